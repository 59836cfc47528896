// Application of the factored block-banded preconditioner, z = P^{-1} r
// (Sec. 4.2 and App. A: the banded linear Jacobian, factored by block LU),
// in FP32 over an FP32 copy of the FP64 factors.
//
// The sweeps are a chain of 2M dependent slice steps: forward
//   y_k = x_k - sum_{i=k-h}^{k-1} L_ki y_i,
// backward
//   z_k = D_k^-1 y_k - sum_{j=k+1}^{k+h} W_kj z_j.
// Of the blocks a step multiplies, only one meets a vector finished by the
// step just before (L_k,k-1 y_k-1 forward, W_k,k+1 z_k+1 backward, D^-1 y at
// the turn); every other term uses vectors finished two or more steps
// earlier.
//
// Dataflow instead of a grid barrier: every entry of y and z is one 64-bit
// word holding the FP32 value and a tag naming the launch and step that wrote
// it, stored and loaded with single-copy-atomic relaxed accesses.  A CTA
// computes the independent terms of its next step, loads the one dependent
// block into registers, and then each thread spins only on the tags of the
// vector entries it multiplies.  The critical path per step is one
// producer-to-consumer trip through L2 plus a short dot product; the other
// blocks stream while the CTA waits, and the blocks of step s+2 are prefetched
// to L2.  Tags grow with every launch (the buffers are zeroed when the
// preconditioner is factored, tags start at 1), so an entry left by an earlier
// launch never matches.
//
// Rows are dealt round-robin to one CTA per SM (row = blockIdx + j G); each
// thread owns CPT columns, so a block's rows of a CTA are RPC x CPT values
// per thread, reduced through warp shuffles and shared memory.  The
// preconditioner only steers GMRES; the Newton residual and the converged
// solution do not depend on its rounding.
//
// The launch is cooperative (all CTAs resident), so every awaited entry is
// eventually written.  Each spin is still bounded (about a second); a thread
// that gives up raises bit 2 of the context flag and the CTA returns at its
// next step boundary.
#include "bfs_internal.cuh"

namespace bfs {

struct FlowArgs {
    const float *pc;               // FP32 factors: block (k, m) row r at ((k nd + m - k + h) nb + r) ldp
    const double *r;               // right-hand side, order of u
    double *z;                     // result, order of u (may equal r)
    unsigned long long *X, *Y;     // tagged slice-ordered vectors, M * nb each
    int nb, NB, M, h;
    int ldp;                       // padded row length of the FP32 factors (multiple of 4)
    int nslot;                     // shared-memory ring depth (TMA kernel)
    unsigned int *tagp;            // device word: tag of this launch's step 0; step s writes
                                   // tag0 + s, and block 0 advances the word by 2M on exit
    int *flag;
};

constexpr int FL_TPB = 512;
constexpr int FL_WARPS = FL_TPB / 32;
constexpr unsigned int FL_SPIN = 1u << 20;  // polls of one entry before giving up (~1 s)

__device__ __forceinline__ unsigned long long ld_word(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_word(unsigned long long *p, float v, unsigned int tag)
{
    const unsigned long long w = ((unsigned long long)tag << 32) | __float_as_uint(v);
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(w) : "memory");
}

__device__ __forceinline__ unsigned int ld_tag(const unsigned int *p)
{
    unsigned int v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Block 0 ends after every CTA has stored its rows of step 2M-2, so every
// CTA has read the launch's tag by then: the next launch may use the next
// 2M tags.
__device__ __forceinline__ void advance_tag(unsigned int *p, unsigned int tag0, int M)
{
    const unsigned int next = tag0 + 2u * (unsigned int)M;
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(next) : "memory");
}

// Value of a tagged entry once its tag is `tag`; false on timeout.
__device__ __forceinline__ bool await_word(const unsigned long long *p, unsigned int tag, float &v)
{
    unsigned long long w = ld_word(p);
    unsigned int spins = 0;
    while ((unsigned int)(w >> 32) != tag) {
        if (++spins > FL_SPIN) return false;
        __nanosleep(32);
        w = ld_word(p);
    }
    v = __uint_as_float((unsigned int)w);
    return true;
}

template <int RPC, int CPT>
__global__ void __launch_bounds__(FL_TPB, 1) k_apply_flow(FlowArgs a)
{
    __shared__ float red[RPC][FL_WARPS];
    __shared__ unsigned int tag_sh;
    const float *pc = a.pc;
    const int nb = a.nb, NB = a.NB, M = a.M, h = a.h, nd = 2 * h + 1, G = gridDim.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if ((int)blockIdx.x >= nb) return;  // no rows here
    if (tid == 0) tag_sh = ld_tag(a.tagp);
    __syncthreads();
    const unsigned int tag0 = tag_sh;

    int row[RPC];
    bool rv[RPC];
#pragma unroll
    for (int j = 0; j < RPC; j++) {
        row[j] = blockIdx.x + j * G;
        rv[j] = row[j] < nb;
        if (!rv[j]) row[j] = 0;
    }
    int col[CPT];
    bool cv[CPT];
#pragma unroll
    for (int q = 0; q < CPT; q++) {
        col[q] = tid + q * FL_TPB;
        cv[q] = col[q] < nb;
        if (!cv[q]) col[q] = 0;
    }
    // the thread that finishes row j (tid == j) and its index in the order of u
    const int my_j = tid < RPC ? tid : -1;
    const bool my_rv = my_j >= 0 && blockIdx.x + my_j * G < nb;
    size_t my_e = 0;
    if (my_rv) {
        const int rw = blockIdx.x + my_j * G, g = rw / NB, p = rw - g * NB;
        my_e = (size_t)g * NB * M + p;  // + l NB for slice l
    }

    auto step_of = [&](int s, int &pass, int &k, int &lo, int &hi, int &crit) {
        pass = s < M ? 0 : 1;
        k = pass == 0 ? s : 2 * M - 1 - s;
        if (pass == 0) {
            lo = max(0, k - h); hi = k - 1;
            crit = (k >= 1 && h >= 1) ? k - 1 : -1;
        } else {
            lo = k; hi = min(M - 1, k + h);
            crit = (k == M - 1) ? k : (h >= 1 ? k + 1 : -1);
        }
    };
    // step that wrote the vector multiplied by block (k, m) in pass `pass`
    auto producer = [&](int pass, int k, int m) { return (pass == 0 || m == k) ? m : 2 * M - 1 - m; };
    auto vec = [&](int pass, int k, int m) -> const unsigned long long * {
        return (pass == 0 || m == k) ? a.Y + (size_t)m * nb : a.X + (size_t)m * nb;
    };
    const int ldp = a.ldp;
    auto block_row = [&](int k, int m, int j) { return pc + (((size_t)k * nd + (m - k + h)) * nb + row[j]) * ldp; };
    auto prefetch = [&](int s) {
        if (s >= 2 * M) return;
        int pass, k, lo, hi, crit;
        step_of(s, pass, k, lo, hi, crit);
        constexpr int per_line = 32;  // floats per 128-byte line
        const int nlines = (nb + per_line - 1) / per_line;
        for (int m = lo; m <= hi; m++)
            for (int idx = tid; idx < RPC * nlines; idx += FL_TPB) {
                const int j = idx / nlines, ln = idx - j * nlines;
                const int rw = blockIdx.x + j * G;
                if (rw < nb) {
                    const float *bp = pc + (((size_t)k * nd + (m - k + h)) * nb + rw) * ldp + ln * per_line;
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(bp));
                }
            }
    };

    prefetch(0);
    prefetch(1);
    bool ok = true;
    for (int s = 0; s < 2 * M; s++) {
        int pass, k, lo, hi, crit;
        step_of(s, pass, k, lo, hi, crit);
        prefetch(s + 2);
        float acc[RPC];
#pragma unroll
        for (int j = 0; j < RPC; j++) acc[j] = 0.f;
        double xk = 0.0;
        if (pass == 0 && my_rv) xk = a.r[my_e + (size_t)k * NB];

        // terms whose vectors were finished two or more steps ago, two blocks
        // in flight at a time (their tags are checked all the same)
        for (int m = lo; m <= hi; m++) {
            if (m == crit) continue;
            int m2 = m + 1;
            if (m2 == crit) m2++;
            const bool two = m2 <= hi;
            float f[2][RPC][CPT], v[2][CPT];
#pragma unroll
            for (int bb = 0; bb < 2; bb++) {
                const int mm = (bb == 0 || !two) ? m : m2;
                const bool use = bb == 0 || two;
                const unsigned long long *vp = vec(pass, k, mm);
                const unsigned int tg = tag0 + producer(pass, k, mm);
#pragma unroll
                for (int q = 0; q < CPT; q++) {
                    v[bb][q] = 0.f;
                    if (ok && use && cv[q]) ok = await_word(vp + col[q], tg, v[bb][q]);
                }
#pragma unroll
                for (int j = 0; j < RPC; j++) {
                    const float *bp = block_row(k, mm, j);
#pragma unroll
                    for (int q = 0; q < CPT; q++) f[bb][j][q] = (use && rv[j] && cv[q]) ? __ldg(bp + col[q]) : 0.f;
                }
            }
#pragma unroll
            for (int bb = 0; bb < 2; bb++) {
                const int mm = (bb == 0 || !two) ? m : m2;
                const float sg = (pass == 1 && mm == k) ? 1.f : -1.f;
#pragma unroll
                for (int j = 0; j < RPC; j++) {
                    float t = 0.f;
#pragma unroll
                    for (int q = 0; q < CPT; q++) t = fmaf(f[bb][j][q], v[bb][q], t);
                    acc[j] = fmaf(sg, t, acc[j]);
                }
            }
            if (two) m = m2;
        }

        // the dependent block: registers first, then wait for its vector
        if (crit >= 0) {
            float cf[RPC][CPT];
#pragma unroll
            for (int j = 0; j < RPC; j++) {
                const float *bp = block_row(k, crit, j);
#pragma unroll
                for (int q = 0; q < CPT; q++) cf[j][q] = (rv[j] && cv[q]) ? __ldg(bp + col[q]) : 0.f;
            }
            const float sg = (pass == 1 && crit == k) ? 1.f : -1.f;
            const unsigned long long *vp = vec(pass, k, crit);
            const unsigned int tg = tag0 + (unsigned int)(s - 1);
            float v[CPT];
#pragma unroll
            for (int q = 0; q < CPT; q++) {
                v[q] = 0.f;
                if (ok && cv[q]) ok = await_word(vp + col[q], tg, v[q]);
            }
#pragma unroll
            for (int j = 0; j < RPC; j++) {
                float t = 0.f;
#pragma unroll
                for (int q = 0; q < CPT; q++) t = fmaf(cf[j][q], v[q], t);
                acc[j] = fmaf(sg, t, acc[j]);
            }
        }
#pragma unroll
        for (int j = 0; j < RPC; j++) {
            float t = acc[j];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            if (lane == 0) red[j][warp] = t;
        }
        if (!__syncthreads_and(ok)) {
            if (tid == 0) {
                atomicOr(a.flag, 2);
                if (blockIdx.x == 0) advance_tag(a.tagp, tag0, M);
            }
            return;
        }
        if (my_rv) {
            float t = 0.f;
#pragma unroll
            for (int w = 0; w < FL_WARPS; w++) t += red[my_j][w];
            const size_t si = (size_t)k * nb + blockIdx.x + my_j * G;
            const unsigned int tg = tag0 + (unsigned int)s;
            if (pass == 0) {
                st_word(a.Y + si, (float)(xk + (double)t), tg);
            } else {
                st_word(a.X + si, t, tg);
                a.z[my_e + (size_t)k * NB] = (double)t;
            }
        }
        __syncthreads();  // red is rewritten by the next step
    }
    if (blockIdx.x == 0 && tid == 0) advance_tag(a.tagp, tag0, M);
}

// TMA variant for slice blocks that fit its tiles (rows per CTA <= RPC,
// nb <= CT CPT, at most BMAX blocks per step).  Each CTA owns a contiguous
// run of rows, so its rows of one block are one contiguous span of the padded
// FP32 factors.  A producer warp streams the spans of every block of a step
// into a ring of `nslot` shared-memory slots with 1-D bulk copies
// (cp.async.bulk, completion counted in bytes on a "full" mbarrier per slot),
// up to nslot - 1 steps ahead; the compute warps release a slot on its
// "empty" mbarrier once they have read it.  No compute thread spends issue
// slots or load-queue entries on the factors: the vector words of a step's
// independent terms are loaded when the previous step has stored, and only
// the awaited entries of the dependent term remain on the critical path.
__device__ __forceinline__ unsigned int smem_u32(const void *p)
{
    return (unsigned int)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ bool mbar_wait(unsigned int bar, unsigned int parity)
{
    for (unsigned int i = 0; i < FL_SPIN; i++) {
        unsigned int done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// barrier 1 over the CT compute threads, AND of their predicates
__device__ __forceinline__ bool compute_sync_and(bool pred, int ct)
{
    unsigned int r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.and.pred q, 1, %2, p;\n selp.u32 %0, 1, 0, q;\n}"
        : "=r"(r)
        : "r"((unsigned int)pred), "r"(ct)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ void compute_sync(int ct)
{
    asm volatile("bar.sync 1, %0;" ::"r"(ct) : "memory");
}

template <int CT, int RPC, int CPT, int BMAX>
__global__ void __launch_bounds__(CT + 32, 1) k_apply_tma(FlowArgs a)
{
    // Block positions of a step (slot layout): forward step k multiplies
    // L_k,k-p at position p = 1..h (p = 1 is the dependent one); backward
    // step k multiplies D_k^-1 at p = 0 and W_k,k+p at p = 1..h (p = 1
    // dependent; at k = M-1 the D^-1 term is the dependent one).
    constexpr int WARPS = CT / 32;
    constexpr int MAXSLOT = 8;
    constexpr int HW = BMAX - 2 > 0 ? BMAX - 2 : 1;  // vectors kept from earlier steps
    extern __shared__ __align__(128) float ring[];  // nslot x BMAX x RPC x ldp
    __shared__ __align__(8) unsigned long long full[MAXSLOT], empty[MAXSLOT];
    __shared__ float red[2][RPC][WARPS];
    __shared__ unsigned int tag_sh;
    const float *pc = a.pc;
    const int nb = a.nb, NB = a.NB, M = a.M, h = a.h, nd = 2 * h + 1, ldp = a.ldp;
    const int nslot = a.nslot, G = gridDim.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const size_t slot_floats = (size_t)BMAX * RPC * ldp;
    // rows [r0, r0 + nrv): the first nb % G CTAs take one row more
    const int base = nb / G, extra = nb % G;
    const int nrv = base + (blockIdx.x < extra ? 1 : 0);
    const int r0 = blockIdx.x * base + min((int)blockIdx.x, extra);
    // block column m at position p of step s (-1: no block there)
    auto pos_m = [&](int s, int p) {
        if (s < M) {
            const int k = s, m = k - p;
            return (p >= 1 && p <= h && m >= 0) ? m : -1;
        }
        const int k = 2 * M - 1 - s, m = k + p;
        return (p <= h && m <= M - 1) ? m : -1;
    };

    if (nrv == 0) return;  // no rows here
    if (tid == 0) {
        tag_sh = ld_tag(a.tagp);
        for (int i = 0; i < nslot; i++) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full[i])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[i])) : "memory");
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const unsigned int tag0 = tag_sh;

    if (warp == WARPS) {
        // producer warp: lane L copies row L % RPC of position L / RPC
        const int p = lane / RPC, j = lane % RPC;
        int q = 0;
        bool fine = true;
        for (; q < 2 * M; q++) {
            const int slot = q % nslot;
            if (q >= nslot) {
                int w = 1;
                if (lane == 0) w = mbar_wait(smem_u32(&empty[slot]), (unsigned int)((q / nslot - 1) & 1)) ? 1 : 0;
                w = __shfl_sync(0xffffffffu, w, 0);
                if (!w) {
                    if (lane == 0) atomicOr(a.flag, 2);
                    fine = false;
                    break;
                }
            }
            const int k = q < M ? q : 2 * M - 1 - q;
            int npos = 0;
            for (int pp = 0; pp < BMAX; pp++) npos += pos_m(q, pp) >= 0 ? 1 : 0;
            const unsigned int fb = smem_u32(&full[slot]);
            const unsigned int row_bytes = (unsigned int)(ldp * 4);
            if (lane == 0) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb),
                             "r"(row_bytes * (unsigned int)(npos * nrv))
                             : "memory");
            }
            __syncwarp();
            const int m = p < BMAX ? pos_m(q, p) : -1;
            if (m >= 0 && j < nrv) {
                const float *src = pc + (((size_t)k * nd + (m - k + h)) * nb + r0 + j) * ldp;
                float *dst = ring + (size_t)slot * slot_floats + ((size_t)p * RPC + j) * ldp;
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                        smem_u32(dst)),
                    "l"(src), "r"(row_bytes), "r"(fb)
                    : "memory");
            }
        }
        // every copy issued must land before the CTA may end
        if (lane == 0) {
            const int last = fine ? 2 * M - 1 : q - 1;
            for (int pq = max(0, last - nslot + 1); pq <= last; pq++)
                if (!mbar_wait(smem_u32(&full[pq % nslot]), (unsigned int)((pq / nslot) & 1))) break;
        }
        return;
    }

    // compute warps
    int col[CPT];
    bool cv[CPT];
#pragma unroll
    for (int q = 0; q < CPT; q++) {
        col[q] = tid + q * CT;
        cv[q] = col[q] < nb;
        if (!cv[q]) col[q] = 0;
    }
    const int my_j = tid < nrv ? tid : -1;
    size_t my_e = 0;
    if (my_j >= 0) {
        const int rw = r0 + my_j, g = rw / NB, pp = rw - g * NB;
        my_e = (size_t)g * NB * M + pp;
    }
    float win[HW][CPT];  // forward: y_{k-2-i}; backward: z_{k+2+i} (this thread's columns)
    unsigned long long yw[CPT];  // backward: the word of y_k, loaded one step early
#pragma unroll
    for (int q = 0; q < CPT; q++) {
        yw[q] = 0ull;
#pragma unroll
        for (int i = 0; i < HW; i++) win[i][q] = 0.f;
    }
    auto dot = [&](const float *S, int p, const float (&v)[CPT], float (&acc)[RPC], float sg) {
#pragma unroll
        for (int j = 0; j < RPC; j++) {
            float u = 0.f;
#pragma unroll
            for (int q = 0; q < CPT; q++)
                if (cv[q] && j < nrv) u = fmaf(S[((size_t)p * RPC + j) * ldp + col[q]], v[q], u);
            acc[j] = fmaf(sg, u, acc[j]);
        }
    };

    bool ok = true;
    for (int s = 0; s < 2 * M; s++) {
        const int pass = s < M ? 0 : 1;
        const int k = pass == 0 ? s : 2 * M - 1 - s;
        double xk = 0.0;
        if (pass == 0 && my_j >= 0) xk = a.r[my_e + (size_t)k * NB];
        const int slot = s % nslot;
        const float *S = ring + (size_t)slot * slot_floats;
        ok = mbar_wait(smem_u32(&full[slot]), (unsigned int)((s / nslot) & 1));
        float acc[RPC];
#pragma unroll
        for (int j = 0; j < RPC; j++) acc[j] = 0.f;
        // terms whose vectors this thread already holds
#pragma unroll
        for (int p = 2; p < BMAX; p++)
            if (ok && pos_m(s, p) >= 0) dot(S, p, win[p - 2], acc, -1.f);
        if (ok && pass == 1 && k < M - 1) {
            float v[CPT];
#pragma unroll
            for (int q = 0; q < CPT; q++) {
                v[q] = 0.f;
                if (cv[q]) {
                    if ((unsigned int)(yw[q] >> 32) == tag0 + (unsigned int)k) v[q] = __uint_as_float((unsigned int)yw[q]);
                    else if (ok) ok = await_word(a.Y + (size_t)k * nb + col[q], tag0 + (unsigned int)k, v[q]);
                }
            }
            dot(S, 0, v, acc, 1.f);
        }
        // the dependent term: the vector finished by step s-1
        const bool turn = pass == 1 && k == M - 1;
        if (ok && (turn || pos_m(s, 1) >= 0)) {
            const unsigned long long *vp = turn ? a.Y + (size_t)k * nb
                                                : (pass == 0 ? a.Y + (size_t)(k - 1) * nb : a.X + (size_t)(k + 1) * nb);
            const unsigned int tg = tag0 + (unsigned int)(s - 1);
            float v[CPT];
#pragma unroll
            for (int q = 0; q < CPT; q++) {
                v[q] = 0.f;
                if (ok && cv[q]) ok = await_word(vp + col[q], tg, v[q]);
            }
            if (turn) {
                dot(S, 0, v, acc, 1.f);
            } else {
                dot(S, 1, v, acc, -1.f);
#pragma unroll
                for (int q = 0; q < CPT; q++) {
#pragma unroll
                    for (int i = HW - 1; i > 0; i--) win[i][q] = win[i - 1][q];
                    win[0][q] = v[q];
                }
            }
        }
        if (turn) {  // the backward window starts empty
#pragma unroll
            for (int q = 0; q < CPT; q++)
#pragma unroll
                for (int i = 0; i < HW; i++) win[i][q] = 0.f;
        }
        float(&rd)[RPC][WARPS] = red[s & 1];
#pragma unroll
        for (int j = 0; j < RPC; j++) {
            float u = acc[j];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) u += __shfl_xor_sync(0xffffffffu, u, o);
            if (lane == 0) rd[j][warp] = u;
        }
        if (!compute_sync_and(ok, CT)) {
            if (tid == 0) {
                atomicOr(a.flag, 2);
                if (blockIdx.x == 0) advance_tag(a.tagp, tag0, M);
            }
            return;  // the producer drains its copies and returns
        }
        if (tid == 0)  // every compute warp has read slot `slot`
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&empty[slot])) : "memory");
        if (my_j >= 0) {
            float u = 0.f;
#pragma unroll
            for (int w = 0; w < WARPS; w++) u += rd[my_j][w];
            const size_t si = (size_t)k * nb + r0 + my_j;
            const unsigned int tg = tag0 + (unsigned int)s;
            if (pass == 0) {
                st_word(a.Y + si, (float)(xk + (double)u), tg);
            } else {
                st_word(a.X + si, u, tg);
                a.z[my_e + (size_t)k * NB] = (double)u;
            }
        }
        // y_k of the next backward step (finished long before)
        if (s + 1 > M && s + 1 < 2 * M) {
            const int kn = 2 * M - 2 - s;
#pragma unroll
            for (int q = 0; q < CPT; q++) yw[q] = cv[q] ? ld_word(a.Y + (size_t)kn * nb + col[q]) : 0ull;
        }
        // red[s & 1] is next written at step s + 2, after every thread has
        // passed the barrier of step s + 1
    }
    if (blockIdx.x == 0 && tid == 0) advance_tag(a.tagp, tag0, M);
}

constexpr int TMA_CT = 288, TMA_RPC = 4, TMA_CPT = 2, TMA_BMAX = 4, TMA_MAXSLOT = 8;
constexpr size_t TMA_SMEM_MAX = 200 * 1024;


using FlowKernel = void (*)(FlowArgs);

static FlowKernel pick_flow(int rpc, int cpt)
{
    if (rpc <= 4 && cpt <= 2) return k_apply_flow<4, 2>;
    if (rpc <= 8 && cpt <= 2) return k_apply_flow<8, 2>;
    if (rpc <= 8 && cpt <= 3) return k_apply_flow<8, 3>;
    return nullptr;
}

// FP32 copy of the factors with rows padded from nb to ldp entries (zeros),
// so that every row starts on a 16-byte boundary.
__global__ void k_cast_f32(const double *__restrict__ in, float *__restrict__ out, size_t rows, int nb, int ldp)
{
    const size_t n = rows * (size_t)ldp;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const size_t r = i / ldp;
        const int c = (int)(i - r * ldp);
        out[i] = c < nb ? (float)in[r * nb + c] : 0.f;
    }
}

__global__ void k_set_tag(unsigned int *p, unsigned int v) { *p = v; }

// Zero the tagged vectors and restart the tags at 1 (so no stale entry can
// carry a tag a later launch waits for).
static int flow_reset(bfs_ctx *c, cudaStream_t s)
{
    const size_t nv = (size_t)c->M * c->nb;
    BFS_CUDA_TRY(c, cudaMemsetAsync(c->d_flow, 0, sizeof(unsigned long long) * (2 * nv + 1), s));
    k_set_tag<<<1, 1, 0, s>>>(reinterpret_cast<unsigned int *>(c->d_flow + 2 * nv), 1u);
    c->launches++;
    c->flow_count = 0;
    BFS_CUDA_TRY(c, cudaGetLastError());
    return BFS_OK;
}

// Before each FP32 sweep launch (direct or inside a graph): restart the tags
// well before they could wrap.
int flow_wrap_check(bfs_ctx *c, cudaStream_t s)
{
    const unsigned long long steps = 2ull * (unsigned long long)c->M;
    if ((c->flow_count + 2) * steps >= 0xFFFFFFFFull - 0xFFFFull) return flow_reset(c, s);
    return BFS_OK;
}

int precond_make_f32(bfs_ctx *c, cudaStream_t s)
{
    const int ldp = (c->nb + 3) / 4 * 4;
    const size_t rows = (size_t)c->nb * c->M * (2 * c->pc_h + 1);
    const size_t cnt = rows * ldp;
    const size_t nv = (size_t)c->M * c->nb;
    c->ldp32 = ldp;
    cudaFree(c->d_pc32);
    cudaFree(c->d_flow);
    c->d_pc32 = nullptr;
    c->d_flow = nullptr;
    if (cudaMalloc(&c->d_pc32, sizeof(float) * cnt) != cudaSuccess ||
        cudaMalloc(&c->d_flow, sizeof(unsigned long long) * (2 * nv + 1)) != cudaSuccess) {
        cudaGetLastError();
        c->err = "FP32 preconditioner copy: out of device memory";
        return BFS_ENOMEM;
    }
    int rc = flow_reset(c, s);
    if (rc) return rc;
    k_cast_f32<<<4 * num_sms(c->device), 256, 0, s>>>(c->d_pc, c->d_pc32, rows, c->nb, ldp);
    c->launches++;
    BFS_CUDA_TRY(c, cudaGetLastError());
    return BFS_OK;
}

// Returns 1 if launched, 0 if this apply is not for the FP32 sweep kernels
// (FP64 sweeps, or slice blocks wider than their tiles), or a negative code.
int apply_flow_launch(bfs_ctx *c, const double *r, double *z, cudaStream_t s)
{
    if (c->opt.precond_precision != BFS_FP32C || !c->d_pc32 || !c->d_flow) return 0;
    const int G = num_sms(c->device);
    const int rpc = (c->nb + G - 1) / G, cpt = (c->nb + FL_TPB - 1) / FL_TPB;
    const size_t slot_bytes = (size_t)TMA_BMAX * TMA_RPC * c->ldp32 * sizeof(float);
    int nslot = (int)std::min<size_t>(TMA_MAXSLOT, TMA_SMEM_MAX / slot_bytes);
    nslot = std::min(nslot, 6);
    const bool tma = rpc <= TMA_RPC && c->nb <= TMA_CT * TMA_CPT && c->pc_h < TMA_BMAX && nslot >= 2;
    FlowKernel kern = tma ? k_apply_tma<TMA_CT, TMA_RPC, TMA_CPT, TMA_BMAX> : pick_flow(rpc, cpt);
    const int tpb = tma ? TMA_CT + 32 : FL_TPB;
    const size_t dyn = tma ? slot_bytes * nslot : 0;
    if (!kern) return 0;
    if (!c->flow_checked) {
        if (tma)  // one ceiling for every context, whatever its ring depth
            BFS_CUDA_TRY(c, cudaFuncSetAttribute((const void *)kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)TMA_SMEM_MAX));
        int per_sm = 0;
        BFS_CUDA_TRY(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, tpb, dyn));
        if (per_sm < 1) return 0;
        c->flow_checked = 1;
    }
    if (!c->capturing) {
        int rc = flow_wrap_check(c, s);
        if (rc) return rc;
    }
    FlowArgs a;
    a.pc = c->d_pc32;
    a.r = r; a.z = z;
    a.Y = c->d_flow;
    a.X = c->d_flow + (size_t)c->M * c->nb;
    a.nb = c->nb; a.NB = c->N + 1; a.M = c->M; a.h = c->pc_h;
    a.ldp = c->ldp32;
    a.nslot = nslot;
    a.tagp = reinterpret_cast<unsigned int *>(c->d_flow + 2 * (size_t)c->M * c->nb);
    a.flag = c->d_flag;
    void *args[] = {&a};
    BFS_CUDA_TRY(c, cudaLaunchCooperativeKernel((const void *)kern, dim3(G), dim3(tpb), args, dyn, s));
    c->launches++;
    c->flow_count++;
    return 1;
}

}  // namespace bfs
