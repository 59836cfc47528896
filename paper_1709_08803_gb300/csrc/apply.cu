// Application of the factored block-banded preconditioner, z = P^{-1} r
// (Sec. 4.2 and App. A: the banded linear Jacobian, factored by block LU),
// in FP32 over an FP32 copy of the FP64 factors.
//
// The sweeps are chains of dependent slice steps.  With the one-ended LU
// (factored from slice 0 down) they are forward
//   y_k = x_k - sum_{i=k-h}^{k-1} L_ki y_i,
// then backward
//   z_k = D_k^-1 y_k - sum_{j=k+1}^{k+h} W_kj z_j,
// 2M steps in one chain.  The two-ended ("twisted") LU eliminates slices
// 0..t-1 downwards and M-1..t+h upwards; the two chains touch only the h
// middle slices, whose Schur complement C is inverted whole.  Its sweeps run
// as two chains side by side: forward from the top and upward from the bottom
// (y_k = x_k - sum U'_kj y_j, j = k+1..k+h), the middle y (both chains' terms),
// z_mid = C^-1 y_mid, and the back substitutions outwards -- about M dependent
// steps instead of 2M.
//
// Every step, in either form, is one task of a host-built table: the slice it
// finishes, whether it writes y (and adds the right-hand side) or z, and the
// stored blocks it multiplies, each with the vector slice it multiplies and the
// task that wrote that slice.  CTAs are split into as many groups as there are
// chains; a group runs its tasks in order, each CTA owning a contiguous run of
// rows of every slice.
//
// Dataflow instead of a grid barrier: every entry of y and z is one 64-bit
// word holding the FP32 value and a tag naming the launch and task that wrote
// it, stored and loaded with single-copy-atomic relaxed accesses.  A CTA loads
// the vector words of all its blocks at the start of a step, multiplies the
// ones that are ready, and then each thread spins only on the tags of the
// entries still missing -- in practice those the group's previous task wrote.
// The critical path per step is one producer-to-consumer trip through L2 plus
// a short dot product.  Tags grow with every launch (the buffers are zeroed
// when the preconditioner is factored or a wait has timed out, tags start at
// 1), so an entry left by an earlier launch never matches.
//
// The launches are cooperative (all CTAs resident), so every awaited entry is
// eventually written.  Each spin is still bounded (about a second by default,
// the option wait_polls otherwise); a thread that gives up raises bit 2 of the
// context flag and the CTA returns at its next step boundary.  A launch that
// finds bit 2 already raised does nothing: the host clears it, and resets the
// tagged vectors, when it reads the flag.
#include <string.h>

#include <algorithm>
#include <vector>

#include "bfs_internal.cuh"

namespace bfs {

struct FlowArgs {
    const float *pc;               // FP32 factors: block (k, m) row r at ((k nd + m - k + h) nb + r) ldp
    const double *r;               // right-hand side, order of u
    double *z;                     // result, order of u (may equal r)
    unsigned long long *X, *Y;     // tagged slice-ordered vectors, M * nb each
    int nb, NB, M, h;
    int ldp;                       // padded row length of the FP32 factors (multiple of 4)
    int nslot;                     // shared-memory ring depth (task-table kernel)
    unsigned int *tagp;            // device word: tag of this launch's first step; step (task) s
                                   // writes tag0 + s, and block 0 advances the word by ntags on exit
    int *flag;
    unsigned int spin;             // polls of one wait before giving up
    const SweepTask *tasks;        // task table: group 0's tasks, then group 1's
    int ntask0, ntask1;            // tasks per group
    int G0;                        // CTAs of group 0 (the rest form group 1)
    int ntags;                     // tags one launch uses (= ntask0 + ntask1)
};

constexpr int FL_TPB = 512;
constexpr int FL_WARPS = FL_TPB / 32;
constexpr unsigned int FL_SPIN = 1u << 20;  // default polls of one entry before giving up (~1 s)

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

// The launch's last CTA to depend on every other one advances the tag word,
// so every CTA has read this launch's tag by then and the next launch may use
// the next tags.
__device__ __forceinline__ void advance_tag(unsigned int *p, unsigned int tag0, unsigned int ntags)
{
    const unsigned int next = tag0 + ntags;
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(next) : "memory");
}

// Value of a tagged entry once its tag is `tag`; false after `spin` polls.
__device__ __forceinline__ bool await_word(const unsigned long long *p, unsigned int tag, float &v,
                                           unsigned int spin)
{
    unsigned long long w = ld_word(p);
    unsigned int spins = 0;
    while ((unsigned int)(w >> 32) != tag) {
        if (++spins > spin) return false;
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
    __shared__ int abort_sh;
    if ((int)blockIdx.x >= nb) return;  // no rows here
    if (tid == 0) {
        abort_sh = (ld_tag(reinterpret_cast<const unsigned int *>(a.flag)) & 2u) != 0;
        tag_sh = ld_tag(a.tagp);
    }
    __syncthreads();
    if (abort_sh) return;  // an earlier wait timed out: the host resets the vectors first
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
                    if (ok && use && cv[q]) ok = await_word(vp + col[q], tg, v[bb][q], a.spin);
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
                if (ok && cv[q]) ok = await_word(vp + col[q], tg, v[q], a.spin);
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
                if (blockIdx.x == 0) advance_tag(a.tagp, tag0, 2u * (unsigned int)M);
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
    if (blockIdx.x == 0 && tid == 0) advance_tag(a.tagp, tag0, 2u * (unsigned int)M);
}

// ---------------------------------------------------------------------------
// Task-table kernel for slice blocks that fit its tiles (rows of a slice per
// CTA <= RPC, nb <= CT CPT, at most SW_BMAX blocks per task).  Each CTA owns a
// contiguous run of rows, so its rows of one block are one contiguous span of
// the padded FP32 factors.  A producer warp streams the spans of every block
// of a task into a ring of `nslot` shared-memory slots with 1-D bulk copies
// (cp.async.bulk, completion counted in bytes on a "full" mbarrier per slot),
// up to nslot - 1 tasks ahead; the compute warps release a slot on its "empty"
// mbarrier once they have read it.  No compute thread spends issue slots or
// load-queue entries on the factors.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned int smem_u32(const void *p)
{
    return (unsigned int)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ bool mbar_wait(unsigned int bar, unsigned int parity, unsigned int spin)
{
    for (unsigned int i = 0; i < spin; i++) {
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

// Sums v[j] (j < R, R a power of two <= 32) over the 32 lanes of a warp by a
// reduce-scatter: each halving step trades half of the rows with the partner
// lane, so R rows cost log2(R) + (R - 1) shuffles instead of 5 R.  Lane l ends
// with the warp total of row `row`; the 32 / R lanes that share a row hold the
// same total.
template <int R>
__device__ __forceinline__ float warp_rows_sum(const float (&acc)[R], int lane, int &row)
{
    float v[R];
#pragma unroll
    for (int i = 0; i < R; i++) v[i] = acc[i];
    int r = 0, off = 16;
#pragma unroll
    for (int n = R; n > 1; n >>= 1) {
        const bool up = (lane & off) != 0;
        const int hlf = n >> 1;
#pragma unroll
        for (int i = 0; i < hlf; i++) {
            const float send = up ? v[i] : v[i + hlf];
            const float keep = up ? v[i + hlf] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
        }
        if (up) r += hlf;
        off >>= 1;
    }
    for (; off >= 1; off >>= 1) v[0] += __shfl_xor_sync(0xffffffffu, v[0], off);
    row = r;
    return v[0];
}

template <int CT, int RPC, int CPT>
__global__ void __launch_bounds__(CT + 32, 1) k_apply_sweep(FlowArgs a)
{
    constexpr int WARPS = CT / 32;
    constexpr int BM = SW_BMAX;
    constexpr int MAXSLOT = 8;
    static_assert(32 % RPC == 0 && RPC * BM >= 1, "rows per CTA must divide the warp");
    extern __shared__ __align__(128) float ring[];  // nslot x BM x RPC x ldp, then the group's tasks
    __shared__ __align__(8) unsigned long long full[MAXSLOT], empty[MAXSLOT];
    __shared__ float red[2][RPC][WARPS];
    __shared__ unsigned int tag_sh;
    __shared__ int abort_sh;
    const float *pc = a.pc;
    const int nb = a.nb, NB = a.NB, h = a.h, nd = 2 * h + 1, ldp = a.ldp;
    const int nslot = a.nslot;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const size_t slot_floats = (size_t)BM * RPC * ldp;
    // CTA group and its tasks
    const int grp = (int)blockIdx.x < a.G0 ? 0 : 1;
    const int Gg = grp ? (int)gridDim.x - a.G0 : a.G0;
    const int lb = grp ? (int)blockIdx.x - a.G0 : (int)blockIdx.x;
    const SweepTask *gtasks = a.tasks + (grp ? a.ntask0 : 0);
    const int ntask = grp ? a.ntask1 : a.ntask0;
    // the task table, staged once: a descriptor read from global memory at
    // every step would put an L2 round trip in front of each step's waits
    SweepTask *tasks = reinterpret_cast<SweepTask *>(ring + (size_t)nslot * slot_floats);
    // rows [r0, r0 + nrv) of every slice: the first nb % Gg CTAs take one row more
    const int base = nb / Gg, extra = nb % Gg;
    const int nrv = base + (lb < extra ? 1 : 0);
    const int r0 = lb * base + min(lb, extra);

    if (nrv == 0 || ntask == 0) return;  // no rows here
    if (tid == 0) {
        abort_sh = (ld_tag(reinterpret_cast<const unsigned int *>(a.flag)) & 2u) != 0;
        tag_sh = ld_tag(a.tagp);
        for (int i = 0; i < nslot; i++) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full[i])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[i])) : "memory");
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    {
        const int *src = reinterpret_cast<const int *>(gtasks);
        int *dst = reinterpret_cast<int *>(tasks);
        const int words = ntask * (int)(sizeof(SweepTask) / sizeof(int));
        for (int i = tid; i < words; i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    if (abort_sh) return;  // an earlier wait timed out: the host resets the vectors first
    const unsigned int tag0 = tag_sh;

    if (warp == WARPS) {
        // producer warp: the rows [r0, r0 + nrv) of every block of task q into slot q % nslot
        int q = 0;
        bool fine = true;
        const unsigned int row_bytes = (unsigned int)(ldp * 4);
        for (; q < ntask; q++) {
            const int slot = q % nslot;
            if (q >= nslot) {
                int w = 1;
                if (lane == 0)
                    w = mbar_wait(smem_u32(&empty[slot]), (unsigned int)((q / nslot - 1) & 1), a.spin) ? 1 : 0;
                w = __shfl_sync(0xffffffffu, w, 0);
                if (!w) {
                    if (lane == 0) atomicOr(a.flag, 2);
                    fine = false;
                    break;
                }
            }
            const int k = tasks[q].k, nblk = tasks[q].nblk;
            const unsigned int fb = smem_u32(&full[slot]);
            if (lane == 0) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb),
                             "r"(row_bytes * (unsigned int)(nblk * nrv))
                             : "memory");
            }
            __syncwarp();
            for (int idx = lane; idx < nblk * RPC; idx += 32) {
                const int p = idx / RPC, j = idx - p * RPC;
                if (j >= nrv) continue;
                const int m = tasks[q].m[p];
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
            const int last = fine ? ntask - 1 : q - 1;
            for (int pq = max(0, last - nslot + 1); pq <= last; pq++)
                if (!mbar_wait(smem_u32(&full[pq % nslot]), (unsigned int)((pq / nslot) & 1), a.spin)) break;
        }
        return;
    }

    // compute warps: thread tid owns the columns tid + q CT of every block
    int col[CPT];
    bool cv[CPT];
#pragma unroll
    for (int q = 0; q < CPT; q++) {
        col[q] = tid + q * CT;
        cv[q] = col[q] < nb;
        if (!cv[q]) col[q] = 0;
    }
    const int my_j = tid < nrv ? tid : -1;  // the row this thread finishes
    size_t my_e = 0;                        // its index in the order of u (+ k NB for slice k)
    if (my_j >= 0) {
        const int rw = r0 + my_j, g = rw / NB, pp = rw - g * NB;
        my_e = (size_t)g * NB * a.M + pp;
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
    auto vec_ptr = [&](int vec, int m) { return ((vec & 1) ? a.X : a.Y) + (size_t)m * nb; };
    // words of a task's prefetched blocks (SW_EARLY), loaded at the end of the step before
    unsigned long long pre[BM][CPT];
    auto prefetch = [&](int s) {
#pragma unroll
        for (int p = 0; p < BM; p++) {
            const bool use = s < ntask && p < tasks[s].nblk && ((tasks[s].vec[p] >> 2) & 3) == SW_EARLY;
            const unsigned long long *vp = use ? vec_ptr(tasks[s].vec[p], tasks[s].m[p]) : a.Y;
#pragma unroll
            for (int q = 0; q < CPT; q++) pre[p][q] = (use && cv[q]) ? ld_word(vp + col[q]) : 0ull;
        }
    };
    // this thread's columns of the last SW_HW vectors that were a task's critical one
    float win[SW_HW][CPT];
#pragma unroll
    for (int i = 0; i < SW_HW; i++)
#pragma unroll
        for (int q = 0; q < CPT; q++) win[i][q] = 0.f;

    bool ok = true;
    prefetch(0);
    for (int s = 0; s < ntask; s++) {
        const int k = tasks[s].k, nblk = tasks[s].nblk, out = tasks[s].out;
        // the critical vector: its first poll goes out before anything else
        int cp = -1;
#pragma unroll
        for (int p = 0; p < BM; p++)
            if (p < nblk && ((tasks[s].vec[p] >> 2) & 3) == SW_CRIT) cp = p;
        const int cvec = cp >= 0 ? tasks[s].vec[cp] : 0;
        const unsigned long long *cptr = vec_ptr(cvec, cp >= 0 ? tasks[s].m[cp] : 0);
        const unsigned int ctag = tag0 + (unsigned int)(cp >= 0 ? tasks[s].uid[cp] : 0);
        unsigned long long wc[CPT];
#pragma unroll
        for (int q = 0; q < CPT; q++) wc[q] = (cp >= 0 && cv[q]) ? ld_word(cptr + col[q]) : 0ull;
        double xk = 0.0;
        if (out == 0 && my_j >= 0) xk = a.r[my_e + (size_t)k * NB];
        const int slot = s % nslot;
        const float *S = ring + (size_t)slot * slot_floats;
        ok = ok && mbar_wait(smem_u32(&full[slot]), (unsigned int)((s / nslot) & 1), a.spin);
        float acc[RPC];
#pragma unroll
        for (int j = 0; j < RPC; j++) acc[j] = 0.f;
        // terms whose vectors this thread holds or has prefetched
#pragma unroll
        for (int p = 0; p < BM; p++) {
            if (p < nblk && ok) {
                const int vec = tasks[s].vec[p], src = (vec >> 2) & 3;
                const float sg = (vec & 2) ? 1.f : -1.f;
                float v[CPT];
                if (src == SW_WIN) {
                    const int wi = (vec >> 4) & 3;
#pragma unroll
                    for (int q = 0; q < CPT; q++) {
                        v[q] = win[0][q];
#pragma unroll
                        for (int i = 1; i < SW_HW; i++)
                            if (wi == i) v[q] = win[i][q];
                    }
                    dot(S, p, v, acc, sg);
                } else if (src == SW_EARLY) {
                    const unsigned int tg = tag0 + (unsigned int)tasks[s].uid[p];
                    const unsigned long long *vp = vec_ptr(vec, tasks[s].m[p]);
#pragma unroll
                    for (int q = 0; q < CPT; q++) {
                        v[q] = 0.f;
                        if (!cv[q]) continue;
                        if ((unsigned int)(pre[p][q] >> 32) == tg) v[q] = __uint_as_float((unsigned int)pre[p][q]);
                        else if (ok) ok = await_word(vp + col[q], tg, v[q], a.spin);
                    }
                    dot(S, p, v, acc, sg);
                }
            }
        }
        // the critical term last: the vector the group's previous task wrote
        if (cp >= 0 && ok) {
            float v[CPT];
#pragma unroll
            for (int q = 0; q < CPT; q++) {
                v[q] = 0.f;
                if (!cv[q]) continue;
                if ((unsigned int)(wc[q] >> 32) == ctag) v[q] = __uint_as_float((unsigned int)wc[q]);
                else if (ok) ok = await_word(cptr + col[q], ctag, v[q], a.spin);
            }
#pragma unroll
            for (int p = 0; p < BM; p++)
                if (p == cp) dot(S, p, v, acc, (cvec & 2) ? 1.f : -1.f);
#pragma unroll
            for (int q = 0; q < CPT; q++) {
#pragma unroll
                for (int i = SW_HW - 1; i > 0; i--) win[i][q] = win[i - 1][q];
                win[0][q] = v[q];
            }
        }
        float(&rd)[RPC][WARPS] = red[s & 1];
        {
            int row;
            const float t = warp_rows_sum<RPC>(acc, lane, row);
            if ((lane & (32 / RPC - 1)) == 0) rd[row][warp] = t;
        }
        if (!compute_sync_and(ok, CT)) {
            if (tid == 0) atomicOr(a.flag, 2);
            return;  // the producer drains its copies and returns
        }
        if (tid == 0)  // every compute warp has read slot `slot`
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&empty[slot])) : "memory");
        if (my_j >= 0) {
            float u = 0.f;
#pragma unroll
            for (int q = 0; q < WARPS; q++) u += rd[my_j][q];
            const size_t si = (size_t)k * nb + r0 + my_j;
            const unsigned int tg = tag0 + (unsigned int)((grp ? a.ntask0 : 0) + s);
            if (out == 0) {
                st_word(a.Y + si, (float)(xk + (double)u), tg);
            } else {
                st_word(a.X + si, u, tg);
                a.z[my_e + (size_t)k * NB] = (double)u;
            }
        }
        prefetch(s + 1);
        // red[s & 1] is next written at task s + 2, after every thread has
        // passed the barrier of task s + 1
    }
    if (blockIdx.x == 0 && tid == 0) advance_tag(a.tagp, tag0, (unsigned int)a.ntags);
}

constexpr int SW_CT = 288, SW_CPT = 2, SW_MAXSLOT = 6;
constexpr size_t SW_SMEM_MAX = 220 * 1024;

// ---------------------------------------------------------------------------
// Host: the task table.  Tasks of group 0 come first; the task with index s
// in group g has uid s (g = 0) or ntask0 + s (g = 1), and writes its slice
// with tag tag0 + uid.
// ---------------------------------------------------------------------------
int sweep_plan(int M, int h, int twisted, SweepPlan &P)
{
    P = SweepPlan();
    if (M < 1 || h < 0 || h + 1 > SW_BMAX) return BFS_EINVAL;
    const bool two = twisted && h >= 1 && M - h >= 2;
    std::vector<SweepTask> G[2];
    auto task = [](int k, int out) {
        SweepTask t;
        memset(&t, 0, sizeof t);
        t.k = k;
        t.out = out;
        return t;
    };
    auto blk = [](SweepTask &t, int m, int x, int plus) {
        t.m[t.nblk] = m;
        t.vec[t.nblk] = x | (plus << 1);
        t.nblk++;
    };
    if (!two) {
        for (int k = 0; k < M; k++) {  // forward: y_k = x_k - L_ki y_i
            SweepTask t = task(k, 0);
            for (int i = std::max(0, k - h); i < k; i++) blk(t, i, 0, 0);
            G[0].push_back(t);
        }
        for (int k = M - 1; k >= 0; k--) {  // backward: z_k = D_k^-1 y_k - W_kj z_j
            SweepTask t = task(k, 1);
            blk(t, k, 0, 1);
            for (int j = k + 1; j <= std::min(M - 1, k + h); j++) blk(t, j, 1, 0);
            G[0].push_back(t);
        }
    } else {
        const int t0 = (M - h) / 2, t1 = t0 + h;  // middle slices [t0, t1)
        for (int k = 0; k < t0; k++) {  // top chain, forward
            SweepTask t = task(k, 0);
            for (int i = std::max(0, k - h); i < k; i++) blk(t, i, 0, 0);
            G[0].push_back(t);
        }
        for (int k = M - 1; k >= t1; k--) {  // bottom chain, upward: y_k = x_k - U'_kj y_j
            SweepTask t = task(k, 0);
            for (int j = k + 1; j <= std::min(M - 1, k + h); j++) blk(t, j, 0, 0);
            G[1].push_back(t);
        }
        for (int g = 0; g < 2; g++)  // middle y: both chains' terms (the groups alternate slices)
            for (int m = t0 + g; m < t1; m += 2) {
                SweepTask t = task(m, 0);
                for (int i = std::max(0, m - h); i < t0; i++) blk(t, i, 0, 0);
                for (int j = t1; j <= std::min(M - 1, m + h); j++) blk(t, j, 0, 0);
                G[g].push_back(t);
            }
        for (int g = 0; g < 2; g++)  // middle z = C^-1 y_mid
            for (int m = t0 + g; m < t1; m += 2) {
                SweepTask t = task(m, 1);
                for (int q = t0; q < t1; q++) blk(t, q, 0, 1);
                G[g].push_back(t);
            }
        for (int k = t0 - 1; k >= 0; k--) {  // top chain, backward
            SweepTask t = task(k, 1);
            blk(t, k, 0, 1);
            for (int j = k + 1; j <= std::min(M - 1, k + h); j++) blk(t, j, 1, 0);
            G[0].push_back(t);
        }
        for (int k = t1; k < M; k++) {  // bottom chain, downward: z_k = D_k^-1 y_k - W'_kj z_j
            SweepTask t = task(k, 1);
            blk(t, k, 0, 1);
            for (int j = std::max(0, k - h); j < k; j++) blk(t, j, 1, 0);
            G[1].push_back(t);
        }
        P.twist = t0;
        P.groups = 2;
    }
    P.ntask[0] = (int)G[0].size();
    P.ntask[1] = (int)G[1].size();
    std::vector<int> prodY(M, -1), prodX(M, -1);
    for (int g = 0; g < 2; g++)
        for (int s = 0; s < P.ntask[g]; s++) {
            int &pr = (G[g][s].out ? prodX : prodY)[G[g][s].k];
            if (pr >= 0) return BFS_EINVAL;  // every vector slice has one writer
            pr = (g ? P.ntask[0] : 0) + s;
        }
    for (int g = 0; g < 2; g++)
        for (int s = 0; s < P.ntask[g]; s++) {
            SweepTask &t = G[g][s];
            const int prev = s > 0 ? (g ? P.ntask[0] : 0) + s - 1 : -1;
            int last = -1;
            for (int p = 0; p < t.nblk; p++) {
                const int u = ((t.vec[p] & 1) ? prodX : prodY)[t.m[p]];
                if (u < 0) return BFS_EINVAL;
                t.uid[p] = u;
                if (u == prev) last = p;
            }
            if (last >= 0 && last != t.nblk - 1) {  // the freshest vector last
                std::swap(t.m[last], t.m[t.nblk - 1]);
                std::swap(t.vec[last], t.vec[t.nblk - 1]);
                std::swap(t.uid[last], t.uid[t.nblk - 1]);
            }
        }
    // where each thread finds its columns of a block's vector: the group's
    // previous task wrote it (SW_CRIT: polled last); one of the last SW_HW
    // critical vectors the thread holds in registers (SW_WIN, with its index);
    // otherwise loaded at the end of the step before (SW_EARLY)
    for (int g = 0; g < 2; g++) {
        std::vector<int> win;  // uids of the vectors in the register window, newest first
        for (int s = 0; s < P.ntask[g]; s++) {
            SweepTask &t = G[g][s];
            const int prev = s > 0 ? (g ? P.ntask[0] : 0) + s - 1 : -1;
            int crit = -1;
            for (int p = 0; p < t.nblk; p++) {
                int src = SW_EARLY, wi = 0;
                if (t.uid[p] == prev) {
                    src = SW_CRIT;
                    crit = t.uid[p];
                } else {
                    for (int i = 0; i < (int)win.size(); i++)
                        if (win[i] == t.uid[p]) { src = SW_WIN; wi = i; }
                }
                t.vec[p] = (t.vec[p] & 3) | (src << 2) | (wi << 4);
            }
            if (crit >= 0) {
                win.insert(win.begin(), crit);
                if ((int)win.size() > SW_HW) win.pop_back();
            }
        }
    }
    P.tasks = G[0];
    P.tasks.insert(P.tasks.end(), G[1].begin(), G[1].end());
    return BFS_OK;
}

using FlowKernel = void (*)(FlowArgs);

static FlowKernel pick_flow(int rpc, int cpt)
{
    if (rpc <= 4 && cpt <= 2) return k_apply_flow<4, 2>;
    if (rpc <= 8 && cpt <= 2) return k_apply_flow<8, 2>;
    if (rpc <= 8 && cpt <= 3) return k_apply_flow<8, 3>;
    return nullptr;
}

// Shape of the task-table kernel for nb-wide slice blocks, half band h,
// `groups` CTA groups on G SMs and at most ntask tasks per group (staged in
// shared memory after the ring); false if its tiles do not take them.
static bool sweep_shape(int nb, int h, int groups, int G, int ntask, FlowKernel &kern, int &rpc, int &nslot,
                        size_t &dyn)
{
    const int ldp = (nb + 3) / 4 * 4;
    if (nb > SW_CT * SW_CPT || h + 1 > SW_BMAX || G < groups) return false;
    const int Gg = G / groups;  // the smaller group
    const int rows = (nb + Gg - 1) / Gg;
    if (rows <= 4) {
        rpc = 4;
        kern = k_apply_sweep<SW_CT, 4, SW_CPT>;
    } else if (rows <= 8) {
        rpc = 8;
        kern = k_apply_sweep<SW_CT, 8, SW_CPT>;
    } else {
        return false;
    }
    const size_t slot = (size_t)SW_BMAX * rpc * ldp * sizeof(float);
    const size_t tbytes = (size_t)ntask * sizeof(SweepTask);
    if (tbytes + 2 * slot > SW_SMEM_MAX) return false;
    nslot = (int)std::min<size_t>(SW_MAXSLOT, (SW_SMEM_MAX - tbytes) / slot);
    dyn = slot * nslot + tbytes;
    return true;
}

// 1 if the FP32 sweeps of this context can run the two-chain (twisted)
// schedule for half band h, so that the factorisation should take that order.
int sweep_twist_ok(bfs_ctx *c, int h)
{
    if (c->opt.precond_precision != BFS_FP32C || c->opt.surface_tension != 0.0) return 0;
    if (h < 1 || c->M - h < 2) return 0;
    SweepPlan P;
    if (sweep_plan(c->M, h, 1, P) != BFS_OK || P.groups != 2) return 0;
    FlowKernel kern;
    int rpc, nslot;
    size_t dyn;
    if (!sweep_shape(3 * (c->N + 1), h, 2, num_sms(c->device), std::max(P.ntask[0], P.ntask[1]), kern, rpc,
                     nslot, dyn))
        return 0;
    BFS_CUDA_TRY(c, cudaFuncSetAttribute((const void *)kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)SW_SMEM_MAX));
    int per_sm = 0;
    BFS_CUDA_TRY(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, SW_CT + 32, dyn));
    return per_sm >= 1 ? 1 : 0;
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
int flow_reset(bfs_ctx *c, cudaStream_t s)
{
    if (!c->d_flow) return BFS_OK;
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
    const unsigned long long steps = (unsigned long long)std::max(c->sweep_ntags, 2 * c->M);
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
    cudaFree(c->d_tasks);
    c->d_pc32 = nullptr;
    c->d_flow = nullptr;
    c->d_tasks = nullptr;
    c->sweep_table = 0;
    if (cudaMalloc(&c->d_pc32, sizeof(float) * cnt) != cudaSuccess ||
        cudaMalloc(&c->d_flow, sizeof(unsigned long long) * (2 * nv + 1)) != cudaSuccess) {
        cudaGetLastError();
        c->err = "FP32 preconditioner copy: out of device memory";
        return BFS_ENOMEM;
    }
    // the task table: two chains if the factors are in the two-ended order
    const int twisted = c->pc_twist >= 0;
    FlowKernel kern;
    int rpc = 0, nslot = 0;
    size_t dyn = 0;
    c->sweep_ntags = 2 * c->M;
    SweepPlan P;
    const bool planned = sweep_plan(c->M, c->pc_h, twisted, P) == BFS_OK;  // h <= 3 only
    if (twisted && (!planned || P.twist != c->pc_twist)) {
        c->err = "sweep schedule does not match the factor order";
        return BFS_EINVAL;
    }
    if (planned && sweep_shape(c->nb, c->pc_h, twisted ? 2 : 1, num_sms(c->device),
                               std::max(P.ntask[0], P.ntask[1]), kern, rpc, nslot, dyn)) {
        BFS_CUDA_TRY(c, cudaMalloc(&c->d_tasks, sizeof(SweepTask) * P.tasks.size()));
        BFS_CUDA_TRY(c, cudaMemcpy(c->d_tasks, P.tasks.data(), sizeof(SweepTask) * P.tasks.size(),
                                   cudaMemcpyHostToDevice));
        c->h_tasks = P.tasks;
        c->sweep_table = 1;
        c->sweep_groups = P.groups;
        c->sweep_ntask[0] = P.ntask[0];
        c->sweep_ntask[1] = P.ntask[1];
        c->sweep_ntags = P.ntask[0] + P.ntask[1];
        c->sweep_rpc = rpc;
        c->sweep_nslot = nslot;
        c->sweep_dyn = dyn;
    } else if (twisted) {
        c->err = "two-ended factors need the task-table sweep kernel";
        return BFS_EINVAL;
    }
    int rc = flow_reset(c, s);
    if (rc) return rc;
    k_cast_f32<<<4 * num_sms(c->device), 256, 0, s>>>(c->d_pc, c->d_pc32, rows, c->nb, ldp);
    c->launches++;
    BFS_CUDA_TRY(c, cudaGetLastError());
    return BFS_OK;
}

static unsigned int spin_limit(const bfs_ctx *c)
{
    return c->opt.wait_polls > 0 ? (unsigned int)c->opt.wait_polls : FL_SPIN;
}

// Returns 1 if launched, 0 if this apply is not for the FP32 sweep kernels
// (FP64 sweeps, or slice blocks wider than their tiles), or a negative code.
int apply_flow_launch(bfs_ctx *c, const double *r, double *z, cudaStream_t s)
{
    if (c->opt.precond_precision != BFS_FP32C || !c->d_pc32 || !c->d_flow) return 0;
    const int G = num_sms(c->device);
    FlowArgs a;
    a.pc = c->d_pc32;
    a.r = r; a.z = z;
    a.Y = c->d_flow;
    a.X = c->d_flow + (size_t)c->M * c->nb;
    a.nb = c->nb; a.NB = c->N + 1; a.M = c->M; a.h = c->pc_h;
    a.ldp = c->ldp32;
    a.tagp = reinterpret_cast<unsigned int *>(c->d_flow + 2 * (size_t)c->M * c->nb);
    a.flag = c->d_flag;
    a.spin = spin_limit(c);
    a.tasks = c->d_tasks;
    a.ntask0 = c->sweep_ntask[0];
    a.ntask1 = c->sweep_ntask[1];
    a.G0 = c->sweep_groups == 2 ? G / 2 : G;
    a.ntags = c->sweep_ntags;
    a.nslot = c->sweep_nslot;
    FlowKernel kern;
    int tpb;
    size_t dyn = 0;
    if (c->sweep_table) {
        kern = c->sweep_rpc == 4 ? k_apply_sweep<SW_CT, 4, SW_CPT> : k_apply_sweep<SW_CT, 8, SW_CPT>;
        tpb = SW_CT + 32;
        dyn = c->sweep_dyn;
    } else {
        const int rpc = (c->nb + G - 1) / G, cpt = (c->nb + FL_TPB - 1) / FL_TPB;
        kern = pick_flow(rpc, cpt);
        tpb = FL_TPB;
        if (!kern) return 0;
    }
    if (!c->flow_checked) {
        if (c->sweep_table)  // one ceiling for every context, whatever its ring depth
            BFS_CUDA_TRY(c, cudaFuncSetAttribute((const void *)kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)SW_SMEM_MAX));
        int per_sm = 0;
        BFS_CUDA_TRY(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, tpb, dyn));
        if (per_sm < 1) {
            if (c->pc_twist >= 0) {
                c->err = "the two-chain sweep kernel cannot be resident";
                return BFS_ECUDA;
            }
            return 0;
        }
        c->flow_checked = 1;
    }
    if (!c->capturing) {
        int rc = flow_wrap_check(c, s);
        if (rc) return rc;
    }
    // test hook: one wait of this launch is for a vector no task writes
    const bool stall = c->sweep_table && c->dbg_stall_task >= 0 && !c->capturing;
    if (stall) {
        std::vector<SweepTask> bad = c->h_tasks;
        SweepTask &t = bad[c->dbg_stall_task];
        if (t.nblk > 0) t.uid[0] = c->sweep_ntags;  // the tag of the next launch's first task
        BFS_CUDA_TRY(c, cudaMemcpyAsync(c->d_tasks, bad.data(), sizeof(SweepTask) * bad.size(),
                                        cudaMemcpyHostToDevice, s));
        BFS_CUDA_TRY(c, cudaStreamSynchronize(s));
    }
    void *args[] = {&a};
    cudaError_t e = cudaLaunchCooperativeKernel((const void *)kern, dim3(G), dim3(tpb), args, dyn, s);
    if (stall) {
        c->dbg_stall_task = -1;
        BFS_CUDA_TRY(c, cudaMemcpyAsync(c->d_tasks, c->h_tasks.data(), sizeof(SweepTask) * c->h_tasks.size(),
                                        cudaMemcpyHostToDevice, s));
        BFS_CUDA_TRY(c, cudaStreamSynchronize(s));
    }
    BFS_CUDA_TRY(c, e);
    c->launches++;
    c->flow_count++;
    return 1;
}

}  // namespace bfs

extern "C" {

int bfs_sweep_schedule(int M, int half_band, int twisted, int *tasks_out, int cap, int *ntask_out)
{
    bfs::SweepPlan P;
    if (bfs::sweep_plan(M, half_band, twisted, P) != BFS_OK) return BFS_EINVAL;
    if (ntask_out) {
        ntask_out[0] = P.ntask[0];
        ntask_out[1] = P.ntask[1];
    }
    const int n = (int)P.tasks.size();
    if (tasks_out) {
        if (cap < n) return BFS_EINVAL;
        static_assert(sizeof(bfs::SweepTask) == sizeof(int) * (4 + 3 * bfs::SW_BMAX), "task layout");
        memcpy(tasks_out, P.tasks.data(), sizeof(bfs::SweepTask) * n);
    }
    return n;
}

int bfs_debug_stall_sweep(bfs_ctx *c, int task)
{
    if (!c) return BFS_EINVAL;
    if (!c->pc_ready || !c->sweep_table) {
        c->err = "the stall hook needs the FP32 task-table sweeps";
        return BFS_EINVAL;
    }
    if (task < 0 || task >= (int)c->h_tasks.size() || c->h_tasks[task].nblk == 0) {
        c->err = "no waiting block in that task";
        return BFS_EINVAL;
    }
    c->dbg_stall_task = task;
    return BFS_OK;
}

}  // extern "C"
