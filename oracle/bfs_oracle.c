/*
 * bfs_oracle.c -- plain, slow, FP64 CPU oracle for the boundary-integral
 * collocation scheme of Buttle, Pethiyagoda, Moroney & McCue,
 * "Three-dimensional free-surface flow over arbitrary bottom topography"
 * (arXiv:1709.08803).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or
 * calls this file: only tests/, __graft_entry__.smoke() and bench.py's CPU
 * baseline leg use it.  It shares no code, header, table or helper with the
 * CUDA library under paper_1709_08803_gb300/csrc.
 *
 * Everything here follows the paper's steps in the paper's order, with no
 * blocking, fusion or reordering:
 *   - unknown vector u and its slice layout ............ Sec. 3.1, the vector of unknowns
 *   - trapezoid reconstruction of nodal values ......... Sec. 3.1 ("trapezoidal rule"),
 *                                                         implied by the App. B Jacobian
 *   - boundary integral equation, kernels K1, K2 ....... Sec. 2.2, boundary integral equation
 *   - singularity subtraction I2 = I2' + I2'' .......... Sec. 3.1
 *   - collocation at half mesh points (top, bottom) .... Sec. 3.1
 *   - combined dynamic condition ....................... Sec. 2.1, combined dynamic condition
 *   - radiation conditions (Scullen) ................... Sec. 3.1, Scullen conditions
 *   - residual ordering ................................ App. B
 *   - linearised discrete system, kernels K5, K6, K7 ... Sec. 4.2, App. B
 *   - preconditioner = Jacobian of the linear system ... Sec. 4.2, App. A (banding)
 *   - damped inexact Newton, right-preconditioned GMRES,
 *     finite-difference Jacobian-vector product ........ Sec. 3.2
 *
 * Readings taken where the paper is silent or at odds with itself:
 *   R1  y-derivatives at nodes: second-order central differences, second-order
 *       one-sided at the outer rows; mirror ghost (derivative 0) on y = 0 in the
 *       half domain.                                           (Sec. 3.1 is silent)
 *   R2  values at half mesh points are the mean of the two neighbouring nodes
 *       (the App. B Jacobian coefficients 1/2, 3/4, 1/4 are exactly this).
 *   R3  bottom collocation swaps the roles of the sheets: the bottom is the
 *       self sheet, its double layer carries the (psi - psi*) subtraction and
 *       its single layer the S2 subtraction (App. B, F7).
 *   R4  the bottom single layer I4 carries a sign sigma; Green's second
 *       identity with outward normals and the bottom kinematic condition give
 *       sigma = -1, the paper prints +1.  sigma is an input here.
 *   R5  closed-form I2'' is the rectangle sum of the printed antiderivative,
 *       evaluated in a cancellation-free form where its log argument is small.
 *   R6  half domain: nodes with y >= 0, y1 = 0, mirrored images (x, -y) of the
 *       rows j >= 2 added as sources with zeta_y, beta_y negated.
 *   R14 surface tension (Sec. 6 names the term, tension times mean curvature
 *       in the dynamic condition, and leaves it to future work): F1 gains
 *       -tau * kappa with kappa = div(grad zeta / sqrt(1 + |grad zeta|^2)),
 *       expanded as ((1+zy^2) zxx - 2 zx zy zxy + (1+zx^2) zyy) / w^(3/2),
 *       w = 1 + zx^2 + zy^2, at the half point: zx, zy its averages, zxx and
 *       zxy the x-differences of the nodal zeta_x, zeta_y across it, zyy the
 *       mean of the nodal second y-differences (central; second-order
 *       one-sided on outer rows; mirror ghost on y = 0 of the half domain).
 *       The linearised system gains -tau (zxx + zyy).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

typedef struct {
    int N, M;              /* nodes in x and in y (Sec. 3.1) */
    int half;              /* 1: half domain y >= 0 with mirror images (R6) */
    double x1, y1, dx, dy; /* first node and spacings (Sec. 3.1) */
    double F;              /* depth-based Froude number (Sec. 2.1) */
    double n_rad;          /* upstream decay rate n of the radiation condition */
    double sigma;          /* sign of the bottom single layer I4 (R4) */
    const double *psurf;   /* applied surface pressure at the nodes, or NULL
                              (the pressure-distribution problem of Sec. 4.1:
                              p adds to the dynamic condition) */
    double tau;            /* surface tension parameter (0: none): the dynamic
                              condition gains -tau * kappa, kappa the mean-curvature
                              operator of the surface (Sec. 6, reading R14) */
} orc_problem;

typedef struct {
    int newton_its, krylov_its, residual_evals, status;
    double fnorm_inf, fnorm_2;
} orc_stats;

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

static int orc_n(const orc_problem *P) { return 3 * (P->N + 1) * P->M; }

int orc_lu_factor(int n, double *A, int *piv);
void orc_lu_solve(int n, const double *LU, const int *piv, const double *b, double *x);

/* ------------------------------------------------------------------ */
/* Unknown vector -> nodal values (Sec. 3.1, the vector of unknowns).          */
/* Per slice j and field q: u holds q(x1, y_j) followed by q_x at the   */
/* N nodes; nodal values follow from the trapezoid rule in x.           */
/* ------------------------------------------------------------------ */
static void orc_unpack_field(const orc_problem *P, const double *u, int field,
                             double *q, double *qx)
{
    int N = P->N, M = P->M;
    for (int j = 0; j < M; j++) {
        const double *s = u + (size_t)field * (N + 1) * M + (size_t)j * (N + 1);
        double *qj = q + (size_t)j * N, *qxj = qx + (size_t)j * N;
        for (int i = 0; i < N; i++) qxj[i] = s[1 + i];
        qj[0] = s[0];
        for (int i = 1; i < N; i++) qj[i] = qj[i - 1] + 0.5 * P->dx * (qxj[i - 1] + qxj[i]);
    }
}

/* y-derivative at the nodes (reading R1). */
static void orc_ydiff(const orc_problem *P, const double *q, double *qy)
{
    int N = P->N, M = P->M;
    double h = P->dy;
    for (int j = 0; j < M; j++)
        for (int i = 0; i < N; i++) {
            double v;
#define Q(jj) q[(size_t)(jj) * N + i]
            if (j == 0) {
                if (P->half) v = 0.0; /* mirror ghost: q(-y) = q(y) */
                else v = (-3.0 * Q(0) + 4.0 * Q(1) - Q(2)) / (2.0 * h);
            } else if (j == M - 1) {
                v = (3.0 * Q(M - 1) - 4.0 * Q(M - 2) + Q(M - 3)) / (2.0 * h);
            } else {
                v = (Q(j + 1) - Q(j - 1)) / (2.0 * h);
            }
#undef Q
            qy[(size_t)j * N + i] = v;
        }
}

/* Second y-derivative of the nodal field q at node (i, j) (reading R14):
   central (q_{j-1} - 2 q_j + q_{j+1}) / dy^2 inside; on an outer row the
   second-order one-sided (2 q_0 - 5 q_1 + 4 q_2 - q_3) / dy^2 (first-order
   q_0 - 2 q_1 + q_2 when M = 3); on y = 0 of the half domain the mirror ghost
   q_{-1} = q_1 gives (2 q_1 - 2 q_0) / dy^2. */
static double orc_yy(const orc_problem *P, const double *q, int i, int j)
{
    int N = P->N, M = P->M;
    double h2 = P->dy * P->dy;
#define Q(jj) q[(size_t)(jj) * N + i]
    double v;
    if (j == 0) {
        if (P->half) v = 2.0 * (Q(1) - Q(0));
        else if (M >= 4) v = 2.0 * Q(0) - 5.0 * Q(1) + 4.0 * Q(2) - Q(3);
        else v = Q(0) - 2.0 * Q(1) + Q(2);
    } else if (j == M - 1) {
        if (M >= 4) v = 2.0 * Q(M - 1) - 5.0 * Q(M - 2) + 4.0 * Q(M - 3) - Q(M - 4);
        else v = Q(M - 1) - 2.0 * Q(M - 2) + Q(M - 3);
    } else {
        v = Q(j - 1) - 2.0 * Q(j) + Q(j + 1);
    }
#undef Q
    return v / h2;
}

/* ------------------------------------------------------------------ */
/* Closed form of the integral of S2 over a rectangle (Sec. 3.1).       */
/* The antiderivative of (A s^2 + B s t + C t^2)^(-1/2) is              */
/*   G = t/sqrt(A) ln(2As + Bt + 2 sqrt(A Q)) + s/sqrt(C) ln(2Ct + Bs + 2 sqrt(C Q)). */
/* Where 2As + Bt < 0 the log argument is rewritten with                */
/*   (2As+Bt+2sqrt(AQ))(2sqrt(AQ)-2As-Bt) = (4AC-B^2) t^2  (reading R5). */
/* ------------------------------------------------------------------ */
static double orc_G(double A, double B, double C, double s, double t)
{
    double Q = A * s * s + B * s * t + C * t * t;
    double D = 4.0 * A * C - B * B;
    double g = 0.0;
    if (t != 0.0) { /* t/sqrt(A) ln(2As + Bt + 2 sqrt(AQ)); the product is 0 at t = 0 */
        double lin = 2.0 * A * s + B * t, r = 2.0 * sqrt(A * Q);
        double L = lin >= 0.0 ? log(lin + r) : log(D * t * t) - log(r - lin);
        g += t / sqrt(A) * L;
    }
    if (s != 0.0) { /* s/sqrt(C) ln(2Ct + Bs + 2 sqrt(CQ)); the product is 0 at s = 0 */
        double lin = 2.0 * C * t + B * s, r = 2.0 * sqrt(C * Q);
        double L = lin >= 0.0 ? log(lin + r) : log(D * s * s) - log(r - lin);
        g += s / sqrt(C) * L;
    }
    return g;
}

double orc_rect_S2(double A, double B, double C, double s1, double s2, double t1, double t2)
{
    return orc_G(A, B, C, s2, t2) - orc_G(A, B, C, s1, t2) - orc_G(A, B, C, s2, t1) +
           orc_G(A, B, C, s1, t1);
}

/* ------------------------------------------------------------------ */
/* Kernels of the boundary integral equation (Sec. 2.2).               */
/* ------------------------------------------------------------------ */
static double orc_K1(double s, double t, double a, double b, double c, double d)
{
    double r2 = s * s + t * t + (a - d) * (a - d);
    return (a - d - s * b - t * c) / (r2 * sqrt(r2));
}

static double orc_K2(double s, double t, double a, double d)
{
    return 1.0 / sqrt(s * s + t * t + (a - d) * (a - d));
}

/* Trapezoid weight of node (i, j) (Sec. 3.1); the half domain counts the
   row y = 0 once as an interior row (R6). */
static double orc_weight(const orc_problem *P, int i, int j)
{
    double cx = (i == 0 || i == P->N - 1) ? 0.5 : 1.0;
    double cy;
    if (P->half) cy = (j == P->M - 1) ? 0.5 : 1.0;
    else cy = (j == 0 || j == P->M - 1) ? 0.5 : 1.0;
    return P->dx * P->dy * cx * cy;
}

/* A sheet z = h(x, y) with double-layer density d and single-layer density s,
   all at the N x M nodes (index i + N j). */
typedef struct {
    const double *h, *hx, *hy, *d, *s;
} orc_sheet;

/* One collocation point on a sheet. */
typedef struct {
    double x, y;   /* position */
    double z;      /* height of the sheet there */
    double u;      /* double-layer density there */
    double sd;     /* single-layer density there */
    double px, py; /* slopes of the self sheet there (for S2) */
} orc_target;

/*
 * Green's second identity at a point on the self sheet (Sec. 2.2, boundary integral equation
 * and Sec. 3.1).  Returns
 *   sum over the top sheet of    w [ d K1(top) + s K2(top) ]
 * + sum over the bottom sheet of w [ d (-K1(bot)) + s K2(bot) ]
 * with, on the self sheet, d replaced by (d - u*) and s K2 replaced by
 * s K2 - s* S2, plus s* times the closed-form integral of S2.  The caller
 * subtracts 2 pi u*.  *scale receives the sum of the absolute values of all
 * terms (used to normalise parity checks).
 */
double orc_bie_point(const orc_problem *P, const orc_sheet *top, const orc_sheet *bot,
                     int self_bottom, const orc_target *T, double *scale)
{
    int N = P->N, M = P->M;
    double A = 1.0 + T->px * T->px, B = 2.0 * T->px * T->py, C = 1.0 + T->py * T->py;
    double sum = 0.0, sabs = 0.0;
    int nimg = P->half ? 2 : 1;
    for (int img = 0; img < nimg; img++) {
        double ysgn = img ? -1.0 : 1.0;
        for (int j = 0; j < M; j++) {
            if (img && j == 0) continue; /* y = 0 row has no separate image */
            double yj = ysgn * (P->y1 + j * P->dy);
            for (int i = 0; i < N; i++) {
                size_t q = (size_t)j * N + i;
                double w = orc_weight(P, i, j);
                double s = P->x1 + i * P->dx - T->x, t = yj - T->y;
                /* top sheet */
                {
                    double k1 = orc_K1(s, t, top->h[q], top->hx[q], ysgn * top->hy[q], T->z);
                    double k2 = orc_K2(s, t, top->h[q], T->z);
                    double dd = top->d[q] - (self_bottom ? 0.0 : T->u);
                    double a = w * dd * k1, b = w * top->s[q] * k2, c = 0.0;
                    if (!self_bottom) c = -w * T->sd / sqrt(A * s * s + B * s * t + C * t * t);
                    sum += a + b + c;
                    sabs += fabs(a) + fabs(b) + fabs(c);
                }
                /* bottom sheet */
                {
                    double k1 = orc_K1(s, t, bot->h[q], bot->hx[q], ysgn * bot->hy[q], T->z);
                    double k2 = orc_K2(s, t, bot->h[q], T->z);
                    double dd = bot->d[q] - (self_bottom ? T->u : 0.0);
                    double a = -w * dd * k1, b = w * bot->s[q] * k2, c = 0.0;
                    if (self_bottom) c = -w * T->sd / sqrt(A * s * s + B * s * t + C * t * t);
                    sum += a + b + c;
                    sabs += fabs(a) + fabs(b) + fabs(c);
                }
            }
        }
    }
    double ylo = P->half ? -(P->y1 + (M - 1) * P->dy) : P->y1;
    double yhi = P->y1 + (M - 1) * P->dy;
    double xhi = P->x1 + (N - 1) * P->dx;
    double cf = T->sd * orc_rect_S2(A, B, C, P->x1 - T->x, xhi - T->x, ylo - T->y, yhi - T->y);
    sum += cf;
    sabs += fabs(cf);
    if (scale) *scale = sabs;
    return sum;
}

/* ------------------------------------------------------------------ */
/* Nonlinear residual F(u) (Sec. 3.1; ordering App. B).                 */
/* ------------------------------------------------------------------ */
typedef struct {
    double *z, *zx, *zy, *ph, *phx, *phy, *ps, *psx, *f, *g, *bs;
} orc_nodal;

static void orc_nodal_alloc(const orc_problem *P, orc_nodal *nd)
{
    size_t n = (size_t)P->N * P->M;
    double *b = (double *)calloc(11 * n, sizeof(double));
    nd->z = b; nd->zx = b + n; nd->zy = b + 2 * n; nd->ph = b + 3 * n; nd->phx = b + 4 * n;
    nd->phy = b + 5 * n; nd->ps = b + 6 * n; nd->psx = b + 7 * n; nd->f = b + 8 * n;
    nd->g = b + 9 * n; nd->bs = b + 10 * n;
}

static void orc_nodal_free(orc_nodal *nd) { free(nd->z); }

static void orc_nodal_fill(const orc_problem *P, const double *u, const double *bx,
                           orc_nodal *nd)
{
    int N = P->N, M = P->M;
    orc_unpack_field(P, u, 0, nd->z, nd->zx);
    orc_unpack_field(P, u, 1, nd->ph, nd->phx);
    orc_unpack_field(P, u, 2, nd->ps, nd->psx);
    orc_ydiff(P, nd->z, nd->zy);
    orc_ydiff(P, nd->ph, nd->phy);
    for (int j = 0; j < M; j++)
        for (int i = 0; i < N; i++) {
            size_t q = (size_t)j * N + i;
            double x = P->x1 + i * P->dx;
            nd->f[q] = nd->ph[q] - x;
            nd->g[q] = nd->ps[q] - x;
            nd->bs[q] = P->sigma * (bx ? bx[q] : 0.0);
        }
}

/* Row index of each equation in F (App. B ordering). */
static size_t orc_row_F1(const orc_problem *P, int k, int l) { return (size_t)l * (P->N + 1) + 2 + k; }
static size_t orc_row_F2(const orc_problem *P, int k, int l) { return (size_t)(P->N + 1) * P->M + orc_row_F1(P, k, l); }
static size_t orc_row_F7(const orc_problem *P, int k, int l) { return 2 * (size_t)(P->N + 1) * P->M + orc_row_F1(P, k, l); }

/* Radiation conditions (Sec. 3.1, Scullen conditions); second derivatives at
   x1 are the forward difference of the first derivatives. */
static void orc_radiation(const orc_problem *P, const orc_nodal *nd, double *Fv, double *sc)
{
    int N = P->N, M = P->M;
    size_t blk = (size_t)(N + 1) * M;
    double x1 = P->x1, n = P->n_rad, h = P->dx;
    for (int l = 0; l < M; l++) {
        size_t q = (size_t)l * N, r = (size_t)l * (N + 1);
        double z1 = nd->z[q], zx1 = nd->zx[q], zx2 = nd->zx[q + 1];
        double p1 = nd->ph[q], px1 = nd->phx[q], px2 = nd->phx[q + 1];
        double s1 = nd->ps[q], sx1 = nd->psx[q], sx2 = nd->psx[q + 1];
        double t[12];
        t[0] = x1 * zx1;          t[1] = n * z1;                      /* F5 */
        t[2] = x1 * (zx2 - zx1) / h; t[3] = n * zx1;                  /* F6 */
        t[4] = x1 * (px1 - 1.0);  t[5] = n * (p1 - x1);               /* F3 */
        t[6] = x1 * (px2 - px1) / h; t[7] = n * (px1 - 1.0);          /* F4 */
        t[8] = x1 * (sx1 - 1.0);  t[9] = n * (s1 - x1);               /* F8 */
        t[10] = x1 * (sx2 - sx1) / h; t[11] = n * (sx1 - 1.0);        /* F9 */
        size_t rows[6] = {r, r + 1, blk + r, blk + r + 1, 2 * blk + r, 2 * blk + r + 1};
        for (int e = 0; e < 6; e++) {
            Fv[rows[e]] = t[2 * e] + t[2 * e + 1];
            if (sc) sc[rows[e]] = fabs(t[2 * e]) + fabs(t[2 * e + 1]);
        }
    }
}

/* Combined dynamic condition at a half point (Sec. 2.1, combined dynamic
   condition); an applied surface pressure p* enters as + p* (Sec. 4.1). */
static double orc_bernoulli(double F, double z, double zx, double zy, double px, double py,
                            double *sc)
{
    double num = (1.0 + zx * zx) * py * py + (1.0 + zy * zy) * px * px - 2.0 * zx * zy * px * py;
    double kin = 0.5 * num / (1.0 + zx * zx + zy * zy);
    double grav = z / (F * F);
    if (sc) *sc = fabs(kin) + fabs(grav) + 0.5;
    return kin + grav - 0.5;
}

/*
 * F(u): u has 3(N+1)M entries (Sec. 3.1), beta/beta_x/beta_y are nodal
 * (index i + N j).  Fout receives 3(N+1)M residuals in App. B order; scale
 * (optional) the per-row sum of absolute term values.
 */
void orc_residual(const orc_problem *P, const double *beta, const double *bx, const double *by,
                  const double *u, double *Fout, double *scale)
{
    int N = P->N, M = P->M;
    orc_nodal nd;
    orc_nodal_alloc(P, &nd);
    orc_nodal_fill(P, u, bx, &nd);
    orc_sheet top = {nd.z, nd.zx, nd.zy, nd.f, nd.zx};
    orc_sheet bot = {beta, bx, by, nd.g, nd.bs};
    orc_radiation(P, &nd, Fout, scale);
    int nt = (N - 1) * M;
#pragma omp parallel for schedule(dynamic, 4)
    for (int e = 0; e < nt; e++) {
        int k = e % (N - 1), l = e / (N - 1);
        size_t a = (size_t)l * N + k, b = a + 1;
#define AV(arr) (0.5 * ((arr)[a] + (arr)[b]))
        double xs = P->x1 + (k + 0.5) * P->dx, ys = P->y1 + l * P->dy;
        /* half-point values (reading R2) */
        double zs = AV(nd.z), zxs = AV(nd.zx), zys = AV(nd.zy);
        double pxs = AV(nd.phx), pys = AV(nd.phy), fs = AV(nd.f), gs = AV(nd.g);
        double bts = AV(beta), bxs = AV(bx), bys = AV(by);
#undef AV
        double sc2, sc7, sc1;
        orc_target Tt = {xs, ys, zs, fs, zxs, zxs, zys};
        double I = orc_bie_point(P, &top, &bot, 0, &Tt, &sc2);
        Fout[orc_row_F2(P, k, l)] = I - 2.0 * ORC_PI * fs;
        orc_target Tb = {xs, ys, bts, gs, P->sigma * bxs, bxs, bys};
        double J = orc_bie_point(P, &top, &bot, 1, &Tb, &sc7);
        Fout[orc_row_F7(P, k, l)] = J - 2.0 * ORC_PI * gs;
        Fout[orc_row_F1(P, k, l)] = orc_bernoulli(P->F, zs, zxs, zys, pxs, pys, &sc1);
        if (P->tau != 0.0) {
            /* mean curvature at the half point: zeta_xx, zeta_xy as x-differences
               of the nodal zeta_x, zeta_y across the half point, zeta_yy the mean
               of the two nodal second y-differences (reading R14) */
            double zxx = (nd.zx[b] - nd.zx[a]) / P->dx;
            double zxy = (nd.zy[b] - nd.zy[a]) / P->dx;
            double zyy = 0.5 * (orc_yy(P, nd.z, k, l) + orc_yy(P, nd.z, k + 1, l));
            double w = 1.0 + zxs * zxs + zys * zys;
            double kap = ((1.0 + zys * zys) * zxx - 2.0 * zxs * zys * zxy + (1.0 + zxs * zxs) * zyy) /
                         (w * sqrt(w));
            Fout[orc_row_F1(P, k, l)] -= P->tau * kap;
            sc1 += fabs(P->tau * kap);
        }
        if (P->psurf) {
            double pstar = 0.5 * (P->psurf[a] + P->psurf[b]);
            Fout[orc_row_F1(P, k, l)] += pstar;
            sc1 += fabs(pstar);
        }
        if (scale) {
            scale[orc_row_F2(P, k, l)] = sc2 + 2.0 * ORC_PI * fabs(fs);
            scale[orc_row_F7(P, k, l)] = sc7 + 2.0 * ORC_PI * fabs(gs);
            scale[orc_row_F1(P, k, l)] = sc1;
        }
    }
    orc_nodal_free(&nd);
}

/* Nodal reconstruction exposed for tests: zeta, zeta_x, zeta_y, phi, phi_x,
   phi_y, psi, psi_x, each N*M (index i + N j). */
void orc_nodal_values(const orc_problem *P, const double *u, double *out)
{
    size_t n = (size_t)P->N * P->M;
    orc_nodal nd;
    orc_nodal_alloc(P, &nd);
    orc_nodal_fill(P, u, NULL, &nd);
    memcpy(out + 0 * n, nd.z, n * sizeof(double));
    memcpy(out + 1 * n, nd.zx, n * sizeof(double));
    memcpy(out + 2 * n, nd.zy, n * sizeof(double));
    memcpy(out + 3 * n, nd.ph, n * sizeof(double));
    memcpy(out + 4 * n, nd.phx, n * sizeof(double));
    memcpy(out + 5 * n, nd.phy, n * sizeof(double));
    memcpy(out + 6 * n, nd.ps, n * sizeof(double));
    memcpy(out + 7 * n, nd.psx, n * sizeof(double));
    orc_nodal_free(&nd);
}

/* ------------------------------------------------------------------ */
/* Linearised discrete system (Sec. 4.2, App. B).                       */
/* K5 = 1/r, K6 = (r^2+1)^(-3/2), K7 = (r^2+1)^(-1/2), r the horizontal */
/* distance from node (i,j) to the half point (k,l).                    */
/* ------------------------------------------------------------------ */
void orc_residual_linear(const orc_problem *P, const double *bx, const double *u, double *Fout)
{
    int N = P->N, M = P->M;
    orc_nodal nd;
    orc_nodal_alloc(P, &nd);
    orc_nodal_fill(P, u, NULL, &nd);
    orc_radiation(P, &nd, Fout, NULL);
    double ylo = P->half ? -(P->y1 + (M - 1) * P->dy) : P->y1;
    double yhi = P->y1 + (M - 1) * P->dy, xhi = P->x1 + (N - 1) * P->dx;
    int nt = (N - 1) * M;
#pragma omp parallel for schedule(dynamic, 4)
    for (int e = 0; e < nt; e++) {
        int k = e % (N - 1), l = e / (N - 1);
        size_t a = (size_t)l * N + k, b = a + 1;
        double xs = P->x1 + (k + 0.5) * P->dx, ys = P->y1 + l * P->dy;
        double zs = 0.5 * (nd.z[a] + nd.z[b]), zxs = 0.5 * (nd.zx[a] + nd.zx[b]);
        double pxs = 0.5 * (nd.phx[a] + nd.phx[b]);
        double fs = 0.5 * (nd.f[a] + nd.f[b]), gs = 0.5 * (nd.g[a] + nd.g[b]);
        double bxs = bx ? 0.5 * (bx[a] + bx[b]) : 0.0;
        double s2 = 0.0, s7 = 0.0;
        int nimg = P->half ? 2 : 1;
        for (int img = 0; img < nimg; img++)
            for (int j = 0; j < M; j++) {
                if (img && j == 0) continue;
                double yj = (img ? -1.0 : 1.0) * (P->y1 + j * P->dy);
                for (int i = 0; i < N; i++) {
                    size_t q = (size_t)j * N + i;
                    double w = orc_weight(P, i, j);
                    double s = P->x1 + i * P->dx - xs, t = yj - ys, r2 = s * s + t * t;
                    double K5 = 1.0 / sqrt(r2), K7 = 1.0 / sqrt(r2 + 1.0), K6 = K7 * K7 * K7;
                    double bxq = bx ? bx[q] : 0.0;
                    s2 += w * ((nd.zx[q] - zxs) * K5 + P->sigma * bxq * K7 + nd.g[q] * K6);
                    s7 += w * (nd.zx[q] * K7 + P->sigma * (bxq - bxs) * K5 + nd.f[q] * K6);
                }
            }
        double iK5 = orc_rect_S2(1.0, 0.0, 1.0, P->x1 - xs, xhi - xs, ylo - ys, yhi - ys);
        Fout[orc_row_F1(P, k, l)] = pxs + zs / (P->F * P->F) - 1.0;
        if (P->tau != 0.0) /* linearised curvature: zeta_xx + zeta_yy */
            Fout[orc_row_F1(P, k, l)] -= P->tau * ((nd.zx[b] - nd.zx[a]) / P->dx +
                                                    0.5 * (orc_yy(P, nd.z, k, l) + orc_yy(P, nd.z, k + 1, l)));
        Fout[orc_row_F2(P, k, l)] = s2 + zxs * iK5 - 2.0 * ORC_PI * fs;
        Fout[orc_row_F7(P, k, l)] = s7 + P->sigma * bxs * iK5 - 2.0 * ORC_PI * gs;
    }
    orc_nodal_free(&nd);
}

/*
 * Jacobian of the linear discrete system (Sec. 4.2: P = J~).  The system is
 * affine in u, so column c is F_lin(e_c) - F_lin(0), exactly.  J is n x n,
 * row-major (J[r*n + c]).  If half_band >= 0, entries whose row slice and
 * column slice differ by more than half_band are dropped (App. A banding).
 */
void orc_jtilde(const orc_problem *P, int half_band, double *J)
{
    int n = orc_n(P);
    double *e = (double *)calloc((size_t)n, sizeof(double));
    double *F0 = (double *)malloc((size_t)n * sizeof(double));
    double *Fc = (double *)malloc((size_t)n * sizeof(double));
    orc_residual_linear(P, NULL, e, F0);
    for (int c = 0; c < n; c++) {
        e[c] = 1.0;
        orc_residual_linear(P, NULL, e, Fc);
        e[c] = 0.0;
        for (int r = 0; r < n; r++) J[(size_t)r * n + c] = Fc[r] - F0[r];
    }
    if (half_band >= 0) {
        int per = P->N + 1, blk = per * P->M;
        for (int r = 0; r < n; r++)
            for (int c = 0; c < n; c++) {
                int sr = (r % blk) / per, sc = (c % blk) / per;
                if (abs(sr - sc) > half_band) J[(size_t)r * n + c] = 0.0;
            }
    }
    free(e); free(F0); free(Fc);
}

/* ------------------------------------------------------------------ */
/* Banded linear Jacobian, block by block (Sec. 4.2 with the banding of */
/* App. A), for meshes whose dense J~ does not fit in memory.           */
/* ------------------------------------------------------------------ */
/*
 * Unknowns and equations regrouped slice by slice: slice l owns the
 * nb = 3(N+1) equations [F5, F6, F1(1..N-1) | F3, F4, F2(1..N-1) | F8, F9,
 * F7(1..N-1)] and the nb unknowns [zeta(1), zeta_x(1..N) | phi(1), phi_x |
 * psi(1), psi_x] of that slice, i.e. the rows and columns of J~ with slice
 * index l, in the order they have in F and in u.  Block (l, m), |l - m| <= h,
 * is stored at Bk + (l (2h+1) + m - l + h) nb^2, row-major.
 *
 * The linear system is affine in u, so column c of J~ is the change of the
 * linear residual of orc_residual_linear when unknown c goes from 0 to 1
 * (the constants of f = phi - x, g = psi - x, the -1 of the dynamic condition
 * and of the radiation conditions cancel).  That unknown changes the nodal
 * values of its own slice m only (the trapezoid rule acts along x; the linear
 * residual uses no y-derivative), so the change of each sum over sources
 * comes from the sources of slice m and, in the half domain, their mirror
 * images; the target's own half-point values enter only the rows of slice m.
 * Surface tension, whose curvature term couples slices, is not supported.
 */
int orc_jtilde_band(const orc_problem *P, int h, double *Bk)
{
    int N = P->N, M = P->M, NB = N + 1, nb = 3 * NB, nd = 2 * h + 1;
    size_t bsz = (size_t)nb * nb;
    if (P->tau != 0.0 || h < 0) return -1;
    memset(Bk, 0, (size_t)M * nd * bsz * sizeof(double));
    double ylo = P->half ? -(P->y1 + (M - 1) * P->dy) : P->y1;
    double yhi = P->y1 + (M - 1) * P->dy, xhi = P->x1 + (N - 1) * P->dx;
    int nt = (N - 1) * M;
    /* per target: sum over all sources of w K5 (the subtraction of zeta_x*)
       and the closed-form integral of K5 over the truncated domain */
    double *R5 = (double *)malloc((size_t)nt * sizeof(double));
    double *I5 = (double *)malloc((size_t)nt * sizeof(double));
#pragma omp parallel for schedule(dynamic, 4)
    for (int e = 0; e < nt; e++) {
        int k = e % (N - 1), l = e / (N - 1);
        double xs = P->x1 + (k + 0.5) * P->dx, ys = P->y1 + l * P->dy, acc = 0.0;
        for (int img = 0; img < (P->half ? 2 : 1); img++)
            for (int j = 0; j < M; j++) {
                if (img && j == 0) continue;
                double yj = (img ? -1.0 : 1.0) * (P->y1 + j * P->dy);
                for (int i = 0; i < N; i++) {
                    double s = P->x1 + i * P->dx - xs, t = yj - ys;
                    acc += orc_weight(P, i, j) / sqrt(s * s + t * t);
                }
            }
        R5[e] = acc;
        I5[e] = orc_rect_S2(1.0, 0.0, 1.0, P->x1 - xs, xhi - xs, ylo - ys, yhi - ys);
    }
#pragma omp parallel
    {
        double *e = (double *)calloc((size_t)orc_n(P), sizeof(double));
        double *q = (double *)malloc((size_t)N * M * sizeof(double));
        double *qx = (double *)malloc((size_t)N * M * sizeof(double));
#pragma omp for schedule(dynamic, 8)
        for (int col = 0; col < M * nb; col++) {
            int m = col / nb, cl = col % nb, g = cl / NB, p = cl % NB;
            size_t uc = (size_t)g * NB * M + (size_t)m * NB + p; /* index in u */
            e[uc] = 1.0;
            orc_unpack_field(P, e, g, q, qx); /* nodal change of field g (slice m only) */
            e[uc] = 0.0;
            const double *dq = q + (size_t)m * N, *dqx = qx + (size_t)m * N;
            /* per field: zeta enters through zeta_x (K5 top, K7 bottom targets) and
               zeta (dynamic condition); phi through f (K6 at bottom targets) and
               phi_x (dynamic condition); psi through g (K6 at top targets) */
            for (int l = (m - h > 0 ? m - h : 0); l <= (m + h < M - 1 ? m + h : M - 1); l++) {
                double *blk = Bk + ((size_t)l * nd + (m - l + h)) * bsz;
                for (int k = 0; k < N - 1; k++) {
                    double xs = P->x1 + (k + 0.5) * P->dx, ys = P->y1 + l * P->dy;
                    double s2 = 0.0, s7 = 0.0;
                    for (int img = 0; img < (P->half ? 2 : 1); img++) {
                        if (img && m == 0) continue;
                        double yj = (img ? -1.0 : 1.0) * (P->y1 + m * P->dy);
                        for (int i = 0; i < N; i++) {
                            double w = orc_weight(P, i, m);
                            double s = P->x1 + i * P->dx - xs, t = yj - ys, r2 = s * s + t * t;
                            double K5 = 1.0 / sqrt(r2), K7 = 1.0 / sqrt(r2 + 1.0), K6 = K7 * K7 * K7;
                            if (g == 0) { s2 += w * dqx[i] * K5; s7 += w * dqx[i] * K7; }
                            else if (g == 1) s7 += w * dq[i] * K6;
                            else s2 += w * dq[i] * K6;
                        }
                    }
                    double F1 = 0.0, F2 = s2, F7 = s7;
                    if (l == m) { /* the target's own half-point values */
                        double hq = 0.5 * (dq[k] + dq[k + 1]), hqx = 0.5 * (dqx[k] + dqx[k + 1]);
                        int et = l * (N - 1) + k;
                        if (g == 0) { F1 = hq / (P->F * P->F); F2 += hqx * (I5[et] - R5[et]); }
                        else if (g == 1) { F1 = hqx; F2 -= 2.0 * ORC_PI * hq; }
                        else F7 -= 2.0 * ORC_PI * hq;
                    }
                    blk[(size_t)(0 * NB + 2 + k) * nb + cl] = F1;
                    blk[(size_t)(1 * NB + 2 + k) * nb + cl] = F2;
                    blk[(size_t)(2 * NB + 2 + k) * nb + cl] = F7;
                }
                if (l == m) { /* radiation rows of slice m: their linear parts */
                    double x1 = P->x1, n = P->n_rad, hx = P->dx;
                    double v1 = dq[0], d1 = dqx[0], d2 = dqx[1];
                    blk[(size_t)(g * NB + 0) * nb + cl] = x1 * d1 + n * v1;
                    blk[(size_t)(g * NB + 1) * nb + cl] = x1 * (d2 - d1) / hx + n * d1;
                }
            }
        }
        free(e); free(q); free(qx);
    }
    free(R5); free(I5);
    return 0;
}

/*
 * In-place block LU of the banded matrix (App. A: no pivoting across blocks,
 * partial pivoting inside each diagonal block):
 *   for k = 0..M-1:  D_k = B(k,k) = Pi L U (orc_lu_factor, pivots at piv + k nb);
 *     B(k,j) <- D_k^-1 B(k,j)          for j = k+1..k+h
 *     B(i,j) <- B(i,j) - B(i,k) B(k,j)  for i, j = k+1..k+h
 * Returns -1 on a zero pivot.
 */
int orc_band_factor(int M, int nb, int h, double *Bk, int *piv)
{
    int nd = 2 * h + 1;
    size_t bsz = (size_t)nb * nb;
#define ORC_B(l, m) (Bk + ((size_t)(l) * nd + ((m) - (l) + h)) * bsz)
    double *col = (double *)malloc((size_t)nb * sizeof(double));
    for (int k = 0; k < M; k++) {
        double *D = ORC_B(k, k);
        if (orc_lu_factor(nb, D, piv + (size_t)k * nb)) { free(col); return -1; }
        int hi = k + h < M - 1 ? k + h : M - 1;
        for (int j = k + 1; j <= hi; j++) {
            double *U = ORC_B(k, j);
            for (int c = 0; c < nb; c++) {
                for (int r = 0; r < nb; r++) col[r] = U[(size_t)r * nb + c];
                orc_lu_solve(nb, D, piv + (size_t)k * nb, col, col);
                for (int r = 0; r < nb; r++) U[(size_t)r * nb + c] = col[r];
            }
        }
        for (int i = k + 1; i <= hi; i++)
            for (int j = k + 1; j <= hi; j++) {
                const double *L = ORC_B(i, k), *U = ORC_B(k, j);
                double *S = ORC_B(i, j);
#pragma omp parallel for schedule(static)
                for (int r = 0; r < nb; r++)
                    for (int t = 0; t < nb; t++) {
                        double a = L[(size_t)r * nb + t];
                        if (a != 0.0)
                            for (int c = 0; c < nb; c++) S[(size_t)r * nb + c] -= a * U[(size_t)t * nb + c];
                    }
            }
    }
    free(col);
    return 0;
}

/*
 * z = P^-1 r with the factors of orc_band_factor; r in the order of F, z in
 * the order of u (both regrouped by slice inside):
 *   forward  w_k = D_k^-1 (r_k - sum_{i=k-h}^{k-1} B(k,i) w_i)
 *   backward z_k = w_k - sum_{j=k+1}^{k+h} B(k,j) z_j
 */
void orc_band_solve(int N, int M, int h, const double *Bk, const int *piv, const double *r, double *z)
{
    int NB = N + 1, nb = 3 * NB, nd = 2 * h + 1;
    size_t bsz = (size_t)nb * nb;
    double *w = (double *)malloc((size_t)M * nb * sizeof(double));
    for (int l = 0; l < M; l++)
        for (int g = 0; g < 3; g++)
            for (int p = 0; p < NB; p++)
                w[(size_t)l * nb + g * NB + p] = r[(size_t)g * NB * M + (size_t)l * NB + p];
    for (int k = 0; k < M; k++) {
        double *wk = w + (size_t)k * nb;
        for (int i = (k - h > 0 ? k - h : 0); i < k; i++) {
            const double *L = ORC_B(k, i), *wi = w + (size_t)i * nb;
            for (int a = 0; a < nb; a++) {
                double s = 0.0;
                for (int b = 0; b < nb; b++) s += L[(size_t)a * nb + b] * wi[b];
                wk[a] -= s;
            }
        }
        orc_lu_solve(nb, ORC_B(k, k), piv + (size_t)k * nb, wk, wk);
    }
    for (int k = M - 1; k >= 0; k--) {
        double *zk = w + (size_t)k * nb;
        for (int j = k + 1; j <= (k + h < M - 1 ? k + h : M - 1); j++) {
            const double *U = ORC_B(k, j), *zj = w + (size_t)j * nb;
            for (int a = 0; a < nb; a++) {
                double s = 0.0;
                for (int b = 0; b < nb; b++) s += U[(size_t)a * nb + b] * zj[b];
                zk[a] -= s;
            }
        }
    }
    for (int l = 0; l < M; l++)
        for (int g = 0; g < 3; g++)
            for (int p = 0; p < NB; p++)
                z[(size_t)g * NB * M + (size_t)l * NB + p] = w[(size_t)l * nb + g * NB + p];
    free(w);
#undef ORC_B
}

/* Finite-difference Jacobian of F (column c: (F(u + h e_c) - F(u)) / h). */
void orc_fd_jacobian(const orc_problem *P, const double *beta, const double *bx,
                     const double *by, const double *u, double *J)
{
    int n = orc_n(P);
    double *up = (double *)malloc((size_t)n * sizeof(double));
    double *F0 = (double *)malloc((size_t)n * sizeof(double));
    double *Fc = (double *)malloc((size_t)n * sizeof(double));
    memcpy(up, u, (size_t)n * sizeof(double));
    orc_residual(P, beta, bx, by, u, F0, NULL);
    for (int c = 0; c < n; c++) {
        double h = 1.4901161193847656e-08 * fmax(fabs(u[c]), 1.0);
        up[c] = u[c] + h;
        h = up[c] - u[c];
        orc_residual(P, beta, bx, by, up, Fc, NULL);
        up[c] = u[c];
        for (int r = 0; r < n; r++) J[(size_t)r * n + c] = (Fc[r] - F0[r]) / h;
    }
    free(up); free(F0); free(Fc);
}

/* ------------------------------------------------------------------ */
/* Dense LU with partial pivoting (textbook Doolittle, row-major).      */
/* ------------------------------------------------------------------ */
int orc_lu_factor(int n, double *A, int *piv)
{
    for (int k = 0; k < n; k++) {
        int p = k;
        double best = fabs(A[(size_t)k * n + k]);
        for (int i = k + 1; i < n; i++)
            if (fabs(A[(size_t)i * n + k]) > best) { best = fabs(A[(size_t)i * n + k]); p = i; }
        piv[k] = p;
        if (best == 0.0) return -1;
        if (p != k)
            for (int c = 0; c < n; c++) {
                double t = A[(size_t)k * n + c];
                A[(size_t)k * n + c] = A[(size_t)p * n + c];
                A[(size_t)p * n + c] = t;
            }
        double d = A[(size_t)k * n + k];
#pragma omp parallel for schedule(static)
        for (int i = k + 1; i < n; i++) {
            double l = A[(size_t)i * n + k] / d;
            A[(size_t)i * n + k] = l;
            if (l != 0.0)
                for (int c = k + 1; c < n; c++) A[(size_t)i * n + c] -= l * A[(size_t)k * n + c];
        }
    }
    return 0;
}

void orc_lu_solve(int n, const double *LU, const int *piv, const double *b, double *x)
{
    if (x != b) memcpy(x, b, (size_t)n * sizeof(double));
    for (int k = 0; k < n; k++)
        if (piv[k] != k) { double t = x[k]; x[k] = x[piv[k]]; x[piv[k]] = t; }
    for (int i = 0; i < n; i++) {
        double s = x[i];
        for (int c = 0; c < i; c++) s -= LU[(size_t)i * n + c] * x[c];
        x[i] = s;
    }
    for (int i = n - 1; i >= 0; i--) {
        double s = x[i];
        for (int c = i + 1; c < n; c++) s -= LU[(size_t)i * n + c] * x[c];
        x[i] = s / LU[(size_t)i * n + i];
    }
}

/* ------------------------------------------------------------------ */
/* Jacobian-free Newton-Krylov (Sec. 3.2).                              */
/* ------------------------------------------------------------------ */
static double orc_norm2(int n, const double *v)
{
    double s = 0.0;
    for (int i = 0; i < n; i++) s += v[i] * v[i];
    return sqrt(s);
}

static double orc_norminf(int n, const double *v)
{
    double s = 0.0;
    for (int i = 0; i < n; i++) s = fmax(s, fabs(v[i]));
    return s;
}

typedef struct {
    const orc_problem *P;
    const double *beta, *bx, *by;
    const double *LU; const int *piv; /* preconditioner P = LU (dense) or NULL */
    int n, evals;
    double *tmp_u, *tmp_F;
    const double *Bk; const int *bpiv; int h; /* or the banded block LU of orc_band_factor */
} orc_ctx;

static void orc_eval(orc_ctx *c, const double *u, double *Fv)
{
    orc_residual(c->P, c->beta, c->bx, c->by, u, Fv, NULL);
    c->evals++;
}

static void orc_prec(orc_ctx *c, const double *r, double *z)
{
    if (c->LU) orc_lu_solve(c->n, c->LU, c->piv, r, z);
    else if (c->Bk) orc_band_solve(c->P->N, c->P->M, c->h, c->Bk, c->bpiv, r, z);
    else if (z != r) memcpy(z, r, (size_t)c->n * sizeof(double));
}

/* J z ~ (F(u + h z) - F(u)) / h, h = sqrt(eps) (1 + |u|) / |z| (Sec. 3.2). */
static void orc_jv(orc_ctx *c, const double *u, const double *Fu, const double *z, double *Jz)
{
    int n = c->n;
    double zn = orc_norm2(n, z);
    if (zn == 0.0) { memset(Jz, 0, (size_t)n * sizeof(double)); return; }
    double h = 1.4901161193847656e-08 * (1.0 + orc_norm2(n, u)) / zn;
    for (int i = 0; i < n; i++) c->tmp_u[i] = u[i] + h * z[i];
    orc_eval(c, c->tmp_u, c->tmp_F);
    for (int i = 0; i < n; i++) Jz[i] = (c->tmp_F[i] - Fu[i]) / h;
}

/*
 * Right-preconditioned restarted GMRES (Saad & Schultz) for J P^-1 y = -F,
 * returning du = P^-1 y.  Modified Gram-Schmidt Arnoldi, Givens rotations.
 * Stops when the residual estimate is <= eta |F|.  Returns iterations used.
 */
static int orc_gmres(orc_ctx *c, const double *u, const double *Fu, double eta, int m,
                     int maxit, double *du)
{
    int n = c->n, its = 0;
    double *V = (double *)malloc((size_t)(m + 1) * n * sizeof(double));
    double *H = (double *)calloc((size_t)(m + 1) * m, sizeof(double));
    double *cs = (double *)malloc((size_t)m * sizeof(double));
    double *sn = (double *)malloc((size_t)m * sizeof(double));
    double *g = (double *)malloc((size_t)(m + 1) * sizeof(double));
    double *y = (double *)malloc((size_t)m * sizeof(double));
    double *z = (double *)malloc((size_t)n * sizeof(double));
    double *w = (double *)malloc((size_t)n * sizeof(double));
    double fn = orc_norm2(n, Fu);
    memset(du, 0, (size_t)n * sizeof(double));
    double *r = (double *)malloc((size_t)n * sizeof(double));
    for (int i = 0; i < n; i++) r[i] = -Fu[i];
    while (its < maxit) {
        double beta = orc_norm2(n, r);
        if (beta <= eta * fn) break;
        for (int i = 0; i < n; i++) V[i] = r[i] / beta;
        memset(g, 0, (size_t)(m + 1) * sizeof(double));
        g[0] = beta;
        int j;
        for (j = 0; j < m && its < maxit; j++, its++) {
            orc_prec(c, V + (size_t)j * n, z);
            orc_jv(c, u, Fu, z, w);
            for (int i = 0; i <= j; i++) {
                double h = 0.0;
                for (int q = 0; q < n; q++) h += w[q] * V[(size_t)i * n + q];
                H[(size_t)i * m + j] = h;
                for (int q = 0; q < n; q++) w[q] -= h * V[(size_t)i * n + q];
            }
            double hn = orc_norm2(n, w);
            H[(size_t)(j + 1) * m + j] = hn;
            if (hn > 0.0)
                for (int q = 0; q < n; q++) V[(size_t)(j + 1) * n + q] = w[q] / hn;
            for (int i = 0; i < j; i++) {
                double a = H[(size_t)i * m + j], b = H[(size_t)(i + 1) * m + j];
                H[(size_t)i * m + j] = cs[i] * a + sn[i] * b;
                H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * b;
            }
            double a = H[(size_t)j * m + j], b = H[(size_t)(j + 1) * m + j];
            double d = sqrt(a * a + b * b);
            cs[j] = d > 0.0 ? a / d : 1.0;
            sn[j] = d > 0.0 ? b / d : 0.0;
            H[(size_t)j * m + j] = d;
            H[(size_t)(j + 1) * m + j] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            if (fabs(g[j + 1]) <= eta * fn || hn == 0.0) { j++; its++; break; }
        }
        /* y = H^-1 g, x += P^-1 V y */
        for (int i = j - 1; i >= 0; i--) {
            double s = g[i];
            for (int q = i + 1; q < j; q++) s -= H[(size_t)i * m + q] * y[q];
            y[i] = s / H[(size_t)i * m + i];
        }
        memset(w, 0, (size_t)n * sizeof(double));
        for (int i = 0; i < j; i++)
            for (int q = 0; q < n; q++) w[q] += y[i] * V[(size_t)i * n + q];
        orc_prec(c, w, z);
        for (int q = 0; q < n; q++) du[q] += z[q];
        if (fabs(g[j]) <= eta * fn || its >= maxit) break;
        /* restart: r = -F - J du */
        orc_jv(c, u, Fu, du, w);
        for (int q = 0; q < n; q++) r[q] = -Fu[q] - w[q];
    }
    free(V); free(H); free(cs); free(sn); free(g); free(y); free(z); free(w); free(r);
    return its;
}

/*
 * Damped inexact Newton with backtracking line search (Sec. 3.2).
 * half_band = -1 means the full linear Jacobian J~ as preconditioner; >= 0
 * its banded form (dense storage); -2 no preconditioner; -3 - h the banded
 * form with half band h in block storage, factored by orc_band_factor (for
 * meshes whose dense J~ does not fit in memory).  Returns 0 when
 * |F|_inf <= tol, 1 when the iteration limit is reached, 2 when the line
 * search fails, 3 on a singular preconditioner.
 */
int orc_jfnk(const orc_problem *P, const double *beta, const double *bx, const double *by,
             double *u, int half_band, double tol, int max_newton, int restart,
             int max_krylov, double eta, orc_stats *st)
{
    int n = orc_n(P);
    orc_ctx c = {P, beta, bx, by, NULL, NULL, n, 0, NULL, NULL, NULL, NULL, 0};
    c.tmp_u = (double *)malloc((size_t)n * sizeof(double));
    c.tmp_F = (double *)malloc((size_t)n * sizeof(double));
    double *LU = NULL; int *piv = NULL;
    int status = 1;
    memset(st, 0, sizeof(*st));
    if (half_band <= -3) {
        /* banded block LU (orc_jtilde_band + orc_band_factor), half band -3 - half_band */
        int h = -3 - half_band, nb = 3 * (P->N + 1);
        LU = (double *)malloc((size_t)P->M * (2 * h + 1) * nb * nb * sizeof(double));
        piv = (int *)malloc((size_t)P->M * nb * sizeof(int));
        if (orc_jtilde_band(P, h, LU) || orc_band_factor(P->M, nb, h, LU, piv)) { status = 3; goto done; }
        c.Bk = LU; c.bpiv = piv; c.h = h;
    } else if (half_band != -2) {
        LU = (double *)malloc((size_t)n * n * sizeof(double));
        piv = (int *)malloc((size_t)n * sizeof(int));
        orc_jtilde(P, half_band < 0 ? -1 : half_band, LU);
        if (orc_lu_factor(n, LU, piv)) { status = 3; goto done; }
        c.LU = LU; c.piv = piv;
    }
    double *Fv = (double *)malloc((size_t)n * sizeof(double));
    double *du = (double *)malloc((size_t)n * sizeof(double));
    double *ut = (double *)malloc((size_t)n * sizeof(double));
    double *Ft = (double *)malloc((size_t)n * sizeof(double));
    orc_eval(&c, u, Fv);
    for (int k = 0; ; k++) {
        st->fnorm_inf = orc_norminf(n, Fv);
        st->fnorm_2 = orc_norm2(n, Fv);
        if (st->fnorm_inf <= tol) { status = 0; break; }
        if (k >= max_newton) { status = 1; break; }
        st->krylov_its += orc_gmres(&c, u, Fv, eta, restart, max_krylov, du);
        double f0 = st->fnorm_2, mu = 1.0;
        int ok = 0;
        while (mu >= 1e-4) {
            for (int i = 0; i < n; i++) ut[i] = u[i] + mu * du[i];
            orc_eval(&c, ut, Ft);
            if (orc_norm2(n, Ft) <= (1.0 - 1e-4 * mu) * f0) { ok = 1; break; }
            mu *= 0.5;
        }
        if (!ok) { status = 2; break; }
        memcpy(u, ut, (size_t)n * sizeof(double));
        memcpy(Fv, Ft, (size_t)n * sizeof(double));
        st->newton_its = k + 1;
    }
    free(Fv); free(du); free(ut); free(Ft);
done:
    st->residual_evals = c.evals;
    st->status = status;
    free(c.tmp_u); free(c.tmp_F); free(LU); free(piv);
    return status;
}

/*
 * Newton with the dense finite-difference Jacobian and a direct solve, for
 * tiny meshes; the same line search and stopping rule as orc_jfnk.
 */
int orc_newton_dense(const orc_problem *P, const double *beta, const double *bx,
                     const double *by, double *u, double tol, int max_newton, orc_stats *st)
{
    int n = orc_n(P), status = 1;
    double *J = (double *)malloc((size_t)n * n * sizeof(double));
    int *piv = (int *)malloc((size_t)n * sizeof(int));
    double *Fv = (double *)malloc((size_t)n * sizeof(double));
    double *du = (double *)malloc((size_t)n * sizeof(double));
    double *ut = (double *)malloc((size_t)n * sizeof(double));
    double *Ft = (double *)malloc((size_t)n * sizeof(double));
    memset(st, 0, sizeof(*st));
    orc_residual(P, beta, bx, by, u, Fv, NULL);
    st->residual_evals = 1;
    for (int k = 0; ; k++) {
        st->fnorm_inf = orc_norminf(n, Fv);
        st->fnorm_2 = orc_norm2(n, Fv);
        if (st->fnorm_inf <= tol) { status = 0; break; }
        if (k >= max_newton) { status = 1; break; }
        orc_fd_jacobian(P, beta, bx, by, u, J);
        st->residual_evals += n + 1;
        if (orc_lu_factor(n, J, piv)) { status = 3; break; }
        for (int i = 0; i < n; i++) du[i] = -Fv[i];
        orc_lu_solve(n, J, piv, du, du);
        double f0 = st->fnorm_2, mu = 1.0;
        int ok = 0;
        while (mu >= 1e-4) {
            for (int i = 0; i < n; i++) ut[i] = u[i] + mu * du[i];
            orc_residual(P, beta, bx, by, ut, Ft, NULL);
            st->residual_evals++;
            if (orc_norm2(n, Ft) <= (1.0 - 1e-4 * mu) * f0) { ok = 1; break; }
            mu *= 0.5;
        }
        if (!ok) { status = 2; break; }
        memcpy(u, ut, (size_t)n * sizeof(double));
        memcpy(Fv, Ft, (size_t)n * sizeof(double));
        st->newton_its = k + 1;
    }
    st->status = status;
    free(J); free(piv); free(Fv); free(du); free(ut); free(Ft);
    return status;
}

/* ------------------------------------------------------------------ */
/* Pressure on the bottom (Sec. 2.1: Bernoulli's equation along the    */
/* bottom, with the bottom kinematic condition folded in, written for   */
/* psi the bottom potential) and the force of the fluid on the          */
/* topography, integral of p (beta_x, beta_y, -1) dx dy by the          */
/* trapezoid rule (the outward normal of the fluid on the bottom times  */
/* dS is (beta_x, beta_y, -1) dx dy).  p: N*M nodal values; force: 3.   */
/* The half domain counts the mirror image of every row but y = 0 and   */
/* gives force[1] = 0.                                                  */
/* ------------------------------------------------------------------ */
void orc_bottom_pressure(const orc_problem *P, const double *beta, const double *bx,
                         const double *by, const double *u, double *p, double *force)
{
    int N = P->N, M = P->M;
    size_t n = (size_t)N * M;
    double *ps = (double *)malloc(n * sizeof(double)), *psx = (double *)malloc(n * sizeof(double));
    double *psy = (double *)malloc(n * sizeof(double));
    orc_unpack_field(P, u, 2, ps, psx);
    orc_ydiff(P, ps, psy);
    double fx = 0.0, fy = 0.0, fz = 0.0;
    for (int j = 0; j < M; j++)
        for (int i = 0; i < N; i++) {
            size_t q = (size_t)j * N + i;
            double a = bx[q], b = by[q], gx = psx[q], gy = psy[q];
            double kin = 0.5 * ((1.0 + a * a) * gy * gy + (1.0 + b * b) * gx * gx - 2.0 * a * b * gx * gy) /
                         (1.0 + a * a + b * b);
            double pv = 0.5 - kin - beta[q] / (P->F * P->F);
            p[q] = pv;
            double w = orc_weight(P, i, j) * ((P->half && j > 0) ? 2.0 : 1.0);
            fx += w * pv * a;
            fy += w * pv * b;
            fz -= w * pv;
        }
    force[0] = fx;
    force[1] = P->half ? 0.0 : fy;
    force[2] = fz;
    free(ps); free(psx); free(psy);
}
