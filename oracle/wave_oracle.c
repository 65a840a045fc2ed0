/*
 * wave_oracle.c -- plain, slow FP64 CPU oracle for the acoustic wave path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no code with the CUDA path.
 *
 * What it computes (FP64 throughout, arrays C-order [x][y][z], z contiguous,
 * the layout of the paper's generated code, Sec. 3.2.1 "CSE"):
 *
 *   Laplacian     L u = sum_a h_a^-2 [ c_0 u + sum_{k=1..r} c_k (u(+k e_a) + u(-k e_a)) ]
 *                 with u = 0 outside the grid (or periodic wrap, for the
 *                 plane-wave pin).  The c_k are an input (oracle/coeffs.py).
 *                 The paper only names Taylor's theorem (Sec. 2.1) and space
 *                 orders 4..16 (Sec. 5.8.1); the radius is r = so/2, the
 *                 minimum skew of Table "AWE results" (Sec. 5.8.2).
 *   Time step     leapfrog for m u_tt + damp u_t - lap u = f with a centred
 *                 damping term:
 *                 u^{n+1} = alpha (2 m u^n - (m - eta) u^{n-1} + dt^2 (L u^n + f^n)),
 *                 eta = damp dt / 2, alpha = 1 / (m + eta), u^0 = u^-1 = 0.
 *   Sources       f^n[p] = sum_s w_{s,p} q_s(t_n), trilinear weights over the
 *                 8 corners of the cell holding the source, no 1/h^3 factor.
 *   Receivers     d^n[r] = sum_p w_{r,p} u^{n+1}[p], n = 0..nt-1.
 *   Adjoint       lambda^k = dJ/du^k of J = sum_n <res^n, d^n>, obtained by
 *                 transposing each step of the forward recursion (no reuse
 *                 of the forward scheme).
 *   Gradient      dJ/dm = - sum_n lambda^{n+1} alpha (u^{n+1} - 2 u^n + u^{n-1}).
 *   Time tiling   the paper's skewed, time-tiled loop nest with min/max
 *                 bounds (Sec. 4.1 "Skewing", Sec. 4.2.2 "Min/max bounds"),
 *                 OpenMP on the incremental x loop (Sec. 4.2.3), with a
 *                 time buffer of tt+2 levels (Sec. 5.2.1 bound n + t with
 *                 n = 2 for leapfrog).  It must equal the untiled loop bitwise
 *                 (Sec. 4.3 "Test suite", Sec. 5.4.3 "Functional correctness").
 *
 * The damping form, source/receiver convention, adjoint and gradient are not
 * in the paper (its acoustic operator is "propagation only", Sec. 5.8.1); they
 * are the textbook readings listed in the design notes of this repository.
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -fPIC -shared (oracle/build.py).
 * -ffp-contract=off keeps every expression evaluated exactly as written, so
 * the untiled and tiled loops (which call the same point update) agree bitwise
 * on every host architecture.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------- */
/* Grid helpers                                                              */
/* ------------------------------------------------------------------------- */

static long npts(const int n[3]) { return (long)n[0] * n[1] * n[2]; }

static long at(const int n[3], long x, long y, long z)
{
    return (x * n[1] + y) * n[2] + z;
}

/* Value of u at (x,y,z) with a zero halo outside the grid, or periodic wrap. */
static double val(const int n[3], int periodic, const double *u, long x, long y, long z)
{
    if (periodic) {
        x = ((x % n[0]) + n[0]) % n[0];
        y = ((y % n[1]) + n[1]) % n[1];
        z = ((z % n[2]) + n[2]) % n[2];
        return u[at(n, x, y, z)];
    }
    if (x < 0 || x >= n[0] || y < 0 || y >= n[1] || z < 0 || z >= n[2]) return 0.0;
    return u[at(n, x, y, z)];
}

/* Order-2r central second-difference Laplacian at one point. */
static double lap_at(const int n[3], const double h[3], int r, const double *c,
                     int periodic, const double *u, long x, long y, long z)
{
    const long e[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    double sum = 0.0;
    for (int a = 0; a < 3; a++) {
        double acc = c[0] * val(n, periodic, u, x, y, z);
        for (int k = 1; k <= r; k++) {
            double plus = val(n, periodic, u, x + k * e[a][0], y + k * e[a][1], z + k * e[a][2]);
            double minus = val(n, periodic, u, x - k * e[a][0], y - k * e[a][1], z - k * e[a][2]);
            acc = acc + c[k] * (plus + minus);
        }
        sum = sum + acc / (h[a] * h[a]);
    }
    return sum;
}

/* One leapfrog point update with centred damping. */
static double update_point(double m, double damp, double dt,
                           double u, double um, double lap, double f)
{
    double eta = damp * dt / 2.0;
    double alpha = 1.0 / (m + eta);
    return alpha * (2.0 * m * u - (m - eta) * um + dt * dt * (lap + f));
}

/* ------------------------------------------------------------------------- */
/* Sparse points: trilinear weights over the 8 corners of the holding cell.  */
/* ------------------------------------------------------------------------- */

/* Corner c = 4*dx + 2*dy + dz; cell index floor(x/h) clamped to [0, n-2] so a
 * point on the upper face is still inside a cell. */
static void trilinear(const int n[3], const double h[3], const double *xyz,
                      long corner[8], double w[8])
{
    long cell[3];
    double f[3];
    for (int a = 0; a < 3; a++) {
        double s = xyz[a] / h[a];
        long i = (long)floor(s);
        if (i < 0) i = 0;
        if (i > n[a] - 2) i = n[a] - 2;
        cell[a] = i;
        f[a] = s - (double)i;
    }
    for (int cidx = 0; cidx < 8; cidx++) {
        int dx = (cidx >> 2) & 1, dy = (cidx >> 1) & 1, dz = cidx & 1;
        double wx = dx ? f[0] : 1.0 - f[0];
        double wy = dy ? f[1] : 1.0 - f[1];
        double wz = dz ? f[2] : 1.0 - f[2];
        corner[cidx] = at(n, cell[0] + dx, cell[1] + dy, cell[2] + dz);
        w[cidx] = wx * wy * wz;
    }
}

/* Sources: for every grid point, the list of (source, weight) contributions in
 * ascending source order.  slot[p] = -1 or an index into the unique points. */
typedef struct {
    int nsrc;
    long *slot;      /* [N] */
    int nuniq;
    long *first;     /* [nuniq+1] into contrib arrays */
    int *csrc;       /* [8*nsrc] source index per contribution */
    double *cw;      /* [8*nsrc] weight per contribution */
} srcmap_t;

static int srcmap_build(srcmap_t *sm, const int n[3], const double h[3],
                        int nsrc, const double *xyz)
{
    long N = npts(n);
    memset(sm, 0, sizeof(*sm));
    sm->nsrc = nsrc;
    sm->slot = (long *)malloc(sizeof(long) * N);
    if (!sm->slot) return -1;
    for (long p = 0; p < N; p++) sm->slot[p] = -1;
    if (nsrc <= 0) return 0;
    long *pts = (long *)malloc(sizeof(long) * 8 * nsrc);
    double *wts = (double *)malloc(sizeof(double) * 8 * nsrc);
    long *count = (long *)calloc(8 * (size_t)nsrc + 1, sizeof(long));
    sm->first = (long *)calloc(8 * (size_t)nsrc + 1, sizeof(long));
    sm->csrc = (int *)malloc(sizeof(int) * 8 * nsrc);
    sm->cw = (double *)malloc(sizeof(double) * 8 * nsrc);
    if (!pts || !wts || !count || !sm->first || !sm->csrc || !sm->cw) return -1;
    for (int s = 0; s < nsrc; s++) trilinear(n, h, xyz + 3 * s, pts + 8 * s, wts + 8 * s);
    /* unique points in first-appearance order */
    int nu = 0;
    for (int j = 0; j < 8 * nsrc; j++) {
        if (sm->slot[pts[j]] < 0) sm->slot[pts[j]] = nu++;
        count[sm->slot[pts[j]]]++;
    }
    sm->nuniq = nu;
    sm->first[0] = 0;
    for (int u = 0; u < nu; u++) sm->first[u + 1] = sm->first[u] + count[u];
    for (int u = 0; u < nu; u++) count[u] = 0;
    /* contributions in ascending source order (j runs over sources in order) */
    for (int j = 0; j < 8 * nsrc; j++) {
        long u = sm->slot[pts[j]];
        long k = sm->first[u] + count[u]++;
        sm->csrc[k] = j / 8;
        sm->cw[k] = wts[j];
    }
    free(pts);
    free(wts);
    free(count);
    return 0;
}

static void srcmap_free(srcmap_t *sm)
{
    free(sm->slot);
    free(sm->first);
    free(sm->csrc);
    free(sm->cw);
}

/* f^n at grid point p (0 if p holds no source). q is [nt][nsrc]. */
static double src_term(const srcmap_t *sm, const double *q, int step, long p)
{
    long u = sm->slot[p];
    if (u < 0) return 0.0;
    double f = 0.0;
    for (long k = sm->first[u]; k < sm->first[u + 1]; k++)
        f = f + sm->cw[k] * q[(long)step * sm->nsrc + sm->csrc[k]];
    return f;
}

/* Receivers: 8 corners and weights per receiver; a per-point list of the
 * (receiver, corner) slots that read it so that values can be recorded at the
 * moment a point is computed (needed by the tiled loop, whose time buffer
 * forgets old levels). */
typedef struct {
    int nrec;
    long *corner;    /* [8*nrec] */
    double *w;       /* [8*nrec] */
    long *slot;      /* [N] -1 or index into unique */
    long *first;     /* [nuniq+1] */
    long *cslot;     /* [8*nrec] receiver-corner slot (8*rec + c) */
} recmap_t;

static int recmap_build(recmap_t *rm, const int n[3], const double h[3],
                        int nrec, const double *xyz)
{
    long N = npts(n);
    memset(rm, 0, sizeof(*rm));
    rm->nrec = nrec;
    rm->slot = (long *)malloc(sizeof(long) * N);
    if (!rm->slot) return -1;
    for (long p = 0; p < N; p++) rm->slot[p] = -1;
    if (nrec <= 0) return 0;
    rm->corner = (long *)malloc(sizeof(long) * 8 * nrec);
    rm->w = (double *)malloc(sizeof(double) * 8 * nrec);
    rm->first = (long *)calloc(8 * (size_t)nrec + 1, sizeof(long));
    rm->cslot = (long *)malloc(sizeof(long) * 8 * nrec);
    long *count = (long *)calloc(8 * (size_t)nrec + 1, sizeof(long));
    if (!rm->corner || !rm->w || !rm->first || !rm->cslot || !count) return -1;
    for (int r = 0; r < nrec; r++) trilinear(n, h, xyz + 3 * r, rm->corner + 8 * r, rm->w + 8 * r);
    long nu = 0;
    for (long j = 0; j < 8L * nrec; j++) {
        if (rm->slot[rm->corner[j]] < 0) rm->slot[rm->corner[j]] = nu++;
        count[rm->slot[rm->corner[j]]]++;
    }
    for (long u = 0; u < nu; u++) rm->first[u + 1] = rm->first[u] + count[u];
    for (long u = 0; u < nu; u++) count[u] = 0;
    for (long j = 0; j < 8L * nrec; j++) {
        long u = rm->slot[rm->corner[j]];
        rm->cslot[rm->first[u] + count[u]++] = j;
    }
    free(count);
    return 0;
}

static void recmap_free(recmap_t *rm)
{
    free(rm->corner);
    free(rm->w);
    free(rm->slot);
    free(rm->first);
    free(rm->cslot);
}

/* Store the value of point p at a level into every receiver-corner slot that
 * reads p.  corners is [nt][8*nrec]. */
static void rec_record(const recmap_t *rm, double *corners, int step, long p, double v)
{
    long u = rm->slot[p];
    if (u < 0) return;
    for (long k = rm->first[u]; k < rm->first[u + 1]; k++)
        corners[(long)step * 8 * rm->nrec + rm->cslot[k]] = v;
}

/* d^n[r] = sum_c w_c * corner value, corners in ascending order. */
static void rec_finish(const recmap_t *rm, const double *corners, int nt, double *d)
{
    for (int s = 0; s < nt; s++)
        for (int r = 0; r < rm->nrec; r++) {
            double acc = 0.0;
            for (int c = 0; c < 8; c++)
                acc = acc + rm->w[8 * r + c] * corners[(long)s * 8 * rm->nrec + 8 * r + c];
            d[(long)s * rm->nrec + r] = acc;
        }
}

/* ------------------------------------------------------------------------- */
/* Public entry points (called through ctypes by oracle/__init__.py)         */
/* ------------------------------------------------------------------------- */

void oracle_set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* out = L u (zero halo, or periodic). */
void oracle_laplacian(const int *n, const double *h, int r, const double *c,
                      int periodic, const double *u, double *out)
{
#pragma omp parallel for schedule(static)
    for (long x = 0; x < n[0]; x++)
        for (long y = 0; y < n[1]; y++)
            for (long z = 0; z < n[2]; z++)
                out[at(n, x, y, z)] = lap_at(n, h, r, c, periodic, u, x, y, z);
}

/* Untiled forward.
 *   src_xyz [nsrc][3], src_q [nt][nsrc]; rec_xyz [nrec][3], rec_d [nt][nrec] out.
 *   u0, um1: optional initial levels u^0, u^-1 (NULL = zero).
 *   u_last [2][N] out: u^{nt}, u^{nt-1}.
 *   u_all  optional [nt+2][N] out: u^{-1}, u^0, ..., u^{nt}.
 * Returns 0 or -1 on allocation failure. */
int oracle_forward(const int *n, const double *h, double dt, int nt, int r, const double *c,
                   const double *m, const double *damp,
                   int nsrc, const double *src_xyz, const double *src_q,
                   int nrec, const double *rec_xyz, double *rec_d,
                   int periodic, const double *u0, const double *um1,
                   double *u_last, double *u_all)
{
    long N = npts(n);
    srcmap_t sm;
    recmap_t rm;
    if (srcmap_build(&sm, n, h, nsrc, src_xyz) || recmap_build(&rm, n, h, nrec, rec_xyz)) return -1;
    double *um = (double *)calloc(N, sizeof(double));
    double *u = (double *)calloc(N, sizeof(double));
    double *up = (double *)calloc(N, sizeof(double));
    double *corners = (double *)calloc((size_t)nt * 8 * (nrec > 0 ? nrec : 1), sizeof(double));
    if (!um || !u || !up || !corners) return -1;
    if (u0) memcpy(u, u0, sizeof(double) * N);
    if (um1) memcpy(um, um1, sizeof(double) * N);
    if (u_all) {
        memcpy(u_all, um, sizeof(double) * N);
        memcpy(u_all + N, u, sizeof(double) * N);
    }
    for (int step = 0; step < nt; step++) {
#pragma omp parallel for schedule(static)
        for (long x = 0; x < n[0]; x++)
            for (long y = 0; y < n[1]; y++)
                for (long z = 0; z < n[2]; z++) {
                    long p = at(n, x, y, z);
                    double lap = lap_at(n, h, r, c, periodic, u, x, y, z);
                    double f = src_term(&sm, src_q, step, p);
                    up[p] = update_point(m[p], damp[p], dt, u[p], um[p], lap, f);
                    rec_record(&rm, corners, step, p, up[p]);
                }
        double *t = um;
        um = u;
        u = up;
        up = t;
        if (u_all) memcpy(u_all + (long)(step + 2) * N, u, sizeof(double) * N);
    }
    if (nrec > 0 && rec_d) rec_finish(&rm, corners, nt, rec_d);
    if (u_last) {
        memcpy(u_last, u, sizeof(double) * N);
        memcpy(u_last + N, um, sizeof(double) * N);
    }
    free(um);
    free(u);
    free(up);
    free(corners);
    srcmap_free(&sm);
    recmap_free(&rm);
    return 0;
}

/* The Laplace (heat) operator of Sec. 5.7, explicit Euler in time:
 *   u^{n+1} = u^n + dt kappa (L u^n + f^n)
 * with the same Laplacian, zero halo, source spread and receiver recording
 * (receivers read u^{n+1}) as oracle_forward.  kappa may be NULL (1). */
int oracle_heat(const int *n, const double *h, double dt, int nt, int r, const double *c,
                const double *kappa, const double *u0,
                int nsrc, const double *src_xyz, const double *src_q,
                int nrec, const double *rec_xyz, double *rec_d, double *u_last)
{
    long N = npts(n);
    srcmap_t sm;
    recmap_t rm;
    if (srcmap_build(&sm, n, h, nsrc, src_xyz) || recmap_build(&rm, n, h, nrec, rec_xyz)) return -1;
    double *u = (double *)calloc(N, sizeof(double));
    double *up = (double *)calloc(N, sizeof(double));
    double *corners = (double *)calloc((size_t)nt * 8 * (nrec > 0 ? nrec : 1), sizeof(double));
    if (!u || !up || !corners) return -1;
    if (u0) memcpy(u, u0, sizeof(double) * N);
    for (int step = 0; step < nt; step++) {
#pragma omp parallel for schedule(static)
        for (long x = 0; x < n[0]; x++)
            for (long y = 0; y < n[1]; y++)
                for (long z = 0; z < n[2]; z++) {
                    long p = at(n, x, y, z);
                    double lap = lap_at(n, h, r, c, 0, u, x, y, z);
                    double f = src_term(&sm, src_q, step, p);
                    double k = kappa ? kappa[p] : 1.0;
                    up[p] = u[p] + dt * k * (lap + f);
                    rec_record(&rm, corners, step, p, up[p]);
                }
        double *t = u;
        u = up;
        up = t;
    }
    if (nrec > 0 && rec_d) rec_finish(&rm, corners, nt, rec_d);
    if (u_last) memcpy(u_last, u, sizeof(double) * N);
    free(u);
    free(up);
    free(corners);
    srcmap_free(&sm);
    recmap_free(&rm);
    return 0;
}

static long lmax(long a, long b) { return a > b ? a : b; }
static long lmin(long a, long b) { return a < b ? a : b; }

/* The paper's time-tiled loop nest for the same forward problem (zero halo).
 * Time is tiled by tt, x and y are skewed by the stencil radius r per time
 * step (the minimum legal factor, Sec. 2.3.2.1) and tiled by bx, by; z stays
 * the innermost, untiled loop.  Each time tile uses local time tl = t - t_blk
 * for the skew; min/max bounds keep every access inside the grid.  Tile loops
 * run sequentially; the incremental x loop is parallel (Sec. 4.2.3).
 * Levels live in a buffer of tt+2 slots: level L is in slot (L+1) mod (tt+2). */
int oracle_forward_tiled(const int *n, const double *h, double dt, int nt, int r, const double *c,
                         const double *m, const double *damp,
                         int nsrc, const double *src_xyz, const double *src_q,
                         int nrec, const double *rec_xyz, double *rec_d,
                         int tt, int bx, int by, double *u_last)
{
    long N = npts(n);
    if (tt < 1 || bx < 1 || by < 1) return -2;
    srcmap_t sm;
    recmap_t rm;
    if (srcmap_build(&sm, n, h, nsrc, src_xyz) || recmap_build(&rm, n, h, nrec, rec_xyz)) return -1;
    const int K = tt + 2;
    double *buf = (double *)calloc((size_t)K * N, sizeof(double));
    double *corners = (double *)calloc((size_t)nt * 8 * (nrec > 0 ? nrec : 1), sizeof(double));
    if (!buf || !corners) return -1;
    const long sk = r; /* skew factor */
    for (long t_blk = 0; t_blk < nt; t_blk += tt) {
        long t_end = lmin(nt, t_blk + tt);
        long xext = n[0] + sk * (t_end - t_blk - 1); /* skewed x extent of this time tile */
        long yext = n[1] + sk * (t_end - t_blk - 1);
        for (long x_blk = 0; x_blk < xext; x_blk += bx)
            for (long y_blk = 0; y_blk < yext; y_blk += by)
                for (long t = t_blk; t < t_end; t++) {
                    long tl = t - t_blk;
                    long xlo = lmax(sk * tl, x_blk), xhi = lmin(n[0] + sk * tl, x_blk + bx);
                    long ylo = lmax(sk * tl, y_blk), yhi = lmin(n[1] + sk * tl, y_blk + by);
                    const double *u = buf + ((t + 1) % K) * N;     /* level t   */
                    const double *um = buf + ((t + K) % K) * N;    /* level t-1 */
                    double *up = buf + ((t + 2) % K) * N;          /* level t+1 */
#pragma omp parallel for schedule(static)
                    for (long xs = xlo; xs < xhi; xs++)
                        for (long ys = ylo; ys < yhi; ys++)
                            for (long z = 0; z < n[2]; z++) {
                                long x = xs - sk * tl, y = ys - sk * tl;
                                long p = at(n, x, y, z);
                                double lap = lap_at(n, h, r, c, 0, u, x, y, z);
                                double f = src_term(&sm, src_q, (int)t, p);
                                up[p] = update_point(m[p], damp[p], dt, u[p], um[p], lap, f);
                                rec_record(&rm, corners, (int)t, p, up[p]);
                            }
                }
    }
    if (nrec > 0 && rec_d) rec_finish(&rm, corners, nt, rec_d);
    if (u_last) {
        memcpy(u_last, buf + ((long)(nt + 1) % K) * N, sizeof(double) * N);
        memcpy(u_last + N, buf + ((long)nt % K) * N, sizeof(double) * N);
    }
    free(buf);
    free(corners);
    srcmap_free(&sm);
    recmap_free(&rm);
    return 0;
}

/* Transposed recursion.  With J = sum_n <res^n, d^n> (res = dJ/dd for any
 * misfit), lambda^k = dJ/du^k satisfies, for k = nt..1,
 *   lambda^k = R^T res^{k-1} + 2 m alpha lambda^{k+1} + dt^2 L(alpha lambda^{k+1})
 *              - (m - eta) alpha lambda^{k+2},           lambda^{nt+1} = lambda^{nt+2} = 0,
 * since u^{k+1} = alpha (2 m u^k + dt^2 L u^k - (m - eta) u^{k-1} + ...) and L is
 * symmetric.  If lam_all != NULL it receives lambda^1..lambda^nt as [nt][N]
 * (index k-1).  src_grad [nt][nsrc] = dJ/dq_s^n = dt^2 sum_p w_{s,p} alpha_p lambda^{n+1}_p.
 * lam_last [2][N] = lambda^1, lambda^2. */
static int adjoint_core(const int *n, const double *h, double dt, int nt, int r, const double *c,
                        const double *m, const double *damp,
                        int nrec, const double *rec_xyz, const double *res,
                        double *lam_all, double *lam_last,
                        int nsrc, const double *src_xyz, double *src_grad)
{
    long N = npts(n);
    recmap_t rm;
    if (recmap_build(&rm, n, h, nrec, rec_xyz)) return -1;
    double *l1 = (double *)calloc(N, sizeof(double)); /* lambda^{k+1} */
    double *l2 = (double *)calloc(N, sizeof(double)); /* lambda^{k+2} */
    double *lk = (double *)calloc(N, sizeof(double)); /* lambda^k */
    double *al = (double *)calloc(N, sizeof(double)); /* alpha * lambda^{k+1} */
    double *lap = (double *)calloc(N, sizeof(double));
    double *alpha = (double *)calloc(N, sizeof(double));
    if (!l1 || !l2 || !lk || !al || !lap || !alpha) return -1;
    for (long p = 0; p < N; p++) alpha[p] = 1.0 / (m[p] + damp[p] * dt / 2.0);
    long *spts = NULL;
    double *swts = NULL;
    if (nsrc > 0) {
        spts = (long *)malloc(sizeof(long) * 8 * nsrc);
        swts = (double *)malloc(sizeof(double) * 8 * nsrc);
        for (int s = 0; s < nsrc; s++) trilinear(n, h, src_xyz + 3 * s, spts + 8 * s, swts + 8 * s);
    }
    for (int k = nt; k >= 1; k--) {
        for (long p = 0; p < N; p++) al[p] = alpha[p] * l1[p];
        oracle_laplacian(n, h, r, c, 0, al, lap);
        for (long p = 0; p < N; p++) {
            double eta = damp[p] * dt / 2.0;
            lk[p] = 2.0 * m[p] * alpha[p] * l1[p] + dt * dt * lap[p] - (m[p] - eta) * alpha[p] * l2[p];
        }
        /* R^T res^{k-1}: receivers read u^k at step k-1 */
        for (int rr = 0; rr < nrec; rr++)
            for (int cc = 0; cc < 8; cc++)
                lk[rm.corner[8 * rr + cc]] += rm.w[8 * rr + cc] * res[(long)(k - 1) * nrec + rr];
        if (lam_all) memcpy(lam_all + (long)(k - 1) * N, lk, sizeof(double) * N);
        /* dJ/dq^{k-1}: u^k holds alpha dt^2 f^{k-1} */
        for (int s = 0; s < nsrc; s++) {
            double acc = 0.0;
            for (int cc = 0; cc < 8; cc++) {
                long p = spts[8 * s + cc];
                acc = acc + swts[8 * s + cc] * alpha[p] * lk[p];
            }
            if (src_grad) src_grad[(long)(k - 1) * nsrc + s] = dt * dt * acc;
        }
        double *t = l2;
        l2 = l1;
        l1 = lk;
        lk = t;
    }
    if (lam_last) {
        memcpy(lam_last, l1, sizeof(double) * N);     /* lambda^1 */
        memcpy(lam_last + N, l2, sizeof(double) * N); /* lambda^2 */
    }
    free(l1);
    free(l2);
    free(lk);
    free(al);
    free(lap);
    free(alpha);
    free(spts);
    free(swts);
    recmap_free(&rm);
    return 0;
}

int oracle_adjoint(const int *n, const double *h, double dt, int nt, int r, const double *c,
                   const double *m, const double *damp,
                   int nrec, const double *rec_xyz, const double *res,
                   int nsrc, const double *src_xyz, double *src_grad,
                   double *lam_last)
{
    return adjoint_core(n, h, dt, nt, r, c, m, damp, nrec, rec_xyz, res, NULL, lam_last,
                        nsrc, src_xyz, src_grad);
}

/* dJ/dm for J = sum_n <res^n, d^n> with res fixed:
 *   g = - sum_{n=0}^{nt-1} lambda^{n+1} alpha (u^{n+1} - 2 u^n + u^{n-1}),
 * because d(alpha N)/dm = -alpha (alpha N - 2 u^n + u^{n-1}) for
 * N = 2 m u^n - (m - eta) u^{n-1} + dt^2 (L u^n + f^n).
 * Plain: stores every forward level and every adjoint level (small grids). */
int oracle_gradient(const int *n, const double *h, double dt, int nt, int r, const double *c,
                    const double *m, const double *damp,
                    int nsrc, const double *src_xyz, const double *src_q,
                    int nrec, const double *rec_xyz, const double *res,
                    double *grad)
{
    long N = npts(n);
    double *u_all = (double *)malloc(sizeof(double) * (size_t)(nt + 2) * N);
    double *lam_all = (double *)malloc(sizeof(double) * (size_t)nt * N);
    if (!u_all || !lam_all) return -1;
    int rc = oracle_forward(n, h, dt, nt, r, c, m, damp, nsrc, src_xyz, src_q, 0, NULL, NULL,
                            0, NULL, NULL, NULL, u_all);
    if (rc) return rc;
    rc = adjoint_core(n, h, dt, nt, r, c, m, damp, nrec, rec_xyz, res, lam_all, NULL, 0, NULL, NULL);
    if (rc) return rc;
    for (long p = 0; p < N; p++) {
        double alpha = 1.0 / (m[p] + damp[p] * dt / 2.0);
        double g = 0.0;
        for (int s = 0; s < nt; s++) {
            /* u_all index j holds u^{j-1}: u^{s+1} at s+2, u^s at s+1, u^{s-1} at s */
            double d2 = u_all[(long)(s + 2) * N + p] - 2.0 * u_all[(long)(s + 1) * N + p]
                        + u_all[(long)s * N + p];
            g = g - lam_all[(long)s * N + p] * alpha * d2;
        }
        grad[p] = g;
    }
    free(u_all);
    free(lam_all);
    return 0;
}

/* Born (linearised) modelling: the derivative of the forward map m -> d in
 * the direction dm (not in the paper; the textbook linearisation of the
 * scheme above).  With N = 2 m u^n - (m - eta) u^{n-1} + dt^2 (L u^n + f^n),
 * u^{n+1} = alpha N and d alpha / dm = -alpha^2, d N / dm = 2 u^n - u^{n-1}:
 *   du^{n+1} = alpha (2 m du^n - (m - eta) du^{n-1} + dt^2 L du^n)
 *              - alpha dm (u^{n+1} - 2 u^n + u^{n-1}),
 *   du^0 = du^-1 = 0,   dd^n[r] = sum_p w_{r,p} du^{n+1}[p].
 * Each step advances u over the whole grid first, then du. */
int oracle_born(const int *n, const double *h, double dt, int nt, int r, const double *c,
                const double *m, const double *damp, const double *dm,
                int nsrc, const double *src_xyz, const double *src_q,
                int nrec, const double *rec_xyz, double *rec_dd, double *du_last)
{
    long N = npts(n);
    srcmap_t sm;
    recmap_t rm;
    if (srcmap_build(&sm, n, h, nsrc, src_xyz) || recmap_build(&rm, n, h, nrec, rec_xyz)) return -1;
    double *um = (double *)calloc(N, sizeof(double));
    double *u = (double *)calloc(N, sizeof(double));
    double *up = (double *)calloc(N, sizeof(double));
    double *vm = (double *)calloc(N, sizeof(double));
    double *v = (double *)calloc(N, sizeof(double));
    double *vp = (double *)calloc(N, sizeof(double));
    double *corners = (double *)calloc((size_t)nt * 8 * (nrec > 0 ? nrec : 1), sizeof(double));
    if (!um || !u || !up || !vm || !v || !vp || !corners) return -1;
    for (int step = 0; step < nt; step++) {
#pragma omp parallel for schedule(static)
        for (long x = 0; x < n[0]; x++)
            for (long y = 0; y < n[1]; y++)
                for (long z = 0; z < n[2]; z++) {
                    long p = at(n, x, y, z);
                    double lap = lap_at(n, h, r, c, 0, u, x, y, z);
                    double f = src_term(&sm, src_q, step, p);
                    up[p] = update_point(m[p], damp[p], dt, u[p], um[p], lap, f);
                }
#pragma omp parallel for schedule(static)
        for (long x = 0; x < n[0]; x++)
            for (long y = 0; y < n[1]; y++)
                for (long z = 0; z < n[2]; z++) {
                    long p = at(n, x, y, z);
                    double eta = damp[p] * dt / 2.0;
                    double alpha = 1.0 / (m[p] + eta);
                    double lap = lap_at(n, h, r, c, 0, v, x, y, z);
                    double d2 = up[p] - 2.0 * u[p] + um[p];
                    vp[p] = alpha * (2.0 * m[p] * v[p] - (m[p] - eta) * vm[p] + dt * dt * lap)
                            - alpha * dm[p] * d2;
                    rec_record(&rm, corners, step, p, vp[p]);
                }
        double *t = um;
        um = u;
        u = up;
        up = t;
        t = vm;
        vm = v;
        v = vp;
        vp = t;
    }
    if (nrec > 0 && rec_dd) rec_finish(&rm, corners, nt, rec_dd);
    if (du_last) {
        memcpy(du_last, v, sizeof(double) * N);
        memcpy(du_last + N, vm, sizeof(double) * N);
    }
    free(um);
    free(u);
    free(up);
    free(vm);
    free(v);
    free(vp);
    free(corners);
    srcmap_free(&sm);
    recmap_free(&rm);
    return 0;
}

/* A multi-step (time dependence 2) form of the Laplace operator: the
 * two-step Adams-Bashforth scheme for u_t = kappa (lap u + f), the kind of
 * multi-step linear method the paper names for stencils with a larger time
 * dependence (Sec. 6, "Time-tiling with larger time dependences"):
 *   F^n     = L u^n + f^n,
 *   u^{n+1} = u^n + dt kappa (3/2 F^n - 1/2 F^{n-1}),   n >= 1,
 *   u^1     = u^0 + dt kappa F^0                          (Euler start),
 * receivers reading u^{n+1} as oracle_heat.  kappa may be NULL (1). */
int oracle_heat_ab2(const int *n, const double *h, double dt, int nt, int r, const double *c,
                    const double *kappa, const double *u0,
                    int nsrc, const double *src_xyz, const double *src_q,
                    int nrec, const double *rec_xyz, double *rec_d, double *u_last)
{
    long N = npts(n);
    srcmap_t sm;
    recmap_t rm;
    if (srcmap_build(&sm, n, h, nsrc, src_xyz) || recmap_build(&rm, n, h, nrec, rec_xyz)) return -1;
    double *u = (double *)calloc(N, sizeof(double));
    double *up = (double *)calloc(N, sizeof(double));
    double *F = (double *)calloc(N, sizeof(double));
    double *Fm = (double *)calloc(N, sizeof(double));
    double *corners = (double *)calloc((size_t)nt * 8 * (nrec > 0 ? nrec : 1), sizeof(double));
    if (!u || !up || !F || !Fm || !corners) return -1;
    if (u0) memcpy(u, u0, sizeof(double) * N);
    for (int step = 0; step < nt; step++) {
#pragma omp parallel for schedule(static)
        for (long x = 0; x < n[0]; x++)
            for (long y = 0; y < n[1]; y++)
                for (long z = 0; z < n[2]; z++) {
                    long p = at(n, x, y, z);
                    F[p] = lap_at(n, h, r, c, 0, u, x, y, z) + src_term(&sm, src_q, step, p);
                }
#pragma omp parallel for schedule(static)
        for (long p = 0; p < N; p++) {
            double k = kappa ? kappa[p] : 1.0;
            double rate = step == 0 ? F[p] : 1.5 * F[p] - 0.5 * Fm[p];
            up[p] = u[p] + dt * k * rate;
        }
        for (long x = 0; x < n[0]; x++)
            for (long y = 0; y < n[1]; y++)
                for (long z = 0; z < n[2]; z++) {
                    long p = at(n, x, y, z);
                    rec_record(&rm, corners, step, p, up[p]);
                }
        double *t = u;
        u = up;
        up = t;
        t = Fm;
        Fm = F;
        F = t;
    }
    if (nrec > 0 && rec_d) rec_finish(&rm, corners, nt, rec_d);
    if (u_last) memcpy(u_last, u, sizeof(double) * N);
    free(u);
    free(up);
    free(F);
    free(Fm);
    free(corners);
    srcmap_free(&sm);
    recmap_free(&rm);
    return 0;
}
