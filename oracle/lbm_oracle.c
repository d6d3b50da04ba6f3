/*
 * lbm_oracle.c -- plain, slow, FP64 CPU oracle for the lattice-BGK step with the
 * entropic equilibrium of Hosseini & Karlin, "Entropic equilibrium for the lattice
 * Boltzmann method: Hydrodynamics and numerical properties" (arXiv 2303.08163).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or calls
 * this file; only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark do.  It shares no source with the CUDA path.
 *
 * What it computes, in the paper's order and notation (lattice units dr = dt = 1):
 *   - Sec. II: D1Q3 velocities c in {-1,0,1}, weights {1/6, 2/3, 1/6}; D2Q9 / D3Q27
 *     as tensor products.
 *   - Eq. (eq:Entropic_isothermal_EDF): f_i^eq = w_i rho prod_a (2 - S_a) Z_a^{c_ia},
 *     S_a = sqrt((u_a/vs)^2 + 1), Z_a = (2 u_a + S_a) / (1 - u_a); Z^-1 is taken as 1/Z
 *     (literal form, with the divisions).
 *   - Eq. (eq:Poly2_isothermal_EDF): the quadratic polynomial equilibrium.
 *   - Eq. (eq:Product_isothermal_EDF): the product-form equilibrium.
 *   - Eq. (eq:relaxation_frequency): beta = dt / (2 nu / vs^2 + dt), 2 beta = 1/tau.
 *   - Eqs. (eq:entropic_bulk), (eq:LBGK_bulk): the bulk coefficient A; Eqs.
 *     (eq:redefined_relaxation rate) and (_poly): the locally corrected beta.  In 2-D
 *     and 3-D the per-cell A is min over axes of A(u_a) (the paper derives A in 1-D
 *     only; this reading reduces to the paper's case for flow along one axis).
 *   - Eq. (1): f_i(r + c_i, t + 1) - f_i(r, t) = 2 beta (f_i^eq - f_i): collide, then
 *     stream, periodic, on two arrays.
 *
 * Population index convention (shared as an interface convention only):
 *   i = (c_x + 1) + 3 (c_y + 1) + 9 (c_z + 1); opposite(i) = Q - 1 - i.
 * Cell index: x fastest, idx = x + Nx (y + Ny z).  Arrays are SoA: f[i * ncell + idx].
 *
 * Built with -O2 -ffp-contract=off and IEEE sqrt / division.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_EQ_ENTROPIC 0
#define OR_EQ_POLY2 1
#define OR_EQ_PRODUCT 2

typedef struct {
    int D, Q;
    int c[27][3];
    double w[27];
} or_lattice;

/* Sec. II: first-neighbour D1Q3 lattice and its tensor products. */
static void or_make_lattice(int D, or_lattice *L)
{
    static const double w1[3] = {1.0 / 6.0, 2.0 / 3.0, 1.0 / 6.0}; /* for c = -1, 0, 1 */
    int Q = 1, i, a;
    for (a = 0; a < D; ++a) Q *= 3;
    L->D = D;
    L->Q = Q;
    for (i = 0; i < Q; ++i) {
        int rem = i;
        L->w[i] = 1.0;
        for (a = 0; a < 3; ++a) {
            if (a < D) {
                int digit = rem % 3;
                rem /= 3;
                L->c[i][a] = digit - 1;
                L->w[i] *= w1[digit];
            } else {
                L->c[i][a] = 0;
            }
        }
    }
}

int oracle_lattice(int D, int *c_out /* [Q][3] */, double *w_out /* [Q] */)
{
    or_lattice L;
    int i;
    if (D < 1 || D > 3) return -1;
    or_make_lattice(D, &L);
    for (i = 0; i < L.Q; ++i) {
        c_out[3 * i + 0] = L.c[i][0];
        c_out[3 * i + 1] = L.c[i][1];
        c_out[3 * i + 2] = L.c[i][2];
        w_out[i] = L.w[i];
    }
    return L.Q;
}

/* Lattice sound speed vs = dr / (sqrt(3) dt), Sec. II. */
static double or_vs(void) { return 1.0 / sqrt(3.0); }

/* Eq. (eq:Entropic_isothermal_EDF), literal: Z_a and X^-1 from their closed forms. */
static void or_feq_entropic(const or_lattice *L, double rho, const double *u, double *feq)
{
    double vs = or_vs();
    double Z[3], Zinv[3], Xinv = rho;
    int a, i;
    for (a = 0; a < L->D; ++a) {
        double x = u[a] / vs;
        double S = sqrt(x * x + 1.0);
        Z[a] = (2.0 * u[a] + S) / (1.0 - u[a]);
        Zinv[a] = 1.0 / Z[a];
        Xinv *= (2.0 - S);
    }
    for (i = 0; i < L->Q; ++i) {
        double p = 1.0;
        for (a = 0; a < L->D; ++a) {
            if (L->c[i][a] == 1) p *= Z[a];
            else if (L->c[i][a] == -1) p *= Zinv[a];
        }
        feq[i] = L->w[i] * Xinv * p;
    }
}

/* Eq. (eq:Poly2_isothermal_EDF). */
static void or_feq_poly2(const or_lattice *L, double rho, const double *u, double *feq)
{
    double vs = or_vs();
    double vs2 = vs * vs;
    double uu = 0.0;
    int a, i;
    for (a = 0; a < L->D; ++a) uu += u[a] * u[a];
    for (i = 0; i < L->Q; ++i) {
        double cu = 0.0;
        for (a = 0; a < L->D; ++a) cu += L->c[i][a] * u[a];
        feq[i] = L->w[i] * rho *
                 (1.0 + cu / vs2 + (cu * cu) / (2.0 * vs2 * vs2) - uu / (2.0 * vs2));
    }
}

/* Eq. (eq:Product_isothermal_EDF). */
static void or_feq_product(const or_lattice *L, double rho, const double *u, double *feq)
{
    double vs = or_vs();
    double vs2 = vs * vs;
    int a, i;
    for (i = 0; i < L->Q; ++i) {
        double p = rho;
        for (a = 0; a < L->D; ++a) {
            int c = L->c[i][a];
            if (c == 0) p *= (1.0 - vs2 - u[a] * u[a]);
            else p *= (c * u[a] + vs2 + u[a] * u[a]) / 2.0;
        }
        feq[i] = p;
    }
}

static int or_feq(const or_lattice *L, int eq_kind, double rho, const double *u, double *feq)
{
    switch (eq_kind) {
    case OR_EQ_ENTROPIC: or_feq_entropic(L, rho, u, feq); return 0;
    case OR_EQ_POLY2: or_feq_poly2(L, rho, u, feq); return 0;
    case OR_EQ_PRODUCT: or_feq_product(L, rho, u, feq); return 0;
    default: return -1;
    }
}

int oracle_feq(int D, int eq_kind, double rho, const double *u, double *feq)
{
    or_lattice L;
    double uu[3] = {0.0, 0.0, 0.0};
    int a;
    if (D < 1 || D > 3) return -1;
    or_make_lattice(D, &L);
    for (a = 0; a < D; ++a) uu[a] = u[a];
    return or_feq(&L, eq_kind, rho, uu, feq);
}

/*
 * Bulk coefficient A of one axis.
 * Entropic: Eq. (eq:entropic_bulk), with x = u / vs:
 *   A = 1 - (3/2) u^2 / vs^2 + (x^2 + 3 x^4 - 2 sqrt(x^2 + 1) + 2) / (2 x^2 + 2).
 * Polynomial and product form: Eq. (eq:LBGK_bulk), A = 1 - (3/2) u^2 / vs^2.
 */
double oracle_bulk_A(int eq_kind, double u)
{
    double vs = or_vs();
    double vs2 = vs * vs;
    if (eq_kind == OR_EQ_ENTROPIC) {
        double x = u / vs;
        double x2 = x * x;
        return 1.0 - 1.5 * u * u / vs2 +
               (x2 + 3.0 * x2 * x2 - 2.0 * sqrt(x2 + 1.0) + 2.0) / (2.0 * x2 + 2.0);
    }
    return 1.0 - 1.5 * u * u / vs2;
}

/*
 * Collision frequency 2 beta for one cell.
 * bulk_corr = 0: Eq. (eq:relaxation_frequency) with nu = vs^2 (tau - 1/2), i.e. 1/tau.
 * bulk_corr = 1: Eq. (eq:redefined_relaxation rate), beta = 1 / (2 nu / (A vs^2) + 1),
 *                A = min_a A(u_a).
 */
double oracle_omega(int D, int eq_kind, int bulk_corr, double tau, const double *u)
{
    double vs = or_vs();
    double vs2 = vs * vs;
    double nu = vs2 * (tau - 0.5);
    double beta;
    if (!bulk_corr) {
        beta = 1.0 / (2.0 * nu / vs2 + 1.0);
    } else {
        double A = oracle_bulk_A(eq_kind, u[0]);
        int a;
        for (a = 1; a < D; ++a) {
            double Aa = oracle_bulk_A(eq_kind, u[a]);
            if (Aa < A) A = Aa;
        }
        beta = 1.0 / (2.0 * nu / (A * vs2) + 1.0);
    }
    return 2.0 * beta;
}

static void or_moments_cell(const or_lattice *L, const double *f, int64_t ncell, int64_t idx,
                            double *rho, double *u)
{
    double r = 0.0, j[3] = {0.0, 0.0, 0.0};
    int i, a;
    for (i = 0; i < L->Q; ++i) {
        double fi = f[(int64_t)i * ncell + idx];
        r += fi;
        for (a = 0; a < L->D; ++a) j[a] += L->c[i][a] * fi;
    }
    *rho = r;
    for (a = 0; a < 3; ++a) u[a] = (a < L->D) ? j[a] / r : 0.0;
}

static int64_t or_wrap(int64_t v, int64_t n)
{
    v %= n;
    return v < 0 ? v + n : v;
}

/* f = f^eq(rho, u) for every cell (the initial state; the paper is silent on it). */
int oracle_init(int D, const int64_t *dims, int eq_kind, const double *rho, const double *u,
                double *f)
{
    or_lattice L;
    int64_t ncell = dims[0] * dims[1] * dims[2], idx;
    double feq[27];
    int i, a;
    if (D < 1 || D > 3) return -1;
    or_make_lattice(D, &L);
    for (idx = 0; idx < ncell; ++idx) {
        double uc[3] = {0.0, 0.0, 0.0};
        for (a = 0; a < D; ++a) uc[a] = u[(int64_t)a * ncell + idx];
        if (or_feq(&L, eq_kind, rho[idx], uc, feq)) return -1;
        for (i = 0; i < L.Q; ++i) f[(int64_t)i * ncell + idx] = feq[i];
    }
    return 0;
}

/*
 * Host threads of oracle_step (1 by default).  The cells of one step are independent:
 * each reads the state f and writes its post-collision values to distinct slots of g,
 * so the rows of the lattice are shared out between threads without changing any
 * cell's arithmetic; the result is the same bit for bit for every thread count.  Builds
 * without OpenMP run one thread whatever is asked.
 */
static int or_threads = 1;

int oracle_set_threads(int n)
{
    or_threads = n < 1 ? 1 : n;
#ifdef _OPENMP
    return or_threads;
#else
    return 1;
#endif
}

/*
 * n time steps of Eq. (1) on two arrays: for each cell compute rho and u from the
 * populations, the equilibrium, the collision frequency, the post-collision value
 * f_i + 2 beta (f_i^eq - f_i), and write it to cell r + c_i (periodic).  f holds the
 * state on entry and on exit; g is a work array of the same size.
 */
int oracle_step(int D, const int64_t *dims, int eq_kind, int bulk_corr, double tau, int64_t n,
                double *f, double *g)
{
    or_lattice L;
    int64_t nx = dims[0], ny = dims[1], nz = dims[2];
    int64_t ncell = nx * ny * nz, nrow = ny * nz, s;
    if (D < 1 || D > 3) return -1;
    if (eq_kind != OR_EQ_ENTROPIC && eq_kind != OR_EQ_POLY2 && eq_kind != OR_EQ_PRODUCT) return -1;
    or_make_lattice(D, &L);
    for (s = 0; s < n; ++s) {
        int64_t row;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(or_threads)
#endif
        for (row = 0; row < nrow; ++row) {
            int64_t y = row % ny, z = row / ny, x;
            double feq[27];
            for (x = 0; x < nx; ++x) {
                int64_t idx = x + nx * (y + ny * z);
                double rho, u[3], om;
                int i;
                or_moments_cell(&L, f, ncell, idx, &rho, u);
                or_feq(&L, eq_kind, rho, u, feq);
                om = oracle_omega(D, eq_kind, bulk_corr, tau, u);
                for (i = 0; i < L.Q; ++i) {
                    double fi = f[(int64_t)i * ncell + idx];
                    double post = fi + om * (feq[i] - fi);
                    int64_t xd = or_wrap(x + L.c[i][0], nx);
                    int64_t yd = or_wrap(y + L.c[i][1], ny);
                    int64_t zd = or_wrap(z + L.c[i][2], nz);
                    g[(int64_t)i * ncell + xd + nx * (yd + ny * zd)] = post;
                }
            }
        }
        memcpy(f, g, sizeof(double) * (size_t)(ncell * L.Q));
    }
    return 0;
}

/* rho and u (SoA, u[a * ncell + idx]) of every cell. */
int oracle_moments(int D, const int64_t *dims, const double *f, double *rho, double *u)
{
    or_lattice L;
    int64_t ncell = dims[0] * dims[1] * dims[2], idx;
    int a;
    if (D < 1 || D > 3) return -1;
    or_make_lattice(D, &L);
    for (idx = 0; idx < ncell; ++idx) {
        double r, uc[3];
        or_moments_cell(&L, f, ncell, idx, &r, uc);
        rho[idx] = r;
        for (a = 0; a < D; ++a) u[(int64_t)a * ncell + idx] = uc[a];
    }
    return 0;
}

static void or_kahan_add(double *sum, double *comp, double v)
{
    double y = v - *comp;
    double t = *sum + y;
    *comp = (t - *sum) - y;
    *sum = t;
}

/*
 * Global diagnostics with compensated summation:
 * out[0] = sum rho, out[1..3] = sum rho u_a, out[4] = sum rho |u|^2 / 2, out[5] = max |u_a|.
 */
int oracle_diagnostics(int D, const int64_t *dims, const double *f, double *out)
{
    or_lattice L;
    int64_t ncell = dims[0] * dims[1] * dims[2], idx;
    double s[5] = {0, 0, 0, 0, 0}, c[5] = {0, 0, 0, 0, 0}, umax = 0.0;
    int a;
    if (D < 1 || D > 3) return -1;
    or_make_lattice(D, &L);
    for (idx = 0; idx < ncell; ++idx) {
        double r, u[3], e = 0.0;
        or_moments_cell(&L, f, ncell, idx, &r, u);
        or_kahan_add(&s[0], &c[0], r);
        for (a = 0; a < 3; ++a) {
            or_kahan_add(&s[1 + a], &c[1 + a], r * u[a]);
            e += u[a] * u[a];
            if (fabs(u[a]) > umax) umax = fabs(u[a]);
        }
        or_kahan_add(&s[4], &c[4], 0.5 * r * e);
    }
    for (a = 0; a < 5; ++a) out[a] = s[a];
    out[5] = umax;
    return 0;
}

/*
 * Fourier projection of rho and j = rho u on the wave vector k = 2 pi (n_x/N_x, n_y/N_y,
 * n_z/N_z): out = [Re, Im] of sum_r q(r) exp(-i k.r) for q = rho, j_x, j_y, j_z.
 */
int oracle_probe(int D, const int64_t *dims, const double *f, const int *kvec, double *out)
{
    or_lattice L;
    int64_t nx = dims[0], ny = dims[1], nz = dims[2];
    int64_t ncell = nx * ny * nz;
    int64_t x, y, z;
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const double twopi = 6.283185307179586476925286766559;
    int q;
    if (D < 1 || D > 3) return -1;
    or_make_lattice(D, &L);
    for (z = 0; z < nz; ++z)
        for (y = 0; y < ny; ++y)
            for (x = 0; x < nx; ++x) {
                int64_t idx = x + nx * (y + ny * z);
                double r, u[3], ph, cr, ci, val[4];
                or_moments_cell(&L, f, ncell, idx, &r, u);
                ph = twopi * ((double)(kvec[0] * x % nx) / (double)nx +
                              (double)(kvec[1] * y % ny) / (double)ny +
                              (double)(kvec[2] * z % nz) / (double)nz);
                cr = cos(ph);
                ci = -sin(ph);
                val[0] = r;
                val[1] = r * u[0];
                val[2] = r * u[1];
                val[3] = r * u[2];
                for (q = 0; q < 4; ++q) {
                    acc[2 * q] += val[q] * cr;
                    acc[2 * q + 1] += val[q] * ci;
                }
            }
    for (q = 0; q < 8; ++q) out[q] = acc[q];
    return 0;
}

/*
 * Run n steps, recording a probe sample (oracle_probe) of the state at t = 0, K, 2K, ...
 * while t < n.  probes_out holds ceil(n / K) samples of 8 doubles.  Used for the batched
 * linear-mode sweep, one instance at a time.
 */
int oracle_run_probed(int D, const int64_t *dims, int eq_kind, int bulk_corr, double tau,
                      int64_t n, int64_t every_k, const int *kvec, double *f, double *g,
                      double *probes_out)
{
    int64_t t, ns = 0;
    if (every_k < 1) return -1;
    for (t = 0; t < n; ++t) {
        if (t % every_k == 0) {
            if (oracle_probe(D, dims, f, kvec, probes_out + 8 * ns)) return -1;
            ++ns;
        }
        if (oracle_step(D, dims, eq_kind, bulk_corr, tau, 1, f, g)) return -1;
    }
    return 0;
}
