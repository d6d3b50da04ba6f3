// k_vn.cu -- von Neumann analysis of the D2Q9 scheme on the GPU (Sec. V.A of the paper):
// batched eigenvalues of the amplification matrix M = E (delta + J) (Eq. eq:VN_eigen) and
// the linear-stability limit of Sec. V.A.2, one parameter point per thread, in FP64.
//
// J is the Jacobian of the collision operator Omega_i = 2 beta (f_i^eq - f_i) at the
// equilibrium state f = f^eq(rho, u).  The derivative of a locally corrected 2 beta
// multiplies f^eq - f = 0 there, so J = 2 beta (d f^eq / d f - I) with
//   d f_i^eq / d f_j = d f_i^eq / d rho + sum_a d f_i^eq / d u_a (c_ja - u_a) / rho
// (rho = sum f, rho u = sum c f).  The partial derivatives of f^eq(rho, u) come from
// forward-mode dual numbers evaluated through the same equilibrium formulas as the step
// kernels, so they are exact to rounding.  E_ij = exp(-i c_i . k) delta_ij.
//
// Eigenvalues: reduction to upper Hessenberg form by complex Givens rotations, then
// single-shift QR with Wilkinson shifts and deflation (the standard complex Schur
// iteration), on a 9 x 9 matrix held by one thread.
#include <cmath>

#include "lbm.h"
#include "lbm_device.cuh"
#include "lbm_internal.h"

namespace lbmd {

// ------------------------------------------------------------------------- dual numbers

struct Dual {  // value and derivatives with respect to (rho, u_x, u_y)
    double v, d[3];
};
__host__ __device__ __forceinline__ Dual dconst(double c) { return {c, {0, 0, 0}}; }
__host__ __device__ __forceinline__ Dual operator+(Dual a, Dual b) {
    return {a.v + b.v, {a.d[0] + b.d[0], a.d[1] + b.d[1], a.d[2] + b.d[2]}};
}
__host__ __device__ __forceinline__ Dual operator-(Dual a, Dual b) {
    return {a.v - b.v, {a.d[0] - b.d[0], a.d[1] - b.d[1], a.d[2] - b.d[2]}};
}
__host__ __device__ __forceinline__ Dual operator*(Dual a, Dual b) {
    return {a.v * b.v, {a.d[0] * b.v + a.v * b.d[0], a.d[1] * b.v + a.v * b.d[1], a.d[2] * b.v + a.v * b.d[2]}};
}
__host__ __device__ __forceinline__ Dual operator*(double c, Dual a) { return {c * a.v, {c * a.d[0], c * a.d[1], c * a.d[2]}}; }
__host__ __device__ __forceinline__ Dual dsqrt(Dual a) {
    const double s = sqrt(a.v), h = 0.5 / s;
    return {s, {h * a.d[0], h * a.d[1], h * a.d[2]}};
}

// f^eq_i(rho, u) of D2Q9 as dual numbers (same formulas as the step kernels' equilibria).
template <int EQ>
__host__ __device__ void feq_dual(Dual rho, Dual ux, Dual uy, Dual (&f)[9]) {
    if (EQ == EQ_POLY2) {
        const Dual uu = ux * ux + uy * uy;
        for (int i = 0; i < 9; ++i) {
            const Dual cu = (double)cxo(i) * ux + (double)cyo(i) * uy;
            const Dual p = dconst(1.0) + 3.0 * cu + 4.5 * (cu * cu) - 1.5 * uu;
            f[i] = wq<2>(i) * (rho * p);
        }
        return;
    }
    Dual tx[3], ty[3];  // per-axis factors t(c) = a(c) / w(c), indexed by c + 1
    const Dual u[2] = {ux, uy};
    for (int a = 0; a < 2; ++a) {
        Dual *t = a == 0 ? tx : ty;
        if (EQ == EQ_ENT) {
            const Dual S = dsqrt(dconst(1.0) + 3.0 * (u[a] * u[a]));
            t[1] = dconst(2.0) - S;
            t[2] = 2.0 * S - dconst(1.0) + 3.0 * u[a];
            t[0] = 2.0 * S - dconst(1.0) - 3.0 * u[a];
        } else {
            const Dual u2 = u[a] * u[a];
            t[1] = dconst(1.0) - 1.5 * u2;
            t[2] = dconst(1.0) + 3.0 * u[a] + 3.0 * u2;
            t[0] = dconst(1.0) - 3.0 * u[a] + 3.0 * u2;
        }
    }
    for (int i = 0; i < 9; ++i) f[i] = wq<2>(i) * (rho * (tx[cxo(i) + 1] * ty[cyo(i) + 1]));
}

// -------------------------------------------------------------------- complex helpers

struct cplx {
    double re, im;
};
__host__ __device__ __forceinline__ cplx cadd(cplx a, cplx b) { return {a.re + b.re, a.im + b.im}; }
__host__ __device__ __forceinline__ cplx csub(cplx a, cplx b) { return {a.re - b.re, a.im - b.im}; }
__host__ __device__ __forceinline__ cplx cmul(cplx a, cplx b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__host__ __device__ __forceinline__ cplx cconj(cplx a) { return {a.re, -a.im}; }
__host__ __device__ __forceinline__ cplx cscale(double s, cplx a) { return {s * a.re, s * a.im}; }
__host__ __device__ __forceinline__ double cabs2(cplx a) { return a.re * a.re + a.im * a.im; }
__host__ __device__ __forceinline__ double cabsd(cplx a) { return hypot(a.re, a.im); }
__host__ __device__ __forceinline__ cplx cdiv(cplx a, cplx b) {
    const double d = cabs2(b);
    return {(a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d};
}
__host__ __device__ __forceinline__ cplx csqrt_(cplx z) {
    const double r = cabsd(z);
    if (r == 0.0) return {0.0, 0.0};
    double x = sqrt(0.5 * (r + fabs(z.re)));
    double y = 0.5 * z.im / x;
    if (z.re >= 0.0) return {x, y};
    return {fabs(y), z.im >= 0.0 ? x : -x};
}

// Givens rotation G = [[c, s], [-conj(s), c]] (c real) with G [a; b] = [r; 0].
__host__ __device__ __forceinline__ void givens(cplx a, cplx b, double &c, cplx &s) {
    const double na = cabsd(a), nb = cabsd(b);
    if (nb == 0.0) {
        c = 1.0;
        s = {0.0, 0.0};
        return;
    }
    if (na == 0.0) {
        c = 0.0;
        s = {1.0, 0.0};
        return;
    }
    const double r = hypot(na, nb);
    c = na / r;
    s = cscale(1.0 / (na * r), cmul(a, cconj(b)));
}

constexpr int kN = 9;

// Rotate rows p, q of H (columns lo..hi) by G.
__host__ __device__ __forceinline__ void rot_rows(cplx (&H)[kN][kN], int p, int q, double c, cplx s, int lo, int hi) {
    for (int j = lo; j <= hi; ++j) {
        const cplx x = H[p][j], y = H[q][j];
        H[p][j] = cadd(cscale(c, x), cmul(s, y));
        H[q][j] = csub(cscale(c, y), cmul(cconj(s), x));
    }
}

// Multiply columns p, q of H (rows lo..hi) by G^H on the right.
__host__ __device__ __forceinline__ void rot_cols(cplx (&H)[kN][kN], int p, int q, double c, cplx s, int lo, int hi) {
    for (int j = lo; j <= hi; ++j) {
        const cplx x = H[j][p], y = H[j][q];
        H[j][p] = cadd(cscale(c, x), cmul(cconj(s), y));
        H[j][q] = csub(cscale(c, y), cmul(s, x));
    }
}

// Eigenvalues of H (overwritten).  Returns the number of QR iterations used, or -1 if
// the iteration limit was reached (eigenvalues then hold the last diagonal).
__host__ __device__ int eig_hessenberg_qr(cplx (&H)[kN][kN], cplx (&lam)[kN]) {
    // Hessenberg reduction
    for (int k = 0; k < kN - 2; ++k) {
        for (int i = kN - 1; i >= k + 2; --i) {
            double c;
            cplx s;
            givens(H[i - 1][k], H[i][k], c, s);
            rot_rows(H, i - 1, i, c, s, 0, kN - 1);
            rot_cols(H, i - 1, i, c, s, 0, kN - 1);
            H[i][k] = {0.0, 0.0};
        }
    }
    const double eps = 2.220446049250313e-16;
    int hi = kN - 1, iters = 0, since = 0;
    while (hi >= 0) {
        if (hi == 0) {
            lam[0] = H[0][0];
            break;
        }
        // deflation: smallest l with a negligible subdiagonal above the active block
        int l = hi;
        while (l > 0) {
            const double tol = eps * (cabsd(H[l - 1][l - 1]) + cabsd(H[l][l]));
            if (cabsd(H[l][l - 1]) <= tol) {
                H[l][l - 1] = {0.0, 0.0};
                break;
            }
            --l;
        }
        if (l == hi) {
            lam[hi] = H[hi][hi];
            --hi;
            since = 0;
            continue;
        }
        if (++iters > 60 * kN) return -1;
        ++since;
        // Wilkinson shift: eigenvalue of the trailing 2 x 2 block closest to H[hi][hi]
        const cplx a = H[hi - 1][hi - 1], b = H[hi - 1][hi], cc = H[hi][hi - 1], d = H[hi][hi];
        const cplx half = cscale(0.5, csub(a, d));
        const cplx disc = csqrt_(cadd(cmul(half, half), cmul(b, cc)));
        cplx mu1 = cadd(d, csub(half, disc)), mu2 = cadd(d, cadd(half, disc));
        cplx mu = cabs2(csub(mu1, d)) <= cabs2(csub(mu2, d)) ? mu1 : mu2;
        if (since % 11 == 10) mu = cadd(d, cscale(0.75, {cabsd(cc), 0.0}));  // exceptional shift
        // one QR step on the active block l..hi: H - mu I = Q R, H <- R Q + mu I
        for (int k = l; k <= hi; ++k) H[k][k] = csub(H[k][k], mu);
        double cs[kN];
        cplx sn[kN];
        for (int k = l; k < hi; ++k) {
            givens(H[k][k], H[k + 1][k], cs[k], sn[k]);
            rot_rows(H, k, k + 1, cs[k], sn[k], k, hi);
            H[k + 1][k] = {0.0, 0.0};
        }
        for (int k = l; k < hi; ++k) rot_cols(H, k, k + 1, cs[k], sn[k], l, k + 2 < hi ? k + 2 : hi);
        for (int k = l; k <= hi; ++k) H[k][k] = cadd(H[k][k], mu);
    }
    return iters;
}

// M = E (delta + J) of the D2Q9 scheme at (tau, rho, u) and wave vector k.
template <int EQ, bool BULK>
__host__ __device__ void vn_matrix(double tau, double rho, double ux, double uy, double kx, double ky,
                          cplx (&M)[kN][kN]) {
    Dual f[9];
    feq_dual<EQ>(Dual{rho, {1, 0, 0}}, Dual{ux, {0, 1, 0}}, Dual{uy, {0, 0, 1}}, f);
    double om = 1.0 / tau;
    if (BULK) {
        const double nu = (tau - 0.5) / 3.0;
        double A;
        if (EQ == EQ_ENT) {
            const double S = fmax(sqrt(1.0 + 3.0 * ux * ux), sqrt(1.0 + 3.0 * uy * uy));
            A = (2.0 - S) / (S * S);
        } else {
            A = 1.0 - 4.5 * fmax(ux * ux, uy * uy);
        }
        om = 2.0 * A / (6.0 * nu + A);
    }
    for (int i = 0; i < 9; ++i) {
        const double ph = -(cxo(i) * kx + cyo(i) * ky);
        double sp, cp;
        sincos(ph, &sp, &cp);
        for (int j = 0; j < 9; ++j) {
            const double dfdf = f[i].d[0] + f[i].d[1] * (cxo(j) - ux) / rho + f[i].d[2] * (cyo(j) - uy) / rho;
            const double a = (i == j ? 1.0 : 0.0) + om * (dfdf - (i == j ? 1.0 : 0.0));
            M[i][j] = {cp * a, sp * a};
        }
    }
}

template <int EQ, bool BULK>
__global__ void __launch_bounds__(128) k_vn_eigs(int64_t count, const double *params, double *out,
                                                 int32_t *status) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < count;
         p += (int64_t)gridDim.x * blockDim.x) {
        const double *q = params + 6 * p;
        cplx M[kN][kN], lam[kN];
        vn_matrix<EQ, BULK>(q[0], q[1], q[2], q[3], q[4], q[5], M);
        if (eig_hessenberg_qr(M, lam) < 0) atomicExch(status, 1);
        // sort by decreasing modulus (insertion sort)
        for (int a = 1; a < kN; ++a) {
            const cplx v = lam[a];
            const double m = cabs2(v);
            int b = a - 1;
            while (b >= 0 && cabs2(lam[b]) < m) {
                lam[b + 1] = lam[b];
                --b;
            }
            lam[b + 1] = v;
        }
        for (int a = 0; a < kN; ++a) {
            out[(p * kN + a) * 2] = lam[a].re;
            out[(p * kN + a) * 2 + 1] = lam[a].im;
        }
    }
}

// One bisection probe: for every (pair, k-point), the spectral radius of M at the pair's
// trial speed u_try along angle theta; the maximum over k-points is accumulated per pair
// with an integer atomicMax on the bit pattern (order-preserving for values >= 0).
template <int EQ>
__global__ void __launch_bounds__(128) k_vn_radius(int64_t npairs, const double *tau, const double *theta,
                                                   const double *u_try, int nk,
                                                   unsigned long long *radius_bits, int32_t *status) {
    const int64_t total = npairs * nk * nk;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t pr = t / ((int64_t)nk * nk);
        const int kk = (int)(t - pr * nk * nk);
        const int ix = kk % nk, iy = kk / nk;
        const double pi = 3.14159265358979323846;
        const double kx = nk > 1 ? pi * ix / (nk - 1) : 0.0, ky = nk > 1 ? pi * iy / (nk - 1) : 0.0;
        double st, ct;
        sincos(theta[pr], &st, &ct);
        const double u = u_try[pr];
        cplx M[kN][kN], lam[kN];
        vn_matrix<EQ, false>(tau[pr], 1.0, u * ct, u * st, kx, ky, M);
        if (eig_hessenberg_qr(M, lam) < 0) atomicExch(status, 1);
        double r = 0.0;
        for (int a = 0; a < kN; ++a) r = fmax(r, cabsd(lam[a]));
        if (!(r >= 0.0)) r = 1e300;  // NaN: treat as unstable
        atomicMax(radius_bits + pr, (unsigned long long)__double_as_longlong(r));
    }
}

}  // namespace lbmd

namespace lbmh {

using namespace lbmd;

static int grid_n(int64_t n, int threads) {
    int64_t g = (n + threads - 1) / threads;
    return (int)(g < 1 ? 1 : (g > 152 * 64 ? 152 * 64 : g));
}

cudaError_t vn_eigs(int eq, int bulk, int64_t count, const double *params, double *out, int32_t *status,
                    cudaStream_t s) {
    const int g = grid_n(count, 128);
#define LBM_VN(EQv)                                                                                  \
    if (eq == EQv) {                                                                                 \
        if (bulk) k_vn_eigs<EQv, true><<<g, 128, 0, s>>>(count, params, out, status);                \
        else k_vn_eigs<EQv, false><<<g, 128, 0, s>>>(count, params, out, status);                    \
        return cudaGetLastError();                                                                   \
    }
    LBM_VN(EQ_ENT)
    LBM_VN(EQ_POLY2)
    LBM_VN(EQ_PROD)
#undef LBM_VN
    return cudaErrorInvalidValue;
}

cudaError_t vn_radius(int eq, int64_t npairs, const double *tau, const double *theta, const double *u_try, int nk,
                      unsigned long long *radius_bits, int32_t *status, cudaStream_t s) {
    const int g = grid_n(npairs * nk * nk, 128);
    if (eq == EQ_ENT) k_vn_radius<EQ_ENT><<<g, 128, 0, s>>>(npairs, tau, theta, u_try, nk, radius_bits, status);
    else if (eq == EQ_POLY2) k_vn_radius<EQ_POLY2><<<g, 128, 0, s>>>(npairs, tau, theta, u_try, nk, radius_bits, status);
    else if (eq == EQ_PROD) k_vn_radius<EQ_PROD><<<g, 128, 0, s>>>(npairs, tau, theta, u_try, nk, radius_bits, status);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

}  // namespace lbmh
