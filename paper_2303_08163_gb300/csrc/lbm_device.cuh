// lbm_device.cuh -- device-side lattice constants, storage formats and the fused
// equilibrium + BGK collision of one cell (arXiv 2303.08163, Sec. II and Sec. V.B).
//
// Populations are held shifted, ft_i = f_i - w_i rho0.  The collision of one cell:
//   moments     rho = rho0 + sum ft_i, j = sum c_i ft_i (sum w_i c_i = 0), u = j / rho
//   equilibrium f_i^eq - w_i rho0 = w_i (drho + rho h_i), drho = rho - rho0, with
//     entropic (Eq. eq:Entropic_isothermal_EDF): f^eq_i = w_i rho prod_a t_a(c_ia),
//       t(0) = 2 - S, t(+-1) = (2 - S) Z^{+-1} = 2 S - 1 +- 3u, S = sqrt(1 + 3 u^2).
//       (The identity (2 - S)(2u + S) = (2S - 1 + 3u)(1 - u) follows from S^2 = 1 + 3u^2
//       and removes the division by 1 - u.)  With d = t - 1:
//       d(0) = -(S - 1), d(+-1) = 2 (S - 1) +- 3u, S - 1 = 3u^2 / (1 + S) (no cancellation),
//       h_i = prod_a (1 + d_a) - 1 built by nested fused multiply-adds.
//     product form (Eq. eq:Product_isothermal_EDF): same structure with
//       t(0) = 1 - 3/2 u^2, t(+-1) = 1 +- 3u + 3u^2 (i.e. the 1-D factors divided by w).
//     quadratic (Eq. eq:Poly2_isothermal_EDF): h_i = 3 c.u + 9/2 (c.u)^2 - 3/2 u^2.
//   relaxation  2 beta = 1 / tau, or with the local bulk correction (Eq. eq:redefined_
//     relaxation rate) 2 beta = 2 A vs^2 / (2 nu + A vs^2) = 2 A / (6 nu + A), where
//     A = min_a A(u_a).  For the entropic equilibrium Eq. (eq:entropic_bulk) simplifies,
//     with S^2 = 1 + x^2, to A = (2 - S) / S^2, which decreases with |u|, so the minimum
//     is taken at the largest S.  For the polynomial forms A = 1 - 9/2 u^2 (Eq. eq:LBGK_bulk).
//   collide     ft*_i = ft_i + 2 beta (ft^eq_i - ft_i) = (1 - 2beta) ft_i + 2beta w_i (drho + rho h_i).
#pragma once

#include <cuda_fp16.h>
#include <stdint.h>

namespace lbmd {

enum { P_F64 = 0, P_F32 = 1, P_F16S = 2 };
enum { EQ_ENT = 0, EQ_POLY2 = 1, EQ_PROD = 2 };

__host__ __device__ constexpr int qof(int D) { return D == 2 ? 9 : 27; }
// population index i = (cx + 1) + 3 (cy + 1) + 9 (cz + 1); opposite = Q - 1 - i
__host__ __device__ constexpr int cxo(int i) { return i % 3 - 1; }
__host__ __device__ constexpr int cyo(int i) { return (i / 3) % 3 - 1; }
__host__ __device__ constexpr int czo(int i) { return i / 9 - 1; }
__host__ __device__ constexpr double w1d(int c) { return c == 0 ? 2.0 / 3.0 : 1.0 / 6.0; }
template <int D>
__host__ __device__ constexpr double wq(int i) {
    return D == 2 ? w1d(cxo(i)) * w1d(cyo(i)) : w1d(cxo(i)) * w1d(cyo(i)) * w1d(czo(i));
}
// weight class: number of nonzero velocity components (0 .. D); for D = 2 only the
// first two digits of the index are velocity components
template <int D>
__host__ __device__ constexpr int wclass(int i) {
    return (cxo(i) != 0) + (cyo(i) != 0) + (D == 3 && czo(i) != 0);
}
// weight of a population with n nonzero components: (1/6)^n (2/3)^(D - n)
template <int D>
__host__ __device__ constexpr double wclass_weight(int n) {
    return (n >= 1 ? 1.0 / 6.0 : 1.0) * (n >= 2 ? 1.0 / 6.0 : 1.0) * (n >= 3 ? 1.0 / 6.0 : 1.0) *
           (D - n >= 1 ? 2.0 / 3.0 : 1.0) * (D - n >= 2 ? 2.0 / 3.0 : 1.0) *
           (D - n >= 3 ? 2.0 / 3.0 : 1.0);
}

template <int P> struct Storage;
template <> struct Storage<P_F64> {
    using T = double;
    using R = double;
    static __host__ __device__ __forceinline__ R load(T v) { return v; }
    static __host__ __device__ __forceinline__ T store(R v) { return v; }
};
template <> struct Storage<P_F32> {
    using T = float;
    using R = float;
    static __host__ __device__ __forceinline__ R load(T v) { return v; }
    static __host__ __device__ __forceinline__ T store(R v) { return v; }
};
template <> struct Storage<P_F16S> {
    using T = __half;
    using R = float;
    static __host__ __device__ __forceinline__ R load(T v) { return __half2float(v); }
    static __host__ __device__ __forceinline__ T store(R v) { return __float2half_rn(v); }
};

// Arithmetic helpers: FP64 keeps IEEE sqrt and division (parity path); FP32 uses the
// hardware reciprocal square root and fast division (a few ulp, far below the
// storage rounding of the FP32 and binary16 formats).
__host__ __device__ __forceinline__ double sqrt_r(double x) { return sqrt(x); }
__host__ __device__ __forceinline__ float sqrt_r(float x) {
#ifdef __CUDA_ARCH__
    return x * rsqrtf(x);
#else
    return sqrtf(x);
#endif
}
__host__ __device__ __forceinline__ double div_r(double a, double b) { return a / b; }
__host__ __device__ __forceinline__ float div_r(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fdividef(a, b);
#else
    return a / b;
#endif
}
__host__ __device__ __forceinline__ double fma_r(double a, double b, double c) { return fma(a, b, c); }
__host__ __device__ __forceinline__ float fma_r(float a, float b, float c) { return fmaf(a, b, c); }

template <typename R> struct CellMoments {
    R rho;   // density
    R u[3];  // velocity (u[2] = 0 in 2-D)
};

// Per-axis equilibrium factors d(c) = t(c) - 1 for c = -1, 0, +1; also returns the
// quantity the bulk coefficient depends on (S for the entropic form, u^2 otherwise).
template <int EQ, typename R>
__host__ __device__ __forceinline__ void axis_factors(R u, R &dm, R &d0, R &dp, R &key) {
    const R u2 = u * u;
    if constexpr (EQ == EQ_ENT) {
        const R s2 = fma_r(R(3), u2, R(1));
        const R S = sqrt_r(s2);
        const R sm1 = div_r(R(3) * u2, R(1) + S);  // S - 1 without cancellation
        d0 = -sm1;
        dp = fma_r(R(2), sm1, R(3) * u);
        dm = fma_r(R(2), sm1, R(-3) * u);
        key = S;
    } else {  // product form (also used for the per-axis key of the polynomial form)
        const R t3 = R(3) * u2;
        d0 = R(-1.5) * u2;
        dp = fma_r(R(3), u, t3);
        dm = fma_r(R(-3), u, t3);
        key = u2;
    }
}

// The per-axis factors of all D axes.  In FP64 the entropic form's D divisions
// 3u_a^2 / (1 + S_a) share one reciprocal of the product of the (1 + S_a), each axis
// multiplying it by the other axes' factors (a few ulp, one IEEE division instead of D;
// FP64 divisions are long instruction sequences on the FP64 pipe).
template <int D, int EQ, typename R>
__host__ __device__ __forceinline__ void all_axis_factors(const R (&u)[3], R (&dm)[3], R (&d0)[3],
                                                          R (&dp)[3], R (&key)[3]) {
    if constexpr (EQ == EQ_ENT && sizeof(R) == 8) {
        R u2[3], S[3], op[3];
#pragma unroll
        for (int a = 0; a < D; ++a) {
            u2[a] = u[a] * u[a];
            S[a] = sqrt_r(fma_r(R(3), u2[a], R(1)));
            op[a] = R(1) + S[a];
        }
        R inv[3];
        if constexpr (D == 2) {
            const R r = R(1) / (op[0] * op[1]);
            inv[0] = r * op[1];
            inv[1] = r * op[0];
        } else {
            const R yz = op[1] * op[2];
            const R r = R(1) / (op[0] * yz);
            inv[0] = r * yz;
            inv[1] = r * (op[0] * op[2]);
            inv[2] = r * (op[0] * op[1]);
        }
#pragma unroll
        for (int a = 0; a < D; ++a) {
            const R sm1 = R(3) * u2[a] * inv[a];  // S - 1 without cancellation
            d0[a] = -sm1;
            dp[a] = fma_r(R(2), sm1, R(3) * u[a]);
            dm[a] = fma_r(R(2), sm1, R(-3) * u[a]);
            key[a] = S[a];
        }
    } else {
#pragma unroll
        for (int a = 0; a < D; ++a) axis_factors<EQ>(u[a], dm[a], d0[a], dp[a], key[a]);
    }
}

// Local collision frequency 2 beta from the largest per-axis key.
template <int EQ, bool BULK, typename R>
__host__ __device__ __forceinline__ R collision_rate(R key_max, R omega0, R six_nu) {
    if constexpr (!BULK) {
        return omega0;
    } else if constexpr (EQ == EQ_ENT) {
        const R S = key_max;
        const R A2 = R(2) - S;                      // A S^2
        return div_r(R(2) * A2, fma_r(six_nu, S * S, A2));
    } else {
        const R A = fma_r(R(-4.5), key_max, R(1));  // 1 - 3/2 u^2 / vs^2
        return div_r(R(2) * A, six_nu + A);
    }
}

// h_i such that f^eq_i - w_i rho0 = w_i (drho + rho h_i), for all i; returns the
// largest per-axis key (see axis_factors) for the bulk correction.
template <int D, int EQ, typename R>
__host__ __device__ __forceinline__ R equilibrium_h(const R (&u)[3], R (&h)[qof(D)]) {
    constexpr int Q = qof(D);
    if constexpr (EQ == EQ_POLY2) {
        // h = 3 cu + 9/2 cu^2 - 3/2 u^2
        R uu = u[0] * u[0] + u[1] * u[1];
        if constexpr (D == 3) uu = fma_r(u[2], u[2], uu);
        const R m = R(-1.5) * uu;
        R cxy[9];
#pragma unroll
        for (int p = 0; p < 9; ++p) {
            const int cx = cxo(p), cy = cyo(p);
            R v = R(0);
            if (cx == 1) v = u[0];
            if (cx == -1) v = -u[0];
            if (cy == 1) v = v + u[1];
            if (cy == -1) v = v - u[1];
            cxy[p] = v;
        }
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int cz = (D == 3) ? czo(i) : 0;
            R cu = cxy[i % 9];
            if (cz == 1) cu = cu + u[2];
            if (cz == -1) cu = cu - u[2];
            h[i] = fma_r(cu, fma_r(R(4.5), cu, R(3)), m);
        }
        R k = u[0] * u[0];
        k = fmax(k, u[1] * u[1]);
        if constexpr (D == 3) k = fmax(k, u[2] * u[2]);
        return k;
    } else {
        R dm[3], d0[3], dp[3], key[3];
        all_axis_factors<D, EQ>(u, dm, d0, dp, key);
        R kmax = fmax(key[0], key[1]);
        if constexpr (D == 3) kmax = fmax(kmax, key[2]);
        // d and t = 1 + d per axis, indexed by c + 1
        R dx[3] = {dm[0], d0[0], dp[0]};
        R dy[3] = {dm[1], d0[1], dp[1]};
        R tx[3] = {R(1) + dm[0], R(1) + d0[0], R(1) + dp[0]};
        if constexpr (D == 2) {
#pragma unroll
            for (int i = 0; i < 9; ++i) h[i] = fma_r(dy[cyo(i) + 1], tx[cxo(i) + 1], dx[cxo(i) + 1]);
        } else {
            R ty[3] = {R(1) + dm[1], R(1) + d0[1], R(1) + dp[1]};
            R dz[3] = {dm[2], d0[2], dp[2]};
            R exy[9], txy[9];
#pragma unroll
            for (int p = 0; p < 9; ++p) {
                exy[p] = fma_r(dy[cyo(p) + 1], tx[cxo(p) + 1], dx[cxo(p) + 1]);
                txy[p] = tx[cxo(p) + 1] * ty[cyo(p) + 1];
            }
#pragma unroll
            for (int i = 0; i < 27; ++i) h[i] = fma_r(dz[czo(i) + 1], txy[i % 9], exy[i % 9]);
        }
        return kmax;
    }
}

// Density and momentum of one cell from shifted populations.  The partial sums follow the
// tensor structure of the lattice (first over c_z, then c_y, then c_x).
template <int D, typename R>
__host__ __device__ __forceinline__ void moment_sums(const R (&f)[qof(D)], R rho0, R &rho, R (&j)[3]) {
    R a[9], bz[9];
    if constexpr (D == 2) {
#pragma unroll
        for (int p = 0; p < 9; ++p) a[p] = f[p];
    } else {
#pragma unroll
        for (int p = 0; p < 9; ++p) {
            a[p] = (f[p] + f[p + 9]) + f[p + 18];
            bz[p] = f[p + 18] - f[p];
        }
    }
    const R c0 = (a[0] + a[3]) + a[6];  // c_x = -1
    const R c1 = (a[1] + a[4]) + a[7];  // c_x = 0
    const R c2 = (a[2] + a[5]) + a[8];  // c_x = +1
    const R rt = (c0 + c1) + c2;
    j[0] = c2 - c0;
    j[1] = ((a[6] + a[7]) + a[8]) - ((a[0] + a[1]) + a[2]);
    j[2] = R(0);
    if constexpr (D == 3) {
        j[2] = ((bz[0] + bz[1]) + (bz[2] + bz[3])) + ((bz[4] + bz[5]) + (bz[6] + bz[7])) + bz[8];
    }
    rho = rho0 + rt;
}

// Moments of one cell from shifted populations: rho and u = j / rho.
template <int D, typename R>
__host__ __device__ __forceinline__ CellMoments<R> moments_shifted(const R (&f)[qof(D)], R rho0) {
    CellMoments<R> m;
    R jv[3];
    moment_sums<D, R>(f, rho0, m.rho, jv);
    const R jx = jv[0], jy = jv[1], jz = jv[2];
    const R inv = div_r(R(1), m.rho);
    m.u[0] = jx * inv;
    m.u[1] = jy * inv;
    m.u[2] = jz * inv;
    return m;
}

// The relaxation f* = (1 - 2beta) f + 2beta w_i (drho + rho h_i) of one direction of
// weight class c, in one of two forms.  TWO_FMA: two FMAs per direction, with the
// per-class products 2beta w rho and 2beta w drho formed once per cell (fewest
// instructions: used where instruction issue is the bound, FP64 and D2Q9 with binary16
// storage).  Otherwise the factored form 2beta w (rho h + drho) + (1 - 2beta) f, which
// measured faster for the bandwidth-bound FP32 and D3Q27 binary16 steps (fewer live
// registers).  Both kernels of a lattice use the same form, so their states agree bit for
// bit.
template <int D, int P>
__host__ __device__ constexpr bool relax_two_fma() {
    return P == P_F64 || (D == 2 && P == P_F16S);
}

template <typename R, bool TWO_FMA = (sizeof(R) == 8)> struct Relax {
    R keep, rho, drho, omw[4], wr[4], wd[4];
    __host__ __device__ __forceinline__ Relax(R om, double w0, double w1, double w2, double w3, R rho_,
                                              R drho_)
        : keep(R(1) - om), rho(rho_), drho(drho_) {
        const double w[4] = {w0, w1, w2, w3};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            omw[c] = om * R(w[c]);
            wr[c] = omw[c] * rho;
            wd[c] = omw[c] * drho;
        }
    }
    __host__ __device__ __forceinline__ R operator()(int c, R h, R f) const {
        if constexpr (TWO_FMA) return fma_r(wr[c], h, fma_r(keep, f, wd[c]));
        else return fma_r(omw[c], fma_r(rho, h, drho), keep * f);
    }
};

// FP64 entropic collisions: the moments and the per-axis factors with one IEEE division.
// With T_a = rho S_a = sqrt(rho^2 + 3 j_a^2) and q_a = rho + T_a = rho (1 + S_a), the
// identities 1/rho = (prod_a q_a) / (rho prod_a q_a) and S_a - 1 = 3 u_a^2 / (1 + S_a) =
// 3 j_a^2 / (rho q_a) let one reciprocal of rho prod_a q_a serve 1/rho and every axis
// (exact rewrites, a few ulp apart from the separate divisions).
template <int D, typename R>
__host__ __device__ __forceinline__ void entropic_factors_one_division(
    const R (&f)[qof(D)], R rho0, CellMoments<R> &m, R (&dm)[3], R (&d0)[3], R (&dp)[3], R (&key)[3]) {
    R j[3];
    moment_sums<D, R>(f, rho0, m.rho, j);
    const R rho = m.rho, rho2 = rho * rho;
    R j3[3], T[3], q[3], cof[3];
#pragma unroll
    for (int a = 0; a < D; ++a) {
        j3[a] = R(3) * j[a];
        T[a] = sqrt_r(fma_r(j3[a], j[a], rho2));
        q[a] = rho + T[a];
    }
    R qprod;
    if constexpr (D == 2) {
        cof[0] = q[1];
        cof[1] = q[0];
        qprod = q[0] * q[1];
    } else {
        cof[0] = q[1] * q[2];
        cof[1] = q[0] * q[2];
        cof[2] = q[0] * q[1];
        qprod = q[0] * cof[0];
    }
    const R r = R(1) / (rho * qprod);
    const R irho = r * qprod;
    m.u[2] = R(0);
#pragma unroll
    for (int a = 0; a < D; ++a) {
        m.u[a] = j[a] * irho;
        const R sm1 = (j3[a] * j[a]) * (r * cof[a]);  // S - 1 without cancellation
        const R u3 = j3[a] * irho;
        d0[a] = -sm1;
        dp[a] = fma_r(R(2), sm1, u3);
        dm[a] = fma_r(R(2), sm1, -u3);
        key[a] = T[a] * irho;
    }
}

// The fused collision of one cell, in place on shifted populations.  Returns the
// pre-collision moments (the macroscopic state at the current time step).  The
// equilibrium term h_i of each direction is formed inside the relaxation loop from the
// per-axis factors, so only the Q populations and O(D^2) factors stay live.
template <int D, int EQ, bool BULK, typename R, bool TWO_FMA = (sizeof(R) == 8)>
__host__ __device__ __forceinline__ CellMoments<R> collide(R (&f)[qof(D)], R rho0, R omega0, R six_nu) {
    constexpr int Q = qof(D);
    // weights per number of nonzero velocity components, folded at compile time
    constexpr double kW0 = wclass_weight<D>(0), kW1 = wclass_weight<D>(1);
    constexpr double kW2 = wclass_weight<D>(2), kW3 = wclass_weight<D>(D >= 3 ? 3 : 0);
    CellMoments<R> m;
    R dm[3], d0[3], dp[3], key[3];  // per-axis factors (entropic and product forms)
    if constexpr (EQ == EQ_ENT && sizeof(R) == 8) {
        entropic_factors_one_division<D, R>(f, rho0, m, dm, d0, dp, key);
    } else {
        m = moments_shifted<D, R>(f, rho0);
        if constexpr (EQ != EQ_POLY2) all_axis_factors<D, EQ>(m.u, dm, d0, dp, key);
    }
    const R drho = m.rho - rho0;
    if constexpr (EQ == EQ_POLY2) {
        R uu = m.u[0] * m.u[0] + m.u[1] * m.u[1];
        if constexpr (D == 3) uu = fma_r(m.u[2], m.u[2], uu);
        R k = fmax(m.u[0] * m.u[0], m.u[1] * m.u[1]);
        if constexpr (D == 3) k = fmax(k, m.u[2] * m.u[2]);
        const R om = collision_rate<EQ, BULK, R>(k, omega0, six_nu);
        const R mh = R(-1.5) * uu;
        const Relax<R, TWO_FMA> relax(om, kW0, kW1, kW2, kW3, m.rho, drho);
        const R upm = m.u[0] + m.u[1], umm = m.u[0] - m.u[1];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int cx = cxo(i), cy = cyo(i), cz = (D == 3) ? czo(i) : 0;
            R cu;
            if (cx == 0 && cy == 0) cu = R(0);
            else if (cx == 0) cu = cy > 0 ? m.u[1] : -m.u[1];
            else if (cy == 0) cu = cx > 0 ? m.u[0] : -m.u[0];
            else if (cx == cy) cu = cx > 0 ? upm : -upm;
            else cu = cx > 0 ? umm : -umm;
            if (cz == 1) cu = cu + m.u[2];
            if (cz == -1) cu = cu - m.u[2];
            const R h = fma_r(cu, fma_r(R(4.5), cu, R(3)), mh);
            f[i] = relax(wclass<D>(i), h, f[i]);
        }
    } else {
        R kmax = fmax(key[0], key[1]);
        if constexpr (D == 3) kmax = fmax(kmax, key[2]);
        const R om = collision_rate<EQ, BULK, R>(kmax, omega0, six_nu);
        const Relax<R, TWO_FMA> relax(om, kW0, kW1, kW2, kW3, m.rho, drho);
        const R dx[3] = {dm[0], d0[0], dp[0]};
        const R dy[3] = {dm[1], d0[1], dp[1]};
        const R tx[3] = {R(1) + dm[0], R(1) + d0[0], R(1) + dp[0]};
        if constexpr (D == 2) {
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const R h = fma_r(dy[cyo(i) + 1], tx[cxo(i) + 1], dx[cxo(i) + 1]);
                f[i] = relax(wclass<D>(i), h, f[i]);
            }
        } else {
            const R ty[3] = {R(1) + dm[1], R(1) + d0[1], R(1) + dp[1]};
            const R dz[3] = {dm[2], d0[2], dp[2]};
#pragma unroll
            for (int p = 0; p < 9; ++p) {
                // h = prod (1 + d) - 1 over x, y, z = e_xy + d_z (1 + e_xy)
                const R exy = fma_r(dy[cyo(p) + 1], tx[cxo(p) + 1], dx[cxo(p) + 1]);
                const R txy = tx[cxo(p) + 1] * ty[cyo(p) + 1];
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    const int i = p + 9 * q;
                    const R h = fma_r(dz[q], txy, exy);
                    f[i] = relax(wclass<D>(i), h, f[i]);
                }
            }
        }
    }
    return m;
}

}  // namespace lbmd
