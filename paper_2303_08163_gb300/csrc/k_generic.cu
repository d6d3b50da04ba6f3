// k_generic.cu -- auxiliary kernels of a single lattice: initialisation f = f^eq(rho, u),
// moments, canonical population export / import (undoing the AA odd-step slot
// permutation), sampled export, diagnostics of a state, the fixed-order final reduction
// of diagnostics, the bounded-wait self test, and the generic step dispatcher.
#include "lbm_common.cuh"
#include "ptx.cuh"

namespace lbmh {
cudaError_t step_generic_d2(const StepArgs &a, int blocks, int threads, cudaStream_t s);
cudaError_t step_generic_d3(const StepArgs &a, int blocks, int threads, cudaStream_t s);
}  // namespace lbmh

namespace lbmd {

static inline int grid_for(int64_t n, int threads, int cap = 152 * 32) {
    int64_t g = (n + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

// f = f^eq(rho, u), written in the even (canonical) layout, shifted by w_i rho0.
template <int D, int P, int EQ, typename In>
__global__ void k_init(lbmh::Lattice lat, double rho0d, const In *__restrict__ rho,
                       const In *__restrict__ u) {
    using St = Storage<P>;
    using R = typename St::R;
    constexpr int Q = qof(D);
    auto *A = static_cast<typename St::T *>(lat.A);
    const R rho0 = R(rho0d);
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < lat.ncell;
         c += (int64_t)gridDim.x * blockDim.x) {
        const R r = R(rho[c]);
        R uu[3] = {R(u[c]), R(u[lat.ncell + c]), D == 3 ? R(u[2 * lat.ncell + c]) : R(0)};
        R h[Q];
        equilibrium_h<D, EQ, R>(uu, h);
        const R drho = r - rho0;
#pragma unroll
        for (int i = 0; i < Q; ++i) A[(int64_t)i * lat.plane + c] = St::store(R(wq<D>(i)) * fma_r(r, h[i], drho));
    }
}

template <int D, int P>
__device__ __forceinline__ void load_canonical(const lbmh::Lattice &lat, int odd, int64_t c,
                                               typename Storage<P>::R (&f)[qof(D)], int &x,
                                               int &y, int &z) {
    using St = Storage<P>;
    const auto *A = static_cast<const typename St::T *>(lat.A);
    x = (int)(c % lat.nx);
    const int64_t r = c / lat.nx;
    y = (int)(r % lat.ny);
    z = (int)(r / lat.ny);
#pragma unroll
    for (int i = 0; i < qof(D); ++i)
        f[i] = St::load(A[aa_index<D>(i, x, y, z, lat.nx, lat.ny, lat.nz, lat.plane, odd)]);
}

template <int D, int P, typename Out>
__global__ void k_moments(lbmh::Lattice lat, double rho0d, int odd, Out *__restrict__ rho,
                          Out *__restrict__ u) {
    using R = typename Storage<P>::R;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < lat.ncell;
         c += (int64_t)gridDim.x * blockDim.x) {
        R f[qof(D)];
        int x, y, z;
        load_canonical<D, P>(lat, odd, c, f, x, y, z);
        const CellMoments<R> m = moments_shifted<D, R>(f, R(rho0d));
        rho[c] = Out(m.rho);
        u[c] = Out(m.u[0]);
        u[lat.ncell + c] = Out(m.u[1]);
        if (D == 3) u[2 * lat.ncell + c] = Out(m.u[2]);
    }
}

template <int D, int P, typename Out>
__global__ void k_get_pop(lbmh::Lattice lat, double rho0, int odd, Out *__restrict__ f) {
    using R = typename Storage<P>::R;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < lat.ncell;
         c += (int64_t)gridDim.x * blockDim.x) {
        R g[qof(D)];
        int x, y, z;
        load_canonical<D, P>(lat, odd, c, g, x, y, z);
#pragma unroll
        for (int i = 0; i < qof(D); ++i) f[(int64_t)i * lat.ncell + c] = Out((double)g[i] + wq<D>(i) * rho0);
    }
}

template <int D, int P, typename In>
__global__ void k_set_pop(lbmh::Lattice lat, double rho0, int odd, const In *__restrict__ f) {
    using St = Storage<P>;
    using R = typename St::R;
    auto *A = static_cast<typename St::T *>(lat.A);
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < lat.ncell;
         c += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(c % lat.nx);
        const int64_t r = c / lat.nx;
        const int y = (int)(r % lat.ny), z = (int)(r / lat.ny);
#pragma unroll
        for (int i = 0; i < qof(D); ++i) {
            const double v = (double)f[(int64_t)i * lat.ncell + c] - wq<D>(i) * rho0;
            A[aa_index<D>(i, x, y, z, lat.nx, lat.ny, lat.nz, lat.plane, odd)] = St::store(R(v));
        }
    }
}

// Raw stored (shifted) values in the canonical layout, bit for bit.
template <int D, int P>
__global__ void k_get_pop_raw(lbmh::Lattice lat, int odd, typename Storage<P>::T *__restrict__ f) {
    const auto *A = static_cast<const typename Storage<P>::T *>(lat.A);
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < lat.ncell;
         c += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(c % lat.nx);
        const int64_t r = c / lat.nx;
        const int y = (int)(r % lat.ny), z = (int)(r / lat.ny);
#pragma unroll
        for (int i = 0; i < qof(D); ++i)
            f[(int64_t)i * lat.ncell + c] = A[aa_index<D>(i, x, y, z, lat.nx, lat.ny, lat.nz, lat.plane, odd)];
    }
}

template <int D, int P>
__global__ void k_set_pop_raw(lbmh::Lattice lat, int odd, const typename Storage<P>::T *__restrict__ f) {
    auto *A = static_cast<typename Storage<P>::T *>(lat.A);
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < lat.ncell;
         c += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(c % lat.nx);
        const int64_t r = c / lat.nx;
        const int y = (int)(r % lat.ny), z = (int)(r / lat.ny);
#pragma unroll
        for (int i = 0; i < qof(D); ++i)
            A[aa_index<D>(i, x, y, z, lat.nx, lat.ny, lat.nz, lat.plane, odd)] = f[(int64_t)i * lat.ncell + c];
    }
}

template <int D, int P>
__global__ void k_sample_pop(lbmh::Lattice lat, double rho0, int odd, const int64_t *cells,
                             int64_t count, double *out) {
    using R = typename Storage<P>::R;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < count;
         k += (int64_t)gridDim.x * blockDim.x) {
        R g[qof(D)];
        int x, y, z;
        load_canonical<D, P>(lat, odd, cells[k], g, x, y, z);
#pragma unroll
        for (int i = 0; i < qof(D); ++i) out[k * qof(D) + i] = (double)g[i] + wq<D>(i) * rho0;
    }
}

template <int D, int P>
__global__ void __launch_bounds__(256) k_diag_state(lbmh::Lattice lat, double rho0d, int odd,
                                                    double *partials) {
    using R = typename Storage<P>::R;
    DiagAcc acc;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < lat.ncell;
         c += (int64_t)gridDim.x * blockDim.x) {
        R f[qof(D)];
        int x, y, z;
        load_canonical<D, P>(lat, odd, c, f, x, y, z);
        const CellMoments<R> m = moments_shifted<D, R>(f, R(rho0d));
        acc.add(m.rho, m.u);
    }
    diag_block_store(acc, partials + (int64_t)blockIdx.x * lbmh::kDiagWords);
}

// record = {mass, jx, jy, jz, kinetic, max|u|, nonfinite, step}: sums of the per-block
// partials in a fixed order (thread t takes blocks t, t + 256, ..., then a fixed tree).
__global__ void __launch_bounds__(256) k_diag_finalize(const double *partials, int blocks,
                                                       int64_t step, double *record) {
    __shared__ double red[256][7];
    double s[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < blocks; b += blockDim.x) {
#pragma unroll
        for (int q = 0; q < 7; ++q) {
            const double v = partials[(int64_t)b * lbmh::kDiagWords + q];
            s[q] = (q == 5) ? fmax(s[q], v) : s[q] + v;
        }
    }
#pragma unroll
    for (int q = 0; q < 7; ++q) red[threadIdx.x][q] = s[q];
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
#pragma unroll
            for (int q = 0; q < 7; ++q) {
                const double o = red[threadIdx.x + w][q];
                red[threadIdx.x][q] = (q == 5) ? fmax(red[threadIdx.x][q], o) : red[threadIdx.x][q] + o;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < 7; ++q) record[q] = red[0][q];
        record[7] = (double)step;
    }
}

__global__ void k_selftest_wait(int64_t timeout_ns, int32_t *status) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_barrier_init();
    }
    __syncthreads();
    const bool ok = mbar_wait_bounded(&bar, 0, timeout_ns);
    if (threadIdx.x == 0) *status = ok ? 0 : -5; /* LBM_ETIMEOUT */
}

}  // namespace lbmd

namespace lbmh {

using namespace lbmd;

int diag_blocks_generic(int64_t ncell) { return grid_for(ncell, 256, 152 * 8); }

cudaError_t step_generic(const StepArgs &a, int blocks, int threads, cudaStream_t s) {
    return a.lat.D == 2 ? step_generic_d2(a, blocks, threads, s) : step_generic_d3(a, blocks, threads, s);
}

#define LBM_DISPATCH_DP(D_, P_, CALL)                                                      \
    do {                                                                                   \
        if ((D_) == 2 && (P_) == P_F64) { constexpr int DD = 2, PP = P_F64; CALL; }        \
        else if ((D_) == 2 && (P_) == P_F32) { constexpr int DD = 2, PP = P_F32; CALL; }   \
        else if ((D_) == 2 && (P_) == P_F16S) { constexpr int DD = 2, PP = P_F16S; CALL; } \
        else if ((D_) == 3 && (P_) == P_F64) { constexpr int DD = 3, PP = P_F64; CALL; }   \
        else if ((D_) == 3 && (P_) == P_F32) { constexpr int DD = 3, PP = P_F32; CALL; }   \
        else if ((D_) == 3 && (P_) == P_F16S) { constexpr int DD = 3, PP = P_F16S; CALL; } \
        else return cudaErrorInvalidValue;                                                 \
    } while (0)

cudaError_t init_fields(const Lattice &lat, int eq, double rho0, const void *rho, const void *u,
                        int dtype, cudaStream_t s) {
    const int g = grid_for(lat.ncell, 256);
#define LBM_INIT_EQ(EQv)                                                                         \
    if (eq == EQv) {                                                                             \
        if (dtype == 0)                                                                          \
            LBM_DISPATCH_DP(lat.D, lat.P, (k_init<DD, PP, EQv, double><<<g, 256, 0, s>>>(        \
                                                lat, rho0, (const double *)rho, (const double *)u))); \
        else                                                                                     \
            LBM_DISPATCH_DP(lat.D, lat.P, (k_init<DD, PP, EQv, float><<<g, 256, 0, s>>>(         \
                                                lat, rho0, (const float *)rho, (const float *)u))); \
        return cudaGetLastError();                                                               \
    }
    LBM_INIT_EQ(EQ_ENT)
    LBM_INIT_EQ(EQ_POLY2)
    LBM_INIT_EQ(EQ_PROD)
#undef LBM_INIT_EQ
    return cudaErrorInvalidValue;
}

cudaError_t moments(const Lattice &lat, double rho0, int odd, void *rho, void *u, int dtype,
                    cudaStream_t s) {
    const int g = grid_for(lat.ncell, 256);
    if (dtype == 0)
        LBM_DISPATCH_DP(lat.D, lat.P, (k_moments<DD, PP, double><<<g, 256, 0, s>>>(lat, rho0, odd, (double *)rho, (double *)u)));
    else
        LBM_DISPATCH_DP(lat.D, lat.P, (k_moments<DD, PP, float><<<g, 256, 0, s>>>(lat, rho0, odd, (float *)rho, (float *)u)));
    return cudaGetLastError();
}

cudaError_t get_populations(const Lattice &lat, double rho0, int odd, void *f, int dtype,
                            cudaStream_t s) {
    const int g = grid_for(lat.ncell, 256);
    if (dtype == 2)
        LBM_DISPATCH_DP(lat.D, lat.P, (k_get_pop_raw<DD, PP><<<g, 256, 0, s>>>(lat, odd, (typename Storage<PP>::T *)f)));
    else if (dtype == 0)
        LBM_DISPATCH_DP(lat.D, lat.P, (k_get_pop<DD, PP, double><<<g, 256, 0, s>>>(lat, rho0, odd, (double *)f)));
    else
        LBM_DISPATCH_DP(lat.D, lat.P, (k_get_pop<DD, PP, float><<<g, 256, 0, s>>>(lat, rho0, odd, (float *)f)));
    return cudaGetLastError();
}

cudaError_t set_populations(const Lattice &lat, double rho0, int odd, const void *f, int dtype,
                            cudaStream_t s) {
    const int g = grid_for(lat.ncell, 256);
    if (dtype == 2)
        LBM_DISPATCH_DP(lat.D, lat.P, (k_set_pop_raw<DD, PP><<<g, 256, 0, s>>>(lat, odd, (const typename Storage<PP>::T *)f)));
    else if (dtype == 0)
        LBM_DISPATCH_DP(lat.D, lat.P, (k_set_pop<DD, PP, double><<<g, 256, 0, s>>>(lat, rho0, odd, (const double *)f)));
    else
        LBM_DISPATCH_DP(lat.D, lat.P, (k_set_pop<DD, PP, float><<<g, 256, 0, s>>>(lat, rho0, odd, (const float *)f)));
    return cudaGetLastError();
}

cudaError_t sample_populations(const Lattice &lat, double rho0, int odd, const int64_t *cells,
                               int64_t count, double *out, cudaStream_t s) {
    const int g = grid_for(count, 128);
    LBM_DISPATCH_DP(lat.D, lat.P, (k_sample_pop<DD, PP><<<g, 128, 0, s>>>(lat, rho0, odd, cells, count, out)));
    return cudaGetLastError();
}

cudaError_t diag_state(const Lattice &lat, double rho0, int odd, double *partials, int blocks,
                       cudaStream_t s) {
    LBM_DISPATCH_DP(lat.D, lat.P, (k_diag_state<DD, PP><<<blocks, 256, 0, s>>>(lat, rho0, odd, partials)));
    return cudaGetLastError();
}

cudaError_t diag_finalize(const double *partials, int blocks, int64_t step, double *record,
                          cudaStream_t s) {
    k_diag_finalize<<<1, 256, 0, s>>>(partials, blocks, step, record);
    return cudaGetLastError();
}

cudaError_t selftest_wait(int64_t timeout_ns, int32_t *status, cudaStream_t s) {
    k_selftest_wait<<<1, 32, 0, s>>>(timeout_ns, status);
    return cudaGetLastError();
}

}  // namespace lbmh
