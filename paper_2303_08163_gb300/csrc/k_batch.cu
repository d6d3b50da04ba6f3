// k_batch.cu -- many independent periodic lattices (the linear-mode sweep of Sec. V)
// advanced for n steps by one persistent launch.
//
// Every instance is owned by exactly one block (a greedy longest-first assignment on the
// host balances the cell counts), so the only synchronisation between steps is the
// block's own barrier: no block ever waits for another.  Each step of an instance is the
// AA-pattern update of the generic kernel in FP64 (the state of the linear sweep is FP64;
// on GB300 this path is bound by the FP64 pipe, not by memory).  On steps t with
// t % every_k == 0 the block also projects rho and j = rho u of the state at t on
// exp(-i k.r) (twiddle tables per axis), reduces them in a fixed order and records one
// sample per instance; a non-finite mass marks the instance's status with t + 1.
#include "k_generic_step.cuh"

namespace lbmd {

struct ProbeAcc {
    double v[8];  // re, im of rho, jx, jy, jz
};

template <int D, int EQ, bool BULK>
__global__ void __launch_bounds__(256) k_step_batch(const lbmh::BatchArgs a) {
    __shared__ double red[8][8];
    const int b0 = a.block_start[blockIdx.x], b1 = a.block_start[blockIdx.x + 1];
    constexpr int Q = qof(D);
    for (int64_t s = 0; s < a.nsteps; ++s) {
        const int64_t t = a.step0 + s;
        const int odd = (int)(t & 1);
        const bool probe = a.every_k > 0 && (t % a.every_k) == 0;
        for (int ii = b0; ii < b1; ++ii) {
            const int k = a.order[ii];
            const int nx = a.dims[3 * k], ny = a.dims[3 * k + 1], nz = a.dims[3 * k + 2];
            const int64_t c0 = a.cell_start[k];
            const int64_t ncell = a.cell_start[k + 1] - c0;
            double *A = a.arena + (int64_t)Q * c0;
            const double om = a.omega0[k], sn = a.six_nu[k];
            const double2 *tw = a.twiddle + a.tw_offset[k];
            double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            for (int64_t c = threadIdx.x; c < ncell; c += blockDim.x) {
                const int x = (int)(c % nx);
                const int64_t r = c / nx;
                const int y = (int)(r % ny);
                const int z = (int)(r / ny);
                const CellMoments<double> m =
                    aa_cell_step<D, P_F64, EQ, BULK>(A, ncell, nx, ny, nz, x, y, z, odd, a.rho0, om, sn);
                if (probe) {
                    // exp(-i k.r) = tw_x[x] tw_y[y] tw_z[z]
                    const double2 tx = tw[x], ty = tw[nx + y];
                    double pr = tx.x * ty.x - tx.y * ty.y;
                    double pi = tx.x * ty.y + tx.y * ty.x;
                    if (D == 3) {
                        const double2 tz = tw[nx + ny + z];
                        const double qr = pr * tz.x - pi * tz.y;
                        pi = pr * tz.y + pi * tz.x;
                        pr = qr;
                    }
                    const double q[4] = {m.rho, m.rho * m.u[0], m.rho * m.u[1], m.rho * m.u[2]};
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        acc[2 * j] += q[j] * pr;
                        acc[2 * j + 1] += q[j] * pi;
                    }
                }
            }
            if (probe) {
                // fixed-order block reduction: warps by shuffle, then warps in order
#pragma unroll
                for (int off = 16; off > 0; off >>= 1)
#pragma unroll
                    for (int j = 0; j < 8; ++j) acc[j] += __shfl_down_sync(0xffffffffu, acc[j], off);
                const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
                if (lane == 0)
#pragma unroll
                    for (int j = 0; j < 8; ++j) red[warp][j] = acc[j];
                __syncthreads();
                if (threadIdx.x == 0) {
                    double sum[8] = {0, 0, 0, 0, 0, 0, 0, 0};
                    const int nw = (blockDim.x + 31) >> 5;
                    for (int w = 0; w < nw; ++w)
                        for (int j = 0; j < 8; ++j) sum[j] += red[w][j];
                    const int64_t sample = t / a.every_k;
                    if (sample < a.max_samples) {
                        double *out = a.series + ((int64_t)k * a.max_samples + sample) * 8;
                        for (int j = 0; j < 8; ++j) out[j] = sum[j];
                    }
                    bool fin = true;
                    for (int j = 0; j < 8; ++j) fin = fin && isfinite(sum[j]);
                    if (!fin && a.status[k] == 0) a.status[k] = (int32_t)(t + 1);
                }
                __syncthreads();
            }
        }
        __syncthreads();  // step boundary: the block's instances are complete at t + 1
    }
}

// Instance of a packed global cell index (binary search over cell_start).
__device__ __forceinline__ int find_instance(const int64_t *cell_start, int64_t count, int64_t g) {
    int64_t lo = 0, hi = count - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (cell_start[mid] <= g) lo = mid;
        else hi = mid - 1;
    }
    return (int)lo;
}

template <int D, int EQ, typename In>
__global__ void k_batch_init(double *arena, const int64_t *cell_start, const int32_t *dims,
                             int64_t count, double rho0, const In *rho, const In *u,
                             int64_t total) {
    constexpr int Q = qof(D);
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int k = find_instance(cell_start, count, g);
        const int64_t c0 = cell_start[k], n = cell_start[k + 1] - c0, c = g - c0;
        const double r = (double)rho[g];
        double uu[3] = {0, 0, 0};
        for (int a = 0; a < D; ++a) uu[a] = (double)u[(int64_t)D * c0 + a * n + c];
        double h[Q];
        equilibrium_h<D, EQ, double>(uu, h);
        double *A = arena + (int64_t)Q * c0;
        for (int i = 0; i < Q; ++i) A[(int64_t)i * n + c] = wq<D>(i) * fma(r, h[i], r - rho0);
    }
}

template <int D, typename Out>
__global__ void k_batch_moments(const double *arena, const int64_t *cell_start, const int32_t *dims,
                                int64_t count, double rho0, int odd, Out *rho, Out *u, int64_t total) {
    constexpr int Q = qof(D);
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int k = find_instance(cell_start, count, g);
        const int64_t c0 = cell_start[k], n = cell_start[k + 1] - c0, c = g - c0;
        const int nx = dims[3 * k], ny = dims[3 * k + 1], nz = dims[3 * k + 2];
        const int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / ((int64_t)nx * ny));
        const double *A = arena + (int64_t)Q * c0;
        double f[Q];
        for (int i = 0; i < Q; ++i) f[i] = A[aa_index<D>(i, x, y, z, nx, ny, nz, n, odd)];
        const CellMoments<double> m = moments_shifted<D, double>(f, rho0);
        rho[g] = Out(m.rho);
        for (int a = 0; a < D; ++a) u[(int64_t)D * c0 + a * n + c] = Out(m.u[a]);
    }
}

template <int D, typename Out>
__global__ void k_batch_pop(const double *arena, const int64_t *cell_start, const int32_t *dims,
                            int64_t count, double rho0, int odd, Out *f, int64_t total) {
    constexpr int Q = qof(D);
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int k = find_instance(cell_start, count, g);
        const int64_t c0 = cell_start[k], n = cell_start[k + 1] - c0, c = g - c0;
        const int nx = dims[3 * k], ny = dims[3 * k + 1], nz = dims[3 * k + 2];
        const int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / ((int64_t)nx * ny));
        const double *A = arena + (int64_t)Q * c0;
        for (int i = 0; i < Q; ++i)
            f[(int64_t)Q * c0 + (int64_t)i * n + c] = Out(A[aa_index<D>(i, x, y, z, nx, ny, nz, n, odd)] + wq<D>(i) * rho0);
    }
}

}  // namespace lbmd

namespace lbmh {

using namespace lbmd;

const void *batch_kernel(int D, int eq, int bulk) {
#define LBM_BK(Dv, EQv)                                                                        \
    if (D == Dv && eq == EQv)                                                                  \
        return bulk ? (const void *)k_step_batch<Dv, EQv, true> : (const void *)k_step_batch<Dv, EQv, false>;
    LBM_BK(2, EQ_ENT)
    LBM_BK(2, EQ_POLY2)
    LBM_BK(2, EQ_PROD)
    LBM_BK(3, EQ_ENT)
    LBM_BK(3, EQ_POLY2)
    LBM_BK(3, EQ_PROD)
#undef LBM_BK
    return nullptr;
}

cudaError_t step_batch(const BatchArgs &a, int blocks, int threads, cudaStream_t s) {
    const void *fn = batch_kernel(a.D, a.eq, a.bulk);
    if (!fn) return cudaErrorInvalidValue;
    BatchArgs aa = a;
    void *args[] = {(void *)&aa};
    return cudaLaunchKernel(fn, dim3(blocks), dim3(threads), args, 0, s);
}

static int grid_cells(int64_t n) {
    int64_t g = (n + 255) / 256;
    return (int)(g < 1 ? 1 : (g > 152 * 32 ? 152 * 32 : g));
}

cudaError_t batch_init(double *arena, const int64_t *cell_start, const int32_t *dims,
                       int64_t count, int D, int eq, double rho0, const void *rho, const void *u,
                       int dtype, int64_t total, cudaStream_t s) {
    const int g = grid_cells(total);
#define LBM_BI(Dv, EQv)                                                                                    \
    if (D == Dv && eq == EQv) {                                                                            \
        if (dtype == 0)                                                                                    \
            k_batch_init<Dv, EQv, double><<<g, 256, 0, s>>>(arena, cell_start, dims, count, rho0,          \
                                                            (const double *)rho, (const double *)u, total); \
        else                                                                                               \
            k_batch_init<Dv, EQv, float><<<g, 256, 0, s>>>(arena, cell_start, dims, count, rho0,           \
                                                           (const float *)rho, (const float *)u, total);    \
        return cudaGetLastError();                                                                         \
    }
    LBM_BI(2, EQ_ENT)
    LBM_BI(2, EQ_POLY2)
    LBM_BI(2, EQ_PROD)
    LBM_BI(3, EQ_ENT)
    LBM_BI(3, EQ_POLY2)
    LBM_BI(3, EQ_PROD)
#undef LBM_BI
    return cudaErrorInvalidValue;
}

cudaError_t batch_moments(const double *arena, const int64_t *cell_start, const int32_t *dims,
                          int64_t count, int D, double rho0, int odd, void *rho, void *u,
                          int dtype, int64_t total, cudaStream_t s) {
    const int g = grid_cells(total);
    if (D == 2 && dtype == 0) k_batch_moments<2, double><<<g, 256, 0, s>>>(arena, cell_start, dims, count, rho0, odd, (double *)rho, (double *)u, total);
    else if (D == 2) k_batch_moments<2, float><<<g, 256, 0, s>>>(arena, cell_start, dims, count, rho0, odd, (float *)rho, (float *)u, total);
    else if (dtype == 0) k_batch_moments<3, double><<<g, 256, 0, s>>>(arena, cell_start, dims, count, rho0, odd, (double *)rho, (double *)u, total);
    else k_batch_moments<3, float><<<g, 256, 0, s>>>(arena, cell_start, dims, count, rho0, odd, (float *)rho, (float *)u, total);
    return cudaGetLastError();
}

cudaError_t batch_populations(const double *arena, const int64_t *cell_start,
                              const int32_t *dims, int64_t count, int D, double rho0, int odd,
                              void *f, int dtype, int64_t total, cudaStream_t s) {
    const int g = grid_cells(total);
    if (D == 2 && dtype == 0) k_batch_pop<2, double><<<g, 256, 0, s>>>(arena, cell_start, dims, count, rho0, odd, (double *)f, total);
    else if (D == 2) k_batch_pop<2, float><<<g, 256, 0, s>>>(arena, cell_start, dims, count, rho0, odd, (float *)f, total);
    else if (dtype == 0) k_batch_pop<3, double><<<g, 256, 0, s>>>(arena, cell_start, dims, count, rho0, odd, (double *)f, total);
    else k_batch_pop<3, float><<<g, 256, 0, s>>>(arena, cell_start, dims, count, rho0, odd, (float *)f, total);
    return cudaGetLastError();
}

}  // namespace lbmh
