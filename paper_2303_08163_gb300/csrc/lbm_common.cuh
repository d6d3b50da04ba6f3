// lbm_common.cuh -- shared device helpers: periodic indexing of the AA pattern and the
// deterministic FP64 block reduction of the fused diagnostics.
#pragma once

#include "lbm_device.cuh"
#include "lbm_internal.h"

namespace lbmd {

__device__ __forceinline__ int wrapi(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// The first error a kernel reports sticks in the device status word.
__device__ __forceinline__ void report_status(int32_t *status, int32_t code) { atomicCAS(status, 0, code); }

// Checked builds (-DLBM_CHECKED): device-side bounds and alignment checks.  A failed check
// records LBM_ECHECK (-7) in the status word and the caller skips the access, so an
// indexing mistake shows up as an error code instead of a memory fault.  In normal builds
// every check is the constant true and compiles away.
#ifdef LBM_CHECKED
__device__ __forceinline__ bool lbm_check(bool ok, int32_t *status) {
    if (!ok && status) report_status(status, -7);
    return ok;
}
#define LBM_CHECK(ok, status) ::lbmd::lbm_check((ok), (status))
#else
#define LBM_CHECK(ok, status) true
#endif

// A per-step scalar in the collision precision (no FP64 conversion in FP32 kernels).
template <typename R> __device__ __forceinline__ R step_scalar(double d, float f);
template <> __device__ __forceinline__ double step_scalar<double>(double d, float) { return d; }
template <> __device__ __forceinline__ float step_scalar<float>(double, float f) { return f; }

// Canonical population f_i(r) = A[i][r] after an even number of steps and
// A[opp(i)][r - c_i] after an odd number (AA pattern: the odd step leaves post-collision
// values in the opposite slot of the sending cell).
template <int D>
__device__ __forceinline__ int64_t aa_index(int i, int x, int y, int z, int nx, int ny, int nz,
                                            int64_t plane, int odd) {
    constexpr int Q = qof(D);
    if (!odd) return (int64_t)i * plane + x + (int64_t)nx * (y + (int64_t)ny * z);
    const int xs = wrapi(x - cxo(i), nx);
    const int ys = wrapi(y - cyo(i), ny);
    const int zs = (D == 3) ? wrapi(z - czo(i), nz) : z;
    return (int64_t)(Q - 1 - i) * plane + xs + (int64_t)nx * (ys + (int64_t)ny * zs);
}

struct DiagAcc {
    double m = 0, jx = 0, jy = 0, jz = 0, ke = 0, umax = 0, nf = 0;

    template <typename R>
    __device__ __forceinline__ void add(R rho, const R (&u)[3]) {
        const double r = rho, ux = u[0], uy = u[1], uz = u[2];
        const bool fin = isfinite(r) && isfinite(ux) && isfinite(uy) && isfinite(uz);
        if (!fin) nf += 1.0;
        m += r;
        jx += r * ux;
        jy += r * uy;
        jz += r * uz;
        ke += 0.5 * r * (ux * ux + uy * uy + uz * uz);
        umax = fmax(umax, fmax(fabs(ux), fmax(fabs(uy), fabs(uz))));
    }

    __device__ __forceinline__ void merge(const DiagAcc &o) {
        m += o.m;
        jx += o.jx;
        jy += o.jy;
        jz += o.jz;
        ke += o.ke;
        umax = fmax(umax, o.umax);
        nf += o.nf;
    }
};

// Partial diagnostics of a few cells in the collision precision R, flushed into the FP64
// accumulator once per job (FP64 arithmetic is a small fraction of the FP32 rate on
// this GPU, so per-cell FP64 sums would dominate a diagnostics step).  Mass is summed as
// rho - rho0 so the FP32 partials carry only the small deviations.
template <typename R>
struct DiagLocal {
    R dm = 0, jx = 0, jy = 0, jz = 0, ke = 0, umax = 0;
    int nf = 0, count = 0;

    __device__ __forceinline__ void add(R rho, const R (&u)[3], R rho0) {
        const bool fin = isfinite(rho) && isfinite(u[0]) && isfinite(u[1]) && isfinite(u[2]);
        nf += fin ? 0 : 1;
        ++count;
        dm += rho - rho0;
        jx += rho * u[0];
        jy += rho * u[1];
        jz += rho * u[2];
        ke += R(0.5) * rho * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        umax = fmax(umax, fmax(fabs(u[0]), fmax(fabs(u[1]), fabs(u[2]))));
    }

    __device__ __forceinline__ void flush(DiagAcc &acc, double rho0) {
        acc.m += (double)count * rho0 + (double)dm;
        acc.jx += (double)jx;
        acc.jy += (double)jy;
        acc.jz += (double)jz;
        acc.ke += (double)ke;
        acc.umax = fmax(acc.umax, (double)umax);
        acc.nf += (double)nf;
        *this = DiagLocal<R>();
    }
};

__device__ __forceinline__ double shfl_down_d(double v, int off) {
    return __shfl_down_sync(0xffffffffu, v, off);
}

// Fixed-order reduction of one DiagAcc per thread to one record of kDiagWords doubles
// per block (warp shuffle, then warps in order).  All threads of the block must call it.
__device__ __forceinline__ void diag_block_store(DiagAcc acc, double *out) {
    __shared__ double red[32][8];
    double v[7] = {acc.m, acc.jx, acc.jy, acc.jz, acc.ke, acc.umax, acc.nf};
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
        for (int q = 0; q < 7; ++q) {
            const double o = shfl_down_d(v[q], off);
            v[q] = (q == 5) ? fmax(v[q], o) : v[q] + o;
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q < 7; ++q) red[warp][q] = v[q];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        double s[7] = {0, 0, 0, 0, 0, 0, 0};
        for (int w = 0; w < nw; ++w) {
#pragma unroll
            for (int q = 0; q < 7; ++q) s[q] = (q == 5) ? fmax(s[q], red[w][q]) : s[q] + red[w][q];
        }
#pragma unroll
        for (int q = 0; q < 7; ++q) out[q] = s[q];
        out[7] = 0.0;
    }
}

}  // namespace lbmd
