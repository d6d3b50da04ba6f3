// noalloc.cu -- diagnostics of caller-owned populations without any device allocation.
//
// Some callers cannot call cudaMalloc: code running inside another framework's memory
// pool or arena, applications that reserve all device memory up front, and stream-capture
// regions where an allocation would break the capture.  For them this entry point
// computes the global diagnostics of a population array they already own, into an
// output buffer they already own.  Its only scratch memory (the per-block partial sums)
// is a file-scope static device array of fixed size that lives for the lifetime of the
// library on every device that loads it; nothing is allocated or freed per call.
#include <cstdio>
#include <mutex>

#include "lbm.h"
#include "lbm_common.cuh"

namespace {

// Scratch of lbm_diagnostics_noalloc: one record of kDiagWords doubles per block.
constexpr int kNoAllocMaxBlocks = 1024;  // 64 KiB of device memory per device
static __device__ __align__(256) double g_noalloc_partials[kNoAllocMaxBlocks * lbmh::kDiagWords];

// Device address of g_noalloc_partials, looked up once per device (the host-side name of
// a __device__ array is only a stand-in; kernels need the address the runtime reports).
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
double *g_noalloc_ptr[kMaxDevices] = {nullptr};

}  // namespace

namespace lbmd {

// The state-diagnostics reduction of k_diag_state, reading canonical (not shifted) FP64
// populations f[Q][ncell] instead of a context's stored layout.
template <int D>
__global__ void __launch_bounds__(256) k_diag_canonical(const double *__restrict__ f, int64_t ncell,
                                                        double *partials) {
    constexpr int Q = qof(D);
    DiagAcc acc;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < ncell;
         c += (int64_t)gridDim.x * blockDim.x) {
        double rho = 0, j[3] = {0, 0, 0};
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const double v = f[(int64_t)i * ncell + c];
            rho += v;
            j[0] += cxo(i) * v;
            j[1] += cyo(i) * v;
            if (D == 3) j[2] += czo(i) * v;
        }
        const double u[3] = {j[0] / rho, j[1] / rho, j[2] / rho};
        acc.add(rho, u);
    }
    diag_block_store(acc, partials + (int64_t)blockIdx.x * lbmh::kDiagWords);
}

// Same fixed-order final pass as k_diag_finalize, writing the caller's 8 doubles.
__global__ void __launch_bounds__(256) k_noalloc_finalize(const double *partials, int blocks,
                                                         double *out) {
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
        // mass, momentum[3], kinetic, max_u, the non-finite count, 0
        for (int q = 0; q < 7; ++q) out[q] = red[0][q];
        out[7] = 0.0;
    }
}

}  // namespace lbmd

static int noalloc_fail(int code, const char *msg) { return lbmh::set_last_error(code, msg); }

extern "C" int lbm_diagnostics_noalloc(int lattice, const int64_t dims[3], const double *f,
                                       int64_t blocks, double *out, void *cuda_stream) {
    if (!dims || !f || !out) return noalloc_fail(LBM_EINVAL, "null argument");
    if (lattice != LBM_D2Q9 && lattice != LBM_D3Q27) return noalloc_fail(LBM_EINVAL, "bad lattice");
    for (int a = 0; a < 3; ++a)
        if (dims[a] < 1 || dims[a] > (1 << 30)) return noalloc_fail(LBM_EINVAL, "dims must be in [1, 2^30]");
    if (lattice == LBM_D2Q9 && dims[2] != 1) return noalloc_fail(LBM_EINVAL, "D2Q9 needs dims[2] == 1");
    // the same size limits as lbm_create: no int64 overflow of the cell count, at most 2^40 cells
    const int64_t xy = dims[0] * dims[1];
    if (xy / dims[0] != dims[1] || dims[2] > (((int64_t)1 << 40) / xy))
        return noalloc_fail(LBM_EINVAL, "lattice too large (more than 2^40 cells)");
    if (blocks < 1 || blocks > kNoAllocMaxBlocks)
        return noalloc_fail(LBM_EINVAL,
                            "blocks must be in [1, 1024]: the static scratch holds 1024 partial sums");
    const int64_t ncell = dims[0] * dims[1] * dims[2];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return noalloc_fail(LBM_ECUDA, "no current CUDA device");
    }
    double *scratch;
    {
        // First call on this device: look up the array's device address (no allocation).
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void *p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();
                return noalloc_fail(LBM_ECUDA, "cudaGetSymbolAddress of the static scratch failed");
            }
            g_noalloc_ptr[dev] = static_cast<double *>(p);
        }
        scratch = g_noalloc_ptr[dev];
    }
    // Every block writes its whole partial record before the final pass reads records
    // [0, blocks), so nothing in the shared scratch has to be cleared between calls.
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    if (lattice == LBM_D2Q9)
        lbmd::k_diag_canonical<2><<<(int)blocks, 256, 0, s>>>(f, ncell, scratch);
    else
        lbmd::k_diag_canonical<3><<<(int)blocks, 256, 0, s>>>(f, ncell, scratch);
    lbmd::k_noalloc_finalize<<<1, 256, 0, s>>>(scratch, (int)blocks, out);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return noalloc_fail(LBM_ECUDA, cudaGetErrorString(e));
    return LBM_OK;
}
