// k_tma_host.cu -- geometry and launch of the TMA row-staged step kernel.
#include "k_tma.cuh"

namespace lbmh {

#define LBM_DECL_CAP(d, c) const void *tma_kernel_d##d##_c##c(int P, int eq, int bulk);
LBM_DECL_CAP(2, 1024)
LBM_DECL_CAP(2, 2048)
LBM_DECL_CAP(2, 4096)
LBM_DECL_CAP(2, 8192)
LBM_DECL_CAP(3, 1024)
LBM_DECL_CAP(3, 2048)
LBM_DECL_CAP(3, 4096)
LBM_DECL_CAP(3, 8192)
#undef LBM_DECL_CAP

static const void *tma_kernel(const Lattice &lat, int eq, int bulk, int cap) {
    if (lat.D == 2) {
        switch (cap) {
        case 1024: return tma_kernel_d2_c1024(lat.P, eq, bulk);
        case 2048: return tma_kernel_d2_c2048(lat.P, eq, bulk);
        case 4096: return tma_kernel_d2_c4096(lat.P, eq, bulk);
        case 8192: return tma_kernel_d2_c8192(lat.P, eq, bulk);
        }
    } else {
        switch (cap) {
        case 1024: return tma_kernel_d3_c1024(lat.P, eq, bulk);
        case 2048: return tma_kernel_d3_c2048(lat.P, eq, bulk);
        case 4096: return tma_kernel_d3_c4096(lat.P, eq, bulk);
        case 8192: return tma_kernel_d3_c8192(lat.P, eq, bulk);
        }
    }
    return nullptr;
}

static int esize(int P) { return P == lbmd::P_F64 ? 8 : (P == lbmd::P_F32 ? 4 : 2); }

bool tma_supported(const Lattice &lat) {
    const int es = esize(lat.P);
    return ((int64_t)lat.nx * es) % 16 == 0 && (lat.plane * es) % 16 == 0 && lat.nx >= 16 / es;
}

static lbmd::TmaGeom geom(const Lattice &lat, const TmaShape &t) {
    const int U = 16 / esize(lat.P);
    lbmd::TmaGeom g;
    g.stages = t.stages;
    g.seg = t.seg >= lat.nx ? lat.nx : t.seg;
    g.nseg = (lat.nx + g.seg - 1) / g.seg;
    g.rows = g.nseg > 1 ? 1 : (t.rows < 1 ? 1 : (t.rows > lat.ny ? lat.ny : t.rows));
    g.ygroups = (lat.ny + g.rows - 1) / g.rows;
    g.halo = g.nseg > 1 ? U : 0;
    g.rowstride = g.seg + 2 * g.halo;
    g.bufstride = t.cap / esize(lat.P);
    g.njobs = (int64_t)lat.nz * g.ygroups * g.nseg;
    return g;
}

// Dynamic shared memory of a shape, or -1 when the shape is invalid: the segment must be
// a multiple of the 16-byte unit, the rows of a job must fit the direction buffer and
// the stage count must be in [2, 8].
int tma_thread_limit(const Lattice &lat) { return lbmd::tma_max_threads(lat.D, lat.P); }

int tma_smem_bytes(const Lattice &lat, const TmaShape &t) {
    const int U = 16 / esize(lat.P);
    if (t.stages < 2 || t.stages > kTmaMaxStages) return -1;
    if (t.cap != 1024 && t.cap != 2048 && t.cap != 4096 && t.cap != 8192) return -1;
    if (t.seg < lat.nx && (t.seg % U) != 0) return -1;
    const lbmd::TmaGeom g = geom(lat, t);
    if ((int64_t)g.rows * g.rowstride > g.bufstride) return -1;
    if (g.njobs >= ((int64_t)1 << 31)) return -1;
    if (t.threads < 32 || t.threads > lbmd::tma_max_threads(lat.D, lat.P) || t.threads % 32) return -1;
    const int64_t bytes = (int64_t)t.stages * lbmd::qof(lat.D) * t.cap;
    return bytes > 227 * 1024 ? -1 : (int)bytes;
}

cudaError_t tma_prepare(const Lattice &lat, int eq, int bulk, int cap, int smem_bytes) {
    const void *fn = tma_kernel(lat, eq, bulk, cap);
    if (!fn) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
}

int tma_max_blocks_per_sm(const Lattice &lat, int eq, int bulk, const TmaShape &t) {
    const void *fn = tma_kernel(lat, eq, bulk, t.cap);
    int n = 0;
    if (!fn) return 0;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, t.smem_bytes) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, t.threads + 32, t.smem_bytes) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

cudaError_t step_tma(const StepArgs &a, const TmaShape &t, cudaStream_t s) {
    const void *fn = tma_kernel(a.lat, a.eq, a.bulk, t.cap);
    if (!fn) return cudaErrorInvalidValue;
    lbmd::TmaGeom g = geom(a.lat, t);
    StepArgs aa = a;
    void *args[] = {(void *)&aa, (void *)&g};
    // t.threads consumer threads plus the producer warp
    return cudaLaunchKernel(fn, dim3(t.blocks), dim3(t.threads + 32), args, (size_t)t.smem_bytes, s);
}

}  // namespace lbmh
