// k_generic_step.cuh -- the generic fused stream-collide kernel: one cell per thread
// (grid-stride), populations read and written directly in global memory by the AA
// pattern.  Works for any lattice size and every storage precision; used for ragged
// sizes, for FP64 storage (bound by the FP64 pipe, not by memory) and as the fallback
// of the TMA row-staged kernel.
//
// AA pattern (in place, one array).  Even step: cell r reads its own slots A[i][r],
// collides, and writes f*_i to the opposite slot A[opp(i)][r].  Odd step: cell r reads
// f_i = A[opp(i)][r - c_i] (the value the neighbour r - c_i left for it), collides, and
// writes f*_i to A[i][r + c_i].  Every location is read and written by the same cell, so
// no two threads touch one location within a step.  Two steps together perform two
// collide-then-stream updates of Eq. (1).
#pragma once

#include "lbm_common.cuh"

namespace lbmd {

// One AA-pattern update of cell (x, y, z) of a lattice stored as Q planes of `plane`
// elements at A; returns the cell's pre-collision moments.
template <int D, int P, int EQ, bool BULK>
__device__ __forceinline__ CellMoments<typename Storage<P>::R> aa_cell_step(
    typename Storage<P>::T *__restrict__ A, int64_t plane, int nx, int ny, int nz, int x, int y,
    int z, int odd, typename Storage<P>::R rho0, typename Storage<P>::R omega0,
    typename Storage<P>::R six_nu, int32_t *status = nullptr) {
    using St = Storage<P>;
    using R = typename St::R;
    constexpr int Q = qof(D);
    // checked builds: the cell and (through the periodic wrap) all its neighbours lie
    // inside the lattice, so every index below stays inside the Q planes
    if (!LBM_CHECK(x >= 0 && x < nx && y >= 0 && y < ny && z >= 0 && z < nz &&
                       (int64_t)nx * ny * nz <= plane, status)) {
        CellMoments<R> none{};
        return none;
    }
    const int64_t cell = x + (int64_t)nx * (y + (int64_t)ny * z);
    const int xs[3] = {wrapi(x - 1, nx), x, wrapi(x + 1, nx)};
    const int ys[3] = {wrapi(y - 1, ny), y, wrapi(y + 1, ny)};
    const int zs[3] = {D == 3 ? wrapi(z - 1, nz) : z, z, D == 3 ? wrapi(z + 1, nz) : z};
    R f[Q];
    if (!odd) {
#pragma unroll
        for (int i = 0; i < Q; ++i) f[i] = St::load(A[(int64_t)i * plane + cell]);
    } else {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            // f_i(r) = A[opp(i)][r - c_i]
            const int64_t src = xs[1 - cxo(i)] +
                                (int64_t)nx * (ys[1 - cyo(i)] + (int64_t)ny * zs[1 - (D == 3 ? czo(i) : 0)]);
            f[i] = St::load(A[(int64_t)(Q - 1 - i) * plane + src]);
        }
    }
    const CellMoments<R> m = collide<D, EQ, BULK, R, relax_two_fma<D, P>()>(f, rho0, omega0, six_nu);
    if (!odd) {
#pragma unroll
        for (int i = 0; i < Q; ++i) A[(int64_t)(Q - 1 - i) * plane + cell] = St::store(f[i]);
    } else {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int64_t dst = xs[1 + cxo(i)] +
                                (int64_t)nx * (ys[1 + cyo(i)] + (int64_t)ny * zs[1 + (D == 3 ? czo(i) : 0)]);
            A[(int64_t)i * plane + dst] = St::store(f[i]);
        }
    }
    return m;
}

template <int D, int P, int EQ, bool BULK>
__global__ void __launch_bounds__(256) k_step_generic(const lbmh::StepArgs a) {
    using St = Storage<P>;
    using T = typename St::T;
    using R = typename St::R;
    T *__restrict__ A = static_cast<T *>(a.lat.A);
    const int nx = a.lat.nx, ny = a.lat.ny, nz = a.lat.nz;
    const R rho0 = step_scalar<R>(a.rho0, a.rho0f), omega0 = step_scalar<R>(a.omega0, a.omega0f),
            six_nu = step_scalar<R>(a.six_nu, a.six_nuf);
    DiagAcc acc;
    DiagLocal<R> loc;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const bool small = a.lat.ncell < ((int64_t)1 << 31);
    for (int64_t cell = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; cell < a.lat.ncell;
         cell += stride) {
        int x, y, z;
        if (small) {  // 32-bit index arithmetic
            const unsigned c = (unsigned)cell;
            const unsigned rowi = c / (unsigned)nx;
            x = (int)(c - rowi * (unsigned)nx);
            const unsigned zq = rowi / (unsigned)ny;
            y = (int)(rowi - zq * (unsigned)ny);
            z = (int)zq;
        } else {
            x = (int)(cell % nx);
            const int64_t rowi = cell / nx;
            y = (int)(rowi % ny);
            z = (int)(rowi / ny);
        }
        const CellMoments<R> m = aa_cell_step<D, P, EQ, BULK>(A, a.lat.plane, nx, ny, nz, x, y, z,
                                                              a.odd, rho0, omega0, six_nu, a.status);
        if (a.diag) {
            loc.add(m.rho, m.u, rho0);
            if (loc.count == 16) loc.flush(acc, a.rho0);
        }
    }
    if (a.diag) {
        loc.flush(acc, a.rho0);
        diag_block_store(acc, a.partials + (int64_t)blockIdx.x * lbmh::kDiagWords);
    }
}

template <int D, int P>
cudaError_t launch_generic_dp(const lbmh::StepArgs &a, int blocks, int threads, cudaStream_t s) {
#define LBM_GEN(EQv, Bv)                                                                   \
    if (a.eq == EQv && a.bulk == Bv) {                                                     \
        k_step_generic<D, P, EQv, Bv><<<blocks, threads, 0, s>>>(a);                        \
        return cudaGetLastError();                                                          \
    }
    LBM_GEN(EQ_ENT, false)
    LBM_GEN(EQ_ENT, true)
    LBM_GEN(EQ_POLY2, false)
    LBM_GEN(EQ_POLY2, true)
    LBM_GEN(EQ_PROD, false)
    LBM_GEN(EQ_PROD, true)
#undef LBM_GEN
    return cudaErrorInvalidValue;
}

}  // namespace lbmd
