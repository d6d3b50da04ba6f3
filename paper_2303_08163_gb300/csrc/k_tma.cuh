// k_tma.cuh -- the TMA row-staged fused stream-collide kernel (AA pattern, in place).
//
// A job is a group of `rows` consecutive x-rows of one z-plane, or one aligned segment
// of `seg` cells of a row when the row is too long for shared memory.  For every
// population direction b the job needs one row piece ("buffer b"):
//   even step: plane b of the job's own rows, read at x, written back as the opposite
//              direction's post-collision value at x;
//   odd step:  plane opp(b) of the rows shifted by -c_b in y and z; cell x reads it at
//              x - c_bx (pulling f_b from its neighbour) and the same cell writes its
//              post-collision value of direction opp(b) there.
// Every position of buffer b is read by exactly one cell of the job and written by the
// same cell (the AA pattern's own property), so the collision runs in place in shared
// memory and buffer b is stored back to exactly the global location it was loaded from.
// Different jobs touch disjoint global locations, so jobs need no ordering.
//
// Data movement (warp specialised): the last warp of the block is the producer, the
// others collide.  Lane b of the producer issues the cp.async.bulk copies of buffer b
// (global -> shared, completion counted in transaction bytes on the stage's `full`
// mbarrier) and later the cp.async.bulk stores of the same buffer (shared -> global) in
// its own bulk async-group, so each lane orders its own store before its own refill of
// that buffer.  Consumer warps wait on `full`, collide the job in place, fence their
// shared-memory writes for the async proxy and arrive on the stage's `empty` mbarrier;
// the producer then stores the stage back and refills it `stages` jobs ahead.  Rows must
// be 16-byte multiples (Nx * sizeof(storage) % 16 == 0).
//
// Segmented rows (seg < Nx) carry a halo of U = 16 / sizeof(storage) cells on each side.
// In the odd step the cells of a segment touch positions [X0 - 1, X0 + len - 1) of the
// buffers with c_x = +1 and [X0 + 1, X0 + len + 1) of those with c_x = -1: the aligned
// interior goes back by bulk stores and the U ragged cells at each end by plain stores,
// so neighbouring segments never write the same location.
#pragma once

#include "lbm_common.cuh"
#include "ptx.cuh"

namespace lbmd {

using lbmh::kTmaMaxStages;
constexpr int kTmaMaxThreads = 256;  // consumer threads of the D3Q27 kernels; one producer warp more
// D2Q9 binary16 kernels (under 100 registers) may run up to 512 consumers
__host__ __device__ constexpr int tma_max_threads(int D, int P) { return D == 2 && P == 2 ? 512 : kTmaMaxThreads; }

// bufstride (elements between direction buffers) equals the compile-time buffer
// capacity CAPB / sizeof(storage) of the kernel instantiation.
struct TmaGeom {
    int stages, rows, seg, nseg, ygroups, halo, rowstride, bufstride;
    int64_t njobs;
};

constexpr int kTmaCaps[4] = {1024, 2048, 4096, 8192};  // bytes per direction buffer

struct JobPos {
    int z, y0, nrows, X0, len;
};

__device__ __forceinline__ JobPos decode_job(const lbmh::StepArgs &a, const TmaGeom &g, int64_t job) {
    JobPos j;
    const unsigned jb = (unsigned)job;  // njobs < 2^31 (checked on the host)
    const unsigned rest = jb / (unsigned)g.nseg;
    const int s = (int)(jb - rest * (unsigned)g.nseg);
    const unsigned zq = rest / (unsigned)g.ygroups;
    const int yg = (int)(rest - zq * (unsigned)g.ygroups);
    j.z = (int)zq;
    j.y0 = yg * g.rows;
    j.nrows = min(g.rows, a.lat.ny - j.y0);
    j.X0 = s * g.seg;
    j.len = min(g.seg, a.lat.nx - j.X0);
    return j;
}

// Global row (plane, y, z) of buffer b of a job.
template <int D, typename T>
__device__ __forceinline__ T *buffer_row(const lbmh::StepArgs &a, int b, int z, int y) {
    constexpr int Q = qof(D);
    const int plane = a.odd ? Q - 1 - b : b;
    const int zz = (D == 3 && a.odd) ? wrapi(z - czo(b), a.lat.nz) : z;
    const int yy = a.odd ? wrapi(y - cyo(b), a.lat.ny) : y;
    return static_cast<T *>(a.lat.A) + (int64_t)plane * a.lat.plane +
           ((int64_t)zz * a.lat.ny + yy) * a.lat.nx;
}

// Bytes of one job's loads (all buffers), for the stage's expect-tx.
template <int D, typename T>
__device__ __forceinline__ uint32_t tma_job_bytes(const lbmh::StepArgs &a, const TmaGeom &g, const JobPos &j) {
    constexpr int Q = qof(D);
    constexpr int U = 16 / (int)sizeof(T);
    uint32_t bytes = (uint32_t)(Q * j.nrows * j.len * (int)sizeof(T));
    if (a.odd && g.nseg > 1) bytes += (uint32_t)((2 * Q / 3) * U * (int)sizeof(T));
    return bytes;
}

// Checked builds: a bulk copy of `bytes` between global `gp` and shared `sp` stays inside
// the population array and the stage, and meets the 16-byte rules of cp.async.bulk.
template <int D, typename T>
__device__ __forceinline__ bool bulk_ok(const lbmh::StepArgs &a, const TmaGeom &g, const T *stage,
                                        const T *sp, const T *gp, uint32_t bytes) {
#ifdef LBM_CHECKED
    constexpr int Q = qof(D);
    const T *A0 = static_cast<const T *>(a.lat.A);
    const int64_t n = (int64_t)bytes / (int64_t)sizeof(T);
    const bool ok = bytes > 0 && (bytes & 15u) == 0 && ((uintptr_t)gp & 15u) == 0 &&
                    (smem_u32(sp) & 15u) == 0 && gp >= A0 && gp + n <= A0 + (int64_t)Q * a.lat.plane &&
                    sp >= stage && sp + n <= stage + (int64_t)Q * g.bufstride;
    return LBM_CHECK(ok, a.status);
#else
    return true;
#endif
}

// Loads of buffer b of a job into its stage (issued by producer lane b).
template <int D, typename T>
__device__ __forceinline__ void tma_issue_loads(const lbmh::StepArgs &a, const TmaGeom &g,
                                                const JobPos &j, int b, T *st, uint64_t *bar) {
    constexpr int U = 16 / (int)sizeof(T);
    const int nx = a.lat.nx, ny = a.lat.ny;
    T *sbuf = st + (int64_t)b * g.bufstride;
    int r = 0;
    while (r < j.nrows) {
        const int ysrc = a.odd ? wrapi(j.y0 + r - cyo(b), ny) : j.y0 + r;
        const int run = min(j.nrows - r, ny - ysrc);
        const T *src = buffer_row<D, T>(a, b, j.z, j.y0 + r) + j.X0;
        T *dst = sbuf + r * g.rowstride + g.halo;
        const uint32_t bytes = (uint32_t)(run * j.len * (int)sizeof(T));
        if (bulk_ok<D, T>(a, g, st, dst, src, bytes)) bulk_g2s(dst, src, bytes, bar);
        r += run;
    }
    if (a.odd && g.nseg > 1) {
        const T *grow = buffer_row<D, T>(a, b, j.z, j.y0);
        if (cxo(b) == 1) {
            const int xs = j.X0 == 0 ? nx - U : j.X0 - U;
            if (bulk_ok<D, T>(a, g, st, sbuf, grow + xs, U * sizeof(T))) bulk_g2s(sbuf, grow + xs, U * sizeof(T), bar);
        } else if (cxo(b) == -1) {
            const int xs = (j.X0 + j.len == nx) ? 0 : j.X0 + j.len;
            T *dst = sbuf + g.halo + j.len;
            if (bulk_ok<D, T>(a, g, st, dst, grow + xs, U * sizeof(T))) bulk_g2s(dst, grow + xs, U * sizeof(T), bar);
        }
    }
}

// Stores of buffer b of a job back to global memory (issued by producer lane b).
template <int D, typename T>
__device__ __forceinline__ void tma_issue_stores(const lbmh::StepArgs &a, const TmaGeom &g,
                                                 const JobPos &j, int b, T *st) {
    constexpr int U = 16 / (int)sizeof(T);
    const int ny = a.lat.ny;
    T *sbuf = st + (int64_t)b * g.bufstride;
    if (!(a.odd && g.nseg > 1)) {
        int r = 0;
        while (r < j.nrows) {
            const int ysrc = a.odd ? wrapi(j.y0 + r - cyo(b), ny) : j.y0 + r;
            const int run = min(j.nrows - r, ny - ysrc);
            T *dst = buffer_row<D, T>(a, b, j.z, j.y0 + r) + j.X0;
            const T *src = sbuf + r * g.rowstride + g.halo;
            const uint32_t bytes = (uint32_t)(run * j.len * (int)sizeof(T));
            if (bulk_ok<D, T>(a, g, st, src, dst, bytes)) bulk_s2g(dst, src, bytes);
            r += run;
        }
    } else {
        T *grow = buffer_row<D, T>(a, b, j.z, j.y0);
        if (cxo(b) == 0) {
            const uint32_t bytes = (uint32_t)(j.len * (int)sizeof(T));
            if (bulk_ok<D, T>(a, g, st, sbuf + g.halo, grow + j.X0, bytes)) bulk_s2g(grow + j.X0, sbuf + g.halo, bytes);
        } else if (j.len > U) {
            const int off = cxo(b) == 1 ? 0 : U;  // skip the ragged end the plain stores take
            const uint32_t bytes = (uint32_t)((j.len - U) * (int)sizeof(T));
            if (bulk_ok<D, T>(a, g, st, sbuf + g.halo + off, grow + j.X0 + off, bytes))
                bulk_s2g(grow + j.X0 + off, sbuf + g.halo + off, bytes);
        }
    }
}

// Plain stores of the ragged ends of segmented odd steps (U cells per buffer with c_x != 0).
template <int D, typename T>
__device__ __forceinline__ void tma_plain_stores(const lbmh::StepArgs &a, const TmaGeom &g,
                                                 const JobPos &j, const T *st, int tid, int nthr) {
    constexpr int Q = qof(D);
    constexpr int U = 16 / (int)sizeof(T);
    constexpr int NB = 2 * Q / 3;
    const int nx = a.lat.nx;
    for (int t = tid; t < NB * U; t += nthr) {
        const int k = t / U, e = t - (t / U) * U;
        const int b = (k >> 1) * 3 + ((k & 1) ? 2 : 0);  // k-th direction with c_x != 0
        T *grow = buffer_row<D, T>(a, b, j.z, j.y0);
        const T *srow = st + (int64_t)b * g.bufstride;
        int gx, sx;
        if (cxo(b) == 1) {
            if (e == 0) { gx = j.X0 == 0 ? nx - 1 : j.X0 - 1; sx = g.halo - 1; }
            else { gx = j.X0 + j.len - U + e - 1; sx = g.halo + j.len - U + e - 1; }
        } else {
            if (e == 0) { gx = (j.X0 + j.len == nx) ? 0 : j.X0 + j.len; sx = g.halo + j.len; }
            else { gx = j.X0 + e; sx = g.halo + e; }
        }
        if (LBM_CHECK(gx >= 0 && gx < nx && sx >= 0 && sx < g.bufstride, a.status)) grow[gx] = srow[sx];
    }
}

// Shared-memory positions of one cell's populations (see the header comment): in the
// even step direction i is read at x and written (as direction opp(i)) at x; in the odd
// step it is read at x - c_ix and written at x + c_ix, wrapping inside a whole row.
struct CellPos {
    int row, x, xm, xp;
};

__device__ __forceinline__ CellPos cell_pos(const TmaGeom &g, int r, int xl, int len) {
    CellPos p;
    p.row = r * g.rowstride + g.halo;
    p.x = xl;
    p.xm = xl - 1;
    p.xp = xl + 1;
    if (g.nseg == 1) {
        p.xm = xl == 0 ? len - 1 : p.xm;
        p.xp = xl == len - 1 ? 0 : p.xp;
    }
    return p;
}

template <int D, int P, int CAPB>
__device__ __forceinline__ void tma_load_cell(const typename Storage<P>::T *st, const CellPos &p,
                                              int odd, typename Storage<P>::R (&f)[qof(D)]) {
    using St = Storage<P>;
    constexpr int bs = CAPB / (int)sizeof(typename St::T);  // compile-time offsets between buffers
    const typename St::T *row = st + p.row;
    if (!odd) {
#pragma unroll
        for (int i = 0; i < qof(D); ++i) f[i] = St::load(row[i * bs + p.x]);
    } else {
#pragma unroll
        for (int i = 0; i < qof(D); ++i) {
            const int x = cxo(i) == 1 ? p.xm : (cxo(i) == -1 ? p.xp : p.x);
            f[i] = St::load(row[i * bs + x]);
        }
    }
}

template <int D, int P, int CAPB>
__device__ __forceinline__ void tma_store_cell(typename Storage<P>::T *st, const CellPos &p, int odd,
                                               const typename Storage<P>::R (&f)[qof(D)]) {
    using St = Storage<P>;
    constexpr int Q = qof(D);
    constexpr int bs = CAPB / (int)sizeof(typename St::T);
    typename St::T *row = st + p.row;
    if (!odd) {
#pragma unroll
        for (int i = 0; i < Q; ++i) row[(Q - 1 - i) * bs + p.x] = St::store(f[i]);
    } else {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int x = cxo(i) == 1 ? p.xp : (cxo(i) == -1 ? p.xm : p.x);
            row[(Q - 1 - i) * bs + x] = St::store(f[i]);
        }
    }
}

// Collide every cell of a job in place in its stage, one cell per thread per iteration.
template <int D, int P, int EQ, bool BULK, int CAPB>
__device__ __forceinline__ void tma_compute(const lbmh::StepArgs &a, const TmaGeom &g,
                                            const JobPos &j, typename Storage<P>::T *st,
                                            DiagAcc &acc, int tid, int nthr) {
    using St = Storage<P>;
    using R = typename St::R;
    constexpr int Q = qof(D);
    const R rho0 = step_scalar<R>(a.rho0, a.rho0f), omega0 = step_scalar<R>(a.omega0, a.omega0f),
            six_nu = step_scalar<R>(a.six_nu, a.six_nuf);
    const int ncells = j.nrows * j.len;
    DiagLocal<R> loc;
    int r = tid / j.len;
    int xl = tid - r * j.len;
    for (int c = tid; c < ncells; c += nthr) {
        const CellPos p = cell_pos(g, r, xl, j.len);
        // checked builds: every position the cell touches lies inside its direction buffer
        if (LBM_CHECK(p.row + min(p.xm, p.x) >= 0 && p.row + max(p.xp, p.x) < g.bufstride, a.status)) {
            R f[Q];
            tma_load_cell<D, P, CAPB>(st, p, a.odd, f);
            const CellMoments<R> m = collide<D, EQ, BULK, R, relax_two_fma<D, P>()>(f, rho0, omega0, six_nu);
            tma_store_cell<D, P, CAPB>(st, p, a.odd, f);
            if (a.diag) loc.add(m.rho, m.u, rho0);
        }
        xl += nthr;
        while (xl >= j.len) {
            xl -= j.len;
            ++r;
        }
    }
    if (a.diag) loc.flush(acc, a.rho0);
}

// binary16 storage: the same collision, two neighbouring cells per thread per iteration,
// so that every buffer position pair the two cells own at an even offset moves as one
// 32-bit shared-memory access and one paired conversion.  Even step: cells (x, x + 1),
// x even, own the pair at x in every buffer.  Odd step, whole rows: cells (x, x + 1), x
// odd (the last pair is (len - 1, 0)), own the pairs at x - 1 and x + 1 in the buffers
// with c_x != 0; the c_x = 0 buffers go one half at a time.  Odd step, segments (no wrap
// inside the job): cells (x, x + 1), x even, own the pair at x in the c_x = 0 buffers and
// go one half at a time elsewhere.  The conversions round exactly as the one-cell path
// does, so the stored state is the same bit for bit.
__device__ __forceinline__ float2 ld_pair(const __half *b, int p) {
    return __half22float2(*reinterpret_cast<const __half2 *>(b + p));
}
__device__ __forceinline__ void st_pair(__half *b, int p, float lo, float hi) {
    *reinterpret_cast<__half2 *>(b + p) = __floats2half2_rn(lo, hi);
}

// MODE 0: even step; 1: odd step, whole rows; 2: odd step, segments; -1: chosen at run
// time from the step parity and the job layout (one loop body for all three).
template <int D, int EQ, bool BULK, int CAPB, int MODE>
__device__ __forceinline__ void tma_compute_pairs(const lbmh::StepArgs &a, const TmaGeom &g,
                                                  const JobPos &j, __half *st, DiagAcc &acc,
                                                  int tid, int nthr) {
    constexpr int Q = qof(D);
    constexpr int bs = CAPB / 2;  // halves between direction buffers
    const int mode = MODE >= 0 ? MODE : (!a.odd ? 0 : (g.nseg == 1 ? 1 : 2));
    const float rho0 = a.rho0f, omega0 = a.omega0f, six_nu = a.six_nuf;
    const int hl = j.len >> 1;  // len is a multiple of 8 cells (16-byte rows)
    const int npairs = j.nrows * hl;
    DiagLocal<float> loc;
    int r = tid / hl;
    int xh = tid - r * hl;
    for (int c = tid; c < npairs; c += nthr) {
        __half *row = st + r * g.rowstride + g.halo;
        // cells xa and xb = xa + 1 (the odd pairing of whole rows wraps its last pair to
        // cell 0); pm = xa - 1 and pp = xb + 1 are the outer neighbours, inside the row for
        // whole rows (xa >= 1 in the odd pairing) and in the halos for segments
        const int xa = 2 * xh + (mode == 1 ? 1 : 0);
        const int xb = (mode == 1 && xa + 1 == j.len) ? 0 : xa + 1;
        const int pm = xa - 1;
        const int pp = xb + 1;
        // checked builds: every position the pair touches lies inside its direction buffer
        const int row_off = r * g.rowstride + g.halo;
        const int lo = mode == 0 ? xa : min(min(pm, xa), xb);
        const int hi = mode == 0 ? xa + 1 : max(max(xb + 1, pp), xa);
        if (LBM_CHECK(row_off + lo >= 0 && row_off + hi < bs, a.status)) {
            float fa[Q], fb[Q];
            if (mode == 0) {
    #pragma unroll
                for (int i = 0; i < Q; ++i) {
                    const float2 v = ld_pair(row + i * bs, xa);
                    fa[i] = v.x;
                    fb[i] = v.y;
                }
            } else if (mode == 1) {
    #pragma unroll
                for (int i = 0; i < Q; ++i) {
                    const __half *b = row + i * bs;
                    if (cxo(i) == 0) {
                        fa[i] = __half2float(b[xa]);
                        fb[i] = __half2float(b[xb]);
                    } else {
                        const float2 v = ld_pair(b, cxo(i) == 1 ? pm : xb);
                        fa[i] = v.x;
                        fb[i] = v.y;
                    }
                }
            } else {
    #pragma unroll
                for (int i = 0; i < Q; ++i) {
                    const __half *b = row + i * bs;
                    if (cxo(i) == 0) {
                        const float2 v = ld_pair(b, xa);
                        fa[i] = v.x;
                        fb[i] = v.y;
                    } else if (cxo(i) == 1) {
                        fa[i] = __half2float(b[pm]);
                        fb[i] = __half2float(b[xa]);
                    } else {
                        fa[i] = __half2float(b[xb]);
                        fb[i] = __half2float(b[pp]);
                    }
                }
            }
            const CellMoments<float> ma = collide<D, EQ, BULK, float, relax_two_fma<D, P_F16S>()>(fa, rho0, omega0, six_nu);
            const CellMoments<float> mb = collide<D, EQ, BULK, float, relax_two_fma<D, P_F16S>()>(fb, rho0, omega0, six_nu);
            if (mode == 0) {
    #pragma unroll
                for (int i = 0; i < Q; ++i) st_pair(row + (Q - 1 - i) * bs, xa, fa[i], fb[i]);
            } else if (mode == 1) {
    #pragma unroll
                for (int i = 0; i < Q; ++i) {
                    __half *b = row + (Q - 1 - i) * bs;
                    if (cxo(i) == 0) {
                        b[xa] = __float2half_rn(fa[i]);
                        b[xb] = __float2half_rn(fb[i]);
                    } else {
                        st_pair(b, cxo(i) == 1 ? xb : pm, fa[i], fb[i]);
                    }
                }
            } else {
    #pragma unroll
                for (int i = 0; i < Q; ++i) {
                    __half *b = row + (Q - 1 - i) * bs;
                    if (cxo(i) == 0) {
                        st_pair(b, xa, fa[i], fb[i]);
                    } else if (cxo(i) == 1) {
                        b[xb] = __float2half_rn(fa[i]);
                        b[pp] = __float2half_rn(fb[i]);
                    } else {
                        b[pm] = __float2half_rn(fa[i]);
                        b[xa] = __float2half_rn(fb[i]);
                    }
                }
            }
            if (a.diag) {
                loc.add(ma.rho, ma.u, rho0);
                loc.add(mb.rho, mb.u, rho0);
            }
        }
        xh += nthr;
        while (xh >= hl) {
            xh -= hl;
            ++r;
        }
    }
    if (a.diag) loc.flush(acc, a.rho0);
}

template <int D, int P, int EQ, bool BULK, int CAPB>
__global__ void __launch_bounds__(tma_max_threads(D, P) + 32) k_step_tma(const lbmh::StepArgs a, const TmaGeom g) {
    using T = typename Storage<P>::T;
    constexpr int Q = qof(D);
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full[kTmaMaxStages];
    __shared__ __align__(8) uint64_t empty[kTmaMaxStages];
    T *sm = reinterpret_cast<T *>(smem_raw);
    const int64_t stage_elems = (int64_t)Q * (CAPB / (int)sizeof(T));
    const int S = g.stages;
    const int64_t G = gridDim.x;
    const int ncons = (int)blockDim.x - 32;  // consumer threads; the last warp produces
    const int lane = threadIdx.x & 31;
    const bool producer = (int)threadIdx.x >= ncons;
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], ncons / 32);
        }
        fence_barrier_init();
    }
    __syncthreads();
    DiagAcc acc;
    bool failed = false;
    if (producer) {
        int64_t k = 0;
        for (;; ++k) {
            const int64_t job = blockIdx.x + k * G;
            if (job >= g.njobs) break;
            const int s = (int)(k % S);
            const JobPos jp = decode_job(a, g, job);
            if (k >= S) {
                // stage s still holds job k - S: wait for its collision, store it back
                const int64_t q = k - S;
                const bool ok = mbar_wait_bounded(&empty[s], (uint32_t)((q / S) & 1), a.timeout_ns);
                if (__any_sync(0xffffffffu, !ok)) {
                    failed = true;
                    break;
                }
                const JobPos jq = decode_job(a, g, blockIdx.x + q * G);
                if (a.odd && g.nseg > 1) {
                    tma_plain_stores<D, T>(a, g, jq, sm + s * stage_elems, lane, 32);
                    __syncwarp();  // every lane's plain stores read the stage before any refill
                }
                if (lane == 0) mbar_arrive_expect_tx(&full[s], tma_job_bytes<D, T>(a, g, jp));
                if (lane < Q) {
                    // each lane stores its direction's buffer, waits until that store has
                    // read shared memory, and refills the same buffer; lanes do not wait
                    // for one another (the stage's phase completes once all bytes land)
                    tma_issue_stores<D, T>(a, g, jq, lane, sm + s * stage_elems);
                    bulk_commit();
                    bulk_wait_read<0>();
                    tma_issue_loads<D, T>(a, g, jp, lane, sm + s * stage_elems, &full[s]);
                }
            } else {
                if (lane == 0) mbar_arrive_expect_tx(&full[s], tma_job_bytes<D, T>(a, g, jp));
                if (lane < Q) tma_issue_loads<D, T>(a, g, jp, lane, sm + s * stage_elems, &full[s]);
            }
        }
        const int64_t issued = k;
        if (!failed) {
            // store back the last stages
            for (int64_t q = (issued > S ? issued - S : 0); q < issued; ++q) {
                const int s = (int)(q % S);
                const bool ok = mbar_wait_bounded(&empty[s], (uint32_t)((q / S) & 1), a.timeout_ns);
                if (__any_sync(0xffffffffu, !ok)) {
                    failed = true;
                    break;
                }
                const JobPos jq = decode_job(a, g, blockIdx.x + q * G);
                if (a.odd && g.nseg > 1) tma_plain_stores<D, T>(a, g, jq, sm + s * stage_elems, lane, 32);
                if (lane < Q) {
                    tma_issue_stores<D, T>(a, g, jq, lane, sm + s * stage_elems);
                    bulk_commit();
                }
            }
        }
        bulk_wait_all();
        if (failed) {
            // let loads still in flight land before the block's shared memory is released
            for (int64_t q = (issued > S ? issued - S : 0); q < issued; ++q)
                (void)mbar_wait_bounded(&full[q % S], (uint32_t)((q / S) & 1), a.timeout_ns);
        }
    } else {
        for (int64_t k = 0;; ++k) {
            const int64_t job = blockIdx.x + k * G;
            if (job >= g.njobs) break;
            const int s = (int)(k % S);
            const bool ok = mbar_wait_bounded(&full[s], (uint32_t)((k / S) & 1), a.timeout_ns);
            if (__any_sync(0xffffffffu, !ok)) {
                failed = true;
                break;
            }
            T *st = sm + s * stage_elems;
            const JobPos jp = decode_job(a, g, job);
            if constexpr (P == P_F16S && D == 3) {
                // the D3Q27 pair body is long: one copy serves the three pairings (three
                // specialised copies measured slower)
                tma_compute_pairs<D, EQ, BULK, CAPB, -1>(a, g, jp, st, acc, threadIdx.x, ncons);
            } else if constexpr (P == P_F16S) {
                if (!a.odd)
                    tma_compute_pairs<D, EQ, BULK, CAPB, 0>(a, g, jp, st, acc, threadIdx.x, ncons);
                else if (g.nseg == 1)
                    tma_compute_pairs<D, EQ, BULK, CAPB, 1>(a, g, jp, st, acc, threadIdx.x, ncons);
                else
                    tma_compute_pairs<D, EQ, BULK, CAPB, 2>(a, g, jp, st, acc, threadIdx.x, ncons);
            } else
                tma_compute<D, P, EQ, BULK, CAPB>(a, g, jp, st, acc, threadIdx.x, ncons);
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive_cta(&empty[s]);
        }
    }
    if (failed && lane == 0) report_status(a.status, -5); /* LBM_ETIMEOUT */
    if (a.diag) diag_block_store(acc, a.partials + (int64_t)blockIdx.x * lbmh::kDiagWords);
}

template <int D, int P, int CAPB>
const void *tma_kernel_dpc(int eq, int bulk) {
    if (eq == EQ_ENT) return bulk ? (const void *)k_step_tma<D, P, EQ_ENT, true, CAPB> : (const void *)k_step_tma<D, P, EQ_ENT, false, CAPB>;
    if (eq == EQ_POLY2) return bulk ? (const void *)k_step_tma<D, P, EQ_POLY2, true, CAPB> : (const void *)k_step_tma<D, P, EQ_POLY2, false, CAPB>;
    if (eq == EQ_PROD) return bulk ? (const void *)k_step_tma<D, P, EQ_PROD, true, CAPB> : (const void *)k_step_tma<D, P, EQ_PROD, false, CAPB>;
    return nullptr;
}

template <int D, int CAPB>
const void *tma_kernel_dc(int P, int eq, int bulk) {
    switch (P) {
    case P_F64: return tma_kernel_dpc<D, P_F64, CAPB>(eq, bulk);
    case P_F32: return tma_kernel_dpc<D, P_F32, CAPB>(eq, bulk);
    case P_F16S: return tma_kernel_dpc<D, P_F16S, CAPB>(eq, bulk);
    default: return nullptr;
    }
}

}  // namespace lbmd
