// lbm_internal.h -- host-side launch interface between the C ABI (api.cu) and the
// kernel translation units.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lbmh {

// Layout of one lattice's populations: Q planes of `plane` elements (plane >= ncell,
// padded so that every plane starts on a 256-byte boundary), x fastest within a plane.
struct Lattice {
    void *A;
    int64_t plane;
    int nx, ny, nz;
    int64_t ncell;
    int D, P;  // dimension (2 or 3), storage precision (lbmd::P_*)
};

// Per-step arguments shared by every step kernel.
struct StepArgs {
    Lattice lat;
    int eq, bulk;
    double rho0, omega0, six_nu;  // reference density, 1/tau, 6 nu
    float rho0f, omega0f, six_nuf; // the same in single precision (FP32 collisions)
    int odd;                      // AA pattern: 0 = even step, 1 = odd step
    int diag;                     // 1 = reduce diagnostics into partials
    double *partials;             // [blocks][8] when diag
    int32_t *status;              // device status word (LBM_ETIMEOUT on a timed-out wait)
    int64_t timeout_ns;           // limit of every bounded device wait
};

// Launch shape of the TMA row-staged kernel.
struct TmaShape {
    int threads;    // consumer threads per block (one producer warp is added)
    int blocks;     // grid size (persistent blocks)
    int stages;     // shared-memory pipeline depth (>= 2)
    int rows;       // rows per job (>= 1; 1 when the row is split into segments)
    int seg;        // cells per row segment (== nx for whole rows)
    int cap;        // bytes per direction buffer in shared memory (1024, 2048, 4096, 8192)
    int smem_bytes; // dynamic shared memory per block
};

constexpr int kDiagWords = 8;  // mass, jx, jy, jz, kinetic, max|u|, nonfinite, unused
constexpr int kTmaMaxStages = 8;  // deepest shared-memory pipeline of the TMA row kernel

// api.cu: record the message of a failed call for lbm_last_error(); returns code.
int set_last_error(int code, const char *msg);

// k_generic.cu
cudaError_t step_generic(const StepArgs &a, int blocks, int threads, cudaStream_t s);
cudaError_t init_fields(const Lattice &lat, int eq, double rho0, const void *rho, const void *u,
                        int dtype, cudaStream_t s);
cudaError_t moments(const Lattice &lat, double rho0, int odd, void *rho, void *u, int dtype,
                    cudaStream_t s);
cudaError_t get_populations(const Lattice &lat, double rho0, int odd, void *f, int dtype,
                            cudaStream_t s);
cudaError_t set_populations(const Lattice &lat, double rho0, int odd, const void *f, int dtype,
                            cudaStream_t s);
cudaError_t sample_populations(const Lattice &lat, double rho0, int odd, const int64_t *cells,
                               int64_t count, double *out, cudaStream_t s);
cudaError_t diag_state(const Lattice &lat, double rho0, int odd, double *partials, int blocks,
                       cudaStream_t s);
cudaError_t diag_finalize(const double *partials, int blocks, int64_t step, double *record,
                          cudaStream_t s);
cudaError_t selftest_wait(int64_t timeout_ns, int32_t *status, cudaStream_t s);
int diag_blocks_generic(int64_t ncell);

// k_tma_*.cu
bool tma_supported(const Lattice &lat);
int tma_smem_bytes(const Lattice &lat, const TmaShape &t);
// Largest number of colliding threads per block of the TMA kernel for the lattice.
int tma_thread_limit(const Lattice &lat);
cudaError_t tma_prepare(const Lattice &lat, int eq, int bulk, int cap, int smem_bytes);
cudaError_t step_tma(const StepArgs &a, const TmaShape &t, cudaStream_t s);
int tma_max_blocks_per_sm(const Lattice &lat, int eq, int bulk, const TmaShape &t);

// k_batch.cu -- many independent lattices in one arena (FP64, shifted).  Instance k has
// ncell_k = cell_start[k + 1] - cell_start[k] cells; its populations are Q planes of
// ncell_k doubles starting at arena + Q * cell_start[k].
struct BatchArgs {
    double *arena;
    const int64_t *cell_start;   // [count + 1]
    const int32_t *dims;         // [count][3]
    const double *omega0;        // [count] 1/tau_k
    const double *six_nu;        // [count] 6 nu_k
    const int32_t *order;        // instance ids, grouped per block
    const int32_t *block_start;  // [blocks + 1] range of `order` owned by each block
    const double2 *twiddle;      // exp(-i 2 pi n_a x_a / N_a) per instance, [Nx | Ny | Nz]
    const int64_t *tw_offset;    // [count] offset of instance k's twiddles
    double *series;              // [count][max_samples][8] (re, im of rho, jx, jy, jz)
    int64_t max_samples;
    int32_t *status;             // [count] 0, or first non-finite probed step + 1
    int64_t count;
    int D, eq, bulk;
    double rho0;
    int64_t step0, nsteps, every_k;  // first step, steps in this launch, probe period (0 = off)
};
cudaError_t step_batch(const BatchArgs &a, int blocks, int threads, cudaStream_t s);
const void *batch_kernel(int D, int eq, int bulk);
cudaError_t batch_init(double *arena, const int64_t *cell_start, const int32_t *dims,
                       int64_t count, int D, int eq, double rho0, const void *rho, const void *u,
                       int dtype, int64_t total_cells, cudaStream_t s);
cudaError_t batch_moments(const double *arena, const int64_t *cell_start, const int32_t *dims,
                          int64_t count, int D, double rho0, int odd, void *rho, void *u,
                          int dtype, int64_t total_cells, cudaStream_t s);
cudaError_t batch_populations(const double *arena, const int64_t *cell_start,
                              const int32_t *dims, int64_t count, int D, double rho0, int odd,
                              void *f, int dtype, int64_t total_cells, cudaStream_t s);

// k_vn.cu
cudaError_t vn_eigs(int eq, int bulk, int64_t count, const double *params, double *out, int32_t *status,
                    cudaStream_t s);
cudaError_t vn_radius(int eq, int64_t npairs, const double *tau, const double *theta, const double *u_try, int nk,
                      unsigned long long *radius_bits, int32_t *status, cudaStream_t s);

}  // namespace lbmh
