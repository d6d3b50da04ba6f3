/*
 * lbm.h -- C ABI of the GB300 (sm_103a) lattice-BGK library with the entropic
 * equilibrium of Hosseini & Karlin, arXiv 2303.08163.
 *
 * The library advances periodic D2Q9 / D3Q27 lattices by the lattice-BGK evolution
 * equation (Eq. 1 of the paper):
 *
 *     f_i(r + c_i dt, t + dt) - f_i(r, t) = 2 beta (f_i^eq(rho, u) - f_i(r, t)),
 *
 * one collide-then-stream step per call unit, with
 *   - the entropic equilibrium (Eq. eq:Entropic_isothermal_EDF),
 *     f_i^eq = w_i rho prod_a (2 - S_a) Z_a^{c_ia},  S_a = sqrt(1 + 3 u_a^2),
 *     Z_a = (2 u_a + S_a) / (1 - u_a), in lattice units (dr = dt = 1, vs^2 = 1/3);
 *   - the quadratic polynomial equilibrium (Eq. eq:Poly2_isothermal_EDF) or the product
 *     form (Eq. eq:Product_isothermal_EDF) as comparison paths;
 *   - 2 beta = 1 / tau (Eq. eq:relaxation_frequency with nu = (tau - 1/2) / 3), or the
 *     local bulk-viscosity correction beta = 1 / (2 nu / (A vs^2) + 1) of Eq.
 *     (eq:redefined_relaxation rate), A = min_a A(u_a) from Eq. (eq:entropic_bulk) for
 *     the entropic equilibrium and Eq. (eq:LBGK_bulk) for the others.
 *
 * Conventions used by every entry point
 * -------------------------------------
 * Population index: i = (c_x + 1) + 3 (c_y + 1) + 9 (c_z + 1), Q = 9 or 27; the
 *   opposite direction of i is Q - 1 - i.  Weights are products of the D1Q3 weights
 *   {1/6, 2/3, 1/6} (Sec. II).
 * Cell index: x fastest, idx = x + Nx (y + Ny z).  dims = {Nx, Ny, Nz}; Nz = 1 for D2Q9.
 * Field buffers: rho[ncell]; u[D][ncell] (structure of arrays).
 * Population buffers: f[Q][ncell] (structure of arrays), canonical meaning: the
 *   post-stream, pre-collision populations f_i(r, t) at the current step t.
 * Storage: populations live in device memory owned by the library, as shifted values
 *   f_i - w_i rho0 in FP64, FP32 or IEEE binary16 (round-to-nearest-even); the collision
 *   runs in FP64 for FP64 storage and in FP32 otherwise.
 * dtype arguments: LBM_DT_F64 (double) or LBM_DT_F32 (float) for caller buffers;
 *   population calls also take LBM_DT_STORAGE (exact checkpoint of the stored values).
 * on_device: 0 = caller pointer is host memory (pageable or pinned), 1 = device memory
 *   on the context's device.  Page-locked host buffers (cudaHostAlloc, cudaHostRegister)
 *   of the field calls are read or written by the kernels directly across the CPU-GPU
 *   link; pageable ones go through a device staging buffer.  The results are the same.
 * Ownership: the library owns its objects and all device memory it allocates; caller
 *   buffers are borrowed for the duration of the call only.
 * Streams: every call is ordered on the stream given at creation (NULL = legacy default
 *   stream).  Calls that return data in host memory synchronise that stream first.
 * Errors: every int-returning call returns LBM_OK (0) or a negative status code.  The
 *   message of the last failure on the calling thread is returned by lbm_last_error().
 *   LBM_ECUDA, LBM_ETIMEOUT and LBM_ENOMEM are sticky: the object refuses further work
 *   (LBM_ESTATE) until destroyed.  A step kernel whose bounded wait ran out records
 *   LBM_ETIMEOUT in the object's device status word; every call that synchronises (lbm_sync,
 *   lbm_diagnostics, lbm_diag_history, lbm_step with diagnostics, and the calls that return
 *   data in host memory) reads that word and returns the error.  Calls that only enqueue
 *   work (lbm_step without diagnostics, device-memory outputs) do not synchronise, so the
 *   error surfaces at the next synchronising call.
 * Threads: an object may be used by one host thread at a time.
 */
#ifndef LBM_H
#define LBM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx;     /* one periodic lattice (opaque, library-owned) */
typedef struct lbm_batch lbm_batch; /* many independent small lattices (opaque) */

enum lbm_lattice { LBM_D2Q9 = 0, LBM_D3Q27 = 1 };

enum lbm_eq_kind {
    LBM_EQ_ENTROPIC = 0, /* Eq. eq:Entropic_isothermal_EDF */
    LBM_EQ_POLY2 = 1,    /* Eq. eq:Poly2_isothermal_EDF */
    LBM_EQ_PRODUCT = 2   /* Eq. eq:Product_isothermal_EDF */
};

enum lbm_precision {
    LBM_F64 = 0, /* FP64 storage, FP64 collision */
    LBM_F32 = 1, /* FP32 storage of f - w rho0, FP32 collision */
    LBM_F16S = 2 /* binary16 storage of f - w rho0 (RN-even), FP32 collision */
};

enum lbm_dtype {
    LBM_DT_F64 = 0,    /* double */
    LBM_DT_F32 = 1,    /* float */
    LBM_DT_STORAGE = 2 /* populations only: the stored shifted values f - w rho0 in the
                          storage type (double, float or binary16), bit for bit */
};

enum lbm_status {
    LBM_OK = 0,
    LBM_EINVAL = -1,     /* invalid argument (bad enum, size, tau <= 1/2, null pointer) */
    LBM_ENOMEM = -2,     /* device or host allocation failed */
    LBM_ECUDA = -3,      /* a CUDA runtime call or kernel launch failed */
    LBM_ENONFINITE = -4, /* fused diagnostics saw a non-finite mass or momentum */
    LBM_ETIMEOUT = -5,   /* a bounded device wait ran out; the kernel returned early */
    LBM_ESTATE = -6,     /* object is in an error state or the call is out of order */
    LBM_ECHECK = -7      /* checked builds only (compiled with -DLBM_CHECKED): a device-side
                            bounds or alignment check failed and the access was skipped */
};

/* Options for lbm_set_option. */
enum lbm_option {
    LBM_OPT_DIAG_EVERY = 0, /* fused diagnostics every K steps (0 = off, the default) */
    LBM_OPT_KERNEL = 1,     /* 0 = auto, 1 = generic one-cell-per-thread kernel,
                               2 = TMA row-staged kernel (needs Nx * sizeof % 16 == 0) */
    LBM_OPT_USE_GRAPH = 2,  /* 1 = replay steps from a captured CUDA graph (default 0) */
    LBM_OPT_TUNE = 3        /* 1 = time the candidate launch shapes now and keep the best */
};

/* Global diagnostics of one state (FP64, deterministic fixed-order reduction). */
typedef struct {
    double mass;        /* sum rho */
    double momentum[3]; /* sum rho u_a */
    double kinetic;     /* sum rho |u|^2 / 2 */
    double max_u;       /* max over cells and axes of |u_a| */
    int64_t step;       /* time step t of the state the values describe */
    int64_t nonfinite;  /* number of cells whose rho or u was not finite */
} lbm_diag;

/* ------------------------------------------------------------------------------------
 * Single lattice
 * ------------------------------------------------------------------------------------ */

/*
 * Create a periodic lattice of dims[0] x dims[1] x dims[2] cells.
 *   lattice    LBM_D2Q9 (dims[2] must be 1) or LBM_D3Q27.
 *   tau        relaxation time, 2 beta = 1 / tau, nu = (tau - 1/2) / 3 (Sec. II);
 *              must be > 1/2 (beta in (0, 1)).
 *   eq_kind    lbm_eq_kind.  bulk_corr: 0 or 1 (Sec. V.B local correction).
 *   precision  lbm_precision.  rho0: reference density of the shifted storage.
 *   cuda_stream  a cudaStream_t (or NULL) on which all work of this object is ordered.
 * Allocates Q * ncell populations in device memory (zero = the rest state rho = rho0,
 * u = 0).  Returns LBM_EINVAL for bad arguments, LBM_ENOMEM if allocation fails.
 */
int lbm_create(lbm_ctx **out, int lattice, const int64_t dims[3], double tau, int eq_kind,
               int bulk_corr, int precision, double rho0, void *cuda_stream);

/*
 * Set an lbm_option.  LBM_OPT_TUNE times every candidate launch shape on a proxy lattice
 * with the same row geometry (the same Nx, and Ny for D3Q27) and at most 2 GiB of
 * populations in whole z-planes (y-rows for D2Q9), filled from the current state's first
 * planes; the context's own state is not touched.  It keeps the fastest shape (among
 * shapes within 0.5 % of it, the one with the least shared memory, then the fewest stages
 * and threads), remembers it for lattices of the same kind and size (and in the file named
 * by the environment variable LBM_TUNE_CACHE, if set; a remembered shape is checked
 * against the lattice and the device before it is used).  A candidate whose bounded wait
 * ran out is discarded.  Returns LBM_ENOMEM, with the context still usable, if the proxy
 * cannot be allocated.
 */
int lbm_set_option(lbm_ctx *ctx, int option, int64_t value);

/*
 * Set the state to f = f^eq(rho, u) of the context's equilibrium (step counter = 0).
 * rho: [ncell], u: [D][ncell] in dtype, host or device memory.
 */
int lbm_init_fields(lbm_ctx *ctx, const void *rho, const void *u, int dtype, int on_device);

/*
 * Advance n >= 0 time steps of Eq. (1).  Each step is one launch of the fused
 * stream-collide kernel (AA pattern, in place).  When LBM_OPT_DIAG_EVERY = K > 0 the
 * step kernels of steps t with t % K == 0 also reduce the diagnostics of state t; the
 * call then synchronises and returns LBM_ENONFINITE if any of them saw a non-finite
 * cell (the state is kept for inspection).
 */
int lbm_step(lbm_ctx *ctx, int64_t n);

/* rho [ncell] and u [D][ncell] of the current state, in dtype, host or device memory. */
int lbm_moments(lbm_ctx *ctx, void *rho, void *u, int dtype, int on_device);

/* Diagnostics of the current state (synchronises). */
int lbm_diagnostics(lbm_ctx *ctx, lbm_diag *out);

/*
 * Fused diagnostics recorded by lbm_step since the last lbm_init_fields or
 * lbm_set_populations (oldest first, at most the last 65536).  Copies up to max
 * records to out and stores the number available in *count (synchronises).
 */
int lbm_diag_history(lbm_ctx *ctx, lbm_diag *out, int64_t max, int64_t *count);

/* Canonical populations f[Q][ncell] of the current state: not shifted for LBM_DT_F64 and
 * LBM_DT_F32, the stored shifted values for LBM_DT_STORAGE. */
int lbm_get_populations(lbm_ctx *ctx, void *f, int dtype, int on_device);

/* Replace the current state with canonical populations f[Q][ncell] (same dtype meaning
 * as lbm_get_populations); the step counter is kept.  A checkpoint that resumes bit for
 * bit is (lbm_get_populations(LBM_DT_STORAGE), lbm_step_count). */
int lbm_set_populations(lbm_ctx *ctx, const void *f, int dtype, int on_device);

/* Set the step counter t.  The stored layout depends on the parity of t, so a change of
 * parity moves the current state into the new layout (the state is unchanged).  To resume a
 * checkpoint: lbm_set_step_count(t), then lbm_set_populations(f). */
int lbm_set_step_count(lbm_ctx *ctx, int64_t step);

/*
 * Canonical populations (FP64, not shifted) of count sampled cells.
 * cells: host array of count cell indices idx = x + Nx (y + Ny z);
 * out: host array [count][Q].  Synchronises.
 */
int lbm_sample_populations(lbm_ctx *ctx, const int64_t *cells, int64_t count, double *out);

/* Current step counter t. */
int lbm_step_count(lbm_ctx *ctx, int64_t *out);

/*
 * Launch shape of the step kernel chosen for this context: out[0] = kernel (1 generic,
 * 2 TMA row-staged), out[1] = threads per block, out[2] = blocks, out[3] = pipeline
 * stages, out[4] = rows per job, out[5] = cells per row segment, out[6] = dynamic
 * shared memory bytes, out[7] = population storage bytes.
 */
int lbm_launch_info(lbm_ctx *ctx, int64_t out[8]);

/*
 * Choose the step kernel's launch shape explicitly.  shape = {kernel, threads, stages,
 * rows, seg, cap}: kernel 1 = generic (threads per block, the rest ignored), 2 = TMA
 * row-staged with `threads` colliding threads per block (a multiple of 32, at most 256,
 * 512 for D2Q9 with binary16 storage; one copy-issuing warp is added), `stages`
 * shared-memory stages (2..8), `rows` rows per job when whole rows fit, `seg` cells per
 * row segment (seg >= Nx for whole rows; otherwise a multiple of 16 / sizeof(storage), and
 * never below it) and `cap` bytes per direction buffer (1024, 2048, 4096 or 8192).  The
 * one-cell kernel takes at most 256 threads.  The block count is the largest that fits on
 * the device.  Returns LBM_EINVAL for a negative entry, an entry above INT32_MAX, or a
 * shape the lattice or the device cannot run.
 */
int lbm_set_launch_shape(lbm_ctx *ctx, const int64_t shape[6]);

/* Wait for all work of the object's stream; returns a sticky error if one occurred. */
int lbm_sync(lbm_ctx *ctx);

/* Free the object and its device memory (synchronises its stream).  NULL is allowed. */
void lbm_destroy(lbm_ctx *ctx);

/* ------------------------------------------------------------------------------------
 * Batch of independent periodic lattices (the linear-mode sweep of Sec. V)
 * ------------------------------------------------------------------------------------ */

/*
 * Create count independent periodic lattices of one lattice type and equilibrium, with
 * per-instance sizes dims[count][3] (int32, host) and relaxation times tau[count]
 * (host).  Storage is FP64 (precision must be LBM_F64) packed in one arena in instance
 * order, each instance structure-of-arrays.
 */
int lbm_batch_create(lbm_batch **out, int lattice, int64_t count, const int32_t *dims,
                     const double *tau, int eq_kind, int bulk_corr, int precision, double rho0,
                     void *cuda_stream);

/* f = f^eq(rho, u) for every instance; rho and u packed in instance order, each
 * instance's u as [D][ncell_k]; step counter = 0. */
int lbm_batch_init_fields(lbm_batch *b, const void *rho, const void *u, int dtype,
                          int on_device);

/*
 * Record, at every step t with t % every_k == 0 (t counted from the last init), the
 * Fourier projections sum_r q(r) exp(-i k.r) of q = rho, j_x, j_y, j_z (FP64, j = rho u)
 * of the state at t, for the per-instance wave vector
 * k = 2 pi (kvec[k][0] / Nx, kvec[k][1] / Ny, kvec[k][2] / Nz).
 * kvec: host int32 [count][3].  every_k >= 1.
 */
int lbm_batch_set_probe(lbm_batch *b, const int32_t *kvec, int64_t every_k);

/* Advance every instance by n steps in one persistent kernel launch, replayed from a
 * captured CUDA graph. */
int lbm_batch_step(lbm_batch *b, int64_t n);

/*
 * Copy the probe series to host: out[count][max_samples][4][2] (re, im of rho, j_x, j_y,
 * j_z); *nsamples receives the number of samples recorded so far (synchronises).  Pass
 * out = NULL to query *nsamples only.
 */
int lbm_batch_probe_series(lbm_batch *b, double *out, int64_t max_samples, int64_t *nsamples);

/* Per-instance status, host int32 [count]: 0 = finite so far, s + 1 = the first probed
 * step s at which the instance's mass or momentum was not finite (synchronises). */
int lbm_batch_status(lbm_batch *b, int32_t *status);

/* rho and u of every instance (packed as in lbm_batch_init_fields). */
int lbm_batch_moments(lbm_batch *b, void *rho, void *u, int dtype, int on_device);

/* Canonical populations of every instance, packed in instance order as [Q][ncell_k]. */
int lbm_batch_get_populations(lbm_batch *b, void *f, int dtype, int on_device);

/* Number of cells of all instances together, and the current step counter. */
int lbm_batch_info(lbm_batch *b, int64_t *total_cells, int64_t *step);

/* Launch shape of the batched kernel: out[0] = threads per block, out[1] = blocks,
 * out[2] = largest per-block cell load, out[3] = mean per-block cell load. */
int lbm_batch_launch_info(lbm_batch *b, int64_t out[4]);

/*
 * Choose the batched kernel's launch shape: `threads` per block (a multiple of 32 in
 * [32, 256]) and `blocks` (1 .. min(count, 32 x the SM count)).  Instances are
 * re-assigned to the blocks longest-first (each to the least-loaded block so far); a
 * block owns whole instances, so blocks never wait for one another and more blocks than
 * fit on the GPU at once simply run in waves.  Returns LBM_EINVAL for other values.
 */
int lbm_batch_set_launch_shape(lbm_batch *b, int threads, int64_t blocks);

/*
 * Launch-shape autotuner of the batched kernel: times `steps` steps (1 .. 100000) of the
 * current state under each candidate shape (64, 128 or 256 threads; 1, 2, 3, 4, 6, 8, 12
 * or 16 blocks per SM), twice, and keeps the fastest (among shapes within 0.5 % of it, the
 * one with the fewest blocks, then threads).  The state, the step counter and the status
 * are restored afterwards, so the call changes only the launch shape; the probes of the
 * timed steps are written to samples that the next lbm_batch_step rewrites.  Needs one
 * temporary copy of the state (Q x total cells doubles): LBM_ENOMEM, with the object
 * still usable, if it cannot be allocated.  Synchronises.
 */
int lbm_batch_autotune(lbm_batch *b, int64_t steps);

int lbm_batch_sync(lbm_batch *b);
void lbm_batch_destroy(lbm_batch *b);

/* ------------------------------------------------------------------------------------
 * Linear stability (von Neumann analysis of the D2Q9 scheme, Sec. V.A)
 * ------------------------------------------------------------------------------------ */

/*
 * Eigenvalues of the amplification matrix M = E (delta + J) of Eq. (eq:VN_eigen) for count
 * parameter points, computed on the GPU in FP64 (one point per thread).  J = 2 beta
 * (d f^eq / d f - I) is the Jacobian of the collision operator at f = f^eq(rho, u), with
 * the exact derivatives of the eq_kind equilibrium; E_ij = exp(-i c_i . k) delta_ij.
 * With bulk_corr = 1, 2 beta is the corrected rate of Eq. (eq:redefined_relaxation rate)
 * at u.  params: host [count][6] = {tau, rho, u_x, u_y, k_x, k_y}; out: host
 * [count][9][2] (re, im), each point's eigenvalues sorted by decreasing modulus.  A mode
 * exp(i (k.r - Omega t)) has lambda = exp(-i Omega): decay -ln|lambda| per step, phase
 * speed -arg(lambda) / |k|.  Synchronises.  LBM_ECUDA also when the QR iteration of some
 * point did not converge.
 */
int lbm_vn_eigenvalues(int eq_kind, int bulk_corr, int64_t count, const double *params, double *out,
                       void *cuda_stream);

/*
 * Linear-stability limit of Sec. V.A.2: for each of npairs (nu, theta) pairs, the largest
 * speed |u| in [0, u_hi] such that every eigenvalue of M has modulus <= 1 + tol for all
 * wave vectors of an nk x nk grid of [0, pi]^2, with u = |u| (cos theta, sin theta),
 * rho = 1 and tau = 1/2 + 3 nu (constant relaxation).  Found by `iterations` bisection
 * steps (stability is taken to hold below the limit); umax: host [npairs].
 * nu, theta: host [npairs].  Synchronises.
 */
int lbm_vn_stability_limit(int eq_kind, int64_t npairs, const double *nu, const double *theta, int nk,
                           double u_hi, int iterations, double tol, double *umax, void *cuda_stream);

/* ------------------------------------------------------------------------------------
 * Library
 * ------------------------------------------------------------------------------------ */

/* Message of the last failed call on this host thread ("" if none). */
const char *lbm_last_error(void);

/*
 * Global diagnostics of populations the caller owns, computed without allocating any
 * device memory.  The paper has no counterpart: this is a utility for callers that
 * cannot call cudaMalloc (code running inside another framework's memory pool, programs
 * that reserve all device memory up front, or work recorded inside a stream capture).
 *   lattice  LBM_D2Q9 (dims[2] == 1) or LBM_D3Q27.
 *   f        device pointer to canonical FP64 populations f[Q][ncell] (not shifted;
 *            population and cell order as above), read only.
 *   blocks   number of per-block partial sums, 1 <= blocks <= 1024.  The partial sums
 *            live in one static device array of 1024 records (64 KiB), which every
 *            device that loads the library holds until the process exits; larger values
 *            return LBM_EINVAL.
 *   out      device pointer to 8 doubles written on the stream: mass, momentum[3],
 *            kinetic, max |u_a|, number of non-finite cells, 0.
 *   cuda_stream  the stream the two kernels are ordered on (NULL = legacy stream).
 * The call does not synchronise.  Its first call on a device looks up the static
 * array's device address for that device (the device current at the call), so make the
 * first call on each device before any stream capture.  All calls share the one static
 * array: calls whose kernels overlap on the GPU (different streams, or host threads
 * without ordering between them) race and corrupt each other's results; order them on
 * one stream.  Every call rewrites the records it reads, so no clearing is needed.
 */
int lbm_diagnostics_noalloc(int lattice, const int64_t dims[3], const double *f, int64_t blocks,
                            double *out, void *cuda_stream);

/* Library version as major * 10000 + minor * 100 + patch. */
int lbm_version(void);

/*
 * Self-test of the bounded device wait used by every kernel that waits on a shared
 * memory barrier: launches one block that waits on an mbarrier nothing arrives on,
 * with a limit of timeout_ns nanoseconds.  *status_out receives LBM_ETIMEOUT when the
 * wait ran out as it should, LBM_OK if it completed.  Synchronises the stream.
 */
int lbm_selftest_bounded_wait(void *cuda_stream, int64_t timeout_ns, int32_t *status_out);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
