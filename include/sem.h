/*
 * sem.h -- C-ABI of the GB300 spectral-element Poisson library (libsem.so).
 *
 * The library implements the hot path of the Nekbone/Neko-style SEM Poisson
 * solve studied in "Enabling mixed-precision in spectral element codes"
 * (arXiv 2503.02134):
 *   - the matrix-free element operator w_L = sum_a D_a^T (sum_b G_ab D_b u_L)
 *     (Sec. 3.1, profiling table, kernel `ax`: local_grad3, geometric
 *     factors, local_grad3_t);
 *   - the direct-stiffness summation Sigma' = Q Q^T over shared GLL nodes
 *     (Sec. 3.3, "Global communication and gather-scatter modes");
 *   - the Jacobi preconditioner z = J^{-1} r, J^{-1} = 1/diag(A) (Sec. 4.3);
 *   - the preconditioned CG loop of the profiling table, in FP64 and in the
 *     paper's mixed strategy (FP32 loop operations, FP64 gather-scatter
 *     accumulation and FP64 dot products; Sec. 3.3 and 4.3, Table
 *     "Evaluation of mixed-precision strategies in Neko"), plus an FP64
 *     residual / iterative-refinement outer loop.
 *
 * Conventions shared by every entry point
 *   - Vectors are LOCAL (unassembled) vectors of L = E*(N+1)^3 values,
 *     element-major; inside an element, node (i,j,k) is at i + n*j + n*n*k
 *     with n = N+1 (i runs along the reference direction r).
 *   - Pointers may be device pointers (cudaMalloc, PyTorch CUDA tensors) or
 *     host pointers; host buffers are staged through device buffers owned by
 *     the handle (copies are enqueued on the handle's stream).  The caller
 *     owns every pointer it passes; the library never frees them.
 *   - All device work is enqueued on the stream given to sem_setup.  Calls
 *     that return scalars (solve info) synchronise that stream.
 *   - Return codes: 0 ok; negative = error (SEM_EINVAL -1 invalid argument,
 *     SEM_ECUDA -2 CUDA error or no device, SEM_ENOMEM -3 out of device
 *     memory, SEM_ETIMEOUT -4 a bounded device wait gave up); positive =
 *     non-fatal solver outcome (SEM_MAXIT 1 maxit reached before tol,
 *     SEM_STAGNATED 2 stagnation not cured by refinement, SEM_BREAKDOWN 3
 *     p.Ap <= 0 or non-finite).  sem_last_error() returns the message of the
 *     last failing call on the calling thread.  There is no CPU fallback.
 */
#ifndef SEM_H_
#define SEM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  SEM_OK = 0,
  SEM_EINVAL = -1,
  SEM_ECUDA = -2,
  SEM_ENOMEM = -3,
  SEM_ETIMEOUT = -4,
  SEM_MAXIT = 1,
  SEM_STAGNATED = 2,
  SEM_BREAKDOWN = 3
};

/* Arithmetic of a call (vector dtype at the boundary in brackets).
 *  SEM_FP64        everything in FP64                         [double]
 *  SEM_MIXED_FP32  FP32 operator / vectors / updates, FP64 gather-scatter
 *                  accumulation, FP64-quality dots and scalars (the paper's
 *                  converging strategy)                        [float]
 *  SEM_MIXED_TF32  as MIXED_FP32 with the D-contractions on tensor cores in
 *                  TF32 (FP32 accumulate)                      [float]
 *  SEM_MIXED_BF16X3 as MIXED_FP32 with the D-contractions as three BF16
 *                  products hi*hi + hi*lo + lo*hi, FP32 accumulate  [float]
 *  SEM_FP32_ALL    everything FP32, including gather-scatter accumulation
 *                  and dot products (the paper's stagnating strategy) [float]
 * sem_pcg_solve takes FP64 f/x0/x for every precision. */
typedef enum {
  SEM_FP64 = 0,
  SEM_MIXED_FP32 = 1,
  SEM_MIXED_TF32 = 2,
  SEM_MIXED_BF16X3 = 3,
  SEM_FP32_ALL = 4
} sem_precision;

typedef struct sem_handle_s* sem_handle;

/* Mesh description.  With gid == NULL the mesh is the kx*ky*kz box on
 * [lo, hi] (element e = ex + kx*(ey + ky*ez)), numbered on its
 * (kx N+1)(ky N+1)(kz N+1) grid of GLL points, Dirichlet on all six faces,
 * optionally deformed (deform_kind 1: x += a sin(2 pi y) sin(2 pi z) and
 * cyclic permutations, evaluated from the undeformed coordinates at every
 * GLL node).  With gid != NULL the caller gives a general conforming hex
 * mesh: gid (host, E*n^3 ids in [0, 2^31)), coords (host, 3*E*n^3 doubles,
 * x block then y then z, local layout), and dirichlet_faces (host, E bytes;
 * bit f set = face f of the element is Dirichlet, faces ordered
 * r=-1, r=+1, s=-1, s=+1, t=-1, t=+1).  E = kx*ky*kz in both cases. */
typedef struct {
  int kx, ky, kz;
  double lo[3], hi[3];
  double deform_amp;
  int deform_kind;
  const int64_t* gid;
  const double* coords;
  const uint8_t* dirichlet_faces;
} sem_mesh;

typedef struct {
  int N, n;
  int64_t E, L, U;       /* elements, local DOFs, unique global nodes */
  int64_t n_shared;      /* local entries with multiplicity > 1 */
  int64_t n_segments;    /* global nodes with multiplicity > 1 */
  int64_t device_bytes;  /* device memory held by the handle */
} sem_sizes;

typedef struct {
  int iters;             /* PCG iterations (inner iterations summed) */
  int refinements;       /* FP64 residual replacements (mode 0) or restarts (mode 1) */
  int status;            /* 0, SEM_MAXIT, SEM_STAGNATED or SEM_BREAKDOWN */
  double relres;         /* final recursive ||r||_c/||b||_c of the last (inner) solve, relative to b */
  double relres_true;    /* ||b - A x||_c/||b||_c recomputed in FP64 */
  double solve_ms;       /* device time of the solve (CUDA events) */
  int64_t launches;      /* kernels this solve launched (graph nodes counted) */
} sem_info;

/* Solver options (sem_pcg_solve_ex).  Zero-initialised fields take defaults. */
typedef struct {
  double tol;            /* relative residual ||r||_c/||b||_c target (default 1e-8) */
  int maxit;             /* iteration cap over all inner solves (default 1000) */
  sem_precision precision;
  int fixed_iters;       /* > 0: run exactly this many iterations, no convergence test */
  int no_refine;         /* mixed only: 1 = one inner solve, no FP64 outer loop */
  double inner_tol;      /* mixed only: per-cycle residual reduction floor (default 1e-5) */
  int max_cycles;        /* mixed only: FP64 outer cycles cap (default 20) */
  int use_graph;         /* 0 (default) or 1: replay iteration chunks as CUDA graphs; -1: plain launches */
  int chunk;             /* iterations per convergence poll (default 32) */
  int precond;           /* 1 Jacobi (default), -1 identity, 2 multigrid (sem_mg_apply's
                            V-cycle; FP64, or mixed: reliable updates as for Jacobi,
                            refine_mode 1 restarts FP32 inner solves whose residual
                            reduction is inner_tol, default 1e-4) */
  double* history;       /* optional host array of maxit+1 recursive residuals (or NULL) */
  int refine_mode;       /* mixed only: 0 reliable updates (default): the FP64 true residual
                            replaces the FP32 one each time it fell by replace_factor, CG
                            continues with the same search direction; 1 restarted refinement:
                            a new inner solve of A d = r64 per FP64 cycle */
  double replace_factor; /* mixed, refine_mode 0: residual drop between replacements (1e-2) */
} sem_solve_opts;

/* Set up a problem: GLL nodes/weights and the derivative matrix
 * (textbook GLL rule the paper's SEM relies on, Sec. 3 and its reference
 * Deville-Fischer-Mund), node coordinates, geometric factors G1..G6 and
 * mass B (FP64, with an FP32 copy), the gather-scatter map (sorted
 * shared-node segments), multiplicities, the Dirichlet mask and the Jacobi
 * diagonal (FP64, with a one-time FP32 copy, Sec. 4.3).  N in [1, 15].
 * stream: a cudaStream_t (NULL = legacy default stream).
 * geom_flags: reserved, pass 0.  On success *out owns all device memory. */
int sem_setup(const sem_mesh* mesh, int N, int geom_flags, void* stream, sem_handle* out);
void sem_destroy(sem_handle h);
const char* sem_last_error(void);
int sem_get_sizes(sem_handle h, sem_sizes* out);

/* w = mask * QQ^T (A_L u): the assembled, masked SEM Laplacian applied to a
 * local vector (profiling table, `ax`, including the gather-scatter and the
 * Dirichlet mask).  u, w: L values of the precision's dtype; may not alias. */
int sem_ax(sem_handle h, const void* u, void* w, sem_precision p);

/* w_L = mask * A_L u: the element operator only (no gather-scatter). */
int sem_ax_local(sem_handle h, const void* u, void* w, sem_precision p);

/* v = QQ^T v in place (direct-stiffness summation, Sec. 3.3).  FP64 and the
 * mixed precisions accumulate every shared-node sum in FP64; SEM_FP32_ALL
 * accumulates in FP32.  Every copy receives the same rounded sum. */
int sem_gs(sem_handle h, void* v, sem_precision p);

/* Weighted inner product sum_i a_i c_i b_i with c = mask/multiplicity
 * (glsc3 of the profiling table).  a, b: L values of the precision's dtype.
 * FP64 reduction for every precision except SEM_FP32_ALL. */
int sem_glsc3(sem_handle h, const void* a, const void* b, sem_precision p, double* out);

/* Copy an internal field to `out` (L doubles unless stated):
 * 0 G (6*L, per element [6][n^3]), 1 B (mass), 2 Jacobi inverse J^{-1},
 * 3 multiplicity, 4 mask, 5 c = mask/multiplicity, 6 coordinates (3*L,
 * x block, y block, z block), 7 GLL nodes (n), 8 GLL weights (n),
 * 9 derivative matrix D (n*n, row-major D[i][j] = l_j'(xi_i)),
 * 10 Jacobian determinant. */
int sem_get_field(sem_handle h, int which, double* out);

/* Right-hand sides (FP64, L values, masked, continuous):
 * kind 0: b = mask QQ^T(B * 3 pi^2 sin(pi x) sin(pi y) sin(pi z));
 * kind 1: b_g uniform in [-1,1) per global node g from SplitMix64 output
 *         number g+1 of state `seed` (Steele-Lea-Flood 2014), masked. */
int sem_rhs(sem_handle h, int kind, uint64_t seed, double* b);

/* Random Fourier right-hand side b = mask QQ^T(B f) (FP64, L values):
 * f = sum over k in {1..8}^3 of a_k sin(pi k1 x) sin(pi k2 y) sin(pi k3 z),
 * a_k = xi_k / |k|^2, xi_k uniform in [-1,1) from SplitMix64 output number
 * sample*512 + (k1-1) + 8(k2-1) + 64(k3-1) + 1 of state `seed`.  Training
 * and test data of the learned initial guess. */
int sem_rhs_fourier(sem_handle h, uint64_t seed, uint64_t sample, double* b);

/* Jacobi PCG for A x = f (f assembled and masked, FP64).  x0 may be NULL
 * (zero initial guess).  x receives the FP64 solution.  Stopping test:
 * recursive ||r||_c/||b||_c <= tol (FP64 path) or the FP64 true residual
 * <= tol (mixed path with refinement). */
int sem_pcg_solve(sem_handle h, const double* f, const double* x0, double* x,
                  double tol, int maxit, sem_precision p, sem_info* info);
int sem_pcg_solve_ex(sem_handle h, const double* f, const double* x0, double* x,
                     const sem_solve_opts* opts, sem_info* info);

/* ---- Learned initial guess (the paper has no learned component) ----
 * An element-local network (inputs: the element's b_L / s_e, the element
 * mean and standard deviation of G1..G6, the mean of b_L over each face
 * neighbour / s_e; s_e the RMS of b_L on the element; 530 inputs padded to
 * 544 -> hidden -> hidden -> n^3, ReLU) predicts u_L / (s_e t), t the RMS
 * of the training targets u_L / s_e; the guess is
 * x0 = c * QQ^T(s_e t y) (continuity projection, c = mask / multiplicity),
 * optionally scaled by the energy-optimal alpha = <b,c,x0>/<x0,c,A x0>,
 * which never increases the A-norm error over x0 = 0.  Box meshes only.
 * Weights: FP32 master + BF16 copies; products in BF16 with FP32
 * accumulation; Adam (lr as given, betas 0.9/0.999, eps 1e-8).
 * sem_x0_add_pair appends the E (features, x_L / s_e) rows of one solved
 * pair (b, x: device FP64 vectors) to the model's training set;
 * sem_x0_train runs `epochs` passes of shuffled mini-batches;
 * sem_x0_predict writes x0 (device FP64).  sem_x0_params gets (set = 0) or
 * sets (set = 1) the FP32 master parameters (host array laid out as
 * sem_x0_param_count's offsets: W1 [544 x H], b1, W2 [H x H], b2, W3 [H x n^3],
 * b3, row-major); sem_x0_gradients runs one forward/backward pass on `rows`
 * host rows (X: rows x 544, T: rows x n^3, FP32) in BF16 (bf16_mode = 1) or
 * FP32 arithmetic and returns the gradient of mean((y - T)^2) in the same
 * layout; sem_x0_features writes the FP32 features (E x 544) and scales.
 * The BF16 products run on the tcgen05 tensor cores (FP32 accumulator in
 * tensor memory; the FP32 gradient-check mode on the CUDA cores).
 * sem_x0_set_option keys:
 *   "umma"          1 (default): BF16 products by tcgen05.mma; 0: by the
 *                   warp-level mma.sync kernel (m16n8k16), for comparison
 *   "pair_rows"     element rows kept per training pair: a seeded random
 *                   subset (seed: the pair's index); 0 (default) keeps all E
 *   "reserve_rows"  allocate the training set for this many rows at once
 *   "coarse_cycles" c > 0: the features also carry a coarse approximation
 *                   of the solution, z = c FP32 multigrid-Richardson steps
 *                   (z += M^{-1}(b - A z) from 0, sem_mg_apply's V-cycle),
 *                   at the element's 8 vertices and its element mean, / s_e,
 *                   times 1 / (RMS of the first training pair's x_L / s_e),
 *                   a constant of the model that keeps them O(1) (inputs
 *                   539 of 544; fixed once pairs are stored)
 *   "post_cycles"   p > 0: sem_x0_predict ends with p steps
 *                   x0 += M^{-1}(b - A x0) (FP64 residual, FP32 V-cycle)
 * sem_x0_predict returns once x0 is written; its energy scaling runs on the
 * device (no host round trip). */
typedef struct sem_x0_model_s* sem_x0_model;
int sem_x0_create(sem_handle h, int hidden, uint64_t seed, sem_x0_model* out);
int sem_x0_param_count(sem_x0_model m, int64_t* sizes6, int64_t* offsets6);
int sem_x0_params(sem_x0_model m, float* host, int set);
int sem_x0_features(sem_x0_model m, const double* b, float* X, double* scale);
int sem_x0_gradients(sem_x0_model m, const float* X, const float* T, int rows, int bf16_mode,
                     float* grads, double* loss);
int sem_x0_add_pair(sem_x0_model m, const double* b, const double* x);
int sem_x0_train(sem_x0_model m, int epochs, int batch, float lr, uint64_t seed, double* final_loss);
int sem_x0_predict(sem_x0_model m, const double* b, double* x0, int energy_scale);
int sem_x0_set_option(sem_x0_model m, const char* key, int64_t value);
void sem_x0_destroy(sem_x0_model m);

/* ---- Batched solves: many independent problems of uneven E and N ----
 * sem_batch_setup builds one sub-handle per problem (meshes[i], Ns[i]; odd
 * N in 1..9), all on one stream, and the work lists of the batched kernels:
 * each phase of a PCG iteration (operator, gather-scatter, update + dots) is
 * ONE persistent launch over every problem's work items (for box-mesh
 * problems with N = 7 the gather-scatter is folded into the update, as with
 * the handle option "fuse_gs"), and chunks of
 * iterations are replayed as a CUDA graph.  A project autotuner picks the
 * operator's pipeline depth and grid at set-up.  The solve is the mixed
 * path with reliable updates (as sem_pcg_solve_ex, refine_mode 0), per
 * problem; f[i], x[i] are device pointers to problem i's FP64 vectors,
 * infos[i] receives problem i's outcome.  sem_batch_problem returns the
 * sub-handle of problem i (owned by the batch) for sem_rhs, sem_ax, ...
 * Returns the worst per-problem status (0 when all converged). */
typedef struct sem_batch_s* sem_batch;
int sem_batch_setup(const sem_mesh* meshes, const int* Ns, int count, void* stream,
                    sem_batch* out);
int sem_batch_problem(sem_batch b, int i, sem_handle* out);
int sem_batch_pcg_solve(sem_batch b, const double* const* f, double* const* x,
                        const sem_solve_opts* opts, sem_info* infos);
/* keys: "work_items", "launches", "fused_problems" (problems whose
 * gather-scatter is folded into the update), and per GLL points per direction n (2..10,
 * even): "variant_n<n>", "grid_n<n>" (autotuned launch), "tune_ms_n<n>_v<0..3>" */
int sem_batch_get_option(sem_batch b, const char* key, double* value);
void sem_batch_destroy(sem_batch b);

/* Allocation-free weighted dot product: *result = sum_i a_i c_i b_i over n
 * FP64 values, the same quantity as sem_glsc3 with the weights passed in.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory (no cudaMalloc allowed: an allocation-free
 * section of a host application, a sandbox with a fixed memory budget).  It
 * needs no handle and allocates nothing: its block partial sums live in a
 * static device array of 4096 doubles (32 KiB) that every GPU loading this
 * library holds until the process exits, so n may not exceed 33,554,432
 * (larger n returns SEM_EINVAL and changes nothing).  a, b, c: device
 * pointers to n doubles; result: device pointer to one double; stream: a
 * cudaStream_t (NULL = legacy default stream); the call is asynchronous.
 * The first call on a device looks up the array's device address on the
 * current device and keeps it for the life of the process; make that first
 * call before any stream capture.  The kept address belongs to the device's
 * context of that moment: after cudaDeviceReset the library's module may be
 * loaded at another address, so do not call this entry point on a device
 * after resetting it.  All calls
 * share the one array (the call zeroes its counter first), so calls that
 * overlap on the GPU -- on different streams, or from several threads --
 * race and must be serialised by the caller. */
int sem_glsc3_noalloc(const double* a, const double* b, const double* c, int64_t n,
                      double* result, void* stream);

/* Measured FMA throughput of the CUDA cores (the paper has no counterpart:
 * it is the roofline denominator of the compute-bound FP64 operator).
 * Launches, on the current device and the legacy default stream, 8 blocks
 * of 256 threads per SM, each thread running 8 independent FMA chains for
 * `iters` steps (a multiple of 4 is used), once to warm up and once timed
 * with CUDA events; *tflops = 2 * 8 * steps * threads / time.  fp64: 1 for
 * FP64 (DFMA), 0 for FP32 (FFMA).  Changes no clock or power setting.
 * Returns SEM_EINVAL for iters < 4 or a null result, SEM_ECUDA on a CUDA
 * error. */
int sem_fma_peak(int fp64, int iters, double* tflops);

/* Tuning knobs and diagnostics of the implementation (the paper has no
 * counterpart; they never change results beyond rounding).  Keys:
 *   "ax_variant", "ax_variant_pcg"  launch variant (0..4) of the bulk-copy
 *                                   staged FP32 operator, plain / PCG mode;
 *                                   sem_setup's autotuner picks the fastest
 *                                   (4: G in one buffer refilled after the
 *                                   geometric step, u or p_old in two, r and
 *                                   J^-1 in one refilled once p is formed;
 *                                   n = 6 .. 14 only).  A variant whose
 *                                   stages do not fit runs the unstaged kernel
 *   "ax_grid_cap" largest grid of the staged FP32 operator (0, the default:
 *                 resident blocks on every SM); a small cap makes every block
 *                 walk many element groups, so that small meshes go through
 *                 the stage reuse of the copy pipeline
 *   "use_tma"     1 (default) staged FP32 operator where it applies, 0 off
 *   "gs_acc"      mixed-path gather-scatter accumulation: 2 error-free
 *                 FP32 TwoSum (default), 0 FP64, 1 plain FP32
 *   "l2_persist"  1: during a mixed solve keep the operator output resident
 *                 in L2 (access-policy window on the handle's stream and a
 *                 persisting carve-out of the context, released at the end);
 *                 0 (default: measured no faster with the summation folded
 *                 into the update, slower with the separate pass)
 *   "l2_hints"    1: in FP32 PCG iterations the streamed vectors and G pass
 *                 through L2 with evict-first priority and the operator
 *                 output w is written evict-last (per-access cache hints),
 *                 instead of the access-policy window of "l2_persist";
 *                 0 (default) off
 *   "fuse_gs"     1 (default): in FP32 and mixed PCG iterations on a box mesh
 *                 (sem_setup without gid) with an even n the
 *                 direct-stiffness summation is folded into the vector update
 *                 -- each copy of a shared node gathers the others, found from
 *                 its position (whole rows of float4, or float2 pairs where n
 *                 is not a multiple of 4), in ascending local index with the
 *                 accumulation "gs_acc" selects, which gives the separate
 *                 pass's bits; 2: folded for odd n as well (node by node,
 *                 slower than the separate pass); 0: separate pass
 *   "upd_tma"     1: the folded update at N = 7 stages its streams in shared
 *                 memory by bulk copies (two stages, bounded waits) and reads
 *                 only the other copies of shared nodes directly; 0 (default) off
 *   "upd_variant" launch shape of the folded update kernel: register budget
 *                 for 0 (default) four, 1 five, 2 six 256-thread blocks per
 *                 SM; 3 four blocks and an L2 prefetch of each thread's next
 *                 float4 group; 4 four blocks with 64-bit indices; 5 five
 *                 blocks.  0 and 5 index in 32 bits where the vectors'
 *                 float4 indices fit in 31 bits (else 4 and 1)
 *   "mg_hcoarsen" 1 (default): the multigrid preconditioner continues below
 *                 its N = 1 level on halved meshes (see sem_mg_apply); 0:
 *                 orders only.  Changing it discards the built levels.
 *   "kernel_timing" 1: PCG solves run without graphs and time each
 *                 iteration's operator, gather-scatter and update launches
 *                 with CUDA events on the handle's stream (the events add
 *                 small gaps between launches); 0 (default) off.  Setting
 *                 it, either way, clears the sums.
 * sem_get_option also reads "ax_tune_ms_plain_<v>", "ax_tune_ms_pcg_<v>"
 * (autotuner timings, ms; -1 for a variant whose stages do not fit in shared
 * memory at this order), "launches" (kernels enqueued so far),
 * "mg_levels" (0 before the first multigrid use), "mg_omega_<l>" (damping of
 * level l, any number of digits; -1 for a level that does not exist),
 * "l2_window_bytes", "l2_max_persist", "l2_max_window" (the L2 window of
 * the last mixed solve and the device limits it was cut to),
 * "kt_iters" (iterations timed) and "kt_ms_ax", "kt_ms_gs",
 * "kt_ms_update" (average device time per launch, ms).
 * Unknown keys and out-of-range values return SEM_EINVAL. */
/* Multigrid preconditioner z = M^{-1} r (box meshes only).  The paper runs
 * Nekbone with its multigrid preconditioner (Sec. 3.1, profiling table;
 * Sec. 4, the Schwarz weights' square roots kept in FP64) without giving
 * its algorithm; this one is a symmetric V-cycle over orders N,
 * floor(N/2), ..., 1 on the same mesh (tensor-product interpolation between
 * orders) and then, with option "mg_hcoarsen" (default), over the N = 1
 * problem on the mesh halved in every direction while kx, ky, kz are even
 * and their halves at least 2 (trilinear interpolation between meshes);
 * restriction is the adjoint of interpolation on unique nodes; additive
 * overlapping Schwarz smoothing on every level (each element extended by
 * one node layer, separable local operator solved by fast diagonalisation,
 * weights 1/sqrt(blocks holding the node) computed in FP64, damping
 * 1/lambda_max from a power iteration); the coarsest level applies the
 * smoother only (no direct coarse solve).  r, z: L
 * device values, FP64 for SEM_FP64 or FP32 for SEM_MIXED_FP32 (the FP32
 * cycle sums shared nodes error-free); r continuous and masked.  Builds
 * the levels on first use (handles of their own, kept with this one). */
int sem_mg_apply(sem_handle h, const void* r, void* z, sem_precision p);

int sem_set_option(sem_handle h, const char* key, int64_t value);
int sem_get_option(sem_handle h, const char* key, double* value);

#ifdef __cplusplus
}
#endif
#endif /* SEM_H_ */
