// Internal declarations of libsem: the handle, device buffers and kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/sem.h"

namespace sem {

constexpr int kMaxN = 15;
constexpr int kTmaVariants = 5;   // launch variants of the bulk-copy staged FP32 operator
constexpr int kMaxn = kMaxN + 1;

// Per-iteration scalars of one PCG solve, resident on the device so that no
// host round trip sits between the kernels of an iteration.
struct PcgScalars {
  double rtz;        // <r, c, z> of the current iteration
  double rtz_old;    // previous rtz (beta = rtz / rtz_old)
  double pap;        // <p, c, A p>
  double rtr;        // <r, c, r>
  double alpha, beta;
  double bnorm;      // ||b||_c of the system being solved
  double tol;        // stop when sqrt(rtr)/bnorm <= tol
  double relres;     // last sqrt(rtr)/bnorm
  double best_rtr;   // stagnation watch: smallest rtr seen
  int best_it;       // iteration at which best_rtr was seen
  int iter;          // iterations done
  int maxit;         // iteration cap of this solve
  int fixed;         // 1: no convergence test
  int done;          // set once converged, capped, stagnated or broken down
  int status;        // 0 / SEM_MAXIT / SEM_STAGNATED / SEM_BREAKDOWN
  int stag_window;   // iterations without a 10% drop of ||r|| that mean stagnation (0 = off)
  int err;           // set by a kernel whose bounded wait gave up
  unsigned int counter[4];   // last-block election counters (reset by the last block)
  double hist_dummy;
};

// Where to write residual history (device array of maxit+1 doubles) or null.
struct MgData;

struct Handle {
  int N = 0, n = 0;
  int64_t E = 0, L = 0, U = 0;
  int kx = 0, ky = 0, kz = 0;
  bool gid_user = false;               // mesh numbered by the caller (no box structure)
  double mesh_lo[3] = {}, mesh_hi[3] = {};   // box mesh description (for multigrid levels)
  double deform_amp = 0.0;
  int deform_kind = 0;
  MgData* mg = nullptr;                // multigrid preconditioner, built on first use
  cudaStream_t stream = nullptr;       // internal work stream (never the legacy stream)
  cudaStream_t user_stream = nullptr;  // stream given to sem_setup
  bool own_stream = false;
  int num_sms = 0;
  int device = 0;

  // 1-D tables (FP64 master + FP32 copies)
  double* xi = nullptr;     // n
  double* wq = nullptr;     // n
  double* D64 = nullptr;    // n*n, D[i][j] row-major
  float* D32 = nullptr;
  float D32_host[kMaxn * kMaxn] = {};   // host copies of D32, D64 (kernel parameters by value)
  double D64_host[kMaxn * kMaxn] = {};

  // geometry
  double* coords = nullptr;  // 3*L
  double* G64 = nullptr;     // E*6*n^3
  float* G32 = nullptr;
  double* B64 = nullptr;     // L
  double* detJ = nullptr;    // L

  // connectivity
  int* gid = nullptr;          // L
  uint8_t* bfaces = nullptr;   // E (Dirichlet face bits)
  double* mask64 = nullptr;    // L
  double* mult64 = nullptr;    // L
  double* c64 = nullptr;       // L   mask / multiplicity
  float* c32 = nullptr;
  uint8_t* cw8 = nullptr;      // L: multiplicity on interior nodes, 0 on the Dirichlet boundary
  int* seg_off = nullptr;      // n_segments + 1
  int* perm = nullptr;         // n_shared local indices grouped by global node
  int64_t n_segments = 0, n_shared = 0;
  int* gs_slots = nullptr;     // bucketed, transposed copy indices (-1 = padding)
  int2* gs_chunks = nullptr;   // per 32-segment chunk: {copies m, first slot}
  int64_t n_chunks = 0, n_slots = 0;
  bool use_tma = true;         // FP32 operator: bulk-copy staged kernel where it applies
  int ax_grid_cap = 0;         // staged FP32 operator: largest grid (0: no cap)
  int ax_variant = 0;          // launch variant of the staged FP32 operator (plain / PCG mode)
  int ax_variant_pcg = 0;
  float ax_tune_ms[2][kTmaVariants] = {};  // autotuner timings [plain, PCG][variant]
  bool l2_persist = false;     // mixed solve: keep w resident in L2 (access-policy window)
  bool l2_hints = false;       // PCG kernels: per-access L2 eviction priorities keep w resident
  int64_t l2_window_bytes = 0;     // window of the last mixed solve (0: none set)
  int64_t l2_max_persist = 0, l2_max_window = 0;   // device limits read then
  int gs_acc = 2;              // mixed-path accumulation: 2 TwoSum (default), 0 FP64, 1 FP32
  int fuse_gs = 1;             // FP32 PCG on box meshes: summation folded into the update
                               // (1: n a multiple of 4, 2: every n, 0: never)
  int upd_gs_occ[24] = {};     // resident blocks per SM of the fused update kernels (0: not yet read)
  int upd_variant = 0;         // fused update launch shape (0..5, see pcg_kernels.cu UpdShape)
  bool upd_tma = false;        // fused update (n = 8): bulk-copy staged variant
  bool mg_hcoarsen = true;     // multigrid: h-levels below the N = 1 level

  // Jacobi
  double* minv64 = nullptr;
  float* minv32 = nullptr;

  // solver work space
  double *x64 = nullptr, *r64 = nullptr, *p64 = nullptr, *w64 = nullptr, *b64 = nullptr;
  float *x32 = nullptr, *r32 = nullptr, *p32 = nullptr, *w32 = nullptr, *b32 = nullptr;
  double* partials = nullptr;  // reduction partials (2 * max_blocks)
  int max_blocks = 0;
  PcgScalars* scal = nullptr;      // device, solver scalars
  PcgScalars* scal_aux = nullptr;  // device, scalars of residual checks / glsc3
  double* partials_aux = nullptr;  // reduction partials of residual checks / glsc3
  PcgScalars* scal_host = nullptr; // pinned host mirror
  double* dot_out = nullptr;       // device scalar of sem_glsc3
  double* hist_dev = nullptr;  // residual history (device), lazily sized
  int hist_cap = 0;

  // host staging
  void* stage_a = nullptr;     // device buffers of L doubles for host pointers
  void* stage_b = nullptr;
  void* stage_c = nullptr;

  int64_t device_bytes = 0;
  int* dev_err = nullptr;        // &scal->err: error word of the bounded device waits
  int64_t launches = 0;          // kernels enqueued (graph replays count their nodes)

  // graphs cache: one per (precision, chunk) combination
  cudaGraphExec_t graph_exec[8] = {};
  int graph_chunk[8] = {};
  int64_t graph_nodes[8] = {};

  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;

  // Per-kernel timing of PCG iterations (option "kernel_timing"): graphs
  // off, an event before and after each of the operator, gather-scatter and
  // update launches of every iteration of a chunk, read after the chunk.
  bool kernel_timing = false;
  std::vector<cudaEvent_t> kt_events;   // 4 per iteration of the current chunk
  int kt_recorded = 0;                  // iterations recorded in the current chunk
  double kt_ms[3] = {};                 // summed device time [operator, gs, update]
  int64_t kt_iters = 0;                 // iterations summed
};

// ------------------------------------------------------------------ errors
void set_error(const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

#define SEM_CUDA(call)                                  \
  do {                                                  \
    cudaError_t _e = (call);                            \
    if (_e != cudaSuccess) return ::sem::cuda_fail(_e, #call); \
  } while (0)

// Two timing events, destroyed when the scope ends (early error returns
// included).
struct ScopedEvents {
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t create() {
    cudaError_t e = cudaEventCreate(&a);
    return e == cudaSuccess ? cudaEventCreate(&b) : e;
  }
  ~ScopedEvents() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
};

// ------------------------------------------------------------------ launchers
// setup_kernels.cu
int launch_gll(Handle& h);
int launch_box_connectivity(Handle& h);
int launch_user_connectivity(Handle& h, const int64_t* gid_host, const uint8_t* faces_host);
int launch_geometry(Handle& h, const double* user_coords_dev, double amp, int deform_kind,
                    const double lo[3], const double hi[3]);
int launch_gs_map(Handle& h);
int launch_jacobi(Handle& h);
int launch_rhs(Handle& h, int kind, uint64_t seed, double* b);
int launch_rhs_fourier(Handle& h, uint64_t seed, uint64_t sample, double* b);

// ax_kernels.cu
// w = mask * A_L u (element operator, masked); optional PCG prologue/epilogue.
struct AxPrologue {
  // when r != nullptr: u := minv * r + beta * p_old, written to p (u is p)
  const void* r = nullptr;
  const void* minv = nullptr;
  const PcgScalars* scal = nullptr;
  // when pap_partials != nullptr: accumulate sum_l u_l w_l per block
  double* pap_partials = nullptr;
};
int launch_ax_local(Handle& h, sem_precision p, const void* u, void* w, const AxPrologue* pro);

int autotune_ax32(Handle& h);
bool ax32_variant_fits(int n, bool pcg, int v);   // staged FP32 operator variant fits in smem

// gs_kernels.cu
int launch_gs(Handle& h, sem_precision p, void* v);
int launch_gs_acc(Handle& h, sem_precision p, void* v, int acc);
int build_gs_buckets(Handle& h);

// pcg_kernels.cu
int launch_glsc3(Handle& h, sem_precision p, const void* a, const void* b, double* out_dev);

// solver.cu
int read_scalars(Handle& h, PcgScalars* dev, PcgScalars* out);
int fp64_residual(Handle& h, const double* f, bool x_is_zero, double* relres,
                  double* bnorm = nullptr);
int pcg_solve(Handle& h, const double* f, const double* x0, double* x, const sem_solve_opts& o,
              sem_info* info);

// helpers
inline int div_up(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }
bool is_device_ptr(const void* p);
int alloc(Handle& h, void** p, size_t bytes);
template <typename T>
int alloc_t(Handle& h, T** p, size_t count) {
  return alloc(h, reinterpret_cast<void**>(p), count * sizeof(T));
}

}  // namespace sem

// The opaque C handle is the internal handle.
struct sem_handle_s : public sem::Handle {};
