// C-ABI entry points of libsem (declared in include/sem.h).
#include <stdio.h>
#include <string.h>

#include <string>
#include <vector>

#include "pcg.cuh"

namespace sem {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

int cuda_fail(cudaError_t e, const char* what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  if (e == cudaErrorMemoryAllocation) return SEM_ENOMEM;
  return SEM_ECUDA;
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int alloc(Handle& h, void** p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    return cuda_fail(e, "cudaMalloc");
  }
  h.device_bytes += (int64_t)bytes;
  return 0;
}

void mg_free(Handle& h);
int mg_apply(Handle& h, sem_precision p, const void* r, void* z);
double mg_omega(Handle& h, int level);
int mg_levels(Handle& h);

static void free_handle(Handle* h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  for (int q = 0; q < 8; ++q)
    if (h->graph_exec[q]) cudaGraphExecDestroy(h->graph_exec[q]);
  void* ptrs[] = {h->xi,     h->wq,      h->D64,    h->D32,      h->coords,   h->G64,
                  h->G32,    h->B64,     h->detJ,   h->gid,      h->bfaces,   h->mask64,
                  h->mult64, h->c64,     h->c32, h->cw8,    h->seg_off,  h->perm, h->gs_slots, h->gs_chunks,     h->minv64,
                  h->minv32, h->x64,     h->r64,    h->p64,      h->w64,      h->x32,
                  h->r32,    h->p32,     h->w32,    h->b32,      h->partials, h->partials_aux,
                  h->scal,   h->scal_aux, h->dot_out, h->hist_dev, h->stage_a, h->stage_b,
                  h->stage_c};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (h->scal_host) cudaFreeHost(h->scal_host);
  if (h->ev0) cudaEventDestroy(h->ev0);
  if (h->ev1) cudaEventDestroy(h->ev1);
  if (h->ev_in) cudaEventDestroy(h->ev_in);
  if (h->ev_out) cudaEventDestroy(h->ev_out);
  for (cudaEvent_t e : h->kt_events) cudaEventDestroy(e);
  mg_free(*h);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete static_cast<sem_handle_s*>(h);
}

// Order the handle's work stream after the caller's stream (entry) and the
// caller's stream after the work stream (exit), so device pointers produced
// or consumed on the caller's stream see the right data.
struct StreamScope {
  Handle& h;
  bool ok = true;
  explicit StreamScope(Handle& hh) : h(hh) {
    if (h.own_stream) {
      if (cudaEventRecord(h.ev_in, h.user_stream) != cudaSuccess ||
          cudaStreamWaitEvent(h.stream, h.ev_in, 0) != cudaSuccess)
        ok = false;
    }
  }
  ~StreamScope() {
    if (h.own_stream) {
      cudaEventRecord(h.ev_out, h.stream);
      cudaStreamWaitEvent(h.user_stream, h.ev_out, 0);
    }
  }
};

// Device view of a caller pointer: device pointers pass through; host
// pointers are copied into a handle-owned staging buffer (when `in`).
static int stage_in(Handle& h, const void* p, size_t bytes, void* stage, const void** out) {
  if (!p) {
    *out = nullptr;
    return 0;
  }
  if (is_device_ptr(p)) {
    *out = p;
    return 0;
  }
  SEM_CUDA(cudaMemcpyAsync(stage, p, bytes, cudaMemcpyHostToDevice, h.stream));
  *out = stage;
  return 0;
}

static int ensure_stage(Handle& h) {
  int rc;
  if (!h.stage_a) {
    if ((rc = alloc(h, &h.stage_a, sizeof(double) * h.L))) return rc;
    if ((rc = alloc(h, &h.stage_b, sizeof(double) * h.L))) return rc;
    if ((rc = alloc(h, &h.stage_c, sizeof(double) * h.L))) return rc;
  }
  return 0;
}

static size_t elem_size(sem_precision p) { return p == SEM_FP64 ? 8 : 4; }

static bool valid_precision(sem_precision p) {
  return p == SEM_FP64 || p == SEM_MIXED_FP32 || p == SEM_MIXED_TF32 || p == SEM_MIXED_BF16X3 ||
         p == SEM_FP32_ALL;
}

}  // namespace sem

using namespace sem;

extern "C" {

const char* sem_last_error(void) { return g_last_error.c_str(); }

int sem_setup(const sem_mesh* mesh, int N, int geom_flags, void* stream, sem_handle* out) {
  (void)geom_flags;
  if (!mesh || !out) {
    set_error("sem_setup: null argument");
    return SEM_EINVAL;
  }
  *out = nullptr;
  if (N < 1 || N > kMaxN || mesh->kx < 1 || mesh->ky < 1 || mesh->kz < 1) {
    set_error("sem_setup: need 1 <= N <= 15 and kx, ky, kz >= 1");
    return SEM_EINVAL;
  }
  const int64_t n = N + 1;
  const int64_t E = (int64_t)mesh->kx * mesh->ky * mesh->kz;
  if (E * n * n * n >= ((int64_t)1 << 31)) {
    set_error("sem_setup: more than 2^31 local nodes");
    return SEM_EINVAL;
  }
  if (mesh->gid && !mesh->coords) {
    set_error("sem_setup: a user numbering (gid) needs user coordinates");
    return SEM_EINVAL;
  }
  int ndev = 0;
  cudaError_t ce = cudaGetDeviceCount(&ndev);
  if (ce != cudaSuccess || ndev == 0) {
    set_error("sem_setup: no CUDA device");
    return SEM_ECUDA;
  }
  sem_handle_s* h = new sem_handle_s();
  int rc = 0;
  auto fail = [&](int code) {
    free_handle(h);
    return code;
  };
  h->N = N;
  h->n = (int)n;
  h->E = E;
  h->L = E * n * n * n;
  h->kx = mesh->kx;
  h->ky = mesh->ky;
  h->kz = mesh->kz;
  h->user_stream = (cudaStream_t)stream;
  cudaGetDevice(&h->device);
  cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
  h->max_blocks = h->num_sms * 16;
  if (stream == nullptr) {
    if ((ce = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking)) != cudaSuccess)
      return fail(cuda_fail(ce, "cudaStreamCreate"));
    h->own_stream = true;
  } else {
    h->stream = (cudaStream_t)stream;
  }
  if ((ce = cudaEventCreate(&h->ev0)) != cudaSuccess || (ce = cudaEventCreate(&h->ev1)) != cudaSuccess ||
      (ce = cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming)) != cudaSuccess ||
      (ce = cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming)) != cudaSuccess)
    return fail(cuda_fail(ce, "cudaEventCreate"));
  if (h->own_stream) {
    // setup reads only host data, but order it after the caller's stream anyway
    if ((ce = cudaEventRecord(h->ev_in, h->user_stream)) != cudaSuccess ||
        (ce = cudaStreamWaitEvent(h->stream, h->ev_in, 0)) != cudaSuccess)
      return fail(cuda_fail(ce, "cudaStreamWaitEvent"));
  }

  const size_t L = (size_t)h->L;
  if ((rc = alloc_t(*h, &h->xi, n)) || (rc = alloc_t(*h, &h->wq, n)) ||
      (rc = alloc_t(*h, &h->D64, n * n)) || (rc = alloc_t(*h, &h->D32, n * n)) ||
      (rc = alloc_t(*h, &h->coords, 3 * L)) || (rc = alloc_t(*h, &h->G64, 6 * L)) ||
      (rc = alloc_t(*h, &h->G32, 6 * L)) || (rc = alloc_t(*h, &h->B64, L)) ||
      (rc = alloc_t(*h, &h->detJ, L)) || (rc = alloc_t(*h, &h->gid, L)) ||
      (rc = alloc_t(*h, &h->bfaces, (size_t)E)) || (rc = alloc_t(*h, &h->mask64, L)) ||
      (rc = alloc_t(*h, &h->mult64, L)) || (rc = alloc_t(*h, &h->c64, L)) ||
      (rc = alloc_t(*h, &h->c32, L)) || (rc = alloc_t(*h, &h->cw8, L)) || (rc = alloc_t(*h, &h->minv64, L)) ||
      (rc = alloc_t(*h, &h->minv32, L)) || (rc = alloc_t(*h, &h->x64, L)) ||
      (rc = alloc_t(*h, &h->r64, L)) || (rc = alloc_t(*h, &h->p64, L)) ||
      (rc = alloc_t(*h, &h->w64, L)) || (rc = alloc_t(*h, &h->x32, L)) ||
      (rc = alloc_t(*h, &h->r32, L)) || (rc = alloc_t(*h, &h->p32, L)) ||
      (rc = alloc_t(*h, &h->w32, L)) || (rc = alloc_t(*h, &h->b32, L)) ||
      (rc = alloc_t(*h, &h->partials, 3 * (size_t)h->max_blocks)) ||
      (rc = alloc_t(*h, &h->partials_aux, 3 * (size_t)h->max_blocks)) ||
      (rc = alloc_t(*h, &h->scal, 1)) || (rc = alloc_t(*h, &h->scal_aux, 1)) ||
      (rc = alloc_t(*h, &h->dot_out, 1)))
    return fail(rc);
  if ((ce = cudaMallocHost((void**)&h->scal_host, sizeof(PcgScalars))) != cudaSuccess)
    return fail(cuda_fail(ce, "cudaMallocHost"));
  if ((ce = cudaMemsetAsync(h->scal, 0, sizeof(PcgScalars), h->stream)) != cudaSuccess ||
      (ce = cudaMemsetAsync(h->scal_aux, 0, sizeof(PcgScalars), h->stream)) != cudaSuccess)
    return fail(cuda_fail(ce, "cudaMemset"));

  h->dev_err = &h->scal->err;
  if ((rc = launch_gll(*h))) return fail(rc);
  if ((ce = cudaMemcpyAsync(h->D32_host, h->D32, sizeof(float) * n * n, cudaMemcpyDeviceToHost,
                            h->stream)) != cudaSuccess ||
      (ce = cudaMemcpyAsync(h->D64_host, h->D64, sizeof(double) * n * n, cudaMemcpyDeviceToHost,
                            h->stream)) != cudaSuccess ||
      (ce = cudaStreamSynchronize(h->stream)) != cudaSuccess)
    return fail(cuda_fail(ce, "sem_setup: D to host"));
  double* ucoords = nullptr;
  if (mesh->gid) {
    h->gid_user = true;
    if ((rc = launch_user_connectivity(*h, mesh->gid, mesh->dirichlet_faces))) return fail(rc);
    if ((ce = cudaMalloc((void**)&ucoords, sizeof(double) * 3 * L)) != cudaSuccess)
      return fail(cuda_fail(ce, "cudaMalloc"));
    if ((ce = cudaMemcpy(ucoords, mesh->coords, sizeof(double) * 3 * L, cudaMemcpyHostToDevice)) !=
        cudaSuccess) {
      cudaFree(ucoords);
      return fail(cuda_fail(ce, "cudaMemcpy"));
    }
  } else {
    if ((rc = launch_box_connectivity(*h))) return fail(rc);
  }
  double lo[3], hi[3];
  for (int d = 0; d < 3; ++d) {
    lo[d] = mesh->lo[d];
    hi[d] = mesh->hi[d];
    if (!mesh->gid && !(hi[d] > lo[d])) {
      set_error("sem_setup: need hi > lo in every direction");
      return fail(SEM_EINVAL);
    }
  }
  for (int d = 0; d < 3; ++d) {
    h->mesh_lo[d] = lo[d];
    h->mesh_hi[d] = hi[d];
  }
  h->deform_amp = mesh->deform_amp;
  h->deform_kind = mesh->deform_kind;
  rc = launch_geometry(*h, ucoords, mesh->deform_amp, mesh->deform_kind, lo, hi);
  if (ucoords) cudaFree(ucoords);
  if (rc) return fail(rc);
  if ((rc = launch_gs_map(*h))) return fail(rc);
  if ((rc = launch_jacobi(*h))) return fail(rc);
  if ((rc = autotune_ax32(*h))) return fail(rc);
  if ((ce = cudaStreamSynchronize(h->stream)) != cudaSuccess)
    return fail(cuda_fail(ce, "sem_setup"));
  *out = h;
  return SEM_OK;
}

void sem_destroy(sem_handle h) { free_handle(h); }

int sem_get_sizes(sem_handle h, sem_sizes* out) {
  if (!h || !out) {
    set_error("sem_get_sizes: null argument");
    return SEM_EINVAL;
  }
  out->N = h->N;
  out->n = h->n;
  out->E = h->E;
  out->L = h->L;
  out->U = h->U;
  out->n_shared = h->n_shared;
  out->n_segments = h->n_segments;
  out->device_bytes = h->device_bytes;
  return SEM_OK;
}

static int ax_common(sem_handle h, const void* u, void* w, sem_precision p, bool assemble) {
  if (!h || !u || !w || !valid_precision(p)) {
    set_error("sem_ax: invalid argument");
    return SEM_EINVAL;
  }
  if (u == w) {
    set_error("sem_ax: u and w may not alias");
    return SEM_EINVAL;
  }
  StreamScope scope(*h);
  int rc;
  const size_t bytes = elem_size(p) * (size_t)h->L;
  const bool w_dev = is_device_ptr(w);
  if ((!w_dev || !is_device_ptr(u)) && (rc = ensure_stage(*h))) return rc;
  const void* ud;
  if ((rc = stage_in(*h, u, bytes, h->stage_a, &ud))) return rc;
  void* wd = w_dev ? w : h->stage_b;
  if ((rc = launch_ax_local(*h, p, ud, wd, nullptr))) return rc;
  if (assemble && (rc = launch_gs(*h, p, wd))) return rc;
  if (!w_dev) {
    SEM_CUDA(cudaMemcpyAsync(w, wd, bytes, cudaMemcpyDeviceToHost, h->stream));
    SEM_CUDA(cudaStreamSynchronize(h->stream));
  }
  return SEM_OK;
}

int sem_ax(sem_handle h, const void* u, void* w, sem_precision p) {
  return ax_common(h, u, w, p, true);
}

int sem_ax_local(sem_handle h, const void* u, void* w, sem_precision p) {
  return ax_common(h, u, w, p, false);
}

int sem_gs(sem_handle h, void* v, sem_precision p) {
  if (!h || !v || !valid_precision(p)) {
    set_error("sem_gs: invalid argument");
    return SEM_EINVAL;
  }
  StreamScope scope(*h);
  int rc;
  const size_t bytes = elem_size(p) * (size_t)h->L;
  if (is_device_ptr(v)) return launch_gs(*h, p, v);
  if ((rc = ensure_stage(*h))) return rc;
  SEM_CUDA(cudaMemcpyAsync(h->stage_a, v, bytes, cudaMemcpyHostToDevice, h->stream));
  if ((rc = launch_gs(*h, p, h->stage_a))) return rc;
  SEM_CUDA(cudaMemcpyAsync(v, h->stage_a, bytes, cudaMemcpyDeviceToHost, h->stream));
  SEM_CUDA(cudaStreamSynchronize(h->stream));
  return SEM_OK;
}

int sem_glsc3(sem_handle h, const void* a, const void* b, sem_precision p, double* out) {
  if (!h || !a || !b || !out || !valid_precision(p)) {
    set_error("sem_glsc3: invalid argument");
    return SEM_EINVAL;
  }
  StreamScope scope(*h);
  int rc;
  const size_t bytes = elem_size(p) * (size_t)h->L;
  if ((!is_device_ptr(a) || !is_device_ptr(b)) && (rc = ensure_stage(*h))) return rc;
  const void *ad, *bd;
  if ((rc = stage_in(*h, a, bytes, h->stage_a, &ad))) return rc;
  if ((rc = stage_in(*h, b, bytes, h->stage_b, &bd))) return rc;
  if ((rc = launch_glsc3(*h, p, ad, bd, h->dot_out))) return rc;
  SEM_CUDA(cudaMemcpyAsync(h->scal_host, h->dot_out, sizeof(double), cudaMemcpyDeviceToHost,
                           h->stream));
  SEM_CUDA(cudaStreamSynchronize(h->stream));
  memcpy(out, h->scal_host, sizeof(double));
  return SEM_OK;
}

int sem_get_field(sem_handle h, int which, double* out) {
  if (!h || !out) {
    set_error("sem_get_field: null argument");
    return SEM_EINVAL;
  }
  StreamScope scope(*h);
  const size_t L = (size_t)h->L;
  const double* src = nullptr;
  size_t count = L;
  switch (which) {
    case 0: src = h->G64; count = 6 * L; break;
    case 1: src = h->B64; break;
    case 2: src = h->minv64; break;
    case 3: src = h->mult64; break;
    case 4: src = h->mask64; break;
    case 5: src = h->c64; break;
    case 6: src = h->coords; count = 3 * L; break;
    case 7: src = h->xi; count = (size_t)h->n; break;
    case 8: src = h->wq; count = (size_t)h->n; break;
    case 9: src = h->D64; count = (size_t)h->n * h->n; break;
    case 10: src = h->detJ; break;
    default: set_error("sem_get_field: unknown field"); return SEM_EINVAL;
  }
  SEM_CUDA(cudaMemcpyAsync(out, src, sizeof(double) * count, cudaMemcpyDefault, h->stream));
  SEM_CUDA(cudaStreamSynchronize(h->stream));
  return SEM_OK;
}

int sem_rhs(sem_handle h, int kind, uint64_t seed, double* b) {
  if (!h || !b) {
    set_error("sem_rhs: null argument");
    return SEM_EINVAL;
  }
  StreamScope scope(*h);
  int rc;
  if (is_device_ptr(b)) return launch_rhs(*h, kind, seed, b);
  if ((rc = ensure_stage(*h))) return rc;
  if ((rc = launch_rhs(*h, kind, seed, (double*)h->stage_a))) return rc;
  SEM_CUDA(cudaMemcpyAsync(b, h->stage_a, sizeof(double) * h->L, cudaMemcpyDeviceToHost, h->stream));
  SEM_CUDA(cudaStreamSynchronize(h->stream));
  return SEM_OK;
}

int sem_rhs_fourier(sem_handle h, uint64_t seed, uint64_t sample, double* b) {
  if (!h || !b) {
    set_error("sem_rhs_fourier: null argument");
    return SEM_EINVAL;
  }
  StreamScope scope(*h);
  int rc;
  if (is_device_ptr(b)) return launch_rhs_fourier(*h, seed, sample, b);
  if ((rc = ensure_stage(*h))) return rc;
  if ((rc = launch_rhs_fourier(*h, seed, sample, (double*)h->stage_a))) return rc;
  SEM_CUDA(cudaMemcpyAsync(b, h->stage_a, sizeof(double) * h->L, cudaMemcpyDeviceToHost, h->stream));
  SEM_CUDA(cudaStreamSynchronize(h->stream));
  return SEM_OK;
}

int sem_pcg_solve_ex(sem_handle h, const double* f, const double* x0, double* x,
                     const sem_solve_opts* opts, sem_info* info) {
  if (!h || !f || !x || !opts) {
    set_error("sem_pcg_solve: null argument");
    return SEM_EINVAL;
  }
  if (!valid_precision(opts->precision) || opts->precision == SEM_MIXED_TF32 ||
      opts->precision == SEM_MIXED_BF16X3) {
    set_error("sem_pcg_solve: precision not supported by the solver");
    return SEM_EINVAL;
  }
  if (opts->tol < 0 || opts->maxit < 0 || opts->fixed_iters < 0) {
    set_error("sem_pcg_solve: negative tol / maxit / fixed_iters");
    return SEM_EINVAL;
  }
  StreamScope scope(*h);
  int rc;
  const size_t bytes = sizeof(double) * (size_t)h->L;
  const bool x_dev = is_device_ptr(x);
  if ((!x_dev || !is_device_ptr(f) || (x0 && !is_device_ptr(x0))) && (rc = ensure_stage(*h)))
    return rc;
  const void *fd, *x0d;
  if ((rc = stage_in(*h, f, bytes, h->stage_a, &fd))) return rc;
  if ((rc = stage_in(*h, x0, bytes, h->stage_b, &x0d))) return rc;
  double* xd = x_dev ? x : (double*)h->stage_c;
  sem_solve_opts o = *opts;
  o.use_graph = o.use_graph >= 0 ? 1 : 0;   // 0 (default) or 1: graphs on; -1: off
  rc = pcg_solve(*h, (const double*)fd, (const double*)x0d, xd, o, info);
  if (rc < 0) return rc;
  if (!x_dev) {
    SEM_CUDA(cudaMemcpyAsync(x, xd, bytes, cudaMemcpyDeviceToHost, h->stream));
    SEM_CUDA(cudaStreamSynchronize(h->stream));
  }
  return rc;
}

int sem_pcg_solve(sem_handle h, const double* f, const double* x0, double* x, double tol,
                  int maxit, sem_precision p, sem_info* info) {
  sem_solve_opts o;
  memset(&o, 0, sizeof(o));
  o.tol = tol;
  o.maxit = maxit;
  o.precision = p;
  o.use_graph = 1;
  return sem_pcg_solve_ex(h, f, x0, x, &o, info);
}

static void drop_graphs(Handle& h) {
  for (int q = 0; q < 8; ++q) {
    if (h.graph_exec[q]) cudaGraphExecDestroy(h.graph_exec[q]);
    h.graph_exec[q] = nullptr;
  }
}

int sem_mg_apply(sem_handle h, const void* r, void* z, sem_precision p) {
  if (!h || !r || !z) {
    set_error("sem_mg_apply: null argument");
    return SEM_EINVAL;
  }
  if (p != SEM_FP64 && p != SEM_MIXED_FP32) {
    set_error("sem_mg_apply: precision must be SEM_FP64 or SEM_MIXED_FP32");
    return SEM_EINVAL;
  }
  if (!is_device_ptr(r) || !is_device_ptr(z)) {
    set_error("sem_mg_apply: r and z must be device pointers");
    return SEM_EINVAL;
  }
  StreamScope scope(*h);
  return mg_apply(*h, p, r, z);
}

int sem_set_option(sem_handle h, const char* key, int64_t value) {
  if (!h || !key) {
    set_error("sem_set_option: null argument");
    return SEM_EINVAL;
  }
  const std::string k(key);
  if ((k == "ax_variant" || k == "ax_variant_pcg") && value >= 0 && value < kTmaVariants) {
    (k == "ax_variant" ? h->ax_variant : h->ax_variant_pcg) = (int)value;
  } else if (k == "ax_grid_cap" && value >= 0 && value <= (1 << 30)) {
    h->ax_grid_cap = (int)value;
  } else if (k == "use_tma" && (value == 0 || value == 1)) {
    h->use_tma = value != 0;
  } else if (k == "gs_acc" && value >= 0 && value <= 2) {
    h->gs_acc = (int)value;
  } else if (k == "l2_persist" && (value == 0 || value == 1)) {
    h->l2_persist = value != 0;
  } else if (k == "upd_tma" && (value == 0 || value == 1)) {
    h->upd_tma = value != 0;
  } else if (k == "mg_hcoarsen" && (value == 0 || value == 1)) {
    if (h->mg_hcoarsen != (value != 0)) mg_free(*h);   // rebuilt on next use
    h->mg_hcoarsen = value != 0;
  } else if (k == "upd_variant" && value >= 0 && value <= 5) {
    h->upd_variant = (int)value;
  } else if (k == "l2_hints" && (value == 0 || value == 1)) {
    h->l2_hints = value != 0;
  } else if (k == "fuse_gs" && value >= 0 && value <= 2) {
    h->fuse_gs = (int)value;
  } else if (k == "kernel_timing" && (value == 0 || value == 1)) {
    h->kernel_timing = value != 0;   // setting it (either way) clears the sums
    h->kt_ms[0] = h->kt_ms[1] = h->kt_ms[2] = 0.0;
    h->kt_iters = 0;
    h->kt_recorded = 0;
  } else {
    set_error("sem_set_option: unknown key or value out of range: " + k);
    return SEM_EINVAL;
  }
  drop_graphs(*h);   // captured graphs hold the old launch choices
  return SEM_OK;
}

int sem_get_option(sem_handle h, const char* key, double* value) {
  if (!h || !key || !value) {
    set_error("sem_get_option: null argument");
    return SEM_EINVAL;
  }
  const std::string k(key);
  if (k == "ax_variant") *value = h->ax_variant;
  else if (k == "ax_variant_pcg") *value = h->ax_variant_pcg;
  else if (k == "use_tma") *value = h->use_tma ? 1 : 0;
  else if (k == "ax_grid_cap") *value = h->ax_grid_cap;
  else if (k == "gs_acc") *value = h->gs_acc;
  else if (k == "l2_persist") *value = h->l2_persist ? 1 : 0;
  else if (k == "fuse_gs") *value = h->fuse_gs;
  else if (k == "l2_hints") *value = h->l2_hints ? 1 : 0;
  else if (k == "upd_variant") *value = h->upd_variant;
  else if (k == "upd_tma") *value = h->upd_tma ? 1 : 0;
  else if (k == "mg_hcoarsen") *value = h->mg_hcoarsen ? 1 : 0;
  else if (k == "mg_levels") *value = mg_levels(*h);
  else if (k.rfind("mg_omega_", 0) == 0 && k.size() > 9 && k.size() <= 12 &&
           k.find_first_not_of("0123456789", 9) == std::string::npos) {
    // level index: any number of decimal digits (the level count grows with
    // log2 of the mesh size once h-levels are built)
    *value = mg_omega(*h, std::stoi(k.substr(9)));   // -1 for a level that does not exist
  }
  else if (k == "l2_window_bytes") *value = (double)h->l2_window_bytes;
  else if (k == "l2_max_persist") *value = (double)h->l2_max_persist;
  else if (k == "l2_max_window") *value = (double)h->l2_max_window;
  else if (k == "launches") *value = (double)h->launches;
  else if (k == "kernel_timing") *value = h->kernel_timing ? 1 : 0;
  else if (k == "kt_iters") *value = (double)h->kt_iters;
  else if (k == "kt_ms_ax" || k == "kt_ms_gs" || k == "kt_ms_update") {
    const int q = k == "kt_ms_ax" ? 0 : k == "kt_ms_gs" ? 1 : 2;
    *value = h->kt_iters ? h->kt_ms[q] / (double)h->kt_iters : 0.0;
  }
  else if (k.rfind("ax_tune_ms_plain_", 0) == 0 && k.size() == 18 && k[17] >= '0' && k[17] < '0' + kTmaVariants)
    *value = h->ax_tune_ms[0][k[17] - '0'];
  else if (k.rfind("ax_tune_ms_pcg_", 0) == 0 && k.size() == 16 && k[15] >= '0' && k[15] < '0' + kTmaVariants)
    *value = h->ax_tune_ms[1][k[15] - '0'];
  else {
    set_error("sem_get_option: unknown key: " + k);
    return SEM_EINVAL;
  }
  return SEM_OK;
}

}  // extern "C"
