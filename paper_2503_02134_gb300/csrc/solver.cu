// Host driver of the Jacobi PCG solve.
//
// FP64 path: the CG loop of the paper's profiling table (Sec. 3.1), one
// iteration = [preconditioner + add2s1 + ax + glsc3(w,c,p)] (one fused
// kernel), the gather-scatter, and [add2s2 x2 + glsc3(r,c,r) +
// glsc3(r,c,z)] (one fused kernel).  Scalars stay on the device; the host
// only polls a `done` flag once per chunk of iterations, and a chunk is
// replayed as a CUDA graph.
//
// Mixed path: the paper's converging strategy (Sec. 3.3, 4.3): FP32
// operator, preconditioner and vector updates; FP64 gather-scatter sums;
// FP64-quality dot products and FP64 scalars.  Around it sits an FP64
// residual / iterative-refinement loop (x64 += d, r64 = f - A64 x64) so the
// final residual is judged in FP64 and stagnation of the FP32 recursion is
// cured by a restart.  All-FP32 variant (the paper's stagnating strategy):
// FP32 gather-scatter sums and FP32 dots, no refinement.
#include <math.h>

#include <algorithm>
#include <vector>

#include "pcg.cuh"

namespace sem {

int ax_dispatch_fp64(Handle& h, const double* u, double* w, const AxPrologue* pro);
int ax_dispatch_fp32(Handle& h, const float* u, float* w, const AxPrologue* pro, int dm);

int ax_dispatch_tc(Handle& h, const float* u, float* w, sem_precision p);

int launch_ax_local(Handle& h, sem_precision p, const void* u, void* w, const AxPrologue* pro) {
  if (p == SEM_FP64) return ax_dispatch_fp64(h, (const double*)u, (double*)w, pro);
  if ((p == SEM_MIXED_TF32 || p == SEM_MIXED_BF16X3) && !pro)
    return ax_dispatch_tc(h, (const float*)u, (float*)w, p);
  const int dm = p == SEM_FP32_ALL ? kDotFP32 : kDotDot2;
  return ax_dispatch_fp32(h, (const float*)u, (float*)w, pro, dm);
}

int read_scalars(Handle& h, PcgScalars* dev, PcgScalars* out) {
  SEM_CUDA(cudaMemcpyAsync(h.scal_host, dev, sizeof(PcgScalars), cudaMemcpyDeviceToHost, h.stream));
  SEM_CUDA(cudaStreamSynchronize(h.stream));
  *out = *h.scal_host;
  return 0;
}

// r64 = f - A64 x64 in FP64; returns ||r64||_c / ||f||_c through *relres
// (and ||f||_c through *bnorm when asked).
int fp64_residual(Handle& h, const double* f, bool x_is_zero, double* relres,
                  double* bnorm) {
  int rc;
  if ((rc = launch_scal_setup(h, h.scal_aux, 0.0, 1, 1, 0))) return rc;
  if (!x_is_zero) {
    if ((rc = ax_dispatch_fp64(h, h.x64, h.w64, nullptr))) return rc;
    if ((rc = launch_gs(h, SEM_FP64, h.w64))) return rc;
  }
  double* saved = h.partials;
  h.partials = h.partials_aux;
  rc = launch_cg_init64(h, h.r64, f, x_is_zero ? nullptr : h.w64, h.minv64, h.scal_aux, nullptr);
  h.partials = saved;
  if (rc) return rc;
  PcgScalars s;
  if ((rc = read_scalars(h, h.scal_aux, &s))) return rc;
  *relres = s.relres;
  if (bnorm) *bnorm = s.bnorm;
  return 0;
}


namespace {

// A restart of the inner FP32 recursion is forced when its residual has not
// fallen by 10 % for this many iterations (CG residuals plateau for tens of
// iterations on hard problems, so the window is long).
constexpr int kStagWindow = 200;

enum GraphKind { kG64 = 0, kGMixed = 1, kGFP32 = 2 };

// Timing mode: record event q (0..3) of iteration `it` of the chunk on the
// handle's stream (events are created once and kept).
int kt_mark(Handle& h, int it, int q) {
  const size_t idx = 4 * (size_t)it + q;
  while (h.kt_events.size() <= idx) {
    cudaEvent_t e = nullptr;
    SEM_CUDA(cudaEventCreate(&e));
    h.kt_events.push_back(e);
  }
  SEM_CUDA(cudaEventRecord(h.kt_events[idx], h.stream));
  return 0;
}

// Timing mode: add the kernel times of the first `ran` recorded iterations
// of the chunk (the stream has been synchronised by the caller); launches
// after the solve finished return at once and are not counted.
int kt_collect(Handle& h, int ran) {
  const int m = std::max(0, std::min(h.kt_recorded, ran));
  for (int it = 0; it < m; ++it) {
    for (int q = 0; q < 3; ++q) {
      float ms = 0.f;
      SEM_CUDA(cudaEventElapsedTime(&ms, h.kt_events[4 * it + q], h.kt_events[4 * it + q + 1]));
      h.kt_ms[q] += ms;
    }
  }
  h.kt_iters += m;
  h.kt_recorded = 0;
  return 0;
}

// Enqueue `iters` PCG iterations (no host interaction).
int enqueue_iterations(Handle& h, GraphKind kind, int iters) {
  AxPrologue pro;
  pro.scal = h.scal;
  pro.pap_partials = h.partials;
  const bool kt = h.kernel_timing;
  for (int it = 0; it < iters; ++it) {
    int rc;
    if (kt && (rc = kt_mark(h, it, 0))) return rc;
    if (kind == kG64) {
      pro.r = h.r64;
      pro.minv = h.minv64;
      if ((rc = ax_dispatch_fp64(h, h.p64, h.w64, &pro))) return rc;
      if (kt && (rc = kt_mark(h, it, 1))) return rc;
      if ((rc = launch_gs(h, SEM_FP64, h.w64))) return rc;
      if (kt && (rc = kt_mark(h, it, 2))) return rc;
      if ((rc = launch_cg_update64(h, h.x64, h.r64, h.p64, h.w64, h.scal, h.hist_dev))) return rc;
    } else {
      const int dm = kind == kGFP32 ? kDotFP32 : kDotDot2;
      const sem_precision gp = kind == kGFP32 ? SEM_FP32_ALL : SEM_MIXED_FP32;
      pro.r = h.r32;
      pro.minv = h.minv32;
      if ((rc = ax_dispatch_fp32(h, h.p32, h.w32, &pro, dm))) return rc;
      if (kt && (rc = kt_mark(h, it, 1))) return rc;
      if (gs_fusable(h)) {
        // box mesh: QQ^T folded into the update (no separate pass)
        if (kt && (rc = kt_mark(h, it, 2))) return rc;
        const int acc = kind == kGFP32 ? 1 : h.gs_acc;
        if ((rc = launch_cg_update32_gs(h, dm, acc, h.x32, h.r32, h.p32, h.w32, h.minv32,
                                        h.scal, h.hist_dev)))
          return rc;
      } else {
        if ((rc = launch_gs(h, gp, h.w32))) return rc;
        if (kt && (rc = kt_mark(h, it, 2))) return rc;
        if ((rc = launch_cg_update32(h, dm, h.x32, h.r32, h.p32, h.w32, h.minv32, h.scal,
                                     h.hist_dev)))
          return rc;
      }
    }
    if (kt && (rc = kt_mark(h, it, 3))) return rc;
  }
  if (kt) h.kt_recorded = iters;
  return 0;
}

int run_chunk(Handle& h, GraphKind kind, int chunk, bool use_graph) {
  // per-kernel timing records events between launches: no graphs
  if (!use_graph || h.kernel_timing) return enqueue_iterations(h, kind, chunk);
  if (!h.graph_exec[kind] || h.graph_chunk[kind] != chunk) {
    if (h.graph_exec[kind]) {
      cudaGraphExecDestroy(h.graph_exec[kind]);
      h.graph_exec[kind] = nullptr;
    }
    cudaGraph_t g = nullptr;
    const int64_t before = h.launches;
    SEM_CUDA(cudaStreamBeginCapture(h.stream, cudaStreamCaptureModeThreadLocal));
    int rc = enqueue_iterations(h, kind, chunk);
    cudaError_t e = cudaStreamEndCapture(h.stream, &g);
    h.graph_nodes[kind] = h.launches - before;   // kernels per replay
    h.launches = before;                          // capture itself runs nothing
    if (rc) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&h.graph_exec[kind], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    h.graph_chunk[kind] = chunk;
  }
  SEM_CUDA(cudaGraphLaunch(h.graph_exec[kind], h.stream));
  h.launches += h.graph_nodes[kind];
  return 0;
}

// Iterate until the device says done; returns 0 or an error.  On entry
// *fin holds the scalars as they stand (read by the caller).
int iterate(Handle& h, GraphKind kind, int chunk, bool use_graph, PcgScalars* fin) {
  int base = fin->iter;
  for (;;) {
    int rc = run_chunk(h, kind, chunk, use_graph);
    if (rc) return rc;
    if ((rc = read_scalars(h, h.scal, fin))) return rc;
    if (h.kernel_timing) {
      if ((rc = kt_collect(h, fin->iter - base))) return rc;
      base = fin->iter;
    }
    if (fin->err) {
      set_error("pcg: a bounded device wait gave up (bulk copy did not complete)");
      return SEM_ETIMEOUT;
    }
    if (fin->done) return 0;
  }
}

int ensure_history(Handle& h, int maxit) {
  if (h.hist_cap >= maxit + 1) return 0;
  if (h.hist_dev) cudaFree(h.hist_dev);
  h.hist_dev = nullptr;
  int cap = std::max(maxit + 1, 1024);
  SEM_CUDA(cudaMalloc((void**)&h.hist_dev, sizeof(double) * cap));
  h.hist_cap = cap;
  // graphs captured the old pointer
  for (int q = 0; q < 8; ++q) {
    if (h.graph_exec[q]) cudaGraphExecDestroy(h.graph_exec[q]);
    h.graph_exec[q] = nullptr;
  }
  return 0;
}

}  // namespace

// Keep the FP32 operator output w resident in L2 between the three kernels
// of an iteration (written by the operator, gathered and scattered by the
// gather-scatter, read by the update): an access-policy window marks it
// persisting for kernels on the handle's stream.  The context's persisting
// carve-out is released when the solve ends.
struct L2Window {
  Handle& h;
  bool on = false;
  L2Window(Handle& hh, const void* base, size_t bytes) : h(hh) {
    if (!h.l2_persist || h.l2_hints || !base) return;
    int max_persist = 0, max_window = 0;
    if (cudaDeviceGetAttribute(&max_persist, cudaDevAttrMaxPersistingL2CacheSize, h.device) != cudaSuccess ||
        cudaDeviceGetAttribute(&max_window, cudaDevAttrMaxAccessPolicyWindowSize, h.device) != cudaSuccess ||
        max_persist <= 0 || max_window <= 0) {
      cudaGetLastError();
      return;
    }
    const size_t want = std::min(bytes, (size_t)std::min(max_persist, max_window));
    h.l2_window_bytes = (int64_t)want;
    h.l2_max_persist = max_persist;
    h.l2_max_window = max_window;
    if (cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, want) != cudaSuccess) {
      cudaGetLastError();
      return;
    }
    cudaStreamAttrValue a{};
    a.accessPolicyWindow.base_ptr = const_cast<void*>(base);
    a.accessPolicyWindow.num_bytes = want;
    a.accessPolicyWindow.hitRatio = 1.0f;
    a.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
    a.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
    if (cudaStreamSetAttribute(h.stream, cudaStreamAttributeAccessPolicyWindow, &a) != cudaSuccess) {
      cudaGetLastError();
      return;
    }
    on = true;
  }
  ~L2Window() {
    if (!on) return;
    cudaStreamAttrValue a{};
    a.accessPolicyWindow.num_bytes = 0;
    cudaStreamSetAttribute(h.stream, cudaStreamAttributeAccessPolicyWindow, &a);
    cudaStreamSynchronize(h.stream);
    cudaCtxResetPersistingL2Cache();
    cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, 0);
    cudaGetLastError();
  }
};

int pcg_mg_solve(Handle& h, const double* f, const double* x0, double* x, double tol, int maxit,
                 sem_precision prec, double inner_floor, int max_cycles, int refine_mode,
                 double replace_factor, sem_info* info);

int pcg_solve(Handle& h, const double* f, const double* x0, double* x, const sem_solve_opts& o,
              sem_info* info) {
  if (o.precond == 2) {
    // multigrid-preconditioned CG (FP64, or mixed with FP64 restarts)
    if (o.precision != SEM_FP64 && o.precision != SEM_MIXED_FP32) {
      set_error("pcg: the multigrid preconditioner supports SEM_FP64 and SEM_MIXED_FP32");
      return SEM_EINVAL;
    }
    return pcg_mg_solve(h, f, x0, x, o.tol > 0 ? o.tol : 1e-8, o.maxit > 0 ? o.maxit : 1000,
                        o.precision, o.inner_tol > 0 ? o.inner_tol : 1e-4,
                        o.max_cycles > 0 ? o.max_cycles : 20, o.refine_mode, o.replace_factor,
                        info);
  }
  const double tol = o.tol > 0 ? o.tol : 1e-8;
  const int maxit = o.maxit > 0 ? o.maxit : 1000;
  const int fixed = o.fixed_iters > 0 ? o.fixed_iters : 0;
  const bool use_graph = o.use_graph != 0;
  const int chunk = o.chunk > 0 ? o.chunk : 32;
  const sem_precision prec = o.precision;
  const double inner_floor = o.inner_tol > 0 ? o.inner_tol : 1e-5;
  const int max_cycles = o.max_cycles > 0 ? o.max_cycles : 20;
  const bool identity = o.precond < 0;
  int rc;
  const int cap_it = fixed ? fixed : maxit;
  if ((rc = ensure_history(h, cap_it))) return rc;

  sem_info res{};
  const int64_t launches0 = h.launches;
  std::vector<double> hist_host;
  SEM_CUDA(cudaEventRecord(h.ev0, h.stream));

  // The identity preconditioner reuses the kernels with J^{-1} = mask.
  double* minv64 = h.minv64;
  float* minv32 = h.minv32;
  float* minv32_copy = nullptr;
  auto drop_graphs = [&]() {
    for (int q = 0; q < 8; ++q) {
      if (h.graph_exec[q]) cudaGraphExecDestroy(h.graph_exec[q]);
      h.graph_exec[q] = nullptr;
    }
  };
  if (identity) {
    SEM_CUDA(cudaMallocAsync((void**)&minv32_copy, sizeof(float) * h.L, h.stream));
    if ((rc = launch_cast64to32(h, h.mask64, minv32_copy))) return rc;
    h.minv64 = h.mask64;
    h.minv32 = minv32_copy;
    drop_graphs();   // graphs captured the Jacobi pointers
  }
  auto restore = [&]() {
    h.minv64 = minv64;
    h.minv32 = minv32;
    if (minv32_copy) {
      cudaFreeAsync(minv32_copy, h.stream);
      drop_graphs();
    }
  };

  if (prec == SEM_FP64) {
    if ((rc = launch_masked_copy64(h, x0, h.x64))) { restore(); return rc; }
    if (x0) {
      if ((rc = ax_dispatch_fp64(h, h.x64, h.w64, nullptr))) { restore(); return rc; }
      if ((rc = launch_gs(h, SEM_FP64, h.w64))) { restore(); return rc; }
    }
    SEM_CUDA(cudaMemsetAsync(h.p64, 0, sizeof(double) * h.L, h.stream));
    if ((rc = launch_scal_setup(h, h.scal, tol, cap_it, fixed ? 1 : 0, 0))) { restore(); return rc; }
    if ((rc = launch_cg_init64(h, h.r64, f, x0 ? h.w64 : nullptr, h.minv64, h.scal, h.hist_dev))) {
      restore();
      return rc;
    }
    PcgScalars fin;
    if ((rc = read_scalars(h, h.scal, &fin))) { restore(); return rc; }
    if (!fin.done && (rc = iterate(h, kG64, chunk, use_graph, &fin))) { restore(); return rc; }
    res.iters = fin.iter;
    res.status = fin.status;
    res.relres = fin.relres;
    if (o.history) {
      hist_host.resize(fin.iter + 1);
      SEM_CUDA(cudaMemcpy(hist_host.data(), h.hist_dev, sizeof(double) * (fin.iter + 1),
                          cudaMemcpyDeviceToHost));
    }
    SEM_CUDA(cudaEventRecord(h.ev1, h.stream));
    if ((rc = fp64_residual(h, f, false, &res.relres_true))) { restore(); return rc; }
  } else if (prec != SEM_FP32_ALL && !o.no_refine && !fixed && o.refine_mode == 0) {
    L2Window l2(h, h.w32, sizeof(float) * (size_t)h.L);
    // Mixed with reliable updates: one FP32 CG recursion for A x = f with
    // x = x64 + x32.  Each time its residual has fallen by `delta` the
    // correction is folded into x64, the FP64 true residual is recomputed and
    // replaces r32, and the recursion continues with the same p.
    const double delta = o.replace_factor > 0 ? o.replace_factor : 1e-2;
    if ((rc = launch_masked_copy64(h, x0, h.x64))) { restore(); return rc; }
    double relres_true = 1.0, bnorm = 0.0;
    if ((rc = fp64_residual(h, f, x0 == nullptr, &relres_true, &bnorm))) { restore(); return rc; }
    res.status = 0;
    int replacements = 0, slow = 0;
    PcgScalars fin{};
    if (bnorm > 0.0 && relres_true > tol) {
      SEM_CUDA(cudaMemsetAsync(h.x32, 0, sizeof(float) * h.L, h.stream));
      SEM_CUDA(cudaMemsetAsync(h.p32, 0, sizeof(float) * h.L, h.stream));
      if ((rc = launch_cast64to32(h, h.r64, h.b32))) { restore(); return rc; }
      double seg_tol = std::max(tol, delta * relres_true);
      if ((rc = launch_scal_setup(h, h.scal, seg_tol, maxit, 0, 0))) { restore(); return rc; }
      if ((rc = launch_cg_init32(h, kDotDot2, h.r32, h.b32, nullptr, h.minv32, h.scal,
                                 h.hist_dev))) {
        restore();
        return rc;
      }
      if ((rc = launch_set_bnorm(h, h.scal, bnorm, h.hist_dev))) { restore(); return rc; }
      for (;;) {
        if ((rc = read_scalars(h, h.scal, &fin))) { restore(); return rc; }
        if (!fin.done && (rc = iterate(h, kGMixed, chunk, use_graph, &fin))) { restore(); return rc; }
        if ((rc = launch_add32to64(h, h.x64, h.x32))) { restore(); return rc; }
        SEM_CUDA(cudaMemsetAsync(h.x32, 0, sizeof(float) * h.L, h.stream));
        const double prev = relres_true;
        if ((rc = fp64_residual(h, f, false, &relres_true))) { restore(); return rc; }
        if (relres_true <= tol) break;
        if (fin.status == SEM_BREAKDOWN) { res.status = SEM_BREAKDOWN; break; }
        if (fin.iter >= maxit) { res.status = SEM_MAXIT; break; }
        slow = relres_true > 0.5 * prev ? slow + 1 : 0;
        if (slow >= 3 || replacements >= 4 * max_cycles) { res.status = SEM_STAGNATED; break; }
        seg_tol = std::max(tol, delta * relres_true);
        if ((rc = launch_cg_replace32(h, kDotDot2, h.r64, h.r32, h.minv32, seg_tol, h.scal))) {
          restore();
          return rc;
        }
        ++replacements;
      }
      if (o.history) {
        hist_host.resize(fin.iter + 1);
        SEM_CUDA(cudaMemcpy(hist_host.data(), h.hist_dev, sizeof(double) * (fin.iter + 1),
                            cudaMemcpyDeviceToHost));
      }
    }
    res.iters = fin.iter;
    res.refinements = replacements;
    res.relres = fin.relres;
    res.relres_true = relres_true;
    SEM_CUDA(cudaEventRecord(h.ev1, h.stream));
  } else {
    const bool all32 = prec == SEM_FP32_ALL;
    const bool refine = !all32 && !o.no_refine && !fixed;
    const GraphKind kind = all32 ? kGFP32 : kGMixed;
    const int dm = all32 ? kDotFP32 : kDotDot2;
    if ((rc = launch_masked_copy64(h, x0, h.x64))) { restore(); return rc; }
    bool x_zero = x0 == nullptr;
    int total_it = 0;
    int cycles = 0;
    double relres_true = 1.0;
    res.status = 0;
    for (;;) {
      // FP64 outer residual r64 = f - A x64 (first cycle with x0 = 0: r64 = f)
      if (refine || cycles == 0) {
        if ((rc = fp64_residual(h, f, x_zero, &relres_true))) { restore(); return rc; }
      }
      if (refine && relres_true <= tol) break;
      if (refine && cycles >= max_cycles) {
        res.status = SEM_STAGNATED;
        break;
      }
      if (refine && total_it >= maxit) {
        res.status = SEM_MAXIT;
        break;
      }
      // inner mixed solve of A d = r64 (FP32 copy), d0 = 0
      if ((rc = launch_cast64to32(h, h.r64, h.b32))) { restore(); return rc; }
      SEM_CUDA(cudaMemsetAsync(h.x32, 0, sizeof(float) * h.L, h.stream));
      SEM_CUDA(cudaMemsetAsync(h.p32, 0, sizeof(float) * h.L, h.stream));
      double inner_tol = tol;
      int inner_max = fixed ? fixed : maxit - total_it;
      if (refine) inner_tol = std::max(inner_floor, 0.5 * tol / std::max(relres_true, 1e-300));
      if ((rc = launch_scal_setup(h, h.scal, inner_tol, inner_max, fixed ? 1 : 0,
                                   refine ? kStagWindow : 0))) {
        restore();
        return rc;
      }
      if ((rc = launch_cg_init32(h, dm, h.r32, h.b32, nullptr, h.minv32, h.scal, h.hist_dev))) {
        restore();
        return rc;
      }
      PcgScalars fin;
      if ((rc = read_scalars(h, h.scal, &fin))) { restore(); return rc; }
      if (!fin.done && (rc = iterate(h, kind, chunk, use_graph, &fin))) { restore(); return rc; }
      if (o.history) {
        std::vector<double> hcyc(fin.iter + 1);
        SEM_CUDA(cudaMemcpy(hcyc.data(), h.hist_dev, sizeof(double) * (fin.iter + 1),
                            cudaMemcpyDeviceToHost));
        const double scale = refine ? relres_true : 1.0;
        for (int q = (cycles == 0 ? 0 : 1); q <= fin.iter; ++q) hist_host.push_back(hcyc[q] * scale);
      }
      total_it += fin.iter;
      res.relres = fin.relres * (refine ? relres_true : 1.0);
      if ((rc = launch_add32to64(h, h.x64, h.x32))) { restore(); return rc; }
      x_zero = false;
      ++cycles;
      if (fin.status == SEM_BREAKDOWN) {
        res.status = SEM_BREAKDOWN;
        break;
      }
      if (!refine) {
        res.status = fin.status;
        break;
      }
    }
    res.iters = total_it;
    res.refinements = refine ? cycles - 1 : 0;
    SEM_CUDA(cudaEventRecord(h.ev1, h.stream));
    if (!refine) {
      if ((rc = fp64_residual(h, f, false, &relres_true))) { restore(); return rc; }
    }
    res.relres_true = relres_true;
  }
  restore();
  // solution out
  SEM_CUDA(cudaMemcpyAsync(x, h.x64, sizeof(double) * h.L, cudaMemcpyDeviceToDevice, h.stream));
  SEM_CUDA(cudaStreamSynchronize(h.stream));
  float ms = 0.f;
  SEM_CUDA(cudaEventElapsedTime(&ms, h.ev0, h.ev1));
  res.solve_ms = ms;
  res.launches = h.launches - launches0;
  if (o.history) {
    const int cnt = std::min<int>((int)hist_host.size(), cap_it + 1);
    for (int q = 0; q < cnt; ++q) o.history[q] = hist_host[q];
  }
  if (info) *info = res;
  return res.status;
}

}  // namespace sem
