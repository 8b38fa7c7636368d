// FP32 instantiations of the element operator (CUDA cores), plain and PCG-fused
// with the compensated (Dot2) or the plain FP32 pap reduction.
#include "ax_tma.cuh"

namespace sem {

static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// Staged launch of variant V in the requested mode; nonzero `*fit` is
// cleared when that variant's stages do not fit in shared memory.
template <int n, int V>
static int tma_variant(Handle& h, const float* u, float* w, const AxPrologue* pro, int dm,
                       bool* fit) {
  if (!pro) {
    if constexpr (tma_fits<n, false, V>()) return ax_tma_launch<n, false, kDotDot2, V>(h, u, w, nullptr);
  } else {
    if constexpr (tma_fits<n, true, V>()) {
      if (dm == kDotFP32) return ax_tma_launch<n, true, kDotFP32, V>(h, u, w, pro);
      return ax_tma_launch<n, true, kDotDot2, V>(h, u, w, pro);
    }
  }
  *fit = false;
  return 0;
}

// Whether launch variant v of the staged operator fits at order n (mode pcg).
template <int n>
static bool tma_fits_rt(bool pcg, int v) {
  switch (v) {
    case 0: return pcg ? tma_fits<n, true, 0>() : tma_fits<n, false, 0>();
    case 1: return pcg ? tma_fits<n, true, 1>() : tma_fits<n, false, 1>();
    case 2: return pcg ? tma_fits<n, true, 2>() : tma_fits<n, false, 2>();
    case 4: return pcg ? tma_fits<n, true, 4>() : tma_fits<n, false, 4>();
    default: return pcg ? tma_fits<n, true, 3>() : tma_fits<n, false, 3>();
  }
}

template <int n>
static int run32(Handle& h, const float* u, float* w, const AxPrologue* pro, int dm) {
  // bulk-copy staged kernel: even n (16-byte element blocks)
  if constexpr (n % 2 == 0) {
    const bool ok = h.use_tma && aligned16(u) && aligned16(w) &&
                    (!pro || (aligned16(pro->r) && aligned16(pro->minv)));
    if (ok) {
      const int v = pro ? h.ax_variant_pcg : h.ax_variant;
      bool fit = true;
      int rc;
      switch (v) {
        case 1: rc = tma_variant<n, 1>(h, u, w, pro, dm, &fit); break;
        case 2: rc = tma_variant<n, 2>(h, u, w, pro, dm, &fit); break;
        case 3: rc = tma_variant<n, 3>(h, u, w, pro, dm, &fit); break;
        case 4: rc = tma_variant<n, 4>(h, u, w, pro, dm, &fit); break;
        default: rc = tma_variant<n, 0>(h, u, w, pro, dm, &fit); break;
      }
      if (fit) return rc;
      // no staged variant of this mode fits (PCG mode at n = 16): unstaged kernel
    }
  }
  if (!pro) return ax_launch<n, float, false, kDotDot2>(h, u, w, h.G32, h.D32, nullptr);
  if (dm == kDotFP32) return ax_launch<n, float, true, kDotFP32>(h, u, w, h.G32, h.D32, pro);
  return ax_launch<n, float, true, kDotDot2>(h, u, w, h.G32, h.D32, pro);
}

bool ax32_variant_fits(int n, bool pcg, int v) {
  switch (n) {
    case 2: return tma_fits_rt<2>(pcg, v);
    case 4: return tma_fits_rt<4>(pcg, v);
    case 6: return tma_fits_rt<6>(pcg, v);
    case 8: return tma_fits_rt<8>(pcg, v);
    case 10: return tma_fits_rt<10>(pcg, v);
    case 12: return tma_fits_rt<12>(pcg, v);
    case 14: return tma_fits_rt<14>(pcg, v);
    case 16: return tma_fits_rt<16>(pcg, v);
    default: return false;
  }
}

int ax_dispatch_fp32(Handle& h, const float* u, float* w, const AxPrologue* pro, int dm) {
  switch (h.n) {
    case 2: return run32<2>(h, u, w, pro, dm);
    case 3: return run32<3>(h, u, w, pro, dm);
    case 4: return run32<4>(h, u, w, pro, dm);
    case 5: return run32<5>(h, u, w, pro, dm);
    case 6: return run32<6>(h, u, w, pro, dm);
    case 7: return run32<7>(h, u, w, pro, dm);
    case 8: return run32<8>(h, u, w, pro, dm);
    case 9: return run32<9>(h, u, w, pro, dm);
    case 10: return run32<10>(h, u, w, pro, dm);
    case 11: return run32<11>(h, u, w, pro, dm);
    case 12: return run32<12>(h, u, w, pro, dm);
    case 13: return run32<13>(h, u, w, pro, dm);
    case 14: return run32<14>(h, u, w, pro, dm);
    case 15: return run32<15>(h, u, w, pro, dm);
    case 16: return run32<16>(h, u, w, pro, dm);
    default: set_error("ax: unsupported order"); return SEM_EINVAL;
  }
}

}  // namespace sem

namespace sem {

int launch_scal_setup(Handle& h, PcgScalars* s, double tol, int maxit, int fixed, int stag_window);

// Project autotuner of the staged FP32 operator: times every launch variant
// (elements per block x pipeline stages) of both modes on this handle's mesh
// with CUDA events and keeps the fastest.  Runs once, at set-up.
int autotune_ax32(Handle& h) {
  if (h.n % 2 != 0 || !h.use_tma) return 0;
  ScopedEvents ev;
  SEM_CUDA(ev.create());
  cudaEvent_t a = ev.a, b = ev.b;
  // positive data (0x3f3f3f3f ~ 0.747) so the PCG-mode pap stays positive
  SEM_CUDA(cudaMemsetAsync(h.b32, 0x3f, sizeof(float) * h.L, h.stream));
  SEM_CUDA(cudaMemsetAsync(h.x32, 0x3f, sizeof(float) * h.L, h.stream));
  int rc = launch_scal_setup(h, h.scal_aux, 0.0, 1, 0, 0);
  AxPrologue pro;
  pro.r = h.b32;
  pro.minv = h.minv32;
  pro.scal = h.scal_aux;
  pro.pap_partials = h.partials_aux;
  const int reps = 3;
  for (int mode = 0; mode < 2 && !rc; ++mode) {
    float best = 1e30f;
    int best_v = 0;
    for (int v = 0; v < kTmaVariants && !rc; ++v) {
      if (!ax32_variant_fits(h.n, mode == 1, v)) {
        h.ax_tune_ms[mode][v] = -1.f;   // not launched: its stages exceed shared memory
        continue;
      }
      if (mode == 0) h.ax_variant = v; else h.ax_variant_pcg = v;
      const AxPrologue* pp = mode ? &pro : nullptr;
      if ((rc = ax_dispatch_fp32(h, h.x32, h.w32, pp, kDotDot2))) break;
      SEM_CUDA(cudaEventRecord(a, h.stream));
      for (int q = 0; q < reps && !rc; ++q) rc = ax_dispatch_fp32(h, h.x32, h.w32, pp, kDotDot2);
      SEM_CUDA(cudaEventRecord(b, h.stream));
      SEM_CUDA(cudaEventSynchronize(b));
      float ms = 0.f;
      SEM_CUDA(cudaEventElapsedTime(&ms, a, b));
      h.ax_tune_ms[mode][v] = ms / reps;
      if (ms < best) {
        best = ms;
        best_v = v;
      }
    }
    if (mode == 0) h.ax_variant = best_v; else h.ax_variant_pcg = best_v;
  }
  if (!rc) rc = launch_scal_setup(h, h.scal_aux, 0.0, 1, 0, 0);
  return rc;
}

}  // namespace sem
