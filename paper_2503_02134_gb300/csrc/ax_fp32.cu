// FP32 instantiations of the element operator (CUDA cores), plain and PCG-fused
// with the compensated (Dot2) or the plain FP32 pap reduction.
#include "ax_tma.cuh"

namespace sem {

static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

template <int n>
static int run32(Handle& h, const float* u, float* w, const AxPrologue* pro, int dm) {
  // bulk-copy staged kernel: even n (16-byte element blocks) up to n = 10
  if constexpr (n % 2 == 0 && n <= 10) {
    const bool ok = h.use_tma && aligned16(u) && aligned16(w) &&
                    (!pro || (aligned16(pro->r) && aligned16(pro->minv)));
    if (ok) {
      if (!pro) return ax_tma_launch<n, false, kDotDot2>(h, u, w, nullptr);
      if (dm == kDotFP32) return ax_tma_launch<n, true, kDotFP32>(h, u, w, pro);
      return ax_tma_launch<n, true, kDotDot2>(h, u, w, pro);
    }
  }
  if (!pro) return ax_launch<n, float, false, kDotDot2>(h, u, w, h.G32, h.D32, nullptr);
  if (dm == kDotFP32) return ax_launch<n, float, true, kDotFP32>(h, u, w, h.G32, h.D32, pro);
  return ax_launch<n, float, true, kDotDot2>(h, u, w, h.G32, h.D32, pro);
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
