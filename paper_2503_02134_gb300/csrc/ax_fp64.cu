// FP64 instantiations of the element operator (plain and PCG-fused).
#include "ax_kernel.cuh"

namespace sem {

template <int n>
static int run64(Handle& h, const double* u, double* w, const AxPrologue* pro) {
  if (pro) return ax_launch<n, double, true, kDotFP64>(h, u, w, h.G64, h.D64, pro);
  return ax_launch<n, double, false, kDotFP64>(h, u, w, h.G64, h.D64, nullptr);
}

int ax_dispatch_fp64(Handle& h, const double* u, double* w, const AxPrologue* pro) {
  switch (h.n) {
    case 2: return run64<2>(h, u, w, pro);
    case 3: return run64<3>(h, u, w, pro);
    case 4: return run64<4>(h, u, w, pro);
    case 5: return run64<5>(h, u, w, pro);
    case 6: return run64<6>(h, u, w, pro);
    case 7: return run64<7>(h, u, w, pro);
    case 8: return run64<8>(h, u, w, pro);
    case 9: return run64<9>(h, u, w, pro);
    case 10: return run64<10>(h, u, w, pro);
    case 11: return run64<11>(h, u, w, pro);
    case 12: return run64<12>(h, u, w, pro);
    case 13: return run64<13>(h, u, w, pro);
    case 14: return run64<14>(h, u, w, pro);
    case 15: return run64<15>(h, u, w, pro);
    case 16: return run64<16>(h, u, w, pro);
    default: set_error("ax: unsupported order"); return SEM_EINVAL;
  }
}

}  // namespace sem
