// Zonal kernels specialised on the zone, anti-diagonals 5..8 (16 <= r <= 43): split
// from adct_codec.cu so that the instantiations compile in parallel.
#include "adct_codec_kernel.cuh"

namespace adct {

KernelFn pick_zonal_kernel_hi(int kind, int qmode, int zs) {
  switch (zs) {
    case 5: return pick_zone<5>(kind, qmode);
    case 6: return pick_zone<6>(kind, qmode);
    case 7: return pick_zone<7>(kind, qmode);
    case 8: return pick_zone<8>(kind, qmode);
    default: return nullptr;
  }
}

}  // namespace adct
