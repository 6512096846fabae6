// Zonal kernels specialised on the zone, anti-diagonals 0..4 (r <= 15): split
// from adct_codec.cu so that the instantiations compile in parallel.
#include "adct_codec_kernel.cuh"

namespace adct {

KernelFn pick_zonal_kernel_lo(int kind, int qmode, int zs) {
  switch (zs) {
    case 0: return pick_zone<0>(kind, qmode);
    case 1: return pick_zone<1>(kind, qmode);
    case 2: return pick_zone<2>(kind, qmode);
    case 3: return pick_zone<3>(kind, qmode);
    case 4: return pick_zone<4>(kind, qmode);
    default: return nullptr;
  }
}

}  // namespace adct
