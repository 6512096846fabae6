// Codec kernels for channel-interleaved images (HWC: 3 or 4 channels per
// pixel) with edge blocks, every kind that reads or writes pixels, with the
// full zone.
#include "adct_codec_kernel.cuh"

namespace adct {

KernelFn pick_interleaved_edge_kernel(int kind, int qmode, bool evenq, int nch) {
  if (nch == 3) return pick_full<3, kEdgeBlocks>(kind, qmode, evenq);
  if (nch == 4) return pick_full<4, kEdgeBlocks>(kind, qmode, evenq);
  return nullptr;
}

}  // namespace adct
