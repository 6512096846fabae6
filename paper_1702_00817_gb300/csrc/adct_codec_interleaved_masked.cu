// Codec kernels for the interiors of channel-interleaved images (3 or 4
// channels) with edge blocks: full blocks only, the last block column of each
// block row masked (it goes to the edge launch).
#include "adct_codec_kernel.cuh"

namespace adct {

KernelFn pick_interleaved_masked_kernel(int kind, int qmode, bool evenq, int nch) {
  if (nch == 3) return pick_full<3, kEdgeMasked>(kind, qmode, evenq);
  if (nch == 4) return pick_full<4, kEdgeMasked>(kind, qmode, evenq);
  return nullptr;
}

}  // namespace adct
