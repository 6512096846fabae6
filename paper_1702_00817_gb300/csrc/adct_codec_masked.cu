// Codec kernels for the interiors of planar images with edge blocks: every
// block has 8 x 8 valid pixels, and each block row runs over the whole
// coefficient row with its last block column masked (that column goes to
// the edge launch), so that tiles stay aligned with the image's rows.
#include "adct_codec_kernel.cuh"

namespace adct {

KernelFn pick_masked_kernel(int kind, int qmode, bool evenq) { return pick_full<1, kEdgeMasked>(kind, qmode, evenq); }

}  // namespace adct
