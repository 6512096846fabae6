// Codec kernels for planar images whose sides are not multiples of 8 (edge
// blocks replicate the last column and row), every kind that reads or writes
// pixels, with the full zone.  Images without edge blocks use the kernels of
// adct_codec.cu, which compile the edge handling out.
#include "adct_codec_kernel.cuh"

namespace adct {

KernelFn pick_edge_kernel(int kind, int qmode, bool evenq) { return pick_full<1, kEdgeBlocks>(kind, qmode, evenq); }

}  // namespace adct
