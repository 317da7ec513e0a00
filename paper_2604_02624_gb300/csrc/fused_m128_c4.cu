// Cluster-resident sweeps for M = 128 (= 8 x 16, 8 threads per line): clusters of 4 CTAs, 16 lines per CTA.
#include "dos_fused.cuh"
namespace dos {
const FusedOps* fused_ops_m128_c4() { return FusedLaunch<Line<8, 16, 8>, 4, 16>::ops(); }
}  // namespace dos
