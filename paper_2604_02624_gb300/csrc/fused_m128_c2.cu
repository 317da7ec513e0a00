// Cluster-resident sweeps for M = 128 (= 8 x 16, 8 threads per line): clusters of 2 CTAs, 16 lines per CTA.
#include "dos_fused.cuh"
namespace dos {
const FusedOps* fused_ops_m128_c2() { return FusedLaunch<Line<8, 16, 8>, 2, 16>::ops(); }
}  // namespace dos
