// Cluster-resident sweeps for M = 512 (= 16 x 32, 16 threads per line): clusters of 8 CTAs, 8 lines per CTA.
#include "dos_fused.cuh"
namespace dos {
const FusedOps* fused_ops_m512_c8l8() { return FusedLaunch<Line<16, 32, 16>, 8, 8>::ops(); }
}  // namespace dos
