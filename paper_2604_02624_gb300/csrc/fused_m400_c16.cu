// Cluster-resident sweeps for M = 400 (= 20 x 20, 20 threads per line): clusters of 16 CTAs, 13 lines per CTA.
#include "dos_fused.cuh"
namespace dos {
const FusedOps* fused_ops_m400_c16() { return FusedLaunch<Line<20, 20, 20>, 16, 13>::ops(); }
}  // namespace dos
