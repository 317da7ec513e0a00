// Cluster-resident sweeps for M = 400 (= 20 x 20, 20 threads per line): clusters of 5 CTAs, 20 lines per CTA.
#include "dos_fused.cuh"
namespace dos {
const FusedOps* fused_ops_m400_c5() { return FusedLaunch<Line<20, 20, 20>, 5, 20>::ops(); }
}  // namespace dos
