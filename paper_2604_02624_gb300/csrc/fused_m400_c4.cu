// Cluster-resident sweeps for M = 400 (= 20 x 20, 20 threads per line): clusters of 4 CTAs, 10 lines per CTA.
#include "dos_fused.cuh"
namespace dos {
const FusedOps* fused_ops_m400_c4() { return FusedLaunch<Line<20, 20, 20>, 4, 10>::ops(); }
}  // namespace dos
