// Cluster-resident sweeps for M = 400 (= 20 x 20, 20 threads per line): clusters of 4 CTAs, 17 lines per CTA.
#include "dos_fused.cuh"
namespace dos {
const FusedOps* fused_ops_m400_c4l17() { return FusedLaunch<Line<20, 20, 20>, 4, 17>::ops(); }
}  // namespace dos
