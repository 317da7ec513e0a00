// Cluster-resident sweeps for M = 400 (= 20 x 20, 20 threads per line): clusters of 4 CTAs, 16 lines per CTA.
#include "dos_fused.cuh"
namespace dos {
const FusedOps* fused_ops_m400_c4l16() { return FusedLaunch<Line<20, 20, 20>, 4, 16>::ops(); }
}  // namespace dos
