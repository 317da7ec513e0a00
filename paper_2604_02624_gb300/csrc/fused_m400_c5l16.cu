// Cluster-resident sweeps for M = 400 (= 20 x 20, 20 threads per line): clusters of 5 CTAs, 16 lines per CTA.
#include "dos_fused.cuh"
namespace dos {
const FusedOps* fused_ops_m400_c5l16() { return FusedLaunch<Line<20, 20, 20>, 5, 16>::ops(); }
}  // namespace dos
