// Cluster-resident sweeps for M = 400 (= 20 x 20, 20 threads per line): clusters of 8 CTAs, 16 lines per CTA.
#include "dos_fused.cuh"
namespace dos {
const FusedOps* fused_ops_m400_c8l16() { return FusedLaunch<Line<20, 20, 20>, 8, 16>::ops(); }
}  // namespace dos
