// Fused (cluster-resident) configurations compiled for each padded size M.
#include "dos_fused.cuh"

namespace dos {
const FusedOps* fused_ops_m400_c4l16();
const FusedOps* fused_ops_m400_c4l17();
const FusedOps* fused_ops_m400_c5();
const FusedOps* fused_ops_m400_c5l16();
const FusedOps* fused_ops_m400_c8();
const FusedOps* fused_ops_m400_c8l16();
const FusedOps* fused_ops_m400_c10();
const FusedOps* fused_ops_m512_c8();
const FusedOps* fused_ops_m512_c8l8();
const FusedOps* fused_ops_m512_c16();
const FusedOps* fused_ops_m128_c2();
const FusedOps* fused_ops_m128_c4();

int fused_ops_for_m(int m, const FusedOps** out, int cap) {
  const FusedOps* list[16];
  int k = 0;
  switch (m) {
    case 400:
      list[k++] = fused_ops_m400_c5();
      list[k++] = fused_ops_m400_c5l16();
      list[k++] = fused_ops_m400_c4l16();
      list[k++] = fused_ops_m400_c4l17();
      list[k++] = fused_ops_m400_c8();
      list[k++] = fused_ops_m400_c8l16();
      list[k++] = fused_ops_m400_c10();
      break;
    case 512:
      list[k++] = fused_ops_m512_c8();
      list[k++] = fused_ops_m512_c8l8();
      list[k++] = fused_ops_m512_c16();
      break;
    case 128:
      list[k++] = fused_ops_m128_c2();
      list[k++] = fused_ops_m128_c4();
      break;
    default:
      break;
  }
  for (int i = 0; i < k && i < cap; ++i) out[i] = list[i];
  return k;
}
}  // namespace dos
