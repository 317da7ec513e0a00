// Dispatch from the padded size M to its compiled row/column pass kernels.
#include "dos_internal.h"

namespace dos {
const PassOps* pass_ops_16();
const PassOps* pass_ops_32();
const PassOps* pass_ops_64();
const PassOps* pass_ops_128();
const PassOps* pass_ops_200();
const PassOps* pass_ops_256();
const PassOps* pass_ops_400();
const PassOps* pass_ops_512();

static const int kSupported[] = {16, 32, 64, 128, 200, 256, 400, 512};

const PassOps* pass_ops_for_m(int m) {
  switch (m) {
    case 16: return pass_ops_16();
    case 32: return pass_ops_32();
    case 64: return pass_ops_64();
    case 128: return pass_ops_128();
    case 200: return pass_ops_200();
    case 256: return pass_ops_256();
    case 400: return pass_ops_400();
    case 512: return pass_ops_512();
    default: return nullptr;
  }
}

int supported_m_list(int* out, int cap) {
  const int n = (int)(sizeof(kSupported) / sizeof(kSupported[0]));
  for (int i = 0; i < n && i < cap; ++i) out[i] = kSupported[i];
  return n;
}
}  // namespace dos
