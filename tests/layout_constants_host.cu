// Prints the shared-memory layout constants of the compiled pass kernels, one
// line per padded size M, as the kernels' own headers define them (compiled
// by nvcc as host code; no kernel is instantiated, no GPU is needed).  The
// bank-mapping checks of tests/test_bank_layout_cpu.py run on these values.
#include <cstdio>

#include "../paper_2604_02624_gb300/csrc/dos_pass_bulk.cuh"

template <int P, int Q, int T, int RL>
static void print_shape() {
  using LF = dos::Line<P, Q, T>;
  using PB = dos::PassBulk<LF, RL, true>;
  using PS = dos::Pass<LF>;
  std::printf(
      "{\"M\": %d, \"P\": %d, \"Q\": %d, \"T\": %d, \"RL\": %d, \"RP\": %d, \"ZS\": %d, \"TWP\": %d, \"TWS\": %d, "
      "\"RZL\": %d, \"SR\": %d, \"COLL\": %d, \"GW\": %d, \"GT\": %d, \"ZX\": %d, \"ZLB\": %d, \"HP\": %d, "
      "\"HB\": %d, \"STAGE_H\": %d, \"SLOT_H\": %d, \"GROUP_BARS\": %d}\n",
      LF::M, P, Q, T, RL, LF::RP, LF::ZS, LF::TWP, LF::TWS, PS::RZL, PB::SR, PS::COLL, PB::GW, PB::GT, PB::ZX,
      PB::ZLB, PB::HP, PB::HB, (int)PB::STAGE_H, (int)PB::SLOT_H, (int)PB::GROUP_BARS);
}

int main() {
  // (M, P, Q, T, rows per block of the bulk row passes) as pass_m*.cu compile them
  print_shape<4, 4, 4, 16>();
  print_shape<4, 8, 4, 16>();
  print_shape<8, 8, 8, 16>();
  print_shape<8, 16, 8, 16>();
  print_shape<10, 20, 10, 16>();
  print_shape<16, 16, 16, 16>();
  print_shape<20, 20, 20, 8>();
  print_shape<16, 32, 16, 8>();
  return 0;
}
