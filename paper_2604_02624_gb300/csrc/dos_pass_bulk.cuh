// dos_pass_bulk.cuh - the multi-pass row and column passes with bulk-async prefetch.
//
// Same arithmetic as dos_pass.cuh; what changes is how the input reaches the
// block.  Blocks loop over several work items and the bulk-copy engine
// (cp.async.bulk global -> shared, completion counted in bytes on an
// mbarrier) fetches the next item while the block computes the current one:
//   column pass : item = a mirrored pair of 8-column groups of one channel
//                 (persistent blocks); tensor copies (TMA) of both groups'
//                 input rows and of the transfer-table tile they share;
//   row passes  : item = the block's RL rows of the next channel of its chunk;
//                 one cp.async.bulk per row (rows padded in shared memory
//                 against bank conflicts): spectra rows, the rows of the
//                 input-field table in the first forward pass, and spectra
//                 plus checkpoint rows in the adjoint pass.
// One staging buffer per input suffices: the item is moved from the stage to
// registers and the next copy is issued at the first block barrier after
// that (the one inside the item's first line DFT), so the copy overlaps most
// of the item's DFT / modulation / DFT / store.
// Every wait is bounded (one second of global time).  Each thread times its
// own wait, and the block takes one verdict from them (a block-wide AND at the
// barrier after the wait), so that no thread goes on with an item another
// thread gave up on: when any wait expires the whole block issues no further
// copy, leaves its loop without writing partial results, waits once more
// (bounded) for the copy it was waiting for (its only one in flight) and sets
// *err.
// PassArgs::stall (fault injection for tests): 1 makes the blocks announce
// their bytes without copying them, so that the first wait of every block
// expires; 2 lets the copies land but makes the odd threads of every block
// give up their first wait (a split verdict that the block-wide AND resolves).
#pragma once

#include <cuda.h>

#include <algorithm>
#include <cstdint>

#include "dos_pass.cuh"

namespace dos {

constexpr unsigned long long kBulkWaitNs = 1000000000ull;  // bounded wait: one second
constexpr long kBulkSpin = 1L << 30;                        // and an iteration cap behind it

__device__ __forceinline__ uint32_t sh_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
// First 16-byte boundary at or after p: the line DFTs read the twiddle table
// in 16-byte pairs (the layouts reserve one extra float2 for the shift).
__device__ __forceinline__ float2* tw_align(float2* p) { return p + ((sh_addr(p) >> 3) & 1u); }

__device__ __forceinline__ void bulk_bar_init(uint64_t* b) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sh_addr(b)));
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void bulk_expect(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sh_addr(b)), "r"(bytes) : "memory");
}
// global -> shared copy of `bytes` (multiple of 16, both addresses 16-byte aligned)
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* b) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   sh_addr(dst)),
               "l"(src), "r"(bytes), "r"(sh_addr(b))
               : "memory");
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// true once the phase with this parity has completed; false after kBulkWaitNs
// (or at once when `give_up` is set: the injected split verdict of the tests)
__device__ __forceinline__ bool bulk_wait(uint64_t* b, uint32_t parity, bool give_up = false) {
  if (give_up) return false;
  const unsigned long long t0 = global_ns();
  for (long it = 0; it < kBulkSpin; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(sh_addr(b)), "r"(parity)
        : "memory");
    if (done) return true;
    if ((it & 15) == 15 && global_ns() - t0 > kBulkWaitNs) return false;
  }
  return false;
}

// Injected split verdict (PassArgs::stall == 2, tests only): the odd threads
// of every block give up their first wait although the copy lands.
__device__ __forceinline__ bool split_verdict(const PassArgs& a, int item) {
  return a.stall == 2 && item == 0 && (threadIdx.x & 1);
}

// Row stride of the row passes' staging buffer: a warp reads the rows of two
// or more lines at once, and these strides make those 8-byte reads free of
// bank conflicts (enumerated on the host for the compiled line shapes).
constexpr int row_stage_stride(int m) {
  return m == 400 ? 404 : m == 200 ? 202 : m == 128 ? 132 : m == 64 ? 68 : m == 32 ? 34 : m == 16 ? 18 : m;
}

// HALF: the pruned line DFTs and field-half loops of Pass<LF, true> (N <= M / 2).
template <class LF, int RL, bool HALF = false>
struct PassBulk {
  static constexpr int T = LF::T, E = LF::E, M = LF::M;
  static constexpr int NZF = Pass<LF, HALF>::NZF, NOI = Pass<LF, HALF>::NOI, EF = Pass<LF, HALF>::EF;
  // packed FP32-pair butterflies in every bulk pass (faster than scalar ones
  // in each of them on the 400-point line)
  static constexpr bool PKR = true, PKC = true;
  static constexpr int COLL = Pass<LF>::COLL, ZL = Pass<LF>::ZL, RZL = Pass<LF>::RZL;
  static constexpr int SR = row_stage_stride(M);  // even: every staged row starts 16-byte aligned
  static_assert(SR % 2 == 0 && SR >= M, "staged rows must be 16-byte aligned and hold M values");
  static_assert(Pass<LF>::RZL >= LF::ZS, "exchange buffers must not overlap");
  static constexpr int CT = T * COLL, RT = T * RL;

  // ------------------------------------------------------------ column pass
  // An item is a mirrored pair of column groups of one channel: columns
  // c0 .. c0+7 (lines 0-7) and M-c0-8 .. M-c0-1 (lines 8-15), c0 = 8 p for
  // p < M/16.  H depends on |kx| only, and the two groups' |kx| are c0 .. c0+8,
  // so one tile of 10 |kx| values (c0 .. c0+9) serves all 16 columns.  The
  // quadrant table is symmetric, H(|ky|, |kx|) = H(|kx|, |ky|) (the setup forms
  // q = k^2 - (fx^2 + fy^2), the same in either order), so the tile is fetched
  // as the table's rows c0 .. c0+9, all M/2 + 2 entries each (box {M/2+2, 10,
  // 1}; a row is a 16-byte multiple), and held as tile[|kx| - c0][|ky|]: then
  // the 16 reads of a half-warp (8 lines x 2 element owners) fall on distinct
  // bank pairs.  Per item, three tensor copies: the two groups' input rows (box
  // {8, in_r1 - in_r0, 1} of the row spectra, one dense [rows][8] block per
  // group) and the H tile.  The spectra of the next item are fetched at the
  // barrier inside the forward DFT (the stage has been read) and waited for at
  // the top of the item, with one block-wide verdict; the H tile of an item is
  // fetched at its top (every thread is past the previous item's multiply)
  // and waited for just before the H multiply, so its copy overlaps the
  // forward DFT.  A thread whose H wait expires marks a shared flag (its
  // item's results are then invalid, and reported so) that the next
  // block-wide verdict reads.
  static constexpr int GW = Pass<LF>::COLL / 2;       // columns per group
  static constexpr int HW = GW + 2;                   // |kx| values per H tile (c0 .. c0+9)
  static constexpr int HP = M / 2 + 2;                // quadrant pitch (rows and columns)
  static_assert(GW == 8, "column groups of 8");
  // The H tile is staged in a region of its own where the block still fits
  // twice on an SM with it and a table row fits one box (M <= 400: 96.8 KB
  // at N = 200).  At M = 512 the exchange buffers alone take 66 KB and a
  // separate tile would leave one block per SM, so each group stages its own
  // 8 rows of the table in its stage slot instead (SLOT_H): the copy is
  // issued once the group's input rows are in registers (at the barrier
  // inside the forward DFT) and waited for just before the H multiply, and
  // the next item's input rows are fetched at the barrier inside the inverse
  // DFT, when the group is past its H reads.  A table row of M/2 + 2 > 256
  // entries is then two boxes of HB entries, at x = 0 and x = HP - HB.
  static constexpr bool STAGE_H = M <= 400;
  static constexpr bool SLOT_H = !STAGE_H;
  static_assert(!STAGE_H || HP <= 256, "a staged H tile row is one box row (at most 256 entries)");
  static constexpr int HTILE = STAGE_H ? HW * HP : 0;  // float2 of the H tile in shared memory
  static_assert(HTILE % 2 == 0, "the exchange buffers after the tile start 16-byte aligned");
  static constexpr int HB = (HP / 2 + 1) / 2 * 2;         // SLOT_H box width: even (16-byte box rows)
  static constexpr int HSLOT = SLOT_H ? 2 * GW * HB : 0;  // float2 of a group's H tile: [2 boxes][8][HB]
  static_assert(!SLOT_H || (HB <= 256 && (HP - HB) % 2 == 0 && 2 * HB >= HP),
                "two 16-byte aligned boxes cover a table row");
  // every register's |ky| range (over the T element owners) lies in one box
  static constexpr bool slot_boxes_cover() {
    for (int i = 0; i < E; ++i) {
      const int lo = i < E / 2 ? T * i : M - T * i - T + 1, hi = i < E / 2 ? T * i + T - 1 : M - T * i;
      if (!(hi < HB || lo >= HP - HB)) return false;
    }
    return true;
  }
  static_assert(!SLOT_H || slot_boxes_cover(), "each register's H values come from one box");
  // group stride in the stage (float2): whole 128-byte lines for any row
  // count, and room for the group's H tile under SLOT_H
  __host__ __device__ static int col_group_stride(int rows) {
    const int s = (rows + 1) / 2 * 2 * GW, h = (HSLOT + 15) / 16 * 16;
    return s > h ? s : h;
  }
  // The two groups of an item share only the H tile: a group's 8 lines are
  // held by warps of their own (thread = group g, line lc, element owner t:
  // g = tid / GT, lc = tid % 8, t = (tid % GT) / 8), so the exchanges inside
  // the line DFTs synchronise the group's warps on a named barrier, and only
  // the top of an item is a block-wide barrier.  With GT not a multiple of the
  // warp size (M = 200) the groups share warps and the block barrier serves.
  static constexpr int GT = GW * T;                    // threads of a group
  static constexpr bool GROUP_BARS = GT % 32 == 0;
  // Exchange matrices of the column lines: even pitch ZX (row entries k1,
  // k1 + 1 are one 16-byte access), stride ZLB between the lines at least
  // Q ZX and 2 mod 16.  A group warp holds 8 lines x 4 consecutive element
  // owners; its 8-byte accesses (the column side of either layout) then fall
  // on distinct bank pairs in each half-warp (8 lines x 2 owners) and its
  // 16-byte ones (the row side) on distinct bank quads in each quarter-warp
  // (8 lines, one owner).
  static constexpr int ZX = LF::P + (LF::P & 1), ZSX = LF::Q * ZX;
  static constexpr int ZLB = ZSX + ((2 - ZSX % 16) + 16) % 16;
  static_assert(ZX % 2 == 0 && ZLB % 16 == 2, "16-byte aligned rows, conflict-free line stride");
  __device__ static __forceinline__ void group_sync(int g) {
    if constexpr (GROUP_BARS) {
      // g is uniform over a warp; immediate barrier ids keep the count of
      // barriers the kernel reserves at three
      if (g == 0) asm volatile("bar.sync 1, %0;" ::"n"(GT) : "memory");
      else asm volatile("bar.sync 2, %0;" ::"n"(GT) : "memory");
    } else {
      __syncthreads();
    }
  }
  // dynamic shared memory (from a 128-byte aligned base):
  //   stage[2][rows][8] | H tile[10][M/2+2] | exchange[COLL][ZLB] | tw[TWS] | barrier[4] | flag
  static size_t col_smem(int n) {
    return 128 + sizeof(float2) * (2 * (size_t)col_group_stride(n) + (size_t)HTILE + (size_t)COLL * ZLB +
                                   LF::TWS + 1) + 4 * sizeof(uint64_t) + sizeof(int);
  }

  template <bool ADJ>
  __device__ static void col(const PassArgs& a, const CUtensorMap* smap, const CUtensorMap* hmap) {
    extern __shared__ __align__(16) unsigned char col_raw[];
    // 128-byte aligned start, by pointer arithmetic on the shared array: the
    // compiler keeps seeing shared-memory pointers (an integer round trip
    // would turn every access below into a generic one)
    float2* stage = reinterpret_cast<float2*>(col_raw + ((128u - (sh_addr(col_raw) & 127u)) & 127u));
    const int GS = col_group_stride(a.n);
    float2* htile = stage + 2 * (size_t)GS;
    float2* zb = htile + HTILE;
    float2* tw = tw_align(zb + (size_t)COLL * ZLB);
    // [0], [1] spectra of group 0, 1; [2] transfer-table tile (STAGE_H), or
    // [2], [3] the H tiles of group 0, 1 (SLOT_H)
    uint64_t* bar = reinterpret_cast<uint64_t*>(tw + LF::TWS);
    int* h_late = reinterpret_cast<int*>(bar + 4);  // an H wait of this block expired
    const int g = threadIdx.x / GT, lc = threadIdx.x % GW, t = (threadIdx.x % GT) / GW;
    const bool leader = threadIdx.x % GT == 0;  // issues the group's copies
    float2* z = zb + (g * GW + lc) * ZLB;
    constexpr int npairs = M / (2 * GW);
    const int items = a.nw * npairs;
    const uint32_t sbytes = GW * 8u * (uint32_t)(a.in_r1 - a.in_r0);
    constexpr uint32_t hbytes = (uint32_t)HW * HP * 8u;
    constexpr uint32_t hsbytes = (uint32_t)HSLOT * 8u;
    if (threadIdx.x == 0) {
      bulk_bar_init(&bar[0]);
      bulk_bar_init(&bar[1]);
      bulk_bar_init(&bar[2]);
      bulk_bar_init(&bar[3]);
      *h_late = 0;
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(smap)) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(hmap)) : "memory");
    }
    for (int i = threadIdx.x; i < LF::TWS; i += blockDim.x) tw[i] = a.tw[i];
    __syncthreads();
    auto tensor_copy = [](float2* dst, const CUtensorMap* map, int x, int y, int zc, uint64_t* b) {
      asm volatile(
          "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
          "[%5];" ::"r"(sh_addr(dst)),
          "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(zc), "r"(sh_addr(b))
          : "memory");
    };
    // the input rows of group gg of item it (its leader)
    auto fetch_s = [&](int it, int gg) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      bulk_expect(&bar[gg], sbytes);
      if (a.stall == 1) return;  // injected fault: the expected bytes never arrive
      const int w = it / npairs, c0 = GW * (it % npairs);
      tensor_copy(stage + gg * GS, smap, gg == 0 ? c0 : M - c0 - GW, a.in_r0, a.tmap_w0 + w, &bar[gg]);
    };
    // the H tile of item it (thread 0)
    auto fetch_h = [&](int it) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      bulk_expect(&bar[2], hbytes);
      if (a.stall == 1) return;
      const int w = it / npairs, c0 = GW * (it % npairs);
      tensor_copy(htile, hmap, 0, c0, a.hmap_z0 + w, &bar[2]);
    };
    // the 8 table rows |kx| = c0 + gg .. c0 + gg + 7 that group gg of item it
    // reads, into its stage slot (its leader; SLOT_H)
    auto fetch_hs = [&](int it, int gg) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      bulk_expect(&bar[2 + gg], hsbytes);
      if (a.stall == 1) return;
      const int w = it / npairs, c0 = GW * (it % npairs);
      float2* dst = stage + gg * GS;
      tensor_copy(dst, hmap, 0, c0 + gg, a.hmap_z0 + w, &bar[2 + gg]);
      tensor_copy(dst + GW * HB, hmap, HP - HB, c0 + gg, a.hmap_z0 + w, &bar[2 + gg]);
    };
    bool ok = true;
    int k = 0;
    if ((int)blockIdx.x < items && leader) fetch_s(blockIdx.x, g);
    for (int it = blockIdx.x; it < items; it += gridDim.x, ++k) {
      const int w = it / npairs, c0 = GW * (it % npairs);
      const int cc = g == 0 ? c0 + lc : M - c0 - GW + lc;  // this line's column
      const int hc = g == 0 ? lc : GW - lc;                 // its |kx| - c0: the column in the H tile
      // this group's input rows, and no expired H wait in the previous item
      const bool got = bulk_wait(&bar[g], (uint32_t)(k & 1), split_verdict(a, k)) && *h_late == 0;
      ok = __syncthreads_and(got) != 0;  // one verdict for the whole block
      if (!ok) break;
      // every thread is past the previous item's H multiply: this item's tile
      // may land (it is waited for just before the multiply)
      if (STAGE_H && threadIdx.x == 0) fetch_h(it);
      float2 r[E];
      const float2* sg = stage + (size_t)g * GS + lc - (ptrdiff_t)a.in_r0 * GW;  // row y at sg[y * GW]
#pragma unroll
      for (int i = 0; i < E; ++i) {
        const int row = t + T * i;
        r[i] = (i < EF && row >= a.in_r0 && row < a.in_r1) ? sg[row * GW] : czero();
      }
      LF::template step1<false, NZF, PKC, false, ZX>(r, t, z, tw);
      group_sync(g);  // the group is past its stage reads: its next rows (or its H tile) may land there
      if constexpr (SLOT_H) {
        if (leader) fetch_hs(it, g);
      } else {
        if (leader && it + (int)gridDim.x < items) fetch_s(it + gridDim.x, g);
      }
      LF::template step2<false, LF::Q, PKC, false, ZX>(r, t, z);
      // square lines: the inverse DFT below writes the exchange matrix in
      // the transposed layout, i.e. only what this thread just read
      if constexpr (!LF::SQUARE) group_sync(g);
      // H(|ky|, |kx|) from the tile: |ky| = k below M/2 and M - k above, both
      // affine in i at compile time
      // (injected, tests: the wait of the block's last item gives up)
      const bool give_up_h = a.stall == 3 && it + (int)gridDim.x >= items;
      if (STAGE_H && !bulk_wait(&bar[2], (uint32_t)(k & 1), give_up_h)) *h_late = 1;
      if (SLOT_H && !bulk_wait(&bar[2 + g], (uint32_t)(k & 1), give_up_h)) *h_late = 1;
      // STAGE_H: tile[hc][|ky|] (pitch HP).  SLOT_H: box b of the group's
      // tile, [hc - g][|ky| - b (HP - HB)] (pitch HB); box 0 holds |ky| < HB,
      // box 1 |ky| >= HP - HB, and which one a register's |ky| range lies in
      // is known at compile time.
      const float2* hlo = STAGE_H ? htile + hc * HP + t : stage + (size_t)g * GS + (hc - g) * HB + t;
      const float2* hhi = STAGE_H ? htile + hc * HP + (M - t) : stage + (size_t)g * GS + (hc - g) * HB + (M - t);
      const float* Sw = a.mis.sq ? a.mis.sq + (size_t)w * a.hs * a.hs : nullptr;
#pragma unroll
      for (int i = 0; i < E; ++i) {
        float2 h;
        if constexpr (STAGE_H) {
          h = i < E / 2 ? hlo[T * i] : hhi[-T * i];
        } else {
          // |ky| in [T i, T i + T - 1] (i < E/2) or [M - T i - T + 1, M - T i]
          constexpr int B1 = GW * HB - (HP - HB);  // offset of box 1, less its first |ky|
          if (i < E / 2) h = T * i + T - 1 < HB ? hlo[T * i] : hlo[B1 + T * i];
          else h = M - T * i < HB ? hhi[-T * i] : hhi[B1 - T * i];
        }
        if (Sw) {
          const int kk = t + T * i;
          h = cmul(h, misalign_factor(a.mis, kk, cc, M, Sw[(size_t)min(kk, M - kk) * a.hs + c0 + hc]));
        }
        r[i] = ADJ ? cmulc(r[i], h) : cmul(r[i], h);
      }
      LF::template step1<true, LF::P, PKC, LF::SQUARE, ZX>(r, t, z, tw);
      group_sync(g);
      // SLOT_H: the group is past its H reads: its next rows may land in the slot
      if (SLOT_H && leader && it + (int)gridDim.x < items) fetch_s(it + gridDim.x, g);
      // no trailing barrier: the exchange buffer is next written after the
      // barrier at the top of the next item
      LF::template step2<true, NOI, PKC, LF::SQUARE, ZX>(r, t, z);
      float2* dst = a.S + (size_t)w * a.n * M + cc;
#pragma unroll
      for (int i = 0; i < E; ++i) {
        const int row = t + T * i;
        if (i < EF && row >= a.out_r0 && row < a.out_r1) dst[(size_t)row * M] = r[i];
      }
    }
    // An H wait that expired in the block's last item has no later verdict
    // to read it: every thread (the loop ends for all of them together)
    // takes it here.
    const bool late = __syncthreads_or(*h_late != 0) != 0;
    if ((!ok || late) && threadIdx.x == 0) {
      // The copies in flight land (bounded) before the block leaves: after a
      // failed verdict at item k both groups' rows of item k, and after an
      // expired H wait in item k - 1 that tile (no tile of item k was issued).
      if (!ok) {
        (void)bulk_wait(&bar[0], (uint32_t)(k & 1));
        (void)bulk_wait(&bar[1], (uint32_t)(k & 1));
      }
      if (STAGE_H && late) (void)bulk_wait(&bar[2], (uint32_t)((k - 1) & 1));
      if (SLOT_H && late) {
        (void)bulk_wait(&bar[2], (uint32_t)((k - 1) & 1));
        (void)bulk_wait(&bar[3], (uint32_t)((k - 1) & 1));
      }
      atomicExch(a.err, 1);
    }
  }

  // ------------------------------------------------------------- row passes
  // dynamic shared memory: stage[RL][SR] | exchange[RL][RZL] | tw[TWS] | barrier
  static size_t row_smem() {
    return sizeof(float2) * ((size_t)RL * SR + (size_t)RL * RZL + LF::TWS + 1) + sizeof(uint64_t);
  }

  // Rows [blockIdx.x * RL, +RL) of the channels of chunk blockIdx.y.
  //   ADJ false : forward layer pass (as Pass::row_fwd), FLAG = save the checkpoint
  //   ADJ true  : adjoint layer pass (as Pass::row_adj), FLAG = first layer; it
  //               runs only for odd N (the checkpoint rows are then not 16-byte
  //               multiples and are read directly), row_adj_staged otherwise
  template <bool ADJ, bool FLAG>
  __device__ static void row(const PassArgs& a) {
    extern __shared__ __align__(16) float2 smem[];
    float2* stage = smem;
    float2* zb = stage + (size_t)RL * SR;
    float2* tw = tw_align(zb + (size_t)RL * RZL);
    uint64_t* bar = reinterpret_cast<uint64_t*>(tw + LF::TWS);
    const int l = threadIdx.x / T, t = threadIdx.x % T;
    float2* z = zb + l * RZL;
    const int r0 = blockIdx.x * RL;
    const int nrows = min(RL, a.n - r0);
    const int row = r0 + l;
    const bool ok = l < nrows;
    const int rr = ok ? row : r0;
    const int w0 = blockIdx.y * a.chunk;
    const int w1 = min(a.nw, w0 + a.chunk);
    const uint32_t bytes = (uint32_t)nrows * M * 8u;
    if (threadIdx.x == 0) bulk_bar_init(bar);
    for (int i = threadIdx.x; i < LF::TWS; i += blockDim.x) tw[i] = a.tw[i];
    __syncthreads();
    // thread 0 copies the block's rows of channel w, one bulk copy (M * 8 bytes) per row
    auto fetch = [&](int w) {
      if (threadIdx.x != 0) return;
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      bulk_expect(bar, bytes);
      if (a.stall == 1) return;  // injected fault: the expected bytes never arrive
      const float2* src = a.S + ((size_t)w * a.n + r0) * M;
      for (int q = 0; q < nrows; ++q) bulk_g2s(stage + (size_t)q * SR, src + (size_t)q * M, M * 8u, bar);
    };
    // the thickness row is held in registers by the forward pass; the adjoint
    // pass (which also carries its gradient and the checkpoint) re-reads it
    // from L1 per channel
    const float* hrow = a.h + (size_t)rr * a.n;
    float hv[ADJ ? 1 : E];
    if constexpr (!ADJ) {
#pragma unroll
      for (int i = 0; i < E; ++i) {
        const int x = t + T * i;
        hv[i] = (i < EF && x < a.n) ? __ldg(hrow + x) : 0.f;
      }
    }
    float g[E];
#pragma unroll
    for (int i = 0; i < E; ++i) g[i] = 0.f;
    bool okw = true;
    if (w0 < w1) fetch(w0);
    int k = 0;
    // the next channel's constants are loaded one iteration ahead
    ChanConst cnext = a.chan[w0 < w1 ? w0 : 0];
    for (int w = w0; w < w1; ++w, ++k) {
      const ChanConst cc = cnext;
      if (w + 1 < w1) cnext = a.chan[w + 1];
      okw = __syncthreads_and(bulk_wait(bar, (uint32_t)(k & 1), split_verdict(a, k))) != 0;  // one verdict for the whole block
      if (!okw) break;
      float2 r[E];
#pragma unroll
      for (int i = 0; i < E; ++i) r[i] = stage[(size_t)(ok ? l : 0) * SR + t + T * i];
      LF::template step1<true, LF::P, PKR>(r, t, z, tw);
      __syncthreads();  // every thread is past its stage reads: the next channel may land there
      if (w + 1 < w1) fetch(w + 1);
      LF::template step2<true, NOI, PKR>(r, t, z);
      // square lines: the forward DFT below writes the exchange matrix in the
      // transposed layout (only what this thread just read); the adjoint's
      // forward DFT does too
      if constexpr (!LF::SQUARE) __syncthreads();
      float2* srow = a.S + ((size_t)w * a.n + rr) * M;
      if constexpr (!ADJ) {
        float2* ck = a.ckpt + ((size_t)w * a.n + rr) * a.n;
#pragma unroll
        for (int i = 0; i < E; ++i) {
          const int x = t + T * i;
          if (i < EF && x < a.n) {
            const float2 v = r[i];
            if (FLAG && ok) ck[x] = v;
            r[i] = cmul(transmission(hv[i], cc), v);
          } else {
            r[i] = czero();
          }
        }
        LF::template fft<false, NZF, LF::Q, false, PKR, LF::SQUARE>(r, t, z, tw);
        if (ok) {
#pragma unroll
          for (int i = 0; i < E; ++i) srow[t + T * i] = r[i];
        }
      } else {
        const float2* ck = a.ckpt + ((size_t)w * a.n + rr) * a.n;
#pragma unroll
        for (int i = 0; i < E; ++i) {
          const int x = t + T * i;
          if (i < EF && x < a.n) {
            const float2 au = r[i];
            const float2 tt = transmission(__ldg(hrow + x), cc);
            const float2 cu = cmul(make_float2(cc.c_re, cc.c_im), cmul(tt, ck[x]));
            g[i] = fmaf(au.x, cu.x, fmaf(au.y, cu.y, g[i]));
            r[i] = cmulc(au, tt);
          } else {
            r[i] = czero();
          }
        }
        if constexpr (!FLAG) {
          LF::template fft<false, NZF, LF::Q, false, PKR, LF::SQUARE>(r, t, z, tw);
          if (ok) {
#pragma unroll
            for (int i = 0; i < E; ++i) srow[t + T * i] = r[i];
          }
        }
      }
    }
    if (!okw) {
      if (threadIdx.x == 0) {
        (void)bulk_wait(bar, (uint32_t)(k & 1));  // a late copy lands (bounded) before the block leaves
        atomicExch(a.err, 1);
      }
      return;
    }
    if constexpr (ADJ) {
      if (ok) {
        float* prow = a.partial + ((size_t)blockIdx.y * a.n + row) * a.n;
#pragma unroll
        for (int i = 0; i < E; ++i) {
          const int x = t + T * i;
          if (i < EF && x < a.n) prow[x] = g[i];
        }
      }
    }
  }

  // -------------------------------------------------------- first row pass
  // t(h) * v1 -> pad -> DFT (as Pass::row_first) with the next channel's rows
  // of the input-field table v1 (fin) staged by bulk copies.  Needs N even.
  // dynamic shared memory: stage[RL][cks] | exchange[RL][RZL] | tw[TWS] | barrier
  static size_t first_smem(int n) {
    return sizeof(float2) * ((size_t)RL * ck_stride(n) + (size_t)RL * RZL + LF::TWS + 1) + sizeof(uint64_t);
  }

  __device__ static void row_first_staged(const PassArgs& a) {
    extern __shared__ __align__(16) float2 smem[];
    const int cks = ck_stride(a.n);
    float2* stage = smem;
    float2* zb = stage + (size_t)RL * cks;
    float2* tw = tw_align(zb + (size_t)RL * RZL);
    uint64_t* bar = reinterpret_cast<uint64_t*>(tw + LF::TWS);
    const int l = threadIdx.x / T, t = threadIdx.x % T;
    float2* z = zb + l * RZL;
    const int r0 = blockIdx.x * RL;
    const int nrows = min(RL, a.n - r0);
    const int row = r0 + l;
    const bool ok = l < nrows;
    const int rr = ok ? row : r0;
    const int lr = ok ? l : 0;
    const int w0 = blockIdx.y * a.chunk;
    const int w1 = min(a.nw, w0 + a.chunk);
    const uint32_t bytes = (uint32_t)nrows * a.n * 8u;
    if (threadIdx.x == 0) bulk_bar_init(bar);
    for (int i = threadIdx.x; i < LF::TWS; i += blockDim.x) tw[i] = a.tw[i];
    __syncthreads();
    auto fetch = [&](int w) {
      if (threadIdx.x != 0) return;
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      bulk_expect(bar, bytes);
      if (a.stall == 1) return;  // injected fault: the expected bytes never arrive
      const float2* src = a.fin + ((size_t)w * a.n + r0) * a.n;
      for (int q = 0; q < nrows; ++q) bulk_g2s(stage + (size_t)q * cks, src + (size_t)q * a.n, a.n * 8u, bar);
    };
    const float* hrow = a.h + (size_t)rr * a.n;
    float hv[E];
#pragma unroll
    for (int i = 0; i < E; ++i) {
      const int x = t + T * i;
      hv[i] = (i < EF && x < a.n) ? __ldg(hrow + x) : 0.f;
    }
    bool okw = true;
    if (w0 < w1) fetch(w0);
    int k = 0;
    // the next channel's constants are loaded one iteration ahead
    ChanConst cnext = a.chan[w0 < w1 ? w0 : 0];
    for (int w = w0; w < w1; ++w, ++k) {
      const ChanConst cc = cnext;
      if (w + 1 < w1) cnext = a.chan[w + 1];
      okw = __syncthreads_and(bulk_wait(bar, (uint32_t)(k & 1), split_verdict(a, k))) != 0;  // one verdict for the whole block
      if (!okw) break;
      float2 r[E];
#pragma unroll
      for (int i = 0; i < E; ++i) {
        const int x = t + T * i;
        r[i] = (i < EF && x < a.n) ? cmul(transmission(hv[i], cc), stage[(size_t)lr * cks + x]) : czero();
      }
      LF::template step1<false, NZF, PKR>(r, t, z, tw);
      __syncthreads();  // every thread is past its stage reads: the next channel may land there
      if (w + 1 < w1) fetch(w + 1);
      LF::template step2<false, LF::Q, PKR>(r, t, z);  // next z write follows the loop-top barrier
      if (ok) {
        float2* srow = a.S + ((size_t)w * a.n + rr) * M;
#pragma unroll
        for (int i = 0; i < E; ++i) srow[t + T * i] = r[i];
      }
    }
    if (!okw && threadIdx.x == 0) {
      (void)bulk_wait(bar, (uint32_t)(k & 1));  // a late copy lands (bounded) before the block leaves
      atomicExch(a.err, 1);
    }
  }

  // Row stride in shared memory of staged N-point rows (checkpoint, input
  // field): >= N, and congruent to SR mod 16, so that the rows of consecutive
  // lines fall in different banks the same way as in the staged spectra.
  __host__ __device__ static int ck_stride(int n) { return n + (((SR - n) % 16) + 16) % 16; }

  // ------------------------------------------- adjoint row pass, both inputs staged
  // Both inputs of a channel arrive by bulk copies: its spectra rows (into a
  // stage that is emptied into registers at the top of the iteration, so the
  // next channel's copy overlaps the whole iteration) and its checkpoint rows
  // (read after the inverse DFT; the next channel's copy is issued as soon as
  // every thread is past them, at the barrier inside the forward DFT).  With
  // few rows per block three blocks fit on an SM.  Needs N even.
  // SHARE (32 elements per thread, M = 512): the two inputs take turns in one
  // stage, which leaves room for three blocks per SM: the channel's checkpoint
  // rows are fetched at the barrier inside its inverse DFT (every thread is
  // past its spectra reads) and the next channel's spectra rows at the
  // barrier inside its forward DFT (every thread is past its checkpoint reads).
  static constexpr bool SHARE = LF::E > 20;
  // dynamic shared memory: stage[RL][SR] | ck[RL][cks] (not with SHARE) | exchange[RL][RZL] | tw[TWS] | barrier[2]
  static size_t adj_staged_smem(int n) {
    return sizeof(float2) * ((size_t)RL * SR + (SHARE ? 0 : (size_t)RL * ck_stride(n)) + (size_t)RL * RZL +
                             LF::TWS + 1) +
           2 * sizeof(uint64_t);
  }

  template <bool FIRST>
  __device__ static void row_adj_staged(const PassArgs& a) {
    extern __shared__ __align__(16) float2 smem[];
    const int cks = ck_stride(a.n);
    float2* stage = smem;
    float2* ckb = SHARE ? stage : stage + (size_t)RL * SR;
    float2* zb = SHARE ? stage + (size_t)RL * SR : ckb + (size_t)RL * cks;
    static_assert(!SHARE || SR % 2 == 0, "the checkpoint rows share the 16-byte aligned stage");
    float2* tw = tw_align(zb + (size_t)RL * RZL);
    uint64_t* bar = reinterpret_cast<uint64_t*>(tw + LF::TWS);  // [0] spectra rows, [1] checkpoint rows
    const int l = threadIdx.x / T, t = threadIdx.x % T;
    float2* z = zb + l * RZL;
    const int r0 = blockIdx.x * RL;
    const int nrows = min(RL, a.n - r0);
    const int row = r0 + l;
    const bool ok = l < nrows;
    const int rr = ok ? row : r0;
    const int lr = ok ? l : 0;
    const int w0 = blockIdx.y * a.chunk;
    const int w1 = min(a.nw, w0 + a.chunk);
    if (threadIdx.x == 0) {
      bulk_bar_init(&bar[0]);
      bulk_bar_init(&bar[1]);
    }
    for (int i = threadIdx.x; i < LF::TWS; i += blockDim.x) tw[i] = a.tw[i];
    __syncthreads();
    // thread 0 copies the block's rows of channel w: spectra (M * 8 bytes a
    // row) into the stage, checkpoint (N * 8 bytes a row) into ck
    auto fetch_s = [&](int w) {
      if (threadIdx.x != 0) return;
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      bulk_expect(&bar[0], (uint32_t)nrows * M * 8u);
      if (a.stall == 1) return;  // injected fault: the expected bytes never arrive
      const float2* src = a.S + ((size_t)w * a.n + r0) * M;
      for (int q = 0; q < nrows; ++q) bulk_g2s(stage + (size_t)q * SR, src + (size_t)q * M, M * 8u, &bar[0]);
    };
    auto fetch_c = [&](int w) {
      if (threadIdx.x != 0) return;
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      bulk_expect(&bar[1], (uint32_t)nrows * a.n * 8u);
      if (a.stall == 1) return;
      const float2* src = a.ckpt + ((size_t)w * a.n + r0) * a.n;
      for (int q = 0; q < nrows; ++q) bulk_g2s(ckb + (size_t)q * cks, src + (size_t)q * a.n, a.n * 8u, &bar[1]);
    };
    // the thickness row stays in registers across the chunk's channels
    const float* hrow = a.h + (size_t)rr * a.n;
    float hv[E];
#pragma unroll
    for (int i = 0; i < E; ++i) {
      const int x = t + T * i;
      hv[i] = (i < EF && x < a.n) ? __ldg(hrow + x) : 0.f;
    }
    float g[E];
#pragma unroll
    for (int i = 0; i < E; ++i) g[i] = 0.f;
    bool okw = true;
    int issued_s = 0, issued_c = 0, done_s = 0, done_c = 0;  // copies per barrier (thread 0's view)
    if (w0 < w1) {
      fetch_s(w0);
      issued_s = 1;
      if constexpr (!SHARE) {
        fetch_c(w0);
        issued_c = 1;
      }
    }
    for (int w = w0; w < w1; ++w) {
      okw = __syncthreads_and(bulk_wait(&bar[0], (uint32_t)(done_s & 1), split_verdict(a, done_s))) != 0;  // one verdict for the block
      if (!okw) break;
      ++done_s;
      float2 r[E];
#pragma unroll
      for (int i = 0; i < E; ++i) r[i] = stage[(size_t)lr * SR + t + T * i];
      LF::template step1<true, LF::P, PKR>(r, t, z, tw);
      __syncthreads();  // every thread is past its stage reads: the next channel (SHARE: this channel's checkpoint) may land there
      if constexpr (SHARE) {
        fetch_c(w);
        ++issued_c;
      } else if (w + 1 < w1) {
        fetch_s(w + 1);
        ++issued_s;
      }
      LF::template step2<true, NOI, PKR>(r, t, z);  // the barrier below also ends its z reads
      okw = __syncthreads_and(bulk_wait(&bar[1], (uint32_t)(done_c & 1))) != 0;
      if (!okw) break;
      ++done_c;
      // the channel's constants, loaded here rather than held through the
      // inverse DFT (the registers they would take there spill)
      const ChanConst cc = a.chan[w];
      const float2* ck = ckb + (size_t)lr * cks;
#pragma unroll
      for (int i = 0; i < E; ++i) {
        const int x = t + T * i;
        if (i < EF && x < a.n) {
          const float2 au = r[i];
          const float2 tt = transmission(hv[i], cc);
          const float2 cu = cmul(make_float2(cc.c_re, cc.c_im), cmul(tt, ck[x]));
          g[i] = fmaf(au.x, cu.x, fmaf(au.y, cu.y, g[i]));
          r[i] = cmulc(au, tt);
        } else {
          r[i] = czero();
        }
      }
      if constexpr (!FIRST) {
        LF::template step1<false, NZF, PKR, LF::SQUARE>(r, t, z, tw);
        __syncthreads();  // every thread is past its checkpoint reads
        if (w + 1 < w1) {
          if constexpr (SHARE) {
            fetch_s(w + 1);
            ++issued_s;
          } else {
            fetch_c(w + 1);
            ++issued_c;
          }
        }
        LF::template step2<false, LF::Q, PKR, LF::SQUARE>(r, t, z);  // next z write follows the loop-top barrier
        if (ok) {
          float2* srow = a.S + ((size_t)w * a.n + rr) * M;
#pragma unroll
          for (int i = 0; i < E; ++i) srow[t + T * i] = r[i];
        }
      } else {
        __syncthreads();  // every thread is past its checkpoint reads
        if (w + 1 < w1) {
          if constexpr (SHARE) {
            fetch_s(w + 1);
            ++issued_s;
          } else {
            fetch_c(w + 1);
            ++issued_c;
          }
        }
      }
    }
    if (!okw) {
      // copies still in flight land (bounded waits) before the block leaves
      if (threadIdx.x == 0) {
        if (issued_s > done_s) (void)bulk_wait(&bar[0], (uint32_t)(done_s & 1));
        if (issued_c > done_c) (void)bulk_wait(&bar[1], (uint32_t)(done_c & 1));
        atomicExch(a.err, 1);
      }
      return;
    }
    if (ok) {
      float* prow = a.partial + ((size_t)blockIdx.y * a.n + row) * a.n;
#pragma unroll
      for (int i = 0; i < E; ++i) {
        const int x = t + T * i;
        if (i < EF && x < a.n) prow[x] = g[i];
      }
    }
  }
};

// the staged adjoint row pass: three blocks of few rows per SM
template <class LF, int RL, bool HALF, bool FIRST>
__global__ void __launch_bounds__(LF::T * RL, 3) k_row_adj_staged(PassArgs a) {
  PassBulk<LF, RL, HALF>::template row_adj_staged<FIRST>(a);
}
// two blocks per SM for every line shape: one leaves too few warps to hide the
// DFT's barriers and dependencies (M = 512: 8.5 ms per launch with one)
template <class LF, int RL, bool HALF, bool ADJ>
__global__ void __launch_bounds__(LF::T * Pass<LF>::COLL, 2)
    k_col_bulk(PassArgs a, const __grid_constant__ CUtensorMap smap, const __grid_constant__ CUtensorMap hmap) {
  PassBulk<LF, RL, HALF>::template col<ADJ>(a, &smap, &hmap);
}
// the row passes: as many resident blocks as their shared memory allows
template <class LF, int RL>
constexpr int row_bulk_min_blocks() { return LF::E <= 20 ? (RL <= 8 ? 4 : 2) : 1; }
template <class LF, int RL, bool HALF, bool ADJ, bool FLAG>
__global__ void __launch_bounds__(LF::T * RL, row_bulk_min_blocks<LF, RL>()) k_row_bulk(PassArgs a) {
  PassBulk<LF, RL, HALF>::template row<ADJ, FLAG>(a);
}
template <class LF, int RL, bool HALF>
__global__ void __launch_bounds__(LF::T * RL, row_bulk_min_blocks<LF, RL>()) k_row_first_staged(PassArgs a) {
  PassBulk<LF, RL, HALF>::row_first_staged(a);
}

// Launchers.  The column pass runs one persistent block per resident slot
// (blocks per SM from the occupancy calculator x SMs); the row passes run
// (row blocks) x (channel chunks) blocks, each looping over its chunk.
template <class LF, int RL>
struct PassBulkLaunch {
  using PB = PassBulk<LF, RL>;
  template <typename K>
  static cudaError_t slots(K kernel, int threads, size_t smem, int* out) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0, dev = 0, sms = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem)) != cudaSuccess) return e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    *out = std::max(1, per_sm) * sms;
    return cudaSuccess;
  }
  // The tensor copy needs a map whose box holds the input rows (at most 256);
  // without one the plain kernel runs.
  static bool half(const PassArgs& a) { return 2 * a.n <= LF::M; }
  template <bool H>
  static cudaError_t col_h(const PassArgs& a, bool adj, size_t sm, cudaStream_t s) {
    const int items = a.nw * (LF::M / PB::COLL);
    if (items == 0) return cudaSuccess;
    int n_slots = 0;
    auto kern = adj ? k_col_bulk<LF, RL, H, true> : k_col_bulk<LF, RL, H, false>;
    cudaError_t e = slots(kern, PB::CT, sm, &n_slots);
    if (e != cudaSuccess) return e;
    kern<<<std::min(items, n_slots), PB::CT, sm, s>>>(a, *static_cast<const CUtensorMap*>(a.tmap),
                                                     *static_cast<const CUtensorMap*>(a.hmap));
    return cudaGetLastError();
  }
  // The tensor copies need maps whose boxes hold the input rows (at most 256)
  // and the H tile, and M a multiple of 16 (whole mirrored pairs of 8-column
  // groups); otherwise the plain kernel runs.
  static cudaError_t col(const PassArgs& a, bool adj, cudaStream_t s) {
    const size_t sm = PB::col_smem(a.n);
    if (!a.tmap || !a.hmap || a.tmap_rows != a.in_r1 - a.in_r0 || a.tmap_rows > 256 ||
        LF::M % 16 != 0 ||
        sm > 227 * 1024)
      return PassLaunch<LF>::col(a, adj, false, s);
    return half(a) ? col_h<true>(a, adj, sm, s) : col_h<false>(a, adj, sm, s);
  }
  template <bool H>
  static cudaError_t row_fwd_h(const PassArgs& a, bool save, cudaStream_t s) {
    const dim3 g((a.n + RL - 1) / RL, a.n_chunks);
    const size_t sm = PB::row_smem();
    return save ? launch_k(k_row_bulk<LF, RL, H, false, true>, g, PB::RT, sm, a, s)
                : launch_k(k_row_bulk<LF, RL, H, false, false>, g, PB::RT, sm, a, s);
  }
  static cudaError_t row_fwd(const PassArgs& a, bool save, cudaStream_t s) {
    return half(a) ? row_fwd_h<true>(a, save, s) : row_fwd_h<false>(a, save, s);
  }
  // the first forward row pass (t * v1 -> DFT) with staged input rows; the
  // plain kernel where N is odd or the stage does not fit
  static cudaError_t row_first(const PassArgs& a, cudaStream_t s) {
    const size_t sm = PB::first_smem(a.n);
    if (a.n % 2 != 0 || sm > 227 * 1024) return PassLaunch<LF>::row_first(a, s);
    const dim3 g((a.n + RL - 1) / RL, a.n_chunks);
    return half(a) ? launch_k(k_row_first_staged<LF, RL, true>, g, PB::RT, sm, a, s)
                   : launch_k(k_row_first_staged<LF, RL, false>, g, PB::RT, sm, a, s);
  }
  // rows per block of the staged adjoint row pass
  static constexpr int RLA = RL >= 16 ? RL / 2 : RL;
  using PBA = PassBulk<LF, RLA>;
  template <bool H>
  static cudaError_t row_adj_h(const PassArgs& a, bool first, cudaStream_t s) {
    if (a.n % 2 == 0 && PBA::adj_staged_smem(a.n) <= 227 * 1024) {
      const dim3 g((a.n + RLA - 1) / RLA, a.n_chunks);
      const size_t sm = PBA::adj_staged_smem(a.n);
      return first ? launch_k(k_row_adj_staged<LF, RLA, H, true>, g, PBA::RT, sm, a, s)
                   : launch_k(k_row_adj_staged<LF, RLA, H, false>, g, PBA::RT, sm, a, s);
    }
    // odd N: the spectra rows staged, the checkpoint read directly
    const dim3 g((a.n + RL - 1) / RL, a.n_chunks);
    const size_t sm = PB::row_smem();
    return first ? launch_k(k_row_bulk<LF, RL, H, true, true>, g, PB::RT, sm, a, s)
                 : launch_k(k_row_bulk<LF, RL, H, true, false>, g, PB::RT, sm, a, s);
  }
  static cudaError_t row_adj(const PassArgs& a, bool first, cudaStream_t s) {
    return half(a) ? row_adj_h<true>(a, first, s) : row_adj_h<false>(a, first, s);
  }
};

// The launchers of one padded size, plain and bulk-prefetching.
template <class LF, int RL>
const PassOps* pass_ops_table() {
  using PL = PassLaunch<LF>;
  using PBL = PassBulkLaunch<LF, RL>;
  static const PassOps o = {LF::M,       LF::P,          LF::Q,          LF::T,
                            Pass<LF>::ROWL, Pass<LF>::COLL, &PL::col,    &PL::row_fwd,
                            &PL::row_out, &PL::row_seed,  &PL::row_adj,  &PL::row_in,
                            &PL::row_back, &PL::row_first, &PBL::col, &PBL::row_fwd,
                            &PBL::row_adj, &PBL::row_first, PassBulk<LF, RL>::GW,
                            PassBulk<LF, RL>::STAGE_H ? PassBulk<LF, RL>::HP : PassBulk<LF, RL>::HB,
                            PassBulk<LF, RL>::STAGE_H ? PassBulk<LF, RL>::HW : PassBulk<LF, RL>::GW};
  return &o;
}

}  // namespace dos

// One translation unit per padded size: defines dos::pass_ops_<M>() (RL_ rows
// per block in the bulk-prefetching row passes).
#define DOS_DEFINE_PASS_OPS(M_, P_, Q_, T_, RL_)                                              \
  namespace dos {                                                                             \
  const PassOps* pass_ops_##M_() { return pass_ops_table<Line<P_, Q_, T_>, RL_>(); }          \
  }
