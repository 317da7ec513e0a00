// dos_gemm.cu - split-BF16 DFT-GEMM form of the propagation (tcgen05, TMEM).
//
// See dos_gemm.cuh for the formulation.  The GEMM kernel is persistent and
// warp-specialised: one CTA per SM walks its share of the 128 x 256 output
// tiles.  Warp 0 (one lane) streams the operands: both are kept in global
// memory tile by tile in the tensor core's K-major core-matrix order
// (gemm_tiled), so a K chunk of 64 is two bulk copies (16 KB of A, 32 KB of B,
// cp.async.bulk with completion counted in bytes on the stage's "full"
// mbarrier) into a GSTAGES-deep ring.  Warp 1 (one lane) issues the MMAs into
// one of two TMEM accumulators (2 x 256 columns) and frees each stage through
// tcgen05.commit on its "empty" mbarrier; a commit on "acc_full" hands a
// finished accumulator to the sixteen epilogue warps, which drain it (warp w
// reads TMEM lanes 32 (w % 4) .. +31 and a quarter of the columns) while the
// MMAs of the next tile run into the other accumulator, and release it on
// "acc_empty".  Every wait is bounded and watches a shared abort flag: on
// expiry the CTA records the error flag, lets its copies and MMAs in flight
// finish (bounded) and ends cleanly.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>

#include "dos_gemm.cuh"
#include "dos_internal.h"
#include "dos_pass.cuh"

namespace dos {

constexpr int GTM = 128, GTN = 256, GTK = 64;  // one tile and MMA: 128 x 256, K steps of 16
constexpr int GSTAGES = 4;                      // 48 KB per stage
constexpr int kEpiWarps = 16;                   // 4 per TMEM lane quarter, a quarter of the columns each
constexpr int kGemmThreads = 32 * (2 + kEpiWarps);
constexpr long kSpinLimit = 1L << 26;           // bounded mbarrier wait (a fraction of a second)

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t kmajor_desc(uint32_t saddr) {
  // start >> 4 | LBO 128 B (next 8 k) | SBO 1024 B (next 8 rows) | descriptor version 1 | no swizzle
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46);
}

// kind::f16 instruction descriptor: D f32, A and B bf16, both K-major, N = 256, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(GTN >> 3) << 17) |
                            ((uint32_t)(GTM >> 4) << 24);

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}
// bounded wait; gives up early when another role of the CTA raised *abort
// (then returns false without raising it again)
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort = nullptr) {
  for (long it = 0; it < kSpinLimit; ++it) {
    if (mbar_try(bar, parity)) return true;
    if (abort && (it & 255) == 255 && *abort) return false;
  }
  if (abort) *abort = 1;
  return false;
}

__device__ __forceinline__ void bar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// one contiguous global -> shared bulk copy, completion counted on `bar`
__device__ __forceinline__ void bulk_tile(void* dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

struct __align__(1024) GemmSmem {
  uint8_t a[GSTAGES][GTM * GTK * 2];  // 16 KB per stage
  uint8_t b[GSTAGES][GTN * GTK * 2];  // 32 KB per stage
  uint64_t full[GSTAGES];             // copies of the stage landed
  uint64_t empty[GSTAGES];            // MMAs reading the stage done
  uint64_t acc_full[2];               // accumulator ready for the epilogue
  uint64_t acc_empty[2];              // accumulator drained (one arrival per epilogue warp)
  uint32_t tmem;
  int abort;
};

// ------------------------------------------------------------ epilogues
// x -> bf16 parts: each the round-to-nearest of what the earlier parts leave
__device__ __forceinline__ void split_store(const Parts& P, size_t i, float v) {
  const __nv_bfloat16 h = __float2bfloat16_rn(v);
  P.p[0][i] = h;
  const float r1 = v - __bfloat162float(h);
  const __nv_bfloat16 m = __float2bfloat16_rn(r1);
  P.p[1][i] = m;
  if (P.k > 2) P.p[2][i] = __float2bfloat16_rn(r1 - __bfloat162float(m));
}

// x -> bf16 parts of 8 consecutive K entries (8-aligned) of one operand row:
// one 16-byte store per part
__device__ __forceinline__ void split_store8(const Parts& P, size_t at, const float* x) {
  uint32_t w0[4], w1[4], w2[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    __nv_bfloat16 h[2], m[2], l[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const float v = x[2 * e + q];
      h[q] = __float2bfloat16_rn(v);
      const float r1 = v - __bfloat162float(h[q]);
      m[q] = __float2bfloat16_rn(r1);
      l[q] = __float2bfloat16_rn(r1 - __bfloat162float(m[q]));
    }
    w0[e] = (uint32_t)__bfloat16_as_ushort(h[0]) | ((uint32_t)__bfloat16_as_ushort(h[1]) << 16);
    w1[e] = (uint32_t)__bfloat16_as_ushort(m[0]) | ((uint32_t)__bfloat16_as_ushort(m[1]) << 16);
    w2[e] = (uint32_t)__bfloat16_as_ushort(l[0]) | ((uint32_t)__bfloat16_as_ushort(l[1]) << 16);
  }
  *reinterpret_cast<uint4*>(P.p[0] + at) = make_uint4(w0[0], w0[1], w0[2], w0[3]);
  *reinterpret_cast<uint4*>(P.p[1] + at) = make_uint4(w1[0], w1[1], w1[2], w1[3]);
  if (P.k > 2) *reinterpret_cast<uint4*>(P.p[2] + at) = make_uint4(w2[0], w2[1], w2[2], w2[3]);
}

// Transfer-function values of accumulator row r = (w, kx), columns cb ..
// cb+31 = sixteen ky (spectrum epilogue): loaded before the accumulator is,
// so that the table's latency overlaps the tensor-memory load
__device__ __forceinline__ void spectrum_h(const GemmArgs& g, int r, int cb, float2 (&hv)[16]) {
  const int m = g.m, w = r / m, kx = r - w * m;
  const int bx = min(kx, m - kx);
  const float2* Hw = g.Hq + (size_t)w * g.hs * g.hs;
  const int ky0 = cb >> 1;
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const int ky = ky0 + q;
    hv[q] = ky < m ? __ldg(Hw + (size_t)min(ky, m - ky) * g.hs + bx) : make_float2(0.f, 0.f);
  }
}

// accumulator row r, columns cb .. cb+31 (values v) -> the destination of MODE
// (hv: the spectrum epilogue's transfer-function values, from spectrum_h)
template <int MODE>
__device__ __forceinline__ void epilogue(const GemmArgs& g, int r, int cb, const float* v, const float2 (&hv)[16]) {
  if constexpr (MODE == GEMM_OUT_ROWS) {
    const int k = r >> 1, p = r & 1;
    if (g.nj % 8 == 0) {
      // 8-aligned groups never straddle a channel: one 16-byte store per part
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int c = cb + 8 * q;
        if (c >= g.vcols) break;
        const int w = c / g.nj, j = c - w * g.nj;
        split_store8(g.xo, gemm_tiled((size_t)w * g.nk + k, p * g.nj + j, g.kpo), v + 8 * q);
      }
    } else {
      for (int q = 0; q < 32; ++q) {
        const int c = cb + q;
        if (c >= g.vcols) break;
        const int w = c / g.nj, j = c - w * g.nj;
        split_store(g.xo, gemm_tiled((size_t)w * g.nk + k, p * g.nj + j, g.kpo), v[q]);
      }
    }
  } else if constexpr (MODE == GEMM_OUT_SPECTRUM) {
    // row r = (w, kx); columns 2ky + {0, 1}: sixteen spectrum values
    const int m = g.m, w = r / m, kx = r - w * m;
    const int bx = min(kx, m - kx);
    const float* Sw = g.mis.sq ? g.mis.sq + (size_t)w * g.hs * g.hs : nullptr;
    const int ky0 = cb >> 1;  // multiple of 16
    if (ky0 >= m) return;
    float re[16], im[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int ky = ky0 + q;
      float2 val = make_float2(0.f, 0.f);
      if (ky < m) {
        float2 h = hv[q];
        if (Sw) h = cmul(h, misalign_factor(g.mis, ky, kx, m, Sw[(size_t)min(ky, m - ky) * g.hs + bx]));
        const float2 b = make_float2(v[2 * q], v[2 * q + 1]);
        val = g.adj ? cmulc(b, h) : cmul(b, h);
      }
      re[q] = val.x;
      im[q] = val.y;
    }
    // m is a multiple of 8 for every compiled size: whole groups of 8
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      if (ky0 + 8 * q >= m) break;
      split_store8(g.xo, gemm_tiled((size_t)r, ky0 + 8 * q, g.kpo), re + 8 * q);
      split_store8(g.xo, gemm_tiled((size_t)r, m + ky0 + 8 * q, g.kpo), im + 8 * q);
    }
  } else {
    // row r = (w, y); columns 2x + {0, 1}: sixteen field values
    const int n = g.n, w = r / n, y = r - w * n;
    const int x0 = cb >> 1;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int x = x0 + q;
      if (x >= n) break;
      const float2 val = make_float2(v[2 * q], v[2 * q + 1]);
      if (g.o) {
        const int fy = y - g.of, fx = x - g.of;
        if (fy >= 0 && fy < g.fov && fx >= 0 && fx < g.fov) {
          const size_t qo = ((size_t)w * g.fov + fy) * g.fov + fx;
          g.o[qo] = val;
          if (g.I) g.I[qo] = fmaf(val.x, val.x, val.y * val.y);
        }
      } else {
        g.fld[((size_t)w * n + y) * n + x] = val;
      }
    }
  }
}

template <int MODE>
__global__ void __launch_bounds__(kGemmThreads, 1) k_tc_gemm(const __grid_constant__ GemmArgs g) {
  extern __shared__ __align__(1024) uint8_t gsm_raw[];
  GemmSmem& sm = *reinterpret_cast<GemmSmem*>(gsm_raw);
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  volatile int* abort = &sm.abort;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&sm.tmem)),
                 "r"(2 * GTN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 32) {
    for (int s = 0; s < GSTAGES; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&sm.full[s])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&sm.empty[s])));
    }
    for (int b = 0; b < 2; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&sm.acc_full[b])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&sm.acc_empty[b])), "r"(kEpiWarps));
    }
    sm.abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = sm.tmem;
  const int kchunks = g.K / GTK;
  const int total = g.nseg * kchunks;  // K chunks per tile
  // tiles, the DFT matrix's (few) tiles the fast index: the CTAs that share a
  // data tile run together
  const int tilesA = g.rows / GTM, tilesB = (g.cols + GTN - 1) / GTN;
  const int ntiles = tilesA * tilesB;
  auto tile_of = [&](int t, int& mt, int& nt) {
    if (g.w_is_b) {
      nt = t % tilesB;
      mt = t / tilesB;
    } else {
      mt = t % tilesA;
      nt = t / tilesA;
    }
  };
  if (warp == 0) {
    // ---------------------------------------------------------------- producer
    if (lane == 0) {
      int c = 0;
      int last[GSTAGES];
      for (int s = 0; s < GSTAGES; ++s) last[s] = -1;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        int mt, nt;
        tile_of(t, mt, nt);
        for (int it = 0; it < total; ++it, ++c) {
          const int st = c % GSTAGES;
          if (c >= GSTAGES &&
              !mbar_wait(smem_addr(&sm.empty[st]), (uint32_t)(((c / GSTAGES) - 1) & 1), abort)) {
            ok = false;
            break;
          }
          const int seg = it / kchunks, kc = it % kchunks;
          const uint32_t fb = smem_addr(&sm.full[st]);
          bar_expect_tx(fb, (GTM + GTN) * GTK * 2);
          // 128-row A tile mt: half (mt & 1) of the stored 256-row tile mt / 2
          bulk_tile(sm.a[st], g.a[seg] + (((size_t)(mt >> 1) * kchunks + kc) << 14) + ((size_t)(mt & 1) << 13),
                    GTM * GTK * 2, fb);
          bulk_tile(sm.b[st], g.b[seg] + (((size_t)nt * kchunks + kc) << 14), GTN * GTK * 2, fb);
          last[st] = c;
        }
      }
      // no copy may still target shared memory when the CTA ends
      for (int s = 0; s < GSTAGES; ++s)
        if (last[s] >= 0) (void)mbar_wait(smem_addr(&sm.full[s]), (uint32_t)((last[s] / GSTAGES) & 1));
    }
    __syncwarp();
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA issue
    if (lane == 0) {
      int c = 0, tc = 0;
      uint32_t last_bar = 0, last_par = 0;  // the latest commit (covers every MMA before it)
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++tc) {
        const int b = tc & 1;
        if (tc >= 2 && !mbar_wait(smem_addr(&sm.acc_empty[b]), (uint32_t)(((tc >> 1) - 1) & 1), abort)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t acc0 = tmem + (uint32_t)(b * GTN);
        for (int it = 0; it < total; ++it, ++c) {
          const int st = c % GSTAGES;
          if (!mbar_wait(smem_addr(&sm.full[st]), (uint32_t)((c / GSTAGES) & 1), abort)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;");
          const uint32_t sa = smem_addr(sm.a[st]), sb = smem_addr(sm.b[st]);
#pragma unroll
          for (int kk = 0; kk < GTK / 16; ++kk) {
            const uint64_t da = kmajor_desc(sa + kk * 256), db = kmajor_desc(sb + kk * 256);
            const uint32_t acc = (it > 0 || kk > 0) ? 1u : 0u;
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(acc0),
                "l"(da), "l"(db), "r"(kIdesc), "r"(acc));
          }
          last_bar = smem_addr(&sm.empty[st]);
          last_par = (uint32_t)((c / GSTAGES) & 1);
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(last_bar));
        }
        if (!ok) break;
        last_bar = smem_addr(&sm.acc_full[b]);
        last_par = (uint32_t)((tc >> 1) & 1);
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(last_bar));
      }
      // no MMA may still write tensor memory when it is released
      if (last_bar) (void)mbar_wait(last_bar, last_par);
    }
    __syncwarp();
  } else {
    // ---------------------------------------------------------------- epilogue
    const int q = warp & 3;                 // TMEM lane quarter
    const int part = (warp - 2) >> 2;       // column quarter
    int tc = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++tc) {
      const int b = tc & 1;
      if (!mbar_wait(smem_addr(&sm.acc_full[b]), (uint32_t)((tc >> 1) & 1), abort)) break;
      asm volatile("tcgen05.fence::after_thread_sync;");
      int mt, nt;
      tile_of(t, mt, nt);
      const int r = mt * GTM + q * 32 + lane;  // accumulator row of this thread
#pragma unroll 1
      for (int c0 = part * (GTN / 4); c0 < (part + 1) * (GTN / 4); c0 += 32) {
        float2 hv[16];
        if constexpr (MODE == GEMM_OUT_SPECTRUM) {
          if (r < g.vrows) spectrum_h(g, r, nt * GTN + c0, hv);
        }
        uint32_t u[32];
        const uint32_t addr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * GTN + c0);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
            "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]),
              "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]), "=r"(u[15]),
              "=r"(u[16]), "=r"(u[17]), "=r"(u[18]), "=r"(u[19]), "=r"(u[20]), "=r"(u[21]), "=r"(u[22]), "=r"(u[23]),
              "=r"(u[24]), "=r"(u[25]), "=r"(u[26]), "=r"(u[27]), "=r"(u[28]), "=r"(u[29]), "=r"(u[30]), "=r"(u[31])
            : "r"(addr));
        asm volatile("tcgen05.wait::ld.sync.aligned;");
        if (r < g.vrows) {
          float v[32];
#pragma unroll
          for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(u[j]);
          epilogue<MODE>(g, r, nt * GTN + c0, v, hv);
        }
      }
      // this warp is done with the accumulator
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&sm.acc_empty[b])) : "memory");
    }
  }
  __syncthreads();
  if (tid == 0 && sm.abort) atomicExch(g.err, 1);
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * GTN));
}

template <int MODE>
static cudaError_t launch_mode(const GemmArgs& g, cudaStream_t s) {
  // attribute and SM count of the current device, every launch (contexts may
  // live on different devices of one process; both calls are host-side only)
  const size_t sm = sizeof(GemmSmem) + 1024;
  cudaError_t e = cudaFuncSetAttribute(k_tc_gemm<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  int dev = 0, sms = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int tiles = (g.rows / GTM) * ((g.cols + GTN - 1) / GTN);
  k_tc_gemm<MODE><<<std::min(tiles, sms), kGemmThreads, sm, s>>>(g);
  return cudaGetLastError();
}

cudaError_t launch_tc_gemm(const GemmArgs& g, cudaStream_t s) {
  switch (g.mode) {
    case GEMM_OUT_ROWS: return launch_mode<GEMM_OUT_ROWS>(g, s);
    case GEMM_OUT_SPECTRUM: return launch_mode<GEMM_OUT_SPECTRUM>(g, s);
    default: return launch_mode<GEMM_OUT_FIELD>(g, s);
  }
}

// ------------------------------------------------------------ constant matrices

// W rows r: output o = r / 2 (re for even r, im for odd r); K index c: input
// element c (its real part) for c < kin, input c - kin (imaginary part) for
// kin <= c < 2 kin.  Entry exp(sign 2 pi j o x / m) in FP64, split into bf16.
__global__ void k_dft_matrix(Parts W, int rows_pad, int kpad, int nout, int kin, int m, int sign) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)rows_pad * kpad) return;
  const int r = (int)(i / kpad), c = (int)(i % kpad);
  const int o = r / 2;
  const size_t at = gemm_tiled((size_t)r, c, kpad);
  float v = 0.f;
  if (o < nout && c < 2 * kin) {
    const int x = c < kin ? c : c - kin;
    const long e = ((long)o * x) % m;
    double s, co;
    sincospi(2.0 * sign * (double)e / (double)m, &s, &co);
    // row 2o: [Re W, -Im W];  row 2o+1: [Im W, Re W]
    if ((r & 1) == 0) v = (float)(c < kin ? co : -s);
    else v = (float)(c < kin ? s : co);
  }
  split_store(W, at, v);
}

cudaError_t launch_build_dft(GemmPlan& p, cudaStream_t s) {
  const size_t nf = (size_t)p.rp1 * p.kp1, ng = (size_t)p.rp2 * p.kp2;
  k_dft_matrix<<<(unsigned)((nf + 255) / 256), 256, 0, s>>>(p.F, p.rp1, p.kp1, p.m, p.n, p.m, -1);
  k_dft_matrix<<<(unsigned)((ng + 255) / 256), 256, 0, s>>>(p.G, p.rp2, p.kp2, p.n, p.m, p.m, +1);
  return cudaGetLastError();
}

// ------------------------------------------------------------ conversion kernels
// field (complex [w][y][x]) -> X rows (w, y): [Re(u), Im(u), 0 ...] of length kp.
// mode 0: u = v;  mode 1: checkpoint v, u = t(h) v (forward layer);  mode 2: aperture.
__global__ void k_prep_field(const float2* __restrict__ v, float2* __restrict__ ckpt, const float* __restrict__ h,
                             const ChanConst* __restrict__ chan, Parts X, int n, int kp, int mode, int a_off,
                             int a_w) {
  const int wy = blockIdx.x;  // w * n + y
  const int w = wy / n, y = wy % n;
  for (int c = threadIdx.x; c < kp; c += blockDim.x) {
    float val = 0.f;
    if (c < 2 * n) {
      const int x = c < n ? c : c - n;
      float2 u;
      if (mode == 2) {
        const bool in = y >= a_off && y < a_off + a_w && x >= a_off && x < a_off + a_w;
        u = make_float2(in ? 1.f : 0.f, 0.f);
      } else {
        const float2 vv = v[(size_t)wy * n + x];
        if (mode == 1) {
          if (c < n) ckpt[(size_t)wy * n + x] = vv;
          u = cmul(transmission(h[(size_t)y * n + x], chan[w]), vv);
        } else {
          u = vv;
        }
      }
      val = c < n ? u.x : u.y;
    }
    split_store(X, gemm_tiled((size_t)wy, c, kp), val);
  }
}

// zero the K entries [k_from, kp) of operand rows [0, rows) (the padding of
// K past the data, which the epilogues do not write)
__global__ void k_zero_kpad(Parts X, size_t rows, int k_from, int kp) {
  const int wk = kp - k_from;
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows * (size_t)wk) return;
  const size_t r = i / wk;
  const int k = k_from + (int)(i % wk);
  const size_t at = gemm_tiled(r, k, kp);
  const __nv_bfloat16 z = __float2bfloat16_rn(0.f);
  for (int q = 0; q < X.k; ++q) X.p[q][at] = z;
}

// adjoint seed on the FOV: 2 dL/dI o, zero elsewhere
__global__ void k_field_seed(float2* __restrict__ field, const float2* __restrict__ o, const float* __restrict__ dLdI,
                             int n, int of, int fov, size_t total) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  const size_t w = i / ((size_t)n * n);
  const int y = (int)((i / n) % n), x = (int)(i % n);
  const int fy = y - of, fx = x - of;
  float2 g = make_float2(0.f, 0.f);
  if (fy >= 0 && fy < fov && fx >= 0 && fx < fov) {
    const size_t q = (w * fov + fy) * fov + fx;
    g = cscale(o[q], 2.0f * dLdI[q]);
  }
  field[i] = g;
}

// adjoint layer: per pixel, over the chunk's channels in order:
//   partial += Re(conj(grad_u) c t v);  grad_v = conj(t) grad_u (in place)
__global__ void k_field_adj(float2* __restrict__ field, const float2* __restrict__ ckpt, size_t ckpt_stride,
                            const float* __restrict__ h, const ChanConst* __restrict__ chan, float* __restrict__ partial,
                            int nwc, int n) {
  const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t n2 = (size_t)n * n;
  if (p >= n2) return;
  const float hv = h[p];
  float acc = 0.f;
  for (int w = 0; w < nwc; ++w) {
    const ChanConst cc = chan[w];
    const float2 au = field[w * n2 + p];
    const float2 tt = transmission(hv, cc);
    const float2 cu = cmul(make_float2(cc.c_re, cc.c_im), cmul(tt, ckpt[(size_t)w * ckpt_stride + p]));
    acc = fmaf(au.x, cu.x, fmaf(au.y, cu.y, acc));
    field[w * n2 + p] = cmulc(au, tt);
  }
  partial[p] = acc;
}

// ------------------------------------------------------------ one propagation
// The kept products of the parts: (0,0), (0,1), (1,0) and, with three parts,
// (0,2), (2,0), (1,1).  The tensor core's FP32 accumulation loses a little of
// every partial sum (measured: the relative error grows with the number of
// accumulation steps at the accumulator's magnitude), so the small products go
// first and the large (0,0) product last: the error is then that of the (0,0)
// product alone.
static void set_terms(GemmArgs& g, const Parts& A, const Parts& B) {
  static const int ta2[3] = {0, 1, 0}, tb2[3] = {1, 0, 0};
  static const int ta3[6] = {1, 0, 2, 0, 1, 0}, tb3[6] = {1, 2, 0, 1, 0, 0};
  const bool three = A.k == 3;
  g.nseg = three ? 6 : 3;
  for (int t = 0; t < g.nseg; ++t) {
    g.a[t] = A.p[three ? ta3[t] : ta2[t]];
    g.b[t] = B.p[three ? tb3[t] : tb2[t]];
  }
}

static cudaError_t zero_kpad(const Parts& X, size_t rows, int k_from, int kp, int* launches, cudaStream_t s) {
  if (k_from >= kp) return cudaSuccess;
  const size_t total = rows * (size_t)(kp - k_from);
  k_zero_kpad<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(X, rows, k_from, kp);
  ++*launches;
  return cudaGetLastError();
}

// X rows (w, y) of the chunk hold the field; computes the propagated field
// (into fld) or, with o non-null, the output plane.  Operands alternate
// between the X and Y buffers: X1 (field) -> Y (after the row DFT) -> X (after
// the column DFT and H) -> Y (after the column IDFT) -> field.
cudaError_t gemm_propagate(GemmPlan& p, int nwc, const float2* Hq, int hs, bool adj, float2* o, float* I, int of,
                           int fov, const Misalign& mis, int* launches, cudaStream_t s) {
  const int n = p.n, m = p.m;
  auto pad256 = [](int v) { return (v + 255) / 256 * 256; };
  const int c1 = nwc * n, c2 = nwc * m;
  cudaError_t e;
  GemmArgs g;
  std::memset(&g, 0, sizeof(g));
  g.err = p.err;
  // row DFT: D = F X1^T -> Y rows (w, kx), K = p n + y
  if ((e = zero_kpad(p.Y, (size_t)pad256(c2), 2 * n, p.kp1, launches, s)) != cudaSuccess) return e;
  set_terms(g, p.F, p.X);
  g.rows = p.rp1; g.cols = c1; g.K = p.kp1; g.w_is_b = 0;
  g.mode = GEMM_OUT_ROWS; g.vrows = 2 * m; g.vcols = c1; g.nk = m; g.nj = n; g.xo = p.Y; g.kpo = p.kp1;
  if ((e = launch_tc_gemm(g, s)) != cudaSuccess) return e;
  ++*launches;
  // column DFT and H: D = Y F^T -> X rows (w, kx), K = ky | m + ky
  if ((e = zero_kpad(p.X, (size_t)pad256(c2), 2 * m, p.kp2, launches, s)) != cudaSuccess) return e;
  set_terms(g, p.Y, p.F);
  g.rows = pad256(c2); g.cols = 2 * m; g.K = p.kp1; g.w_is_b = 1;
  g.mode = GEMM_OUT_SPECTRUM; g.vrows = c2; g.vcols = 2 * m; g.xo = p.X; g.kpo = p.kp2;
  g.Hq = Hq; g.hs = hs; g.m = m; g.adj = adj ? 1 : 0; g.mis = mis;
  if ((e = launch_tc_gemm(g, s)) != cudaSuccess) return e;
  ++*launches;
  // column IDFT: D = G X^T -> Y rows (w, y), K = p m + kx
  if ((e = zero_kpad(p.Y, (size_t)pad256(c1), 2 * m, p.kp2, launches, s)) != cudaSuccess) return e;
  set_terms(g, p.G, p.X);
  g.rows = p.rp2; g.cols = c2; g.K = p.kp2; g.w_is_b = 0;
  g.mode = GEMM_OUT_ROWS; g.vrows = 2 * n; g.vcols = c2; g.nk = n; g.nj = m; g.xo = p.Y; g.kpo = p.kp2;
  if ((e = launch_tc_gemm(g, s)) != cudaSuccess) return e;
  ++*launches;
  // row IDFT: D = Y G^T -> field (or the output plane)
  set_terms(g, p.Y, p.G);
  g.rows = pad256(c1); g.cols = 2 * n; g.K = p.kp2; g.w_is_b = 1;
  g.mode = GEMM_OUT_FIELD; g.vrows = c1; g.vcols = 2 * n; g.fld = p.fld; g.o = o; g.I = I; g.n = n; g.of = of;
  g.fov = fov;
  if ((e = launch_tc_gemm(g, s)) != cudaSuccess) return e;
  ++*launches;
  return cudaSuccess;
}

cudaError_t gemm_prep_field(GemmPlan& p, int nwc, const float2* v, float2* ckpt, const float* h,
                            const ChanConst* chan, int mode, int a_off, int a_w, cudaStream_t s) {
  k_prep_field<<<nwc * p.n, 128, 0, s>>>(v, ckpt, h, chan, p.X, p.n, p.kp1, mode, a_off, a_w);
  return cudaGetLastError();
}

cudaError_t gemm_seed(GemmPlan& p, int nwc, const float2* o, const float* dLdI, int of, int fov, cudaStream_t s) {
  const size_t total = (size_t)nwc * p.n * p.n;
  k_field_seed<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(p.fld, o, dLdI, p.n, of, fov, total);
  return cudaGetLastError();
}

cudaError_t gemm_adj_layer(GemmPlan& p, int nwc, const float2* ckpt, size_t ckpt_stride, const float* h,
                           const ChanConst* chan, float* partial, cudaStream_t s) {
  const size_t n2 = (size_t)p.n * p.n;
  k_field_adj<<<(unsigned)((n2 + 255) / 256), 256, 0, s>>>(p.fld, ckpt, ckpt_stride, h, chan, partial, nwc, p.n);
  return cudaGetLastError();
}

}  // namespace dos

