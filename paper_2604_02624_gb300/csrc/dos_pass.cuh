// dos_pass.cuh - row and column passes of the angular-spectrum cascade.
//
// One free-space gap (Eq. 4-5 realised as P_z(u) = crop(IDFT(H * DFT(pad u))))
// is split into a row pass and a column pass over an [nw][n][m] buffer S of
// row spectra.  The N x N layer occupies rows/columns [0, N) of the padded
// M x M grid; by shift invariance of circular convolution this equals the
// centred placement.
//
//   row pass    : per (channel, row): inverse row DFT of the previous column
//                 pass (-> field, cropped to N), modulation by the layer's
//                 transmission t (Eq. 1-2) or the adjoint chain, zero pad,
//                 forward row DFT.  One read and one write of a row of M.
//   column pass : per (channel, column tile): forward column DFT of the
//                 N non-zero rows, multiply by H (conj H for the adjoint),
//                 inverse column DFT, keep the rows that are needed.
//
// Each kernel keeps every element of a line in registers across both of its
// transforms; the only shared-memory traffic is the one exchange inside each
// line DFT.
#pragma once

#include "dos_fft.cuh"
#include "dos_internal.h"

namespace dos {

// Transmission of Eq. 1 at thickness h (Eq. 2 base folded into the constants):
// t = exp(-2 pi kappa h / lambda) exp(-j 2 pi (n - n_med) h / lambda).
// The phase in cycles is formed as a float-pair product (exact product error
// by fma) and reduced modulo 1 before sincospi, which keeps ~1e-7 cycle
// accuracy for any thickness.
__device__ __forceinline__ float2 transmission(float h, const ChanConst& cc) {
  const float p = cc.a_hi * h;
  float e = fmaf(cc.a_hi, h, -p);
  e = fmaf(cc.a_lo, h, e);
  float f = (p - rintf(p)) + (e + cc.pc_base);
  f -= rintf(f);
  float s, c;
  sincospif(2.0f * f, &s, &c);
  const float amp = exp2f(cc.amp_k * h) * cc.amp_base;
  return make_float2(amp * c, -amp * s);
}

// Stride between the lines' exchange buffers in the row passes.  There the
// T threads of a line are consecutive (line = tid / T), so a warp straddles
// two or more lines; these strides make the 8-byte exchange accesses of such
// warps free of bank conflicts (least-conflict for M = 200), found by
// enumerating the bank pattern of every access of the compiled line shapes.
constexpr int row_line_stride(int m, int zs) {
  return m == 400 ? 420 : m == 200 ? 222 : m == 128 ? 148 : m == 32 ? 42 : zs;
}

// HALF (N <= M / 2, every compiled design with M = 2N): the field half of a
// line, x < M / 2, holds every non-zero input of a forward DFT and every output
// that is kept of an inverse one.  Thread t's elements t + T i with i < E / 2
// are exactly that half, and so are the first P / 2 inputs of each first-step
// sub-DFT and the first Q / 2 outputs of each second-step one: the line DFTs
// are pruned at compile time (NZF, NOI) and the field-domain loops stop at EF.
template <class LF, bool HALF = false>
struct Pass {
  static constexpr int T = LF::T, E = LF::E, M = LF::M;
  static constexpr int NZF = HALF ? LF::P / 2 : LF::P;  // forward DFT of a field: non-zero inputs per sub-DFT
  static constexpr int NOI = HALF ? LF::Q / 2 : LF::Q;  // inverse DFT to a field: outputs kept per sub-DFT
  static constexpr int EF = HALF ? E / 2 : E;           // field-domain elements of a thread
  static_assert(!HALF || (LF::P % 2 == 0 && LF::Q % 2 == 0), "halving needs even factors");
  // Packed FP32-pair butterflies (Line::fft's PK) where they measured faster
  // on the 400-point line: the row passes but the adjoint one (PKA) and not
  // this column pass (PKC), whose three-blocks-per-SM register budget they
  // overflow.
  static constexpr bool PKR = true, PKA = false, PKC = false;
  static constexpr int ROWL = 16;  // rows per block in the row passes
  static constexpr int COLL = 16;  // columns per block in the column pass
  // column pass: line = tid % COLL, an odd stride keeps the lines apart
  static constexpr int ZL = LF::ZS + 1;
  static constexpr int RZL = row_line_stride(M, LF::ZS);
  static constexpr size_t smem_bytes(int lines) { return sizeof(float2) * (LF::TWS + (size_t)lines * ZL); }
  static constexpr size_t row_smem_bytes(int lines) { return sizeof(float2) * (LF::TWS + (size_t)lines * RZL); }

  __device__ static __forceinline__ void load_tw(float2* tw, const float2* g) {
    for (int i = threadIdx.x; i < LF::TWS; i += blockDim.x) tw[i] = g[i];
    __syncthreads();
  }

  // ------------------------------------------------------------ column pass
  template <bool ADJ, bool APERTURE>
  __device__ static void col(const PassArgs& a) {
    extern __shared__ __align__(16) float2 smem[];
    float2* tw = smem;
    const int l = threadIdx.x % COLL;
    const int t = threadIdx.x / COLL;
    float2* z = smem + LF::TWS + l * ZL;
    load_tw(tw, a.tw);
    const int w = blockIdx.y;
    const int c = blockIdx.x * COLL + l;
    const bool ok = c < M;
    const int cc = ok ? c : 0;
    float2 r[E];
    if constexpr (APERTURE) {
      // spectrum of the square aperture: Arow[ky] * Arow[kx]
      const float2 ac = a.arow[cc];
#pragma unroll
      for (int i = 0; i < E; ++i) r[i] = cmul(a.arow[t + T * i], ac);
    } else {
      const float2* src = a.S + (size_t)w * a.n * M + cc;
#pragma unroll
      for (int i = 0; i < E; ++i) {
        const int row = t + T * i;
        r[i] = (i < EF && ok && row >= a.in_r0 && row < a.in_r1) ? src[(size_t)row * M] : czero();
      }
      LF::template fft<false, NZF, LF::Q, true, PKC>(r, t, z, tw);
    }
    const float2* Hw = a.Hq + (size_t)w * a.hs * a.hs;
    const float* Sw = a.mis.sq ? a.mis.sq + (size_t)w * a.hs * a.hs : nullptr;
    const int bc = min(cc, M - cc);
#pragma unroll
    for (int i = 0; i < E; ++i) {
      const int k = t + T * i;
      const size_t qi = (size_t)min(k, M - k) * a.hs + bc;
      float2 hv = Hw[qi];
      if (Sw) hv = cmul(hv, misalign_factor(a.mis, k, cc, M, Sw[qi]));
      r[i] = ADJ ? cmulc(r[i], hv) : cmul(r[i], hv);
    }
    LF::template fft<true, LF::P, NOI, true, PKC>(r, t, z, tw);
    float2* dst = a.S + (size_t)w * a.n * M + cc;
#pragma unroll
    for (int i = 0; i < E; ++i) {
      const int row = t + T * i;
      if (i < EF && ok && row >= a.out_r0 && row < a.out_r1) dst[(size_t)row * M] = r[i];
    }
  }

  // ------------------------------------------------------------- row passes
  struct RowCtx {
    int l, t;
    float2* z;
    float2* tw;
  };
  __device__ static __forceinline__ RowCtx row_ctx(const PassArgs& a) {
    extern __shared__ __align__(16) float2 smem[];
    RowCtx rc;
    rc.l = threadIdx.x / T;
    rc.t = threadIdx.x % T;
    rc.tw = smem;
    rc.z = smem + LF::TWS + rc.l * RZL;
    load_tw(rc.tw, a.tw);
    return rc;
  }

  // forward, layer l: IDFT -> v (crop) -> [checkpoint] -> t*v -> pad -> DFT
  template <bool SAVE>
  __device__ static void row_fwd(const PassArgs& a) {
    const RowCtx rc = row_ctx(a);
    const int t = rc.t;
    const int w = blockIdx.y;
    const int row = blockIdx.x * ROWL + rc.l;
    const bool ok = row < a.n;
    const int rr = ok ? row : 0;
    float2* srow = a.S + ((size_t)w * a.n + rr) * M;
    float2 r[E];
#pragma unroll
    for (int i = 0; i < E; ++i) r[i] = srow[t + T * i];
    LF::template fft<true, LF::P, NOI, true, PKR>(r, t, rc.z, rc.tw);
    const ChanConst cc = a.chan[w];
    const float* hrow = a.h + (size_t)rr * a.n;
    float2* ck = a.ckpt + ((size_t)w * a.n + rr) * a.n;
#pragma unroll
    for (int i = 0; i < E; ++i) {
      const int x = t + T * i;
      if (i < EF && x < a.n) {
        const float2 v = r[i];
        if (SAVE && ok) ck[x] = v;
        r[i] = cmul(transmission(hrow[x], cc), v);
      } else {
        r[i] = czero();
      }
    }
    LF::template fft<false, NZF, LF::Q, true, PKR>(r, t, rc.z, rc.tw);
    if (ok) {
#pragma unroll
      for (int i = 0; i < E; ++i) srow[t + T * i] = r[i];
    }
  }

  // first layer from the create-time input field v1 = P_z0(aperture) (a.fin):
  // u = t(h) v1 -> pad -> forward row DFT.  No inverse DFT, and no checkpoint:
  // the table itself is the first layer's incoming field.
  __device__ static void row_first(const PassArgs& a) {
    const RowCtx rc = row_ctx(a);
    const int t = rc.t;
    const int w = blockIdx.y;
    const int row = blockIdx.x * ROWL + rc.l;
    const bool ok = row < a.n;
    const int rr = ok ? row : 0;
    const float2* vrow = a.fin + ((size_t)w * a.n + rr) * a.n;
    const float* hrow = a.h + (size_t)rr * a.n;
    const ChanConst cc = a.chan[w];
    float2 r[E];
#pragma unroll
    for (int i = 0; i < E; ++i) {
      const int x = t + T * i;
      r[i] = (i < EF && x < a.n) ? cmul(transmission(hrow[x], cc), vrow[x]) : czero();
    }
    LF::template fft<false, NZF, LF::Q, true, PKR>(r, t, rc.z, rc.tw);
    if (ok) {
      float2* srow = a.S + ((size_t)w * a.n + row) * M;
#pragma unroll
      for (int i = 0; i < E; ++i) srow[t + T * i] = r[i];
    }
  }

  // output plane: IDFT of the FOV rows -> o (complex) and I = |o|^2; a
  // block's lines are consecutive (channel, FOV row) pairs, so no block is
  // left with a few rows of a channel
  __device__ static void row_out(const PassArgs& a) {
    const RowCtx rc = row_ctx(a);
    const int t = rc.t;
    const int line = blockIdx.x * ROWL + rc.l;
    const bool ok = line < a.nw * a.fov;
    const int w = ok ? line / a.fov : 0;
    const int fr = ok ? line % a.fov : 0;  // FOV row
    const int row = a.of + fr;
    const float2* srow = a.S + ((size_t)w * a.n + row) * M;
    float2 r[E];
#pragma unroll
    for (int i = 0; i < E; ++i) r[i] = srow[t + T * i];
    LF::template fft<true, LF::P, NOI, true, PKR>(r, t, rc.z, rc.tw);
    if (ok) {
      float2* orow = a.o + ((size_t)w * a.fov + fr) * a.fov;
      float* irow = a.I ? a.I + ((size_t)w * a.fov + fr) * a.fov : nullptr;
#pragma unroll
      for (int i = 0; i < E; ++i) {
        const int x = t + T * i - a.of;
        if (i < EF && x >= 0 && x < a.fov) {
          orow[x] = r[i];
          if (irow) irow[x] = fmaf(r[i].x, r[i].x, r[i].y * r[i].y);
        }
      }
    }
  }

  // adjoint seed: grad_o = 2 dL/dI o on the FOV, zero elsewhere -> DFT of the FOV rows
  // (lines as in row_out)
  __device__ static void row_seed(const PassArgs& a) {
    const RowCtx rc = row_ctx(a);
    const int t = rc.t;
    const int line = blockIdx.x * ROWL + rc.l;
    const bool ok = line < a.nw * a.fov;
    const int w = ok ? line / a.fov : 0;
    const int fr = ok ? line % a.fov : 0;
    const float2* orow = a.o + ((size_t)w * a.fov + fr) * a.fov;
    const float* grow = a.dLdI + ((size_t)w * a.fov + fr) * a.fov;
    float2 r[E];
#pragma unroll
    for (int i = 0; i < E; ++i) {
      const int x = t + T * i - a.of;
      r[i] = (i < EF && ok && x >= 0 && x < a.fov) ? cscale(orow[x], 2.0f * grow[x]) : czero();
    }
    LF::template fft<false, NZF, LF::Q, true, PKR>(r, t, rc.z, rc.tw);
    if (ok) {
      float2* srow = a.S + ((size_t)w * a.n + a.of + fr) * M;
#pragma unroll
      for (int i = 0; i < E; ++i) srow[t + T * i] = r[i];
    }
  }

  // adjoint, layer l, for a chunk of channels:
  //   IDFT -> grad_u (crop); u = t v from the checkpoint;
  //   dL/dh += Re(conj(grad_u) c u) (accumulated over the chunk in registers);
  //   grad_v = conj(t) grad_u -> pad -> DFT (skipped for the first layer)
  template <bool FIRST>
  __device__ static void row_adj(const PassArgs& a) {
    const RowCtx rc = row_ctx(a);
    const int t = rc.t;
    const int row = blockIdx.x * ROWL + rc.l;
    const bool ok = row < a.n;
    const int rr = ok ? row : 0;
    const int w0 = blockIdx.y * a.chunk;
    const int w1 = min(a.nw, w0 + a.chunk);
    const float* hrow = a.h + (size_t)rr * a.n;
    float g[E];
#pragma unroll
    for (int i = 0; i < E; ++i) g[i] = 0.f;
    for (int w = w0; w < w1; ++w) {
      float2* srow = a.S + ((size_t)w * a.n + rr) * M;
      const float2* ck = a.ckpt + ((size_t)w * a.n + rr) * a.n;
      float2 r[E];
#pragma unroll
      for (int i = 0; i < E; ++i) r[i] = srow[t + T * i];
      LF::template fft<true, LF::P, NOI, true, PKA>(r, t, rc.z, rc.tw);
      const ChanConst cc = a.chan[w];
#pragma unroll
      for (int i = 0; i < E; ++i) {
        const int x = t + T * i;
        if (i < EF && x < a.n) {
          const float2 au = r[i];
          const float2 tt = transmission(hrow[x], cc);
          const float2 cu = cmul(make_float2(cc.c_re, cc.c_im), cmul(tt, ck[x]));
          g[i] = fmaf(au.x, cu.x, fmaf(au.y, cu.y, g[i]));
          r[i] = cmulc(au, tt);
        } else {
          r[i] = czero();
        }
      }
      if constexpr (!FIRST) {
        LF::template fft<false, NZF, LF::Q, true, PKA>(r, t, rc.z, rc.tw);
        if (ok) {
#pragma unroll
          for (int i = 0; i < E; ++i) srow[t + T * i] = r[i];
        }
      }
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

  // caller field -> pad -> row DFT (dos_propagate)
  __device__ static void row_in(const PassArgs& a) {
    const RowCtx rc = row_ctx(a);
    const int t = rc.t;
    const int w = blockIdx.y;
    const int row = blockIdx.x * ROWL + rc.l;
    const bool ok = row < a.n;
    const int rr = ok ? row : 0;
    const float2* frow = a.fin + ((size_t)w * a.n + rr) * a.n;
    float2 r[E];
#pragma unroll
    for (int i = 0; i < E; ++i) {
      const int x = t + T * i;
      r[i] = (i < EF && x < a.n) ? frow[x] : czero();
    }
    LF::template fft<false, NZF, LF::Q, true, PKR>(r, t, rc.z, rc.tw);
    if (ok) {
      float2* srow = a.S + ((size_t)w * a.n + row) * M;
#pragma unroll
      for (int i = 0; i < E; ++i) srow[t + T * i] = r[i];
    }
  }

  // row spectra -> IDFT -> crop -> caller field (dos_propagate)
  __device__ static void row_back(const PassArgs& a) {
    const RowCtx rc = row_ctx(a);
    const int t = rc.t;
    const int w = blockIdx.y;
    const int row = blockIdx.x * ROWL + rc.l;
    const bool ok = row < a.n;
    const int rr = ok ? row : 0;
    const float2* srow = a.S + ((size_t)w * a.n + rr) * M;
    float2 r[E];
#pragma unroll
    for (int i = 0; i < E; ++i) r[i] = srow[t + T * i];
    LF::template fft<true, LF::P, NOI, true, PKR>(r, t, rc.z, rc.tw);
    if (ok) {
      float2* frow = a.fout + ((size_t)w * a.n + row) * a.n;
#pragma unroll
      for (int i = 0; i < E; ++i) {
        const int x = t + T * i;
        if (i < EF && x < a.n) frow[x] = r[i];
      }
    }
  }
};

// ------------------------------------------------------------------ kernels
// The forward row pass of lines with up to 20 elements per thread fits three
// blocks per SM in 64 registers per thread without spills (measured faster than
// two; the column pass is faster with its own register allocation).
template <class LF>
constexpr int pass_min_blocks() { return LF::E <= 20 ? 3 : 1; }
// column pass: the halved kernel fits three blocks per SM without spills
template <class LF, bool HALF>
constexpr int col_min_blocks() { return HALF && LF::M == 400 ? 3 : 0; }

template <class LF, bool HALF, bool ADJ, bool APERTURE>
__global__ void __launch_bounds__(LF::T * Pass<LF>::COLL, col_min_blocks<LF, HALF>()) k_col(PassArgs a) {
  Pass<LF, HALF>::template col<ADJ, APERTURE>(a);
}
template <class LF, bool HALF, bool SAVE>
__global__ void __launch_bounds__(LF::T * Pass<LF>::ROWL, pass_min_blocks<LF>()) k_row_fwd(PassArgs a) {
  Pass<LF, HALF>::template row_fwd<SAVE>(a);
}
template <class LF, bool HALF>
__global__ void __launch_bounds__(LF::T * Pass<LF>::ROWL, pass_min_blocks<LF>()) k_row_first(PassArgs a) {
  Pass<LF, HALF>::row_first(a);
}
// the output and seed passes: three blocks per SM where the lines are short
// (the register count would otherwise drift past 64 and leave two)
template <class LF, bool HALF>
__global__ void __launch_bounds__(LF::T * Pass<LF>::ROWL, pass_min_blocks<LF>()) k_row_out(PassArgs a) {
  Pass<LF, HALF>::row_out(a);
}
template <class LF, bool HALF>
__global__ void __launch_bounds__(LF::T * Pass<LF>::ROWL, pass_min_blocks<LF>()) k_row_seed(PassArgs a) {
  Pass<LF, HALF>::row_seed(a);
}
template <class LF, bool HALF, bool FIRST>
__global__ void __launch_bounds__(LF::T * Pass<LF>::ROWL, col_min_blocks<LF, HALF>()) k_row_adj(PassArgs a) {
  Pass<LF, HALF>::template row_adj<FIRST>(a);
}
template <class LF, bool HALF>
__global__ void __launch_bounds__(LF::T * Pass<LF>::ROWL) k_row_in(PassArgs a) {
  Pass<LF, HALF>::row_in(a);
}
template <class LF, bool HALF>
__global__ void __launch_bounds__(LF::T * Pass<LF>::ROWL) k_row_back(PassArgs a) {
  Pass<LF, HALF>::row_back(a);
}

template <typename K>
static cudaError_t launch_k(K kernel, dim3 grid, int threads, size_t smem, const PassArgs& a,
                            cudaStream_t s) {
  if (grid.x == 0 || grid.y == 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kernel<<<grid, threads, smem, s>>>(a);
  return cudaGetLastError();
}

// Each launcher picks the halved (pruned) kernels when the design allows it.
template <class LF>
struct PassLaunch {
  using PS = Pass<LF>;
  static constexpr int RT = LF::T * PS::ROWL;
  static constexpr int CT = LF::T * PS::COLL;
  static int row_blocks(int rows) { return (rows + PS::ROWL - 1) / PS::ROWL; }
  static bool half(const PassArgs& a) { return 2 * a.n <= LF::M; }

  template <bool H>
  static cudaError_t col_h(const PassArgs& a, bool adj, bool ap, cudaStream_t s) {
    const dim3 g((LF::M + PS::COLL - 1) / PS::COLL, a.nw);
    const size_t sm = PS::smem_bytes(PS::COLL);
    if (ap) return adj ? launch_k(k_col<LF, H, true, true>, g, CT, sm, a, s)
                       : launch_k(k_col<LF, H, false, true>, g, CT, sm, a, s);
    return adj ? launch_k(k_col<LF, H, true, false>, g, CT, sm, a, s)
               : launch_k(k_col<LF, H, false, false>, g, CT, sm, a, s);
  }
  static cudaError_t col(const PassArgs& a, bool adj, bool ap, cudaStream_t s) {
    return half(a) ? col_h<true>(a, adj, ap, s) : col_h<false>(a, adj, ap, s);
  }
  template <bool H>
  static cudaError_t row_fwd_h(const PassArgs& a, bool save, cudaStream_t s) {
    const dim3 g(row_blocks(a.n), a.nw);
    const size_t sm = PS::row_smem_bytes(PS::ROWL);
    return save ? launch_k(k_row_fwd<LF, H, true>, g, RT, sm, a, s)
                : launch_k(k_row_fwd<LF, H, false>, g, RT, sm, a, s);
  }
  static cudaError_t row_fwd(const PassArgs& a, bool save, cudaStream_t s) {
    return half(a) ? row_fwd_h<true>(a, save, s) : row_fwd_h<false>(a, save, s);
  }
  static cudaError_t row_first(const PassArgs& a, cudaStream_t s) {
    const dim3 g(row_blocks(a.n), a.nw);
    const size_t sm = PS::row_smem_bytes(PS::ROWL);
    return half(a) ? launch_k(k_row_first<LF, true>, g, RT, sm, a, s)
                   : launch_k(k_row_first<LF, false>, g, RT, sm, a, s);
  }
  static cudaError_t row_out(const PassArgs& a, cudaStream_t s) {
    const dim3 g(row_blocks(a.nw * a.fov));
    const size_t sm = PS::row_smem_bytes(PS::ROWL);
    return half(a) ? launch_k(k_row_out<LF, true>, g, RT, sm, a, s) : launch_k(k_row_out<LF, false>, g, RT, sm, a, s);
  }
  static cudaError_t row_seed(const PassArgs& a, cudaStream_t s) {
    const dim3 g(row_blocks(a.nw * a.fov));
    const size_t sm = PS::row_smem_bytes(PS::ROWL);
    return half(a) ? launch_k(k_row_seed<LF, true>, g, RT, sm, a, s)
                   : launch_k(k_row_seed<LF, false>, g, RT, sm, a, s);
  }
  template <bool H>
  static cudaError_t row_adj_h(const PassArgs& a, bool first, cudaStream_t s) {
    const dim3 g(row_blocks(a.n), a.n_chunks);
    const size_t sm = PS::row_smem_bytes(PS::ROWL);
    return first ? launch_k(k_row_adj<LF, H, true>, g, RT, sm, a, s)
                 : launch_k(k_row_adj<LF, H, false>, g, RT, sm, a, s);
  }
  static cudaError_t row_adj(const PassArgs& a, bool first, cudaStream_t s) {
    return half(a) ? row_adj_h<true>(a, first, s) : row_adj_h<false>(a, first, s);
  }
  static cudaError_t row_in(const PassArgs& a, cudaStream_t s) {
    const dim3 g(row_blocks(a.n), a.nw);
    const size_t sm = PS::row_smem_bytes(PS::ROWL);
    return half(a) ? launch_k(k_row_in<LF, true>, g, RT, sm, a, s) : launch_k(k_row_in<LF, false>, g, RT, sm, a, s);
  }
  static cudaError_t row_back(const PassArgs& a, cudaStream_t s) {
    const dim3 g(row_blocks(a.n), a.nw);
    const size_t sm = PS::row_smem_bytes(PS::ROWL);
    return half(a) ? launch_k(k_row_back<LF, true>, g, RT, sm, a, s)
                   : launch_k(k_row_back<LF, false>, g, RT, sm, a, s);
  }
};

}  // namespace dos
