// dos_fused.cuh - cluster-resident forward and adjoint sweeps (one launch each).
//
// A thread-block cluster of C CTAs owns one wavelength channel at a time and
// carries it through every gap of the cascade (Eq. 1-5) without the field
// leaving the chip.  The N x M plane of row spectra is distributed over the
// cluster's shared memory by interleaved rows (row r lives in CTA r mod C at
// local slot r / C):
//
//   row phase    : each CTA transforms its own rows in local shared memory
//                  (IDFT, crop, checkpoint, Eq. 1 modulation, pad, DFT);
//   column phase : each CTA owns M/C columns, gathers them from every CTA's
//                  shared memory (distributed shared memory), runs the column
//                  DFT, multiplies by H (L2-resident table of the channel),
//                  runs the inverse DFT and scatters the N rows back.
//
// The layer must fit in half the padded grid (N <= M/2, as for M = 2N): then
// only the first half of each line is ever non-zero on input or needed on
// output, and every line DFT is pruned at compile time.
//
// Two cluster barriers per gap separate the phases.  Global memory sees only
// the checkpoints (written forward, read by the adjoint), the transfer table,
// the thickness, the output field and the gradient partials.  Clusters take
// channels w = cluster, cluster + n_clusters, ... so every result, including
// the gradient sum, is reproducible run to run.
#pragma once

#include <cooperative_groups.h>

#include "dos_pass.cuh"

namespace dos {

namespace cg = cooperative_groups;

constexpr int kMaxGaps = 65;

struct FusedArgs {
  const float2* Hq;          // [n_slots][nw][hs][hs]
  size_t hq_slot_stride;     // nw * hs * hs
  int gap_slot[kMaxGaps];    // gap -> table slot
  const float2* arow;        // [m]
  const float2* tw;          // [Q * RP]
  const ChanConst* chan;     // [nw]
  const float* h;            // [K][n][n]
  float2* ckpt;              // [K][nw][n][n] incoming field v of each layer
  const float2* v1;          // [nw][n][n] create-time input field v1 = P_z0(aperture), or null:
                             // then layer 1 starts from it (no gap-0 phase) and it is layer 1's checkpoint
  float2* ckt;               // [K][nw][n][n] transmission t of each layer and channel
  float2* o;                 // [nw][fov][fov]
  float* I;                  // [nw][fov][fov] or null
  const float* dLdI;         // [nw][fov][fov]
  float* partial;            // [n_clusters][K][n][n]
  int n, nw, K, fov, of, hs;
  int save;
  const float* sq;             // [nw][hs][hs] signed sqrt(|q|) when layers are misaligned, else null
  float df;                    // DFT bin spacing [1/m]
  float mis[kMaxGaps][3];      // per gap: lateral shift (x, y) and length change [m]
};

constexpr int ct_gcd(int a, int b) { return b == 0 ? a : ct_gcd(b, a % b); }

template <class LF, int C, int LINES>
struct Fused {
  static constexpr int T = LF::T, E = LF::E, M = LF::M, ZS = LF::ZS, ZL = ZS + 1;
  static constexpr int NT = LINES * T;
  static constexpr int EH = E / 2;             // elements of a thread inside [0, M/2), the only ones in the layer
  static constexpr int PH = LF::P / 2, QH = LF::Q / 2;  // pruning: half the inputs are padding, half the outputs cropped
  static constexpr bool FPK = false;  // packed FP32-pair butterflies measured 1 % slower here
  static constexpr int MC = (M + C - 1) / C;  // columns per CTA
  // rows t + T*i of a column: owner (row mod C) repeats with this period in i
  static constexpr int PERIOD = (T % C) == 0 ? 1 : C / ct_gcd(T % C, C);
  static constexpr int LR_STEP = T * PERIOD / C;  // local-row step per period
  static_assert((T * PERIOD) % C == 0, "row ownership period");
  static_assert(E % PERIOD == 0, "elements per thread must cover whole periods");
  static_assert(LF::P % 2 == 0 && LF::Q % 2 == 0 && E % 2 == 0, "pruned halves");

  // Transfer-table values of a column are issued before its forward DFT when
  // the register budget (65536 / threads) leaves room for them.
  static constexpr bool kPrefetchH = NT <= 400;

  // H(|ky|, |kx|) for the thread's frequencies k = t + T*i of column cc:
  // |k| = k below M/2 and M - k above, both affine in i at compile time.
  __device__ static __forceinline__ void load_h(float2 (&hreg)[E], const float2* __restrict__ Hw, int hs, int t,
                                                int cc, const float* __restrict__ Sw, const Misalign& mg) {
    const int bc = min(cc, M - cc);
    const float2* lo = Hw + (size_t)t * hs + bc;
    const float2* hi = Hw + (size_t)(M - t) * hs + bc;
#pragma unroll
    for (int i = 0; i < E; ++i)
      hreg[i] = i < EH ? __ldg(lo + (size_t)T * i * hs) : __ldg(hi - (size_t)T * i * hs);
    if (Sw) {
      const float* slo = Sw + (size_t)t * hs + bc;
      const float* shi = Sw + (size_t)(M - t) * hs + bc;
#pragma unroll
      for (int i = 0; i < E; ++i) {
        const float sv = i < EH ? __ldg(slo + (size_t)T * i * hs) : __ldg(shi - (size_t)T * i * hs);
        hreg[i] = cmul(hreg[i], misalign_factor(mg, t + T * i, cc, M, sv));
      }
    }
  }

  static size_t smem_bytes(int n) {
    const int R = (n + C - 1) / C;
    return sizeof(float2) * (tw_offset(R) + LF::TWS);
  }
  // the twiddle table starts on a 16-byte boundary (Line reads it in pairs)
  __host__ __device__ static constexpr size_t tw_offset(int R) {
    return ((size_t)R * ZS + (size_t)LINES * ZL + 1) & ~(size_t)1;
  }

  struct Sm {
    float2* sp;    // [R][ZS] this CTA's rows of the spectrum plane (also their DFT exchange)
    float2* colz;  // [LINES][ZL] exchange buffers of the column lines
    float2* tw;    // [TWS]
    int R;
  };

  __device__ static Sm carve(const FusedArgs& a) {
    extern __shared__ __align__(16) float2 smem[];
    Sm s;
    s.R = (a.n + C - 1) / C;
    s.sp = smem;
    s.colz = smem + (size_t)s.R * ZS;
    s.tw = smem + tw_offset(s.R);
    for (int i = threadIdx.x; i < LF::TWS; i += NT) s.tw[i] = a.tw[i];
    __syncthreads();
    return s;
  }

  // ------------------------------------------------------------- column phase
  // Columns [rank*MC, rank*MC + MC) of the plane; rows [in_r0, in_r1) are read
  // (others are zero), rows [out_r0, out_r1) are written back.
  template <bool ADJ, bool APERTURE>
  __device__ static void col_phase(const cg::cluster_group& cl, const Sm& s, const float2* __restrict__ Hw,
                                   const float2* __restrict__ arow, int n, int hs, int in_r0, int in_r1,
                                   int out_r0, int out_r1, const float* __restrict__ Sw, const Misalign& mg) {
    const int l = threadIdx.x % LINES;
    const int t = threadIdx.x / LINES;
    const int rank = (int)cl.block_rank();
    float2* z = s.colz + l * ZL;
    // remote row bases of this thread's rows t + T*(p + PERIOD*m)
    float2* rb[PERIOD];
#pragma unroll
    for (int p = 0; p < PERIOD; ++p) {
      const int row = t + T * p;
      rb[p] = cl.map_shared_rank(s.sp, (unsigned)(row % C)) + (size_t)(row / C) * ZS;
    }
    const int c0 = rank * MC;
    // the next round's column values are fetched from the peers' shared memory
    // while the current round computes (software pipeline over rounds)
    float2 rnext[EH];
    auto fetch = [&](int cb, float2 (&dst)[EH]) {
      const int c = c0 + cb + l;
      const bool ok = (cb + l) < MC && c < M;
      const int cc = ok ? c : c0;
#pragma unroll
      for (int i = 0; i < EH; ++i) {
        const int row = t + T * i;
        const float2* src = rb[i % PERIOD] + (size_t)(i / PERIOD) * LR_STEP * ZS + cc;
        dst[i] = (ok && row >= in_r0 && row < in_r1) ? *src : czero();
      }
    };
    if constexpr (!APERTURE) fetch(0, rnext);
    for (int cb = 0; cb < MC; cb += LINES) {
      const int c = c0 + cb + l;
      const bool ok = (cb + l) < MC && c < M;
      const int cc = ok ? c : c0;
      float2 r[E];
      float2 hreg[E];
      if constexpr (kPrefetchH) load_h(hreg, Hw, hs, t, cc, Sw, mg);
      if constexpr (APERTURE) {
        const float2 ac = arow[cc];
#pragma unroll
        for (int i = 0; i < E; ++i) r[i] = cmul(arow[t + T * i], ac);
      } else {
#pragma unroll
        for (int i = 0; i < EH; ++i) r[i] = rnext[i];
        if (cb + LINES < MC) fetch(cb + LINES, rnext);
        LF::template fft<false, PH, LF::Q, true, FPK>(r, t, z, s.tw);
      }
      if constexpr (!kPrefetchH) load_h(hreg, Hw, hs, t, cc, Sw, mg);
#pragma unroll
      for (int i = 0; i < E; ++i) r[i] = ADJ ? cmulc(r[i], hreg[i]) : cmul(r[i], hreg[i]);
      LF::template fft<true, LF::P, QH, true, FPK>(r, t, z, s.tw);
#pragma unroll
      for (int i = 0; i < EH; ++i) {
        const int row = t + T * i;
        if (ok && row >= out_r0 && row < out_r1 && row < n)
          rb[i % PERIOD][(size_t)(i / PERIOD) * LR_STEP * ZS + cc] = r[i];
      }
    }
  }

  // --------------------------------------------------------------- row phases
  // Local slot j holds plane row rank + C*j.  Lines take slots j0 + l.
  struct RowLine {
    int t, l;
  };

  // forward, layer l (0-based): IDFT -> v -> [checkpoint v, t] -> t v -> pad -> DFT.
  // The IDFT exchanges through the row's own slot, the DFT through the line's
  // column buffer (idle in this phase), so a round needs three barriers.
  __device__ static void row_fwd_phase(const cg::cluster_group& cl, const Sm& s, const FusedArgs& a,
                                       int layer, int w) {
    const int t = threadIdx.x % T;
    const int l = threadIdx.x / T;
    const int rank = (int)cl.block_rank();
    const ChanConst cc = a.chan[w];
    const float* hl = a.h + (size_t)layer * a.n * a.n;
    float2* ck = a.ckpt + ((size_t)layer * a.nw + w) * a.n * a.n;
    float2* ct = a.ckt + ((size_t)layer * a.nw + w) * a.n * a.n;
    const bool from_v1 = layer == 0 && a.v1;
    // the column buffers double as row-phase exchange space, at the row-slot
    // stride (ZS): with the row phase's thread layout that stride is conflict-free
    float2* zc = s.colz + l * ZS;
    for (int j0 = 0; j0 < s.R; j0 += LINES) {
      const int j = j0 + l;
      const int row = rank + C * j;
      const bool ok = j < s.R && row < a.n;
      float2* z = j < s.R ? s.sp + (size_t)j * ZS : zc;
      const float* hrow = hl + (size_t)(ok ? row : 0) * a.n;
      float hv[EH];
#pragma unroll
      for (int i = 0; i < EH; ++i) {
        const int x = t + T * i;
        hv[i] = (ok && x < a.n) ? __ldg(hrow + x) : 0.f;
      }
      float2 r[E];
      const size_t ro = (size_t)(ok ? row : 0) * a.n;
      if (from_v1) {
        // layer 1 from the input-field table (uniform across the block); the
        // barrier keeps the previous round's readers of zc ahead of this
        // round's forward DFT, as the inverse DFT's barriers do otherwise
        const float2* vrow = a.v1 + (size_t)w * a.n * a.n + ro;
#pragma unroll
        for (int i = 0; i < E; ++i) {
          const int x = t + T * i;
          r[i] = (i < EH && ok && x < a.n) ? vrow[x] : czero();
        }
        __syncthreads();
      } else {
#pragma unroll
        for (int i = 0; i < E; ++i) r[i] = z[t + T * i];
        __syncthreads();
        LF::template fft<true, LF::P, QH, false, FPK>(r, t, z, s.tw);
      }
#pragma unroll
      for (int i = 0; i < EH; ++i) {
        const int x = t + T * i;
        if (x < a.n) {
          const float2 v = r[i];
          const float2 tt = transmission(hv[i], cc);
          if (ok && a.save) {
            if (!from_v1) ck[ro + x] = v;
            ct[ro + x] = tt;
          }
          r[i] = cmul(tt, v);
        } else {
          r[i] = czero();
        }
      }
      LF::template fft<false, PH, LF::Q, false, FPK>(r, t, zc, s.tw);
#pragma unroll
      for (int i = 0; i < E; ++i) z[t + T * i] = r[i];
    }
    __syncthreads();
  }

  // first local slot whose row is >= r0
  __device__ static int first_slot(int rank, int r0) { return r0 > rank ? (r0 - rank + C - 1) / C : 0; }

  // output plane: FOV rows -> IDFT -> o, I
  __device__ static void out_phase(const cg::cluster_group& cl, const Sm& s, const FusedArgs& a, int w) {
    const int t = threadIdx.x % T;
    const int l = threadIdx.x / T;
    const int rank = (int)cl.block_rank();
    const int jb = first_slot(rank, a.of);
    const int je = first_slot(rank, a.of + a.fov);
    for (int j0 = jb; j0 < je; j0 += LINES) {
      const int j = j0 + l;
      const int row = rank + C * j;
      const bool ok = j < je;
      float2* z = ok ? s.sp + (size_t)j * ZS : s.colz + l * ZL;
      float2 r[E];
#pragma unroll
      for (int i = 0; i < E; ++i) r[i] = z[t + T * i];
      __syncthreads();
      LF::template fft<true, LF::P, QH, true, FPK>(r, t, z, s.tw);
      if (ok) {
        const int fr = row - a.of;
        float2* orow = a.o + ((size_t)w * a.fov + fr) * a.fov;
        float* irow = a.I ? a.I + ((size_t)w * a.fov + fr) * a.fov : nullptr;
#pragma unroll
        for (int i = 0; i < EH; ++i) {
          const int x = t + T * i - a.of;
          if (x >= 0 && x < a.fov) {
            orow[x] = r[i];
            if (irow) irow[x] = fmaf(r[i].x, r[i].x, r[i].y * r[i].y);
          }
        }
      }
    }
  }

  // adjoint seed: 2 dL/dI o on the FOV rows -> DFT -> plane rows
  __device__ static void seed_phase(const cg::cluster_group& cl, const Sm& s, const FusedArgs& a, int w) {
    const int t = threadIdx.x % T;
    const int l = threadIdx.x / T;
    const int rank = (int)cl.block_rank();
    const int jb = first_slot(rank, a.of);
    const int je = first_slot(rank, a.of + a.fov);
    for (int j0 = jb; j0 < je; j0 += LINES) {
      const int j = j0 + l;
      const int row = rank + C * j;
      const bool ok = j < je;
      float2* z = ok ? s.sp + (size_t)j * ZS : s.colz + l * ZL;
      const int fr = ok ? row - a.of : 0;
      const float2* orow = a.o + ((size_t)w * a.fov + fr) * a.fov;
      const float* grow = a.dLdI + ((size_t)w * a.fov + fr) * a.fov;
      float2 r[E];
#pragma unroll
      for (int i = 0; i < EH; ++i) {
        const int x = t + T * i - a.of;
        r[i] = (ok && x >= 0 && x < a.fov) ? cscale(orow[x], 2.0f * grow[x]) : czero();
      }
      LF::template fft<false, PH, LF::Q, true, FPK>(r, t, z, s.tw);
      if (ok) {
#pragma unroll
        for (int i = 0; i < E; ++i) z[t + T * i] = r[i];
      }
      __syncthreads();
    }
  }

  // adjoint, layer l: IDFT -> grad_u; u = t v (both checkpointed by the forward
  // sweep); partial += Re(conj(grad_u) c u); grad_v = conj(t) grad_u -> pad ->
  // DFT (not for the first layer)
  __device__ static void row_adj_phase(const cg::cluster_group& cl, const Sm& s, const FusedArgs& a,
                                       int layer, int w, float* part, bool first_channel) {
    const int t = threadIdx.x % T;
    const int l = threadIdx.x / T;
    const int rank = (int)cl.block_rank();
    const ChanConst cc = a.chan[w];
    const float2* ck = (layer == 0 && a.v1) ? a.v1 + (size_t)w * a.n * a.n
                                            : a.ckpt + ((size_t)layer * a.nw + w) * a.n * a.n;
    const float2* ct = a.ckt + ((size_t)layer * a.nw + w) * a.n * a.n;
    float* pl = part + (size_t)layer * a.n * a.n;
    const bool last = layer == 0;
    // the column buffers double as row-phase exchange space, at the row-slot
    // stride (ZS): with the row phase's thread layout that stride is conflict-free
    float2* zc = s.colz + l * ZS;
    for (int j0 = 0; j0 < s.R; j0 += LINES) {
      const int j = j0 + l;
      const int row = rank + C * j;
      const bool ok = j < s.R && row < a.n;
      float2* z = j < s.R ? s.sp + (size_t)j * ZS : zc;
      const size_t ro = (size_t)(ok ? row : 0) * a.n;
      float2 tv[EH];
      float2 vv[EH];
      float pv[EH];
#pragma unroll
      for (int i = 0; i < EH; ++i) {
        const int x = t + T * i;
        const bool in = ok && x < a.n;
        tv[i] = in ? ct[ro + x] : czero();
        vv[i] = in ? ck[ro + x] : czero();
        pv[i] = (in && !first_channel) ? pl[ro + x] : 0.f;
      }
      float2 r[E];
#pragma unroll
      for (int i = 0; i < E; ++i) r[i] = z[t + T * i];
      __syncthreads();
      LF::template fft<true, LF::P, QH, false, FPK>(r, t, z, s.tw);
      const float2 cf = make_float2(cc.c_re, cc.c_im);
#pragma unroll
      for (int i = 0; i < EH; ++i) {
        const int x = t + T * i;
        if (x < a.n) {
          const float2 au = r[i];
          const float2 cu = cmul(cf, cmul(tv[i], vv[i]));
          if (ok) pl[ro + x] = fmaf(au.x, cu.x, fmaf(au.y, cu.y, pv[i]));
          r[i] = cmulc(au, tv[i]);
        } else {
          r[i] = czero();
        }
      }
      if (!last) {
        LF::template fft<false, PH, LF::Q, false, FPK>(r, t, zc, s.tw);
#pragma unroll
        for (int i = 0; i < E; ++i) z[t + T * i] = r[i];
      }
    }
    __syncthreads();
  }

  __device__ static const float2* table(const FusedArgs& a, int gap, int w) {
    return a.Hq + (size_t)a.gap_slot[gap] * a.hq_slot_stride + (size_t)w * a.hs * a.hs;
  }
  __device__ static const float* sqt(const FusedArgs& a, int w) {
    return a.sq ? a.sq + (size_t)w * a.hs * a.hs : nullptr;
  }
  __device__ static Misalign mis(const FusedArgs& a, int gap) {
    Misalign m;
    m.sq = a.sq;
    m.df = a.df;
    m.ax = a.mis[gap][0];
    m.ay = a.mis[gap][1];
    m.dz = a.mis[gap][2];
    return m;
  }

  // --------------------------------------------------------------- sweeps
  __device__ static void forward(const FusedArgs& a) {
    cg::cluster_group cl = cg::this_cluster();
    const Sm s = carve(a);
    const int cid = blockIdx.x / C;
    const int ncl = gridDim.x / C;
    for (int w = cid; w < a.nw; w += ncl) {
      if (!a.v1) {  // gap 0 from the aperture (the table is not used with displaced layers)
        col_phase<false, true>(cl, s, table(a, 0, w), a.arow, a.n, a.hs, 0, 0, 0, a.n, sqt(a, w), mis(a, 0));
        cl.sync();
      }
      for (int layer = 0; layer < a.K; ++layer) {
        row_fwd_phase(cl, s, a, layer, w);
        cl.sync();
        const bool lastgap = layer == a.K - 1;
        col_phase<false, false>(cl, s, table(a, layer + 1, w), a.arow, a.n, a.hs, 0, a.n,
                                lastgap ? a.of : 0, lastgap ? a.of + a.fov : a.n, sqt(a, w), mis(a, layer + 1));
        cl.sync();
      }
      out_phase(cl, s, a, w);
      cl.sync();
    }
  }

  __device__ static void adjoint(const FusedArgs& a) {
    cg::cluster_group cl = cg::this_cluster();
    const Sm s = carve(a);
    const int cid = blockIdx.x / C;
    const int ncl = gridDim.x / C;
    float* part = a.partial + (size_t)cid * a.K * a.n * a.n;
    for (int w = cid; w < a.nw; w += ncl) {
      seed_phase(cl, s, a, w);
      cl.sync();
      for (int layer = a.K - 1; layer >= 0; --layer) {
        const bool lastgap = layer == a.K - 1;
        col_phase<true, false>(cl, s, table(a, layer + 1, w), a.arow, a.n, a.hs,
                               lastgap ? a.of : 0, lastgap ? a.of + a.fov : a.n, 0, a.n, sqt(a, w), mis(a, layer + 1));
        cl.sync();
        row_adj_phase(cl, s, a, layer, w, part, w == cid);
        cl.sync();
      }
    }
  }
};

template <class LF, int C, int LINES>
__global__ void __launch_bounds__(LINES * LF::T, 1) k_fused_fwd(FusedArgs a) {
  Fused<LF, C, LINES>::forward(a);
}
template <class LF, int C, int LINES>
__global__ void __launch_bounds__(LINES * LF::T, 1) k_fused_adj(FusedArgs a) {
  Fused<LF, C, LINES>::adjoint(a);
}

// Host side of one fused configuration.
struct FusedOps {
  int m, C, lines, threads;
  size_t (*smem)(int n);
  // max co-resident clusters for n (0 = does not fit)
  int (*max_clusters)(int n);
  cudaError_t (*launch)(const FusedArgs&, bool adjoint, int n_clusters, cudaStream_t);
};

template <class LF, int C, int LINES>
struct FusedLaunch {
  using FS = Fused<LF, C, LINES>;
  static size_t smem(int n) { return FS::smem_bytes(n); }
  template <typename K>
  static cudaError_t prep(K k, size_t sm) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    if (C > 8) e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    return e;
  }
  static cudaLaunchConfig_t config(int n_clusters, size_t sm, cudaStream_t s, cudaLaunchAttribute* at) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(n_clusters * C);
    cfg.blockDim = dim3(FS::NT);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = s;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cfg;
  }
  static int max_clusters(int n) {
    const size_t sm = smem(n);
    if (sm > 227 * 1024) return 0;
    if (prep(k_fused_fwd<LF, C, LINES>, sm) != cudaSuccess) {
      (void)cudaGetLastError();
      return 0;
    }
    cudaLaunchAttribute at[1];
    cudaLaunchConfig_t cfg = config(1, sm, nullptr, at);
    int nc = 0;
    if (cudaOccupancyMaxActiveClusters(&nc, k_fused_fwd<LF, C, LINES>, &cfg) != cudaSuccess) {
      (void)cudaGetLastError();
      return 0;
    }
    return nc;
  }
  static cudaError_t launch(const FusedArgs& a, bool adjoint, int n_clusters, cudaStream_t s) {
    const size_t sm = smem(a.n);
    cudaLaunchAttribute at[1];
    cudaLaunchConfig_t cfg = config(n_clusters, sm, s, at);
    cudaError_t e;
    if (adjoint) {
      e = prep(k_fused_adj<LF, C, LINES>, sm);
      if (e == cudaSuccess) e = cudaLaunchKernelEx(&cfg, k_fused_adj<LF, C, LINES>, a);
    } else {
      e = prep(k_fused_fwd<LF, C, LINES>, sm);
      if (e == cudaSuccess) e = cudaLaunchKernelEx(&cfg, k_fused_fwd<LF, C, LINES>, a);
    }
    return e;
  }
  static const FusedOps* ops() {
    static const FusedOps o = {LF::M, C, LINES, FS::NT, &smem, &max_clusters, &launch};
    return &o;
  }
};

// fused configurations compiled for a padded size (fused_table.cu)
int fused_ops_for_m(int m, const FusedOps** out, int cap);

}  // namespace dos
