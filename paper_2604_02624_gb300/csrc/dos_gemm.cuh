// dos_gemm.cuh - split-BF16 DFT-as-GEMM propagation on the tcgen05 tensor cores.
//
// The 2D DFTs of the angular-spectrum step (Eq. 4-5) are dense complex matrix
// products with two constant matrices shared by every channel:
//   F[k][x] = exp(-2 pi j k x / M)   (M x N: DFT of N non-zero inputs)
//   G[x][k] = exp(+2 pi j x k / M)   (N x M: inverse DFT keeping N outputs)
// One propagation of a field U (N x N) is
//   A = F U^T-rows  (row DFT),  B = F A (column DFT),  B *= H,
//   C = G B (column IDFT),      V = C G^T-rows (row IDFT),
// each written as Y = W X with the data matrix X stacked over channels.  The
// GEMM epilogues write the next product's operand directly (no FP32 output
// round trip): the row DFT and the column IDFT as D = W X^T, whose accumulator
// rows (one output frequency or position, re or im) map to contiguous runs of
// the next operand's rows; the column DFT (with the multiply by H) and the row
// IDFT as D = X W^T, whose accumulator rows are one data row each.
//
// Precision: every operand is split into bf16 parts, x = x0 + x1 (+ x2), each
// the bf16 rounding of what the earlier parts leave.  Two parts carry ~2^-17
// relative and a product keeps three terms, W0 X0 + W0 X1 + W1 X0; three parts
// carry ~2^-26 and a product keeps six, adding W0 X2 + W2 X0 + W1 X1 (the
// dropped terms are below 2^-26).  Terms accumulate in FP32 in tensor memory.  In real form a complex W (m x k) is a 2m x 2k
// matrix whose row 2o is [Re W_o, -Im W_o] and row 2o+1 is [Im W_o, Re W_o];
// the data column is [Re x; Im x], so lanes 2o / 2o+1 of the accumulator hold
// the real / imaginary part of output o.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "dos_internal.h"

namespace dos {

// Element (row, k) of an operand with kp (a multiple of 64) columns of K in
// the tiled order the GEMM reads: tiles of 256 rows x 64 K, 32 KB each,
// row-tile major; inside a tile the tensor core's K-major core-matrix order
// (8 rows x 8 K = 128 bytes per core matrix, 8 core matrices along K, then
// the next 8 rows).
__host__ __device__ inline size_t gemm_tiled(size_t row, int k, int kp) {
  return ((((row >> 8) * (size_t)(kp >> 6)) + (size_t)(k >> 6)) << 14) +
         ((size_t)((((int)(row & 255) >> 3) << 3) + ((k & 63) >> 3)) << 6) + ((row & 7) << 3) + (size_t)(k & 7);
}

// One GEMM D[rows][cols] (f32, row-major, leading dimension ldd) =
//   sum over segments s of A_s[rows][K] * B_s[cols][K]^T, A_s / B_s bf16 in
//   the tiled order above.  rows % 256 == 0, K % 64 == 0; cols may be ragged
//   (B must then hold whole 256-row tiles; rows past cols are never stored).
constexpr int kMaxGemmTerms = 6;

// The bf16 parts of one operand (parts 1 or 2 unused when there are fewer).
struct Parts {
  __nv_bfloat16* p[3];
  int k;  // 2 or 3
};

// What the epilogue does with the accumulator D (rows x cols):
enum {
  GEMM_OUT_ROWS = 0,      // D = W X^T, row 2k+p = part p (re, im) of output k; column c = (w, j):
                          //   next operand row (w, k), K index p * nj + j
  GEMM_OUT_SPECTRUM = 1,  // D = X W^T, row (w, kx), columns 2ky+p: times H_w(ky, kx) (conj H for the
                          //   adjoint, with the misalignment factor): next operand row (w, kx), K ky / m + ky
  GEMM_OUT_FIELD = 2      // D = X W^T, row (w, y), columns 2x+p: field[w][y][x], or o / I on the FOV
};

struct GemmArgs {
  const __nv_bfloat16* a[kMaxGemmTerms];
  const __nv_bfloat16* b[kMaxGemmTerms];
  int nseg;
  int rows, cols, K;  // tiles of the A operand (rows) and B operand (cols), 256 each
  int w_is_b;         // the DFT matrix is the B operand (raster: its tiles fastest)
  int* err;           // set to 1 when a bounded wait gave up
  int mode;           // GEMM_OUT_*
  int vrows, vcols;   // D rows / columns that hold results
  int nk, nj;         // ROWS: outputs and inputs per channel
  Parts xo;           // ROWS / SPECTRUM: the next operand
  int kpo;            // its K pitch
  const float2* Hq;   // SPECTRUM: [nwc][hs][hs] transfer tables of the chunk
  int hs, m, adj;
  Misalign mis;       // SPECTRUM: misalignment (sq offset to the chunk), or sq null
  float2* fld;        // FIELD: [nwc][n][n]
  float2* o;          // FIELD: FOV output [nwc][fov][fov] (then fld unused)
  float* I;           //        and its intensity (may be null)
  int n, of, fov;
};

cudaError_t launch_tc_gemm(const GemmArgs& g, cudaStream_t s);

// Context-level buffers and constants of the DFT-GEMM path.
struct GemmPlan {
  int n, m, nwc;            // layer side, padded size, channels per chunk
  int kp1, kp2;             // padded K of the N- and M-point products (multiples of 64)
  int rp1, rp2;             // padded rows of F (2M) and G (2N) (multiples of 256)
  int parts;                // bf16 parts per operand: 2 (three products) or 3 (six)
  Parts F;                  // [rp1][kp1] each
  Parts G;                  // [rp2][kp2] each
  Parts X;                  // data operand (product input), whole 256-row tiles
  Parts Y;                  // the other data operand buffer (products alternate X -> Y -> X -> Y)
  float2* fld;              // FP32 working field [nwc][n][n]
  int* err;
};

cudaError_t launch_build_dft(GemmPlan& p, cudaStream_t s);

// One propagation (forward H or conj H) of the chunk's field held in X rows
// (w, y); the result goes to p.fld, or to o / I on the FOV when o is given.
// Adds the number of kernels it launched to *launches.
cudaError_t gemm_propagate(GemmPlan& p, int nwc, const float2* Hq, int hs, bool adj, float2* o, float* I, int of,
                           int fov, const Misalign& mis, int* launches, cudaStream_t s);
// field -> X rows: mode 0 copy, mode 1 checkpoint + Eq. 1 modulation, mode 2 aperture.
cudaError_t gemm_prep_field(GemmPlan& p, int nwc, const float2* v, float2* ckpt, const float* h,
                            const ChanConst* chan, int mode, int a_off, int a_w, cudaStream_t s);
// p.fld = 2 dL/dI o on the FOV, zero elsewhere
cudaError_t gemm_seed(GemmPlan& p, int nwc, const float2* o, const float* dLdI, int of, int fov, cudaStream_t s);
// gradient partial of one layer over the chunk, p.fld <- conj(t) p.fld
cudaError_t gemm_adj_layer(GemmPlan& p, int nwc, const float2* ckpt, size_t ckpt_stride, const float* h,
                           const ChanConst* chan, float* partial, cudaStream_t s);

}  // namespace dos
