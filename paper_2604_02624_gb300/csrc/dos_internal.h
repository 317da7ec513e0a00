// dos_internal.h - declarations shared by the CUDA translation units of libdos.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>

namespace dos {

// Per-channel constants of Eq. 1 (one wavelength), built on the device at create.
struct ChanConst {
  float a_hi, a_lo;   // (n - n_medium) / lambda as a float pair [cycles per metre]
  float pc_base;      // phase of the base thickness, frac((n - n_medium) h_base / lambda) [cycles]
  float amp_k;        // -2 pi kappa / (lambda ln 2): amplitude = exp2(amp_k * h) * amp_base
  float amp_base;     // exp(-2 pi kappa h_base / lambda)
  float c_re, c_im;   // c = dt/dh / t = -2 pi (kappa + j (n - n_medium)) / lambda
  float pad;
};

// Misaligned layers (Section 3, "vaccination"): gap g carries the lateral
// shift (ax, ay) and the length change dz; the transfer function becomes
// H * exp(-2 pi j (fx ax + fy ay)) * H(dz), with H(dz) from the signed
// root table sq = +sqrt(q) (propagating) or -sqrt(-q) (evanescent).
struct Misalign {
  const float* sq;   // [nw][hs][hs] signed sqrt(|q|) [1/m], or null when off
  float df;          // DFT bin spacing 1 / (M pitch) [1/m]
  float ax, ay, dz;  // this gap [m]
};

// exp(-2 pi j (fx ax + fy ay)) * H(dz) for bins (ky, kx) of an M-point grid
__device__ __forceinline__ float2 misalign_factor(const Misalign& g, int ky, int kx, int m, float sq) {
  const float fx = (float)(kx < m / 2 ? kx : kx - m) * g.df;
  const float fy = (float)(ky < m / 2 ? ky : ky - m) * g.df;
  float ph = -fmaf(fx, g.ax, fy * g.ay);  // cycles
  float amp = 1.0f;
  if (sq >= 0.0f) ph = fmaf(g.dz, sq, ph);
  else amp = expf(6.283185307179586f * g.dz * sq);
  float sn, cs;
  sincospif(2.0f * ph, &sn, &cs);
  return make_float2(amp * cs, amp * sn);
}

// Arguments of one propagation pass (all channels of the context).
struct PassArgs {
  float2* S;              // [nw][n][m] spectra of the rows (row pass output / column pass in-out)
  const float2* Hq;       // [nw][hs][hs] transfer function of this gap, 1/M^2 folded in
  const float2* arow;     // [m] DFT of one aperture row (lambda independent)
  const float2* tw;       // [Q*RP] line twiddles exp(-2 pi j q k1 / M)
  const ChanConst* chan;  // [nw]
  const float* h;         // [n][n] thickness of this layer
  float2* ckpt;           // [nw][n][n] incoming field of this layer (checkpoint)
  float2* o;              // [nw][fov][fov] complex output field
  float* I;               // [nw][fov][fov] intensity (may be null)
  const float* dLdI;      // [nw][fov][fov]
  float* partial;         // [n_chunks][n][n] gradient partials of this layer
  const float2* fin;      // [nw][n][n] caller field (propagate entry)
  float2* fout;           // [nw][n][n] caller field (propagate entry)
  int n, m, nw, fov, of, hs;
  int in_r0, in_r1;       // column pass: rows that may be non-zero on input
  int out_r0, out_r1;     // column pass: rows stored on output
  int chunk;              // channels per block of the adjoint row pass
  int n_chunks;
  Misalign mis;           // misaligned layers (mis.sq null: none)
  int* err;               // set to 1 by a bulk-copy pass whose bounded wait expired
  int stall;              // fault injection (tests): 1 = the bulk pass expects bytes that are never
                          // copied; 2 = its copies land but odd threads give up their first wait;
                          // 3 = (column pass) the H tile of each block's last item lands but every
                          // thread gives up its wait for it
  const void* tmap;       // host CUtensorMap of S as [nw][n][m] 8-byte elements (bulk column pass), or null
  int tmap_rows;          // rows of its box: the bulk column pass uses it when they are in_r1 - in_r0
  const void* hmap;       // host CUtensorMap of the transfer tables as [slots * nw][hs][hs] 8-byte elements
  int hmap_z0;            // its channel coordinate of this gap's table slot and channel range: slot * nw + w0
  int tmap_w0;            // channel coordinate of channel 0 of this range in the spectra maps
};

// Kernel launchers of one padded size M (one translation unit per M).
struct PassOps {
  int m, P, Q, T;
  int row_lines, col_lines;
  cudaError_t (*col)(const PassArgs&, bool adjoint, bool aperture, cudaStream_t);
  cudaError_t (*row_fwd)(const PassArgs&, bool save, cudaStream_t);
  cudaError_t (*row_out)(const PassArgs&, cudaStream_t);
  cudaError_t (*row_seed)(const PassArgs&, cudaStream_t);
  cudaError_t (*row_adj)(const PassArgs&, bool first, cudaStream_t);
  cudaError_t (*row_in)(const PassArgs&, cudaStream_t);    // caller field -> row spectra
  cudaError_t (*row_back)(const PassArgs&, cudaStream_t);  // row spectra -> caller field
  cudaError_t (*row_first)(const PassArgs&, cudaStream_t); // t(h) * field (fin) -> row spectra
  // the same column / forward row / adjoint row passes with bulk-async prefetch
  // (dos_pass_bulk.cuh)
  cudaError_t (*bulk_col)(const PassArgs&, bool adjoint, cudaStream_t);
  cudaError_t (*bulk_row_fwd)(const PassArgs&, bool save, cudaStream_t);
  cudaError_t (*bulk_row_adj)(const PassArgs&, bool first, cudaStream_t);
  cudaError_t (*bulk_row_first)(const PassArgs&, cudaStream_t);  // t(h) * field (fin) -> row spectra
  // boxes of the bulk column pass's tensor copies: spectra {col_group, rows, 1},
  // transfer table {h_box_cols, h_box_rows, 1} (h_box_cols 0: no staged H tile)
  int col_group, h_box_cols, h_box_rows;
};

const PassOps* pass_ops_for_m(int m);

// Message returned by dos_last_error() for the calling thread.
void set_last_error(const char* msg);
int supported_m_list(int* out, int cap);

// Setup kernels (dos_setup.cu).
cudaError_t launch_htable(float2* Hq, const double* d_lambda, int nw, double z, double n_medium,
                          double pitch, int m, int hs, int evanescent, cudaStream_t s);
cudaError_t launch_arow(float2* arow, int m, int offset, int width, cudaStream_t s);
cudaError_t launch_sqtable(float* sq, const double* d_lambda, int nw, double n_medium, double pitch, int m, int hs,
                           cudaStream_t s);
cudaError_t launch_twiddles(float2* tw, int P, int Q, int TWP, int m, cudaStream_t s);
cudaError_t launch_chan(ChanConst* chan, const double* d_lambda, const double* d_nidx,
                        const double* d_kappa, int nw, double n_medium, double h_base,
                        cudaStream_t s);

// Objective kernels (dos_loss.cu).
struct LossStats {
  double sse;      // sum_p (I - T)^2
  double sigma;    // sum I T / sum I^2
  double sse_sc;   // sum_p (sigma I - T)^2
  double pad;
};
// o: [nw][fov][fov] output field; T: [nw][fov/bin][fov/bin] targets of the
// detector pixels (bin x bin simulation pixels each); dLdI: [nw][fov][fov] or
// null (then not written); norm: the loss's divisor; mode: DOS_LOSS_*
cudaError_t launch_loss_stats(const float2* o, const float* T, LossStats* st, int nw, int fov, int bin,
                              float* dLdI, double norm, int mode, cudaStream_t s);
// det2: detector pixels per channel (PSNR mean)
cudaError_t launch_loss_final(const LossStats* st, int nw, int det2, double norm, int mode,
                              double* d_loss, float* d_psnr, cudaStream_t s);
cudaError_t launch_grad_reduce(const float* partial, float* grad, int n_chunks, size_t count,
                               size_t chunk_stride, cudaStream_t s);
cudaError_t launch_grad_reduce_flat(const float* partial, float* grad, int n_parts, size_t count,
                                    cudaStream_t s);

// Evaluation variants (dos_eval.cu).
cudaError_t launch_quantize(const float* h, float* q, size_t count, double h_max, int bits, cudaStream_t s);
cudaError_t launch_efficiency(const float2* o, float* eta, int nw, int fov2, int aperture, cudaStream_t s);

}  // namespace dos
