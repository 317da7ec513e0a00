// dos_loss.cu - objective, quality metric and the gradient reduction.
//
// Section 2: the design minimises an MSE between the output intensity O_w of
// every channel and its target; reconstruction quality is a PSNR.  The
// detector (Section 4: the FOV divided into output pixels) reads pixel (y, x)
// as the sum of the b x b simulation intensities it covers (b = 1: I itself).
// Per-pixel arithmetic and each thread's strided partial sums run in FP32 (a
// thread sums at most a few hundred terms), the block tree and everything
// after it in FP64 (GB300's FP64 rate is a small fraction of its FP32 rate);
// every sum has a fixed order, so results are reproducible bit for bit.
#include "dos_internal.h"

#include "../../include/dos.h"

namespace dos {

constexpr int kRedThreads = 256;

__device__ __forceinline__ double block_sum(double v, double* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int s = kRedThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}

__device__ __forceinline__ float intensity(float2 o) { return fmaf(o.x, o.x, o.y * o.y); }

// detector pixel p = (y, x) of a channel's F x F output field: sum over its b x b block
__device__ __forceinline__ float detector(const float2* ow, int fov, int b, int p) {
  if (b == 1) return intensity(ow[p]);
  const int fd = fov / b, y = (p / fd) * b, x = (p % fd) * b;
  float s = 0.f;
  for (int i = 0; i < b; ++i)
    for (int j = 0; j < b; ++j) s += intensity(ow[(size_t)(y + i) * fov + x + j]);
  return s;
}

// per channel: sum (D-T)^2, sigma = sum D T / sum D^2, sum (sigma D - T)^2,
// and (dLdI not null) dL/dI of the channel's simulation pixels: dL/dD of the
// detector pixel covering it, 2 (D - T) / norm, or 2 sigma (sigma D - T) / norm
// for the scaled loss (scale = 2 / norm)
__global__ void __launch_bounds__(kRedThreads) k_loss_stats(const float2* __restrict__ o,
                                                            const float* __restrict__ T,
                                                            LossStats* __restrict__ st, int fov, int b,
                                                            float* __restrict__ dLdI, float scale, int mode) {
  __shared__ double sh[kRedThreads];
  const int w = blockIdx.x;
  const int fd = fov / b, det2 = fd * fd;
  const float2* ow = o + (size_t)w * fov * fov;
  const float* tw = T + (size_t)w * det2;
  float fse = 0.f, fit = 0.f, fii = 0.f;
  for (int p = threadIdx.x; p < det2; p += kRedThreads) {
    const float I = detector(ow, fov, b, p);
    const float t = tw[p];
    const float d = I - t;
    fse = fmaf(d, d, fse);
    fit = fmaf(I, t, fit);
    fii = fmaf(I, I, fii);
  }
  const double sse = block_sum(fse, sh);
  const double sit = block_sum(fit, sh);
  const double sii = block_sum(fii, sh);
  const double sigma = sii > 0.0 ? sit / sii : 0.0;
  const float sg = (float)sigma;
  float fsc = 0.f;
  for (int p = threadIdx.x; p < det2; p += kRedThreads) {
    const float d = fmaf(sg, detector(ow, fov, b, p), -tw[p]);
    fsc = fmaf(d, d, fsc);
  }
  const double ssc = block_sum(fsc, sh);
  if (threadIdx.x == 0) {
    LossStats s;
    s.sse = sse;
    s.sigma = sigma;
    s.sse_sc = ssc;
    s.pad = 0;
    st[w] = s;
  }
  if (dLdI) {
    const int fov2 = fov * fov;
    float* gw = dLdI + (size_t)w * fov2;
    for (int q = threadIdx.x; q < fov2; q += kRedThreads) {
      const int p = ((q / fov) / b) * fd + (q % fov) / b;  // detector pixel covering q
      const float I = detector(ow, fov, b, p);
      const float t = tw[p];
      gw[q] = mode == DOS_LOSS_MSE_SCALED ? scale * sg * fmaf(sg, I, -t) : scale * (I - t);
    }
  }
}

cudaError_t launch_loss_stats(const float2* o, const float* T, LossStats* st, int nw, int fov, int bin,
                              float* dLdI, double norm, int mode, cudaStream_t s) {
  const float scale = (float)(2.0 / norm);  // dL/dD = 2 (D - T) / norm
  k_loss_stats<<<nw, kRedThreads, 0, s>>>(o, T, st, fov, bin, dLdI, scale, mode);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(kRedThreads) k_loss_final(const LossStats* __restrict__ st, int nw,
                                                            int fov2, double norm, int mode,
                                                            double* __restrict__ d_loss,
                                                            float* __restrict__ psnr) {
  __shared__ double sh[kRedThreads];
  double acc = 0;
  for (int w = threadIdx.x; w < nw; w += kRedThreads) {
    const LossStats s = st[w];
    acc += mode == DOS_LOSS_MSE_SCALED ? s.sse_sc : s.sse;
    if (psnr) psnr[w] = (float)(10.0 * log10((double)fov2 / s.sse_sc));
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) *d_loss = acc / norm;
}

cudaError_t launch_loss_final(const LossStats* st, int nw, int fov2, double norm, int mode,
                              double* d_loss, float* d_psnr, cudaStream_t s) {
  k_loss_final<<<1, kRedThreads, 0, s>>>(st, nw, fov2, norm, mode, d_loss, d_psnr);
  return cudaGetLastError();
}

// grad[g] = sum over chunks c (in order) of partial[layer(g)][c][pixel(g)]
__global__ void k_grad_reduce(const float* __restrict__ partial, float* __restrict__ grad,
                              int n_chunks, size_t count, size_t n2) {
  const size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= count) return;
  const size_t layer = g / n2, px = g % n2;
  const float* p = partial + layer * n_chunks * n2 + px;
  double acc = 0.0;
  for (int c = 0; c < n_chunks; ++c) acc += (double)p[(size_t)c * n2];
  grad[g] = (float)acc;
}

cudaError_t launch_grad_reduce(const float* partial, float* grad, int n_chunks, size_t count,
                               size_t n2, cudaStream_t s) {
  k_grad_reduce<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(partial, grad, n_chunks, count, n2);
  return cudaGetLastError();
}

}  // namespace dos

namespace dos {
// grad[g] = sum over c < n_parts (in order) of partial[c * count + g]
__global__ void k_grad_reduce_flat(const float* __restrict__ partial, float* __restrict__ grad,
                                   int n_parts, size_t count) {
  const size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= count) return;
  double acc = 0.0;
  for (int c = 0; c < n_parts; ++c) acc += (double)partial[(size_t)c * count + g];
  grad[g] = (float)acc;
}

cudaError_t launch_grad_reduce_flat(const float* partial, float* grad, int n_parts, size_t count,
                                    cudaStream_t s) {
  k_grad_reduce_flat<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(partial, grad, n_parts, count);
  return cudaGetLastError();
}
}  // namespace dos
