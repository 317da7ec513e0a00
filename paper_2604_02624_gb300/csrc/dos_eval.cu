// dos_eval.cu - evaluation variants of a design on the forward path.
//
//  * phase bit depth B (Fig. 7): the learnable thickness, limited to
//    [0, h_max], takes one of 2^B evenly spaced levels;
//  * output diffraction efficiency (Figs. 5-6): power on the output FOV over
//    the power of the unit-amplitude input aperture.
#include "../../include/dos.h"
#include "dos_internal.h"

namespace dos {

__global__ void k_quantize(const float* __restrict__ h, float* __restrict__ q, size_t count, float hmax, float s,
                           float step) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const float hc = fminf(fmaxf(h[i], 0.0f), hmax);
  const float k = rintf(__fmul_rn(hc, s));
  q[i] = __fmul_rn(k, step);
}

cudaError_t launch_quantize(const float* h, float* q, size_t count, double h_max, int bits, cudaStream_t st) {
  const double levels = (double)((1u << bits) - 1u);
  k_quantize<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(h, q, count, (float)h_max, (float)(levels / h_max),
                                                              (float)(h_max / levels));
  return cudaGetLastError();
}

// eta_w = sum over the FOV of |o|^2 / aperture^2 (FP64 sums, fixed order)
__global__ void __launch_bounds__(256) k_efficiency(const float2* __restrict__ o, float* __restrict__ eta, int fov2,
                                                    double inv_power) {
  __shared__ double sh[256];
  const int w = blockIdx.x;
  const float2* ow = o + (size_t)w * fov2;
  double acc = 0.0;
  for (int p = threadIdx.x; p < fov2; p += 256) acc += (double)fmaf(ow[p].x, ow[p].x, ow[p].y * ow[p].y);
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) eta[w] = (float)(sh[0] * inv_power);
}

cudaError_t launch_efficiency(const float2* o, float* eta, int nw, int fov2, int aperture, cudaStream_t s) {
  k_efficiency<<<nw, 256, 0, s>>>(o, eta, fov2, 1.0 / ((double)aperture * aperture));
  return cudaGetLastError();
}

}  // namespace dos
