// dos_setup.cu - tables built once per context (dos_create), all on the device.
//
//  * H_z for every (distinct gap, wavelength): the angular-spectrum transfer
//    function of the Rayleigh-Sommerfeld impulse response (Eq. 4),
//    exp(j 2 pi z sqrt((n/lambda)^2 - fx^2 - fy^2)).  With gaps of hundreds of
//    wavelengths the phase is hundreds of cycles, so it is formed and reduced
//    modulo one cycle in FP64; only the reduced value is rounded to FP32.
//    H depends on fx^2 and fy^2 only, so one quadrant (M/2+1)^2 per table
//    covers the whole M x M grid.  The 1/M^2 of the inverse DFT is folded in.
//  * the DFT of one row of the square input aperture (lambda independent);
//  * the line-FFT twiddles exp(-2 pi j q k / M);
//  * per-channel constants of the transmission of Eq. 1-2.
#include "dos_internal.h"

#include "../../include/dos.h"

namespace dos {

__global__ void k_htable(float2* __restrict__ Hq, const double* __restrict__ lam, double z,
                         double n_medium, double pitch, int m, int hs, int evanescent) {
  const int w = blockIdx.y;
  const int a = blockIdx.x;
  const double df = 1.0 / ((double)m * pitch);  // frequency spacing of the DFT bins
  const double k = n_medium / lam[w];
  const double k2 = k * k;
  const double scale = 1.0 / ((double)m * (double)m);
  const double fa = a * df;
  for (int b = threadIdx.x; b < hs; b += blockDim.x) {
    const double fb = b * df;
    // fx^2 + fy^2 first: the table is exactly symmetric, H(a, b) = H(b, a)
    // (the bulk column pass reads a quadrant column as a table row)
    const double q = k2 - (fa * fa + fb * fb);
    float2 h;
    if (q >= 0.0) {
      const double cyc = z * sqrt(q);
      const double fr = cyc - rint(cyc);
      double s, c;
      sincospi(2.0 * fr, &s, &c);
      h = make_float2((float)(c * scale), (float)(s * scale));
    } else if (evanescent == DOS_EVAN_DECAY) {
      const double d = 2.0 * 3.14159265358979323846 * z * sqrt(-q);
      h = make_float2((float)(exp(-d) * scale), 0.f);
    } else {
      h = make_float2(0.f, 0.f);
    }
    Hq[((size_t)w * hs + a) * hs + b] = h;
  }
}

cudaError_t launch_htable(float2* Hq, const double* d_lambda, int nw, double z, double n_medium,
                          double pitch, int m, int hs, int evanescent, cudaStream_t s) {
  k_htable<<<dim3(hs, nw), 256, 0, s>>>(Hq, d_lambda, z, n_medium, pitch, m, hs, evanescent);
  return cudaGetLastError();
}

// signed root of q = (n/lambda)^2 - fx^2 - fy^2 on the quadrant (FP64, rounded once)
__global__ void k_sqtable(float* __restrict__ sq, const double* __restrict__ lam, double n_medium, double pitch, int m,
                          int hs) {
  const int w = blockIdx.y;
  const int a = blockIdx.x;
  const double df = 1.0 / ((double)m * pitch);
  const double k = n_medium / lam[w];
  const double fa = a * df;
  for (int b = threadIdx.x; b < hs; b += blockDim.x) {
    const double fb = b * df;
    const double q = k * k - fa * fa - fb * fb;
    sq[((size_t)w * hs + a) * hs + b] = (float)(q >= 0.0 ? sqrt(q) : -sqrt(-q));
  }
}

cudaError_t launch_sqtable(float* sq, const double* d_lambda, int nw, double n_medium, double pitch, int m, int hs,
                           cudaStream_t s) {
  k_sqtable<<<dim3(hs, nw), 256, 0, s>>>(sq, d_lambda, n_medium, pitch, m, hs);
  return cudaGetLastError();
}

// Arow[k] = sum_{x = offset}^{offset + width - 1} exp(-2 pi j k x / m)
__global__ void k_arow(float2* __restrict__ arow, int m, int offset, int width) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= m) return;
  double re = 0.0, im = 0.0;
  for (int x = offset; x < offset + width; ++x) {
    const long e = ((long)k * x) % m;
    double s, c;
    sincospi(-2.0 * (double)e / (double)m, &s, &c);
    re += c;
    im += s;
  }
  arow[k] = make_float2((float)re, (float)im);
}

cudaError_t launch_arow(float2* arow, int m, int offset, int width, cudaStream_t s) {
  k_arow<<<(m + 127) / 128, 128, 0, s>>>(arow, m, offset, width);
  return cudaGetLastError();
}

// tw[q*RP + k] = exp(-2 pi j q k / m) for q < Q, k < P; padding entries zero.
__global__ void k_twiddles(float2* __restrict__ tw, int P, int Q, int TWP, int m) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Q * TWP) return;
  const int q = i / TWP, k = i % TWP;
  float2 v = make_float2(0.f, 0.f);
  if (k < P) {
    const long e = ((long)q * k) % m;
    double s, c;
    sincospi(-2.0 * (double)e / (double)m, &s, &c);
    v = make_float2((float)c, (float)s);
  }
  tw[i] = v;
}

cudaError_t launch_twiddles(float2* tw, int P, int Q, int TWP, int m, cudaStream_t s) {
  const int n = Q * TWP;
  k_twiddles<<<(n + 127) / 128, 128, 0, s>>>(tw, P, Q, TWP, m);
  return cudaGetLastError();
}

__global__ void k_chan(ChanConst* __restrict__ chan, const double* __restrict__ lam,
                       const double* __restrict__ nidx, const double* __restrict__ kap, int nw,
                       double n_medium, double h_base) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= nw) return;
  const double pi = 3.14159265358979323846;
  const double l = lam[w];
  const double kappa = kap ? kap[w] : 0.0;
  const double a = (nidx[w] - n_medium) / l;  // phase cycles per metre of thickness
  ChanConst c;
  c.a_hi = (float)a;
  c.a_lo = (float)(a - (double)c.a_hi);
  const double pb = a * h_base;
  c.pc_base = (float)(pb - rint(pb));
  c.amp_k = (float)(-2.0 * pi * kappa / (l * 0.69314718055994530942));
  c.amp_base = (float)exp(-2.0 * pi * kappa * h_base / l);
  c.c_re = (float)(-2.0 * pi * kappa / l);
  c.c_im = (float)(-2.0 * pi * (nidx[w] - n_medium) / l);
  c.pad = 0.f;
  chan[w] = c;
}

cudaError_t launch_chan(ChanConst* chan, const double* d_lambda, const double* d_nidx,
                        const double* d_kappa, int nw, double n_medium, double h_base,
                        cudaStream_t s) {
  k_chan<<<(nw + 127) / 128, 128, 0, s>>>(chan, d_lambda, d_nidx, d_kappa, nw, n_medium, h_base);
  return cudaGetLastError();
}

}  // namespace dos
