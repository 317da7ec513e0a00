// Host check of the register DFTs and the cooperative line DFT of
// csrc/dos_fft.cuh against a direct FP64 DFT (built and run by
// tests/test_line_dft_host.py; no GPU needed: the templates are
// __host__ __device__, and a block of T threads is emulated by running step 1
// for every thread, then step 2 for every thread, as the barrier between them
// orders it on the GPU).
//
// Inputs outside a pruning mask are set to NaN, so reading one shows up as a
// non-finite output; outputs outside the mask are not compared.
#include <cmath>
#include <complex>
#include <cstdio>
#include <random>
#include <vector>

#include "../paper_2604_02624_gb300/csrc/dos_fft.cuh"

using namespace dos;
using cd = std::complex<double>;

static int g_fail = 0, g_checks = 0;
static double g_worst = 0.0;

static void record(const char* what, double err, bool finite) {
  ++g_checks;
  if (err > g_worst) g_worst = err;
  if (!(err <= 2e-6) || !finite) {
    ++g_fail;
    std::printf("FAIL %s: relative error %.3e%s\n", what, err, finite ? "" : " (non-finite)");
  }
}

static cd w_turn(long e, long n, bool inv) {
  const double a = 2.0 * M_PI * (double)e / (double)n;
  return inv ? cd(std::cos(a), std::sin(a)) : cd(std::cos(a), -std::sin(a));
}

// one register DFT with the given pruning masks
template <int N, bool INV, ct::mask_t IM, ct::mask_t OM>
static void check_dftm(unsigned seed) {
  std::mt19937 rng(seed);
  std::normal_distribution<double> nd;
  float2 x[N];
  cd xd[N];
  for (int j = 0; j < N; ++j) {
    if (ct::has(IM, j)) {
      x[j] = make_float2((float)nd(rng), (float)nd(rng));
      xd[j] = cd(x[j].x, x[j].y);
    } else {
      x[j] = make_float2(NAN, NAN);
      xd[j] = 0.0;
    }
  }
  dftm<N, INV, IM, OM>(x);
  double num = 0.0, den = 0.0;
  bool finite = true;
  for (int k = 0; k < N; ++k) {
    if (!ct::has(OM, k)) continue;
    cd ref = 0.0;
    for (int j = 0; j < N; ++j) ref += xd[j] * w_turn((long)j * k, N, INV);
    const cd got(x[k].x, x[k].y);
    finite = finite && std::isfinite(got.real()) && std::isfinite(got.imag());
    num += std::norm(got - ref);
    den += std::norm(ref);
  }
  char what[128];
  std::snprintf(what, sizeof what, "dft N=%d inv=%d im=%llx om=%llx", N, (int)INV, IM, OM);
  record(what, den > 0 ? std::sqrt(num / den) : std::sqrt(num), finite);
}

template <int N>
static void check_sizes() {
  constexpr ct::mask_t F = ct::lead_mask(N), H = ct::lead_mask(N / 2), L = ct::lead_mask((N + 1) / 2);
  // a scattered mask: every third element and the last
  constexpr ct::mask_t S = []() {
    ct::mask_t m = 0;
    for (int i = 0; i < N; i += 3) m |= 1ull << i;
    return m | (1ull << (N - 1));
  }();
  check_dftm<N, false, F, F>(N);
  check_dftm<N, true, F, F>(N + 1);
  check_dftm<N, false, H | 1ull, F>(N + 2);
  check_dftm<N, true, F, H | 1ull>(N + 3);
  check_dftm<N, false, L, H | 1ull>(N + 4);
  check_dftm<N, true, S, S>(N + 5);
  check_dftm<N, false, F & ~S, S>(N + 6);
  check_dftm<N, true, 1ull, F>(N + 7);
}

// the cooperative M = P Q point line DFT of T threads (Line<P, Q, T>)
template <int P, int Q, int T, bool INV, int NZP, int NOQ, bool TR, int ZR = -1>
static void check_line(unsigned seed) {
  using LF = Line<P, Q, T>;
  constexpr int M = P * Q, E = M / T;
  constexpr int ZP = ZR < 0 ? LF::RP : ZR;  // exchange pitch
  std::vector<float2> tw(LF::TWS), z((size_t)(P > Q ? P : Q) * ZP, make_float2(NAN, NAN));
  for (int q = 0; q < Q; ++q)
    for (int k1 = 0; k1 < P; ++k1) {
      const cd w = w_turn((long)q * k1, M, false);
      tw[q * LF::TWP + k1] = make_float2((float)w.real(), (float)w.imag());
    }
  std::mt19937 rng(seed);
  std::normal_distribution<double> nd;
  // first-step sub-DFT q reads x[q + Q p] for p < NZP: inputs n < Q NZP may be non-zero
  std::vector<cd> xd(M, 0.0);
  std::vector<std::vector<float2>> r(T, std::vector<float2>(E));
  for (int t = 0; t < T; ++t)
    for (int i = 0; i < E; ++i) {
      const int n = t + T * i;
      if (n < Q * NZP) {
        r[t][i] = make_float2((float)nd(rng), (float)nd(rng));
        xd[n] = cd(r[t][i].x, r[t][i].y);
      } else {
        r[t][i] = make_float2(NAN, NAN);
      }
    }
  for (int t = 0; t < T; ++t) {
    float2(&rt)[E] = *reinterpret_cast<float2(*)[E]>(r[t].data());
    LF::template step1<INV, NZP, false, TR, ZP>(rt, t, z.data(), tw.data());
  }
  for (int t = 0; t < T; ++t) {
    float2(&rt)[E] = *reinterpret_cast<float2(*)[E]>(r[t].data());
    LF::template step2<INV, NOQ, false, TR, ZP>(rt, t, z.data());
  }
  // outputs k = k1 + P k2 with k2 < NOQ, i.e. k < P NOQ, are produced
  double num = 0.0, den = 0.0;
  bool finite = true;
  for (int t = 0; t < T; ++t)
    for (int i = 0; i < E; ++i) {
      const int k = t + T * i;
      if (k >= P * NOQ) continue;
      cd ref = 0.0;
      for (int n = 0; n < Q * NZP; ++n) ref += xd[n] * w_turn((long)n * k, M, INV);
      const cd got(r[t][i].x, r[t][i].y);
      finite = finite && std::isfinite(got.real()) && std::isfinite(got.imag());
      num += std::norm(got - ref);
      den += std::norm(ref);
    }
  char what[128];
  std::snprintf(what, sizeof what, "line %dx%d T=%d inv=%d nzp=%d noq=%d tr=%d pitch=%d", P, Q, T, (int)INV, NZP,
                NOQ, (int)TR, ZP);
  record(what, std::sqrt(num / den), finite);
}

// every use the passes make of a line shape: forward DFT of a full or a
// half-zero field, inverse DFT to a full or a cropped field, both layouts of
// the exchange on square lines, with the odd pitch and with the even one
// (paired 16-byte accesses)
template <int P, int Q, int T>
static void check_shape() {
  constexpr bool SQ = Line<P, Q, T>::SQUARE;
  constexpr int ZE = P + (P & 1);  // the bulk column pass's even exchange pitch
  check_line<P, Q, T, false, P, Q, false>(P * 100 + 1);
  check_line<P, Q, T, false, P / 2, Q, false>(P * 100 + 2);
  check_line<P, Q, T, true, P, Q, false>(P * 100 + 3);
  check_line<P, Q, T, true, P, Q / 2, false>(P * 100 + 4);
  check_line<P, Q, T, false, P / 2, Q, false, ZE>(P * 100 + 7);
  check_line<P, Q, T, true, P, Q / 2, false, ZE>(P * 100 + 8);
  if constexpr (SQ) {
    check_line<P, Q, T, false, P / 2, Q, true>(P * 100 + 5);
    check_line<P, Q, T, true, P, Q / 2, true>(P * 100 + 6);
    check_line<P, Q, T, false, P / 2, Q, true, ZE>(P * 100 + 9);
    check_line<P, Q, T, true, P, Q / 2, true, ZE>(P * 100 + 10);
  }
}

int main() {
  check_sizes<2>();
  check_sizes<3>();
  check_sizes<4>();
  check_sizes<5>();
  check_sizes<6>();
  check_sizes<8>();
  check_sizes<10>();
  check_sizes<12>();
  check_sizes<15>();
  check_sizes<16>();
  check_sizes<20>();
  check_sizes<25>();
  check_sizes<32>();
  check_shape<4, 4, 4>();
  check_shape<4, 8, 4>();
  check_shape<8, 8, 8>();
  check_shape<8, 16, 8>();
  check_shape<10, 20, 10>();
  check_shape<16, 16, 16>();
  check_shape<20, 20, 20>();
  check_shape<16, 32, 16>();
  std::printf("%s: %d checks, %d failed, worst relative error %.3e\n", g_fail ? "FAIL" : "OK", g_checks, g_fail,
              g_worst);
  return g_fail ? 1 : 0;
}
