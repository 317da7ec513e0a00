// dos_fft.cuh - FP32 complex DFTs for the angular-spectrum passes (sm_103a).
//
// Two levels:
//  * dft<N, INV, NZ, NO>(x): an N-point DFT held entirely in one thread's
//    registers, natural order in and out, built at compile time from radix
//    2/3/4/5 butterflies.  Composite sizes split by Good-Thomas (prime factor
//    algorithm: coprime factors, index maps by the Chinese remainder theorem,
//    no twiddles between the stages) or by Cooley-Tukey, whichever a
//    compile-time operation count finds cheaper (20 = 4 x 5 goes Good-Thomas).
//    Twiddles are compile-time constants (cos/sin of rational turns evaluated
//    by a constexpr series), so they become instruction immediates. NZ
//    leading inputs may be non-zero, NO leading outputs are needed:
//    zero-padding and cropping prune work, tracked as bit masks through the
//    splits.
//  * Line<P, Q, T>::fft: an M = P*Q point DFT shared by T threads, one shared
//    memory exchange. Thread t holds x[t + T*i] in r[i] on input *and* output,
//    so an inverse followed by a forward transform (crop -> modulate -> pad of
//    Eq. 1/5) needs no data movement between them.
//
// Sign convention: forward = exp(-2 pi j k n / M), inverse = exp(+2 pi j k n / M),
// both unnormalised (the 1/M^2 of the inverse 2D DFT is folded into H).
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

#define DOS_HD __host__ __device__ __forceinline__

namespace dos {

// ---------------------------------------------------------------- complex ops
DOS_HD float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
DOS_HD float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
DOS_HD float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
DOS_HD float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
DOS_HD float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
DOS_HD float2 czero() { return make_float2(0.f, 0.f); }

// Complex add / subtract as one packed FP32-pair instruction (add/sub.f32x2 of
// the sm_100 family) when PK is set, as two scalar ones otherwise.  Packed
// operands are opaque to the compiler (no folding of known zeros), so only the
// unpruned butterflies use them.
template <bool PK>
DOS_HD float2 vadd(float2 a, float2 b) {
#if defined(__CUDA_ARCH__)
  if constexpr (PK) {
    float2 d;
    asm("{\n .reg .b64 pa, pb, pd;\n mov.b64 pa, {%2, %3};\n mov.b64 pb, {%4, %5};\n"
        " add.rn.f32x2 pd, pa, pb;\n mov.b64 {%0, %1}, pd;\n}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
  }
#endif
  return cadd(a, b);
}
template <bool PK>
DOS_HD float2 vsub(float2 a, float2 b) {
#if defined(__CUDA_ARCH__)
  if constexpr (PK) {
    float2 d;
    asm("{\n .reg .b64 pa, pb, pd;\n mov.b64 pa, {%2, %3};\n mov.b64 pb, {%4, %5};\n"
        " sub.rn.f32x2 pd, pa, pb;\n mov.b64 {%0, %1}, pd;\n}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
  }
#endif
  return csub(a, b);
}

// a * (c, c) + acc and a * (c, c) for a scalar constant c: one packed FP32-pair
// instruction (fma / mul .rn.f32x2) when PK is set, two scalar ones otherwise
template <bool PK>
DOS_HD float2 vfma_bc(float2 a, float c, float2 acc) {
#if defined(__CUDA_ARCH__)
  if constexpr (PK) {
    float2 d;
    asm("{\n .reg .b64 pa, pc, pacc, pd;\n mov.b64 pa, {%2, %3};\n mov.b64 pc, {%4, %4};\n"
        " mov.b64 pacc, {%5, %6};\n fma.rn.f32x2 pd, pa, pc, pacc;\n mov.b64 {%0, %1}, pd;\n}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(c), "f"(acc.x), "f"(acc.y));
    return d;
  }
#endif
  return make_float2(fmaf(c, a.x, acc.x), fmaf(c, a.y, acc.y));
}
template <bool PK>
DOS_HD float2 vmul_bc(float2 a, float c) {
#if defined(__CUDA_ARCH__)
  if constexpr (PK) {
    float2 d;
    asm("{\n .reg .b64 pa, pc, pd;\n mov.b64 pa, {%2, %3};\n mov.b64 pc, {%4, %4};\n"
        " mul.rn.f32x2 pd, pa, pc;\n mov.b64 {%0, %1}, pd;\n}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(c));
    return d;
  }
#endif
  return make_float2(a.x * c, a.y * c);
}

// ------------------------------------------------- compile-time trigonometry
namespace ct {
constexpr double kPi = 3.14159265358979323846264338327950288;
constexpr double taylor_sin(double x) {
  double term = x, sum = x;
  for (int i = 1; i < 14; ++i) {
    term *= -x * x / ((2.0 * i) * (2.0 * i + 1.0));
    sum += term;
  }
  return sum;
}
constexpr double taylor_cos(double x) {
  double term = 1.0, sum = 1.0;
  for (int i = 1; i < 14; ++i) {
    term *= -x * x / ((2.0 * i - 1.0) * (2.0 * i));
    sum += term;
  }
  return sum;
}
// cos(2 pi k / n) for integers, by quarter-turn symmetry and a series on [0, pi/4].
constexpr double cos_turn(long k, long n) {
  k %= n;
  if (k < 0) k += n;
  const long q = (4 * k) / n;
  const long r = 4 * k - q * n;                 // angle = (q + r/n) * pi/2
  const double x = (double)r / (double)n * (kPi / 2);
  const double sx = x > kPi / 4 ? taylor_cos(kPi / 2 - x) : taylor_sin(x);
  const double cx = x > kPi / 4 ? taylor_sin(kPi / 2 - x) : taylor_cos(x);
  return q == 0 ? cx : q == 1 ? -sx : q == 2 ? -cx : sx;
}
// sin(2 pi k / n) = cos(2 pi (4k - n) / (4n))
constexpr double sin_turn(long k, long n) { return cos_turn(4 * k - n, 4 * n); }

constexpr int first_factor(int n) {
  return n % 4 == 0 && n != 4 ? 4 : n % 5 == 0 && n != 5 ? 5 : n % 3 == 0 && n != 3 ? 3 : 2;
}
constexpr bool is_base(int n) { return n == 2 || n == 3 || n == 4 || n == 5; }
constexpr int butterfly_cost(int n) { return n == 2 ? 4 : n == 3 ? 16 : n == 4 ? 16 : 36; }

// ---- pruning masks: bit i of an input mask = input i may be non-zero; bit k
// of an output mask = output k is needed (N <= 64)
using mask_t = unsigned long long;
constexpr mask_t lead_mask(int n) { return n <= 0 ? 0ull : n >= 64 ? ~0ull : ((1ull << n) - 1ull); }
constexpr bool has(mask_t m, int i) { return ((m >> i) & 1ull) != 0; }
constexpr int popcount(mask_t m) {
  int c = 0;
  for (; m; m >>= 1) c += (int)(m & 1ull);
  return c;
}
constexpr int lowest(mask_t m) {
  int i = 0;
  while (m && !(m & 1ull)) m >>= 1, ++i;
  return i;
}
// w^e is +-1 or +-j: a sign change or a swap, no arithmetic
constexpr bool trivial_turn(long e, long n) {
  e %= n;
  return e == 0 || 2 * e == n || 4 * e == n || 4 * e == 3 * n;
}
constexpr int gcd(int a, int b) { return b == 0 ? a : gcd(b, a % b); }
constexpr int inv_mod(int a, int m) {
  for (int x = 1; x < m; ++x)
    if ((a * x) % m == 1) return x;
  return 1;
}
// Good-Thomas (prime factor) indexing of N = P1 P2 with gcd(P1, P2) = 1:
// input n = (P2 i1 + P1 i2) mod N; output k with k = k1 (mod P1), k = k2 (mod P2)
// (Chinese remainder theorem).  Then X[k] = sum_i1 w_P1^(k1 i1) sum_i2 w_P2^(k2 i2)
// x[n]: two sets of short DFTs with no twiddle factors between them.
constexpr int pfa_in_index(int P1, int P2, int i1, int i2) { return (P2 * i1 + P1 * i2) % (P1 * P2); }
constexpr int pfa_out_index(int P1, int P2, int k1, int k2) {
  return (k1 * P2 * inv_mod(P2 % P1, P1) + k2 * P1 * inv_mod(P1 % P2, P2)) % (P1 * P2);
}
// masks of the sub-DFTs.  PFA: stage 1 = P2-point DFTs over i2 (one per i1),
// stage 2 = P1-point DFTs over i1 (one per k2).
constexpr mask_t pfa_in1(int P1, int P2, mask_t im, int i1) {
  mask_t m = 0;
  for (int i2 = 0; i2 < P2; ++i2)
    if (has(im, pfa_in_index(P1, P2, i1, i2))) m |= 1ull << i2;
  return m;
}
constexpr mask_t pfa_out1(int P1, int P2, mask_t om) {
  mask_t m = 0;
  for (int k = 0; k < P1 * P2; ++k)
    if (has(om, k)) m |= 1ull << (k % P2);
  return m;
}
constexpr mask_t pfa_in2(int P1, int P2, mask_t im) {
  mask_t m = 0;
  for (int i1 = 0; i1 < P1; ++i1)
    if (pfa_in1(P1, P2, im, i1)) m |= 1ull << i1;
  return m;
}
constexpr mask_t pfa_out2(int P1, int P2, mask_t om, int k2) {
  mask_t m = 0;
  for (int k1 = 0; k1 < P1; ++k1)
    if (has(om, pfa_out_index(P1, P2, k1, k2))) m |= 1ull << k1;
  return m;
}
// Cooley-Tukey N = A B: input n = B a + b, output k = k1 + A k2; stage 1 =
// A-point DFTs over a (one per b), twiddles w_N^(b k1), stage 2 = B-point DFTs
// over b (one per k1).
constexpr mask_t ct_in1(int A, int B, mask_t im, int b) {
  mask_t m = 0;
  for (int a = 0; a < A; ++a)
    if (has(im, B * a + b)) m |= 1ull << a;
  return m;
}
constexpr mask_t ct_out1(int A, int B, mask_t om) {
  mask_t m = 0;
  for (int k = 0; k < A * B; ++k)
    if (has(om, k)) m |= 1ull << (k % A);
  return m;
}
constexpr mask_t ct_in2(int A, int B, mask_t im) {
  mask_t m = 0;
  for (int b = 0; b < B; ++b)
    if (ct_in1(A, B, im, b)) m |= 1ull << b;
  return m;
}
constexpr mask_t ct_out2(int A, int B, mask_t om, int k1) {
  mask_t m = 0;
  for (int k2 = 0; k2 < B; ++k2)
    if (has(om, k1 + A * k2)) m |= 1ull << k2;
  return m;
}

// ---- plans: the cheapest way (estimated scalar FP32 instructions) to
// compute the needed outputs of an N-point DFT from its non-zero inputs
enum PlanKind : int { kNone, kZero, kOne, kDirect, kButterfly, kPfa, kCt };
struct Plan {
  int cost, kind, p1;
};
// X[k] = sum over inputs of x[j] w^(jk) for the needed k
constexpr int direct_cost(int n, mask_t im, mask_t om) {
  const int j0 = lowest(im);
  int c = 0;
  for (int k = 0; k < n; ++k) {
    if (!has(om, k)) continue;
    c += trivial_turn((long)j0 * k, n) ? 0 : 4;
    for (int j = j0 + 1; j < n; ++j)
      if (has(im, j)) c += 2 + (trivial_turn((long)j * k, n) ? 0 : 4);
  }
  return c;
}
constexpr Plan plan(int n, mask_t im, mask_t om) {
  im &= lead_mask(n);
  om &= lead_mask(n);
  if (n == 1 || om == 0) return Plan{0, kNone, 0};
  if (im == 0) return Plan{0, kZero, 0};
  if (popcount(im) == 1) {
    const int j = lowest(im);
    int c = 0;
    for (int k = 0; k < n; ++k)
      if (has(om, k) && !trivial_turn((long)j * k, n)) c += 4;
    return Plan{c, kOne, 0};
  }
  if (is_base(n)) {
    const bool full = im == lead_mask(n) && om == lead_mask(n);
    const int d = full ? 1 << 30 : direct_cost(n, im, om);
    return d < butterfly_cost(n) ? Plan{d, kDirect, 0} : Plan{butterfly_cost(n), kButterfly, 0};
  }
  Plan best{1 << 30, kCt, 0};
  // Good-Thomas splits (both orders of every coprime factor pair)
  for (int p1 = 2; p1 < n; ++p1) {
    if (n % p1 != 0 || gcd(p1, n / p1) != 1) continue;
    const int p2 = n / p1;
    const mask_t om1 = pfa_out1(p1, p2, om), im2 = pfa_in2(p1, p2, im);
    int c = 0;
    for (int i1 = 0; i1 < p1; ++i1) c += plan(p2, pfa_in1(p1, p2, im, i1), om1).cost;
    for (int k2 = 0; k2 < p2; ++k2)
      if (has(om1, k2)) c += plan(p1, im2, pfa_out2(p1, p2, om, k2)).cost;
    if (c < best.cost) best = Plan{c, kPfa, p1};
  }
  // Cooley-Tukey split with twiddles
  {
    const int a = first_factor(n), b = n / a;
    const mask_t om1 = ct_out1(a, b, om), im2 = ct_in2(a, b, im);
    int c = 0;
    for (int bb = 0; bb < b; ++bb) {
      const mask_t m = ct_in1(a, b, im, bb);
      if (!m) continue;
      c += plan(a, m, om1).cost;
      for (int k1 = 0; k1 < a; ++k1)
        if (has(om1, k1) && !trivial_turn((long)bb * k1, n)) c += 4;
    }
    for (int k1 = 0; k1 < a; ++k1)
      if (has(om1, k1)) c += plan(b, im2, ct_out2(a, b, om, k1)).cost;
    if (c < best.cost) best = Plan{c, kCt, a};
  }
  return best;
}
}  // namespace ct

template <int B, int E, typename F>
DOS_HD void static_for(F&& f) {
  if constexpr (B < E) {
    f(std::integral_constant<int, B>{});
    static_for<B + 1, E>(f);
  }
}

// x * w^E with w = exp(-2 pi j / N) (forward) or exp(+2 pi j / N) (inverse).
template <int N, long E, bool INV>
DOS_HD float2 twiddle(float2 x) {
  constexpr long e = ((E % N) + N) % N;
  if constexpr (e == 0) {
    return x;
  } else if constexpr (2 * e == N) {
    return make_float2(-x.x, -x.y);
  } else if constexpr (4 * e == N) {  // forward -j, inverse +j
    if constexpr (INV) return make_float2(-x.y, x.x);
    else return make_float2(x.y, -x.x);
  } else if constexpr (4 * e == 3 * N) {  // forward +j, inverse -j
    if constexpr (INV) return make_float2(x.y, -x.x);
    else return make_float2(-x.y, x.x);
  } else {
    constexpr float c = (float)ct::cos_turn(e, N);
    constexpr float s = INV ? (float)ct::sin_turn(e, N) : -(float)ct::sin_turn(e, N);
    return make_float2(fmaf(x.x, c, -x.y * s), fmaf(x.x, s, x.y * c));
  }
}

// ------------------------------------------------------------- butterflies
template <bool INV, bool PK = false>
DOS_HD void bfly2(float2* x) {
  const float2 a = x[0], b = x[1];
  x[0] = vadd<PK>(a, b);
  x[1] = vsub<PK>(a, b);
}
template <bool INV, bool PK = false>
DOS_HD void bfly3(float2* x) {
  constexpr float c = -0.5f;
  constexpr float s = INV ? 0.86602540378443864676f : -0.86602540378443864676f;
  const float2 t = vadd<PK>(x[1], x[2]);
  const float2 d = vsub<PK>(x[1], x[2]);
  const float2 m = make_float2(fmaf(c, t.x, x[0].x), fmaf(c, t.y, x[0].y));
  x[0] = vadd<PK>(x[0], t);
  // j*s*d
  const float2 jd = make_float2(-s * d.y, s * d.x);
  x[1] = cadd(m, jd);
  x[2] = csub(m, jd);
}
template <bool INV, bool PK = false>
DOS_HD void bfly4(float2* x) {
  const float2 t0 = vadd<PK>(x[0], x[2]);
  const float2 t1 = vsub<PK>(x[0], x[2]);
  const float2 t2 = vadd<PK>(x[1], x[3]);
  const float2 d = vsub<PK>(x[1], x[3]);
  // forward: -j*d, inverse: +j*d
  const float2 t3 = INV ? make_float2(-d.y, d.x) : make_float2(d.y, -d.x);
  x[0] = vadd<PK>(t0, t2);
  x[2] = vsub<PK>(t0, t2);
  x[1] = cadd(t1, t3);
  x[3] = csub(t1, t3);
}
template <bool INV, bool PK = false>
DOS_HD void bfly5(float2* x) {
  constexpr float c1 = 0.30901699437494742410f;   // cos(2 pi / 5)
  constexpr float c2 = -0.80901699437494742410f;  // cos(4 pi / 5)
  constexpr float s1 = 0.95105651629515357212f;   // sin(2 pi / 5)
  constexpr float s2 = 0.58778525229247312917f;   // sin(4 pi / 5)
  const float2 x0 = x[0];
  const float2 t1 = vadd<PK>(x[1], x[4]);
  const float2 t2 = vadd<PK>(x[2], x[3]);
  const float2 t3 = vsub<PK>(x[1], x[4]);
  const float2 t4 = vsub<PK>(x[2], x[3]);
  const float2 a1 = vfma_bc<PK>(t2, c2, vfma_bc<PK>(t1, c1, x0));
  const float2 a2 = vfma_bc<PK>(t2, c1, vfma_bc<PK>(t1, c2, x0));
  const float2 b1 = vfma_bc<PK>(t4, s2, vmul_bc<PK>(t3, s1));
  const float2 b2 = vfma_bc<PK>(t4, -s1, vmul_bc<PK>(t3, s2));
  // forward: X1 = a1 - j b1, X4 = a1 + j b1, X2 = a2 - j b2, X3 = a2 + j b2
  const float2 jb1 = INV ? make_float2(-b1.y, b1.x) : make_float2(b1.y, -b1.x);
  const float2 jb2 = INV ? make_float2(-b2.y, b2.x) : make_float2(b2.y, -b2.x);
  x[0] = vadd<PK>(vadd<PK>(x0, t1), t2);
  x[1] = cadd(a1, jb1);
  x[4] = csub(a1, jb1);
  x[2] = cadd(a2, jb2);
  x[3] = csub(a2, jb2);
}

// Direct sum X[k] = sum over the non-zero inputs j of x[j] w^(jk), needed k only.
template <int N, bool INV, ct::mask_t IM, ct::mask_t OM>
DOS_HD void dft_direct(float2* x) {
  constexpr int j0 = ct::lowest(IM);
  float2 out[N];
  static_for<0, N>([&](auto kk) {
    constexpr int k = kk;
    if constexpr (ct::has(OM, k)) {
      float2 acc = twiddle<N, (long)j0 * k, INV>(x[j0]);
      static_for<j0 + 1, N>([&](auto jj) {
        constexpr int j = jj;
        if constexpr (ct::has(IM, j)) acc = cadd(acc, twiddle<N, (long)j * k, INV>(x[j]));
      });
      out[k] = acc;
    }
  });
  static_for<0, N>([&](auto kk) {
    if constexpr (ct::has(OM, kk)) x[kk] = out[kk];
  });
}

// N-point DFT in registers, natural order in and out: only the inputs in IM
// are read (the others are zero), only the outputs in OM are produced (the
// others are left undefined).  The split is chosen at compile time by
// ct::plan: a radix-2/3/4/5 butterfly or a direct sum for the base sizes, and
// for composite sizes the cheaper of the Good-Thomas splits (coprime factors,
// no twiddles between the stages) and a Cooley-Tukey split (with twiddles).
template <int N, bool INV, ct::mask_t IM, ct::mask_t OM, bool PK = false>
DOS_HD void dftm(float2* x) {
  constexpr ct::Plan pl = ct::plan(N, IM, OM);
  constexpr ct::mask_t im = IM & ct::lead_mask(N), om = OM & ct::lead_mask(N);
  if constexpr (pl.kind == ct::kNone) {
    return;
  } else if constexpr (pl.kind == ct::kZero) {
    static_for<0, N>([&](auto k) {
      if constexpr (ct::has(om, k)) x[k] = czero();
    });
  } else if constexpr (pl.kind == ct::kOne) {
    constexpr int j = ct::lowest(im);
    const float2 v = x[j];
    static_for<0, N>([&](auto kk) {
      constexpr int k = kk;
      if constexpr (ct::has(om, k)) x[k] = twiddle<N, (long)j * k, INV>(v);
    });
  } else if constexpr (pl.kind == ct::kDirect) {
    dft_direct<N, INV, im, om>(x);
  } else if constexpr (pl.kind == ct::kButterfly) {
    static_for<0, N>([&](auto j) {
      if constexpr (!ct::has(im, j)) x[j] = czero();
    });
    constexpr bool pk = PK && im == ct::lead_mask(N);  // zero inputs fold only in scalar form
    if constexpr (N == 2) bfly2<INV, pk>(x);
    else if constexpr (N == 3) bfly3<INV, pk>(x);
    else if constexpr (N == 4) bfly4<INV, pk>(x);
    else bfly5<INV, pk>(x);
  } else if constexpr (pl.kind == ct::kPfa) {
    constexpr int P1 = pl.p1, P2 = N / P1;
    constexpr ct::mask_t OM1 = ct::pfa_out1(P1, P2, om), IM2 = ct::pfa_in2(P1, P2, im);
    float2 y[N];  // y[i1 * P2 + k2]
    static_for<0, P1>([&](auto ii) {
      constexpr int i1 = ii;
      constexpr ct::mask_t m = ct::pfa_in1(P1, P2, im, i1);
      if constexpr (m != 0) {
        float2 t[P2];
        static_for<0, P2>([&](auto jj) {
          constexpr int i2 = jj;
          if constexpr (ct::has(m, i2)) t[i2] = x[ct::pfa_in_index(P1, P2, i1, i2)];
        });
        dftm<P2, INV, m, OM1, PK>(t);
        static_for<0, P2>([&](auto kk) {
          if constexpr (ct::has(OM1, kk)) y[i1 * P2 + kk] = t[kk];
        });
      }
    });
    static_for<0, P2>([&](auto kk) {
      constexpr int k2 = kk;
      if constexpr (ct::has(OM1, k2)) {
        constexpr ct::mask_t o2 = ct::pfa_out2(P1, P2, om, k2);
        float2 t[P1];
        static_for<0, P1>([&](auto ii) {
          if constexpr (ct::has(IM2, ii)) t[ii] = y[ii * P2 + k2];
        });
        dftm<P1, INV, IM2, o2, PK>(t);
        static_for<0, P1>([&](auto k1) {
          if constexpr (ct::has(o2, k1)) x[ct::pfa_out_index(P1, P2, k1, k2)] = t[k1];
        });
      }
    });
  } else {
    constexpr int A = pl.p1, B = N / A;
    constexpr ct::mask_t OM1 = ct::ct_out1(A, B, om), IM2 = ct::ct_in2(A, B, im);
    float2 y[N];  // y[b * A + k1]
    static_for<0, B>([&](auto bb) {
      constexpr int b = bb;
      constexpr ct::mask_t m = ct::ct_in1(A, B, im, b);
      if constexpr (m != 0) {
        float2 t[A];
        static_for<0, A>([&](auto aa) {
          if constexpr (ct::has(m, aa)) t[aa] = x[B * aa + b];
        });
        dftm<A, INV, m, OM1, PK>(t);
        static_for<0, A>([&](auto kk) {
          constexpr int k1 = kk;
          if constexpr (ct::has(OM1, k1)) y[b * A + k1] = twiddle<N, (long)b * k1, INV>(t[k1]);
        });
      }
    });
    static_for<0, A>([&](auto kk) {
      constexpr int k1 = kk;
      if constexpr (ct::has(OM1, k1)) {
        constexpr ct::mask_t o2 = ct::ct_out2(A, B, om, k1);
        float2 t[B];
        static_for<0, B>([&](auto bb) {
          if constexpr (ct::has(IM2, bb)) t[bb] = y[bb * A + k1];
        });
        dftm<B, INV, IM2, o2, PK>(t);
        static_for<0, B>([&](auto k2) {
          if constexpr (ct::has(o2, k2)) x[k1 + A * k2] = t[k2];
        });
      }
    });
  }
}

// N-point DFT in registers; only x[0..NZ) are read, only X[0..NO) are produced.
template <int N, bool INV, int NZ = N, int NO = N, bool PK = false>
DOS_HD void dft(float2* x) {
  static_assert(NZ >= 0 && NZ <= N && NO >= 0 && NO <= N && N <= 64, "bad pruning");
  dftm<N, INV, ct::lead_mask(NZ), ct::lead_mask(NO), PK>(x);
}

// --------------------------------------------------- line FFT over T threads
// M = P*Q points shared by T threads (T | P, T | Q). Thread t holds element
// t + T*i in r[i], i < M/T, both before and after the transform.
// z: this line's exchange buffer (ZS float2 in shared memory).
// tw: shared table tw[q*TWP + k1] = exp(-2 pi j q k1 / M) (forward sign), 16-byte
// aligned, read two twiddles at a time.
// Every thread of the block must call fft() the same number of times (it
// contains two block-wide barriers).
// Pitch of the twiddle table rows: the smallest TWP >= p with TWP = 2 mod 4.
// Even, so that twiddles k1, k1 + 1 (k1 even) are one 16-byte load; and a
// row is an odd number of 16-byte units, so the loads of 8 consecutive rows
// (one quarter-warp of consecutive threads) fall on distinct bank quads.
constexpr int twiddle_pitch(int p) { return p + ((2 - p % 4) + 4) % 4; }

template <int P_, int Q_, int T_>
struct Line {
  static constexpr int P = P_, Q = Q_, T = T_, M = P * Q, E = M / T;
  static constexpr int QJ = Q / T, PJ = P / T;
  static constexpr int RP = (P % 2 == 0) ? P + 1 : P;  // odd pitch: conflict-free columns
  static constexpr int ZS = Q * RP;
  // twiddle table [Q][TWP] (twiddle_pitch): TWS entries, the space kernels
  // reserve for it in shared memory
  static constexpr int TWP = twiddle_pitch(P), TWS = Q * TWP;
  static_assert(P % T == 0 && Q % T == 0, "T must divide P and Q");
  // TR: the exchange matrix stored transposed (entry (q, k1) at k1 * RP + q).
  // For a square line (P = Q = T) step 1 of thread t writes exactly the
  // entries that step 2 of thread t read in the other layout, so two line
  // DFTs in alternating layouts need no barrier between them.
  static constexpr bool SQUARE = P == Q && T == P;

  // Step 1: the Q/T sub-DFTs of length P owned by thread t (q = t + T*j),
  // twiddled and written to the exchange matrix z[q][k1].
  // NZP: leading non-zero inputs of each sub-DFT (zero padding).
  // ZR: pitch of the exchange matrix (RP, or an even pitch for kernels whose
  // lines are laid out so that 16-byte accesses are conflict-free: then a
  // thread's entries k1, k1 + 1 (k1 even) of a row are one 16-byte store, and
  // in step 2 of the transposed layout q, q + 1 are one 16-byte load).
  template <bool INV, int NZP = P, bool PK = false, bool TR = false, int ZR = RP>
  DOS_HD static void step1(const float2 (&r)[E], int t, float2* z, const float2* tw) {
    static_assert(!TR || SQUARE, "the transposed exchange is for square lines");
    static_assert(ZR >= P && (!TR || ZR >= Q), "the pitch holds a row");
    constexpr bool V = !TR && ZR % 2 == 0;  // paired row stores
    static_for<0, QJ>([&](auto jj) {
      constexpr int j = jj;
      float2 a[P];
      static_for<0, NZP>([&](auto pp) { a[pp] = r[j + QJ * pp]; });
      dft<P, INV, NZP, P, PK>(a);
      const int q = t + T * j;
      const float4* twq = reinterpret_cast<const float4*>(tw + q * TWP);  // twiddle pairs
      float2* zq = TR ? z + q : z + q * ZR;
      constexpr int ZK = TR ? ZR : 1;  // stride of k1
      static_for<0, (P + 1) / 2>([&](auto pp) {
        constexpr int k0 = 2 * pp, k1 = 2 * pp + 1;
        const float4 w = twq[pp];
        float2 o0 = a[k0], o1;
        if constexpr (k0 > 0) {
          const float2 w0 = make_float2(w.x, w.y);
          o0 = INV ? cmulc(a[k0], w0) : cmul(a[k0], w0);
        }
        if constexpr (k1 < P) {
          const float2 w1 = make_float2(w.z, w.w);
          o1 = INV ? cmulc(a[k1], w1) : cmul(a[k1], w1);
        }
        if constexpr (V && k1 < P) {
          *reinterpret_cast<float4*>(zq + k0) = make_float4(o0.x, o0.y, o1.x, o1.y);
        } else {
          zq[k0 * ZK] = o0;
          if constexpr (k1 < P) zq[k1 * ZK] = o1;
        }
      });
    });
  }
  // Step 2: the P/T sub-DFTs of length Q owned by thread t (k1 = t + T*j),
  // read as columns of z; outputs k1 + P*k2 land in r[j + (P/T)*k2].
  // NOQ: leading outputs of each sub-DFT that are needed (cropping).
  template <bool INV, int NOQ = Q, bool PK = false, bool TR = false, int ZR = RP>
  DOS_HD static void step2(float2 (&r)[E], int t, const float2* z) {
    constexpr bool V = TR && ZR % 2 == 0;  // paired row loads
    static_for<0, PJ>([&](auto jj) {
      constexpr int j = jj;
      const int k1 = t + T * j;
      float2 b[Q];
      if constexpr (V) {
        const float4* zr = reinterpret_cast<const float4*>(z + k1 * ZR);
        static_for<0, Q / 2>([&](auto qq) {
          const float4 v = zr[qq];
          b[2 * qq] = make_float2(v.x, v.y);
          b[2 * qq + 1] = make_float2(v.z, v.w);
        });
        if constexpr (Q % 2 == 1) b[Q - 1] = z[k1 * ZR + Q - 1];
      } else {
        static_for<0, Q>([&](auto qq) { b[qq] = TR ? z[k1 * ZR + qq] : z[qq * ZR + k1]; });
      }
      dft<Q, INV, Q, NOQ, PK>(b);
      static_for<0, NOQ>([&](auto k2) { r[j + PJ * k2] = b[k2]; });
    });
  }
  // TRAIL: end with a barrier so that z may be rewritten right away; callers
  // that next write a different buffer (and reach another barrier before
  // reusing z) pass false.
  // PK: the unpruned butterflies add and subtract in packed FP32 pairs
  template <bool INV, int NZP = P, int NOQ = Q, bool TRAIL = true, bool PK = false, bool TR = false>
  __device__ static __forceinline__ void fft(float2 (&r)[E], int t, float2* z, const float2* tw) {
    step1<INV, NZP, PK, TR>(r, t, z, tw);
    __syncthreads();
    step2<INV, NOQ, PK, TR>(r, t, z);
    if constexpr (TRAIL) __syncthreads();
  }
};

}  // namespace dos
