// Batched 1-D mixed-radix DFTs of odd length on lines held in shared memory.
//
// Self-sorting (Stockham) formulation: stage s with radix R and
// Ns = product of the previous radices takes butterfly j (0 <= j < N/R) from
// positions j + r N/R, multiplies input r by w_N^(r (j mod Ns) N/(Ns R)),
// runs an R-point DFT and writes output r to (j div Ns) Ns R + (j mod Ns) +
// r Ns.  The result is in natural order after the last stage.  Forward
// transforms use w_N = exp(-2 pi i / N) (numpy's sign), inverse transforms
// the conjugate, both unnormalised.
//
// Odd radices 3, 5, 7, 11 use the symmetric form of the R-point DFT
// (pairs x_r +- x_(R-r)); composite radices 9, 15, 21, 25 nest two of them
// in registers; even radices 2, 4, 8 (even grids, Appendix C) nest the
// two-point butterfly; other primes use a direct sum, one output per thread.
// Stages alternate between two shared-memory buffers.
#pragma once
#include <type_traits>

#include "common.cuh"
#include "dfloat.cuh"

#define RVE_MAX_STAGES 16
// Threads per block of every kernel that runs the four-step line DFTs below;
// their work loops stride by this constant, not by blockDim.x, so that the
// compiler can fold the index arithmetic of each unrolled round.
#ifndef FFT_THREADS
#define FFT_THREADS 256
#endif

// Unsigned division by a run-time constant d through one 64-bit multiply:
// q = (a * ceil(2^40 / d)) >> 40, exact whenever a * d < 2^40 (all indices
// here are below 2^20).  The multiplier is computed on the host (a 64-bit
// division on the device would run on the FP64 pipe).
struct FastDiv {
  unsigned long long m;
  unsigned d;
  RVE_DEV unsigned div(unsigned a) const { return (unsigned)(((unsigned long long)a * m) >> 40); }
};

inline FastDiv make_fastdiv(unsigned d) {
  FastDiv f;
  f.d = d ? d : 1;
  f.m = ((1ull << 40) + f.d - 1) / f.d;
  return f;
}

struct AxisPlan {
  int n;
  int nst;
  int rad[RVE_MAX_STAGES];
  FastDiv fNs[RVE_MAX_STAGES];  // divide by the product of the earlier radices
  FastDiv fnb[RVE_MAX_STAGES];  // divide by n / rad[s] (butterflies per line)
  FastDiv fN;                   // divide by n
};

// Maps line index l to its first element in shared memory:
//   base(l) = (l >> gshift) * gstride + (l & (2^gshift - 1)) * lstride,
// element e at base + e*es (the group size is a power of two).
// lf != 0 assigns consecutive threads to consecutive lines (strided layouts),
// otherwise to consecutive butterflies of one line (contiguous layouts).
struct LineMap {
  int gshift, gstride, lstride, es, lf;
  RVE_DEV int base(int l) const {
    return (l >> gshift) * gstride + (l & ((1 << gshift) - 1)) * lstride;
  }
};

// ---------------------------------------------------------------------------
// Roots of unity as compile-time constants: cos and sin of 2 pi m / M by
// reduction to [0, pi/4] and the Taylor series there (the terms beyond
// x^25 / 25! are below 1e-30).  Used only in constant expressions.
// ---------------------------------------------------------------------------
constexpr double kPi = 3.14159265358979323846264338327950288;

constexpr double taylor_sin(double x) {
  double t = x, s = x;
  for (int k = 1; k < 13; ++k) {
    t *= -x * x / ((2.0 * k) * (2.0 * k + 1.0));
    s += t;
  }
  return s;
}

constexpr double taylor_cos(double x) {
  double t = 1.0, s = 1.0;
  for (int k = 1; k < 13; ++k) {
    t *= -x * x / ((2.0 * k - 1.0) * (2.0 * k));
    s += t;
  }
  return s;
}

// (cos, sin)(2 pi f) for f in [0, 1/4]
constexpr double quarter_cos(double f) {
  return f <= 0.125 ? taylor_cos(2.0 * kPi * f) : taylor_sin(2.0 * kPi * (0.25 - f));
}
constexpr double quarter_sin(double f) {
  return f <= 0.125 ? taylor_sin(2.0 * kPi * f) : taylor_cos(2.0 * kPi * (0.25 - f));
}

constexpr double cos2pi(int m, int M) {
  m %= M;
  if (m < 0) m += M;
  // 4m/M selects the quadrant; the remainder is exact in integers
  const int q = (4 * m) / M;
  const double f = (double)(4 * m - q * M) / (4.0 * M);  // in [0, 1/4)
  return q == 0 ? quarter_cos(f) : q == 1 ? -quarter_sin(f) : q == 2 ? -quarter_cos(f)
                                                                     : quarter_sin(f);
}

constexpr double sin2pi(int m, int M) {
  m %= M;
  if (m < 0) m += M;
  const int q = (4 * m) / M;
  const double f = (double)(4 * m - q * M) / (4.0 * M);
  return q == 0 ? quarter_sin(f) : q == 1 ? quarter_cos(f) : q == 2 ? -quarter_sin(f)
                                                                    : -quarter_cos(f);
}

// All M-th roots of unity exp(2 pi i m / M).
template <int M>
struct Roots {
  double c[M], s[M];
  constexpr Roots() : c(), s() {
    for (int m = 0; m < M; ++m) {
      c[m] = cos2pi(m, M);
      s[m] = sin2pi(m, M);
    }
  }
};

// Packed float pairs (one 64-bit register pair holding re, im) and the
// sm_100+ two-wide float instructions on them.
namespace f2 {
typedef unsigned long long u64;
RVE_DEV u64 pk(float lo, float hi) {
  u64 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
RVE_DEV float2 up(u64 r) {
  float2 f;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(f.x), "=f"(f.y) : "l"(r));
  return f;
}
RVE_DEV u64 add(u64 a, u64 b) {
  u64 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
RVE_DEV u64 sub(u64 a, u64 b) {
  u64 d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
RVE_DEV u64 fma(u64 a, u64 b, u64 c) {
  u64 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
RVE_DEV u64 mul(u64 a, u64 b) {
  u64 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
}  // namespace f2

// The symmetric odd-length DFT on packed pairs: the sums and differences of
// x_r, x_(R-r) and the accumulation over the roots take one two-wide
// instruction per complex value instead of two.
template <int RAD, bool INV>
RVE_DEV void dft_odd_f2(cplx<float> (&v)[RAD], const float (&cs)[RAD], const float (&sn)[RAD]) {
  constexpr int H = (RAD - 1) / 2;
  f2::u64 a[H], b[H];
#pragma unroll
  for (int r = 1; r <= H; ++r) {
    const f2::u64 p = f2::pk(v[r].x, v[r].y), q = f2::pk(v[RAD - r].x, v[RAD - r].y);
    a[r - 1] = f2::add(p, q);
    b[r - 1] = f2::sub(p, q);
  }
  const f2::u64 x0 = f2::pk(v[0].x, v[0].y);
  f2::u64 s = x0;
#pragma unroll
  for (int r = 0; r < H; ++r) s = f2::add(s, a[r]);
#pragma unroll
  for (int k = 1; k <= H; ++k) {
    f2::u64 re = x0, im;
#pragma unroll
    for (int r = 1; r <= H; ++r) {
      const int m = (r * k) % RAD;
      re = f2::fma(f2::pk(cs[m], cs[m]), a[r - 1], re);
      im = (r == 1) ? f2::mul(f2::pk(sn[m], sn[m]), b[r - 1])
                    : f2::fma(f2::pk(sn[m], sn[m]), b[r - 1], im);
    }
    const float2 e = f2::up(re), o = f2::up(im);
    if (!INV) {
      v[k] = {e.x + o.y, e.y - o.x};
      v[RAD - k] = {e.x - o.y, e.y + o.x};
    } else {
      v[k] = {e.x - o.y, e.y + o.x};
      v[RAD - k] = {e.x + o.y, e.y - o.x};
    }
  }
  const float2 s0 = f2::up(s);
  v[0] = {s0.x, s0.y};
}

template <typename R, int RAD, bool INV, bool PK = true>
RVE_DEV void dft_odd(cplx<R> (&v)[RAD], const R (&cs)[RAD], const R (&sn)[RAD]) {
  if constexpr (PK && std::is_same<R, float>::value) {
    dft_odd_f2<RAD, INV>(v, cs, sn);
    return;
  }
  constexpr int H = (RAD - 1) / 2;
  cplx<R> a[H], b[H];
#pragma unroll
  for (int r = 1; r <= H; ++r) {
    a[r - 1] = c_add(v[r], v[RAD - r]);
    b[r - 1] = c_sub(v[r], v[RAD - r]);
  }
  const cplx<R> x0 = v[0];
  cplx<R> s = x0;
#pragma unroll
  for (int r = 0; r < H; ++r) s = c_add(s, a[r]);
#pragma unroll
  for (int k = 1; k <= H; ++k) {
    cplx<R> re = x0, im = {R(0), R(0)};
#pragma unroll
    for (int r = 1; r <= H; ++r) {
      const int m = (r * k) % RAD;
      re.x = fma(cs[m], a[r - 1].x, re.x);
      re.y = fma(cs[m], a[r - 1].y, re.y);
      im.x = fma(sn[m], b[r - 1].x, im.x);
      im.y = fma(sn[m], b[r - 1].y, im.y);
    }
    // forward: X_k = re - i im, X_(R-k) = re + i im
    if (!INV) {
      v[k] = {re.x + im.y, re.y - im.x};
      v[RAD - k] = {re.x - im.y, re.y + im.x};
    } else {
      v[k] = {re.x - im.y, re.y + im.x};
      v[RAD - k] = {re.x + im.y, re.y - im.x};
    }
  }
  v[0] = s;
}

// One Stockham stage from `src` to `dst` (two shared-memory buffers): every
// thread takes butterflies b = tid, tid + nthr, ... of all L lines, so each
// butterfly is loaded, transformed and stored without waiting on others; one
// barrier ends the stage.  Strided layouts (lm.lf) give consecutive threads
// consecutive lines; contiguous layouts consecutive butterflies of a line.
template <typename R, int RAD, bool INV>
RVE_DEV void stage_pp(const cplx<R>* __restrict__ src, cplx<R>* __restrict__ dst, const LineMap lm,
                      int L, const FastDiv fL, int N, int Ns, const FastDiv fNs, const FastDiv fnb,
                      const cplx<R>* tw) {
  const int nb = N / RAD;
  const int tws = N / (Ns * RAD);
  R cs[RAD], sn[RAD];
#pragma unroll
  for (int m = 0; m < RAD; ++m) {
    const cplx<R> w = tw[m * nb];  // exp(-2 pi i m / RAD)
    cs[m] = w.x;
    sn[m] = -w.y;
  }
  const int total = L * nb;
  for (int b = threadIdx.x; b < total; b += blockDim.x) {
    int l, j;
    if (lm.lf) {
      j = (int)fL.div((unsigned)b);
      l = b - j * L;
    } else {
      l = (int)fnb.div((unsigned)b);
      j = b - l * nb;
    }
    const int jq = (int)fNs.div((unsigned)j);
    const int jr = j - jq * Ns;
    const int base = lm.base(l);
    cplx<R> v[RAD];
#pragma unroll
    for (int r = 0; r < RAD; ++r) v[r] = src[base + (j + r * nb) * lm.es];
    if (jr != 0) {  // all twiddles are 1 for the first butterfly of a group
#pragma unroll
      for (int r = 1; r < RAD; ++r) {
        const cplx<R> w = tw[r * jr * tws];
        v[r] = INV ? c_mulc(v[r], w) : c_mul(v[r], w);
      }
    }
    dft_odd<R, RAD, INV>(v, cs, sn);
    const int d = jq * Ns * RAD + jr;
#pragma unroll
    for (int r = 0; r < RAD; ++r) dst[base + (d + r * Ns) * lm.es] = v[r];
  }
  __syncthreads();
}

// R-point DFT with compile-time roots (cs[m] = cos(2 pi m/R), sn[m] =
// sin(2 pi m/R); the forward transform multiplies by exp(-2 pi i m/R)).
template <typename R, int RAD, bool INV, bool PK = true>
RVE_DEV void dft_const(cplx<R> (&v)[RAD]) {
  constexpr Roots<RAD> T{};
  R cs[RAD], sn[RAD];
#pragma unroll
  for (int m = 0; m < RAD; ++m) {
    cs[m] = (R)T.c[m];
    sn[m] = (R)T.s[m];
  }
  dft_odd<R, RAD, INV, PK>(v, cs, sn);
}

constexpr int smallest_factor(int m) {
  for (int p = 2; p * p <= m; ++p)
    if (m % p == 0) return p;
  return m;
}

template <typename R, int M, bool INV, bool PK = true>
RVE_DEV void dft_reg(cplx<R> (&v)[M]);

// M = R1 R2 point DFT in registers, natural order in and out, by one
// Cooley-Tukey split: with r = R2 a + b and k = k1 + R1 k2,
//   X_k = sum_b w_R2^(b k2) [w_M^(b k1) sum_a w_R1^(a k1) x_(R2 a + b)]
// (w_M = exp(-2 pi i / M) forward, its conjugate inverse).
template <typename R, int R1, int R2, bool INV, bool PK = true>
RVE_DEV void dft_split(cplx<R> (&v)[R1 * R2]) {
  constexpr int M = R1 * R2;
  constexpr Roots<M> T{};
#pragma unroll
  for (int b = 0; b < R2; ++b) {
    cplx<R> t[R1];
#pragma unroll
    for (int a = 0; a < R1; ++a) t[a] = v[R2 * a + b];
    dft_reg<R, R1, INV, PK>(t);
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) {
      cplx<R> y = t[k1];
      if (b > 0 && k1 > 0) {
        const R c = (R)T.c[(b * k1) % M];
        const R sg = INV ? (R)T.s[(b * k1) % M] : -(R)T.s[(b * k1) % M];
        y = {y.x * c - y.y * sg, fma(y.x, sg, y.y * c)};
      }
      v[R2 * k1 + b] = y;
    }
  }
  cplx<R> o[M];
#pragma unroll
  for (int k1 = 0; k1 < R1; ++k1) {
    cplx<R> t[R2];
#pragma unroll
    for (int b = 0; b < R2; ++b) t[b] = v[R2 * k1 + b];
    dft_reg<R, R2, INV, PK>(t);
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) o[k1 + R1 * k2] = t[k2];
  }
#pragma unroll
  for (int k = 0; k < M; ++k) v[k] = o[k];
}

// M-point DFT in registers: the two-point butterfly, the symmetric form for
// an odd prime, otherwise split off the smallest prime factor.
template <typename R, int M, bool INV, bool PK>
RVE_DEV void dft_reg(cplx<R> (&v)[M]) {
  if constexpr (M == 1) {
    return;
  } else if constexpr (M == 2) {
    const cplx<R> a = v[0];
    v[0] = c_add(a, v[1]);
    v[1] = c_sub(a, v[1]);
  } else if constexpr (smallest_factor(M) == M) {
    dft_const<R, M, INV, PK>(v);
  } else {
    dft_split<R, smallest_factor(M), M / smallest_factor(M), INV, PK>(v);
  }
}

// A Stockham stage of composite radix R1 R2 (the same data movement as
// stage_pp with RAD = R1 R2; the butterfly is dft_split): two stages for
// the price of one pass through shared memory.
template <typename R, int R1, int R2, bool INV>
RVE_DEV void stage_pp2(const cplx<R>* __restrict__ src, cplx<R>* __restrict__ dst,
                       const LineMap lm, int L, const FastDiv fL, int N, int Ns,
                       const FastDiv fNs, const FastDiv fnb, const cplx<R>* tw) {
  constexpr int RAD = R1 * R2;
  const int nb = N / RAD;
  const int tws = N / (Ns * RAD);
  const int total = L * nb;
  for (int b = threadIdx.x; b < total; b += blockDim.x) {
    int l, j;
    if (lm.lf) {
      j = (int)fL.div((unsigned)b);
      l = b - j * L;
    } else {
      l = (int)fnb.div((unsigned)b);
      j = b - l * nb;
    }
    const int jq = (int)fNs.div((unsigned)j);
    const int jr = j - jq * Ns;
    const int base = lm.base(l);
    cplx<R> v[RAD];
#pragma unroll
    for (int r = 0; r < RAD; ++r) v[r] = src[base + (j + r * nb) * lm.es];
    if (jr != 0) {
      const int step = jr * tws;
#pragma unroll
      for (int r = 1; r < RAD; ++r) {
        const cplx<R> w = tw[r * step];
        v[r] = INV ? c_mulc(v[r], w) : c_mul(v[r], w);
      }
    }
    dft_split<R, R1, R2, INV>(v);
    const int d = jq * Ns * RAD + jr;
#pragma unroll
    for (int r = 0; r < RAD; ++r) dst[base + (d + r * Ns) * lm.es] = v[r];
  }
  __syncthreads();
}

// A Stockham stage of any compile-time radix M (used for the even radices
// 2, 4, 8): the data movement of stage_pp, butterfly dft_reg<M>.
template <typename R, int M, bool INV>
RVE_DEV void stage_ppM(const cplx<R>* __restrict__ src, cplx<R>* __restrict__ dst,
                       const LineMap lm, int L, const FastDiv fL, int N, int Ns,
                       const FastDiv fNs, const FastDiv fnb, const cplx<R>* tw) {
  const int nb = N / M;
  const int tws = N / (Ns * M);
  const int total = L * nb;
  for (int b = threadIdx.x; b < total; b += blockDim.x) {
    int l, j;
    if (lm.lf) {
      j = (int)fL.div((unsigned)b);
      l = b - j * L;
    } else {
      l = (int)fnb.div((unsigned)b);
      j = b - l * nb;
    }
    const int jq = (int)fNs.div((unsigned)j);
    const int jr = j - jq * Ns;
    const int base = lm.base(l);
    cplx<R> v[M];
#pragma unroll
    for (int r = 0; r < M; ++r) v[r] = src[base + (j + r * nb) * lm.es];
    if (jr != 0) {
      const int step = jr * tws;
#pragma unroll
      for (int r = 1; r < M; ++r) {
        const cplx<R> w = tw[r * step];
        v[r] = INV ? c_mulc(v[r], w) : c_mul(v[r], w);
      }
    }
    dft_reg<R, M, INV>(v);
    const int d = jq * Ns * M + jr;
#pragma unroll
    for (int r = 0; r < M; ++r) dst[base + (d + r * Ns) * lm.es] = v[r];
  }
  __syncthreads();
}

// Direct R-point DFT for any prime R: one output element per thread.
template <typename R, bool INV>
RVE_DEV void stage_pp_generic(const cplx<R>* __restrict__ src, cplx<R>* __restrict__ dst,
                              const LineMap lm, int L, const FastDiv fL, int N, int Ns, int RAD,
                              const FastDiv fNs, const FastDiv fnb, const FastDiv fN,
                              const cplx<R>* tw) {
  const int nb = N / RAD;
  const int tws = N / (Ns * RAD);
  const int total = L * N;
  for (int o = threadIdx.x; o < total; o += blockDim.x) {
    int l, q;
    if (lm.lf) {
      q = (int)fL.div((unsigned)o);
      l = o - q * L;
    } else {
      l = (int)fN.div((unsigned)o);
      q = o - l * N;
    }
    const int k = (int)fnb.div((unsigned)q);
    const int j = q - k * nb;
    const int jq = (int)fNs.div((unsigned)j);
    const int jr = j - jq * Ns;
    const int base = lm.base(l);
    const int m = jr * tws + k * nb;  // < N
    cplx<R> acc = {R(0), R(0)};
    int e = 0;
    for (int r = 0; r < RAD; ++r) {
      const cplx<R> x = src[base + (j + r * nb) * lm.es];
      const cplx<R> w = tw[e];
      acc = c_add(acc, INV ? c_mulc(x, w) : c_mul(x, w));
      e += m;
      if (e >= N) e -= N;
    }
    dst[base + (jq * Ns * RAD + jr + k * Ns) * lm.es] = acc;
  }
  __syncthreads();
}

// Copies an axis plan into shared memory (indexing a kernel parameter with a
// run-time stage number would force a local-memory copy per thread).
RVE_DEV void load_plan(AxisPlan* dst, const AxisPlan& src) {
  const int* s = reinterpret_cast<const int*>(&src);
  int* d = reinterpret_cast<int*>(dst);
  for (int i = threadIdx.x; i < (int)(sizeof(AxisPlan) / sizeof(int)); i += blockDim.x) d[i] = s[i];
}

// All stages of the plan on L lines, ping-ponging between buffers a and b
// (same layout).  tw[k] = exp(-2 pi i k / N) must be in shared memory.
// Returns the buffer that holds the result.  Caller synchronises before.
template <typename R, bool INV>
RVE_DEV cplx<R>* fft_lines(cplx<R>* a, cplx<R>* b, const LineMap& lm, int L, const FastDiv fL,
                           const AxisPlan& p, const cplx<R>* tw) {
  int Ns = 1;
  for (int s = 0; s < p.nst; ++s) {
    const int rad = p.rad[s];
    const FastDiv fNs = p.fNs[s], fnb = p.fnb[s];
    switch (rad) {
      case 3: stage_pp<R, 3, INV>(a, b, lm, L, fL, p.n, Ns, fNs, fnb, tw); break;
      case 5: stage_pp<R, 5, INV>(a, b, lm, L, fL, p.n, Ns, fNs, fnb, tw); break;
      case 7: stage_pp<R, 7, INV>(a, b, lm, L, fL, p.n, Ns, fNs, fnb, tw); break;
      case 11: stage_pp<R, 11, INV>(a, b, lm, L, fL, p.n, Ns, fNs, fnb, tw); break;
      case 2: stage_ppM<R, 2, INV>(a, b, lm, L, fL, p.n, Ns, fNs, fnb, tw); break;
      case 4: stage_ppM<R, 4, INV>(a, b, lm, L, fL, p.n, Ns, fNs, fnb, tw); break;
      case 8: stage_ppM<R, 8, INV>(a, b, lm, L, fL, p.n, Ns, fNs, fnb, tw); break;
      default:
        if constexpr (!is_dfl<R>::value) {  // float-float plans have no composite radices
          if (rad == 9) {
            stage_pp2<R, 3, 3, INV>(a, b, lm, L, fL, p.n, Ns, fNs, fnb, tw);
            break;
          } else if (rad == 15) {
            stage_pp2<R, 5, 3, INV>(a, b, lm, L, fL, p.n, Ns, fNs, fnb, tw);
            break;
          } else if (rad == 21) {
            stage_pp2<R, 7, 3, INV>(a, b, lm, L, fL, p.n, Ns, fNs, fnb, tw);
            break;
          } else if (rad == 25) {
            stage_pp2<R, 5, 5, INV>(a, b, lm, L, fL, p.n, Ns, fNs, fnb, tw);
            break;
          }
        }
        stage_pp_generic<R, INV>(a, b, lm, L, fL, p.n, Ns, rad, fNs, fnb, p.fN, tw);
        break;
    }
    cplx<R>* t = a;
    a = b;
    b = t;
    Ns *= rad;
  }
  return a;
}

// Out-of-line entry for kernels that run several transforms (the x pass):
// each call gets its own register allocation.
template <typename R, bool INV>
__device__ __noinline__ cplx<R>* fft_lines_call(cplx<R>* a, cplx<R>* b, const LineMap lm, int L,
                                                const FastDiv fL, const AxisPlan* p,
                                                const cplx<R>* tw) {
  return fft_lines<R, INV>(a, b, lm, L, fL, *p, tw);
}

// ---------------------------------------------------------------------------
// In-place DFTs of compile-time length N = N1 N2 on the L lines of a
// compile-time layout LM in one shared buffer (line l, element e at
// LM::base(l) + e LM::ES; consecutive threads take consecutive lines, and
// every shared-memory offset inside a work item is a constant).  Four-step
// split with n = N2 m + n2, k = k1 + N1 k2:
//   phase A (per line and n2):  Y_n2(k1) = w_N^(n2 k1) sum_m w_N1^(m k1) x_(N2 m + n2)
//   phase B (per line and k1):  X_(k1 + N1 k2) = sum_n2 w_N2^(n2 k2) Y_n2(k1)
// Each work item reads and writes the same N1 (phase A) or N2 (phase B)
// positions, so no second buffer is needed; the forward result is stored
// transposed: X_(k1 + N1 k2) at position N2 k1 + k2 (fs_freq / fs_pos).  The
// inverse runs the conjugate phases in reverse order and takes that
// transposed order back to natural order.  tw2[n2 N1 + k1] = w_N^(n2 k1).
// ---------------------------------------------------------------------------
template <int G_, int GS_, int LS_, int ES_, int L_>
struct FsLayout {
  static constexpr int G = G_, GS = GS_, LS = LS_, ES = ES_, L = L_;
  static RVE_DEV int base(int l) { return (l / G) * GS + (l % G) * LS; }
};

template <int N1, int N2>
RVE_DEV int fs_freq(int pos) { return pos / N2 + N1 * (pos % N2); }
template <int N1, int N2>
RVE_DEV int fs_pos(int k) { return N2 * (k % N1) + k / N1; }

// tw2[n2 N1 + k1] = tw[n2 k1] (tw[k] = exp(-2 pi i k / N)), built by the block
template <typename R, int N1, int N2>
RVE_DEV void fs_twiddles(cplx<R>* tw2, const cplx<R>* tw) {
  for (int j = threadIdx.x; j < N1 * N2; j += FFT_THREADS) {
    const int n2 = j / N1, k1 = j - (j / N1) * N1;
    tw2[j] = tw[n2 * k1];
  }
}

template <typename R, int N1, int N2, bool INV, typename LM>
RVE_DEV void fs_phase_a(cplx<R>* buf, const cplx<R>* tw2) {
  constexpr int total = LM::L * N2;
  for (int i = threadIdx.x; i < total; i += FFT_THREADS) {
    const int n2 = i / LM::L;
    const int l = i - n2 * LM::L;
    cplx<R>* line = buf + LM::base(l) + n2 * LM::ES;
    const cplx<R>* w = tw2 + n2 * N1;
    cplx<R> v[N1];
#pragma unroll
    for (int m = 0; m < N1; ++m) v[m] = line[m * N2 * LM::ES];
    if (INV && n2 != 0) {
#pragma unroll
      for (int k1 = 1; k1 < N1; ++k1) v[k1] = c_mulc(v[k1], w[k1]);
    }
    dft_reg<R, N1, INV>(v);
    if (!INV && n2 != 0) {
#pragma unroll
      for (int k1 = 1; k1 < N1; ++k1) v[k1] = c_mul(v[k1], w[k1]);
    }
#pragma unroll
    for (int m = 0; m < N1; ++m) line[m * N2 * LM::ES] = v[m];
  }
}

template <typename R, int N1, int N2, bool INV, typename LM, bool PK = true>
RVE_DEV void fs_phase_b(cplx<R>* buf) {
  constexpr int total = LM::L * N1;
  for (int i = threadIdx.x; i < total; i += FFT_THREADS) {
    const int k1 = i / LM::L;
    const int l = i - k1 * LM::L;
    cplx<R>* line = buf + LM::base(l) + N2 * k1 * LM::ES;
    cplx<R> u[N2];
#pragma unroll
    for (int j = 0; j < N2; ++j) u[j] = line[j * LM::ES];
    dft_reg<R, N2, INV, PK>(u);
#pragma unroll
    for (int j = 0; j < N2; ++j) line[j * LM::ES] = u[j];
  }
}

// Forward: natural order in, transposed order out.  Inverse: transposed in,
// natural out.  Caller synchronises before; returns after a barrier.
template <typename R, int N1, int N2, bool INV, typename LM>
RVE_DEV void fs_lines(cplx<R>* buf, const cplx<R>* tw2) {
  if (!INV) {
    fs_phase_a<R, N1, N2, false, LM>(buf, tw2);
    __syncthreads();
    if (N2 > 1) fs_phase_b<R, N1, N2, false, LM>(buf);
    __syncthreads();
  } else {
    if (N2 > 1) fs_phase_b<R, N1, N2, true, LM>(buf);
    __syncthreads();
    fs_phase_a<R, N1, N2, true, LM>(buf, tw2);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// The same two phases with one end in global memory, for passes whose lines
// are tile rows: `gl(l)` gives line l's first element in global memory, its
// element stride and whether it may be read / written (the caller's tile
// bounds).  A phase reading global memory loads its N1 (or N2) values
// straight into registers, a phase writing global memory stores them from
// registers, so the tile makes a single trip through shared memory.
// ---------------------------------------------------------------------------
template <typename R>
struct GLine {
  cplx<R>* p;
  size_t stride;
  bool rd, wr;
};

// forward phase A: natural order from global, result to shared memory
template <typename R, int N1, int N2, typename LM, typename GL, bool PK = true>
RVE_DEV void fs_phase_a_g2s(cplx<R>* buf, const cplx<R>* tw2, const GL& gl) {
  constexpr int total = LM::L * N2;
  for (int i = threadIdx.x; i < total; i += FFT_THREADS) {
    const int n2 = i / LM::L;
    const int l = i - n2 * LM::L;
    const GLine<R> g = gl(l);
    cplx<R> v[N1];
#pragma unroll
    for (int m = 0; m < N1; ++m)
      v[m] = g.rd ? g.p[(size_t)(N2 * m + n2) * g.stride] : cplx<R>{R(0), R(0)};
    dft_reg<R, N1, false, PK>(v);
    if (n2 != 0) {
      const cplx<R>* w = tw2 + n2 * N1;
#pragma unroll
      for (int k1 = 1; k1 < N1; ++k1) v[k1] = c_mul(v[k1], w[k1]);
    }
    cplx<R>* line = buf + LM::base(l) + n2 * LM::ES;
#pragma unroll
    for (int m = 0; m < N1; ++m) line[m * N2 * LM::ES] = v[m];
  }
}

// forward phase B: from shared memory, natural-order result to global
template <typename R, int N1, int N2, typename LM, typename GL>
RVE_DEV void fs_phase_b_s2g(const cplx<R>* buf, const GL& gl) {
  constexpr int total = LM::L * N1;
  for (int i = threadIdx.x; i < total; i += FFT_THREADS) {
    const int k1 = i / LM::L;
    const int l = i - k1 * LM::L;
    const cplx<R>* line = buf + LM::base(l) + N2 * k1 * LM::ES;
    cplx<R> u[N2];
#pragma unroll
    for (int j = 0; j < N2; ++j) u[j] = line[j * LM::ES];
    dft_reg<R, N2, false>(u);
    const GLine<R> g = gl(l);
    if (g.wr) {
#pragma unroll
      for (int k2 = 0; k2 < N2; ++k2) g.p[(size_t)(k1 + N1 * k2) * g.stride] = u[k2];
    }
  }
}

// inverse phase B: natural-order spectrum from global, to shared memory
template <typename R, int N1, int N2, typename LM, typename GL>
RVE_DEV void fs_phase_b_g2s(cplx<R>* buf, const GL& gl) {
  constexpr int total = LM::L * N1;
  for (int i = threadIdx.x; i < total; i += FFT_THREADS) {
    const int k1 = i / LM::L;
    const int l = i - k1 * LM::L;
    const GLine<R> g = gl(l);
    cplx<R> u[N2];
#pragma unroll
    for (int j = 0; j < N2; ++j)
      u[j] = g.rd ? g.p[(size_t)(k1 + N1 * j) * g.stride] : cplx<R>{R(0), R(0)};
    dft_reg<R, N2, true>(u);
    cplx<R>* line = buf + LM::base(l) + N2 * k1 * LM::ES;
#pragma unroll
    for (int j = 0; j < N2; ++j) line[j * LM::ES] = u[j];
  }
}

// inverse phase A: from shared memory, natural-order result to global
template <typename R, int N1, int N2, typename LM, typename GL>
RVE_DEV void fs_phase_a_s2g(const cplx<R>* buf, const cplx<R>* tw2, const GL& gl) {
  constexpr int total = LM::L * N2;
  for (int i = threadIdx.x; i < total; i += FFT_THREADS) {
    const int n2 = i / LM::L;
    const int l = i - n2 * LM::L;
    const cplx<R>* line = buf + LM::base(l) + n2 * LM::ES;
    cplx<R> v[N1];
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) v[k1] = line[k1 * N2 * LM::ES];
    if (n2 != 0) {
      const cplx<R>* w = tw2 + n2 * N1;
#pragma unroll
      for (int k1 = 1; k1 < N1; ++k1) v[k1] = c_mulc(v[k1], w[k1]);
    }
    dft_reg<R, N1, true>(v);
    const GLine<R> g = gl(l);
    if (g.wr) {
#pragma unroll
      for (int m = 0; m < N1; ++m) g.p[(size_t)(N2 * m + n2) * g.stride] = v[m];
    }
  }
}
