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
// (pairs x_r +- x_(R-r)); other primes use a direct sum, one output per
// thread.  Stages alternate between two shared-memory buffers.
#pragma once
#include "common.cuh"

#define RVE_MAX_STAGES 16

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

template <typename R, int RAD, bool INV>
RVE_DEV void dft_odd(cplx<R> (&v)[RAD], const R (&cs)[RAD], const R (&sn)[RAD]) {
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
#pragma unroll
    for (int r = 1; r < RAD; ++r) {
      const cplx<R> w = tw[r * jr * tws];
      v[r] = INV ? c_mulc(v[r], w) : c_mul(v[r], w);
    }
    dft_odd<R, RAD, INV>(v, cs, sn);
    const int d = jq * Ns * RAD + jr;
#pragma unroll
    for (int r = 0; r < RAD; ++r) dst[base + (d + r * Ns) * lm.es] = v[r];
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
      default: stage_pp_generic<R, INV>(a, b, lm, L, fL, p.n, Ns, rad, fNs, fnb, p.fN, tw); break;
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
