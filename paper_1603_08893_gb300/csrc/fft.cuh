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
// thread.  All stages of a line run in place: each thread loads its
// butterflies into registers, the block synchronises, then stores.
#pragma once
#include "common.cuh"

#define RVE_MAX_STAGES 16

struct AxisPlan {
  int n;
  int nst;
  int rad[RVE_MAX_STAGES];
};

// Maps line index l to its first element in shared memory:
//   base(l) = (l / grp) * gstride + (l % grp) * lstride, element e at base + e*es.
// lf != 0 assigns consecutive threads to consecutive lines (strided layouts),
// otherwise to consecutive butterflies of one line (contiguous layouts).
struct LineMap {
  int grp, gstride, lstride, es, lf;
  RVE_DEV int base(int l) const { return (l / grp) * gstride + (l % grp) * lstride; }
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

template <typename R, int RAD, bool INV>
__device__ __noinline__ void fft_stage(cplx<R>* buf, const LineMap lm, int nlines, int N, int Ns,
                                       const cplx<R>* tw) {
  constexpr int MAXB = (RAD <= 3) ? 2 : 1;
  const int nb = N / RAD;
  const int tws = N / (Ns * RAD);
  R cs[RAD], sn[RAD];
#pragma unroll
  for (int m = 0; m < RAD; ++m) {
    const cplx<R> w = tw[m * nb];  // exp(-2 pi i m / RAD)
    cs[m] = w.x;
    sn[m] = -w.y;
  }
  const int nthr = blockDim.x;
  int lpc = (nthr * MAXB) / nb;
  if (lpc < 1) lpc = 1;
  for (int l0 = 0; l0 < nlines; l0 += lpc) {
    const int nl = min(lpc, nlines - l0);
    const int cnt = nl * nb;
    cplx<R> v[MAXB][RAD];
#pragma unroll
    for (int t = 0; t < MAXB; ++t) {
      const int b = t * nthr + threadIdx.x;
      if (b < cnt) {
        int l, j;
        if (lm.lf) { l = b % nl; j = b / nl; } else { l = b / nb; j = b - (b / nb) * nb; }
        const cplx<R>* base = buf + lm.base(l0 + l);
        const int jr = j % Ns;
#pragma unroll
        for (int r = 0; r < RAD; ++r) v[t][r] = base[(j + r * nb) * lm.es];
#pragma unroll
        for (int r = 1; r < RAD; ++r) {
          const cplx<R> w = tw[r * jr * tws];
          v[t][r] = INV ? c_mulc(v[t][r], w) : c_mul(v[t][r], w);
        }
        dft_odd<R, RAD, INV>(v[t], cs, sn);
      }
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < MAXB; ++t) {
      const int b = t * nthr + threadIdx.x;
      if (b < cnt) {
        int l, j;
        if (lm.lf) { l = b % nl; j = b / nl; } else { l = b / nb; j = b - (b / nb) * nb; }
        cplx<R>* base = buf + lm.base(l0 + l);
        const int jr = j % Ns;
        const int d = (j / Ns) * Ns * RAD + jr;
#pragma unroll
        for (int r = 0; r < RAD; ++r) base[(d + r * Ns) * lm.es] = v[t][r];
      }
    }
    __syncthreads();
  }
}

// Direct R-point DFT for any prime R: one output element per thread.
template <typename R, bool INV>
__device__ __noinline__ void fft_stage_generic(cplx<R>* buf, const LineMap lm, int nlines, int N,
                                               int Ns, int RAD, const cplx<R>* tw) {
  constexpr int MAXO = 2;
  const int nb = N / RAD;
  const int tws = N / (Ns * RAD);
  const int nthr = blockDim.x;
  int lpc = (nthr * MAXO) / N;
  if (lpc < 1) lpc = 1;
  for (int l0 = 0; l0 < nlines; l0 += lpc) {
    const int nl = min(lpc, nlines - l0);
    const int cnt = nl * N;
    cplx<R> out[MAXO];
#pragma unroll
    for (int t = 0; t < MAXO; ++t) {
      const int o = t * nthr + threadIdx.x;
      if (o < cnt) {
        int l, q;
        if (lm.lf) { l = o % nl; q = o / nl; } else { l = o / N; q = o - (o / N) * N; }
        const int k = q / nb, j = q - (q / nb) * nb;
        const cplx<R>* base = buf + lm.base(l0 + l);
        const int m = (j % Ns) * tws + k * nb;  // < N
        cplx<R> acc = {R(0), R(0)};
        int e = 0;
        for (int r = 0; r < RAD; ++r) {
          const cplx<R> x = base[(j + r * nb) * lm.es];
          const cplx<R> w = tw[e];
          const cplx<R> p = INV ? c_mulc(x, w) : c_mul(x, w);
          acc = c_add(acc, p);
          e += m;
          if (e >= N) e -= N;
        }
        out[t] = acc;
      }
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < MAXO; ++t) {
      const int o = t * nthr + threadIdx.x;
      if (o < cnt) {
        int l, q;
        if (lm.lf) { l = o % nl; q = o / nl; } else { l = o / N; q = o - (o / N) * N; }
        const int k = q / nb, j = q - (q / nb) * nb;
        cplx<R>* base = buf + lm.base(l0 + l);
        const int d = (j / Ns) * Ns * RAD + (j % Ns) + k * Ns;
        base[d * lm.es] = out[t];
      }
    }
    __syncthreads();
  }
}

// All stages of the plan on `nlines` lines.  tw[k] = exp(-2 pi i k / N) must
// be readable by every thread (shared memory).  Caller synchronises before.
template <typename R, bool INV>
RVE_DEV void fft_lines(cplx<R>* buf, const LineMap& lm, int nlines, const AxisPlan& p,
                       const cplx<R>* tw) {
  int Ns = 1;
  for (int s = 0; s < p.nst; ++s) {
    const int rad = p.rad[s];
    switch (rad) {
      case 3: fft_stage<R, 3, INV>(buf, lm, nlines, p.n, Ns, tw); break;
      case 5: fft_stage<R, 5, INV>(buf, lm, nlines, p.n, Ns, tw); break;
      case 7: fft_stage<R, 7, INV>(buf, lm, nlines, p.n, Ns, tw); break;
      case 11: fft_stage<R, 11, INV>(buf, lm, nlines, p.n, Ns, tw); break;
      default: fft_stage_generic<R, INV>(buf, lm, nlines, p.n, Ns, rad, tw); break;
    }
    Ns *= rad;
  }
}
