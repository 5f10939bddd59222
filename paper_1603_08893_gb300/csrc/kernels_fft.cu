// FFT pass kernels of the projected tangent operator  p -> G : (K : p)
// (Eq. iter:system; G-hat of Eq. G, applied in the reduced form of
// Eq. G_red).  Fields are component-major [9][nx][ny][nz] (z fastest); the
// half spectrum is [9][nx][ny][hzp] complex with kz in [0, nz/2].
//
//   zfwd   : per z-line: CG direction update, tangent contraction K : p,
//            then a real-to-complex DFT along z (two real components are
//            packed into one complex line and split by Hermitian symmetry).
//   fft_y  : complex DFT along y on (kz-tile x ny) tiles.
//   fft_x  : forward DFT along x, projection, inverse DFT along x, on
//            (kz-tile x nx x 9 components) tiles that stay in shared memory.
//   zinv   : complex-to-real inverse DFT along z and the output stage
//            (plain copy, CG product p.Ap, or residual / CG initialisation).
#include <algorithm>
#include <map>
#include <mutex>

#include "kernels.h"

#include "fft_pass.cuh"

template <typename R, int SRC, int TAN>
__global__ void FFT_BOUNDS(R) k_zfwd(const ZfwdParams<R> P) {
  if (P.done && *P.done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nz = P.g.nz, lz = P.lz;
  cplx<R>* tw = reinterpret_cast<cplx<R>*>(smem_raw);
  cplx<R>* bufA = tw + ((nz + 1) & ~1);  // [5][lz][nz]
  cplx<R>* bufB = bufA + 5 * lz * nz;
  for (int i = threadIdx.x; i < nz; i += blockDim.x) tw[i] = P.tw[i];
  __shared__ AxisPlan plan;
  load_plan(&plan, axis_plan<R>(P.g, 2));
  const int nlines = P.g.nx * P.g.ny;
  const int l0 = blockIdx.x * lz;
  const int nl = min(lz, nlines - l0);
  const int nvox = nl * nz;
  const size_t v0 = (size_t)l0 * nz;
  const ZfwdScalars<R> sc = zfwd_scalars<R, SRC>(P);
  double pkp = 0.0;
  for (int i = threadIdx.x; i < lz * nz; i += blockDim.x) {
    R out[9];
    if (i < nvox) {
      zfwd_voxel<R, SRC, TAN>(P, sc, v0 + i, out, pkp);
    } else {
#pragma unroll
      for (int c = 0; c < 9; ++c) out[c] = R(0);
    }
#pragma unroll
    for (int k = 0; k < 5; ++k)
      bufA[k * lz * nz + i] = {out[2 * k], (2 * k + 1 < 9) ? out[2 * k + 1] : R(0)};
  }
  __syncthreads();
  const LineMap lm{30, 0, nz, 1, 0};
  const cplx<R>* res = fft_lines<R, false>(bufA, bufB, lm, 5 * lz, P.g.f_hz, plan, tw);
  const int hz = P.g.hz, hzp = P.g.hzp;
  const size_t ss = P.g.sstride;
  const FastDiv dhz = P.g.f_hz, dlz = sizeof(R) == 4 ? P.g.f_lzf : P.g.f_lzd;
  for (int i = threadIdx.x; i < 5 * lz * hz; i += blockDim.x) {
    const int rest = (int)dhz.div((unsigned)i);
    const int kz = i - rest * hz;
    const int k = (int)dlz.div((unsigned)rest);
    const int li = rest - k * lz;
    if (li >= nl) continue;
    const cplx<R> z1 = res[(k * lz + li) * nz + kz];
    cplx<R> z2 = res[(k * lz + li) * nz + (kz ? nz - kz : 0)];
    z2.y = -z2.y;
    const size_t o = (size_t)(l0 + li) * hzp + kz;
    P.spec[(size_t)(2 * k) * ss + o] = {R(0.5) * (z1.x + z2.x), R(0.5) * (z1.y + z2.y)};
    if (2 * k + 1 < 9) {
      // B = (z1 - conj(z_-k)) / (2i)
      const R dx = R(0.5) * (z1.x - z2.x), dy = R(0.5) * (z1.y - z2.y);
      P.spec[(size_t)(2 * k + 1) * ss + o] = {dy, -dx};
    }
  }
  if (SRC == SRC_CGPX) zfwd_step_length<R>(P, pkp, blockIdx.x, gridDim.x);
}

// Complex DFT along y (forward or inverse) on tiles of (grp component-x
// rows) x ny x (T consecutive kz); the tile is fetched with cp.async and the
// stages ping-pong between two shared buffers.
template <typename R, bool INV>
__global__ void FFT_BOUNDS(R) k_fft_y(const LineParams<R> P) {
  if (P.done && *P.done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int ny = P.g.ny, T = P.t, grp = P.grp;
  const int ts = __ffs(T) - 1;  // T is a power of two
  const int tile_elems = grp * ny * T;
  cplx<R>* tw = reinterpret_cast<cplx<R>*>(smem_raw);
  cplx<R>* bufA = tw + ((ny + 1) & ~1);  // 16-byte aligned
  cplx<R>* bufB = bufA + tile_elems;
  const int hz = P.g.hz, hzp = P.g.hzp;
  const int ngroups = 9 * P.g.nx;
  const int ntk = (hz + T - 1) >> ts;
  const FastDiv dntk = sizeof(R) == 4 ? P.g.f_ntky_f : P.g.f_ntky_d;
  const int tile = blockIdx.x;
  const int tg = (int)dntk.div((unsigned)tile);
  const int k0 = (tile - tg * ntk) * T, g0 = tg * grp;
  const int ng = min(grp, ngroups - g0);
  cplx<R>* gbase = P.spec + (size_t)g0 * ny * hzp + k0;
  issue_tile<R>(bufA, gbase, (size_t)hzp, ng * ny, T, ts, k0, hzp, P.spec);
  cp_async_commit();
  for (int i = threadIdx.x; i < ny; i += blockDim.x) tw[i] = P.tw[i];
  __shared__ AxisPlan plan;
  load_plan(&plan, axis_plan<R>(P.g, 1));
  cp_async_wait<0>();
  __syncthreads();
  const LineMap lm{ts, ny * T, 1, T, 1};
  const FastDiv fL = sizeof(R) == 4 ? P.g.f_Ly_f : P.g.f_Ly_d;
  const cplx<R>* res = fft_lines<R, INV>(bufA, bufB, lm, grp * T, fL, plan, tw);
  const int tc = min(T, hz - k0);
  const int tot = ng * ny * T;
  for (int i = threadIdx.x; i < tot; i += blockDim.x) {
    const int t = i & (T - 1);
    if (t < tc) gbase[(size_t)(i >> ts) * hzp + t] = res[i];
  }
}

// Forward DFT along x, projection, inverse DFT along x.  The projection
// A_ij <- xi_j (sum_l xi_l A_il) / |xi|^2 (Eq. G_red) couples only the three
// components of one tensor row i, so a tile is (row i) x nx x (T kz) for one
// ky.
// 1/a: float reciprocal, or for float64 the Newton-Raphson iteration
// x <- x (2 - a x) from the float reciprocal (about 24 correct bits, doubled
// by each step; two steps, written with FMAs as e = 1 - a x, x <- x + x e),
// which avoids a float64 division per element on a part whose float64
// rate is 1/64 of its float32 rate.
RVE_DEV float recip(float a) { return 1.0f / a; }
RVE_DEV double recip(double a) {
  double x = (double)__frcp_rn((float)a);
  double e = fma(-a, x, 1.0);
  x = fma(x, e, x);
  e = fma(-a, x, 1.0);
  return fma(x, e, x);
}

template <typename R>
__global__ void FFT_BOUNDS(R) k_fft_x_proj(const LineParams<R> P) {
  if (P.done && *P.done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nx = P.g.nx, ny = P.g.ny, T = P.t;
  const int ts = __ffs(T) - 1;
  const int tile_elems = 3 * nx * T;
  cplx<R>* tw = reinterpret_cast<cplx<R>*>(smem_raw);
  cplx<R>* bufA = tw + ((nx + 1) & ~1);
  cplx<R>* bufB = bufA + tile_elems;
  const int hz = P.g.hz, hzp = P.g.hzp;
  const int ntk = (hz + T - 1) >> ts;
  const FastDiv dntk = sizeof(R) == 4 ? P.g.f_ntkx_f : P.g.f_ntkx_d, dny = P.g.f_ny;
  const size_t rs = (size_t)ny * hzp;  // stride of spectrum rows (c*nx + x)
  // tile = (irow * ny + y) * ntk + tk
  const int tile = blockIdx.x;
  const int q = (int)dntk.div((unsigned)tile);
  const int k0 = (tile - q * ntk) * T;
  const int irow = (int)dny.div((unsigned)q);
  const int y = q - irow * ny;
  cplx<R>* gbase = P.spec + (size_t)(3 * irow) * nx * rs + (size_t)y * hzp + k0;
  issue_tile<R>(bufA, gbase, rs, 3 * nx, T, ts, k0, hzp, P.spec);
  cp_async_commit();
  for (int i = threadIdx.x; i < nx; i += blockDim.x) tw[i] = P.tw[i];
  __shared__ AxisPlan plan;
  load_plan(&plan, axis_plan<R>(P.g, 0));
  cp_async_wait<0>();
  __syncthreads();
  const LineMap lm{ts, nx * T, 1, T, 1};
  const FastDiv fL = sizeof(R) == 4 ? P.g.f_Lx_f : P.g.f_Lx_d;
  cplx<R>* X = fft_lines_call<R, false>(bufA, bufB, lm, 3 * T, fL, &plan, tw);
  cplx<R>* Y = (X == bufA) ? bufB : bufA;
  using RQ = typename std::conditional<is_dfl<R>::value, double, R>::type;
  const RQ qy_ = signed_freq<RQ>(y, ny) / (RQ)ny;
  const RQ sc_ = (RQ)P.scale;
  // Nyquist frequencies of even axes: G-hat = 0 there (Appendix C)
  const bool nyq_y = (ny % 2 == 0) && (2 * y == ny);
  // blockDim.x is a multiple of T: each thread keeps one t (one kz), so its
  // xi_z and z-Nyquist test once
  const int t0 = (int)(threadIdx.x & (T - 1));
  const RQ qz_ = (RQ)(k0 + t0) / (RQ)P.g.nz;
  const bool nyq_z = (P.g.nz % 2 == 0) && (2 * (k0 + t0) == P.g.nz);
  const RQ inv_nx = RQ(1) / (RQ)nx;
  for (int i = threadIdx.x; i < nx * T; i += blockDim.x) {
    const int x = i >> ts;
    // frequencies and 1/|xi|^2 in R (float-float: in float64, then split)
    const RQ qx_ = signed_freq<RQ>(x, nx) * inv_nx;
    const RQ q2 = qx_ * qx_ + qy_ * qy_ + qz_ * qz_;
    const bool nyq = nyq_y || nyq_z || ((nx % 2 == 0) && (2 * x == nx));
    const R f = R((q2 > RQ(0) && !nyq) ? sc_ * recip(q2) : RQ(0));
    const R qx = R(qx_), qy = R(qy_), qz = R(qz_);
    const cplx<R> A0 = X[i], A1 = X[nx * T + i], A2 = X[2 * nx * T + i];
    const R sx = f * (qx * A0.x + qy * A1.x + qz * A2.x);
    const R sy = f * (qx * A0.y + qy * A1.y + qz * A2.y);
    X[i] = {sx * qx, sy * qx};
    X[nx * T + i] = {sx, sy};
  }
  __syncthreads();
  // row j of the projected spectrum is s xi_j and xi_y, xi_z are constant
  // along an x line: components 1 and 2 are xi_y and xi_z times the inverse
  // transform of s -- two inverse transforms per tensor row instead of three
  FastDiv f2L;  // lines of two components: 2T, a power of two
  f2L.d = 2u * (unsigned)T;
  f2L.m = (1ull << 40) / f2L.d;
  const cplx<R>* res = fft_lines_call<R, true>(X, Y, lm, 2 * T, f2L, &plan, tw);
  const int tc = min(T, hz - k0);
  const int tot = 3 * nx * T;
  const R qy = R(qy_), qz = R(qz_);
  for (int i = threadIdx.x; i < tot; i += blockDim.x) {
    const int t = i & (T - 1);
    if (t >= tc) continue;
    const int row = i >> ts;  // component c of the row, times nx, plus x
    if (row < nx) {
      gbase[(size_t)row * rs + t] = res[i];
    } else {
      const int c2 = row >= 2 * nx;
      const cplx<R> u = res[i - c2 * nx * T];
      const R fq = c2 ? qz : qy;
      gbase[(size_t)row * rs + t] = {fq * u.x, fq * u.y};
    }
  }
}

template <typename R, typename RC, int OUT>
__global__ void FFT_BOUNDS(R) k_zinv(const ZinvParams<R, RC> P) {
  if (P.done && *P.done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nz = P.g.nz, lz = P.lz, hz = P.g.hz, hzp = P.g.hzp;
  cplx<R>* tw = reinterpret_cast<cplx<R>*>(smem_raw);
  cplx<R>* bufA = tw + ((nz + 1) & ~1);  // [5][lz][nz]
  cplx<R>* bufB = bufA + 5 * lz * nz;
  for (int i = threadIdx.x; i < nz; i += blockDim.x) tw[i] = P.tw[i];
  __shared__ AxisPlan plan;
  load_plan(&plan, axis_plan<R>(P.g, 2));
  const size_t n = P.g.n;
  const size_t ss = P.g.sstride;
  const int nlines = P.g.nx * P.g.ny;
  const int l0 = blockIdx.x * lz;
  const int nl = min(lz, nlines - l0);
  // rebuild the full z spectrum of the packed lines z = a + i b
  constexpr int U = sizeof(R) == 4 ? 4 : 2;  // (A, B) pairs in flight per thread
  const FastDiv dhz = P.g.f_hz, dlz = sizeof(R) == 4 ? P.g.f_lzf : P.g.f_lzd;
  const int nthr = blockDim.x;
  const int totl = 5 * lz * hz;
  for (int i0 = threadIdx.x; i0 < totl; i0 += U * nthr) {
    cplx<R> A[U], B[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = i0 + u * nthr;
      const int rest = (int)dhz.div((unsigned)i);
      const int kz = i - rest * hz;
      const int k = (int)dlz.div((unsigned)rest);
      const int li = rest - k * lz;
      A[u] = {R(0), R(0)};
      B[u] = {R(0), R(0)};
      if (i < totl && li < nl) {
        const size_t o = (size_t)(l0 + li) * hzp + kz;
        A[u] = P.spec[(size_t)(2 * k) * ss + o];
        if (2 * k + 1 < 9) B[u] = P.spec[(size_t)(2 * k + 1) * ss + o];
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = i0 + u * nthr;
      if (i >= totl) continue;
      const int rest = (int)dhz.div((unsigned)i);
      const int kz = i - rest * hz;
      const int k = (int)dlz.div((unsigned)rest);
      const int li = rest - k * lz;
      cplx<R>* line = bufA + (k * lz + li) * nz;
      line[kz] = {A[u].x - B[u].y, A[u].y + B[u].x};
      if (kz > 0) line[nz - kz] = {A[u].x + B[u].y, B[u].x - A[u].y};
    }
  }
  __syncthreads();
  const LineMap lm{30, 0, nz, 1, 0};
  const cplx<R>* res = fft_lines<R, true>(bufA, bufB, lm, 5 * lz, P.g.f_hz, plan, tw);
  const size_t v0 = (size_t)l0 * nz;
  double acc = 0.0;
  for (int i = threadIdx.x; i < nl * nz; i += blockDim.x) {
    R out[9];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      const cplx<R> z = res[k * lz * nz + i];
      out[2 * k] = z.x;
      if (2 * k + 1 < 9) out[2 * k + 1] = z.y;
    }
    const size_t v = v0 + i;
    if constexpr (OUT == OUT_PLAIN) {
      if constexpr (is_dfl<R>::value) {
#pragma unroll
        for (int c = 0; c < 9; ++c) P.dst64[(size_t)c * n + v] = (double)out[c];
      } else {
#pragma unroll
        for (int c = 0; c < 9; ++c) P.dst[(size_t)c * n + v] = out[c];
      }
    } else if constexpr (OUT == OUT_CGR) {
      const R alpha = (R)P.st->alpha;
      R rv[9];
#pragma unroll
      for (int c = 0; c < 9; ++c) rv[c] = (R)P.r_out[(size_t)c * n + v];
      R s = 0;
#pragma unroll
      for (int c = 0; c < 9; ++c) {
        rv[c] = fma(-alpha, out[c], rv[c]);
        P.r_out[(size_t)c * n + v] = (RC)rv[c];
        s = fma(rv[c], rv[c], s);
      }
      if constexpr (!is_dfl<R>::value)
        if (P.mn_ell >= 0.f) s = mnorm_k0<R>(rv, (R)P.mn_ell);
      acc += (double)s;
    } else if constexpr (OUT == OUT_CGAP) {
      R pv[9];
#pragma unroll
      for (int c = 0; c < 9; ++c) pv[c] = (R)P.p_in[(size_t)c * n + v];
      R s = 0;
#pragma unroll
      for (int c = 0; c < 9; ++c) {
        P.dst[(size_t)c * n + v] = out[c];
        s = fma(pv[c], out[c], s);
      }
      acc += (double)s;
    } else {
      R s = R(0);
#pragma unroll
      for (int c = 0; c < 9; ++c) {
        P.r_out[(size_t)c * n + v] = (RC)out[c];
        P.x_out[(size_t)c * n + v] = (RC)0;
        s = fma(out[c], out[c], s);
      }
      if constexpr (!is_dfl<R>::value)
        if (P.mn_ell >= 0.f) s = mnorm_k0<R>(out, (R)P.mn_ell);
      acc += (double)s;
    }
  }
  if (OUT == OUT_PLAIN) return;
  double v1[1] = {acc}, tot[1];
  const int slot = (OUT == OUT_CGAP) ? SLOT_PAP : (OUT == OUT_CGR ? SLOT_RR : SLOT_BB);
  if (last_block_sum<1>(v1, P.partials, &P.st->counter[slot], tot) && threadIdx.x == 0) {
    SolverState* st = P.st;
    if (OUT == OUT_CGR) {
      cg_after_rr(st, tot[0]);
    } else if (OUT == OUT_CGAP) {
      const double pap = tot[0];
      st->pAp = pap;
      if (!isfinite(pap)) {
        st->status = RVE_DEV_ERR_NONFINITE;
        st->done = 1;
      } else if (pap == 0.0) {
        // CG as in the library routine the method is written for: the sign
        // of p.Ap is not tested (the J2 tangent may be mildly indefinite);
        // only an exact zero stops it
        st->status = RVE_DEV_ERR_CG_BREAKDOWN;
        st->done = 1;
      } else {
        st->alpha = st->rr / pap;
      }
    } else {
      cg_after_bb(st, tot[0]);
    }
  }
}

// --------------------------------------------------------------------------
// launchers
// --------------------------------------------------------------------------
template <typename R>
static int lz_of(const GridGeom& g) { return sizeof(R) == 4 ? g.lz_f : g.lz_d; }

template <typename R>
void launch_zfwd(const GridGeom& g, int src, const TangentView<R>& tan, const R* field, const R* r,
                 R* p, const double* unif, SolverState* st, const int* done, cplx<R>* spec,
                 const Twiddles<R>& tw, cudaStream_t s, R* x, double* partials) {
  ZfwdParams<R> P{};
  P.g = g;
  P.lz = lz_of<R>(g);
  P.src = src;
  P.tan = tan;
  P.field = field;
  P.r = r;
  P.p = p;
  P.unif = unif;
  P.st = st;
  P.done = done;
  P.spec = spec;
  P.tw = tw.z;
  P.x = x;
  P.partials = partials;
  if (sizeof(R) == 4 && g.fsz_n1 && src == SRC_CGPX) {
    launch_zfwd4(reinterpret_cast<const ZfwdParams<float>&>(P), s);
    return;
  }
  const int nlines = g.nx * g.ny;
  const dim3 grid((nlines + P.lz - 1) / P.lz);
  const size_t sm = sizeof(cplx<R>) * ((size_t)((g.nz + 1) & ~1) + 10 * (size_t)P.lz * g.nz);
#define ZF(S, T) k_zfwd<R, S, T><<<grid, FFT_THREADS, sm, s>>>(P)
  const int tm = tan.mode;
  if (src == SRC_FIELD) {
    if (tm == TAN_FULL81) ZF(SRC_FIELD, TAN_FULL81);
    else if (tm == TAN_SYM45) ZF(SRC_FIELD, TAN_SYM45);
    else if (tm == TAN_SVK) ZF(SRC_FIELD, TAN_SVK);
    else ZF(SRC_FIELD, 0);
  } else if (src == SRC_CGP) {
    if (tm == TAN_FULL81) ZF(SRC_CGP, TAN_FULL81);
    else if (tm == TAN_SYM45) ZF(SRC_CGP, TAN_SYM45);
    else ZF(SRC_CGP, TAN_SVK);
  } else if (src == SRC_CGPX) {
    if (tm == TAN_FULL81) ZF(SRC_CGPX, TAN_FULL81);
    else if (tm == TAN_SYM45) ZF(SRC_CGPX, TAN_SYM45);
    else ZF(SRC_CGPX, TAN_SVK);
  } else {
    if (tm == TAN_FULL81) ZF(SRC_UNIFORM, TAN_FULL81);
    else if (tm == TAN_SYM45) ZF(SRC_UNIFORM, TAN_SYM45);
    else ZF(SRC_UNIFORM, TAN_SVK);
  }
#undef ZF
}

template <typename R>
void launch_fft_y(const GridGeom& g, bool inverse, cplx<R>* spec, const int* done,
                  const Twiddles<R>& tw, cudaStream_t s) {
  if (sizeof(R) == 4 && g.fsy_n1) {
    launch_fft_y4(g, inverse, reinterpret_cast<cplx<float>*>(spec), done,
                  reinterpret_cast<const cplx<float>*>(tw.y), s);
    return;
  }
  LineParams<R> P{};
  P.g = g;
  P.t = sizeof(R) == 4 ? g.ty_f : g.ty_d;
  P.grp = sizeof(R) == 4 ? g.gy_f : g.gy_d;
  P.scale = 1.0;
  P.spec = spec;
  P.done = done;
  P.tw = tw.y;
  const int ntiles = ((g.hz + P.t - 1) / P.t) * ((9 * g.nx + P.grp - 1) / P.grp);
  const size_t sm = sizeof(cplx<R>) * ((size_t)((g.ny + 1) & ~1) + 2 * (size_t)P.grp * g.ny * P.t);
  if (inverse) k_fft_y<R, true><<<ntiles, FFT_THREADS, sm, s>>>(P);
  else k_fft_y<R, false><<<ntiles, FFT_THREADS, sm, s>>>(P);
}

template <typename R>
void launch_fft_x_proj(const GridGeom& g, double scale, cplx<R>* spec, const int* done,
                       const Twiddles<R>& tw, cudaStream_t s, bool gamma0) {
  if (sizeof(R) == 4 && (g.fsx_n1 || gamma0)) {
    launch_fft_x4(g, scale, reinterpret_cast<cplx<float>*>(spec), done,
                  reinterpret_cast<const cplx<float>*>(tw.x), s, gamma0);
    return;
  }
  LineParams<R> P{};
  P.g = g;
  P.t = sizeof(R) == 4 ? g.tx_f : g.tx_d;
  P.grp = 1;
  P.scale = scale;
  P.spec = spec;
  P.done = done;
  P.tw = tw.x;
  const int ntiles = 3 * g.ny * ((g.hz + P.t - 1) / P.t);
  const size_t sm = sizeof(cplx<R>) * ((size_t)((g.nx + 1) & ~1) + 2 * 3 * (size_t)g.nx * P.t);
  k_fft_x_proj<R><<<ntiles, FFT_THREADS, sm, s>>>(P);
}

template <typename R, typename RC>
void launch_zinv(const GridGeom& g, int out, const cplx<R>* spec, R* dst, RC* r_out, RC* x_out,
                 const RC* p_in, SolverState* st, double* partials, const int* done,
                 const Twiddles<R>& tw, cudaStream_t s, bool mnorm) {
  ZinvParams<R, RC> P{};
  P.g = g;
  P.mn_ell = mnorm ? g.pc_ell : -1.f;
  P.lz = lz_of<R>(g);
  P.spec = spec;
  P.dst = dst;
  P.r_out = r_out;
  P.x_out = x_out;
  P.p_in = p_in;
  P.st = st;
  P.partials = partials;
  P.done = done;
  P.tw = tw.z;
  if (sizeof(R) == 4 && sizeof(RC) == 4 && g.fsz_n1 && out == OUT_CGR) {
    launch_zinv4(reinterpret_cast<const ZinvParams<float, float>&>(P), s);
    return;
  }
  const int nlines = g.nx * g.ny;
  const dim3 grid((nlines + P.lz - 1) / P.lz);
  const size_t sm = sizeof(cplx<R>) * ((size_t)((g.nz + 1) & ~1) + 10 * (size_t)P.lz * g.nz);
  if (out == OUT_PLAIN) k_zinv<R, RC, OUT_PLAIN><<<grid, FFT_THREADS, sm, s>>>(P);
  else if (out == OUT_CGAP) k_zinv<R, RC, OUT_CGAP><<<grid, FFT_THREADS, sm, s>>>(P);
  else if (out == OUT_CGR) k_zinv<R, RC, OUT_CGR><<<grid, FFT_THREADS, sm, s>>>(P);
  else k_zinv<R, RC, OUT_RESID><<<grid, FFT_THREADS, sm, s>>>(P);
}

size_t fft_max_blocks(const GridGeom& g) {
  const size_t nlines = (size_t)g.nx * g.ny;
  int lz = g.lz_f < g.lz_d ? g.lz_f : g.lz_d;
  if (g.fsz_n1 && g.fsz_lz < lz) lz = g.fsz_lz;
  if (g.fsz_n1 && fs_zt_lz(g.nz) >= 1 && fs_zt_lz(g.nz) < lz) lz = fs_zt_lz(g.nz);
  return (nlines + lz - 1) / lz;
}

// Dynamic shared memory of these kernels stays below 200 KB (checked when the
// grid geometry is built); the opt-in limit leaves room for static shared
// memory (reduction scratch) within the 227 KB per block.
// g_init_err is shared by every caller of fft_kernels_init, which holds
// g_init_mu for the whole set-up so that host threads creating handles and
// the allocation-free entry point can set it up at the same time.
static cudaError_t g_init_err = cudaSuccess;
static std::mutex g_init_mu;

template <typename K>
static void allow_big_smem(K kernel) {
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 208 * 1024);
  if (e != cudaSuccess && g_init_err == cudaSuccess) g_init_err = e;
}

template <typename R>
static void init_r() {
  allow_big_smem(k_zfwd<R, SRC_FIELD, TAN_FULL81>);
  allow_big_smem(k_zfwd<R, SRC_FIELD, TAN_SVK>);
  allow_big_smem(k_zfwd<R, SRC_FIELD, 0>);
  allow_big_smem(k_zfwd<R, SRC_CGP, TAN_FULL81>);
  allow_big_smem(k_zfwd<R, SRC_CGP, TAN_SVK>);
  allow_big_smem(k_zfwd<R, SRC_CGPX, TAN_FULL81>);
  allow_big_smem(k_zfwd<R, SRC_CGPX, TAN_SVK>);
  allow_big_smem(k_zfwd<R, SRC_UNIFORM, TAN_FULL81>);
  allow_big_smem(k_zfwd<R, SRC_UNIFORM, TAN_SVK>);
  allow_big_smem(k_zfwd<R, SRC_FIELD, TAN_SYM45>);
  allow_big_smem(k_zfwd<R, SRC_CGP, TAN_SYM45>);
  allow_big_smem(k_zfwd<R, SRC_CGPX, TAN_SYM45>);
  allow_big_smem(k_zfwd<R, SRC_UNIFORM, TAN_SYM45>);
  allow_big_smem(k_fft_y<R, true>);
  allow_big_smem(k_fft_y<R, false>);
  allow_big_smem(k_fft_x_proj<R>);
}

bool launch_G_df(const GridGeom& g, const double* in, double scale, int out_mode, double* out64,
                 float* r_out, float* x_out, SolverState* st, double* partials, cplx<dfl>* spec,
                 const Twiddles<dfl>& tw, cudaStream_t s) {
  const int nlines = g.nx * g.ny;
  const int lz = g.lz_d;
  const dim3 grid((nlines + lz - 1) / lz);
  const size_t smz = sizeof(cplx<dfl>) * ((size_t)((g.nz + 1) & ~1) + 10 * (size_t)lz * g.nz);
  // four-step kernels where the axis length has a compiled split, the
  // Stockham engine otherwise
  if (!launch_zfwd4_df(g, in, spec, tw.z, s)) {
    ZfwdParams<dfl> P{};
    P.g = g;
    P.lz = lz;
    P.src = SRC_FIELD;
    P.field64 = in;
    P.st = st;
    P.spec = spec;
    P.tw = tw.z;
    k_zfwd<dfl, SRC_FIELD, 0><<<grid, FFT_THREADS, smz, s>>>(P);
  }
  if (!launch_fft_y4_df(g, false, spec, tw.y, s)) launch_fft_y<dfl>(g, false, spec, nullptr, tw, s);
  if (!launch_fft_x4_df(g, scale, spec, tw.x, s)) launch_fft_x_proj<dfl>(g, scale, spec, nullptr, tw, s);
  if (!launch_fft_y4_df(g, true, spec, tw.y, s)) launch_fft_y<dfl>(g, true, spec, nullptr, tw, s);
  if (launch_zinv4_df(g, out_mode, spec, out64, r_out, x_out, st, partials, tw.z, s))
    return out_mode == OUT_PLAIN_MEANX;
  if (out_mode != OUT_RESID) {
    ZinvParams<dfl, double> P{};
    P.g = g;
    P.lz = lz;
    P.spec = spec;
    P.dst64 = out64;
    P.st = st;
    P.partials = partials;
    P.tw = tw.z;
    k_zinv<dfl, double, OUT_PLAIN><<<grid, FFT_THREADS, smz, s>>>(P);
  } else {
    ZinvParams<dfl, float> P{};
    P.g = g;
    P.lz = lz;
    P.spec = spec;
    P.r_out = r_out;
    P.x_out = x_out;
    P.st = st;
    P.partials = partials;
    P.tw = tw.z;
    k_zinv<dfl, float, OUT_RESID><<<grid, FFT_THREADS, smz, s>>>(P);
  }
  return false;
}

cudaError_t fft_kernels_init() {
  std::lock_guard<std::mutex> lock(g_init_mu);
  g_init_err = cudaSuccess;
  init_r<float>();
  init_r<double>();
  allow_big_smem(k_zinv<double, double, OUT_PLAIN>);
  allow_big_smem(k_zinv<double, double, OUT_CGAP>);
  allow_big_smem(k_zinv<double, double, OUT_RESID>);
  allow_big_smem(k_zinv<double, float, OUT_RESID>);
  allow_big_smem(k_zinv<float, float, OUT_PLAIN>);
  allow_big_smem(k_zinv<float, float, OUT_CGAP>);
  allow_big_smem(k_zinv<float, float, OUT_CGR>);
  allow_big_smem(k_zinv<double, double, OUT_CGR>);
  allow_big_smem(k_zinv<float, float, OUT_RESID>);
  allow_big_smem(k_zfwd<dfl, SRC_FIELD, 0>);
  allow_big_smem(k_fft_y<dfl, true>);
  allow_big_smem(k_fft_y<dfl, false>);
  allow_big_smem(k_fft_x_proj<dfl>);
  allow_big_smem(k_zinv<dfl, double, OUT_PLAIN>);
  allow_big_smem(k_zinv<dfl, float, OUT_RESID>);
  if (g_init_err == cudaSuccess) g_init_err = fft4_kernels_init();
  return g_init_err;
}

// Column of the homogenised tangent: < K : (U + x) > over the voxels, the
// tangent applied exactly as in the first z pass (same storage modes), the
// sums in float64 with the deterministic last-block reduction.
template <typename R, int TAN>
__global__ void __launch_bounds__(256) k_tangent_mean(TangentView<R> T, const R* __restrict__ x,
                                                      const double* __restrict__ U, size_t n,
                                                      double* out9, double* partials,
                                                      unsigned int* counter) {
  double s[9];
  R u[9];
#pragma unroll
  for (int c = 0; c < 9; ++c) {
    s[c] = 0.0;
    u[c] = (R)U[c];
  }
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
    TanPre<R> q;
    tangent_pre<R, TAN>(T, v, n, q);
    R in[9], out[9];
#pragma unroll
    for (int c = 0; c < 9; ++c) in[c] = x ? u[c] + x[(size_t)c * n + v] : u[c];
    tangent_post<R, TAN>(T, v, n, q, in, out);
#pragma unroll
    for (int c = 0; c < 9; ++c) s[c] += (double)out[c];
  }
  double tot[9];
  if (last_block_sum<9>(s, partials, counter, tot) && threadIdx.x == 0)
#pragma unroll
    for (int c = 0; c < 9; ++c) out9[c] = tot[c] / (double)n;
}

template <typename R>
void launch_tangent_mean(const TangentView<R>& tan, const R* x, const double* U, size_t n,
                         double* out9, double* partials, unsigned int* counter, cudaStream_t s) {
  const size_t blocks = std::min<size_t>((n + 255) / 256, vec_max_blocks());
  const dim3 grid((unsigned)std::max<size_t>(blocks, 1));
  if (tan.mode == TAN_FULL81)
    k_tangent_mean<R, TAN_FULL81><<<grid, 256, 0, s>>>(tan, x, U, n, out9, partials, counter);
  else if (tan.mode == TAN_SYM45)
    k_tangent_mean<R, TAN_SYM45><<<grid, 256, 0, s>>>(tan, x, U, n, out9, partials, counter);
  else
    k_tangent_mean<R, TAN_SVK><<<grid, 256, 0, s>>>(tan, x, U, n, out9, partials, counter);
}

// explicit instantiations
template void launch_tangent_mean<float>(const TangentView<float>&, const float*, const double*,
                                         size_t, double*, double*, unsigned int*, cudaStream_t);
template void launch_tangent_mean<double>(const TangentView<double>&, const double*,
                                          const double*, size_t, double*, double*, unsigned int*,
                                          cudaStream_t);
template void launch_zfwd<float>(const GridGeom&, int, const TangentView<float>&, const float*,
                                 const float*, float*, const double*, SolverState*, const int*,
                                 cplx<float>*, const Twiddles<float>&, cudaStream_t, float*,
                                 double*);
template void launch_zfwd<double>(const GridGeom&, int, const TangentView<double>&, const double*,
                                  const double*, double*, const double*, SolverState*, const int*,
                                  cplx<double>*, const Twiddles<double>&, cudaStream_t, double*,
                                  double*);
template void launch_fft_y<float>(const GridGeom&, bool, cplx<float>*, const int*,
                                  const Twiddles<float>&, cudaStream_t);
template void launch_fft_y<double>(const GridGeom&, bool, cplx<double>*, const int*,
                                   const Twiddles<double>&, cudaStream_t);
template void launch_fft_x_proj<float>(const GridGeom&, double, cplx<float>*, const int*,
                                       const Twiddles<float>&, cudaStream_t, bool);
template void launch_fft_x_proj<double>(const GridGeom&, double, cplx<double>*, const int*,
                                        const Twiddles<double>&, cudaStream_t, bool);
template void launch_zinv<double, double>(const GridGeom&, int, const cplx<double>*, double*,
                                          double*, double*, const double*, SolverState*, double*,
                                          const int*, const Twiddles<double>&, cudaStream_t, bool);
template void launch_zinv<double, float>(const GridGeom&, int, const cplx<double>*, double*,
                                         float*, float*, const float*, SolverState*, double*,
                                         const int*, const Twiddles<double>&, cudaStream_t, bool);
template void launch_zinv<float, float>(const GridGeom&, int, const cplx<float>*, float*, float*,
                                        float*, const float*, SolverState*, double*, const int*,
                                        const Twiddles<float>&, cudaStream_t, bool);
template void launch_fft_y<dfl>(const GridGeom&, bool, cplx<dfl>*, const int*,
                                const Twiddles<dfl>&, cudaStream_t);
template void launch_fft_x_proj<dfl>(const GridGeom&, double, cplx<dfl>*, const int*,
                                     const Twiddles<dfl>&, cudaStream_t, bool);
