// Float y and x passes on the in-place four-step line DFT (fs_lines) for
// axis lengths with a compiled split N = N1 N2 (RVE_FS_SIZES).  Same data
// flow as k_fft_y / k_fft_x_proj: a tile of 128-byte spectrum rows (16 kz
// values) is fetched with cp.async into ONE shared buffer, transformed in
// place and written back; the transposed order the forward transform leaves
// is undone in the addressing of the global stores (forward y), loads
// (inverse y) or of the projection (x pass).
#include <algorithm>
#include <vector>

#include "fft_pass.cuh"

namespace {

// three CTAs per SM when both factors fit the register budget
template <typename R, int N1, int N2>
struct Fs4Occ {
  static constexpr int value = (sizeof(R) == 4 && N1 <= 27 && N2 <= 27) ? 3 : 2;
};

// Complex DFT along y on tiles of (GRP component-x rows) x ny x (T kz),
// T and GRP compile-time (fs_y_t, fs_y_grp).  The last phase writes its
// values straight to global memory (forward: phase A then B; inverse: B
// then A), and the inverse's first phase reads them straight from global
// memory (N2 = 25 loads per thread in flight), so the transposed
// intermediate order never leaves shared memory.
template <typename R, int N1, int N2, bool INV, int T>
RVE_DEV void fft_y4_tile(const LineParams<R>& P, const int tile) {
  constexpr int N = N1 * N2;
  constexpr int GRP = fs_y_grp(N);
  using LM = FsLayout<T, N * T, 1, T, GRP * T>;
  if (P.done && *P.done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<R>* tw2 = reinterpret_cast<cplx<R>*>(smem_raw);
  cplx<R>* buf = tw2 + ((N + 1) & ~1);
  const int hz = P.g.hz, hzp = P.g.hzp;  // kz extent (z axis), not this axis
  const int ngroups = 9 * P.g.nx;
  const int ntk = (hz + T - 1) / T;
  // the float-float tiles have their own height: plain division there
  const int tg = is_dfl<R>::value ? tile / ntk : (int)P.g.f_fsy_ntk.div((unsigned)tile);
  const int k0 = (tile - tg * ntk) * T, g0 = tg * GRP;
  const int ng = min(GRP, ngroups - g0);
  cplx<R>* gbase = P.spec + (size_t)g0 * N * hzp + k0;
  // line l = (group l / T, kz k0 + l % T): rows y at stride hzp
  auto gl = [&](int l) {
    const int gi = l / T, t = l - (l / T) * T;
    return GLine<R>{gbase + (size_t)gi * N * hzp + t, (size_t)hzp, gi < ng && k0 + t < hz,
                    gi < ng && k0 + t < hz};
  };
  if (!INV) {
    // forward: the whole tile by cp.async first (phase A alone would keep
    // only N1 loads in flight per thread), phase A in place, phase B to global
    constexpr int EPC = 16 / sizeof(cplx<R>);
    constexpr int CPR = T / EPC;  // 16-byte chunks per row
    const int nch = ng * N * CPR;
    for (int c = threadIdx.x; c < nch; c += FFT_THREADS) {
      const int row = c / CPR;
      const int t = (c - row * CPR) * EPC;
      const bool ok = (k0 + t) < hzp;
      const cplx<R>* src = ok ? gbase + (size_t)row * hzp + t : P.spec;
      cp_async16(buf + row * T + t, src, ok ? 16 : 0);
    }
    cp_async_commit();
    fs_twiddles<R, N1, N2>(tw2, P.tw);
    cp_async_wait<0>();
    __syncthreads();
    fs_phase_a<R, N1, N2, false, LM>(buf, tw2);
    __syncthreads();
    fs_phase_b_s2g<R, N1, N2, LM>(buf, gl);
  } else {
    fs_twiddles<R, N1, N2>(tw2, P.tw);
    __syncthreads();
    fs_phase_b_g2s<R, N1, N2, LM>(buf, gl);
    __syncthreads();
    fs_phase_a_s2g<R, N1, N2, LM>(buf, tw2, gl);
  }
}

template <typename R, int N1, int N2, bool INV, int T>
__global__ void __launch_bounds__(FFT_THREADS, (Fs4Occ<R, N1, N2>::value) + (N1 * N2 <= 125 ? 1 : 0))
    k_fft_y4(const LineParams<R> P) {
  fft_y4_tile<R, N1, N2, INV, T>(P, blockIdx.x);
}

// k / n in the pass's arithmetic.  Float: the rounded quotient.
// Float-float: the rounded quotient h plus the rounded quotient of the
// remainder k - h n, which one fma gives exactly (the remainder of a
// correctly rounded division is representable).
template <typename R>
RVE_DEV R fs_ratio(int k, int n);
template <>
RVE_DEV float fs_ratio<float>(int k, int n) {
  return (float)k / (float)n;
}
template <>
RVE_DEV dfl fs_ratio<dfl>(int k, int n) {
  const float kf = (float)k, nf = (float)n;
  const float h = __fdiv_rn(kf, nf);
  return fast_two_sum(h, __fdiv_rn(fmaf(-h, nf, kf), nf));
}

RVE_DEV bool fs_positive(float a) { return a > 0.0f; }
RVE_DEV bool fs_positive(dfl a) { return a.hi > 0.0f; }

// 1 / a.  Float: the correctly rounded reciprocal.  Float-float: one Newton
// step from it, r = r0 + r0 e with e = 1 - a r0 formed from the exact
// product a.hi r0 = p + pe (fma) -- 1 - p is exact since p is within an
// ulp of 1 -- so the relative error is of order e^2 ~ 2^-48.
RVE_DEV float fs_rcp(float a) { return __frcp_rn(a); }
RVE_DEV dfl fs_rcp(dfl a) {
  const float r0 = __frcp_rn(a.hi);
  const float p = a.hi * r0;
  const float pe = fmaf(a.hi, r0, -p);
  const float e = ((1.0f - p) - pe) - a.lo * r0;
  return fast_two_sum(r0, r0 * e);
}

// Forward DFT along x, projection A_ij <- xi_j (sum_l xi_l A_il) / |xi|^2
// (Eq. G_red) in the transposed order, inverse DFT along x; tile = (tensor
// row i) x nx x (T kz) for one ky, T compile-time (fs_x_t).
template <typename R, int N1, int N2, int T>
RVE_DEV void fft_x4_tile(const LineParams<R>& P, const int tile) {
  constexpr int N = N1 * N2;
  using LM = FsLayout<T, N * T, 1, T, 3 * T>;
  if (P.done && *P.done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<R>* tw2 = reinterpret_cast<cplx<R>*>(smem_raw);
  cplx<R>* buf = tw2 + ((N + 1) & ~1);
  const int ny = P.g.ny;
  const int hz = P.g.hz, hzp = P.g.hzp;
  const int ntk = (hz + T - 1) / T;
  const size_t rs = (size_t)ny * hzp;  // stride of spectrum rows (c*nx + x)
  const int q = (int)P.g.f_fsx_ntk.div((unsigned)tile);
  const int k0 = (tile - q * ntk) * T;
  const int irow = (int)P.g.f_ny.div((unsigned)q);
  const int y = q - irow * ny;
  cplx<R>* gbase = P.spec + (size_t)(3 * irow) * N * rs + (size_t)y * hzp + k0;
  // line l = (component l / T of the row, kz k0 + l % T): rows x at stride rs
  auto gl = [&](int l) {
    const int c = l / T, t = l - (l / T) * T;
    return GLine<R>{gbase + (size_t)c * N * rs + t, rs, k0 + t < hz, k0 + t < hz};
  };
  fs_twiddles<R, N1, N2>(tw2, P.tw);
  __syncthreads();
  fs_phase_a_g2s<R, N1, N2, LM, decltype(gl), false>(buf, tw2, gl);
  __syncthreads();
  fs_phase_b<R, N1, N2, false, LM, false>(buf);
  const R qy = fs_ratio<R>(signed_freq<int>(y, ny), ny);
  const R sc = (R)P.scale;
  // xi_x of each transposed position and xi_z of each kz of the tile
  R* qxs = reinterpret_cast<R*>(buf + 3 * N * T);  // [N]
  R* qzs = qxs + N;                                // [T]
  for (int i = threadIdx.x; i < N + T; i += FFT_THREADS) {
    if (i < N) qxs[i] = fs_ratio<R>(signed_freq<int>(fs_freq<N1, N2>(i), N), N);
    else qzs[i - N] = fs_ratio<R>(k0 + i - N, P.g.nz);
  }
  __syncthreads();
  // Nyquist frequencies of even y / z axes: G-hat = 0 there (Appendix C;
  // this kernel's x length is odd)
  const bool nyq_y = (ny % 2 == 0) && (2 * y == ny);
  const int kz_nyq = (P.g.nz % 2 == 0) ? P.g.nz / 2 : -1;
  for (int i = threadIdx.x; i < N * T; i += FFT_THREADS) {
    const R qx = qxs[i / T];
    const R qz = qzs[i % T];
    const R q2 = qx * qx + qy * qy + qz * qz;
    const bool nyq = nyq_y || (k0 + i % T == kz_nyq);
    const R f = (fs_positive(q2) && !nyq) ? sc * fs_rcp(q2) : R(0);
    const cplx<R> A0 = buf[i], A1 = buf[N * T + i], A2 = buf[2 * N * T + i];
    const R sx = f * (qx * A0.x + qy * A1.x + qz * A2.x);
    const R sy = f * (qx * A0.y + qy * A1.y + qz * A2.y);
    buf[i] = {sx * qx, sy * qx};
    buf[N * T + i] = {sx, sy};
  }
  __syncthreads();
  // Row j of the projected tensor is s xi_j with s = xi.A_i / |xi|^2, and
  // xi_y, xi_z are constant along an x line: the inverse x transforms of
  // components 1 and 2 are xi_y and xi_z times the one of s.  Two inverse
  // transforms per tensor row instead of three.
  using LM2 = FsLayout<T, N * T, 1, T, 2 * T>;
  fs_phase_b<R, N1, N2, true, LM2, false>(buf);
  __syncthreads();
  constexpr int total = 2 * T * N2;
  for (int i = threadIdx.x; i < total; i += FFT_THREADS) {
    const int n2 = i / (2 * T);
    const int l = i - n2 * (2 * T);
    const cplx<R>* line = buf + LM2::base(l) + n2 * LM2::ES;
    cplx<R> v[N1];
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) v[k1] = line[k1 * N2 * LM2::ES];
    if (n2 != 0) {
      const cplx<R>* w = tw2 + n2 * N1;
#pragma unroll
      for (int k1 = 1; k1 < N1; ++k1) v[k1] = c_mulc(v[k1], w[k1]);
    }
    dft_reg<R, N1, true, false>(v);
    const int t = l % T;
    if (k0 + t < hz) {
      if (l < T) {
        cplx<R>* g = gbase + t;
#pragma unroll
        for (int m = 0; m < N1; ++m) g[(size_t)(N2 * m + n2) * rs] = v[m];
      } else {
        const R qz = qzs[t];
        cplx<R>* g1 = gbase + (size_t)N * rs + t;
        cplx<R>* g2 = gbase + (size_t)(2 * N) * rs + t;
#pragma unroll
        for (int m = 0; m < N1; ++m) {
          g1[(size_t)(N2 * m + n2) * rs] = {qy * v[m].x, qy * v[m].y};
          g2[(size_t)(N2 * m + n2) * rs] = {qz * v[m].x, qz * v[m].y};
        }
      }
    }
  }
}

template <typename R, int N1, int N2, int T>
__global__ void __launch_bounds__(FFT_THREADS, (Fs4Occ<R, N1, N2>::value))
    k_fft_x4(const LineParams<R> P) {
  fft_x4_tile<R, N1, N2, T>(P, blockIdx.x);
}

// The y and x passes of G in float-float arithmetic (the float64-accurate
// residual and projection of the mixed solver): the same tiles with 16-byte
// complex values, two blocks per SM for the registers that the N2-point
// float-float DFTs hold.  T = 16 kz per tile where the tile fits 100 KB
// (x pass: 8 or 4 beyond), so that the N2-point DFTs of the second phase
// still give most of the 256 threads a line (tile lines x N1 items).
constexpr int fs_y_t_df() { return 16; }
constexpr int fs_x_t_df(int n) {
  return 16 * 2 * n * 16 <= 102400 ? 16 : (16 * 2 * n * 8 <= 102400 ? 8 : 4);
}
// z lines per tile of the float-float z passes: the most whose five packed
// lines fit 104 KB (two blocks per SM)
constexpr int fs_zd_lz(int n) {
  int best = 1;
  for (int lz = 1; lz <= 64; ++lz)
    if (16 * ((size_t)((n + 1) & ~1) + (size_t)n * ((5 * lz) | 1)) <= 104 * 1024) best = lz;
  return best;
}

template <int N1, int N2, bool INV>
__global__ void __launch_bounds__(FFT_THREADS, 2) k_fft_y4_df(const LineParams<dfl> P) {
  fft_y4_tile<dfl, N1, N2, INV, fs_y_t_df()>(P, blockIdx.x);
}

// Phase B of the float-float x pass with its N2-point DFTs split once more
// where N2 is composite, N2 = Na Nb (Na its smallest factor), through the
// shared buffer: sub-phase 1 runs Na-point DFTs on stride Nb within each
// N2 block, times w_N2^(b ka) (twb[m] = w_N2^m), sub-phase 2 Nb-point DFTs on
// its contiguous runs, leaving frequency ka + Na kb of the block at position
// Nb ka + kb (fs_freq_df).  A float-float N2-point DFT is long, and the x
// tile's 2T lines give only 2T N1 of them (160 for 256 threads at 125);
// the sub-phases give 2T N1 Nb and 2T N1 Na short ones.  The inverse runs
// the conjugate steps in reverse order.
template <int N1, int N2>
RVE_DEV int fs_freq_df(int p) {
  constexpr int Na = smallest_factor(N2), Nb = N2 / Na;
  if constexpr (Na == N2) {
    return fs_freq<N1, N2>(p);
  } else {
    const int s = p % N2;
    return p / N2 + N1 * (s / Nb + Na * (s % Nb));
  }
}

template <int N1, int N2, bool INV, typename LM>
RVE_DEV void df_phase_b(cplx<dfl>* buf, const cplx<dfl>* twb) {
  using R = dfl;
  constexpr int Na = smallest_factor(N2), Nb = N2 / Na;
  if constexpr (Na == N2) {
    fs_phase_b<R, N1, N2, INV, LM>(buf);
  } else {
    constexpr int tot1 = LM::L * N1 * Nb, tot2 = LM::L * N1 * Na;
    auto sub1 = [&]() {  // items (line, k1, b): positions Nb a + b of the block
      for (int i = threadIdx.x; i < tot1; i += FFT_THREADS) {
        const int l = i % LM::L, r = i / LM::L;
        const int b = r % Nb, k1 = r / Nb;
        cplx<R>* line = buf + LM::base(l) + (N2 * k1 + b) * LM::ES;
        cplx<R> t[Na];
#pragma unroll
        for (int a = 0; a < Na; ++a) t[a] = line[Nb * a * LM::ES];
        if (INV && b != 0) {
#pragma unroll
          for (int ka = 1; ka < Na; ++ka) t[ka] = c_mulc(t[ka], twb[b * ka]);
        }
        dft_reg<R, Na, INV>(t);
        if (!INV && b != 0) {
#pragma unroll
          for (int ka = 1; ka < Na; ++ka) t[ka] = c_mul(t[ka], twb[b * ka]);
        }
#pragma unroll
        for (int a = 0; a < Na; ++a) line[Nb * a * LM::ES] = t[a];
      }
    };
    auto sub2 = [&]() {  // items (line, k1, ka): positions Nb ka + kb of the block
      for (int i = threadIdx.x; i < tot2; i += FFT_THREADS) {
        const int l = i % LM::L, r = i / LM::L;
        const int ka = r % Na, k1 = r / Na;
        cplx<R>* line = buf + LM::base(l) + (N2 * k1 + Nb * ka) * LM::ES;
        cplx<R> u[Nb];
#pragma unroll
        for (int b = 0; b < Nb; ++b) u[b] = line[b * LM::ES];
        dft_reg<R, Nb, INV>(u);
#pragma unroll
        for (int b = 0; b < Nb; ++b) line[b * LM::ES] = u[b];
      }
    };
    if (!INV) {
      sub1();
      __syncthreads();
      sub2();
    } else {
      sub2();
      __syncthreads();
      sub1();
    }
  }
}

// x pass of G in float-float.  xi_y and xi_z are constant along an x line,
// so the sum over l of xi_l A^_il needs only two forward transforms per
// tensor row: A_i0 and B_i = xi_y A_i1 + xi_z A_i2, formed while the tile
// is loaded (xi . A^_i = xi_x A^_i0 + B^_i); with the two inverse
// transforms of the projection, four line DFTs per row instead of five --
// the DFTs being most of this pass's float-float arithmetic.
template <int N1, int N2, int T>
RVE_DEV void fft_x4_df_tile(const LineParams<dfl>& P, const int tile) {
  using R = dfl;
  constexpr int N = N1 * N2;
  using LM = FsLayout<T, N * T, 1, T, 2 * T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<R>* tw2 = reinterpret_cast<cplx<R>*>(smem_raw);
  cplx<R>* buf = tw2 + ((N + 1) & ~1);
  R* qxs = reinterpret_cast<R*>(buf + 2 * N * T);  // [N]
  R* qzs = qxs + N;                                // [T]
  // w_N2^m, after qzs rounded to 16 bytes
  cplx<R>* twb = reinterpret_cast<cplx<R>*>(qzs + T + ((N + T) & 1));
  const int ny = P.g.ny;
  const int hz = P.g.hz, hzp = P.g.hzp;
  const int ntk = (hz + T - 1) / T;
  const size_t rs = (size_t)ny * hzp;  // stride of spectrum rows (c*nx + x)
  const int q = tile / ntk;
  const int k0 = (tile - q * ntk) * T;
  const int irow = (int)P.g.f_ny.div((unsigned)q);
  const int y = q - irow * ny;
  cplx<R>* gbase = P.spec + (size_t)(3 * irow) * N * rs + (size_t)y * hzp + k0;
  const R qy = fs_ratio<R>(signed_freq<int>(y, ny), ny);
  fs_twiddles<R, N1, N2>(tw2, P.tw);
  for (int i = threadIdx.x; i < N + T + N2; i += FFT_THREADS) {
    if (i < N) qxs[i] = fs_ratio<R>(signed_freq<int>(fs_freq_df<N1, N2>(i), N), N);
    else if (i < N + T) qzs[i - N] = fs_ratio<R>(k0 + i - N, P.g.nz);
    else twb[i - N - T] = P.tw[N1 * (i - N - T)];
  }
  __syncthreads();
  // forward phase A from global: line l < T is A_i0 at kz k0 + l, line
  // T + t is B_i at kz k0 + t
  constexpr int totA = 2 * T * N2;
  for (int i = threadIdx.x; i < totA; i += FFT_THREADS) {
    const int n2 = i / (2 * T);
    const int l = i - n2 * (2 * T);
    const int t = l % T;
    const bool ok = k0 + t < hz;
    cplx<R> v[N1];
    if (l < T) {
#pragma unroll
      for (int m = 0; m < N1; ++m)
        v[m] = ok ? gbase[(size_t)(N2 * m + n2) * rs + t] : cplx<R>{R(0.0f, 0.0f), R(0.0f, 0.0f)};
    } else {
      const R qz = qzs[t];
#pragma unroll
      for (int m = 0; m < N1; ++m) {
        if (ok) {
          const size_t o = (size_t)(N2 * m + n2) * rs + t;
          const cplx<R> a1 = gbase[(size_t)N * rs + o], a2 = gbase[(size_t)(2 * N) * rs + o];
          v[m] = {qy * a1.x + qz * a2.x, qy * a1.y + qz * a2.y};
        } else {
          v[m] = {R(0.0f, 0.0f), R(0.0f, 0.0f)};
        }
      }
    }
    dft_reg<R, N1, false>(v);
    if (n2 != 0) {
      const cplx<R>* w = tw2 + n2 * N1;
#pragma unroll
      for (int k1 = 1; k1 < N1; ++k1) v[k1] = c_mul(v[k1], w[k1]);
    }
    cplx<R>* line = buf + LM::base(l) + n2 * LM::ES;
#pragma unroll
    for (int m = 0; m < N1; ++m) line[m * N2 * LM::ES] = v[m];
  }
  __syncthreads();
  df_phase_b<N1, N2, false, LM>(buf, twb);
  __syncthreads();
  const R sc = (R)P.scale;
  const bool nyq_y = (ny % 2 == 0) && (2 * y == ny);
  const int kz_nyq = (P.g.nz % 2 == 0) ? P.g.nz / 2 : -1;
  for (int i = threadIdx.x; i < N * T; i += FFT_THREADS) {
    const R qx = qxs[i / T];
    const R qz = qzs[i % T];
    const R q2 = qx * qx + qy * qy + qz * qz;
    const bool nyq = nyq_y || (k0 + i % T == kz_nyq);
    const R f = (fs_positive(q2) && !nyq) ? sc * fs_rcp(q2) : R(0.0f, 0.0f);
    const cplx<R> A0 = buf[i], B = buf[N * T + i];
    const R sx = f * (qx * A0.x + B.x);
    const R sy = f * (qx * A0.y + B.y);
    buf[i] = {sx * qx, sy * qx};
    buf[N * T + i] = {sx, sy};
  }
  __syncthreads();
  // inverse: row j of the projected tensor is s xi_j; components 1 and 2
  // are xi_y and xi_z times the inverse transform of s
  df_phase_b<N1, N2, true, LM>(buf, twb);
  __syncthreads();
  constexpr int total = 2 * T * N2;
  for (int i = threadIdx.x; i < total; i += FFT_THREADS) {
    const int n2 = i / (2 * T);
    const int l = i - n2 * (2 * T);
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
    const int t = l % T;
    if (k0 + t < hz) {
      if (l < T) {
        cplx<R>* g = gbase + t;
#pragma unroll
        for (int m = 0; m < N1; ++m) g[(size_t)(N2 * m + n2) * rs] = v[m];
      } else {
        const R qz = qzs[t];
        cplx<R>* g1 = gbase + (size_t)N * rs + t;
        cplx<R>* g2 = gbase + (size_t)(2 * N) * rs + t;
#pragma unroll
        for (int m = 0; m < N1; ++m) {
          g1[(size_t)(N2 * m + n2) * rs] = {qy * v[m].x, qy * v[m].y};
          g2[(size_t)(N2 * m + n2) * rs] = {qz * v[m].x, qz * v[m].y};
        }
      }
    }
  }
}

template <int N1, int N2>
__global__ void __launch_bounds__(FFT_THREADS, 2) k_fft_x4_df(const LineParams<dfl> P) {
  fft_x4_df_tile<N1, N2, fs_x_t_df(N1 * N2)>(P, blockIdx.x);
}

RVE_DEV dfl dfl_half(dfl a) { return {0.5f * a.hi, 0.5f * a.lo}; }  // exact

// First z pass of G in float-float, persistent: each block walks tiles of
// lz z-lines (stride gridDim.x) -- the float64 field split into hi + lo
// pairs (integer operations, dfl_from_bits), components 2k and 2k+1 packed as the real and imaginary parts of
// complex line k (five per voxel line), in-place four-step DFT, half
// spectrum out (the two real spectra separated by the Hermitian symmetry).
template <int N1, int N2>
__global__ void __launch_bounds__(FFT_THREADS, 2) k_zfwd4_df(const ZfwdParams<dfl> P) {
  using R = dfl;
  constexpr int N = N1 * N2;
  constexpr int lz = fs_zd_lz(N), LP = (5 * lz) | 1, hz = N / 2 + 1;
  using LM = FsLayout<5 * lz, 0, 1, LP, 5 * lz>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<R>* tw2 = reinterpret_cast<cplx<R>*>(smem_raw);
  cplx<R>* buf = tw2 + ((N + 1) & ~1);
  fs_twiddles<R, N1, N2>(tw2, P.tw);
  const size_t n = P.g.n;
  const int nlines = P.g.nx * P.g.ny;
  const int ntiles = (nlines + lz - 1) / lz;
  const int hzp = P.g.hzp;
  const size_t ss = P.g.sstride;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int l0 = tile * lz;
    const int nl = min(lz, nlines - l0);
    const int nvox = nl * N;
    const size_t v0 = (size_t)l0 * N;
    for (int i = threadIdx.x; i < lz * N; i += FFT_THREADS) {
      R out[9];
      if (i < nvox) {
        double d[9];
#pragma unroll
        for (int c = 0; c < 9; ++c) d[c] = P.field64[(size_t)c * n + v0 + i];
#pragma unroll
        for (int c = 0; c < 9; ++c) out[c] = dfl_from_bits(d[c]);
      } else {
#pragma unroll
        for (int c = 0; c < 9; ++c) out[c] = R(0.0f, 0.0f);
      }
      const int li = i / N;
      cplx<R>* e = buf + (i - li * N) * LP + li;
#pragma unroll
      for (int k = 0; k < 5; ++k)
        e[k * lz] = {out[2 * k], (2 * k + 1 < 9) ? out[2 * k + 1] : R(0.0f, 0.0f)};
    }
    __syncthreads();
    fs_lines<R, N1, N2, false, LM>(buf, tw2);
    // spectrum k of line z = a + i b: A = (Z_k + conj Z_-k) / 2,
    // B = (Z_k - conj Z_-k) / (2i)
    for (int i = threadIdx.x; i < 5 * lz * hz; i += FFT_THREADS) {
      const int rest = i / hz;
      const int kz = i - rest * hz;
      const int k = rest / lz;
      const int li = rest - k * lz;
      if (li >= nl) continue;
      const int l = k * lz + li;
      const cplx<R> z1 = buf[fs_pos<N1, N2>(kz) * LP + l];
      const cplx<R> z2 = buf[fs_pos<N1, N2>(kz ? N - kz : 0) * LP + l];
      const size_t o = (size_t)(l0 + li) * hzp + kz;
      P.spec[(size_t)(2 * k) * ss + o] = {dfl_half(z1.x + z2.x), dfl_half(z1.y - z2.y)};
      if (2 * k + 1 < 9)
        P.spec[(size_t)(2 * k + 1) * ss + o] = {dfl_half(z1.y + z2.y), dfl_half(z2.x - z1.x)};
    }
    __syncthreads();  // the buffer is refilled by the next tile
  }
}

// Last z pass of G in float-float, persistent: the full z spectrum of each
// packed line rebuilt from the two half spectra (Z_k = A_k + i B_k, Z_-k =
// conj A_k + i conj B_k), in-place inverse four-step DFT, then OUT_PLAIN:
// the float64 result (OUT_PLAIN_MEANX: and its component means, summed in
// float-float per thread, in float64 across threads and blocks, into
// st->meanX); OUT_RESID: r = result (float32), x = 0, and the CG start
// from b.b.
template <int N1, int N2, typename RC, int OUT>
__global__ void __launch_bounds__(FFT_THREADS, 2) k_zinv4_df(const ZinvParams<dfl, RC> P) {
  using R = dfl;
  constexpr int N = N1 * N2;
  constexpr int lz = fs_zd_lz(N), LP = (5 * lz) | 1, hz = N / 2 + 1;
  using LM = FsLayout<5 * lz, 0, 1, LP, 5 * lz>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<R>* tw2 = reinterpret_cast<cplx<R>*>(smem_raw);
  cplx<R>* buf = tw2 + ((N + 1) & ~1);
  fs_twiddles<R, N1, N2>(tw2, P.tw);
  const size_t n = P.g.n;
  const int nlines = P.g.nx * P.g.ny;
  const int ntiles = (nlines + lz - 1) / lz;
  const int hzp = P.g.hzp;
  const size_t ss = P.g.sstride;
  double acc = 0.0;
  dfl msum[9];
#pragma unroll
  for (int c = 0; c < 9; ++c) msum[c] = dfl(0.0f, 0.0f);
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int l0 = tile * lz;
    const int nl = min(lz, nlines - l0);
    const int nvox = nl * N;
    const size_t v0 = (size_t)l0 * N;
    for (int i = threadIdx.x; i < 5 * lz * hz; i += FFT_THREADS) {
      const int rest = i / hz;
      const int kz = i - rest * hz;
      const int k = rest / lz;
      const int li = rest - k * lz;
      const int l = k * lz + li;
      const R zero(0.0f, 0.0f);
      cplx<R> A = {zero, zero}, B = {zero, zero};
      if (li < nl) {
        const size_t o = (size_t)(l0 + li) * hzp + kz;
        A = P.spec[(size_t)(2 * k) * ss + o];
        if (2 * k + 1 < 9) B = P.spec[(size_t)(2 * k + 1) * ss + o];
      }
      buf[fs_pos<N1, N2>(kz) * LP + l] = {A.x - B.y, A.y + B.x};
      if (kz > 0) buf[fs_pos<N1, N2>(N - kz) * LP + l] = {A.x + B.y, B.x - A.y};
    }
    __syncthreads();
    fs_lines<R, N1, N2, true, LM>(buf, tw2);
    for (int i = threadIdx.x; i < nvox; i += FFT_THREADS) {
      const int li = i / N;
      const cplx<R>* e = buf + (i - li * N) * LP + li;
      R out[9];
#pragma unroll
      for (int k = 0; k < 5; ++k) {
        const cplx<R> z = e[k * lz];
        out[2 * k] = z.x;
        if (2 * k + 1 < 9) out[2 * k + 1] = z.y;
      }
      const size_t v = v0 + i;
      if constexpr (OUT == OUT_PLAIN || OUT == OUT_PLAIN_MEANX) {
#pragma unroll
        for (int c = 0; c < 9; ++c) P.dst64[(size_t)c * n + v] = (double)out[c];
        if constexpr (OUT == OUT_PLAIN_MEANX) {
#pragma unroll
          for (int c = 0; c < 9; ++c) msum[c] = msum[c] + out[c];
        }
      } else {
        R s(0.0f, 0.0f);
#pragma unroll
        for (int c = 0; c < 9; ++c) {
          P.r_out[(size_t)c * n + v] = (RC)out[c];
          P.x_out[(size_t)c * n + v] = (RC)0;
          s = fma(out[c], out[c], s);
        }
        acc += (double)s;
      }
    }
    __syncthreads();  // the buffer is refilled by the next tile
  }
  if constexpr (OUT == OUT_RESID) {
    double v1[1] = {acc}, tot[1];
    if (last_block_sum_of<1>(v1, P.partials, &P.st->counter[SLOT_BB], tot, blockIdx.x, gridDim.x) &&
        threadIdx.x == 0)
      cg_after_bb(P.st, tot[0]);
  } else if constexpr (OUT == OUT_PLAIN_MEANX) {
    double v9[9], tot[9];
#pragma unroll
    for (int c = 0; c < 9; ++c) v9[c] = (double)msum[c];
    if (last_block_sum_of<9>(v9, P.partials, &P.st->counter[SLOT_MEAN], tot, blockIdx.x,
                             gridDim.x) &&
        threadIdx.x == 0) {
      for (int c = 0; c < 9; ++c) P.st->meanX[c] = tot[c] / (double)n;
    }
  }
}

// x pass of the preconditioned CG iteration: as k_fft_x4, with the
// reference-medium Green operator Gamma0 = pinv(G K0 G) G in place of G-hat.
// Per frequency, with a_i = sum_l A_il xi_l / |xi|^2 (the coefficient of
// Eq. G_red) and d = xi . a / |xi|^2, the inverse acoustic tensor of the
// isotropic K0 (mu0 = 1) gives C_ij = (a_i - c xi_i d) xi_j,
// c = (lambda0 + mu0) / (lambda0 + 2 mu0).  d couples the three tensor rows,
// so a tile holds all nine components: (9 components) x nx x (T kz), one ky.
template <typename R, int N1, int N2>
__global__ void __launch_bounds__(FFT_THREADS, 2) k_fft_x4_g0(const LineParams<R> P) {
  constexpr int N = N1 * N2;
  constexpr int T = fs_x_t_g0(N);
  using LM = FsLayout<T, N * T, 1, T, 9 * T>;
  if (P.done && *P.done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<R>* tw2 = reinterpret_cast<cplx<R>*>(smem_raw);
  cplx<R>* buf = tw2 + ((N + 1) & ~1);
  const int ny = P.g.ny;
  const int hz = P.g.hz, hzp = P.g.hzp;
  const int ntk = (hz + T - 1) / T;
  const size_t rs = (size_t)ny * hzp;  // stride of spectrum rows (c*nx + x)
  const int tile = blockIdx.x;
  const int y = tile / ntk;
  const int k0 = (tile - y * ntk) * T;
  cplx<R>* gbase = P.spec + (size_t)y * hzp + k0;
  // line l = (component l / T, kz k0 + l % T): rows x at stride rs
  auto gl = [&](int l) {
    const int c = l / T, t = l - (l / T) * T;
    return GLine<R>{gbase + (size_t)c * N * rs + t, rs, k0 + t < hz, k0 + t < hz};
  };
  fs_twiddles<R, N1, N2>(tw2, P.tw);
  __syncthreads();
  fs_phase_a_g2s<R, N1, N2, LM>(buf, tw2, gl);
  __syncthreads();
  fs_phase_b<R, N1, N2, false, LM>(buf);
  const R qy = signed_freq<R>(y, ny) / (R)ny;
  const R sc = (R)P.scale;
  const R cc = (R)P.g.pc_c;
  R* qxs = reinterpret_cast<R*>(buf + 9 * N * T);  // [N]
  R* qzs = qxs + N;                                // [T]
  for (int i = threadIdx.x; i < N + T; i += FFT_THREADS) {
    if (i < N) qxs[i] = signed_freq<R>(fs_freq<N1, N2>(i), N) / (R)N;
    else qzs[i - N] = (R)(k0 + i - N) / (R)P.g.nz;
  }
  __syncthreads();
  const bool nyq_y = (ny % 2 == 0) && (2 * y == ny);
  const int kz_nyq = (P.g.nz % 2 == 0) ? P.g.nz / 2 : -1;
  constexpr int NT = N * T;
  for (int i = threadIdx.x; i < NT; i += FFT_THREADS) {
    const R q[3] = {qxs[i / T], qy, qzs[i % T]};
    const R q2 = q[0] * q[0] + q[1] * q[1] + q[2] * q[2];
    const bool nyq = nyq_y || (k0 + i % T == kz_nyq);
    const R inv = (q2 > R(0) && !nyq) ? __frcp_rn(q2) : R(0);
    R ax[3], ay[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const cplx<R> A0 = buf[(3 * r) * NT + i], A1 = buf[(3 * r + 1) * NT + i],
                    A2 = buf[(3 * r + 2) * NT + i];
      ax[r] = sc * inv * (q[0] * A0.x + q[1] * A1.x + q[2] * A2.x);
      ay[r] = sc * inv * (q[0] * A0.y + q[1] * A1.y + q[2] * A2.y);
    }
    const R dx = cc * inv * (q[0] * ax[0] + q[1] * ax[1] + q[2] * ax[2]);
    const R dy = cc * inv * (q[0] * ay[0] + q[1] * ay[1] + q[2] * ay[2]);
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const R bx = ax[r] - q[r] * dx, by = ay[r] - q[r] * dy;
#pragma unroll
      for (int j = 0; j < 3; ++j) buf[(3 * r + j) * NT + i] = {bx * q[j], by * q[j]};
    }
  }
  __syncthreads();
  fs_phase_b<R, N1, N2, true, LM>(buf);
  __syncthreads();
  fs_phase_a_s2g<R, N1, N2, LM>(buf, tw2, gl);
}

// L2 prefetch of the first-pass inputs of a tile (r and F, after the first
// iteration p and x, the phase bytes): one bulk prefetch per component's
// range, issued by one thread.
template <typename R, int SRC, int TAN>
RVE_DEV void zfwd_prefetch_tile(const ZfwdParams<R>& P, const ZfwdScalars<R>& sc, size_t v0,
                                int nvox) {
  if constexpr (SRC == SRC_CGPX && TAN == TAN_SVK) {
    const size_t n = P.g.n;
    const int nf = sc.first ? 18 : 36;
    if (threadIdx.x == 0) {
      for (int a = 0; a < nf; ++a) {
        const R* b = a < 9 ? P.r : a < 18 ? P.tan.Fop : a < 27 ? P.p : P.x;
        bulk_prefetch_l2(b + (size_t)(a % 9) * n + v0, (size_t)nvox * sizeof(R));
      }
      if (P.tan.mat.phase) bulk_prefetch_l2(P.tan.mat.phase + v0, (size_t)nvox);
    }
  }
}

// First pass of the fused float CG iteration on the four-step z DFT,
// persistent: each thread block walks tiles of lz z-lines (stride gridDim.x)
// -- voxel stage (p, lagged x, tangent, p.(K:p)) into a transposed buffer
// (element z of line l at z * LP + l, LP odd), in-place DFT of the 5 lz
// packed lines, half spectrum out -- and prefetches its next tile's inputs
// into L2 before the DFT, so that they arrive while it computes.
template <typename R, int SRC, int TAN, int N1, int N2>
RVE_DEV void zfwd4_blocks(const ZfwdParams<R>& P, const int bid, const int nblk) {
  constexpr int N = N1 * N2;
  constexpr int lz = fs_zf_lz(N), LP = (5 * lz) | 1, hz = N / 2 + 1;
  using LM = FsLayout<5 * lz, 0, 1, LP, 5 * lz>;
  if (P.done && *P.done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<R>* tw2 = reinterpret_cast<cplx<R>*>(smem_raw);
  cplx<R>* buf = tw2 + ((N + 1) & ~1);
  fs_twiddles<R, N1, N2>(tw2, P.tw);
  const int nlines = P.g.nx * P.g.ny;
  const int ntiles = (nlines + lz - 1) / lz;
  const ZfwdScalars<R> sc = zfwd_scalars<R, SRC>(P);
  const int hzp = P.g.hzp;
  const size_t ss = P.g.sstride;
  double pkp = 0.0;
  for (int tile = bid; tile < ntiles; tile += nblk) {
    const int l0 = tile * lz;
    const int nl = min(lz, nlines - l0);
    const int nvox = nl * N;
    const size_t v0 = (size_t)l0 * N;
    R tpk = 0;  // this tile's share of p.(K:p): a few voxels per thread
    for (int i = threadIdx.x; i < lz * N; i += FFT_THREADS) {
      R out[9];
      if (i < nvox) {
        zfwd_voxel<R, SRC, TAN>(P, sc, v0 + i, out, tpk);
      } else {
#pragma unroll
        for (int c = 0; c < 9; ++c) out[c] = 0;
      }
      const int li = i / N;
      cplx<R>* e = buf + (i - li * N) * LP + li;
#pragma unroll
      for (int k = 0; k < 5; ++k) e[k * lz] = {out[2 * k], (2 * k + 1 < 9) ? out[2 * k + 1] : R(0)};
    }
    pkp += (double)tpk;
    __syncthreads();
    const int next = tile + nblk;
    if (next < ntiles) {
      const int nl2 = min(lz, nlines - next * lz);
      zfwd_prefetch_tile<R, SRC, TAN>(P, sc, (size_t)next * lz * N, nl2 * N);
    }
    fs_lines<R, N1, N2, false, LM>(buf, tw2);
    // half spectrum, two kz per thread (16-byte stores); with hz odd the
    // last pair's second value lands in the row padding as zero
    constexpr int hz2 = (hz + 1) / 2;
    for (int i = threadIdx.x; i < 5 * lz * hz2; i += FFT_THREADS) {
      const int rest = i / hz2;
      const int kz = 2 * (i - rest * hz2);
      const int k = rest / lz;
      const int li = rest - k * lz;
      if (li >= nl) continue;
      const int l = k * lz + li;
      float4 a, b;
      {
        const cplx<R> z1 = buf[fs_pos<N1, N2>(kz) * LP + l];
        cplx<R> z2 = buf[fs_pos<N1, N2>(kz ? N - kz : 0) * LP + l];
        z2.y = -z2.y;
        // A = (z1 + conj(z_-k)) / 2, B = (z1 - conj(z_-k)) / (2i)
        a.x = R(0.5) * (z1.x + z2.x);
        a.y = R(0.5) * (z1.y + z2.y);
        b.x = R(0.5) * (z1.y - z2.y);
        b.y = -R(0.5) * (z1.x - z2.x);
      }
      if (kz + 1 < hz) {
        const cplx<R> z1 = buf[fs_pos<N1, N2>(kz + 1) * LP + l];
        cplx<R> z2 = buf[fs_pos<N1, N2>(N - kz - 1) * LP + l];
        z2.y = -z2.y;
        a.z = R(0.5) * (z1.x + z2.x);
        a.w = R(0.5) * (z1.y + z2.y);
        b.z = R(0.5) * (z1.y - z2.y);
        b.w = -R(0.5) * (z1.x - z2.x);
      } else {
        a.z = a.w = b.z = b.w = R(0);
      }
      const size_t o = (size_t)(l0 + li) * hzp + kz;
      *reinterpret_cast<float4*>(P.spec + (size_t)(2 * k) * ss + o) = a;
      if (2 * k + 1 < 9) *reinterpret_cast<float4*>(P.spec + (size_t)(2 * k + 1) * ss + o) = b;
    }
    __syncthreads();  // the buffer is refilled by the next tile
  }
  if (SRC == SRC_CGPX) zfwd_step_length<R>(P, pkp, bid, nblk);
}

template <typename R, int SRC, int TAN, int N1, int N2>
__global__ void __launch_bounds__(FFT_THREADS, (Fs4Occ<R, N1, N2>::value))
    k_zfwd4(const ZfwdParams<R> P) {
  zfwd4_blocks<R, SRC, TAN, N1, N2>(P, blockIdx.x, gridDim.x);
}

// First pass of the fused float CG iteration for the SVK tangent with a
// phase map, persistent and pipelined: the inputs of a tile -- r and F,
// after the first iteration also p and x, and the phase bytes -- arrive in
// shared memory by bulk asynchronous copies (TMA) that one thread issues for
// the block's NEXT tile as soon as the current tile's voxel stage has read
// its staged copy, so that they land while the block runs the current
// tile's DFT and stores.  Each copy covers the 16-byte-aligned span around
// one component's range of the tile (the arrays start 256-byte aligned
// inside one allocation with slack after the last one, so the span stays in
// it); soffs[a] is where the range starts in its staged copy.  Completion is
// tracked by one mbarrier whose phase flips per tile; a bounded wait that
// gives up marks the solver state (the last block then reports a timeout).
template <int N1, int N2>
__global__ void __launch_bounds__(FFT_THREADS, 3) k_zfwd4p(const ZfwdParams<float> P) {
  using R = float;
  constexpr int N = N1 * N2;
  constexpr int lz = fs_zt_lz(N), hz = N / 2 + 1;
  constexpr Z4tLayout Lt = z4t_layout(N, lz);
  constexpr int LP = Lt.lp, SP = Lt.sp;
  using LM = FsLayout<5 * lz, 0, 1, LP, 5 * lz>;
  if (P.done && *P.done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) unsigned long long bar;
  __shared__ int soffs[37];
  cplx<R>* tw2 = reinterpret_cast<cplx<R>*>(smem_raw);
  cplx<R>* buf = tw2 + ((N + 1) & ~1);
  float* stage = reinterpret_cast<float*>(smem_raw + Lt.stage_off);
  unsigned char* sphase = smem_raw + Lt.phase_off;
  const size_t n = P.g.n;
  const int nlines = P.g.nx * P.g.ny;
  const int ntiles = (nlines + lz - 1) / lz;
  const int hzp = P.g.hzp;
  const size_t ss = P.g.sstride;
  const ZfwdScalars<R> sc = zfwd_scalars<R, SRC_CGPX>(P);
  const int narr = sc.first ? 18 : 36;  // r, F, then p, x
  // thread 0: stage the inputs of tile t (expected bytes first, then copies)
  auto issue = [&](int t) {
    const int nl = min(lz, nlines - t * lz);
    const int nvox = nl * N;
    const size_t v0 = (size_t)t * lz * N;
    auto span = [&](int a, uintptr_t& lo16, unsigned& bytes) {
      uintptr_t lo, hi;
      if (a < narr) {
        const float* b = a < 9 ? P.r : a < 18 ? P.tan.Fop : a < 27 ? P.p : P.x;
        const float* src = b + (size_t)(a % 9) * n + v0;
        lo = reinterpret_cast<uintptr_t>(src);
        hi = reinterpret_cast<uintptr_t>(src + nvox);
      } else {
        lo = reinterpret_cast<uintptr_t>(P.tan.mat.phase + v0);
        hi = lo + (uintptr_t)nvox;
      }
      lo16 = lo & ~(uintptr_t)15;
      bytes = (unsigned)(((hi + 15) & ~(uintptr_t)15) - lo16);
      return (int)(lo - lo16) / (a < narr ? 4 : 1);
    };
    unsigned total = 0;
    for (int a = 0; a <= narr; ++a) {
      uintptr_t lo16;
      unsigned bytes;
      soffs[a] = span(a, lo16, bytes);
      total += bytes;
    }
    mbar_arrive_expect_tx(&bar, total);
    for (int a = 0; a <= narr; ++a) {
      uintptr_t lo16;
      unsigned bytes;
      span(a, lo16, bytes);
      void* dst = a < narr ? (void*)(stage + (size_t)a * SP) : (void*)sphase;
      bulk_load(dst, reinterpret_cast<const void*>(lo16), bytes, &bar);
    }
  };
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  __syncthreads();
  if (threadIdx.x == 0 && (int)blockIdx.x < ntiles) issue(blockIdx.x);
  fs_twiddles<R, N1, N2>(tw2, P.tw);
  double pkp = 0.0;
  unsigned parity = 0;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int l0 = tile * lz;
    const int nl = min(lz, nlines - l0);
    const int nvox = nl * N;
    const size_t v0 = (size_t)l0 * N;
    if (!mbar_wait_bounded(&bar, parity, P.g.wait_polls)) {
      atomicOr(&P.st->dev_timeout, 1);
      mbar_wait_bounded(&bar, parity, kDefaultWaitPolls);  // let the copies land before going on
    }
    parity ^= 1u;
    const int pofs = soffs[narr];
    for (int i = threadIdx.x; i < lz * N; i += FFT_THREADS) {
      R out[9];
      if (i < nvox) {
        const size_t v = v0 + i;
        TanPre<R> q;
#pragma unroll
        for (int c = 0; c < 9; ++c) q.F[c] = stage[(9 + c) * SP + soffs[9 + c] + i];
        const int ph = sphase[pofs + i];
        q.lam = P.tan.mat.table[ph * P.tan.mat.nparam];
        q.mu = P.tan.mat.table[ph * P.tan.mat.nparam + 1];
        R in[9];
        if (sc.first) {
#pragma unroll
          for (int c = 0; c < 9; ++c) in[c] = stage[c * SP + soffs[c] + i];
        } else {
#pragma unroll
          for (int c = 0; c < 9; ++c) {
            const R rr = stage[c * SP + soffs[c] + i];
            const R pp = stage[(18 + c) * SP + soffs[18 + c] + i];
            const R xx = stage[(27 + c) * SP + soffs[27 + c] + i];
            P.x[(size_t)c * n + v] = fma(sc.alpha_prev, pp, xx);
            in[c] = fma(sc.beta, pp, rr);
          }
        }
        tangent_post<R, TAN_SVK>(P.tan, v, n, q, in, out);
        R sp = 0;
#pragma unroll
        for (int c = 0; c < 9; ++c) {
          P.p[(size_t)c * n + v] = in[c];
          sp = fma(in[c], out[c], sp);
        }
        pkp += (double)sp;
      } else {
#pragma unroll
        for (int c = 0; c < 9; ++c) out[c] = 0;
      }
      const int li = i / N;
      cplx<R>* e = buf + (i - li * N) * LP + li;
#pragma unroll
      for (int k = 0; k < 5; ++k) e[k * lz] = {out[2 * k], (2 * k + 1 < 9) ? out[2 * k + 1] : R(0)};
    }
    __syncthreads();  // staged copy consumed: refill it with the next tile
    if (threadIdx.x == 0 && tile + (int)gridDim.x < ntiles) issue(tile + gridDim.x);
    fs_lines<R, N1, N2, false, LM>(buf, tw2);
    for (int i = threadIdx.x; i < 5 * lz * hz; i += FFT_THREADS) {
      const int rest = i / hz;
      const int kz = i - rest * hz;
      const int k = rest / lz;
      const int li = rest - k * lz;
      if (li >= nl) continue;
      const int l = k * lz + li;
      const cplx<R> z1 = buf[fs_pos<N1, N2>(kz) * LP + l];
      cplx<R> z2 = buf[fs_pos<N1, N2>(kz ? N - kz : 0) * LP + l];
      z2.y = -z2.y;
      const size_t o = (size_t)(l0 + li) * hzp + kz;
      P.spec[(size_t)(2 * k) * ss + o] = {R(0.5) * (z1.x + z2.x), R(0.5) * (z1.y + z2.y)};
      if (2 * k + 1 < 9) {
        const R dx = R(0.5) * (z1.x - z2.x), dy = R(0.5) * (z1.y - z2.y);
        P.spec[(size_t)(2 * k + 1) * ss + o] = {dy, -dx};
      }
    }
    __syncthreads();  // the DFT buffer is refilled by the next tile
  }
  zfwd_step_length<R>(P, pkp, blockIdx.x, gridDim.x);
}

// L2 prefetch of the last pass's inputs of a tile: the tile's half spectrum
// (per component nl consecutive rows of hzp values, contiguous) and its r
// range, one bulk prefetch each, issued by one thread.
template <typename R>
RVE_DEV void zinv_prefetch_tile(const ZinvParams<R, R>& P, int l0, int nl, size_t v0, int nvox) {
  if (threadIdx.x == 0) {
    const size_t ss = P.g.sstride;
    const int hzp = P.g.hzp;
    for (int c = 0; c < 9; ++c) {
      bulk_prefetch_l2(P.spec + (size_t)c * ss + (size_t)l0 * hzp, (size_t)nl * hzp * sizeof(cplx<R>));
      bulk_prefetch_l2(P.r_out + (size_t)c * P.g.n + v0, (size_t)nvox * sizeof(R));
    }
  }
}

// Last pass of the fused float CG iteration, persistent like k_zfwd4: per
// tile the nine r ranges are fetched by bulk asynchronous copies (TMA, one
// thread, completion on an mbarrier whose phase flips per tile; the spans
// are the 16-byte-aligned ones around each range, rofs[c] the offset of the
// range in its copy) while the half spectrum is expanded into the
// transposed order (two kz per thread, 16-byte loads) and transformed back;
// then r -= alpha Ap in place and r.r.  The next tile's inputs are
// prefetched into L2 before the DFT stage.
template <typename R, int N1, int N2>
RVE_DEV void zinv4_cgr_blocks(const ZinvParams<R, R>& P, const int bid, const int nblk) {
  static_assert(sizeof(R) == 4, "float32 CG iteration");
  constexpr int N = N1 * N2;
  constexpr int lz = fs_z_lz(N), LP = (5 * lz) | 1, hz = N / 2 + 1;
  constexpr int SP = (lz * N + 8 + 3) & ~3;  // staged floats per r component
  constexpr int hz2 = (hz + 1) / 2;          // kz pairs per line
  using LM = FsLayout<5 * lz, 0, 1, LP, 5 * lz>;
  if (P.done && *P.done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) unsigned long long bar;
  __shared__ int rofs[9];
  const int hzp = P.g.hzp;
  cplx<R>* tw2 = reinterpret_cast<cplx<R>*>(smem_raw);
  cplx<R>* buf = tw2 + ((N + 1) & ~1);
  R* rt = reinterpret_cast<R*>(smem_raw + z4inv_stage_off(N, lz));  // [9][SP]
  const size_t n = P.g.n;
  const size_t ss = P.g.sstride;
  const int nlines = P.g.nx * P.g.ny;
  const int ntiles = (nlines + lz - 1) / lz;
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  fs_twiddles<R, N1, N2>(tw2, P.tw);
  const R alpha = (R)P.st->alpha;
  const R mn_ell = (R)P.mn_ell;
  __syncthreads();
  double acc = 0.0;
  unsigned parity = 0;
  for (int tile = bid; tile < ntiles; tile += nblk) {
    const int l0 = tile * lz;
    const int nl = min(lz, nlines - l0);
    const int nvox = nl * N;
    const size_t v0 = (size_t)l0 * N;
    if (threadIdx.x == 0) {
      unsigned total = 0;
      uintptr_t lo16[9];
      unsigned bytes[9];
      for (int c = 0; c < 9; ++c) {
        const uintptr_t lo = reinterpret_cast<uintptr_t>(P.r_out + (size_t)c * n + v0);
        const uintptr_t hi = lo + sizeof(R) * (uintptr_t)nvox;
        lo16[c] = lo & ~(uintptr_t)15;
        bytes[c] = (unsigned)(((hi + 15) & ~(uintptr_t)15) - lo16[c]);
        rofs[c] = (int)(lo - lo16[c]) / (int)sizeof(R);
        total += bytes[c];
      }
      mbar_arrive_expect_tx(&bar, total);
      for (int c = 0; c < 9; ++c)
        bulk_load(rt + (size_t)c * SP, reinterpret_cast<const void*>(lo16[c]), bytes[c], &bar);
    }
    // full z spectrum of the packed lines z = a + i b, written transposed;
    // item = (component pair k, line li, kz pair); a pair's second kz may
    // lie in the row padding (hz odd), where nothing is read or written
    // two rounds of items per batch: both rounds' spectrum loads are in
    // flight before the first round's stores
    constexpr int totl = 5 * lz * hz2;
    constexpr int NR = (totl + FFT_THREADS - 1) / FFT_THREADS;
#pragma unroll
    for (int r0 = 0; r0 < NR; r0 += 2) {
      float4 A[2], B[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int i = threadIdx.x + (r0 + u) * FFT_THREADS;
        const int rest = i / hz2;
        const int kz = 2 * (i - rest * hz2);
        const int k = rest / lz;
        const int li = rest - k * lz;
        A[u] = B[u] = float4{0.f, 0.f, 0.f, 0.f};
        if (r0 + u < NR && i < totl && li < nl) {
          const size_t o = (size_t)(l0 + li) * hzp + kz;
          A[u] = *reinterpret_cast<const float4*>(P.spec + (size_t)(2 * k) * ss + o);
          if (2 * k + 1 < 9) B[u] = *reinterpret_cast<const float4*>(P.spec + (size_t)(2 * k + 1) * ss + o);
        }
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int i = threadIdx.x + (r0 + u) * FFT_THREADS;
        if (r0 + u >= NR || i >= totl) continue;
        const int rest = i / hz2;
        const int kz = 2 * (i - rest * hz2);
        const int k = rest / lz;
        const int li = rest - k * lz;
        const int l = k * lz + li;
        const float4 a = A[u], b = B[u];
        buf[fs_pos<N1, N2>(kz) * LP + l] = {a.x - b.y, a.y + b.x};
        if (kz > 0) buf[fs_pos<N1, N2>(N - kz) * LP + l] = {a.x + b.y, b.x - a.y};
        if (kz + 1 < hz) {
          buf[fs_pos<N1, N2>(kz + 1) * LP + l] = {a.z - b.w, a.w + b.z};
          buf[fs_pos<N1, N2>(N - kz - 1) * LP + l] = {a.z + b.w, b.z - a.w};
        }
      }
    }
    __syncthreads();
    const int next = tile + nblk;
    if (next < ntiles) {
      const int nl2 = min(lz, nlines - next * lz);
      zinv_prefetch_tile<R>(P, next * lz, nl2, (size_t)next * lz * N, nl2 * N);
    }
    fs_lines<R, N1, N2, true, LM>(buf, tw2);
    if (!mbar_wait_bounded(&bar, parity, P.g.wait_polls)) {
      atomicOr(&P.st->dev_timeout, 1);
      mbar_wait_bounded(&bar, parity, kDefaultWaitPolls);  // let the copies land before going on
    }
    parity ^= 1u;
    R tacc = 0;  // this tile's share of r.r: a few voxels per thread
    for (int i = threadIdx.x; i < nvox; i += FFT_THREADS) {
      const int li = i / N;
      const cplx<R>* e = buf + (i - li * N) * LP + li;
      R out[9];
#pragma unroll
      for (int k = 0; k < 5; ++k) {
        const cplx<R> z = e[k * lz];
        out[2 * k] = z.x;
        if (2 * k + 1 < 9) out[2 * k + 1] = z.y;
      }
      R s = 0;
#pragma unroll
      for (int c = 0; c < 9; ++c) {
        out[c] = fma(-alpha, out[c], rt[c * SP + rofs[c] + i]);
        P.r_out[(size_t)c * n + v0 + i] = out[c];
        s = fma(out[c], out[c], s);
      }
      if (mn_ell >= R(0)) s = mnorm_k0<R>(out, mn_ell);
      tacc += s;
    }
    acc += (double)tacc;
    __syncthreads();  // buffer, r copy and rofs are refilled by the next tile
  }
  double v1[1] = {acc}, tot[1];
  if (last_block_sum_of<1>(v1, P.partials, &P.st->counter[SLOT_RR], tot, bid, nblk) &&
      threadIdx.x == 0) {
    if (P.st->dev_timeout) {
      P.st->status = RVE_DEV_ERR_TIMEOUT;
      P.st->done = 1;
    } else {
      cg_after_rr(P.st, tot[0]);
    }
  }
}

template <typename R, int N1, int N2>
__global__ void __launch_bounds__(FFT_THREADS, (Fs4Occ<R, N1, N2>::value))
    k_zinv4_cgr(const ZinvParams<R, R> P) {
  zinv4_cgr_blocks<R, N1, N2>(P, blockIdx.x, gridDim.x);
}

cudaError_t g_err4 = cudaSuccess;

template <typename K>
void allow_smem(K kernel) {
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 208 * 1024);
  if (e != cudaSuccess && g_err4 == cudaSuccess) g_err4 = e;
}

}  // namespace

// ---------------------------------------------------------------------------
// Recording of the four-step launches for batched passes (see kernels.h).
// ---------------------------------------------------------------------------
namespace {
// one kind of pass (0 first z, 1 y forward, 2 x, 3 y inverse, 4 last z)
// for every recorded cell
struct Fs4Pass {
  std::vector<char> params;  // per cell, one parameter struct of the kind
  std::vector<int> axis, tan, nblk;
  std::vector<int2> blk;     // per block of the batched launch: (cell, block)
  size_t smem = 0;
  char* d_params = nullptr;
  int *d_axis = nullptr, *d_tan = nullptr, *d_nblk = nullptr;
  int2* d_blk = nullptr;
};
thread_local Fs4Batch* t_rec = nullptr;

constexpr bool fs4_batch_size(int n) {
  return n == 15 || n == 21 || n == 27 || n == 33 || n == 45 || n == 63;
}
}  // namespace

struct Fs4Batch {
  Fs4Pass pass[5];
  bool bad = false;  // a launch that cannot be batched was recorded
};

namespace {
template <typename PT>
void rec_add(int kind, const PT& P, int axis, int tan, int grid, size_t sm) {
  Fs4Pass& p = t_rec->pass[kind];
  if (!fs4_batch_size(axis)) t_rec->bad = true;
  const int c = (int)p.axis.size();
  const char* raw = reinterpret_cast<const char*>(&P);
  p.params.insert(p.params.end(), raw, raw + sizeof(PT));
  p.axis.push_back(axis);
  p.tan.push_back(tan);
  p.nblk.push_back(grid);
  for (int b = 0; b < grid; ++b) p.blk.push_back(make_int2(c, b));
  p.smem = std::max(p.smem, sm);
}
}  // namespace

void launch_fft_y4(const GridGeom& g, bool inverse, cplx<float>* spec, const int* done,
                   const cplx<float>* tw, cudaStream_t s) {
  LineParams<float> P;
  P.g = g;
  P.t = g.fsy_t;
  P.grp = g.fsy_grp;
  P.scale = 1.0;
  P.spec = spec;
  P.done = done;
  P.tw = tw;
  const int ntiles = ((g.hz + P.t - 1) / P.t) * ((9 * g.nx + P.grp - 1) / P.grp);
  const size_t sm = sizeof(cplx<float>) * ((size_t)((g.ny + 1) & ~1) + (size_t)P.grp * g.ny * P.t);
  if (t_rec) {
    rec_add(inverse ? 3 : 1, P, g.ny, 0, ntiles, sm);
    return;
  }
  switch (g.ny) {
#define RVE_FS_Y(N, A, B)                                                                       \
  case N:                                                                                       \
    if (P.t == fs_y_t()) {                                                                      \
      if (inverse) k_fft_y4<float, A, B, true, fs_y_t()><<<ntiles, FFT_THREADS, sm, s>>>(P);    \
      else k_fft_y4<float, A, B, false, fs_y_t()><<<ntiles, FFT_THREADS, sm, s>>>(P);           \
    } else {                                                                                    \
      if (inverse) k_fft_y4<float, A, B, true, fs_y_t2()><<<ntiles, FFT_THREADS, sm, s>>>(P);   \
      else k_fft_y4<float, A, B, false, fs_y_t2()><<<ntiles, FFT_THREADS, sm, s>>>(P);          \
    }                                                                                           \
    break;
    RVE_FS_SIZES(RVE_FS_Y)
#undef RVE_FS_Y
    default:
      break;
  }
}

void launch_fft_x4(const GridGeom& g, double scale, cplx<float>* spec, const int* done,
                   const cplx<float>* tw, cudaStream_t s, bool gamma0) {
  LineParams<float> P;
  P.g = g;
  if (gamma0 && t_rec) {
    t_rec->bad = true;
    return;
  }
  if (gamma0) {
    P.t = 0;
    P.grp = 1;
    P.scale = scale;
    P.spec = spec;
    P.done = done;
    P.tw = tw;
    switch (g.nx) {
#define RVE_FS_XG(N, A, B)                                                                      case N: {                                                                                       constexpr int T = fs_x_t_g0(N);                                                               const int ntiles = g.ny * ((g.hz + T - 1) / T);                                               const size_t sm = sizeof(cplx<float>) * ((size_t)((N + 1) & ~1) + 9 * (size_t)N * T) +                          sizeof(float) * ((size_t)N + T);                                            k_fft_x4_g0<float, A, B><<<ntiles, FFT_THREADS, sm, s>>>(P);                                  break;                                                                                      }
      RVE_FS_SIZES(RVE_FS_XG)
#undef RVE_FS_XG
      default:
        break;
    }
    return;
  }
  P.t = g.fsx_t;
  P.grp = 1;
  P.scale = scale;
  P.spec = spec;
  P.done = done;
  P.tw = tw;
  const int ntiles = 3 * g.ny * ((g.hz + P.t - 1) / P.t);
  const size_t sm = sizeof(cplx<float>) * ((size_t)((g.nx + 1) & ~1) + 3 * (size_t)g.nx * P.t) +
                    sizeof(float) * ((size_t)g.nx + P.t);
  if (t_rec) {
    rec_add(2, P, g.nx, 0, ntiles, sm);
    return;
  }
  switch (g.nx) {
#define RVE_FS_X(N, A, B)                                                        \
  case N:                                                                        \
    if (P.t == fs_x_t(N)) k_fft_x4<float, A, B, fs_x_t(N)><<<ntiles, FFT_THREADS, sm, s>>>(P); \
    else k_fft_x4<float, A, B, fs_x_t2(N)><<<ntiles, FFT_THREADS, sm, s>>>(P);   \
    break;
    RVE_FS_SIZES(RVE_FS_X)
#undef RVE_FS_X
    default:
      break;
  }
}

bool launch_fft_y4_df(const GridGeom& g, bool inverse, cplx<dfl>* spec, const cplx<dfl>* tw,
                      cudaStream_t s) {
  LineParams<dfl> P;
  P.g = g;
  P.t = fs_y_t_df();
  P.scale = 1.0;
  P.spec = spec;
  P.done = nullptr;
  P.tw = tw;
  constexpr int T = fs_y_t_df();
  switch (g.ny) {
#define RVE_FS_YD(N, A, B)                                                                       \
  case N: {                                                                                      \
    constexpr int GRP = fs_y_grp(N);                                                             \
    P.grp = GRP;                                                                                 \
    const int ntiles = ((g.hz + T - 1) / T) * ((9 * g.nx + GRP - 1) / GRP);                      \
    const size_t sm = sizeof(cplx<dfl>) * ((size_t)((N + 1) & ~1) + (size_t)GRP * N * T);         \
    if (inverse) k_fft_y4_df<A, B, true><<<ntiles, FFT_THREADS, sm, s>>>(P);                     \
    else k_fft_y4_df<A, B, false><<<ntiles, FFT_THREADS, sm, s>>>(P);                            \
    return true;                                                                                 \
  }
    RVE_FS_SIZES(RVE_FS_YD)
#undef RVE_FS_YD
    default:
      return false;
  }
}

static int sm_count();

bool launch_zfwd4_df(const GridGeom& g, const double* in, cplx<dfl>* spec, const cplx<dfl>* tw,
                     cudaStream_t s) {
  ZfwdParams<dfl> P{};
  P.g = g;
  P.src = SRC_FIELD;
  P.field64 = in;
  P.spec = spec;
  P.tw = tw;
  const int nlines = g.nx * g.ny;
  switch (g.nz) {
#define RVE_FS_ZFD(N, A, B)                                                                      \
  case N: {                                                                                      \
    constexpr int lz = fs_zd_lz(N);                                                              \
    const int nblk = std::min((nlines + lz - 1) / lz, 2 * sm_count());                           \
    const size_t sm = sizeof(cplx<dfl>) * ((size_t)((N + 1) & ~1) + (size_t)N * ((5 * lz) | 1)); \
    k_zfwd4_df<A, B><<<nblk, FFT_THREADS, sm, s>>>(P);                                           \
    return true;                                                                                 \
  }
    RVE_FS_SIZES(RVE_FS_ZFD)
#undef RVE_FS_ZFD
    default:
      return false;
  }
}

bool launch_zinv4_df(const GridGeom& g, int out_mode, const cplx<dfl>* spec, double* out64,
                     float* r_out, float* x_out, SolverState* st, double* partials,
                     const cplx<dfl>* tw, cudaStream_t s) {
  const int nlines = g.nx * g.ny;
  switch (g.nz) {
#define RVE_FS_ZID(N, A, B)                                                                      \
  case N: {                                                                                      \
    constexpr int lz = fs_zd_lz(N);                                                              \
    const int nblk = std::min((nlines + lz - 1) / lz, 2 * sm_count());                           \
    const size_t sm = sizeof(cplx<dfl>) * ((size_t)((N + 1) & ~1) + (size_t)N * ((5 * lz) | 1)); \
    if (out_mode != OUT_RESID) {                                                                 \
      ZinvParams<dfl, double> P{};                                                               \
      P.g = g;                                                                                   \
      P.spec = spec;                                                                             \
      P.dst64 = out64;                                                                           \
      P.st = st;                                                                                 \
      P.partials = partials;                                                                     \
      P.tw = tw;                                                                                 \
      if (out_mode == OUT_PLAIN_MEANX)                                                           \
        k_zinv4_df<A, B, double, OUT_PLAIN_MEANX><<<nblk, FFT_THREADS, sm, s>>>(P);              \
      else                                                                                       \
        k_zinv4_df<A, B, double, OUT_PLAIN><<<nblk, FFT_THREADS, sm, s>>>(P);                    \
    } else {                                                                                     \
      ZinvParams<dfl, float> P{};                                                                \
      P.g = g;                                                                                   \
      P.spec = spec;                                                                             \
      P.r_out = r_out;                                                                           \
      P.x_out = x_out;                                                                           \
      P.st = st;                                                                                 \
      P.partials = partials;                                                                     \
      P.tw = tw;                                                                                 \
      k_zinv4_df<A, B, float, OUT_RESID><<<nblk, FFT_THREADS, sm, s>>>(P);                       \
    }                                                                                            \
    return true;                                                                                 \
  }
    RVE_FS_SIZES(RVE_FS_ZID)
#undef RVE_FS_ZID
    default:
      return false;
  }
}

bool launch_fft_x4_df(const GridGeom& g, double scale, cplx<dfl>* spec, const cplx<dfl>* tw,
                      cudaStream_t s) {
  LineParams<dfl> P;
  P.g = g;
  P.grp = 1;
  P.scale = scale;
  P.spec = spec;
  P.done = nullptr;
  P.tw = tw;
  switch (g.nx) {
#define RVE_FS_XD(N, A, B)                                                                       \
  case N: {                                                                                      \
    constexpr int T = fs_x_t_df(N);                                                              \
    P.t = T;                                                                                     \
    const int ntiles = 3 * g.ny * ((g.hz + T - 1) / T);                                          \
    const size_t sm = sizeof(cplx<dfl>) * ((size_t)((N + 1) & ~1) + 2 * (size_t)N * T + B) +      \
                      sizeof(dfl) * ((size_t)N + T + 1);                                         \
    k_fft_x4_df<A, B><<<ntiles, FFT_THREADS, sm, s>>>(P);                                        \
    return true;                                                                                 \
  }
    RVE_FS_SIZES(RVE_FS_XD)
#undef RVE_FS_XD
    default:
      return false;
  }
}

// SMs of the current device (persistent grids: three blocks per SM)
static int sm_count() {
  static int cache[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (!cache[dev]) {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cache[dev] = sms > 0 ? sms : 1;
  }
  return cache[dev];
}

static size_t z4_smem(const GridGeom& g, bool with_r) {
  if (with_r) return z4inv_stage_off(g.nz, g.fsz_lz) + sizeof(float) * 9 * (size_t)z4inv_sp(g.nz, g.fsz_lz);
  const int LP = (5 * g.fszf_lz) | 1;
  return sizeof(cplx<float>) * ((size_t)((g.nz + 1) & ~1) + (size_t)g.nz * LP);
}

void launch_zfwd4(const ZfwdParams<float>& P0, cudaStream_t s) {
  ZfwdParams<float> P = P0;
  const GridGeom& g = P.g;
  if (g.zstage && P.tan.mode == TAN_SVK && P.tan.mat.phase && !P.tan.Sop && fs_zt_lz(g.nz) >= 1) {
    if (t_rec) {
      t_rec->bad = true;
      return;
    }
    const int lz = fs_zt_lz(g.nz);
    P.lz = lz;
    const int grid = std::min((g.nx * g.ny + lz - 1) / lz, std::max(1, g.zblk) * sm_count());
    const size_t sm = z4t_layout(g.nz, lz).total;
    switch (g.nz) {
#define RVE_FS_ZP(N, A, B)                                    \
  case N:                                                     \
    k_zfwd4p<A, B><<<grid, FFT_THREADS, sm, s>>>(P);          \
    return;
      RVE_FS_SIZES(RVE_FS_ZP)
#undef RVE_FS_ZP
      default:
        break;
    }
  }
  P.lz = g.fszf_lz;
  const int nlines = g.nx * g.ny;
  // persistent: as many thread blocks as are resident at once
  const int grid = std::min((nlines + P.lz - 1) / P.lz, std::max(1, g.zblk) * sm_count());
  const size_t sm = z4_smem(g, false);
  const int tm = P.tan.mode;
  if (t_rec) {
    if (tm != TAN_SVK && tm != TAN_SYM45) t_rec->bad = true;
    rec_add(0, P, g.nz, tm, grid, sm);
    return;
  }
  switch (g.nz) {
#define RVE_FS_ZF(N, A, B)                                                                    \
  case N:                                                                                     \
    if (tm == TAN_FULL81) k_zfwd4<float, SRC_CGPX, TAN_FULL81, A, B><<<grid, FFT_THREADS, sm, s>>>(P); \
    else if (tm == TAN_SYM45) k_zfwd4<float, SRC_CGPX, TAN_SYM45, A, B><<<grid, FFT_THREADS, sm, s>>>(P); \
    else k_zfwd4<float, SRC_CGPX, TAN_SVK, A, B><<<grid, FFT_THREADS, sm, s>>>(P);            \
    break;
    RVE_FS_SIZES(RVE_FS_ZF)
#undef RVE_FS_ZF
    default:
      break;
  }
}

void launch_zinv4(const ZinvParams<float, float>& P0, cudaStream_t s) {
  ZinvParams<float, float> P = P0;
  const GridGeom& g = P.g;
  P.lz = g.fsz_lz;
  const int nlines = g.nx * g.ny;
  const int grid = std::min((nlines + P.lz - 1) / P.lz, std::max(1, g.zblk) * sm_count());
  const size_t sm = z4_smem(g, true);
  if (t_rec) {
    if (P.mn_ell >= 0.f) t_rec->bad = true;
    rec_add(4, P, g.nz, 0, grid, sm);
    return;
  }
  switch (g.nz) {
#define RVE_FS_ZI(N, A, B)                                          \
  case N:                                                           \
    k_zinv4_cgr<float, A, B><<<grid, FFT_THREADS, sm, s>>>(P);       \
    break;
    RVE_FS_SIZES(RVE_FS_ZI)
#undef RVE_FS_ZI
    default:
      break;
  }
}

// ---------------------------------------------------------------------------
// Batched passes: block blockIdx.x runs block blk.y of cell blk.x's own
// launch of that pass (its parameters, its block count), dispatched on the
// cell's axis length.
// ---------------------------------------------------------------------------
#define RVE_FS_BATCH_SIZES(X) X(15, 5, 3) X(21, 7, 3) X(27, 9, 3) X(33, 11, 3) X(45, 9, 5) X(63, 9, 7)

namespace {
struct Fs4Tab {
  const int2* blk;
  const int* axis;
  const int* tan;
  const int* nblk;
  const char* params;
};

// out of line: each size gets its own register allocation (inlined into one
// switch, the six first-pass bodies spill heavily at the 80-register bound)
template <int TAN, int N1, int N2>
__device__ __noinline__ void zfwd4_blocks_call(const ZfwdParams<float>* P, int bid, int nblk) {
  zfwd4_blocks<float, SRC_CGPX, TAN, N1, N2>(*P, bid, nblk);
}

__global__ void __launch_bounds__(FFT_THREADS, 3) k_fs4_batch_zfwd(const Fs4Tab T) {
  const int2 b = T.blk[blockIdx.x];
  const ZfwdParams<float>& P = reinterpret_cast<const ZfwdParams<float>*>(T.params)[b.x];
  const int nb = T.nblk[b.x];
  const bool sym = T.tan[b.x] == TAN_SYM45;
  switch (T.axis[b.x]) {
#define RVE_B_ZF(N, A, B)                                                  \
  case N:                                                                  \
    if (sym) zfwd4_blocks_call<TAN_SYM45, A, B>(&P, b.y, nb);              \
    else zfwd4_blocks_call<TAN_SVK, A, B>(&P, b.y, nb);                    \
    break;
    RVE_FS_BATCH_SIZES(RVE_B_ZF)
#undef RVE_B_ZF
    default:
      break;
  }
}

template <bool INV>
__global__ void __launch_bounds__(FFT_THREADS, 4) k_fs4_batch_y(const Fs4Tab T) {
  const int2 b = T.blk[blockIdx.x];
  const LineParams<float>& P = reinterpret_cast<const LineParams<float>*>(T.params)[b.x];
  switch (T.axis[b.x]) {
#define RVE_B_Y(N, A, B)                                         \
  case N:                                                        \
    if (P.t == fs_y_t()) fft_y4_tile<float, A, B, INV, fs_y_t()>(P, b.y);   \
    else fft_y4_tile<float, A, B, INV, fs_y_t2()>(P, b.y);       \
    break;
    RVE_FS_BATCH_SIZES(RVE_B_Y)
#undef RVE_B_Y
    default:
      break;
  }
}

__global__ void __launch_bounds__(FFT_THREADS, 4) k_fs4_batch_x(const Fs4Tab T) {
  const int2 b = T.blk[blockIdx.x];
  const LineParams<float>& P = reinterpret_cast<const LineParams<float>*>(T.params)[b.x];
  switch (T.axis[b.x]) {
#define RVE_B_X(N, A, B)                                         \
  case N:                                                        \
    if (P.t == fs_x_t(N)) fft_x4_tile<float, A, B, fs_x_t(N)>(P, b.y);      \
    else fft_x4_tile<float, A, B, fs_x_t2(N)>(P, b.y);           \
    break;
    RVE_FS_BATCH_SIZES(RVE_B_X)
#undef RVE_B_X
    default:
      break;
  }
}

__global__ void __launch_bounds__(FFT_THREADS, 3) k_fs4_batch_zinv(const Fs4Tab T) {
  const int2 b = T.blk[blockIdx.x];
  const ZinvParams<float, float>& P =
      reinterpret_cast<const ZinvParams<float, float>*>(T.params)[b.x];
  const int nb = T.nblk[b.x];
  switch (T.axis[b.x]) {
#define RVE_B_ZI(N, A, B)                               \
  case N:                                               \
    zinv4_cgr_blocks<float, A, B>(P, b.y, nb);          \
    break;
    RVE_FS_BATCH_SIZES(RVE_B_ZI)
#undef RVE_B_ZI
    default:
      break;
  }
}
}  // namespace

cudaError_t fft4_kernels_init() {
  g_err4 = cudaSuccess;
#define RVE_FS_INIT(N, A, B)                                \
  allow_smem(k_fft_y4<float, A, B, true, fs_y_t()>);        \
  allow_smem(k_fft_y4<float, A, B, false, fs_y_t()>);       \
  allow_smem(k_fft_y4<float, A, B, true, fs_y_t2()>);       \
  allow_smem(k_fft_y4<float, A, B, false, fs_y_t2()>);      \
  allow_smem(k_fft_x4<float, A, B, fs_x_t(N)>);             \
  allow_smem(k_fft_x4<float, A, B, fs_x_t2(N)>);            \
  allow_smem(k_fft_x4_g0<float, A, B>);                     \
  allow_smem(k_zfwd4<float, SRC_CGPX, TAN_FULL81, A, B>);   \
  allow_smem(k_zfwd4<float, SRC_CGPX, TAN_SVK, A, B>);      \
  allow_smem(k_zfwd4<float, SRC_CGPX, TAN_SYM45, A, B>);    \
  allow_smem(k_zinv4_cgr<float, A, B>);                     \
  allow_smem(k_zfwd4p<A, B>);                               \
  allow_smem(k_fft_y4_df<A, B, true>);                      \
  allow_smem(k_fft_y4_df<A, B, false>);                     \
  allow_smem(k_fft_x4_df<A, B>);                            \
  allow_smem(k_zfwd4_df<A, B>);                             \
  allow_smem(k_zinv4_df<A, B, double, OUT_PLAIN>);          \
  allow_smem(k_zinv4_df<A, B, double, OUT_PLAIN_MEANX>);    \
  allow_smem(k_zinv4_df<A, B, float, OUT_RESID>);
  RVE_FS_SIZES(RVE_FS_INIT)
#undef RVE_FS_INIT
  allow_smem(k_fs4_batch_zfwd);
  allow_smem(k_fs4_batch_y<false>);
  allow_smem(k_fs4_batch_y<true>);
  allow_smem(k_fs4_batch_x);
  allow_smem(k_fs4_batch_zinv);
  return g_err4;
}

Fs4Batch* fs4_batch_new() { return new Fs4Batch(); }

void fs4_batch_free(Fs4Batch* b) {
  if (!b) return;
  for (auto& p : b->pass) {
    cudaFree(p.d_params);
    cudaFree(p.d_axis);
    cudaFree(p.d_tan);
    cudaFree(p.d_nblk);
    cudaFree(p.d_blk);
  }
  delete b;
}

bool fs4_batch_eligible(const GridGeom& g, bool mixed, int tan_mode, bool precond) {
  return mixed && !precond && !g.zstage && g.fsx_n1 && g.fsy_n1 && g.fsz_n1 &&
         fs4_batch_size(g.nx) && fs4_batch_size(g.ny) && fs4_batch_size(g.nz) &&
         (tan_mode == TAN_SVK || tan_mode == TAN_SYM45);
}

void fs4_batch_record(Fs4Batch* b) { t_rec = b; }

int fs4_batch_cells(const Fs4Batch* b) {
  if (!b || b->bad) return -1;
  const size_t c = b->pass[0].axis.size();
  for (const auto& p : b->pass)
    if (p.axis.size() != c) return -1;
  return (int)c;
}

cudaError_t fs4_batch_upload(Fs4Batch* b) {
  if (fs4_batch_cells(b) < 0) return cudaErrorInvalidValue;
  for (auto& p : b->pass) {
    auto put = [](auto** dst, const auto& v) {
      cudaFree(*dst);
      *dst = nullptr;
      const size_t bytes = v.size() * sizeof(v[0]);
      if (!bytes) return cudaSuccess;
      cudaError_t e = cudaMalloc(reinterpret_cast<void**>(dst), bytes);
      if (e != cudaSuccess) return e;
      return cudaMemcpy(*dst, v.data(), bytes, cudaMemcpyHostToDevice);
    };
    cudaError_t e;
    if ((e = put(&p.d_params, p.params)) != cudaSuccess) return e;
    if ((e = put(&p.d_axis, p.axis)) != cudaSuccess) return e;
    if ((e = put(&p.d_tan, p.tan)) != cudaSuccess) return e;
    if ((e = put(&p.d_nblk, p.nblk)) != cudaSuccess) return e;
    if ((e = put(&p.d_blk, p.blk)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

void fs4_batch_launch(const Fs4Batch* b, cudaStream_t s) {
  for (int k = 0; k < 5; ++k) {
    const Fs4Pass& p = b->pass[k];
    if (p.blk.empty()) continue;
    const Fs4Tab T{p.d_blk, p.d_axis, p.d_tan, p.d_nblk, p.d_params};
    const unsigned grid = (unsigned)p.blk.size();
    switch (k) {
      case 0: k_fs4_batch_zfwd<<<grid, FFT_THREADS, p.smem, s>>>(T); break;
      case 1: k_fs4_batch_y<false><<<grid, FFT_THREADS, p.smem, s>>>(T); break;
      case 2: k_fs4_batch_x<<<grid, FFT_THREADS, p.smem, s>>>(T); break;
      case 3: k_fs4_batch_y<true><<<grid, FFT_THREADS, p.smem, s>>>(T); break;
      default: k_fs4_batch_zinv<<<grid, FFT_THREADS, p.smem, s>>>(T); break;
    }
  }
}
