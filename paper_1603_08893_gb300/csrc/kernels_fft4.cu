// Float y and x passes on the in-place four-step line DFT (fs_lines) for
// axis lengths with a compiled split N = N1 N2 (RVE_FS_SIZES).  Same data
// flow as k_fft_y / k_fft_x_proj: a tile of 128-byte spectrum rows (16 kz
// values) is fetched with cp.async into ONE shared buffer, transformed in
// place and written back; the transposed order the forward transform leaves
// is undone in the addressing of the global stores (forward y), loads
// (inverse y) or of the projection (x pass).
#include "fft_pass.cuh"

namespace {

// three CTAs per SM when both factors fit the register budget
template <typename R, int N1, int N2>
struct Fs4Occ {
  static constexpr int value = (sizeof(R) == 4 && N1 <= 27 && N2 <= 27) ? 3 : 2;
};

// Complex DFT along y on tiles of (grp component-x rows) x ny x (T kz).
// Forward: natural rows in, transposed order in shared memory, natural rows
// out.  Inverse: rows loaded into transposed positions, natural out.
template <typename R, int N1, int N2, bool INV>
__global__ void __launch_bounds__(FFT_THREADS, (Fs4Occ<R, N1, N2>::value))
    k_fft_y4(const LineParams<R> P) {
  constexpr int N = N1 * N2;
  if (P.done && *P.done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int T = P.t, grp = P.grp;
  const int ts = __ffs(T) - 1;
  cplx<R>* tw = reinterpret_cast<cplx<R>*>(smem_raw);
  cplx<R>* buf = tw + ((N + 1) & ~1);
  const int hz = P.g.hz, hzp = P.g.hzp;
  const int ngroups = 9 * P.g.nx;
  const int ntk = (hz + T - 1) >> ts;
  const int tile = blockIdx.x;
  const int tg = (int)P.g.f_fsy_ntk.div((unsigned)tile);
  const int k0 = (tile - tg * ntk) * T, g0 = tg * grp;
  const int ng = min(grp, ngroups - g0);
  cplx<R>* gbase = P.spec + (size_t)g0 * N * hzp + k0;
  {
    constexpr int EPC = 16 / sizeof(cplx<R>);
    const int cpr = T / EPC;
    const int cs = __ffs(cpr) - 1;
    const int nch = ng * N * cpr;
    for (int c = threadIdx.x; c < nch; c += blockDim.x) {
      const int row = c >> cs;
      const int t = (c & (cpr - 1)) * EPC;
      const int gi = row / N;
      const int y = row - gi * N;
      const int srow = INV ? gi * N + fs_pos<N1, N2>(y) : row;
      const bool ok = (k0 + t) < hzp;
      const cplx<R>* src = ok ? gbase + (size_t)row * hzp + t : P.spec;
      cp_async16(buf + (srow << ts) + t, src, ok ? 16 : 0);
    }
  }
  cp_async_commit();
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = P.tw[i];
  cp_async_wait<0>();
  __syncthreads();
  const LineMap lm{ts, N * T, 1, T, 1};
  fs_lines<R, N1, N2, INV>(buf, lm, grp * T, P.g.f_fsy_L, tw);
  const int tc = min(T, hz - k0);
  const int tot = ng * N * T;
  for (int i = threadIdx.x; i < tot; i += blockDim.x) {
    const int t = i & (T - 1);
    const int srow = i >> ts;
    const int gi = srow / N;
    const int pos = srow - gi * N;
    const int y = INV ? pos : fs_freq<N1, N2>(pos);
    if (t < tc) gbase[(size_t)(gi * N + y) * hzp + t] = buf[i];
  }
}

// Forward DFT along x, projection A_ij <- xi_j (sum_l xi_l A_il) / |xi|^2
// (Eq. G_red) in the transposed order, inverse DFT along x; tile = (tensor
// row i) x nx x (T kz) for one ky.
template <typename R, int N1, int N2>
__global__ void __launch_bounds__(FFT_THREADS, (Fs4Occ<R, N1, N2>::value))
    k_fft_x4(const LineParams<R> P) {
  constexpr int N = N1 * N2;
  if (P.done && *P.done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int ny = P.g.ny, T = P.t;
  const int ts = __ffs(T) - 1;
  cplx<R>* tw = reinterpret_cast<cplx<R>*>(smem_raw);
  cplx<R>* buf = tw + ((N + 1) & ~1);
  const int hz = P.g.hz, hzp = P.g.hzp;
  const int ntk = (hz + T - 1) >> ts;
  const size_t rs = (size_t)ny * hzp;  // stride of spectrum rows (c*nx + x)
  const int tile = blockIdx.x;
  const int q = (int)P.g.f_fsx_ntk.div((unsigned)tile);
  const int k0 = (tile - q * ntk) * T;
  const int irow = (int)P.g.f_ny.div((unsigned)q);
  const int y = q - irow * ny;
  cplx<R>* gbase = P.spec + (size_t)(3 * irow) * N * rs + (size_t)y * hzp + k0;
  issue_tile<R>(buf, gbase, rs, 3 * N, T, ts, k0, hzp, P.spec);
  cp_async_commit();
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = P.tw[i];
  cp_async_wait<0>();
  __syncthreads();
  const LineMap lm{ts, N * T, 1, T, 1};
  fs_lines<R, N1, N2, false>(buf, lm, 3 * T, P.g.f_fsx_L, tw);
  const R qy = signed_freq<R>(y, ny) / (R)ny;
  const R sc = (R)P.scale;
  for (int i = threadIdx.x; i < N * T; i += blockDim.x) {
    const int t = i & (T - 1);
    const int kx = fs_freq<N1, N2>(i >> ts);
    const R qx = signed_freq<R>(kx, N) / (R)N;
    const R qz = (R)(k0 + t) / (R)P.g.nz;
    const R q2 = qx * qx + qy * qy + qz * qz;
    const R f = (q2 > R(0)) ? sc / q2 : R(0);
    const cplx<R> A0 = buf[i], A1 = buf[N * T + i], A2 = buf[2 * N * T + i];
    const R sx = f * (qx * A0.x + qy * A1.x + qz * A2.x);
    const R sy = f * (qx * A0.y + qy * A1.y + qz * A2.y);
    buf[i] = {sx * qx, sy * qx};
    buf[N * T + i] = {sx * qy, sy * qy};
    buf[2 * N * T + i] = {sx * qz, sy * qz};
  }
  __syncthreads();
  fs_lines<R, N1, N2, true>(buf, lm, 3 * T, P.g.f_fsx_L, tw);
  const int tc = min(T, hz - k0);
  const int tot = 3 * N * T;
  for (int i = threadIdx.x; i < tot; i += blockDim.x) {
    const int t = i & (T - 1);
    if (t < tc) gbase[(size_t)(i >> ts) * rs + t] = buf[i];
  }
}

cudaError_t g_err4 = cudaSuccess;

template <typename K>
void allow_smem(K kernel) {
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 208 * 1024);
  if (e != cudaSuccess && g_err4 == cudaSuccess) g_err4 = e;
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
  switch (g.ny) {
#define RVE_FS_Y(N, A, B)                                                   \
  case N:                                                                   \
    if (inverse) k_fft_y4<float, A, B, true><<<ntiles, FFT_THREADS, sm, s>>>(P); \
    else k_fft_y4<float, A, B, false><<<ntiles, FFT_THREADS, sm, s>>>(P);   \
    break;
    RVE_FS_SIZES(RVE_FS_Y)
#undef RVE_FS_Y
    default:
      break;
  }
}

void launch_fft_x4(const GridGeom& g, double scale, cplx<float>* spec, const int* done,
                   const cplx<float>* tw, cudaStream_t s) {
  LineParams<float> P;
  P.g = g;
  P.t = g.fsx_t;
  P.grp = 1;
  P.scale = scale;
  P.spec = spec;
  P.done = done;
  P.tw = tw;
  const int ntiles = 3 * g.ny * ((g.hz + P.t - 1) / P.t);
  const size_t sm = sizeof(cplx<float>) * ((size_t)((g.nx + 1) & ~1) + 3 * (size_t)g.nx * P.t);
  switch (g.nx) {
#define RVE_FS_X(N, A, B)                                       \
  case N:                                                       \
    k_fft_x4<float, A, B><<<ntiles, FFT_THREADS, sm, s>>>(P);   \
    break;
    RVE_FS_SIZES(RVE_FS_X)
#undef RVE_FS_X
    default:
      break;
  }
}

cudaError_t fft4_kernels_init() {
  g_err4 = cudaSuccess;
#define RVE_FS_INIT(N, A, B)                  \
  allow_smem(k_fft_y4<float, A, B, true>);    \
  allow_smem(k_fft_y4<float, A, B, false>);   \
  allow_smem(k_fft_x4<float, A, B>);
  RVE_FS_SIZES(RVE_FS_INIT)
#undef RVE_FS_INIT
  return g_err4;
}
