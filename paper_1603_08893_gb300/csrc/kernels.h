// Host-side launchers of the device kernels (implemented in the .cu files).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "common.cuh"
#include "dfloat.cuh"
#include "fft.cuh"

// tangent storage modes
enum { TAN_FULL81 = 1, TAN_SVK = 2, TAN_SYM45 = 3 };

// Packed symmetric tangent: the 9x9 matrix M[r][c] = dP_r / dF_c
// (r = 3i + j for P_ij, c = 3k + l for F_kl) is symmetric for the
// hyperelastic SVK law and the J2 update with frozen history (major symmetry
// K_ijkl = K_lkji); its upper triangle r <= c is stored row by row.
__host__ __device__ constexpr int sym45_index(int r, int c) {
  return r <= c ? r * 9 - r * (r - 1) / 2 + (c - r) : c * 9 - c * (c - 1) / 2 + (r - c);
}
// sources of the forward pass input
// SRC_CGPX: fused CG iteration front: p = r + beta p, lagged x += alpha p,
// and p.(K:p) (= p.Ap for compatible p, G being an orthogonal projector)
enum { SRC_FIELD = 0, SRC_CGP = 1, SRC_UNIFORM = 2, SRC_CGPX = 3 };
// outputs of the inverse z pass
// OUT_CGR: fused CG iteration end: r -= alpha Ap in place, r.r, CG control
enum { OUT_PLAIN = 0, OUT_CGAP = 1, OUT_RESID = 2, OUT_CGR = 3 };
// OUT_PLAIN plus the component means of the result into st->meanX (the
// float-float projection of dF on the four-step z kernels)
enum { OUT_PLAIN_MEANX = 4 };

struct GridGeom {
  int nx, ny, nz;
  int hz, hzp;        // nz/2+1 and its padded row length
  size_t n;           // nx*ny*nz
  size_t sstride;     // nx*ny*hzp (complex elements per spectrum component)
  AxisPlan px, py, pz;
  AxisPlan pxs, pys, pzs;  // prime radices only (float-float passes)
  int lz_f, lz_d;     // z lines per CTA (float, double)
  int ty_f, ty_d, gy_f, gy_d;  // y tile (kz) and groups per CTA
  int tx_f, tx_d;     // x tile (kz)
  // host-computed divisors used in index arithmetic
  FastDiv f_hz, f_lzf, f_lzd, f_ny, f_ntky_f, f_ntky_d, f_ntkx_f, f_ntkx_d;
  FastDiv f_Ly_f, f_Ly_d, f_Lx_f, f_Lx_d;  // lines per y / x tile
  // float y and x passes on the in-place four-step kernels (fs_n1 != 0:
  // the axis length has a compiled N1 x N2 split, see RVE_FS_SIZES)
  int fsy_n1, fsx_n1, fsz_n1;
  int zblk;    // persistent four-step z passes: thread blocks per SM in the grid
  int zstage;  // first z pass with TMA-staged, pipelined inputs (SVK, phase map);
               // off by default (slower at 125^3: its tiles are half as large),
               // a candidate of the autotuner
  int fsy_t, fsy_grp, fsx_t, fsz_lz, fszf_lz;
  FastDiv f_fsy_ntk, f_fsx_ntk, f_fsy_L, f_fsx_L, f_fsz_L, f_fsz_lz;
  // reference medium of the preconditioned CG (lambda0 / mu0 and
  // (lambda0 + mu0) / (lambda0 + 2 mu0), with mu0 scaled to 1)
  float pc_ell, pc_c;
  // polls of a thread block's bounded wait on its own asynchronous copies
  // before it gives up and reports a timeout (kDefaultWaitPolls; 0 in the
  // failure tests: every first wait gives up at once)
  unsigned wait_polls;
};

constexpr unsigned kDefaultWaitPolls = 1u << 20;

// Axis lengths with compiled four-step kernels: X(N, N1, N2), N = N1 N2.
#define RVE_FS_SIZES(X) \
  X(15, 5, 3)           \
  X(21, 7, 3)           \
  X(27, 9, 3)           \
  X(33, 11, 3)          \
  X(45, 9, 5)           \
  X(63, 9, 7)           \
  X(125, 5, 25)         \
  X(243, 9, 27)         \
  X(315, 21, 15)

// Tile shapes of the four-step kernels, compile-time functions of the axis
// length so that every shared-memory offset of a DFT work item is constant.
constexpr int fs_y_t() { return 16; }  // kz values per y tile row (128 bytes)
// The autotuner's alternative tile heights (half the kz values per tile, so
// twice the tiles, half the shared memory each): y pass 8, x pass fs_x_t / 2.
constexpr int fs_y_t2() { return 8; }
constexpr int fs_y_grp(int n) { return 49152 / (8 * n * 16) > 1 ? 49152 / (8 * n * 16) : 1; }
constexpr int fs_x_t(int n) {
  return 8 * 3 * n * 16 <= 65536 ? 16 : (8 * 3 * n * 8 <= 65536 ? 8 : 4);
}
constexpr int fs_x_t2(int n) { return fs_x_t(n) / 2 >= 2 ? fs_x_t(n) / 2 : fs_x_t(n); }
// first z pass: tiles of about 32 KB (larger tiles measured slower)
// x pass of the preconditioned iteration: all nine components per tile
// (the reference-medium operator couples the tensor rows), tiles of at most
// 96 KB
constexpr int fs_x_t_g0(int n) {
  return 72 * n * 16 <= 98304 ? 16 : (72 * n * 8 <= 98304 ? 8 : (72 * n * 4 <= 98304 ? 4 : 2));
}
constexpr int fs_zf_lz(int n) {
  return (32768 / (8 * n) - 1) / 5 < 1 ? 1 : ((32768 / (8 * n) - 1) / 5 > 64 ? 64 : (32768 / (8 * n) - 1) / 5);
}
constexpr int fs_z_lz(int n) {
  return (32768 / (8 * n) - 1) / 5 < 1 ? 1 : ((32768 / (8 * n) - 1) / 5 > 64 ? 64 : (32768 / (8 * n) - 1) / 5);
}

// Shared-memory layout (bytes) of the TMA-staged first z pass: twiddles |
// transposed DFT buffer | staged inputs [36][sp] floats | staged phase bytes.
struct Z4tLayout {
  int lp, sp, spb;
  size_t stage_off, phase_off, total;
};

__host__ __device__ constexpr Z4tLayout z4t_layout(int nz, int lz) {
  Z4tLayout L{};
  L.lp = (5 * lz) | 1;
  L.sp = (lz * nz + 8 + 3) & ~3;
  L.spb = (lz * nz + 32 + 15) & ~15;
  const size_t head = 8 * ((size_t)((nz + 1) & ~1) + (size_t)nz * L.lp);
  L.stage_off = (head + 15) & ~(size_t)15;
  L.phase_off = L.stage_off + 4 * 36 * (size_t)L.sp;
  L.total = L.phase_off + (size_t)L.spb;
  return L;
}

// Last z pass: twiddles | transposed DFT buffer | r staged per component
// ([9][sp] floats, 16-byte aligned)
__host__ __device__ constexpr int z4inv_sp(int nz, int lz) { return (lz * nz + 8 + 3) & ~3; }
__host__ __device__ constexpr size_t z4inv_stage_off(int nz, int lz) {
  return (8 * ((size_t)((nz + 1) & ~1) + (size_t)nz * ((5 * lz) | 1)) + 15) & ~(size_t)15;
}

// z lines per tile of the staged pass: the most that fit 72 KB (three
// thread blocks per SM); 0 if not even one line fits
constexpr int fs_zt_lz(int nz) {
  int best = 0;
  for (int lz = 1; lz <= 64; ++lz)
    if (z4t_layout(nz, lz).total <= 72 * 1024) best = lz;
  return best;
}

inline int fs_split_n1(int n) {
  switch (n) {
#define RVE_FS_CASE(N, A, B) \
  case N:                    \
    return A;
    RVE_FS_SIZES(RVE_FS_CASE)
#undef RVE_FS_CASE
    default:
      return 0;
  }
}

// a 3x3 tensor passed by value to a kernel (row-major)
struct W9 {
  double w[9];
};

template <typename R>
struct TangentView {
  int mode;           // TAN_FULL81 / TAN_SYM45 / TAN_SVK / 0 (plain copy)
  const R* K4;        // [81][n] (FULL81) or [45][n] (SYM45)
  const R* Fop;       // [9][n]
  const R* Sop;       // [6][n] or null (compute S from F)
  MatView<R> mat;     // lambda, mu
};

template <typename R>
struct Twiddles {
  const cplx<R>* x;
  const cplx<R>* y;
  const cplx<R>* z;
};

// Forward transform chain front: (optional p-update) -> tangent -> R2C along z.
template <typename R>
void launch_zfwd(const GridGeom& g, int src, const TangentView<R>& tan, const R* field, const R* r,
                 R* p, const double* unif, SolverState* st, const int* done, cplx<R>* spec,
                 const Twiddles<R>& tw, cudaStream_t s, R* x = nullptr, double* partials = nullptr);
template <typename R>
void launch_fft_y(const GridGeom& g, bool inverse, cplx<R>* spec, const int* done,
                  const Twiddles<R>& tw, cudaStream_t s);
// gamma0: the reference-medium Green operator (preconditioned CG, float
// four-step x lengths only) in place of G-hat
template <typename R>
void launch_fft_x_proj(const GridGeom& g, double scale, cplx<R>* spec, const int* done,
                       const Twiddles<R>& tw, cudaStream_t s, bool gamma0 = false);
// Inverse z transform and output stage.
// mnorm: the CG reductions of OUT_CGR / OUT_RESID take the reference-medium
// norm z.(K0:z) instead of z.z (preconditioned CG)
template <typename R, typename RC>
void launch_zinv(const GridGeom& g, int out, const cplx<R>* spec, R* dst, RC* r_out, RC* x_out,
                 const RC* p_in, SolverState* st, double* partials, const int* done,
                 const Twiddles<R>& tw, cudaStream_t s, bool mnorm = false);

// four-step float kernels (kernels_fft4.cu); used when g.fsy_n1 / g.fsx_n1
void launch_fft_y4(const GridGeom& g, bool inverse, cplx<float>* spec, const int* done,
                   const cplx<float>* tw, cudaStream_t s);
void launch_fft_x4(const GridGeom& g, double scale, cplx<float>* spec, const int* done,
                   const cplx<float>* tw, cudaStream_t s, bool gamma0 = false);
// the y and x passes of G in float-float arithmetic on the four-step
// kernels; false (nothing launched) when the axis has no four-step split
bool launch_fft_y4_df(const GridGeom& g, bool inverse, cplx<dfl>* spec, const cplx<dfl>* tw,
                      cudaStream_t s);
bool launch_fft_x4_df(const GridGeom& g, double scale, cplx<dfl>* spec, const cplx<dfl>* tw,
                      cudaStream_t s);
// the z passes of G in float-float on the four-step kernels (float64 field
// in; OUT_PLAIN: float64 out, OUT_RESID: float32 r, x = 0, CG start)
bool launch_zfwd4_df(const GridGeom& g, const double* in, cplx<dfl>* spec, const cplx<dfl>* tw,
                     cudaStream_t s);
bool launch_zinv4_df(const GridGeom& g, int out_mode, const cplx<dfl>* spec, double* out64,
                     float* r_out, float* x_out, SolverState* st, double* partials,
                     const cplx<dfl>* tw, cudaStream_t s);
// per-voxel parameters in device memory to the internal form (kernels_mat.cu)
void launch_voxel_params(const double* vp, size_t n, int nparam, double* v64, float* v32,
                         double* sums, double* partials, unsigned int* counter, cudaStream_t s);
cudaError_t fft4_kernels_init();

// Batched passes of the fused float32 CG iteration (kernels_fft4.cu) for
// cells whose three axes all have four-step kernels of the batch sizes
// (15, 21, 27, 33, 45, 63).  While a batch records on this host thread, the
// four-step launchers store each launch (parameters, grid, shared memory)
// in it instead of launching; fs4_batch_launch then runs each of the five
// passes of one CG iteration for every recorded cell in ONE launch, every
// cell's blocks doing exactly what its own launch would (same tiles, same
// block count, same reductions), so results are bit-identical to solving
// the cell alone.
struct Fs4Batch;
Fs4Batch* fs4_batch_new();
void fs4_batch_free(Fs4Batch* b);
bool fs4_batch_eligible(const GridGeom& g, bool mixed, int tan_mode, bool precond);
void fs4_batch_record(Fs4Batch* b);  // nullptr ends recording
int fs4_batch_cells(const Fs4Batch* b);
cudaError_t fs4_batch_upload(Fs4Batch* b);  // device copies of the launch tables
void fs4_batch_launch(const Fs4Batch* b, cudaStream_t s);

// G : in in float-float arithmetic on the float32 pipe (float64 in and out):
// out_mode OUT_PLAIN writes out64 = scale * G:in; OUT_RESID writes
// r_out = scale * G:in (float32), x_out = 0 and initialises the CG state;
// OUT_PLAIN_MEANX is OUT_PLAIN that also stores the component means of the
// result in st->meanX where the z axis has four-step kernels.  Returns
// whether the means were stored.
bool launch_G_df(const GridGeom& g, const double* in, double scale, int out_mode, double* out64,
                 float* r_out, float* x_out, SolverState* st, double* partials, cplx<dfl>* spec,
                 const Twiddles<dfl>& tw, cudaStream_t s);

// out9 = < K : (U + x) > over the voxels, U a uniform tensor (device, 9
// doubles), x a [9][n] field or null; K applied as in the first z pass
template <typename R>
void launch_tangent_mean(const TangentView<R>& tan, const R* x, const double* U, size_t n,
                         double* out9, double* partials, unsigned int* counter, cudaStream_t s);

cudaError_t fft_kernels_init();  // opt-in to large dynamic shared memory
size_t fft_max_blocks(const GridGeom& g);

// ---- vector / material kernels (kernels_mat.cu) ----
template <typename R>
void launch_cg_finish(size_t n9, R* x, const R* p, const SolverState* st, cudaStream_t s);
template <typename R>
void launch_cg_update(size_t n9, R* x, R* r, const R* p, const R* Ap, SolverState* st,
                      double* partials, cudaStream_t s);
template <typename T>
void launch_mean9(const T* A, size_t n, double* out9, double* partials, unsigned int* counter,
                  int post, SolverState* st, cudaStream_t s);
void launch_shifted_norm(const double* F, size_t n, SolverState* st, double* partials,
                         cudaStream_t s);
template <typename RC>
void launch_newton_update(double* F, const RC* x, size_t n, SolverState* st, double* partials,
                          int add_dfbar, cudaStream_t s);
template <typename RO>
void launch_svk_constitutive(const double* F, size_t n, MatView<double> mat, double* P,
                             int tan_mode, RO* K4, RO* Fop, RO* Sop, SolverState* st,
                             cudaStream_t s);
// the SVK update of mixed handles with the recomputed tangent in float-float
// arithmetic (P float64, Fop = F in float32; no K4, no S)
void launch_svk_constitutive_df(const double* F, size_t n, MatView<double> mat, double* P,
                                float* Fop, SolverState* st, cudaStream_t s);
void launch_svk_k4_full(const double* F, size_t v0, size_t count, size_t n,
                        MatView<double> mat, double* dst, cudaStream_t s);
template <typename Ti, typename To>
void launch_convert(const Ti* in, To* out, size_t count, cudaStream_t s);

template <typename RC>
void launch_cg_init(size_t n9, const double* b, const double* Ax, RC* r, RC* x, SolverState* st,
                    double* partials, cudaStream_t s);
template <typename RC>
void launch_accumulate(size_t n9, double* y, const RC* x, cudaStream_t s);
void launch_adjoint_grad(const double* F, const double* lam, const double W[9], size_t n, double* g,
                         double* gK, cudaStream_t s);

// ---- finite-strain J2 (kernels_j2.cu) ----
template <typename RO>
void launch_j2_constitutive(const double* F, size_t n, MatView<double> mat, const double* hc,
                            double* ht, double* P, RO* K4, SolverState* st, cudaStream_t s,
                            int sym45 = 0);
void launch_j2_k4_full(const double* F, size_t v0, size_t count, size_t n, MatView<double> mat,
                       const double* hc, double* dst, cudaStream_t s);
// reverse sweep of the J2 adjoint through the history of a path (central
// differences of the return map): gF = (dH/dF)^T a; one backward step with
// c = W/n [last] - lambda: g += c : dP/dp + a . dH/dp, a_out = c : dP/dh + a . dH/dh
void launch_j2_path_gF(const double* F, size_t n, MatView<double> mat, const double* hs,
                       const double* a, double* gF, cudaStream_t s);
void launch_j2_path_step(const double* F, size_t n, MatView<double> mat, const double* hs,
                         const double* lam, const double W[9], int last, const double* a_in,
                         double* a_out, double* g, cudaStream_t s);
// out[4][n]: dJ/d(K, mu, tau_y0, H) per voxel, J = W : P-bar, history hs fixed
void launch_j2_adjoint_grad(const double* F, size_t n, MatView<double> mat, const double* hs,
                            const double* lam, const double W[9], double* out, cudaStream_t s);
size_t vec_max_blocks();

// mean9 post-processing modes
enum { MEAN_PLAIN = 0, MEAN_DFBAR = 1, MEAN_X = 2, MEAN_PBAR = 3 };
