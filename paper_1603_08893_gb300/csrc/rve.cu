// C ABI and host orchestration of the Newton-CG solver (Algorithm 1).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <tuple>
#include <mutex>
#include <map>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/rve.h"
#include "kernels.h"

namespace {

const double kDivergedUpdate = 0.5;  // ||dF||/||F|| above this ends Newton as diverged
// float32 CG stops after this many iterations without a 10% drop of ||r||
// (its accuracy limit on high-contrast cells); float64 CG never does
const int kMixedStagnation = 200;
const int kMaxMacro = 30;            // Newton iterations on the free F-bar components
const double kSingularPivot = 1e-10; // relative pivot of a singular homogenised tangent

struct TimedLaunch {
  cudaEvent_t a, b;
  long long solve;
  int iter;
};

struct Arena {
  char* base = nullptr;
  size_t off = 0, cap = 0;
  bool dry = true;
  template <typename T>
  T* take(size_t count) {
    off = (off + 255) & ~(size_t)255;
    T* p = dry ? nullptr : reinterpret_cast<T*>(base + off);
    off += count * sizeof(T);
    return p;
  }
};

bool factor_plan(int n, AxisPlan* p, bool composite = true) {
  p->n = n;
  p->nst = 0;
  int m = n;
  // pairs of small primes become one composite stage (two radix passes for
  // one trip through shared memory); then single radices
  const int fixed[] = {25, 21, 15, 9, 8, 11, 7, 5, 4, 3, 2};
  for (int f : fixed)
    while (m % f == 0 && (composite || f == 11 || f == 7 || f == 5 || f == 3 || f <= 8)) {
      if (p->nst >= RVE_MAX_STAGES) return false;
      p->rad[p->nst++] = f;
      m /= f;
    }
  for (int q = 13; m > 1; q += 2)
    while (m % q == 0) {
      if (p->nst >= RVE_MAX_STAGES) return false;
      p->rad[p->nst++] = q;
      m /= q;
    }
  {
    int ns = 1;
    for (int s = 0; s < p->nst; ++s) {
      p->fNs[s] = make_fastdiv((unsigned)ns);
      p->fnb[s] = make_fastdiv((unsigned)(n / p->rad[s]));
      ns *= p->rad[s];
    }
    p->fN = make_fastdiv((unsigned)n);
  }
  // capacity of the in-register stage scheme with 256 threads per block
  for (int s = 0; s < p->nst; ++s) {
    const int r = p->rad[s];
    const int nb = n / r;
    if (r == 3 && nb > 512) return false;
    if ((r == 5 || r == 7 || r == 11 || r == 9 || r == 15 || r == 21 || r == 25 || r == 2 ||
         r == 4 || r == 8) && nb > 1024)
      return false;
    if (r > 11 && r != 15 && r != 21 && r != 25 && n > 512) return false;
  }
  return true;
}

int pick_lz(int nz, size_t csize, size_t budget) {
  long lz = (long)((budget / csize - (size_t)nz) / (5 * (size_t)nz));
  if (lz < 1) lz = 1;
  if (lz > 64) lz = 64;
  return (int)lz;
}

bool make_geom(int nx, int ny, int nz, GridGeom* g) {
  if (nx < 1 || ny < 1 || nz < 1) return false;
  if (nx > 2047 || ny > 2047 || nz > 2047) return false;
  g->nx = nx;
  g->ny = ny;
  g->nz = nz;
  g->hz = nz / 2 + 1;
  g->hzp = (g->hz + 3) & ~3;
  g->n = (size_t)nx * ny * nz;
  g->sstride = (size_t)nx * ny * g->hzp;
  g->wait_polls = kDefaultWaitPolls;
  if (!factor_plan(nx, &g->px) || !factor_plan(ny, &g->py) || !factor_plan(nz, &g->pz)) return false;
  if (!factor_plan(nx, &g->pxs, false) || !factor_plan(ny, &g->pys, false) ||
      !factor_plan(nz, &g->pzs, false))
    return false;
  // z passes: two buffers of 5 packed lines x lz x nz (ping-pong stages)
  g->lz_f = pick_lz(nz, 8, 32 * 1024);
  g->lz_d = pick_lz(nz, 16, 32 * 1024);
  if ((size_t)16 * (nz + 1 + 10 * (size_t)g->lz_d * nz) > 200 * 1024) return false;
  // strided passes: tiles of 64-byte rows (8 float or 4 double complex kz
  // values), double buffered in shared memory
  g->ty_f = 8;
  g->ty_d = 4;
  g->gy_f = std::max(1, std::min(9 * nx, (int)(24576 / (8 * (size_t)ny * g->ty_f))));
  g->gy_d = std::max(1, std::min(9 * nx, (int)(24576 / (16 * (size_t)ny * g->ty_d))));
  if (8 * ((size_t)ny + 1 + 2 * (size_t)g->gy_f * ny * g->ty_f) > 200 * 1024) return false;
  if (16 * ((size_t)ny + 1 + 2 * (size_t)g->gy_d * ny * g->ty_d) > 200 * 1024) return false;
  g->tx_f = 8;
  g->tx_d = 4;
  g->f_hz = make_fastdiv((unsigned)g->hz);
  g->f_lzf = make_fastdiv((unsigned)g->lz_f);
  g->f_lzd = make_fastdiv((unsigned)g->lz_d);
  g->f_ny = make_fastdiv((unsigned)ny);
  g->f_ntky_f = make_fastdiv((unsigned)((g->hz + g->ty_f - 1) / g->ty_f));
  g->f_ntky_d = make_fastdiv((unsigned)((g->hz + g->ty_d - 1) / g->ty_d));
  g->f_ntkx_f = make_fastdiv((unsigned)((g->hz + g->tx_f - 1) / g->tx_f));
  g->f_ntkx_d = make_fastdiv((unsigned)((g->hz + g->tx_d - 1) / g->tx_d));
  g->f_Ly_f = make_fastdiv((unsigned)(g->gy_f * g->ty_f));
  g->f_Ly_d = make_fastdiv((unsigned)(g->gy_d * g->ty_d));
  g->f_Lx_f = make_fastdiv((unsigned)(3 * g->tx_f));
  g->f_Lx_d = make_fastdiv((unsigned)(3 * g->tx_d));
  if (8 * ((size_t)nx + 1 + 6 * (size_t)nx * g->tx_f) > 200 * 1024) return false;
  if (16 * ((size_t)nx + 1 + 6 * (size_t)nx * g->tx_d) > 200 * 1024) return false;
  // four-step float y / x passes: 128-byte tile rows (16 kz values) where
  // the tile fits 48-64 KB, about 48 lines per CTA
  g->fsy_n1 = fs_split_n1(ny);
  g->fsx_n1 = fs_split_n1(nx);
  g->fsy_t = fs_y_t();
  g->fsy_grp = fs_y_grp(ny);
  g->fsx_t = fs_x_t(nx);
  if (8 * ((size_t)nx + 1 + 3 * (size_t)nx * g->fsx_t) > 200 * 1024) g->fsx_n1 = 0;
  g->f_fsy_ntk = make_fastdiv((unsigned)((g->hz + g->fsy_t - 1) / g->fsy_t));
  g->f_fsx_ntk = make_fastdiv((unsigned)((g->hz + g->fsx_t - 1) / g->fsx_t));
  g->f_fsy_L = make_fastdiv((unsigned)(g->fsy_grp * g->fsy_t));
  g->f_fsx_L = make_fastdiv((unsigned)(3 * g->fsx_t));
  // four-step float z passes of the CG iteration: one buffer of
  // 5 lz lines x nz (about 32 KB) plus, in the last pass, the r tile
  g->fsz_n1 = fs_split_n1(nz);
  g->fsz_lz = fs_z_lz(nz);
  g->fszf_lz = fs_zf_lz(nz);
  g->zblk = 3;
  g->zstage = 0;
  g->f_fsz_L = make_fastdiv((unsigned)(5 * g->fsz_lz));
  g->f_fsz_lz = make_fastdiv((unsigned)g->fsz_lz);
  return true;
}

}  // namespace

// Grid geometry for other translation units of the library.
bool rve_internal_make_geom(int nx, int ny, int nz, GridGeom* g) { return make_geom(nx, ny, nz, g); }

struct rve_s {
  int model = RVE_SVK;
  rve_options opt{};
  cudaStream_t s = nullptr;
  GridGeom g{};
  size_t n = 0;
  bool mixed = false;
  int tan = TAN_SVK;
  int nparam = 2;
  // memory
  char* ws = nullptr;
  size_t ws_bytes = 0;
  bool own_ws = false;
  double *F = nullptr, *Ft = nullptr, *P = nullptr, *tmp64 = nullptr;
  void *x = nullptr, *r = nullptr, *p = nullptr, *Ap = nullptr;
  void* K4 = nullptr;
  void* Fop = nullptr;
  void* Sop = nullptr;
  void* spec_op = nullptr;
  cplx<double>* spec64 = nullptr;
  size_t spec64_bytes = 0;
  uint8_t* phase = nullptr;
  double* table64 = nullptr;
  float* table32 = nullptr;
  double* vox64 = nullptr;
  float* vox32 = nullptr;
  double* partials = nullptr;
  SolverState* st = nullptr;
  SolverState* hst = nullptr;  // pinned mirror
  cplx<float>* twf_all = nullptr;
  cplx<double>* twd_all = nullptr;
  cplx<dfl>* twdf_all = nullptr;
  Twiddles<float> twf{};
  Twiddles<double> twd{};
  Twiddles<dfl> twdf{};
  bool floatfloat = false;  // mixed: float64-accuracy transforms in float-float
  bool precond = false;     // reference-medium preconditioned float32 CG
  int knobs[9] = {1, 3, 1, 1, 1, 0, 0, 0, 0};  // kernel variants (rve_tuning)
  double Fbar[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
  double Fbar_committed[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};  // F-bar of the last committed state
  double* adj_b = nullptr;  // adjoint right-hand side [9][n] (SVK)
  double* adj_l = nullptr;  // adjoint solution [9][n] (SVK)
  double* hc = nullptr;     // J2 history, committed [7][n]
  double* ht = nullptr;     // J2 history, trial [7][n]
  double* hprev = nullptr;  // J2 history at the start of the last committed increment
  // J2 path tape (rve_tape): per committed increment its F and starting history
  bool tape_on = false;
  std::vector<double*> tape_F, tape_h;
  std::string err;
  long long launches = 0;
  // instrumentation
  int timing_family = -1;
  std::vector<TimedLaunch> timed;
  std::vector<cudaEvent_t> ev_pool;
  long long solve_id = 0;
  std::vector<std::pair<long long, int>> solve_iters;  // (solve id, effective iterations)
  cudaEvent_t e0 = nullptr, e1 = nullptr;
};

static void tape_clear(rve_t h);

namespace {

// NVTX range for the solver phases (visible in Nsight timelines; no cost
// without an attached tool)
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

int fail(rve_t h, int code, const std::string& msg) {
  if (h) h->err = msg;
  return code;
}

#define CK(call)                                                                       \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return fail(h, RVE_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

cudaEvent_t ev_get(rve_t h) {
  if (!h->ev_pool.empty()) {
    cudaEvent_t e = h->ev_pool.back();
    h->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}

struct FamilyTimer {
  rve_t h;
  int fam, iter;
  cudaEvent_t a = nullptr;
  FamilyTimer(rve_t h_, int fam_, int iter_) : h(h_), fam(fam_), iter(iter_) {
    if (h->timing_family == fam) {
      a = ev_get(h);
      cudaEventRecord(a, h->s);
    }
  }
  ~FamilyTimer() {
    if (a) {
      cudaEvent_t b = ev_get(h);
      cudaEventRecord(b, h->s);
      h->timed.push_back({a, b, h->solve_id, iter});
    }
  }
};

template <typename T>
T* as(void* p) { return reinterpret_cast<T*>(p); }

template <typename R>
MatView<R> mat_view(rve_t h) {
  MatView<R> m;
  m.phase = h->phase;
  m.nparam = h->nparam;
  m.n = h->n;
  if (sizeof(R) == 8) {
    m.table = reinterpret_cast<const R*>(h->table64);
    m.vox = reinterpret_cast<const R*>(h->vox64);
  } else {
    m.table = reinterpret_cast<const R*>(h->table32);
    m.vox = reinterpret_cast<const R*>(h->vox32);
  }
  return m;
}

template <typename R>
TangentView<R> tangent_view(rve_t h) {
  TangentView<R> t;
  t.mode = h->tan;
  t.K4 = as<R>(h->K4);
  t.Fop = as<R>(h->Fop);
  t.Sop = as<R>(h->Sop);
  t.mat = mat_view<R>(h);
  return t;
}

template <typename R>
const Twiddles<R>& twiddles(rve_t h);
template <>
const Twiddles<float>& twiddles<float>(rve_t h) { return h->twf; }
template <>
const Twiddles<double>& twiddles<double>(rve_t h) { return h->twd; }

// one CG iteration on the device, Ap = G:(K:p) through five passes.
// float64 (the oracle's recurrence): the p-update is fused into the first
// pass, p.Ap into the last, then a vector pass updates x and r.
// float32: the whole iteration lives in the five passes.  The first pass
// forms p, applies the previous step x += alpha p_prev and reduces
// p.(K:p), which equals p.Ap because p is compatible and G an orthogonal
// projector, so alpha is known before the inverse transforms; the last pass
// updates r -= alpha Ap in place and Ap is never stored.  x lags one step;
// enqueue_cg_finish adds the last one.
template <typename R>
void enqueue_cg_iteration(rve_t h, int iter) {
  const GridGeom& g = h->g;
  const Twiddles<R>& tw = twiddles<R>(h);
  const int* done = &h->st->done;
  cplx<R>* spec = as<cplx<R>>(h->spec_op);
  constexpr bool fused = std::is_same<R, float>::value;
  {
    FamilyTimer t(h, 0, iter);
    if (fused)
      launch_zfwd<R>(g, SRC_CGPX, tangent_view<R>(h), nullptr, as<R>(h->r), as<R>(h->p),
                     nullptr, h->st, done, spec, tw, h->s, as<R>(h->x), h->partials);
    else
      launch_zfwd<R>(g, SRC_CGP, tangent_view<R>(h), nullptr, as<R>(h->r), as<R>(h->p),
                     nullptr, h->st, done, spec, tw, h->s);
  }
  {
    FamilyTimer t(h, 1, iter);
    launch_fft_y<R>(g, false, spec, done, tw, h->s);
  }
  {
    FamilyTimer t(h, 2, iter);
    launch_fft_x_proj<R>(g, 1.0 / (double)h->n, spec, done, tw, h->s, fused && h->precond);
  }
  {
    FamilyTimer t(h, 3, iter);
    launch_fft_y<R>(g, true, spec, done, tw, h->s);
  }
  if (fused) {
    FamilyTimer t(h, 4, iter);
    launch_zinv<R, R>(g, OUT_CGR, spec, nullptr, as<R>(h->r), nullptr, nullptr, h->st,
                      h->partials, done, tw, h->s, h->precond);
    h->launches += 5;
    return;
  }
  {
    FamilyTimer t(h, 4, iter);
    launch_zinv<R, R>(g, OUT_CGAP, spec, as<R>(h->Ap), nullptr, nullptr, as<R>(h->p), h->st,
                      h->partials, done, tw, h->s);
  }
  {
    FamilyTimer t(h, 5, iter);
    launch_cg_update<R>(9 * h->n, as<R>(h->x), as<R>(h->r), as<R>(h->p), as<R>(h->Ap), h->st,
                        h->partials, h->s);
  }
  h->launches += 6;
}

// Preconditioned CG (reference medium, float32 path): the residual r of
// the right-hand side just set up is replaced by z = Gamma0 r (the inverse
// acoustic tensor of K0 applied in Fourier space, in the x pass) and the CG
// state restarts on it with the norm z.(K0:z) = r.z.  The iteration then
// updates z instead of r: z -= alpha Gamma0 (K:p), one transform round trip
// per iteration as without preconditioning; p.Ap = p.(K:p) as before.
void enqueue_precondition(rve_t h) {
  const GridGeom& g = h->g;
  const Twiddles<float>& tw = h->twf;
  cplx<float>* spec = as<cplx<float>>(h->spec_op);
  TangentView<float> plain{};
  plain.mode = 0;
  launch_zfwd<float>(g, SRC_FIELD, plain, as<float>(h->r), nullptr, nullptr, nullptr, h->st,
                     nullptr, spec, tw, h->s);
  launch_fft_y<float>(g, false, spec, nullptr, tw, h->s);
  launch_fft_x_proj<float>(g, 1.0 / (double)h->n, spec, nullptr, tw, h->s, true);
  launch_fft_y<float>(g, true, spec, nullptr, tw, h->s);
  launch_zinv<float, float>(g, OUT_RESID, spec, nullptr, as<float>(h->r), as<float>(h->x), nullptr,
                            h->st, h->partials, nullptr, tw, h->s, true);
  h->launches += 5;
}

// The last lagged step x += alpha p of a float32 CG solve.
template <typename R>
void enqueue_cg_finish(rve_t h) {
  if (!std::is_same<R, float>::value) return;
  launch_cg_finish<R>(9 * h->n, as<R>(h->x), as<R>(h->p), h->st, h->s);
  h->launches += 1;
}

// b = -G:P in float64 (float-float for mixed handles by default); r = b (in
// the CG precision), x = 0, CG state reset.
template <typename RC>
void enqueue_residual(rve_t h) {
  const GridGeom& g = h->g;
  if (std::is_same<RC, float>::value && h->floatfloat) {
    launch_G_df(g, h->P, -1.0 / (double)h->n, OUT_RESID, nullptr, as<float>(h->r),
                as<float>(h->x), h->st, h->partials, reinterpret_cast<cplx<dfl>*>(h->spec64),
                h->twdf, h->s);
    h->launches += 5;
    return;
  }
  TangentView<double> plain{};
  plain.mode = 0;
  launch_zfwd<double>(g, SRC_FIELD, plain, h->P, nullptr, nullptr, nullptr, h->st, nullptr,
                      h->spec64, h->twd, h->s);
  launch_fft_y<double>(g, false, h->spec64, nullptr, h->twd, h->s);
  launch_fft_x_proj<double>(g, -1.0 / (double)h->n, h->spec64, nullptr, h->twd, h->s);
  launch_fft_y<double>(g, true, h->spec64, nullptr, h->twd, h->s);
  launch_zinv<double, RC>(g, OUT_RESID, h->spec64, nullptr, as<RC>(h->r), as<RC>(h->x), nullptr,
                          h->st, h->partials, nullptr, h->twd, h->s);
  h->launches += 5;
}

// buf <- G : buf in float64 (Eq. weak:discr:FFT-intermediate), in place;
// in float-float arithmetic for mixed handles unless hardware float64 is
// asked for.
// With mean_x, also the component means of the result into st->meanX
// where the float-float passes can fuse them; returns whether they did.
bool enqueue_project_fp64(rve_t h, double* buf, bool allow_floatfloat = true,
                          bool mean_x = false) {
  const GridGeom& g = h->g;
  if (h->floatfloat && allow_floatfloat) {
    const bool m = launch_G_df(g, buf, 1.0 / (double)h->n, mean_x ? (int)OUT_PLAIN_MEANX : (int)OUT_PLAIN,
                               buf, nullptr, nullptr, h->st, h->partials,
                               reinterpret_cast<cplx<dfl>*>(h->spec64), h->twdf, h->s);
    h->launches += 5;
    return m;
  }
  TangentView<double> plain{};
  plain.mode = 0;
  launch_zfwd<double>(g, SRC_FIELD, plain, buf, nullptr, nullptr, nullptr, h->st, nullptr,
                      h->spec64, h->twd, h->s);
  launch_fft_y<double>(g, false, h->spec64, nullptr, h->twd, h->s);
  launch_fft_x_proj<double>(g, 1.0 / (double)h->n, h->spec64, nullptr, h->twd, h->s);
  launch_fft_y<double>(g, true, h->spec64, nullptr, h->twd, h->s);
  launch_zinv<double, double>(g, OUT_PLAIN, h->spec64, buf, nullptr, nullptr, nullptr, h->st,
                              h->partials, nullptr, h->twd, h->s);
  h->launches += 5;
  return false;
}

// Newton update of a mixed handle from its float32 CG solution x: dF = x in
// float64, projected onto the compatible fields (float32 CG leaves dF
// compatible only up to float32 round-off amplified by the cancellation in
// the CG sum; Sec. 2.3), its mean (zero up to round-off, Eq. mean:zero)
// removed, F += dF (+ dF-bar on the first iteration of an increment).
template <typename R>
void enqueue_mixed_update(rve_t h, bool first) {
  launch_convert<R, double>(as<R>(h->x), h->tmp64, 9 * h->n, h->s);
  if (!enqueue_project_fp64(h, h->tmp64, true, true)) {
    launch_mean9<double>(h->tmp64, h->n, nullptr, h->partials, &h->st->counter[SLOT_MEAN],
                         MEAN_X, h->st, h->s);
    h->launches += 1;
  }
  launch_newton_update<double>(h->F, h->tmp64, h->n, h->st, h->partials, first, h->s);
  h->launches += 2;
}

// Float64 view of the SVK tangent at the current F (mixed handles keep only
// float32 tangent data, so S is recomputed from F).
TangentView<double> tangent64_view(rve_t h) {
  if (!h->mixed) {
    TangentView<double> t = tangent_view<double>(h);
    if (t.mode == TAN_SVK) t.Fop = h->F;
    return t;
  }
  TangentView<double> t{};
  t.mode = TAN_SVK;
  t.K4 = nullptr;
  t.Fop = h->F;
  t.Sop = nullptr;
  t.mat = mat_view<double>(h);
  return t;
}

// out = G : (K : in) in float64 (src SRC_FIELD) or G : (K : U) for the
// uniform field U stored in the device state (src SRC_UNIFORM); scale 1/n.
void enqueue_operator64(rve_t h, int src, const double* in, const double* unif, double* out) {
  const GridGeom& g = h->g;
  launch_zfwd<double>(g, src, tangent64_view(h), in, nullptr, nullptr, unif, h->st, nullptr,
                      h->spec64, h->twd, h->s);
  launch_fft_y<double>(g, false, h->spec64, nullptr, h->twd, h->s);
  launch_fft_x_proj<double>(g, 1.0 / (double)h->n, h->spec64, nullptr, h->twd, h->s);
  launch_fft_y<double>(g, true, h->spec64, nullptr, h->twd, h->s);
  launch_zinv<double, double>(g, OUT_PLAIN, h->spec64, out, nullptr, nullptr, nullptr, h->st,
                              h->partials, nullptr, h->twd, h->s);
  h->launches += 5;
}

// predictor right-hand side b = -G:(K_(0) : dFbar) (Eq. bc:lin) in the
// operator precision; dFbar = Fbar - <F> computed on the device.
// With from_mean false the uniform field is the dFbar already in the device
// state (a column of the homogenised tangent).
template <typename R>
void enqueue_predictor(rve_t h, bool from_mean = true) {
  const GridGeom& g = h->g;
  const Twiddles<R>& tw = twiddles<R>(h);
  cplx<R>* spec = as<cplx<R>>(h->spec_op);
  if (from_mean) {
    launch_mean9<double>(h->F, h->n, nullptr, h->partials, &h->st->counter[SLOT_MEAN], MEAN_DFBAR,
                         h->st, h->s);
    h->launches += 1;
  }
  launch_zfwd<R>(g, SRC_UNIFORM, tangent_view<R>(h), nullptr, nullptr, nullptr, h->st->dFbar,
                 h->st, nullptr, spec, tw, h->s);
  launch_fft_y<R>(g, false, spec, nullptr, tw, h->s);
  launch_fft_x_proj<R>(g, -1.0 / (double)h->n, spec, nullptr, tw, h->s);
  launch_fft_y<R>(g, true, spec, nullptr, tw, h->s);
  launch_zinv<R, R>(g, OUT_RESID, spec, nullptr, as<R>(h->r), as<R>(h->x), nullptr, h->st,
                    h->partials, nullptr, tw, h->s);
  h->launches += 5;
}

int enqueue_constitutive(rve_t h) {
  NvtxRange nv("rve constitutive");
  MatView<double> m = mat_view<double>(h);
  cudaMemsetAsync(&h->st->err_flags, 0, sizeof(int), h->s);  // flags of this evaluation only
  if (h->model == RVE_J2) {
    const int sym = h->tan == TAN_SYM45;
    if (h->mixed)
      launch_j2_constitutive<float>(h->F, h->n, m, h->hc, h->ht, h->P, as<float>(h->K4), h->st, h->s,
                                    sym);
    else
      launch_j2_constitutive<double>(h->F, h->n, m, h->hc, h->ht, h->P, as<double>(h->K4), h->st,
                                     h->s, sym);
    h->launches += 1;
    return RVE_OK;
  }
  if (h->mixed && h->floatfloat && h->tan == TAN_SVK)
    launch_svk_constitutive_df(h->F, h->n, m, h->P, as<float>(h->Fop), h->st, h->s);
  else if (h->mixed)
    launch_svk_constitutive<float>(h->F, h->n, m, h->P, h->tan, as<float>(h->K4),
                                   as<float>(h->Fop), nullptr, h->st, h->s);
  else
    launch_svk_constitutive<double>(h->F, h->n, m, h->P, h->tan, as<double>(h->K4), nullptr,
                                    as<double>(h->Sop), h->st, h->s);
  h->launches += 1;
  return RVE_OK;
}

int sync_state(rve_t h) {
  CK(cudaMemcpyAsync(h->hst, h->st, sizeof(SolverState), cudaMemcpyDeviceToHost, h->s));
  CK(cudaStreamSynchronize(h->s));
  return RVE_OK;
}

int push_state(rve_t h) {
  CK(cudaMemcpyAsync(h->st, h->hst, sizeof(SolverState), cudaMemcpyHostToDevice, h->s));
  return RVE_OK;
}

// CG loop: iterations are enqueued in chunks; kernels of iterations after
// convergence return at once (device flag), so overshoot costs launches only.
template <typename R>
int cg_solve(rve_t h, int* iters) {
  NvtxRange nv("rve cg_solve");
  int launched = 0;
  int chunk = 4;
  h->solve_id++;
  if (std::is_same<R, float>::value && h->precond) enqueue_precondition(h);
  int rc = sync_state(h);
  if (rc) return rc;
  while (!h->hst->done) {
    for (int k = 0; k < chunk; ++k) enqueue_cg_iteration<R>(h, launched + k);
    launched += chunk;
    CK(cudaGetLastError());
    rc = sync_state(h);
    if (rc) return rc;
    if (h->hst->done) break;
    // the device counts iterations and stops at maxit; this host bound only
    // guards against a state that no longer advances
    if (launched > h->hst->maxit + 4096)
      return fail(h, RVE_ERR_TIMEOUT, "CG state stopped advancing");
    const int it = h->hst->it;
    const double rr = h->hst->rr, bb = h->hst->bb, tol2 = h->hst->tol2;
    int pred = chunk;
    if (it > 0 && rr < bb && rr > 0.0 && tol2 > 0.0) {
      const double rate = std::log(rr / bb) / it;  // log decrease per iteration (<0)
      const double need = std::log(tol2 / rr) / rate;
      pred = (int)std::ceil(need * 1.05) + 1;
    }
    chunk = std::max(2, std::min(pred, 256));
    chunk = std::min(chunk, std::max(1, h->hst->maxit - it));
  }
  enqueue_cg_finish<R>(h);
  *iters = h->hst->it;
  h->solve_iters.push_back({h->solve_id, h->hst->it});
  // float32 CG can reach p.Ap = 0 once its residual is at the float32 noise
  // level; the iterate so far is kept and the float64 Newton residual
  // decides whether more work is needed.
  if (h->mixed && h->hst->status == RVE_DEV_ERR_CG_BREAKDOWN && h->hst->it >= 1) return RVE_OK;
  return h->hst->status;
}

// Flags of the last constitutive evaluation.  A Newton iterate may pass
// through det F <= 0 in some voxel (the stress is still defined); only the
// converged state (final = true) must have det F > 0 everywhere.
int check_flags(rve_t h, bool final = true) {
  if (h->hst->err_flags & 2) return fail(h, RVE_ERR_NONFINITE, "non-finite stress or det F");
  if (final && (h->hst->err_flags & 1)) return fail(h, RVE_ERR_DETF, "det F <= 0 in some voxel");
  return RVE_OK;
}

int copy_in(rve_t h, void* dst, const void* src, size_t bytes, int on_device) {
  CK(cudaMemcpyAsync(dst, src, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                     h->s));
  return RVE_OK;
}

int copy_out(rve_t h, void* dst, const void* src, size_t bytes, int on_device) {
  CK(cudaMemcpyAsync(dst, src, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                     h->s));
  CK(cudaStreamSynchronize(h->s));
  return RVE_OK;
}

size_t layout(rve_t h, Arena& a) {
  const size_t n = h->n, n9 = 9 * n;
  const size_t ro = h->mixed ? 4 : 8;
  const size_t ns = 9 * h->g.sstride;
  h->F = a.take<double>(n9);
  h->Ft = a.take<double>(n9);
  h->P = a.take<double>(n9);
  h->tmp64 = a.take<double>(n9);
  h->x = a.take<char>(n9 * ro);
  h->r = a.take<char>(n9 * ro);
  h->p = a.take<char>(n9 * ro);
  h->Ap = a.take<char>(n9 * ro);
  h->K4 = nullptr;
  h->Fop = nullptr;
  h->Sop = nullptr;
  if (h->tan == TAN_FULL81) {
    h->K4 = a.take<char>(81 * n * ro);
  } else if (h->tan == TAN_SYM45) {
    h->K4 = a.take<char>(45 * n * ro);
  } else {
    if (h->mixed) h->Fop = a.take<char>(n9 * ro);
    else h->Sop = a.take<char>(6 * n * ro);
  }
  h->spec64 = a.take<cplx<double>>(ns);
  h->spec64_bytes = ns * sizeof(cplx<double>);
  h->spec_op = h->mixed ? (void*)a.take<cplx<float>>(ns) : (void*)h->spec64;
  if (h->model == RVE_J2) {
    h->hc = a.take<double>(7 * n);
    h->ht = a.take<double>(7 * n);
    h->hprev = a.take<double>(7 * n);
  } else {
    h->hc = h->ht = h->hprev = nullptr;
  }
  h->adj_b = a.take<double>(n9);
  h->adj_l = a.take<double>(n9);
  h->table64 = a.take<double>(256 * 4);
  h->table32 = a.take<float>(256 * 4);
  h->vox64 = nullptr;
  h->vox32 = nullptr;
  const size_t blocks = std::max(fft_max_blocks(h->g), vec_max_blocks());
  h->partials = a.take<double>(blocks * 9 + 64);
  h->st = a.take<SolverState>(1);
  const int gx[3] = {h->g.nx, h->g.ny, h->g.nz};
  h->twf_all = a.take<cplx<float>>((size_t)gx[0] + gx[1] + gx[2]);
  h->twd_all = a.take<cplx<double>>((size_t)gx[0] + gx[1] + gx[2]);
  h->twdf_all = a.take<cplx<dfl>>((size_t)gx[0] + gx[1] + gx[2]);
  return a.off;
}

size_t layout_material(rve_t h, Arena& a, bool use_phase) {
  if (use_phase) {
    h->phase = a.take<uint8_t>(h->n);
  } else {
    h->phase = nullptr;
    h->vox64 = a.take<double>((size_t)h->nparam * h->n);
    h->vox32 = h->mixed ? a.take<float>((size_t)h->nparam * h->n) : nullptr;
  }
  // slack after the last array: bulk copies read the 16-byte-aligned span
  // around a range, up to 15 bytes past an array's end
  a.take<char>(256);
  return a.off;
}

// ---------------------------------------------------------------------------
// Autotuner of the float32 CG iteration (not in the paper).  Knobs: the
// DFT engine of each pass (four-step kernels where the axis length has a
// compiled split, else Stockham), the grid of the persistent z passes
// (blocks per SM), composite radices in the Stockham plans and the
// TMA-staged first z pass.  Coordinate
// descent from the defaults; each candidate is timed on the handle itself
// (CUDA events, the best of three runs of eight CG iterations on a predictor
// right-hand side, after two warm-up iterations).  Results are cached per
// (grid, device, tangent) for the process.
// ---------------------------------------------------------------------------
struct TuneKey {
  int nx, ny, nz, dev, tan;
  bool operator<(const TuneKey& o) const {
    return std::tie(nx, ny, nz, dev, tan) < std::tie(o.nx, o.ny, o.nz, o.dev, o.tan);
  }
};
// autotuner knobs: the six of rve_tuning knobs[0..5], then the x and y tile
// heights (0 default, 1 half)
typedef std::array<int, 8> Knobs;
std::mutex g_tune_mu;
std::map<TuneKey, Knobs> g_tune_cache;

void apply_knobs(rve_t h, const Knobs& k) {
  GridGeom& g = h->g;
  GridGeom base;
  make_geom(g.nx, g.ny, g.nz, &base);
  g.fsz_n1 = k[0] ? base.fsz_n1 : 0;
  g.zblk = k[1];
  g.fsy_n1 = k[2] ? base.fsy_n1 : 0;
  g.fsx_n1 = k[3] ? base.fsx_n1 : 0;
  g.px = k[4] ? base.px : base.pxs;
  g.py = k[4] ? base.py : base.pys;
  g.pz = k[4] ? base.pz : base.pzs;
  g.zstage = k[5];
  // tile heights of the four-step x and y passes: the default or half
  g.fsx_t = k[6] ? fs_x_t2(g.nx) : fs_x_t(g.nx);
  g.fsy_t = k[7] ? fs_y_t2() : fs_y_t();
  g.f_fsy_ntk = make_fastdiv((unsigned)((g.hz + g.fsy_t - 1) / g.fsy_t));
  g.f_fsx_ntk = make_fastdiv((unsigned)((g.hz + g.fsx_t - 1) / g.fsx_t));
  g.f_fsy_L = make_fastdiv((unsigned)(g.fsy_grp * g.fsy_t));
  g.f_fsx_L = make_fastdiv((unsigned)(3 * g.fsx_t));
  for (int i = 0; i < 6; ++i) h->knobs[i] = k[i];
  h->knobs[7] = k[6];
  h->knobs[8] = k[7];
}

// Milliseconds per float32 CG iteration with the current knobs; < 0 if the
// CG state did not stay active.
double time_cg_iteration(rve_t h) {
  SolverState* hs = h->hst;
  std::memset(hs, 0, sizeof(SolverState));
  hs->cg_tol = 0.0;
  hs->cg_atol = 0.0;
  hs->maxit = 1 << 30;
  for (int c = 0; c < 9; ++c) hs->Fbar[c] = (c % 4 == 0 ? 1.0 : 0.0) + (c == 1 ? 0.01 : 0.0);
  if (push_state(h)) return -1.0;
  enqueue_predictor<float>(h);
  for (int k = 0; k < 2; ++k) enqueue_cg_iteration<float>(h, -1);
  double best = 1e30;
  for (int rep = 0; rep < 3; ++rep) {
    cudaEventRecord(h->e0, h->s);
    for (int k = 0; k < 8; ++k) enqueue_cg_iteration<float>(h, -1);
    cudaEventRecord(h->e1, h->s);
    if (cudaEventSynchronize(h->e1) != cudaSuccess) return -1.0;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, h->e0, h->e1);
    best = std::min(best, (double)ms / 8.0);
  }
  if (sync_state(h) || h->hst->done) return -1.0;
  return best;
}

int autotune(rve_t h) {
  NvtxRange nv("rve autotune");
  int dev = 0;
  cudaGetDevice(&dev);
  const TuneKey key{h->g.nx, h->g.ny, h->g.nz, dev, h->tan + 16 * (int)h->precond};
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      apply_knobs(h, it->second);
      h->knobs[6] = 1;
      return RVE_OK;
    }
  }
  Knobs best = {1, 3, 1, 1, 1, 0, 0, 0};
  apply_knobs(h, best);
  double tbest = time_cg_iteration(h);
  if (tbest < 0) return fail(h, RVE_ERR_CUDA, "autotune: CG timing run failed");
  const std::vector<int> choices[8] = {{1, 0}, {3, 2, 1}, {1, 0}, {1, 0}, {1, 0}, {0, 1},
                                       {0, 1}, {0, 1}};
  for (int knob = 0; knob < 8; ++knob)
    for (int v : choices[knob]) {
      if (v == best[knob]) continue;
      Knobs cand = best;
      cand[knob] = v;
      apply_knobs(h, cand);
      const double t = time_cg_iteration(h);
      if (t > 0 && t < tbest) {
        tbest = t;
        best = cand;
      }
    }
  apply_knobs(h, best);
  h->knobs[6] = 1;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = best;
  }
  return RVE_OK;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

void rve_default_options(rve_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->precision = RVE_FP64;
  o->tangent = RVE_TAN_AUTO;
  o->max_newton = 50;
  o->max_cg = 10000;
  o->cg_tol_floor = 1e-5;
  o->cg_atol = 0.0;
  o->mixed_refine = 0;
  o->residual = RVE_RES_FLOATFLOAT;
  o->autotune = 0;
  o->precond = RVE_PRECOND_NONE;
}

const char* rve_status_string(int code) {
  switch (code) {
    case RVE_OK: return "ok";
    case RVE_ERR_INVALID: return "invalid argument";
    case RVE_ERR_CUDA: return "CUDA error";
    case RVE_ERR_NOMEM: return "out of device memory";
    case RVE_ERR_CG_MAXIT: return "CG did not converge within max_cg iterations";
    case RVE_ERR_CG_BREAKDOWN: return "CG breakdown (p.Ap = 0)";
    case RVE_ERR_NEWTON_MAXIT: return "Newton did not converge within max_newton iterations";
    case RVE_ERR_NONFINITE: return "non-finite value";
    case RVE_ERR_DETF: return "det F <= 0";
    case RVE_ERR_TIMEOUT: return "device wait timed out";
    case RVE_ERR_UNSUPPORTED: return "unsupported";
    default: return "unknown status";
  }
}

const char* rve_last_error(rve_t h) {
  if (!h) return "null handle";
  return h->err.c_str();
}

static int resolve_options(const rve_options* in, rve_options* out, int model, int* tan) {
  if (in) *out = *in;
  else rve_default_options(out);
  if (out->precision != RVE_FP64 && out->precision != RVE_MIXED) return RVE_ERR_INVALID;
  if (out->max_newton <= 0) out->max_newton = 50;
  if (out->max_cg <= 0) out->max_cg = 10000;
  if (!(out->cg_tol_floor >= 0.0)) return RVE_ERR_INVALID;
  if (!(out->cg_atol >= 0.0)) return RVE_ERR_INVALID;
  if (out->mixed_refine < 0 || out->mixed_refine > 8) return RVE_ERR_INVALID;
  if (out->residual != RVE_RES_FLOATFLOAT && out->residual != RVE_RES_FP64) return RVE_ERR_INVALID;
  if (out->autotune != 0 && out->autotune != 1) return RVE_ERR_INVALID;
  if (out->precond != RVE_PRECOND_NONE && out->precond != RVE_PRECOND_REFERENCE)
    return RVE_ERR_INVALID;
  if (out->precond == RVE_PRECOND_REFERENCE && out->precision != RVE_MIXED)
    return RVE_ERR_UNSUPPORTED;
  if (model == RVE_SVK) {
    if (out->tangent == RVE_TAN_AUTO || out->tangent == RVE_TAN_RECOMPUTE) *tan = TAN_SVK;
    else if (out->tangent == RVE_TAN_FULL81) *tan = TAN_FULL81;
    else if (out->tangent == RVE_TAN_SYM45) *tan = TAN_SYM45;
    else return RVE_ERR_INVALID;
  } else if (model == RVE_J2) {
    // the J2 tangent is stored: packed symmetric (45 values per voxel) by
    // default, or all 81
    if (out->tangent == RVE_TAN_AUTO || out->tangent == RVE_TAN_SYM45) *tan = TAN_SYM45;
    else if (out->tangent == RVE_TAN_FULL81) *tan = TAN_FULL81;
    else return RVE_ERR_INVALID;
  } else {
    return RVE_ERR_INVALID;
  }
  return RVE_OK;
}

int rve_workspace_size(int nx, int ny, int nz, int model, const rve_options* opt, size_t* bytes) {
  if (!bytes) return RVE_ERR_INVALID;
  rve_s tmp;
  if (!make_geom(nx, ny, nz, &tmp.g)) return RVE_ERR_INVALID;
  int tan = 0;
  int rc = resolve_options(opt, &tmp.opt, model, &tan);
  if (rc) return rc;
  tmp.n = tmp.g.n;
  tmp.mixed = tmp.opt.precision == RVE_MIXED;
  tmp.tan = tan;
  tmp.nparam = (model == RVE_J2) ? 4 : 2;
  tmp.model = model;
  Arena a;
  layout(&tmp, a);
  Arena b = a;
  size_t with_vox = layout_material(&tmp, b, false);
  Arena c = a;
  size_t with_phase = layout_material(&tmp, c, true);
  *bytes = std::max(with_vox, with_phase) + 256;
  return RVE_OK;
}

int rve_create(rve_t* out, int nx, int ny, int nz, int model, int nphase, const uint8_t* phase,
               const double* phase_params, const double* voxel_params, const rve_options* opt) {
  if (!out) return RVE_ERR_INVALID;
  *out = nullptr;
  rve_t h = new rve_s();
  auto bail = [&](int code, const std::string& msg) {
    rve_destroy(h);
    std::fprintf(stderr, "rve_create: %s\n", msg.c_str());
    return code;
  };
  if (model != RVE_SVK && model != RVE_J2) return bail(RVE_ERR_INVALID, "unknown model");
  h->model = model;
  if (!make_geom(nx, ny, nz, &h->g))
    return bail(RVE_ERR_INVALID, "grid sizes must be positive and supported by the DFT plan");
  int tan = 0;
  int rc = resolve_options(opt, &h->opt, model, &tan);
  if (rc) return bail(rc, rc == RVE_ERR_UNSUPPORTED ? "option combination not supported"
                                                    : "invalid options");
  h->n = h->g.n;
  h->mixed = h->opt.precision == RVE_MIXED;
  h->floatfloat = h->mixed && h->opt.residual == RVE_RES_FLOATFLOAT;
  h->precond = h->opt.precond == RVE_PRECOND_REFERENCE;
  if (h->precond && !fs_split_n1(nx))
    return bail(RVE_ERR_UNSUPPORTED, "preconditioned CG needs an x length with a four-step DFT kernel");
  h->tan = tan;
  h->nparam = (model == RVE_J2) ? 4 : 2;
  h->s = (cudaStream_t)h->opt.stream;
  if (phase) {
    if (nphase < 1 || nphase > 256 || !phase_params)
      return bail(RVE_ERR_INVALID, "phase map needs 1..256 phases with parameters");
    for (size_t v = 0; v < h->n; ++v)
      if (phase[v] >= nphase) return bail(RVE_ERR_INVALID, "phase index >= nphase");
  } else if (!voxel_params) {
    return bail(RVE_ERR_INVALID, "either a phase map or per-voxel parameters are required");
  }
  // sizes
  Arena dry;
  layout(h, dry);
  Arena dry2 = dry;
  const size_t need = layout_material(h, dry2, phase != nullptr) + 256;
  if (h->opt.workspace) {
    if (h->opt.workspace_bytes < need) return bail(RVE_ERR_NOMEM, "workspace too small");
    h->ws = (char*)h->opt.workspace;
    h->own_ws = false;
  } else {
    if (cudaMalloc(&h->ws, need) != cudaSuccess) {
      h->ws = nullptr;
      return bail(RVE_ERR_NOMEM, "cudaMalloc of the workspace failed");
    }
    h->own_ws = true;
  }
  h->ws_bytes = need;
  Arena a;
  a.dry = false;
  a.base = h->ws;
  a.cap = need;
  layout(h, a);
  layout_material(h, a, phase != nullptr);
  if (cudaMallocHost(&h->hst, sizeof(SolverState)) != cudaSuccess) return bail(RVE_ERR_NOMEM, "pinned alloc");
  std::memset(h->hst, 0, sizeof(SolverState));
  {
    cudaError_t e = fft_kernels_init();
    if (e != cudaSuccess) return bail(RVE_ERR_CUDA, std::string("kernel attributes: ") + cudaGetErrorString(e));
  }
  cudaEventCreate(&h->e0);
  cudaEventCreate(&h->e1);

  cudaError_t first_err = cudaSuccess;
  auto ck = [&](cudaError_t e) {
    if (e != cudaSuccess && first_err == cudaSuccess) first_err = e;
    return e == cudaSuccess;
  };
  bool ok = true;
  ok &= ck(cudaMemsetAsync(h->ws, 0, need, h->s));
  // twiddles exp(-2 pi i k / N) per axis, from float64 host evaluation
  {
    const int dims[3] = {h->g.nx, h->g.ny, h->g.nz};
    std::vector<cplx<double>> td;
    std::vector<cplx<float>> tf;
    std::vector<cplx<dfl>> tdf;
    for (int d = 0; d < 3; ++d)
      for (int k = 0; k < dims[d]; ++k) {
        const double ang = 2.0 * kPi * (double)k / (double)dims[d];
        td.push_back({std::cos(ang), -std::sin(ang)});
        tf.push_back({(float)std::cos(ang), (float)-std::sin(ang)});
        tdf.push_back({dfl(std::cos(ang)), dfl(-std::sin(ang))});
      }
    ok &= ck(cudaMemcpyAsync(h->twd_all, td.data(), td.size() * sizeof(td[0]), cudaMemcpyHostToDevice, h->s));
    ok &= ck(cudaMemcpyAsync(h->twf_all, tf.data(), tf.size() * sizeof(tf[0]), cudaMemcpyHostToDevice, h->s));
    ok &= ck(cudaMemcpyAsync(h->twdf_all, tdf.data(), tdf.size() * sizeof(tdf[0]), cudaMemcpyHostToDevice, h->s));
    h->twd = {h->twd_all, h->twd_all + dims[0], h->twd_all + dims[0] + dims[1]};
    h->twf = {h->twf_all, h->twf_all + dims[0], h->twf_all + dims[0] + dims[1]};
    h->twdf = {h->twdf_all, h->twdf_all + dims[0], h->twdf_all + dims[0] + dims[1]};
    ok &= ck(cudaStreamSynchronize(h->s));
  }
  // materials: (lambda, mu) with lambda = K - 2 mu / 3 (Eq. elas:C)
  bool vp_on_device = false;
  double vp_sums[2] = {0.0, 0.0};
  if (!phase && voxel_params) {
    cudaPointerAttributes pa{};
    if (cudaPointerGetAttributes(&pa, voxel_params) == cudaSuccess)
      vp_on_device = pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged;
    cudaGetLastError();  // a plain host pointer may leave an error on older drivers
  }
  if (phase) {
    std::vector<double> t64(256 * 4, 0.0);
    std::vector<float> t32(256 * 4, 0.0f);
    for (int k = 0; k < nphase; ++k) {
      const double K = phase_params[k * h->nparam], mu = phase_params[k * h->nparam + 1];
      t64[k * h->nparam] = K - 2.0 * mu / 3.0;
      t64[k * h->nparam + 1] = mu;
      for (int q = 2; q < h->nparam; ++q) t64[k * h->nparam + q] = phase_params[k * h->nparam + q];
      for (int q = 0; q < h->nparam; ++q) t32[k * h->nparam + q] = (float)t64[k * h->nparam + q];
    }
    ok &= ck(cudaMemcpyAsync(h->table64, t64.data(), t64.size() * 8, cudaMemcpyHostToDevice, h->s));
    ok &= ck(cudaMemcpyAsync(h->table32, t32.data(), t32.size() * 4, cudaMemcpyHostToDevice, h->s));
    ok &= ck(cudaMemcpyAsync(h->phase, phase, h->n, cudaMemcpyHostToDevice, h->s));
    ok &= ck(cudaStreamSynchronize(h->s));
  } else if (vp_on_device) {
    // device parameters: converted and averaged by a kernel, only the two
    // sums of the reference medium come back to the host
    unsigned int* cnt = &h->st->counter[SLOT_MISC];
    ok &= ck(cudaMemsetAsync(cnt, 0, sizeof(unsigned int), h->s));
    launch_voxel_params(voxel_params, h->n, h->nparam, h->vox64, h->vox32, h->tmp64, h->partials, cnt,
                        h->s);
    ok &= ck(cudaGetLastError());
    ok &= ck(cudaMemcpyAsync(vp_sums, h->tmp64, sizeof(vp_sums), cudaMemcpyDeviceToHost, h->s));
    ok &= ck(cudaStreamSynchronize(h->s));
  } else {
    std::vector<double> v64((size_t)h->nparam * h->n);
    for (size_t v = 0; v < h->n; ++v) {
      const double K = voxel_params[v], mu = voxel_params[h->n + v];
      v64[v] = K - 2.0 * mu / 3.0;
      v64[h->n + v] = mu;
    }
    for (int q = 2; q < h->nparam; ++q)
      for (size_t v = 0; v < h->n; ++v) v64[q * h->n + v] = voxel_params[q * h->n + v];
    ok &= ck(cudaMemcpyAsync(h->vox64, v64.data(), v64.size() * 8, cudaMemcpyHostToDevice, h->s));
    std::vector<float> v32;
    if (h->vox32) {
      v32.assign(v64.begin(), v64.end());
      ok &= ck(cudaMemcpyAsync(h->vox32, v32.data(), v32.size() * 4, cudaMemcpyHostToDevice, h->s));
    }
    ok &= ck(cudaStreamSynchronize(h->s));
  }
  if (!ok) return bail(RVE_ERR_CUDA, std::string("initial copies failed: ") + cudaGetErrorString(first_err));
  {
    // reference medium of the preconditioner: voxel averages of the Lame
    // parameters (only lambda0 / mu0 matters)
    double lam0 = 0.0, mu0 = 0.0;
    if (phase) {
      std::vector<size_t> cnt(256, 0);
      for (size_t v = 0; v < h->n; ++v) cnt[phase[v]]++;
      for (int k = 0; k < nphase; ++k) {
        const double K = phase_params[k * h->nparam], mu = phase_params[k * h->nparam + 1];
        lam0 += (double)cnt[k] * (K - 2.0 * mu / 3.0);
        mu0 += (double)cnt[k] * mu;
      }
    } else if (vp_on_device) {
      lam0 = vp_sums[0];
      mu0 = vp_sums[1];
    } else {
      for (size_t v = 0; v < h->n; ++v) {
        lam0 += voxel_params[v] - 2.0 * voxel_params[h->n + v] / 3.0;
        mu0 += voxel_params[h->n + v];
      }
    }
    if (h->precond && !(mu0 > 0.0 && lam0 + 2.0 * mu0 / 3.0 > 0.0))
      return bail(RVE_ERR_INVALID, "reference medium needs positive average moduli");
    const double ell = mu0 > 0.0 ? lam0 / mu0 : 0.0;
    h->g.pc_ell = (float)ell;
    h->g.pc_c = (float)((ell + 1.0) / (ell + 2.0));
  }
  // F = I, evaluate the material there
  {
    std::vector<double> I(9 * h->n, 0.0);
    for (int c : {0, 4, 8})
      for (size_t v = 0; v < h->n; ++v) I[c * h->n + v] = 1.0;
    ok &= ck(cudaMemcpyAsync(h->F, I.data(), I.size() * 8, cudaMemcpyHostToDevice, h->s));
    ok &= ck(cudaMemcpyAsync(h->Ft, I.data(), I.size() * 8, cudaMemcpyHostToDevice, h->s));
    ok &= ck(cudaStreamSynchronize(h->s));
  }
  if (h->model == RVE_J2) {
    // history: Cp^-1 = I, eps_p = 0 (Algorithm 1, first line)
    std::vector<double> H0(7 * h->n, 0.0);
    for (int c = 0; c < 3; ++c)
      for (size_t v = 0; v < h->n; ++v) H0[c * h->n + v] = 1.0;
    ok &= ck(cudaMemcpyAsync(h->hc, H0.data(), H0.size() * 8, cudaMemcpyHostToDevice, h->s));
    ok &= ck(cudaMemcpyAsync(h->ht, H0.data(), H0.size() * 8, cudaMemcpyHostToDevice, h->s));
    ok &= ck(cudaMemcpyAsync(h->hprev, H0.data(), H0.size() * 8, cudaMemcpyHostToDevice, h->s));
    ok &= ck(cudaStreamSynchronize(h->s));
  }
  if (h->tan == TAN_SVK && !h->mixed) h->Fop = h->F;  // FP64 recompute reads F itself
  enqueue_constitutive(h);
  ok &= ck(cudaStreamSynchronize(h->s));
  ok &= ck(cudaGetLastError());
  if (!ok)
    return bail(RVE_ERR_CUDA, std::string("initial constitutive evaluation failed: ") +
                                  cudaGetErrorString(first_err));
  if (h->mixed && h->opt.autotune) {
    const int arc = autotune(h);
    if (arc) return bail(arc, "autotune failed");
  }
  *out = h;
  return RVE_OK;
}

// ---------------------------------------------------------------------------
// Checkpoint / resume.  File: a fixed header (CkptHeader) followed by tagged
// blocks {char tag[8]; uint64 bytes; data}, host byte order.  Saved: F, the
// committed F, P, the tangent data, the J2 histories, the material buffers
// in their internal form (so that a resumed run is bit-identical), and on
// the host F-bar, the committed F-bar and the kernel variants.
// ---------------------------------------------------------------------------
struct CkptHeader {
  char magic[8];
  int version, nx, ny, nz, model, nparam, use_phase, precision, tangent, residual;
  int max_newton, max_cg, mixed_refine;
  double cg_tol_floor, cg_atol;
  int knobs[9];
  int precond;
  double Fbar[9], Fbar_committed[9];
};

struct CkptBlock {
  const char* tag;
  void* dev;
  size_t bytes;
};

static std::vector<CkptBlock> ckpt_blocks(rve_t h) {
  const size_t n = h->n, ro = h->mixed ? 4 : 8;
  std::vector<CkptBlock> b = {{"F", h->F, 9 * n * 8}, {"Ft", h->Ft, 9 * n * 8}, {"P", h->P, 9 * n * 8}};
  if (h->K4) b.push_back({"K4", h->K4, (h->tan == TAN_SYM45 ? 45 : 81) * n * ro});
  if (h->Fop && h->Fop != (void*)h->F) b.push_back({"Fop", h->Fop, 9 * n * ro});
  if (h->Sop) b.push_back({"Sop", h->Sop, 6 * n * ro});
  if (h->hc) b.push_back({"hc", h->hc, 7 * n * 8});
  if (h->ht) b.push_back({"ht", h->ht, 7 * n * 8});
  if (h->hprev) b.push_back({"hprev", h->hprev, 7 * n * 8});
  if (h->phase) {
    b.push_back({"phase", h->phase, n});
    b.push_back({"t64", h->table64, 256 * 4 * 8});
    b.push_back({"t32", h->table32, 256 * 4 * 4});
  } else {
    b.push_back({"v64", h->vox64, (size_t)h->nparam * n * 8});
    if (h->vox32) b.push_back({"v32", h->vox32, (size_t)h->nparam * n * 4});
  }
  return b;
}

int rve_save(rve_t h, const char* path) {
  NvtxRange nv("rve save");
  if (!h || !path) return RVE_ERR_INVALID;
  FILE* f = std::fopen(path, "wb");
  if (!f) return fail(h, RVE_ERR_INVALID, std::string("cannot open ") + path);
  CkptHeader hd;
  std::memset(&hd, 0, sizeof(hd));
  std::memcpy(hd.magic, "RVECKPT1", 8);
  hd.version = 3;
  hd.nx = h->g.nx;
  hd.ny = h->g.ny;
  hd.nz = h->g.nz;
  hd.model = h->model;
  hd.nparam = h->nparam;
  hd.use_phase = h->phase != nullptr;
  hd.precision = h->opt.precision;
  hd.tangent = h->tan == TAN_FULL81 ? RVE_TAN_FULL81 : (h->tan == TAN_SYM45 ? RVE_TAN_SYM45 : RVE_TAN_RECOMPUTE);
  hd.residual = h->opt.residual;
  hd.max_newton = h->opt.max_newton;
  hd.max_cg = h->opt.max_cg;
  hd.mixed_refine = h->opt.mixed_refine;
  hd.cg_tol_floor = h->opt.cg_tol_floor;
  hd.cg_atol = h->opt.cg_atol;
  hd.precond = h->opt.precond;
  std::memcpy(hd.knobs, h->knobs, sizeof(hd.knobs));
  std::memcpy(hd.Fbar, h->Fbar, sizeof(hd.Fbar));
  std::memcpy(hd.Fbar_committed, h->Fbar_committed, sizeof(hd.Fbar_committed));
  bool ok = std::fwrite(&hd, sizeof(hd), 1, f) == 1;
  std::vector<char> host;
  for (const CkptBlock& b : ckpt_blocks(h)) {
    if (!ok) break;
    host.resize(b.bytes);
    if (cudaMemcpyAsync(host.data(), b.dev, b.bytes, cudaMemcpyDeviceToHost, h->s) != cudaSuccess ||
        cudaStreamSynchronize(h->s) != cudaSuccess) {
      std::fclose(f);
      return fail(h, RVE_ERR_CUDA, "checkpoint copy failed");
    }
    char tag[8] = {0};
    std::strncpy(tag, b.tag, 8);
    const unsigned long long nb = b.bytes;
    ok = std::fwrite(tag, 8, 1, f) == 1 && std::fwrite(&nb, 8, 1, f) == 1 &&
         std::fwrite(host.data(), 1, b.bytes, f) == b.bytes;
  }
  ok = (std::fclose(f) == 0) && ok;
  return ok ? RVE_OK : fail(h, RVE_ERR_INVALID, std::string("write failed: ") + path);
}

int rve_load(rve_t* out, const char* path, const rve_options* opt) {
  NvtxRange nv("rve load");
  if (!out || !path) return RVE_ERR_INVALID;
  *out = nullptr;
  FILE* f = std::fopen(path, "rb");
  if (!f) return RVE_ERR_INVALID;
  CkptHeader hd;
  if (std::fread(&hd, sizeof(hd), 1, f) != 1 || std::memcmp(hd.magic, "RVECKPT1", 8) != 0 ||
      hd.version != 3) {
    std::fclose(f);
    return RVE_ERR_INVALID;
  }
  // all blocks into host memory first
  std::map<std::string, std::vector<char>> blocks;
  for (;;) {
    char tag[9] = {0};
    unsigned long long nb = 0;
    if (std::fread(tag, 8, 1, f) != 1) break;
    if (std::fread(&nb, 8, 1, f) != 1 || nb > ((unsigned long long)1 << 40)) {
      std::fclose(f);
      return RVE_ERR_INVALID;
    }
    std::vector<char> data(nb);
    if (std::fread(data.data(), 1, nb, f) != nb) {
      std::fclose(f);
      return RVE_ERR_INVALID;
    }
    blocks[tag] = std::move(data);
  }
  std::fclose(f);
  const size_t n = (size_t)hd.nx * hd.ny * hd.nz;
  // material in the user's form (the internal buffers are restored below)
  std::vector<double> params;
  std::vector<uint8_t> ph;
  int nphase = 0;
  if (hd.use_phase) {
    auto& pb = blocks["phase"];
    auto& tb = blocks["t64"];
    if (pb.size() != n || tb.size() != 256 * 4 * 8) return RVE_ERR_INVALID;
    ph.assign(pb.begin(), pb.end());
    for (uint8_t v : ph) nphase = std::max(nphase, (int)v + 1);
    const double* t = reinterpret_cast<const double*>(tb.data());
    params.assign((size_t)nphase * hd.nparam, 0.0);
    for (int k = 0; k < nphase; ++k) {
      for (int q = 0; q < hd.nparam; ++q) params[k * hd.nparam + q] = t[k * hd.nparam + q];
      params[k * hd.nparam] = t[k * hd.nparam] + 2.0 * t[k * hd.nparam + 1] / 3.0;  // K
    }
  } else {
    auto& vb = blocks["v64"];
    if (vb.size() != (size_t)hd.nparam * n * 8) return RVE_ERR_INVALID;
    const double* v = reinterpret_cast<const double*>(vb.data());
    params.assign(v, v + (size_t)hd.nparam * n);
    for (size_t i = 0; i < n; ++i) params[i] = v[i] + 2.0 * v[n + i] / 3.0;  // K
  }
  rve_options o;
  rve_default_options(&o);
  o.precision = hd.precision;
  o.tangent = hd.tangent;
  o.residual = hd.residual;
  o.max_newton = hd.max_newton;
  o.max_cg = hd.max_cg;
  o.mixed_refine = hd.mixed_refine;
  o.cg_tol_floor = hd.cg_tol_floor;
  o.cg_atol = hd.cg_atol;
  o.precond = hd.precond;
  if (opt) {
    o.stream = opt->stream;
    o.workspace = opt->workspace;
    o.workspace_bytes = opt->workspace_bytes;
  }
  rve_t h = nullptr;
  int rc = rve_create(&h, hd.nx, hd.ny, hd.nz, hd.model, nphase, hd.use_phase ? ph.data() : nullptr,
                      hd.use_phase ? params.data() : nullptr, hd.use_phase ? nullptr : params.data(), &o);
  if (rc) return rc;
  for (const CkptBlock& b : ckpt_blocks(h)) {
    auto it = blocks.find(b.tag);
    if (it == blocks.end() || it->second.size() != b.bytes) {
      rve_destroy(h);
      return RVE_ERR_INVALID;
    }
    if (cudaMemcpyAsync(b.dev, it->second.data(), b.bytes, cudaMemcpyHostToDevice, h->s) != cudaSuccess ||
        cudaStreamSynchronize(h->s) != cudaSuccess) {
      rve_destroy(h);
      return RVE_ERR_CUDA;
    }
  }
  std::memcpy(h->Fbar, hd.Fbar, sizeof(hd.Fbar));
  std::memcpy(h->Fbar_committed, hd.Fbar_committed, sizeof(hd.Fbar_committed));
  Knobs k;
  for (int i = 0; i < 6; ++i) k[i] = hd.knobs[i];
  k[6] = hd.knobs[7];
  k[7] = hd.knobs[8];
  apply_knobs(h, k);
  h->knobs[6] = hd.knobs[6];
  *out = h;
  return RVE_OK;
}

int rve_model(rve_t h) { return h ? h->model : RVE_ERR_INVALID; }

int rve_grid(rve_t h, int dims[3]) {
  if (!h || !dims) return RVE_ERR_INVALID;
  dims[0] = h->g.nx;
  dims[1] = h->g.ny;
  dims[2] = h->g.nz;
  return RVE_OK;
}

int rve_set_tuning(rve_t h, const int knobs[9]) {
  if (!h || !knobs) return RVE_ERR_INVALID;
  for (int i : {0, 2, 3, 4, 5, 7, 8})
    if (knobs[i] != 0 && knobs[i] != 1) return fail(h, RVE_ERR_INVALID, "tuning knobs are 0 or 1");
  if (knobs[1] < 1 || knobs[1] > 3) return fail(h, RVE_ERR_INVALID, "z blocks per SM in 1..3");
  CK(cudaStreamSynchronize(h->s));
  Knobs k;
  for (int i = 0; i < 6; ++i) k[i] = knobs[i];
  k[6] = knobs[7];
  k[7] = knobs[8];
  apply_knobs(h, k);
  h->knobs[6] = 0;
  return RVE_OK;
}

int rve_tuning(rve_t h, int knobs[9]) {
  if (!h || !knobs) return RVE_ERR_INVALID;
  for (int i = 0; i < 9; ++i) knobs[i] = h->knobs[i];
  return RVE_OK;
}

void rve_destroy(rve_t h) {
  if (h) tape_clear(h);
  if (!h) return;
  if (h->s) cudaStreamSynchronize(h->s);
  else cudaDeviceSynchronize();
  if (h->own_ws && h->ws) cudaFree(h->ws);
  if (h->hst) cudaFreeHost(h->hst);
  for (auto& t : h->timed) {
    cudaEventDestroy(t.a);
    cudaEventDestroy(t.b);
  }
  for (auto e : h->ev_pool) cudaEventDestroy(e);
  if (h->e0) cudaEventDestroy(h->e0);
  if (h->e1) cudaEventDestroy(h->e1);
  delete h;
}

int rve_set_macro_F(rve_t h, const double Fbar[9]) {
  if (!h || !Fbar) return RVE_ERR_INVALID;
  for (int c = 0; c < 9; ++c)
    if (!std::isfinite(Fbar[c])) return fail(h, RVE_ERR_INVALID, "non-finite F-bar");
  std::memcpy(h->Fbar, Fbar, sizeof(h->Fbar));
  return RVE_OK;
}

}  // extern "C"

// Stores the converged state of an increment: F, F-bar, P-bar and (J2) the
// trial history of the last constitutive evaluation, after which the
// constitutive response is re-evaluated with it (Algorithm 1, i = 0 of the
// next increment).
static int commit_state(rve_t h) {
  CK(cudaMemcpyAsync(h->Ft, h->F, 9 * h->n * 8, cudaMemcpyDeviceToDevice, h->s));
  std::memcpy(h->Fbar_committed, h->Fbar, sizeof(h->Fbar));
  launch_mean9<double>(h->P, h->n, nullptr, h->partials, &h->st->counter[SLOT_MEAN], MEAN_PBAR,
                       h->st, h->s);
  h->launches += 1;
  if (h->model == RVE_J2) {
    // the trial history becomes the committed one; the former committed
    // one is kept as the start of this increment (for the adjoint)
    double* start = h->hc;
    h->hc = h->ht;
    h->ht = h->hprev;
    h->hprev = start;
    if (h->tape_on) {
      double *tf = nullptr, *th = nullptr;
      if (cudaMalloc(&tf, 9 * h->n * 8) != cudaSuccess || cudaMalloc(&th, 7 * h->n * 8) != cudaSuccess) {
        cudaFree(tf);
        return fail(h, RVE_ERR_NOMEM, "tape: allocation failed");
      }
      CK(cudaMemcpyAsync(tf, h->F, 9 * h->n * 8, cudaMemcpyDeviceToDevice, h->s));
      CK(cudaMemcpyAsync(th, h->hprev, 7 * h->n * 8, cudaMemcpyDeviceToDevice, h->s));
      h->tape_F.push_back(tf);
      h->tape_h.push_back(th);
    }
    enqueue_constitutive(h);
  }
  return RVE_OK;
}

static void tape_clear(rve_t h) {
  if (!h->tape_F.empty() || !h->tape_h.empty()) cudaStreamSynchronize(h->s);
  for (double* p : h->tape_F) cudaFree(p);
  for (double* p : h->tape_h) cudaFree(p);
  h->tape_F.clear();
  h->tape_h.clear();
}

// One increment to h->Fbar.  commit = false leaves a converged state
// uncommitted: F, P and the J2 trial history stay those of the converged
// iterate while the committed state (Ft, history) is kept, so that a later
// increment still starts the return map from the committed history (the
// iterates of mixed control).  A failure always rolls back to the
// committed state.
template <typename R>
static int solve_increment_t(rve_t h, double tol_newton, double tol_cg, rve_stats* st,
                             bool commit = true) {
  NvtxRange nv("rve solve_increment");
  const size_t n9 = 9 * h->n;
  CK(cudaEventRecord(h->e0, h->s));
  // device state for this increment
  SolverState* hs = h->hst;
  std::memset(hs, 0, sizeof(SolverState));
  hs->cg_tol = h->mixed ? std::max(tol_cg, h->opt.cg_tol_floor) : tol_cg;
  hs->cg_atol = h->opt.cg_atol;
  hs->maxit = h->opt.max_cg;
  hs->stag = h->mixed ? kMixedStagnation : 0;
  std::memcpy(hs->Fbar, h->Fbar, sizeof(hs->Fbar));
  int rc = push_state(h);
  if (rc) return rc;
  // predictor (i = 0 right-hand side) and ||F_(0) + dFbar||
  enqueue_predictor<R>(h);
  // ||F_(0) + dFbar|| (F itself is updated together with the first dF)
  launch_shifted_norm(h->F, h->n, h->st, h->partials, h->s);
  h->launches += 1;
  int result = RVE_OK;
  bool converged = false;
  int newton = 0;
  int cg_total = 0;
  int extra_refine = h->mixed ? h->opt.mixed_refine : 0;
  double prev_rel = 0.0, prev2_rel = 0.0;
  for (int i = 0; i < h->opt.max_newton; ++i) {
    int its = 0;
    CK(cudaGetLastError());
    rc = cg_solve<R>(h, &its);
    cg_total += its;
    if (st && i < RVE_MAX_NEWTON_LOG) st->cg_iters[i] = its;
    if (rc) {
      result = fail(h, rc, std::string("linear solve: ") + rve_status_string(rc));
      break;
    }
    if (h->mixed) {
      // float32 CG leaves dF compatible only up to float32 round-off
      // amplified by the cancellation in the CG sum; project it onto the
      // compatible fields in float64 so that F stays compatible (Sec. 2.3)
      enqueue_mixed_update<R>(h, i == 0);
    } else {
      launch_mean9<R>(as<R>(h->x), h->n, nullptr, h->partials, &h->st->counter[SLOT_MEAN], MEAN_X,
                      h->st, h->s);
      launch_newton_update<R>(h->F, as<R>(h->x), h->n, h->st, h->partials, i == 0, h->s);
      h->launches += 2;
    }
    enqueue_constitutive(h);
    enqueue_residual<R>(h);
    rc = sync_state(h);
    if (rc) {
      result = rc;
      break;
    }
    newton = i + 1;
    const double rel = std::sqrt(hs->dF2 / hs->Fn2);
    if (st && i < RVE_MAX_NEWTON_LOG) {
      st->rel_update[i] = rel;
      st->residual[i] = std::sqrt(hs->bb);
    }
    rc = check_flags(h, false);
    if (rc) {
      result = rc;
      break;
    }
    if (!std::isfinite(rel)) {
      result = fail(h, RVE_ERR_NONFINITE, "non-finite Newton update");
      break;
    }
    // divergence: an update larger than half of F, or updates that grew in
    // two consecutive equilibrium iterations
    if (rel > kDivergedUpdate || (i >= 3 && rel > prev_rel && prev_rel > prev2_rel)) {
      result = fail(h, RVE_ERR_NEWTON_MAXIT, "Newton diverged");
      break;
    }
    prev2_rel = prev_rel;
    prev_rel = rel;
    if (rel < tol_newton && i > 0) {
      if (extra_refine > 0) {
        --extra_refine;
        continue;
      }
      converged = true;
      result = check_flags(h, true);  // the converged state must have det F > 0
      break;
    }
  }
  if (result == RVE_OK && !converged)
    result = fail(h, RVE_ERR_NEWTON_MAXIT, "Newton did not converge");
  if (result == RVE_OK) {
    if (commit) {
      rc = commit_state(h);
      if (rc) return rc;
    }
  } else {
    // roll back to the last committed state
    CK(cudaMemcpyAsync(h->F, h->Ft, n9 * 8, cudaMemcpyDeviceToDevice, h->s));
    enqueue_constitutive(h);
  }
  CK(cudaEventRecord(h->e1, h->s));
  rc = sync_state(h);
  if (rc) return rc;
  CK(cudaGetLastError());
  if (st) {
    st->status = result;
    st->newton_iters = newton;
    st->cg_iters_total = cg_total;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, h->e0, h->e1);
    st->elapsed_ms = ms;
  }
  return result;
}

extern "C" {

int rve_solve_increment(rve_t h, double tol_newton, double tol_cg, rve_stats* st) {
  if (!h) return RVE_ERR_INVALID;
  if (!(tol_newton > 0.0) || !(tol_cg > 0.0)) return fail(h, RVE_ERR_INVALID, "tolerances must be > 0");
  if (st) std::memset(st, 0, sizeof(*st));
  h->err.clear();
  return h->mixed ? solve_increment_t<float>(h, tol_newton, tol_cg, st)
                  : solve_increment_t<double>(h, tol_newton, tol_cg, st);
}

int rve_solve_step(rve_t h, const double Fbar[9], double tol_newton, double tol_cg, int max_cuts,
                   rve_stats* st) {
  NvtxRange nv("rve solve_step");
  if (!h || !Fbar || max_cuts < 0) return RVE_ERR_INVALID;
  for (int c = 0; c < 9; ++c)
    if (!std::isfinite(Fbar[c])) return fail(h, RVE_ERR_INVALID, "non-finite F-bar");
  double F0[9], target[9];
  std::memcpy(F0, h->Fbar_committed, sizeof(F0));
  std::memcpy(target, Fbar, sizeof(target));
  rve_stats acc;
  std::memset(&acc, 0, sizeof(acc));
  double done = 0.0, step = 1.0;
  const double min_step = std::ldexp(1.0, -max_cuts);
  int cuts = 0, sub = 0, streak = 0;
  int result = RVE_OK;
  while (done < 1.0) {
    const double to = std::min(1.0, done + step);
    double Fb[9];
    for (int c = 0; c < 9; ++c) Fb[c] = (to >= 1.0) ? target[c] : F0[c] + to * (target[c] - F0[c]);
    rve_set_macro_F(h, Fb);
    rve_stats s1;
    const int rc = rve_solve_increment(h, tol_newton, tol_cg, &s1);
    acc.newton_iters += s1.newton_iters;
    acc.cg_iters_total += s1.cg_iters_total;
    acc.elapsed_ms += s1.elapsed_ms;
    if (rc == RVE_OK) {
      done = to;
      if (sub < RVE_MAX_NEWTON_LOG) acc.substep_to[sub] = to;
      ++sub;
      // grow only after two successes at this size (growing after every
      // success alternates success and failure on a hard stretch)
      if (++streak >= 2) {
        step = std::min(2.0 * step, 1.0);
        streak = 0;
      }
    } else if (rc == RVE_ERR_NEWTON_MAXIT || rc == RVE_ERR_CG_MAXIT || rc == RVE_ERR_NONFINITE ||
               rc == RVE_ERR_DETF || rc == RVE_ERR_CG_BREAKDOWN) {
      // the state was rolled back: retry with half the step
      ++cuts;
      streak = 0;
      step *= 0.5;
      if (step < min_step) {
        result = rc;
        break;
      }
    } else {
      result = rc;
      break;
    }
  }
  std::memcpy(h->Fbar, target, sizeof(h->Fbar));
  if (st) {
    *st = acc;
    st->status = result;
    st->substeps = sub;
    st->cuts = cuts;
  }
  return result;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Mixed macroscopic control.  Not in the paper: Sec. 3.1 prescribes the full
// F-bar and leaves other boundary conditions to the literature.  The
// stress-controlled components S have P-bar_S prescribed and F-bar_S free;
// the state sought is the equilibrium of one increment from the committed
// state with <F> = F-bar and <P>_S = P*_S.  Newton on F-bar_S: every iterate
// is an ordinary (uncommitted) increment; the Jacobian is the homogenised
// tangent dP-bar_a/dF-bar_b = <K : (E_b + dF_b)>_a, where dF_b solves the
// predictor system G:K:dF_b = -G:K:E_b (Eq. bc:lin with dF-bar = E_b), taken
// exactly at the first iterate and again whenever the stress residual fell
// by less than 4x, with Broyden's rank-one update in between.
// ---------------------------------------------------------------------------

// Solves A u = b in place (m x m row-major, m <= 9) by Gaussian elimination
// with partial pivoting; false if a pivot is below rel * max |A_ij|.
static bool small_solve(int m, double* A, double* b, double rel) {
  double amax = 0.0;
  for (int i = 0; i < m * m; ++i) amax = std::max(amax, std::fabs(A[i]));
  if (!(amax > 0.0)) return false;
  for (int k = 0; k < m; ++k) {
    int piv = k;
    for (int i = k + 1; i < m; ++i)
      if (std::fabs(A[i * m + k]) > std::fabs(A[piv * m + k])) piv = i;
    if (!(std::fabs(A[piv * m + k]) > rel * amax)) return false;
    if (piv != k) {
      for (int j = 0; j < m; ++j) std::swap(A[k * m + j], A[piv * m + j]);
      std::swap(b[k], b[piv]);
    }
    for (int i = k + 1; i < m; ++i) {
      const double f = A[i * m + k] / A[k * m + k];
      for (int j = k; j < m; ++j) A[i * m + j] -= f * A[k * m + j];
      b[i] -= f * b[k];
    }
  }
  for (int k = m - 1; k >= 0; --k) {
    double v = b[k];
    for (int j = k + 1; j < m; ++j) v -= A[k * m + j] * b[j];
    b[k] = v / A[k * m + k];
  }
  return true;
}

static int rollback_state(rve_t h) {
  CK(cudaMemcpyAsync(h->F, h->Ft, 9 * h->n * 8, cudaMemcpyDeviceToDevice, h->s));
  enqueue_constitutive(h);
  return sync_state(h);
}

// Columns cols[0..ncol) of dP-bar/dF-bar at the current converged state into
// C[a * ncol + k] (a = component of P-bar), one CG solve each.
template <typename R>
static int homogenized_tangent_t(rve_t h, const int* cols, int ncol, double tol_cg, double* C,
                                 int* cg_iters) {
  NvtxRange nv("rve homogenized_tangent");
  SolverState* hs = h->hst;
  for (int k = 0; k < ncol; ++k) {
    std::memset(hs, 0, sizeof(SolverState));
    hs->cg_tol = h->mixed ? std::max(tol_cg, h->opt.cg_tol_floor) : tol_cg;
    hs->cg_atol = h->opt.cg_atol;
    hs->maxit = h->opt.max_cg;
    hs->stag = h->mixed ? kMixedStagnation : 0;
    hs->dFbar[cols[k]] = 1.0;
    int rc = push_state(h);
    if (rc) return rc;
    enqueue_predictor<R>(h, false);
    int its = 0;
    rc = cg_solve<R>(h, &its);
    *cg_iters += its;
    if (rc) return fail(h, rc, std::string("homogenised tangent solve: ") + rve_status_string(rc));
    launch_tangent_mean<R>(tangent_view<R>(h), as<R>(h->x), h->st->dFbar, h->n, h->st->Kmean,
                           h->partials, &h->st->counter[SLOT_MISC], h->s);
    h->launches += 1;
    CK(cudaGetLastError());
    rc = sync_state(h);
    if (rc) return rc;
    for (int a = 0; a < 9; ++a) C[a * ncol + k] = hs->Kmean[a];
  }
  return RVE_OK;
}

// P-bar of the current F into Pb (device P-bar slot and host copy)
static int current_Pbar(rve_t h, double Pb[9]) {
  launch_mean9<double>(h->P, h->n, nullptr, h->partials, &h->st->counter[SLOT_MEAN], MEAN_PBAR,
                       h->st, h->s);
  h->launches += 1;
  const int rc = sync_state(h);
  if (rc) return rc;
  std::memcpy(Pb, h->hst->Pbar, 9 * sizeof(double));
  return RVE_OK;
}

// One increment under mixed control to (Fb_in on the strain-controlled
// components, Pt on S); commits on success, rolls back on failure.
template <typename R>
static int mixed_increment_t(rve_t h, const double Fb_in[9], const double Pt[9], const int* S,
                             int ns, double tol_stress, double tol_newton, double tol_cg,
                             rve_stats* acc) {
  NvtxRange nv("rve mixed_increment");
  double Fb[9];
  std::memcpy(Fb, Fb_in, sizeof(Fb));
  for (int k = 0; k < ns; ++k) Fb[S[k]] = h->Fbar_committed[S[k]];
  double J[81], Rprev[9], dprev[9], rprev = 0.0;
  bool have_J = false;
  for (int m = 1; m <= kMaxMacro; ++m) {
    std::memcpy(h->Fbar, Fb, sizeof(Fb));
    rve_stats s1;
    std::memset(&s1, 0, sizeof(s1));
    int rc = solve_increment_t<R>(h, tol_newton, tol_cg, &s1, false);
    acc->newton_iters += s1.newton_iters;
    acc->cg_iters_total += s1.cg_iters_total;
    acc->macro_iters += 1;
    if (rc) return rc;  // rolled back to the committed state
    double Pb[9];
    rc = current_Pbar(h, Pb);
    if (rc) return rc;
    double Rs[9], rn = 0.0, pn = 0.0;
    for (int c = 0; c < 9; ++c) pn += Pb[c] * Pb[c];
    for (int k = 0; k < ns; ++k) {
      Rs[k] = Pb[S[k]] - Pt[S[k]];
      rn += Rs[k] * Rs[k];
    }
    rn = std::sqrt(rn);
    if (!std::isfinite(rn)) {
      rollback_state(h);
      return fail(h, RVE_ERR_NONFINITE, "mixed control: non-finite P-bar");
    }
    if (ns == 0 || rn <= tol_stress * std::sqrt(pn)) return commit_state(h);
    if (m == kMaxMacro) break;
    if (!have_J || rn > 0.25 * rprev) {
      double Cfull[81];
      int its = 0;
      rc = homogenized_tangent_t<R>(h, S, ns, tol_cg, Cfull, &its);
      acc->cg_iters_total += its;
      acc->tangent_solves += ns;
      if (rc) {
        rollback_state(h);
        return rc;
      }
      for (int i = 0; i < ns; ++i)
        for (int j = 0; j < ns; ++j) J[i * ns + j] = Cfull[S[i] * ns + j];
      have_J = true;
    } else {
      // Broyden: J += ((R - R_prev) - J d) d^T / (d.d)
      double dd = 0.0;
      for (int j = 0; j < ns; ++j) dd += dprev[j] * dprev[j];
      for (int i = 0; i < ns; ++i) {
        double y = Rs[i] - Rprev[i];
        for (int j = 0; j < ns; ++j) y -= J[i * ns + j] * dprev[j];
        for (int j = 0; j < ns; ++j) J[i * ns + j] += y * dprev[j] / dd;
      }
    }
    double A[81], d[9];
    std::memcpy(A, J, sizeof(double) * ns * ns);
    for (int k = 0; k < ns; ++k) d[k] = -Rs[k];
    if (!small_solve(ns, A, d, kSingularPivot)) {
      rollback_state(h);
      return fail(h, RVE_ERR_INVALID,
                  "mixed control: homogenised tangent singular on the stress-controlled "
                  "components (leave a rotation-fixing set of F-bar components prescribed)");
    }
    for (int k = 0; k < ns; ++k) {
      Fb[S[k]] += d[k];
      Rprev[k] = Rs[k];
      dprev[k] = d[k];
    }
    rprev = rn;
  }
  rollback_state(h);
  return fail(h, RVE_ERR_NEWTON_MAXIT, "mixed control: macroscopic Newton did not converge");
}

extern "C" {

int rve_solve_mixed(rve_t h, const double Fbar[9], const double Pbar[9], const int mask[9],
                    double tol_stress, double tol_newton, double tol_cg, int max_cuts,
                    rve_stats* st) {
  NvtxRange nv("rve solve_mixed");
  if (!h || !Fbar || !Pbar || !mask || max_cuts < 0) return RVE_ERR_INVALID;
  if (!(tol_stress > 0.0) || !(tol_newton > 0.0) || !(tol_cg > 0.0))
    return fail(h, RVE_ERR_INVALID, "tolerances must be > 0");
  int S[9], ns = 0;
  for (int c = 0; c < 9; ++c) {
    if (mask[c]) S[ns++] = c;
    if ((!mask[c] && !std::isfinite(Fbar[c])) || (mask[c] && !std::isfinite(Pbar[c])))
      return fail(h, RVE_ERR_INVALID, "non-finite prescribed component");
  }
  h->err.clear();
  const auto t0 = std::chrono::steady_clock::now();
  // the path starts at the committed state: its F-bar and P-bar
  double F0[9], P0[9];
  std::memcpy(F0, h->Fbar_committed, sizeof(F0));
  int rc = current_Pbar(h, P0);
  if (rc) return rc;
  rve_stats acc;
  std::memset(&acc, 0, sizeof(acc));
  double done = 0.0, step = 1.0;
  const double min_step = std::ldexp(1.0, -max_cuts);
  int cuts = 0, sub = 0, streak = 0, result = RVE_OK;
  while (done < 1.0) {
    const double to = std::min(1.0, done + step);
    double Fb[9], Pt[9];
    for (int c = 0; c < 9; ++c) {
      Fb[c] = to >= 1.0 ? Fbar[c] : F0[c] + to * (Fbar[c] - F0[c]);
      Pt[c] = to >= 1.0 ? Pbar[c] : P0[c] + to * (Pbar[c] - P0[c]);
    }
    h->err.clear();
    rc = h->mixed ? mixed_increment_t<float>(h, Fb, Pt, S, ns, tol_stress, tol_newton, tol_cg, &acc)
                  : mixed_increment_t<double>(h, Fb, Pt, S, ns, tol_stress, tol_newton, tol_cg,
                                              &acc);
    if (rc == RVE_OK) {
      done = to;
      if (sub < RVE_MAX_NEWTON_LOG) acc.substep_to[sub] = to;
      ++sub;
      if (++streak >= 2) {
        step = std::min(2.0 * step, 1.0);
        streak = 0;
      }
    } else if (rc == RVE_ERR_NEWTON_MAXIT || rc == RVE_ERR_CG_MAXIT || rc == RVE_ERR_NONFINITE ||
               rc == RVE_ERR_DETF || rc == RVE_ERR_CG_BREAKDOWN) {
      ++cuts;
      streak = 0;
      step *= 0.5;
      if (step < min_step) {
        result = rc;
        break;
      }
    } else {
      result = rc;
      break;
    }
  }
  if (st) {
    *st = acc;
    st->status = result;
    st->substeps = sub;
    st->cuts = cuts;
    st->elapsed_ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  return result;
}

int rve_macro_F(rve_t h, double Fbar[9]) {
  if (!h || !Fbar) return RVE_ERR_INVALID;
  std::memcpy(Fbar, h->Fbar_committed, 9 * sizeof(double));
  return RVE_OK;
}

int rve_get_F(rve_t h, double* dst, int on_device) {
  if (!h || !dst) return RVE_ERR_INVALID;
  return copy_out(h, dst, h->F, 9 * h->n * 8, on_device);
}

int rve_get_P(rve_t h, double* dst, int on_device) {
  if (!h || !dst) return RVE_ERR_INVALID;
  return copy_out(h, dst, h->P, 9 * h->n * 8, on_device);
}

int rve_get_K4(rve_t h, double* dst, int on_device) {
  if (!h || !dst) return RVE_ERR_INVALID;
  // evaluated in float64 in chunks through the spectrum buffer
  size_t chunk = h->spec64_bytes / (81 * sizeof(double));
  if (chunk == 0) return fail(h, RVE_ERR_NOMEM, "scratch too small");
  double* scratch = reinterpret_cast<double*>(h->spec64);
  MatView<double> m = mat_view<double>(h);
  for (size_t v0 = 0; v0 < h->n; v0 += chunk) {
    const size_t cnt = std::min(chunk, h->n - v0);
    if (h->model == RVE_J2) launch_j2_k4_full(h->F, v0, cnt, h->n, m, h->hc, scratch, h->s);
    else launch_svk_k4_full(h->F, v0, cnt, h->n, m, scratch, h->s);
    h->launches += 1;
    CK(cudaMemcpy2DAsync(dst + v0, h->n * sizeof(double), scratch, cnt * sizeof(double),
                         cnt * sizeof(double), 81,
                         on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->s));
  }
  CK(cudaStreamSynchronize(h->s));
  return RVE_OK;
}

}  // extern "C"

// Adjoint solve A lambda = G:(K:W)/n with the CG operator of the handle;
// float32 handles refine in float64 (residual b - A64 lambda).
template <typename RC>
static int adjoint_solve(rve_t h, double tol, int* total_iters) {
  const size_t n9 = 9 * h->n;
  if (std::is_same<RC, float>::value && h->model == RVE_J2) {
    // a mixed J2 handle keeps its tangent in float32 only: one float32 solve
    // of the adjoint system (no float64 refinement), then the float64
    // projection onto compatible fields
    const GridGeom& g = h->g;
    const Twiddles<float>& tw = h->twf;
    cplx<float>* spec = as<cplx<float>>(h->spec_op);
    launch_zfwd<float>(g, SRC_UNIFORM, tangent_view<float>(h), nullptr, nullptr, nullptr,
                       h->st->adjW, h->st, nullptr, spec, tw, h->s);
    launch_fft_y<float>(g, false, spec, nullptr, tw, h->s);
    launch_fft_x_proj<float>(g, 1.0 / (double)h->n, spec, nullptr, tw, h->s);
    launch_fft_y<float>(g, true, spec, nullptr, tw, h->s);
    launch_zinv<float, float>(g, OUT_RESID, spec, nullptr, as<float>(h->r), as<float>(h->x),
                              nullptr, h->st, h->partials, nullptr, tw, h->s);
    h->launches += 5;
    int its = 0;
    const int rc = cg_solve<float>(h, &its);
    if (rc) return fail(h, rc, std::string("adjoint solve: ") + rve_status_string(rc));
    launch_convert<float, double>(as<float>(h->x), h->adj_l, n9, h->s);
    enqueue_project_fp64(h, h->adj_l);
    h->launches += 1;
    *total_iters = its;
    return RVE_OK;
  }
  // b = G : (K : W/n) in float64
  enqueue_operator64(h, SRC_UNIFORM, nullptr, h->st->adjW, h->adj_b);
  CK(cudaMemsetAsync(h->adj_l, 0, n9 * sizeof(double), h->s));
  double b0 = -1.0;
  int its_total = 0;
  const int rounds = h->mixed ? 6 : 1;
  for (int round = 0; round < rounds; ++round) {
    if (round > 0) enqueue_operator64(h, SRC_FIELD, h->adj_l, nullptr, h->tmp64);
    launch_cg_init<RC>(n9, h->adj_b, round > 0 ? h->tmp64 : nullptr, as<RC>(h->r), as<RC>(h->x),
                       h->st, h->partials, h->s);
    h->launches += 1;
    int rc = sync_state(h);
    if (rc) return rc;
    const double bb = std::sqrt(h->hst->bb);
    if (round == 0) b0 = bb;
    if (bb <= tol * b0 || bb == 0.0) break;
    int its = 0;
    rc = cg_solve<RC>(h, &its);
    its_total += its;
    if (rc) return fail(h, rc, std::string("adjoint solve: ") + rve_status_string(rc));
    launch_accumulate<RC>(n9, h->adj_l, as<RC>(h->x), h->s);
    h->launches += 1;
    // float32 increments are compatible only up to float32 round-off; the
    // incompatible part would enter lambda : dP/dmu directly
    if (h->mixed) enqueue_project_fp64(h, h->adj_l);
  }
  *total_iters = its_total;
  return RVE_OK;
}

extern "C" {

int rve_adjoint_grad_mu(rve_t h, const double W[9], double tol_cg, double* grad, int on_device,
                        int* cg_iters) {
  if (!grad) return RVE_ERR_INVALID;
  return rve_adjoint_grad(h, W, tol_cg, nullptr, grad, on_device, cg_iters);
}

}  // extern "C"

// Adjoint gradients of J = W : P-bar for every per-voxel parameter, into
// h->tmp64 as [nparam][n] in the order of rve_create (K, mu[, tau_y0, H]).
// J2: the tangent and the parameter derivatives are those of the last
// committed increment, i.e. with the history at its start (h->hprev).
static int adjoint_grads(rve_t h, const double W[9], double tol_cg, int* cg_iters) {
  int rc = sync_state(h);
  if (rc) return rc;
  SolverState* hs = h->hst;
  std::memset(hs->counter, 0, sizeof(hs->counter));
  for (int c = 0; c < 9; ++c) hs->adjW[c] = W[c] / (double)h->n;
  hs->cg_tol = h->mixed ? std::max(tol_cg, h->opt.cg_tol_floor) : tol_cg;
  hs->cg_atol = h->opt.cg_atol;
  hs->maxit = h->opt.max_cg;
  hs->stag = h->mixed ? kMixedStagnation : 0;
  hs->done = 0;
  rc = push_state(h);
  if (rc) return rc;
  MatView<double> m = mat_view<double>(h);
  const int sym = h->tan == TAN_SYM45;
  if (h->model == RVE_J2) {
    // the consistent tangent of the increment: F with its starting history
    if (h->mixed)
      launch_j2_constitutive<float>(h->F, h->n, m, h->hprev, nullptr, nullptr, as<float>(h->K4),
                                    h->st, h->s, sym);
    else
      launch_j2_constitutive<double>(h->F, h->n, m, h->hprev, nullptr, nullptr,
                                     as<double>(h->K4), h->st, h->s, sym);
    h->launches += 1;
  }
  int its = 0;
  rc = h->mixed ? adjoint_solve<float>(h, tol_cg, &its) : adjoint_solve<double>(h, tol_cg, &its);
  if (h->model == RVE_J2) {
    // back to the tangent of the committed state
    if (h->mixed)
      launch_j2_constitutive<float>(h->F, h->n, m, h->hc, nullptr, nullptr, as<float>(h->K4),
                                    h->st, h->s, sym);
    else
      launch_j2_constitutive<double>(h->F, h->n, m, h->hc, nullptr, nullptr, as<double>(h->K4),
                                     h->st, h->s, sym);
    h->launches += 1;
  }
  if (rc) return rc;
  if (cg_iters) *cg_iters = its;
  if (h->model == RVE_J2) {
    launch_j2_adjoint_grad(h->F, h->n, m, h->hprev, h->adj_l, W, h->tmp64, h->s);
  } else {
    // [K][n] then [mu][n]
    launch_adjoint_grad(h->F, h->adj_l, W, h->n, h->tmp64 + h->n, h->tmp64, h->s);
  }
  h->launches += 1;
  CK(cudaGetLastError());
  return RVE_OK;
}

extern "C" {

int rve_adjoint_grad(rve_t h, const double W[9], double tol_cg, double* grad_K, double* grad_mu,
                     int on_device, int* cg_iters) {
  NvtxRange nv("rve adjoint_grad");
  if (!h || !W || !(grad_K || grad_mu) || !(tol_cg > 0.0)) return RVE_ERR_INVALID;
  int rc = adjoint_grads(h, W, tol_cg, cg_iters);
  if (rc) return rc;
  if (grad_mu) {
    rc = copy_out(h, grad_mu, h->tmp64 + h->n, h->n * sizeof(double), on_device);
    if (rc) return rc;
  }
  if (grad_K) return copy_out(h, grad_K, h->tmp64, h->n * sizeof(double), on_device);
  return RVE_OK;
}

int rve_adjoint_grad_params(rve_t h, const double W[9], double tol_cg, double* grads,
                            int on_device, int* cg_iters) {
  NvtxRange nv("rve adjoint_grad_params");
  if (!h || !W || !grads || !(tol_cg > 0.0)) return RVE_ERR_INVALID;
  const int rc = adjoint_grads(h, W, tol_cg, cg_iters);
  if (rc) return rc;
  return copy_out(h, grads, h->tmp64, (size_t)h->nparam * h->n * sizeof(double), on_device);
}

int rve_tape(rve_t h, int enable) {
  if (!h) return RVE_ERR_INVALID;
  if (h->model != RVE_J2) return fail(h, RVE_ERR_UNSUPPORTED, "tape: J2 only");
  tape_clear(h);
  h->tape_on = enable != 0;
  return RVE_OK;
}

int rve_tape_length(rve_t h) { return h ? (int)h->tape_F.size() : RVE_ERR_INVALID; }

// Reverse sweep over the taped increments (J2, float64 handles): per
// increment m = M..1 the tangent at (F_m, h_{m-1}), the adjoint field of
// G K G lambda = G g with g = (1/n) K W [m = M] + (dH/dF)^T a, then the
// parameter gradient and a = dJ/dh_{m-1}; finally the state's tangent and
// trial history are evaluated again at the current F.
int rve_adjoint_grad_path(rve_t h, const double W[9], double tol_cg, double* grads,
                          int on_device, int* cg_iters) {
  NvtxRange nv("rve adjoint_grad_path");
  if (!h || !W || !grads || !(tol_cg > 0.0)) return RVE_ERR_INVALID;
  if (h->model != RVE_J2 || h->mixed)
    return fail(h, RVE_ERR_UNSUPPORTED, "path adjoint: float64 J2 handles only");
  const int M = (int)h->tape_F.size();
  if (M < 1) return fail(h, RVE_ERR_INVALID, "path adjoint: empty tape (rve_tape before the increments)");
  const size_t n = h->n, n9 = 9 * n;
  int rc = sync_state(h);
  if (rc) return rc;
  SolverState* hs = h->hst;
  std::memset(hs->counter, 0, sizeof(hs->counter));
  for (int c = 0; c < 9; ++c) hs->adjW[c] = W[c] / (double)n;
  hs->cg_tol = tol_cg;
  hs->cg_atol = h->opt.cg_atol;
  hs->maxit = h->opt.max_cg;
  hs->stag = 0;
  hs->done = 0;
  rc = push_state(h);
  if (rc) return rc;
  MatView<double> m = mat_view<double>(h);
  const int sym = h->tan == TAN_SYM45;
  // scratch: g in tmp64 [4][n]; a = dJ/dh in ht and Ft (both rebuilt below)
  double* g = h->tmp64;
  double* a_cur = h->ht;
  double* a_next = h->Ft;
  CK(cudaMemsetAsync(g, 0, 4 * n * sizeof(double), h->s));
  int its_total = 0;
  for (int k = M - 1; k >= 0; --k) {
    const bool last = k == M - 1;
    const double* Fk = h->tape_F[k];
    const double* hk = h->tape_h[k];
    launch_j2_constitutive<double>(Fk, n, m, hk, nullptr, nullptr, as<double>(h->K4), h->st, h->s,
                                   sym);
    h->launches += 1;
    // right-hand side G g
    if (last) {
      enqueue_operator64(h, SRC_UNIFORM, nullptr, h->st->adjW, h->adj_b);
    } else {
      launch_j2_path_gF(Fk, n, m, hk, a_cur, h->adj_b, h->s);
      enqueue_project_fp64(h, h->adj_b);
      h->launches += 1;
    }
    launch_cg_init<double>(n9, h->adj_b, nullptr, as<double>(h->r), as<double>(h->x), h->st,
                           h->partials, h->s);
    h->launches += 1;
    rc = sync_state(h);
    if (rc) return rc;
    int its = 0;
    rc = cg_solve<double>(h, &its);
    its_total += its;
    if (rc) {
      fail(h, rc, std::string("path adjoint solve: ") + rve_status_string(rc));
      break;
    }
    launch_j2_path_step(Fk, n, m, hk, as<double>(h->x), W, last ? 1 : 0, last ? nullptr : a_cur,
                        a_next, g, h->s);
    h->launches += 1;
    std::swap(a_cur, a_next);
  }
  // back to the committed state: tangent and trial history at (F, hc), Ft = F
  launch_j2_constitutive<double>(h->F, n, m, h->hc, h->ht, nullptr, as<double>(h->K4), h->st,
                                 h->s, sym);
  h->launches += 1;
  CK(cudaMemcpyAsync(h->Ft, h->F, n9 * 8, cudaMemcpyDeviceToDevice, h->s));
  if (rc) {
    sync_state(h);
    return rc;
  }
  CK(cudaGetLastError());
  if (cg_iters) *cg_iters = its_total;
  return copy_out(h, grads, g, 4 * n * sizeof(double), on_device);
}

int rve_get_history(rve_t h, double* dst, int on_device) {
  if (!h || !dst || h->model != RVE_J2) return RVE_ERR_INVALID;
  return copy_out(h, dst, h->hc, 7 * h->n * 8, on_device);
}

int rve_homogenized_P(rve_t h, double Pbar[9]) {
  if (!h || !Pbar) return RVE_ERR_INVALID;
  launch_mean9<double>(h->P, h->n, nullptr, h->partials, &h->st->counter[SLOT_MEAN], MEAN_PBAR,
                       h->st, h->s);
  h->launches += 1;
  int rc = sync_state(h);
  if (rc) return rc;
  std::memcpy(Pbar, h->hst->Pbar, sizeof(double) * 9);
  return RVE_OK;
}

int rve_set_F(rve_t h, const double* F, int on_device) {
  if (!h || !F) return RVE_ERR_INVALID;
  int rc = copy_in(h, h->F, F, 9 * h->n * 8, on_device);
  if (rc) return rc;
  {
    // the macroscopic state of the new field
    launch_mean9<double>(h->F, h->n, nullptr, h->partials, &h->st->counter[SLOT_MEAN], MEAN_PBAR,
                         h->st, h->s);
    h->launches += 1;
    rc = sync_state(h);
    if (rc) return rc;
    std::memcpy(h->Fbar_committed, h->hst->Pbar, sizeof(h->Fbar_committed));
  }
  CK(cudaMemcpyAsync(h->Ft, h->F, 9 * h->n * 8, cudaMemcpyDeviceToDevice, h->s));
  if (h->hprev)  // no increment since: the committed history is its own start
    CK(cudaMemcpyAsync(h->hprev, h->hc, 7 * h->n * 8, cudaMemcpyDeviceToDevice, h->s));
  tape_clear(h);  // a new path starts here
  std::memset(h->hst, 0, sizeof(SolverState));
  rc = push_state(h);
  if (rc) return rc;
  enqueue_constitutive(h);
  rc = sync_state(h);
  if (rc) return rc;
  CK(cudaGetLastError());
  return check_flags(h);
}

int rve_apply_operator(rve_t h, const double* dF, double* out, int on_device) {
  if (!h || !dF || !out) return RVE_ERR_INVALID;
  const size_t n9 = 9 * h->n;
  int rc = copy_in(h, h->tmp64, dF, n9 * 8, on_device);
  if (rc) return rc;
  const GridGeom& g = h->g;
  if (h->mixed) {
    float* in = as<float>(h->p);
    float* o = as<float>(h->Ap);
    cplx<float>* spec = as<cplx<float>>(h->spec_op);
    launch_convert<double, float>(h->tmp64, in, n9, h->s);
    launch_zfwd<float>(g, SRC_FIELD, tangent_view<float>(h), in, nullptr, nullptr, nullptr, h->st,
                       nullptr, spec, h->twf, h->s);
    launch_fft_y<float>(g, false, spec, nullptr, h->twf, h->s);
    launch_fft_x_proj<float>(g, 1.0 / (double)h->n, spec, nullptr, h->twf, h->s);
    launch_fft_y<float>(g, true, spec, nullptr, h->twf, h->s);
    launch_zinv<float, float>(g, OUT_PLAIN, spec, o, nullptr, nullptr, nullptr, h->st, h->partials,
                              nullptr, h->twf, h->s);
    launch_convert<float, double>(o, h->tmp64, n9, h->s);
    h->launches += 7;
  } else {
    double* o = as<double>(h->Ap);
    launch_zfwd<double>(g, SRC_FIELD, tangent_view<double>(h), h->tmp64, nullptr, nullptr, nullptr,
                        h->st, nullptr, h->spec64, h->twd, h->s);
    launch_fft_y<double>(g, false, h->spec64, nullptr, h->twd, h->s);
    launch_fft_x_proj<double>(g, 1.0 / (double)h->n, h->spec64, nullptr, h->twd, h->s);
    launch_fft_y<double>(g, true, h->spec64, nullptr, h->twd, h->s);
    launch_zinv<double, double>(g, OUT_PLAIN, h->spec64, o, nullptr, nullptr, nullptr, h->st,
                                h->partials, nullptr, h->twd, h->s);
    launch_convert<double, double>(o, h->tmp64, n9, h->s);
    h->launches += 6;
  }
  CK(cudaGetLastError());
  return copy_out(h, out, h->tmp64, n9 * 8, on_device);
}

int rve_project(rve_t h, const double* A, double* out, int on_device) {
  if (!h || !A || !out) return RVE_ERR_INVALID;
  const size_t n9 = 9 * h->n;
  int rc = copy_in(h, h->tmp64, A, n9 * 8, on_device);
  if (rc) return rc;
  enqueue_project_fp64(h, h->tmp64);
  CK(cudaGetLastError());
  return copy_out(h, out, h->tmp64, n9 * 8, on_device);
}

int rve_launch_count(rve_t h, long long* count) {
  if (!h || !count) return RVE_ERR_INVALID;
  *count = h->launches;
  return RVE_OK;
}

int rve_kernel_timing(rve_t h, int family, int enable) {
  if (!h || family < 0 || family > 5) return RVE_ERR_INVALID;
  cudaStreamSynchronize(h->s);
  for (auto& t : h->timed) {
    h->ev_pool.push_back(t.a);
    h->ev_pool.push_back(t.b);
  }
  h->timed.clear();
  h->solve_iters.clear();
  h->timing_family = enable ? family : -1;
  return RVE_OK;
}

int rve_set_wait_polls(rve_t h, unsigned polls) {
  if (!h) return RVE_ERR_INVALID;
  h->g.wait_polls = polls;
  return RVE_OK;
}

int rve_kernel_time(rve_t h, double* total_ms, long long* launches) {
  if (!h || !total_ms || !launches) return RVE_ERR_INVALID;
  CK(cudaStreamSynchronize(h->s));
  double tot = 0.0;
  long long cnt = 0;
  for (auto& t : h->timed) {
    // only launches of iterations that did work (those after convergence
    // return at once and are not counted)
    int eff = -1;
    for (auto& si : h->solve_iters)
      if (si.first == t.solve) eff = si.second;
    if (eff < 0 || t.iter >= eff) continue;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, t.a, t.b) == cudaSuccess) {
      tot += ms;
      cnt++;
    }
  }
  *total_ms = tot;
  *launches = cnt;
  return RVE_OK;
}

}  // extern "C"

// ===========================================================================
// Batches of independent cells.  Every cell keeps its own handle, buffers and
// device state; the cells' per-iteration kernel chains run on a pool of
// streams as independent branches of one CUDA graph (a graph launch advances
// every cell by kGraphIters CG iterations; cells whose CG has finished return
// at once from each kernel).  Newton steps run in lockstep on the host with
// converged cells masked out.
// ===========================================================================
namespace {
constexpr int kBatchStreams = 64;
constexpr int kGraphIters = 4;
// once few cells are left (the long CG runs of hard cells), more iterations
// per graph launch: fewer host round trips; iterations enqueued after a
// cell's CG has finished return at once
constexpr int kGraphItersFew = 16;
constexpr size_t kFewCells = 8;

__global__ void k_gather_cg(SolverState* const* st, int nrve, int* out) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nrve; b += gridDim.x * blockDim.x) {
    out[3 * b] = st[b]->done;
    out[3 * b + 1] = st[b]->status;
    out[3 * b + 2] = st[b]->it;
  }
}
}  // namespace

struct rve_batch_s {
  std::vector<rve_t> rv;
  std::vector<cudaStream_t> streams;
  cudaStream_t s0 = nullptr;
  bool mixed = false;
  cudaGraphExec_t exec = nullptr;
  std::vector<int> graph_members;  // cells captured in exec
  int graph_iters = kGraphIters;   // CG iterations per graph launch
  Fs4Batch* fs4 = nullptr;         // batched passes of the captured iteration
  int fs4_cells = 0;               // cells in it (the others are graph branches)
  SolverState** d_states = nullptr;
  int* d_info = nullptr;
  int* h_info = nullptr;
  std::string err;
  long long launches = 0;
};

namespace {

int bfail(rve_batch_t b, int code, const std::string& msg) {
  if (b) b->err = msg;
  return code;
}

void batch_sync_all(rve_batch_t b) {
  for (auto s : b->streams) cudaStreamSynchronize(s);
  cudaStreamSynchronize(b->s0);
}

// capture kGraphIters CG iterations of the given cells as parallel branches
template <typename R>
int batch_capture(rve_batch_t b, const std::vector<int>& cells) {
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  const int iters = cells.size() <= kFewCells ? kGraphItersFew : kGraphIters;
  b->graph_iters = iters;
  // float32 CG of cells whose passes all have batched four-step kernels:
  // their launches are recorded (not run) and become one launch per pass
  fs4_batch_free(b->fs4);
  b->fs4 = nullptr;
  b->fs4_cells = 0;
  std::vector<int> branch;
  if constexpr (std::is_same<R, float>::value) {
    std::vector<int> batched;
    for (int c : cells) {
      rve_t h = b->rv[c];
      if (fs4_batch_eligible(h->g, h->mixed, h->tan, h->precond)) batched.push_back(c);
      else branch.push_back(c);
    }
    if (batched.size() > 1) {
      b->fs4 = fs4_batch_new();
      fs4_batch_record(b->fs4);
      for (int c : batched) {  // recorded, not launched: the cell's count stays
        const long long l0 = b->rv[c]->launches;
        enqueue_cg_iteration<R>(b->rv[c], -1);
        b->rv[c]->launches = l0;
      }
      fs4_batch_record(nullptr);
      const int nb = fs4_batch_cells(b->fs4);
      if (nb != (int)batched.size() || fs4_batch_upload(b->fs4) != cudaSuccess) {
        fs4_batch_free(b->fs4);
        b->fs4 = nullptr;
        return RVE_ERR_CUDA;
      }
      b->fs4_cells = nb;
    } else {
      branch.insert(branch.end(), batched.begin(), batched.end());
    }
  } else {
    branch = cells;
  }
  cudaGraph_t graph;
  cudaEvent_t fork;
  if (cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess) return RVE_ERR_CUDA;
  std::vector<cudaEvent_t> joins(b->streams.size());
  for (auto& e : joins) cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
  if (cudaStreamBeginCapture(b->s0, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return RVE_ERR_CUDA;
  cudaEventRecord(fork, b->s0);
  std::vector<bool> used(b->streams.size(), false);
  if (b->fs4)
    for (int k = 0; k < iters; ++k) fs4_batch_launch(b->fs4, b->s0);
  for (int c : branch) {
    rve_t h = b->rv[c];
    const size_t si = (size_t)c % b->streams.size();
    if (!used[si]) {
      cudaStreamWaitEvent(b->streams[si], fork, 0);
      used[si] = true;
    }
    for (int k = 0; k < iters; ++k) enqueue_cg_iteration<R>(h, -1);
  }
  for (size_t si = 0; si < b->streams.size(); ++si)
    if (used[si]) {
      cudaEventRecord(joins[si], b->streams[si]);
      cudaStreamWaitEvent(b->s0, joins[si], 0);
    }
  const cudaError_t e1 = cudaStreamEndCapture(b->s0, &graph);
  cudaEventDestroy(fork);
  for (auto& e : joins) cudaEventDestroy(e);
  if (e1 != cudaSuccess) return RVE_ERR_CUDA;
  const cudaError_t e2 = cudaGraphInstantiate(&b->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e2 != cudaSuccess) return RVE_ERR_CUDA;
  b->graph_members = cells;
  return RVE_OK;
}

// CG for every cell in `active` (their right-hand sides are set up):
// graph launches until every cell's CG reports done.
template <typename R>
int batch_cg_phase(rve_batch_t b, const std::vector<int>& active, std::vector<int>& iters,
                   std::vector<int>& status) {
  const int nrve = (int)b->rv.size();
  if (active.empty()) return RVE_OK;
  if (b->graph_members != active) {
    int rc = batch_capture<R>(b, active);
    if (rc) return bfail(b, rc, "graph capture of the batched CG iteration failed");
  }
  for (int c : active)
    if (b->rv[c]->precond) enqueue_precondition(b->rv[c]);
  batch_sync_all(b);
  long long guard = 0;
  const long long max_launch = (long long)b->rv[active[0]]->opt.max_cg / kGraphIters + 4096;
  while (true) {
    if (cudaGraphLaunch(b->exec, b->s0) != cudaSuccess) return bfail(b, RVE_ERR_CUDA, "graph launch");
    b->launches += ((b->fs4 ? 5 : 0) + (long long)(b->graph_members.size() - b->fs4_cells) *
                                          (b->mixed ? 5 : 6)) * b->graph_iters;
    k_gather_cg<<<(nrve + 127) / 128, 128, 0, b->s0>>>(b->d_states, nrve, b->d_info);
    cudaMemcpyAsync(b->h_info, b->d_info, sizeof(int) * 3 * nrve, cudaMemcpyDeviceToHost, b->s0);
    if (cudaStreamSynchronize(b->s0) != cudaSuccess) return bfail(b, RVE_ERR_CUDA, "batched CG");
    bool all = true;
    for (int c : active) all = all && b->h_info[3 * c];
    if (all) break;
    // a batched launch schedules the blocks of every member cell, finished
    // or not: once half of the members have finished, capture the rest
    if (b->fs4) {
      std::vector<int> running;
      for (int c : b->graph_members)
        if (!b->h_info[3 * c]) running.push_back(c);
      if (2 * running.size() <= b->graph_members.size()) {
        int rc = batch_capture<R>(b, running);
        if (rc) return bfail(b, rc, "graph capture of the batched CG iteration failed");
      }
    }
    if (++guard > max_launch) return bfail(b, RVE_ERR_TIMEOUT, "batched CG state stopped advancing");
  }
  for (int c : active) {
    enqueue_cg_finish<R>(b->rv[c]);
    iters[c] = b->h_info[3 * c + 2];
    int st = b->h_info[3 * c + 1];
    if (b->mixed && st == RVE_DEV_ERR_CG_BREAKDOWN && iters[c] >= 1) st = RVE_OK;
    status[c] = st;
  }
  return RVE_OK;
}

// One increment for the cells in `cells` (F-bar of cell c at Fbar + 9 c);
// result[c] receives each cell's status.
template <typename R>
int batch_solve_t(rve_batch_t b, const double* Fbar, double tol_newton, double tol_cg,
                  rve_stats* stats, const std::vector<int>& cells, std::vector<int>& result) {
  const int nrve = (int)b->rv.size();
  std::vector<int> active, newton(nrve, 0), cgtot(nrve, 0);
  std::vector<int> iters(nrve, 0), status(nrve, 0);
  std::vector<double> prev(nrve, 0.0), prev2(nrve, 0.0);
  for (int c : cells) result[c] = RVE_OK;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  batch_sync_all(b);
  cudaEventRecord(e0, b->s0);
  for (int c : cells) {
    rve_t h = b->rv[c];
    rve_set_macro_F(h, Fbar + 9 * c);
    SolverState* hs = h->hst;
    std::memset(hs, 0, sizeof(SolverState));
    hs->cg_tol = h->mixed ? std::max(tol_cg, h->opt.cg_tol_floor) : tol_cg;
    hs->cg_atol = h->opt.cg_atol;
    hs->maxit = h->opt.max_cg;
    hs->stag = h->mixed ? kMixedStagnation : 0;
    std::memcpy(hs->Fbar, h->Fbar, sizeof(hs->Fbar));
    push_state(h);
    enqueue_predictor<R>(h);
    launch_shifted_norm(h->F, h->n, h->st, h->partials, h->s);
    h->launches += 1;
    active.push_back(c);
  }
  const int max_newton = b->rv[0]->opt.max_newton;
  for (int i = 0; i < max_newton && !active.empty(); ++i) {
    int rc = batch_cg_phase<R>(b, active, iters, status);
    if (rc) return rc;
    std::vector<int> still;
    for (int c : active) {
      rve_t h = b->rv[c];
      cgtot[c] += iters[c];
      if (stats && i < RVE_MAX_NEWTON_LOG) stats[c].cg_iters[i] = iters[c];
      if (status[c]) {
        result[c] = status[c];
        continue;
      }
      if (h->mixed) {
        enqueue_mixed_update<R>(h, i == 0);
      } else {
        launch_mean9<R>(as<R>(h->x), h->n, nullptr, h->partials, &h->st->counter[SLOT_MEAN],
                        MEAN_X, h->st, h->s);
        launch_newton_update<R>(h->F, as<R>(h->x), h->n, h->st, h->partials, i == 0, h->s);
        h->launches += 2;
      }
      enqueue_constitutive(h);
      enqueue_residual<R>(h);
      still.push_back(c);
    }
    active.clear();
    for (int c : still) {
      rve_t h = b->rv[c];
      if (sync_state(h)) return bfail(b, RVE_ERR_CUDA, "batched Newton step");
      newton[c] = i + 1;
      const double rel = std::sqrt(h->hst->dF2 / h->hst->Fn2);
      if (stats && i < RVE_MAX_NEWTON_LOG) {
        stats[c].rel_update[i] = rel;
        stats[c].residual[i] = std::sqrt(h->hst->bb);
      }
      int frc = check_flags(h, false);
      if (!frc && !std::isfinite(rel)) frc = RVE_ERR_NONFINITE;
      if (!frc && (rel > kDivergedUpdate || (i >= 3 && rel > prev[c] && prev[c] > prev2[c])))
        frc = RVE_ERR_NEWTON_MAXIT;
      prev2[c] = prev[c];
      prev[c] = rel;
      if (frc) {
        result[c] = frc;
        continue;
      }
      if (rel < tol_newton && i > 0) {  // converged; det F > 0 required there
        result[c] = check_flags(h, true);
        continue;
      }
      active.push_back(c);
    }
    // cells that left the active set must not iterate in later graph launches
    for (int c : still)
      if (std::find(active.begin(), active.end(), c) == active.end()) {
        const int one = 1;
        cudaMemcpyAsync(&b->rv[c]->st->done, &one, sizeof(int), cudaMemcpyHostToDevice,
                        b->rv[c]->s);
      }
  }
  for (int c : active) result[c] = RVE_ERR_NEWTON_MAXIT;
  int worst = RVE_OK;
  for (int c : cells) {
    rve_t h = b->rv[c];
    const size_t n9 = 9 * h->n;
    if (result[c] == RVE_OK) {
      commit_state(h);
    } else {
      cudaMemcpyAsync(h->F, h->Ft, n9 * 8, cudaMemcpyDeviceToDevice, h->s);
      enqueue_constitutive(h);
      if (worst == RVE_OK) worst = result[c];
    }
  }
  batch_sync_all(b);
  cudaEventRecord(e1, b->s0);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (stats)
    for (int c : cells) {
      stats[c].status = result[c];
      stats[c].newton_iters += newton[c];
      stats[c].cg_iters_total += cgtot[c];
      stats[c].elapsed_ms += ms;
    }
  if (cudaGetLastError() != cudaSuccess) return bfail(b, RVE_ERR_CUDA, "batched increment");
  if (worst) b->err = "at least one cell failed (see its stats)";
  return worst;
}

}  // namespace

extern "C" {

int rve_batch_create(rve_batch_t* out, int nrve, const int* dims, int model, const int* nphase,
                     const uint8_t* const* phase, const double* const* phase_params,
                     const rve_options* opt) {
  if (!out || nrve < 1 || !dims || !nphase || !phase || !phase_params) return RVE_ERR_INVALID;
  *out = nullptr;
  rve_batch_t b = new rve_batch_s();
  rve_options o;
  if (opt) o = *opt;
  else rve_default_options(&o);
  if (o.workspace) {
    delete b;
    return RVE_ERR_INVALID;  // every cell allocates its own workspace
  }
  b->mixed = o.precision == RVE_MIXED;
  // the batch runs on streams of its own (graph capture needs a non-default
  // stream); every batch call synchronises them before returning
  if (cudaStreamCreateWithFlags(&b->s0, cudaStreamNonBlocking) != cudaSuccess) {
    delete b;
    return RVE_ERR_CUDA;
  }
  const int ns = std::min(nrve, kBatchStreams);
  for (int i = 0; i < ns; ++i) {
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      rve_batch_destroy(b);
      return RVE_ERR_CUDA;
    }
    b->streams.push_back(s);
  }
  for (int c = 0; c < nrve; ++c) {
    rve_options oc = o;
    oc.stream = b->streams[c % ns];
    rve_t h = nullptr;
    const int rc = rve_create(&h, dims[3 * c], dims[3 * c + 1], dims[3 * c + 2], model, nphase[c],
                              phase[c], phase_params[c], nullptr, &oc);
    if (rc) {
      rve_batch_destroy(b);
      return rc;
    }
    b->rv.push_back(h);
  }
  std::vector<SolverState*> ptrs(nrve);
  for (int c = 0; c < nrve; ++c) ptrs[c] = b->rv[c]->st;
  if (cudaMalloc(&b->d_states, sizeof(SolverState*) * nrve) != cudaSuccess ||
      cudaMalloc(&b->d_info, sizeof(int) * 3 * nrve) != cudaSuccess ||
      cudaMallocHost(&b->h_info, sizeof(int) * 3 * nrve) != cudaSuccess) {
    rve_batch_destroy(b);
    return RVE_ERR_NOMEM;
  }
  cudaMemcpy(b->d_states, ptrs.data(), sizeof(SolverState*) * nrve, cudaMemcpyHostToDevice);
  *out = b;
  return RVE_OK;
}

void rve_batch_destroy(rve_batch_t b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  fs4_batch_free(b->fs4);
  for (rve_t h : b->rv) rve_destroy(h);
  for (auto s : b->streams) {
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  }
  if (b->d_states) cudaFree(b->d_states);
  if (b->d_info) cudaFree(b->d_info);
  if (b->h_info) cudaFreeHost(b->h_info);
  if (b->s0) {
    cudaStreamSynchronize(b->s0);
    cudaStreamDestroy(b->s0);
  }
  delete b;
}

int rve_batch_solve(rve_batch_t b, const double* Fbar, double tol_newton, double tol_cg,
                    rve_stats* stats) {
  return rve_batch_solve_step(b, Fbar, tol_newton, tol_cg, 0, stats);
}

int rve_batch_solve_step(rve_batch_t b, const double* Fbar, double tol_newton, double tol_cg,
                         int max_cuts, rve_stats* stats) {
  NvtxRange nv("rve batch_solve_step");
  if (!b || !Fbar || !(tol_newton > 0.0) || !(tol_cg > 0.0) || max_cuts < 0)
    return RVE_ERR_INVALID;
  b->err.clear();
  const int nrve = (int)b->rv.size();
  if (stats) std::memset(stats, 0, sizeof(rve_stats) * nrve);
  // every cell follows the straight path from its committed F-bar; failed
  // increments (rolled back) are retried with half the step, two successes
  // in a row double it (as rve_solve_step)
  std::vector<double> F0(9 * nrve), target(Fbar, Fbar + 9 * nrve), sub(9 * nrve);
  std::vector<double> done(nrve, 0.0), step(nrve, 1.0);
  std::vector<int> cuts(nrve, 0), nsub(nrve, 0), result(nrve, RVE_OK), fin(nrve, RVE_OK);
  std::vector<int> streak(nrve, 0);
  const double min_step = std::ldexp(1.0, -max_cuts);
  for (int c = 0; c < nrve; ++c) std::memcpy(&F0[9 * c], b->rv[c]->Fbar_committed, 9 * sizeof(double));
  std::vector<int> open;
  for (int c = 0; c < nrve; ++c) open.push_back(c);
  int worst = RVE_OK;
  while (!open.empty()) {
    std::vector<double> to(nrve, 0.0);
    for (int c : open) {
      to[c] = std::min(1.0, done[c] + step[c]);
      for (int k = 0; k < 9; ++k)
        sub[9 * c + k] = (to[c] >= 1.0) ? target[9 * c + k]
                                        : F0[9 * c + k] + to[c] * (target[9 * c + k] - F0[9 * c + k]);
    }
    const int rc = b->mixed ? batch_solve_t<float>(b, sub.data(), tol_newton, tol_cg, stats, open, result)
                            : batch_solve_t<double>(b, sub.data(), tol_newton, tol_cg, stats, open, result);
    if (rc == RVE_ERR_CUDA || rc == RVE_ERR_TIMEOUT) return rc;
    std::vector<int> next;
    for (int c : open) {
      if (result[c] == RVE_OK) {
        done[c] = to[c];
        if (nsub[c] < RVE_MAX_NEWTON_LOG && stats) stats[c].substep_to[nsub[c]] = to[c];
        ++nsub[c];
        if (++streak[c] >= 2) {
          step[c] = std::min(2.0 * step[c], 1.0);
          streak[c] = 0;
        }
        if (done[c] < 1.0) next.push_back(c);
      } else {
        ++cuts[c];
        streak[c] = 0;
        step[c] *= 0.5;
        if (step[c] >= min_step) {
          next.push_back(c);
        } else {
          fin[c] = result[c];
          if (worst == RVE_OK) worst = result[c];
        }
      }
    }
    open.swap(next);
  }
  for (int c = 0; c < nrve; ++c) std::memcpy(b->rv[c]->Fbar, &target[9 * c], 9 * sizeof(double));
  if (stats)
    for (int c = 0; c < nrve; ++c) {
      stats[c].status = fin[c];
      stats[c].substeps = nsub[c];
      stats[c].cuts = cuts[c];
    }
  if (worst) b->err = "at least one cell failed (see its stats)";
  return worst;
}

int rve_batch_size(rve_batch_t b) { return b ? (int)b->rv.size() : 0; }

rve_t rve_batch_cell(rve_batch_t b, int i) {
  if (!b || i < 0 || i >= (int)b->rv.size()) return nullptr;
  return b->rv[i];
}

int rve_batch_homogenized_P(rve_batch_t b, double* Pbar) {
  if (!b || !Pbar) return RVE_ERR_INVALID;
  for (size_t c = 0; c < b->rv.size(); ++c) {
    const int rc = rve_homogenized_P(b->rv[c], Pbar + 9 * c);
    if (rc) return rc;
  }
  return RVE_OK;
}

int rve_batch_launch_count(rve_batch_t b, long long* count) {
  if (!b || !count) return RVE_ERR_INVALID;
  long long t = b->launches;
  for (rve_t h : b->rv) t += h->launches;
  *count = t;
  return RVE_OK;
}

const char* rve_batch_last_error(rve_batch_t b) { return b ? b->err.c_str() : "null batch"; }

}  // extern "C"
