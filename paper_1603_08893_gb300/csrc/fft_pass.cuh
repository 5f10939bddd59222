// Pieces shared by the FFT pass kernels (kernels_fft.cu, kernels_fft4.cu).
#pragma once
#include "kernels.h"

#ifndef FFT_THREADS
#define FFT_THREADS 256
#endif
// float kernels: three CTAs per SM (<= 85 registers); double: two (<= 128)
#define FFT_BOUNDS(R) __launch_bounds__(FFT_THREADS, sizeof(R) == 4 ? 3 : 2)

template <typename R>
RVE_DEV R signed_freq(int k, int n) {
  return (R)((k <= (n - 1) / 2) ? k : k - n);
}

template <typename R>
struct LineParams {
  GridGeom g;
  int t, grp;  // kz tile and groups (y pass)
  double scale;
  cplx<R>* spec;
  const int* done;
  const cplx<R>* tw;
};

// ---------------------------------------------------------------------------
// 16-byte asynchronous global->shared copies (cp.async): a tile's loads are
// in flight while the previous tile is transformed.  bytes = 0 zero-fills.
// ---------------------------------------------------------------------------
RVE_DEV void cp_async16(void* sdst, const void* gsrc, int bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gsrc), "r"(bytes));
}
RVE_DEV void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
RVE_DEV void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// Tiles of the strided passes: `rows` rows of T complex values (T a power of
// two, 64 bytes); row r of the tile starts at gbase + r * rstride.  Rows are
// copied in 16-byte chunks; chunks past the padded row length are zero-filled
// and not read.
template <typename R>
RVE_DEV void issue_tile(cplx<R>* sbuf, const cplx<R>* gbase, size_t rstride, int rows, int T,
                        int ts, int kz0, int hzp, const cplx<R>* any_valid) {
  constexpr int EPC = 16 / sizeof(cplx<R>);  // complex values per chunk
  const int cpr = T / EPC;                   // chunks per row (power of two)
  const int cs = __ffs(cpr) - 1;
  const int nch = rows * cpr;
  for (int c = threadIdx.x; c < nch; c += blockDim.x) {
    const int row = c >> cs;
    const int t = (c & (cpr - 1)) * EPC;
    const bool ok = (kz0 + t) < hzp;
    const cplx<R>* src = ok ? gbase + (size_t)row * rstride + t : any_valid;
    cp_async16(sbuf + (row << ts) + t, src, ok ? 16 : 0);
  }
}


// --------------------------------------------------------------------------
// Input stage: tangent contraction of one voxel.
//   FULL81: out_(3a+b) = (K : in)_ab = sum_kl K_(b a k l) in_(3k+l)
//           (delta P_ji = K_ijkl delta F_kl, Eq. iter:varP)
//   SVK   : linearisation of P = F.S with S = lambda tr(E) I + 2 mu E:
//           dP = dF.S + F.(lambda tr(dE) I + 2 mu dE), dE = sym(F^T dF)
// --------------------------------------------------------------------------
// The SVK inputs of the tangent (F, S or its parameters) are loaded by
// tangent_pre before the caller's other loads and stores, so that every
// global load of a voxel is in flight at once; tangent_post contracts.
template <typename R>
struct TanPre {
  R F[9];
  R S[6];  // from T.Sop when given
  R lam, mu;
};

template <typename R, int TAN>
RVE_DEV void tangent_pre(const TangentView<R>& T, size_t v, size_t n, TanPre<R>& q) {
  if constexpr (TAN == TAN_SVK) {
#pragma unroll
    for (int c = 0; c < 9; ++c) q.F[c] = __ldg(T.Fop + (size_t)c * n + v);
    q.lam = T.mat.get(v, 0);
    q.mu = T.mat.get(v, 1);
    if (T.Sop) {
#pragma unroll
      for (int c = 0; c < 6; ++c) q.S[c] = __ldg(T.Sop + (size_t)c * n + v);
    }
  }
}

template <typename R, int TAN>
RVE_DEV void tangent_post(const TangentView<R>& T, size_t v, size_t n, const TanPre<R>& q,
                          const R (&in)[9], R (&out)[9]) {
  if constexpr (TAN == TAN_FULL81) {
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        R s = 0;
#pragma unroll
        for (int kl = 0; kl < 9; ++kl) s = fma(__ldg(T.K4 + (size_t)((b * 3 + a) * 9 + kl) * n + v), in[kl], s);
        out[3 * a + b] = s;
      }
  } else if constexpr (TAN == TAN_SYM45) {
#pragma unroll
    for (int r = 0; r < 9; ++r) {
      R s = 0;
#pragma unroll
      for (int c = 0; c < 9; ++c) s = fma(__ldg(T.K4 + (size_t)sym45_index(r, c) * n + v), in[c], s);
      out[r] = s;
    }
  } else if constexpr (TAN == TAN_SVK) {
    const R* F = q.F;
    const R lam = q.lam, mu = q.mu;
    R S[3][3];
    if (T.Sop) {
      S[0][0] = q.S[0]; S[1][1] = q.S[1]; S[2][2] = q.S[2];
      S[0][1] = S[1][0] = q.S[3]; S[0][2] = S[2][0] = q.S[4]; S[1][2] = S[2][1] = q.S[5];
    } else {
      R E[3][3];
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          R c = F[a] * F[b] + F[3 + a] * F[3 + b] + F[6 + a] * F[6 + b];
          E[a][b] = R(0.5) * (c - (a == b ? R(1) : R(0)));
        }
      const R tr = E[0][0] + E[1][1] + E[2][2];
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) S[a][b] = 2 * mu * E[a][b] + (a == b ? lam * tr : R(0));
    }
    // dE = sym(F^T in)
    R dE[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const R fa = F[a] * in[b] + F[3 + a] * in[3 + b] + F[6 + a] * in[6 + b];
        const R fb = F[b] * in[a] + F[3 + b] * in[3 + a] + F[6 + b] * in[6 + a];
        dE[a][b] = R(0.5) * (fa + fb);
      }
    const R trd = dE[0][0] + dE[1][1] + dE[2][2];
    R dS[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) dS[a][b] = 2 * mu * dE[a][b] + (a == b ? lam * trd : R(0));
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        R s = 0;
#pragma unroll
        for (int c = 0; c < 3; ++c) s += in[3 * a + c] * S[c][b] + F[3 * a + c] * dS[c][b];
        out[3 * a + b] = s;
      }
  } else {
#pragma unroll
    for (int c = 0; c < 9; ++c) out[c] = in[c];
  }
}

template <typename R>
struct ZfwdParams {
  GridGeom g;
  int lz;
  int src;
  TangentView<R> tan;
  const R* field;
  const double* field64;  // SRC_FIELD input of the float-float passes
  const R* r;
  R* p;
  const double* unif;
  SolverState* st;
  const int* done;
  cplx<R>* spec;
  const cplx<R>* tw;
  R* x;               // SRC_CGPX
  double* partials;   // SRC_CGPX
};


// CG scalars every voxel of the first pass needs, read once per CTA before
// any block can overwrite them (the step length is written by the last
// block of the same kernel).
template <typename R>
struct ZfwdScalars {
  bool first;
  R beta, alpha_prev;
};

template <typename R, int SRC>
RVE_DEV ZfwdScalars<R> zfwd_scalars(const ZfwdParams<R>& P) {
  ZfwdScalars<R> s{true, R(0), R(0)};
  if (SRC == SRC_CGP || SRC == SRC_CGPX) {
    s.first = (P.st->it == 0);
    s.beta = (R)P.st->beta;
    s.alpha_prev = (R)P.st->alpha;
  }
  return s;
}

// Input stage of the first pass for voxel v: the field itself, the CG
// direction p = r + beta p (SRC_CGPX also applies the previous step
// x += alpha p and accumulates p.(K:p)), or a uniform tensor; then the
// tangent.  Every global load of the voxel is issued before its stores.
template <typename R, int SRC, int TAN, typename A>
RVE_DEV void zfwd_voxel(const ZfwdParams<R>& P, const ZfwdScalars<R>& sc, size_t v, R (&out)[9],
                        A& pkp) {
  const size_t n = P.g.n;
  TanPre<R> q;
  tangent_pre<R, TAN>(P.tan, v, n, q);
  R in[9];
  if constexpr (SRC == SRC_FIELD) {
    if constexpr (is_dfl<R>::value) {
#pragma unroll
      for (int c = 0; c < 9; ++c) in[c] = R(P.field64[(size_t)c * n + v]);
    } else {
#pragma unroll
      for (int c = 0; c < 9; ++c) in[c] = P.field[(size_t)c * n + v];
    }
  } else if constexpr (SRC == SRC_CGP) {
    R rr[9], pp[9];
#pragma unroll
    for (int c = 0; c < 9; ++c) rr[c] = P.r[(size_t)c * n + v];
    if (!sc.first) {
#pragma unroll
      for (int c = 0; c < 9; ++c) pp[c] = P.p[(size_t)c * n + v];
    }
#pragma unroll
    for (int c = 0; c < 9; ++c) in[c] = sc.first ? rr[c] : fma(sc.beta, pp[c], rr[c]);
  } else if constexpr (SRC == SRC_CGPX) {
    R rr[9], pp[9], xx[9];
#pragma unroll
    for (int c = 0; c < 9; ++c) rr[c] = P.r[(size_t)c * n + v];
    if (!sc.first) {
#pragma unroll
      for (int c = 0; c < 9; ++c) {
        pp[c] = P.p[(size_t)c * n + v];
        xx[c] = P.x[(size_t)c * n + v];
      }
#pragma unroll
      for (int c = 0; c < 9; ++c) P.x[(size_t)c * n + v] = fma(sc.alpha_prev, pp[c], xx[c]);
    }
#pragma unroll
    for (int c = 0; c < 9; ++c) in[c] = sc.first ? rr[c] : fma(sc.beta, pp[c], rr[c]);
  } else {
#pragma unroll
    for (int c = 0; c < 9; ++c) in[c] = (R)P.unif[c];
  }
  tangent_post<R, TAN>(P.tan, v, n, q, in, out);
  if constexpr (SRC == SRC_CGP || SRC == SRC_CGPX) {
#pragma unroll
    for (int c = 0; c < 9; ++c) P.p[(size_t)c * n + v] = in[c];
  }
  if constexpr (SRC == SRC_CGPX) {
    R sp = 0;
#pragma unroll
    for (int c = 0; c < 9; ++c) sp = fma(in[c], out[c], sp);
    pkp += (A)sp;
  }
}

RVE_DEV void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

// One thread: bulk prefetch into L2 of the 16-byte-aligned span around
// [p, p + bytes) (the span stays inside the allocation: arrays start 256-byte
// aligned in one workspace with slack after the last one)
RVE_DEV void bulk_prefetch_l2(const void* p, size_t bytes) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(p) & ~(uintptr_t)15;
  const uintptr_t e = (reinterpret_cast<uintptr_t>(p) + bytes + 15) & ~(uintptr_t)15;
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"((unsigned)(e - a))
               : "memory");
}

// Step length of the fused CG iteration from sum p.(K:p):
// p.Ap = p.G(K p) = (G p).(K p) = p.(K p) for compatible p (G is an
// orthogonal projector), so alpha is known before the inverse transforms.
template <typename R>
RVE_DEV void zfwd_step_length(const ZfwdParams<R>& P, double pkp, unsigned bid, unsigned nblk) {
  double v1[1] = {pkp}, tot[1];
  if (last_block_sum_of<1>(v1, P.partials, &P.st->counter[SLOT_PAP], tot, bid, nblk) &&
      threadIdx.x == 0) {
    SolverState* st = P.st;
    const double pap = tot[0];
    st->pAp = pap;
    if (st->dev_timeout) {
      st->status = RVE_DEV_ERR_TIMEOUT;
      st->alpha = 0.0;
      st->done = 1;
    } else if (!isfinite(pap)) {
      st->status = RVE_DEV_ERR_NONFINITE;
      st->alpha = 0.0;
      st->done = 1;
    } else if (pap == 0.0) {
      st->status = RVE_DEV_ERR_CG_BREAKDOWN;
      st->alpha = 0.0;
      st->done = 1;
    } else {
      st->alpha = st->rr / pap;
    }
  }
}

template <typename R, typename RC>
struct ZinvParams {
  GridGeom g;
  int lz;
  const cplx<R>* spec;
  R* dst;
  double* dst64;  // OUT_PLAIN output of the float-float passes
  RC* r_out;
  RC* x_out;
  const RC* p_in;
  SolverState* st;
  double* partials;
  const int* done;
  const cplx<R>* tw;
  float mn_ell;  // >= 0: reduce z.(K0:z) with lambda0/mu0 = mn_ell (mu0 = 1), else z.z
};

// z.(K0:z) for the reference medium K0:z = ell tr(z) I + z + z^T (mu0 = 1):
// the squared norm the preconditioned CG monitors (z = M^+ r, r.z = z.(K0:z)
// for compatible z)
template <typename R>
RVE_DEV R mnorm_k0(const R (&z)[9], R ell) {
  const R tr = z[0] + z[4] + z[8];
  const R d2 = z[0] * z[0] + z[4] * z[4] + z[8] * z[8];
  const R o2 = z[1] * z[1] + z[3] * z[3] + z[2] * z[2] + z[6] * z[6] + z[5] * z[5] + z[7] * z[7];
  const R x2 = z[1] * z[3] + z[2] * z[6] + z[5] * z[7];
  return ell * tr * tr + R(2) * d2 + o2 + R(2) * x2;
}

// Four-step float z passes of the fused CG iteration (kernels_fft4.cu),
// used when the z length has a compiled split (g.fsz_n1 != 0).
void launch_zfwd4(const ZfwdParams<float>& P, cudaStream_t s);
void launch_zinv4(const ZinvParams<float, float>& P, cudaStream_t s);

RVE_DEV void cp_async4(void* sdst, const void* gsrc) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gsrc));
}

// Axis plans: the float-float passes use prime radices only (a composite
// float-float butterfly does not fit the register budget).
template <typename R>
RVE_DEV const AxisPlan& axis_plan(const GridGeom& g, int axis) {
  if constexpr (is_dfl<R>::value) return axis == 0 ? g.pxs : (axis == 1 ? g.pys : g.pzs);
  else return axis == 0 ? g.px : (axis == 1 ? g.py : g.pz);
}

// ---------------------------------------------------------------------------
// Bulk asynchronous copies (TMA, cp.async.bulk) into shared memory with
// completion on an mbarrier.  Addresses and sizes are multiples of 16 bytes.
// ---------------------------------------------------------------------------
RVE_DEV unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

RVE_DEV void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

RVE_DEV void mbar_arrive_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

RVE_DEV void bulk_load(void* sdst, const void* gsrc, unsigned bytes, unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(sdst)),
      "l"(gsrc), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

RVE_DEV bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}" : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
  return ok != 0;
}

// Waits for phase `parity` of the barrier, giving up after `limit` polls
// (each poll itself suspends for a bounded time); returns false on giving up.
RVE_DEV bool mbar_wait_bounded(unsigned long long* bar, unsigned parity, unsigned limit) {
  for (unsigned it = 0; it < limit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
