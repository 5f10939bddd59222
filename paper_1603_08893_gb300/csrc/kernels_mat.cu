// Per-voxel kernels: CG vector update, Newton update, reductions and the
// Saint Venant-Kirchhoff constitutive update (Sec. 4.2-4.3).
#include "kernels.h"

#define VEC_THREADS 256
#define VEC_BLOCKS 1216  // 152 SMs x 8 resident blocks; fixed, so reductions are deterministic

size_t vec_max_blocks() { return VEC_BLOCKS; }

// x += alpha p ; r -= alpha Ap ; rr_new = r.r ; then convergence test and
// beta = rr_new / rr (standard CG, Sec. 2.6).  Fields are 9n long.
template <typename R>
__global__ void __launch_bounds__(VEC_THREADS) k_cg_update(size_t n9, R* __restrict__ x,
                                                           R* __restrict__ r, const R* __restrict__ p,
                                                           const R* __restrict__ Ap,
                                                           SolverState* st, double* partials) {
  if (st->done) return;
  const R alpha = (R)st->alpha;
  double acc = 0.0;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n9; i += stride) {
    const R pi = p[i];
    x[i] = fma(alpha, pi, x[i]);
    const R ri = fma(-alpha, Ap[i], r[i]);
    r[i] = ri;
    acc += (double)ri * (double)ri;
  }
  double v[1] = {acc}, tot[1];
  if (last_block_sum<1>(v, partials, &st->counter[SLOT_RR], tot) && threadIdx.x == 0)
    cg_after_rr(st, tot[0]);
}

// Completes a CG solve run with the fused iteration (x is updated one
// iteration late): x += alpha p with the last step length.
template <typename R>
__global__ void __launch_bounds__(VEC_THREADS) k_cg_finish(size_t n9, R* __restrict__ x,
                                                           const R* __restrict__ p,
                                                           const SolverState* st) {
  if (st->it == 0) return;
  const R alpha = (R)st->alpha;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n9; i += stride)
    x[i] = fma(alpha, p[i], x[i]);
}

// Component means of a [9][n] field.  post selects what the last block does
// with them: MEAN_DFBAR: dFbar = Fbar - <F>; MEAN_X: store <dF>; MEAN_PBAR:
// store P-bar; MEAN_PLAIN: write out9.
template <typename T>
__global__ void __launch_bounds__(VEC_THREADS) k_mean9(const T* __restrict__ A, size_t n,
                                                       double* out9, double* partials,
                                                       unsigned int* counter, int post,
                                                       SolverState* st) {
  double s[9];
#pragma unroll
  for (int c = 0; c < 9; ++c) s[c] = 0.0;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
#pragma unroll
    for (int c = 0; c < 9; ++c) s[c] += (double)A[(size_t)c * n + v];
  double tot[9];
  if (last_block_sum<9>(s, partials, counter, tot) && threadIdx.x == 0) {
    for (int c = 0; c < 9; ++c) {
      const double m = tot[c] / (double)n;
      if (post == MEAN_DFBAR) {
        st->meanF[c] = m;
        st->dFbar[c] = st->Fbar[c] - m;
      } else if (post == MEAN_X) {
        st->meanX[c] = m;
      } else if (post == MEAN_PBAR) {
        st->Pbar[c] = m;
      } else {
        out9[c] = m;
      }
    }
  }
}

// ||F + dFbar||^2 -> Fn2 (F itself is not changed; the macroscopic increment
// is added together with the first Newton update)
__global__ void __launch_bounds__(VEC_THREADS) k_shifted_norm(const double* __restrict__ F, size_t n,
                                                              SolverState* st, double* partials) {
  double d[9];
#pragma unroll
  for (int c = 0; c < 9; ++c) d[c] = st->dFbar[c];
  double acc = 0.0;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
#pragma unroll
    for (int c = 0; c < 9; ++c) {
      const double f = F[(size_t)c * n + v] + d[c];
      acc += f * f;
    }
  double a[1] = {acc}, tot[1];
  if (last_block_sum<1>(a, partials, &st->counter[SLOT_NORM], tot) && threadIdx.x == 0)
    st->Fn2 = tot[0];
}

// F += dF - <dF> (+ dFbar on the first iteration of an increment, Algorithm 1:
// F_(1) = F_(0) + dFbar + dF).  The exact mean of dF is zero (Eq. mean:zero);
// the mean of the computed dF is round-off and is removed.
// ||dF - <dF>||^2 -> dF2
template <typename RC>
__global__ void __launch_bounds__(VEC_THREADS) k_newton_update(double* __restrict__ F,
                                                               const RC* __restrict__ x, size_t n,
                                                               SolverState* st, double* partials,
                                                               int add_dfbar) {
  double m[9], u[9];
#pragma unroll
  for (int c = 0; c < 9; ++c) {
    m[c] = st->meanX[c];
    u[c] = add_dfbar ? st->dFbar[c] : 0.0;
  }
  double acc = 0.0;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
#pragma unroll
    for (int c = 0; c < 9; ++c) {
      const double d = (double)x[(size_t)c * n + v] - m[c];
      F[(size_t)c * n + v] += u[c] + d;
      acc += d * d;
    }
  double a[1] = {acc}, tot[1];
  if (last_block_sum<1>(a, partials, &st->counter[SLOT_NORM], tot) && threadIdx.x == 0)
    st->dF2 = tot[0];
}

// Saint Venant-Kirchhoff in FP64: E = (F^T F - I)/2, S = lambda tr(E) I +
// 2 mu E (Eq. elas:S with Eq. elas:C), P = F S (Eq. elas:S-P).  Tangent
// storage: FULL81 writes K_ijkl = S_li d_jk + lambda F_ji F_kl + mu F_jl F_ki
// + mu d_il (F F^T)_jk (Eq. elas:K written out in components) in RO;
// SVK writes F (and, in FP64, S) for on-the-fly recomputation.
template <typename RO>
__global__ void __launch_bounds__(VEC_THREADS) k_svk(const double* __restrict__ F, size_t n,
                                                     MatView<double> mat, double* __restrict__ P,
                                                     int tan_mode, RO* __restrict__ K4,
                                                     RO* __restrict__ Fop, RO* __restrict__ Sop,
                                                     SolverState* st) {
  int flags = 0;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
    double f[9];
#pragma unroll
    for (int c = 0; c < 9; ++c) f[c] = F[(size_t)c * n + v];
    const double lam = mat.get(v, 0), mu = mat.get(v, 1);
    double E[3][3], S[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b)
        E[a][b] = 0.5 * (f[a] * f[b] + f[3 + a] * f[3 + b] + f[6 + a] * f[6 + b] - (a == b ? 1.0 : 0.0));
    const double tr = E[0][0] + E[1][1] + E[2][2];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) S[a][b] = 2.0 * mu * E[a][b] + (a == b ? lam * tr : 0.0);
    double pmax = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const double pv = f[3 * a] * S[0][b] + f[3 * a + 1] * S[1][b] + f[3 * a + 2] * S[2][b];
        P[(size_t)(3 * a + b) * n + v] = pv;
        pmax = fmax(pmax, fabs(pv));
      }
    const double det = f[0] * (f[4] * f[8] - f[5] * f[7]) - f[1] * (f[3] * f[8] - f[5] * f[6]) +
                       f[2] * (f[3] * f[7] - f[4] * f[6]);
    if (!(det > 0.0)) flags |= 1;
    if (!isfinite(pmax) || !isfinite(det)) flags |= 2;
    if (tan_mode == TAN_FULL81) {
      double B[3][3];  // F F^T
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
          B[a][b] = f[3 * a] * f[3 * b] + f[3 * a + 1] * f[3 * b + 1] + f[3 * a + 2] * f[3 * b + 2];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
          for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int l = 0; l < 3; ++l) {
              double kv = lam * f[3 * j + i] * f[3 * k + l] + mu * f[3 * j + l] * f[3 * k + i];
              if (j == k) kv += S[l][i];
              if (i == l) kv += mu * B[j][k];
              K4[(size_t)(((i * 3 + j) * 3 + k) * 3 + l) * n + v] = (RO)kv;
            }
    } else if (tan_mode == TAN_SYM45) {
      double B[3][3];  // F F^T
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
          B[a][b] = f[3 * a] * f[3 * b] + f[3 * a + 1] * f[3 * b + 1] + f[3 * a + 2] * f[3 * b + 2];
      // K_ijkl is M[r][c] with r = 3j + i, c = 3k + l; upper triangle only
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
          for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int l = 0; l < 3; ++l) {
              if (3 * j + i > 3 * k + l) continue;
              double kv = lam * f[3 * j + i] * f[3 * k + l] + mu * f[3 * j + l] * f[3 * k + i];
              if (j == k) kv += S[l][i];
              if (i == l) kv += mu * B[j][k];
              K4[(size_t)sym45_index(3 * j + i, 3 * k + l) * n + v] = (RO)kv;
            }
    } else if (tan_mode == TAN_SVK) {
      if (Fop) {
#pragma unroll
        for (int c = 0; c < 9; ++c) Fop[(size_t)c * n + v] = (RO)f[c];
      }
      if (Sop) {
        Sop[v] = (RO)S[0][0];
        Sop[n + v] = (RO)S[1][1];
        Sop[2 * n + v] = (RO)S[2][2];
        Sop[3 * n + v] = (RO)S[0][1];
        Sop[4 * n + v] = (RO)S[0][2];
        Sop[5 * n + v] = (RO)S[1][2];
      }
    }
  }
  if (flags) atomicOr(&st->err_flags, flags);
}

// The same update for the mixed solver with the tangent recomputed from F
// in the CG (Fop = F in float32, no stored K4 or S) in float-float
// arithmetic, written in the displacement gradient H = F - I (exact in
// float64 for the diagonal, F_aa in [1/2, 2]): E = (H + H^T + H^T H) / 2
// and P = S + H S, so that the cancellation in F^T F - I costs nothing
// and P is accurate to about 2^-46 relative, the accuracy of the
// float-float residual G:P it feeds.  F, H and the parameters are split and
// P assembled from the float64 bits by integer operations (dfloat.cuh), so
// the float64 units, a small fraction of the float32 rate on this
// hardware, only form the three diagonal entries of H and add the two
// parts of each P entry.  det F (the failure test) is taken in float32
// from the high parts of F.
__global__ void __launch_bounds__(VEC_THREADS) k_svk_df(const double* __restrict__ F, size_t n,
                                                        MatView<double> mat,
                                                        double* __restrict__ P,
                                                        float* __restrict__ Fop,
                                                        SolverState* st) {
  int flags = 0;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
    double fd[9];
#pragma unroll
    for (int c = 0; c < 9; ++c) fd[c] = F[(size_t)c * n + v];
    const double lamd = mat.get(v, 0), mud = mat.get(v, 1);
    dfl hm[9];
    float fh[9];
#pragma unroll
    for (int c = 0; c < 9; ++c) {
      fh[c] = dfl_from_bits(fd[c]).hi;
      hm[c] = dfl_from_bits(c % 4 == 0 ? fd[c] - 1.0 : fd[c]);
    }
    const dfl lam = dfl_from_bits(lamd), mu = dfl_from_bits(mud);
    dfl E[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = a; b < 3; ++b) {
        const dfl e = (hm[3 * a + b] + hm[3 * b + a]) +
                      (hm[a] * hm[b] + hm[3 + a] * hm[3 + b] + hm[6 + a] * hm[6 + b]);
        E[a][b] = E[b][a] = dfl(0.5f * e.hi, 0.5f * e.lo);
      }
    const dfl ltr = lam * (E[0][0] + E[1][1] + E[2][2]);
    const dfl mu2(2.0f * mu.hi, 2.0f * mu.lo);
    dfl S[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = a; b < 3; ++b) {
        dfl sv = mu2 * E[a][b];
        if (a == b) sv = sv + ltr;
        S[a][b] = S[b][a] = sv;
      }
    float pmax = 0.0f;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const dfl pv =
            S[a][b] + (hm[3 * a] * S[0][b] + hm[3 * a + 1] * S[1][b] + hm[3 * a + 2] * S[2][b]);
        P[(size_t)(3 * a + b) * n + v] = (double)pv;
        pmax = fmaxf(pmax, fabsf(pv.hi));
      }
    const float det = fh[0] * (fh[4] * fh[8] - fh[5] * fh[7]) -
                      fh[1] * (fh[3] * fh[8] - fh[5] * fh[6]) +
                      fh[2] * (fh[3] * fh[7] - fh[4] * fh[6]);
    if (!(det > 0.0f)) flags |= 1;
    if (!isfinite(pmax) || !isfinite(det)) flags |= 2;
#pragma unroll
    for (int c = 0; c < 9; ++c) Fop[(size_t)c * n + v] = fh[c];
  }
  if (flags) atomicOr(&st->err_flags, flags);
}

// FP64 K4 of a voxel range [v0, v0+count) into dst[81][count].
__global__ void __launch_bounds__(VEC_THREADS) k_svk_k4(const double* __restrict__ F, size_t v0,
                                                        size_t count, size_t n,
                                                        MatView<double> mat, double* dst) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t u = (size_t)blockIdx.x * blockDim.x + threadIdx.x; u < count; u += stride) {
    const size_t v = v0 + u;
    double f[9];
#pragma unroll
    for (int c = 0; c < 9; ++c) f[c] = F[(size_t)c * n + v];
    const double lam = mat.get(v, 0), mu = mat.get(v, 1);
    double S[3][3], B[3][3];
    double E[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        E[a][b] = 0.5 * (f[a] * f[b] + f[3 + a] * f[3 + b] + f[6 + a] * f[6 + b] - (a == b ? 1.0 : 0.0));
        B[a][b] = f[3 * a] * f[3 * b] + f[3 * a + 1] * f[3 * b + 1] + f[3 * a + 2] * f[3 * b + 2];
      }
    const double tr = E[0][0] + E[1][1] + E[2][2];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) S[a][b] = 2.0 * mu * E[a][b] + (a == b ? lam * tr : 0.0);
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j)
        for (int k = 0; k < 3; ++k)
          for (int l = 0; l < 3; ++l) {
            double kv = lam * f[3 * j + i] * f[3 * k + l] + mu * f[3 * j + l] * f[3 * k + i];
            if (j == k) kv += S[l][i];
            if (i == l) kv += mu * B[j][k];
            dst[(size_t)(((i * 3 + j) * 3 + k) * 3 + l) * count + u] = kv;
          }
  }
}

// CG start for A x = b - Ax0: r = b - Ax0 (in the CG precision), x = 0,
// ||r||^2 and the CG state as after a residual evaluation.
template <typename RC>
__global__ void __launch_bounds__(VEC_THREADS) k_cg_init(size_t n9, const double* __restrict__ b,
                                                         const double* __restrict__ Ax,
                                                         RC* __restrict__ r, RC* __restrict__ x,
                                                         SolverState* st, double* partials) {
  double acc = 0.0;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n9; i += stride) {
    const double ri = b[i] - (Ax ? Ax[i] : 0.0);
    r[i] = (RC)ri;
    x[i] = (RC)0;
    acc += ri * ri;
  }
  double a[1] = {acc}, tot[1];
  if (last_block_sum<1>(a, partials, &st->counter[SLOT_BB], tot) && threadIdx.x == 0)
    cg_after_bb(st, tot[0]);
}

// y += (double) x
template <typename RC>
__global__ void __launch_bounds__(VEC_THREADS) k_accumulate(size_t n9, double* __restrict__ y,
                                                            const RC* __restrict__ x) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n9; i += stride)
    y[i] += (double)x[i];
}

// dJ/dmu_k = (1/n) W : (dP/dmu)_k - lambda_k : (dP/dmu)_k with
// dP/dmu = F . (2 dev E) at fixed bulk modulus (S = lambda tr(E) I + 2 mu E,
// lambda = K - 2 mu / 3).
// dJ/dmu (g) and, when gK != null, dJ/dK per voxel from the adjoint field:
// (W/n - lambda) : dP/dq with dP/dmu = F . (2 dev E), dP/dK = F . (tr(E) I).
__global__ void __launch_bounds__(VEC_THREADS) k_adjoint_grad(const double* __restrict__ F,
                                                              const double* __restrict__ lam,
                                                              W9 W, size_t n, double* __restrict__ g,
                                                              double* __restrict__ gK) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  const double inv_n = 1.0 / (double)n;
  for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
    double f[9];
#pragma unroll
    for (int c = 0; c < 9; ++c) f[c] = F[(size_t)c * n + v];
    double E[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b)
        E[a][b] = 0.5 * (f[a] * f[b] + f[3 + a] * f[3 + b] + f[6 + a] * f[6 + b] - (a == b ? 1.0 : 0.0));
    const double tr = E[0][0] + E[1][1] + E[2][2];
    double acc = 0.0, accK = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        double d = 0.0;  // (F . 2 dev E)_ab
#pragma unroll
        for (int c = 0; c < 3; ++c) d += f[3 * a + c] * 2.0 * (E[c][b] - (c == b ? tr / 3.0 : 0.0));
        const double wl = W.w[3 * a + b] * inv_n - lam[(size_t)(3 * a + b) * n + v];
        acc += wl * d;
        accK += wl * f[3 * a + b] * tr;  // (F . tr(E) I)_ab
      }
    g[v] = acc;
    if (gK) gK[v] = accK;
  }
}

template <typename Ti, typename To>
__global__ void k_convert(const Ti* __restrict__ in, To* __restrict__ out, size_t count) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride)
    out[i] = (To)in[i];
}

// --------------------------------------------------------------------------
static unsigned int grid_for(size_t work) {
  size_t b = (work + VEC_THREADS - 1) / VEC_THREADS;
  if (b > VEC_BLOCKS) b = VEC_BLOCKS;
  if (b < 1) b = 1;
  return (unsigned int)b;
}

// Per-voxel parameters [nparam][n] (K, mu, ...) already in device memory to
// the internal form (lambda = K - 2 mu / 3, mu, ...) in float64 and, if
// v32, float32; sums[0..1] = the sums of lambda and mu over the voxels
// (deterministic last-block reduction), for the preconditioner's reference
// medium.
__global__ void __launch_bounds__(VEC_THREADS) k_voxel_params(const double* __restrict__ vp, size_t n,
                                                              int nparam, double* __restrict__ v64,
                                                              float* __restrict__ v32, double* sums,
                                                              double* partials, unsigned int* counter) {
  double a[2] = {0.0, 0.0}, tot[2];
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
    const double K = vp[v], mu = vp[n + v];
    const double lam = K - 2.0 * mu / 3.0;
    v64[v] = lam;
    v64[n + v] = mu;
    if (v32) {
      v32[v] = (float)lam;
      v32[n + v] = (float)mu;
    }
    for (int q = 2; q < nparam; ++q) {
      const double x = vp[(size_t)q * n + v];
      v64[(size_t)q * n + v] = x;
      if (v32) v32[(size_t)q * n + v] = (float)x;
    }
    a[0] += lam;
    a[1] += mu;
  }
  if (last_block_sum<2>(a, partials, counter, tot) && threadIdx.x == 0) {
    sums[0] = tot[0];
    sums[1] = tot[1];
  }
}

void launch_voxel_params(const double* vp, size_t n, int nparam, double* v64, float* v32,
                         double* sums, double* partials, unsigned int* counter, cudaStream_t s) {
  k_voxel_params<<<grid_for(n), VEC_THREADS, 0, s>>>(vp, n, nparam, v64, v32, sums, partials, counter);
}

template <typename R>
void launch_cg_update(size_t n9, R* x, R* r, const R* p, const R* Ap, SolverState* st,
                      double* partials, cudaStream_t s) {
  k_cg_update<R><<<grid_for(n9), VEC_THREADS, 0, s>>>(n9, x, r, p, Ap, st, partials);
}

template <typename R>
void launch_cg_finish(size_t n9, R* x, const R* p, const SolverState* st, cudaStream_t s) {
  k_cg_finish<R><<<grid_for(n9), VEC_THREADS, 0, s>>>(n9, x, p, st);
}

template <typename T>
void launch_mean9(const T* A, size_t n, double* out9, double* partials, unsigned int* counter,
                  int post, SolverState* st, cudaStream_t s) {
  k_mean9<T><<<grid_for(n), VEC_THREADS, 0, s>>>(A, n, out9, partials, counter, post, st);
}

void launch_shifted_norm(const double* F, size_t n, SolverState* st, double* partials,
                         cudaStream_t s) {
  k_shifted_norm<<<grid_for(n), VEC_THREADS, 0, s>>>(F, n, st, partials);
}

template <typename RC>
void launch_newton_update(double* F, const RC* x, size_t n, SolverState* st, double* partials,
                          int add_dfbar, cudaStream_t s) {
  k_newton_update<RC><<<grid_for(n), VEC_THREADS, 0, s>>>(F, x, n, st, partials, add_dfbar);
}

template <typename RO>
void launch_svk_constitutive(const double* F, size_t n, MatView<double> mat, double* P,
                             int tan_mode, RO* K4, RO* Fop, RO* Sop, SolverState* st,
                             cudaStream_t s) {
  k_svk<RO><<<grid_for(n), VEC_THREADS, 0, s>>>(F, n, mat, P, tan_mode, K4, Fop, Sop, st);
}

void launch_svk_constitutive_df(const double* F, size_t n, MatView<double> mat, double* P,
                                float* Fop, SolverState* st, cudaStream_t s) {
  k_svk_df<<<grid_for(n), VEC_THREADS, 0, s>>>(F, n, mat, P, Fop, st);
}

void launch_svk_k4_full(const double* F, size_t v0, size_t count, size_t n,
                        MatView<double> mat, double* dst, cudaStream_t s) {
  k_svk_k4<<<grid_for(count), VEC_THREADS, 0, s>>>(F, v0, count, n, mat, dst);
}

template <typename RC>
void launch_cg_init(size_t n9, const double* b, const double* Ax, RC* r, RC* x, SolverState* st,
                    double* partials, cudaStream_t s) {
  k_cg_init<RC><<<grid_for(n9), VEC_THREADS, 0, s>>>(n9, b, Ax, r, x, st, partials);
}

template <typename RC>
void launch_accumulate(size_t n9, double* y, const RC* x, cudaStream_t s) {
  k_accumulate<RC><<<grid_for(n9), VEC_THREADS, 0, s>>>(n9, y, x);
}

void launch_adjoint_grad(const double* F, const double* lam, const double W[9], size_t n, double* g,
                         double* gK, cudaStream_t s) {
  W9 w;
  for (int c = 0; c < 9; ++c) w.w[c] = W[c];
  k_adjoint_grad<<<grid_for(n), VEC_THREADS, 0, s>>>(F, lam, w, n, g, gK);
}

template <typename Ti, typename To>
void launch_convert(const Ti* in, To* out, size_t count, cudaStream_t s) {
  k_convert<Ti, To><<<grid_for(count), VEC_THREADS, 0, s>>>(in, out, count);
}

template void launch_cg_update<float>(size_t, float*, float*, const float*, const float*,
                                      SolverState*, double*, cudaStream_t);
template void launch_cg_update<double>(size_t, double*, double*, const double*, const double*,
                                       SolverState*, double*, cudaStream_t);
template void launch_mean9<float>(const float*, size_t, double*, double*, unsigned int*, int,
                                  SolverState*, cudaStream_t);
template void launch_mean9<double>(const double*, size_t, double*, double*, unsigned int*, int,
                                   SolverState*, cudaStream_t);
template void launch_newton_update<float>(double*, const float*, size_t, SolverState*, double*,
                                          int, cudaStream_t);
template void launch_newton_update<double>(double*, const double*, size_t, SolverState*, double*,
                                           int, cudaStream_t);
template void launch_svk_constitutive<float>(const double*, size_t, MatView<double>, double*, int,
                                             float*, float*, float*, SolverState*, cudaStream_t);
template void launch_svk_constitutive<double>(const double*, size_t, MatView<double>, double*,
                                              int, double*, double*, double*, SolverState*,
                                              cudaStream_t);
template void launch_convert<double, float>(const double*, float*, size_t, cudaStream_t);
template void launch_convert<float, double>(const float*, double*, size_t, cudaStream_t);
template void launch_convert<double, double>(const double*, double*, size_t, cudaStream_t);
template void launch_cg_init<float>(size_t, const double*, const double*, float*, float*,
                                    SolverState*, double*, cudaStream_t);
template void launch_cg_init<double>(size_t, const double*, const double*, double*, double*,
                                     SolverState*, double*, cudaStream_t);
template void launch_accumulate<float>(size_t, double*, const float*, cudaStream_t);
template void launch_accumulate<double>(size_t, double*, const double*, cudaStream_t);
template void launch_cg_finish<float>(size_t, float*, const float*, const SolverState*, cudaStream_t);
template void launch_cg_finish<double>(size_t, double*, const double*, const SolverState*, cudaStream_t);
