// Finite-strain J2 elasto-plasticity (Sec. 5) per voxel, float64:
// be = F Cp^-1 F^T, eps = ln(be)/2 (principal), Kirchhoff stress
// tau = K tr(eps) I + 2 mu dev(eps) (Eq. elas:C acting on the logarithmic
// strain), von Mises yield phi = tau_eq - (tau_y0 + H eps_p) (Eq. simo:flow),
// plastic branch for phi > -1e-10 tau_y (on the yield surface too, with
// dgamma = max(phi, 0)/(3 mu + H) = 0 there: elasto-plastic tangent),
// radial return in principal logarithmic strains, P = tau F^-T (pull-back),
// trial history Cp^-1 = F^-1 be F^-T, eps_p += dgamma.  The tangent is the
// exact derivative dP/dF of this update (committed history frozen), with the
// derivative of the matrix logarithm from divided differences of ln in the
// eigenbasis of be.  Stored as K_ijkl = dP_ji / dF_kl (Eq. iter:varP).
#include <algorithm>

#include "kernels.h"

#define J2_THREADS 128

// relative margin below the yield stress within which a state counts as on
// the yield surface (round-off of the return map's consistency phi = 0)
constexpr double kYieldSurfaceTol = 1e-10;

namespace {

// Cyclic Jacobi rotations: A (symmetric, in/out, becomes diagonal) and the
// orthogonal V with A_in = V diag(A_out) V^T.  Sweeps stop when the
// off-diagonal part is below 1e-30 of the diagonal (at most 12 sweeps).
RVE_DEV void jacobi3(double (&A)[3][3], double (&V)[3][3]) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) V[i][j] = (i == j) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 12; ++sweep) {
    const double off = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
    const double dia = A[0][0] * A[0][0] + A[1][1] * A[1][1] + A[2][2] * A[2][2];
    if (off <= 1e-30 * dia) break;
#pragma unroll
    for (int pq = 0; pq < 3; ++pq) {
      const int p = (pq == 2) ? 1 : 0;
      const int q = (pq == 0) ? 1 : 2;
      const double apq = A[p][q];
      if (apq == 0.0) continue;
      // rotation angle zeroing A[p][q]: tan(2 phi) = 2 apq / (aqq - app)
      const double theta = (A[q][q] - A[p][p]) / (2.0 * apq);
      const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
      const double c = 1.0 / sqrt(t * t + 1.0);
      const double s = t * c;
      // A <- R^T A R with R the rotation in the (p, q) plane
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const double akp = A[k][p], akq = A[k][q];
        A[k][p] = c * akp - s * akq;
        A[k][q] = s * akp + c * akq;
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const double apk = A[p][k], aqk = A[q][k];
        A[p][k] = c * apk - s * aqk;
        A[q][k] = s * apk + c * aqk;
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const double vkp = V[k][p], vkq = V[k][q];
        V[k][p] = c * vkp - s * vkq;
        V[k][q] = s * vkp + c * vkq;
      }
    }
  }
}

// divided difference of ln: (ln x - ln y)/(x - y) = atanh(t)/(m t),
// t = (x - y)/(x + y), m = (x + y)/2; 1/m at t = 0
RVE_DEV double dd_log(double x, double y) {
  const double m = 0.5 * (x + y);
  const double t = (x - y) / (x + y);
  if (t == 0.0) return 1.0 / m;
  return atanh(t) / (m * t);
}

}  // namespace

// hc: committed history [7][n] (Cp^-1: 00,11,22,01,02,12; eps_p),
// ht: trial history written here.  K4 (RO) and/or K64 (float64, voxel range
// [v0, v0+cnt) into [81][cnt]) are optional.
template <typename RO>
__global__ void __launch_bounds__(J2_THREADS) k_j2(const double* __restrict__ F, size_t n,
                                                   size_t v0, size_t cnt, MatView<double> mat,
                                                   const double* __restrict__ hc,
                                                   double* __restrict__ ht, double* __restrict__ P,
                                                   RO* __restrict__ K4, double* __restrict__ K64,
                                                   SolverState* st, int sym45) {
  int flags = 0;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t u = (size_t)blockIdx.x * blockDim.x + threadIdx.x; u < cnt; u += stride) {
    const size_t v = v0 + u;
    double f[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) f[i][j] = F[(size_t)(3 * i + j) * n + v];
    double C[3][3];
    C[0][0] = hc[v];
    C[1][1] = hc[n + v];
    C[2][2] = hc[2 * n + v];
    C[0][1] = C[1][0] = hc[3 * n + v];
    C[0][2] = C[2][0] = hc[4 * n + v];
    C[1][2] = C[2][1] = hc[5 * n + v];
    const double ep = hc[6 * n + v];
    const double lam_l = mat.get(v, 0), mu = mat.get(v, 1), ty0 = mat.get(v, 2), H = mat.get(v, 3);
    const double Kb = lam_l + 2.0 * mu / 3.0;  // bulk modulus
    // FC = F Cp^-1, be = FC F^T
    double FC[3][3], be[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) FC[i][j] = f[i][0] * C[0][j] + f[i][1] * C[1][j] + f[i][2] * C[2][j];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) be[i][j] = FC[i][0] * f[j][0] + FC[i][1] * f[j][1] + FC[i][2] * f[j][2];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = i + 1; j < 3; ++j) be[i][j] = be[j][i] = 0.5 * (be[i][j] + be[j][i]);
    double Q[3][3];
    jacobi3(be, Q);
    double lam[3], eps[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      lam[a] = be[a][a];
      eps[a] = 0.5 * log(lam[a]);
    }
    const double tr = eps[0] + eps[1] + eps[2];
    double dev[3], s[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      dev[a] = eps[a] - tr / 3.0;
      s[a] = 2.0 * mu * dev[a];
    }
    const double teq = sqrt(1.5 * (s[0] * s[0] + s[1] * s[1] + s[2] * s[2]));
    const double phi = teq - (ty0 + H * ep);
    // plastic branch also on the yield surface (a state that yielded in the
    // last increment): dgamma = 0 there, elasto-plastic tangent
    const bool plastic = phi > -kYieldSurfaceTol * (ty0 + H * ep);
    const double dg = plastic ? fmax(phi, 0.0) / (3.0 * mu + H) : 0.0;
    const double beta = plastic ? 1.0 - 3.0 * mu * dg / teq : 1.0;
    double taup[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) taup[a] = Kb * tr + beta * s[a];
    // tau = Q diag(taup) Q^T
    double tau[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j)
        tau[i][j] = Q[i][0] * taup[0] * Q[j][0] + Q[i][1] * taup[1] * Q[j][1] + Q[i][2] * taup[2] * Q[j][2];
    // F^-1 by the adjugate
    const double det = f[0][0] * (f[1][1] * f[2][2] - f[1][2] * f[2][1]) -
                       f[0][1] * (f[1][0] * f[2][2] - f[1][2] * f[2][0]) +
                       f[0][2] * (f[1][0] * f[2][1] - f[1][1] * f[2][0]);
    if (!(det > 0.0)) flags |= 1;
    const double id = 1.0 / det;
    double Fi[3][3];  // F^-1
    Fi[0][0] = (f[1][1] * f[2][2] - f[1][2] * f[2][1]) * id;
    Fi[0][1] = (f[0][2] * f[2][1] - f[0][1] * f[2][2]) * id;
    Fi[0][2] = (f[0][1] * f[1][2] - f[0][2] * f[1][1]) * id;
    Fi[1][0] = (f[1][2] * f[2][0] - f[1][0] * f[2][2]) * id;
    Fi[1][1] = (f[0][0] * f[2][2] - f[0][2] * f[2][0]) * id;
    Fi[1][2] = (f[0][2] * f[1][0] - f[0][0] * f[1][2]) * id;
    Fi[2][0] = (f[1][0] * f[2][1] - f[1][1] * f[2][0]) * id;
    Fi[2][1] = (f[0][1] * f[2][0] - f[0][0] * f[2][1]) * id;
    Fi[2][2] = (f[0][0] * f[1][1] - f[0][1] * f[1][0]) * id;
    // P = tau F^-T : P_ij = tau_ik Fi_jk
    double Pm[3][3];
    double pmax = 0.0;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        Pm[i][j] = tau[i][0] * Fi[j][0] + tau[i][1] * Fi[j][1] + tau[i][2] * Fi[j][2];
        pmax = fmax(pmax, fabs(Pm[i][j]));
      }
    if (!isfinite(pmax) || !isfinite(det)) flags |= 2;
    if (P) {
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) P[(size_t)(3 * i + j) * n + v] = Pm[i][j];
    }
    if (ht) {
      // trial history: be_new = Q diag(exp(2 eps_e)) Q^T, Cp^-1 = F^-1 be_new F^-T
      double bn[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) bn[a] = exp(2.0 * (tr / 3.0 + beta * dev[a]));
      double G[3][3];  // F^-1 Q
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int a = 0; a < 3; ++a) G[i][a] = Fi[i][0] * Q[0][a] + Fi[i][1] * Q[1][a] + Fi[i][2] * Q[2][a];
      double Cn[3][3];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) Cn[i][j] = G[i][0] * bn[0] * G[j][0] + G[i][1] * bn[1] * G[j][1] + G[i][2] * bn[2] * G[j][2];
      ht[v] = Cn[0][0];
      ht[n + v] = Cn[1][1];
      ht[2 * n + v] = Cn[2][2];
      ht[3 * n + v] = 0.5 * (Cn[0][1] + Cn[1][0]);
      ht[4 * n + v] = 0.5 * (Cn[0][2] + Cn[2][0]);
      ht[5 * n + v] = 0.5 * (Cn[1][2] + Cn[2][1]);
      ht[6 * n + v] = ep + dg;
    }
    if (!K4 && !K64) continue;
    // ---- consistent tangent, one unit direction dF = e_k (x) e_l at a time
    double f1[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) f1[a][b] = dd_log(lam[a], lam[b]);
    // Qt_FC[a][l] = (Q^T FC)_al
    double QFC[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int l = 0; l < 3; ++l) QFC[a][l] = Q[0][a] * FC[0][l] + Q[1][a] * FC[1][l] + Q[2][a] * FC[2][l];
    const double c1 = plastic ? 1.0 / (3.0 * mu + H) - dg / teq : 0.0;
    for (int k = 0; k < 3; ++k)
      for (int l = 0; l < 3; ++l) {
        // d(be) = e_k (x) v + v (x) e_k, v = FC[:, l]; in the eigenbasis
        // (Q^T d(be) Q)_ab = Q_ka QFC_bl + QFC_al Q_kb
        double dq[3][3];
        double dtr = 0.0;
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
          for (int b = 0; b < 3; ++b) {
            dq[a][b] = 0.5 * f1[a][b] * (Q[k][a] * QFC[b][l] + QFC[a][l] * Q[k][b]);  // d(eps)
          }
        dtr = dq[0][0] + dq[1][1] + dq[2][2];
        double dteq = 0.0, dbeta = 0.0;
        if (plastic) {
          // s_tr : ds_tr = 2 mu sum_a s_a d(eps)_aa (s_tr is diagonal, traceless)
          dteq = 1.5 * 2.0 * mu * (s[0] * dq[0][0] + s[1] * dq[1][1] + s[2] * dq[2][2]) / teq;
          dbeta = -3.0 * mu * dteq * c1 / teq;
        }
        // d(tau) in the eigenbasis
        double dt[3][3];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
          for (int b = 0; b < 3; ++b) {
            double x = beta * 2.0 * mu * (dq[a][b] - (a == b ? dtr / 3.0 : 0.0));
            if (a == b) x += Kb * dtr + dbeta * s[a];
            dt[a][b] = x;
          }
        // d(tau) global = Q dt Q^T
        double dT[3][3], QdT[3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int b = 0; b < 3; ++b) QdT[i][b] = Q[i][0] * dt[0][b] + Q[i][1] * dt[1][b] + Q[i][2] * dt[2][b];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int j = 0; j < 3; ++j) dT[i][j] = QdT[i][0] * Q[j][0] + QdT[i][1] * Q[j][1] + QdT[i][2] * Q[j][2];
        // dP = d(tau) F^-T - P[:, l] (x) F^-T[k, :]  (F^-T[k][j] = Fi[j][k])
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int j = 0; j < 3; ++j) {
            const double dP = dT[i][0] * Fi[j][0] + dT[i][1] * Fi[j][1] + dT[i][2] * Fi[j][2] - Pm[i][l] * Fi[j][k];
            // K_jikl = dP_ij, i.e. M[3i + j][3k + l]
            const size_t comp = (size_t)((j * 3 + i) * 3 + k) * 3 + l;
            if (K4) {
              if (!sym45) K4[comp * n + v] = (RO)dP;
              else if (3 * i + j <= 3 * k + l) K4[(size_t)sym45_index(3 * i + j, 3 * k + l) * n + v] = (RO)dP;
            }
            if (K64) K64[comp * cnt + u] = dP;
          }
      }
  }
  if (flags && st) atomicOr(&st->err_flags, flags);
}

// Adjoint gradient of J = W : P-bar with respect to the per-voxel
// parameters (K, mu, tau_y0, H) at fixed F and fixed history hs (the one at
// the start of the increment): out[k][v] = (1/n) W : dP/dp_k - lambda : dP/dp_k.
// At fixed F and history the eigenbasis of be is fixed; with e the
// principal deviatoric log strain, q = sqrt(3/2 e.e), tau_y = tau_y0 + H eps_p
// and dgamma = (2 mu q - tau_y) / (3 mu + H) on the plastic branch,
// s = 2 mu e - 3 mu dgamma e / q and
//   d tau_p/dK = tr(eps),  d s/dmu = 2 e - 3 (dgamma + mu (2 q H + 3 tau_y)/(3 mu + H)^2) e/q,
//   d s/dtau_y0 = 3 mu/(3 mu + H) e/q,  d s/dH = 3 mu (eps_p + dgamma)/(3 mu + H) e/q
// (elastic: 2 e for mu, 0 for tau_y0 and H); dP = d tau F^-T.
__global__ void __launch_bounds__(J2_THREADS) k_j2_adjoint_grad(
    const double* __restrict__ F, size_t n, MatView<double> mat, const double* __restrict__ hs,
    const double* __restrict__ lam, W9 w, double* __restrict__ out) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  const double inv_n = 1.0 / (double)n;
  for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
    double f[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) f[i][j] = F[(size_t)(3 * i + j) * n + v];
    double C[3][3];
    C[0][0] = hs[v];
    C[1][1] = hs[n + v];
    C[2][2] = hs[2 * n + v];
    C[0][1] = C[1][0] = hs[3 * n + v];
    C[0][2] = C[2][0] = hs[4 * n + v];
    C[1][2] = C[2][1] = hs[5 * n + v];
    const double ep = hs[6 * n + v];
    const double mu = mat.get(v, 1), ty0 = mat.get(v, 2), H = mat.get(v, 3);
    double FC[3][3], be[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) FC[i][j] = f[i][0] * C[0][j] + f[i][1] * C[1][j] + f[i][2] * C[2][j];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) be[i][j] = FC[i][0] * f[j][0] + FC[i][1] * f[j][1] + FC[i][2] * f[j][2];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = i + 1; j < 3; ++j) be[i][j] = be[j][i] = 0.5 * (be[i][j] + be[j][i]);
    double Q[3][3];
    jacobi3(be, Q);
    double eps[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) eps[a] = 0.5 * log(be[a][a]);
    const double tr = eps[0] + eps[1] + eps[2];
    double e[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) e[a] = eps[a] - tr / 3.0;
    const double q = sqrt(1.5 * (e[0] * e[0] + e[1] * e[1] + e[2] * e[2]));
    const double teq = 2.0 * mu * q;
    const double ty = ty0 + H * ep;
    const double phi = teq - ty;
    const bool plastic = phi > -kYieldSurfaceTol * ty;
    const double den = 3.0 * mu + H;
    const double dg = plastic ? fmax(phi, 0.0) / den : 0.0;
    // principal derivatives of tau for (K, mu, tau_y0, H)
    double d[4][3];
    const double iq = plastic ? 1.0 / q : 0.0;
    const double cmu = plastic ? 3.0 * (dg + mu * (2.0 * q * H + 3.0 * ty) / (den * den)) : 0.0;
    const double cty = plastic ? 3.0 * mu / den : 0.0;
    const double cH = plastic ? 3.0 * mu * (ep + dg) / den : 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      d[0][a] = tr;
      d[1][a] = 2.0 * e[a] - cmu * e[a] * iq;
      d[2][a] = cty * e[a] * iq;
      d[3][a] = cH * e[a] * iq;
    }
    const double det = f[0][0] * (f[1][1] * f[2][2] - f[1][2] * f[2][1]) -
                       f[0][1] * (f[1][0] * f[2][2] - f[1][2] * f[2][0]) +
                       f[0][2] * (f[1][0] * f[2][1] - f[1][1] * f[2][0]);
    const double id = 1.0 / det;
    double Fi[3][3];
    Fi[0][0] = (f[1][1] * f[2][2] - f[1][2] * f[2][1]) * id;
    Fi[0][1] = (f[0][2] * f[2][1] - f[0][1] * f[2][2]) * id;
    Fi[0][2] = (f[0][1] * f[1][2] - f[0][2] * f[1][1]) * id;
    Fi[1][0] = (f[1][2] * f[2][0] - f[1][0] * f[2][2]) * id;
    Fi[1][1] = (f[0][0] * f[2][2] - f[0][2] * f[2][0]) * id;
    Fi[1][2] = (f[0][2] * f[1][0] - f[0][0] * f[1][2]) * id;
    Fi[2][0] = (f[1][0] * f[2][1] - f[1][1] * f[2][0]) * id;
    Fi[2][1] = (f[0][1] * f[2][0] - f[0][0] * f[2][1]) * id;
    Fi[2][2] = (f[0][0] * f[1][1] - f[0][1] * f[1][0]) * id;
    // c_ab = (1/n) W_ab - lambda_ab; g_k = sum_ab c_ab (d tau_k F^-T)_ab
    double c[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) c[i][j] = inv_n * w.w[3 * i + j] - lam[(size_t)(3 * i + j) * n + v];
    // sum_ab c_ab tau_ac Fi_bc = sum_ac tau_ac (c Fi)_ac with (c Fi)_ac = sum_b c_ab Fi_bc
    double cF[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int k = 0; k < 3; ++k) cF[i][k] = c[i][0] * Fi[0][k] + c[i][1] * Fi[1][k] + c[i][2] * Fi[2][k];
    // tau = Q diag(t) Q^T: sum_ac Q_a p t_p Q_c p cF_ac = sum_p t_p (Q^T cF Q)_pp
    double m[3];
#pragma unroll
    for (int p = 0; p < 3; ++p) {
      double acc = 0.0;
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k) acc += Q[i][p] * cF[i][k] * Q[k][p];
      m[p] = acc;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) out[(size_t)k * n + v] = d[k][0] * m[0] + d[k][1] * m[1] + d[k][2] * m[2];
  }
}

// ---------------------------------------------------------------------------
// Adjoint through the history of a path of increments (reverse sweep): the
// return map's derivatives with respect to the history h = (Cp^-1_00, _11,
// _22, _01, _02, _12, eps_p), to F and to the parameters (K, mu, tau_y0, H),
// in closed form: every step of the return map linearised (the matrix
// logarithm and exponential by Daleckii-Krein divided differences in the
// eigenbasis of be, the radial return, the pull-backs with
// d(F^-1) = -F^-1 dF F^-1), one directional derivative per unit direction.
// ---------------------------------------------------------------------------

// The return map of one voxel and the pieces its linearisation needs.
struct J2State {
  double f[3][3], C[3][3], ep;  // F, committed Cp^-1 and eps_p
  double K, mu, ty0, H;         // bulk and shear moduli, yield stress, hardening
  double Q[3][3];               // eigenvectors of be (columns)
  double f1[3][3];              // divided differences of ln at the eigenvalues of be
  double tr, dev[3];            // trace and principal deviator of the trial log strain
  double teq, dg, beta;
  bool plastic;
  double Fi[3][3];              // F^-1
  double tau[3][3];             // Kirchhoff stress
  double g1[3][3];              // divided differences of exp(2 x), x the elastic log strain
  double bn[3][3];              // new elastic be = exp(2 eps_e)
};

// sinh(x)/x, 1 + x^2/6 near 0
RVE_DEV double sinhc(double x) { return fabs(x) < 1e-8 ? 1.0 + x * x / 6.0 : sinh(x) / x; }

RVE_DEV void j2_state(const double (&Fv)[9], const double (&hs)[7], double Kb, double mu,
                      double ty0, double H, J2State& S) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) S.f[i][j] = Fv[3 * i + j];
  S.C[0][0] = hs[0];
  S.C[1][1] = hs[1];
  S.C[2][2] = hs[2];
  S.C[0][1] = S.C[1][0] = hs[3];
  S.C[0][2] = S.C[2][0] = hs[4];
  S.C[1][2] = S.C[2][1] = hs[5];
  S.ep = hs[6];
  S.K = Kb;
  S.mu = mu;
  S.ty0 = ty0;
  S.H = H;
  double FC[3][3], be[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      FC[i][j] = S.f[i][0] * S.C[0][j] + S.f[i][1] * S.C[1][j] + S.f[i][2] * S.C[2][j];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      be[i][j] = FC[i][0] * S.f[j][0] + FC[i][1] * S.f[j][1] + FC[i][2] * S.f[j][2];
  for (int i = 0; i < 3; ++i)
    for (int j = i + 1; j < 3; ++j) be[i][j] = be[j][i] = 0.5 * (be[i][j] + be[j][i]);
  jacobi3(be, S.Q);
  double lam[3], eps[3];
  for (int a = 0; a < 3; ++a) {
    lam[a] = be[a][a];
    eps[a] = 0.5 * log(lam[a]);
  }
  for (int a = 0; a < 3; ++a)
    for (int c = 0; c < 3; ++c) S.f1[a][c] = dd_log(lam[a], lam[c]);
  S.tr = eps[0] + eps[1] + eps[2];
  double sp[3];
  for (int a = 0; a < 3; ++a) {
    S.dev[a] = eps[a] - S.tr / 3.0;
    sp[a] = 2.0 * mu * S.dev[a];
  }
  S.teq = sqrt(1.5 * (sp[0] * sp[0] + sp[1] * sp[1] + sp[2] * sp[2]));
  const double phi = S.teq - (ty0 + H * S.ep);
  S.plastic = phi > -kYieldSurfaceTol * (ty0 + H * S.ep);
  S.dg = S.plastic ? fmax(phi, 0.0) / (3.0 * mu + H) : 0.0;
  S.beta = S.plastic ? 1.0 - 3.0 * mu * S.dg / (S.teq > 0.0 ? S.teq : 1.0) : 1.0;
  const double (&f)[3][3] = S.f;
  const double det = f[0][0] * (f[1][1] * f[2][2] - f[1][2] * f[2][1]) -
                     f[0][1] * (f[1][0] * f[2][2] - f[1][2] * f[2][0]) +
                     f[0][2] * (f[1][0] * f[2][1] - f[1][1] * f[2][0]);
  const double id = 1.0 / det;
  S.Fi[0][0] = (f[1][1] * f[2][2] - f[1][2] * f[2][1]) * id;
  S.Fi[0][1] = (f[0][2] * f[2][1] - f[0][1] * f[2][2]) * id;
  S.Fi[0][2] = (f[0][1] * f[1][2] - f[0][2] * f[1][1]) * id;
  S.Fi[1][0] = (f[1][2] * f[2][0] - f[1][0] * f[2][2]) * id;
  S.Fi[1][1] = (f[0][0] * f[2][2] - f[0][2] * f[2][0]) * id;
  S.Fi[1][2] = (f[0][2] * f[1][0] - f[0][0] * f[1][2]) * id;
  S.Fi[2][0] = (f[1][0] * f[2][1] - f[1][1] * f[2][0]) * id;
  S.Fi[2][1] = (f[0][1] * f[2][0] - f[0][0] * f[2][1]) * id;
  S.Fi[2][2] = (f[0][0] * f[1][1] - f[0][1] * f[1][0]) * id;
  double taup[3], x[3], e2[3];
  for (int a = 0; a < 3; ++a) {
    taup[a] = Kb * S.tr + S.beta * sp[a];
    x[a] = S.tr / 3.0 + S.beta * S.dev[a];
    e2[a] = exp(2.0 * x[a]);
  }
  for (int a = 0; a < 3; ++a)
    for (int c = 0; c < 3; ++c) S.g1[a][c] = 2.0 * exp(x[a] + x[c]) * sinhc(x[a] - x[c]);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double t = 0.0, b = 0.0;
      for (int a = 0; a < 3; ++a) {
        t += S.Q[i][a] * taup[a] * S.Q[j][a];
        b += S.Q[i][a] * e2[a] * S.Q[j][a];
      }
      S.tau[i][j] = t;
      S.bn[i][j] = b;
    }
}

// M <- Q (W o (Q^T A Q)) Q^T: a function's derivative in the eigenbasis Q
// with divided differences W
RVE_DEV void eig_apply(const double (&Q)[3][3], const double (&W)[3][3], const double (&A)[3][3],
                       double (&M)[3][3]) {
  double T[3][3], U[3][3];
  for (int a = 0; a < 3; ++a)
    for (int j = 0; j < 3; ++j) T[a][j] = Q[0][a] * A[0][j] + Q[1][a] * A[1][j] + Q[2][a] * A[2][j];
  for (int a = 0; a < 3; ++a)
    for (int c = 0; c < 3; ++c)
      U[a][c] = W[a][c] * (T[a][0] * Q[0][c] + T[a][1] * Q[1][c] + T[a][2] * Q[2][c]);
  for (int i = 0; i < 3; ++i)
    for (int c = 0; c < 3; ++c) T[i][c] = Q[i][0] * U[0][c] + Q[i][1] * U[1][c] + Q[i][2] * U[2][c];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) M[i][j] = T[i][0] * Q[j][0] + T[i][1] * Q[j][1] + T[i][2] * Q[j][2];
}

RVE_DEV void mm3(const double (&A)[3][3], const double (&B)[3][3], double (&C)[3][3]) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) C[i][j] = A[i][0] * B[0][j] + A[i][1] * B[1][j] + A[i][2] * B[2][j];
}

// A B^T
RVE_DEV void mmt3(const double (&A)[3][3], const double (&B)[3][3], double (&C)[3][3]) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) C[i][j] = A[i][0] * B[j][0] + A[i][1] * B[j][1] + A[i][2] * B[j][2];
}

// Directional derivative of the return map at S in the direction (dF, dC
// (symmetric), dep, dp = (dK, dmu, dtau_y0, dH)): dP (row-major 9) and the
// new history's dh (7).
RVE_DEV void j2_dir(const J2State& S, const double (&dF)[3][3], const double (&dC)[3][3],
                    double dep, const double (&dp)[4], double (&dP)[9], double (&dh)[7]) {
  const double dK = dp[0], dmu = dp[1], dty = dp[2], dH = dp[3];
  const double I[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  // d(be) = dF C F^T + F C dF^T + F dC F^T
  double A[3][3], B[3][3], dbe[3][3];
  mm3(dF, S.C, A);
  mmt3(A, S.f, dbe);
  mm3(S.f, dC, B);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      const double fcdf = (S.f[i][0] * S.C[0][0] + S.f[i][1] * S.C[1][0] + S.f[i][2] * S.C[2][0]) * dF[j][0] +
                          (S.f[i][0] * S.C[0][1] + S.f[i][1] * S.C[1][1] + S.f[i][2] * S.C[2][1]) * dF[j][1] +
                          (S.f[i][0] * S.C[0][2] + S.f[i][1] * S.C[1][2] + S.f[i][2] * S.C[2][2]) * dF[j][2];
      const double fdcf = B[i][0] * S.f[j][0] + B[i][1] * S.f[j][1] + B[i][2] * S.f[j][2];
      dbe[i][j] += fcdf + fdcf;
    }
  // trial log strain: d(eps) = (1/2) Dln(be)[d(be)]
  double hf1[3][3], deps[3][3];
  for (int a = 0; a < 3; ++a)
    for (int c = 0; c < 3; ++c) hf1[a][c] = 0.5 * S.f1[a][c];
  eig_apply(S.Q, hf1, dbe, deps);
  const double dtr = deps[0][0] + deps[1][1] + deps[2][2];
  double Ed[3][3], dEd[3][3], s_tr[3][3], ds_tr[3][3];
  double ssum = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      Ed[i][j] = S.Q[i][0] * S.dev[0] * S.Q[j][0] + S.Q[i][1] * S.dev[1] * S.Q[j][1] +
                 S.Q[i][2] * S.dev[2] * S.Q[j][2];
      dEd[i][j] = deps[i][j] - dtr * I[i][j] / 3.0;
      s_tr[i][j] = 2.0 * S.mu * Ed[i][j];
      ds_tr[i][j] = 2.0 * S.mu * dEd[i][j] + 2.0 * dmu * Ed[i][j];
      ssum += s_tr[i][j] * ds_tr[i][j];
    }
  // radial return
  const double den = 3.0 * S.mu + S.H;
  const double tsafe = S.teq > 0.0 ? S.teq : 1.0;
  const double dteq = S.plastic ? 1.5 * ssum / tsafe : 0.0;
  const double dphi = dteq - dty - dH * S.ep - S.H * dep;
  const double ddg = S.plastic ? (dphi - S.dg * (3.0 * dmu + dH)) / den : 0.0;
  const double dbeta = S.plastic ? -3.0 * (dmu * S.dg + S.mu * ddg) / tsafe +
                                       3.0 * S.mu * S.dg * dteq / (tsafe * tsafe)
                                 : 0.0;
  // stress and its pull-back: dP = d(tau) F^-T + tau d(F^-1)^T
  double dtau[3][3], dFi[3][3], deps_e[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      dtau[i][j] = (dK * S.tr + S.K * dtr) * I[i][j] + dbeta * s_tr[i][j] + S.beta * ds_tr[i][j];
      deps_e[i][j] = dtr * I[i][j] / 3.0 + dbeta * Ed[i][j] + S.beta * dEd[i][j];
    }
  mm3(S.Fi, dF, A);
  mm3(A, S.Fi, dFi);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) dFi[i][j] = -dFi[i][j];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      dP[3 * i + j] = dtau[i][0] * S.Fi[j][0] + dtau[i][1] * S.Fi[j][1] + dtau[i][2] * S.Fi[j][2] +
                      S.tau[i][0] * dFi[j][0] + S.tau[i][1] * dFi[j][1] + S.tau[i][2] * dFi[j][2];
  // new history: d(be_new) = Dexp2(eps_e)[d(eps_e)], Cp^-1 = F^-1 be_new F^-T
  double dbn[3][3], T1[3][3], dCn[3][3];
  eig_apply(S.Q, S.g1, deps_e, dbn);
  mm3(dFi, S.bn, A);
  mmt3(A, S.Fi, dCn);       // dF^-1 be F^-T
  mm3(S.Fi, dbn, A);
  mmt3(A, S.Fi, T1);        // F^-1 dbe F^-T
  mm3(S.Fi, S.bn, A);
  mmt3(A, dFi, B);          // F^-1 be dF^-T
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) dCn[i][j] += T1[i][j] + B[i][j];
  dh[0] = dCn[0][0];
  dh[1] = dCn[1][1];
  dh[2] = dCn[2][2];
  dh[3] = 0.5 * (dCn[0][1] + dCn[1][0]);
  dh[4] = 0.5 * (dCn[0][2] + dCn[2][0]);
  dh[5] = 0.5 * (dCn[1][2] + dCn[2][1]);
  dh[6] = dep + ddg;
}

// unit direction k of the history h = (C00, C11, C22, C01, C02, C12, eps_p)
RVE_DEV void hist_unit(int k, double (&dC)[3][3], double& dep) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) dC[i][j] = 0.0;
  dep = 0.0;
  switch (k) {
    case 0: dC[0][0] = 1.0; break;
    case 1: dC[1][1] = 1.0; break;
    case 2: dC[2][2] = 1.0; break;
    case 3: dC[0][1] = dC[1][0] = 1.0; break;
    case 4: dC[0][2] = dC[2][0] = 1.0; break;
    case 5: dC[1][2] = dC[2][1] = 1.0; break;
    default: dep = 1.0; break;
  }
}

// gF[c][v] = sum_k a_k dH_k/dF_c (the functional's sensitivity to F_m
// through the history h_m)
__global__ void __launch_bounds__(J2_THREADS) k_j2_path_gF(const double* __restrict__ F, size_t n,
                                                         MatView<double> mat,
                                                         const double* __restrict__ hs,
                                                         const double* __restrict__ a,
                                                         double* __restrict__ gF) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
    double Fv[9], h[7], av[7];
    for (int c = 0; c < 9; ++c) Fv[c] = F[(size_t)c * n + v];
    for (int k = 0; k < 7; ++k) {
      h[k] = hs[(size_t)k * n + v];
      av[k] = a[(size_t)k * n + v];
    }
    const double mu = mat.get(v, 1), ty0 = mat.get(v, 2), H = mat.get(v, 3);
    const double Kb = mat.get(v, 0) + 2.0 * mu / 3.0;
    J2State S;
    j2_state(Fv, h, Kb, mu, ty0, H, S);
    const double zC[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    const double zp[4] = {0, 0, 0, 0};
    double dF[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, dP[9], dh[7];
    for (int c = 0; c < 9; ++c) {
      dF[c / 3][c % 3] = 1.0;
      j2_dir(S, dF, zC, 0.0, zp, dP, dh);
      dF[c / 3][c % 3] = 0.0;
      double s = 0.0;
      for (int k = 0; k < 7; ++k) s += av[k] * dh[k];
      gF[(size_t)c * n + v] = s;
    }
  }
}

// One backward step at (F_m, h_{m-1}): with c = (1/n) W [last] - lambda,
//   g[p][v]     += c : dP/dp + a . dH/dp          (p = K, mu, tau_y0, H),
//   a_out[k][v]  = c : dP/dh_k + a . dH/dh_k.
__global__ void __launch_bounds__(J2_THREADS) k_j2_path_step(
    const double* __restrict__ F, size_t n, MatView<double> mat, const double* __restrict__ hs,
    const double* __restrict__ lam, W9 w, int last, const double* __restrict__ a_in,
    double* __restrict__ a_out, double* __restrict__ g) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  const double inv_n = 1.0 / (double)n;
  for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
    double Fv[9], h[7], av[7], c[9];
    for (int q = 0; q < 9; ++q) {
      Fv[q] = F[(size_t)q * n + v];
      c[q] = (last ? inv_n * w.w[q] : 0.0) - lam[(size_t)q * n + v];
    }
    for (int k = 0; k < 7; ++k) {
      h[k] = hs[(size_t)k * n + v];
      av[k] = a_in ? a_in[(size_t)k * n + v] : 0.0;
    }
    const double mu = mat.get(v, 1);
    J2State S;
    j2_state(Fv, h, mat.get(v, 0) + 2.0 * mu / 3.0, mu, mat.get(v, 2), mat.get(v, 3), S);
    const double zF[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    double dC[3][3], dep, dP[9], dh[7];
    double dp[4] = {0, 0, 0, 0};
    for (int k = 0; k < 7; ++k) {
      hist_unit(k, dC, dep);
      j2_dir(S, zF, dC, dep, dp, dP, dh);
      double s = 0.0;
      for (int q = 0; q < 9; ++q) s += c[q] * dP[q];
      for (int j = 0; j < 7; ++j) s += av[j] * dh[j];
      a_out[(size_t)k * n + v] = s;
    }
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) dC[i][j] = 0.0;
    for (int t = 0; t < 4; ++t) {
      dp[t] = 1.0;
      j2_dir(S, zF, dC, 0.0, dp, dP, dh);
      dp[t] = 0.0;
      double s = 0.0;
      for (int q = 0; q < 9; ++q) s += c[q] * dP[q];
      for (int j = 0; j < 7; ++j) s += av[j] * dh[j];
      g[(size_t)t * n + v] += s;
    }
  }
}

template <typename RO>
void launch_j2_constitutive(const double* F, size_t n, MatView<double> mat, const double* hc,
                            double* ht, double* P, RO* K4, SolverState* st, cudaStream_t s,
                            int sym45) {
  size_t b = (n + J2_THREADS - 1) / J2_THREADS;
  if (b > 4864) b = 4864;
  if (b < 1) b = 1;
  k_j2<RO><<<(unsigned)b, J2_THREADS, 0, s>>>(F, n, 0, n, mat, hc, ht, P, K4, nullptr, st, sym45);
}

void launch_j2_k4_full(const double* F, size_t v0, size_t count, size_t n, MatView<double> mat,
                       const double* hc, double* dst, cudaStream_t s) {
  size_t b = (count + J2_THREADS - 1) / J2_THREADS;
  if (b > 4864) b = 4864;
  if (b < 1) b = 1;
  k_j2<double><<<(unsigned)b, J2_THREADS, 0, s>>>(F, n, v0, count, mat, hc, nullptr, nullptr,
                                                   nullptr, dst, nullptr, 0);
}

void launch_j2_adjoint_grad(const double* F, size_t n, MatView<double> mat, const double* hs,
                           const double* lam, const double W[9], double* out, cudaStream_t s) {
  W9 w;
  for (int c = 0; c < 9; ++c) w.w[c] = W[c];
  const size_t b = std::min<size_t>((n + J2_THREADS - 1) / J2_THREADS, 65535);
  k_j2_adjoint_grad<<<(unsigned)std::max<size_t>(b, 1), J2_THREADS, 0, s>>>(F, n, mat, hs, lam, w, out);
}

void launch_j2_path_gF(const double* F, size_t n, MatView<double> mat, const double* hs,
                       const double* a, double* gF, cudaStream_t s) {
  const size_t b = std::min<size_t>((n + J2_THREADS - 1) / J2_THREADS, 65535);
  k_j2_path_gF<<<(unsigned)std::max<size_t>(b, 1), J2_THREADS, 0, s>>>(F, n, mat, hs, a, gF);
}

void launch_j2_path_step(const double* F, size_t n, MatView<double> mat, const double* hs,
                         const double* lam, const double W[9], int last, const double* a_in,
                         double* a_out, double* g, cudaStream_t s) {
  W9 w;
  for (int c = 0; c < 9; ++c) w.w[c] = W[c];
  const size_t b = std::min<size_t>((n + J2_THREADS - 1) / J2_THREADS, 65535);
  k_j2_path_step<<<(unsigned)std::max<size_t>(b, 1), J2_THREADS, 0, s>>>(F, n, mat, hs, lam, w,
                                                                          last, a_in, a_out, g);
}

template void launch_j2_constitutive<float>(const double*, size_t, MatView<double>, const double*,
                                            double*, double*, float*, SolverState*, cudaStream_t,
                                            int);
template void launch_j2_constitutive<double>(const double*, size_t, MatView<double>,
                                             const double*, double*, double*, double*,
                                             SolverState*, cudaStream_t, int);
