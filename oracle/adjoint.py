"""Gradient of a homogenised-stress functional with respect to per-voxel
material parameters by one adjoint solve: shear and bulk moduli for Saint
Venant-Kirchhoff (Sec. 4), and K, mu, tau_y0, H for J2 (Sec. 5) with the
history at the start of the increment held fixed (below).

Not in the paper; derived from its equilibrium equations.  With
F = Fbar + w (w compatible, zero mean) the converged state satisfies
R(w, mu) = G : P(Fbar + w, mu) = 0 (Eq. weak:discr:FFT).  For
J = W : P-bar = (1/n) sum_v W_ab P_ab(F_v, mu_v):

  dJ/dmu_k = (1/n) W : (dP/dmu)_k + <dJ/dF, dw/dmu_k>,
  dw/dmu_k = -A^-1 G : (dP/dmu_k e_k),   A = G K G on compatible fields.

K (the matrix of Eq. iter:varP, dP_ab = D_ab,cd dF_cd) is symmetric for a
hyper-elastic material, so dJ/dF = (1/n) D W and the adjoint field solves
A lambda = G : (K : W) / n -- the same CG system as the Newton steps.  Then

  dJ/dmu_k = (1/n) W : (dP/dmu)_k - lambda_k : (dP/dmu)_k,
  (dP/dmu)_k = F_k . (2 dev E_k)   (S = lambda tr(E) I + 2 mu E with
                                    lambda = K - 2 mu/3, K fixed),
and in the same way, with the same lambda, for the bulk moduli
  (dP/dK)_k = F_k . (tr(E_k) I)    (mu fixed).
"""
import numpy as np

from . import fourier, j2, solver, svk, tensor as t


def dP_dmu(F):
    """(dP/dmu) = F . (2 dev E) at fixed bulk modulus, [3,3,*grid]."""
    E = svk.green_lagrange(F)
    I = t.EYE.reshape((3, 3) + (1,) * (F.ndim - 2))
    devE = E - np.trace(E) / 3.0 * I
    return t.dot_2_2(F, 2.0 * devE)


def dP_dK(F):
    """(dP/dK) = F . (tr(E) I) at fixed shear modulus, [3,3,*grid]."""
    E = svk.green_lagrange(F)
    I = t.EYE.reshape((3, 3) + (1,) * (F.ndim - 2))
    return t.dot_2_2(F, np.trace(E) * I)


def adjoint_field(problem, W, tol_cg=1e-12, cg_atol=0.0):
    """lambda solving G K G lambda = G (K : W) / n at the converged state."""
    W = np.asarray(W, dtype=np.float64)
    grid = problem.shape
    n = int(np.prod(grid))
    _, K4 = problem.constitutive(problem.F)
    op = solver.tangent_operator(K4)
    b = fourier.G(svk.tangent_apply(K4, t.uniform(W, grid)) / n)
    lam, _, _ = solver.cg(op, b, tol_cg, atol=cg_atol)
    return lam


def grad_params(problem, W, tol_cg=1e-12, cg_atol=0.0):
    """(dJ/dK, dJ/dmu) per voxel for J = W : P-bar, from one adjoint field."""
    W = np.asarray(W, dtype=np.float64)
    n = problem.F[0, 0].size
    lam = adjoint_field(problem, W, tol_cg, cg_atol)
    out = []
    for d in (dP_dK(problem.F), dP_dmu(problem.F)):
        out.append(np.einsum("ab,ab...->...", W, d) / n - np.einsum("ab...,ab...->...", lam, d))
    return tuple(out)


def grad_mu(problem, W, tol_cg=1e-12, cg_atol=0.0):
    """dJ/dmu per voxel for J = W : P-bar at the problem's converged state."""
    W = np.asarray(W, dtype=np.float64)
    grid = problem.shape
    n = int(np.prod(grid))
    _, K4 = problem.constitutive(problem.F)
    op = solver.tangent_operator(K4)
    g = svk.tangent_apply(K4, t.uniform(W, grid)) / n        # dJ/dF = (1/n) D W
    b = fourier.G(g)
    lam, _, _ = solver.cg(op, b, tol_cg, atol=cg_atol)
    d = dP_dmu(problem.F)
    explicit = np.einsum("ab,ab...->...", W, d) / n
    return explicit - np.einsum("ab...,ab...->...", lam, d)


def localization(problem, W, tol_cg=1e-12, cg_atol=0.0):
    """Microscopic response L = W + dF to a unit macroscopic perturbation W
    (the predictor system of Eq. bc:lin with dFbar = W); gives the same
    gradient through dJ/dmu_k = (1/n) L_k : (dP/dmu)_k."""
    W = np.asarray(W, dtype=np.float64)
    grid = problem.shape
    _, K4 = problem.constitutive(problem.F)
    op = solver.tangent_operator(K4)
    U = t.uniform(W, grid)
    dF, _, _ = solver.cg(op, -op(U), tol_cg, atol=cg_atol)
    return U + dF


# ---------------------------------------------------------------------------
# J2 (Sec. 5).  Reading: the derivative is taken for the last increment with
# the committed history at its start (Cp^-1_n, eps_p,n) held fixed -- the
# exact total derivative for a path of one increment from the virgin state.
# The consistent tangent of the increment is symmetric (major symmetry), so
# the adjoint system is the SVK one with the J2 tangent.  At fixed F and
# history the eigenbasis of be = F Cp^-1 F^T does not depend on the
# parameters; in it, with e the principal deviatoric log strain,
# q = sqrt(3/2 e.e), tau_eq = 2 mu q, tau_y = tau_y0 + H eps_p,n,
# dgamma = (tau_eq - tau_y)/(3 mu + H) on the plastic branch:
#   tau_p = K tr(eps) + s_p,   s_p = 2 mu e - 3 mu dgamma e / q,
#   d tau_p / dK      = tr(eps),
#   d s_p / dmu       = 2 e - 3 (dgamma + mu d dgamma/dmu) e / q,
#                       d dgamma/dmu = (2 q H + 3 tau_y) / (3 mu + H)^2,
#   d s_p / dtau_y0   = 3 mu / (3 mu + H) e / q,
#   d s_p / dH        = 3 mu (eps_p,n + dgamma) / (3 mu + H) e / q,
# (elastic branch: 2 e for mu, 0 for tau_y0 and H), and dP = d tau F^-T.
# ---------------------------------------------------------------------------
def j2_dP_dparams(F, Cpi, ep, K, mu, ty0, H):
    """(dP/dK, dP/dmu, dP/dtau_y0, dP/dH) for voxels: F, Cpi [n,3,3]; ep and
    the parameters [n].  Returns [4, n, 3, 3]."""
    st = j2.return_map(F, Cpi, ep, K, mu, ty0, H)
    Q, e, tr = st["Q"], st["dev"], st["tr"]
    plastic, dg, teq = st["plastic"], st["dg"], st["teq"]
    q = np.where(plastic, teq / (2.0 * mu), 1.0)
    den = 3.0 * mu + H
    ty = ty0 + H * ep
    ddg_dmu = (2.0 * q * H + 3.0 * ty) / den ** 2
    eq = e / q[:, None]
    d = np.zeros((4,) + e.shape)
    d[0] = tr[:, None]
    d[1] = 2.0 * e - np.where(plastic, 3.0 * (dg + mu * ddg_dmu), 0.0)[:, None] * eq
    d[2] = np.where(plastic, 3.0 * mu / den, 0.0)[:, None] * eq
    d[3] = np.where(plastic, 3.0 * mu * (ep + dg) / den, 0.0)[:, None] * eq
    dtau = np.einsum("nab,knb,ncb->knac", Q, d, Q)
    return np.einsum("knac,nbc->knab", dtau, st["Finv"])


def j2_grad_params(F, Cpi, ep, K, mu, ty0, H, W, tol_cg=1e-12, cg_atol=0.0):
    """dJ/d(K, mu, tau_y0, H) per voxel, [4, *grid], for J = W : P-bar at a
    converged J2 increment: F [3,3,*grid], the history at the start of the
    increment (Cpi [n,3,3], ep [n]) and the parameters ([n] each)."""
    W = np.asarray(W, dtype=np.float64)
    grid = F.shape[-3:]
    n = int(np.prod(grid))
    Fv = np.moveaxis(F.reshape(3, 3, -1), -1, 0)
    st = j2.return_map(Fv, Cpi, ep, K, mu, ty0, H)
    K4v = j2.tangent(Fv, Cpi, K, mu, H, st)
    K4 = np.moveaxis(K4v, 0, -1).reshape((3, 3, 3, 3) + tuple(grid))
    op = solver.tangent_operator(K4)
    b = fourier.G(svk.tangent_apply(K4, t.uniform(W, grid)) / n)
    lam, _, _ = solver.cg(op, b, tol_cg, atol=cg_atol)
    lamv = np.moveaxis(lam.reshape(3, 3, -1), -1, 0)
    dP = j2_dP_dparams(Fv, Cpi, ep, K, mu, ty0, H)
    g = np.einsum("ab,knab->kn", W, dP) / n - np.einsum("nab,knab->kn", lamv, dP)
    return g.reshape((4,) + tuple(grid))


# ---------------------------------------------------------------------------
# J2 through the history of a path of increments (reverse sweep).  With
# h_m = H(F_m, h_{m-1}) the history after increment m, F_m in equilibrium
# G:P(F_m, h_{m-1}) = 0 at <F_m> = F-bar_m, and J = W : P-bar after the last
# increment M, a backward sweep over m = M..1 carries a_m = dJ/dh_m
# (a_M = 0):
#   g_m      = (1/n) K_M W [m = M] + (dH/dF)^T a_m          (dJ/dF_m),
#   lambda_m : G K_m G lambda_m = G g_m                     (K_m symmetric),
#   c_m      = (1/n) W [m = M] - lambda_m,
#   dJ/dp   += c_m : dP/dp + (dH/dp)^T a_m,
#   a_{m-1}  = c_m : dP/dh + (dH/dh)^T a_m,
# all local derivatives at (F_m, h_{m-1}): in closed form (the return map
# linearised step by step, below) or by central differences per voxel; the
# parameter derivative of P is the closed form above.
# ---------------------------------------------------------------------------
def _hist_pack(Cpi, ep):
    return np.stack([Cpi[:, 0, 0], Cpi[:, 1, 1], Cpi[:, 2, 2], Cpi[:, 0, 1], Cpi[:, 0, 2],
                     Cpi[:, 1, 2], ep], axis=1)


def _hist_unpack(h):
    C = np.empty((h.shape[0], 3, 3))
    for k, (i, j) in enumerate(((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))):
        C[:, i, j] = h[:, k]
        C[:, j, i] = h[:, k]
    return C, h[:, 6].copy()


def j2_local_jacobians(F, Cpi, ep, K, mu, ty0, H, step=1e-7):
    """Central differences of the return map per voxel at (F, history) --
    step 1e-7: the truncation error of the logarithm / exponential of nearly
    equal eigenvalues (small strains) is still visible at 1e-6:
    dP/dh [n,9,7], dH/dF [n,7,9], dH/dh [n,7,7], dH/dp [n,7,4], with
    h = (Cp^-1_00, _11, _22, _01, _02, _12, eps_p) and p = (K, mu, tau_y0, H)."""
    n = F.shape[0]
    h0 = _hist_pack(Cpi, ep)
    prm = [K, mu, ty0, H]

    def run(Fx, hx, px):
        C, e = _hist_unpack(hx)
        st = j2.return_map(Fx, C, e, *px)
        return st["P"].reshape(n, 9), _hist_pack(st["Cpi_new"], st["ep_new"])

    dPdh = np.zeros((n, 9, 7))
    dHdh = np.zeros((n, 7, 7))
    for k in range(7):
        d = np.zeros_like(h0)
        d[:, k] = step
        Pp, Hp = run(F, h0 + d, prm)
        Pm, Hm = run(F, h0 - d, prm)
        dPdh[:, :, k] = (Pp - Pm) / (2 * step)
        dHdh[:, :, k] = (Hp - Hm) / (2 * step)
    dHdF = np.zeros((n, 7, 9))
    for a in range(9):
        d = np.zeros_like(F)
        d[:, a // 3, a % 3] = step
        _, Hp = run(F + d, h0, prm)
        _, Hm = run(F - d, h0, prm)
        dHdF[:, :, a] = (Hp - Hm) / (2 * step)
    dHdp = np.zeros((n, 7, 4))
    for t in range(4):
        s = step * np.abs(prm[t])
        pp = [q.copy() for q in prm]
        pm = [q.copy() for q in prm]
        pp[t] = prm[t] + s
        pm[t] = prm[t] - s
        _, Hp = run(F, h0, pp)
        _, Hm = run(F, h0, pm)
        dHdp[:, :, t] = (Hp - Hm) / (2 * s)[:, None]
    return dPdh, dHdF, dHdh, dHdp


def j2_path_grad_params(states, K, mu, ty0, H, W, tol_cg=1e-12, cg_atol=0.0, local="closed"):
    """dJ/d(K, mu, tau_y0, H) per voxel, [4, *grid], for J = W : P-bar after
    a path of increments.  ``states``: per increment, in order, (F_m
    [3,3,*grid] converged, Cpi_{m-1} [n,3,3], ep_{m-1} [n]) -- the field
    and the history at the increment's start.  ``local``: the return map's
    derivatives in closed form ("closed") or by central differences ("fd")."""
    W = np.asarray(W, dtype=np.float64)
    grid = states[0][0].shape[-3:]
    n = int(np.prod(grid))
    prm = (K, mu, ty0, H)
    a = np.zeros((n, 7))
    g = np.zeros((4, n))
    last = len(states) - 1
    for m in range(last, -1, -1):
        F, Cpi, ep = states[m]
        Fv = np.moveaxis(F.reshape(3, 3, -1), -1, 0)
        st = j2.return_map(Fv, Cpi, ep, *prm)
        K4v = j2.tangent(Fv, Cpi, K, mu, H, st)
        K4 = np.moveaxis(K4v, 0, -1).reshape((3, 3, 3, 3) + tuple(grid))
        jac = j2_local_jacobians_closed if local == "closed" else j2_local_jacobians
        dPdh, dHdF, dHdh, dHdp = jac(Fv, Cpi, ep, *prm)
        gF = np.einsum("nka,nk->na", dHdF, a)
        gfield = np.moveaxis(gF, 0, -1).reshape((3, 3) + tuple(grid))
        if m == last:
            gfield = gfield + svk.tangent_apply(K4, t.uniform(W, grid)) / n
        op = solver.tangent_operator(K4)
        lam, _, _ = solver.cg(op, fourier.G(gfield), tol_cg, atol=cg_atol)
        c = -np.moveaxis(lam.reshape(3, 3, -1), -1, 0).reshape(n, 9)
        if m == last:
            c = c + W.reshape(9) / n
        dPdp = j2_dP_dparams(Fv, Cpi, ep, *prm).reshape(4, n, 9)
        g += np.einsum("na,tna->tn", c, dPdp) + np.einsum("nk,nkt->tn", a, dHdp)
        a = np.einsum("na,nak->nk", c, dPdh) + np.einsum("nk,nkj->nj", a, dHdh)
    return g.reshape((4,) + tuple(grid))


def _sinhc(x):
    """sinh(x)/x, 1 at x = 0."""
    with np.errstate(invalid="ignore", divide="ignore"):
        return np.where(np.abs(x) < 1e-8, 1.0 + x * x / 6.0, np.sinh(x) / np.where(x == 0, 1.0, x))


def j2_return_map_directional(F, Cpi, ep, K, mu, ty0, H, dF=None, dC=None, dep=None, dprm=None):
    """Directional derivative of the J2 return map per voxel, in closed form:
    (dP [n,3,3], dh_new [n,7]) for perturbations dF [n,3,3], dC [n,3,3]
    (symmetric), dep [n] and dprm [4, n] of (K, mu, tau_y0, H).  Each step
    of ``j2.return_map`` linearised: the logarithm by the Daleckii-Krein
    divided differences of ln, the radial return, the exponential of the
    elastic log strain by those of exp(2 x), the pull-backs with
    d(F^-1) = -F^-1 dF F^-1."""
    n = F.shape[0]
    Z = np.zeros((n, 3, 3))
    dF = Z if dF is None else dF
    dC = Z if dC is None else dC
    dep = np.zeros(n) if dep is None else dep
    dK, dmu, dty, dH = (np.zeros((4, n)) if dprm is None else dprm)
    st = j2.return_map(F, Cpi, ep, K, mu, ty0, H)
    Q, lam, plastic = st["Q"], st["lam"], st["plastic"]
    teq, dg, beta, tr = st["teq"], st["dg"], st["beta"], st["tr"]
    Finv = st["Finv"]
    FT = np.swapaxes(F, -1, -2)
    QT = np.swapaxes(Q, -1, -2)
    I = np.eye(3)
    # trial log strain
    dbe = dF @ Cpi @ FT + F @ Cpi @ np.swapaxes(dF, -1, -2) + F @ dC @ FT
    deps = Q @ (0.5 * j2._f1(lam) * (QT @ dbe @ Q)) @ QT
    dtr = np.trace(deps, axis1=-2, axis2=-1)
    Ed = np.einsum("nab,nb,ncb->nac", Q, st["dev"], Q)             # deviatoric log strain
    dEd = deps - dtr[:, None, None] * I / 3.0
    s_tr = 2.0 * mu[:, None, None] * Ed
    ds_tr = 2.0 * mu[:, None, None] * dEd + 2.0 * dmu[:, None, None] * Ed
    den = 3.0 * mu + H
    tsafe = np.where(teq > 0, teq, 1.0)
    dteq = np.where(plastic, 1.5 * (s_tr * ds_tr).sum((-2, -1)) / tsafe, 0.0)
    dphi = dteq - dty - dH * ep - H * dep
    ddg = np.where(plastic, (dphi - dg * (3.0 * dmu + dH)) / den, 0.0)
    dbeta = np.where(plastic, -3.0 * (dmu * dg + mu * ddg) / tsafe
                     + 3.0 * mu * dg * dteq / tsafe ** 2, 0.0)
    tau = st["tau"]
    dtau = ((dK * tr + K * dtr)[:, None, None] * I + dbeta[:, None, None] * s_tr
            + beta[:, None, None] * ds_tr)
    dFinv = -Finv @ dF @ Finv
    dP = dtau @ st["FinvT"] + tau @ np.swapaxes(dFinv, -1, -2)
    # new history
    x = tr[:, None] / 3.0 + beta[:, None] * st["dev"]                 # principal elastic log strain
    deps_e = dtr[:, None, None] * I / 3.0 + dbeta[:, None, None] * Ed + beta[:, None, None] * dEd
    xa, xb = x[:, :, None], x[:, None, :]
    g1 = 2.0 * np.exp(xa + xb) * _sinhc(xa - xb)                     # divided differences of exp(2x)
    dbn = Q @ (g1 * (QT @ deps_e @ Q)) @ QT
    bn = np.einsum("nab,nb,ncb->nac", Q, np.exp(2.0 * x), Q)
    dCn = dFinv @ bn @ st["FinvT"] + Finv @ dbn @ st["FinvT"] + Finv @ bn @ np.swapaxes(dFinv, -1, -2)
    dCn = 0.5 * (dCn + np.swapaxes(dCn, -1, -2))
    dh = _hist_pack(dCn, dep + ddg)
    return dP, dh


def j2_local_jacobians_closed(F, Cpi, ep, K, mu, ty0, H):
    """Same outputs as ``j2_local_jacobians`` from the closed-form
    directional derivatives."""
    n = F.shape[0]
    prm = (K, mu, ty0, H)
    dPdh = np.zeros((n, 9, 7))
    dHdh = np.zeros((n, 7, 7))
    for k in range(7):
        e = np.zeros((n, 7))
        e[:, k] = 1.0
        dC, dep = _hist_unpack(e)
        dP, dh = j2_return_map_directional(F, Cpi, ep, *prm, dC=dC, dep=dep)
        dPdh[:, :, k] = dP.reshape(n, 9)
        dHdh[:, :, k] = dh
    dHdF = np.zeros((n, 7, 9))
    for a in range(9):
        dF = np.zeros((n, 3, 3))
        dF[:, a // 3, a % 3] = 1.0
        _, dh = j2_return_map_directional(F, Cpi, ep, *prm, dF=dF)
        dHdF[:, :, a] = dh
    dHdp = np.zeros((n, 7, 4))
    for t in range(4):
        d = np.zeros((4, n))
        d[t] = 1.0
        _, dh = j2_return_map_directional(F, Cpi, ep, *prm, dprm=d)
        dHdp[:, :, t] = dh
    return dPdh, dHdF, dHdh, dHdp
