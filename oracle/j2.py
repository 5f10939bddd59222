"""Finite-strain J2 elasto-plasticity (Sec. 5): multiplicative split
F = Fe.Fp, Kirchhoff stress linear in the logarithmic elastic strain
(tau = C : (1/2) ln be, C of Eq. elas:C), von Mises yield function
phi = tau_eq - tau_y(eps_p) <= 0 (Eq. simo:flow) with linear hardening
tau_y = tau_y0 + H eps_p, associative flow integrated with an elastic
predictor / plastic corrector, and the pull-back P = tau . F^-T.

The paper gives the structure and defers the return mapping and the
algorithmic tangent to Simo (1992) and Geers (2004); the readings used here
(written out from the mechanics, not taken from those references):

* history per voxel: Cp^-1 = Fp^-1 Fp^-T (symmetric) and eps_p; initially
  I and 0;
* trial: be = F Cp^-1 F^T, eps_tr = (1/2) ln be (principal logarithm),
  tau_tr = K tr(eps_tr) I + 2 mu dev(eps_tr);
* tau_eq = sqrt(3/2 dev(tau):dev(tau)); the plastic branch is taken when
  phi_tr > -1e-10 tau_y, i.e. also ON the yield surface, where dgamma =
  max(phi_tr, 0) / (3 mu + H) = 0 leaves the stress elastic and the tangent
  is the elasto-plastic one.  A state that yielded in the last increment
  starts the next one exactly on the surface (phi = 0 up to round-off), and
  Algorithm 1 evaluates the predictor tangent there; Sec. 5.3 says the
  discrete switch affects the convergence only around the yield point and
  Sec. 5.5 reports two Newton iterations per increment in the plastic
  regime, which the elastic tangent on the surface would not give;
* radial return in logarithmic strain: dgamma = phi_tr / (3 mu + H),
  dev(tau) = beta dev(tau_tr), beta = 1 - 3 mu dgamma / tau_eq_tr,
  eps_p += dgamma, elastic strain eps_e = tr(eps_tr)/3 I + beta dev(eps_tr),
  be = exp(2 eps_e), trial history Cp^-1 = F^-1 be F^-T;
* tangent: the exact derivative dP/dF of this update with the committed
  history frozen: d(be) = dF Cp^-1 F^T + F Cp^-1 dF^T,
  d(eps_tr) = (1/2) Dln(be)[d(be)] with the Daleckii-Krein formula
  (Q^T d(eps) Q)_ab = (1/2) f1(l_a, l_b) (Q^T d(be) Q)_ab,
  f1(x, y) = (ln x - ln y)/(x - y) = atanh(t)/(m t), t = (x-y)/(x+y),
  m = (x+y)/2 (f1 = 1/m at t = 0); then d(tau) from the return map and
  dP = d(tau) F^-T - tau F^-T dF^T F^-T.  Stored in the convention of
  Eq. iter:varP: K_ijkl = dP_ji / dF_kl.

Parameters per voxel: K (bulk), mu (shear), tau_y0, H.
"""
import numpy as np


def _sym_eig(A):
    """Eigen-decomposition of stacked symmetric 3x3 matrices [..., 3, 3]."""
    return np.linalg.eigh(A)


def _f1(lam):
    """Divided differences f1(l_a, l_b) of ln, [..., 3, 3]."""
    x = lam[..., :, None]
    y = lam[..., None, :]
    m = 0.5 * (x + y)
    t = (x - y) / (x + y)
    with np.errstate(invalid="ignore", divide="ignore"):
        f = np.where(t == 0.0, 1.0 / m, np.arctanh(t) / (m * np.where(t == 0.0, 1.0, t)))
    return f


def _to_voxels(A):
    """[3, 3, *grid] -> [n, 3, 3]."""
    return np.moveaxis(A.reshape(3, 3, -1), -1, 0)


def _to_grid(A, grid):
    """[n, 3, 3] -> [3, 3, *grid]."""
    return np.moveaxis(A, 0, -1).reshape((3, 3) + tuple(grid))


def return_map(F, Cpi, ep, K, mu, ty0, H):
    """Stress and trial history for voxels.  F, Cpi: [n,3,3]; ep, K, mu,
    ty0, H: [n].  Returns dict with P, tau, Cpi_new, ep_new and the pieces
    the tangent needs."""
    I = np.eye(3)
    be = F @ Cpi @ np.swapaxes(F, -1, -2)
    be = 0.5 * (be + np.swapaxes(be, -1, -2))
    lam, Q = _sym_eig(be)
    eps = 0.5 * np.log(lam)                               # principal log strains
    tr = eps.sum(-1)
    dev = eps - tr[:, None] / 3.0
    s_tr = 2.0 * mu[:, None] * dev                        # principal deviatoric trial stress
    teq = np.sqrt(1.5 * (s_tr * s_tr).sum(-1))
    phi = teq - (ty0 + H * ep)
    plastic = phi > -1e-10 * (ty0 + H * ep)
    dg = np.where(plastic, np.maximum(phi, 0.0) / (3.0 * mu + H), 0.0)
    with np.errstate(invalid="ignore", divide="ignore"):
        beta = np.where(plastic, 1.0 - 3.0 * mu * dg / np.where(teq > 0, teq, 1.0), 1.0)
    tau_p = K[:, None] * tr[:, None] + beta[:, None] * s_tr   # principal Kirchhoff stress
    tau = np.einsum("nab,nb,ncb->nac", Q, tau_p, Q)
    Finv = np.linalg.inv(F)
    FinvT = np.swapaxes(Finv, -1, -2)
    P = tau @ FinvT
    eps_e = tr[:, None] / 3.0 + beta[:, None] * dev
    be_new = np.einsum("nab,nb,ncb->nac", Q, np.exp(2.0 * eps_e), Q)
    Cpi_new = Finv @ be_new @ FinvT
    Cpi_new = 0.5 * (Cpi_new + np.swapaxes(Cpi_new, -1, -2))
    return dict(P=P, tau=tau, Cpi_new=Cpi_new, ep_new=ep + dg, lam=lam, Q=Q, dev=dev,
                s_tr=s_tr, teq=teq, dg=dg, beta=beta, plastic=plastic, Finv=Finv,
                FinvT=FinvT, tr=tr)


def tangent(F, Cpi, K, mu, H, st):
    """K_ijkl = dP_ji/dF_kl for voxels ([n,3,3,3,3]) by linearising every
    step of return_map in a unit direction dF = e_k (x) e_l."""
    n = F.shape[0]
    Q, lam = st["Q"], st["lam"]
    f1 = _f1(lam)
    FT = np.swapaxes(F, -1, -2)
    tau, FinvT = st["tau"], st["FinvT"]
    plastic, teq, dg, beta = st["plastic"], st["teq"], st["dg"], st["beta"]
    K4 = np.zeros((n, 3, 3, 3, 3))
    for k in range(3):
        for l in range(3):
            dF = np.zeros((n, 3, 3))
            dF[:, k, l] = 1.0
            dbe = dF @ Cpi @ FT + F @ Cpi @ np.swapaxes(dF, -1, -2)
            dbe_q = np.swapaxes(Q, -1, -2) @ dbe @ Q           # eigenbasis of be
            deps_q = 0.5 * f1 * dbe_q                           # Daleckii-Krein
            deps = Q @ deps_q @ np.swapaxes(Q, -1, -2)
            dtr = np.trace(deps, axis1=-2, axis2=-1)
            ddev = deps - dtr[:, None, None] * np.eye(3) / 3.0
            ds_tr = 2.0 * mu[:, None, None] * ddev
            # trial deviatoric stress in the global basis
            s_tr = np.einsum("nab,nb,ncb->nac", Q, st["s_tr"], Q)
            with np.errstate(invalid="ignore", divide="ignore"):
                dteq = np.where(plastic, 1.5 * (s_tr * ds_tr).sum((-2, -1))
                                / np.where(teq > 0, teq, 1.0), 0.0)
                dbeta = np.where(plastic, -3.0 * mu * (dteq / (3.0 * mu + H) - dg * dteq
                                                       / np.where(teq > 0, teq, 1.0))
                                 / np.where(teq > 0, teq, 1.0), 0.0)
            ds = beta[:, None, None] * ds_tr + dbeta[:, None, None] * s_tr
            dtau = K[:, None, None] * dtr[:, None, None] * np.eye(3) + ds
            dP = dtau @ FinvT - tau @ FinvT @ np.swapaxes(dF, -1, -2) @ FinvT
            K4[:, :, :, k, l] = np.swapaxes(dP, -1, -2)         # K_ijkl = dP_ji
    return K4


class J2Material:
    """Per-voxel J2 material with committed history."""

    def __init__(self, grid, K, mu, ty0, H):
        self.grid = tuple(grid)
        n = int(np.prod(self.grid))
        b = lambda a: np.broadcast_to(np.asarray(a, dtype=np.float64), self.grid).reshape(-1).copy()
        self.K, self.mu, self.ty0, self.H = b(K), b(mu), b(ty0), b(H)
        self.Cpi = np.broadcast_to(np.eye(3), (n, 3, 3)).copy()
        self.ep = np.zeros(n)
        self._trial = None

    def constitutive(self, F):
        """(P, K4) at F with the committed history; remembers the trial history."""
        Fv = _to_voxels(F)
        st = return_map(Fv, self.Cpi, self.ep, self.K, self.mu, self.ty0, self.H)
        K4 = tangent(Fv, self.Cpi, self.K, self.mu, self.H, st)
        self._trial = (st["Cpi_new"], st["ep_new"])
        P = _to_grid(st["P"], self.grid)
        K4g = np.moveaxis(K4, 0, -1).reshape((3, 3, 3, 3) + self.grid)
        return P, K4g

    def stress(self, F):
        Fv = _to_voxels(F)
        st = return_map(Fv, self.Cpi, self.ep, self.K, self.mu, self.ty0, self.H)
        return _to_grid(st["P"], self.grid)

    def commit(self):
        """Store history variables (Algorithm 1, after convergence)."""
        self.Cpi, self.ep = self._trial
