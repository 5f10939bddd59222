"""Seeded synthetic microstructures and load schedules.

This module holds no arithmetic of the homogenisation method: it only draws
phase maps, per-voxel moduli and macroscopic deformation ramps.  Both the FP64
oracle (``oracle/``) and the GPU path's tests and benchmark take their inputs
from here, so that the two sides see identical data.

Conventions
-----------
* Grids are ``[nx, ny, nz]`` arrays in C order (z fastest), voxel centres at
  integer coordinates.
* ``phase`` is ``uint8``; ``phase_params`` is ``[nphase, nparam]`` float64.
  For Saint Venant-Kirchhoff the parameters are ``(K, mu)`` (bulk and shear
  modulus); for J2 plasticity ``(K, mu, tau_y0, H)``.
* Macroscopic deformation gradients are 3x3 arrays with
  ``F[i, j] = dx_i / dX_j``.

The recipes (sphere packing, Voronoi cells, lognormal moduli) are the readings
of the benchmark configurations recorded in the design notes of this
repository; each function's docstring states its rule.
"""
from __future__ import annotations

import numpy as np

# Moduli of the paper's examples (Sec. 4.4 and the printed 31^3 example of
# Appendix B): matrix K = 0.833, mu = 0.386; the inclusion is 10x stiffer.
K_SOFT = 0.833
MU_SOFT = 0.386


def cube_inclusion(n: int = 31, size: int = 9) -> np.ndarray:
    """Two-phase grid with a ``size``^3 cube of phase 1 in one corner.

    Same geometry as the paper's example of Sec. 4.4 (Appendix B): phase 1
    occupies ``x >= n-size``, ``y < size``, ``z >= n-size``.
    """
    ph = np.zeros((n, n, n), dtype=np.uint8)
    ph[n - size:, :size, n - size:] = 1
    return ph


def laminate(shape, normal_axis: int, fraction: float = 0.5) -> np.ndarray:
    """Layered two-phase grid whose phase depends on one coordinate only.

    Phase 1 fills the first ``round(fraction * N)`` layers along
    ``normal_axis``.
    """
    shape = tuple(int(s) for s in shape)
    nl = shape[normal_axis]
    k = int(round(fraction * nl))
    idx = [None, None, None]
    idx[normal_axis] = slice(None)
    layer = np.zeros(nl, dtype=np.uint8)
    layer[:k] = 1
    ph = np.broadcast_to(layer[tuple(idx)], shape).astype(np.uint8).copy()
    return ph


def _periodic_delta(a: np.ndarray, n: int) -> np.ndarray:
    d = np.abs(a) % n
    return np.minimum(d, n - d)


def spheres(n: int, fraction: float, rmin: float, rmax: float,
            rng: np.random.Generator, max_reject: int = 10_000):
    """Random sequential addition of non-overlapping periodic spheres.

    Draw a centre uniformly in ``[0, n)^3`` and a radius ``r ~ U[rmin, rmax]``;
    reject the candidate if its periodic centre distance to an accepted sphere
    is below the sum of radii.  A voxel (centre at integer coordinates) is
    inside a sphere if its periodic distance to the centre is ``<= r``.  Stop
    as soon as the voxel fraction reaches ``fraction``, or after
    ``max_reject`` consecutive rejections.  The radius range is clipped to
    ``r_max = min(rmax, (n-1)//4)`` for small cells.

    Returns ``(phase uint8 [n,n,n], achieved_fraction)``.
    """
    r_hi = min(float(rmax), float((n - 1) // 4))
    r_lo = min(float(rmin), r_hi)
    ph = np.zeros((n, n, n), dtype=np.uint8)
    centres = np.zeros((0, 3))
    radii = np.zeros(0)
    filled = 0
    target = fraction * n ** 3
    rejects = 0
    while filled < target and rejects < max_reject:
        c = rng.uniform(0.0, n, size=3)
        r = rng.uniform(r_lo, r_hi)
        if len(radii):
            d = _periodic_delta(centres - c, n)
            if np.any(np.sqrt((d * d).sum(axis=1)) < r + radii):
                rejects += 1
                continue
        rejects = 0
        centres = np.vstack([centres, c])
        radii = np.append(radii, r)
        # mark voxels within a bounding box, with periodic wrap (the box is
        # narrower than the cell, so the wrapped indices are distinct)
        lo = np.floor(c - r).astype(int)
        hi = np.ceil(c + r).astype(int)
        ax = [np.arange(lo[k], hi[k] + 1) for k in range(3)]
        dx = _periodic_delta(ax[0] - c[0], n)[:, None, None]
        dy = _periodic_delta(ax[1] - c[1], n)[None, :, None]
        dz = _periodic_delta(ax[2] - c[2], n)[None, None, :]
        inside = (dx * dx + dy * dy + dz * dz) <= r * r
        sel = np.ix_(np.mod(ax[0], n), np.mod(ax[1], n), np.mod(ax[2], n))
        before = int(ph[sel].sum(dtype=np.int64))
        ph[sel] |= inside.astype(np.uint8)
        filled += int(ph[sel].sum(dtype=np.int64)) - before
    return ph, filled / n ** 3


def voronoi(n: int, ncells: int, rng: np.random.Generator,
            nhard: int | None = None) -> tuple[np.ndarray, np.ndarray]:
    """Periodic Voronoi tessellation with cells assigned soft (0) / hard (1).

    ``ncells`` seed points uniform in ``[0, n)^3``; each voxel centre goes to
    the seed at the smallest periodic (minimum-image) Euclidean distance, ties
    to the lowest seed index.  A seeded permutation makes exactly ``nhard``
    cells (default half) hard.  Returns ``(phase uint8, cell_id int32)``.
    """
    if nhard is None:
        nhard = ncells // 2
    seeds = rng.uniform(0.0, n, size=(ncells, 3))
    perm = rng.permutation(ncells)
    cell_phase = np.zeros(ncells, dtype=np.uint8)
    cell_phase[perm[:nhard]] = 1
    cell = np.empty((n, n, n), dtype=np.int32)
    coords = np.arange(n, dtype=np.float64)
    # squared periodic offsets per seed and axis; d2 = (dx^2 + dy^2) + dz^2
    # in the same order of operations for every voxel
    dx2 = np.stack([_periodic_delta(coords - seeds[s, 0], n) ** 2 for s in range(ncells)])
    dy2 = np.stack([_periodic_delta(coords - seeds[s, 1], n) ** 2 for s in range(ncells)])
    dz2 = np.stack([_periodic_delta(coords - seeds[s, 2], n) ** 2 for s in range(ncells)])
    best = np.empty((n, n))
    d2 = np.empty((n, n))
    better = np.empty((n, n), dtype=bool)
    for x in range(n):
        best.fill(np.inf)
        arg = np.zeros((n, n), dtype=np.int32)
        for s in range(ncells):
            np.add((dx2[s, x] + dy2[s])[:, None], dz2[s][None, :], out=d2)
            np.less(d2, best, out=better)
            np.copyto(best, d2, where=better)
            arg[better] = s
        cell[x] = arg
    return cell_phase[cell], cell


def lognormal_mu(shape, rng: np.random.Generator, mean: float = MU_SOFT,
                 sigma: float = 0.5) -> np.ndarray:
    """i.i.d. lognormal shear modulus with the given arithmetic mean.

    ``mu = exp(m + sigma Z)``, ``Z ~ N(0, 1)``, ``m = ln(mean) - sigma^2/2``.
    """
    m = np.log(mean) - 0.5 * sigma * sigma
    return np.exp(m + sigma * rng.standard_normal(size=tuple(shape)))


def simple_shear(gamma: float) -> np.ndarray:
    """``F = I + gamma e_x (x) e_y`` (Eq. elas:deform)."""
    F = np.eye(3)
    F[0, 1] += gamma
    return F


def uniaxial(eps: float) -> np.ndarray:
    """``F = diag(1 + eps, 1, 1)``."""
    return np.diag([1.0 + eps, 1.0, 1.0])


# Mixed control masks: True where the P-bar component (3i+j) is prescribed
# and F-bar is free; False where F-bar is prescribed.
def uniaxial_stress_mask() -> np.ndarray:
    """Uniaxial stress along x: F11 prescribed, F21 = F31 = F32 prescribed
    (they fix the rotation), P12, P13, P22, P23, P33 prescribed."""
    m = np.zeros(9, dtype=bool)
    m[[1, 2, 4, 5, 8]] = True
    return m


def ramp(final: np.ndarray, nincr: int) -> list[np.ndarray]:
    """Equal increments from I to ``final``: ``I + (k/m)(final - I)``."""
    final = np.asarray(final, dtype=np.float64)
    eye = np.eye(3)
    return [eye + (k / nincr) * (final - eye) for k in range(1, nincr + 1)]


def two_phase_params(contrast: float, k0: float = K_SOFT,
                     mu0: float = MU_SOFT) -> np.ndarray:
    """``[[K, mu] matrix, [K, mu] inclusion]`` with inclusion = contrast x matrix."""
    return np.array([[k0, mu0], [contrast * k0, contrast * mu0]],
                    dtype=np.float64)


def random_field(shape, rng: np.random.Generator, scale: float = 1.0):
    """Gaussian real field of the given shape (test data only)."""
    return scale * rng.standard_normal(size=tuple(shape))


def random_F(shape, rng: np.random.Generator, amp: float = 0.2):
    """Deformation gradients ``I + amp * U[-1,1]`` per voxel, ``[3,3,*shape]``."""
    shape = tuple(shape)
    F = amp * rng.uniform(-1.0, 1.0, size=(3, 3) + shape)
    for i in range(3):
        F[i, i] += 1.0
    return F


# ---------------------------------------------------------------------------
# Named workloads
# ---------------------------------------------------------------------------

def config_cube31():
    """31^3, 9^3 corner cube, contrast 10, simple shear to 0.1 in 10 steps."""
    return dict(name="svk31_cube", shape=(31, 31, 31), model="svk",
                phase=cube_inclusion(31, 9),
                phase_params=two_phase_params(10.0),
                schedule=ramp(simple_shear(0.1), 10),
                tol_newton=1e-5, tol_cg=1e-8)


def config_spheres(n: int = 125, seed: int = 1, nincr: int = 20,
                   eps: float = 0.2):
    """Spheres (fraction 0.3, r in [4,10], contrast 100), uniaxial ramp."""
    rng = np.random.default_rng(seed)
    ph, frac = spheres(n, 0.3, 4.0, 10.0, rng)
    return dict(name=f"svk{n}_spheres", shape=(n, n, n), model="svk",
                phase=ph, fraction=frac,
                phase_params=two_phase_params(100.0),
                schedule=ramp(uniaxial(eps), nincr),
                tol_newton=1e-5, tol_cg=1e-8)


def config_voronoi_j2(n: int = 315, seed: int = 2, nincr: int = 20,
                      gamma: float = 0.2):
    """64-cell periodic Voronoi, 32 soft / 32 hard, J2, simple shear ramp.

    E = 1, nu = 0.3 -> K = 1/1.2, mu = 1/2.6; tau_y0 = 0.003 / 0.006;
    H = 0.01 in both phases.
    """
    rng = np.random.default_rng(seed)
    ph, _ = voronoi(n, 64, rng)
    K, mu = 1.0 / 1.2, 1.0 / 2.6
    params = np.array([[K, mu, 0.003, 0.01], [K, mu, 0.006, 0.01]])
    return dict(name=f"j2_{n}_voronoi", shape=(n, n, n), model="j2",
                phase=ph, phase_params=params,
                schedule=ramp(simple_shear(gamma), nincr),
                tol_newton=1e-5, tol_cg=1e-8)


def config_batch(nrve: int = 256, seed: int = 3,
                 sizes=(15, 21, 27, 33, 45, 63)):
    """Batch of SVK RVEs of uneven size, each with its own spheres and F."""
    rng = np.random.default_rng(seed)
    rves = []
    for _ in range(nrve):
        n = int(rng.choice(sizes))
        frac = rng.uniform(0.1, 0.4)
        contrast = rng.uniform(2.0, 100.0)
        ph, got = spheres(n, frac, 4.0, 10.0, rng)
        Fbar = np.eye(3) + rng.uniform(-0.05, 0.05, size=(3, 3))
        rves.append(dict(shape=(n, n, n), phase=ph, fraction=got,
                         phase_params=two_phase_params(contrast),
                         Fbar=Fbar))
    return rves


def config_lognormal(n: int = 243, seed: int = 4, gamma: float = 0.05):
    """Lognormal mu field (sigma 0.5, mean 0.386), K = 0.833, shear 0.05."""
    rng = np.random.default_rng(seed)
    mu = lognormal_mu((n, n, n), rng)
    K = np.full((n, n, n), K_SOFT)
    return dict(name=f"svk{n}_lognormal", shape=(n, n, n), model="svk",
                voxel_params=np.stack([K, mu]),
                schedule=[simple_shear(gamma)],
                tol_newton=1e-5, tol_cg=1e-8)
