"""Discrete Fourier transform and the compatibility projection G.

Follows Sec. 2.3-2.5 (Eq. weak:discr:FFT-intermediate, Eq. G) and
Appendix D (Eq. G_red); grids of even size along an axis follow Appendix C:
G-hat is zero at every frequency vector with a Nyquist component (the
variant that keeps the deformation gradient compatible).

Readings of the paper used here:
* The ``fftshift``/``ifftshift`` pair of the paper's listing only re-centres
  the frequency axis; for a multiplier whose frequencies are assigned with the
  same centring the shifts cancel, so standard-order DFTs with signed integer
  frequencies are used.
* xi_i = q_i / L_i with L_i the cell size; voxels are unit cubes, so
  L_i = N_i.  On cubic grids the scaling cancels in xi (x) xi / |xi|^2.
* The inverse transform's result is real (G-hat is real and even in q, with
  the Nyquist frequencies of even axes zeroed); the imaginary round-off is
  dropped, as the listing does.
"""
import numpy as np

try:  # optional multi-threaded backend for large timing runs
    import scipy.fft as _sfft
except Exception:  # pragma: no cover
    _sfft = None

_BACKEND = {"name": "numpy", "workers": 1}


def set_backend(name: str = "numpy", workers: int = 1):
    """Choose the DFT routine: 'naive' (dense matrices, O(N^4) per 3-D
    transform), 'numpy' (numpy.fft) or 'scipy' (scipy.fft, multi-threaded)."""
    if name not in ("naive", "numpy", "scipy"):
        raise ValueError(name)
    if name == "scipy" and _sfft is None:
        raise RuntimeError("scipy.fft not available")
    _BACKEND["name"] = name
    _BACKEND["workers"] = int(workers)


def get_backend():
    return dict(_BACKEND)


def frequencies(n: int) -> np.ndarray:
    """Signed integer frequencies in standard DFT order: k for
    k <= (n-1)/2, else k - n.  Odd n: the centred range -(n-1)/2 .. (n-1)/2
    of the paper's listing, in unshifted order; even n: -n/2 .. n/2-1 (the
    listing of Appendix C), the Nyquist index n/2 carrying -n/2."""
    k = np.arange(n)
    return np.where(k <= (n - 1) // 2, k, k - n)


def nyquist_mask(grid_shape) -> np.ndarray:
    """True at the frequency vectors with a component at the Nyquist index
    n/2 of an axis of even size n (Appendix C), shape [nx, ny, nz]."""
    m = [(np.arange(n) == n // 2) & (n % 2 == 0) for n in grid_shape]
    X, Y, Z = np.meshgrid(*m, indexing="ij")
    return X | Y | Z


def dft_matrix(n: int, inverse: bool = False) -> np.ndarray:
    """W[j, k] = exp(-+ 2 pi i ((j k) mod n) / n); the exponent is reduced in
    integers before the FP64 angle is formed."""
    j = np.arange(n)
    e = np.mod(np.outer(j, j), n).astype(np.float64)
    sign = 1.0 if inverse else -1.0
    return np.exp(sign * 2j * np.pi * e / n)


def _dft_axis_naive(A, axis, inverse):
    n = A.shape[axis]
    W = dft_matrix(n, inverse)
    out = np.tensordot(A, W, axes=([axis], [0]))  # new axis goes last
    out = np.moveaxis(out, -1, axis)
    if inverse:
        out = out / n
    return out


def dft3(A, inverse: bool = False):
    """Unnormalised forward DFT (sign -1) or normalised inverse (1/n) over the
    last three axes, using the selected backend."""
    name = _BACKEND["name"]
    axes = (-3, -2, -1)
    if name == "numpy":
        return np.fft.ifftn(A, axes=axes) if inverse else np.fft.fftn(A, axes=axes)
    if name == "scipy":
        w = _BACKEND["workers"]
        return (_sfft.ifftn(A, axes=axes, workers=w) if inverse
                else _sfft.fftn(A, axes=axes, workers=w))
    out = np.asarray(A, dtype=np.complex128)
    for ax in axes:
        out = _dft_axis_naive(out, ax, inverse)
    return out


def scaled_frequencies(grid_shape):
    """xi[k] on the grid, shape [3, nx, ny, nz]; xi_i = q_i / N_i."""
    nx, ny, nz = grid_shape
    qx = frequencies(nx) / nx
    qy = frequencies(ny) / ny
    qz = frequencies(nz) / nz
    X, Y, Z = np.meshgrid(qx, qy, qz, indexing="ij")
    return np.stack([X, Y, Z])


def ghat_reduced(grid_shape):
    """g-hat_jl(q) = xi_j xi_l / |xi|^2, zero at q = 0 (Eq. G_red) and at
    Nyquist frequencies (Appendix C).  Shape [3, 3, nx, ny, nz]."""
    xi = scaled_frequencies(grid_shape)
    n2 = (xi * xi).sum(axis=0)
    g = np.einsum("j...,l...->jl...", xi, xi)
    keep = (n2 != 0) & ~nyquist_mask(grid_shape)
    g[:, :, keep] /= n2[keep]
    g[:, :, ~keep] = 0.0
    return g


def ghat4(grid_shape):
    """The full G-hat_ijlm(q) = d_im xi_j xi_l / |xi|^2 (Eq. G), zero at
    q = 0 and at Nyquist frequencies.  Shape [3,3,3,3,*grid] -- for small
    grids only (81 reals/node)."""
    g = ghat_reduced(grid_shape)
    return np.einsum("im,jl...->ijlm...", np.eye(3), g)


def apply_ghat(Ahat, g):
    """C_ij = G-hat_ijlm A_ml = d_im g_jl A_ml = g_jl A_il (Eq. G_red)."""
    return np.einsum("jl...,il...->ij...", g, Ahat)


def G(A):
    """Projection G : A = F^-1{ G-hat : F{A} } (Eq. weak:discr:FFT-
    intermediate) of a real second-order field ``[3, 3, *grid]``."""
    A = np.asarray(A, dtype=np.float64)
    g = ghat_reduced(A.shape[-3:])
    return np.real(dft3(apply_ghat(dft3(A), g), inverse=True))


def G_literal(A):
    """Same as :func:`G` but contracting with the full 81-component G-hat of
    Eq. G (small grids only)."""
    A = np.asarray(A, dtype=np.float64)
    G4 = ghat4(A.shape[-3:])
    Ahat = dft3(A)
    Chat = np.einsum("ijlm...,ml...->ij...", G4, Ahat)
    return np.real(dft3(Chat, inverse=True))
