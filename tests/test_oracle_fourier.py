"""Pins of the oracle's DFT and projection (CPU only).

The projection G is pinned by what Appendix D and Sec. 2.5 prove about it:
idempotent, symmetric, zero mean (Eq. G:mean), range = compatible fields
(curl-free rows, Appendix D), identity on zero-mean compatible fields; and by
brute force: on tiny grids its matrix equals the orthogonal projector onto
gradients of periodic trigonometric displacement fields, computed by least
squares without G-hat, and has rank 3(n-1).
"""
import numpy as np
import pytest

from oracle import fourier, tensor as t

SIZES = [1, 3, 5, 7, 9, 11, 13, 15, 21, 27, 31, 33, 45, 63]


@pytest.fixture(autouse=True)
def _numpy_backend():
    fourier.set_backend("numpy")
    yield
    fourier.set_backend("numpy")


@pytest.mark.parametrize("n", SIZES + [125, 243, 315])
def test_naive_dft_matches_numpy_fft(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal((4, n)) + 1j * rng.standard_normal((4, n))
    W = fourier.dft_matrix(n)
    ref = np.fft.fft(x, axis=-1)
    got = x @ W
    assert np.abs(got - ref).max() <= 1e-13 * max(1.0, np.abs(ref).max()) * np.sqrt(n)
    Wi = fourier.dft_matrix(n, inverse=True)
    back = (got @ Wi) / n
    assert np.abs(back - x).max() < 1e-12


@pytest.mark.parametrize("shape", [(3, 5, 7), (9, 1, 5), (11, 13, 3)])
def test_dft3_backends_parseval_roundtrip(shape):
    rng = np.random.default_rng(1)
    A = rng.standard_normal((3, 3) + shape)
    ref = fourier.dft3(A)
    fourier.set_backend("naive")
    got = fourier.dft3(A)
    back = fourier.dft3(got, inverse=True)
    fourier.set_backend("numpy")
    assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()
    assert np.abs(back.real - A).max() < 1e-13
    n = np.prod(shape)
    assert np.isclose((np.abs(ref) ** 2).sum() / n, (A ** 2).sum(), rtol=1e-13)


def test_frequencies_are_centred_set():
    for n in SIZES:
        q = fourier.frequencies(n)
        assert sorted(q) == list(range(-(n - 1) // 2, (n - 1) // 2 + 1))
        assert q[0] == 0
    # even sizes: the listing's range -n/2 .. n/2 - 1 (Appendix C)
    for n in (2, 4, 6, 16):
        q = fourier.frequencies(n)
        assert sorted(q) == list(range(-n // 2, n // 2))
        assert q[0] == 0 and q[n // 2] == -n // 2
    m = fourier.nyquist_mask((4, 3, 6))
    assert m.sum() == 3 * 6 + 4 * 3 - 3 and m[2, 0, 0] and m[0, 1, 3] and not m[1, 1, 1]


@pytest.mark.parametrize("shape", [(5, 7, 9), (31, 31, 31), (3, 11, 5)])
def test_projection_idempotent_symmetric_zero_mean(shape):
    rng = np.random.default_rng(2)
    A = rng.standard_normal((3, 3) + shape)
    B = rng.standard_normal((3, 3) + shape)
    GA, GB = fourier.G(A), fourier.G(B)
    scale = np.abs(GA).max()
    assert np.abs(fourier.G(GA) - GA).max() < 1e-13 * scale
    assert abs((A * GB).sum() - (GA * B).sum()) < 1e-12 * np.abs(A).sum()
    assert np.abs(t.grid_mean(GA)).max() < 1e-14 * scale
    # uniform fields (q = 0 only) are annihilated
    U = t.uniform(rng.standard_normal((3, 3)), shape)
    assert np.abs(fourier.G(U)).max() < 1e-14


def _compatible_field(shape, rng):
    """Zero-mean compatible field A_ij = d phi_i / dX_j of a random periodic
    trigonometric potential: A-hat_ij = i 2 pi xi_j phi-hat_i."""
    phi = rng.standard_normal((3,) + shape)
    phihat = np.fft.fftn(phi, axes=(-3, -2, -1))
    xi = fourier.scaled_frequencies(shape)
    Ahat = 2j * np.pi * np.einsum("i...,j...->ij...", phihat, xi)
    return np.real(np.fft.ifftn(Ahat, axes=(-3, -2, -1)))


@pytest.mark.parametrize("shape", [(5, 7, 9), (15, 15, 15), (1, 9, 5)])
def test_projection_identity_on_compatible_and_curl_free(shape):
    rng = np.random.default_rng(3)
    A = _compatible_field(shape, rng)
    GA = fourier.G(A)
    assert np.abs(GA - A).max() < 1e-12 * np.abs(A).max()
    # rows of the projection of an arbitrary field are curl free: xi x a = 0
    B = rng.standard_normal((3, 3) + shape)
    Chat = np.fft.fftn(fourier.G(B), axes=(-3, -2, -1))
    xi = fourier.scaled_frequencies(shape)
    for i in range(3):
        cr = np.cross(xi, Chat[i], axis=0)
        assert np.abs(cr).max() < 1e-12 * np.abs(Chat).max()


def _matrix_of(op, shape):
    n = int(np.prod(shape))
    M = np.zeros((9 * n, 9 * n))
    for k in range(9 * n):
        e = np.zeros(9 * n)
        e[k] = 1.0
        M[:, k] = op(e.reshape((3, 3) + shape)).reshape(-1)
    return M


def _gradient_matrix(shape):
    """Matrix of u (3n) -> grad u (9n), (grad u)_ij = du_i/dX_j, by spectral
    differentiation of the trigonometric interpolant (no G-hat involved)."""
    n = int(np.prod(shape))
    xi = fourier.scaled_frequencies(shape)
    D = np.zeros((9 * n, 3 * n))
    for k in range(3 * n):
        e = np.zeros(3 * n)
        e[k] = 1.0
        u = e.reshape((3,) + shape)
        uh = np.fft.fftn(u, axes=(-3, -2, -1))
        gh = 2j * np.pi * np.einsum("i...,j...->ij...", uh, xi)
        D[:, k] = np.real(np.fft.ifftn(gh, axes=(-3, -2, -1))).reshape(-1)
    return D


@pytest.mark.parametrize("shape", [(3, 3, 3), (3, 5, 1), (5, 3, 3)])
def test_projection_matrix_equals_least_squares_projector(shape):
    M = _matrix_of(fourier.G, shape)
    D = _gradient_matrix(shape)
    Pd = D @ np.linalg.pinv(D, rcond=1e-10)
    assert np.abs(M - Pd).max() < 1e-12
    n = int(np.prod(shape))
    assert np.linalg.matrix_rank(M, tol=1e-9) == 3 * (n - 1)
    assert np.abs(M - M.T).max() < 1e-13
    assert np.abs(M @ M - M).max() < 1e-12


def test_literal_and_reduced_projection_agree():
    rng = np.random.default_rng(4)
    A = rng.standard_normal((3, 3, 5, 3, 7))
    assert np.abs(fourier.G_literal(A) - fourier.G(A)).max() < 1e-14


# ---- even grids (Appendix C): Nyquist frequencies zeroed ----

def _compatible_field_no_nyquist(shape, rng):
    phi = rng.standard_normal((3,) + shape)
    phihat = np.fft.fftn(phi, axes=(-3, -2, -1))
    phihat[:, fourier.nyquist_mask(shape)] = 0.0
    xi = fourier.scaled_frequencies(shape)
    Ahat = 2j * np.pi * np.einsum("i...,j...->ij...", phihat, xi)
    return np.real(np.fft.ifftn(Ahat, axes=(-3, -2, -1)))


@pytest.mark.parametrize("shape", [(4, 6, 8), (2, 5, 4), (16, 16, 16)])
def test_even_grid_projection(shape):
    rng = np.random.default_rng(8)
    A = rng.standard_normal((3, 3) + shape)
    B = rng.standard_normal((3, 3) + shape)
    GA, GB = fourier.G(A), fourier.G(B)
    scale = np.abs(GA).max()
    assert np.abs(fourier.G(GA) - GA).max() < 1e-13 * scale
    assert abs((A * GB).sum() - (GA * B).sum()) < 1e-12 * np.abs(A).sum()
    assert np.abs(t.grid_mean(GA)).max() < 1e-14 * scale
    # nothing at the Nyquist frequencies; the listing's explicit loop agrees
    GAh = np.fft.fftn(GA, axes=(-3, -2, -1))
    assert np.abs(GAh[:, :, fourier.nyquist_mask(shape)]).max() < 1e-12 * np.abs(GAh).max()
    assert np.abs(fourier.G_literal(A) - GA).max() < 1e-13 * scale
    # compatible fields without Nyquist content are kept
    C = _compatible_field_no_nyquist(shape, rng)
    assert np.abs(fourier.G(C) - C).max() < 1e-12 * np.abs(C).max()


@pytest.mark.parametrize("shape", [(4, 3, 3), (2, 4, 3)])
def test_even_grid_matrix_equals_least_squares_projector(shape):
    """On even grids G is the orthogonal projector onto the gradients of
    trigonometric displacements without Nyquist content."""
    M = _matrix_of(fourier.G, shape)
    n = int(np.prod(shape))
    xi = fourier.scaled_frequencies(shape)
    mask = fourier.nyquist_mask(shape)
    D = np.zeros((9 * n, 3 * n))
    for k in range(3 * n):
        e = np.zeros(3 * n)
        e[k] = 1.0
        uh = np.fft.fftn(e.reshape((3,) + shape), axes=(-3, -2, -1))
        uh[:, mask] = 0.0
        gh = 2j * np.pi * np.einsum("i...,j...->ij...", uh, xi)
        D[:, k] = np.real(np.fft.ifftn(gh, axes=(-3, -2, -1))).reshape(-1)
    Pd = D @ np.linalg.pinv(D, rcond=1e-10)
    assert np.abs(M - Pd).max() < 1e-12
    assert np.linalg.matrix_rank(M, tol=1e-9) == 3 * (n - 1 - int(mask.sum()))
