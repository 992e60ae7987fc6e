"""Pins of the oracle's sparsity dictionary Psi (Sec. 3: a collection of b orthonormal bases)."""
import numpy as np
import pytest

from oracle import wavelets as W
from oracle import pd as PD


@pytest.mark.parametrize("p", range(1, 9))
def test_daubechies_filter_identities(p):
    h = W.daubechies_lowpass(p)
    L = len(h)
    assert L == 2 * p
    assert h.sum() == pytest.approx(np.sqrt(2.0), abs=1e-13)
    # double-shift orthonormality: sum_k h_k h_{k+2m} = delta_m
    for m in range(0, p):
        acc = sum(h[k] * h[k + 2 * m] for k in range(L - 2 * m))
        assert acc == pytest.approx(1.0 if m == 0 else 0.0, abs=1e-12)
    # p vanishing moments of the high-pass filter: sum_k (-1)^k k^q h_k = 0 for q < p
    k = np.arange(L, dtype=np.float64)
    for q in range(p):
        mom = np.sum((-1.0) ** k * k ** q * h)
        assert abs(mom) <= 1e-9 * max(1.0, np.sum(k ** q * np.abs(h)))
    # minimum phase: sum_k h_k z^(L-1-k) = (z + 1)^p Q(z) with every zero of Q inside the unit circle
    quot, rem = np.polydiv(h, np.poly(-np.ones(p)))
    assert np.max(np.abs(rem)) < 1e-12
    if p > 1:
        assert np.all(np.abs(np.roots(quot)) < 1.0)


def test_haar_and_db2_closed_forms():
    assert np.allclose(W.daubechies_lowpass(1), [1 / np.sqrt(2), 1 / np.sqrt(2)], atol=1e-16)
    s3 = np.sqrt(3.0)
    db2 = np.array([1 + s3, 3 + s3, 3 - s3, 1 - s3]) / (4 * np.sqrt(2.0))
    assert np.allclose(W.daubechies_lowpass(2), db2, atol=1e-15)


def test_haar_2d_one_level_closed_form():
    x = np.array([[1.0, 2.0], [3.0, 5.0]])
    c = W.dwt2(x, W.daubechies_lowpass(1), 1)
    # rows then columns of the orthonormal Haar pair
    assert c[0, 0] == pytest.approx((1 + 2 + 3 + 5) / 2)
    assert c[0, 1] == pytest.approx(((1 - 2) + (3 - 5)) / 2)   # row detail, column approx
    assert c[1, 0] == pytest.approx(((1 + 2) - (3 + 5)) / 2)   # row approx, column detail
    assert c[1, 1] == pytest.approx(((1 - 2) - (3 - 5)) / 2)


def test_constant_image_haar_packs_into_coarsest_corner():
    x = np.full((16, 16), 3.0)
    c = W.dwt2(x, W.daubechies_lowpass(1), 3)
    assert np.allclose(c[:2, :2], 3.0 * 2 ** 3)
    c[:2, :2] = 0
    assert np.allclose(c, 0.0, atol=1e-13)


@pytest.mark.parametrize("p", [1, 2, 4, 8])
def test_polynomial_interior_detail_vanishes(p):
    # away from the periodic seam, the detail of a polynomial of degree < p is zero
    m = 256
    i = np.arange(m, dtype=np.float64) / m
    coef = np.random.default_rng(p).normal(size=p)
    x = np.tile(sum(coef[q] * i ** q for q in range(p)), (4, 1))
    h = W.daubechies_lowpass(p)
    d = W.analysis_1d(x, h, axis=1)[:, m // 2:]
    interior = d[:, : m // 2 - len(h)]
    assert np.max(np.abs(interior)) < 1e-10 * np.max(np.abs(x))
    # and the detail of a degree-p polynomial is not (the moment count is exact)
    x2 = np.tile((np.arange(m) / 16.0) ** p, (4, 1))
    d2 = W.analysis_1d(x2, h, axis=1)[:, m // 2:]
    assert np.max(np.abs(d2[:, : m // 2 - len(h)])) > 1e-6 * np.max(np.abs(x2[:, : m - len(h)])) * 16.0 ** -p


@pytest.mark.parametrize("basis", range(0, 9))
@pytest.mark.parametrize("shape,levels", [((32, 32), 3), ((16, 32), 2), ((16, 16), 3)])
def test_perfect_reconstruction_and_parseval(basis, shape, levels):
    # (16,16) at 3 levels leaves a 4x4 coarsest band: db3..db8 wrap more than once
    rng = np.random.default_rng(basis * 7 + levels)
    x = rng.normal(size=shape)
    c = W.psi_j_adj(x, basis, levels)
    assert np.linalg.norm(c) == pytest.approx(np.linalg.norm(x), rel=1e-12)
    assert np.allclose(W.psi_j(c, basis, levels), x, atol=1e-12)
    # the analysis is also a left inverse of the synthesis (square orthogonal map)
    s = rng.normal(size=shape)
    assert np.allclose(W.psi_j_adj(W.psi_j(s, basis, levels), basis, levels), s, atol=1e-12)


def test_psi_collection_adjoint_and_unit_norm():
    rng = np.random.default_rng(5)
    ids = list(range(9))
    x = rng.normal(size=(32, 32))
    s = rng.normal(size=(9, 32, 32))
    lhs = np.sum(W.psi_adj(x, ids, 2) * s)
    rhs = np.sum(x * W.psi(s, ids, 2))
    assert lhs == pytest.approx(rhs, rel=1e-12)
    # Psi Psi^H = I, so the power method gives ||Psi||_S^2 = 1
    assert np.allclose(W.psi(W.psi_adj(x, ids, 2), ids, 2), x, atol=1e-12)
    lam, _ = PD.power_method(lambda z: W.psi(W.psi_adj(z, ids, 2), ids, 2), x, tol=1e-14)
    assert lam == pytest.approx(1.0, rel=1e-12)


def test_dirac_basis_is_identity():
    x = np.random.default_rng(0).normal(size=(8, 8))
    assert np.array_equal(W.psi_j_adj(x, 0, 3), x)
    assert np.array_equal(W.psi_j(x, 0, 3), x)
