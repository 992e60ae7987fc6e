"""Pins of the oracle's measurement operator Phi = G F Z (Sec. 2) against things other than itself."""
import numpy as np
import pytest
from scipy.integrate import quad

from oracle import measurement as meas
from paper_1610_08895_gb300 import synth


def nudft_direct(x, uv):
    """Brute-force non-uniform DFT of the discretised model (Sec. 2, no DDEs), written as loops."""
    ny, nx = x.shape
    out = np.zeros(len(uv), dtype=np.complex128)
    for m, (u, v) in enumerate(uv):
        acc = 0.0 + 0.0j
        for iy in range(ny):
            for ix in range(nx):
                acc += x[iy, ix] * np.exp(-1j * (u * (ix - nx // 2) + v * (iy - ny // 2)))
        out[m] = acc
    return out


def i0_series(z):
    """Modified Bessel I0 by its power series sum (z/2)^(2k) / (k!)^2."""
    total, term, k = 1.0, 1.0, 0
    while term > 1e-18 * total:
        k += 1
        term *= (z / 2.0) ** 2 / (k * k)
        total += term
    return total


@pytest.mark.parametrize("J", [4, 8])
def test_kernel_values_against_series(J):
    beta = meas.kb_beta_default(J)
    t = np.linspace(-J / 2, J / 2, 37)
    ref = np.array([i0_series(beta * np.sqrt(max(0.0, 1 - (2 * s / J) ** 2))) for s in t])
    got = meas.kb_kernel(t, J, beta)
    assert np.allclose(got, ref, rtol=1e-13, atol=0)
    assert meas.kb_kernel(np.array([J / 2 + 1e-9, -J]), J, beta).tolist() == [0.0, 0.0]


def test_default_beta_values():
    # Beatty et al. rule at alpha = 2: beta = pi sqrt(0.5625 J^2 - 0.8)
    assert meas.kb_beta_default(4) == pytest.approx(np.pi * np.sqrt(8.2), rel=1e-15)
    assert meas.kb_beta_default(8) == pytest.approx(np.pi * np.sqrt(35.2), rel=1e-15)


@pytest.mark.parametrize("J", [4, 6, 8])
def test_kernel_fourier_closed_form_against_quadrature(J):
    beta = meas.kb_beta_default(J)
    for xi in [0.0, 0.05, 0.125, 0.25, 0.4, 1.7]:
        re, _ = quad(lambda t: meas.kb_kernel(np.array([t]), J, beta)[0] * np.cos(2 * np.pi * xi * t),
                     -J / 2, J / 2, limit=400, epsabs=0, epsrel=1e-13)
        got = meas.kb_fourier(np.array([xi]), J, beta)[0]
        assert got == pytest.approx(re, rel=1e-9, abs=1e-9 * abs(meas.kb_fourier(np.array([0.0]), J, beta)[0]))


def test_fft_step_against_brute_force_dft():
    rng = np.random.default_rng(1)
    g = rng.normal(size=(8, 16)) + 1j * rng.normal(size=(8, 16))
    Ky, Kx = g.shape
    ref = np.zeros_like(g)
    for ky in range(Ky):
        for kx in range(Kx):
            for my in range(Ky):
                for mx in range(Kx):
                    ref[ky, kx] += g[my, mx] * np.exp(-2j * np.pi * (ky * my / Ky + kx * mx / Kx))
    assert np.allclose(meas.Geometry.fft(g), ref, rtol=0, atol=1e-12)
    # F^H is the conjugate transpose: <F a, b> = <a, F^H b>
    b = rng.normal(size=g.shape) + 1j * rng.normal(size=g.shape)
    lhs = np.vdot(b, meas.Geometry.fft(g))
    rhs = np.vdot(meas.Geometry.fft_adj(b), g)
    assert abs(lhs - rhs) <= 1e-11 * abs(lhs)


def test_zpad_places_centre_pixel_at_origin():
    geo = meas.Geometry(8, 16, 4)
    x = np.zeros((8, 16))
    x[4, 8] = 1.0
    g = geo.zpad(x)
    assert g[0, 0] == pytest.approx(geo.cy[4] * geo.cx[8])
    assert np.count_nonzero(g) == 1
    x[0, 0] = 2.0            # top-left pixel sits at centred coordinates (-4, -8)
    g = geo.zpad(x)
    assert g[16 - 4, 32 - 8] == pytest.approx(2.0 * geo.cy[0] * geo.cx[0])


def test_centred_point_source_gives_unit_visibilities():
    # the continuous model of a point at the phase centre has y(u) = 1 for every u
    geo = meas.Geometry(32, 32, 8)
    x = np.zeros((32, 32))
    x[16, 16] = 1.0
    uv = synth.uv_gaussian(300, seed=3)
    y = geo.phi(x, uv)
    assert np.max(np.abs(y - 1.0)) < 1e-4


@pytest.mark.parametrize("n", [16])
def test_phi_against_direct_nudft_error_falls_with_kernel_width(n):
    x = synth.test_image(n, seed=2)
    uv = synth.uv_gaussian(200, seed=4)
    ref = nudft_direct(x, uv)
    errs = {}
    for J in (4, 6, 8):
        geo = meas.Geometry(n, n, J)
        y = geo.phi(x, uv)
        errs[J] = np.linalg.norm(y - ref) / np.linalg.norm(ref)
    assert errs[4] > errs[6] > errs[8]
    # frozen from the first measurement (J=4: 4.6e-4, J=6: 3.8e-6, J=8: 3.1e-8), 3x margin
    assert errs[4] < 1.5e-3
    assert errs[6] < 1.2e-5
    assert errs[8] < 1e-7


def test_phi_against_direct_nudft_rectangular_and_band_edge():
    rng = np.random.default_rng(7)
    x = rng.uniform(0, 1, size=(8, 16))
    uv = np.concatenate([synth.uv_gaussian(50, seed=5),
                         np.array([[-np.pi, -np.pi], [np.pi - 1e-12, 0.0], [0.0, np.pi - 1e-9]])])
    geo = meas.Geometry(8, 16, 8)
    ref = nudft_direct(x, uv)
    y = geo.phi(x, uv)
    assert np.linalg.norm(y - ref) / np.linalg.norm(ref) < 1e-5


@pytest.mark.parametrize("J,shape", [(4, (16, 16)), (8, (8, 16)), (8, (32, 32))])
def test_phi_adjoint_identity(J, shape):
    rng = np.random.default_rng(11)
    geo = meas.Geometry(shape[0], shape[1], J)
    uv = synth.uv_gaussian(150, seed=6)
    x = rng.normal(size=shape)
    y = rng.normal(size=150) + 1j * rng.normal(size=150)
    lhs = np.real(np.vdot(y, geo.phi(x, uv)))      # Re <Phi x, y>
    rhs = np.dot(x.ravel(), geo.phi_adj(y, uv).ravel())
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0) * 10


def test_grid_is_transpose_of_degrid_including_wrap():
    rng = np.random.default_rng(3)
    geo = meas.Geometry(8, 8, 8)       # 16x16 grid, 8x8 taps: every point wraps
    uv = np.array([[-np.pi, -np.pi], [3.0, 3.1], [0.1, -0.2], [-3.1, 2.9]])
    b = rng.normal(size=(16, 16)) + 1j * rng.normal(size=(16, 16))
    v = rng.normal(size=4) + 1j * rng.normal(size=4)
    lhs = np.vdot(v, geo.degrid(b, uv))
    rhs = np.vdot(geo.grid(v, uv), b)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    # brute-force dense G on this tiny case, entry by entry from the kernel definition
    Gd = np.zeros((4, 256))
    for m, (u, vv) in enumerate(uv):
        gx, gy = u * 16 / (2 * np.pi), vv * 16 / (2 * np.pi)
        for ky in range(-20, 36):
            for kx in range(-20, 36):
                w = meas.kb_kernel(np.array([gx - kx]), 8, geo.beta)[0] * \
                    meas.kb_kernel(np.array([gy - ky]), 8, geo.beta)[0]
                if w and (np.floor(gx) - 3 <= kx <= np.floor(gx) + 4) and (np.floor(gy) - 3 <= ky <= np.floor(gy) + 4):
                    Gd[m, (ky % 16) * 16 + (kx % 16)] += w
    assert np.allclose(geo.degrid(b, uv), Gd @ b.ravel(), rtol=1e-13)


def test_adjoint_at_pixels_equals_full_adjoint():
    rng = np.random.default_rng(12)
    geo = meas.Geometry(16, 32, 8)
    uv = synth.uv_gaussian(400, seed=8)
    y = rng.normal(size=400) + 1j * rng.normal(size=400)
    full = geo.phi_adj(y, uv)
    pix = [(0, 0), (7, 31), (15, 3), (8, 16), (3, 29)]
    got = geo.phi_adj_at(y, uv, pix)
    assert np.allclose(got, [full[iy, ix] for iy, ix in pix], rtol=1e-11, atol=1e-11 * np.abs(full).max())


def test_uv_coverage_with_holes():
    # Sec. 5: holes cut predominantly in the high frequencies (inverse Gaussian profile)
    from paper_1610_08895_gb300 import synth
    uv, holes = synth.uv_gaussian_holes(20000, seed=3, nholes=40)
    assert uv.shape == (20000, 2) and np.all((uv >= -np.pi) & (uv < np.pi))
    d2 = (uv[:, None, 0] - holes[None, :, 0]) ** 2 + (uv[:, None, 1] - holes[None, :, 1]) ** 2
    assert np.all(d2 >= holes[None, :, 2] ** 2)                      # no point inside a hole
    r = np.hypot(holes[:, 0], holes[:, 1])
    r_unif = np.hypot(*np.random.default_rng(0).uniform(-np.pi, np.pi, (100000, 2)).T)
    assert np.mean(r) > np.mean(r_unif)                             # centres lean to high frequencies
    uv2, holes2 = synth.uv_gaussian_holes(20000, seed=3, nholes=40)
    assert np.array_equal(uv, uv2) and np.array_equal(holes, holes2)
