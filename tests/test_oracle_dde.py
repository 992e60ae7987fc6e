"""Pins of the oracle's DDE-aware G (Sec. 2: G models compact-support DDEs as a
convolution in the Fourier domain, besides interpolating) against things other than
itself: the identity DDE, the adjoint identity, the DFT shift theorem and a
brute-force non-uniform DFT of the DDE-modulated image."""
import numpy as np
import pytest

from oracle import measurement as meas
from oracle import pd as PD
from paper_1610_08895_gb300 import synth


def random_dde(m, d, seed):
    rng = np.random.default_rng(seed)
    k = 0.2 * (rng.normal(size=(m, d, d)) + 1j * rng.normal(size=(m, d, d)))
    k[:, d // 2, d // 2] += 1.0                  # near-identity kernels, like smooth gains
    return k


def test_identity_dde_is_plain_interpolation():
    geo = meas.Geometry(16, 16, 6)
    uv = synth.uv_gaussian(300, seed=1)
    rng = np.random.default_rng(0)
    grid = rng.normal(size=(32, 32)) + 1j * rng.normal(size=(32, 32))
    v = rng.normal(size=300) + 1j * rng.normal(size=300)
    for d in (1, 3):
        dde = np.zeros((300, d, d), dtype=np.complex128)
        dde[:, d // 2, d // 2] = 1.0
        assert np.array_equal(geo.degrid_dde(grid, uv, dde), geo.degrid(grid, uv))
        assert np.array_equal(geo.grid_dde(v, uv, dde), geo.grid(v, uv))


@pytest.mark.parametrize("J,d", [(4, 3), (6, 3), (4, 5)])
def test_dde_adjoint_identity(J, d):
    geo = meas.Geometry(16, 16, J)
    uv = synth.uv_gaussian(200, seed=2)
    dde = random_dde(200, d, seed=3)
    rng = np.random.default_rng(4)
    b = rng.normal(size=(32, 32)) + 1j * rng.normal(size=(32, 32))
    v = rng.normal(size=200) + 1j * rng.normal(size=200)
    lhs = np.vdot(v, geo.degrid_dde(b, uv, dde))          # <v, G b>
    rhs = np.vdot(geo.grid_dde(v, uv, dde), b)            # <G^H v, b>
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_shift_dde_is_a_linear_phase_on_the_image():
    # D = delta at grid offset (ky, kx) = (0, 1): by the DFT shift theorem, Phi_D x equals
    # Phi applied to x exp(-2 pi i (ix - nx/2) / Kx), to rounding -- this fixes which axis
    # the offsets run along and the sign of the convolution.
    geo = meas.Geometry(16, 16, 6)
    uv = synth.uv_gaussian(150, seed=5)
    x = synth.test_image(16, seed=6)
    dde = np.zeros((150, 3, 3), dtype=np.complex128)
    dde[:, 1, 2] = 1.0
    y_dde = geo.degrid_dde(geo.fft(geo.zpad(x)), uv, dde)
    ix = np.arange(16) - 8
    xm = x * np.exp(-2j * np.pi * ix / 32)[None, :]
    y_ref = geo.degrid(geo.fft(geo.zpad(xm)), uv)            # Z and F act on the complex image
    assert np.linalg.norm(y_dde - y_ref) <= 1e-12 * np.linalg.norm(y_ref)


def nudft_modulated(x, uv, dde, Ky, Kx):
    """sum_n x_n d_m(n) exp(-i (u (ix - nx/2) + v (iy - ny/2))) with the image-domain DDE
    d_m(n) = sum_k D_m[k] exp(-2 pi i (ky (iy - ny/2) / Ky + kx (ix - nx/2) / Kx)), by loops."""
    ny, nx = x.shape
    d = dde.shape[1]
    h = (d - 1) // 2
    out = np.zeros(len(uv), dtype=np.complex128)
    for m, (u, v) in enumerate(uv):
        acc = 0.0 + 0.0j
        for iy in range(ny):
            ly = iy - ny // 2
            for ixx in range(nx):
                lx = ixx - nx // 2
                dm = 0.0 + 0.0j
                for a in range(d):
                    for b in range(d):
                        dm += dde[m, a, b] * np.exp(-2j * np.pi * ((a - h) * ly / Ky + (b - h) * lx / Kx))
                acc += x[iy, ixx] * dm * np.exp(-1j * (u * lx + v * ly))
        out[m] = acc
    return out


@pytest.mark.parametrize("J,d,tol", [(6, 3, 1e-5), (8, 1, 1e-7)])   # measured 3.5e-6, 3.0e-8: the plain J accuracy
def test_dde_phi_against_modulated_nudft(J, d, tol):
    geo = meas.Geometry(16, 16, J)
    uv = synth.uv_gaussian(60, seed=7)
    x = synth.test_image(16, seed=8)
    dde = random_dde(60, d, seed=9)
    prob = PD.Problem(geo, uv, np.zeros(60, np.int32), 1, [0], 1, dde=dde)
    y = prob.phi(x)
    ref = nudft_modulated(x, uv, dde, 32, 32)
    assert np.linalg.norm(y - ref) / np.linalg.norm(ref) < tol


def test_dde_problem_adjoint_and_blocks():
    geo = meas.Geometry(16, 16, 4)
    uv = synth.uv_gaussian(120, seed=10)
    dde = random_dde(120, 3, seed=11)
    blk = (np.arange(120) % 3).astype(np.int32)
    prob = PD.Problem(geo, uv, blk, 3, [0], 1, dde=dde)
    rng = np.random.default_rng(12)
    x = rng.normal(size=(16, 16))
    v = rng.normal(size=120) + 1j * rng.normal(size=120)
    # Re <v, Phi x> = <Phi^H v, x> for the real-image adjoint
    assert abs(np.real(np.vdot(v, prob.phi(x))) - np.dot(prob.phi_adj(v).ravel(), x.ravel())) < 1e-11 * np.abs(v).sum()
    # block rows are the rows of the whole operator
    b = geo.fft(geo.zpad(x))
    full = prob.degrid_rows(b, np.arange(120))
    for i in range(3):
        ix = prob.block_index[i]
        assert np.allclose(prob.degrid_rows(b, ix), full[ix], rtol=1e-14, atol=0)
