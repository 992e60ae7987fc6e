"""GPU parity of the operators Phi, Phi^H, Psi^H, Psi and the power method against the oracle.

Sizes span several gridding tiles and FFT tiles with ragged work lists; both
precisions. Everything goes through the C ABI via the ctypes binding."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from gpu_util import TOL_OP32, TOL_OP64, make_problem, rel  # noqa: E402
from oracle import measurement as meas  # noqa: E402
from oracle import pd as PD  # noqa: E402
from oracle import wavelets as W  # noqa: E402
from paper_1610_08895_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__ as ge
    ge.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _plan(prob, precision, tile=0):
    from paper_1610_08895_gb300.api import Plan
    g = prob.geom
    return Plan(g.nx, g.ny, prob.uv, prob.block_of_vis, prob.nblocks, kernel_width=g.J,
                basis_ids=prob.basis_ids, levels=prob.levels, precision=precision, tile=tile)


CASES = [
    # n, M, blocks, J, bases, levels, tile
    (16, 300, 4, 4, (0, 1, 2), 2, 0),        # one 32x32 tile, every tap wraps
    (64, 4096, 4, 4, (0, 1, 2, 3, 4), 3, 0),  # C1 shape: 4 tiles
    (64, 5000, 16, 8, (0, 1, 8), 3, 32),      # 16 tiles, ragged chunks
    (256, 65536, 16, 8, tuple(range(9)), 4, 0),  # C2 shape: 64 tiles
]


@pytest.mark.parametrize("precision", ["f32", "f64"])
@pytest.mark.parametrize("case", CASES)
def test_phi_and_adjoint_match_oracle(case, precision):
    n, m, d, J, bases, L, tile = case
    prob, x_true = make_problem(n, m, d, J, bases, L)
    plan = _plan(prob, precision, tile)
    rdt = torch.float32 if precision == "f32" else torch.float64
    x = torch.tensor(x_true, dtype=rdt, device="cuda")
    y = plan.pd_apply_phi(x)
    y_ref = prob.phi(x_true)
    tol = TOL_OP32 if precision == "f32" else TOL_OP64
    assert rel(y.cpu().numpy(), y_ref) < tol
    v = synth.uniform_vis(m, seed=5)
    vt = torch.tensor(v, dtype=plan.cplx_dtype, device="cuda")
    xa = plan.pd_apply_phi_adj(vt)
    xa_ref = prob.phi_adj(v)
    assert rel(xa.cpu().numpy(), xa_ref) < tol
    # adjoint identity on the GPU operators themselves
    lhs = float(np.real(np.vdot(v, y.cpu().numpy().astype(np.complex128))))
    rhs = float(np.dot(x_true.ravel(), xa.cpu().numpy().astype(np.float64).ravel()))
    assert abs(lhs - rhs) <= (1e-5 if precision == "f32" else 1e-11) * np.linalg.norm(v) * np.linalg.norm(
        y_ref) * 10


@pytest.mark.parametrize("precision", ["f32", "f64"])
@pytest.mark.parametrize("nx,ny", [(64, 32), (32, 128), (16, 256)])
def test_phi_rectangular_images(nx, ny, precision):
    """Non-square images: the row and column passes see different lengths and panel counts."""
    from paper_1610_08895_gb300.api import Plan
    m = 3000
    uv = synth.uv_gaussian(m, seed=13)
    plan = Plan(nx, ny, uv, np.zeros(m, np.int32), 1, kernel_width=8, precision=precision)
    geo = meas.Geometry(ny, nx, 8)
    rng = np.random.default_rng(2)
    x0 = rng.uniform(size=(ny, nx))
    rdt = torch.float32 if precision == "f32" else torch.float64
    y = plan.pd_apply_phi(torch.tensor(x0, dtype=rdt, device="cuda"))
    tol = TOL_OP32 if precision == "f32" else TOL_OP64
    assert rel(y.cpu().numpy(), geo.phi(x0, uv)) < tol
    v = rng.normal(size=m) + 1j * rng.normal(size=m)
    xa = plan.pd_apply_phi_adj(torch.tensor(v, dtype=plan.cplx_dtype, device="cuda"))
    assert rel(xa.cpu().numpy(), geo.phi_adj(v, uv)) < tol


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_phi_batched_and_edge_points(precision):
    n = 32
    uv = np.concatenate([synth.uv_gaussian(500, seed=9),
                         np.array([[-np.pi, -np.pi], [np.pi - 1e-12, 0.0], [0.0, np.pi - 1e-7], [0.0, 0.0]])])
    blk = (np.arange(len(uv)) % 3).astype(np.int32)
    prob = PD.Problem(meas.Geometry(n, n, 8), uv, blk, 3, [0], 1)
    plan = _plan(prob, precision)
    xs = synth.random_images(3, n, n, seed=4)
    rdt = torch.float32 if precision == "f32" else torch.float64
    y = plan.pd_apply_phi(torch.tensor(xs, dtype=rdt, device="cuda")).cpu().numpy()
    tol = TOL_OP32 if precision == "f32" else TOL_OP64
    for k in range(3):
        assert rel(y[k], prob.phi(xs[k])) < tol
    vs = synth.uniform_vis(len(uv), seed=3, batch=2)
    xa = plan.pd_apply_phi_adj(torch.tensor(vs, dtype=plan.cplx_dtype, device="cuda")).cpu().numpy()
    for k in range(2):
        assert rel(xa[k], prob.phi_adj(vs[k])) < tol


@pytest.mark.parametrize("precision", ["f32", "f64"])
@pytest.mark.parametrize("n,levels,bases", [(16, 3, tuple(range(9))), (64, 3, (0, 1, 2, 3, 4)),
                                            (256, 4, tuple(range(9))), (32, 1, (8, 0, 3))])
def test_psi_and_adjoint_match_oracle(n, levels, bases, precision):
    rng = np.random.default_rng(n + levels)
    x = rng.normal(size=(n, n))
    prob = PD.Problem(meas.Geometry(n, n, 4), np.zeros((1, 2)), np.zeros(1, np.int32), 1, list(bases), levels)
    plan = _plan(prob, precision)
    rdt = torch.float32 if precision == "f32" else torch.float64
    c = plan.pd_apply_psi_adj(torch.tensor(x, dtype=rdt, device="cuda")).cpu().numpy()
    c_ref = W.psi_adj(x, list(bases), levels)
    tol = TOL_OP32 if precision == "f32" else TOL_OP64
    assert rel(c, c_ref) < tol
    s = rng.normal(size=(len(bases), n, n))
    xs = plan.pd_apply_psi(torch.tensor(s, dtype=rdt, device="cuda")).cpu().numpy()
    assert rel(xs, W.psi(s, list(bases), levels)) < tol
    # perfect reconstruction through the GPU pair
    back = plan.pd_apply_psi(torch.tensor(c, dtype=rdt, device="cuda")).cpu().numpy()
    assert rel(back, x) < tol


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_operator_norms_match_oracle_power_method(precision):
    prob, _ = make_problem(64, 4096, 4, 4, (0, 1, 2), 2)
    plan = _plan(prob, precision)
    x0 = synth.start_vector(64, 64, seed=9)
    rdt = torch.float32 if precision == "f32" else torch.float64
    phi2, psi2, it = plan.pd_operator_norms(torch.tensor(x0, dtype=rdt, device="cuda"), max_iter=2000, tol=1e-9)
    phi2_ref, psi2_ref = PD.operator_norms(prob, x0, max_iter=2000, tol=1e-12)
    assert phi2 == pytest.approx(phi2_ref, rel=1e-5 if precision == "f32" else 1e-8)
    assert psi2 == pytest.approx(psi2_ref, rel=1e-5 if precision == "f32" else 1e-12)


def test_plan_rejects_bad_descriptions():
    from paper_1610_08895_gb300._binding import PDError
    from paper_1610_08895_gb300.api import Plan
    uv = synth.uv_gaussian(10, seed=1)
    blk = np.zeros(10, np.int32)
    with pytest.raises(PDError):
        Plan(48, 32, uv, blk, 1)                       # not a power of two
    with pytest.raises(PDError):
        Plan(32, 32, uv, blk, 1, kernel_width=5)        # odd kernel
    bad = uv.copy()
    bad[0, 0] = np.pi
    with pytest.raises(PDError):
        Plan(32, 32, bad, blk, 1)                       # outside [-pi, pi)
    with pytest.raises(PDError):
        Plan(32, 32, uv, blk + 1, 1)                    # block index out of range
    with pytest.raises(PDError):
        Plan(32, 32, uv, blk, 1, basis_ids=(9,))        # unknown basis
