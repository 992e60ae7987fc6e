"""G held as a sparse matrix (pd_plan_desc.g_mode = PD_G_CSR): Phi, Phi^H and Algorithm 1
against the oracle and against the plan that evaluates G in the kernels.

The oracle's G is its own dense-footprint interpolation (Sec. 2); the CSR plan must give
the same operator to the working precision, at sizes that span several gridding tiles
with ragged work lists, for every kernel width it supports (J <= 8)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from gpu_util import TOL_IT32, TOL_IT64, TOL_OP32, TOL_OP64, make_problem, rel  # noqa: E402
from oracle import pd as PD  # noqa: E402
from paper_1610_08895_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__ as ge
    ge.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _plan(prob, precision, g_mode, tile=0):
    from paper_1610_08895_gb300.api import Plan
    g = prob.geom
    return Plan(g.nx, g.ny, prob.uv, prob.block_of_vis, prob.nblocks, kernel_width=g.J,
                basis_ids=prob.basis_ids, levels=prob.levels, precision=precision, tile=tile, g_mode=g_mode)


CASES = [
    # n, M, blocks, J, tile
    (16, 300, 4, 4, 0),        # one tile, every tap wraps
    (32, 2000, 4, 2, 0),       # smallest kernel
    (64, 4096, 4, 6, 16),      # 16 tiles of 16
    (64, 5000, 16, 8, 32),     # ragged chunks over 16 tiles
    (128, 20000, 16, 8, 32),   # 64 tiles
]


@pytest.mark.parametrize("precision", ["f32", "f64"])
@pytest.mark.parametrize("case", CASES)
def test_csr_phi_and_adjoint_match_oracle(case, precision):
    n, m, d, J, tile = case
    prob, x_true = make_problem(n, m, d, J, (0,), 1)
    plan = _plan(prob, precision, "csr", tile)
    rdt = torch.float32 if precision == "f32" else torch.float64
    tol = TOL_OP32 if precision == "f32" else TOL_OP64
    y = plan.pd_apply_phi(torch.tensor(x_true, dtype=rdt, device="cuda")).cpu().numpy()
    assert rel(y, prob.phi(x_true)) < tol
    v = synth.uniform_vis(m, seed=5)
    xa = plan.pd_apply_phi_adj(torch.tensor(v, dtype=plan.cplx_dtype, device="cuda")).cpu().numpy()
    assert rel(xa, prob.phi_adj(v)) < tol
    # the same operator as the plan that evaluates the weights in the kernels
    fly = _plan(prob, precision, "on_the_fly", tile)
    y2 = fly.pd_apply_phi(torch.tensor(x_true, dtype=rdt, device="cuda")).cpu().numpy()
    assert rel(y, y2) < (2e-6 if precision == "f32" else 1e-13)


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_csr_batched_apply_and_determinism(precision):
    n, m = 64, 6000
    prob, _ = make_problem(n, m, 9, 8, (0,), 1)
    plan = _plan(prob, precision, "csr", 16)
    rdt = torch.float32 if precision == "f32" else torch.float64
    tol = TOL_OP32 if precision == "f32" else TOL_OP64
    xs = synth.random_images(3, n, n, seed=4)
    y = plan.pd_apply_phi(torch.tensor(xs, dtype=rdt, device="cuda")).cpu().numpy()
    for k in range(3):
        assert rel(y[k], prob.phi(xs[k])) < tol
    vs = synth.uniform_vis(m, seed=3, batch=2)
    vt = torch.tensor(vs, dtype=plan.cplx_dtype, device="cuda")
    xa = plan.pd_apply_phi_adj(vt)
    for k in range(2):
        assert rel(xa[k].cpu().numpy(), prob.phi_adj(vs[k])) < tol
    # fixed summation order: a second application gives the same bits
    assert torch.equal(xa, plan.pd_apply_phi_adj(vt))


def _steps(prob):
    x0 = synth.start_vector(prob.geom.ny, prob.geom.nx, seed=9)
    phi2, psi2 = PD.operator_norms(prob, x0, max_iter=500, tol=1e-8)
    return dict(tau=0.49, sigma=1.0 / psi2, varsigma=1.0 / phi2, kappa=1e-3, psi_norm=float(np.sqrt(psi2)))


@pytest.mark.parametrize("precision,per_block", [("f64", False), ("f32", False), ("f64", True)])
def test_csr_pd_iterations_match_oracle(precision, per_block):
    from paper_1610_08895_gb300.api import State
    # uneven annuli, half the blocks and bases active per iteration
    prob, _ = make_problem(64, 8192, 16, 8, (0, 1, 2), 2, uv_kind="radial", blocks="annuli", nannuli=16)
    kw = _steps(prob)
    args = dict(seed=3, p_block=[0.5] * 16, p_basis=[0.5] * 3, **kw)
    niter = 30
    st_ref, draws = PD.pd_run(prob, niter, **args)
    plan = _plan(prob, precision, "csr")
    st = State(plan)
    st.pd_state_set_data(torch.tensor(prob.y, dtype=plan.cplx_dtype, device="cuda"), prob.eps)
    st.pd_iterate(niter, per_block=per_block, **args)
    rep = st.report()
    assert list(rep["block_active"]) == list(draws[-1][0])
    tol = TOL_IT64 if precision == "f64" else TOL_IT32
    assert rel(st.x().cpu().numpy(), st_ref.x) < tol
    assert rel(st.v().cpu().numpy(), st_ref.v) < tol


def test_csr_needs_narrow_kernel():
    from paper_1610_08895_gb300._binding import PDError
    from paper_1610_08895_gb300.api import Plan
    uv = synth.uv_gaussian(100, seed=1)
    with pytest.raises(PDError):
        Plan(32, 32, uv, np.zeros(100, np.int32), 1, kernel_width=10, g_mode="csr")
