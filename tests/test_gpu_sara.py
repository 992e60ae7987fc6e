"""GPU parity of the reweighted analysis prior (SARA, Sec. 2): the reweighting rule
pd_sara_weights and Algorithm 1 with per-coefficient weights, against the oracle."""
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


def _plan(prob, precision):
    from paper_1610_08895_gb300.api import Plan
    g = prob.geom
    return Plan(g.nx, g.ny, prob.uv, prob.block_of_vis, prob.nblocks, kernel_width=g.J,
                basis_ids=prob.basis_ids, levels=prob.levels, precision=precision)


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_sara_weights_match_oracle(precision):
    prob, x_true = make_problem(64, 2000, 4, 8, tuple(range(9)), 3)
    plan = _plan(prob, precision)
    rdt = torch.float32 if precision == "f32" else torch.float64
    w = plan.pd_sara_weights(torch.tensor(x_true, dtype=rdt, device="cuda"), 0.02).cpu().numpy()
    w_ref = PD.sara_weights(prob, x_true, 0.02)
    assert rel(w, w_ref) < (TOL_OP32 if precision == "f32" else TOL_OP64)
    assert np.all((w > 0) & (w <= 1))


def _steps(prob):
    x0 = synth.start_vector(prob.geom.ny, prob.geom.nx, seed=9)
    phi2, psi2 = PD.operator_norms(prob, x0, max_iter=500, tol=1e-8)
    return dict(tau=0.49, sigma=1.0 / psi2, varsigma=1.0 / phi2, kappa=1e-3, psi_norm=float(np.sqrt(psi2)))


@pytest.mark.parametrize("precision,use_graph,per_block", [("f64", False, False), ("f32", True, False),
                                                           ("f64", False, True)])
def test_reweighted_iterations_match_oracle(precision, use_graph, per_block):
    from paper_1610_08895_gb300.api import State
    prob, x_true = make_problem(64, 8192, 16, 8, (0, 1, 2, 3), 3)
    kw = _steps(prob)
    args = dict(seed=2, p_block=[0.5] * 16, p_basis=[0.75] * 4, **kw)
    # weights from a rough image (reweighting from the truth would be too kind to the test)
    x_rough = np.clip(x_true + 0.1 * np.random.default_rng(3).normal(size=x_true.shape), 0, None)
    wts = PD.sara_weights(prob, x_rough, 0.01)
    niter = 40
    st_ref, draws = PD.pd_run(prob, niter, weights=wts, **args)
    plan = _plan(prob, precision)
    st = State(plan)
    st.pd_state_set_data(torch.tensor(prob.y, dtype=plan.cplx_dtype, device="cuda"), prob.eps)
    wt = torch.tensor(wts, dtype=plan.real_dtype, device="cuda")
    st.pd_iterate(niter, use_graph=use_graph, per_block=per_block, weights=wt, **args)
    rep = st.report()
    assert list(rep["basis_active"]) == list(draws[-1][1])
    tol = TOL_IT64 if precision == "f64" else TOL_IT32
    assert rel(st.x().cpu().numpy(), st_ref.x) < tol
    assert rel(st.s().cpu().numpy(), st_ref.s) < tol
    # the weights matter: the unweighted run is elsewhere
    st_l1, _ = PD.pd_run(prob, niter, **args)
    assert rel(st_l1.s, st_ref.s) > 100 * tol
