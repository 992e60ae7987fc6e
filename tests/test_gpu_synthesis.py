"""GPU parity of the synthesis formulation (x = Psi alpha, l1 on the coefficients,
positivity as a dual; Sec. 2's synthesis approach with the primal-dual template of
Sec. 3) against the oracle, through pd_synthesis_iterate."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from gpu_util import TOL_IT32, TOL_IT64, make_problem, rel  # noqa: E402
from oracle import pd as PD  # noqa: E402
from oracle import synthesis as SY  # noqa: E402
from paper_1610_08895_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__ as ge
    ge.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


@pytest.mark.parametrize("precision,case", [("f64", "c1"), ("f32", "c1"), ("f32", "annuli")])
def test_synthesis_iterations_match_oracle(precision, case):
    from paper_1610_08895_gb300.api import Plan, State
    if case == "c1":
        prob, _ = make_problem(64, 4096, 4, 4, (0, 1, 2, 3, 4), 3)
        pb = [0.75] * 4
    else:
        prob, _ = make_problem(64, 8192, 16, 8, (0, 1, 2), 2, uv_kind="radial", blocks="annuli", nannuli=16)
        pb = [0.5] * 16
    x0 = synth.start_vector(prob.geom.ny, prob.geom.nx, seed=9)
    phi2, _ = PD.operator_norms(prob, x0, max_iter=500, tol=1e-8)
    kw = dict(tau=0.49, sigma=1.0, varsigma=1.0 / phi2, kappa=1e-3)
    niter = 40
    st_ref, draws = SY.synthesis_run(prob, niter, seed=6, p_block=pb, **kw)
    g = prob.geom
    plan = Plan(g.nx, g.ny, prob.uv, prob.block_of_vis, prob.nblocks, kernel_width=g.J,
                basis_ids=prob.basis_ids, levels=prob.levels, precision=precision)
    st = State(plan)
    st.pd_state_set_data(torch.tensor(prob.y, dtype=plan.cplx_dtype, device="cuda"), prob.eps)
    st.pd_synthesis_iterate(niter, seed=6, p_block=pb, **kw)
    rep = st.report()
    assert rep["t"] == niter
    assert list(rep["block_active"]) == list(draws[-1])
    tol = TOL_IT64 if precision == "f64" else TOL_IT32
    alpha = st.s().cpu().numpy()
    assert rel(alpha, st_ref.alpha) < tol
    assert rel(st.x().cpu().numpy(), st_ref.x(prob)) < tol
    assert rel(st.v().cpu().numpy(), st_ref.v) < tol
    # the l1 step leaves exact zeros, in the same places up to coefficients at the threshold
    z_gpu, z_ref = alpha == 0, st_ref.alpha == 0
    assert np.mean(z_gpu != z_ref) < (1e-12 if precision == "f64" else 1e-3)


def test_synthesis_refuses_graph_and_adaptive():
    from paper_1610_08895_gb300 import _binding as B
    from paper_1610_08895_gb300.api import Plan, State
    prob, _ = make_problem(32, 500, 4, 4, (0, 1), 1)
    g = prob.geom
    plan = Plan(g.nx, g.ny, prob.uv, prob.block_of_vis, 4, kernel_width=4, basis_ids=(0, 1), levels=1,
                precision="f64")
    st = State(plan)
    st.pd_state_set_data(torch.tensor(prob.y, dtype=plan.cplx_dtype, device="cuda"), prob.eps)
    import ctypes
    pb = np.ones(4)
    prm = B.PdParams(tau=0.49, sigma=1.0, varsigma=1e-3, kappa=1e-3, seed=0, p_block=pb.ctypes.data, use_graph=1)
    with pytest.raises(B.PDError):
        B.call("pd_synthesis_iterate", plan.handle, st._h, ctypes.byref(prm), 1, None)
