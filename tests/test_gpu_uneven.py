"""GPU against the oracle on uneven blocks drawn with a uniform probability: radially
decaying coverage in 64 equal-width annuli (the inner annuli hold few points, the outer
many), every block drawn with p = 0.25, all nine bases, 300 iterations. This is the
configuration in which the synthetic convergence study saw the SNR of the GPU path fall
back; the oracle decides whether that is the method or the kernels."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from gpu_util import TOL_IT32, make_problem, rel  # noqa: E402
from oracle import experiment as EX  # noqa: E402
from oracle import pd as PD  # noqa: E402
from paper_1610_08895_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu

NITER = 300
CHECK = (100, 200, 300)


@pytest.fixture(scope="module")
def oracle_run():
    import __graft_entry__ as ge
    ge.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    prob, x_true = make_problem(128, 65536, 64, 8, tuple(range(9)), 4, uv_kind="radial", blocks="annuli",
                                nannuli=64)
    x0 = synth.start_vector(128, 128, seed=9)
    phi2, psi2 = PD.operator_norms(prob, x0, max_iter=500, tol=1e-8)
    kw = dict(tau=0.49, sigma=1.0 / psi2, varsigma=1.0 / phi2, kappa=1e-3, psi_norm=float(np.sqrt(psi2)), seed=0,
              p_block=[0.25] * 64, p_basis=[1.0] * 9)
    st = PD.PDState(prob)
    snaps, draws = {}, []
    for t in range(1, NITER + 1):
        draws.append(PD.pd_iteration(prob, st, **kw))
        if t in CHECK:
            snaps[t] = st.x.copy()
    return prob, x_true, kw, snaps, draws, st


@pytest.mark.parametrize("use_graph", [False, True])
def test_uniform_p_on_uneven_annuli_matches_oracle(oracle_run, use_graph):
    from paper_1610_08895_gb300.api import Plan, State
    prob, x_true, kw, snaps, draws, st_ref = oracle_run
    g = prob.geom
    plan = Plan(g.nx, g.ny, prob.uv, prob.block_of_vis, prob.nblocks, kernel_width=g.J, basis_ids=prob.basis_ids,
                levels=prob.levels, precision="f32")
    st = State(plan)
    st.pd_state_set_data(torch.tensor(prob.y, dtype=torch.complex64, device="cuda"), prob.eps)
    done = 0
    for t in CHECK:
        st.pd_iterate(t - done, use_graph=use_graph, **kw)
        done = t
        rep = st.report()
        assert list(rep["block_active"]) == list(draws[t - 1][0])
        x = st.x().cpu().numpy().astype(np.float64)
        err = rel(x, snaps[t])
        snr_gpu, snr_ref = EX.snr_db(x_true, x), EX.snr_db(x_true, snaps[t])
        print(f"t={t} rel={err:.2e} SNR gpu {snr_gpu:.2f} dB oracle {snr_ref:.2f} dB")
        assert err < TOL_IT32
    assert rel(st.v().cpu().numpy(), st_ref.v) < TOL_IT32
    assert rel(st.s().cpu().numpy(), st_ref.s) < TOL_IT32
    st.close()
    plan.close()
