"""The split iteration (pd_iterate_dual / pd_state_u / pd_iterate_primal) with the data
blocks spread over two shards, both on this GPU in one process: the shards' gridded dual
contributions are summed on the device in place of the all-reduce between GPUs, and
each shard runs the same primal step. The result must match the oracle's single-process
run of Algorithm 1 and the unsplit pd_iterate."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from gpu_util import TOL_IT32, TOL_IT64, make_problem, rel  # noqa: E402
from oracle import pd as PD  # noqa: E402
from paper_1610_08895_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__ as ge
    ge.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_two_shards_match_oracle_and_unsplit_iteration(precision):
    from paper_1610_08895_gb300 import distributed as D
    from paper_1610_08895_gb300.api import Plan, State
    prob, _ = make_problem(128, 30000, 16, 8, (0, 1, 2), 3, uv_kind="radial", blocks="annuli", nannuli=16)
    x0 = synth.start_vector(128, 128, seed=9)
    phi2, psi2 = PD.operator_norms(prob, x0, max_iter=200, tol=1e-8)
    kw = dict(tau=0.49, sigma=1.0 / psi2, varsigma=1.0 / phi2, kappa=1e-3, psi_norm=float(np.sqrt(psi2)), seed=4,
              p_block=[0.5] * 16, p_basis=[0.5] * 3)
    niter = 15
    st_ref, _ = PD.pd_run(prob, niter, **kw)
    cdt = torch.complex64 if precision == "f32" else torch.complex128
    groups = D.shard_blocks(prob.uv, prob.block_of_vis, prob.nblocks, 2)
    shards = []
    for g in groups:
        sh = D.GpuShard(128, 128, prob.uv, prob.block_of_vis, prob.nblocks, g, kw, kernel_width=8,
                        basis_ids=prob.basis_ids, levels=prob.levels, precision=precision)
        sh.set_data(torch.tensor(prob.y[sh.vis], dtype=cdt, device="cuda"), prob.eps)
        shards.append(sh)
    for _ in range(niter):
        for sh in shards:
            sh.dual_step()
        u = shards[0].u_sum_buffer() + shards[1].u_sum_buffer()
        for sh in shards:
            sh.primal_step(u)
    x0_, x1_ = shards[0].x().cpu().numpy(), shards[1].x().cpu().numpy()
    assert np.array_equal(x0_, x1_)                   # the replicated primal update agrees bit for bit
    tol = TOL_IT64 if precision == "f64" else TOL_IT32
    assert rel(x0_, st_ref.x) < tol
    plan = Plan(128, 128, prob.uv, prob.block_of_vis, prob.nblocks, kernel_width=8, basis_ids=prob.basis_ids,
                levels=prob.levels, precision=precision)
    st = State(plan)
    st.pd_state_set_data(torch.tensor(prob.y, dtype=cdt, device="cuda"), prob.eps)
    st.pd_iterate(niter, **kw)
    assert rel(x0_, st.x().cpu().numpy()) < (1e-12 if precision == "f64" else 1e-5)
