"""GPU parity of Algorithm 1 (pd_iterate) against the oracle's step-by-step PD-R run."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from gpu_util import TOL_IT32, TOL_IT64, make_problem, rel  # noqa: E402
from oracle import pd as PD  # noqa: E402
from oracle import philox as PH  # noqa: E402
from paper_1610_08895_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__ as ge
    ge.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _setup(prob, precision, tile=0):
    from paper_1610_08895_gb300.api import Plan, State
    g = prob.geom
    plan = Plan(g.nx, g.ny, prob.uv, prob.block_of_vis, prob.nblocks, kernel_width=g.J,
                basis_ids=prob.basis_ids, levels=prob.levels, precision=precision, tile=tile)
    st = State(plan)
    st.pd_state_set_data(torch.tensor(prob.y, dtype=plan.cplx_dtype, device="cuda"), prob.eps)
    return plan, st


def _steps(prob):
    x0 = synth.start_vector(prob.geom.ny, prob.geom.nx, seed=9)
    phi2, psi2 = PD.operator_norms(prob, x0, max_iter=500, tol=1e-8)
    return dict(tau=0.49, sigma=1.0 / psi2, varsigma=1.0 / phi2, kappa=1e-3, psi_norm=float(np.sqrt(psi2)))


def test_deterministic_pd_fp64_config1_shape():
    # 64x64 image, 128x128 grid, M = 4096, 4 equal blocks, 4x4 kernel, Dirac + db1-db4, 3 levels, p = 1
    prob, _ = make_problem(64, 4096, 4, 4, (0, 1, 2, 3, 4), 3)
    kw = _steps(prob)
    niter = 200
    st_ref, _ = PD.pd_run(prob, niter, seed=0, p_block=[1.0] * 4, p_basis=[1.0] * 5, **kw)
    plan, st = _setup(prob, "f64")
    st.pd_iterate(niter, seed=0, p_block=[1.0] * 4, p_basis=[1.0] * 5, **kw)
    x = st.x().cpu().numpy()
    assert rel(x, st_ref.x) < TOL_IT64
    assert rel(st.s().cpu().numpy(), st_ref.s) < TOL_IT64
    assert rel(st.v().cpu().numpy(), st_ref.v) < TOL_IT64
    rep = st.report()
    assert rep["t"] == niter
    assert rep["dx2"] >= 0 and rep["x2"] == pytest.approx(np.sum(st_ref.x ** 2), rel=1e-9)


@pytest.mark.parametrize("use_graph", [False, True])
def test_randomised_pd_fp32_config2_shape(use_graph):
    # 256x256, 512x512 grid, M = 65536, 16 blocks p = 0.5, 9 bases p = 0.5, 4 levels, 8x8 kernel
    prob, _ = make_problem(256, 65536, 16, 8, tuple(range(9)), 4)
    kw = _steps(prob)
    niter = 40
    pb, ps = [0.5] * 16, [0.5] * 9
    st_ref, draws = PD.pd_run(prob, niter, seed=0, p_block=pb, p_basis=ps, **kw)
    plan, st = _setup(prob, "f32")
    st.pd_iterate(niter, seed=0, p_block=pb, p_basis=ps, use_graph=use_graph, **kw)
    rep = st.report()
    assert list(rep["block_active"]) == list(draws[-1][0])      # same seeded draws
    assert list(rep["basis_active"]) == list(draws[-1][1])
    assert rel(st.x().cpu().numpy(), st_ref.x) < TOL_IT32
    assert rel(st.v().cpu().numpy(), st_ref.v) < TOL_IT32


def test_adaptive_probabilities_uneven_blocks():
    # radially decaying coverage split in annuli (uneven blocks), probabilities by eq. prob-choice
    prob, _ = make_problem(64, 16384, 16, 8, (0, 1, 2), 2, uv_kind="radial", blocks="annuli", nannuli=16)
    kw = _steps(prob)
    ad = {"n": 4.0, "p_min": 0.05, "p_max": 0.5}
    niter = 30
    st_ref, draws = PD.pd_run(prob, niter, seed=3, p_block=None, p_basis=[1.0] * 3, adaptive=ad, **kw)
    plan, st = _setup(prob, "f32")
    st.pd_iterate(niter, seed=3, p_basis=[1.0] * 3, adaptive=ad, **kw)
    rep = st.report()
    assert list(rep["block_active"]) == list(draws[-1][0])
    assert rel(st.x().cpu().numpy(), st_ref.x) < TOL_IT32
    assert np.allclose(rep["res_norm"], st_ref.res_norm, rtol=1e-4)
    assert rep["p_block"].sum() == pytest.approx(4.0, rel=1e-9)


def test_checkpoint_resume_matches_uninterrupted_run():
    prob, _ = make_problem(64, 8192, 4, 8, (0, 1, 2), 2)
    kw = _steps(prob)
    args = dict(seed=7, p_block=[0.5] * 4, p_basis=[0.5] * 3, **kw)
    plan, st = _setup(prob, "f64")
    st.pd_iterate(10, **args)
    buf = st.save()
    st.pd_iterate(10, **args)
    x_full = st.x().cpu().numpy()
    from paper_1610_08895_gb300.api import State
    st2 = State(plan)
    st2.load(buf)
    st2.pd_iterate(10, **args)
    assert st2.report()["t"] == 20
    assert rel(st2.x().cpu().numpy(), x_full) < 1e-12


def test_draws_match_oracle_philox_every_iteration():
    prob, _ = make_problem(32, 2000, 9, 4, (0, 1), 1)
    kw = _steps(prob)
    plan, st = _setup(prob, "f32")
    pb = [0.3] * 9
    ps = [0.6, 0.6]
    for t in range(1, 16):
        st.pd_iterate(1, seed=11, p_block=pb, p_basis=ps, **kw)
        rep = st.report()
        assert list(rep["block_active"]) == PH.active_set(11, t, 0, pb)
        assert list(rep["basis_active"]) == PH.active_set(11, t, 1, ps)


def test_tile_autotuner_picks_a_working_tile():
    from paper_1610_08895_gb300.api import autotune_tile
    prob, _ = make_problem(128, 30000, 16, 8, (0, 1, 2), 3, uv_kind="radial", blocks="annuli", nannuli=16)
    g = prob.geom
    best, times = autotune_tile(g.nx, g.ny, prob.uv, prob.block_of_vis, prob.nblocks, kernel_width=8,
                                basis_ids=prob.basis_ids, levels=prob.levels, candidates=(4, 16, 32, 64), iters=3)
    assert times[4] < 0                      # below the kernel width: rejected by the plan
    assert best in (16, 32, 64) and times[best] == min(t for t in times.values() if t > 0)


@pytest.mark.parametrize("use_graph", [False, True])
def test_adaptive_probabilities_exact_reading(use_graph):
    # Sec. 4's c_i from ||Phi_i x^(t) - y_i|| of every block after every iteration
    prob, _ = make_problem(64, 16384, 16, 8, (0, 1, 2), 2, uv_kind="radial", blocks="annuli", nannuli=16)
    kw = _steps(prob)
    ad = {"n": 4.0, "p_min": 0.05, "p_max": 0.5, "exact": True}
    niter = 30
    st_ref, draws = PD.pd_run(prob, niter, seed=3, p_block=None, p_basis=[1.0] * 3, adaptive=ad, **kw)
    plan, st = _setup(prob, "f32")
    st.pd_iterate(niter, seed=3, p_basis=[1.0] * 3, adaptive=ad, use_graph=use_graph, **kw)
    rep = st.report()
    assert list(rep["block_active"]) == list(draws[-1][0])
    assert rel(st.x().cpu().numpy(), st_ref.x) < TOL_IT32
    assert np.allclose(rep["res_norm"], st_ref.res_norm, rtol=1e-4)
    assert rep["p_block"].sum() == pytest.approx(4.0, rel=1e-9)


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_per_block_form_matches_batched_form_and_oracle(precision):
    # one launch per active block per operator (host draws) against the batched form and
    # the oracle: same draws, same iterates up to the rounding order
    prob, _ = make_problem(64, 8192, 16, 8, (0, 1, 2), 2, uv_kind="radial", blocks="annuli", nannuli=16)
    kw = _steps(prob)
    args = dict(seed=5, p_block=[0.5] * 16, p_basis=[0.5] * 3, **kw)
    niter = 20
    st_ref, draws = PD.pd_run(prob, niter, **args)
    plan, st = _setup(prob, precision)
    st.pd_iterate(niter, per_block=True, **args)
    rep = st.report()
    assert rep["t"] == niter
    assert list(rep["block_active"]) == list(draws[-1][0])
    assert list(rep["basis_active"]) == list(draws[-1][1])
    x_pb = st.x().cpu().numpy()
    plan2, st2 = _setup(prob, precision)
    st2.pd_iterate(niter, **args)
    x_b = st2.x().cpu().numpy()
    tol_it = TOL_IT64 if precision == "f64" else TOL_IT32
    assert rel(x_pb, st_ref.x) < tol_it
    assert rel(st.v().cpu().numpy(), st_ref.v) < tol_it
    assert rel(x_pb, x_b) < (1e-12 if precision == "f64" else 1e-5)
