"""Parity at the sizes and lengths of the named workloads, against oracle runs made in
worker processes (tests/oracle_jobs.py; started when this module is collected):

* 256^2, 65,536 Gaussian points, 16 blocks and 9 bases at p = 0.5: 500 iterations;
* 512^2, 1,048,576 radial points in 64 annuli, adaptive probabilities (n = 16,
  p_min = 0.05, p_max = 0.5), 9 bases x 4 levels, graph replay: 20 iterations, full x, s, v;
* the bench workload (2048^2 image, 4096^2 grid, 16,777,216 radial points, 256 uneven
  blocks): the full image of Re(Phi^H w), and one iteration of Algorithm 1 from non-zero
  start values (x~ != 0, s != 0, v != 0, so U != 0 before the gridding) in the graph form
  the bench times.

This module runs last among the parity tests (the bench-size cases at its end)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from gpu_util import TOL_IT32, TOL_OP32, rel  # noqa: E402
from paper_1610_08895_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__ as ge
    ge.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _plan_state(n, uv, blk, d, res, bases=range(9), levels=4):
    from paper_1610_08895_gb300.api import Plan, State
    plan = Plan(n, n, uv, blk, d, kernel_width=8, basis_ids=list(bases), levels=levels, precision="f32")
    st = State(plan)
    st.pd_state_set_data(torch.tensor(res["y"], dtype=torch.complex64, device="cuda"), res["eps"])
    return plan, st


def test_c2_500_iterations(oracle_job):
    res = oracle_job("c2_run")
    uv = synth.uv_gaussian(65536, seed=1)
    plan, st = _plan_state(256, uv, synth.blocks_equal(uv, 16), 16, res)
    st.pd_iterate(500, use_graph=True, **res["kw"])
    rep = st.report()
    assert list(rep["block_active"]) == list(res["last_draw"][0])
    s_gpu = st.s().cpu().numpy()
    ex, es, ev = rel(st.x().cpu().numpy(), res["x"]), rel(s_gpu, res["s"]), rel(st.v().cpu().numpy(), res["v"])
    # s = clip(s + Psi^H x~ / sqrt(b), -kappa, kappa) holds small differences of much larger
    # analysis coefficients: its FP32 rounding is relative to ||Psi^H x~||, not to ||s||
    es_w = float(np.linalg.norm((s_gpu - res["s"]).ravel()) / res["w_norm"])
    print(f"c2 500 iterations: rel x {ex:.2e} s {es:.2e} (of ||Psi^H x~||: {es_w:.2e}) v {ev:.2e} "
          f"(oracle SNR {res['snr']:.2f} dB)")
    assert ex < TOL_IT32 and ev < TOL_IT32
    assert es_w < TOL_OP32


def test_c3_adaptive_graph_20_iterations(oracle_job):
    res = oracle_job("c3_run")
    uv = synth.uv_radial(1_048_576, seed=1)
    plan, st = _plan_state(512, uv, synth.blocks_annuli(uv, 64, 1), 64, res)
    kw = dict(res["kw"])
    for t in range(20):
        st.pd_iterate(1, use_graph=True, **kw)
        assert list(st.report()["block_active"]) == list(res["draws"][t])
    rep = st.report()
    ex, es, ev = (rel(st.x().cpu().numpy(), res["x"]), rel(st.s().cpu().numpy(), res["s"]),
                  rel(st.v().cpu().numpy(), res["v"]))
    print(f"c3 20 adaptive iterations: rel x {ex:.2e} s {es:.2e} v {ev:.2e}")
    assert ex < TOL_IT32 and es < TOL_IT32 and ev < TOL_IT32
    assert np.allclose(rep["res_norm"], res["res_norm"], rtol=1e-4)
    assert rep["p_block"].sum() == pytest.approx(16.0, rel=1e-9)


def test_c5_phi_adjoint_full_image(oracle_job):
    from paper_1610_08895_gb300.api import Plan
    from oracle_jobs import bench_inputs
    uv, blk = bench_inputs(2048, 16_777_216, 32, 8)
    plan = Plan(2048, 2048, uv, blk, 256, kernel_width=8, basis_ids=list(range(9)), levels=4, precision="f32")
    w = torch.tensor(synth.uniform_vis(len(uv), seed=5), dtype=torch.complex64, device="cuda")
    xa = plan.pd_apply_phi_adj(w).cpu().numpy()
    ref = oracle_job("c5_phi_adj")["x"]
    e = rel(xa, ref)
    print(f"c5 Phi^H full image: rel {e:.2e}")
    assert e < TOL_OP32
    plan.close()


def test_c5_one_graph_iteration_from_nonzero_start(oracle_job):
    from oracle_jobs import bench_inputs, c5_start
    from paper_1610_08895_gb300.api import Plan, State
    uv, blk = bench_inputs(2048, 16_777_216, 32, 8)
    x0, xt0, s0, v0, y = c5_start()
    plan = Plan(2048, 2048, uv, blk, 256, kernel_width=8, basis_ids=list(range(9)), levels=4, precision="f32")
    st = State(plan)
    res = oracle_job("c5_iteration")
    st.pd_state_set_data(torch.tensor(y, dtype=torch.complex64, device="cuda"), res["eps"])
    f32 = lambda a: torch.tensor(a, dtype=torch.float32, device="cuda")   # noqa: E731
    st.pd_state_set_start(f32(x0), f32(xt0), f32(s0), torch.tensor(v0, dtype=torch.complex64, device="cuda"))
    st.pd_iterate(1, use_graph=True, **res["kw"])
    rep = st.report()
    assert list(rep["block_active"]) == list(res["act"]) and list(rep["basis_active"]) == list(res["actb"])
    x = st.x().cpu().numpy().astype(np.float64)
    s = st.s().cpu().numpy()
    v = st.v().cpu().numpy()
    # the update itself (x^(1) - x^(0)), not only x^(1), which keeps most of x^(0)
    ex = rel(x - x0, res["x"] - x0)
    es = rel(s[4], res["s4"])
    ev = rel(v[res["v_idx"]], res["v"])
    print(f"c5 one iteration: rel dx {ex:.2e} s(db4) {es:.2e} v(sample) {ev:.2e}; oracle: "
          f"{res['frac_pos']:.2f} of x positive, |dx|/|x0| {res['dx']:.2e}, {res['frac_clip']:.2f} of s clipped")
    assert ex < TOL_IT32 and es < TOL_IT32 and ev < TOL_IT32
    assert np.allclose(np.linalg.norm(s.reshape(9, -1).astype(np.float64), axis=1), res["s_norms"], rtol=1e-4)
