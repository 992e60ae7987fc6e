"""GPU parity of the DDE-aware G (Sec. 2: G models compact-support DDEs as a convolution
in the Fourier domain besides interpolating), stored as complex CSR rows: Phi, Phi^H and
Algorithm 1 against the oracle, at sizes spanning several tiles with ragged work lists."""
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


def random_dde(m, d, seed):
    """Near-identity complex Fourier-domain kernels (smooth direction-dependent gains)."""
    rng = np.random.default_rng(seed)
    k = 0.2 * (rng.normal(size=(m, d, d)) + 1j * rng.normal(size=(m, d, d)))
    k[:, d // 2, d // 2] += 1.0
    return k


def _dde_problem(n, m, nblocks, J, d, seed=0, **kw):
    prob, x_true = make_problem(n, m, nblocks, J, (0, 1, 2), 2, seed=seed, **kw)
    prob.dde = random_dde(m, d, seed + 50)
    # data of the DDE-aware model
    from oracle import experiment as EX
    phix = prob.phi(x_true)
    sn = EX.noise_sigma(phix, 30.0)
    prob.y = phix + sn * synth.complex_noise(m, seed=seed + 3)
    prob.eps = EX.epsilon_bounds(sn, [max(len(ix), 1) for ix in prob.block_index])
    return prob, x_true


def _plan(prob, precision, tile=0):
    from paper_1610_08895_gb300.api import Plan
    g = prob.geom
    return Plan(g.nx, g.ny, prob.uv, prob.block_of_vis, prob.nblocks, kernel_width=g.J,
                basis_ids=prob.basis_ids, levels=prob.levels, precision=precision, tile=tile, g_mode="csr",
                dde_kernels=prob.dde)


CASES = [
    # n, M, blocks, J, d, tile
    (16, 300, 4, 4, 3, 0),       # footprint 6, one tile per side pair, taps wrap
    (64, 4096, 4, 4, 5, 16),     # footprint 8 over 16-cell tiles
    (64, 5000, 16, 6, 3, 32),    # footprint 8, ragged chunks
    (128, 20000, 16, 4, 3, 32),  # footprint 6, 64 tiles
]


@pytest.mark.parametrize("precision", ["f32", "f64"])
@pytest.mark.parametrize("case", CASES)
def test_dde_phi_and_adjoint_match_oracle(case, precision):
    n, m, nb, J, d, tile = case
    prob, x_true = _dde_problem(n, m, nb, J, d)
    plan = _plan(prob, precision, tile)
    rdt = torch.float32 if precision == "f32" else torch.float64
    tol = TOL_OP32 if precision == "f32" else TOL_OP64
    y = plan.pd_apply_phi(torch.tensor(x_true, dtype=rdt, device="cuda")).cpu().numpy()
    assert rel(y, prob.phi(x_true)) < tol
    v = synth.uniform_vis(m, seed=5)
    xa = plan.pd_apply_phi_adj(torch.tensor(v, dtype=plan.cplx_dtype, device="cuda")).cpu().numpy()
    assert rel(xa, prob.phi_adj(v)) < tol


def test_identity_dde_equals_the_plain_operator():
    from paper_1610_08895_gb300.api import Plan
    prob, x_true = make_problem(64, 4000, 4, 6, (0,), 1)
    dde = np.zeros((4000, 3, 3), dtype=np.complex128)
    dde[:, 1, 1] = 1.0
    g = prob.geom
    for precision, tol in (("f32", 2e-6), ("f64", 1e-13)):
        rdt = torch.float32 if precision == "f32" else torch.float64
        x = torch.tensor(x_true, dtype=rdt, device="cuda")
        a = Plan(g.nx, g.ny, prob.uv, prob.block_of_vis, 4, kernel_width=6, precision=precision, g_mode="csr",
                 dde_kernels=dde).pd_apply_phi(x).cpu().numpy()
        b = Plan(g.nx, g.ny, prob.uv, prob.block_of_vis, 4, kernel_width=6, precision=precision,
                 g_mode="csr").pd_apply_phi(x).cpu().numpy()
        assert rel(a, b) < tol


def _steps(prob):
    x0 = synth.start_vector(prob.geom.ny, prob.geom.nx, seed=9)
    phi2, psi2 = PD.operator_norms(prob, x0, max_iter=500, tol=1e-8)
    return dict(tau=0.49, sigma=1.0 / psi2, varsigma=1.0 / phi2, kappa=1e-3, psi_norm=float(np.sqrt(psi2)))


@pytest.mark.parametrize("precision,use_graph", [("f64", False), ("f32", True)])
def test_dde_pd_iterations_match_oracle(precision, use_graph):
    from paper_1610_08895_gb300.api import State
    prob, _ = _dde_problem(64, 8192, 16, 6, 3, uv_kind="radial", blocks="annuli", nannuli=16)
    kw = _steps(prob)
    args = dict(seed=4, p_block=[0.5] * 16, p_basis=[0.5] * 3, **kw)
    niter = 25
    st_ref, draws = PD.pd_run(prob, niter, **args)
    plan = _plan(prob, precision)
    st = State(plan)
    st.pd_state_set_data(torch.tensor(prob.y, dtype=plan.cplx_dtype, device="cuda"), prob.eps)
    st.pd_iterate(niter, use_graph=use_graph, **args)
    rep = st.report()
    assert list(rep["block_active"]) == list(draws[-1][0])
    tol = TOL_IT64 if precision == "f64" else TOL_IT32
    assert rel(st.x().cpu().numpy(), st_ref.x) < tol
    assert rel(st.v().cpu().numpy(), st_ref.v) < tol


def test_dde_plans_refused():
    from paper_1610_08895_gb300._binding import PDError
    from paper_1610_08895_gb300.api import Plan
    uv = synth.uv_gaussian(50, seed=1)
    blk = np.zeros(50, np.int32)
    with pytest.raises(PDError):
        Plan(32, 32, uv, blk, 1, kernel_width=4, dde_kernels=random_dde(50, 3, 0))            # not CSR
    with pytest.raises(PDError):
        Plan(32, 32, uv, blk, 1, kernel_width=8, g_mode="csr", dde_kernels=random_dde(50, 3, 0))  # 10 > 8
    with pytest.raises(PDError):
        Plan(32, 32, uv, blk, 1, kernel_width=4, g_mode="csr", dde_kernels=random_dde(50, 2, 0))  # even d
