"""Pins of the oracle's Algorithm 1 (PD-R) and power method against independent computations."""
import numpy as np
import pytest

from oracle import experiment as EX
from oracle import measurement as meas
from oracle import pd as PD
from oracle import prox as PX
from paper_1610_08895_gb300 import synth


def tiny_problem(n=8, m=256, nblocks=2, basis_ids=(0, 1), levels=2, J=4, snr=30.0, seed=0):
    geo = meas.Geometry(n, n, J)
    uv = synth.uv_gaussian(m, seed=seed + 1)
    blk = synth.blocks_equal(uv, nblocks) if int(np.sqrt(nblocks)) ** 2 == nblocks else \
        (np.arange(m) % nblocks).astype(np.int32)
    x_true = synth.test_image(n, seed=seed + 2)
    prob = PD.Problem(geo, uv, blk, nblocks, list(basis_ids), levels)
    phix = prob.phi(x_true)
    sn = EX.noise_sigma(phix, snr)
    prob.y = phix + sn * synth.complex_noise(m, seed=seed + 3)
    prob.eps = EX.epsilon_bounds(sn, [len(ix) for ix in prob.block_index])
    return prob, x_true


def dense_phi(prob):
    """Columns of Phi as a real 2M x N matrix [Re; Im], by applying it to unit images."""
    g = prob.geom
    cols = []
    for k in range(g.ny * g.nx):
        e = np.zeros(g.ny * g.nx)
        e[k] = 1.0
        y = prob.phi(e.reshape(g.ny, g.nx))
        cols.append(np.concatenate([y.real, y.imag]))
    return np.array(cols).T


def test_power_method_matches_dense_eigenvalue():
    prob, _ = tiny_problem()
    A = dense_phi(prob)
    lam_dense = np.linalg.eigvalsh(A.T @ A)[-1]
    x0 = synth.start_vector(8, 8, seed=9)
    phi2, psi2 = PD.operator_norms(prob, x0, max_iter=5000, tol=1e-13)
    assert phi2 == pytest.approx(lam_dense, rel=1e-8)
    assert psi2 == pytest.approx(1.0, rel=1e-12)


def admm_reference(prob, iters=30000, rho=1.0, weights=None):
    """Independent solver of problem (basic-min-problem) on dense matrices.

    ADMM on min ||W x||_1 + i_{x>=0}(x) + sum_i i_{B_i}(A_i x) with the splitting
    z = K x, K = [W; I; A_1; ...; A_d]; the x-step is a dense linear solve.
    weights: per-coefficient weights of the reweighted prior (W = diag(w) Psi^H).
    """
    g = prob.geom
    N = g.ny * g.nx
    W = np.array([prob.psi_adj(e.reshape(g.ny, g.nx)).ravel() for e in np.eye(N)]).T
    if weights is not None:
        W = np.asarray(weights).ravel()[:, None] * W
    A = dense_phi(prob)
    M = len(prob.uv)
    rows = []
    for ix in prob.block_index:
        rows.append(np.concatenate([ix, ix + M]))
    K = np.vstack([W, np.eye(N)] + [A[r] for r in rows])
    ys = [np.concatenate([prob.y[ix].real, prob.y[ix].imag]) for ix in prob.block_index]
    nW = W.shape[0]
    sizes = [nW, N] + [len(r) for r in rows]
    offs = np.concatenate([[0], np.cumsum(sizes)])
    KtK_inv = np.linalg.inv(K.T @ K)
    x = np.zeros(N)
    z = K @ x
    u = np.zeros_like(z)
    for _ in range(iters):
        x = KtK_inv @ (K.T @ (z - u))
        kx = K @ x
        q = kx + u
        zn = np.empty_like(q)
        a = q[offs[0]:offs[1]]
        zn[offs[0]:offs[1]] = np.sign(a) * np.maximum(np.abs(a) - 1.0 / rho, 0.0)
        zn[offs[1]:offs[2]] = np.maximum(q[offs[1]:offs[2]], 0.0)
        for i, yi in enumerate(ys):
            seg = q[offs[2 + i]:offs[3 + i]]
            zn[offs[2 + i]:offs[3 + i]] = PX.proj_l2ball(seg, yi, prob.eps[i])
        z = zn
        u = u + kx - z
    return x.reshape(g.ny, g.nx)


@pytest.mark.slow
def test_pd_converges_to_independent_solver_solution():
    prob, x_true = tiny_problem()
    x0 = synth.start_vector(8, 8, seed=9)
    phi2, psi2 = PD.operator_norms(prob, x0, max_iter=5000, tol=1e-13)
    # measured: the distance to the ADMM point falls ~6x per 2500 iterations (3.8e-5 at 10000)
    st, _ = PD.pd_run(prob, 11000, tau=0.49, sigma=1.0 / psi2, varsigma=1.0 / phi2, kappa=0.1,
                      psi_norm=np.sqrt(psi2), seed=0, p_block=[1.0] * 2, p_basis=[1.0] * 2)
    x_ref = admm_reference(prob)
    # both are feasible and reach the same objective and point
    assert np.all(st.x >= 0)
    res = PD.block_residuals(prob, st.x)
    assert np.all(res <= prob.eps * (1 + 1e-4))
    assert np.all(PD.block_residuals(prob, x_ref) <= prob.eps * (1 + 1e-9))
    f_pd, f_ref = PD.objective(prob, st.x), PD.objective(prob, x_ref)
    assert f_pd == pytest.approx(f_ref, rel=1e-4)
    assert np.linalg.norm(st.x - x_ref) / np.linalg.norm(x_ref) < 1e-4


def test_pd_iteration_invariants_and_step_structure():
    prob, _ = tiny_problem(nblocks=4, basis_ids=(0, 1, 2), levels=1)
    alpha = 0.02
    st = PD.PDState(prob)
    x_prev = st.x.copy()
    for _ in range(30):
        act, actb = PD.pd_iteration(prob, st, tau=0.49, sigma=1.0, varsigma=1e-4, kappa=alpha,
                                    psi_norm=1.0, seed=3, p_block=[0.5] * 4, p_basis=[0.5] * 3)
        assert np.all(st.x >= 0)                                   # P_C
        assert np.all(np.abs(st.s) <= alpha + 1e-15)               # step 13 keeps s in [-alpha, alpha]
        assert np.allclose(st.x_tilde, 2 * st.x - x_prev)          # step 18
        x_prev = st.x.copy()


def test_inactive_blocks_and_bases_keep_their_duals():
    prob, _ = tiny_problem(nblocks=4, basis_ids=(0, 1, 2), levels=1)
    st = PD.PDState(prob)
    for _ in range(3):
        PD.pd_iteration(prob, st, 0.49, 1.0, 1e-4, 0.02, 1.0, 5, [1.0] * 4, [1.0] * 3)
    v0, s0 = st.v.copy(), st.s.copy()
    act, actb = PD.pd_iteration(prob, st, 0.49, 1.0, 1e-4, 0.02, 1.0, 5, [0.5] * 4, [0.5] * 3)
    assert not all(act) or not all(actb)
    for i, on in enumerate(act):
        if not on:                                                 # step 11
            assert np.array_equal(st.v[prob.block_index[i]], v0[prob.block_index[i]])
    for k, on in enumerate(actb):
        if not on:
            assert np.array_equal(st.s[k], s0[k])


@pytest.mark.slow
def test_randomised_pd_reaches_the_same_solution():
    # with p = 0.5 the iterates still converge to the solution of (basic-min-problem),
    # roughly 2x slower than p = 1 (Sec. 5); measured 1.4e-3 after 10000 iterations
    prob, _ = tiny_problem()
    x0 = synth.start_vector(8, 8, seed=9)
    phi2, psi2 = PD.operator_norms(prob, x0, max_iter=5000, tol=1e-12)
    x_ref = admm_reference(prob)
    st_rnd, draws = PD.pd_run(prob, 10000, tau=0.49, sigma=1.0 / psi2, varsigma=1.0 / phi2, kappa=0.1,
                              psi_norm=np.sqrt(psi2), seed=1, p_block=[0.5, 0.5], p_basis=[0.5, 1.0])
    assert 0.45 < np.mean([a for d in draws for a in d[0]]) < 0.55
    assert np.linalg.norm(st_rnd.x - x_ref) / np.linalg.norm(x_ref) < 3e-3


def test_adaptive_pd_runs_and_keeps_probability_budget():
    prob, _ = tiny_problem(nblocks=4, m=256)
    st = PD.PDState(prob)
    ad = {"n": 1.0, "p_min": 0.05, "p_max": 0.5}
    counts = 0
    for _ in range(40):
        act, _ = PD.pd_iteration(prob, st, 0.49, 1.0, 1e-3, 0.1, 1.0, 2, None, [1.0] * 2, adaptive=ad)
        counts += sum(act)
    assert 0 < counts < 40 * 4


def test_exact_adaptive_with_full_budget_is_the_deterministic_run():
    # n = d forces every p_i = 1 (sum p_i = n, p_i <= 1), whatever the c_i: the exact
    # reading must then reproduce the deterministic Algorithm 1 exactly
    prob, _ = tiny_problem(nblocks=4, m=256)
    kw = dict(tau=0.49, sigma=1.0, varsigma=1e-3, kappa=0.1, psi_norm=1.0, seed=2, p_basis=[1.0] * 2)
    st_det, _ = PD.pd_run(prob, 25, p_block=[1.0] * 4, **kw)
    st_ex, draws = PD.pd_run(prob, 25, p_block=None, adaptive={"n": 4.0, "p_min": 0.05, "p_max": 1.0,
                                                             "exact": True}, **kw)
    assert all(all(a) for a, _ in draws)
    assert np.array_equal(st_ex.x, st_det.x)


def test_exact_adaptive_norms_are_those_of_the_current_iterate():
    # the exact reading keeps ||Phi_i x^(t) - y_i|| for every block (Sec. 4), whereas the
    # lagged reading keeps the norm of the last pass in which the block was active
    prob, _ = tiny_problem(nblocks=4, m=256)
    st = PD.PDState(prob)
    ad = {"n": 1.0, "p_min": 0.05, "p_max": 0.5, "exact": True}
    for _ in range(10):
        PD.pd_iteration(prob, st, 0.49, 1.0, 1e-3, 0.1, 1.0, 2, None, [1.0] * 2, adaptive=ad)
        direct = np.array([np.linalg.norm(meas.Geometry(8, 8, 4).phi(st.x, prob.uv[ix]) - prob.y[ix])
                           for ix in prob.block_index])
        assert np.allclose(st.res_norm, direct, rtol=1e-12)


def test_lagged_adaptive_norms_follow_the_last_active_pass():
    # default reading of Sec. 4's c_i: after iteration t, an active block i holds
    # ||Phi_i x~^(t-1) - y_i|| (the residual of step 8, on the x~ the iteration started
    # from); an inactive block keeps its previous value bit for bit; before the first
    # iteration every block holds ||Phi_i x^(0) - y_i|| = ||y_i||
    prob, _ = tiny_problem(nblocks=4, m=256)
    st = PD.PDState(prob)
    assert np.array_equal(st.res_norm, np.array([np.linalg.norm(prob.y[ix]) for ix in prob.block_index]))
    ad = {"n": 2.0, "p_min": 0.05, "p_max": 0.9}
    geo = meas.Geometry(8, 8, 4)
    seen_inactive = seen_active = 0
    for _ in range(12):
        xt_prev = st.x_tilde.copy()
        prev = st.res_norm.copy()
        act, _ = PD.pd_iteration(prob, st, 0.49, 1.0, 1e-3, 0.1, 1.0, 4, None, [1.0] * 2, adaptive=ad)
        for i, ix in enumerate(prob.block_index):
            if act[i]:
                direct = np.linalg.norm(geo.phi(xt_prev, prob.uv[ix]) - prob.y[ix])
                assert st.res_norm[i] == pytest.approx(direct, rel=1e-12)
                seen_active += 1
            else:
                assert st.res_norm[i] == prev[i]
                seen_inactive += 1
    assert seen_active > 0 and seen_inactive > 0


def test_snr_of_a_known_error():
    # 20 log10(||x|| / ||x - x_hat||): x_hat = 0.9 x leaves 10% of ||x|| as error -> 20 dB
    x = synth.test_image(16, seed=4)
    assert EX.snr_db(x, 0.9 * x) == pytest.approx(20.0, abs=1e-12)
    e = np.zeros_like(x)
    e[3, 5] = 0.01 * np.linalg.norm(x)                           # one pixel off by 1% of ||x|| -> 40 dB
    assert EX.snr_db(x, x + e) == pytest.approx(40.0, abs=1e-9)
