"""Pins of the oracle's synthesis formulation (Sec. 2's synthesis approach, solved with
the primal-dual template of Sec. 3) against an independent solver of the same problem
and the structure of its steps."""
import numpy as np
import pytest

from oracle import pd as PD
from oracle import prox as PX
from oracle import synthesis as SY
from paper_1610_08895_gb300 import synth
from test_oracle_pd import dense_phi, tiny_problem


def admm_synthesis(prob, iters=30000, rho=1.0):
    """Independent solver on dense matrices: ADMM on
    min ||alpha||_1 + i_{>=0}(Psi alpha) + sum_i i_{B_i}(A_i Psi alpha), splitting z = K alpha
    with K = [I; Psi; A_1 Psi; ...] and a dense solve for the alpha-step."""
    g = prob.geom
    N = g.ny * g.nx
    b = len(prob.basis_ids)
    nc = b * N
    S = np.array([prob.psi(e.reshape(b, g.ny, g.nx)).ravel() for e in np.eye(nc)]).T     # N x bN
    A = dense_phi(prob)
    M = len(prob.uv)
    rows = [np.concatenate([ix, ix + M]) for ix in prob.block_index]
    K = np.vstack([np.eye(nc), S] + [A[r] @ S for r in rows])
    ys = [np.concatenate([prob.y[ix].real, prob.y[ix].imag]) for ix in prob.block_index]
    sizes = [nc, N] + [len(r) for r in rows]
    offs = np.concatenate([[0], np.cumsum(sizes)])
    KtK_inv = np.linalg.inv(K.T @ K)
    a = np.zeros(nc)
    z = K @ a
    w = np.zeros_like(z)
    for _ in range(iters):
        a = KtK_inv @ (K.T @ (z - w))
        ka = K @ a
        q = ka + w
        zn = np.empty_like(q)
        zn[:nc] = np.sign(q[:nc]) * np.maximum(np.abs(q[:nc]) - 1.0 / rho, 0.0)
        zn[offs[1]:offs[2]] = np.maximum(q[offs[1]:offs[2]], 0.0)
        for i, yi in enumerate(ys):
            zn[offs[2 + i]:offs[3 + i]] = PX.proj_l2ball(q[offs[2 + i]:offs[3 + i]], yi, prob.eps[i])
        z = zn
        w = w + ka - z
    return a.reshape(b, g.ny, g.nx)


def test_synthesis_step_structure():
    prob, _ = tiny_problem(nblocks=4, basis_ids=(0, 1, 2), levels=1)
    st = SY.SynthesisState(prob)
    a_prev = st.alpha.copy()
    v0 = None
    for k in range(20):
        if k == 10:
            v0 = st.v.copy()
        act = SY.synthesis_iteration(prob, st, tau=0.49, sigma=1.0, varsigma=1e-3, kappa=0.05, seed=2,
                                     p_block=[0.5] * 4)
        assert np.all(st.u <= 0)                                             # dual of positivity
        assert np.allclose(st.alpha_tilde, 2 * st.alpha - a_prev)            # step 18
        a_prev = st.alpha.copy()
        if k == 10:
            for i, on in enumerate(act):
                if not on:                                                   # inactive blocks keep v_i
                    assert np.array_equal(st.v[prob.block_index[i]], v0[prob.block_index[i]])
    assert np.count_nonzero(st.alpha) < st.alpha.size                          # the l1 prox zeroes entries


@pytest.mark.slow
def test_synthesis_converges_to_independent_solver_solution():
    prob, _ = tiny_problem()
    x0 = synth.start_vector(8, 8, seed=9)
    phi2, _ = PD.operator_norms(prob, x0, max_iter=5000, tol=1e-13)
    st, _ = SY.synthesis_run(prob, 12000, tau=0.49, sigma=1.0, varsigma=1.0 / phi2, kappa=0.1, seed=0,
                             p_block=[1.0] * 2)
    a_ref = admm_synthesis(prob)
    x = st.x(prob)
    assert np.all(x >= -1e-6)
    assert np.all(PD.block_residuals(prob, x) <= prob.eps * (1 + 1e-4))
    # the minimiser over a redundant dictionary need not be unique (measured: the two
    # coefficient vectors differ by 1.5%), the minimum is: compare it, and check that the
    # reference point is feasible too
    f, f_ref = np.abs(st.alpha).sum(), np.abs(a_ref).sum()
    assert f == pytest.approx(f_ref, rel=1e-4)
    x_ref = prob.psi(a_ref)
    assert np.all(x_ref >= -1e-9)
    assert np.all(PD.block_residuals(prob, x_ref) <= prob.eps * (1 + 1e-9))


@pytest.mark.slow
def test_synthesis_with_the_dirac_basis_is_the_analysis_problem():
    # with Psi = I (the Dirac basis alone) both formulations minimise ||x||_1 over the same
    # constraint set: Algorithm 1 and the synthesis iterations reach the same minimum
    prob, _ = tiny_problem(basis_ids=(0,), levels=1)
    x0 = synth.start_vector(8, 8, seed=9)
    phi2, psi2 = PD.operator_norms(prob, x0, max_iter=5000, tol=1e-13)
    st_a, _ = PD.pd_run(prob, 8000, tau=0.49, sigma=1.0 / psi2, varsigma=1.0 / phi2, kappa=0.1,
                        psi_norm=np.sqrt(psi2), seed=0, p_block=[1.0] * 2, p_basis=[1.0])
    st_s, _ = SY.synthesis_run(prob, 8000, tau=0.49, sigma=1.0, varsigma=1.0 / phi2, kappa=0.1, seed=0,
                               p_block=[1.0] * 2)
    xs = st_s.x(prob)
    assert np.abs(xs).sum() == pytest.approx(np.abs(st_a.x).sum(), rel=1e-4)
    assert np.all(PD.block_residuals(prob, xs) <= prob.eps * (1 + 1e-4))
