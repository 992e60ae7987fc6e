"""Pins of the oracle's reweighted analysis prior (SARA, Sec. 2): the weighted soft
threshold, the reweighting rule, and Algorithm 1 with weights against an independent
solver of the weighted problem."""
import numpy as np
import pytest

from oracle import pd as PD
from oracle import prox as PX
from paper_1610_08895_gb300 import synth
from test_oracle_pd import admm_reference, tiny_problem


def test_weighted_soft_threshold_is_componentwise():
    rng = np.random.default_rng(0)
    z = rng.normal(size=(3, 8, 8))
    z[0, 0, 0] = 0.0
    a = rng.uniform(0.0, 1.5, size=z.shape)
    a[1, 2, 3] = abs(z[1, 2, 3])                       # exactly at the threshold
    out = PX.soft_threshold(z, a)
    ref = np.array([PX.soft_threshold(np.array([zz]), aa)[0] for zz, aa in zip(z.ravel(), a.ravel())])
    assert np.array_equal(out.ravel(), ref)
    assert out[1, 2, 3] == 0.0 and out[0, 0, 0] == 0.0
    # Moreau: z = S_a(z) + P_[-a, a](z) with per-coefficient a (eq. prox-L1 and its conjugate)
    assert np.allclose(out + np.clip(z, -a, a), z, rtol=0, atol=1e-15)
    # the step-13 update with weights is the clip to the weighted box
    s = rng.normal(size=z.shape) * 0.1
    w = rng.normal(size=z.shape)
    assert np.allclose(PX.dual_sparsity_update(s, w, a), np.clip(s + w, -a, a), rtol=0, atol=1e-15)


def test_unit_weights_reproduce_the_unweighted_run():
    prob, _ = tiny_problem(nblocks=4, basis_ids=(0, 1, 2), levels=1)
    kw = dict(tau=0.49, sigma=1.0, varsigma=1e-3, kappa=0.02, psi_norm=1.0, seed=3,
              p_block=[0.5] * 4, p_basis=[0.5] * 3)
    st_a, _ = PD.pd_run(prob, 25, **kw)
    st_b, _ = PD.pd_run(prob, 25, weights=np.ones((3, 8, 8)), **kw)
    assert np.array_equal(st_a.x, st_b.x) and np.array_equal(st_a.s, st_b.s)


def test_weights_bound_each_coefficient_of_s():
    prob, _ = tiny_problem(nblocks=4, basis_ids=(0, 1, 2), levels=1)
    rng = np.random.default_rng(4)
    wts = rng.uniform(0.05, 1.0, size=(3, 8, 8))
    alpha = 0.02
    st = PD.PDState(prob)
    for _ in range(30):
        PD.pd_iteration(prob, st, 0.49, 1.0, 1e-4, alpha, 1.0, 3, [0.5] * 4, [0.5] * 3, weights=wts)
        assert np.all(np.abs(st.s) <= alpha * wts + 1e-15)


def test_sara_weights_closed_forms():
    prob, _ = tiny_problem(basis_ids=(0,), levels=1)
    rng = np.random.default_rng(2)
    x = rng.normal(size=(8, 8))
    delta = 0.3
    w = PD.sara_weights(prob, x, delta)
    # Dirac basis alone: Psi^H x = x
    assert np.allclose(w[0], delta / (delta + np.abs(x)), rtol=1e-15)
    prob2, _ = tiny_problem(basis_ids=(0, 1), levels=2)
    w2 = PD.sara_weights(prob2, x, delta)
    assert w2.shape == (2, 8, 8)
    assert np.allclose(w2[0], delta / (delta + np.abs(x) / np.sqrt(2)), rtol=1e-15)
    assert np.all((w2 > 0) & (w2 <= 1))
    # a zero coefficient keeps weight 1; |c| = delta gives 1/2
    z = np.zeros((8, 8))
    assert np.array_equal(PD.sara_weights(prob, z, delta), np.ones((1, 8, 8)))
    z[3, 4] = delta
    assert PD.sara_weights(prob, z, delta)[0, 3, 4] == 0.5


@pytest.mark.slow
def test_weighted_pd_converges_to_independent_solver_solution():
    prob, x_true = tiny_problem()
    x0 = synth.start_vector(8, 8, seed=9)
    phi2, psi2 = PD.operator_norms(prob, x0, max_iter=5000, tol=1e-13)
    wts = PD.sara_weights(prob, x_true, delta=0.05)
    st, _ = PD.pd_run(prob, 11000, tau=0.49, sigma=1.0 / psi2, varsigma=1.0 / phi2, kappa=0.1,
                      psi_norm=np.sqrt(psi2), seed=0, p_block=[1.0] * 2, p_basis=[1.0] * 2, weights=wts)
    x_ref = admm_reference(prob, weights=wts)
    assert np.all(st.x >= 0)
    assert np.all(PD.block_residuals(prob, st.x) <= prob.eps * (1 + 1e-4))
    f_pd = np.abs(wts * prob.psi_adj(st.x)).sum()
    f_ref = np.abs(wts * prob.psi_adj(x_ref)).sum()
    assert f_pd == pytest.approx(f_ref, rel=1e-4)
    assert np.linalg.norm(st.x - x_ref) / np.linalg.norm(x_ref) < 1e-4      # measured 8e-12
    # the weighted problem has another solution than the unweighted one
    x_l1 = admm_reference(prob)
    assert np.linalg.norm(x_l1 - x_ref) / np.linalg.norm(x_ref) > 1e-3
