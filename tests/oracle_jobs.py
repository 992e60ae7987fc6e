"""Oracle computations of the full-size parity tests, run in worker processes.

Each job builds its problem from the seeded generators in paper_1610_08895_gb300.synth
and computes the expected values with oracle/ only (FP64, CPU). The largest take
minutes, so the session starts them in a spawn-context process pool (no CUDA in the
workers) when the GPU tests that need them are collected, and the tests wait for them
at the end of the run (see conftest.py). Run inline, they give the same results."""
import numpy as np

from oracle import experiment as EX
from oracle import measurement as meas
from oracle import pd as PD
from paper_1610_08895_gb300 import synth


def bench_inputs(n, m, nannuli, nsectors, seed=0):
    """The bench's workload generators: radial uv, annuli x sectors blocks."""
    uv = synth.uv_radial(m, seed=seed + 1)
    blk = synth.blocks_annuli(uv, nannuli, nsectors)
    return uv, blk


def steps(prob, n_power, seed=9):
    """Step sizes from the oracle's power method (tau (sigma ||Psi||^2 + varsigma ||Phi||^2) < 1)."""
    x0 = synth.start_vector(prob.geom.ny, prob.geom.nx, seed=seed)
    phi2, psi2 = PD.operator_norms(prob, x0, max_iter=n_power, tol=1e-7)
    return dict(tau=0.49, sigma=1.0 / psi2, varsigma=1.0 / phi2, kappa=1e-3, psi_norm=float(np.sqrt(psi2)))


def problem(n, uv, blk, d, J, bases, levels, snr=30.0, seed=0):
    x_true = synth.test_image(n, seed=seed + 2)
    prob = PD.Problem(meas.Geometry(n, n, J), uv, blk, d, list(bases), levels)
    phix = prob.phi(x_true)
    sn = EX.noise_sigma(phix, snr)
    prob.y = phix + sn * synth.complex_noise(len(uv), seed=seed + 3)
    prob.eps = EX.epsilon_bounds(sn, [max(len(ix), 1) for ix in prob.block_index])
    return prob, x_true


def c2_run(niter=500):
    """256^2 image, 65,536 Gaussian points, 16 equal blocks at p = 0.5, 9 bases x 4 levels
    at p = 0.5, J = 8, 30 dB: niter oracle iterations with seed 0."""
    uv = synth.uv_gaussian(65536, seed=1)
    blk = synth.blocks_equal(uv, 16)
    prob, x_true = problem(256, uv, blk, 16, 8, range(9), 4)
    kw = steps(prob, 200)
    kw.update(seed=0, p_block=[0.5] * 16, p_basis=[0.5] * 9)
    st, draws = PD.pd_run(prob, niter, **kw)
    w_norm = float(np.linalg.norm(prob.psi_adj(st.x_tilde)))
    return dict(y=prob.y, eps=prob.eps, kw=kw, x=st.x, s=st.s, v=st.v, last_draw=draws[-1],
                snr=EX.snr_db(x_true, st.x), w_norm=w_norm)


def c3_run(niter=20):
    """512^2 image, 1,048,576 radial points in 64 equal-width annuli, adaptive probabilities
    (n = 16, p_min = 0.05, p_max = 0.5, lagged c_i), 9 bases x 4 levels, J = 8, 30 dB."""
    uv = synth.uv_radial(1_048_576, seed=1)
    blk = synth.blocks_annuli(uv, 64, 1)
    prob, x_true = problem(512, uv, blk, 64, 8, range(9), 4)
    kw = steps(prob, 40)
    ad = {"n": 16.0, "p_min": 0.05, "p_max": 0.5}
    kw.update(seed=0, p_block=None, p_basis=[1.0] * 9, adaptive=ad)
    st, draws = PD.pd_run(prob, niter, **kw)
    return dict(y=prob.y, eps=prob.eps, kw=kw, x=st.x, s=st.s, v=st.v, res_norm=st.res_norm,
                draws=[d[0] for d in draws])


def c5_phi_adj():
    """Re(Phi^H w) on the full bench workload (2048^2 image, 4096^2 grid, 16,777,216 radial
    points, J = 8) for the seeded complex vector w = synth.uniform_vis(M, seed=5)."""
    uv, _ = bench_inputs(2048, 16_777_216, 32, 8)
    geo = meas.Geometry(2048, 2048, 8)
    return dict(x=geo.phi_adj(synth.uniform_vis(len(uv), seed=5), uv))


def c5_start():
    """Seeded non-zero start values of one Algorithm 1 iteration on the bench workload:
    x^(0) = a blob image, x~^(0) = 2 x^(0) - x_prev, s^(0) small random coefficients,
    v^(0) small random duals; y = Phi-free synthetic data (noise scaled to the image)."""
    n, m = 2048, 16_777_216
    rng = np.random.Generator(np.random.PCG64(77))
    x0 = synth.test_image(n, seed=12)
    x_prev = 0.9 * x0 + 0.01 * rng.uniform(0.0, 1.0, size=(n, n))
    s0 = 1e-4 * rng.normal(size=(9, n, n))
    v0 = 1e-2 * synth.uniform_vis(m, seed=13)
    y = 10.0 * synth.uniform_vis(m, seed=14)
    return x0, 2.0 * x0 - x_prev, s0, v0, y


def c5_iteration():
    """One oracle iteration (p = 0.5 for blocks and bases, seed 0) on the bench workload from
    the c5_start values. Returns x^(1), s^(1) of basis 4 (db4), v^(1) at 200,000 sampled
    points and the draws."""
    uv, blk = bench_inputs(2048, 16_777_216, 32, 8)
    prob = PD.Problem(meas.Geometry(2048, 2048, 8), uv, blk, 256, list(range(9)), 4)
    x0, xt0, s0, v0, y = c5_start()
    prob.y = y
    prob.eps = np.full(256, 50.0 * np.sqrt(np.bincount(blk, minlength=256).max()))
    st = PD.PDState.__new__(PD.PDState)        # the given start values of Alg. 1 step 1
    st.x, st.x_tilde, st.s, st.v, st.t = x0.copy(), xt0.copy(), s0.copy(), v0.copy(), 0
    st.res_norm = np.zeros(256)                # written for active blocks, not read (fixed p)
    kw = dict(tau=0.49, sigma=1.0, varsigma=2e-9, kappa=0.05, psi_norm=1.0, seed=0,
              p_block=[0.5] * 256, p_basis=[0.5] * 9)
    act, actb = PD.pd_iteration(prob, st, **kw)
    sample = np.random.Generator(np.random.PCG64(5)).choice(m := len(uv), size=200_000, replace=False)
    return dict(eps=prob.eps, kw=kw, x=st.x, s4=st.s[4], s_norms=np.linalg.norm(st.s.reshape(9, -1), axis=1),
                v_idx=sample, v=st.v[sample], act=np.array(act), actb=np.array(actb),
                frac_pos=float(np.mean(st.x > 0)), dx=float(np.linalg.norm(st.x - x0) / np.linalg.norm(x0)),
                frac_clip=float(np.mean(np.abs(st.s[4]) >= 0.05 * (1 - 1e-12))))


JOBS = {"c2_run": c2_run, "c3_run": c3_run, "c5_phi_adj": c5_phi_adj, "c5_iteration": c5_iteration}


def run(name):
    return JOBS[name]()
