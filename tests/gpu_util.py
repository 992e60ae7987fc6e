"""Shared helpers of the GPU parity tests: seeded problems built from synth, and
the oracle counterparts. Inputs come only from paper_1610_08895_gb300.synth;
expected values only from oracle/."""
import numpy as np

from oracle import experiment as EX
from oracle import measurement as meas
from oracle import pd as PD
from paper_1610_08895_gb300 import synth

# relative l2 tolerances: FP32 per operator application and iterate (stated by the
# task for complex64 bulk arithmetic); FP64 ones from the accumulated rounding of
# ~10^2 operations per output at 1.1e-16 with margin.
TOL_OP32 = 1e-5
TOL_IT32 = 1e-4
TOL_OP64 = 1e-12
TOL_IT64 = 1e-9


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def make_problem(n, m, nblocks, J, basis_ids, levels, uv_kind="gaussian", blocks="equal", snr=30.0, seed=0,
                 nannuli=None, nsectors=1):
    uv = synth.uv_gaussian(m, seed=seed + 1) if uv_kind == "gaussian" else synth.uv_radial(m, seed=seed + 1)
    if blocks == "equal":
        blk = synth.blocks_equal(uv, nblocks)
    else:
        blk = synth.blocks_annuli(uv, nannuli, nsectors)
    x_true = synth.test_image(n, seed=seed + 2)
    geo = meas.Geometry(n, n, J)
    prob = PD.Problem(geo, uv, blk, nblocks, list(basis_ids), levels)
    phix = prob.phi(x_true)
    sn = EX.noise_sigma(phix, snr)
    prob.y = phix + sn * synth.complex_noise(m, seed=seed + 3)
    prob.eps = EX.epsilon_bounds(sn, [max(len(ix), 1) for ix in prob.block_index])
    return prob, x_true
