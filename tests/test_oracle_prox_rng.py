"""Pins of the proximity operators (Sec. 3), the Philox draws (Alg. 1 step 3),
the adaptive probabilities (Sec. 4) and the chi-square bounds (Sec. 5)."""
import numpy as np
import pytest

from oracle import adaptive as AD
from oracle import experiment as EX
from oracle import philox as PH
from oracle import prox as PX


# ---------------------------------------------------------------- P_B (eq. proj-L2)
def test_ball_projection_closed_form_and_properties():
    rng = np.random.default_rng(0)
    y = rng.normal(size=50) + 1j * rng.normal(size=50)
    eps = 2.0
    for scale in [0.1, 0.5, 1.0, 3.0, 10.0]:
        z = y + scale * (rng.normal(size=50) + 1j * rng.normal(size=50)) / np.sqrt(50)
        p = PX.proj_l2ball(z, y, eps)
        dist = np.linalg.norm(z - y)
        if dist <= eps:
            assert np.array_equal(p, z)                      # identity inside (closed ball)
        else:
            assert np.linalg.norm(p - y) == pytest.approx(eps, rel=1e-14)   # on the sphere
            # along the ray from y through z
            assert np.allclose((p - y) * dist, (z - y) * eps, atol=1e-12)
        assert np.allclose(PX.proj_l2ball(p, y, eps), p, atol=1e-14)     # idempotent
    # non-expansive
    a = y + 5 * rng.normal(size=50)
    b = y + 5 * rng.normal(size=50)
    assert np.linalg.norm(PX.proj_l2ball(a, y, eps) - PX.proj_l2ball(b, y, eps)) <= np.linalg.norm(a - b)
    # boundary point exactly on the sphere stays
    z = y + eps * np.ones(50) / np.sqrt(50)
    assert np.allclose(PX.proj_l2ball(z, y, eps), z, atol=1e-14)


def test_dual_data_update_is_scaled_residual():
    # step 8 equals (z - y) max(0, 1 - eps / ||z - y||) with z = v + G b
    rng = np.random.default_rng(1)
    y = rng.normal(size=20) + 1j * rng.normal(size=20)
    for eps in [0.1, 1.0, 100.0]:
        v = rng.normal(size=20) + 1j * rng.normal(size=20)
        gb = rng.normal(size=20) + 1j * rng.normal(size=20)
        r = v + gb - y
        ref = r * max(0.0, 1.0 - eps / np.linalg.norm(r))
        assert np.allclose(PX.dual_data_update(v, gb, y, eps), ref, atol=1e-13)


# ---------------------------------------------------------------- S_alpha (eq. prox-L1)
def test_soft_threshold_closed_form_ties_and_moreau():
    z = np.array([-3.0, -1.0, -0.5, 0.0, 0.5, 1.0, 2.5])
    out = PX.soft_threshold(z, 1.0)
    assert np.array_equal(out, [-2.0, 0.0, 0.0, 0.0, 0.0, 0.0, 1.5])
    # Moreau decomposition (Sec. 3): z = S_alpha(z) + P_{||.||_inf <= alpha}(z)
    rng = np.random.default_rng(2)
    w = rng.normal(size=1000) * 3
    for alpha in [0.0, 0.3, 1.7]:
        assert np.allclose(PX.soft_threshold(w, alpha) + np.clip(w, -alpha, alpha), w, atol=1e-15)
    # hence step 13 is a clip onto [-alpha, alpha]
    s = rng.normal(size=1000)
    assert np.allclose(PX.dual_sparsity_update(s, w, 0.7), np.clip(s + w, -0.7, 0.7), atol=1e-15)


# ---------------------------------------------------------------- P_C (eq. proj-plus)
def test_positive_projection():
    z = np.array([1.5 + 2j, -0.5 + 1j, 0.0 - 3j, 2.0])
    assert np.array_equal(PX.proj_positive(z), [1.5, 0.0, 0.0, 2.0])


# ---------------------------------------------------------------- Philox (Alg. 1 step 3)
@pytest.mark.parametrize("key0,ctr", [(0, (0, 0, 0, 0)), (5, (0, 0, 0, 0)),
                                      (0xDEADBEEFCAFEF00D, (17, 1, 123456, 0)),
                                      (2 ** 64 - 1, (2 ** 64 - 2, 2 ** 63, 7, 9))])
def test_philox_matches_numpy_bit_generator(key0, ctr):
    # numpy's Philox pre-increments the 256-bit counter before each block of 4 words
    bg = np.random.Philox(key=np.array([key0, 0], dtype=np.uint64),
                          counter=np.array(ctr, dtype=np.uint64))
    raw = bg.random_raw(8)
    c = list(ctr)
    for blk in range(2):
        # increment the counter as a little-endian 256-bit integer
        val = sum(w << (64 * k) for k, w in enumerate(c)) + 1
        c = [(val >> (64 * k)) & ((1 << 64) - 1) for k in range(4)]
        got = PH.philox4x64_10(c, (key0, 0))
        assert [int(w) for w in raw[4 * blk: 4 * blk + 4]] == list(got)


def test_active_set_frequencies_follow_probabilities():
    probs = [0.05, 0.25, 0.5, 0.9, 1.0]
    n = 4000
    counts = np.zeros(len(probs))
    for t in range(1, n + 1):
        counts += PH.active_set(7, t, PH.STREAM_BLOCKS, probs)
    freq = counts / n
    for p, f in zip(probs, freq):
        sd = np.sqrt(max(p * (1 - p), 1e-12) / n)
        assert abs(f - p) <= 5 * sd + 1e-12
    assert counts[-1] == n                    # p = 1 always active


def test_draws_are_independent_of_stream_and_deterministic():
    a = [PH.uniform(3, t, 0, 5) for t in range(1, 50)]
    b = [PH.uniform(3, t, 1, 5) for t in range(1, 50)]
    assert a != b
    assert a == [PH.uniform(3, t, 0, 5) for t in range(1, 50)]
    assert all(0.0 <= u < 1.0 for u in a + b)


# ---------------------------------------------------------------- adaptive p (Sec. 4)
def _a_by_bisection(q, cap, target):
    lo, hi = 0.0, cap + 1.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if np.minimum(q + mid, cap).sum() < target:
            lo = mid
        else:
            hi = mid
    return hi


@pytest.mark.parametrize("seed", range(6))
def test_adaptive_probabilities_invariants(seed):
    rng = np.random.default_rng(seed)
    d, n, pmin, pmax = 16, 4.0, 0.05, 0.5
    c = rng.exponential(size=d) ** 3 * (rng.uniform(size=d) < 0.7)
    p = AD.probabilities(c, n, pmin, pmax)
    assert p.sum() == pytest.approx(n, rel=1e-12)
    assert np.all(p >= pmin - 1e-15) and np.all(p <= pmax + 1e-15)
    if c.sum() > 0:
        q = (n - d * pmin) * c / c.sum()
        a = _a_by_bisection(q, pmax - pmin, n - d * pmin)
        assert np.allclose(p, pmin + np.minimum(q + a, pmax - pmin), atol=1e-10)
        # monotone in c
        order = np.argsort(c)
        assert np.all(np.diff(p[order]) >= -1e-15)


def test_adaptive_probabilities_special_cases():
    # uniform fallback when every residual is inside its ball
    assert np.allclose(AD.probabilities(np.zeros(8), 2.0, 0.05, 0.5), 0.25)
    # no saturation: a = 0 and p is affine in c
    c = np.array([1.0, 1.0, 2.0, 0.0])
    p = AD.probabilities(c, 1.0, 0.1, 0.9)
    assert np.allclose(p, 0.1 + 0.6 * c / 4.0)
    # all mass on one block: it saturates and the rest share equally
    p = AD.probabilities(np.array([5.0, 0, 0, 0]), 2.0, 0.1, 0.5)
    assert np.allclose(p, [0.5, 0.5, 0.5, 0.5])
    # c_i definition
    assert np.allclose(AD.residual_distance([3.0, 1.0], [2.0, 2.0]), [0.25, 0.0])
    with pytest.raises(ValueError):
        AD.probabilities(np.ones(4), 3.0, 0.1, 0.5)       # p_max < n / d


# ---------------------------------------------------------------- epsilon (Sec. 5)
def test_epsilon_is_the_099_quantile_of_the_noise_norm():
    rng = np.random.default_rng(3)
    mi, sigma_n, trials = 64, 0.7, 20000
    eps = EX.epsilon_bounds(sigma_n, [mi])[0]
    w = (rng.normal(size=(trials, mi)) + 1j * rng.normal(size=(trials, mi))) / np.sqrt(2) * sigma_n
    frac = np.mean(np.linalg.norm(w, axis=1) <= eps)
    assert abs(frac - 0.99) < 5 * np.sqrt(0.99 * 0.01 / trials)
    # and the noise scale matches the requested input SNR
    phi_x = rng.normal(size=5000) + 1j * rng.normal(size=5000)
    s = EX.noise_sigma(phi_x, 30.0)
    noise = (rng.normal(size=5000) + 1j * rng.normal(size=5000)) / np.sqrt(2) * s
    snr = 20 * np.log10(np.linalg.norm(phi_x) / np.linalg.norm(noise))
    assert snr == pytest.approx(30.0, abs=0.3)
