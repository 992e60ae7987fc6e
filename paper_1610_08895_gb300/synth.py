"""Seeded synthetic inputs for the PD-R RI imaging workloads.

This module holds input generation only -- images, uv coverages, block
partitions, standard complex noise and random start vectors -- and none of the
method's arithmetic. Both the CUDA path and the test oracle consume what it
produces. Recipes (stand-ins for the paper's M31 image and simulated coverage,
Sec. 5 of arXiv:1610.08895, which are not available here):

* image: 20 Gaussian blobs (width 1-4 px at 64x64, scaled with n/64) with
  centres uniform over the image, plus 10 single-pixel point sources;
  amplitudes uniform in (0, 1]. Nonnegative.
* uv "gaussian": 2-D Gaussian of standard deviation 0.25 pi per axis (the band
  edge is pi), points outside [-pi, pi)^2 redrawn.
* uv "radial": area density proportional to 8^(-r/pi) for r < pi (the inner
  density is 8x the outer), uniform angle.
* uv "gaussian with holes": the Gaussian coverage with circular holes cut mostly in
  the high frequencies (Sec. 5: holes placed with an inverse Gaussian profile): hole
  centres are drawn with density proportional to 1 - exp(-r^2 / (2 s^2)) (low at the
  origin, high towards the band edge), and points falling in a hole are redrawn.
* blocks "equal": sqrt(d) equal-count strips in u, each cut into sqrt(d)
  equal-count pieces in v (compact uv regions, Sec. 3).
* blocks "annuli": equal-width radial annuli over [0, pi); "annuli_sectors"
  further cuts each annulus into angular sectors.
* noise: standard complex normal, E|w|^2 = 1, to be scaled by the caller.
"""
import numpy as np


def _rng(seed):
    return np.random.Generator(np.random.PCG64(int(seed)))


def test_image(n, seed=0, nblobs=20, npoints=10, ny=None):
    """Nonnegative blob + point-source image of shape [ny, n] (row-major, float64)."""
    ny = n if ny is None else ny
    rng = _rng(seed)
    scale = max(n, ny) / 64.0
    img = np.zeros((ny, n))
    yy = np.arange(ny)[:, None]
    xx = np.arange(n)[None, :]
    for _ in range(nblobs):
        cy, cx = rng.uniform(0, ny), rng.uniform(0, n)
        sd = rng.uniform(1.0, 4.0) * scale
        amp = 1.0 - rng.uniform(0.0, 1.0)            # in (0, 1]
        img += amp * np.exp(-((yy - cy) ** 2 + (xx - cx) ** 2) / (2.0 * sd * sd))
    for _ in range(npoints):
        iy, ix = rng.integers(0, ny), rng.integers(0, n)
        img[iy, ix] += 1.0 - rng.uniform(0.0, 1.0)
    return img


def random_images(batch, ny, nx, seed=0):
    """Batch of images uniform in [0, 1)."""
    return _rng(seed).uniform(0.0, 1.0, size=(batch, ny, nx))


def uv_gaussian(m, seed=0, sd=0.25 * np.pi):
    """m points (u, v) in [-pi, pi)^2 from a clipped (redrawn) 2-D Gaussian."""
    rng = _rng(seed)
    out = np.empty((0, 2))
    while len(out) < m:
        cand = rng.normal(0.0, sd, size=(2 * (m - len(out)) + 16, 2))
        ok = np.all((cand >= -np.pi) & (cand < np.pi), axis=1)
        out = np.concatenate([out, cand[ok]])
    return out[:m].copy()


def uv_gaussian_holes(m, seed=0, sd=0.25 * np.pi, nholes=40, hole_radius=(0.05 * np.pi, 0.15 * np.pi),
                      profile_sd=0.5 * np.pi):
    """m points of the clipped 2-D Gaussian coverage with nholes circular holes; returns
    (uv [m, 2], holes [nholes, 3] as (centre u, centre v, radius))."""
    rng = _rng(seed)
    centres = np.empty((0, 2))
    while len(centres) < nholes:
        c = rng.uniform(-np.pi, np.pi, size=(4 * nholes, 2))
        keep = rng.uniform(0.0, 1.0, len(c)) < 1.0 - np.exp(-np.sum(c * c, axis=1) / (2.0 * profile_sd ** 2))
        centres = np.concatenate([centres, c[keep]])
    centres = centres[:nholes]
    radii = rng.uniform(hole_radius[0], hole_radius[1], nholes)
    holes = np.column_stack([centres, radii])

    def outside(p):
        d2 = (p[:, None, 0] - centres[None, :, 0]) ** 2 + (p[:, None, 1] - centres[None, :, 1]) ** 2
        return np.all(d2 >= radii[None, :] ** 2, axis=1)
    out = np.empty((0, 2))
    while len(out) < m:
        cand = rng.normal(0.0, sd, size=(2 * (m - len(out)) + 16, 2))
        ok = np.all((cand >= -np.pi) & (cand < np.pi), axis=1)
        cand = cand[ok]
        keep = np.zeros(len(cand), dtype=bool)
        for a in range(0, len(cand), 1 << 16):
            keep[a:a + (1 << 16)] = outside(cand[a:a + (1 << 16)])
        out = np.concatenate([out, cand[keep]])
    return out[:m].copy(), holes


def uv_radial(m, seed=0, contrast=8.0):
    """m points in the disc r < pi with area density proportional to contrast^(-r/pi)."""
    rng = _rng(seed)
    out = np.empty((0, 2))
    while len(out) < m:
        k = 4 * (m - len(out)) + 64
        r = np.pi * np.sqrt(rng.uniform(0.0, 1.0, k))
        th = rng.uniform(0.0, 2.0 * np.pi, k)
        keep = rng.uniform(0.0, 1.0, k) < contrast ** (-r / np.pi)
        pts = np.stack([r * np.cos(th), r * np.sin(th)], axis=1)[keep]
        ok = np.all((pts >= -np.pi) & (pts < np.pi), axis=1)
        out = np.concatenate([out, pts[ok]])
    return out[:m].copy()


def blocks_equal(uv, d):
    """Equal-count compact blocks: sqrt(d) strips in u, each split into sqrt(d) in v."""
    s = int(round(np.sqrt(d)))
    if s * s != d:
        raise ValueError("equal blocks need a square block count")
    m = len(uv)
    blk = np.empty(m, dtype=np.int32)
    order_u = np.argsort(uv[:, 0], kind="stable")
    strips = np.array_split(order_u, s)
    for a, idx in enumerate(strips):
        sub = idx[np.argsort(uv[idx, 1], kind="stable")]
        for b, piece in enumerate(np.array_split(sub, s)):
            blk[piece] = a * s + b
    return blk


def blocks_annuli(uv, nannuli, nsectors=1):
    """Blocks by equal-width radial annuli over [0, pi), optionally cut into angular sectors."""
    r = np.hypot(uv[:, 0], uv[:, 1])
    ring = np.minimum((r / np.pi * nannuli).astype(np.int64), nannuli - 1)
    if nsectors == 1:
        return ring.astype(np.int32)
    th = np.mod(np.arctan2(uv[:, 1], uv[:, 0]), 2.0 * np.pi)
    sec = np.minimum((th / (2.0 * np.pi) * nsectors).astype(np.int64), nsectors - 1)
    return (ring * nsectors + sec).astype(np.int32)


def complex_noise(m, seed=0):
    """Standard complex normal vector (real and imaginary parts of variance 1/2)."""
    rng = _rng(seed)
    return (rng.normal(size=m) + 1j * rng.normal(size=m)) / np.sqrt(2.0)


def start_vector(ny, nx, seed=0):
    """Random start image for the power method."""
    return _rng(seed).normal(size=(ny, nx))


def uniform_vis(m, seed=0, batch=None):
    """Random complex visibilities (for adjoint tests)."""
    rng = _rng(seed)
    shape = (m,) if batch is None else (batch, m)
    return rng.normal(size=shape) + 1j * rng.normal(size=shape)
