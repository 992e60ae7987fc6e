"""FP64 sparsity dictionary Psi: a collection of b orthonormal bases (oracle; test infrastructure).

Sec. 3 of arXiv:1610.08895 takes Psi as a collection of b bases (the SARA
dictionary: the Dirac basis plus the Daubechies wavelets db1..db8). The paper
prints no filter coefficients and no transform convention; the readings used:

* db_p is the minimum-phase spectral factor of the maximally flat half-band
  polynomial (Daubechies 1988): |H(w)|^2 = 2 cos^{2p}(w/2) P(sin^2(w/2)) with
  P(y) = sum_{k<p} C(p-1+k, k) y^k. Coefficients are derived here in FP64.
* Periodic 1-D analysis: a_k = sum_j h_j x_{(2k+j) mod m},
  d_k = sum_j g_j x_{(2k+j) mod m}, with g_j = (-1)^j h_{L-1-j}; synthesis is
  its transpose. Filters longer than the signal wrap modulo m repeatedly.
* 2-D: rows, then columns; L levels; packed layout with the coarsest
  approximation in the top-left corner, so each basis has exactly N coefficients.
* Psi = b^{-1/2} [Psi_1 ... Psi_b], so Psi Psi^H = I and ||Psi||_S = 1.
* Basis id 0 is the Dirac basis (identity); id k in 1..8 is db_k.
"""
import numpy as np
from math import comb


def daubechies_lowpass(p):
    """Low-pass filter h of db_p (length 2p), sum h = sqrt(2), largest tap first."""
    if p == 1:
        return np.array([1.0, 1.0]) / np.sqrt(2.0)
    # P(y), coefficients in decreasing powers of y for np.roots
    poly_y = np.array([comb(p - 1 + k, k) for k in range(p)][::-1], dtype=np.float64)
    y_roots = np.roots(poly_y)
    z_roots = []
    for yr in y_roots:
        # sin^2(w/2) = (2 - z - 1/z)/4 = yr  <=>  z^2 - (2 - 4 yr) z + 1 = 0
        c = 1.0 - 2.0 * yr
        disc = np.sqrt(c * c - 1.0 + 0j)
        z1, z2 = c + disc, c - disc
        z_roots.append(z1 if abs(z1) < 1.0 else z2)   # minimum phase: inside the unit circle
    roots = np.concatenate([-np.ones(p), np.array(z_roots)])
    h = np.real(np.poly(roots))
    return h * (np.sqrt(2.0) / h.sum())


def highpass_from_lowpass(h):
    """Quadrature mirror: g_j = (-1)^j h_{L-1-j}."""
    L = len(h)
    return np.array([(-1) ** j * h[L - 1 - j] for j in range(L)])


def analysis_1d(x, h, axis):
    """One periodic analysis level along ``axis``: returns [a | d] along that axis."""
    g = highpass_from_lowpass(h)
    m = x.shape[axis]
    k = np.arange(m // 2)
    a = 0.0
    d = 0.0
    for j in range(len(h)):
        xs = np.take(x, (2 * k + j) % m, axis=axis)
        a = a + h[j] * xs
        d = d + g[j] * xs
    return np.concatenate([a, d], axis=axis)


def synthesis_1d(c, h, axis):
    """Transpose of ``analysis_1d``: scatter a_k h_j + d_k g_j to position (2k + j) mod m."""
    g = highpass_from_lowpass(h)
    m = c.shape[axis]
    k = np.arange(m // 2)
    a = np.take(c, np.arange(m // 2), axis=axis)
    d = np.take(c, np.arange(m // 2, m), axis=axis)
    x = np.zeros_like(c)
    for j in range(len(h)):
        idx = (2 * k + j) % m        # distinct for a fixed j, so plain fancy-index add is exact
        contrib = h[j] * a + g[j] * d
        if axis == 0:
            x[idx, ...] += contrib
        else:
            x[:, idx] += contrib
    return x


def dwt2(x, h, levels):
    """L-level periodic 2-D analysis (rows then columns), packed Mallat layout."""
    out = np.array(x, dtype=np.float64, copy=True)
    my, mx = out.shape
    for _ in range(levels):
        region = out[:my, :mx]
        region = analysis_1d(region, h, axis=1)
        region = analysis_1d(region, h, axis=0)
        out[:my, :mx] = region
        my //= 2
        mx //= 2
    return out


def idwt2(c, h, levels):
    """Inverse (= transpose) of ``dwt2``."""
    out = np.array(c, dtype=np.float64, copy=True)
    ny, nx = out.shape
    for lev in reversed(range(levels)):
        my, mx = ny >> lev, nx >> lev
        region = out[:my, :mx]
        region = synthesis_1d(region, h, axis=0)
        region = synthesis_1d(region, h, axis=1)
        out[:my, :mx] = region
    return out


def basis_filter(basis_id):
    if basis_id == 0:
        return None
    if not 1 <= basis_id <= 8:
        raise ValueError("basis id must be 0 (Dirac) or 1..8 (db1..db8)")
    return daubechies_lowpass(basis_id)


def psi_j_adj(x, basis_id, levels):
    """Psi_j^T x for one orthonormal basis (no 1/sqrt(b))."""
    h = basis_filter(basis_id)
    return np.array(x, dtype=np.float64, copy=True) if h is None else dwt2(x, h, levels)


def psi_j(c, basis_id, levels):
    """Psi_j c for one orthonormal basis (no 1/sqrt(b))."""
    h = basis_filter(basis_id)
    return np.array(c, dtype=np.float64, copy=True) if h is None else idwt2(c, h, levels)


def psi_adj(x, basis_ids, levels):
    """Psi^H x = b^{-1/2} [Psi_1^T x, ..., Psi_b^T x], shape [b, ny, nx] (Sec. 3)."""
    b = len(basis_ids)
    return np.stack([psi_j_adj(x, j, levels) for j in basis_ids]) / np.sqrt(b)


def psi(s, basis_ids, levels):
    """Psi s = b^{-1/2} sum_j Psi_j s_j, for s of shape [b, ny, nx] (Sec. 3)."""
    b = len(basis_ids)
    return sum(psi_j(s[k], j, levels) for k, j in enumerate(basis_ids)) / np.sqrt(b)
