"""Proximity operators used by Algorithm 1 (oracle; test infrastructure).

* ``proj_l2ball``: P_B of eq. (proj-L2), Sec. 3. The ball is closed: a point with
  ||z - y|| <= eps is returned unchanged.
* ``soft_threshold``: S_alpha of eq. (prox-L1), Sec. 3, componentwise on real
  coefficients; |z| = alpha and z = 0 both give 0.
* ``proj_positive``: P_C of eq. (proj-plus), Sec. 3: Re(z) where Re(z) > 0, else 0.
* ``dual_data_update``: step 8 of Algorithm 1, v + Gb - P_B(v + Gb).
* ``dual_sparsity_update``: step 13 of Algorithm 1, s + w - S_alpha(s + w)
  (alpha scalar, or per coefficient for the reweighted prior).
"""
import numpy as np


def proj_l2ball(z, y, eps):
    """P_B(z) onto {z : ||z - y||_2 <= eps} (eq. proj-L2)."""
    r = z - y
    nr = np.linalg.norm(r)
    if nr > eps:
        return eps * r / nr + y
    return np.array(z, copy=True)


def soft_threshold(z, alpha):
    """S_alpha(z)_k = z_k {|z_k| - alpha_k}_+ / |z_k| for |z_k| > 0, else 0 (eq. prox-L1).

    alpha is a scalar, or an array of z's shape for the weighted l1 norm
    sum_k alpha_k |z_k| (the reweighted prior of SARA, Sec. 2), whose proximity
    operator is the same componentwise shrinkage with per-coefficient sizes."""
    z = np.asarray(z, dtype=np.float64)
    a = np.broadcast_to(np.asarray(alpha, dtype=np.float64), z.shape)
    mag = np.abs(z)
    out = np.zeros_like(z)
    nz = mag > 0
    out[nz] = z[nz] * np.maximum(mag[nz] - a[nz], 0.0) / mag[nz]
    return out


def proj_positive(z):
    """P_C(z)_k = Re(z_k) if Re(z_k) > 0 else 0 (eq. proj-plus)."""
    re = np.real(z)
    return np.where(re > 0, re, 0.0)


def dual_data_update(v, gb, y, eps):
    """Step 8: v_i <- v_i + G_i b_i - P_B(v_i + G_i b_i)."""
    z = v + gb
    return z - proj_l2ball(z, y, eps)


def dual_sparsity_update(s, w, alpha):
    """Step 13: s <- s + w - S_alpha(s + w), with w = Psi^H x~."""
    q = s + w
    return q - soft_threshold(q, alpha)
