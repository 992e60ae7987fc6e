"""Algorithm 1 (randomised forward-backward primal-dual, PD-R) in FP64 (oracle; test infrastructure).

Follows Sec. 3 of arXiv:1610.08895 step by step, in the paper's order and
notation. Plain choices where the paper is silent:

* Initial values x^(0), x~^(0), s^(0), v^(0) are all zero, so v~^(0) = G^T v^(0) = 0.
* Step 11 keeps v_i and v~_i = G_i^T v_i of inactive blocks. The sum
  sum_i M_i^T v~_i in step 17 is therefore G^T v over all blocks, and the oracle
  recomputes it in full every iteration from the current v.
* The soft-threshold size is kappa ||Psi||_S (step 13).
* Sparsity bases can also be drawn at random (probability p_basis_j); an
  inactive basis keeps s_j, mirroring step 11 for the data blocks. With all
  p_basis_j = 1 this is exactly step 13 of the paper.
* For adaptive probabilities (Sec. 4), c_i uses the residual norm
  ||G_i b_i - y_i|| computed in step 8 of the last iteration in which block i
  was active (that is, Phi_i applied to x~ of the previous iteration); the
  initial norms come from one full pass with x^(0). p^(t) is computed before the
  draw of iteration t. With adaptive["exact"] the norms are instead
  ||Phi_i x^(t) - y_i|| of the primal iterate after every iteration, for all
  blocks (Sec. 4 defines c_i on Phi_i x^(t); this costs one full Phi per iteration).
* The stopping rule "until convergence" (step 19) is a fixed iteration count.
* Reweighted analysis prior (SARA, cited in Sec. 2 but not defined there): with
  weights W (one per coefficient of Psi^H x, all in (0, 1]) the objective is
  ||W Psi^H x||_1, and step 13 becomes the weighted soft threshold of size
  kappa ||Psi||_S W. ``sara_weights`` gives the usual reweighting rule
  W = delta / (delta + |Psi^H x|) (reweighted l1, Candes, Wakin and Boyd 2008, as used
  by SARA) for the caller's delta; the outer loop that recomputes W and lowers delta
  between runs of Algorithm 1 is the caller's.
"""
import numpy as np

from . import adaptive as _adaptive
from . import philox as _philox
from . import prox as _prox
from . import wavelets as _wav


class Problem:
    """Data of problem (basic-min-problem): geometry, uv, blocks, Psi, y, epsilon."""

    def __init__(self, geom, uv, block_of_vis, nblocks, basis_ids, levels, y=None, eps=None, dde=None):
        self.geom = geom
        # optional Fourier-domain DDE kernels [M][d][d] of the DDE-aware G (Sec. 2)
        self.dde = None if dde is None else np.asarray(dde, dtype=np.complex128)
        self.uv = np.asarray(uv, dtype=np.float64)
        self.block_of_vis = np.asarray(block_of_vis, dtype=np.int64)
        self.nblocks = int(nblocks)
        self.basis_ids = list(basis_ids)
        self.levels = int(levels)
        self.block_index = [np.nonzero(self.block_of_vis == i)[0] for i in range(self.nblocks)]
        self.y = None if y is None else np.asarray(y, dtype=np.complex128)
        self.eps = None if eps is None else np.asarray(eps, dtype=np.float64)

    # G restricted to the visibilities ix (G_i of eq. data-split), and G^H of all of them
    def degrid_rows(self, grid, ix):
        if self.dde is None:
            return self.geom.degrid(grid, self.uv[ix])
        return self.geom.degrid_dde(grid, self.uv[ix], self.dde[ix])

    def grid_all(self, v):
        if self.dde is None:
            return self.geom.grid(v, self.uv)
        return self.geom.grid_dde(v, self.uv, self.dde)

    # operators of the split problem (eq. data-split)
    def phi(self, x):
        g = self.geom
        return self.degrid_rows(g.fft(g.zpad(x)), np.arange(len(self.uv)))

    def phi_adj(self, y):
        g = self.geom
        return np.real(g.zpad_adj(g.fft_adj(self.grid_all(y))))

    def psi_adj(self, x):
        return _wav.psi_adj(x, self.basis_ids, self.levels)

    def psi(self, s):
        return _wav.psi(s, self.basis_ids, self.levels)


def power_method(apply_normal, x0, max_iter=1000, tol=1e-10):
    """Largest eigenvalue of a symmetric positive operator A (Sec. 5: norms by the power method).

    x <- A x / ||A x||; the estimate is ||A x|| for the unit-norm iterate.
    Returns (lambda, iterations). ||Phi||_S^2 = lambda for A = Re(Phi^H Phi).
    """
    x = np.asarray(x0, dtype=np.float64)
    x = x / np.linalg.norm(x)
    lam_prev = 0.0
    lam = 0.0
    for k in range(1, max_iter + 1):
        z = apply_normal(x)
        lam = np.linalg.norm(z)
        if lam == 0.0:
            return 0.0, k
        x = z / lam
        if abs(lam - lam_prev) <= tol * lam:
            return lam, k
        lam_prev = lam
    return lam, max_iter


def operator_norms(problem, x0, max_iter=1000, tol=1e-10):
    """(||Phi||_S^2, ||Psi||_S^2) by the power method from the start image x0."""
    phi2, _ = power_method(lambda x: problem.phi_adj(problem.phi(x)), x0, max_iter, tol)
    psi2, _ = power_method(lambda x: problem.psi(problem.psi_adj(x)), x0, max_iter, tol)
    return phi2, psi2


class PDState:
    """Primal and dual variables of Algorithm 1."""

    def __init__(self, problem):
        g = problem.geom
        self.x = np.zeros((g.ny, g.nx))
        self.x_tilde = np.zeros((g.ny, g.nx))
        self.s = np.zeros((len(problem.basis_ids), g.ny, g.nx))
        self.v = np.zeros(len(problem.uv), dtype=np.complex128)
        self.t = 0
        # residual norms ||Phi_i x^(0) - y_i|| for the adaptive probabilities
        r = problem.phi(self.x) - problem.y
        self.res_norm = np.array([np.linalg.norm(r[ix]) for ix in problem.block_index])


def pd_iteration(problem, st, tau, sigma, varsigma, kappa, psi_norm, seed,
                 p_block, p_basis, adaptive=None, weights=None):
    """One iteration t of Algorithm 1 (steps 3-18). Returns the active sets drawn.
    weights: None, or [b][ny][nx] per-coefficient weights of the reweighted prior."""
    st.t += 1
    t = st.t
    # step 3: generate the active set (Sec. 3; Sec. 4 for adaptive p)
    if adaptive is not None:
        c = _adaptive.residual_distance(st.res_norm, problem.eps)
        p_block = _adaptive.probabilities(c, adaptive["n"], adaptive["p_min"], adaptive["p_max"])
    active = _philox.active_set(seed, t, _philox.STREAM_BLOCKS, p_block)
    active_basis = _philox.active_set(seed, t, _philox.STREAM_BASES, p_basis)
    # step 4: b~ = F Z x~^(t-1)
    b_tilde = problem.geom.fft(problem.geom.zpad(st.x_tilde))
    # steps 5-9 for i in A; step 11 (inactive blocks keep v_i) is implicit
    for i in range(problem.nblocks):
        if not active[i]:
            continue
        ix = problem.block_index[i]
        gb = problem.degrid_rows(b_tilde, ix)                                  # G_i M_i b~
        st.res_norm[i] = np.linalg.norm(gb - problem.y[ix])
        st.v[ix] = _prox.dual_data_update(st.v[ix], gb, problem.y[ix], problem.eps[i])   # step 8
    # step 13 for the active sparsity bases
    alpha = kappa * psi_norm
    b = len(problem.basis_ids)
    for k, j in enumerate(problem.basis_ids):
        if not active_basis[k]:
            continue
        w = _wav.psi_j_adj(st.x_tilde, j, problem.levels) / np.sqrt(b)            # (Psi^H x~)_j
        st.s[k] = _prox.dual_sparsity_update(st.s[k], w, alpha if weights is None else alpha * weights[k])
    # step 14: s~ = Psi s
    s_tilde = problem.psi(st.s)
    # step 9 / 17: sum_i M_i^T v~_i = G^T v, then Z^T F^H
    back = np.real(problem.geom.zpad_adj(problem.geom.fft_adj(problem.grid_all(st.v))))
    # step 17: primal update with the positivity projection
    x_new = _prox.proj_positive(st.x - tau * (sigma * s_tilde + varsigma * back))
    # step 18: over-relaxation
    st.x_tilde = 2.0 * x_new - st.x
    st.x = x_new
    if adaptive is not None and adaptive.get("exact", False):
        # Sec. 4, exact reading: c_i for the next draw from Phi_i x^(t) of every block
        st.res_norm = block_residuals(problem, st.x)
    return active, active_basis


def pd_run(problem, niter, tau, sigma, varsigma, kappa, psi_norm, seed,
           p_block, p_basis, adaptive=None, state=None, weights=None):
    """Run ``niter`` iterations of Algorithm 1; returns (state, list of active sets)."""
    st = PDState(problem) if state is None else state
    draws = []
    for _ in range(niter):
        draws.append(pd_iteration(problem, st, tau, sigma, varsigma, kappa, psi_norm, seed,
                                  p_block, p_basis, adaptive, weights))
    return st, draws


def sara_weights(problem, x, delta):
    """Reweighting rule of the reweighted analysis prior: W = delta / (delta + |Psi^H x|),
    per coefficient of the normalised dictionary Psi = b^{-1/2} [Psi_1 ... Psi_b]."""
    return delta / (delta + np.abs(problem.psi_adj(x)))


def objective(problem, x):
    """||Psi^H x||_1 (the objective of problem analysis-l1 under the constraints)."""
    return np.abs(problem.psi_adj(x)).sum()


def block_residuals(problem, x):
    r = problem.phi(x) - problem.y
    return np.array([np.linalg.norm(r[ix]) for ix in problem.block_index])
