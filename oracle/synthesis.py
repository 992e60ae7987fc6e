"""Synthesis formulation solved by randomised primal-dual iterations, FP64 (oracle; test infrastructure).

Sec. 2 names, besides the analysis problem (analysis-l1-problem) that Algorithm 1
solves, a synthesis approach: the image is x = Psi alpha and the sparsity prior acts
on the coefficients alpha themselves. Here that problem is

    minimise_alpha  kappa ||alpha||_1
    subject to      ||y_i - Phi_i Psi alpha||_2 <= eps_i for every block i,  Psi alpha >= 0,

with Psi = b^{-1/2} [Psi_1 ... Psi_b] the same normalised dictionary. It is solved by
the forward-backward primal-dual template of Algorithm 1 (Sec. 3) with the roles of
the two non-smooth terms exchanged: the l1 norm is now a function of the primal
variable (its proximity operator, the soft threshold of eq. prox-L1, is the primal
step), and positivity of Psi alpha becomes a dual variable u (the indicator of the
positive orthant, whose conjugate's proximity operator is z - P_C(z) = min(z, 0)).
Per iteration t, in the order of Algorithm 1:

  3.     draw the active blocks (the same Philox draws, stream 0);
  4.     x~ = Psi alpha~ and b~ = F Z x~;
  5-8.   v_i <- v_i + G_i b~ - P_B(v_i + G_i b~) for the active blocks (inactive keep v_i);
  13'.   u <- min(u + x~, 0);
  17'.   alpha <- S_{tau kappa}(alpha - tau Psi^H(sigma u + varsigma Re(Phi^H v)));
  18.    alpha~ = 2 alpha^(t) - alpha^(t-1).

Start values are zero. The step sizes obey the same condition as Algorithm 1 with
||Psi|| = 1 (tau (sigma ||Psi||^2 + varsigma ||Phi Psi||^2) < 1, e.g. sigma = 1,
varsigma = 1/||Phi||^2, tau = 0.49). The sparsity bases are not drawn at random here:
the coefficients are primal, all of them are updated every iteration.
"""
import numpy as np

from . import philox as _philox
from . import prox as _prox


class SynthesisState:
    """alpha, alpha~ (coefficients [b][ny][nx]), the data duals v and the positivity dual u."""

    def __init__(self, problem):
        g = problem.geom
        b = len(problem.basis_ids)
        self.alpha = np.zeros((b, g.ny, g.nx))
        self.alpha_tilde = np.zeros((b, g.ny, g.nx))
        self.v = np.zeros(len(problem.uv), dtype=np.complex128)
        self.u = np.zeros((g.ny, g.nx))
        self.t = 0

    def x(self, problem):
        """The image Psi alpha."""
        return problem.psi(self.alpha)


def synthesis_iteration(problem, st, tau, sigma, varsigma, kappa, seed, p_block):
    """One iteration of the synthesis form (steps above); returns the active blocks."""
    st.t += 1
    active = _philox.active_set(seed, st.t, _philox.STREAM_BLOCKS, p_block)
    g = problem.geom
    x_tilde = problem.psi(st.alpha_tilde)                                   # step 4
    b_tilde = g.fft(g.zpad(x_tilde))
    for i in range(problem.nblocks):                                        # steps 5-8
        if not active[i]:
            continue
        ix = problem.block_index[i]
        gb = problem.degrid_rows(b_tilde, ix)
        st.v[ix] = _prox.dual_data_update(st.v[ix], gb, problem.y[ix], problem.eps[i])
    z = st.u + x_tilde                                                      # step 13'
    st.u = z - _prox.proj_positive(z)
    back = np.real(g.zpad_adj(g.fft_adj(problem.grid_all(st.v))))          # Re(Phi^H v)
    grad = problem.psi_adj(sigma * st.u + varsigma * back)
    alpha_new = _prox.soft_threshold(st.alpha - tau * grad, tau * kappa)    # step 17'
    st.alpha_tilde = 2.0 * alpha_new - st.alpha                             # step 18
    st.alpha = alpha_new
    return active


def synthesis_run(problem, niter, tau, sigma, varsigma, kappa, seed, p_block, state=None):
    st = SynthesisState(problem) if state is None else state
    draws = [synthesis_iteration(problem, st, tau, sigma, varsigma, kappa, seed, p_block) for _ in range(niter)]
    return st, draws
