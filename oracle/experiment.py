"""Noise level and data-fidelity bounds of the simulations (oracle; test infrastructure).

Sec. 5 of arXiv:1610.08895: complex Gaussian noise at a given input SNR, and
bounds epsilon_i at the 0.99 quantile of the chi-square law with 2 M_i degrees
of freedom that models the block residual norm. Reading: the noise has
n_m ~ CN(0, sigma_n^2) (each of the real and imaginary parts of variance
sigma_n^2 / 2) with sigma_n = ||Phi x|| / sqrt(M) * 10^(-SNR/20), so
||n_i||^2 = (sigma_n^2 / 2) chi2(2 M_i) and
epsilon_i = sigma_n / sqrt(2) * sqrt(chi2_{0.99}(2 M_i)).
"""
import numpy as np
from scipy.stats import chi2


def noise_sigma(phi_x, snr_db):
    phi_x = np.asarray(phi_x)
    return np.linalg.norm(phi_x) / np.sqrt(phi_x.size) * 10.0 ** (-snr_db / 20.0)


def epsilon_bounds(sigma_n, block_sizes, quantile=0.99):
    m = np.asarray(block_sizes, dtype=np.float64)
    return sigma_n / np.sqrt(2.0) * np.sqrt(chi2.ppf(quantile, 2.0 * m))


def snr_db(x_true, x_hat):
    """SNR = 20 log10(||x|| / ||x - x_hat||) (Sec. 5)."""
    return 20.0 * np.log10(np.linalg.norm(x_true) / np.linalg.norm(x_true - x_hat))
