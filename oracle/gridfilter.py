"""Point-mass (grid) filter for one-dimensional state-space models (FP64).

The stochastic-volatility model has no closed-form filter; a deterministic
quadrature filter on a fine uniform grid is its near-exact reference (a
reading of this library: the paper evaluates only on a linear-Gaussian model,
Section 6.1).  On a grid x_1..x_G with spacing h:

    predict:  p_n(x_i) = sum_j phi_f(x_i | x_j) p~_{n-1}(x_j) h
    update:   p~_n(x_i) = p_n(x_i) g(x_i, y_n) / Z_n,   Z_n = sum_i p_n(x_i) g(x_i, y_n) h

and log p(y_0..y_{T-1}) = sum_n log Z_n.  The transition density phi_f is a
Gaussian N(phi x_j, sigma^2) (SV) or N(a x_j, q) (scalar linear-Gaussian).
"""
from __future__ import annotations

import numpy as np


def _gauss(x, m, var):
    return np.exp(-0.5 * (x - m) ** 2 / var) / np.sqrt(2 * np.pi * var)


def grid_filter_1d(trans_coef: float, trans_var: float, init_mean: float, init_var: float,
                   log_g, y: np.ndarray, lo: float, hi: float, G: int = 4096):
    """Generic 1-D grid filter.  log_g(x_grid, y_n) -> log density of y_n given x."""
    y = np.asarray(y, dtype=np.float64).reshape(len(y), -1)
    x = np.linspace(lo, hi, G)
    h = x[1] - x[0]
    K = _gauss(x[:, None], trans_coef * x[None, :], trans_var) * h   # K[i, j] = f(x_i | x_j) h
    p = _gauss(x, init_mean, init_var)
    T = y.shape[0]
    means = np.empty(T)
    incs = np.empty(T)
    for n in range(T):
        if n > 0:
            p = K @ p
        lg = log_g(x, y[n])
        mx = np.max(lg)
        w = p * np.exp(lg - mx)
        Z = np.sum(w) * h
        incs[n] = np.log(Z) + mx
        p = w / Z
        means[n] = np.sum(p * x) * h
    return dict(mean=means[:, None], inc=incs, loglik=float(np.sum(incs)))


def sv_grid_filter(model, y: np.ndarray, G: int = 4096, width: float = 8.0):
    """Grid filter for the SV model on [-width, width] stationary standard deviations."""
    sd0 = model.sigma / np.sqrt(1.0 - model.phi ** 2)
    beta2 = model.beta ** 2

    def log_g(x, yn):
        yy = float(yn[0])
        return -0.5 * np.log(2 * np.pi * beta2) - 0.5 * x - yy * yy * np.exp(-x) / (2 * beta2)

    return grid_filter_1d(model.phi, model.sigma ** 2, 0.0, sd0 ** 2, log_g, y,
                          -width * sd0, width * sd0, G)


def lg_scalar_grid_filter(model, y: np.ndarray, G: int = 4096, width: float = 10.0):
    """Grid filter for a scalar linear-Gaussian model (used to pin the grid filter to Kalman)."""
    a = float(model.A[0, 0])
    q = float(model.Lq[0, 0] ** 2)
    hcoef = float(model.H[0, 0])
    r = float(model.Lr[0, 0] ** 2)
    v0 = float(model.L0[0, 0] ** 2)
    m0 = float(model.m0[0])
    sd = np.sqrt(max(v0, q / max(1e-12, 1 - a * a)))

    def log_g(x, yn):
        return -0.5 * np.log(2 * np.pi * r) - 0.5 * (float(yn[0]) - hcoef * x) ** 2 / r

    return grid_filter_1d(a, q, m0, v0, log_g, y, m0 - width * sd, m0 + width * sd, G)
