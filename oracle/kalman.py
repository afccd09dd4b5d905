"""Kalman filter (FP64): the exact filter for linear-Gaussian models.

Section 6.1 measures every particle filter against the Kalman recursions
(Kalman, 1960) on a model where they are exact.  For

    X_0 ~ N(m0, P0),  X_n = A X_{n-1} + eta_n (cov Q),  Y_n = H X_n + eps_n (cov R),  n >= 0,

the recursion (prediction -> update) gives the filtering mean E[X_n | y_0..y_n],
its covariance, and log p(y_0..y_{T-1}) = sum_n log N(y_n; H m_pred, H P_pred H^T + R).
"""
from __future__ import annotations

import numpy as np


def kalman_filter(model, y: np.ndarray):
    """Returns dict(mean (T,d), cov (T,d,d), loglik float, inc (T,))."""
    y = np.asarray(y, dtype=np.float64).reshape(len(y), -1)
    T = y.shape[0]
    A, H = model.A, model.H
    Q = model.Lq @ model.Lq.T
    R = model.Lr @ model.Lr.T
    m = model.m0.astype(np.float64).copy()
    P = model.L0 @ model.L0.T
    d = A.shape[0]
    means = np.empty((T, d))
    covs = np.empty((T, d, d))
    incs = np.empty(T)
    for n in range(T):
        if n > 0:
            m = A @ m
            P = A @ P @ A.T + Q
        S = H @ P @ H.T + R
        resid = y[n] - H @ m
        Sc = np.linalg.cholesky(S)
        z = np.linalg.solve(Sc, resid)
        incs[n] = -0.5 * z @ z - np.sum(np.log(np.diag(Sc))) - 0.5 * len(resid) * np.log(2 * np.pi)
        K = np.linalg.solve(S, H @ P).T          # P H^T S^{-1}  (S, P symmetric)
        m = m + K @ resid
        P = P - K @ S @ K.T
        P = 0.5 * (P + P.T)
        means[n], covs[n] = m, P
    return dict(mean=means, cov=covs, inc=incs, loglik=float(np.sum(incs)))
