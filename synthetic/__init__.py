"""Seeded synthetic inputs shared by the tests, the bench and the oracle checks.

This module only *describes* state-space models and *simulates* observation
series from them with numpy's PCG64 generator.  It holds none of the particle
filter's arithmetic (no weighting, resampling, Philox stream or likelihood):
both the CUDA path and the FP64 oracle receive the same model parameters and
observation arrays from here and do all of the method's work themselves.

Models follow the hidden Markov model of Section 1.1 of Heine, Whiteley and
Cemgil (arXiv 1812.01502):  X_0 ~ pi_0,  X_n | X_{n-1} ~ f,  Y_n | X_n ~ g,
observations for n >= 0.

* ``LinearGaussian``:  X_n = A X_{n-1} + Lq eps,  Y_n = H X_n + Lr w,
  X_0 ~ N(m0, L0 L0^T)   (the paper's experiment in Section 6.1 is the special
  case A = I, Lq = I, H = I, Lr = I/2, m0 = 0, L0 = I).
* ``StochVol``:  X_n = phi X_{n-1} + sigma v_n,  Y_n = beta exp(X_n / 2) w_n,
  X_0 from the stationary law N(0, sigma^2 / (1 - phi^2)).

Workload presets reproduce the shapes of the filtering problems this library
is measured on (state dimension, particle count, radices, horizon).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np

__all__ = [
    "LinearGaussian", "StochVol", "Workload",
    "simulate", "lg_scalar", "lg_dense", "sv_model", "random_walk",
    "workload", "WORKLOADS", "batched_specs", "simulate_batch", "serving_stream",
]


@dataclass
class LinearGaussian:
    """Linear-Gaussian HMM (all matrices float64, row-major)."""
    A: np.ndarray            # d x d transition matrix
    Lq: np.ndarray           # d x d lower-triangular factor of the transition covariance
    H: np.ndarray            # dy x d observation matrix
    Lr: np.ndarray           # dy x dy lower-triangular factor of the observation covariance
    m0: np.ndarray           # d initial mean
    L0: np.ndarray           # d x d lower-triangular factor of the initial covariance
    kind: str = field(default="lg", init=False)

    @property
    def d(self) -> int:
        return self.A.shape[0]

    @property
    def dy(self) -> int:
        return self.H.shape[0]


@dataclass
class StochVol:
    """Univariate stochastic-volatility HMM."""
    phi: float
    sigma: float
    beta: float
    kind: str = field(default="sv", init=False)

    @property
    def d(self) -> int:
        return 1

    @property
    def dy(self) -> int:
        return 1


def lg_scalar(a: float = 0.9, q: float = 1.0, r: float = 1.0) -> LinearGaussian:
    """x_n = a x_{n-1} + N(0, q), y_n = x_n + N(0, r), x_0 ~ N(0, 1)."""
    one = np.ones((1, 1))
    return LinearGaussian(A=a * one, Lq=np.sqrt(q) * one, H=one.copy(),
                          Lr=np.sqrt(r) * one, m0=np.zeros(1), L0=one.copy())


def lg_dense(d: int, seed: int, diag: float = 0.9, offdiag: float = 0.01) -> LinearGaussian:
    """A = diag*I plus seeded off-diagonal N(0, offdiag^2) entries; Q = R = I; H = I."""
    rng = np.random.default_rng(seed)
    z = rng.standard_normal((d, d))
    A = offdiag * z
    np.fill_diagonal(A, diag)
    rho = max(abs(np.linalg.eigvals(A)))
    if rho >= 1.0:
        raise ValueError(f"transition matrix is not stable (spectral radius {rho})")
    eye = np.eye(d)
    return LinearGaussian(A=A, Lq=eye.copy(), H=eye.copy(), Lr=eye.copy(),
                          m0=np.zeros(d), L0=eye.copy())


def random_walk(d: int = 7, obs_std: float = 0.5) -> LinearGaussian:
    """The Gaussian random walk of Section 6.1: A = I, Q = I, R = obs_std^2 I."""
    eye = np.eye(d)
    return LinearGaussian(A=eye.copy(), Lq=eye.copy(), H=eye.copy(), Lr=obs_std * eye,
                          m0=np.zeros(d), L0=eye.copy())


def sv_model(phi: float = 0.98, sigma: float = 0.16, beta: float = 0.7) -> StochVol:
    return StochVol(phi=phi, sigma=sigma, beta=beta)


def simulate(model, T: int, seed: int) -> Tuple[np.ndarray, np.ndarray]:
    """Simulate (x[0:T], y[0:T]) from the HMM with numpy PCG64(seed).

    Returns float64 arrays x of shape (T, d) and y of shape (T, dy).
    """
    rng = np.random.default_rng(seed)
    d, dy = model.d, model.dy
    x = np.empty((T, d))
    y = np.empty((T, dy))
    if model.kind == "lg":
        xt = model.m0 + model.L0 @ rng.standard_normal(d)
        for n in range(T):
            if n > 0:
                xt = model.A @ xt + model.Lq @ rng.standard_normal(d)
            x[n] = xt
            y[n] = model.H @ xt + model.Lr @ rng.standard_normal(dy)
    elif model.kind == "sv":
        sd0 = model.sigma / np.sqrt(1.0 - model.phi ** 2)
        xt = sd0 * rng.standard_normal()
        for n in range(T):
            if n > 0:
                xt = model.phi * xt + model.sigma * rng.standard_normal()
            x[n, 0] = xt
            y[n, 0] = model.beta * np.exp(xt / 2.0) * rng.standard_normal()
    else:
        raise ValueError(model.kind)
    return x, y


@dataclass
class Workload:
    name: str
    model: object
    N: int
    radices: Tuple[int, ...]
    T: int
    data_seed: int
    filter_seed: int

    def observations(self, T: Optional[int] = None) -> np.ndarray:
        """Observation series y[0:T] (float64, shape (T, dy)), simulated with the data seed."""
        return simulate(self.model, self.T if T is None else T, self.data_seed)[1]

    def truth(self, T: Optional[int] = None) -> np.ndarray:
        return simulate(self.model, self.T if T is None else T, self.data_seed)[0]


def _mk(name: str) -> Workload:
    if name == "lg1d_n1024":
        return Workload(name, lg_scalar(), 1 << 10, (2,) * 10, 100, 1, 1000)
    if name == "lg8d_n1m":
        return Workload(name, lg_dense(8, seed=2), 1 << 20, (32, 32, 32, 32), 1000, 2, 2000)
    if name == "sv_n16m":
        return Workload(name, sv_model(), 1 << 24, (16,) * 6, 2000, 3, 3000)
    if name == "rw7d_paper":
        # Section 6.1 workload: d = 7 random walk, R = I/4, n_max = 8000 observations.
        return Workload(name, random_walk(7), 1 << 14, (16, 16, 16, 4), 8000, 7, 7000)
    raise KeyError(name)


WORKLOADS = ("lg1d_n1024", "lg8d_n1m", "sv_n16m", "rw7d_paper")


def workload(name: str) -> Workload:
    """Named workload presets.

    lg1d_n1024 : 1-D LG x=0.9x+N(0,1), y=x+N(0,1), T=100, N=2^10, radix-2 (m=10)
    lg8d_n1m   : 8-D LG, A = 0.9 I + 0.01 N(0,1) off-diagonal, Q=R=I, T=1000, N=2^20, radices (32,)*4
    sv_n16m    : SV phi=0.98, sigma=0.16, beta=0.7, T=2000, N=2^24, radix 16 (m=6)
    rw7d_paper : Section 6.1 random walk, d=7, R=I/4, T=8000
    """
    return _mk(name)


def _factor_radices(N: int, rng: np.random.Generator, allowed=(2, 4, 8, 16, 32)) -> Tuple[int, ...]:
    """A random factorisation of the power of two N into factors drawn from ``allowed``."""
    out: List[int] = []
    rem = N
    while rem > 1:
        choices = [a for a in allowed if rem % a == 0]
        a = int(rng.choice(choices))
        out.append(a)
        rem //= a
    return tuple(out)


def batched_specs(n_filters: int = 4096, T: int = 500, seed: int = 4,
                  dims: Sequence[int] = (1, 4, 8), log2n: Tuple[int, int] = (8, 16)):
    """Independent LG filters with uneven d, N and radices.

    d uniform over ``dims``; N = 2^round(U(log2n)); radices a random factorisation
    of N into {2,4,8,16,32}.  Each filter gets its own model (seeded dense A) and
    its own observation series (data seed derived from ``seed`` and the filter id).
    Returns a list of Workload objects.
    """
    rng = np.random.default_rng(seed)
    specs = []
    for f in range(n_filters):
        d = int(rng.choice(dims))
        ln = int(np.rint(rng.uniform(log2n[0], log2n[1])))
        N = 1 << ln
        radices = _factor_radices(N, rng)
        model = lg_dense(d, seed=seed * 1_000_003 + f) if d > 1 else lg_scalar()
        specs.append(Workload(f"batch{f}", model, N, radices, T,
                              data_seed=seed * 7919 + f, filter_seed=seed * 104729 + f))
    return specs


def simulate_batch(specs, T: int) -> np.ndarray:
    """Observations of many linear-Gaussian workloads at once, vectorised over the
    filters of equal dimension: returns y of shape (F, T, dy_max), zero padded.
    Each filter's series uses its own data seed (numpy PCG64), so it differs from
    ``simulate(model, T, seed)`` draw by draw but has the same law."""
    F = len(specs)
    dy_max = max(w.model.dy for w in specs)
    y = np.zeros((F, T, dy_max))
    by_d = {}
    for f, w in enumerate(specs):
        if w.model.kind != "lg":
            y[f, :, :1] = simulate(w.model, T, w.data_seed)[1]
            continue
        by_d.setdefault((w.model.d, w.model.dy), []).append(f)
    for (d, dy), idx in by_d.items():
        A = np.stack([specs[f].model.A for f in idx])
        Lq = np.stack([specs[f].model.Lq for f in idx])
        H = np.stack([specs[f].model.H for f in idx])
        Lr = np.stack([specs[f].model.Lr for f in idx])
        m0 = np.stack([specs[f].model.m0 for f in idx])
        L0 = np.stack([specs[f].model.L0 for f in idx])
        gens = [np.random.default_rng(specs[f].data_seed) for f in idx]
        eps = np.stack([g.standard_normal((T, d + dy)) for g in gens])       # (Fd, T, d + dy)
        x = m0 + np.einsum("fij,fj->fi", L0, eps[:, 0, :d])
        for n in range(T):
            if n > 0:
                x = np.einsum("fij,fj->fi", A, x) + np.einsum("fij,fj->fi", Lq, eps[:, n, :d])
            y[idx, n, :dy] = np.einsum("fij,fj->fi", H, x) + np.einsum("fij,fj->fi", Lr, eps[:, n, d:])
    return y


def serving_stream(n_requests: int, rate_hz: float, seed: int = 5,
                   log2n: Tuple[int, int] = (10, 20), T_range: Tuple[int, int] = (100, 2000)):
    """Poisson arrival stream of filtering requests.

    Each request: model uniform over {LG d=1, LG d=4, LG d=8, SV}; N = 2^U{log2n};
    radices a random factorisation of N; T uniform in T_range.  Returns a list of
    (arrival_time_s, Workload) sorted by arrival time.
    """
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for r in range(n_requests):
        t += rng.exponential(1.0 / rate_hz)
        kind = int(rng.integers(0, 4))
        ln = int(rng.integers(log2n[0], log2n[1] + 1))
        N = 1 << ln
        radices = _factor_radices(N, rng)
        T = int(rng.integers(T_range[0], T_range[1] + 1))
        if kind == 0:
            model = lg_scalar()
        elif kind == 1:
            model = lg_dense(4, seed=seed * 31 + r)
        elif kind == 2:
            model = lg_dense(8, seed=seed * 31 + r)
        else:
            model = sv_model()
        out.append((t, Workload(f"req{r}", model, N, radices, T,
                                data_seed=seed * 8191 + r, filter_seed=seed * 65537 + r)))
    return out
