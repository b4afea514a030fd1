"""Dual-averaging step-size adaptation -- TEST INFRASTRUCTURE ONLY (part of the oracle).

The paper tunes the leapfrog step to about 80% acceptance (Sec. 4.2.3) and prints no
procedure; the reading taken is dual averaging of log eps (Hoffman and Gelman 2014,
Sec. 3.2, the step-size part of their Algorithm 5), driven by the mean over all
chains of the Metropolis acceptance probability min(1, exp(-dH)) of each warm-up
trajectory, a non-finite dH counting as 0.

With m = 1, 2, ... the update number, delta the target and a_m that mean:
    Hbar_m      = (1 - 1/(m + t0)) Hbar_{m-1} + (delta - a_m) / (m + t0),  Hbar_0 = 0
    log eps_m   = mu - sqrt(m) / gamma * Hbar_m,                          mu = log(10 eps_0)
    log ebar_m  = m^-kappa log eps_m + (1 - m^-kappa) log ebar_{m-1},     log ebar_0 = 0
eps_m is the step of trajectory m + 1; ebar_n, after the last update, is the step kept.
Plain float64 Python, one update at a time.
"""
import math

import numpy as np

GAMMA, T0, KAPPA = 0.05, 10.0, 0.75


def accept_stat(dH_row):
    """Mean over chains of min(1, exp(-dH)); a non-finite dH contributes 0."""
    tot = 0.0
    for v in np.asarray(dH_row, dtype=np.float64).ravel():
        if math.isfinite(v):
            tot += 1.0 if v <= 0.0 else math.exp(-v)    # min(1, e^-v) without overflowing e^-v
    return tot / np.asarray(dH_row).size


class DualAveraging:
    """The recursion above, one update at a time."""

    def __init__(self, eps0, target, gamma=GAMMA, t0=T0, kappa=KAPPA):
        self.mu = math.log(10.0 * eps0)
        self.target, self.gamma, self.t0, self.kappa = target, gamma, t0, kappa
        self.m, self.hbar, self.lbar = 0, 0.0, 0.0

    def update(self, a):
        """One update with acceptance statistic a; returns (eps_m, ebar_m)."""
        self.m += 1
        m = self.m
        w = 1.0 / (m + self.t0)
        self.hbar = (1.0 - w) * self.hbar + w * (self.target - a)
        log_eps = self.mu - math.sqrt(m) / self.gamma * self.hbar
        eta = m ** (-self.kappa)
        self.lbar = eta * log_eps + (1.0 - eta) * self.lbar
        return math.exp(log_eps), math.exp(self.lbar)


def dual_averaging(stats, eps0, target, gamma=GAMMA, t0=T0, kappa=KAPPA):
    """Step sizes after each update for the acceptance statistics a_1..a_n:
    returns [n][2] = (eps_m, ebar_m)."""
    da = DualAveraging(eps0, target, gamma, t0, kappa)
    out = np.zeros((len(stats), 2))
    for i, a in enumerate(stats):
        out[i] = da.update(a)
    return out


def dual_averaging_dH(dH, eps0, target):
    """dual_averaging() on the statistics of energy errors dH[n][chains]."""
    return dual_averaging([accept_stat(r) for r in dH], eps0, target)


def warmup(orc, q, L, eps0, n, target, seed, first_traj, problem=0):
    """The whole warm-up on the oracle: trajectory m (index first_traj + m - 1) from the
    current chain states with the current step, then one update; `problem` selects the
    random stream (a problem of a batch draws from its own).  Returns the [n][2] trace
    and the final states."""
    q = np.array(q, dtype=np.float64)
    da = DualAveraging(eps0, target)
    eps = eps0
    out = np.zeros((n, 2))
    for m in range(1, n + 1):
        _, _, dH, q = orc.sample(q, eps, L, 1, seed=seed, first_traj=first_traj + m - 1, problem=problem)
        out[m - 1] = da.update(accept_stat(dH[0]))
        eps = out[m - 1, 0]
    return out, q
