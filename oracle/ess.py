"""Effective sample size by Geyer's initial monotone sequence estimator.

TEST AND MEASUREMENT INFRASTRUCTURE (same rules as the rest of ``oracle/``).

For one chain x_1..x_n: normalised autocorrelations rho_t; pair sums
Gamma_m = rho_{2m} + rho_{2m+1}; keep Gamma_m while positive, force them to be
non-increasing, then tau = -1 + 2 sum_m Gamma_m and ESS = n / tau
(Geyer, Statistical Science 7, 1992).  Chains are independent, so the ESS of a
set of chains is the sum of their ESS values.
"""
import numpy as np


def autocorr(x):
    x = np.asarray(x, dtype=np.float64)
    n = x.shape[0]
    x = x - x.mean()
    nfft = 1
    while nfft < 2 * n:
        nfft *= 2
    f = np.fft.rfft(x, nfft)
    acov = np.fft.irfft(f * np.conj(f), nfft)[:n] / n
    if acov[0] <= 0:
        return np.ones(n)
    return acov / acov[0]


def ess_geyer(x):
    """ESS of one scalar chain (length n)."""
    x = np.asarray(x, dtype=np.float64)
    n = x.shape[0]
    if n < 4 or np.all(x == x[0]):
        return 0.0 if n >= 4 else float(n)
    rho = autocorr(x)
    gam = []
    for m in range(n // 2):
        g = rho[2 * m] + rho[2 * m + 1]
        if g <= 0:
            break
        if gam and g > gam[-1]:
            g = gam[-1]
        gam.append(g)
    tau = -1.0 + 2.0 * float(np.sum(gam))
    tau = max(tau, 1.0 / np.log10(max(n, 10)))
    return n / tau


def ess_chains(samples):
    """samples [n][C][k] -> ESS per parameter summed over chains, shape [k]."""
    s = np.asarray(samples, dtype=np.float64)
    n, C, k = s.shape
    out = np.zeros(k)
    for c in range(C):
        for j in range(k):
            out[j] += ess_geyer(s[:, c, j])
    return out


def ess_summary(samples):
    e = ess_chains(samples)
    return {"min": float(e.min()) if e.size else 0.0, "median": float(np.median(e)) if e.size else 0.0}
