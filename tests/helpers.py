"""Shared test helpers: golden-fixture loader and textbook closed forms.

The closed forms here (Black, Bachelier, CEV) are the independent references the
oracle's special cases are checked against; they are not part of the method.
"""
import os

import numpy as np
from scipy.stats import norm

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


class Golden:
    def __init__(self, name):
        self.meta = {}
        self.rows = []
        with open(os.path.join(GOLDEN, name)) as fh:
            for line in fh:
                line = line.strip()
                if not line or line.startswith("#"):
                    continue
                head, *rest = line.split()
                try:
                    self.rows.append([float(head)] + [float(x) for x in rest])
                except ValueError:
                    self.meta[head] = rest
        self.rows = np.array(self.rows)

    def floats(self, key):
        return [float(x) for x in self.meta[key]]


def black_call(f, K, T, sigma):
    s = sigma * np.sqrt(T)
    d1 = (np.log(f / K) + 0.5 * s * s) / s
    return f * norm.cdf(d1) - K * norm.cdf(d1 - s)


def bachelier_call(f, K, T, sigma_n):
    s = sigma_n * np.sqrt(T)
    d = (f - K) / s
    return (f - K) * norm.cdf(d) + s * norm.pdf(d)


def cev_call(f, K, T, alpha, beta):
    """Call on dF = alpha F^beta dW (SABR with nu = 0), 0 <= beta < 1, F
    absorbed at 0.  Y = F^(2(1-beta)) / (alpha (1-beta))^2 is a squared
    Bessel process of dimension delta = (1 - 2 beta)/(1 - beta) (Ito); the
    process absorbed at 0 is the h-transform, h(y) = y^((2-delta)/2), of the
    squared Bessel process of dimension 4 - delta, whose Y_T/T is noncentral
    chi-square (4 - delta degrees, noncentrality Y_0/T).  With
    (Y_0/Y)^((2-delta)/2) = f/F this gives
        E[(F_T - K)^+] = f E'[(1 - K/F_T)^+]
    under the dimension 4 - delta law, evaluated here by one quadrature."""
    from scipy.integrate import quad
    from scipy.stats import ncx2
    b1 = 1.0 - beta
    c = 1.0 / (alpha * b1) ** 2
    k = (3.0 - 2.0 * beta) / b1
    lam = c * f ** (2 * b1) / T
    uK = c * K ** (2 * b1) / T
    hi = lam + k + 60.0 * np.sqrt(2 * (k + 2 * lam))
    inv_f = lambda u: ((u * T / c) ** (-1.0 / (2 * b1)))  # 1 / F at Y = u T
    tail, _ = quad(lambda u: ncx2.pdf(u, k, lam) * inv_f(u), uK, hi, limit=400, epsabs=1e-14, epsrel=1e-10)
    return f * (ncx2.sf(uK, k, lam) - K * tail)


# Exact law of the Sec. 6.3 cliquet when the forward is a geometric Brownian
# motion (SABR with nu = 0, beta = 1): the local returns are i.i.d. with
# 1 + R lognormal of mean 1.
def clipped_return_pmf(sigma, dt, fl, cl, n_cells):
    """Law of max(min(R, cl), fl) on the grid fl + j (cl - fl)/n_cells: atoms
    at both ends, each cell's mass split between its two end nodes."""
    s = sigma * np.sqrt(dt)
    x = np.linspace(fl, cl, n_cells + 1)
    cdf = norm.cdf((np.log1p(x) + 0.5 * s * s) / s)  # P(R <= x)
    pmf = np.zeros(n_cells + 1)
    cell = np.diff(cdf)
    pmf[:-1] += 0.5 * cell
    pmf[1:] += 0.5 * cell
    pmf[0] += cdf[0]
    pmf[-1] += 1.0 - cdf[-1]
    return x, pmf


def exact_gbm_cliquet(sigma, T, n_resets, fl, cl, fg, cg, n_cells=4000):
    dt = T / n_resets
    x, pmf = clipped_return_pmf(sigma, dt, fl, cl, n_cells)
    tot = pmf
    for _ in range(n_resets - 2):
        tot = np.convolve(tot, pmf)
    k = n_resets - 1
    grid = k * fl + (cl - fl) / n_cells * np.arange(tot.size)
    return float(np.sum(tot * np.clip(grid, fg, cg)))
