"""Shared test helpers: golden-fixture loader and textbook closed forms.

The closed forms here (Black, Bachelier) are the independent references the
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
