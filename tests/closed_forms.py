"""Closed forms used as references by several tests (test code only)."""
import math

import numpy as np


def dirichlet(N, S):
    """Closed form of the geometric series sum_{n=0}^{N-1} exp(2 i pi S n).

    n is an integer, so only sigma = S - rint(S) matters:
    exp(i pi (N-1) sigma) sin(pi N sigma) / sin(pi sigma), with the series
    N (1 - pi^2 (N^2-1) sigma^2 / 6) for |sigma| < 1e-9."""
    S = np.asarray(S, dtype=np.float64)
    sig = S - np.rint(S)
    small = np.abs(sig) < 1e-9
    with np.errstate(invalid="ignore", divide="ignore"):
        ratio = np.where(small, N * (1.0 - (math.pi ** 2) * (N * N - 1) * sig * sig / 6.0),
                         np.sin(math.pi * N * sig) / np.sin(math.pi * sig))
    return np.exp(1j * math.pi * (N - 1) * sig) * ratio


def parallelepiped_closed_form(n, S):
    """Amplitude of n[0] x n[1] x n[2] atoms at integer positions 0..n-1, f=1."""
    S = np.asarray(S)
    return dirichlet(n[0], S[:, 0]) * dirichlet(n[1], S[:, 1]) * dirichlet(n[2], S[:, 2])


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))
