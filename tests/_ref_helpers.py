"""Independent brute-force helpers for pinning the oracle (test code only).

Nothing here is shared with the oracle or with the CUDA path: each helper is
the textbook definition of a quantity, written with numpy.
"""
from __future__ import annotations

import itertools
import math

import numpy as np


def all_label_vectors(M: int, nt: int) -> np.ndarray:
    """Every vector of Q^nt as labels, shape [M^nt][nt] (user order)."""
    return np.array(list(itertools.product(range(M), repeat=nt)), dtype=np.int64)


def ml_metrics(H: np.ndarray, y: np.ndarray, cand_syms: np.ndarray) -> np.ndarray:
    """||y - H s||^2 for every candidate symbol vector (rows of cand_syms)."""
    r = y[None, :] - cand_syms @ H.T
    return np.sum(np.abs(r) ** 2, axis=1)


def bit_of(labels, b: int, B: int):
    return (np.asarray(labels) >> (B - 1 - b)) & 1


def maxlog_llr_bruteforce(metrics: np.ndarray, cand_labels: np.ndarray, B: int, sigma2: float,
                          llr_max: float) -> np.ndarray:
    """Max-log LLR per (user, bit) from a candidate list; positive means bit 0."""
    nt = cand_labels.shape[1]
    out = np.zeros((nt, B))
    for k in range(nt):
        for b in range(B):
            bits = bit_of(cand_labels[:, k], b, B)
            m1 = metrics[bits == 1].min() if np.any(bits == 1) else np.inf
            m0 = metrics[bits == 0].min() if np.any(bits == 0) else np.inf
            if np.isinf(m1):
                out[k, b] = llr_max
            elif np.isinf(m0):
                out[k, b] = -llr_max
            else:
                out[k, b] = (m1 - m0) / sigma2
    return out


def qfunc(x: float) -> float:
    return 0.5 * math.erfc(x / math.sqrt(2.0))


def mrc_rayleigh_bpsk_ber(gamma_b: float, L: int) -> float:
    """Closed-form BER of coherent BPSK with L-branch MRC over i.i.d. Rayleigh
    fading (Proakis, Digital Communications, eq. 14.4-15), gamma_b = average
    SNR per bit per branch."""
    mu = math.sqrt(gamma_b / (1.0 + gamma_b))
    s = 0.0
    for k in range(L):
        s += math.comb(L - 1 + k, k) * ((1.0 + mu) / 2.0) ** k
    return ((1.0 - mu) / 2.0) ** L * s
