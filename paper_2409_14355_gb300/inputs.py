"""Seeded synthetic slots for the MPNL uplink: channel, transmit symbols, noise.

This module models the transmitter and the radio channel only; it holds none
of the detector's arithmetic.  Both the CUDA path and the FP64 oracle are fed
from it.

* Transmit symbols: uniform random bits, Gray-mapped per 3GPP TS 38.211
  §5.1.3-5.1.5 (written here from the standard's mapping formulas; the
  detector sides carry their own independent copies).
* Channel: one H per subcarrier, constant over the 14 OFDM symbols of a slot
  (the paper's 30 km/h at 3.5 GHz gives a coherence time of about 4 ms, far
  above the 0.5 ms slot, §III-B).  Either i.i.d. CN(0, 1) Rayleigh or the
  Kronecker model H = L_r H_w L_t^H with exponential correlation
  [rho^|i-j|] at both ends.  These stand in for the CDL-B/CDL-D channels of
  §III-A, whose generator is not available.
* Noise: CN(0, sigma2 I) with sigma2 = Nt / SNR (SNR per receive antenna,
  E|h|^2 = 1, unit-energy symbols).
* Seed: numpy PCG64 with seed = 240914355 + 1000 * config + snr_index.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

SEED_BASE = 240914355
BITS = {4: 2, 16: 4, 64: 6}


def seed_for(config: int, snr_index: int = 0) -> int:
    return SEED_BASE + 1000 * config + snr_index


def tx_constellation(qam: int) -> np.ndarray:
    """Label-indexed TS 38.211 Gray constellation, unit average energy."""
    B = BITS[qam]
    labels = np.arange(qam)
    b = [(labels >> (B - 1 - i)) & 1 for i in range(B)]
    s = [1 - 2 * x for x in b]  # 1 - 2 b_i
    if qam == 4:
        re, im, scale = s[0], s[1], np.sqrt(2.0)
    elif qam == 16:
        re = s[0] * (2 - s[2])
        im = s[1] * (2 - s[3])
        scale = np.sqrt(10.0)
    else:
        re = s[0] * (4 - s[2] * (2 - s[4]))
        im = s[1] * (4 - s[3] * (2 - s[5]))
        scale = np.sqrt(42.0)
    return (re + 1j * im).astype(np.complex128) / scale


def exp_corr_chol(n: int, rho: float) -> np.ndarray:
    idx = np.arange(n)
    C = rho ** np.abs(idx[:, None] - idx[None, :])
    return np.linalg.cholesky(C)


@dataclass
class Slot:
    H: np.ndarray        # complex64 [n_sc][nr][nt]
    Y: np.ndarray        # complex64 [n_sc][n_sym][nr]
    labels: np.ndarray   # uint8 [n_sc][n_sym][nt] transmitted symbol labels
    sigma2: float
    nr: int
    nt: int
    qam: int
    snr_db: float

    @property
    def n_sc(self) -> int:
        return self.H.shape[0]

    @property
    def n_sym(self) -> int:
        return self.Y.shape[1]


def make_slot(nr: int, nt: int, qam: int, n_sc: int, n_sym: int = 14, snr_db: float = 10.0,
              channel: str = "iid", rho: float = 0.3, seed: int = SEED_BASE,
              noise: bool = True) -> Slot:
    rng = np.random.Generator(np.random.PCG64(seed))
    g = (rng.standard_normal((n_sc, nr, nt)) + 1j * rng.standard_normal((n_sc, nr, nt))) / np.sqrt(2)
    if channel == "iid":
        H = g
    elif channel == "kronecker":
        Lr = exp_corr_chol(nr, rho)
        Lt = exp_corr_chol(nt, rho)
        H = Lr[None] @ g @ Lt.conj().T[None]
    else:
        raise ValueError(f"unknown channel model {channel!r}")
    labels = rng.integers(0, qam, size=(n_sc, n_sym, nt), dtype=np.int64)
    s = tx_constellation(qam)[labels]                       # [n_sc][n_sym][nt]
    snr_lin = 10.0 ** (snr_db / 10.0)
    sigma2 = nt / snr_lin
    Y = np.einsum("crt,cst->csr", H, s)
    if noise:
        w = (rng.standard_normal(Y.shape) + 1j * rng.standard_normal(Y.shape)) * np.sqrt(sigma2 / 2)
        Y = Y + w
    return Slot(H=H.astype(np.complex64), Y=Y.astype(np.complex64),
                labels=labels.astype(np.uint8), sigma2=float(sigma2), nr=nr, nt=nt, qam=qam,
                snr_db=float(snr_db))


# The workloads, by what they are (Nr x Nt, QAM, subcarriers, SNR points, N_pe).
WORKLOADS = {
    "4x4-qpsk-64sc": dict(config=1, nr=4, nt=4, qam=4, n_sc=64, channel="iid",
                          snrs=[10.0], n_pe=[16, 256]),
    "8x8-16qam-936sc": dict(config=2, nr=8, nt=8, qam=16, n_sc=936, channel="kronecker",
                            snrs=[10.0, 13.0, 16.0, 19.0, 22.0, 25.0], n_pe=[64]),
    "16x16-64qam-3276sc": dict(config=3, nr=16, nt=16, qam=64, n_sc=3276, channel="iid",
                               snrs=[15.0, 18.0, 21.0, 24.0, 27.0, 30.0], n_pe=[64, 128, 256]),
}


def workload_slot(name: str, snr_index: int = 0, n_sc: int | None = None, extra_seed: int = 0,
                  noise: bool = True) -> Slot:
    w = WORKLOADS[name]
    return make_slot(w["nr"], w["nt"], w["qam"], n_sc if n_sc is not None else w["n_sc"],
                     14, w["snrs"][snr_index], w["channel"], 0.3,
                     seed_for(w["config"], snr_index) + 7919 * extra_seed, noise)


# Mixed batch of radio units (config 4): rx antennas in {4, 8, 16}, users
# uniform in rx/2..rx, QAM in {4, 16, 64}, subcarriers in {312, 936, 3276},
# N_pe in {16, 32, 64, 128, 256} (capped at QAM^users), all uniform; i.i.d.
# or Kronecker (rho 0.3) channels; SNR per unit drawn around a level where
# the QAM order is usable (QPSK 8-14 dB, 16-QAM 14-20 dB, 64-QAM 20-26 dB).
MIXED_CONFIG = 4
MIXED_RX = (4, 8, 16)
MIXED_QAM = (4, 16, 64)
MIXED_SC = (312, 936, 3276)
MIXED_NPE = (16, 32, 64, 128, 256)
MIXED_SNR_LO = {4: 8.0, 16: 14.0, 64: 20.0}


@dataclass
class UnitSpec:
    nr: int
    nt: int
    qam: int
    n_sc: int
    n_pe: int
    snr_db: float
    channel: str
    seed: int


def mixed_units(n_units: int = 64, seed: int | None = None, sc_scale: float = 1.0,
                config: int = MIXED_CONFIG) -> list[UnitSpec]:
    """Sizes of a mixed batch.  sc_scale shrinks the subcarrier counts (for
    tests) without changing the other draws."""
    rng = np.random.Generator(np.random.PCG64(seed_for(config) if seed is None else seed))
    out = []
    for k in range(n_units):
        nr = int(rng.choice(MIXED_RX))
        nt = int(rng.integers(nr // 2, nr + 1))
        qam = int(rng.choice(MIXED_QAM))
        n_sc = max(1, int(round(int(rng.choice(MIXED_SC)) * sc_scale)))
        n_pe = int(min(int(rng.choice(MIXED_NPE)), qam ** nt))
        snr = float(MIXED_SNR_LO[qam] + 6.0 * rng.random())
        channel = "iid" if rng.random() < 0.5 else "kronecker"
        out.append(UnitSpec(nr, nt, qam, n_sc, n_pe, snr, channel,
                            int(rng.integers(0, 2 ** 31 - 1))))
    return out


def unit_slot(u: UnitSpec, n_sym: int = 14, noise: bool = True) -> Slot:
    return make_slot(u.nr, u.nt, u.qam, u.n_sc, n_sym, u.snr_db, u.channel, 0.3, u.seed, noise)
