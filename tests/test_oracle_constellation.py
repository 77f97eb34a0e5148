"""Pins of the oracle's constellation (TS 38.211 §5.1) against its defining
properties and the standard's printed mapping."""
import numpy as np
import pytest

import oracle
from paper_2409_14355_gb300 import inputs
from tests._ref_helpers import bit_of

GOLDEN = __import__("os").path.join(__import__("os").path.dirname(__file__), "golden",
                                    "ts38211_constellations.txt")


def _load_golden():
    rows = {}
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            qam, bits, re, im, scale = line.split()
            rows.setdefault(int(qam), {})[int(bits, 2)] = complex(int(re), int(im)) / np.sqrt(int(scale))
    return rows


@pytest.mark.parametrize("qam", [4, 16, 64])
def test_unit_energy_and_square_grid(qam):
    pts = oracle.constellation(qam)
    assert np.isclose(np.mean(np.abs(pts) ** 2), 1.0, atol=1e-14)
    L = int(round(np.sqrt(qam)))
    scale = np.sqrt(2.0 * (qam - 1) / 3.0)  # average energy of the odd-integer grid
    grid = set(range(-(L - 1), L, 2))
    for p in pts:
        assert round(p.real * scale) in grid and round(p.imag * scale) in grid
        assert abs(p.real * scale - round(p.real * scale)) < 1e-12
    assert len({(round(p.real * scale), round(p.imag * scale)) for p in pts}) == qam


@pytest.mark.parametrize("qam", [4, 16, 64])
def test_gray_neighbours_differ_in_one_bit(qam):
    pts = oracle.constellation(qam)
    B = int(np.log2(qam))
    dmin = np.min([abs(a - b) for i, a in enumerate(pts) for j, b in enumerate(pts) if i != j])
    for i in range(qam):
        for j in range(qam):
            if i != j and abs(abs(pts[i] - pts[j]) - dmin) < 1e-12:
                assert bin(i ^ j).count("1") == 1


@pytest.mark.parametrize("qam", [4, 16, 64])
def test_matches_standard_table_and_generator(qam):
    gold = _load_golden()[qam]
    pts = oracle.constellation(qam)
    for lab, val in gold.items():
        assert abs(pts[lab] - val) < 1e-14, (qam, lab)
    # the transmitter's independent copy in the input generator agrees
    np.testing.assert_allclose(inputs.tx_constellation(qam), pts, atol=1e-15)


@pytest.mark.parametrize("qam", [4, 16, 64])
def test_first_bits_give_quadrant(qam):
    # b0 selects the sign of the real part and b1 that of the imaginary part
    pts = oracle.constellation(qam)
    B = int(np.log2(qam))
    labels = np.arange(qam)
    assert np.all((pts.real < 0) == (bit_of(labels, 0, B) == 1))
    assert np.all((pts.imag < 0) == (bit_of(labels, 1, B) == 1))
