"""Mixed-precision walk (mpnl_detect_mixed) against the FP64 oracle.

The walks choose their vectors with FP16 residuals; every metric they report
(best and runner-up PED, each LLR minimum) is the FP32 metric ||z - R s||^2
of a chosen vector.  So the outputs are exact FP32 functions of the FP16
walks' list: the reported best PED is the metric of the decided vector, LLR
signs agree with the decided bits, and the results do not depend on the
scale of the inputs (FP16's range is covered by power-of-two scaling).
Where FP16 rounding changes a ranking the list can hold other vectors than
the FP32 walks' list: the decision-mismatch rate and the BER delta against
the FP64 oracle are reported per SNR point, the BER delta held to the 1e-3
of the acceptance rule, and bit-exact decisions at FP32's tie width are
recorded as an expected failure of this form.
"""
import numpy as np
import pytest

import oracle
from paper_2409_14355_gb300 import inputs
from tests import _parity as P
from tests._ref_helpers import bit_of

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U16 = 2.0 ** -11


@pytest.fixture(scope="module")
def dev():
    from paper_2409_14355_gb300 import mpnl

    assert torch.cuda.is_available()
    mpnl.load_library()
    d = torch.device("cuda", 0)
    torch.cuda.set_device(d)
    return d


def _t(a, dev):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def _run(dev, sl, n_pe, precision):
    from paper_2409_14355_gb300 import mpnl

    Rr, pr, Zr, _ = P.oracle_front(sl.H.astype(np.complex128), sl.Y.astype(np.complex128))
    R32, Z32, inv32 = P.to_fp32_inputs(Rr, Zr)
    paths = np.stack([oracle.select_paths(np.real(np.diag(R32[c])).astype(np.float64), sl.sigma2,
                                          sl.qam, n_pe)[0] for c in range(sl.n_sc)])
    hard, llr, ped2 = mpnl.detect(_t(P.pack_upper(R32), dev), _t(inv32, dev),
                                  _t(pr.astype(np.uint8), dev), _t(paths, dev), _t(Z32, dev),
                                  sl.sigma2, sl.qam, precision=precision)
    mpnl.check_status()
    g = dict(hard=hard.cpu().numpy(), llr=llr.cpu().numpy().astype(np.float64),
             ped2=ped2.cpu().numpy().astype(np.float64))
    ref = P.oracle_detect_all(R32.astype(np.complex128), Z32.astype(np.complex128), pr, paths,
                              sl.sigma2, sl.qam)
    return g, ref, R32.astype(np.complex128), Z32.astype(np.complex128), pr


def _ber(hard, labels, B):
    return sum(np.sum(bit_of(hard, b, B) != bit_of(labels, b, B)) for b in range(B)) / (labels.size * B)


@pytest.mark.parametrize("name,snr_index,n_pe,n_sc", [
    ("16x16-64qam-3276sc", 0, 64, 64),
    ("16x16-64qam-3276sc", 2, 256, 48),
    ("16x16-64qam-3276sc", 5, 128, 48),
    ("8x8-16qam-936sc", 0, 64, 128),
    ("8x8-16qam-936sc", 5, 64, 128),
    ("4x4-qpsk-64sc", 0, 16, None),
])
def test_mixed_precision_vs_oracle(dev, name, snr_index, n_pe, n_sc):
    sl = inputs.workload_slot(name, snr_index, n_sc=n_sc)
    g, ref, R, Z, perm = _run(dev, sl, n_pe, "fp16")
    pts = oracle.constellation(sl.qam)
    B = oracle.BITS[sl.qam]
    # 1. the FP32 re-check: the reported best PED is the metric of the decided vector
    for c in range(sl.n_sc):
        s_det = pts[g["hard"][c][:, perm[c]]]                     # detection order
        metric = np.sum(np.abs(Z[c] - s_det @ R[c].T) ** 2, axis=1)  # [n_sym]
        scale = np.sum(np.real(np.diag(R[c])) ** 2)
        np.testing.assert_allclose(g["ped2"][c, :, 0], metric, rtol=1e-4, atol=1e-6 * scale)
        assert np.all(g["ped2"][c, :, 1] >= g["ped2"][c, :, 0])
    # 2. decision mismatch on the oracle's unique decisions, and BER delta
    m = P.comparable(ref, sl.sigma2)["decision"]
    mismatch = np.mean(~np.all(g["hard"] == ref["hard"], axis=-1)[m])
    dber = _ber(g["hard"], sl.labels, B) - _ber(ref["hard"], sl.labels, B)
    # 3. LLRs of unique minima: error relative to the two PED minima
    ml = P.comparable(ref, sl.sigma2)["llr"]
    d1 = ref["ped2"][..., 0][..., None, None]
    scale = 2 * d1 / sl.sigma2 + np.abs(ref["llr"]) + 1.0
    rel = (np.abs(g["llr"] - ref["llr"]) / scale)[ml]
    same = np.all(g["hard"] == ref["hard"], axis=-1)
    print(f"\n{name} snr={sl.snr_db} n_pe={n_pe}: fp16 decision mismatch {mismatch:.4f} "
          f"(all {np.mean(~same):.4f}), BER delta {dber:+.2e}, LLR rel err median "
          f"{np.median(rel):.2e} p99 {np.quantile(rel, 0.99):.2e} max {np.max(rel):.2e}, "
          f"LLRs within 1e-4: {np.mean(rel <= 1e-4):.4f}")
    assert abs(dber) <= 1e-3
    assert mismatch <= 0.05
    # 4. LLR signs agree with the decided bits (each side's minimum is a
    #    metric of the list, and the decided vector holds the smaller one)
    for b in range(B):
        bits = bit_of(g["hard"], b, B)
        L = g["llr"][..., b]
        assert np.all(L[bits == 0] >= 0) and np.all(L[bits == 1] <= 0)


@pytest.mark.xfail(reason="FP16 residuals flip rankings that FP32 resolves: the FP16 walks' "
                          "list differs from the FP32 walks' list on some detections that "
                          "are unique at FP32's tie width", strict=False)
def test_mixed_precision_decisions_bit_exact_at_fp32_tie_width(dev):
    sl = inputs.workload_slot("16x16-64qam-3276sc", 2, n_sc=48)
    g, ref, _, _, _ = _run(dev, sl, 256, "fp16")
    m = P.comparable(ref, sl.sigma2)["decision"]
    assert np.all(np.all(g["hard"] == ref["hard"], axis=-1)[m])


@pytest.mark.parametrize("precision", ["fp16", "fp32"])
def test_walks_do_not_depend_on_the_input_scale(dev, precision):
    # scaling R, z by 2^k (1/R_ll by 2^-k, sigma2 by 2^2k) is exact in any
    # precision that represents the scaled values: decisions and LLRs stay
    # bit-identical and the PEDs scale by 2^2k -- for FP16 residuals only
    # because the kernel normalises each subcarrier by a power of two
    from paper_2409_14355_gb300 import mpnl

    sl = inputs.workload_slot("16x16-64qam-3276sc", 4, n_sc=24)
    Rr, pr, Zr, _ = P.oracle_front(sl.H.astype(np.complex128), sl.Y.astype(np.complex128))
    R32, Z32, inv32 = P.to_fp32_inputs(Rr, Zr)
    paths = np.stack([oracle.select_paths(np.real(np.diag(R32[c])).astype(np.float64), sl.sigma2,
                                          sl.qam, 128)[0] for c in range(sl.n_sc)])
    out = {}
    for k in (0, 12, -12):
        f = np.float32(2.0 ** k)
        h, l, p = mpnl.detect(_t(P.pack_upper(R32) * f, dev), _t(inv32 / f, dev),
                              _t(pr.astype(np.uint8), dev), _t(paths, dev), _t(Z32 * f, dev),
                              sl.sigma2 * float(f) ** 2, sl.qam, precision=precision)
        out[k] = (h.cpu().numpy(), l.cpu().numpy(), p.cpu().numpy())
    for k in (12, -12):
        assert np.array_equal(out[k][0], out[0][0]), k
        assert np.array_equal(out[k][1], out[0][1]), k
        assert np.array_equal(out[k][2], out[0][2] * np.float32(2.0 ** (2 * k))), k


def test_mixed_and_fp32_agree_on_most_decisions(dev):
    from paper_2409_14355_gb300 import mpnl

    sl = inputs.workload_slot("16x16-64qam-3276sc", 3, n_sc=256)
    H, Y = _t(sl.H, dev), _t(sl.Y, dev)
    R, inv_diag, perm, Z = mpnl.preprocess(H, Y)
    paths = mpnl.select_paths(R, sl.sigma2, 64, 128, 16)
    h32, _, _ = mpnl.detect(R, inv_diag, perm, paths, Z, sl.sigma2, 64)
    h16, _, _ = mpnl.detect(R, inv_diag, perm, paths, Z, sl.sigma2, 64, precision="fp16")
    agree = torch.all(h32 == h16, dim=-1).float().mean().item()
    assert agree >= 0.95, agree
