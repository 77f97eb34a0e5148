"""Mixed-precision walk (mpnl_detect_mixed) against the FP64 oracle.

FP16 residuals change some rankings, so decisions may differ from the
oracle's; the tests bound and report the decision-mismatch rate and the BER
delta per SNR point, and check exactly what the FP32 re-check guarantees:
the reported best PED is the FP32 metric ||z - R s||^2 of the decided vector.
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
    print(f"\n{name} snr={sl.snr_db} n_pe={n_pe}: fp16 decision mismatch {mismatch:.4f}, "
          f"BER delta {dber:+.2e}")
    assert mismatch <= 0.05
    assert abs(dber) <= 2e-3
    # 3. LLRs of unique minima: error relative to the two PED minima
    ml = P.comparable(ref, sl.sigma2)["llr"]
    d1 = ref["ped2"][..., 0][..., None, None]
    scale = 2 * d1 / sl.sigma2 + np.abs(ref["llr"]) + 1.0
    rel = (np.abs(g["llr"] - ref["llr"]) / scale)[ml]
    assert np.median(rel) <= 64 * U16 and np.quantile(rel, 0.99) <= 0.25


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


def test_ffma_probe_runs_and_counts_its_flops(dev):
    # measurement helper used for the roofline's measured FP32 peak
    from paper_2409_14355_gb300 import mpnl
    out = torch.empty(3 * 256, dtype=torch.float32, device=dev)
    fl = mpnl.probe_ffma(3, 100, out)
    torch.cuda.synchronize()
    assert fl == 2 * 8 * 256 * 3 * 100
    v = out.cpu().numpy()
    assert np.all(np.isfinite(v)) and np.all(v > 0)
    with pytest.raises(mpnl.MpnlError):
        mpnl.probe_ffma(0, 100, torch.empty(0, dtype=torch.float32, device=dev))
    with pytest.raises(mpnl.MpnlError):
        mpnl.probe_ffma(3, 10 ** 9, out)            # more than 1e13 flop
