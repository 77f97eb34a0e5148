"""Serving loop: every slot request's results in the continuous-batching mix
equal the per-call path (factor, selection, Q^H y, walks) on that RU alone
with the channel that applied to it; z from a stored Q matches the oracle."""
import numpy as np
import pytest

from paper_2409_14355_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def dev():
    from paper_2409_14355_gb300 import mpnl

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    mpnl.load_library()
    d = torch.device("cuda", 0)
    torch.cuda.set_device(d)
    return d


@pytest.mark.parametrize("nr,nt,qam,n_sc,mmse_qr", [(8, 8, 16, 37, False), (16, 16, 64, 9, False),
                                                     (7, 12, 4, 21, True), (4, 2, 64, 33, False)])
def test_factor_and_stored_q_match_oracle(dev, nr, nt, qam, n_sc, mmse_qr):
    from paper_2409_14355_gb300 import mpnl
    from tests import _parity as P
    sl = inputs.make_slot(nr, nt, qam, n_sc, 14, 18.0, "iid", 0.3, 500 + nr + nt)
    H = torch.from_numpy(sl.H).to(dev)
    Y = torch.from_numpy(sl.Y).to(dev)
    Q, R, inv_diag, perm = mpnl.factor(H, sl.sigma2 if mmse_qr else None)
    Z = mpnl.qhy(Q, Y)
    torch.cuda.synchronize()
    H64 = sl.H.astype(np.complex128)
    Y64 = sl.Y.astype(np.complex128)
    if mmse_qr:
        Rr, pr, Zr, gap = P.oracle_front_mmse(H64, Y64, sl.sigma2)
        Ha = np.concatenate([H64, np.broadcast_to(np.sqrt(sl.sigma2) * np.eye(nt),
                                                  (n_sc, nt, nt))], axis=1)
    else:
        Rr, pr, Zr, gap = P.oracle_front(H64, Y64)
        Ha = H64
    kappa = np.linalg.cond(Ha)
    ok = np.all(gap > 1e-4, axis=1)
    assert ok.mean() > 0.8
    pg = perm.cpu().numpy()
    np.testing.assert_array_equal(pg[ok], pr[ok])
    Rg = P.unpack_upper(R.cpu().numpy().astype(np.complex128), nt)
    Zg = Z.cpu().numpy().astype(np.complex128)
    Qg = Q.cpu().numpy().astype(np.complex128)
    for c in np.flatnonzero(ok):
        assert np.max(np.abs(Rg[c] - Rr[c])) <= 100 * U32 * kappa[c] * np.linalg.norm(Ha[c])
        ynorm = np.max(np.linalg.norm(Y64[c], axis=-1))
        assert np.max(np.abs(Zg[c] - Zr[c])) <= 100 * U32 * kappa[c] * ynorm
        # the stored antenna rows of Q reproduce H P = Q R on those rows
        Hp = H64[c][:, pg[c]]
        assert np.max(np.abs(Qg[c] @ Rg[c] - Hp)) <= 100 * U32 * kappa[c] * np.linalg.norm(Ha[c])


def _alone(dev, ru, H, Y):
    from paper_2409_14355_gb300 import mpnl, serving
    Hd = H.to(dev)
    Q, R, inv_diag, perm = mpnl.factor(Hd, ru.sigma2 if ru.mmse_qr else None)
    if ru.precision == "fp16":
        mpnl.refine_qr(Hd, None, R, inv_diag, perm, Q=Q, sigma2=ru.sigma2 if ru.mmse_qr else None,
                       cond_threshold=serving.REFINE_COND)
    paths = mpnl.select_paths(R, ru.sigma2, ru.qam, ru.n_pe, ru.nt)
    Z = mpnl.qhy(Q, Y.to(dev), precision=ru.precision)
    hard, llr, _ = mpnl.detect(R, inv_diag, perm, paths, Z, ru.sigma2, ru.qam,
                               precision=ru.precision)
    return hard.cpu(), llr.cpu()


def test_serving_results_equal_each_request_alone(dev):
    _serve_and_compare(dev)


def test_serving_with_llrs_left_on_the_device(dev):
    """llr_to_host=False: the LLRs are computed into each slot's device
    buffer and not copied back; they equal the per-call path's."""
    server = _serve_and_compare(dev, llr_to_host=False)
    assert all(b.llr_host is None for ru in server.rus.values() for b in ru.pool)


def test_serving_on_an_sm_split_equals_each_request_alone(dev):
    """The same with the small units' rounds on a group of SMs of their own
    (green contexts) and the large ones on the rest: the class boundary is
    set so that both groups serve some of the units."""
    from paper_2409_14355_gb300 import serving
    specs = inputs.mixed_units(6, seed=31, sc_scale=0.02)
    costs = sorted(serving.RU(0, u.nr, u.nt, u.qam, u.n_sc, u.n_pe, 1.0).cost for u in specs)
    server = _serve_and_compare(dev, sm_split=16, big_cost=costs[len(costs) // 2])
    assert server.split_sms is not None and server.split_sms[0] >= 16


def _serve_and_compare(dev, **server_kw):
    from paper_2409_14355_gb300 import mpnl, serving
    specs = inputs.mixed_units(6, seed=31, sc_scale=0.02)
    specs[1] = inputs.UnitSpec(4, 6, 16, 29, 64, 18.0, "iid", 77)   # more users than antennas
    server = serving.Server(dev, mem_budget=64 << 20, max_units_per_round=8, max_inflight=2,
                            keep_results=True, **server_kw)
    payloads, first_H = {}, {}
    for k, u in enumerate(specs):
        sl = inputs.unit_slot(u)
        ru = serving.RU(k, u.nr, u.nt, u.qam, u.n_sc, u.n_pe, sl.sigma2, mmse_qr=u.nt > u.nr,
                        precision="fp16" if k % 3 == 2 else "fp32")
        server.register(ru, torch.from_numpy(sl.H))
        first_H[k] = torch.from_numpy(sl.H)
        alt = [inputs.unit_slot(inputs.UnitSpec(**{**u.__dict__, "seed": u.seed + j}))
               for j in (1, 2)]
        payloads[k] = {"slot": [torch.from_numpy(a.Y).pin_memory() for a in [sl] + alt],
                       "channel": [torch.from_numpy(a.H).pin_memory() for a in alt]}
    trace = serving.poisson_trace(specs, rate_per_s=40000.0, duration_s=0.002,
                                  coherence_slots=3, seed=3)
    assert any(kind == "channel" for _, _, kind in trace)
    reqs = serving.run_trace(server, trace, payloads)
    server.close()
    mpnl.check_status()
    assert all(q.done >= 0 for q in reqs)
    assert max(server.round_sizes) > 1  # requests were batched together
    current = dict(first_H)
    n_cmp = 0
    for q in reqs:  # per-RU order is submission order
        if q.kind == "channel":
            current[q.ru] = q.payload
            continue
        ru = server.rus[q.ru]
        hard, llr = _alone(dev, ru, current[q.ru], q.payload)
        assert torch.equal(q.hard, hard), (q.rid, q.ru)
        assert torch.equal(q.llr.cpu(), llr), (q.rid, q.ru)
        assert q.llr.device.type == ("cpu" if server.llr_to_host else "cuda")
        n_cmp += 1
    assert n_cmp > 20
    if "big_cost" in server_kw:   # both size classes were served
        assert len({server.rus[q.ru].cost >= server.big_cost for q in reqs}) == 2
    return server


def test_sm_split_streams_run_the_path(dev):
    """mpnl_sm_split_*: two disjoint SM groups covering at most the device's
    SMs; the whole path enqueued on a stream of either group gives the
    results of the default stream; bad arguments are refused."""
    from paper_2409_14355_gb300 import mpnl
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    sl = inputs.make_slot(8, 8, 16, 150, 14, 16.0, "iid", 0.3, 901)
    H = torch.from_numpy(sl.H).to(dev)
    Y = torch.from_numpy(sl.Y).to(dev)

    def path():
        R, inv_diag, perm, Z = mpnl.preprocess(H, Y)
        paths = mpnl.select_paths(R, sl.sigma2, sl.qam, 64, sl.nt)
        hard, llr, ped2 = mpnl.detect(R, inv_diag, perm, paths, Z, sl.sigma2, sl.qam)
        return hard, llr, ped2

    want = [t.cpu() for t in path()]
    split = mpnl.SmSplit.get(16, dev)
    assert mpnl.SmSplit.get(16, dev) is split
    assert split.sms[0] >= 16 and split.sms[1] >= 1 and sum(split.sms) <= n_sm
    for part in (0, 1):
        st = split.stream(part)
        assert split.stream(part) is st
        st.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(st):
            got = path()
        st.synchronize()
        for a, b in zip(got, want):
            assert torch.equal(a.cpu(), b)
    mpnl.check_status()
    for bad in (0, n_sm, -3):
        with pytest.raises(mpnl.MpnlError):
            mpnl.SmSplit(bad, dev)


def test_sm_split_create_and_destroy_through_the_abi(dev):
    """Create, streams, destroy at the C ABI (nothing enqueued: a split
    whose streams torch has used stays for the life of the process)."""
    import ctypes
    from paper_2409_14355_gb300 import mpnl
    lib = mpnl.load_library()
    ctx = mpnl.context(dev.index)
    h = ctypes.c_void_p()
    sms = (ctypes.c_int * 2)()
    assert lib.mpnl_sm_split_create(ctx, 24, ctypes.byref(h), sms) == mpnl.OK
    assert sms[0] >= 24 and sms[1] >= 1
    streams = []
    for part in (0, 1, 1):
        p = ctypes.c_void_p()
        assert lib.mpnl_sm_split_stream(ctx, h, part, 0, ctypes.byref(p)) == mpnl.OK and p.value
        streams.append(p.value)
    assert len(set(streams)) == 3
    p = ctypes.c_void_p()
    assert lib.mpnl_sm_split_stream(ctx, h, 2, 0, ctypes.byref(p)) == mpnl.ERR_INVALID_ARG
    assert lib.mpnl_sm_split_create(ctx, 24, None, sms) == mpnl.ERR_INVALID_ARG
    assert lib.mpnl_sm_split_destroy(ctx, h) == mpnl.OK
    assert lib.mpnl_sm_split_destroy(ctx, None) == mpnl.OK


def test_memory_budget_limits_rounds(dev):
    from paper_2409_14355_gb300 import serving
    specs = inputs.mixed_units(3, seed=8, sc_scale=0.05)
    server = serving.Server(dev, mem_budget=1, max_units_per_round=8, max_inflight=1)
    payloads = {}
    for k, u in enumerate(specs):
        sl = inputs.unit_slot(u)
        server.register(serving.RU(k, u.nr, u.nt, u.qam, u.n_sc, u.n_pe, sl.sigma2),
                        torch.from_numpy(sl.H))
        payloads[k] = {"slot": [torch.from_numpy(sl.Y).pin_memory()], "channel": []}
    # a budget smaller than any request admits nothing: the loop gives up at its limit
    trace = [(0.0, 0, "slot")]
    reqs = serving.run_trace(server, trace, payloads, t_limit_s=0.2)
    assert reqs[0].done < 0 and server.n_rounds == 0
    server.close()


def test_serve_round_refuses_bad_requests(dev):
    # mpnl_serve_round checks every request before it enqueues anything
    import ctypes

    from paper_2409_14355_gb300 import mpnl, serving
    u = inputs.mixed_units(1, seed=5, sc_scale=0.02)[0]
    sl = inputs.unit_slot(u)
    server = serving.Server(dev, mem_budget=64 << 20, max_units_per_round=4, max_inflight=1)
    ru = serving.RU(0, u.nr, u.nt, u.qam, u.n_sc, u.n_pe, sl.sigma2)
    server.register(ru, torch.from_numpy(sl.H))
    reqs = [(0.0, 0, "slot")]
    payloads = {0: {"slot": [torch.from_numpy(sl.Y).pin_memory()], "channel": []}}
    serving.run_trace(server, reqs, payloads)            # creates the round's batch
    r = server.rounds[0]
    assert r.batch is not None
    rc = (mpnl.RoundReqC * 4)()
    lib = mpnl.load_library()
    st = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    b = ru.pool[0]
    rc[0].unit = ctypes.pointer(ru.item)
    rc[0].kind = 7                                        # no such kind
    rc[0].payload, rc[0].staging = payloads[0]["slot"][0].data_ptr(), b.Y.data_ptr()
    assert lib.mpnl_serve_round(r.batch._ctx, r.batch._h, rc, 1, 0, st) == mpnl.ERR_INVALID_ARG
    rc[0].kind = mpnl.ROUND_SLOT                          # a slot without its output buffers
    assert lib.mpnl_serve_round(r.batch._ctx, r.batch._h, rc, 1, 0, st) == mpnl.ERR_INVALID_ARG
    assert lib.mpnl_serve_round(r.batch._ctx, r.batch._h, rc, 5, 0, st) == mpnl.ERR_INVALID_ARG
    assert lib.mpnl_serve_round(r.batch._ctx, r.batch._h, rc, 1, 1 << 20, st) \
        == mpnl.ERR_INVALID_ARG
    server.close()
