"""Host logic of the serving loop (no GPU): arrivals, request sizes and the
admission rules (memory budget, per-RU order, channel updates)."""
import numpy as np
import torch

from paper_2409_14355_gb300 import inputs, serving


def _server(budget=1 << 30, units=4):
    s = serving.Server(device="cpu", mem_budget=budget, max_units_per_round=8)
    for k in range(units):
        s.rus[k] = serving.RU(k, 4, 4, 16, 12 + k, 16, 0.1)
        s.rus[k].pool = [object(), object()]  # two free buffer sets
    return s


def _req(rid, ru, kind):
    return serving.Request(rid, ru, kind, rid * 1e-6, torch.zeros(1))


def test_poisson_trace_is_sorted_with_periodic_channel_updates():
    units = inputs.mixed_units(5, seed=2, sc_scale=0.01)
    tr = serving.poisson_trace(units, 5000.0, 0.1, coherence_slots=4, seed=1)
    times = [t for t, _, _ in tr]
    assert times == sorted(times)
    per = {}
    for t, k, kind in tr:
        per.setdefault(k, []).append(kind)
    for kinds in per.values():
        slots = 0
        for a, kind in enumerate(kinds):
            if kind == "channel":
                assert slots % 4 == 3 and kinds[a + 1] == "slot"
            else:
                slots += 1
    n_slots = sum(1 for _, _, k in tr if k == "slot")
    assert abs(n_slots - 500) < 5 * np.sqrt(500)


def test_request_bytes_counts_inputs_scratch_and_outputs():
    ru = serving.RU(0, 8, 4, 64, 10, 16, 0.1)
    slot = serving.request_bytes(ru, "slot", llr=True)
    assert slot == 10 * 14 * (8 * 8 + 4 * 8 + 4 + 8) + 10 * 14 * 4 * 6 * 4
    assert serving.request_bytes(ru, "slot", llr=False) == slot - 10 * 14 * 4 * 6 * 4
    assert serving.request_bytes(ru, "channel", llr=True) == 10 * 8 * 4 * 8


def test_admission_keeps_per_ru_order_and_budget():
    s = _server()
    reqs = [_req(0, 3, "slot"), _req(1, 0, "slot"), _req(2, 3, "slot"), _req(3, 1, "slot")]
    for q in reqs:
        s.submit(q)
    chosen, nbytes = s._form()
    # smallest RUs first; RU 3's two slots stay in arrival order
    assert [q.rid for q in chosen] == [1, 3, 0, 2]
    assert nbytes == sum(serving.request_bytes(s.rus[q.ru], q.kind, True) for q in chosen)
    # a budget for one request admits one, the rest wait in arrival order
    s = _server(budget=serving.request_bytes(serving.RU(0, 4, 4, 16, 13, 16, 0.1), "slot", True))
    for q in reqs:
        s.submit(q)
    chosen, _ = s._form()
    assert [q.rid for q in chosen] == [1]
    assert [q.rid for q in s.waiting] == [0, 2, 3]


def test_channel_update_waits_for_rounds_reading_the_state():
    s = _server()
    s.rus[2].busy_rounds.add(7)
    for q in (_req(0, 2, "channel"), _req(1, 2, "slot"), _req(2, 0, "slot")):
        s.submit(q)
    chosen, _ = s._form()
    assert [q.rid for q in chosen] == [2]          # RU 2 is held behind its update
    s.rus[2].busy_rounds.clear()
    chosen, _ = s._form()
    assert [q.rid for q in chosen] == [0, 1]       # update, then its slot, same round


def test_slot_waits_while_its_rus_update_runs_in_another_round():
    # round 1 (in flight) holds RU 2's channel update; a later slot of RU 2
    # must not go into the next round, which runs on another stream and
    # could read the state while the update still rewrites it
    s = _server()
    s.submit(_req(0, 2, "channel"))
    chosen, _ = s._form()
    assert [q.rid for q in chosen] == [0]
    s.rus[2].busy_rounds.add(1)
    s.rus[2].update_round = 1        # what the launch records for the update
    for q in (_req(1, 2, "slot"), _req(2, 0, "slot")):
        s.submit(q)
    chosen, _ = s._form()
    assert [q.rid for q in chosen] == [2]
    assert [q.rid for q in s.waiting] == [1]
    # the update's round retires: the slot goes into the next round
    s.rus[2].busy_rounds.clear()
    s.rus[2].update_round = -1
    chosen, _ = s._form()
    assert [q.rid for q in chosen] == [1]


def test_poll_clears_the_update_mark_with_its_round():
    s = _server()
    ru = s.rus[1]
    q = _req(0, 1, "channel")

    class Done:
        def query(self):
            return True

    r = s.rounds[0]
    r.requests, r.event, r.round_id, r.bytes = [q], Done(), 5, 0
    ru.busy_rounds.add(5)
    ru.update_round = 5
    assert s.poll() == 1
    assert ru.update_round == -1 and not ru.busy_rounds


def test_slots_wait_for_a_free_buffer_set_of_their_ru():
    s = _server()
    for q in (_req(0, 1, "slot"), _req(1, 1, "slot"), _req(2, 1, "slot"), _req(3, 2, "slot")):
        s.submit(q)
    chosen, _ = s._form()
    assert [q.rid for q in chosen] == [0, 1, 3]    # RU 1 (smaller) has two buffer sets
    assert [q.rid for q in s.waiting] == [2]


def test_update_never_shares_a_round_with_an_earlier_slot_of_its_ru():
    s = _server()
    for q in (_req(0, 1, "slot"), _req(1, 1, "channel"), _req(2, 1, "slot")):
        s.submit(q)
    chosen, _ = s._form()
    assert [q.rid for q in chosen] == [0]
    assert [q.rid for q in s.waiting] == [1, 2]


def test_small_and_large_units_form_separate_rounds():
    s = _server()
    s.rus[3] = serving.RU(3, 16, 16, 64, 3276, 256, 0.1)
    s.rus[3].pool = [object(), object()]
    for q in (_req(0, 3, "slot"), _req(1, 0, "slot"), _req(2, 1, "slot")):
        s.submit(q)
    chosen, _ = s._form()
    assert [q.rid for q in chosen] == [1, 2]       # the small units' round
    chosen, _ = s._form()
    assert [q.rid for q in chosen] == [0]          # then the large unit's


def test_large_rounds_leave_room_for_small_units():
    s = serving.Server(device="cpu", mem_budget=1 << 30, max_units_per_round=8, max_inflight=4,
                       max_large_rounds=1)
    for k in range(2):
        s.rus[k] = serving.RU(k, 4, 4, 16, 12 + k, 16, 0.1)
        s.rus[k].pool = [object(), object()]
    for k in (2, 3):
        s.rus[k] = serving.RU(k, 16, 16, 64, 3276, 256, 0.1)
        s.rus[k].pool = [object(), object()]
    # one large unit's round in flight: the other large unit waits, small ones go
    s.rounds[0].big = True
    s.rounds[0].event = object()
    for q in (_req(0, 3, "slot"), _req(1, 0, "slot"), _req(2, 2, "slot")):
        s.submit(q)
    chosen, _ = s._form()
    assert [q.rid for q in chosen] == [1]
    chosen, _ = s._form()
    assert chosen == []
    s.rounds[0].event = None                       # the large round completed
    chosen, _ = s._form()
    assert [q.rid for q in chosen] == [0, 2]       # both large units, one round


def test_latency_statistics_per_size_class():
    reqs = []
    # ten small-unit slots at 0.1 .. 1.0 ms, five large-unit slots at 2 ms,
    # a channel update and an unfinished slot that must not count
    for k in range(10):
        q = _req(k, 0, "slot")
        q.arrival, q.done = 0.0, (k + 1) * 1e-4
        reqs.append(q)
    for k in range(5):
        q = _req(10 + k, 3, "slot")
        q.arrival, q.done = 1.0, 1.0 + 2e-3
        reqs.append(q)
    ch = _req(20, 0, "channel")
    ch.arrival, ch.done = 0.0, 5.0
    reqs.append(ch)
    reqs.append(_req(21, 0, "slot"))                 # never done
    st = serving.latency_stats(reqs, deadline_s=0.5e-3, dets_of=lambda q: 100,
                               big_of=lambda q: q.ru == 3)
    assert st["requests"] == 17 and st["slots_done"] == 15
    assert abs(st["small_units"]["p50_ms"] - 0.55) < 1e-9
    assert st["small_units"]["miss_rate"] == 0.5     # 0.6 .. 1.0 ms are over 0.5 ms
    assert st["large_units"]["miss_rate"] == 1.0 and abs(st["large_units"]["p50_ms"] - 2.0) < 1e-9
    assert abs(st["miss_rate"] - 10 / 15) < 1e-12
    assert abs(st["detections_per_s"] - 15 * 100 / (1.0 + 2e-3)) < 1e-6


def test_a_radio_unit_that_disappears_mid_trace():
    # RU 1 drops out: its waiting requests are dropped and reported, later
    # submissions for it are refused, the other RUs are served as before,
    # and its state is released once the round still using it retires
    s = _server()
    s.rus[1].state = {"Q": None}
    s.rus[1].busy_rounds.add(3)                  # a round in flight holds one of its slots
    for q in (_req(0, 1, "slot"), _req(1, 0, "slot"), _req(2, 1, "channel"), _req(3, 2, "slot")):
        s.submit(q)
    dropped = s.deregister(1)
    assert [q.rid for q in dropped] == [0, 2] and all(q.done == -2.0 for q in dropped)
    assert 1 in s.rus                            # still read by round 3
    assert not s.submit(_req(4, 1, "slot")) and s.dropped[-1].rid == 4
    chosen, _ = s._form()
    assert [q.rid for q in chosen] == [1, 3]

    class Done:
        def query(self):
            return True

    r = s.rounds[0]
    inflight = _req(9, 1, "slot")
    r.requests, r.event, r.round_id, r.bytes = [inflight], Done(), 3, 0
    assert s.poll() == 1
    assert inflight.done >= 0 and inflight in s.completed   # its last slot completed
    assert 1 not in s.rus                                   # state released
    assert not s.submit(_req(5, 1, "slot"))
    # an RU with nothing in flight is released at once
    s.deregister(2)
    assert 2 not in s.rus

