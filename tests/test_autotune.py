"""Host-side logic of the launch-shape autotuner (no GPU needed)."""
from paper_2409_14355_gb300 import autotune, inputs, mpnl


def test_tuning_dict_round_trip():
    t = mpnl.Tuning()
    t.detect_sym[2][2][1] = 1
    t.select_warps[0][1][0] = 4
    t.persistent_ctas_per_sm = 2
    t.persistent_select_warps = 4
    u = autotune.from_dict(autotune.to_dict(t))
    assert autotune.to_dict(u) == autotune.to_dict(t)
    c = mpnl.Tuning()
    autotune.ctypes_copy(c, t)
    assert autotune.to_dict(c) == autotune.to_dict(t)


def test_representative_is_largest_unit_per_class():
    units = inputs.mixed_units(40, seed=5)
    rep = autotune._representative(units)
    for c, u in rep.items():
        same = [v for v in units if mpnl.problem_class(v.nt, v.qam, v.n_pe) == c]
        assert u.n_sc * u.n_pe == max(v.n_sc * v.n_pe for v in same)
    assert set(rep) == {mpnl.problem_class(v.nt, v.qam, v.n_pe) for v in units}


def test_problem_class_bounds():
    assert mpnl.problem_class(4, 4, 16) == (0, 0, 0)
    assert mpnl.problem_class(5, 16, 255) == (1, 1, 0)
    assert mpnl.problem_class(16, 64, 256) == (2, 2, 1)


def test_mixed_units_follow_the_size_rules():
    for u in inputs.mixed_units(64):
        assert u.nr in (4, 8, 16) and u.nr // 2 <= u.nt <= u.nr
        assert u.qam in (4, 16, 64) and u.n_sc in (312, 936, 3276)
        assert u.n_pe <= min(256, u.qam ** u.nt) and u.n_pe >= 1
