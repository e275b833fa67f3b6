"""Admission policy of the served loop (host logic, no GPU): which waiting request
starts next under a device budget, one out-of-core slot and one large in-core build
at a time."""
import types

from paper_2302_05002_gb300.serve import pick_request


def req(name, need, mode="in-core", n=1_000_000):
    return types.SimpleNamespace(name=name, need=need, mode=mode, n=n)


BIG = 1 << 24


def pick(queue, free=100, ooc=True, big_active=0, big_slots=1, max_bypass=None):
    r = pick_request(queue, free, ooc, BIG, big_active, big_slots, max_bypass)
    return None if r is None else r.name


def test_first_fit_in_arrival_order():
    q = [req("a", 150), req("b", 60), req("c", 10)]
    assert pick(q) == "b"                      # a does not fit, b is the first that does


def test_nothing_fits():
    assert pick([req("a", 150), req("b", 101)]) is None
    assert pick([]) is None


def test_out_of_core_goes_first_when_a_slot_is_free():
    q = [req("a", 10), req("o", 50, "out-of-core"), req("b", 10)]
    assert pick(q) == "o"
    assert pick(q, ooc=False) == "a"            # no host slot: the in-core requests go on
    assert pick(q, free=40) == "a"              # the arena does not fit: same


def test_one_large_in_core_build_at_a_time():
    q = [req("big", 10, n=BIG), req("small", 10, n=BIG - 1)]
    assert pick(q) == "big"
    assert pick(q, big_active=1) == "small"     # a large one runs: only smaller ones start
    assert pick([req("big", 10, n=2 * BIG)], big_active=1) is None


def test_budget_is_inclusive():
    assert pick([req("a", 100)]) == "a"


def test_incore_need_per_point():
    # the cloud, its outputs and the largest stage workspace: about 120 B per point for
    # large clouds, so a 24 GB budget (in core up to three quarters) holds ~160M points
    from paper_2302_05002_gb300 import fastpoints as fp
    from paper_2302_05002_gb300.serve import incore_need
    prm = fp.params()
    per = incore_need(160_000_000, prm) / 160_000_000
    assert 100 < per < 130
    assert incore_need(155_000_000, prm) <= (24 << 30) * 3 // 4 < incore_need(165_000_000, prm)


def test_large_in_core_builds_up_to_the_slots():
    q = [req("big", 10, n=BIG), req("small", 10, n=BIG - 1)]
    assert pick(q, big_active=1, big_slots=2) == "big"    # a second large build may start
    assert pick(q, big_active=2, big_slots=2) == "small"


def test_aging_stops_bypassing_the_oldest_request():
    big = req("big", 150)
    q = [big, req("s1", 10), req("s2", 10)]
    assert pick(q, max_bypass=2) == "s1"        # the oldest does not fit: a later one starts
    big.bypassed = 2                            # passed over twice: nothing else starts ...
    assert pick(q, max_bypass=2) is None
    assert pick(q, free=150, max_bypass=2) == "big"   # ... until it fits
    assert pick(q, max_bypass=None) == "s1"     # no aging bound: first fit as before
