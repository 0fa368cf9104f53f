"""Host arithmetic of bench.py (the figures it reports); no GPU."""
import importlib.util
import os

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


B = _bench()


def test_algorithmic_bytes():
    # 16 + 56 S per tet-period: 72, 184 and 464 B at S = 1, 3 and 8
    assert [B.engine_bytes_per_entry(s) for s in (1, 3, 8)] == [72, 184, 464]
    # the bar: 8 species, reactions (tet volume) and a reaction mask
    assert B.algorithmic_bytes_per_tet_period(8, 14, True) == 476
    assert B.algorithmic_bytes_per_tet_period(3, 3, False) == 192
    assert B.algorithmic_bytes_per_tet_period(1, 0, False) == 72


def test_host_cores_within_the_machine():
    n = B.host_cores()
    assert 1 <= n <= (os.cpu_count() or 1)


def test_engine_tail_split_and_idle_share():
    """Three simulations on two clusters: spans built from a cost per period
    and a cost per entry are split back into those costs; the share of the
    launch with fewer than two running is the tail after the second ends."""
    per_period, per_entry = 20_000.0, 5.0        # ns
    P = np.array([100, 300, 50])
    E = np.array([1_000, 20_000, 3_000])
    span = P * per_period + E * per_entry
    start = np.array([0.0, 0.0, span[0]])
    end = start + span
    st = np.stack([start + 1e9, end + 1e9, E], axis=1)   # device clock offset
    out = B.engine_tail(st, P, [10, 20, 30], in_flight=2)
    assert out["us_per_period"] == pytest.approx(per_period / 1e3)
    assert out["ns_per_entry"] == pytest.approx(per_entry)
    t1 = end.max()
    both = min(end[1], end[2])                   # two running until the first of them ends
    assert out["launch_ms"] == pytest.approx(t1 / 1e6)
    assert out["frac_below_full"] == pytest.approx((t1 - both) / t1)
    assert out["longest_sim_periods"] == 300 and out["longest_sim_tets"] == 20
    assert out["max_running"] == 2
    assert out["mean_running"] == pytest.approx(span.sum() / t1)


def test_engine_tail_ignores_slots_never_timed():
    st = np.array([[0, 0, 0], [5, 15, 7]], dtype=np.int64)
    out = B.engine_tail(st, [3, 4], [1, 2], in_flight=1)
    assert out["longest_sim_tets"] == 2 and out["launch_ms"] == pytest.approx(10 / 1e6)
    assert B.engine_tail(np.zeros((2, 3)), [1, 1], [1, 1], in_flight=1) is None
