"""The stored oracle runs (tests/golden/oracle_runs.json), which the GPU
parity tests compare against at full size, still equal what the oracle
computes: every stored run with a recorded oracle time of at most 0.5 s is
rerun here and its digest compared.  A change to the oracle's arithmetic
that is not followed by rewriting the stored runs fails this test."""
import importlib.util
import json
import os

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def _make_golden():
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(HERE, "golden", "make_golden.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


MG = _make_golden()
STORED = json.load(open(MG.OUT))
CHEAP = sorted(k for k, v in STORED.items() if v["oracle_seconds"] <= 0.5)


def test_cheap_stored_runs_exist():
    assert len(CHEAP) >= 10
    kinds = {STORED[k]["kind"] for k in CHEAP}
    assert {"diffusion", "ensemble", "request"} <= kinds


@pytest.mark.parametrize("name", CHEAP)
def test_stored_run_is_reproduced(oracle, name):
    entry = MG.entries()[name]
    got_name, rec = MG.run_entry((name, entry))
    assert got_name == name
    want = STORED[name]
    assert rec["sha256"] == want["sha256"], name
    assert rec["period"] == want["period"] and rec["totals"] == want["totals"]
