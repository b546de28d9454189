"""JSON-lines metrics log (host logic, on a stand-in context)."""
import io
import json
import math

import numpy as np

from paper_1312_2213_gb300 import ISING2D, POLYMER3D
from paper_1312_2213_gb300.log import JsonlLog, record


class FakeCtx:
    def __init__(self, system=ISING2D, L=4, q=2, p=8):
        self.system, self.L, self.q, self.p = system, L, q, p
        self.N = L if system == POLYMER3D else L * L

    def metrics(self):
        return {"iteration": 3, "accepted": 500, "tunnelling_events": 2, "sweeps": 10,
                "acceptance_rate": 500 / (self.p * self.N * 10), "accepted_total": 1500,
                "tunnelling_events_total": 4}

    def histogram(self):
        return np.array([4, 0, 8, 0, 12], dtype=np.uint64)

    def lnW(self):
        return np.array([0.0, -np.inf, 1.0, 2.0, 3.0])  # bin 1 unreachable


def test_record_fields():
    r = record(FakeCtx(), seconds=0.5, tag="x")
    assert r["system"] == "ising2d" and r["L"] == 4 and r["p"] == 8
    assert r["bins_reachable"] == 4 and r["bins_visited"] == 3  # bin 3 reachable, not visited
    assert r["h_min"] == 0.0 and r["h_max"] == 12.0 and math.isclose(r["h_mean"], 6.0)
    assert r["h_min_over_mean"] == 0.0
    assert math.isclose(r["attempts_per_s"], 8 * 16 * 10 / 0.5)
    assert r["tunnelling_events"] == 2 and r["iteration"] == 3 and r["tag"] == "x"


def test_polymer_record_names_beads():
    r = record(FakeCtx(system=POLYMER3D, L=13, q=0, p=4))
    assert r["N"] == 13 and "L" not in r and "attempts_per_s" not in r


def test_jsonl_lines():
    buf = io.StringIO()
    log = JsonlLog(buf)
    for _ in range(3):
        log.log(FakeCtx())
    lines = buf.getvalue().splitlines()
    assert len(lines) == 3
    assert all(json.loads(x)["accepted"] == 500 for x in lines)
