"""The configuration files under configs/ (one per benchmark configuration) parse and name valid
systems and sizes; the runner's argument handling (no GPU needed)."""
import glob
import json
import os

import pytest

from paper_1312_2213_gb300 import SYSTEM_NAMES

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CONFIGS = sorted(glob.glob(os.path.join(ROOT, "configs", "*.json")))


def test_there_is_a_config_per_benchmark_configuration():
    assert len(CONFIGS) == 5


@pytest.mark.parametrize("path", CONFIGS, ids=os.path.basename)
def test_config_is_valid(path):
    with open(path) as f:
        cfg = json.load(f)
    names = set(SYSTEM_NAMES.values())
    assert cfg["iterations"] >= 1 and cfg["sweeps"] >= 1
    for s in cfg["systems"]:
        assert s["system"] in names
        assert s["p"] >= 1
        if s["system"] == "polymer3d":
            assert 2 <= s["L"] <= 128
            assert s.get("window") == "pilot" or len(s["window"]) == 2
        else:
            assert s["L"] in (4, 8, 12, 16, 24, 32, 48, 64)
            if s["system"] == "potts2d":
                assert 2 <= s["q"] <= 16
            if s["system"] == "ising2d_muma":
                assert s["beta"] > 0


def test_pilot_windows_exist_for_the_polymer_config():
    from paper_1312_2213_gb300.run import _pilot_window

    with open(os.path.join(ROOT, "configs", "polymer_N13_N128_p4096.json")) as f:
        cfg = json.load(f)
    for s in cfg["systems"]:
        lo, hi = _pilot_window(s["L"])
        assert hi > lo
