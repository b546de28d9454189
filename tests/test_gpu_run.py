"""The configuration runner (python -m paper_1312_2213_gb300.run) on shortened versions of the
configurations: the 8x8 Ising configuration ends in the same reweighting as the oracle run with
the same seed, and the batched mix (one graph per iteration) and the polymer configuration run
through with their per-iteration JSON lines."""
import io
import json
import os

import numpy as np
import pytest

import oracle
from paper_1312_2213_gb300 import run as runner
from paper_1312_2213_gb300.log import JsonlLog

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _cfg(name, **over):
    with open(os.path.join(ROOT, "configs", name)) as f:
        cfg = json.load(f)
    cfg.update(over)
    return cfg


def test_ising_L8_config_matches_the_oracle():
    cfg = _cfg("ising2d_L8_p64.json", iterations=4, sweeps=300)
    buf = io.StringIO()
    res = runner.run(cfg, JsonlLog(buf), out=io.StringIO())
    lines = [json.loads(x) for x in buf.getvalue().splitlines()]
    assert [r["iteration"] for r in lines] == [1, 2, 3, 4]
    o = oracle.Run(0, 8, 2, 64, 1)
    o.init()
    for _ in range(4):
        o.iterate(300, 8)
        o.update()
    for beta in cfg["reweight_betas"]:
        want, _ = o.reweight(beta)
        got = np.array(res["systems"][0]["reweight"][str(beta)])
        np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12)
    assert lines[-1]["accepted"] == int(o.metrics()[0])


def test_mix_and_polymer_configs_run():
    buf = io.StringIO()
    res = runner.run(_cfg("mix_ising_potts_2048.json", iterations=2, sweeps=10), JsonlLog(buf), out=io.StringIO())
    assert res["iterations"] == 2 and len(res["systems"]) == 9
    assert len(buf.getvalue().splitlines()) == 2 * 9
    buf = io.StringIO()
    res = runner.run(_cfg("polymer_N13_N128_p4096.json", iterations=1, sweeps=3), JsonlLog(buf), out=io.StringIO())
    assert [s["N"] for s in res["systems"]] == [13, 32, 64, 128]
    assert all(len(s["reweight"]) == 3 for s in res["systems"])
