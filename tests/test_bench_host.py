"""bench.py host logic without a GPU: the clock record taken during the timed region (median SM
clock under load, its maximum, and the throttle reasons seen)."""
import importlib.util
import os
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


class _Proc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _sampler_with(lines):
    bench = _bench()
    s = bench.ClockSampler(0)
    fd, s.path = tempfile.mkstemp(suffix=".csv")
    with os.fdopen(fd, "w") as f:
        f.write("\n".join(lines) + "\n")
    s.proc = _Proc()
    return s


def test_clock_record_median_max_and_reasons():
    lines = ["0, 2070, 2070, 910.2, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
             "0, 1980, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
             "0, 2070, 2070, 1200.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
             "garbage line",
             "0, [N/A], 2070, 0.0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    s = _sampler_with(lines)
    path = s.path
    rec = s.stop()
    assert rec == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    assert not os.path.exists(path)


def test_clock_record_flags_thermal_slowdown():
    lines = ["0, 1500, 2070, 1400.0, 0x0000000000000040, Not Active, Active, Not Active, Not Active",
             "0, 1600, 2070, 1400.0, 0x0000000000000020, Not Active, Not Active, Active, Not Active"]
    rec = _sampler_with(lines).stop()
    assert rec["reasons"] == ["hw_thermal_slowdown", "sw_thermal_slowdown"]
    assert rec["sm_mhz"] == 1550.0


def test_no_samples_gives_no_record():
    assert _sampler_with(["not csv"]).stop() is None
    assert _bench().ClockSampler(0).stop() is None   # nvidia-smi never started


def test_mix_iteration_lengths_follow_eq4():
    """The mix's third regime runs every system at its own M_opt from the fits of Eq. 4 at
    p = 2048: 5.7 L^2.51 / p for Ising, 24 L^2.67 / p (the 8-Potts fit) for q = 10 Potts."""
    bench = _bench()
    got = dict(zip(bench.MIX, bench.mix_mopt()))
    for (system, L, q), m_opt in got.items():
        exact = (5.7 * L ** 2.51 if system == 0 else 24.0 * L ** 2.67) / 2048
        assert m_opt == max(1, round(exact)) and abs(m_opt - exact) <= 0.5
    assert got[(0, 64, 2)] == 95 and got[(1, 48, 10)] == 361
