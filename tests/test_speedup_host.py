"""Host logic of the statistical-speedup study (Eq. 4 sweep counts, Eq. 6 speedup)."""
import math

import paper_1312_2213_gb300 as m
from paper_1312_2213_gb300 import speedup


def test_m_opt_follows_eq4():
    assert speedup.m_opt(m.ISING2D, 16, 1) == round(5.7 * 16 ** 2.51)
    assert speedup.m_opt(m.ISING2D, 32, 64) == round(5.7 * 32 ** 2.51 / 64)
    assert speedup.m_opt(m.POTTS2D, 16, 4) == round(24 * 16 ** 2.67 / 4)
    assert speedup.m_opt(m.ISING2D_MUMA, 16, 8) == speedup.m_opt(m.ISING2D, 16, 8)
    assert speedup.m_opt(m.ISING2D, 8, 10 ** 6) == 1  # never below one sweep


def test_s_star_is_eq6(monkeypatch):
    fake = {1: [40, 44], 4: [12, 12], 64: [3, 5]}
    monkeypatch.setattr(speedup, "iterations_to_flat",
                        lambda system, L, q, p, seeds, M, max_iter, ratio, beta: fake[p])
    rows = speedup.study(m.ISING2D, 16, 2, [1, 4, 64], 2, 100)
    by_p = {r["p"]: r for r in rows}
    base = 42 * speedup.m_opt(m.ISING2D, 16, 1)
    for p, n in ((4, 12), (64, 4)):
        assert math.isclose(by_p[p]["S_star"], base / (n * speedup.m_opt(m.ISING2D, 16, p)))
    assert by_p[1]["S_star"] == 1.0
    assert math.isclose(by_p[1]["n_iter_err"], 2.0)


def test_unconverged_seeds_are_left_out(monkeypatch):
    monkeypatch.setattr(speedup, "iterations_to_flat",
                        lambda system, L, q, p, seeds, M, max_iter, ratio, beta: [10, None, 14])
    rows = speedup.study(m.ISING2D, 8, 2, [1], 3, 100)
    assert rows[0]["converged"] == 2 and rows[0]["n_iter_mean"] == 12.0


def test_s_star_relative_to_the_smallest_p(monkeypatch):
    """Without p = 1 the study reports p0 S*_p / S*_p0 against the smallest converged p0."""
    fake = {16: [20, 22], 64: [None, None], 256: [30, 30]}
    monkeypatch.setattr(speedup, "iterations_to_flat",
                        lambda system, L, q, p, seeds, M, max_iter, ratio, beta: fake[p])
    rows = speedup.study(m.ISING2D, 32, 2, [16, 64, 256], 2, 100)
    by_p = {r["p"]: r for r in rows}
    assert by_p[16]["S_star_rel"] == 16.0 and by_p[16]["S_star_rel_to_p"] == 16
    assert math.isnan(by_p[64]["S_star_rel"]) and math.isnan(by_p[16]["S_star"])
    want = 16 * 21 * speedup.m_opt(m.ISING2D, 32, 16) / (30 * speedup.m_opt(m.ISING2D, 32, 256))
    assert math.isclose(by_p[256]["S_star_rel"], want)
