"""The statistical-speedup driver (Eq. 4 sweeps per iteration, Eq. 6 S*_p) on the GPU against the
same study run on the oracle.

Every seed's GPU histograms are bit-identical to the oracle's, so the iteration at which a seed's
merged histogram first becomes flat must be the same on both sides, seed by seed, and with it the
mean iteration counts and S*_p.  A mistake in the driver (a seed merged into another, the stopping
rule, the sweep count of an iteration) shows up as a differing count."""
import numpy as np
import pytest

import oracle
import paper_1312_2213_gb300 as m
from paper_1312_2213_gb300 import speedup

pytestmark = pytest.mark.gpu
NT = 8


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def oracle_iterations_to_flat(system, L, q, p, seeds, sweeps, max_iter, ratio=0.5, beta=0.0):
    out = []
    for s in seeds:
        r = oracle.Run(system, L, q, p, int(s), beta=beta)
        r.init()
        n = None
        for it in range(1, max_iter + 1):
            r.iterate(sweeps, NT)
            r.update()
            if r.is_flat(ratio)[0]:
                n = it
                break
        out.append(n)
    return out


@pytest.mark.parametrize("system,q,beta", [(m.ISING2D, 2, None), (m.POTTS2D, 8, None), (m.ISING2D_MUMA, 2, 0.4407)])
def test_study_matches_the_oracle_seed_by_seed(system, q, beta):
    L, p_values, n_seeds, max_iter, seed0 = 8, [1, 16, 64], 4, 400, 1000
    rows = speedup.study(system, L, q, p_values, n_seeds, max_iter, beta=beta, seed0=seed0)
    cost = {}
    for r in rows:
        p = r["p"]
        M = speedup.m_opt(system, L, p, q)
        assert r["sweeps_per_iteration"] == M
        seeds = [seed0 + 7919 * k + p for k in range(n_seeds)]
        g = speedup.iterations_to_flat(system, L, q, p, seeds, M, max_iter, beta=beta)
        o = oracle_iterations_to_flat(system, L, q, p, seeds, M, max_iter, beta=beta or 0.0)
        assert g == o, (p, g, o)
        assert all(n is not None for n in o)
        assert r["converged"] == n_seeds
        assert r["n_iter_mean"] == pytest.approx(np.mean(o), rel=1e-12)
        cost[p] = np.mean(o) * M
    by_p = {r["p"]: r for r in rows}
    for p in p_values:
        assert by_p[p]["S_star"] == pytest.approx(cost[1] / cost[p], rel=1e-12)
    assert by_p[16]["S_star"] > 4.0
