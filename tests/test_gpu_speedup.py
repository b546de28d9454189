"""The statistical-speedup driver on the GPU: a tiny study converges and S*_p grows with p."""
import pytest

import paper_1312_2213_gb300 as m
from paper_1312_2213_gb300 import speedup

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_small_study_converges():
    rows = speedup.study(m.ISING2D, 8, 2, [1, 16], 4, 400)
    assert all(r["converged"] == 4 for r in rows)
    by_p = {r["p"]: r for r in rows}
    assert by_p[1]["S_star"] == 1.0
    assert by_p[16]["S_star"] > 4.0
