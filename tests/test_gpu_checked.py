"""The checked build (MUCA_DEBUG=1 -> libmuca_checked.so, -DMUCA_CHECKED): every shared-memory
table access of the spin sweeps is bounds-checked.  On healthy runs it must change nothing (bit
for bit against the oracle in every sweep form and in a batch); its failure path is exercised by
the "debug_check" hook, which makes every check fail while every access still reads the table's
first entry, so that no access leaves the table: the next synchronising call reports
MUCA_ERR_CHECK and the context continues from a checkpoint.  The checked library is loaded in a
child process (one library per process)."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
MUCA_ERR_CHECK = -7


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_regular_build_refuses_the_hook():
    import paper_1312_2213_gb300 as m

    g = m.Muca(m.ISING2D, 8, 2, 32, 1)
    with pytest.raises(m.MucaError) as e:
        g.set_param("debug_check", 1)
    assert e.value.code == -1


def test_checked_build_is_bit_exact_and_reports_failed_checks():
    env = dict(os.environ, MUCA_DEBUG="1", PYTHONPATH=ROOT + os.pathsep + os.path.join(ROOT, "tests"))
    r = subprocess.run([sys.executable, os.path.abspath(__file__)], env=env, cwd=ROOT, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "checked build ok" in r.stdout


def _child():
    import numpy as np

    import oracle
    import paper_1312_2213_gb300 as m
    from gpu_util import compare_state

    m.load()
    assert m.library_path().endswith("libmuca_checked.so")
    for system, L, q, pipeline, block in [(m.ISING2D, 16, 2, 2, 64), (m.ISING2D_MUMA, 16, 2, 2, 32),
                                          (m.POTTS2D, 16, 6, 2, 64), (m.ISING2D, 16, 2, 1, 64),
                                          (m.POTTS2D, 16, 6, 1, 64), (m.ISING2D, 16, 2, 0, 64),
                                          (m.POTTS2D, 8, 3, 0, 32), (m.POTTS2D, 64, 10, 2, 32),
                                          (m.POTTS2D, 64, 10, 2, 64)]:
        beta = 0.4407 if system == m.ISING2D_MUMA else 0.0
        g = m.Muca(system, L, q, 70, 5, beta=beta if system == m.ISING2D_MUMA else None, block=block)
        g.set_param("pipeline", pipeline)
        o = oracle.Run(system, L, q, 70, 5, beta=beta)
        o.init()
        for _ in range(3):
            g.iterate(40)
            g.merge_and_update()
            o.iterate(40, 8)
            o.update()
        compare_state(g, o, "checked build, system %d pipeline %d" % (system, pipeline))
        # the failure path: every check fails, every access reads the first table entry
        blob = g.get_state()
        g.set_param("debug_check", 1)
        g.iterate(3)
        try:
            g.synchronize()
            raise AssertionError("no MUCA_ERR_CHECK")
        except m.MucaError as e:
            assert e.code == MUCA_ERR_CHECK, e
        g.set_param("debug_check", 0)
        g.set_state(blob)
        g.iterate(40)
        g.merge_and_update()
        o.iterate(40, 8)
        o.update()
        compare_state(g, o, "after a reported check and a restore")
    mix = [(m.ISING2D, 16, 2, 64, 1), (m.POTTS2D, 16, 10, 64, 2), (m.ISING2D, 32, 2, 40, 3)]
    ref = [m.Muca(s, L, q, p, seed) for s, L, q, p, seed in mix]
    for _ in range(2):
        for c in ref:
            c.iterate(15)
            c.merge_and_update()
    sys_ = [m.Muca(s, L, q, p, seed) for s, L, q, p, seed in mix]
    for form in (1, 0):
        b = m.Batch(sys_, form=form)
        b.run(1, 15, use_graph=form == 1)
        b.close()
    for r, c in zip(ref, sys_):
        np.testing.assert_array_equal(r.lnW().view(np.uint64), c.lnW().view(np.uint64))
        np.testing.assert_array_equal(r.spins(), c.spins())
        c.synchronize()
    print("checked build ok")


if __name__ == "__main__":
    _child()
