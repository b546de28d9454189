"""Helpers for the GPU parity tests: run the CUDA path and the oracle side by side."""
import numpy as np

import oracle
import paper_1312_2213_gb300 as m


def lattice_equal(gpu_spins, orc_spins):
    return np.array_equal(gpu_spins.astype(np.int8), orc_spins.astype(np.int8))


def compare_state(g, o, what=""):
    np.testing.assert_array_equal(g.bins(), o.bins(), err_msg="bins " + what)
    np.testing.assert_array_equal(g.spins(), o.spins(), err_msg="spins " + what)
    np.testing.assert_array_equal(g.thresholds(), o.thresholds(), err_msg="thresholds " + what)
    # ln W bit for bit (compare the binary64 encodings, -inf included)
    np.testing.assert_array_equal(g.lnW().view(np.uint64), o.lnW().view(np.uint64), err_msg="lnW " + what)
    np.testing.assert_array_equal(g.lnW_sampled().view(np.uint64), o.lnW_sampled().view(np.uint64),
                                  err_msg="lnW_sampled " + what)
    np.testing.assert_array_equal(g.histogram(), o.histogram(), err_msg="H " + what)


def run_pair(system, L, q, p, seed, iters, sweeps, beta=0.0, record=0, block=None, nthreads=8, check_each=True,
             pipeline=None, recursion=0):
    g = m.Muca(system, L, q, p, seed, beta=beta if system == m.ISING2D_MUMA else None, record=record, block=block)
    if pipeline is not None:
        g.set_param("pipeline", pipeline)
    if recursion:
        g.set_param("recursion", recursion)
    o = oracle.Run(system, L, q, p, seed, beta=beta, record=record, recursion=recursion)
    o.init()
    compare_state(g, o, "after init")
    for it in range(iters):
        g.iterate(sweeps)
        g.merge_and_update()
        o.iterate(sweeps, nthreads)
        o.update()
        if check_each or it == iters - 1:
            compare_state(g, o, "after iteration %d" % it)
    return g, o
