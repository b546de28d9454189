"""GPU parity of the spin hot path (sweep -> histogram -> merge -> recursion -> thresholds)
against the oracle, through the C ABI.  Ising / Potts / multimagnetic histograms, lattices,
walker bins, ln W and thresholds must agree bit for bit (the integer-threshold acceptance
and the deterministic binary64 recursion make the two paths identical)."""
import numpy as np
import pytest

import oracle
import paper_1312_2213_gb300 as m
from gpu_util import compare_state, run_pair

pytestmark = pytest.mark.gpu

NT = 16


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    m.load()


def test_det_math_bitwise_equals_oracle():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.uniform(-23, 0, 200000), rng.uniform(-745, 709, 50000), [0.0, -1e-300, -800.0]])
    ge = m.muca_det_math(0, x)
    oe = np.array([oracle.det_exp(v) for v in x])
    np.testing.assert_array_equal(ge.view(np.uint64), oe.view(np.uint64))
    y = np.concatenate([rng.integers(1, 2**53, 200000).astype(np.float64), 10.0 ** rng.uniform(-300, 300, 50000),
                        [1.0, 2.0, 5e-324, np.inf]])
    gl = m.muca_det_math(1, y)
    ol = np.array([oracle.det_log(v) for v in y])
    np.testing.assert_array_equal(gl.view(np.uint64), ol.view(np.uint64))


@pytest.mark.parametrize("system,L,q,p", [
    (m.ISING2D, 4, 2, 37), (m.ISING2D, 8, 2, 64), (m.ISING2D, 12, 2, 33), (m.ISING2D, 16, 2, 100),
    (m.ISING2D, 24, 2, 70), (m.ISING2D, 32, 2, 130), (m.ISING2D, 48, 2, 40), (m.ISING2D, 64, 2, 35),
    (m.POTTS2D, 4, 3, 37), (m.POTTS2D, 8, 8, 64), (m.POTTS2D, 16, 10, 65), (m.POTTS2D, 32, 8, 96),
    (m.POTTS2D, 48, 10, 33), (m.POTTS2D, 16, 2, 40), (m.POTTS2D, 12, 16, 40),
    (m.ISING2D_MUMA, 8, 2, 50), (m.ISING2D_MUMA, 32, 2, 100), (m.ISING2D_MUMA, 64, 2, 33),
])
def test_iterations_bit_exact(system, L, q, p):
    """Several tiles and a ragged last block; every iteration compared."""
    sweeps = max(2, 4000 // (L * L))
    run_pair(system, L, q, p, seed=1000 + L + q, iters=4, sweeps=sweeps, beta=0.4407, nthreads=NT)


@pytest.mark.parametrize("system,L,q,p", [(m.ISING2D, 32, 2, 100), (m.POTTS2D, 16, 10, 70), (m.ISING2D_MUMA, 24, 2, 65),
                                          (m.POTTS2D, 48, 8, 40), (m.ISING2D, 64, 2, 33)])
def test_one_warp_form_bit_exact(system, L, q, p):
    """pipeline = 0 (one warp runs its walkers' random numbers and chains) gives the same bits."""
    run_pair(system, L, q, p, seed=77 + L, iters=3, sweeps=max(2, 3000 // (L * L)), beta=0.4407, nthreads=NT,
             pipeline=0)


@pytest.mark.parametrize("system,L,q,p", [(m.ISING2D, 32, 2, 100), (m.POTTS2D, 16, 10, 70), (m.ISING2D_MUMA, 24, 2, 65),
                                          (m.ISING2D, 64, 2, 33)])
def test_random_pipeline_bit_exact(system, L, q, p):
    """pipeline = 1 (producer warps compute the random numbers only) gives the same bits."""
    run_pair(system, L, q, p, seed=91 + L, iters=3, sweeps=max(2, 3000 // (L * L)), beta=0.4407, nthreads=NT,
             pipeline=1)


@pytest.mark.parametrize("system,L,q,p,block", [
    (m.ISING2D, 8, 2, 64, None), (m.ISING2D, 16, 2, 100, None), (m.ISING2D, 24, 2, 70, None),
    (m.ISING2D, 32, 2, 130, None), (m.ISING2D, 48, 2, 40, None), (m.ISING2D, 64, 2, 35, None),
    (m.ISING2D_MUMA, 8, 2, 50, None), (m.ISING2D_MUMA, 32, 2, 100, None), (m.ISING2D_MUMA, 48, 2, 33, None),
    (m.POTTS2D, 8, 3, 64, None), (m.POTTS2D, 12, 5, 45, None), (m.POTTS2D, 16, 10, 100, None),
    (m.POTTS2D, 24, 8, 70, None), (m.POTTS2D, 32, 8, 130, None), (m.POTTS2D, 32, 2, 40, None),
    (m.POTTS2D, 48, 10, 40, 32)])
def test_code_pipeline_bit_exact(system, L, q, p, block):
    """pipeline = 2 (the producer also computes the per-site codes) gives the same bits; Potts L = 48
    with 32 walkers a block runs the two-row ring, the others the four-row ring."""
    run_pair(system, L, q, p, seed=500 + L + q, iters=4, sweeps=max(2, 4000 // (L * L)), beta=0.4407, nthreads=NT,
             pipeline=2, block=block)


@pytest.mark.parametrize("system,L,q,p", [(m.ISING2D, 16, 2, 64), (m.POTTS2D, 16, 8, 70), (m.ISING2D_MUMA, 16, 2, 40),
                                          (m.ISING2D, 32, 2, 100)])
def test_plain_recursion_bit_exact(system, L, q, p):
    """recursion = 1 (the plain W/H update) matches the oracle bit for bit at every iteration."""
    run_pair(system, L, q, p, seed=123 + L, iters=5, sweeps=max(2, 3000 // (L * L)), beta=0.4407, nthreads=NT,
             recursion=1)


def test_config_ising_L8_p64_full_length():
    """Ising L = 8, p = 64, 10 iterations of 1e4 sweeps: bit-exact at every iteration."""
    g, o = run_pair(m.ISING2D, 8, 2, 64, seed=1, iters=10, sweeps=10000, nthreads=NT)
    flat, _ = o.is_flat(0.5)
    assert flat and g.merge_and_update is not None


@pytest.mark.parametrize("pipeline", [0, 1, 2])
def test_record_per_sweep(pipeline):
    """record = 1 (one count per walker per sweep) in every form of the sweep."""
    run_pair(m.ISING2D, 16, 2, 64, seed=5, iters=3, sweeps=50, record=1, nthreads=NT, pipeline=pipeline)
    run_pair(m.POTTS2D, 16, 5, 64, seed=6, iters=3, sweeps=50, record=1, nthreads=NT, pipeline=pipeline)
    run_pair(m.ISING2D_MUMA, 16, 2, 40, seed=7, iters=3, sweeps=50, beta=0.4407, record=1, nthreads=NT,
             pipeline=pipeline)


@pytest.mark.parametrize("block", [32, 64, 96, 256, 512])
def test_block_size_does_not_change_results(block):
    """Explicit walkers per block (the default for q-Potts at p = 300 is 32: every block has an
    SM to itself); 64 is the code form's two-consumer block."""
    run_pair(m.POTTS2D, 16, 8, 300, seed=7, iters=2, sweeps=20, block=block, nthreads=NT)


def test_full_size_first_iteration_sampled_walkers():
    """Config sizes (Ising L=32, Potts q=8 L=32, MUMA L=32; p = 8192): one full iteration of
    1e4 sweeps in the benchmark's launch configuration; sampled walkers recomputed one by one
    by the oracle must match bit for bit, and the merged histogram must hold p*sweeps*N counts."""
    sweeps = 10000
    for system, q in ((m.ISING2D, 2), (m.POTTS2D, 8), (m.ISING2D_MUMA, 2)):
        p, L = 8192, 32
        g = m.Muca(system, L, q, p, 11, beta=0.4407 if system == m.ISING2D_MUMA else None)
        g.iterate(sweeps)
        g.merge_and_update()
        assert int(g.histogram().sum()) == p * sweeps * L * L
        gs, gb = g.spins(), g.bins()
        o = oracle.Run(system, L, q, p, 11, beta=0.4407)
        o.init()
        sample = [0, 1, 31, 32, 4095, 8191]
        for w in sample:
            o.iterate_range(sweeps, w, w + 1, 1)
        os_, ob = o.spins(), o.bins()
        for w in sample:
            np.testing.assert_array_equal(gs[w], os_[w])
            assert gb[w] == ob[w]


def test_full_size_bookkeeping_after_several_iterations():
    """At full size the walkers' bins always equal the bins recomputed from their lattices."""
    from test_oracle_muca import bins_from_spins

    for system, q in ((m.ISING2D, 2), (m.POTTS2D, 8), (m.ISING2D_MUMA, 2)):
        g = m.Muca(system, 32, q, 8192, 12, beta=0.4407 if system == m.ISING2D_MUMA else None)
        for _ in range(3):
            g.iterate(300)
            g.merge_and_update()
        np.testing.assert_array_equal(g.bins(), bins_from_spins(g.spins(), system))
        assert int(g.histogram().sum()) == 8192 * 300 * 1024
        assert g.sweep_counter() == 900


def test_reweight_matches_oracle():
    g, o = run_pair(m.ISING2D, 8, 2, 64, seed=3, iters=6, sweeps=3000, nthreads=NT, check_each=False)
    for beta in (0.2, 0.44, 0.8):
        go, glp = g.reweight(beta)
        oo, olp = o.reweight(beta)
        np.testing.assert_allclose(go, oo, rtol=1e-12, atol=1e-12)
        fin = np.isfinite(olp)
        np.testing.assert_array_equal(np.isfinite(glp), fin)
        np.testing.assert_allclose(glp[fin], olp[fin], rtol=1e-12, atol=1e-11)
    gm, om_ = run_pair(m.ISING2D_MUMA, 8, 2, 64, seed=4, iters=5, sweeps=2000, beta=0.4407, nthreads=NT,
                       check_each=False)
    go, _ = gm.reweight(0.0)
    oo, _ = om_.reweight(0.0)
    np.testing.assert_allclose(go, oo, rtol=1e-12, atol=1e-12)


def test_checkpoint_resume_is_bit_exact():
    a = m.Muca(m.POTTS2D, 16, 8, 200, 21)
    for _ in range(4):
        a.iterate(100)
        a.merge_and_update()
    b = m.Muca(m.POTTS2D, 16, 8, 200, 21)
    for _ in range(2):
        b.iterate(100)
        b.merge_and_update()
    b.iterate(30)                 # an open (unmerged) iteration is part of the state
    st = b.get_state()
    c = m.Muca(m.POTTS2D, 16, 8, 200, 21)
    c.set_state(st)
    c.iterate(70)
    c.merge_and_update()
    for _ in range(1):
        c.iterate(100)
        c.merge_and_update()
    for f in ("lnW", "histogram", "spins", "bins", "thresholds"):
        np.testing.assert_array_equal(getattr(a, f)(), getattr(c, f)())
    assert a.sweep_counter() == c.sweep_counter()


def test_walker_shards_reproduce_one_context():
    """Two contexts holding walkers [0, 60) and [60, 128) (walker_offset) draw the same streams
    as one context of 128 walkers: lattices agree and the histograms add up (the merge is an
    integer sum)."""
    full = m.Muca(m.ISING2D, 16, 2, 128, 9)
    s0 = m.Muca(m.ISING2D, 16, 2, 60, 9)
    s1 = m.Muca(m.ISING2D, 16, 2, 68, 9, walker_offset=60)
    for c in (full, s0, s1):
        c.iterate(40)
        c.merge_and_update()
    np.testing.assert_array_equal(full.spins()[:60], s0.spins())
    np.testing.assert_array_equal(full.spins()[60:], s1.spins())
    np.testing.assert_array_equal(full.histogram(), s0.histogram() + s1.histogram())


def test_torch_arena_and_stream():
    import torch

    s = torch.cuda.Stream()
    a = m.Muca(m.ISING2D, 16, 2, 64, 5, arena="torch", stream=s)
    b = m.Muca(m.ISING2D, 16, 2, 64, 5)
    for c in (a, b):
        c.iterate(25)
        c.merge_and_update()
    np.testing.assert_array_equal(a.histogram(), b.histogram())
    np.testing.assert_array_equal(a.lnW(), b.lnW())


def test_errors_are_reported_not_raised_in_c():
    with pytest.raises(m.MucaError):
        m.Muca(m.ISING2D, 30, 2, 64, 1)
    g = m.Muca(m.ISING2D, 8, 2, 8, 1)
    with pytest.raises(m.MucaError):
        m.muca_get_lnW(g.h, np.zeros(3))
    g.iterate(1)
    with pytest.raises(m.MucaError) as e:
        g.set_param("record", 1)
    assert e.value.code == -5
    with pytest.raises(m.MucaError):
        g.set_param("nonsense", 1)
    with pytest.raises(m.MucaError):
        g.iterate(0)
    bad = np.zeros(10, dtype=np.uint8)
    with pytest.raises(m.MucaError):
        g.set_state(bad)


def test_p_equals_one_and_tiny_lattice():
    run_pair(m.ISING2D, 4, 2, 1, seed=8, iters=3, sweeps=200, nthreads=1)
    run_pair(m.POTTS2D, 4, 16, 1, seed=8, iters=3, sweeps=200, nthreads=1)
    run_pair(m.ISING2D_MUMA, 4, 2, 1, seed=8, iters=3, sweeps=200, beta=0.4407, nthreads=1)
    # one walker in a 32-lane consumer warp of the code form (31 inactive lanes)
    run_pair(m.ISING2D, 8, 2, 1, seed=9, iters=3, sweeps=100, nthreads=1, pipeline=2)
    run_pair(m.POTTS2D, 8, 5, 1, seed=9, iters=3, sweeps=100, nthreads=1, pipeline=2)


@pytest.mark.parametrize("pipeline,L,p", [(0, 8, 64), (1, 16, 70), (2, 16, 70), (2, 32, 100)])
def test_observables_bit_exact(pipeline, L, p):
    """Per-sweep sums of 1, |M| and M^2 per energy bin (Ising) match the oracle bit for bit in
    every sweep form, and the Eq. 2 reweighting of them agrees to rounding."""
    S = max(2, 2000 // (L * L))
    g = m.Muca(m.ISING2D, L, 2, p, 41)
    g.set_param("pipeline", pipeline)
    g.set_param("observables", 1)
    o = oracle.Run(0, L, 2, p, 41, observables=1)
    o.init()
    for _ in range(3):
        g.iterate(S)
        g.merge_and_update()
        o.iterate(S, NT)
        o.update()
        out, sums = g.observables(0.4)
        np.testing.assert_array_equal(sums, o.observable_sums())
        assert int(sums[:, 0].sum()) == p * S
        np.testing.assert_allclose(out, o.reweight_observables(0.4), rtol=1e-12, atol=0)
    compare_state(g, o, "with observables")


def test_observables_refused_where_not_recorded():
    g = m.Muca(m.POTTS2D, 8, 3, 8, 1)
    with pytest.raises(m.MucaError):
        g.set_param("observables", 1)
    h = m.Muca(m.ISING2D, 8, 2, 8, 1)
    with pytest.raises(m.MucaError):
        h.observables(0.4)


def _state_offsets(g, C):
    """Byte offsets of the lattice and bin sections in a spin state buffer (header first)."""
    WR = (4 * g.L + 31) // 32 if g.system == m.POTTS2D else (g.L + 31) // 32
    pstride = (g.p + 31) // 32 * 32
    lat_b = g.L * WR * pstride * 4
    sizes = [lat_b, 4 * g.p] + [8 * g.B] * 6 + [4 * g.B * C, 48 * g.B, 64, g.p]
    blob = g.get_state()
    head = blob.nbytes - sum(sizes)
    return blob, head, head + lat_b, WR, pstride


@pytest.mark.parametrize("system,L,q,C", [(m.ISING2D, 24, 2, 5), (m.POTTS2D, 16, 5, 9), (m.ISING2D_MUMA, 16, 2, 10)])
def test_state_buffer_must_be_consistent(system, L, q, C):
    """muca_set_state refuses a buffer whose walker bin disagrees with its lattice, a Potts colour
    >= q, or set bits past a row's last site (the sweeps would move such a bin off the tables);
    the untouched buffer is accepted."""
    g = m.Muca(system, L, q, 40, 3, beta=0.4407 if system == m.ISING2D_MUMA else None)
    g.iterate(20)
    g.merge_and_update()
    blob, head, bins_off, WR, pstride = _state_offsets(g, C)
    c = m.Muca(system, L, q, 40, 3, beta=0.4407 if system == m.ISING2D_MUMA else None)
    c.set_state(blob)  # consistent
    np.testing.assert_array_equal(c.spins(), g.spins())

    bad = blob.copy()
    bins = bad[bins_off:bins_off + 4 * 40].view(np.int32)
    bins[7] += 1 if bins[7] + 1 < g.B else -1  # a bin that is not its lattice's
    with pytest.raises(m.MucaError) as e:
        c.set_state(bad)
    assert e.value.code == -1 and "bin" in str(e.value)

    bad = blob.copy()
    lat = bad[head:bins_off].view(np.uint32)
    if system == m.POTTS2D:
        lat[0 * pstride + 5] = (lat[0 * pstride + 5] & ~np.uint32(0xF)) | np.uint32(q)  # colour q at site 0
    else:
        lat[0 * pstride + 5] |= np.uint32(1 << (L % 32 if L % 32 else 31))  # past the row (L = 24) or a site
    with pytest.raises(m.MucaError):
        c.set_state(bad)
    c.set_state(blob)
    c.iterate(5)
    g.iterate(5)
    np.testing.assert_array_equal(c.spins(), g.spins())


@pytest.mark.parametrize("record", [0, 1])
@pytest.mark.parametrize("pipeline", [2, 0])
def test_potts_L64_bit_exact(record, pipeline):
    """q-Potts at L = 64: 8193 bins x 9 columns of 32-bit thresholds (295 KB) do not fit a block's
    shared memory.  The code form (pipeline 2) keeps 16-bit stand-ins of their upper halves there,
    decides on those and redoes a walker's row exactly when one of its sites had equal halves (u
    recomputed from its Philox block, T read from the global table); the one-warp form
    (pipeline 0) reads the full table from global memory.  Bit-exact against the oracle over 64
    walkers x 3 x 10 sweeps = 7.9e6 attempts; in the second and third iterations, where the
    thresholds are no longer all 'always', a few tens of sites tie (2^-16 an attempt), and about
    half of them the full words accept where the halves alone would have rejected."""
    run_pair(m.POTTS2D, 64, 10, 64, 17, 3, 10, record=record, nthreads=NT, pipeline=pipeline)


@pytest.mark.parametrize("q,block", [(10, 64), (5, 32)])
def test_potts_L64_many_redone_rows(q, block):
    """The row redo behind the split table at scale: 608 walkers x 3 x 12 sweeps = 9e7 attempts, of
    which some 700 tie on the 16-bit stand-ins (2^-16 an attempt whose threshold is not 'always'),
    so rows with a tie on the last site, with two ties, and ties in both blocks' consumers all
    occur.  Bit-exact against the oracle after every iteration."""
    run_pair(m.POTTS2D, 64, q, 608, 23, 3, 12, block=block, nthreads=NT)


def test_potts_L64_q2_split_table():
    """q = 2 at L = 64 in the code form: the odd bins are unreachable (threshold 0 into them)."""
    run_pair(m.POTTS2D, 64, 2, 40, 5, 2, 8, nthreads=NT)


def test_potts_L64_in_a_batch():
    """Side by side (form 1) a batch runs it; the persistent tile form refuses it."""
    cfg = [(m.POTTS2D, 64, 10, 40, 3), (m.ISING2D, 16, 2, 64, 4)]
    ref = [m.Muca(s, L, q, p, seed) for s, L, q, p, seed in cfg]
    for _ in range(2):
        for c in ref:
            c.iterate(8)
            c.merge_and_update()
    sys_ = [m.Muca(s, L, q, p, seed) for s, L, q, p, seed in cfg]
    b = m.Batch(sys_)
    with pytest.raises(m.MucaError):
        b.set_form(0)
    b.run(2, 8, use_graph=True)
    for r, c in zip(ref, sys_):
        np.testing.assert_array_equal(r.lnW().view(np.uint64), c.lnW().view(np.uint64))
        np.testing.assert_array_equal(r.spins(), c.spins())
        assert r.metrics() == c.metrics()
    b.close()


@pytest.mark.parametrize("system,q", [(m.ISING2D, 2), (m.POTTS2D, 8), (m.ISING2D_MUMA, 2)])
def test_full_size_bit_exact_with_nontrivial_weights(system, q):
    """Benchmark size and launch configuration (L = 32, p = 8192, code form, 64 walkers a block):
    four short iterations, so that the later ones run on weights the earlier histograms set
    (thresholds below "always"), compared with the oracle over all walkers bit for bit."""
    run_pair(system, 32, q, 8192, 23, 4, 20, beta=0.4407 if system == m.ISING2D_MUMA else 0.0, nthreads=NT)


@pytest.mark.parametrize("system,L,q", [(m.ISING2D, 8, 2), (m.POTTS2D, 8, 4), (m.ISING2D_MUMA, 8, 2)])
def test_flatness_matches_oracle(system, L, q):
    """The device's flatness statistic (min, mean, max over the reachable bins) and its flat
    decision equal the oracle's after every iteration."""
    beta = 0.4407 if system == m.ISING2D_MUMA else 0.0
    g = m.Muca(system, L, q, 48, 6, beta=beta if system == m.ISING2D_MUMA else None)
    o = oracle.Run(system, L, q, 48, 6, beta=beta)
    o.init()
    for _ in range(8):
        g.iterate(200)
        flat_g = g.merge_and_update(want_flat=True)
        o.iterate(200, NT)
        o.update()
        flat_o, st = o.is_flat(0.5)
        np.testing.assert_array_equal(g.flatness(), st)
        assert flat_g == flat_o
