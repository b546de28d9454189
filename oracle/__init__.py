"""CPU oracle of the parallel multicanonical method (arXiv:1312.2213).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library; the C source (``muca_oracle.c``) is a plain, slow,
one-walker-at-a-time restatement of the method, and ``exact.py`` holds exact
reference results (transfer matrices, Kaufman's closed form) used to pin it.
"""
from __future__ import annotations

import ctypes
import functools
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "muca_oracle.c")
_LIB = os.path.join(_HERE, "libmuca_oracle.so")
_lock = threading.Lock()
_lib = None

ISING, POTTS, MUMA, POLYMER = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the oracle with -O2 -ffp-contract=off (no FMA contraction, no fast-math)."""
    srcs = [_SRC, os.path.join(_HERE, "polymer_oracle.c")]
    srcs = [s for s in srcs if os.path.exists(s)]
    newest = max(os.path.getmtime(s) for s in srcs + [os.path.join(_HERE, "muca_oracle.h")])
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-pthread", "-D_DEFAULT_SOURCE", "-o", tmp] + srcs + ["-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            u32p = ctypes.POINTER(ctypes.c_uint32)
            L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
            L.orc_det_exp.argtypes = [ctypes.c_double]
            L.orc_det_exp.restype = ctypes.c_double
            L.orc_det_log.argtypes = [ctypes.c_double]
            L.orc_det_log.restype = ctypes.c_double
            L.orc_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_uint64, ctypes.c_double, ctypes.c_int]
            L.orc_create.restype = ctypes.c_void_p
            for name in ("orc_free", "orc_init", "orc_update"):
                getattr(L, name).argtypes = [ctypes.c_void_p]
            for name in ("orc_num_bins", "orc_num_cols", "orc_num_sites"):
                getattr(L, name).argtypes = [ctypes.c_void_p]
                getattr(L, name).restype = ctypes.c_int
            L.orc_set_recursion.argtypes = [ctypes.c_void_p, ctypes.c_int]
            L.orc_set_lnW.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
            L.orc_set_observables.argtypes = [ctypes.c_void_p, ctypes.c_int]
            L.orc_get_observables.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
            L.orc_reweight_obs.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_double, ctypes.c_void_p]
            L.orc_reweight_observables.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p]
            L.orc_iterate.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int]
            L.orc_iterate_range.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_int]
            L.orc_advance.argtypes = [ctypes.c_void_p, ctypes.c_int64]
            L.orc_is_flat.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p]
            L.orc_is_flat.restype = ctypes.c_int
            L.orc_reweight.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p]
            for name in ("orc_reachable", "orc_get_lnW", "orc_get_lnW_sampled", "orc_get_histogram",
                         "orc_get_thresholds", "orc_get_spins", "orc_get_bins", "orc_set_open_histogram",
                         "orc_get_open_histogram", "orc_get_metrics"):
                getattr(L, name).argtypes = [ctypes.c_void_p, ctypes.c_void_p]
            L.orc_get_sweep_counter.argtypes = [ctypes.c_void_p]
            L.orc_get_sweep_counter.restype = ctypes.c_int64
            L.orc_bruteforce_ising.argtypes = [ctypes.c_int, ctypes.c_void_p]
            L.orc_bruteforce_ising_EM.argtypes = [ctypes.c_int, ctypes.c_void_p]
            L.orc_bruteforce_potts.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
            for name in ("orc_bruteforce_ising", "orc_bruteforce_ising_EM", "orc_bruteforce_potts"):
                getattr(L, name).restype = ctypes.c_int
            L.orc_tm_ising.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
            L.orc_tm_ising.restype = ctypes.c_int
            L.orc_tm_potts.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
            L.orc_tm_potts.restype = ctypes.c_int
            if hasattr(L, "orc_poly_create"):
                _bind_polymer(L)
            _lib = L
    return _lib


def _bind_polymer(L):
    c = ctypes
    L.orc_poly_create.argtypes = [c.c_int, c.c_int, c.c_uint64, c.c_double, c.c_double, c.c_double,
                                  c.c_double, c.c_int]
    L.orc_poly_create.restype = c.c_void_p
    L.orc_poly_free.argtypes = [c.c_void_p]
    L.orc_poly_init.argtypes = [c.c_void_p]
    L.orc_poly_num_bins.argtypes = [c.c_void_p]
    L.orc_poly_num_bins.restype = c.c_int
    L.orc_poly_iterate.argtypes = [c.c_void_p, c.c_int64, c.c_int]
    L.orc_poly_iterate_range.argtypes = [c.c_void_p, c.c_int64, c.c_int, c.c_int, c.c_int]
    L.orc_poly_advance.argtypes = [c.c_void_p, c.c_int64]
    L.orc_poly_update.argtypes = [c.c_void_p]
    for name in ("orc_poly_get_lnW", "orc_poly_get_lnW_sampled", "orc_poly_get_histogram", "orc_poly_get_coords",
                 "orc_poly_get_energy", "orc_poly_get_bins", "orc_poly_get_counters", "orc_poly_get_metrics"):
        getattr(L, name).argtypes = [c.c_void_p, c.c_void_p]
    L.orc_poly_set_beta.argtypes = [c.c_void_p, c.c_double]
    L.orc_poly_set_model.argtypes = [c.c_void_p, c.c_int]
    L.orc_poly_set_moves.argtypes = [c.c_void_p, c.c_int]
    L.orc_poly_set_grid.argtypes = [c.c_void_p, c.c_int, c.c_double]
    L.orc_poly_set_grid.restype = c.c_int
    L.orc_poly_reweight.argtypes = [c.c_void_p, c.c_double, c.c_void_p, c.c_void_p]
    L.orc_poly_get_walker_events.argtypes = [c.c_void_p, c.c_void_p]
    L.orc_poly_refresh_energy.argtypes = [c.c_void_p]
    L.orc_poly_refresh_energy.restype = c.c_double
    L.orc_poly_energy.argtypes = [c.c_int, c.c_void_p, c.c_int]
    L.orc_poly_energy.restype = c.c_double
    L.orc_poly_pair.argtypes = [c.c_double, c.c_int, c.c_int]
    L.orc_poly_pair.restype = c.c_double
    L.orc_poly_get_first_events.argtypes = [c.c_void_p, c.c_void_p]
    L.orc_poly_get_delta.argtypes = [c.c_void_p, c.c_void_p]
    L.orc_poly_get_drift.argtypes = [c.c_void_p]
    L.orc_poly_get_drift.restype = c.c_double
    L.orc_poly_set_trace.argtypes = [c.c_void_p, c.c_void_p]
    L.orc_poly_set_tau.argtypes = [c.c_void_p, c.c_double]
    L.orc_poly_set_perturbation.argtypes = [c.c_void_p, c.c_double, c.c_uint64]
    L.orc_poly_set_lnW.argtypes = [c.c_void_p, c.c_void_p]
    L.orc_poly_pair_scale.argtypes = [c.c_double, c.c_int, c.c_int]
    L.orc_poly_pair_scale.restype = c.c_double


# One record of the oracle's polymer trace (orc_poly_trace_rec).
POLY_TRACE_DTYPE = np.dtype([("dE", "<f8"), ("scale", "<f8"), ("E", "<f8"), ("delta", "<f8"), ("bin_new", "<i4"),
                             ("bin_after", "<i4"), ("flags", "<i4"), ("pad", "<i4")])


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def philox(ctr, key) -> np.ndarray:
    """One Philox4x32-10 block."""
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32))
    out = np.zeros(4, dtype=np.uint32)
    u32p = ctypes.POINTER(ctypes.c_uint32)
    lib().orc_philox4x32_10(c.ctypes.data_as(u32p), k.ctypes.data_as(u32p), out.ctypes.data_as(u32p))
    return out


def det_exp(x: float) -> float:
    return lib().orc_det_exp(float(x))


def det_log(x: float) -> float:
    return lib().orc_det_log(float(x))


class Run:
    """One oracle MUCA/MUMA run: p walkers sharing one ln W (Fig. 1 scheme)."""

    def __init__(self, system: int, L: int, q: int, p: int, seed: int, beta: float = 0.0, record: int = 0,
                 recursion: int = 0, observables: int = 0):
        self._lib = lib()
        self.h = self._lib.orc_create(system, L, q, p, seed, beta, record)
        if not self.h:
            raise ValueError("oracle: unsupported configuration")
        self._lib.orc_set_recursion(self.h, recursion)
        self._lib.orc_set_observables(self.h, observables)
        self.system, self.L, self.q, self.p, self.seed = system, L, q, p, seed
        self.B = self._lib.orc_num_bins(self.h)
        self.K = self._lib.orc_num_cols(self.h)
        self.N = self._lib.orc_num_sites(self.h)

    def __del__(self):
        if getattr(self, "h", None):
            self._lib.orc_free(self.h)
            self.h = None

    def init(self):
        self._lib.orc_init(self.h)

    def iterate(self, sweeps: int, nthreads: int = 1):
        self._lib.orc_iterate(self.h, sweeps, nthreads)

    def iterate_range(self, sweeps: int, w0: int, w1: int, nthreads: int = 1):
        self._lib.orc_iterate_range(self.h, sweeps, w0, w1, nthreads)

    def advance(self, sweeps: int):
        self._lib.orc_advance(self.h, sweeps)

    def update(self):
        self._lib.orc_update(self.h)

    def set_lnW(self, lnW):
        """Run on at fixed weights: ln W of the reachable bins, -inf elsewhere; thresholds rebuilt."""
        w = np.ascontiguousarray(lnW, dtype=np.float64)
        assert w.shape == (self.B,)
        self._lib.orc_set_lnW(self.h, _ptr(w))

    def observable_sums(self) -> np.ndarray:
        """Per-bin sums (samples, |M|, M^2) of the last update, shape (B, 3)."""
        a = np.zeros(3 * self.B, dtype=np.uint64)
        self._lib.orc_get_observables(self.h, _ptr(a))
        return a.reshape(self.B, 3)

    def reweight_observables(self, beta: float) -> np.ndarray:
        out = np.zeros(3, dtype=np.float64)
        self._lib.orc_reweight_observables(self.h, beta, _ptr(out))
        return out

    def set_open_histogram(self, H):
        H = np.ascontiguousarray(np.asarray(H, dtype=np.uint64))
        assert H.shape == (self.B,)
        self._lib.orc_set_open_histogram(self.h, _ptr(H))

    def open_histogram(self):
        return self._get("orc_get_open_histogram", self.B, np.uint64)

    def is_flat(self, ratio: float = 0.5):
        st = np.zeros(3)
        f = self._lib.orc_is_flat(self.h, ratio, _ptr(st))
        return bool(f), st

    def reweight(self, beta: float):
        out = np.zeros(4)
        lnP = np.zeros(self.B)
        self._lib.orc_reweight(self.h, beta, _ptr(out), _ptr(lnP))
        return out, lnP

    def _get(self, name, n, dtype):
        a = np.zeros(n, dtype=dtype)
        getattr(self._lib, name)(self.h, _ptr(a))
        return a

    def reachable(self):
        return self._get("orc_reachable", self.B, np.uint8).astype(bool)

    def lnW(self):
        return self._get("orc_get_lnW", self.B, np.float64)

    def lnW_sampled(self):
        return self._get("orc_get_lnW_sampled", self.B, np.float64)

    def histogram(self):
        return self._get("orc_get_histogram", self.B, np.uint64)

    def thresholds(self):
        return self._get("orc_get_thresholds", self.B * self.K, np.uint32).reshape(self.B, self.K)

    def spins(self):
        return self._get("orc_get_spins", self.p * self.N, np.int8).reshape(self.p, self.L, self.L)

    def bins(self):
        return self._get("orc_get_bins", self.p, np.int32)

    def sweep_counter(self) -> int:
        return int(self._lib.orc_get_sweep_counter(self.h))

    def metrics(self) -> np.ndarray:
        """{accepted, tunnelling events} of the last closed iteration, the same totals over all
        closed iterations, and the closed iteration's sweeps (uint64[5])."""
        return self._get("orc_get_metrics", 5, np.uint64)


def reweight_obs(N: int, sums: np.ndarray, lnW_sampled: np.ndarray, beta: float) -> np.ndarray:
    """Eq. (2) on per-bin sums (samples, |M|, M^2) of an Ising run (reading R9)."""
    sums = np.ascontiguousarray(np.asarray(sums, dtype=np.uint64).reshape(-1))
    lw = np.ascontiguousarray(np.asarray(lnW_sampled, dtype=np.float64))
    B = lw.size
    assert sums.size == 3 * B
    out = np.zeros(3, dtype=np.float64)
    lib().orc_reweight_obs(B, N, _ptr(sums), _ptr(lw), beta, _ptr(out))
    return out


def bruteforce_ising(L: int) -> np.ndarray:
    N = L * L
    out = np.zeros(N + 1, dtype=np.uint64)
    assert lib().orc_bruteforce_ising(L, _ptr(out)) == 0
    return out


def bruteforce_ising_EM(L: int) -> np.ndarray:
    N = L * L
    out = np.zeros((N + 1) * (N + 1), dtype=np.uint64)
    assert lib().orc_bruteforce_ising_EM(L, _ptr(out)) == 0
    return out.reshape(N + 1, N + 1)


def bruteforce_potts(L: int, q: int) -> np.ndarray:
    N = L * L
    out = np.zeros(2 * N + 1, dtype=np.uint64)
    assert lib().orc_bruteforce_potts(L, q, _ptr(out)) == 0
    return out


def _u128(a: np.ndarray) -> list:
    return [int(a[2 * i]) + (int(a[2 * i + 1]) << 64) for i in range(a.size // 2)]


@functools.lru_cache(maxsize=None)
def tm_ising(L: int) -> list:
    """Exact Omega(E) of the periodic L x L Ising model (Python ints), index (E+2N)/4."""
    N = L * L
    out = np.zeros(2 * (N + 1), dtype=np.uint64)
    assert lib().orc_tm_ising(L, 0, _ptr(out)) == 0
    return _u128(out)


@functools.lru_cache(maxsize=None)
def tm_ising_EM(L: int) -> list:
    """Exact Omega(E, M), as a list of rows [(E+2N)/4][(M+N)/2] of Python ints."""
    N = L * L
    out = np.zeros(2 * (N + 1) * (N + 1), dtype=np.uint64)
    assert lib().orc_tm_ising(L, 1, _ptr(out)) == 0
    flat = _u128(out)
    return [flat[i * (N + 1):(i + 1) * (N + 1)] for i in range(N + 1)]


@functools.lru_cache(maxsize=None)
def tm_potts(L: int, q: int) -> list:
    """Exact Omega(E) of the periodic L x L q-state Potts model, index E+2N."""
    N = L * L
    out = np.zeros(2 * (2 * N + 1), dtype=np.uint64)
    assert lib().orc_tm_potts(L, q, _ptr(out)) == 0
    return _u128(out)


class PolyRun:
    """Oracle multicanonical run of a bead-spring polymer of N beads (p walkers)."""

    def __init__(self, N: int, p: int, seed: int, e_lo: float, e_hi: float, K: float = 40.0, R: float = 1.5,
                 record: int = 0, beta: float = 0.0, model: int = 0, moves: int = 0, bin_k: int = 10,
                 step_q: int = 1229):
        self._lib = lib()
        self.h = self._lib.orc_poly_create(N, p, seed, e_lo, e_hi, K, R, record)
        if not self.h:
            raise ValueError("oracle: bad polymer configuration")
        self.N, self.p = N, p
        if (bin_k, step_q) != (10, 1229) and self._lib.orc_poly_set_grid(self.h, bin_k, float(step_q)) < 0:
            raise ValueError("oracle: bad bin width or step")
        self.B = self._lib.orc_poly_num_bins(self.h)
        if beta > 0:
            self._lib.orc_poly_set_beta(self.h, beta)
        if model:
            self._lib.orc_poly_set_model(self.h, model)
        if moves:
            self._lib.orc_poly_set_moves(self.h, moves)

    def __del__(self):
        if getattr(self, "h", None):
            self._lib.orc_poly_free(self.h)
            self.h = None

    def init(self):
        self._lib.orc_poly_init(self.h)

    def iterate(self, sweeps: int, nthreads: int = 1):
        self._lib.orc_poly_iterate(self.h, sweeps, nthreads)

    def iterate_range(self, sweeps: int, w0: int, w1: int, nthreads: int = 1):
        self._lib.orc_poly_iterate_range(self.h, sweeps, w0, w1, nthreads)

    def advance(self, sweeps: int):
        self._lib.orc_poly_advance(self.h, sweeps)

    def update(self):
        self._lib.orc_poly_update(self.h)

    def refresh_energy(self) -> float:
        return self._lib.orc_poly_refresh_energy(self.h)

    def drift(self) -> float:
        """Largest change of a running energy at the refresh after a call, since init."""
        return self._lib.orc_poly_get_drift(self.h)

    def first_events(self) -> np.ndarray:
        """Per walker, the attempt index (sweep * N + bead) of the first event of the last call,
        N * sweeps if only its closing refresh was one, -1 if none."""
        return self._get("orc_poly_get_first_events", self.p, np.int64)

    def delta(self) -> np.ndarray:
        """Per walker, the bound on the energy difference of an FP32 implementation."""
        return self._get("orc_poly_get_delta", self.p, np.float64)

    def set_perturbation(self, perturb: float, seed: int = 99):
        """Plant an error of up to perturb * sigma in every pair term (tests of the event rule)."""
        self._lib.orc_poly_set_perturbation(self.h, perturb, seed)

    def set_lnW(self, lnW):
        lnW = np.ascontiguousarray(lnW, dtype=np.float64)
        assert lnW.shape == (self.B,)
        self._lib.orc_poly_set_lnW(self.h, _ptr(lnW))

    def iterate_traced(self, sweeps: int, nthreads: int = 1) -> np.ndarray:
        """Run `sweeps` sweeps and return the record of every attempt, shape (p, sweeps, N)."""
        t = np.zeros(self.p * sweeps * self.N, dtype=POLY_TRACE_DTYPE)
        self._lib.orc_poly_set_trace(self.h, t.ctypes.data_as(ctypes.c_void_p))
        try:
            self.iterate(sweeps, nthreads)
        finally:
            self._lib.orc_poly_set_trace(self.h, None)
        return t.reshape(self.p, sweeps, self.N)

    def iterate_range_traced(self, sweeps: int, w0: int, w1: int, nthreads: int = 1) -> np.ndarray:
        """Run `sweeps` sweeps of walkers [w0, w1) (the sweep counter does not advance: call
        advance() once for all ranges) and return their records, shape (w1 - w0, sweeps, N)."""
        t = np.zeros((w1 - w0) * sweeps * self.N, dtype=POLY_TRACE_DTYPE)
        self._lib.orc_poly_set_trace(self.h, t.ctypes.data_as(ctypes.c_void_p))
        try:
            self.iterate_range(sweeps, w0, w1, nthreads)
        finally:
            self._lib.orc_poly_set_trace(self.h, None)
        return t.reshape(w1 - w0, sweeps, self.N)

    def walker_energies(self, idx) -> tuple:
        """(energies, bounds delta) of the given walkers."""
        idx = np.asarray(idx)
        return self.energy()[idx], self.delta()[idx]

    def _get(self, name, n, dtype):
        a = np.zeros(n, dtype=dtype)
        getattr(self._lib, name)(self.h, _ptr(a))
        return a

    def lnW(self):
        return self._get("orc_poly_get_lnW", self.B, np.float64)

    def lnW_sampled(self):
        return self._get("orc_poly_get_lnW_sampled", self.B, np.float64)

    def histogram(self):
        return self._get("orc_poly_get_histogram", self.B, np.uint64)

    def coords(self):
        return self._get("orc_poly_get_coords", self.p * self.N * 3, np.float64).reshape(self.p, self.N, 3)

    def energy(self):
        return self._get("orc_poly_get_energy", self.p, np.float64)

    def bins(self):
        return self._get("orc_poly_get_bins", self.p, np.int32)

    def counters(self):
        return self._get("orc_poly_get_counters", 2, np.int64)

    def walker_events(self):
        return self._get("orc_poly_get_walker_events", 2 * self.p, np.int64).reshape(self.p, 2)

    def metrics(self) -> np.ndarray:
        return self._get("orc_poly_get_metrics", 5, np.uint64)

    def reweight(self, beta: float):
        out = np.zeros(4)
        lnP = np.zeros(self.B)
        self._lib.orc_poly_reweight(self.h, beta, _ptr(out), _ptr(lnP))
        return out, lnP


def poly_energy(X: np.ndarray, model: int = 0) -> float:
    X = np.ascontiguousarray(X, dtype=np.float64)
    return lib().orc_poly_energy(X.shape[0], _ptr(X), model)


def poly_pair(r: float, sep: int, model: int = 0) -> float:
    return lib().orc_poly_pair(float(r), int(sep), int(model))


def poly_pair_scale(r: float, sep: int, model: int = 0) -> float:
    """First-order error scale |v(r)| + |r v'(r)| of a pair term."""
    return lib().orc_poly_pair_scale(float(r), int(sep), int(model))
