"""GB300 (sm_103a) parallel multicanonical simulations (arXiv:1312.2213).

A thin Python layer over the C ABI in ``include/muca.h``: the functions below
carry the same names and only marshal arguments; every step of the method runs
in the CUDA library ``libmuca.so``.  PyTorch is used only to hand over CUDA
streams (``muca_set_stream``) and, optionally, a device arena (``Muca(...,
arena="torch")``).
"""
from __future__ import annotations

import ctypes

import numpy as np

from ._native import MucaError, check, library_path, load

ISING2D, POTTS2D, ISING2D_MUMA, POLYMER3D = 0, 1, 2, 3
SYSTEM_NAMES = {ISING2D: "ising2d", POTTS2D: "potts2d", ISING2D_MUMA: "ising2d_muma", POLYMER3D: "polymer3d"}

__all__ = ["Muca", "MucaError", "ISING2D", "POTTS2D", "ISING2D_MUMA", "POLYMER3D", "library_path", "load",
           "muca_init", "muca_init_ex", "muca_workspace_size", "muca_set_param", "muca_set_stream",
           "muca_iterate", "muca_merge_and_update", "muca_num_bins", "muca_get_lnW", "muca_get_lnW_sampled",
           "muca_get_histogram", "muca_get_flatness", "muca_get_reweight", "muca_get_observables", "muca_get_metrics",
           "muca_merge_open", "muca_update_with",
           "muca_get_state", "muca_set_state",
           "muca_get_spins", "muca_get_walker_bins", "muca_get_thresholds", "muca_get_sweep_counter",
           "muca_synchronize", "muca_free", "muca_last_error", "muca_det_math",
           "muca_iterate_noalloc", "muca_set_lnW", "muca_poly_trace", "POLY_TRACE_DTYPE", "muca_get_coords", "muca_get_drift", "muca_batch_create", "muca_batch_run", "muca_batch_free", "muca_batch_set_form", "muca_batch_set_sweeps", "Batch"]


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


# ---- one-to-one wrappers of the C ABI --------------------------------------------------------
def muca_last_error() -> str:
    return (load().muca_last_error() or b"").decode(errors="replace")


def muca_init(system: int, L_or_N: int, q: int, p: int, seed: int):
    h = ctypes.c_void_p()
    check(load().muca_init(ctypes.byref(h), system, L_or_N, q, p, seed), "muca_init")
    return h


def muca_workspace_size(system: int, L_or_N: int, q: int, p: int) -> int:
    n = ctypes.c_size_t()
    check(load().muca_workspace_size(system, L_or_N, q, p, ctypes.byref(n)), "muca_workspace_size")
    return n.value


def muca_init_ex(system: int, L_or_N: int, q: int, p: int, seed: int, device_arena: int, arena_bytes: int):
    h = ctypes.c_void_p()
    check(load().muca_init_ex(ctypes.byref(h), system, L_or_N, q, p, seed, ctypes.c_void_p(device_arena),
                              arena_bytes), "muca_init_ex")
    return h


def muca_set_param(h, key: str, value: float):
    check(load().muca_set_param(h, key.encode(), float(value)), "muca_set_param(%s)" % key)


def muca_set_stream(h, stream: int):
    check(load().muca_set_stream(h, ctypes.c_void_p(stream)), "muca_set_stream")


def muca_iterate(h, sweeps: int):
    check(load().muca_iterate(h, sweeps), "muca_iterate")


def muca_merge_and_update(h, want_flat: bool = False):
    if want_flat:
        f = ctypes.c_int()
        check(load().muca_merge_and_update(h, ctypes.byref(f)), "muca_merge_and_update")
        return bool(f.value)
    check(load().muca_merge_and_update(h, None), "muca_merge_and_update")
    return None


def muca_num_bins(h) -> int:
    n = ctypes.c_int()
    check(load().muca_num_bins(h, ctypes.byref(n)), "muca_num_bins")
    return n.value


def muca_set_lnW(h, lnW: np.ndarray):
    lnW = np.ascontiguousarray(lnW, dtype=np.float64)
    check(load().muca_set_lnW(h, _p(lnW), lnW.size), "muca_set_lnW")


def muca_poly_trace(h, dev_ptr: int, n_records: int):
    check(load().muca_poly_trace(h, ctypes.c_void_p(dev_ptr), int(n_records)), "muca_poly_trace")


# One record of muca_poly_trace (32 bytes).
POLY_TRACE_DTYPE = np.dtype([("dq", "<i8"), ("E", "<i8"), ("bn", "<i4"), ("b", "<i4"), ("flags", "<i4"),
                             ("pad", "<i4")])


def muca_get_lnW(h, out: np.ndarray):
    check(load().muca_get_lnW(h, _p(out), out.size), "muca_get_lnW")


def muca_get_lnW_sampled(h, out: np.ndarray):
    check(load().muca_get_lnW_sampled(h, _p(out), out.size), "muca_get_lnW_sampled")


def muca_get_histogram(h, out: np.ndarray):
    check(load().muca_get_histogram(h, _p(out), out.size), "muca_get_histogram")


def muca_get_flatness(h, out: np.ndarray):
    check(load().muca_get_flatness(h, _p(out)), "muca_get_flatness")


def muca_merge_open(h, dev_ptr: int):
    check(load().muca_merge_open(h, ctypes.c_void_p(dev_ptr)), "muca_merge_open")


def muca_update_with(h, dev_ptr: int, want_flat: bool = False):
    flat = ctypes.c_int(0)
    check(load().muca_update_with(h, ctypes.c_void_p(dev_ptr), ctypes.byref(flat) if want_flat else None),
          "muca_update_with")
    return bool(flat.value) if want_flat else None


def muca_get_observables(h, beta: float, out: np.ndarray, sums: np.ndarray | None = None):
    n = 0 if sums is None else sums.size // 3
    check(load().muca_get_observables(h, float(beta), _p(out), None if sums is None else _p(sums), n),
          "muca_get_observables")


def muca_get_metrics(h, out: np.ndarray):
    check(load().muca_get_metrics(h, _p(out)), "muca_get_metrics")


def muca_get_reweight(h, beta: float, out: np.ndarray, lnP: np.ndarray | None = None):
    check(load().muca_get_reweight(h, float(beta), _p(out), None if lnP is None else _p(lnP)), "muca_get_reweight")


def muca_get_state(h, buf: np.ndarray | None = None) -> int:
    n = ctypes.c_size_t(0 if buf is None else buf.nbytes)
    check(load().muca_get_state(h, None if buf is None else _p(buf), ctypes.byref(n)), "muca_get_state")
    return n.value


def muca_set_state(h, buf: np.ndarray):
    check(load().muca_set_state(h, _p(buf), buf.nbytes), "muca_set_state")


def muca_get_spins(h, out: np.ndarray):
    check(load().muca_get_spins(h, _p(out), out.size), "muca_get_spins")


def muca_get_walker_bins(h, out: np.ndarray):
    check(load().muca_get_walker_bins(h, _p(out), out.size), "muca_get_walker_bins")


def muca_get_thresholds(h, out: np.ndarray):
    check(load().muca_get_thresholds(h, _p(out), out.size), "muca_get_thresholds")


def muca_get_sweep_counter(h) -> int:
    v = ctypes.c_int64()
    check(load().muca_get_sweep_counter(h, ctypes.byref(v)), "muca_get_sweep_counter")
    return v.value


def muca_get_coords(h, coords: np.ndarray, energies: np.ndarray | None = None):
    check(load().muca_get_coords(h, _p(coords), coords.size, None if energies is None else _p(energies),
                                 0 if energies is None else energies.size), "muca_get_coords")


def muca_get_drift(h) -> float:
    v = ctypes.c_double()
    check(load().muca_get_drift(h, ctypes.byref(v)), "muca_get_drift")
    return v.value


def muca_det_math(fn: int, x: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.zeros_like(x)
    check(load().muca_det_math(fn, _p(x), _p(out), x.size), "muca_det_math")
    return out


def muca_iterate_noalloc(h, sweeps: int, dev_H_out: int):
    """Sweeps + merge into a caller-provided device buffer, with no device allocation
    (partial histograms in the library's static device array; see include/muca.h)."""
    check(load().muca_iterate_noalloc(h, sweeps, ctypes.c_void_p(dev_H_out)), "muca_iterate_noalloc")


def muca_batch_create(handles):
    arr = (ctypes.c_void_p * len(handles))(*[h.value if isinstance(h, ctypes.c_void_p) else h for h in handles])
    b = ctypes.c_void_p()
    check(load().muca_batch_create(arr, len(handles), ctypes.byref(b)), "muca_batch_create")
    return b


def muca_batch_run(b, n_iter: int, sweeps: int, use_graph: bool = True):
    check(load().muca_batch_run(b, n_iter, sweeps, 1 if use_graph else 0), "muca_batch_run")


def muca_batch_set_form(b, form: int):
    check(load().muca_batch_set_form(b, int(form)), "muca_batch_set_form")


def muca_batch_set_sweeps(b, sweeps):
    """Per-system sweeps of every batch iteration, or None for the run's argument."""
    if sweeps is None:
        check(load().muca_batch_set_sweeps(b, None, 0), "muca_batch_set_sweeps")
        return
    arr = np.ascontiguousarray(sweeps, dtype=np.int64)
    check(load().muca_batch_set_sweeps(b, _p(arr), arr.size), "muca_batch_set_sweeps")


def muca_batch_free(b):
    check(load().muca_batch_free(b), "muca_batch_free")


class Batch:
    """Several Muca systems advanced together: per iteration every system's own sweep kernel on a
    stream of its own, side by side (form 1, default), or one persistent sweep launch over all
    systems (form 0); then batched merge, recursion and thresholds; optionally the whole run as
    one CUDA graph."""

    def __init__(self, systems, form: int = 1):
        self.systems = list(systems)
        self.h = muca_batch_create([s.h for s in self.systems])
        if form != 1:
            self.set_form(form)

    def set_form(self, form: int):
        muca_batch_set_form(self.h, form)

    def set_sweeps(self, sweeps):
        """Each system's own sweeps an iteration (e.g. its M_opt, Eq. 4), or None."""
        muca_batch_set_sweeps(self.h, sweeps)

    def run(self, n_iter: int, sweeps: int, use_graph: bool = True):
        muca_batch_run(self.h, n_iter, sweeps, use_graph)

    def close(self):
        if getattr(self, "h", None) is not None:
            muca_batch_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def muca_synchronize(h):
    check(load().muca_synchronize(h), "muca_synchronize")


def muca_free(h):
    check(load().muca_free(h), "muca_free")


# ---- convenience object -----------------------------------------------------------------------
class Muca:
    """One system of p walkers on the current CUDA device (owns a muca_ctx)."""

    def __init__(self, system: int, L: int, q: int = 2, p: int = 64, seed: int = 1, *, beta: float | None = None,
                 record: int = 0, block: int | None = None, walker_offset: int = 0, stream=None,
                 arena: str | None = None, window: tuple | None = None):
        self.system, self.L, self.q, self.p, self.seed = system, L, q, p, seed
        self._arena = None
        if arena == "torch":
            import torch

            nbytes = muca_workspace_size(system, L, q, p)
            self._arena = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
            ptr = (self._arena.data_ptr() + 255) // 256 * 256
            self.h = muca_init_ex(system, L, q, p, seed, ptr, nbytes)
        else:
            self.h = muca_init(system, L, q, p, seed)
        self.N = L if system == POLYMER3D else L * L
        self.C = {ISING2D: 5, POTTS2D: 9, ISING2D_MUMA: 10}.get(system, 0)
        if stream is not None:
            muca_set_stream(self.h, int(getattr(stream, "cuda_stream", stream)))
        self.beta = beta
        if beta is not None:
            muca_set_param(self.h, "beta", beta)
        if record:
            muca_set_param(self.h, "record", record)
        if block is not None:
            muca_set_param(self.h, "block", block)
        if walker_offset:
            muca_set_param(self.h, "walker_offset", walker_offset)
        # the polymer's energy window (the library's default is [2N, 6N))
        self.window = window if window is not None or system != POLYMER3D else (2.0 * L, 6.0 * L)
        if window is not None:
            muca_set_param(self.h, "e_lo", window[0])
            muca_set_param(self.h, "e_hi", window[1])
        self.B = muca_num_bins(self.h)

    def close(self):
        if getattr(self, "h", None) is not None:
            muca_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_param(self, key: str, value: float):
        muca_set_param(self.h, key, value)
        if key in ("e_lo", "e_hi", "bin_width"):  # the polymer's bin count follows the window
            self.B = muca_num_bins(self.h)
            if key != "bin_width" and self.window is not None:
                lo, hi = self.window
                self.window = (float(value), hi) if key == "e_lo" else (lo, float(value))

    def set_stream(self, stream):
        muca_set_stream(self.h, int(getattr(stream, "cuda_stream", stream)))

    def iterate(self, sweeps: int):
        muca_iterate(self.h, sweeps)

    def merge_and_update(self, want_flat: bool = False):
        return muca_merge_and_update(self.h, want_flat)

    def merge_open(self, dev_buf):
        """Sum the open histogram into a device tensor of B int64 and clear it (sharded runs);
        returns when the buffer holds the sum."""
        muca_merge_open(self.h, dev_buf.data_ptr())
        muca_synchronize(self.h)

    def update_with(self, dev_buf, want_flat: bool = False):
        """Close the iteration with a summed histogram held in a device tensor (sharded runs)."""
        return muca_update_with(self.h, dev_buf.data_ptr(), want_flat)

    def set_lnW(self, lnW: np.ndarray):
        muca_set_lnW(self.h, lnW)

    def iterate_traced(self, sweeps: int, walkers=None) -> np.ndarray:
        """Polymer: run `sweeps` sweeps and return the record of every attempt, shape
        (p, sweeps, N), dtype POLY_TRACE_DTYPE (muca_poly_trace); with `walkers` (indices) only
        their records are copied back, shape (len(walkers), sweeps, N)."""
        import torch

        n = self.p * sweeps * self.N
        buf = torch.empty(n * POLY_TRACE_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
        muca_poly_trace(self.h, buf.data_ptr(), n)
        muca_iterate(self.h, sweeps)
        muca_synchronize(self.h)
        rows = buf.view(self.p, -1)
        if walkers is not None:
            rows = rows[torch.as_tensor(np.asarray(walkers), device="cuda")]
        k = rows.shape[0]
        return rows.cpu().numpy().reshape(-1).view(POLY_TRACE_DTYPE).reshape(k, sweeps, self.N)

    def lnW(self) -> np.ndarray:
        a = np.zeros(self.B, dtype=np.float64)
        muca_get_lnW(self.h, a)
        return a

    def lnW_sampled(self) -> np.ndarray:
        a = np.zeros(self.B, dtype=np.float64)
        muca_get_lnW_sampled(self.h, a)
        return a

    def histogram(self) -> np.ndarray:
        a = np.zeros(self.B, dtype=np.uint64)
        muca_get_histogram(self.h, a)
        return a

    def flatness(self) -> np.ndarray:
        a = np.zeros(3, dtype=np.float64)
        muca_get_flatness(self.h, a)
        return a

    def reweight(self, beta: float):
        out = np.zeros(4, dtype=np.float64)
        lnP = np.zeros(self.B, dtype=np.float64)
        muca_get_reweight(self.h, beta, out, lnP)
        return out, lnP

    def observables(self, beta: float):
        """Eq. (2) for |M| and M^2 (Ising with observables on): ({<|M|>/N, <M^2>/N^2, chi per
        site}, per-bin sums of shape (B, 3))."""
        out = np.zeros(3, dtype=np.float64)
        sums = np.zeros(3 * self.B, dtype=np.uint64)
        muca_get_observables(self.h, beta, out, sums)
        return out, sums.reshape(self.B, 3)

    def metrics(self) -> dict:
        """Counts of the last closed iteration and of all closed iterations: accepted moves,
        tunnelling events (arrivals at one end of the reachable bins after the other end, the bin
        sampled at every sweep's end), the iteration's sweeps and its acceptance rate."""
        a = np.zeros(6, dtype=np.uint64)
        muca_get_metrics(self.h, a)
        acc, ev, acc_t, ev_t, sw, it = (int(x) for x in a)
        attempts = self.p * self.N * sw
        return {"iteration": it, "accepted": acc, "tunnelling_events": ev, "sweeps": sw,
                "acceptance_rate": acc / attempts if attempts else float("nan"),
                "accepted_total": acc_t, "tunnelling_events_total": ev_t}

    def spins(self) -> np.ndarray:
        a = np.zeros(self.p * self.N, dtype=np.int8)
        muca_get_spins(self.h, a)
        return a.reshape(self.p, self.L, self.L)

    def bins(self) -> np.ndarray:
        a = np.zeros(self.p, dtype=np.int32)
        muca_get_walker_bins(self.h, a)
        return a

    def thresholds(self) -> np.ndarray:
        a = np.zeros(self.B * self.C, dtype=np.uint32)
        muca_get_thresholds(self.h, a)
        return a.reshape(self.B, self.C)

    def sweep_counter(self) -> int:
        return muca_get_sweep_counter(self.h)

    def coords(self) -> np.ndarray:
        c = np.zeros(self.p * self.N * 3, dtype=np.float64)
        muca_get_coords(self.h, c)
        return c.reshape(self.p, self.N, 3)

    def energies(self) -> np.ndarray:
        c = np.zeros(self.p * self.N * 3, dtype=np.float64)
        e = np.zeros(self.p, dtype=np.float64)
        muca_get_coords(self.h, c, e)
        return e

    def drift(self) -> float:
        return muca_get_drift(self.h)

    def get_state(self) -> np.ndarray:
        n = muca_get_state(self.h, None)
        buf = np.zeros(n, dtype=np.uint8)
        muca_get_state(self.h, buf)
        return buf

    def set_state(self, buf: np.ndarray):
        muca_set_state(self.h, np.ascontiguousarray(buf, dtype=np.uint8))

    def synchronize(self):
        muca_synchronize(self.h)
