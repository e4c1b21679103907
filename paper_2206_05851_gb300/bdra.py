"""Python binding of the C ABI in include/bdra.h (argument marshalling only).

Every function here has the name of the C entry point it calls and does no
arithmetic of the method: it converts numpy arrays / torch tensors into
pointers, checks sizes and raises on a non-OK status. All work runs in the
CUDA library libbdra.so; importing this module fails if that library has not
been built (there is no CPU fallback).

Arrays may live on the host (numpy, CPU tensors) or on the current CUDA
device (torch tensors); the library detects which. PyTorch serves only for
device memory and streams.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbdra.so")

BD_OK, BD_E_INVALID, BD_E_CUDA, BD_E_OOM, BD_E_STATE, BD_E_TIMEOUT, BD_E_CAPACITY = range(7)
BD_PREC_FP64, BD_PREC_FP32 = 0, 1
BD_CRIT_ISF, BD_CRIT_TSF, BD_CRIT_RSF = 1, 2, 4
BD_FLAG_IDENTICAL_NOISE = 1
BD_FLAG_CONFORMATION = 2
BD_FLAG_TEST_TC_STALL = 4


class BdError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_status_name(status)}: {message}")
        self.status = status


class bd_chain_desc(ctypes.Structure):
    _fields_ = [("n_beads", ctypes.c_int32), ("n_replicas", ctypes.c_int32),
                ("spring", ctypes.c_int32), ("flow", ctypes.c_int32),
                ("H", ctypes.c_double), ("b", ctypes.c_double), ("rate", ctypes.c_double),
                ("f_c", ctypes.c_double), ("k0", ctypes.c_double), ("dx", ctypes.c_double),
                ("r0", ctypes.c_double), ("lj_u", ctypes.c_double), ("lj_sigma", ctypes.c_double),
                ("hi_a", ctypes.c_double), ("vwf_fa", ctypes.c_double), ("vwf_fb", ctypes.c_double),
                ("vwf_xmax", ctypes.c_double)]


class bd_config(ctypes.Structure):
    _fields_ = [("n_chains", ctypes.c_int32), ("window_steps", ctypes.c_int32),
                ("chains", ctypes.POINTER(bd_chain_desc)), ("dt", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("precision", ctypes.c_int32),
                ("flags", ctypes.c_int32), ("thr_mask", ctypes.c_int32),
                ("bell_mask", ctypes.c_int32), ("max_windows", ctypes.c_int64),
                ("s_min", ctypes.c_double), ("stream", ctypes.c_void_p),
                ("lanes_hint", ctypes.c_int32), ("layout_hint", ctypes.c_int32),
                ("checkpoint_steps", ctypes.c_int32), ("chain_id_base", ctypes.c_int32)]


class bd_event(ctypes.Structure):
    _fields_ = [("chain", ctypes.c_int32), ("spring", ctypes.c_int32),
                ("criterion", ctypes.c_int32), ("kind", ctypes.c_int32),
                ("step", ctypes.c_int64)]


class bd_info(ctypes.Structure):
    _fields_ = [("n_springs", ctypes.c_int64), ("step", ctypes.c_int64),
                ("windows_done", ctypes.c_int64), ("overextensions", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("kernel_launches", ctypes.c_int64),
                ("n_launch_classes", ctypes.c_int32),
                ("precision", ctypes.c_int32)]


EVENT_DTYPE = np.dtype([("chain", np.int32), ("spring", np.int32), ("criterion", np.int32),
                        ("kind", np.int32), ("step", np.int64)])

_lib = None


def load() -> ctypes.CDLL:
    """Load libbdra.so (raises if it was not built: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(LIB_PATH)
    P, vp = ctypes.POINTER, ctypes.c_void_p
    st = ctypes.c_int
    sig = {
        "bd_create": ([P(bd_config), vp, P(vp)], st),
        "bd_spawn_replicas": ([vp], st),
        "bd_step": ([vp, ctypes.c_int64], st),
        "bd_replica_average": ([vp, ctypes.c_int64, vp], st),
        "bd_time_average": ([vp, ctypes.c_int64, vp], st),
        "bd_conformation": ([vp, ctypes.c_int64, vp, vp, vp], st),
        "bd_detect_events": ([vp, vp, ctypes.c_int64, P(ctypes.c_int64), vp], st),
        "bd_get_kinetics": ([vp, vp, vp, vp], st),
        "bd_get_positions": ([vp, ctypes.c_int32, vp, P(ctypes.c_int64)], st),
        "bd_set_positions": ([vp, vp, ctypes.c_int64], st),
        "bd_get_info": ([vp, P(bd_info)], st),
        "bd_autotune": ([vp, ctypes.c_int32, ctypes.c_int32], st),
        "bd_get_plan": ([vp, vp, vp, vp], st),
        "bd_enable_timing": ([vp, ctypes.c_int32], st),
        "bd_kernel_times": ([vp, P(ctypes.c_double), P(ctypes.c_int64)], st),
        "bd_adjoint": ([vp, vp, vp, vp], st),
        "bd_probe_philox_rounds": ([vp, P(ctypes.c_double)], st),
        "bd_probe_fp32_fma": ([vp, P(ctypes.c_double)], st),
        "bd_probe_fp64_fma": ([vp, P(ctypes.c_double)], st),
        "bd_probe_mufu": ([vp, P(ctypes.c_double)], st),
        "bd_probe_issue": ([vp, P(ctypes.c_double)], st),
        "bd_probe_int_alu": ([vp, P(ctypes.c_double)], st),
        "bd_philox_normals": ([ctypes.c_uint64, ctypes.c_int64, vp, ctypes.c_int32, vp, vp], st),
        "bd_compact_events_noalloc": ([vp, vp, ctypes.c_int64, vp, ctypes.c_int32, vp,
                                       ctypes.c_int64, vp, vp], st),
        "bd_last_error": ([vp], ctypes.c_char_p),
        "bd_status_string": ([ctypes.c_int], ctypes.c_char_p),
        "bd_destroy": ([vp], None),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _status_name(s: int) -> str:
    try:
        return load().bd_status_string(s).decode()
    except Exception:
        return f"status {s}"


def _check(status: int, ctx=None) -> None:
    if status != BD_OK:
        msg = load().bd_last_error(ctx).decode() if ctx else ""
        raise BdError(status, msg)


def _ptr(a) -> Tuple[int, int]:
    """(address, nbytes) of a contiguous numpy array or torch tensor."""
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data, a.nbytes
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr(), a.numel() * a.element_size()
    raise TypeError(f"unsupported array type {type(a)}")


def _need(a, nbytes: int, what: str) -> int:
    p, n = _ptr(a)
    if n < nbytes:
        raise ValueError(f"{what}: buffer of {n} bytes, needs {nbytes}")
    return p


def make_config(chains: Sequence, dt: float, window_steps: int, seed: int, precision: int,
                max_windows: int, thr_mask: int = 0, bell_mask: int = 0, flags: int = 0,
                s_min: float = 1e-3, stream: Optional[int] = None,
                lanes_hint: int = 0, layout_hint: int = 0,
                checkpoint_steps: int = 0, chain_id_base: int = 0) -> Tuple[bd_config, ctypes.Array]:
    """Build a bd_config (and the chain array it points to) from chain records
    with the fields of bd_chain_desc."""
    arr = (bd_chain_desc * len(chains))(*[
        bd_chain_desc(int(c.n_beads), int(c.n_replicas), int(c.spring), int(c.flow),
                      float(c.H), float(c.b), float(c.rate), float(c.f_c), float(c.k0),
                      float(c.dx), float(getattr(c, "r0", 0.0)), float(getattr(c, "lj_u", 0.0)),
                      float(getattr(c, "lj_sigma", 0.0)), float(getattr(c, "hi_a", 0.0)),
                      float(getattr(c, "vwf_fa", 0.0)), float(getattr(c, "vwf_fb", 0.0)),
                      float(getattr(c, "vwf_xmax", 0.0)))
              for c in chains])
    cfg = bd_config(len(chains), int(window_steps), arr, float(dt), int(seed), int(precision),
                    int(flags), int(thr_mask), int(bell_mask), int(max_windows), float(s_min),
                    stream, int(lanes_hint), int(layout_hint), int(checkpoint_steps),
                    int(chain_id_base))
    return cfg, arr


def bd_create(cfg: bd_config, init_pos) -> int:
    lib = load()
    n_beads = sum(cfg.chains[i].n_beads for i in range(cfg.n_chains))
    p = _need(init_pos, 24 * n_beads, "init_pos")
    out = ctypes.c_void_p()
    _check(lib.bd_create(ctypes.byref(cfg), p, ctypes.byref(out)))
    return out.value


def bd_destroy(ctx: int) -> None:
    load().bd_destroy(ctx)


def bd_spawn_replicas(ctx: int) -> None:
    _check(load().bd_spawn_replicas(ctx), ctx)


def bd_step(ctx: int, n_steps: int) -> None:
    _check(load().bd_step(ctx, int(n_steps)), ctx)


def bd_get_info(ctx: int) -> bd_info:
    info = bd_info()
    _check(load().bd_get_info(ctx, ctypes.byref(info)), ctx)
    return info


def bd_replica_average(ctx: int, window: int, out) -> None:
    M = bd_get_info(ctx).n_springs
    _check(load().bd_replica_average(ctx, int(window), _need(out, 8 * M, "out")), ctx)


def bd_time_average(ctx: int, window: int, out) -> None:
    M = bd_get_info(ctx).n_springs
    _check(load().bd_time_average(ctx, int(window), _need(out, 8 * M, "out")), ctx)


def bd_conformation(ctx: int, window: int, dbar=None, dbead=None, rgz=None) -> None:
    """Eq. 5 diagnostics of a completed window into the given arrays (any may
    be None): dbar [sum R][3], dbead [sum N][3], rgz [n_chains] float64."""
    args = [_ptr(a)[0] if a is not None else None for a in (dbar, dbead, rgz)]
    _check(load().bd_conformation(ctx, int(window), *args), ctx)


def bd_detect_events(ctx: int, out, capacity: int, log_surv=None) -> int:
    """Returns the number of events (raises BdError BD_E_CAPACITY if > capacity)."""
    n = ctypes.c_int64(0)
    po = _need(out, 24 * capacity, "out") if capacity > 0 else None
    pl = _ptr(log_surv)[0] if log_surv is not None else None
    _check(load().bd_detect_events(ctx, po, int(capacity), ctypes.byref(n), pl), ctx)
    return int(n.value)


def bd_get_kinetics(ctx: int, hazard=None, first_thr=None, first_bell=None) -> None:
    M = bd_get_info(ctx).n_springs
    args = [_need(a, 24 * M, name) if a is not None else None
            for a, name in ((hazard, "hazard"), (first_thr, "first_thr"),
                            (first_bell, "first_bell"))]
    _check(load().bd_get_kinetics(ctx, *args), ctx)


def bd_get_positions(ctx: int, all_slots: bool, out) -> int:
    step = ctypes.c_int64(0)
    _check(load().bd_get_positions(ctx, int(bool(all_slots)), _ptr(out)[0], ctypes.byref(step)),
           ctx)
    return int(step.value)


def bd_set_positions(ctx: int, pos, step: int = 0) -> None:
    _check(load().bd_set_positions(ctx, _ptr(pos)[0], int(step)), ctx)


def bd_autotune(ctx: int, probe_steps: int = 32, force: bool = False) -> None:
    _check(load().bd_autotune(ctx, int(probe_steps), int(bool(force))), ctx)


def bd_get_plan(ctx: int, n_chains: int, precision: int = BD_PREC_FP32):
    """(variant per chain, groups per chain, {variant: cost ns per warp-step})."""
    v = np.zeros(n_chains, dtype=np.int32)
    g = np.zeros(n_chains, dtype=np.int32)
    names = ([2, 4, 7, 10, 13, 16, 202, 204, 205, 207, 216] if precision == BD_PREC_FP64
             else [4, 7, 10, 13, 16, 104, 107, 202, 204, 205, 207, 216,
                   5, 6, 8, 9, 11, 12, 14, 15, 105, 106])
    c = np.zeros(len(names))
    _check(load().bd_get_plan(ctx, v.ctypes.data, g.ctypes.data, c.ctypes.data), ctx)
    return v, g, dict(zip(names, c.tolist()))


def bd_enable_timing(ctx: int, enable: bool) -> None:
    _check(load().bd_enable_timing(ctx, int(bool(enable))), ctx)


def bd_kernel_times(ctx: int):
    """((parent_ms, replica_ms), (parent_launches, replica_launches)) since last call."""
    ms = (ctypes.c_double * 2)()
    n = (ctypes.c_int64 * 2)()
    _check(load().bd_kernel_times(ctx, ms, n), ctx)
    return (ms[0], ms[1]), (n[0], n[1])


def bd_adjoint(ctx: int, n_chains: int, M: int, windows: int, grad_rsf=None,
               grad_log_surv=None, out=None):
    """dL/d(rate, b, H) per chain, [n_chains][3] float64, for
    L = sum grad_rsf * RSF + sum grad_log_surv * log S (RSF-criterion Bell
    log-survival). grad_rsf [windows][M], grad_log_surv [n_chains]: host or
    device arrays, or None."""
    out = np.zeros((n_chains, 3)) if out is None else out
    g = _need(grad_rsf, 8 * windows * M, "grad_rsf") if grad_rsf is not None else None
    l = _need(grad_log_surv, 8 * n_chains, "grad_log_surv") if grad_log_surv is not None else None
    _check(load().bd_adjoint(ctx, g, l, _need(out, 24 * n_chains, "grad_params")), ctx)
    return out


def bd_probe_philox_rounds(stream: Optional[int] = None) -> float:
    """Measured Philox4x32 rounds per second of the current device."""
    r = ctypes.c_double(0.0)
    _check(load().bd_probe_philox_rounds(stream, ctypes.byref(r)))
    return r.value


def bd_probe_fp32_fma(stream: Optional[int] = None) -> float:
    """Measured float32 FMA throughput of the current device, FLOP/s."""
    r = ctypes.c_double(0.0)
    _check(load().bd_probe_fp32_fma(stream, ctypes.byref(r)))
    return r.value


def bd_probe_fp64_fma(stream: Optional[int] = None) -> float:
    """Measured float64 FMA throughput of the current device, FLOP/s."""
    r = ctypes.c_double(0.0)
    _check(load().bd_probe_fp64_fma(stream, ctypes.byref(r)))
    return r.value


def bd_probe_mufu(stream: Optional[int] = None) -> float:
    """Measured special-function (approximate rsqrt) throughput, ops/s."""
    r = ctypes.c_double(0.0)
    _check(load().bd_probe_mufu(stream, ctypes.byref(r)))
    return r.value


def bd_probe_issue(stream: Optional[int] = None) -> float:
    """Measured instruction-issue rate (mixed float32 / integer stream) of the
    current device, thread-instructions per second."""
    r = ctypes.c_double(0.0)
    _check(load().bd_probe_issue(stream, ctypes.byref(r)))
    return r.value


def bd_probe_int_alu(stream: Optional[int] = None) -> float:
    """Measured integer-ALU (three-input logic) throughput, ops/s."""
    r = ctypes.c_double(0.0)
    _check(load().bd_probe_int_alu(stream, ctypes.byref(r)))
    return r.value


NOALLOC_MAX_SPRINGS = 1 << 20


def bd_compact_events_noalloc(first_thr, first_bell, n_springs: int, spring_offsets,
                              n_chains: int, out, capacity: int, n_out,
                              stream: Optional[int] = None) -> None:
    """Allocation-free event compaction; every array is device memory."""
    _check(load().bd_compact_events_noalloc(
        _ptr(first_thr)[0], _ptr(first_bell)[0], int(n_springs), _ptr(spring_offsets)[0],
        int(n_chains), _ptr(out)[0] if capacity > 0 else None, int(capacity), _ptr(n_out)[0],
        stream))


def bd_philox_normals(seed: int, ctr, precision: int, out, stream: Optional[int] = None) -> None:
    p, nb = _ptr(ctr)
    n = nb // 16
    _check(load().bd_philox_normals(int(seed), n, p, int(precision), _need(out, 24 * n, "out"),
                                    stream))


# ---------------------------------------------------------------------------
# Convenience wrapper (still marshalling only)
# ---------------------------------------------------------------------------

class Context:
    """Owns one bd_ctx; methods forward to the C entry points."""

    def __init__(self, chains: Sequence, dt: float, window_steps: int, seed: int,
                 init_pos, precision: int = BD_PREC_FP32, max_windows: int = 1024,
                 thr_mask: int = 0, bell_mask: int = 0, flags: int = 0,
                 s_min: float = 1e-3, stream: Optional[int] = None, lanes_hint: int = 0,
                 layout_hint: int = 0, checkpoint_steps: int = 0, chain_id_base: int = 0):
        self.chains = list(chains)
        self.cfg, self._arr = make_config(self.chains, dt, window_steps, seed, precision,
                                          max_windows, thr_mask, bell_mask, flags, s_min,
                                          stream, lanes_hint, layout_hint, checkpoint_steps,
                                          chain_id_base)
        self.ptr = bd_create(self.cfg, init_pos)
        self.M = sum(c.n_beads - 1 for c in self.chains)
        self.n_beads = sum(c.n_beads for c in self.chains)
        self.n_slot_beads = sum(c.n_beads * (c.n_replicas + 1) for c in self.chains)

    def close(self) -> None:
        if self.ptr:
            bd_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n: int) -> None:
        bd_step(self.ptr, n)

    def spawn(self) -> None:
        bd_spawn_replicas(self.ptr)

    def info(self) -> bd_info:
        return bd_get_info(self.ptr)

    def replica_average(self, window: int, out=None) -> np.ndarray:
        out = np.zeros(self.M) if out is None else out
        bd_replica_average(self.ptr, window, out)
        return out

    def time_average(self, window: int, out=None) -> np.ndarray:
        out = np.zeros(self.M) if out is None else out
        bd_time_average(self.ptr, window, out)
        return out

    def positions(self, all_slots: bool = False) -> np.ndarray:
        n = self.n_slot_beads if all_slots else self.n_beads
        out = np.zeros((n, 3))
        bd_get_positions(self.ptr, all_slots, out)
        return out

    def set_positions(self, pos, step: int = 0) -> None:
        bd_set_positions(self.ptr, pos, step)

    def autotune(self, probe_steps: int = 32, force: bool = False) -> None:
        bd_autotune(self.ptr, probe_steps, force)

    def plan(self):
        return bd_get_plan(self.ptr, len(self.chains), self.cfg.precision)

    def conformation(self, window: int):
        """(dbar [sum R][3], dbead [sum N][3], rgz [n_chains]) of a completed
        window (needs BD_FLAG_CONFORMATION)."""
        dbar = np.zeros((sum(c.n_replicas for c in self.chains), 3))
        dbead = np.zeros((self.n_beads, 3))
        rgz = np.zeros(len(self.chains))
        bd_conformation(self.ptr, window, dbar, dbead, rgz)
        return dbar, dbead, rgz

    def kinetics(self):
        haz = np.zeros((3, self.M))
        ft = np.zeros((3, self.M), dtype=np.int64)
        fb = np.zeros((3, self.M), dtype=np.int64)
        bd_get_kinetics(self.ptr, haz, ft, fb)
        return haz, ft, fb

    def adjoint(self, grad_rsf=None, grad_log_surv=None, out=None):
        """Gradient [n_chains][3] of sum grad_rsf * RSF + sum grad_log_surv *
        log S with respect to (rate, b, H); see bd_adjoint."""
        windows = self.info().windows_done
        return bd_adjoint(self.ptr, len(self.chains), self.M, windows, grad_rsf,
                          grad_log_surv, out)

    def events(self, capacity: int = 1 << 16):
        out = np.zeros(capacity, dtype=EVENT_DTYPE)
        ls = np.zeros((len(self.chains), 3))
        n = bd_detect_events(self.ptr, out, capacity, ls)
        return out[:n], ls
