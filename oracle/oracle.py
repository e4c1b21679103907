"""ctypes loader for the CPU FP64 oracle (bd_oracle.c).

TEST INFRASTRUCTURE ONLY. Only the test-suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this module. The product
library never imports it, and the two share no code. Inputs come from
``paper_2206_05851_gb300.inputs`` (seeded generators with none of the
method's arithmetic); everything the oracle computes is its own.

Every oracle function is pinned in ``tests/test_oracle_*.py`` against values
the physics and the paper fix, and Philox against an independent
implementation (the CUDA toolkit's host-side generator);
``tests/test_oracle_planted.py`` checks that the pins catch planted mistakes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Dict, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bd_oracle.c")
_LIB = os.path.join(_HERE, "libbdoracle.so")
# A prebuilt oracle library to load instead (the planted-mistake tests point
# this at copies of the oracle with one mistake compiled in).
_LIB_OVERRIDE = os.environ.get("BD_ORACLE_LIB")

ISF, TSF, RSF = 0, 1, 2
S_MIN_DEFAULT = 1e-3


def build(force: bool = False) -> str:
    """Compile bd_oracle.c with gcc (OpenMP over chains) into libbdoracle.so."""
    if _LIB_OVERRIDE:
        return _LIB_OVERRIDE
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "bd_oracle.h"))):
        tmp = f"{_LIB}.{os.getpid()}.tmp"      # then renamed: concurrent builds never see half a file
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Chain(ctypes.Structure):
    _fields_ = [("n_beads", ctypes.c_int32), ("n_replicas", ctypes.c_int32),
                ("spring", ctypes.c_int32), ("flow", ctypes.c_int32),
                ("H", ctypes.c_double), ("b", ctypes.c_double), ("rate", ctypes.c_double),
                ("f_c", ctypes.c_double), ("k0", ctypes.c_double), ("dx", ctypes.c_double),
                ("r0", ctypes.c_double), ("lj_u", ctypes.c_double), ("lj_sigma", ctypes.c_double),
                ("hi_a", ctypes.c_double), ("vwf_fa", ctypes.c_double), ("vwf_fb", ctypes.c_double),
                ("vwf_xmax", ctypes.c_double)]


class _Problem(ctypes.Structure):
    _fields_ = [("n_chains", ctypes.c_int32), ("window_steps", ctypes.c_int32),
                ("chains", ctypes.POINTER(_Chain)), ("dt", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("identical_noise", ctypes.c_int32),
                ("thr_mask", ctypes.c_int32), ("bell_mask", ctypes.c_int32),
                ("s_min", ctypes.c_double), ("chain_ids", ctypes.POINTER(ctypes.c_int32))]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.POINTER
        u32p, f64p, i64p = P(ctypes.c_uint32), P(ctypes.c_double), P(ctypes.c_int64)
        _lib.ora_philox4x32_10.argtypes = [u32p, u32p, u32p]
        _lib.ora_uniform.argtypes = [ctypes.c_uint32]
        _lib.ora_uniform.restype = ctypes.c_double
        _lib.ora_uniform21.argtypes = [ctypes.c_uint32]
        _lib.ora_uniform21.restype = ctypes.c_double
        _lib.ora_normals3.argtypes = [ctypes.c_uint64] + [ctypes.c_uint32] * 5 + [f64p]
        _lib.ora_exp1.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                  ctypes.c_uint32]
        _lib.ora_exp1.restype = ctypes.c_double
        _lib.ora_spring_force.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_double, f64p, f64p, f64p]
        _lib.ora_lj_forces.argtypes = [P(_Chain), f64p, f64p]
        _lib.ora_spring_force.restype = ctypes.c_int
        _lib.ora_flow_gradient.argtypes = [ctypes.c_int, ctypes.c_double, f64p]
        _lib.ora_em_step.argtypes = [P(_Chain), ctypes.c_double, ctypes.c_double, f64p, f64p]
        _lib.ora_em_step.restype = ctypes.c_int64
        _lib.ora_tensions.argtypes = [P(_Chain), ctypes.c_double, f64p, f64p]
        _lib.ora_run.argtypes = [P(_Problem), ctypes.c_int64, f64p, f64p, f64p, f64p, f64p,
                                 i64p, i64p, f64p, i64p, ctypes.c_int]
        _lib.ora_run.restype = ctypes.c_int
        _lib.ora_criteria_update.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                             P(_Chain), ctypes.c_double, ctypes.c_double,
                                             ctypes.c_int64, ctypes.c_double, f64p, i64p, i64p]
        _lib.ora_philox_many.argtypes = [ctypes.c_int64, u32p, u32p, u32p]
        _lib.ora_normals3_many.argtypes = [ctypes.c_uint64, ctypes.c_int64, u32p, f64p]
        _lib.ora_max_threads.restype = ctypes.c_int
        _lib.ora_rsf_tangent.argtypes = [P(_Problem), ctypes.c_int64, f64p, f64p, f64p, ctypes.c_int]
        _lib.ora_rsf_tangent.restype = ctypes.c_int
        _lib.ora_run_conformation.argtypes = [P(_Problem), ctypes.c_int64, f64p, f64p, f64p, f64p,
                                              ctypes.c_int]
        _lib.ora_run_conformation.restype = ctypes.c_int
        _lib.ora_rpy_block.argtypes = [ctypes.c_double, f64p, f64p]
        _lib.ora_rpy_matrix.argtypes = [ctypes.c_int, ctypes.c_double, f64p, f64p]
        _lib.ora_cholesky.argtypes = [ctypes.c_int, f64p, f64p]
        _lib.ora_cholesky.restype = ctypes.c_int
        _lib.ora_chain_spring_force.argtypes = [P(_Chain), ctypes.c_int, ctypes.c_double, f64p, f64p, f64p]
        _lib.ora_chain_spring_force.restype = ctypes.c_int
    return _lib


def _p(a: np.ndarray, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _chain_struct(ch) -> _Chain:
    return _Chain(int(ch.n_beads), int(ch.n_replicas), int(ch.spring), int(ch.flow),
                  float(ch.H), float(ch.b), float(ch.rate), float(ch.f_c), float(ch.k0),
                  float(ch.dx), float(getattr(ch, "r0", 0.0)), float(getattr(ch, "lj_u", 0.0)),
                  float(getattr(ch, "lj_sigma", 0.0)), float(getattr(ch, "hi_a", 0.0)),
                  float(getattr(ch, "vwf_fa", 0.0)), float(getattr(ch, "vwf_fb", 0.0)),
                  float(getattr(ch, "vwf_xmax", 0.0)))


# ---------------------------------------------------------------------------
# Generators
# ---------------------------------------------------------------------------

def philox(ctr: Sequence[int], key: Sequence[int]) -> np.ndarray:
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().ora_philox4x32_10(_p(c, ctypes.c_uint32), _p(k, ctypes.c_uint32),
                            _p(out, ctypes.c_uint32))
    return out


def philox_many(ctr: np.ndarray, key: Sequence[int]) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    k = np.asarray(key, dtype=np.uint32)
    out = np.zeros_like(c)
    lib().ora_philox_many(len(c), _p(c, ctypes.c_uint32), _p(k, ctypes.c_uint32),
                          _p(out, ctypes.c_uint32))
    return out


def uniform(x: int) -> float:
    return lib().ora_uniform(int(x))


def uniform21(m: int) -> float:
    return lib().ora_uniform21(int(m))


def normals3(seed: int, bead: int, slot: int, stream: int, step: int, chain: int) -> np.ndarray:
    xi = np.zeros(3)
    lib().ora_normals3(seed, bead, slot, stream, step, chain, _p(xi, ctypes.c_double))
    return xi


def normals3_many(seed: int, ctr: np.ndarray) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    xi = np.zeros((len(c), 3))
    lib().ora_normals3_many(seed, len(c), _p(c, ctypes.c_uint32), _p(xi, ctypes.c_double))
    return xi


def exp1(seed: int, spring: int, criterion: int, chain: int) -> float:
    return lib().ora_exp1(seed, spring, criterion, chain)


# ---------------------------------------------------------------------------
# Model pieces
# ---------------------------------------------------------------------------

def spring_force(spring: int, H: float, b: float, Q, s_min: float = S_MIN_DEFAULT,
                 r0: float = 0.0):
    q = np.ascontiguousarray(Q, dtype=np.float64)
    F = np.zeros(3)
    t = np.zeros(1)
    fl = lib().ora_spring_force(spring, H, b, r0, s_min, _p(q, ctypes.c_double),
                                _p(F, ctypes.c_double), _p(t, ctypes.c_double))
    return F, float(t[0]), int(fl)


def chain_spring_force(chain, i: int, Q, s_min: float = S_MIN_DEFAULT):
    """(force [3], signed tension, floored) of spring i of `chain` under its law."""
    q = np.ascontiguousarray(Q, dtype=np.float64)
    F = np.zeros(3)
    t = np.zeros(1)
    cs = _chain_struct(chain)
    fl = lib().ora_chain_spring_force(ctypes.byref(cs), int(i), s_min, _p(q, ctypes.c_double),
                                      _p(F, ctypes.c_double), _p(t, ctypes.c_double))
    return F, float(t[0]), int(fl)


def lj_forces(chain, r: np.ndarray) -> np.ndarray:
    """Lennard-Jones forces [N][3] between the non-adjacent beads of r [N][3]."""
    rr = np.ascontiguousarray(r, dtype=np.float64)
    F = np.zeros_like(rr)
    cs = _chain_struct(chain)
    lib().ora_lj_forces(ctypes.byref(cs), _p(rr, ctypes.c_double), _p(F, ctypes.c_double))
    return F


def rpy_block(a: float, d) -> np.ndarray:
    """Eq. 3 / D_0 for the separation d = r_j - r_i of two beads of radius a."""
    dd = np.ascontiguousarray(d, dtype=np.float64)
    out = np.zeros(9)
    lib().ora_rpy_block(a, _p(dd, ctypes.c_double), _p(out, ctypes.c_double))
    return out.reshape(3, 3)


def rpy_matrix(a: float, r: np.ndarray) -> np.ndarray:
    """The 3N x 3N diffusion tensor / D_0 of conformation r [N][3]."""
    rr = np.ascontiguousarray(r, dtype=np.float64)
    N = len(rr)
    D = np.zeros((3 * N, 3 * N))
    lib().ora_rpy_matrix(N, a, _p(rr, ctypes.c_double), _p(D, ctypes.c_double))
    return D


def cholesky(A: np.ndarray):
    """(lower factor, status) of the oracle's Cholesky."""
    a = np.ascontiguousarray(A, dtype=np.float64)
    L = np.zeros_like(a)
    st = lib().ora_cholesky(len(a), _p(a, ctypes.c_double), _p(L, ctypes.c_double))
    return L, int(st)


def flow_gradient(flow: int, rate: float) -> np.ndarray:
    k = np.zeros(9)
    lib().ora_flow_gradient(flow, rate, _p(k, ctypes.c_double))
    return k.reshape(3, 3)


def em_step(chain, dt: float, r: np.ndarray, xi: np.ndarray,
            s_min: float = S_MIN_DEFAULT) -> int:
    """One Eq. 1 step in place on r [N][3] with given noise xi [N][3]."""
    assert r.dtype == np.float64 and r.flags.c_contiguous
    x = np.ascontiguousarray(xi, dtype=np.float64)
    cs = _chain_struct(chain)
    return int(lib().ora_em_step(ctypes.byref(cs), dt, s_min, _p(r, ctypes.c_double),
                                 _p(x, ctypes.c_double)))


def tensions(chain, r: np.ndarray, s_min: float = S_MIN_DEFAULT) -> np.ndarray:
    x = np.ascontiguousarray(r, dtype=np.float64)
    f = np.zeros(chain.n_beads - 1)
    cs = _chain_struct(chain)
    lib().ora_tensions(ctypes.byref(cs), s_min, _p(x, ctypes.c_double), _p(f, ctypes.c_double))
    return f


def criteria_update(q: int, thr_on: bool, bell_on: bool, chain, f: float, dT: float,
                    step: int, E: float, state: Dict[str, float]) -> None:
    lam = np.array([state["lam"]])
    ft = np.array([state["first_thr"]], dtype=np.int64)
    fb = np.array([state["first_bell"]], dtype=np.int64)
    cs = _chain_struct(chain)
    lib().ora_criteria_update(q, int(thr_on), int(bell_on), ctypes.byref(cs), f, dT, step, E,
                              _p(lam, ctypes.c_double), _p(ft, ctypes.c_int64),
                              _p(fb, ctypes.c_int64))
    state["lam"], state["first_thr"], state["first_bell"] = float(lam[0]), int(ft[0]), int(fb[0])


def max_threads() -> int:
    return int(lib().ora_max_threads())


# ---------------------------------------------------------------------------
# The method
# ---------------------------------------------------------------------------

def run(chains, dt: float, window_steps: int, n_steps: int, seed: int, pos0: np.ndarray,
        thr_mask: int = 7, bell_mask: int = 7, identical_noise: bool = False,
        s_min: float = S_MIN_DEFAULT, n_threads: int = 1,
        want_replicas: bool = True, want_windows: bool = True,
        chain_ids: Optional[Sequence[int]] = None) -> Dict[str, np.ndarray]:
    """Run the replica-averaging method from global step 0 on all chains.

    ``thr_mask`` / ``bell_mask`` use bit q for criterion q (0 ISF, 1 TSF,
    2 RSF). ``chain_ids`` gives each chain's id in the noise counter (default
    0, 1, ...), so a sample of a larger problem can be run on its own.
    Returns laboratory-frame parent positions, replica positions,
    per-window RSF/TSF profiles, Bell hazards, first-event steps (-1 none),
    Exp(1) thresholds and FENE-floor counts.
    """
    C = len(chains)
    cs = (_Chain * C)(*[_chain_struct(c) for c in chains])
    ids = None if chain_ids is None else np.ascontiguousarray(chain_ids, dtype=np.int32)
    prob = _Problem(C, int(window_steps), cs, float(dt), int(seed), int(bool(identical_noise)),
                    int(thr_mask), int(bell_mask), float(s_min),
                    _p(ids, ctypes.c_int32) if ids is not None
                    else ctypes.POINTER(ctypes.c_int32)())
    n_beads = sum(c.n_beads for c in chains)
    M = sum(c.n_beads - 1 for c in chains)
    n_rep_beads = sum(c.n_beads * c.n_replicas for c in chains)
    nw = n_steps // window_steps
    pos = np.ascontiguousarray(pos0, dtype=np.float64).copy().reshape(n_beads, 3)
    rep = np.zeros((n_rep_beads, 3)) if want_replicas else None
    rsf = np.zeros((nw, M)) if want_windows else None
    tsf = np.zeros((nw, M)) if want_windows else None
    lam = np.zeros((3, M))
    ft = np.full((3, M), -1, dtype=np.int64)
    fb = np.full((3, M), -1, dtype=np.int64)
    e1 = np.zeros((3, M))
    over = np.zeros(C, dtype=np.int64)
    nul = ctypes.POINTER(ctypes.c_double)()
    rc = lib().ora_run(ctypes.byref(prob), int(n_steps), _p(pos, ctypes.c_double),
                       _p(rep, ctypes.c_double) if rep is not None else nul,
                       _p(rsf, ctypes.c_double) if rsf is not None else nul,
                       _p(tsf, ctypes.c_double) if tsf is not None else nul,
                       _p(lam, ctypes.c_double), _p(ft, ctypes.c_int64), _p(fb, ctypes.c_int64),
                       _p(e1, ctypes.c_double), _p(over, ctypes.c_int64), int(n_threads))
    if rc != 0:
        raise ValueError("oracle rejected the problem")
    return dict(pos=pos, rep=rep, rsf=rsf, tsf=tsf, lam=lam, first_thr=ft, first_bell=fb,
                exp1=e1, overext=over)


def conformation(chains, dt: float, window_steps: int, n_steps: int, seed: int,
                 pos0: np.ndarray, identical_noise: bool = False,
                 s_min: float = S_MIN_DEFAULT, n_threads: int = 1,
                 chain_ids: Optional[Sequence[int]] = None):
    """Eq. 5 diagnostics of every completed window: (dbar [W][sum R][3],
    dbead [W][sum N][3], rgz [W][C]) - see ora_run_conformation."""
    C = len(chains)
    cs = (_Chain * C)(*[_chain_struct(c) for c in chains])
    ids = None if chain_ids is None else np.ascontiguousarray(chain_ids, dtype=np.int32)
    prob = _Problem(C, int(window_steps), cs, float(dt), int(seed), int(bool(identical_noise)),
                    0, 0, float(s_min),
                    _p(ids, ctypes.c_int32) if ids is not None
                    else ctypes.POINTER(ctypes.c_int32)())
    n_beads = sum(c.n_beads for c in chains)
    n_rep = sum(c.n_replicas for c in chains)
    nw = n_steps // window_steps
    pos = np.ascontiguousarray(pos0, dtype=np.float64).copy().reshape(n_beads, 3)
    dbar = np.zeros((nw, n_rep, 3))
    dbead = np.zeros((nw, n_beads, 3))
    rgz = np.zeros((nw, C))
    rc = lib().ora_run_conformation(ctypes.byref(prob), int(n_steps), _p(pos, ctypes.c_double),
                                    _p(dbar, ctypes.c_double), _p(dbead, ctypes.c_double),
                                    _p(rgz, ctypes.c_double), int(n_threads))
    if rc != 0:
        raise ValueError("oracle rejected the problem")
    return dbar, dbead, rgz


def rsf_tangent(chains, dt: float, window_steps: int, n_steps: int, seed: int, pos0: np.ndarray,
                identical_noise: bool = False, s_min: float = S_MIN_DEFAULT, n_threads: int = 1,
                chain_ids: Optional[Sequence[int]] = None):
    """RSF [W][M] and its pathwise derivative (frozen noise) [3][W][M] with
    respect to each chain's (rate, b, H)."""
    C = len(chains)
    cs = (_Chain * C)(*[_chain_struct(c) for c in chains])
    ids = None if chain_ids is None else np.ascontiguousarray(chain_ids, dtype=np.int32)
    prob = _Problem(C, int(window_steps), cs, float(dt), int(seed), int(bool(identical_noise)),
                    0, 0, float(s_min),
                    _p(ids, ctypes.c_int32) if ids is not None
                    else ctypes.POINTER(ctypes.c_int32)())
    n_beads = sum(c.n_beads for c in chains)
    M = sum(c.n_beads - 1 for c in chains)
    W = n_steps // window_steps
    pos = np.ascontiguousarray(pos0, dtype=np.float64).copy().reshape(n_beads, 3)
    rsf = np.zeros((W, M))
    drsf = np.zeros((3, W, M))
    rc = lib().ora_rsf_tangent(ctypes.byref(prob), int(n_steps), _p(pos, ctypes.c_double),
                               _p(rsf, ctypes.c_double), _p(drsf, ctypes.c_double),
                               int(n_threads))
    if rc != 0:
        raise ValueError("oracle rejected the problem")
    return rsf, drsf


def com_frame(pos: np.ndarray, n_beads: Sequence[int]) -> np.ndarray:
    """Subtract each chain's centre of mass (Eq. 5 frame)."""
    out = np.array(pos, dtype=np.float64, copy=True).reshape(-1, 3)
    o = 0
    for n in n_beads:
        out[o:o + n] -= out[o:o + n].mean(axis=0)
        o += n
    return out
