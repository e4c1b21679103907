"""Float32 parity of profiles and events against the FP64 oracle (helpers for
the GPU tests; not collected by pytest).

Reading of the criteria of Sec. II (threshold on ISF, TSF, RSF) and Sec. III
(Bell rate k0 exp(f dx) with the survival integral) for a float32 run:

- Force profiles (RSF, TSF) are one result per chain and window: each
  (chain, window) row is compared normwise, relative to that row's largest
  force, so a wrong force on a few low-tension springs is not hidden under
  the largest spring of another chain or window. For the laws with a rest
  length r0 (the collapsed chain's harmonic springs, the vWF springs) the
  force H (|Q| - r0) is a small difference of bond lengths times a large
  stiffness: the bond length carries the trajectory's relative error, so
  the force error scales with H r0, not with the force. Their rows are
  compared relative to max(largest force, H r0), H the chain's stiffest
  spring.
- Event steps (first threshold crossing, first Bell passage) must equal the
  oracle's, except at a near-tie. A float32 and a float64 run that differ in
  the force by a small relative error can take a boundary decision on
  different sides only where the oracle's own quantity sits at the boundary
  at the earlier of the two event steps t (at t one side has crossed and the
  other has not):
    * threshold: |f_ora(t) - f_c| < 1e-4 |f_c| (the near-tie band of a
      float32 run);
    * Bell: |ln Lambda_ora(t) - ln E| within the float32 log-hazard
      tolerance, 1e-4 |ln E| + 2e-3. A relative force error e moves the
      log of every hazard increment k0 exp(dx f) dT by dx f e, and the
      workloads' dx F_max = 20 with e = 1e-4 gives the 2e-3; a sum of
      positive increments has at most the largest relative error of its
      terms.
  f_ora(t) and Lambda_ora(t) are the oracle's, re-computed for each
  mismatch by running that spring's chain alone up to step t (same global
  chain id in the noise counter, so the same draws). Window criteria read
  the oracle's stored RSF / TSF row of the window that ends at t.
- Near-ties are counted and returned, and kept apart from the exact-match
  set, which must be equal element by element.
"""
from __future__ import annotations

from typing import Dict, Optional, Sequence

import numpy as np

from oracle import oracle as O
from paper_2206_05851_gb300 import inputs as I

THR_BAND = 1e-4          # threshold near-tie band, relative to |f_c|
LOG_HAZ_REL, LOG_HAZ_ABS = 1e-4, 2e-3


def log_hazard_close(lg: np.ndarray, lr: np.ndarray) -> np.ndarray:
    """Float32 hazards against the oracle's, in log space."""
    return np.abs(lg - lr) <= LOG_HAZ_REL * np.abs(lr) + LOG_HAZ_ABS


def force_scale(ch) -> float:
    """H r0 of a law with a rest length (0 for FENE and Hookean springs)."""
    if ch.spring == I.SPRING_HARMONIC:
        return ch.H * ch.r0
    if ch.spring == I.SPRING_VWF:
        return max(ch.H, ch.vwf_fa + ch.vwf_fb) * ch.r0
    return 0.0


def profile_rows_rel_err(got: np.ndarray, want: np.ndarray, chains) -> float:
    """Largest normwise relative error over the (chain, window) rows of a
    [W][M] profile history."""
    offs = I.spring_offsets(chains)
    worst = 0.0
    for c in range(len(chains)):
        g, w = got[:, offs[c]:offs[c + 1]], want[:, offs[c]:offs[c + 1]]
        if g.size == 0:
            continue
        den = np.maximum(np.maximum(np.abs(w).max(axis=1), force_scale(chains[c])), 1e-300)
        worst = max(worst, float((np.abs(g - w).max(axis=1) / den).max()))
    return worst


def check_profiles(g: Dict, r: Dict, chains, tol: float, keys=("rsf", "tsf")) -> None:
    for key in keys:
        assert g[key].shape == r[key].shape, key
        if g[key].size:
            err = profile_rows_rel_err(g[key], r[key], chains)
            assert err <= tol, f"{key}: per-(chain, window) rel err {err:.3e} > {tol}"


class OracleReplay:
    """The oracle's state of one chain at a given step, from a run of that
    chain alone from the same start (for the near-tie checks)."""

    def __init__(self, chains, dt, S, seed, pos0, thr_mask, bell_mask,
                 chain_ids: Optional[Sequence[int]] = None):
        self.chains, self.dt, self.S, self.seed = chains, dt, S, seed
        self.pos0 = np.asarray(pos0, dtype=np.float64).reshape(-1, 3)
        self.thr, self.bell = thr_mask, bell_mask
        self.ids = list(range(len(chains))) if chain_ids is None else list(chain_ids)
        self.boff = I.bead_offsets(chains)
        self._cache = {}

    def at(self, c: int, n_steps: int):
        """(integrated hazards [3][N-1], ISF tensions [N-1]) of chain c after
        n_steps steps."""
        key = (c, n_steps)
        if key not in self._cache:
            ch = self.chains[c]
            p0 = self.pos0[self.boff[c]:self.boff[c + 1]]
            r = O.run([ch], self.dt, self.S, n_steps, self.seed, p0, thr_mask=self.thr,
                      bell_mask=self.bell, want_replicas=False, want_windows=False,
                      chain_ids=[self.ids[c]])
            self._cache[key] = (r["lam"], O.tensions(ch, r["pos"]))
        return self._cache[key]


def compare_events_fp32(g: Dict, r: Dict, chains, S: int, replay: OracleReplay,
                        cols: Optional[np.ndarray] = None) -> Dict[str, int]:
    """Event steps of a float32 run equal the oracle's except at near-ties.

    g: GPU results (first_thr, first_bell [3][M_gpu]); r: oracle results of
    `chains` (first_thr, first_bell, exp1, rsf, tsf, [3][M] / [W][M]); cols:
    the GPU columns of the oracle's springs when the oracle ran a sample.
    Returns counts of exact matches and near-ties per kind."""
    offs = I.spring_offsets(chains)
    chain_of = np.repeat(np.arange(len(chains)), np.diff(offs))
    counts = dict(thr_equal=0, thr_near_tie=0, bell_equal=0, bell_near_tie=0)
    for kind, key in (("thr", "first_thr"), ("bell", "first_bell")):
        got = g[key] if cols is None else g[key][:, cols]
        want = r[key]
        assert got.shape == want.shape
        counts[f"{kind}_equal"] = int(((got == want) & (want >= 0)).sum())
        for q, m in zip(*np.nonzero(got != want)):
            a, b = int(got[q, m]), int(want[q, m])
            t = min(x for x in (a, b) if x >= 0)
            c = int(chain_of[m])
            i = int(m - offs[c])
            ch = chains[c]
            where = f"criterion {q} chain {c} spring {i}: gpu step {a}, oracle step {b}"
            if kind == "thr":
                if q == O.ISF:
                    f = replay.at(c, t)[1][i]
                else:
                    assert t % S == 0, where
                    f = r["rsf" if q == O.RSF else "tsf"][t // S - 1, m]
                gap = abs(f - ch.f_c) / abs(ch.f_c)
                assert gap < THR_BAND, f"{where}: threshold event differs, |f - f_c|/f_c = {gap:.2e}"
            else:
                lam = replay.at(c, t)[0][q, i]
                E = r["exp1"][q, m]
                assert lam > 0, f"{where}: Bell passage differs with no hazard"
                ok = log_hazard_close(np.log(lam), np.log(E))
                assert ok, f"{where}: Bell passage differs, ln(Lambda/E) = {np.log(lam / E):.2e}"
            counts[f"{kind}_near_tie"] += 1
    return counts


def compare_hazards_fp32(g_haz: np.ndarray, r_lam: np.ndarray) -> None:
    """Float32 hazards in log space where the oracle's are positive, and
    exactly zero where the oracle's are zero."""
    gh, rl = np.ravel(g_haz), np.ravel(r_lam)
    pos = rl > 0
    ok = log_hazard_close(np.log(gh[pos]), np.log(rl[pos]))
    assert ok.all(), (np.nonzero(pos)[0][~ok][:5], gh[pos][~ok][:5], rl[pos][~ok][:5])
    np.testing.assert_array_equal(gh[~pos], rl[~pos])
