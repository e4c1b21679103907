"""Mechano-reactive kinetics over long runs (Sec. III): the Bell first-passage
rupture times and locations of an ensemble of chains in start-up uniaxial
flow, per force criterion (ISF, TSF, RSF).

- Same Philox draws, FP64: every chain's rupture step and spring equal the
  oracle's exactly.
- Independent noise streams, the batched FP32 path against the FP64 oracle:
  the rupture-time distributions (censored at the end of the run) agree by
  two-sample Kolmogorov-Smirnov tests, and the rupture-location histograms by
  chi-square tests, each at the 95% level with a Bonferroni correction over
  the three criteria (p > 0.05 / 3).
"""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2206_05851_gb300 import bdra
from paper_2206_05851_gb300 import inputs as I

pytestmark = pytest.mark.gpu

N, C, R, S, DT, STEPS = 10, 1024, 8, 50, 2e-3, 4000
ALPHA = 0.05 / 3


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    from paper_2206_05851_gb300 import build as B
    B.build()
    torch.cuda.init()


def _chains():
    b = 50.0
    fmax = I.fene_fmax(1.0, b)
    return [I.Chain(n_beads=N, n_replicas=R, spring=I.SPRING_FENE, flow=I.FLOW_UNIAXIAL, b=b,
                    rate=0.3, f_c=0.9 * fmax, k0=1e-6, dx=20.0 / fmax) for _ in range(C)]


def _gpu(seed, pos0, prec):
    import torch
    ctx = bdra.Context(_chains(), DT, S, seed, pos0, precision=prec, max_windows=STEPS // S + 1,
                       thr_mask=0, bell_mask=I.CRIT_ALL,
                       stream=torch.cuda.current_stream().cuda_stream)
    ctx.step(STEPS)
    _, _, fb = ctx.kinetics()
    ctx.close()
    return fb


def _oracle(seed, pos0):
    r = O.run(_chains(), DT, S, STEPS, seed, pos0, thr_mask=0, bell_mask=I.CRIT_ALL,
              n_threads=os.cpu_count() or 1, want_replicas=False)
    return r["first_bell"]


def _first_rupture(first_bell):
    """Per criterion and chain: (step of the first Bell rupture, spring), step
    STEPS + 1 and spring -1 where the chain survived."""
    t = np.where(first_bell >= 0, first_bell, STEPS + 1).reshape(3, C, N - 1)
    step = t.min(axis=2)
    loc = np.where(step <= STEPS, t.argmin(axis=2), -1)
    return step, loc


def test_same_noise_fp64_rupture_steps_and_springs_exact():
    pos0 = I.initial_positions(I.custom(_chains(), DT, S, STEPS), seed=31)
    g = _gpu(3, pos0, bdra.BD_PREC_FP64)
    o = _oracle(3, pos0)
    np.testing.assert_array_equal(g, o)
    step, _ = _first_rupture(o)
    assert (step <= STEPS).mean() > 0.5          # the run does exercise the kinetics


@pytest.fixture(scope="module")
def independent():
    from scipy import stats  # noqa: F401  (fail early if missing)
    wl = I.custom(_chains(), DT, S, STEPS)
    g = _first_rupture(_gpu(101, I.initial_positions(wl, seed=41), bdra.BD_PREC_FP32))
    o = _first_rupture(_oracle(202, I.initial_positions(wl, seed=42)))
    return g, o


@pytest.mark.parametrize("q", [0, 1, 2])
def test_rupture_time_distributions_agree(independent, q):
    from scipy import stats
    (gs, _), (os_, _) = independent
    assert 0.3 < (gs[q] <= STEPS).mean() < 1.0 and 0.3 < (os_[q] <= STEPS).mean() < 1.0
    p = stats.ks_2samp(gs[q], os_[q]).pvalue
    assert p > ALPHA, f"criterion {q}: KS p = {p:.4f}"


@pytest.mark.parametrize("q", [0, 1, 2])
def test_rupture_location_histograms_agree(independent, q):
    from scipy import stats
    (_, gl), (_, ol) = independent
    table = np.array([[np.sum(gl[q] == i) for i in range(-1, N - 1)],
                      [np.sum(ol[q] == i) for i in range(-1, N - 1)]])
    table = table[:, table.sum(axis=0) >= 10]     # merge-free: drop bins too sparse for chi-square
    p = stats.chi2_contingency(table).pvalue
    assert p > ALPHA, f"criterion {q}: chi-square p = {p:.4f}\n{table}"
