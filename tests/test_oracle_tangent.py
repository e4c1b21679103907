"""Pins of the oracle's pathwise derivatives (frozen noise) of the RSF profile
with respect to each chain's strain rate, FENE extensibility b and spring
constant H: central finite differences with common random numbers through
the pinned forward oracle, and special cases that must vanish."""
import dataclasses
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2206_05851_gb300 import inputs as I


def _chains():
    return [I.Chain(n_beads=6, n_replicas=4, spring=I.SPRING_FENE, flow=I.FLOW_UNIAXIAL, b=30.0,
                    rate=0.4, H=1.1),
            I.Chain(n_beads=9, n_replicas=3, spring=I.SPRING_FENE, flow=I.FLOW_SHEAR, b=50.0,
                    rate=1.5, H=0.9),
            I.Chain(n_beads=5, n_replicas=2, spring=I.SPRING_HOOKE, flow=I.FLOW_PLANAR, b=20.0,
                    rate=0.3, H=1.3)]


PARAMS = ["rate", "b", "H"]


@pytest.mark.parametrize("j", [0, 1, 2])
def test_tangent_matches_common_random_number_finite_differences(j):
    chains = _chains()
    dt, S, n, seed = 2e-3, 25, 100, 5
    pos0 = I.initial_positions(I.custom(chains, dt, S, n), seed=3)
    rsf, drsf = O.rsf_tangent(chains, dt, S, n, seed, pos0)
    h = 1e-5
    fd = np.zeros_like(rsf)
    o = 0
    for c, ch in enumerate(chains):
        nb = ch.n_beads - 1
        val = getattr(ch, PARAMS[j])
        step = h * val
        runs = []
        for sgn in (1, -1):
            cc = list(chains)
            cc[c] = dataclasses.replace(ch, **{PARAMS[j]: val + sgn * step})
            r = O.run(cc, dt, S, n, seed, pos0, thr_mask=0, bell_mask=0, want_replicas=False)
            assert r["overext"].sum() == 0
            runs.append(r["rsf"][:, o:o + nb])
        fd[:, o:o + nb] = (runs[0] - runs[1]) / (2 * step)
        o += nb
    scale = np.abs(drsf[j]).max()
    assert scale > 0 or j == 1
    np.testing.assert_allclose(drsf[j], fd, rtol=1e-5, atol=1e-6 * max(scale, 1e-3))


def test_tangent_vanishes_where_the_parameter_does_not_enter():
    ch = [I.Chain(n_beads=5, n_replicas=3, spring=I.SPRING_FENE, flow=I.FLOW_NONE, b=30.0,
                  rate=0.7),
          I.Chain(n_beads=4, n_replicas=2, spring=I.SPRING_HOOKE, flow=I.FLOW_SHEAR, b=30.0,
                  rate=0.7)]
    pos0 = I.initial_positions(I.custom(ch, 1e-3, 10, 40), seed=1)
    _, drsf = O.rsf_tangent(ch, 1e-3, 10, 40, 2, pos0)
    assert np.all(drsf[0][:, :4] == 0.0)          # no flow: the rate does nothing
    assert np.all(drsf[1][:, 4:] == 0.0)          # Hookean spring: b does nothing
    assert np.abs(drsf[2]).max() > 0


def test_tangent_rsf_equals_forward_rsf():
    chains = _chains()
    pos0 = I.initial_positions(I.custom(chains, 2e-3, 25, 75), seed=4)
    rsf, _ = O.rsf_tangent(chains, 2e-3, 25, 75, 9, pos0)
    ref = O.run(chains, 2e-3, 25, 75, 9, pos0, thr_mask=0, bell_mask=0)["rsf"]
    np.testing.assert_array_equal(rsf, ref)
