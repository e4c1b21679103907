"""Pins of the oracle's collapsed-chain model (Sec. II): harmonic springs with
rest length 2a, U_s = (kappa/2)(|Q| - 2a)^2, and Lennard-Jones cohesion
between non-adjacent beads, U_LJ = u [(2a/r)^12 - 2 (2a/r)^6], in units of
the bead radius a and kT.

- The bead forces of one zero-noise Euler step equal -grad U (numerical
  derivative of the total potential) on random conformations.
- Three beads at rest (no flow): the stationary density is exp(-U); the
  bond length and the bond-angle cosine of a long ensemble match 3-D
  quadrature over (r1, r2, cos theta) with the Jacobian r1^2 r2^2. The angle
  is set by the 0-2 Lennard-Jones term alone (uniform without it), so a
  wrong sign, factor or range of the pair force moves it.
"""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import oracle as O
from paper_2206_05851_gb300 import inputs as I

KAPPA, R0, U_LJ, SIG = 400.0, 2.0, 1.0, 2.0


def _chain(N, R=1, flow=I.FLOW_NONE, rate=0.0):
    return I.Chain(n_beads=N, n_replicas=R, spring=I.SPRING_HARMONIC, flow=flow, rate=rate,
                   H=KAPPA, r0=R0, lj_u=U_LJ, lj_sigma=SIG)


def _potential(r):
    N = len(r)
    U = 0.0
    for i in range(N - 1):
        U += 0.5 * KAPPA * (np.linalg.norm(r[i + 1] - r[i]) - R0) ** 2
    for i in range(N):
        for j in range(i + 2, N):
            x = SIG / np.linalg.norm(r[j] - r[i])
            U += U_LJ * (x ** 12 - 2 * x ** 6)
    return U


def test_eq4_signed_spring_force():
    for q in (1.7, 2.0, 2.3):
        Q = np.array([0.0, 0.0, q])
        F, f, fl = O.spring_force(I.SPRING_HARMONIC, KAPPA, 1.0, Q, r0=R0)
        assert f == pytest.approx(KAPPA * (q - R0), abs=1e-12) and fl == 0
        np.testing.assert_allclose(F, [0, 0, KAPPA * (q - R0)], atol=1e-12)


@pytest.mark.parametrize("N", [3, 6])
def test_zero_noise_step_moves_beads_down_the_potential_gradient(N):
    rng = np.random.default_rng(N)
    ch = _chain(N)
    # a compact random walk with bonds near 2a, so that LJ terms are active
    r = np.cumsum(rng.normal(size=(N, 3)), axis=0)
    for i in range(1, N):
        d = r[i] - r[i - 1]
        r[i] = r[i - 1] + d / np.linalg.norm(d) * (R0 + 0.1 * rng.normal())
    dt = 1e-7
    r1 = r.copy()
    O.em_step(ch, dt, r1, np.zeros((N, 3)))
    F = (r1 - r) / (0.25 * dt)                    # bead diffusivity 1/4 in these units
    g = np.zeros_like(r)
    h = 1e-6
    for i in range(N):
        for k in range(3):
            rp, rm = r.copy(), r.copy()
            rp[i, k] += h
            rm[i, k] -= h
            g[i, k] = (_potential(rp) - _potential(rm)) / (2 * h)
    np.testing.assert_allclose(F, -g, rtol=1e-5, atol=1e-4 * np.abs(g).max())


def test_three_beads_at_rest_match_the_stationary_density():
    # A softer spring and a deeper well than the paper's (kappa 50, u 2) so that
    # the bond angle equilibrates within a short run; the force laws are the same.
    kappa, u = 50.0, 2.0

    def weight(r1, r2, c):
        r02 = math.sqrt(max(r1 * r1 + r2 * r2 - 2 * r1 * r2 * c, 1e-12))   # c: cos of the bead angle
        x = SIG / r02
        return r1 * r1 * r2 * r2 * math.exp(-0.5 * kappa * ((r1 - R0) ** 2 + (r2 - R0) ** 2)
                                            - u * (x ** 12 - 2 * x ** 6))

    lo, hi = R0 - 1.0, R0 + 1.0
    opts = dict(epsabs=1e-13, epsrel=1e-8)
    Z = integrate.tplquad(lambda c, r2, r1: weight(r1, r2, c), lo, hi, lo, hi, -1, 1, **opts)[0]
    mc = integrate.tplquad(lambda c, r2, r1: c * weight(r1, r2, c), lo, hi, lo, hi, -1, 1, **opts)[0] / Z
    mr = integrate.tplquad(lambda c, r2, r1: r1 * weight(r1, r2, c), lo, hi, lo, hi, -1, 1, **opts)[0] / Z
    # the oracle: 8 chains x 600 replicas from a straight start, one window of
    # 80 time units (five rotational relaxation times)
    R, dt, steps = 600, 2e-3, 40000
    chains = [I.Chain(n_beads=3, n_replicas=R, spring=I.SPRING_HARMONIC, H=kappa, r0=R0,
                      lj_u=u, lj_sigma=SIG) for _ in range(8)]
    pos0 = np.zeros((24, 3))
    pos0[:, 2] = np.tile([0.0, 2.0, 4.0], 8)
    out = O.run(chains, dt, steps, steps, seed=13, pos0=pos0, thr_mask=0, bell_mask=0, n_threads=8)
    rep = out["rep"].reshape(8 * R, 3, 3)
    q1, q2 = rep[:, 1] - rep[:, 0], rep[:, 2] - rep[:, 1]
    n1, n2 = np.linalg.norm(q1, axis=1), np.linalg.norm(q2, axis=1)
    cos_bead = -(q1 * q2).sum(axis=1) / (n1 * n2)         # angle at bead 1 between its bonds
    for est, want in ((cos_bead, mc), (n1, mr)):
        sd = est.std() / math.sqrt(est.size)
        assert abs(est.mean() - want) < 5 * sd + 0.005 * abs(want), (est.mean(), want, sd)
    assert mc > 0.05       # the 0-2 cohesion bends the trimer (without it <cos> = 0)
