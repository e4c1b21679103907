"""Pins of the oracle's coarse-grained vWF chain (supplementary material,
Table S1): A2 domains (a FENE spring in parallel with a harmonic spring) on
the even springs, disulfide bonds (harmonic) on the odd springs, rest length
2a, Lennard-Jones cohesion; Bell unfolding of the A2 domains only.

- Forces: a zero-noise step moves the beads by (dt/4)(-grad U) with U written
  out here as potentials (the A2 domain's FENE part -(f_A x_max^2 / 2)
  ln(1 - x^2/x_max^2)), on random conformations of 4 and 7 beads.
- The A2 domain's small-extension stiffness is f_A + f_B; the disulfide
  bond's is H; the FENE part's floor applies and is counted.
- Kinetics: with a large Bell rate every A2 domain unfolds and no disulfide
  bond does, under all three criteria.
- Statics: three beads (one A2 domain, one disulfide bond) at rest sample
  exp(-U): bond lengths and bead angle against 3-D quadrature.
- Units: every library-unit constant of the chain follows from Table S1's
  printed SI values (`tests/golden/vwf_table_s1.txt`), and the conversion
  reproduces the supplement's mean-force unfolding time 1 / (25 k0 exp(f /
  f_u)) computed in seconds from those values.
"""
import math
import os

import numpy as np
import pytest
from scipy import integrate

from oracle import oracle as O
from paper_2206_05851_gb300 import inputs as I

R0, SIG = 2.0, 2.0
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "vwf_table_s1.txt")


def _chain(N, R=1, fa=20.0, fb=30.0, xmax=0.8, H=50.0, u=2.0, **kw):
    return I.Chain(n_beads=N, n_replicas=R, spring=I.SPRING_VWF, H=H, r0=R0, lj_u=u, lj_sigma=SIG,
                   vwf_fa=fa, vwf_fb=fb, vwf_xmax=xmax, **kw)


def _potential(r, ch):
    U = 0.0
    for i in range(len(r) - 1):
        x = np.linalg.norm(r[i + 1] - r[i]) - ch.r0
        if i % 2 == 0:
            U += 0.5 * ch.vwf_fb * x * x - 0.5 * ch.vwf_fa * ch.vwf_xmax ** 2 * math.log(1 - (x / ch.vwf_xmax) ** 2)
        else:
            U += 0.5 * ch.H * x * x
    for i in range(len(r)):
        for j in range(i + 2, len(r)):
            s = ch.lj_sigma / np.linalg.norm(r[j] - r[i])
            U += ch.lj_u * (s ** 12 - 2 * s ** 6)
    return U


@pytest.mark.parametrize("N", [4, 7])
def test_zero_noise_step_is_minus_grad_u(N):
    rng = np.random.default_rng(N)
    ch = _chain(N)
    r = np.zeros((N, 3))
    for i in range(1, N):
        d = rng.normal(size=3)
        r[i] = r[i - 1] + d / np.linalg.norm(d) * (R0 + 0.4 * (rng.random() - 0.5))
    dt = 1e-7
    r1 = r.copy()
    O.em_step(ch, dt, r1, np.zeros((N, 3)))
    g = np.zeros_like(r)
    h = 1e-6
    for i in range(N):
        for k in range(3):
            rp, rm = r.copy(), r.copy()
            rp[i, k] += h
            rm[i, k] -= h
            g[i, k] = (_potential(rp, ch) - _potential(rm, ch)) / (2 * h)
    np.testing.assert_allclose((r1 - r) / (0.25 * dt), -g, rtol=1e-5, atol=1e-5 * np.abs(g).max())


def test_small_extension_stiffness_and_floor():
    ch = _chain(3)
    e = np.array([0.3, -0.4, 0.866])
    e /= np.linalg.norm(e)
    x = 1e-6
    _, fa2, fl = O.chain_spring_force(ch, 0, (R0 + x) * e)
    assert fa2 / x == pytest.approx(ch.vwf_fa + ch.vwf_fb, rel=1e-9) and fl == 0
    _, fds, _ = O.chain_spring_force(ch, 1, (R0 - x) * e)
    assert fds / -x == pytest.approx(ch.H, rel=1e-9)
    # beyond the FENE limit the denominator is floored (and counted)
    F, f, fl = O.chain_spring_force(ch, 2, (R0 + 1.2 * ch.vwf_xmax) * e, s_min=1e-3)
    assert fl == 1
    xx = 1.2 * ch.vwf_xmax
    assert f == pytest.approx(ch.vwf_fb * xx + ch.vwf_fa * xx / 1e-3, rel=1e-12)
    np.testing.assert_allclose(F, f * e, rtol=1e-12)


def test_only_a2_domains_unfold():
    N = 9
    chains = [_chain(N, R=4, k0=500.0, dx=0.2) for _ in range(3)]
    pos0 = I.initial_positions(I.custom(chains, 1e-4, 20, 400), seed=3)
    out = O.run(chains, 1e-4, 20, 400, seed=2, pos0=pos0, thr_mask=0, bell_mask=7, n_threads=4)
    fb = out["first_bell"].reshape(3, len(chains), N - 1)
    lam = out["lam"].reshape(3, len(chains), N - 1)
    assert (fb[:, :, 0::2] >= 0).all()
    assert (fb[:, :, 1::2] < 0).all() and (lam[:, :, 1::2] == 0).all()


def test_three_beads_at_rest_match_the_stationary_density():
    ch = _chain(3)

    def weight(r1, r2, c):
        x1, x2 = r1 - R0, r2 - R0
        if abs(x1) >= ch.vwf_xmax:
            return 0.0
        u_a2 = 0.5 * ch.vwf_fb * x1 * x1 - 0.5 * ch.vwf_fa * ch.vwf_xmax ** 2 * math.log(1 - (x1 / ch.vwf_xmax) ** 2)
        r02 = math.sqrt(max(r1 * r1 + r2 * r2 - 2 * r1 * r2 * c, 1e-12))
        s = SIG / r02
        return r1 * r1 * r2 * r2 * math.exp(-u_a2 - 0.5 * ch.H * x2 * x2 - ch.lj_u * (s ** 12 - 2 * s ** 6))

    lo1, hi1 = R0 - ch.vwf_xmax, R0 + ch.vwf_xmax
    lo2, hi2 = R0 - 1.0, R0 + 1.0
    opts = dict(epsabs=1e-13, epsrel=1e-8)
    Z = integrate.tplquad(lambda c, r2, r1: weight(r1, r2, c), lo1, hi1, lo2, hi2, -1, 1, **opts)[0]
    mom = {}
    for name, fn in (("cos", lambda r1, r2, c: c), ("r1", lambda r1, r2, c: r1), ("r2", lambda r1, r2, c: r2)):
        mom[name] = integrate.tplquad(lambda c, r2, r1: fn(r1, r2, c) * weight(r1, r2, c),
                                      lo1, hi1, lo2, hi2, -1, 1, **opts)[0] / Z
    R, dt, steps = 600, 2e-3, 40000
    chains = [_chain(3, R=R) for _ in range(8)]
    pos0 = np.zeros((24, 3))
    pos0[:, 2] = np.tile([0.0, 2.0, 4.0], 8)
    out = O.run(chains, dt, steps, steps, seed=19, pos0=pos0, thr_mask=0, bell_mask=0, n_threads=8)
    rep = out["rep"].reshape(8 * R, 3, 3)
    q1, q2 = rep[:, 1] - rep[:, 0], rep[:, 2] - rep[:, 1]
    n1, n2 = np.linalg.norm(q1, axis=1), np.linalg.norm(q2, axis=1)
    cos_bead = -(q1 * q2).sum(axis=1) / (n1 * n2)
    for est, want in ((cos_bead, mom["cos"]), (n1, mom["r1"]), (n2, mom["r2"])):
        sd = est.std() / math.sqrt(est.size)
        assert abs(est.mean() - want) < 5 * sd + 0.003 * abs(want), (est.mean(), want, sd)
    assert out["overext"].sum() == 0


def _table_s1():
    vals = {}
    with open(GOLDEN) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                name, value, _unit = line.split()
                vals[name] = float(value)
    return vals


def test_library_units_follow_table_s1():
    # lengths in a, energies in kT = epsilon, time unit tau / 4 with
    # tau = 6 pi eta a^3 / kT (the collapsed chain's units)
    t = _table_s1()
    a, kT = t["a"], t["epsilon"]
    assert 1.380649e-2 * t["T"] == pytest.approx(kT, rel=1e-3)      # k_B T at 300 K in pN nm
    tau_s = 6 * math.pi * t["eta"] * a ** 3 / kT * 1e-6               # us -> s
    assert I.VWF_TAU_S == pytest.approx(tau_s, rel=1e-12)
    ch = I.vwf_chain(1)
    assert ch.H == pytest.approx(t["f_harm"] * a * a / kT, rel=1e-12)
    assert ch.vwf_fa == pytest.approx(t["f_A"] * a * a / kT, rel=1e-12)
    assert ch.vwf_fb == pytest.approx(t["f_B"] * a * a / kT, rel=1e-12)
    assert ch.vwf_xmax == pytest.approx(t["r_max"] / a, rel=1e-12)
    assert ch.k0 == pytest.approx(t["k0"] * tau_s / 4, rel=1e-12)
    assert ch.dx == pytest.approx((kT / a) / t["f_u"], rel=1e-12)
    assert ch.spring == I.SPRING_VWF and ch.lj_u == 1.0 and ch.r0 == 2.0 and ch.lj_sigma == 2.0


def test_unit_conversion_reproduces_the_mean_force_unfolding_time():
    # Supplementary material: MFTU = 1 / [25 k0 exp(<f>/f_u)] in seconds,
    # straight from the printed SI values
    t = _table_s1()
    want = 1.0 / (25 * t["k0"] * math.exp(t["mean_a2_force"] / t["f_u"]))
    ch = I.vwf_chain(1)
    f = t["mean_a2_force"] / I.VWF_FORCE_UNIT_PN                     # the same force in kT / a
    got = I.vwf_mftu_seconds(25 * ch.k0 * math.exp(ch.dx * f))
    assert got == pytest.approx(want, rel=1e-12)
