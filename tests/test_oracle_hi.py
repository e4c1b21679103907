"""Pins of the oracle's hydrodynamic interaction (Eqs. 1-3): the
Rotne-Prager-Yamakawa diffusion tensor, its Cholesky factor and the
correlated Euler-Maruyama step.

Tensor (in units of the single-bead diffusivity D_0, bead radius a):
- at contact (r = 2a) both branches give the textbook RPY mobilities 5/8
  (along the line of centres) and 7/16 (across it);
- as r -> 0 the overlap branch tends to the self term I of Eq. 2;
- far apart it tends to the Oseen tensor (3a / 4r)(I + d d / r^2);
- it is divergence-free in the separation (both branches), which is why
  Eq. 1 needs no drift correction;
- the 3N x 3N tensor is positive definite, overlaps included.
Step:
- the factor is lower triangular with a positive diagonal and L L^T = D;
- zero-force steps have displacement covariance (dt/2) D (noise sqrt(2 D_0
  dt) L xi with D_0 = 1/4);
- zero-noise steps move the beads by (dt/4) D (-grad U);
- a vanishing radius gives back the free-draining step;
- statics: three collapsed beads with hydrodynamic interaction sample the
  same stationary density exp(-U) as without it (3-D quadrature).
"""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import oracle as O
from paper_2206_05851_gb300 import inputs as I


def _unit(rng):
    u = rng.normal(size=3)
    return u / np.linalg.norm(u)


@pytest.mark.parametrize("a", [1.0, 0.7])
def test_contact_mobilities(a):
    rng = np.random.default_rng(1)
    for _ in range(4):
        e = _unit(rng)
        for r in (2 * a, 2 * a * (1 - 1e-12), 2 * a * (1 + 1e-12)):
            B = O.rpy_block(a, r * e)
            assert e @ B @ e == pytest.approx(5 / 8, abs=1e-9)
            p = np.cross(e, _unit(rng))
            p /= np.linalg.norm(p)
            assert p @ B @ p == pytest.approx(7 / 16, abs=1e-9)


def test_overlap_limit_is_the_self_term():
    B = O.rpy_block(1.0, [1e-9, 2e-9, -1e-9])
    np.testing.assert_allclose(B, np.eye(3), atol=1e-8)


def test_far_field_is_oseen():
    rng = np.random.default_rng(2)
    a = 1.0
    for r in (1e3, 1e4):
        e = _unit(rng)
        B = O.rpy_block(a, r * e)
        oseen = 3 * a / (4 * r) * (np.eye(3) + np.outer(e, e))
        assert np.abs(B - oseen).max() <= 1.0 * (a / r) ** 3      # next term is O((a/r)^3)


@pytest.mark.parametrize("r", [0.3, 1.2, 1.9, 2.5, 7.0])
def test_divergence_free(r):
    rng = np.random.default_rng(int(r * 10))
    a, h = 1.0, 1e-5
    for _ in range(3):
        d = r * _unit(rng)
        div = np.zeros(3)
        for y in range(3):
            dp, dm = d.copy(), d.copy()
            dp[y] += h
            dm[y] -= h
            div += (O.rpy_block(a, dp)[:, y] - O.rpy_block(a, dm)[:, y]) / (2 * h)
        assert np.abs(div).max() < 1e-7


def test_tensor_positive_definite_and_factor():
    rng = np.random.default_rng(3)
    for N, spread in ((5, 0.8), (12, 2.0), (30, 3.0)):
        r = rng.normal(scale=spread, size=(N, 3))           # many overlapping pairs
        D = O.rpy_matrix(1.0, r)
        np.testing.assert_allclose(D, D.T, atol=1e-15)
        assert np.linalg.eigvalsh(D).min() > 0
        L, st = O.cholesky(D)
        assert st == 0
        assert np.all(np.triu(L, 1) == 0) and np.all(np.diag(L) > 0)
        np.testing.assert_allclose(L @ L.T, D, atol=1e-13)
    _, st = O.cholesky(np.array([[1.0, 2.0], [2.0, 1.0]]))
    assert st == 1                                          # indefinite: reported


def _chain(N, a=1.0, H=1e-12):
    return I.Chain(n_beads=N, n_replicas=1, spring=I.SPRING_HOOKE, H=H, hi_a=a)


def test_noise_covariance_is_2_D_dt():
    rng = np.random.default_rng(4)
    N, dt, n = 3, 1e-2, 40000
    r0 = np.array([[0.0, 0.0, 0.0], [1.5, 0.3, 0.0], [2.0, 2.2, 0.4]])
    ch = _chain(N)
    xs = rng.normal(size=(n, N, 3))
    disp = np.empty((n, 3 * N))
    for k in range(n):
        r = r0.copy()
        O.em_step(ch, dt, r, xs[k])
        disp[k] = (r - r0).ravel()
    cov = disp.T @ disp / n
    want = (dt / 2) * O.rpy_matrix(1.0, r0)
    assert np.abs(cov - want).max() < 0.04 * np.abs(want).max()
    # the displacement is linear in xi with the lower factor: check one draw exactly
    r = r0.copy()
    O.em_step(ch, dt, r, xs[0])
    L, _ = O.cholesky(O.rpy_matrix(1.0, r0))
    np.testing.assert_allclose((r - r0).ravel(), math.sqrt(dt / 2) * L @ xs[0].ravel(), atol=1e-14)


def _potential(r, kappa, r0, u, sig):
    U = 0.0
    N = len(r)
    for i in range(N - 1):
        U += 0.5 * kappa * (np.linalg.norm(r[i + 1] - r[i]) - r0) ** 2
    for i in range(N):
        for j in range(i + 2, N):
            x = sig / np.linalg.norm(r[j] - r[i])
            U += u * (x ** 12 - 2 * x ** 6)
    return U


def test_zero_noise_drift_is_mobility_times_force():
    rng = np.random.default_rng(5)
    N = 5
    ch = I.Chain(n_beads=N, n_replicas=1, spring=I.SPRING_HARMONIC, H=400.0, r0=2.0, lj_u=1.0,
                 lj_sigma=2.0, hi_a=1.0)
    r = np.cumsum(rng.normal(size=(N, 3)), axis=0)
    for i in range(1, N):
        d = r[i] - r[i - 1]
        r[i] = r[i - 1] + d / np.linalg.norm(d) * (2.0 + 0.1 * rng.normal())
    dt = 1e-7
    r1 = r.copy()
    O.em_step(ch, dt, r1, np.zeros((N, 3)))
    g = np.zeros(3 * N)
    h = 1e-6
    for p in range(3 * N):
        rp, rm = r.copy().ravel(), r.copy().ravel()
        rp[p] += h
        rm[p] -= h
        g[p] = (_potential(rp.reshape(N, 3), 400.0, 2.0, 1.0, 2.0)
                - _potential(rm.reshape(N, 3), 400.0, 2.0, 1.0, 2.0)) / (2 * h)
    want = 0.25 * dt * O.rpy_matrix(1.0, r) @ (-g)
    got = (r1 - r).ravel()
    np.testing.assert_allclose(got, want, rtol=1e-5, atol=1e-5 * np.abs(want).max())


def test_vanishing_radius_is_free_draining():
    rng = np.random.default_rng(6)
    N = 6
    r = np.cumsum(rng.normal(size=(N, 3)), axis=0)
    xi = rng.normal(size=(N, 3))
    base = I.Chain(n_beads=N, n_replicas=1, spring=I.SPRING_FENE, b=50.0, flow=I.FLOW_SHEAR, rate=1.0)
    hi = I.Chain(n_beads=N, n_replicas=1, spring=I.SPRING_FENE, b=50.0, flow=I.FLOW_SHEAR, rate=1.0,
                 hi_a=1e-9)
    r_a, r_b = r.copy(), r.copy()
    O.em_step(base, 1e-3, r_a, xi)
    O.em_step(hi, 1e-3, r_b, xi)
    np.testing.assert_allclose(r_b, r_a, atol=1e-10)


@pytest.mark.slow
def test_three_beads_with_hi_keep_the_stationary_density():
    # as the collapsed-chain pin (kappa 50, u 2, rest 2, sigma 2), now with
    # hydrodynamic interaction: the dynamics change, exp(-U) does not
    kappa, u, R0, SIG = 50.0, 2.0, 2.0, 2.0

    def weight(r1, r2, c):
        r02 = math.sqrt(max(r1 * r1 + r2 * r2 - 2 * r1 * r2 * c, 1e-12))
        x = SIG / r02
        return r1 * r1 * r2 * r2 * math.exp(-0.5 * kappa * ((r1 - R0) ** 2 + (r2 - R0) ** 2)
                                            - u * (x ** 12 - 2 * x ** 6))

    lo, hi = R0 - 1.0, R0 + 1.0
    opts = dict(epsabs=1e-13, epsrel=1e-8)
    Z = integrate.tplquad(lambda c, r2, r1: weight(r1, r2, c), lo, hi, lo, hi, -1, 1, **opts)[0]
    mc = integrate.tplquad(lambda c, r2, r1: c * weight(r1, r2, c), lo, hi, lo, hi, -1, 1, **opts)[0] / Z
    mr = integrate.tplquad(lambda c, r2, r1: r1 * weight(r1, r2, c), lo, hi, lo, hi, -1, 1, **opts)[0] / Z
    R, dt, steps = 300, 2e-3, 40000
    chains = [I.Chain(n_beads=3, n_replicas=R, spring=I.SPRING_HARMONIC, H=kappa, r0=R0,
                      lj_u=u, lj_sigma=SIG, hi_a=1.0) for _ in range(16)]
    pos0 = np.zeros((48, 3))
    pos0[:, 2] = np.tile([0.0, 2.0, 4.0], 16)
    out = O.run(chains, dt, steps, steps, seed=17, pos0=pos0, thr_mask=0, bell_mask=0, n_threads=16)
    rep = out["rep"].reshape(16 * R, 3, 3)
    q1, q2 = rep[:, 1] - rep[:, 0], rep[:, 2] - rep[:, 1]
    n1, n2 = np.linalg.norm(q1, axis=1), np.linalg.norm(q2, axis=1)
    cos_bead = -(q1 * q2).sum(axis=1) / (n1 * n2)
    for est, want in ((cos_bead, mc), (n1, mr)):
        sd = est.std() / math.sqrt(est.size)
        assert abs(est.mean() - want) < 5 * sd + 0.005 * abs(want), (est.mean(), want, sd)
