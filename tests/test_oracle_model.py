"""Pins of the oracle's model: spring laws, flows and the Eq. 1 update.

Each check compares the oracle with something the physics fixes, computed
here independently: potentials differentiated numerically, the exact linear
(Rouse) map of a Hookean chain under Euler-Maruyama, its exact mean and
covariance after n steps, the FENE equilibrium law, and the stationary FENE
dumbbell density in a potential flow evaluated by quadrature, and the
stationary three-bead density in the same flow by importance sampling.
"""
import math

import numpy as np
import pytest
from scipy import integrate, linalg, stats

from oracle import oracle as O
from paper_2206_05851_gb300 import inputs as I


def _fene_potential(Q, H, b):
    return -0.5 * b * math.log(1.0 - H * float(np.dot(Q, Q)) / b)


@pytest.mark.parametrize("H,b", [(1.0, 50.0), (1.7, 20.0), (0.6, 200.0)])
def test_fene_force_is_gradient_of_potential(H, b):
    rng = np.random.default_rng(0)
    for _ in range(20):
        Q = rng.normal(size=3)
        Q *= rng.uniform(0.05, 0.9) * math.sqrt(b / H) / np.linalg.norm(Q)
        F, f, fl = O.spring_force(I.SPRING_FENE, H, b, Q)
        h = 1e-6
        grad = np.array([(_fene_potential(Q + h * e, H, b) - _fene_potential(Q - h * e, H, b))
                         / (2 * h) for e in np.eye(3)])
        assert fl == 0
        np.testing.assert_allclose(F, grad, rtol=1e-6, atol=1e-6 * np.linalg.norm(grad))
        assert f == pytest.approx(np.linalg.norm(grad), rel=1e-6)


def test_hooke_force_is_gradient_of_quadratic_potential():
    Q = np.array([0.3, -1.2, 2.0])
    F, f, _ = O.spring_force(I.SPRING_HOOKE, 2.5, 1.0, Q)
    h = 1e-6
    U = lambda q: 0.5 * 2.5 * float(np.dot(q, q))
    grad = np.array([(U(Q + h * e) - U(Q - h * e)) / (2 * h) for e in np.eye(3)])
    np.testing.assert_allclose(F, grad, rtol=1e-8)


def test_fene_small_extension_limit_is_hookean():
    Q = np.array([1e-4, -2e-4, 3e-4])
    F, _, _ = O.spring_force(I.SPRING_FENE, 1.3, 80.0, Q)
    Fh, _, _ = O.spring_force(I.SPRING_HOOKE, 1.3, 80.0, Q)
    np.testing.assert_allclose(F, Fh, rtol=1e-8)


def test_fene_floor_applies_past_full_extension():
    b = 10.0
    Q = np.array([math.sqrt(b) * 1.01, 0.0, 0.0])
    F, f, fl = O.spring_force(I.SPRING_FENE, 1.0, b, Q, s_min=1e-3)
    assert fl == 1
    assert F[0] == pytest.approx(Q[0] / 1e-3)
    assert f == pytest.approx(Q[0] / 1e-3)


def test_flow_gradients():
    # Sec. II: shear v = gdot z x_hat (x streamwise, z gradient direction).
    k = O.flow_gradient(I.FLOW_SHEAR, 2.0)
    np.testing.assert_array_equal(k @ np.array([0.0, 0.0, 1.0]), [2.0, 0.0, 0.0])
    np.testing.assert_array_equal(k @ np.array([1.0, 1.0, 0.0]), [0.0, 0.0, 0.0])
    for flow in (I.FLOW_UNIAXIAL, I.FLOW_PLANAR, I.FLOW_SHEAR, I.FLOW_NONE):
        assert np.trace(O.flow_gradient(flow, 0.7)) == pytest.approx(0.0)   # incompressible
    ku = O.flow_gradient(I.FLOW_UNIAXIAL, 0.7)
    assert np.allclose(ku, ku.T) and ku[0, 0] == pytest.approx(0.7)
    assert ku[1, 1] == pytest.approx(ku[2, 2])                               # axisymmetric
    kp = O.flow_gradient(I.FLOW_PLANAR, 0.7)
    assert kp[0, 0] == pytest.approx(0.7) and kp[1, 1] == pytest.approx(-0.7)
    assert kp[2, 2] == 0.0                                                   # neutral axis


def _chain(n, spring=I.SPRING_HOOKE, flow=I.FLOW_NONE, rate=0.0, H=1.0, b=50.0, R=1):
    return I.Chain(n_beads=n, n_replicas=R, spring=spring, flow=flow, H=H, b=b, rate=rate)


def test_free_bead_noise_amplitude():
    # No spring (H = 0) and no flow: Eq. 1 reduces to r' = r + R with
    # <R R> = 2 D dt and D = kT/zeta = 1/4 in Hookean units.
    ch = _chain(2, H=0.0)
    r = np.array([[0.1, 0.2, 0.3], [1.0, -1.0, 0.5]])
    xi = np.array([[1.0, -2.0, 0.5], [0.25, 3.0, -1.0]])
    r0 = r.copy()
    O.em_step(ch, 0.02, r, xi)
    np.testing.assert_allclose(r - r0, math.sqrt(2 * 0.25 * 0.02) * xi, rtol=1e-13)


def test_shear_advection_direction():
    ch = _chain(2, H=0.0, flow=I.FLOW_SHEAR, rate=3.0)
    r = np.array([[0.0, 0.0, 2.0], [0.0, 0.0, -1.0]])
    O.em_step(ch, 0.01, r, np.zeros((2, 3)))
    np.testing.assert_allclose(r, [[0.06, 0.0, 2.0], [-0.03, 0.0, -1.0]], rtol=1e-14)


def _rouse(n_springs):
    return 2 * np.eye(n_springs) - np.eye(n_springs, k=1) - np.eye(n_springs, k=-1)


def test_zero_noise_rouse_modes_decay_exactly():
    # Hookean chain, no flow, no noise: the connectors obey Q' = (I - dt/4 A) Q
    # with A the Rouse matrix; mode j decays by (1 - dt a_j / 4) per step,
    # a_j = 4 sin^2(j pi / (2N)).
    N, dt, n = 9, 0.05, 60
    ch = _chain(N)
    A = _rouse(N - 1)
    lam, V = np.linalg.eigh(A)
    np.testing.assert_allclose(np.sort(lam),
                               4 * np.sin(np.arange(1, N) * np.pi / (2 * N)) ** 2, atol=1e-12)
    rng = np.random.default_rng(1)
    r = rng.normal(size=(N, 3))
    amp0 = V.T @ np.diff(r, axis=0)
    for _ in range(n):
        O.em_step(ch, dt, r, np.zeros((N, 3)))
    amp = V.T @ np.diff(r, axis=0)
    np.testing.assert_allclose(amp, ((1 - dt * lam / 4) ** n)[:, None] * amp0, rtol=1e-10,
                               atol=1e-12)


def test_zero_noise_no_flow_conserves_centre_of_mass():
    ch = _chain(7, spring=I.SPRING_FENE, b=30.0)
    rng = np.random.default_rng(2)
    r = np.cumsum(rng.normal(scale=0.8, size=(7, 3)), axis=0)
    c0 = r.mean(axis=0)
    for _ in range(50):
        O.em_step(ch, 0.01, r, np.zeros((7, 3)))
    np.testing.assert_allclose(r.mean(axis=0), c0, atol=1e-12)


def _bond_map(N, dt, kappa):
    """Exact one-step map of the Hookean connectors (3(N-1) vector, spring-major):
    Q' = M Q + sqrt(dt/2) B xi with B B^T = A (x) I3."""
    A = _rouse(N - 1)
    M = np.kron(np.eye(N - 1), np.eye(3) + dt * kappa) - (dt / 4.0) * np.kron(A, np.eye(3))
    Cn = (dt / 2.0) * np.kron(A, np.eye(3))
    return M, Cn


@pytest.mark.parametrize("flow,rate", [(I.FLOW_SHEAR, 1.5), (I.FLOW_UNIAXIAL, 0.2),
                                       (I.FLOW_PLANAR, 0.3)])
def test_hookean_replica_ensemble_matches_exact_gaussian(flow, rate):
    # Replicas spawned from one parent and evolved n steps are iid draws of
    # the Euler map started there; for Hookean springs that law is Gaussian
    # with mean M^n q0 and covariance Sigma_n = M Sigma_{n-1} M^T + Cn.
    N, R, n, dt = 4, 3000, 150, 0.01
    ch = _chain(N, flow=flow, rate=rate, R=R)
    rng = np.random.default_rng(5)
    pos0 = np.cumsum(rng.normal(size=(N, 3)), axis=0)
    out = O.run([ch], dt, n, n, seed=17, pos0=pos0, thr_mask=0, bell_mask=0, n_threads=8)
    rep = out["rep"].reshape(R, N, 3)
    Q = np.diff(rep, axis=1).reshape(R, -1)
    M, Cn = _bond_map(N, dt, O.flow_gradient(flow, rate))
    mu = np.linalg.matrix_power(M, n) @ np.diff(pos0, axis=0).reshape(-1)
    Sig = np.zeros_like(M)
    for _ in range(n):
        Sig = M @ Sig @ M.T + Cn
    sd = np.sqrt(np.diag(Sig))
    assert np.all(np.abs(Q.mean(axis=0) - mu) < 5 * sd / math.sqrt(R))
    emp = np.cov(Q.T)
    tol = 5 * np.sqrt((Sig ** 2 + np.outer(np.diag(Sig), np.diag(Sig))) / R)
    assert np.all(np.abs(emp - Sig) < tol)


def test_hookean_stationary_covariance_is_discrete_lyapunov():
    # Long evolution: the connector covariance of the Euler scheme is the
    # solution of Sigma = M Sigma M^T + Cn (continuum limit: <Q^2> = 3/H).
    N, R, dt = 3, 3000, 0.05
    n = 800                                       # 40 lambda_H >> lambda_1 = 4/3
    ch = _chain(N, R=R)
    out = O.run([ch], dt, n, n, seed=23, pos0=np.zeros((N, 3)), thr_mask=0, bell_mask=0,
                n_threads=8)
    Q = np.diff(out["rep"].reshape(R, N, 3), axis=1).reshape(R, -1)
    M, Cn = _bond_map(N, dt, np.zeros((3, 3)))
    Sig = linalg.solve_discrete_lyapunov(M, Cn)
    np.testing.assert_allclose(np.cov(Q.T), Sig, atol=5 * math.sqrt(2.0 / R) * Sig.max())
    q2 = (Q.reshape(R, N - 1, 3) ** 2).sum(axis=2).mean(axis=0)
    np.testing.assert_allclose(q2, 3.0, rtol=0.05)


@pytest.mark.parametrize("b", [10.0, 50.0])
def test_fene_equilibrium_spring_length(b):
    # Free-draining FENE springs at equilibrium are independent with
    # p(Q) ~ Q^2 (1 - Q^2/b)^(b/2): Q^2/b ~ Beta(3/2, b/2 + 1), <Q^2> = 3b/(b+5).
    R, dt, n = 3000, 5e-3, 2400
    ch = _chain(2, spring=I.SPRING_FENE, b=b, R=R)
    pos0 = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0]])
    out = O.run([ch], dt, n, n, seed=29, pos0=pos0, thr_mask=0, bell_mask=0, n_threads=8)
    Q = np.diff(out["rep"].reshape(R, 2, 3), axis=1).reshape(R, 3)
    x = (Q ** 2).sum(axis=1) / b
    mean = 3.0 / (b + 5.0)
    sd = math.sqrt(stats.beta(1.5, b / 2 + 1).var() / R)
    assert abs(x.mean() - mean) < 5 * sd + 0.01 * mean        # + Euler O(dt) bias
    assert stats.kstest(x, stats.beta(1.5, b / 2 + 1).cdf).pvalue > 1e-4
    assert out["overext"][0] == 0


def test_fene_dumbbell_in_uniaxial_flow_matches_quadrature():
    # Dumbbell in a potential flow: the stationary connector density is
    # psi ~ (1 - Q^2/b)^(b/2) exp(Q . kappa . Q) (Fokker-Planck with drift
    # kappa Q - F/2 and diffusivity 1/2). Axisymmetric quadrature of <Qx^2>.
    b, eps = 20.0, 0.3
    w = lambda qx, rho: (1 - (qx * qx + rho * rho) / b) ** (b / 2) * \
        math.exp(eps * (qx * qx - 0.5 * rho * rho)) * rho
    lim = math.sqrt(b)
    hi = lambda qx: math.sqrt(max(b - qx * qx, 0.0))
    Z = integrate.dblquad(lambda rho, qx: w(qx, rho), -lim, lim, 0.0, hi)[0]
    qx2 = integrate.dblquad(lambda rho, qx: qx * qx * w(qx, rho), -lim, lim, 0.0, hi)[0] / Z
    R, dt, n = 4000, 2e-3, 6000
    ch = _chain(2, spring=I.SPRING_FENE, b=b, flow=I.FLOW_UNIAXIAL, rate=eps, R=R)
    out = O.run([ch], dt, n, n, seed=31, pos0=np.zeros((2, 3)), thr_mask=0, bell_mask=0,
                n_threads=8)
    Q = np.diff(out["rep"].reshape(R, 2, 3), axis=1).reshape(R, 3)
    est = (Q[:, 0] ** 2).mean()
    sd = (Q[:, 0] ** 2).std() / math.sqrt(R)
    assert abs(est - qx2) < 5 * sd + 0.01 * qx2
    assert qx2 > 1.3          # the flow really stretches the dumbbell here


def test_fene_three_bead_chain_in_uniaxial_flow_matches_stationary_density():
    # Three free-draining beads in a potential flow: with bead diffusivity
    # 1/4 the stationary density of the internal coordinates is
    # exp(-U + 2 sum_i r_i . kappa . r_i) in the centre-of-mass frame, which
    # for bonds Q1, Q2 is p0(Q1) p0(Q2) exp(4/3 (Q1.k.Q1 + Q2.k.Q2 + Q1.k.Q2))
    # with p0 the FENE equilibrium density. Its moments by importance
    # sampling from p0 (exact rejection sampler) against a long ensemble run.
    b, eps = 20.0, 0.1
    rng = np.random.default_rng(11)
    n = 400_000
    q1 = I.sample_connectors(rng, n, I.SPRING_FENE, 1.0, b)
    q2 = I.sample_connectors(rng, n, I.SPRING_FENE, 1.0, b)
    kq = lambda a, c: eps * (a[:, 0] * c[:, 0] - 0.5 * a[:, 1] * c[:, 1] - 0.5 * a[:, 2] * c[:, 2])
    logw = (4.0 / 3.0) * (kq(q1, q1) + kq(q2, q2) + kq(q1, q2))
    w = np.exp(logw - logw.max())
    w /= w.sum()
    want_xx = float(np.sum(w * 0.5 * (q1[:, 0] ** 2 + q2[:, 0] ** 2)))
    want_x12 = float(np.sum(w * q1[:, 0] * q2[:, 0]))
    # the oracle: 8 chains x 1000 independent replicas, one window of n steps from a straight start
    R, dt, steps = 1000, 2e-3, 15000
    chains = [_chain(3, spring=I.SPRING_FENE, b=b, flow=I.FLOW_UNIAXIAL, rate=eps, R=R)
              for _ in range(8)]
    out = O.run(chains, dt, steps, steps, seed=33, pos0=np.zeros((24, 3)), thr_mask=0,
                bell_mask=0, n_threads=8)
    Q = np.diff(out["rep"].reshape(8 * R, 3, 3), axis=1)          # [replica][bond][3]
    # (halving the cross term of the density would move <Q1x Q2x> by about six standard errors)
    xx = 0.5 * (Q[:, 0, 0] ** 2 + Q[:, 1, 0] ** 2)
    x12 = Q[:, 0, 0] * Q[:, 1, 0]
    for est, want in ((xx, want_xx), (x12, want_x12)):
        sd = est.std() / math.sqrt(est.size)
        assert abs(est.mean() - want) < 5 * sd + 0.02 * abs(want), (est.mean(), want, sd)
    assert want_x12 > 0.1        # the flow couples the two bonds
