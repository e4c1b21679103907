"""Pins of the oracle's conformation diagnostics of Eq. 5 (Sec. III): the
bead-mean |COM-frame position difference| between a replica after the
evolution time and the halted parent it was formed from, its per-bead form,
and the z contribution to the parent's radius of gyration.

- A straight chain along z: R_GZ = a sqrt((N^2 - 1) / 12) exactly.
- Two beads: the COM-frame positions are -Q/2 and +Q/2, so every per-bead
  difference and the bead mean equal |Q_rep - Q_parent| / 2 per component.
- Hookean springs, no flow: a replica's bonds after n Euler steps are
  Gaussian with mean M^n q0 and covariance Sigma_n (exact recursion), so
  each COM-frame bead displacement is Gaussian with known mean mu and
  standard deviation s, and E|X| = s sqrt(2/pi) exp(-mu^2 / 2 s^2)
  + mu (1 - 2 Phi(-mu / s)); the replica mean of the per-bead difference
  must match it.
"""
import math

import numpy as np
from scipy import stats

from oracle import oracle as O
from paper_2206_05851_gb300 import inputs as I


def test_rgz_of_a_straight_chain_along_z():
    N, a = 9, 0.7
    ch = I.Chain(n_beads=N, n_replicas=2, spring=I.SPRING_HOOKE)
    pos0 = np.zeros((N, 3))
    pos0[:, 2] = a * np.arange(N)
    pos0[:, 0] = 3.0                  # a translation changes nothing
    _, _, rgz = O.conformation([ch], 1e-3, 5, 10, 1, pos0)
    assert abs(rgz[0, 0] - a * math.sqrt((N * N - 1) / 12.0)) < 1e-14
    assert rgz[1, 0] > 0


def test_two_beads_reduce_to_half_the_bond_change():
    ch = I.Chain(n_beads=2, n_replicas=5, spring=I.SPRING_FENE, b=20.0, flow=I.FLOW_SHEAR, rate=1.0)
    pos0 = np.array([[0.3, -0.2, 1.0], [1.2, 0.4, 0.1]])
    S = 40
    dbar, dbead, _ = O.conformation([ch], 2e-3, S, S, 9, pos0)
    run = O.run([ch], 2e-3, S, S, 9, pos0, thr_mask=0, bell_mask=0)
    Qrep = np.diff(run["rep"].reshape(5, 2, 3), axis=1)[:, 0, :]
    half = np.abs(Qrep - (pos0[1] - pos0[0])) / 2
    np.testing.assert_allclose(dbar[0], half, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(dbead[0, 0], half.mean(axis=0), rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(dbead[0, 1], half.mean(axis=0), rtol=1e-13, atol=1e-15)


def test_hookean_per_bead_difference_matches_exact_gaussian_expectation():
    N, R, n, dt = 5, 4000, 60, 0.01
    ch = I.Chain(n_beads=N, n_replicas=R, spring=I.SPRING_HOOKE)
    rng = np.random.default_rng(3)
    pos0 = np.cumsum(rng.normal(size=(N, 3)), axis=0)
    _, dbead, _ = O.conformation([ch], dt, n, n, 21, pos0, n_threads=4)
    # exact one-step map of the bonds (one Cartesian component; no flow, so
    # the three components are independent and identically structured)
    A = 2 * np.eye(N - 1) - np.eye(N - 1, k=1) - np.eye(N - 1, k=-1)
    Mst = np.eye(N - 1) - (dt / 4.0) * A
    Cn = (dt / 2.0) * A
    Sig = np.zeros((N - 1, N - 1))
    for _ in range(n):
        Sig = Mst @ Sig @ Mst.T + Cn
    # bonds -> COM-frame bead positions: r_i = sum_{m<i} Q_m, minus the mean
    B = np.tril(np.ones((N, N - 1)), k=-1)
    B = B - B.mean(axis=0)
    Mn = np.linalg.matrix_power(Mst, n)
    q0 = np.diff(pos0, axis=0)                        # [N-1][3]
    for j in range(3):
        mu = B @ ((Mn - np.eye(N - 1)) @ q0[:, j])
        s = np.sqrt(np.diag(B @ Sig @ B.T))
        e_abs = s * math.sqrt(2 / math.pi) * np.exp(-mu ** 2 / (2 * s ** 2)) \
            + mu * (1 - 2 * stats.norm.cdf(-mu / s))
        var_abs = mu ** 2 + s ** 2 - e_abs ** 2
        np.testing.assert_array_less(np.abs(dbead[0, :, j] - e_abs), 5 * np.sqrt(var_abs / R))
