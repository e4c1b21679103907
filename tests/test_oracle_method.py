"""Pins of the oracle's method: the RSF/TSF/ISF procedure of Sec. II, the
replica-average estimator and its 1/sqrt(N_R) spread (Sec. III), threshold and
Bell kinetics (Sec. I; Sec. III, vWF) and chain-reversal symmetry.
"""
import math

import numpy as np
import pytest
from scipy import integrate, stats

from oracle import oracle as O
from paper_2206_05851_gb300 import inputs as I


def _chain(n, R, spring=I.SPRING_FENE, flow=I.FLOW_NONE, rate=0.0, H=1.0, b=50.0,
           f_c=math.inf, k0=0.0, dx=0.0):
    return I.Chain(n_beads=n, n_replicas=R, spring=spring, flow=flow, H=H, b=b, rate=rate,
                   f_c=f_c, k0=k0, dx=dx)


def _brute_force(chains, dt, S, n_steps, seed, pos0, identical=False):
    """The procedure of Sec. II written out with the pinned primitives only:
    per window, replicas copied from the halted parent and evolved S steps
    (noise slot k), one force sample each at the end; then the parent
    continues S steps (slot 0) with a force sample per step."""
    out_rsf, out_tsf, isf = [], [], []
    parents, reps = [], []
    off = 0
    for c, ch in enumerate(chains):
        N, R = ch.n_beads, ch.n_replicas
        par = np.array(pos0[off:off + N], dtype=np.float64)
        off += N
        rep = [par.copy() for _ in range(R)]
        rs, ts, fi = [], [], []
        t = 0
        while t < n_steps:
            Sw = min(S, n_steps - t)
            for k in range(1, R + 1):
                rep[k - 1] = par.copy()
                for s in range(Sw):
                    xi = np.array([O.normals3(seed, i, 0 if identical else k, 0, t + s, c)
                                   for i in range(N)])
                    O.em_step(ch, dt, rep[k - 1], xi)
            if Sw == S:
                rs.append(np.mean([O.tensions(ch, rep[k]) for k in range(R)], axis=0))
            acc = np.zeros(N - 1)
            for s in range(Sw):
                xi = np.array([O.normals3(seed, i, 0, 0, t + s, c) for i in range(N)])
                O.em_step(ch, dt, par, xi)
                f = O.tensions(ch, par)
                acc += f
                fi.append(f)
            if Sw == S:
                ts.append(acc / S)
            t += Sw
        out_rsf.append(rs); out_tsf.append(ts); isf.append(fi)
        parents.append(par); reps.append(np.concatenate(rep))
    return dict(rsf=np.concatenate([np.array(x) for x in out_rsf], axis=1),
                tsf=np.concatenate([np.array(x) for x in out_tsf], axis=1),
                pos=np.concatenate(parents), rep=np.concatenate(reps), isf=isf)


def test_run_matches_procedure_written_out():
    chains = [_chain(3, 2, flow=I.FLOW_SHEAR, rate=0.8, b=20.0),
              _chain(4, 3, flow=I.FLOW_UNIAXIAL, rate=0.3, b=30.0)]
    pos0 = I.initial_positions(I.custom(chains, 0.01, 4, 14), seed=3)
    ref = _brute_force(chains, 0.01, 4, 14, 99, pos0)
    out = O.run(chains, 0.01, 4, 14, 99, pos0, thr_mask=0, bell_mask=0)
    np.testing.assert_array_equal(out["pos"], ref["pos"])
    np.testing.assert_array_equal(out["rep"], ref["rep"])
    np.testing.assert_allclose(out["rsf"], ref["rsf"], rtol=1e-15)
    np.testing.assert_allclose(out["tsf"], ref["tsf"], rtol=1e-14)


def test_identical_noise_replicas_reproduce_parent():
    ch = _chain(6, 16, flow=I.FLOW_PLANAR, rate=0.5, b=40.0)
    pos0 = I.initial_positions(I.custom([ch], 1e-3, 50, 100), seed=4)
    out = O.run([ch], 1e-3, 50, 100, 5, pos0, thr_mask=0, bell_mask=0, identical_noise=True)
    rep = out["rep"].reshape(16, 6, 3)
    for k in range(16):
        np.testing.assert_array_equal(rep[k], out["pos"])
    # RSF of the last window = ISF of the parent at its end (16 equal samples,
    # summed in sequence: equal up to the rounding of that sum).
    np.testing.assert_allclose(out["rsf"][-1], O.tensions(ch, out["pos"]), rtol=8e-16)


def test_rsf_mean_is_conditional_mean_force_hookean():
    # Given the parent q0, a replica's connector after S steps is Gaussian,
    # N(M^S q0, Sigma_S) (exact for Hookean springs under Euler), so
    # E[RSF_i] = E|H Q_i| under that law; evaluated here by Monte Carlo with
    # an independent generator.
    N, R, S, dt = 5, 4000, 40, 0.01
    ch = _chain(N, R, spring=I.SPRING_HOOKE, flow=I.FLOW_SHEAR, rate=1.0)
    rng = np.random.default_rng(8)
    pos0 = np.cumsum(rng.normal(size=(N, 3)), axis=0)
    out = O.run([ch], dt, S, S, 77, pos0, thr_mask=0, bell_mask=0, n_threads=8)
    A = 2 * np.eye(N - 1) - np.eye(N - 1, k=1) - np.eye(N - 1, k=-1)
    kap = O.flow_gradient(I.FLOW_SHEAR, 1.0)
    M = np.kron(np.eye(N - 1), np.eye(3) + dt * kap) - dt / 4 * np.kron(A, np.eye(3))
    Cn = dt / 2 * np.kron(A, np.eye(3))
    mu = np.linalg.matrix_power(M, S) @ np.diff(pos0, axis=0).reshape(-1)
    Sig = np.zeros_like(M)
    for _ in range(S):
        Sig = M @ Sig @ M.T + Cn
    draws = rng.multivariate_normal(mu, Sig, size=400_000).reshape(-1, N - 1, 3)
    f = np.linalg.norm(draws, axis=2)
    expect, sd = f.mean(axis=0), f.std(axis=0)
    assert np.all(np.abs(out["rsf"][0] - expect) < 5 * sd / math.sqrt(R) + 1e-3 * expect)


def test_rsf_spread_scales_as_inverse_sqrt_replicas():
    # Sec. III: sigma(RSF) ~ N_R^(-1/2). Same parent, independent seeds.
    N, S, dt = 6, 30, 1e-3
    pos0 = I.initial_positions(I.custom([_chain(N, 1)], dt, S, S), seed=9)
    vals = {}
    for R in (10, 40):
        ch = _chain(N, R, b=30.0, flow=I.FLOW_UNIAXIAL, rate=0.2)
        vals[R] = np.array([O.run([ch], dt, S, S, 1000 + s, pos0, thr_mask=0, bell_mask=0)
                            ["rsf"][0] for s in range(120)])
    ratio = vals[10].std(axis=0) / vals[40].std(axis=0)
    assert np.all(np.abs(ratio - 2.0) < 0.5)
    # averaging does not move the mean (Sec. III, Fig. 1 discussion)
    se = np.sqrt(vals[10].var(axis=0) / 120 + vals[40].var(axis=0) / 120)
    assert np.all(np.abs(vals[10].mean(axis=0) - vals[40].mean(axis=0)) < 5 * se)


def test_threshold_events_recount_from_window_profiles():
    b = 30.0
    chains = [_chain(8, 8, b=b, flow=I.FLOW_UNIAXIAL, rate=1.2, f_c=0.6 * math.sqrt(b)),
              _chain(5, 4, b=b, flow=I.FLOW_SHEAR, rate=4.0, f_c=0.5 * math.sqrt(b))]
    S, n, dt = 20, 2000, 2e-3
    pos0 = I.initial_positions(I.custom(chains, dt, S, n), seed=11)
    out = O.run(chains, dt, S, n, 12, pos0, thr_mask=7, bell_mask=0)
    fc = np.concatenate([[c.f_c] * (c.n_beads - 1) for c in chains])
    for q, key in ((O.RSF, "rsf"), (O.TSF, "tsf")):
        prof = out[key]
        hit = prof >= fc[None, :]
        expect = np.where(hit.any(axis=0), (hit.argmax(axis=0) + 1) * S, -1)
        np.testing.assert_array_equal(out["first_thr"][q], expect)
    assert (out["first_thr"][O.RSF] >= 0).sum() > 0        # the case has events
    # ISF: at its first-event step the parent's spring force reaches f_c, and
    # a run stopped one step earlier has not yet seen it.
    m = int(np.argmax(out["first_thr"][O.ISF] >= 0))
    t_star = int(out["first_thr"][O.ISF][m])
    c = 0 if m < 7 else 1
    i = m if c == 0 else m - 7
    at = O.run(chains, dt, S, t_star, 12, pos0, thr_mask=7, bell_mask=0)
    before = O.run(chains, dt, S, t_star - 1, 12, pos0, thr_mask=7, bell_mask=0)
    off = 0 if c == 0 else 8
    f_at = O.tensions(chains[c], at["pos"][off:off + chains[c].n_beads])
    assert f_at[i] >= chains[c].f_c
    assert before["first_thr"][O.ISF][m] == -1


def test_bell_constant_force_survival_closed_form():
    # Constant force f: hazard k = k0 exp(f dx); integrated hazard after n
    # windows of length dT is n k dT and the survival is exp(-k t) (Bell 1978).
    ch = _chain(2, 1, k0=1e-3, dx=0.7)
    f, dT, E = 3.0, 0.5, 0.9
    k = 1e-3 * math.exp(3.0 * 0.7)
    st = dict(lam=0.0, first_thr=-1, first_bell=-1)
    for w in range(1, 300):
        O.criteria_update(O.RSF, False, True, ch, f, dT, w * 100, E, st)
        assert st["lam"] == pytest.approx(w * k * dT, rel=1e-12)
        assert math.exp(-st["lam"]) == pytest.approx(math.exp(-k * w * dT), rel=1e-12)
    n_star = math.ceil(E / (k * dT))
    assert st["first_bell"] == n_star * 100


def test_bell_isf_hazard_at_equilibrium_matches_quadrature():
    # Hookean dumbbell at rest. Its Euler map Q' = (1 - dt/2) Q + sqrt(dt) eta
    # has the exact stationary law N(0, s2 I), s2 = 1/(1 - dt/4), so the ISF
    # hazard rate is k0 E[exp(dx s chi_3)] (1D quadrature). (For a FENE
    # spring this mean diverges: f grows without bound at full extension.)
    dx, k0, dt = 1.0, 1e-2, 5e-3
    s = 1.0 / math.sqrt(1.0 - dt / 4.0)
    chi = stats.chi(3)
    rate = k0 * integrate.quad(lambda r: math.exp(dx * s * r) * chi.pdf(r), 0, 40)[0]
    C, n = 400, 20000
    chains = [_chain(2, 1, spring=I.SPRING_HOOKE, k0=k0, dx=dx) for _ in range(C)]
    rng = np.random.default_rng(13)
    pos0 = np.concatenate([[[0.0, 0.0, 0.0], list(rng.normal(scale=s, size=3))]
                           for _ in range(C)])
    out = O.run(chains, dt, 100, n, 14, pos0, thr_mask=0, bell_mask=1, n_threads=8,
                want_replicas=False)
    per_chain = out["lam"][O.ISF] / (n * dt)
    est, sd = per_chain.mean(), per_chain.std() / math.sqrt(C)
    assert abs(est - rate) < 5 * sd + 2e-3 * rate


def test_jensen_ordering_of_hazards():
    # Averaging before the convex rate law lowers the hazard: ISF >= RSF, and
    # ISF >= TSF (the ordering of Table 1).
    b = 50.0
    fmax = math.sqrt(b)
    chains = [_chain(10, 16, b=b, flow=I.FLOW_UNIAXIAL, rate=0.02, k0=1e-6, dx=20.0 / fmax)
              for _ in range(8)]
    pos0 = I.initial_positions(I.custom(chains, 1e-3, 20, 2000), seed=15)
    out = O.run(chains, 1e-3, 20, 2000, 16, pos0, thr_mask=0, bell_mask=7, n_threads=8,
                want_replicas=False)
    lam = out["lam"].sum(axis=1)
    assert lam[O.ISF] > lam[O.RSF] and lam[O.ISF] > lam[O.TSF]


def test_mean_tension_profile_end_to_end_symmetry():
    # Reversing bead order maps the free-draining chain in any of the flows
    # onto itself, so <f_i> = <f_{N-2-i}>.
    N, C = 8, 64
    chains = [_chain(N, 4, b=40.0, flow=I.FLOW_PLANAR, rate=0.15) for _ in range(C)]
    pos0 = I.initial_positions(I.custom(chains, 2e-3, 50, 6000), seed=17)
    out = O.run(chains, 2e-3, 50, 6000, 18, pos0, thr_mask=0, bell_mask=0, n_threads=8,
                want_replicas=False)
    prof = out["rsf"][20:].reshape(-1, C, N - 1).mean(axis=0)     # per-chain window means
    d = prof - prof[:, ::-1]
    se = d.std(axis=0) / math.sqrt(C)
    assert np.all(np.abs(d.mean(axis=0)) < 5 * se + 1e-9)
    # the profile is not flat: the middle spring carries more than the ends
    m = prof.mean(axis=0)
    assert m[(N - 1) // 2] > m[0]
