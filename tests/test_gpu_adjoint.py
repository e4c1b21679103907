"""GPU adjoint (bd_adjoint and its torch.autograd.Function) against the FP64
oracle's pathwise tangent - the same Philox draws, the noise held fixed - and
against central finite differences of the GPU forward run with common random
numbers.

Objective: L = sum_{w,m} G[w][m] RSF_w[m] + sum_c g_c log S_c, with log S_c
the Bell log-survival of chain c under the RSF criterion. The oracle side is
sum_{w,m of c} (G[w][m] - g_c k0 dx exp(dx RSF_w[m]) S dt) dRSF_w[m]/dtheta_c.

Tolerances: FP64 1e-10 relative to the largest gradient of each parameter
(the two sides differentiate the same discrete map and differ by rounding
order only; measured 1e-14). FP32: the integration runs in float32, so the
gradient carries the float32 trajectory's deviation from the float64 one;
bound 1e-3 of the largest gradient (measured up to 1.2e-4 on the 256-chain
workload, 1e-5 on the small cases).
"""
import dataclasses

import numpy as np
import pytest

from oracle import oracle as O
from paper_2206_05851_gb300 import bdra
from paper_2206_05851_gb300 import inputs as I

pytestmark = pytest.mark.gpu

F64, F32 = bdra.BD_PREC_FP64, bdra.BD_PREC_FP32
PARAMS = ("rate", "b", "H")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    from paper_2206_05851_gb300 import build as B
    B.build()
    torch.cuda.init()


def _stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


def mixed_chains():
    """Adjoint replica tiles 4, 7 and 16 (N = 6, 150, 300, 2), forward parent
    tiles 2, 7 and 10, several replicas per warp with ragged groups, shear,
    uniaxial and planar flow, FENE and Hookean springs."""
    return [
        I.Chain(n_beads=6, n_replicas=40, spring=I.SPRING_FENE, flow=I.FLOW_UNIAXIAL, b=30.0,
                rate=0.4, H=1.1, k0=1e-3, dx=0.3),
        I.Chain(n_beads=150, n_replicas=3, spring=I.SPRING_FENE, flow=I.FLOW_SHEAR, b=50.0,
                rate=0.05, H=0.9, k0=1e-3, dx=0.2),
        I.Chain(n_beads=300, n_replicas=2, spring=I.SPRING_HOOKE, flow=I.FLOW_PLANAR, b=20.0,
                rate=0.01, H=1.3, k0=1e-3, dx=0.1),
        I.Chain(n_beads=2, n_replicas=5, spring=I.SPRING_FENE, flow=I.FLOW_UNIAXIAL, b=10.0,
                rate=0.5, H=1.0, k0=1e-2, dx=0.5),
    ]


def seeds(chains, W, seed):
    rng = np.random.default_rng(seed)
    M = sum(c.n_beads - 1 for c in chains)
    return rng.normal(size=(W, M)), rng.normal(size=len(chains))


def oracle_grad(chains, rsf, drsf, G, gls, dt, S):
    offs = I.spring_offsets(chains)
    out = np.zeros((len(chains), 3))
    for c, ch in enumerate(chains):
        sl = slice(offs[c], offs[c + 1])
        seed = G[:, sl].copy()
        if gls is not None:
            seed -= gls[c] * ch.k0 * ch.dx * np.exp(ch.dx * rsf[:, sl]) * S * dt
        for j in range(3):
            out[c, j] = float((seed * drsf[j][:, sl]).sum())
    return out


def gpu_forward(chains, dt, S, n, seed, pos0, prec, K, restart=None):
    ctx = bdra.Context(chains, dt, S, seed, pos0, precision=prec, max_windows=n // S + 1,
                       bell_mask=I.CRIT_RSF, stream=_stream(), checkpoint_steps=K)
    if restart is not None:
        t, pos = restart
        ctx.step(t)
        ctx.set_positions(pos, t)
        ctx.step(n - t)
    else:
        ctx.step(n)
    return ctx


def objective(ctx, G, gls, w_lo=0):
    W = ctx.info().windows_done
    rsf = np.array([ctx.replica_average(w) for w in range(W)]).reshape(W, ctx.M)
    _, ls = ctx.events()
    return float((G[w_lo:W] * rsf[w_lo:W]).sum() + (gls * ls[:, 2]).sum()), rsf


def assert_close(got, want, rtol, what=""):
    for j in range(3):
        scale = np.abs(want[:, j]).max()
        err = np.abs(got[:, j] - want[:, j]).max()
        assert err <= rtol * max(scale, 1e-300), \
            f"{what} {PARAMS[j]}: max err {err:.3e}, scale {scale:.3e}\n{got[:, j]}\n{want[:, j]}"


DT, S, SEED = 2e-3, 25, 11


@pytest.mark.parametrize("K,n", [(25, 100), (50, 100), (100, 100), (50, 110), (75, 175)])
def test_fp64_adjoint_matches_oracle_tangent(K, n):
    chains = mixed_chains()
    pos0 = I.initial_positions(I.custom(chains, DT, S, n), seed=21)
    W = n // S
    G, gls = seeds(chains, W, 1)
    rsf, drsf = O.rsf_tangent(chains, DT, S, W * S, SEED, pos0, n_threads=4)
    want = oracle_grad(chains, rsf, drsf, G, gls, DT, S)
    ctx = gpu_forward(chains, DT, S, n, SEED, pos0, F64, K)
    _, grsf = objective(ctx, G, gls)
    np.testing.assert_allclose(grsf, rsf, rtol=1e-10, atol=1e-12)
    got = ctx.adjoint(G, gls)
    ctx.close()
    assert_close(got, want, 1e-10, f"K={K} n={n}")
    assert np.all(got[2, 1] == 0.0)           # Hookean chain: b does not enter


def test_fp32_adjoint_matches_oracle_tangent():
    chains = mixed_chains()
    n, K = 100, 50
    pos0 = I.initial_positions(I.custom(chains, DT, S, n), seed=21)
    G, gls = seeds(chains, n // S, 2)
    rsf, drsf = O.rsf_tangent(chains, DT, S, n, SEED, pos0, n_threads=4)
    want = oracle_grad(chains, rsf, drsf, G, gls, DT, S)
    ctx = gpu_forward(chains, DT, S, n, SEED, pos0, F32, K)
    got = ctx.adjoint(G, gls)
    ctx.close()
    assert_close(got, want, 1e-3, "fp32")


def test_device_arrays_and_objective_parts():
    import torch
    chains = mixed_chains()
    n, K = 100, 50
    pos0 = I.initial_positions(I.custom(chains, DT, S, n), seed=22)
    G, gls = seeds(chains, n // S, 3)
    ctx = gpu_forward(chains, DT, S, n, SEED, pos0, F64, K)
    both = ctx.adjoint(G, gls)
    only_rsf = ctx.adjoint(G, None)
    only_ls = ctx.adjoint(None, gls)
    none = ctx.adjoint(None, None)
    dev = torch.empty((len(chains), 3), dtype=torch.float64, device="cuda")
    bdra.bd_adjoint(ctx.ptr, len(chains), ctx.M, n // S,
                    torch.from_numpy(G).cuda(), torch.from_numpy(gls).cuda(), dev)
    ctx.close()
    np.testing.assert_allclose(only_rsf + only_ls, both, rtol=1e-12, atol=1e-14 * np.abs(both).max())
    assert np.all(none == 0.0)
    np.testing.assert_allclose(dev.cpu().numpy(), both, rtol=1e-12, atol=1e-14 * np.abs(both).max())


@pytest.mark.parametrize("c,j", [(0, 0), (0, 1), (0, 2), (1, 0), (1, 2), (2, 0), (3, 1)])
def test_fp64_adjoint_matches_crn_finite_differences(c, j):
    """Central differences of the GPU forward run, h = 1e-4 relative, same
    seed (common random numbers)."""
    chains = mixed_chains()
    n, K = 100, 50
    pos0 = I.initial_positions(I.custom(chains, DT, S, n), seed=23)
    G, gls = seeds(chains, n // S, 4)
    ctx = gpu_forward(chains, DT, S, n, SEED, pos0, F64, K)
    g = ctx.adjoint(G, gls)[c, j]
    ctx.close()
    val = getattr(chains[c], PARAMS[j])
    h = 1e-4 * val
    L = []
    for sgn in (1, -1):
        cc = list(chains)
        cc[c] = dataclasses.replace(chains[c], **{PARAMS[j]: val + sgn * h})
        x = gpu_forward(cc, DT, S, n, SEED, pos0, F64, K)
        assert x.info().overextensions == 0
        L.append(objective(x, G, gls)[0])
        x.close()
    fd = (L[0] - L[1]) / (2 * h)
    assert abs(g - fd) <= 1e-6 * abs(fd) + 1e-12, (g, fd)


def test_restart_moves_the_origin():
    """After bd_set_positions(pos, t) the objective covers windows from t / S
    on, with the conformation at t held fixed: rows before are ignored and
    finite differences of the restarted run agree."""
    chains = mixed_chains()
    n, t, K = 200, 100, 50
    pos0 = I.initial_positions(I.custom(chains, DT, S, n), seed=24)
    pos1 = I.initial_positions(I.custom(chains, DT, S, n), seed=25)
    G, gls = seeds(chains, n // S, 5)
    ctx = gpu_forward(chains, DT, S, n, SEED, pos0, F64, K, restart=(t, pos1))
    g = ctx.adjoint(G, gls)
    G2 = G.copy()
    G2[: t // S] = 0.0
    np.testing.assert_allclose(ctx.adjoint(G2, gls), g, rtol=1e-13, atol=1e-15 * np.abs(g).max())
    ctx.close()
    c, j = 0, 0
    val = chains[c].rate
    h = 1e-4 * val
    L = []
    for sgn in (1, -1):
        cc = list(chains)
        cc[c] = dataclasses.replace(chains[c], rate=val + sgn * h)
        x = gpu_forward(cc, DT, S, n, SEED, pos0, F64, K, restart=(t, pos1))
        L.append(objective(x, G, gls, w_lo=t // S)[0])
        x.close()
    fd = (L[0] - L[1]) / (2 * h)
    assert abs(g[c, j] - fd) <= 1e-6 * abs(fd), (g[c, j], fd)


def test_no_complete_window_gives_zero_and_missing_checkpoints_is_a_state_error():
    chains = mixed_chains()[:2]
    pos0 = I.initial_positions(I.custom(chains, DT, S, 10), seed=26)
    ctx = gpu_forward(chains, DT, S, S - 1, SEED, pos0, F32, S)
    assert np.all(ctx.adjoint(None, np.ones(2)) == 0.0)
    ctx.close()
    ctx = gpu_forward(chains, DT, S, 2 * S, SEED, pos0, F32, 0)
    with pytest.raises(bdra.BdError) as e:
        ctx.adjoint(None, np.ones(2))
    assert e.value.status == bdra.BD_E_STATE
    ctx.close()


def test_autograd_function_backward_is_the_adjoint():
    import torch
    from paper_2206_05851_gb300.autograd import RunSpec, chain_params, replica_averaged_run
    chains = mixed_chains()
    n, K = 100, 50
    pos0 = I.initial_positions(I.custom(chains, DT, S, n), seed=27)
    G, gls = seeds(chains, n // S, 6)
    spec = RunSpec(chains, DT, S, n, SEED, pos0, K, precision=F64)
    params = chain_params(chains).requires_grad_(True)
    rsf, ls = replica_averaged_run(params, spec)
    assert rsf.shape == (n // S, sum(c.n_beads - 1 for c in chains)) and ls.shape == (4,)
    loss = (rsf * torch.from_numpy(G).to(rsf.device)).sum() + (ls * torch.from_numpy(gls).to(ls.device)).sum()
    loss.backward()
    r, dr = O.rsf_tangent(chains, DT, S, n, SEED, pos0, n_threads=4)
    np.testing.assert_allclose(rsf.detach().cpu().numpy(), r, rtol=1e-10, atol=1e-12)
    assert_close(params.grad.numpy(), oracle_grad(chains, r, dr, G, gls, DT, S), 1e-10, "autograd")
    # a loss on the RSF alone (no gradient reaches the survival output)
    params.grad = None
    rsf, ls = replica_averaged_run(params, spec)
    (rsf[:, 2].sum()).backward()
    G1 = np.zeros_like(G)
    G1[:, 2] = 1.0
    assert_close(params.grad.numpy(), oracle_grad(chains, r, dr, G1, None, DT, S), 1e-10, "rsf only")


def test_autograd_releases_device_memory():
    """Forward and backward through the autograd function twice, on chains
    shaped like the 256-chain adjoint workload (N = 200, 32 replicas,
    checkpoints every 1000 steps) but fewer: the device memory of the run's
    context (state, histories, checkpoints, the adjoint's replay buffers) is
    returned after each backward pass, and a second backward through a
    released graph raises instead of touching freed memory."""
    import gc
    import torch
    from paper_2206_05851_gb300.autograd import RunSpec, chain_params, release_run, replica_averaged_run
    wl = I.adjoint_256(n_steps=2000, n_chains=16)
    pos0 = I.initial_positions(wl)
    spec = RunSpec(wl.chains, wl.dt, wl.window_steps, wl.n_steps, wl.seed, pos0,
                   I.ADJOINT_CHECKPOINT_STEPS, precision=F32)

    def free_bytes():
        gc.collect()
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        return torch.cuda.mem_get_info()[0]

    base = free_bytes()
    grads = []
    for _ in range(2):
        params = chain_params(wl.chains).requires_grad_(True)
        rsf, ls = replica_averaged_run(params, spec)
        assert free_bytes() < base              # the context holds its buffers until backward
        loss = rsf[:, 99].sum() + ls.sum()
        loss.backward(retain_graph=True)
        grads.append(params.grad.clone())
        assert free_bytes() >= base - (16 << 20), "context not released by backward"
        with pytest.raises(RuntimeError, match="released"):
            loss.backward()
        del rsf, ls, loss
    # the float64 gradient partials meet in atomics: equal up to their order
    np.testing.assert_allclose(grads[0].numpy(), grads[1].numpy(), rtol=1e-12, atol=0)
    assert free_bytes() >= base - (16 << 20)
    # kept for a second backward on request; released early on request
    params = chain_params(wl.chains).requires_grad_(True)
    rsf, ls = replica_averaged_run(params, dataclasses.replace(spec, retain_run=True))
    rsf.sum().backward(retain_graph=True)
    g1 = params.grad.clone()
    params.grad = None
    rsf.sum().backward()
    np.testing.assert_allclose(params.grad.numpy(), g1.numpy(), rtol=1e-12, atol=0)
    release_run(rsf)
    assert free_bytes() >= base - (16 << 20)
    del rsf, ls


def test_adjoint_workload_full_size_sampled_chains():
    """256 FENE chains, N=200, 32 replicas, Wi=5, 2e4 steps, checkpoints every 1000
    steps, float32: the mid-chain RSF averaged over the windows plus the
    Bell log-survival; the gradients of two sampled chains against the FP64
    oracle's tangent of those chains (with their own noise streams)."""
    wl = I.adjoint_256()
    chains, S_, n = wl.chains, wl.window_steps, wl.n_steps
    pos0 = I.initial_positions(wl)
    W = n // S_
    offs = I.spring_offsets(chains)
    G = np.zeros((W, int(offs[-1])))
    for c, ch in enumerate(chains):
        G[:, offs[c] + (ch.n_beads - 1) // 2] = 1.0 / W
    gls = np.ones(len(chains))
    ctx = bdra.Context(chains, wl.dt, S_, wl.seed, pos0, precision=F32, max_windows=W,
                       bell_mask=I.CRIT_RSF, stream=_stream(),
                       checkpoint_steps=I.ADJOINT_CHECKPOINT_STEPS)
    ctx.step(n)
    got = ctx.adjoint(G, gls)
    ctx.close()
    assert np.all(np.isfinite(got))
    sample = [0, len(chains) - 1]
    sub = [chains[c] for c in sample]
    bo = I.bead_offsets(chains)
    p0 = np.concatenate([pos0[bo[c]:bo[c + 1]] for c in sample])
    r, dr = O.rsf_tangent(sub, wl.dt, S_, n, wl.seed, p0, n_threads=2, chain_ids=sample)
    so = I.spring_offsets(sub)
    Gs = np.concatenate([G[:, offs[c]:offs[c + 1]] for c in sample], axis=1)
    want = oracle_grad(sub, r, dr, Gs, gls[sample], wl.dt, S_)
    assert so[-1] == Gs.shape[1]
    assert_close(got[sample], want, 1e-3, "adjoint workload")
