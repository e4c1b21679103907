"""Seeded synthetic inputs for replica-averaged Brownian dynamics.

This module is shared by the CUDA path, the tests and the benchmark. It
holds no part of the method's arithmetic (no integrator, no spring force, no
noise stream, no sampling or kinetics): it only draws initial chain
conformations and builds the per-chain parameter tables of the workloads.

Units are Hookean ones: length l_H = sqrt(kT/H0), time lambda_H = zeta/(4 H0),
force kT/l_H, kT = 1. A spring's dimensionless stiffness ``H`` is its spring
constant in units of H0 (1 by default), and the FENE extensibility is
b = H Q0^2 / kT.

Workload shapes follow the configurations the replica-averaging method is
benchmarked on: free-draining FENE chains under uniaxial / planar elongation
and steady shear, tens of replicas per chain, re-spawned every window of
100 steps (Sec. II of the paper describes the replica procedure; the FENE
spring is named in its supplementary vWF model, Table S1). The paper's own
model is here too, in units of the bead radius a (see COLLAPSED_DT): the
collapsed chain (harmonic springs with rest length 2a, Lennard-Jones
cohesion), with RPY hydrodynamic interaction, and the coarse-grained vWF
chain of Table S1; its starting conformations are compact globules.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

SPRING_HOOKE = 0
SPRING_FENE = 1
SPRING_HARMONIC = 2     # harmonic with a rest length r0 (the paper's collapsed-chain springs)
SPRING_VWF = 3          # vWF: A2 domains (FENE || harmonic) alternating with disulfide bonds

FLOW_NONE = 0
FLOW_SHEAR = 1
FLOW_UNIAXIAL = 2
FLOW_PLANAR = 3

CRIT_ISF = 1
CRIT_TSF = 2
CRIT_RSF = 4
CRIT_ALL = CRIT_ISF | CRIT_TSF | CRIT_RSF


@dataclasses.dataclass
class Chain:
    """Parameters of one parent chain and its replica set."""

    n_beads: int
    n_replicas: int
    spring: int = SPRING_FENE
    flow: int = FLOW_NONE
    H: float = 1.0
    b: float = 50.0
    rate: float = 0.0      # strain rate (elongation) or shear rate, 1/lambda_H
    f_c: float = math.inf  # threshold-rupture force
    k0: float = 0.0        # Bell zero-force rate, 1/lambda_H
    dx: float = 0.0        # Bell distance to transition state, l_H
    r0: float = 0.0        # rest length of SPRING_HARMONIC
    lj_u: float = 0.0      # Lennard-Jones depth between non-adjacent beads (0: none)
    lj_sigma: float = 0.0  # Lennard-Jones zero-force (minimum) distance
    hi_a: float = 0.0      # bead radius of the RPY hydrodynamic interaction (0: free draining)
    vwf_fa: float = 0.0    # SPRING_VWF A2 domain: FENE spring constant
    vwf_fb: float = 0.0    # SPRING_VWF A2 domain: harmonic spring constant
    vwf_xmax: float = 0.0  # SPRING_VWF A2 domain: FENE maximum extension beyond r0


@dataclasses.dataclass
class Workload:
    """A complete problem: chains, integration settings and criteria."""

    name: str
    chains: List[Chain]
    dt: float
    window_steps: int
    n_steps: int
    seed: int
    thr_mask: int = CRIT_RSF
    bell_mask: int = 0
    init_seed: int = 12345

    @property
    def n_chains(self) -> int:
        return len(self.chains)

    def bead_steps(self, n_steps: Optional[int] = None) -> int:
        """chains x replicas x beads x steps (parent chain not counted)."""
        n = self.n_steps if n_steps is None else n_steps
        return sum(c.n_replicas * c.n_beads for c in self.chains) * n


def rouse_longest_time(n_beads: int) -> float:
    """Longest Rouse relaxation time of an N-bead Hookean chain, in lambda_H.

    lambda_1 = 1 / (2 sin^2(pi / (2N))); the dumbbell (N = 2) gives 1.
    """
    return 1.0 / (2.0 * math.sin(math.pi / (2.0 * n_beads)) ** 2)


def rate_from_wi(wi: float, n_beads: int) -> float:
    """Flow rate (1/lambda_H) for Weissenberg number Wi = rate * lambda_1."""
    return wi / rouse_longest_time(n_beads)


def fene_fmax(H: float, b: float) -> float:
    """FENE force scale F_max = H Q0 = sqrt(H b) (kT = 1)."""
    return math.sqrt(H * b)


def sample_connectors(rng: np.random.Generator, n: int, spring: int,
                      H: float, b: float) -> np.ndarray:
    """n iid connector vectors from the equilibrium spring density.

    Hookean: Q ~ N(0, I/H). FENE: p(Q) ~ (1 - H Q^2/b)^(b/2) on |Q| < sqrt(b/H),
    drawn by rejection from N(0, I/H) (the ratio of the two densities,
    (1 - x)^(b/2) e^(b x / 2) with x = H Q^2 / b, never exceeds 1).
    """
    out = np.empty((n, 3))
    filled = 0
    sd = 1.0 / math.sqrt(H)
    while filled < n:
        m = max(16, 2 * (n - filled))
        q = rng.normal(0.0, sd, size=(m, 3))
        if spring == SPRING_HOOKE:
            acc = q
        else:
            x = H * np.sum(q * q, axis=1) / b
            ok = x < 1.0
            q, x = q[ok], x[ok]
            logr = 0.5 * b * (np.log1p(-x) + x)
            acc = q[rng.random(len(q)) < np.exp(logr)]
        take = min(len(acc), n - filled)
        out[filled:filled + take] = acc[:take]
        filled += take
    return out


def initial_globule(rng: np.random.Generator, chain: Chain, tries: int = 48) -> np.ndarray:
    """Compact conformation [N][3] of a harmonic or vWF chain, centre of mass at 0.

    A walk with bonds of the rest length r0 (1 if r0 = 0): each new bead is
    the candidate, among `tries` random directions, nearest the beads placed
    so far (their centroid) that keeps at least 0.95 lj_sigma from every
    earlier non-adjacent bead. When no direction does (the walk has buried
    its end), up to 16 more sets of directions are drawn; if still none, the
    walk steps back four beads and regrows them taking the valid direction
    farthest from the centroid. With lj_sigma = 0 the walk is freely jointed
    (first candidate taken). This stands in for an equilibrated globule: the
    Lennard-Jones contacts start near their minimum, none overlapping.
    """
    N = chain.n_beads
    r0 = chain.r0 if chain.r0 > 0 else 1.0
    dmin = 0.95 * chain.lj_sigma
    r = np.zeros((N, 3))
    escape = 0          # beads still to grow away from the centroid
    backtracks = 0
    i = 1
    while i < N:
        if dmin <= 0 or i < 2:
            u = rng.normal(size=3)
            r[i] = r[i - 1] + r0 * u / np.linalg.norm(u)
            i += 1
            continue
        chosen = None
        for _ in range(17):
            u = rng.normal(size=(tries, 3))
            u /= np.linalg.norm(u, axis=1, keepdims=True)
            cand = r[i - 1] + r0 * u
            d = np.linalg.norm(cand[:, None, :] - r[None, :i - 1, :], axis=2).min(axis=1)
            ok = np.flatnonzero(d >= dmin)
            if ok.size:
                dist = np.linalg.norm(cand[ok] - r[:i].mean(axis=0), axis=1)
                chosen = cand[ok[np.argmax(dist) if escape else np.argmin(dist)]]
                break
        if chosen is None and backtracks < 1000:
            backtracks += 1
            i = max(2, i - 4)
            escape = 4
            continue
        if chosen is None:                       # give up: the farthest candidate
            chosen = cand[np.argmax(d)]
        r[i] = chosen
        escape = max(0, escape - 1)
        i += 1
    r -= r.mean(axis=0)
    return r


def initial_coil(rng: np.random.Generator, chain: Chain) -> np.ndarray:
    """Equilibrium random-walk conformation [N][3], centre of mass at 0
    (for harmonic chains, the compact walk of initial_globule)."""
    if chain.spring in (SPRING_HARMONIC, SPRING_VWF):
        return initial_globule(rng, chain)
    q = sample_connectors(rng, chain.n_beads - 1, chain.spring, chain.H, chain.b)
    r = np.zeros((chain.n_beads, 3))
    r[1:] = np.cumsum(q, axis=0)
    r -= r.mean(axis=0)
    return r


def initial_positions(workload: Workload, seed: Optional[int] = None) -> np.ndarray:
    """Concatenated initial conformations of all chains, [sum N][3] float64."""
    rng = np.random.default_rng(workload.init_seed if seed is None else seed)
    return np.concatenate([initial_coil(rng, c) for c in workload.chains], axis=0)


def spring_offsets(chains: Sequence[Chain]) -> np.ndarray:
    """Exclusive prefix sum of N_c - 1 (spring index base of each chain)."""
    return np.concatenate([[0], np.cumsum([c.n_beads - 1 for c in chains])]).astype(np.int64)


def bead_offsets(chains: Sequence[Chain]) -> np.ndarray:
    return np.concatenate([[0], np.cumsum([c.n_beads for c in chains])]).astype(np.int64)


# ---------------------------------------------------------------------------
# Named workloads
# ---------------------------------------------------------------------------

def single_chain_fp64(n_steps: int = 10_000) -> Workload:
    """One FENE chain, N=20, b=50, uniaxial Wi=2, dt=1e-3, 16 replicas,
    window 100, seed 0, threshold rupture at 0.9 F_max."""
    n, b = 20, 50.0
    ch = Chain(n_beads=n, n_replicas=16, spring=SPRING_FENE, flow=FLOW_UNIAXIAL,
               H=1.0, b=b, rate=rate_from_wi(2.0, n), f_c=0.9 * fene_fmax(1.0, b))
    return Workload("fene_n20_r16_uniaxial_wi2", [ch], dt=1e-3, window_steps=100,
                    n_steps=n_steps, seed=0, thr_mask=CRIT_RSF, bell_mask=0, init_seed=0)


def planar_1024(n_steps: int = 100_000, n_chains: int = 1024) -> Workload:
    """1024 FENE chains, N=100, b=100, planar elongation Wi=5, 64 replicas,
    dt=5e-4, window 100, seed 1. Threshold at 0.9 F_max and a Bell rate with
    k0 = 1e-6, dx F_max = 20 on the replica-averaged force."""
    n, b = 100, 100.0
    fmax = fene_fmax(1.0, b)
    chains = [Chain(n_beads=n, n_replicas=64, spring=SPRING_FENE, flow=FLOW_PLANAR,
                    H=1.0, b=b, rate=rate_from_wi(5.0, n), f_c=0.9 * fmax,
                    k0=1e-6, dx=20.0 / fmax) for _ in range(n_chains)]
    return Workload("fene_1024x_n100_r64_planar_wi5", chains, dt=5e-4, window_steps=100,
                    n_steps=n_steps, seed=1, thr_mask=CRIT_RSF, bell_mask=CRIT_RSF,
                    init_seed=1)


def uneven_4096(n_steps: int = 10_000, n_chains: int = 4096, gen_seed: int = 2) -> Workload:
    """4096 FENE chains, N ~ U{20..500}, R ~ {8,16,32,64,128}, half steady shear
    Wi ~ U[1,50], half uniaxial Wi ~ U[0.5,10], b ~ U[20,200], dt=1e-3."""
    rng = np.random.default_rng(gen_seed)
    chains = []
    for c in range(n_chains):
        n = int(rng.integers(20, 501))
        r = int(rng.choice([8, 16, 32, 64, 128]))
        b = float(rng.uniform(20.0, 200.0))
        if c % 2 == 0:
            flow, wi = FLOW_SHEAR, float(rng.uniform(1.0, 50.0))
        else:
            flow, wi = FLOW_UNIAXIAL, float(rng.uniform(0.5, 10.0))
        fmax = fene_fmax(1.0, b)
        chains.append(Chain(n_beads=n, n_replicas=r, spring=SPRING_FENE, flow=flow, H=1.0,
                            b=b, rate=rate_from_wi(wi, n), f_c=0.9 * fmax,
                            k0=1e-6, dx=20.0 / fmax))
    return Workload("fene_4096x_uneven_n20-500_r8-128", chains, dt=1e-3, window_steps=100,
                    n_steps=n_steps, seed=2, thr_mask=CRIT_RSF, bell_mask=CRIT_RSF,
                    init_seed=2)


def bell_16384(n_steps: int = 250_000, n_chains: int = 16384) -> Workload:
    """16384 FENE chains, N=50, b=100, start-up uniaxial Wi=10 from equilibrium,
    32 replicas, Bell k0=1e-6 and dx F_max = 20 on ISF, TSF and RSF."""
    n, b = 50, 100.0
    fmax = fene_fmax(1.0, b)
    chains = [Chain(n_beads=n, n_replicas=32, spring=SPRING_FENE, flow=FLOW_UNIAXIAL, H=1.0,
                    b=b, rate=rate_from_wi(10.0, n), f_c=0.9 * fmax, k0=1e-6,
                    dx=20.0 / fmax) for _ in range(n_chains)]
    return Workload("fene_16384x_n50_r32_uniaxial_wi10_bell", chains, dt=1e-3,
                    window_steps=100, n_steps=n_steps, seed=4, thr_mask=CRIT_ALL,
                    bell_mask=CRIT_ALL, init_seed=4)


# The collapsed-chain model of Sec. II in these units: length a (bead radius),
# energy kT, and a time unit of tau / 4 (tau the single-bead diffusion time,
# so that the bead diffusivity is 1/4 as in Eq. 1 above): a time of x tau is
# 4x here, so the paper's time step of 1e-5 tau is 4e-5, its shear rate
# 30 / tau is 7.5, and its evolution time S = 0.015 tau is 1500 steps.
COLLAPSED_DT = 4e-5
COLLAPSED_TAU = 4.0      # tau in these time units


def collapsed_chain(n_replicas: int, rate: float = 7.5, n_beads: int = 50) -> Chain:
    """The paper's collapsed chain: N = 50, kappa = 400 kT/a^2, rest length
    2a, Lennard-Jones depth u = 1 kT and minimum 2a between non-adjacent
    beads; steady shear (v_x = rate z)."""
    return Chain(n_beads=n_beads, n_replicas=n_replicas, spring=SPRING_HARMONIC,
                 flow=FLOW_SHEAR if rate else FLOW_NONE, rate=rate, H=400.0, r0=2.0,
                 lj_u=1.0, lj_sigma=2.0)


def collapsed_1024(n_steps: int = 15_000, n_chains: int = 1024) -> Workload:
    """1024 collapsed chains (N=50, kappa=400, u=1) in shear at gamma-dot = 30
    / tau, 50 replicas each, dt = 1e-5 tau, evolution time S = 0.015 tau
    (1500 steps), compact initial globules; force sampling only (no
    criteria)."""
    chains = [collapsed_chain(50) for _ in range(n_chains)]
    return Workload("collapsed_1024x_n50_r50_shear30", chains, dt=COLLAPSED_DT,
                    window_steps=1500, n_steps=n_steps, seed=6, thr_mask=0, bell_mask=0,
                    init_seed=6)


def collapsed_hi_128(n_steps: int = 1_500, n_chains: int = 128) -> Workload:
    """The paper's full model (Eqs. 1-3): 128 collapsed chains (N=50,
    kappa=400, u=1) with RPY hydrodynamic interaction (bead radius a) in shear
    at gamma-dot = 30 / tau, 50 replicas each, dt = 1e-5 tau, evolution time
    S = 0.015 tau (1500 steps); force sampling only."""
    chains = []
    for _ in range(n_chains):
        ch = collapsed_chain(50)
        ch.hi_a = 1.0
        chains.append(ch)
    return Workload("collapsed_hi_128x_n50_r50_shear30", chains, dt=COLLAPSED_DT,
                    window_steps=1500, n_steps=n_steps, seed=8, thr_mask=0, bell_mask=0,
                    init_seed=8)


# The coarse-grained vWF chain of the supplementary material (Table S1), in the
# units above (length a = 15 nm, energy kT, time tau / 4): a monomer is two
# beads joined by an A2 domain (a FENE spring in parallel with a harmonic
# spring), monomers are joined by disulfide bonds (harmonic springs), and
# non-adjacent beads attract with the Lennard-Jones energy epsilon = 1 kT.
VWF_A_NM = 15.0                 # bead radius a
VWF_KT_PN_NM = 4.143            # kT at 300 K (= the Lennard-Jones epsilon of Table S1)
VWF_ETA = 0.001                 # viscosity, pN us / nm^2
VWF_TAU_S = 6.0 * math.pi * VWF_ETA * VWF_A_NM ** 3 / VWF_KT_PN_NM * 1e-6   # 6 pi eta a^3 / kT
VWF_TIME_UNIT_S = VWF_TAU_S / COLLAPSED_TAU
VWF_FORCE_UNIT_PN = VWF_KT_PN_NM / VWF_A_NM          # kT / a
VWF_SPRING_UNIT = VWF_KT_PN_NM / VWF_A_NM ** 2       # kT / a^2 in pN / nm
VWF_K0_PER_S = 7e-4             # zero-force A2 unfolding rate
VWF_FU_PN = 1.1                 # force scale of the unfolding rate k0 exp(f / f_u)


def vwf_chain(n_replicas: int, n_beads: int = 50, hi: bool = True) -> Chain:
    """The vWF chain (Table S1): 25 monomers, 50 beads; disulfide bonds 7.5
    pN/nm, A2 domains 0.116 pN/nm (FENE, maximum extension 51.46 nm beyond the
    rest length 2a) in parallel with 5 pN/nm (harmonic); Lennard-Jones u = 1 kT
    at 2a; Bell unfolding of the A2 domains, k = k0 exp(f / f_u); no flow; RPY
    hydrodynamic interaction (bead radius a) unless hi is False."""
    return Chain(n_beads=n_beads, n_replicas=n_replicas, spring=SPRING_VWF, flow=FLOW_NONE,
                 H=7.5 / VWF_SPRING_UNIT, r0=2.0, lj_u=1.0, lj_sigma=2.0,
                 vwf_fa=0.116 / VWF_SPRING_UNIT, vwf_fb=5.0 / VWF_SPRING_UNIT,
                 vwf_xmax=51.46 / VWF_A_NM, k0=VWF_K0_PER_S * VWF_TIME_UNIT_S,
                 dx=VWF_FORCE_UNIT_PN / VWF_FU_PN, hi_a=1.0 if hi else 0.0)


def vwf_mftu_seconds(hazard_rate: float) -> float:
    """Mean first time to unfold any A2 domain (Table 1's MFTU) for a chain
    whose A2 domains unfold at the summed rate `hazard_rate` (per time unit):
    1 / rate, in seconds."""
    return VWF_TIME_UNIT_S / hazard_rate


def vwf_64(n_steps: int = 1_500, n_chains: int = 64, n_replicas: int = 40,
           window_steps: int = 1_500) -> Workload:
    """64 vWF chains at rest (Table 1's set-up): 50 beads, N_R = 40,
    dt = 1e-5 tau, evolution time S = 0.015 tau (1500 steps), Bell unfolding
    on ISF, TSF and RSF."""
    chains = [vwf_chain(n_replicas) for _ in range(n_chains)]
    return Workload("vwf_64x_n50_r40_rest", chains, dt=COLLAPSED_DT, window_steps=window_steps,
                    n_steps=n_steps, seed=10, thr_mask=0, bell_mask=CRIT_ALL, init_seed=10)


def adjoint_256(n_steps: int = 20_000, n_chains: int = 256) -> Workload:
    """256 FENE chains, N=200, b=100, H=1, 32 replicas, uniaxial elongation
    Wi=5, dt=1e-3, window 100, Bell k0=1e-6 and dx F_max = 20 on the
    replica-averaged force; differentiated with parent checkpoints every 1000
    steps."""
    n, b = 200, 100.0
    fmax = fene_fmax(1.0, b)
    chains = [Chain(n_beads=n, n_replicas=32, spring=SPRING_FENE, flow=FLOW_UNIAXIAL, H=1.0,
                    b=b, rate=rate_from_wi(5.0, n), f_c=0.9 * fmax, k0=1e-6,
                    dx=20.0 / fmax) for _ in range(n_chains)]
    return Workload("fene_256x_n200_r32_uniaxial_wi5_adjoint", chains, dt=1e-3,
                    window_steps=100, n_steps=n_steps, seed=5, thr_mask=0,
                    bell_mask=CRIT_RSF, init_seed=5)


ADJOINT_CHECKPOINT_STEPS = 1000


def custom(chains: Sequence[Chain], dt: float, window_steps: int, n_steps: int,
           seed: int = 0, thr_mask: int = CRIT_ALL, bell_mask: int = CRIT_ALL,
           init_seed: int = 7, name: str = "custom") -> Workload:
    return Workload(name, list(chains), dt=dt, window_steps=window_steps, n_steps=n_steps,
                    seed=seed, thr_mask=thr_mask, bell_mask=bell_mask, init_seed=init_seed)
