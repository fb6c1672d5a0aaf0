"""Seeded synthetic workloads for the ETD2RKds hot path.

This module is shared by the FP64 oracle, the tests and the benchmark.  It
holds problem descriptions (grid, domain, coefficients, reaction model, step
size) and seeded initial data, and nothing of the time-stepping method's
arithmetic.  Random numbers come from SplitMix64 (Steele, Lea & Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014), a
counter-based generator with a published definition, so every consumer sees
the same bits on x86 and Arm.

Problem statement (two-component ADR system, homogeneous Neumann boundaries
on a box domain) follows Sec. 1, Eq. (1) of Caliari & Cassini,
arXiv:2307.10684.  The reaction models are the Schnakenberg model
(Sec. 4.1), a FitzHugh-Nagumo variant with advection, and the advective
Brusselator (Sec. 4.6).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence, Tuple

import numpy as np

# Reaction model identifiers (mirrors the C ABI enum adr_model).
SCHNAKENBERG = 0
FHN = 1
BRUSSELATOR = 2
NO_REACTION = 3
FHN_RHO = 4
DIB = 5
MODEL_NAMES = {SCHNAKENBERG: "schnakenberg", FHN: "fhn", BRUSSELATOR: "brusselator",
               NO_REACTION: "none", FHN_RHO: "fhn_rho", DIB: "dib"}

# Scheme identifiers (mirrors the C ABI enum adr_scheme).
ETD2RKDS = 0
LAWSON2B = 1

# State modes (mirrors the C ABI enum adr_state_mode).
STATE_AUTO = 0
STATE_PLAIN = 1
STATE_COMPENSATED = 2

# Precision identifiers (mirrors the C ABI enum adr_precision).
FP64 = 0
FP32 = 1
TF32X3 = 2
BF16X3 = 3
PRECISION_NAMES = {FP64: "fp64", FP32: "fp32", TF32X3: "tf32x3", BF16X3: "bf16x3"}


@dataclasses.dataclass
class Problem:
    """One ADR solve: u_t = K^u u + g^u(u,v), v_t = K^v v + g^v(u,v).

    n[mu] is the number of grid points along direction mu (mu = 0 is x_1,
    the contiguous axis).  State arrays have numpy shape (n_d, ..., n_1),
    i.e. x_1 fastest, which is the column-major vec ordering of Sec. 2.
    diff[c] is the diffusion coefficient of component c (0 = u, 1 = v);
    adv[c][mu] the advection velocity of the term -adv . grad(c).
    params: Schnakenberg (gamma, a, b); FHN (eps, a1, a0); Brusselator (a, b).
    """

    d: int
    n: Tuple[int, ...]
    lo: Tuple[float, ...]
    hi: Tuple[float, ...]
    diff: Tuple[float, float]
    adv: Tuple[Tuple[float, ...], Tuple[float, ...]]
    model: int
    params: Tuple[float, ...]
    tau: float
    nsteps: int
    precision: int = FP32
    seed: int = 0
    name: str = ""
    scheme: int = 0   # 0 = ETD2RKds (Eq. 11), 1 = Lawson2b (Eq. 7)
    state: int = 0    # adr_state_mode: 0 = library's choice, 1 = plain, 2 = compensated

    @property
    def shape(self) -> Tuple[int, ...]:
        """numpy shape of a state tensor: (n_d, ..., n_1)."""
        return tuple(reversed(self.n[: self.d]))

    @property
    def npoints(self) -> int:
        return int(np.prod(self.n[: self.d]))

    def replace(self, **kw) -> "Problem":
        return dataclasses.replace(self, **kw)


# ---------------------------------------------------------------- SplitMix64
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Outputs offset..offset+count-1 of SplitMix64 started from `seed`.

    Output k is the finaliser applied to seed + (k+1) * golden gamma, so any
    slice of the stream can be produced without generating the prefix.
    """
    k = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Doubles in [0, 1): top 53 bits of each SplitMix64 output times 2^-53."""
    z = splitmix64(seed, count, offset)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Standard normal deviates by Box-Muller over consecutive uniform pairs."""
    m = (count + 1) // 2
    u = uniform01(seed, 2 * m, 2 * offset)
    u1 = 1.0 - u[0::2]  # (0, 1]
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * m)
    z[0::2] = r * np.cos(2.0 * math.pi * u2)
    z[1::2] = r * np.sin(2.0 * math.pi * u2)
    return z[:count]


# ---------------------------------------------------------------- equilibria
def equilibrium(model: int, params: Sequence[float]) -> Tuple[float, float]:
    """Spatially constant steady state of the reaction terms."""
    if model == SCHNAKENBERG:
        _, a, b = params[:3]
        return a + b, b / (a + b) ** 2
    if model == BRUSSELATOR:
        a, b = params[:2]
        return a, b / a
    if model == NO_REACTION:
        return 1.0, 1.0
    if model == FHN_RHO:
        return 0.0, 0.0
    if model == DIB:
        return 0.0, params[4]
    if model == FHN:
        # u - u^3 - v = 0 and u - a1 v - a0 = 0  ->  u(1 - 1/a1) - u^3 + a0/a1 = 0;
        # take the root of smallest magnitude by Newton from u = 0.
        _, a1, a0 = params[:3]
        u = 0.0
        for _ in range(100):
            f = u * (1.0 - 1.0 / a1) - u ** 3 + a0 / a1
            fp = (1.0 - 1.0 / a1) - 3.0 * u ** 2
            u -= f / fp
        return u, (u - a0) / a1
    raise ValueError(f"unknown model {model}")


# ---------------------------------------------------------------- initial data
def initial_data(p: Problem, kind: str = "auto", amp: float | None = None):
    """Seeded initial data (u0, v0) as float64 arrays of shape p.shape.

    kind "uniform": equilibrium + amp * U[-1, 1] (amp defaults to 0.01);
    kind "uniform01": equilibrium + amp * U[0, 1] (amp defaults to 1e-5; the
    paper's perturbation of its Sec. 4.1, 4.2 and 4.4 examples);
    kind "normal": amp * N(0, 1) about 0 (amp defaults to 0.05);
    kind "auto": normal for FHN, uniform otherwise.
    The u field takes stream outputs [0, N), the v field [N, 2N).
    """
    N = p.npoints
    if kind == "auto":
        kind = "normal" if p.model == FHN else "uniform"
    if kind == "uniform":
        a = 0.01 if amp is None else amp
        ue, ve = equilibrium(p.model, p.params)
        r = uniform01(p.seed, 2 * N)
        u = ue + a * (2.0 * r[:N] - 1.0)
        v = ve + a * (2.0 * r[N:] - 1.0)
    elif kind == "uniform01":
        a = 1e-5 if amp is None else amp
        ue, ve = equilibrium(p.model, p.params)
        r = uniform01(p.seed, 2 * N)
        u = ue + a * r[:N]
        v = ve + a * r[N:]
    elif kind == "normal":
        a = 0.05 if amp is None else amp
        z = normal(p.seed, 2 * N)
        u = a * z[:N]
        v = a * z[N:]
    else:
        raise ValueError(kind)
    return u.reshape(p.shape), v.reshape(p.shape)


def brusselator_e6_initial(p: Problem):
    """Deterministic data of the paper's 3D advective Brusselator example
    (Sec. 4.6): u0 = 1 + sin(2 pi x1) sin(2 pi x2) sin(2 pi x3), v0 = 3."""
    xs = [np.linspace(p.lo[m], p.hi[m], p.n[m]) for m in range(p.d)]
    grids = np.meshgrid(*reversed(xs), indexing="ij")  # axis 0 = x_d
    s = np.ones(p.shape)
    for g in grids:
        s = s * np.sin(2.0 * math.pi * g)
    return 1.0 + s, 3.0 * np.ones(p.shape)


def round_to(x: np.ndarray, precision: int) -> np.ndarray:
    """Round FP64 data to the run precision and promote back to FP64, so that
    the oracle and the GPU start from identical values."""
    if precision == FP64:
        return np.array(x, dtype=np.float64)
    return np.asarray(x, dtype=np.float32).astype(np.float64)


# ---------------------------------------------------------------- configurations
def schnakenberg_64(precision: int = FP64) -> Problem:
    """2D Schnakenberg on [0,1]^2, 64x64, gamma=1000, a=0.1, b=0.9, D=(1,10),
    tau = 5e-4, 200 steps (T = 0.1); data = equilibrium + U[-0.01, 0.01]."""
    return Problem(d=2, n=(64, 64), lo=(0.0, 0.0), hi=(1.0, 1.0), diff=(1.0, 10.0),
                   adv=((0.0, 0.0), (0.0, 0.0)), model=SCHNAKENBERG,
                   params=(1000.0, 0.1, 0.9), tau=5e-4, nsteps=200,
                   precision=precision, seed=1, name="schnakenberg2d_64")


def fhn_1024(precision: int = FP32, n: int = 1024, nsteps: int = 500) -> Problem:
    """2D FitzHugh-Nagumo variant with advection on [0,100]^2, n x n (1024),
    D=(1,20), velocity (0.5,0.5), eps=0.05, a1=2, a0=-0.03, tau=1e-2,
    500 steps; data ~ N(0, 0.05^2)."""
    return Problem(d=2, n=(n, n), lo=(0.0, 0.0), hi=(100.0, 100.0), diff=(1.0, 20.0),
                   adv=((0.5, 0.5), (0.5, 0.5)), model=FHN, params=(0.05, 2.0, -0.03),
                   tau=1e-2, nsteps=nsteps, precision=precision, seed=2,
                   name=f"fhn2d_adv_{n}")


def brusselator_256(precision: int = FP32, n: int = 256, nsteps: int = 100) -> Problem:
    """3D advective Brusselator on [0,1]^3, n^3 (256^3), a=1, b=3,
    D=(0.02,0.1), velocity (-0.5,-0.5,-0.5), tau=1e-2, 100 steps;
    data = (a, b/a) + U[-0.01, 0.01]."""
    v = (-0.5, -0.5, -0.5)
    return Problem(d=3, n=(n, n, n), lo=(0.0,) * 3, hi=(1.0,) * 3, diff=(0.02, 0.1),
                   adv=(v, v), model=BRUSSELATOR, params=(1.0, 3.0), tau=1e-2,
                   nsteps=nsteps, precision=precision, seed=3,
                   name=f"brusselator3d_adv_{n}")


def dib_parameters():
    """(rho, a1u, a2u, a3u, a4u, a1v, a2v, a3v, a4v, a5v) of Sec. 4.4, with a4v
    derived so that (0, a4u) is an equilibrium."""
    rho, a1u, a2u, a3u, a4u = 25.0 / 4.0, 10.0, 1.0, 66.0, 0.5
    a1v, a2v, a3v, a5v = 3.0, 2.5, 0.2, 1.5
    a4v = a1v * (1.0 - a4u) * (1.0 - a3v + a3v * a4u) / (a4u * (1.0 + a3v * a4u))
    return (rho, a1u, a2u, a3u, a4u, a1v, a2v, a3v, a4v, a5v)


def dib_200(precision: int = FP32, n: int = 200, nsteps: int = 1250) -> Problem:
    """2D DIB model of Sec. 4.4 on [0,20]^2, n x n (200), D = (1, 20),
    T = 2.5 in `nsteps` steps; data (0, a4u) + 1e-5 U(0,1)."""
    return Problem(d=2, n=(n, n), lo=(0.0, 0.0), hi=(20.0, 20.0), diff=(1.0, 20.0),
                   adv=((0.0, 0.0), (0.0, 0.0)), model=DIB, params=dib_parameters(),
                   tau=2.5 / nsteps, nsteps=nsteps, precision=precision, seed=123,
                   name=f"dib2d_{n}")


def fhn_rho(d: int = 2, precision: int = FP32, n: int | None = None,
            nsteps: int = 20000) -> Problem:
    """FitzHugh-Nagumo of Sec. 4.2 (2D, n = 100, rho = 65.731) and Sec. 4.3
    (3D, n = 64, rho = 24.649) on [0, pi]^d, D = (1, 42.1887), a1 = 11,
    a2 = 0.1, T = 10; data 1e-3 U(0,1) about (0, 0)."""
    n = n or (100 if d == 2 else 64)
    rho = 65.731 if d == 2 else 24.649
    return Problem(d=d, n=(n,) * d, lo=(0.0,) * d, hi=(math.pi,) * d, diff=(1.0, 42.1887),
                   adv=((0.0,) * d, (0.0,) * d), model=FHN_RHO, params=(rho, 11.0, 0.1),
                   tau=10.0 / nsteps, nsteps=nsteps, precision=precision, seed=0,
                   name=f"fhn_rho{d}d_{n}")


BATCH_SIDES = (64, 96, 128, 192, 256, 384, 512)


def schnakenberg_tau(gamma: float) -> float:
    """Step for batched and served Schnakenberg solves: 1.25e-4 (1000/gamma),
    clipped to [6.25e-5, 1.25e-3].  The reaction time scale is 1/gamma; over
    100 steps the Turing-unstable modes with D_v/D_u up to 40 amplify FP32
    rounding, and at twice this step the FP64 conditioning floor alone
    reaches 1e-5 for the stiffest solves."""
    return min(max(1.25e-4 * (1000.0 / gamma), 6.25e-5), 1.25e-3)


def batched_512(count: int = 512, nsteps: int = 100, precision: int = FP32) -> List[Problem]:
    """512 independent 2D solves: sides iid from BATCH_SIDES (non-square
    allowed), half Schnakenberg on [0,1]^2 (gamma ~ U[100,2000], step
    schnakenberg_tau), half FHN on [0,100]^2 (tau = 1e-2, velocity (0.5,
    0.5)); D_u = 1, D_v/D_u ~ U[5,40]; solve i uses seed 1000 + i."""
    r = uniform01(4, 8 * count)
    out = []
    for i in range(count):
        q = r[8 * i: 8 * i + 8]
        n1 = BATCH_SIDES[int(q[0] * len(BATCH_SIDES))]
        n2 = BATCH_SIDES[int(q[1] * len(BATCH_SIDES))]
        dv = 5.0 + 35.0 * q[3]
        if q[2] < 0.5:
            gamma = 100.0 + 1900.0 * q[4]
            tau = schnakenberg_tau(gamma)
            p = Problem(d=2, n=(n1, n2), lo=(0.0, 0.0), hi=(1.0, 1.0), diff=(1.0, dv),
                        adv=((0.0, 0.0), (0.0, 0.0)), model=SCHNAKENBERG,
                        params=(gamma, 0.1, 0.9), tau=tau, nsteps=nsteps,
                        precision=precision, seed=1000 + i, name=f"batch{i}")
        else:
            p = Problem(d=2, n=(n1, n2), lo=(0.0, 0.0), hi=(100.0, 100.0), diff=(1.0, dv),
                        adv=((0.5, 0.5), (0.5, 0.5)), model=FHN, params=(0.05, 2.0, -0.03),
                        tau=1e-2, nsteps=nsteps, precision=precision, seed=1000 + i,
                        name=f"batch{i}")
        out.append(p)
    return out


SERVE_SIDES_2D = (128, 192, 256, 384, 512, 768, 1024)
SERVE_SIDES_3D = (64, 96, 128, 160, 192)


def serving_stream(count: int = 2000, rate: float = 200.0, precision: int = FP32,
                   seed: int = 5) -> List[Tuple[float, Problem]]:
    """Poisson request stream: (arrival time in s, problem).  Half 2D grids
    (sides from SERVE_SIDES_2D), half 3D (SERVE_SIDES_3D); model uniform over
    the three; coefficients within +-50% of the base configurations with the
    cell Peclet number kept below 1; horizons uniform on {50..1000} steps."""
    r = uniform01(seed, 16 * count)
    t = 0.0
    out = []
    for i in range(count):
        q = r[16 * i: 16 * i + 16]
        t += -math.log(1.0 - q[0]) / rate
        three_d = q[1] >= 0.5
        if three_d:
            s = SERVE_SIDES_3D[int(q[2] * len(SERVE_SIDES_3D))]
            n = (s, s, s)
        else:
            s = SERVE_SIDES_2D[int(q[2] * len(SERVE_SIDES_2D))]
            n = (s, s)
        d = len(n)
        model = int(q[3] * 3)
        f = lambda x: 0.5 + x  # factor in [0.5, 1.5)
        if model == SCHNAKENBERG:
            base = schnakenberg_64()
            params = (base.params[0] * f(q[4]), 0.1, 0.9)
            diff = (1.0 * f(q[5]), 10.0 * f(q[6]))
            vel = (0.0,) * d
            L = 1.0
            tau = schnakenberg_tau(params[0])
        elif model == FHN:
            params = (0.05 * f(q[4]), 2.0, -0.03)
            diff = (1.0 * f(q[5]), 20.0 * f(q[6]))
            vel = (0.5 * f(q[7]),) * d
            L = 100.0
            tau = 1e-2
        else:
            params = (1.0, 3.0 * f(q[4]))
            diff = (0.02 * f(q[5]), 0.1 * f(q[6]))
            vel = (-0.5 * f(q[7]),) * d
            L = 1.0
            tau = 1e-2
        # keep the cell Peclet number |alpha| h / (2 delta) below 1
        h = L / (min(n) - 1)
        vmax = 0.9 * 2.0 * min(diff) / h
        vel = tuple(max(-vmax, min(vmax, a)) for a in vel)
        steps = 50 + int(q[8] * 951)
        p = Problem(d=d, n=n, lo=(0.0,) * d, hi=(L,) * d, diff=diff, adv=(vel, vel),
                    model=model, params=params, tau=tau, nsteps=steps,
                    precision=precision, seed=100000 + i, name=f"req{i}")
        out.append((t, p))
    return out
