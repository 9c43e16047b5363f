"""Seeded synthetic inputs for the fast Monte Carlo pipeline.

This module only draws the *inputs* of a study: the machine system, the
disturbance model and the sampling settings.  It holds none of the method's
arithmetic (no equilibrium, no dynamics, no KL basis, no sampling; the only
network sum it forms is each machine's resistive load at zero angles, to place
the mechanical powers where an operating point exists); the CUDA library and
the FP64 oracle each compute the method themselves from these inputs.  Parameter draws use numpy's PCG64 generator seeded explicitly; the
random numbers of the method itself (the Latin hypercube design) are drawn
inside each implementation from the seed carried here.

Workloads (the paper's IEEE 39-bus case, its PSS/E models and its wind record
are not available, so these stand in for them):

* ``smib_case``   -- single machine against an infinite bus, one OU disturbance
  on the mechanical power, K = 100, T = 10 s, dt = 0.01 s, N = 1000.
* ``multimachine_case`` -- a Kron-reduced classical system of ``n`` machines
  shaped like the 39-bus case's 10 generators: symmetric off-diagonal
  susceptances U[1,8] and conductances U[0,0.3] p.u., diagonally dominant,
  H ~ U[3,10] s, D ~ U[1,2], E ~ U[1.0,1.1], mechanical power of machine i =
  its resistive load sum_j E_i E_j G_ij plus U[-1,2] p.u. (machine 0 balances),
  ``d`` OU disturbances (theta ~ U[0.5,2] /s, sigma ~ U[0.02,0.1]) each on the
  mechanical power of a distinct machine (machines repeat when d > n).
* ``batched_cases`` -- many such systems with uneven sizes.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

LHS = 0
SRS = 1
LHS_MIDPOINT = 2
SRS_EM = 3  # the paper's traditional Monte Carlo: a fresh normal per step (no KL expansion)

RK4 = 0
HEUN = 1

BASIS_SINE = 0    # Brownian eigenbasis
BASIS_COSINE = 1  # the paper's cosine white-noise basis

FORCING_INCREMENTS = 0  # Euler-Maruyama on the KL increments of each step
FORCING_SMOOTH = 1      # the random ODE of Eq. (eqkl): the smooth KL forcing at the RK stage times

CORR_NONE = 0   # the design's random permutations (Section IV-B step 2) as they are
CORR_RANK = 1   # the correlation-reducing permutation (rank method of Iman and Conover)


@dataclasses.dataclass
class Scenario:
    """One uncertainty-evaluation problem: system, disturbances, KL and sampling."""

    n: int
    d: int
    K: int
    T: float
    dt: float
    N: int
    seed: int
    omega_s: float
    G: np.ndarray        # [n, n]
    B: np.ndarray        # [n, n]
    H: np.ndarray        # [n]
    D: np.ndarray        # [n]
    E: np.ndarray        # [n]
    Pm: np.ndarray       # [n]; Pm[0] is balanced by the equilibrium without an infinite bus
    theta: np.ndarray    # [d]
    sigma: np.ndarray    # [d]
    inject: np.ndarray   # [n, d]
    has_inf_bus: bool = False
    Ginf: np.ndarray | None = None
    Binf: np.ndarray | None = None
    Vinf: float = 1.0
    sampling: int = LHS
    integrator: int = RK4
    basis: int = BASIS_SINE
    # an event in the style of the paper's generator trip: from t = event_time on
    # (rounded to the grid) machine event_machine's mechanical power changes by
    # event_dpm p.u.; None: no event
    event_machine: int | None = None
    event_time: float = 0.0
    event_dpm: float = 0.0
    # general Ito disturbances (one dict per disturbance, see ito_* below), or
    # None: every disturbance is Ornstein-Uhlenbeck with theta, sigma
    ito: list | None = None
    # how the KL path drives the disturbances: FORCING_INCREMENTS (the GPU library
    # and the oracle) or FORCING_SMOOTH (the oracle only, so far)
    forcing: int = FORCING_INCREMENTS
    # Section IV-B step 2: CORR_NONE (the design's random permutations as they
    # are) or CORR_RANK (the correlation-reducing permutation)
    correlation: int = 0

    @property
    def Nt(self) -> int:
        return int(round(self.T / self.dt))

    @property
    def M(self) -> int:
        return self.d * self.K

    def replace(self, **kw) -> "Scenario":
        return dataclasses.replace(self, **kw)

    def machine_steps(self) -> int:
        return int(self.N) * self.Nt * self.n


# One-dimensional Ito processes of the paper's Table I (unit rate) and the wind
# model it identifies (Eq. windito): drift m0 + m1 x + m2 x^2; diffusion either
# s0 + s1 x + s2 x^2 (kind 1) or the square root of v0 + v1 x + v2 x^2 + v3 |x - a|
# (kind 2); x0 = the start (the mean of the stationary law, or the drift's
# stable root).
def ito_gaussian(a: float, b: float) -> dict:
    return dict(kind=2, m=(a, -1.0, 0.0), v=(2.0 * b, 0.0, 0.0, 0.0), a=0.0, x0=a)


def ito_beta(a: float, b: float) -> dict:
    return dict(kind=2, m=(a / (a + b), -1.0, 0.0), v=(0.0, 2.0 / (a + b), -2.0 / (a + b), 0.0), a=0.0,
                x0=a / (a + b))


def ito_gamma(a: float, b: float) -> dict:
    return dict(kind=2, m=(a / b, -1.0, 0.0), v=(0.0, 2.0 / b, 0.0, 0.0), a=0.0, x0=a / b)


def ito_laplace(a: float, b: float) -> dict:
    return dict(kind=2, m=(a, -1.0, 0.0), v=(2.0 * b * b, 0.0, 0.0, 2.0 * b), a=a, x0=a)


def ito_wind() -> dict:
    m = (0.0535, -0.0899, 0.0349)
    # the stable root of the drift (where it decreases)
    r = np.roots([m[2], m[1], m[0]])
    x0 = float(min(r.real))
    return dict(kind=1, m=m, s=(-0.410, 0.919, -0.505), a=0.0, x0=x0)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def smib_case(N: int = 1000, K: int = 100, T: float = 10.0, dt: float = 0.01, seed: int = 0,
              H: float = 5.0, D: float = 1.0, E: float = 1.1, V: float = 1.0, X: float = 0.5,
              Pm: float = 0.8, theta: float = 1.0, sigma: float = 0.05) -> Scenario:
    """Single machine, infinite bus: Pe = E V / X sin(delta)."""
    return Scenario(
        n=1, d=1, K=K, T=T, dt=dt, N=N, seed=seed, omega_s=2.0 * math.pi * 50.0,
        G=_f64([[0.0]]), B=_f64([[-1.0 / X]]),
        H=_f64([H]), D=_f64([D]), E=_f64([E]), Pm=_f64([Pm]),
        theta=_f64([theta]), sigma=_f64([sigma]), inject=_f64([[1.0]]),
        has_inf_bus=True, Ginf=_f64([0.0]), Binf=_f64([1.0 / X]), Vinf=V,
    )


def random_network(rng: np.random.Generator, n: int):
    """Symmetric Kron-reduced admittance, diagonally dominant."""
    Boff = rng.uniform(1.0, 8.0, size=(n, n))
    Goff = rng.uniform(0.0, 0.3, size=(n, n))
    Boff = np.triu(Boff, 1)
    Goff = np.triu(Goff, 1)
    Boff = Boff + Boff.T
    Goff = Goff + Goff.T
    G = Goff.copy()
    B = Boff.copy()
    for i in range(n):
        G[i, i] = Goff[i].sum() + rng.uniform(0.1, 0.5)
        B[i, i] = -Boff[i].sum() - rng.uniform(0.5, 2.0)
    return _f64(G), _f64(B)


def multimachine_case(n: int = 10, d: int = 3, K: int = 200, T: float = 20.0, dt: float = 0.005,
                      N: int = 1 << 16, seed: int = 0, system_seed: int | None = None) -> Scenario:
    """Classical multi-machine system shaped like the 39-bus case's generators.

    ``system_seed`` draws the system; ``seed`` keys the Latin hypercube design.
    """
    rng = np.random.default_rng(seed if system_seed is None else system_seed)
    G, B = random_network(rng, n)
    H = rng.uniform(3.0, 10.0, size=n)
    Dm = rng.uniform(1.0, 2.0, size=n)
    E = rng.uniform(1.0, 1.1, size=n)
    # mechanical power: the resistive load of the machine at nominal voltages and
    # angles (sum_j E_i E_j G_ij) plus a margin U[-1, 2] p.u., so that an operating
    # point exists for any machine count (the positive conductances grow with n)
    Pm = E * (G @ E) + rng.uniform(-1.0, 2.0, size=n)
    theta = rng.uniform(0.5, 2.0, size=d)
    sigma = rng.uniform(0.02, 0.1, size=d)
    gens = rng.choice(n, size=d, replace=(d > n))
    inject = np.zeros((n, d))
    for w, g in enumerate(gens):
        inject[g, w] = 1.0
    return Scenario(n=n, d=d, K=K, T=T, dt=dt, N=N, seed=seed, omega_s=2.0 * math.pi * 50.0,
                    G=G, B=B, H=_f64(H), D=_f64(Dm), E=_f64(E), Pm=_f64(Pm),
                    theta=_f64(theta), sigma=_f64(sigma), inject=_f64(inject))


def batched_cases(count: int = 64, seed: int = 0, n_range=(3, 50), d_range=(1, 8), K_range=(50, 300),
                  T_range=(5.0, 60.0), dt: float = 0.005, N_range=(1000, 256 * 1024)) -> list[Scenario]:
    """Uneven scenarios: machines, disturbances, KL order, horizon and N all drawn."""
    rng = np.random.default_rng(seed)
    out = []
    for c in range(count):
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        d = int(rng.integers(d_range[0], d_range[1] + 1))
        K = int(rng.integers(K_range[0], K_range[1] + 1))
        steps = int(rng.integers(int(T_range[0] / dt), int(T_range[1] / dt) + 1))
        N = int(rng.integers(N_range[0], N_range[1] + 1))
        out.append(multimachine_case(n=n, d=d, K=K, T=steps * dt, dt=dt, N=N, seed=seed * 1000 + c,
                                     system_seed=int(rng.integers(0, 2**31))))
    return out
