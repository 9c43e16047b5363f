"""FP64 CPU oracle for the fast Monte Carlo method (arXiv 2007.03847).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product library
(``paper_2007_03847_gb300``) never imports, links or executes it, and the two
share no code: the oracle is the plain C in ``fmc_oracle.c``, compiled with gcc
by ``build()``, and this file only marshals numpy arrays into it.

Functions and the passages they follow:

* ``philox4x32_10``           -- the counter-based generator of Salmon et al., SC'11.
* ``lhs_stratum``, ``lhs_uniform``, ``lhs_sample`` -- Section IV-B steps 1-2,
  Algorithm 1 step 1.
* ``ppnd16``                  -- inverse normal CDF, Wichura AS 241 (1988).
* ``kl_increment_basis``, ``kl_path_basis``, ``kle_reconstruct`` -- Eqs. (kl),
  (kle), (eqkl); Algorithm 1 step 2.  Two bases: the Brownian eigenbasis (the
  Karhunen-Loeve basis of min(s, t)) and the paper's cosine basis, Eq. (klb2).
* ``em_normal``, ``em_increments``, ``simulate_em`` -- the traditional Monte
  Carlo the paper compares against (Section V-B): Eq. (distito) with a fresh
  normal per step.
* ``electrical_power``, ``equilibrium`` -- Eqs. (state)/(algebra) for the
  classical model; equilibrium at t = 0 as in Section V-A.
* ``lhs_decorrelate``         -- Section IV-B step 2, the correlation-reducing
  permutation, by the rank method of Iman and Conover (1982).
* ``ito_objective``, ``ito_identify`` -- the Appendix's identification of an Ito
  model from a record (Eqs. likelihood, like, reprob, ident).
* ``simulate``                -- Algorithm 1 steps 2-4.
* ``moments_twopass``         -- Algorithm 1 step 4.

Pins (tests/test_oracle_*.py): Philox known-answer vectors, every LHS stratum
hit once, Phi(Phi^-1(p)) = p, the KL variance identity at t = T (and W(T)
exact for the cosine basis, its bridge-tail bound), the per-step normals as
Philox words through scipy's inverse CDF, the exact EM-OU variance, the OU and
Lyapunov closed forms, constant equilibrium, RK4 order, product vs pairwise
electrical power.  End-to-end moments of the nonlinear multi-machine system
have no published values: parity unpinned beyond those invariants.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fmc_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

LHS, SRS, LHS_MIDPOINT = 0, 1, 2
PE_PAIRWISE, PE_PRODUCT = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (strict IEEE FP64: no contraction, no fast-math)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm", "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Ito(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("pad", ctypes.c_int32), ("m0", ctypes.c_double), ("m1", ctypes.c_double),
                ("m2", ctypes.c_double), ("s0", ctypes.c_double), ("s1", ctypes.c_double), ("s2", ctypes.c_double),
                ("v0", ctypes.c_double), ("v1", ctypes.c_double), ("v2", ctypes.c_double), ("v3", ctypes.c_double),
                ("a", ctypes.c_double), ("x0", ctypes.c_double)]


def _ito_struct(spec) -> _Ito:
    """spec: dict(kind=1|2, m=(m0, m1, m2), s=(s0, s1, s2) | v=(v0, v1, v2, v3), a=..., x0=...), or None (OU)."""
    it = _Ito()
    if spec is None:
        return it
    it.kind = int(spec["kind"])
    it.m0, it.m1, it.m2 = (float(c) for c in spec["m"])
    if it.kind == 1:
        it.s0, it.s1, it.s2 = (float(c) for c in spec["s"])
    else:
        it.v0, it.v1, it.v2, it.v3 = (float(c) for c in spec["v"])
    it.a = float(spec.get("a", 0.0))
    it.x0 = float(spec.get("x0", 0.0))
    return it


class _System(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int32), ("d", ctypes.c_int32), ("K", ctypes.c_int32), ("Nt", ctypes.c_int32),
        ("T", ctypes.c_double), ("dt", ctypes.c_double), ("omega_s", ctypes.c_double),
        ("has_inf_bus", ctypes.c_int32), ("integrator", ctypes.c_int32), ("Vinf", ctypes.c_double),
        ("G", ctypes.c_void_p), ("B", ctypes.c_void_p), ("Ginf", ctypes.c_void_p), ("Binf", ctypes.c_void_p),
        ("H", ctypes.c_void_p), ("D", ctypes.c_void_p), ("E", ctypes.c_void_p), ("Pm", ctypes.c_void_p),
        ("theta", ctypes.c_void_p), ("sigma", ctypes.c_void_p), ("inject", ctypes.c_void_p),
        ("init_delta", ctypes.c_void_p), ("basis", ctypes.c_int32), ("em", ctypes.c_int32),
        ("em_seed", ctypes.c_uint64), ("em_k0", ctypes.c_int64), ("event_machine", ctypes.c_int32),
        ("event_step", ctypes.c_int32), ("event_dpm", ctypes.c_double), ("ito", ctypes.c_void_p),
        ("smooth", ctypes.c_int32),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u32p = ctypes.POINTER(ctypes.c_uint32)
            lib.oracle_philox4x32_10.argtypes = [u32p, u32p, u32p]
            lib.oracle_lhs_stratum.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32, ctypes.c_int64]
            lib.oracle_lhs_stratum.restype = ctypes.c_uint32
            lib.oracle_lhs_uniform.argtypes = [ctypes.c_uint64, ctypes.c_int32, ctypes.c_int64]
            lib.oracle_lhs_uniform.restype = ctypes.c_double
            lib.oracle_ppnd16.argtypes = [ctypes.c_double]
            lib.oracle_ppnd16.restype = ctypes.c_double
            lib.oracle_lhs_sample.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                              ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]
            lib.oracle_lhs_sample.restype = ctypes.c_int
            lib.oracle_kl_increment_basis.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_int32,
                                                      ctypes.c_void_p]
            lib.oracle_kl_path_basis.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_int32, ctypes.c_void_p]
            lib.oracle_em_increments.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32,
                                                 ctypes.c_int32, ctypes.c_double, ctypes.c_void_p]
            lib.oracle_em_normal.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32]
            lib.oracle_em_normal.restype = ctypes.c_double
            lib.oracle_ito_paths.argtypes = [ctypes.POINTER(_Ito), ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                             ctypes.c_double, ctypes.c_int32, ctypes.c_void_p]
            lib.oracle_kl_increment_basis_ex.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                                         ctypes.c_int32, ctypes.c_void_p]
            lib.oracle_kl_path_basis_ex.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                                    ctypes.c_int32, ctypes.c_void_p]
            lib.oracle_kle_reconstruct.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                                   ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]
            lib.oracle_electrical_power.argtypes = [ctypes.POINTER(_System), ctypes.c_void_p, ctypes.c_void_p,
                                                    ctypes.c_int32]
            lib.oracle_equilibrium.argtypes = [ctypes.POINTER(_System), ctypes.c_void_p, ctypes.c_void_p]
            lib.oracle_equilibrium.restype = ctypes.c_int
            lib.oracle_simulate.argtypes = [ctypes.POINTER(_System), ctypes.c_void_p, ctypes.c_int64,
                                            ctypes.c_int32, ctypes.c_int32] + [ctypes.c_void_p] * 7
            lib.oracle_simulate.restype = ctypes.c_int
            lib.oracle_ou_em.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_double, ctypes.c_void_p]
            lib.oracle_moments_twopass.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                                   ctypes.c_void_p, ctypes.c_void_p]
            lib.oracle_kl_forcing_basis_ex.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                                       ctypes.c_int32, ctypes.c_void_p]
            lib.oracle_smooth_paths.argtypes = [ctypes.POINTER(_System), ctypes.c_void_p, ctypes.c_int64,
                                                ctypes.c_int32, ctypes.c_void_p]
            lib.oracle_smooth_paths.restype = ctypes.c_int
            lib.oracle_plant_stage_forcing.argtypes = [ctypes.c_int32]
            lib.oracle_lhs_decorrelate.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
            lib.oracle_lhs_decorrelate.restype = ctypes.c_int
            lib.oracle_ito_objective.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                                 ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p]
            lib.oracle_ito_objective.restype = ctypes.c_double
            lib.oracle_ito_identify.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_int64, ctypes.c_double,
                                                ctypes.c_void_p]
            lib.oracle_ito_identify.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def philox4x32_10(ctr, key) -> np.ndarray:
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    u32p = ctypes.POINTER(ctypes.c_uint32)
    lib.oracle_philox4x32_10(c.ctypes.data_as(u32p), k.ctypes.data_as(u32p), out.ctypes.data_as(u32p))
    return out


def lhs_stratum(seed: int, N: int, dim: int, k: int) -> int:
    return int(_load().oracle_lhs_stratum(seed, N, dim, k))


def lhs_uniform(seed: int, dim: int, k: int) -> float:
    return float(_load().oracle_lhs_uniform(seed, dim, k))


def ppnd16(p: float) -> float:
    return float(_load().oracle_ppnd16(float(p)))


def lhs_sample(seed: int, N: int, M: int, mode: int = LHS, k0: int = 0, count: int | None = None,
               with_strata: bool = False):
    """Rows k0..k0+count-1 of the N-sample design: zeta [count, M] (and strata [M, count])."""
    count = N - k0 if count is None else count
    zeta = np.zeros((count, M), dtype=np.float64)
    strata = np.zeros((M, count), dtype=np.uint32) if with_strata else None
    rc = _load().oracle_lhs_sample(seed, N, k0, count, M, mode, _ptr(zeta), _ptr(strata))
    if rc != 0:
        raise ValueError("oracle_lhs_sample: invalid arguments")
    return (zeta, strata) if with_strata else zeta


def lhs_decorrelate(seed: int, N: int, M: int, mode: int = LHS, want_rstar: bool = False):
    """Section IV-B step 2 by the rank method of Iman and Conover: the N-sample
    design with each column rearranged so that the columns' correlation is
    minimised.  Returns (zeta [N, M], strata [M, N]) or, with want_rstar, also
    the decorrelated scores R* [N, M] whose ranks give the strata."""
    zeta = np.zeros((N, M), dtype=np.float64)
    strata = np.zeros((M, N), dtype=np.uint32)
    rstar = np.zeros((N, M), dtype=np.float64) if want_rstar else None
    rc = _load().oracle_lhs_decorrelate(seed, N, M, mode, _ptr(zeta), _ptr(strata), _ptr(rstar))
    if rc == -2:
        raise ValueError("oracle_lhs_decorrelate: the score correlation is not positive definite")
    if rc != 0:
        raise ValueError("oracle_lhs_decorrelate: invalid arguments (needs N > M and an LHS mode)")
    return (zeta, strata, rstar) if want_rstar else (zeta, strata)


ITO_SIGMA_POLY, ITO_SIGMA_SQUARED_POLY = 1, 2


def ito_objective(kind: int, q, xi, h: float, derivatives: bool = False):
    """The Appendix's objective L' (Eq. ident) of the record xi for the model
    mu = q0 + q1 x + q2 x^2 and sigma = q3 + q4 x + q5 x^2 (kind 1) or
    sigma^2 = q3 + q4 x + q5 x^2 (kind 2); with derivatives, (L', grad, Hessian)."""
    q = np.ascontiguousarray(q, dtype=np.float64)
    xi = np.ascontiguousarray(xi, dtype=np.float64)
    g = np.zeros(6) if derivatives else None
    H = np.zeros((6, 6)) if derivatives else None
    L = _load().oracle_ito_objective(kind, _ptr(q), _ptr(xi), xi.size, h, _ptr(g), _ptr(H))
    return (L, g, H) if derivatives else L


def ito_identify(kind: int, xi, h: float, q0):
    """Newton's method on L' from q0 -> (q, iterations); raises if it does not converge."""
    q = np.array(q0, dtype=np.float64)
    xi = np.ascontiguousarray(xi, dtype=np.float64)
    it = _load().oracle_ito_identify(kind, _ptr(xi), xi.size, h, _ptr(q))
    if it < 0:
        raise RuntimeError("oracle_ito_identify did not converge")
    return q, it


BASIS_SINE = 0    # Brownian eigenbasis (the Karhunen-Loeve basis of min(s, t))
BASIS_COSINE = 1  # the paper's Eq. (klb2)


def kl_increment_basis(K: int, T: float, Nt: int, basis: int = BASIS_SINE) -> np.ndarray:
    phi = np.zeros((K, Nt), dtype=np.float64)
    _load().oracle_kl_increment_basis_ex(basis, K, T, Nt, _ptr(phi))
    return phi


def kl_path_basis(K: int, T: float, Nt: int, basis: int = BASIS_SINE) -> np.ndarray:
    psi = np.zeros((K, Nt + 1), dtype=np.float64)
    _load().oracle_kl_path_basis_ex(basis, K, T, Nt, _ptr(psi))
    return psi


def kl_forcing_basis(K: int, T: float, Nt: int, basis: int = BASIS_SINE) -> np.ndarray:
    """m_k(j dt / 2), j = 0..2 Nt: the time derivatives of the KL basis functions (the
    smooth forcing of Eq. eqkl is sum_k zeta_k m_k(t)); [K, 2 Nt + 1]."""
    mdot = np.zeros((K, 2 * Nt + 1), dtype=np.float64)
    _load().oracle_kl_forcing_basis_ex(basis, K, T, Nt, _ptr(mdot))
    return mdot


def kle_reconstruct(zeta: np.ndarray, d: int, K: int, T: float, Nt: int, basis: int = BASIS_SINE) -> np.ndarray:
    zeta = np.ascontiguousarray(zeta, dtype=np.float64)
    count = zeta.shape[0]
    phi = kl_increment_basis(K, T, Nt, basis)
    dW = np.zeros((count, d, Nt), dtype=np.float64)
    _load().oracle_kle_reconstruct(_ptr(zeta), count, d, K, _ptr(phi), Nt, _ptr(dW))
    return dW


class _Holder:
    """Keeps the numpy arrays behind a _System alive."""

    def __init__(self, sc, integrator=None, init_delta=None):
        f = lambda a: np.ascontiguousarray(a, dtype=np.float64)
        self.arrays = {
            "G": f(sc.G), "B": f(sc.B), "H": f(sc.H), "D": f(sc.D), "E": f(sc.E), "Pm": f(sc.Pm),
            "theta": f(sc.theta), "sigma": f(sc.sigma), "inject": f(sc.inject),
            "Ginf": f(sc.Ginf if sc.has_inf_bus else np.zeros(sc.n)),
            "Binf": f(sc.Binf if sc.has_inf_bus else np.zeros(sc.n)),
        }
        s = _System()
        s.n, s.d, s.K, s.Nt = sc.n, sc.d, sc.K, sc.Nt
        s.T, s.dt, s.omega_s = float(sc.T), float(sc.dt), float(sc.omega_s)
        s.has_inf_bus = 1 if sc.has_inf_bus else 0
        s.integrator = int(sc.integrator if integrator is None else integrator)
        s.Vinf = float(sc.Vinf)
        s.basis = int(getattr(sc, "basis", BASIS_SINE))
        ev = getattr(sc, "event_machine", -1)
        s.event_machine = int(ev if ev is not None else -1)
        s.event_step = int(round(float(getattr(sc, "event_time", 0.0)) / float(sc.dt)))
        s.event_dpm = float(getattr(sc, "event_dpm", 0.0))
        s.smooth = 1 if int(getattr(sc, "forcing", 0)) == 1 else 0
        specs = getattr(sc, "ito", None)
        if specs is not None:
            self.ito = (_Ito * sc.d)(*[_ito_struct(sp) for sp in specs])
            s.ito = ctypes.cast(self.ito, ctypes.c_void_p)
        if init_delta is not None:
            self.arrays["init_delta"] = f(init_delta)
        for name, arr in self.arrays.items():
            setattr(s, name, arr.ctypes.data)
        self.s = s


def smooth_paths(sc, zeta, q: int = 0, integrator=None) -> np.ndarray:
    """Disturbance q alone under the smooth forcing (the random ODE of Eq. eqkl), by the
    scenario's integrator (or the one given) and the simulation's own step:
    x [count, Nt + 1] for the coefficient rows zeta [count, d K]."""
    h = _Holder(sc, integrator=integrator)
    zeta = np.ascontiguousarray(zeta, dtype=np.float64)
    count = zeta.shape[0]
    x = np.zeros((count, sc.Nt + 1), dtype=np.float64)
    rc = _load().oracle_smooth_paths(ctypes.byref(h.s), _ptr(zeta), count, q, _ptr(x))
    if rc != 0:
        raise ValueError("oracle_smooth_paths: invalid arguments")
    return x


def plant_stage_forcing(mode: int) -> None:
    """Test hook: plants a known mistake in the disturbance values the RK stages see
    (1: x_n at every stage; 2: x_{n+1} at the midpoint stages; 0: none), so that a
    pin can show it catches it.  Process-wide; reset to 0 after use."""
    _load().oracle_plant_stage_forcing(int(mode))


def electrical_power(sc, delta, form: int = PE_PAIRWISE) -> np.ndarray:
    h = _Holder(sc)
    delta = np.ascontiguousarray(delta, dtype=np.float64)
    pe = np.zeros(sc.n)
    _load().oracle_electrical_power(ctypes.byref(h.s), _ptr(delta), _ptr(pe), form)
    return pe


def equilibrium(sc):
    """Returns (delta0, pm_eq, iterations)."""
    h = _Holder(sc)
    delta0 = np.zeros(sc.n)
    pm_eq = np.zeros(sc.n)
    it = _load().oracle_equilibrium(ctypes.byref(h.s), _ptr(delta0), _ptr(pm_eq))
    if it < 0:
        raise RuntimeError("oracle equilibrium: Newton did not converge")
    return delta0, pm_eq, it


def simulate(sc, zeta: np.ndarray, *, want_traj: bool = False, want_dW: bool = False,
             want_moments: bool = True, pe_form: int = PE_PAIRWISE, nthreads: int = 1, integrator=None,
             init_delta=None):
    """Runs Algorithm 1 steps 2-4 on the given coefficient rows.

    Returns a dict with delta0, pm_eq and, on request, dW [S, d, Nt],
    traj [S, Nt+1, 2n] (delta_0..delta_{n-1}, domega_0..domega_{n-1}) and
    mean/var [Nt+1, 2n].  ``init_delta`` replaces the equilibrium angles as the
    initial state (speeds still start at zero).
    """
    h = _Holder(sc, integrator, init_delta)
    return _simulate_holder(h, sc, zeta, want_traj=want_traj, want_dW=want_dW, want_moments=want_moments,
                            pe_form=pe_form, nthreads=nthreads)


def _simulate_holder(h, sc, zeta, *, want_traj: bool = False, want_dW: bool = False, want_moments: bool = True,
                     pe_form: int = PE_PAIRWISE, nthreads: int = 1):
    zeta = np.ascontiguousarray(zeta, dtype=np.float64)
    S = zeta.shape[0]
    assert zeta.shape[1] == sc.d * sc.K
    n, Nt = sc.n, sc.Nt
    out = {"delta0": np.zeros(n), "pm_eq": np.zeros(n)}
    dW = np.zeros((S, sc.d, Nt)) if want_dW else None
    traj = np.zeros((S, Nt + 1, 2 * n)) if want_traj else None
    mean = np.zeros((Nt + 1, 2 * n)) if want_moments else None
    var = np.zeros((Nt + 1, 2 * n)) if want_moments else None
    rrf = np.zeros(S)
    rc = _load().oracle_simulate(ctypes.byref(h.s), _ptr(zeta), S, pe_form, nthreads, _ptr(out["delta0"]),
                                 _ptr(out["pm_eq"]), _ptr(dW), _ptr(traj), _ptr(mean), _ptr(var), _ptr(rrf))
    if rc != 0:
        raise RuntimeError(f"oracle_simulate failed ({rc})")
    if want_dW:
        out["dW"] = dW
    if want_traj:
        out["traj"] = traj
    if want_moments:
        out["mean"], out["var"] = mean, var
    # the response function of every sample (RMS centre-of-inertia speed deviation)
    out["rrf"] = rrf
    return out


def em_increments(seed: int, k0: int, count: int, d: int, Nt: int, dt: float) -> np.ndarray:
    """The "traditional MCs" increments (Eq. distito, fresh normal per step): dW [count, d, Nt]."""
    dW = np.zeros((count, d, Nt), dtype=np.float64)
    _load().oracle_em_increments(seed, k0, count, d, Nt, dt, _ptr(dW))
    return dW


def em_normal(seed: int, k: int, w: int, n: int) -> float:
    return float(_load().oracle_em_normal(seed, k, w, n))


def simulate_em(sc, k0: int = 0, count: int | None = None, **kw):
    """``simulate`` with the per-step normal increments of samples k0..k0+count-1
    (the paper's traditional Monte Carlo) instead of the KL expansion."""
    count = sc.N - k0 if count is None else count
    integrator = kw.pop("integrator", None)
    init_delta = kw.pop("init_delta", None)
    h = _Holder(sc, integrator, init_delta)
    h.s.em, h.s.em_seed, h.s.em_k0 = 1, int(sc.seed), int(k0)
    return _simulate_holder(h, sc, np.zeros((count, sc.d * sc.K)), **kw)


def ito_paths(spec, dW: np.ndarray, dt: float, stratonovich: bool) -> np.ndarray:
    """Paths x [S, Nt+1] of a general disturbance (Table I / Eq. windito) driven by
    increments dW [S, Nt]; stratonovich: subtract sigma sigma'/2 from the drift
    (increments of a smooth KL path)."""
    dW = np.ascontiguousarray(dW, dtype=np.float64)
    S, Nt = dW.shape
    x = np.zeros((S, Nt + 1))
    it = _ito_struct(spec)
    _load().oracle_ito_paths(ctypes.byref(it), _ptr(dW), S, Nt, dt, 1 if stratonovich else 0, _ptr(x))
    return x


def ou_em(dW: np.ndarray, dt: float, theta: float, sigma: float) -> np.ndarray:
    """OU paths x [S, Nt+1] driven by increments dW [S, Nt]."""
    dW = np.ascontiguousarray(dW, dtype=np.float64)
    S, Nt = dW.shape
    x = np.zeros((S, Nt + 1))
    _load().oracle_ou_em(_ptr(dW), S, Nt, dt, theta, sigma, _ptr(x))
    return x


def moments_twopass(x: np.ndarray):
    x = np.ascontiguousarray(x, dtype=np.float64)
    N = x.shape[0]
    C = int(np.prod(x.shape[1:])) if x.ndim > 1 else 1
    mean = np.zeros(C)
    var = np.zeros(C)
    _load().oracle_moments_twopass(_ptr(x), N, C, _ptr(mean), _ptr(var))
    shape = x.shape[1:]
    return mean.reshape(shape), var.reshape(shape)
