"""GB300 (sm_103a) implementation of the fast Monte Carlo method of Qiu et al.,
"Fast Monte Carlo Simulation of Dynamic Power Systems Under Continuous Random
Disturbances" (arXiv 2007.03847).

The compute path lives in ``lib/libfastmc.so`` (CUDA C++ with a C ABI declared
in ``include/fastmc.h``).  This module only marshals arguments: PyTorch tensors
supply device memory and the current CUDA stream; every step of Algorithm 1 runs
in the library's kernels.  There is no CPU fallback: if the library is missing
or no GPU is present, the calls raise.

Entry points (same names as the C ABI without the ``fmc_`` prefix):
``lhs_sample``, ``lhs_sample_split``, ``kl_basis``, ``kle_reconstruct``,
``equilibrium``, ``simulate``, ``simulate_sums``, ``simulate_rrf``, ``moments``,
``lhs_decorrelate``, ``ito_objective``, ``ito_identify``, the ``Batch`` and
``Server`` forms, plus ``Context``, ``device_status``, the fused kernel's choice
(``set_kernel_policy``: "auto", "per_sample", "split", "split_tc";
``set_launch_rules``) and the diagnostics of ``include/fastmc_diag.h``
(``profile``/``profile_read``, ``check_wait_path``, ``kernel_choice``,
``net_matrix``).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# FASTMC_LIB may point at another build of the same library (A/B comparisons)
LIB_PATH = os.environ.get("FASTMC_LIB") or os.path.join(HERE, "lib", "libfastmc.so")

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, NOT_READY, EBUSY, ECANCELLED, EUNSUPPORTED, ENOCONVERGE = range(10)
LHS, SRS, LHS_MIDPOINT, SRS_EM = 0, 1, 2, 3
PREC_F32, PREC_BF16, PREC_BF16X3 = 0, 1, 2
RK4, HEUN = 0, 1
PATH_FUSED, PATH_PLAIN = 0, 1
PH_LHS, PH_BASIS, PH_EQ, PH_FUSED, PH_REDUCE, PH_CONTRACT, PH_INTEGRATE, PH_MOMENTS, PH_BATCH = range(9)
MAX_MACHINES, MAX_MACHINES_PLAIN, MAX_DISTURBANCES = 52, 16, 8

_PRECISION = {"f32": PREC_F32, "bf16": PREC_BF16, "bf16x3": PREC_BF16X3}
_PATH = {"fused": PATH_FUSED, "plain": PATH_PLAIN}


class FastMCError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"fastmc error {code}: {msg}")
        self.code = code


class _Ito(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("reserved", ctypes.c_int32), ("m", ctypes.c_double * 3),
                ("s", ctypes.c_double * 3), ("v", ctypes.c_double * 4), ("a", ctypes.c_double),
                ("x0", ctypes.c_double)]


ITO_OU, ITO_POLY, ITO_SQRT = 0, 1, 2


class _Scenario(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int32), ("d", ctypes.c_int32), ("K", ctypes.c_int32), ("sampling", ctypes.c_int32),
        ("T", ctypes.c_double), ("dt", ctypes.c_double), ("N", ctypes.c_int64), ("seed", ctypes.c_uint64),
        ("precision", ctypes.c_int32), ("integrator", ctypes.c_int32), ("has_inf_bus", ctypes.c_int32),
        ("basis", ctypes.c_int32), ("omega_s", ctypes.c_double), ("Vinf", ctypes.c_double),
        ("G", ctypes.c_void_p), ("B", ctypes.c_void_p), ("Ginf", ctypes.c_void_p), ("Binf", ctypes.c_void_p),
        ("H", ctypes.c_void_p), ("D", ctypes.c_void_p), ("E", ctypes.c_void_p), ("Pm", ctypes.c_void_p),
        ("theta", ctypes.c_void_p), ("sigma", ctypes.c_void_p), ("inject", ctypes.c_void_p),
        ("event_machine", ctypes.c_int32), ("forcing", ctypes.c_int32), ("event_time", ctypes.c_double),
        ("event_dpm", ctypes.c_double), ("ito", ctypes.c_void_p), ("correlation", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
    ]


class LaunchRule(ctypes.Structure):
    """fmc_launch_rule: a measured launch shape for a range of (n, d, N)."""
    _fields_ = [("n_min", ctypes.c_int32), ("n_max", ctypes.c_int32), ("d_min", ctypes.c_int32),
                ("d_max", ctypes.c_int32), ("N_min", ctypes.c_int64), ("N_max", ctypes.c_int64),
                ("kernel", ctypes.c_int32), ("max_ctas", ctypes.c_int32), ("TC", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class _Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("replicates", ctypes.c_int32), ("latency_us", ctypes.c_double),
                ("queue_us", ctypes.c_double), ("device_bytes", ctypes.c_uint64), ("n_used", ctypes.c_int64),
                ("err_E", ctypes.c_double), ("err_Var", ctypes.c_double), ("target_met", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("message", ctypes.c_char * 256)]


_lib = None
_lib_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compiles libfastmc.so in-tree with nvcc (sm_103a)."""
    from . import _buildlib
    return _buildlib.build(force=force)


def load_library():
    """Loads libfastmc.so; raises if it has not been built."""
    global _lib
    with _lib_lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise FastMCError(ECUDA, f"{LIB_PATH} is missing: build it with paper_2007_03847_gb300.build()")
        lib = ctypes.CDLL(LIB_PATH)
        vp, i32, i64, u64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
        sig = {
            "fmc_create": ([ctypes.POINTER(vp), ctypes.c_int, ctypes.c_size_t], ctypes.c_int),
            "fmc_destroy": ([vp], ctypes.c_int),
            "fmc_last_error": ([vp], ctypes.c_char_p),
            "fmc_device_info": ([vp, ctypes.POINTER(ctypes.c_int), ctypes.c_char_p, ctypes.c_size_t], ctypes.c_int),
            "fmc_lhs_sample": ([vp, u64, i64, i64, i64, i32, i32, vp, vp, vp], ctypes.c_int),
            "fmc_lhs_sample_split": ([vp, u64, i64, i64, i64, i32, i32, i32, vp, vp, vp], ctypes.c_int),
            "fmc_kl_basis": ([vp, i32, dbl, i32, i32, vp, vp], ctypes.c_int),
            "fmc_kle_reconstruct": ([vp, vp, i64, i32, i32, dbl, dbl, i32, vp, vp], ctypes.c_int),
            "fmc_equilibrium": ([vp, ctypes.POINTER(_Scenario), vp, vp], ctypes.c_int),
            "fmc_simulate": ([vp, ctypes.POINTER(_Scenario), i32, vp, vp, vp, vp], ctypes.c_int),
            "fmc_moments": ([vp, vp, i64, i64, vp, vp, vp], ctypes.c_int),
            "fmc_device_status": ([vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
            "fmc_profile": ([vp, i32, i64], ctypes.c_int),
            "fmc_profile_read": ([vp, i32, ctypes.POINTER(dbl), ctypes.POINTER(i64)], ctypes.c_int),
            "fmc_last_fused_occupancy": ([vp, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
            "fmc_diag_net_matrix": ([vp, i32, i32, vp, i64], ctypes.c_int),
            "fmc_diag_kernel_choice": ([vp, i32, i32, i64, vp], ctypes.c_int),
            "fmc_set_kernel_policy": ([vp, ctypes.c_int32], ctypes.c_int),
            "fmc_test_sincos": ([vp, vp, i64, vp, vp, vp, vp, vp], ctypes.c_int),
            "fmc_batch_create": ([vp, ctypes.POINTER(_Scenario), i32, i32, ctypes.POINTER(vp), ctypes.POINTER(vp),
                                  i32, ctypes.POINTER(vp)], ctypes.c_int),
            "fmc_batch_launch": ([vp, vp], ctypes.c_int),
            "fmc_batch_destroy": ([vp], ctypes.c_int),
            "fmc_simulate_batch": ([vp, ctypes.POINTER(_Scenario), i32, i32, ctypes.POINTER(vp), ctypes.POINTER(vp),
                                    vp], ctypes.c_int),
            "fmc_server_create": ([ctypes.c_int, i32, ctypes.c_size_t, ctypes.POINTER(vp)], ctypes.c_int),
            "fmc_server_destroy": ([vp], ctypes.c_int),
            "fmc_submit": ([vp, ctypes.POINTER(_Scenario), i32, vp, vp, ctypes.POINTER(u64)], ctypes.c_int),
            "fmc_simulate_rrf": ([vp, ctypes.POINTER(_Scenario), i32, vp, vp, vp, vp], ctypes.c_int),
            "fmc_submit_target": ([vp, ctypes.POINTER(_Scenario), i32, dbl, dbl, i64, vp, vp, ctypes.POINTER(u64)],
                                  ctypes.c_int),
            "fmc_poll": ([vp, u64, ctypes.POINTER(_Result)], ctypes.c_int),
            "fmc_wait": ([vp, u64, i64, ctypes.POINTER(_Result)], ctypes.c_int),
            "fmc_cancel": ([vp, u64], ctypes.c_int),
            "fmc_server_stats": ([vp, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_size_t)],
                                 ctypes.c_int),
            "fmc_kle_reconstruct_noalloc": ([vp, vp, i64, i32, i32, dbl, dbl, i32, vp, vp], ctypes.c_int),
            "fmc_check_wait_path": ([vp, i32, i64, vp], ctypes.c_int),
            "fmc_lhs_decorrelate": ([vp, u64, i64, i32, i32, vp, vp, vp], ctypes.c_int),
            "fmc_set_launch_rules": ([vp, ctypes.POINTER(LaunchRule), i32], ctypes.c_int),
            "fmc_ito_objective": ([vp, i32, vp, vp, i64, dbl, ctypes.POINTER(dbl), vp, vp, vp], ctypes.c_int),
            "fmc_ito_identify": ([vp, i32, vp, i64, dbl, vp, ctypes.POINTER(i32), vp], ctypes.c_int),
            "fmc_simulate_sums": ([vp, ctypes.POINTER(_Scenario), i64, i64, i32, vp, vp, vp, vp, vp], ctypes.c_int),
            "fmc_moments_from_sums": ([vp, vp, vp, vp, i64, i64, i32, vp, vp, vp], ctypes.c_int),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


class Context:
    """A library context on one CUDA device (workspace, kernel timing)."""

    def __init__(self, device: int = 0, mem_budget_bytes: int = 0):
        import torch
        if not torch.cuda.is_available():
            raise FastMCError(ECUDA, "no CUDA device is available")
        torch.cuda.init()
        self.lib = load_library()
        self.device = device
        h = ctypes.c_void_p()
        rc = self.lib.fmc_create(ctypes.byref(h), device, mem_budget_bytes)
        if rc != OK:
            raise FastMCError(rc, self.lib.fmc_last_error(None).decode())
        self.h = h
        # the launch shapes the autotuner measured on this GPU model, if cached
        from . import autotune
        autotune.apply_cached(self)

    def close(self):
        if getattr(self, "h", None):
            self.lib.fmc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self, rc: int):
        if rc != OK:
            raise FastMCError(rc, self.lib.fmc_last_error(self.h).decode())

    def info(self):
        sms = ctypes.c_int()
        name = ctypes.create_string_buffer(256)
        self.check(self.lib.fmc_device_info(self.h, ctypes.byref(sms), name, 256))
        return sms.value, name.value.decode()


_default_ctx = None


def default_context() -> Context:
    global _default_ctx
    if _default_ctx is None:
        _default_ctx = Context(0)
    return _default_ctx


def _stream(stream=None):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise FastMCError(EINVAL, "device tensor expected")
    if not t.is_contiguous():
        raise FastMCError(EINVAL, "contiguous tensor expected")
    return ctypes.c_void_p(t.data_ptr())


class ScenarioStruct:
    """fmc_scenario built from an object with the fields of fmc_synth.Scenario."""

    def __init__(self, sc, precision=None, sampling=None, integrator=None):
        f = lambda a: np.ascontiguousarray(np.asarray(a, dtype=np.float64))
        self.keep = {k: f(getattr(sc, k)) for k in ("G", "B", "H", "D", "E", "Pm", "theta", "sigma", "inject")}
        s = _Scenario()
        s.n, s.d, s.K = int(sc.n), int(sc.d), int(sc.K)
        s.sampling = int(getattr(sc, "sampling", LHS) if sampling is None else sampling)
        s.T, s.dt, s.N, s.seed = float(sc.T), float(sc.dt), int(sc.N), int(sc.seed)
        prec = getattr(sc, "precision", PREC_BF16X3) if precision is None else precision
        s.precision = _PRECISION.get(prec, prec) if isinstance(prec, str) else int(prec)
        s.integrator = int(getattr(sc, "integrator", RK4) if integrator is None else integrator)
        s.has_inf_bus = 1 if sc.has_inf_bus else 0
        s.basis = int(getattr(sc, "basis", BASIS_SINE))
        s.forcing = int(getattr(sc, "forcing", FORCING_INCREMENTS))
        s.correlation = int(getattr(sc, "correlation", CORR_NONE))
        specs = getattr(sc, "ito", None)
        if specs is not None:
            arr = (_Ito * int(sc.d))()
            for q, sp in enumerate(specs):
                it = arr[q]
                if sp is None:
                    continue
                it.kind = int(sp["kind"])
                it.m[:] = [float(c) for c in sp["m"]]
                if it.kind == ITO_POLY:
                    it.s[:] = [float(c) for c in sp["s"]]
                elif it.kind == ITO_SQRT:
                    it.v[:] = [float(c) for c in sp["v"]]
                it.a = float(sp.get("a", 0.0))
                it.x0 = float(sp.get("x0", 0.0))
            self.ito = arr
            s.ito = ctypes.cast(arr, ctypes.c_void_p)
        ev = getattr(sc, "event_machine", None)
        s.event_machine = -1 if ev is None else int(ev)
        s.event_time = float(getattr(sc, "event_time", 0.0))
        s.event_dpm = float(getattr(sc, "event_dpm", 0.0))
        s.omega_s, s.Vinf = float(sc.omega_s), float(sc.Vinf)
        if sc.has_inf_bus:
            self.keep["Ginf"] = f(sc.Ginf)
            self.keep["Binf"] = f(sc.Binf)
        for k, a in self.keep.items():
            setattr(s, k, a.ctypes.data)
        self.s = s
        self.Nt = int(round(sc.T / sc.dt))


# ---------------------------------------------------------------------------- entry points


def lhs_sample(seed: int, N: int, M: int, mode: int = LHS, k0: int = 0, count: int | None = None, zeta=None,
               strata=None, ctx: Context | None = None, stream=None):
    """Algorithm 1 step 1: rows k0..k0+count-1 of the N-sample design -> zeta [count, M] float32."""
    import torch
    ctx = ctx or default_context()
    count = N - k0 if count is None else count
    if zeta is None:
        zeta = torch.empty((count, M), dtype=torch.float32, device="cuda")
    ctx.check(ctx.lib.fmc_lhs_sample(ctx.h, seed, N, k0, count, M, mode, _ptr(zeta), _ptr(strata), _stream(stream)))
    return zeta, strata


def lhs_decorrelate(seed: int, N: int, M: int, mode: int = LHS, zeta=None, strata=None,
                    ctx: "Context | None" = None, stream=None):
    """fmc_lhs_decorrelate: the N x M design with the correlation-reducing
    permutation (Section IV-B step 2) -> (zeta [N, M] float32, strata [M, N] int32
    holding uint32 values) device tensors."""
    import torch
    ctx = ctx or default_context()
    zeta = torch.empty((N, M), dtype=torch.float32, device="cuda") if zeta is None else zeta
    strata = torch.empty((M, N), dtype=torch.int32, device="cuda") if strata is None else strata
    ctx.check(ctx.lib.fmc_lhs_decorrelate(ctx.h, seed, N, M, mode, _ptr(zeta), _ptr(strata), _stream(stream)))
    return zeta, strata


IDENT_SIGMA, IDENT_SIGMA2 = 1, 2


def ito_objective(kind: int, q, xi, h: float, derivatives: bool = False, ctx: "Context | None" = None, stream=None):
    """fmc_ito_objective: the Appendix's L' of the device record xi (float64) at q;
    with derivatives (L', grad [6], Hessian [6, 6]) as numpy arrays."""
    ctx = ctx or default_context()
    qa = np.ascontiguousarray(q, dtype=np.float64)
    L = ctypes.c_double()
    g = np.zeros(6) if derivatives else None
    H = np.zeros((6, 6)) if derivatives else None
    ctx.check(ctx.lib.fmc_ito_objective(ctx.h, kind, qa.ctypes.data_as(ctypes.c_void_p), _ptr(xi), xi.numel(), h,
                                        ctypes.byref(L), None if g is None else g.ctypes.data_as(ctypes.c_void_p),
                                        None if H is None else H.ctypes.data_as(ctypes.c_void_p), _stream(stream)))
    return (L.value, g, H) if derivatives else L.value


def ito_identify(kind: int, xi, h: float, q0, ctx: "Context | None" = None, stream=None):
    """fmc_ito_identify: Newton's method on L' from q0 over the device record xi
    (float64) -> (q numpy [6], iterations)."""
    ctx = ctx or default_context()
    q = np.array(q0, dtype=np.float64)
    it = ctypes.c_int32()
    ctx.check(ctx.lib.fmc_ito_identify(ctx.h, kind, _ptr(xi), xi.numel(), h, q.ctypes.data_as(ctypes.c_void_p),
                                       ctypes.byref(it), _stream(stream)))
    return q, it.value


def lhs_sample_split(seed: int, N: int, d: int, K: int, mode: int = LHS, k0: int = 0, count: int | None = None,
                     ctx: Context | None = None, stream=None):
    """Split-BF16 design [count, d, round_up(K, 8)] as (hi, lo) bfloat16 tensors."""
    import torch
    ctx = ctx or default_context()
    count = N - k0 if count is None else count
    Ks = (K + 7) // 8 * 8
    hi = torch.empty((count, d, Ks), dtype=torch.bfloat16, device="cuda")
    lo = torch.empty_like(hi)
    ctx.check(ctx.lib.fmc_lhs_sample_split(ctx.h, seed, N, k0, count, d, K, mode, _ptr(hi), _ptr(lo),
                                           _stream(stream)))
    return hi, lo


BASIS_SINE, BASIS_COSINE = 0, 1
FORCING_INCREMENTS, FORCING_SMOOTH = 0, 1
CORR_NONE, CORR_RANK = 0, 1


def kl_basis(K: int, T: float, Nt: int, basis: int = BASIS_SINE, phi=None, ctx: Context | None = None,
             stream=None):
    """Increment basis phi [K, Nt] float32 (FP64 on the GPU, rounded)."""
    import torch
    ctx = ctx or default_context()
    if phi is None:
        phi = torch.empty((K, Nt), dtype=torch.float32, device="cuda")
    ctx.check(ctx.lib.fmc_kl_basis(ctx.h, K, T, Nt, int(basis), _ptr(phi), _stream(stream)))
    return phi


def kle_reconstruct(zeta, d: int, K: int, T: float, dt: float, precision="f32", dW=None, ctx: Context | None = None,
                    stream=None):
    """Algorithm 1 step 2: increments dW [count, d, Nt] float32 from zeta [count, d*K]."""
    import torch
    ctx = ctx or default_context()
    count = zeta.shape[0]
    Nt = int(round(T / dt))
    prec = _PRECISION.get(precision, precision) if isinstance(precision, str) else precision
    if dW is None:
        dW = torch.empty((count, d, Nt), dtype=torch.float32, device="cuda")
    ctx.check(ctx.lib.fmc_kle_reconstruct(ctx.h, _ptr(zeta), count, d, K, T, dt, prec, _ptr(dW), _stream(stream)))
    return dW


def kle_reconstruct_noalloc(zeta, d: int, K: int, T: float, dt: float, precision="bf16x3", dW=None,
                            ctx: Context | None = None, stream=None):
    """fmc_kle_reconstruct_noalloc: the same increments as kle_reconstruct, computed with
    the library's fixed scratch array instead of allocated working memory.  The
    caller provides dW (or this wrapper creates it, which allocates through torch)."""
    import torch
    ctx = ctx or default_context()
    count = zeta.shape[0]
    Nt = int(round(T / dt))
    prec = _PRECISION.get(precision, precision) if isinstance(precision, str) else precision
    if dW is None:
        dW = torch.empty((count, d, Nt), dtype=torch.float32, device="cuda")
    ctx.check(ctx.lib.fmc_kle_reconstruct_noalloc(ctx.h, _ptr(zeta), count, d, K, T, dt, prec, _ptr(dW),
                                                  _stream(stream)))
    return dW


def equilibrium(scenario, ctx: Context | None = None):
    """FP64 Newton equilibrium on the GPU -> (delta0, pm_eq) numpy arrays."""
    ctx = ctx or default_context()
    ss = ScenarioStruct(scenario)
    delta0 = np.zeros(scenario.n)
    pm = np.zeros(scenario.n)
    ctx.check(ctx.lib.fmc_equilibrium(ctx.h, ctypes.byref(ss.s), delta0.ctypes.data_as(ctypes.c_void_p),
                                      pm.ctypes.data_as(ctypes.c_void_p)))
    return delta0, pm


def simulate(scenario, path="fused", precision=None, sampling=None, integrator=None, mean=None, var=None,
             traj=None, want_traj: bool = False, ctx: Context | None = None, stream=None):
    """Algorithm 1 steps 1-4 for one scenario.

    Returns (mean, var[, traj]) as device tensors: mean/var [Nt+1, 2n] float64,
    traj [N, Nt+1, 2n] float32 when requested.
    """
    import torch
    ctx = ctx or default_context()
    p = _PATH.get(path, path) if isinstance(path, str) else path
    if precision is None:
        precision = "f32" if p == PATH_PLAIN else "bf16x3"
    ss = ScenarioStruct(scenario, precision=precision, sampling=sampling, integrator=integrator)
    Nt1, S = ss.Nt + 1, 2 * scenario.n
    if mean is None:
        mean = torch.empty((Nt1, S), dtype=torch.float64, device="cuda")
    if var is None:
        var = torch.empty((Nt1, S), dtype=torch.float64, device="cuda")
    if want_traj and traj is None:
        traj = torch.empty((scenario.N, Nt1, S), dtype=torch.float32, device="cuda")
    ctx.check(ctx.lib.fmc_simulate(ctx.h, ctypes.byref(ss.s), p, _ptr(mean), _ptr(var), _ptr(traj),
                                   _stream(stream)))
    return (mean, var, traj) if (want_traj or traj is not None) else (mean, var)


def simulate_rrf(scenario, path="fused", precision=None, sampling=None, integrator=None, ctx: Context | None = None,
                 stream=None):
    """The paper's response function (RMS of the centre-of-inertia speed deviation over
    the horizon) of every sample, reduced to (E[RRF], Var[RRF]) as a [2] float64 device
    tensor, with the moment trajectories mean, var [Nt+1, 2n]."""
    import torch
    ctx = ctx or default_context()
    p = _PATH.get(path, path) if isinstance(path, str) else path
    if precision is None:
        precision = "f32" if p == PATH_PLAIN else "bf16x3"
    ss = ScenarioStruct(scenario, precision=precision, sampling=sampling, integrator=integrator)
    rrf = torch.empty(2, dtype=torch.float64, device="cuda")
    mean = torch.empty((ss.Nt + 1, 2 * scenario.n), dtype=torch.float64, device="cuda")
    var = torch.empty_like(mean)
    ctx.check(ctx.lib.fmc_simulate_rrf(ctx.h, ctypes.byref(ss.s), p, _ptr(rrf), _ptr(mean), _ptr(var),
                                       _stream(stream)))
    return rrf, mean, var


def simulate_sums(scenario, k0: int, count: int, path="fused", precision=None, sampling=None, integrator=None,
                  traj=None, ctx: Context | None = None, stream=None):
    """Samples k0..k0+count-1 of the design -> (S1, S2, shift) device float64 tensors:
    S1, S2 [Nt+1, 2n] shifted sums, shift [2n]."""
    import torch
    ctx = ctx or default_context()
    p = _PATH.get(path, path) if isinstance(path, str) else path
    if precision is None:
        precision = "f32" if p == PATH_PLAIN else "bf16x3"
    ss = ScenarioStruct(scenario, precision=precision, sampling=sampling, integrator=integrator)
    Nt1, S = ss.Nt + 1, 2 * scenario.n
    S1 = torch.empty((Nt1, S), dtype=torch.float64, device="cuda")
    S2 = torch.empty_like(S1)
    shift = torch.empty(S, dtype=torch.float64, device="cuda")
    ctx.check(ctx.lib.fmc_simulate_sums(ctx.h, ctypes.byref(ss.s), k0, count, p, _ptr(S1), _ptr(S2), _ptr(shift),
                                        _ptr(traj), _stream(stream)))
    return S1, S2, shift


def moments_from_sums(S1, S2, shift, N: int, mean=None, var=None, ctx: Context | None = None, stream=None):
    """mean, var [rows, S] float64 from shifted sums over N samples."""
    import torch
    ctx = ctx or default_context()
    rows, S = S1.shape
    mean = torch.empty_like(S1) if mean is None else mean
    var = torch.empty_like(S1) if var is None else var
    ctx.check(ctx.lib.fmc_moments_from_sums(ctx.h, _ptr(S1), _ptr(S2), _ptr(shift), N, rows, S, _ptr(mean),
                                            _ptr(var), _stream(stream)))
    return mean, var


class Batch:
    """fmc_batch: many scenarios run concurrently; with use_graph the whole batch is one
    captured CUDA graph that launch() replays.  Results: self.mean[i], self.var[i]
    ([Nt_i+1, 2 n_i] float64 device tensors)."""

    def __init__(self, scenarios, path="fused", precision=None, use_graph: bool = True, ctx: Context | None = None):
        import torch
        self.ctx = ctx or default_context()
        p = _PATH.get(path, path) if isinstance(path, str) else path
        if precision is None:
            precision = "f32" if p == PATH_PLAIN else "bf16x3"
        self.structs = [ScenarioStruct(sc, precision=precision) for sc in scenarios]
        arr = (_Scenario * len(scenarios))(*[ss.s for ss in self.structs])
        self.mean = [torch.empty((ss.Nt + 1, 2 * sc.n), dtype=torch.float64, device="cuda")
                     for ss, sc in zip(self.structs, scenarios)]
        self.var = [torch.empty_like(m) for m in self.mean]
        mp = (ctypes.c_void_p * len(scenarios))(*[m.data_ptr() for m in self.mean])
        vp_ = (ctypes.c_void_p * len(scenarios))(*[v.data_ptr() for v in self.var])
        h = ctypes.c_void_p()
        self.ctx.check(self.ctx.lib.fmc_batch_create(self.ctx.h, arr, len(scenarios), p, mp, vp_,
                                                     1 if use_graph else 0, ctypes.byref(h)))
        self.h = h

    def launch(self, stream=None):
        self.ctx.check(self.ctx.lib.fmc_batch_launch(self.h, _stream(stream)))
        return self.mean, self.var

    def close(self):
        if getattr(self, "h", None):
            self.ctx.lib.fmc_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """fmc_server: requests admitted by device memory into `slots` concurrent slots.

    submit() returns a handle; poll()/wait() return (result dict, mean, var) once the
    request is done (mean/var: [Nt+1, 2n] float64 device tensors), or None.
    """

    def __init__(self, device: int = 0, slots: int = 8, mem_budget_bytes: int = 0):
        import torch
        if not torch.cuda.is_available():
            raise FastMCError(ECUDA, "no CUDA device is available")
        torch.cuda.init()
        self.lib = load_library()
        h = ctypes.c_void_p()
        rc = self.lib.fmc_server_create(device, slots, mem_budget_bytes, ctypes.byref(h))
        if rc != OK:
            raise FastMCError(rc, "fmc_server_create failed")
        self.h = h
        self.pending = {}

    def submit(self, scenario, path="fused", precision="bf16x3", tol_E: float = 0.0, tol_Var: float = 0.0,
               max_N: int = 0):
        """Queues a request.  With tol_E or tol_Var > 0 the server draws four
        independent designs of scenario.N samples, growing N until the replicate
        spread meets the targets or 4 N would pass max_N (fmc_submit_target)."""
        import torch
        p = _PATH.get(path, path) if isinstance(path, str) else path
        ss = ScenarioStruct(scenario, precision=precision)
        mean = torch.empty((ss.Nt + 1, 2 * scenario.n), dtype=torch.float64, device="cuda")
        var = torch.empty_like(mean)
        hd = ctypes.c_uint64()
        if tol_E > 0 or tol_Var > 0:
            rc = self.lib.fmc_submit_target(self.h, ctypes.byref(ss.s), p, float(tol_E), float(tol_Var), int(max_N),
                                            _ptr(mean), _ptr(var), ctypes.byref(hd))
        else:
            rc = self.lib.fmc_submit(self.h, ctypes.byref(ss.s), p, _ptr(mean), _ptr(var), ctypes.byref(hd))
        if rc != OK:
            raise FastMCError(rc, "fmc_submit failed")
        self.pending[hd.value] = (mean, var)
        return hd.value

    def _finish(self, handle, res):
        mean, var = self.pending.pop(handle)
        out = {"status": res.status, "latency_us": res.latency_us, "queue_us": res.queue_us,
               "device_bytes": res.device_bytes, "n_used": res.n_used, "replicates": res.replicates,
               "err_E": res.err_E, "err_Var": res.err_Var, "target_met": bool(res.target_met),
               "message": res.message.decode()}
        return out, mean, var

    def poll(self, handle):
        res = _Result()
        rc = self.lib.fmc_poll(self.h, handle, ctypes.byref(res))
        if rc == NOT_READY:
            return None
        if rc != OK:
            raise FastMCError(rc, "fmc_poll failed")
        return self._finish(handle, res)

    def wait(self, handle, timeout_s: float = 60.0):
        res = _Result()
        rc = self.lib.fmc_wait(self.h, handle, int(timeout_s * 1e6), ctypes.byref(res))
        if rc == ETIMEOUT:
            return None
        if rc != OK:
            raise FastMCError(rc, "fmc_wait failed")
        return self._finish(handle, res)

    def cancel(self, handle) -> int:
        return self.lib.fmc_cancel(self.h, handle)

    def stats(self):
        q, r, b = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_size_t()
        self.lib.fmc_server_stats(self.h, ctypes.byref(q), ctypes.byref(r), ctypes.byref(b))
        return {"queued": q.value, "running": r.value, "bytes_in_use": b.value}

    def close(self):
        if getattr(self, "h", None):
            self.lib.fmc_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def moments(x, mean=None, var=None, ctx: Context | None = None, stream=None):
    """Algorithm 1 step 4: column mean and unbiased variance of x [N, C] float32 -> float64 [C]."""
    import torch
    ctx = ctx or default_context()
    N = x.shape[0]
    C = int(np.prod(x.shape[1:])) if x.dim() > 1 else 1
    if mean is None:
        mean = torch.empty(x.shape[1:], dtype=torch.float64, device="cuda")
    if var is None:
        var = torch.empty(x.shape[1:], dtype=torch.float64, device="cuda")
    ctx.check(ctx.lib.fmc_moments(ctx.h, _ptr(x), N, C, _ptr(mean), _ptr(var), _stream(stream)))
    return mean, var


def device_status(ctx: Context | None = None):
    """(equilibrium iterations, kernel error code) after synchronising; raises on errors."""
    ctx = ctx or default_context()
    it, err = ctypes.c_int(), ctypes.c_int()
    ctx.check(ctx.lib.fmc_device_status(ctx.h, ctypes.byref(it), ctypes.byref(err)))
    return it.value, err.value


def check_wait_path(target: int = 0, poll_limit: int = 1000, ctx: Context | None = None, stream=None):
    """fmc_check_wait_path: a bounded device wait that runs out on purpose (no fault);
    the next device_status raises FastMCError with code ETIMEOUT.  target 0: the
    context's status word; 1: the allocation-free reconstruction's."""
    ctx = ctx or default_context()
    ctx.check(ctx.lib.fmc_check_wait_path(ctx.h, target, poll_limit, _stream(stream)))


def profile(enable: bool, max_records: int = 100000, ctx: Context | None = None):
    ctx = ctx or default_context()
    ctx.check(ctx.lib.fmc_profile(ctx.h, 1 if enable else 0, max_records))


def profile_read(phase: int, ctx: Context | None = None):
    """(total milliseconds, launches) of one kernel phase since profiling was enabled."""
    ctx = ctx or default_context()
    ms, cnt = ctypes.c_double(), ctypes.c_int64()
    ctx.check(ctx.lib.fmc_profile_read(ctx.h, phase, ctypes.byref(ms), ctypes.byref(cnt)))
    return ms.value, cnt.value


def test_sincos(x, ctx: Context | None = None, stream=None):
    """The integrator's sin/cos and CUDA's sincosf on x (float32 device tensor)."""
    import torch
    ctx = ctx or default_context()
    outs = [torch.empty_like(x) for _ in range(4)]
    ctx.check(ctx.lib.fmc_test_sincos(ctx.h, _ptr(x), x.numel(), *[_ptr(o) for o in outs], _stream(stream)))
    return outs


KERNEL_AUTO, KERNEL_PER_SAMPLE, KERNEL_SPLIT, KERNEL_SPLIT_TC = 0, 1, 2, 3
_KERNEL = {"auto": KERNEL_AUTO, "per_sample": KERNEL_PER_SAMPLE, "split": KERNEL_SPLIT,
           "split_tc": KERNEL_SPLIT_TC}


def set_launch_rules(rules, ctx: "Context | None" = None) -> None:
    """fmc_set_launch_rules from dicts with the fields of LaunchRule (missing
    fields: the whole range / 0); an empty list clears the rules."""
    ctx = ctx or default_context()
    arr = (LaunchRule * max(1, len(rules)))()
    for k, r in enumerate(rules):
        arr[k] = LaunchRule(int(r.get("n_min", 1)), int(r.get("n_max", 1 << 30)), int(r.get("d_min", 1)),
                            int(r.get("d_max", 1 << 30)), int(r.get("N_min", 1)), int(r.get("N_max", 1 << 62)),
                            int(r.get("kernel", 0)), int(r.get("max_ctas", 0)), int(r.get("TC", 0)), 0)
    ctx.check(ctx.lib.fmc_set_launch_rules(ctx.h, arr, len(rules)))


def net_matrix(scenario, nmt: int, H: int = 4):
    """fmc_diag_net_matrix: the split kernel's tensor-core network matrix as the
    library builds it for a launch (host only, no GPU): (Net_hi, Net_lo), each
    float32 [NN][NN]."""
    lib = load_library()
    kh = (2 * nmt + 3) & ~3
    nn = (H * kh + 15) & ~15
    out = np.zeros(2 * nn * nn, dtype=np.float32)
    ss = ScenarioStruct(scenario)
    rc = lib.fmc_diag_net_matrix(ctypes.byref(ss.s), int(nmt), int(H), out.ctypes.data, out.size)
    if rc != OK:
        raise FastMCError(rc, "fmc_diag_net_matrix failed")
    return out[: nn * nn].reshape(nn, nn), out[nn * nn:].reshape(nn, nn)


def kernel_choice(scenario, policy="auto", path="fused", count=None):
    """fmc_diag_kernel_choice: the kernel and layout of a single-scenario fused
    launch (host only, no GPU, no launch rules) as a dict, or FastMCError with the
    launch's refusal."""
    lib = load_library()
    out = np.zeros(5, dtype=np.int32)
    ss = ScenarioStruct(scenario)
    p = _PATH.get(path, path) if isinstance(path, str) else path
    pol = _KERNEL.get(policy, policy) if isinstance(policy, str) else policy
    rc = lib.fmc_diag_kernel_choice(ctypes.byref(ss.s), int(p), int(pol), int(scenario.N if count is None else count),
                                    out.ctypes.data)
    if rc != OK:
        raise FastMCError(rc, "fmc_diag_kernel_choice refused")
    names = {KERNEL_PER_SAMPLE: "per_sample", KERNEL_SPLIT: "split", KERNEL_SPLIT_TC: "split_tc"}
    return {"kernel": names[int(out[0])], "nmt": int(out[1]), "H": int(out[2]), "nd": int(out[3]),
            "bus": bool(out[4])}


def set_kernel_policy(policy, ctx: Context | None = None) -> None:
    """Fused-path kernel for later single-scenario calls: "auto", "per_sample", "split" or
    "split_tc"."""
    ctx = ctx or default_context()
    ctx.check(ctx.lib.fmc_set_kernel_policy(ctx.h, _KERNEL.get(policy, policy)))


def fused_occupancy(ctx: Context | None = None) -> int:
    ctx = ctx or default_context()
    v = ctypes.c_int()
    ctx.check(ctx.lib.fmc_last_fused_occupancy(ctx.h, ctypes.byref(v)))
    return v.value
