"""The precision form at full size: the 10-machine, 3-disturbance, K = 200 system at
N = 2^20 samples in one fused launch, against the FP64 oracle.

The horizon is shortened to T = 0.5 s (100 steps) so that the oracle can run all
2^20 samples in the test; the launch shape (8192 CTAs of 128 samples, 13.5
waves, a 20-bit Feistel domain with cycle walking) is that of the full-horizon
run.  Checked:
* LHS strata of every dimension and every sample bit-exact against the oracle;
* trajectories of the first 4096 samples and of samples spread over the design
  within 1e-4 (normwise, delta and omega separately) for BF16x3;
* mean and variance of all 2^20 samples within 1e-5 of the oracle's (BF16x3);
* the first 4096 samples as their own block (the sums entry point) against the
  oracle's moments of the same 4096;
* BF16: the stated error bound of the unsplit contraction (2e-2), with the
  errors printed.
"""
import concurrent.futures as cf
import os

import numpy as np
import pytest

import fmc_synth as fs
from gpu_common import need_gpu, normwise_rel, traj_errors

pytestmark = pytest.mark.gpu

N = 1 << 20
BLOCK = 1 << 14


def _case():
    return fs.multimachine_case(n=10, d=3, K=200, T=0.5, dt=0.005, N=N, seed=0)


def _chan(parts):
    """Combine (count, mean, M2) triples of disjoint blocks (Chan, Golub, LeVeque)."""
    n, m, M2 = parts[0]
    for nb, mb, M2b in parts[1:]:
        tot = n + nb
        delta = mb - m
        m = m + delta * (nb / tot)
        M2 = M2 + M2b + delta * delta * (n * nb / tot)
        n = tot
    return n, m, M2


@pytest.fixture(scope="module")
def oracle_design(orc):
    """Per block of the design: strata [M, count], and the oracle's mean/var."""
    sc = _case()

    def block(k0):
        z, strata = orc.lhs_sample(sc.seed, sc.N, sc.M, k0=k0, count=BLOCK, with_strata=True)
        out = orc.simulate(sc, z, nthreads=1)
        return k0, strata, out["mean"], out["var"]

    workers = max(1, min(32, os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(workers) as ex:   # ctypes calls release the GIL
        blocks = sorted(ex.map(block, range(0, N, BLOCK)), key=lambda b: b[0])
    return sc, blocks


def test_c3_strata_bit_exact(orc, oracle_design):
    fmc = need_gpu()
    import torch
    sc, blocks = oracle_design
    strata = torch.empty((sc.M, sc.N), dtype=torch.int32, device="cuda")
    fmc.lhs_sample(sc.seed, sc.N, sc.M, strata=strata)
    for k0, sr, _, _ in blocks:
        sg = strata[:, k0:k0 + BLOCK].cpu().numpy().view(np.uint32)
        assert np.array_equal(sg, sr), k0


@pytest.mark.parametrize("precision,traj_tol,mom_tol", [("bf16x3", 1e-4, 1e-5), ("bf16", 2e-2, 2e-2)])
def test_c3_full_launch(orc, oracle_design, precision, traj_tol, mom_tol):
    fmc = need_gpu()
    import torch
    sc, blocks = oracle_design
    n = sc.n
    mean, var, traj = fmc.simulate(sc, path="fused", precision=precision, want_traj=True)
    fmc.device_status()
    # trajectories: the first 4096 samples, and samples spread over the design
    picks = list(range(4096)) + [N // 2 - 1, N // 2, 777777, N - 129, N - 1]
    zr = np.concatenate([orc.lhs_sample(sc.seed, sc.N, sc.M, k0=0, count=4096)] +
                        [orc.lhs_sample(sc.seed, sc.N, sc.M, k0=k, count=1) for k in picks[4096:]])
    ref = orc.simulate(sc, zr, want_traj=True, want_moments=False, nthreads=os.cpu_count() or 1)
    got = traj[torch.tensor(picks, device="cuda")].cpu().numpy()
    ed, ew = traj_errors(got, ref["traj"], n)
    del traj
    torch.cuda.empty_cache()
    # moments of all 2^20 samples against the oracle's, its blocks combined in FP64
    cnt, rm, M2 = _chan([(float(BLOCK), m, v * (BLOCK - 1)) for _, _, m, v in blocks])
    rv = M2 / (cnt - 1)
    m, v = mean.cpu().numpy(), var.cpu().numpy()
    em = max(np.max(np.abs(m[:, sl] - rm[:, sl])) / np.max(np.sqrt(rm[:, sl] ** 2 + rv[:, sl]))
             for sl in (slice(0, n), slice(n, 2 * n)))
    ev = max(normwise_rel(v[:, sl], rv[:, sl]) for sl in (slice(0, n), slice(n, 2 * n)))
    # the first 4096 samples as a block of their own
    S1, S2, shift = fmc.simulate_sums(sc, 0, 4096, path="fused", precision=precision)
    m4, v4 = fmc.moments_from_sums(S1, S2, shift, 4096)
    r4 = orc.simulate(sc, zr[:4096], nthreads=os.cpu_count() or 1)
    m4, v4 = m4.cpu().numpy(), v4.cpu().numpy()
    em4 = max(np.max(np.abs(m4[:, sl] - r4["mean"][:, sl])) / np.max(np.sqrt(r4["mean"][:, sl] ** 2 + r4["var"][:, sl]))
              for sl in (slice(0, n), slice(n, 2 * n)))
    ev4 = max(normwise_rel(v4[:, sl], r4["var"][:, sl]) for sl in (slice(0, n), slice(n, 2 * n)))
    print(f"c3 {precision}: traj delta {ed:.2e} omega {ew:.2e}; all 2^20: E {em:.2e} Var {ev:.2e}; "
          f"first 4096: E {em4:.2e} Var {ev4:.2e}")
    assert ed <= traj_tol and ew <= traj_tol, (ed, ew)
    assert em <= mom_tol and ev <= mom_tol, (em, ev)
    assert em4 <= mom_tol and ev4 <= mom_tol, (em4, ev4)
