"""The allocation-free reconstruction entry point against the allocating one.

fmc_kle_reconstruct_noalloc serves callers that cannot allocate device memory
(for example a process whose device memory is all reserved for its own pool, or
a loop that must not pay for cudaMalloc's device synchronisation): its working
memory is a fixed array inside the library.  Called through the C ABI twice in
a row with different shapes, it must reproduce fmc_kle_reconstruct within the
tolerance the reconstruction tests use, and a call larger than the array must
be refused with a clear error.  This file is collected last.
"""
import numpy as np
import pytest

from gpu_common import need_gpu

pytestmark = pytest.mark.gpu

CASES = [  # count, d, K, T, dt, precision, tolerance factor on sum_k |zeta_k phi_k|
    (300, 2, 50, 1.0, 0.01, "bf16x3", 2.0**-15),
    (129, 3, 200, 2.0, 0.005, "bf16", 2.0**-7),
    (257, 1, 100, 10.0, 0.01, "f32", None),
]


def _tolerance(orc, zeta, d, K, T, Nt, factor):
    z64 = zeta.cpu().numpy().astype(np.float64)
    phi = orc.kl_increment_basis(K, T, Nt)
    absum = np.einsum("swk,kn->swn", np.abs(z64.reshape(z64.shape[0], d, K)), np.abs(phi))
    return (K * 2.0**-23 if factor is None else factor) * absum + 1e-12


def test_noalloc_matches_allocating_entry_point(orc):
    fmc = need_gpu()
    for count, d, K, T, dt, prec, factor in CASES:  # consecutive calls share the scratch array
        Nt = int(round(T / dt))
        zeta, _ = fmc.lhs_sample(11, count, d * K)
        ref = fmc.kle_reconstruct(zeta, d, K, T, dt, precision=prec).cpu().numpy()
        got = fmc.kle_reconstruct_noalloc(zeta, d, K, T, dt, precision=prec)
        fmc.device_status()
        got = got.cpu().numpy()
        tol = _tolerance(orc, zeta, d, K, T, Nt, factor)
        assert np.all(np.abs(got.astype(np.float64) - ref) <= tol)


def test_noalloc_refuses_oversize_calls():
    fmc = need_gpu()
    import torch
    count, d, K, T, dt = 1 << 14, 8, 300, 1.0, 0.01
    zeta = torch.zeros((count, d * K), dtype=torch.float32, device="cuda")
    dW = torch.empty((count, d, 100), dtype=torch.float32, device="cuda")
    with pytest.raises(fmc.FastMCError) as e:
        fmc.kle_reconstruct_noalloc(zeta, d, K, T, dt, precision="bf16x3", dW=dW)
    assert e.value.code == fmc.EINVAL and "working memory" in str(e.value)
