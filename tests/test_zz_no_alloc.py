"""The allocation-free reconstruction entry point against the allocating one.

fmc_kle_reconstruct_noalloc serves callers that cannot allocate device memory
(for example a process whose device memory is all reserved for its own pool, or
a loop that must not pay for cudaMalloc's device synchronisation): its working
memory is a fixed array inside the library.  Both entry points run the same
split, basis and contraction kernels on the same inputs, so, called through the
C ABI several times in a row with different shapes, the allocation-free form
must reproduce fmc_kle_reconstruct bit for bit (a wrong offset into the shared
array or a stale operand would show), its error word must read clean through
fmc_device_status, and a call larger than the array must be refused with a
clear error.  This file is collected last.
"""
import numpy as np
import pytest

from gpu_common import need_gpu

pytestmark = pytest.mark.gpu

CASES = [  # count, d, K, T, dt, precision
    (300, 2, 50, 1.0, 0.01, "bf16x3"),
    (129, 3, 200, 2.0, 0.005, "bf16"),
    (257, 1, 100, 10.0, 0.01, "f32"),
    (300, 2, 50, 1.0, 0.01, "bf16x3"),
]


def test_noalloc_matches_allocating_entry_point():
    fmc = need_gpu()
    for count, d, K, T, dt, prec in CASES:  # consecutive calls share the scratch array
        zeta, _ = fmc.lhs_sample(11 + count, count, d * K)
        ref = fmc.kle_reconstruct(zeta, d, K, T, dt, precision=prec).cpu().numpy()
        got = fmc.kle_reconstruct_noalloc(zeta, d, K, T, dt, precision=prec)
        _, err = fmc.device_status()   # reads the allocation-free call's error word too
        assert err == 0
        assert np.array_equal(got.cpu().numpy(), ref), (count, d, K, prec)


def test_noalloc_refuses_oversize_calls():
    fmc = need_gpu()
    import torch
    count, d, K, T, dt = 1 << 14, 8, 300, 1.0, 0.01
    zeta = torch.zeros((count, d * K), dtype=torch.float32, device="cuda")
    dW = torch.empty((count, d, 100), dtype=torch.float32, device="cuda")
    with pytest.raises(fmc.FastMCError) as e:
        fmc.kle_reconstruct_noalloc(zeta, d, K, T, dt, precision="bf16x3", dW=dW)
    assert e.value.code == fmc.EINVAL and "working memory" in str(e.value)


def test_noalloc_timeout_surfaces_and_clears():
    # a bounded wait that runs out on purpose (no fault: an mbarrier nothing
    # arrives at) lands in the allocation-free call's error word; the next
    # allocation-free call clears it
    fmc = need_gpu()
    fmc.check_wait_path(target=1, poll_limit=1000)
    with pytest.raises(fmc.FastMCError) as e:
        fmc.device_status()
    assert e.value.code == fmc.ETIMEOUT and "allocation-free" in str(e.value)
    zeta, _ = fmc.lhs_sample(5, 64, 40)
    fmc.kle_reconstruct_noalloc(zeta, 1, 40, 1.0, 0.01, precision="bf16x3")
    assert fmc.device_status()[1] == 0
