"""The fused path's kernel and layout choice (host logic, no GPU): which kernel a
launch takes, the split kernel's slots per thread and warps per sample, the
disturbance-slot bucket the instantiations exist for, the infinite-bus form, and
the refusals -- the combinations the launch relies on."""
import pytest

import fmc_synth as fs


@pytest.fixture(scope="module")
def fmc():
    import paper_2007_03847_gb300 as m
    m.build()
    return m


def _sc(n, d=3, **kw):
    return fs.multimachine_case(n=n, d=d, K=20, T=0.1, dt=0.005, N=1024, seed=n).replace(**kw)


def _bus(sc):
    import numpy as np
    return sc.replace(has_inf_bus=True, Ginf=np.zeros(sc.n), Binf=np.full(sc.n, 2.0), Vinf=1.0)


@pytest.mark.parametrize("n,kernel,nmt,H", [
    (1, "per_sample", 0, 4), (10, "per_sample", 0, 4), (16, "per_sample", 0, 4),
    (17, "split_tc", 9, 2), (18, "split_tc", 9, 2), (19, "split_tc", 10, 2), (20, "split_tc", 10, 2),
    (21, "split_tc", 11, 2), (22, "split_tc", 11, 2), (23, "split_tc", 12, 2), (24, "split_tc", 12, 2),
    (25, "split_tc", 13, 2), (26, "split_tc", 13, 2), (27, "split_tc", 14, 2), (28, "split_tc", 14, 2),
    (29, "split_tc", 10, 4), (40, "split_tc", 10, 4), (41, "split_tc", 13, 4), (52, "split_tc", 13, 4)])
def test_automatic_choice(fmc, n, kernel, nmt, H):
    c = fmc.kernel_choice(_sc(n))
    assert (c["kernel"], c["nmt"], c["H"], c["nd"], c["bus"]) == (kernel, nmt, H, 4, False)


def test_two_warps_per_sample_needs_the_tmem_and_the_bucket(fmc):
    # 8 disturbances: 16-step chunks of 8 columns plus the product's 144 exceed a
    # CTA's 256 columns at two CTAs per SM
    c = fmc.kernel_choice(_sc(20, d=8))
    assert (c["H"], c["nmt"], c["nd"]) == (4, 5, 8)
    c = fmc.kernel_choice(_sc(20, d=7))
    assert (c["H"], c["nmt"], c["nd"]) == (2, 10, 8)
    # 13 and 14 slots exist for buckets up to 4 disturbance slots: 4 disturbances
    # and a generator trip fill the 8-slot bucket
    c = fmc.kernel_choice(_sc(25, d=4))
    assert (c["H"], c["nmt"], c["nd"]) == (2, 13, 4)
    c = fmc.kernel_choice(_sc(25, d=4, event_machine=3, event_time=0.05, event_dpm=-0.5))
    assert (c["H"], c["nmt"], c["nd"]) == (4, 7, 8)
    c = fmc.kernel_choice(_sc(27, d=5))
    assert (c["H"], c["nmt"]) == (4, 7)


def test_policies(fmc):
    assert fmc.kernel_choice(_sc(13), policy="split_tc")["kernel"] == "split_tc"
    assert fmc.kernel_choice(_sc(13), policy="split") == {"kernel": "split", "nmt": 4, "H": 4, "nd": 4,
                                                          "bus": False}
    assert fmc.kernel_choice(_sc(40), policy="split")["kernel"] == "split"
    with pytest.raises(fmc.FastMCError) as e:
        fmc.kernel_choice(_sc(12), policy="split_tc")     # below 13 machines
    assert e.value.code == fmc.EUNSUPPORTED
    with pytest.raises(fmc.FastMCError) as e:
        fmc.kernel_choice(_sc(20), policy="per_sample")   # above 16 machines
    assert e.value.code == fmc.EUNSUPPORTED
    with pytest.raises(fmc.FastMCError) as e:              # smooth forcing: per-sample kernel only
        fmc.kernel_choice(_sc(20, forcing=fs.FORCING_SMOOTH))
    assert e.value.code == fmc.EUNSUPPORTED


def test_infinite_bus(fmc):
    # the bus takes the last slot of a four-warp layout in the 8-slot bucket
    c = fmc.kernel_choice(_bus(_sc(19)))
    assert c == {"kernel": "split_tc", "nmt": 5, "H": 4, "nd": 8, "bus": True}
    c = fmc.kernel_choice(_bus(_sc(44, d=2)))
    assert c == {"kernel": "split_tc", "nmt": 13, "H": 4, "nd": 8, "bus": True}
    # no free slot: the FP32 split kernel, or a refusal when forced
    c = fmc.kernel_choice(_bus(_sc(20)))
    assert (c["kernel"], c["bus"]) == ("split", False)
    with pytest.raises(fmc.FastMCError) as e:
        fmc.kernel_choice(_bus(_sc(20)), policy="split_tc")
    assert e.value.code == fmc.EUNSUPPORTED
