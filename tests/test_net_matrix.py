"""The split kernel's tensor-core network matrix as the library builds it for a
launch (host code, no GPU): its layout, the TF32 hi/lo split, and the network
sums it forms, against the Kron-reduced network written out here:
    du_i = sum_{j != i} E_i E_j (G_ij gamma_j - B_ij eta_j)
    dv_i = sum_{j != i} E_i E_j (B_ij gamma_j + G_ij eta_j)
(the deviation form of P_e, Sec. II), with an infinite bus as one more node at
E = V, G_ib = Ginf_i, B_ib = Binf_i."""
import numpy as np
import pytest

import fmc_synth as fs


@pytest.fixture(scope="module")
def fmc():
    import paper_2007_03847_gb300 as m
    m.build()
    return m


def _slot(i, H, KH):
    return (i % H) * KH + 2 * (i // H)


def _is_tf32(a):
    bits = np.asarray(a, dtype=np.float32).view(np.uint32)
    return np.all(bits & np.uint32(0x1FFF) == 0)


def _check(fmc, sc, nmt, H, bus_slot=None):
    hi, lo = fmc.net_matrix(sc, nmt, H)
    n, KH = sc.n, (2 * nmt + 3) & ~3
    NN = (H * KH + 15) & ~15
    assert hi.shape == (NN, NN) and lo.shape == (NN, NN)
    assert _is_tf32(hi) and _is_tf32(lo)
    net = hi.astype(np.float64) + lo.astype(np.float64)
    # the split: lo is the rounded remainder, below 2^-11 of hi
    assert np.all(np.abs(lo) <= 2.0**-11 * np.abs(hi) + 1e-30)
    E, G, B = sc.E, sc.G, sc.B
    expect = np.zeros((NN, NN))
    for i in range(n):
        ru = _slot(i, H, KH)
        for j in range(n):
            if j == i:
                continue
            cg = _slot(j, H, KH)
            ge, be = E[i] * E[j] * G[i, j], E[i] * E[j] * B[i, j]
            expect[ru, cg], expect[ru, cg + 1] = ge, -be
            expect[ru + 1, cg], expect[ru + 1, cg + 1] = be, ge
        if bus_slot is not None:
            cb = _slot(bus_slot, H, KH)
            ge, be = E[i] * sc.Vinf * sc.Ginf[i], E[i] * sc.Vinf * sc.Binf[i]
            expect[ru, cb], expect[ru, cb + 1] = ge, -be
            expect[ru + 1, cb], expect[ru + 1, cb + 1] = be, ge
    # hi + lo carries every entry to 2^-21 of itself; everything else is zero
    assert np.all(np.abs(net - expect) <= 2.0**-21 * np.abs(expect))
    assert np.all(net[expect == 0] == 0)
    # the sums it forms, for seeded deviations, against the formula above
    rng = np.random.default_rng(nmt * 10 + H)
    gam, eta = rng.normal(0, 1e-2, n), rng.normal(0, 1e-2, n)
    x = np.zeros(NN)
    for j in range(n):
        x[_slot(j, H, KH)], x[_slot(j, H, KH) + 1] = gam[j], eta[j]
    y = net @ x
    for i in range(n):
        ru = _slot(i, H, KH)
        du = sum(E[i] * E[j] * (G[i, j] * gam[j] - B[i, j] * eta[j]) for j in range(n) if j != i)
        dv = sum(E[i] * E[j] * (B[i, j] * gam[j] + G[i, j] * eta[j]) for j in range(n) if j != i)
        scale = sum(E[i] * E[j] * (abs(G[i, j]) + abs(B[i, j])) for j in range(n)) * 1e-2
        assert abs(y[ru] - du) <= 1e-6 * scale and abs(y[ru + 1] - dv) <= 1e-6 * scale


@pytest.mark.parametrize("n,nmt,H", [(13, 4, 4), (20, 5, 4), (20, 10, 2), (23, 12, 2), (27, 14, 2), (41, 13, 4),
                                     (52, 13, 4)])
def test_network_matrix_layout_and_sums(fmc, n, nmt, H):
    _check(fmc, fs.multimachine_case(n=n, d=2, K=10, T=0.1, dt=0.005, N=128, seed=n), nmt, H)


def _with_bus(sc):
    n = sc.n
    return sc.replace(has_inf_bus=True, Ginf=np.linspace(0.0, 0.3, n), Binf=np.linspace(1.0, 2.0, n), Vinf=1.05)


@pytest.mark.parametrize("n,nmt,H", [(19, 10, 2), (44, 13, 4)])
def test_network_matrix_with_an_infinite_bus(fmc, n, nmt, H):
    sc = _with_bus(fs.multimachine_case(n=n, d=2, K=10, T=0.1, dt=0.005, N=128, seed=n))
    _check(fmc, sc, nmt, H, bus_slot=H * nmt - 1)


def test_network_matrix_refusals(fmc):
    sc = fs.multimachine_case(n=20, d=2, K=10, T=0.1, dt=0.005, N=128, seed=3)
    for nmt, H in ((4, 4), (10, 3), (0, 4)):       # too few slots; H not 2 or 4; no slots
        with pytest.raises(fmc.FastMCError):
            fmc.net_matrix(sc, nmt, H)
    with pytest.raises(fmc.FastMCError):           # an infinite bus needs a free slot
        fmc.net_matrix(_with_bus(sc), 10, 2)
