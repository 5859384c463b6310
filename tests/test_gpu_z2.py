"""Z2-symmetric MERA on the GPU (mera_config.z2 = 1, Sec. 6): the ternary
network in the setting of Fig. 2 (Ising chain, chi = 8, two transition
layers) and the binary network where its chain runs unsliced (blocked spin
pairs in the parity-ordered basis); every network contraction runs as its two
charge sectors.  Against the oracles and the dense GPU path on the same
symmetric point: energy and every partial derivative at 1e-12 in FP64, within
the mixed-precision bound for 3xTF32, derivatives exactly symmetric; L-BFGS
keeps the tensors symmetric and follows the dense path; non-symmetric tensors
or Hamiltonians, and the sliced chain, are refused."""
import numpy as np
import pytest

from oracle import ternary as ot
from oracle import z2
from paper_2007_03638_gb300 import inputs as inp

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module")
def gm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2007_03638_gb300 import build as b
    b.build()
    from paper_2007_03638_gb300 import mera
    return mera


def _flat(us, ws):
    return [t for p in zip(us, ws) for t in p]


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _cfg(gm, chi, L, **kw):
    return gm.default_config(2, chi, L, network=gm.MERA_TERNARY, **kw)


def _parities(chi, L):
    dims = inp.ternary_layer_dims(2, chi, L)
    out = []
    for l in range(L + 1):
        cf, cc = dims[l], dims[min(l + 1, L)]
        pu = inp.fused_parities(cf, cf)
        out.append((pu, pu))
        out.append((inp.fused_parities(cf, cf, cf), inp.z2_parities(cc)))
    return out


@pytest.mark.parametrize("chi,L,seed", [(4, 1, 0), (8, 2, 1)])
def test_z2_sectors_match_dense_and_oracle(gm, chi, L, seed):
    h = inp.ising_bond(1.0)
    us, ws = inp.random_z2_ternary_mera(chi, L, seed=seed)
    pt = _flat(us, ws)
    dense = gm.Mera(_cfg(gm, chi, L), h)
    dense.set_tensors(pt)
    sym = gm.Mera(_cfg(gm, chi, L, z2=1), h)
    sym.set_tensors(pt)
    e0, G0, D0 = dense.energy_grad(deriv=True)
    e1, G1, D1 = sym.energy_grad(deriv=True)
    e_ref, ds, _ = ot.energy_grad(h, us, ws)
    assert abs(e1 - e_ref) <= TOL * max(1.0, abs(e_ref)), (e1, e_ref)
    assert abs(e1 - e0) <= TOL * max(1.0, abs(e0))
    for i, (d_ref, (rp, cp)) in enumerate(zip(ds, _parities(chi, L))):
        assert _rel(D1[i], d_ref) < TOL, (i, _rel(D1[i], d_ref))
        assert _rel(D1[i], D0[i]) < TOL, i
        assert z2.violation(D1[i], rp, cp) == 0.0, i
        assert z2.violation(G1[i], rp, cp) == 0.0, i


def test_z2_mixed_precision(gm):
    h = inp.ising_bond(1.0)
    us, ws = inp.random_z2_ternary_mera(8, 2, seed=2)
    m = gm.Mera(_cfg(gm, 8, 2, z2=1, prec=gm.PREC_3XTF32), h)
    m.set_tensors(_flat(us, ws))
    e, G, D = m.energy_grad(deriv=True)
    e_ref, ds, _ = ot.energy_grad(h, us, ws)
    assert abs(e - e_ref) / max(1.0, abs(e_ref)) < 2e-6
    assert max(_rel(D[i], ds[i]) for i in range(len(ds))) < 2e-5


def test_z2_lbfgs_stays_symmetric_and_follows_dense(gm):
    h = inp.ising_bond(1.0)
    us, ws = inp.random_z2_ternary_mera(8, 2, seed=3)
    pt = _flat(us, ws)
    runs = {}
    for flag in (0, 1):
        m = gm.Mera(_cfg(gm, 8, 2, z2=flag), h)
        m.set_tensors(pt)
        runs[flag] = ([m.lbfgs_step()["energy"] for _ in range(10)], m.get_tensors())
    es, tensors = runs[1]
    assert all(b <= a + 1e-12 for a, b in zip(es, es[1:]))
    assert max(abs(a - b) for a, b in zip(es, runs[0][0])) < 1e-9
    for t, (rp, cp) in zip(tensors, _parities(8, 2)):
        assert z2.violation(t, rp, cp) <= 1e-12 * np.abs(t).max()


def test_z2_refusals(gm):
    h = inp.ising_bond(1.0)
    with pytest.raises(gm.MeraError) as ei:
        gm.Mera(_cfg(gm, 8, 2, z2=1), inp.ising_bond(1.0, 0.3))  # a longitudinal field breaks Z2
    assert ei.value.code == -1
    m = gm.Mera(_cfg(gm, 8, 2, z2=1), h)
    us, ws = inp.random_ternary_mera(2, 8, 2, seed=4)  # generic tensors
    with pytest.raises(gm.MeraError) as ei:
        m.set_tensors(_flat(us, ws))
    assert ei.value.code == -1
    with pytest.raises(gm.MeraError) as ei:
        gm.Mera(gm.default_config(2, 8, 0, network=gm.MERA_MPS, z2=1), h)
    assert ei.value.code == -8


@pytest.mark.parametrize("chi,L,seed,prec,tol", [(4, 2, 0, 0, TOL), (8, 3, 1, 0, TOL), (8, 3, 2, 1, 2e-6)])
def test_z2_binary_matches_dense_and_oracle(gm, chi, L, seed, prec, tol):
    from oracle import mera as om
    h3 = inp.parity_ordered_three_site(inp.three_site_blocked(inp.ising_bond(1.0)))
    us, ws = inp.random_z2_mera(4, chi, L, seed=seed)
    pt = _flat(us, ws)
    sym = gm.Mera(gm.default_config(4, chi, L, z2=1, prec=prec), h3)
    sym.set_tensors(pt)
    e, G, D = sym.energy_grad(deriv=True)
    e_ref, ds, _ = om.energy_grad(h3, us, ws)
    assert abs(e - e_ref) <= tol * max(1.0, abs(e_ref)), (e, e_ref)
    dims = inp.layer_dims(4, chi, L)
    for i, d_ref in enumerate(ds):
        assert _rel(D[i], d_ref) < 10 * tol, (i, _rel(D[i], d_ref))
        c = dims[i // 2]
        cp = dims[min(i // 2 + 1, L)]
        pair = inp.fused_parities(c, c)
        cols = pair if i % 2 == 0 else inp.z2_parities(cp)
        assert z2.violation(D[i], pair, cols) == 0.0, i
    if prec == 0:
        dense = gm.Mera(gm.default_config(4, chi, L), h3)
        dense.set_tensors(pt)
        e0, G0 = dense.energy_grad()
        assert abs(e - e0) <= TOL * max(1.0, abs(e0))
        for a, b in zip(G, G0):
            assert np.abs(a - b).max() < TOL * max(1.0, np.abs(b).max())


def test_z2_binary_refusals(gm):
    h3 = inp.parity_ordered_three_site(inp.three_site_blocked(inp.ising_bond(1.0)))
    with pytest.raises(gm.MeraError) as ei:  # the chi^9 chain of chi = 32 is sliced
        gm.Mera(gm.default_config(4, 32, 3, z2=1, prec=2), h3)
    assert ei.value.code == -8
    with pytest.raises(gm.MeraError) as ei:  # the product basis of a blocked pair is not graded first-half-even
        gm.Mera(gm.default_config(4, 8, 3, z2=1), inp.three_site_blocked(inp.ising_bond(1.0)))
    assert ei.value.code == -1
