"""GPU (CUDA, FP64 path) against the CPU FP64 oracle, element by element,
through the C ABI.  Tolerance: 1e-12 relative (normwise per tensor) for the
FP64 path."""
import numpy as np
import pytest

from oracle import geometry as geo
from oracle import mera as om
from oracle import optim as oo
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


def _ham(d_b, kind="ising", seed=0):
    if kind == "ising":
        bond = inp.ising_bond(1.0)
    elif kind == "xxz":
        bond = inp.xxz_bond(1.0)
    else:
        rng = np.random.default_rng(seed)
        a = rng.standard_normal((d_b**3, d_b**3))
        return 0.5 * (a + a.T)
    return inp.three_site_blocked(bond) if d_b == 4 else inp.three_site_unblocked(bond)


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _flat(us, ws):
    return [t for p in zip(us, ws) for t in p]


CASES = [
    (4, 4, 2, "ising", 0),   # config-1 shapes
    (4, 4, 2, "xxz", 3),
    (2, 3, 2, "ising", 1),   # ragged tiles: dims 2,3,3
    (3, 5, 2, "random", 2),  # odd dims 3,5,5
    (4, 8, 3, "ising", 4),   # config-2 chi=8
]


@pytest.mark.parametrize("d_b,chi,L,kind,seed", CASES)
def test_energy_grad_parity(gm, d_b, chi, L, kind, seed):
    us, ws = inp.random_mera(d_b, chi, L, seed=seed)
    h3 = _ham(d_b, kind, seed)
    m = gm.Mera(gm.default_config(d_b, chi, L), h3)
    m.set_tensors(_flat(us, ws))
    e, G, D = m.energy_grad(deriv=True)
    e_ref, ds, _ = om.energy_grad(h3, us, ws)
    assert abs(e - e_ref) <= TOL * max(1.0, abs(e_ref)), (e, e_ref)
    pt = _flat(us, ws)
    for i, (W, d_ref) in enumerate(zip(pt, ds)):
        kind_i = geo.STIEFEL if i % 2 == 0 else geo.GRASSMANN
        g_ref = geo.project(W, d_ref, kind_i)
        assert _rel(D[i], d_ref) < TOL, (i, _rel(D[i], d_ref))
        if np.abs(g_ref).max() > 1e-13:
            assert np.abs(G[i] - g_ref).max() < TOL * np.abs(d_ref).max(), i
    # second call reuses the Krylov warm starts: same result
    e2, G2 = m.energy_grad()
    assert abs(e2 - e) <= 1e-13 * max(1, abs(e))
    assert max(np.abs(a - b).max() for a, b in zip(G, G2)) < 1e-12 * max(np.abs(g).max() for g in G)


@pytest.mark.slow
def test_energy_grad_parity_chi12(gm):
    """Config-2 chi=12 (3 transition layers), one seed."""
    us, ws = inp.random_mera(4, 12, 3, seed=5)
    h3 = _ham(4)
    m = gm.Mera(gm.default_config(4, 12, 3), h3)
    m.set_tensors(_flat(us, ws))
    e, G, D = m.energy_grad(deriv=True)
    e_ref, ds, _ = om.energy_grad(h3, us, ws)
    assert abs(e - e_ref) <= TOL * abs(e_ref)
    for i in range(len(ds)):
        assert _rel(D[i], ds[i]) < TOL, i


def test_product_state(gm):
    """Closed form: u = 1, w|k> = |k>|0> gives e = 2 <00|bond|00> per bottom site."""
    us, ws = inp.product_state_mera(4, 2)
    m = gm.Mera(gm.default_config(4, 4, 2), _ham(4, "xxz"))
    m.set_tensors(_flat(us, ws))
    assert abs(m.energy() / 2 - 1.0) < 1e-12


def test_not_isometric_rejected(gm):
    us, ws = inp.random_mera(4, 4, 2, seed=0)
    m = gm.Mera(gm.default_config(4, 4, 2), _ham(4))
    bad = _flat(us, ws)
    bad[1] = bad[1] * 1.01
    with pytest.raises(gm.MeraError) as ex:
        m.set_tensors(bad)
    assert ex.value.code == -6
    m.set_tensors(_flat(us, ws))  # object still usable
    assert np.isfinite(m.energy())


def test_geometry_parity(gm):
    us, ws = inp.random_mera(4, 4, 2, seed=7)
    pt = _flat(us, ws)
    h3 = _ham(4)
    m = gm.Mera(gm.default_config(4, 4, 2), h3)
    m.set_tensors(pt)
    rng = np.random.default_rng(1)
    kinds = [geo.STIEFEL if i % 2 == 0 else geo.GRASSMANN for i in range(len(pt))]
    Draw = [rng.standard_normal(t.shape) for t in pt]
    X = m.project(Draw)
    X_ref = [geo.project(W, d, k) for W, d, k in zip(pt, Draw, kinds)]
    for a, b in zip(X, X_ref):
        assert np.abs(a - b).max() < 1e-13
    Y = [geo.project(W, rng.standard_normal(W.shape), k) for W, k in zip(pt, kinds)]
    assert abs(m.inner(X, Y) - geo.inner(X_ref, Y)) < 1e-12 * abs(geo.inner(X_ref, Y))
    alpha = 0.3
    TY = m.transport(X_ref, alpha, Y)
    for W, x, y, ty in zip(pt, X_ref, Y, TY):
        assert np.abs(ty - geo.transport(W, x, alpha, y)).max() < 1e-12
    # preconditioner with the density matrices of this point
    e, G = m.energy_grad()
    e_ref, ds, info = om.energy_grad(h3, us, ws)
    rv = om.tensor_density_matrices(info["rho"], ws)
    Gr = [geo.project(W, d, k) for W, d, k in zip(pt, ds, kinds)]
    deltas = [float(np.linalg.norm(g)) for g in Gr]
    Xt = m.precondition(X_ref)
    for W, x, r, dl, k, xt in zip(pt, X_ref, rv, deltas, kinds, Xt):
        ref = geo.precondition(W, x, r, dl, k)
        assert np.abs(xt - ref).max() < 1e-11 * max(1, np.abs(ref).max())
    Xp = m.retract(X_ref, alpha, want_xprime=True)
    Wn = m.get_tensors()
    for W, x, wn, xp in zip(pt, X_ref, Wn, Xp):
        assert np.abs(wn - geo.polar(geo.retract(W, x, alpha))).max() < 1e-12
        assert np.abs(xp - geo.transport(W, x, alpha, x)).max() < 1e-12
        assert np.abs(wn.T @ wn - np.eye(wn.shape[1])).max() < 1e-14


def test_lbfgs_matches_oracle_trajectory(gm):
    """Config-1 shapes: the first L-BFGS iterations of the GPU follow the
    oracle's energies (same starting point, same algorithm)."""
    us, ws = inp.random_mera(4, 4, 2, seed=0)
    h3 = _ham(4)
    m = gm.Mera(gm.default_config(4, 4, 2), h3)
    m.set_tensors(_flat(us, ws))
    got = [m.lbfgs_step() for _ in range(8)]
    prob = oo.MeraProblem(h3)
    _, _, hist = oo.lbfgs(prob, _flat(us, ws), m=8, maxiter=9)
    ref = [h["energy"] for h in hist[1:9]]
    for g, r in zip(got, ref):
        assert abs(g["energy"] - r) < 1e-9 * abs(r), (g, r)
    # isometry kept
    for t in m.get_tensors():
        assert np.abs(t.T @ t - np.eye(t.shape[1])).max() < 1e-13


@pytest.mark.parametrize("kind,seed", [("ising", 0), ("xxz", 2)])
def test_cg_matches_oracle_trajectory(gm, kind, seed):
    """Config-1 shapes: the first nonlinear-CG iterations (preconditioned
    Hager-Zhang beta with its eta bound, Sec. 3) follow the oracle's energies
    and gradient norms (same starting point, same algorithm)."""
    us, ws = inp.random_mera(4, 4, 2, seed=seed)
    h3 = _ham(4, kind)
    m = gm.Mera(gm.default_config(4, 4, 2), h3)
    m.set_tensors(_flat(us, ws))
    got = [m.cg_step() for _ in range(8)]
    prob = oo.MeraProblem(h3)
    _, _, hist = oo.cg(prob, _flat(us, ws), maxiter=9)
    for g, r in zip(got, hist[1:9]):
        assert abs(g["energy"] - r["energy"]) < 1e-9 * abs(r["energy"]), (g, r)
        assert abs(g["gnorm"] - r["gnorm"]) < 1e-6 * r["gnorm"], (g, r)
    for t in m.get_tensors():
        assert np.abs(t.T @ t - np.eye(t.shape[1])).max() < 1e-13


def test_cg_decreases(gm):
    us, ws = inp.random_mera(4, 4, 2, seed=2)
    m = gm.Mera(gm.default_config(4, 4, 2), _ham(4, "xxz"))
    m.set_tensors(_flat(us, ws))
    e0 = m.energy()
    es = [m.cg_step()["energy"] for _ in range(6)]
    assert es[-1] < e0
    assert all(b <= a + 1e-12 for a, b in zip(es, es[1:]))


MIXED = [
    (1, 2e-6, 4, 4, 2, "ising", 0),
    (1, 2e-6, 4, 8, 3, "xxz", 1),
    (1, 2e-6, 3, 5, 2, "random", 2),
    (2, 2e-4, 4, 4, 2, "ising", 0),
    (2, 2e-4, 4, 8, 3, "ising", 3),
    (3, 2e-6, 4, 4, 2, "ising", 0),
    (3, 2e-6, 4, 8, 3, "xxz", 1),
    (3, 2e-6, 3, 5, 2, "random", 2),
    (3, 2e-6, 4, 8, 3, "ising", 3),
]


@pytest.mark.parametrize("prec,tol,d_b,chi,L,kind,seed", MIXED)
def test_energy_grad_mixed_precision(gm, prec, tol, d_b, chi, L, kind, seed):
    """Tensor-core path (1 = 3xTF32, 2 = split-BF16; FP32 accumulation, FP64
    Krylov solves and reductions) against the FP64 oracle."""
    us, ws = inp.random_mera(d_b, chi, L, seed=seed)
    h3 = _ham(d_b, kind, seed)
    m = gm.Mera(gm.default_config(d_b, chi, L, prec=prec), h3)
    m.set_tensors(_flat(us, ws))
    e, G, D = m.energy_grad(deriv=True)
    e_ref, ds, _ = om.energy_grad(h3, us, ws)
    err_e = abs(e - e_ref) / max(1.0, abs(e_ref))
    err_d = max(_rel(D[i], ds[i]) for i in range(len(ds)))
    print(f"prec={prec} chi={chi}: energy rel err {err_e:.2e}, max derivative rel err {err_d:.2e}")
    assert err_e < tol
    assert err_d < 10 * tol
    st = m.stats()
    assert st["gett_launches"] > 0


def test_preconditioner_large_rho_warm_start(gm):
    """rho_u of the scale-invariant layer is 81 x 81 (d_b=3, chi=9): the
    eigen-decomposition runs on the multi-CTA Jacobi path; the second
    evaluation (after a retraction) starts from the previous eigenbasis."""
    us, ws = inp.random_mera(3, 9, 1, seed=11)
    h3 = _ham(3, "random", 4)
    m = gm.Mera(gm.default_config(3, 9, 1), h3)
    pt = _flat(us, ws)
    m.set_tensors(pt)
    kinds = [geo.STIEFEL if i % 2 == 0 else geo.GRASSMANN for i in range(len(pt))]
    rng = np.random.default_rng(2)
    for rep in range(2):
        e, G = m.energy_grad()
        us_c, ws_c = pt[0::2], pt[1::2]
        e_ref, ds, info = om.energy_grad(h3, us_c, ws_c)
        assert abs(e - e_ref) < 1e-12 * max(1, abs(e_ref))
        rv = om.tensor_density_matrices(info["rho"], ws_c)
        Gr = [geo.project(W, d, k) for W, d, k in zip(pt, ds, kinds)]
        X = [geo.project(W, rng.standard_normal(W.shape), k) for W, k in zip(pt, kinds)]
        Xt = m.precondition(X)
        for W, x, r, g, k, xt in zip(pt, X, rv, Gr, kinds, Xt):
            ref = geo.precondition(W, x, r, float(np.linalg.norm(g)), k)
            assert np.abs(xt - ref).max() < 1e-10 * max(1, np.abs(ref).max()), rep
        step = [-0.05 * g for g in G]
        m.retract(step, 1.0)
        pt = m.get_tensors()


@pytest.mark.parametrize("prec,chunk,tol", [(0, 2, 1e-12), (0, 4, 1e-12), (1, 2, 2e-6)])
def test_sliced_chain_parity(gm, prec, chunk, tol):
    """The chi^9 chain evaluated one slice of the middle coarse leg at a time
    (as at chi=32) gives the oracle's energy and derivatives (chi=8)."""
    us, ws = inp.random_mera(4, 8, 3, seed=6)
    h3 = _ham(4, "xxz")
    m = gm.Mera(gm.default_config(4, 8, 3, prec=prec, b_chunk=chunk), h3)
    m.set_tensors(_flat(us, ws))
    e, G, D = m.energy_grad(deriv=True)
    e_ref, ds, _ = om.energy_grad(h3, us, ws)
    assert abs(e - e_ref) <= tol * max(1.0, abs(e_ref))
    for i in range(len(ds)):
        assert _rel(D[i], ds[i]) < 10 * tol, i
    with pytest.raises(gm.MeraError):
        gm.Mera(gm.default_config(4, 8, 3, b_chunk=3), h3)


def test_recompute_env_same_result(gm):
    """Reusing the up-sweep's intermediates and recomputing them give the same gradient."""
    us, ws = inp.random_mera(4, 8, 3, seed=8)
    h3 = _ham(4, "xxz")
    out = []
    for rec in (0, 1):
        m = gm.Mera(gm.default_config(4, 8, 3, recompute_env=rec), h3)
        m.set_tensors(_flat(us, ws))
        out.append(m.energy_grad(deriv=True))
    assert out[0][0] == out[1][0]
    for a, b in zip(out[0][2], out[1][2]):
        assert np.array_equal(a, b)
