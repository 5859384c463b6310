"""Pins of the oracle's MERA networks, fixed point and derivatives against
brute force, closed forms and finite differences (CPU only)."""
import numpy as np
import pytest

from oracle import mera as om
from paper_2007_03638_gb300 import inputs as inp
from tests import bruteforce as bf


def _rand_herm(rng, n, pd=False):
    a = rng.standard_normal((n, n))
    if pd:
        a = a @ a.T + 0.1 * np.eye(n)
        return a / np.trace(a)
    return 0.5 * (a + a.T)


def test_bruteforce_finite_mera_energy_and_rdm():
    """16-spin periodic binary MERA: state vector vs ascending/descending maps.

    Two layers (spin dim 2 -> 4 -> 4), a random top state on 4 sites of dim 4.
    The energy density of the dense state must equal Tr(Abar(Abar(h)) rho_top)
    and the averaged 3-site density matrix at the bottom must equal
    Dbar(Dbar(rho_top)) (Sec. 4 networks; both causal-cone parities)."""
    rng = np.random.default_rng(7)
    u0 = inp._haar_like(rng, 4, 4, np.float64)
    w0 = inp._haar_like(rng, 4, 4, np.float64)
    u1 = inp._haar_like(rng, 16, 16, np.float64)
    w1 = inp._haar_like(rng, 16, 4, np.float64)
    top = rng.standard_normal((4, 4, 4, 4))
    top /= np.linalg.norm(top)
    psi = bf.finite_mera_state(top, [(u1, w1), (u0, w0)])
    assert psi.shape == (2,) * 16
    assert abs(np.linalg.norm(psi) - 1) < 1e-12
    bond = inp.ising_bond(1.0)
    e_bf = bf.energy_density(psi, bond)
    h3 = inp.three_site_unblocked(bond)
    rho_top = bf.averaged_rdm3(top)
    e_or = np.trace(om.ascend(om.ascend(h3, u0, w0), u1, w1) @ rho_top)
    assert abs(e_bf - e_or) < 1e-13
    rho_bf = bf.averaged_rdm3(psi)
    rho_or = om.descend(om.descend(rho_top, u1, w1), u0, w0)
    assert np.abs(rho_bf - rho_or).max() < 1e-13


def test_bruteforce_8_sites_complex():
    """Complex tensors on 8 spins (one layer 2 -> 4 plus a 4-site top)."""
    rng = np.random.default_rng(3)
    u0 = inp._haar_like(rng, 4, 4, np.complex128)
    w0 = inp._haar_like(rng, 4, 4, np.complex128)
    top = rng.standard_normal((4,) * 4) + 1j * rng.standard_normal((4,) * 4)
    top /= np.linalg.norm(top)
    psi = bf.finite_mera_state(top, [(u0, w0)])
    bond = inp.xxz_bond(0.7)
    e_bf = bf.energy_density(psi, bond)
    e_or = np.trace(om.ascend(inp.three_site_unblocked(bond), u0, w0) @ bf.averaged_rdm3(top))
    assert abs(e_bf - e_or) < 1e-13


@pytest.mark.parametrize("side", ["L", "R"])
@pytest.mark.parametrize("dt", [np.float64, np.complex128])
def test_descend_matches_dense_cone(side, dt):
    """Each one-sided descending map equals the partial trace of V rho V^dag
    with V the dense causal-cone isometry (u on (2j+1, 2j+2))."""
    rng = np.random.default_rng(11)
    u = inp._haar_like(rng, 9, 9, dt)
    w = inp._haar_like(rng, 9, 2, dt)
    r = rng.standard_normal((8, 8)) + (1j * rng.standard_normal((8, 8)) if dt == np.complex128 else 0)
    assert np.abs(om.descend_side(r, u, w, side) - bf.dense_descend(r, u, w, side)).max() < 1e-13


def test_unitality_trace_and_adjointness():
    rng = np.random.default_rng(5)
    us, ws = inp.random_mera(4, 4, 1, seed=5)
    u, w = us[0], ws[0]
    one = np.eye(64)
    assert np.abs(om.ascend(one, u, w) - one).max() < 1e-13
    r = _rand_herm(rng, 64, pd=True)
    assert abs(np.trace(om.descend(r, u, w)) - 1) < 1e-13
    o = rng.standard_normal((64, 64))
    lhs = np.trace(om.ascend(o, u, w) @ r)
    rhs = np.trace(o @ om.descend(r, u, w))
    assert abs(lhs - rhs) < 1e-13


@pytest.mark.parametrize("bond,exact", [(inp.ising_bond(1.0), -1.0), (inp.xxz_bond(1.0), 1.0),
                                        (inp.xxz_bond(0.3), 0.3)])
def test_product_state_closed_form(bond, exact):
    """u = 1, w|k> = |k>|0>: the MERA is the product state |00...>; its energy
    per spin is <00|bond|00> and the fixed point is |000><000|."""
    us, ws = inp.product_state_mera(4, 2)
    h3 = inp.three_site_blocked(bond)
    e, ds, info = om.energy_grad(h3, us, ws)
    assert abs(e / 2 - exact) < 1e-12
    rho = info["rho"][-1]
    target = np.zeros_like(rho)
    target[0, 0] = 1.0
    assert np.abs(rho - target).max() < 1e-12


def _dense_super(u, w):
    """Dense matrix of Dbar_S built from the brute-force cone isometries."""
    c = w.shape[1]
    n = c**3
    M = np.zeros((n * n, n * n), dtype=np.result_type(u, w))
    for k in range(n * n):
        e = np.zeros(n * n, dtype=M.dtype)
        e[k] = 1
        E = e.reshape(n, n)
        M[:, k] = 0.5 * (bf.dense_descend(E, u, w, "L") + bf.dense_descend(E, u, w, "R")).ravel()
    return M


@pytest.mark.parametrize("chi", [2, 3])
def test_fixed_point_and_series_vs_dense(chi):
    """App. B: rho_S is the unit-trace eigenvector of Dbar_S for eigenvalue 1;
    x solves x (1 - A') = <h| with A' = A - |rho><1|.  Both checked against a
    dense eigendecomposition / dense linear solve of the brute-force
    superoperator; the spectrum of Dbar_S lies in the unit disk."""
    rng = np.random.default_rng(chi)
    u = inp._haar_like(rng, chi * chi, chi * chi, np.float64)
    w = inp._haar_like(rng, chi * chi, chi, np.float64)
    M = _dense_super(u, w)
    vals, vecs = np.linalg.eig(M)
    k = np.argmax(np.abs(vals))
    assert abs(vals[k] - 1) < 1e-12
    assert np.sort(np.abs(vals))[-2] < 1 - 1e-6
    rho_dense = vecs[:, k].reshape(chi**3, chi**3)
    rho_dense = (rho_dense / np.trace(rho_dense)).real
    rho, lam = om.si_fixed_point(u, w)
    assert abs(lam - 1) < 1e-12
    assert np.abs(rho - rho_dense).max() < 1e-11
    assert np.abs(rho - rho.T).max() < 1e-15
    assert np.linalg.eigvalsh(rho).min() > -1e-12
    h = _rand_herm(rng, chi**3)
    n = chi**6
    # Abar is the transpose of Dbar in the vectorised Hilbert-Schmidt pairing.
    perm = np.arange(n).reshape(chi**3, chi**3).T.ravel()
    A_T = M[perm][:, perm]  # vec(D(r))^T-pairing: <h|A = vec of Abar(h)
    # operator x -> x - Abar(x) + Tr(x rho) 1, dense
    Aasc = A_T.T
    one = np.eye(chi**3).ravel()
    op = np.eye(n) - Aasc + np.outer(one, rho.T.ravel())
    x_dense = np.linalg.solve(op, h.ravel()).reshape(chi**3, chi**3)
    x = om.si_env_series(h, rho, u, w)
    assert np.abs(x - x_dense).max() < 1e-10 * max(1, np.abs(x_dense).max())
    # ascending map via the dense matrix agrees with the network
    assert np.abs((Aasc @ h.ravel()).reshape(chi**3, chi**3) - om.ascend(h, u, w)).max() < 1e-13


def _tangent(rng, W, kind):
    X = rng.standard_normal(W.shape)
    if kind == "stiefel":
        return X - 0.5 * W @ (W.T @ X + X.T @ W)
    return X - W @ (W.T @ X)


@pytest.mark.parametrize("which", ["u0", "w0", "u1", "w1", "uS", "wS", "all"])
def test_gradient_finite_differences(which):
    """Central differences of C(W + eps X) against Re Tr D^dag X (Sec. 2.3) for
    tangent directions X on single tensors and on all tensors at once."""
    us, ws = inp.random_mera(4, 4, 2, seed=21)
    h3 = inp.three_site_blocked(inp.ising_bond(1.0))
    pt = [t for pair in zip(us, ws) for t in pair]
    e, ds, _ = om.energy_grad(h3, us, ws)
    names = ["u0", "w0", "u1", "w1", "uS", "wS"]
    rng = np.random.default_rng(100 + (names + ["all"]).index(which))
    eps = 1e-5
    for trial in range(2):
        X = [np.zeros_like(t) for t in pt]
        for i, nm in enumerate(names):
            if which in ("all", nm):
                X[i] = _tangent(rng, pt[i], "stiefel" if nm[0] == "u" else "grassmann")
        def C(t):
            p = [a + t * x for a, x in zip(pt, X)]
            return om.energy(h3, p[0::2], p[1::2])
        fd = (C(eps) - C(-eps)) / (2 * eps)
        an = sum(float(np.sum(d * x)) for d, x in zip(ds, X))
        assert abs(fd - an) < 1e-7 * max(1.0, abs(an)), (which, fd, an)


def test_identity_shift_and_level_independence():
    """Adding c*1 to h shifts e by c and leaves the projected gradient unchanged
    (App. A/B); Tr(h_l rho_l) is the same at every level."""
    from oracle import geometry as geo
    us, ws = inp.random_mera(4, 4, 2, seed=4)
    h3 = inp.three_site_blocked(inp.ising_bond(1.0))
    e1, d1, info = om.energy_grad(h3, us, ws)
    e2, d2, _ = om.energy_grad(h3 + 0.75 * np.eye(64), us, ws)
    assert abs(e2 - e1 - 0.75) < 1e-12
    pt = [t for pair in zip(us, ws) for t in pair]
    for i, (W, a, b) in enumerate(zip(pt, d1, d2)):
        kind = "stiefel" if i % 2 == 0 else "grassmann"
        assert np.abs(geo.project(W, a, kind) - geo.project(W, b, kind)).max() < 1e-11
    for l in range(3):
        assert abs(np.trace(info["h"][l] @ info["rho"][l]) - e1) < 1e-12


def test_grassmann_gauge_invariance():
    """w_0 -> w_0 U with u_1 -> (U^dag (x) U^dag) u_1 leaves the state, hence the
    energy, unchanged (Sec. 4 footnote on the Grassmann manifold)."""
    us, ws = inp.random_mera(4, 4, 2, seed=9)
    h3 = inp.three_site_blocked(inp.xxz_bond(1.0))
    rng = np.random.default_rng(1)
    U = inp._haar_like(rng, 4, 4, np.float64)
    us2, ws2 = list(us), list(ws)
    ws2[0] = ws[0] @ U
    us2[1] = np.kron(U.T, U.T) @ us[1]
    e1 = om.energy(h3, us, ws)
    e2 = om.energy(h3, us2, ws2)
    assert abs(e1 - e2) < 1e-12


def _site_rdm(psi, sites):
    """Reduced density matrix of the listed sites (in that order) of a state tensor."""
    d = [psi.shape[k] for k in sites]
    p = np.moveaxis(psi, sites, list(range(len(sites)))).reshape(int(np.prod(d)), -1)
    return p @ p.conj().T / np.vdot(psi, psi).real


@pytest.mark.parametrize("dt", [np.float64, np.complex128])
def test_tensor_density_matrices_vs_dense_sites(dt):
    """rho_w and rho_u of the binary network (Sec. 4: the density matrix on a
    tensor's top legs) from a 3-site density matrix that is NOT averaged over
    positions: the reduced state of coarse sites (0, 1, 2) of a random
    periodic 4-site state.  rho_w must be the one-site state of coarse site 1
    (the middle site); rho_u the two-site state of the fine pair (1, 2) of
    W|psi> -- the right output of w on coarse site 0 and the left output of w
    on coarse site 1, the pair a disentangler acts on -- both by partial trace
    of the dense state.  A wrong site, a wrong pair, a transposed or
    conjugated w fails here (the state has no symmetry that hides them)."""
    rng = np.random.default_rng(21)
    c, cp = 2, 3
    w = inp._haar_like(rng, c * c, cp, dt)
    top = rng.standard_normal((cp,) * 4) + (1j * rng.standard_normal((cp,) * 4) if dt == np.complex128 else 0)
    top /= np.linalg.norm(top)
    rho3 = _site_rdm(top, [0, 1, 2])
    ru, rw = om.tensor_density_matrices([rho3], [w])
    assert np.abs(rw - _site_rdm(top, [1])).max() < 1e-14
    fine = bf.apply_isometry_layer(top, w)  # 8 fine sites, no disentanglers
    assert np.abs(ru - _site_rdm(fine, [1, 2])).max() < 1e-14
    # the other choices differ on this state (so the comparison above is sharp)
    assert np.abs(rw - _site_rdm(top, [0])).max() > 1e-3
    assert np.abs(ru - _site_rdm(fine, [3, 4])).max() > 1e-3
    assert np.abs(ru - _site_rdm(fine, [0, 1])).max() > 1e-3


@pytest.mark.parametrize("dt", [np.float64, np.complex128])
def test_tensor_density_matrices_vs_dense_average(dt):
    """With the position-averaged 3-site density matrix of a periodic 4-site
    state (the form the MERA's level density matrices have), rho_w is the
    average one-site state and rho_u the average, over the four disentangler
    positions (2j+1, 2j+2) of the fine chain W|psi>, of the two-site state;
    both have unit trace and are Hermitian, positive semidefinite."""
    rng = np.random.default_rng(22)
    c, cp = 2, 3
    w = inp._haar_like(rng, c * c, cp, dt)
    top = rng.standard_normal((cp,) * 4) + (1j * rng.standard_normal((cp,) * 4) if dt == np.complex128 else 0)
    top /= np.linalg.norm(top)
    ru, rw = om.tensor_density_matrices([bf.averaged_rdm3(top)], [w])
    one = sum(_site_rdm(top, [k]) for k in range(4)) / 4
    assert np.abs(rw - one).max() < 1e-14
    fine = bf.apply_isometry_layer(top, w)
    two = sum(_site_rdm(fine, [(2 * j + 1) % 8, (2 * j + 2) % 8]) for j in range(4)) / 4
    assert np.abs(ru - two).max() < 1e-14
    for r in (ru, rw):
        assert abs(np.trace(r) - 1) < 1e-13
        assert np.abs(r - r.conj().T).max() < 1e-15
        assert np.linalg.eigvalsh(r).min() > -1e-14


def test_tensor_density_matrices_levels():
    """Layer l's matrices come from the level above (rho_{l+1}); the
    scale-invariant layer's from rho_S itself."""
    rng = np.random.default_rng(23)
    ws = [inp._haar_like(rng, 4, 3, np.float64), inp._haar_like(rng, 9, 3, np.float64)]
    rhos = []
    for _ in range(2):
        t = rng.standard_normal((3,) * 4)
        rhos.append(bf.averaged_rdm3(t / np.linalg.norm(t)))
    out = om.tensor_density_matrices(rhos, ws)
    r0 = om.tensor_density_matrices([rhos[1]], [ws[0]])
    r1 = om.tensor_density_matrices([rhos[1]], [ws[1]])
    for a, b in zip(out, r0 + r1):
        assert np.abs(a - b).max() == 0.0
