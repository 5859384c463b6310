"""The seeded input recipes (CPU): the sign-fixed QR-of-Gaussian starting point
of the MERA workloads and the Poisson request stream of the serving workload
(arrival rate, model mix, parameter ranges, bond dimensions)."""
import numpy as np
import pytest

from paper_2007_03638_gb300 import inputs as inp


@pytest.mark.parametrize("dt", [np.float64, np.complex128])
def test_random_mera_is_the_sign_fixed_qr_of_gaussians(dt):
    d_b, chi, L, seed = 4, 8, 3, 11
    us, ws = inp.random_mera(d_b, chi, L, seed=seed, dtype=dt)
    dims = inp.layer_dims(d_b, chi, L)
    assert [u.shape for u in us] == [(c * c, c * c) for c in dims]
    assert [w.shape for w in ws] == [(dims[l] ** 2, dims[min(l + 1, L)]) for l in range(L + 1)]
    # regenerate the Gaussians in the recipe's order and check Q^dag G = R
    rng = np.random.default_rng(seed)
    for l in range(L + 1):
        for W in (us[l], ws[l]):
            n, p = W.shape
            G = rng.standard_normal((n, p))
            if dt == np.complex128:
                G = G + 1j * rng.standard_normal((n, p))
            R = W.conj().T @ G
            assert np.abs(W.conj().T @ W - np.eye(p)).max() < 1e-13
            assert np.abs(np.tril(R, -1)).max() < 1e-11 * np.abs(G).max()
            assert np.diag(R).real.min() > 0


def test_poisson_stream_recipe():
    serve = pytest.importorskip("paper_2007_03638_gb300.serve")
    n, rate = 2000, 50.0
    reqs = serve.poisson_stream(n, rate=rate, chis=(4, 8), seed=7)
    t = np.array([r["t"] for r in reqs])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0)
    assert abs(gaps.mean() * rate - 1.0) < 5 / np.sqrt(n)          # exponential gaps, mean 1/rate
    assert abs(gaps.std() * rate - 1.0) < 0.1
    ising = np.array([r["model"] == "ising" for r in reqs])
    assert abs(ising.mean() - 0.5) < 5 * 0.5 / np.sqrt(n)
    for r in reqs:
        assert r["chi"] in (4, 8)
        lo, hi = (0.5, 1.5) if r["model"] == "ising" else (0.0, 2.0)
        assert lo <= r["param"] <= hi
        h = r["h3"]
        assert np.abs(h - h.T).max() < 1e-14
    for r in reqs[:20]:
        for W in r["tensors"]:
            assert np.abs(W.T @ W - np.eye(W.shape[1])).max() < 1e-13
    again = serve.poisson_stream(5, rate=rate, chis=(4, 8), seed=7)
    assert [(a["t"], a["model"], a["param"], a["chi"]) for a in again] == \
        [(a["t"], a["model"], a["param"], a["chi"]) for a in reqs[:5]]


def test_z2_inputs_of_the_binary_network():
    """Blocked spin pairs in the parity-ordered basis: the Ising and Heisenberg
    three-site terms commute with the parity under the first-half-even grading
    (they do not in the plain product basis) and keep their spectrum; the
    seeded symmetric binary MERA is made of symmetric isometries."""
    from oracle import z2
    p3 = inp.fused_parities(4, 4, 4)
    for bond in (inp.ising_bond(1.0), inp.xxz_bond(1.0)):
        h = inp.three_site_blocked(bond)
        ho = inp.parity_ordered_three_site(h)
        assert z2.violation(ho, p3, p3) == 0.0
        assert np.allclose(np.linalg.eigvalsh(ho), np.linalg.eigvalsh(h), atol=1e-12)
    assert z2.violation(inp.three_site_blocked(inp.ising_bond(1.0)), p3, p3) > 0.1
    us, ws = inp.random_z2_mera(4, 8, 3, seed=2)
    dims = inp.layer_dims(4, 8, 3)
    for l, (u, w) in enumerate(zip(us, ws)):
        c, cp = dims[l], dims[min(l + 1, 3)]
        pair = inp.fused_parities(c, c)
        assert z2.violation(u, pair, pair) == 0.0 and z2.violation(w, pair, inp.z2_parities(cp)) == 0.0
        assert np.abs(w.T @ w - np.eye(cp)).max() < 1e-13
