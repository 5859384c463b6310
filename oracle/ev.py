"""Evenbly-Vidal tensor updates for the binary MERA, FP64 (the comparator the
paper sets its Riemannian optimisers against).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

App. ev_steplimit (with the Evenbly-Vidal paragraph of Sec. 4): one tensor W
is updated at a time with the others held fixed.  The cost is redefined with
the shifted Hamiltonian H_gamma = H - gamma 1 (gamma large enough that
H_gamma is negative definite, so that minimising the energy is maximising
|C|); the environment D_gamma = 2 dC_gamma / d conj(W) of that cost is
polar-decomposed, D_gamma = Q P, and W is replaced by the polar factor.  The
sign is irrelevant to C (every tensor enters with even powers); this oracle
takes W <- -Q, which keeps W's sign near a fixed point (there
D_gamma = W (S - gamma rho) with S - gamma rho negative definite, so Q = -W).
A sweep updates u_0, w_0, ..., u_S, w_S in that order, each with a freshly
computed environment.  Fixed points are exactly the points where the
Stiefel gradient of D_gamma vanishes.

Reading: the shift is applied to the 3-site term (h3 - gamma 1), which
shifts the energy per bottom site by -gamma; the environment is computed
exactly for that Hamiltonian (no first-order formula).

Pins (tests/test_oracle_ev.py): the polar factor maximises Re Tr(D^dag W)
over isometries; a point built as W = -polar(D) is a fixed point with zero
Stiefel gradient; sweeps lower the energy of a small critical-Ising MERA.
"""
from __future__ import annotations

import numpy as np

from . import mera as om


def polar_factor(D):
    """(App. ev_steplimit) Q of the polar decomposition D = Q P (Q isometric, P = Q^dag D Hermitian
    positive semidefinite): Q = U V^dag from the thin SVD D = U S V^dag."""
    u, _, vh = np.linalg.svd(D, full_matrices=False)
    return u @ vh


def ev_update(D):
    """The new tensor for environment D: -Q (App. ev_steplimit; the sign is
    discussed in the module docstring)."""
    return -polar_factor(D)


def ev_sweep(h3, us, ws, gamma, tol=1e-14, network="binary"):
    """One Evenbly-Vidal sweep (Sec. 4, App. ev_steplimit): for i = 0..2L+1 (u_0, w_0, ..., u_S, w_S), recompute the
    environments of the shifted cost at the current point and replace tensor
    i by -polar(D_i).  Returns (us, ws, energies) with energies[i] the energy
    per bottom site (unshifted) after update i.  network: "binary" (h3 a
    three-site term) or "ternary" (a two-site term, oracle/ternary.py)."""
    if network == "ternary":
        from . import ternary as net
    else:
        net = om
    us = [u.copy() for u in us]
    ws = [w.copy() for w in ws]
    hs = np.asarray(h3) - gamma * np.eye(np.asarray(h3).shape[0])
    energies = []
    for i in range(2 * len(us)):
        _, ds, _ = net.energy_grad(hs, us, ws, tol=tol)
        l, k = divmod(i, 2)
        if k == 0:
            us[l] = ev_update(ds[i])
        else:
            ws[l] = ev_update(ds[i])
        energies.append(net.energy(h3, us, ws, tol=tol))
    return us, ws, energies
