"""Plain CPU FP64 oracle for the MERA energy/gradient and the Riemannian step.

TEST INFRASTRUCTURE ONLY.  This package is the slow, obviously-correct
restatement of the method (Hauru, Van Damme, Haegeman, "Riemannian
optimization of isometric tensor networks", arXiv:2007.03638) that the CUDA
library is checked against.  Only the test-suite, ``__graft_entry__.smoke()``
and ``bench.py``'s CPU-baseline / reference leg may import it; the product
path (``paper_2007_03638_gb300``) never does, and the two share no code.

Modules
-------
``mera``      binary MERA networks (ascending/descending superoperators, Sec. 4),
              the scale-invariant fixed point and environment series (App. B),
              partial derivatives D_v (Sec. 4).
``geometry``  tangent projection, exponential retraction, vector transport,
              metric, Hilbert-space preconditioner (Sec. 2, Sec. 3).
``optim``     Hager-Zhang line search, L-BFGS two-loop and nonlinear CG on the
              product manifold (Sec. 3).
``ternary``   the ternary MERA's three ascending maps of two-site operators,
              its scale-invariant layer and derivatives (Sec. 4, App. B).
``ev``        Evenbly-Vidal updates and sweeps (App. ev_steplimit).
``mps``       the uniform MPS: transfer maps, energy, derivative and
              preconditioner (Sec. 5).
``z2``        Z2 symmetry: charge violation, blockwise geometry (Sec. 6).
``rng``       the seeded generator and sign-fixed QR-of-Gaussian isometries of
              the library's random initialisation.
"""
