"""FP64 CPU oracle for the heat-kernel Sinkhorn on S^2 (the SHOT method).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, deliberately
unoptimised restatement of the method in float64 numpy, written from the
paper's text:

* Gauss-Legendre grid and area weights (App. C.1 "Gauss-Legendre"; App. C.2,
  a^T 1 = 4 pi),
* orthonormal associated Legendre functions and spherical harmonics (App. B),
* the semi-naive spherical harmonic transform: longitude DFT + per-order
  Legendre projection (App. C.1, last paragraph),
* the heat convolution HeatConv(v; h) = F^{-1}(h (.) F(v)), h_l = exp(-t l(l+1))
  (Sec. 3.2),
* the dense heat matrix from the Legendre series (addition theorem) for tiny
  grids,
* Algorithm 1 (balanced and unbalanced Sinkhorn with the translation-invariant
  step, the periodic marginal check of App. C.3, the dual-objective return of
  App. C.2) and the Sinkhorn divergence of eq. (sinkhorn-divergence),
* finite-difference and envelope gradients of the divergence.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import it.  It shares no code with
the CUDA library and never imports it; the CUDA path never imports this.
"""
