"""Plain, slow, FP64 CPU oracle for the 2D Fourier Continuation (2D-FC) hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The CUDA library never imports, links or calls anything here, and this
package shares no code, table or constant generator with it: the only module both
sides use is ``workloads.py`` (seeded inputs, no method arithmetic).

Every function follows Bruno & Paul, "Two-dimensional Fourier Continuation and
applications" (arXiv 2010.03901), and cites the section / equation it restates.

Modules
-------
fc_matrices   Section 2.2 + Remark "Blending to zero on a refined grid": Gram QR,
              oversampled Gram values, SVD least-squares trig fit, A and A_r.
              (50-digit ``decimal`` arithmetic; cached in tests/golden.)
fc1d          Section 2.3, eq. (2.5): the 1D-FC continuation (used as a pin).
geometry      Section 3.1, eqs. (3.1)-(3.5): boundary, normals, grid, crossings,
              inside test, feet of normals and the strip set H cap V+.
fc2d          Sections 3.2-3.6: matching values, blending, interpolation onto the
              Cartesian strip, the 2D-FC extension and its DFT.
poisson       Section 4.1, eqs. (4.1)-(4.6): particular solution, boundary
              interpolation, Laplace BIE correction.
wave          Section 4.2, eqs. (4.7)-(4.13): Fourier Forwarding.

Functions whose result the paper does not fix numerically and that no closed form
or brute force pins are marked "parity unpinned" in their docstring.
"""
