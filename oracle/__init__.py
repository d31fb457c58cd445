"""FP64 CPU oracle for the exact-gradient path of SIMP compliance minimisation.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or link this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` use it.  It shares no code with the CUDA
library; the only common inputs are the seeded arrays of
``paper_2104_12282_gb300.problems``.

What it computes (the plain definitions of §III-D, Eq. 4 and Eq. 5):

* ``fem``      -- hex8 unit stiffness K0 (2x2x2 Gauss, exact), element DOF map, sparse
                  assembly of K(rho) and the same operator applied element by element;
* ``solve``    -- K_ff u_f = f_f by a sparse direct factorisation or Jacobi-PCG;
* ``filt``     -- the density filter P = diag(1/Hs) H with cone weights, forward and
                  transposed (the volume gradient is P^T v);
* ``oc``       -- the optimality-criteria update with bisection on the multiplier;
* ``topopt``   -- compliance, sensitivities (Eq. 5 with the SIMP chain rule), the
                  filtered gradient and the OC loop.

Every function is pinned by ``tests/test_oracle_*.py`` against facts fixed by the
mathematics or the paper (rigid-body modes, exact symbolic integration, patch test,
energy identity, finite differences, beam theory, Table 1 counts, closed-form OC
multiplier).  The absolute compliance values of the named workloads are not printed in
the paper; for those the oracle is checked only through the pinned components.
"""
