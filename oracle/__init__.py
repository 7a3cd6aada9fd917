"""Plain FP64 CPU oracle for the FDLB solver of the simplified Enskog equation in
cylindrical and spherical geometry (Busuioc, arXiv 2403.15051).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, calls or links this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
legs of ``bench.py`` use it.  It shares no code with the CUDA library.

Modules (each function cites the passage of the paper it restates):

* ``quadrature``  - full-range and half-range Gauss-Hermite rules (Sec. III.A).
* ``equilibrium`` - discrete per-axis equilibria g^H and g^h (Sec. III.C).
* ``kmatrix``     - momentum-derivative matrices K (Sec. III.B).
* ``model``       - Carnahan-Starling chi, transport coefficients, Kn <-> C (Sec. II).
* ``geometry``    - radial grid, metric factors and Fischer-Methfessel weights (App. A).
* ``solver``      - moments, closure, RHS, diffuse walls and the SSP-RK3 step (Sec. II-III).
"""
