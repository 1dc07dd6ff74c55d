"""FP64 CPU oracle for the spectral-element wave step and its Hilbert reordering.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package. The product path (``paper_2104_08416_gb300`` and its CUDA library)
never imports it, and this package imports nothing from the product.

It is a plain, slow, direct restatement of what the paper's method computes
(Araujo, Gross, Xavier-de-Souza, "Boosting memory access locality of the
spectral element method with Hilbert space-filling curves", 2021), in float64:

* ``gll``       -- GLL nodes, weights and the Lagrange derivative matrix
                   (nodal basis / quadrature, Section 4.2, Eqs. dual_sys,
                   numerical_integ).
* ``mesh``      -- canonical global numbering mu(p, e) of the SEM nodes of a
                   quad mesh, bilinear element maps and Jacobians
                   (Section 4.2, element map and Eq. deriv_u).
* ``sem``       -- lumped diagonal mass (Eq. Abar with A = M = 1/K), dense
                   element stiffness matrices and their assembly
                   (Eq. u_change_r_effic), the Ricker point source snapped to a
                   node (Eq. u_change, Algorithm 3), leapfrog time stepping,
                   discrete energy, CFL step.
* ``hilbert``   -- the standard Hilbert curve as defined by Listing 1
                   (Section 3), a textbook index-to-cell map used to pin it,
                   and the generalized W x H curve used by the element
                   reordering (Section 4.3, after Cerveny 2020).
* ``ordering``  -- element reordering by the curve (Section 4.3, steps 1-4),
                   node renumbering by first touch sorted by degree
                   (Section 4.3, Cuthill-McKee-like procedure), and the
                   row-major / random baselines (Section 6.1, "No Strategy").
* ``cpp``       -- the same mass, stiffness and leapfrog as ``sem`` in plain
                   C loops with OpenMP (``sem_ref.c``): the multi-core CPU
                   baseline that bench.py times, pinned to ``sem``.

Readings of passages the paper leaves open are listed in the repository's
design notes and repeated in the docstring of the function that takes them.
Parity status: every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, brute force, hand-traced values of Listing 1 or
published test vectors; none is "parity unpinned".
"""
from . import gll, mesh, sem, hilbert, ordering  # noqa: F401
