"""FP64 CPU oracle of the coupled IMEX domain-decomposition scheme for ES-BGK.

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously-correct
reference against which the CUDA library is checked.  Only the tests, the
``smoke()`` entry of ``__graft_entry__`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import it.  The product path (the
CUDA library and its Python binding) never imports, links or calls anything in
here, and nothing in here imports the product package.  Both sides are fed by
the seeded generators in ``workloads``, which hold none of the method's
arithmetic.

Every function follows a numbered place of Caparello & Tenna, "A Coupled IMEX
Domain Decomposition Method for High-Order Time Integration of the ES-BGK Model
of the Boltzmann Equation" (arXiv 2512.03586); the citation is in each
docstring.  Where the paper is silent the reading taken is stated in the
docstring as "Reading R<n>".

Arithmetic is numpy float64.  Library primitives used as steps: ``np.sum``,
``np.einsum``, ``np.linalg.solve``/``inv``/``det``/``eigvalsh``.

Parity status per function (what pins it is in ``tests/test_oracle_*.py``):
pinned -- moments, Gaussian, projected Gaussian, relaxation, CWENO3, transport,
Euler flux, regime criterion, tableaux, stepper (order, conservation, limits),
and the learned switch in ``oracle.cnn`` (network forward and gradients,
features, Adam, the learned map rule).
The dissipation speed of the Euler flux (local Lax-Friedrichs,
max |u_n| + sqrt(gamma P / rho)) is pinned by the closed-form linearisation
of the scheme about a uniform moving state (tests/test_oracle_transport.py).
Parity unpinned beyond invariants: the CWENO epsilon value and linear weights
(d_0 = 1/2, d_L = d_R = 1/4: any weights give the optimal parabola on smooth
data by construction of P_0), the choice of the
quadratic moment projection and the criterion constants (paper's printed
d_v = 3 values), which are readings, not results the paper fixes.
"""

from .kinetic import (velocity_grid, moments, macro_from_moments, gaussian,
                      projected_gaussian, maxwellian_hat, es_gaussian_of, relax,
                      cons_from_prim, prim_from_cons, cons_from_moments)
from .transport import pad_cells, cweno3_faces, cweno3_indicators, kinetic_transport, euler_phi, euler_flux
from .scheme import (Problem, State, ARS233, IMEX_EULER, ARS222, SSP2_332, Tableau, init_state,
                     regime_indicators, regime_update, convert, buffer_mask,
                     advance, step, totals, macro)
from . import cnn

__all__ = [n for n in dir() if not n.startswith("_")]
