"""Plain, slow FP64 CPU oracle of the energy-conserving MRT finite-difference
lattice Boltzmann model (Chen, Xu, Zhang, Li; D2V16, arXiv 0908.3749).

THIS PACKAGE IS TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
it. The GPU library never calls it and shares no code, table or constant with it.

Modules
-------
lattice   Eq. 4 velocity set, Eqs. 5a-5p moment matrix M, M^-1 by Gauss-Jordan.
scheme    Eq. 14 equilibria, Eq. 3 collision, Eq. A.1 time/space discretisation,
          ghost-node boundary conditions of Sec. V, initial state, macroscopics.
exact     Reference solutions used to pin the scheme: exact Riemann solver,
          Rankine-Hugoniot (normal and oblique) shocks, Couette series, the
          relative error E of Sec. V.A.

Every function states the passage of the paper it follows. Readings of places
where the paper is silent or ambiguous are listed in the module docstrings.
Parity status: every function here is pinned by a ``-m "not gpu"`` test except
those whose docstring says "parity unpinned".
"""
