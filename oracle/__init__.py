"""CPU oracle for the D2Q37 thermal lattice Boltzmann time step.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import anything under ``oracle/``.
The product path (the CUDA library and its Python binding) never calls it and
shares no code, table or constant generator with it.

The oracle is plain NumPy in float64 (and complex128 for complex-step
derivatives), vectorised over lattice sites, looping over the 37 populations
in the notation of the paper:

* ``oracle.lattice``  - the D2Q37 velocity set and its quadrature weights,
  solved here from the isotropy conditions (the paper names the model in
  Sect. 2 and delegates its definition to the works it cites).
* ``oracle.model``    - eq. (1) (BGK evolution), eq. (2) (macroscopic fields),
  the Hermite equilibrium, propagate, bc and collide of Sect. 2, and the time
  loop.
* ``oracle.adjoint``  - the discrete adjoint of one time step.

Where the paper is silent the readings used are listed in each module's
docstring.
"""
