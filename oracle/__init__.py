"""FP64 CPU oracle for the COLA particle-mesh hot path (ICE-COLA, Izard, Crocce &
Fosalba 2016, arXiv:1509.04685).

This package is TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
The product path (the CUDA library in ``paper_1509_04685_gb300``) never imports,
links or executes anything from here, and this package shares no code, table or
constant generator with it.

Everything is plain NumPy/SciPy in float64, written to be checked by eye against
the paper and the textbook definitions it relies on:

* ``cosmology`` -- E(a), Eisenstein & Hu no-wiggle P(k), sigma_8 normalisation,
  growth factors D1, D2, kick/drift integrals, time nodes (Eq. 3).
* ``philox``    -- Philox-4x32-10 counter RNG and the Box-Muller normal draw
  used for the seeded white noise of the initial conditions (Sec. 2.2).
* ``lpt``       -- linear field and 2LPT displacements Psi1, Psi2 (Sec. 2.2).
* ``pm``        -- CIC deposit, k-space Green's function + ik gradient, CIC
  gather: the particle-mesh force (Sec. 2.2, Eq. 2 right-hand side).
* ``cola``      -- the COLA kick-drift-kick loop in the LPT frame (Eqs. 1-2).
* ``power``     -- the matter P(k) estimator (Sec. 2.5).
* ``fof``       -- friends-of-friends groups (linking length b of the mean
  spacing), halo catalogue with Warren masses, mass function (Secs. 2.1, 2.4).
* ``dft``       -- a direct O(N^2) DFT used to pin numpy's FFT.
* ``learned``   -- FP64 forward/backward of the learned coarse-mesh force
  correction (k-space filter + 3-layer 3D conv net).  The paper has no such
  part; it is pinned by finite differences.

Parity status per function is stated in each module header.
"""
