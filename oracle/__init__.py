"""Plain, slow FP64 CPU oracle for the lattice-field hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the C-ABI library
``liblqcd.so`` and its Python binding ``paper_1105_2279_gb300``) imports,
links or runs this package.  Only ``tests/``, ``__graft_entry__.smoke()``
and ``bench.py`` (its ``cpu_baseline`` leg and ``--impl reference`` arm)
may use it.

What it computes, each in complex128 numpy with whole-lattice array
operations (``np.roll`` for shifts, ``@`` for 3x3 products):

* ``lattice``  -- geometry and the periodic ``shift`` of the paper's
  Listing 1 (Sec. 6): ``shift(f, FORWARD, mu)(x) = f(x + mu)``.
* ``su3``      -- adjoint, trace, traceless anti-Hermitian projection.
* ``expm``     -- brute-force matrix exponential (scaling and squaring of a
  30-term Taylor series) and its Frechet derivative via the 2n x 2n block
  matrix identity.
* ``stout``    -- stout link smearing (staple sum, Omega, Q, Cayley-Hamilton
  exp(iQ), link update), following Morningstar & Peardon, Phys. Rev. D 69
  (2004) 054501, Secs. II-III.  The paper this project accelerates
  (Winter, "Accelerating QDP++ using GPUs", Sec. 6) uses a smearing routine
  as its application; stout smearing is the routine taken here.
* ``gauge``    -- plaquette, Wilson action, per-site action, gauge
  transformations and the Wilson-action gradient.
* ``backward`` -- reverse-mode gradient of a scalar through n stout steps,
  built only from the chain rule, ``expm`` and its Frechet derivative
  (independent of the closed-form stout-force formulas).
* ``expr``     -- the reference semantics of the fused expression programs
  and of the Jacobi smearing routine of Listing 1.
* ``ape``      -- APE link smearing (Albanese et al., Phys. Lett. B 192
  (1987) 163): links mixed with their staples, projected back to SU(3) by
  the unitary polar factor with the determinant phase removed.
* ``ape_force`` -- reverse-mode gradient through APE steps: the SU(3)
  projection's gradient from Jacobi's determinant formula and the
  Daleckii-Krein formula for the Frechet derivative of A^(-1/2), and the
  staple sum's from ``backward``.
* ``hyp``      -- HYP smearing (Hasenfratz and Knechtli, Phys. Rev. D 64
  (2001) 034504): three nested APE-type levels with staples confined to the
  hypercubes attached to the link.
* ``hyp_force`` -- reverse-mode gradient through HYP steps: the three levels
  backwards, each through the projection's gradient of ``ape_force`` and a
  two-field staple gradient.

Field convention: a link field is an array of shape (Lt, Lz, Ly, Lx, 4, 3, 3)
complex128, i.e. site-major with x fastest, direction mu = 0,1,2,3 = x,y,z,t,
then row, column.  Its C-order bytes are the host interchange (AoS) layout.

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, invariants, library routines or brute force.
"""
