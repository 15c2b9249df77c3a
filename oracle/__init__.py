"""FP64 CPU oracle for the FMM vortex-particle hot path.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports, links or runs
anything in this package; only the test-suite, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / reference arm of ``bench.py`` use it.  It shares no code
with the CUDA implementation: it has its own pair formula, its own Morton keys,
octree and dual-tree traversal, and its own expansion basis (Cartesian Taylor
expansions, where the CUDA path uses spherical harmonics).

Modules
  pairs      -- Eq. (1)-(3) pair terms S, T and a vectorised pair sum (numpy).
  direct     -- the same direct sum in plain C (direct.c), through ctypes.
  periodic   -- Fourier-space periodic sum, Taylor-Green closed form,
                brute-force cubic image sum and the dipole term.
  tree       -- Morton keys, stable sort, octree, radii, Algorithms 1-2.
  cartesian  -- Cartesian Taylor P2M, M2M, M2L, L2L, L2P.
  fmm        -- the plain FMM that strings them together (free or periodic).
"""
