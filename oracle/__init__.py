"""FP64 CPU oracle for the FC-based spectral ISPH hot path.

TEST INFRASTRUCTURE ONLY.  This package is the slow, plain, obviously-correct
reference that the CUDA path is checked against.  Only the test-suite, the
smoke check and the CPU-baseline leg of the benchmark may import or run it;
the library itself never does, and the oracle imports nothing from the
library.  Everything here is float64 numpy, written step by step in the order
and notation of the paper (Lin, Fourtakas & Rogers, "A high-order Fourier
Continuation (FC)-based spectral ISPH scheme ..."):

  kernels  -- high-order Gaussian kernels, Appendix A moment recipe, Sec. 3.3
  dft      -- naive O(N^2) DFT / DCT-I matrices (Eqs. 11, 31, 32)
  fc       -- Fourier continuation tables: the paper's polynomial fit +
              extrapolation + blending (Sec. 4, Eqs. 14-29) and an FC(Gram)
              construction (Sec. 4.5 names it; built here from its
              mathematical definition); extension of lines/planes (Eq. 30)
  symbols  -- Fourier symbols of the sampled, minimum-image kernel
              derivatives (Eq. 13, Fig. 1)
  ops      -- spectral SPH operators on the FC-extended grid (Eqs. 11, 13)
  ppe      -- spectral PPE on the physical nodes (Eqs. 31-33)
  step     -- FOP / low-storage RK3 projection step (Eqs. 5-9, Sec. 2.2)
  advection -- Gaussian vortex convection with inflow/outflow (Sec. 6.2)
  channel3d -- the same operators, PPE and step in three dimensions (x, z
              periodic, walls in y)
  norms    -- L2 norm of Eq. 34 and companions

Pins: every function here is pinned by a ``-m "not gpu"`` test against
closed forms, printed values, invariants or brute force (tests/test_oracle_*).
Parity unpinned: the FC(Gram) table construction itself (the paper gives no
construction; its table is pinned only through the properties it must have:
exact reproduction of low-degree polynomials and smoothness of the extension).
"""
