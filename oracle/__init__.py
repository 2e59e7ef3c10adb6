"""Plain FP64 CPU oracle for CCD in pure neutron matter (arXiv:1611.06765).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` are the only callers.  The oracle shares no code with the CUDA
library and does not import it.

Parts:
  ``channel``  ctypes front end of ``pnm_oracle.c``: basis, Minnesota V, HF energies,
               E_ref, MBPT2 and the channel/intermediate CCD engine.
  ``dense``    Eq. (ccd) / Eq. (ccd3) evaluated term by term on dense 4-index arrays.
  ``pairing``  the four-particle, eight-state pairing model of Sec. "Developing a
               numerical project" (a small test case for the dense engine).
  ``exact2``   exact diagonalisation of two neutrons in the P = 0, S_z = 0 block.
  ``pw``       an independent numpy restatement of the plane-wave basis and the
               antisymmetrized Minnesota elements (for the dense engine).
"""
