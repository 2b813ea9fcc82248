"""FP64 CPU oracle for the BOUNCE velocity-jump integrator (arXiv 2002.07109).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously correct
restatement of what the method computes, used to check the CUDA library.
Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its
``cpu_baseline`` leg and ``--impl reference`` arm) may import it.  The product
path (the C-ABI library and its Python binding) never imports, links or calls
anything here, and this package shares no code, tables or constants
generators with the CUDA path.

Modules
-------
philox        Philox4x32-10 counter-based generator (Salmon et al., SC'11).
forcefield    Pair potential W (Coulomb or Ewald-erfc, plus Lennard-Jones),
              switching function chi, short/long gradient split (Sec. IV.A),
              bonded terms, energies.
bounds        L_ab = sup |chi W'_ab| by a dense grid plus refinement (Sec. IV.A).
neighbors     Brute-force candidate rows (exact FP64 set, ascending index) and
              an independent cell-list construction used only to pin it.
poisson       Poisson counts by chunked FP32 inversion, with the FP32 exp(-x)
              this project defines (range reduction plus Taylor series).
integrate     BAOAB and BJAOAJB (BOUNCE) steps, the jump half-step J of
              Sec. IV.B, the O step, and the RESPA outer kick (Sec. V).
ewald         Plain Ewald sum (direct erfc + reciprocal k-sum + self term) for
              periodic boxes; the smooth particle-mesh (SPME) reciprocal part.
observables   Energies, O-O distance histograms, mean-square displacement.

Parity status of every function is given in its docstring; a function whose
result is pinned by nothing but itself says "parity unpinned".
"""
