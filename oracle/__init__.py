"""FP64 CPU oracle for the improved W-stacking gridder/degridder.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may call it.  It shares no code,
tables or constants with the CUDA library under ``paper_2101_11172_gb300/``.

Modules (each function cites the passage of Ye, Gull, Tan & Nikolic 2021,
"High accuracy wide field imaging method in radio interferometry", that it
follows):

* :mod:`oracle.lmfit`    -- least-misfit gridding function C and correction h
  (Section 3.3, Eq. csum2, Eq. norm_bound), the error bound E and the map error
  l(x); the top-hat case of Section 6 (W_z = 1, h = 1/sinc).
* :mod:`oracle.geometry` -- normalised coordinates and plan sizes
  (Section 5.1, Eq. z-on-sphere, Eq. n_params, Eq. N_{w'}+W, Eq. N_w).
* :mod:`oracle.wstack`   -- Algorithms 1, 2 (1-D), 3, 4 (original W-stacking)
  and 5, 6 (3-D improved W-stacking) written step by step in FP64 with
  numpy's FFT.
* :mod:`oracle.explore`  -- the curves of Figures 3, 5 and 7 (E against W and
  x0), the top-hat error and the layer counts.
* :mod:`oracle.dft`      -- the exact operator (Eq. fourier_visibility and its
  adjoint) by brute force, in plain C with a numpy fallback.

Parity status: the individual values of C(u') and h(x) are *parity unpinned*
(the paper prints them only as a figure).  They are pinned indirectly through
the error bound E (Section 6: E = 1.3e-7 for W = 7, x0 = 0.25; the layer
multipliers quoted for Figure 3) and through the brute-force DFT.
"""
