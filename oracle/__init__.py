"""FP64 CPU oracle of the particle-mesh lensing forward model, its adjoint and
its tangent-linear model.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may use it.  It shares no code with the CUDA path; the only common
module is ``pm_inputs`` (seeded inputs, no arithmetic of the method).

Every step is written plainly in float64 with numpy/scipy primitives (FFT,
quadrature, ODE integration, interpolation), following the paper's method:

* Eq. (conv) and the lensing kernel q(chi) -- Born convergence (``lightcone``)
* Sec. 3 (package design) -- FastPM kick/drift stepping, box replication with
  rotation, the sub-evolution projection, PGD sharpening (``nbody``,
  ``lightcone``, ``mesh``)
* Appendix A -- comoving distance integral, Eisenstein-Hu linear power,
  finite-difference cosmology derivatives (``cosmology``, ``adjoint``)
* Sec. 3 / Fig. 8 -- the forward-mode derivative along a noise direction
  (``jvp``), pinned to the reverse sweep by the dot-product identity
* Sec. 4 (Fig. accuracy) -- shot-noise runs with uniformly random particles and
  the flat-sky angular power spectrum of the maps (``shotnoise``)

Readings of points the paper leaves open are stated in each function's
docstring.  The Eisenstein-Hu transfer function is pinned through its CDM part
(the Omega_b -> 0 limit against EH98's separately published zero-baryon fit, 1.5%)
and its averaged baryon suppression (the no-wiggle fit, 2%) and sound horizon;
the sigma_8 normalisation through the top-hat window's series and exact values
and the closed-form variance of power laws.  Parity unpinned: the amplitude of
the baryon wiggles (the constants of alpha_b, beta_node, beta_b and k_silk),
which no independent formula in reach fixes.
"""
