"""FP64 CPU oracle for spherical-cap GGX VNDF sampling (test infrastructure).

Plain, slow, obviously-correct numpy restatements of what the CUDA library
computes, each function citing the section or equation of Dupuy & Benyoub,
"Sampling Visible GGX Normals with Spherical Caps" (HPG 2023) it follows.
Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import anything here; the library itself never does, and the
two share no code.  Modules:

* ``philox``      Philox4x32-10 (Salmon et al., SC'11) and the u-mapping
* ``vndf``        the sampler (cap and prior), NDF, G1 and the VNDF pdf
* ``microfacet``  G2, Fresnel, BRDF, reflection pdf, albedo estimator and quadrature
* ``grad``        complex-step and finite-difference derivatives of (wm, pdf)
* ``brute``       ray casting against the truncated ellipsoid (definition of the VNDF)
"""
