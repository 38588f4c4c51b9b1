"""FP64 CPU oracle for least-misfit gridding and degridding (Ye, Gull, Tan & Nikolic 2019).

TEST INFRASTRUCTURE ONLY. Nothing in the product imports this package: only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference`` legs of
``bench.py`` may call it. It shares no code, table, constant generator or helper with the
CUDA library under ``paper_1906_07102_gb300/``.

Modules
-------
``design``   the least-misfit function: quadrature nodes, the per-offset linear systems
             (normal equations with Cholesky, or least squares with QR), the map error
             l(x) and the integrated misfit E, the Levenberg-Marquardt optimisation of the
             correcting function h, the look-up table and the grid-correction factors
             (Section 2.1, Appendices A, B, E, F).
``imaging``  the support rule, table lookup, gridding, FFT dirty image with correction and
             crop, its adjoint (pad, correct, FFT, degrid), the brute-force DFT references
             and the Cauchy-Schwarz misfit bound (Section 2.1 Eqs. 3-9, Section 4).

Everything is plain numpy/scipy in float64, written step by step in the paper's order.
Library primitives used as single steps: ``scipy.optimize.leastsq`` (MINPACK
Levenberg-Marquardt, the routine the paper names in Appendix A), ``scipy.linalg`` Cholesky
and triangular solves, ``numpy.linalg.qr`` (Householder QR, Appendix B) and ``numpy.fft``.

Parity status: C(u), h(x) and E are pinned by closed forms in two limits (tests/prolate.py,
tests/small_field.py): at support W = 1 the design is exactly the prolate spheroidal
eigenproblem (E_min = 1 - lambda_0(pi x0) / (2 x0), h and C proportional to S_00), and for
W = 1..5 on a small field the optimum has a moment-matching closed form (rational even
moments, E proportional to (2 pi x0)^(2W)); the oracle approaches both at second order
(W = 5 through the least-squares route of Appendix B, which keeps the digits there). At
the working x0 (0.25) the paper prints no values (its figures are lost), so for W >= 2 the
exact values of C(u) and h(x) there are **parity unpinned**: the same code is pinned in
those limits (for W <= 5), and the values themselves only indirectly, by stationarity, by
the paper's ordering and bound claims and by route agreement (see tests/test_oracle_*.py).
"""
