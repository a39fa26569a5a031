"""FP64 CPU oracle for the S-ADI scheme (arXiv 2312.06206).

This package is TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
it.  The CUDA library never calls it and shares no code, table or constant
generator with it.

Contents
--------
weights  -- the 1D Riesz weights a_i (closed form, Sec. 2 eq. "single coefficient
            discrete Riesz"), the 2D fractional-Laplacian weights a_ij (Sec. 2,
            eq. "center discretization"; trapezoid + Richardson, with a
            Bessel-integral cross check).
sadi     -- the discrete operators L_h, delta_x, delta_y (Sec. 2), the ADI factor
            H (Sec. 3), the S-ADI step in the factored increment form (Sec. 3,
            eq. "ADI scheme equivalent") and the literal three-level form
            (Sec. 2, eqs. "ADI scheme" and "ADI scheme initial"), the
            Gohberg-Semencul solve (Proposition 1, Algorithm 1), the discrete
            energy of the stability theorem (Sec. 4) and the Error_1/Error_2
            estimators of Sec. 6.
diffusion -- S-ADI for the fractional Laplacian diffusion equation, the further
            application the conclusion (Sec. 7) names without a scheme: the
            splitting of Secs. 2-3 with Crank-Nicolson on the Riesz parts, the
            remainder and g extrapolated to t_{n+1/2}, and the factorisation
            term on the second difference (the reading is in its docstring).

Every function is plain FP64 numpy/scipy and cites the passage it follows.
Parity status of each function is listed in its docstring; every function
used by the parity tests is pinned by a ``-m "not gpu"`` test against values
fixed by the paper or by mathematics (closed forms, brute force, limits).
"""
