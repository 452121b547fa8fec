"""CPU oracle for density-fitted self-consistent GW (test infrastructure).

A plain, slow, fp64/complex128 NumPy restatement of the method, used only by
the test suite, the smoke check and the benchmark's CPU-baseline leg.  It
shares no code with the CUDA library and never imports it.  Modules:

* grids         -- Chebyshev tau nodes, tau <-> Matsubara transforms (Eqs. tau_to_iw, iw_to_tau)
* gw            -- one scGW iteration step by step (Eqs. HF_J, HF_K, tilde_P0_tau,
                   P0t_to_P0w, tilde_P_omega, Piw_to_Pt, tilde_sigma2, Dyson)
* brute         -- four-index (non-density-fitted) route (Eqs. U_decompose, W, P0_tau, tilde_sigma)
* closed_forms  -- non-interacting G0 and P~0, single-orbital model
"""
