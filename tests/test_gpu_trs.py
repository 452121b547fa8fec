"""Time-reversal symmetry (GW_TRS): the forward P~0, screened solve and Sigma~
run only on the irreducible q (k) of the mesh and fill the others by conjugation.
On a time-reversal-symmetric system (3x2x1 mesh: 4 irreducible points of 6) the
reduced context must match the unreduced one to rounding and the oracle to the
FP64 target; a system without the symmetry is rejected by gw_init."""
import numpy as np
import pytest

from gpu_helpers import gpu, oracle_state, system

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,tol_full,tol_oracle", [("fp64", 1e-12, 1e-10), ("split_f16", 1e-7, 1e-6)])
def test_trs_reduction_matches_full(precision, tol_full, tol_oracle):
    sysd = system(5, 20, (3, 2, 1), 24, 40.0, 71, trs=True)
    full = gpu(sysd, precision=precision, damping=0.5)
    red = gpu(sysd, precision=precision, damping=0.5, trs=True)
    full.iterate(2)
    red.iterate(2)
    st = oracle_state(sysd, damping=0.5)
    st.iterate()
    st.iterate()
    for q in ("G_tau", "Sigma_iw", "Sigma_inf", "P_tau", "Sigma_tau"):
        a, b = red.get(q), full.get(q)
        assert np.abs(a - b).max() <= tol_full * max(1.0, np.abs(b).max()), q
    for q in ("G_tau", "Sigma_iw", "Sigma_inf"):
        assert np.abs(red.get(q) - getattr(st, q)).max() < tol_oracle, q
    assert abs(red.get("mu") - st.mu) < (1e-8 if precision == "fp64" else 1e-6)


def test_trs_flag_rejects_asymmetric_system():
    from paper_2206_07660_gb300 import GWError
    sysd = system(4, 8, (3, 1, 1), 12, 20.0, 72, trs=False)
    with pytest.raises(GWError) as e:
        gpu(sysd, trs=True)
    assert e.value.status == 1 and "time-reversal" in str(e.value)
