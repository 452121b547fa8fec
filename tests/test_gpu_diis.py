"""Device DIIS self-consistency (gw_iterate_diis) against the oracle's DIIS.

Both sides iterate the same fixed-point map x -> F(x), x = (Sigma_inf, Sigma~(i w)),
F = Dyson with the mu search, then the GW self-energy of the new G, from x = 0,
keeping the last m steps and continuing from the affine combination of least
residual.  On the small configuration the FP64 paths agree step by step (residual
norms and the final self-energy); the residual falls where damped mixing stalls."""
import numpy as np
import pytest

from gpu_helpers import gpu, oracle_state
from oracle.diis import DIIS
from synth import make_config_system

pytestmark = pytest.mark.gpu


def test_diis_matches_oracle_c1():
    sysd = make_config_system("C1")
    n, m, mix = 6, 4, 0.5
    g = gpu(sysd)
    res = g.iterate_diis(n, m=m, mix=mix)
    st = oracle_state(sysd)
    d = DIIS(m=m, mix=mix)
    ores = []
    for _ in range(n):
        st.dyson()
        Sinf, _, Siw = st.sigma()
        (xi, xw), rn = d.push([st.Sigma_inf, st.Sigma_iw], [Sinf, Siw])
        ores.append(rn)
        st.Sigma_inf, st.Sigma_iw = xi, xw
    st.dyson()
    np.testing.assert_allclose(res, ores, rtol=1e-8)
    assert np.abs(g.get("Sigma_inf") - st.Sigma_inf).max() < 1e-9
    assert np.abs(g.get("Sigma_iw") - st.Sigma_iw).max() < 1e-9
    assert np.abs(g.get("G_tau") - st.G_tau).max() < 1e-9
