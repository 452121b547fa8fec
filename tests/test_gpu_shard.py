"""q-sharding through the C ABI on one GPU: two contexts own disjoint q blocks
(gw_set_q_range), their partial Sigma~(tau) are summed on the host and written
back (gw_selfenergy_partial / gw_set / gw_selfenergy_finish), as the ranks of
a multi-GPU run would after their all-reduce.  The contexts run one after the
other (no kernel of one waits on the other).  The summed result must equal the
unsharded context and the oracle."""
import numpy as np
import pytest

from gpu_helpers import gpu, oracle_state
from synth import make_config_system

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "split_tf32"])
def test_two_q_blocks_sum_to_full_iteration(precision):
    from paper_2206_07660_gb300.shard import attach
    sysd = make_config_system("C1")
    full = gpu(sysd, precision=precision)
    full.iterate(1)
    parts = [gpu(sysd, precision=precision) for _ in range(2)]
    for r, g in enumerate(parts):
        attach(g, r, 2)
        g.dyson()
        g.polarization()
        g.screened()
        g.selfenergy_partial()
    partial = [g.get("Sigma_tau") for g in parts]
    S = partial[0] + partial[1]
    for g in parts:
        g.set("Sigma_tau", S)
        g.selfenergy_finish()
        g.dyson()
    st = oracle_state(sysd)
    st.iterate()
    # mixed path: 2e-6 of |Sigma~| (FP32 accumulation in the tensor pipe; see test_gpu_parity)
    tol = 1e-10 if precision == "fp64" else 2e-6 * max(1.0, float(np.abs(st.Sigma_tau).max()))
    for g in parts:
        for q in ("G_tau", "Sigma_iw", "Sigma_inf"):
            assert np.abs(g.get(q) - full.get(q)).max() < (1e-12 if precision == "fp64" else 1e-7), q
        assert np.abs(g.get("G_tau") - st.G_tau).max() < tol
        assert np.abs(g.get("Sigma_iw") - st.Sigma_iw).max() < tol
        assert abs(g.get("mu") - st.mu) < (1e-8 if precision == "fp64" else 1e-5)
    # a partial Sigma~(tau) alone is not the full one (both blocks contribute)
    assert np.abs(S - partial[0]).max() > 1e-3 * np.abs(S).max()


def test_q_range_rejects_bad_blocks():
    from paper_2206_07660_gb300 import GWError
    sysd = make_config_system("C1")
    g = gpu(sysd)
    for q0, q1 in ((-1, 2), (3, 3), (0, 9), (5, 2)):
        with pytest.raises(GWError):
            g.set_q_range(q0, q1)
