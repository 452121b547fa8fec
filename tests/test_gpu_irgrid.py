"""GW iterations on an IR sparse-sampling grid (gw_init_grid) against the oracle.

The paper represents functions of tau and i w on the IR basis and samples them at
the basis' own points (Sec. "Representation on the imaginary axes").  The oracle
builds that basis from its own singular value expansion (oracle.ir, pinned in
test_oracle_ir*.py); the CUDA library takes the resulting grid from the caller:
ntau tau points, nwf fermionic and nwb bosonic Matsubara points (rectangular
transforms, nwf != ntau or nwb != ntau here).  Damped iterations on the small
configuration's system must match the oracle's on the same grid: FP64 to 1e-10 Ha,
the mixed path to 2e-6 of |Sigma~| (its FP32-accumulation bound)."""
import numpy as np
import pytest

from gpu_helpers import gpu
from oracle import gw as ogw
from oracle.ir import IRGrid
from synth import make_config_system

pytestmark = pytest.mark.gpu


def _ctx(sysd, grid, **kw):
    import torch
    from paper_2206_07660_gb300 import GW
    torch.cuda.set_device(0)
    ntau = len(grid["tau"]) if isinstance(grid, dict) else grid.ntau
    return GW(sysd["H0"], sysd["S"], sysd["V"], sysd["kmesh"], ntau, sysd["beta"], n_elec=sysd["n_elec"],
              grid=grid, **kw)


@pytest.mark.parametrize("lam", [600.0, 2000.0])
@pytest.mark.parametrize("precision", ["fp64", "split_f16"])
def test_iterations_on_ir_grid(lam, precision):
    sysd = make_config_system("C1")
    grid = IRGrid(sysd["beta"], lam, 1e-10)
    assert (grid.ntau, len(grid.fermi_n), len(grid.bose_m)) != (grid.ntau,) * 3   # rectangular
    g = _ctx(sysd, grid, precision=precision, damping=0.5)
    assert g.get("TFf").shape == (len(grid.fermi_n), grid.ntau)
    assert np.abs(g.get("TBb") - grid.TBb).max() == 0.0
    st = ogw.State(sysd, damping=0.5, grid=grid)
    for it in range(2):
        g.iterate(1)
        st.iterate()
        scale = max(1.0, float(np.abs(st.Sigma_tau).max()))
        tol = 1e-10 if precision == "fp64" else 2e-6 * scale
        for q in ("G_tau", "Sigma_iw", "Sigma_inf", "Sigma_tau"):
            err = float(np.abs(g.get(q) - getattr(st, q)).max())
            assert err < tol, (it, q, err)
        assert abs(g.get("mu") - st.mu) < (1e-8 if precision == "fp64" else 1e-6)
    assert g.get("G_iw").shape[0] == len(grid.fermi_n)
    assert g.get("P_iw").shape[1] == len(grid.bose_m)


def test_grid_validation():
    from paper_2206_07660_gb300 import GWError
    sysd = make_config_system("C1")
    grid = IRGrid(sysd["beta"], 600.0, 1e-10)
    bad = {k: getattr(grid, k) for k in ("tau", "fermi_n", "bose_m", "TFf", "TBf", "TFb", "TBb", "lb")}
    bad["fermi_n"] = np.concatenate([grid.fermi_n[:-1], grid.fermi_n[:1]])   # a repeated index
    with pytest.raises(GWError):
        _ctx(sysd, bad)
