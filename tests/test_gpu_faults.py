"""Failure paths on the GPU that fault nothing: bad inputs rejected by gw_init's
checks, a chemical potential that cannot be bracketed, and checkpoint files that
are missing, truncated, corrupt or of another size; plus a bit-identical resume."""
import os

import numpy as np
import pytest

from gpu_helpers import gpu, system
from synth import make_config_system

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("which", ["V", "H0", "S"])
def test_non_finite_input_is_rejected(which):
    from paper_2206_07660_gb300 import GWError
    sysd = system(3, 4, (2, 1, 1), 8, 10.0, 2)
    x = sysd[which].copy()
    x.flat[5] = np.nan
    with pytest.raises(GWError) as e:
        gpu(dict(sysd, **{which: x}))
    assert e.value.status == 1 and ("non-finite value in " + which) in str(e.value)


def test_unreachable_electron_count_is_not_converged():
    from paper_2206_07660_gb300 import GWError
    sysd = system(3, 4, (2, 1, 1), 8, 10.0, 2)
    g = gpu(dict(sysd, n_elec=2 * 3 + 1.0), mu_maxit=40)     # more electrons than spin-orbitals
    with pytest.raises(GWError) as e:
        g.dyson()
    assert e.value.status == 4
    g.close()
    g = gpu(sysd)          # the device and the library stay usable
    g.dyson()


def test_checkpoint_resume_is_bit_identical(tmp_path):
    sysd = make_config_system("C1")
    a = gpu(sysd, damping=0.5)
    a.iterate(1)
    path = str(tmp_path / "state.gw")
    a.save_state(path)
    a.iterate(1)
    b = gpu(sysd, damping=0.5)
    b.load_state(path)
    b.iterate(1)
    for q in ("G_tau", "Sigma_iw", "Sigma_inf"):
        assert np.array_equal(a.get(q), b.get(q)), q
    assert a.get("mu") == b.get("mu")


def test_checkpoint_rejects_bad_files(tmp_path):
    from paper_2206_07660_gb300 import GWError
    sysd = make_config_system("C1")
    a = gpu(sysd)
    a.iterate(1)
    path = str(tmp_path / "s.gw")
    a.save_state(path)
    raw = open(path, "rb").read()
    b = gpu(sysd)
    for name, data in (("truncated", raw[:-100]), ("corrupt", raw[:500] + bytes([raw[500] ^ 1]) + raw[501:]),
                       ("extra", raw + b"x")):
        p = str(tmp_path / name)
        open(p, "wb").write(data)
        with pytest.raises(GWError) as e:
            b.load_state(p)
        assert e.value.status == 1, name
    with pytest.raises(GWError):
        b.load_state(str(tmp_path / "missing.gw"))
    other = gpu(system(4, 8, (2, 1, 1), 16, 100.0, 3))
    with pytest.raises(GWError) as e:
        other.load_state(path)
    assert "sizes" in str(e.value)
    b.load_state(path)          # the good file still loads after the failures
    assert np.array_equal(b.get("G_tau"), a.get("G_tau"))
