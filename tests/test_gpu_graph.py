"""Captured-graph iterations and the multi-system batch against plain
iterations of the same systems (same kernels, so agreement is to roundoff of
the mu bisection: G and Sigma to 1e-10).  The grids resolve the systems'
spectra (ntau >= 24 at beta <= 50): on coarser grids the sampled electron
count N(mu) is not monotone far from the spectrum and the bracket search
started from the previous mu may not find a root."""
import numpy as np
import pytest

from gpu_helpers import gpu, oracle_state, system

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "split_tf32"])
def test_graph_iterations_match_plain(precision):
    sysd = system(6, 24, (2, 2, 1), 32, 50.0, 41)
    a = gpu(sysd, precision=precision, damping=0.5)
    b = gpu(sysd, precision=precision, damping=0.5)
    a.iterate(3)
    st = b.iterate_graph(3)
    assert abs(st["n_elec"] - 6.0) <= 1e-9
    for q in ("G_tau", "Sigma_iw", "Sigma_inf"):
        assert np.abs(a.get(q) - b.get(q)).max() < 1e-10, q
    assert abs(a.get("mu") - b.get("mu")) < 1e-8
    # replaying the same graph again keeps matching
    a.iterate(1)
    b.iterate_graph(1)
    assert np.abs(a.get("G_tau") - b.get("G_tau")).max() < 1e-10


def test_batch_of_uneven_systems():
    from paper_2206_07660_gb300.gw import batch_iterate
    shapes = [(4, 16, (2, 1, 1), 32), (8, 32, (2, 2, 1), 32), (3, 24, (3, 1, 1), 24)]
    plain, batched = [], []
    for i, (nao, naux, km, nt) in enumerate(shapes):
        sysd = system(nao, naux, km, nt, 40.0, 50 + i)
        p = gpu(sysd, precision="split_tf32", damping=0.5)
        p.iterate(2)
        plain.append(p)
        batched.append(gpu(sysd, precision="split_tf32", damping=0.5))
    batch_iterate(batched, 2)
    for p, b in zip(plain, batched):
        assert np.abs(p.get("G_tau") - b.get("G_tau")).max() < 1e-10
        assert np.abs(p.get("Sigma_iw") - b.get("Sigma_iw")).max() < 1e-10


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("split_f16", 1e-6), ("split_tf32", 1e-6)])
def test_batch_of_uneven_systems_against_oracle(precision, tol):
    # four systems of different orbital counts, auxiliary sizes, k-meshes and grids iterated
    # together (captured graphs on per-system streams), each compared with the oracle's
    # own damped iterations of that system: the FP64 path to 1e-10 Ha, the mixed paths to 1e-6 Ha
    from paper_2206_07660_gb300.gw import batch_iterate
    shapes = [(4, 16, (2, 1, 1), 32, 40.0), (8, 32, (2, 2, 1), 32, 40.0), (3, 24, (3, 1, 1), 24, 30.0),
              (6, 40, (2, 2, 2), 32, 50.0)]
    systems, ctxs = [], []
    for i, (nao, naux, km, nt, beta) in enumerate(shapes):
        sysd = system(nao, naux, km, nt, beta, 60 + i)
        systems.append(sysd)
        ctxs.append(gpu(sysd, precision=precision, damping=0.5))
    batch_iterate(ctxs, 3)
    for i, (sysd, g) in enumerate(zip(systems, ctxs)):
        st = oracle_state(sysd, damping=0.5)
        for _ in range(3):
            st.iterate()
        for q in ("G_tau", "Sigma_iw", "Sigma_inf"):
            err = float(np.abs(g.get(q) - getattr(st, q)).max())
            assert err < tol, (i, q, err)
        assert abs(g.get("mu") - st.mu) < max(tol, 1e-8), i
