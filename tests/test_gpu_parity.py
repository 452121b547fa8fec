"""GPU parity: the CUDA path through the C ABI against the CPU oracle, stage by
stage and for full iterations, on seeded inputs whose sizes span several
64-wide tiles and ragged tails.

Tolerances (fp64 path): the two sides evaluate the same discrete definition
with different summation orders, so they agree to roundoff amplified by the
conditioning of each step: ~1e-13 relative for the contractions, cond(TF) x
1e-15 for the transforms, and 1e-10 Ha absolute for Sigma and G after a full
iteration (the target accuracy for the fp64 path).
"""
import numpy as np
import pytest

from gpu_helpers import gpu, hermitian_noise, oracle_state, rel, system
from oracle import gw as ogw
from oracle.grids import Grid
from synth import make_config_system, matsubara_indices

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("ntau,beta", [(8, 20.0), (32, 100.0), (92, 1000.0), (100, 1000.0)])
def test_transform_matrices(ntau, beta):
    sysd = system(2, 3, (1, 1, 1), ntau, beta, 1)
    g = gpu(sysd)
    fn, bm = matsubara_indices(ntau)
    o = Grid(beta, ntau, fn, bm)
    assert rel(g.get("TFf"), o.TFf) < 1e-13
    assert rel(g.get("TFb"), o.TFb) < 1e-13
    assert rel(g.get("TBf"), o.TBf) < 1e-15 * np.linalg.cond(o.TFf) * 20
    assert rel(g.get("TBb"), o.TBb) < 1e-15 * np.linalg.cond(o.TFb) * 20
    assert np.abs(g.get("lb") - o.lb).max() < 1e-12 * np.abs(o.lb).max()
    assert np.abs(g.get("tau") - o.tau).max() < 1e-12 * beta


@pytest.mark.parametrize("nao,naux,kmesh,ntau,beta", [(3, 5, (1, 1, 1), 8, 10.0), (8, 32, (2, 2, 2), 32, 100.0),
                                                      (13, 20, (3, 1, 1), 24, 200.0)])
def test_dyson_noninteracting(nao, naux, kmesh, ntau, beta):
    sysd = system(nao, naux, kmesh, ntau, beta, 7)
    g = gpu(sysd)
    mu = g.dyson()
    st = oracle_state(sysd)
    st.dyson()
    assert abs(g.get("n_elec") - nao) <= 1e-9
    assert abs(mu - st.mu) < 1e-8
    assert np.abs(g.get("G_tau") - st.G_tau).max() < 1e-10
    # G(i w) ~ 1/w near the lowest frequency, so it carries the bisection's
    # last-digit freedom in mu amplified by |G|^2: compare it relatively
    assert rel(g.get("G_iw"), st.G_iw) < 1e-10


def _perturbed_green(sysd, seed):
    st = oracle_state(sysd)
    st.dyson()
    G = st.G_tau + hermitian_noise(st.G_tau.shape, 0.02, seed)
    return st, G


@pytest.mark.parametrize("nao,naux,kmesh,ntau", [(5, 70, (3, 1, 1), 12), (8, 32, (2, 2, 2), 32),
                                                 (17, 9, (1, 2, 1), 10), (1, 1, (1, 1, 1), 8)])
def test_polarization(nao, naux, kmesh, ntau):
    sysd = system(nao, naux, kmesh, ntau, 60.0, 11)
    st, G = _perturbed_green(sysd, 3)
    g = gpu(sysd)
    g.set("G_tau", G)
    g.polarization()
    P0 = ogw.polarization_tau(st.V, G, st.km)
    P0iw = ogw.to_matsubara(st.grid.TFb, P0, 1)
    assert rel(g.get("P0_tau"), P0) < 1e-13
    assert rel(g.get("P0_iw"), P0iw) < 1e-12


@pytest.mark.parametrize("naux,nq,ntau", [(130, 2, 6), (64, 3, 5), (7, 1, 9)])
def test_screened(naux, nq, ntau):
    # seeded P~0(i Omega) with a negative-definite Hermitian part (as the
    # polarization has), so that I - P~0 is well conditioned
    sysd = system(2, naux, (nq, 1, 1), ntau, 30.0, 5)
    rng = np.random.default_rng(9)
    A = (rng.standard_normal((nq, ntau, naux, naux)) + 1j * rng.standard_normal((nq, ntau, naux, naux))) / np.sqrt(naux)
    P0 = -0.5 * (A @ np.conj(np.swapaxes(A, -1, -2))) + 0.3 * (A - np.conj(np.swapaxes(A, -1, -2)))
    g = gpu(sysd)
    g.set("P0_iw", P0)
    g.screened()
    P = ogw.screened(P0)
    o = Grid(30.0, ntau, *matsubara_indices(ntau))
    Pt = ogw.herm(ogw.to_matsubara(o.TBb, P, 1))
    assert rel(g.get("P_iw"), P) < 1e-12
    assert rel(g.get("P_tau"), Pt) < 1e-12


@pytest.mark.parametrize("nao,naux,kmesh,ntau", [(5, 70, (3, 1, 1), 12), (8, 32, (2, 2, 2), 32),
                                                 (17, 9, (1, 2, 1), 10)])
def test_selfenergy(nao, naux, kmesh, ntau):
    sysd = system(nao, naux, kmesh, ntau, 60.0, 13)
    st, G = _perturbed_green(sysd, 4)
    nk = st.km.nk
    P = hermitian_noise((nk, ntau, naux, naux), 0.1, 8)
    g = gpu(sysd)
    g.set("G_tau", G)
    g.set("P_tau", P)
    g.selfenergy()
    S = ogw.selfenergy_tau(st.V, G, P, st.km)
    Siw = ogw.to_matsubara(st.grid.TFf, S, 0)
    gam = ogw.density_matrix(st.grid, G)
    Sinf = ogw.hartree(st.V, gam) + ogw.exchange(st.V, gam)
    assert rel(g.get("Sigma_tau"), S) < 1e-13
    assert rel(g.get("Sigma_iw"), Siw) < 1e-12
    assert rel(g.get("Sigma_inf_new"), Sinf) < 1e-13
    assert rel(g.get("gamma"), gam) < 1e-13


@pytest.mark.parametrize("trs", [False, True])
def test_full_iterations_c1(trs):
    sysd = make_config_system("C1", trs=trs)
    g = gpu(sysd, damping=0.5)
    st = oracle_state(sysd, damping=0.5)
    for it in range(2):
        stats = g.iterate(1)
        st.iterate()
        assert abs(stats["n_elec"] - st.n_elec) <= 1e-9
        assert np.abs(g.get("Sigma_inf") - st.Sigma_inf).max() < 1e-10
        assert np.abs(g.get("Sigma_iw") - st.Sigma_iw).max() < 1e-10
        assert np.abs(g.get("Sigma_tau") - st.Sigma_tau).max() < 1e-10
        assert np.abs(g.get("G_tau") - st.G_tau).max() < 1e-10
        assert abs(g.get("mu") - st.mu) < 1e-8


def test_single_orbital_closed_form():
    # nao = naux = nk = 1 with the exact G at the nodes: P~0 is the constant
    # -s v^2 f (1-f) and Sigma~ has a closed form (see oracle.closed_forms)
    from oracle import closed_forms as cf
    ntau, beta, eps, v, mu = 16, 10.0, 0.3, 0.7, 0.05
    fn, bm = matsubara_indices(ntau)
    sysd = dict(H0=np.full((1, 1, 1), eps, dtype=np.complex128), S=np.ones((1, 1, 1), dtype=np.complex128),
                V=np.full((1, 1, 1, 1, 1), v, dtype=np.complex128), kmesh=(1, 1, 1), ntau=ntau, beta=beta,
                fermi_n=fn, bose_m=bm, n_elec=1.0)
    o = Grid(beta, ntau, fn, bm)
    cl = cf.single_orbital(beta, eps, v, mu, o.tau)
    g = gpu(sysd)
    g.set("G_tau", cl["G"].reshape(ntau, 1, 1, 1).astype(np.complex128))
    g.polarization()
    assert np.abs(g.get("P0_tau") - cl["c"]).max() < 1e-14
    g.screened()
    tol = 50 * np.linalg.cond(o.TFb) * np.finfo(float).eps * (1 + abs(beta * cl["c"]))
    assert np.abs(g.get("P_tau") - cl["P_tau"]).max() < tol * abs(cl["P_tau"])
    g.selfenergy()
    assert np.abs(g.get("Sigma_tau")[:, 0, 0, 0] - cl["Sigma_tau"]).max() < tol * np.abs(cl["Sigma_tau"]).max()
    assert abs(g.get("Sigma_inf_new")[0, 0, 0] - (cl["J"] + cl["K"])) < 1e-13


def test_lowp_contractions_c1_fp32():
    # complex64 SIMT products against the fp64 oracle: errors stay at the 1e-5 Ha
    # level of plain fp32 arithmetic
    sysd = make_config_system("C1")
    g = gpu(sysd, precision="fp32")
    st = oracle_state(sysd)
    g.iterate(1)
    st.iterate()
    err = np.abs(g.get("Sigma_tau") - st.Sigma_tau).max()
    assert err < 1e-5, err
    assert np.abs(g.get("Sigma_inf") - st.Sigma_inf).max() < 1e-5


# Accuracy of the mixed path: the split products and the 16/22-bit intermediates are
# exact to ~2^-22 relative (a CPU emulation of their rounding at C1 moves Sigma~ by
# 4e-8 Ha), but the tensor pipe accumulates each MMA chunk in FP32 with truncation
# (measured at C1: 1.9 / 2.7 / 3.0e-6 Ha for drains every 1 / 2 / 4 stages), which
# leaves ~1.2e-6 of |Sigma~| in absolute terms.  Where |Sigma~| < ~0.8 Ha -- the C2
# and C3 workloads, where the C2 / C3 sampled tests check 1e-6 Ha -- that is within
# the 1e-6 Ha target; C1's interaction (|Sigma~| = 1.8 Ha) is 25x stronger, so its
# bound is 2e-6 of max |Sigma~| (3.7e-6 Ha).
MIXED_REL = 2e-6


@pytest.mark.parametrize("precision,small", [("split_tf32", "simt"), ("split_tf32", "tensor"), ("split_f16", "auto")])
def test_mixed_path_c1(precision, small):
    # the mixed path (split-TF32 or row-scaled split-fp16 tensor-core contractions, FP64
    # elsewhere) against the FP64 oracle over two damped iterations
    sysd = make_config_system("C1")
    g = gpu(sysd, precision=precision, small_steps=small, damping=0.5)
    st = oracle_state(sysd, damping=0.5)
    for it in range(2):
        g.iterate(1)
        st.iterate()
        scale = max(float(np.abs(st.Sigma_tau).max()), float(np.abs(st.Sigma_inf).max()))
        errs = {q: float(np.abs(g.get(q) - getattr(st, q)).max())
                for q in ("Sigma_inf", "Sigma_tau", "Sigma_iw", "G_tau")}
        assert max(errs.values()) < MIXED_REL * scale, (it, errs, scale)
        assert errs["Sigma_inf"] < 1e-6, errs      # HF: FP32 SIMT exchange, no tensor-pipe accumulation
        assert abs(g.get("mu") - st.mu) < 1e-6


def test_split_bf16_c1_error():
    # bf16 pieces carry 16 significant bits: the error against the FP64 oracle after one
    # iteration is bounded at the 1e-4 Ha level (and reported by the benchmark)
    sysd = make_config_system("C1")
    g = gpu(sysd, precision="split_bf16")
    st = oracle_state(sysd)
    g.iterate(1)
    st.iterate()
    err = max(float(np.abs(g.get("Sigma_tau") - st.Sigma_tau).max()),
              float(np.abs(g.get("Sigma_inf") - st.Sigma_inf).max()))
    assert err < 1e-4, err


def test_get_refuses_unwritten_quantities():
    # gw_get returns GW_ERR_STATE for buffers that nothing has written yet
    from paper_2206_07660_gb300 import GWError
    sysd = system(3, 5, (2, 1, 1), 8, 10.0, 2)
    g = gpu(sysd)
    for name in ("G_tau", "G_iw", "Sigma_tau", "P0_tau", "P0_iw", "P_iw", "P_tau", "gamma", "Sigma_inf_new", "mu"):
        with pytest.raises(GWError) as e:
            g.get(name)
        assert e.value.status == 7, name
    assert np.abs(g.get("Sigma_inf")).max() == 0.0      # zero self-energy from the start
    assert np.abs(g.get("Sigma_iw")).max() == 0.0
    g.get("TFf"); g.get("tau")
    g.dyson()
    g.get("G_tau"); g.get("G_iw"); g.get("mu")
    g.polarization()
    g.get("P0_tau"); g.get("P0_iw")
    with pytest.raises(GWError):
        g.get("P_iw")
    g.screened()
    g.get("P_iw"); g.get("P_tau")
    with pytest.raises(GWError):
        g.get("P0_iw")                                  # replaced by P~(i Omega)
    g.selfenergy()
    g.get("Sigma_tau"); g.get("gamma"); g.get("Sigma_inf_new")


def test_rejects_bad_inputs():
    from paper_2206_07660_gb300 import GWError
    sysd = system(3, 4, (2, 1, 1), 8, 10.0, 2)
    V = sysd["V"].copy()
    V[0, 1] += 0.1
    bad = dict(sysd, V=V)
    with pytest.raises(GWError):
        gpu(bad)
    H = sysd["H0"].copy()
    H[0, 0, 1] += 0.1
    with pytest.raises(GWError):
        gpu(dict(sysd, H0=H))
    g = gpu(sysd)
    with pytest.raises(GWError):
        g.polarization()     # no G yet


@pytest.mark.parametrize("precision,small", [("fp32", "auto"), ("split_tf32", "simt"), ("split_tf32", "tensor"),
                                             ("split_f16", "auto"), ("split_bf16", "auto")])
@pytest.mark.parametrize("nao,naux,kmesh,ntau", [(5, 70, (3, 1, 1), 12), (13, 20, (2, 1, 1), 10),
                                                 (64, 9, (1, 1, 1), 6), (65, 6, (1, 1, 1), 4)])
def test_lowp_stages(nao, naux, kmesh, ntau, precision, small):
    # ragged sizes (K = 2 nao^2 and 2 naux not multiples of the 32-wide tensor-core K
    # block; nao = 64 is the largest batched-small-product size, 65 takes the general kernel)
    sysd = system(nao, naux, kmesh, ntau, 60.0, 21)
    st, G = _perturbed_green(sysd, 6)
    nk = st.km.nk
    P = hermitian_noise((nk, ntau, naux, naux), 0.1, 9)
    g = gpu(sysd, precision=precision, small_steps=small)
    g.set("G_tau", G)
    g.polarization()
    tol = 3e-4 if precision == "split_bf16" else 2e-5
    P0 = ogw.polarization_tau(st.V, G, st.km)
    assert rel(g.get("P0_tau"), P0) < tol
    g.set("P_tau", P)
    g.selfenergy()
    S = ogw.selfenergy_tau(st.V, G, P, st.km)
    assert rel(g.get("Sigma_tau"), S) < tol


@pytest.mark.parametrize("precision", ["fp64", "split_tf32"])
def test_transforms_tensor_vs_native_fp64(precision):
    # the tau <-> i nu transforms as digit-split tensor-core products agree with the
    # FP64 SIMT kernel to FP64 roundoff over full iterations
    sysd = make_config_system("C1")
    a = gpu(sysd, precision=precision, fp64_gemm="tensor")
    b = gpu(sysd, precision=precision, fp64_gemm="native")
    a.iterate(2)
    b.iterate(2)
    for q in ("G_tau", "Sigma_iw", "P_tau"):
        x, y = a.get(q), b.get(q)
        assert np.abs(x - y).max() <= 1e-11 * max(1.0, np.abs(y).max()), q
