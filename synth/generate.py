"""Seeded synthetic inputs (numpy PCG64), shaped like the paper's workloads.

The paper's inputs are PySCF integrals of real solids (Sec. "scGW workflow");
none are available here, so seeded random tensors with the same structure
stand in for them:

* Gamma-centred n1 x n2 x n3 k-mesh, k = (i1 n2 + i2) n3 + i3.
* H0(k) = U diag(e) U^H with e ~ Uniform[-1, 1] Ha and U Haar-random.
* S(k) = I + 0.05 (A + A^H)/2, A_ij ~ CN(0, 1/nao), redrawn until
  lambda_min >= 0.5 (positive definite overlap, Eq. scalar_S).
* V^{kk'}_ij(Q) ~ CN(0, 1) c_V exp(-Q/8), c_V = 1/sqrt(nao), with the pairing
  V^{k'k}(Q) = V^{kk'}(Q)^H (so that U of Eq. U_decompose is Hermitian) and
  V^{kk}(Q) Hermitian.  naux/nao = 4..8 as in the paper's "3~10" range.
* Optional time-reversal variant: H0(-k) = conj H0(k), S(-k) = conj S(k),
  V^{-k,-k'} = conj V^{kk'}.

Sampled Matsubara integers.  The paper takes its sparse-sampling points from
the IR basis package; here the tau grid is Chebyshev and the ntau sampled
frequencies follow a fixed integer rule: the first positive indices are
consecutive and later ones follow kappa * h * tan(pi (i + 1/2) / (2 (h + 1)))
with kappa = 0.4, h = ceil(ntau/2).  Fermionic sets are symmetric
(n and -n-1); bosonic sets hold 0, pairs +-m and one extra positive m.  The
rule only depends on ntau (the transform matrices scale with beta alone).
"""
import numpy as np

SEED_BASE = 2206076600

# Workloads: sizes of the paper-scale synthetic systems.
CONFIGS = {
    "C1": dict(nao=8, naux=32, kmesh=(2, 2, 2), ntau=32, beta=100.0, cV_scale=1.0),
    "C2": dict(nao=26, naux=200, kmesh=(3, 3, 3), ntau=92, beta=1000.0, cV_scale=0.35),
    "C3": dict(nao=52, naux=400, kmesh=(4, 4, 4), ntau=100, beta=1000.0, cV_scale=0.35),
}
CONFIG_INDEX = {"C1": 1, "C2": 2, "C3": 3, "C4": 4, "C5": 5}


def config_seed(name, system=0):
    return SEED_BASE + 10 * CONFIG_INDEX[name] + system


def kmesh_size(kmesh):
    return int(kmesh[0]) * int(kmesh[1]) * int(kmesh[2])


def _positive_rule(h, kappa=0.4):
    i = np.arange(h)
    raw = np.floor(kappa * h * np.tan(np.pi * (i + 0.5) / (2 * (h + 1)))).astype(np.int64)
    out = np.empty(h, dtype=np.int64)
    prev = -1
    for t in range(h):
        v = max(int(raw[t]), prev + 1)
        out[t] = v
        prev = v
    return out


def matsubara_indices(ntau):
    """(fermi_n, bose_m): sorted int64 arrays of length ntau.

    Fermionic frequency (2n+1) pi / beta, bosonic 2 m pi / beta.
    """
    ntau = int(ntau)
    hf = (ntau + 1) // 2
    p = _positive_rule(hf)
    fermi = np.concatenate([p, -p[: ntau - hf] - 1])
    hb = ntau // 2
    pb = _positive_rule(hb) + 1 if hb > 0 else np.zeros(0, dtype=np.int64)
    bose = np.concatenate([[0], pb, -pb[: ntau - 1 - hb]])
    fermi = np.sort(fermi).astype(np.int64)
    bose = np.sort(bose).astype(np.int64)
    assert len(set(fermi.tolist())) == ntau and len(set(bose.tolist())) == ntau
    return fermi, bose


def _cn(rng, shape):
    """Complex normal CN(0, 1): E|z|^2 = 1."""
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2.0)


def _haar(rng, n, real=False):
    if real:
        z = rng.standard_normal((n, n))
    else:
        z = _cn(rng, (n, n))
    q, r = np.linalg.qr(z)
    d = np.diag(r)
    ph = d / np.abs(d)
    return q * ph[None, :]


def _kvec(nk3):
    n1, n2, n3 = nk3
    return np.array([(a, b, c) for a in range(n1) for b in range(n2) for c in range(n3)])


def _kidx(v, nk3):
    n1, n2, n3 = nk3
    return (int(v[0]) % n1 * n2 + int(v[1]) % n2) * n3 + int(v[2]) % n3


def make_system(nao, naux, kmesh, seed, trs=False, cV=None, s_pert=0.05, v_decay=8.0,
                materialize_V=True, **_):
    """Draw one synthetic system.  Returns a dict of complex128 arrays.

    H0, S: [nk, nao, nao];  V: [nk, nk, naux, nao, nao] with
    V[k, k2, Q, i, j] = V^{k k2}_{ij}(Q).  With materialize_V=False the
    tensor is not built; v_slab(sys, k, k2) draws any (k, k2) slab on demand
    (each unordered pair has its own seed, so slabs are reproducible).
    """
    nao, naux = int(nao), int(naux)
    kmesh = tuple(int(x) for x in kmesh)
    nk = kmesh_size(kmesh)
    rng = np.random.Generator(np.random.PCG64(int(seed)))
    if cV is None:
        cV = 1.0 / np.sqrt(nao)
    kv = _kvec(kmesh)
    minus = np.array([_kidx(-kv[k], kmesh) for k in range(nk)])

    H0 = np.zeros((nk, nao, nao), dtype=np.complex128)
    S = np.zeros((nk, nao, nao), dtype=np.complex128)
    done = np.zeros(nk, dtype=bool)
    for k in range(nk):
        if done[k]:
            continue
        self_conj = trs and minus[k] == k
        e = rng.uniform(-1.0, 1.0, nao)
        U = _haar(rng, nao, real=self_conj)
        H = (U * e[None, :]) @ U.conj().T
        H = 0.5 * (H + H.conj().T)
        while True:
            A = rng.standard_normal((nao, nao)) / np.sqrt(nao) if self_conj else \
                _cn(rng, (nao, nao)) / np.sqrt(nao)
            Sk = np.eye(nao) + s_pert * 0.5 * (A + A.conj().T)
            if np.linalg.eigvalsh(Sk).min() >= 0.5:
                break
        H0[k], S[k] = H, Sk
        done[k] = True
        if trs and not self_conj:
            H0[minus[k]] = H.conj()
            S[minus[k]] = Sk.conj()
            done[minus[k]] = True

    decay = cV * np.exp(-np.arange(naux) / v_decay)
    out = dict(H0=H0, S=S, nao=nao, naux=naux, kmesh=kmesh, nk=nk,
               seed=int(seed), trs=bool(trs), cV=float(cV), v_decay=float(v_decay))
    if trs:
        V = np.stack([np.stack([_v_raw(seed, k, k2, naux, nao, decay) for k2 in range(nk)])
                      for k in range(nk)])
        # group average over (k,k') -> (k',k) [^H] and (k,k') -> (-k,-k') [conj]
        Vh = np.conj(np.swapaxes(V, 3, 4))                    # V^{kk'}^H
        t1 = np.swapaxes(Vh, 0, 1)                            # (V^{k'k})^H at [k,k']
        t2 = np.conj(V[minus][:, minus])                      # conj V^{-k,-k'}
        t3 = np.swapaxes(np.swapaxes(V[minus][:, minus], 0, 1), 3, 4)  # (V^{-k',-k})^T
        out["V"] = 0.25 * (V + t1 + t2 + t3)
    elif materialize_V:
        V = np.empty((nk, nk, naux, nao, nao), dtype=np.complex128)
        for k in range(nk):
            for k2 in range(k, nk):
                V[k, k2] = v_slab(out, k, k2)
                if k2 != k:
                    V[k2, k] = np.conj(np.swapaxes(V[k, k2], 1, 2))
        out["V"] = V
    return out


def _v_raw(seed, k, k2, naux, nao, decay):
    rng = np.random.Generator(np.random.PCG64([int(seed), 7, int(k), int(k2)]))
    return _cn(rng, (naux, nao, nao)) * decay[:, None, None]


def v_slab(sysd, k, k2):
    """V^{k k2}(Q) as [naux, nao, nao], drawn from a per-pair seed.

    The unordered pair (min, max) owns the draw; the other order is its
    conjugate transpose, and the diagonal pair is made Hermitian.
    """
    if sysd.get("V") is not None:
        return sysd["V"][k, k2]
    naux, nao = sysd["naux"], sysd["nao"]
    decay = sysd["cV"] * np.exp(-np.arange(naux) / sysd["v_decay"])
    a, b = min(k, k2), max(k, k2)
    raw = _v_raw(sysd["seed"], a, b, naux, nao, decay)
    if a == b:
        return (raw + np.conj(np.swapaxes(raw, 1, 2))) / np.sqrt(2.0)
    return raw if k <= k2 else np.conj(np.swapaxes(raw, 1, 2))




def batch_configs(n_systems=16, nao_set=(8, 12, 16, 26, 40), mesh_set=(2, 3, 4), ntau=64, beta=100.0,
                  name="C4"):
    """Sizes of the uneven batch: per system nao from nao_set and an n x n x n
    mesh from mesh_set, drawn from the system's own seed; naux = 8 nao."""
    out = []
    for s in range(n_systems):
        rng = np.random.Generator(np.random.PCG64(config_seed(name, s) + 1))
        nao = int(rng.choice(nao_set))
        n = int(rng.choice(mesh_set))
        out.append(dict(nao=nao, naux=8 * nao, kmesh=(n, n, n), ntau=ntau, beta=beta, cV_scale=0.35,
                        seed=config_seed(name, s)))
    return out


def make_batch_system(cfg, materialize_V=True):
    cV = cfg.get("cV_scale", 1.0) / np.sqrt(cfg["nao"])
    sysd = make_system(cfg["nao"], cfg["naux"], cfg["kmesh"], cfg["seed"], materialize_V=materialize_V, cV=cV)
    fn, bm = matsubara_indices(cfg["ntau"])
    sysd.update(ntau=int(cfg["ntau"]), beta=float(cfg["beta"]), fermi_n=fn, bose_m=bm, n_elec=float(cfg["nao"]))
    return sysd


def make_config_system(name, system=0, trs=False, materialize_V=True, **over):
    """System plus grid integers for a named workload (sizes overridable)."""
    cfg = dict(CONFIGS[name])
    cfg.update(over)
    cV = cfg.get("cV_scale", 1.0) / np.sqrt(cfg["nao"])
    sysd = make_system(cfg["nao"], cfg["naux"], cfg["kmesh"], config_seed(name, system),
                       trs=trs, materialize_V=materialize_V, cV=cV)
    fn, bm = matsubara_indices(cfg["ntau"])
    sysd.update(ntau=int(cfg["ntau"]), beta=float(cfg["beta"]), fermi_n=fn, bose_m=bm,
                n_elec=float(cfg.get("n_elec", cfg["nao"])))
    return sysd


class LazyV:
    """V^{kk'}(Q) slabs drawn on demand, indexable as V[k, k'] (for oracle samples
    of workloads whose full V tensor does not fit in host memory)."""

    def __init__(self, sysd):
        self.sysd = sysd
        nk, naux, nao = sysd["nk"], sysd["naux"], sysd["nao"]
        self.shape = (nk, nk, naux, nao, nao)
        self.cache = {}

    def __getitem__(self, idx):
        k, k2 = idx
        if isinstance(k, np.ndarray):
            return np.stack([self[(int(a), int(b))] for a, b in zip(k, k2)])
        key = (int(k), int(k2))
        if key not in self.cache:
            self.cache[key] = v_slab(self.sysd, *key)
        return self.cache[key]


def device_V(sysd, threads=16):
    """The full V tensor [nk, nk, naux, nao, nao] complex128 in GPU memory, drawn
    slab by slab on host threads (each unordered pair once, its partner by
    conjugate transposition on the device)."""
    import concurrent.futures as cf
    import os
    import torch
    nk, naux, nao = sysd["nk"], sysd["naux"], sysd["nao"]
    V = torch.empty((nk, nk, naux, nao, nao), dtype=torch.complex128, device="cuda")
    pairs = [(k, k2) for k in range(nk) for k2 in range(k, nk)]

    def draw(p):
        return p, torch.from_numpy(v_slab(sysd, *p)).pin_memory()

    with cf.ThreadPoolExecutor(max_workers=min(threads, os.cpu_count() or 4)) as ex:
        for (k, k2), h in ex.map(draw, pairs):
            d = h.to("cuda", non_blocking=False)
            V[k, k2] = d
            if k2 != k:
                V[k2, k] = d.transpose(-1, -2).conj()
    torch.cuda.synchronize()
    return V

