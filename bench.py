#!/usr/bin/env python
"""Benchmark of one full self-consistent GW iteration on one GB300.

A step is one GW iteration (density matrix and HF, P~0, screened solve,
Sigma~, transforms, chemical-potential search and Dyson) over a seeded
synthetic system resident in HBM.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload C3] [--precision fp32]
  python bench.py --impl reference ...   # the CPU oracle on a bounded sample
  python bench.py --peaks                # fp64 / fp32 / tf32 matmul rates of this GPU
  python bench.py --gemm M N K B F64     # one tensor-core GEMM shape (profiling cases)
"""
import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GW iteration seconds and P/Sigma TFLOP/s, FP64 vs mixed, at stated Sigma error"
SM_COUNT = 152
SM_MAX_MHZ = 2070.0
# per-SM per-clock flop rates of the SIMT pipes used by the contraction kernel
FP32_FLOPS_PER_CLK_SM = 128 * 2       # 128 FP32 lanes x FMA
FP64_FLOPS_PER_CLK_SM = 2 * 2         # 2 FP64 FMA per SM per clock (1.26 TFLOP/s at 2.07 GHz)


def bf16_peak(sustained=True):
    """The measured dense bf16 rate: the seconds-long sustained figure for a kernel timed
    inside a long step (the contraction kernel, timed across a whole iteration), else the
    burst figure; the profiling recipe's fallbacks without the measurement file."""
    try:
        d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        if sustained and d.get("bf16_tflops_sustained"):
            return float(d["bf16_tflops_sustained"])
        return float(d["bf16_tflops"])
    except Exception:
        return 1700.0 if sustained else 1900.0


def tf32_peak():
    return bf16_peak() * 1.1 / 2.25


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gw", choices=["gw", "reference"])
    p.add_argument("--workload", default="C3", choices=["C1", "C2", "C3", "C4", "C5"])
    p.add_argument("--c5-vjp", action="store_true", help="C5: also time the FP64 adjoint chains")
    p.add_argument("--precision", default="split_f16",
                   choices=["split_f16", "split_bf16", "split_tf32", "fp32", "fp64"])
    p.add_argument("--fp64-gemm", default="tensor", choices=["tensor", "native"],
                   help="FP64 tau<->i nu transforms: digit-split tensor-core products or the FP64 SIMT kernel")
    p.add_argument("--small-steps", default="auto", choices=["auto", "tensor", "simt"],
                   help="placement of the nao-sized chain steps in the split_tf32 path")
    p.add_argument("--e2e-steps", type=int, default=1)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-slices", action="store_true", help="skip the oracle slices and the fp64-path timing")
    p.add_argument("--no-fp64", action="store_true", help="skip the fp64 path on the slices")
    p.add_argument("--no-phi", action="store_true", help="skip the grand-potential call after the timed loop")
    p.add_argument("--cpu-samples", type=int, default=3, help="single-pair oracle samples in the CPU baseline")
    p.add_argument("--peaks", action="store_true")
    p.add_argument("--gemm", nargs=5, type=int, action="append", metavar=("M", "N", "K", "B", "F64"),
                   help="time the tensor-core GEMM on this shape (--steps launches) and exit")
    p.add_argument("--gemm-bn", type=int, default=0)
    p.add_argument("--gemm-f16", action="store_true")
    p.add_argument("--kmesh", default=None, help="override the k-mesh, e.g. 2,2,2 (profiling cases)")
    return p.parse_args()


# ---------------------------------------------------------------- flop accounting

def flops(cfg):
    nao, naux, ntau = cfg["nao"], cfg["naux"], cfg["ntau"]
    nk = cfg["kmesh"][0] * cfg["kmesh"][1] * cfg["kmesh"][2]
    contr = 8.0 * nk * nk * ntau * (naux * naux * nao * nao + 2 * naux * nao ** 3)
    return dict(P0=contr, Sigma=contr, screened=8.0 * naux ** 3 * nk * ntau,
                transforms=16.0 * nk * naux * naux * ntau * ntau + 16.0 * nk * nao * nao * ntau * ntau,
                K=16.0 * nk * nk * naux * nao ** 3)


# ---------------------------------------------------------------- clocks

class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self):
        self.proc = None
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(int(os.environ.get("LOCAL_RANK", "0")))],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1])); mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- inputs

HOST_V_LIMIT = 8e9   # bytes; larger V tensors are drawn slab by slab straight into HBM


def max_over_ranks(value, device):
    """The job's time is its slowest rank's: max of a per-rank float over all ranks
    of the default process group (the value itself without one)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def make_inputs(workload, seed_offset=0, kmesh=None):
    from synth import CONFIGS, make_config_system
    cfg = dict(CONFIGS[workload])
    over = {}
    if kmesh:
        cfg["kmesh"] = over["kmesh"] = tuple(int(x) for x in kmesh.split(","))
    nk = cfg["kmesh"][0] * cfg["kmesh"][1] * cfg["kmesh"][2]
    vbytes = nk * nk * cfg["naux"] * cfg["nao"] ** 2 * 16
    sysd = make_config_system(workload, system=seed_offset, materialize_V=vbytes <= HOST_V_LIMIT, **over)
    return cfg, sysd


def oracle_V(sysd):
    from synth import LazyV
    return sysd["V"] if sysd.get("V") is not None else LazyV(sysd)


def source_sha(precision):
    """Hash of the contraction kernel's source (the counters are void once it changes)."""
    kern = "k_umma.cu" if precision.startswith("split") else "k_gett.cu"
    src = os.path.join(ROOT, "paper_2206_07660_gb300", "csrc", kern)
    return hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]


def traffic_from_profiles(workload, precision):
    """Per-launch DRAM bytes of the contraction kernel from the committed ncu
    summary, if it was taken on the current sources (else None)."""
    sha = source_sha(precision)
    path = os.path.join(ROOT, "profiles", "contraction_%s_%s.md" % (workload, precision))
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m1 = re.search(r"kernel_source_sha:\s*([0-9a-f]+)", txt)
    m2 = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    if not m1 or not m2 or m1.group(1) != sha:
        return None
    return float(m2.group(1))


# ---------------------------------------------------------------- CPU oracle sample

def pair_list(nk, n, offset=0):
    """n distinct (q, k) pairs spread over the mesh (offset rotates the choice)."""
    out, i = [], offset
    while len(out) < n:
        q, k = (7 * i + 3) % nk, (5 * i + 1) % nk
        if (q, k) not in out:
            out.append((q, k))
        i += 1
    return out


def cpu_state(sysd):
    """The oracle's state at the non-interacting G0: its own mu search and Dyson
    step, timed.  Returns (state, seconds)."""
    from oracle import gw as ogw
    t0 = time.perf_counter()
    st = ogw.State(dict(sysd, V=oracle_V(sysd)))
    st.dyson()
    return st, time.perf_counter() - t0


def tau_subset(ntau, half):
    """The first and last `half` tau indices: a set closed under tau_j -> tau_{ntau-1-j},
    so that G(-tau) = -G(beta - tau) of a point in it stays in it."""
    import numpy as np
    if 2 * half >= ntau:
        return np.arange(ntau)
    return np.r_[0:half, ntau - half:ntau]


def cpu_sample(cfg, sysd, state, n_pairs=1, offset=0, tau_half=4):
    """Time the oracle on a bounded slice of one iteration and extrapolate.

    The slice: A2 (P~0) and A6 (Sigma~) on n_pairs (q, k) pairs and 2 tau_half
    tau points (every tau point is an independent batch of the same products);
    the screened solve with its two transforms for one q; Hartree for one k and
    the exchange term for one (k, k') pair; one electron count N(mu) (a Dyson
    inversion at every (n, k) and a trace), the G(tau) transform and the Sigma~
    transform.  Seconds per iteration = each part x (total units / sampled
    units), with the mu search counted as the number of N(mu) evaluations the
    oracle's bisection made on the state it was given.
    """
    import numpy as np
    from oracle import gw as ogw
    V = oracle_V(sysd)
    st = state
    G, km, grid = st.G_tau, st.km, st.grid
    nk, ntau = km.nk, G.shape[0]
    ts = tau_subset(ntau, tau_half)
    Gs = np.ascontiguousarray(G[ts])
    pairs = pair_list(nk, n_pairs, offset)
    for q, k in pairs:                    # draw the V slabs the sample reads before the clock starts
        for a, b in ((k, km.add(k, q)), (k, km.sub(k, q))):
            V[a, b], V[b, a]
    V[0, 0], V[pairs[0][0], pairs[0][1]], V[pairs[0][1], pairs[0][0]]
    t_p = t_s = 0.0
    P = {}
    for q, k in pairs:
        t0 = time.perf_counter()
        P[q] = ogw.polarization_tau(V, Gs, km, qs=[q], ks=[k])[q]
        t_p += time.perf_counter() - t0
    for q, k in pairs:
        t0 = time.perf_counter()
        ogw.selfenergy_tau(V, Gs, {q: P[q]}, km, qs=[q], ks=[k])
        t_s += time.perf_counter() - t0
    # the screened solve of one q from a full-length P~0(tau) of that q
    q0 = pairs[0][0]
    P0q = np.zeros((ntau,) + P[q0].shape[1:], dtype=np.complex128)
    P0q[ts] = P[q0]
    t0 = time.perf_counter()
    Piw = ogw.to_matsubara(grid.TFb, P0q, 0)
    ogw.herm(ogw.to_matsubara(grid.TBb, ogw.screened(Piw), 0))
    t_w = time.perf_counter() - t0
    t0 = time.perf_counter()
    gam = ogw.density_matrix(grid, G)
    t_j = time.perf_counter() - t0
    t0 = time.perf_counter()
    ogw.hartree(V, gam[:1])                 # the k = 0 term of the k' sum and row
    t_j1 = time.perf_counter() - t0
    t0 = time.perf_counter()
    ogw.exchange(V, gam, kps=[pairs[0][1]], ks=[pairs[0][0]])
    t_k = time.perf_counter() - t0
    t0 = time.perf_counter()
    Giw = ogw.dyson_inverse(grid, st.H0, st.S, st.Sigma_inf, st.Sigma_iw, st.mu)
    ogw.electron_count(grid, st.S, Giw)
    t_n = time.perf_counter() - t0
    t0 = time.perf_counter()
    ogw.green_tau(grid, Giw)
    ogw.to_matsubara(grid.TFf, G, 0)      # the Sigma~ transform (an array of Sigma~'s shape)
    t_tr = time.perf_counter() - t0
    n_eval = st.mu_steps + 4              # bracket ends, first midpoint, bisection steps, final inversion
    npairs = len(pairs)
    t_pairs = (t_p + t_s) * (nk * nk) / npairs * (ntau / float(len(ts)))
    t_hf = t_j + t_j1 * nk + t_k * nk * nk
    t_rest = t_n * n_eval + t_tr
    per_iter = t_pairs + t_w * nk + t_hf + t_rest
    cores = len(os.sched_getaffinity(0))
    what = ("A2+A6 on %d of %d x %d (q, k) pairs and %d of %d tau points, A4 with its transforms on 1 of %d q, "
            "Hartree on 1 of %d k, exchange on 1 of %d x %d (k, k') pairs, one N(mu) evaluation (scaled by the %d "
            "inversions of the oracle's mu search and Dyson step), the G(tau) and Sigma~ transforms"
            % (npairs, nk, nk, len(ts), ntau, nk, nk, nk, nk, n_eval))
    return per_iter, dict(cores=cores, parts_s=dict(pairs=t_pairs, screened=t_w * nk, hf=t_hf, rest=t_rest),
                          sample="oracle (NumPy complex128): " + what + "; each part scaled by total/sampled units")


# ---------------------------------------------------------------- sampled slices against the oracle

def slice_inputs(sysd, state, q=None, k0=None, ks=None):
    """Inputs of the sampled parity slices (the same construction as the full-size
    tests): G nonzero at k0, k0+q, k0+2q only (two (k, k+q) pairs contribute to
    P~0^q), and a P~(tau) nonzero for one q only, of the workload's own magnitude."""
    import numpy as np
    from oracle import gw as ogw
    st, km = state, state.km
    nk = km.nk
    q = nk // 4 if q is None else q
    k0 = 5 % nk if k0 is None else k0
    ks = (9 % nk) if ks is None else ks
    kk = [k0, km.add(k0, q), km.add(km.add(k0, q), q)]
    Gs = np.zeros_like(st.G_tau)
    Gs[:, kk] = st.G_tau[:, kk]
    V = oracle_V(sysd)
    npair = 2 if len(set(kk)) == 3 else len(set(kk)) - 1 or 1
    P0 = ogw.polarization_tau(V, Gs, km, qs=[q], ks=kk[:2])[q]
    Pw = ogw.screened(ogw.to_matsubara(st.grid.TFb, P0 * (nk / float(npair)), 0))
    Pq = ogw.herm(ogw.to_matsubara(st.grid.TBb, Pw, 0))
    Sref = ogw.selfenergy_tau(V, st.G_tau, {q: Pq}, km, qs=[q], ks=[ks])[:, ks]
    gam = ogw.density_matrix(st.grid, st.G_tau)
    Sinf = ogw.hartree(V, gam)[ks] + ogw.exchange(V, gam, ks=[ks])[ks]
    return dict(q=q, ks=ks, Gs=Gs, P0=P0, Pq=Pq, Sref=Sref, Sinf_ref=Sinf)


def run_slices(g, sl, G0, torch):
    """Sampled outputs of context g on the slice inputs, with device times of the
    P~0 stage (one q, every k), the screened solve (one q) and the Sigma~ stage
    (one q, every k) and of the q-independent rest (HF, transform, Dyson)."""
    import numpy as np
    nq = g.nk

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3

    q = sl["q"]
    g.set_q_range(q, q + 1)
    g.set("G_tau", sl["Gs"])
    t_p = timed(g.polarization)
    out = torch.empty(g.shape_of("P0_tau"), dtype=torch.complex128, device="cuda")
    g.get("P0_tau", out=out)
    P0 = out[q].cpu().numpy()
    t_w = timed(g.screened)
    out.zero_()
    out[q] = torch.from_numpy(sl["Pq"]).cuda()
    g.set("P_tau", out)
    del out
    g.set("G_tau", G0)
    t_s = timed(g.selfenergy_partial)
    S = g.get("Sigma_tau")[:, sl["ks"]]
    t_rest = timed(lambda: (g.selfenergy_finish(), g.dyson()))
    Sinf = g.get("Sigma_inf_new")[sl["ks"]]
    g.set_q_range(0, nq)
    return dict(P0_err=float(np.abs(P0 - sl["P0"]).max()), Sigma_tilde_err=float(np.abs(S - sl["Sref"]).max()),
                Sigma_inf_err=float(np.abs(Sinf - sl["Sinf_ref"]).max()),
                s_per_iteration_extrapolated=(t_p + t_w + t_s) * nq + t_rest,
                stage_s=dict(P0_one_q=t_p, screened_one_q=t_w, Sigma_one_q=t_s, rest=t_rest))


# ---------------------------------------------------------------- peaks

def measure_peaks():
    import torch
    out = {"gpu": torch.cuda.get_device_name(0)}
    for name, dt, n, tf32 in [("fp64", torch.float64, 8192, False), ("fp32_simt", torch.float32, 8192, False),
                              ("tf32", torch.float32, 8192, True), ("bf16", torch.bfloat16, 8192, False)]:
        torch.backends.cuda.matmul.allow_tf32 = tf32
        a = torch.randn(n, n, device="cuda", dtype=dt)
        b = torch.randn(n, n, device="cuda", dtype=dt)
        for _ in range(2):
            a @ b
        torch.cuda.synchronize()
        best = 1e9
        for _ in range(5):
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record(); a @ b; e.record(); torch.cuda.synchronize()
            best = min(best, s.elapsed_time(e) / 1e3)
        out[name + "_tflops"] = 2.0 * n ** 3 / best / 1e12
    out["host_cores"] = len(os.sched_getaffinity(0))
    print(json.dumps(out))


def gemm_timing(args):
    """--gemm M N K B F64 [...]: device time of the split tensor-core GEMM on given
    shapes with pseudo-random operands (C[z] (M x N, real) += A[z] (M x K) B (N x K)^T,
    three products; fp64 accumulating output when F64 = 1).  --gemm-bn forces the N tile,
    --gemm-f16 takes fp16 pieces (kind::f16) instead of TF32 pieces."""
    import ctypes
    import torch
    from paper_2206_07660_gb300 import load
    torch.cuda.set_device(0)
    lib = load()
    fn = lib.gwdbg_umma_bench_f16 if args.gemm_f16 else lib.gwdbg_umma_bench
    fn.argtypes = [ctypes.c_int] * 6 + [ctypes.POINTER(ctypes.c_double)]
    fn.restype = ctypes.c_int
    lib.gwdbg_umma_force_bn.argtypes = [ctypes.c_int]
    lib.gwdbg_umma_force_bn.restype = ctypes.c_int
    blk = 64 if args.gemm_f16 else 32
    old = lib.gwdbg_umma_force_bn(args.gemm_bn)
    rc = 0
    try:
        for (m, n, k, b, f) in args.gemm:
            ms = ctypes.c_double()
            kpad = (k + blk - 1) // blk * blk
            st = fn(m, n, kpad, b, f, args.steps, ctypes.byref(ms))
            tf = 6.0 * m * n * kpad * b / (ms.value * 1e-3) / 1e12 if st == 0 and ms.value > 0 else 0.0
            print(json.dumps({"gemm": [m, n, kpad, b, f], "bn": args.gemm_bn or "auto",
                              "pieces": "f16" if args.gemm_f16 else "tf32", "status": st, "ms": ms.value,
                              "tensor_tflops": tf}), flush=True)
            rc = rc or st
    finally:
        lib.gwdbg_umma_force_bn(old)
    return rc


# ---------------------------------------------------------------- reference arm

def run_reference(args):
    """The oracle (fp64 NumPy on the host cores) on the same workload: every step
    times a bounded sample (one (q, k) pair of both contractions on a tau subset,
    one q of the screened solve, one k of Hartree, one (k, k') pair of the
    exchange, one N(mu) evaluation and the transforms) and extrapolates it to one
    iteration.  The oracle's G0 (its own mu search and Dyson step) is computed
    once before the steps; its time is reported beside the sampled estimate of
    the same q-independent rest."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cfg, sysd = make_inputs(args.workload, kmesh=args.kmesh)
    st, t_dyson = cpu_state(sysd)
    vals, walls, rests = [], [], []
    info = None
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        v, info = cpu_sample(cfg, sysd, st, 1, offset=i)
        if i >= args.warmup:
            vals.append(v)
            walls.append(time.perf_counter() - t0)
            rests.append(info["parts_s"]["rest"])
    value = statistics.median(vals)
    ms_step = statistics.median(walls) * 1e3
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "s/iteration",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
            "data": "synthetic", "config": workload_config(cfg, args.workload, args.precision),
            "reference_note": "the CPU oracle (fp64 NumPy) on a bounded sample of the same workload per step; "
                              "value = the sample's time extrapolated to one full iteration (median over steps), "
                              "ms_per_step = the wall time of one sampled step",
            "mu_search_and_dyson_s": {"full_once": t_dyson, "sampled_median": statistics.median(rests),
                                      "mu_evaluations": st.mu_steps + 3},
            "cpu_baseline": {"value": value, "unit": "s/iteration", "cores": info["cores"], "kind": "oracle",
                             "sample": info["sample"]},
            "e2e": {"value": value, "unit": "s/iteration", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def workload_config(cfg, name, precision):
    nk = cfg["kmesh"][0] * cfg["kmesh"][1] * cfg["kmesh"][2]
    return {"workload": "%s: nao=%d naux=%d k-mesh %dx%dx%d (nk=%d) ntau=nw=%d beta=%g, %s contractions, "
                        "fp64 screened solve/transforms/Dyson/mu" % (name, cfg["nao"], cfg["naux"], *cfg["kmesh"], nk,
                                                                     cfg["ntau"], cfg["beta"], precision),
            "nao": cfg["nao"], "naux": cfg["naux"], "nk": nk, "ntau": cfg["ntau"], "beta": cfg["beta"],
            "contract_precision": precision, "l2": "inputs larger than L2 (V is %.2f GB)" %
            (nk * nk * cfg["naux"] * cfg["nao"] ** 2 * 16 / 1e9), "parallelism": "single GPU"}


# ---------------------------------------------------------------- GPU arm

def make_context(sysd, Vd, precision, args, **kw):
    import torch
    from paper_2206_07660_gb300 import GW
    if Vd is not None:
        return GW(torch.from_numpy(sysd["H0"]).cuda(), torch.from_numpy(sysd["S"]).cuda(), Vd, sysd["kmesh"],
                  sysd["ntau"], sysd["beta"], sysd["fermi_n"], sysd["bose_m"], n_elec=sysd["n_elec"], damping=0.5,
                  precision=precision, borrow_V=True, small_steps=args.small_steps, fp64_gemm=args.fp64_gemm, **kw)
    return GW(sysd["H0"], sysd["S"], sysd["V"], sysd["kmesh"], sysd["ntau"], sysd["beta"], sysd["fermi_n"],
              sysd["bose_m"], n_elec=sysd["n_elec"], damping=0.5, precision=precision,
              small_steps=args.small_steps, fp64_gemm=args.fp64_gemm, **kw)


def run_gw(args):
    import numpy as np
    import torch
    import torch.distributed as dist
    from oracle import gw as ogw   # sampled parity slices and the CPU baseline only
    from paper_2206_07660_gb300.shard import attach, sharded_iteration
    from synth import device_V

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    # one system; with N > 1 ranks every rank owns a block of q-points (strong scaling)
    cfg, sysd = make_inputs(args.workload, kmesh=args.kmesh)
    # the oracle's state (the error slices below use it too) and the CPU baseline, timed
    # first, in a process that has not touched the GPU yet (as the reference arm does)
    st = None
    cpu_line = None
    if rank == 0 and world == 1 and not (args.no_slices and args.no_cpu_baseline):
        st, _ = cpu_state(sysd)
    if st is not None and not args.no_cpu_baseline:
        # the reference arm's per-step sample (one (q, k) pair), median over a few pairs
        vs = []
        for i in range(args.cpu_samples):
            v, info = cpu_sample(cfg, sysd, st, 1, offset=i)
            vs.append(v)
        cpu_line = {"value": statistics.median(vs), "unit": "s/iteration", "cores": info["cores"], "kind": "oracle",
                    "sample": "median over %d samples of: %s" % (len(vs), info["sample"])}

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")

    def barrier():
        if world > 1:
            dist.barrier()

    fl = flops(cfg)
    Vd = device_V(sysd) if sysd.get("V") is None else None
    g = make_context(sysd, Vd, args.precision, args)
    if world > 1:
        attach(g, rank, world)
    g.dyson()
    G0 = g.get("G_tau")
    mu0 = g.get("mu")

    def step():
        if world > 1:
            sharded_iteration(g)
            return None
        return g.iterate(1)

    for _ in range(args.warmup):
        step()
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    clocks = Clocks()
    clocks.start()
    l0 = g.kernel_launches()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    stage = {"ms_polarization": 0.0, "ms_screened": 0.0, "ms_selfenergy": 0.0, "ms_dyson": 0.0}
    last = None
    for _ in range(args.steps):
        last = step()
        if last is not None:
            for kk in stage:
                stage[kk] += last[kk]
    ev1.record(stream)
    torch.cuda.synchronize()
    launches = g.kernel_launches() - l0
    barrier()
    clk = clocks.stop()
    ms = max_over_ranks(ev0.elapsed_time(ev1), "cuda")
    s_per_iter = ms / args.steps / 1e3
    K = args.steps
    norms = {"Sigma_inf_max_abs": float(np.abs(g.get("Sigma_inf")).max()),
             "Sigma_tilde_tau_max_abs": float(np.abs(g.get("Sigma_tau")).max())}

    # one more iteration with per-launch CUDA events around every contraction GEMM (on
    # the launching stream): the roofline of the dominant kernel, kept out of the timed loop
    g.profile(True)
    step()
    torch.cuda.synchronize()
    prof = g.profile_read()
    g.profile(False)
    dominant = "tensor" if args.precision.startswith("split") else "simt"
    gemm_ms, gemm_flops, gemm_launches = prof[dominant]
    p_tflops = s_tflops = None
    if last is not None and stage["ms_polarization"] > 0:
        p_tflops = fl["P0"] / (stage["ms_polarization"] / K / 1e3) / 1e12
        s_tflops = fl["Sigma"] / (stage["ms_selfenergy"] / K / 1e3) / 1e12

    # the grand potential Phi~ (Eq. tilde_Phi_GW) of the last iteration's P~0, outside the timed loop
    phi = None
    if not args.no_phi:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        v = g.grand_potential()
        phi = {"Phi_tilde_Ha": v, "s": time.perf_counter() - t0,
               "note": "one gw_grand_potential call after the timed loop (FP64 transform and LU trace-log "
                       "of I - P~0 at every (q, Omega) of this rank's q block)"}

    # end to end through the public API: each step's input G(tau) from pinned host memory,
    # one iteration, G(tau) and Sigma(i w) read back (H0, S, V stay resident from gw_init)
    e2e_t = []
    hG = torch.from_numpy(G0).pin_memory()
    outG = torch.empty_like(hG).pin_memory()
    outS = torch.empty(g.shape_of("Sigma_iw"), dtype=torch.complex128).pin_memory()
    g.reset_sigma()
    for _ in range(args.e2e_steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g.set("G_tau", hG)
        g.set("mu", mu0)
        step()
        g.get("G_tau", out=outG)
        g.get("Sigma_iw", out=outS)
        e2e_t.append(time.perf_counter() - t0)
    e2e = None
    if e2e_t:
        e2e_v = max_over_ranks(statistics.median(e2e_t), "cuda")
        e2e = {"value": e2e_v, "unit": "s/iteration", "h2d_bytes_per_step": hG.numel() * 16,
               "d2h_bytes_per_step": (outG.numel() + outS.numel()) * 16,
               "copies": "G(tau) host->device before, G(tau) and Sigma(i w) device->host after each iteration"}

    # sampled slices against the oracle (rank 0, single GPU): the mixed path's errors in Ha, and the
    # FP64 path's errors and its seconds per iteration extrapolated from one q
    extra = {}
    if rank == 0 and world == 1 and not args.no_slices:
        sl = slice_inputs(sysd, st)
        r_mixed = run_slices(g, sl, st.G_tau, torch)
        g.close()
        g = None
        r64 = None
        if not args.no_fp64:
            g64 = make_context(sysd, Vd, "fp64", args)
            g64.dyson()
            r64 = run_slices(g64, sl, st.G_tau, torch)
            g64.close()
        scale = {"Sigma_tilde_ref_max_abs": float(np.abs(sl["Sref"]).max()),
                 "Sigma_inf_ref_max_abs": float(np.abs(sl["Sinf_ref"]).max()),
                 "P0_ref_max_abs": float(np.abs(sl["P0"]).max())}
        slice_desc = ("vs the fp64 oracle on sampled slices of this workload: P~0^q(tau) of q=%d from a G(tau) "
                      "nonzero at three k (two (k, k+q) pairs), Sigma~^k(tau) of k=%d from the oracle's G0 and a "
                      "P~(tau) nonzero for q=%d only, Sigma_inf^k of k=%d from G0" % (sl["q"], sl["ks"], sl["q"],
                                                                                       sl["ks"]))
        extra = {"sigma_err_Ha": {"Sigma_inf": r_mixed["Sigma_inf_err"], "Sigma_tilde_tau": r_mixed["Sigma_tilde_err"],
                                  "P0_tau": r_mixed["P0_err"], "against": slice_desc, "reference_magnitudes": scale,
                                  "iteration_magnitudes": norms, "target_Ha": 1e-6},
                 "mixed_slice_s_per_iteration_extrapolated": r_mixed["s_per_iteration_extrapolated"]}
        if r64 is not None:
            extra.update({
                 "fp64_path": {"s_per_iteration": r64["s_per_iteration_extrapolated"],
                               "extrapolated": "from one q of the P~0, screened and Sigma~ stages (x nq) plus the "
                                               "q-independent HF, transform and Dyson step, timed on the sampled "
                                               "slices",
                               "stage_s": r64["stage_s"],
                               "P_tflops": fl["P0"] / g_nk(cfg) / r64["stage_s"]["P0_one_q"] / 1e12,
                               "Sigma_tflops": fl["Sigma"] / g_nk(cfg) / r64["stage_s"]["Sigma_one_q"] / 1e12,
                               "sigma_err_Ha": {"Sigma_inf": r64["Sigma_inf_err"],
                                                "Sigma_tilde_tau": r64["Sigma_tilde_err"], "P0_tau": r64["P0_err"],
                                                "target_Ha": 1e-10}},
                 "mixed_speedup_over_fp64": r64["s_per_iteration_extrapolated"] / s_per_iter})

    achieved = gemm_flops / (gemm_ms / 1e3) / 1e12 if gemm_ms > 0 else 0.0
    traffic = traffic_from_profiles(args.workload, args.precision)
    if args.precision == "split_tf32":
        peak = tf32_peak()
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": "umma_pkernel (tcgen05 kind::tf32, split hi/lo, 3 products)",
                "split_products": 3, "tensor_pipe_frac": 3.0 * achieved / peak,
                "peak_basis": "of measured: bf16 dense %.1f TFLOP/s sustained (MEASURED_PEAKS.json; the kernel is "
                              "timed across a whole iteration) x nominal tf32/bf16 ratio 1.1/2.25" % bf16_peak(),
                "frac_of_burst_peak": achieved / (bf16_peak(False) * 1.1 / 2.25)}
    elif args.precision in ("split_f16", "split_bf16"):
        peak = bf16_peak()
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": traffic,
                "kernel": "umma_pkernel (tcgen05 kind::f16, %s hi/lo pieces, 3 products)" % args.precision[6:],
                "split_products": 3, "tensor_pipe_frac": 3.0 * achieved / peak,
                "peak_basis": "of measured: bf16 dense %.1f TFLOP/s sustained (MEASURED_PEAKS.json; the kernel is "
                              "timed across a whole iteration; fp16 has the same nominal rate)" % bf16_peak(),
                "frac_of_burst_peak": achieved / bf16_peak(False)}
    else:
        peak = (SM_COUNT * (FP32_FLOPS_PER_CLK_SM if args.precision == "fp32" else FP64_FLOPS_PER_CLK_SM)
                * SM_MAX_MHZ * 1e6 / 1e12)
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": "gett_kernel<%s> (complex contraction, SIMT FMA)" % args.precision,
                "peak_basis": "152 SMs x %d flop/clk x 2070 MHz (unit counts and max SM clock)" %
                              (FP32_FLOPS_PER_CLK_SM if args.precision == "fp32" else FP64_FLOPS_PER_CLK_SM)}
    roof.update({"launches": gemm_launches, "algorithmic_flops_per_launch": gemm_flops / max(1, gemm_launches),
                 "avg_launch_ms": gemm_ms / max(1, gemm_launches),
                 "measured_in": "one profiled iteration after the timed loop (CUDA events around every launch "
                                "of the kernel, on its stream)",
                 "flops_definition": "useful complex-contraction flops, 8 per complex multiply-add",
                 "other_kernel": {k: {"ms": v[0], "tflops": v[1] / max(1e-9, v[0] / 1e3) / 1e12, "launches": v[2]}
                                  for k, v in prof.items() if k != dominant}})
    conf = workload_config(cfg, args.workload, args.precision)
    if world > 1:
        conf["parallelism"] = "q-sharded over %d GPUs (contiguous q blocks, one all-reduce of Sigma~(tau))" % world
    line = {"metric": METRIC, "value": s_per_iter, "unit": "s/iteration", "n_gpus": world, "steps": K,
            "warmup": args.warmup, "ms_per_step": ms / K, "higher_is_better": False,
            "scaling": "strong" if world > 1 else "weak",
            "vs_baseline": None, "dtype": {"fp32": "c64", "fp64": "c128", "split_tf32": "tf32x3/c64", "split_f16": "f16x3/c64",
                                  "split_bf16": "bf16x3/c64"}[args.precision],
            "data": "synthetic", "config": conf,
            "P_tflops": p_tflops, "Sigma_tflops": s_tflops,
            "stage_ms_per_iteration": {k: v / K for k, v in stage.items()},
            "gpu_launches": launches, "clocks": clk, "roofline": roof, "e2e": e2e}
    line.update(extra)
    if phi is not None:
        line["grand_potential"] = phi
    if g is not None:
        g.close()
    if cpu_line is not None:
        line["cpu_baseline"] = cpu_line
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def g_nk(cfg):
    return cfg["kmesh"][0] * cfg["kmesh"][1] * cfg["kmesh"][2]


def run_batch(args):
    """C4: 16 seeded systems of uneven sizes, iterated together from captured graphs."""
    import numpy as np
    import torch
    from paper_2206_07660_gb300 import GW
    from paper_2206_07660_gb300.gw import batch_iterate
    from synth import batch_configs, device_V, make_batch_system
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    prec = args.precision
    cfgs = batch_configs()
    systems, gws = [], []
    for cfg in cfgs:
        nk = cfg["kmesh"][0] ** 3
        big = nk * nk * cfg["naux"] * cfg["nao"] ** 2 * 16 > HOST_V_LIMIT
        sysd = make_batch_system(cfg, materialize_V=not big)
        if big:
            Vd = device_V(sysd)
            g = GW(torch.from_numpy(sysd["H0"]).cuda(), torch.from_numpy(sysd["S"]).cuda(), Vd, sysd["kmesh"],
                   sysd["ntau"], sysd["beta"], sysd["fermi_n"], sysd["bose_m"], n_elec=sysd["n_elec"], damping=0.5,
                   precision=prec, borrow_V=True)
            g._keep = Vd
        else:
            g = GW(sysd["H0"], sysd["S"], sysd["V"], sysd["kmesh"], sysd["ntau"], sysd["beta"], sysd["fermi_n"],
                   sysd["bose_m"], n_elec=sysd["n_elec"], damping=0.5, precision=prec)
        systems.append(sysd)
        gws.append(g)
    flop = sum(flops(dict(c))["P0"] * 2 for c in cfgs)
    batch_iterate(gws, args.warmup)
    torch.cuda.synchronize()
    clocks = Clocks()
    clocks.start()
    l0 = gws[0].kernel_launches()
    t0 = time.perf_counter()
    batch_iterate(gws, args.steps)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / args.steps
    launches = gws[0].kernel_launches() - l0
    clk = clocks.stop()
    # the same systems one after another, plain (uncaptured) iterations
    t0 = time.perf_counter()
    for g in gws:
        g.iterate(1)
    torch.cuda.synchronize()
    seq = time.perf_counter() - t0
    line = {"metric": METRIC, "value": dt, "unit": "s/batch-iteration (16 systems)", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32": "c64", "fp64": "c128", "split_tf32": "tf32x3/c64", "split_f16": "f16x3/c64",
                                  "split_bf16": "bf16x3/c64"}[prec],
            "data": "synthetic",
            "config": {"workload": "C4: 16 systems, nao in {8,12,16,26,40}, naux = 8 nao, k-meshes 2^3..4^3, "
                                   "ntau = nw = 64, beta = 100, %s contractions, captured graphs on per-system "
                                   "streams" % prec,
                       "systems": [{"nao": c["nao"], "nk": c["kmesh"][0] ** 3} for c in cfgs],
                       "l2": "inputs larger than L2", "parallelism": "single GPU"},
            "contraction_tflops": flop / dt / 1e12, "sequential_plain_s": seq, "batch_speedup": seq / dt,
            "gpu_launches": launches, "clocks": clk}
    if not args.no_cpu_baseline:
        tot, parts = 0.0, []
        for cfg, sysd in zip(cfgs, systems):
            v, info = cpu_sample(cfg, sysd, cpu_state(sysd)[0], 1)
            tot += v
        line["cpu_baseline"] = {"value": tot, "unit": "s/batch-iteration (16 systems)", "cores": info["cores"],
                                "kind": "oracle", "sample": "per system: " + info["sample"] + "; summed"}
    for g in gws:
        g.close()
    print(json.dumps(line))


def run_differentiation(args):
    """C5 (C2 sizes): the tangent of the whole self-consistency map and Newton-Krylov
    self-consistency built on it, against damped iterations from the same start."""
    import numpy as np
    import torch
    from paper_2206_07660_gb300 import GW
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    cfg, sysd = make_inputs("C2", kmesh=args.kmesh)
    prec = args.precision

    def ctx(damping):
        return GW(sysd["H0"], sysd["S"], sysd["V"], sysd["kmesh"], sysd["ntau"], sysd["beta"], sysd["fermi_n"],
                  sysd["bose_m"], n_elec=sysd["n_elec"], damping=damping, precision=prec, mu_tol=1e-10)

    def ev():
        return torch.cuda.Event(enable_timing=True)

    # damped reference: residual ||F(x) - x|| per iteration (one extra unmixed map per step)
    g = ctx(1.0)
    g.iterate(2)
    start_i, start_w = g.get("Sigma_inf"), g.get("Sigma_iw")
    # tangent timing at the start point
    g.polarization()
    g.screened()
    vi = torch.randn(*g.shape_of("Sigma_inf"), dtype=torch.complex128, device="cuda")
    vw = torch.randn(*g.shape_of("Sigma_iw"), dtype=torch.complex128, device="cuda")
    for _ in range(max(1, args.warmup)):
        g.sc_jvp(vi, vw)
    torch.cuda.synchronize()
    e0, e1 = ev(), ev()
    e0.record()
    for _ in range(args.steps):
        g.sc_jvp(vi, vw)
    e1.record()
    torch.cuda.synchronize()
    jvp_s = e0.elapsed_time(e1) / 1e3 / args.steps
    e0, e1 = ev(), ev()
    e0.record()
    g.iterate(1)
    e1.record()
    torch.cuda.synchronize()
    fwd_s = e0.elapsed_time(e1) / 1e3
    g.close()
    # Newton-Krylov from the start point
    n_outer, m = 4, 6
    gn = ctx(1.0)
    gn.set("Sigma_inf", start_i)
    gn.set("Sigma_iw", start_w)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res_nk = gn.iterate_newton(n_outer, m=m, tol=1e-10)
    torch.cuda.synchronize()
    nk_s = time.perf_counter() - t0
    gn.close()
    # damped iterations (mixing 0.5) from the same start, for the same wall time
    gd = ctx(0.5)
    gd.set("Sigma_inf", start_i)
    gd.set("Sigma_iw", start_w)
    res_d, t0 = [], time.perf_counter()
    while time.perf_counter() - t0 < nk_s and len(res_d) < 200:
        st = gd.iterate(1)
        res_d.append(float(st["max_dSigma"]))
    torch.cuda.synchronize()
    gd.close()
    line = {"metric": METRIC, "value": nk_s / n_outer, "unit": "s/Newton-Krylov step (GMRES(%d), %s)" % (m, prec),
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": nk_s / n_outer * 1e3,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32": "c64", "fp64": "c128", "split_tf32": "tf32x3/c64", "split_f16": "f16x3/c64",
                                  "split_bf16": "bf16x3/c64"}[prec], "data": "synthetic",
            "config": dict(workload_config(cfg, "C5", prec),
                           workload="C5: C2 sizes, tangent of the self-consistency map and Newton-Krylov "
                                    "self-consistency (GMRES(%d)) vs damped (0.5) iterations" % m),
            "sc_jvp_s": jvp_s, "forward_iteration_s": fwd_s,
            "newton_residual_l2": res_nk, "newton_wall_s": nk_s,
            "damped_max_dSigma_same_wall_time": res_d[-3:], "damped_iterations_same_wall_time": len(res_d)}
    if args.c5_vjp:
        import numpy as np
        g = GW(sysd["H0"], sysd["S"], sysd["V"], sysd["kmesh"], sysd["ntau"], sysd["beta"], sysd["fermi_n"],
               sysd["bose_m"], n_elec=sysd["n_elec"], precision=prec)
        g.iterate(1)
        Pbar = torch.randn(*g.shape_of("P_tau"), dtype=torch.complex128, device="cuda")
        Sbar = torch.randn(*g.shape_of("Sigma_tau"), dtype=torch.complex128, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g.polarization_vjp(Pbar)
        g.selfenergy_vjp(Sbar)
        torch.cuda.synchronize()
        line["fp64_vjp_pair_s"] = time.perf_counter() - t0
        g.close()
    print(json.dumps(line))


def main():
    args = parse()
    if args.peaks:
        return measure_peaks()
    if args.gemm:
        return gemm_timing(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "C4":
        return run_batch(args)
    if args.workload == "C5":
        return run_differentiation(args)
    return run_gw(args)


if __name__ == "__main__":
    main()
