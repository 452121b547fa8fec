"""The CPU baseline's bounded sample (bench.py): the tau subset it times is closed
under tau -> beta - tau, the oracle's contractions on that subset give exactly
the full results' rows at those tau (so timing a subset and scaling by
ntau / |subset| counts the same work), and a sample at C1 returns a finite
extrapolation whose parts add up."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from oracle import gw as ogw  # noqa: E402


@pytest.mark.parametrize("ntau,half", [(100, 4), (32, 4), (7, 2), (6, 3), (5, 4)])
def test_tau_subset_closed_under_reflection(ntau, half):
    ts = bench.tau_subset(ntau, half)
    assert len(set(ts.tolist())) == len(ts) == min(ntau, 2 * half)
    assert set((ntau - 1 - ts).tolist()) == set(ts.tolist())
    assert np.all(np.diff(ts) > 0)


@pytest.fixture(scope="module")
def c1():
    cfg, sysd = bench.make_inputs("C1")
    st, t = bench.cpu_state(sysd)
    assert t > 0
    return cfg, sysd, st


def test_contractions_on_tau_subset_are_rows_of_full(c1):
    _, sysd, st = c1
    V, G, km = sysd["V"], st.G_tau, st.km
    ts = bench.tau_subset(G.shape[0], 4)
    q, k = 3, 5
    full = ogw.polarization_tau(V, G, km, qs=[q], ks=[k])[q]
    sub = ogw.polarization_tau(V, np.ascontiguousarray(G[ts]), km, qs=[q], ks=[k])[q]
    assert np.abs(sub - full[ts]).max() <= 1e-14 * np.abs(full).max()
    Sf = ogw.selfenergy_tau(V, G, {q: full}, km, qs=[q], ks=[k])
    Ss = ogw.selfenergy_tau(V, np.ascontiguousarray(G[ts]), {q: full[ts]}, km, qs=[q], ks=[k])
    assert np.abs(Ss - Sf[ts]).max() <= 1e-14 * np.abs(Sf).max()


def test_sample_at_c1(c1):
    cfg, sysd, st = c1
    v, info = bench.cpu_sample(cfg, sysd, st, 2, offset=1)
    parts = info["parts_s"]
    assert np.isfinite(v) and v > 0
    assert abs(v - sum(parts.values())) <= 1e-9 * v
    assert info["cores"] >= 1 and "8 of 32 tau points" in info["sample"]
