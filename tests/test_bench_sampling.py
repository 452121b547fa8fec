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


def test_traffic_record_is_keyed_to_the_kernel_source(tmp_path, monkeypatch):
    # the committed record carries the source hash of the contraction kernel it was taken
    # on; the bench reports its bytes only while that hash matches the current source
    import re
    txt0 = open(os.path.join(ROOT, "profiles", "contraction_C3_split_f16.md")).read()
    keyed = re.search(r"kernel_source_sha:\s*([0-9a-f]+)", txt0).group(1) == bench.source_sha("split_f16")
    v = bench.traffic_from_profiles("C3", "split_f16")
    assert (v is not None) == keyed
    if v is not None:
        assert 1e8 < v < 1e11
    prof = tmp_path / "profiles"
    prof.mkdir()
    txt = open(os.path.join(ROOT, "profiles", "contraction_C3_split_f16.md")).read()
    (prof / "contraction_C3_split_f16.md").write_text(txt.replace(bench.source_sha("split_f16"), "0" * 16))
    src = tmp_path / "paper_2206_07660_gb300" / "csrc"
    src.mkdir(parents=True)
    (src / "k_umma.cu").write_bytes(open(os.path.join(ROOT, "paper_2206_07660_gb300", "csrc", "k_umma.cu"), "rb").read())
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_from_profiles("C3", "split_f16") is None
    assert bench.traffic_from_profiles("C9", "split_f16") is None
