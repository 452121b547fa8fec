"""The q-sharded split of one GW problem (paper_2206_07660_gb300.shard) on CPU.

Two gloo ranks (127.0.0.1) each own a contiguous block of q-points; every rank
computes its share of P~0, the screened solve and Sigma~ and the partial
Sigma~(tau) are summed with one all-reduce.  The contexts here are stand-ins
that evaluate each stage with the oracle (so the test needs no GPU and checks
the host logic: the partition, the reduction and the replicated rest); the
result must equal one unsharded oracle iteration.
"""
import os
import socket

import numpy as np
import pytest

from oracle import gw as ogw
from oracle import thermo
from paper_2206_07660_gb300.shard import q_block, sharded_grand_potential, sharded_iteration
from gpu_helpers import system


class OracleContext:
    """Stand-in with the binding's method names; every stage is the oracle's."""

    def __init__(self, sysd):
        self.st = ogw.State(sysd)
        self.st.dyson()
        self.nk = self.st.km.nk
        self.q0, self.q1 = 0, self.nk
        self.Stau = None

    def shape_of(self, name):
        return self.st.G_tau.shape

    def set_q_range(self, q0, q1):
        self.q0, self.q1 = q0, q1

    def polarization(self):
        st, qs = self.st, list(range(self.q0, self.q1))
        self.P0 = ogw.polarization_tau(st.V, st.G_tau, st.km, qs=qs)

    def screened(self):
        st, qs = self.st, list(range(self.q0, self.q1))
        self.P = np.zeros_like(self.P0)
        Pw = ogw.screened(ogw.to_matsubara(st.grid.TFb, self.P0[qs], 1))
        self.P[qs] = ogw.herm(ogw.to_matsubara(st.grid.TBb, Pw, 1))

    def selfenergy_partial(self):
        st = self.st
        self.Stau = ogw.selfenergy_tau(st.V, st.G_tau, self.P, st.km, qs=list(range(self.q0, self.q1)))

    def get(self, name, out=None):
        assert name == "Sigma_tau"
        out.copy_(__import__("torch").from_numpy(self.Stau))
        return out

    def set(self, name, value):
        assert name == "Sigma_tau"
        self.Stau = value.numpy().copy()

    def selfenergy_finish(self):
        st = self.st
        gam = ogw.density_matrix(st.grid, st.G_tau)
        st.Sigma_inf = ogw.hartree(st.V, gam) + ogw.exchange(st.V, gam)
        st.Sigma_iw = ogw.to_matsubara(st.grid.TFf, self.Stau, 0)
        st.have_sigma = True

    def dyson(self):
        return self.st.dyson()

    def grand_potential(self):
        # the rank's share of Eq. tilde_Phi_GW: its q block, normalised by the full nk
        qs = list(range(self.q0, self.q1))
        return thermo.phi_tilde(self.st.grid, self.P0[qs]) * len(qs) / self.nk


def test_q_blocks_cover_every_q_once():
    for nq in range(1, 70):
        for world in range(1, min(nq, 9) + 1):
            blocks = [q_block(nq, r, world) for r in range(world)]
            assert blocks[0][0] == 0 and blocks[-1][1] == nq
            assert all(a[1] == b[0] for a, b in zip(blocks, blocks[1:]))
            sizes = [b - a for a, b in blocks]
            assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 1
    with pytest.raises(ValueError):
        q_block(3, 0, 4)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _sysd():
    return system(4, 12, (2, 2, 1), 16, 20.0, 77)


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    from paper_2206_07660_gb300.shard import attach
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g = OracleContext(_sysd())
        blk = attach(g, rank, world)
        mu = sharded_iteration(g, device="cpu")
        phi = sharded_grand_potential(g)
        out[rank] = (blk, mu, g.Stau, g.st.G_tau, phi)
    finally:
        dist.destroy_process_group()


def test_two_rank_q_sharded_iteration_matches_unsharded():
    import torch.multiprocessing as mp
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    ref = ogw.State(_sysd())
    ref.dyson()
    phi_ref = thermo.phi_tilde(ref.grid, ogw.polarization_tau(ref.V, ref.G_tau, ref.km))
    ref.iterate()
    assert res[0][0] == (0, 2) and res[1][0] == (2, 4)
    for r in range(world):
        assert np.abs(res[r][2] - ref.Sigma_tau).max() < 1e-13     # summed partials = full Sigma~(tau)
        assert np.abs(res[r][3] - ref.G_tau).max() < 1e-12        # replicated Dyson step
        assert abs(res[r][1] - ref.mu) < 1e-12
        assert abs(res[r][4] - phi_ref) <= 1e-12 * abs(phi_ref)   # summed q blocks = full Phi~
