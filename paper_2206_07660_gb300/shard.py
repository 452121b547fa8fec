"""One GW problem split over several GPUs by blocks of q-points.

Per q-point, the polarization P~0^q (Eq. tilde_P0_tau), its transform, the
screened solve (Eq. tilde_P_omega) and the transform back are independent of
every other q, and the self-energy (Eq. tilde_sigma2) is a sum of one term
per q.  The paper's GPU scheme distributes the q-points over MPI ranks and
reduces the self-energy (Sec. "GPU acceleration"); here every rank holds one
context restricted to a contiguous q block (gw_set_q_range) and the partial
sums Sigma~^k(tau) are added with one all-reduce per iteration.  Hartree-Fock,
the transform of Sigma~, the damping and the Dyson step are replicated: every
rank gets the same summed Sigma~(tau), so every rank computes the same G.

The functions take any object with the GW binding's methods, so the same
host logic runs on GPU contexts and, in the CPU tests, on stand-ins.
"""


def q_block(nq, rank, world):
    """Contiguous q range [q0, q1) of `rank`: block sizes differ by at most one."""
    if not (0 <= rank < world) or nq < world:
        raise ValueError("need 0 <= rank < world <= nq")
    base, extra = divmod(nq, world)
    q0 = rank * base + min(rank, extra)
    return q0, q0 + base + (1 if rank < extra else 0)


def sum_over_ranks(x, group=None):
    """In-place sum of a tensor over the ranks of `group` (no-op without one)."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(x, op=dist.ReduceOp.SUM, group=group)
    return x


def attach(g, rank, world):
    """Restrict the context `g` to this rank's q block; returns the block."""
    q0, q1 = q_block(g.nk, rank, world)
    g.set_q_range(q0, q1)
    return q0, q1


def sharded_iteration(g, device="cuda", group=None, reduce=sum_over_ranks):
    """One GW iteration of a q-sharded context (the rank's share of P~0, screened
    solve and Sigma~, one reduction of Sigma~(tau), the replicated rest).
    Returns mu after the Dyson step."""
    import torch
    g.polarization()
    g.screened()
    g.selfenergy_partial()
    S = torch.empty(g.shape_of("Sigma_tau"), dtype=torch.complex128, device=device)
    g.get("Sigma_tau", out=S)
    reduce(S, group)
    g.set("Sigma_tau", S)
    g.selfenergy_finish()
    return g.dyson()


def sharded_grand_potential(g, group=None, reduce=sum_over_ranks):
    """Phi~ (Eq. tilde_Phi_GW) of a q-sharded problem: each rank's context sums its
    own q block (gw_grand_potential) and one all-reduce adds the blocks.  Call it
    after the rank's polarization step."""
    import torch
    x = torch.tensor([g.grand_potential()], dtype=torch.float64)
    reduce(x, group)
    return float(x[0])
