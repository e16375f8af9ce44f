"""World-size-2 gloo test of the sharded form of the path (CPU, no GPU).

Columns are independent given V_eff (Sec. 3, "Spectral weights, nodes and electronic fields"), so
ranks take disjoint column ranges and need one collective: a sum of the K+1 moment sums before the
Fermi solve (the paper's single global reduction, Eq. Ne).  Each rank then forms its own part of
rho.  On the CPU the per-column moments come from the oracle (the library's recursion needs a GPU);
the Fermi level and the weights after the allreduce come from the library's pure host entry points
sq_fermi_level and sq_fermi_weights, the calls a sharded GPU run makes.  The result must equal the
single-process oracle solve."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_path):
    import torch
    from oracle import oracle
    from paper_2011_13517_gb300 import cells
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    c = cells.tiny_cell()
    lo, hi = oracle.spectral_bounds(c)
    omega, tau = oracle.scale_shift(lo, hi)
    cols = np.array_split(np.arange(c.N_d), world)[rank]
    mu = oracle.moments(c, omega, tau, cols=cols, nthreads=2)
    msum = torch.from_numpy(mu.sum(axis=0))
    dist.all_reduce(msum, op=dist.ReduceOp.SUM)
    from paper_2011_13517_gb300 import sq
    lam_f = sq.sq_fermi_level(msum.numpy(), c.K, omega, tau, lo, hi, c.kT, c.N_e)
    coef, dcoef, _ = sq.sq_fermi_weights(lam_f, c.K, omega, tau, c.kT)
    rho_part = torch.from_numpy(2.0 * (mu @ coef) / float(np.prod(c.h)))
    U = 2.0 * float(dcoef @ msum.numpy())
    # gather the density parts (equal-sized shards here: 3570 = 2 x 1785)
    parts = [torch.zeros_like(rho_part) for _ in range(world)]
    dist.all_gather(parts, rho_part)
    if rank == 0:
        np.savez(out_path, lam_f=lam_f, msum=msum.numpy(), rho=torch.cat(parts).numpy(), U=U)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.slow
def test_two_rank_column_shard_matches_single_process(tmp_path):
    from oracle import oracle
    from paper_2011_13517_gb300 import cells
    out = str(tmp_path / "r0.npz")
    mp.spawn(_worker, args=(2, _free_port(), out), nprocs=2, join=True)
    got = np.load(out)
    c = cells.tiny_cell()
    ref = oracle.sq_solve(c, force=False)
    assert abs(float(got["lam_f"]) - ref["lam_f"]) < 1e-12
    np.testing.assert_allclose(got["msum"], ref["Msum"], rtol=1e-13, atol=1e-12)
    np.testing.assert_allclose(got["rho"], ref["rho"], rtol=1e-12, atol=1e-14)
    assert abs(float(got["U"]) - ref["U"]) < 1e-11 * abs(ref["U"])
