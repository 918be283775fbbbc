"""Multi-rank logic on CPU: two gloo ranks (127.0.0.1) shard the 2D ray set, step their own rays
with the CPU oracle (no collective on the data path) and combine timing with a MAX and throughput
with the whole-job formula; a ray-sharded adjoint sums the objective and the opacity-scale
gradient over the ranks with one all-reduce."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip('torch')
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(('127.0.0.1', 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR='127.0.0.1', MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group('gloo', rank=rank, world_size=world)
    import bench
    from oracle import mgfld_oracle as O
    from paper_1809_05608_gb300 import problems
    rpr = 3
    mine = bench.workload(world, rank, rays_per_rank=rpr)
    full = problems.make_problem(bench.CONFIG_ID, n_ray=rpr * world)
    sl = bench.shard(world, rank, rpr)
    same = all(np.array_equal(mine[k], full[k][sl]) for k in ('psi0', 'ye0', 'T0'))
    same &= np.array_equal(mine['problem']['kappa_abs'], full['problem']['kappa_abs'][sl])
    # Step one ray of the shard with the oracle (on reduced sizes to stay fast).
    small = problems.make_problem(bench.CONFIG_ID, n_ray=rpr * world, n_r=12, n_e=4)
    sub = problems.subset_rays(small, slice(sl.start, sl.start + 1))
    res = O.step(sub['problem'], sub['psi0'], sub['ye0'], sub['T0'])
    ms = torch.tensor([10.0 * (rank + 1)], dtype=torch.float64)
    dist.all_reduce(ms, op=dist.ReduceOp.MAX)
    ups = bench.updates_per_step(mine)
    value = bench.job_throughput(ups, world, float(ms.item()))
    psi_sum = torch.tensor([float(res['psi'].sum())], dtype=torch.float64)
    dist.all_reduce(psi_sum, op=dist.ReduceOp.SUM)
    out[rank] = (same, float(ms.item()), value, ups, float(psi_sum.item()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_rays_and_take_the_slowest_rank():
    world = 2
    port = _free_port()
    mgr = mp.get_context('spawn').Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, join=True, start_method='spawn')
    assert sorted(out.keys()) == [0, 1]
    for r in range(world):
        same, ms, value, ups, _ = out[r]
        assert same                                   # shard = the right block of the full ray set
        assert ms == 20.0                             # MAX over ranks
        assert ups == 3 * 4 * 512 * 20
        assert value == pytest.approx(ups * world / 20e-3)
    assert out[0][4] == out[1][4]                     # the SUM reached both ranks


def _adjoint_rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR='127.0.0.1', MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group('gloo', rank=rank, world_size=world)
    from oracle import mgfld_adjoint_oracle as A
    from paper_1809_05608_gb300 import adjoint, problems
    from tests import small_problems as SP
    inp = SP.strong(n_ray=2 * world, n_r=8, n_e=3, kabs=1e16, kscat=1e15, nes=10.0)
    mine = problems.subset_rays(inp, slice(2 * rank, 2 * rank + 2))
    scale = np.ones((4, 3)) * (1.0 + 0.05 * np.arange(12).reshape(4, 3))
    J, g_psi, g_s = A.objective_and_gradients(mine['problem'], mine['psi0'], mine['ye0'], mine['T0'], scale, 2)
    Jt, gt = adjoint.reduce_over_ranks(float(J.sum()), torch.as_tensor(g_s))
    out[rank] = (float(Jt), gt.numpy().copy(), g_psi.copy())
    dist.barrier()
    dist.destroy_process_group()


def test_ray_sharded_adjoint_sums_objective_and_scale_gradient_over_ranks():
    """The oracle adjoint on each rank's two rays, reduced over two gloo ranks, equals the oracle
    adjoint on all four rays: J and dJ/dscale summed, dJ/dpsi0 the rank's own block."""
    from oracle import mgfld_adjoint_oracle as A
    from tests import small_problems as SP
    world = 2
    port = _free_port()
    mgr = mp.get_context('spawn').Manager()
    out = mgr.dict()
    mp.start_processes(_adjoint_rank, args=(world, port, out), nprocs=world, join=True, start_method='spawn')
    inp = SP.strong(n_ray=2 * world, n_r=8, n_e=3, kabs=1e16, kscat=1e15, nes=10.0)
    scale = np.ones((4, 3)) * (1.0 + 0.05 * np.arange(12).reshape(4, 3))
    J, g_psi, g_s = A.objective_and_gradients(inp['problem'], inp['psi0'], inp['ye0'], inp['T0'], scale, 2)
    for r in range(world):
        Jr, gr, gpr = out[r]
        assert Jr == pytest.approx(float(J.sum()), rel=1e-12)
        assert np.allclose(gr, g_s, rtol=1e-11, atol=1e-11 * np.max(np.abs(g_s)))
        assert np.allclose(gpr, g_psi[2 * r:2 * r + 2], rtol=1e-11, atol=1e-11 * np.max(np.abs(g_psi)))
    assert np.max(np.abs(g_s)) > 0.0
