"""Node-sharded ensembles (the path's multi-process form): the collocation
nodes are independent runs (Sec. 2.4 step 5), so an ensemble splits into
contiguous node ranges, one per process, whose moment sums S1 = sum a_j Q_j,
S2 = sum a_j Q_j^2 and weight sums are added by an all-reduce and finished as
mean = S1/W, var = S2/W - mean^2 (Eq. quad_moments).

CPU tests: the partition, the configuration checks, and a world-size-2 gloo
run of the exchange on oracle shards against the unsharded oracle moments.
"""
import os
import socket

import numpy as np
import pytest

from paper_2508_18202_gb300 import sclbm as S
from paper_2508_18202_gb300 import workloads as W

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("n", [1, 2, 5, 13, 29, 69, 121])
def test_shard_partition_covers_the_rule(n):
    for world in range(1, min(n, 9) + 1):
        ranges = [S.shard_nodes(n, world, r) for r in range(world)]
        assert ranges[0][0] == 0
        for (b0, c0), (b1, _) in zip(ranges, ranges[1:]):
            assert b0 + c0 == b1
        assert sum(c for _, c in ranges) == n
        assert max(c for _, c in ranges) - min(c for _, c in ranges) <= 1
    with pytest.raises(ValueError):
        S.shard_nodes(3, 4, 0)


def test_node_range_checked():
    wl = W.URBAN_LES   # 13 nodes
    assert S.sc_lbm_workspace_size(S.make_config(wl, node_begin=5, node_count=8)) < \
        S.sc_lbm_workspace_size(S.make_config(wl))
    for b, c in ((13, 0), (5, 9), (-1, 2)):
        with pytest.raises(S.ScError) as ei:
            S.sc_lbm_workspace_size(S.make_config(wl, node_begin=b, node_count=c))
        assert ei.value.code == S.SC_ERR_ARG
    Z, a = S.sc_lbm_quadrature(S.make_config(wl, node_begin=5, node_count=8), 0)
    assert len(a) == 13   # the rule itself is always reported whole


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_path):
    import torch.distributed as dist
    from oracle import oracle as O
    from helpers import oracle_domain, oracle_nodes
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    O.set_threads(1)
    wl = dict(W.CHANNEL_CUBE, domains=[dict(nx=24, ny=12, nz=12, boxes=[[6, 4, 0, 10, 8, 6]],
                                            bc=W.CHANNEL_BC, quad_level=5)], steps=40)
    p, flags = oracle_domain(O, wl)
    Z, a = oracle_nodes(O, wl)
    b, c = S.shard_nodes(len(a), world, rank)
    Q = O.ensemble(p, flags, Z[b:b + c], wl["inputs"], wl["u_ref"], wl["alpha"], 0.0, p.nz, wl["steps"])
    w = a[b:b + c]
    s1 = torch.from_numpy(w @ Q)
    s2 = torch.from_numpy(w @ (Q * Q))
    ws = torch.tensor([w.sum()], dtype=torch.float64)
    for t in (s1, s2, ws):
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    mean = s1.numpy() / ws.item()
    std = np.sqrt(np.maximum(s2.numpy() / ws.item() - mean * mean, 0.0))
    if rank == 0:
        Qa = O.ensemble(p, flags, Z, wl["inputs"], wl["u_ref"], wl["alpha"], 0.0, p.nz, wl["steps"])
        m_ref, s_ref, _ = O.moments_two_pass(a, Qa)
        np.savez(out_path, mean=mean, std=std, m_ref=m_ref, s_ref=s_ref)
    dist.barrier()
    dist.destroy_process_group()


def test_gloo_two_rank_exchange(tmp_path):
    """Two gloo ranks run their node shards, all-reduce the sums and finish
    the moments; the result equals the unsharded oracle moments."""
    import sys
    import torch.multiprocessing as mp
    here = os.path.dirname(os.path.abspath(__file__))
    sys.path.insert(0, here)
    out = str(tmp_path / "moments.npz")
    mp.start_processes(_rank_main, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
    r = np.load(out)
    assert np.max(np.abs(r["mean"] - r["m_ref"])) < 1e-14
    assert np.max(np.abs(r["std"] - r["s_ref"])) < 1e-9


@pytest.mark.gpu
def test_shards_on_one_gpu_match_the_whole_ensemble():
    """Two node-range handles on one GPU (an all-reduce emulated by adding
    their sums) reproduce the whole ensemble's moments and gPC coefficients;
    a one-process NCCL group runs the same exchange through sharded_moments."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    wl = dict(W.CHANNEL_CUBE, precision=W.FP32_SHIFT)
    full = S.Ensemble(S.make_config(wl))
    full.step(120)
    ref = full.moments(0, gpc=True)
    n = full.ncell(0)
    s1 = torch.empty(n, dtype=torch.float64, device="cuda")
    s2 = torch.empty_like(s1)
    gs = torch.empty((5, n), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    wsum = []
    for r in range(2):
        b, c = S.shard_nodes(5, 2, r)
        sh = S.Ensemble(S.make_config(wl, node_begin=b, node_count=c))
        assert sh.n_nodes[0] == c
        sh.step(120)
        # the second shard continues the first one's sums on the device
        S.sc_lbm_moment_sums(sh.h, 0, s1, s2, gs, accumulate=r > 0)
        sh.sync()
        wsum.append(S.sc_lbm_weight_sum(sh.h, 0))
        sh.close()
    W_rule = S.sc_lbm_rule_weight_sum(S.make_config(wl), 0)
    assert abs(W_rule - sum(wsum)) < 1e-15
    mean, std = torch.empty_like(s1), torch.empty_like(s1)
    S.sc_lbm_moments_from_sums(full.h, 0, s1, s2, W_rule, mean, std)
    full.sync()
    # node ranges continued one after another give the whole reduction's bits
    # for S1 and S2; the gPC pair sums agree to their 48-bit rounding
    assert torch.equal(mean, ref["mean"])
    assert torch.equal(std, ref["std"])
    assert torch.max(torch.abs(gs - ref["coef"])).item() < 1e-15
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(_free_port())
    dist.init_process_group("nccl", rank=0, world_size=1)
    try:
        out = full.sharded_moments(0, gpc=True)
        torch.cuda.synchronize()
        assert torch.max(torch.abs(out["mean"] - ref["mean"])).item() < 1e-12
        assert torch.max(torch.abs(out["coef"] - ref["coef"])).item() < 1e-15
    finally:
        dist.destroy_process_group()
    full.close()


def test_waves_reject_bad_arguments():
    with pytest.raises(ValueError):
        S.run_in_waves(W.URBAN_BATCHED, 10, 4)          # several domains
    with pytest.raises(ValueError):
        S.run_in_waves(W.CHANNEL_CUBE, 10, 0)


@pytest.mark.gpu
def test_waves_match_the_whole_ensemble():
    """An ensemble run in waves of two nodes (three waves over the 5-node
    rule, one wave's workspace held at a time) gives the whole ensemble's
    moments and gPC coefficients."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    wl = dict(W.CHANNEL_CUBE, precision=W.FP32_SHIFT)
    full = S.Ensemble(S.make_config(wl))
    full.step(120)
    ref = full.moments(0, gpc=True)
    full.sync()
    out = S.run_in_waves(wl, 120, 2, gpc=True)
    assert out["waves"] == 3
    # the waves continue one sum per cell node by node: the same bits for S1
    # and S2, the gPC pair sums to their 48-bit rounding
    assert torch.equal(out["mean"], ref["mean"])
    assert torch.equal(out["std"], ref["std"])
    assert torch.max(torch.abs(out["coef"] - ref["coef"])).item() < 1e-15
    full.close()


def _product_rank_main(rank, world, port, out_path):
    """One rank of the product's node-sharded path: a node-range Ensemble on
    the GPU, stepped, then Ensemble.sharded_moments over a gloo group (the
    all-reduce of the FP64 moment sums, gPC sums and weight sums)."""
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    wl = dict(W.CHANNEL_CUBE, precision=W.FP32_SHIFT)
    b, c = S.shard_nodes(5, world, rank)
    ens = S.Ensemble(S.make_config(wl, node_begin=b, node_count=c))
    ens.step(120)
    out = ens.sharded_moments(0, group=dist.group.WORLD, gpc=True)
    torch.cuda.synchronize()
    if rank == 0:
        np.savez(out_path, mean=out["mean"].cpu().numpy(), std=out["std"].cpu().numpy(),
                 coef=out["coef"].cpu().numpy())
    ens.close()
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.gpu
def test_gloo_two_rank_product_sharding(tmp_path):
    """Two processes, each holding a node-range ensemble on the one GPU (their
    kernels are independent), exchange through Ensemble.sharded_moments over a
    gloo group; the result equals the whole ensemble's moments and gPC
    coefficients (1e-12)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import sys
    import torch.multiprocessing as mp
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    out = str(tmp_path / "sharded.npz")
    mp.start_processes(_product_rank_main, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
    r = np.load(out)
    wl = dict(W.CHANNEL_CUBE, precision=W.FP32_SHIFT)
    full = S.Ensemble(S.make_config(wl))
    full.step(120)
    ref = full.moments(0, gpc=True)
    full.sync()
    assert np.max(np.abs(r["mean"] - ref["mean"].cpu().numpy())) < 1e-12
    assert np.max(np.abs(r["std"] - ref["std"].cpu().numpy())) < 1e-9
    assert np.max(np.abs(r["coef"] - ref["coef"].cpu().numpy())) < 1e-12
    full.close()
