"""The multi-rank path: targets sharded over two gloo ranks, energy shares combined with the
float64 all-reduce; the result equals the single-process apply and energy.

On the CPU each rank's W and energy share come from the FP64 oracle (the partitioning and the
collective are what is tested).  Where a GPU is present, the same two ranks run the library's
own sharded path (paper_2401_04189_gb300.sharding.exchange_apply_sharded and energy_share, on
cuda:0 each; the ranks' kernels never wait on one another) and are checked against the oracle."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle as O
import workloads as W
from _helpers import W_TOL, E_TOL, rel
from paper_2401_04189_gb300.sharding import combine_energy, target_range


def test_target_range_partitions_every_size():
    for n in (0, 1, 5, 64, 65):
        for world in (1, 2, 3, 8):
            got = [target_range(n, world, r) for r in range(world)]
            assert got[0][0] == 0 and got[-1][1] == n
            assert all(got[r][1] == got[r + 1][0] for r in range(world - 1))
            sizes = [b - a for a, b in got]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        target_range(4, 2, 2)


def _system(gpu):
    # the tensor-core paths need n3 % 4 == 0; the float32 path takes any grid
    return W.config_small(n=16, n_orb=5, rank=6, T=4, L=4.0) if gpu else W.config_small(n=14, n_orb=5, rank=6, T=4, L=4.0)


def _rank_main(rank, world, port, outdir, gpu):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        s = _system(gpu)
        if gpu:
            import paper_2401_04189_gb300 as P
            from paper_2401_04189_gb300.sharding import energy_share, exchange_apply_sharded
            torch.cuda.set_device(0)
            ctx = P.Context.from_system(s, precision="fp32")
            psi = torch.from_numpy(np.ascontiguousarray(s.psi, dtype=np.float32)).cuda()
            a, b, Wl_t = exchange_apply_sharded(ctx, psi, world, rank)
            e_t = energy_share(ctx, psi[a:b], Wl_t)
            torch.cuda.synchronize()
            Wl = Wl_t.cpu().numpy().astype(np.float64)
            e = float(e_t.item())
            ctx.destroy()
        else:
            S = O.Setup.from_system(s)
            a, b = target_range(s.psi.shape[0], world, rank)
            Wl = O.exchange_apply(s.psi, S, psi_tgt=s.psi[a:b])
            e = O.exchange_energy(s.psi[a:b], S, W=Wl)      # 1/2 sum over this rank's targets
        etot = combine_energy(torch.tensor(e, dtype=torch.float64))
        np.save(os.path.join(outdir, f"w{rank}.npy"), Wl)
        np.save(os.path.join(outdir, f"e{rank}.npy"), np.array([e, float(etot)]))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as so:
        so.bind(("127.0.0.1", 0))
        return so.getsockname()[1]


def _run(tmp_path, gpu):
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path), gpu), nprocs=world, join=True)
    s = _system(gpu)
    S = O.Setup.from_system(s)
    W_full = O.exchange_apply(s.psi, S)
    E_full = O.exchange_energy(s.psi, S, W_full)
    shards = [np.load(tmp_path / f"w{r}.npy") for r in range(world)]
    e = [np.load(tmp_path / f"e{r}.npy") for r in range(world)]
    return np.concatenate(shards), W_full, e, E_full


def test_two_gloo_ranks_match_single_process(tmp_path):
    Wc, W_full, e, E_full = _run(tmp_path, gpu=False)
    np.testing.assert_allclose(Wc, W_full, rtol=0, atol=1e-12 * np.abs(W_full).max())
    assert abs(e[0][0] + e[1][0] - E_full) <= 1e-12 * abs(E_full)
    # every rank holds the combined energy after the all-reduce
    for r in range(2):
        assert abs(e[r][1] - E_full) <= 1e-12 * abs(E_full)


@pytest.mark.gpu
def test_two_gloo_ranks_run_the_library_sharded_path(tmp_path):
    Wc, W_full, e, E_full = _run(tmp_path, gpu=True)
    assert rel(Wc, W_full) < W_TOL["fp32"]
    assert abs(e[0][0] + e[1][0] - E_full) <= E_TOL["fp32"] * abs(E_full)
    for r in range(2):
        assert abs(e[r][1] - (e[0][0] + e[1][0])) <= 1e-15 * abs(E_full) + 1e-300
