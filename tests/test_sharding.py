"""The multi-rank path on CPU: targets sharded over two gloo ranks, each rank's W computed by
the FP64 oracle for its targets, energy shares combined with the float64 all-reduce; the
result equals the single-process apply and energy."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle as O
import workloads as W
from paper_2401_04189_gb300.sharding import combine_energy, energy_share, target_range


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


def _system():
    return W.config_small(n=14, n_orb=5, rank=6, T=4, L=4.0)


def _rank_main(rank, world, port, outdir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        s = _system()
        S = O.Setup.from_system(s)
        a, b = target_range(s.psi.shape[0], world, rank)
        Wl = O.exchange_apply(s.psi, S, psi_tgt=s.psi[a:b])
        e = energy_share(torch.from_numpy(s.psi[a:b]), torch.from_numpy(Wl), *s.w)
        etot = combine_energy(e)
        np.save(os.path.join(outdir, f"w{rank}.npy"), Wl)
        np.save(os.path.join(outdir, f"e{rank}.npy"), np.array([float(e), float(etot)]))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as so:
        so.bind(("127.0.0.1", 0))
        return so.getsockname()[1]


def test_two_gloo_ranks_match_single_process(tmp_path):
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    s = _system()
    S = O.Setup.from_system(s)
    W_full = O.exchange_apply(s.psi, S)
    E_full = O.exchange_energy(s.psi, S, W_full)
    shards = [np.load(tmp_path / f"w{r}.npy") for r in range(world)]
    np.testing.assert_allclose(np.concatenate(shards), W_full, rtol=0, atol=1e-12 * np.abs(W_full).max())
    e = [np.load(tmp_path / f"e{r}.npy") for r in range(world)]
    assert abs(e[0][0] + e[1][0] - E_full) <= 1e-12 * abs(E_full)
    # every rank holds the combined energy after the all-reduce
    for r in range(world):
        assert abs(e[r][1] - E_full) <= 1e-12 * abs(E_full)
