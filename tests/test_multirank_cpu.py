"""The N > 1 path of bench.py on CPU: two gloo ranks (world_size 2).

Ranks run disjoint realizations with no data-path collective; the only
collectives are the timing reduction (max over ranks) and the eigenpair count
(sum over ranks).  This checks both, and that the realization indices of the
ranks never overlap, without a GPU.
"""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    cpu = torch.device("cpu")
    # rank r reports device time 1 + r, wall time 2 + r and 10 + r passing eigenpairs
    t_dev, wall, pairs, pairs_wall = bench.reduce_ranks(torch, cpu, dist, 1.0 + rank, 2.0 + rank, 10 + rank,
                                                         7.5 + rank)
    mine = [bench.timed_realization(k, world, rank) for k in range(5)]
    mine += [bench.warmup_realization(w, world, rank) for w in range(3)]
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    spec = bench.BATCHED["batched64_L16_L18"]
    seeds = [(m.L, tuple(m.h)) for k in range(2)
             for m in bench.batched_models(spec, 1000 * bench.timed_realization(k, world, rank))[0]]
    all_seeds = [None] * world
    dist.all_gather_object(all_seeds, seeds)
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
        f.write(repr((t_dev, wall, pairs, pairs_wall, gathered, [len(set(x)) for x in all_seeds],
                      len(set(all_seeds[0]) & set(all_seeds[1])))))


def test_two_gloo_ranks_reduce_and_shard(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    res = [eval(open(tmp_path / f"rank{r}.txt").read()) for r in range(2)]
    for t_dev, wall, pairs, pairs_wall, gathered, n_unique, n_shared in res:
        assert (t_dev, wall, pairs, pairs_wall) == (2.0, 3.0, 21.0, 16.0)  # max, max, sum, sum
        a, b = set(gathered[0]), set(gathered[1])
        assert len(a) == len(gathered[0]) and not (a & b)  # disjoint realizations
        assert n_unique == [128, 128] and n_shared == 0  # batched workloads: distinct field sets per rank


def test_credited_pairs_by_overlap():
    import bench
    runs = [(0.0, 10.0, 100), (10.0, 20.0, 50), (20.0, 40.0, 80)]
    # half of run 0, half of run 1, none of run 2
    assert abs(bench.credited_pairs(runs, 5.0, 15.0) - 75.0) < 1e-12
    # all of run 1 and a quarter of run 2
    assert abs(bench.credited_pairs(runs, 10.0, 25.0) - 70.0) < 1e-12
    # one run at a constant rate: the credited rate equals the run's rate
    assert abs(bench.credited_pairs([(0.0, 8.0, 40)], 2.0, 6.0) / 4.0 - 5.0) < 1e-12
