"""The multi-GPU host logic on CPU ranks (gloo, world size 2).

* wavelength_shard: whole batches, disjoint, covering every wavelength;
* the one exchange of the sharded Lambda iteration: each rank reduces the
  radiative rates of its own wavelength range (J zero elsewhere) over the full
  grid -- here with the float64 oracle as the per-rank computation -- and the
  float64 sum-allreduce over the ranks equals the rates of the whole J;
* the benchmark's reductions: the slowest rank's time (max) and the units of
  every rank's atmosphere (sum).
"""

import os
import socket
import tempfile

import numpy as np
import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")


def test_wavelength_shard_partitions_whole_batches():
    from paper_2511_08498_gb300.distributed import wavelength_shard
    for L in (1, 7, 8, 9, 32, 96, 100):
        for W in (1, 4, 8):
            for world in (1, 2, 3, 5, 16):
                ranges = [wavelength_shard(L, W, r, world) for r in range(world)]
                cover = []
                for l0, l1 in ranges:
                    assert l0 <= l1
                    assert l0 % W == 0 or l0 == L
                    assert l1 == L or l1 % W == 0
                    cover.extend(range(l0, l1))
                assert cover == list(range(L))
                sizes = [-(-(l1 - l0) // W) for l0, l1 in ranges]
                assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        wavelength_shard(8, 8, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import synth
    from oracle import atom as oa
    from paper_2511_08498_gb300.distributed import allreduce_sum_, reduce_scalar, wavelength_shard
    from synth.atom import line_wavelength_grid, populations_atmosphere, three_level_atom
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    ad = three_level_atom()
    m = populations_atmosphere(32, 32, seed=synth.SEED_BASE + 500)
    lam, tag = line_wavelength_grid(8, 4)
    T = m["temperature"].reshape(-1)
    L = lam.size
    J = np.random.default_rng(11).uniform(0.1, 2.0, (L, T.size)) * 1e-5
    l0, l1 = wavelength_shard(L, 8, rank, world)
    Jr = np.zeros_like(J)
    Jr[l0:l1] = J[l0:l1]
    part = torch.from_numpy(oa.jbar(ad, lam, tag, T, Jr))
    allreduce_sum_(part)
    full = oa.jbar(ad, lam, tag, T, J)
    err = float(np.abs(part.numpy() - full).max() / np.abs(full).max())
    t_max = reduce_scalar(1.0 + rank, "max")
    u_sum = reduce_scalar(10.0 * (rank + 1), "sum")
    with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as fh:
        fh.write(f"{err} {t_max} {u_sum} {l0} {l1}\n")
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_rates_allreduce_on_two_cpu_ranks():
    import torch.multiprocessing as mp
    world = 2
    with tempfile.TemporaryDirectory() as d:
        mp.spawn(_rank_main, args=(world, _free_port(), d), nprocs=world, join=True)
        rows = [open(os.path.join(d, f"rank{r}.txt")).read().split() for r in range(world)]
    for r, row in enumerate(rows):
        err, t_max, u_sum = float(row[0]), float(row[1]), float(row[2])
        assert err < 1e-12, (r, err)
        assert t_max == 2.0 and u_sum == 30.0
    # the two ranks held different, adjacent wavelength ranges
    assert rows[0][4] == rows[1][3] and rows[0][3] == "0"


def test_single_process_reductions_are_identity():
    from paper_2511_08498_gb300.distributed import allreduce_sum_, reduce_scalar
    t = torch.arange(5, dtype=torch.float64)
    assert torch.equal(allreduce_sum_(t.clone()), t)
    assert reduce_scalar(3.5, "max") == 3.5
