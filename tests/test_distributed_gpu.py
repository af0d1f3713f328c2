"""The wavelength-sharded Lambda iteration on one GPU.

* one rank: identical to the unsharded accelerated iteration;
* two ranks emulated by two host threads, each with its own context and
  stream, exchanging the float64 rates on the host between iterations (no
  kernel waits on another): populations within 1e-12 of the unsharded run --
  every wavelength batch is solved by the same kernels on the same data, only
  the order of the rate sum differs;
* the linearity the exchange relies on, on the rates kernel itself.
"""

import threading

import numpy as np
import pytest

import synth
from synth.atom import line_wavelength_grid, populations_atmosphere, three_level_atom

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N = 48


@pytest.fixture(scope="module")
def setup():
    from paper_2511_08498_gb300 import api
    ad = three_level_atom()
    m = populations_atmosphere(N, N, seed=synth.SEED_BASE + 500)
    lam, tag = line_wavelength_grid(8, 4)
    atom = api.Atom.from_dict(ad, m["cell_cm"])
    dev = {k: torch.from_numpy(np.ascontiguousarray(m[k]).reshape(-1)).cuda() for k in ("temperature", "ne", "nh")}
    dirs, w = synth.directions(16)
    return dict(api=api, atom=atom, lam=lam, tag=tag, dev=dev, dirs=dirs, w=w, m=m)


def _unsharded(s, ctx):
    api, d = s["api"], s["dev"]
    return api.lambda_iteration(ctx, s["atom"], s["lam"], s["tag"], d["temperature"], d["ne"], d["nh"], N, N,
                                s["dirs"], s["w"], 6, accelerated=True, iod=1e-2).cpu().numpy()


def test_one_rank_equals_unsharded(setup):
    from paper_2511_08498_gb300 import distributed
    s = setup
    ctx = s["api"].Context(0)
    d = s["dev"]
    ref = _unsharded(s, ctx)
    got = distributed.lambda_iteration_sharded(ctx, s["atom"], s["lam"], s["tag"], d["temperature"], d["ne"],
                                               d["nh"], N, N, s["dirs"], s["w"], 6).cpu().numpy()
    ctx.check()
    assert np.array_equal(got, ref)


def test_two_emulated_ranks_match_unsharded(setup):
    from paper_2511_08498_gb300 import distributed
    s = setup
    api, d = s["api"], s["dev"]
    ref = _unsharded(s, api.Context(0))
    world = 2
    bar = threading.Barrier(world, timeout=120)
    host = [None] * world
    out, errors = [None] * world, []

    def rank_main(r):
        try:
            stream = torch.cuda.Stream()
            with torch.cuda.stream(stream):
                ctx = api.Context(0, stream=stream)

                def reduce(jbar):
                    ctx.check()
                    host[r] = jbar.cpu()
                    bar.wait()
                    total = host[0] + host[1]
                    bar.wait()
                    jbar.copy_(total)

                pops = distributed.lambda_iteration_sharded(ctx, s["atom"], s["lam"], s["tag"], d["temperature"],
                                                            d["ne"], d["nh"], N, N, s["dirs"], s["w"], 6, rank=r,
                                                            world=world, reduce=reduce)
                ctx.check()
                out[r] = pops.cpu().numpy()
        except Exception as e:  # surfaced below
            errors.append(e)
            bar.abort()

    threads = [threading.Thread(target=rank_main, args=(r,)) for r in range(world)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    live = s["m"]["temperature"].reshape(-1) > 0
    for r in range(world):
        rel = np.abs(out[r] - ref) / np.maximum(np.abs(ref), 1e-300)
        assert rel[:, live].max() < 1e-12, (r, rel[:, live].max())


def test_rates_are_linear_in_J(setup):
    from paper_2511_08498_gb300.distributed import wavelength_shard
    s = setup
    api, d = s["api"], s["dev"]
    ctx = api.Context(0)
    L = s["lam"].size
    J = torch.from_numpy(np.random.default_rng(4).uniform(0.1, 2.0, (L, N * N)).astype(np.float32) * 1e-5).cuda()
    full = api.rates_accumulate(ctx, s["atom"], s["lam"], s["tag"], d["temperature"], J)
    acc = torch.zeros_like(full)
    for r in range(3):
        l0, l1 = wavelength_shard(L, 8, r, 3)
        Jr = torch.zeros_like(J)
        Jr[l0:l1] = J[l0:l1]
        acc += api.rates_accumulate(ctx, s["atom"], s["lam"], s["tag"], d["temperature"], Jr)
    ctx.check()
    rel = ((acc - full).abs() / full.abs().clamp_min(1e-300)).max().item()
    assert rel < 1e-13
