"""Multi-rank sharding of projections (host logic, gloo on CPU)."""
import os
import socket

import pytest

from paper_2503_20146_gb300.shard import projection_cost, rank_loads, shard_projections

# the mixed-size workload: 16 projections each of 256^2, 768^2, 1536^2, 2048^2, K = 25
MIXED = [(n, n, 25) for n in (256, 768, 1536, 2048) for _ in range(16)]


@pytest.mark.parametrize("world", [1, 2, 3, 4, 8])
def test_shards_partition_and_balance(world):
    shards = [shard_projections(MIXED, world, r) for r in range(world)]
    flat = sorted(i for s in shards for i in s)
    assert flat == list(range(len(MIXED)))               # every projection exactly once
    loads = rank_loads(MIXED, world)
    biggest = max(projection_cost(*s) for s in MIXED)
    assert max(loads) - min(loads) <= biggest            # LPT bound


def test_bad_rank_rejected():
    with pytest.raises(ValueError):
        shard_projections(MIXED, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    mine = shard_projections(MIXED, world, rank)
    # each rank "solves" its share: here a stand-in value per projection
    local = {i: float(i) * 2.0 for i in mine}
    gathered = [None] * world
    dist.all_gather_object(gathered, local)
    t = torch.tensor([len(mine)], dtype=torch.int64)
    dist.all_reduce(t)
    if rank == 0:
        merged = {}
        for g in gathered:
            assert not (set(g) & set(merged))
            merged.update(g)
        q.put((sorted(merged), int(t.item())))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gloo_gather_covers_the_series():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    keys, total = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert keys == list(range(len(MIXED))) and total == len(MIXED)


# a small uneven series for the solve test: (ny, nx, n_modes) per projection
SMALL = [(32, 32, 0), (48, 48, 0), (32, 32, 0), (48, 48, 0), (32, 32, 0)]


def _small_inputs(i):
    """Seeded inputs of projection i of SMALL (measurement from the oracle)."""
    import numpy as np
    from oracle import pwf_oracle as O
    from paper_2503_20146_gb300 import synth as S
    ny, nx, _ = SMALL[i]
    w = S.WORKLOADS["blob512_iotf"]
    g = O.Geometry(ny, nx, w.pixel_m, w.wavelength_m, w.L1_m, w.L2_m, w.xcoh_m, w.ycoh_m, w.gamma, w.alpha, w.eta)
    t = S.diffuser(ny, nx, S.rng_for(w.config, 99))
    psi_true = S.complex_phase_from(S.blob_phase(ny, nx, S.rng_for(w.config, 10 + i)))
    y = S.poisson_measurement(O.intensity(psi_true, t, g), 1e4, S.rng_for(w.config, 60 + i))
    return g, t, np.asarray(y, np.float64)


def _solve_one(i, iters=4):
    from oracle import pwf_oracle as O
    g, t, y = _small_inputs(i)
    return O.solve(y, t, g, iters).psi


def _solve_worker(rank, world, port, q):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    mine = shard_projections(SMALL, world, rank)
    local = {i: _solve_one(i) for i in mine}          # no exchange during the iterations
    gathered = [None] * world
    dist.all_gather_object(gathered, local)           # one gather of the results at the end
    if rank == 0:
        merged = {}
        for g in gathered:
            merged.update(g)
        q.put(merged)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gloo_solves_match_one_process():
    """Each of two gloo ranks solves its cost-balanced share of an uneven series
    (the FP64 oracle stands in for the GPU solve on this CPU-only test) and the
    results are gathered once: the same iterates as one process solving all."""
    import numpy as np
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_solve_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    merged = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert sorted(merged) == list(range(len(SMALL)))
    assert shard_projections(SMALL, 2, 0) and shard_projections(SMALL, 2, 1)   # both ranks had work
    for i in range(len(SMALL)):
        assert np.array_equal(merged[i], _solve_one(i))
