"""Host logic of batched spots (no GPU): bucket planning, workspace sizing,
sharding over ranks, and the gather of per-rank doses over a two-rank gloo
process group."""
import os
import socket

import numpy as np
import pytest

from paper_2504_00340_gb300 import spots as S
from paper_2504_00340_gb300.workloads import spot_batch


@pytest.fixture(scope="module")
def batch():
    return spot_batch()


def test_spot_batch_recipe(batch):
    assert len(batch) == 256
    e0 = np.array([w.beam["e0"] for w in batch])
    assert e0.min() >= 70.0 and e0.max() <= 200.0
    for w in batch:
        assert w.ng == int(np.ceil(w.beam["e0"] / 0.5))
        assert (w.ny == 64) == (w.beam["e0"] <= 135.0) and w.ny in (64, 96)
        rng_cm = 0.0022 * w.beam["e0"] ** 1.77
        assert w.n_steps == int(np.ceil((rng_cm + 1.0) / 0.05))
    centres = {(round(w.beam["yc"], 6), round(w.beam["zc"], 6)) for w in batch}
    assert len(centres) == 256  # a 16 x 16 grid of distinct centres


@pytest.mark.parametrize("max_gb,waste", [(48, 0.1), (8, 0.05), (200, 0.2)])
def test_plan_buckets_invariants(batch, max_gb, waste):
    buckets = S.plan_buckets(batch, max_bytes=max_gb << 30, max_waste=waste)
    seen = sorted(i for b in buckets for i in b.members)
    assert seen == list(range(len(batch)))  # every spot exactly once
    for b in buckets:
        ws = [batch[i] for i in b.members]
        assert len({S._grid_key(w) for w in ws}) == 1
        assert all(w.ng >= (1 - waste) * b.ng and w.e_max <= b.e_max for w in ws)
        assert b.steps == [w.n_steps for w in ws]
        assert all(x >= y for x, y in zip(b.steps, b.steps[1:]))
        w = ws[0]
        assert S.workspace_bytes(w.ny, w.nz, w.nu, w.nv, b.ng, b.nx, w.n_scatter, len(ws), w.precision) \
            <= max_gb << 30
    processed = sum(S.bucket_cost(b, batch) for b in buckets)
    useful = S.useful_cost(batch)
    assert useful <= processed <= useful / (1 - waste) * 1.001


def test_workspace_bytes_single_beam_regions():
    # primary only, FP32: psi dominates; two scattered components add R/src and P^2
    a = S.workspace_bytes(8, 8, 4, 4, 10, 3, 0, 1, "fp32")
    psi = 10 * 2 * 16 * 64 * 4
    assert psi < a < psi + 64 * 1024
    b = S.workspace_bytes(8, 8, 4, 4, 10, 3, 2, 1, "mixed")
    assert b > 3 * psi + 4 * 10 * 16 * 64 * 2


def test_plan_rejects_oversize_spot(batch):
    with pytest.raises(ValueError):
        S.plan_buckets(batch[:4], max_bytes=1 << 20)


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_shard_buckets_partition(batch, world):
    buckets = S.plan_buckets(batch)
    shards = S.shard_buckets(buckets, batch, world)
    flat = sorted(j for r in shards for j in r)
    assert flat == list(range(len(buckets)))
    loads = [sum(S.bucket_cost(buckets[j], batch) for j in r) for r in shards]
    biggest = max(S.bucket_cost(b, batch) for b in buckets)
    assert max(loads) - min(loads) <= biggest  # LPT bound


def _fake_march(b, spots):
    return {i: np.full((b.steps[j], 2, 2), float(i)) for j, i in enumerate(b.members)}, 1.0, 5, (8, 0)


def _worker(rank, world, port, out_path):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sp = spot_batch(n_beams=40)
        doses, stats = S.run_shard(sp, rank, world, march=_fake_march)
        merged = S.gather_doses(doses, rank, world)
        if rank == 0:
            np.savez(out_path, keys=np.array(list(merged.keys())),
                     ok=np.array([np.all(v == k) and v.shape[0] == sp[k].n_steps for k, v in merged.items()]),
                     buckets=np.array([stats["buckets"]]))
    finally:
        dist.destroy_process_group()


def test_two_rank_gather_gloo(tmp_path):
    import torch.multiprocessing as mp
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    out = str(tmp_path / "gather.npz")
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    r = np.load(out)
    assert list(r["keys"]) == list(range(40))
    assert r["ok"].all()
