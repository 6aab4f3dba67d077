"""Host logic of the lateral domain decomposition (Remark 2: only the
lateral transport couples lateral points): the row split, the halo exchange
plan, and the exchange itself over torch.distributed with gloo ranks on the
CPU.  A stand-in for the transport substep (a linear stencil reaching four
rows on either side, zero outside the grid) marched on the parts with an
exchange before every application equals the stencil marched on the whole
grid, which is the property the four halo rows exist for."""
import os
import socket

import numpy as np
import pytest

from paper_2504_00340_gb300.domain import HALO, assemble_rows, halo_plan, split_rows


@pytest.mark.parametrize("ny,n", [(128, 2), (130, 3), (37, 4), (8, 2), (9, 1)])
def test_split_rows_tiles_the_grid(ny, n):
    lay = split_rows(ny, n)
    assert lay[0].y_offset == 0 and lay[0].halo_lo == 0
    assert lay[-1].y_offset + lay[-1].ny == ny and lay[-1].halo_hi == 0
    for a, b in zip(lay, lay[1:]):
        assert a.own_end == b.own_start
        assert a.halo_hi == HALO and b.halo_lo == HALO
    own = [x.own_end - x.own_start for x in lay]
    assert sum(own) == ny and max(own) - min(own) <= 1


def test_split_rows_rejects_parts_thinner_than_the_halo():
    with pytest.raises(ValueError):
        split_rows(7, 2)
    with pytest.raises(ValueError):
        split_rows(3, 4)


@pytest.mark.parametrize("ny,n", [(64, 2), (50, 3), (41, 5)])
def test_halo_plan_pairs_up(ny, n):
    """What part r sends to part r' is exactly what r' receives from r, and
    both name the same rows of the grid: r's own rows that r' mirrors."""
    lay = split_rows(ny, n)
    for r in range(n):
        for m in halo_plan(lay, r):
            back = [x for x in halo_plan(lay, m.peer) if x.peer == r]
            assert len(back) == 1
            b = back[0]
            assert m.n_send == b.n_recv and m.n_recv == b.n_send
            sent = np.arange(m.send_first, m.send_first + m.n_send) + lay[r].y_offset
            got = np.arange(b.recv_first, b.recv_first + b.n_recv) + lay[m.peer].y_offset
            assert np.array_equal(sent, got)
            assert sent.min() >= lay[r].own_start and sent.max() < lay[r].own_end


def _stencil(x):
    """Linear stand-in for a transport substep: each row becomes a weighted
    sum of the rows up to four away on either side (zero beyond the edges),
    per plane and column.  x: [planes][rows][cols]."""
    w = np.array([0.01, -0.03, 0.07, 0.2, 0.5, 0.15, -0.02, 0.05, 0.004])
    pad = np.pad(x, ((0, 0), (4, 4), (0, 0)))
    out = np.zeros_like(x)
    for k, wk in enumerate(w):
        out += wk * pad[:, k:k + x.shape[1]]
    return out


def _worker(rank, world, port, ny, out_path):
    import torch
    import torch.distributed as dist

    from paper_2504_00340_gb300.domain import exchange_halos
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        planes, nz = 3, 5
        glob = np.random.default_rng(7).random((planes, ny, nz))
        lay = split_rows(ny, world)
        me = lay[rank]
        local = torch.full((planes, me.ny, nz), float("nan"), dtype=torch.float64)
        own = slice(me.halo_lo, me.ny - me.halo_hi)
        local[:, own] = torch.from_numpy(glob[:, me.own_start:me.own_end])

        def pack(first, n):
            return local[:, first:first + n].contiguous()

        def unpack(first, n, buf):
            local[:, first:first + n] = buf.view(planes, n, nz)

        def alloc(n):
            return torch.empty((planes, n, nz), dtype=torch.float64)

        # one exchange fills the halos with the neighbours' rows of the grid
        exchange_halos(lay, rank, pack, unpack, alloc)
        filled = np.array_equal(local.numpy(), glob[:, me.y_offset:me.y_offset + me.ny])
        # a march of the stencil: exchange, apply (zero ghosts at the part's edges)
        ref = glob.copy()
        for _ in range(6):
            exchange_halos(lay, rank, pack, unpack, alloc)
            local[:] = torch.from_numpy(_stencil(local.numpy()))
            ref = _stencil(ref)
        mine = local.numpy()[:, own]
        gathered = [None] * world
        dist.all_gather_object(gathered, (filled, mine))
        if rank == 0:
            whole = np.concatenate([g[1] for g in gathered], axis=1)
            np.savez(out_path, filled=np.array([g[0] for g in gathered]), err=np.abs(whole - ref).max(),
                     scale=np.abs(ref).max())
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,ny", [(2, 20), (3, 27)])
def test_gloo_halo_exchange_reproduces_the_whole_grid(tmp_path, world, ny):
    import torch.multiprocessing as mp
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    out = str(tmp_path / "halo.npz")
    mp.spawn(_worker, args=(world, port, ny, out), nprocs=world, join=True)
    r = np.load(out)
    assert r["filled"].all()
    # the parts' own rows equal the undivided march to rounding (the
    # stencil's sums run in the same order on both sides)
    assert r["err"] <= 1e-15 * r["scale"]


def test_assemble_rows():
    lay = split_rows(13, 2)
    glob = np.arange(2 * 13 * 3, dtype=float).reshape(2, 13, 3)
    parts = [glob[:, x.y_offset:x.y_offset + x.ny] for x in lay]
    assert np.array_equal(assemble_rows(lay, parts), glob)
