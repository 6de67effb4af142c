"""Block decomposition (Sec. III-A) host logic on CPU: block extents and
neighbours, the halo layout, the halo exchange and the wave-speed reduction,
with world sizes 1, 2 and 4 over gloo.

Each block's packed sides are filled here from a global random array by this
file's own packer, written from the layout the library documents
(include/mfc.h: a segment per side with a neighbour, [field][layer][plane],
plane index x fastest; low side = the block's cells 0..2, high side = n-3..n-1).
After ``exchange_halos`` every halo segment must hold exactly the global
array's cells beyond that side (wrapped on periodic dimensions) -- the ghost
values the undecomposed grid reads there."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2409_10729_gb300 import decomp as D  # noqa: E402
from paper_2409_10729_gb300 import inputs as I  # noqa: E402

NF = 4   # fields per cell in these tests


def _cases():
    p3 = I.make_params(3, [10, 9, 7], [0.0] * 3, [1.0] * 3, [[1, 1], [0, 0], [0, 0]])
    p2 = I.make_params(2, [12, 8], [0.0] * 2, [1.0] * 2, [[1, 1], [1, 1]])
    p1 = I.make_params(1, [20], [0.0], [1.0], [[1, 1]])
    p3t = I.make_params(3, [8, 8, 9], [0.0] * 3, [1.0] * 3, I.TRANSMISSIVE)
    return [(p3, (2, 2, 1)), (p2, (2, 2)), (p1, (4,)), (p3t, (1, 2, 3)), (p2, (2, 1))]


def _global(p, seed=0):
    n = [int(p["n"][d]) if d < p["ndim"] else 1 for d in range(3)]
    return np.random.default_rng(seed).normal(size=(NF, n[2], n[1], n[0]))


def _layers(G, axis_d, idx, zyx):
    """Cells `idx` along dimension axis_d of G restricted to the block's other
    two ranges, as [field][layer][plane] flattened (plane x fastest)."""
    ax = 3 - axis_d
    sub = G[(slice(None),) + tuple(zyx[k] if k != ax - 1 else slice(None) for k in range(3))]
    return np.stack([np.take(sub, j, axis=ax) for j in idx], axis=1).reshape(-1)


def _block_ranges(b):
    return tuple(slice(b["lo"][2 - k], b["lo"][2 - k] + b["n"][2 - k]) for k in range(3))   # z, y, x


def _pack(grid, bid, G):
    b = grid.blocks[bid]
    _, tot = grid.layout(bid, NF)
    out = np.zeros(max(tot, 1))
    zyx = _block_ranges(b)
    for d in range(3):
        for s in (0, 1):
            if b["nbr"][d][s] is None:
                continue
            o, ln = grid.segment(bid, d, s, NF)
            idx = [b["lo"][d] + l for l in range(3)] if s == 0 else [b["lo"][d] + b["n"][d] - 3 + l for l in range(3)]
            out[o:o + ln] = _layers(G, d, idx, zyx)
    return out


def _expected_halo(grid, bid, G):
    b = grid.blocks[bid]
    _, tot = grid.layout(bid, NF)
    out = np.zeros(max(tot, 1))
    zyx = _block_ranges(b)
    for d in range(3):
        for s in (0, 1):
            if b["nbr"][d][s] is None:
                continue
            o, ln = grid.segment(bid, d, s, NF)
            idx = [b["lo"][d] - 3 + l for l in range(3)] if s == 0 else [b["lo"][d] + b["n"][d] + l for l in range(3)]
            idx = [j % grid.N[d] for j in idx]        # only periodic dimensions reach past the boundary
            out[o:o + ln] = _layers(G, d, idx, zyx)
    return out


def test_block_extents_neighbours_and_layout():
    p, counts = _cases()[0]                          # 10 x 9 x 7, periodic in x only, 2 x 2 x 1 blocks
    g = D.BlockGrid(p, counts)
    assert [b["n"] for b in g.blocks] == [[5, 5, 7], [5, 5, 7], [5, 4, 7], [5, 4, 7]]
    assert [b["lo"] for b in g.blocks] == [[0, 0, 0], [5, 0, 0], [0, 5, 0], [5, 5, 0]]
    b0 = g.blocks[0]
    assert b0["nbr"][0] == [1, 1]                     # periodic x: both sides are block 1
    assert b0["nbr"][1] == [None, 2]                  # transmissive y: low side is the domain boundary
    assert b0["nbr"][2] == [None, None]               # one block along z
    off, tot = g.layout(0, NF)
    # x sides: planes of 5 (y) x 7 (z); y high: 5 (x) x 7 (z); no y low, no z sides
    assert off == [0, NF * 3 * 35, -1, 2 * NF * 3 * 35, -1, -1]
    assert tot == 3 * NF * 3 * 35
    with pytest.raises(ValueError):
        D.BlockGrid(I.make_params(1, [5], [0.0], [1.0], [[0, 0]]), (2,))   # a 2-cell block with a neighbour


@pytest.mark.parametrize("case", range(5))
def test_single_process_exchange_fills_every_halo(case):
    p, counts = _cases()[case]
    g = D.BlockGrid(p, counts)
    G = _global(p, case)
    ids = range(len(g.blocks))
    packs = {b: torch.from_numpy(_pack(g, b, G)) for b in ids}
    halos = {b: torch.full_like(packs[b], float("nan")) for b in ids}
    D.exchange_halos(g, ids, packs, halos, NF, D.default_owner(len(g.blocks), 1), 0, None)
    for b in ids:
        assert np.array_equal(halos[b].numpy(), _expected_halo(g, b, G))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys
    import torch.distributed as dist
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    import test_decomp_cpu as T
    from paper_2409_10729_gb300 import decomp as D
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    group = dist.group.WORLD
    ok = []
    for case in range(5):
        p, counts = T._cases()[case]
        g = D.BlockGrid(p, counts)
        G = T._global(p, case)
        owner = D.default_owner(len(g.blocks), world)
        owned = [b for b in range(len(g.blocks)) if owner(b) == rank]
        packs = {b: torch.from_numpy(T._pack(g, b, G)) for b in owned}
        halos = {b: torch.full_like(packs[b], float("nan")) for b in owned}
        D.exchange_halos(g, owned, packs, halos, T.NF, owner, rank, group)
        ok.append(all(np.array_equal(halos[b].numpy(), T._expected_halo(g, b, G)) for b in owned))
    # the wave-speed reduction: every rank gets the max over all ranks' blocks
    s = D.global_max([1.0 + rank, 0.5 * rank], group)
    out.put((rank, ok, s))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
def test_multi_process_exchange_and_wave_speed_reduction(world):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    res = sorted(q.get(timeout=180) for _ in procs)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    for rank, ok, s in res:
        assert all(ok), f"rank {rank}: halo mismatch in cases {[i for i, v in enumerate(ok) if not v]}"
        assert s == float(world)                   # max over ranks of 1 + rank
