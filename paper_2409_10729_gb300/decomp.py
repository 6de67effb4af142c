"""Block decomposition of the grid (arXiv 2409.10729, Sec. III-A).

The global grid is cut into a Cartesian arrangement of blocks, one library
context per block (``mfc_create_block``).  A block needs three ghost layers of
the stage state beyond every side that borders another block; they are
exchanged once per SSP-RK3 stage, and every step's dt = CFL / S uses the wave
speed S reduced (max) over all blocks.  This module holds the host side of
that exchange:

* ``BlockGrid`` -- the blocks' extents and neighbours, and the halo layout
  the library uses (one segment per side with a neighbour, in the order
  x low, x high, y low, y high, z low, z high; a segment is
  [field][layer 0..2][plane]);
* ``exchange_halos`` -- hands each packed side to the facing halo segment of
  the neighbour: a device-to-device copy when both blocks live in this
  process, a point-to-point message (``torch.distributed``: NCCL between GPUs,
  gloo between CPU processes) otherwise;
* ``global_max`` -- the wave-speed reduction over blocks and processes;
* ``DecomposedSolver`` -- steps a decomposed grid: begin step, then per stage
  pack -> exchange -> sweeps, all of whose arithmetic runs in the library's
  kernels.

The result is bit-identical to the undecomposed grid's: a cell's update
depends only on its stencil cells and on dt, and every block reads at its
ghost positions exactly the values the undecomposed grid holds there.
"""
from __future__ import annotations

import numpy as np


def split_extent(n: int, parts: int):
    """Start indices and sizes of `parts` nearly equal pieces of n cells."""
    base, extra = divmod(n, parts)
    sizes = [base + (1 if i < extra else 0) for i in range(parts)]
    starts = [sum(sizes[:i]) for i in range(parts)]
    return starts, sizes


class BlockGrid:
    """Blocks of the grid of params dict ``p`` with ``counts[d]`` blocks along
    dimension d (missing or beyond ndim: 1)."""

    def __init__(self, p: dict, counts):
        self.p = p
        self.ndim = int(p["ndim"])
        self.N = [int(p["n"][d]) if d < self.ndim else 1 for d in range(3)]
        self.counts = [int(counts[d]) if d < len(counts) and d < self.ndim else 1 for d in range(3)]
        self.periodic = [d < self.ndim and int(p["bc"][d][0]) == 1 for d in range(3)]
        ext = [split_extent(self.N[d], self.counts[d]) for d in range(3)]
        self.blocks = []
        for k in range(self.counts[2]):
            for j in range(self.counts[1]):
                for i in range(self.counts[0]):
                    c = (i, j, k)
                    lo = [ext[d][0][c[d]] for d in range(3)]
                    n = [ext[d][1][c[d]] for d in range(3)]
                    self.blocks.append({"id": len(self.blocks), "coord": c, "lo": lo, "n": n})
        for b in self.blocks:
            b["nbr"] = [[self._neighbour(b, d, s) for s in (0, 1)] for d in range(3)]
            for d in range(3):
                if (b["nbr"][d][0] is not None or b["nbr"][d][1] is not None) and b["n"][d] < 3:
                    raise ValueError(f"block {b['id']} has {b['n'][d]} cells along dimension {d}: "
                                     "a block with a neighbour needs at least 3")

    def _index(self, c):
        return c[0] + self.counts[0] * (c[1] + self.counts[1] * c[2])

    def _neighbour(self, b, d, s):
        """Id of the block beyond side s of dimension d, or None where the BC
        applies (non-periodic boundary, or one block spanning a periodic
        dimension, which wraps onto itself)."""
        if d >= self.ndim or self.counts[d] == 1:
            return None
        c = list(b["coord"])
        c[d] += 1 if s else -1
        if c[d] < 0 or c[d] >= self.counts[d]:
            if not self.periodic[d]:
                return None
            c[d] %= self.counts[d]
        return self._index(c)

    def layout(self, bid: int, nfields: int):
        """Element offsets of the six side segments (-1 where no neighbour) and
        the total, as mfc_halo_layout reports them."""
        b = self.blocks[bid]
        cells = b["n"][0] * b["n"][1] * b["n"][2]
        off, tot = [], 0
        for d in range(3):
            for s in (0, 1):
                if b["nbr"][d][s] is None:
                    off.append(-1)
                else:
                    off.append(tot)
                    tot += nfields * 3 * (cells // b["n"][d])
        return off, tot

    def segment(self, bid: int, d: int, s: int, nfields: int):
        """(start, length) of side (d, s)'s segment of block bid."""
        off, _ = self.layout(bid, nfields)
        b = self.blocks[bid]
        cells = b["n"][0] * b["n"][1] * b["n"][2]
        return off[2 * d + s], nfields * 3 * (cells // b["n"][d])

    def slices(self, bid: int):
        """numpy index of the block's cells in a global [field][z][y][x] array."""
        b = self.blocks[bid]
        return (slice(None), slice(b["lo"][2], b["lo"][2] + b["n"][2]), slice(b["lo"][1], b["lo"][1] + b["n"][1]),
                slice(b["lo"][0], b["lo"][0] + b["n"][0]))


def default_owner(nblocks: int, world: int):
    """Contiguous runs of block ids per process."""
    return lambda bid: bid * world // nblocks


def exchange_halos(grid: BlockGrid, owned, packs: dict, halos: dict, nfields: int, owner, rank: int = 0,
                   group=None):
    """Fill the halo buffers of the blocks in ``owned`` from their neighbours'
    packed sides.  packs[b], halos[b] (1-D tensors in the halo layout) exist
    for every owned block b.  Side (d, s) of block b receives the packed side
    (d, 1 - s) of the neighbour beyond it: copied when that neighbour is owned
    here, else received from its owner, which sends it.  Message tags name
    the receiving segment (6 b + 2 d + s), so every pair of blocks, however
    many sides they share (two blocks along a periodic dimension share two),
    exchanges unambiguously."""
    owned = list(owned)
    local = set(owned)
    reqs = []
    if group is not None or any(owner(nb) != rank for b in owned for d in range(3) for nb in grid.blocks[b]["nbr"][d]
                                if nb is not None):
        import torch.distributed as dist
        for b in owned:   # receives first, then sends: both non-blocking
            for d in range(3):
                for s in (0, 1):
                    nb = grid.blocks[b]["nbr"][d][s]
                    if nb is None or nb in local:
                        continue
                    o, ln = grid.segment(b, d, s, nfields)
                    reqs.append(dist.irecv(halos[b][o:o + ln], src=owner(nb), group=group, tag=6 * b + 2 * d + s))
        for b in owned:
            for d in range(3):
                for s in (0, 1):
                    nb = grid.blocks[b]["nbr"][d][s]
                    if nb is None or nb in local:
                        continue
                    o, ln = grid.segment(b, d, s, nfields)
                    reqs.append(dist.isend(packs[b][o:o + ln], dst=owner(nb), group=group,
                                           tag=6 * nb + 2 * d + (1 - s)))
    for b in owned:
        for d in range(3):
            for s in (0, 1):
                nb = grid.blocks[b]["nbr"][d][s]
                if nb is None or nb not in local:
                    continue
                o, ln = grid.segment(b, d, s, nfields)
                so, sl = grid.segment(nb, d, 1 - s, nfields)
                assert sl == ln
                halos[b][o:o + ln].copy_(packs[nb][so:so + sl])
    for r in reqs:
        r.wait()


def global_max(values, group=None, device=None) -> float:
    """Max of this process's values and, with a process group, of every
    process's (all-reduce MAX)."""
    m = max(float(v) for v in values) if len(values) else 0.0
    if group is None:
        return m
    import torch
    import torch.distributed as dist
    t = torch.tensor([m], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


class DecomposedSolver:
    """SSP-RK3 on a block-decomposed grid: the blocks of ``counts`` owned by
    this process (all of them without a process group) each in its own
    context on the current CUDA device."""

    def __init__(self, p: dict, counts, precision="fp64", group=None, owner=None):
        import torch

        from . import mfc
        self.grid = BlockGrid(p, counts)
        self.p = p
        self.group = group
        if group is not None:
            import torch.distributed as dist
            self.rank, self.world = dist.get_rank(group), dist.get_world_size(group)
        else:
            self.rank, self.world = 0, 1
        nb = len(self.grid.blocks)
        self.owner = owner or default_owner(nb, self.world)
        self.owned = [b for b in range(nb) if self.owner(b) == self.rank]
        self.solvers, self.packs, self.halos = {}, {}, {}
        for b in self.owned:
            blk = self.grid.blocks[b]
            s = mfc.Solver(p, precision, block=(blk["lo"], blk["n"]))
            off, tot, el = s.halo_layout()
            nfields = s.neq + (1 if el == 4 else 0)
            exp_off, exp_tot = self.grid.layout(b, nfields)
            if off != exp_off or tot != exp_tot:
                raise RuntimeError(f"halo layout of block {b}: library {off, tot}, expected {exp_off, exp_tot}")
            dt = torch.float64 if el == 8 else torch.float32
            self.solvers[b] = s
            self.packs[b] = torch.empty(max(tot, 1), dtype=dt, device="cuda")
            self.halos[b] = torch.empty(max(tot, 1), dtype=dt, device="cuda")
            self.nfields = nfields
        self.neq = 2 * len(p["gamma"]) + int(p["ndim"])
        self.nonphysical = False

    def close(self):
        for s in self.solvers.values():
            s.close()
        self.solvers = {}

    # -- state ---------------------------------------------------------------
    def set_state_prim(self, w):
        for b, s in self.solvers.items():
            s.set_state_prim(np.ascontiguousarray(w[self.grid.slices(b)]))

    def set_state(self, q):
        for b, s in self.solvers.items():
            s.set_state(np.ascontiguousarray(q[self.grid.slices(b)]))

    def set_mlp_weights(self, w):
        for s in self.solvers.values():
            s.set_mlp_weights(w)

    def get_blocks(self):
        """{block id: its state} of the blocks owned here."""
        return {b: s.get_state() for b, s in self.solvers.items()}

    def get_state(self):
        """The global state assembled from every block (all blocks must be
        owned by this process)."""
        if len(self.owned) != len(self.grid.blocks):
            raise RuntimeError("get_state needs every block in this process; use get_blocks")
        nz, ny, nx = self.grid.N[2], self.grid.N[1], self.grid.N[0]
        q = np.empty((self.neq, nz, ny, nx))
        for b, qb in self.get_blocks().items():
            q[self.grid.slices(b)] = qb
        return q

    # -- stepping --------------------------------------------------------------
    def _exchange(self, stage: int):
        for b, s in self.solvers.items():
            s.block_pack(stage, self.packs[b])
        exchange_halos(self.grid, self.owned, self.packs, self.halos, self.nfields, self.owner, self.rank,
                       self.group)

    def wavespeed(self) -> float:
        vals = []
        for s in self.solvers.values():
            v, st = s.block_wavespeed(allow_nonphysical=True)
            self.nonphysical |= st != 0
            vals.append(v)
        return global_max(vals, self.group, "cuda" if self._nccl() else "cpu")

    def _nccl(self):
        if self.group is None:
            return False
        import torch.distributed as dist
        return dist.get_backend(self.group) == "nccl"

    def step_rk3(self, cfl: float, nsteps: int, allow_nonphysical=False) -> float:
        """nsteps steps, each with dt = cfl / S(q^n) over all blocks; returns
        the time advanced (the dt summed in step order)."""
        t = 0.0
        for _ in range(nsteps):
            S = self.wavespeed()
            dt = cfl / S
            for s in self.solvers.values():
                s.block_begin_step(dt)
            for k in (1, 2, 3):
                self._exchange(k)
                for b, s in self.solvers.items():
                    s.block_stage(k, self.halos[b])
            t += dt
        self.wavespeed()   # the status of the last step
        if self.nonphysical and not allow_nonphysical:
            from . import mfc
            raise mfc.MfcError(mfc.MFC_ENONPHYSICAL, "DecomposedSolver.step_rk3")
        return t

    def rhs_blocks(self):
        """{block id: L(q^n) of the block} for the blocks owned here."""
        self._exchange(1)
        return {b: s.block_rhs(self.halos[b]) for b, s in self.solvers.items()}

    def rhs(self):
        nz, ny, nx = self.grid.N[2], self.grid.N[1], self.grid.N[0]
        L = np.empty((self.neq, nz, ny, nx))
        for b, Lb in self.rhs_blocks().items():
            L[self.grid.slices(b)] = Lb
        return L
