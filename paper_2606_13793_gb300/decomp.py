"""Spatial decomposition of one unigrid FMM solve over several ranks (z slabs).

A multi-GPU solve would give every rank a slab of leaf boxes along z and keep
each step local except for three exchanges, all fixed by the geometry of the
hierarchy (Sec. 2, Fig. 1):

* Near field (eq. direct): a cell's sources lie in the leaf boxes at Chebyshev
  distance <= 1 from its own, so a slab needs one leaf box (b cells) of density
  from each side.
* M2L (Sec. 2.2): the interaction list of a level-l box is made of children of
  its parent's 27 neighbours, so its sources lie within two level-l boxes of it
  along every axis; a slab needs two boxes of multipoles per level from each
  side, from whichever ranks own them.
* Coarse levels: below the split level the slabs would be thinner than a box.
  The split level's multipoles are all-gathered once, and every rank runs the
  levels above it whole (M2M, M2L and L2L), which costs little.

The slab boundaries are box boundaries of the split level, so every parent of
an owned box is owned and M2M / L2L never cross ranks.  This module holds the
plan only (index ranges and who sends what to whom); it does no arithmetic.
"""
from __future__ import annotations

from dataclasses import dataclass


def level_extents(shape, leaf):
    """Boxes per axis of every level, level 0 (root) first: the leaf grid is
    shape / leaf, each coarser level halves it rounding up (phantom boxes past
    the domain hold no mass)."""
    nx, ny, nz = (int(v) for v in shape)
    if leaf <= 0 or nx % leaf or ny % leaf or nz % leaf:
        raise ValueError("every axis must be a multiple of the leaf size")
    ext = [(nx // leaf, ny // leaf, nz // leaf)]
    while any(e > 1 for e in ext[-1]):
        ext.append(tuple((e + 1) // 2 for e in ext[-1]))
    return ext[::-1]


@dataclass(frozen=True)
class Transfer:
    """Boxes [lo, hi) along z of one level that rank `src` sends to rank `dst`."""
    level: int
    src: int
    dst: int
    lo: int
    hi: int


class SlabDecomposition:
    """z-slab plan for `world` ranks.

    split: the coarsest level with at least `world` boxes along z; its boxes are
    shared out in contiguous, balanced runs.  Levels finer than the split are
    distributed (each rank owns the boxes below its run), the split level is
    distributed for the upward pass and all-gathered afterwards, and coarser
    levels are replicated.
    """

    M2L_HALO = 2  # boxes: the interaction list reaches one parent box (two boxes) away
    NEAR_HALO = 1  # leaf boxes: the near field reaches the adjacent boxes

    def __init__(self, shape, leaf: int, world: int):
        if world < 1:
            raise ValueError("world must be >= 1")
        self.shape = tuple(int(v) for v in shape)
        self.leaf = int(leaf)
        self.world = int(world)
        self.ext = level_extents(self.shape, self.leaf)
        self.L = len(self.ext) - 1
        nz = [e[2] for e in self.ext]
        cand = [l for l in range(self.L + 1) if nz[l] >= self.world]
        if not cand:
            raise ValueError(f"{nz[self.L]} leaf boxes along z cannot be shared by {world} ranks")
        self.split = cand[0]
        n = nz[self.split]
        self._bounds = [(r * n) // self.world for r in range(self.world + 1)]

    # -- ownership -------------------------------------------------------------
    def owned(self, rank: int, level: int):
        """Owned box range [lo, hi) along z at `level` (the whole axis above the split)."""
        nz = self.ext[level][2]
        if level < self.split:
            return 0, nz
        f = 1 << (level - self.split)
        return min(self._bounds[rank] * f, nz), min(self._bounds[rank + 1] * f, nz)

    def owner(self, level: int, z: int) -> int:
        """Rank owning box row z of a distributed level (level >= split)."""
        for r in range(self.world):
            lo, hi = self.owned(r, level)
            if lo <= z < hi:
                return r
        raise ValueError(f"box {z} outside level {level}")

    def cells(self, rank: int):
        """Owned cell range [z0, z1) along z."""
        lo, hi = self.owned(rank, self.L)
        return lo * self.leaf, hi * self.leaf

    # -- exchanges ---------------------------------------------------------------
    def _halo_transfers(self, level: int, width: int):
        out = []
        nz = self.ext[level][2]
        for dst in range(self.world):
            lo, hi = self.owned(dst, level)
            if lo >= hi:
                continue
            want = set(range(max(0, lo - width), lo)) | set(range(hi, min(nz, hi + width)))
            for src in range(self.world):
                if src == dst:
                    continue
                slo, shi = self.owned(src, level)
                got = sorted(z for z in want if slo <= z < shi)
                # an owner's share of a halo is contiguous (slabs are contiguous runs)
                if got:
                    out.append(Transfer(level, src, dst, got[0], got[-1] + 1))
        return out

    def multipole_halos(self, level: int, width: int | None = None):
        """Transfers of multipole boxes the M2L of a distributed level needs
        (levels finer than the split; the split level itself is all-gathered)."""
        if level <= self.split:
            return []
        return self._halo_transfers(level, self.M2L_HALO if width is None else width)

    def density_halos(self, width: int | None = None):
        """Transfers of leaf boxes of density for the near field (in leaf boxes;
        multiply by the leaf size for cells)."""
        return self._halo_transfers(self.L, self.NEAR_HALO if width is None else width)

    def received_bytes(self, rank: int, ncoef: int, elem_bytes: int = 4, density_bytes: int = 4):
        """Bytes `rank` receives in one solve, by exchange: the density halo
        (cells of density_bytes), the multipole halos of each distributed level
        (ncoef coefficients of elem_bytes per box) and the all-gather of the
        split level (every box it does not own)."""
        nx, ny, _ = self.shape
        out = {"density": sum((t.hi - t.lo) * self.leaf * nx * ny * density_bytes
                              for t in self.density_halos() if t.dst == rank)}
        for l in range(self.L, self.split, -1):
            ex, ey, _ = self.ext[l]
            out[f"multipoles level {l}"] = sum((t.hi - t.lo) * ex * ey * ncoef * elem_bytes
                                               for t in self.multipole_halos(l) if t.dst == rank)
        ex, ey, ez = self.ext[self.split]
        lo, hi = self.owned(rank, self.split)
        out[f"allgather level {self.split}"] = (ez - (hi - lo)) * ex * ey * ncoef * elem_bytes
        return out

    def exchanges(self):
        """Every exchange of one solve, in order: density halos, multipole
        halos of each distributed level (finest first), then the all-gather of
        the split level."""
        steps = [("density", self.density_halos())]
        for l in range(self.L, self.split, -1):
            steps.append(("multipoles", self.multipole_halos(l)))
        steps.append(("allgather", self.split))
        return steps
