"""Spatial decomposition of one solve over ranks (z slabs), checked on CPU.

Each gloo rank holds only its slab of the density and runs the oracle's single
operators (P2M, M2M, M2L, L2L, L2P and the near-field sum of Sec. 2) on the
boxes it owns; everything else reaches it through the exchanges that
paper_2606_13793_gb300.decomp plans: density halos for the near field,
multipole halos of every level finer than the split level, and the all-gather
of the split level (coarser levels run whole on every rank).  The gathered
potential must equal the single-domain oracle solve to rounding.  Every value
a rank neither owns nor received is NaN, so a missing or too narrow exchange
cannot pass: with one box of multipole halo instead of two the solve fails.
"""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2606_13793_gb300 import decomp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _ilist(ext, level, i, j, k):
    """Interaction list of box (i, j, k) (Sec. 2.2): children of the parent's
    27 neighbours at Chebyshev distance >= 2, clipped to the level."""
    n = ext[level]
    pn = ext[level - 1]
    out = []
    for qk in range(k // 2 - 1, k // 2 + 2):
        for qj in range(j // 2 - 1, j // 2 + 2):
            for qi in range(i // 2 - 1, i // 2 + 2):
                if not (0 <= qi < pn[0] and 0 <= qj < pn[1] and 0 <= qk < pn[2]):
                    continue
                for c in range(8):
                    si, sj, sk = 2 * qi + (c & 1), 2 * qj + ((c >> 1) & 1), 2 * qk + (c >> 2)
                    if si >= n[0] or sj >= n[1] or sk >= n[2]:
                        continue
                    if max(abs(si - i), abs(sj - j), abs(sk - k)) >= 2:
                        out.append((si, sj, sk))
    return out


def _exchange(transfers, rank, arrays, scale=1):
    """Point-to-point copies of z-ranges [lo, hi) * scale of arrays[level]."""
    reqs, recv = [], []
    for t in transfers:
        a = arrays[t.level] if isinstance(arrays, dict) else arrays
        sl = slice(t.lo * scale, t.hi * scale)
        if t.src == rank:
            reqs.append(dist.isend(torch.from_numpy(np.ascontiguousarray(a[sl])), dst=t.dst))
        elif t.dst == rank:
            buf = torch.empty(a[sl].shape, dtype=torch.float64)
            reqs.append(dist.irecv(buf, src=t.src))
            recv.append((a, sl, buf))
    for r in reqs:
        r.wait()
    for a, sl, buf in recv:
        a[sl] = buf.numpy()


def _slab_solve(rank, world, port, shape, b, p, m2l_halo, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from paper_2606_13793_gb300 import inputs

    o = oracle.Oracle(oracle.load())
    D = decomp.SlabDecomposition(shape, b, world)
    ext, L, S = D.ext, D.L, D.split
    nc = o.ncoef(p)
    full = inputs.gaussian_blobs(shape, seed=31).astype(np.float64)  # [z][y][x]
    z0, z1 = D.cells(rank)
    rho = np.full_like(full, np.nan)
    rho[z0:z1] = full[z0:z1]
    _exchange(D.density_halos(), rank, rho, scale=b)

    def h(l):
        return b * (1 << (L - l))

    def centre(l, i, j, k):
        return np.array([(i + 0.5) * h(l), (j + 0.5) * h(l), (k + 0.5) * h(l)])

    def boxes(l, whole=False):
        lo, hi = (0, ext[l][2]) if whole else D.owned(rank, l)
        for k in range(lo, hi):
            for j in range(ext[l][1]):
                for i in range(ext[l][0]):
                    yield i, j, k

    # upward pass: P2M and M2M on the owned boxes down to the split level
    M = {l: np.full((ext[l][2], ext[l][1], ext[l][0], nc), np.nan) for l in range(L + 1)}
    for i, j, k in boxes(L):
        M[L][k, j, i] = o.p2m_region(rho, (i * b, j * b, k * b), (b, b, b), centre(L, i, j, k), p)

    def m2m_into(l, i, j, k):
        acc = np.zeros(nc)
        cp = centre(l, i, j, k)
        for c in range(8):
            si, sj, sk = 2 * i + (c & 1), 2 * j + ((c >> 1) & 1), 2 * k + (c >> 2)
            if si < ext[l + 1][0] and sj < ext[l + 1][1] and sk < ext[l + 1][2]:
                acc += o.m2m(M[l + 1][sk, sj, si], centre(l + 1, si, sj, sk) - cp, p)
        M[l][k, j, i] = acc

    for l in range(L - 1, S - 1, -1):
        for box in boxes(l):
            m2m_into(l, *box)
    # all-gather of the split level, then the coarse levels whole
    for r in range(world):
        lo, hi = D.owned(r, S)
        t = torch.from_numpy(np.ascontiguousarray(M[S][lo:hi]))
        dist.broadcast(t, src=r)
        M[S][lo:hi] = t.numpy()
    for l in range(S - 1, -1, -1):
        for box in boxes(l, whole=True):
            m2m_into(l, *box)
    # multipole halos of the distributed levels
    for l in range(L, S, -1):
        _exchange(D.multipole_halos(l, width=m2l_halo), rank, M)

    # downward pass: coarse levels whole, then the owned boxes
    Lx = {0: np.zeros((1, 1, 1, nc))}
    for l in range(1, L + 1):
        Lx[l] = np.full((ext[l][2], ext[l][1], ext[l][0], nc), np.nan)
        for i, j, k in boxes(l, whole=l < S):
            ct = centre(l, i, j, k)
            acc = o.l2l(Lx[l - 1][k // 2, j // 2, i // 2], ct - centre(l - 1, i // 2, j // 2, k // 2), p)
            for si, sj, sk in _ilist(ext, l, i, j, k):
                acc += o.m2l(M[l][sk, sj, si], ct - centre(l, si, sj, sk), p)
            Lx[l][k, j, i] = acc

    # leaf: L2P plus the near field over the adjacent leaf boxes (eq. direct)
    nz, ny, nx = full.shape
    phi = np.zeros((z1 - z0, ny, nx))
    cz, cy, cx = np.meshgrid(np.arange(b), np.arange(b), np.arange(b), indexing="ij")
    for i, j, k in boxes(L):
        c = centre(L, i, j, k)
        zl, zh = max(0, (k - 1) * b), min(nz, (k + 2) * b)
        yl, yh = max(0, (j - 1) * b), min(ny, (j + 2) * b)
        xl, xh = max(0, (i - 1) * b), min(nx, (i + 2) * b)
        src = rho[zl:zh, yl:yh, xl:xh]
        sz, sy, sx = np.meshgrid(np.arange(zl, zh), np.arange(yl, yh), np.arange(xl, xh), indexing="ij")
        for z, y, x in zip(cz.ravel() + k * b, cy.ravel() + j * b, cx.ravel() + i * b):
            r = np.sqrt((x - sx) ** 2 + (y - sy) ** 2 + (z - sz) ** 2)
            g = np.where(r <= 1.0, -1.0, -1.0 / np.maximum(r, 1.0))
            far = o.l2p(Lx[L][k, j, i], np.array([x + 0.5, y + 0.5, z + 0.5]) - c, p)
            phi[z - z0, y, x] = far + float(np.sum(src * g))

    # gather on rank 0 and compare with the single-domain solve
    whole = np.zeros_like(full)
    for r in range(world):
        a, e = D.cells(r)
        t = torch.from_numpy(np.ascontiguousarray(phi)) if r == rank else torch.empty((e - a, ny, nx),
                                                                                      dtype=torch.float64)
        dist.broadcast(t, src=r)
        whole[a:e] = t.numpy()
    if rank == 0:
        ref = o.fmm(full, b, p)["phi"]
        finite = bool(np.all(np.isfinite(whole)))
        err = float(np.max(np.abs(whole - ref)) / np.max(np.abs(ref))) if finite else float("nan")
        out["result"] = (finite, err, S, L)
    dist.barrier()
    dist.destroy_process_group()


def _run(world, shape=(24, 20, 40), b=4, p=4, m2l_halo=None):
    import oracle

    oracle.load()  # built once here, before the ranks load it
    with mp.get_context("spawn").Manager() as mgr:  # no fork of a threaded process
        out = mgr.dict()
        mp.spawn(_slab_solve, args=(world, _free_port(), shape, b, p, m2l_halo, out), nprocs=world, join=True)
        return out["result"]


def test_plan_geometry():
    D = decomp.SlabDecomposition((24, 20, 40), 4, 3)
    assert [e[2] for e in D.ext] == [1, 2, 3, 5, 10] and D.split == 2
    assert [D.owned(r, 4) for r in range(3)] == [(0, 4), (4, 8), (8, 10)]
    assert [D.owned(r, 1) for r in range(3)] == [(0, 2)] * 3  # replicated above the split
    assert [D.cells(r) for r in range(3)] == [(0, 16), (16, 32), (32, 40)]
    # every owned box's parent is owned (M2M and L2L stay local)
    for r in range(3):
        for l in range(D.split + 1, D.L + 1):
            lo, hi = D.owned(r, l)
            plo, phi_ = D.owned(r, l - 1)
            assert plo <= lo // 2 and (hi - 1) // 2 < phi_
    # halos: two boxes each side per distributed level, from their owners
    t = {(x.src, x.dst): (x.lo, x.hi) for x in D.multipole_halos(4)}
    assert t == {(1, 0): (4, 6), (0, 1): (2, 4), (2, 1): (8, 10), (1, 2): (6, 8)}
    assert D.multipole_halos(D.split) == []
    assert {(x.src, x.dst): (x.lo, x.hi) for x in D.density_halos()} == {
        (1, 0): (4, 5), (0, 1): (3, 4), (2, 1): (8, 9), (1, 2): (7, 8)}
    # odd extents: the last slab is clipped to the boxes that exist
    D9 = decomp.SlabDecomposition((8, 8, 36), 4, 3)
    assert [e[2] for e in D9.ext] == [1, 2, 3, 5, 9] and D9.split == 2
    assert [D9.owned(r, 4) for r in range(3)] == [(0, 4), (4, 8), (8, 9)]
    assert {(x.src, x.dst): (x.lo, x.hi) for x in D9.multipole_halos(4) if x.dst == 2} == {(1, 2): (6, 8)}
    assert {(x.src, x.dst): (x.lo, x.hi) for x in D9.multipole_halos(3) if x.dst == 1} == {
        (0, 1): (0, 2), (2, 1): (4, 5)}


def test_received_bytes_count_the_halo_boxes():
    D = decomp.SlabDecomposition((24, 20, 40), 4, 3)  # leaf boxes 6 x 5 x 10, split level 2
    nc = 35
    for r in range(3):
        got = D.received_bytes(r, nc, elem_bytes=8, density_bytes=8)
        lo, hi = D.cells(r)
        # density: the cells within one leaf box (4 cells) of the slab, along z
        cells = len([z for z in range(40) if (lo - 4 <= z < lo) or (hi <= z < hi + 4)])
        assert got["density"] == cells * 24 * 20 * 8
        for l in (4, 3):
            blo, bhi = D.owned(r, l)
            nz = D.ext[l][2]
            boxes = len([z for z in range(nz) if (blo - 2 <= z < blo) or (bhi <= z < bhi + 2)])
            assert got[f"multipoles level {l}"] == boxes * D.ext[l][0] * D.ext[l][1] * nc * 8
        slo, shi = D.owned(r, 2)
        assert got["allgather level 2"] == (D.ext[2][2] - (shi - slo)) * D.ext[2][0] * D.ext[2][1] * nc * 8


@pytest.mark.parametrize("world", [2, 3, 4])
def test_slab_solve_equals_single_domain(world):
    finite, err, split, L = _run(world)
    print(f"{world} ranks: split level {split} of {L}, max |phi - phi_single| / max |phi| = {err:.2e}")
    assert finite and err <= 1e-12


def test_one_box_multipole_halo_is_not_enough():
    finite, err, _, _ = _run(2, m2l_halo=1)
    assert not finite or err > 1e-6
