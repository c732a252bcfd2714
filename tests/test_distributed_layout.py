"""The pencil distribution (paper_1905_10388_gb300.distributed) on CPU ranks.

* index logic, in one process for 1, 2, 3 and 5 simulated ranks with uneven
  blocks: packing on every rank, routing the blocks as an all-to-all would,
  and unpacking reproduce the global arrays exactly in both directions;
* two gloo ranks (world size 2, uneven: 15 pencils, 45 dealiased z rows):
  the distributed backward transform -- Chebyshev z per local pencil, one
  grouped transpose of all fields, Fourier x per local row -- gathered on
  rank 0 equals the single-rank transform bit for bit, and the forward
  transform back through the other transpose returns the single-rank
  coefficients bit for bit.  The local one-dimensional transforms are the
  oracle's (test infrastructure), applied column by column on both sides,
  so that only the layout, packing and exchange are under test.

Not run on GPUs here (one GPU per machine in this environment): the
exchange then goes through NCCL with the same code.
"""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1905_10388_gb300.distributed import PencilLayout, block_range

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_block_ranges_partition():
    for n in (0, 1, 7, 15, 45, 256):
        for w in (1, 2, 3, 5, 8):
            rs = [block_range(n, w, r) for r in range(w)]
            assert rs[0][0] == 0 and rs[-1][1] == n
            assert all(rs[i][1] == rs[i + 1][0] for i in range(w - 1))
            sizes = [b - a for a, b in rs]
            assert max(sizes) - min(sizes) <= 1


@pytest.mark.parametrize("world", [1, 2, 3, 5])
def test_pack_route_unpack_round_trip(world):
    P, R, nf = 15, 45, 4
    rng = np.random.default_rng(world)
    full = rng.standard_normal((nf, R, P)) + 1j * rng.standard_normal((nf, R, P))
    lay = PencilLayout(P, R, world)
    # pencil layout -> row layout
    sends = []
    for r in range(world):
        p0, p1 = lay.pencils[r]
        sends.append(lay.pack_to_rows(r, full[:, :, p0:p1].copy()))
    for r in range(world):
        recv = []
        for s in range(world):
            cnt_s, _ = lay.split_to_rows(s, nf)
            off = sum(cnt_s[:r])
            recv.append(sends[s][off:off + cnt_s[r]])
        rows = lay.unpack_to_rows(r, np.concatenate(recv), nf)
        z0, z1 = lay.rows[r]
        assert np.array_equal(rows, full[:, z0:z1, :])
    # row layout -> pencil layout
    sends = []
    for r in range(world):
        z0, z1 = lay.rows[r]
        sends.append(lay.pack_to_pencils(r, full[:, z0:z1, :].copy()))
    for r in range(world):
        recv = []
        for s in range(world):
            cnt_s, _ = lay.split_to_pencils(s, nf)
            off = sum(cnt_s[:r])
            recv.append(sends[s][off:off + cnt_s[r]])
        pen = lay.unpack_to_pencils(r, np.concatenate(recv), nf)
        p0, p1 = lay.pencils[r]
        assert np.array_equal(pen, full[:, :, p0:p1])


# --- two gloo ranks ---------------------------------------------------------------

NX, NZ, NF = 30, 30, 3          # P = 15 pencils, N_gz = 45 rows, N_gx = 45


def _z_backward(c_p, ngz):
    from oracle import bases
    return bases.chebyshev_backward(c_p, ngz)


def _x_backward(row, ngx):
    from oracle import bases
    return bases.fourier_backward(row, ngx)


def _x_forward(grow, nx):
    from oracle import bases
    return bases.fourier_forward(grow, nx)


def _z_forward(col, nz):
    from oracle import bases
    return bases.chebyshev_forward(col, nz)


def _coefficients():
    rng = np.random.default_rng(11)
    c = rng.standard_normal((NF, NX // 2, NZ)) + 1j * rng.standard_normal((NF, NX // 2, NZ))
    c[:, 0, :] = c[:, 0, :].real
    return c


def _single_rank(c):
    """Column by column: z backward per pencil, x backward per row, and back."""
    P, ngz, ngx = NX // 2, 3 * NZ // 2, 3 * NX // 2
    gz = np.empty((NF, ngz, P), complex)
    for f in range(NF):
        for p in range(P):
            gz[f, :, p] = _z_backward(c[f, p], ngz)
    g = np.empty((NF, ngz, ngx))
    for f in range(NF):
        for z in range(ngz):
            g[f, z] = _x_backward(gz[f, z], ngx)
    h = np.empty((NF, ngz, P), complex)
    for f in range(NF):
        for z in range(ngz):
            h[f, z] = _x_forward(g[f, z], NX)
    back = np.empty((NF, P, NZ), complex)
    for f in range(NF):
        for p in range(P):
            back[f, p] = _z_forward(h[f, :, p], NZ)
    return g, back


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1905_10388_gb300.distributed import PencilLayout, to_pencils, to_rows
    P, ngz, ngx = NX // 2, 3 * NZ // 2, 3 * NX // 2
    lay = PencilLayout(P, ngz, world)
    c = _coefficients()
    p0, p1 = lay.pencils[rank]
    z0, z1 = lay.rows[rank]
    # pencil layout: z backward of the local pencils
    gz = np.empty((NF, ngz, p1 - p0), complex)
    for f in range(NF):
        for i, p in enumerate(range(p0, p1)):
            gz[f, :, i] = _z_backward(c[f, p], ngz)
    rows = to_rows(lay, rank, torch.from_numpy(gz)).numpy()          # [NF][rows][P]
    g = np.empty((NF, z1 - z0, ngx))
    for f in range(NF):
        for i in range(z1 - z0):
            g[f, i] = _x_backward(rows[f, i], ngx)
    # forward: x per local row, transpose back, z per local pencil
    h = np.empty((NF, z1 - z0, P), complex)
    for f in range(NF):
        for i in range(z1 - z0):
            h[f, i] = _x_forward(g[f, i], NX)
    hp = to_pencils(lay, rank, torch.from_numpy(h)).numpy()           # [NF][ngz][P_r]
    back = np.empty((NF, p1 - p0, NZ), complex)
    for f in range(NF):
        for i in range(p1 - p0):
            back[f, i] = _z_forward(hp[f, :, i], NZ)
    q.put((rank, (z0, z1), g, (p0, p1), back))
    dist.destroy_process_group()


def test_two_gloo_ranks_reassemble_the_single_rank_transforms():
    world = 2
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get() for _ in range(world)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    g_ref, back_ref = _single_rank(_coefficients())
    g = np.empty_like(g_ref)
    back = np.empty_like(back_ref)
    for rank, (z0, z1), gr, (p0, p1), br in res:
        g[:, z0:z1] = gr
        back[:, p0:p1] = br
    assert np.array_equal(g, g_ref)
    assert np.array_equal(back, back_ref)
