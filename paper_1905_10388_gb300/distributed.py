"""Pencil distribution over ranks: layouts and the grouped transposes between
them (Sec. "Distributor / Layout": the data of one transform is distributed
so that the axis being transformed is local, and a global transpose moves
between layouts; all fields of one right-hand-side evaluation travel in one
exchange).

Two layouts of a two-dimensional problem with P = N_x / 2 stored k_x modes
(pencils) and N_gz dealiased z points, over W ranks:

* pencil layout (coefficients, Chebyshev transforms, pencil solves): rank r
  holds the pencils [p0_r, p1_r), a balanced block of k_x, with every
  Chebyshev mode or z point -- the z axis is local;
* row layout (Fourier x transforms, products on the grid): rank r holds the
  z rows [z0_r, z1_r) of the dealiased grid with every k_x -- the x axis is
  local.

The buffers follow the library's z-transformed layout ``[field][z][pencil]``
(complex): the z kernels write ``[f][N_gz][P_r]`` for their own pencils, the
x-row kernel reads ``[f][rows_r][P]``.  One right-hand-side evaluation is

    z backward (pencil layout) -> to_rows (all fields, one all-to-all)
    -> x backward, products, x forward (row layout)
    -> to_pencils (all products, one all-to-all) -> z forward, pencil solves.

Each rank sends every other rank one contiguous block per exchange, whose
size follows from the two block partitions; packing copies the slices into
one send buffer ordered by destination, unpacking scatters the received
blocks.  The pencil solves need no communication (each pencil is local).
The exchange runs through ``torch.distributed.all_to_all_single`` (NCCL
between GPUs, gloo between CPU ranks); complex data travel as pairs of
reals.  This module holds the index logic and the exchange only; the
transforms on either side are the library's kernels on each rank's GPU.
"""
import numpy as np


def block_range(n, world, rank):
    """[start, stop) of rank's block of a balanced partition of n items (the
    first n mod world ranks get one item more)."""
    base, extra = divmod(int(n), int(world))
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


class PencilLayout:
    def __init__(self, n_pencils, n_rows, world):
        self.P, self.R, self.W = int(n_pencils), int(n_rows), int(world)
        self.pencils = [block_range(self.P, self.W, r) for r in range(self.W)]
        self.rows = [block_range(self.R, self.W, r) for r in range(self.W)]

    def n_pencils(self, rank):
        p0, p1 = self.pencils[rank]
        return p1 - p0

    def n_rows(self, rank):
        z0, z1 = self.rows[rank]
        return z1 - z0

    # -- pencil layout -> row layout ------------------------------------------
    def split_to_rows(self, rank, nf):
        """Element counts (complex) sent to / received from each rank."""
        send = [nf * self.n_rows(d) * self.n_pencils(rank) for d in range(self.W)]
        recv = [nf * self.n_rows(rank) * self.n_pencils(s) for s in range(self.W)]
        return send, recv

    def pack_to_rows(self, rank, local):
        """local [nf][R][P_rank] -> send buffer: destination d's z rows, in
        destination order, each block [nf][rows_d][P_rank] contiguous."""
        parts = [local[:, z0:z1, :].reshape(-1) for (z0, z1) in self.rows]
        return _cat(parts, local)

    def unpack_to_rows(self, rank, recv, nf):
        """Received blocks (source s: [nf][rows_rank][P_s]) -> [nf][rows_rank][P]."""
        nr = self.n_rows(rank)
        out = _empty(recv, (nf, nr, self.P))
        off = 0
        for s, (p0, p1) in enumerate(self.pencils):
            cnt = nf * nr * (p1 - p0)
            out[:, :, p0:p1] = recv[off:off + cnt].reshape(nf, nr, p1 - p0)
            off += cnt
        return out

    # -- row layout -> pencil layout ------------------------------------------
    def split_to_pencils(self, rank, ne):
        send = [ne * self.n_rows(rank) * self.n_pencils(d) for d in range(self.W)]
        recv = [ne * self.n_rows(s) * self.n_pencils(rank) for s in range(self.W)]
        return send, recv

    def pack_to_pencils(self, rank, rows_local):
        """rows_local [ne][rows_rank][P] -> send buffer: destination d's
        pencils, each block [ne][rows_rank][P_d] contiguous."""
        parts = [rows_local[:, :, p0:p1].reshape(-1) for (p0, p1) in self.pencils]
        return _cat(parts, rows_local)

    def unpack_to_pencils(self, rank, recv, ne):
        """Received blocks (source s: [ne][rows_s][P_rank]) -> [ne][R][P_rank]."""
        npr = self.n_pencils(rank)
        out = _empty(recv, (ne, self.R, npr))
        off = 0
        for s, (z0, z1) in enumerate(self.rows):
            cnt = ne * (z1 - z0) * npr
            out[:, z0:z1, :] = recv[off:off + cnt].reshape(ne, z1 - z0, npr)
            off += cnt
        return out


def _cat(parts, like):
    if isinstance(like, np.ndarray):
        return np.concatenate(parts)
    import torch
    return torch.cat(parts)


def _empty(like, shape):
    if isinstance(like, np.ndarray):
        return np.empty(shape, dtype=like.dtype)
    import torch
    return torch.empty(shape, dtype=like.dtype, device=like.device)


def _exchange(send, send_counts, recv_counts, group=None):
    """all-to-all of a complex torch buffer with per-rank element counts."""
    import torch
    import torch.distributed as dist
    s = torch.view_as_real(send.contiguous()).reshape(-1)
    r = torch.empty(2 * sum(recv_counts), dtype=s.dtype, device=s.device)
    dist.all_to_all_single(r, s, output_split_sizes=[2 * c for c in recv_counts],
                           input_split_sizes=[2 * c for c in send_counts], group=group)
    return torch.view_as_complex(r.reshape(-1, 2))


def to_rows(layout, rank, local, group=None):
    """Grouped transpose, pencil layout -> row layout, of all nf fields in
    ``local`` [nf][R][P_rank] (complex torch tensor): one all-to-all."""
    nf = local.shape[0]
    send, recv = layout.split_to_rows(rank, nf)
    got = _exchange(layout.pack_to_rows(rank, local), send, recv, group)
    return layout.unpack_to_rows(rank, got, nf)


def to_pencils(layout, rank, rows_local, group=None):
    """Grouped transpose, row layout -> pencil layout, of all ne fields in
    ``rows_local`` [ne][rows_rank][P]: one all-to-all."""
    ne = rows_local.shape[0]
    send, recv = layout.split_to_pencils(rank, ne)
    got = _exchange(layout.pack_to_pencils(rank, rows_local), send, recv, group)
    return layout.unpack_to_pencils(rank, got, ne)
