"""Face exchange between the sub-domains of a cut lattice (lqcd_halo_*).

Sub-domain ranks are numbered lexicographically over their coordinates
(x fastest): rank = ((ct * pz + cz) * py + cy) * px + cx.  For every cut
direction mu a sub-domain sends its face segment (mu, 0) to its backward
neighbour and (mu, 1) to its forward neighbour (periodic), and receives its
segment (mu, 0) from the forward neighbour and (mu, 1) from the backward one
(include/lqcd.h, halo section).  The segments' offsets and lengths come
from lqcd_halo_layout.

This module moves bytes only: the faces are computed by lqcd_halo_pack and
consumed by lqcd_halo_dslash.  exchange() runs the transfers as
torch.distributed point-to-point operations (one process per sub-domain;
NCCL between GPUs, or gloo); exchange_local() copies between the buffers of
sub-domains held in one process (one GPU holding several sub-domains).
"""
from __future__ import annotations

import numpy as np


def rank_of(coord, part):
    """Rank of the sub-domain at coord (x fastest)."""
    r = 0
    for mu in (3, 2, 1, 0):
        r = r * max(1, part[mu]) + coord[mu]
    return r


def coord_of(rank, part):
    c = []
    for mu in range(4):
        p = max(1, part[mu])
        c.append(rank % p)
        rank //= p
    return tuple(c)


def neighbour(coord, part, mu, step):
    c = list(coord)
    c[mu] = (c[mu] + step) % max(1, part[mu])
    return rank_of(c, part)


def plan(coord, part):
    """Transfers of one sub-domain: a list of (mu, side, send_to, recv_from),
    send segment (mu, side) to rank send_to and receive segment (mu, side)
    from rank recv_from, in increasing mu and side."""
    out = []
    for mu in range(4):
        if max(1, part[mu]) < 2:
            continue
        fwd, bwd = neighbour(coord, part, mu, +1), neighbour(coord, part, mu, -1)
        out.append((mu, 0, bwd, fwd))
        out.append((mu, 1, fwd, bwd))
    return out


def _segment(buf, off, length, rhs, total):
    start = rhs * total + off
    return buf[start:start + length]


def exchange(send, recv, layout, coord, part, nrhs=1, group=None):
    """Point-to-point exchange of one sub-domain's faces: send, recv are its
    uint8 buffers (nrhs sets of layout[2] bytes), layout = lqcd_halo_layout's
    (offsets, lengths, total).  Every rank of the group calls it; the
    messages of one (mu, side) carry tag 2 mu + side (with two sub-domains
    along mu both neighbours are the same rank)."""
    import torch.distributed as dist
    off, ln, total = layout
    ops = []
    for mu, side, to, frm in plan(coord, part):
        k = 2 * mu + side
        for r in range(nrhs):
            tag = k + 8 * r
            ops.append(dist.P2POp(dist.isend, _segment(send, off[k], ln[k], r, total), to, group=group, tag=tag))
            ops.append(dist.P2POp(dist.irecv, _segment(recv, off[k], ln[k], r, total), frm, group=group, tag=tag))
    if ops:
        for req in dist.batch_isend_irecv(ops):
            req.wait()


def exchange_local(sends, recvs, layout, part, nrhs=1):
    """The same exchange among sub-domains held in one process: sends[rank],
    recvs[rank] are the buffers of every sub-domain (ranks as rank_of)."""
    off, ln, total = layout
    for rank in range(len(sends)):
        coord = coord_of(rank, part)
        for mu, side, to, frm in plan(coord, part):
            k = 2 * mu + side
            for r in range(nrhs):
                _segment(recvs[rank], off[k], ln[k], r, total).copy_(_segment(sends[frm], off[k], ln[k], r, total))


def split_field(field, part, coord):
    """The sub-domain's part of a canonical [t][z][y][x]... array (numpy)."""
    lt, lz, ly, lx = field.shape[:4]
    ext = (lx // max(1, part[0]), ly // max(1, part[1]), lz // max(1, part[2]), lt // max(1, part[3]))
    sl = tuple(slice(coord[mu] * ext[mu], (coord[mu] + 1) * ext[mu]) for mu in (3, 2, 1, 0))
    return np.ascontiguousarray(field[sl])


def local_dims(dims, part):
    return tuple(dims[mu] // max(1, part[mu]) for mu in range(4))
