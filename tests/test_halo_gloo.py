"""The face exchange of a cut lattice (paper_1103_1363_gb300.halo) with one
gloo process per sub-domain on the CPU: 2 sub-domains along t and 2 x 2
along z and t.  Every rank fills its send segments with a pattern naming
(rank, mu, side, rhs); after the exchange its receive segment (mu, 0) must
hold the pattern of its forward neighbour along mu and (mu, 1) that of its
backward neighbour, as include/lqcd.h specifies, with the segment layout
the library reports (lqcd_halo_layout, no GPU needed)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _pattern(rank, k, r, n):
    # distinct bytes per (source rank, segment, rhs): a ramp offset by a key
    key = (rank * 37 + k * 11 + r * 5) % 251
    return ((torch.arange(n, dtype=torch.int64) + key) % 256).to(torch.uint8)


def _expected_source(coord, part, mu, side):
    c = list(coord)
    c[mu] = (c[mu] + (1 if side == 0 else -1)) % part[mu]
    # rank numbering independent of the module under test: x fastest
    return ((c[3] * part[2] + c[2]) * part[1] + c[1]) * part[0] + c[0]


def _worker(rank, world, port, dims, part, nrhs, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1103_1363_gb300 import halo, lqcd
    coord = halo.coord_of(rank, part)
    ctx = lqcd.lqcd_create(halo.local_dims(dims, part), precisions=("f64", "f32"), part=part, coord=coord)
    ok = 1
    for prec in ("f32", "f64"):
        layout = lqcd.lqcd_halo_layout(ctx, prec)
        off, ln, total = layout
        send = torch.zeros(nrhs * total, dtype=torch.uint8)
        recv = torch.zeros(nrhs * total, dtype=torch.uint8)
        for k in range(8):
            for r in range(nrhs):
                if ln[k]:
                    send[r * total + off[k]:r * total + off[k] + ln[k]] = _pattern(rank, k, r, ln[k])
        halo.exchange(send, recv, layout, coord, part, nrhs=nrhs)
        for mu in range(4):
            for side in range(2):
                k = 2 * mu + side
                if part[mu] < 2:
                    ok &= int(ln[k] == 0)
                    continue
                real = 8 if prec == "f64" else 4
                ldims = halo.local_dims(dims, part)
                nf = ldims[0] * ldims[1] * ldims[2] * ldims[3] // ldims[mu] // 2
                ok &= int(ln[k] == nf * 12 * real)
                src = _expected_source(coord, part, mu, side)
                for r in range(nrhs):
                    got = recv[r * total + off[k]:r * total + off[k] + ln[k]]
                    ok &= int(torch.equal(got, _pattern(src, k, r, ln[k])))
    lqcd.lqcd_destroy(ctx)
    out[rank] = ok
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("dims,part,nrhs", [((4, 4, 4, 8), (1, 1, 1, 2), 2), ((4, 4, 8, 8), (1, 1, 2, 2), 1)],
                         ids=["t2", "z2t2"])
def test_face_exchange_gloo(dims, part, nrhs):
    from paper_1103_1363_gb300 import _build
    _build.build()
    world = part[0] * part[1] * part[2] * part[3]
    out = torch.zeros(world, dtype=torch.int32).share_memory_()
    mp.start_processes(_worker, args=(world, _free_port(), dims, part, nrhs, out), nprocs=world,
                       start_method="spawn")
    assert out.tolist() == [1] * world


def test_plan_pairs_every_send_with_a_receive():
    """Across all ranks, each (mu, side) transfer sent to a rank is expected
    by that rank from the sender (host logic only)."""
    from paper_1103_1363_gb300 import halo
    for part in ((1, 1, 1, 2), (1, 1, 2, 2), (2, 1, 1, 4), (1, 2, 3, 2)):
        world = part[0] * part[1] * part[2] * part[3]
        sends = set()
        recvs = set()
        for rank in range(world):
            for mu, side, to, frm in halo.plan(halo.coord_of(rank, part), part):
                sends.add((rank, to, mu, side))
                recvs.add((frm, rank, mu, side))
            assert halo.rank_of(halo.coord_of(rank, part), part) == rank
        assert sends == recvs
