"""The hopping term and the Wilson Schur operator of a lattice cut into
sub-domains (one GPU emulating the ranks: every sub-domain is a context of
its own, the faces travel by device copies), assembled and compared element
by element with the FP64 oracle on the uncut lattice.  Cuts along t (2 and
4 sub-domains, crossing the antiperiodic t boundary), along z and t (2 x 2),
and along x (the checkerboarded direction).  FP64 and FP32 storage, plain
and dagger, both output parities; the interior pass and the face pass run
as separate calls with the exchange between them.  The sub-domains' FP64
norms add up to the global norm."""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests.gpu_helpers import hop_ref, rel, require_cuda, restrict

pytestmark = pytest.mark.gpu

CASES = [((4, 4, 4, 8), (1, 1, 1, 2)), ((4, 4, 4, 16), (1, 1, 1, 4)), ((4, 4, 8, 8), (1, 1, 2, 2)),
         ((8, 4, 4, 4), (2, 1, 1, 1))]
TOL = {"f64": 1e-12, "f32": 1e-6}


class Domains:
    def __init__(self, lq, dims, part, U, prec):
        from paper_1103_1363_gb300 import halo
        self.halo, self.lq, self.dims, self.part, self.prec = halo, lq, dims, part, prec
        self.n = part[0] * part[1] * part[2] * part[3]
        self.coords = [halo.coord_of(r, part) for r in range(self.n)]
        self.ld = halo.local_dims(dims, part)
        self.lats = []
        for c in self.coords:
            lat = lq.Lattice(self.ld, precisions=("f64", "f32"), part=part, coord=c)
            lat.gauge_load(halo.split_field(U, part, c))
            self.lats.append(lat)
        self.layout = lq.lqcd_halo_layout(self.lats[0].ctx, prec)
        tot = self.layout[2]
        self.send = [torch.zeros(tot, dtype=torch.uint8, device="cuda") for _ in range(self.n)]
        self.recv = [torch.zeros(tot, dtype=torch.uint8, device="cuda") for _ in range(self.n)]

    def fields(self, psi, parity):
        fs = []
        for lat, c in zip(self.lats, self.coords):
            f = lat.new_field(self.prec)
            lat.pack(f, self.halo.split_field(psi, self.part, c), parity, self.prec)
            fs.append(f)
        return fs

    def hop(self, fin, in_parity, dag, epi=0, y=None, a=1.0):
        """out_p = epi(H fin) on every sub-domain: pack, exchange, interior, faces."""
        lq = self.lq
        outs = []
        for lat, f, s in zip(self.lats, fin, self.send):
            lq.lqcd_halo_pack(lat.ctx, s, f, in_parity, dag, self.prec)
        for lat, f, k in zip(self.lats, fin, range(self.n)):
            o = lat.new_field(self.prec)
            lq.lqcd_halo_dslash(lat.ctx, o, f, None, 1 - in_parity, dag, epi, y[k] if y else None, a, 1, self.prec)
            outs.append(o)
        torch.cuda.synchronize()
        self.halo.exchange_local(self.send, self.recv, self.layout, self.part)
        for lat, f, o, r, k in zip(self.lats, fin, outs, self.recv, range(self.n)):
            lq.lqcd_halo_dslash(lat.ctx, o, f, r, 1 - in_parity, dag, epi, y[k] if y else None, a, 2, self.prec)
        return outs

    def assemble(self, fields, parity):
        lt, lz, ly, lx = self.dims[3], self.dims[2], self.dims[1], self.dims[0]
        out = np.zeros((lt, lz, ly, lx, 4, 3), np.complex128)
        for lat, f, c in zip(self.lats, fields, self.coords):
            loc = lat.canonical_spinor()
            lat.unpack(loc, f, parity, self.prec)
            torch.cuda.synchronize()
            ld = self.ld
            out[c[3] * ld[3]:(c[3] + 1) * ld[3], c[2] * ld[2]:(c[2] + 1) * ld[2],
                c[1] * ld[1]:(c[1] + 1) * ld[1], c[0] * ld[0]:(c[0] + 1) * ld[0]] = loc.cpu().numpy()
        return out


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("dims,part", CASES, ids=["t2", "t4", "z2t2", "x2"])
def test_halo_hop_matches_oracle(dims, part, prec):
    lq = require_cuda()
    U = synth.smooth_gauge(dims, 0.5, 41)
    psi = synth.gaussian_spinor(dims, 42)
    D = Domains(lq, dims, part, U, prec)
    for par in (0, 1):
        fin = D.fields(psi, 1 - par)
        for dag in (False, True):
            got = D.assemble(D.hop(fin, 1 - par, dag), par)
            want = hop_ref(U, psi, dims, par, dag=dag)
            err = rel(got, want)
            print("halo hop %s %s par %d dag %d: %.2e" % (part, prec, par, dag, err))
            assert err < TOL[prec]
        # the sub-domains' FP64 norms add up to the global one
        n2 = sum(lq.lqcd_norm2(lat.ctx, f, 1 - par, prec)[0] for lat, f in zip(D.lats, fin))
        want = np.sum(np.abs(restrict(psi, dims, 1 - par)) ** 2)
        assert abs(n2 - want) / want < (1e-13 if prec == "f64" else 1e-6)


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("dims,part", CASES[:3], ids=["t2", "t4", "z2t2"])
def test_halo_schur_matches_oracle(dims, part, prec):
    """Mhat = 1 - kappa^2 H_oe H_eo (Wilson, csw = 0) with one exchange per
    sweep: t_e = H_eo in_o, then out_o = in_o - kappa^2 H_oe t_e."""
    lq = require_cuda()
    kappa = 0.13
    U = synth.smooth_gauge(dims, 0.5, 43)
    psi = synth.gaussian_spinor(dims, 44)
    D = Domains(lq, dims, part, U, prec)
    fin = D.fields(psi, 1)
    for dag in (False, True):
        te = D.hop(fin, 1, dag, epi=0)
        out = D.hop(te, 0, dag, epi=2, y=fin, a=-kappa * kappa)
        got = D.assemble(out, 1)
        want = oracle.schur(U, None, None, kappa, restrict(psi, dims, 1), dag=dag)
        err = rel(got, restrict(want, dims, 1))
        print("halo schur %s %s dag %d: %.2e" % (part, prec, dag, err))
        assert err < TOL[prec]


def test_halo_rejects_uncut_and_unsupported():
    lq = require_cuda()
    dims = (4, 4, 4, 4)
    lat = lq.Lattice(dims, precisions=("f64", "f32"))
    f = lat.new_field("f32")
    with pytest.raises(lq.LqcdError) as e:
        lq.lqcd_halo_pack(lat.ctx, f, f, 1, False, "f32")
    assert e.value.status == 4  # not a sub-domain
    cut = lq.Lattice(dims, precisions=("f64", "f32", "f16"), part=(1, 1, 1, 2), coord=(0, 0, 0, 1))
    cut.gauge_load(synth.smooth_gauge(dims, 0.5, 45))
    g = cut.new_field("f16")
    with pytest.raises(lq.LqcdError) as e:
        lq.lqcd_halo_pack(cut.ctx, g, g, 1, False, "f16")
    assert e.value.status == 1
    with pytest.raises(lq.LqcdError) as e:
        cut.clover_compute(0.13, 1.0)  # clover leaves need the neighbours' links
    assert e.value.status == 4
    with pytest.raises(lq.LqcdError) as e:
        cut.dslash(f, g, 0, prec="f32")
    assert e.value.status == 4
