"""SAP on the GPU (FP32; one CTA per block with the block residual in shared
memory) against the FP64 oracle's Schwarz alternating procedure (Sec. 5) on
the same seeded inputs, element by element; SAP in the FGCR slot, verified
by the oracle's true residual and compared with the oracle's SAP-FGCR.

Tolerance: the block solve is a short chain of FP32 operator applications
and FP32 CTA reductions, so the result carries a few times the FP32
operator error (1e-6): 2e-5 relative L2."""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests.gpu_helpers import gauge, gpu_apply, rel, require_cuda

pytestmark = pytest.mark.gpu

TOL = 2e-5

# dims, block, clover, recon, ncycle, nmr
CASES = [
    ((8, 8, 8, 8), (4, 4, 4, 4), True, 12, 1, 4),
    ((8, 4, 8, 16), (4, 2, 4, 4), False, 18, 2, 3),    # non-cubic, Wilson, two cycles
    ((16, 8, 16, 8), (8, 4, 8, 4), True, 12, 1, 4),    # 8x4x8x4: 1024 sites, four sites per thread
    ((16, 4, 4, 20), (8, 2, 2, 10), True, 12, 1, 4),   # 8x2x2x10: 320 sites, ragged second pass
    ((16, 4, 12, 12), (8, 2, 6, 6), True, 18, 1, 4),   # 8x2x6x6: 576 sites
    ((12, 8, 8, 12), (2, 2, 2, 6), True, 12, 2, 2),    # 48 sites: idle lanes in the last warp
    ((4, 4, 4, 4), (2, 2, 2, 2), True, 18, 3, 1),      # 16-site blocks, nmr 1
]


@pytest.fixture(scope="module")
def lq():
    return require_cuda()


@pytest.mark.parametrize("dims,block,clover,recon,ncycle,nmr", CASES)
def test_sap_matches_oracle(lq, dims, block, clover, recon, ncycle, nmr):
    kappa, csw = (0.135, 1.0) if clover else (0.12, 0.0)
    U = gauge(dims, "smooth", seed=51)
    r = synth.gaussian_spinor(dims, 52)
    lat = lq.Lattice(dims, recon=recon)
    lat.gauge_load(U)
    lat.clover_compute(kappa, csw)
    A = oracle.clover(U, kappa, csw) if clover else None
    got = gpu_apply(lat, "f32", r, -1, -1, lambda z, rr: lat.sap_apply(z, rr, block, ncycle, nmr), full=True)
    want = oracle.sap(U, A, kappa, r, block, ncycle, nmr)
    err = rel(got, want)
    print("sap %s block %s ncycle %d nmr %d: %.3e" % (dims, block, ncycle, nmr, err))
    assert err < TOL
    # the preconditioner did work: |r - M z| < |r|
    res = np.linalg.norm(r - oracle.wilson_clover(U, A, kappa, got)) / np.linalg.norm(r)
    assert res < 0.9


def test_sap_zero_residual(lq):
    """r = 0: every MR step meets q = 0 and stops; z = 0 exactly."""
    dims, block = (8, 8, 8, 8), (4, 4, 4, 4)
    lat = lq.Lattice(dims)
    lat.gauge_load(gauge(dims, "smooth", seed=53))
    lat.clover_compute(0.135, 1.0)
    got = gpu_apply(lat, "f32", np.zeros(dims + (4, 3), complex), -1, -1,
                    lambda z, rr: lat.sap_apply(z, rr, block, 2, 4), full=True)
    assert not np.any(got)


def test_sap_rejects_bad_blocks(lq):
    dims = (8, 8, 8, 8)
    lat = lq.Lattice(dims)
    lat.gauge_load(gauge(dims, "smooth", seed=54))
    z = lat.new_field("f32", full=True)
    r = lat.new_field("f32", full=True)
    for block in ((3, 4, 4, 4),        # does not divide
                  (8, 4, 4, 4),        # one block in x
                  (4, 4, 4, 5),        # does not divide
                  (2, 2, 2, 8)):       # one block in t
        with pytest.raises(lq.LqcdError):
            lat.sap_apply(z, r, block)
    big = lq.Lattice((16, 16, 16, 16))
    big.gauge_load(gauge((16, 16, 16, 16), "smooth", seed=55))
    with pytest.raises(lq.LqcdError):
        big.set_sap((8, 4, 8, 8))      # 2048 sites per block
    with pytest.raises(lq.LqcdError):
        lat.set_sap((4, 4, 4, 4), ncycle=0)


def test_fgcr_with_sap(lq):
    """SAP-FGCR on 8^4 (clover): converges to 1e-10 (oracle true residual),
    in fewer iterations than unpreconditioned GCR and within a few
    iterations (FP32 recursion vs FP64) of the oracle's SAP-FGCR."""
    dims, block = (8, 8, 8, 8), (4, 4, 4, 4)
    kappa, csw = 0.135, 1.0
    U = synth.smooth_gauge(dims, 0.5, 56)
    A = oracle.clover(U, kappa, csw)
    b = synth.gaussian_spinor(dims, 57)
    lat = lq.Lattice(dims, gcr_nkrylov=16)
    lat.gauge_load(U)
    lat.clover_compute(kappa, csw)
    bt = torch.from_numpy(b).cuda()
    x = lat.canonical_spinor()
    _, st_id = lat.solve(x, bt, 1e-10, solver=lq.SOLVER_FGCR, inner_prec="f32", nkrylov=16)
    lat.set_sap(block, ncycle=1, nmr=4)
    x = lat.canonical_spinor()
    _, st = lat.solve(x, bt, 1e-10, solver=lq.SOLVER_FGCR, inner_prec="f32", nkrylov=16)
    xs = x.cpu().numpy()
    res = oracle.true_residual(U, A, kappa, b, xs)
    _, it_o, res_o, ok = oracle.fgcr(U, A, kappa, b, 1e-10, nkrylov=16,
                                     prec=lambda r: oracle.sap(U, A, kappa, r, block, 1, 4))
    print("fgcr identity %d, SAP %d (oracle SAP-FGCR %d), res %.2e, fallback %d"
          % (st_id["iterations"], st["iterations"], it_o, res, st["preconditioner_fallback"]))
    assert ok and res <= 1e-10
    assert st["preconditioner_fallback"] == 0
    assert st["iterations"] < st_id["iterations"]
    assert abs(st["iterations"] - it_o) <= max(3, it_o // 8)
    lat.set_sap(None)


def test_fgcr_with_strong_sap_restarts_in_time(lq):
    """5 SAP cycles leave ~4e-3 of the residual per application, so the FP32
    recursion reaches FP32's resolution of the cycle's starting residual
    within a few iterations; the cycle must then end and restart from the
    FP64 residual (8^4, kappa 0.13: this diverged when the cycle ran on)."""
    dims, block = (8, 8, 8, 8), (4, 4, 4, 4)
    kappa, csw = 0.13, 1.0
    U = synth.smooth_gauge(dims, 0.5, 124)
    A = oracle.clover(U, kappa, csw)
    b = synth.gaussian_spinor(dims, 1124)
    lat = lq.Lattice(dims, gcr_nkrylov=20)
    lat.gauge_load(U)
    lat.clover_compute(kappa, csw)
    bt = torch.from_numpy(b).cuda()
    for ncycle in (3, 5, 8):
        lat.set_sap(block, ncycle=ncycle, nmr=4)
        x = lat.canonical_spinor()
        rc, st = lat.solve(x, bt, 1e-10, solver=lq.SOLVER_FGCR, inner_prec="f32", nkrylov=20, maxiter=400)
        res = oracle.true_residual(U, A, kappa, b, x.cpu().numpy())
        print("SAP ncycle %d: %d iterations, %d restarts, res %.2e" % (ncycle, st["iterations"], st["restarts"], res))
        assert rc == 0 and res <= 1e-10
        assert st["iterations"] <= 30
    lat.set_sap(None)
