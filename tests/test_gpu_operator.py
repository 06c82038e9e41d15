"""GPU parity of the hopping term, clover term, Schur complement and full
operator against the FP64 CPU oracle, element by element (rel-L2 over all
real components, in FP64).

Tolerances: FP64 1e-13 (1e-12 where an inverted clover block enters);
FP32 1e-6 (the requirement on the FP32 dslash); FP16 / BF16 storage with a
per-site norm: 3e-3 / 2e-2, i.e. a few units of the format's rounding
(2^-11, 2^-8) - their errors are also printed.
"""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_helpers import (gauge, gpu_apply, hop_ref, parity_mask, rel, require_cuda,
                               restrict)

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-13, "f32": 1e-6, "f16": 3e-3, "bf16": 2e-2, "f16links": 3e-3, "bf16links": 2e-2,
       "f16spinors": 3e-3, "bf16spinors": 2e-2}
ALL = ("f64", "f32", "f16", "bf16", "f16links", "bf16links", "f16spinors", "bf16spinors")

# several tiles with a ragged tail (Vh = 288, 1152+...), the 2^4 degenerate
# lattice (x+mu = x-mu), and a non-cubic shape
LATTICES = [(2, 2, 2, 2), (6, 4, 4, 6), (8, 4, 6, 4), (8, 8, 8, 16)]


@pytest.fixture(scope="module")
def lq():
    return require_cuda()


@pytest.mark.parametrize("dims", LATTICES)
@pytest.mark.parametrize("recon", [12, 18])
def test_hop_all_precisions(lq, dims, recon):
    U = gauge(dims, "haar", seed=3)
    psi = synth.gaussian_spinor(dims, 4)
    lat = lq.Lattice(dims, recon=recon)
    lat.gauge_load(U)
    for prec in ALL:
        for par in (0, 1):
            for dag in (False, True):
                got = gpu_apply(lat, prec, psi, 1 - par, par,
                                lambda o, i: lat.dslash(o, i, par, prec=prec, dag=dag))
                want = hop_ref(U, psi, dims, par, dag)
                err = rel(got, want)
                print("hop %s recon %d par %d dag %d: %.3e" % (prec, recon, par, dag, err))
                assert err < TOL[prec], (prec, par, dag, err)


def test_hop_periodic_t(lq):
    dims = (4, 4, 4, 6)
    U = gauge(dims, "haar", seed=5)
    psi = synth.gaussian_spinor(dims, 6)
    lat = lq.Lattice(dims, t_antiperiodic=0)
    lat.gauge_load(U)
    got = gpu_apply(lat, "f64", psi, 1, 0, lambda o, i: lat.dslash(o, i, 0, prec="f64"))
    src = restrict(psi, dims, 1)
    want = restrict(oracle.hop(U, src, tanti=0), dims, 0)
    assert rel(got, want) < 1e-13


@pytest.mark.parametrize("prec", ALL)
def test_clover_apply(lq, prec):
    dims = (6, 4, 4, 8)
    kappa, csw = 0.135, 1.0
    U = gauge(dims, "smooth", seed=7)
    psi = synth.gaussian_spinor(dims, 8)
    lat = lq.Lattice(dims)
    lat.gauge_load(U)
    lat.clover_compute(kappa, csw)
    A = oracle.clover(U, kappa, csw)
    Ainv, bad = oracle.invert_site_matrices(A)
    assert bad == 0
    tol = TOL[prec]
    for par in (0, 1):
        for inv, M in ((0, A), (1, Ainv)):
            got = gpu_apply(lat, prec, psi, par, par,
                            lambda o, i: lat.clover_apply(o, i, par, inv, prec=prec))
            want = restrict(oracle.apply_site_matrices(M, psi), dims, par)
            err = rel(got, want)
            print("clover %s par %d inv %d: %.3e" % (prec, par, inv, err))
            assert err < tol


@pytest.mark.parametrize("dims,kind", [((4, 4, 4, 4), "haar"), ((8, 6, 4, 6), "smooth"),
                                       ((16, 16, 16, 32), "smooth")])
def test_schur_and_full_operator(lq, dims, kind):
    """Mhat (odd Schur complement, clover) and M, with and without dagger.
    16^3x32 is the even-odd Wilson-clover FP32 workload (kappa 0.135, csw 1)."""
    kappa, csw = 0.135, 1.0
    U = gauge(dims, kind, seed=9)
    psi = synth.gaussian_spinor(dims, 10)
    lat = lq.Lattice(dims)
    lat.gauge_load(U)
    lat.clover_compute(kappa, csw)
    A = oracle.clover(U, kappa, csw)
    Ainv, _ = oracle.invert_site_matrices(A)
    precs = ("f64", "f32") if dims[3] >= 32 else ALL
    for prec in precs:
        tol = {"f64": 1e-12, "f32": 1e-6, "f16": 5e-3, "bf16": 3e-2, "f16links": 5e-3,
               "bf16links": 3e-2, "f16spinors": 5e-3, "bf16spinors": 3e-2}[prec]
        for dag in (False, True):
            got = gpu_apply(lat, prec, psi, 1, 1, lambda o, i: lat.dslash(
                o, i, 1, kappa, csw, op=lq.OP_SCHUR, dag=dag, prec=prec))
            want = oracle.schur(U, A, Ainv, kappa, psi, dag=dag)
            err = rel(got, want)
            print("schur %s dag %d: %.3e" % (prec, dag, err))
            assert err < tol
            got = gpu_apply(lat, prec, psi, 0, 0, lambda o, i: lat.dslash(
                o, i, 0, kappa, csw, op=lq.OP_FULL, dag=dag, prec=prec), full=True)
            want = oracle.wilson_clover(U, A, kappa, psi, dag=dag)
            err = rel(got, want)
            print("full %s dag %d: %.3e" % (prec, dag, err))
            assert err < tol


def test_wilson_without_clover(lq):
    dims = (4, 4, 4, 8)
    kappa = 0.12
    U = gauge(dims, "haar", seed=11)
    psi = synth.gaussian_spinor(dims, 12)
    lat = lq.Lattice(dims)
    lat.gauge_load(U)
    got = gpu_apply(lat, "f64", psi, 0, 0, lambda o, i: lat.dslash(
        o, i, 0, kappa, 0.0, op=lq.OP_FULL, prec="f64"), full=True)
    assert rel(got, oracle.wilson_clover(U, None, kappa, psi)) < 1e-13
    got = gpu_apply(lat, "f64", psi, 1, 1, lambda o, i: lat.dslash(
        o, i, 1, kappa, 0.0, op=lq.OP_SCHUR, prec="f64"))
    assert rel(got, oracle.schur(U, None, None, kappa, psi)) < 1e-13


@pytest.mark.parametrize("prec", ["f32", "f16", "f16spinors", "bf16links"])
def test_multi_rhs_matches_single(lq, prec):
    """nrhs fields in one launch give bit-identical results to one per call,
    for the hopping term and for the Schur operator (A^{-1} and x-pay
    epilogues), plain and dagger."""
    import torch
    dims = (8, 4, 4, 8)
    R = 5
    kappa, csw = 0.13, 1.0
    U = gauge(dims, "smooth", seed=13)
    psis = synth.gaussian_spinor(dims, 14, nfields=R)
    lat = lq.Lattice(dims, max_nrhs=R)
    lat.gauge_load(U)
    lat.clover_compute(kappa, csw)
    fb = lat.field_bytes(prec)
    fin = lat.new_field(prec, nrhs=R)
    fout = lat.new_field(prec, nrhs=R)
    single = torch.empty(fb, dtype=torch.uint8, device="cuda")
    for par in (0, 1):
        lat.pack(fin, psis, 1 - par, prec, nrhs=R)
        for dag in (False, True):
            lat.dslash(fout, fin, par, prec=prec, nrhs=R, dag=dag)
            for r in range(R):
                lat.dslash(single, fin[r * fb:(r + 1) * fb], par, prec=prec, dag=dag)
                torch.cuda.synchronize()
                assert torch.equal(single, fout[r * fb:(r + 1) * fb]), ("hop", par, dag, r)
    lat.pack(fin, psis, 1, prec, nrhs=R)
    for dag in (False, True):
        lat.dslash(fout, fin, 1, kappa, csw, op=lq.OP_SCHUR, dag=dag, prec=prec, nrhs=R)
        for r in range(R):
            lat.dslash(single, fin[r * fb:(r + 1) * fb], 1, kappa, csw, op=lq.OP_SCHUR, dag=dag, prec=prec)
            torch.cuda.synchronize()
            assert torch.equal(single, fout[r * fb:(r + 1) * fb]), ("schur", dag, r)


@pytest.mark.parametrize("prec", ["f32", "f16spinors", "bf16spinors"])
@pytest.mark.parametrize("dims", [(8, 8, 8, 8), (12, 4, 6, 4), (32, 4, 2, 2), (8, 6, 4, 4)])
def test_staged_kernel_matches_gather_and_oracle(lq, prec, dims):
    """The shared-memory staged hopping kernel (LQCD_BLOCK_STAGED) gives the
    gathering kernel's results bit for bit, for the hopping term (both
    parities, plain and dagger, 3 right-hand sides in one launch) and for the
    Schur operator whose A^-1 sweeps it runs; and the hop matches the oracle.
    (8, 6, 4, 4): Ly is no multiple of the tile's 4 rows, so the launch falls
    back to the gathering kernel.)"""
    import torch
    R = 3
    kappa, csw = 0.13, 1.0
    U = gauge(dims, "smooth", seed=21)
    psis = synth.gaussian_spinor(dims, 22, nfields=R)
    lat = lq.Lattice(dims, max_nrhs=R)
    lat.gauge_load(U)
    lat.clover_compute(kappa, csw)
    fin = lat.new_field(prec, nrhs=R)
    fg = lat.new_field(prec, nrhs=R)
    fs = lat.new_field(prec, nrhs=R)
    gather, staged = (128, 128, 128, 128), (lq.BLOCK_STAGED, 128, lq.BLOCK_STAGED, 128)
    fb = lat.field_bytes(prec)
    for par in (0, 1):
        lat.pack(fin, psis, 1 - par, prec, nrhs=R)
        for dag in (False, True):
            fg.fill_(0xff)  # the same bytes in the padding past V/2 sites, which no kernel writes
            fs.fill_(0xff)
            lq.lqcd_tune_set(lat.ctx, prec, gather)
            lat.dslash(fg, fin, par, prec=prec, nrhs=R, dag=dag)
            lq.lqcd_tune_set(lat.ctx, prec, staged)
            lat.dslash(fs, fin, par, prec=prec, nrhs=R, dag=dag)
            torch.cuda.synchronize()
            assert torch.equal(fg, fs), ("hop", par, dag)
            out = lat.canonical_spinor()
            lat.unpack(out, fs[fb:2 * fb], par, prec)
            torch.cuda.synchronize()
            assert rel(out.cpu().numpy(), hop_ref(U, psis[1], dims, par, dag=dag)) < TOL[prec], ("oracle", par, dag)
    lat.pack(fin, psis, 1, prec, nrhs=R)
    for dag in (False, True):
        fg.fill_(0xff)
        fs.fill_(0xff)
        lq.lqcd_tune_set(lat.ctx, prec, gather)
        lat.dslash(fg, fin, 1, kappa, csw, op=lq.OP_SCHUR, dag=dag, prec=prec, nrhs=R)
        lq.lqcd_tune_set(lat.ctx, prec, staged)
        lat.dslash(fs, fin, 1, kappa, csw, op=lq.OP_SCHUR, dag=dag, prec=prec, nrhs=R)
        torch.cuda.synchronize()
        assert torch.equal(fg, fs), ("schur", dag)


def test_tune_set_validates(lq):
    """lqcd_tune_set accepts the tuner's block sizes, and the staged kernel for
    the plain classes only; it rejects anything else."""
    lat = lq.Lattice((4, 4, 4, 4))
    lq.lqcd_tune_set(lat.ctx, "f32", (lq.BLOCK_STAGED, 64, 32, 96), (0, 4))
    for block, sites in (((lq.BLOCK_STAGED, lq.BLOCK_STAGED, 128, 128), None), ((100, 128, 128, 128), None),
                         ((128, 128, 128, 128), (-1, 0)), ((128, 128, 128, 128), (0, 65))):
        with pytest.raises(lq.LqcdError):
            lq.lqcd_tune_set(lat.ctx, "f32", block, sites)


def test_pack_roundtrip(lq):
    dims = (6, 4, 4, 6)
    psi = synth.gaussian_spinor(dims, 15)
    lat = lq.Lattice(dims)
    for prec, tol in (("f64", 0.0), ("f32", 1e-7), ("f16", 1e-3), ("bf16", 8e-3)):
        f = lat.new_field(prec, full=True)
        lat.pack(f, psi, -1, prec)
        out = lat.canonical_spinor()
        lat.unpack(out, f, -1, prec)
        import torch
        torch.cuda.synchronize()
        assert rel(out.cpu().numpy(), psi) <= tol


@pytest.mark.slow
def test_hop_full_size_sampled(lq):
    """32^3x64, FP32 recon-12 (the benchmark's dslash): sampled output sites
    against the oracle computed site by site."""
    dims = (32, 32, 32, 64)
    U = gauge(dims, "smooth", seed=3, eps=0.4)
    psi = synth.gaussian_spinor(dims, 0)
    lat = lq.Lattice(dims, precisions=("f64", "f32"))
    lat.gauge_load(U)
    rng = np.random.default_rng(0)
    for par in (0, 1):
        got = gpu_apply(lat, "f32", psi, 1 - par, par, lambda o, i: lat.dslash(o, i, par, prec="f32"))
        src = restrict(psi, dims, 1 - par)
        mask = parity_mask(dims).reshape(-1)
        cand = np.nonzero(mask == par)[0]
        sites = np.sort(rng.choice(cand, 4096, replace=False))
        want = oracle.hop_sites(U, src, sites)
        g = got.reshape(-1, 4, 3)[sites]
        err = rel(g, want)
        print("full-size hop par %d: %.3e" % (par, err))
        assert err < 1e-6


def test_autotuner_keeps_results(lq):
    """lqcd_tune picks a block size per precision, dagger and reduction; results are
    unchanged by the choice."""
    dims = (8, 8, 8, 8)
    U = gauge(dims, "haar", seed=17)
    psi = synth.gaussian_spinor(dims, 18)
    lat = lq.Lattice(dims)
    lat.gauge_load(U)
    for prec in ("f32", "f16"):
        best = lq.lqcd_tune(lat.ctx, prec)
        assert all(b in (32, 64, 96, 128) for b in best["block"][1::2])  # reducing classes
        assert all(b in (32, 64, 96, 128, lq.BLOCK_STAGED) for b in best["block"][0::2])
        assert all(s in (0, 1, 4, 16) for s in best["sites_per_thread"])
        got = gpu_apply(lat, prec, psi, 1, 0, lambda o, i: lat.dslash(o, i, 0, prec=prec))
        assert rel(got, hop_ref(U, psi, dims, 0)) < TOL[prec]


@pytest.mark.parametrize("prec,tol", [("f64", 1e-14), ("f32", 1e-6), ("f16", 1e-6), ("bf16", 1e-6)])
def test_norm2_matches_numpy(lq, prec, tol):
    """lqcd_norm2 (the deterministic two-stage FP64 reduction of the solvers'
    dots) against numpy's FP64 sum of |psi|^2 over the same stored values:
    per right-hand side, one parity and both (parity -1); the stored values
    are read back with lqcd_unpack, so storage rounding cancels out."""
    import torch
    dims = (8, 6, 4, 6)
    R = 3
    psis = synth.gaussian_spinor(dims, 23, nfields=R)
    lat = lq.Lattice(dims, max_nrhs=R)
    for par in (0, 1, -1):
        f = lat.new_field(prec, nrhs=R, full=(par == -1))
        lat.pack(f, psis, par, prec, nrhs=R)
        got = lq.lqcd_norm2(lat.ctx, f, par, prec, nrhs=R)
        fb = lat.field_bytes(prec) * (2 if par == -1 else 1)
        for r in range(R):
            out = lat.canonical_spinor()
            out.zero_()
            lat.unpack(out, f[r * fb:(r + 1) * fb], par, prec)
            torch.cuda.synchronize()
            want = float(np.sum(np.abs(out.cpu().numpy()) ** 2))
            assert abs(got[r] - want) <= tol * want, (prec, par, r, got[r], want)
