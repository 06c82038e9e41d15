"""GPU solves, each verified by the FP64 CPU oracle: the true residual
|b - M x| / |b| <= 1e-10, computed by one oracle operator application on
the GPU's solution (self-pinning: the oracle operator is pinned by the
CPU tests).  On 4^4 the solution is also compared with the oracle's own
CG solution."""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests.gpu_helpers import gauge, rel, require_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lq():
    return require_cuda()


def check_solution(U, A, kappa, b, x, tol=1e-10):
    res = oracle.true_residual(U, A, kappa, b, x)
    assert res <= tol, res
    return res


def test_cgnr_fp64_4444(lq):
    """Plain Wilson CG on the normal equations, FP64: 4^4, Haar links,
    kappa 0.12, no clover, Gaussian source seed 0."""
    dims = (4, 4, 4, 4)
    kappa = 0.12
    U = synth.haar_gauge(dims, 1)
    b = synth.gaussian_spinor(dims, 0)
    lat = lq.Lattice(dims)
    lat.gauge_load(U)
    lat.clover_compute(kappa, 0.0)
    x = lat.canonical_spinor()
    _, st = lat.solve(x, torch.from_numpy(b).cuda(), 1e-10, solver=lq.SOLVER_CG_FULL, inner_prec="f64")
    xg = x.cpu().numpy()
    res = check_solution(U, None, kappa, b, xg)
    xo, it, ores, ok = oracle.cgnr(U, None, kappa, b)
    assert ok
    assert rel(xg, xo) < 1e-8
    print("cgnr fp64: %d iters (oracle %d), res %.2e, device res %.2e" % (
        st["iterations"], it, res, st["true_residual"]))


@pytest.mark.parametrize("inner", ["bf16", "bf16links", "f16", "bf16spinors"])
def test_eo_cg_bf16_16c16(lq, inner):
    """BF16 storage (8 mantissa bits) converges on the 16^4 system of the
    32^3x64 ensemble (exp(0.4 i H), kappa 0.1355) but needs several times the
    FP32 iteration count; on harder systems it can stall (the operator's
    rounding, amplified by the condition number of the normal equations,
    stops the defect correction from contracting)."""
    dims = (16, 16, 16, 16)
    kappa, csw = 0.1355, 1.0
    U = synth.smooth_gauge(dims, 0.4, 3)
    b = synth.gaussian_spinor(dims, 0)
    lat = lq.Lattice(dims)
    lat.gauge_load(U)
    lat.clover_compute(kappa, csw)
    x = lat.canonical_spinor()
    _, st = lat.solve(x, torch.from_numpy(b).cuda(), 1e-10, inner_prec=inner, maxiter=5000)
    res = check_solution(U, oracle.clover(U, kappa, csw), kappa, b, x.cpu().numpy())
    print("16^4 %s: %d iters, res %.2e" % (inner, st["iterations"], res))


@pytest.mark.parametrize("inner", ["f64", "f32", "f16", "f16links", "f16spinors"])
def test_eo_cg_clover(lq, inner):
    dims = (8, 8, 8, 8)
    kappa, csw = 0.13, 1.0
    U = synth.smooth_gauge(dims, 0.5, 2)
    b = synth.gaussian_spinor(dims, 0)
    lat = lq.Lattice(dims)
    lat.gauge_load(U)
    lat.clover_compute(kappa, csw)
    x = lat.canonical_spinor()
    _, st = lat.solve(x, torch.from_numpy(b).cuda(), 1e-10, inner_prec=inner)
    A = oracle.clover(U, kappa, csw)
    res = check_solution(U, A, kappa, b, x.cpu().numpy())
    assert abs(st["true_residual"] - res) < 1e-11
    print("eo cg %s: %d iters, %d reliable updates, res %.2e" % (
        inner, st["iterations"], st["reliable_updates"], res))


@pytest.mark.parametrize("inner", ["f32", "f16"])
def test_full_cgnr_mixed(lq, inner):
    dims = (4, 4, 4, 8)
    kappa, csw = 0.125, 1.0
    U = synth.smooth_gauge(dims, 0.5, 3)
    b = synth.gaussian_spinor(dims, 1)
    lat = lq.Lattice(dims)
    lat.gauge_load(U)
    lat.clover_compute(kappa, csw)
    x = lat.canonical_spinor()
    lat.solve(x, torch.from_numpy(b).cuda(), 1e-10, solver=lq.SOLVER_CG_FULL, inner_prec=inner)
    check_solution(U, oracle.clover(U, kappa, csw), kappa, b, x.cpu().numpy())


def test_eo_cg_16c32_fp32(lq):
    """Even-odd Wilson-clover, FP32 inner: 16^3x32, exp(0.5 i H) links,
    kappa 0.135, csw 1.0, Gaussian source."""
    dims = (16, 16, 16, 32)
    kappa, csw = 0.135, 1.0
    U = synth.smooth_gauge(dims, 0.5, 2)
    b = synth.gaussian_spinor(dims, 0)
    lat = lq.Lattice(dims, precisions=("f64", "f32"))
    lat.gauge_load(U)
    lat.clover_compute(kappa, csw)
    x = lat.canonical_spinor()
    _, st = lat.solve(x, torch.from_numpy(b).cuda(), 1e-10, inner_prec="f32")
    res = check_solution(U, oracle.clover(U, kappa, csw), kappa, b, x.cpu().numpy())
    print("16^3x32 fp32: %d iters, res %.2e, %.3f s" % (st["iterations"], res, st["seconds"]))


def test_multi_rhs_and_graph(lq):
    """Three right-hand sides solved together (fused CG update and norm
    epilogues on all of them in each launch), with and without graph replay,
    for 16-bit, FP32 and FP16-spinor inner storage; every solution checked by
    the oracle."""
    dims = (8, 8, 8, 8)
    kappa, csw = 0.13, 1.0
    R = 3
    U = synth.smooth_gauge(dims, 0.5, 4)
    b = synth.gaussian_spinor(dims, 5, nfields=R)
    stream = torch.cuda.Stream()
    lat = lq.Lattice(dims, max_nrhs=R, stream=stream)
    lat.gauge_load(U)
    lat.clover_compute(kappa, csw)
    A = oracle.clover(U, kappa, csw)
    bt = torch.from_numpy(b).cuda()
    torch.cuda.synchronize()
    for inner, graph in (("f16", 0), ("f16", 1), ("f32", 1), ("f16spinors", 1)):
        x = lat.canonical_spinor(nrhs=R)
        torch.cuda.synchronize()
        _, st = lat.solve(x, bt, 1e-10, nrhs=R, inner_prec=inner, use_graph=graph)
        xs = x.cpu().numpy()
        for r in range(R):
            check_solution(U, A, kappa, b[r], xs[r])
        print("multi-rhs %s graph=%d: %d iters" % (inner, graph, st["iterations"]))


def test_host_buffers(lq):
    dims = (4, 4, 4, 8)
    kappa, csw = 0.13, 1.0
    U = synth.smooth_gauge(dims, 0.5, 6)
    b = synth.gaussian_spinor(dims, 7)
    lat = lq.Lattice(dims)
    lat.gauge_load(U)  # host numpy links go through the staging path as a tensor copy
    lat.clover_compute(kappa, csw)
    bh = torch.from_numpy(b).pin_memory()
    xh = torch.zeros_like(bh).pin_memory()
    lat.solve(xh, bh, 1e-10, inner_prec="f32")
    check_solution(U, oracle.clover(U, kappa, csw), kappa, b, xh.numpy())


def test_host_gauge_load(lq):
    """Canonical links in host memory are staged in t slices."""
    dims = (4, 4, 4, 8)
    U = synth.haar_gauge(dims, 8)
    psi = synth.gaussian_spinor(dims, 9)
    lat = lq.Lattice(dims)
    lq.lqcd_gauge_load(lat.ctx, torch.from_numpy(U).pin_memory())
    from tests.gpu_helpers import gpu_apply, hop_ref
    got = gpu_apply(lat, "f64", psi, 1, 0, lambda o, i: lat.dslash(o, i, 0, prec="f64"))
    assert rel(got, hop_ref(U, psi, dims, 0)) < 1e-13


def test_not_converged_and_errors(lq):
    dims = (4, 4, 4, 4)
    U = synth.haar_gauge(dims, 1)
    b = synth.gaussian_spinor(dims, 0)
    lat = lq.Lattice(dims)
    lat.gauge_load(U)
    lat.clover_compute(0.12, 0.0)
    x = lat.canonical_spinor()
    rc, st = lat.solve(x, torch.from_numpy(b).cuda(), 1e-10, raise_on_error=False, maxiter=3,
                       check_interval=1, inner_prec="f64")
    assert rc == 5 and st["iterations"] == 3
    assert 1e-10 < st["true_residual"] < 1.0
    # the partial solution is returned and is what the device residual describes
    res = oracle.true_residual(U, None, 0.12, b, x.cpu().numpy())
    assert abs(res - st["true_residual"]) < 1e-12
    f = lat.new_field("f32")
    with pytest.raises(lq.LqcdError) as e:
        lat.dslash(f, f, 0, prec="f32")  # aliasing
    assert e.value.status == 1
    g = lat.new_field("f32")
    with pytest.raises(lq.LqcdError) as e:
        lat.dslash(g, f, 1, 0.12, 1.0, op=lq.OP_SCHUR, prec="f32")  # csw mismatch
    assert e.value.status == 4
    with pytest.raises(lq.LqcdError) as e:
        lat.dslash(g, f, 0, 0.12, 0.0, op=lq.OP_SCHUR, prec="f32")  # Schur on even
    assert e.value.status == 1
