"""Batched solves: 12 point sources (every spin and colour at the origin) on
24^3x48 in one multi-right-hand-side solve, and an uneven batch of 8^4,
12^4 and 16^3x32 lattices solved together with one CUDA graph per
iteration block.  Each solution is verified by one oracle operator
application."""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests.gpu_helpers import require_cuda

pytestmark = pytest.mark.gpu


def test_uneven_lattice_batch_single_graph():
    lq = require_cuda()
    specs = [((8, 8, 8, 8), 0.120, 4), ((12, 12, 12, 12), 0.1275, 5), ((16, 16, 16, 32), 0.135, 6)]
    stream = torch.cuda.Stream()
    lats, xs, bs, Us = [], [], [], []
    for dims, kappa, seed in specs:
        U = synth.smooth_gauge(dims, 0.5, seed)
        lat = lq.Lattice(dims, precisions=("f64", "f32"), stream=stream)
        lat.gauge_load(U)
        lat.clover_compute(kappa, 1.0)
        b = synth.gaussian_spinor(dims, seed + 100)
        lats.append(lat)
        Us.append(U)
        bs.append(torch.from_numpy(b).cuda())
        xs.append(torch.zeros_like(bs[-1]))
    torch.cuda.synchronize()
    p = lq.solver_params(inner_prec="f32", use_graph=1)
    rc, stats = lq.lqcd_solve_batch([l.ctx for l in lats], xs, bs, [1e-10] * 3, p)
    assert rc == 0
    for (dims, kappa, _), U, x, b, st in zip(specs, Us, xs, bs, stats):
        A = oracle.clover(U, kappa, 1.0)
        res = oracle.true_residual(U, A, kappa, b.cpu().numpy(), x.cpu().numpy())
        print(dims, st["iterations"], "%.2e" % res, st["kernel_launches"])
        assert res <= 1e-10


@pytest.mark.slow
def test_twelve_point_sources_24c48():
    lq = require_cuda()
    dims = (24, 24, 24, 48)
    kappa, csw = 0.135, 1.0
    U = synth.smooth_gauge(dims, 0.5, 4)
    srcs = np.stack([synth.point_source(dims, s, c) for s in range(4) for c in range(3)])
    lat = lq.Lattice(dims, precisions=("f64", "f32", "f16"), max_nrhs=12, stream=torch.cuda.Stream())
    lat.gauge_load(U)
    lat.clover_compute(kappa, csw)
    b = torch.from_numpy(srcs).cuda()
    x = torch.zeros_like(b)
    torch.cuda.synchronize()
    _, st = lat.solve(x, b, 1e-10, nrhs=12, inner_prec="f32", use_graph=1)
    print("12 point sources: %d iters, %.3f s, %d launches" % (st["iterations"], st["seconds"], st["kernel_launches"]))
    A = oracle.clover(U, kappa, csw)
    xh = x.cpu().numpy()
    for r in (0, 5, 11):
        assert oracle.true_residual(U, A, kappa, srcs[r], xh[r]) <= 1e-10
    assert st["true_residual"] <= 1e-10


@pytest.mark.slow
def test_point_source_fp16_spinors_24c48():
    """One point source with FP16-spinor inner storage.  Far from the source
    the iterates' components drop below the smallest normal FP32 number, and
    the per-site-norm codec used to turn those sites into NaN (breakdown
    after the first check interval)."""
    lq = require_cuda()
    dims = (24, 24, 24, 48)
    kappa, csw = 0.135, 1.0
    U = synth.smooth_gauge(dims, 0.5, 4)
    b = synth.point_source(dims, 0, 0)
    lat = lq.Lattice(dims, precisions=("f64", "f32", "f16spinors"), stream=torch.cuda.Stream())
    lat.gauge_load(U)
    lat.clover_compute(kappa, csw)
    x = lat.canonical_spinor()
    rc, st = lat.solve(x, torch.from_numpy(b).cuda(), 1e-10, inner_prec="f16spinors")
    print("point source, FP16 spinors: %d iters, true residual %.2e" % (st["iterations"], st["true_residual"]))
    assert rc == 0 and st["true_residual"] <= 1e-10
    A = oracle.clover(U, kappa, csw)
    assert oracle.true_residual(U, A, kappa, b, x.cpu().numpy()) <= 1e-10


def _uneven_batch(lq, stream):
    specs = [((8, 8, 8, 8), 0.120, 4), ((12, 12, 12, 12), 0.1275, 5), ((16, 16, 16, 32), 0.135, 6)]
    lats, bs, Us = [], [], []
    for dims, kappa, seed in specs:
        U = synth.smooth_gauge(dims, 0.5, seed)
        lat = lq.Lattice(dims, precisions=("f64", "f32"), stream=stream)
        lat.gauge_load(U)
        lat.clover_compute(kappa, 1.0)
        lats.append(lat)
        Us.append(U)
        bs.append(torch.from_numpy(synth.gaussian_spinor(dims, seed + 100)).cuda())
    return specs, lats, bs, Us


@pytest.mark.parametrize("inner", ["f32", "f16spinors"])
def test_uneven_batch_persistent_launch(inner):
    """The uneven batch with every iteration block as one persistent
    cooperative launch over the three lattices: each solution passes the
    oracle's true residual, and the iteration counts match the
    launch-per-stage path (the global sums differ only in summation order)."""
    lq = require_cuda()
    stream = torch.cuda.Stream()
    specs, lats, bs, Us = _uneven_batch(lq, stream)
    its = {}
    for persistent in (0, 1):
        xs = [torch.zeros_like(b) for b in bs]
        torch.cuda.synchronize()
        p = lq.solver_params(inner_prec=inner, use_graph=1, persistent=persistent)
        rc, stats = lq.lqcd_solve_batch([l.ctx for l in lats], xs, bs, [1e-10] * 3, p)
        assert rc == 0
        its[persistent] = [st["iterations"] for st in stats]
        for (dims, kappa, _), U, x, b, st in zip(specs, Us, xs, bs, stats):
            A = oracle.clover(U, kappa, 1.0)
            res = oracle.true_residual(U, A, kappa, b.cpu().numpy(), x.cpu().numpy())
            print(inner, "persistent" if persistent else "per-stage", dims, st["iterations"], "%.2e" % res,
                  st["kernel_launches"])
            assert res <= 1e-10
    for a, b in zip(its[0], its[1]):
        assert abs(a - b) <= 10


def test_persistent_multi_rhs_and_reliable_updates():
    """Three right-hand sides of one 8^4 lattice in the persistent launch,
    with reliable updates every 20 iterations (blocks that end in one) and a
    check interval that does not divide it; every solution checked by the
    oracle."""
    lq = require_cuda()
    dims = (8, 8, 8, 8)
    kappa, csw = 0.13, 1.0
    R = 3
    U = synth.smooth_gauge(dims, 0.5, 7)
    b = synth.gaussian_spinor(dims, 8, nfields=R)
    lat = lq.Lattice(dims, precisions=("f64", "f32"), max_nrhs=R, stream=torch.cuda.Stream())
    lat.gauge_load(U)
    lat.clover_compute(kappa, csw)
    A = oracle.clover(U, kappa, csw)
    for inner in ("f32", "f16spinors"):
        x = lat.canonical_spinor(nrhs=R)
        torch.cuda.synchronize()
        rc, st = lat.solve(x, torch.from_numpy(b).cuda(), 1e-10, nrhs=R, inner_prec=inner, persistent=1,
                           reliable_interval=20, check_interval=7)
        assert rc == 0 and st["reliable_updates"] >= 1
        xs = x.cpu().numpy()
        for r in range(R):
            assert oracle.true_residual(U, A, kappa, b[r], xs[r]) <= 1e-10
        print(inner, st["iterations"], st["reliable_updates"], st["kernel_launches"])


def test_persistent_barrier_timeout_is_reported():
    """A grid-barrier wait bound of 1 us runs out inside the first iteration
    (a hopping stage takes longer): the launch aborts, the solve returns
    LQCD_ERR_TIMEOUT and lqcd_sync reports the error word; the context then
    solves normally."""
    lq = require_cuda()
    dims = (8, 8, 8, 8)
    kappa, csw = 0.13, 1.0
    U = synth.smooth_gauge(dims, 0.5, 9)
    b = torch.from_numpy(synth.gaussian_spinor(dims, 10)).cuda()
    lat = lq.Lattice(dims, precisions=("f64", "f32"), stream=torch.cuda.Stream())
    lat.gauge_load(U)
    lat.clover_compute(kappa, csw)
    x = lat.canonical_spinor()
    rc, _ = lat.solve(x, b, 1e-10, raise_on_error=False, inner_prec="f32", persistent=1, persistent_wait_us=1)
    assert rc == 7
    with pytest.raises(lq.LqcdError) as e:
        lat.sync()
    assert e.value.status == 7
    x = lat.canonical_spinor()
    rc, st = lat.solve(x, b, 1e-10, raise_on_error=False, inner_prec="f32", persistent=1)
    assert rc == 0
    A = oracle.clover(U, kappa, csw)
    assert oracle.true_residual(U, A, kappa, b.cpu().numpy(), x.cpu().numpy()) <= 1e-10


def test_persistent_rejects_unsupported_solves():
    lq = require_cuda()
    dims = (4, 4, 4, 4)
    lat = lq.Lattice(dims, precisions=("f64", "f32", "f16"))
    lat.gauge_load(synth.smooth_gauge(dims, 0.5, 11))
    lat.clover_compute(0.12, 1.0)
    b = torch.from_numpy(synth.gaussian_spinor(dims, 12)).cuda()
    for kw in (dict(inner_prec="f16"), dict(inner_prec="f32", solver=lq.SOLVER_CG_FULL)):
        x = lat.canonical_spinor()
        rc, _ = lat.solve(x, b, 1e-10, raise_on_error=False, persistent=1, **kw)
        assert rc == 1, kw
