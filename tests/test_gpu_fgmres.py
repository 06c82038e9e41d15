"""FGMRES-DR on the GPU (FP32 Arnoldi, FP64 restarts) against the FP64
oracle (Sec. 7): the iterate after the same iterations, with and without a
deflated restart, and converged solutions checked by the oracle's true
residual, with the identity and with SAP as right preconditioner."""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests.gpu_helpers import require_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lq():
    return require_cuda()


def setup(lq, dims, kappa, csw, seed=61, K=24):
    U = synth.smooth_gauge(dims, 0.5, seed)
    A = oracle.clover(U, kappa, csw) if csw else None
    b = synth.gaussian_spinor(dims, seed + 1)
    lat = lq.Lattice(dims, gcr_nkrylov=K)
    lat.gauge_load(U)
    lat.clover_compute(kappa, csw)
    return U, A, b, lat


def gpu_solve(lq, lat, b, m, k, maxiter=100000, tol=1e-10):
    x = lat.canonical_spinor()
    rc, st = lat.solve(x, torch.from_numpy(b).cuda(), tol, raise_on_error=False, solver=lq.SOLVER_FGMRES_DR,
                       inner_prec="f32", nkrylov=m, ndefl=k, maxiter=maxiter)
    return x.cpu().numpy(), rc, st


@pytest.mark.parametrize("k", [0, 3])
def test_iterate_matches_oracle(lq, k):
    """After one full cycle of 8 (and, with deflation, 5 more iterations
    after a deflated restart) the GPU iterate equals the oracle's to FP32
    accuracy of the Arnoldi recursion."""
    dims, kappa = (8, 8, 8, 8), 0.12
    U, A, b, lat = setup(lq, dims, kappa, 0.0)
    for maxiter in ((8,) if k == 0 else (8, 13)):
        xg, rc, st = gpu_solve(lq, lat, b, 8, k, maxiter=maxiter)
        assert st["iterations"] == maxiter
        xo, it, _, _ = oracle.fgmres_dr(U, A, kappa, b, m=8, k=k, maxiter=maxiter)
        err = np.linalg.norm(xg - xo) / np.linalg.norm(xo)
        print("k %d after %d: rel diff %.2e" % (k, maxiter, err))
        assert err < 1e-4


@pytest.mark.parametrize("m,k", [(8, 0), (12, 4), (20, 6)])
def test_converges_identity(lq, m, k):
    dims, kappa, csw = (8, 8, 8, 8), 0.13, 1.0
    U, A, b, lat = setup(lq, dims, kappa, csw)
    xg, rc, st = gpu_solve(lq, lat, b, m, k)
    res = oracle.true_residual(U, A, kappa, b, xg)
    _, it_o, _, ok = oracle.fgmres_dr(U, A, kappa, b, m=m, k=k)
    print("m %d k %d: %d iterations (oracle %d), %d restarts, res %.2e" % (m, k, st["iterations"], it_o,
                                                                            st["restarts"], res))
    assert rc == 0 and ok and res <= 1e-10
    assert st["iterations"] <= 1.5 * it_o + 10


def test_sap_preconditioned(lq):
    dims, kappa, csw = (8, 8, 8, 8), 0.135, 1.0
    U, A, b, lat = setup(lq, dims, kappa, csw)
    _, _, st_id = gpu_solve(lq, lat, b, 16, 4)
    lat.set_sap((4, 4, 4, 4), ncycle=2, nmr=4)
    xg, rc, st = gpu_solve(lq, lat, b, 16, 4)
    lat.set_sap(None)
    res = oracle.true_residual(U, A, kappa, b, xg)
    print("SAP-FGMRES-DR %d iterations (identity %d), res %.2e" % (st["iterations"], st_id["iterations"], res))
    assert rc == 0 and res <= 1e-10
    assert st["iterations"] < st_id["iterations"]


def test_many_deflated_restarts(lq):
    """A short space (m = 6, k = 3) forces dozens of deflated restarts, each
    transforming the kept V and Z in place on the device."""
    dims, kappa, csw = (8, 8, 8, 8), 0.13, 1.0
    U, A, b, lat = setup(lq, dims, kappa, csw)
    xg, rc, st = gpu_solve(lq, lat, b, 6, 3)
    res = oracle.true_residual(U, A, kappa, b, xg)
    print("m 6 k 3: %d iterations, %d restarts, res %.2e" % (st["iterations"], st["restarts"], res))
    assert rc == 0 and res <= 1e-10 and st["restarts"] > 10


def test_rejects_bad_parameters(lq):
    dims = (8, 8, 8, 8)
    U, A, b, lat = setup(lq, dims, 0.12, 0.0, K=8)
    for m, k in ((9, 0), (8, 8), (1, 0), (8, 17)):  # m > cfg.gcr_nkrylov, k >= m, m < 2, k > 16
        with pytest.raises(lq.LqcdError):
            x = lat.canonical_spinor()
            lat.solve(x, torch.from_numpy(b).cuda(), 1e-10, solver=lq.SOLVER_FGMRES_DR, inner_prec="f32",
                      nkrylov=m, ndefl=k)
