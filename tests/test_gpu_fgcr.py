"""Flexible GCR on the GPU: identity, a fixed polynomial preconditioner
expressed as a one-layer network (1 + kappa H, the first term of the
hopping expansion of M^{-1} without clover), and a random network; every
solution verified by one oracle operator application."""
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


def solve(lq, lat, b, **kw):
    x = lat.canonical_spinor()
    rc, st = lat.solve(x, torch.from_numpy(b).cuda(), 1e-10, solver=lq.SOLVER_FGCR,
                       inner_prec="f32", nkrylov=20, **kw)
    return x.cpu().numpy(), st


def test_fgcr_identity_and_hopping_preconditioner(lq):
    dims = (8, 8, 8, 8)
    kappa = 0.12
    U = synth.smooth_gauge(dims, 0.5, 41)
    b = synth.gaussian_spinor(dims, 0)
    lat = lq.Lattice(dims, gcr_nkrylov=20)
    lat.gauge_load(U)
    lat.clover_compute(kappa, 0.0)
    x, st_id = solve(lq, lat, b)
    assert oracle.true_residual(U, None, kappa, b, x) <= 1e-10
    # N = 1 + kappa H: W_0 = 1, W_{+mu} = kappa (1 - g_mu), W_{-mu} = kappa (1 + g_mu)
    net = lq.Net(lat, (1, 1), bf16=False)
    W = np.zeros((9, 4, 4), complex)
    W[0] = np.eye(4)
    for mu in range(4):
        g = oracle.gamma(mu)
        W[2 * mu + 1] = kappa * (np.eye(4) - g)
        W[2 * mu + 2] = kappa * (np.eye(4) + g)
    net.set_weights(W.reshape(-1))
    net.use_as_preconditioner()
    x, st_p = solve(lq, lat, b)
    res = oracle.true_residual(U, None, kappa, b, x)
    print("fgcr identity %d iters, 1+kH %d iters, res %.2e" % (st_id["iterations"], st_p["iterations"], res))
    assert res <= 1e-10
    assert st_p["iterations"] < st_id["iterations"]
    net.use_as_preconditioner(False)


def hopping_net_weights(kappa, chans, rng, noise):
    """Weights of a (1, C, C, 1) network that computes 1 + kappa H through
    channel 0 (identity in the first layers, the hopping expansion in the
    last), plus small random weights everywhere."""
    ws = []
    for l in range(3):
        cin, cout = chans[l], chans[l + 1]
        w = noise * (rng.standard_normal((9, 4 * cout, 4 * cin)) + 1j * rng.standard_normal((9, 4 * cout, 4 * cin)))
        w[0, :4, :4] += np.eye(4)
        if l == 2:
            for mu in range(4):
                g = oracle.gamma(mu)
                w[2 * mu + 1, :4, :4] += kappa * (np.eye(4) - g)
                w[2 * mu + 2, :4, :4] += kappa * (np.eye(4) + g)
        ws.append(w.reshape(-1))
    return np.concatenate(ws)


@pytest.mark.parametrize("bf16", [False, True])
def test_fgcr_clover_three_layer_net(lq, bf16):
    """A (1, 12, 12, 1) network near 1 + kappa H (perturbed by noise) in the
    FGCR slot, FP32 and BF16 tensor-core layers, with clover."""
    dims = (8, 8, 8, 8)
    kappa, csw = 0.13, 1.0
    U = synth.smooth_gauge(dims, 0.5, 42)
    b = synth.gaussian_spinor(dims, 1)
    lat = lq.Lattice(dims, gcr_nkrylov=20)
    lat.gauge_load(U)
    lat.clover_compute(kappa, csw)
    _, st_id = solve(lq, lat, b)
    net = lq.Net(lat, (1, 12, 12, 1), bf16=bf16)
    net.set_weights(hopping_net_weights(kappa, (1, 12, 12, 1), np.random.default_rng(3), 0.002))
    net.use_as_preconditioner()
    x, st = solve(lq, lat, b)
    res = oracle.true_residual(U, oracle.clover(U, kappa, csw), kappa, b, x)
    print("fgcr 3-layer net bf16=%d: %d iters (identity %d), res %.2e" % (
        bf16, st["iterations"], st_id["iterations"], res))
    assert res <= 1e-10
    assert st["iterations"] < st_id["iterations"]
