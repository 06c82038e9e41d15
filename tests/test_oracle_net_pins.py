"""Pins of the oracle's parallel-transport convolution layer (no GPU).

* With one channel and the weights W_0 = 1, W_{+mu} = -kappa (1 - g_mu),
  W_{-mu} = -kappa (1 + g_mu) the layer IS the Wilson operator M = 1 - kappa H,
  which the free-field closed form already fixes.  This pins the transport
  direction, the link (not its adjoint) on forward hops and the t sign.
* The adjoint layer satisfies <phi, N psi> = <N^dag phi, psi>.
* Gauge equivariance N[U'](g psi) = g N[U](psi).
* The weight gradient equals central finite differences of a real loss.
"""
import numpy as np
import pytest

import oracle
import synth


def rand_w(rng, cout, cin, scale=0.3):
    return scale * (rng.standard_normal((9, 4 * cout, 4 * cin))
                    + 1j * rng.standard_normal((9, 4 * cout, 4 * cin)))


def test_layer_reduces_to_wilson_operator():
    dims = (4, 4, 6, 4)
    U = synth.haar_gauge(dims, 3)
    kappa = 0.125
    W = np.zeros((9, 4, 4), complex)
    W[0] = np.eye(4)
    for mu in range(4):
        g = oracle.gamma(mu)
        W[2 * mu + 1] = -kappa * (np.eye(4) - g)
        W[2 * mu + 2] = -kappa * (np.eye(4) + g)
    psi = synth.gaussian_spinor(dims, 4)
    out = oracle.net_layer(U, W, psi[..., None, :, :])[..., 0, :, :]
    want = oracle.wilson_clover(U, None, kappa, psi)
    assert np.linalg.norm(out - want) / np.linalg.norm(want) < 1e-14


def test_layer_adjoint():
    dims = (4, 2, 4, 6)
    rng = np.random.default_rng(1)
    U = synth.haar_gauge(dims, 5)
    cin, cout = 2, 3
    W = rand_w(rng, cout, cin)
    psi = synth.gaussian_spinor(dims, 6, nfields=cin)
    psi = np.moveaxis(psi, 0, 4)
    phi = np.moveaxis(synth.gaussian_spinor(dims, 7, nfields=cout), 0, 4)
    lhs = np.vdot(phi.reshape(-1), oracle.net_layer(U, W, psi).reshape(-1))
    rhs = np.vdot(oracle.net_layer_adj(U, W, phi).reshape(-1), psi.reshape(-1))
    assert abs(lhs - rhs) / abs(lhs) < 1e-13


def test_layer_equivariance():
    dims = (4, 4, 4, 4)
    rng = np.random.default_rng(2)
    U = synth.haar_gauge(dims, 8)
    G = synth.random_gauge_transform(dims, 9)
    Up = np.empty_like(U)
    for mu in range(4):
        Gf = np.roll(G, -1, axis=3 - mu)
        Up[..., mu, :, :] = G @ U[..., mu, :, :] @ np.swapaxes(Gf.conj(), -1, -2)
    W = rand_w(rng, 2, 1)
    psi = synth.gaussian_spinor(dims, 10)[..., None, :, :]
    gpsi = np.einsum("...ab,...csb->...csa", G, psi)
    out = oracle.net_layer(Up, W, gpsi)
    want = np.einsum("...ab,...csb->...csa", G, oracle.net_layer(U, W, psi))
    assert np.linalg.norm(out - want) / np.linalg.norm(want) < 1e-13


def test_weight_gradient_finite_differences():
    """L(W) = |N_W(psi) - e|^2 ; G_W = dL/dRe W + i dL/dIm W, G_out = 2 (N psi - e)."""
    dims = (2, 2, 2, 4)
    rng = np.random.default_rng(3)
    U = synth.smooth_gauge(dims, 0.5, 11)
    cin, cout = 2, 2
    W = rand_w(rng, cout, cin)
    psi = np.moveaxis(synth.gaussian_spinor(dims, 12, nfields=cin), 0, 4)
    e = np.moveaxis(synth.gaussian_spinor(dims, 13, nfields=cout), 0, 4)

    def loss(Wx):
        r = oracle.net_layer(U, Wx, psi) - e
        return np.sum(np.abs(r) ** 2)

    gout = 2 * (oracle.net_layer(U, W, psi) - e)
    G = oracle.net_layer_wgrad(U, psi, gout, cout)
    h = 1e-6
    for (hh, i, j) in [(0, 0, 0), (3, 5, 2), (8, 7, 7), (4, 1, 6)]:
        for unit in (1.0, 1j):
            Wp = W.copy(); Wp[hh, i, j] += h * unit
            Wm = W.copy(); Wm[hh, i, j] -= h * unit
            fd = (loss(Wp) - loss(Wm)) / (2 * h)
            an = G[hh, i, j].real if unit == 1.0 else G[hh, i, j].imag
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an))
    # input gradient: dL/dRe psi + i dL/dIm psi = N^dag G_out
    gin = oracle.net_layer_adj(U, W, gout)
    for idx in [(0, 0, 0, 0, 0, 1, 2), (3, 1, 1, 0, 1, 3, 0)]:
        for unit in (1.0, 1j):
            pp = psi.copy(); pp[idx] += h * unit
            pm = psi.copy(); pm[idx] -= h * unit
            fd = (np.sum(np.abs(oracle.net_layer(U, W, pp) - e) ** 2)
                  - np.sum(np.abs(oracle.net_layer(U, W, pm) - e) ** 2)) / (2 * h)
            an = gin[idx].real if unit == 1.0 else gin[idx].imag
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an))
