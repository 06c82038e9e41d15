"""GPU parity of the parallel-transport convolution network against the FP64
oracle: each layer, its adjoint (input gradient) and its weight gradient;
the whole-network gradient of a training step against oracle backprop.

Tolerances: FP32 path rel-L2 <= 1e-5 (FP32 rounding of sums of ~900
terms).  BF16 tensor-core path: each operand is rounded to an 8-bit
significand (unit roundoff 2^-9 = 2.0e-3) and the products are summed in
FP32, so a layer's output, input gradient and weight gradient carry a
relative error of about 2^-9 (measured 2.3-3.4e-3 on the cases here, the
multi-channel layers also reading BF16 activations); the tolerance is 5e-3
for one layer and 6e-3 for a training step's gradient, which chains five
BF16 contractions (measured 2.6e-3).

The persistent BF16 kernels stride over 128-site tiles (64-site tiles for
the multi-channel weight gradient; one CTA per SM, or per SM and group of
hops).  Cases with a CTA cap (lqcd_net_set_max_ctas) and the 8^4 x 16 batch
make every CTA run several tiles, so the next-tile prefetch, the mbarrier
phases across tiles and the weight gradients' accumulation in tensor memory
across tiles are compared with the oracle too.  The one-channel layers (the
first, and the last one's adjoint and weight gradient) take their own
folded-hop kernels, which every (1, C, C', 1) case here exercises."""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests.gpu_helpers import rel, require_cuda

pytestmark = pytest.mark.gpu

DIMS = (4, 4, 6, 8)


def rand_w(rng, cout, cin, scale=0.2):
    return (scale * (rng.standard_normal((9, 4 * cout, 4 * cin))
                     + 1j * rng.standard_normal((9, 4 * cout, 4 * cin)))).astype(np.complex128)


def field(dims, ch, seed, batch=1):
    f = synth.gaussian_spinor(dims, seed, nfields=batch * ch)
    lt, lz, ly, lx = dims[3], dims[2], dims[1], dims[0]
    f = f.reshape(batch, ch, lt, lz, ly, lx, 4, 3)
    return np.ascontiguousarray(np.moveaxis(f, 1, 5))  # (B, Lt, Lz, Ly, Lx, ch, 4, 3)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).astype(np.complex64)).cuda()


@pytest.fixture(scope="module")
def lq():
    return require_cuda()


TOL_BF16_LAYER = 5e-3
TOL_BF16_STEP = 6e-3


def make(lq, channels, bf16, U, max_batch=2, dims=DIMS, max_ctas=0):
    lat = lq.Lattice(dims, max_nrhs=1)
    lat.gauge_load(U)
    net = lq.Net(lat, channels, bf16=bf16, max_batch=max_batch)
    net.set_max_ctas(max_ctas)
    return lat, net


# (dims, channels, bf16, batch, CTA cap)
# 4x4x6x8: 768 sites, six full 128-site tiles of the tensor-core kernel;
# 4x4x6x6: 576 sites, a ragged last tile (64 sites); 2x2x2x2: one tile
# that is mostly padding; odd widths exercise the K and N padding.
# Multi-tile cases: cap 1 puts all 12 tiles (batch 2) through one CTA per
# launch (per hop for the weight gradient); cap 3 on 4x4x6x6 gives each CTA
# 3-4 tiles with ragged tiles inside its loop; 8^4 x 16 is 512 tiles at the
# default grid: >= 3 per layer CTA and 32 per weight-gradient CTA.
CASES = [(DIMS, (1, 12, 12, 1), False, 2, 0), (DIMS, (1, 12, 12, 1), True, 2, 0),
         ((4, 4, 6, 6), (1, 12, 12, 1), True, 2, 0), ((2, 2, 2, 2), (1, 5, 3, 1), True, 2, 0),
         (DIMS, (1, 12, 12, 1), True, 2, 1), ((4, 4, 6, 6), (1, 12, 12, 1), True, 2, 3),
         (DIMS, (1, 12, 12, 1), False, 2, 1), ((8, 8, 8, 8), (1, 12, 12, 1), True, 16, 0)]
CASE_IDS = ["f32", "bf16", "bf16-ragged", "bf16-tiny-odd", "bf16-1cta", "bf16-ragged-3cta", "f32-1cta",
            "bf16-8c8-batch16"]


@pytest.mark.parametrize("dims,chans,bf16,B,cap", CASES, ids=CASE_IDS)
def test_layers_forward_adjoint_wgrad(lq, dims, chans, bf16, B, cap):
    U = synth.smooth_gauge(dims, 0.5, 31)
    rng = np.random.default_rng(0)
    Ws = [rand_w(rng, chans[l + 1], chans[l]) for l in range(3)]
    lat, net = make(lq, chans, bf16, U, dims=dims, max_batch=B, max_ctas=cap)
    net.set_weights(np.concatenate([w.reshape(-1) for w in Ws]))
    tol = TOL_BF16_LAYER if bf16 else 1e-5
    for l in range(3):
        cin, cout = chans[l], chans[l + 1]
        x = field(dims, cin, 40 + l, B)
        g = field(dims, cout, 50 + l, B)
        out = torch.empty(x.shape[:5] + (cout, 4, 3), dtype=torch.complex64, device="cuda")
        net.layer_apply(l, out, dev(x), batch=B)
        gin = torch.empty(x.shape, dtype=torch.complex64, device="cuda")
        net.layer_apply(l, gin, dev(g), batch=B, adjoint=True)
        net.layer_wgrad(l, dev(x), dev(g), batch=B, zero=True)
        torch.cuda.synchronize()
        _, grad = net.get_weights(grad=True)
        off = sum(w.size for w in Ws[:l])
        gW = grad.numpy()[off:off + Ws[l].size].reshape(Ws[l].shape)
        want_out = np.stack([oracle.net_layer(U, Ws[l], x[b]) for b in range(B)])
        want_gin = np.stack([oracle.net_layer_adj(U, Ws[l], g[b]) for b in range(B)])
        want_gW = sum(oracle.net_layer_wgrad(U, x[b], g[b], cout) for b in range(B))
        e1, e2 = rel(out.cpu().numpy(), want_out), rel(gin.cpu().numpy(), want_gin)
        e3 = rel(gW, want_gW)
        print("layer %d bf16=%d: fwd %.2e adj %.2e wgrad %.2e" % (l, bf16, e1, e2, e3))
        assert e1 < tol and e2 < tol and e3 < tol


@pytest.mark.parametrize("bf16,cap", [(False, 0), (True, 0), (True, 1), (True, 2)],
                         ids=["f32", "bf16", "bf16-1cta", "bf16-2cta"])
def test_train_step_gradient_matches_oracle_backprop(lq, bf16, cap):
    U = synth.smooth_gauge(DIMS, 0.5, 32)
    rng = np.random.default_rng(1)
    chans = (1, 4, 3, 1)
    Ws = [rand_w(rng, chans[l + 1], chans[l]) for l in range(3)]
    lat, net = make(lq, chans, bf16, U, max_batch=2, max_ctas=cap)
    net.set_weights(np.concatenate([w.reshape(-1) for w in Ws]))
    B = 2
    r = field(DIMS, 1, 60, B)
    e = field(DIMS, 1, 61, B)
    rs = r[:, :, :, :, :, 0]
    es = e[:, :, :, :, :, 0]
    loss = net.train_step(dev(rs), dev(es), B, lr=0.0)
    torch.cuda.synchronize()
    _, grad = net.get_weights(grad=True)
    # oracle: forward, loss, backprop
    acts = [r]
    for l in range(3):
        acts.append(np.stack([oracle.net_layer(U, Ws[l], acts[-1][b]) for b in range(B)]))
    y = acts[-1]
    en2 = np.array([np.sum(np.abs(e[b]) ** 2) for b in range(B)])
    want_loss = np.mean([np.sum(np.abs(y[b] - e[b]) ** 2) / en2[b] for b in range(B)])
    assert abs(loss - want_loss) / want_loss < (TOL_BF16_STEP if bf16 else 1e-5)
    g = np.stack([2 * (y[b] - e[b]) / (B * en2[b]) for b in range(B)])
    want = []
    for l in range(2, -1, -1):
        want.insert(0, sum(oracle.net_layer_wgrad(U, acts[l][b], g[b], chans[l + 1]) for b in range(B)))
        g = np.stack([oracle.net_layer_adj(U, Ws[l], g[b]) for b in range(B)])
    want = np.concatenate([w.reshape(-1) for w in want])
    err = rel(grad.numpy(), want)
    print("train-step gradient rel err %.2e (bf16=%d)" % (err, bf16))
    assert err < (TOL_BF16_STEP if bf16 else 1e-5)


def test_training_reduces_loss(lq):
    U = synth.smooth_gauge(DIMS, 0.5, 33)
    lat, net = make(lq, (1, 4, 1), True, U, max_batch=4)
    rng = np.random.default_rng(2)
    net.set_weights(np.concatenate([rand_w(rng, 4, 1, 0.1).reshape(-1), rand_w(rng, 1, 4, 0.1).reshape(-1)]))
    # targets made by a fixed random linear map of the same form: learnable exactly
    Wt = [rand_w(rng, 4, 1, 0.3), rand_w(rng, 1, 4, 0.3)]
    r = field(DIMS, 1, 70, 4)
    e = np.stack([oracle.net_layer(U, Wt[1], oracle.net_layer(U, Wt[0], r[b])) for b in range(4)])
    rd, ed = dev(r[..., 0, :, :]), dev(e[..., 0, :, :])
    losses = [net.train_step(rd, ed, 4, lr=2e-2) for _ in range(150)]
    print("loss %.3e -> %.3e" % (losses[0], losses[-1]))
    assert losses[-1] < 0.05 * losses[0]


@pytest.mark.parametrize("bf16", [False, True], ids=["f32", "bf16"])
def test_network_gauge_equivariance(lq, bf16):
    """N_{U^g}(g psi) = g N_U(psi) for a random SU(3) gauge transformation g,
    U^g_mu(x) = g(x) U_mu(x) g(x + mu)^dag: the whole 1-12-12-1 network on
    the GPU (lqcd_net_forward), FP32 and BF16 tensor-core paths.  The two
    BF16 runs round different operands, so their bound is a few times the
    per-layer tolerance; a transport on the wrong side or a missing dagger
    gives an O(1) difference."""
    dims = (8, 8, 8, 8)
    U = synth.smooth_gauge(dims, 0.5, 70)
    G = synth.random_gauge_transform(dims, 71)
    Ug = np.empty_like(U)
    for mu in range(4):
        Gf = np.roll(G, -1, axis=3 - mu)
        Ug[..., mu, :, :] = G @ U[..., mu, :, :] @ np.swapaxes(Gf.conj(), -1, -2)
    rng = np.random.default_rng(5)
    chans = (1, 12, 12, 1)
    w = np.concatenate([rand_w(rng, chans[l + 1], chans[l]).reshape(-1) for l in range(3)])
    psi = synth.gaussian_spinor(dims, 72)
    gpsi = np.einsum("...ab,...sb->...sa", G, psi)
    outs = []
    for links, src in ((U, psi), (Ug, gpsi)):
        lat, net = make(lq, chans, bf16, links, max_batch=1, dims=dims)
        net.set_weights(w)
        out = torch.empty(psi.shape, dtype=torch.complex64, device="cuda")
        net.forward(out, dev(src), batch=1)
        torch.cuda.synchronize()
        outs.append(out.cpu().numpy().astype(np.complex128))
    want = np.einsum("...ab,...sb->...sa", G, outs[0])
    err = rel(outs[1], want)
    print("equivariance bf16=%d: %.2e" % (bf16, err))
    assert err < (3 * TOL_BF16_LAYER if bf16 else 1e-5)


def test_expired_wait_is_reported_and_net_stays_usable(lq):
    """The tensor-core kernels' bounded mbarrier waits: with
    lqcd_net_set_wait's expiry test each CTA's last wait is for a phase that
    nothing completes, bounded by 1 ms, so it runs out; the CTA then waits for
    its own MMAs and copies, frees its tensor memory and exits.  lqcd_sync
    reports LQCD_ERR_TIMEOUT (once), after a forward (the folded first layer,
    the 12 -> 12 layer, the stacked 12 -> 1 contraction) and after a training
    step (the three weight-gradient kernels); with the default bound and the
    weights set again the same network then reproduces its earlier output bit
    for bit."""
    dims = (8, 8, 8, 8)
    U = synth.smooth_gauge(dims, 0.5, 80)
    rng = np.random.default_rng(6)
    chans = (1, 12, 12, 1)
    lat, net = make(lq, chans, True, U, max_batch=2, dims=dims)
    w = np.concatenate([rand_w(rng, chans[l + 1], chans[l]).reshape(-1) for l in range(3)])
    net.set_weights(w)
    psi = dev(synth.gaussian_spinor(dims, 81))
    ref = torch.empty_like(psi)
    net.forward(ref, psi, batch=1)
    lat.sync()
    net.set_wait(1_000_000, expire_test=True)
    out = torch.empty_like(psi)
    net.forward(out, psi, batch=1)
    with pytest.raises(lq.LqcdError) as e:
        lat.sync()
    assert e.value.status == 7
    lat.sync()  # reported once
    r = dev(field(dims, 1, 82, 2)[:, :, :, :, :, 0])
    t = dev(field(dims, 1, 83, 2)[:, :, :, :, :, 0])
    net.train_step(r, t, 2, lr=0.0)
    with pytest.raises(lq.LqcdError) as e:
        lat.sync()
    assert e.value.status == 7
    net.set_wait(0, expire_test=False)
    net.set_weights(w)  # the aborted step's Adam moments and weights are not to be trusted
    out = torch.empty_like(psi)
    net.forward(out, psi, batch=1)
    lat.sync()
    assert torch.equal(out, ref)
