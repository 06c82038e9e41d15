"""The learned preconditioner end to end on a small lattice: pairs from the
library's own 20-iteration CG, training on the GPU, and FGCR(20) with the
trained network against the untrained network and the identity; every
solution checked by one oracle operator application."""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests.gpu_helpers import require_cuda

pytestmark = pytest.mark.gpu


def test_pairs_satisfy_m_e_equals_r():
    lq = require_cuda()
    from paper_1103_1363_gb300 import learned
    dims = (4, 4, 4, 8)
    kappa, csw = 0.13, 1.0
    U = synth.smooth_gauge(dims, 0.5, 5)
    lat = lq.Lattice(dims, max_nrhs=4, precisions=("f64", "f32"))
    lat.gauge_load(U)
    lat.clover_compute(kappa, csw)
    R, E = learned.make_pairs(lat, 4, seed=3)
    A = oracle.clover(U, kappa, csw)
    for i in range(4):
        r, e = R[i].cpu().numpy().astype(np.complex128), E[i].cpu().numpy().astype(np.complex128)
        me = oracle.wilson_clover(U, A, kappa, e)
        assert np.linalg.norm(me - r) / np.linalg.norm(r) < 1e-5  # complex64 storage
        assert np.linalg.norm(r) > 0


def test_training_pair_matches_oracle():
    """lqcd_training_pair: e = x* - x and r = M e (FP64, rounded to FP32 once)
    against the oracle's operator, over more right-hand sides than the
    context's solver vectors hold (chunked), and with x = 0 (r = M x*)."""
    lq = require_cuda()
    dims = (4, 4, 6, 8)
    kappa, csw = 0.13, 1.0
    U = synth.smooth_gauge(dims, 0.5, 6)
    lat = lq.Lattice(dims, max_nrhs=2, precisions=("f64", "f32"))
    lat.gauge_load(U)
    lat.clover_compute(kappa, csw)
    n = 5
    xs = synth.gaussian_spinor(dims, 20, nfields=n)
    x = synth.gaussian_spinor(dims, 21, nfields=n)
    A = oracle.clover(U, kappa, csw)
    shape = (n,) + xs.shape[1:]
    for xx in (x, None):
        R = torch.empty(shape, dtype=torch.complex64, device="cuda")
        E = torch.empty_like(R)
        lq.lqcd_training_pair(lat.ctx, R, E, torch.from_numpy(xs).cuda(),
                              None if xx is None else torch.from_numpy(xx).cuda(), n)
        torch.cuda.synchronize()
        for i in range(n):
            e_want = xs[i] - (0 if xx is None else xx[i])
            r_want = oracle.wilson_clover(U, A, kappa, e_want)
            e_got = E[i].cpu().numpy().astype(np.complex128)
            r_got = R[i].cpu().numpy().astype(np.complex128)
            assert np.linalg.norm(e_got - e_want) / np.linalg.norm(e_want) < 1e-7
            assert np.linalg.norm(r_got - r_want) / np.linalg.norm(r_want) < 1e-7


def test_trained_net_reduces_fgcr_iterations():
    require_cuda()
    from paper_1103_1363_gb300 import learned
    out = learned.run_experiment(dims=(8, 8, 8, 8), eps=0.5, kappa=0.13, csw=1.0, train_seeds=range(100, 104),
                                 test_seeds=range(124, 126), npairs=256, channels=(1, 8, 8, 1), epochs=8,
                                 batch=8, lr=2e-3, log=print)
    s = out["summary"]
    for k, v in s.items():
        assert v["all_converged"] and v["true_residual_max"] <= 1e-10, k
    print({k: v["iterations_mean"] for k, v in s.items()})
    assert out["loss_history"][-1] < out["loss_history"][0]
    assert s["fgcr_trained"]["iterations_mean"] < s["fgcr_identity"]["iterations_mean"]
