"""Learned preconditioner: training pairs, training loop and evaluation.

This module only sequences library calls; every step runs in liblqcd.so's
kernels (operator, CG, network forward / backward, Adam).

Pairs (r, e): for a gauge field, draw x* (complex Gaussian), form b = M x*,
run 20 iterations of CG on the normal equations of M from x = 0 (the
library's solver, FP32 inner iteration), and keep e = x* - x_20 and
r = M e = b - M x_20 (lqcd_training_pair, which also rounds them to the
network's FP32 layout).  The network N is trained to map r
to e (loss |N(r) - e|^2 / |e|^2, Adam), i.e. to act as M^{-1} on the
residuals that plain CG leaves behind, and is then used as the right
preconditioner of flexible GCR(20).

Initialisation (a choice; the paper has no network): every weight is drawn
from N(0, scale^2) (real and imaginary parts) and the spin identity is
added to hop 0 of channel 0 in every layer, so the untrained network is
close to the identity preconditioner.
"""
from __future__ import annotations

import time

import numpy as np
import torch

from . import lqcd


def init_weights(channels, seed, scale=0.01):
    rng = np.random.default_rng(seed)
    ws = []
    for l in range(len(channels) - 1):
        cin, cout = channels[l], channels[l + 1]
        w = scale * (rng.standard_normal((9, 4 * cout, 4 * cin)) + 1j * rng.standard_normal((9, 4 * cout, 4 * cin)))
        w[0, :4, :4] += np.eye(4)
        ws.append(w.reshape(-1))
    return np.concatenate(ws).astype(np.complex64)


def apply_full_operator(lat, out_canon, in_canon, nrhs):
    """out = M in for nrhs canonical FP64 spinors on the device (M of the
    lattice's last lqcd_clover_compute)."""
    f_in = lat.new_field("f64", nrhs=nrhs, full=True)
    f_out = lat.new_field("f64", nrhs=nrhs, full=True)
    lat.pack(f_in, in_canon, -1, "f64", nrhs=nrhs)
    lqcd.lqcd_dslash(lat.ctx, f_out, f_in, 0, lat.kappa, lat.csw, lqcd.OP_FULL, "f64", nrhs)
    lat.unpack(out_canon, f_out, -1, "f64", nrhs=nrhs)


def make_pairs(lat, npairs, seed, cg_iters=20, with_start=True, chunk=None):
    """(r, e) as complex64 device tensors of shape (npairs, Lt, Lz, Ly, Lx, 4, 3).

    Each CG run gives its pair after cg_iters iterations and, when
    with_start, also its pair at iteration 0, (b, x*): the 20-iteration
    residuals carry almost no high-mode content, and a network trained on
    them alone learns nothing about the high modes of a Gaussian source.
    With with_start, npairs // 2 runs are made (npairs even)."""
    chunk = chunk or lat.max_nrhs
    lx, ly, lz, lt = lat.dims
    shape = (lt, lz, ly, lx, 4, 3)
    R = torch.empty((npairs,) + shape, dtype=torch.complex64, device=lat.device)
    E = torch.empty_like(R)
    runs = npairs // 2 if with_start else npairs
    # x* drawn on the device (seeded): complex Gaussian, E|z|^2 = 1 per component
    gen = torch.Generator(device=lat.device).manual_seed(int(seed))
    k = 0
    for p0 in range(0, runs, chunk):
        n = min(chunk, runs - p0)
        xs = torch.randn((n,) + shape, dtype=torch.complex128, device=lat.device, generator=gen)
        b = torch.empty_like(xs)
        apply_full_operator(lat, b, xs, n)
        x20 = torch.zeros_like(xs)
        lat.solve(x20, b, 1e-30, nrhs=n, raise_on_error=False, solver=lqcd.SOLVER_CG_FULL, inner_prec="f32",
                  maxiter=cg_iters, check_interval=10, reliable_interval=0)
        # e = x* - x_20, r = M e: the residual and error of the 20-iteration iterate
        lqcd.lqcd_training_pair(lat.ctx, R[k:k + n], E[k:k + n], xs, x20, n)
        k += n
        if with_start:  # x = 0: e = x*, r = M x* = b
            lqcd.lqcd_training_pair(lat.ctx, R[k:k + n], E[k:k + n], xs, None, n)
            k += n
    torch.cuda.synchronize(lat.device)
    return R[:k], E[:k]


def train(net, fields, epochs, batch, lr=1e-3, seed=0, log=None):
    """Adam on mean |N(r) - e|^2 / |e|^2 over shuffled mini-batches.

    fields: list of (lat_f, R, E) with lat_f a Lattice holding that gauge
    field's links (loaded once) and R, E its pairs.  The network transports
    with the links of the context it is bound to, so every mini-batch is
    drawn from one field and the network is bound to that field's context
    (lqcd_net_bind: no links are reloaded).  Mini-batches of all fields are
    shuffled together.  Returns the mean loss per epoch."""
    gen = torch.Generator(device="cpu").manual_seed(seed)
    hist = []
    for ep in range(epochs):
        batches = []
        for f, (_, R, _) in enumerate(fields):
            perm = torch.randperm(R.shape[0], generator=gen)
            for i in range(0, R.shape[0] - batch + 1, batch):
                batches.append((f, perm[i:i + batch]))
        order = torch.randperm(len(batches), generator=gen).tolist()
        tot = 0.0
        for j in order:
            f, idx = batches[j]
            lat_f, R, E = fields[f]
            if net.bound is not lat_f:
                net.bind(lat_f)
            idx = idx.to(R.device)
            tot += net.train_step(R.index_select(0, idx).contiguous(), E.index_select(0, idx).contiguous(),
                                  batch, lr=lr)
        hist.append(tot / max(len(order), 1))
        if log:
            log("epoch %d loss %.4e" % (ep, hist[-1]))
    return hist


def fgcr_solve(lat, b, tol=1e-10, nkrylov=20, maxiter=20000):
    x = torch.zeros_like(b)
    torch.cuda.synchronize(lat.device)
    t0 = time.perf_counter()
    rc, st = lat.solve(x, b, tol, raise_on_error=False, solver=lqcd.SOLVER_FGCR, inner_prec="f32",
                       nkrylov=nkrylov, maxiter=maxiter)
    st["wall_s"] = time.perf_counter() - t0
    st["status"] = rc
    return x, st


def eo_cg_solve(lat, b, tol=1e-10, inner="f32"):
    x = torch.zeros_like(b)
    torch.cuda.synchronize(lat.device)
    t0 = time.perf_counter()
    rc, st = lat.solve(x, b, tol, raise_on_error=False, inner_prec=inner)
    st["wall_s"] = time.perf_counter() - t0
    st["status"] = rc
    return x, st


def run_experiment(dims=(16, 16, 16, 16), eps=0.5, kappa=0.134, csw=1.0, train_seeds=range(100, 124),
                   test_seeds=range(124, 132), npairs=4096, channels=(1, 12, 12, 1), epochs=10, batch=16,
                   lr=1e-3, net_seed=7, device="cuda", log=print, sap_block=(4, 4, 4, 4), sap_ncycle=5,
                   sap_nmr=4):
    """The learned-preconditioner workload: train on pairs from the training
    fields, then solve one Gaussian source per held-out field with FGCR(20)
    + trained net, FGCR(20) + untrained net, FGCR(20) + identity, FGCR(20) +
    SAP (the paper's preconditioner in the same slot) and mixed-precision
    even-odd CG (FP32 and FP16-spinor inner), all to true residual 1e-10."""
    import synth
    lat = lqcd.Lattice(dims, precisions=("f64", "f32"), max_nrhs=64, gcr_nkrylov=20, device=device)
    train_seeds, test_seeds = list(train_seeds), list(test_seeds)
    per = [npairs // len(train_seeds) + (1 if i < npairs % len(train_seeds) else 0)
           for i in range(len(train_seeds))]
    fields = []
    t0 = time.perf_counter()
    for s, n in zip(train_seeds, per):
        U = torch.from_numpy(synth.smooth_gauge(dims, eps, s)).to(device)
        lat.gauge_load(U)
        lat.clover_compute(kappa, csw)
        R, E = make_pairs(lat, n, seed=10000 + s)
        # the field's links stay resident in a small context of their own
        lat_f = lqcd.Lattice(dims, precisions=("f64", "f32"), max_nrhs=1, device=device)
        lat_f.gauge_load(U)
        fields.append((lat_f, R, E))
    t_pairs = time.perf_counter() - t0
    log("pairs: %d in %.1f s" % (sum(per), t_pairs))
    net = lqcd.Net(lat, channels, bf16=True, max_batch=batch)
    w0 = init_weights(channels, net_seed)
    net.set_weights(w0)
    t0 = time.perf_counter()
    hist = train(net, fields, epochs, batch, lr=lr, log=log)
    torch.cuda.synchronize(device)
    t_train = time.perf_counter() - t0
    net.bind(lat)
    w_trained = net.get_weights()
    for lat_f, _, _ in fields:
        lat_f.close()
    del fields
    results = []
    for s in test_seeds:
        U = torch.from_numpy(synth.smooth_gauge(dims, eps, s)).to(device)
        lat.gauge_load(U)
        lat.clover_compute(kappa, csw)
        b = torch.from_numpy(synth.gaussian_spinor(dims, 1000 + s)).to(device)
        row = {"seed": s}
        net.use_as_preconditioner(False)
        _, row["fgcr_identity"] = fgcr_solve(lat, b)
        net.set_weights(w0)
        net.use_as_preconditioner(True)
        _, row["fgcr_untrained"] = fgcr_solve(lat, b)
        net.set_weights(w_trained)
        _, row["fgcr_trained"] = fgcr_solve(lat, b)
        net.use_as_preconditioner(False)
        if sap_block is not None:
            lat.set_sap(sap_block, sap_ncycle, sap_nmr)
            _, row["fgcr_sap"] = fgcr_solve(lat, b)
            lat.set_sap(None)
        _, row["eo_cg_f32"] = eo_cg_solve(lat, b)
        _, row["eo_cg_f16spinors"] = eo_cg_solve(lat, b, inner="f16spinors")
        results.append(row)
        log("test %d: " % s + ", ".join("%s %d it %.3f s res %.1e" % (k, v["iterations"], v["wall_s"],
                                                                       v["true_residual"])
                                        for k, v in row.items() if k != "seed"))
    summary = {}
    for k in [k for k in results[0] if k != "seed"]:
        summary[k] = {"iterations_mean": float(np.mean([r[k]["iterations"] for r in results])),
                      "wall_s_mean": float(np.mean([r[k]["wall_s"] for r in results])),
                      "true_residual_max": float(max(r[k]["true_residual"] for r in results)),
                      "all_converged": all(r[k]["status"] == 0 for r in results)}
    return {"pairs_s": t_pairs, "train_s": t_train, "loss_history": hist, "summary": summary,
            "per_field": [{k: (v if k == "seed" else {q: v[q] for q in ("iterations", "wall_s", "true_residual")})
                           for k, v in r.items()} for r in results]}


if __name__ == "__main__":
    import json
    import sys
    import os
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    out = run_experiment()
    print(json.dumps(out))
