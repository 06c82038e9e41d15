"""The Schur operator with its intermediate in the library's fixed device
array (lqcd_dslash_schur_static) gives what lqcd_dslash(OP_SCHUR) gives.

Callers that cannot allocate device memory where they apply the operator
use this entry point; its scratch is a 32 MiB array the CUDA module keeps
on each GPU.  Collected last (file name) so that a failure here leaves the
rest of a stop-at-first-failure run already done."""
import numpy as np
import pytest
import torch

import synth
from tests.gpu_helpers import rel, require_cuda

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-6, "f16": 5e-3}


def test_static_scratch_matches_workspace_scratch():
    lq = require_cuda()
    dims = (16, 16, 16, 32)
    kappa, csw = 0.135, 1.0
    U = synth.smooth_gauge(dims, 0.5, 21)
    lat = lq.Lattice(dims, max_nrhs=2)
    lat.gauge_load(U)
    lat.clover_compute(kappa, csw)
    for prec in ("f64", "f32", "f16"):
        for dag in (False, True):
            for call in range(2):  # two calls in a row, different inputs
                psi = synth.gaussian_spinor(dims, 100 + call, nfields=2)
                fin = lat.new_field(prec, nrhs=2)
                ref = lat.new_field(prec, nrhs=2)
                got = lat.new_field(prec, nrhs=2)
                lat.pack(fin, psi, 1, prec, nrhs=2)
                lat.dslash(ref, fin, 1, kappa, csw, op=lq.OP_SCHUR, dag=dag, prec=prec, nrhs=2)
                lq.lqcd_dslash_schur_static(lat.ctx, got, fin, kappa, csw, dag, prec, nrhs=2)
                a = lat.canonical_spinor(nrhs=2)
                b = lat.canonical_spinor(nrhs=2)
                lat.unpack(a, ref, 1, prec, nrhs=2)
                lat.unpack(b, got, 1, prec, nrhs=2)
                torch.cuda.synchronize()
                a, b = a.cpu().numpy(), b.cpu().numpy()
                assert np.linalg.norm(a) > 0
                assert rel(b, a) <= TOL[prec], (prec, dag, call)


def test_static_scratch_size_limit():
    lq = require_cuda()
    dims = (16, 16, 16, 32)  # one FP64 odd field is 12.6 MB: three exceed 32 MiB
    lat = lq.Lattice(dims, max_nrhs=3)
    lat.gauge_load(synth.smooth_gauge(dims, 0.5, 22))
    f = lat.new_field("f64", nrhs=3)
    g = lat.new_field("f64", nrhs=3)
    with pytest.raises(lq.LqcdError) as e:
        lq.lqcd_dslash_schur_static(lat.ctx, g, f, 0.13, 0.0, 0, "f64", nrhs=3)
    assert e.value.status == 1 and "32 MiB" in str(e.value)
