"""lqcd_dslash_schur_static: the Schur operator with its even-parity
intermediate in a 32 MiB array that the library's CUDA module keeps on each
GPU, for callers that cannot allocate device memory where they apply the
operator (a fixed memory budget, an allocator that must not grow, code
running where cudaMalloc is not allowed).

Checked on two calls in a row with different inputs: the result equals
lqcd_dslash(OP_SCHUR) (the workspace path) and the FP64 oracle's Schur
operator; the call writes nothing in the context's workspace (the library's
solver vectors stay intact) and PyTorch's allocator sees no new device
memory.  Collected last (file name) so that a failure here leaves the rest
of a stop-at-first-failure run already done."""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests.gpu_helpers import rel, require_cuda, restrict

pytestmark = pytest.mark.gpu

# against the workspace path (same kernels, same order: bit-identical in
# practice) and against the FP64 oracle (the storage precision's rounding)
TOL = {"f64": 1e-12, "f32": 1e-6, "f16": 5e-3}
TOL_ORACLE = {"f64": 1e-12, "f32": 1e-6, "f16": 5e-3}


def test_static_scratch_matches_workspace_and_oracle():
    lq = require_cuda()
    dims = (16, 16, 16, 32)
    kappa, csw = 0.135, 1.0
    U = synth.smooth_gauge(dims, 0.5, 21)
    lat = lq.Lattice(dims, max_nrhs=2)
    lat.gauge_load(U)
    lat.clover_compute(kappa, csw)
    A = oracle.clover(U, kappa, csw)
    Ainv, _ = oracle.invert_site_matrices(A)
    for prec in ("f64", "f32", "f16"):
        for dag in (False, True):
            for call in range(2):  # two calls in a row, different inputs
                psi = synth.gaussian_spinor(dims, 100 + call, nfields=2)
                fin = lat.new_field(prec, nrhs=2)
                ref = lat.new_field(prec, nrhs=2)
                got = lat.new_field(prec, nrhs=2)
                a = lat.canonical_spinor(nrhs=2)
                b = lat.canonical_spinor(nrhs=2)
                lat.pack(fin, psi, 1, prec, nrhs=2)
                lat.dslash(ref, fin, 1, kappa, csw, op=lq.OP_SCHUR, dag=dag, prec=prec, nrhs=2)
                torch.cuda.synchronize()
                ws_before = lat.workspace.clone()
                torch.cuda.synchronize()
                # torch's count of allocation requests, and the device's free
                # memory (the first call may load the library's module on the
                # device, with its 32 MiB array: compared from the second call)
                nalloc = torch.cuda.memory_stats()["allocation.all.allocated"]
                free_before = torch.cuda.mem_get_info()[0]
                lq.lqcd_dslash_schur_static(lat.ctx, got, fin, kappa, csw, dag, prec, nrhs=2)
                torch.cuda.synchronize()
                assert torch.cuda.memory_stats()["allocation.all.allocated"] == nalloc
                if call == 1:
                    assert torch.cuda.mem_get_info()[0] >= free_before
                assert torch.equal(lat.workspace, ws_before), "the static call wrote into the workspace"
                del ws_before
                lat.unpack(a, ref, 1, prec, nrhs=2)
                lat.unpack(b, got, 1, prec, nrhs=2)
                torch.cuda.synchronize()
                a, b = a.cpu().numpy(), b.cpu().numpy()
                assert np.linalg.norm(a) > 0
                assert rel(b, a) <= TOL[prec], (prec, dag, call)
                if call == 1 or prec == "f64":
                    for r in range(2):
                        want = oracle.schur(U, A, Ainv, kappa, restrict(psi[r], dims, 1), dag=dag)
                        want = restrict(want, dims, 1)
                        assert rel(b[r], want) <= TOL_ORACLE[prec], (prec, dag, call, r)


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
