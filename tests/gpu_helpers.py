"""Shared helpers of the GPU parity tests (host side only: reference values
come from the FP64 CPU oracle, inputs from the seeded generators)."""
import numpy as np
import pytest

import oracle
import synth


def require_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test run without a CUDA device")
    from paper_1103_1363_gb300 import lqcd  # raises if liblqcd.so is missing
    return lqcd


def parity_mask(dims):
    lx, ly, lz, lt = dims
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
    return (x + y + z + t) % 2


def restrict(psi, dims, parity):
    out = psi.copy()
    out[..., parity_mask(dims) != parity, :, :] = 0
    return out


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def hop_ref(U, psi, dims, out_parity, dag=False):
    """Oracle H_{p,1-p} (dag: g5 H g5) restricted to parities."""
    src = restrict(psi, dims, 1 - out_parity)
    if dag:
        out = oracle.gamma5(oracle.hop(U, oracle.gamma5(src)))
    else:
        out = oracle.hop(U, src)
    return restrict(out, dims, out_parity)


def gauge(dims, kind="smooth", seed=1, eps=0.5):
    return synth.gauge_field(dims, kind, seed, eps=eps)


def gpu_apply(lat, fn_prec, psi, in_parity, out_parity, run, full=False):
    """Pack psi (one parity, or full), run(out_field, in_field), unpack."""
    import torch
    fin = lat.new_field(fn_prec, full=full)
    fout = lat.new_field(fn_prec, full=full)
    fout.zero_()
    lat.pack(fin, psi, -1 if full else in_parity, fn_prec)
    run(fout, fin)
    out = lat.canonical_spinor()
    lat.unpack(out, fout, -1 if full else out_parity, fn_prec)
    torch.cuda.synchronize()
    return out.cpu().numpy()
