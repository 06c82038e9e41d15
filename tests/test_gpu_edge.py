"""Degenerate inputs of the solvers, through the C ABI on the GPU:

- b = 0: every solver returns x = 0 exactly, with status OK and no
  iteration (|b - M x| = 0 already).
- b = M x* for a plane wave x* on a unit-link lattice without clover: the
  Krylov space of b is one-dimensional for FGCR / FGMRES (M b is parallel
  to b), so they converge in one iteration (the invariant-subspace case of
  GMRES); CG on the normal equations reaches r = 0 after one iteration and
  must survive the remaining iterations of its check interval (0/0 steps).
- 16-bit spinor storage with per-site norms keeps sites whose values are
  subnormal in FP32 from turning into NaN (stored as zero).
- The smallest lattice (2^4, where x + mu and x - mu coincide) solves to
  1e-10 with every solver, checked by the oracle.  Its rough Haar links make
  the normal equations so ill-conditioned that 16-bit search directions
  stagnate (|r|/|r0| ~ 2e-4); the CG then switches its inner storage to FP32
  and says so in the stats.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests.gpu_helpers import require_cuda

pytestmark = pytest.mark.gpu

SOLVERS = [("cg_eo", dict(inner_prec="f32")), ("cg_eo_f16spinors", dict(inner_prec="f16spinors")),
           ("cg_full", dict(solver=1, inner_prec="f32")), ("fgcr", dict(solver=2, inner_prec="f32", nkrylov=8)),
           ("fgmres_dr", dict(solver=3, inner_prec="f32", nkrylov=8, ndefl=2))]


@pytest.fixture(scope="module")
def lq():
    return require_cuda()


@pytest.mark.parametrize("name,kw", SOLVERS, ids=[s[0] for s in SOLVERS])
def test_zero_source(lq, name, kw):
    dims = (4, 4, 4, 8)
    lat = lq.Lattice(dims, gcr_nkrylov=8)
    lat.gauge_load(synth.smooth_gauge(dims, 0.5, 71))
    lat.clover_compute(0.13, 1.0)
    x = lat.canonical_spinor()
    x.fill_(7.0)
    rc, st = lat.solve(x, torch.zeros_like(x), 1e-10, **kw)
    assert rc == 0 and st["iterations"] == 0
    assert not torch.any(x)


@pytest.mark.parametrize("name,kw", SOLVERS, ids=[s[0] for s in SOLVERS])
def test_plane_wave_source(lq, name, kw):
    """Free field (unit links, csw 0, periodic in t): a plane wave of
    momentum p with a fixed spinor u is an eigenvector of the hopping term
    only if u is an eigenvector of the momentum's gamma combination; a zero
    momentum wave is one for any u: H psi = 8 psi, M psi = (1 - 8 kappa) psi."""
    dims = (4, 4, 4, 4)
    kappa = 0.1
    U = synth.unit_gauge(dims)
    u = synth.gaussian_spinor((1, 1, 1, 1), 72)[0, 0, 0, 0]
    xstar = np.broadcast_to(u, dims + (4, 3)).copy()
    b = oracle.wilson_clover(U, None, kappa, xstar, tanti=0)
    assert np.allclose(b, (1 - 8 * kappa) * xstar)
    lat = lq.Lattice(dims, t_antiperiodic=0, gcr_nkrylov=8)
    lat.gauge_load(U)
    lat.clover_compute(kappa, 0.0)
    x = lat.canonical_spinor()
    rc, st = lat.solve(x, torch.from_numpy(b).cuda(), 1e-10, **kw)
    xg = x.cpu().numpy()
    assert rc == 0
    assert np.linalg.norm(xg - xstar) / np.linalg.norm(xstar) < 1e-10
    if name.startswith("fg"):  # CG checks its residual only every check_interval iterations
        assert st["iterations"] <= 2, st["iterations"]


@pytest.mark.parametrize("prec", ["f16spinors", "bf16spinors", "f16", "bf16"])
def test_subnormal_sites_in_16bit_spinors(lq, prec):
    """Per-site-norm codec: a site whose largest component is below the
    smallest normal FP32 number (2^-126) is stored as zero.  Dividing by
    its norm overflowed to infinity and made the site NaN, which broke
    FP16-spinor solves of point sources at 24^3x48.  Normal sites keep
    16-bit accuracy relative to their own norm, down to 1e-36."""
    dims = (4, 4, 4, 4)
    lat = lq.Lattice(dims, precisions=("f64", "f32", prec))
    b = synth.gaussian_spinor(dims, 76)
    exps = [0, 5, 10, 20, 30, 36, 39, 41, 43]
    lt, lz, ly, lx = b.shape[:4]
    scale = np.empty((lt, lz, ly, lx))
    for n, idx in enumerate(np.ndindex(lt, lz, ly, lx)):
        scale[idx] = 10.0 ** -exps[n % len(exps)]
    b = b * scale[..., None, None]
    f = lat.new_field(prec)
    lat.pack(f, b, 1, prec)
    out = torch.zeros(b.shape, dtype=torch.complex128, device="cuda")
    lat.unpack(out, f, 1, prec)
    u = out.cpu().numpy()
    assert np.all(np.isfinite(u))
    t, z, y, x = np.indices((lt, lz, ly, lx))
    odd = ((t + z + y + x) & 1) == 1
    vmax = np.abs(b).reshape(lt, lz, ly, lx, -1).max(axis=-1)
    err = np.abs(u - b).reshape(lt, lz, ly, lx, -1).max(axis=-1)
    tol = 2.0 ** -10 if prec.startswith("f16") else 2.0 ** -7
    normal = odd & (vmax > 1e-36)
    tiny = odd & (vmax < 1e-38)
    assert normal.sum() > 0 and tiny.sum() > 0
    assert np.all(err[normal] <= tol * vmax[normal])
    assert np.all(u.reshape(lt, lz, ly, lx, -1)[tiny] == 0)


@pytest.mark.parametrize("name,kw", SOLVERS, ids=[s[0] for s in SOLVERS])
def test_smallest_lattice(lq, name, kw):
    dims = (2, 2, 2, 2)
    kappa, csw = 0.12, 1.0
    U = synth.haar_gauge(dims, 73)
    A = oracle.clover(U, kappa, csw)
    b = synth.gaussian_spinor(dims, 74)
    lat = lq.Lattice(dims, gcr_nkrylov=8)
    lat.gauge_load(U)
    lat.clover_compute(kappa, csw)
    x = lat.canonical_spinor()
    rc, st = lat.solve(x, torch.from_numpy(b).cuda(), 1e-10, **kw)
    assert rc == 0
    assert oracle.true_residual(U, A, kappa, b, x.cpu().numpy()) <= 1e-10
    assert st["precision_fallback"] == (1 if "f16" in name else 0)


def test_singular_clover_block_reported(lq):
    """csw = 1 / (kappa sin theta) in a constant abelian field makes the clover
    matrix singular on every site (the oracle's inverse reports all of them,
    tests/test_oracle_pins.py); lqcd_clover_compute returns
    LQCD_ERR_CLOVER_SINGULAR and lqcd_sync reports it too.  At 90 % of that
    csw the build succeeds and A^{-1} matches the oracle."""
    dims = (4, 4, 6, 8)
    U = synth.constant_abelian_gauge(dims, 0, 1, 1)
    kappa = 0.13
    csw = 1.0 / (kappa * np.sin(2 * np.pi / dims[0]))
    lat = lq.Lattice(dims, precisions=("f64", "f32"))
    lat.gauge_load(U)
    with pytest.raises(lq.LqcdError) as e:
        lat.clover_compute(kappa, csw)
    assert e.value.status == 8
    with pytest.raises(lq.LqcdError) as e:
        lat.sync()
    assert e.value.status == 8
    lat.clover_compute(kappa, 0.9 * csw)
    lat.sync()
    psi = synth.gaussian_spinor(dims, 77)
    fin, fout = lat.new_field("f64"), lat.new_field("f64")
    lat.pack(fin, psi, 1, "f64")
    lat.clover_apply(fout, fin, 1, True, prec="f64")
    out = lat.canonical_spinor()
    lat.unpack(out, fout, 1, "f64")
    torch.cuda.synchronize()
    Ainv, bad = oracle.invert_site_matrices(oracle.clover(U, kappa, 0.9 * csw))
    assert bad == 0
    t, z, y, x = np.indices(dims[::-1])
    odd = (((t + z + y + x) & 1) == 1)[..., None, None]
    want = oracle.apply_site_matrices(Ainv, np.where(odd, psi, 0))
    got = out.cpu().numpy()
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 1e-12


def test_entry_points_restore_the_current_device(lq):
    """Every call makes the context's device current and then gives the
    caller's current device back (needs two GPUs to observe)."""
    if torch.cuda.device_count() < 2:
        pytest.skip("one GPU: the context's device is always the current one")
    dims = (4, 4, 4, 4)
    lat = lq.Lattice(dims, device="cuda:1", precisions=("f64", "f32"))
    torch.cuda.set_device(0)
    lat.gauge_load(synth.smooth_gauge(dims, 0.5, 78))
    assert torch.cuda.current_device() == 0
    lat.clover_compute(0.13, 1.0)
    assert torch.cuda.current_device() == 0


def test_fma_peak_measures_and_validates(lq):
    """lqcd_fma_peak returns positive multiply-add rates (FP64 below FP32, a
    packed pair at least the scalar rate within noise) and rejects an
    unknown kind."""
    f32 = lq.lqcd_fma_peak(0, 0)
    f32x2 = lq.lqcd_fma_peak(0, 1)
    f64 = lq.lqcd_fma_peak(0, 2)
    assert f32 > 1.0 and f64 > 0.0 and f64 < f32
    assert f32x2 > 0.8 * f32
    with pytest.raises(lq.LqcdError):
        lq.lqcd_fma_peak(0, 3)
