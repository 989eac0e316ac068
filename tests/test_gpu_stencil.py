"""GPU parity of the nearest-neighbour operations (Sec. 6, Summary and Outlook: Cshift, the
colour part of the Dslash hopping term and the Wilson hopping term with spin) against the CPU
oracle.

  * su3s_cshift is a copy of stored objects: its stored values are bit exact
    against the oracle's shift of the source's stored values (computed from the
    host data by the oracle's rounding; rows 0 and 1 for two-row matrices), in
    every storage format and layout.
  * su3s_hop: FP64 storage; native FP64 and fixed point within 1e-13, the
    pair arithmetic within 8e-13 (8 products of up to 6 terms each, operands
    of magnitude <= 1), per real component.
  * su3s_dslash (spinors as colour-vector fields with 4 spin components):
    FP64 storage, spinor components of magnitude <= 1; native FP64 and fixed
    point within 2e-13, the pair arithmetic within 1.6e-12 (each output
    real sums 8 half-spinor products of magnitude <= 6, each with the pair
    arithmetic's ~2^-46 relative error of its 6 terms), per real component.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from helpers import cplx

pytestmark = pytest.mark.gpu

SEED = synth.SEED_BASE + 21
TOL = 1e-13
DIMS = [(3, 2, 5, 4), (1, 3, 1, 2), (8, 8, 8, 9)]
LAYOUTS = [("soa", 0, 0), ("aosoa4", 1, 4), ("aosoa32", 1, 32)]


@pytest.fixture(scope="module")
def su3s(gpu_lib):
    return gpu_lib


def field(su3s, lat, kind, nmu, prec, lay, arr):
    f = su3s.Field(lat, kind, nmu, prec, lay[1], lay[2] or 64)
    f.upload(arr)
    return f


def host(kind, n, fid):
    if kind == "matrix":
        return synth.su3(SEED, fid, n)
    if kind == "vector":
        return synth.gauss_vector(SEED, fid, n)
    return synth.uniform_real(SEED, fid, n)


def stored_values(arr, prec):
    """The values a field of format `prec` stores for the canonical array `arr`,
    from the oracle: rows 0, 1 of two-row matrices, rounded to the format."""
    x = arr
    if prec in ("F64_C12", "F32_C12"):
        x = arr.reshape(-1, 3, 3, 2)[:, :2]
    fmt = {"F32": "f32", "F32_C12": "f32", "BF16": "bf16", "F16": "f16"}.get(prec)
    x = np.ascontiguousarray(x)
    return oracle.round_to(x, fmt) if fmt else x


@pytest.mark.parametrize("dims", DIMS)
@pytest.mark.parametrize("lay", LAYOUTS, ids=lambda x: x[0])
@pytest.mark.parametrize("kind,prec,nmu", [
    ("matrix", "F64", 1), ("matrix", "F64", 4), ("vector", "F64", 1), ("real", "F64", 1),
    ("matrix", "F32", 4), ("matrix", "BF16", 1), ("matrix", "F64_C12", 1), ("vector", "F16", 1)])
def test_cshift_is_exact(su3s, dims, lay, kind, prec, nmu):
    lat = su3s.Lattice(dims)
    v = synth.volume(dims)
    K = {"matrix": su3s.MATRIX, "vector": su3s.VECTOR, "real": su3s.REAL}[kind]
    h = host(kind, v * nmu, 0)
    src = field(su3s, lat, K, nmu, getattr(su3s, prec), lay, h)
    ref_in = stored_values(h, prec).reshape(v, -1)
    dst = src.like()
    for dim in range(4):
        for shift in (1, -1, 2, -5, dims[dim]):
            su3s.cshift(dst, src, dim, shift)
            got = dst.download_stored().double().numpy().reshape(v, -1)
            assert np.array_equal(got, oracle.cshift(ref_in, dims, dim, shift)), (dim, shift)


@pytest.mark.parametrize("dims", DIMS)
@pytest.mark.parametrize("lay", LAYOUTS, ids=lambda x: x[0])
@pytest.mark.parametrize("kind", ["vector", "matrix"])
@pytest.mark.parametrize("math", [1, 2, 3], ids=["f64", "df32", "fx"])
def test_hop_matches_oracle(su3s, dims, lay, kind, math):
    lat = su3s.Lattice(dims)
    v = synth.volume(dims)
    u = synth.su3(SEED, 1, 4 * v)
    x = host(kind, v, 2)
    x = x / np.abs(x).max()                      # operand magnitudes <= 1
    K = su3s.MATRIX if kind == "matrix" else su3s.VECTOR
    U = field(su3s, lat, su3s.MATRIX, 4, su3s.F64, lay, u)
    X = field(su3s, lat, K, 1, su3s.F64, lay, x)
    Z = X.like()
    su3s.hop(Z, U, X, math)
    ref = oracle.hop(u, x, dims)
    tol = 8 * TOL if math == 2 else TOL
    assert np.abs(Z.download() - ref).max() < tol


def test_hop_is_hermitian_on_gpu(su3s):
    """<a, H b> = <H a, b>: the backward links are daggered and taken at x - mu."""
    dims = (8, 6, 4, 10)
    lat = su3s.Lattice(dims)
    v = synth.volume(dims)
    U = field(su3s, lat, su3s.MATRIX, 4, su3s.F64, LAYOUTS[0], synth.su3(SEED, 1, 4 * v))
    a = field(su3s, lat, su3s.VECTOR, 1, su3s.F64, LAYOUTS[0], synth.gauss_vector(SEED, 3, v))
    b = field(su3s, lat, su3s.VECTOR, 1, su3s.F64, LAYOUTS[0], synth.gauss_vector(SEED, 4, v))
    Ha, Hb = a.like(), b.like()
    su3s.hop(Ha, U, a, 3)
    su3s.hop(Hb, U, b, 3)
    lhs = np.vdot(cplx(a.download()), cplx(Hb.download()))
    rhs = np.vdot(cplx(Ha.download()), cplx(b.download()))
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)
    assert su3s.device_error() == 0


@pytest.mark.parametrize("kind", ["vector", "matrix"])
def test_hop_full_size_48(su3s, kind):
    """The 48^4 lattice the stencil study times (default arithmetic), against
    the oracle's hopping term over the whole lattice, on sampled sites and the
    first and last site."""
    dims = (48, 48, 48, 48)
    lat = su3s.Lattice(dims)
    v = synth.volume(dims)
    u = synth.su3(SEED, 1, 4 * v)
    x = host(kind, v, 2)
    x = x / np.abs(x).max()
    K = su3s.MATRIX if kind == "matrix" else su3s.VECTOR
    U = field(su3s, lat, su3s.MATRIX, 4, su3s.F64, LAYOUTS[0], u)
    X = field(su3s, lat, K, 1, su3s.F64, LAYOUTS[0], x)
    Z = X.like()
    su3s.hop(Z, U, X)
    rng = np.random.default_rng(21)
    idx = np.unique(np.concatenate([rng.choice(v, 3000, replace=False), [0, v - 1]]))
    got = Z.unpack()[torch.from_numpy(idx).cuda()].cpu().numpy()
    del U, X, Z
    torch.cuda.empty_cache()
    ref = oracle.hop(u, x, dims)[idx]
    assert np.abs(got - ref).max() < 8 * TOL


# ------------------------------------------ Wilson hopping term with spin
def spinor(n_sites, fid, seed=SEED):
    x = synth.gauss_vector(seed, fid, 4 * n_sites).reshape(n_sites, 4, 3, 2)
    return x / np.abs(x).max()                   # components of magnitude <= 1


DSLASH_TOL = {1: 2 * TOL, 2: 16 * TOL, 3: 2 * TOL}


@pytest.mark.parametrize("dims", DIMS + [(1, 1, 1, 1), (2, 2, 2, 2)])
@pytest.mark.parametrize("lay", LAYOUTS, ids=lambda x: x[0])
@pytest.mark.parametrize("math", [1, 2, 3], ids=["f64", "df32", "fx"])
def test_dslash_matches_oracle(su3s, dims, lay, math):
    lat = su3s.Lattice(dims)
    v = synth.volume(dims)
    u = synth.su3(SEED, 1, 4 * v)
    psi = spinor(v, 2)
    U = field(su3s, lat, su3s.MATRIX, 4, su3s.F64, lay, u)
    P = field(su3s, lat, su3s.VECTOR, 4, su3s.F64, lay, psi.reshape(4 * v, 3, 2))
    Z = P.like()
    su3s.dslash(Z, U, P, math)
    ref = oracle.dslash(u, psi, dims).reshape(4 * v, 3, 2)
    assert np.abs(Z.download() - ref).max() < DSLASH_TOL[math]


def test_dslash_is_gamma5_hermitian_on_gpu(su3s):
    """<a, D b> = <g5 D g5 a, b> with the GPU's D: the projectors' signs, the
    daggered backward links and the gamma basis together."""
    dims = (8, 6, 4, 10)
    lat = su3s.Lattice(dims)
    v = synth.volume(dims)
    U = field(su3s, lat, su3s.MATRIX, 4, su3s.F64, LAYOUTS[0], synth.su3(SEED, 1, 4 * v))
    a, b = spinor(v, 3), spinor(v, 4)
    g5 = np.array([1.0, 1.0, -1.0, -1.0])[None, :, None, None]
    A = field(su3s, lat, su3s.VECTOR, 4, su3s.F64, LAYOUTS[0], (g5 * a).reshape(4 * v, 3, 2))
    B = field(su3s, lat, su3s.VECTOR, 4, su3s.F64, LAYOUTS[0], b.reshape(4 * v, 3, 2))
    DA, DB = A.like(), B.like()
    su3s.dslash(DA, U, A, 1)
    su3s.dslash(DB, U, B, 1)
    lhs = np.vdot(cplx(a.reshape(4 * v, 3, 2)), cplx(DB.download()))
    rhs = np.vdot(cplx((g5 * DA.download().reshape(v, 4, 3, 2)).reshape(4 * v, 3, 2)),
                  cplx(b.reshape(4 * v, 3, 2)))
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)
    assert su3s.device_error() == 0


def test_dslash_full_size_48(su3s):
    """The 48^4 lattice the stencil study times (default arithmetic, default
    launch), against the oracle's Wilson term over the whole lattice, on
    sampled sites and the first and last site."""
    dims = (48, 48, 48, 48)
    lat = su3s.Lattice(dims)
    v = synth.volume(dims)
    u = synth.su3(SEED, 1, 4 * v)
    psi = spinor(v, 2)
    U = field(su3s, lat, su3s.MATRIX, 4, su3s.F64, LAYOUTS[0], u)
    P = field(su3s, lat, su3s.VECTOR, 4, su3s.F64, LAYOUTS[0], psi.reshape(4 * v, 3, 2))
    Z = P.like()
    su3s.dslash(Z, U, P)
    rng = np.random.default_rng(22)
    idx = np.unique(np.concatenate([rng.choice(v, 3000, replace=False), [0, v - 1]]))
    got = Z.unpack().reshape(v, 4, 3, 2)[torch.from_numpy(idx).cuda()].cpu().numpy()
    del U, P, Z
    torch.cuda.empty_cache()
    ref = oracle.dslash(u, psi, dims)[idx]
    assert np.abs(got - ref).max() < DSLASH_TOL[2]
