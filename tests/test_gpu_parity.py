"""Parity of the CUDA path with the CPU oracle, through the C ABI.

Tolerances:
  * FP64 storage (native FP64, pair-of-FP32 or fixed-point arithmetic): 1e-13 per real
    component for products of SU(3) matrices (sum_t |x_t y_t| <= 1 there); for
    Gaussian operands the same bound scaled by max(1, sum_t |x_t y_t|).
  * FP32/BF16/FP16 storage with FP32 accumulation: against the oracle that
    rounds the inputs to the format, multiplies in FP64 and rounds the output,
    at most one unit in the last place of the output format plus 8*2^-24.
  * Integer/layout work (pack/unpack, copies): bit-exact.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from helpers import BOUND_VS_F64, E1, E2, E3, ULP, cplx, lattice_fields

pytestmark = pytest.mark.gpu

SEED = synth.SEED_BASE
TOL = 1e-13
# arithmetics for FP64 storage: native FP64, pair of FP32, shared-exponent fixed point
MATHS = [1, 2, 3]
MATH_IDS = ["f64", "df32", "fx"]
DIMS = [(1, 1, 1, 1), (2, 2, 2, 2), (3, 2, 1, 5), (6, 5, 7, 3), (8, 8, 8, 8)]
LAYOUTS = [("soa", 0, 0), ("aosoa4", 1, 4), ("aosoa32", 1, 32), ("aosoa128", 1, 128)]


def layout_id(x):
    return x[0]


@pytest.fixture(scope="module")
def su3s(gpu_lib):
    return gpu_lib


def upload(su3s, lat, arr, kind=None, nmu=1, prec=None, layout=0, block=0):
    kind = su3s.MATRIX if kind is None else kind
    prec = su3s.F64 if prec is None else prec
    f = su3s.Field(lat, kind, nmu, prec, layout, block or 64)
    f.upload(arr)
    return f


def tree_expr(tree, fields):
    op = tree[0]
    if op == "leaf":
        return fields[tree[1]].expr()
    if op == "mul":
        return tree_expr(tree[1], fields) * tree_expr(tree[2], fields)
    if op == "add":
        return tree_expr(tree[1], fields) + tree_expr(tree[2], fields)
    if op == "sub":
        return tree_expr(tree[1], fields) - tree_expr(tree[2], fields)
    if op == "scale":
        return float(tree[1]) * tree_expr(tree[2], fields)
    return tree_expr(tree[1], fields).adj()


# ------------------------------------------------------------------ products
@pytest.mark.parametrize("math", MATHS, ids=MATH_IDS)
@pytest.mark.parametrize("lay", LAYOUTS, ids=layout_id)
@pytest.mark.parametrize("dims", DIMS, ids=str)
def test_mm(su3s, dims, lay, math):
    lat = su3s.Lattice(dims)
    f = lattice_fields(dims, SEED)
    a = upload(su3s, lat, f["a"], layout=lay[1], block=lay[2])
    b = upload(su3s, lat, f["b"], layout=lay[1], block=lay[2])
    z = a.like()
    su3s.evaluate(z, a * b, math)
    err = np.abs(z.download() - oracle.mm(f["a"], f["b"])).max()
    assert err < TOL


@pytest.mark.parametrize("math", MATHS, ids=MATH_IDS)
@pytest.mark.parametrize("lay", LAYOUTS[:2], ids=layout_id)
@pytest.mark.parametrize("dims", [(3, 2, 1, 5), (8, 8, 8, 8)], ids=str)
def test_mv(su3s, dims, lay, math):
    lat = su3s.Lattice(dims)
    f = lattice_fields(dims, SEED, names=("a", "v"))
    a = upload(su3s, lat, f["a"], layout=lay[1], block=lay[2])
    v = upload(su3s, lat, f["v"], kind=su3s.VECTOR, layout=lay[1], block=lay[2])
    z = v.like()
    su3s.evaluate(z, a * v, math)
    ref = oracle.mv(f["a"], f["v"])
    scale = max(1.0, np.abs(cplx(f["v"])).sum(axis=1).max())
    assert np.abs(z.download() - ref).max() < TOL * scale


@pytest.mark.parametrize("math", MATHS, ids=MATH_IDS)
@pytest.mark.parametrize("lay", [LAYOUTS[0], LAYOUTS[2]], ids=layout_id)
def test_lorentz_links(su3s, lay, math):
    dims = (6, 5, 7, 3)
    lat = su3s.Lattice(dims)
    f = lattice_fields(dims, SEED, nmu=4)
    a = upload(su3s, lat, f["a"], nmu=4, layout=lay[1], block=lay[2])
    b = upload(su3s, lat, f["b"], nmu=4, layout=lay[1], block=lay[2])
    z = a.like()
    su3s.evaluate(z, a * b, math)
    assert np.abs(z.download() - oracle.mm(f["a"], f["b"])).max() < TOL


@pytest.mark.parametrize("layout,block", [(0, 0), (1, 1024)], ids=["soa", "aosoa1024"])
def test_largest_link_count_and_site_block(su3s, layout, block):
    """The API's limits of the field shape: 8 objects per site, and the largest
    site block (1024, more than the lattice's 630 sites: one padded block), for
    a product, a fused tree and its reverse mode."""
    dims = (6, 5, 7, 3)
    v = synth.volume(dims)
    lat = su3s.Lattice(dims)
    f = lattice_fields(dims, SEED + 11, nmu=8, names=("a", "b", "c", "d", "w"))
    F = {n: upload(su3s, lat, f[n], nmu=8, layout=layout, block=block) for n in "abcdw"}
    z = F["a"].like()
    su3s.evaluate(z, F["a"] * F["b"])
    assert np.abs(z.download() - oracle.mm(f["a"], f["b"])).max() < TOL
    su3s.evaluate(z, F["a"] * F["b"] + F["c"] * F["d"])
    assert np.abs(z.download() - oracle.eval_tree(E1, f)).max() < 2 * TOL
    grads = [F["a"].like() for _ in range(4)]
    su3s.eval_adjoint(F["a"] * F["b"] + F["c"] * F["d"], F["w"], grads)
    ref = oracle.eval_adjoint(E1, {n: f[n] for n in "abcd"}, f["w"])
    wscale = np.abs(f["w"]).max() * 3
    for n, g in zip("abcd", grads):
        assert np.abs(g.download() - ref[n]).max() < TOL * wscale, n


@pytest.mark.parametrize("math", MATHS, ids=MATH_IDS)
def test_gaussian_operands(su3s, math):
    dims = (6, 5, 7, 3)
    v = synth.volume(dims)
    lat = su3s.Lattice(dims)
    ga, gb = synth.gauss_matrix(SEED, 0, v), synth.gauss_matrix(SEED, 1, v)
    a, b = upload(su3s, lat, ga), upload(su3s, lat, gb)
    z = a.like()
    su3s.evaluate(z, a * b, math)
    scale = np.einsum("nij,njk->nik", np.abs(cplx(ga)), np.abs(cplx(gb)))   # sum_j |a_ij||b_jk|
    err = np.abs(cplx(z.download()) - cplx(oracle.mm(ga, gb)))
    assert (err <= TOL * np.maximum(1.0, 2 * scale)).all()


def test_dest_aliases_leaf(su3s):
    dims = (6, 5, 7, 3)
    lat = su3s.Lattice(dims)
    f = lattice_fields(dims, SEED)
    a, b = upload(su3s, lat, f["a"]), upload(su3s, lat, f["b"])
    su3s.evaluate(b, a * b)          # b <- a*b in place
    assert np.abs(b.download() - oracle.mm(f["a"], f["b"])).max() < TOL


def test_dest_aliases_leaf_every_pipeline(su3s):
    """A destination that is one of the tree's leaves, in every data-movement
    mode, with many tiles per warp (the staged kernels fetch the next tile
    while the current one is stored): c <- a*b + c*d, and a <- adj(a)*b - b*adj(a),
    which reads the overwritten leaf twice."""
    dims = (16, 16, 16, 18)          # a volume of its own: the forced launch stays here
    lat = su3s.Lattice(dims)
    f = lattice_fields(dims, SEED + 12, names=("a", "b", "c", "d"))
    ref1, ref3 = oracle.eval_tree(E1, f), oracle.eval_tree(E3, f)
    try:
        for mode in (su3s.PIPE_PLAIN, su3s.PIPE_TMA, su3s.PIPE_TMA_LEAF, su3s.PIPE_TMA_RING,
                     su3s.PIPE_TMA_PAIR):
            su3s.set_pipeline(mode)
            F = {n: upload(su3s, lat, f[n]) for n in "abcd"}
            e1 = F["a"] * F["b"] + F["c"] * F["d"]
            su3s.set_launch(F["c"], e1, 32, 1)        # 152 one-warp blocks: ~15 tiles each
            su3s.evaluate(F["c"], e1)
            assert np.abs(F["c"].download() - ref1).max() < 2 * TOL, mode
            e3 = F["a"].adj() * F["b"] - F["b"] * F["a"].adj()
            su3s.set_launch(F["a"], e3, 32, 1)
            su3s.evaluate(F["a"], e3)
            assert np.abs(F["a"].download() - ref3).max() < 2 * TOL, mode
    finally:
        su3s.set_pipeline(su3s.PIPE_AUTO)
    assert su3s.device_error() == 0


def test_zero_and_identity_inputs(su3s):
    dims = (3, 2, 1, 5)
    lat = su3s.Lattice(dims)
    v = synth.volume(dims)
    eye = np.zeros((v, 3, 3, 2))
    eye[:, [0, 1, 2], [0, 1, 2], 0] = 1.0
    f = lattice_fields(dims, SEED)
    for math in MATHS:
        a, i = upload(su3s, lat, f["a"]), upload(su3s, lat, eye)
        z = a.like()
        su3s.evaluate(z, a * i, math)
        if math == 1:   # native FP64: multiplying by the identity is exact
            assert np.array_equal(z.download() + 0.0, f["a"] + 0.0)
        else:           # pair arithmetic and fixed point carry >= 48 significant bits
            assert np.abs(z.download() - f["a"]).max() <= 2.0 ** -46
        zero = upload(su3s, lat, np.zeros_like(eye))
        su3s.evaluate(z, a * zero, math)
        assert np.array_equal(z.download() + 0.0, np.zeros_like(eye))


# -------------------------------------------------------------- fused trees
@pytest.mark.parametrize("math", MATHS, ids=MATH_IDS)
@pytest.mark.parametrize("name,tree", [("E1", E1), ("E2", E2), ("E3", E3)], ids=["E1", "E2", "E3"])
@pytest.mark.parametrize("lay", [LAYOUTS[0], LAYOUTS[2]], ids=layout_id)
def test_fused_trees(su3s, name, tree, lay, math):
    dims = (6, 5, 7, 3)
    lat = su3s.Lattice(dims)
    names = oracle.leaf_names(tree)
    f = lattice_fields(dims, SEED, names=tuple(names))
    fields = {n: upload(su3s, lat, f[n], layout=lay[1], block=lay[2]) for n in names}
    e = tree_expr(tree, fields)
    assert e.signature() in {s for (_, s, p, m) in su3s.catalogue() if p == "f64"}
    z = fields[names[0]].like()
    su3s.evaluate(z, e, math)
    ref = oracle.eval_tree(tree, f)
    assert np.abs(z.download() - ref).max() < TOL * 2


COMM = ("sub", ("mul", ("leaf", "a"), ("leaf", "b")), ("mul", ("leaf", "b"), ("leaf", "a")))


@pytest.mark.parametrize("math", MATHS, ids=MATH_IDS)
def test_commutator_tree(su3s, math):
    """a*b - b*a, a catalogued tree whose two products share both leaves (the
    staged kernel forms its output row by row): every data movement gives the
    same bits, the oracle's value within the bound, a traceless result (the
    trace of a commutator vanishes), and exactly zero when b is the identity
    (both products then combine the same values)."""
    dims = (8, 8, 8, 9)
    lat = su3s.Lattice(dims)
    f = lattice_fields(dims, SEED, names=("a", "b"))
    a, b = (upload(su3s, lat, f[n]) for n in "ab")
    e = a * b - b * a
    assert e.signature() in {s for (_, s, p, m) in su3s.catalogue() if p == "f64"}
    outs = []
    try:
        for mode in (su3s.PIPE_PLAIN, su3s.PIPE_TMA, su3s.PIPE_TMA_LEAF, su3s.PIPE_TMA_RING,
                     su3s.PIPE_TMA_PAIR):
            su3s.set_pipeline(mode)
            z = a.like()
            su3s.evaluate(z, e, math)
            outs.append(z.download())
    finally:
        su3s.set_pipeline(su3s.PIPE_AUTO)
    for o in outs[1:]:
        assert np.array_equal(outs[0], o)
    ref = oracle.eval_tree(COMM, f)
    assert np.abs(outs[0] - ref).max() < 2 * TOL
    tr = cplx(outs[0])[:, [0, 1, 2], [0, 1, 2]].sum(axis=1)
    assert np.abs(tr).max() < 2 * TOL
    eye = np.zeros_like(f["a"])
    eye[:, [0, 1, 2], [0, 1, 2], 0] = 1.0
    i = upload(su3s, lat, eye)
    z = a.like()
    su3s.evaluate(z, a * i - i * a, math)
    assert np.array_equal(z.download() + 0.0, np.zeros_like(eye))
    assert su3s.device_error() == 0


@pytest.mark.parametrize("math", MATHS, ids=MATH_IDS)
def test_fused_equals_term_by_term_on_gpu(su3s, math):
    dims = (8, 8, 8, 8)
    lat = su3s.Lattice(dims)
    f = lattice_fields(dims, SEED, names=("a", "b", "c", "d"))
    F = {n: upload(su3s, lat, f[n]) for n in "abcd"}
    fused, t1, t2, tot = (F["a"].like() for _ in range(4))
    su3s.evaluate(fused, F["a"] * F["b"] + F["c"] * F["d"], math)
    su3s.evaluate(t1, F["a"] * F["b"], math)
    su3s.evaluate(t2, F["c"] * F["d"], math)
    su3s.evaluate(tot, t1 + t2, math)
    # two evaluations compared with each other: each is within the FP64
    # tolerance of the exact value
    tol = 2e-15 if math == 1 else TOL
    assert np.abs(fused.download() - tot.download()).max() < tol


@pytest.mark.parametrize("math", MATHS, ids=MATH_IDS)
def test_interpreter_for_uncatalogued_trees(su3s, math):
    dims = (6, 5, 7, 3)
    lat = su3s.Lattice(dims)
    f = lattice_fields(dims, SEED, names=("a", "b", "c", "d", "v"))
    F = {n: upload(su3s, lat, f[n], kind=(su3s.VECTOR if n == "v" else su3s.MATRIX)) for n in "abcdv"}
    trees = [
        ("sub", ("mul", ("add", ("mul", ("leaf", "a"), ("leaf", "b")), ("leaf", "c")),
                 ("adj", ("leaf", "d"))), ("scale", 2.5, ("leaf", "a"))),
        ("mul", ("adj", ("mul", ("leaf", "a"), ("leaf", "b"))), ("leaf", "v")),
        ("add", ("scale", -0.25, ("mul", ("leaf", "c"), ("leaf", "v"))),
         ("mul", ("leaf", "d"), ("mul", ("leaf", "a"), ("leaf", "v")))),
    ]
    cat = {s for (_, s, p, m) in su3s.catalogue()}
    for tree in trees:
        e = tree_expr(tree, F)
        assert e.signature() not in cat
        kind = su3s.VECTOR if tree[0] != "sub" else su3s.MATRIX
        z = F["v"].like() if kind == su3s.VECTOR else F["a"].like()
        su3s.evaluate(z, e, math)
        leaves = {n: f[n] for n in oracle.leaf_names(tree)}
        ref = oracle.eval_tree(tree, leaves)
        scale = max(1.0, np.abs(ref).max())
        assert np.abs(z.download() - ref).max() < 4 * TOL * scale


def test_listing2_real_fields(su3s):
    import os
    rows = [ln.split() for ln in open(os.path.join(os.path.dirname(__file__), "golden",
                                                   "listing2.txt"))
            if ln.strip() and not ln.startswith("#")]
    dims = (6, 5, 7, 3)
    v = synth.volume(dims)
    lat = su3s.Lattice(dims)
    for math in MATHS:
        for v1, v2, expr, v3 in rows:
            f1 = upload(su3s, lat, np.full(v, float(v1)), kind=su3s.REAL)
            f2 = upload(su3s, lat, np.full(v, float(v2)), kind=su3s.REAL)
            out = f1.like()
            e = f1 + f2 if expr == "v1+v2" else f1 + f2 + f1 * f2
            su3s.evaluate(out, e, math)
            assert np.array_equal(out.download(), np.full(v, float(v3)))


def test_real_field_trees_random(su3s):
    dims = (6, 5, 7, 3)
    v = synth.volume(dims)
    lat = su3s.Lattice(dims)
    r1, r2 = synth.uniform_real(SEED, 6, v), synth.uniform_real(SEED, 7, v)
    a, b = upload(su3s, lat, r1, kind=su3s.REAL), upload(su3s, lat, r2, kind=su3s.REAL)
    tree = ("add", ("add", ("leaf", "x"), ("leaf", "y")), ("mul", ("leaf", "x"), ("leaf", "y")))
    ref = oracle.eval_tree(tree, {"x": r1, "y": r2})
    for math in MATHS:
        z = a.like()
        su3s.evaluate(z, a + b + a * b, math)
        assert np.abs(z.download() - ref).max() < TOL


# ---------------------------------------------------------- reduced precision


@pytest.mark.parametrize("fmt", ["f32", "bf16", "f16"])
@pytest.mark.parametrize("lay", [LAYOUTS[0], LAYOUTS[1], LAYOUTS[2]], ids=layout_id)
@pytest.mark.parametrize("dims", [(3, 2, 1, 5), (8, 8, 8, 8), (16, 16, 16, 32)], ids=str)
def test_reduced_precision_mm(su3s, fmt, lay, dims):
    prec = {"f32": su3s.F32, "bf16": su3s.BF16, "f16": su3s.F16}[fmt]
    lat = su3s.Lattice(dims)
    f = lattice_fields(dims, SEED)
    a = upload(su3s, lat, f["a"], prec=prec, layout=lay[1], block=lay[2])
    b = upload(su3s, lat, f["b"], prec=prec, layout=lay[1], block=lay[2])
    z = a.like()
    su3s.evaluate(z, a * b)
    got = z.download()
    # oracle (i): inputs rounded to the format, FP64 product, output rounded
    ref_i = oracle.round_to(oracle.mm(oracle.round_to(f["a"], fmt), oracle.round_to(f["b"], fmt)), fmt)
    assert (np.abs(got - ref_i) <= ULP[fmt](ref_i) + 8 * 2.0 ** -24).all()
    # (ii) against the exact FP64 product: the a priori bound
    err = np.abs(got - oracle.mm(f["a"], f["b"])).max()
    assert err < BOUND_VS_F64[fmt]


@pytest.mark.parametrize("fmt", ["f32", "bf16", "f16"])
def test_reduced_precision_mv(su3s, fmt):
    prec = {"f32": su3s.F32, "bf16": su3s.BF16, "f16": su3s.F16}[fmt]
    dims = (6, 5, 7, 3)
    lat = su3s.Lattice(dims)
    f = lattice_fields(dims, SEED, names=("a", "v"))
    vv = f["v"] / 4.0   # keep FP16 far from overflow
    a = upload(su3s, lat, f["a"], prec=prec)
    v = upload(su3s, lat, vv, kind=su3s.VECTOR, prec=prec)
    z = v.like()
    su3s.evaluate(z, a * v)
    ref_i = oracle.round_to(oracle.mv(oracle.round_to(f["a"], fmt), oracle.round_to(vv, fmt)), fmt)
    assert (np.abs(z.download() - ref_i) <= ULP[fmt](ref_i) + 8 * 2.0 ** -24).all()


# ------------------------------------------------------------- two-row SU(3)
@pytest.mark.parametrize("math", MATHS, ids=MATH_IDS)
@pytest.mark.parametrize("lay", [LAYOUTS[0], LAYOUTS[2]], ids=layout_id)
def test_c12_f64(su3s, lay, math):
    dims = (6, 5, 7, 3)
    lat = su3s.Lattice(dims)
    f = lattice_fields(dims, SEED)
    a = upload(su3s, lat, f["a"], prec=su3s.F64_C12, layout=lay[1], block=lay[2])
    b = upload(su3s, lat, f["b"], prec=su3s.F64_C12, layout=lay[1], block=lay[2])
    z = a.like()
    su3s.evaluate(z, a * b, math)
    got = z.download()
    ea, eb = (oracle.c12_expand(f[n][:, :2].copy()) for n in "ab")
    ref = oracle.mm(ea, eb)
    assert np.abs(got[:, :2] - ref[:, :2]).max() < TOL            # stored rows
    assert np.abs(got - oracle.c12_expand(ref[:, :2].copy())).max() < TOL
    assert np.abs(got - oracle.mm(f["a"], f["b"])).max() < 1e-12


def test_c12_f32(su3s):
    dims = (6, 5, 7, 3)
    lat = su3s.Lattice(dims)
    f = lattice_fields(dims, SEED)
    a = upload(su3s, lat, f["a"], prec=su3s.F32_C12)
    b = upload(su3s, lat, f["b"], prec=su3s.F32_C12)
    z = a.like()
    su3s.evaluate(z, a * b)
    got = z.download()
    ra, rb = (oracle.round_to(f[n][:, :2].copy(), "f32") for n in "ab")
    ref = oracle.mm(oracle.c12_expand(ra), oracle.c12_expand(rb))
    # FP32 rebuild + FP32 accumulation: a few FP32 ulps of O(1) values
    assert np.abs(got[:, :2] - ref[:, :2]).max() < 3e-6
    assert np.abs(got - oracle.mm(f["a"], f["b"])).max() < 5e-6


# --------------------------------------------------------- pack and unpack
@pytest.mark.parametrize("prec,fmt", [(0, None), (1, "f32"), (2, "bf16"), (3, "f16")],
                         ids=["f64", "f32", "bf16", "f16"])
@pytest.mark.parametrize("lay", LAYOUTS, ids=layout_id)
def test_pack_unpack_roundtrip(su3s, prec, fmt, lay):
    dims = (3, 2, 1, 5)
    lat = su3s.Lattice(dims)
    f = lattice_fields(dims, SEED, nmu=4, names=("a", "v"))
    for kind, arr in ((su3s.MATRIX, f["a"]), (su3s.VECTOR, f["v"])):
        x = upload(su3s, lat, arr, kind=kind, nmu=4, prec=prec, layout=lay[1], block=lay[2])
        want = arr if fmt is None else oracle.round_to(arr, fmt)
        assert np.array_equal(x.download(), want)
        dev = torch.from_numpy(arr.copy()).cuda()
        y = x.like()
        y.pack(dev)
        assert torch.equal(y.unpack().cpu(), torch.from_numpy(want))


def test_pack_zeroes_pad_sites(su3s):
    dims = (3, 2, 1, 5)   # 30 sites, padded to 64
    lat = su3s.Lattice(dims)
    f = lattice_fields(dims, SEED)
    x = su3s.Field(lat, su3s.MATRIX, 1, su3s.F64, su3s.SOA)
    x.tensor.fill_(float("nan"))
    x.upload(f["a"])
    t = x.tensor.view(9, 64, 2)
    assert torch.all(t[:, 30:, :] == 0)
    assert not torch.isnan(t[:, :30, :]).any()


STORED = [(0, None, torch.float64), (1, "f32", torch.float32), (2, "bf16", torch.bfloat16),
          (3, "f16", torch.float16), (4, None, torch.float64), (5, "f32", torch.float32)]


def stored_of(arr, prec, fmt, dtype, kind):
    """Stored-format array of canonical `arr` computed from the oracle: rows 0,1
    for the two-row formats, values rounded to the storage format."""
    x = arr
    if prec in (4, 5):
        x = arr[:, :2].reshape(arr.shape[0], 6, 2)
    if fmt is not None:
        x = oracle.round_to(x, fmt)
    x = np.ascontiguousarray(x).reshape(arr.shape[0], -1, 2)
    return torch.from_numpy(x).to(dtype)   # exact: the values fit the format


@pytest.mark.parametrize("prec,fmt,dtype", STORED, ids=["f64", "f32", "bf16", "f16", "f64c12", "f32c12"])
@pytest.mark.parametrize("lay", LAYOUTS, ids=layout_id)
def test_stored_format_transfer(su3s, prec, fmt, dtype, lay):
    """Stored-format download of a packed field equals the oracle's rounding
    (bitwise); a stored-format upload unpacks to the oracle's widening (and row
    rebuild) and downloads to the same bytes."""
    dims = (3, 2, 1, 5)
    lat = su3s.Lattice(dims)
    f = lattice_fields(dims, SEED + 7, nmu=4, names=("a", "v"))
    cases = [(su3s.MATRIX, f["a"])] + ([] if prec >= 4 else [(su3s.VECTOR, f["v"])])
    for kind, arr in cases:
        x = upload(su3s, lat, arr, kind=kind, nmu=4, prec=prec, layout=lay[1], block=lay[2])
        want = stored_of(arr, prec, fmt, dtype, kind)
        got = x.download_stored()
        assert got.dtype == dtype and tuple(got.shape) == x.stored_shape
        assert torch.equal(got.view(torch.uint8), want.view(torch.uint8))
        y = x.like()
        y.tensor.fill_(255 if y.tensor.dtype == torch.uint8 else float("nan"))
        y.upload_stored(want)
        assert torch.equal(y.download_stored().view(torch.uint8), want.view(torch.uint8))
        canon = want.double().numpy()
        if prec in (4, 5):
            # rows 0,1 exact; row 2 rebuilt in FP64: each real part is a sum of
            # four products of values of modulus <= 1, so contraction and
            # summation order move it by at most 8 * 2^-53
            canon = oracle.c12_expand(canon.reshape(-1, 2, 3, 2))
            got = y.download()
            assert np.array_equal(got[:, :2], canon[:, :2])
            assert np.abs(got[:, 2] - canon[:, 2]).max() <= 8 * 2.0 ** -53
        else:
            assert np.array_equal(y.download(), canon.reshape(arr.shape))
        assert torch.equal(y.tensor, x.tensor)     # pad sites zeroed, same layout bytes


@pytest.mark.parametrize("prec,dtype", [(0, torch.float64), (2, torch.bfloat16), (5, torch.float32)],
                         ids=["f64", "bf16", "f32c12"])
def test_stored_transfer_moves_bytes_unchanged(su3s, prec, dtype):
    """Arbitrary bit patterns (NaN payloads, infinities, subnormals) survive an
    upload and download in the stored format."""
    dims = (6, 5, 7, 3)
    lat = su3s.Lattice(dims)
    x = su3s.Field(lat, su3s.MATRIX, 1, prec, su3s.AOSOA, 32)
    g = torch.Generator().manual_seed(SEED)
    nbytes = int(np.prod(x.stored_shape)) * torch.empty(0, dtype=dtype).element_size()
    raw = torch.randint(0, 256, (nbytes,), dtype=torch.uint8, generator=g)
    host = raw.view(dtype).view(x.stored_shape).pin_memory()
    st = torch.cuda.Stream()
    x.upload_stored(host, stream=st)
    out = torch.empty_like(host).pin_memory()
    x.download_stored(out=out, stream=st)
    st.synchronize()
    assert torch.equal(out.reshape(-1).view(torch.uint8), raw)


def test_stored_transfer_real_field(su3s):
    dims = (3, 2, 1, 5)
    lat = su3s.Lattice(dims)
    r = synth.uniform_real(SEED, 3, 30 * 2)
    x = su3s.Field(lat, su3s.REAL, 2, su3s.F64, su3s.SOA)
    x.upload_stored(torch.from_numpy(r))
    assert np.array_equal(x.download(), r)
    assert torch.equal(x.download_stored(), torch.from_numpy(r))


# ---------------------------------------------------------- reverse mode
@pytest.mark.parametrize("math", MATHS, ids=MATH_IDS)
@pytest.mark.parametrize("name,tree", [("MM", ("mul", ("leaf", "a"), ("leaf", "b"))), ("E1", E1),
                                       ("E2", E2), ("E3", E3)], ids=["MM", "E1", "E2", "E3"])
def test_adjoint_kernels(su3s, name, tree, math):
    dims = (6, 5, 7, 3)
    lat = su3s.Lattice(dims)
    names = oracle.leaf_names(tree)
    f = lattice_fields(dims, SEED, names=tuple(names) + ("w",))
    F = {n: upload(su3s, lat, f[n]) for n in names}
    G = upload(su3s, lat, f["w"])
    grads = [F[n].like() for n in names]
    su3s.eval_adjoint(tree_expr(tree, F), G, grads, math)
    ref = oracle.eval_adjoint(tree, {n: f[n] for n in names}, f["w"])
    wscale = np.abs(f["w"]).max() * 3
    for n, g in zip(names, grads):
        assert np.abs(g.download() - ref[n]).max() < TOL * wscale, n


E1SUB = ("sub", ("mul", ("leaf", "a"), ("leaf", "b")), ("mul", ("leaf", "c"), ("leaf", "d")))
E1LIN = ("add", ("scale", 0.75, ("mul", ("leaf", "a"), ("leaf", "b"))),
         ("scale", -1.5, ("mul", ("leaf", "c"), ("leaf", "d"))))


@pytest.mark.parametrize("math", MATHS, ids=MATH_IDS)
@pytest.mark.parametrize("name,tree", [("E1", E1), ("E1Sub", E1SUB), ("E1Lin", E1LIN)],
                         ids=["E1", "E1Sub", "E1Lin"])
@pytest.mark.parametrize("pipeline", [-1, 0, 2], ids=["auto", "plain", "leaf"])
def test_adjoint_split_and_fused_agree(su3s, name, tree, math, pipeline):
    # a sum of two products of distinct leaves: one fused pass and two
    # single-product passes give the oracle's gradients (E1: bit for bit the
    # same, each half repeats the fused kernel's operations for its product)
    dims = (6, 5, 7, 3)
    lat = su3s.Lattice(dims)
    names = oracle.leaf_names(tree)
    f = lattice_fields(dims, SEED + 5, names=tuple(names) + ("w",))
    F = {n: upload(su3s, lat, f[n]) for n in names}
    G = upload(su3s, lat, f["w"])
    ref = oracle.eval_adjoint(tree, {n: f[n] for n in names}, f["w"])
    wscale = np.abs(f["w"]).max() * 3 * 1.5
    got = {}
    su3s.set_pipeline(pipeline)
    try:
        for mode in (0, 1):
            su3s.set_adjoint_split(mode)
            grads = [F[n].like() for n in names]
            su3s.eval_adjoint(tree_expr(tree, F), G, grads, math)
            got[mode] = [g.download() for g in grads]
    finally:
        su3s.set_adjoint_split(-1)
        su3s.set_pipeline(-1)
    for mode in (0, 1):
        for n, g in zip(names, got[mode]):
            assert np.abs(g - ref[n]).max() < TOL * wscale, (mode, n)
    if name == "E1":
        for a, b in zip(got[0], got[1]):
            assert a.tobytes() == b.tobytes()


@pytest.mark.parametrize("math", MATHS, ids=MATH_IDS)
def test_adjoint_matrix_vector(su3s, math):
    dims = (6, 5, 7, 3)
    lat = su3s.Lattice(dims)
    v = synth.volume(dims)
    f = lattice_fields(dims, SEED, names=("a", "v"))
    gz = synth.gauss_vector(SEED, 9, v)
    a = upload(su3s, lat, f["a"])
    x = upload(su3s, lat, f["v"], kind=su3s.VECTOR)
    G = upload(su3s, lat, gz, kind=su3s.VECTOR)
    ga, gv = a.like(), x.like()
    su3s.eval_adjoint(a * x, G, [ga, gv], math)
    ref = oracle.eval_adjoint(("mul", ("leaf", "a"), ("leaf", "v")), f, gz)
    s = np.abs(gz).max() * np.abs(f["v"]).max() * 6
    assert np.abs(ga.download() - ref["a"]).max() < TOL * s
    assert np.abs(gv.download() - ref["v"]).max() < TOL * s


def test_autograd_gradient_16x4(su3s):
    """L = sum_x Re tr(W^dagger (a*b)) on a 16^4 lattice: gradients against the
    oracle's closed form and against central finite differences."""
    dims = (16, 16, 16, 16)
    lat = su3s.Lattice(dims)
    f = lattice_fields(dims, synth.SEED_BASE + 4, names=("a", "b", "w"))
    a, b, w = (upload(su3s, lat, f[n]) for n in "abw")
    ta = a.tensor.clone().requires_grad_(True)
    tb = b.tensor.clone().requires_grad_(True)
    z = su3s.lattice_expr(("mul", ("leaf", 0), ("leaf", 1)), lat, [ta, tb])
    loss = (w.tensor * z).sum()   # pad sites of W are zero
    loss.backward()
    ga = su3s.Field(lat, tensor=ta.grad.contiguous()).download()
    gb = su3s.Field(lat, tensor=tb.grad.contiguous()).download()
    ref = oracle.eval_adjoint(("mul", ("leaf", "a"), ("leaf", "b")), f, f["w"])
    assert np.abs(ga - ref["a"]).max() < TOL * 8
    assert np.abs(gb - ref["b"]).max() < TOL * 8
    # the loss itself against the oracle
    lo = oracle.redot(f["w"], oracle.mm(f["a"], f["b"]))
    assert abs(loss.item() - lo) <= 1e-11 * abs(lo) + 1e-9
    # central differences on 64 random real components of a and b (L is linear
    # in each, so the difference quotient is exact up to rounding)
    rng = np.random.default_rng(11)
    h = 1e-3
    zf = a.like()
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    for name, grad in (("a", ga), ("b", gb)):
        flat = f[name].reshape(-1)
        for k in rng.choice(flat.size, 32, replace=False):
            vals = []
            for sgn in (1, -1):
                pert = f[name].copy()
                pert.reshape(-1)[k] += sgn * h
                x = upload(su3s, lat, pert)
                su3s.evaluate(zf, (x * b) if name == "a" else (a * x), su3s.MATH_F64)
                vals.append(su3s.redot(w, zf, out).item())
            fd = (vals[0] - vals[1]) / (2 * h)
            assert abs(fd - grad.reshape(-1)[k]) < 1e-7 * max(1.0, abs(lo)) ** 0.5


@pytest.mark.parametrize("math", MATHS, ids=MATH_IDS)
def test_autograd_fused_tree(su3s, math):
    dims = (6, 5, 7, 3)
    lat = su3s.Lattice(dims)
    f = lattice_fields(dims, SEED, names=("a", "b", "c", "d", "w"))
    F = {n: upload(su3s, lat, f[n]) for n in "abcdw"}
    ts = [F[n].tensor.clone().requires_grad_(True) for n in "abcd"]
    tree = ("add", ("mul", ("leaf", 0), ("leaf", 1)), ("mul", ("leaf", 2), ("leaf", 3)))
    z = su3s.lattice_expr(tree, lat, ts, math=math)
    (F["w"].tensor * z).sum().backward()
    ref = oracle.eval_adjoint(E1, {n: f[n] for n in "abcd"}, f["w"])
    for n, t in zip("abcd", ts):
        g = su3s.Field(lat, tensor=t.grad.contiguous()).download()
        assert np.abs(g - ref[n]).max() < TOL * 16


# --------------------------------------------------------- batched launches
def config4_volumes(seed, n=64):
    shapes = [(4, 4, 4, 4), (8, 8, 8, 8), (12, 12, 12, 12), (16, 16, 16, 32), (24, 24, 24, 24)]
    picks = (synth.uniform_real(seed, 40, n) + 1.0) / 2.0 * len(shapes)
    return [shapes[min(int(p), len(shapes) - 1)] for p in picks]


@pytest.mark.parametrize("math", MATHS, ids=MATH_IDS)
def test_batch_matches_separate_evaluations(su3s, math):
    seed = synth.SEED_BASE + 4
    shapes = config4_volumes(seed, 12)
    items = []
    b = su3s.Batch()
    for i, dims in enumerate(shapes):
        lat = su3s.Lattice(dims)
        v = synth.volume(dims)
        host = {n: synth.su3(seed + 1000 * i, synth.FIELD[n], v) for n in "abcd"}
        F = {n: upload(su3s, lat, host[n]) for n in "abcd"}
        z = F["a"].like()
        b.add(z, F["a"] * F["b"] + F["c"] * F["d"])
        items.append((lat, host, F, z))
    # one extra item the persistent kernels do not cover (interpreter inside the graph)
    _, host0, F0, _ = items[0]
    zi = F0["a"].like()
    b.add(zi, (F0["a"] + F0["b"]) * F0["c"].adj())
    # an item that cannot be staged (4-site blocks): plain-load persistent kernel
    lat0 = items[0][0]
    F4 = {n: upload(su3s, lat0, host0[n], layout=1, block=4) for n in "abcd"}
    z4 = F4["a"].like()
    b.add(z4, F4["a"] * F4["b"] + F4["c"] * F4["d"])
    # a second staged tree with a real factor, on Lorentz-indexed links
    lat1, host1 = items[1][0], items[1][1]
    v1 = synth.volume(shapes[1])
    hl = {n: synth.su3(seed + 77, synth.FIELD[n], 4 * v1) for n in "abcd"}
    FL = {n: upload(su3s, lat1, hl[n], nmu=4) for n in "abcd"}
    zl = FL["a"].like()
    b.add(zl, FL["a"] * FL["b"] * FL["c"] + 0.5 * FL["d"])
    b.build(math)
    for _ in range(2):
        b.launch()
    torch.cuda.synchronize()
    for lat, host, F, z in items:
        ref = oracle.mm(host["a"], host["b"]) + oracle.mm(host["c"], host["d"])
        got = z.download()
        assert np.abs(got - ref).max() < 2 * TOL
        sep = z.like()
        su3s.evaluate(sep, F["a"] * F["b"] + F["c"] * F["d"], math)
        assert np.array_equal(sep.download(), got)   # same arithmetic, same bits
    ref = oracle.eval_tree(("mul", ("add", ("leaf", "a"), ("leaf", "b")), ("adj", ("leaf", "c"))),
                           host0)
    assert np.abs(zi.download() - ref).max() < 4 * TOL
    ref4 = oracle.mm(host0["a"], host0["b"]) + oracle.mm(host0["c"], host0["d"])
    assert np.abs(z4.download() - ref4).max() < 2 * TOL
    refl = oracle.eval_tree(E2, hl)
    assert np.abs(zl.download() - refl).max() < 4 * TOL
    sepl = zl.like()
    su3s.evaluate(sepl, FL["a"] * FL["b"] * FL["c"] + 0.5 * FL["d"], math)
    assert np.array_equal(sepl.download(), zl.download())
    assert su3s.device_error() == 0
    sites, tiles = b.info()
    assert sites > 0 and tiles > 0


@pytest.mark.parametrize("math", MATHS, ids=MATH_IDS)
def test_batch_covers_every_persistent_tree(su3s, math):
    """One item of each tree the persistent kernels cover, on a lattice that the
    staged kernel takes (SoA) and on one that the plain-load kernel takes
    (4-site blocks): same bits as a separate evaluation, and the oracle's value."""
    dims = (4, 4, 4, 6)
    v = synth.volume(dims)
    lat = su3s.Lattice(dims)
    seed = synth.SEED_BASE + 9
    host = {n: synth.su3(seed, synth.FIELD[n], v) for n in "abcd"}
    hv = synth.gauss_vector(seed, synth.FIELD["v"], v)
    al, be = 0.75, -1.25
    trees = {
        "MM": (("mul", ("leaf", "a"), ("leaf", "b")), lambda F: F["a"] * F["b"]),
        "E1": (E1, lambda F: F["a"] * F["b"] + F["c"] * F["d"]),
        "MV": (("mul", ("leaf", "a"), ("leaf", "v")), lambda F: F["a"] * F["v"]),
        "E2": (E2, lambda F: F["a"] * F["b"] * F["c"] + 0.5 * F["d"]),
        "E3": (E3, lambda F: F["a"].adj() * F["b"] - F["b"] * F["a"].adj()),
        "MMM": (("mul", ("mul", ("leaf", "a"), ("leaf", "b")), ("leaf", "c")),
                lambda F: F["a"] * F["b"] * F["c"]),
        "E1Lin": (("add", ("scale", al, ("mul", ("leaf", "a"), ("leaf", "b"))),
                   ("scale", be, ("mul", ("leaf", "c"), ("leaf", "d")))),
                  lambda F: al * (F["a"] * F["b"]) + be * (F["c"] * F["d"])),
        "AdjMM": (("mul", ("adj", ("leaf", "a")), ("leaf", "b")), lambda F: F["a"].adj() * F["b"]),
    }
    b = su3s.Batch()
    items = []
    for lay in ((0, 0), (1, 4)):
        for name, (tree, mk) in trees.items():
            # every item reads its own copies: batch items must not overlap
            F = {n: upload(su3s, lat, host[n], layout=lay[0], block=lay[1]) for n in "abcd"}
            F["v"] = upload(su3s, lat, hv, kind=su3s.VECTOR, layout=lay[0], block=lay[1])
            z = (F["v"] if name == "MV" else F["a"]).like()
            b.add(z, mk(F))
            items.append((name, tree, mk, F, z))
    b.build(math)
    b.launch()
    torch.cuda.synchronize()
    leaves = dict(host, v=hv)
    for name, tree, mk, F, z in items:
        sep = z.like()
        su3s.evaluate(sep, mk(F), math)
        got = z.download()
        assert np.array_equal(sep.download(), got), name
        ref = oracle.eval_tree(tree, {n: leaves[n] for n in oracle.leaf_names(tree)})
        scale = max(1.0, np.abs(hv).max() * 3) if name == "MV" else 1.0
        assert np.abs(got - ref).max() < 4 * TOL * scale, name
    assert su3s.device_error() == 0


@pytest.mark.parametrize("math", MATHS, ids=MATH_IDS)
def test_batch_tune_keeps_results(su3s, math):
    """The batch autotuner rebuilds the graph in other launch shapes; the
    results of the tuned batch are the same bits as the default build's."""
    seed = synth.SEED_BASE + 4
    shapes = config4_volumes(seed, 6)
    b = su3s.Batch()
    outs = []
    for i, dims in enumerate(shapes):
        lat = su3s.Lattice(dims)
        v = synth.volume(dims)
        host = {n: synth.su3(seed + 1000 * i, synth.FIELD[n], v) for n in "abcd"}
        lay = (1, 4) if i == 0 else (0, 0)          # one item on the plain-load kernels
        F = {n: upload(su3s, lat, host[n], layout=lay[0], block=lay[1]) for n in "abcd"}
        z = F["a"].like()
        b.add(z, F["a"] * F["b"] + F["c"] * F["d"])
        outs.append((F, z))
    b.build(math)
    b.launch()
    torch.cuda.synchronize()
    ref = [z.download() for _, z in outs]
    th, tile, bps, ms = b.tune(math)
    assert th in (64, 128, 256) and tile in (th, 2 * th, 4 * th) and bps in (0, 1, 2, 4) and ms > 0
    for _, z in outs:
        z.tensor.zero_()
    b.launch()
    torch.cuda.synchronize()
    for r, (_, z) in zip(ref, outs):
        assert np.array_equal(z.download(), r)
    assert su3s.device_error() == 0


# --------------------------------------------- staged vs plain data movement
@pytest.mark.parametrize("math", MATHS, ids=MATH_IDS)
@pytest.mark.parametrize("lay", [LAYOUTS[0], LAYOUTS[2], LAYOUTS[3]], ids=layout_id)
def test_tma_staging_is_bitwise_identical(su3s, lay, math):
    """The TMA-staged kernels (bulk copies into shared memory, one 32-site tile
    per warp: whole tile, per leaf, or through a ring of buffers) and the
    plain-load kernels run the same arithmetic per site."""
    PIPES = (su3s.PIPE_PLAIN, su3s.PIPE_TMA, su3s.PIPE_TMA_LEAF, su3s.PIPE_TMA_RING,
             su3s.PIPE_TMA_PAIR)
    dims = (8, 8, 8, 9)
    lat = su3s.Lattice(dims)
    f = lattice_fields(dims, SEED, nmu=4, names=("a", "b", "c", "d", "w"))
    F = {n: upload(su3s, lat, f[n], nmu=4, layout=lay[1], block=lay[2]) for n in "abcdw"}
    a, b, c, d = (F[n] for n in "abcd")
    exprs = [a * b, a * b + c * d, a.adj() * b - b * a.adj(), a * b * c + 0.5 * d]
    try:
        for e in exprs:
            outs = []
            for mode in PIPES:
                su3s.set_pipeline(mode)
                z = a.like()
                su3s.evaluate(z, e, math)
                outs.append(z.download())
            for o in outs[1:]:
                assert np.array_equal(outs[0], o)
        grads = []
        for mode in PIPES:
            su3s.set_pipeline(mode)
            g = [a.like() for _ in range(4)]
            su3s.eval_adjoint(a * b + c * d, F["w"], g, math)
            g2 = [a.like() for _ in range(4)]
            su3s.eval_adjoint(a * b * c + 0.5 * d, F["w"], g2, math)
            grads.append([x.download() for x in g + g2])
        for xs in zip(*grads):
            for y in xs[1:]:
                assert np.array_equal(xs[0], y)
    finally:
        su3s.set_pipeline(su3s.PIPE_AUTO)
    assert su3s.device_error() == 0
    ref = oracle.eval_tree(E1, f)
    z = a.like()
    su3s.evaluate(z, a * b + c * d, math)
    assert np.abs(z.download() - ref).max() < 2 * TOL


def test_ring_staging_over_many_tiles_per_warp(su3s):
    """The ring-staged kernels prefetch into the warp's next tile; with many
    tiles per warp (a small forced grid, and a 24^4 lattice for the reverse
    mode) they stay bitwise equal to plain loads."""
    dims = (24, 24, 24, 24)
    lat = su3s.Lattice(dims)
    f = lattice_fields(dims, SEED + 11, names=("a", "b", "c", "d", "w"))
    F = {n: upload(su3s, lat, f[n]) for n in "abcdw"}
    a, b, c, d = (F[n] for n in "abcd")
    try:
        for math in MATHS:
            for e in (a * b + c * d, a * b * c + 0.5 * d):
                outs = []
                for mode in (su3s.PIPE_PLAIN, su3s.PIPE_TMA_RING):
                    su3s.set_pipeline(mode)
                    z = a.like()
                    su3s.set_launch(z, e, 32, 1, math)   # 152 one-warp blocks: ~68 tiles each
                    su3s.evaluate(z, e, math)
                    outs.append(z.download())
                assert np.array_equal(outs[0], outs[1])
            for e, n in ((a * b + c * d, 4), (a * b, 2)):
                gs = []
                for mode in (su3s.PIPE_PLAIN, su3s.PIPE_TMA_RING):
                    su3s.set_pipeline(mode)
                    g = [a.like() for _ in range(n)]
                    su3s.eval_adjoint(e, F["w"], g, math)
                    gs.append([x.download() for x in g])
                for x, y in zip(*gs):
                    assert np.array_equal(x, y)
    finally:
        su3s.set_pipeline(su3s.PIPE_AUTO)
    assert su3s.device_error() == 0



@pytest.mark.parametrize("dims,nmu,lay", [((17, 17, 17, 17), 1, LAYOUTS[2]),
                                          ((6, 6, 6, 6), 4, LAYOUTS[2]),
                                          ((3, 3, 3, 3), 1, LAYOUTS[0])],
                         ids=["17^4-aosoa32", "6^4-nmu4-aosoa32", "3^4-soa"])
def test_pair_kernels_bitwise_over_odd_tiles(su3s, dims, nmu, lay):
    """The two-sites-per-lane kernels (mode 4: a warp takes two 32-site tiles
    per step, every pair-arithmetic operation packed over the two sites) give
    the plain-load kernels' results bit for bit.  With 32-site blocks the
    lattices have an odd number of tiles, so the last step has one; 17^4 with
    152 one-warp blocks gives each warp ~9 steps; 3^4 is one step of padded
    sites.  Every adjoint placement in a product, a sum and a difference of
    products, and the reverse mode with both gradients and with one."""
    lat = su3s.Lattice(dims)
    if lay[2] == 32:
        assert ((np.prod(dims) + 31) // 32) % 2 == 1
    f = lattice_fields(dims, SEED + 13, nmu=nmu, names=("a", "b", "c", "d", "w"))
    F = {n: upload(su3s, lat, f[n], nmu=nmu, layout=lay[1], block=lay[2]) for n in "abcdw"}
    a, b, c, d, w = (F[n] for n in "abcdw")
    exprs = [a * b, a.adj() * b, a * b.adj(), a.adj() * b.adj(), a * b + c * d, a * b - c * d]
    try:
        for e in exprs:
            outs = []
            for mode in (su3s.PIPE_PLAIN, su3s.PIPE_TMA_PAIR):
                su3s.set_pipeline(mode)
                z = a.like()
                if dims[0] == 17:
                    su3s.set_launch(z, e, 32, 1)    # 152 one-warp blocks
                elif dims[0] == 6:
                    # 256 threads: a sum's staging (37 KB per warp) fits 6 warps
                    # of a block, so the launch is cut to 192 threads
                    su3s.set_launch(z, e, 256, 0)
                su3s.evaluate(z, e)
                outs.append(z.download())
            assert np.array_equal(outs[0], outs[1])
        for e in (a * b, a.adj() * b, a * b.adj()):
            for want in ((True, True), (True, False), (False, True)):
                gs = []
                for mode in (su3s.PIPE_PLAIN, su3s.PIPE_TMA_PAIR):
                    su3s.set_pipeline(mode)
                    g = [a.like() if k else None for k in want]
                    su3s.eval_adjoint(e, w, g)
                    gs.append([x.download() for x in g if x is not None])
                for x, y in zip(*gs):
                    assert np.array_equal(x, y)
    finally:
        su3s.set_pipeline(su3s.PIPE_AUTO)
    assert su3s.device_error() == 0
    # and against the oracle
    ref = oracle.eval_tree(E1, f)
    su3s.set_pipeline(su3s.PIPE_TMA_PAIR)
    try:
        z = a.like()
        su3s.evaluate(z, a * b + c * d)
    finally:
        su3s.set_pipeline(su3s.PIPE_AUTO)
    assert np.abs(z.download() - ref).max() < 2 * TOL

# ---------------------------------------------------------- tuning
def test_launch_geometry_does_not_change_results(su3s):
    dims = (8, 8, 8, 8)
    lat = su3s.Lattice(dims)
    f = lattice_fields(dims, SEED, names=("a", "b", "c", "d"))
    F = {n: upload(su3s, lat, f[n]) for n in "abcd"}
    e = F["a"] * F["b"] + F["c"] * F["d"]
    outs = []
    for math in MATHS:
        ref = None
        for th, bps in ((64, 0), (128, 2), (256, 0), (256, 8), (96, 1)):
            z = F["a"].like()
            su3s.set_launch(z, e, th, bps, math)
            su3s.evaluate(z, e, math)
            got = z.download()
            if ref is None:
                ref = got
            assert np.array_equal(got, ref)
        th, bps, var, ms = su3s.tune(z, e, math)
        su3s.evaluate(z, e, math)
        assert np.array_equal(z.download(), ref) and th in (64, 128, 256) and ms > 0
        assert var in (0, 1, 2, 3)
        outs.append(ref)


# --------------------------------------------------- reductions, projection
def test_redot(su3s):
    dims = (6, 5, 7, 3)
    lat = su3s.Lattice(dims)
    f = lattice_fields(dims, SEED, nmu=4, names=("a", "w"))
    a, w = upload(su3s, lat, f["a"], nmu=4), upload(su3s, lat, f["w"], nmu=4)
    got = su3s.redot(a, w).item()
    want = oracle.redot(f["a"], f["w"])
    assert abs(got - want) <= 1e-12 * max(1.0, abs(want))
    # deterministic
    assert su3s.redot(a, w).item() == got


@pytest.mark.parametrize("prec,fmt,tol", [(0, None, 1e-13), (1, "f32", 1e-6)], ids=["f64", "f32"])
def test_reunitarize(su3s, prec, fmt, tol):
    dims = (6, 5, 7, 3)
    lat = su3s.Lattice(dims)
    v = synth.volume(dims)
    noisy = synth.su3(SEED, 0, v) + 1e-3 * synth.gauss_matrix(SEED, 5, v)
    x = upload(su3s, lat, noisy, prec=prec)
    y = x.like()
    su3s.reunitarize(y, x)
    src = noisy if fmt is None else oracle.round_to(noisy, fmt)
    ref = oracle.reunitarize(src)
    if fmt is not None:
        ref = oracle.round_to(ref, fmt)
    assert np.abs(y.download() - ref).max() < tol
    u = cplx(y.download())
    assert np.abs(u @ np.conj(np.swapaxes(u, 1, 2)) - np.eye(3)).max() < max(tol, 1e-13) * 10


# ------------------------------------------------------ failure detection
def test_bounded_wait_gives_up_and_context_survives(su3s):
    """A staging wait that nothing completes (no copy issued, nothing arrives)
    gives up after its poll limit, records code 1 in the device error word, and
    the kernel returns: the context stays usable and the next evaluation is
    right.  The measured time per poll gives the pipelines' give-up time."""
    import json
    assert su3s.device_error() == 0
    polls = 4096
    cycles = su3s.selftest_bounded_wait(polls)
    assert cycles > 0
    assert su3s.device_error() == 1
    assert su3s.device_error() == 0          # the read cleared it
    dims = (3, 2, 1, 5)
    lat = su3s.Lattice(dims)
    f = lattice_fields(dims, SEED)
    a, b = upload(su3s, lat, f["a"]), upload(su3s, lat, f["b"])
    z = a.like()
    su3s.evaluate(z, a * b)
    assert np.abs(z.download() - oracle.mm(f["a"], f["b"])).max() < TOL
    assert su3s.device_error() == 0
    print(json.dumps({"bounded_wait_polls": polls, "cycles": cycles,
                      "cycles_per_poll": cycles / polls,
                      "pipeline_give_up_cycles": cycles / polls * (1 << 18)}))


# ------------------------------------------------------ full-size sampling
@pytest.mark.parametrize("math", MATHS, ids=MATH_IDS)
def test_full_size_48_sampled(su3s, math):
    """The 48^4 configuration in the launch geometry the benchmark uses:
    z=a*b, z=a*v and Lorentz z_mu=a_mu*b_mu checked on sampled sites."""
    dims = (48, 48, 48, 48)
    v = synth.volume(dims)
    seed = synth.SEED_BASE + 1
    lat = su3s.Lattice(dims)
    rng = np.random.default_rng(2)
    sample = np.unique(np.concatenate([rng.choice(v, 3000, replace=False), [0, v - 1]]))
    for nmu, vec in ((1, False), (1, True), (4, False)):
        ha = synth.su3(seed, 0, v * nmu)
        hb = synth.gauss_vector(seed, 4, v * nmu) if vec else synth.su3(seed, 1, v * nmu)
        a = upload(su3s, lat, ha, nmu=nmu)
        b = upload(su3s, lat, hb, kind=su3s.VECTOR if vec else su3s.MATRIX, nmu=nmu)
        z = b.like()
        su3s.evaluate(z, a * b, math)
        idx = (sample[:, None] * nmu + np.arange(nmu)[None, :]).reshape(-1)
        got = z.unpack()[torch.from_numpy(idx).cuda()].cpu().numpy()
        ref = oracle.mv(ha[idx], hb[idx]) if vec else oracle.mm(ha[idx], hb[idx])
        scale = 1.0 if not vec else max(1.0, np.abs(cplx(hb[idx])).sum(axis=1).max())
        assert np.abs(got - ref).max() < TOL * scale
        del a, b, z
        torch.cuda.empty_cache()


@pytest.mark.parametrize("dims", [(128, 128, 128, 512), (128, 128, 128, 513)],
                         ids=["V=2^30", "V>2^30"])
def test_largest_soa_fields(su3s, dims):
    """z = a*v into v on the largest lattices the device holds: at V = 2^30 the
    staged kernels copy at tensor column 2^31 - 64, the top of the signed
    32-bit coordinate range; beyond it the fields take the plain-load kernels.
    A 155 GB Gaussian matrix field and a 52 GB vector field (seeded on the
    device); sampled sites, the sites around 2^30 and the last site are checked
    against the oracle."""
    v = synth.volume(dims)
    need = v * (144 + 48)
    torch.cuda.empty_cache()          # memory cached by earlier tests counts as used
    if torch.cuda.mem_get_info()[0] < need + (4 << 30):
        pytest.skip("needs %.0f GB of free device memory" % (need / 1e9))
    lat = su3s.Lattice(dims)
    a = su3s.Field(lat, su3s.MATRIX, 1, su3s.F64, su3s.SOA)
    x = su3s.Field(lat, su3s.VECTOR, 1, su3s.F64, su3s.SOA)
    g = torch.Generator(device="cuda").manual_seed(SEED)
    a.tensor.normal_(generator=g)
    x.tensor.normal_(generator=g)
    vpad = a.tensor.numel() // 18
    rng = np.random.default_rng(5)
    edge = [0, 1, (1 << 30) - 33, (1 << 30) - 32, (1 << 30) - 1, v - 33, v - 32, v - 1]
    sample = np.unique(np.concatenate([rng.choice(v, 4000, replace=False), edge]))
    sample = sample[sample < v]
    idx = torch.from_numpy(sample).cuda()

    def gather(f, nc):
        t = f.tensor.view(nc, vpad, 2)[:, idx, :].permute(1, 0, 2).contiguous()
        return t.cpu().numpy().reshape((-1, 3, 3, 2) if nc == 9 else (-1, 3, 2))
    ha, hx = gather(a, 9), gather(x, 3)
    su3s.evaluate(x, a * x)
    got = gather(x, 3)
    torch.cuda.synchronize()
    del a, x
    torch.cuda.empty_cache()
    ref = oracle.mv(ha, hx)
    scale = np.einsum("nij,nj->ni", np.abs(cplx(ha)), np.abs(cplx(hx)))
    err = np.abs(cplx(got) - cplx(ref))
    assert (err <= TOL * np.maximum(1.0, 2 * scale)).all()


def test_empty_batch_builds_and_launches(su3s):
    b = su3s.Batch()
    b.build()
    b.launch()
    torch.cuda.synchronize()
    assert b.info() == (0, 0)
