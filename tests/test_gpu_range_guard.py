"""Range guard of the FP64-accurate arithmetics, through the C ABI.

The pair-of-FP32 (DF32) and fixed-point (FX) arithmetics hold FP64 values in
narrower formats and represent neither Inf nor NaN.  Every kernel that
evaluates in them checks each site's FP64 inputs as it reads them; a site
with an input that is NaN, +-Inf or at least 2^t(d) in magnitude (t(2) = 58,
t(3) = 38) is evaluated again in native FP64 before anything of it is stored.

These tests plant such values (and values just inside the range, and tiny
ones) in otherwise random fields and check every output against the FP64
oracle with IEEE semantics: NaN exactly where the oracle has NaN, the same
infinities, finite values within 1e-13 times the site's magnitude.  A site
that trips the guard must also equal the native-FP64 kernel bit for bit,
which shows that the FP64 path, not the narrow arithmetic, produced it.
"""
import numpy as np
import pytest

import oracle
import synth
from helpers import E1, E2, lattice_fields

pytestmark = pytest.mark.gpu

SEED = synth.SEED_BASE + 23
TOL = 1e-13
GUARDED = [2, 3]            # SU3S_MATH_DF32, SU3S_MATH_FX
GUARDED_IDS = ["df32", "fx"]
F64 = 1
DIMS = (6, 5, 7, 3)         # 630 sites: many tiles, a ragged tail
# (value, whether it trips the guard of a degree-2 tree)
SPECIALS = [(np.nan, True), (np.inf, True), (-np.inf, True), (1e40, True), (-3e300, True),
            (2.0 ** 59, True), (-(2.0 ** 57), False), (1e-40, False), (5e-324, False),
            (-0.0, False)]


@pytest.fixture(scope="module")
def su3s(gpu_lib):
    return gpu_lib


def plant(arr, first_site, values=SPECIALS, stride=37):
    """Put each special value into one real of one site object (sites
    first_site, first_site + stride, ...); returns the sites touched."""
    flat = arr.reshape(arr.shape[0], -1)
    sites = []
    for k, (val, _) in enumerate(values):
        s = (first_site + stride * k) % arr.shape[0]
        flat[s, (5 * k + 1) % flat.shape[1]] = val
        sites.append(s)
    return sites


def site_scale(*arrs):
    """Per-object magnitude bound of a product term: 6 x the product of the
    operands' largest finite magnitudes (at least 1)."""
    m = np.ones(arrs[0].shape[0])
    for a in arrs:
        x = np.abs(a.reshape(a.shape[0], -1))
        x = np.where(np.isfinite(x), x, 0.0)
        m = m * np.maximum(x.max(axis=1), 1.0)
    return 6.0 * m


def assert_ieee(got, ref, scale):
    got = got.reshape(got.shape[0], -1)
    ref = ref.reshape(ref.shape[0], -1)
    assert np.array_equal(np.isnan(got), np.isnan(ref))
    inf = np.isinf(ref)
    assert np.array_equal(got[inf], ref[inf])
    fin = np.isfinite(ref)
    assert np.isfinite(got[fin]).all()
    err = np.abs(got - ref)
    assert (err[fin] <= (TOL * scale[:, None] * np.ones_like(ref))[fin]).all(), err[fin].max()


def fields(su3s, dims, arrs, kinds=None, nmu=1, layout=0, block=64):
    lat = su3s.Lattice(dims)
    out = {}
    for n, a in arrs.items():
        kind = (kinds or {}).get(n, su3s.MATRIX)
        f = su3s.Field(lat, kind, nmu, su3s.F64, layout, block)
        f.upload(a)
        out[n] = f
    return out


@pytest.mark.parametrize("math", GUARDED, ids=GUARDED_IDS)
@pytest.mark.parametrize("pipeline", [-1, 0, 1, 2, 3, 4],
                         ids=["auto", "plain", "tile", "leaf", "ring", "pair"])
def test_product_with_special_inputs(su3s, math, pipeline):
    f = lattice_fields(DIMS, SEED, names=("a", "b"))
    trips = plant(f["a"], 3) + plant(f["b"], 200)
    F = fields(su3s, DIMS, f)
    su3s.set_pipeline(pipeline)
    try:
        z = F["a"].like()
        su3s.evaluate(z, F["a"] * F["b"], math)
        zf = F["a"].like()
        su3s.evaluate(zf, F["a"] * F["b"], F64)
    finally:
        su3s.set_pipeline(-1)
    got = z.download()
    assert_ieee(got, oracle.mm(f["a"], f["b"]), site_scale(f["a"], f["b"]))
    ref64 = zf.download()
    for (val, trip), s in zip(SPECIALS * 2, trips):
        if trip:
            assert got[s].tobytes() == ref64[s].tobytes(), (val, s)


@pytest.mark.parametrize("math", GUARDED, ids=GUARDED_IDS)
def test_in_place_product_reads_its_inputs_before_the_fallback(su3s, math):
    # z = a*b into a: a tripped site must still see its own inputs
    f = lattice_fields(DIMS, SEED + 1, names=("a", "b"))
    plant(f["a"], 11)
    plant(f["b"], 300)
    F = fields(su3s, DIMS, f)
    su3s.evaluate(F["a"], F["a"] * F["b"], math)
    assert_ieee(F["a"].download(), oracle.mm(f["a"], f["b"]), site_scale(f["a"], f["b"]))


@pytest.mark.parametrize("math", GUARDED, ids=GUARDED_IDS)
@pytest.mark.parametrize("layout,block", [(0, 64), (1, 32), (1, 4)], ids=["soa", "aosoa32", "aosoa4"])
@pytest.mark.parametrize("pipeline", [-1, 4], ids=["auto", "pair"])
def test_fused_sum_of_products(su3s, math, layout, block, pipeline):
    f = lattice_fields(DIMS, SEED + 2, names=("a", "b", "c", "d"))
    plant(f["a"], 5)
    plant(f["d"], 150)
    F = fields(su3s, DIMS, f, layout=layout, block=block)
    z = F["a"].like()
    su3s.set_pipeline(pipeline)
    try:
        su3s.evaluate(z, F["a"] * F["b"] + F["c"] * F["d"], math)
    finally:
        su3s.set_pipeline(-1)
    scale = site_scale(f["a"], f["b"]) + site_scale(f["c"], f["d"])
    assert_ieee(z.download(), oracle.eval_tree(E1, f), scale)


@pytest.mark.parametrize("math", GUARDED, ids=GUARDED_IDS)
def test_degree_three_tree_uses_the_tighter_bound(su3s, math):
    # (a*b)*c + 0.5 d has degree 3: 2^38 is its bound, so 1e15 trips it
    f = lattice_fields(DIMS, SEED + 3, names=("a", "b", "c", "d"))
    vals = [(1e15, True), (-(2.0 ** 37), False), (np.nan, True)]
    trips = plant(f["c"], 9, vals)
    F = fields(su3s, DIMS, f)
    z = F["a"].like()
    su3s.evaluate(z, (F["a"] * F["b"]) * F["c"] + 0.5 * F["d"], math)
    zf = F["a"].like()
    su3s.evaluate(zf, (F["a"] * F["b"]) * F["c"] + 0.5 * F["d"], F64)
    got = z.download()
    scale = 6.0 * site_scale(f["a"], f["b"], f["c"]) + site_scale(f["d"])
    assert_ieee(got, oracle.eval_tree(E2, f), scale)
    ref64 = zf.download()
    for (val, trip), s in zip(vals, trips):
        if trip:
            assert got[s].tobytes() == ref64[s].tobytes(), val


@pytest.mark.parametrize("math", GUARDED, ids=GUARDED_IDS)
@pytest.mark.parametrize("alpha", [1e300, np.nan, 2.0 ** 60], ids=["1e300", "nan", "2^60"])
def test_real_factor_out_of_range_sends_every_site_to_fp64(su3s, math, alpha):
    f = lattice_fields(DIMS, SEED + 4, names=("a", "b", "c", "d"))
    F = fields(su3s, DIMS, f)
    e = alpha * (F["a"] * F["b"]) + 0.25 * (F["c"] * F["d"])
    z = F["a"].like()
    su3s.evaluate(z, e, math)
    zf = F["a"].like()
    su3s.evaluate(zf, e, F64)
    tree = ("add", ("scale", alpha, ("mul", ("leaf", "a"), ("leaf", "b"))),
            ("scale", 0.25, ("mul", ("leaf", "c"), ("leaf", "d"))))
    got = z.download()
    ref = oracle.eval_tree(tree, f)
    scale = site_scale(f["a"], f["b"]) * (abs(alpha) if np.isfinite(alpha) else 1.0) + 1.0
    assert_ieee(got, ref, scale)
    assert got.tobytes() == zf.download().tobytes()


@pytest.mark.parametrize("math", GUARDED, ids=GUARDED_IDS)
def test_interpreter_tree(su3s, math):
    # adj(a*b)*c is outside the compiled catalogue: the interpreter runs it
    f = lattice_fields(DIMS, SEED + 5, names=("a", "b", "c"))
    plant(f["b"], 17, [(np.inf, True), (1e20, True), (np.nan, True), (1e-40, False)])
    F = fields(su3s, DIMS, f)
    e = (F["a"] * F["b"]).adj() * F["c"]
    z = F["a"].like()
    su3s.evaluate(z, e, math)
    tree = ("mul", ("adj", ("mul", ("leaf", "a"), ("leaf", "b"))), ("leaf", "c"))
    assert_ieee(z.download(), oracle.eval_tree(tree, f), 6.0 * site_scale(f["a"], f["b"], f["c"]))


@pytest.mark.parametrize("math", GUARDED, ids=GUARDED_IDS)
@pytest.mark.parametrize("pipeline", [-1, 0, 2, 3, 4], ids=["auto", "plain", "leaf", "ring", "pair"])
@pytest.mark.parametrize("tree,split", [("ab", -1), ("e1", -1), ("e1", 0)],
                         ids=["ab", "e1", "e1-fused"])
def test_reverse_mode_with_special_inputs(su3s, math, pipeline, tree, split):
    names = ("a", "b") if tree == "ab" else ("a", "b", "c", "d")
    f = lattice_fields(DIMS, SEED + 6, names=names + ("w",))
    plant(f["a"], 21)
    plant(f["w"], 400, [(np.nan, True), (-np.inf, True), (3e60, True), (1e-40, False)])
    leaves = {n: f[n] for n in names}
    F = fields(su3s, DIMS, f)
    if tree == "ab":
        e, t = F["a"] * F["b"], ("mul", ("leaf", "a"), ("leaf", "b"))
    else:
        e, t = F["a"] * F["b"] + F["c"] * F["d"], E1
    grads = [F[n].like() for n in names]
    su3s.set_pipeline(pipeline)
    su3s.set_adjoint_split(split)
    try:
        su3s.eval_adjoint(e, F["w"], grads, math)
    finally:
        su3s.set_pipeline(-1)
        su3s.set_adjoint_split(-1)
    ref = oracle.eval_adjoint(t, leaves, f["w"])
    for n, g in zip(names, grads):
        others = [f[m] for m in names if m != n] + [f["w"]]
        assert_ieee(g.download(), ref[n], 2.0 * site_scale(*others))


@pytest.mark.parametrize("math", GUARDED, ids=GUARDED_IDS)
def test_batch_items_with_special_inputs(su3s, math):
    f = lattice_fields(DIMS, SEED + 7, names=("a", "b", "c", "d"))
    plant(f["a"], 2)
    plant(f["c"], 99)
    F = fields(su3s, DIMS, f)
    z1, z2 = F["a"].like(), F["a"].like()
    b = su3s.Batch()
    b.add(z1, F["a"] * F["b"])
    b.add(z2, F["a"] * F["b"] + F["c"] * F["d"])
    b.build(math)
    b.launch()
    assert_ieee(z1.download(), oracle.mm(f["a"], f["b"]), site_scale(f["a"], f["b"]))
    assert_ieee(z2.download(), oracle.eval_tree(E1, f),
                site_scale(f["a"], f["b"]) + site_scale(f["c"], f["d"]))


@pytest.mark.parametrize("math", GUARDED, ids=GUARDED_IDS)
@pytest.mark.parametrize("kind", ["vector", "matrix"])
def test_hopping_term_with_special_inputs(su3s, math, kind):
    v = synth.volume(DIMS)
    u = synth.su3(SEED + 8, 0, v * 4)
    x = synth.gauss_vector(SEED + 8, 1, v) if kind == "vector" else synth.su3(SEED + 8, 1, v)
    plant(u, 40, [(np.nan, True), (1e30, True), (1e-40, False)])
    plant(x, 333, [(-np.inf, True), (2.0 ** 70, True)])
    lat = su3s.Lattice(DIMS)
    K = su3s.VECTOR if kind == "vector" else su3s.MATRIX
    U = su3s.Field(lat, su3s.MATRIX, 4, su3s.F64)
    U.upload(u)
    X = su3s.Field(lat, K, 1, su3s.F64)
    X.upload(x)
    out = X.like()
    su3s.hop(out, U, X, math)
    ref = oracle.hop(u, x, DIMS)
    got = out.download()
    assert np.array_equal(np.isnan(got), np.isnan(ref))
    inf = np.isinf(ref)
    assert np.array_equal(got[inf], ref[inf])
    fin = np.isfinite(ref)
    # the neighbour sums mix sites: bound each output by its largest input
    assert (np.abs(got - ref)[fin] <= TOL * np.maximum(1.0, np.abs(ref[fin])) * 64).all()
