"""C ABI checks that need no GPU: the library loads, exports every declared
entry point, and its host-side logic (validation, layouts, type rules,
canonical signatures, catalogue) behaves as documented in include/su3s.h.

Fields are wrapped around a fake, aligned device address: wrapping never
touches memory, and no call here launches a kernel.
"""
import ctypes
import os
import re

import pytest

import paper_1710_09409_gb300 as su3s

HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "su3s.h")
FAKE = 1 << 40  # 16-byte aligned, never dereferenced


@pytest.fixture(scope="module")
def L():
    return su3s.load(build_if_missing=True)


def declared():
    text = open(HDR).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(su3s_\w+)\s*\(", text, re.M)))


def test_every_declared_symbol_is_exported(L):
    names = declared()
    assert len(names) >= 30
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_no_undeclared_exports(L):
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", su3s.lib_path()], capture_output=True,
                         text=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    assert exported == set(declared())


def _lat(L, dims):
    h = ctypes.c_void_p()
    rc = L.su3s_lattice_create(*dims, ctypes.byref(h))
    return rc, h


def test_lattice_validation(L):
    rc, h = _lat(L, (0, 2, 2, 2))
    assert rc == 1 and b"extents" in L.su3s_last_error()
    rc, h = _lat(L, (1291, 1291, 1291, 1))   # volume >= 2^31
    assert rc == 1
    rc, h = _lat(L, (3, 2, 1, 5))
    assert rc == 0
    v = ctypes.c_int64()
    assert L.su3s_lattice_volume(h, ctypes.byref(v)) == 0 and v.value == 30
    assert L.su3s_lattice_destroy(h) == 0
    assert L.su3s_lattice_destroy(None) == 0


@pytest.mark.parametrize("kind,prec,ncomp,eb", [
    (su3s.MATRIX, su3s.F64, 9, 16), (su3s.MATRIX, su3s.F32, 9, 8), (su3s.MATRIX, su3s.BF16, 9, 4),
    (su3s.MATRIX, su3s.F16, 9, 4), (su3s.MATRIX, su3s.F64_C12, 6, 16),
    (su3s.MATRIX, su3s.F32_C12, 6, 8), (su3s.VECTOR, su3s.F64, 3, 16), (su3s.REAL, su3s.F64, 1, 8)])
@pytest.mark.parametrize("layout,block", [(su3s.SOA, 0), (su3s.AOSOA, 4), (su3s.AOSOA, 64)])
def test_field_bytes_formula(L, kind, prec, ncomp, eb, layout, block):
    rc, lat = _lat(L, (3, 2, 1, 5))   # V = 30: ragged for every block
    for nmu in (1, 4):
        n = ctypes.c_size_t()
        assert L.su3s_field_bytes(lat, kind, nmu, prec, layout, block, ctypes.byref(n)) == 0
        q = 64 if layout == su3s.SOA else max(block, 4)
        vpad = (30 + q - 1) // q * q
        assert n.value == vpad * nmu * ncomp * eb


def test_field_validation(L):
    rc, lat = _lat(L, (2, 2, 2, 2))
    n = ctypes.c_size_t()
    h = ctypes.c_void_p()
    assert L.su3s_field_bytes(lat, su3s.MATRIX, 1, su3s.F64, su3s.SOA, 0, ctypes.byref(n)) == 0
    assert L.su3s_field_wrap(lat, su3s.MATRIX, 1, su3s.F64, su3s.SOA, 0, FAKE + 8, n.value,
                             ctypes.byref(h)) == 1
    assert b"aligned" in L.su3s_last_error()
    assert L.su3s_field_wrap(lat, su3s.MATRIX, 1, su3s.F64, su3s.SOA, 0, FAKE, n.value - 16,
                             ctypes.byref(h)) == 3
    assert L.su3s_field_wrap(lat, su3s.REAL, 1, su3s.F32, su3s.SOA, 0, FAKE, 1 << 20,
                             ctypes.byref(h)) == 6
    assert L.su3s_field_wrap(lat, su3s.VECTOR, 1, su3s.F64_C12, su3s.SOA, 0, FAKE, 1 << 20,
                             ctypes.byref(h)) == 6
    assert L.su3s_field_wrap(lat, su3s.MATRIX, 1, su3s.F64, su3s.AOSOA, 48, FAKE, 1 << 20,
                             ctypes.byref(h)) == 1
    assert L.su3s_field_wrap(lat, su3s.MATRIX, 9, su3s.F64, su3s.SOA, 0, FAKE, 1 << 20,
                             ctypes.byref(h)) == 1
    assert L.su3s_field_wrap(lat, su3s.MATRIX, 1, su3s.F64, su3s.SOA, 0, None, 1 << 20,
                             ctypes.byref(h)) == 1


class Tree:
    """Expression handles over fake-pointer fields, for host-side checks."""

    def __init__(self, L, dims=(2, 2, 2, 2), nmu=1, prec=su3s.F64, layout=su3s.SOA, block=0):
        self.L = L
        rc, self.lat = _lat(L, dims)
        self.nmu, self.prec, self.layout, self.block = nmu, prec, layout, block
        self.keep = []

    def field(self, kind=su3s.MATRIX, prec=None, lat=None, nmu=None):
        h = ctypes.c_void_p()
        rc = self.L.su3s_field_wrap(lat or self.lat, kind, nmu or self.nmu,
                                    self.prec if prec is None else prec,
                                    self.layout, self.block, FAKE, 1 << 40, ctypes.byref(h))
        assert rc == 0, self.L.su3s_last_error()
        return h

    def leaf(self, f):
        e = ctypes.c_void_p()
        assert self.L.su3s_expr_leaf(f, ctypes.byref(e)) == 0
        return e

    def op(self, name, *args):
        e = ctypes.c_void_p()
        rc = getattr(self.L, "su3s_expr_" + name)(*args, ctypes.byref(e))
        return rc, e

    def sig(self, e):
        buf = ctypes.create_string_buffer(256)
        assert self.L.su3s_expr_signature(e, buf, 256) == 0
        return buf.value.decode()


def test_type_rules(L):
    t = Tree(L)
    m, v, r = t.leaf(t.field()), t.leaf(t.field(su3s.VECTOR)), t.leaf(t.field(su3s.REAL))
    assert t.op("mul", m, m)[0] == 0
    assert t.op("mul", m, v)[0] == 0
    assert t.op("mul", r, r)[0] == 0
    assert t.op("mul", v, m)[0] == 2
    assert t.op("mul", m, r)[0] == 2
    assert t.op("add", m, v)[0] == 2
    assert t.op("sub", v, r)[0] == 2
    assert t.op("adj", v)[0] == 2
    assert t.op("adj", m)[0] == 0
    assert t.op("scale", ctypes.c_double(2.0), v)[0] == 0


def test_canonical_signatures(L):
    t = Tree(L)
    a, b, c, d = (t.leaf(t.field()) for _ in range(4))
    _, ab = t.op("mul", a, b)
    _, cd = t.op("mul", c, d)
    _, e1 = t.op("add", ab, cd)
    assert t.sig(e1) == "add(mul(M0,M1),mul(M2,M3))"
    _, abc = t.op("mul", ab, c)
    _, hd = t.op("scale", ctypes.c_double(0.5), d)
    _, e2 = t.op("add", abc, hd)
    assert t.sig(e2) == "add(mul(mul(M0,M1),M2),scale(s0,M3))"
    _, aa = t.op("adj", a)
    _, l3 = t.op("mul", aa, b)
    _, r3 = t.op("mul", b, aa)
    _, e3 = t.op("sub", l3, r3)
    assert t.sig(e3) == "sub(mul(adj(M0),M1),mul(M1,adj(M0)))"
    n = ctypes.c_int()
    assert L.su3s_expr_num_leaves(e3, ctypes.byref(n)) == 0 and n.value == 2
    # the same field twice is one leaf slot
    _, sq = t.op("mul", a, a)
    assert t.sig(sq) == "mul(M0,M0)"
    # children may be freed before the parent (reference counting)
    for h in (a, b, c, d, ab, cd, abc, hd, aa, l3, r3):
        assert L.su3s_expr_free(h) == 0
    assert t.sig(e1) == "add(mul(M0,M1),mul(M2,M3))"
    for h in (e1, e2, e3, sq):
        assert L.su3s_expr_free(h) == 0


def test_catalogue_covers_hot_path_rows(L):
    cat = set(su3s.catalogue())
    for math in ("f64", "df32", "fx"):
        for sig in ("mul(M0,M1)", "mul(M0,V1)", "add(mul(M0,M1),mul(M2,M3))",
                    "add(mul(mul(M0,M1),M2),scale(s0,M3))", "sub(mul(adj(M0),M1),mul(M1,adj(M0)))",
                    "add(add(R0,R1),mul(R0,R1))"):
            assert ("eval", sig, "f64", math) in cat
        for sig in ("mul(M0,M1)", "add(mul(M0,M1),mul(M2,M3))", "mul(M0,V1)"):
            assert ("adjoint", sig, "f64", math) in cat
    for p in ("f32", "bf16", "f16"):
        assert ("eval", "mul(M0,M1)", p, "f32") in cat
    assert ("eval", "mul(M0,M1)", "f64_c12", "df32") in cat
    assert ("eval", "mul(M0,M1)", "f64_c12", "fx") in cat
    assert ("eval", "mul(M0,M1)", "f64_c12", "f64") in cat
    assert ("eval", "mul(M0,M1)", "f32_c12", "f32") in cat


def test_eval_validation_before_any_launch(L):
    t = Tree(L)
    a, b = t.leaf(t.field()), t.leaf(t.field())
    _, ab = t.op("mul", a, b)
    vdest = t.field(su3s.VECTOR)
    assert L.su3s_eval_math(vdest, ab, 0, None) == 2                 # kind mismatch
    rc, lat2 = _lat(L, (2, 2, 2, 3))
    other = t.field(lat=lat2)
    assert L.su3s_eval_math(other, ab, 0, None) == 3                 # other lattice
    f32 = t.field(prec=su3s.F32)
    assert L.su3s_eval_math(f32, ab, 0, None) == 3                   # precision mismatch
    assert L.su3s_eval_math(t.field(), ab, 7, None) == 1             # bad arithmetic
    c12 = Tree(L, prec=su3s.F64_C12)
    x, y = c12.leaf(c12.field()), c12.leaf(c12.field())
    _, s = c12.op("add", x, y)
    assert L.su3s_eval_math(c12.field(), s, 0, None) == 6            # sums leave SU(3)
    many = [t.leaf(t.field()) for _ in range(7)]
    acc = many[0]
    for h in many[1:]:
        _, acc = t.op("add", acc, h)
    assert L.su3s_eval_math(t.field(), acc, 0, None) == 6            # too many leaves
    assert L.su3s_set_default_math(5) == 1
    assert L.su3s_set_default_math(0) == 1
    assert L.su3s_set_default_math(su3s.MATH_FX) == 0
    assert L.su3s_set_default_math(su3s.MATH_DF32) == 0


def test_adjoint_validation(L):
    t = Tree(L)
    a, b = t.leaf(t.field()), t.leaf(t.field())
    _, ab = t.op("mul", a, b)
    g = t.field()
    arr = (ctypes.c_void_p * 2)(t.field(), t.field())
    assert L.su3s_eval_adjoint(ab, g, arr, 1, 0, None) == 1          # wrong count
    assert L.su3s_eval_adjoint(ab, t.field(su3s.VECTOR), arr, 2, 0, None) == 2
    arr2 = (ctypes.c_void_p * 2)(t.field(su3s.VECTOR), None)
    assert L.su3s_eval_adjoint(ab, g, arr2, 2, 0, None) == 2          # gradient kind
    assert L.su3s_tune_adjoint(ab, g, arr, 1, 0, None, None, None, None, None) == 1
    assert L.su3s_tune_adjoint(ab, g, arr2, 2, 0, None, None, None, None, None) == 2
    assert L.su3s_tune_adjoint(ab, g, arr, 2, 9, None, None, None, None, None) == 1  # arithmetic


def test_batch_validation(L):
    t = Tree(L)
    b = ctypes.c_void_p()
    assert L.su3s_batch_create(ctypes.byref(b)) == 0
    a, c = t.leaf(t.field()), t.leaf(t.field())
    _, ac = t.op("mul", a, c)
    assert L.su3s_batch_add(b, t.field(su3s.VECTOR), ac) == 2
    assert L.su3s_batch_add(b, t.field(prec=su3s.F32), ac) == 6
    assert L.su3s_batch_launch(b, None) == 1                          # not built
    assert L.su3s_batch_build(b, 0, 100, 0, None) == 1                # bad threads
    assert L.su3s_batch_destroy(b) == 0


def test_package_never_reaches_the_oracle():
    """The product package has no host implementation of the method: none of
    its Python files import the oracle or the input generator."""
    pkg = os.path.dirname(su3s.__file__)
    for fn in os.listdir(pkg):
        if fn.endswith(".py"):
            src = open(os.path.join(pkg, fn)).read()
            for mod in ("oracle", "synth"):
                assert "import %s" % mod not in src and "from %s" % mod not in src, fn


def test_pipeline_modes(L):
    for mode in (-1, 0, 1, 2, 3, 4):
        assert L.su3s_set_pipeline(mode) == 0
    assert L.su3s_set_pipeline(5) == 1
    assert L.su3s_set_pipeline(-2) == 1
    assert L.su3s_set_pipeline(-1) == 0


def _wrap(L, lat, kind, nmu, prec, addr):
    n = ctypes.c_size_t()
    assert L.su3s_field_bytes(lat, kind, nmu, prec, su3s.SOA, 0, ctypes.byref(n)) == 0
    h = ctypes.c_void_p()
    assert L.su3s_field_wrap(lat, kind, nmu, prec, su3s.SOA, 0, addr, n.value, ctypes.byref(h)) == 0
    return h


def test_neighbour_operation_validation(L):
    """Argument checks of su3s_cshift and su3s_hop (nothing reaches the GPU)."""
    rc, lat = _lat(L, (2, 2, 2, 2))
    rc2, other = _lat(L, (2, 2, 2, 3))
    gap = 1 << 24
    m1 = _wrap(L, lat, su3s.MATRIX, 1, su3s.F64, FAKE)
    m2 = _wrap(L, lat, su3s.MATRIX, 1, su3s.F64, FAKE + gap)
    v1 = _wrap(L, lat, su3s.VECTOR, 1, su3s.F64, FAKE + 2 * gap)
    v2 = _wrap(L, lat, su3s.VECTOR, 1, su3s.F64, FAKE + 3 * gap)
    u4 = _wrap(L, lat, su3s.MATRIX, 4, su3s.F64, FAKE + 4 * gap)
    f32 = _wrap(L, lat, su3s.MATRIX, 1, su3s.F32, FAKE + 5 * gap)
    mo = _wrap(L, other, su3s.MATRIX, 1, su3s.F64, FAKE + 6 * gap)
    assert L.su3s_cshift(m1, m2, 4, 1, None) == 1                 # direction
    assert L.su3s_cshift(m1, m2, -1, 1, None) == 1
    assert L.su3s_cshift(m1, m1, 0, 1, None) == 1                 # overlap
    assert L.su3s_cshift(m1, v1, 0, 1, None) == 2                 # kind
    assert L.su3s_cshift(m1, f32, 0, 1, None) == 3                # precision
    assert L.su3s_cshift(m1, mo, 0, 1, None) == 3                 # lattice
    assert L.su3s_hop(v2, m2, v1, 0, None) == 2                   # links need 4 per site
    assert L.su3s_hop(m1, u4, v1, 0, None) == 2                   # destination kind
    assert L.su3s_hop(v1, u4, v1, 0, None) == 1                   # overlap
    assert L.su3s_hop(f32, u4, m2, 0, None) == 6                  # FP64 only
    assert L.su3s_hop(mo, u4, m2, 0, None) == 3                   # lattice
    assert L.su3s_hop(v2, u4, v1, 9, None) == 1                   # arithmetic
    # the Wilson hopping term: spinors are vector fields with 4 spin components
    s1 = _wrap(L, lat, su3s.VECTOR, 4, su3s.F64, FAKE + 7 * gap)
    s2 = _wrap(L, lat, su3s.VECTOR, 4, su3s.F64, FAKE + 8 * gap)
    s32 = _wrap(L, lat, su3s.VECTOR, 4, su3s.F32, FAKE + 9 * gap)
    so = _wrap(L, other, su3s.VECTOR, 4, su3s.F64, FAKE + 10 * gap)
    assert L.su3s_dslash(s2, m2, s1, 0, None) == 2                # links need 4 per site
    assert L.su3s_dslash(s2, u4, v1, 0, None) == 2                # psi: 4 spin components
    assert L.su3s_dslash(v2, u4, s1, 0, None) == 2                # dst: 4 spin components
    assert L.su3s_dslash(s1, u4, s1, 0, None) == 1                # overlap
    assert L.su3s_dslash(s32, u4, s1, 0, None) == 6               # FP64 only
    assert L.su3s_dslash(so, u4, s1, 0, None) == 3                # lattice
    assert L.su3s_dslash(s2, u4, s1, 9, None) == 1                # arithmetic
    assert L.su3s_dslash(None, u4, s1, 0, None) == 1              # null


def test_batch_rejects_items_that_touch_each_other(L):
    """Batch items run concurrently: an item may not write what another reads."""
    rc, lat = _lat(L, (2, 2, 2, 2))
    gap = 1 << 24
    f = [_wrap(L, lat, su3s.MATRIX, 1, su3s.F64, FAKE + k * gap) for k in range(5)]
    lv = []
    for h in f:
        e = ctypes.c_void_p()
        assert L.su3s_expr_leaf(h, ctypes.byref(e)) == 0
        lv.append(e)
    p01, p23 = ctypes.c_void_p(), ctypes.c_void_p()
    assert L.su3s_expr_mul(lv[0], lv[1], ctypes.byref(p01)) == 0
    assert L.su3s_expr_mul(lv[2], lv[3], ctypes.byref(p23)) == 0
    b = ctypes.c_void_p()
    assert L.su3s_batch_create(ctypes.byref(b)) == 0
    assert L.su3s_batch_add(b, f[2], p01) == 0       # item 0 writes f2 ...
    assert L.su3s_batch_add(b, f[4], p23) == 0       # ... which item 1 reads
    assert L.su3s_batch_build(b, 0, 0, 0, None) == 1
    assert b"item" in L.su3s_last_error()
    assert L.su3s_batch_tune(b, 0, None, None, None, None, None) == 1
    assert b"item" in L.su3s_last_error()
    assert L.su3s_batch_tune(b, 9, None, None, None, None, None) == 1
    assert L.su3s_batch_tune(None, 0, None, None, None, None, None) == 1
    assert L.su3s_batch_destroy(b) == 0


@pytest.mark.parametrize("kind,prec,ncomp,eb", [
    (su3s.MATRIX, su3s.F64, 9, 16), (su3s.MATRIX, su3s.F32, 9, 8), (su3s.MATRIX, su3s.BF16, 9, 4),
    (su3s.MATRIX, su3s.F16, 9, 4), (su3s.MATRIX, su3s.F64_C12, 6, 16),
    (su3s.MATRIX, su3s.F32_C12, 6, 8), (su3s.VECTOR, su3s.BF16, 3, 4), (su3s.REAL, su3s.F64, 1, 8)])
def test_stored_transfer_sizes_and_validation(L, kind, prec, ncomp, eb):
    """The stored-format array has V*nmu*ncomp elements of the stored size (no
    padding); a wrong size or a null pointer is refused before any copy."""
    rc, lat = _lat(L, (3, 2, 1, 5))   # V = 30
    for nmu in (1, 4):
        h = _wrap(L, lat, kind, nmu, prec, FAKE)
        n = ctypes.c_size_t()
        assert L.su3s_field_stored_bytes(h, ctypes.byref(n)) == 0
        assert n.value == 30 * nmu * ncomp * eb
        buf = ctypes.create_string_buffer(n.value + 16)
        assert L.su3s_field_upload_stored(h, buf, n.value - eb, None) == 3
        assert L.su3s_field_download_stored(h, buf, n.value + eb, None) == 3
        assert b"stores" in L.su3s_last_error()
        assert L.su3s_field_upload_stored(h, None, n.value, None) == 1
        assert L.su3s_field_download_stored(None, buf, n.value, None) == 1
        assert L.su3s_field_stored_bytes(h, None) == 1
        assert L.su3s_field_destroy(h) == 0


def test_version_and_last_error(L):
    """su3s_version is 10000*major + 100*minor + patch; a successful call leaves
    the thread's message empty, a failed one sets it."""
    v = L.su3s_version()
    assert v >= 10000 and v % 100 < 100 and (v // 100) % 100 < 100
    rc, lat = _lat(L, (2, 2, 2, 2))
    assert rc == 0 and L.su3s_last_error() == b""
    assert L.su3s_lattice_volume(None, None) == 1 and L.su3s_last_error() != b""


def test_bounded_wait_selftest_validation(L):
    c = ctypes.c_int64()
    assert L.su3s_selftest_bounded_wait(0, ctypes.byref(c), None) == 1
    assert L.su3s_selftest_bounded_wait((1 << 20) + 1, ctypes.byref(c), None) == 1
    assert L.su3s_selftest_bounded_wait(16, None, None) == 1
