"""Plain CPU oracle for site-local lattice expression evaluation (FP64).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg may use it; the product path never does.  It is a thin ctypes
wrapper over ``su3_oracle.c`` (single-threaded C, no FMA contraction) and
shares no code with the CUDA library.

Each function cites the passage of arXiv:1710.09409 it follows (see the C file
for the definitions):
  mm, mv          Sec. 4, Listing 3 (z = x*y per site)
  eval_tree       Sec. 3, Listing 1 (per-site recursive evaluation of an
                  expression) and Listing 2 (composite expressions)
  eval_adjoint    reverse mode of eval_tree (gradient of a real loss)
  round_to        storage precisions, IEEE 754 round-to-nearest-even
  c12_expand      third row of an SU(3) matrix rebuilt from rows 0 and 1
  redot           sum_x Re tr(X^dagger Y)
  reunitarize     projection to SU(3): Gram-Schmidt over rows, det phase removed
  cshift          Sec. 6 (Cshift): circular shift along one lattice direction
  hop             Sec. 6 (Dslash): colour part of the nearest-neighbour
                  hopping term, sum_mu U_mu(x) v(x+mu) + U_mu(x-mu)^dagger v(x-mu)
  dslash          Sec. 6 (Dslash): the Wilson hopping term with its spin
                  structure, sum_mu (1 - g_mu) U_mu(x) psi(x+mu)
                  + (1 + g_mu) U_mu(x-mu)^dagger psi(x-mu) on spinor fields
  gamma           the Euclidean gamma matrices (chiral basis) dslash uses

Parity status: every function here is pinned by the CPU tests in
tests/test_oracle.py (brute force against numpy/torch, closed forms,
identities, invariants, finite differences).

Trees are nested tuples:
  ("leaf", name) | ("mul", x, y) | ("add", x, y) | ("sub", x, y)
  | ("scale", s, x) | ("adj", x)
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "su3_oracle.c")
_LIB = os.path.join(_HERE, "_oracle.so")
_lib = None

MATRIX, VECTOR, REAL = 0, 1, 2
_OPS = {"leaf": 0, "mul": 1, "add": 2, "sub": 3, "scale": 4, "adj": 5}
FORMATS = {"f32": 0, "bf16": 1, "f16": 2}


class _Node(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int), ("a", ctypes.c_int), ("b", ctypes.c_int),
                ("leaf", ctypes.c_int), ("s", ctypes.c_double)]


def build(force=False):
    """Compile the oracle with gcc (-O2, no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _bind(lib):
    """Declare the C signatures on a loaded oracle library."""
    P, I64 = ctypes.c_void_p, ctypes.c_int64
    lib.oracle_mm.argtypes = [P, P, P, I64]
    lib.oracle_mv.argtypes = [P, P, P, I64]
    lib.oracle_eval.argtypes = [P, ctypes.c_int, ctypes.c_int, P, P, ctypes.c_int, I64, P]
    lib.oracle_eval.restype = ctypes.c_int
    lib.oracle_eval_adjoint.argtypes = [P, ctypes.c_int, ctypes.c_int, P, P, ctypes.c_int,
                                        I64, P, P]
    lib.oracle_eval_adjoint.restype = ctypes.c_int
    lib.oracle_round.argtypes = [P, P, I64, ctypes.c_int]
    lib.oracle_round.restype = ctypes.c_int
    lib.oracle_c12_expand.argtypes = [P, P, I64]
    lib.oracle_redot.argtypes = [P, P, I64]
    lib.oracle_redot.restype = ctypes.c_double
    lib.oracle_reunitarize.argtypes = [P, P, I64]
    lib.oracle_cshift.argtypes = [P, P, P, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.oracle_cshift.restype = None
    lib.oracle_hop.argtypes = [P, P, P, P, ctypes.c_int]
    lib.oracle_hop.restype = None
    lib.oracle_dslash.argtypes = [P, P, P, P, ctypes.c_int]
    lib.oracle_dslash.restype = None
    lib.oracle_gamma.argtypes = [ctypes.c_int, P]
    lib.oracle_gamma.restype = ctypes.c_int
    return lib


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = _bind(ctypes.CDLL(_LIB))
    return _lib


def _c(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a


def _kind_of(arr):
    tail = arr.shape[1:]
    if tail == (3, 3, 2):
        return MATRIX
    if tail == (3, 2):
        return VECTOR
    if tail == ():
        return REAL
    raise ValueError("unrecognised field shape %r" % (arr.shape,))


def mm(x, y):
    """z = x*y for every element; x, y canonical (n,3,3,2) float64."""
    x, y = _c(x), _c(y)
    assert x.shape == y.shape and x.shape[1:] == (3, 3, 2)
    z = np.empty_like(x)
    _load().oracle_mm(x.ctypes.data, y.ctypes.data, z.ctypes.data, x.shape[0])
    return z


def mv(x, v):
    """z = x*v for every element; x (n,3,3,2), v (n,3,2)."""
    x, v = _c(x), _c(v)
    assert x.shape[0] == v.shape[0] and x.shape[1:] == (3, 3, 2) and v.shape[1:] == (3, 2)
    z = np.empty_like(v)
    _load().oracle_mv(x.ctypes.data, v.ctypes.data, z.ctypes.data, x.shape[0])
    return z


def compile_tree(tree, names):
    """Flatten a nested-tuple tree into postfix nodes (children first).

    `names` is the ordered list of leaf names (leaf slot = index)."""
    nodes = []

    def rec(t):
        op = t[0]
        if op == "leaf":
            nodes.append((0, -1, -1, names.index(t[1]), 0.0))
        elif op in ("mul", "add", "sub"):
            a = rec(t[1])
            b = rec(t[2])
            nodes.append((_OPS[op], a, b, -1, 0.0))
        elif op == "scale":
            a = rec(t[2])
            nodes.append((4, a, -1, -1, float(t[1])))
        elif op == "adj":
            a = rec(t[1])
            nodes.append((5, a, -1, -1, 0.0))
        else:
            raise ValueError("unknown op %r" % (op,))
        return len(nodes) - 1

    root = rec(tree)
    arr = (_Node * len(nodes))(*[_Node(*n) for n in nodes])
    return arr, len(nodes), root


def leaf_names(tree, acc=None):
    """Leaf names in order of first appearance."""
    acc = [] if acc is None else acc
    if tree[0] == "leaf":
        if tree[1] not in acc:
            acc.append(tree[1])
    elif tree[0] == "scale":
        leaf_names(tree[2], acc)
    else:
        for sub in tree[1:]:
            leaf_names(sub, acc)
    return acc


def _result_shape(tree, leaves):
    op = tree[0]
    if op == "leaf":
        return leaves[tree[1]].shape[1:]
    if op == "mul":
        return _result_shape(tree[2], leaves)
    if op in ("add", "sub"):
        return _result_shape(tree[1], leaves)
    if op == "scale":
        return _result_shape(tree[2], leaves)
    return (3, 3, 2)


def eval_tree(tree, leaves):
    """Value of `tree` at every element; `leaves` maps names to canonical arrays."""
    names = leaf_names(tree)
    arrs = [_c(leaves[n]) for n in names]
    n = arrs[0].shape[0]
    assert all(a.shape[0] == n for a in arrs)
    nodes, nn, root = compile_tree(tree, names)
    ptrs = (ctypes.c_void_p * len(arrs))(*[a.ctypes.data for a in arrs])
    kinds = (ctypes.c_int * len(arrs))(*[_kind_of(a) for a in arrs])
    out = np.empty((n,) + tuple(_result_shape(tree, leaves)), dtype=np.float64)
    rc = _load().oracle_eval(ctypes.addressof(nodes), nn, root, ptrs, kinds, len(arrs), n,
                             out.ctypes.data)
    if rc != 0:
        raise ValueError("ill-typed or malformed expression tree")
    return out


def eval_adjoint(tree, leaves, gz):
    """Gradients dL/d(leaf) of a real loss with dL/d(tree value) = gz."""
    names = leaf_names(tree)
    arrs = [_c(leaves[n]) for n in names]
    n = arrs[0].shape[0]
    gz = _c(gz)
    nodes, nn, root = compile_tree(tree, names)
    grads = [np.zeros_like(a) for a in arrs]
    ptrs = (ctypes.c_void_p * len(arrs))(*[a.ctypes.data for a in arrs])
    gptrs = (ctypes.c_void_p * len(arrs))(*[g.ctypes.data for g in grads])
    kinds = (ctypes.c_int * len(arrs))(*[_kind_of(a) for a in arrs])
    rc = _load().oracle_eval_adjoint(ctypes.addressof(nodes), nn, root, ptrs, kinds, len(arrs),
                                     n, gz.ctypes.data, gptrs)
    if rc != 0:
        raise ValueError("ill-typed or malformed expression tree")
    return dict(zip(names, grads))


def round_to(x, fmt):
    """Round every value to FP32 / BF16 / FP16 (nearest, ties to even); float64 out."""
    x = _c(x)
    out = np.empty_like(x)
    rc = _load().oracle_round(x.ctypes.data, out.ctypes.data, x.size, FORMATS[fmt])
    if rc != 0:
        raise ValueError(fmt)
    return out


def c12_expand(rows01):
    """Full (n,3,3,2) matrices from rows 0,1 (n,2,3,2): row 2 = conj(row0 x row1)."""
    r = _c(rows01)
    assert r.shape[1:] == (2, 3, 2)
    out = np.empty((r.shape[0], 3, 3, 2))
    _load().oracle_c12_expand(r.ctypes.data, out.ctypes.data, r.shape[0])
    return out


def redot(x, y):
    """sum over all reals of x*y (= sum_x Re tr(X^dagger Y) for matrix fields)."""
    x, y = _c(x), _c(y)
    assert x.shape == y.shape
    return _load().oracle_redot(x.ctypes.data, y.ctypes.data, x.size)


def reunitarize(x):
    """Projection of every matrix to SU(3) (Gram-Schmidt over rows, det phase removed)."""
    x = _c(x)
    out = np.empty_like(x)
    _load().oracle_reunitarize(x.ctypes.data, out.ctypes.data, x.shape[0])
    return out


def _dims(dims):
    d = (ctypes.c_int * 4)(*[int(x) for x in dims])
    assert all(x >= 1 for x in dims)
    return d


def cshift(x, dims, dim, shift):
    """dst(s) = x(s + shift * e_dim), periodic (the Cshift of Sec. 6).  x: canonical
    field array whose first axis runs over sites (all links and components of
    a site follow)."""
    x = _c(x)
    v = int(np.prod(dims))
    assert x.shape[0] == v and 0 <= dim < 4
    out = np.empty_like(x)
    _load().oracle_cshift(x.ctypes.data, out.ctypes.data, _dims(dims), x.size // v, dim, shift)
    return out


def hop(u, x, dims):
    """out(s) = sum_mu U_mu(s) x(s+mu) + U_mu(s-mu)^dagger x(s-mu): the colour part
    of the Dslash hopping term (Sec. 6).  u: (V*4, 3, 3, 2) links; x: (V, 3, 3, 2)
    matrices or (V, 3, 2) vectors."""
    u, x = _c(u), _c(x)
    v = int(np.prod(dims))
    assert u.shape == (4 * v, 3, 3, 2) and x.shape[0] == v
    kind = {(3, 3, 2): 0, (3, 2): 1}[x.shape[1:]]
    out = np.empty_like(x)
    _load().oracle_hop(u.ctypes.data, x.ctypes.data, out.ctypes.data, _dims(dims), kind)
    return out


def gamma(mu):
    """gamma_mu (mu = 0..3, directions x, y, z, t) or gamma_5 (mu = 4) of the
    chiral basis dslash uses, as a complex (4, 4) array."""
    out = np.empty((4, 4, 2))
    if _load().oracle_gamma(int(mu), out.ctypes.data) != 0:
        raise ValueError(mu)
    return out[..., 0] + 1j * out[..., 1]


def dslash(u, psi, dims, r=1):
    """out(s) = sum_mu (1 - r g_mu) U_mu(s) psi(s+mu) + (1 + r g_mu) U_mu(s-mu)^dagger psi(s-mu):
    the Wilson hopping term with spin (Sec. 6; r = 1 is the operator, r = -1
    swaps the projectors).  u: (V*4, 3, 3, 2) links; psi: (V*4, 3, 2) or
    (V, 4, 3, 2) spinors (spin s of site x at row 4x + s)."""
    u, psi = _c(u), _c(psi)
    v = int(np.prod(dims))
    assert u.shape == (4 * v, 3, 3, 2) and psi.size == 24 * v
    out = np.empty_like(psi)
    _load().oracle_dslash(u.ctypes.data, psi.ctypes.data, out.ctypes.data, _dims(dims), int(r))
    return out
