"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each check compares the oracle with something other than itself: numpy/torch
library routines (brute force on tiny lattices), closed forms, group
identities and invariants, the values of the paper's Listing 2, and finite
differences.  Tolerances follow from FP64 rounding of O(1) quantities.
"""
import os

import numpy as np
import pytest

import oracle
import synth
from helpers import E1, E2, E3, cplx, lattice_fields, real_view

TINY = [(1, 1, 1, 1), (2, 2, 2, 2), (3, 2, 1, 5)]
SEED = synth.SEED_BASE + 0


def adj(c):
    return np.conj(np.swapaxes(c, -1, -2))


# ---------------------------------------------------------------- brute force
@pytest.mark.parametrize("dims", TINY)
def test_mm_matches_numpy_matmul(dims):
    f = lattice_fields(dims, SEED)
    z = oracle.mm(f["a"], f["b"])
    ref = np.matmul(cplx(f["a"]), cplx(f["b"]))
    assert np.abs(cplx(z) - ref).max() < 1e-14


@pytest.mark.parametrize("dims", TINY)
def test_mm_gaussian_matches_einsum(dims):
    v = synth.volume(dims)
    a = synth.gauss_matrix(SEED, 0, v)
    b = synth.gauss_matrix(SEED, 1, v)
    ref = np.einsum("nij,njk->nik", cplx(a), cplx(b))
    assert np.abs(cplx(oracle.mm(a, b)) - ref).max() < 1e-13


@pytest.mark.parametrize("dims", TINY)
def test_mv_matches_einsum(dims):
    f = lattice_fields(dims, SEED, names=("a", "v"))
    z = oracle.mv(f["a"], f["v"])
    ref = np.einsum("nij,nj->ni", cplx(f["a"]), cplx(f["v"]))
    assert np.abs(cplx(z) - ref).max() < 1e-14


def test_lorentz_equals_four_independent_products():
    dims = (3, 2, 1, 5)
    v = synth.volume(dims)
    f = lattice_fields(dims, SEED, nmu=4)
    z = oracle.mm(f["a"], f["b"])
    for mu in range(4):
        zmu = oracle.mm(f["a"][mu::4].copy(), f["b"][mu::4].copy())
        assert np.array_equal(z[mu::4], zmu)
    assert z.shape == (4 * v, 3, 3, 2)


def test_tree_single_product_is_mm():
    f = lattice_fields((2, 2, 2, 2), SEED)
    z = oracle.eval_tree(("mul", ("leaf", "a"), ("leaf", "b")), f)
    assert np.array_equal(z, oracle.mm(f["a"], f["b"]))


# ----------------------------------------------------------- group identities
def _identity(n):
    e = np.zeros((n, 3, 3), complex)
    e[:, [0, 1, 2], [0, 1, 2]] = 1.0
    return real_view(e)


def test_identity_products_exact():
    f = lattice_fields((2, 2, 2, 2), SEED)
    n = f["a"].shape[0]
    eye = _identity(n)
    # a*I = a and I*b = b exactly (up to the sign of zero: + 0.0 folds -0 to +0)
    assert np.array_equal(oracle.mm(f["a"], eye) + 0.0, f["a"] + 0.0)
    assert np.array_equal(oracle.mm(eye, f["b"]) + 0.0, f["b"] + 0.0)


def test_inverse_is_adjoint():
    f = lattice_fields((3, 2, 1, 5), SEED)
    z = oracle.eval_tree(("mul", ("leaf", "a"), ("adj", ("leaf", "a"))), f)
    assert np.abs(cplx(z) - np.eye(3)).max() < 1e-14
    z = oracle.eval_tree(("mul", ("adj", ("leaf", "a")), ("leaf", "a")), f)
    assert np.abs(cplx(z) - np.eye(3)).max() < 1e-14


def test_trace_cyclicity():
    dims = (2, 2, 2, 2)
    v = synth.volume(dims)
    a = synth.gauss_matrix(SEED, 0, v)
    b = synth.gauss_matrix(SEED, 1, v)
    tab = np.trace(cplx(oracle.mm(a, b)), axis1=1, axis2=2)
    tba = np.trace(cplx(oracle.mm(b, a)), axis1=1, axis2=2)
    assert np.abs(tab - tba).max() < 1e-13


def test_products_of_su3_stay_in_su3():
    f = lattice_fields((3, 2, 1, 5), SEED)
    z = cplx(oracle.mm(f["a"], f["b"]))
    assert np.abs(z @ adj(z) - np.eye(3)).max() < 1e-12
    assert np.abs(np.linalg.det(z) - 1.0).max() < 1e-12


def test_associativity():
    f = lattice_fields((2, 2, 2, 2), SEED, names=("a", "b", "c"))
    left = oracle.mm(oracle.mm(f["a"], f["b"]), f["c"])
    right = oracle.mm(f["a"], oracle.mm(f["b"], f["c"]))
    assert np.abs(left - right).max() < 1e-13


def test_matrix_vector_preserves_norm():
    f = lattice_fields((3, 2, 1, 5), SEED, names=("a", "v"))
    z = cplx(oracle.mv(f["a"], f["v"]))
    nv = np.linalg.norm(cplx(f["v"]), axis=1)
    assert np.abs(np.linalg.norm(z, axis=1) - nv).max() < 1e-13


# --------------------------------------------------------------- closed forms
def _diag_phase(al, be):
    n = al.shape[0]
    d = np.zeros((n, 3, 3), complex)
    d[:, 0, 0] = np.exp(1j * al)
    d[:, 1, 1] = np.exp(1j * be)
    d[:, 2, 2] = np.exp(-1j * (al + be))
    return d


def test_closed_form_diagonal_phases():
    rng = np.random.default_rng(7)
    a1, b1, a2, b2 = (rng.uniform(-3, 3, 50) for _ in range(4))
    z = cplx(oracle.mm(real_view(_diag_phase(a1, b1)), real_view(_diag_phase(a2, b2))))
    assert np.abs(z - _diag_phase(a1 + a2, b1 + b2)).max() < 1e-15


def test_closed_form_rotations_compose():
    th1, th2 = np.linspace(-3, 3, 40), np.linspace(2, -1, 40)

    def rot(t):
        r = np.zeros((t.shape[0], 3, 3), complex)
        r[:, 0, 0] = r[:, 1, 1] = np.cos(t)
        r[:, 0, 1] = -np.sin(t) * 1j
        r[:, 1, 0] = -np.sin(t) * 1j
        r[:, 2, 2] = 1.0
        return r

    z = cplx(oracle.mm(real_view(rot(th1)), real_view(rot(th2))))
    assert np.abs(z - rot(th1 + th2)).max() < 1e-15


def test_closed_form_cyclic_permutation():
    p = np.zeros((1, 3, 3), complex)
    p[0, 0, 1] = p[0, 1, 2] = p[0, 2, 0] = 1.0
    pp = real_view(p)
    p3 = oracle.eval_tree(("mul", ("mul", ("leaf", "p"), ("leaf", "p")), ("leaf", "p")), {"p": pp})
    assert np.array_equal(cplx(p3), np.eye(3)[None].astype(complex))


# ------------------------------------------------------------- golden (paper)
def _listing2_rows():
    path = os.path.join(os.path.dirname(__file__), "golden", "listing2.txt")
    rows = []
    for line in open(path):
        line = line.strip()
        if line and not line.startswith("#"):
            v1, v2, expr, v3 = line.split()
            rows.append((float(v1), float(v2), expr, float(v3)))
    return rows


def test_listing2_composite_real_expressions():
    rows = _listing2_rows()
    assert len(rows) == 2
    dims = (3, 2, 1, 5)
    v = synth.volume(dims)
    trees = {"v1+v2": ("add", ("leaf", "v1"), ("leaf", "v2")),
             "v1+v2+v1*v2": ("add", ("add", ("leaf", "v1"), ("leaf", "v2")),
                             ("mul", ("leaf", "v1"), ("leaf", "v2")))}
    for v1, v2, expr, v3 in rows:
        leaves = {"v1": np.full(v, v1), "v2": np.full(v, v2)}
        out = oracle.eval_tree(trees[expr], leaves)
        assert np.array_equal(out, np.full(v, v3))


# -------------------------------------------------------------- fused trees
def test_fused_trees_equal_term_by_term():
    f = lattice_fields((3, 2, 1, 5), SEED, names=("a", "b", "c", "d"))
    ab = oracle.mm(f["a"], f["b"])
    e1 = oracle.eval_tree(E1, f)
    assert np.abs(e1 - (ab + oracle.mm(f["c"], f["d"]))).max() < 1e-15
    e2 = oracle.eval_tree(E2, f)
    assert np.abs(e2 - (oracle.mm(ab, f["c"]) + 0.5 * f["d"])).max() < 1e-15
    ca = cplx(f["a"])
    cb = cplx(f["b"])
    e3 = cplx(oracle.eval_tree(E3, f))
    assert np.abs(e3 - (adj(ca) @ cb - cb @ adj(ca))).max() < 1e-14
    assert np.abs(np.trace(e3, axis1=1, axis2=2)).max() < 1e-13


def test_commutator_tree():
    """a*b - b*a: numpy's matrix products, a vanishing trace (tr(ab) = tr(ba)),
    and exactly zero when b is the identity or when b = a."""
    dims = (3, 2, 1, 5)
    f = lattice_fields(dims, SEED, names=("a", "b"))
    comm = ("sub", ("mul", ("leaf", "a"), ("leaf", "b")), ("mul", ("leaf", "b"), ("leaf", "a")))
    ca, cb = cplx(f["a"]), cplx(f["b"])
    z = cplx(oracle.eval_tree(comm, f))
    assert np.abs(z - (ca @ cb - cb @ ca)).max() < 1e-14
    assert np.abs(np.trace(z, axis1=1, axis2=2)).max() < 1e-14
    eye = np.zeros_like(f["a"])
    eye[:, [0, 1, 2], [0, 1, 2], 0] = 1.0
    zi = oracle.eval_tree(comm, {"a": f["a"], "b": eye})
    assert np.array_equal(zi + 0.0, np.zeros_like(eye))
    za = oracle.eval_tree(comm, {"a": f["a"], "b": f["a"]})
    assert np.array_equal(za + 0.0, np.zeros_like(eye))


def test_ill_typed_trees_are_rejected():
    f = lattice_fields((1, 1, 1, 1), SEED, names=("a", "v"))
    with pytest.raises(ValueError):
        oracle.eval_tree(("mul", ("leaf", "v"), ("leaf", "a")), f)
    with pytest.raises(ValueError):
        oracle.eval_tree(("add", ("leaf", "v"), ("leaf", "a")), f)
    with pytest.raises(ValueError):
        oracle.eval_tree(("adj", ("leaf", "v")), f)


# ------------------------------------------------------------------ rounding
def _edge_values():
    rng = np.random.default_rng(3)
    x = np.concatenate([
        rng.standard_normal(20000),
        rng.standard_normal(2000) * 1e-30,
        rng.standard_normal(2000) * 1e-42,      # FP32 subnormal range
        rng.standard_normal(2000) * 1e-6,       # FP16 subnormal range
        rng.standard_normal(2000) * 1e4,
        np.array([0.0, -0.0, 65504.0, 65519.9, 65520.0, 1e39, -1e39, 3.4028235e38,
                  1.0 + 2.0 ** -24, 1.0 + 3 * 2.0 ** -24, 1.0 + 2.0 ** -11, 1.0 + 3 * 2.0 ** -11,
                  2.0 ** -149, 2.0 ** -150, 3 * 2.0 ** -151, 2.0 ** -24, 2.0 ** -25,
                  6e-8, 5.960464477539063e-08]),
    ])
    return x


def test_round_f32_matches_numpy():
    x = _edge_values()
    with np.errstate(over="ignore"):
        ref = x.astype(np.float32).astype(np.float64)
    assert np.array_equal(oracle.round_to(x, "f32"), ref)


def test_round_f16_matches_numpy():
    x = _edge_values()
    with np.errstate(over="ignore"):
        ref = x.astype(np.float16).astype(np.float64)
    assert np.array_equal(oracle.round_to(x, "f16"), ref)


def test_round_bf16_matches_torch_on_fp32_values():
    torch = pytest.importorskip("torch")
    x = _edge_values()
    with np.errstate(over="ignore"):
        x32 = x.astype(np.float32)
    x32 = x32[np.isfinite(x32)].astype(np.float64)   # values exact in FP32: no double rounding
    ref = torch.from_numpy(x32).to(torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(oracle.round_to(x32, "bf16"), ref)


def test_round_bf16_ties_to_even():
    # 1 + 2^-8 is halfway between 1 and 1 + 2^-7: ties go to the even significand (1.0)
    x = np.array([1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -8 + 2.0 ** -30])
    assert np.array_equal(oracle.round_to(x, "bf16"),
                          np.array([1.0, 1.0 + 2 * 2.0 ** -7, 1.0 + 2.0 ** -7]))


# ---------------------------------------------------------------- 12 reals
def test_c12_expand_recovers_su3():
    f = lattice_fields((3, 2, 1, 5), SEED)
    u = f["a"]
    full = oracle.c12_expand(u[:, :2].copy())
    assert np.abs(full - u).max() < 1e-15


def test_c12_expand_closed_form_identity_rows():
    r = np.zeros((1, 2, 3, 2))
    r[0, 0, 0, 0] = 1.0
    r[0, 1, 1, 0] = 1.0
    full = oracle.c12_expand(r)
    assert np.array_equal(cplx(full)[0] + 0.0, np.eye(3).astype(complex))


# ------------------------------------------------------------------ adjoint
def test_adjoint_closed_form_for_product():
    dims = (3, 2, 1, 5)
    f = lattice_fields(dims, SEED, names=("a", "b", "w"))
    g = oracle.eval_adjoint(("mul", ("leaf", "a"), ("leaf", "b")), f, f["w"])
    ca, cb, cw = cplx(f["a"]), cplx(f["b"]), cplx(f["w"])
    assert np.abs(cplx(g["a"]) - cw @ adj(cb)).max() < 1e-14
    assert np.abs(cplx(g["b"]) - adj(ca) @ cw).max() < 1e-14


def test_adjoint_closed_form_for_matrix_vector():
    dims = (2, 2, 2, 2)
    f = lattice_fields(dims, SEED, names=("a", "v"))
    v = synth.volume(dims)
    gz = synth.gauss_vector(SEED, 9, v)
    g = oracle.eval_adjoint(("mul", ("leaf", "a"), ("leaf", "v")), f, gz)
    ca, cv, cg = cplx(f["a"]), cplx(f["v"]), cplx(gz)
    assert np.abs(cplx(g["a"]) - np.einsum("ni,nj->nij", cg, np.conj(cv))).max() < 1e-14
    assert np.abs(cplx(g["v"]) - np.einsum("nji,nj->ni", np.conj(ca), cg)).max() < 1e-14


def test_adjoint_dot_product_identity():
    # Re<dZ, dA*B> = Re<dZ*B^dagger, dA> for a perturbation dA
    dims = (3, 2, 1, 5)
    f = lattice_fields(dims, SEED, names=("a", "b", "w"))
    v = synth.volume(dims)
    da = synth.gauss_matrix(SEED, 11, v)
    g = oracle.eval_adjoint(("mul", ("leaf", "a"), ("leaf", "b")), f, f["w"])
    lhs = oracle.redot(f["w"], oracle.mm(da, f["b"]))
    rhs = oracle.redot(g["a"], da)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


@pytest.mark.parametrize("tree", [("mul", ("leaf", "a"), ("leaf", "b")), E1, E2, E3,
                                  ("sub", ("scale", -1.5, ("adj", ("leaf", "b"))),
                                   ("mul", ("leaf", "a"), ("adj", ("leaf", "a"))))])
def test_adjoint_matches_central_differences(tree):
    dims = (2, 1, 1, 3)
    names = oracle.leaf_names(tree)
    f = lattice_fields(dims, SEED, names=tuple(names) + ("w",))
    leaves = {n: f[n] for n in names}
    g = oracle.eval_adjoint(tree, leaves, f["w"])

    def loss(lv):
        return oracle.redot(f["w"], oracle.eval_tree(tree, lv))

    rng = np.random.default_rng(5)
    h = 1e-3
    for name in names:
        flat = leaves[name].reshape(-1)
        for k in rng.choice(flat.size, 12, replace=False):
            up = {n: a.copy() for n, a in leaves.items()}
            dn = {n: a.copy() for n, a in leaves.items()}
            up[name].reshape(-1)[k] += h
            dn[name].reshape(-1)[k] -= h
            fd = (loss(up) - loss(dn)) / (2 * h)
            an = g[name].reshape(-1)[k]
            # the loss is at most quadratic in one component (a leaf may appear
            # twice), so the central difference is exact up to rounding
            assert abs(fd - an) <= 1e-9 * max(1.0, abs(an))


def test_adjoint_real_fields():
    v1 = np.array([1.0, -2.0, 0.5])
    v2 = np.array([3.0, 4.0, -1.0])
    tree = ("add", ("add", ("leaf", "v1"), ("leaf", "v2")), ("mul", ("leaf", "v1"), ("leaf", "v2")))
    g = oracle.eval_adjoint(tree, {"v1": v1, "v2": v2}, np.ones(3))
    assert np.array_equal(g["v1"], 1.0 + v2)
    assert np.array_equal(g["v2"], 1.0 + v1)


# ------------------------------------------------------------- reductions
def test_redot_matches_numpy():
    x = synth.gauss_matrix(SEED, 0, 100)
    y = synth.gauss_matrix(SEED, 1, 100)
    ref = np.real(np.sum(np.conj(cplx(x)) * cplx(y)))
    assert abs(oracle.redot(x, y) - ref) < 1e-12


# ------------------------------------------------------------- reunitarise
def test_reunitarize_projects_to_su3():
    n = 500
    g = synth.gauss_matrix(SEED, 3, n)
    u = cplx(oracle.reunitarize(g))
    assert np.abs(u @ adj(u) - np.eye(3)).max() < 1e-14
    assert np.abs(np.linalg.det(u) - 1.0).max() < 1e-14


def test_reunitarize_fixes_su3_and_matches_qr_rows():
    n = 200
    u = synth.su3(SEED, 0, n)
    assert np.abs(oracle.reunitarize(u) - u).max() < 1e-14
    # Gram-Schmidt over rows = QR of the transpose; compare up to the det phase
    g = synth.gauss_matrix(SEED, 4, n)
    r = cplx(oracle.reunitarize(g))
    q, rr = np.linalg.qr(np.swapaxes(cplx(g), 1, 2))
    ph = np.diagonal(rr, axis1=1, axis2=2) / np.abs(np.diagonal(rr, axis1=1, axis2=2))
    rows = np.swapaxes(q * ph[:, None, :], 1, 2)          # rows with positive R diagonal
    det = np.linalg.det(rows)
    rows = rows * np.exp(-1j * np.angle(det) / 3)[:, None, None]
    assert np.abs(r - rows).max() < 1e-13


# ------------------------------------------------------------- generator
def test_generator_is_counter_based_and_thread_independent():
    full = synth.su3(123, 0, 10000, nthreads=1)
    par = synth.su3(123, 0, 10000, nthreads=7)
    assert np.array_equal(full, par)
    assert np.array_equal(synth.su3(123, 0, 50, first=4321), full[4321:4371])
    assert not np.array_equal(synth.su3(123, 1, 50), full[:50])
    assert not np.array_equal(synth.su3(124, 0, 50), full[:50])


def test_generator_su3_properties():
    u = cplx(synth.su3(99, 2, 20000))
    assert np.abs(u @ adj(u) - np.eye(3)).max() < 1e-14
    assert np.abs(np.linalg.det(u) - 1.0).max() < 1e-14


def test_generator_gaussian_moments():
    g = synth.gauss_matrix(5, 5, 100000).reshape(-1)
    assert abs(g.mean()) < 0.01 and abs(g.std() - 1.0) < 0.01
    s = synth.uniform_real(5, 6, 100000)
    assert s.min() > -1.0 and s.max() < 1.0 and abs(s.mean()) < 0.01


# ------------------------------------------------ neighbours (Sec. 6)
STENCIL_DIMS = [(3, 2, 5, 4), (1, 3, 1, 2), (4, 4, 4, 4)]


def lattice_axis(dim):
    """Axis of a site-major array reshaped to (Lt, Lz, Ly, Lx, ...) for direction dim."""
    return 3 - dim


def as_grid(a, dims):
    return a.reshape(tuple(reversed(dims)) + a.shape[1:])


@pytest.mark.parametrize("dims", STENCIL_DIMS)
def test_cshift_matches_numpy_roll(dims):
    v = synth.volume(dims)
    links = synth.su3(SEED, 0, 4 * v).reshape(v, 4, 3, 3, 2)   # 4 links per site
    for dim in range(4):
        for shift in (-3, -1, 1, 2, 5):
            got = oracle.cshift(links, dims, dim, shift)
            # dst(x) = src(x + shift e_dim)  <=>  roll by -shift along that axis
            ref = np.roll(as_grid(links, dims), -shift, axis=lattice_axis(dim)).reshape(links.shape)
            assert np.array_equal(got, ref)


def test_cshift_inverse_and_period():
    dims = (3, 2, 5, 4)
    x = synth.gauss_vector(SEED, 4, synth.volume(dims))
    for dim in range(4):
        assert np.array_equal(oracle.cshift(oracle.cshift(x, dims, dim, 1), dims, dim, -1), x)
        assert np.array_equal(oracle.cshift(x, dims, dim, dims[dim]), x)
        y = x
        for _ in range(dims[dim]):
            y = oracle.cshift(y, dims, dim, 1)
        assert np.array_equal(y, x)


def hop_numpy(u, x, dims):
    """Independent restatement with numpy rolls and einsum."""
    v = synth.volume(dims)
    U = as_grid(cplx(u).reshape(v, 4, 3, 3), dims)
    X = as_grid(cplx(x), dims)
    out = np.zeros_like(X)
    mat = X.ndim == 6
    for mu in range(4):
        ax = lattice_axis(mu)
        Um = U[..., mu, :, :]
        fwd = np.roll(X, -1, axis=ax)                    # x(s + mu)
        bwd = np.roll(X, 1, axis=ax)                     # x(s - mu)
        Ub = np.conj(np.swapaxes(np.roll(Um, 1, axis=ax), -1, -2))   # U_mu(s - mu)^dagger
        if mat:
            out += np.einsum("...ij,...jk->...ik", Um, fwd) + np.einsum("...ij,...jk->...ik", Ub, bwd)
        else:
            out += np.einsum("...ij,...j->...i", Um, fwd) + np.einsum("...ij,...j->...i", Ub, bwd)
    return out.reshape((v,) + out.shape[4:])


@pytest.mark.parametrize("dims", STENCIL_DIMS)
@pytest.mark.parametrize("kind", ["vector", "matrix"])
def test_hop_matches_numpy(dims, kind):
    v = synth.volume(dims)
    u = synth.su3(SEED, 0, 4 * v)
    x = synth.gauss_vector(SEED, 4, v) if kind == "vector" else synth.gauss_matrix(SEED, 5, v)
    got = cplx(oracle.hop(u, x, dims))
    assert np.abs(got - hop_numpy(u, x, dims)).max() < 1e-13


def test_hop_unit_links_constant_field():
    dims = (3, 2, 5, 4)
    v = synth.volume(dims)
    u = np.zeros((4 * v, 3, 3, 2))
    u[:, [0, 1, 2], [0, 1, 2], 0] = 1.0
    # dyadic components with few bits: every partial sum is exact
    x = np.broadcast_to(np.round(16 * synth.gauss_vector(SEED, 4, 1)) / 16, (v, 3, 2)).copy()
    assert np.array_equal(oracle.hop(u, x, dims), 8.0 * x)


def test_hop_is_hermitian():
    dims = (3, 2, 5, 4)
    v = synth.volume(dims)
    u = synth.su3(SEED, 0, 4 * v)
    a, b = synth.gauss_vector(SEED, 4, v), synth.gauss_vector(SEED + 1, 4, v)
    lhs = np.vdot(cplx(a), cplx(oracle.hop(u, b, dims)))
    rhs = np.vdot(cplx(oracle.hop(u, a, dims)), cplx(b))
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)


def test_hop_gauge_covariance():
    """U'_mu(x) = g(x) U_mu(x) g(x+mu)^dagger, v'(x) = g(x) v(x) give hop'(x) = g(x) hop(x)."""
    dims = (3, 2, 5, 4)
    v = synth.volume(dims)
    u = synth.su3(SEED, 0, 4 * v)
    x = synth.gauss_matrix(SEED, 5, v)
    g = synth.su3(SEED + 9, 2, v)
    G, U = cplx(g), cplx(u).reshape(v, 4, 3, 3)
    Up = np.empty_like(U)
    for mu in range(4):
        gn = cplx(oracle.cshift(g, dims, mu, 1))          # g(x + mu)
        Up[:, mu] = G @ U[:, mu] @ np.conj(np.swapaxes(gn, -1, -2))
    xp = G @ cplx(x)
    up = np.stack([Up.real, Up.imag], -1).reshape(4 * v, 3, 3, 2)
    hp = oracle.hop(up, np.stack([xp.real, xp.imag], -1), dims)
    assert np.abs(cplx(hp) - G @ cplx(oracle.hop(u, x, dims))).max() < 1e-13


# ------------------------------------ Wilson hopping term with spin (Sec. 6)
def spinor(seed, field, v):
    """Gaussian spinor field: 4 spin components of a colour vector per site."""
    return synth.gauss_vector(seed, field, 4 * v).reshape(v, 4, 3, 2)


def test_gamma_matrices_form_the_euclidean_clifford_algebra():
    g = [oracle.gamma(mu) for mu in range(4)]
    g5 = oracle.gamma(4)
    eye = np.eye(4)
    for a in range(4):
        assert np.array_equal(g[a], np.conj(g[a].T))             # hermitian
        for b in range(4):
            assert np.array_equal(g[a] @ g[b] + g[b] @ g[a], 2.0 * eye * (a == b))
        assert np.array_equal(g[a] @ g5 + g5 @ g[a], np.zeros((4, 4)))
    assert np.array_equal(g[0] @ g[1] @ g[2] @ g[3], g5)
    assert np.array_equal(g5, np.diag([1, 1, -1, -1]))           # chiral basis
    for a in range(4):                                           # (1 -+ g)/2: rank-2 projectors
        for sg in (1, -1):
            p = 0.5 * (eye + sg * g[a])
            assert np.array_equal(p @ p, p) and np.linalg.matrix_rank(p) == 2


@pytest.mark.parametrize("dims", STENCIL_DIMS)
def test_dslash_projector_sum_is_twice_the_colour_hopping_term(dims):
    # (1 - g) + (1 + g) = 2: the operator plus its projector-swapped form is
    # twice the colour hopping term, applied to each spin component
    v = synth.volume(dims)
    u = synth.su3(SEED, 0, 4 * v)
    psi = spinor(SEED, 4, v)
    both = oracle.dslash(u, psi, dims, 1) + oracle.dslash(u, psi, dims, -1)
    hop = np.stack([oracle.hop(u, np.ascontiguousarray(psi[:, s]), dims) for s in range(4)], 1)
    assert np.abs(both - 2.0 * hop).max() < 1e-13


def test_dslash_is_gamma5_hermitian():
    # <a, D b> = <g5 D g5 a, b>: the hopping term's adjoint is g5 D g5
    dims = (3, 2, 5, 4)
    v = synth.volume(dims)
    u = synth.su3(SEED, 0, 4 * v)
    a, b = spinor(SEED, 4, v), spinor(SEED + 1, 4, v)
    g5 = np.array([1.0, 1.0, -1.0, -1.0])[None, :, None, None]
    lhs = np.vdot(cplx(a), cplx(oracle.dslash(u, b, dims)))
    rhs = np.vdot(cplx(g5 * oracle.dslash(u, g5 * a, dims)), cplx(b))
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)
    # and it is not hermitian itself (the projectors do not commute with g5)
    rhs_h = np.vdot(cplx(oracle.dslash(u, a, dims)), cplx(b))
    assert abs(lhs - rhs_h) > 1e-3 * abs(lhs)


def test_dslash_gauge_covariance():
    dims = (3, 2, 5, 4)
    v = synth.volume(dims)
    u = synth.su3(SEED, 0, 4 * v)
    psi = spinor(SEED, 4, v)
    g = synth.su3(SEED + 9, 2, v)
    G, U = cplx(g), cplx(u).reshape(v, 4, 3, 3)
    Up = np.empty_like(U)
    for mu in range(4):
        gn = cplx(oracle.cshift(g, dims, mu, 1))
        Up[:, mu] = G @ U[:, mu] @ np.conj(np.swapaxes(gn, -1, -2))
    up = np.stack([Up.real, Up.imag], -1).reshape(4 * v, 3, 3, 2)
    pp = np.einsum("nij,nsj->nsi", G, cplx(psi))
    out_p = oracle.dslash(up, np.stack([pp.real, pp.imag], -1), dims)
    ref = np.einsum("nij,nsj->nsi", G, cplx(oracle.dslash(u, psi, dims)))
    assert np.abs(cplx(out_p) - ref).max() < 1e-13


@pytest.mark.parametrize("dims", [(4, 3, 2, 5), (2, 2, 2, 2)])
def test_dslash_free_field_plane_wave(dims):
    # unit links, psi(x) = exp(i p.x) u: D psi = sum_mu [(1 - g_mu) e^{i p_mu}
    # + (1 + g_mu) e^{-i p_mu}] psi, a 4x4 matrix in spin space only
    v = synth.volume(dims)
    links = np.zeros((4 * v, 3, 3, 2))
    links[:, [0, 1, 2], [0, 1, 2], 0] = 1.0
    n = np.array([1, 2, 1, 3])
    p = 2 * np.pi * n / np.array(dims)
    x = np.stack(np.meshgrid(*[np.arange(L) for L in dims], indexing="ij"), -1)
    x = x.transpose(3, 2, 1, 0, 4).reshape(v, 4)                # site order x fastest
    phase = np.exp(1j * (x @ p))
    rng = np.random.default_rng(7)
    u0 = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
    psi = phase[:, None, None] * u0[None]
    eye = np.eye(4)
    m = sum((eye - oracle.gamma(mu)) * np.exp(1j * p[mu]) + (eye + oracle.gamma(mu)) * np.exp(-1j * p[mu])
            for mu in range(4))
    ref = phase[:, None, None] * (m @ u0)[None]
    got = cplx(oracle.dslash(links, np.stack([psi.real, psi.imag], -1), dims))
    assert np.abs(got - ref).max() < 1e-13
