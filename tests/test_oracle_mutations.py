"""The oracle pins catch plausible mistakes.

Each case plants one mistake (a flipped sign, a transposed operand, a dropped
term, a missing conjugation, a wrong rounding) in a copy of the oracle's C
source, builds it on the CPU, and checks that at least one pin from
test_oracle.py fails against the mutated oracle while it passes against the
original.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle
import synth
from helpers import cplx, lattice_fields

SEED = synth.SEED_BASE
SRC = os.path.join(os.path.dirname(oracle.__file__), "su3_oracle.c")


def adj(c):
    return np.conj(np.swapaxes(c, -1, -2))


def pin_mm_brute_force():
    f = lattice_fields((3, 2, 1, 5), SEED)
    return np.abs(cplx(oracle.mm(f["a"], f["b"])) - cplx(f["a"]) @ cplx(f["b"])).max() < 1e-14


def pin_mv_brute_force():
    f = lattice_fields((3, 2, 1, 5), SEED, names=("a", "v"))
    ref = np.einsum("nij,nj->ni", cplx(f["a"]), cplx(f["v"]))
    return np.abs(cplx(oracle.mv(f["a"], f["v"])) - ref).max() < 1e-14


def pin_inverse():
    f = lattice_fields((2, 2, 2, 2), SEED)
    z = oracle.eval_tree(("mul", ("leaf", "a"), ("adj", ("leaf", "a"))), f)
    return np.abs(cplx(z) - np.eye(3)).max() < 1e-14


def pin_c12():
    u = synth.su3(SEED, 0, 100)
    return np.abs(oracle.c12_expand(u[:, :2].copy()) - u).max() < 1e-15


def pin_grad_closed_form():
    f = lattice_fields((2, 2, 2, 2), SEED, names=("a", "b", "w"))
    g = oracle.eval_adjoint(("mul", ("leaf", "a"), ("leaf", "b")), f, f["w"])
    ok_a = np.abs(cplx(g["a"]) - cplx(f["w"]) @ adj(cplx(f["b"]))).max() < 1e-14
    ok_b = np.abs(cplx(g["b"]) - adj(cplx(f["a"])) @ cplx(f["w"])).max() < 1e-14
    return ok_a and ok_b


def pin_round():
    x = np.random.default_rng(1).standard_normal(10000)
    return (np.array_equal(oracle.round_to(x, "f32"), x.astype(np.float32).astype(np.float64))
            and np.array_equal(oracle.round_to(x, "f16"), x.astype(np.float16).astype(np.float64)))


def pin_round_bf16_ties():
    x = np.array([1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8])
    return np.array_equal(oracle.round_to(x, "bf16"), np.array([1.0, 1.0 + 2 * 2.0 ** -7]))


def pin_reunitarize_det():
    u = cplx(oracle.reunitarize(synth.gauss_matrix(SEED, 3, 200)))
    return (np.abs(u @ adj(u) - np.eye(3)).max() < 1e-14
            and np.abs(np.linalg.det(u) - 1).max() < 1e-14)


def pin_cshift_roll():
    dims = (3, 2, 5, 4)
    x = synth.gauss_vector(SEED, 4, synth.volume(dims))
    g = x.reshape(4, 5, 2, 3, 3, 2)
    return all(np.array_equal(oracle.cshift(x, dims, d, 1),
                              np.roll(g, -1, axis=3 - d).reshape(x.shape)) for d in range(4))


def pin_hop_hermitian():
    dims = (3, 2, 5, 4)
    v = synth.volume(dims)
    u = synth.su3(SEED, 0, 4 * v)
    a, b = synth.gauss_vector(SEED, 4, v), synth.gauss_vector(SEED + 1, 4, v)
    lhs = np.vdot(cplx(a), cplx(oracle.hop(u, b, dims)))
    rhs = np.vdot(cplx(oracle.hop(u, a, dims)), cplx(b))
    return abs(lhs - rhs) <= 1e-13 * abs(lhs)


def pin_dslash_gamma5_hermitian():
    dims = (3, 2, 5, 4)
    v = synth.volume(dims)
    u = synth.su3(SEED, 0, 4 * v)
    a = synth.gauss_vector(SEED, 4, 4 * v).reshape(v, 4, 3, 2)
    b = synth.gauss_vector(SEED + 1, 4, 4 * v).reshape(v, 4, 3, 2)
    g5 = np.array([1.0, 1.0, -1.0, -1.0])[None, :, None, None]
    lhs = np.vdot(cplx(a), cplx(oracle.dslash(u, b, dims)))
    rhs = np.vdot(cplx(g5 * oracle.dslash(u, g5 * a, dims)), cplx(b))
    return abs(lhs - rhs) <= 1e-13 * abs(lhs)


def pin_dslash_projector_sum():
    dims = (3, 2, 5, 4)
    v = synth.volume(dims)
    u = synth.su3(SEED, 0, 4 * v)
    psi = synth.gauss_vector(SEED, 4, 4 * v).reshape(v, 4, 3, 2)
    both = oracle.dslash(u, psi, dims, 1) + oracle.dslash(u, psi, dims, -1)
    hop = np.stack([oracle.hop(u, np.ascontiguousarray(psi[:, s]), dims) for s in range(4)], 1)
    return np.abs(both - 2.0 * hop).max() < 1e-13


def pin_dslash_plane_wave():
    dims = (4, 3, 2, 5)
    v = synth.volume(dims)
    links = np.zeros((4 * v, 3, 3, 2))
    links[:, [0, 1, 2], [0, 1, 2], 0] = 1.0
    p = 2 * np.pi * np.array([1, 2, 1, 3]) / np.array(dims)
    x = np.stack(np.meshgrid(*[np.arange(L) for L in dims], indexing="ij"), -1)
    x = x.transpose(3, 2, 1, 0, 4).reshape(v, 4)
    phase = np.exp(1j * (x @ p))
    u0 = np.arange(12).reshape(4, 3) + 0.5j
    psi = phase[:, None, None] * u0[None]
    # the closed form with the gamma matrices written out here (chiral basis)
    i = 1j
    g = [np.array([[0, 0, 0, i], [0, 0, i, 0], [0, -i, 0, 0], [-i, 0, 0, 0]]),
         np.array([[0, 0, 0, -1], [0, 0, 1, 0], [0, 1, 0, 0], [-1, 0, 0, 0]]),
         np.array([[0, 0, i, 0], [0, 0, 0, -i], [-i, 0, 0, 0], [0, i, 0, 0]]),
         np.array([[0, 0, 1, 0], [0, 0, 0, 1], [1, 0, 0, 0], [0, 1, 0, 0]])]
    m = sum((np.eye(4) - g[mu]) * np.exp(1j * p[mu]) + (np.eye(4) + g[mu]) * np.exp(-1j * p[mu])
            for mu in range(4))
    ref = phase[:, None, None] * (m @ u0)[None]
    got = cplx(oracle.dslash(links, np.stack([psi.real, psi.imag], -1), dims))
    return np.abs(got - ref).max() < 1e-12


MUTATIONS = [
    ("mm sign", "re -= xi * yi;", "re += xi * yi;", pin_mm_brute_force),
    ("mm transposed operand", "double yr = y[2 * (3 * j + k)], yi = y[2 * (3 * j + k) + 1];",
     "double yr = y[2 * (3 * k + j)], yi = y[2 * (3 * k + j) + 1];", pin_mm_brute_force),
    ("mm dropped term", "                im += xi * yr;\n", "\n", pin_mm_brute_force),
    ("mv wrong index", "double vr = v[2 * j], vi = v[2 * j + 1];",
     "double vr = v[2 * i], vi = v[2 * i + 1];", pin_mv_brute_force),
    ("adj without conjugation", "z[2 * (3 * i + j) + 1] = -x[2 * (3 * j + i) + 1];",
     "z[2 * (3 * i + j) + 1] = x[2 * (3 * j + i) + 1];", pin_inverse),
    ("c12 without conjugation", "f[12 + 2 * c + 1] = -im;", "f[12 + 2 * c + 1] = im;", pin_c12),
    ("c12 swapped cross product", "int j = (c + 1) % 3, k = (c + 2) % 3;",
     "int j = (c + 2) % 3, k = (c + 1) % 3;", pin_c12),
    ("grad missing dagger", "mat_adj(y->v, u);\n                    mat_mul(G, u, t);",
     "memcpy(u, y->v, sizeof u);\n                    mat_mul(G, u, t);", pin_grad_closed_form),
    ("grad operand order", "mat_adj(x->v, u);\n                    mat_mul(u, G, t);\n                    for (int r = 0; r < 18; ++r) gy[r] += t[r];",
     "mat_adj(x->v, u);\n                    mat_mul(G, u, t);\n                    for (int r = 0; r < 18; ++r) gy[r] += t[r];", pin_grad_closed_form),
    ("rounding truncates", "double q = rint(ldexp(x, -k));", "double q = trunc(ldexp(x, -k));", pin_round),
    ("rounding ties away", "double q = rint(ldexp(x, -k));", "double q = round(ldexp(x, -k));",
     pin_round_bf16_ties),
    ("reunitarize keeps det phase", "double phi = atan2(di, dr);", "double phi = 0.0 * atan2(di, dr);",
     pin_reunitarize_det),
    ("cshift wrong direction", "int64_t m = ((c[dim] + shift) % L[dim] + L[dim]) % L[dim];",
     "int64_t m = ((c[dim] - shift) % L[dim] + L[dim]) % L[dim];", pin_cshift_roll),
    ("hop backward link not daggered", "mat_adj(U + 18 * (4 * bw + mu), a);\n            if (kind",
     "memcpy(a, U + 18 * (4 * bw + mu), sizeof a);\n            if (kind", pin_hop_hermitian),
    ("hop backward link at the site", "mat_adj(U + 18 * (4 * bw + mu), a);\n            if (kind",
     "mat_adj(U + 18 * (4 * s + mu), a);\n            if (kind", pin_hop_hermitian),
    ("dslash projectors swapped", "spin_project_add(o, (const double(*)[6])chi, mu, -(double)r);",
     "spin_project_add(o, (const double(*)[6])chi, mu, (double)r);", pin_dslash_gamma5_hermitian),
    ("dslash gamma_y entry sign", "{{0, 0}, {0, 0}, {0, 0}, {-1, 0}},",
     "{{0, 0}, {0, 0}, {0, 0}, {1, 0}},", pin_dslash_plane_wave),
    ("dslash imaginary part of the projector dropped", "                o[6 * a + 2 * c] -= pi * xi;\n",
     "\n", pin_dslash_plane_wave),
    ("dslash backward link not daggered", "mat_adj(U + 18 * (4 * bw + mu), a);\n            for (int sp",
     "memcpy(a, U + 18 * (4 * bw + mu), sizeof a);\n            for (int sp", pin_dslash_projector_sum),
]


@pytest.mark.parametrize("name,old,new,pin", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pin_catches_planted_mistake(name, old, new, pin, tmp_path, monkeypatch):
    src = open(SRC).read()
    assert src.count(old) == 1, "mutation anchor must occur exactly once"
    assert pin(), "pin must pass on the unmodified oracle"
    mut_c = tmp_path / "mut.c"
    mut_c.write_text(src.replace(old, new))
    so = tmp_path / "mut.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                           "-o", str(so), str(mut_c), "-lm"])
    monkeypatch.setattr(oracle, "_lib", oracle._bind(ctypes.CDLL(str(so))))
    assert not pin(), "planted mistake %r went unnoticed" % name
