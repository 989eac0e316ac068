"""The stated errors: every output of the configurations' lattices against the
FP64 oracle, for each arithmetic of FP64 storage and each storage format.

  * storage formats, z = a*b on 32^4 and 16^3x32 SU(3) lattices: the maximum
    absolute error against the exact FP64 product, within the a priori bound of
    the format (FP32 2e-6, BF16 2.5e-2, FP16 3e-3; two-row FP64 1e-13, two-row
    FP32 5e-6);
  * FP64 storage, the fused trees on 32^4 and z = a*b on 48^4: the maximum
    absolute error of native FP64, the pair-of-FP32 and the fixed-point
    arithmetic, within 1e-13, with each arithmetic's own bound (native FP64 and
    fixed point 5e-15, pair arithmetic 1e-13).

Each case prints one JSON line (pytest -s shows them).
"""
import json

import numpy as np
import pytest

import oracle
import synth
from helpers import E1, E2, E3

pytestmark = pytest.mark.gpu

SEED = synth.SEED_BASE + 2
MM = ("mul", ("leaf", "a"), ("leaf", "b"))
STORAGE = [("f64", "F64", 1e-13), ("f32", "F32", 2e-6), ("bf16", "BF16", 2.5e-2),
           ("f16", "F16", 3e-3), ("f64_c12", "F64_C12", 1e-13), ("f32_c12", "F32_C12", 5e-6)]
MATHS = [("f64", 1, 5e-15), ("df32", 2, 1e-13), ("fx", 3, 5e-15)]


@pytest.fixture(scope="module")
def su3s(gpu_lib):
    return gpu_lib


def upload(su3s, lat, arr, prec):
    f = su3s.Field(lat, su3s.MATRIX, 1, prec, su3s.SOA)
    f.upload(arr)
    return f


@pytest.mark.parametrize("dims", [(32, 32, 32, 32), (16, 16, 16, 32)], ids=str)
def test_storage_format_errors(su3s, dims):
    v = synth.volume(dims)
    lat = su3s.Lattice(dims)
    ha, hb = synth.su3(SEED, 0, v), synth.su3(SEED, 1, v)
    exact = oracle.mm(ha, hb)
    for name, prec, bound in STORAGE:
        a, b = upload(su3s, lat, ha, getattr(su3s, prec)), upload(su3s, lat, hb, getattr(su3s, prec))
        z = a.like()
        su3s.evaluate(z, a * b)
        err = float(np.abs(z.download() - exact).max())
        print(json.dumps({"study": "storage error", "lattice": list(dims), "storage": name,
                          "outputs": int(exact.size), "max_abs_err_vs_fp64_oracle": err}))
        assert err <= bound, (name, err)


@pytest.mark.parametrize("dims,trees", [((32, 32, 32, 32), ("a*b", "E1", "E2", "E3")),
                                        ((48, 48, 48, 48), ("a*b",))], ids=["32^4", "48^4"])
def test_fp64_arithmetic_errors(su3s, dims, trees):
    v = synth.volume(dims)
    lat = su3s.Lattice(dims)
    host = {n: synth.su3(SEED + 3, i, v) for i, n in enumerate("abcd")}
    F = {n: upload(su3s, lat, host[n], su3s.F64) for n in "abcd"}
    a, b, c, d = (F[n] for n in "abcd")
    cases = {"a*b": (MM, a * b), "E1": (E1, a * b + c * d), "E2": (E2, a * b * c + 0.5 * d),
             "E3": (E3, a.adj() * b - b * a.adj())}
    z = a.like()
    for name in trees:
        tree, expr = cases[name]
        ref = oracle.eval_tree(tree, host)
        line = {"study": "fp64 error vs oracle", "lattice": list(dims), "tree": name,
                "outputs": int(ref.size)}
        for mname, math, bound in MATHS:
            su3s.evaluate(z, expr, math)
            err = float(np.abs(z.download() - ref).max())
            line["max_abs_err_" + mname] = err
            assert err <= bound, (name, mname, err)
        print(json.dumps(line))


def _rows(t, shape):
    return t.reshape((-1,) + shape).numpy()


def test_bench_step_errors_at_48(gpu_lib):
    """Every output of every FP64-storage row of the benchmark step at its size
    (48^4, 5,308,416 sites; the 64 batch lattices in full), tuned and run as
    the benchmark runs them, against the oracle: the maximum absolute error per
    row in the default (pair) arithmetic, within 1e-13 (Gaussian operands: the
    bound scaled by their size, as in the parity tests)."""
    import torch

    import bench
    from helpers import cplx
    su3s = gpu_lib
    want = lambda n: n.startswith(("A2", "A3", "A4", "A5", "A7 z=a*b f64", "A8", "A9"))
    rows, keep = bench.build_rows(su3s, synth, torch, True, want=want)
    stream = torch.cuda.Stream()
    for r in rows:
        if r.tune is not None:
            r.tune(stream)
    for r in rows:
        r.run(stream)
    stream.synchronize()
    assert su3s.device_error() == 0
    trees = {"A5 z=a*b+c*d": E1, "A5 z=a*b*c+0.5*d": E2, "A5 z=adj(a)*b-b*adj(a)": E3}
    line = {"study": "fp64 error vs oracle, benchmark step", "lattice": [48, 48, 48, 48],
            "arithmetic": "df32"}
    for r in rows:
        ins = [h for _, h in r.inputs]
        outs = [f for f, _ in r.outputs]
        name = r.name
        if name in ("A2 z=a*b", "A4 z_mu=a_mu*b_mu"):
            err, n = np.abs(outs[0].download() - oracle.mm(_rows(ins[0], (3, 3, 2)),
                                                            _rows(ins[1], (3, 3, 2)))).max(), 1.0
        elif name == "A3 z=a*v":
            X = _rows(ins[1], (3, 2))
            n = max(1.0, np.abs(cplx(X)).sum(axis=1).max())
            err = np.abs(outs[0].download() - oracle.mv(_rows(ins[0], (3, 3, 2)), X)).max()
        elif name in trees:
            leaves = {k: _rows(h, (3, 3, 2)) for k, h in zip("abcd", ins)}
            err, n = np.abs(outs[0].download() - oracle.eval_tree(trees[name], leaves)).max(), 1.0
        elif name == "A7 z=a*b f64_c12":
            A, B = (_rows(h, (3, 3, 2)) for h in ins)
            ref = oracle.mm(oracle.c12_expand(A[:, :2].copy()), oracle.c12_expand(B[:, :2].copy()))
            got = outs[0].download()
            err, n = max(np.abs(got[:, :2] - ref[:, :2]).max(),
                         np.abs(got - oracle.c12_expand(ref[:, :2].copy())).max()), 1.0
        elif name.startswith("A8"):
            err, n = 0.0, 1.0
            for i, z in enumerate(outs):
                leaves = {k: _rows(h, (3, 3, 2)) for k, h in zip("abcd", ins[4 * i:4 * i + 4])}
                err = max(err, np.abs(z.download() - oracle.eval_tree(E1, leaves)).max())
        elif name.startswith("A9"):
            tree = MM if name == "A9 adjoint of z=a*b" else E1
            names = "ab" if tree is MM else "abcd"
            leaves = {k: _rows(h, (3, 3, 2)) for k, h in zip(names, ins)}
            W = _rows(ins[len(names)], (3, 3, 2))
            ref = oracle.eval_adjoint(tree, leaves, W)
            n = np.abs(W).max() * 3
            err = max(np.abs(g.download() - ref[k]).max() for k, g in zip(names, outs))
        else:
            continue
        line[name] = {"max_abs_err": float(err), "bound": 1e-13 * n}
        assert err <= 1e-13 * n, (name, err)
    print(json.dumps(line))
