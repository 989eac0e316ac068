"""Parity of the benchmark's own step at its full size (48^4 lattice, 5,308,416
sites), in the launch configuration the benchmark times: the rows are built by
bench.build_rows from the same seeded inputs, tuned by the library's autotuner
as the benchmark does, run once, and every row's outputs are checked against
the oracle on sampled sites (plus the first and last sites).  The batch row is
checked on sampled sites of each of its 64 lattices.

Tolerances as in test_gpu_parity: FP64 storage 1e-13 per real component (2e-13
for the fused trees, scaled by the operands' size for Gaussian ones); reduced
precision one unit in the last place of the output format plus 8*2^-24 against
the oracle that rounds inputs and output; two-row FP32 3e-6.
"""
import numpy as np
import pytest
import torch

import bench
import oracle
import synth
from helpers import E1, E2, E3, ULP, cplx

pytestmark = pytest.mark.gpu

TOL = 1e-13
MM = ("mul", ("leaf", "a"), ("leaf", "b"))
TREES = {"A5 z=a*b+c*d": E1, "A5 z=a*b*c+0.5*d": E2, "A5 z=adj(a)*b-b*adj(a)": E3}


def host_rows(t, shape, idx):
    """Rows `idx` of a flat canonical host array viewed as objects of `shape`."""
    return t.view((-1,) + shape)[torch.from_numpy(idx)].numpy()


def dev_rows(f, idx):
    """Rows `idx` of the field's canonical (FP64, row 2 rebuilt) contents."""
    return f.unpack()[torch.from_numpy(idx).cuda()].cpu().numpy()


def check_row(r, idx):
    name = r.name
    ins = [(f, h) for f, h in r.inputs]
    outs = [f for f, _ in r.outputs]
    if name in ("A2 z=a*b", "A4 z_mu=a_mu*b_mu"):
        nmu = outs[0].nmu
        ii = (idx[:, None] * nmu + np.arange(nmu)[None, :]).reshape(-1)
        A, B = (host_rows(h, (3, 3, 2), ii) for _, h in ins)
        assert np.abs(dev_rows(outs[0], ii) - oracle.mm(A, B)).max() < TOL
    elif name == "A3 z=a*v":
        A, X = host_rows(ins[0][1], (3, 3, 2), idx), host_rows(ins[1][1], (3, 2), idx)
        scale = max(1.0, np.abs(cplx(X)).sum(axis=1).max())
        assert np.abs(dev_rows(outs[0], idx) - oracle.mv(A, X)).max() < TOL * scale
    elif name in TREES:
        leaves = {n: host_rows(h, (3, 3, 2), idx) for n, (_, h) in zip("abcd", ins)}
        ref = oracle.eval_tree(TREES[name], leaves)
        assert np.abs(dev_rows(outs[0], idx) - ref).max() < 2 * TOL
    elif name.startswith("A6"):
        fmt = name.split()[-1]
        A, B = (host_rows(h, (3, 3, 2), idx) for _, h in ins)
        ref = oracle.round_to(oracle.mm(oracle.round_to(A, fmt), oracle.round_to(B, fmt)), fmt)
        assert (np.abs(dev_rows(outs[0], idx) - ref) <= ULP[fmt](ref) + 8 * 2.0 ** -24).all()
    elif name == "A7 z=a*b f64_c12":
        A, B = (host_rows(h, (3, 3, 2), idx) for _, h in ins)
        ref = oracle.mm(oracle.c12_expand(A[:, :2].copy()), oracle.c12_expand(B[:, :2].copy()))
        got = dev_rows(outs[0], idx)
        assert np.abs(got[:, :2] - ref[:, :2]).max() < TOL
        assert np.abs(got - oracle.c12_expand(ref[:, :2].copy())).max() < TOL
    elif name == "A7 z=a*b f32_c12":
        A, B = (host_rows(h, (3, 3, 2), idx) for _, h in ins)
        ra, rb = (oracle.round_to(x[:, :2].copy(), "f32") for x in (A, B))
        ref = oracle.mm(oracle.c12_expand(ra), oracle.c12_expand(rb))
        assert np.abs(dev_rows(outs[0], idx)[:, :2] - ref[:, :2]).max() < 3e-6
    elif name.startswith("A8"):
        rng = np.random.default_rng(12)
        assert len(outs) == 64 and len(ins) == 4 * 64
        for i, z in enumerate(outs):
            nv = z.lattice.volume
            ii = np.unique(np.concatenate([rng.choice(nv, min(nv, 64), replace=False), [nv - 1]]))
            leaves = {n: host_rows(h, (3, 3, 2), ii) for n, (_, h) in zip("abcd", ins[4 * i:4 * i + 4])}
            ref = oracle.eval_tree(E1, leaves)
            assert np.abs(dev_rows(z, ii) - ref).max() < 2 * TOL, i
    elif name.startswith("A9"):
        tree = MM if name == "A9 adjoint of z=a*b" else E1
        names = "ab" if tree is MM else "abcd"
        leaves = {n: host_rows(h, (3, 3, 2), idx) for n, (_, h) in zip(names, ins)}
        W = host_rows(ins[len(names)][1], (3, 3, 2), idx)
        ref = oracle.eval_adjoint(tree, leaves, W)
        wscale = np.abs(W).max() * 3
        for n, g in zip(names, outs):
            assert np.abs(dev_rows(g, idx) - ref[n]).max() < TOL * wscale, n
    else:
        raise AssertionError("no oracle check for row %r" % name)


def test_every_bench_row_at_full_size_matches_oracle(gpu_lib):
    su3s = gpu_lib
    rows, keep = bench.build_rows(su3s, synth, torch, True)
    assert [r.name for r in rows] == bench.ROW_NAMES
    stream = torch.cuda.Stream()
    for r in rows:
        if r.tune is not None:
            r.tune(stream)
    for r in rows:
        r.run(stream)
    stream.synchronize()
    assert su3s.device_error() == 0
    v = synth.volume(bench.DIMS)
    rng = np.random.default_rng(11)
    idx = np.unique(np.concatenate([rng.choice(v, 1500, replace=False), [0, 1, v - 1]]))
    for r in rows:
        check_row(r, idx)
