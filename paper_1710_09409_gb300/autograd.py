"""torch.autograd bridge: differentiable evaluation of lattice expressions.

Forward runs the fused evaluation kernel; backward runs the hand-written
reverse-mode kernel (for z = a*b: dA = G B^dagger, dB = A^dagger G; sums,
real factors and adjoints by the chain rule), both through the C ABI.  Tensors
are FP64 fields in a device layout (flat float64 CUDA tensors of the field's
size); the gradient convention is the one PyTorch uses for real tensors, i.e.
dL/dRe and dL/dIm per stored real, which for complex entries is
dL/dRe + i dL/dIm.
"""
import torch

from . import F64, MATH_DEFAULT, MATRIX, SOA, Field, eval_adjoint, evaluate


def _leaf_order(tree, acc=None):
    acc = [] if acc is None else acc
    op = tree[0]
    if op == "leaf":
        if tree[1] not in acc:
            acc.append(tree[1])
    elif op == "scale":
        _leaf_order(tree[2], acc)
    else:
        for sub in tree[1:]:
            _leaf_order(sub, acc)
    return acc


def _build(tree, fields):
    op = tree[0]
    if op == "leaf":
        return fields[tree[1]].expr()
    if op == "mul":
        return _build(tree[1], fields) * _build(tree[2], fields)
    if op == "add":
        return _build(tree[1], fields) + _build(tree[2], fields)
    if op == "sub":
        return _build(tree[1], fields) - _build(tree[2], fields)
    if op == "scale":
        return float(tree[1]) * _build(tree[2], fields)
    if op == "adj":
        return _build(tree[1], fields).adj()
    raise ValueError(op)


def _result_kind(tree, kinds):
    op = tree[0]
    if op == "leaf":
        return kinds[tree[1]]
    if op == "mul":
        return _result_kind(tree[2], kinds)
    if op in ("add", "sub"):
        return _result_kind(tree[1], kinds)
    if op == "scale":
        return _result_kind(tree[2], kinds)
    return MATRIX


class LatticeFunction(torch.autograd.Function):
    """apply(spec, *tensors); spec = (tree, lattice, kinds, nmu, layout, block, math)."""

    @staticmethod
    def forward(ctx, spec, *tensors):
        tree, lattice, kinds, nmu, layout, block, math = spec
        fields = [Field(lattice, kinds[i], nmu, F64, layout, block, tensor=t.detach())
                  for i, t in enumerate(tensors)]
        out_kind = _result_kind(tree, kinds)
        dest = Field(lattice, out_kind, nmu, F64, layout, block)
        evaluate(dest, _build(tree, fields), math)
        ctx.spec = spec
        ctx.out_kind = out_kind
        ctx.save_for_backward(*tensors)
        return dest.tensor

    @staticmethod
    def backward(ctx, grad):
        tree, lattice, kinds, nmu, layout, block, math = ctx.spec
        tensors = ctx.saved_tensors
        fields = [Field(lattice, kinds[i], nmu, F64, layout, block, tensor=t.detach())
                  for i, t in enumerate(tensors)]
        g = Field(lattice, ctx.out_kind, nmu, F64, layout, block,
                  tensor=grad.detach().contiguous())
        order = _leaf_order(tree)
        grads = [None] * len(tensors)
        gfields = []
        for i in order:
            if ctx.needs_input_grad[1 + i]:
                grads[i] = Field(lattice, kinds[i], nmu, F64, layout, block)
                gfields.append(grads[i])
            else:
                gfields.append(None)
        eval_adjoint(_build(tree, fields), g, gfields, math)
        return (None,) + tuple(f.tensor if f is not None else None for f in grads)


def lattice_expr(tree, lattice, tensors, kinds=None, nmu=1, layout=SOA, block=64,
                 math=MATH_DEFAULT):
    """Differentiable dest = tree(tensors) for FP64 fields in a device layout.

    `tree` is a nested tuple ("leaf", i) | ("mul", x, y) | ("add", x, y) |
    ("sub", x, y) | ("scale", s, x) | ("adj", x) with leaf i = tensors[i]."""
    kinds = tuple(kinds) if kinds is not None else (MATRIX,) * len(tensors)
    spec = (tree, lattice, kinds, nmu, layout, block, math)
    return LatticeFunction.apply(spec, *tensors)
