"""Python binding of su3s, the GB300 library for site-local lattice expressions.

Argument marshalling only: every step of the computation runs in the CUDA
kernels of ``lib/libsu3s.so`` (built from ``csrc/`` by ``build.py``), reached
through its C ABI (``include/su3s.h``) with ctypes.  PyTorch provides device
memory (fields wrap torch tensors) and streams.  There is no CPU fallback:
if the library cannot be loaded, every call raises.

Objects follow arXiv:1710.09409: a ``Lattice`` is the grid (Sec. 3, Listing
2), a ``Field`` a lattice-wide array of site objects (colour matrices, colour
vectors or reals, optionally ``nmu`` per site), an ``Expr`` a tree of
products, sums, differences, real factors and adjoints (the expression
template of Sec. 3, Listing 1), and ``evaluate(dest, expr)`` computes
dest[x] = expr[x] for every site x in one pass (Sec. 4, Listing 3: z = x*y).
"""
import ctypes
import numbers
import os

import numpy as np

from . import build as _build

MATRIX, VECTOR, REAL = 0, 1, 2
F64, F32, BF16, F16, F64_C12, F32_C12 = 0, 1, 2, 3, 4, 5
SOA, AOSOA = 0, 1
MATH_DEFAULT, MATH_F64, MATH_DF32, MATH_FX = 0, 1, 2, 3
WIDTH = {MATRIX: 18, VECTOR: 6, REAL: 1}
PREC_NAMES = {F64: "f64", F32: "f32", BF16: "bf16", F16: "f16", F64_C12: "f64_c12",
              F32_C12: "f32_c12"}

_lib = None


class Su3sError(RuntimeError):
    """A call into the library returned a non-zero status."""

    def __init__(self, code, msg):
        super().__init__("su3s error %d: %s" % (code, msg))
        self.code = code


def lib_path():
    return _build.LIB


def load(build_if_missing=False):
    """Load the CUDA library (raises if it is not built and cannot be)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError("su3s CUDA library %s is not built; run __graft_entry__.build()"
                           % _build.LIB)
    L = ctypes.CDLL(_build.LIB)
    P, I, D, SZ, I64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t, ctypes.c_int64
    PP = ctypes.POINTER(ctypes.c_void_p)
    sigs = {
        "su3s_last_error": ([], ctypes.c_char_p),
        "su3s_version": ([], I),
        "su3s_lattice_create": ([I, I, I, I, PP], I),
        "su3s_lattice_destroy": ([P], I),
        "su3s_lattice_volume": ([P, ctypes.POINTER(I64)], I),
        "su3s_field_bytes": ([P, I, I, I, I, I, ctypes.POINTER(SZ)], I),
        "su3s_field_wrap": ([P, I, I, I, I, I, P, SZ, PP], I),
        "su3s_field_destroy": ([P], I),
        "su3s_field_pack": ([P, P, P], I),
        "su3s_field_unpack": ([P, P, P], I),
        "su3s_field_upload": ([P, P, SZ, P], I),
        "su3s_field_download": ([P, P, SZ, P], I),
        "su3s_field_download_static": ([P, P, SZ, P], I),
        "su3s_field_stored_bytes": ([P, ctypes.POINTER(SZ)], I),
        "su3s_field_upload_stored": ([P, P, SZ, P], I),
        "su3s_field_download_stored": ([P, P, SZ, P], I),
        "su3s_expr_leaf": ([P, PP], I),
        "su3s_expr_mul": ([P, P, PP], I),
        "su3s_expr_add": ([P, P, PP], I),
        "su3s_expr_sub": ([P, P, PP], I),
        "su3s_expr_scale": ([D, P, PP], I),
        "su3s_expr_adj": ([P, PP], I),
        "su3s_expr_free": ([P], I),
        "su3s_expr_signature": ([P, ctypes.c_char_p, SZ], I),
        "su3s_expr_num_leaves": ([P, ctypes.POINTER(I)], I),
        "su3s_eval": ([P, P, P], I),
        "su3s_eval_math": ([P, P, I, P], I),
        "su3s_set_default_math": ([I], I),
        "su3s_catalogue": ([ctypes.c_char_p, SZ], I),
        "su3s_set_launch": ([P, P, I, I, I], I),
        "su3s_set_pipeline": ([I], I),
        "su3s_device_error": ([ctypes.POINTER(I), P], I),
        "su3s_selftest_bounded_wait": ([ctypes.c_uint32, ctypes.POINTER(I64), P], I),
        "su3s_tune": ([P, P, I, P, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I),
                       ctypes.POINTER(ctypes.c_float)], I),
        "su3s_batch_create": ([PP], I),
        "su3s_batch_add": ([P, P, P], I),
        "su3s_batch_build": ([P, I, I, I, P], I),
        "su3s_batch_tune": ([P, I, P, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I),
                             ctypes.POINTER(ctypes.c_float)], I),
        "su3s_batch_launch": ([P, P], I),
        "su3s_batch_info": ([P, ctypes.POINTER(I64), ctypes.POINTER(I64)], I),
        "su3s_batch_destroy": ([P], I),
        "su3s_eval_adjoint": ([P, P, PP, I, I, P], I),
        "su3s_tune_adjoint": ([P, P, PP, I, I, P, ctypes.POINTER(I), ctypes.POINTER(I),
                               ctypes.POINTER(I), ctypes.POINTER(ctypes.c_float)], I),
        "su3s_field_redot": ([P, P, P, P], I),
        "su3s_reunitarize": ([P, P, P], I),
        "su3s_cshift": ([P, P, I, I, P], I),
        "su3s_hop": ([P, P, P, I, P], I),
        "su3s_dslash": ([P, P, P, I, P], I),
        "su3s_set_adjoint_split": ([I], I),
    }
    for name, (args, res) in sigs.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


def _check(rc):
    if rc != 0:
        raise Su3sError(rc, _lib.su3s_last_error().decode())


def _stream(stream):
    """cudaStream_t of a torch stream (None = torch's current stream)."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def catalogue():
    """(kind, signature, precision, arithmetic) of every compiled kernel."""
    L = load()
    buf = ctypes.create_string_buffer(1 << 16)
    _check(L.su3s_catalogue(buf, len(buf)))
    return [tuple(line.split()) for line in buf.value.decode().splitlines()]


def set_default_math(math):
    _check(load().su3s_set_default_math(math))


PIPE_AUTO, PIPE_PLAIN, PIPE_TMA, PIPE_TMA_LEAF, PIPE_TMA_RING, PIPE_TMA_PAIR = -1, 0, 1, 2, 3, 4


def set_pipeline(mode):
    """-1 the library's choice, 0 plain loads, 1 TMA-staged tiles, 2 TMA-staged
    per leaf, 3 TMA-staged through a ring of buffers, 4 TMA-staged two tiles at
    a time with two sites per lane (FP64 storage; layouts that keep 32 sites
    contiguous; trees without a kernel of that mode use their default)."""
    _check(load().su3s_set_pipeline(mode))


def device_error(stream=None):
    """Read and clear the device error word (0 = every bounded wait completed)."""
    c = ctypes.c_int()
    _check(load().su3s_device_error(ctypes.byref(c), _stream(stream)))
    return c.value


# ---------------------------------------------------------------- lattice
def selftest_bounded_wait(polls=4096, stream=None):
    """Run the bounded-wait diagnostic (a wait that nothing completes gives up
    after `polls` polls); returns the SM cycles the wait took.  The device
    error word is left at 1 (read it with device_error())."""
    c = ctypes.c_int64()
    _check(load().su3s_selftest_bounded_wait(polls, ctypes.byref(c), _stream(stream)))
    return c.value


class Lattice:
    """A 4-d lattice Lx*Ly*Lz*Lt (site index x + Lx*(y + Ly*(z + Lz*t)))."""

    def __init__(self, dims):
        L = load()
        self.dims = tuple(int(d) for d in dims)
        assert len(self.dims) == 4
        h = ctypes.c_void_p()
        _check(L.su3s_lattice_create(*self.dims, ctypes.byref(h)))
        self._h = h
        v = ctypes.c_int64()
        _check(L.su3s_lattice_volume(h, ctypes.byref(v)))
        self.volume = v.value

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.su3s_lattice_destroy(self._h)
            self._h = None


# ------------------------------------------------------------------ fields
class Field:
    """A field wrapping torch-owned device memory in one of the device layouts.

    FP64 storage is held in a float64 tensor (usable with autograd); other
    precisions in a uint8 tensor.
    """

    def __init__(self, lattice, kind=MATRIX, nmu=1, prec=F64, layout=SOA, block=64, tensor=None):
        import torch
        L = load()
        self.lattice, self.kind, self.nmu, self.prec = lattice, kind, nmu, prec
        self.layout, self.block = layout, (block if layout == AOSOA else 0)
        nb = ctypes.c_size_t()
        _check(L.su3s_field_bytes(lattice._h, kind, nmu, prec, layout, block, ctypes.byref(nb)))
        self.nbytes = nb.value
        if tensor is None:
            if prec == F64:
                tensor = torch.empty(nb.value // 8, dtype=torch.float64, device="cuda")
            else:
                tensor = torch.empty(nb.value, dtype=torch.uint8, device="cuda")
        if not tensor.is_cuda or not tensor.is_contiguous():
            raise ValueError("field storage must be a contiguous CUDA tensor")
        tb = tensor.numel() * tensor.element_size()
        h = ctypes.c_void_p()
        _check(L.su3s_field_wrap(lattice._h, kind, nmu, prec, layout, block,
                                 ctypes.c_void_p(tensor.data_ptr()), tb, ctypes.byref(h)))
        self._h = h
        self.tensor = tensor

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.su3s_field_destroy(self._h)
            self._h = None

    @property
    def canonical_shape(self):
        tail = {MATRIX: (3, 3, 2), VECTOR: (3, 2), REAL: ()}[self.kind]
        return (self.lattice.volume * self.nmu,) + tail

    def like(self, prec=None, kind=None):
        """A new field of the same lattice, links and layout."""
        return Field(self.lattice, self.kind if kind is None else kind, self.nmu,
                     self.prec if prec is None else prec, self.layout, self.block or 64)

    # transfers -----------------------------------------------------------
    def upload(self, host, stream=None):
        """Copy a canonical float64 host array (numpy or CPU tensor; pinned for
        an asynchronous copy) into the field."""
        import torch
        if isinstance(host, np.ndarray):
            arr = np.ascontiguousarray(host, dtype=np.float64)
            ptr, n, keep = arr.ctypes.data, arr.size, arr
        else:
            assert host.dtype == torch.float64 and not host.is_cuda and host.is_contiguous()
            ptr, n, keep = host.data_ptr(), host.numel(), host
        _check(_lib.su3s_field_upload(self._h, ctypes.c_void_p(ptr), n, _stream(stream)))
        if isinstance(host, np.ndarray):
            torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()
        del keep

    def download(self, out=None, stream=None):
        """Canonical float64 copy of the field on the host (synchronous unless
        `out` is a pinned CPU tensor and a stream is given)."""
        import torch
        shape = self.canonical_shape
        if out is None:
            res = np.empty(shape, dtype=np.float64)
            _check(_lib.su3s_field_download(self._h, ctypes.c_void_p(res.ctypes.data), res.size,
                                            _stream(stream)))
            (torch.cuda.current_stream() if stream is None else stream).synchronize()
            return res
        _check(_lib.su3s_field_download(self._h, ctypes.c_void_p(out.data_ptr()), out.numel(),
                                        _stream(stream)))
        return out

    def download_static(self, stream=None):
        """Canonical float64 copy on the host through the library's fixed
        staging array: no device memory is allocated (fields up to 2^21
        doubles; synchronous)."""
        import torch
        res = np.empty(self.canonical_shape, dtype=np.float64)
        _check(_lib.su3s_field_download_static(self._h, ctypes.c_void_p(res.ctypes.data), res.size,
                                               _stream(stream)))
        (torch.cuda.current_stream() if stream is None else stream).synchronize()
        return res

    @property
    def stored_shape(self):
        """Shape of the stored-format host array: (V*nmu, ncomp, 2) (ncomp = 9,
        6 for two-row matrices, 3 for vectors) or (V*nmu,) for reals."""
        if self.kind == REAL:
            return (self.lattice.volume * self.nmu,)
        nc = 3 if self.kind == VECTOR else 6 if self.prec in (F64_C12, F32_C12) else 9
        return (self.lattice.volume * self.nmu, nc, 2)

    @property
    def stored_dtype(self):
        """torch dtype of one stored real of the field."""
        import torch
        if self.kind == REAL:
            return torch.float64
        return {F64: torch.float64, F64_C12: torch.float64, F32: torch.float32,
                F32_C12: torch.float32, BF16: torch.bfloat16, F16: torch.float16}[self.prec]

    def _check_stored(self, t):
        if t.is_cuda or not t.is_contiguous():
            raise ValueError("stored-format array must be a contiguous CPU tensor (got %s, "
                             "shape %s, strides %s)" % (t.device, tuple(t.shape), t.stride()))
        if t.dtype != self.stored_dtype or tuple(t.shape) != self.stored_shape:
            raise ValueError("stored-format array is %s %s; the field needs %s %s"
                             % (t.dtype, tuple(t.shape), self.stored_dtype, self.stored_shape))

    def upload_stored(self, host, stream=None):
        """Copy a stored-format CPU tensor (`stored_shape`, `stored_dtype`; pinned
        for an asynchronous copy) into the field, bytes unchanged."""
        import torch
        self._check_stored(host)
        _check(_lib.su3s_field_upload_stored(self._h, ctypes.c_void_p(host.data_ptr()),
                                             host.numel() * host.element_size(), _stream(stream)))
        if not host.is_pinned():
            (torch.cuda.current_stream() if stream is None else stream).synchronize()

    def download_stored(self, out=None, stream=None):
        """The field's stored bytes as a CPU tensor (`stored_shape`, `stored_dtype`);
        synchronous unless `out` is a pinned CPU tensor and a stream is given."""
        import torch
        sync = out is None
        if out is None:
            out = torch.empty(self.stored_shape, dtype=self.stored_dtype)
        self._check_stored(out)
        _check(_lib.su3s_field_download_stored(self._h, ctypes.c_void_p(out.data_ptr()),
                                               out.numel() * out.element_size(), _stream(stream)))
        if sync:
            (torch.cuda.current_stream() if stream is None else stream).synchronize()
        return out

    def pack(self, dev_canonical, stream=None):
        """Fill the field from a canonical float64 CUDA tensor."""
        assert dev_canonical.is_cuda and dev_canonical.is_contiguous()
        assert dev_canonical.numel() == int(np.prod(self.canonical_shape))
        _check(_lib.su3s_field_pack(self._h, ctypes.c_void_p(dev_canonical.data_ptr()),
                                    _stream(stream)))

    def unpack(self, stream=None):
        """Canonical float64 CUDA tensor of the field."""
        import torch
        out = torch.empty(self.canonical_shape, dtype=torch.float64, device="cuda")
        _check(_lib.su3s_field_unpack(self._h, ctypes.c_void_p(out.data_ptr()), _stream(stream)))
        return out

    # expressions ---------------------------------------------------------
    def expr(self):
        return Expr._leaf(self)

    def __mul__(self, o):
        return self.expr() * o

    def __rmul__(self, o):
        return o * self.expr()

    def __add__(self, o):
        return self.expr() + o

    def __sub__(self, o):
        return self.expr() - o

    def __neg__(self):
        return -self.expr()

    def adj(self):
        return self.expr().adj()


def _as_expr(x):
    if isinstance(x, Expr):
        return x
    if isinstance(x, Field):
        return x.expr()
    raise TypeError("expected a Field or an Expr, got %r" % (type(x),))


class Expr:
    """Immutable expression tree node (owns one reference to its C handle)."""

    def __init__(self, handle, fields):
        self._h = handle
        self.fields = fields  # keep leaf fields alive

    @classmethod
    def _leaf(cls, f):
        h = ctypes.c_void_p()
        _check(_lib.su3s_expr_leaf(f._h, ctypes.byref(h)))
        return cls(h, [f])

    def _bin(self, fn, other):
        other = _as_expr(other)
        h = ctypes.c_void_p()
        _check(fn(self._h, other._h, ctypes.byref(h)))
        return Expr(h, self.fields + other.fields)

    def __mul__(self, o):
        if isinstance(o, numbers.Real):
            return self._scale(float(o))
        return self._bin(_lib.su3s_expr_mul, o)

    def __rmul__(self, o):
        if isinstance(o, numbers.Real):
            return self._scale(float(o))
        return _as_expr(o)._bin(_lib.su3s_expr_mul, self)

    def __add__(self, o):
        return self._bin(_lib.su3s_expr_add, o)

    def __sub__(self, o):
        return self._bin(_lib.su3s_expr_sub, o)

    def __neg__(self):
        return self._scale(-1.0)

    def _scale(self, s):
        h = ctypes.c_void_p()
        _check(_lib.su3s_expr_scale(s, self._h, ctypes.byref(h)))
        return Expr(h, self.fields)

    def adj(self):
        h = ctypes.c_void_p()
        _check(_lib.su3s_expr_adj(self._h, ctypes.byref(h)))
        return Expr(h, self.fields)

    def signature(self):
        buf = ctypes.create_string_buffer(512)
        _check(_lib.su3s_expr_signature(self._h, buf, len(buf)))
        return buf.value.decode()

    def num_leaves(self):
        n = ctypes.c_int()
        _check(_lib.su3s_expr_num_leaves(self._h, ctypes.byref(n)))
        return n.value

    def unique_fields(self):
        out = []
        for f in self.fields:
            if not any(f is g for g in out):
                out.append(f)
        return out

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.su3s_expr_free(self._h)
            self._h = None


# -------------------------------------------------------------- evaluation
def evaluate(dest, expr, math=MATH_DEFAULT, stream=None):
    """dest = expr at every site, one pass, asynchronous on `stream`."""
    expr = _as_expr(expr)
    _check(_lib.su3s_eval_math(dest._h, expr._h, math, _stream(stream)))
    return dest


def set_launch(dest, expr, threads, blocks_per_sm=0, math=MATH_DEFAULT):
    _check(_lib.su3s_set_launch(dest._h, _as_expr(expr)._h, math, threads, blocks_per_sm))


def tune(dest, expr, math=MATH_DEFAULT, stream=None):
    """Autotune data movement and launch geometry; returns
    (threads, blocks_per_sm, variant, ms)."""
    t, b, v, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_float()
    _check(_lib.su3s_tune(dest._h, _as_expr(expr)._h, math, _stream(stream), ctypes.byref(t),
                          ctypes.byref(b), ctypes.byref(v), ctypes.byref(ms)))
    return t.value, b.value, v.value, ms.value


def eval_adjoint(expr, grad_out, grads, math=MATH_DEFAULT, stream=None):
    """Write dL/d(leaf) into `grads` (one Field or None per unique leaf, in
    order of first appearance) for dL/d(expr) = grad_out."""
    expr = _as_expr(expr)
    arr = (ctypes.c_void_p * max(1, len(grads)))(*[(g._h if g is not None else None) for g in grads])
    _check(_lib.su3s_eval_adjoint(expr._h, grad_out._h, arr, len(grads), math, _stream(stream)))


def set_adjoint_split(mode):
    """Reverse mode of a sum of two products: -1 tuned (split when untuned),
    0 one fused pass, 1 two single-product passes."""
    _check(load().su3s_set_adjoint_split(int(mode)))


def tune_adjoint(expr, grad_out, grads, math=MATH_DEFAULT, stream=None):
    """Autotune the reverse-mode kernel of `expr` (arguments as for
    eval_adjoint; `grads` are overwritten); returns (threads, blocks_per_sm,
    variant, ms)."""
    expr = _as_expr(expr)
    arr = (ctypes.c_void_p * max(1, len(grads)))(*[(g._h if g is not None else None) for g in grads])
    t, b, v, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_float()
    _check(_lib.su3s_tune_adjoint(expr._h, grad_out._h, arr, len(grads), math, _stream(stream),
                                  ctypes.byref(t), ctypes.byref(b), ctypes.byref(v),
                                  ctypes.byref(ms)))
    return t.value, b.value, v.value, ms.value


def redot(x, y, out=None, stream=None):
    """sum over all reals of x*y (= sum_x Re tr(X^dagger Y)) as a 1-element
    float64 CUDA tensor."""
    import torch
    if out is None:
        out = torch.empty(1, dtype=torch.float64, device="cuda")
    _check(_lib.su3s_field_redot(x._h, y._h, ctypes.c_void_p(out.data_ptr()), _stream(stream)))
    return out


def reunitarize(dst, src, stream=None):
    """dst = projection of src to SU(3) at every site."""
    _check(_lib.su3s_reunitarize(dst._h, src._h, _stream(stream)))
    return dst


def cshift(dst, src, dim, shift, stream=None):
    """dst(x) = src(x + shift e_dim), periodic (directions 0..3 = x, y, z, t)."""
    _check(_lib.su3s_cshift(dst._h, src._h, int(dim), int(shift), _stream(stream)))
    return dst


def hop(dst, links, v, math=MATH_DEFAULT, stream=None):
    """dst(x) = sum_mu U_mu(x) v(x+mu) + U_mu(x-mu)^dagger v(x-mu), the colour
    part of the Dslash hopping term; `links` holds the 4 links of every site."""
    _check(_lib.su3s_hop(dst._h, links._h, v._h, math, _stream(stream)))
    return dst


def dslash(dst, links, psi, math=MATH_DEFAULT, stream=None):
    """dst(x) = sum_mu (1 - gamma_mu) U_mu(x) psi(x+mu) + (1 + gamma_mu)
    U_mu(x-mu)^dagger psi(x-mu), the Wilson hopping term with spin (chiral
    gamma basis); psi and dst are colour-vector fields with 4 spin components
    per site (nmu = 4), `links` holds the 4 links of every site."""
    _check(_lib.su3s_dslash(dst._h, links._h, psi._h, math, _stream(stream)))
    return dst


class Batch:
    """Many (dest, expr) items in one persistent launch captured in a CUDA graph."""

    def __init__(self):
        h = ctypes.c_void_p()
        _check(load().su3s_batch_create(ctypes.byref(h)))
        self._h = h
        self._keep = []

    def add(self, dest, expr):
        expr = _as_expr(expr)
        _check(_lib.su3s_batch_add(self._h, dest._h, expr._h))
        self._keep.append((dest, expr))

    def build(self, math=MATH_DEFAULT, threads=0, tile_sites=0, stream=None):
        _check(_lib.su3s_batch_build(self._h, math, threads, tile_sites, _stream(stream)))

    def tune(self, math=MATH_DEFAULT, stream=None):
        """Build with the fastest launch shape (destinations are overwritten);
        returns (threads, tile_sites, blocks_per_sm, ms per launch)."""
        th, tile, bps, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_float()
        _check(_lib.su3s_batch_tune(self._h, math, _stream(stream), ctypes.byref(th),
                                    ctypes.byref(tile), ctypes.byref(bps), ctypes.byref(ms)))
        return th.value, tile.value, bps.value, ms.value

    def launch(self, stream=None):
        _check(_lib.su3s_batch_launch(self._h, _stream(stream)))

    def info(self):
        s, t = ctypes.c_int64(), ctypes.c_int64()
        _check(_lib.su3s_batch_info(self._h, ctypes.byref(s), ctypes.byref(t)))
        return s.value, t.value

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.su3s_batch_destroy(self._h)
            self._h = None


from .autograd import LatticeFunction, lattice_expr  # noqa: E402,F401
