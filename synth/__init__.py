"""Seeded synthetic lattice fields shared by the oracle side and the CUDA side.

Holds no arithmetic of the method under test: it only draws random fields
(SplitMix64 counter stream -> uniforms -> Box-Muller normals -> SU(3) by
Gram-Schmidt over rows and removal of the determinant phase).  Every element is
a pure function of (seed, field id, element index), so a slice can be
regenerated on its own (used to check sampled sites of large lattices).

Arrays are in the canonical host layout of a field: float64 of shape
(n, 3, 3, 2) for matrices, (n, 3, 2) for vectors, (n,) for reals, where
n = volume * links and the element index is m = site * links + mu, with
site = x + Lx*(y + Ly*(z + Lz*t)).
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "su3_synth.c")
_LIB = os.path.join(_HERE, "_synth.so")
_lib = None

#: Seed of each benchmark configuration: SEED_BASE + configuration number.
SEED_BASE = 1710094090
#: Field ids of the standard operands.
FIELD = {"a": 0, "b": 1, "c": 2, "d": 3, "v": 4, "w": 5, "s": 6}

KIND_SU3, KIND_GAUSS_MATRIX, KIND_GAUSS_VECTOR, KIND_UNIFORM = 0, 1, 2, 3
_SHAPE = {0: (3, 3, 2), 1: (3, 3, 2), 2: (3, 2), 3: ()}


def build(force=False):
    """Compile the generator (gcc, no fused multiply-add contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        lib.synth_fill.restype = ctypes.c_int
        lib.synth_fill.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int64,
                                   ctypes.c_int64, ctypes.c_void_p, ctypes.c_int]
        _lib = lib
    return _lib


def _threads():
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:
        return os.cpu_count() or 1


def fill(kind, seed, field, count, first=0, out=None, nthreads=None):
    """Elements first..first+count-1 of a field as float64 in canonical layout."""
    shape = (count,) + _SHAPE[kind]
    if out is None:
        out = np.empty(shape, dtype=np.float64)
    assert out.dtype == np.float64 and out.flags.c_contiguous and out.size == int(np.prod(shape))
    rc = _load().synth_fill(kind, seed, field, first, count, out.ctypes.data,
                            nthreads if nthreads is not None else _threads())
    if rc != 0:
        raise ValueError("synth_fill rejected its arguments")
    return out


def su3(seed, field, count, first=0, **kw):
    """SU(3) matrices: Gaussian, Gram-Schmidt over rows, det phase removed."""
    return fill(KIND_SU3, seed, field, count, first, **kw)


def gauss_matrix(seed, field, count, first=0, **kw):
    """Complex 3x3 matrices with independent standard normal real and imaginary parts."""
    return fill(KIND_GAUSS_MATRIX, seed, field, count, first, **kw)


def gauss_vector(seed, field, count, first=0, **kw):
    """Complex 3-vectors with independent standard normal components."""
    return fill(KIND_GAUSS_VECTOR, seed, field, count, first, **kw)


def uniform_real(seed, field, count, first=0, **kw):
    """Reals drawn uniformly from (-1, 1)."""
    return fill(KIND_UNIFORM, seed, field, count, first, **kw)


def volume(dims):
    v = 1
    for d in dims:
        v *= int(d)
    return v


def site_index(x, y, z, t, dims):
    """Canonical site index, x fastest."""
    lx, ly, lz, _ = dims
    return x + lx * (y + ly * (z + lz * t))


def as_complex(arr):
    """View a canonical float64 array (..., 2) as complex128 (...)."""
    return arr.view(np.complex128).reshape(arr.shape[:-1])
