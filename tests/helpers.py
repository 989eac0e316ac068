"""Small helpers shared by the tests (no method arithmetic)."""
import numpy as np

import synth


def cplx(a):
    return synth.as_complex(np.ascontiguousarray(a))


def real_view(c):
    """complex128 (...) -> float64 (..., 2)."""
    c = np.ascontiguousarray(c)
    return c.view(np.float64).reshape(c.shape + (2,))


def lattice_fields(dims, seed, nmu=1, names=("a", "b")):
    v = synth.volume(dims)
    out = {}
    for n in names:
        fid = synth.FIELD[n]
        if n == "v":
            out[n] = synth.gauss_vector(seed, fid, v * nmu)
        elif n == "w":
            out[n] = synth.gauss_matrix(seed, fid, v * nmu)
        else:
            out[n] = synth.su3(seed, fid, v * nmu)
    return out


E1 = ("add", ("mul", ("leaf", "a"), ("leaf", "b")), ("mul", ("leaf", "c"), ("leaf", "d")))
E2 = ("add", ("mul", ("mul", ("leaf", "a"), ("leaf", "b")), ("leaf", "c")),
      ("scale", 0.5, ("leaf", "d")))
E3 = ("sub", ("mul", ("adj", ("leaf", "a")), ("leaf", "b")),
      ("mul", ("leaf", "b"), ("adj", ("leaf", "a"))))


# one unit in the last place of a value stored in each reduced format, and the
# a priori error bound of a product of SU(3) matrices in each format against
# the exact FP64 product (|entries| <= 1, sum_j |a_ij||b_jk| <= 1)
ULP = {"f32": lambda x: np.spacing(np.abs(x).astype(np.float32)).astype(np.float64),
       "f16": lambda x: np.spacing(np.abs(x).astype(np.float16)).astype(np.float64),
       "bf16": lambda x: 2.0 ** (np.floor(np.log2(np.maximum(np.abs(x), 2.0 ** -126))) - 7)}
BOUND_VS_F64 = {"f32": 2e-6, "f16": 3e-3, "bf16": 2.5e-2}
