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
