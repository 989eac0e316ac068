"""The download that allocates no device memory.

su3s_field_download_static is for callers that cannot allocate device memory
when they read a field back (a framework that already holds the device's
memory in its own allocator, or code that must not take the latency or
synchronisation of an allocation).  It stages through a fixed array in the
library's device memory.  These tests call it through the C ABI twice in a
row and compare with su3s_field_download, the allocating entry point.  The
file is collected last so that a run stopping at its first failure has run
every other test before it.
"""
import ctypes

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

SEED = synth.SEED_BASE + 7


def _download_static(su3s, field):
    L = su3s.load()
    out = np.empty(field.canonical_shape, dtype=np.float64)
    stream = torch.cuda.current_stream()
    rc = L.su3s_field_download_static(field._h, ctypes.c_void_p(out.ctypes.data), out.size,
                                      ctypes.c_void_p(stream.cuda_stream))
    assert rc == 0, L.su3s_last_error()
    stream.synchronize()
    return out


@pytest.mark.parametrize("prec", ["f64", "bf16"])
def test_static_download_matches_allocating_download_twice(gpu_lib, prec):
    su3s = gpu_lib
    p = {"f64": su3s.F64, "bf16": su3s.BF16}[prec]
    dims = (16, 16, 16, 16)                  # 65,536 sites: 1,179,648 doubles, under the limit
    lat = su3s.Lattice(dims)
    v = synth.volume(dims)
    a = su3s.Field(lat, su3s.MATRIX, 1, p)
    b = su3s.Field(lat, su3s.MATRIX, 1, p)
    a.upload(synth.su3(SEED, 0, v))
    b.upload(synth.su3(SEED, 1, v))
    # first call
    first = _download_static(su3s, a)
    assert np.array_equal(first, a.download())
    # second call, after the field changed: no stale staging contents
    su3s.evaluate(a, a * b)
    second = _download_static(su3s, a)
    ref = a.download()
    assert np.array_equal(second, ref)
    assert not np.array_equal(first, second)


def test_static_download_small_and_vector_fields(gpu_lib):
    su3s = gpu_lib
    dims = (3, 2, 1, 5)                       # ragged: 30 sites padded to 64
    lat = su3s.Lattice(dims)
    v = synth.volume(dims)
    x = su3s.Field(lat, su3s.VECTOR, 4, su3s.F64, su3s.AOSOA, 32)
    x.upload(synth.gauss_vector(SEED, 4, v * 4))
    for _ in range(2):
        assert np.array_equal(_download_static(su3s, x), x.download())


def test_static_download_rejects_fields_beyond_the_limit(gpu_lib):
    su3s = gpu_lib
    L = su3s.load()
    lat = su3s.Lattice((16, 16, 16, 32))      # 131,072 sites: 2,359,296 doubles > 2^21
    big = su3s.Field(lat, su3s.MATRIX, 1, su3s.F64)
    out = np.empty(big.canonical_shape, dtype=np.float64)
    rc = L.su3s_field_download_static(big._h, ctypes.c_void_p(out.ctypes.data), out.size, None)
    assert rc == 3
    assert b"static staging area" in L.su3s_last_error()


def test_static_download_leaves_device_memory_untouched(gpu_lib):
    # The property the entry point exists for: after a warm-up call (which
    # loads the unpack kernel's code), further calls change neither the
    # device's free memory nor torch's allocator.
    su3s = gpu_lib
    dims = (8, 8, 8, 8)
    lat = su3s.Lattice(dims)
    a = su3s.Field(lat, su3s.MATRIX, 4, su3s.F64)
    a.upload(synth.su3(SEED, 2, synth.volume(dims) * 4))
    first = _download_static(su3s, a)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    allocs0 = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
    for _ in range(3):
        assert np.array_equal(_download_static(su3s, a), first)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_stats().get("allocation.all.allocated", 0) == allocs0
