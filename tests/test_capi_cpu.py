"""CPU-only checks of the C ABI: the library builds, loads, and exports every
entry point include/torontonian.h declares; the binding declares the same set.
No compute call is made (there is no GPU here)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "torontonian.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b((?:tor|gbs)_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2009_01177_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("tor_single", "tor_batch", "tor_bounds", "gbs_sample_step", "tor_create",
                     "tor_destroy", "tor_last_error", "tor_chunks"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_declares_exactly_the_header(lib):
    from paper_2009_01177_gb300 import tor
    assert sorted(tor.SIGNATURES) == declared_functions()


def test_create_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2009_01177_gb300 import tor
    tor.load_library()
    h = ctypes.c_void_p()
    rc = tor._lib.tor_create(ctypes.byref(h), 0)
    assert rc != tor.TOR_OK
    assert tor._lib.tor_last_error().decode()


def test_fixed_point_conversion_on_host(lib):
    # tor_fixed_to_result is pure host code: 3 * 2^128 -> 3.0; -0.5 -> (-0.5)
    from paper_2009_01177_gb300 import tor
    tor.load_library()
    three = [0, 0, 3, 0, 0, 0, 3, 0]
    r = tor.fixed_to_result(three, 5)
    assert (r.hi, r.lo, r.sum_abs) == (3.0, 0.0, 3.0)
    neg_half = (-(1 << 127)) & ((1 << 256) - 1)
    limbs = [(neg_half >> (64 * i)) & 0xFFFFFFFFFFFFFFFF for i in range(4)] + [0, 0, 1, 0]
    r = tor.fixed_to_result(limbs, 5)
    assert (r.hi, r.lo, r.sum_abs) == (-0.5, 0.0, 1.0)
    # hi + lo split of 1 + 2^-100
    v = (1 << 128) + (1 << 28)
    limbs = [(v >> (64 * i)) & 0xFFFFFFFFFFFFFFFF for i in range(4)] + [0, 0, 1, 0]
    r = tor.fixed_to_result(limbs, 5)
    assert (r.hi, r.lo) == (1.0, 2.0 ** -100)


def test_fixed_point_conversion_of_384_bit_partials(lib):
    # the 256-bit tier's partials: two 6-limb values with 192 fraction bits
    from paper_2009_01177_gb300 import tor
    tor.load_library()

    def limbs6(v):
        v &= (1 << 384) - 1
        return [(v >> (64 * i)) & 0xFFFFFFFFFFFFFFFF for i in range(6)]

    r = tor.fixed_to_result(limbs6(3 << 192) + limbs6(5 << 192), 7, "fx256")
    assert (r.hi, r.lo, r.sum_abs, r.tier) == (3.0, 0.0, 5.0, 4)
    # -(2^-100 + 2^-190): its low part lies far below the 128-bit tiers' resolution
    v = -((1 << 92) + (1 << 2))
    r = tor.fixed_to_result(limbs6(v) + limbs6(1 << 192), 7, "fx256")
    assert (r.hi, r.lo) == (-(2.0 ** -100), -(2.0 ** -190))
    # error model: 4k u sum_abs with u = 2^-186
    assert r.err_est == 4 * 7 * 2.0 ** -186 * 1.0
    with pytest.raises(ValueError):
        tor.fixed_to_result(limbs6(1) + limbs6(1), 7, "fp64")   # 12 limbs given, 8 expected


def test_shard_sums_of_384_bit_partials():
    from paper_2009_01177_gb300 import shard
    a = shard.ints_to_limbs(-(1 << 300), 1 << 300, limbs=12)
    b = shard.ints_to_limbs(3, 7, limbs=12)
    tot = shard.sum_partials(np.stack([a, b]))
    assert tot.shape == (12,)
    lo, hi = shard.limbs_to_ints(tot)
    assert lo == (3 - (1 << 300)) % (1 << 384) and hi == (1 << 300) + 7
