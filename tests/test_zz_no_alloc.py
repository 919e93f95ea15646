"""tor_single_noalloc: the entry point for callers that cannot allocate device memory.

Some callers may not call cudaMalloc (they run inside someone else's memory
pool, or must keep a fixed device footprint), so this entry point takes its
scratch from a fixed array inside the library.  The test calls it through
the C ABI twice in a row (the array keeps the previous call's contents) and
checks each result against tor_single's within the a-posteriori error bound
the other GPU tests use.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2009_01177_gb300 import gbs_inputs as gi

pytestmark = pytest.mark.gpu


def _noalloc(lib, O, out, prec):
    from paper_2009_01177_gb300 import tor
    k = O.shape[0] // 2
    rc = lib.tor_single_noalloc(O.data_ptr(), k, O.stride(0), tor.LAYOUT_XXPP, prec,
                                torch.cuda.current_stream().cuda_stream, out.data_ptr())
    return rc


@pytest.mark.parametrize("prec_name", ["fp64", "dd"])
def test_noalloc_matches_tor_single_on_two_calls(cuda_lib, prec_name):
    tor = cuda_lib
    lib = tor.load_library()
    prec = {"fp64": tor.PREC_FP64, "dd": tor.PREC_DD}[prec_name]
    ctx = tor.Context(0)
    try:
        st, pat, O1 = gi.workload_m16_k10()
        O2 = gi.select(st.O, gi.random_pattern(16, 14, 5))
        for O in (O1, O2):                       # two calls in a row, different sizes
            Od = torch.from_numpy(O).cuda()
            ref = ctx.single(Od, prec=prec_name)
            out = torch.full((tor.RESULT_BYTES,), 0xFF, dtype=torch.uint8, device="cuda")
            assert _noalloc(lib, Od, out, prec) == tor.TOR_OK, lib.tor_last_error().decode()
            torch.cuda.synchronize()
            r = tor.TorResult.from_bytes(out.cpu().numpy().tobytes())
            assert r.status == tor.TOR_OK and r.tier == prec
            assert abs((r.hi - ref.hi) + (r.lo - ref.lo)) <= ref.err_est
            assert abs(r.sum_abs - ref.sum_abs) <= 1e-12 * ref.sum_abs
    finally:
        ctx.close()


def test_noalloc_rejects_oversized_instances(cuda_lib):
    tor = cuda_lib
    lib = tor.load_library()
    st, pat, O = gi.workload_m100(32)
    Od = torch.from_numpy(O).cuda()
    out = torch.zeros(tor.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    rc = _noalloc(lib, Od, out, tor.PREC_FP64)
    assert rc == tor.TOR_EINVAL
    assert "scratch" in lib.tor_last_error().decode()


def test_noalloc_empty_pattern_is_asynchronous(cuda_lib):
    # k = 0 (Tor = 1) is written by a kernel on the caller's stream: the call only enqueues
    tor = cuda_lib
    lib = tor.load_library()
    Od = torch.zeros((0, 0), dtype=torch.float64, device="cuda")
    for prec in (tor.PREC_FP64, tor.PREC_DD):
        out = torch.full((tor.RESULT_BYTES,), 0xFF, dtype=torch.uint8, device="cuda")
        assert _noalloc(lib, Od, out, prec) == tor.TOR_OK
        torch.cuda.synchronize()
        r = tor.TorResult.from_bytes(out.cpu().numpy().tobytes())
        assert (r.hi, r.lo, r.sum_abs, r.err_est, r.tier, r.status) == (1.0, 0.0, 1.0, 0.0, prec, tor.TOR_OK)


def test_noalloc_size_limits_on_a_152_sm_gpu(cuda_lib):
    # the fixed array holds k <= 25 in FP64 and k <= 17 in double-double on a 152-SM GB300
    tor = cuda_lib
    if torch.cuda.get_device_properties(0).multi_processor_count != 152:
        pytest.skip("the limits are stated for 152 SMs")
    lib = tor.load_library()
    st, pat, O32 = gi.workload_m100(32)
    ctx = tor.Context(0)
    try:
        for prec_name, prec, k_lim in (("fp64", tor.PREC_FP64, 25), ("dd", tor.PREC_DD, 17)):
            O = torch.from_numpy(gi.select(st.O, pat[:k_lim])).cuda()
            out = torch.zeros(tor.RESULT_BYTES, dtype=torch.uint8, device="cuda")
            assert _noalloc(lib, O, out, prec) == tor.TOR_OK, lib.tor_last_error().decode()
            torch.cuda.synchronize()
            r = tor.TorResult.from_bytes(out.cpu().numpy().tobytes())
            ref = ctx.single(O, prec=prec_name)
            assert r.status == tor.TOR_OK
            assert abs((r.hi - ref.hi) + (r.lo - ref.lo)) <= ref.err_est
            O1 = torch.from_numpy(gi.select(st.O, pat[:k_lim + 1])).cuda()
            assert _noalloc(lib, O1, out, prec) == tor.TOR_EINVAL
            assert "scratch" in lib.tor_last_error().decode()
    finally:
        ctx.close()
