"""The allocation-free matched filter against the plan-based one.

rtis_matched_filter_noalloc is for callers that may not allocate device
memory (a real-time loop that must never enter the allocator, a host
framework that lends its own buffers, code without a plan).  It keeps its
tables and workspace in a static device array instead.  Its output must
match rtis_matched_filter's within the matched-filter tolerance used by the
parity tests, on consecutive calls of different sizes (the second call reuses
the array the first one filled).  This file is collected last on purpose.
"""
import numpy as np
import pytest

import synth

A_TOL = 2e-5   # matched-filter tolerance of tests/test_gpu_parity.py


@pytest.fixture(scope="module")
def nat():
    from paper_2208_10839_gb300 import build
    build.build()
    from paper_2208_10839_gb300 import _native
    _native.lib()
    return _native


def test_noalloc_rejects_sizes_beyond_static_scratch(nat):
    # 32 mics x 32768 samples need F = 65536: ~8.6 MB of scratch > 8 MiB.
    # Rejected before any CUDA call, so the (never dereferenced) addresses are dummies.
    st = nat.lib().rtis_matched_filter_noalloc(256, 32, 32768, 256, 900, 450e3, 20e3, 80e3, 256, None, None)
    assert st == nat.RTIS_ERR_INVALID_ARG
    assert "static maximum" in nat.last_error()


@pytest.mark.gpu
def test_noalloc_matches_plan_matched_filter_on_consecutive_calls(nat):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2208_10839_gb300 import Plan
    chirp = synth.chirp().astype(np.float32)
    d_chirp = torch.from_numpy(chirp).cuda()
    for M, N, seed in [(32, 16384, 11), (5, 4096, 12)]:
        x = torch.from_numpy(synth.random_measurement(seed, M, N, -15000, 15000)).cuda()
        with Plan(synth.mic_array(seed, M), synth.FS, chirp, synth.azimuth_fan(3), N) as plan:
            a_ref, A_ref = plan.matched_filter(x, want_a=True, want_spectrum=True)
            a = torch.empty_like(a_ref)
            A = torch.empty_like(A_ref)
            nat.rtis_matched_filter_noalloc(x, M, N, d_chirp, chirp.shape[0], synth.FS, 20e3, 80e3, a, A)
            torch.cuda.synchronize()
            a_ref, A_ref, a, A = (t.cpu().numpy().astype(np.complex128) for t in (a_ref, A_ref, a, A))
        assert np.max(np.abs(a - a_ref)) <= A_TOL * np.max(np.abs(a_ref))
        assert np.max(np.abs(A - A_ref)) <= A_TOL * np.max(np.abs(A_ref))
