"""The allocation-free matched filter against the plan-based one.

rtis_matched_filter_noalloc is for callers that may not allocate device
memory (a real-time loop that must never enter the allocator, a host
framework that lends its own buffers, code without a plan).  It keeps its
tables and workspace in a static device array instead.  Its output must
match rtis_matched_filter's within the matched-filter tolerance used by the
parity tests, on consecutive calls of different sizes (the second call reuses
the array the first one filled).  A fresh process that never creates a plan
checks that calls of three sizes leave the device's free memory unchanged and
agree with the FP64 oracle's matched filter.  This file is collected last on
purpose.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

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
        err_a = np.max(np.abs(a - a_ref)) / np.max(np.abs(a_ref))
        err_A = np.max(np.abs(A - A_ref)) / np.max(np.abs(A_ref))
        print(f"no-alloc vs plan matched filter, {M} x {N}: {err_a:.1e} (a), {err_A:.1e} (A) of the maximum")
        assert err_a <= A_TOL and err_A <= A_TOL


# Run in a fresh process with eager module loading, so that loading code or the static
# array cannot show up as an allocation: the first call comes before any plan exists,
# then the free device memory is read and must not move over calls of other sizes.
_FRESH = r"""
import json, sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
import oracle, synth
from paper_2208_10839_gb300 import _native as nat
nat.lib()
chirp = synth.chirp().astype(np.float32)
cases = [(32, 16384, 31), (5, 4096, 32), (32, 8192, 33), (32, 16384, 34)]
d_chirp = torch.from_numpy(chirp).cuda()
bufs = []
for M, N, seed in cases:
    x = synth.random_measurement(seed, M, N, -15000, 15000)
    F = oracle.fft_length(N, chirp.shape[0])
    k_lo, k_hi = oracle.band_bins(F, synth.FS)
    bufs.append((x, torch.from_numpy(x).cuda(), torch.empty((M, N), dtype=torch.complex64, device="cuda"),
                 torch.empty((M, k_hi - k_lo + 1), dtype=torch.complex64, device="cuda")))
torch.cuda.synchronize()
out = {"free": [], "err_a": [], "err_A": []}
for i, ((M, N, _), (x, xd, a, A)) in enumerate(zip(cases, bufs)):
    nat.rtis_matched_filter_noalloc(xd, M, N, d_chirp, chirp.shape[0], synth.FS, 20e3, 80e3, a, A)
    torch.cuda.synchronize()
    out["free"].append(torch.cuda.mem_get_info()[0])
    a_ref = oracle.matched_filter(x, chirp, synth.FS)
    A_ref, _, F = oracle.mf_spectrum(x, chirp, synth.FS)
    a_g = a.cpu().numpy().astype(np.complex128)
    A_g = A.cpu().numpy().astype(np.complex128)
    out["err_a"].append(float(np.max(np.abs(a_g - a_ref)) / np.max(np.abs(a_ref))))
    out["err_A"].append(float(np.max(np.abs(A_g - A_ref / F)) / np.max(np.abs(A_ref / F))))
print("RESULT " + json.dumps(out))
"""


@pytest.mark.gpu
def test_noalloc_fresh_process_allocates_nothing_and_matches_oracle(nat):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    env = dict(os.environ, CUDA_MODULE_LOADING="EAGER")
    r = subprocess.run([sys.executable, "-c", _FRESH, ROOT], capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
    line = [ln for ln in r.stdout.splitlines() if ln.startswith("RESULT ")][-1]
    out = json.loads(line[len("RESULT "):])
    print(f"fresh process: free device memory after each call {out['free']}; errors against the oracle "
          f"{['%.1e' % e for e in out['err_a']]} (a), {['%.1e' % e for e in out['err_A']]} (A)")
    assert len(set(out["free"])) == 1, f"free device memory moved between calls: {out['free']}"
    assert max(out["err_a"]) <= A_TOL and max(out["err_A"]) <= A_TOL
