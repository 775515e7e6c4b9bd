"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (FP32 path): energyscape max |E_gpu - E_oracle| <= 1e-4 x peak and
the peak (direction, range bin) identical; matched-filter stage within
2e-5 x max|a| (an FP32 FFT of <= 2^14 points in <= 4 passes carries a few
1e-7 relative error per pass).
"""
import numpy as np
import pytest

import oracle as orc
import synth

pytestmark = pytest.mark.gpu

E_TOL = 1e-4
A_TOL = 2e-5


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2208_10839_gb300 import build
    build.build()
    return torch


def make_plan(cfg, **kw):
    from paper_2208_10839_gb300 import Plan
    return Plan(cfg["mic_xyz"], cfg["fs"], cfg["chirp"], cfg["dirs"], cfg["n_samples"], **kw)


def to_dev(torch, x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def assert_energyscape(E_gpu, E_ref, tol=E_TOL, check_peak=True):
    E_gpu = np.asarray(E_gpu, dtype=np.float64)
    assert E_gpu.shape == E_ref.shape
    assert np.all(np.isfinite(E_gpu))
    peak = float(np.max(E_ref))
    err = float(np.max(np.abs(E_gpu - E_ref)))
    assert err <= tol * peak, f"max err {err:.3e} vs peak {peak:.3e} ({err / peak:.2e} relative)"
    if check_peak:
        i_ref = np.unravel_index(np.argmax(E_ref), E_ref.shape)
        i_gpu = np.unravel_index(np.argmax(E_gpu), E_gpu.shape)
        if i_ref != i_gpu:
            # tie rule: accept only if the oracle's top two values differ by less than the tolerance
            flat = np.sort(E_ref.ravel())
            assert flat[-1] - E_ref[i_gpu] <= tol * peak, (i_ref, i_gpu)
    return err / peak


# ----------------------------------------------------------------------------- matched filter
@pytest.mark.parametrize("N,M,seed", [(4096, 32, 0), (5000, 5, 1), (8192, 32, 2), (16384, 32, 3), (32768, 3, 4)])
def test_matched_filter_matches_oracle(torch_cuda, N, M, seed):
    torch = torch_cuda
    x = synth.random_measurement(seed, M, N, -12000, 12000)
    mic = synth.mic_array(seed, M)
    cfg = dict(mic_xyz=mic, fs=synth.FS, chirp=synth.chirp().astype(np.float32), dirs=synth.azimuth_fan(5),
               n_samples=N)
    with make_plan(cfg) as p:
        a, A = p.matched_filter(to_dev(torch, x), want_a=True, want_spectrum=True)
        torch.cuda.synchronize()
        assert p.sync() == 0
        a_ref = orc.matched_filter(x, cfg["chirp"], cfg["fs"])
        A_ref, k_lo, F = orc.mf_spectrum(x, cfg["chirp"], cfg["fs"])
        assert (k_lo, F) == (p.info.k_lo, p.info.fft_len)
        a_gpu = a.cpu().numpy().astype(np.complex128)
        err = np.max(np.abs(a_gpu - a_ref)) / np.max(np.abs(a_ref))
        assert err <= A_TOL, err
        A_gpu = A.cpu().numpy().astype(np.complex128)
        errA = np.max(np.abs(A_gpu - A_ref / F)) / np.max(np.abs(A_ref / F))
        assert errA <= A_TOL, errA


def test_matched_filter_extremes_and_zero(torch_cuda):
    torch = torch_cuda
    N, M = 4096, 4
    x = np.zeros((M, N), np.int16)
    x[1, ::3] = 32767
    x[2, 1::2] = -32768
    cfg = dict(mic_xyz=synth.mic_array(0, M), fs=synth.FS, chirp=synth.chirp().astype(np.float32),
               dirs=synth.azimuth_fan(3), n_samples=N)
    with make_plan(cfg) as p:
        a, _ = p.matched_filter(to_dev(torch, x))
        a_gpu = a.cpu().numpy().astype(np.complex128)
        a_ref = orc.matched_filter(x, cfg["chirp"], cfg["fs"])
        assert np.all(a_gpu[0] == 0)            # silent channel stays exactly zero
        assert np.max(np.abs(a_gpu - a_ref)) <= A_TOL * np.max(np.abs(a_ref))


# ----------------------------------------------------------------------------- steering table
def test_steering_table_matches_oracle(torch_cuda):
    cfg = synth.hemisphere(n_samples=4096, n_dirs=300)
    with make_plan(cfg) as p:
        shift, weight = p.steering_table()
        shift = shift.cpu().numpy()
        weight = weight.cpu().numpy().astype(np.float64)
    delta = orc.steering_delays(cfg["mic_xyz"], cfg["dirs"], cfg["fs"], cfg["c"])
    j = np.floor(delta)
    w_ref = np.stack(orc.catmull_rom(delta - j), axis=-1)
    same = shift == j
    # floor may differ only where delta sits on an integer to FP64 rounding
    assert np.all(same | (np.abs(delta - np.rint(delta)) < 1e-9))
    np.testing.assert_allclose(weight[same], w_ref[same], atol=2e-7)


# ----------------------------------------------------------------------------- beamformer
def test_beamform_td_from_oracle_mf(torch_cuda):
    """The DAS + envelope kernel alone, fed the oracle's matched-filter output."""
    torch = torch_cuda
    cfg = synth.single_sensor()
    a_ref = orc.matched_filter(cfg["x"], cfg["chirp"], cfg["fs"])
    delta = orc.steering_delays(cfg["mic_xyz"], cfg["dirs"], cfg["fs"], cfg["c"])
    E_ref = orc.envelope_decimate(orc.das_td(a_ref, delta), orc.lpf_taps())
    with make_plan(cfg) as p:
        a_dev = to_dev(torch, a_ref.astype(np.complex64))
        E = p.beamform_td(a_dev)
        assert p.sync() == 0
        rel = assert_energyscape(E.cpu().numpy(), E_ref)
    assert rel < 1e-5


def test_process_single_sensor_config(torch_cuda):
    """32 mics x 8192 samples x 181 azimuth directions, whole chain."""
    torch = torch_cuda
    cfg = synth.single_sensor()
    E_ref = orc.energyscape(cfg["x"], cfg["chirp"], cfg["mic_xyz"], cfg["dirs"], cfg["fs"], cfg["c"])
    with make_plan(cfg) as p:
        E = p.process(to_dev(torch, cfg["x"]))
        assert p.sync() == 0
        assert_energyscape(E.cpu().numpy(), E_ref)


@pytest.mark.parametrize("M,N,D,decim,taps", [
    (1, 4096, 1, 10, None),          # one mic, one direction
    (7, 4100, 13, 10, None),         # N not a multiple of the tile, ragged D
    (32, 6000, 9, 7, 29),            # other decimation / low-pass length
    (32, 2048, 40, 10, 1),           # single-tap (no) low-pass
    (17, 1000, 33, 3, 13),           # short record, tile covers all of it
    (4, 64000, 5, 10, None),         # near the longest record (F = 65536)
])
def test_process_edge_shapes(torch_cuda, M, N, D, decim, taps):
    torch = torch_cuda
    rng = np.random.default_rng(M * 1000 + N)
    mic = synth.mic_array(M, M)
    dirs = synth.fibonacci_hemisphere(D)
    chirp = synth.chirp().astype(np.float32)
    x = synth.random_measurement(N + D, M, N, -20000, 20000)
    h = None
    if taps is not None:
        h = rng.uniform(0.0, 1.0, size=taps).astype(np.float32)
    E_ref = orc.energyscape(x, chirp, mic, dirs, synth.FS, synth.C_SOUND, R=decim,
                            h=None if h is None else h.astype(np.float64))
    cfg = dict(mic_xyz=mic, fs=synth.FS, chirp=chirp, dirs=dirs, n_samples=N)
    with make_plan(cfg, decim=decim, lpf_taps=h) as p:
        E = p.process(to_dev(torch, x))
        assert p.sync() == 0
        assert_energyscape(E.cpu().numpy(), E_ref)


def test_process_far_delays_reach_outside_record(torch_cuda):
    """A wide array: delays of ~100 samples reach before sample 0 and past N-1."""
    torch = torch_cuda
    M, N = 8, 1024
    mic = synth.mic_array(3, M, side=0.16)
    dirs = synth.azimuth_fan(19)
    x = synth.random_measurement(5, M, N)
    chirp = synth.chirp().astype(np.float32)
    E_ref = orc.energyscape(x, chirp, mic, dirs, synth.FS, synth.C_SOUND)
    with make_plan(dict(mic_xyz=mic, fs=synth.FS, chirp=chirp, dirs=dirs, n_samples=N)) as p:
        assert p.info.max_shift >= 100
        E = p.process(to_dev(torch, x))
        assert p.sync() == 0
        assert_energyscape(E.cpu().numpy(), E_ref)


def test_process_all_zero_input_is_zero(torch_cuda):
    torch = torch_cuda
    cfg = synth.single_sensor(n_samples=4096, n_dirs=20)
    with make_plan(cfg) as p:
        E = p.process(torch.zeros((32, 4096), dtype=torch.int16, device="cuda"))
        assert p.sync() == 0
        assert torch.count_nonzero(E).item() == 0


def test_process_repeatable_and_stream_ordered(torch_cuda):
    torch = torch_cuda
    cfg = synth.single_sensor(n_samples=4096, n_dirs=64)
    s = torch.cuda.Stream()
    with make_plan(cfg) as p:
        x = to_dev(torch, cfg["x"])
        E1 = p.process(x).clone()
        with torch.cuda.stream(s):
            E2 = p.process(x, stream=s)
        s.synchronize()
        assert torch.equal(E1, E2)


@pytest.mark.slow
def test_process_hemisphere_full_size_sampled(torch_cuda):
    """Metric size (32 x 16384 x 2048): every direction on a sample, plus the
    GPU's 32 strongest directions, computed by the oracle one by one."""
    torch = torch_cuda
    cfg = synth.hemisphere()
    with make_plan(cfg) as p:
        E = p.process(to_dev(torch, cfg["x"]))
        assert p.sync() == 0
        E = E.cpu().numpy().astype(np.float64)
    a = orc.matched_filter(cfg["x"], cfg["chirp"], cfg["fs"])
    delta = orc.steering_delays(cfg["mic_xyz"], cfg["dirs"], cfg["fs"], cfg["c"])
    rng = np.random.default_rng(0)
    top = np.argsort(E.max(axis=1))[-32:]
    pick = np.unique(np.concatenate([top, rng.choice(E.shape[0], 64, replace=False), [0, E.shape[0] - 1]]))
    E_ref = orc.envelope_decimate(orc.das_td(a, delta[pick]), orc.lpf_taps())
    peak = E.max()
    err = np.max(np.abs(E[pick] - E_ref))
    assert err <= E_TOL * E_ref.max()
    d_gpu, i_gpu = np.unravel_index(np.argmax(E), E.shape)
    d_ref, i_ref = np.unravel_index(np.argmax(E_ref), E_ref.shape)
    assert (pick[d_ref], i_ref) == (d_gpu, i_gpu)
    assert abs(E_ref.max() - peak) <= E_TOL * peak


# ----------------------------------------------------------------------------- frequency-domain path
def test_beamform_fd_from_oracle_spectrum(torch_cuda):
    """The frequency-domain DAS + envelope kernel alone, fed the oracle's in-band spectra."""
    torch = torch_cuda
    cfg = synth.single_sensor()
    A, k_lo, F = orc.mf_spectrum(cfg["x"], cfg["chirp"], cfg["fs"])
    delta = orc.steering_delays(cfg["mic_xyz"], cfg["dirs"], cfg["fs"], cfg["c"])
    E_ref = orc.envelope_decimate(orc.das_fd(A, k_lo, F, cfg["n_samples"], delta), orc.lpf_taps())
    with make_plan(cfg, path="fd") as p:
        E = p.beamform_fd(to_dev(torch, (A / F).astype(np.complex64)))
        assert p.sync() == 0
        rel = assert_energyscape(E.cpu().numpy(), E_ref)
    assert rel < 1e-5


def test_process_fd_single_sensor_config(torch_cuda):
    torch = torch_cuda
    cfg = synth.single_sensor()
    E_ref = orc.energyscape(cfg["x"], cfg["chirp"], cfg["mic_xyz"], cfg["dirs"], cfg["fs"], cfg["c"], path="fd")
    with make_plan(cfg, path="fd") as p:
        E = p.process(to_dev(torch, cfg["x"]))
        assert p.sync() == 0
        assert_energyscape(E.cpu().numpy(), E_ref)


@pytest.mark.parametrize("M,N,D,decim,taps", [
    (1, 4096, 1, 10, None),
    (7, 4100, 13, 10, None),
    (17, 1000, 33, 3, 13),
    (32, 6000, 9, 7, 29),
])
def test_process_fd_edge_shapes(torch_cuda, M, N, D, decim, taps):
    torch = torch_cuda
    rng = np.random.default_rng(M * 1000 + N + 7)
    mic = synth.mic_array(M, M)
    dirs = synth.fibonacci_hemisphere(D)
    chirp = synth.chirp().astype(np.float32)
    x = synth.random_measurement(N + D + 1, M, N, -20000, 20000)
    h = None if taps is None else rng.uniform(0.0, 1.0, size=taps).astype(np.float32)
    E_ref = orc.energyscape(x, chirp, mic, dirs, synth.FS, synth.C_SOUND, path="fd", R=decim,
                            h=None if h is None else h.astype(np.float64))
    cfg = dict(mic_xyz=mic, fs=synth.FS, chirp=chirp, dirs=dirs, n_samples=N)
    with make_plan(cfg, decim=decim, lpf_taps=h, path="fd") as p:
        E = p.process(to_dev(torch, x))
        assert p.sync() == 0
        assert_energyscape(E.cpu().numpy(), E_ref)


@pytest.mark.parametrize("N,D,decim,taps", [
    (32768, 24, 10, None),   # F = 65536: 512-thread kernel, pruned first pass, register fold
    (33000, 9, 9, 13),       # custom short low-pass, ragged N
    (32768, 7, 15, 61),      # a low-pass longer than the register fold takes: the general kernel
])
def test_process_fd_longest_records(torch_cuda, N, D, decim, taps):
    """The frequency-domain path at F = 65536 (records of 32768 samples and more)."""
    torch = torch_cuda
    cfg = synth.hemisphere(seed_scene=11, n_samples=N, n_dirs=D)
    rng = np.random.default_rng(N + D)
    h = None if taps is None else rng.uniform(0.0, 1.0, size=taps).astype(np.float32)
    E_ref = orc.energyscape(cfg["x"], cfg["chirp"], cfg["mic_xyz"], cfg["dirs"], cfg["fs"], cfg["c"], path="fd",
                            R=decim, h=None if h is None else h.astype(np.float64))
    with make_plan(cfg, decim=decim, lpf_taps=h, path="fd") as p:
        assert p.info.fft_len == 65536
        E = p.process(to_dev(torch, cfg["x"]))
        assert p.sync() == 0
        rel = assert_energyscape(E.cpu().numpy(), E_ref)
    print(f"FD at F = 65536, N = {N}: {rel:.1e} of the peak")


@pytest.mark.slow
def test_process_fd_hemisphere_full_size_sampled(torch_cuda):
    torch = torch_cuda
    cfg = synth.hemisphere()
    with make_plan(cfg, path="fd") as p:
        E = p.process(to_dev(torch, cfg["x"]))
        assert p.sync() == 0
        E = E.cpu().numpy().astype(np.float64)
    A, k_lo, F = orc.mf_spectrum(cfg["x"], cfg["chirp"], cfg["fs"])
    delta = orc.steering_delays(cfg["mic_xyz"], cfg["dirs"], cfg["fs"], cfg["c"])
    rng = np.random.default_rng(1)
    top = np.argsort(E.max(axis=1))[-16:]
    pick = np.unique(np.concatenate([top, rng.choice(E.shape[0], 32, replace=False)]))
    E_ref = orc.envelope_decimate(orc.das_fd(A, k_lo, F, cfg["n_samples"], delta[pick]), orc.lpf_taps())
    assert np.max(np.abs(E[pick] - E_ref)) <= E_TOL * E_ref.max()
    d_gpu, i_gpu = np.unravel_index(np.argmax(E), E.shape)
    d_ref, i_ref = np.unravel_index(np.argmax(E_ref), E_ref.shape)
    assert (pick[d_ref], i_ref) == (d_gpu, i_gpu)
