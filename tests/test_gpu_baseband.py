"""Complex-baseband path (RTIS_PATH_BB) through the C ABI against the FP64 oracle.

Parity: the same definition as oracle.energyscape(path="bb") (demodulated
analytic signal every 4th sample, carrier-phase-corrected Catmull-Rom delays,
coarse-grid low-pass); FP32 bar as the other paths, max |E_gpu - E_oracle| <=
1e-4 x peak and the same peak.  Property: within 1e-2 of the peak of the
exact-delay (frequency-domain) energyscape of the same plan.
"""
import numpy as np
import pytest

import oracle as orc
import synth

pytestmark = pytest.mark.gpu

E_TOL = 1e-4


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2208_10839_gb300 import build
    build.build()
    return torch


def run_bb(torch, cfg, dirs=None, **kw):
    from paper_2208_10839_gb300 import Plan
    dirs = cfg["dirs"] if dirs is None else dirs
    with Plan(cfg["mic_xyz"], cfg["fs"], cfg["chirp"], dirs, cfg["n_samples"], path="bb", **kw) as p:
        E = p.process(torch.from_numpy(np.ascontiguousarray(cfg["x"])).cuda()).cpu().numpy()
        assert p.sync() == 0
    return E


def assert_close(E_gpu, E_ref, tol=E_TOL):
    E_gpu = np.asarray(E_gpu, dtype=np.float64)
    assert E_gpu.shape == E_ref.shape
    assert np.all(np.isfinite(E_gpu))
    peak = float(np.max(E_ref))
    err = float(np.max(np.abs(E_gpu - E_ref)))
    assert err <= tol * peak, f"max err {err:.3e} vs peak {peak:.3e} ({err / peak:.2e} relative)"
    i_ref = np.unravel_index(np.argmax(E_ref), E_ref.shape)
    i_gpu = np.unravel_index(np.argmax(E_gpu), E_gpu.shape)
    if i_ref != i_gpu:
        assert float(np.max(E_ref)) - E_ref[i_gpu] <= tol * peak, (i_ref, i_gpu)
    return err / peak


@pytest.mark.parametrize("n_samples,n_dirs,decim", [(8192, 181, 10), (4100, 13, 7), (2048, 40, 3), (64, 5, 1)])
def test_baseband_matches_oracle(torch_cuda, n_samples, n_dirs, decim):
    cfg = synth.single_sensor(n_samples=n_samples, n_dirs=n_dirs)
    E = run_bb(torch_cuda, cfg, decim=decim)
    ref = orc.energyscape(cfg["x"], cfg["chirp"], cfg["mic_xyz"], cfg["dirs"], cfg["fs"], cfg["c"], path="bb",
                          R=decim)
    assert_close(E, ref)


def test_baseband_hemisphere_sampled_directions(torch_cuda):
    # full size (32 x 16384 x 2048, the bench workload); the oracle on 24 sampled rows
    cfg = synth.hemisphere()
    E = run_bb(torch_cuda, cfg)
    pick = np.sort(np.random.default_rng(3).choice(cfg["dirs"].shape[0], 24, replace=False))
    ref = orc.energyscape(cfg["x"], cfg["chirp"], cfg["mic_xyz"], cfg["dirs"][pick], cfg["fs"], cfg["c"], path="bb")
    full_peak_row = int(np.argmax(E.max(axis=1)))
    assert_close(E[pick], ref)
    # the sampled rows' peak is also not above the full image's
    assert E[pick].max() <= E[full_peak_row].max()


def test_baseband_custom_taps_and_calibration(torch_cuda):
    torch = torch_cuda
    from paper_2208_10839_gb300 import Plan
    cfg = synth.single_sensor(n_samples=6144, n_dirs=33, seed_scene=4)
    taps = np.hanning(13)[1:-1].astype(np.float32)    # 11 taps, unnormalised
    rng = np.random.default_rng(6)
    gain = rng.uniform(0.8, 1.2, size=32).astype(np.float32)
    delay = rng.uniform(-2e-6, 2e-6, size=32).astype(np.float32)
    with Plan(cfg["mic_xyz"], cfg["fs"], cfg["chirp"], cfg["dirs"], 6144, path="bb", decim=6, lpf_taps=taps) as p:
        p.set_calibration(gain=torch.from_numpy(gain).cuda(), delay_s=torch.from_numpy(delay).cuda())
        E = p.process(torch.from_numpy(cfg["x"]).cuda()).cpu().numpy()
        assert p.sync() == 0
    ref = orc.energyscape(cfg["x"], cfg["chirp"], cfg["mic_xyz"], cfg["dirs"], cfg["fs"], cfg["c"], path="bb", R=6,
                          h=taps.astype(np.float64), gain=gain.astype(np.float64), delay_s=delay.astype(np.float64))
    assert_close(E, ref)


def test_baseband_tracks_exact_delay_energyscape(torch_cuda):
    torch = torch_cuda
    from paper_2208_10839_gb300 import Plan
    cfg = synth.single_sensor()
    x = torch.from_numpy(cfg["x"]).cuda()
    out = {}
    for path in ("bb", "fd", "td"):
        with Plan(cfg["mic_xyz"], cfg["fs"], cfg["chirp"], cfg["dirs"], cfg["n_samples"], path=path) as p:
            out[path] = p.process(x).cpu().numpy().astype(np.float64)
            assert p.sync() == 0
    peak = out["fd"].max()
    assert np.max(np.abs(out["bb"] - out["fd"])) < 1e-2 * peak
    assert np.unravel_index(np.argmax(out["bb"]), out["bb"].shape) == \
        np.unravel_index(np.argmax(out["fd"]), out["fd"].shape)


def test_baseband_silence(torch_cuda):
    torch = torch_cuda
    from paper_2208_10839_gb300 import Plan
    cfg = synth.single_sensor(n_samples=4096, n_dirs=16)
    with Plan(cfg["mic_xyz"], cfg["fs"], cfg["chirp"], cfg["dirs"], 4096, path="bb") as p:
        E = p.process(torch.zeros((32, 4096), dtype=torch.int16, device="cuda")).cpu().numpy()
        assert p.sync() == 0
    assert E.shape == (16, 409) and np.all(E == 0.0)


def test_baseband_signal_and_stage_split(torch_cuda):
    # the two stages through their own entry points: z against the oracle's
    # demodulated every-4th-sample signal (2e-5 of max |z|, the matched-filter
    # FP32 bar), and beamform_bb(z) equal to process() bit for bit
    torch = torch_cuda
    from paper_2208_10839_gb300 import Plan, RtisError
    cfg = synth.single_sensor(n_samples=8192, n_dirs=24)
    x = torch.from_numpy(cfg["x"]).cuda()
    with Plan(cfg["mic_xyz"], cfg["fs"], cfg["chirp"], cfg["dirs"], 8192, path="bb") as p:
        z = p.baseband_signal(x)
        E_split = p.beamform_bb(z).cpu().numpy()
        E = p.process(x).cpu().numpy()
        assert p.sync() == 0
        z = z.cpu().numpy()
    a = orc.matched_filter(cfg["x"], cfg["chirp"], cfg["fs"])
    F = orc.fft_length(8192, cfg["chirp"].size)
    k_c = orc.baseband_centre_bin(*orc.band_bins(F, cfg["fs"]))
    z_ref = orc.baseband_signal(a, k_c, F)
    assert z.shape == z_ref.shape
    assert np.max(np.abs(z - z_ref)) <= 2e-5 * np.max(np.abs(z_ref))
    assert np.array_equal(E_split, E)
    # stage entry points refuse plans of another path
    with Plan(cfg["mic_xyz"], cfg["fs"], cfg["chirp"], cfg["dirs"], 8192) as p:
        with pytest.raises(RtisError):
            p.baseband_signal(x)


def test_autotuner_timings_are_reported(torch_cuda):
    # the autotuners keep every layout's time; the chosen layout is the fastest tried
    from paper_2208_10839_gb300 import Plan
    cfg = synth.single_sensor(n_samples=8192, n_dirs=64)
    with Plan(cfg["mic_xyz"], cfg["fs"], cfg["chirp"], cfg["dirs"], 8192, path="bb") as p:
        i = p.info
        td = [v for v in i.td_layout_ms]
        bb = [v for v in i.bb_layout_ms]
    for times, variant, tuned in ((td, i.td_variant, i.td_tuned_ms), (bb, i.bb_variant, i.bb_tuned_ms)):
        tried = [v for v in times if v > 0]
        assert len(tried) >= 4
        assert min(tried) == pytest.approx(tuned, rel=1e-6)
        assert min(times[2 * variant], times[2 * variant + 1] or 1e30) == pytest.approx(tuned, rel=1e-6)


def test_every_layout_and_grid_gives_the_same_energyscape(torch_cuda):
    # forced layouts and grids (the persistent grid loops over many tiles, the baseband
    # one prefetching the next tile's rows) against the autotuned plan: bit for bit,
    # since every layout sums the mics in the same order; the autotuned plan itself
    # is held to the oracle by the other tests
    torch = torch_cuda
    from paper_2208_10839_gb300 import Plan
    cfg = synth.hemisphere(n_dirs=1024, n_samples=8192)
    x = torch.from_numpy(cfg["x"]).cuda()
    args = (cfg["mic_xyz"], cfg["fs"], cfg["chirp"], cfg["dirs"], 8192)
    ref = {}
    for path in ("td", "bb"):
        with Plan(*args, path=path) as p:
            ref[path] = p.process(x).cpu().numpy()
            assert p.sync() == 0
    for grid in ("tile", "persistent"):
        for v in range(5):
            with Plan(*args, td_layout=v, grid=grid) as p:
                assert (p.info.td_variant, p.info.td_grid > 0) == (v, True)
                E = p.process(x).cpu().numpy()
                assert p.sync() == 0
            assert np.array_equal(E, ref["td"]), ("td", v, grid)
        for v in range(6):
            with Plan(*args, path="bb", bb_layout=v, grid=grid) as p:
                assert p.info.bb_variant == v
                E = p.process(x).cpu().numpy()
                assert p.sync() == 0
            assert np.array_equal(E, ref["bb"]), ("bb", v, grid)


@pytest.mark.parametrize("M,N,D,decim", [(1, 4096, 1, 10), (4, 64000, 5, 10), (32, 4104, 3, 9), (13, 2052, 21, 4)])
def test_baseband_edge_shapes(torch_cuda, M, N, D, decim):
    # one mic and one direction; near the longest record (F = 65536); N/4 odd (padded
    # rows of z); R a multiple of 4 (a single low-pass residue)
    torch = torch_cuda
    from paper_2208_10839_gb300 import Plan
    mic = synth.mic_array(M + 100, M)
    dirs = synth.fibonacci_hemisphere(D)
    chirp = synth.chirp().astype(np.float32)
    x = synth.random_measurement(N + 7 * D, M, N, -20000, 20000)
    with Plan(mic, synth.FS, chirp, dirs, N, path="bb", decim=decim) as p:
        E = p.process(torch.from_numpy(x).cuda()).cpu().numpy()
        assert p.sync() == 0
    ref = orc.energyscape(x, chirp, mic, dirs, synth.FS, synth.C_SOUND, path="bb", R=decim)
    assert_close(E, ref)
