"""rtis_process_many's frequency-domain path with the inverse transform as two
dense DFT stages on the tcgen05 tensor cores (rtis_options.fd_ifft = TC): the
energyscapes must match the FFT form of the same path and the FP64 oracle to
the FP32 tolerance (1e-4 of the peak, same peak index).  The tensor-core form
takes F = 32768 only, so every case records 16384 samples; the direction and
measurement counts leave ragged item lists (fewer items than CTAs, one
measurement, a count that does not divide the CTA groups)."""
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


def measurements(n, n_dirs, n_samples=16384):
    cfgs = [synth.single_sensor(seed_scene=40 + i, n_samples=n_samples, n_dirs=n_dirs) for i in range(n)]
    return cfgs[0], np.stack([c["x"] for c in cfgs])


def both_forms(torch, cfg, xs, n_samples, **kw):
    from paper_2208_10839_gb300 import Plan
    x = torch.from_numpy(xs).cuda()
    out = {}
    for form in ("tc", "fft"):
        with Plan(cfg["mic_xyz"], cfg["fs"], cfg["chirp"], cfg["dirs"], n_samples, path="fd",
                  max_batch=xs.shape[0], fd_ifft=form, **kw) as p:
            assert p.info.fd_ifft == (2 if form == "tc" else 1)
            out[form] = p.process_many(x).cpu().numpy().astype(np.float64)
            assert p.sync() == 0
    return out["tc"], out["fft"]


@pytest.mark.parametrize("n,n_dirs", [(1, 5), (1, 37), (3, 181), (8, 64)])
def test_tc_ifft_matches_fft_form_and_oracle(torch_cuda, n, n_dirs):
    cfg, xs = measurements(n, n_dirs)
    E_tc, E_fft = both_forms(torch_cuda, cfg, xs, 16384)
    errs = []
    for t in range(n):
        peak = E_fft[t].max()
        errs.append(np.max(np.abs(E_tc[t] - E_fft[t])) / peak)
        assert errs[-1] <= E_TOL
        assert np.argmax(E_tc[t]) == np.argmax(E_fft[t])
    print(f"tensor-core vs FFT form, max error / peak: {max(errs):.2e}")
    for t in sorted({0, n - 1}):
        E_ref = orc.energyscape(xs[t], cfg["chirp"], cfg["mic_xyz"], cfg["dirs"], cfg["fs"], cfg["c"], path="fd")
        err = np.max(np.abs(E_tc[t] - E_ref)) / E_ref.max()
        print(f"tensor-core form vs oracle, measurement {t}: {err:.2e}")
        assert err <= E_TOL
        assert np.argmax(E_tc[t]) == np.argmax(E_ref)


def test_tc_ifft_custom_lowpass_and_calibration(torch_cuda):
    """Another decimation and an asymmetric taper (output bins straddle the tiles'
    runs at other offsets), with per-mic gains and delays."""
    torch = torch_cuda
    from paper_2208_10839_gb300 import Plan
    cfg, xs = measurements(2, 23)
    R, taps = 7, np.hanning(33)[1:-1] * np.linspace(1.0, 2.0, 31)
    taps = (taps / taps.sum()).astype(np.float32)
    rng = np.random.default_rng(11)
    gain = rng.uniform(0.8, 1.2, 32).astype(np.float32)
    delay = rng.uniform(-2e-6, 2e-6, 32).astype(np.float32)
    x = torch.from_numpy(xs).cuda()
    with Plan(cfg["mic_xyz"], cfg["fs"], cfg["chirp"], cfg["dirs"], 16384, path="fd", max_batch=2, decim=R,
              lpf_taps=taps, fd_ifft="tc") as p:
        p.set_calibration(None, torch.from_numpy(gain).cuda(), torch.from_numpy(delay).cuda())
        E = p.process_many(x).cpu().numpy().astype(np.float64)
        assert p.sync() == 0
    for t in (0, 1):
        E_ref = orc.energyscape(xs[t], cfg["chirp"], cfg["mic_xyz"], cfg["dirs"], cfg["fs"], cfg["c"], path="fd",
                                gain=gain, delay_s=delay, R=R, h=taps.astype(np.float64))
        assert E.shape[2] == 16384 // R
        assert np.max(np.abs(E[t] - E_ref)) <= E_TOL * E_ref.max()
        assert np.argmax(E[t]) == np.argmax(E_ref)


def test_tc_ifft_is_deterministic(torch_cuda):
    """Bins whose taps straddle two tiles receive two partial sums by atomic adds onto
    zero; with two addends the order cannot change the result."""
    torch = torch_cuda
    from paper_2208_10839_gb300 import Plan
    cfg, xs = measurements(4, 96)
    x = torch.from_numpy(xs).cuda()
    with Plan(cfg["mic_xyz"], cfg["fs"], cfg["chirp"], cfg["dirs"], 16384, path="fd", max_batch=4,
              fd_ifft="tc") as p:
        first = p.process_many(x).clone()
        for _ in range(3):
            assert torch.equal(p.process_many(x), first)
        assert p.sync() == 0


def test_tc_ifft_only_at_its_fft_length(torch_cuda):
    from paper_2208_10839_gb300 import Plan, _native as nat
    cfg, _ = measurements(1, 5, n_samples=8192)
    with pytest.raises(nat.RtisError):
        Plan(cfg["mic_xyz"], cfg["fs"], cfg["chirp"], cfg["dirs"], 8192, path="fd", max_batch=2, fd_ifft="tc")
    with Plan(cfg["mic_xyz"], cfg["fs"], cfg["chirp"], cfg["dirs"], 8192, path="fd", max_batch=2) as p:
        assert p.info.fd_ifft == 1  # auto falls back to the FFT form
