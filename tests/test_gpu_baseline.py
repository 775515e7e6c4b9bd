"""The comparison baseline (cuFFT matched filter, one-thread-per-sample
delay-and-sum, separate low-pass kernel) computes the same energyscape as the
fused time-domain path and the FP64 oracle."""
import numpy as np
import pytest

import oracle as orc
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2208_10839_gb300 import build
    build.build()
    return torch


@pytest.mark.parametrize("n_samples,n_dirs,decim", [(8192, 181, 10), (4100, 13, 7)])
def test_baseline_matches_fused_path_and_oracle(torch_cuda, n_samples, n_dirs, decim):
    torch = torch_cuda
    from paper_2208_10839_gb300 import Plan, _native as nat
    cfg = synth.single_sensor(n_samples=n_samples, n_dirs=n_dirs)
    x = torch.from_numpy(cfg["x"]).cuda()
    with Plan(cfg["mic_xyz"], cfg["fs"], cfg["chirp"], cfg["dirs"], n_samples, decim=decim) as p:
        E = p.process(x)
        b = nat.rtis_baseline_create(p.handle)
        try:
            Eb = torch.empty_like(E)
            nat.rtis_baseline_process(b, x, Eb)
            torch.cuda.synchronize()
        finally:
            nat.rtis_baseline_destroy(b)
        assert p.sync() == 0
    E, Eb = E.cpu().numpy().astype(np.float64), Eb.cpu().numpy().astype(np.float64)
    E_ref = orc.energyscape(cfg["x"], cfg["chirp"], cfg["mic_xyz"], cfg["dirs"], cfg["fs"], cfg["c"], R=decim)
    peak = E_ref.max()
    assert np.max(np.abs(Eb - E_ref)) <= 1e-4 * peak
    assert np.max(np.abs(Eb - E)) <= 1e-4 * peak
    assert np.argmax(Eb) == np.argmax(E_ref)
