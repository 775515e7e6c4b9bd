"""rtis_process_many: several measurements per call.  On the frequency-domain
path their delay-and-sum runs as one batched tcgen05 GEMM (measurements as
frames) followed by the per-direction phase IFFTs; the result must match the
per-measurement path and the FP64 oracle to the FP32 energyscape tolerance.
On the time-domain path it is rtis_process per measurement, bit for bit."""
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


def measurements(n, n_samples, n_dirs):
    cfgs = [synth.single_sensor(seed_scene=10 + i, n_samples=n_samples, n_dirs=n_dirs) for i in range(n)]
    return cfgs[0], np.stack([c["x"] for c in cfgs])


@pytest.mark.parametrize("n,max_batch", [(1, 4), (3, 4), (16, 16), (24, 64)])
def test_fd_batched_gemm_matches_per_measurement(torch_cuda, n, max_batch):
    torch = torch_cuda
    from paper_2208_10839_gb300 import Plan
    cfg, xs = measurements(n, 8192, 181)
    x = torch.from_numpy(xs).cuda()
    with Plan(cfg["mic_xyz"], cfg["fs"], cfg["chirp"], cfg["dirs"], 8192, path="fd", max_batch=max_batch) as p:
        E = p.process_many(x)
        ref = torch.stack([p.process(x[t]) for t in range(n)])
        assert p.sync() == 0
    E, ref = E.cpu().numpy().astype(np.float64), ref.cpu().numpy().astype(np.float64)
    for t in range(n):
        peak = ref[t].max()
        assert np.max(np.abs(E[t] - ref[t])) <= E_TOL * peak
        assert np.argmax(E[t]) == np.argmax(ref[t])
    for t in sorted({0, n - 1}):  # and against the oracle itself
        E_ref = orc.energyscape(xs[t], cfg["chirp"], cfg["mic_xyz"], cfg["dirs"], cfg["fs"], cfg["c"], path="fd")
        assert np.max(np.abs(E[t] - E_ref)) <= E_TOL * E_ref.max()
        assert np.argmax(E[t]) == np.argmax(E_ref)


def test_fd_batched_gemm_with_calibration(torch_cuda):
    """Gains and per-mic delays reach the GEMM through the steering table."""
    torch = torch_cuda
    from paper_2208_10839_gb300 import Plan
    cfg, xs = measurements(4, 4096, 37)
    rng = np.random.default_rng(3)
    gain = rng.uniform(0.8, 1.2, 32).astype(np.float32)
    delay = rng.uniform(-2e-6, 2e-6, 32).astype(np.float32)
    x = torch.from_numpy(xs).cuda()
    with Plan(cfg["mic_xyz"], cfg["fs"], cfg["chirp"], cfg["dirs"], 4096, path="fd", max_batch=4) as p:
        p.set_calibration(None, torch.from_numpy(gain).cuda(), torch.from_numpy(delay).cuda())
        E = p.process_many(x).cpu().numpy().astype(np.float64)
        assert p.sync() == 0
    for t in (0, 3):
        E_ref = orc.energyscape(xs[t], cfg["chirp"], cfg["mic_xyz"], cfg["dirs"], cfg["fs"], cfg["c"], path="fd",
                                gain=gain, delay_s=delay)
        assert np.max(np.abs(E[t] - E_ref)) <= E_TOL * E_ref.max()


@pytest.mark.slow
def test_fd_batched_gemm_hemisphere_sampled(torch_cuda):
    torch = torch_cuda
    from paper_2208_10839_gb300 import Plan
    cfgs = [synth.hemisphere(seed_scene=1 + i) for i in range(16)]
    cfg = cfgs[0]
    x = torch.from_numpy(np.stack([c["x"] for c in cfgs])).cuda()
    with Plan(cfg["mic_xyz"], cfg["fs"], cfg["chirp"], cfg["dirs"], cfg["n_samples"], path="fd", max_batch=64) as p:
        E = p.process_many(x)
        ref = torch.stack([p.process(x[t]) for t in (0, 15)])
        assert p.sync() == 0
    E = E.cpu().numpy().astype(np.float64)
    ref = ref.cpu().numpy().astype(np.float64)
    for j, t in enumerate((0, 15)):
        assert np.max(np.abs(E[t] - ref[j])) <= E_TOL * ref[j].max()
        assert np.argmax(E[t]) == np.argmax(ref[j])


def test_td_many_is_per_measurement(torch_cuda):
    torch = torch_cuda
    from paper_2208_10839_gb300 import Plan
    cfg, xs = measurements(3, 4096, 24)
    x = torch.from_numpy(xs).cuda()
    with Plan(cfg["mic_xyz"], cfg["fs"], cfg["chirp"], cfg["dirs"], 4096) as p:
        E = p.process_many(x)
        for t in range(3):
            assert torch.equal(E[t], p.process(x[t]))
        assert p.sync() == 0


def test_many_rejects_more_than_max_batch(torch_cuda):
    torch = torch_cuda
    from paper_2208_10839_gb300 import Plan, RtisError
    cfg, xs = measurements(3, 4096, 8)
    with Plan(cfg["mic_xyz"], cfg["fs"], cfg["chirp"], cfg["dirs"], 4096, path="fd", max_batch=2) as p:
        with pytest.raises(RtisError):
            p.process_many(torch.from_numpy(xs).cuda())


def test_both_paths_from_one_matched_filter(torch_cuda):
    """paths=("td", "fd"): the time-domain energyscapes are bit-identical to
    rtis_process on the TD path, the frequency-domain ones match the
    per-measurement FD path."""
    torch = torch_cuda
    from paper_2208_10839_gb300 import Plan
    cfg, xs = measurements(16, 8192, 64)
    x = torch.from_numpy(xs).cuda()
    args = (cfg["mic_xyz"], cfg["fs"], cfg["chirp"], cfg["dirs"], 8192)
    with Plan(*args, max_batch=16) as p, Plan(*args, path="fd") as pf:
        E_td, E_fd = p.process_many(x, paths=("td", "fd"))
        for t in (0, 7, 15):
            assert torch.equal(E_td[t], p.process(x[t]))
            ref = pf.process(x[t]).cpu().numpy().astype(np.float64)
            got = E_fd[t].cpu().numpy().astype(np.float64)
            assert np.max(np.abs(got - ref)) <= E_TOL * ref.max()
        assert p.sync() == 0 and pf.sync() == 0


def test_fd_batched_gemm_longest_records(torch_cuda):
    """F = 65536 (32768-sample records, the ring's longest sensors): the batched GEMM over
    8738 in-band bins and the 512-thread IFFT kernel reading its output, against the
    per-measurement path and the oracle."""
    torch = torch_cuda
    from paper_2208_10839_gb300 import Plan
    cfgs = [synth.hemisphere(seed_scene=40 + i, n_samples=32768, n_dirs=16) for i in range(2)]
    cfg = cfgs[0]
    xs = np.stack([c["x"] for c in cfgs])
    x = torch.from_numpy(xs).cuda()
    with Plan(cfg["mic_xyz"], cfg["fs"], cfg["chirp"], cfg["dirs"], 32768, path="fd", max_batch=2) as p:
        assert p.info.fft_len == 65536
        E = p.process_many(x)
        ref = torch.stack([p.process(x[t]) for t in range(2)])
        assert p.sync() == 0
    E, ref = E.cpu().numpy().astype(np.float64), ref.cpu().numpy().astype(np.float64)
    for t in range(2):
        E_ref = orc.energyscape(xs[t], cfg["chirp"], cfg["mic_xyz"], cfg["dirs"], cfg["fs"], cfg["c"], path="fd")
        for got in (E[t], ref[t]):
            assert np.max(np.abs(got - E_ref)) <= E_TOL * E_ref.max()
            assert np.argmax(got) == np.argmax(E_ref)


@pytest.mark.parametrize("N", [16384, 20000, 31000])
def test_fd_batched_f32768_record_lengths(torch_cuda, N):
    """F = 32768 on the batched path for records from 16384 samples (the hemisphere) to
    31000 (each phase then needs more than half of its P-point IFFT's outputs)."""
    torch = torch_cuda
    from paper_2208_10839_gb300 import Plan
    cfgs = [synth.hemisphere(seed_scene=60 + i, n_samples=N, n_dirs=40) for i in range(3)]
    cfg = cfgs[0]
    xs = np.stack([c["x"] for c in cfgs])
    x = torch.from_numpy(xs).cuda()
    with Plan(cfg["mic_xyz"], cfg["fs"], cfg["chirp"], cfg["dirs"], N, path="fd", max_batch=4) as p:
        assert p.info.fft_len == 32768
        E = p.process_many(x)
        assert p.sync() == 0
    E = E.cpu().numpy().astype(np.float64)
    for t in range(3):
        E_ref = orc.energyscape(xs[t], cfg["chirp"], cfg["mic_xyz"], cfg["dirs"], cfg["fs"], cfg["c"], path="fd")
        err = np.max(np.abs(E[t] - E_ref)) / E_ref.max()
        print(f"batched FD, N = {N}, measurement {t}: {err:.1e} of the peak")
        assert err <= E_TOL
        assert np.argmax(E[t]) == np.argmax(E_ref)
