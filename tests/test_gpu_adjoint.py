"""Reverse pass of the time-domain energyscape (rtis_backward) against the
FP64 oracle adjoint, the autograd wrapper, and finite differences of the
GPU forward.

The gradient sums FP32 products over every direction and sample, so it is
compared per quantity with max |g_gpu - g_ref| <= GRAD_TOL x max |g_ref|.
"""
import numpy as np
import pytest

import oracle as orc
import synth

pytestmark = pytest.mark.gpu

GRAD_TOL = 1e-6   # measured: at most 4.9e-7 over every case below (2x margin)
E_TOL = 1e-4


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2208_10839_gb300 import build
    build.build()
    return torch


def to_dev(torch, x, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    return t if dtype is None else t.to(dtype)


def calib_case(seed, M, N, D, n_refl=6):
    """A recording made by a perturbed array (positions, gains, delays)."""
    rng = np.random.default_rng(np.random.SeedSequence([0xAD70, seed]))
    mic_nom = synth.mic_array(seed, M).astype(np.float64)
    mic_true = mic_nom + rng.normal(0.0, 1e-3, size=mic_nom.shape)
    gain = rng.uniform(0.8, 1.2, size=M)
    delay = rng.uniform(-2e-6, 2e-6, size=M)
    r_max = 0.75 * N / synth.FS * synth.C_SOUND / 2  # echoes inside the recording
    sc = synth.reflectors_hemisphere(seed + 7, n_refl, r=(0.3, r_max))
    x = synth.quantise(synth.render_echoes(mic_true, sc, N, mic_gain=gain, mic_delay_s=delay), seed, 20.0)
    return dict(x=x, mic_nom=mic_nom.astype(np.float32), mic_true=mic_true.astype(np.float32),
                gain=gain.astype(np.float32), delay=delay.astype(np.float32),
                dirs=synth.fibonacci_hemisphere(D), chirp=synth.chirp().astype(np.float32), fs=synth.FS,
                c=synth.C_SOUND, N=N)


def assert_close(g, ref, tol=GRAD_TOL, what=""):
    g = np.asarray(g, dtype=np.float64)
    assert np.all(np.isfinite(g)), what
    scale = float(np.max(np.abs(ref)))
    err = float(np.max(np.abs(g - ref)))
    assert scale > 0, what
    print(f"gradient {what}: max |g - g64| / max |g64| = {err / scale:.2e}")
    assert err <= tol * scale, f"{what}: max err {err:.3e} vs scale {scale:.3e} ({err / scale:.2e})"


def gpu_grads(torch, cfg, G, mic, gain, delay, decim=10):
    from paper_2208_10839_gb300 import Plan
    with Plan(cfg["mic_nom"], cfg["fs"], cfg["chirp"], cfg["dirs"], cfg["N"], c=cfg["c"], decim=decim) as p:
        p.set_calibration(to_dev(torch, mic), to_dev(torch, gain), to_dev(torch, delay))
        x = to_dev(torch, cfg["x"])
        E = p.process(x)
        gx, gg, gd = p.backward(x, to_dev(torch, G.astype(np.float32)))
        torch.cuda.synchronize()
        assert p.sync() == 0
        return E.cpu().numpy(), gx.cpu().numpy(), gg.cpu().numpy(), gd.cpu().numpy()


@pytest.mark.parametrize("M,N,D,decim,seed", [
    (32, 4096, 48, 10, 0),   # several range tiles, D a multiple of 8
    (5, 5000, 13, 10, 1),    # ragged: N not a multiple of R or of the tile, D not a multiple of 8
    (32, 8192, 24, 8, 2),    # another decimation
])
def test_backward_matches_oracle(torch_cuda, M, N, D, decim, seed):
    torch = torch_cuda
    cfg = calib_case(seed, M, N, D)
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((D, N // decim))
    E, gx, gg, gd = gpu_grads(torch, cfg, G, cfg["mic_true"], cfg["gain"], cfg["delay"], decim)
    E_ref, gx_ref, gg_ref, gd_ref = orc.energyscape_vjp(
        cfg["x"], cfg["chirp"], cfg["mic_true"], cfg["dirs"], cfg["fs"], cfg["c"], G, gain=cfg["gain"],
        delay_s=cfg["delay"], R=decim)
    assert np.max(np.abs(E - E_ref)) <= E_TOL * np.max(E_ref)
    assert_close(gx, gx_ref, what="dL/dp")
    assert_close(gg, gg_ref, what="dL/dg")
    assert_close(gd, gd_ref, what="dL/dDelta")


def test_backward_l2_loss_cotangent(torch_cuda):
    """The calibration loss L = ||E - E_ref||^2: G = 2 (E - E_ref), sparse in range."""
    torch = torch_cuda
    cfg = calib_case(3, 32, 4096, 40)
    with_nominal = orc.energyscape(cfg["x"], cfg["chirp"], cfg["mic_nom"], cfg["dirs"], cfg["fs"], cfg["c"])
    E_true = orc.energyscape(cfg["x"], cfg["chirp"], cfg["mic_true"], cfg["dirs"], cfg["fs"], cfg["c"],
                             gain=cfg["gain"], delay_s=cfg["delay"])
    G = 2.0 * (E_true - with_nominal)
    G[:, : G.shape[1] // 2] = 0.0  # a cotangent that is zero on whole tiles
    _, gx, gg, gd = gpu_grads(torch, cfg, G, cfg["mic_true"], cfg["gain"], cfg["delay"])
    _, gx_ref, gg_ref, gd_ref = orc.energyscape_vjp(
        cfg["x"], cfg["chirp"], cfg["mic_true"], cfg["dirs"], cfg["fs"], cfg["c"], G, gain=cfg["gain"],
        delay_s=cfg["delay"])
    assert_close(gx, gx_ref, what="dL/dp")
    assert_close(gg, gg_ref, what="dL/dg")
    assert_close(gd, gd_ref, what="dL/dDelta")


def test_backward_zero_cotangent_and_determinism(torch_cuda):
    torch = torch_cuda
    cfg = calib_case(4, 32, 4096, 16)
    G0 = np.zeros((16, 409))
    _, gx, gg, gd = gpu_grads(torch, cfg, G0, cfg["mic_true"], cfg["gain"], cfg["delay"])
    assert not np.any(gx) and not np.any(gg) and not np.any(gd)
    G = np.random.default_rng(4).standard_normal((16, 409))
    r1 = gpu_grads(torch, cfg, G, cfg["mic_true"], cfg["gain"], cfg["delay"])
    r2 = gpu_grads(torch, cfg, G, cfg["mic_true"], cfg["gain"], cfg["delay"])
    for a, b in zip(r1[1:], r2[1:]):
        assert np.array_equal(a, b)  # fixed-order reductions: bit-identical


def test_backward_full_size_sampled_directions(torch_cuda):
    """32 mics x 16384 samples x 2048 directions; the cotangent is nonzero on 48
    sampled directions only, so the oracle needs just those directions."""
    torch = torch_cuda
    cfg = calib_case(5, 32, 16384, 2048, n_refl=10)
    rng = np.random.default_rng(5)
    sel = np.sort(rng.choice(2048, size=48, replace=False))
    G = np.zeros((2048, 1638))
    G[sel] = rng.standard_normal((48, 1638))
    _, gx, gg, gd = gpu_grads(torch, cfg, G, cfg["mic_true"], cfg["gain"], cfg["delay"])
    _, gx_ref, gg_ref, gd_ref = orc.energyscape_vjp(
        cfg["x"], cfg["chirp"], cfg["mic_true"], cfg["dirs"][sel], cfg["fs"], cfg["c"], G[sel], gain=cfg["gain"],
        delay_s=cfg["delay"])
    assert_close(gx, gx_ref, what="dL/dp")
    assert_close(gg, gg_ref, what="dL/dg")
    assert_close(gd, gd_ref, what="dL/dDelta")


def test_autograd_function_and_finite_differences(torch_cuda):
    """energyscape() under torch.autograd gives rtis_backward's gradient, and a
    central difference of the GPU forward along a random direction agrees."""
    torch = torch_cuda
    from paper_2208_10839_gb300 import Plan, energyscape
    cfg = calib_case(6, 32, 4096, 32)
    rng = np.random.default_rng(6)
    G = to_dev(torch, rng.standard_normal((32, 409)).astype(np.float32))
    x = to_dev(torch, cfg["x"])
    with Plan(cfg["mic_nom"], cfg["fs"], cfg["chirp"], cfg["dirs"], cfg["N"], c=cfg["c"]) as p:
        mic = to_dev(torch, cfg["mic_true"]).requires_grad_(True)
        gain = to_dev(torch, cfg["gain"]).requires_grad_(True)
        delay = to_dev(torch, cfg["delay"]).requires_grad_(True)
        L = (energyscape(p, x, mic, gain, delay) * G).sum()
        L.backward()
        torch.cuda.synchronize()
        assert p.sync() == 0
        _, gx_ref, gg_ref, gd_ref = orc.energyscape_vjp(
            cfg["x"], cfg["chirp"], cfg["mic_true"], cfg["dirs"], cfg["fs"], cfg["c"], G.cpu().numpy(),
            gain=cfg["gain"], delay_s=cfg["delay"])
        assert_close(mic.grad.cpu().numpy(), gx_ref, what="autograd dL/dp")
        assert_close(gain.grad.cpu().numpy(), gg_ref, what="autograd dL/dg")
        assert_close(delay.grad.cpu().numpy(), gd_ref, what="autograd dL/dDelta")

        def loss(mv, gv, dv):
            with torch.no_grad():
                return float((energyscape(p, x, mv, gv, dv).double() * G.double()).sum())

        # one direction per parameter group, steps of a few thousandths of a sample of
        # delay: the Catmull-Rom interpolant is only C1 in t, so the central
        # difference has an O(step) error (0.5 % at 4 um on this case, by the FP64 oracle)
        for name, base, grad, eps in (("delay", delay, delay.grad, 1e-8), ("gain", gain, gain.grad, 1e-3),
                                      ("xyz", mic, mic.grad, 4e-6)):
            v = torch.from_numpy(rng.standard_normal(tuple(base.shape)).astype(np.float32)).cuda()
            args_p = [mic.detach(), gain.detach(), delay.detach()]
            args_m = list(args_p)
            k = {"xyz": 0, "gain": 1, "delay": 2}[name]
            args_p[k] = base.detach() + eps * v
            args_m[k] = base.detach() - eps * v
            fd = (loss(*args_p) - loss(*args_m)) / (2 * eps)
            an = float((grad.double() * v.double()).sum())
            assert abs(fd - an) <= 2e-2 * abs(an), (name, fd, an)


def test_loss_l2_matches_numpy(torch_cuda):
    torch = torch_cuda
    from paper_2208_10839_gb300 import Plan, _native as nat
    cfg = calib_case(7, 4, 4096, 19)
    rng = np.random.default_rng(7)
    with Plan(cfg["mic_nom"], cfg["fs"], cfg["chirp"], cfg["dirs"], cfg["N"], c=cfg["c"]) as p:
        E = rng.standard_normal((19, p.n_out)).astype(np.float32)
        Er = rng.standard_normal((19, p.n_out)).astype(np.float32)
        G = torch.empty((19, p.n_out), dtype=torch.float32, device="cuda")
        L = torch.empty(1, dtype=torch.float32, device="cuda")
        nat.rtis_loss_l2(p.handle, to_dev(torch, E), to_dev(torch, Er), G, L)
        torch.cuda.synchronize()
        r = E.astype(np.float64) - Er
        assert np.array_equal(G.cpu().numpy(), 2 * (E - Er))
        assert abs(float(L) - np.sum(r * r)) <= 1e-5 * np.sum(r * r)


def test_calibration_descent_and_checkpoint(torch_cuda, tmp_path):
    """Self-calibration on a known scene: the loss falls, and a checkpoint
    taken mid-run resumes to the bit-identical trajectory."""
    torch = torch_cuda
    from paper_2208_10839_gb300 import Plan
    from paper_2208_10839_gb300.calibrate import Calibrator
    M, N, D = 32, 4096, 128
    rng = np.random.default_rng(np.random.SeedSequence([0xAD70, 9]))
    mic_nom = synth.mic_array(9, M).astype(np.float64)
    mic_true = mic_nom + rng.normal(0, 1e-3, size=mic_nom.shape)
    gain = rng.uniform(0.8, 1.2, size=M)
    delay = rng.uniform(-2e-6, 2e-6, size=M)
    sc = synth.reflectors_hemisphere(20, 8, r=(0.3, 1.1))
    x = synth.quantise(synth.render_echoes(mic_true, sc, N, mic_gain=gain, mic_delay_s=delay), 9, 20.0)
    x_ref = synth.quantise(synth.render_echoes(mic_nom, sc, N), 9, 200.0)
    dirs = synth.fibonacci_hemisphere(D)
    chirp = synth.chirp().astype(np.float32)
    with Plan(mic_nom.astype(np.float32), synth.FS, chirp, dirs, N, c=synth.C_SOUND) as p:
        E_ref = p.process(to_dev(torch, x_ref)).clone()  # the known scene through the nominal array
        xd = to_dev(torch, x)
        cal = Calibrator(p, mic_nom)
        losses = [float(cal.step(xd, E_ref)) for _ in range(6)]
        ck = tmp_path / "cal.npz"
        cal.save(ck)
        cont = [float(cal.step(xd, E_ref)) for _ in range(10)]
        cal2 = Calibrator(p, mic_nom)
        cal2.load(ck)
        resumed = [float(cal2.step(xd, E_ref)) for _ in range(10)]
        assert p.sync() == 0
    assert resumed == cont
    traj = losses + cont
    assert all(np.isfinite(traj))
    assert traj[-1] < 0.8 * traj[0], traj
