"""Frequency-domain beamforming GEMM on tcgen05 vs the FP64 oracle.

Tolerances, relative to max |Y_oracle| of each case: FP32 mode (three BF16
products) 1e-4; BF16 and FP16 operands 1e-2 (the reduced-precision bound).
"""
import numpy as np
import pytest

import oracle as orc
import synth

pytestmark = pytest.mark.gpu
TOL = {"fp32": 1e-4, "bf16": 1e-2, "fp16": 1e-2}


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2208_10839_gb300 import build
    build.build()
    return torch


def run_gemm(torch, mic, dirs, freqs, X, prec, gain=None, delay=None):
    from paper_2208_10839_gb300 import FdGemm
    with FdGemm(mic, dirs, freqs, X.shape[2], gain=gain, delay_s=delay, precision=prec) as g:
        Y = g.run(torch.from_numpy(X.astype(np.complex64)).cuda())
        torch.cuda.synchronize()
        return Y.cpu().numpy().astype(np.complex128)


def rel_err(Y, Y_ref):
    return float(np.max(np.abs(Y - Y_ref)) / np.max(np.abs(Y_ref)))


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp16"])
@pytest.mark.parametrize("D,T,M", [(150, 64, 32), (64, 7, 32), (200, 33, 20), (1, 64, 1)])
def test_fd_gemm_random(torch_cuda, prec, D, T, M):
    rng = np.random.default_rng(D * 100 + T + M)
    mic = synth.mic_array(M, M)
    dirs = synth.fibonacci_hemisphere(D)
    freqs = np.array([20e3, 20e3 + 50 * 37, 51e3, 79.95e3])
    X = (rng.normal(size=(4, M, T)) + 1j * rng.normal(size=(4, M, T))) * 1e3
    gain = rng.uniform(0.8, 1.2, size=M)
    delay = rng.uniform(-2e-6, 2e-6, size=M)
    Y = run_gemm(torch_cuda, mic, dirs, freqs, X, prec, gain, delay)
    W = orc.steering_matrix(freqs, mic, dirs, synth.C_SOUND, gain.astype(np.float32).astype(np.float64),
                            delay.astype(np.float32).astype(np.float64))
    Y_ref = orc.fd_gemm(W, X.astype(np.complex64).astype(np.complex128))
    assert rel_err(Y, Y_ref) <= TOL[prec], (prec, rel_err(Y, Y_ref))


def test_fd_gemm_focuses_plane_wave(torch_cuda):
    """A plane wave from direction d* sums coherently to M at d* (FP32 mode)."""
    mic = synth.mic_array(0)
    dirs = synth.fibonacci_hemisphere(256)
    freqs = np.array([25e3, 60e3])
    d_star = 77
    pu = mic.astype(np.float64) @ dirs[d_star].astype(np.float64)
    X = np.exp(2j * np.pi * freqs[:, None] * pu[None, :] / synth.C_SOUND)[:, :, None] * np.ones((1, 1, 16))
    Y = run_gemm(torch_cuda, mic, dirs, freqs, X, "fp32")
    assert np.all(np.argmax(np.abs(Y[:, :, 0]), axis=1) == d_star)
    np.testing.assert_allclose(np.abs(Y[:, d_star, :]), 32.0, rtol=1e-5)


@pytest.mark.slow
@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp16"])
def test_fd_gemm_full_size_sampled_bins(torch_cuda, prec):
    """1200 bins x 32 mics x 64 frames -> 2048 directions; oracle on sampled bins."""
    torch = torch_cuda
    cfg = synth.gemm_frames()
    from paper_2208_10839_gb300 import FdGemm
    X = cfg["X"]
    with FdGemm(cfg["mic_xyz"], cfg["dirs"], cfg["freqs"], X.shape[2], precision=prec) as g:
        Y = g.run(torch.from_numpy(X.astype(np.complex64)).cuda())
        torch.cuda.synchronize()
        picks = [0, 1, 311, 600, 977, 1199]
        Ys = Y[picks].cpu().numpy().astype(np.complex128)
    W = orc.steering_matrix(cfg["freqs"][picks], cfg["mic_xyz"], cfg["dirs"], cfg["c"])
    Y_ref = orc.fd_gemm(W, X[picks].astype(np.complex64).astype(np.complex128))
    err = rel_err(Ys, Y_ref)
    assert err <= TOL[prec], (prec, err)
