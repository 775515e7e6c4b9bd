"""PDM front end (rtis_pdm_demodulate) through the C ABI against the FP64/integer oracle.

The demodulation is integer arithmetic on both sides, so the int16 output is
compared bit for bit; the chain behind it is the PCM chain and keeps its FP32
bar (1e-4 of the peak) against the oracle fed with the same int16 recording.
"""
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


def words_dev(torch, words):
    return torch.from_numpy(np.ascontiguousarray(words).view(np.int32)).cuda()


def demod_gpu(torch, words, M, N, decim=10, taps=None, shift=0):
    from paper_2208_10839_gb300 import pdm_demodulate
    x = pdm_demodulate(words_dev(torch, words), M, N, decim, taps, shift)
    torch.cuda.synchronize()
    return x.cpu().numpy()


def test_pdm_hemisphere_bit_exact(torch_cuda):
    cfg = synth.hemisphere_pdm()
    x = demod_gpu(torch_cuda, cfg["words"], 32, 16384)
    ref = orc.pdm_demodulate(orc.pdm_unpack(cfg["words"], 32), orc.cic_taps(10, 4), 10, 16384)
    assert np.array_equal(x, ref)
    assert np.abs(ref).max() > 1000  # a real signal, not silence


@pytest.mark.parametrize("M,N,decim,ntap,shift,short", [
    (5, 4100, 10, None, 0, 37),        # ragged N, record shorter than N decim (edge zeros)
    (32, 1000, 8, 15, 3, 0),           # custom odd taps with a rounding shift
    (1, 1, 16, 4, 1, 0),               # a single output, even-length taps
    (7, 333, 1, 1, 0, 5),              # decim 1, one tap: unpacking alone
    (32, 640, 64, None, 12, 0),        # the largest decim (CIC length 253), shifted to int16 range
])
def test_pdm_shapes_taps_and_edges(torch_cuda, M, N, decim, ntap, shift, short):
    rng = np.random.default_rng(M * 1000 + N)
    K = N * decim - short
    words = rng.integers(0, 2 ** 32, size=K, dtype=np.uint64).astype(np.uint32)
    taps = None if ntap is None else rng.integers(-300, 900, size=ntap).astype(np.int32)
    x = demod_gpu(torch_cuda, words, M, N, decim, taps, shift)
    g = orc.cic_taps(decim, 4) if taps is None else taps
    ref = orc.pdm_demodulate(orc.pdm_unpack(words, M), g, decim, N, shift)
    assert np.array_equal(x, ref)


def test_pdm_saturates_like_the_oracle(torch_cuda):
    # all-ones bits through a CIC with decim 16: sum 16^4 = 65536 > int16 range
    words = np.full(16 * 200, 0xFFFFFFFF, dtype=np.uint32)
    x = demod_gpu(torch_cuda, words, 3, 200, 16)
    ref = orc.pdm_demodulate(orc.pdm_unpack(words, 3), orc.cic_taps(16, 4), 16, 200)
    assert np.array_equal(x, ref) and x.max() == 32767


def test_pdm_chain_energyscape(torch_cuda):
    # words -> Plan.process_pdm: the demodulated recording goes through the PCM chain;
    # parity against the oracle's energyscape of the oracle's demodulated recording,
    # and the same peak as the PCM recording of the same scene
    torch = torch_cuda
    from paper_2208_10839_gb300 import Plan
    cfg = synth.single_sensor_pdm()
    with Plan(cfg["mic_xyz"], cfg["fs"], cfg["chirp"], cfg["dirs"], cfg["n_samples"]) as p:
        E = p.process_pdm(words_dev(torch, cfg["words"])).cpu().numpy().astype(np.float64)
        assert p.sync() == 0
    x = orc.pdm_demodulate(orc.pdm_unpack(cfg["words"], 32), orc.cic_taps(10, 4), 10, cfg["n_samples"])
    ref = orc.energyscape(x, cfg["chirp"], cfg["mic_xyz"], cfg["dirs"], cfg["fs"], synth.C_SOUND)
    assert np.max(np.abs(E - ref)) <= 1e-4 * ref.max()
    pcm = synth.single_sensor()
    E_pcm = orc.energyscape(pcm["x"], pcm["chirp"], pcm["mic_xyz"], pcm["dirs"], pcm["fs"], pcm["c"])
    assert np.unravel_index(np.argmax(E), E.shape) == np.unravel_index(np.argmax(E_pcm), E_pcm.shape)
