"""PDM (pulse-density modulated) recordings: the eRTIS microphones deliver a
1-bit sigma-delta stream (Sec. 2), which this module synthesises.

* Rate: the bit clock is PDM_DECIM = 10 times the 450 kHz PCM rate (4.5 MHz).
* Modulator: second order, noise transfer function (1 - z^-1)^2, error feedback:
  v[k] = u[k] - 2 e[k-1] + e[k-2], y[k] = +1 if v[k] >= 0 else -1, e[k] = y[k] - v[k].
* Packing: one uint32 word per bit-clock tick, bit m = mic m (a synchronous
  32-line capture); bit value 1 stands for +1, 0 for -1.

Like the rest of this package it makes inputs only; the demodulation is the
library's (and the oracle's) job.
"""
from __future__ import annotations

import numpy as np

from .scene import FS, chirp, fibonacci_hemisphere, mic_array, reflectors_hemisphere, reflectors_planar, \
    azimuth_fan, render_echoes, _noise_rng

__all__ = ["PDM_DECIM", "sigma_delta2", "pdm_pack", "pdm_measurement", "hemisphere_pdm", "single_sensor_pdm"]

PDM_DECIM = 10


def sigma_delta2(u):
    """Second-order sigma-delta modulation of u [M][K] (|u| <= about 0.5) -> bits [M][K] uint8."""
    u = np.asarray(u, dtype=np.float64)
    M, K = u.shape
    e1 = np.zeros(M)
    e2 = np.zeros(M)
    bits = np.empty((M, K), dtype=np.uint8)
    for k in range(K):
        v = u[:, k] - 2.0 * e1 + e2
        y = np.where(v >= 0.0, 1.0, -1.0)
        e2 = e1
        e1 = y - v
        bits[:, k] = y > 0.0
    return bits


def pdm_pack(bits):
    """bits [M][K] (0/1, M <= 32) -> uint32 words [K], bit m of word k = bits[m][k]."""
    bits = np.asarray(bits, dtype=np.uint32)
    M = bits.shape[0]
    if M > 32:
        raise ValueError("at most 32 channels per word")
    words = np.zeros(bits.shape[1], dtype=np.uint32)
    for m in range(M):
        words |= bits[m] << np.uint32(m)
    return words


def pdm_measurement(mic, scene, n_samples: int, seed: int, snr_db: float = 20.0, level: float = 0.5,
                    decim: int = PDM_DECIM):
    """Echoes rendered at the bit clock (decim x 450 kHz), white noise at snr_db against
    the clean power, scaled to peak `level`, sigma-delta modulated and packed.
    Returns (words [n_samples * decim], bits [M][n_samples * decim])."""
    K = n_samples * decim
    clean = render_echoes(mic, scene, K, fs=FS * decim)
    p_sig = float(np.mean(clean * clean))
    sigma = np.sqrt(p_sig / 10.0 ** (snr_db / 10.0)) if p_sig > 0 else 1.0
    u = clean + sigma * _noise_rng(seed).normal(size=clean.shape)
    u *= level / max(float(np.max(np.abs(u))), 1e-300)
    bits = sigma_delta2(u)
    return pdm_pack(bits), bits


def single_sensor_pdm(seed_scene: int = 0, seed_mics: int = 0, n_samples: int = 8192, n_dirs: int = 181,
                      n_reflectors: int = 3):
    mic = mic_array(seed_mics)
    sc = reflectors_planar(seed_scene, n_reflectors)
    words, bits = pdm_measurement(mic, sc, n_samples, seed_scene)
    return dict(mic_xyz=mic, dirs=azimuth_fan(n_dirs), chirp=chirp().astype(np.float32), words=words, bits=bits,
                scene=sc, fs=FS, n_samples=n_samples, decim=PDM_DECIM)


def hemisphere_pdm(seed_scene: int = 1, seed_mics: int = 0, n_samples: int = 16384, n_dirs: int = 2048,
                   n_reflectors: int = 20):
    mic = mic_array(seed_mics)
    sc = reflectors_hemisphere(seed_scene, n_reflectors)
    words, bits = pdm_measurement(mic, sc, n_samples, seed_scene)
    return dict(mic_xyz=mic, dirs=fibonacci_hemisphere(n_dirs), chirp=chirp().astype(np.float32), words=words,
                bits=bits, scene=sc, fs=FS, n_samples=n_samples, decim=PDM_DECIM)
