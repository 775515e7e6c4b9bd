"""Seeded synthetic scenes for the eRTIS imaging sonar (inputs only).

The paper (Sec. 2) describes the eRTIS sensor: one emitter sending a broadband
FM sweep and a known, irregular array of 32 microphones sampled at 450 kHz.
It gives no recordings, so every input here is synthetic and seeded:

* the emitted chirp: linear FM 80 -> 20 kHz, 2 ms, symmetric Hann window;
* microphone positions: uniform in a 12 cm x 12 cm square in the z = 0 plane;
* steering directions: a 1-degree azimuth fan or a Fibonacci half-sphere;
* recordings: point reflectors, spherical propagation emitter -> reflector ->
  microphone at c = 343 m/s (no spreading loss, no absorption), white
  Gaussian noise at a stated SNR, quantised to int16.

Direction frame: the array faces +z; u(az, el) = (sin az cos el, sin el,
cos az cos el).  Nothing here performs matched filtering, beamforming or
envelope detection.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

FS = 450e3          # sampling rate (Sec. 2: 450 kHz)
C_SOUND = 343.0     # speed of sound, m/s
CHIRP_F0 = 80e3     # sweep start (Hz)
CHIRP_F1 = 20e3     # sweep end (Hz)
CHIRP_T = 2e-3      # sweep duration (s)
N_MICS = 32         # Sec. 2: 32 microphones


# --------------------------------------------------------------------------
# emitted signal
# --------------------------------------------------------------------------
def chirp_length(fs: float = FS, T: float = CHIRP_T) -> int:
    return int(round(T * fs))


def chirp_continuous(t, fs: float = FS, f0: float = CHIRP_F0, f1: float = CHIRP_F1,
                     T: float = CHIRP_T):
    """Emitted sweep at continuous times t (s): symmetric Hann x linear FM.

    The Hann window spans the L sample instants 0..(L-1)/fs so that sampling
    this function at t = n/fs gives exactly :func:`chirp` below.
    """
    t = np.asarray(t, dtype=np.float64)
    L = chirp_length(fs, T)
    span = (L - 1) / fs
    k = (f1 - f0) / T
    phase = 2.0 * np.pi * (f0 * t + 0.5 * k * t * t)
    win = 0.5 * (1.0 - np.cos(2.0 * np.pi * t / span))
    inside = (t >= 0.0) & (t <= span)
    return np.where(inside, win * np.cos(phase), 0.0)


def chirp(fs: float = FS, f0: float = CHIRP_F0, f1: float = CHIRP_F1, T: float = CHIRP_T):
    """Sampled emitted sweep s[n], n = 0..L-1 (float64)."""
    L = chirp_length(fs, T)
    return chirp_continuous(np.arange(L) / fs, fs, f0, f1, T)


# --------------------------------------------------------------------------
# geometry
# --------------------------------------------------------------------------
def mic_array(seed: int, n_mics: int = N_MICS, side: float = 0.12):
    """Irregular planar array: uniform in [-side/2, side/2]^2 at z = 0."""
    rng = np.random.default_rng(np.random.SeedSequence([0x6D1C, seed]))
    xy = rng.uniform(-side / 2, side / 2, size=(n_mics, 2))
    return np.concatenate([xy, np.zeros((n_mics, 1))], axis=1).astype(np.float32)


def unit_vector(az, el):
    az = np.asarray(az, dtype=np.float64)
    el = np.asarray(el, dtype=np.float64)
    return np.stack([np.sin(az) * np.cos(el), np.sin(el), np.cos(az) * np.cos(el)], axis=-1)


def azimuth_fan(n: int = 181, lo_deg: float = -90.0, hi_deg: float = 90.0):
    """Horizontal fan of n directions, evenly spaced in azimuth, elevation 0."""
    az = np.deg2rad(np.linspace(lo_deg, hi_deg, n))
    return unit_vector(az, np.zeros_like(az)).astype(np.float32)


def fibonacci_hemisphere(n: int):
    """n directions on the frontal (+z) half-sphere, Fibonacci lattice."""
    i = np.arange(n, dtype=np.float64)
    z = (i + 0.5) / n
    phi = i * np.pi * (3.0 - math.sqrt(5.0))
    rho = np.sqrt(1.0 - z * z)
    return np.stack([rho * np.cos(phi), rho * np.sin(phi), z], axis=1).astype(np.float32)


# --------------------------------------------------------------------------
# scenes
# --------------------------------------------------------------------------
@dataclass
class Scene:
    """Point reflectors in the sensor (or world) frame."""
    pos: np.ndarray              # [Q][3] metres
    amp: np.ndarray              # [Q]
    meta: dict = field(default_factory=dict)


def reflectors_planar(seed: int, n: int = 3, r=(0.5, 4.0), az_deg=(-60.0, 60.0), amp=(0.2, 1.0)):
    rng = np.random.default_rng(np.random.SeedSequence([0x5CE0, seed]))
    rr = rng.uniform(*r, size=n)
    az = np.deg2rad(rng.uniform(*az_deg, size=n))
    a = rng.uniform(*amp, size=n)
    pos = rr[:, None] * unit_vector(az, np.zeros(n))
    return Scene(pos, a, {"range": rr, "az": az, "el": np.zeros(n)})


def reflectors_hemisphere(seed: int, n: int = 20, r=(0.3, 6.0), amp=(0.1, 1.0)):
    """Reflectors uniform over the frontal half-sphere; log-uniform amplitudes."""
    rng = np.random.default_rng(np.random.SeedSequence([0x5CE1, seed]))
    rr = rng.uniform(*r, size=n)
    v = rng.normal(size=(n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    v[:, 2] = np.abs(v[:, 2])
    a = np.exp(rng.uniform(math.log(amp[0]), math.log(amp[1]), size=n))
    return Scene(rr[:, None] * v, a, {"range": rr, "dir": v})


def _noise_rng(seed: int):
    return np.random.default_rng(np.random.SeedSequence([0x0015E, seed]))


def render_echoes(mic_xyz, scene: Scene, n_samples: int, fs: float = FS, c: float = C_SOUND,
                  emitters=None, mic_gain=None, mic_delay_s=None):
    """Clean recording [M][N] (float64) of a point-reflector scene.

    Mic m receives, from reflector q and each emitter e, the sweep delayed by
    (|q - e| + |q - p_m|)/c (+ the mic's own hardware delay) and scaled by
    the reflector amplitude (and the mic's gain).  Emitters default to a
    single one at the origin; all fire at t = 0 (Sec. 2: synchronised
    emission).
    """
    mic = np.asarray(mic_xyz, dtype=np.float64)
    M = mic.shape[0]
    em = np.zeros((1, 3)) if emitters is None else np.asarray(emitters, dtype=np.float64)
    gain = np.ones(M) if mic_gain is None else np.asarray(mic_gain, dtype=np.float64)
    dly = np.zeros(M) if mic_delay_s is None else np.asarray(mic_delay_s, dtype=np.float64)
    L = chirp_length(fs)
    out = np.zeros((M, n_samples))
    for m in range(M):
        for q in range(scene.pos.shape[0]):
            for e in range(em.shape[0]):
                tau = (np.linalg.norm(scene.pos[q] - em[e]) + np.linalg.norm(scene.pos[q] - mic[m])) / c
                tau += dly[m]
                n0 = int(math.floor(tau * fs))
                lo, hi = max(n0, 0), min(n0 + L + 2, n_samples)
                if lo >= hi:
                    continue
                t = np.arange(lo, hi) / fs - tau
                out[m, lo:hi] += gain[m] * scene.amp[q] * chirp_continuous(t, fs)
    return out


def quantise(clean, seed: int, snr_db: float = 20.0, full_scale: float = 30000.0):
    """Add white Gaussian noise at snr_db (vs mean clean power) and round to int16.
    A recording with no echo in its window is noise alone (unit variance before
    the full-scale normalisation), as a real sensor's would be."""
    clean = np.asarray(clean, dtype=np.float64)
    p_sig = float(np.mean(clean * clean))
    sigma = math.sqrt(p_sig / 10.0 ** (snr_db / 10.0)) if p_sig > 0 else 1.0
    noisy = clean + sigma * _noise_rng(seed).normal(size=clean.shape)
    peak = float(np.max(np.abs(noisy)))
    scale = full_scale / peak if peak > 0 else 1.0
    return np.clip(np.rint(noisy * scale), -32768, 32767).astype(np.int16)


# --------------------------------------------------------------------------
# workloads (the five benchmark configurations)
# --------------------------------------------------------------------------
def single_sensor(seed_scene: int = 0, seed_mics: int = 0, n_samples: int = 8192, n_dirs: int = 181,
                  n_reflectors: int = 3, snr_db: float = 20.0):
    """32 mics, 1-degree azimuth fan, 3 planar reflectors (0.5-4 m, +-60 deg)."""
    mic = mic_array(seed_mics)
    dirs = azimuth_fan(n_dirs)
    sc = reflectors_planar(seed_scene, n_reflectors)
    x = quantise(render_echoes(mic, sc, n_samples), seed_scene, snr_db)
    return dict(mic_xyz=mic, dirs=dirs, chirp=chirp().astype(np.float32), x=x, scene=sc,
                fs=FS, c=C_SOUND, n_samples=n_samples, name=f"single-sensor {N_MICS}ch x {n_samples} x {n_dirs} az")


def hemisphere(seed_scene: int = 1, seed_mics: int = 0, n_samples: int = 16384, n_dirs: int = 2048,
               n_reflectors: int = 20, snr_db: float = 20.0):
    """32 mics, Fibonacci half-sphere directions, 20 reflectors 0.3-6 m."""
    mic = mic_array(seed_mics)
    dirs = fibonacci_hemisphere(n_dirs)
    sc = reflectors_hemisphere(seed_scene, n_reflectors)
    x = quantise(render_echoes(mic, sc, n_samples), seed_scene, snr_db)
    return dict(mic_xyz=mic, dirs=dirs, chirp=chirp().astype(np.float32), x=x, scene=sc,
                fs=FS, c=C_SOUND, n_samples=n_samples,
                name=f"hemisphere {N_MICS}ch x {n_samples} x {n_dirs} fibonacci")


def measurement_batch(n_frames: int, seed0: int = 200, **kw):
    """n_frames independent seeded measurements of the same array/directions."""
    out = [hemisphere(seed_scene=seed0 + i, **kw) for i in range(n_frames)]
    return out


def gemm_frames(n_bins: int = 1200, f_start: float = 20e3, f_step: float = 50.0, n_frames: int = 64,
                n_dirs: int = 2048, seed_mics: int = 0, seed0: int = 100, n_reflectors: int = 20,
                snr_db: float = 20.0):
    """Channel spectra X[k][m][t] for the frequency-domain beamforming GEMM.

    Frame t is an independent hemisphere scene; bin k sits at f_k = f_start +
    k*f_step.  Each mic's spectrum is the plane/spherical-wave model
    sum_q amp_q exp(-j 2 pi f_k tau_qm) (tau_qm: emitter -> reflector -> mic
    flight time) plus complex white noise at snr_db.
    """
    mic = mic_array(seed_mics).astype(np.float64)
    dirs = fibonacci_hemisphere(n_dirs)
    f = f_start + f_step * np.arange(n_bins)
    M = mic.shape[0]
    X = np.zeros((n_bins, M, n_frames), dtype=np.complex128)
    for t in range(n_frames):
        sc = reflectors_hemisphere(seed0 + t, n_reflectors)
        tau = (np.linalg.norm(sc.pos, axis=1)[:, None]
               + np.linalg.norm(sc.pos[:, None, :] - mic[None, :, :], axis=2)) / C_SOUND   # [Q][M]
        ph = np.exp(-2j * np.pi * f[:, None, None] * tau[None, :, :])                       # [K][Q][M]
        clean = np.einsum("q,kqm->km", sc.amp, ph)
        p = float(np.mean(np.abs(clean) ** 2))
        rng = _noise_rng(seed0 + t)
        sig = math.sqrt(p / 10 ** (snr_db / 10) / 2)
        X[:, :, t] = clean + sig * (rng.normal(size=clean.shape) + 1j * rng.normal(size=clean.shape))
    return dict(mic_xyz=mic.astype(np.float32), dirs=dirs, freqs=f, X=X, fs=FS, c=C_SOUND,
                name=f"fd-gemm {n_bins} bins x {M} mics x {n_frames} frames -> {n_dirs} dirs")


def ring_sensors(n_sensors: int = 8, radius: float = 0.3, n_reflectors: int = 30, seed_scene: int = 3,
                 seed_mics0: int = 10, lengths=(4096, 8192, 16384, 32768), dir_counts=(512, 1024, 2048, 4096),
                 snr_db: float = 20.0, all_emitters: bool = True):
    """Sensors on a ring, radial +z axes, one shared scene; ragged N and D.

    Each recording length and each direction-set size is used
    n_sensors/len(...) times, assigned to sensors by a seeded permutation.
    Returns per-sensor inputs in each sensor's own frame.
    """
    rng = np.random.default_rng(np.random.SeedSequence([0x818C, seed_scene]))
    reps = n_sensors // len(lengths)
    Ns = rng.permutation(np.repeat(np.asarray(lengths), reps))
    Ds = rng.permutation(np.repeat(np.asarray(dir_counts), n_sensors // len(dir_counts)))
    Q = n_reflectors
    rr = rng.uniform(0.5, 6.0, size=Q)
    az = rng.uniform(0.0, 2 * np.pi, size=Q)
    el = np.deg2rad(rng.uniform(-30.0, 30.0, size=Q))
    refl = np.stack([rr * np.cos(el) * np.cos(az), rr * np.cos(el) * np.sin(az), rr * np.sin(el)], axis=1)
    amp = rng.uniform(0.2, 1.0, size=Q)
    centres, rots = [], []
    for s in range(n_sensors):
        th = 2 * np.pi * s / n_sensors
        centres.append(radius * np.array([np.cos(th), np.sin(th), 0.0]))
        # columns: local x, local y, local z expressed in world coordinates
        rots.append(np.array([[-np.sin(th), 0.0, np.cos(th)],
                              [np.cos(th), 0.0, np.sin(th)],
                              [0.0, 1.0, 0.0]]))
    emitters = np.array(centres) if all_emitters else np.array(centres[:1])
    sensors = []
    for s in range(n_sensors):
        mic_local = mic_array(seed_mics0 + s).astype(np.float64)
        mic_world = centres[s][None, :] + mic_local @ rots[s].T
        sc = Scene(refl, amp)
        clean = render_echoes(mic_world, sc, int(Ns[s]), emitters=emitters)
        x = quantise(clean, seed_scene * 100 + s, snr_db)
        sensors.append(dict(mic_xyz=mic_local.astype(np.float32), dirs=fibonacci_hemisphere(int(Ds[s])),
                            chirp=chirp().astype(np.float32), x=x, n_samples=int(Ns[s]), fs=FS, c=C_SOUND,
                            centre=centres[s], rot=rots[s]))
    return dict(sensors=sensors, reflectors=Scene(refl, amp),
                name=f"ring of {n_sensors} sensors, N in {sorted(set(Ns.tolist()))}, D in {sorted(set(Ds.tolist()))}")


def calibration(seed: int = 4, n_samples: int = 16384, n_dirs: int = 2048, n_reflectors: int = 10,
                pos_sigma: float = 1e-3, gain_range=(0.8, 1.2), delay_range_s=(-2e-6, 2e-6),
                snr_db: float = 20.0, seed_mics: int = 0):
    """Array self-calibration workload.

    The recording is made with the *true* array: nominal positions plus
    N(0, pos_sigma) on every coordinate, per-mic gains and hardware delays.
    The reference recording of the same known scene uses the nominal array
    and no gain/delay errors (noise-free).
    """
    rng = np.random.default_rng(np.random.SeedSequence([0xCA11, seed]))
    mic_nom = mic_array(seed_mics).astype(np.float64)
    mic_true = mic_nom + rng.normal(0.0, pos_sigma, size=mic_nom.shape)
    gain = rng.uniform(*gain_range, size=mic_nom.shape[0])
    delay = rng.uniform(*delay_range_s, size=mic_nom.shape[0])
    sc = reflectors_hemisphere(seed + 1000, n_reflectors)
    x = quantise(render_echoes(mic_true, sc, n_samples, mic_gain=gain, mic_delay_s=delay), seed, snr_db)
    ref_clean = render_echoes(mic_nom, sc, n_samples)
    x_ref = quantise(ref_clean, seed, snr_db=200.0)
    return dict(mic_nominal=mic_nom.astype(np.float32), mic_true=mic_true.astype(np.float32),
                gain_true=gain, delay_true_s=delay, x=x, x_ref=x_ref, dirs=fibonacci_hemisphere(n_dirs),
                chirp=chirp().astype(np.float32), scene=sc, n_samples=n_samples, fs=FS, c=C_SOUND)


def random_measurement(seed: int, n_mics: int, n_samples: int, lo: int = -32768, hi: int = 32767):
    """Uniform random int16 samples (edge-case and parity fodder)."""
    rng = np.random.default_rng(np.random.SeedSequence([0x4A4D, seed]))
    return rng.integers(lo, hi + 1, size=(n_mics, n_samples), dtype=np.int64).astype(np.int16)
