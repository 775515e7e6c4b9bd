"""Plain FP64 NumPy oracle of the eRTIS energyscape chain.

TEST INFRASTRUCTURE ONLY: imported by the tests, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; never by the library.  It shares no
code with the CUDA path.

The paper (arXiv 2208.10839) describes the processing in words only:

* Fig. 3 caption and Sec. 4.1 -- the recorded channels go through a matched
  filter against the emitted broadband FM sweep, a delay-and-sum beamformer
  forms one beam per direction of interest, and an envelope detector turns
  each beam into a reflector distribution whose time axis is range.
* Sec. 4.3 -- filters are applied as FFT convolutions, the filters' group
  delay is removed, and the envelope is subsampled.

Every function below writes one of those steps out plainly in FP64, with the
readings of the unstated details given in its docstring:

1. input   x_m[n] = int16 / 32768, n in [0, N)
2. matched filter + analytic signal (Sec. 4.1, 4.3): with F the smallest
   power of two >= N + L - 1, A_m[k] = 2 X_m[k] conj(S[k]) for k in
   [ceil(20 kHz F/fs), floor(80 kHz F/fs)], zero elsewhere;
   a_m = IFFT_F(A_m)[0:N] (correlation aligned at lag 0, which removes the
   filter's group delay)
3. far-field steering delays delta_dm = -fs (p_m . u_d)/c + fs Delta_m
4. time-domain delay-and-sum (Sec. 4.1): b_d[n] = sum_m g_m I(a_m, n + delta_dm),
   I = Catmull-Rom (Keys, a = -1/2) interpolation, a = 0 outside [0, N)
   or frequency-domain delay-and-sum: B_d[k] = sum_m g_m e^{+j 2 pi k delta_dm / F} A_m[k],
   b_d = IFFT_F(B_d)[0:N]
5. envelope |b|, zero-phase low-pass FIR h (4R+1 taps) and subsampling by R
   (Sec. 4.3): E[d][i] = sum_j h[j] |b_d|[R i + j - 2R], i < floor(N/R)

Complex-baseband variant (the paper subsamples the signal before the matched
filter, Sec. 4.3; here the subsampling moves behind it, onto the demodulated
analytic signal, where the 60 kHz band allows it):

6. z_m[j] = a_m[Q j] exp(-j 2 pi k_c Q j / F), j < ceil(N/Q), with k_c the
   mid-band bin (the analytic signal shifted to 0 Hz and kept every Q-th sample)
7. b_d[j] = sum_m g_m exp(+j 2 pi k_c delta_dm / F) I(z_m, j + delta_dm / Q)
   (the envelope delayed on the coarse grid, the carrier's phase exactly)
8. E[d][i] = sum_j h_Ri(Q j - R i) |b_d[j]|: the same windowed-sinc low-pass
   sampled at the coarse grid's offsets from R i, renormalised to unit DC gain

PDM front end (the microphones record through a 1-bit sigma-delta ADC, Sec. 2;
the GPU unpacks the bits and demodulates them with a low-pass filter before
the matched filter, Sec. 4.3):

0a. unpack: bit m of word k is mic m's k-th bit; b_m[k] = +1 for 1, -1 for 0
0b. demodulate: x_m[n] = sum_j g[j] b_m[D n + j - c], c = (len(g) - 1) // 2,
    b = 0 outside the record: an integer FIR evaluated at every D-th bit (by
    default the CIC kernel, D = 10, order 4), rounded right shift, int16
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "fft_length", "band_bins", "to_float", "mf_spectrum", "matched_filter", "catmull_rom", "catmull_rom_deriv",
    "lpf_adjoint", "energyscape_vjp",
    "steering_delays", "das_td", "das_td_bruteforce", "das_fd", "lpf_taps", "envelope_decimate",
    "energyscape", "steering_matrix", "fd_gemm", "DEFAULT_BAND", "DEFAULT_DECIM",
    "DEFAULT_BB_DECIM", "baseband_centre_bin", "baseband_signal", "das_bb", "das_bb_bruteforce", "lpf_window",
    "envelope_decimate_bb", "pdm_unpack", "cic_taps", "pdm_demodulate",
]

DEFAULT_BAND = (20e3, 80e3)   # chirp band: the 80 -> 20 kHz sweep
DEFAULT_DECIM = 10            # R: 8192 samples -> 8192/10 range bins
DEFAULT_BB_DECIM = 4          # Q: baseband samples per full-rate sample (112.5 kHz complex rate)


# --------------------------------------------------------------------------
# sizes
# --------------------------------------------------------------------------
def fft_length(n_samples: int, chirp_len: int) -> int:
    """Smallest power of two F with F >= N + L - 1 (linear, not circular, correlation)."""
    F = 1
    while F < n_samples + chirp_len - 1:
        F *= 2
    return F


def band_bins(F: int, fs: float, band=DEFAULT_BAND):
    """First and last FFT bin inside the chirp band: ceil(f_lo F/fs), floor(f_hi F/fs)."""
    k_lo = int(math.ceil(band[0] * F / fs))
    k_hi = int(math.floor(band[1] * F / fs))
    return k_lo, k_hi


def to_float(x_int16):
    """Step 1: int16 samples to real values in [-1, 1)."""
    return np.asarray(x_int16, dtype=np.float64) / 32768.0


# --------------------------------------------------------------------------
# matched filter (Fig. 3, Sec. 4.1; FFT convolution and group delay: Sec. 4.3)
# --------------------------------------------------------------------------
def mf_spectrum(x_int16, chirp, fs: float, band=DEFAULT_BAND):
    """Band-limited one-sided matched-filter spectrum.

    Returns (A, k_lo, F) with A[m][k - k_lo] = 2 X_m[k] conj(S[k]) for the
    in-band bins k = k_lo..k_hi.  X_m and S are F-point DFTs of the
    zero-padded channel and chirp.  Multiplying by conj(S) correlates the
    channel with the sweep; keeping only positive in-band frequencies (x2)
    makes the inverse transform the analytic signal of the band-limited
    correlation.
    """
    x = to_float(x_int16)
    s = np.asarray(chirp, dtype=np.float64)
    M, N = x.shape
    F = fft_length(N, s.shape[0])
    k_lo, k_hi = band_bins(F, fs, band)
    X = np.fft.fft(x, n=F, axis=1)
    S = np.fft.fft(s, n=F)
    k = np.arange(k_lo, k_hi + 1)
    A = 2.0 * X[:, k] * np.conj(S[k])[None, :]
    return A, k_lo, F


def matched_filter(x_int16, chirp, fs: float, band=DEFAULT_BAND, mask: str = "band"):
    """Analytic matched-filter output a_m[n], n in [0, N) (complex128 [M][N]).

    mask="band": the in-band one-sided spectrum of :func:`mf_spectrum`.
    mask="analytic": no band limit -- the textbook analytic-signal mask
    (1 at DC and F/2, 2 on positive bins, 0 on negative bins), so that the
    real part is exactly the linear correlation sum_l x[n+l] s[l].
    """
    x = to_float(x_int16)
    s = np.asarray(chirp, dtype=np.float64)
    M, N = x.shape
    F = fft_length(N, s.shape[0])
    if mask == "band":
        A, k_lo, _ = mf_spectrum(x_int16, chirp, fs, band)
        full = np.zeros((M, F), dtype=np.complex128)
        full[:, k_lo:k_lo + A.shape[1]] = A
    elif mask == "analytic":
        X = np.fft.fft(x, n=F, axis=1)
        S = np.fft.fft(s, n=F)
        H = np.zeros(F)
        H[0] = 1.0
        H[F // 2] = 1.0
        H[1:F // 2] = 2.0
        full = X * np.conj(S)[None, :] * H[None, :]
    else:
        raise ValueError(mask)
    return np.fft.ifft(full, axis=1)[:, :N]


# --------------------------------------------------------------------------
# delay-and-sum (Fig. 3, Sec. 4.1)
# --------------------------------------------------------------------------
def catmull_rom(mu):
    """Catmull-Rom (Keys a = -1/2) weights for taps j-1, j, j+1, j+2 at fraction mu."""
    mu = np.asarray(mu, dtype=np.float64)
    mu2 = mu * mu
    mu3 = mu2 * mu
    w_m1 = 0.5 * (-mu3 + 2.0 * mu2 - mu)
    w_0 = 0.5 * (3.0 * mu3 - 5.0 * mu2 + 2.0)
    w_1 = 0.5 * (-3.0 * mu3 + 4.0 * mu2 + mu)
    w_2 = 0.5 * (mu3 - mu2)
    return w_m1, w_0, w_1, w_2


def catmull_rom_deriv(mu):
    """d/dmu of the Catmull-Rom weights (taps j-1, j, j+1, j+2)."""
    mu = np.asarray(mu, dtype=np.float64)
    mu2 = mu * mu
    return (0.5 * (-3.0 * mu2 + 4.0 * mu - 1.0), 0.5 * (9.0 * mu2 - 10.0 * mu),
            0.5 * (-9.0 * mu2 + 8.0 * mu + 1.0), 0.5 * (3.0 * mu2 - 2.0 * mu))


def steering_delays(mic_xyz, dirs, fs: float, c: float, delay_s=None):
    """Far-field steering delays in samples: delta_dm = fs (Delta_m - (p_m . u_d)/c).

    A plane wave from direction u reaches mic m earlier by (p_m . u)/c than
    the array origin; reading channel m at n + delta_dm lines all channels
    up on the origin's time axis.  Delta_m is an optional per-mic hardware
    delay (seconds) that is advanced out.
    """
    p = np.asarray(mic_xyz, dtype=np.float64)
    u = np.asarray(dirs, dtype=np.float64)
    tau = -(u @ p.T) / c
    if delay_s is not None:
        tau = tau + np.asarray(delay_s, dtype=np.float64)[None, :]
    return fs * tau


def _zero_padded(a, pad):
    M, N = a.shape
    out = np.zeros((M, N + 2 * pad), dtype=np.complex128)
    out[:, pad:pad + N] = a
    return out


def das_td(a, delta, gain=None, chunk: int = 64):
    """Time-domain delay-and-sum with Catmull-Rom fractional delays.

    b_d[n] = sum_m g_m sum_{q=-1..2} w_q(mu) a_m[j+q], with t = n + delta_dm,
    j = floor(t), mu = t - j, and a_m = 0 outside [0, N).
    """
    a = np.asarray(a, dtype=np.complex128)
    delta = np.asarray(delta, dtype=np.float64)
    M, N = a.shape
    D = delta.shape[0]
    g = np.ones(M) if gain is None else np.asarray(gain, dtype=np.float64)
    pad = int(math.ceil(np.max(np.abs(delta)))) + 4 if delta.size else 4
    ap = _zero_padded(a, pad)
    n = np.arange(N, dtype=np.float64)
    b = np.zeros((D, N), dtype=np.complex128)
    for d0 in range(0, D, chunk):
        dd = delta[d0:d0 + chunk]
        for m in range(M):
            t = n[None, :] + dd[:, m:m + 1]
            j = np.floor(t)
            w = catmull_rom(t - j)
            idx = j.astype(np.int64) + pad
            acc = (w[0] * ap[m][idx - 1] + w[1] * ap[m][idx]
                   + w[2] * ap[m][idx + 1] + w[3] * ap[m][idx + 2])
            b[d0:d0 + chunk] += g[m] * acc
    return b


def das_td_bruteforce(a, delta, gain=None):
    """Triple loop over (d, n, m) of the same definition (tiny inputs only)."""
    a = np.asarray(a, dtype=np.complex128)
    M, N = a.shape
    D = delta.shape[0]
    g = np.ones(M) if gain is None else gain
    b = np.zeros((D, N), dtype=np.complex128)
    for d in range(D):
        for n in range(N):
            acc = 0j
            for m in range(M):
                t = n + float(delta[d][m])
                j = math.floor(t)
                mu = t - j
                ws = catmull_rom(mu)
                for q, wq in zip((-1, 0, 1, 2), ws):
                    if 0 <= j + q < N:
                        acc += g[m] * float(wq) * a[m][j + q]
            b[d][n] = acc
    return b


def das_fd(A_band, k_lo: int, F: int, n_samples: int, delta, gain=None):
    """Frequency-domain delay-and-sum.

    B_d[k] = sum_m g_m exp(+j 2 pi k delta_dm / F) A_m[k] on the in-band bins
    (zero elsewhere); b_d = IFFT_F(B_d)[0:N].  The +j sign makes the phase
    ramp a circular advance by delta_dm, matching the time-domain reading.
    """
    A_band = np.asarray(A_band, dtype=np.complex128)
    M, Kb = A_band.shape
    delta = np.asarray(delta, dtype=np.float64)
    D = delta.shape[0]
    g = np.ones(M) if gain is None else np.asarray(gain, dtype=np.float64)
    k = np.arange(k_lo, k_lo + Kb, dtype=np.float64)
    b = np.zeros((D, n_samples), dtype=np.complex128)
    for d in range(D):
        W = g[None, :] * np.exp(2j * np.pi * np.outer(k, delta[d]) / F)     # [Kb][M]
        B = np.zeros(F, dtype=np.complex128)
        B[k_lo:k_lo + Kb] = np.sum(W * A_band.T, axis=1)
        b[d] = np.fft.ifft(B)[:n_samples]
    return b


# --------------------------------------------------------------------------
# envelope, low-pass and subsampling (Fig. 3, Sec. 4.1, Sec. 4.3)
# --------------------------------------------------------------------------
def lpf_window(t, R: int = DEFAULT_DECIM):
    """The envelope low-pass before normalisation, at full-rate offset t:
    sinc(t/R) * (1 + cos(pi t/(2R+1)))/2 for |t| <= 2R, 0 beyond (a Hann
    window whose zeros fall one sample beyond the ends)."""
    t = np.asarray(t, dtype=np.float64)
    return np.where(np.abs(t) <= 2 * R, np.sinc(t / R) * 0.5 * (1.0 + np.cos(np.pi * t / (2 * R + 1))), 0.0)


def lpf_taps(R: int = DEFAULT_DECIM):
    """Zero-phase low-pass FIR for the envelope: 4R+1 taps, cutoff fs/(2R).

    h[j] = lpf_window(j - 2R), scaled to unit DC gain (sum h = 1).
    """
    t = np.arange(-2 * R, 2 * R + 1, dtype=np.float64)
    h = lpf_window(t, R)
    return h / np.sum(h)


def envelope_decimate(b, h, R: int = DEFAULT_DECIM):
    """E[d][i] = sum_{j=0}^{len(h)-1} h[j] |b_d|[R i + j - (len(h)-1)/2], |b| = 0 outside [0, N)."""
    env = np.abs(np.asarray(b))
    D, N = env.shape
    h = np.asarray(h, dtype=np.float64)
    half = (h.shape[0] - 1) // 2
    n_out = N // R
    ep = np.zeros((D, N + 2 * half + R))
    ep[:, half:half + N] = env
    E = np.zeros((D, n_out))
    for j in range(h.shape[0]):
        E += h[j] * ep[:, j:j + R * n_out:R]
    return E


def lpf_adjoint(G, h, R: int, n_samples: int):
    """Transpose of envelope_decimate's low-pass + subsampling (linear in |b|):
    G_env[d][n] = sum_i G[d][i] h[n - R i + half], n in [0, N)."""
    G = np.asarray(G, dtype=np.float64)
    h = np.asarray(h, dtype=np.float64)
    D, n_out = G.shape
    half = (h.shape[0] - 1) // 2
    out = np.zeros((D, n_samples + 2 * half + R))
    for j in range(h.shape[0]):
        out[:, j:j + R * n_out:R] += h[j] * G
    return out[:, half:half + n_samples]


def energyscape_vjp(x_int16, chirp, mic_xyz, dirs, fs: float, c: float, G, gain=None, delay_s=None,
                    R: int = DEFAULT_DECIM, h=None, band=DEFAULT_BAND, chunk: int = 32):
    """Time-domain energyscape E and the gradient of <G, E> with respect to the
    mic positions, gains and delays (hand-derived reverse pass, FP64).

    With t = n + delta_dm, I = sum_q w_q(mu) a[j+q] and I' = dI/dt:
      G_env = lpf_adjoint(G);  G_b = G_env b / |b|  (0 where b = 0)
      dL/d delta_dm = g_m sum_n Re(conj(G_b) I'),  dL/d g_m = sum_{d,n} Re(conj(G_b) I)
      dL/d Delta_m = fs sum_d dL/d delta_dm,  dL/d p_m = -(fs/c) sum_d dL/d delta_dm u_d
    Returns (E, grad_xyz [M][3], grad_gain [M], grad_delay [M] (per second)).
    """
    a = matched_filter(x_int16, chirp, fs, band)
    M, N = a.shape
    u = np.asarray(dirs, dtype=np.float64)
    D = u.shape[0]
    g = np.ones(M) if gain is None else np.asarray(gain, dtype=np.float64)
    delta = steering_delays(mic_xyz, dirs, fs, c, delay_s)
    h = lpf_taps(R) if h is None else np.asarray(h, dtype=np.float64)
    pad = int(math.ceil(np.max(np.abs(delta)))) + 4
    ap = _zero_padded(a, pad)
    n = np.arange(N, dtype=np.float64)
    b = np.zeros((D, N), dtype=np.complex128)
    for d0 in range(0, D, chunk):
        dd = delta[d0:d0 + chunk]
        for m in range(M):
            t = n[None, :] + dd[:, m:m + 1]
            j = np.floor(t)
            w = catmull_rom(t - j)
            idx = j.astype(np.int64) + pad
            b[d0:d0 + chunk] += g[m] * sum(w[q] * ap[m][idx + q - 1] for q in range(4))
    E = envelope_decimate(b, h, R)
    G_env = lpf_adjoint(G, h, R, N)
    mag = np.abs(b)
    G_b = np.where(mag > 0, G_env / np.where(mag > 0, mag, 1.0), 0.0) * b
    d_delta = np.zeros((D, M))
    grad_gain = np.zeros(M)
    for d0 in range(0, D, chunk):
        dd = delta[d0:d0 + chunk]
        gb = G_b[d0:d0 + chunk]
        for m in range(M):
            t = n[None, :] + dd[:, m:m + 1]
            j = np.floor(t)
            mu = t - j
            w = catmull_rom(mu)
            wd = catmull_rom_deriv(mu)
            idx = j.astype(np.int64) + pad
            taps = [ap[m][idx + q - 1] for q in range(4)]
            I = sum(w[q] * taps[q] for q in range(4))
            Id = sum(wd[q] * taps[q] for q in range(4))
            d_delta[d0:d0 + chunk, m] = g[m] * np.sum(np.real(np.conj(gb) * Id), axis=1)
            grad_gain[m] += np.sum(np.real(np.conj(gb) * I))
    grad_delay = fs * np.sum(d_delta, axis=0)
    grad_xyz = -(fs / c) * (d_delta.T @ u)
    return E, grad_xyz, grad_gain, grad_delay


def energyscape(x_int16, chirp, mic_xyz, dirs, fs: float, c: float, path: str = "td",
                R: int = DEFAULT_DECIM, gain=None, delay_s=None, band=DEFAULT_BAND, h=None,
                return_stages: bool = False, Q: int = DEFAULT_BB_DECIM):
    """Whole chain: int16 [M][N] -> energyscape E [D][floor(N/R)].
    path: "td" (steps 1-5 with das_td), "fd" (das_fd), "bb" (steps 6-8; Q, no h)."""
    N = np.asarray(x_int16).shape[1]
    delta = steering_delays(mic_xyz, dirs, fs, c, delay_s)
    h_given = h
    h = lpf_taps(R) if h is None else np.asarray(h, dtype=np.float64)
    if path == "td":
        a = matched_filter(x_int16, chirp, fs, band)
        b = das_td(a, delta, gain)
    elif path == "fd":
        A, k_lo, F = mf_spectrum(x_int16, chirp, fs, band)
        a = None
        b = das_fd(A, k_lo, F, N, delta, gain)
    elif path == "bb":
        a = matched_filter(x_int16, chirp, fs, band)
        F = fft_length(N, np.asarray(chirp).shape[0])
        k_c = baseband_centre_bin(*band_bins(F, fs, band))
        z = baseband_signal(a, k_c, F, Q)
        b = das_bb(z, delta, k_c, F, Q, gain)
        E = envelope_decimate_bb(b, N, R, Q, None if h_given is None else h)
        return (E, dict(a=a, z=z, b=b, delta=delta, k_c=k_c)) if return_stages else E
    else:
        raise ValueError(path)
    E = envelope_decimate(b, h, R)
    if return_stages:
        return E, dict(a=a, b=b, delta=delta, h=h)
    return E


# --------------------------------------------------------------------------
# complex-baseband delay-and-sum (subsampling moved behind the matched filter)
# --------------------------------------------------------------------------
def baseband_centre_bin(k_lo: int, k_hi: int) -> int:
    """k_c: the mid-band bin, floor((k_lo + k_hi) / 2); the band k_lo..k_hi maps to
    about +-30 kHz around 0 after demodulation by k_c."""
    return (int(k_lo) + int(k_hi)) // 2


def baseband_signal(a, k_c: int, F: int, Q: int = DEFAULT_BB_DECIM):
    """z_m[j] = a_m[Q j] exp(-j 2 pi k_c Q j / F) for j < ceil(N/Q).

    a is the full-rate analytic matched-filter output (complex [M][N]); the
    band-limited analytic signal demodulated to 0 Hz and kept every Q-th
    sample.  Nothing is filtered: a's spectrum is already confined to the band.
    """
    a = np.asarray(a, dtype=np.complex128)
    N = a.shape[1]
    j = np.arange((N + Q - 1) // Q, dtype=np.float64)
    return a[:, ::Q] * np.exp(-2j * np.pi * k_c * Q * j / F)[None, :]


def das_bb(z, delta, k_c: int, F: int, Q: int = DEFAULT_BB_DECIM, gain=None):
    """Baseband delay-and-sum on the coarse grid.

    b_d[j] = sum_m g_m exp(+j 2 pi k_c delta_dm / F) sum_{q=-1..2} w_q(mu) z_m[J+q]
    with u = j + delta_dm / Q, J = floor(u), mu = u - J (Catmull-Rom, as in
    das_td), z_m = 0 outside [0, Nb).  Since a_m(t) = z_m(t/Q) exp(+j 2 pi k_c t/F),
    |b_d[j]| approximates the full-rate |b_d[Q j]|: the envelope moves by the
    interpolated delay, the carrier by its exact phase.
    """
    z = np.asarray(z, dtype=np.complex128)
    delta = np.asarray(delta, dtype=np.float64)
    M, Nb = z.shape
    D = delta.shape[0]
    g = np.ones(M) if gain is None else np.asarray(gain, dtype=np.float64)
    dq = delta / Q
    rot = g[None, :] * np.exp(2j * np.pi * k_c * delta / F)            # [D][M]
    pad = int(math.ceil(np.max(np.abs(dq)))) + 4 if delta.size else 4
    zp = _zero_padded(z, pad)
    j = np.arange(Nb, dtype=np.float64)
    b = np.zeros((D, Nb), dtype=np.complex128)
    for m in range(M):
        u = j[None, :] + dq[:, m:m + 1]
        J = np.floor(u)
        w = catmull_rom(u - J)
        idx = J.astype(np.int64) + pad
        s = w[0] * zp[m][idx - 1] + w[1] * zp[m][idx] + w[2] * zp[m][idx + 1] + w[3] * zp[m][idx + 2]
        b += rot[:, m:m + 1] * s
    return b


def das_bb_bruteforce(z, delta, k_c: int, F: int, Q: int = DEFAULT_BB_DECIM, gain=None):
    """Triple loop over (d, j, m) of the das_bb definition (tiny inputs only)."""
    z = np.asarray(z, dtype=np.complex128)
    M, Nb = z.shape
    D = delta.shape[0]
    g = np.ones(M) if gain is None else gain
    b = np.zeros((D, Nb), dtype=np.complex128)
    for d in range(D):
        for j in range(Nb):
            acc = 0j
            for m in range(M):
                dl = float(delta[d][m])
                u = j + dl / Q
                J = math.floor(u)
                ws = catmull_rom(u - J)
                s = 0j
                for q, wq in zip((-1, 0, 1, 2), ws):
                    if 0 <= J + q < Nb:
                        s += float(wq) * z[m][J + q]
                acc += g[m] * complex(math.cos(2 * math.pi * k_c * dl / F), math.sin(2 * math.pi * k_c * dl / F)) * s
            b[d][j] = acc
    return b


def envelope_decimate_bb(b, n_samples: int, R: int = DEFAULT_DECIM, Q: int = DEFAULT_BB_DECIM, h=None):
    """E[d][i] = sum_j h_i(Q j - R i) |b_d[j]| for i < floor(N/R).

    b sits on the coarse grid (full-rate times Q j).  Output bin i keeps the
    full-rate position R i; its taps are the low-pass at the offsets
    t = Q j - R i inside its support, renormalised to sum 1 (unit DC gain, as
    lpf_taps): lpf_window(t, R) by default, or h[t + (len(h)-1)/2] for a given
    odd-length h.  |b| = 0 outside [0, Nb).  With Q = 1 this is envelope_decimate.
    """
    env = np.abs(np.asarray(b))
    D, Nb = env.shape
    half = 2 * R if h is None else (len(h) - 1) // 2
    n_out = n_samples // R
    E = np.zeros((D, n_out))
    for i in range(n_out):
        jlo = -((half - R * i) // Q)           # ceil((R i - half) / Q)
        jhi = (R * i + half) // Q
        jj = np.arange(jlo, jhi + 1)
        t = Q * jj - R * i
        w = lpf_window(t, R) if h is None else np.asarray(h, dtype=np.float64)[t + half]
        w = w / np.sum(w)
        ok = (jj >= 0) & (jj < Nb)
        E[:, i] = env[:, jj[ok]] @ w[ok]
    return E


# --------------------------------------------------------------------------
# PDM front end (Sec. 2: 1-bit sigma-delta microphones; Sec. 4.3: bit
# unpacking and a demodulating low-pass before the matched filter)
# --------------------------------------------------------------------------
def pdm_unpack(words, n_mics: int):
    """uint32 words [K] -> bits [n_mics][K] (0/1): bit m of word k is mic m's k-th bit."""
    w = np.asarray(words, dtype=np.uint64)
    return np.stack([((w >> np.uint64(m)) & np.uint64(1)).astype(np.int64) for m in range(n_mics)])


def cic_taps(decim: int = 10, order: int = 4):
    """Integer impulse response of an order-K CIC decimator: the length-D boxcar
    convolved with itself K times (length K (D - 1) + 1, sum D^K)."""
    h = np.ones(1, dtype=np.int64)
    for _ in range(order):
        h = np.convolve(h, np.ones(decim, dtype=np.int64))
    return h


def pdm_demodulate(bits, taps, decim: int, n_samples: int, shift: int = 0):
    """x_m[n] = sum_j g[j] b_m[D n + j - c] with b = 2 bits - 1 (0 outside [0, K)),
    c = (len(g) - 1) // 2, then (x + 2^(shift-1)) >> shift for shift > 0 (an
    arithmetic shift: rounds halves up), clamped to int16.  All integer."""
    b = 2 * np.asarray(bits, dtype=np.int64) - 1
    g = np.asarray(taps, dtype=np.int64)
    M, K = b.shape
    L = g.shape[0]
    c = (L - 1) // 2
    pad = np.zeros((M, K + decim * n_samples + 2 * L), dtype=np.int64)
    pad[:, L:L + K] = b
    x = np.zeros((M, n_samples), dtype=np.int64)
    idx = decim * np.arange(n_samples, dtype=np.int64) - c + L     # index of tap j = 0 in pad
    for j in range(L):
        x += g[j] * pad[:, idx + j]
    if shift > 0:
        x = (x + (1 << (shift - 1))) >> shift
    return np.clip(x, -32768, 32767).astype(np.int16)


# --------------------------------------------------------------------------
# frequency-domain beamforming as a batched complex GEMM
# --------------------------------------------------------------------------
def steering_matrix(freqs, mic_xyz, dirs, c: float, gain=None, delay_s=None):
    """W[k][d][m] = g_m exp(+j 2 pi f_k tau_dm), tau_dm = Delta_m - (p_m . u_d)/c."""
    tau = steering_delays(mic_xyz, dirs, 1.0, c, delay_s)            # seconds, [D][M]
    f = np.asarray(freqs, dtype=np.float64)
    M = tau.shape[1]
    g = np.ones(M) if gain is None else np.asarray(gain, dtype=np.float64)
    return g[None, None, :] * np.exp(2j * np.pi * f[:, None, None] * tau[None, :, :])


def fd_gemm(W, X):
    """Y[k][d][t] = sum_m W[k][d][m] X[k][m][t] (per-bin complex matrix product)."""
    return np.matmul(np.asarray(W, dtype=np.complex128), np.asarray(X, dtype=np.complex128))
