"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test ties one step of the oracle to a closed form, an invariant, brute
force, or an independent library routine, so that a dropped term, a sign
flip, a transposed operand or an off-by-one in it fails here.  CPU only.
"""
import math
import os

import numpy as np
import pytest
import scipy.signal

import oracle as orc
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
FS = synth.FS
C = synth.C_SOUND


def _short_chirp(L=40):
    n = np.arange(L)
    return np.hanning(L) * np.cos(2 * np.pi * (0.15 * n + 0.002 * n * n))


# -------------------------------------------------------------- sizes / band
def test_band_bins_golden():
    rows = [list(map(int, ln.split())) for ln in open(os.path.join(GOLDEN, "band_bins.txt"))
            if ln.strip() and not ln.startswith("#")]
    L = synth.chirp_length()
    assert L == 900
    for N, F, k_lo, k_hi, Kb, n_out in rows:
        assert orc.fft_length(N, L) == F
        assert orc.band_bins(F, FS) == (k_lo, k_hi)
        assert k_hi - k_lo + 1 == Kb
        assert N // orc.DEFAULT_DECIM == n_out


# -------------------------------------------------------------- matched filter
def test_mf_analytic_real_part_is_bruteforce_correlation():
    rng = np.random.default_rng(1)
    M, N, L = 2, 150, 40
    x = rng.integers(-3000, 3000, size=(M, N)).astype(np.int16)
    s = _short_chirp(L)
    a = orc.matched_filter(x, s, FS, mask="analytic")
    xf = x.astype(np.float64) / 32768.0
    F = orc.fft_length(N, L)
    for m in range(M):
        # circular correlation over F (no wrap for n < N since F >= N + L - 1)
        c_circ = np.zeros(F)
        for n in range(F):
            for l in range(L):
                j = (n + l) % F
                if j < N:
                    c_circ[n] += xf[m][j] * s[l]
        np.testing.assert_allclose(a[m].real, c_circ[:N], rtol=0, atol=1e-13)
        # imaginary part: the textbook analytic signal of the same sequence
        h = scipy.signal.hilbert(c_circ)
        np.testing.assert_allclose(a[m].imag, h.imag[:N], rtol=0, atol=1e-12)


def test_chirp_autocorrelation_peak_equals_energy():
    s_q = np.rint(synth.chirp() * 2 ** 14)
    N = 2048
    x = np.zeros((1, N), dtype=np.int16)
    x[0, :s_q.size] = s_q.astype(np.int16)
    s = s_q / 32768.0                        # the template equals the recorded sweep
    a = orc.matched_filter(x, s, FS, mask="analytic")
    energy = float(np.sum(s * s))
    assert abs(a[0, 0].real - energy) <= 1e-12 * energy
    # the analytic envelope peaks at lag 0 and |a[0]| >= its real part
    assert int(np.argmax(np.abs(a[0]))) == 0


@pytest.mark.parametrize("n0", [0, 1, 333, 1000])
def test_mf_band_alignment_integer_onset(n0):
    s = synth.chirp()
    N = 4096
    x = np.zeros((1, N), dtype=np.int16)
    x[0, n0:n0 + s.size] = np.rint(s * 20000).astype(np.int16)
    a = orc.matched_filter(x, s.astype(np.float32), FS)
    assert int(np.argmax(np.abs(a[0]))) == n0


def test_mf_band_limit_removes_out_of_band_tone():
    # a long Hann-windowed 150 kHz tone lies outside [20, 80] kHz: the banded
    # filter output is tiny while the unbanded one is not.
    N = 8192
    n = np.arange(N)
    tone = np.hanning(N) * np.cos(2 * np.pi * 150e3 / FS * n)
    x = np.rint(tone * 30000).astype(np.int16)[None, :]
    s = np.cos(2 * np.pi * 150e3 / FS * np.arange(64)) * np.hanning(64)
    a_band = orc.matched_filter(x, s, FS)
    a_full = orc.matched_filter(x, s, FS, mask="analytic")
    assert np.max(np.abs(a_band)) < 1e-6 * np.max(np.abs(a_full))


# -------------------------------------------------------------- interpolation
def test_catmull_rom_partition_identity_and_quadratics():
    mu = np.linspace(0, 1, 101)
    w = orc.catmull_rom(mu)
    np.testing.assert_allclose(sum(w), 1.0, atol=1e-15)
    w0 = orc.catmull_rom(0.0)
    assert [float(v) for v in w0] == [0.0, 1.0, 0.0, 0.0]
    w1 = orc.catmull_rom(1.0)
    assert [float(v) for v in w1] == [0.0, 0.0, 1.0, 0.0]
    j = 7
    for coeffs in ([2.0, 0, 0], [0.5, -3.0, 0], [1.0, 0.25, -0.75]):
        f = lambda t: coeffs[0] + coeffs[1] * t + coeffs[2] * t * t
        interp = sum(wq * f(j + q) for wq, q in zip(w, (-1, 0, 1, 2)))
        np.testing.assert_allclose(interp, f(j + mu), atol=1e-12)
    cubic = lambda t: t ** 3
    interp = sum(wq * cubic(j + q) for wq, q in zip(w, (-1, 0, 1, 2)))
    assert np.max(np.abs(interp - cubic(j + mu))) > 1e-3      # third order is not reproduced


# -------------------------------------------------------------- delay-and-sum
def test_das_td_vectorised_equals_bruteforce():
    rng = np.random.default_rng(7)
    M, N, D = 3, 48, 4
    a = rng.normal(size=(M, N)) + 1j * rng.normal(size=(M, N))
    delta = rng.uniform(-12, 12, size=(D, M))
    delta[0, 0] = -0.25          # reads before sample 0
    delta[1, 2] = 3.0            # exactly integer
    g = rng.uniform(0.5, 1.5, size=M)
    b_vec = orc.das_td(a, delta, g)
    b_bf = orc.das_td_bruteforce(a, delta, g)
    np.testing.assert_allclose(b_vec, b_bf, rtol=0, atol=1e-13)


def test_das_td_integer_delays_is_plain_shift():
    rng = np.random.default_rng(8)
    M, N, D = 4, 64, 3
    a = rng.normal(size=(M, N)) + 1j * rng.normal(size=(M, N))
    delta = rng.integers(-9, 9, size=(D, M)).astype(np.float64)
    b = orc.das_td(a, delta)
    ref = np.zeros((D, N), dtype=complex)
    for d in range(D):
        for m in range(M):
            s = int(delta[d, m])
            for n in range(N):
                if 0 <= n + s < N:
                    ref[d, n] += a[m, n + s]
    np.testing.assert_allclose(b, ref, atol=1e-13)


def test_steering_delays_sign_convention():
    # a mic displaced by +x sees a wave from +x (az = +90 deg) earlier by x/c:
    # it must be read later (positive n index shift is an advance -> negative delta)
    mic = np.array([[0.01, 0.0, 0.0]])
    u = synth.unit_vector(np.deg2rad([90.0, -90.0, 0.0]), np.zeros(3))
    d = orc.steering_delays(mic, u, FS, C)
    np.testing.assert_allclose(d[:, 0], [-FS * 0.01 / C, FS * 0.01 / C, 0.0], atol=1e-12)


def test_td_equals_fd_on_integer_delays():
    rng = np.random.default_rng(11)
    M, N, L = 3, 512, 40
    x = rng.integers(-20000, 20000, size=(M, N)).astype(np.int16)
    s = _short_chirp(L)
    fs = 450e3
    A, k_lo, F = orc.mf_spectrum(x, s, fs)
    a = orc.matched_filter(x, s, fs)
    delta = rng.integers(-20, 20, size=(5, M)).astype(np.float64)
    b_td = orc.das_td(a, delta)
    b_fd = orc.das_fd(A, k_lo, F, N, delta)
    lo = int(np.max(np.maximum(0, -delta)))
    hi = N - int(np.max(np.maximum(0, delta)))
    np.testing.assert_allclose(b_td[:, lo:hi], b_fd[:, lo:hi], rtol=0, atol=1e-12 * np.max(np.abs(b_td)))


def _plane_wave_case(n0=2000, M=8, N=4096, d_star=37):
    """Mics placed so the true direction has integer delays -k_m; echo onset n0 - k_m."""
    rng = np.random.default_rng(5)
    dirs = synth.azimuth_fan(91).astype(np.float64)
    u = dirs[d_star]
    perp = np.array([u[2], 0.0, -u[0]])                # in the horizontal plane, orthogonal to u
    k = rng.integers(-6, 7, size=M)
    mic = (k[:, None] * (C / FS)) * u[None, :] + rng.uniform(-0.05, 0.05, size=(M, 1)) * perp[None, :]
    mic += rng.uniform(-0.05, 0.05, size=(M, 1)) * np.array([0.0, 1.0, 0.0])[None, :]
    s = synth.chirp()
    sq = np.rint(s * 16000).astype(np.int16)
    x = np.zeros((M, N), dtype=np.int16)
    for m in range(M):
        x[m, n0 - k[m]:n0 - k[m] + s.size] = sq
    return x, s.astype(np.float32), mic, dirs, k


def test_plane_wave_point_reflector_peaks_exactly():
    n0, M, d_star = 2000, 8, 37
    x, s, mic, dirs, k = _plane_wave_case(n0, M, 4096, d_star)
    delta = orc.steering_delays(mic, dirs, FS, C)
    np.testing.assert_allclose(delta[d_star], -k, atol=1e-9)
    E = orc.energyscape(x, s, mic, dirs, FS, C)
    d_pk, i_pk = np.unravel_index(np.argmax(E), E.shape)
    assert d_pk == d_star
    assert i_pk == n0 // orc.DEFAULT_DECIM
    # coherent sum: the beam at the true direction is M times one channel's
    # matched-filter output (channel 0 shifted to onset n0)
    single = np.zeros((1, x.shape[1]), dtype=np.int16)
    single[0, n0:n0 + s.size] = x[0, n0 - k[0]:n0 - k[0] + s.size]
    a1 = orc.matched_filter(single, s, FS)
    E1 = orc.envelope_decimate(M * a1, orc.lpf_taps())
    np.testing.assert_allclose(E[d_star].max(), E1.max(), rtol=1e-12)


def test_spherical_scene_peak_near_truth():
    cfg = synth.single_sensor()
    E = orc.energyscape(cfg["x"], cfg["chirp"], cfg["mic_xyz"], cfg["dirs"], cfg["fs"], cfg["c"])
    sc = cfg["scene"]
    d_pk, i_pk = np.unravel_index(np.argmax(E), E.shape)
    az = np.deg2rad(np.linspace(-90, 90, 181))
    hits = []
    for q in range(sc.pos.shape[0]):
        r = sc.meta["range"][q]
        tof_bin = (2 * r / C) * FS / orc.DEFAULT_DECIM
        d_true = int(np.argmin(np.abs(az - sc.meta["az"][q])))
        hits.append(abs(i_pk - tof_bin) <= 1.5 and abs(d_pk - d_true) <= 2)
    assert any(hits)


# -------------------------------------------------------------- envelope / LPF
def test_lpf_unit_dc_gain_and_stopband():
    R = orc.DEFAULT_DECIM
    h = orc.lpf_taps(R)
    assert h.size == 4 * R + 1
    np.testing.assert_allclose(np.sum(h), 1.0, atol=1e-15)
    np.testing.assert_allclose(h, h[::-1], atol=0)
    # response at the first alias of the decimated rate, f = fs/R
    t = np.arange(-2 * R, 2 * R + 1)
    resp = abs(np.sum(h * np.exp(-2j * np.pi * t / R)))
    assert resp < 1e-2
    # a constant envelope passes unchanged away from the edges
    b = np.ones((1, 400), dtype=complex) * (3 + 4j)
    E = orc.envelope_decimate(b, h, R)
    np.testing.assert_allclose(E[0, 3:-3], 5.0, rtol=1e-14)
    # at i = 0 only the right half of the taps sees signal
    np.testing.assert_allclose(E[0, 0], 5.0 * np.sum(h[2 * R:]), rtol=1e-14)


def test_envelope_decimate_bruteforce():
    rng = np.random.default_rng(3)
    b = rng.normal(size=(2, 97)) + 1j * rng.normal(size=(2, 97))
    h = rng.uniform(size=9)
    R = 4
    E = orc.envelope_decimate(b, h, R)
    assert E.shape == (2, 97 // R)
    for d in range(2):
        for i in range(97 // R):
            acc = 0.0
            for j in range(9):
                n = R * i + j - 4
                if 0 <= n < 97:
                    acc += h[j] * abs(b[d, n])
            assert abs(E[d, i] - acc) < 1e-13


# -------------------------------------------------------------- FD GEMM
def test_steering_matrix_focuses_plane_wave_to_gain_M():
    mic = synth.mic_array(0).astype(np.float64)
    dirs = synth.fibonacci_hemisphere(64).astype(np.float64)
    f = np.array([20e3, 47e3, 80e3])
    W = orc.steering_matrix(f, mic, dirs, C)
    d_star = 21
    # plane wave from u*: mic m is advanced by (p_m . u*)/c -> phase +2 pi f (p.u)/c
    X = np.exp(2j * np.pi * f[:, None] * (mic @ dirs[d_star])[None, :] / C)[:, :, None]
    Y = orc.fd_gemm(W, X)[:, :, 0]
    M = mic.shape[0]
    np.testing.assert_allclose(Y[:, d_star], M, atol=1e-10)
    assert np.all(np.abs(Y) <= M + 1e-9)
    assert np.all(np.argmax(np.abs(Y), axis=1) == d_star)


def test_fd_gemm_bruteforce():
    rng = np.random.default_rng(4)
    K, D, M, T = 3, 5, 4, 2
    W = rng.normal(size=(K, D, M)) + 1j * rng.normal(size=(K, D, M))
    X = rng.normal(size=(K, M, T)) + 1j * rng.normal(size=(K, M, T))
    Y = orc.fd_gemm(W, X)
    for k in range(K):
        for d in range(D):
            for t in range(T):
                acc = 0j
                for m in range(M):
                    acc += W[k, d, m] * X[k, m, t]
                assert abs(Y[k, d, t] - acc) < 1e-12


# -------------------------------------------------------------- adjoint
def test_lpf_adjoint_dot_product():
    rng = np.random.default_rng(12)
    R, N = 7, 301
    h = rng.normal(size=29)
    b = rng.normal(size=(3, N))          # a nonnegative "envelope" is not needed: the map is linear in |b|
    env = np.abs(b)
    G = rng.normal(size=(3, N // R))
    lhs = np.sum(orc.envelope_decimate(env, h, R) * G)
    rhs = np.sum(env * orc.lpf_adjoint(G, h, R, N))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_catmull_rom_derivative_matches_difference():
    mu = np.linspace(0.02, 0.98, 25)
    eps = 1e-6
    for wq, dq in zip(zip(*[orc.catmull_rom(mu + s) for s in (eps, -eps)]), orc.catmull_rom_deriv(mu)):
        np.testing.assert_allclose((wq[0] - wq[1]) / (2 * eps), dq, atol=1e-8)


def _tiny_calibration_case():
    rng = np.random.default_rng(21)
    M, N, D = 4, 600, 5
    s = synth.chirp()[:200]
    mic = rng.uniform(-0.05, 0.05, size=(M, 3))
    mic[:, 2] = 0.0
    dirs = synth.fibonacci_hemisphere(D).astype(np.float64)
    x = np.zeros((M, N), dtype=np.int16)
    for m in range(M):
        x[m, 150 + 3 * m:150 + 3 * m + s.size] = np.rint(s * 12000).astype(np.int16)
    x = (x + rng.integers(-300, 300, size=(M, N))).astype(np.int16)
    gain = rng.uniform(0.8, 1.2, size=M)
    delay = rng.uniform(-2e-6, 2e-6, size=M)
    G = rng.normal(size=(D, N // orc.DEFAULT_DECIM))
    return x, s, mic, dirs, gain, delay, G


def test_adjoint_matches_central_differences():
    x, s, mic, dirs, gain, delay, G = _tiny_calibration_case()
    fs, c = synth.FS, synth.C_SOUND
    E, gx, gg, gd = orc.energyscape_vjp(x, s, mic, dirs, fs, c, G, gain, delay)
    np.testing.assert_allclose(E, orc.energyscape(x, s, mic, dirs, fs, c, gain=gain, delay_s=delay), rtol=1e-12)
    loss = lambda mic_, g_, d_: np.sum(G * orc.energyscape(x, s, mic_, dirs, fs, c, gain=g_, delay_s=d_))
    for m in (0, 3):
        for k in range(3):
            hstep = 1e-7
            mp, mm = mic.copy(), mic.copy()
            mp[m, k] += hstep
            mm[m, k] -= hstep
            fd = (loss(mp, gain, delay) - loss(mm, gain, delay)) / (2 * hstep)
            assert abs(fd - gx[m, k]) <= 1e-5 * (abs(gx[m, k]) + 1e-3 * np.max(np.abs(gx)))
        hstep = 1e-6
        gp, gm = gain.copy(), gain.copy()
        gp[m] += hstep
        gm[m] -= hstep
        fd = (loss(mic, gp, delay) - loss(mic, gm, delay)) / (2 * hstep)
        assert abs(fd - gg[m]) <= 1e-6 * abs(gg[m]) + 1e-9
        hstep = 1e-9
        dp, dm = delay.copy(), delay.copy()
        dp[m] += hstep
        dm[m] -= hstep
        fd = (loss(mic, gain, dp) - loss(mic, gain, dm)) / (2 * hstep)
        assert abs(fd - gd[m]) <= 1e-5 * (abs(gd[m]) + 1e-3 * np.max(np.abs(gd)))


def test_adjoint_gain_gradient_is_exact_for_linear_scaling():
    # E is positively homogeneous in the common gain: sum_m g_m dE/dg_m = E, so
    # <G, E> = sum_m g_m dL/dg_m
    x, s, mic, dirs, gain, delay, G = _tiny_calibration_case()
    E, gx, gg, gd = orc.energyscape_vjp(x, s, mic, dirs, synth.FS, synth.C_SOUND, G, gain, delay)
    np.testing.assert_allclose(np.sum(gain * gg), np.sum(G * E), rtol=1e-10)


# -------------------------------------------------------------- complex baseband
def _tiny_mf_case(seed=21, M=2, N=103, L=40):
    rng = np.random.default_rng(seed)
    x = rng.integers(-20000, 20000, size=(M, N)).astype(np.int16)
    return x, _short_chirp(L), 450e3


def test_baseband_signal_is_the_shifted_band_sum():
    # z_m[j] written as the inverse DFT of the in-band spectrum moved down by k_c and
    # read at the coarse times Q j: an explicit double loop, no FFT and no matched_filter
    x, s, fs = _tiny_mf_case()
    A, k_lo, F = orc.mf_spectrum(x, s, fs)
    k_hi = k_lo + A.shape[1] - 1
    k_c = orc.baseband_centre_bin(k_lo, k_hi)
    assert k_c == (k_lo + k_hi) // 2
    for Q in (1, 2, 4):
        z = orc.baseband_signal(orc.matched_filter(x, s, fs), k_c, F, Q)
        Nb = (x.shape[1] + Q - 1) // Q
        assert z.shape == (2, Nb)
        ref = np.zeros_like(z)
        for m in range(2):
            for j in range(Nb):
                acc = 0j
                for kk in range(A.shape[1]):
                    kap = k_lo + kk - k_c
                    acc += A[m, kk] * complex(math.cos(2 * math.pi * kap * Q * j / F),
                                              math.sin(2 * math.pi * kap * Q * j / F))
                ref[m, j] = acc / F
        np.testing.assert_allclose(z, ref, rtol=0, atol=1e-12 * np.max(np.abs(ref)))


def test_das_bb_vectorised_equals_bruteforce():
    rng = np.random.default_rng(22)
    M, Nb, D, Q, F, k_c = 3, 40, 4, 4, 1024, 113
    z = rng.normal(size=(M, Nb)) + 1j * rng.normal(size=(M, Nb))
    delta = rng.uniform(-30, 30, size=(D, M))
    delta[0, 0] = -0.5           # reads before sample 0
    delta[1, 2] = 8.0            # a whole number of coarse samples
    delta[2, 1] = 3.0            # whole on the fine grid only
    g = rng.uniform(0.5, 1.5, size=M)
    np.testing.assert_allclose(orc.das_bb(z, delta, k_c, F, Q, g), orc.das_bb_bruteforce(z, delta, k_c, F, Q, g),
                               rtol=0, atol=1e-13)


def test_das_bb_on_whole_coarse_delays_is_the_full_rate_beam():
    # delta = Q J exactly: interpolation is the identity and the carrier phase
    # exp(+j 2 pi k_c Q J / F) puts back what demodulation took out, so
    # b_bb[j] exp(+j 2 pi k_c Q j / F) equals the full-rate beam at n = Q j
    x, s, fs = _tiny_mf_case(seed=23, M=3, N=257)
    a = orc.matched_filter(x, s, fs)
    F = orc.fft_length(x.shape[1], s.size)
    k_lo, k_hi = orc.band_bins(F, fs)
    k_c = orc.baseband_centre_bin(k_lo, k_hi)
    rng = np.random.default_rng(24)
    for Q in (2, 4):
        delta = (Q * rng.integers(-9, 10, size=(5, 3))).astype(np.float64)
        g = rng.uniform(0.5, 1.5, size=3)
        b_td = orc.das_td(a, delta, g)
        b_bb = orc.das_bb(orc.baseband_signal(a, k_c, F, Q), delta, k_c, F, Q, g)
        j = np.arange(b_bb.shape[1])
        np.testing.assert_allclose(b_bb * np.exp(2j * np.pi * k_c * Q * j / F)[None, :], b_td[:, ::Q],
                                   rtol=0, atol=1e-12 * np.max(np.abs(b_td)))


def test_envelope_decimate_bb_with_q1_is_envelope_decimate():
    rng = np.random.default_rng(25)
    b = rng.normal(size=(3, 203)) + 1j * rng.normal(size=(3, 203))
    for R in (7, 10):
        np.testing.assert_allclose(orc.envelope_decimate_bb(b, 203, R, 1),
                                   orc.envelope_decimate(b, orc.lpf_taps(R), R), rtol=0, atol=1e-14)
    # given taps (any odd length, unnormalised) are read at the offsets and renormalised
    h = rng.uniform(0.1, 1.0, size=9)
    np.testing.assert_allclose(orc.envelope_decimate_bb(b, 203, 5, 1, h),
                               orc.envelope_decimate(b, h / h.sum(), 5), rtol=0, atol=1e-14)
    np.testing.assert_allclose(orc.envelope_decimate_bb(b, 203, 10, 4, orc.lpf_taps(10)),
                               orc.envelope_decimate_bb(b, 203, 10, 4), rtol=0, atol=1e-14)


@pytest.mark.parametrize("R,Q", [(10, 4), (6, 4), (8, 4), (10, 2), (7, 4)])
def test_envelope_decimate_bb_constant_and_ramp(R, Q):
    # unit DC gain per output bin; and where every bin's coarse offsets Q j - R i
    # are symmetric about 0 (R i = 0 or Q/2 mod Q for all i, i.e. Q divides 2R)
    # a linear envelope comes back exactly at the bin's full-rate time R i
    N = 1000
    Nb = (N + Q - 1) // Q
    n_out = N // R
    interior = slice(3, n_out - 3)
    E = orc.envelope_decimate_bb(np.full((1, Nb), 2.5 + 0j), N, R, Q)
    np.testing.assert_allclose(E[0, interior], 2.5, rtol=1e-14)
    E = orc.envelope_decimate_bb((Q * np.arange(Nb, dtype=float))[None, :] + 0j, N, R, Q)
    i = np.arange(n_out)
    if (2 * R) % Q == 0:
        np.testing.assert_allclose(E[0, interior], (R * i)[interior], rtol=1e-13)
    else:  # offsets not symmetric: the ramp is shifted by less than Q/2 full-rate samples
        assert np.max(np.abs(E[0, interior] - (R * i)[interior])) < Q / 2


def test_baseband_energyscape_tracks_exact_delays():
    # the baseband chain against the exact-delay (frequency-domain) energyscape:
    # same peak, and within 1% of the peak everywhere (its interpolation and
    # coarse-envelope error; the full-rate Catmull-Rom chain is at the same level)
    n0, M, d_star = 2000, 8, 37
    x, s, mic, dirs, k = _plane_wave_case(n0, M, 4096, d_star)
    E_bb = orc.energyscape(x, s, mic, dirs, FS, C, path="bb")
    E_fd = orc.energyscape(x, s, mic, dirs, FS, C, path="fd")
    assert E_bb.shape == E_fd.shape
    d_pk, i_pk = np.unravel_index(np.argmax(E_bb), E_bb.shape)
    assert (d_pk, i_pk) == (d_star, n0 // orc.DEFAULT_DECIM)
    assert np.max(np.abs(E_bb - E_fd)) < 1e-2 * E_fd.max()
    cfg = synth.single_sensor()
    E_bb = orc.energyscape(cfg["x"], cfg["chirp"], cfg["mic_xyz"], cfg["dirs"], FS, C, path="bb")
    E_fd = orc.energyscape(cfg["x"], cfg["chirp"], cfg["mic_xyz"], cfg["dirs"], FS, C, path="fd")
    assert np.unravel_index(np.argmax(E_bb), E_bb.shape) == np.unravel_index(np.argmax(E_fd), E_fd.shape)
    assert np.max(np.abs(E_bb - E_fd)) < 1e-2 * E_fd.max()


# -------------------------------------------------------------- PDM front end
def test_pdm_unpack_bruteforce_and_pack_roundtrip():
    rng = np.random.default_rng(31)
    words = rng.integers(0, 2 ** 32, size=57, dtype=np.uint64).astype(np.uint32)
    for M in (1, 5, 32):
        bits = orc.pdm_unpack(words, M)
        assert bits.shape == (M, 57)
        for m in range(M):
            for k in range(57):
                assert bits[m, k] == (int(words[k]) >> m) & 1
    bits = rng.integers(0, 2, size=(7, 40))
    packed = np.array([sum(int(bits[m, k]) << m for m in range(7)) for k in range(40)], dtype=np.uint32)
    np.testing.assert_array_equal(synth.pdm_pack(bits), packed)
    np.testing.assert_array_equal(orc.pdm_unpack(packed, 7), bits)


def test_cic_taps_are_the_recursive_cic_impulse_response():
    for D, K in ((10, 4), (8, 3), (4, 1)):
        h = orc.cic_taps(D, K)
        assert h.shape == (K * (D - 1) + 1,) and h.sum() == D ** K
        np.testing.assert_array_equal(h, h[::-1])
        x = np.zeros(200, dtype=np.int64)
        x[0] = 1
        for _ in range(K):                   # integrators
            x = np.cumsum(x)
        for _ in range(K):                   # combs with lag D (not decimated)
            x = x - np.concatenate([np.zeros(D, dtype=np.int64), x[:-D]])
        np.testing.assert_array_equal(x[:h.size], h)
        assert not x[h.size:].any()


def test_pdm_demodulate_is_the_decimated_recursive_cic():
    # integrators at the bit rate, sampled every D bits at the phase the centred
    # FIR implies (x[n] = f[D n + L - 1 - c] for the causal FIR f), combs at the low rate
    rng = np.random.default_rng(32)
    D, K, M, n_out = 10, 4, 3, 150
    bits = rng.integers(0, 2, size=(M, 1400))
    g = orc.cic_taps(D, K)
    L, c = g.size, (g.size - 1) // 2
    x = orc.pdm_demodulate(bits, g, D, n_out)
    b = np.zeros((M, D * n_out + 2 * L), dtype=np.int64)
    b[:, :1400] = 2 * bits - 1
    I = b.copy()
    for _ in range(K):
        I = np.cumsum(I, axis=1)
    n = np.arange(-K, n_out)
    t = D * n + L - 1 - c
    Is = np.where(t >= 0, I[:, np.clip(t, 0, None)], 0)
    for _ in range(K):
        Is = Is[:, 1:] - Is[:, :-1]
    np.testing.assert_array_equal(x, Is.astype(np.int16))


def test_pdm_demodulate_patterns_and_rounding():
    g = orc.cic_taps(10, 4)
    ones = np.ones((2, 3000), dtype=np.int64)
    x = orc.pdm_demodulate(ones, g, 10, 300)
    assert np.all(x[:, 2:-2] == 10000)                  # full scale +1
    assert np.all(orc.pdm_demodulate(0 * ones, g, 10, 300)[:, 2:-2] == -10000)
    alt = np.tile([1, 0], (1, 1500))
    assert np.all(orc.pdm_demodulate(alt, g, 10, 300)[:, 2:-2] == 0)   # nulled by the even boxcar
    # rounding right shift: (x + 2^(s-1)) >> s, halves go up (towards +inf)
    taps = np.array([1, 2, 1])
    bits = np.array([[1, 1, 0, 0, 1, 0, 1, 1, 1, 0]])
    raw = orc.pdm_demodulate(bits, taps, 1, 10).astype(np.int64)
    b = np.concatenate([[0], 2 * bits[0] - 1, [0]])
    np.testing.assert_array_equal(raw[0], [b[n] + 2 * b[n + 1] + b[n + 2] for n in range(10)])
    for s in (1, 2):
        got = orc.pdm_demodulate(bits, taps, 1, 10, shift=s).astype(np.int64)
        np.testing.assert_array_equal(got[0], [math.floor(v / 2 ** s + 0.5) for v in raw[0]])


def test_sigma_delta_tone_through_the_cic_demodulator():
    # a 0.5 full-scale 50 kHz tone: the demodulated amplitude is the CIC's gain at
    # 50 kHz (sin(pi f D/fb) / (D sin(pi f/fb)))^4 x 0.5 x 10^4, and the in-band noise
    # of the second-order modulator at 10x oversampling stays 45 dB below
    D = synth.PDM_DECIM
    fb = synth.FS * D
    K = 4096 * D
    u = 0.5 * np.sin(2 * np.pi * 50e3 * np.arange(K) / fb)[None, :]
    x = orc.pdm_demodulate(synth.sigma_delta2(u), orc.cic_taps(D, 4), D, 4096).astype(np.float64)[0]
    n = np.arange(4096)[100:-100]
    w = 2 * np.pi * 50e3 / synth.FS
    A = np.stack([np.sin(w * n), np.cos(w * n)], 1)
    coef, *_ = np.linalg.lstsq(A, x[100:-100], rcond=None)
    gain = (math.sin(math.pi * 50e3 * D / fb) / (D * math.sin(math.pi * 50e3 / fb))) ** 4
    assert abs(np.hypot(*coef) / (0.5 * 1e4 * gain) - 1) < 0.01
    res = x[100:-100] - A @ coef
    R = np.fft.rfft(res)
    f = np.fft.rfftfreq(res.size, 1 / synth.FS)
    inb = (f >= 20e3) & (f <= 80e3)
    snr = 10 * np.log10((np.hypot(*coef) ** 2 / 2 * res.size) / (2 * np.sum(np.abs(R[inb]) ** 2) / res.size))
    assert snr > 45


@pytest.mark.parametrize("seed", range(4))
def test_envelope_decimate_bb_bruteforce(seed):
    # the coarse-grid low-pass written as a loop over output bins and full-rate offsets t:
    # taps where Q divides t + R i, renormalised over the taps that exist
    rng = np.random.default_rng(40 + seed)
    Q = int(rng.choice([2, 4]))
    R = int(rng.integers(1, 13))
    N = int(rng.integers(40, 300)) * Q
    Nb = N // Q
    b = rng.normal(size=(2, Nb)) + 1j * rng.normal(size=(2, Nb))
    L = 2 * int(rng.integers(0, 9)) + 1
    h = rng.uniform(0.1, 1.0, size=L)
    half = (L - 1) // 2
    E = orc.envelope_decimate_bb(b, N, R, Q, h)
    for d in range(2):
        for i in range(N // R):
            num = den = 0.0
            for t in range(-half, half + 1):
                if (R * i + t) % Q == 0:
                    j = (R * i + t) // Q
                    den += h[t + half]
                    if 0 <= j < Nb:
                        num += h[t + half] * abs(b[d, j])
            assert abs(E[d, i] - num / den) <= 1e-12 * max(1.0, abs(num / den))


@pytest.mark.parametrize("seed", range(4))
def test_pdm_demodulate_bruteforce(seed):
    # random words, taps (including negative), decimation and shift against a plain loop
    rng = np.random.default_rng(50 + seed)
    M = int(rng.integers(1, 6))
    D = int(rng.integers(1, 9))
    N = int(rng.integers(1, 40))
    K = N * D - int(rng.integers(0, D + 1))
    bits = rng.integers(0, 2, size=(M, K))
    L = int(rng.integers(1, 12))
    g = rng.integers(-50, 200, size=L)
    shift = int(rng.integers(0, 4))
    x = orc.pdm_demodulate(bits, g, D, N, shift)
    c = (L - 1) // 2
    for m in range(M):
        for n in range(N):
            acc = 0
            for j in range(L):
                k = D * n + j - c
                if 0 <= k < K:
                    acc += int(g[j]) * (2 * int(bits[m, k]) - 1)
            if shift:
                acc = (acc + (1 << (shift - 1))) >> shift
            assert x[m, n] == max(-32768, min(32767, acc))
