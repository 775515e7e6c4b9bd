"""Pythonic wrapper around one rtis_plan (device tensors in, device tensors out)."""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _native as nat

_PATHS = {"td": nat.RTIS_PATH_TD, "fd": nat.RTIS_PATH_FD, "bb": nat.RTIS_PATH_BB}
_PRECS = {"fp32": nat.RTIS_PREC_FP32, "bf16": nat.RTIS_PREC_BF16, "fp16": nat.RTIS_PREC_FP16}


class Plan:
    """A fixed configuration of the chain with its device buffers (allocated once).

    mic_xyz [M][3] (m), chirp [L], directions [D][3] (unit), n_samples N.
    """

    def __init__(self, mic_xyz, fs, chirp, directions, n_samples, *, c=343.0, decim=10, lpf_taps=None,
                 band=(20e3, 80e3), path="td", precision="fp32", max_delay_s=10e-6, position_slack_m=0.01,
                 max_batch=0, td_layout=None, bb_layout=None, grid="tile", fd_ifft="auto"):
        import torch  # device memory and streams only
        self._torch = torch
        o = nat.default_options()
        o.c = float(c)
        o.decim = int(decim)
        self._taps = None
        if lpf_taps is not None:
            self._taps = np.ascontiguousarray(lpf_taps, dtype=np.float32)
            o.lpf_len = int(self._taps.shape[0])
            o.lpf_taps = self._taps.ctypes.data_as(C.POINTER(C.c_float))
        o.band_lo_hz, o.band_hi_hz = float(band[0]), float(band[1])
        o.path = _PATHS[path]
        o.precision = _PRECS[precision]
        o.max_delay_s = float(max_delay_s)
        o.position_slack_m = float(position_slack_m)
        o.max_batch = int(max_batch)
        # beamformer stage layouts: None = autotuned at creation; an index forces that layout,
        # with one CTA per tile (grid="tile") or the resident CTAs looping (grid="persistent")
        o.td_layout = 0 if td_layout is None else int(td_layout) + 1
        o.bb_layout = 0 if bb_layout is None else int(bb_layout) + 1
        o.grid_mode = {"tile": 1, "persistent": 2}[grid]
        # process_many's frequency-domain inverse transform: "auto" (the faster form, today the FFT),
        # "fft" (FFT kernel on the FP32 pipe) or "tc" (dense DFT stages on the tensor cores, or fail)
        o.fd_ifft = {"auto": nat.RTIS_FD_IFFT_AUTO, "fft": nat.RTIS_FD_IFFT_FFT, "tc": nat.RTIS_FD_IFFT_TC}[fd_ifft]
        self.handle = nat.rtis_plan_create(mic_xyz, fs, chirp, directions, n_samples, o)
        self.info_path = path
        self.info = nat.rtis_plan_get_info(self.handle)
        self.M, self.N, self.D = self.info.n_mics, self.info.n_samples, self.info.n_dirs
        self.n_out = self.info.n_out
        self.Kb = self.info.k_hi - self.info.k_lo + 1

    # -- lifetime -----------------------------------------------------------
    def close(self):
        if getattr(self, "handle", None):
            nat.rtis_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- entry points -------------------------------------------------------
    def _dev(self):
        return self._torch.device("cuda", self._torch.cuda.current_device())

    def process(self, x, out=None, stream=None):
        """int16 [M][N] device tensor -> energyscape float32 [D][n_out]."""
        if out is None:
            out = self._torch.empty((self.D, self.n_out), dtype=self._torch.float32, device=x.device)
        nat.rtis_process(self.handle, x, out, stream)
        return out

    def process_many(self, x, paths=None, out_td=None, out_fd=None, stream=None):
        """int16 [n][M][N] device tensor -> energyscapes float32 [n][D][n_out].

        paths: None (the plan's own path, one tensor back) or a tuple of "td"/"fd"
        (a tuple of tensors back, one matched filter per measurement feeding both).
        The frequency-domain form runs the n measurements through one batched GEMM
        (n <= max_batch)."""
        t = self._torch
        n = int(x.shape[0])
        want = (self.info_path,) if paths is None else tuple(paths)
        if any(w not in ("td", "fd") for w in want):
            raise ValueError("process_many runs the time- and frequency-domain forms (paths 'td', 'fd')")
        shape = (n, self.D, self.n_out)
        if "td" in want and out_td is None:
            out_td = t.empty(shape, dtype=t.float32, device=x.device)
        if "fd" in want and out_fd is None:
            out_fd = t.empty(shape, dtype=t.float32, device=x.device)
        nat.rtis_process_many(self.handle, x.contiguous(), n, out_td if "td" in want else None,
                              out_fd if "fd" in want else None, stream)
        res = tuple(out_td if w == "td" else out_fd for w in want)
        return res[0] if paths is None else res

    def matched_filter(self, x, want_a=True, want_spectrum=False, stream=None):
        t = self._torch
        a = t.empty((self.M, self.N), dtype=t.complex64, device=x.device) if want_a else None
        A = t.empty((self.M, self.Kb), dtype=t.complex64, device=x.device) if want_spectrum else None
        nat.rtis_matched_filter(self.handle, x, a, A, stream)
        return a, A

    def beamform_td(self, a, out=None, stream=None):
        if out is None:
            out = self._torch.empty((self.D, self.n_out), dtype=self._torch.float32, device=a.device)
        nat.rtis_beamform_td(self.handle, a, out, stream)
        return out

    def beamform_fd(self, A, out=None, stream=None):
        """In-band spectra complex64 [M][Kb] (already / F) -> energyscape via the frequency-domain path."""
        if out is None:
            out = self._torch.empty((self.D, self.n_out), dtype=self._torch.float32, device=A.device)
        nat.rtis_beamform_fd(self.handle, A, out, stream)
        return out

    def baseband_signal(self, x, out=None, stream=None):
        """int16 [M][N] -> z complex64 [M][N/4]: the demodulated analytic signal on the coarse grid
        (plans created with path="bb")."""
        t = self._torch
        if out is None:
            out = t.empty((self.M, self.N // 4), dtype=t.complex64, device=x.device)
        nat.rtis_baseband_signal(self.handle, x, out, stream)
        return out

    def beamform_bb(self, z, out=None, stream=None):
        """z complex64 [M][N/4] (N/4 even) -> energyscape through the baseband delay-and-sum."""
        if out is None:
            out = self._torch.empty((self.D, self.n_out), dtype=self._torch.float32, device=z.device)
        nat.rtis_beamform_bb(self.handle, z, out, stream)
        return out

    def process_pdm(self, words, decim=10, taps=None, shift=0, out=None, stream=None):
        """PDM words (int32/uint32 device tensor [n_words], bit m = mic m) -> energyscape:
        rtis_pdm_demodulate into the plan's int16 input buffer, then process()."""
        t = self._torch
        if getattr(self, "_pdm_x", None) is None or self._pdm_x.device != words.device:
            self._pdm_x = t.empty((self.M, self.N), dtype=t.int16, device=words.device)
        pdm_demodulate(words, self.M, self.N, decim, taps, shift, out=self._pdm_x, stream=stream)
        return self.process(self._pdm_x, out=out, stream=stream)

    def set_calibration(self, mic_xyz=None, gain=None, delay_s=None, stream=None):
        """Device float tensors [M][3], [M], [M] (seconds); None keeps the current value."""
        t = self._torch
        c = lambda v: None if v is None else v.detach().to(t.float32).contiguous()
        mic_xyz, gain, delay_s = c(mic_xyz), c(gain), c(delay_s)
        nat.rtis_set_calibration(self.handle, mic_xyz, gain, delay_s, stream)
        self._keep = (mic_xyz, gain, delay_s)  # alive until the stream-ordered copies ran

    def backward(self, x, grad_out, stream=None):
        """dL/dE [D][n_out] -> (dL/dp [M][3], dL/dg [M], dL/dDelta [M]) for the time-domain path."""
        t = self._torch
        dev = x.device
        gx = t.empty((self.M, 3), dtype=t.float32, device=dev)
        gg = t.empty((self.M,), dtype=t.float32, device=dev)
        gd = t.empty((self.M,), dtype=t.float32, device=dev)
        nat.rtis_backward(self.handle, x, grad_out.contiguous(), gx, gg, gd, stream)
        return gx, gg, gd

    def steering_table(self, stream=None):
        t = self._torch
        dev = self._dev()
        shift = t.empty((self.D, self.M), dtype=t.int32, device=dev)
        weight = t.empty((self.D, self.M, 4), dtype=t.float32, device=dev)
        nat.rtis_steering_table(self.handle, shift, weight, stream)
        return shift, weight

    def sync(self) -> int:
        """Waits for the device; returns (and clears) the device status bits."""
        return nat.rtis_plan_sync(self.handle)

    def set_tracing(self, enable=True):
        """CUDA-event timing of the library's own launches in each later call (see trace())."""
        nat.rtis_plan_set_tracing(self.handle, enable)

    def trace(self):
        """The last traced call's kernel launches as [(kernel name, ms)], in launch order."""
        return nat.rtis_plan_get_trace(self.handle)


def pdm_demodulate(words, n_mics, n_samples, decim=10, taps=None, shift=0, out=None, stream=None):
    """PDM front end: words (int32 or uint32 device tensor [n_words], bit m of word k =
    mic m's k-th bit) -> int16 [n_mics][n_samples], the integer demodulating FIR
    (order-4 CIC when taps is None) at every `decim`-th bit."""
    import torch
    if out is None:
        out = torch.empty((n_mics, n_samples), dtype=torch.int16, device=words.device)
    g = None if taps is None else np.ascontiguousarray(taps, dtype=np.int32)
    nat.rtis_pdm_demodulate(words, int(words.numel()), n_mics, n_samples, decim, g, shift, out, stream)
    return out


class FdGemm:
    """Frequency-domain beamforming GEMM: Y[k][d][t] = sum_m W[k][d][m] X[k][m][t] on tcgen05."""

    def __init__(self, mic_xyz, directions, freqs_hz, n_frames, *, c=343.0, gain=None, delay_s=None,
                 precision="fp32"):
        import torch
        self._torch = torch
        self.handle = nat.rtis_fd_gemm_create(mic_xyz, directions, freqs_hz, n_frames, c, gain, delay_s,
                                              _PRECS[precision])
        self.K = len(freqs_hz)
        self.D = int(np.asarray(directions).shape[0])
        self.M = int(np.asarray(mic_xyz).shape[0])
        self.T = int(n_frames)

    def run(self, X, Y=None, stream=None):
        """X: complex64 [K][M][T] device tensor -> Y complex64 [K][D][T]."""
        if Y is None:
            Y = self._torch.empty((self.K, self.D, self.T), dtype=self._torch.complex64, device=X.device)
        nat.rtis_fd_gemm_run(self.handle, X, Y, stream)
        return Y

    def close(self):
        if getattr(self, "handle", None):
            nat.rtis_fd_gemm_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Batch:
    """Several plans processed together: one batched beamformer launch, autotuned on
    the first run and replayed from a CUDA graph afterwards."""

    def __init__(self, plans):
        import torch
        self._torch = torch
        self.plans = list(plans)
        self.handle = nat.rtis_batch_create([p.handle for p in self.plans])

    @property
    def info(self):
        return nat.rtis_batch_get_info(self.handle)

    def run(self, xs, outs=None, stream=None):
        t = self._torch
        if outs is None:
            outs = [t.empty((p.D, p.n_out), dtype=t.float32, device=x.device) for p, x in zip(self.plans, xs)]
        nat.rtis_batch_run(self.handle, list(xs), list(outs), stream)
        return outs

    def sync(self) -> int:
        return nat.rtis_batch_sync(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            nat.rtis_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def process_batch(plans, xs, outs=None, stream=None):
    """One-shot batched processing without a graph (allocates nothing in the library)."""
    import torch
    if outs is None:
        outs = [torch.empty((p.D, p.n_out), dtype=torch.float32, device=x.device) for p, x in zip(plans, xs)]
    nat.rtis_process_batch([p.handle for p in plans], list(xs), list(outs), stream)
    return outs


def _autograd_function():
    import torch

    class EnergyscapeFn(torch.autograd.Function):
        """E = energyscape(x; p, g, Delta) with the hand-written adjoint (rtis_backward)."""

        @staticmethod
        def forward(ctx, plan, x, mic_xyz, gain, delay_s):
            plan.set_calibration(mic_xyz, gain, delay_s)
            E = plan.process(x)
            ctx.plan = plan
            ctx.save_for_backward(x, mic_xyz, gain, delay_s)
            return E

        @staticmethod
        def backward(ctx, grad_E):
            x, mic_xyz, gain, delay_s = ctx.saved_tensors
            plan = ctx.plan
            plan.set_calibration(mic_xyz, gain, delay_s)
            gx, gg, gd = plan.backward(x, grad_E)
            return None, None, gx.to(mic_xyz.dtype), gg.to(gain.dtype), gd.to(delay_s.dtype)

    return EnergyscapeFn


_FN = None


def energyscape(plan, x, mic_xyz, gain, delay_s):
    """Differentiable time-domain energyscape with respect to the array calibration."""
    global _FN
    if _FN is None:
        _FN = _autograd_function()
    return _FN.apply(plan, x, mic_xyz, gain, delay_s)
