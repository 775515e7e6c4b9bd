"""ctypes binding of the C ABI in include/rtis.h (librtis.so).

Argument marshalling only: every step of the energyscape chain runs in the
library's CUDA kernels.  PyTorch supplies device memory and streams; tensors
are passed by ``data_ptr()``.  There is no CPU fallback: if the library is
missing, :func:`lib` raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "librtis.so")

RTIS_OK = 0
RTIS_ERR_INVALID_ARG = 1
RTIS_ERR_CUDA = 2
RTIS_ERR_OOM = 3
RTIS_ERR_UNSUPPORTED = 4
RTIS_ERR_TIMEOUT = 5
RTIS_ERR_NONFINITE = 6
RTIS_ERR_DEVICE = 7
RTIS_ERR_BUSY = 8
RTIS_DEV_DELAY_RANGE = 0x1
RTIS_DEV_TIMEOUT = 0x2
RTIS_DEV_NONFINITE = 0x4
RTIS_PATH_TD, RTIS_PATH_FD, RTIS_PATH_BB = 0, 1, 2
RTIS_PREC_FP32, RTIS_PREC_BF16, RTIS_PREC_FP16 = 0, 1, 2
RTIS_FD_IFFT_AUTO, RTIS_FD_IFFT_FFT, RTIS_FD_IFFT_TC = 0, 1, 2


class rtis_options(C.Structure):
    _fields_ = [
        ("c", C.c_double),
        ("decim", C.c_int),
        ("lpf_len", C.c_int),
        ("lpf_taps", C.POINTER(C.c_float)),
        ("band_lo_hz", C.c_double),
        ("band_hi_hz", C.c_double),
        ("path", C.c_int),
        ("precision", C.c_int),
        ("max_delay_s", C.c_double),
        ("position_slack_m", C.c_double),
        ("max_batch", C.c_int),
        ("td_layout", C.c_int),
        ("bb_layout", C.c_int),
        ("grid_mode", C.c_int),
        ("fd_ifft", C.c_int),
    ]


class rtis_plan_info(C.Structure):
    _fields_ = [
        ("n_mics", C.c_int), ("n_samples", C.c_int), ("n_dirs", C.c_int), ("chirp_len", C.c_int),
        ("fft_len", C.c_int), ("k_lo", C.c_int), ("k_hi", C.c_int),
        ("decim", C.c_int), ("lpf_len", C.c_int), ("n_out", C.c_int),
        ("halo", C.c_int), ("max_shift", C.c_int), ("workspace_bytes", C.c_size_t),
        ("td_variant", C.c_int), ("td_grid", C.c_int), ("td_tuned_ms", C.c_float),
        ("n_coarse", C.c_int), ("k_c", C.c_int), ("bb_variant", C.c_int), ("bb_grid", C.c_int),
        ("bb_tuned_ms", C.c_float), ("td_layout_ms", C.c_float * 16), ("bb_layout_ms", C.c_float * 16),
        ("fd_ifft", C.c_int),
    ]


class rtis_batch_info(C.Structure):
    _fields_ = [("n_sensors", C.c_int), ("total_tiles", C.c_int), ("tuned", C.c_int), ("variant", C.c_int),
                ("grid", C.c_int), ("tuned_ms", C.c_float)]


class rtis_trace_entry(C.Structure):
    _fields_ = [("kernel", C.c_int), ("index", C.c_int), ("ms", C.c_float)]


# rtis_kernel_id (include/rtis.h): the kernels a traced call can launch
KERNEL_NAMES = {1: "steering_table", 2: "mf_forward", 3: "mf_inverse", 4: "td_beamform", 5: "fd_gemm",
                6: "fd_energyscape", 7: "bb_beamform", 8: "adjoint"}
TRACE_MAX = 32


class RtisError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__(f"{where}: status {status} ({message})")
        self.status = status


_VP = C.c_void_p
_PROTOS = {
    "rtis_options_default": (None, [C.POINTER(rtis_options)]),
    "rtis_plan_create": (C.c_int, [C.POINTER(_VP), C.POINTER(C.c_float), C.c_int, C.c_double, C.POINTER(C.c_float),
                                   C.c_int, C.POINTER(C.c_float), C.c_int, C.c_int, C.POINTER(rtis_options)]),
    "rtis_plan_destroy": (None, [_VP]),
    "rtis_plan_get_info": (C.c_int, [_VP, C.POINTER(rtis_plan_info)]),
    "rtis_process": (C.c_int, [_VP, _VP, _VP, _VP]),
    "rtis_process_many": (C.c_int, [_VP, _VP, C.c_int, _VP, _VP, _VP]),
    "rtis_matched_filter": (C.c_int, [_VP, _VP, _VP, _VP, _VP]),
    "rtis_beamform_td": (C.c_int, [_VP, _VP, _VP, _VP]),
    "rtis_beamform_fd": (C.c_int, [_VP, _VP, _VP, _VP]),
    "rtis_baseband_signal": (C.c_int, [_VP, _VP, _VP, _VP]),
    "rtis_pdm_demodulate": (C.c_int, [_VP, C.c_longlong, C.c_int, C.c_int, C.c_int, _VP, C.c_int, C.c_int, _VP,
                                      _VP]),
    "rtis_beamform_bb": (C.c_int, [_VP, _VP, _VP, _VP]),
    "rtis_steering_table": (C.c_int, [_VP, _VP, _VP, _VP]),
    "rtis_plan_sync": (C.c_int, [_VP, C.POINTER(C.c_uint)]),
    "rtis_set_calibration": (C.c_int, [_VP, _VP, _VP, _VP, _VP]),
    "rtis_backward": (C.c_int, [_VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "rtis_loss_l2": (C.c_int, [_VP, _VP, _VP, _VP, _VP, _VP]),
    "rtis_baseline_create": (C.c_int, [C.POINTER(_VP), _VP]),
    "rtis_baseline_process": (C.c_int, [_VP, _VP, _VP, _VP]),
    "rtis_baseline_destroy": (None, [_VP]),
    "rtis_stream_create": (C.c_int, [C.POINTER(_VP), _VP, C.c_int]),
    "rtis_stream_submit": (C.c_int, [_VP, _VP, _VP, C.POINTER(C.c_int64)]),
    "rtis_stream_wait": (C.c_int, [_VP, C.c_int64, C.c_int]),
    "rtis_stream_destroy": (None, [_VP]),
    "rtis_matched_filter_noalloc": (C.c_int, [_VP, C.c_int, C.c_int, _VP, C.c_int, C.c_double, C.c_double,
                                              C.c_double, _VP, _VP, _VP]),
    "rtis_fd_gemm_create": (C.c_int, [C.POINTER(_VP), C.POINTER(C.c_float), C.c_int, C.POINTER(C.c_float), C.c_int,
                                      C.POINTER(C.c_double), C.c_int, C.c_int, C.c_double, C.POINTER(C.c_float),
                                      C.POINTER(C.c_float), C.c_int]),
    "rtis_fd_gemm_run": (C.c_int, [_VP, _VP, _VP, _VP]),
    "rtis_fd_gemm_destroy": (None, [_VP]),
    "rtis_process_batch": (C.c_int, [C.POINTER(_VP), C.c_int, C.POINTER(_VP), C.POINTER(_VP), _VP]),
    "rtis_batch_create": (C.c_int, [C.POINTER(_VP), C.POINTER(_VP), C.c_int]),
    "rtis_batch_run": (C.c_int, [_VP, C.POINTER(_VP), C.POINTER(_VP), _VP]),
    "rtis_batch_get_info": (C.c_int, [_VP, C.POINTER(rtis_batch_info)]),
    "rtis_batch_sync": (C.c_int, [_VP, C.POINTER(C.c_uint)]),
    "rtis_batch_destroy": (None, [_VP]),
    "rtis_plan_set_tracing": (C.c_int, [_VP, C.c_int]),
    "rtis_plan_get_trace": (C.c_int, [_VP, C.POINTER(rtis_trace_entry), C.c_int, C.POINTER(C.c_int)]),
    "rtis_status_string": (C.c_char_p, [C.c_int]),
    "rtis_last_error": (C.c_char_p, []),
}

_lib = None


def lib():
    """The loaded librtis.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"librtis.so not built ({LIB_PATH}); run paper_2208_10839_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _PROTOS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def last_error() -> str:
    return lib().rtis_last_error().decode()


def check(status: int, where: str):
    if status != RTIS_OK:
        raise RtisError(status, where, last_error())


def _fptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_float))


def ptr(t) -> int | None:
    """Device address of a tensor (or an int address, or None)."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def stream_handle(stream=None) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def default_options() -> rtis_options:
    o = rtis_options()
    lib().rtis_options_default(C.byref(o))
    return o


def rtis_plan_create(mic_xyz, fs, chirp, directions, n_samples, options: rtis_options | None = None):
    """Returns an opaque plan handle (int); see include/rtis.h."""
    mic = np.ascontiguousarray(mic_xyz, dtype=np.float32)
    ch = np.ascontiguousarray(chirp, dtype=np.float32)
    dirs = np.ascontiguousarray(directions, dtype=np.float32)
    h = _VP()
    st = lib().rtis_plan_create(C.byref(h), _fptr(mic), int(mic.shape[0]), float(fs), _fptr(ch), int(ch.shape[0]),
                                _fptr(dirs), int(dirs.shape[0]), int(n_samples),
                                C.byref(options) if options is not None else None)
    check(st, "rtis_plan_create")
    return h.value


def rtis_plan_destroy(plan):
    lib().rtis_plan_destroy(plan)


def rtis_plan_get_info(plan) -> rtis_plan_info:
    info = rtis_plan_info()
    check(lib().rtis_plan_get_info(plan, C.byref(info)), "rtis_plan_get_info")
    return info


def rtis_process(plan, d_in, d_out, stream=None):
    check(lib().rtis_process(plan, ptr(d_in), ptr(d_out), stream_handle(stream)), "rtis_process")


def rtis_process_many(plan, d_in, n, d_out_td=None, d_out_fd=None, stream=None):
    check(lib().rtis_process_many(plan, ptr(d_in), int(n), ptr(d_out_td), ptr(d_out_fd), stream_handle(stream)),
          "rtis_process_many")


def rtis_matched_filter(plan, d_in, d_a, d_A=None, stream=None):
    check(lib().rtis_matched_filter(plan, ptr(d_in), ptr(d_a), ptr(d_A), stream_handle(stream)),
          "rtis_matched_filter")


def rtis_beamform_td(plan, d_a, d_out, stream=None):
    check(lib().rtis_beamform_td(plan, ptr(d_a), ptr(d_out), stream_handle(stream)), "rtis_beamform_td")


def rtis_beamform_fd(plan, d_A, d_out, stream=None):
    check(lib().rtis_beamform_fd(plan, ptr(d_A), ptr(d_out), stream_handle(stream)), "rtis_beamform_fd")


def rtis_baseband_signal(plan, d_in, d_z, stream=None):
    check(lib().rtis_baseband_signal(plan, ptr(d_in), ptr(d_z), stream_handle(stream)), "rtis_baseband_signal")


def rtis_pdm_demodulate(d_words, n_words, n_mics, n_samples, decim, taps, shift, d_x, stream=None):
    """taps: None (order-4 CIC) or a C-contiguous int32 NumPy array (host)."""
    tp, nt = (None, 0) if taps is None else (taps.ctypes.data, int(taps.shape[0]))
    check(lib().rtis_pdm_demodulate(ptr(d_words), int(n_words), int(n_mics), int(n_samples), int(decim), tp, nt,
                                    int(shift), ptr(d_x), stream_handle(stream)), "rtis_pdm_demodulate")


def rtis_beamform_bb(plan, d_z, d_out, stream=None):
    check(lib().rtis_beamform_bb(plan, ptr(d_z), ptr(d_out), stream_handle(stream)), "rtis_beamform_bb")


def rtis_steering_table(plan, d_shift, d_weight, stream=None):
    check(lib().rtis_steering_table(plan, ptr(d_shift), ptr(d_weight), stream_handle(stream)), "rtis_steering_table")


def rtis_matched_filter_noalloc(d_in, n_mics, n_samples, d_chirp, chirp_len, fs, band_lo_hz, band_hi_hz,
                                d_a, d_A=None, stream=None):
    """Matched filter with no device allocation (static scratch; see include/rtis.h)."""
    check(lib().rtis_matched_filter_noalloc(ptr(d_in), int(n_mics), int(n_samples), ptr(d_chirp), int(chirp_len),
                                            float(fs), float(band_lo_hz), float(band_hi_hz), ptr(d_a), ptr(d_A),
                                            stream_handle(stream)), "rtis_matched_filter_noalloc")


def rtis_fd_gemm_create(mic_xyz, directions, freqs_hz, n_frames, c=343.0, gain=None, delay_s=None,
                        precision=RTIS_PREC_FP32):
    """Frequency-domain beamforming GEMM plan (see include/rtis.h); returns a handle."""
    mic = np.ascontiguousarray(mic_xyz, dtype=np.float32)
    dirs = np.ascontiguousarray(directions, dtype=np.float32)
    fr = np.ascontiguousarray(freqs_hz, dtype=np.float64)
    g = None if gain is None else np.ascontiguousarray(gain, dtype=np.float32)
    dl = None if delay_s is None else np.ascontiguousarray(delay_s, dtype=np.float32)
    h = _VP()
    st = lib().rtis_fd_gemm_create(C.byref(h), _fptr(mic), int(mic.shape[0]), _fptr(dirs), int(dirs.shape[0]),
                                   fr.ctypes.data_as(C.POINTER(C.c_double)), int(fr.shape[0]), int(n_frames),
                                   float(c), None if g is None else _fptr(g), None if dl is None else _fptr(dl),
                                   int(precision))
    check(st, "rtis_fd_gemm_create")
    return h.value


def rtis_fd_gemm_run(g, d_X, d_Y, stream=None):
    check(lib().rtis_fd_gemm_run(g, ptr(d_X), ptr(d_Y), stream_handle(stream)), "rtis_fd_gemm_run")


def rtis_fd_gemm_destroy(g):
    lib().rtis_fd_gemm_destroy(g)


def _vp_array(items):
    arr = (_VP * len(items))()
    for i, it in enumerate(items):
        arr[i] = ptr(it)
    return arr


def rtis_process_batch(plans, d_in, d_out, stream=None):
    """Several plans' recordings -> energyscapes, one batched beamformer launch (no graph)."""
    check(lib().rtis_process_batch(_vp_array(plans), len(plans), _vp_array(d_in), _vp_array(d_out),
                                   stream_handle(stream)), "rtis_process_batch")


def rtis_batch_create(plans):
    h = _VP()
    check(lib().rtis_batch_create(C.byref(h), _vp_array(plans), len(plans)), "rtis_batch_create")
    return h.value


def rtis_batch_run(b, d_in, d_out, stream=None):
    check(lib().rtis_batch_run(b, _vp_array(d_in), _vp_array(d_out), stream_handle(stream)), "rtis_batch_run")


def rtis_batch_get_info(b) -> rtis_batch_info:
    info = rtis_batch_info()
    check(lib().rtis_batch_get_info(b, C.byref(info)), "rtis_batch_get_info")
    return info


def rtis_batch_sync(b) -> int:
    bits = C.c_uint(0)
    st = lib().rtis_batch_sync(b, C.byref(bits))
    if st not in (RTIS_OK, RTIS_ERR_TIMEOUT):
        check(st, "rtis_batch_sync")
    return bits.value


def rtis_batch_destroy(b):
    lib().rtis_batch_destroy(b)


def rtis_set_calibration(plan, d_mic_xyz=None, d_gain=None, d_delay_s=None, stream=None):
    check(lib().rtis_set_calibration(plan, ptr(d_mic_xyz), ptr(d_gain), ptr(d_delay_s), stream_handle(stream)),
          "rtis_set_calibration")


def rtis_backward(plan, d_in, d_grad_out, d_grad_xyz=None, d_grad_gain=None, d_grad_delay=None, stream=None):
    check(lib().rtis_backward(plan, ptr(d_in), ptr(d_grad_out), ptr(d_grad_xyz), ptr(d_grad_gain), ptr(d_grad_delay),
                              stream_handle(stream)), "rtis_backward")


def rtis_loss_l2(plan, d_E, d_E_ref, d_grad_out, d_loss, stream=None):
    check(lib().rtis_loss_l2(plan, ptr(d_E), ptr(d_E_ref), ptr(d_grad_out), ptr(d_loss), stream_handle(stream)),
          "rtis_loss_l2")


def rtis_baseline_create(plan):
    out = _VP()
    check(lib().rtis_baseline_create(C.byref(out), plan), "rtis_baseline_create")
    return out.value


def rtis_baseline_process(b, d_in, d_out, stream=None):
    check(lib().rtis_baseline_process(b, ptr(d_in), ptr(d_out), stream_handle(stream)), "rtis_baseline_process")


def rtis_baseline_destroy(b):
    lib().rtis_baseline_destroy(b)


def rtis_stream_create(plan, depth):
    out = _VP()
    check(lib().rtis_stream_create(C.byref(out), plan, int(depth)), "rtis_stream_create")
    return out.value


def _host_ptr(a) -> int:
    """Address of a host array: a NumPy array or a (pinned) CPU torch tensor."""
    return a.ctypes.data if isinstance(a, np.ndarray) else a.data_ptr()


def rtis_stream_submit(s, host_in, host_out) -> int:
    """host_in: C-contiguous int16 [M][N]; host_out: C-contiguous float32 [D][n_out]
    (pinned memory keeps the result copy asynchronous).  Returns the ticket."""
    t = C.c_int64(-1)
    check(lib().rtis_stream_submit(s, _host_ptr(host_in), _host_ptr(host_out), C.byref(t)), "rtis_stream_submit")
    return t.value


def rtis_stream_wait(s, ticket, timeout_ms=1000):
    check(lib().rtis_stream_wait(s, int(ticket), int(timeout_ms)), "rtis_stream_wait")


def rtis_stream_destroy(s):
    lib().rtis_stream_destroy(s)


def rtis_plan_sync(plan) -> int:
    bits = C.c_uint(0)
    st = lib().rtis_plan_sync(plan, C.byref(bits))
    if st not in (RTIS_OK, RTIS_ERR_DEVICE, RTIS_ERR_TIMEOUT, RTIS_ERR_NONFINITE):
        check(st, "rtis_plan_sync")
    return bits.value  # device status bits (RTIS_DEV_*); 0 when all went well


def rtis_plan_set_tracing(plan, enable: bool) -> None:
    check(lib().rtis_plan_set_tracing(plan, 1 if enable else 0), "rtis_plan_set_tracing")


def rtis_plan_get_trace(plan):
    """The last traced call's launches: [(kernel name, milliseconds)] in launch order (waits for them)."""
    buf = (rtis_trace_entry * TRACE_MAX)()
    n = C.c_int(0)
    check(lib().rtis_plan_get_trace(plan, buf, TRACE_MAX, C.byref(n)), "rtis_plan_get_trace")
    return [(KERNEL_NAMES.get(buf[i].kernel, str(buf[i].kernel)), float(buf[i].ms)) for i in range(min(n.value, TRACE_MAX))]


def rtis_status_string(status: int) -> str:
    return lib().rtis_status_string(status).decode()
