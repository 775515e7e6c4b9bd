"""The C ABI library loads on a machine without a GPU, exports every entry
point include/rtis.h declares, and rejects bad arguments before touching the
device.  CPU only (no compute calls)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def nat():
    from paper_2208_10839_gb300 import build
    build.build()
    from paper_2208_10839_gb300 import _native
    _native.lib()
    return _native


def declared_entry_points():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(rtis_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_entry_points()
    for required in ("rtis_plan_create", "rtis_process", "rtis_plan_destroy", "rtis_matched_filter",
                     "rtis_beamform_td", "rtis_plan_sync", "rtis_last_error"):
        assert required in names


def test_every_declared_symbol_is_exported(nat):
    lib = C.CDLL(nat.LIB_PATH)
    missing = [n for n in declared_entry_points() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_abi(nat):
    for n in declared_entry_points():
        if n in ("rtis_options_default", "rtis_last_error"):
            continue
        assert hasattr(nat, n), n


def test_options_default(nat):
    o = nat.default_options()
    assert o.c == 343.0 and o.decim == 10 and o.lpf_len == 0
    assert o.band_lo_hz == 20e3 and o.band_hi_hz == 80e3
    assert o.path == nat.RTIS_PATH_TD and o.precision == nat.RTIS_PREC_FP32
    assert o.max_batch == 0 and o.td_layout == 0 and o.bb_layout == 0 and o.grid_mode == 0
    assert o.fd_ifft == nat.RTIS_FD_IFFT_AUTO


def _args():
    return synth.mic_array(0), synth.chirp().astype(np.float32), synth.azimuth_fan(11)


@pytest.mark.parametrize("kw,status", [
    (dict(n_samples=8190), 1),            # not a multiple of 4
    (dict(n_samples=32), 1),              # too short
    (dict(n_samples=70000), 4),           # FFT longer than 65536
    (dict(fs=-1.0), 1),
    (dict(mics=40), 4),                   # more than 32 mics
    (dict(dirs=0), 1),
    (dict(nan_mic=True), 6),
    (dict(decim=0), 1),
    (dict(band=(80e3, 20e3)), 1),
    (dict(band=(20e3, 150e3)), 4),        # band above fs/4
    (dict(precision=2), 4),               # FP16 storage is not offered
    (dict(precision=1, path=1), 4),       # BF16 storage on the frequency-domain path
    (dict(path=3), 1),                    # no such path
    (dict(td_layout=6), 1),               # 5 time-domain layouts
    (dict(bb_layout=7), 1),               # 6 baseband layouts
    (dict(grid_mode=3), 1),
    (dict(fd_ifft=3), 1),                 # AUTO, FFT or TC
    (dict(fd_ifft=-1), 1),
])
def test_plan_create_rejects(nat, kw, status):
    mic, ch, dirs = _args()
    if "mics" in kw:
        mic = np.zeros((kw["mics"], 3), np.float32)
    if kw.get("nan_mic"):
        mic = mic.copy()
        mic[3, 1] = np.nan
    if "dirs" in kw:
        dirs = dirs[:kw["dirs"]]
    o = nat.default_options()
    if "decim" in kw:
        o.decim = kw["decim"]
    if "band" in kw:
        o.band_lo_hz, o.band_hi_hz = kw["band"]
    if "precision" in kw:
        o.precision = kw["precision"]
    if "path" in kw:
        o.path = kw["path"]
    for f in ("td_layout", "bb_layout", "grid_mode", "fd_ifft"):
        if f in kw:
            setattr(o, f, kw[f])
    with pytest.raises(nat.RtisError) as ei:
        nat.rtis_plan_create(mic, kw.get("fs", 450e3), ch, dirs, kw.get("n_samples", 4096), o)
    assert ei.value.status == status
    assert nat.last_error()


def test_null_arguments(nat):
    lib = nat.lib()
    assert lib.rtis_plan_create(None, None, 32, 450e3, None, 900, None, 10, 4096, None) == nat.RTIS_ERR_INVALID_ARG
    assert lib.rtis_process(None, None, None, None) == nat.RTIS_ERR_INVALID_ARG
    assert lib.rtis_matched_filter(None, None, None, None, None) == nat.RTIS_ERR_INVALID_ARG
    assert lib.rtis_beamform_td(None, None, None, None) == nat.RTIS_ERR_INVALID_ARG
    assert lib.rtis_plan_sync(None, None) == nat.RTIS_ERR_INVALID_ARG
    assert lib.rtis_plan_set_tracing(None, 1) == nat.RTIS_ERR_INVALID_ARG
    assert lib.rtis_plan_get_trace(None, None, 0, None) == nat.RTIS_ERR_INVALID_ARG
    lib.rtis_plan_destroy(None)
    assert nat.rtis_status_string(0) == "ok"


def test_injected_allocation_and_launch_failures(nat, monkeypatch):
    """RTIS_FAULT forces the host error paths without touching the GPU."""
    mic, ch, dirs = _args()
    monkeypatch.setenv("RTIS_FAULT", "alloc")
    with pytest.raises(nat.RtisError) as ei:
        nat.rtis_plan_create(mic, 450e3, ch, dirs, 4096, nat.default_options())
    assert ei.value.status == nat.RTIS_ERR_OOM and "injected" in nat.last_error()
    monkeypatch.setenv("RTIS_FAULT", "launch")
    lib = nat.lib()
    assert lib.rtis_process(None, None, None, None) == nat.RTIS_ERR_CUDA
    assert "injected" in nat.last_error()
    assert lib.rtis_backward(None, None, None, None, None, None, None) == nat.RTIS_ERR_CUDA
    monkeypatch.setenv("RTIS_FAULT", "")
    assert lib.rtis_process(None, None, None, None) == nat.RTIS_ERR_INVALID_ARG


def test_stream_and_baseline_argument_checks(nat):
    lib = nat.lib()
    import ctypes as C
    out = C.c_void_p()
    assert lib.rtis_stream_create(C.byref(out), None, 4) == nat.RTIS_ERR_INVALID_ARG
    assert lib.rtis_stream_create(None, None, 4) == nat.RTIS_ERR_INVALID_ARG
    t = C.c_int64(0)
    assert lib.rtis_stream_submit(None, None, None, C.byref(t)) == nat.RTIS_ERR_INVALID_ARG
    assert lib.rtis_stream_wait(None, 0, 10) == nat.RTIS_ERR_INVALID_ARG
    assert lib.rtis_baseline_create(C.byref(out), None) == nat.RTIS_ERR_INVALID_ARG
    assert lib.rtis_baseline_process(None, None, None, None) == nat.RTIS_ERR_INVALID_ARG
    assert nat.rtis_status_string(nat.RTIS_ERR_BUSY) == "no free slot"


def test_pdm_and_baseband_argument_checks(nat):
    # every check runs on the host before any launch
    lib = nat.lib()
    import ctypes as C
    fake = 1 << 20   # an aligned non-NULL address that is never dereferenced
    taps = (C.c_int32 * 3)(1, 2, 1)
    ok = dict(d_words=fake, n_words=100, n_mics=4, n_samples=10, decim=10, taps=None, n_taps=0, shift=0, d_x=fake)

    def call(**kw):
        a = dict(ok, **kw)
        return lib.rtis_pdm_demodulate(a["d_words"], a["n_words"], a["n_mics"], a["n_samples"], a["decim"],
                                       a["taps"], a["n_taps"], a["shift"], a["d_x"], None)
    E = nat.RTIS_ERR_INVALID_ARG
    assert call(d_x=None) == E
    assert call(d_words=None) == E
    assert call(d_words=fake + 2) == E                     # words 4-byte aligned
    assert call(d_x=fake + 1) == E                         # int16 output 2-byte aligned
    assert call(n_mics=0) == E and call(n_mics=33) == E
    assert call(n_samples=0) == E and call(n_words=-1) == E
    assert call(decim=0) == E and call(decim=65) == E
    assert call(shift=-1) == E and call(shift=31) == E
    assert call(taps=C.cast(taps, C.c_void_p), n_taps=0) == E
    assert call(taps=C.cast(taps, C.c_void_p), n_taps=257) == E
    big = (C.c_int32 * 2)(1 << 30, 1)                      # sum |g| above 2^30
    assert call(taps=C.cast(big, C.c_void_p), n_taps=2) == E
    assert lib.rtis_baseband_signal(None, None, None, None) == E
    assert lib.rtis_beamform_bb(None, None, None, None) == E


def test_binding_mirrors_header_layouts_and_constants(nat, tmp_path):
    """Each ctypes mirror of a header struct has the header's size and field offsets, and each
    constant of the binding the header's value: a mirror that drifted from rtis.h would pass
    wrong arguments to every call that takes it.  A C program built against the header prints
    the header's side."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("gcc not found")
    structs = [nat.rtis_options, nat.rtis_plan_info, nat.rtis_batch_info, nat.rtis_trace_entry]
    consts = [n for n in dir(nat) if re.fullmatch(r"RTIS_(OK|ERR_[A-Z_]+|DEV_[A-Z_]+|PATH_[A-Z]+|PREC_[A-Z0-9]+|"
                                                 r"FD_IFFT_[A-Z]+)", n)]
    kernel_ids = {f"RTIS_KERNEL_{name.upper()}": kid for kid, name in nat.KERNEL_NAMES.items()}
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "rtis.h"', "int main(void) {"]
    for st in structs:
        lines.append(f'printf("{st.__name__} sizeof %zu\\n", sizeof({st.__name__}));')
        for field, _ in st._fields_:
            lines.append(f'printf("{st.__name__} {field} %zu\\n", offsetof({st.__name__}, {field}));')
    for name in consts + sorted(kernel_ids) + ["RTIS_TRACE_MAX"]:
        lines.append(f'printf("const {name} %ld\\n", (long)({name}));')
    lines.append("return 0; }")
    src, exe = tmp_path / "layout.c", tmp_path / "layout"
    src.write_text("\n".join(lines) + "\n")
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                        "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    header = {tuple(ln.split()[:2]): int(ln.split()[2]) for ln in out if ln}
    for st in structs:
        assert header[(st.__name__, "sizeof")] == C.sizeof(st), st.__name__
        for field, _ in st._fields_:
            assert header[(st.__name__, field)] == getattr(st, field).offset, (st.__name__, field)
    for name in consts:
        assert header[("const", name)] == getattr(nat, name), name
    for name, kid in kernel_ids.items():
        assert header[("const", name)] == kid, name
    assert header[("const", "RTIS_TRACE_MAX")] == nat.TRACE_MAX
    assert len(consts) >= 17  # the statuses, device bits, paths, precisions and IFFT forms


def test_header_is_plain_c(tmp_path):
    # the boundary is a C ABI: the header compiles as strict C99 (and as C++), no torch types
    import shutil
    import subprocess
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    src = tmp_path / "use.c"
    src.write_text('#include "rtis.h"\nint main(void) { rtis_options o; rtis_options_default(&o); return o.path; }\n')
    for cc, args in (("gcc", ["-std=c99", "-pedantic"]), ("g++", ["-std=c++17", "-x", "c++"])):
        if shutil.which(cc) is None:
            pytest.skip(f"{cc} not found")
        r = subprocess.run([cc, *args, "-Wall", "-Wextra", "-Werror", "-fsyntax-only",
                            "-I", os.path.join(root, "include"), str(src)], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
    header = open(os.path.join(root, "include", "rtis.h")).read()
    assert "torch" not in header and "at::" not in header
