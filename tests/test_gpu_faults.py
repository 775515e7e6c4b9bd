"""Failure detection on the GPU without a GPU fault: a bounded wait that is
made to run out (the injected stall withholds one TMA copy per CTA), a
non-finite input, and an injected launch failure.  After each, the context
stays usable and the next call gives the normal result."""
import pytest

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


@pytest.fixture
def plan_and_input(torch_cuda):
    from paper_2208_10839_gb300 import Plan
    cfg = synth.single_sensor(n_samples=4096, n_dirs=48)
    p = Plan(cfg["mic_xyz"], cfg["fs"], cfg["chirp"], cfg["dirs"], cfg["n_samples"])
    x = torch_cuda.from_numpy(cfg["x"]).cuda()
    yield p, x
    p.close()


def test_bounded_wait_runs_out_and_context_survives(torch_cuda, plan_and_input, monkeypatch):
    from paper_2208_10839_gb300 import _native as nat
    p, x = plan_and_input
    ref = p.process(x).clone()
    assert p.sync() == 0
    monkeypatch.setenv("RTIS_FAULT", "stall")
    p.process(x)
    bits = p.sync()
    assert bits & nat.RTIS_DEV_TIMEOUT, bits
    monkeypatch.setenv("RTIS_FAULT", "")
    again = p.process(x)
    assert p.sync() == 0
    assert torch_cuda.equal(again, ref)


def test_non_finite_input_is_flagged(torch_cuda, plan_and_input):
    from paper_2208_10839_gb300 import _native as nat
    torch = torch_cuda
    p, x = plan_and_input
    a, _ = p.matched_filter(x)
    a[3, 1000] = complex(float("nan"), 0.0)
    E = p.beamform_td(a)
    bits = p.sync()
    assert bits & nat.RTIS_DEV_NONFINITE, bits
    assert not bool(torch.isfinite(E).all())
    a2, A2 = p.matched_filter(x, want_spectrum=True)
    A2[0, 10] = complex(float("inf"), 0.0)
    p.beamform_fd(A2)
    assert p.sync() & nat.RTIS_DEV_NONFINITE
    p.process(x)
    assert p.sync() == 0


def test_injected_launch_failure(torch_cuda, plan_and_input, monkeypatch):
    from paper_2208_10839_gb300 import RtisError, _native as nat
    p, x = plan_and_input
    monkeypatch.setenv("RTIS_FAULT", "launch")
    with pytest.raises(RtisError) as ei:
        p.process(x)
    assert ei.value.status == nat.RTIS_ERR_CUDA
    monkeypatch.setenv("RTIS_FAULT", "")
    E = p.process(x)
    assert p.sync() == 0
    assert bool(torch_cuda.isfinite(E).all())
