"""Kernel tracing: with tracing on, each call lists its own kernel launches in
launch order with CUDA-event times; the times are positive and add up to no
more than the call's own span on the stream; tracing off stops the listing."""
import numpy as np
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


def test_trace_lists_each_calls_launches(torch_cuda):
    torch = torch_cuda
    from paper_2208_10839_gb300 import Plan, RtisError
    cfg = synth.hemisphere(n_samples=8192, n_dirs=256)
    xs = torch.from_numpy(np.stack([synth.hemisphere(seed_scene=5 + i, n_samples=8192, n_dirs=256)["x"]
                                    for i in range(3)])).cuda()
    with Plan(cfg["mic_xyz"], cfg["fs"], cfg["chirp"], cfg["dirs"], 8192, max_batch=4) as p:
        p.set_tracing(True)
        E = p.process(xs[0])
        assert [k for k, _ in p.trace()] == ["mf_forward", "mf_inverse", "td_beamform"]
        # a calibration rebuilds the steering table: that call's list is the table alone
        p.set_calibration(gain=torch.ones(p.M, device="cuda"))
        assert [k for k, _ in p.trace()] == ["steering_table"]
        p.process(xs[0])
        assert [k for k, _ in p.trace()] == ["mf_forward", "mf_inverse", "td_beamform"]

        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        td, fd = p.process_many(xs, paths=("td", "fd"))
        e1.record()
        tr = p.trace()
        torch.cuda.synchronize()
        assert [k for k, _ in tr] == ["mf_forward", "mf_inverse", "td_beamform", "fd_gemm", "fd_energyscape"], tr
        assert all(ms > 0 for _, ms in tr)
        assert sum(ms for _, ms in tr) <= e0.elapsed_time(e1) * 1.05 + 0.05
        # the traced call computes the same energyscapes as the untraced one
        assert torch.equal(td[0], E)
        p.set_tracing(False)
        p.process(xs[1])
        with pytest.raises(RtisError):
            p.trace()
        assert p.sync() == 0
