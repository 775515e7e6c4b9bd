"""Many sensors in one pass: ragged record lengths, geometries and direction
sets through one batched beamformer launch (and its CUDA graph replay).

The batched result equals each sensor's own rtis_process bit for bit (same
kernels and per-tile arithmetic), and agrees with the FP64 oracle on a
reduced ring to the FP32 energyscape tolerance."""
import numpy as np
import pytest

import oracle as orc
import synth

pytestmark = pytest.mark.gpu
E_TOL = 1e-4


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2208_10839_gb300 import build
    build.build()
    return torch


def plans_for(sensors):
    from paper_2208_10839_gb300 import Plan
    return [Plan(s["mic_xyz"], s["fs"], s["chirp"], s["dirs"], s["n_samples"]) for s in sensors]


def per_sensor(torch, plans, xs):
    return [p.process(x).clone() for p, x in zip(plans, xs)]


@pytest.fixture(scope="module")
def small_ring():
    return synth.ring_sensors(n_sensors=4, lengths=(4096, 8192), dir_counts=(40, 72), n_reflectors=12)


def test_batch_matches_oracle_small_ring(torch_cuda, small_ring):
    torch = torch_cuda
    from paper_2208_10839_gb300 import Batch
    sensors = small_ring["sensors"]
    plans = plans_for(sensors)
    xs = [torch.from_numpy(s["x"]).cuda() for s in sensors]
    with Batch(plans) as b:
        outs = b.run(xs)
        assert b.sync() == 0
        info = b.info
        assert info.tuned == 1 and info.n_sensors == 4
    for s, E in zip(sensors, outs):
        E_ref = orc.energyscape(s["x"], s["chirp"], s["mic_xyz"], s["dirs"], s["fs"], s["c"])
        E = E.cpu().numpy().astype(np.float64)
        assert np.max(np.abs(E - E_ref)) <= E_TOL * E_ref.max()
        assert np.argmax(E) == np.argmax(E_ref)
    for p in plans:
        p.close()


def test_process_batch_and_graph_replay_equal_per_sensor(torch_cuda, small_ring):
    torch = torch_cuda
    from paper_2208_10839_gb300 import Batch, process_batch
    sensors = small_ring["sensors"]
    plans = plans_for(sensors)
    xs = [torch.from_numpy(s["x"]).cuda() for s in sensors]
    ref = per_sensor(torch, plans, xs)
    eager = process_batch(plans, xs)
    with Batch(plans) as b:
        first = [o.clone() for o in b.run(xs)]
        again = [o.clone() for o in b.run(xs)]       # graph replay, same pointers
        outs2 = [torch.empty_like(o) for o in first]
        b.run(xs, outs2)                              # new pointers: re-captured graph
        assert b.sync() == 0
    torch.cuda.synchronize()
    for r, e, f, a, o in zip(ref, eager, first, again, outs2):
        assert torch.equal(r, e)
        assert torch.equal(r, f)
        assert torch.equal(r, a)
        assert torch.equal(r, o)
    for p in plans:
        p.close()


@pytest.mark.slow
def test_ring_of_8_full_size_equals_per_sensor(torch_cuda):
    """8 sensors, N in {4096..32768}, D in {512..4096}, 30 reflectors: one batch."""
    torch = torch_cuda
    from paper_2208_10839_gb300 import Batch
    ring = synth.ring_sensors()
    sensors = ring["sensors"]
    plans = plans_for(sensors)
    xs = [torch.from_numpy(s["x"]).cuda() for s in sensors]
    ref = per_sensor(torch, plans, xs)
    with Batch(plans) as b:
        outs = b.run(xs)
        outs = b.run(xs)
        assert b.sync() == 0
    for r, o in zip(ref, outs):
        assert torch.equal(r, o)
    # oracle on a few directions of the shortest and the longest recording
    for i in (int(np.argmin([s["n_samples"] for s in sensors])), int(np.argmax([s["n_samples"] for s in sensors]))):
        s = sensors[i]
        E = outs[i].cpu().numpy().astype(np.float64)
        pick = np.unique(np.concatenate([np.argsort(E.max(axis=1))[-4:], [0, E.shape[0] // 2]]))
        a = orc.matched_filter(s["x"], s["chirp"], s["fs"])
        delta = orc.steering_delays(s["mic_xyz"], s["dirs"][pick], s["fs"], s["c"])
        E_ref = orc.envelope_decimate(orc.das_td(a, delta), orc.lpf_taps())
        assert np.max(np.abs(E[pick] - E_ref)) <= E_TOL * E_ref.max()
    for p in plans:
        p.close()
