"""Sensor-state checkpoints: a view restored from a checkpoint continues bit-exact.

A trainer that saves its view's state (latency ring, per-env first steps, last step) after step s
and restores it into a fresh view of the same configuration must render steps s+1, s+2, ... exactly
as the uninterrupted view does; the delayed frames it returns come from the restored ring."""
import numpy as np
import pytest

from paper_2602_03002_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SENSOR = W.Sensor(sigma_abs=0.01, sigma_rel=0.02, p_drop=0.05, max_latency=3, seed=(0x51, 0xA7))


@pytest.mark.parametrize("on_device", [False, True])
def test_restored_view_continues_bit_exact(cuda, rpl_lib, on_device):
    torch = cuda
    w = W.config_small(n_steps=8, n_envs=6)
    scene = rpl_lib.Scene.from_workload(w)
    poses = torch.from_numpy(w.poses).cuda()
    a = rpl_lib.View.from_workload(scene, w)
    a.set_sensor(SENSOR)
    ref, ckpt = [], None
    for s in range(8):
        ref.append(a.render(poses[s], s, 5).clone())
        if s == 3:
            n = rpl_lib.rpl_view_state_size(a.h)
            buf = torch.empty(n, dtype=torch.uint8, device="cuda") if on_device else None
            ckpt = a.save_state(buf)
            assert (ckpt.numel() if on_device else ckpt.size) == n
    b = rpl_lib.View.from_workload(scene, w)
    b.set_sensor(SENSOR)
    b.load_state(ckpt)
    for s in range(4, 8):
        assert torch.equal(b.render(poses[s], s, 5), ref[s]), s
    b.sync()
    # the restored view knows its last step: skipping one is refused
    c = rpl_lib.View.from_workload(scene, w)
    c.set_sensor(SENSOR)
    c.load_state(ckpt)
    with pytest.raises(rpl_lib.RplError):
        c.render(poses[6], 6, 5)


def test_state_from_another_configuration_is_refused(cuda, rpl_lib):
    w = W.config_small(n_steps=2, n_envs=4)
    scene = rpl_lib.Scene.from_workload(w)
    a = rpl_lib.View.from_workload(scene, w)
    a.set_sensor(SENSOR)
    ckpt = a.save_state()
    other = W.Sensor(max_latency=1)
    b = rpl_lib.View.from_workload(scene, w)
    b.set_sensor(other)                       # another ring span
    with pytest.raises(rpl_lib.RplError) as ei:
        b.load_state(ckpt)
    assert ei.value.status == 1
    bad = ckpt.copy()
    bad[:4] = np.frombuffer(b"XXXX", np.uint8)
    with pytest.raises(rpl_lib.RplError):
        a.load_state(bad)
    with pytest.raises(rpl_lib.RplError):
        a.load_state(ckpt[:10])
