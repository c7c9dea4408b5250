"""Render server: continuous batching of requests from several trainer threads.

Each request's depth must be the same whether it is rendered alone (rpl_render on a view of its
own) or fused with other trainers' requests in the server (bit-exact: the same kernels with the
same parameters).  Admission refuses a request whose host-buffer staging can never fit; a request
cancelled by its caller still renders, so the view's step sequence stays whole; a trainer thread
that dies without waiting leaves the server serving the others.  Failures are made on the host.
"""
import threading

import numpy as np
import pytest

from paper_2602_03002_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SENSOR = W.Sensor(sigma_abs=0.01, p_drop=0.03, max_latency=2, seed=(0x5E, 0x77))


def _views(rpl, torch, w, scene, shapes):
    """One view per (n_envs, n_cams), with its own pose sequence taken from the workload's envs."""
    out = []
    for k, (E, C) in enumerate(shapes):
        v = rpl.View(scene, E, w.n_links)
        v.set_cameras(w.cameras[:C])
        v.set_sensor(SENSOR)
        envs = (np.arange(E) * 3 + k) % w.n_envs
        poses = torch.from_numpy(np.ascontiguousarray(w.poses[:, envs])).cuda()
        out.append((v, poses, E, C))
    return out


def _workload():
    w = W.config_small(n_steps=5, n_envs=16)
    torso = w.cameras[0].mount_link
    w.cameras = w.cameras + [W.pinhole(24, 18, 80.0, 60.0, torso, (0.0, 0.12, 0.30), 90.0, 50.0, 0.1, 3.0),
                             W.pinhole(24, 18, 80.0, 60.0, torso, (0.0, -0.12, 0.30), -90.0, 50.0, 0.1, 3.0)]
    return w


SHAPES = [(5, 1), (9, 2), (16, 4), (3, 3), (7, 2), (12, 1), (2, 4), (11, 3)]


def test_results_alone_equal_results_in_the_mix(cuda, rpl_lib):
    torch = cuda
    w = _workload()
    scene = rpl_lib.Scene.from_workload(w)
    # alone: every view's five steps with rpl_render
    alone = []
    for v, poses, E, C in _views(rpl_lib, torch, w, scene, SHAPES):
        alone.append([v.render(poses[s], s, 100 * len(alone)).clone() for s in range(5)])
    torch.cuda.synchronize()
    # in the mix: four trainer threads, two views each, device and pinned host buffers
    views = _views(rpl_lib, torch, w, scene, SHAPES)
    server = rpl_lib.Server(scene, max_batch=8, n_streams=2)
    results = {}
    errors = []

    def trainer(t):
        try:
            mine = [2 * t, 2 * t + 1]
            for s in range(5):
                tickets = []
                for k in mine:
                    v, poses, E, C = views[k]
                    if (s + k) % 2:
                        out = v.out_tensor()
                        src = poses[s]
                    else:
                        out = torch.empty((E, v.layout()[1]), dtype=torch.float32).pin_memory()
                        src = poses[s].cpu().pin_memory()
                    tickets.append((k, server.submit(v, src, s, out, 100 * k), out, src))
                for k, tk, out, src in tickets:
                    server.wait(tk)
                    results[(k, s)] = out.cpu().clone()
        except Exception as exc:   # reported by the main thread
            errors.append(exc)

    th = [threading.Thread(target=trainer, args=(t,)) for t in range(4)]
    for x in th:
        x.start()
    for x in th:
        x.join()
    assert not errors, errors
    st = server.stats()
    server.close()
    for k in range(len(SHAPES)):
        for s in range(5):
            assert torch.equal(results[(k, s)], alone[k][s].cpu()), (k, s)
    assert st["completed"] == st["submitted"] == 40 and st["failed"] == 0


def test_request_runs_after_work_queued_on_the_default_stream(cuda, rpl_lib):
    """The server's streams are non-blocking, so a request must be ordered after what the caller
    queued on the default stream before submitting: here a ~20 ms sleep kernel, then the write of
    the right poses over wrong ones and a fill of the output.  Rendered before that work, the request
    would see the wrong poses, or its depth would be overwritten by the fill."""
    torch = cuda
    w = _workload()
    scene = rpl_lib.Scene.from_workload(w)
    (v, poses, E, C), = _views(rpl_lib, torch, w, scene, [(16, 4)])
    alone = [v.render(poses[s], s, 0).clone() for s in range(3)]
    torch.cuda.synchronize()
    (v, poses, E, C), = _views(rpl_lib, torch, w, scene, [(16, 4)])
    server = rpl_lib.Server(scene, max_batch=4, n_streams=2)
    try:
        for s in range(3):
            src = poses[(s + 1) % 3].clone()            # wrong poses, written before the sleep
            out = v.out_tensor()
            out.fill_(-5.0)
            torch.cuda.synchronize()
            torch.cuda._sleep(40_000_000)               # bounded spin on the default stream
            src.copy_(poses[s])
            out.fill_(-7.0)
            tk = server.submit(v, src, s, out)
            server.wait(tk)
            torch.cuda.synchronize()
            assert torch.equal(out, alone[s]), s
    finally:
        server.close()
        v.close()


def test_requests_queued_behind_a_busy_slot_are_fused(cuda, rpl_lib):
    """With one stream slot, requests submitted while a long request occupies it wait in the queue
    and go out together in the next launch, each still equal to its render alone."""
    torch = cuda
    w = _workload()
    scene = rpl_lib.Scene.from_workload(w)
    big = W.config_small(n_steps=1, n_envs=4096)
    vb = rpl_lib.View(scene, 4096, w.n_links)
    vb.set_cameras(w.cameras)
    vb.set_sensor(SENSOR)
    pb = torch.from_numpy(np.ascontiguousarray(big.poses[0])).cuda()
    small = _views(rpl_lib, torch, w, scene, SHAPES[:4])
    alone = [v.render(poses[0], 0, 100 * k).clone() for k, (v, poses, E, C) in enumerate(small)]
    torch.cuda.synchronize()
    small = _views(rpl_lib, torch, w, scene, SHAPES[:4])
    server = rpl_lib.Server(scene, max_batch=8, n_streams=1)
    outs = [v.out_tensor() for v, _, _, _ in small]
    tb = server.submit(vb, pb, 0, vb.out_tensor())
    tks = [server.submit(v, poses[0], 0, outs[k], 100 * k) for k, (v, poses, E, C) in enumerate(small)]
    server.wait(tb)
    for tk in tks:
        server.wait(tk)
    st = server.stats()
    server.close()
    for k in range(len(small)):
        assert torch.equal(outs[k], alone[k]), k
    assert st["batches"] <= 3 and st["max_batch_seen"] >= 2, st


def test_admission_budget_timeout_cancel_and_order(cuda, rpl_lib):
    torch = cuda
    w = _workload()
    scene = rpl_lib.Scene.from_workload(w)
    (v, poses, E, C), (v2, poses2, E2, C2) = _views(rpl_lib, torch, w, scene, [(16, 4), (4, 1)])
    server = rpl_lib.Server(scene, max_batch=4, n_streams=1, staging_bytes=64 << 10)
    # host buffers whose staging exceeds the whole budget are refused; device buffers need none
    big_out = torch.empty((E, v.layout()[1]), dtype=torch.float32).pin_memory()
    with pytest.raises(rpl_lib.RplError) as ei:
        server.submit(v, poses[0].cpu().pin_memory(), 0, big_out)
    assert ei.value.status == 5
    out = v.out_tensor()
    server.wait(server.submit(v, poses[0], 0, out))
    # a wait that runs out reports TIMEOUT and the ticket stays valid
    tk = server.submit(v, poses[1], 1, out)
    try:
        server.wait(tk, 0)
    except rpl_lib.RplError as e:
        assert e.status == 6
        server.wait(tk)
    # a cancelled request still renders; the view continues at the next step
    tk = server.submit(v, poses[2], 2, out)
    server.cancel(tk)
    with pytest.raises(rpl_lib.RplError):
        server.wait(tk)
    server.wait(server.submit(v, poses[3], 3, out))
    # steps of a view advance by 0 or 1
    with pytest.raises(rpl_lib.RplError) as ei:
        server.submit(v, poses[4], 6, out)
    assert ei.value.status == 1
    # small host-buffer requests fit the budget
    small = torch.empty((E2, v2.layout()[1]), dtype=torch.float32).pin_memory()
    server.wait(server.submit(v2, poses2[0].cpu().pin_memory(), 0, small))
    st = server.stats()
    assert st["cancelled"] == 1 and st["failed"] == 0
    server.close()


def test_trainer_that_dies_mid_request_leaves_the_server_serving(cuda, rpl_lib):
    torch = cuda
    w = _workload()
    scene = rpl_lib.Scene.from_workload(w)
    views = _views(rpl_lib, torch, w, scene, [(8, 2), (6, 1)])
    server = rpl_lib.Server(scene)

    def dying_trainer():
        v, poses, E, C = views[0]
        server.submit(v, poses[0], 0, v.out_tensor())
        raise RuntimeError("trainer crashed before waiting")

    t = threading.Thread(target=lambda: pytest.raises(RuntimeError, dying_trainer))
    t.start()
    t.join()
    v, poses, E, C = views[1]
    out = v.out_tensor()
    for s in range(3):
        server.wait(server.submit(v, poses[s], s, out))
    st = server.stats()
    assert st["completed"] >= 3 and st["failed"] == 0
    server.close()   # the abandoned request is drained and freed


def test_small_request_fused_with_a_large_one_completes_first(cuda, rpl_lib):
    """Inside one fused launch the smaller request's tiles run first and it completes by its own flag,
    before the launch ends; both results equal their renders alone."""
    torch = cuda
    w = _workload()
    scene = rpl_lib.Scene.from_workload(w)
    big_w = W.config_small(n_steps=1, n_envs=16384)
    blocker = rpl_lib.View(scene, 16384, w.n_links)
    blocker.set_cameras(w.cameras)
    vb = rpl_lib.View(scene, 16384, w.n_links)
    vb.set_cameras(w.cameras)
    vb.set_sensor(SENSOR)
    pb = torch.from_numpy(np.ascontiguousarray(big_w.poses[0])).cuda()
    (vs, ps, E, C), = _views(rpl_lib, torch, w, scene, [(3, 2)])
    alone_big = vb.render(pb, 0).clone()
    alone_small = vs.render(ps[0], 0, 9).clone()
    torch.cuda.synchronize()
    vb2 = rpl_lib.View(scene, 16384, w.n_links)
    vb2.set_cameras(w.cameras)
    vb2.set_sensor(SENSOR)
    (vs2, _, _, _), = _views(rpl_lib, torch, w, scene, [(3, 2)])
    server = rpl_lib.Server(scene, max_batch=8, n_streams=1)
    ob, os_ = vb2.out_tensor(), vs2.out_tensor()
    t0 = server.submit(blocker, pb, 0, blocker.out_tensor())   # occupies the only slot
    import time
    deadline = time.time() + 5.0
    while server.stats()["batches"] < 1 and time.time() < deadline:   # the blocker is on the GPU
        time.sleep(0.0001)
    tb = server.submit(vb2, pb, 0, ob)
    ts = server.submit(vs2, ps[0], 0, os_, 9)
    lat_s = server.wait(ts)
    lat_b = server.wait(tb)
    server.wait(t0)
    st = server.stats()
    server.close()
    assert torch.equal(ob, alone_big) and torch.equal(os_, alone_small)
    assert st["max_batch_seen"] >= 2, st          # the two were fused
    assert lat_s < lat_b, (lat_s, lat_b)


def test_cancel_while_another_thread_waits(cuda, rpl_lib):
    """A cancel from one thread while another waits on the same ticket ends that wait (with the
    result or an error) without touching a freed request; a second concurrent waiter is refused."""
    torch = cuda
    w = _workload()
    scene = rpl_lib.Scene.from_workload(w)
    big_w = W.config_small(n_steps=1, n_envs=8192)
    vb = rpl_lib.View(scene, 8192, w.n_links)
    vb.set_cameras(w.cameras)
    pb = torch.from_numpy(np.ascontiguousarray(big_w.poses[0])).cuda()
    server = rpl_lib.Server(scene, max_batch=4, n_streams=1)
    for rep in range(3):
        tk = server.submit(vb, pb, rep, vb.out_tensor())
        result = {}

        def waiter():
            try:
                rpl_lib.rpl_server_wait(server.h, tk, -1)
                result["status"] = 0
            except rpl_lib.RplError as e:
                result["status"] = e.status

        th = threading.Thread(target=waiter)
        th.start()
        import time
        time.sleep(0.002)
        try:   # refused while the other thread waits; TIMEOUT or done otherwise, depending on timing
            rpl_lib.rpl_server_wait(server.h, tk, 0)
        except rpl_lib.RplError as e:
            assert e.status in (1, 6)
        try:
            rpl_lib.rpl_server_cancel(server.h, tk)
        except rpl_lib.RplError as e:           # the request completed and was consumed first
            assert e.status == 1
        th.join(10)
        assert not th.is_alive()
        assert result["status"] in (0, 1)
    st = server.stats()
    server.close()
    assert st["submitted"] == 3 and st["failed"] == 0


def test_served_results_match_the_oracle(cuda, rpl_lib):
    """Requests of different env counts and camera sets, with device and pinned host buffers, fused by
    the server into shared launches, compared with the FP64 oracle over three steps with latency,
    noise and dropout: every served frame within the tolerance, dropout decisions bit-exact.  A large
    request occupies the only stream slot while the others are submitted, so they queue and go out
    fused; the server's statistics confirm it."""
    import oracle
    from conftest import compare_depth
    torch = cuda
    w = _workload()
    scene = rpl_lib.Scene.from_workload(w)
    shapes = [(5, 1), (9, 2), (16, 4), (3, 3), (7, 2), (12, 1)]
    views = _views(rpl_lib, torch, w, scene, shapes)
    big_w = W.config_small(n_steps=1, n_envs=16384)
    blocker = rpl_lib.View(scene, 16384, w.n_links)
    blocker.set_cameras(w.cameras)
    pb = torch.from_numpy(np.ascontiguousarray(big_w.poses[0])).cuda()
    ob = blocker.out_tensor()
    server = rpl_lib.Server(scene, max_batch=8, n_streams=1)
    served = {}
    fused = []
    import time
    for s in range(3):
        before = server.stats()["batches"]
        t0 = server.submit(blocker, pb, s, ob)
        deadline = time.time() + 5.0
        while server.stats()["batches"] == before and time.time() < deadline:   # the blocker is on the GPU
            time.sleep(0.0001)
        tickets = []
        for k, (v, poses, E, C) in enumerate(views):
            if (s + k) % 2:
                out, src = v.out_tensor(), poses[s]
            else:
                out = torch.empty((E, v.layout()[1]), dtype=torch.float32).pin_memory()
                src = poses[s].cpu().pin_memory()
            tickets.append((k, server.submit(v, src, s, out, 100 * k), out, src))
        server.wait(t0)
        for k, tk, out, src in tickets:
            server.wait(tk)
            served[(k, s)] = out.cpu().numpy().reshape(-1).copy()
        fused.append(server.stats()["max_batch_seen"])
    st = server.stats()
    server.close()
    assert st["failed"] == 0 and st["max_batch_seen"] >= 2, st
    for k, (v, poses, E, C) in enumerate(views):
        envs = (np.arange(E) * 3 + k) % w.n_envs
        osc = oracle.OracleScene.from_workload(w)
        rays = oracle.all_rays(w.cameras[:C], E)
        for s in range(3):
            ref = osc.render(w.cameras[:C], np.ascontiguousarray(w.poses[:, envs]), s, rays, SENSOR,
                             s_first=np.zeros(E, np.int64), env_offset=100 * k)
            got = served[(k, s)]
            dropped = (ref["flags"] & oracle.FLAG_DROPPED) != 0
            assert np.array_equal(got == np.float32(SENSOR.fill), dropped), (k, s)
            compare_depth(got, ref["depth"], ref["flags"], "served request %d (%d envs x %d cams) step %d" % (k, E, C, s))
        osc.close()
