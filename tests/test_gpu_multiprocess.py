"""The library in several processes on one GPU, the way env-range sharding runs on several GPUs: two
ranks (separate processes, each with its own CUDA context on cuda:0) render their halves of the envs
through librpl.so with env_offset = their first global env id, gather over gloo, and the result
must be bit-identical to one process rendering all envs.  The ranks' kernels never wait on one
another: the only exchange is the host-side gather after rendering."""
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_processes_render_their_env_ranges_bit_identically(cuda, rpl_lib, tmp_path):
    sys.path.insert(0, HERE)
    import multiprocess_render as M
    path = str(tmp_path / "gathered.npy")
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                   PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
        procs.append(subprocess.Popen([sys.executable, os.path.join(HERE, "multiprocess_render.py"), path],
                                      env=env, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True))
    logs = [p.communicate(timeout=600)[0] for p in procs]
    assert all(p.returncode == 0 for p in procs), "\n".join(l[-3000:] for l in logs)
    gathered = np.load(path)                       # [3 steps, E, pixels per env]
    w, _ = M.workload()
    whole = M.render(0, w.n_envs, 1000)
    assert gathered.shape == whole.shape
    assert np.array_equal(gathered, whole)
    # the env offset is part of the key: the same envs rendered at another offset differ
    shifted = M.render(0, w.n_envs, 1001)
    assert not np.array_equal(shifted[2], whole[2])
