"""The bounds-checked build: librpl_checked.so tests every node and triangle index against its array
before reading it and records a violation in the view's error word (compute-sanitizer is not
available, so this is the memory-safety check of the traversal).  On every kind of terrain BVH,
through the server's fused launch, with downsampled cameras, randomised mounts and side masks, and
through the no-allocation entry point, it must record nothing and give the normal build's frames
bit for bit."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_checked_build_records_nothing_and_matches(cuda, rpl_lib, tmp_path):
    from paper_2602_03002_gb300 import build
    build.build(checked=True)
    sys.path.insert(0, HERE)
    import checked_workloads
    normal = checked_workloads.render_all()
    path = tmp_path / "checked.npz"
    env = dict(os.environ, RPL_CHECKED="1", PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    r = subprocess.run([sys.executable, os.path.join(HERE, "checked_workloads.py"), str(path)], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]     # an error word would raise DEVICE_FAULT in sync()
    checked = np.load(path)
    assert sorted(checked.files) == sorted(normal)
    for k in normal:
        assert np.array_equal(checked[k], normal[k]), k
