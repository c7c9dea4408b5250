import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built librpl.so")
    config.addinivalue_line("markers", "slow: long-running (full-size workload)")


# Parity bar for floating-point depth (metres) and the budget of rays that may disagree because
# FP32 legitimately decides differently: only rays the oracle flags as passing within eps of a
# silhouette edge, ending within 1e-4 m of the far plane, or hitting so obliquely that FP32 rounding
# of the ray alone moves the depth by more than a quarter of the tolerance; at most 1e-4 of all
# compared rays.
DEPTH_TOL = 1e-4
MISMATCH_FRAC = 1e-4

# What the allowance excused over the session: rays compared, rays beyond the tolerance, and for the
# latter which flag each one carried (a ray may carry several), plus how many lie within the flat
# 1e-6 m band of a silhouette edge.  Printed at the end of the run (pytest_terminal_summary).
ALLOWANCE = {"comparisons": 0, "rays": 0, "excused": 0, "edge": 0, "edge_1e6": 0, "far": 0, "grazing": 0,
             "worst_frac": 0.0, "worst_what": ""}


def compare_depth(gpu, ref, flags, what="", tol=DEPTH_TOL, frac=MISMATCH_FRAC):
    """Element-wise parity: |gpu - ref| <= tol except on flagged rays, and those at most frac of all.
    Returns the absolute differences; records what the allowance excused in ALLOWANCE."""
    import oracle
    gpu = np.asarray(gpu, np.float64).reshape(-1)
    ref = np.asarray(ref, np.float64).reshape(-1)
    flags = np.asarray(flags).reshape(-1)
    assert gpu.shape == ref.shape == flags.shape
    diff = np.abs(gpu - ref)
    bad = ~(diff <= tol)
    allowed = (flags & oracle.FLAG_FP32_SENSITIVE) != 0
    unexplained = bad & ~allowed
    if unexplained.any():
        i = np.flatnonzero(unexplained)
        raise AssertionError("%s: %d rays differ by more than %g m outside the edge/far bands; worst %g m at %s "
                             "(gpu %r, oracle %r)" % (what, len(i), tol, diff[i].max(), i[np.argmax(diff[i])],
                                                      gpu[i[np.argmax(diff[i])]], ref[i[np.argmax(diff[i])]]))
    budget = max(1, int(frac * gpu.size))
    fb = flags[bad]
    a = ALLOWANCE
    a["comparisons"] += 1
    a["rays"] += int(gpu.size)
    a["excused"] += int(bad.sum())
    a["edge"] += int(np.count_nonzero(fb & oracle.FLAG_EDGE))
    a["edge_1e6"] += int(np.count_nonzero(fb & oracle.FLAG_EDGE_1E6))
    a["far"] += int(np.count_nonzero(fb & oracle.FLAG_FAR))
    a["grazing"] += int(np.count_nonzero(fb & oracle.FLAG_GRAZING))
    f = float(bad.sum()) / max(1, gpu.size)
    if f > a["worst_frac"]:
        a["worst_frac"], a["worst_what"] = f, "%s (%d of %d rays)" % (what, int(bad.sum()), gpu.size)
    assert bad.sum() <= budget, "%s: %d flagged disagreements > %d allowed" % (what, bad.sum(), budget)
    return diff


def pytest_terminal_summary(terminalreporter, exitstatus, config):
    a = ALLOWANCE
    if a["comparisons"] == 0:
        return
    terminalreporter.write_line(
        "parity allowance: %d oracle comparisons, %d rays; %d beyond %g m (%.2e of the rays) were excused: "
        "EDGE %d, FAR %d, GRAZING %d (a ray may carry several flags); %d of them within the flat 1e-6 m edge "
        "band; largest share in one comparison %.2e: %s"
        % (a["comparisons"], a["rays"], a["excused"], DEPTH_TOL, a["excused"] / max(1, a["rays"]), a["edge"],
           a["far"], a["grazing"], a["edge_1e6"], a["worst_frac"], a["worst_what"]))


@pytest.fixture(scope="session")
def rpl_lib():
    from paper_2602_03002_gb300 import build, rpl
    build.build()
    return rpl


@pytest.fixture(scope="session")
def cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("a CUDA GPU is required for tests marked gpu")
    return torch
