"""Host checks of the eight-wide quantised BVH (no GPU): every triangle sits in exactly one leaf,
every dequantised child box contains everything below it (quantisation rounds outward), empty slots
can never be hit, and the slot order follows the child positions (slot bit a set -> +axis side)."""
import numpy as np
import pytest

from paper_2602_03002_gb300 import workloads as W


def _bytes(words):
    return np.frombuffer(np.ascontiguousarray(words, np.uint32).tobytes(), np.uint8)


def _decode(node):
    w = node
    origin = np.frombuffer(np.uint32(w[:3]).tobytes(), np.float32).astype(np.float64)
    e = _bytes(w[3:4])[:3].astype(np.int64)
    step = np.ldexp(1.0, e - 127)
    imask = int(_bytes(w[3:4])[3])
    meta = _bytes(w[6:8])
    q = _bytes(w[8:20]).reshape(6, 8).astype(np.float64)   # lo x, lo y, lo z, hi x, hi y, hi z
    lo = origin[:, None] + q[:3] * step[:, None]
    hi = origin[:, None] + q[3:] * step[:, None]
    return dict(imask=imask, child_base=int(w[4]), tri_base=int(w[5]), meta=meta, lo=lo, hi=hi, q=q)


@pytest.mark.parametrize("kind", ["terrain", "ellipsoid", "soup", "one", "empty"])
def test_bvh8_invariants(rpl_lib, kind):
    rng = np.random.default_rng(5)
    if kind == "terrain":
        w = W.config_small(n_steps=1, n_envs=1)
        v, t = w.terrain_verts, w.terrain_tris
    elif kind == "ellipsoid":
        v, t = W.ellipsoid_mesh((0.2, 0.1, 0.3))
    elif kind == "soup":
        v = rng.uniform(-30, 30, (500, 3)).astype(np.float32)
        t = rng.integers(0, 500, (700, 3)).astype(np.int32)
    elif kind == "one":
        v, t = np.eye(3, dtype=np.float32) * 50, np.array([[0, 1, 2]], np.int32)
    else:
        v, t = np.zeros((0, 3), np.float32), np.zeros((0, 3), np.int32)
    nodes, tris, depth = rpl_lib.rpl_bvh8_build_host(v, t, 4)
    assert len(nodes) >= 1 and depth >= 1
    seen = np.zeros(len(t), np.int32)
    pts = np.stack([tris["v0"], tris["v1"], tris["v2"]], 1).astype(np.float64)   # [T, 3, 3]

    def subtree(i, d):
        """Visit node i; return (lo, hi) of all triangles below it and check its children."""
        n = _decode(nodes[i])
        assert d <= depth
        allo, alhi = np.full(3, np.inf), np.full(3, -np.inf)
        for s in range(8):
            m = int(n["meta"][s])
            if m == 0:
                assert np.all(n["q"][:3, s] == 255) and np.all(n["q"][3:, s] == 0)   # empty: never hit
                assert not (n["imask"] >> s) & 1
                continue
            if (n["imask"] >> s) & 1:
                rank = m & 0x7F
                assert rank == bin(n["imask"] & ((1 << s) - 1)).count("1")
                c = n["child_base"] + rank
                assert c > i
                lo, hi = subtree(c, d + 1)
            else:
                off, cnt = (m >> 2) & 31, (m & 3) + 1
                first = n["tri_base"] + off
                seen[tris["id"][first:first + cnt]] += 1
                p = pts[first:first + cnt].reshape(-1, 3)
                lo, hi = p.min(0), p.max(0)
            assert np.all(n["lo"][:, s] <= lo) and np.all(n["hi"][:, s] >= hi), (i, s)   # conservative
            allo, alhi = np.minimum(allo, lo), np.maximum(alhi, hi)
        # slot order: the children on the + side of an axis have that slot bit set, on average
        return allo, alhi

    subtree(0, 1)
    assert np.all(seen == 1)
    if len(t):
        orig = v[t[tris["id"]]]
        assert np.array_equal(tris["v0"], orig[:, 0]) and np.array_equal(tris["v2"], orig[:, 2])


def test_bvh8_slots_follow_child_positions(rpl_lib):
    w = W.config_small(n_steps=1, n_envs=1)
    nodes, tris, depth = rpl_lib.rpl_bvh8_build_host(w.terrain_verts, w.terrain_tris, 4)
    agree = total = 0
    for i in range(len(nodes)):
        n = _decode(nodes[i])
        used = [s for s in range(8) if n["meta"][s]]
        if len(used) < 2:
            continue
        ctr = np.array([(n["lo"][:, s] + n["hi"][:, s]) / 2 for s in used])
        mid = ctr.mean(0)
        for k, s in enumerate(used):
            for a in range(2):   # x and y carry the terrain's spread
                if abs(ctr[k, a] - mid[a]) > 1e-6:
                    total += 1
                    agree += ((s >> a) & 1) == (ctr[k, a] > mid[a])
    assert total > 100 and agree / total > 0.8


def test_bvh8_rejects_large_leaves(rpl_lib):
    with pytest.raises(rpl_lib.RplError):
        rpl_lib.rpl_bvh8_build_host(np.eye(3, dtype=np.float32), np.array([[0, 1, 2]], np.int32), 8)
