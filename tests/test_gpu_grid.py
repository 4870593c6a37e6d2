"""The grid build against its definition (needs a GPU).

The build sorts the points by the Morton code of (p - min) >> shift (a stable
radix sort), cuts the order into octree leaves and the leaves into groups of
at most 32 consecutive points.  Checked here through the library's internal
state dump: the codes are the interleaved bits computed on the host, in
non-decreasing order, ties in input order; every input point appears once
with its coordinates; the groups tile the order, never cross a leaf and start
at the leaf's first point or 32 points after a group start.
"""
import ctypes

import numpy as np
import pytest

from paper_2311_17604_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pd():
    from paper_2311_17604_gb300 import build
    build.build()
    import paper_2311_17604_gb300.pd as pdm
    return pdm


def _dump(pd, g, what, dtype, count):
    out = np.empty(count, dtype=dtype)
    L = pd.lib()
    L.pd__debug_dump.restype = ctypes.c_int
    rc = L.pd__debug_dump(g.h, what, out.ctypes.data_as(ctypes.c_void_p),
                          ctypes.c_int64(out.nbytes))
    assert rc == 0
    return out


def _spread(v):
    """The bits of v (< 2^21) moved to every third position."""
    v = v.astype(np.uint64)
    out = np.zeros_like(v)
    for b in range(21):
        out |= ((v >> np.uint64(b)) & np.uint64(1)) << np.uint64(3 * b)
    return out


@pytest.mark.parametrize("which", ["room", "random", "dups"])
def test_grid_order_and_groups(pd, which):
    rng = np.random.default_rng(11)
    if which == "room":
        xyz = synth.room_scan(seed=2, n_az=900, n_el=180).xyz
    elif which == "random":
        xyz = rng.integers(-50_000, 50_000, size=(300_001, 3)).astype(np.int32)
    else:  # heavy duplicates and dense clusters: leaves above 32 points at level 0
        base = rng.integers(0, 2_000, size=(20_000, 3)).astype(np.int32)
        xyz = np.concatenate([base, base[:5000], np.repeat(base[:40], 50, axis=0)])
    n = xyz.shape[0]
    ctx = pd.Context()
    g = pd.Grid(ctx, torch.from_numpy(np.ascontiguousarray(xyz)).cuda())
    sc = _dump(pd, g, 8, np.int64, 8)
    ng, ngroups, B, shift, T = int(sc[1]), int(sc[2]), int(sc[3]), int(sc[4]), int(sc[7])
    assert ng == n
    pos = _dump(pd, g, 0, np.int32, 4 * n).reshape(n, 4)
    code = _dump(pd, g, 1, np.uint64, n)
    leaf = _dump(pd, g, 2, np.uint8, n)
    groups = _dump(pd, g, 7, np.int32, 4 * ngroups).reshape(ngroups, 4)
    g.free()
    ctx.close()
    # a permutation of the input, coordinates carried along
    idx = pos[:, 3].astype(np.int64)
    assert np.array_equal(np.sort(idx), np.arange(n))
    assert np.array_equal(pos[:, :3], xyz[idx])
    # the codes are the definition's, sorted, ties in input order (stable)
    u = (xyz.astype(np.int64) - xyz.min(axis=0).astype(np.int64)) >> shift
    want = _spread(u[:, 0]) | (_spread(u[:, 1]) << np.uint64(1)) | (_spread(u[:, 2]) << np.uint64(2))
    assert np.array_equal(code, want[idx])
    assert np.all(code[1:] >= code[:-1])
    tie = code[1:] == code[:-1]
    assert np.all(idx[1:][tie] > idx[:-1][tie])
    # groups: tile [0, n) in order, inside one leaf, aligned to the leaf's start
    order = np.argsort(groups[:, 0], kind="stable")
    gs, gc, gl = groups[order, 0], groups[order, 1], groups[order, 2]
    assert gs[0] == 0 and np.all(gs[1:] == gs[:-1] + gc[:-1]) and gs[-1] + gc[-1] == n
    assert np.all((gc >= 1) & (gc <= 32)) and np.all(gl == leaf[gs])
    for s, c, lv in zip(gs.tolist(), gc.tolist(), gl.tolist()):
        pre = code[s:s + c] >> np.uint64(3 * lv)
        assert np.all(pre == pre[0]) and np.all(leaf[s:s + c] == lv)
        head = s == 0 or (code[s - 1] >> np.uint64(3 * lv)) != pre[0]
        if not head:   # a continuation: 32 points after the previous group of the leaf
            assert s >= 32 and (code[s - 32] >> np.uint64(3 * lv)) == pre[0]
    assert T <= 32
