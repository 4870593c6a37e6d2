"""CUDA path against the oracle, through the C ABI (needs a GPU).

Density-only costs must give bit-identical results: the same k-nearest
squared-distance lists, the same binary64 costs, the same retained index set.
"""
import numpy as np
import pytest

import oracle
from paper_2311_17604_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pd():
    from paper_2311_17604_gb300 import build
    build.build()
    import paper_2311_17604_gb300.pd as pdm
    assert torch.cuda.is_available()
    return pdm


@pytest.fixture(scope="module")
def ctx(pd):
    c = pd.Context()
    yield c
    c.close()


def gpu_decimate(pd, ctx, xyz, k, m, leaf_max=0, **kw):
    g = pd.Grid(ctx, torch.from_numpy(np.ascontiguousarray(xyz)).cuda(), leaf_max=leaf_max)
    keep = pd.pd_decimate_count(g, m, k=k, **kw).cpu().numpy()
    st = g.stats()
    g.free()
    return keep, st


def gpu_knn(pd, ctx, xyz, k, leaf_max=0):
    g = pd.Grid(ctx, torch.from_numpy(np.ascontiguousarray(xyz)).cuda(), leaf_max=leaf_max)
    cost, knn = pd.pd_knn_cost(g, k=k)
    g.free()
    return cost.cpu().numpy(), knn.cpu().numpy()


def d2_of(xyz, idx):
    x = xyz.astype(np.int64)
    out = np.full(idx.shape, np.iinfo(np.int64).max, dtype=np.int64)
    ok = idx >= 0
    rows = np.nonzero(ok)
    diff = x[idx[rows]] - x[rows[0]]
    out[rows] = (diff * diff).sum(axis=1)
    return out


def assert_keep_equal(keep, ref, what):
    bad = np.nonzero(keep != ref)[0]
    assert len(bad) == 0, "%s: %d points differ (first %s)" % (what, len(bad), bad[:10])


# ---------------------------------------------------------------- kNN / cost
@pytest.mark.parametrize("k", [1, 4, 8, 16])
@pytest.mark.parametrize("case", ["dense", "sparse", "plane", "room"])
def test_knn_cost_bit_exact(pd, ctx, k, case):
    if case == "dense":
        x = synth.random_cloud(1, 4000, 30)            # many duplicates and ties
    elif case == "sparse":
        x = synth.random_cloud(2, 3000, 200000)        # 3 points per 10^13 mm^3
    elif case == "plane":
        x = synth.random_cloud(3, 5000, 700, dims=2)
    else:
        x = synth.room_scan(seed=0, n_az=160, n_el=40).xyz
    cost, knn = gpu_knn(pd, ctx, x, k)
    d2r, _, costr = oracle.knn_cost(x, k)
    assert np.array_equal(d2_of(x, knn), d2r)
    assert np.array_equal(cost.view(np.int64), costr.view(np.int64))


@pytest.mark.parametrize("leaf_max", [4, 9, 32])
def test_knn_independent_of_cell_size(pd, ctx, leaf_max):
    x = synth.room_scan(seed=1, n_az=200, n_el=50).xyz
    cost, knn = gpu_knn(pd, ctx, x, 4, leaf_max=leaf_max)
    d2r, _, costr = oracle.knn_cost(x, 4)
    assert np.array_equal(d2_of(x, knn), d2r)
    assert np.array_equal(cost, costr)


# ---------------------------------------------------------------- decimation
@pytest.mark.parametrize("k", [1, 2, 4])
@pytest.mark.parametrize("seed,n,span", [(0, 500, 40), (1, 3000, 1000), (2, 6000, 25),
                                          (3, 20000, 5000)])
def test_decimate_random_bit_exact(pd, ctx, k, seed, n, span):
    x = synth.random_cloud(seed, n, span)
    for ratio in (0.1, 0.5, 0.9):
        m = oracle.target_count(n, ratio)
        keep, _ = gpu_decimate(pd, ctx, x, k, m)
        assert_keep_equal(keep, oracle.decimate(x, k, m), "k=%d ratio=%g" % (k, ratio))


@pytest.mark.parametrize("k", [1, 4])
def test_decimate_room_small(pd, ctx, k):
    s = synth.room_scan(seed=3, n_az=500, n_el=100)
    m = oracle.target_count(s.n, 0.25)
    keep, st = gpu_decimate(pd, ctx, s.xyz, k, m)
    assert int(keep.sum()) == m
    assert_keep_equal(keep, oracle.decimate(s.xyz, k, m), "room k=%d" % k)


def test_decimate_room_200k_k1(pd, ctx):
    """The 200k-point room scan, k = 1, keep 25 %: bit-identical to the oracle."""
    s = synth.room_scan(**synth.ROOM_200K)
    m = oracle.target_count(s.n, 0.25)
    keep, st = gpu_decimate(pd, ctx, s.xyz, 1, m)
    assert_keep_equal(keep, oracle.decimate(s.xyz, 1, m), "room 200k k=1")


def test_decimate_room_200k_k4(pd, ctx):
    s = synth.room_scan(**synth.ROOM_200K)
    m = oracle.target_count(s.n, 0.1)
    keep, st = gpu_decimate(pd, ctx, s.xyz, 4, m)
    assert_keep_equal(keep, oracle.decimate(s.xyz, 4, m), "room 200k k=4")


def test_decimate_outdoor_small_k4(pd, ctx):
    s = synth.outdoor_scan(seed=0, n_az=2000, n_el=400)
    m = oracle.target_count(s.n, 0.1)
    keep, st = gpu_decimate(pd, ctx, s.xyz, 4, m)
    assert_keep_equal(keep, oracle.decimate(s.xyz, 4, m), "outdoor k=4")


# ---------------------------------------------------------------- edge cases
def test_edge_cases(pd, ctx):
    one = np.array([[5, 6, 7]], np.int32)
    for m in (0, 1):
        keep, _ = gpu_decimate(pd, ctx, one, 1, m)
        assert keep.tolist() == [m]
    two = np.array([[0, 0, 0], [3, 4, 0]], np.int32)
    for k in (1, 4):
        keep, _ = gpu_decimate(pd, ctx, two, k, 1)
        assert keep.tolist() == [1, 0]          # equal costs: larger index goes
    dup = np.zeros((50, 3), np.int32)           # all coincident
    for m in (0, 1, 7, 50):
        for k in (1, 3):
            keep, _ = gpu_decimate(pd, ctx, dup, k, m)
            assert_keep_equal(keep, oracle.decimate(dup, k, m), "dups m=%d k=%d" % (m, k))
    line = synth.lattice_line(300)
    keep, _ = gpu_decimate(pd, ctx, line, 1, 100)
    assert np.nonzero(keep)[0].tolist() == list(range(100))
    x = synth.random_cloud(5, 1000, 100)
    for k in (1, 4):
        for m in (0, 1000):
            keep, _ = gpu_decimate(pd, ctx, x, k, m)
            assert int(keep.sum()) == m


def test_errors(pd, ctx):
    big = np.array([[0, 0, 0], [1 << 25, 0, 0]], np.int32)
    with pytest.raises(pd.PdError) as e:
        pd.Grid(ctx, torch.from_numpy(big).cuda())
    assert e.value.code == pd.PD_ERANGE
    x = torch.from_numpy(synth.random_cloud(0, 100, 50)).cuda()
    g = pd.Grid(ctx, x)
    for bad in (dict(m=-1), dict(m=101), dict(m=10, k=0), dict(m=10, k=17)):
        with pytest.raises(pd.PdError) as e:
            pd.pd_decimate_count(g, bad.pop("m"), **bad)
        assert e.value.code == pd.PD_EINVAL
    g.free()


def test_ratio_and_host_entry(pd, ctx):
    s = synth.room_scan(seed=4, n_az=300, n_el=80)
    ratio = 0.3
    m = oracle.target_count(s.n, ratio)
    ref = oracle.decimate(s.xyz, 1, m)
    g = pd.Grid(ctx, torch.from_numpy(s.xyz).cuda())
    keep = pd.pd_decimate_ratio(g, ratio, k=1).cpu().numpy()
    g.free()
    assert_keep_equal(keep, ref, "ratio")
    keep2, st = pd.pd_decimate_host(ctx, s.xyz, m, k=1)
    assert_keep_equal(keep2, ref, "host entry")
    assert st["n"] == s.n and st["m"] == m
