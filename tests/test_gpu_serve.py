"""The serving loop (pd_serve_*) on the GPU.

Scans submitted in a burst run concurrently through a few slots; each must get
exactly the result it gets alone (the workers share no device state, and the
density cost is exact, so the comparison is bit for bit), and the admission
rule must keep the scans running at any moment within the memory budget.
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
    return pdm


@pytest.fixture(scope="module")
def ctx(pd):
    c = pd.Context(use_torch_allocator=False)
    yield c
    c.close()


def _scans(count=8, seed=11):
    out = []
    for sp in synth.batch_specs(seed=seed, count=count, n_lo=2e4, n_hi=4e5):
        s = synth.room_scan(seed=sp["seed"], n_az=sp["n_az"], n_el=sp["n_el"], dims=sp["dims"],
                            scanner=sp["scanner"])
        out.append((s.xyz, sp["ratio"]))
    return out


def _alone(pd, ctx, xyz, m, k, term=0, weight=0.0, params=None):
    g = pd.Grid(ctx, torch.from_numpy(xyz).cuda())
    nrm = None
    if term == pd.PD_TERM_ORIENT:
        feat, pca, _ = pd.pd_normals_pca(g)
        nrm = pd.pd_normals_mlp(ctx, params, feat, pca)
    keep = pd.pd_decimate_count(g, m, k=k, term=term, weight=weight, normals=nrm)
    g.free()
    return keep.cpu().numpy()


@pytest.mark.parametrize("k", [1, 4])
def test_served_results_equal_alone(pd, ctx, k):
    scans = _scans()
    srv = pd.Server(ctx, slots=3, k=k)
    pinned = [pd.pinned_like(x) for x, _ in scans]
    tickets = [srv.submit(p, ratio=r) for p, (_, r) in zip(pinned, scans)]
    results = [srv.poll(t) for t in tickets]
    srv.close()
    for (x, r), (keep, res) in zip(scans, results):
        m = oracle.target_count(x.shape[0], r)
        assert res["status"] == pd.PD_OK and res["m"] == m and int(keep.sum()) == m
        assert res["t_submit_ms"] <= res["t_admit_ms"] <= res["t_done_ms"]
        assert np.array_equal(keep, _alone(pd, ctx, x, m, k))
    # the smallest scan against the oracle itself
    i = int(np.argmin([x.shape[0] for x, _ in scans]))
    x, r = scans[i]
    assert np.array_equal(results[i][0], oracle.decimate(x, k, oracle.target_count(x.shape[0], r)))


def test_served_orientation_term_with_network_normals_equals_alone(pd, ctx):
    train = synth.room_scan(seed=31, n_az=300, n_el=80)
    g = pd.Grid(ctx, torch.from_numpy(train.xyz).cuda())
    feat, pca, valid = pd.pd_normals_pca(g)
    g.free()
    tr = pd.MlpTrainer(seed=2)
    tr.train(ctx, feat, pca, ((valid & pd.PD_NORMAL_PLANAR) != 0).to(torch.uint8), steps=200,
             batch=2048, lr=2e-3, seed=3)
    scans = _scans(count=5, seed=12)
    srv = pd.Server(ctx, slots=3, k=4, term=pd.PD_TERM_ORIENT, weight=0.5,
                    mlp_params=tr.params, normals=True)
    tickets = [srv.submit(pd.pinned_like(x), ratio=r) for x, r in scans]
    results = [srv.poll(t) for t in tickets]
    srv.close()
    for (x, r), (keep, res) in zip(scans, results):
        m = oracle.target_count(x.shape[0], r)
        assert res["status"] == pd.PD_OK and int(keep.sum()) == m
        alone = _alone(pd, ctx, x, m, 4, pd.PD_TERM_ORIENT, 0.5, tr.params)
        assert np.array_equal(keep, alone)


def test_admission_keeps_running_scans_within_budget(pd, ctx):
    scans = _scans(count=10, seed=13)
    est = [pd.PD_SERVE_BYTES_PER_POINT * x.shape[0] + (1 << 20) for x, _ in scans]
    budget = int(max(est) * 1.5)
    srv = pd.Server(ctx, slots=4, k=1, mem_budget=budget)
    tickets = [srv.submit(pd.pinned_like(x), ratio=r) for x, r in scans]
    res = [srv.poll(t)[1] for t in tickets]
    srv.close()
    assert all(r["status"] == pd.PD_OK for r in res)
    # FIFO: admission order is submission order
    admits = [r["t_admit_ms"] for r in res]
    assert admits == sorted(admits)
    # at every admission, the scans then running fit in the budget
    for i, r in enumerate(res):
        t = r["t_admit_ms"]
        run = sum(e for e, q in zip(est, res) if q["t_admit_ms"] <= t < q["t_done_ms"])
        assert run <= budget


def test_rejections(pd, ctx):
    x = synth.random_cloud(0, 50000, 3000)
    srv = pd.Server(ctx, slots=1, k=1, mem_budget=1 << 20)   # smaller than any scan's estimate
    with pytest.raises(pd.PdError) as e:
        srv.submit(x, ratio=0.5)
    assert e.value.code == pd.PD_ENOMEM
    with pytest.raises(pd.PdError) as e:
        srv.submit(x, m=x.shape[0] + 1)
    assert e.value.code == pd.PD_EINVAL
    srv.close()
    with pytest.raises(pd.PdError):
        pd.Server(ctx, term=pd.PD_TERM_ORIENT, weight=0.5)   # nothing would supply normals
