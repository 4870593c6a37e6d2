"""Packed batches: many scans decimated as one grid (needs a GPU).

pd_decimate_batch with PD_BATCH_PACKED moves every scan into its own tile of
one cloud and runs one grid build, one first neighbour pass and one sequence
of removal rounds for all of them; only the removal threshold of a round is
selected per scan.  For the density cost every scan must get exactly its
stand-alone result, which is the oracle's sequential greedy (section
"Sub-sampling algorithm").  With the colour term (section "Additional cost
terms") the rounds differ from a scan's own, so the retained sets are checked
against the oracle within the term's tolerance (>= 99.9 % agreement).
Batches that cannot be packed fall back to slots and still give the
stand-alone results.
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
    c = pd.Context()
    yield c
    c.close()


def _room_scans(seed=3, count=7, n_lo=2e4, n_hi=3e5):
    out = []
    for sp in synth.batch_specs(seed=seed, count=count, n_lo=n_lo, n_hi=n_hi):
        s = synth.room_scan(seed=sp["seed"], n_az=sp["n_az"], n_el=sp["n_el"], dims=sp["dims"],
                            scanner=sp["scanner"], rgb=True)
        out.append((s.xyz, s.rgb, sp["ratio"]))
    return out


def _alone(pd, ctx, xyz, rgb, m, **kw):
    g = pd.Grid(ctx, torch.from_numpy(xyz).cuda(),
                rgb=torch.from_numpy(rgb).cuda() if rgb is not None else None)
    keep = pd.pd_decimate_count(g, m, **kw).cpu().numpy()
    g.free()
    return keep


def _packed(pd, ctx, scans, **kw):
    clouds = [{"xyz": torch.from_numpy(x).cuda(),
               "rgb": torch.from_numpy(r).cuda() if r is not None else None, "ratio": q}
              for x, r, q in scans]
    keeps, stats = pd.pd_decimate_batch(ctx, clouds, concurrency=pd.PD_BATCH_PACKED, **kw)
    return [k.cpu().numpy() for k in keeps], stats


@pytest.mark.parametrize("k", [1, 4])
def test_packed_equals_alone_and_oracle(pd, ctx, k):
    scans = _room_scans()
    # a random cloud with coincident points and equal distances, and a line
    # lattice of equal costs (index ties), beside the room scans
    rc = synth.random_cloud(11, 30000, 40)
    scans.append((rc, None, 0.3))
    scans.append((synth.lattice_line(5000, step=9), None, 0.45))
    keeps, stats = _packed(pd, ctx, scans, k=k)
    assert stats[0]["rounds"] > 0
    for (x, r, q), got, st in zip(scans, keeps, stats):
        m = oracle.target_count(x.shape[0], q)
        assert int(got.sum()) == m and st["m"] == m and st["n"] == x.shape[0]
        assert np.array_equal(got, _alone(pd, ctx, x, None, m, k=k))
        assert np.array_equal(got, oracle.decimate(x, k, m))


def test_packed_many_small_scans(pd, ctx):
    """600 scans (16 tiles per axis), 300-3000 points each, spreads from 2 m
    to 20 m, k = 1 and keep 10-60 %: every retained set is the oracle's."""
    rng = np.random.default_rng(5)
    scans = []
    for i in range(600):
        n = int(rng.integers(300, 3000))
        span = int(rng.integers(2000, 20000))
        scans.append((synth.random_cloud(1000 + i, n, span), None, float(rng.uniform(0.1, 0.6))))
    keeps, _ = _packed(pd, ctx, scans, k=1)
    for (x, _, q), got in zip(scans, keeps):
        m = oracle.target_count(x.shape[0], q)
        assert np.array_equal(got, oracle.decimate(x, 1, m))


@pytest.mark.parametrize("k", [1, 4])
def test_packed_colour_within_tolerance(pd, ctx, k):
    scans = _room_scans(seed=8, count=5, n_lo=2e4, n_hi=1.2e5)
    kw = dict(k=k, term=pd.PD_TERM_COLOR, weight=0.3)
    keeps, _ = _packed(pd, ctx, scans, **kw)
    for (x, r, q), got in zip(scans, keeps):
        m = oracle.target_count(x.shape[0], q)
        assert int(got.sum()) == m
        ref = oracle.decimate(x, k, m, term=oracle.TERM_COLOR, a=0.3, rgb=r)
        agree = float((got == ref).mean())
        assert agree >= 0.999, agree


def test_packed_orientation_within_tolerance(pd, ctx):
    """The orientation term (Eq. 13, w = 1 - 0.5 (1 - |n_p . n_q|)) with the
    generator's analytic normals, packed per scan with the coordinates."""
    scans, clouds = [], []
    for sp in synth.batch_specs(seed=12, count=4, n_lo=2e4, n_hi=8e4):
        sc = synth.room_scan(seed=sp["seed"], n_az=sp["n_az"], n_el=sp["n_el"], dims=sp["dims"],
                             scanner=sp["scanner"], normals=True)
        scans.append((sc, sp["ratio"]))
        clouds.append({"xyz": torch.from_numpy(sc.xyz).cuda(),
                       "normals": torch.from_numpy(sc.normals).cuda(), "ratio": sp["ratio"]})
    keeps, _ = pd.pd_decimate_batch(ctx, clouds, k=4, term=pd.PD_TERM_ORIENT, weight=0.5,
                                    concurrency=pd.PD_BATCH_PACKED)
    for (sc, q), kp in zip(scans, keeps):
        m = oracle.target_count(sc.n, q)
        got = kp.cpu().numpy()
        assert int(got.sum()) == m
        ref = oracle.decimate(sc.xyz, 4, m, term=oracle.TERM_ORIENT, a=0.5, nrm=sc.normals)
        agree = float((got == ref).mean())
        assert agree >= 0.999, agree


def test_packed_fallbacks_give_alone_results(pd, ctx):
    """Not packable: a target of k points or fewer, or a scan with more
    coincident points than it must lose; the batch runs in slots."""
    base = _room_scans(seed=9, count=3, n_lo=2e4, n_hi=5e4)
    tiny = [(x, None, q) for x, _, q in base] + [(synth.random_cloud(3, 500, 3000), None, 0.003)]
    rnd = synth.random_cloud(4, 4000, 5000)
    doubled = [(base[0][0], None, 0.3), (np.concatenate([rnd, rnd]), None, 0.6)]
    for scans, k in ((tiny, 1), (doubled, 4)):
        keeps, _ = _packed(pd, ctx, scans, k=k)
        for (xx, _, q), got in zip(scans, keeps):
            m = oracle.target_count(xx.shape[0], q)
            assert np.array_equal(got, _alone(pd, ctx, xx, None, m, k=k))


def test_packed_rounds_settled_on_host(pd, ctx, monkeypatch):
    """Rounds of a packed batch that the device cannot settle: a danger-pair
    capacity of 8 (k = 4: each scan's largest key goes, per scan) and one
    fixpoint sweep (k = 1: the host finishes the fixpoint)."""
    scans = _room_scans(seed=10, count=3, n_lo=1e4, n_hi=2e4)
    for k, var, val in ((4, "PD_PAIR_CAP", "8"), (1, "PD_FIX_SWEEPS", "1")):
        monkeypatch.setenv(var, val)
        keeps, _ = _packed(pd, ctx, scans, k=k)
        monkeypatch.delenv(var)
        for (x, _, q), got in zip(scans, keeps):
            m = oracle.target_count(x.shape[0], q)
            assert np.array_equal(got, oracle.decimate(x, k, m))
