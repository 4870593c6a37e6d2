"""Normals for the orientation term on the GPU against the normals oracle.

Features are bit-exact (exact integer offsets, one rounding to bfloat16 on
both sides).  PCA normals agree to 1e-6 rad wherever the smallest eigenvalue
is well separated (elsewhere the normal itself is ill-conditioned).  The
network runs bfloat16 operands with float32 accumulation on the tensor cores
against the oracle's binary64 sums of the same bfloat16 values, so outputs and
gradients agree to a few bfloat16 rounding units (2^-8), not bit for bit.
"""
import numpy as np
import pytest

import oracle
from oracle import normals as N
from paper_2311_17604_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U_BF16 = 2.0 ** -8


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


def _gpu_features(pd, ctx, xyz):
    g = pd.Grid(ctx, torch.from_numpy(xyz).cuda())
    feat, pca, valid = pd.pd_normals_pca(g)
    g.free()
    return feat, pca, valid


def _feat_values(feat):
    return N.bf16_from_bits(feat.cpu().numpy().view(np.uint16))


def _well_conditioned(xyz, idx=None, gap=1e-3):
    """Points whose neighbour covariance has a simple, well-separated
    smallest eigenvalue (relative gap > gap)."""
    if idx is None:
        k = min(16, xyz.shape[0] - 1)
        _, idx, _ = oracle.knn_cost(xyz, k)
    x = xyz.astype(np.float64)
    have = idx >= 0
    off = np.where(have[..., None], x[np.maximum(idx, 0)] - x[:, None], 0.0)
    m = np.maximum(have.sum(1), 1)
    mean = off.sum(1) / m[:, None]
    cen = np.where(have[..., None], off - mean[:, None], 0.0)
    w = np.linalg.eigvalsh(np.einsum("nia,nib->nab", cen, cen))
    return (w[:, 1] - w[:, 0]) > gap * np.maximum(w[:, 2], 1e-300)


CLOUDS = {
    "room_14k": lambda: synth.room_scan(seed=2, n_az=240, n_el=60).xyz,
    "dups_ties": lambda: synth.random_cloud(3, 5000, 30),           # many coincident points
    "lattice_line": lambda: synth.lattice_line(200),                 # collinear: no normals
    "tiny": lambda: np.array([[0, 0, 0], [5, 0, 0], [0, 7, 0], [0, 0, 9], [3, 3, 3]], np.int32),
    "seventeen": lambda: synth.random_cloud(9, 17, 100),
}


@pytest.mark.parametrize("name", sorted(CLOUDS))
def test_features_bit_exact_and_pca_close(pd, ctx, name):
    xyz = CLOUDS[name]()
    feat, pca, valid = _gpu_features(pd, ctx, xyz)
    ref_feat, ref_pca, ref_ok, ref_planar = N.features_and_pca(xyz)
    assert np.array_equal(_feat_values(feat), ref_feat)
    flags = valid.cpu().numpy()
    ok = (flags & pd.PD_NORMAL_DEFINED) != 0
    planar = (flags & pd.PD_NORMAL_PLANAR) != 0
    good = _well_conditioned(xyz) & ref_ok
    assert np.array_equal(ok[good], ref_ok[good])
    # planarity is a threshold on a ratio: rows right at it may differ
    assert np.mean(planar[good] == ref_planar[good]) >= 0.999 if good.any() else True
    assert not (planar & ~ok).any()
    ang = N.angle(pca.cpu().numpy()[good], ref_pca[good])
    assert ang.size == 0 or ang.max() < 1e-6
    nrm = np.linalg.norm(pca.cpu().numpy()[ok], axis=1)
    assert np.allclose(nrm, 1.0, atol=1e-6)
    assert np.all(pca.cpu().numpy()[~ok] == 0)


def test_init_is_bit_exact(pd):
    for seed in (0, 7, 2 ** 40 + 3):
        p = pd.pd_mlp_init(seed).cpu().numpy()
        assert np.array_equal(p.view(np.uint32), N.init_params(seed).view(np.uint32))


def _perturbed_params(pd, seed):
    p = pd.pd_mlp_init(seed)
    gen = torch.Generator(device="cpu").manual_seed(seed)
    p += (0.05 * torch.randn(pd.PD_MLP_PARAMS, generator=gen)).cuda()
    return p


def _room(seed, n_az, n_el, normals=False):
    return synth.room_scan(seed=seed, n_az=n_az, n_el=n_el, normals=normals)


def test_forward_matches_oracle(pd, ctx):
    xyz = _room(5, 300, 80).xyz
    feat, _, _ = _gpu_features(pd, ctx, xyz)
    p = _perturbed_params(pd, 1)
    u, nr = pd.pd_mlp_forward(p, feat)
    _, _, o, ref_u = N.forward(p.cpu().numpy().astype(np.float64), _feat_values(feat))
    ang = N.angle(u.cpu().numpy(), ref_u)
    assert np.median(ang) < U_BF16 / 4 and ang.max() < 4 * U_BF16
    rel = np.abs(nr.cpu().numpy() - np.linalg.norm(o, axis=1)) / np.linalg.norm(o, axis=1)
    assert np.median(rel) < U_BF16 / 4 and rel.max() < 4 * U_BF16
    # ragged tail: every row count gives the same rows
    for n in (1, 15, 17, 1000, 4099):
        u2, _ = pd.pd_mlp_forward(p, feat[:n].contiguous())
        assert torch.equal(u2, u[:n])


def test_gradient_matches_oracle(pd, ctx):
    xyz = _room(6, 200, 60).xyz
    feat, pca, valid = _gpu_features(pd, ctx, xyz)
    keep = valid.bool()
    feat, pca = feat[keep].contiguous(), pca[keep].contiguous()
    p = _perturbed_params(pd, 2)
    loss, g = pd.pd_mlp_grad(ctx, p, feat, pca)
    ref_loss, ref_g = N.grad(p.cpu().numpy().astype(np.float64), _feat_values(feat),
                             pca.cpu().numpy().astype(np.float64))
    assert abs(loss - ref_loss) <= 1e-3 * ref_loss
    g = g.cpu().numpy().astype(np.float64)
    for lo, hi in ((N.O_W1, N.O_B1), (N.O_B1, N.O_W2), (N.O_W2, N.O_B2), (N.O_B2, N.O_W3),
                   (N.O_W3, N.O_B3), (N.O_B3, N.N_PARAMS)):
        err = np.linalg.norm(g[lo:hi] - ref_g[lo:hi]) / np.linalg.norm(ref_g[lo:hi])
        assert err < 2 * U_BF16, (lo, err)


def test_adam_steps_match_oracle(pd, ctx):
    xyz = _room(7, 160, 50).xyz
    feat, pca, valid = _gpu_features(pd, ctx, xyz)
    p0 = _perturbed_params(pd, 3)
    tr = pd.MlpTrainer(params=p0.clone())
    lr, steps = 1e-3, 6
    losses = tr.train(ctx, feat, pca, valid, steps=steps, batch=300, lr=lr, seed=99)
    ref_p, ref_l = N.train(p0.cpu().numpy(), _feat_values(feat), pca.cpu().numpy(),
                           valid.cpu().numpy().astype(bool), steps, 300, lr, seed=99)
    assert np.allclose(losses.cpu().numpy(), ref_l, rtol=2e-3)
    d_gpu = tr.params.cpu().numpy().astype(np.float64) - p0.cpu().numpy()
    d_ref = ref_p - p0.cpu().numpy().astype(np.float64)
    # Adam's step is ~lr * sign(g) early on: parameters with a near-zero
    # gradient may move differently; all others move alike
    close = np.abs(d_gpu - d_ref) <= 0.1 * lr * steps
    assert close.mean() > 0.98


def test_training_is_reproducible(pd, ctx):
    xyz = _room(9, 160, 50).xyz
    feat, pca, valid = _gpu_features(pd, ctx, xyz)
    runs = []
    for _ in range(2):
        tr = pd.MlpTrainer(seed=5)
        losses = tr.train(ctx, feat, pca, valid, steps=20, batch=1000, lr=1e-3, seed=7)
        runs.append((tr.params.clone(), losses.clone()))
    assert torch.equal(runs[0][0], runs[1][0]) and torch.equal(runs[0][1], runs[1][1])
    g1 = pd.pd_mlp_grad(ctx, runs[0][0], feat, pca)[1]
    g2 = pd.pd_mlp_grad(ctx, runs[0][0], feat, pca)[1]
    assert torch.equal(g1, g2)


def test_fallback_rules(pd, ctx):
    xyz = _room(8, 120, 40).xyz
    feat, pca, _ = _gpu_features(pd, ctx, xyz)
    p = pd.pd_mlp_init(5)
    assert torch.equal(pd.pd_normals_mlp(ctx, None, feat, pca), pca)
    assert torch.equal(pd.pd_normals_mlp(ctx, p, feat, pca, min_norm=1e30), pca)
    u, nr = pd.pd_mlp_forward(p, feat)
    out = pd.pd_normals_mlp(ctx, p, feat, pca)
    use = (nr >= 1e-3)[:, None]
    assert torch.equal(out, torch.where(use, u, pca))
    # zeroed last layer: every raw output is 0, so all rows fall back
    z = p.clone()
    z[pd.PD_MLP_PARAMS - 3 * 64 - 3:] = 0
    assert torch.equal(pd.pd_normals_mlp(ctx, z, feat, pca), pca)


@pytest.fixture(scope="module")
def trained(pd, ctx):
    """A network trained on the planar rows' PCA normals of one room scan."""
    train = _room(21, 500, 100)
    feat, pca, valid = _gpu_features(pd, ctx, train.xyz)
    planar = ((valid & pd.PD_NORMAL_PLANAR) != 0).to(torch.uint8)
    tr = pd.MlpTrainer(seed=4)
    losses = tr.train(ctx, feat, pca, planar, steps=2000, batch=4096, lr=2e-3, seed=1)
    return tr, losses.cpu().numpy()


def test_training_lowers_the_loss(trained):
    _, losses = trained
    assert losses[-50:].mean() < 0.2 * losses[:10].mean()


def test_trained_network_gain(pd, ctx, trained):
    """What the learned normals add: on a scan the network has not seen they
    match PCA on planar patches, are closer than PCA to the true normals at
    creases (where the 16-NN straddle two faces and PCA blends them), and the
    orientation term fed with them keeps more crease points than the density
    cost alone and than the same term fed with PCA normals."""
    tr, _ = trained
    s = _room(22, 800, 200, normals=True)
    feat, pca, valid = _gpu_features(pd, ctx, s.xyz)
    flags = valid.cpu().numpy()
    ok = (flags & pd.PD_NORMAL_DEFINED) != 0
    planar = (flags & pd.PD_NORMAL_PLANAR) != 0
    mlp = pd.pd_normals_mlp(ctx, tr.params, feat, pca)
    untrained = pd.pd_normals_mlp(ctx, pd.pd_mlp_init(4), feat, pca)
    mlp_h, pca_h = mlp.cpu().numpy(), pca.cpu().numpy()
    assert np.median(N.angle(mlp_h[planar], pca_h[planar])) < np.deg2rad(3)
    assert np.median(N.angle(untrained.cpu().numpy()[planar], pca_h[planar])) > np.deg2rad(30)
    _, idx, _ = oracle.knn_cost(s.xyz, 16)
    dots = np.abs((s.normals[idx] * s.normals[:, None]).sum(-1))
    crease = (dots < np.cos(np.deg2rad(45))).any(1) & ok
    a_mlp = np.median(N.angle(mlp_h[crease], s.normals[crease]))
    a_pca = np.median(N.angle(pca_h[crease], s.normals[crease]))
    assert a_mlp < 0.8 * a_pca, (np.degrees(a_mlp), np.degrees(a_pca))
    m = oracle.target_count(s.n, 0.05)
    xd = torch.from_numpy(s.xyz).cuda()
    keeps = {}
    for name, term, nrm in (("density", 0, None), ("pca", 2, pca), ("mlp", 2, mlp)):
        g = pd.Grid(ctx, xd)
        keeps[name] = pd.pd_decimate_count(g, m, k=4, term=term, weight=0.5,
                                           normals=nrm).cpu().numpy().astype(bool)
        g.free()
    kept = {k: float(v[crease].mean()) for k, v in keeps.items()}
    assert kept["mlp"] > kept["density"] + 0.015, kept
    assert kept["mlp"] > kept["pca"] + 0.005, kept


def test_orientation_term_with_network_normals_matches_oracle(pd, ctx, trained):
    tr, _ = trained
    s = _room(23, 300, 100)
    feat, pca, _ = _gpu_features(pd, ctx, s.xyz)
    mlp = pd.pd_normals_mlp(ctx, tr.params, feat, pca)
    m = oracle.target_count(s.n, 0.25)
    xd = torch.from_numpy(s.xyz).cuda()
    g = pd.Grid(ctx, xd)
    cost, _ = pd.pd_knn_cost(g, k=4, term=2, weight=0.5, normals=mlp)
    g.free()
    nh = mlp.cpu().numpy()
    _, _, ref = oracle.knn_cost(s.xyz, 4, term=2, a=0.5, nrm=nh)
    c = cost.cpu().numpy()
    fin = np.isfinite(ref)
    assert np.array_equal(np.isfinite(c), fin)
    assert (np.abs(c[fin] - ref[fin]) / np.abs(ref[fin])).max() <= 1e-5
    g = pd.Grid(ctx, xd)
    keep = pd.pd_decimate_count(g, m, k=4, term=2, weight=0.5, normals=mlp).cpu().numpy()
    g.free()
    ref_keep = oracle.decimate(s.xyz, 4, m, term=2, a=0.5, nrm=nh)
    assert int(keep.sum()) == m
    assert (keep == ref_keep).mean() >= 0.999
