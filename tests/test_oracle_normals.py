"""Pins of the normals oracle (no GPU).

Each check ties the oracle to something other than itself: the bit-level
definition of bfloat16 rounding, numpy's symmetric eigensolver, exact planes
and lines, central finite differences of the loss, Adam's closed form under
a constant gradient, and the published splitmix64 outputs.
"""
import os

import numpy as np
import pytest

import oracle
from oracle import normals as N
from paper_2311_17604_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- bfloat16
def _bf16_by_bits(f32):
    """Round float32 values to bfloat16 on their bit patterns: add 0x7fff plus
    the lowest kept bit, then drop the low 16 bits (round to nearest even)."""
    u = np.asarray(f32, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def test_round_bf16_special_values():
    one = 1.0
    assert N.round_bf16(one + 2.0 ** -8) == one                    # tie -> even (down)
    assert N.round_bf16(one + 3 * 2.0 ** -8) == one + 2.0 ** -6    # tie -> even (up)
    assert N.round_bf16(one + 2.0 ** -8 + 2.0 ** -30) == one + 2.0 ** -7
    assert N.round_bf16(-(one + 3 * 2.0 ** -8)) == -(one + 2.0 ** -6)
    assert N.round_bf16(0.0) == 0.0
    assert N.round_bf16(1.5 * 2.0 ** -133) == 2.0 ** -132          # subnormal tie -> even


def test_round_bf16_matches_bit_rounding_on_float32_values():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(200000), rng.uniform(-4, 4, 200000),
                        rng.standard_normal(1000) * 1e-30]).astype(np.float32)
    assert np.array_equal(N.round_bf16(x.astype(np.float64)), _bf16_by_bits(x))


# ---------------------------------------------------------------- eigenvectors
def test_smallest_eigvec_matches_numpy_eigh():
    rng = np.random.default_rng(1)
    Q, _ = np.linalg.qr(rng.standard_normal((500, 3, 3)))
    lam = np.sort(rng.uniform(0.1, 10, (500, 3)), axis=1)
    lam[:, 1] += 0.5  # well-separated smallest eigenvalue
    lam[:, 2] += 1.0
    A = np.einsum("nij,nj,nkj->nik", Q, lam, Q)
    v, ok = N.smallest_eigvec(A)
    assert ok.all()
    w, V = np.linalg.eigh(A)
    ref = V[:, :, 0]
    assert np.all(np.abs((v * ref).sum(1)) > 1 - 1e-10)
    assert np.allclose(np.linalg.norm(v, axis=1), 1.0)


def test_smallest_eigvec_diagonal_and_repeated():
    v, ok = N.smallest_eigvec(np.diag([3.0, 1.0, 2.0])[None])
    assert ok[0] and abs(abs(v[0, 1]) - 1.0) < 1e-15
    # repeated smallest eigenvalue: no unique normal
    _, ok = N.smallest_eigvec(np.diag([1.0, 1.0, 5.0])[None])
    assert not ok[0]


def test_pca_normal_of_exact_planes_and_lines():
    rng = np.random.default_rng(2)
    # integer points on the plane x + 2y + 3z = 0 (basis (-2,1,0), (-3,0,1))
    a = rng.integers(-300, 300, 3000)
    b = rng.integers(-300, 300, 3000)
    pts = np.stack([-2 * a - 3 * b, a, b], axis=1)
    pts = np.unique(pts, axis=0).astype(np.int32)
    _, v, ok, planar = N.features_and_pca(pts)
    nrm = np.array([1.0, 2.0, 3.0]) / np.sqrt(14.0)
    assert ok.all() and planar.all()
    assert np.all(N.angle(v, nrm[None]) < 1e-7)
    # collinear points: no normal
    line = np.stack([np.arange(40) * 3, np.arange(40) * 5, np.arange(40) * 7], 1).astype(np.int32)
    _, _, ok, _ = N.features_and_pca(line)
    assert not ok.any()


def test_planarity_flag():
    rng = np.random.default_rng(8)
    blob = rng.integers(-1000, 1000, (2000, 3)).astype(np.int32)   # isotropic: not planar
    _, _, ok, planar = N.features_and_pca(blob)
    assert ok.mean() > 0.99 and planar.mean() < 0.01
    # a slab 2000 x 2000 x 10 mm: planar almost everywhere
    slab = np.stack([rng.integers(0, 2000, 4000), rng.integers(0, 2000, 4000),
                     rng.integers(0, 10, 4000)], 1).astype(np.int32)
    _, v, ok, planar = N.features_and_pca(slab)
    assert planar.mean() > 0.9
    assert np.median(N.angle(v[planar], np.array([[0.0, 0.0, 1.0]]))) < 0.1


def test_pca_close_to_analytic_normals_on_room_scan():
    s = synth.room_scan(seed=4, n_az=240, n_el=60, normals=True, noise_mm=0.0)
    _, v, ok, _ = N.features_and_pca(s.xyz)
    ang = N.angle(v[ok], s.normals[ok])
    # noise-free walls: PCA is the wall normal except where 16-NN straddle an edge
    assert np.median(ang) < 1e-3
    assert np.mean(ang < np.deg2rad(5)) > 0.8


# ---------------------------------------------------------------- features
def test_features_are_scaled_offsets_in_knn_order():
    xyz = synth.random_cloud(5, 400, 3000)
    feat, _, _, _ = N.features_and_pca(xyz)
    # brute force: 16 nearest by (d^2, index)
    x = xyz.astype(np.int64)
    for p in (0, 17, 399):
        d2 = ((x - x[p]) ** 2).sum(1)
        d2[p] = np.iinfo(np.int64).max
        order = np.lexsort((np.arange(len(x)), d2))[:16]
        off = (x[order] - x[p]).astype(np.float64)
        rms = np.sqrt((off ** 2).sum() / 16)
        assert np.array_equal(feat[p], N.round_bf16((off / rms).ravel()))
        # rounded rows still have mean squared length 1 within bf16 rounding
        assert abs((feat[p] ** 2).sum() / 16 - 1.0) < 2e-2


def test_features_of_tiny_clouds_are_padded():
    xyz = np.array([[0, 0, 0], [10, 0, 0], [0, 20, 0]], dtype=np.int32)
    feat, v, ok, _ = N.features_and_pca(xyz)
    assert np.all(feat[:, 6:] == 0)
    assert not ok.any()   # two neighbours: no PCA normal


# ---------------------------------------------------------------- network
def _rand_params(seed):
    return N.init_params(seed).astype(np.float64) + \
        np.random.default_rng(seed).normal(0, 0.02, N.N_PARAMS)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(6)
    p = _rand_params(3)
    x = rng.standard_normal((40, N.NF))
    y = rng.standard_normal((40, 3))
    y /= np.linalg.norm(y, axis=1, keepdims=True)
    _, g = N.grad(p, x, y, rounded=False)
    idx = np.concatenate([rng.choice(N.O_B1, 40, replace=False),
                          np.arange(N.O_B1, N.O_B1 + 5),
                          N.O_W2 + rng.choice(N.NH * N.NH, 40, replace=False),
                          np.arange(N.O_B2, N.O_B2 + 5),
                          N.O_W3 + rng.choice(3 * N.NH, 30, replace=False),
                          np.arange(N.O_B3, N.N_PARAMS)])
    h = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        fd = (N.loss(p + e, x, y, False) - N.loss(p - e, x, y, False)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 + 1e-5 * abs(g[i]), (i, fd, g[i])


def test_loss_is_sign_and_scale_invariant():
    rng = np.random.default_rng(7)
    p = _rand_params(4)
    x = rng.standard_normal((64, N.NF))
    y = rng.standard_normal((64, 3))
    y /= np.linalg.norm(y, axis=1, keepdims=True)
    assert np.isclose(N.loss(p, x, y), N.loss(p, x, -y))
    # the network's own normals give zero loss
    _, _, _, u = N.forward(p, x)
    assert N.loss(p, x, u) < 1e-12
    # scaling the last layer does not change the normals
    q = p.copy()
    q[N.O_W3:] *= 2.0
    assert np.isclose(N.loss(p, x, y), N.loss(q, x, y))


def test_adam_closed_form_under_constant_gradient():
    p0 = np.linspace(-1, 1, 11)
    g = np.linspace(-3, 2, 11)
    p, m, v = p0.copy(), np.zeros(11), np.zeros(11)
    lr = 1e-2
    for t in range(1, 6):
        p, m, v = N.adam_step(p, m, v, g, t, lr)
        # bias correction makes m_hat = g and v_hat = g^2 exactly
        step = lr * g / (np.abs(g) + 1e-8)
        assert np.allclose(p, p0 - t * step, rtol=0, atol=1e-12)


def test_splitmix64_published_outputs():
    ref = [int(l) for l in open(os.path.join(GOLDEN, "splitmix64_seed1234567.txt"))
           if l.strip() and not l.startswith("#")]
    gamma = 0x9E3779B97F4A7C15
    got = [N.splitmix64((1234567 + i * gamma) & N.MASK64) for i in range(5)]
    assert got == ref


def test_init_params_ranges():
    p = N.init_params(11)
    assert p.dtype == np.float32 and p.shape == (N.N_PARAMS,)
    w1 = p[N.O_W1:N.O_B1]
    assert np.abs(w1).max() <= np.sqrt(6 / 48) and np.abs(w1).max() > 0.9 * np.sqrt(6 / 48)
    assert np.all(p[N.O_B1:N.O_W2] == 0) and np.all(p[N.O_B3:] == 0)
    assert abs(w1.mean()) < 0.02   # uniform, zero mean
