"""CPU oracle for the normals that feed the orientation term (Eq. 13).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline leg may import this module; the library itself never does.

The paper treats normals as part of the input (section "Additional cost
terms") and gives no estimator.  This module is the plain definition of the
one the library uses, in binary64 numpy:

  * neighbours: the 16 nearest other points, ascending (d^2, input index)
    (the kd-tree/brute-force kNN of ``pd_oracle.c``);
  * features: offsets q_i - p divided by their RMS length, each rounded once
    to bfloat16 (round to nearest, ties to even);
  * PCA normal: eigenvector of the smallest eigenvalue of the neighbours'
    covariance about their mean, eigenvalue by the trigonometric closed form
    of O. K. Smith (CACM 4(4), 1961), eigenvector as the longest cross
    product of two rows of (A - lambda I);
  * network 48 -> 64 -> 64 -> 3: h1 = relu(x W1^T + b1),
    h2 = relu(h1 W2^T + b2), o = h2 W3^T + b3, u = o / |o|, with the weights,
    x, h1 and h2 rounded to bfloat16 (``rounded=True``) and every product
    summed in binary64; loss 1 - (u . y)^2 averaged over the rows;
  * gradient by the chain rule written out layer by layer, rounding taken as
    the identity (``rounded=False`` turns the rounding off, and then the
    gradient is the exact derivative, which the tests pin by central finite
    differences);
  * Adam (Kingma & Ba, ICLR 2015) and the splitmix64 generator (Steele, Lea,
    Flood, OOPSLA 2014) that draws the initial weights and the training rows.
"""
from __future__ import annotations

import numpy as np

NF, NH, NOUT = 48, 64, 3
K_NORMAL = 16
# parameter vector layout
O_W1 = 0
O_B1 = O_W1 + NH * NF
O_W2 = O_B1 + NH
O_B2 = O_W2 + NH * NH
O_W3 = O_B2 + NH
O_B3 = O_W3 + NOUT * NH
N_PARAMS = O_B3 + NOUT
MASK64 = (1 << 64) - 1


# ---------------------------------------------------------------- rounding
def round_bf16(x):
    """Round binary64 values to the nearest bfloat16 (8 significant bits),
    ties to even; zeros, infinities and NaN pass through."""
    x = np.asarray(x, dtype=np.float64)
    _, e = np.frexp(x)                       # x = m 2^e, 0.5 <= |m| < 1
    # quantum 2^(e - 8); below 2^-126 the subnormal quantum 2^-133
    q = np.maximum(e, -125) - 8
    r = np.ldexp(np.rint(np.ldexp(x, -q)), q)
    return np.where(np.isfinite(x) & (x != 0), r, x)


def bf16_bits(x):
    """16-bit patterns of values that are exact bfloat16 numbers."""
    f = np.asarray(x, dtype=np.float32)
    return (f.view(np.uint32) >> 16).astype(np.uint16)


def bf16_from_bits(b):
    return (np.asarray(b, dtype=np.uint32) << 16).view(np.float32).astype(np.float64)


# ---------------------------------------------------------------- PCA and features
def smallest_eigvec(A, with_mid=False):
    """Unit eigenvector of the smallest eigenvalue of each symmetric 3x3 in A
    [..., 3, 3]; (vector, defined) with defined False when the longest row
    cross product of (A - lambda I) has length <= 1e-6 trace(A)^2 (a repeated
    smallest eigenvalue: the closed form's lambda is then only good to about
    the square root of the rounding error, so the products do not vanish).
    with_mid: also return the middle eigenvalue (closed form, j = 2)."""
    A = np.asarray(A, dtype=np.float64)
    a00, a01, a02 = A[..., 0, 0], A[..., 0, 1], A[..., 0, 2]
    a11, a12, a22 = A[..., 1, 1], A[..., 1, 2], A[..., 2, 2]
    p1 = a01 ** 2 + a02 ** 2 + a12 ** 2
    q = (a00 + a11 + a22) / 3.0
    p = np.sqrt(((a00 - q) ** 2 + (a11 - q) ** 2 + (a22 - q) ** 2 + 2.0 * p1) / 6.0)
    with np.errstate(invalid="ignore", divide="ignore"):
        B = (A - q[..., None, None] * np.eye(3)) / p[..., None, None]
        r = np.clip(np.linalg.det(B) / 2.0, -1.0, 1.0)
        # the three eigenvalues are q + 2 p cos(acos(r)/3 + 2 pi j/3), j = 0, 1, 2;
        # j = 1 gives the smallest
        phi = np.arccos(r) / 3.0
        lam = q + 2.0 * p * np.cos(phi + 2.0 * np.pi / 3.0)
        lmid = q + 2.0 * p * np.cos(phi + 4.0 * np.pi / 3.0)
    dmin = np.minimum(np.minimum(a00, a11), a22)
    dmax = np.maximum(np.maximum(a00, a11), a22)
    lam = np.where(p1 == 0.0, dmin, lam)
    lmid = np.where(p1 == 0.0, a00 + a11 + a22 - dmin - dmax, lmid)
    M = A - lam[..., None, None] * np.eye(3)
    rows = [M[..., 0, :], M[..., 1, :], M[..., 2, :]]
    cands = np.stack([np.cross(rows[0], rows[1]), np.cross(rows[0], rows[2]),
                      np.cross(rows[1], rows[2])], axis=-2)
    nn = (cands ** 2).sum(-1)
    best = np.argmax(nn, axis=-1)
    v = np.take_along_axis(cands, best[..., None, None], axis=-2)[..., 0, :]
    bn = np.take_along_axis(nn, best[..., None], axis=-1)[..., 0]
    tr = a00 + a11 + a22
    ok = bn > 1e-12 * tr ** 4
    with np.errstate(invalid="ignore", divide="ignore"):
        v = np.where(ok[..., None], v / np.sqrt(bn)[..., None], 0.0)
    if with_mid:
        return v, ok, lmid
    return v, ok


PLANAR_RATIO = 0.05


def features_and_pca(xyz, idx=None):
    """Feature rows (bfloat16 values as binary64, [n, 48]), PCA normals
    ([n, 3]), their validity ([n] bool) and planarity ([n] bool: defined and
    n^T C n <= PLANAR_RATIO * the middle eigenvalue of the covariance C) of
    every point.  idx: the 16 nearest neighbours ([n, 16] input indices, -1
    past the found ones); by default from the oracle kNN."""
    import oracle
    xyz = np.asarray(xyz)
    n = xyz.shape[0]
    if idx is None:
        k = min(K_NORMAL, max(n - 1, 1))
        _, idx, _ = oracle.knn_cost(xyz, k)
        if k < K_NORMAL:
            idx = np.concatenate([idx, np.full((n, K_NORMAL - k), -1, np.int32)], axis=1)
    idx = np.asarray(idx)
    have = idx >= 0
    m = have.sum(1)
    x = xyz.astype(np.int64)
    off = np.where(have[..., None], x[np.maximum(idx, 0)] - x[:, None, :], 0)   # exact
    ss = (off * off).sum((1, 2))                                                # exact int64
    with np.errstate(invalid="ignore", divide="ignore"):
        rms = np.sqrt(ss.astype(np.float64) / m)
        feat = np.where((rms > 0)[:, None, None], off / rms[:, None, None], 0.0)
    feat = round_bf16(feat.reshape(n, NF))
    # covariance about the neighbours' mean, binary64
    offd = off.astype(np.float64)
    with np.errstate(invalid="ignore", divide="ignore"):
        mean = offd.sum(1) / m[:, None]
    cen = np.where(have[..., None], offd - mean[:, None, :], 0.0)
    C = np.einsum("nia,nib->nab", cen, cen)
    v, ok, lmid = smallest_eigvec(C, with_mid=True)
    ok &= m >= 3
    v = np.where(ok[:, None], v, 0.0)
    l0 = np.einsum("na,nab,nb->n", v, C, v)
    planar = ok & (lmid > 0) & (l0 <= PLANAR_RATIO * lmid)
    return feat, v, ok, planar


# ---------------------------------------------------------------- network
def split(params):
    p = np.asarray(params, dtype=np.float64)
    return (p[O_W1:O_B1].reshape(NH, NF), p[O_B1:O_W2], p[O_W2:O_B2].reshape(NH, NH),
            p[O_B2:O_W3], p[O_W3:O_B3].reshape(NOUT, NH), p[O_B3:N_PARAMS])


def forward(params, x, rounded=True):
    """Returns (h1, h2, o, u) for feature rows x [n, 48]."""
    rd = round_bf16 if rounded else (lambda a: np.asarray(a, dtype=np.float64))
    W1, b1, W2, b2, W3, b3 = split(params)
    W1, W2, W3 = rd(W1), rd(W2), rd(W3)
    x = rd(x)
    h1 = rd(np.maximum(x @ W1.T + b1, 0.0))
    h2 = rd(np.maximum(h1 @ W2.T + b2, 0.0))
    o = h2 @ W3.T + b3
    nr = np.linalg.norm(o, axis=1)
    with np.errstate(invalid="ignore", divide="ignore"):
        u = np.where(nr[:, None] > 0, o / nr[:, None], 0.0)
    return h1, h2, o, u


def loss(params, x, y, rounded=True):
    """Mean over the rows of 1 - (u . y)^2 (rows with o = 0 count 0)."""
    _, _, o, u = forward(params, x, rounded)
    d = (u * y).sum(1)
    per = np.where(np.linalg.norm(o, axis=1) > 0, 1.0 - d * d, 0.0)
    return per.sum() / x.shape[0]


def grad(params, x, y, rounded=True):
    """(loss, gradient [N_PARAMS]) by the chain rule through each layer."""
    rd = round_bf16 if rounded else (lambda a: np.asarray(a, dtype=np.float64))
    W1, b1, W2, b2, W3, b3 = split(params)
    W2r, W3r = rd(W2), rd(W3)
    xr = rd(x)
    n = x.shape[0]
    h1, h2, o, u = forward(params, x, rounded)
    nr = np.linalg.norm(o, axis=1)
    live = nr > 0
    d = (u * y).sum(1)
    L = np.where(live, 1.0 - d * d, 0.0).sum() / n
    # u = o/|o|: do = (I - u u^T) dL/du / |o|, dL/du = -2 (u.y) y / n
    gu = -2.0 * d[:, None] * y / n
    with np.errstate(invalid="ignore", divide="ignore"):
        do = (gu - (gu * u).sum(1)[:, None] * u) / nr[:, None]
    do = np.where(live[:, None], do, 0.0)
    gW3 = do.T @ h2
    gb3 = do.sum(0)
    dh2 = (do @ W3r) * (h2 > 0)
    gW2 = dh2.T @ h1
    gb2 = dh2.sum(0)
    dh1 = (dh2 @ W2r) * (h1 > 0)
    gW1 = dh1.T @ xr
    gb1 = dh1.sum(0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return L, g


# ---------------------------------------------------------------- generator, init, Adam
def splitmix64(x: int) -> int:
    """Output of the splitmix64 generator for state x (adds the increment
    0x9e3779b97f4a7c15 first, then the two xor-shift-multiply rounds)."""
    z = (x + 0x9E3779B97F4A7C15) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def init_params(seed: int):
    """Initial parameters (float32): weight i = (2u - 1) sqrt(6 / fan_in)
    (last layer sqrt(3 / 64)) with u = the top 24 bits of
    splitmix64(seed * 0x100000001b3 + i) / 2^24; biases 0."""
    p = np.zeros(N_PARAMS, dtype=np.float32)
    scale = {0: np.sqrt(np.float32(6.0) / np.float32(NF)),
             1: np.sqrt(np.float32(6.0) / np.float32(NH)),
             2: np.sqrt(np.float32(3.0) / np.float32(NH))}
    for i in range(N_PARAMS):
        if i < O_B1:
            s = scale[0]
        elif O_W2 <= i < O_B2:
            s = scale[1]
        elif O_W3 <= i < O_B3:
            s = scale[2]
        else:
            continue
        h = splitmix64((seed * 0x100000001B3 + i) & MASK64)
        u = np.float32(h >> 40) * np.float32(2.0 ** -24) * np.float32(2.0) - np.float32(1.0)
        p[i] = np.float32(u * s)
    return p


def sample_rows(pool, seed: int, t: int, b: int):
    """Training rows of step t: pool[splitmix64(seed ^ (t << 32) ^ i) % len(pool)]."""
    pool = np.asarray(pool)
    return np.array([pool[splitmix64((seed ^ (t << 32) ^ i) & MASK64) % len(pool)]
                     for i in range(b)], dtype=np.int64)


def adam_step(p, m, v, g, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (bias-corrected), binary64; returns new (p, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def train(params, x, y, valid, steps, batch, lr, seed, step0=0, rounded=True):
    """Adam on rows drawn by sample_rows from the valid rows; returns
    (params, per-step losses)."""
    p = np.asarray(params, dtype=np.float64).copy()
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    pool = np.nonzero(np.asarray(valid))[0]
    losses = []
    for i in range(steps):
        t = step0 + i + 1
        rows = sample_rows(pool, seed, t, batch)
        L, g = grad(p, x[rows], y[rows], rounded)
        losses.append(L)
        p, m, v = adam_step(p, m, v, g, t, lr)
    return p, np.array(losses)


def angle(a, b):
    """Unoriented angle between rows of unit vectors (radians), as
    atan2(|a x b|, |a . b|): accurate for small angles, where acos(|a . b|)
    would turn a rounding error e of the vectors into an angle of sqrt(2e)."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    a, b = np.broadcast_arrays(a, b)
    c = np.linalg.norm(np.cross(a, b), axis=-1)
    return np.arctan2(c, np.abs((a * b).sum(-1)))
