"""Seeded synthetic terrestrial-LiDAR scans (input generator only).

This module produces the point clouds that both the CUDA path and the CPU
oracle consume.  It holds none of the decimation arithmetic: it casts rays
from a scanner on a regular azimuth x elevation grid, intersects them with a
few analytic primitives, adds Gaussian range noise and quantises the hits to
int32 millimetres.  A stationary LiDAR head sweeps the elevation angle fast and
the azimuth slowly, so the sample density peaks at the poles of the scan; the
paper motivates its method with exactly this pattern (Introduction, Fig. 1).

Point order is the acquisition order: index = azimuth_step * n_el + elev_step
(after ray dropout the survivors keep their relative order).  Every random
number comes from numpy's PCG64 with an explicit seed, except the range noise
of the site scan: its compiled ray caster (synth_site.c) draws it from
splitmix64 keyed by (seed, station, ray) so that a billion rays can be cast on
all host cores with a result independent of the thread count.

Generators
----------
room_scan     single station in a box room with axis-aligned boxes on the floor
outdoor_scan  single station over a ground plane with boxes and spheres
site_scan     several stations in a closed site (merged multi-station cloud)
batch_sizes   per-scan sizes / ratios for many small room scans
random_cloud  uniform random integer clouds for small tests
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Scan", "room_scan", "outdoor_scan", "site_scan", "batch_specs",
    "random_cloud", "lattice_line", "ROOM_200K", "OUTDOOR_20M",
]

_INF = np.inf


@dataclass
class Scan:
    """A generated scan: int32 mm coordinates [n,3] plus optional attributes."""
    xyz: np.ndarray                     # int32 [n, 3], millimetres
    rgb: np.ndarray | None = None       # uint8 [n, 3]
    normals: np.ndarray | None = None   # float32 [n, 3], analytic surface normals
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.xyz.shape[0])


# ----------------------------------------------------------------------------
# ray / primitive intersection (vectorised, float64, metres)
# ----------------------------------------------------------------------------

def _ray_dirs(n_az: int, n_el: int, az0: int, az1: int) -> np.ndarray:
    """Unit directions for azimuth steps [az0, az1) x all elevation steps."""
    az = 2.0 * math.pi * np.arange(az0, az1, dtype=np.float64) / n_az
    el = -0.5 * math.pi + math.pi * (np.arange(n_el, dtype=np.float64) + 0.5) / n_el
    ca, sa = np.cos(az)[:, None], np.sin(az)[:, None]
    ce, se = np.cos(el)[None, :], np.sin(el)[None, :]
    d = np.empty((az1 - az0, n_el, 3), dtype=np.float64)
    d[..., 0] = ca * ce
    d[..., 1] = sa * ce
    d[..., 2] = np.broadcast_to(se, (az1 - az0, n_el))
    return d.reshape(-1, 3)


def _safe_inv(d: np.ndarray) -> np.ndarray:
    dd = np.where(d == 0.0, 1e-300, d)
    return 1.0 / dd


def _hit_box_inside(o, D, lo, hi):
    """Exit distance of rays leaving the inside of box [lo, hi]; inward normal."""
    inv = _safe_inv(D)
    t_hi = (hi[None, :] - o[None, :]) * inv
    t_lo = (lo[None, :] - o[None, :]) * inv
    t_axis = np.where(D > 0, t_hi, t_lo)
    t_axis = np.where(D == 0, _INF, t_axis)
    ax = np.argmin(t_axis, axis=1)
    t = t_axis[np.arange(len(D)), ax]
    nrm = np.zeros_like(D)
    nrm[np.arange(len(D)), ax] = -np.sign(D[np.arange(len(D)), ax])
    return t, nrm


def _hit_box_outside(o, D, lo, hi):
    """Entry distance of rays hitting box [lo, hi] from outside; outward normal."""
    inv = _safe_inv(D)
    t1 = (lo[None, :] - o[None, :]) * inv
    t2 = (hi[None, :] - o[None, :]) * inv
    tmin = np.minimum(t1, t2)
    tmax = np.maximum(t1, t2)
    ax = np.argmax(tmin, axis=1)
    tnear = tmin[np.arange(len(D)), ax]
    tfar = np.min(tmax, axis=1)
    hit = (tnear <= tfar) & (tnear > 1e-9)
    t = np.where(hit, tnear, _INF)
    nrm = np.zeros_like(D)
    nrm[np.arange(len(D)), ax] = -np.sign(D[np.arange(len(D)), ax])
    return t, nrm


def _hit_sphere(o, D, c, r):
    oc = o - c
    b = D @ oc
    cc = float(oc @ oc) - r * r
    disc = b * b - cc
    sq = np.sqrt(np.maximum(disc, 0.0))
    t = -b - sq
    hit = (disc >= 0) & (t > 1e-9)
    t = np.where(hit, t, _INF)
    p = o[None, :] + np.where(hit, t, 0.0)[:, None] * D
    nrm = (p - c[None, :]) / r
    return t, nrm


def _hit_plane_z(o, D, z0):
    """Rays hitting the horizontal plane z = z0 from above; normal +z."""
    with np.errstate(divide="ignore", invalid="ignore"):
        t = (z0 - o[2]) / D[:, 2]
    t = np.where((D[:, 2] < 0) & (t > 1e-9), t, _INF)
    nrm = np.zeros_like(D)
    nrm[:, 2] = 1.0
    return t, nrm


def _hit_cylinder_z(o, D, cx, cy, r, z0, z1):
    """Vertical cylinder side (x-cx)^2+(y-cy)^2=r^2, z in [z0,z1], from outside."""
    ox, oy = o[0] - cx, o[1] - cy
    a = D[:, 0] ** 2 + D[:, 1] ** 2
    b = ox * D[:, 0] + oy * D[:, 1]
    c = ox * ox + oy * oy - r * r
    disc = b * b - a * c
    sq = np.sqrt(np.maximum(disc, 0.0))
    with np.errstate(divide="ignore", invalid="ignore"):
        t = (-b - sq) / a
    z = o[2] + t * D[:, 2]
    hit = (disc >= 0) & (a > 0) & (t > 1e-9) & (z >= z0) & (z <= z1)
    t = np.where(hit, t, _INF)
    px = ox + np.where(hit, t, 0.0) * D[:, 0]
    py = oy + np.where(hit, t, 0.0) * D[:, 1]
    nrm = np.stack([px / r, py / r, np.zeros_like(px)], axis=1)
    return t, nrm



def _culled_rows(prim, o, n_az, n_el, az0, az1):
    """Ray rows of this azimuth chunk that can hit a bounded primitive.

    A primitive with a bounding circle (centre ``bc``, radius ``br`` in the xy
    plane) that excludes the scanner subtends the azimuth interval
    theta_c +- asin(br / dist); rays outside it cannot hit it.  Returns None
    for unbounded primitives (test every ray).
    """
    if "bc" not in prim:
        return None
    cx, cy = prim["bc"][0] - o[0], prim["bc"][1] - o[1]
    dist = math.hypot(cx, cy)
    br = prim["br"]
    if dist <= br * 1.0001:
        return None
    hw = math.asin(br / dist) + 2.0 * math.pi / n_az
    th = math.atan2(cy, cx)
    step = 2.0 * math.pi / n_az
    i = np.arange(az0, az1)
    dth = np.angle(np.exp(1j * (i * step - th)))
    cols = np.nonzero(np.abs(dth) <= hw)[0]
    if len(cols) == 0:
        return np.zeros(0, dtype=np.int64)
    return (cols[:, None] * n_el + np.arange(n_el)[None, :]).reshape(-1)

def _quantise_mm(p: np.ndarray) -> np.ndarray:
    """floor(1000 * x + 0.5): metres -> int32 millimetres."""
    return np.floor(p * 1000.0 + 0.5).astype(np.int32)


def _checker_rgb(base: np.ndarray, p: np.ndarray) -> np.ndarray:
    """Object colour times a 0.5 m checker (factor 1.0 or 0.6)."""
    cell = np.floor(p / 0.5).astype(np.int64).sum(axis=1) & 1
    f = np.where(cell == 0, 1.0, 0.6)[:, None]
    return np.clip(base * f, 0, 255).astype(np.uint8)


def _trace(scanner, prims, n_az, n_el, rng, noise_m, dropout, max_range,
           want_rgb, want_normals, chunk_rays=1 << 21):
    """Cast the full ray grid; return int32 xyz (+ rgb, normals) of the hits."""
    o = np.asarray(scanner, dtype=np.float64)
    per_chunk = max(1, chunk_rays // n_el)
    xs, cs, ns = [], [], []
    for az0 in range(0, n_az, per_chunk):
        az1 = min(n_az, az0 + per_chunk)
        D = _ray_dirs(n_az, n_el, az0, az1)
        m = len(D)
        best_t = np.full(m, _INF)
        best_n = np.zeros((m, 3))
        best_id = np.full(m, -1, dtype=np.int64)
        for pid, prim in enumerate(prims):
            rows = _culled_rows(prim, o, n_az, n_el, az0, az1)
            if rows is None:
                t, nrm = prim["fn"](o, D)
                better = t < best_t
                best_t = np.where(better, t, best_t)
                best_n = np.where(better[:, None], nrm, best_n)
                best_id = np.where(better, pid, best_id)
            elif len(rows):
                t, nrm = prim["fn"](o, D[rows])
                better = t < best_t[rows]
                sel = rows[better]
                best_t[sel] = t[better]
                best_n[sel] = nrm[better]
                best_id[sel] = pid
        # draws are taken for every ray so the stream does not depend on hits
        noise = rng.normal(0.0, noise_m, size=m)
        keep_u = rng.random(size=m)
        ok = np.isfinite(best_t) & (best_t <= max_range) & (keep_u >= dropout)
        r = best_t[ok] + noise[ok]
        p = o[None, :] + r[:, None] * D[ok]
        xs.append(_quantise_mm(p))
        if want_rgb:
            base = np.stack([prims[i]["rgb"] for i in range(len(prims))])[best_id[ok]]
            cs.append(_checker_rgb(base.astype(np.float64), p))
        if want_normals:
            ns.append(best_n[ok].astype(np.float32))
    xyz = np.ascontiguousarray(np.concatenate(xs, axis=0))
    rgb = np.ascontiguousarray(np.concatenate(cs, axis=0)) if want_rgb else None
    nrm = np.ascontiguousarray(np.concatenate(ns, axis=0)) if want_normals else None
    return xyz, rgb, nrm


def _colour(rng) -> np.ndarray:
    return rng.integers(40, 256, size=3).astype(np.float64)


# ----------------------------------------------------------------------------
# scenes
# ----------------------------------------------------------------------------

def room_scan(seed: int = 0, n_az: int = 1000, n_el: int = 200,
              dims=(10.0, 8.0, 3.0), scanner=(4.0, 3.0, 1.5), n_boxes: int = 3,
              noise_mm: float = 2.0, rgb: bool = False, normals: bool = False) -> Scan:
    """Single-station scan of a closed box room [0,W]x[0,D]x[0,H] (metres).

    Six walls plus ``n_boxes`` axis-aligned boxes standing on the floor, sides
    drawn uniformly in [0.4, 1.5] m and placed fully inside the room without
    containing the scanner.  The room is closed, so every ray returns and the
    cloud has exactly n_az * n_el points.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    W, Dp, H = (float(v) for v in dims)
    s = np.asarray(scanner, dtype=np.float64)
    prims = [{"fn": (lambda o, D, lo=np.zeros(3), hi=np.array([W, Dp, H]):
                     _hit_box_inside(o, D, lo, hi)), "rgb": _colour(rng)}]
    boxes = []
    while len(boxes) < n_boxes:
        side = rng.uniform(0.4, 1.5, size=3)
        side[2] = min(side[2], H - 0.2)
        x0 = rng.uniform(0.05, W - side[0] - 0.05)
        y0 = rng.uniform(0.05, Dp - side[1] - 0.05)
        lo = np.array([x0, y0, 0.0])
        hi = lo + side
        if np.all(s >= lo - 0.3) and np.all(s <= hi + 0.3):
            continue  # would contain (or nearly touch) the scanner
        boxes.append((lo, hi))
        prims.append({"fn": (lambda o, D, lo=lo, hi=hi: _hit_box_outside(o, D, lo, hi)),
                      "rgb": _colour(rng), "bc": (lo + hi)[:2] / 2,
                      "br": float(np.linalg.norm(hi[:2] - lo[:2]) / 2)})
    noise_rng = np.random.Generator(np.random.PCG64([seed, 1]))
    xyz, c, nr = _trace(s, prims, n_az, n_el, noise_rng, noise_mm * 1e-3, 0.0,
                        _INF, rgb, normals)
    return Scan(xyz, c, nr, {"scene": "room", "seed": seed, "n_az": n_az, "n_el": n_el,
                             "dims": (W, Dp, H), "scanner": tuple(s), "boxes": boxes})


def outdoor_scan(seed: int = 0, n_az: int = 10000, n_el: int = 2000,
                 dropout: float = 0.15, n_boxes: int = 40, n_spheres: int = 20,
                 scanner_height: float = 1.5, max_range: float = 120.0,
                 noise_mm: float = 2.0, rgb: bool = False, normals: bool = False) -> Scan:
    """Single-station outdoor scan: ground plane, boxes and spheres at 1-60 m.

    The scanner sits ``scanner_height`` above an unbounded ground plane z=0.
    Boxes (footprint 0.5-8 m, height 0.5-12 m) and spheres (radius 0.3-4 m,
    resting on the ground) are centred at horizontal range U[1, 60] m.  Rays
    that hit nothing within ``max_range`` (sky, far ground) give no point, and
    a Bernoulli ``dropout`` removes returns (dark or specular surfaces).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    s = np.array([0.0, 0.0, scanner_height])
    prims = [{"fn": (lambda o, D: _hit_plane_z(o, D, 0.0)), "rgb": _colour(rng)}]
    nb = 0
    while nb < n_boxes:
        rr = rng.uniform(1.0, 60.0)
        th = rng.uniform(0.0, 2 * math.pi)
        w = rng.uniform(0.5, 8.0, size=2)
        h = rng.uniform(0.5, 12.0)
        c = np.array([rr * math.cos(th), rr * math.sin(th)])
        lo = np.array([c[0] - w[0] / 2, c[1] - w[1] / 2, 0.0])
        hi = np.array([c[0] + w[0] / 2, c[1] + w[1] / 2, h])
        if np.all(s[:2] >= lo[:2] - 0.5) and np.all(s[:2] <= hi[:2] + 0.5):
            continue
        prims.append({"fn": (lambda o, D, lo=lo, hi=hi: _hit_box_outside(o, D, lo, hi)),
                      "rgb": _colour(rng), "bc": c, "br": float(np.hypot(w[0], w[1]) / 2)})
        nb += 1
    ns_ = 0
    while ns_ < n_spheres:
        rr = rng.uniform(1.0, 60.0)
        th = rng.uniform(0.0, 2 * math.pi)
        rad = rng.uniform(0.3, 4.0)
        c = np.array([rr * math.cos(th), rr * math.sin(th), rad])
        if np.linalg.norm(c - s) < rad + 0.5:
            continue
        prims.append({"fn": (lambda o, D, c=c, rad=rad: _hit_sphere(o, D, c, rad)),
                      "rgb": _colour(rng), "bc": c[:2], "br": rad})
        ns_ += 1
    noise_rng = np.random.Generator(np.random.PCG64([seed, 1]))
    xyz, c, nr = _trace(s, prims, n_az, n_el, noise_rng, noise_mm * 1e-3, dropout,
                        max_range, rgb, normals)
    return Scan(xyz, c, nr, {"scene": "outdoor", "seed": seed, "n_az": n_az,
                             "n_el": n_el, "dropout": dropout, "max_range": max_range})


def _site_scene(seed, stations, size):
    """Primitives and station positions of the site (numpy PCG64, seeded)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    W, Dp, H = (float(v) for v in size)
    site_rgb = _colour(rng)
    prims = []
    for _ in range(30):  # boxes (buildings, containers)
        w = rng.uniform(2.0, 25.0, size=2)
        h = rng.uniform(2.0, 20.0)
        x0 = rng.uniform(2.0, W - w[0] - 2.0)
        y0 = rng.uniform(2.0, Dp - w[1] - 2.0)
        lo, hi = np.array([x0, y0, 0.0]), np.array([x0 + w[0], y0 + w[1], h])
        prims.append({"box": (lo, hi), "rgb": _colour(rng), "bc": (lo + hi)[:2] / 2,
                      "br": float(np.linalg.norm(hi[:2] - lo[:2]) / 2)})
    for _ in range(30):  # cylinders (columns, tanks, poles)
        r = rng.uniform(0.15, 3.0)
        cx, cy = rng.uniform(5.0, W - 5.0), rng.uniform(5.0, Dp - 5.0)
        h = rng.uniform(2.0, 25.0)
        prims.append({"cyl": (cx, cy, r, h), "rgb": _colour(rng), "bc": np.array([cx, cy]),
                      "br": r})
    pos = []
    while len(pos) < stations:
        p = np.array([rng.uniform(3.0, W - 3.0), rng.uniform(3.0, Dp - 3.0), 1.5])
        inside = False
        for pr in prims:
            if "box" in pr:
                lo, hi = pr["box"]
                if np.all(p >= lo - 0.5) and np.all(p <= hi + 0.5):
                    inside = True
            else:
                cx, cy, r, _ = pr["cyl"]
                if math.hypot(p[0] - cx, p[1] - cy) < r + 0.5:
                    inside = True
        if not inside:
            pos.append(p)
    return prims, pos, site_rgb


_SYNTH_LIB = None


def _synth_lib():
    """The compiled site ray caster (synth_site.c, built with gcc on first use)."""
    global _SYNTH_LIB
    if _SYNTH_LIB is None:
        import ctypes
        import os
        import subprocess
        here = os.path.dirname(os.path.abspath(__file__))
        src = os.path.join(here, "synth_site.c")
        lib = os.path.join(here, "libsynth.so")
        if not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(src):
            tmp = lib + ".%d.tmp" % os.getpid()
            subprocess.run(["gcc", "-O2", "-std=gnu11", "-fopenmp", "-ffp-contract=off",
                            "-fno-fast-math", "-fPIC", "-shared", src, "-o", tmp, "-lm"],
                           check=True)
            os.replace(tmp, lib)
        L = ctypes.CDLL(lib)
        P = ctypes.c_void_p
        L.synth_site.argtypes = [P, ctypes.c_int, P, P, P, ctypes.c_int, ctypes.c_int,
                                 ctypes.c_int, ctypes.c_double, ctypes.c_uint64, P, P, P]
        L.synth_site.restype = ctypes.c_int
        L.synth_threads.restype = ctypes.c_int
        _SYNTH_LIB = L
    return _SYNTH_LIB


def site_scan(seed: int = 0, stations: int = 40, n_az: int = 10000, n_el: int = 2500,
              size=(200.0, 200.0, 30.0), noise_mm: float = 2.0, rgb: bool = True,
              station_ids=None) -> Scan:
    """Merged multi-station scan of a closed site (ground, walls, roof, objects).

    The site is the inside of a W x D x H box with 30 axis-aligned boxes (2-25 m
    footprint, 2-20 m high) and 30 vertical cylinders (radius 0.15-3 m, 2-25 m
    high).  Every station stands 1.5 m above the ground at a random position
    outside every object; the site is closed, so every ray returns and each
    station gives exactly n_az * n_el points.  Stations are concatenated in
    order, so points of different stations on the same surface interleave as
    near-duplicates.  ``station_ids`` selects a subset of the stations (for
    bounded samples).  The rays are cast by the compiled ray caster
    (synth_site.c, all host cores); its range noise is seeded per (seed,
    station, ray), so the output does not depend on the thread count.
    """
    import ctypes
    prims, pos, site_rgb = _site_scene(seed, stations, size)
    ids = list(range(stations)) if station_ids is None else [int(i) for i in station_ids]
    rec = np.zeros((len(prims), 17), dtype=np.float64)
    for q, pr in enumerate(prims):
        if "box" in pr:
            lo, hi = pr["box"]
            rec[q, 0] = 0
            rec[q, 1:4], rec[q, 4:7] = lo, hi
        else:
            cx, cy, r, h = pr["cyl"]
            rec[q, 0] = 1
            rec[q, 7:11] = (cx, cy, r, h)
        rec[q, 11:13] = pr["bc"]
        rec[q, 13] = pr["br"]
        rec[q, 14:17] = pr["rgb"]
    st = np.ascontiguousarray(np.stack([pos[i] for i in ids]), dtype=np.float64)
    sid = np.asarray(ids, dtype=np.int64)
    sz = np.asarray(size, dtype=np.float64)
    srgb = np.asarray(site_rgb, dtype=np.float64)
    n = len(ids) * n_az * n_el
    xyz = np.empty((n, 3), dtype=np.int32)
    col = np.empty((n, 3), dtype=np.uint8) if rgb else None
    P = ctypes.c_void_p
    rc = _synth_lib().synth_site(rec.ctypes.data_as(P), len(prims), sz.ctypes.data_as(P),
                                 st.ctypes.data_as(P), sid.ctypes.data_as(P), len(ids), n_az,
                                 n_el, noise_mm * 1e-3, int(seed),
                                 srgb.ctypes.data_as(P), xyz.ctypes.data_as(P),
                                 None if col is None else col.ctypes.data_as(P))
    if rc != 0:
        raise RuntimeError("synth_site failed (%d)" % rc)
    return Scan(xyz, col, None, {"scene": "site", "seed": seed, "stations": ids,
                                 "n_az": n_az, "n_el": n_el})


def batch_specs(seed: int = 0, count: int = 512, n_lo: float = 5e4, n_hi: float = 5e6,
                r_lo: float = 0.05, r_hi: float = 0.5):
    """Per-scan (n_el, n_az, ratio, room dims, scanner) for a batch of room scans.

    Sizes are log-uniform in [n_lo, n_hi] with an azimuth:elevation grid of 5:1
    (n = 5 * n_el^2), room dimensions are the 10x8x3 m room scaled by U[0.7,1.3]
    per axis and the scanner stands at a random position inside it.
    """
    rng = np.random.Generator(np.random.PCG64([seed, 7]))
    specs = []
    for i in range(count):
        n = math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))
        n_el = max(4, int(round(math.sqrt(n / 5.0))))
        dims = (10.0 * rng.uniform(0.7, 1.3), 8.0 * rng.uniform(0.7, 1.3),
                3.0 * rng.uniform(0.7, 1.3))
        sc = (rng.uniform(1.0, dims[0] - 1.0), rng.uniform(1.0, dims[1] - 1.0),
              rng.uniform(1.0, min(2.0, dims[2] - 0.5)))
        ratio = rng.uniform(r_lo, r_hi)
        specs.append({"i": i, "seed": seed * 100003 + i, "n_el": n_el, "n_az": 5 * n_el,
                      "ratio": ratio, "dims": dims, "scanner": sc})
    return specs


def random_cloud(seed: int, n: int, span: int = 1000, dims: int = 3) -> np.ndarray:
    """Uniform random int32 points in [0, span)^dims (other axes zero)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    xyz = np.zeros((n, 3), dtype=np.int32)
    xyz[:, :dims] = rng.integers(0, span, size=(n, dims), dtype=np.int64).astype(np.int32)
    return xyz


def lattice_line(n: int, step: int = 1) -> np.ndarray:
    """Points at x = step * i (i < n) on a line."""
    xyz = np.zeros((n, 3), dtype=np.int32)
    xyz[:, 0] = step * np.arange(n, dtype=np.int32)
    return xyz


# Named workloads.
ROOM_200K = dict(seed=0, n_az=1000, n_el=200)            # k=1, keep 25 %
OUTDOOR_20M = dict(seed=0, n_az=10000, n_el=2000)        # k=4, keep 10 %
