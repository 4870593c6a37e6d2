#!/usr/bin/env python
"""Benchmark: greedy kNN-cost decimation throughput on one GB300.

A step decimates one synthetic terrestrial-LiDAR scan end to end on the
device: voxel-grid build (Morton radix sort, octree cell table), the first
k-nearest-neighbour/cost pass, the removal rounds and the keep mask.  The
default workload is the merged 40-station site scan (1.0B points, int32 mm +
RGB, all resident in HBM) with the k = 1 density cost, keeping 5 %.

  value   input points / second of device time, inputs resident in HBM
  e2e     the same through pd_decimate_host (host buffers, copies timed)
  roofline  the first full kNN/cost pass (the dominant kernel): algorithmic
            bytes / launch time against the measured copy bandwidth, with the
            integer-issue roofline that binds it, the whole search, the phases
            and the whole step beside it
  cpu_baseline  the CPU oracle on a bounded sector of the same scan
  batched   512 room scans of uneven size (sizes log-uniform 50k-5M, RGB,
            colour term 0.3, keep 5-50 %) decimated as one packed grid
            through pd_decimate_batch; the first 48 also through concurrent
            slots and one at a time
  serving   Poisson arrivals (50 scans/s) of distinct room scans of 100k-10M
            points through the pd_serve_* loop with the orientation term and
            network normals; p50/p99 latency, throughput, normal angular error

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
       python bench.py --impl reference ...   (the CPU oracle as the reference arm)
Multi-GPU (torchrun): every rank decimates its own scan (seed + rank), no
collective on the data path ("weak" scaling); timing is max over ranks.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2311_17604_gb300 import synth  # noqa: E402

METRIC = "decimated points/sec/GB300 (oracle-exact), % of HBM roofline; batched p99 ms"
UNIT = "points/s"

WORKLOADS = {
    "site": dict(desc="merged multi-station site scan, 40 stations x 10000x2500 rays (1.0B points) "
                      "of a closed 200x200x30 m site (ground, walls, roof, 30 boxes, 30 "
                      "cylinders), int32 mm + uint8 RGB, all resident in HBM; k=1 density "
                      "cost; keep 5%",
                 gen=lambda seed: synth.site_scan(seed=seed, stations=40, rgb=True),
                 sample_gen=lambda seed: synth.site_scan(seed=seed, stations=40,
                                                         station_ids=[0], rgb=False),
                 k=1, ratio=0.05, sample=400_000, ref_sample=150_000, tune_sample=100_000_000),
    "site4": dict(desc="merged site scan, 4 stations x 10000x2500 rays (100M points) of the "
                       "200x200x30 m site generator, int32 mm; k=1; keep 5%",
                  gen=lambda seed: synth.site_scan(seed=seed, station_ids=[0, 1, 2, 3], rgb=False),
                  k=1, ratio=0.05, sample=400_000, ref_sample=150_000),
    "site1": dict(desc="one station of the site generator, 10000x2500 rays (25M points), int32 "
                       "mm; k=1; keep 5% (profiling case)",
                  gen=lambda seed: synth.site_scan(seed=seed, station_ids=[0], rgb=False),
                  k=1, ratio=0.05, sample=400_000, ref_sample=150_000),
    "outdoor": dict(desc="outdoor single-station scan, 10000x2000 rays, 15% dropout, "
                         "ground + 40 boxes + 20 spheres at 1-60 m, int32 mm; k=4; keep 10%",
                    gen=lambda seed: synth.outdoor_scan(seed=seed, n_az=10000, n_el=2000),
                    k=4, ratio=0.1, sample=400_000, ref_sample=150_000),
    "room": dict(desc="room single-station scan, 1000x200 rays, 10x8x3 m, 3 boxes, "
                      "2 mm noise, int32 mm; k=1; keep 25%",
                 gen=lambda seed: synth.room_scan(seed=seed, n_az=1000, n_el=200),
                 k=1, ratio=0.25, sample=200_000, ref_sample=200_000),
}


# ------------------------------------------------------------------ helpers
def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def aggregate(local_seconds: float, local_units: int, dist=None):
    """Whole-job numbers: units summed over ranks, time = max over ranks."""
    if dist is None:
        return local_seconds, local_units
    import torch
    dev = "cuda" if torch.cuda.is_available() and dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([local_seconds], dtype=torch.float64, device=dev)
    u = torch.tensor([float(local_units)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), int(u.item())


def oracle_sample(scan_xyz, n_sample, k, ratio):
    """The oracle as it stands on the first n_sample points (an azimuth sector)."""
    import oracle
    x = np.ascontiguousarray(scan_xyz[:n_sample])
    m = oracle.target_count(len(x), ratio)
    t0 = time.perf_counter()
    oracle.decimate(x, k, m)
    dt = time.perf_counter() - t0
    return len(x), dt, oracle.threads()


# ------------------------------------------------------------------ arms
def run_reference(args, wl, rank):
    """CPU oracle on bounded samples of the workload (rank 0 only)."""
    if rank != 0:
        return
    scan = wl.get("sample_gen", wl["gen"])(0)
    ns = min(wl["ref_sample"], scan.n)
    for _ in range(args.warmup):
        pass  # the oracle has no warm-up state; warm-up steps are not repeated
    times = []
    threads = 1
    for _ in range(args.steps):
        n, dt, threads = oracle_sample(scan.xyz, ns, wl["k"], wl["ratio"])
        times.append(dt)
    tot = sum(times)
    value = ns * len(times) / tot
    sample = "first %d points (azimuth sector of the first station) of the workload's scan, " \
             "k=%d, keep %g" % (ns, wl["k"], wl["ratio"])
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "i64+f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": wl["desc"], "sample_points": ns},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)




# ------------------------------------------------------------------ rooflines
# Algorithmic (compulsory) HBM bytes of the hot path per unit of work, as the
# measurement plan counts them:
#   kNN/cost (A4), per query: 12 B read (x, y, z), 12 B key + index, 8 B r_k^2
#                  and 4 k B neighbour indices written: 36 B (k = 1), 48 B (k = 4)
#   removal rounds (A5-A6): 16 B per live point per round
#   grid build (A1-A3), per point: 24 B cell key, 24 B per radix pass, 28 B gather
def knn_bytes(k):
    return 12 + 12 + 8 + 4 * k


ROUND_BYTES_PER_LIVE = 16
ALU_OPS_PER_PAIR = 9   # 3 subtractions, 3 multiply-adds, compare, select, loop: exact int distance test

# DRAM bytes per query of the first full kNN pass (knn_kernel<8,0,0,0>), from an
# ncu capture (dram__bytes_read.sum + dram__bytes_write.sum) of a one-station
# site scan at the leaf capacity below; reported only while the kNN sources
# hash to src_sha and the timed run uses the same leaf capacity and k.
KNN_TRAFFIC = {"k": 1, "leaf_max": 32, "bytes_per_query": 113.9, "src_sha": "d96e267f93cc3f0e"}
KNN_SOURCES = ["paper_2311_17604_gb300/csrc/knn.cu", "paper_2311_17604_gb300/csrc/pd_internal.cuh",
               "paper_2311_17604_gb300/csrc/pd_kernels.h"]


def knn_src_sha():
    import hashlib
    h = hashlib.sha256()
    for f in KNN_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def radix_passes(xyz):
    """Radix passes of the grid build: 8-bit digits over 3 B Morton bits."""
    span = int((xyz.max(axis=0).astype(np.int64) - xyz.min(axis=0)).max())
    B = max(1, min(span.bit_length(), 21))
    return (3 * B + 7) // 8


def rooflines(stats, n, k, leaf, passes, step_ms, clk, device):
    """HBM rooflines from the library's CUDA-event phase timers (on the
    launching stream) and the algorithmic bytes above.  The top level is the
    dominant kernel of a step, the first full kNN/cost pass (one launch per
    step); the whole kNN search (that pass plus the re-searches of the removal
    rounds), its integer-issue view, the other phases and the whole step are
    reported beside it."""
    import torch
    mean = lambda key: statistics.mean(s[key] for s in stats)
    peak, kind = measured_peaks()
    bq = knn_bytes(k)
    q1, ms1 = mean("q_first"), mean("ms_knn_first")
    rq, msr = mean("requeries"), mean("ms_knn_requery")
    pairs = mean("pairs_first")
    ms_knn = ms1 + msr
    gbs = lambda b, ms: b / (ms / 1e3) / 1e9 if ms > 0 else None
    knn_ach = gbs((q1 + rq) * bq, ms_knn)
    first_ach = gbs(q1 * bq, ms1)
    sha = knn_src_sha()
    tr = KNN_TRAFFIC
    # DRAM bytes of the first pass (one launch), from the capture scaled by the
    # queries; reported only for the captured build, leaf capacity and k
    traffic1 = (tr["bytes_per_query"] * q1
                if tr["bytes_per_query"] and tr["src_sha"] == sha and tr["leaf_max"] == leaf
                and tr["k"] == k else None)
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    mhz = clk.get("sm_mhz") or clk.get("sm_max_mhz") or 2070.0
    peak_ops = sms * 4 * 32 * mhz * 1e6
    alu = pairs * ALU_OPS_PER_PAIR / (ms1 / 1e3)
    build_b = n * (24 + 24 * passes + 28)
    round_b = mean("live_rounds") * ROUND_BYTES_PER_LIVE
    step_b = build_b + (q1 + rq) * bq + round_b
    step_ach = gbs(step_b, statistics.mean(step_ms))
    phases = {"grid": mean("ms_grid"), "rebuilds": mean("ms_build"), "knn_first": ms1,
              "knn_requery": msr, "select": mean("ms_select"),
              "rules_other": mean("ms_rules") - mean("ms_select"),
              "total": mean("ms_total")}
    return {"bound": "hbm", "kernel": "knn_kernel<8,0,0,0>: the first full kNN/cost pass (one "
                                      "launch per step)",
            "achieved": first_ach, "peak": peak, "unit": "GB/s", "frac": first_ach / peak,
            "hbm_frac": first_ach / peak, "peak_kind": kind, "traffic": traffic1,
            "traffic_basis": "%s B per query (ncu dram__bytes_read.sum + dram__bytes_write.sum "
                             "of this kernel, one-station site scan, leaf %d, k %d) x the "
                             "launch's queries" % (tr["bytes_per_query"], tr["leaf_max"],
                                                   tr["k"]),
            "units": q1, "unit_name": "queries", "bytes_per_unit": bq, "ms": ms1,
            "pairs_per_query": pairs / max(q1, 1),
            "binding": "alu",
            "alu": {"achieved": alu / 1e9, "peak": peak_ops / 1e9, "unit": "Gop/s",
                    "frac": alu / peak_ops, "ops_per_pair": ALU_OPS_PER_PAIR,
                    "peak_basis": "%d SMs x 4 x 32 lanes x %.0f MHz (median SM clock "
                                  "sampled)" % (sms, mhz)},
            "knn_search": {"what": "first pass + re-searches of the removal rounds",
                           "queries": q1 + rq, "ms": ms_knn, "achieved": knn_ach,
                           "frac": knn_ach / peak},
            "requeries": {"queries": rq, "ms": msr, "achieved": gbs(rq * bq, msr),
                          "frac": (gbs(rq * bq, msr) or 0) / peak},
            "step": {"bytes": step_b, "achieved": step_ach, "frac": step_ach / peak,
                     "bytes_basis": "build %d B/pt (%d radix passes) + %d B per query + %d B "
                                    "per live point per round" % (24 + 24 * passes + 28, passes,
                                                                  bq, ROUND_BYTES_PER_LIVE)},
            "phases_ms": phases, "src_sha": sha}

# ------------------------------------------------------------------ batched and served legs
def _pct(v, q):
    return float(np.percentile(np.asarray(v, dtype=np.float64), q)) if len(v) else None


def _batch_scan(sp):
    s = synth.room_scan(seed=sp["seed"], n_az=sp["n_az"], n_el=sp["n_el"], dims=sp["dims"],
                        scanner=sp["scanner"], rgb=True)
    return s.xyz, s.rgb


def run_batched(args, pd, torch, dev, stream):
    """The batched workload: --batch-count room scans (sizes log-uniform in
    50k-5M, room size and scanner from the seed, RGB, colour term 0.3, k = 1,
    keep 5-50 %) decimated as one packed grid (PD_BATCH_PACKED).  The first
    --batch-compare scans also run through concurrent slots and one at a time
    through the single-scan path, for the comparison."""
    import multiprocessing as mp

    import oracle
    specs = synth.batch_specs(seed=0, count=args.batch_count, n_lo=5e4, n_hi=5e6)
    clouds, total = [], 0
    # the scans are cast on the host cores (a spawned pool: this process
    # already holds a CUDA context)
    with mp.get_context("spawn").Pool(max(1, min(16, os.cpu_count() or 1))) as pool:
        for sp, (xyz, rgb) in zip(specs, pool.imap(_batch_scan, specs, chunksize=1)):
            clouds.append({"xyz": torch.from_numpy(xyz).to(dev),
                           "rgb": torch.from_numpy(rgb).to(dev), "ratio": sp["ratio"]})
            total += xyz.shape[0]
    ctx = pd.Context()
    kw = dict(k=1, term=pd.PD_TERM_COLOR, weight=0.3)
    big = max(clouds, key=lambda c: int(c["xyz"].shape[0]))
    leaf = args.leaf_max or pd.pd_autotune(ctx, big["xyz"], big["ratio"], rgb=big["rgb"],
                                           sample=1_000_000, stream=stream, **kw)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        torch.cuda.synchronize()
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return out, e0.elapsed_time(e1)

    pd.pd_decimate_batch(ctx, clouds[:8], stream=stream, **kw)   # warm (packed)
    l0 = pd.lib().pd__launch_count()
    (keeps, stats), packed_ms = timed(lambda: pd.pd_decimate_batch(
        ctx, clouds, concurrency=pd.PD_BATCH_PACKED, stream=stream, **kw))
    launches = pd.lib().pd__launch_count() - l0
    for c, kp in zip(clouds, keeps):
        assert int(kp.sum().item()) == oracle.target_count(int(c["xyz"].shape[0]), c["ratio"])
    del keeps
    compare = _batch_compare(args, pd, ctx, clouds[:args.batch_compare], kw, timed, stream)
    ctx.close()
    return {"workload": "%d room scans, sizes log-uniform 50k-5M (%d points), RGB, k=1 + 0.3 x "
                        "colour term, keep U[5%%, 50%%]" % (len(clouds), total),
            "mode": "packed: every scan in one grid, one launch per round kernel for all scans",
            "scans": len(clouds), "points": total, "leaf_max": leaf,
            "value": total / (packed_ms / 1e3), "unit": UNIT, "ms": packed_ms,
            "rounds": stats[0]["rounds"], "gpu_launches": int(launches),
            "phases_ms": {key: stats[0][key] for key in ("ms_grid", "ms_knn_first",
                                                        "ms_knn_requery", "ms_select",
                                                        "ms_danger", "ms_build", "ms_rules")},
            "graph_rounds": stats[0]["graph_rounds"],
            "per_scan_ms": {"p50": packed_ms, "p99": packed_ms,
                            "what": "every scan of a packed batch finishes with the batch"},
            "compare": compare}


def _batch_compare(args, pd, ctx, sub, kw, timed, stream):
    """The first scans of the batch packed, through slots and one at a time."""
    if not sub:
        return None
    sub_pts = sum(int(c["xyz"].shape[0]) for c in sub)
    pd.pd_decimate_batch(ctx, sub[:4], concurrency=4, stream=stream, **kw)   # warm (slots)
    (_, sstats), slots_ms = timed(lambda: pd.pd_decimate_batch(
        ctx, sub, concurrency=args.batch_slots, stream=stream, **kw))
    (_, pstats), psub_ms = timed(lambda: pd.pd_decimate_batch(
        ctx, sub, concurrency=pd.PD_BATCH_PACKED, stream=stream, **kw))

    def single():
        for c in sub:
            g = pd.Grid(ctx, c["xyz"], rgb=c["rgb"], stream=stream)
            pd.pd_decimate_ratio(g, c["ratio"], stream=stream, **kw)
            g.free()
    _, single_ms = timed(single)
    per_scan = [st["ms_total"] for st in sstats]
    return {"scans": len(sub), "points": sub_pts,
            "packed": {"value": sub_pts / (psub_ms / 1e3), "ms": psub_ms},
            "slots": {"value": sub_pts / (slots_ms / 1e3), "ms": slots_ms,
                      "slots": args.batch_slots,
                      "per_scan_ms": {"p50": _pct(per_scan, 50), "p99": _pct(per_scan, 99),
                                      "what": "each scan's decimation time on its slot's "
                                              "stream"}},
            "single_scan_loop": {"value": sub_pts / (single_ms / 1e3), "ms": single_ms},
            "packed_vs_single": single_ms / psub_ms}


def _serve_scan(spec):
    seed, n_el = spec
    return synth.room_scan(seed=seed, n_az=5 * n_el, n_el=n_el).xyz


def run_serving(args, pd, torch, dev):
    """Poisson arrivals of room scans (n log-uniform in 100k-10M) at --serve-rate
    scans/s through pd_serve_*, orientation term 0.5 with network normals."""
    import multiprocessing as mp

    from oracle import normals as onorm  # angle helper only (reporting)
    rng = np.random.default_rng(0)
    # one distinct scan per request (--serve-pool 0), or a pool reused
    # round-robin; cast on the host cores (a spawned pool: this process
    # already holds a CUDA context)
    npool = args.serve_pool if args.serve_pool > 0 else args.serve_requests
    sizes = np.exp(rng.uniform(np.log(1e5), np.log(1e7), npool))
    specs = [(100 + i, max(10, int(round(np.sqrt(sz / 5.0))))) for i, sz in enumerate(sizes)]
    pool = []
    with mp.get_context("spawn").Pool(max(1, min(16, os.cpu_count() or 1))) as wp:
        for xyz in wp.imap(_serve_scan, specs, chunksize=1):
            pool.append((pd.pinned_like(xyz), xyz.shape[0]))
    ctx = pd.Context(use_torch_allocator=False)
    # the network: trained on the PCA normals of the planar rows of one scan
    tr_scan = synth.room_scan(seed=99, n_az=1000, n_el=200)
    g = pd.Grid(ctx, torch.from_numpy(tr_scan.xyz).to(dev))
    feat, pca, valid = pd.pd_normals_pca(g)
    g.free()
    pd.MlpTrainer(seed=0).train(ctx, feat, pca, valid, steps=2, batch=256, lr=2e-3, seed=0)
    torch.cuda.synchronize()   # first-call set-up outside the timed training
    trainer = pd.MlpTrainer(seed=0)
    t0 = time.perf_counter()
    losses = trainer.train(ctx, feat, pca, ((valid & pd.PD_NORMAL_PLANAR) != 0).to(torch.uint8),
                           steps=args.train_steps, batch=4096, lr=2e-3, seed=0)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    # angular error of the network against PCA (planar rows) and against the
    # generator's analytic normals (every row) on an unseen scan
    tst = synth.room_scan(seed=100, n_az=int(5 * specs[0][1]), n_el=int(specs[0][1]),
                          normals=True)
    x0 = torch.from_numpy(tst.xyz).to(dev)
    g = pd.Grid(ctx, x0)
    feat, pca, valid = pd.pd_normals_pca(g)
    g.free()
    u, _ = pd.pd_mlp_forward(trainer.params, feat)
    planar = ((valid & pd.PD_NORMAL_PLANAR) != 0).cpu().numpy()
    un, pn = u.cpu().numpy(), pca.cpu().numpy()
    ang = onorm.angle(un[planar], pn[planar])
    ang_true = onorm.angle(un, tst.normals)
    defined = (valid.cpu().numpy() & 1) != 0
    ang_pca_true = onorm.angle(pn[defined], tst.normals[defined])
    ratio, k, w = 0.25, 4, 0.5
    leaf = args.leaf_max or pd.pd_autotune(ctx, x0, ratio, k=k, term=pd.PD_TERM_ORIENT, weight=w,
                                           normals=pd.pd_normals_mlp(ctx, trainer.params, feat,
                                                                     pca),
                                           sample=1_000_000)
    mean_n = float(np.mean([n for _, n in pool]))

    def serve_pass(rate, requests):
        """One Poisson stream of `requests` scans at `rate` scans/s."""
        srv = pd.Server(ctx, slots=args.serve_slots, k=k, term=pd.PD_TERM_ORIENT, weight=w,
                        mlp_params=trainer.params, normals=True)
        srv.poll(srv.submit(pool[int(np.argmin(sizes))][0], ratio=ratio))   # warm
        arrivals = np.cumsum(rng.exponential(1.0 / rate, requests))
        tickets, t_start = [], time.perf_counter()
        for i, at in enumerate(arrivals):
            d = at - (time.perf_counter() - t_start)
            if d > 0:
                time.sleep(d)
            x, n = pool[i % len(pool)]
            tickets.append((srv.submit(x, ratio=ratio), n))
        res = [(srv.poll(t)[1], n) for t, n in tickets]
        srv.close()
        assert all(r["status"] == 0 for r, _ in res)
        lat = [r["t_done_ms"] - r["t_submit_ms"] for r, _ in res]
        qwait = [r["t_admit_ms"] - r["t_submit_ms"] for r, _ in res]
        span_ms = max(r["t_done_ms"] for r, _ in res) - min(r["t_submit_ms"] for r, _ in res)
        return {"rate_per_s": rate, "requests": requests, "offered": mean_n * rate,
                "latency_ms": {"p50": _pct(lat, 50), "p99": _pct(lat, 99), "max": max(lat)},
                "queue_wait_ms": {"p50": _pct(qwait, 50), "p99": _pct(qwait, 99)},
                "throughput": sum(n for _, n in res) / (span_ms / 1e3)}

    main = serve_pass(args.serve_rate, args.serve_requests)
    # a second stream at 70 % of the throughput the first one reached: the
    # latency of the loop when it keeps up with its arrivals
    sustain = serve_pass(0.7 * main["throughput"] / mean_n, max(20, args.serve_requests // 2))
    # the plain single-scan path on the first scans of the pool, one at a time
    single_pool = pool[:args.serve_compare]
    t0 = time.perf_counter()
    for x, n in single_pool:
        xd = torch.from_numpy(np.asarray(x)).to(dev)
        g = pd.Grid(ctx, xd)
        feat, pca, _ = pd.pd_normals_pca(g)
        nrm = pd.pd_normals_mlp(ctx, trainer.params, feat, pca)
        pd.pd_decimate_ratio(g, ratio, k=k, term=pd.PD_TERM_ORIENT, weight=w, normals=nrm)
        g.free()
    torch.cuda.synchronize()
    single_s = time.perf_counter() - t0
    ctx.close()
    return {"workload": "%d requests, Poisson %.0f scans/s, room scans n log-uniform 100k-10M "
                        "(%d distinct scans, mean %.2fM), k=%d + %.1f x orientation term, network "
                        "normals, keep %g%%" % (args.serve_requests, args.serve_rate,
                                                 len(pool), np.mean([n for _, n in pool]) / 1e6,
                                                 k, w, 100 * ratio),
            "slots": args.serve_slots, "leaf_max": leaf,
            "latency_ms": main["latency_ms"], "queue_wait_ms": main["queue_wait_ms"],
            "throughput": main["throughput"], "unit": UNIT, "offered": main["offered"],
            "sustainable": sustain,
            "single_scan_path": {"value": sum(n for _, n in single_pool) / single_s,
                                 "scans": len(single_pool),
                                 "what": "the first scans one at a time, host-timed, inputs on "
                                         "device"},
            "normals": {"train_steps": args.train_steps, "train_s": train_s,
                        "final_loss": float(losses[-20:].mean().item()),
                        "angle_vs_pca_deg": {"median": float(np.degrees(np.median(ang))),
                                             "p90": float(np.degrees(np.percentile(ang, 90))),
                                             "rows": "planar rows"},
                        "angle_vs_analytic_deg": {
                            "network": {"median": float(np.degrees(np.median(ang_true))),
                                        "p90": float(np.degrees(np.percentile(ang_true, 90)))},
                            "pca": {"median": float(np.degrees(np.median(ang_pca_true))),
                                    "p90": float(np.degrees(np.percentile(ang_pca_true, 90)))},
                            "rows": "every point (PCA: where it is defined)"}}}

def run_gpu(args, wl, rank, world, local_rank, dist):
    import torch

    from paper_2311_17604_gb300 import build
    build.build()
    import paper_2311_17604_gb300.pd as pd

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if args.batch_only:
        # profiling aid: the batched leg alone (no step line)
        L = pd.lib()
        L.pd__launch_count.restype = ctypes.c_longlong
        print(json.dumps({"batch_only": True,
                          "batched": run_batched(args, pd, torch, dev,
                                                 torch.cuda.current_stream(dev))}))
        return
    scan = wl["gen"](rank)
    n, k = scan.n, wl["k"]
    import oracle
    m = oracle.target_count(n, wl["ratio"])
    xyz_dev = torch.from_numpy(scan.xyz).to(dev)
    ctx = pd.Context()
    if args.device_budget_gb > 0:
        # clouds beyond device memory: blocks past the budget (and cold ones)
        # live in pinned host memory that the kernels address in place
        ctx.set_device_budget(int(args.device_budget_gb * (1 << 30)))
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > 129 MB L2
    L = pd.lib()
    L.pd__launch_count.restype = ctypes.c_longlong

    def step():
        g = pd.Grid(ctx, xyz_dev, leaf_max=args.leaf_max, stream=stream)
        keep = pd.pd_decimate_count(g, m, k=k, stream=stream)
        st = g.stats()
        g.free()
        return keep, st

    if args.normals_only:
        # profiling aid and measurement: 16-NN + features/PCA, then the network
        # forward over every point, each timed with CUDA events on `stream`
        g = pd.Grid(ctx, xyz_dev, leaf_max=args.leaf_max, stream=stream)
        feat, pca, valid = pd.pd_normals_pca(g, stream=stream)   # warm
        params = pd.pd_mlp_init(0, stream=stream)
        pd.pd_mlp_forward(params, feat, stream=stream)
        torch.cuda.synchronize()
        t = {"normals_pca_ms": [], "mlp_forward_ms": []}
        for _ in range(max(1, args.steps)):
            for key, fn in (("normals_pca_ms", lambda: pd.pd_normals_pca(g, stream=stream)),
                            ("mlp_forward_ms", lambda: pd.pd_mlp_forward(params, feat,
                                                                         stream=stream))):
                flush.fill_(1)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record(stream)
                fn()
                e1.record(stream)
                torch.cuda.synchronize()
                t[key].append(e0.elapsed_time(e1))
        g.free()
        fw = statistics.median(t["mlp_forward_ms"]) / 1e3
        print(json.dumps({"normals_only": True, "n": n,
                          "normals_pca_ms": statistics.median(t["normals_pca_ms"]),
                          "mlp_forward_ms": fw * 1e3,
                          "mlp_tflops": n * 2 * (48 * 64 + 64 * 64 + 64 * 3) / fw / 1e12,
                          "mlp_gbs": n * (96 + 16) / fw / 1e9}))
        return

    if args.knn_only:
        for _ in range(max(1, args.steps)):
            g = pd.Grid(ctx, xyz_dev, leaf_max=args.leaf_max, stream=stream)
            pd.pd_knn_cost(g, k=k, stream=stream)
            g.free()
        torch.cuda.synchronize()
        print(json.dumps({"knn_only": True, "n": n, "k": k}))
        return

    # leaf capacity: autotuned once on a sample (the first 2M points, or the
    # workload's own sample size; outside the timed region), unless given
    leaf = args.leaf_max or pd.pd_autotune(ctx, xyz_dev, wl["ratio"], k=k,
                                           sample=wl.get("tune_sample", 2_000_000), stream=stream)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.3)
    launches0 = L.pd__launch_count()
    step_ms, stats = [], []
    for _ in range(args.steps):
        flush.fill_(1)                       # evict L2 between timed steps
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        keep, st = step()
        e1.record(stream)
        torch.cuda.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        stats.append(st)
    launches = L.pd__launch_count() - launches0
    if dist is not None:
        dist.barrier()
    clk = clocks.stop()
    assert int(keep.sum().item()) == m
    tot_s, units = aggregate(sum(step_ms) / 1e3, n * args.steps, dist)
    value = units / tot_s

    # e2e: the host C-ABI entry with pinned buffers, copies inside the timed region
    e2e = None
    if not args.no_e2e:
        xyz_pin = torch.from_numpy(scan.xyz).pin_memory()
        keep_pin = torch.empty(n, dtype=torch.uint8).pin_memory()
        xyz_np, keep_np = xyz_pin.numpy(), keep_pin.numpy()
        pd.pd_decimate_host(ctx, xyz_np, m, k=k, keep=keep_np, stream=stream)   # warm
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        # the host-buffer leg repeats the same step; at most 5 of them keep a
        # billion-point run within minutes
        e2e_steps = max(1, min(args.steps, args.e2e_steps))
        for _ in range(e2e_steps):
            pd.pd_decimate_host(ctx, xyz_np, m, k=k, keep=keep_np, stream=stream)
        e2e_s, e2e_units = aggregate(time.perf_counter() - t0, n * e2e_steps, dist)
        e2e = {"value": e2e_units / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 12 * n,
               "d2h_bytes_per_step": n, "steps": e2e_steps,
               "timed": "host clock around pd_decimate_host calls (pinned host buffers)"}

    roofline = rooflines(stats, n, k, leaf, radix_passes(scan.xyz), step_ms, clk,
                         torch.cuda.current_device())
    if rank != 0:
        return
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        ns = min(wl["sample"], n)
        nsmp, dt, threads = oracle_sample(scan.xyz, ns, k, wl["ratio"])
        cpu = {"value": nsmp / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": "first %d points (azimuth sector) of the scan, k=%d, keep %g; kNN "
                         "on %d threads, greedy single-threaded; %.1f s"
                         % (nsmp, k, wl["ratio"], threads, dt)}
    batched = serving = None
    # the batched and served legs start from an empty device: the scan and
    # the decimation's cached blocks are released first
    del xyz_dev, flush
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    if world == 1 and not args.no_batch:
        batched = run_batched(args, pd, torch, dev, stream)
    if world == 1 and not args.no_serve:
        serving = run_serving(args, pd, torch, dev)
    mean = {key: statistics.mean(s[key] for s in stats) for key in stats[0]}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.mean(step_ms),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "i64+f64",
            "data": "synthetic",
            "config": {"workload": wl["desc"], "n": n, "m": m, "k": k, "leaf_max": leaf,
                       "leaf_max_from": "option" if args.leaf_max else "pd_autotune",
                       "parallelism": "replicas" if world > 1 else "single",
                       "l2": "256 MiB buffer written between timed steps; working set > L2",
                       **({"device_budget_gb": args.device_budget_gb,
                           "memory": {key: v for key, v in ctx.memory().items()
                                      if key in ("device_peak", "host_peak")}}
                          if args.device_budget_gb > 0 else {})},
            "e2e": e2e,
            "roofline": roofline, "cpu_baseline": cpu, "clocks": clk,
            "batched": batched, "serving": serving,
            "gpu_launches": int(launches),
            "detail": {"rounds": mean["rounds"], "ms_knn": mean["ms_knn"],
                       "ms_build": mean["ms_build"], "ms_rules": mean["ms_rules"],
                       "ms_decimate": mean["ms_total"], "requeries": mean["requeries"],
                       "filtered_queries": mean["filtered_queries"],
                       "danger_queries": mean["danger_queries"],
                       "dup_removed": mean["dup_removed"], "step_ms": step_ms}}
    print(json.dumps(line), flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", default="site", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer leg")
    ap.add_argument("--e2e-steps", type=int, default=5,
                    help="steps of the host-buffer leg (at most --steps)")
    ap.add_argument("--leaf-max", type=int, default=0,
                    help="octree leaf capacity, 4..32 (0: the library default)")
    ap.add_argument("--device-budget-gb", type=float, default=0.0,
                    help="device-memory budget of the library's context (GiB); blocks past "
                         "it live in pinned host memory (0: no budget)")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched leg")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving leg")
    ap.add_argument("--batch-count", type=int, default=512)
    ap.add_argument("--batch-compare", type=int, default=48,
                    help="scans of the batch also run through slots and one at a time")
    ap.add_argument("--batch-slots", type=int, default=8)
    ap.add_argument("--serve-requests", type=int, default=200)
    ap.add_argument("--serve-rate", type=float, default=50.0)
    ap.add_argument("--serve-pool", type=int, default=0,
                    help="distinct scans reused round-robin (0: one per request)")
    ap.add_argument("--serve-compare", type=int, default=24,
                    help="scans also run one at a time through the single-scan path")
    ap.add_argument("--serve-slots", type=int, default=4)
    ap.add_argument("--train-steps", type=int, default=1000)
    ap.add_argument("--normals-only", action="store_true",
                    help="time the 16-NN/PCA pass and the network forward on the workload scan")
    ap.add_argument("--batch-only", action="store_true",
                    help="profiling aid: run the batched leg alone")
    ap.add_argument("--knn-only", action="store_true",
                    help="profiling aid: build the grid and run one full kNN/cost pass")
    args = ap.parse_args(argv)
    wl = WORKLOADS[args.workload]
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, wl, rank)
        return
    dist = None
    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(local_rank)
        tdist.init_process_group("nccl")
        dist = tdist
    run_gpu(args, wl, rank, world, local_rank, dist)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
