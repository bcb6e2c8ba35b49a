"""Benchmark: photon histories/s + ML-EM iterations/s on the 128^3 torso.

One step = the whole hot path on one acquisition: transport + tally of the
histories into the system matrix (CSR + CSC), start image, and the ML-EM
iterations.  The phantom, geometry tables and projections are resident in
HBM before the timed region (a transport plan); L2 is flushed between timed
steps.  Printed as one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (the FP64 C transport + tally) on the
host cores on a bounded sample of the same workload.  With N > 1 (torchrun)
the ranks split one acquisition of N x H histories: history ranges per rank,
events routed to the rank owning their view, ML-EM rows by views with one
all-reduce per iteration (weak scaling); --replicas gives every rank its own
acquisition instead (no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2105_13324_gb300 import phantoms as P  # noqa: E402

METRIC = "photon histories/s + MLEM iter/s (128³, 120 views) vs oracle and HBM roofline"
UNIT = "photon histories/s"

# Algorithmic work model of one history (lane operations; an FMA counts as
# one): Philox4x32-10 is 10 rounds x 10 integer ops per 4 words, plus the
# conversion to a uniform; a Woodcock flight is a log, the move, the box
# test, the voxel index and address, the attenuation and the real/virtual
# test; an accepted scatter includes the cross-section update at the new
# energy, ~2.2 rejection trials, the azimuth and the rotation; emission is
# the start point and direction.
OPS_PER_DRAW = 27.0
OPS_PER_FLIGHT = 32.0
OPS_PER_SCATTER = 90.0
OPS_PER_EMISSION = 30.0
ALU_LANES_PER_SM = 128
# DRAM bytes (read + write) counted by ncu for the present kernels, for the
# `traffic` fields: transport_kernel<float> in one launch of 1e9 histories of
# the 128^3 torso (13.38 MB + 987.47 MB: mostly the escape queue, which a
# launch of 1e8 histories keeps in L2), per history; and one ML-EM iteration's
# forward + back-projection warp-chunk kernels on the benchmark's 1e9-history
# matrix (82.28 + 0.43 MB and 99.64 + 3.52 MB, single-pass capture).  To be
# taken again (or set to None) whenever those kernels change.
TRANSPORT_DRAM_BYTES_PER_HISTORY = (13383168 + 987473664) / 1e9
MLEM_DRAM_BYTES_PER_ITER_1E9 = 82282496 + 432896 + 99639552 + 3522560


# Nominal issue rates per SM and clock of the pipes the transport kernel
# uses: FP32/INT32 lanes, 32x32->64-bit integer multiplies (Philox; the
# wide IMAD issues at half the FP32 rate) and the multi-function unit
# (log, sin/cos, reciprocal, reciprocal square root).
PIPE_RATES = {"fp32_int_lanes": 128, "imad_wide": 64, "mufu": 16}
MUFU_PER_FLIGHT = 1.0      # log of the flight length
MUFU_PER_SCATTER = 2.2 + 5.0  # a reciprocal per rejection trial (~2.2), sin+cos, two rsqrt, a reciprocal
MUFU_PER_EMISSION = 3.0    # sin+cos of the azimuth, rsqrt
IMAD_PER_BLOCK = 20.0      # Philox4x32-10: two wide multiplies per round


def transport_per_pipe(rec, flights, sm_count, sm_mhz, histories_per_s, lane_ops):
    """Per-pipe bounds of the transport kernel from the FP64 trace of a
    history sample: operations per history on each pipe, the histories/s
    that pipe alone would allow at its nominal rate, and the fraction of it
    achieved.  Philox blocks are the words drawn rounded up to blocks (the
    minimum any kernel must generate)."""
    blocks = np.ceil(rec["n_draws"] / 4.0).mean()
    per_hist = {"fp32_int_lanes": float(lane_ops),
                "imad_wide": IMAD_PER_BLOCK * float(blocks),
                "mufu": float((MUFU_PER_FLIGHT * flights + MUFU_PER_SCATTER * rec["n_compton"]).mean()
                              + MUFU_PER_EMISSION)}
    out = {}
    for pipe, n in per_hist.items():
        bound = sm_count * PIPE_RATES[pipe] * sm_mhz * 1e6 / n
        out[pipe] = {"ops_per_history": n, "rate_per_sm_clock": PIPE_RATES[pipe], "bound_histories_per_s": bound,
                     "frac": histories_per_s / bound}
    out["philox_blocks_per_history"] = float(blocks)
    return out


def _launch_histories(g) -> int:
    """Histories per transport launch of an analog FP32 build: the library
    runs the longest power-of-two chunk in 2^27..2^30 whose escape queue
    (40-byte records for the fraction ~1.1 w_max of photons that can reach a
    collimator) fits in 4 GiB."""
    t = g.hole_diam_mm / g.hole_len_mm
    q = min(1.1 * (t / math.sqrt(1.0 + t * t) * 1.02 + 1e-6), 1.0)
    k = 1 << 27
    while k < (1 << 30) and 2 * k * q * 40 <= 2 ** 32:
        k *= 2
    return k


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), float(pk.get("sm_max_mhz", 2070.0)), "measured"
    except Exception:
        return 6800.0, 2070.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self._t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _maxreduce(value: float, ws: int, device=None) -> float:
    if ws == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def shard_seed(base_seed: int, rank: int) -> int:
    """Rank r reconstructs its own acquisition: seed base + 7919 r."""
    return base_seed + 7919 * rank


def whole_job_rate(world_size: int, histories_per_rank: int, max_ms_per_step: float) -> float:
    """Histories per second of the whole job: every rank runs its own
    histories, the slowest rank sets the step time."""
    return world_size * histories_per_rank / (max_ms_per_step * 1e-3)


# ---------------------------------------------------------------------------
# CPU oracle arm (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------
def oracle_sample(w, target_s: float = 12.0, max_histories: int = 400_000_000):
    """Times the oracle (FP64 C transport + tally + count matrix) on the host
    cores over the first H_s histories of the workload, H_s chosen so that
    the run takes about target_s seconds."""
    import oracle
    pr = oracle.Problem(w.phantom, w.geometry)
    threads = os.cpu_count() or 1
    t0 = time.perf_counter()
    one = 200_000
    oracle.run(pr, w.seed, 0, one, 1)
    single = one / max(time.perf_counter() - t0, 1e-6)
    t0 = time.perf_counter()
    cal = 2_000_000
    oracle.run(pr, w.seed, 0, cal, threads)
    rate = cal / max(time.perf_counter() - t0, 1e-6)
    hs = int(min(max_histories, max(cal, rate * target_s)))
    t0 = time.perf_counter()
    rows, cols, fates = oracle.run(pr, w.seed, 0, hs, threads)
    c = oracle.system_counts(rows, cols, pr.n_rows, pr.n_voxels)
    dt = time.perf_counter() - t0
    a = oracle.system_matrix(c, oracle.histories_per_voxel(pr.n_voxels, 0, hs))
    y = np.asarray(a @ w.phantom.activity.ravel().astype(np.float64))
    x = oracle.mlem_init(a, y)
    t1 = time.perf_counter()
    n_it = 3
    oracle.mlem(a, y, x, n_it)
    mlem_s = (time.perf_counter() - t1) / n_it
    return {"value": hs / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"histories 0..{hs - 1} of the {w.name} workload (FP64 C transport + tally + count matrix, "
                      f"{threads} threads), {dt:.1f} s; ML-EM float64 on that sample's matrix (nnz {c.nnz}): "
                      f"{1.0 / mlem_s:.2f} iter/s",
            "histories": hs, "seconds": dt, "mlem_iter_per_s": 1.0 / mlem_s, "mlem_nnz": int(c.nnz),
            "single_core_value": single, "single_core_sample": f"histories 0..{one - 1}, 1 thread"}


def run_reference(args, w):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    per = max(3.0, min(15.0, 150.0 / max(args.steps + args.warmup, 1)))
    import oracle
    oracle.build()
    pr = oracle.Problem(w.phantom, w.geometry)
    threads = os.cpu_count() or 1
    cal = 2_000_000
    t0 = time.perf_counter()
    oracle.run(pr, w.seed, 0, cal, threads)
    rate = cal / max(time.perf_counter() - t0, 1e-6)
    hs = int(max(cal, rate * per))
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        rows, cols, _ = oracle.run(pr, w.seed, i * hs, hs, threads)
        oracle.system_counts(rows, cols, pr.n_rows, pr.n_voxels)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    value = hs * len(times) / sum(times)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(times)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": w.name, "histories_per_step": hs,
                                            "step": "transport + tally only (no ML-EM)",
                                            "note": "CPU oracle on a bounded history sample per step; the GPU "
                                                    "step also runs 50 ML-EM iterations, which the oracle's "
                                                    "ML-EM rate on the benchmark matrix is reported for in the "
                                                    "GPU line (reduced_precision.oracle_mlem_iter_per_s)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"{hs} histories per step of the {w.name} workload, transport + tally"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def spmv_bytes(system, nnz, M, N, val_bytes):
    """Algorithmic bytes of one ML-EM iteration: both matrix streams, the
    pointer arrays, and the vectors over non-empty rows / columns (x gathered
    once, y, r written and read, s, x read and written)."""
    rp, _, _ = system.export_csr()
    cp, _, _, _ = system.export_csc()
    m_nz = int(np.count_nonzero(np.diff(rp)))
    n_nz = int(np.count_nonzero(np.diff(cp)))
    return (2 * nnz * (val_bytes + 4) + 4 * (M + 1) + 4 * (N + 1)
            + 4 * (n_nz + m_nz + 2 * m_nz + n_nz + 2 * n_nz))


def mlem_timing(mc, system, y, x, n_iter, flush, stream, reps=5, label="f32"):
    """Median device time of n_iter ML-EM iterations (L2 flushed before each
    repetition), CUDA events on the launching stream."""
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms = []
    for _ in range(reps):
        flush.zero_()
        mc.mc_mlem_init(system, y, x)
        e0.record(stream)
        mc.mlem_iterate(system, y, x, n_iter)
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    it = float(np.median(ms)) / n_iter
    return {label: {"ms_per_iter": it, "iter_per_s": 1e3 / it}}


def roof_instance(mc, plan, histories, seed, n_iter, flush, stream, hbm_gbs, peak_kind):
    """Build the benchmark geometry with `histories` histories (a matrix far
    larger than L2) and time the SpMV pair against HBM bandwidth."""
    import torch
    s = plan.build(0, histories, seed + 2000)
    inf = s.info()
    M, N = inf["n_rows"], inf["n_cols"]
    y = torch.rand(M, device="cuda", generator=torch.Generator(device="cuda").manual_seed(7)) * 10.0
    x = torch.ones(N, device="cuda")
    out = {"histories": histories, "nnz": inf["nnz"], "build_s": (inf["build_ms_transport"] + inf["build_ms_detect"]
                                                                  + inf["build_ms_assembly"]) / 1e3}
    reps_iter = min(n_iter, 20)
    for vt, vb in (("f32", 4), ("f16", 2)):
        if vt == "f16" and inf["max_count"] > 2048:
            continue
        s.set_value_type(vt)
        mc.mc_mlem_init(s, y, x)
        mc.mlem_iterate(s, y, x, 3)
        t = mlem_timing(mc, s, y, x, reps_iter, flush, stream, reps=3, label=vt)[vt]
        b = spmv_bytes(s, inf["nnz"], M, N, vb)
        gbs = b / (t["ms_per_iter"] * 1e-3) / 1e9
        out[vt] = {"ms_per_iter": t["ms_per_iter"], "bytes_per_iter": b, "achieved_gbs": gbs, "frac": gbs / hbm_gbs}
    out["peak_gbs"] = hbm_gbs
    out["peak_kind"] = peak_kind
    s.free()
    return out


def serving_benchmark(mc, n_phantoms: int, histories: int, n_iter: int, stream):
    """Mixed-size serving batch: n_phantoms torso acquisitions (48^3..128^3,
    40-120 views), each with its own system (`histories` histories) and
    Poisson projections; reconstructed together by the batched graph, and
    one by one for the per-phantom latency: with mlem_iterate (autotuned
    kernels) and as a batch of one (one graph per request)."""
    import torch
    mix = P.serving_mix(n_phantoms, seed=5)
    systems, ys = [], []
    t0 = time.perf_counter()
    for ph, g, counts, seed in mix:
        s = mc.mc_build_system(ph, g, histories, seed)
        q = torch.zeros(s.shape[0], dtype=torch.float32, device="cuda")
        mc.mc_project(s, torch.as_tensor(ph.activity.ravel()).cuda(), q)
        ys.append(torch.as_tensor(P.poisson_counts(q.cpu().numpy(), counts, seed)).cuda())
        systems.append(s)
    build_s = time.perf_counter() - t0
    xs = [torch.zeros(s.shape[1], dtype=torch.float32, device="cuda") for s in systems]
    batch = mc.Batch(systems, ys, xs)
    batch.mlem(n_iter, stream)                 # capture + warm-up
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms = []
    for _ in range(5):
        e0.record(stream)
        batch.mlem(n_iter, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    batch_ms = float(np.median(ms))
    # the same reconstruction with all iterations in one persistent launch
    batch.mlem_persistent(n_iter, stream)
    torch.cuda.synchronize()
    ms_p = []
    for _ in range(5):
        e0.record(stream)
        batch.mlem_persistent(n_iter, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_p.append(e0.elapsed_time(e1))
    batch_persistent_ms = float(np.median(ms_p))
    # one request at a time through a batch of one (compacted system, one
    # CUDA graph per reconstruction); before the autotuner, which may
    # replace a system's streaming tiles by row groups
    lat_g = []
    for s, y, x in zip(systems, ys, xs):
        b1 = mc.Batch([s], [y], [x])
        b1.mlem(n_iter, stream)
        torch.cuda.synchronize()
        e0.record(stream)
        b1.mlem(n_iter, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        lat_g.append(e0.elapsed_time(e1))
        b1.free()
    lat = []
    for s, y, x in zip(systems, ys, xs):
        mc.mc_system_autotune(s)
        mc.mc_mlem_init(s, y, x)
        mc.mlem_iterate(s, y, x, n_iter)
        torch.cuda.synchronize()
        e0.record(stream)
        mc.mc_mlem_init(s, y, x)
        mc.mlem_iterate(s, y, x, n_iter)
        e1.record(stream)
        torch.cuda.synchronize()
        lat.append(e0.elapsed_time(e1))
    sizes = sorted({int(ph.shape[0]) for ph, _, _, _ in mix})
    out = {"phantoms": n_phantoms, "grids": sizes, "histories_per_phantom": histories, "mlem_iters": n_iter,
           "build_s": build_s, "batch_ms": batch_ms, "images_per_s": n_phantoms / (batch_ms * 1e-3),
           "batch_persistent_ms": batch_persistent_ms,
           "persistent_images_per_s": n_phantoms / (batch_persistent_ms * 1e-3),
           "latency_ms_p50": float(np.percentile(lat, 50)), "latency_ms_p99": float(np.percentile(lat, 99)),
           "sequential_images_per_s": n_phantoms / (sum(lat) * 1e-3),
           "latency_graph_ms_p50": float(np.percentile(lat_g, 50)),
           "latency_graph_ms_p99": float(np.percentile(lat_g, 99)),
           "sequential_graph_images_per_s": n_phantoms / (sum(lat_g) * 1e-3),
           "nnz_total": int(sum(s.info()["nnz"] for s in systems))}
    batch.free()
    for s in systems:
        s.free()
    return out


def _segment_means(img, seg):
    """Mean image value in each of the 16 myocardial segments."""
    return np.array([img[seg == k].mean() if np.any(seg == k) else 0.0 for k in range(16)])


def reduced_precision_benchmark(mc, system, y_host, w, n_iter, flush, stream):
    """N1: ML-EM images with the matrix values stored in each type against
    the FP64 oracle image on the same matrix and projections (relative L2
    over the image and the 16 myocardial segment means), with ms per
    iteration.  f32 / f16 / bf16 store the counts (exact here: the largest
    count is far below 256); f16_a / bf16_a store A = C / n_v itself,
    rounded (the conventional reduced-precision storage).  The oracle's
    float64 ML-EM runs on the CPU on the benchmark matrix exported from the
    device, timed as the oracle's ML-EM rate on this matrix.  A synthetic
    count matrix with counts up to 6000 (oracle-built) shows the rounding of
    counts beyond the exact range of half / bfloat16."""
    import torch

    import oracle
    M, N = system.shape
    cp, ri, cnt, nv = system.export_csc()
    c = sp_csc(cnt, ri, cp, (M, N))
    a = oracle.system_matrix(c, nv)
    y = np.asarray(y_host, np.float64)
    t0 = time.perf_counter()
    x_o = oracle.mlem(a, y, oracle.mlem_init(a, y), n_iter)
    oracle_s = time.perf_counter() - t0
    seg = P.segments16(w.phantom).ravel()
    seg_o = _segment_means(x_o, seg)
    yd = torch.as_tensor(np.asarray(y_host, np.float32)).cuda()
    x = torch.zeros(N, dtype=torch.float32, device="cuda")
    out = {"matrix": f"benchmark matrix ({M} x {N}, nnz {c.nnz}, largest count {int(cnt.max()) if cnt.size else 0})",
           "mlem_iters": n_iter, "oracle": "float64 ML-EM (CPU, scipy) on the exported matrix and the same y",
           "oracle_mlem_iter_per_s": n_iter / oracle_s, "types": {}}
    for vt in ("f32", "f16", "bf16", "f16_a", "bf16_a"):
        system.set_value_type(vt)
        t = mlem_timing(mc, system, yd, x, n_iter, flush, stream, label=vt)[vt]
        mc.mc_mlem_init(system, yd, x)
        mc.mlem_iterate(system, yd, x, n_iter)
        img = x.cpu().numpy().astype(np.float64)
        seg_g = _segment_means(img, seg)
        t["rel_l2_vs_oracle"] = float(np.linalg.norm(img - x_o) / np.linalg.norm(x_o))
        t["segment_mean_rel_err_max"] = float(np.max(np.abs(seg_g - seg_o) / np.abs(seg_o)))
        t["segment_mean_rel_err_mean"] = float(np.mean(np.abs(seg_g - seg_o) / np.abs(seg_o)))
        out["types"][vt] = t
    system.set_value_type("f32")
    # counts beyond the exact range (synthetic, oracle-built): 128 x 256
    n_rows, n_cols, H = 128, 256, 5 * 256
    rows, cols = P.random_events(n_rows, n_cols, (10, 30), 6000, seed=31)
    cs = oracle.system_counts(rows, cols, n_rows, n_cols)
    a_s = oracle.system_matrix(cs, oracle.histories_per_voxel(n_cols, 0, H))
    y_s = P.poisson_counts(a_s @ np.ones(n_cols), 50.0 * n_rows, 32)
    want = oracle.mlem(a_s, y_s, oracle.mlem_init(a_s, y_s), 20)
    s_syn = mc.mc_system_from_events(n_rows, n_cols, rows, cols, 0, H)
    ys = torch.as_tensor(y_s).cuda()
    hc = {"matrix": f"synthetic {n_rows} x {n_cols} counts 1..6000 (oracle-built), 20 iterations"}
    for vt in ("f32", "f16", "bf16"):
        s_syn.set_value_type(vt, allow_rounding=True)
        xs = torch.zeros(n_cols, dtype=torch.float32, device="cuda")
        mc.mc_mlem_init(s_syn, ys, xs)
        mc.mlem_iterate(s_syn, ys, xs, 20)
        hc[vt + "_rel_l2_vs_oracle"] = float(np.linalg.norm(xs.cpu().numpy() - want) / np.linalg.norm(want))
    s_syn.free()
    out["high_counts"] = hc
    return out, a, x_o


def sp_csc(data, indices, indptr, shape):
    import scipy.sparse as sp
    return sp.csc_matrix((np.asarray(data, np.int64), indices, indptr), shape=shape)


def penalised_benchmark(mc, system, y_host, a, w, n_iter, stream):
    """N2: the penalised Poisson likelihood solved by EM-preconditioned
    gradient steps through the library (paper Sec. 5.1 likelihood plus a
    quadratic 6-neighbour prior; beta relative to the mean sensitivity),
    against plain FP32 ML-EM on the same matrix: ms per iteration, the final
    objective against the oracle's float64 objective of the same image, and
    the image's relative L2 to the ML-EM image."""
    import torch

    import oracle
    from paper_2105_13324_gb300 import autograd as AG
    M, N = system.shape
    yd = torch.as_tensor(np.asarray(y_host, np.float32)).cuda()
    x_em = torch.zeros(N, dtype=torch.float32, device="cuda")
    mc.mc_mlem_init(system, yd, x_em)
    mc.mlem_iterate(system, yd, x_em, n_iter)
    em = x_em.cpu().numpy().astype(np.float64)
    sens = torch.zeros(N, dtype=torch.float64, device="cuda")
    mc.mc_sensitivity(system, sens)
    s_mean = float(sens.mean())
    shape = w.phantom.shape
    y = np.asarray(y_host, np.float64)
    out = {"iters": n_iter, "beta_basis": f"beta = rel x mean sensitivity ({s_mean:.4g})", "runs": {}}
    for rel in (0.0, 1e-4, 1e-3, 1e-2, 1e-1):
        beta = rel * s_mean
        hist = []
        AG.penalised_reconstruct(system, yd, shape, beta, 2)          # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        x = AG.penalised_reconstruct(system, yd, shape, beta, n_iter, history=hist)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        img = x.cpu().numpy().astype(np.float64)
        phi_o = oracle.penalised_objective(a, y, img, shape, beta)
        out["runs"][f"{rel:g}"] = {"beta": beta, "ms_per_iter": 1e3 * dt / n_iter,
                                   "phi": hist[-1], "phi_oracle": phi_o,
                                   "phi_rel_diff": float(abs(hist[-1] - phi_o) / abs(phi_o)),
                                   "rel_l2_vs_mlem": float(np.linalg.norm(img - em) / np.linalg.norm(em))}
    return out


def _blocks(q, geometry, b=8):
    # projection (views x bins_v x bins_u) summed over b x b bins
    V, bv, bu = geometry.n_views, geometry.n_bins_v, geometry.n_bins_u
    return q.reshape(V, bv // b, b, bu // b, b).sum(axis=(2, 4)).ravel()


def fd_benchmark(mc, w, analog, analog_ms, seed, n_batches, stream):
    """Forced detection against the analog build: throughput, and the
    figure of merit 1 / (relative variance x time) of the projection of the
    phantom's activity summed over 8 x 8-bin blocks, per block, FD over
    analog.  FD: n_batches builds of one history per voxel each (batch
    means give the variance); analog: the benchmark step's matrix, whose
    count variance is Poisson."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    g = w.geometry
    act = torch.as_tensor(w.phantom.activity.ravel().astype(np.float32)).to(dev)
    M, N = analog.shape
    # analog: q = A act, Var(q_j) = sum_v C_jv (act_v / n_v)^2 = (A (act^2 / n_v))_j
    _, _, _, nv = analog.export_csc()
    q = torch.zeros(M, dtype=torch.float32, device=dev)
    mc.mc_project(analog, act, q)
    qa = _blocks(q.cpu().numpy().astype(np.float64), g)
    x2 = torch.as_tensor((w.phantom.activity.ravel().astype(np.float64) ** 2 / np.maximum(nv, 1)).astype(np.float32)).to(dev)
    mc.mc_project(analog, x2, q)
    va = _blocks(q.cpu().numpy().astype(np.float64), g)
    plan = mc.Plan(w.phantom, g, "fp32", forced=True)
    s = plan.build(0, N, seed)                      # warm-up
    s.free()
    qb, t_ms, t_fd, t_asm, events = [], 0.0, 0.0, 0.0, 0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for b in range(n_batches):
        torch.cuda.synchronize()
        e0.record(stream)
        s = plan.build(b * N, N, seed)
        e1.record(stream)
        torch.cuda.synchronize()
        t_ms += e0.elapsed_time(e1)
        inf = s.info()
        t_fd += inf["build_ms_detect"]
        t_asm += inf["build_ms_assembly"]
        events += inf["n_events"]
        mc.mc_project(s, act, q)
        qb.append(_blocks(q.cpu().numpy().astype(np.float64), g))
        s.free()
    plan.free()
    qb = np.array(qb)
    qf = qb.mean(axis=0)
    H = n_batches * N
    out = {"histories": H, "batches": n_batches, "histories_per_batch": N,
           "ms": t_ms, "histories_per_s": H / (t_ms * 1e-3),
           "fd_kernel_ms": t_fd, "assembly_ms": t_asm,
           "weighted_events": events, "events_per_history": events / H,
           "weighted_events_per_s": events / (t_ms * 1e-3),
           "analog_events_per_s": analog.info()["n_events"] / (analog_ms * 1e-3),
           "projection_total_rel_diff": float((qf.sum() - qa.sum()) / qa.sum())}
    if n_batches < 2:
        return out                                   # no batch variance, no figure of merit
    vf = qb.var(axis=0, ddof=1) / n_batches
    ok = (qa > 0) & (va > 0) & (vf > 0)
    if not np.any(ok):
        return out
    fom_a = qa[ok] ** 2 / (va[ok] * analog_ms)
    fom_f = qf[ok] ** 2 / (vf[ok] * t_ms)
    ratio = fom_f / fom_a
    out.update({"fom_block": "projection of the activity over 8x8-bin blocks",
                "fom_ratio_median": float(np.median(ratio)),
                "fom_ratio_p10": float(np.percentile(ratio, 10)), "fom_ratio_p90": float(np.percentile(ratio, 90)),
                "blocks": int(ok.sum()),
                "projection_total_z": float((qf.sum() - qa.sum())
                                            / np.sqrt(va.sum() + qb.sum(axis=1).var(ddof=1) / n_batches))})
    return out


def run_split(args, w):
    """N > 1 ranks (torchrun, one GPU each, NCCL): one acquisition of
    N x H histories split over the ranks (paper_2105_13324_gb300.sharded).
    Rank g runs histories [g N H / N, ...), routes its events to the rank
    owning their view (one all-to-all), assembles the rows of its views, and
    ML-EM runs with one all-reduce of the N-voxel back-projection per
    iteration.  Work per rank is fixed as N grows: weak scaling."""
    import torch
    import torch.distributed as dist

    from paper_2105_13324_gb300 import build as B
    from paper_2105_13324_gb300 import mcspect as mc
    from paper_2105_13324_gb300 import sharded

    ws, rank, local = _dist()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (the CUDA library has no CPU fallback)")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist.init_process_group("nccl", device_id=dev)
    mc.load(B.build())
    H = int(args.histories or w.n_histories)
    total = ws * H
    n_iter = int(args.mlem_iters or w.mlem_iters)
    g = w.geometry
    rpv = g.n_bins_u * g.n_bins_v
    M, N = g.n_views * rpv, int(np.prod(w.phantom.shape))
    comm, ops = sharded.TorchComm(), sharded.LibraryOps(mc)
    stream = torch.cuda.current_stream()
    plan = mc.Plan(w.phantom, g, "fp32")
    # projections of this rank's views: an independent realisation (seed +
    # 1000) projects the activity; Poisson counts at the workload's total x N
    truth, (v0, v1) = sharded.split_build(ops, comm, plan, M, N, rpv, total, w.seed + 1000)
    m_p = (v1 - v0) * rpv
    ybar = torch.zeros(m_p, dtype=torch.float32, device=dev)
    mc.mc_project(truth, torch.as_tensor(w.phantom.activity.ravel()).to(dev), ybar)
    truth.free()
    tot = torch.tensor([float(ybar.double().sum())], dtype=torch.float64, device=dev)
    part = float(tot[0])
    dist.all_reduce(tot)
    y_host = P.poisson_counts(ybar.cpu().numpy(), w.total_counts * ws * part / max(float(tot[0]), 1e-300),
                              w.noise_seed + rank)
    y = torch.as_tensor(y_host).to(dev)
    flush = torch.empty(int(args.flush_mb) * (1 << 20) // 4, dtype=torch.float32, device=dev)

    def step(y_part):
        s, _ = sharded.split_build(ops, comm, plan, M, N, rpv, total, w.seed)
        x = sharded.split_mlem(ops, comm, s, y_part, m_p, N, n_iter)
        return s, x

    for _ in range(args.warmup):
        step(y)[0].free()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    dist.barrier()
    torch.cuda.synchronize()
    l0 = mc.mc_kernel_launches()
    infos = []
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        s, x = step(y)
        ev[k][1].record(stream)
        infos.append(s.info())
        s.free()
    torch.cuda.synchronize()
    launches = mc.mc_kernel_launches() - l0
    dist.barrier()
    clk = clocks.stop()
    ms = _maxreduce(float(np.mean([a.elapsed_time(b) for a, b in ev])), ws, dev)
    # end to end: y from pinned host memory each step, the image read back
    y_pin = torch.as_tensor(y_host).pin_memory()
    x_pin = torch.empty(N, dtype=torch.float32).pin_memory()
    y_dev = torch.empty_like(y)
    e2e_ms = []
    for _ in range(max(2, min(args.steps, 3))):
        flush.zero_()
        torch.cuda.synchronize()
        dist.barrier()
        t0 = time.perf_counter()
        y_dev.copy_(y_pin, non_blocking=True)
        s, x = step(y_dev)
        x_pin.copy_(x, non_blocking=True)
        torch.cuda.synchronize()
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
        s.free()
    e2e_ms = _maxreduce(float(np.mean(e2e_ms)), ws, dev)
    if rank == 0:
        inf = infos[-1]
        line = {
            "metric": METRIC, "value": total / (ms * 1e-3), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name, "grid": list(w.phantom.shape), "views": g.n_views,
                       "bins": [g.n_bins_v, g.n_bins_u], "histories_per_step": total, "histories_per_rank": H,
                       "mlem_iters": n_iter, "l2": f"flushed ({args.flush_mb} MB write) between timed steps",
                       "parallelism": f"split over {ws} GPUs: history ranges per rank, events routed to the rank "
                                      "owning their view (one all-to-all), ML-EM rows by views with one all-reduce "
                                      "of the N-voxel back-projection per iteration"},
            "rank0_part": {"views": [v0, v1], "rows": m_p, "nnz": inf["nnz"],
                           "build_ms_transport": inf["build_ms_transport"]},
            "clocks": clk,
            "e2e": {"value": total / (e2e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": int(4 * m_p),
                    "d2h_bytes_per_step": int(4 * N)},
            "gpu_launches": int(launches),
            "cpu_baseline": None,
        }
        print(json.dumps(line), flush=True)
    plan.free()
    dist.destroy_process_group()
    return 0


def run_ours(args, w):
    import torch

    from paper_2105_13324_gb300 import build as B
    from paper_2105_13324_gb300 import mcspect as mc

    ws, rank, local = _dist()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (the CUDA library has no CPU fallback)")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    mc.load(B.build())
    H = int(args.histories or w.n_histories)
    n_iter = int(args.mlem_iters or w.mlem_iters)
    seed = shard_seed(w.seed, rank)
    stream = torch.cuda.current_stream()

    # inputs resident in HBM: plan (map + tables) and the projections y
    plan = mc.Plan(w.phantom, w.geometry, "fp32")
    truth = plan.build(0, H, seed + 1000)
    act = torch.as_tensor(w.phantom.activity.ravel()).to(dev)
    M, N = truth.shape
    ybar = torch.zeros(M, dtype=torch.float32, device=dev)
    mc.mc_project(truth, act, ybar)
    y_host = P.poisson_counts(ybar.cpu().numpy(), w.total_counts, w.noise_seed + rank)
    truth.free()
    y = torch.as_tensor(y_host).to(dev)
    x = torch.zeros(N, dtype=torch.float32, device=dev)
    flush = torch.empty(int(args.flush_mb) * (1 << 20) // 4, dtype=torch.float32, device=dev)

    def step():
        s = plan.build(0, H, seed)
        mc.mc_mlem_init(s, y, x)
        mc.mlem_iterate(s, y, x, n_iter)
        return s

    for _ in range(args.warmup):
        step().free()
    torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    _barrier(ws)
    torch.cuda.synchronize()
    l0 = mc.mc_kernel_launches()
    t_transport, t_detect, t_assembly, infos = [], [], [], []
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        s = step()
        ev[k][1].record(stream)
        inf = s.info()
        t_transport.append(inf["build_ms_transport"])
        t_detect.append(inf["build_ms_detect"])
        t_assembly.append(inf["build_ms_assembly"])
        infos.append(inf)
        if k == args.steps - 1:
            last = s
        else:
            s.free()
    torch.cuda.synchronize()
    launches = mc.mc_kernel_launches() - l0
    _barrier(ws)
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms = _maxreduce(float(np.mean(step_ms)), ws, dev)
    value = whole_job_rate(ws, H, ms)

    # ML-EM alone on the last system
    inf = infos[-1]
    hbm_gbs, sm_max_mhz, peak_kind = _peaks()
    mlem = mlem_timing(mc, last, y, x, n_iter, flush, stream)
    it_ms = mlem["f32"]["ms_per_iter"]
    mlem_bytes = spmv_bytes(last, inf["nnz"], M, N, 4)
    reduced = penalised = None
    if rank == 0 and not args.no_oracle_images:
        reduced, a_bench, _ = reduced_precision_benchmark(mc, last, y_host, w, n_iter, flush, stream)
        penalised = penalised_benchmark(mc, last, y_host, a_bench, w, int(args.penalised_iters), stream)
        del a_bench

    # SpMV roofline on a matrix larger than L2 (same geometry, more histories)
    roof = None
    if args.roof_histories and rank == 0:
        roof = roof_instance(mc, plan, int(args.roof_histories), seed, n_iter, flush, stream, hbm_gbs, peak_kind)
    serving = None
    if args.serving_phantoms and rank == 0:
        serving = serving_benchmark(mc, int(args.serving_phantoms), int(args.serving_histories), 30, stream)
    fd = None
    if args.fd_batches and rank == 0:
        analog_ms = float(np.mean(t_transport) + np.mean(t_detect) + np.mean(t_assembly))
        fd = fd_benchmark(mc, w, last, analog_ms, seed, int(args.fd_batches), stream)

    # transport roofline (lane-op issue bound), work counted from an FP64
    # trace of a history sample of this workload
    rec = mc.mc_trace_histories(w.phantom, w.geometry, seed, 0, 200_000, precision="fp64")
    esc = (rec["fate"] == 2).astype(np.float64)
    flights = rec["n_virtual"] + rec["n_real"] + esc
    ops = (OPS_PER_DRAW * rec["n_draws"] + OPS_PER_FLIGHT * flights + OPS_PER_SCATTER * rec["n_compton"]
           + OPS_PER_EMISSION).mean()
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    alu_peak = sm_count * ALU_LANES_PER_SM * sm_max_mhz * 1e6 / 1e12  # T lane-ops/s
    t_tr = float(np.mean(t_transport))
    achieved = ops * H / (t_tr * 1e-3) / 1e12
    per_pipe = transport_per_pipe(rec, flights, sm_count, sm_max_mhz, H / (t_tr * 1e-3), ops)

    # end to end through the public API with host buffers
    y_pin = torch.as_tensor(y_host).pin_memory()
    x_pin = torch.empty(N, dtype=torch.float32).pin_memory()
    y_dev = torch.empty_like(y)

    def e2e_step():
        s = mc.mc_build_system(w.phantom, w.geometry, H, seed)
        y_dev.copy_(y_pin, non_blocking=True)
        mc.mc_mlem_init(s, y_dev, x)
        mc.mlem_iterate(s, y_dev, x, n_iter)
        x_pin.copy_(x, non_blocking=True)
        torch.cuda.synchronize()
        s.free()
        return float(x_pin[0])

    e2e_step()
    e2e_ms = []
    for _ in range(max(2, min(args.steps, 5))):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_step()
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
    e2e_val = whole_job_rate(ws, H, _maxreduce(float(np.mean(e2e_ms)), ws, dev))
    n_mat = len(w.phantom.rho)
    V = w.geometry.n_views
    h2d = w.phantom.material.size + 3 * 8 * n_mat + 2 * V * (8 + 4) + 3 * n_mat * (8 + 4) + 4 * M
    d2h = 4 * N + 5 * 8 + 4 + 4 + 4

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = oracle_sample(w, target_s=args.cpu_seconds)
        if reduced is not None:
            # the oracle's float64 ML-EM on the benchmark matrix itself (one
            # thread, scipy), beside the GPU's iterations/s on the same matrix
            cpu["mlem_iter_per_s_benchmark_matrix"] = reduced["oracle_mlem_iter_per_s"]

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name, "grid": list(w.phantom.shape), "voxel_mm": w.phantom.voxel_mm,
                       "views": V, "bins": [w.geometry.n_bins_v, w.geometry.n_bins_u], "histories_per_step": H,
                       "mlem_iters": n_iter, "matrix": "CSR+CSC u32 counts, f32 values",
                       "l2": f"flushed ({args.flush_mb} MB write) between timed steps",
                       "parallelism": f"{ws} independent acquisitions" if ws > 1 else "1 GPU"},
            "mlem_iter_per_s": 1e3 / it_ms,
            "transport_histories_per_s": H / (t_tr * 1e-3),
            "build_histories_per_s": H / ((t_tr + float(np.mean(t_detect)) + float(np.mean(t_assembly))) * 1e-3),
            "step_breakdown_ms": {"transport": t_tr, "detect": float(np.mean(t_detect)),
                                  "assembly": float(np.mean(t_assembly)),
                                  "mlem": it_ms * n_iter},
            "matrix": {"rows": M, "cols": N, "nnz": inf["nnz"], "events": inf["n_events"], "fates": inf["fates"],
                       "max_count": inf["max_count"]},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "T lane-ops/s",
                         "frac": achieved / alu_peak,
                         "traffic": (TRANSPORT_DRAM_BYTES_PER_HISTORY * min(H, _launch_histories(w.geometry))
                                     if w.name == "torso128" else None),
                         "traffic_basis": "DRAM bytes of one launch (min(histories, "
                                          f"{_launch_histories(w.geometry)}) histories), per history from an ncu "
                                          "capture of one 1e9-history torso128 launch",
                         "kernel": "transport_kernel<float>",
                         "ops_per_history": ops,
                         "per_pipe": per_pipe,
                         "peak_basis": f"{sm_count} SMs x {ALU_LANES_PER_SM} lanes x {sm_max_mhz:.0f} MHz"},
            "roofline_mlem": {"bound": "hbm", "achieved": mlem_bytes / (it_ms * 1e-3) / 1e9, "peak": hbm_gbs,
                              "unit": "GB/s", "frac": mlem_bytes / (it_ms * 1e-3) / 1e9 / hbm_gbs,
                              "traffic": (MLEM_DRAM_BYTES_PER_ITER_1E9
                                          if w.name == "torso128" and H == 10 ** 9 else None),
                              "bytes_per_iter": mlem_bytes, "peak_kind": peak_kind,
                              "note": "benchmark matrix; rows of ~3.7 entries: bound by the L1-to-L2 request "
                                      "rate of the vector gathers (one 32-byte request per entry), not by DRAM "
                                      "bytes"},
            "roofline_mlem_roof": roof,
            "serving": serving,
            "forced_detection": fd,
            "reduced_precision": reduced,
            "penalised": penalised,
            "clocks": clk,
            "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": int(launches),
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    last.free()
    plan.free()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", default="torso128")
    ap.add_argument("--histories", type=int, default=None, help="override histories per step")
    ap.add_argument("--mlem-iters", type=int, default=None)
    ap.add_argument("--flush-mb", type=int, default=512)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serving-phantoms", type=int, default=64, help="mixed serving batch size (0: skip)")
    ap.add_argument("--serving-histories", type=float, default=2e7, help="histories per serving phantom")
    ap.add_argument("--fd-batches", type=int, default=8,
                    help="forced-detection builds of one history per voxel each (0: skip)")
    ap.add_argument("--roof-histories", type=float, default=1e11,
                    help="histories of the large-matrix SpMV roofline instance (0: skip)")
    ap.add_argument("--no-oracle-images", action="store_true",
                    help="skip the value-type and penalised-solver comparisons with the oracle's images")
    ap.add_argument("--penalised-iters", type=int, default=20)
    ap.add_argument("--split", action="store_true",
                    help="run the split path even on one rank (under torchrun; checks the multi-GPU code path)")
    ap.add_argument("--replicas", action="store_true",
                    help="with N > 1 ranks: independent acquisitions per rank instead of one split acquisition")
    args = ap.parse_args(argv)
    w = P.workload(args.workload)
    if args.impl == "reference":
        return run_reference(args, w)
    if (_dist()[0] > 1 and not args.replicas) or args.split:
        return run_split(args, w)
    return run_ours(args, w)


if __name__ == "__main__":
    sys.exit(main())
