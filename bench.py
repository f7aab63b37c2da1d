"""Benchmark: online rate-distortion estimation + ground truth on GB300.

One step = one pass of the whole hot path over one field: value range; ZFP
block pass (sampled-block estimate fused with the every-block ground truth);
bin width from the exact MSE_sp; SZ pass (sampled-point estimate fused with
the every-point ground truth); entropy, Huffman costs, selection.  Workload:
a Hurricane-shaped 100x500x500 float32 field (GRF k^-11/3 plus 8 tanh fronts,
scaled to [0, 300]) at eb_rel 1e-4 (the paper's throughput setting) and
r_sp = 5% (its default).  The field (100 MB) fits in L2, so L2 is flushed by
writing a 256 MB buffer before every timed step; the flush is outside the
timed events.

Under torchrun each rank evaluates its own independent field (weak scaling,
no collective on the data path); the timed K steps are bracketed by a barrier
and a synchronize, and the time is the maximum over ranks.

--impl reference times the CPU oracle (the plain restatement of the method)
on a bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "R-D estimate GB/s per GB300 (SZ+ZFP) & % HBM peak; batched vs plain; p99 latency"
WORKLOAD = "hurricane_100x500x500_grf_tanh_f32"
SHAPE = (100, 500, 500)
EB_REL = 1e-4
R_SP = 0.05
FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="rdsel", choices=["rdsel", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-planes", type=int, default=100,
                    help="planes of the field in the CPU-baseline sample")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the batched-snapshot measurement")
    ap.add_argument("--batch-steps", type=int, default=20)
    ap.add_argument("--batch-subset", default="all", choices=["all", "small"],
                    help="small: 20 ATM + 2 Hurricane + 1 512^3 fields (1.3 GB), for profiling")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving-loop measurement")
    ap.add_argument("--no-curve", action="store_true",
                    help="skip the rate-distortion sweep (error bounds 1e-2 .. 1e-6)")
    ap.add_argument("--no-nyx", action="store_true",
                    help="skip the four 512^3 fields at eb_rel 1e-3 and 1e-5")
    ap.add_argument("--no-classic", action="store_true",
                    help="skip the classic SZ truth beside the prequantised one")
    ap.add_argument("--serve-population", type=int, default=256)
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--serve-seconds", type=float, default=10.0,
                    help="longest span of arrivals per rate")
    ap.add_argument("--serve-rates", default="50,100,200,500,1000,2000")
    ap.add_argument("--source-hashes", action="store_true",
                    help="print the source hash of each profiled kernel and exit")
    return ap.parse_args()


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# Translation units of each kernel that profiles/ and traffic.json describe;
# a kernel's recorded DRAM traffic holds only while the hash of its units
# (and the package headers they include) is the one recorded beside it.
KERNEL_UNITS = {
    "range": ("rd_reduce.cu",),
    "huffman": ("rd_reduce.cu",),
    "zfp_pass": ("rd_zfp.cu", "rd_zfp3.cu"),
    "sz_pass": ("rd_sz.cu", "rd_sz_tma.cu"),
    "batch": ("rd_batch.cu",),
    "classic": ("rd_sz_classic.cu",),
}


def kernel_source_hash(kernel: str) -> str:
    """Hash of the sources one profiled kernel is compiled from: its
    translation units and every header they include, followed through the
    package's own headers (the public header included)."""
    csrc = os.path.join(ROOT, "paper_1806_08901_gb300", "csrc")
    inc = os.path.join(ROOT, "include")
    seen, todo = [], list(KERNEL_UNITS[kernel])
    while todo:
        fn = todo.pop(0)
        if fn in seen:
            continue
        seen.append(fn)
        path = os.path.join(csrc, fn)
        if not os.path.exists(path):
            path = os.path.join(inc, fn)
        with open(path, encoding="utf-8") as f:
            todo += re.findall(r'#include "([^"]+)"', f.read())
    h = hashlib.sha256()
    for fn in sorted(seen):
        path = os.path.join(csrc, fn)
        if not os.path.exists(path):
            path = os.path.join(inc, fn)
        with open(path, "rb") as f:
            h.update(fn.encode() + f.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel sources; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    rec = d.get(WORKLOAD, {}).get(kernel)
    if not rec or kernel not in KERNEL_UNITS or rec.get("source_hash") != kernel_source_hash(kernel):
        return None
    return rec.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def _query(self, extra=()):
        return ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                "--format=csv,noheader,nounits", *extra]

    def start(self):
        try:
            self.lines += subprocess.run(self._query(), capture_output=True, text=True,
                                         timeout=20).stdout.splitlines()
            self.proc = subprocess.Popen(self._query(["-lms", "20"]), stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except (OSError, subprocess.SubprocessError):
            self.proc = None

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=10)
                self.lines += out.splitlines()
            except subprocess.SubprocessError:
                self.proc.kill()
        try:
            self.lines += subprocess.run(self._query(), capture_output=True, text=True,
                                         timeout=20).stdout.splitlines()
        except (OSError, subprocess.SubprocessError):
            pass

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


SNAPSHOT = "snapshot_79x1800x3600_13x100x500x500_6x512^3_f32"


def snapshot_alg_bytes(fields, r_sp: float) -> float:
    """Algorithmic bytes of the estimate: one read of every value (range), the
    sampled ZFP blocks and the sampled SZ points with their one-cell halo,
    4 + 4 r + 4 r (5/4)^d bytes per value."""
    tot = 0.0
    for x in fields:
        d = x.dim()
        tot += x.numel() * (4.0 + 4.0 * r_sp + 4.0 * r_sp * (1.25 ** d))
    return tot


def bench_snapshot(R, ctx, stream, steps: int, peak: float, peak_kind: str, subset: str = "all"):
    """The batched estimate of a whole snapshot (79 2D 1800x3600, 13
    100x500x500 and 6 512^3 fields, 6.57 GB, far larger than L2) in one
    rd_select_batch call, against the same fields through per-field rd_select
    calls, both timed with CUDA events on the stream."""
    import ctypes as C

    import torch

    import synth

    specs = synth.snapshot_specs()
    if subset == "small":
        specs = specs[:20] + specs[79:81] + specs[92:93]
    fields = [synth.make_field_torch(sp) for sp in specs]
    torch.cuda.synchronize()
    prms = [R.params(eb=sp["eb_rel"], r_sp=R_SP) for sp in specs]
    nbytes = sum(4 * x.numel() for x in fields)
    call = ctx.batch_call(fields, prms)
    for _ in range(3):  # autotune, capture, replay
        rc = call.run(stream)
        if rc != 0:
            raise R.RdselError(rc, "rd_select_batch", R.status_string(rc))
    cfg = ctx.batch_get_config()
    n0 = ctx.launch_count()
    ms = []
    for _ in range(steps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        call.run(stream)
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
    launches = (ctx.launch_count() - n0) / steps
    batch_ms = statistics.median(ms)
    res = call.results()
    # per-kernel device times of the batched launches (a separate profiled plan)
    ctx.set_profiling(True)
    for _ in range(3):
        call.run(stream)
    ctx.reset_profile()
    nprof = 5
    for _ in range(nprof):
        call.run(stream)
    # per call (the sampled-blocks pass is one launch per dimensionality)
    kstats = {k: v[0] / nprof for k, v in ctx.kernel_stats().items() if v[1] and k.startswith("batch")}
    ctx.set_profiling(False)
    # plain: one rd_select per field, arguments marshalled beforehand
    L = R.lib()
    recs = []
    for x, p in zip(fields, prms):
        f, keep = R.make_field(x)
        recs.append((f, p, R.rd_result(), keep))
    sp = R._stream(stream)
    for _ in range(2):
        for f, p, r, _k in recs:
            L.rd_select(ctx.h, C.byref(f), C.byref(p), C.byref(r), sp)
    pms = []
    for _ in range(max(3, steps // 4)):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for f, p, r, _k in recs:
            L.rd_select(ctx.h, C.byref(f), C.byref(p), C.byref(r), sp)
        b.record(stream)
        b.synchronize()
        pms.append(a.elapsed_time(b))
    plain_ms = statistics.median(pms)
    same = all(R._todict(r) == g for (_f, _p, r, _k), g in zip(recs, res))
    alg = snapshot_alg_bytes(fields, R_SP)
    achieved = alg / (batch_ms / 1e3) / 1e9
    out = {
        "workload": SNAPSHOT if subset == "all" else SNAPSHOT + "_subset20+2+1", "fields": len(fields),
        "field_bytes": nbytes, "r_sp": R_SP,
        "eb_rel": "per field from {1e-3,1e-4,1e-5}", "l2": "inputs 6.6 GB, larger than L2",
        "ms": batch_ms, "value": nbytes / (batch_ms / 1e3) / 1e9, "unit": "GB/s",
        "plain_ms": plain_ms, "plain_value": nbytes / (plain_ms / 1e3) / 1e9,
        "speedup_vs_plain": plain_ms / batch_ms, "gpu_launches": launches,
        "records_equal_plain": same, "split": cfg,
        "kernel_ms": kstats,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "peak_kind": peak_kind,
                     "unit": "GB/s", "frac": achieved / peak, "alg_bytes": alg},
        "selections": {"sz": sum(1 for r in res if r["selection"] == 0),
                       "zfp": sum(1 for r in res if r["selection"] == 1)},
    }
    del fields, call, recs
    torch.cuda.empty_cache()
    return out


SERVE_WORKLOAD = "serving_poisson_2d512-1800x3600_3d64-512cubed_f32"


CURVE_EBS = (1e-2, 1e-3, 1e-4, 1e-5, 1e-6)


def bench_rd_curve(R, ctx, x, stream, reps: int = 5):
    """The rate-distortion sweep of the benchmark field over the error
    bounds 1e-2 .. 1e-6 (rd_rd_curve: Algorithm 1 and its truth at each
    bound, and the selection based on error bound), timed with CUDA events
    over whole sweeps; the choices per bound."""
    import torch

    p = R.params(eb=EB_REL, r_sp=R_SP)
    pts = ctx.rd_curve(x, p, CURVE_EBS, stream)  # warm-up
    ms = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        pts = ctx.rd_curve(x, p, CURVE_EBS, stream)
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
    points = []
    for pt in pts:
        e, t, t2 = pt["est"], pt["truth"], pt["truth_eb"]
        points.append({"eb_rel": pt["eb"], "selection": e["selection"], "optimum_gt": t["best_gt"],
                       "selection_eb": pt["selection_eb"], "best_eb_gt": pt["best_eb_gt"],
                       "br_sz": e["br_sz"], "br_zfp": e["br_zfp"], "psnr_zfp": e["psnr_zfp"],
                       "br_sz_gt": t["br_sz_gt"], "br_zfp_gt": t["br_zfp_gt"],
                       "psnr_sz_gt": t["psnr_sz_gt"], "psnr_zfp_gt": t["psnr_zfp_gt"],
                       "br_sz_eb": pt["est_eb"]["br_sz"], "br_sz_eb_gt": t2["br_sz_gt"],
                       "psnr_sz_eb_gt": t2["psnr_sz_gt"], "psnr_zfp_eb_gt": t2["psnr_zfp_gt"]})
    return {"workload": WORKLOAD, "eb_rel": list(CURVE_EBS), "r_sp": R_SP,
            "ms_per_sweep": statistics.median(ms),
            "calls_per_bound": "rd_evaluate + rd_estimate_sz(2 eb_abs) + rd_ground_truth(eb_abs)",
            "points": points}


def bench_classic(R, ctx, x, stream, reps: int = 3):
    """The classic SZ truth (prediction from reconstructed neighbours, one
    launch per wavefront) beside the prequantised truth at the same bound
    eb_sz = EB_REL * VR, on the benchmark field and on one 1800x3600
    ATM-shaped field: device time per call and what each truth reports."""
    import torch

    import synth

    def timed(fn):
        fn()  # first call, then a captured repeat
        fn()
        ms = []
        for _ in range(reps):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            out = fn()
            b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
        return statistics.median(ms), out

    atm = synth.make_field_torch(synth.snapshot_specs()[0])
    res = {}
    for name, f in (("hurricane_100x500x500", x), ("atm_1800x3600", atm)):
        vr = float(f.max()) - float(f.min())
        eb_sz = EB_REL * vr
        p = R.params(eb=EB_REL, r_sp=R_SP)
        ms_c, tc = timed(lambda: ctx.ground_truth_classic(f, p, eb_sz, stream=stream))
        ms_d, td = timed(lambda: ctx.ground_truth(f, p, eb_sz, stream))
        # the sampled estimate at the same bin: entropy + 0.5 (the paper's
        # offset) against the classic stream's bit-rate
        e = ctx.estimate_sz(f, p, 2.0 * eb_sz, stream)
        res[name] = {"eb_sz": eb_sz, "ms_classic": ms_c, "ms_prequantised": ms_d,
                     "entropy_est": e["entropy"], "br_sz_est": e["br_sz"],
                     "br_sz_huff_est": e["br_sz_huff"],
                     "br_sz_classic": tc["br_sz_gt"], "br_sz_prequantised": td["br_sz_gt"],
                     "psnr_classic": tc["psnr_sz_gt"], "psnr_prequantised": td["psnr_sz_gt"],
                     "nesc_classic": tc["sz_nesc_gt"], "nesc_prequantised": td["sz_nesc_gt"]}
    del atm
    return res


NYX_WORKLOAD = "nyx_512^3_density_exp2G_velocity_grf_f32"


def bench_nyx(R, ctx, stream, peak: float, peak_kind: str, reps: int = 10):
    """rd_evaluate (estimate + full ground truth) on the four 512^3 NYX-shaped
    fields (log-normal density exp(2 G), three velocity GRFs) at eb_rel 1e-3
    and 1e-5, r_sp 5%: device time per call with CUDA events (inputs of
    512 MB, four times L2, so no flush), and the two full passes' fractions of
    the HBM peak (one 4-byte read per value each) from their live events."""
    import torch

    import synth

    fields = synth.config3_fields_torch()
    torch.cuda.synchronize()
    names = ("density", "vx", "vy", "vz")
    cases = []
    for name, x in zip(names, fields):
        nbytes = 4 * x.numel()
        for eb in (1e-3, 1e-5):
            p = R.params(eb=eb, r_sp=R_SP)
            for _ in range(3):
                e, t = ctx.evaluate(x, p, stream)
            ms = []
            for _ in range(reps):
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                ctx.evaluate(x, p, stream)
                b.record(stream)
                b.synchronize()
                ms.append(a.elapsed_time(b))
            ctx.set_profiling(True)
            for _ in range(3):
                ctx.evaluate(x, p, stream)
            ctx.reset_profile()
            for _ in range(reps):
                ctx.evaluate(x, p, stream)
            st = ctx.kernel_stats()
            ctx.set_profiling(False)
            kms = {k: v[0] / v[1] for k, v in st.items() if v[1]}
            step = statistics.median(ms)
            case = {"field": name, "eb_rel": eb, "ms": step,
                    "GB_s": nbytes / (step / 1e3) / 1e9,
                    "frac_hbm_step": 3 * nbytes / (step / 1e3) / 1e9 / peak,
                    "kernel_ms": kms, "selection": e["selection"], "best_gt": t["best_gt"],
                    "br_sz": e["br_sz"], "br_zfp": e["br_zfp"],
                    "br_sz_gt": t["br_sz_gt"], "br_zfp_gt": t["br_zfp_gt"]}
            for k in ("zfp_pass", "sz_pass", "range"):
                if k in kms:
                    case["frac_" + k] = nbytes / (kms[k] / 1e3) / 1e9 / peak
            cases.append(case)
    del fields
    torch.cuda.empty_cache()
    tot_ms = sum(c["ms"] for c in cases)
    return {"workload": NYX_WORKLOAD, "r_sp": R_SP, "peak": peak, "peak_kind": peak_kind,
            "l2": "inputs 512 MB per field, larger than L2",
            "value": sum(4 * 512 ** 3 for _ in cases) / (tot_ms / 1e3) / 1e9, "unit": "GB/s",
            "cases": cases}


def bench_sz_stream(R, ctx, x, stream, reps: int = 5):
    """rd_sz_compress on the benchmark field at eb_sz = EB_REL * VR: the SZ
    stream of the prequantised truth written on the device (truth, symbols,
    offsets, packing; the code lengths built on the host), timed with CUDA
    events per call; its size and compression ratio."""
    import torch

    vr = float(x.max()) - float(x.min())
    eb_sz = EB_REL * vr
    p = R.params(eb=EB_REL, r_sp=R_SP)
    nbits = ctx.sz_compress(x, p, eb_sz, stream=stream)
    out = torch.empty(8 * ((nbits + 63) // 64), dtype=torch.uint8, device=x.device)
    ctx.sz_compress(x, p, eb_sz, out, stream)
    ms = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ctx.sz_compress(x, p, eb_sz, out, stream)
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
    return {"workload": WORKLOAD, "eb_sz": eb_sz, "ms_per_call": statistics.median(ms),
            "stream_bits": nbits, "bits_per_value": nbits / x.numel(),
            "compression_ratio": 32.0 * x.numel() / nbits,
            "GB_s": x.numel() * 4 / (statistics.median(ms) / 1e3) / 1e9}


def _serve_rate(R, srv, fields, prm, rate, n_req, seed, max_s, population):
    """Poisson arrivals at `rate` for at most n_req requests or max_s seconds
    of arrivals; returns throughput, latency percentiles and residency."""
    import time

    import synth

    reqs = [r for r in synth.serving_requests(rate, n_req, seed=seed, population=population)
            if r["t"] <= max_s]
    srv.reset_stats()
    st0 = srv.stats()
    done = 0
    nbytes = 0
    t0 = time.perf_counter()
    for i, r in enumerate(reqs):
        while True:
            now = time.perf_counter() - t0
            if now >= r["t"]:
                break
            if r["t"] - now > 2e-3:
                time.sleep(r["t"] - now - 1e-3)
        eb = min(prm, key=lambda e: abs(e - r["eb_rel"]))
        srv.submit(fields[r["field"]], prm[eb], key=1 + r["field"], tag=i)
        nbytes += 4 * fields[r["field"]].numel()
        done += len(srv.poll(256, wait_ms=0))
    while done < len(reqs):
        done += len(srv.poll(256, wait_ms=5000))
    wall = time.perf_counter() - t0
    st = srv.stats()
    hits = st["resident_hits"] - st0["resident_hits"]
    return {"rate_req_s": rate, "requests": len(reqs), "wall_s": wall,
            "throughput_req_s": len(reqs) / wall, "throughput_GB_s": nbytes / wall / 1e9,
            "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "mean_ms": st["mean_ms"],
            "max_ms": st["max_ms"], "resident_hits": hits, "hit_rate": hits / max(1, len(reqs)),
            "evictions": st["evictions"] - st0["evictions"],
            "resident_bytes": st["resident_bytes"]}


def bench_serving(R, population: int, n_req: int, rates, budget: int = 120 << 30,
                  max_s: float = 10.0, evict_rate: float = 200.0):
    """The serving loop under Poisson arrivals: requests name fields of a
    population held in pinned host memory (2D ny ~ logU[512, 1800], nx ~
    logU[512, 3600], or 3D cubes with side ~ logU[64, 512]; spectra k^a, a ~
    U[-4, -2]) and an error bound from {1e-2 .. 1e-6}; each rate runs for
    n_req requests or max_s seconds of arrivals.  Under the 120 GB budget
    every field stays resident (each is requested once first); a second run
    starts cold under a budget of a quarter of the population, so requests
    miss, copy their field in and evict others."""
    import torch

    import synth

    specs = synth.serving_population(seed=synth.seed_for(5), population=population)
    fields = []
    for sp in specs:
        g = synth.grf_torch(tuple(sp["shape"]), sp["alpha"], sp["seed"])
        h = torch.empty(g.shape, dtype=torch.float32, pin_memory=True)
        h.copy_(g)
        fields.append(h)
        del g
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    prm = {eb: R.params(eb=eb, r_sp=R_SP) for eb in (1e-2, 1e-3, 1e-4, 1e-5, 1e-6)}
    pop_bytes = sum(4 * f.numel() for f in fields)
    out = {"workload": SERVE_WORKLOAD, "population": population, "hbm_budget_bytes": budget,
           "population_bytes": pop_bytes, "slots": 4, "window": 16,
           "requests_per_rate": f"{n_req} or {max_s:g} s of arrivals",
           "slots_are": "host threads, each running one request's launch chain on its own "
                        "stream; concurrent requests overlap on the device, they are not "
                        "merged into one launch",
           "rates": []}
    with R.Server(0, slots=4, window=16, hbm_budget=budget) as srv:
        for i, f in enumerate(fields):  # first touch: copy in
            srv.submit(f, prm[1e-4], key=1 + i, tag=i)
        got = 0
        while got < len(fields):
            got += len(srv.poll(256, wait_ms=5000))
        for k, rate in enumerate(rates):
            out["rates"].append(_serve_rate(R, srv, fields, prm, rate, n_req,
                                            synth.seed_for(5, 100 + k), max_s, population))
    small = pop_bytes // 4
    with R.Server(0, slots=4, window=16, hbm_budget=small) as srv:
        ev = _serve_rate(R, srv, fields, prm, evict_rate, n_req, synth.seed_for(5, 200), max_s,
                         population)
    ev["hbm_budget_bytes"] = small
    out["evicting"] = ev
    del fields
    return out


def host_cpu() -> dict:
    """The host's logical core count and CPU model (lscpu, else /proc/cpuinfo)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() in ("Model name", "Vendor ID") and ":" in line:
                val = line.split(":", 1)[1].strip()
                model = val if model is None else model + " / " + val
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith("model name"):
                        model = line.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    return {"nproc": os.cpu_count(), "cpu_model": model}


def _oracle_step(O, s, p):
    O.select(s, p)
    O.ground_truth(s, p)


def cpu_baseline(x_host, planes: int, steps: int = 1, all_cores: bool = False):
    """Time the oracle (select + ground truth) on the first `planes` planes,
    on one core; with all_cores, also one sample per host core at once in
    threads (the oracle releases the interpreter lock inside its C calls),
    each thread on its own slab of planes."""
    from concurrent.futures import ThreadPoolExecutor

    import oracle as O

    s = x_host[:planes].copy()
    p = O.params(eb=EB_REL, r_sp=R_SP)
    t = []
    for _ in range(steps):
        t0 = time.perf_counter()
        _oracle_step(O, s, p)
        t.append(time.perf_counter() - t0)
    sec = statistics.mean(t)
    out = {"value": 4.0 * s.size / sec / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle",
           "sample": f"first {planes} of {SHAPE[0]} planes ({s.size} points), "
                     f"select + ground truth, {steps} run(s), {sec:.2f} s each",
           **host_cpu()}
    if all_cores:
        n = os.cpu_count() or 1
        n0 = x_host.shape[0]
        slabs = []
        for i in range(n):
            lo = (i * planes) % max(1, n0 - planes + 1)
            slabs.append(x_host[lo:lo + planes].copy())
        t0 = time.perf_counter()
        with ThreadPoolExecutor(max_workers=n) as ex:
            list(ex.map(lambda a: _oracle_step(O, a, p), slabs))
        wall = time.perf_counter() - t0
        tot = sum(a.size for a in slabs)
        out["all_cores"] = {"value": 4.0 * tot / wall / 1e9, "unit": "GB/s", "cores": n,
                            "wall_s": wall,
                            "sample": f"{n} slabs of {planes} planes, one per thread, "
                                      f"select + ground truth"}
    return out


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import numpy as np

    import synth

    x = synth.config2_field()
    # a bounded sample: the whole --steps/--warmup run stays near 90 s of CPU
    # work at the oracle's ~45 ms per 500x500 plane
    planes = int(max(1, min(20, 90.0 / (0.045 * max(1, args.steps + args.warmup)))))
    for _ in range(args.warmup):
        cpu_baseline(x, planes, 1)
    t0 = time.perf_counter()
    res = cpu_baseline(x, planes, args.steps)
    total = time.perf_counter() - t0
    ms = 1e3 * total / max(1, args.steps)
    line = {"impl": "reference", "metric": METRIC, "value": res["value"], "unit": "GB/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+i32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "eb_rel": EB_REL, "r_sp": R_SP,
                       "sample_planes": planes},
            "cpu_baseline": res,
            "e2e": {"value": res["value"], "unit": "GB/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    del np
    print(json.dumps(line))


def max_over_ranks(value: float, world: int, device=None) -> float:
    """The maximum of a per-rank float over all ranks (one all-reduce of the
    time; no data-path collective)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist

    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_value(nbytes_per_rank: int, steps: int, world: int, max_ms: float) -> float:
    """Whole-job GB/s: every rank's fields over the slowest rank's time."""
    return world * nbytes_per_rank * steps / (max_ms / 1e3) / 1e9


def main():
    args = parse()
    if args.source_hashes:
        print(json.dumps({k: kernel_source_hash(k) for k in KERNEL_UNITS}))
        return
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    import torch.distributed as dist

    import synth
    from paper_1806_08901_gb300 import _build, rdsel as R

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    if rank == 0:
        _build.build()
    if world > 1:
        dist.barrier()
    ctx = R.Context(dev.index)
    stream = torch.cuda.current_stream()

    x = synth.config2_field_torch(seed=synth.seed_for(2, rank), shape=SHAPE, device=dev)
    n = x.numel()
    nbytes = 4 * n
    p = R.params(eb=EB_REL, r_sp=R_SP)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def timed_steps(profiled):
        """K steps, each after an L2 flush, bracketed by a barrier and a
        synchronize; with profiled, the call's graph also records a CUDA
        event pair around each of its kernels."""
        ctx.set_profiling(profiled)
        # the first call of a key launches directly, the second captures
        # its graph, later ones replay it
        for _ in range(max(args.warmup, 3)):
            flush.zero_()
            ctx.evaluate(x, p, stream)
        ctx.reset_profile()
        l0 = ctx.launch_count()
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(args.steps):
            flush.zero_()
            starts[i].record(stream)
            ctx.evaluate(x, p, stream)
            ends[i].record(stream)
        torch.cuda.synchronize()
        w = time.perf_counter() - t0
        if world > 1:
            dist.barrier()
        st = ctx.kernel_stats() if profiled else None
        ctx.set_profiling(False)
        return sum(a.elapsed_time(b) for a, b in zip(starts, ends)), w, ctx.launch_count() - l0, st

    est_ref, truth_ref = ctx.evaluate(x, p, stream)
    clocks = ClockSampler(dev.index)
    clocks.start()
    # the headline: the call as a user makes it, no events inside it
    dev_ms, wall, launches, _ = timed_steps(False)
    # the same steps again with per-kernel events (each event pair adds a
    # few microseconds to the step), for the per-kernel times and roofline
    dev_ms_prof, _, _, stats = timed_steps(True)
    clocks.stop()

    dev_ms_max = max_over_ranks(dev_ms, world, dev)
    value = weak_scaling_value(nbytes, args.steps, world, dev_ms_max)

    # estimate-only throughput (rd_select: range + sampled ZFP + sampled SZ)
    est_ms = []
    for _ in range(min(args.steps, 50)):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ctx.select(x, p, stream)
        b.record(stream)
        b.synchronize()
        est_ms.append(a.elapsed_time(b))

    # end to end through the C ABI from pinned host memory (H2D inside)
    xh = torch.empty(x.shape, dtype=torch.float32, pin_memory=True)
    xh.copy_(x)
    e2e_s = []
    for i in range(min(args.steps, 20) + 2):
        t0 = time.perf_counter()
        ctx.evaluate(xh, p, stream)
        if i >= 2:
            e2e_s.append(time.perf_counter() - t0)
    e2e_val = world * nbytes / statistics.mean(e2e_s) / 1e9

    peak, peak_kind = measured_peaks()
    per_kernel = {k: {"ms_per_launch": v[0] / v[1], "launches": v[1], "share": None}
                  for k, v in stats.items() if v[1]}
    total_k = sum(v[0] for v in stats.values())
    for k, v in stats.items():
        if v[1]:
            per_kernel[k]["share"] = v[0] / total_k
    dom = max(per_kernel, key=lambda k: per_kernel[k]["ms_per_launch"] * per_kernel[k]["launches"])
    # algorithmic bytes per launch: each full pass reads the field once
    alg_bytes = {"range": nbytes, "zfp_pass": nbytes, "sz_pass": nbytes}
    ab = alg_bytes.get(dom, 0)
    achieved = ab / (per_kernel[dom]["ms_per_launch"] / 1e3) / 1e9 if ab else 0.0
    roofline = {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": peak,
                "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                "traffic": recorded_traffic(dom),
                "alg_bytes_per_launch": ab}

    line = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dev_ms_max / args.steps,
        "ms_per_step_with_kernel_events": dev_ms_prof / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+i32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "eb_rel": EB_REL, "r_sp": R_SP,
                   "l2": "flushed (256 MB write) before every timed step",
                   "parallelism": f"independent fields per rank x{world}"},
        "roofline": roofline,
        "frac_hbm_step": (3 * nbytes * args.steps / (dev_ms_max / 1e3) / 1e9) / peak,
        "estimate_only": {"value": nbytes / (statistics.mean(est_ms) / 1e3) / 1e9, "unit": "GB/s",
                          "ms": statistics.mean(est_ms)},
        "e2e": {"value": e2e_val, "unit": "GB/s", "h2d_bytes_per_step": nbytes,
                "d2h_bytes_per_step": C_RESULT_BYTES},
        "gpu_launches": launches,
        "kernels": per_kernel,
        "wall_s": wall,
        "clocks": clocks.summary(),
        "result": {"selection": est_ref["selection"], "best_gt": truth_ref["best_gt"],
                   "br_sz": est_ref["br_sz"], "br_zfp": est_ref["br_zfp"],
                   "br_sz_gt": truth_ref["br_sz_gt"], "br_zfp_gt": truth_ref["br_zfp_gt"],
                   "psnr_zfp": est_ref["psnr_zfp"], "psnr_zfp_gt": truth_ref["psnr_zfp_gt"]},
    }
    if not args.no_curve and world == 1:
        line["rd_curve"] = bench_rd_curve(R, ctx, x, stream)
    if not args.no_nyx and world == 1:
        line["nyx_512"] = bench_nyx(R, ctx, stream, peak, peak_kind)
    if not args.no_classic and world == 1:
        line["classic_truth"] = bench_classic(R, ctx, x, stream)
        line["sz_stream"] = bench_sz_stream(R, ctx, x, stream)
    if not args.no_batch and world == 1:
        line["batched"] = bench_snapshot(R, ctx, stream, args.batch_steps, peak, peak_kind,
                                         args.batch_subset)
    if not args.no_serve and world == 1:
        rates = [float(v) for v in args.serve_rates.split(",") if v]
        line["serving"] = bench_serving(R, args.serve_population, args.serve_requests, rates,
                                        max_s=args.serve_seconds)
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(x.cpu().numpy(), args.cpu_planes, 1, all_cores=True)
    if rank == 0:
        print(json.dumps(line))
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


# bytes of the result records read back per call (rd_result + rd_truth + status)
def _result_bytes():
    import ctypes as C

    from paper_1806_08901_gb300 import rdsel as R

    return C.sizeof(R.rd_result) + C.sizeof(R.rd_truth) + 4


C_RESULT_BYTES = None

if __name__ == "__main__":
    C_RESULT_BYTES = _result_bytes()
    main()
