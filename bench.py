#!/usr/bin/env python3
"""Benchmark of the GB300 parallel sparse-blossom decoder.

Default workload (N = 1): one persistent batched launch over 1,000,000 shots of
the rotated surface code, d in {7, 9, ..., 21} with d rounds each (125,000 shots
per d, shuffled), uniform p = 0.003, synthetic syndromes from a seeded sampler.
One step = decoding the whole batch (defect compaction, Alg. 1 level-1
clustering, level-1 and top-level sparse blossom, tracing) with inputs resident
in HBM.  The syndromes (248 MB) exceed the 129 MB L2, so no flush is needed.

Also reported: the plain one-shot-per-launch path on a subsample, the end-to-end
number through the public API with pinned host buffers, the roofline of the
dominant kernel, clocks during the timed region, and the CPU oracle timed on
this host's cores on a bounded sample.

`--impl reference` times the CPU oracle (the reference arm of this build) on
the same workload, a bounded sample per step.

Multi-GPU (torchrun): every rank decodes its own batch (replicas, weak scaling,
no data-path collective); the reported time is the maximum over ranks.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from synth import mixed_batch, rotated_surface_code, rotated_surface_code_circuit, sample_shots  # noqa: E402

METRIC = "shots/s and us per round at d,p (batched vs plain GPU)"
UNIT = "shots/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--shots-per-d", type=int, default=125000)
    ap.add_argument("--p", type=float, default=0.003)
    ap.add_argument("--seed", type=int, default=2026)
    ap.add_argument("--plain-shots", type=int, default=2000)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--quick", action="store_true", help="small workload (profiling)")
    ap.add_argument("--kcap", type=int, default=0, help="detection events per main-pass slab (0 = auto)")
    ap.add_argument("--no-autotune", action="store_true", help="skip the launch-shape autotuner")
    ap.add_argument("--serve-seconds", type=float, default=5.0, help="serving run length (0 = skip); 5 s = 10^6 windows at 200k/s")
    ap.add_argument("--serve-rate", type=float, default=200000.0, help="Poisson arrival rate, windows/s")
    ap.add_argument("--serve-oracle", type=int, default=3000, help="served windows checked against the oracle")
    ap.add_argument("--serve-curve", type=int, default=1, help="also serve at 50k, 100k and 400k windows/s")
    ap.add_argument("--extra-configs", type=int, default=1,
                    help="add the d=5 / d=11 configurations and the d=25..51 per-round scaling to the line")
    ap.add_argument("--serve-curve-seconds", type=float, default=2.0)
    ap.add_argument("--scaling", action="store_true",
                    help="scaling study: d in {25,31,41,51} x p in {.001,.003,.005}, us per round vs d")
    ap.add_argument("--scaling-shots", type=int, default=10000)
    ap.add_argument("--configs", action="store_true",
                    help="d=5 one-shot-per-launch and d=11 non-uniform configurations, batched vs plain vs oracle")
    ap.add_argument("--stream-study", action="store_true",
                    help="sliding-window decoding of long histories (W = 2d, C = d) vs whole-history decoding")
    ap.add_argument("--schedule-study", action="store_true",
                    help="alternative cluster schedules: parallel event count, throughput, Theorem 1 check")
    ap.add_argument("--event-study", action="store_true",
                    help="parallel event count per round, hierarchical vs global, d = 9..49, p = 1e-3..1e-5")
    ap.add_argument("--study-shots", type=int, default=1024)
    ap.add_argument("--study-d", type=int, nargs="*", default=None, help="event study: only these distances")
    ap.add_argument("--study-p", type=float, nargs="*", default=None, help="event study: only these error rates")
    ap.add_argument("--noise", default="phenomenological", choices=["phenomenological", "circuit", "circuit-physical"],
                    help="event study noise model: phenomenological graph, or the circuit-level detector graph "
                         "under the uniform or the physically motivated model")
    ap.add_argument("--study-save", default="", help="directory for the first outputs and diagnostics of every point")
    ap.add_argument("--scaling-save", default="", help="directory for the first outputs of every point")
    return ap.parse_args()


DS = [7, 9, 11, 13, 15, 17, 19, 21]


def workload(args, rank):
    from paper_2609_12262_gb300.replicas import shard_seed
    graphs, gid, offs, syn = mixed_batch(DS, args.shots_per_d, args.p, seed=shard_seed(args.seed, rank))
    return graphs, gid, offs, syn


PROFILE = os.path.join(ROOT, "profiles", "batch_kernel_mixed_d7-21_p003.md")
KERNEL_SOURCES = ["decoder.cu", "qec_internal.h", "capi.cpp"]


_TOKENS = re.compile(r'"(?:\\.|[^"\\])*"|//[^\n]*|/\*.*?\*/', re.S)


def _code_only(text):
    """Source text without comments and with whitespace collapsed (string
    literals kept), so that editing a comment does not count as a change."""
    text = _TOKENS.sub(lambda m: m.group(0) if m.group(0).startswith('"') else " ", text)
    return " ".join(text.split())


def kernel_sha256():
    """SHA-256 over the code (comments and whitespace aside) of the kernel sources."""
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2609_12262_gb300", "csrc", f)) as fh:
            h.update(_code_only(fh.read()).encode())
    return h.hexdigest()


def profile_figure(name):
    """A per-shot figure of the committed ncu summary, or None when it is missing
    or the kernel sources changed since the counters were taken."""
    try:
        text = open(PROFILE).read()
        value = float(re.search(name + r":\s*([0-9.]+)", text).group(1))
        sha = re.search(r"kernel_sources_sha256:\s*([0-9a-f]{64})", text).group(1)
    except Exception:
        return None, "no ncu summary"
    if sha != kernel_sha256():
        return None, "kernel changed since the ncu capture"
    return value, os.path.relpath(PROFILE, ROOT)


def measured_traffic(shots):
    """DRAM bytes per launch of the main pass (per shot from the ncu summary,
    scaled to this launch's shots), or None."""
    per_shot, src = profile_figure("dram_bytes_per_shot")
    if per_shot is None:
        return None, src
    return per_shot * shots, "ncu dram__bytes_read.sum + dram__bytes_write.sum per shot x shots (%s)" % src


# Issue peak of the GB300: 152 SMs x 4 warp schedulers x 1 warp-instruction per
# clock x 2.07 GHz (largest SM clock).
ISSUE_PEAK = 152 * 4 * 2.07e9


def alu_roofline(shots, launch_s):
    """Secondary roofline: warp instructions issued per second (instruction count
    per shot from the ncu summary, live launch time) against the issue peak."""
    per_shot, src = profile_figure("warp_instructions_per_shot")
    if per_shot is None:
        return None
    achieved = per_shot * shots / launch_s
    return {"bound": "alu", "achieved": achieved, "peak": ISSUE_PEAK, "unit": "warp-instructions/s",
            "frac": achieved / ISSUE_PEAK,
            "note": "smsp__inst_executed per shot (%s) x shots / CUDA-event launch time; peak = 152 SMs x 4 "
                    "schedulers x 2.07 GHz" % src}


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            j = json.load(f)
        return float(j["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi samples during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        except Exception:
            return out
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1])); mx.append(float(r[2]))
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if sm:
            out["sm_mhz"] = statistics.median(sm)
            out["sm_max_mhz"] = max(mx)
            out["samples"] = len(sm)
        out["reasons"] = sorted(reasons)
        try:
            os.unlink(self.path)
        except Exception:
            pass
        return out


def dist_setup():
    from paper_2609_12262_gb300.replicas import world
    return world()


def cpu_oracle_rate(graphs, gid, offs, syn, seconds, workers=None):
    """Decode a bounded sample with the CPU oracle on all host cores."""
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from oracle_pool import OraclePool
    ncores = workers or (os.cpu_count() or 1)
    pool = OraclePool(graphs, ncores)
    rng = np.random.default_rng(5)
    order = rng.permutation(gid.shape[0])
    done, t_used, n = 0, 0.0, 8 * ncores
    res = []
    while t_used < seconds and done < order.size:
        sel = order[done:done + n]
        rows = [syn[offs[s]:offs[s] + graphs[gid[s]].words] for s in sel]
        t0 = time.perf_counter()
        w, o, st = pool.decode(gid[sel], rows, mode="hier")
        t_used += time.perf_counter() - t0
        res.append((sel, w, o, st))
        done += sel.size
        n = min(n * 2, 16384)
    pool.close()
    idx = np.concatenate([r[0] for r in res])
    ref = tuple(np.concatenate([r[i] for r in res]) for i in (1, 2, 3))
    return done / t_used, done, t_used, ncores, (idx, ref)


def parity_vs_oracle(checked, gpu_w, gpu_o, gpu_s):
    """Element-by-element comparison of GPU outputs with the oracle's results
    (idx: shot indices, ref: oracle weight, observable, status)."""
    idx, (rw, ro, rs) = checked
    bad = (gpu_w[idx] != rw) | (gpu_o[idx] != ro) | (gpu_s[idx] != rs)
    return {"checked": int(idx.size), "mismatches": int(np.count_nonzero(bad)),
            "against": "oracle (weight, observable, status per shot)"}


def cpu_model():
    """The host CPU's model name (Linux /proc/cpuinfo, else the platform string)."""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu model", "hardware"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def cpu_oracle_one_core(graphs, gid, offs, syn, seconds):
    """The CPU oracle in this process alone (one core) on a bounded sample."""
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from oracle_pool import oracle_decode
    rng = np.random.default_rng(6)
    order = rng.permutation(gid.shape[0])
    done, t_used, n = 0, 0.0, 16
    while t_used < seconds and done < order.size:
        sel = order[done:done + n]
        rows = [syn[offs[s]:offs[s] + graphs[gid[s]].words] for s in sel]
        t0 = time.perf_counter()
        oracle_decode(graphs, gid[sel], rows, mode="hier", workers=1)
        t_used += time.perf_counter() - t0
        done += sel.size
        n = min(n * 2, 4096)
    return done / t_used, done


def serving_data(q, args, n):
    """n windows of the serving workload: d uniform in {9, 13, 17, 21, 25}, d
    rounds, p, shuffled; graphs resident on the device."""
    sds = [9, 13, 17, 21, 25]
    per_d = (n + len(sds) - 1) // len(sds)
    graphs, gid, offs, syn = mixed_batch(sds, per_d, args.p, seed=args.seed + 77)
    return sds, graphs, [q.Graph.from_phys(g) for g in graphs], gid[:n], offs[:n], syn


def serving_run(q, args, dev, data, rate, seconds, oracle_n=0):
    """Poisson arrivals at `rate` windows/s for `seconds` into a qec_stream;
    latency = result time - scheduled arrival."""
    import torch
    sds, graphs, gg, gid_all, offs_all, syn = data
    N = min(int(rate * seconds), gid_all.shape[0])
    gid, offs = gid_all[:N], offs_all[:N]
    rng = np.random.default_rng(args.seed + 78)
    arr = np.cumsum(rng.exponential(1.0 / rate, size=N))
    st = q.Stream(device_budget_bytes=6 << 30, max_inflight=65536)
    try:
        warm = min(2000, N)
        i = 0
        while i < warm:
            i += st.submit_many(gg, gid[i:warm], offs[i:warm], syn, np.arange(i, warm, dtype=np.uint64) + (1 << 40))
        st.flush()
        st.poll()
        # no garbage-collection pauses in the submit / poll loop
        import gc
        gc.collect()
        gc.disable()
        t0 = time.monotonic_ns() + 2_000_000
        sched = t0 + (arr * 1e9).astype(np.int64)
        ids = np.arange(N, dtype=np.uint64)
        got_w = np.zeros(N, np.int64); got_o = np.zeros(N, np.uint64); got_s = np.full(N, -1, np.int32)
        t_done = np.zeros(N, np.int64); t_sub = np.zeros(N, np.int64)
        i, n_done = 0, 0
        deadline = time.monotonic() + 30 + 4 * seconds
        while n_done < N and time.monotonic() < deadline:
            now = time.monotonic_ns()
            j = int(np.searchsorted(sched, now, side="right"))
            if j > i:
                i += st.submit_many(gg, gid[i:j], offs[i:j], syn, ids[i:j])
            r = st.poll()
            if len(r):
                k = r["request_id"].astype(np.int64)
                got_w[k] = r["weight"]; got_o[k] = r["obs"]; got_s[k] = r["status"]; t_done[k] = r["t_done_ns"]
                t_sub[k] = r["t_submit_ns"]
                n_done += len(r)
    finally:
        import gc
        gc.enable()
        st.close()
    ok = got_s >= 0
    lat_us = (t_done[ok] - sched[ok]) / 1e3
    # where the latency goes: the host loop's delay in submitting a window
    # after its scheduled arrival, and submission to result in the library
    sub_us = (t_sub[ok] - sched[ok]) / 1e3
    svc_us = (t_done[ok] - t_sub[ok]) / 1e3
    span = (t_done[ok].max() - t0) / 1e9 if ok.any() else float("nan")
    # same windows through the batched path: every served result must agree
    t_syn = torch.from_numpy(syn.view(np.int32)).to(dev)
    o, w, s_ = q.decode_batch(gg, t_syn, torch.from_numpy(gid.astype(np.int32)).to(dev),
                              torch.from_numpy(offs.astype(np.int64)).to(dev), num_shots=N)
    torch.cuda.synchronize()
    bw, bo, bs = w.cpu().numpy(), q.to_uint64(o), s_.cpu().numpy()
    mism = int(np.count_nonzero(ok & ((bw != got_w) | (bo != got_o) | (bs != got_s))))
    # served results against the oracle, on a uniform sample of the windows
    oracle_check = None
    if oracle_n > 0 and ok.any():
        sys.path.insert(0, os.path.join(ROOT, "tests"))
        from oracle_pool import OraclePool
        pick = np.random.default_rng(args.seed + 79).choice(np.nonzero(ok)[0], size=min(oracle_n, int(ok.sum())),
                                                            replace=False)
        pool = OraclePool(graphs, os.cpu_count() or 1)
        rows = [syn[offs[k]:offs[k] + graphs[gid[k]].words] for k in pick]
        rw, ro, rs = pool.decode(gid[pick], rows, mode="hier")
        pool.close()
        oracle_check = {"checked": int(pick.size), "mismatches": int(np.count_nonzero(
            (rw != got_w[pick]) | (ro != got_o[pick]) | (rs != got_s[pick]))),
            "sample": "uniformly drawn served windows, compared on weight, observable and status"}
    return {"windows": N, "completed": int(ok.sum()), "offered_rate": rate,
            "sustained": float(ok.sum() / span), "unit": "windows/s",
            "p50_us": float(np.percentile(lat_us, 50)), "p99_us": float(np.percentile(lat_us, 99)),
            "p999_us": float(np.percentile(lat_us, 99.9)), "max_us": float(lat_us.max()),
            "submit_delay_p50_us": float(np.percentile(sub_us, 50)), "submit_delay_p99_us": float(np.percentile(sub_us, 99)),
            "submit_delay_max_us": float(sub_us.max()),
            "library_p50_us": float(np.percentile(svc_us, 50)), "library_p99_us": float(np.percentile(svc_us, 99)),
            "library_max_us": float(svc_us.max()),
            "distances": sds, "p": args.p, "mismatch_vs_batch": mism, "oracle": oracle_check,
            "team_warps": q.get_tuning()["team_warps"] or "auto",
            "latency": "result available on the host minus the scheduled Poisson arrival"}


def serving_all(q, args, dev):
    """The serving record at the offered rate of the workload (with the oracle
    check) and the latency at other offered rates (latency versus load)."""
    rates = sorted(set([args.serve_rate] + [r for r in (50000.0, 100000.0, 400000.0) if args.serve_curve]))
    n = max(int(args.serve_rate * args.serve_seconds), max(int(r * args.serve_curve_seconds) for r in rates))
    data = serving_data(q, args, n)
    main = serving_run(q, args, dev, data, args.serve_rate, args.serve_seconds, args.serve_oracle)
    curve = []
    for r in rates:
        if r == args.serve_rate:
            rec = main
        else:
            rec = serving_run(q, args, dev, data, r, args.serve_curve_seconds)
        curve.append({k: rec[k] for k in ("offered_rate", "sustained", "windows", "p50_us", "p99_us", "p999_us",
                                          "submit_delay_p99_us", "library_p99_us", "mismatch_vs_batch")})
    main["latency_vs_load"] = curve
    return main


def scaling_study(q, args, dev):
    """Large single windows: throughput and single-window latency per (d, p)."""
    import torch
    rows = []
    for d in (25, 31, 41, 51):
        for p in (0.001, 0.003, 0.005):
            pg = rotated_surface_code(d, d, p)
            syn, _ = sample_shots(pg, args.scaling_shots, args.seed + d * 1000 + int(p * 1e4))
            pc = np.unpackbits(syn.view(np.uint8), axis=1).sum(axis=1)
            kmax = int(pc.max())
            g = q.Graph.from_phys(pg)
            q.set_tuning(kcap=max(64, int(kmax * 1.1) + 8), blocks_per_sm=-1, warps_per_block=-1)
            t = torch.from_numpy(syn.view(np.int32).reshape(-1)).to(dev)
            S = syn.shape[0]
            out = (torch.empty(S, dtype=torch.int64, device=dev), torch.empty(S, dtype=torch.int64, device=dev),
                   torch.empty(S, dtype=torch.int32, device=dev))
            q.decode_batch([g], t, num_shots=S, out=out)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            q.decode_batch([g], t, num_shots=S, out=out)
            b.record()
            torch.cuda.synchronize()
            ms = a.elapsed_time(b)
            st = out[2].cpu().numpy()
            # single-window latency: one window per launch, one warp (the plain
            # path) and a 16-warp team (one window alone in a batch)
            nl = min(16, S)
            po = (torch.empty(nl, dtype=torch.int64, device=dev), torch.empty(nl, dtype=torch.int64, device=dev),
                  torch.empty(nl, dtype=torch.int32, device=dev))
            q.decode_plain(g, t, num_shots=nl, out=po)
            torch.cuda.synchronize()
            a.record()
            q.decode_plain(g, t, num_shots=nl, out=po)
            b.record()
            torch.cuda.synchronize()
            warp_lat_ms = a.elapsed_time(b) / nl
            q.set_tuning(team_warps=16)
            tl = []
            for k in range(-1, nl):
                kk = max(k, 0)
                r1 = (po[0][kk:kk + 1], po[1][kk:kk + 1], po[2][kk:kk + 1])
                a.record()
                q.decode_batch([g], t[kk * pg.words:(kk + 1) * pg.words], num_shots=1, out=r1)
                b.record()
                torch.cuda.synchronize()
                if k >= 0:
                    tl.append(a.elapsed_time(b))
            q.set_tuning(team_warps=-1)
            lat_ms = float(np.mean(tl))
            row = {"d": d, "rounds": d, "p": p, "windows": S, "mean_events": float(pc.mean()), "max_events": kmax,
                   "batch_ms": ms, "windows_per_s": S / (ms / 1e3), "us_per_round_throughput": ms * 1e3 / S / d,
                   "window_latency_us": lat_ms * 1e3, "us_per_round_latency": lat_ms * 1e3 / d,
                   "one_warp_latency_us": warp_lat_ms * 1e3, "team_speedup": warp_lat_ms / lat_ms,
                   "nonzero_status": int(np.count_nonzero(st))}
            if args.scaling_save:
                os.makedirs(args.scaling_save, exist_ok=True)
                k = min(64, S)
                np.savez(os.path.join(args.scaling_save, "d%d_p%g.npz" % (d, p)), weight=out[1].cpu().numpy()[:k],
                         obs=q.to_uint64(out[0])[:k], status=st[:k], seed=args.seed + d * 1000 + int(p * 1e4))
            rows.append(row)
            print(json.dumps(row), flush=True)
            del t, out
    q.set_tuning(kcap=-1, blocks_per_sm=-1, warps_per_block=-1)
    return rows


def config_study(q, args, dev):
    """The small and non-uniform configurations: d=5 (5 noisy + 1 perfect round,
    p=0.005, 10,000 shots from seed 0) and d=11 (11 rounds, per-edge p ~
    U[0.002, 0.006], 100,000 shots), each decoded batched (one persistent launch)
    and plain (one launch per shot), with the CPU oracle timed on the host cores
    beside them (the CPU baseline)."""
    import torch
    rows = []
    cases = [("d5_p0.005", rotated_surface_code(5, 5, 0.005), 10000, 0, 10000),
             ("d11_U[0.002,0.006]", rotated_surface_code(11, 11, p_range=(0.002, 0.006), p_seed=1), 100000, 1, 4000)]
    for name, pg, S, seed, n_plain in cases:
        syn, _ = sample_shots(pg, S, seed)
        g = q.Graph.from_phys(pg)
        t = torch.from_numpy(syn.view(np.int32).reshape(-1)).to(dev)
        out = (torch.empty(S, dtype=torch.int64, device=dev), torch.empty(S, dtype=torch.int64, device=dev),
               torch.empty(S, dtype=torch.int32, device=dev))
        for _ in range(3):
            q.decode_batch([g], t, num_shots=S, out=out)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 5
        a.record()
        for _ in range(reps):
            q.decode_batch([g], t, num_shots=S, out=out)
        b.record()
        torch.cuda.synchronize()
        batch_rate = reps * S / (a.elapsed_time(b) / 1e3)
        st = out[2].cpu().numpy()
        po = (torch.empty(n_plain, dtype=torch.int64, device=dev), torch.empty(n_plain, dtype=torch.int64, device=dev),
              torch.empty(n_plain, dtype=torch.int32, device=dev))
        q.decode_plain(g, t, num_shots=min(200, n_plain), out=po)
        torch.cuda.synchronize()
        a.record()
        q.decode_plain(g, t, num_shots=n_plain, out=po)
        b.record()
        torch.cuda.synchronize()
        plain_rate = n_plain / (a.elapsed_time(b) / 1e3)
        plain_same = bool(torch.equal(po[1], out[1][:n_plain]) and torch.equal(po[0], out[0][:n_plain]))
        row = {"config": name, "shots": S, "rounds": pg.rounds, "batched_shots_per_s": batch_rate,
               "batched_us_per_round": 1e6 / batch_rate / pg.rounds, "plain_shots_per_s": plain_rate,
               "plain_shots": n_plain, "plain_us_per_round": 1e6 / plain_rate / pg.rounds,
               "batched_over_plain": batch_rate / plain_rate, "plain_equals_batched": plain_same,
               "nonzero_status": int(np.count_nonzero(st)),
               "alg_bytes_per_shot": 4 * pg.words + 20,
               "hbm_frac": batch_rate * (4 * pg.words + 20) / 1e9 / load_peaks()[0]}
        if not args.no_cpu_baseline:
            gid = np.zeros(S, np.int32)
            offs = np.arange(S, dtype=np.int64) * pg.words
            rate, n, secs, cores, _ = cpu_oracle_rate([pg], gid, offs, syn.reshape(-1), args.cpu_seconds)
            row["cpu_baseline"] = {"value": rate, "unit": "shots/s", "cores": cores, "kind": "oracle",
                                   "sample": "%d shots of this configuration in %.1f s" % (n, secs)}
        rows.append(row)
        print(json.dumps(row), flush=True)
        del t, out, po
    return rows


def stream_study(q, args, dev):
    """Sliding-window decoding of long histories: R = 10 d noisy rounds (+ 1
    perfect), windows of W = 2d layers every C = d layers, p = 0.003, many
    streams per launch.  Reports rounds decoded per second and us per round for
    the batch of streams, the latency per round of one stream decoded window
    after window, and whole-history decoding (one window) of the same streams."""
    import torch
    from paper_2609_12262_gb300.window import SlidingWindow
    rows = []
    for d, S in ((11, 20000), (15, 8000), (21, 3000)):
        R = 10 * d
        pg = rotated_surface_code(d, R, 0.003)
        syn, _ = sample_shots(pg, S, args.seed + d)
        t = torch.from_numpy(syn.view(np.int32).reshape(-1)).to(dev)
        whole = q.Graph.from_phys(pg)
        dec = SlidingWindow(whole, pg.nz, 2 * d, d)
        q.set_tuning(kcap=max(64, int(np.unpackbits(syn.view(np.uint8), axis=1).sum(axis=1).max()) + 8),
                     blocks_per_sm=-1, warps_per_block=-1)
        dec.decode(t, S)
        q.decode_batch([whole], t, num_shots=S)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        obs, st = dec.decode(t, S)
        b.record()
        torch.cuda.synchronize()
        ms_sw = a.elapsed_time(b)
        a.record()
        wo, ww, ws = q.decode_batch([whole], t, num_shots=S)
        b.record()
        torch.cuda.synchronize()
        ms_whole = a.elapsed_time(b)
        one = t[:pg.words * 1].clone()
        dec.decode(one, 1)
        torch.cuda.synchronize()
        a.record()
        obs1, st1 = dec.decode(one, 1)
        b.record()
        torch.cuda.synchronize()
        ms_one = a.elapsed_time(b)
        ref1 = (obs1.clone(), st1.clone())
        # the same single stream replayed from one captured CUDA graph
        cg, go1, gs1 = dec.graph(one, 1)
        cg.replay()
        torch.cuda.synchronize()
        a.record()
        cg.replay()
        b.record()
        torch.cuda.synchronize()
        ms_one_graph = a.elapsed_time(b)
        graph_same = bool(torch.equal(go1, ref1[0]) and torch.equal(gs1, ref1[1]))
        row = {"d": d, "rounds": R, "W": 2 * d, "C": d, "p": 0.003, "streams": S, "windows": len(dec.windows),
               "sliding_rounds_per_s": S * R / (ms_sw / 1e3), "sliding_us_per_round": ms_sw * 1e3 / (S * R),
               "whole_history_rounds_per_s": S * R / (ms_whole / 1e3),
               "one_stream_us_per_round": ms_one * 1e3 / R,
               "one_stream_graph_us_per_round": ms_one_graph * 1e3 / R, "graph_same_result": graph_same,
               "same_observable_as_whole": float((obs == wo).double().mean().item()),
               "sliding_nonzero_status": int(torch.count_nonzero(st).item()),
               "whole_nonzero_status": int(torch.count_nonzero(ws).item())}
        rows.append(row)
        print(json.dumps(row), flush=True)
        del t
    q.set_tuning(kcap=-1, blocks_per_sm=-1, warps_per_block=-1)
    return rows


SCHEDULE_CANDIDATES = [
    ("alg3 q=1/10 phi_min=1/100", {}),
    ("alg3 q=1/2 phi_min=1/10", {"q": (1, 2), "phi_min": (1, 10)}),
    ("alg3 q=1/5 phi_min=1/20", {"q": (1, 5), "phi_min": (1, 20)}),
    ("d1 = 2 largest edges", {"d1_edges": 2}),
]
# Larger level-1 buffers (d1 = 3 edges, or b1 = 3 d1) make every level-1
# neighbourhood a search over ~1000 vertices per event: decoding then runs at
# 10^2 - 10^3 shots/s and large shots outgrow the per-shot tables (status
# QEC_SHOT_CAPACITY), so they are left out of the default study.


def schedule_study(q, args, dev):
    """Alternative processing-cluster schedules (Methods, Alg. 3 with other
    (q, phi_min), or a custom level-1 diameter d1 with the level-1 conditions
    kept): parallel event count per round, events resolved at level 1, batched
    throughput, and hierarchical == global on every shot (Theorem 1)."""
    import torch
    rows = []
    for d, p in ((13, 0.001), (21, 0.001), (13, 0.003)):
        pg = rotated_surface_code(d, d, p)
        syn, _ = sample_shots(pg, args.study_shots, args.seed + 31 * d)
        pc = np.unpackbits(syn.view(np.uint8), axis=1).sum(axis=1)
        q.set_tuning(kcap=max(64, int(pc.max() * 1.1) + 8), blocks_per_sm=-1, warps_per_block=-1)
        t = torch.from_numpy(syn.view(np.int32).reshape(-1)).to(dev)
        S = syn.shape[0]
        for name, spec in SCHEDULE_CANDIDATES:
            wi = 2 * int(pg.w.max())
            d1 = spec["d1_edges"] * wi + 1 if "d1_edges" in spec else 0
            b1 = spec["b1_factor"] * d1 if "b1_factor" in spec else 0
            g = q.Graph.from_phys(pg, q=spec.get("q"), phi_min=spec.get("phi_min"), d1=d1, b1=b1)
            o, w, st, dg = q.decode_batch_ex([g], t, mode="hier")
            go, gw, gs, _ = q.decode_batch_ex([g], t, mode="global", diag=False)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(3):
                q.decode_batch([g], t, num_shots=S)
            b.record()
            torch.cuda.synchronize()
            dg = dg.cpu().numpy()
            row = {"d": d, "p": p, "schedule": name, "d1": int(g.info.d_k[0]), "b1": int(g.info.b_k[0]),
                   "e_ideal_per_round": float(dg[:, 0].mean() / d),
                   "level1_fraction": float(dg[:, 4].sum() / max(1, dg[:, 7].sum())),
                   "shots_per_s": 3 * S / (a.elapsed_time(b) / 1e3),
                   "hier_vs_global_mismatch": int((~(torch.eq(o, go) & torch.eq(w, gw) & torch.eq(st, gs))).sum().item()),
                   "nonzero_status": int(torch.count_nonzero(st).item())}
            rows.append(row)
            print(json.dumps(row), flush=True)
        del t
    q.set_tuning(kcap=-1, blocks_per_sm=-1, warps_per_block=-1)
    return rows


def event_study(q, args, dev):
    """Parallel event count per round (Methods, "Numerical evaluation"): E_ideal of
    the hierarchical execution and the event count of global sparse blossom, both
    from the GPU's per-shot diagnostics, for d = 9, 13, ..., 49 (d rounds) and
    p in {1e-3, 1e-4, 1e-5}.  Hierarchical and global results must agree
    (Theorem 1).  --study-save keeps the first 64 shots' outputs of every point
    for an offline comparison."""
    import torch
    rows = []
    for p in (0.001, 0.0001, 0.00001):
        if args.study_p and p not in args.study_p:
            continue
        for d in range(9, 50, 4):
            if args.study_d and d not in args.study_d:
                continue
            if args.noise == "phenomenological":
                pg = rotated_surface_code(d, d, p)
            else:
                pg = rotated_surface_code_circuit(d, d, p, "physical" if args.noise == "circuit-physical" else "uniform")
            seed = args.seed + 7 * d + int(round(-np.log10(p)))
            syn, _ = sample_shots(pg, args.study_shots, seed)
            pc = np.unpackbits(syn.view(np.uint8), axis=1).sum(axis=1)
            g = q.Graph.from_phys(pg)
            q.set_tuning(kcap=max(64, int(pc.max() * 1.1) + 8), blocks_per_sm=-1, warps_per_block=-1)
            t = torch.from_numpy(syn.view(np.int32).reshape(-1)).to(dev)
            res = {}
            for mode in ("hier", "global"):
                if mode == "global" and pc.mean() > 500:
                    # every region explores from t = 0: tables twice as large, and
                    # launches of 256 shots so that each ends well inside the watchdog
                    q.set_tuning(kcap=2 * max(64, int(pc.max() * 1.1) + 8), warps_per_block=1, blocks_per_sm=2)
                    parts = []
                    for c0 in range(0, syn.shape[0], 256):
                        n = min(256, syn.shape[0] - c0)
                        sub = t[c0 * pg.words:(c0 + n) * pg.words]
                        parts.append(q.decode_batch_ex([g], sub, num_shots=n, mode=mode))
                    torch.cuda.synchronize()
                    o, w, st, dg = (torch.cat([x[i] for x in parts]) for i in range(4))
                    q.set_tuning(kcap=max(64, int(pc.max() * 1.1) + 8), warps_per_block=-1, blocks_per_sm=-1)
                else:
                    o, w, st, dg = q.decode_batch_ex([g], t, mode=mode)
                torch.cuda.synchronize()
                res[mode] = (w.cpu().numpy(), q.to_uint64(o), st.cpu().numpy(), dg.cpu().numpy())
            hw, ho, hs, hd = res["hier"]
            gw, go, gs, gd = res["global"]
            R = float(d)
            row = {"d": d, "rounds": d, "p": p, "noise": args.noise, "edges": int(pg.num_edges),
                   "shots": int(syn.shape[0]), "mean_defects": float(pc.mean()),
                   "e_ideal_per_round": float(hd[:, 0].mean() / R), "e_global_per_round": float(gd[:, 0].mean() / R),
                   "e_hier_total_per_round": float(hd[:, 2].mean() / R),
                   "max_e_ideal": int(hd[:, 0].max()), "max_e_global": int(gd[:, 0].max()),
                   "t_ideal_mean": float(hd[:, 1].mean()), "t_global_mean": float(gd[:, 1].mean()),
                   "level1_fraction": float(hd[:, 4].sum() / max(1, hd[:, 7].sum())),
                   "hier_vs_global_mismatch": int(np.count_nonzero((hw != gw) | (ho != go) | (hs != gs))),
                   "nonzero_status": int(np.count_nonzero(hs) + np.count_nonzero(gs))}
            if args.study_save:
                os.makedirs(args.study_save, exist_ok=True)
                k = min(64, syn.shape[0])
                np.savez(os.path.join(args.study_save, "d%d_p%g.npz" % (d, p)), seed=seed,
                         **{"%s_%s" % (m, f): v[:k] for m, r in res.items()
                            for f, v in zip(("weight", "obs", "status", "diag"), r)})
            rows.append(row)
            print(json.dumps(row), flush=True)
            del t
    q.set_tuning(kcap=-1, blocks_per_sm=-1, warps_per_block=-1)
    return rows


def configs_line(q, args, dev):
    """The small and non-uniform configurations in the bench line: d = 5 (p =
    0.005, 10,000 shots from seed 0) and d = 11 (per-edge p ~ U[0.002, 0.006],
    100,000 shots), batched (one persistent launch) and plain (one launch per
    shot), in shots/s and us per round; the plain and batched outputs agree."""
    import torch
    out = {}
    cases = [("d5_p0.005", rotated_surface_code(5, 5, 0.005), 10000, 0, 10000),
             ("d11_U[0.002,0.006]", rotated_surface_code(11, 11, p_range=(0.002, 0.006), p_seed=1), 100000, 1, 4000)]
    for name, pg, S, seed, n_plain in cases:
        syn, _ = sample_shots(pg, S, seed)
        g = q.Graph.from_phys(pg)
        t = torch.from_numpy(syn.view(np.int32).reshape(-1)).to(dev)
        res = (torch.empty(S, dtype=torch.int64, device=dev), torch.empty(S, dtype=torch.int64, device=dev),
               torch.empty(S, dtype=torch.int32, device=dev))
        for _ in range(3):
            q.decode_batch([g], t, num_shots=S, out=res)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 5
        a.record()
        for _ in range(reps):
            q.decode_batch([g], t, num_shots=S, out=res)
        b.record()
        torch.cuda.synchronize()
        batch_rate = reps * S / (a.elapsed_time(b) / 1e3)
        po = (torch.empty(n_plain, dtype=torch.int64, device=dev), torch.empty(n_plain, dtype=torch.int64, device=dev),
              torch.empty(n_plain, dtype=torch.int32, device=dev))
        q.decode_plain(g, t, num_shots=min(200, n_plain), out=po)
        torch.cuda.synchronize()
        a.record()
        q.decode_plain(g, t, num_shots=n_plain, out=po)
        b.record()
        torch.cuda.synchronize()
        plain_rate = n_plain / (a.elapsed_time(b) / 1e3)
        out[name] = {"shots": S, "rounds": pg.rounds, "batched_shots_per_s": batch_rate,
                     "batched_us_per_round": 1e6 / batch_rate / pg.rounds, "plain_shots_per_s": plain_rate,
                     "plain_shots": n_plain, "plain_us_per_round": 1e6 / plain_rate / pg.rounds,
                     "batched_over_plain": batch_rate / plain_rate,
                     "plain_equals_batched": bool(torch.equal(po[1], res[1][:n_plain]) and
                                                  torch.equal(po[0], res[0][:n_plain])),
                     "nonzero_status": int(torch.count_nonzero(res[2]).item())}
        del t, res, po
    return out


def graph_cycles(q, args, dev, n=1000, cycles=300):
    """A real-time decoding loop on small batches (one QEC cycle = copy n
    syndromes of the d = 11 non-uniform graph from pinned host memory, decode,
    copy the results back, wait for them), issued call by call and replayed as
    one captured CUDA graph; wall-clock time per cycle and whether both give
    the same results."""
    import torch
    pg = rotated_surface_code(11, 11, p_range=(0.002, 0.006), p_seed=1)
    syn, _ = sample_shots(pg, n, args.seed + 11)
    g = q.Graph.from_phys(pg)
    h_syn = torch.from_numpy(syn.view(np.int32).reshape(-1)).pin_memory()
    d_syn = torch.empty_like(h_syn, device=dev)
    out = (torch.empty(n, dtype=torch.int64, device=dev), torch.empty(n, dtype=torch.int64, device=dev),
           torch.empty(n, dtype=torch.int32, device=dev))
    h_out = [torch.empty(n, dtype=x.dtype).pin_memory() for x in out]

    def cycle():
        d_syn.copy_(h_syn, non_blocking=True)
        q.decode_batch([g], d_syn, num_shots=n, out=out)
        for h, d_ in zip(h_out, out):
            h.copy_(d_, non_blocking=True)

    res = {}
    for name in ("launches", "graph"):
        if name == "graph":
            cg = torch.cuda.CUDAGraph()
            with torch.cuda.graph(cg):
                cycle()
            run = cg.replay
        else:
            run = cycle
        for _ in range(5):
            run()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(cycles):
            run()
            torch.cuda.current_stream().synchronize()
        res[name] = (time.perf_counter() - t0) / cycles * 1e6
        res[name + "_out"] = [h.clone() for h in h_out]
    same = all(torch.equal(a, b) for a, b in zip(res["launches_out"], res["graph_out"]))
    return {"shots_per_cycle": n, "graph": "d11 per-edge p ~ U[0.002, 0.006]", "cycles": cycles,
            "launch_cycle_us": res["launches"], "graph_cycle_us": res["graph"], "same_results": bool(same),
            "cycle": "H2D syndromes + decode + D2H results + host wait, wall clock"}


def scaling_line(q, args, dev):
    """Per-round decode time versus d at p = 0.003 for single large windows (d
    rounds): batched throughput over many windows (one warp per window) and the
    latency of one window decoded alone (a 16-warp team per window, and one
    warp for comparison); the single windows are checked against the oracle."""
    import torch
    from paper_2609_12262_gb300 import autotune
    out = {}
    checks = []
    # split threshold of the 16-warp teams (windows with fewer detection events
    # go to one warp), tuned on two windows of each distance at p = 0.001 and
    # 0.003 (other seeds than the measured windows)
    samples = []
    for d in (25, 31, 41, 51):
        for p in (0.001, 0.003):
            pg = rotated_surface_code(d, d, p)
            sy, _ = sample_shots(pg, 2, args.seed + 700 + d + int(p * 1e4))
            samples.append((q.Graph.from_phys(pg), torch.from_numpy(sy.view(np.int32).reshape(-1)).to(dev)))
    split, split_totals = autotune.tune_split(samples, reps=1)
    out["team_split_events"] = {"chosen": split, "total_ms": {str(sp): ms for ms, sp in split_totals}}
    for d, n in ((25, 4000), (31, 3000), (41, 2000), (51, 1200)):
        pg = rotated_surface_code(d, d, 0.003)
        syn, _ = sample_shots(pg, n, args.seed + 500 + d)
        K = np.unpackbits(syn.view(np.uint8), axis=1).sum(axis=1)
        g = q.Graph.from_phys(pg)
        t = torch.from_numpy(syn.view(np.int32).reshape(-1)).to(dev)
        q.set_tuning(kcap=max(64, int(K.max() * 1.1) + 8), team_warps=-1)
        res = (torch.empty(n, dtype=torch.int64, device=dev), torch.empty(n, dtype=torch.int64, device=dev),
               torch.empty(n, dtype=torch.int32, device=dev))
        q.decode_batch([g], t, num_shots=n, out=res)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        q.decode_batch([g], t, num_shots=n, out=res)
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        # the team size chosen by the autotuner for this batch (results equal
        # across candidates), against the automatic rule above
        tuned_team, team_ms = autotune.tune_team([g], t, num_shots=n, reps=1)
        ref_auto = tuple(x.cpu() for x in res)
        q.decode_batch([g], t, num_shots=n, out=res)
        torch.cuda.synchronize()
        assert all(torch.equal(x, y.cpu()) for x, y in zip(ref_auto, res))
        tuned_ms = min(m for m, tm in team_ms if tm == tuned_team)
        q.set_tuning(team_warps=-1)
        lat = {}
        one = []
        for team in (16, 1):
            q.set_tuning(team_warps=team, team_split_events=split)
            times = []
            for s in range(-1, 6):
                k = max(s, 0)
                r1 = (res[0][k:k + 1].clone(), res[1][k:k + 1].clone(), res[2][k:k + 1].clone())
                a.record()
                q.decode_batch([g], t[k * pg.words:(k + 1) * pg.words], num_shots=1, out=r1)
                b.record()
                torch.cuda.synchronize()
                if s >= 0:
                    times.append(a.elapsed_time(b))
                    if team == 16:
                        one.append((int(r1[1].item()), int(r1[0].item()) & ((1 << 64) - 1), int(r1[2].item())))
            lat[team] = float(np.mean(times))
        out["d%d" % d] = {"d": d, "rounds": d, "p": 0.003, "windows": n, "mean_events": float(K.mean()),
                          "batched_windows_per_s": n / (ms / 1e3), "batched_us_per_round": ms * 1e3 / n / d,
                          "batched_team_warps": "automatic",
                          "tuned_team_warps": tuned_team, "tuned_windows_per_s": n / (tuned_ms / 1e3),
                          "tuned_us_per_round": tuned_ms * 1e3 / n / d,
                          "team_ms": {str(tm): m for m, tm in team_ms},
                          "latency_us": lat[16] * 1e3, "latency_us_per_round": lat[16] * 1e3 / d,
                          "latency_team_warps": 16, "one_warp_latency_us": lat[1] * 1e3,
                          "team_speedup": lat[1] / lat[16],
                          "nonzero_status": int(torch.count_nonzero(res[2]).item())}
        checks.append((pg, syn[:2], one[:2]))
        del t, res
    q.set_tuning(kcap=-1, team_warps=-1)
    # the first two single windows of every distance against the oracle
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from oracle_pool import oracle_decode
    phys = [c[0] for c in checks]
    gid = np.repeat(np.arange(len(checks), dtype=np.int32), 2)
    rows = [r for c in checks for r in c[1]]
    rw, ro, rs = oracle_decode(phys, gid, rows, chunk=1, workers=min(len(rows), os.cpu_count() or 1))
    got = [x for c in checks for x in c[2]]
    bad = sum(1 for i, (w, o, st) in enumerate(got) if (w, o, st) != (int(rw[i]), int(ro[i]), int(rs[i])))
    out["parity"] = {"checked": len(got), "mismatches": bad, "against": "oracle, the single windows"}
    return out


def reference_arm(args, ws, rank):
    if ws > 1 and rank != 0:
        return
    shots_per_d = max(1, min(args.shots_per_d, 400))
    graphs, gid, offs, syn = mixed_batch(DS, shots_per_d, args.p, seed=args.seed)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from oracle_pool import OraclePool
    ncores = os.cpu_count() or 1
    per_step = max(ncores * 32, 256)
    pool = OraclePool(graphs, ncores)
    rng = np.random.default_rng(9)
    times = []
    for it in range(args.warmup + args.steps):
        sel = rng.choice(gid.shape[0], size=min(per_step, gid.shape[0]), replace=False)
        rows = [syn[offs[s]:offs[s] + graphs[gid[s]].words] for s in sel]
        t0 = time.perf_counter()
        pool.decode(gid[sel], rows, mode="hier")
        dt = time.perf_counter() - t0
        if it >= args.warmup:
            times.append(dt)
    pool.close()
    t = sum(times)
    value = args.steps * per_step / t
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic (seeded phenomenological surface-code syndromes)",
        "config": {"workload": "mixed d in {7..21}, d rounds, p=%g; oracle on a %d-shot sample per step"
                   % (args.p, per_step), "shots_per_step": per_step},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": ncores, "kind": "oracle",
                         "sample": "%d uniformly drawn shots of the mixed batch per step" % per_step},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    ws, rank, local = dist_setup()
    if args.quick:
        args.shots_per_d = min(args.shots_per_d, 2500)
        args.plain_shots = min(args.plain_shots, 200)
        args.no_cpu_baseline = True
        args.serve_seconds = 0
        args.extra_configs = 0
    if args.impl == "reference":
        return reference_arm(args, ws, rank)
    import torch
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2609_12262_gb300 import build as qbuild
    qbuild.build()
    import paper_2609_12262_gb300 as q
    if args.kcap:
        q.set_tuning(kcap=args.kcap)
    if args.scaling:
        scaling_study(q, args, torch.device("cuda", local))
        return
    if args.event_study:
        event_study(q, args, torch.device("cuda", local))
        return
    if args.configs:
        config_study(q, args, torch.device("cuda", local))
        return
    if args.schedule_study:
        schedule_study(q, args, torch.device("cuda", local))
        return
    if args.stream_study:
        stream_study(q, args, torch.device("cuda", local))
        return

    graphs, gid, offs, syn = workload(args, rank)
    S = int(gid.shape[0])
    qgraphs = [q.Graph.from_phys(g) for g in graphs]
    dev = torch.device("cuda", local)
    t_syn = torch.from_numpy(syn.view(np.int32)).to(dev)
    t_gid = torch.from_numpy(gid.astype(np.int32)).to(dev)
    t_off = torch.from_numpy(offs.astype(np.int64)).to(dev)
    out = (torch.empty(S, dtype=torch.int64, device=dev), torch.empty(S, dtype=torch.int64, device=dev),
           torch.empty(S, dtype=torch.int32, device=dev))
    stream = torch.cuda.current_stream()

    tuned = None
    if not args.no_autotune and not args.kcap:
        from paper_2609_12262_gb300 import autotune
        n_tune = min(S, 160000)
        tuned, _ = autotune.tune(qgraphs, t_syn, t_gid[:n_tune], t_off[:n_tune], budget_s=40.0)
        autotune.apply(tuned)

    def step():
        q.decode_batch(qgraphs, t_syn, t_gid, t_off, num_shots=S, out=out, stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    st = out[2].cpu().numpy()
    bad_status = int(np.count_nonzero(st != 0))
    out[0].zero_(); out[1].zero_(); out[2].fill_(-1)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    with Clocks(local) as clk:
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_start.record(stream)
        for i in range(args.steps):
            ev[i][0].record(stream)
            step()
            ev[i][1].record(stream)
        t_end.record(stream)
        barrier()
    total_ms = t_start.elapsed_time(t_end)
    launch_ms = [a.elapsed_time(b) for a, b in ev]
    # outputs of the last timed step (compared with the oracle's below)
    timed_out = (out[1].cpu().numpy(), q.to_uint64(out[0]), out[2].cpu().numpy())
    if dist is not None:
        from paper_2609_12262_gb300.replicas import max_over_ranks
        total_ms = max_over_ranks(total_ms, dev)
    clocks = clk.summary()
    ms_step = total_ms / args.steps
    value = ws * S / (ms_step / 1000.0)
    words = np.array([g.words for g in graphs], np.int64)[gid]
    alg_bytes = int(4 * words.sum() + S * (4 + 8) + S * (8 + 8 + 4))
    peak, peak_kind = load_peaks()
    achieved = alg_bytes / (statistics.mean(launch_ms) / 1000.0) / 1e9
    traffic, traffic_note = measured_traffic(S)
    mean_d = float(np.mean(np.array(DS)[gid]))

    # plain one-shot-per-launch path on a subsample
    plain = None
    if args.plain_shots > 0:
        rng = np.random.default_rng(3)
        per_d = max(1, args.plain_shots // len(DS))
        tot_ms, tot_n = 0.0, 0
        for gi, g in enumerate(graphs):
            sel = np.nonzero(gid == gi)[0][:per_d]
            rows = np.stack([syn[offs[s]:offs[s] + g.words] for s in sel])
            ts = torch.from_numpy(rows.view(np.int32).reshape(-1)).to(dev)
            po = (torch.empty(sel.size, dtype=torch.int64, device=dev), torch.empty(sel.size, dtype=torch.int64, device=dev),
                  torch.empty(sel.size, dtype=torch.int32, device=dev))
            q.decode_plain(qgraphs[gi], ts, num_shots=sel.size, out=po)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            q.decode_plain(qgraphs[gi], ts, num_shots=sel.size, out=po, stream=stream)
            b.record(stream)
            torch.cuda.synchronize()
            tot_ms += a.elapsed_time(b)
            tot_n += sel.size
        plain = tot_n / (tot_ms / 1000.0)

    # end to end through the public API with pinned host buffers
    e2e = None
    if not args.no_e2e:
        h_syn = torch.from_numpy(syn.view(np.int32)).pin_memory()
        h_gid = torch.from_numpy(gid.astype(np.int32)).pin_memory()
        h_off = torch.from_numpy(offs.astype(np.int64)).pin_memory()
        h_out = [torch.empty(S, dtype=torch.int64).pin_memory(), torch.empty(S, dtype=torch.int64).pin_memory(),
                 torch.empty(S, dtype=torch.int32).pin_memory()]

        def e2e_step():
            t_syn.copy_(h_syn, non_blocking=True)
            t_gid.copy_(h_gid, non_blocking=True)
            t_off.copy_(h_off, non_blocking=True)
            q.decode_batch(qgraphs, t_syn, t_gid, t_off, num_shots=S, out=out, stream=stream)
            for h, d_ in zip(h_out, out):
                h.copy_(d_, non_blocking=True)

        e2e_step()
        barrier()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(args.steps):
            e2e_step()
        b.record(stream)
        barrier()
        e_ms = a.elapsed_time(b) / args.steps
        if dist is not None:
            from paper_2609_12262_gb300.replicas import max_over_ranks
            e_ms = max_over_ranks(e_ms, dev)
        h2d = int(h_syn.numel() * 4 + h_gid.numel() * 4 + h_off.numel() * 8)
        d2h = int(S * (8 + 8 + 4))
        e2e = {"value": ws * S / (e_ms / 1000.0), "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h}

    serving = None
    if args.serve_seconds > 0 and rank == 0:
        serving = serving_all(q, args, dev)

    configs = scaling = graphs_rec = None
    if rank == 0 and ws == 1 and args.extra_configs:
        configs = configs_line(q, args, dev)
        graphs_rec = graph_cycles(q, args, dev)
        scaling = scaling_line(q, args, dev)

    cpu = None
    parity = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        rate, n, secs, cores, checked = cpu_oracle_rate(graphs, gid, offs, syn, args.cpu_seconds)
        rate1, n1 = cpu_oracle_one_core(graphs, gid, offs, syn, min(4.0, args.cpu_seconds / 3))
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "%d uniformly drawn shots of the same batch, %.1f s wall on %d processes" % (n, secs, cores),
               "cpu_model": cpu_model(), "one_core": {"value": rate1, "unit": UNIT, "sample": "%d shots" % n1}}
        parity = parity_vs_oracle(checked, timed_out[0], timed_out[1], timed_out[2])

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32",
            "data": "synthetic (seeded phenomenological rotated-surface-code syndromes)",
            "config": {"workload": "batched decode, %d shots: d in {7,...,21} x %d shots, d rounds, p=%g, "
                       "one persistent launch" % (S, args.shots_per_d, args.p),
                       "shots": S, "p": args.p, "distances": DS, "parallelism": "replicas" if ws > 1 else "1 GPU",
                       "l2": ("inputs (%.0f MB of syndromes) larger than the 129 MB L2; no flush" % (4 * words.sum() / 1e6))
                       if 4 * words.sum() > 129e6 else "inputs smaller than L2 (profiling size)"},
            "us_per_round": 1e6 / value * ws / mean_d,
            "plain_gpu": {"value": plain, "unit": UNIT, "shots": args.plain_shots,
                          "speedup_batched": (value / ws / plain) if plain else None},
            "nonzero_status_shots": bad_status,
            "tuning": q.get_tuning(),
            "autotuned": {k: tuned[k] for k in ("candidates", "ms", "shots")} if tuned else None,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "peak_source": peak_kind,
                         "note": "algorithmic bytes: syndrome rows + shot metadata + outputs per launch; "
                                 "traffic: " + traffic_note},
            "roofline_alu": alu_roofline(S, statistics.mean(launch_ms) / 1000.0),
            "clocks": clocks,
            # per step: graph sort (count, scan, scatter) for a mixed batch, main pass, overflow pass
            "gpu_launches": (5 if len(graphs) > 1 else 2) * args.steps,
            "e2e": e2e,
            "serving": serving,
            "cpu_baseline": cpu,
            "parity": parity,
            "configs": configs,
            "cuda_graph_cycles": graphs_rec,
            "scaling_p003": scaling,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
