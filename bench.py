"""Benchmark: batched BP-SF on the [[144,12,12]] code-capacity workload.

Workload (one step): 4 x 10^6 syndromes of the [[144,12,12]] BB code under
i.i.d. Z errors at p in {0.02, 0.04, 0.06, 0.08} (10^6 per p, fixed seeds),
decoded with normalised min-sum (alpha 0.625, max_iter 100), |Phi| = 6
(63 trials per failed shot, short_iter 20), minimum-weight selection.  All
four batches and all trials run in ONE persistent launch per step.

Prints one JSON line.  ``--impl reference`` times the CPU oracle instead (the
reference arm: a plain C implementation run on the host cores).
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

P_LIST = (0.02, 0.04, 0.06, 0.08)
SHOTS_PER_P = 1_000_000
# ncu, one launch of 4 x 400k shots (each batch in four shards):
# 23.24 MB read + 24.54 MB written.
DRAM_BYTES_PER_SHOT = 47.78e6 / 1_600_000
CODE = "bb144"
N_BITS, M_CHECKS, NNZ = 144, 72, 432
PARAMS = dict(max_iter=100, alpha=0.625, w=6, w_max=0, short_iter=20, select=0)
METRIC = "BP-SF shots/sec and p50/p99 latency, [[144,12,12]], batched/served vs plain, equal LER"
WORKLOAD = ("[[144,12,12]] BB code capacity, p in {0.02,0.04,0.06,0.08}, 10^6 shots per p, "
            "max_iter 100, w 6 (63 trials) x short_iter 20, alpha 0.625, min-weight selection")


def _gen_chunk(args):
    import synth
    seed, shot0, n, p = args
    bits = synth.bernoulli_bits(seed, 0, shot0, n, N_BITS, p)
    pad = np.zeros((n, 160), dtype=np.uint8)
    pad[:, :N_BITS] = bits
    return np.packbits(pad.reshape(n, 20, 8), axis=-1, bitorder="little").reshape(n, 20).view(np.uint32)


def gen_errors(pool, p_idx, shot0, n, chunk=1 << 16):
    import synth
    seed = synth.SEEDS["bb144_cc"][p_idx]
    jobs = [(seed, shot0 + a, min(chunk, n - a), P_LIST[p_idx]) for a in range(0, n, chunk)]
    parts = pool.map(_gen_chunk, jobs) if pool else list(map(_gen_chunk, jobs))
    return np.concatenate(parts, axis=0)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def roofline_peak_edge_updates(sm_count, sm_mhz):
    """Peak edge-updates/s of the SM-bound kernel (shared-memory bound: 16 B per
    edge-update against 128 B/clk/SM; the ALU bound of ~10 lane-ops per
    edge-update against 128 lanes/clk/SM is looser)."""
    smem = sm_count * 128.0 * sm_mhz * 1e6 / 16.0
    alu = sm_count * 128.0 * sm_mhz * 1e6 / 10.0
    return min(smem, alu)


# --------------------------------------------------------------------------
# CPU oracle (the reference arm and the cpu_baseline)
# --------------------------------------------------------------------------

def oracle_sample(n_per_p, shot0=0):
    import oracle
    import synth
    hx, _ = oracle.named_code(CODE)
    oc = oracle.Code(hx)
    threads = oracle.max_threads()
    P = oracle.Params(PARAMS["max_iter"], PARAMS["alpha"], PARAMS["w"], PARAMS["w_max"], PARAMS["short_iter"],
                      PARAMS["select"])
    inputs = []
    for k, p in enumerate(P_LIST):
        e = synth.bernoulli_bits(synth.SEEDS["bb144_cc"][k], 0, shot0, n_per_p, N_BITS, p)
        inputs.append((p, oc.syndrome(e)))
    t0 = time.perf_counter()
    for p, s in inputs:
        oc.bpsf_batch(s, p, P, fp32=True, threads=threads)
    dt = time.perf_counter() - t0
    return dict(value=len(P_LIST) * n_per_p / dt, unit="shots/s", cores=threads, kind="oracle",
                sample="%d shots per p (first shots of each p's stream), FP32 oracle, %d host threads"
                       % (n_per_p, threads), seconds=dt)


def _lat_stats(shot_s):
    ms = np.asarray(shot_s) * 1e3
    return {"mean_ms": float(ms.mean()), "p50_ms": float(np.percentile(ms, 50)), "p99_ms": float(np.percentile(ms, 99))}


def oracle_plan():
    """The CPU-baseline plan: the FP32 oracle, one host thread and all host
    threads, on bounded samples of configs 1-4 (shots/s, and each shot's own
    decode time as mean / p50 / p99).  Runs in the spawned pool process."""
    import oracle
    import synth
    threads = oracle.max_threads()
    out = {"cores_all": threads}

    def case(oc, synd, p, P, n1, nall):
        r = {}
        for label, th, n in (("1_thread", 1, n1), ("all_threads", threads, nall)):
            s = np.ascontiguousarray(synd[:n])
            t = np.zeros(s.shape[0], dtype=np.float64)
            t0 = time.perf_counter()
            oc.bpsf_batch(s, p, P, fp32=True, threads=th, shot_s=t)
            dt = time.perf_counter() - t0
            r[label] = dict(shots=int(s.shape[0]), threads=th, shots_per_s=s.shape[0] / dt, **_lat_stats(t))
        return r

    def op(prm):
        return oracle.Params(prm["max_iter"], prm["alpha"], prm["w"], prm["w_max"], prm["short_iter"], prm["select"])

    # Config 1: [[72,12,6]], p = 0.05, max_iter 50, w 4 x short_iter 10.
    hx, _ = oracle.named_code("bb72")
    oc = oracle.Code(hx)
    e = synth.bernoulli_bits(synth.SEEDS["bb72_cc"], 0, 0, 10000, 72, 0.05)
    out["config1_bb72_p0.05"] = case(oc, oc.syndrome(e), 0.05,
                                     op(dict(max_iter=50, alpha=0.625, w=4, w_max=0, short_iter=10, select=0)),
                                     2000, 10000)
    # Config 2: [[144,12,12]] at the four p (the headline workload's settings).
    hx, _ = oracle.named_code(CODE)
    oc = oracle.Code(hx)
    for k, p in enumerate(P_LIST):
        e = synth.bernoulli_bits(synth.SEEDS["bb144_cc"][k], 0, 0, 8000, N_BITS, p)
        out["config2_bb144_p%g" % p] = case(oc, oc.syndrome(e), p, op(PARAMS), 500, 8000)
    # Config 3: 12-round phenomenological [[144]], p = q = 0.002, 0.004.
    oc = oracle.Code(oracle.phenom_code(hx, 12))
    for k, p in enumerate((0.002, 0.004)):
        e = synth.phenom_error_bits(synth.SEEDS["bb144_phenom"][k], 0, 0, 4000, 144, 72, 12, p, p)
        out["config3_phenom_p%g" % p] = case(oc, oc.syndrome(e), p, op(PHENOM_PARAMS), 300, 4000)
    # Config 4: the five BB codes of the mixed batch at p = 0.05 (config-2 parameters).
    for k, name in enumerate(SERVE_BB):
        hx, _ = oracle.named_code(name)
        oc = oracle.Code(hx)
        e = synth.bernoulli_bits(synth.SEEDS["mixed"][k], 0, 0, 4000, oc.N, 0.05)
        out["config4_%s_p0.05" % name] = case(oc, oc.syndrome(e), 0.05, op(PARAMS), 300, 4000)
    return out


def run_reference(args, rank, world):
    if rank != 0:
        return
    n_per_p = args.ref_shots
    oracle_sample(max(n_per_p // 20, 10))  # warm-up: load and page in the oracle
    times, cb = [], None
    for _ in range(args.steps):
        cb = oracle_sample(n_per_p)
        times.append(cb["seconds"])
    shots = len(P_LIST) * n_per_p
    v = shots * len(times) / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "shots/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample_shots_per_p": n_per_p},
            "cpu_baseline": {"value": v, "unit": "shots/s", "cores": cb["cores"], "kind": "oracle",
                             "sample": cb["sample"]},
            "e2e": {"value": v, "unit": "shots/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------
# GPU arm
# --------------------------------------------------------------------------

def run_gpu(args, rank, world, pool):
    import torch
    from paper_2507_00254_gb300 import build as libbuild
    libbuild.build()
    from paper_2507_00254_gb300 import bpsf as B
    from paper_2507_00254_gb300 import codes, harness, replicas

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    n = args.shots_per_p
    shot0 = replicas.shot_offset(rank, n)  # weak scaling: each replica decodes its own 10^6 shots per p
    c = codes.bb(CODE)
    Pm = B.Params(**PARAMS)
    decs = [B.Decoder(c.ptr, c.idx, c.M, c.N, np.full(c.N, p), Pm) for p in P_LIST]
    stream = torch.cuda.current_stream()
    # Inputs: errors from the seeded generator, syndromes by the library's kernel.
    t_gen = time.perf_counter()
    errs, synds = [], []
    for k in range(len(P_LIST)):
        e_np = gen_errors(pool, k, shot0, n)
        e_d = torch.from_numpy(e_np.view(np.int32)).cuda()
        errs.append(e_d)
        synds.append(decs[k].syndrome(e_d))
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t_gen
    # Launch shape: the autotuner's pick for this code.
    if args.tuning:
        tuned = args.tuning
    else:
        tuned = decs[0].autotune(p_sample=0.06, n_sample=1 << 16) if args.autotune else decs[0].tuning
    for d in decs:
        d.tuning = tuned
    outs = [d.outputs(n) for d in decs]
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.int32, device="cuda")  # 512 MB > L2

    def step():
        B.decode_multi(decs, synds, outs=outs, sync=False)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    for d in decs:
        B.bpsf_sync(d.handle, stream.cuda_stream)
    # Each timed step replays a CUDA graph of the step (per code, the counter and
    # queue resets; then the one persistent launch), captured after the warm-up.
    eager = [{k: v.clone() for k, v in o.items()} for o in outs]
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(torch.cuda.current_device())
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t_wall = time.perf_counter()
    work = []
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        graph.replay()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    if dist:
        dist.barrier()
    for d in decs:
        B.bpsf_sync(d.handle, stream.cuda_stream)
        work.append(d.last_work())
    for o, r in zip(outs, eager):  # the replays reproduce the eager steps' results
        assert all(torch.equal(o[k], r[k]) for k in r)
    del eager
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms = replicas.max_over_ranks(float(np.mean(step_ms)), dist, device="cuda")
    shots_step = n * len(P_LIST)
    value = replicas.job_rate(shots_step, world, ms / 1e3)

    # Roofline of the persistent kernel (the one launch per step).
    edge_updates = sum(w["edge_updates"] for w in work)
    props = torch.cuda.get_device_properties(0)
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    peak = roofline_peak_edge_updates(props.multi_processor_count, sm_max)
    achieved = edge_updates / (ms / 1e3)

    # LER per p (harness, on the device) and the plain per-shot form on a sample.
    hx = codes.bb(CODE, 0).dense()
    hz = codes.bb(CODE, 1).dense()
    lx = harness.x_logicals(hx, hz)
    G = torch.from_numpy(np.vstack([hx, lx]).astype(np.float32)).cuda()

    def unpack_dev(words, nb):
        w = words.view(torch.int32)
        bits = (w.unsqueeze(-1) >> torch.arange(32, device=w.device, dtype=torch.int32)) & 1
        return bits.reshape(w.shape[0], -1)[:, :nb]

    def fails(e_words, corr_words, conv):
        out = torch.zeros(e_words.shape[0], dtype=torch.bool, device="cuda")
        for a in range(0, e_words.shape[0], 1 << 18):
            b = min(e_words.shape[0], a + (1 << 18))
            r = unpack_dev(e_words[a:b] ^ corr_words[a:b], N_BITS).float()
            par = torch.remainder(r @ G.T, 2.0) > 0.5
            out[a:b] = par.any(dim=1) | (conv[a:b] == 0)
        return out

    ler, plain = {}, {}
    n_plain = min(args.plain_shots, n)
    for k, p in enumerate(P_LIST):
        f = fails(errs[k], outs[k]["corr"], outs[k]["conv"])
        L = float(f.float().mean().item())
        ler[str(p)] = {"ler": L, "sigma": (L * (1 - L) / n) ** 0.5,
                       "stage_counts": np.bincount(outs[k]["stage"].cpu().numpy(), minlength=3).tolist()}
        # Plain form on the first n_plain shots: per-shot latency and equality with batched.
        po = decs[k].outputs(n_plain)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        decs[k].decode(synds[k][:n_plain].contiguous(), out=po, plain=True)
        dt = time.perf_counter() - t0
        same = all(bool((po[key] == outs[k][key][:n_plain]).all()) for key in ("corr", "conv", "iters", "stage"))
        plain[str(p)] = {"shots": n_plain, "shots_per_s": n_plain / dt, "identical_to_batched": same}
    # Per-shot latency of the plain form (host syndrome in -> host result out, one
    # single-shot request at a time, timed by the library on the host's monotonic
    # clock), all p pooled, on the first 200 shots of each p.
    h_sy = [synds[k][:200].cpu().numpy().view(np.uint32) for k in range(len(P_LIST))]
    lat = []
    for k in range(len(P_LIST)):
        lk, _ = B.plain_replay([decs[k]], None, [0] * 200, [h_sy[k][i:i + 1] for i in range(200)])
        lat.extend(lk[10:].tolist())
    lat_ms = np.array(lat) * 1e3
    plain_total = sum(v["shots"] for v in plain.values())
    plain_time = sum(v["shots"] / v["shots_per_s"] for v in plain.values())

    # End-to-end: host (pinned) syndromes in, host results out, through the C ABI: one
    # bpsf_decode_multi_host call per step (the step's four batches in one launch, as
    # in the device-timed form), after one untimed call that sizes the staging buffers.
    h_synd = [torch.empty((n, 3), dtype=torch.int32, pin_memory=True) for _ in P_LIST]
    for k in range(len(P_LIST)):
        h_synd[k].copy_(synds[k].cpu())
    h_out = [(torch.empty((n, 5), dtype=torch.int32, pin_memory=True), torch.empty(n, dtype=torch.uint8, pin_memory=True),
              torch.empty(n, dtype=torch.int16, pin_memory=True), torch.empty(n, dtype=torch.uint8, pin_memory=True))
             for _ in P_LIST]
    h_jobs = [B.bpsf_job(decs[k].handle, n, h_synd[k].data_ptr(), 3, h_out[k][0].data_ptr(), 5,
                         h_out[k][1].data_ptr(), h_out[k][2].data_ptr(), h_out[k][3].data_ptr())
              for k in range(len(P_LIST))]
    e2e_steps = args.steps  # the same number of steps as the device-timed value
    B.bpsf_decode_multi_host(h_jobs, stream.cuda_stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        B.bpsf_decode_multi_host(h_jobs, stream.cuda_stream)
    e2e_dt = (time.perf_counter() - t0) / e2e_steps
    for k in range(len(P_LIST)):  # the host results are the device form's
        assert torch.equal(h_out[k][0], outs[k]["corr"].cpu()) and torch.equal(h_out[k][3], outs[k]["stage"].cpu())
    h2d = len(P_LIST) * n * 3 * 4
    d2h = len(P_LIST) * n * (5 * 4 + 1 + 2 + 1)

    extras = {}
    if rank == 0 and not args.no_extras:
        extras["long_runs_same_kernel"] = run_long_runs(B, codes, torch, tuned, peak)
        extras["phenomenological"] = run_phenom(B, codes, torch)
        extras["mixed_one_launch"] = run_mixed(B, codes, torch)
        extras["code_capacity_paper_setting"] = run_families(B, codes, torch, harness)
        extras["sampled_trials_complexity"] = run_sampled(B, codes, torch, harness)
        extras["first_success_early_cancel"] = run_first_success(B, codes, torch)
        extras["layered_schedule_bb288"] = run_layered(B, codes, torch, harness)
        extras["served"] = run_served(B, codes, torch, (1e4, 1e5, 1e6, 3.16e6, 1e7), seconds=args.serve_seconds,
                                      tuning=args.serve_tuning)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = pool.apply(oracle_sample, (args.cpu_shots,)) if pool else oracle_sample(args.cpu_shots)
        cpu.pop("seconds", None)
        if not args.no_extras:
            extras["cpu_baseline_plan"] = pool.apply(oracle_plan) if pool else oracle_plan()

    if rank == 0:
        # DRAM bytes per launch of the persistent kernel: ncu's dram__bytes_read + write of one
        # 1.6M-shot launch of this kernel over the same p mix, scaled by shots (the traffic is
        # the shots' I/O and the failed shots' records).
        traffic = args.traffic_bytes if args.traffic_bytes > 0 else DRAM_BYTES_PER_SHOT * shots_step
        line = {
            "metric": METRIC, "value": value, "unit": "shots/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "shots_per_step": shots_step * world, "form": "batched",
                       "launch": "one CUDA-graph replay per step: one persistent decode_multi launch over the 4 batches",
                       "tuning": list(tuned), "l2": "flushed between steps (512 MB write)",
                       "parallelism": "replicas" if world > 1 else "single"},
            "roofline": {"bound": "smem", "achieved": achieved / 1e9, "peak": peak / 1e9, "unit": "Gedge-updates/s",
                         "frac": achieved / peak, "traffic": traffic, "traffic_unit": "bytes per launch",
                         "note": ("peak = SMs x 128 B/clk shared memory / 16 B per edge-update at the max SM clock "
                                  "(nominal shared-memory bandwidth, no measured figure exists for it); the ncu "
                                  "counters read the kernel as latency-bound (issue and shared-memory wavefronts "
                                  "both near half of peak), not bandwidth-bound")},
            "cpu_baseline": cpu,
            "e2e": {"value": shots_step / e2e_dt, "unit": "shots/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": args.steps,
            "clocks": clk,
            "latency_ms": {"batched_step_p50": float(np.percentile(step_ms, 50)),
                           "batched_step_p99": float(np.percentile(step_ms, 99)),
                           "plain_per_shot_p50": float(np.percentile(lat_ms, 50)),
                           "plain_per_shot_p99": float(np.percentile(lat_ms, 99))},
            "forms": {"batched_shots_per_s": value, "plain_shots_per_s": plain_total / plain_time,
                      "plain": plain},
            "ler": ler,
            "work": {"edge_updates_per_step": edge_updates, "failed_shots_per_step": sum(w["failed_shots"] for w in work),
                     "trial_runs_per_step": sum(w["trial_runs"] for w in work),
                     "slot_occupancy": sum(w["iterations"] for w in work) / max(1, sum(w["slot_capacity"] for w in work))},
            "input_gen_s": t_gen, "wall_timed_s": t_wall,
        }
        line.update(extras)
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()



# --------------------------------------------------------------------------
# Secondary measurements (reported beside the headline line)
# --------------------------------------------------------------------------

SERVE_BB = ("bb72", "bb90", "bb108", "bb144", "bb288")
# Served BB codes run latency-oriented teams (a lone slot's iteration is short).
SERVE_TUNING = (1, 1, 15, 0)
PHENOM_PARAMS = dict(max_iter=200, alpha=0.625, w=5, w_max=0, short_iter=30, select=0)


def _packed_errors_dev(torch, bits, wn):
    n, nb = bits.shape
    pad = np.zeros((n, 32 * wn), dtype=np.uint8)
    pad[:, :nb] = bits
    w = np.packbits(pad.reshape(n, wn * 4, 8), axis=-1, bitorder="little").reshape(n, wn * 4)
    return torch.from_numpy(w.view(np.int32).copy()).cuda()


def run_phenom(B, codes, torch, n=100_000):
    """12-round phenomenological [[144,12,12]] (864 x 2592), p = q in {0.002, 0.004}, batched."""
    import synth
    c = codes.phenom("bb144")
    out = {}
    for k, p in enumerate((0.002, 0.004)):
        d = B.Decoder(c.ptr, c.idx, c.M, c.N, np.full(c.N, p), B.Params(**PHENOM_PARAMS))
        e = synth.phenom_error_bits(synth.SEEDS["bb144_phenom"][k], 0, 0, n, 144, 72, 12, p, p)
        synd = d.syndrome(_packed_errors_dev(torch, e, d.Wn))
        o = d.outputs(n)
        d.decode(synd, out=o)  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        d.decode(synd, out=o)
        dt = time.perf_counter() - t0
        w = d.last_work()
        st = np.bincount(o["stage"].cpu().numpy(), minlength=3).tolist()
        out[str(p)] = {"shots": n, "shots_per_s": n / dt, "ms": dt * 1e3, "edge_updates_per_s": w["edge_updates"] / dt,
                       "stage_counts": st, "tuning": list(d.tuning)}
        d.close()
    return out


# The paper's code-capacity setting (Section V, Fig. capacity, the [[154]] study):
# adaptive damping alpha_t = 1 - 2^-t, weight-1 trial vectors over |Phi| bits,
# 50 iterations per run.
FAMILY_SETTINGS = (("bb72", 4), ("bb144", 7), ("cbb126", 6), ("gb254", 13), ("cbb154", 8))


def run_families(B, codes, torch, harness, n=100_000, p_list=(0.04, 0.06)):
    """Code families under the paper's code-capacity setting, batched: shots/s and LER
    (each code's launch shape autotuned once, on a sample at the larger p)."""
    import synth
    out = {}
    for k, (name, w) in enumerate(FAMILY_SETTINGS):
        c = codes.bb(name)
        hx, hz = c.dense(), codes.bb(name, 1).dense()
        lx = harness.x_logicals(hx, hz)
        res = {"n": c.N, "k": int(lx.shape[0]), "phi": w}
        for j, p in enumerate(p_list):
            d = B.Decoder(c.ptr, c.idx, c.M, c.N, np.full(c.N, p),
                          B.Params(max_iter=50, alpha=0.0, w=w, w_max=1, short_iter=50))
            if j == 0:
                d.autotune(p_sample=p_list[-1], n_sample=1 << 15)  # per code; the cache serves the next p
            e = synth.bernoulli_bits(6100 + k, j, 0, n, c.N, p)
            synd = d.syndrome(_packed_errors_dev(torch, e, d.Wn))
            o = d.outputs(n)
            d.decode(synd, out=o)  # warm-up
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            d.decode(synd, out=o)
            dt = time.perf_counter() - t0
            wk = d.last_work()
            # Shot fails iff not converged, or the residual e xor e_hat has a nonzero
            # syndrome or logical (exact: integer sums < 2^24 in float32).
            G = torch.from_numpy(np.vstack([hx, lx]).astype(np.float32)).cuda()
            corr = torch.from_numpy(harness.unpack_rows(o["corr"].cpu().numpy().view(np.uint32), c.N)).cuda()
            r = (torch.from_numpy(e).cuda() ^ corr).float()
            f = (torch.remainder(r @ G.T, 2.0) > 0.5).any(dim=1) | (o["conv"] == 0)
            L = float(f.float().mean().item())
            res[str(p)] = {"shots_per_s": n / dt, "edge_updates_per_s": wk["edge_updates"] / dt,
                           "ler": L, "sigma": (L * (1 - L) / n) ** 0.5,
                           "stage_counts": np.bincount(o["stage"].cpu().numpy(), minlength=3).tolist(),
                           "tuning": list(d.tuning)}
            d.close()
        out[name] = res
    return out


def run_long_runs(B, codes, torch, tuning, peak, n=100_000):
    """The benchmark's kernel and launch shape on runs that are all max_iter long:
    random syndromes (each bit 1/2, almost never satisfied within 100 iterations),
    no trials, four [[144]] streams at the benchmark's priors in one launch.  Shows
    what the BP iteration loop itself reaches against the same roofline, apart
    from the cost of starting and ending the benchmark's short runs."""
    import synth
    c = codes.bb(CODE)
    P = B.Params(max_iter=100, alpha=0.625, w=0, short_iter=1)
    decs, synds = [], []
    for k, p in enumerate(P_LIST):
        d = B.Decoder(c.ptr, c.idx, c.M, c.N, np.full(c.N, p), P)
        d.tuning = tuning
        s = synth.bernoulli_bits(synth.SEEDS["serve"], 40 + k, 0, n, c.M, 0.5)
        synds.append(_packed_errors_dev(torch, s, d.Ws))
        decs.append(d)
    stream = torch.cuda.current_stream()
    B.decode_multi(decs, synds)  # warm-up
    best = None
    for _ in range(3):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        B.decode_multi(decs, synds, sync=False)
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        best = ms if best is None else min(best, ms)
    for d in decs:
        B.bpsf_sync(d.handle, stream.cuda_stream)
    w = [d.last_work() for d in decs]
    eu = sum(x["edge_updates"] for x in w)
    it = sum(x["iterations"] for x in w)
    achieved = eu / (best / 1e3)
    out = {"shots": n * len(P_LIST), "ms": best, "iterations_per_run": it / (n * len(P_LIST)),
           "edge_updates_per_s": achieved, "roofline_frac": achieved / peak,
           "slot_occupancy": it / max(1, sum(x["slot_capacity"] for x in w)), "tuning": list(tuning)}
    for d in decs:
        d.close()
    return out


def run_single_slot(B, codes, torch, reps=5):
    """One failing [[144]] shot (p = 0.05, w = 0) through the plain form: each
    decode is one launch of one block whose single one-warp team runs the shot's
    100 iterations on one slot, the chain that sets the served and plain forms'
    tail latency.  Device time per decode, CUDA events."""
    import synth
    c = codes.bb(CODE)
    P0 = B.Params(max_iter=100, alpha=0.625, w=0, short_iter=20)
    d = B.Decoder(c.ptr, c.idx, c.M, c.N, np.full(c.N, 0.05), P0)
    d.tuning = (1, 1, 1, 0)
    e = synth.bernoulli_bits(synth.SEEDS["serve"], 4, 0, 4096, c.N, 0.05)
    synd = d.syndrome(_packed_errors_dev(torch, e, d.Wn))
    st = d.decode(synd)["stage"].cpu().numpy()
    fail = np.nonzero(st != 0)[0]
    s = synd[int(fail[0]):int(fail[0]) + 1].clone()
    o = d.outputs(1)
    ms = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        d.decode(s, out=o, plain=True)
        b.record()
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    out = {"iters": int(o["iters"][0]), "converged": int(o["conv"][0]), "ms_per_decode": ms,
           "us_per_iteration_median": float(np.median(ms)) * 1e3 / max(1, int(o["iters"][0]))}
    d.close()
    return out


def run_sampled(B, codes, torch, harness, n=100_000, p=0.003):
    """The paper's complexity study (Section V: |Phi| = 50, n_s trial vectors sampled per
    weight 1..w_max, 100 iterations per BP instance, adaptive damping), on the 12-round
    phenomenological [[144]] model at p = q = 0.003 standing in for the circuit-level model:
    LER against BP iterations per shot counted serially, batched throughput."""
    import synth
    c = codes.phenom("bb144")
    h0x, h0z = codes.bb("bb144", 0).dense(), codes.bb("bb144", 1).dense()
    lx = harness.x_logicals(h0x, h0z)
    G = torch.from_numpy(np.vstack([h0x, lx]).astype(np.float32)).cuda()
    e = synth.phenom_error_bits(synth.SEEDS["bb144_phenom"][0], 7, 0, n, 144, 72, 12, p, p)
    out = {"p": p, "shots": n}
    for label, w_max in (("bp", 0), ("sf_wmax2", 2), ("sf_wmax4", 4), ("sf_wmax6", 6)):
        params = B.Params(max_iter=100, alpha=0.0, w=50 if w_max else 0, w_max=w_max, short_iter=100)
        d = B.Decoder(c.ptr, c.idx, c.M, c.N, np.full(c.N, p), params)
        if w_max:
            d.set_trials(synth.sample_trial_masks(7100 + w_max, 50, w_max, 5))
        synd = d.syndrome(_packed_errors_dev(torch, e, d.Wn))
        o = d.outputs(n)
        d.decode(synd, out=o)  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        d.decode(synd, out=o)
        dt = time.perf_counter() - t0
        wk = d.last_work()
        corr = torch.from_numpy(harness.unpack_rows(o["corr"].cpu().numpy().view(np.uint32), c.N)).cuda()
        r = torch.from_numpy(e).cuda() ^ corr
        folded = r[:, :144].clone()
        for t in range(1, 12):
            folded ^= r[:, t * 144:(t + 1) * 144]
        f = (torch.remainder(folded.float() @ G.T, 2.0) > 0.5).any(dim=1) | (o["conv"] == 0)
        L = float(f.float().mean().item())
        out[label] = {"trials_per_failed_shot": B.bpsf_num_trials(d.handle), "ler": L, "sigma": (L * (1 - L) / n) ** 0.5,
                      "bp_iterations_per_shot": wk["iterations"] / n, "shots_per_s": n / dt,
                      "edge_updates_per_s": wk["edge_updates"] / dt,
                      "stage_counts": np.bincount(o["stage"].cpu().numpy(), minlength=3).tolist()}
        d.close()
    return out


def run_first_success(B, codes, torch, n=200_000, n_plain=300, p=0.07):
    """First-success rule with early cancel vs the minimum-weight rule on [[144]] at p:
    batched throughput and work, and the plain form's per-shot latency on failed shots
    (the paper's latency argument: a shot ends when its deciding trial is settled)."""
    import synth
    c = codes.bb(CODE)
    e = synth.bernoulli_bits(synth.SEEDS["bb144_cc"][3], 9, 0, n, c.N, p)
    out = {"p": p, "shots": n}
    for label, sel in (("min_weight", 0), ("first_success", 1)):
        d = B.Decoder(c.ptr, c.idx, c.M, c.N, np.full(c.N, p),
                      B.Params(max_iter=100, alpha=0.625, w=6, short_iter=20, select=sel))
        synd = d.syndrome(_packed_errors_dev(torch, e, d.Wn))
        o = d.outputs(n)
        d.decode(synd, out=o)  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        d.decode(synd, out=o)
        dt = time.perf_counter() - t0
        wk = d.last_work()
        stage = o["stage"].cpu().numpy()
        failed = np.nonzero(stage != 0)[0][:n_plain]
        lat = []
        for i in failed:
            s1 = synd[int(i):int(i) + 1].contiguous()
            po = d.outputs(1)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            d.decode(s1, out=po, plain=True)
            lat.append(time.perf_counter() - t1)
        lat = np.array(lat) * 1e3
        out[label] = {"shots_per_s": n / dt, "iterations_per_shot": wk["iterations"] / n,
                      "trial_runs": wk["trial_runs"], "trials_cancelled": wk["trials_cancelled"],
                      "stage_counts": np.bincount(stage, minlength=3).tolist(),
                      "plain_failed_shot_ms": {"n": int(lat.size), "p50": float(np.percentile(lat, 50)),
                                               "p99": float(np.percentile(lat, 99))}}
        d.close()
    return out


def run_layered(B, codes, torch, harness, n=100_000, p_list=(0.05, 0.07)):
    """Flooding vs layered schedule on [[288,12,18]] under the paper's code-capacity setting
    for that code (|Phi| = 20, weight-1 trials, 50 iterations per run, adaptive damping):
    shots/s, LER and BP iterations per shot."""
    import synth
    c = codes.bb("bb288")
    hx, hz = c.dense(), codes.bb("bb288", 1).dense()
    lx = harness.x_logicals(hx, hz)
    G = torch.from_numpy(np.vstack([hx, lx]).astype(np.float32)).cuda()
    out = {}
    for j, p in enumerate(p_list):
        e = synth.bernoulli_bits(7500, j, 0, n, c.N, p)
        res = {}
        for label, lay in (("flooding", False), ("layered", True)):
            d = B.Decoder(c.ptr, c.idx, c.M, c.N, np.full(c.N, p),
                          B.Params(max_iter=50, alpha=0.0, w=20, w_max=1, short_iter=50, layered=lay))
            synd = d.syndrome(_packed_errors_dev(torch, e, d.Wn))
            o = d.outputs(n)
            d.decode(synd, out=o)  # warm-up
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            d.decode(synd, out=o)
            dt = time.perf_counter() - t0
            wk = d.last_work()
            corr = torch.from_numpy(harness.unpack_rows(o["corr"].cpu().numpy().view(np.uint32), c.N)).cuda()
            r = (torch.from_numpy(e).cuda() ^ corr).float()
            f = (torch.remainder(r @ G.T, 2.0) > 0.5).any(dim=1) | (o["conv"] == 0)
            L = float(f.float().mean().item())
            res[label] = {"shots_per_s": n / dt, "ler": L, "sigma": (L * (1 - L) / n) ** 0.5,
                          "bp_iterations_per_shot": wk["iterations"] / n,
                          "stage_counts": np.bincount(o["stage"].cpu().numpy(), minlength=3).tolist(),
                          "tuning": list(d.tuning)}
            d.close()
        out[str(p)] = res
    return out


def run_mixed(B, codes, torch):
    """[[72]], [[90]], [[108]], [[144]], [[288]] at p = 0.05, counts U{10^3..10^5}, in ONE launch."""
    import synth
    counts = synth.uniform_ints(synth.SEEDS["mixed_counts"], 0, len(SERVE_BB), 1000, 100000)
    decs, synds = [], []
    for k, name in enumerate(SERVE_BB):
        c = codes.bb(name)
        d = B.Decoder(c.ptr, c.idx, c.M, c.N, np.full(c.N, 0.05), B.Params(**PARAMS))
        e = synth.bernoulli_bits(synth.SEEDS["mixed"][k], 0, 0, int(counts[k]), c.N, 0.05)
        synds.append(d.syndrome(_packed_errors_dev(torch, e, d.Wn)))
        decs.append(d)
    # Each code's launch shape from the autotuner (threads per shot, shots per
    # block, iteration chunk), then all five in one launch with those shapes.
    untuned = [d.tuning for d in decs]
    outs = B.decode_multi(decs, synds)  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    B.decode_multi(decs, synds, outs=outs)
    dt0 = time.perf_counter() - t0
    ref = [{k: v.clone() for k, v in o.items()} for o in outs]
    tuned = [d.autotune(p_sample=0.05, n_sample=1 << 14) for d in decs]
    B.decode_multi(decs, synds, outs=outs)  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    B.decode_multi(decs, synds, outs=outs)
    dt = time.perf_counter() - t0
    same = all(torch.equal(o[k], r[k]) for o, r in zip(outs, ref) for k in r)
    total = int(counts.sum())
    res = {"codes": list(SERVE_BB), "shots": [int(x) for x in counts], "shots_per_s": total / dt, "ms": dt * 1e3,
           "tunings": {n: list(t) for n, t in zip(SERVE_BB, tuned)},
           "default_shapes": {"tunings": {n: list(t) for n, t in zip(SERVE_BB, untuned)}, "shots_per_s": total / dt0},
           "identical_to_default_shapes": same}
    for d in decs:
        d.close()
    return res


def _pct(lat_s):
    ms = np.asarray(lat_s) * 1e3
    return {"p50_ms": float(np.percentile(ms, 50)), "p99_ms": float(np.percentile(ms, 99)),
            "p999_ms": float(np.percentile(ms, 99.9)), "mean_ms": float(ms.mean())}


def run_served(B, codes, torch, loads, seconds=2.0, pool_shots=8192, tuning=None, plain_cap_shots=20000):
    """Poisson request stream over the five BB codes (p = 0.05) and the 12-round
    phenomenological [[144]] model (p = q = 0.003), served by bpsf_serve_* and,
    on the same requests, by the plain per-shot form (bpsf_plain_replay).
    Requests carry b = max(1, load / 10000) shots (at most ~10^4 requests/s);
    both traces are replayed by the library on the host's monotonic clock, and
    latency is scheduled arrival -> results in host memory.  Closed loop: one
    single-shot request in flight at a time, per code and over the whole mix.
    The plain form decodes one shot at a time, so above its own rate its
    open-loop latency grows with the trace; its traces are cut to the first
    plain_cap_shots shots (the span is reported)."""
    import synth
    names = list(SERVE_BB) + ["bb144_phenom12"]
    decs, pools = [], []
    for k, name in enumerate(SERVE_BB):
        c = codes.bb(name)
        d = B.Decoder(c.ptr, c.idx, c.M, c.N, np.full(c.N, 0.05), B.Params(**PARAMS))
        if tuning:
            d.tuning = tuning  # team shape of the served BB codes (latency vs throughput)
        e = synth.bernoulli_bits(synth.SEEDS["serve"], 1 + k, 0, pool_shots, c.N, 0.05)
        pools.append(d.syndrome(_packed_errors_dev(torch, e, d.Wn)).cpu().numpy().view(np.uint32))
        decs.append(d)
    c = codes.phenom("bb144")
    d = B.Decoder(c.ptr, c.idx, c.M, c.N, np.full(c.N, 0.003), B.Params(**PHENOM_PARAMS))
    e = synth.phenom_error_bits(synth.SEEDS["serve"], 9, 0, pool_shots // 4, 144, 72, 12, 0.003, 0.003)
    pools.append(d.syndrome(_packed_errors_dev(torch, e, d.Wn)).cpu().numpy().view(np.uint32))
    decs.append(d)

    # Traces: per load, arrivals, codes and request rows (the same for both forms).
    traces = []
    for li, load in enumerate(loads):
        b = max(1, int(load // 10000))
        rate = load / b
        n_req = max(50, int(rate * seconds))
        arrivals = synth.poisson_arrivals(synth.SEEDS["serve"], 100 + li, n_req, rate)
        which = synth.uniform_choice(synth.SEEDS["serve"], 200 + li, n_req, len(decs))
        reqs = []
        cursor = [0] * len(decs)
        for i in range(n_req):
            k = int(which[i])
            nn = b if k < len(SERVE_BB) else max(1, b // 4)
            pool = pools[k]
            a = cursor[k] % (pool.shape[0] - nn)
            cursor[k] += nn
            reqs.append(pool[a:a + nn])
        traces.append((load, b, arrivals, which, reqs))
    n_cl = 200
    mix_which = synth.uniform_choice(synth.SEEDS["serve"], 300, 600, len(decs))
    mix_reqs = [pools[int(k)][i:i + 1] for i, k in enumerate(mix_which)]

    def per_code(lat_s, which):
        out = {}
        for k in range(len(decs)):
            sel = np.asarray(lat_s)[np.asarray(which) == k]
            if sel.size:
                out[names[k]] = [float(np.percentile(sel * 1e3, 50)), float(np.percentile(sel * 1e3, 99))]
        return out

    # The plain form first (no server holds the SMs meanwhile).
    plain_closed, plain_open = {}, []
    for k in range(len(decs)):
        lat, _ = B.plain_replay(decs, None, [k] * n_cl, [pools[k][i:i + 1] for i in range(n_cl)])
        plain_closed[names[k]] = _pct(lat[20:])
    lat, _ = B.plain_replay(decs, None, mix_which, mix_reqs)
    plain_closed["mix"] = _pct(lat[20:])
    for load, b, arrivals, which, reqs in traces:
        m, shots = 0, 0
        while m < len(reqs) and shots + reqs[m].shape[0] <= plain_cap_shots:
            shots += reqs[m].shape[0]
            m += 1
        lat, span = B.plain_replay(decs, arrivals[:m], which[:m], reqs[:m])
        plain_open.append(dict(offered_shots_per_s=load, shots_per_request=b, requests=m,
                               trace_s=float(arrivals[m - 1]), achieved_shots_per_s=shots / span,
                               per_code_p50_p99_ms=per_code(lat, which[:m]), **_pct(lat)))

    srv = B.Server(decs, max_inflight_shots=1 << 16, idle_exit_us=50000)
    served_closed, served_open = {}, []
    try:
        for k in range(len(decs)):
            lat, _ = srv.replay(None, [k] * n_cl, [pools[k][i:i + 1] for i in range(n_cl)])
            served_closed[names[k]] = _pct(lat[20:])
        lat, _ = srv.replay(None, mix_which, mix_reqs)
        served_closed["mix"] = _pct(lat[20:])
        for load, b, arrivals, which, reqs in traces:
            lat, span = srv.replay(arrivals, which, reqs)
            shots = sum(x.shape[0] for x in reqs)
            served_open.append(dict(offered_shots_per_s=load, shots_per_request=b, requests=len(reqs),
                                    trace_s=float(arrivals[-1]), achieved_shots_per_s=shots / span,
                                    per_code_p50_p99_ms=per_code(lat, which), **_pct(lat)))
    finally:
        srv.stop()
    tunings = {names[k]: list(decs[k].tuning) for k in range(len(decs))}
    for dk in decs:
        dk.close()
    cmp = []
    for so, po in zip(served_open, plain_open):
        cmp.append({"offered_shots_per_s": so["offered_shots_per_s"], "served_p99_ms": so["p99_ms"],
                    "plain_p99_ms": po["p99_ms"], "served_p99_below_plain": so["p99_ms"] < po["p99_ms"]})
    return {"mix": names, "tunings": tunings, "clock": "host steady_clock inside the library (both forms)",
            "loads": served_open, "plain_loads": plain_open, "p99_served_vs_plain": cmp,
            "closed_loop": {"served": served_closed, "plain": plain_closed}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--shots-per-p", type=int, default=SHOTS_PER_P)
    ap.add_argument("--plain-shots", type=int, default=2000)
    ap.add_argument("--cpu-shots", type=int, default=15000)
    ap.add_argument("--ref-shots", type=int, default=3000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--autotune", type=int, default=1)
    ap.add_argument("--tuning", type=lambda x: tuple(int(v) for v in x.split(",")), default=None,
                    help="launch shape W,S,B,blocks_per_sm of the batched workload (skips the autotuner)")
    ap.add_argument("--traffic-bytes", type=float, default=0.0)
    ap.add_argument("--no-extras", action="store_true", help="skip the served / phenomenological / mixed lines")
    ap.add_argument("--serve-seconds", type=float, default=2.0)
    ap.add_argument("--only-served", action="store_true", help="run only the served measurement (diagnostics)")
    ap.add_argument("--only", choices=["phenom", "layered", "mixed", "families", "sampled", "first", "long",
                                       "single"],
                    default=None,
                    help="run only one secondary measurement and print its JSON (diagnostics, profiling)")
    ap.add_argument("--serve-tuning", type=lambda x: tuple(int(v) for v in x.split(",")), default=SERVE_TUNING,
                    help="team shape W,S,B,blocks_per_sm of the served BB codes")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.only:
        import torch
        from paper_2507_00254_gb300 import build as libbuild
        libbuild.build()
        from paper_2507_00254_gb300 import bpsf as B
        from paper_2507_00254_gb300 import codes, harness
        fn = {"phenom": lambda: run_phenom(B, codes, torch), "layered": lambda: run_layered(B, codes, torch, harness),
              "mixed": lambda: run_mixed(B, codes, torch), "families": lambda: run_families(B, codes, torch, harness),
              "sampled": lambda: run_sampled(B, codes, torch, harness),
              "first": lambda: run_first_success(B, codes, torch),
              "single": lambda: run_single_slot(B, codes, torch),
              "long": lambda: run_long_runs(B, codes, torch, args.tuning or (1, 8, 13, 0, 1),
                                            roofline_peak_edge_updates(torch.cuda.get_device_properties(0)
                                                                       .multi_processor_count,
                                                                       float(measured_peaks().get("sm_max_mhz",
                                                                                                  2070.0))))}[args.only]
        print(json.dumps(fn()))
        return
    if args.only_served:
        import torch
        from paper_2507_00254_gb300 import build as libbuild
        libbuild.build()
        from paper_2507_00254_gb300 import bpsf as B
        from paper_2507_00254_gb300 import codes
        print(json.dumps(run_served(B, codes, torch, (1e4, 1e5, 1e6, 3.16e6, 1e7), seconds=args.serve_seconds,
                                    tuning=args.serve_tuning)))
        return
    # Input generation and the oracle baseline use a spawn pool created before CUDA starts.
    ctx = mp.get_context("spawn")
    pool = ctx.Pool(processes=max(1, min(16, os.cpu_count() or 1)))
    try:
        run_gpu(args, rank, world, pool)
    finally:
        pool.close()
        pool.join()


if __name__ == "__main__":
    main()
