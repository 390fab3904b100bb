"""Benchmark of the SymFT per-shot sampling engine on B300.

Default workload: pure-Clifford rotated surface-code memory, d=7 with 7 rounds,
uniform circuit-level depolarizing p=1e-3, 1e7 shots per step (the d=5, 5-round
circuit is measured the same way and reported under "per_circuit").  A step is
one symft_sample call over the whole batch: noise + random bits + bit-packed
sign evaluation + record/detector/observable output, all on the GPU.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  With torchrun (N > 1) every rank samples its
own contiguous shot range (shot_offset), no collective touches the data path;
the step time is the max over ranks and `value` counts all ranks' shots.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SHOTS = 10_000_000
WORKLOADS = {
    "surface_d7_r7": dict(d=7, rounds=7, p=1e-3),
    "surface_d5_r5": dict(d=5, rounds=5, p=1e-3),
}
HEADLINE = "surface_d7_r7"
METRIC = "shots/s per circuit on 1 B300 (FP32-batched vs FP64-plain), % of roofline"
HEADLINE_WORKLOAD = ("pure-Clifford rotated surface-code Z memory d=7, 7 rounds, "
                     "depolarizing p=1e-3, bit-packed sign path")


# DRAM traffic of one sign-kernel launch on the headline workload, from an ncu
# capture of dram__bytes_read.sum + dram__bytes_write.sum.  Valid only for the kernel
# source it was taken on (sign.cu and the headers it includes): reported as
# null once any of them changes.
SIGN_TRAFFIC = {"source_sha256": "58eaad7b1283c5325a8e5c8a64859119bbf9987c5518cc10694186845235a374",
                "bytes_per_launch": 25332480 + 869300224}
SIGN_SOURCES = ("sign.cu", "device.cuh", "plan_dev.hpp")


def sign_source_sha256():
    import hashlib
    h = hashlib.sha256()
    for name in SIGN_SOURCES:
        with open(os.path.join(ROOT, "paper_2607_28600_b300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def _sign_traffic():
    try:
        sha = sign_source_sha256()
    except OSError:
        return None
    return SIGN_TRAFFIC["bytes_per_launch"] if sha == SIGN_TRAFFIC["source_sha256"] else None


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


def all_peaks(S):
    """HBM from MEASURED_PEAKS.json (or the fallback); integer, Philox, FP32 /
    FP64 FMA and shared-memory rates measured now by the library's own
    microbenchmarks on this GPU."""
    hbm, kind = _peaks()
    pk = S.symft_measure_peaks()
    pk.update({"hbm_gbs": hbm, "hbm_kind": kind})
    return pk


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        import tempfile
        self.path = os.path.join(tempfile.gettempdir(), f"symft_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=self.f, stderr=subprocess.DEVNULL)
            # start timing only once the sampler is producing lines
            t0 = time.time()
            while time.time() - t0 < 3.0 and os.path.getsize(self.path) == 0:
                time.sleep(0.02)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": smax, "samples": len(sm), "reasons": sorted(reasons)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


_ORACLE_CIRCUIT = None


def _oracle_worker_init():
    """Each host worker parses the headline circuit once."""
    global _ORACLE_CIRCUIT
    from oracle.circuit import parse
    from paper_2607_28600_b300.workloads import rotated_surface_code_memory
    w = WORKLOADS[HEADLINE]
    _ORACLE_CIRCUIT = parse(rotated_surface_code_memory(w["d"], w["rounds"], w["p"]))


def _oracle_chunk(lo_hi):
    """Sample shots [lo, hi) of the headline circuit with the tableau oracle."""
    from oracle import tableau
    lo, hi = lo_hi
    tableau.sample(_ORACLE_CIRCUIT, 1, range(lo, hi))
    return hi - lo


def _oracle_pool(cores):
    # spawn: this process may already hold a CUDA context
    import multiprocessing as mp
    pool = mp.get_context("spawn").Pool(cores, initializer=_oracle_worker_init)
    pool.map(_oracle_chunk, [(0, 8)] * cores)          # imports and parsing, untimed
    return pool


def _oracle_timed(pool, cores, shot0, budget_s, chunk=256):
    """Shots/s of the oracle on `cores` worker processes for about budget_s."""
    n, lo = 0, shot0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < budget_s:
        tasks = [(lo + i * chunk, lo + (i + 1) * chunk) for i in range(cores)]
        n += sum(pool.map(_oracle_chunk, tasks))
        lo += cores * chunk
    return n, time.perf_counter() - t0


def run_reference(args):
    """The oracle on the host cores (a bounded sample of the headline workload per step)."""
    world, rank, _ = _dist()
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    pool = _oracle_pool(cores)
    try:
        for s in range(args.warmup):
            _oracle_timed(pool, cores, 1 << 30, 0.0)
        times, shots = [], []
        for s in range(args.steps):
            n, dt = _oracle_timed(pool, cores, s << 24, 3.0)
            times.append(dt)
            shots.append(n)
    finally:
        pool.close()
        pool.join()
    per = sum(times) / len(times)
    val = sum(shots) / sum(times)
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": "shots/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": per * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": HEADLINE_WORKLOAD, "shots_per_step": sum(shots) // len(shots),
                   "shots_per_word": 64, "parallelism": "host processes"},
        "cpu_baseline": {"value": val, "unit": "shots/s", "cores": cores, "kind": "oracle",
                         "sample": f"about 3 s per step of {HEADLINE} through the "
                                   f"Aaronson-Gottesman tableau oracle on {cores} host processes"},
        "e2e": {"value": val, "unit": "shots/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def cpu_baseline(budget_s=12.0):
    """The tableau oracle as it stands, one worker process per host core."""
    cores = os.cpu_count() or 1
    pool = _oracle_pool(cores)
    try:
        n, dt = _oracle_timed(pool, cores, 0, budget_s)
    finally:
        pool.close()
        pool.join()
    return {"value": n / dt, "unit": "shots/s", "cores": cores, "kind": "oracle",
            "sample": f"{n} shots of {HEADLINE} (d=7, 7 rounds, p=1e-3) through the "
                      f"Aaronson-Gottesman tableau oracle in {dt:.1f} s on {cores} host processes "
                      f"(one per core, {n / dt / cores:.0f} shots/s each)"}


NEAR_CLIFFORD = {
    # name: (generator, postselect, shots per step)
    "c1_surface_d3_r3_T": ("surface_t", 0, 100_000),
    "c3_cultivation_d3_to_d9": ("cultivation", 1, 10_000_000),
    "c4_distill_15to1_encoded": ("distill_encoded", 1, 10_000_000),
    "c4_distill_15to1_literal": ("distill_literal", 1, 1_000_000),
    # coherent over-rotations R_Z(0.02) on surface codes (k_max 4, 8, 12, 24)
    "coherent_d3_r1": ("coherent_3_1", 1, 10_000_000),
    "coherent_d3_r3": ("coherent_3_3", 1, 1_000_000),
    "coherent_d5_r1": ("coherent_5_1", 1, 100_000),
    "coherent_d5_r5": ("coherent_5_5", 1, 64),
}


def _near_clifford_text(kind):
    from paper_2607_28600_b300.workloads import (cultivation_shaped, distillation_15_to_1,
                                                 rotated_surface_code_memory)
    if kind == "surface_t":
        return rotated_surface_code_memory(3, 3, 1e-3, t_on_data0_after_round=0)
    if kind == "cultivation":
        return cultivation_shaped(1e-3)
    if kind == "distill_encoded":
        return distillation_15_to_1(1e-3, "encoded")
    if kind.startswith("coherent_"):
        from paper_2607_28600_b300.workloads import coherent_surface_code_memory
        _, d, r = kind.split("_")
        return coherent_surface_code_memory(int(d), int(r), 1e-3, 0.02)
    return distillation_15_to_1(1e-3, "literal")


def fp32_accuracy(S, torch, plan, dev, stream, shots=1 << 16, seed=77):
    """GPU FP32 executor against the GPU FP64 executor on the same shots (both
    checked against the oracle by the parity tests): the fraction of shots
    whose outputs differ (an active outcome flipped) and the largest branch-
    probability difference over the shots whose outputs agree."""
    import numpy as np
    info = plan.info
    W = (shots + 63) // 64
    res = {}
    for prec in (S.FP32, S.FP64):
        cols = [torch.zeros((max(1, info[k]), W), dtype=torch.int64, device=dev)
                for k in ("n_records", "n_dets", "n_obs")]
        disc = torch.zeros((W,), dtype=torch.int64, device=dev)
        prob = torch.zeros((max(1, info["n_causal"]), shots), dtype=torch.float64, device=dev)
        S.symft_sample_ex(plan, shots, seed, meas_out=cols[0], det_out=cols[1], obs_out=cols[2],
                          discard_out=disc, precision=prec, prob_out=prob, stream=stream, check=True)
        res[prec] = (torch.cat(cols + [disc.view(1, -1)]), prob)
    torch.cuda.synchronize(dev)
    a, pa = res[S.FP32]
    b, pb = res[S.FP64]
    anyw = torch.bitwise_xor(a, b).cpu().numpy().view(np.uint64)
    anyw = np.bitwise_or.reduce(anyw, axis=0)
    flipped = np.unpackbits(anyw.view(np.uint8), bitorder="little").astype(bool)[:shots]
    err = 0.0
    if info["n_causal"] and (~flipped).any():
        keep = torch.from_numpy(~flipped).to(dev)
        err = float((pa - pb).abs()[:, keep].max().item())
    return {"shots": shots, "flip_rate": float(flipped.mean()),
            "max_prob_err_unflipped": err, "n_active_meas": info["n_causal"]}


def dense_floor(info, peaks, fp64=False):
    """Per-shot time floors of the dense instructions when every shot runs the
    whole stream.  On-chip executors: FP arithmetic (FLOPs counted per
    amplitude: PromoteRot 4, diagonal rotation 6, pair rotation 10, diagonal
    measurement 5, pair measurement 13, at two FLOPs per FMA) and
    shared-memory traffic (each instruction reads and writes its vector);
    vectors beyond shared memory: the HBM bytes of the wide executor's fused
    passes.  Under the product-component executor the work is scaled by the
    amplitudes its program touches over those of the monolithic vector."""
    amp = 16 if fp64 else 8
    executor = info["dense_executor"][1 if fp64 else 0]
    in_hbm = executor == "wide"
    # the product-component executor touches pc_work[0] amplitudes per shot
    # where the monolithic vector touches pc_work[1]
    scale = (info["pc_work"][0] / info["pc_work"][1]
             if executor.startswith("components") and info["pc_work"][1] else 1.0)
    if in_hbm:
        b = info["wide_amp_traffic"][1 if fp64 else 0] * amp
        return {"where": "hbm", "executor": executor, "bytes_per_shot": b,
                "floor_s_per_shot": b / (peaks["hbm_gbs"] * 1e9)}
    fl = info["dense_flops"] * scale
    fma = peaks["fp64_fma_per_s"] if fp64 else peaks["fp32_fma_per_s"]
    t_fp = fl / (2.0 * fma)
    sm = info["dense_amp_traffic"] * amp * scale
    t_sm = sm / peaks["smem_bytes_per_s"]
    return {"where": "on-chip", "executor": executor, "flops_per_shot": fl, "smem_bytes_per_shot": sm,
            "fp_floor_s_per_shot": t_fp, "smem_floor_s_per_shot": t_sm,
            "floor_s_per_shot": max(t_fp, t_sm), "bound": "fp" if t_fp >= t_sm else "smem"}


def _time_call(S, torch, dev, stream, plan, shots, seed0, steps, warmup, **kw):
    info = plan.info
    W = (shots + 63) // 64
    meas = torch.empty((max(1, info["n_records"]), W), dtype=torch.int64, device=dev)
    det = torch.empty((max(1, info["n_dets"]), W), dtype=torch.int64, device=dev)
    obs = torch.empty((max(1, info["n_obs"]), W), dtype=torch.int64, device=dev)
    disc = torch.empty((W,), dtype=torch.int64, device=dev)

    def step(i):
        S.symft_sample_ex(plan, shots, seed0 + i, meas_out=meas, det_out=det, obs_out=obs,
                          discard_out=disc, stream=stream, **kw)
    for i in range(warmup):
        step(i)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(steps):
        step(warmup + i)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / steps
    import numpy as np
    words = disc.cpu().numpy().view(np.uint64)
    return {"shots_per_step": shots, "ms_per_step": ms, "shots_per_s": shots / (ms / 1e3),
            "discard_rate": int(np.bitwise_count(words).sum()) / shots,
            "launches_per_step": S.symft_last_launch_count()}


def measure_near_clifford(S, torch, dev, stream, steps, warmup, peaks, scale=1.0, only=None):
    """Attempted shots/s per near-Clifford config: FP32-batched, FP64-batched
    and the paper's GPU design in FP64 (one CTA per shot, in-kernel sampling
    or the packed-column prepass; the faster of the two is the FP64-plain
    figure, as the paper's backend picks per circuit).  Roofline: the dense
    floor of a full shot against the FP32-batched run without postselection,
    where every shot runs the whole instruction stream."""
    out = {}
    for name, (kind, post, shots0) in NEAR_CLIFFORD.items():
        if only is not None and name != only:
            continue
        text = _near_clifford_text(kind)
        plan = S.symft_compile(text, postselect=post)
        info = plan.info
        entry = {"k_max": info["k_max"], "n_qubits": info["n_qubits"],
                 "dense_instructions": sum(info["n_instr"][k] for k in
                                           ("PromoteRot", "ActiveDiagRot", "ActivePairRot",
                                            "ActiveDiagMeas", "ActivePairMeas")),
                 "postselect": bool(post), "simplified": info["simplified"]}
        # per-shot work of the widest configs is large: fewer repetitions
        st_w, st_n = (1, 1) if shots0 < 1000 else (warmup, steps)
        modes = (("fp32_batched", S.FP32, S.PLAIN_OFF, 1.0), ("fp64_batched", S.FP64, S.PLAIN_OFF, 1.0),
                 ("fp64_plain_in_kernel", S.FP64, S.PLAIN_IN_KERNEL, 0.1),
                 ("fp64_plain_prepass", S.FP64, S.PLAIN_PREPASS, 0.1))
        for mode, prec, plain, frac in modes:
            shots = max(128, int(shots0 * scale * frac))
            try:
                entry[mode] = _time_call(S, torch, dev, stream, plan, shots, 100, st_n, st_w,
                                         precision=prec, plain=plain)
            except S.SymftError as e:
                entry[mode] = {"unavailable": str(e)}
        plains = [entry[m] for m in ("fp64_plain_in_kernel", "fp64_plain_prepass") if "shots_per_s" in entry[m]]
        if plains:
            best = max(plains, key=lambda d: d["shots_per_s"])
            entry["fp64_plain"] = {"shots_per_s": best["shots_per_s"],
                                   "form": "prepass" if best is entry["fp64_plain_prepass"] else "in_kernel"}
            entry["fp32_batched_over_fp64_plain"] = entry["fp32_batched"]["shots_per_s"] / best["shots_per_s"]
        if "shots_per_s" in entry["fp64_batched"]:
            entry["fp32_batched_over_fp64_batched"] = (entry["fp32_batched"]["shots_per_s"] /
                                                      entry["fp64_batched"]["shots_per_s"])
        entry["gpu_fp32_vs_gpu_fp64"] = fp32_accuracy(S, torch, plan, dev, stream, shots=min(1 << 16, shots0))
        # roofline of the FP32-batched path: every shot runs the whole stream
        if info["k_max"] > 0:
            fl = dense_floor(info, peaks)
            plan0 = S.symft_compile(text, postselect=0) if post else plan
            rshots = max(128, int(shots0 * scale)) if shots0 >= 1000 else max(32, shots0 // 2)
            run = _time_call(S, torch, dev, stream, plan0, rshots, 500, st_n, st_w, precision=S.FP32)
            t_shot = run["ms_per_step"] / 1e3 / rshots
            fl["no_postselect_shots_per_s"] = run["shots_per_s"]
            fl["frac"] = fl["floor_s_per_shot"] / t_shot
            fl["note"] = ("floor of the dense instructions alone, against the whole step (sign "
                          "kernel, executor, finalize): a lower bound on the executor's own fraction")
            entry["roofline"] = fl
        out[name] = entry
    return out


def measure_mixed_batch(S, torch, dev, stream, steps, warmup, n_circuits=64, target_ms=2.0):
    """64 mixed circuits (k_max <= 20): autotuned FP32 jobs in one graph launch per
    step, against untuned sequential FP64 calls: the paper's GPU design (one CTA
    per shot, the faster of its two forms per circuit) on the circuits whose
    vectors fit its shared memory, and the batched FP64 path on all.  Ratios are
    taken over the same circuits."""
    from paper_2607_28600_b300.workloads import mixed_batch
    plans, texts = [], []
    for name, text, post in mixed_batch(seed=1, n=4 * n_circuits):
        pl = S.symft_compile(text, postselect=post)
        if pl.info["k_max"] > 20:
            continue
        plans.append(pl)
        texts.append((text, post))
        if len(plans) == n_circuits:
            break
    t0 = time.perf_counter()
    tuned = []
    for pl in plans:
        k = pl.info["k_max"]
        S.symft_autotune(pl, int(min(65536, max(256, (1 << 22) >> k))), S.FP32, stream=stream)
        tuned.append(pl.refresh_info()["tuned_ns_per_shot"][0])
    tune_s = time.perf_counter() - t0
    shots = [int(min(10_000_000, max(128, (target_ms * 1e6 / max(ns, 1e-3)) // 128 * 128))) for ns in tuned]
    outs = []
    for pl, n in zip(plans, shots):
        W = (n + 63) // 64
        info = pl.info
        mk = lambda m: torch.empty((max(1, m), W), dtype=torch.int64, device=dev)
        outs.append({"meas_out": mk(info["n_records"]), "det_out": mk(info["n_dets"]),
                     "obs_out": mk(info["n_obs"]),
                     "discard_out": torch.empty((W,), dtype=torch.int64, device=dev)})
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def graph_ms(idx, step0):
        sub = [plans[i] for i in idx]
        jobs = lambda st: [{"plan": j, "shots": shots[i], "seed": 1000 * st + i, "precision": S.FP32,
                            **outs[i]} for j, i in enumerate(idx)]
        for w in range(warmup):
            S.symft_sample_batch(sub, jobs(step0 + w), stream=stream)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for st in range(steps):
            S.symft_sample_batch(sub, jobs(step0 + warmup + st), stream=stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / steps, S.symft_last_launch_count()

    all_idx = list(range(len(plans)))
    ms_all, launches = graph_ms(all_idx, 0)
    # untuned FP64 on fresh plans, one call per circuit, each timed on its own
    fresh = [S.symft_compile(t, postselect=post) for t, post in texts]
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in fresh]

    def per_circuit_ms(**kw):
        res = []
        for (a, b), pl, n, o in zip(ev, fresh, shots, outs):
            try:
                S.symft_sample_ex(pl, n, 7, precision=S.FP64, stream=stream, **kw, **o)   # warm-up
                a.record(stream)
                S.symft_sample_ex(pl, n, 8, precision=S.FP64, stream=stream, **kw, **o)
                b.record(stream)
                res.append((a, b))
            except S.SymftError:
                res.append(None)
        torch.cuda.synchronize(dev)
        return [None if r is None else r[0].elapsed_time(r[1]) for r in res]
    plain_ik = per_circuit_ms(plain=S.PLAIN_IN_KERNEL)
    plain_pp = per_circuit_ms(plain=S.PLAIN_PREPASS)
    batched64 = per_circuit_ms(plain=S.PLAIN_OFF)
    plain_best = [min([x for x in (a, b) if x is not None]) if (a is not None or b is not None) else None
                  for a, b in zip(plain_ik, plain_pp)]
    fits = [i for i in all_idx if plain_best[i] is not None]
    ms_fits, _ = graph_ms(fits, 100)
    total, total_fits = sum(shots), sum(shots[i] for i in fits)
    res = {"n_circuits": len(plans), "total_shots_per_step": total,
           "k_max_hist": {str(k): sum(1 for p in plans if p.info["k_max"] == k)
                          for k in sorted(set(p.info["k_max"] for p in plans))},
           "autotune_s": tune_s,
           "fp32_autotuned_graph": {"ms_per_step": ms_all, "shots_per_s": total / (ms_all / 1e3),
                                    "kernel_launches_per_step": launches, "graph_launches_per_step": 1},
           "fp64_batched_untuned": {"ms": sum(batched64), "shots_per_s": total / (sum(batched64) / 1e3)},
           "fits_plain_design": {
               "n_circuits": len(fits), "shots_per_step": total_fits,
               "fp32_autotuned_graph_ms": ms_fits,
               "fp64_plain_best_form_untuned_ms": sum(plain_best[i] for i in fits),
               "fp64_batched_untuned_ms": sum(batched64[i] for i in fits),
               "plain_form_chosen": {"in_kernel": sum(1 for i in fits if plain_ik[i] is not None and
                                                      plain_ik[i] == plain_best[i]),
                                     "prepass": sum(1 for i in fits if plain_ik[i] is None or
                                                    plain_ik[i] != plain_best[i])}}}
    # each circuit: the tuner's executor, its tuned time per shot and the dense
    # floor of a full shot (on-chip FP / shared memory, or HBM for wide vectors)
    peaks = all_peaks(S)
    circ = []
    for pl, ns in zip(plans, tuned):
        info = pl.refresh_info()
        row = {"k_max": info["k_max"], "executor": info["dense_executor"][0],
               "tuned_ns_per_shot": ns, "shots": shots[plans.index(pl)]}
        if row["executor"] == "wide":
            row["wide_tile_bits"] = info["wide_tile_bits"][0]
        if info["k_max"] > 0:
            fl = dense_floor(info, peaks)
            row["dense_floor_ns_per_shot"] = fl["floor_s_per_shot"] * 1e9
            row["frac_of_tuned_time"] = fl["floor_s_per_shot"] * 1e9 / max(ns, 1e-9)
            row["bound"] = fl.get("bound", fl["where"])
        circ.append(row)
    res["per_circuit"] = circ
    res["executors"] = {k: sum(1 for r in circ if r["executor"] == k) for k in sorted(set(r["executor"] for r in circ))}
    # graph launch overhead: the same graph with 64 shots per job
    tiny = [{"plan": i, "shots": 64, "seed": 5 + i, "precision": S.FP32, **outs[i]} for i in all_idx]
    for _ in range(2):
        S.symft_sample_batch(plans, tiny, stream=stream)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for _ in range(5):
        S.symft_sample_batch(plans, tiny, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    res["graph_with_64_shots_per_job_ms"] = e0.elapsed_time(e1) / 5
    res["graph_overhead_share"] = res["graph_with_64_shots_per_job_ms"] / ms_all
    f = res["fits_plain_design"]
    f["fp32_autotuned_over_fp64_plain"] = f["fp64_plain_best_form_untuned_ms"] / ms_fits
    f["fp32_autotuned_over_fp64_batched"] = f["fp64_batched_untuned_ms"] / ms_fits
    res["fp32_autotuned_over_fp64_batched_all"] = sum(batched64) / ms_all
    return res


def _pinned_worker(args):
    """Tableau oracle pinned to one host core for about budget_s (a child process)."""
    core, budget_s = args
    os.sched_setaffinity(0, {core})
    _oracle_worker_init()
    n, lo = 0, 0
    _oracle_chunk((0, 8))
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < budget_s:
        n += _oracle_chunk((lo, lo + 64))
        lo += 64
    return n, time.perf_counter() - t0


def _symft_oracle_worker(args):
    """Plain SymFT oracle (FP64, one shot at a time) on the cultivation-shaped
    circuit, pinned to one core, for about budget_s."""
    core, budget_s = args
    os.sched_setaffinity(0, {core})
    from oracle import symft as osymft
    from oracle.circuit import parse
    from oracle.noise import NoiseSampler
    text = _near_clifford_text("cultivation")
    c = parse(text)
    plan = osymft.Plan(c)
    noise = NoiseSampler(c, 1)
    osymft.sample_shot(plan, 1, 0, noise)
    n = 0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < budget_s:
        osymft.sample_shot(plan, 1, n, noise)
        n += 1
    return n, time.perf_counter() - t0


def cpu_baselines(budget_s=8.0):
    """The oracle as it stands on the host cores: the tableau sampler on every
    core (the headline workload), the same on one pinned core, and the plain
    SymFT interpreter on one pinned core for the cultivation-shaped circuit."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    out = {"all_cores": cpu_baseline(budget_s)}
    ctx = mp.get_context("spawn")
    with ctx.Pool(1) as pool:
        n, dt = pool.map(_pinned_worker, [(0, budget_s)])[0]
    out["one_core"] = {"value": n / dt, "unit": "shots/s", "cores": 1, "kind": "oracle",
                       "sample": f"{n} shots of {HEADLINE} through the tableau oracle pinned to core 0 "
                                 f"in {dt:.1f} s"}
    with ctx.Pool(1) as pool:
        n, dt = pool.map(_symft_oracle_worker, [(0, budget_s)])[0]
    out["near_clifford_one_core"] = {
        "value": n / dt, "unit": "shots/s", "cores": 1, "kind": "oracle",
        "sample": f"{n} shots of the cultivation-shaped circuit (c3, FP64) through the plain "
                  f"SymFT oracle pinned to core 0 in {dt:.1f} s; host has {cores} cores"}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="b300")
    ap.add_argument("--shots", type=int, default=SHOTS)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--only", default=None,
                    help="run one part (profiling): a surface-code workload name, "
                         "near_clifford, a near-Clifford config name, or mixed_batch")
    ap.add_argument("--no-near-clifford", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    import paper_2607_28600_b300 as S
    from paper_2607_28600_b300.workloads import rotated_surface_code_memory

    world, rank, local = _dist()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    stream = torch.cuda.current_stream(dev)
    shots = args.shots
    W = (shots + 63) // 64
    from paper_2607_28600_b300.sharding import weak_offset
    offset = weak_offset(shots, rank)
    if args.only in ("near_clifford", "mixed_batch") or args.only in NEAR_CLIFFORD:
        if args.only == "mixed_batch":
            res = measure_mixed_batch(S, torch, dev, stream, steps=args.steps, warmup=args.warmup)
        else:
            res = measure_near_clifford(S, torch, dev, stream, steps=args.steps, warmup=args.warmup,
                                        peaks=all_peaks(S),
                                        only=None if args.only == "near_clifford" else args.only)
        if rank == 0:
            print(json.dumps({args.only: res}), flush=True)
        return

    per_circuit = {}
    headline = None
    for name, w in WORKLOADS.items():
        if args.only and name != args.only:
            continue
        plan = S.symft_compile(rotated_surface_code_memory(w["d"], w["rounds"], w["p"]))
        info = plan.info
        meas = torch.empty((info["n_records"], W), dtype=torch.int64, device=dev)
        det = torch.empty((info["n_dets"], W), dtype=torch.int64, device=dev)
        obs = torch.empty((info["n_obs"], W), dtype=torch.int64, device=dev)

        def step(i):
            S.symft_sample_ex(plan, shots, 1000 + i, shot_offset=offset, meas_out=meas,
                              det_out=det, obs_out=obs, stream=stream)

        for i in range(args.warmup):
            step(i)
        launches_per_step = S.symft_last_launch_count()
        torch.cuda.synchronize(dev)
        if world > 1:
            torch.distributed.barrier()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * args.steps)]
        with ClockSampler(local) as clk:
            torch.cuda.synchronize(dev)
            t_host0 = time.perf_counter()
            for i in range(args.steps):
                ev[2 * i].record(stream)
                step(args.warmup + i)
                ev[2 * i + 1].record(stream)
            torch.cuda.synchronize(dev)
            t_host = time.perf_counter() - t_host0
        per_launch_ms = [ev[2 * i].elapsed_time(ev[2 * i + 1]) for i in range(args.steps)]
        total_ms = ev[0].elapsed_time(ev[-1])
        ms = torch.tensor([total_ms / args.steps], device=dev)
        if world > 1:
            torch.distributed.all_reduce(ms, op=torch.distributed.ReduceOp.MAX)
        ms_step = float(ms.item())
        out_bytes = (info["n_records"] + info["n_dets"] + info["n_obs"]) * W * 8
        kernel_ms = sum(per_launch_ms) / len(per_launch_ms)
        per_circuit[name] = {
            "shots_per_s": world * shots / (ms_step / 1e3),
            "ms_per_step": ms_step,
            "kernel_ms": kernel_ms,
            "output_bytes_per_step": out_bytes,
            "launches_per_step": launches_per_step,
            "n_channels": info["n_channels"], "n_records": info["n_records"],
            "n_dets": info["n_dets"],
        }
        # the same circuit through the paper's GPU design in FP64: in-kernel
        # sampling (one CTA per shot, fewer shots) and the packed-column prepass;
        # the faster form is the FP64-plain figure
        pin = _time_call(S, torch, dev, stream, plan, max(128, shots // 20), 50, 3, 2,
                         precision=S.FP64, plain=S.PLAIN_IN_KERNEL)
        ppp = _time_call(S, torch, dev, stream, plan, shots, 60, 3, 2,
                         precision=S.FP64, plain=S.PLAIN_PREPASS)
        best = pin if pin["shots_per_s"] >= ppp["shots_per_s"] else ppp
        per_circuit[name]["fp64_plain_in_kernel"] = pin
        per_circuit[name]["fp64_plain_prepass"] = ppp
        per_circuit[name]["fp64_plain"] = {"shots_per_s": best["shots_per_s"],
                                           "form": "in_kernel" if best is pin else "prepass"}
        per_circuit[name]["batched_over_plain"] = per_circuit[name]["shots_per_s"] / best["shots_per_s"]
        per_circuit[name]["batched_over_plain_in_kernel"] = per_circuit[name]["shots_per_s"] / pin["shots_per_s"]
        if name == HEADLINE:
            headline = dict(plan=plan, info=info, clk=clk.summary(), t_host=t_host,
                            kernel_ms=kernel_ms, out_bytes=out_bytes, ms_step=ms_step,
                            launches=launches_per_step, meas=meas, det=det, obs=obs)
        else:
            del meas, det, obs

    if headline is None:
        if rank == 0:
            print(json.dumps({"per_circuit": per_circuit}), flush=True)
        return
    h = headline
    # end-to-end: the public call with HOST outputs (pinned), D2H inside the timed region
    plan = h["plan"]
    info = h["info"]
    hm = torch.empty((info["n_records"], W), dtype=torch.int64, pin_memory=True)
    hd = torch.empty((info["n_dets"], W), dtype=torch.int64, pin_memory=True)
    ho = torch.empty((info["n_obs"], W), dtype=torch.int64, pin_memory=True)
    if not args.no_e2e:
        S.symft_sample_ex(plan, shots, 7, shot_offset=offset, meas_out=hm, det_out=hd, obs_out=ho,
                          out_location=S.OUT_HOST, stream=stream)
    e2e_steps = 0 if args.no_e2e else max(2, min(args.steps, 5))
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        S.symft_sample_ex(plan, shots, 2000 + i, shot_offset=offset, meas_out=hm, det_out=hd,
                          obs_out=ho, out_location=S.OUT_HOST, stream=stream)
    e2e_s = (time.perf_counter() - t0) / max(1, e2e_steps)
    if world > 1:
        # the slowest rank sets the whole job's end-to-end time, as for `value`
        t = torch.tensor([e2e_s], device=dev, dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e_val = world * shots / e2e_s if e2e_steps else None

    if rank != 0:
        return
    peaks = all_peaks(S)
    peak, peak_kind = peaks["hbm_gbs"], peaks["hbm_kind"]
    achieved = h["out_bytes"] / (h["kernel_ms"] / 1e3) / 1e9
    # integer work of the same launch (plan model) against the measured Philox
    # and LOP3 rates: the time those pipes need at their peaks
    sm = info["sign_model"]
    blocks = (shots + 511) // 512
    ks = h["kernel_ms"] / 1e3
    t_philox = blocks * sm["philox_blocks_per_block"] / peaks["philox_blocks_per_s"]
    t_xor = blocks * sm["xor_ops_per_block"] / peaks["int32_lop3_per_s"]
    t_hbm = h["out_bytes"] / (peak * 1e9)
    alu = {"philox_blocks_per_launch": blocks * sm["philox_blocks_per_block"],
           "achieved_philox_blocks_per_s": blocks * sm["philox_blocks_per_block"] / ks,
           "peak_philox_blocks_per_s": peaks["philox_blocks_per_s"],
           "xor_ops_per_launch": blocks * sm["xor_ops_per_block"],
           "peak_lop3_per_s": peaks["int32_lop3_per_s"],
           "floor_ms": max(t_philox, t_xor) * 1e3, "frac": max(t_philox, t_xor) / ks,
           "philox_floor_ms": t_philox * 1e3, "xor_floor_ms": t_xor * 1e3,
           "peak_kind": "measured now (symft_measure_peaks)"}
    line = {
        "metric": METRIC,
        "value": world * shots / (h["ms_step"] / 1e3),
        "unit": "shots/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": h["ms_step"],
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u64",
        "data": "synthetic",
        "config": {"workload": HEADLINE_WORKLOAD,
                   "shots_per_step": shots, "shots_per_word": 64,
                   "l2": "outputs (%.0f MB per step) exceed the 126 MB L2; no flush needed"
                         % (h["out_bytes"] / 1e6),
                   "parallelism": f"shot ranges x{world}"},
        "per_circuit": per_circuit,
        "roofline": {"bound": "hbm" if t_hbm >= max(t_philox, t_xor) else "alu",
                     "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": _sign_traffic() if shots == SHOTS else None,
                     "kernel": "sign_kernel", "peak_kind": peak_kind,
                     "algorithmic_bytes_per_launch": h["out_bytes"], "hbm_floor_ms": t_hbm * 1e3,
                     "alu": alu},
        "peaks": {k: v for k, v in peaks.items()},
        "e2e": {"value": e2e_val, "unit": "shots/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": h["out_bytes"]},
        "gpu_launches": h["launches"] * args.steps,
        "clocks": h["clk"],
    }
    if not args.no_near_clifford and world == 1:
        line["near_clifford"] = measure_near_clifford(S, torch, dev, stream, steps=5, warmup=3, peaks=peaks)
        line["mixed_batch"] = measure_mixed_batch(S, torch, dev, stream, steps=5, warmup=3)
    if not args.no_cpu_baseline and world == 1:
        cb = cpu_baselines()
        line["cpu_baseline"] = cb["all_cores"]
        line["cpu_baselines"] = cb
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
