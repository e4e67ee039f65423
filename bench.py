"""ParaQAOA hot-path benchmark (one JSON line on rank 0).

Workload (the paper-scale configuration): Erdos-Renyi G(400, 0.1) and
G(400, 0.5), integer weights uniform in {1..10}, seed 0; the balanced
partition gives 21 parts of 20 vertices (2^20 complex64 amplitudes each).
One step solves both graphs end to end: p = 1 grid (16 x 16), 32 Adam steps
at p = 1, INTERP to p = 2, 32 Adam steps at p = 2, a final simulation that
keeps the states, top-16 per part and a beam-256 merge. The metric counts
every amplitude-layer the step simulates (2^n * p per evaluated instance).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) the same workload is sharded across the ranks by
default: each graph's parts are assigned to ranks by longest processing time
first, each rank solves its parts on its GPU, the M x K candidate arrays are
summed onto rank 0 (the one exchange) and rank 0 merges (strong scaling).
--replicas instead gives every rank its own copy of the workload (graph
seeds offset by rank; weak scaling, no data-path collective).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "QAOA amplitude-layer updates/s (%HBM roofline); 16k-vertex time-to-cut"
UNIT = "amp-layer/s"
NV, M, K, BEAM, P_FINAL, GRID, STEPS_ADAM = 400, 21, 16, 256, 2, 16, 32
DENSITIES = (0.1, 0.5)
WMAX = 10


def max_over_ranks(values, dist, device):
    """Element-wise maximum of per-rank timings over all ranks (the job takes
    as long as its slowest rank); the values themselves when not distributed."""
    if dist is None:
        return [float(v) for v in values]
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t]


def job_value(units_per_rank_step: float, steps: int, world: int, ms: float) -> float:
    """Whole-job throughput under weak scaling: the units every rank processed
    over the slowest rank's time (under strong scaling pass world = 1 and the
    whole job's units per step)."""
    return units_per_rank_step * steps * world / (ms / 1e3)


def workload(rank: int):
    """The paper-scale graphs; rank r's own copy has seed r (replica mode),
    the sharded job uses rank 0's."""
    return [synth.erdos_renyi(NV, pe, seed=rank, wmax=WMAX) for pe in DENSITIES]


def amp_layers_per_graph(n: int = 20) -> int:
    """Amplitude-layers one solve of one graph simulates."""
    d = 1 << n
    grid = GRID * GRID * M * d * 1
    adam1 = STEPS_ADAM * 4 * 1 * M * d * 1 + M * d * 1   # shifted evals + final eval
    adam2 = STEPS_ADAM * 4 * 2 * M * d * 2 + M * d * 2
    final = M * d * P_FINAL
    return grid + adam1 + adam2 + final


def config_dict():
    return {"workload": "G(400,0.1)+G(400,0.5), w in {1..10}, seed 0; 21 parts x 20 qubits (2^20 complex64); "
                        "p=1 16x16 grid + 32 Adam -> INTERP -> p=2 32 Adam; top-16; beam-256 merge",
            "graphs": 2, "parts_per_graph": M, "qubits": 20, "p": P_FINAL, "K": K, "beam": BEAM,
            "adam_steps": STEPS_ADAM, "grid": f"{GRID}x{GRID}",
            "l2": "working set > L2: every batch streams >= 1.3 GB of state"}


def read_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


LAYER_PASS_SOURCES = [os.path.join(ROOT, "paper_2603_26232_gb300", "csrc", f)
                      for f in ("layer_pass.cu", "sim_common.cuh")]


def kernel_sources_sha256(paths) -> str:
    """sha256 over the concatenated sources of a kernel (the layer pass and
    the device helpers it includes)."""
    h = hashlib.sha256()
    for path in paths:
        h.update(open(path, "rb").read())
    return h.hexdigest()


def traffic_for(kernel_srcs, alg_bytes_per_launch: float):
    """DRAM bytes per layer-pass launch: the ncu-measured DRAM/algorithmic ratio
    of profiles/layer_pass_traffic.json times this run's algorithmic bytes per
    launch; None when the kernel sources changed since that capture."""
    path = os.path.join(ROOT, "profiles", "layer_pass_traffic.json")
    if not os.path.exists(path):
        return None
    rec = json.load(open(path))
    if rec.get("source_sha256") != kernel_sources_sha256(kernel_srcs):
        return None
    return rec["dram_over_algorithmic"] * alg_bytes_per_launch


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(seconds: float = 15.0):
    """The oracle, as it stands, on this host's cores: <C> evaluations of
    20-qubit parts at p = 2 (the Adam batches of the workload), until about
    `seconds` of CPU work."""
    import oracle
    g = synth.erdos_renyi(NV, 0.1, 0, wmax=WMAX)
    subs = oracle.subgraphs(g, M)
    batch = oracle.Batch(subs)
    gam, bet = synth.random_angles(M, 2, 5)
    done, t0 = 0, time.perf_counter()
    chunk = max(1, oracle.num_threads())
    while time.perf_counter() - t0 < seconds:
        idx = (np.arange(chunk) + done) % M
        oracle.expect_batch(batch, idx.astype(np.int32), gam[idx], bet[idx])
        done += chunk
    dt = time.perf_counter() - t0
    amps = done * (1 << 20) * 2
    rate = amps / dt
    return {"value": rate, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{done} oracle <C> evaluations of 20-qubit parts at p=2 (complex128), {dt:.1f} s",
            # one graph's solve (its amplitude-layers) at the sampled rate
            "projected_time_to_cut_s": amp_layers_per_graph() / rate}


def cpu_baseline_one_core(seconds: float = 6.0):
    """The same oracle sample on one host core: a child process (exec, not a
    fork of this one) with OpenMP limited to one thread."""
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-sample", str(seconds)],
                       env=env, capture_output=True, text=True, timeout=600)
    if r.returncode != 0:
        return {"error": (r.stderr or r.stdout).strip().splitlines()[-1:]}
    return json.loads(r.stdout.strip().splitlines()[-1])


def run_reference(args, rank, world):
    if rank != 0:
        return
    cb = cpu_baseline(seconds=max(5.0, 20.0 / max(1, args.steps + args.warmup)))
    vals = []
    for _ in range(args.warmup):
        cpu_baseline(seconds=2.0)
    for _ in range(args.steps):
        vals.append(cpu_baseline(seconds=max(3.0, 60.0 / max(1, args.steps)))["value"])
    v = statistics.median(vals) if vals else cb["value"]
    cb["value"] = v
    # the oracle runs a bounded sample of each step: a full step's time at
    # the sampled rate
    ms_step = 1e3 * amp_layers_per_graph() * len(DENSITIES) / v if v > 0 else None
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "ms_per_step_basis": "full step projected from the sampled rate", "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(), "cpu_baseline": cb,
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_layer_case(args):
    """168 instances (21 parts x 8 angle sets) of 20 qubits of G(400,
    --layer-density) at p = --layer-p (default 2: one Adam-step batch of the
    workload), <C> only; prints the layer passes' timing."""
    import torch
    import paper_2603_26232_gb300 as pkg
    from paper_2603_26232_gb300 import _capi as capi

    pkg.build()
    g = synth.erdos_renyi(NV, args.layer_density, 0, wmax=WMAX)
    ctx = capi.paraqaoa_create(0)
    G = capi.Graph.of(g)
    part = capi.paraqaoa_partition(G, M)
    ids = np.repeat(np.arange(M, dtype=np.int32), 8)
    P = args.layer_p
    gam, bet = synth.random_angles(len(ids), P, 3)
    capi.paraqaoa_part_upload(ctx, part)
    if args.sched:
        sc = tuple(int(x) for x in args.sched.split(","))
        sc = sc + (0,) * (5 - len(sc))
        capi.paraqaoa_set_schedule(ctx, 20, *sc)
        tuned = {20: sc}
    else:
        tuned = {20: (None,) * 5} if args.no_autotune else capi.paraqaoa_autotune(ctx, part, P)
    for it in range(args.iters):
        if it == args.iters - 1:
            capi.paraqaoa_profile_enable(ctx, True)
        capi.paraqaoa_simulate_batch(ctx, part, ids, P, gam, bet, capi.SIM_EXPECT)
        capi.paraqaoa_expect(ctx, len(ids))
    n_l, ms, by = capi.paraqaoa_profile_read(ctx, capi.KCLASS_LAYER_PASS)
    peak, kind = read_peaks()
    print(json.dumps({"case": "layer_pass", "instances": int(len(ids)), "qubits": 20, "p": P,
                      "tile_bits": tuned[20][0], "reg_bits": tuned[20][1], "min_run_qubits": tuned[20][2],
                      "split": tuned[20][3], "tiles_per_cta_log2": tuned[20][4],
                      "launches": n_l, "ms": ms, "algorithmic_bytes": by,
                      "achieved_gbs": by / (ms / 1e3) / 1e9, "peak_gbs": peak,
                      "frac": by / (ms / 1e3) / 1e9 / peak}), flush=True)
    capi.paraqaoa_part_free(part)
    capi.paraqaoa_destroy(ctx)


LARGE_N, LARGE_P_EDGE, LARGE_M, LARGE_K, LARGE_BEAM, LARGE_DEPTH = 16000, 0.01, 640, 32, 64, 2
LARGE_JUDGE_TOL = 1e-2


def train_large_model(capi, ctx, depth=LARGE_DEPTH, count=2048, epochs=100, seed=7):
    """Angle network for the large workload: labels from the plain form on
    method-generated unit-weight random subgraphs of 12..16 vertices whose
    edge counts span those of the workload's parts (G(n, P), P in
    [0.005, 0.06]); returns the network and the seconds spent."""
    t0 = time.perf_counter()
    specs = synth.graph_specs(count, 12, 16, 0.005, 0.06, seed)
    G, sizes = synth.chain_of_graphs(specs, wmax=1)
    part = capi.paraqaoa_partition(capi.Graph.of(G), len(sizes), capi.PART_SIZES, sizes)
    ids = np.arange(len(sizes), dtype=np.int32)
    g, b, _ = capi.paraqaoa_solve_plain(ctx, part, ids, depth, STEPS_ADAM)
    X = capi.paraqaoa_features(ctx, part, ids)
    capi.paraqaoa_part_free(part)
    T = np.concatenate([g, b], axis=1).astype(np.float32)
    net = capi.paraqaoa_mlp_create(ctx, depth, synth.mlp_init(depth, seed))
    losses = capi.paraqaoa_mlp_train(net, X, T, epochs, 128, 1e-3, synth.epoch_orders(count, epochs, seed))
    return net, time.perf_counter() - t0, float(losses[-1])


def large_learned(capi, pkg, plain: bool = True):
    """16,000-vertex time-to-cut of the learned form (network trained first,
    outside the clock) and, unless plain is False, of the plain form (grid +
    Adam + INTERP + Adam, about three and a half minutes) on the same GPU,
    with their cut and time ratios."""
    import torch
    free, _ = torch.cuda.mem_get_info()
    solver = pkg.Solver(device=torch.cuda.current_device(), hbm_budget=int(0.6 * free))
    g = synth.erdos_renyi(LARGE_N, LARGE_P_EDGE, 0, wmax=1)
    G = capi.Graph.of(g)
    net, train_s, _ = train_large_model(capi, solver.ctx)
    cfg = pkg.SolveConfig(M=LARGE_M, K=LARGE_K, p=LARGE_DEPTH, beam=LARGE_BEAM, mlp=net,
                          fallback_steps=STEPS_ADAM, judge_tol=LARGE_JUDGE_TOL)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = solver.solve(G, cfg)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    capi.paraqaoa_mlp_free(net)
    out = {"workload": f"G({LARGE_N},{LARGE_P_EDGE}) unit weights, seed 0; {LARGE_M} parts of 25-26 qubits; "
                       f"p={LARGE_DEPTH}; top-{LARGE_K}; beam-{LARGE_BEAM}",
           "form": "learned angles + judge + plain fallback", "time_to_cut_s": dt, "cut": int(r.cut),
           "train_s": train_s, "verdicts": {"network": int(np.sum(r.fallback == 0)),
                                            "plain_fallback": int(np.sum(r.fallback == 1)),
                                            "reference": int(np.sum(r.fallback == 2))}}
    if plain:
        cfg_p = pkg.SolveConfig(M=LARGE_M, K=LARGE_K, p=LARGE_DEPTH, grid_points=GRID, adam_steps=STEPS_ADAM,
                                beam=LARGE_BEAM)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rp = solver.solve(G, cfg_p)
        torch.cuda.synchronize()
        dtp = time.perf_counter() - t0
        out["plain_form"] = {"time_to_cut_s": dtp, "cut": int(rp.cut)}
        out["cut_ratio_learned_over_plain"] = int(r.cut) / int(rp.cut)
        out["time_ratio_plain_over_learned"] = dtp / dt
    else:
        out["plain_form"] = "skipped (--no-large-plain); bench.py --case large measures it"
    solver.close()
    return out


def batching_measure(capi, ctx, reps: int = 5):
    """Batching configuration: G(2000, 0.05), unit weights, uneven parts of
    12..24 vertices (about 120), p = 3, random angles, <C> of every part in one
    simulate call, schedules autotuned; amplitude-layers/s over the wall time
    of simulate + expect, with the size classes on side streams (profiling
    off), in order (profiling on), and in the persistent form (one launch per
    tile shape), and the 16 B roofline fraction."""
    import torch
    g = synth.erdos_renyi(2000, 0.05, 0, wmax=1)
    sizes = synth.uneven_sizes(2000, 12, 24, 1)
    part = capi.paraqaoa_partition(capi.Graph.of(g), len(sizes), capi.PART_SIZES, sizes)
    ids = np.arange(len(sizes), dtype=np.int32)
    gam, bet = synth.random_angles(len(sizes), 3, 3)
    capi.paraqaoa_autotune(ctx, part, 3)
    amp_layers = float(np.sum(np.left_shift(1, sizes.astype(np.int64)))) * 3
    peak, _ = read_peaks()
    out = {"workload": "G(2000,0.05) unit weights, seed 0; uneven parts of 12..24 vertices; p=3",
           "parts": int(len(sizes)), "amplitude_layers": amp_layers}
    for name, prof, persistent in (("side_streams", False, False), ("serial", True, False),
                                   ("persistent", False, True)):
        capi.paraqaoa_profile_enable(ctx, prof)
        capi.paraqaoa_set_persistent(ctx, persistent)
        capi.paraqaoa_simulate_batch(ctx, part, ids, 3, gam, bet, capi.SIM_EXPECT)
        capi.paraqaoa_expect(ctx, len(ids))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            capi.paraqaoa_simulate_batch(ctx, part, ids, 3, gam, bet, capi.SIM_EXPECT)
            ex = capi.paraqaoa_expect(ctx, len(ids))
        dt = (time.perf_counter() - t0) / reps
        rate = amp_layers / dt
        out[name] = {"s_per_batch": dt, "amp_layers_per_s": rate, "frac_16B_roofline": rate * 16 / (peak * 1e9)}
    capi.paraqaoa_profile_enable(ctx, False)
    capi.paraqaoa_set_persistent(ctx, False)
    out["mean_expect"] = float(np.mean(ex))
    capi.paraqaoa_part_free(part)
    return out


def run_batching_case(args):
    import paper_2603_26232_gb300 as pkg
    from paper_2603_26232_gb300 import _capi as capi

    pkg.build()
    ctx = capi.paraqaoa_create(0)
    out = dict(case="batching", **batching_measure(capi, ctx))
    capi.paraqaoa_destroy(ctx)
    print(json.dumps(out), flush=True)


def run_tc_case(args):
    """Split-precision tensor-core mixer on the batching configuration
    (G(2000, 0.05), unit weights, 122 parts of 12..24 vertices, p = 3, random
    angles): amplitude-layers/s of paraqaoa_simulate_tc (FP16 and BF16 splits,
    blocks of up to --tc-k qubits) against the FP32 butterfly path, and the largest
    |d<C>| / W against the FP32 path over all parts (itself within 1e-5 W of
    the FP64 oracle) and against the FP64 oracle on the parts of <= 18 qubits."""
    import torch
    import oracle
    import paper_2603_26232_gb300 as pkg
    from paper_2603_26232_gb300 import _capi as capi

    pkg.build()
    ctx = capi.paraqaoa_create(0)
    g = synth.erdos_renyi(2000, 0.05, 0, wmax=1)
    sizes = synth.uneven_sizes(2000, 12, 24, 1)
    part = capi.paraqaoa_partition(capi.Graph.of(g), len(sizes), capi.PART_SIZES, sizes)
    ids = np.arange(len(sizes), dtype=np.int32)
    keep = sizes >= 12
    ids = ids[keep]
    gam, bet = synth.random_angles(len(ids), 3, 3)
    W = np.array([max(int(w), 1) for w in capi.paraqaoa_part_info(part)[3][ids]], float)
    amp_layers = float(np.sum(np.left_shift(1, sizes[keep].astype(np.int64)))) * 3
    subs = oracle.subgraphs(g, len(sizes), 2, sizes)
    small = [i for i, k in enumerate(ids) if sizes[k] <= 18][:24]
    oex = oracle.expect_batch(oracle.Batch([subs[ids[i]] for i in small]), np.arange(len(small), dtype=np.int32),
                              gam[small], bet[small])
    out = {"case": "tc", "workload": "G(2000,0.05) unit weights, seed 0; parts of 12..24 vertices; p=3",
           "parts": int(len(ids)), "oracle_parts": len(small), "block_qubits": args.tc_k}

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(3):
            ex = fn()
        return ex, (time.perf_counter() - t0) / 3

    def fp32():
        capi.paraqaoa_simulate_batch(ctx, part, ids, 3, gam, bet, capi.SIM_EXPECT)
        return capi.paraqaoa_expect(ctx, len(ids))
    ex32, t32 = timed(fp32)
    out["fp32"] = {"amp_layers_per_s": amp_layers / t32,
                   "max_dC_over_W_vs_oracle": float(np.max(np.abs(ex32[small] - oex) / W[small]))}
    for name, prec in (("fp16_split", capi.TC_FP16), ("bf16_split", capi.TC_BF16)):
        def tc():
            capi.paraqaoa_simulate_tc(ctx, part, ids, 3, gam, bet, capi.SIM_EXPECT, prec, args.tc_k)
            return capi.paraqaoa_expect(ctx, len(ids))
        ex, t = timed(tc)
        out[name] = {"amp_layers_per_s": amp_layers / t,
                     "max_dC_over_W_vs_fp32_path": float(np.max(np.abs(ex - ex32) / W)),
                     "max_dC_over_W_vs_oracle": float(np.max(np.abs(ex[small] - oex) / W[small]))}
    capi.paraqaoa_part_free(part)
    capi.paraqaoa_destroy(ctx)
    print(json.dumps(out), flush=True)


def sweep_point(capi, ctx, n: int, reps: int = 3):
    """One point of the amplitude-layer sweep: a batch of parts of n vertices
    (G(*, 0.3) chain below 24 qubits, 0.2 from 24, weights 1..10) with
    sum 2^n >= 2^28 amplitudes, p = 2, <C> only, schedule chosen by the
    autotuner; amplitude-layers/s over the summed device time of every kernel,
    its fraction of the 16 B roofline, and the layer passes' own bandwidth
    against the measured HBM peak (n <= 14 stays on chip: no HBM roofline)."""
    import torch
    peak, _ = read_peaks()
    count = max(1, (1 << 28) >> n)
    sizes = [n] * min(count, 64)
    nv = int(sum(sizes) - (len(sizes) - 1))
    g = synth.erdos_renyi(nv, 0.3 if n < 24 else 0.2, 7, wmax=10)
    part = capi.paraqaoa_partition(capi.Graph.of(g), len(sizes), capi.PART_SIZES, sizes)
    ids = np.resize(np.arange(len(sizes), dtype=np.int32), count)
    gam, bet = synth.random_angles(count, 2, 11)
    tuned = capi.paraqaoa_autotune(ctx, part, 2).get(n) if n >= 15 else None
    capi.paraqaoa_simulate_batch(ctx, part, ids, 2, gam, bet, capi.SIM_EXPECT)  # warm-up
    capi.paraqaoa_expect(ctx, count)
    capi.paraqaoa_profile_enable(ctx, True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        capi.paraqaoa_simulate_batch(ctx, part, ids, 2, gam, bet, capi.SIM_EXPECT)
        capi.paraqaoa_expect(ctx, count)
    dt = time.perf_counter() - t0
    lp = capi.paraqaoa_profile_read(ctx, capi.KCLASS_LAYER_PASS)
    sm = capi.paraqaoa_profile_read(ctx, capi.KCLASS_SMEM_SIM)
    dev_ms = sum(capi.paraqaoa_profile_read(ctx, k)[1] for k in range(6))
    capi.paraqaoa_profile_enable(ctx, False)
    amp_layers = reps * count * (1 << n) * 2
    rate = amp_layers / (dev_ms / 1e3)
    line = {"qubits": n, "instances": count, "p": 2, "amp_layers_per_s": rate,
            "wall_amp_layers_per_s": amp_layers / dt, "roofline_frac_16B": rate * 16 / (peak * 1e9),
            "schedule": tuned}
    if lp[0]:
        gbs = lp[2] / (lp[1] / 1e3) / 1e9
        line.update({"layer_passes": int(lp[0] // reps), "layer_pass_gbs": gbs, "frac_of_measured_hbm": gbs / peak,
                     "hbm_bytes_per_amp_layer": lp[2] / amp_layers})
    else:
        line.update({"on_chip_ms": sm[1] / reps})
    capi.paraqaoa_part_free(part)
    return line


def run_sweep_case(args):
    import paper_2603_26232_gb300 as pkg
    from paper_2603_26232_gb300 import _capi as capi

    pkg.build()
    ctx = capi.paraqaoa_create(0)
    for n in range(args.sweep_lo, args.sweep_hi + 1):
        print(json.dumps(dict(case="sweep", **sweep_point(capi, ctx, n))), flush=True)
    capi.paraqaoa_destroy(ctx)


def run_shapes_case(args):
    """Every distinct layer-pass schedule (tile shape, contiguous run, form:
    classic or split, low or high group first; tiles per CTA) at
    n = sweep-lo..sweep-hi, on the sweep's batch
    (sum 2^n >= 2^28, p = 2, <C> only): the layer passes' summed event time
    per batch, their fraction of the 16 B roofline and their streamed bytes'
    fraction of the measured copy bandwidth; the 12 fastest per n."""
    import paper_2603_26232_gb300 as pkg
    from paper_2603_26232_gb300 import _capi as capi

    pkg.build()
    peak, _ = read_peaks()
    ctx = capi.paraqaoa_create(0)
    shapes = [(12, 5), (12, 4), (13, 5), (13, 4), (14, 4)]
    for n in range(args.sweep_lo, args.sweep_hi + 1):
        count = max(1, (1 << 28) >> n)
        sizes = [n] * min(count, 64)
        nv = int(sum(sizes) - (len(sizes) - 1))
        g = synth.erdos_renyi(nv, 0.3 if n < 24 else 0.2, 7, wmax=10)
        part = capi.paraqaoa_partition(capi.Graph.of(g), len(sizes), capi.PART_SIZES, sizes)
        ids = np.resize(np.arange(len(sizes), dtype=np.int32), count)
        gam, bet = synth.random_angles(count, 2, 11)
        rows, seen = [], set()
        for tb, r in shapes:
            for sp in (0, 1, 2, 3):  # schedule form bits: split, high group first
                for cm in (2, 3, 4):
                    for tpc in range(5):
                        try:
                            capi.paraqaoa_set_schedule(ctx, n, tb, r, cm, sp, tpc)
                        except capi.ParaQAOAError:
                            continue
                        sched = capi.paraqaoa_schedule(n, 2, tb, r, cm, sp)
                        key = (tb, r, sp, tuple((d["c"], d["s"]) for d in sched), tpc)
                        if key in seen:
                            continue
                        seen.add(key)
                        capi.paraqaoa_simulate_batch(ctx, part, ids, 2, gam, bet, capi.SIM_EXPECT)
                        capi.paraqaoa_expect(ctx, count)
                        capi.paraqaoa_profile_enable(ctx, True)
                        capi.paraqaoa_profile_classes(ctx, 1 << capi.KCLASS_LAYER_PASS)
                        for _ in range(3):
                            capi.paraqaoa_simulate_batch(ctx, part, ids, 2, gam, bet, capi.SIM_EXPECT)
                            capi.paraqaoa_expect(ctx, count)
                        lp = capi.paraqaoa_profile_read(ctx, capi.KCLASS_LAYER_PASS)
                        capi.paraqaoa_profile_enable(ctx, False)
                        capi.paraqaoa_profile_classes(ctx, 0xFFFFFFFF)
                        ms = lp[1] / 3
                        frac16 = count * (1 << n) * 2 * 16 / (ms / 1e3) / (peak * 1e9)
                        rows.append({"tile_bits": tb, "reg_bits": r, "split": sp, "c_min": cm, "tiles_per_cta_log2": tpc,
                                     "passes": len(sched), "ms": ms, "frac_16B": frac16,
                                     "pass_frac_of_copy": lp[2] / (lp[1] / 1e3) / 1e9 / peak})
        rows.sort(key=lambda x: x["ms"])
        print(json.dumps({"case": "shapes", "qubits": n, "instances": count, "p": 2, "fastest": rows[:12]}), flush=True)
        capi.paraqaoa_part_free(part)
    capi.paraqaoa_destroy(ctx)


def onchip_measure(capi, ctx, peaks):
    """Roofline of the on-chip kernel (states of 10..14 qubits held in
    registers and shared memory for all p layers): its flops and shared-memory
    bytes over its event time against the probed FP32 and shared-memory peaks.
    Per amplitude-layer it does n butterflies (one FFMA2, 4 flops, each) and a
    phase multiply (6 flops), and moves 16 B through shared memory per
    transpose: 2 transposes per layer (one at n = 10); <C> adds 3 flops per
    amplitude. Workloads: the 12..14-vertex parts of the batching
    configuration (G(2000, 0.05), p = 3) as they come, and 256 angle sets of
    each (the shape of a grid-search batch)."""
    fp32, smem = peaks
    g = synth.erdos_renyi(2000, 0.05, 0, wmax=1)
    sizes = synth.uneven_sizes(2000, 12, 24, 1)
    part = capi.paraqaoa_partition(capi.Graph.of(g), len(sizes), capi.PART_SIZES, sizes)
    small = np.flatnonzero((sizes >= 12) & (sizes <= 14)).astype(np.int32)
    out = {"fp32_peak_tflops": fp32, "smem_peak_tbs": smem, "parts": int(len(small))}
    for name, reps_ids in (("c3_parts", small), ("x256_angle_sets", np.repeat(small, 256))):
        ids = reps_ids.astype(np.int32)
        gam, bet = synth.random_angles(len(ids), 3, 5)
        capi.paraqaoa_simulate_batch(ctx, part, ids, 3, gam, bet, capi.SIM_EXPECT)
        capi.paraqaoa_expect(ctx, len(ids))
        capi.paraqaoa_profile_enable(ctx, True)
        reps = 5
        for _ in range(reps):
            capi.paraqaoa_simulate_batch(ctx, part, ids, 3, gam, bet, capi.SIM_EXPECT)
            capi.paraqaoa_expect(ctx, len(ids))
        n_l, ms, _ = capi.paraqaoa_profile_read(ctx, capi.KCLASS_SMEM_SIM)
        capi.paraqaoa_profile_enable(ctx, False)
        n = sizes[ids].astype(np.int64)
        amps = float(np.sum(np.left_shift(1, n)))
        flops = reps * float(np.sum(np.left_shift(1, n) * (3 * (4 * n + 6) + 3)))
        sbytes = reps * float(np.sum(np.left_shift(1, n) * 3 * np.where(n > 10, 32, 16)))
        sec = ms / 1e3
        out[name] = {"instances": int(len(ids)), "launches": int(n_l), "ms_per_batch": ms / reps,
                     "amp_layers_per_s": reps * amps * 3 / sec,
                     "tflops": flops / sec / 1e12, "frac_fp32": flops / sec / 1e12 / fp32,
                     "smem_tbs": sbytes / sec / 1e12, "frac_smem": sbytes / sec / 1e12 / smem}
    capi.paraqaoa_part_free(part)
    return out


def run_streams_case(args):
    """Plain HBM streams (write only, read only, copy) over 2 GiB buffers:
    the ceilings of the layer passes that only write or only read."""
    import paper_2603_26232_gb300 as pkg
    from paper_2603_26232_gb300 import _capi as capi

    pkg.build()
    peak, kind = read_peaks()
    w, r, c = capi.paraqaoa_probe_streams(0, 1 << 31)
    print(json.dumps({"case": "streams", "bytes": 1 << 31, "write_gbs": w, "read_gbs": r, "copy_gbs": c,
                      "hbm_gbs": peak, "hbm_gbs_source": kind}), flush=True)


def run_onchip_case(args):
    import paper_2603_26232_gb300 as pkg
    from paper_2603_26232_gb300 import _capi as capi

    pkg.build()
    peaks = capi.paraqaoa_probe_peaks(0)
    ctx = capi.paraqaoa_create(0)
    out = dict(case="onchip", **onchip_measure(capi, ctx, peaks))
    capi.paraqaoa_destroy(ctx)
    print(json.dumps(out), flush=True)


def run_merge_levels_case(args):
    """Level-aware merge at the paper's scale (Sec. 3.4.2; Sec. 4.2 runs 600
    vertices with K = 2 and L = 1..3): G(600, P), unit weights, seed 0, for
    P in 0.1 / 0.3 / 0.5 / 0.8, 24 parts of 25-26 vertices, the top-2 of each
    part from the p = 1 grid, and the exhaustive merge over all 2^24 paths
    with the GPU walk filled (at least 2^17 starting paths) for L = 1, 2, 3.
    The paper's worker scaling (K^L walkers, one GPU thread each, fill off) is
    timed on the first 12 parts of the P = 0.1 graph (4096 paths)."""
    import torch
    import paper_2603_26232_gb300 as pkg
    from paper_2603_26232_gb300 import _capi as capi

    pkg.build()
    solver = pkg.Solver()
    ctx = solver.ctx
    out = {"case": "merge_levels", "graphs": []}

    def timed_merge(G, part, cand, K, L, reps=3):
        capi.paraqaoa_merge(ctx, G, part, cand, K, L, 0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            side, cut = capi.paraqaoa_merge(ctx, G, part, cand, K, L, 0)
        return (time.perf_counter() - t0) / reps, int(cut), capi.paraqaoa_set_merge_fill(ctx, -1)

    for pe in (0.1, 0.3, 0.5, 0.8):
        g = synth.erdos_renyi(600, pe, 0, wmax=1)
        G = capi.Graph.of(g)
        M = 24
        part = capi.paraqaoa_partition(G, M)
        ids = np.arange(M, dtype=np.int32)
        gam, bet, _ = capi.paraqaoa_angle_search(ctx, part, ids, 1, 16, 0)
        _, cand, _ = capi.paraqaoa_final_topk(ctx, part, ids, 1, gam, bet, 2)
        row = {"graph": f"G(600,{pe})", "edges": g.num_edges, "parts": M, "K": 2, "paths": 2 ** M, "levels": []}
        for L in (1, 2, 3):
            dt, cut, used = timed_merge(G, part, cand, 2, L)
            row["levels"].append({"L": L, "starting_level_used": used, "s": dt, "cut": cut})
        out["graphs"].append(row)
        print(json.dumps(row), flush=True)
        if pe == 0.1:
            nv12 = 12 * 25 + 1
            g12 = synth.erdos_renyi(nv12, pe, 0, wmax=1)
            G12 = capi.Graph.of(g12)
            p12 = capi.paraqaoa_partition(G12, 12)
            ids12 = np.arange(12, dtype=np.int32)
            g1, b1, _ = capi.paraqaoa_angle_search(ctx, p12, ids12, 1, 16, 0)
            _, c12, _ = capi.paraqaoa_final_topk(ctx, p12, ids12, 1, g1, b1, 2)
            scal = []
            for fill in (0, 1):
                capi.paraqaoa_set_merge_fill(ctx, fill)
                for L in (1, 2, 3):
                    dt, cut, used = timed_merge(G12, p12, c12, 2, L)
                    scal.append({"fill": fill, "L": L, "gpu_walkers": 2 ** used, "s": dt, "cut": cut})
            capi.paraqaoa_set_merge_fill(ctx, 1)
            out["worker_scaling"] = {"graph": f"G({nv12},{pe})", "parts": 12, "K": 2, "paths": 4096, "runs": scal}
            print(json.dumps(out["worker_scaling"]), flush=True)
            capi.paraqaoa_part_free(p12)
        capi.paraqaoa_part_free(part)
    solver.close()
    print(json.dumps(out), flush=True)


def run_ksweep_case(args):
    """Top-K sweep (Sec. 4.2: cut and time against K) and the Performance
    Efficiency Index (Sec. 3.5: PEI = AR x EF x 100, EF = 1 / (1 + exp(alpha
    (T_ALG - T_Base))), alpha = 0.001 per second).
    (a) G(200, P), unit weights, seed 0, P in 0.1 / 0.3 / 0.5 / 0.8: 8 parts
    of 25-26 vertices, p = 1 grid, top-K, exhaustive merge, K = 1, 2, 4, 8;
    solve time and cut per K; AR against the best cut of the sweep (the
    paper's GW reference is out of scope), T_Base = the K = 1 solve.
    (b) G(n, P) for n = 20, 22, 24, 26 (the paper's small-scale sizes): two
    parts, K = 1, 4, 16; AR against the exact maximum cut, the largest entry
    of the whole graph's cut table (computed on the GPU, one part of n
    vertices)."""
    import torch
    import paper_2603_26232_gb300 as pkg
    from paper_2603_26232_gb300 import _capi as capi

    pkg.build()
    solver = pkg.Solver()
    out = {"case": "ksweep", "alpha_per_s": 1e-3, "sweep_200": [], "small_exact": []}
    for pe in (0.1, 0.3, 0.5, 0.8):
        g = synth.erdos_renyi(200, pe, 0, wmax=1)
        rows = []
        for K in (1, 2, 4, 8):
            cfg = pkg.SolveConfig(M=8, K=K, p=1, grid_points=16)
            solver.solve(g, cfg)  # warm-up
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = solver.solve(g, cfg)
            torch.cuda.synchronize()
            rows.append({"K": K, "s": time.perf_counter() - t0, "cut": int(r.cut)})
        best = max(x["cut"] for x in rows)
        for x in rows:
            x["ar_vs_best_of_sweep"] = x["cut"] / best
            x["ef"], x["pei"] = capi.paraqaoa_pei(x["ar_vs_best_of_sweep"], x["s"], rows[0]["s"], 1e-3)
        out["sweep_200"].append({"graph": f"G(200,{pe})", "edges": g.num_edges, "rows": rows})
        print(json.dumps(out["sweep_200"][-1]), flush=True)
    for n in (20, 22, 24, 26):
        for pe in (0.1, 0.3, 0.5, 0.8):
            g = synth.erdos_renyi(n, pe, 0, wmax=1)
            whole = capi.paraqaoa_partition(capi.Graph.of(g), 1)
            opt = int(capi.paraqaoa_cut_table(solver.ctx, whole, 0, n).max())
            capi.paraqaoa_part_free(whole)
            row = {"graph": f"G({n},{pe})", "opt": opt, "rows": []}
            for K in (1, 4, 16):
                t0 = time.perf_counter()
                r = solver.solve(g, pkg.SolveConfig(M=2, K=K, p=1, grid_points=16))
                dt = time.perf_counter() - t0
                ar = r.cut / opt if opt else 1.0
                ef, pei = capi.paraqaoa_pei(ar, dt, dt, 1e-3)
                row["rows"].append({"K": K, "s": dt, "cut": int(r.cut), "ar": ar, "pei_at_parity": pei})
            out["small_exact"].append(row)
            print(json.dumps(row), flush=True)
    solver.close()
    print(json.dumps(out), flush=True)


def run_halved_case(args):
    """Halved states (PARAQAOA_SIM_HALVED: z < 2^(n-1) stored, the top qubit's
    mixer fused into the low-group passes) against full states, on the
    sweep's batches (sum 2^n >= 2^28 amplitudes, p = 2, <C> only) for n = 20,
    22, 24, 26 and on one Adam batch of the paper-scale workload (168 x 2^20):
    amplitude-layers/s counting every one of the 2^n amplitudes (reported
    apart from the 16 B roofline metric: a halved state moves 8 B per
    amplitude-layer), the layer passes' streamed bytes per amplitude-layer and
    their fraction of the measured copy bandwidth, and the largest |d<C>| / W
    between the two forms."""
    import torch
    import paper_2603_26232_gb300 as pkg
    from paper_2603_26232_gb300 import _capi as capi

    pkg.build()
    peak, _ = read_peaks()
    ctx = capi.paraqaoa_create(0)
    cases = []
    for n in (20, 22, 24, 26):
        count = max(1, (1 << 28) >> n)
        sizes = [n] * min(count, 64)
        nv = int(sum(sizes) - (len(sizes) - 1))
        g = synth.erdos_renyi(nv, 0.3 if n < 24 else 0.2, 7, wmax=10)
        cases.append((f"{count} x G(*,{0.3 if n < 24 else 0.2}) parts of {n}", g, sizes,
                      np.resize(np.arange(len(sizes), dtype=np.int32), count), n))
    g400 = synth.erdos_renyi(NV, 0.1, 0, wmax=WMAX)
    cases.append(("168 x 2^20: 21 parts of G(400,0.1) x 8 angle sets", g400, None,
                  np.repeat(np.arange(M, dtype=np.int32), 8), 20))
    for name, g, sizes, ids, n in cases:
        part = (capi.paraqaoa_partition(capi.Graph.of(g), len(sizes), capi.PART_SIZES, sizes) if sizes
                else capi.paraqaoa_partition(capi.Graph.of(g), M))
        gam, bet = synth.random_angles(len(ids), 2, 13)
        W = np.array([max(1, int(w)) for w in capi.paraqaoa_part_info(part)[3][ids]], float)
        row = {"case": "halved", "workload": name, "qubits": n, "instances": int(len(ids)), "p": 2}
        res = {}
        for label, flags in (("full", 0), ("halved", capi.SIM_HALVED)):
            capi.paraqaoa_simulate_batch(ctx, part, ids, 2, gam, bet, capi.SIM_EXPECT | flags)
            capi.paraqaoa_expect(ctx, len(ids))
            capi.paraqaoa_profile_enable(ctx, True)
            reps = 3
            for _ in range(reps):
                capi.paraqaoa_simulate_batch(ctx, part, ids, 2, gam, bet, capi.SIM_EXPECT | flags)
                ex = capi.paraqaoa_expect(ctx, len(ids))
            lp = capi.paraqaoa_profile_read(ctx, capi.KCLASS_LAYER_PASS)
            dev_ms = sum(capi.paraqaoa_profile_read(ctx, k)[1] for k in range(6))
            capi.paraqaoa_profile_enable(ctx, False)
            amp_layers = reps * len(ids) * (1 << n) * 2
            res[label] = ex
            row[label] = {"amp_layers_per_s": amp_layers / (dev_ms / 1e3),
                          "layer_pass_bytes_per_amp_layer": lp[2] / amp_layers,
                          "layer_pass_frac_of_copy": lp[2] / (lp[1] / 1e3) / 1e9 / peak}
        row["speedup"] = row["halved"]["amp_layers_per_s"] / row["full"]["amp_layers_per_s"]
        row["max_dC_over_W"] = float(np.max(np.abs(res["halved"] - res["full"]) / W))
        print(json.dumps(row), flush=True)
        capi.paraqaoa_part_free(part)
    capi.paraqaoa_destroy(ctx)


def run_learned_case(args):
    """Learned-angle configuration: random subgraphs of 12..20 vertices from
    G(n, P), P in [0.05, 0.5], weights in {1..10} (and the same with unit
    weights), labelled by the plain form at p = 1..3; the 64-256-256-2p
    network trained on the GPU; on held-out subgraphs the <C> sum ratio to the
    plain form's angles of the prediction alone, of the best constant
    prediction (mean label) and of the judged learned form."""
    import torch
    import paper_2603_26232_gb300 as pkg
    from paper_2603_26232_gb300 import _capi as capi

    pkg.build()
    solver = pkg.Solver()
    ctx = solver.ctx
    ntr, nte, epochs = args.train_count, args.test_count, 60
    out = {"case": "learned", "train": ntr, "held_out": nte, "epochs": epochs, "results": []}
    for wmax in (10, 1):
        def make(count, seed):
            specs = synth.graph_specs(count, 12, 20, 0.05, 0.5, seed)
            G, sizes = synth.chain_of_graphs(specs, wmax=wmax)
            part = capi.paraqaoa_partition(capi.Graph.of(G), len(sizes), capi.PART_SIZES, sizes)
            return part, np.arange(len(sizes), dtype=np.int32)
        ptr, itr = make(ntr, 1)
        pte, ite = make(nte, 100000)
        Xtr = capi.paraqaoa_features(ctx, ptr, itr)
        Xte = capi.paraqaoa_features(ctx, pte, ite)
        for p in (1, 2, 3):
            t0 = time.perf_counter()
            gl, bl, _ = capi.paraqaoa_solve_plain(ctx, ptr, itr, p, STEPS_ADAM)
            t_label = time.perf_counter() - t0
            T = np.concatenate([gl, bl], axis=1).astype(np.float32)
            net = capi.paraqaoa_mlp_create(ctx, p, synth.mlp_init(p, 0))
            t0 = time.perf_counter()
            losses = capi.paraqaoa_mlp_train(net, Xtr, T, epochs, 256, 1e-3, synth.epoch_orders(ntr, epochs, 1))
            t_train = time.perf_counter() - t0
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            gp, bp, vp = capi.paraqaoa_solve_plain(ctx, pte, ite, p, STEPS_ADAM)
            t_plain = time.perf_counter() - t0
            t0 = time.perf_counter()
            gq, bq, vq, fb = capi.paraqaoa_solve_learned(ctx, pte, ite, net, p, STEPS_ADAM, 0.0)
            t_learned = time.perf_counter() - t0
            g0, b0 = capi.paraqaoa_mlp_predict(net, p, Xte)
            capi.paraqaoa_simulate_batch(ctx, pte, ite, p, g0, b0)
            v0 = capi.paraqaoa_expect(ctx, nte)
            rg, rb = capi.paraqaoa_mlp_reference(net, p)
            capi.paraqaoa_simulate_batch(ctx, pte, ite, p, np.tile(rg, (nte, 1)), np.tile(rb, (nte, 1)))
            vr = capi.paraqaoa_expect(ctx, nte)
            capi.paraqaoa_mlp_free(net)
            m = vp > 0
            r = {"weights": f"1..{wmax}", "p": p, "label_s": t_label, "train_s": t_train, "final_loss": float(losses[-1]),
                 "ratio_prediction": float(v0[m].sum() / vp[m].sum()),
                 "ratio_mean_label": float(vr[m].sum() / vp[m].sum()),
                 "ratio_learned_form": float(vq[m].sum() / vp[m].sum()),
                 "fallback_frac": float(np.mean(fb == 1)), "plain_s": t_plain, "learned_s": t_learned}
            out["results"].append(r)
            print(json.dumps(r), flush=True)
        capi.paraqaoa_part_free(ptr)
        capi.paraqaoa_part_free(pte)
    solver.close()
    print(json.dumps(out), flush=True)


def run_large_case(args):
    """16,000-vertex time-to-cut: G(16000, 0.01), unit weights, 640 parts of
    25-26 qubits (complex64 states of 256-512 MB, batched by the device-memory
    budget), p = 2, top-32, beam-64 merge. The learned form (network trained
    beforehand on small method-generated subgraphs, judge + plain fallback)
    against the plain form (grid + Adam + INTERP + Adam) on the same GPU."""
    import torch
    import paper_2603_26232_gb300 as pkg
    from paper_2603_26232_gb300 import _capi as capi

    pkg.build()
    free, total = torch.cuda.mem_get_info()
    solver = pkg.Solver(hbm_budget=int(0.6 * free))
    g = synth.erdos_renyi(LARGE_N, LARGE_P_EDGE, 0, wmax=1)
    G = capi.Graph.of(g)
    net, train_s, loss = train_large_model(capi, solver.ctx)
    out = {"case": "large", "workload": f"G({LARGE_N},{LARGE_P_EDGE}) unit weights, seed 0; {LARGE_M} parts of "
           f"25-26 qubits; p={LARGE_DEPTH}; top-{LARGE_K}; beam-{LARGE_BEAM}", "edges": g.num_edges,
           "train_s": train_s, "train_loss": loss}
    forms = [("learned", pkg.SolveConfig(M=LARGE_M, K=LARGE_K, p=LARGE_DEPTH, beam=LARGE_BEAM, mlp=net,
                                          fallback_steps=STEPS_ADAM, judge_tol=LARGE_JUDGE_TOL))]
    if not args.learned_only:
        forms.append(("plain", pkg.SolveConfig(M=LARGE_M, K=LARGE_K, p=LARGE_DEPTH, grid_points=GRID,
                                                adam_steps=STEPS_ADAM, beam=LARGE_BEAM)))
    for name, cfg in forms:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = solver.solve(G, cfg)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        out[name] = {"time_to_cut_s": dt, "cut": int(r.cut), "times": r.times,
                     "mean_expect": float(np.mean(r.expect))}
        if r.fallback is not None:
            out[name]["verdicts"] = {"network": int(np.sum(r.fallback == 0)), "plain_fallback": int(np.sum(r.fallback == 1)),
                                     "reference": int(np.sum(r.fallback == 2))}
        print(json.dumps(out), flush=True)
    if "plain" in out:
        out["cut_ratio"] = out["learned"]["cut"] / out["plain"]["cut"]
        out["expect_ratio"] = out["learned"]["mean_expect"] / out["plain"]["mean_expect"]
        out["speedup"] = out["plain"]["time_to_cut_s"] / out["learned"]["time_to_cut_s"]
    capi.paraqaoa_mlp_free(net)
    solver.close()
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--learned-only", action="store_true", help="large case: skip the plain form")
    ap.add_argument("--train-count", type=int, default=20000, help="learned case: training subgraphs")
    ap.add_argument("--test-count", type=int, default=2000, help="learned case: held-out subgraphs")
    ap.add_argument("--tc-k", type=int, default=6, help="tc case: mixer block qubits (5..7)")
    ap.add_argument("--sweep-lo", type=int, default=14)
    ap.add_argument("--sweep-hi", type=int, default=26)
    ap.add_argument("--case", default="solve", choices=["solve", "layer_pass", "large", "learned", "sweep",
                                                        "batching", "tc", "shapes", "onchip", "streams", "merge_levels",
                                                        "ksweep", "halved"],
                    help="layer_pass: only the p=2 <C> batch of one Adam step (168 x 2^20), "
                         "a small case for profiling the layer-pass kernel")
    ap.add_argument("--iters", type=int, default=3)
    ap.add_argument("--layer-p", type=int, default=2, help="layer_pass case: QAOA depth of the batch (1: the "
                                                             "grid batches' two half passes, 2: the Adam batches)")
    ap.add_argument("--layer-density", type=float, default=0.1, help="layer_pass case: edge probability of the "
                                                                     "400-vertex graph (0.1 or 0.5 in the workload)")
    ap.add_argument("--sched", default="", help="fixed schedule of the 20-qubit parts instead of the autotuner: "
                                                "tile_bits,reg_bits,c_min,split[,tiles_per_cta_log2]")
    ap.add_argument("--no-large", action="store_true", help="skip the 16k-vertex time-to-cut")
    ap.add_argument("--no-large-plain", action="store_true",
                    help="16k-vertex time-to-cut: the learned form only (the plain form takes minutes)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batching configuration and the n = 22 / 26 sweep points of the default line")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the context's default tile choice (fixed launch sequence for ncu)")
    ap.add_argument("--replicas", action="store_true",
                    help="N > 1: every rank solves its own copy of the workload (weak scaling) instead of "
                         "one workload sharded across the ranks")
    ap.add_argument("--oracle-sample", type=float, default=0.0,
                    help="print one oracle CPU-baseline sample of about this many seconds and exit")
    args = ap.parse_args()
    if args.oracle_sample > 0:
        print(json.dumps(cpu_baseline(args.oracle_sample)), flush=True)
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.case == "layer_pass":
        return run_layer_case(args)
    if args.case == "large":
        return run_large_case(args)
    if args.case == "learned":
        return run_learned_case(args)
    if args.case == "sweep":
        return run_sweep_case(args)
    if args.case == "batching":
        return run_batching_case(args)
    if args.case == "tc":
        return run_tc_case(args)
    if args.case == "shapes":
        return run_shapes_case(args)
    if args.case == "onchip":
        return run_onchip_case(args)
    if args.case == "streams":
        return run_streams_case(args)
    if args.case == "merge_levels":
        return run_merge_levels_case(args)
    if args.case == "ksweep":
        return run_ksweep_case(args)
    if args.case == "halved":
        return run_halved_case(args)

    import torch
    import paper_2603_26232_gb300 as pkg
    from paper_2603_26232_gb300 import _capi as capi

    pkg.build()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    cb = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = cpu_baseline()  # before the first GPU call of the timed work
        cb["one_core"] = cpu_baseline_one_core()
    stream = torch.cuda.Stream()
    solver = pkg.Solver(device=local)
    capi.paraqaoa_set_stream(solver.ctx, stream.cuda_stream)
    sharded = world > 1 and not args.replicas
    graphs = workload(0 if sharded else rank)
    Gs = [capi.Graph.of(g) for g in graphs]
    cfg = pkg.SolveConfig(M=M, K=K, p=P_FINAL, grid_points=GRID, adam_steps=STEPS_ADAM, beam=BEAM)
    # tile size per qubit count, measured once on this GPU (outside the timed region)
    # schedule of the 20-qubit parts per graph (the two densities have different
    # phase-table sizes and cut structure), measured once on this GPU outside
    # the timed region, or fixed (e.g. to repeat a tuned run's launches under a profiler)
    sched = []
    for G in Gs:
        if args.sched:
            sc = tuple(int(x) for x in args.sched.split(","))
            sched.append(sc + (0,) * (5 - len(sc)))
        else:
            part = capi.paraqaoa_partition(G, M)
            sched.append(capi.paraqaoa_autotune(solver.ctx, part, P_FINAL)[20])
            capi.paraqaoa_part_free(part)

    if sharded:
        from paper_2603_26232_gb300 import sharded as shard
        part_solver, merger = shard.cuda_part_solver(solver.ctx, cfg), shard.cuda_merger(solver.ctx, cfg)

    def step():
        out = []
        for G, sc in zip(Gs, sched):
            capi.paraqaoa_set_schedule(solver.ctx, 20, *sc)
            if sharded:
                out.append(shard.solve_sharded(dist, G, cfg, part_solver, merger, device="cuda"))
            else:
                out.append(solver.solve(G, cfg))
        return out

    for _ in range(max(3, args.warmup)):
        res = step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    # the headline: the product mode (size classes on side streams, Adam
    # steps replayed from a CUDA graph, no event brackets), device time
    # between two events on the context's stream
    clocks = Clocks(local)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        ev0.record(stream)
        for _ in range(args.steps):
            res = step()
        ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    clk = clocks.stop()
    # the roofline's kernel in a separate pass of the same steps: every
    # layer-pass launch bracketed by CUDA events on its stream (profiling
    # runs the size classes in order and the Adam steps launch by launch);
    # the other kernel classes are counted, not timed
    prof_steps = max(1, min(args.steps, 5))
    capi.paraqaoa_profile_enable(solver.ctx, True)
    capi.paraqaoa_profile_classes(solver.ctx, 1 << capi.KCLASS_LAYER_PASS)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        for _ in range(prof_steps):
            step()
    torch.cuda.synchronize()
    prof = {k: capi.paraqaoa_profile_read(solver.ctx, k) for k in range(6)}
    capi.paraqaoa_profile_enable(solver.ctx, False)
    capi.paraqaoa_profile_classes(solver.ctx, 0xFFFFFFFF)
    # end to end through the public API with host buffers: partition, upload,
    # every host<->device copy and the merge readback inside the timed region
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for G in Gs:
            part = capi.paraqaoa_partition(G, M)
            capi.paraqaoa_part_upload(solver.ctx, part, True)
            capi.paraqaoa_part_free(part)
        step()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    ms, e2e_s = max_over_ranks([ms, e2e_s], dist, "cuda")
    large = batching = sweep = halved_step = None
    if rank == 0 and not args.no_extras:
        # the batching configuration and two points of the amplitude-layer
        # sweep, on a context of their own (their autotuning leaves the
        # solver's schedules alone)
        xctx = capi.paraqaoa_create(local)
        try:
            batching = batching_measure(capi, xctx)
            sweep = [sweep_point(capi, xctx, n) for n in (22, 26)]
        finally:
            capi.paraqaoa_destroy(xctx)
        # the same step on halved states (a separate metric: 8 B per
        # amplitude-layer instead of the 16 B the roofline counts)
        hsolver = pkg.Solver(device=local, halved=True)
        capi.paraqaoa_set_stream(hsolver.ctx, stream.cuda_stream)
        try:
            def hstep():
                out = []
                for G, sc in zip(Gs, sched):
                    capi.paraqaoa_set_schedule(hsolver.ctx, 19, *sc)  # halved 20-qubit parts hold 19 qubits
                    out.append(hsolver.solve(G, cfg))
                return out
            for _ in range(2):
                hstep()
            torch.cuda.synchronize()
            hev0, hev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                hev0.record(stream)
                for _ in range(args.steps):
                    hres = hstep()
                hev1.record(stream)
            torch.cuda.synchronize()
            hms = hev0.elapsed_time(hev1)
            halved_step = {"metric": "amplitude-layers/s on halved states (z < 2^(n-1) stored, 8 B per amplitude-layer)",
                           "value": job_value(amp_layers_per_graph() * len(graphs), args.steps, 1, hms),
                           "ms_per_step": hms / args.steps, "speedup_over_full": ms / hms,
                           "cuts": [int(r.cut) for r in hres]}
        finally:
            hsolver.close()
    if rank == 0 and not args.no_large:
        large = large_learned(capi, pkg, plain=not args.no_large_plain)
    amps_step = amp_layers_per_graph() * len(graphs)
    copies = 1 if sharded else world  # sharded: one workload in all; replicas: one per rank
    value = job_value(amps_step, args.steps, copies, ms)
    e2e_value = job_value(amps_step, args.steps, copies, e2e_s * 1e3)
    launches, lp_ms, lp_bytes = prof[capi.KCLASS_LAYER_PASS]
    peak, peak_kind = read_peaks()
    achieved = (lp_bytes / (lp_ms / 1e3)) / 1e9 if lp_ms > 0 else 0.0
    traffic = traffic_for(LAYER_PASS_SOURCES, lp_bytes / max(launches, 1))
    # the kernels of a step are the same in both modes (graph replay repeats
    # the captured step's launches): launches per profiled step x timed steps
    total_launches = sum(v[0] for v in prof.values()) * args.steps // prof_steps
    h2d = sum(int(G.row_ptr.nbytes + G.col.nbytes + G.w.nbytes) for G in Gs)
    d2h = len(Gs) * (M * K * 8 + NV + M * 8 * 3)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "strong" if sharded else "weak", "vs_baseline": None, "dtype": "c64/f32 state, f64 <C>",
            "data": "synthetic (seeded Erdos-Renyi graphs)",
            "config": dict(config_dict(), parallelism=(f"parts sharded over {world} ranks (LPT), candidates "
                                                       "reduced to rank 0, merge on rank 0") if sharded else
                           (f"{world} replicas" if world > 1 else "1 GPU")),
            "time_to_cut_s": (ms / 1e3) / args.steps / len(graphs),
            "cuts": [int(r.cut) for r in res],
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak if peak else None, "traffic": traffic,
                         "kernel": "k_layer_pass (HBM-streaming layer pass)",
                         "launches": launches, "avg_launch_ms": lp_ms / max(launches, 1),
                         "algorithmic_bytes_per_launch": lp_bytes / max(launches, 1),
                         "peak_source": f"{peak_kind} hbm_gbs"},
            "layer_pass_share": (lp_ms / prof_steps) / (ms / args.steps) if ms else None,
            "roofline_pass": {"steps": prof_steps, "mode": "profiled (layer passes bracketed by CUDA events)"},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": int(total_launches),
            "clocks": clk,
            "schedule_20_qubits": [{"graph": f"G({NV},{pe})", "tile_bits": sc[0], "reg_bits": sc[1],
                                    "min_run_qubits": sc[2], "split": sc[3], "tiles_per_cta_log2": sc[4]}
                                   for pe, sc in zip(DENSITIES, sched)],
            "cpu_baseline": cb,
            "time_to_cut_16k": large,
            "batching": batching,
            "sweep": sweep,
            "halved_step": halved_step,
        }
        print(json.dumps(line), flush=True)
    solver.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
