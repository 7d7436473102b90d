#!/usr/bin/env python
"""Benchmark of the IPC time step (Eq. 3) on B300: steps/s.

One "step" is one call of sim_step: the whole Newton solve of one time step
of the workload (culling, assembly, PCG, CCD, line search).  The sampled steps
are spread over the trajectory; one untimed pass runs it and saves the state
before each of them, and each is then replayed from its state (a restarted
step is bit-identical to the step in the trajectory).  Inputs live in HBM;
before each timed step the L2 is flushed by writing a 256 MB buffer outside
the timed events.  Each step is timed with CUDA events on the simulator's
stream; `value` = steps / sum of step times (max over ranks for N > 1, each
rank running its own replica of a single scene, or its own shard of a batch).

Without a cached PCG launch shape, a single-scene workload first times every
shape over the same replayed steps and keeps the fastest total.

`e2e` replays the same steps through the public API with host buffers: the
kinematic transforms go host -> device and the positions come back to host
memory every step, inside the timed region.

`--impl reference` times the plain FP64 CPU oracle on the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "IPC sim steps/s at 1e-5 rel pos error (plain FP64 vs batched/mixed); adjoint ms/step"
UNIT = "steps/s"


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0}, "fallback"


def make_workload(name):
    from paper_2609_25653_b300 import scenes
    if name == "fingertip_press":
        # the plate keeps pressing at 0.1 mm per step; 60 steps cover warm-up, timed and e2e steps
        return scenes.fingertip_press(0, n_steps=60)
    if name == "arm_gripper":
        return scenes.arm_gripper_grasp(0)
    if name == "soft_cylinder":
        # fingertips squeeze a deformable 63k-tet cylinder; the timed steps sit in the contact-rich squeeze
        return scenes.soft_gripper_cylinder(0, n_steps=300, close_per_step=0.25e-3)
    if name.startswith("batched"):
        # "batched" = 64 scenes, "batched16" = 16 scenes, ...
        n = int(name[len("batched"):] or 64)
        return scenes.batched_grasps(n)
    raise SystemExit(f"unknown workload {name}")


def workload_config(wl, name, extra=None):
    scs = wl if isinstance(wl, list) else [wl]
    sc = scs[0]
    cfg = {"workload": sc["name"] if len(scs) == 1 else f"batched_grasps_{len(scs)}scenes",
           "scenes": len(scs), "fem_tets": int(sum(len(s["fem_tets"]) for s in scs)),
           "fem_verts": int(sum(len(s["fem_X"]) for s in scs)),
           "kinematic_bodies": sum(len(s.get("kin", [])) for s in scs), "abd_bodies": sum(len(s.get("abd", [])) for s in scs),
           "dt": sc["params"]["dt"], "dhat": sc["params"]["dhat"], "mu": sc["params"]["mu"],
           "newton_tol": sc["params"]["newton_tol"], "pcg_rtol": sc["params"]["pcg_rtol"],
           "l2": "flushed between timed steps (256 MB write outside the timed events)"}
    if extra:
        cfg.update(extra)
    return cfg


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.gpu = gpu_index
        self.proc = None
        # raw samples (the JSON line carries their summary); BENCH_CLOCKS_DIR keeps them somewhere else
        out_dir = os.environ.get("BENCH_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, f"clocks_bench_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def pcg_work(work, sim, fp32, launches, coarse_n=0):
    """Algorithmic work of the PCG kernel per launch: (bytes, flops), from the per-unit figures of the
    method's solve, independent of how the kernel is built.

    Per iteration: the operator product reads every stored 3x3 block once (9 values + a 4 B column index:
    76 B in FP64, 40 B in FP32) and takes 18 flops per block; the CG vectors move 7 values per DOF
    (56 B in FP64, 28 B in FP32) and take 10 flops per DOF, the block-Jacobi preconditioner 6 flops per
    DOF; every active barrier pair's 12x12 block (144 values + its 32 B record) takes 288 flops, every
    friction pair's 3x3 block, ids and weights (9 values + 48 B) about 60 flops.  The mixed-precision
    solver's inner iterations are FP32: its figures use 4-byte values.  The two-level preconditioner adds,
    per iteration, the product with the dense coarse inverse (n_c x n_c values read once, 2 n_c^2 flops,
    n_c = 6 x aggregates) and the restriction and prolongation (36 flops per FEM DOF)."""
    e = 4 if fp32 else 8
    it = work["pcg_iters"]
    ndof = 3 * sim.n_nodes
    per_it_bytes = work["bsr_blocks"] * (9 * e + 4) + ndof * 7 * e + coarse_n * coarse_n * e
    per_it_flops = work["bsr_blocks"] * 18 + ndof * 16 + 2 * coarse_n * coarse_n + 36 * 3 * sim.nf * (coarse_n > 0)
    total_bytes = it * per_it_bytes + work["pcg_pair_iters"] * (144 * e + 32) + work["pcg_fric_iters"] * (9 * e + 48)
    total_flops = it * per_it_flops + work["pcg_pair_iters"] * 288 + work["pcg_fric_iters"] * 60
    n = max(launches, 1)
    return total_bytes / n, total_flops / n


def pcg_traffic(kernel, workload):
    """DRAM bytes per launch of the PCG kernel from the committed ncu summary, or None when the kernel's
    source has changed since that capture (the summary records the hash of the source it measured)."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "pcg_traffic.json")) as f:
            rec = json.load(f)
    except Exception:
        return None
    src = os.path.join(ROOT, "paper_2609_25653_b300", "csrc", "pcg.cu")
    with open(src, "rb") as f:
        sha = hashlib.sha256(f.read()).hexdigest()[:16]
    for r in rec.get("captures", []):
        if r.get("kernel") == kernel and r.get("workload") == workload and r.get("pcg_cu_sha16") == sha:
            return r.get("dram_bytes_per_launch")
    return None


def slowest_rank(local, device="cuda"):
    """The largest of every rank's value (a timed total), after which all ranks hold it; with one rank, or
    without an initialised process group, the local value."""
    try:
        import torch.distributed as dist
        if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
            return float(local)
    except ImportError:
        return float(local)
    import torch
    t = torch.tensor([float(local)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(t.item())


def timed_indices(n_traj, warmup, steps, sample):
    """Trajectory steps to time: `steps` steps spread evenly over the trajectory after the warm-up
    ("trajectory"), or the `steps` steps right after it ("consecutive")."""
    first = warmup
    room = n_traj - first
    if room < steps:
        raise SystemExit("workload trajectory too short for the requested steps")
    if sample == "consecutive":
        return list(range(first, first + steps))
    if steps == 1:
        return [first]
    return [first + round(j * (room - 1) / (steps - 1)) for j in range(steps)]


def run_ours(args):
    import numpy as np
    import torch
    from paper_2609_25653_b300 import ipcsim

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    wl = make_workload(args.workload)
    batched = isinstance(wl, list)
    if batched and world > 1:
        # independent scenes shard across ranks with no collective: rank r takes scenes r, r + N, ...
        wl = shard_scenes(wl, rank, world)
    precision = args.precision or ("mixed" if batched else "fp64")
    prec = ipcsim.PREC_MIXED if precision == "mixed" else ipcsim.PREC_FP64
    over = {"coarse_rebuild": args.coarse_rebuild,
            "preconditioner": ipcsim.PRECOND_BLOCK_JACOBI if args.preconditioner == "block-jacobi"
            else ipcsim.PRECOND_TWO_LEVEL}
    if batched:
        sim = ipcsim.Simulator.batch(wl, precision=prec, stream=stream, **over)
        sc = sim.scene
    else:
        sc = wl
        sim = ipcsim.Simulator(sc, precision=prec, stream=stream, **over)
    n_sc = len(wl) if batched else 1
    n_traj = sc["kin_T"].shape[0] - 1 if len(sc.get("kin", [])) else sc["params"]["n_steps"]
    timed = timed_indices(n_traj, args.warmup, args.steps, args.sample)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    peaks_dev = ipcsim.device_peaks()  # FP64 / FP32 FMA roofs of this device, measured before the timed region
    from paper_2609_25653_b300 import autotune
    # launch shape: a cached choice; else, for one scene, every shape timed over the sampled steps
    # (replayed from their saved states, below); for a batch (whose steps are too long to replay eight
    # times), every shape timed on the first linear system of the first warm-up step
    tuned_from_cache = autotune.cached(sim, prec) if not args.no_autotune else None
    tune_replay = tuned_from_cache is False and not batched
    if tuned_from_cache is False and batched:
        sim.tuning(autotune_next_step=True)
    for w in range(args.warmup):
        sim.step()
        if w == 0 and tuned_from_cache is False and batched:
            autotune.record(sim, prec)
    # the trajectory, untimed, saving the state before every sampled step
    snaps = []
    for s_idx in timed:
        while sim.step_index < s_idx:
            sim.step()
        snaps.append((sim.get_state(), sim.step_index))
        sim.step()
    end_state, end_index = sim.get_state(), sim.step_index

    def restore(j):
        state, idx = snaps[j]
        sim.set_state(*state)
        if sim.nkb:
            sim.set_kinematic(sc["kin_T"][idx])
        sim.step_index = idx

    def replay(j):
        restore(j)
        with torch.cuda.stream(stream):
            flush.fill_(1.0)
        stream.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = sim.step()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1), st

    tune_ms = None
    if tune_replay:
        _, tune_ms = autotune.tune_on_steps(sim, lambda j: replay(j)[0], len(snaps))
        autotune.record(sim, prec, ms=tune_ms)
    (rowg, bps), _ = sim.tuning()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    # the timed pass: every sampled step replayed from its saved state (the same work as in the
    # trajectory: a restarted step is bit-identical), L2 flushed before each
    sim.profile(True)
    times, stats = [], []
    launches = 0
    with ClockSampler(local) as clk:
        for j in range(len(snaps)):
            l0 = ipcsim.kernel_launches()
            ms, st = replay(j)
            launches += ipcsim.kernel_launches() - l0
            times.append(ms)
            stats.append(st)
    torch.cuda.synchronize()
    prof, work = sim.profile_read()
    sim.profile(False)
    total_ms = slowest_rank(sum(times))
    value = world * args.steps * n_sc / (total_ms / 1e3)

    # e2e through the public API with host buffers (transforms in, positions out), the same sampled steps

    x_host = np.zeros((sim.nf, 3))
    T_pinned = torch.empty((max(sim.nkb, 1), 12), dtype=torch.float64).pin_memory()
    e2e_s = 0.0
    e2e_steps_ms = []
    for j in range(len(timed)):
        restore(j)
        torch.cuda.synchronize()
        T_host = T_pinned.numpy()
        T_host[:sim.nkb] = sc["kin_T"][sim.step_index + 1].reshape(-1, 12) if sim.nkb else 0.0
        t1 = time.perf_counter()
        sim.step(T_host[:sim.nkb].reshape(-1, 3, 4) if sim.nkb else None)
        x_host[:] = sim.get_state()[0]
        dt_s = time.perf_counter() - t1
        e2e_s += dt_s
        e2e_steps_ms.append(round(dt_s * 1e3, 2))
    print("e2e step ms:", e2e_steps_ms, file=sys.stderr)

    # adjoint ms/step: the backward of the same sampled steps (unprojected Hessian re-assembly at the
    # checkpointed end state, FP64 adjoint solve, parameter contractions)
    adjoint = None
    if not batched and not args.no_adjoint:
        gen = torch.Generator(device="cuda").manual_seed(0)
        glogE = torch.zeros(sim.nt, dtype=torch.float64, device="cuda")
        adj_ms = []
        for j in range(len(timed)):
            restore(j)
            z0, zd0 = sim.get_dofs()
            k0 = sim.step_index
            sim.step()
            z1, _ = sim.get_dofs()
            gz = torch.randn(sim.ndof, dtype=torch.float64, device="cuda", generator=gen)
            gzd = 1e-2 * torch.randn(sim.ndof, dtype=torch.float64, device="cuda", generator=gen)
            torch.cuda.synchronize()
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            sim.adjoint(z0, zd0, z1, sc["kin_T"][k0], sc["kin_T"][k0 + 1], gz, gzd, glogE)
            a1.record(stream)
            a1.synchronize()
            adj_ms.append(a0.elapsed_time(a1))
        adjoint = {"ms_per_step": round(sum(adj_ms) / len(adj_ms), 3), "steps": len(adj_ms),
                   "solve": "FP64 PCG on the unprojected Hessian, rtol 1e-12"}
    e2e_s = slowest_rank(e2e_s)
    e2e_value = world * args.steps * n_sc / e2e_s

    # accuracy gate of a batch: the first --gate scenes simulated alone in FP64 over the same steps
    gate = None
    if batched and args.gate > 0:
        xb = end_state[0]
        errs = []
        off = 0
        for k, scn in enumerate(wl):
            nfk = len(scn["fem_X"])
            if k < args.gate:
                single = ipcsim.Simulator(scn, stream=stream)
                for _ in range(end_index):
                    single.step()
                xs = single.get_state()[0]
                errs.append(float(np.max(np.abs(xb[off:off + nfk] - xs)) / single.L))
                single.close()
            off += nfk
        gate = {"scenes": len(errs), "reference": "each scene alone, FP64, same steps",
                "max_rel_pos_err": max(errs), "rel_pos_err": [float("%.3g" % e) for e in errs],
                "within_1e-5": bool(max(errs) < 1e-5)}

    # roofline of the dominant kernel (the PCG solve), from its algorithmic work per launch and its
    # CUDA-event time per launch on the simulator's stream
    peaks, peak_src = load_peaks()
    dom = max(prof, key=lambda k: prof[k]["ms"])
    pcg = prof["pcg"]
    fp32 = prec == ipcsim.PREC_MIXED
    pcg_avg_ms = pcg["ms"] / max(pcg["n"], 1)
    pcg_grid, pcg_resident = sim.pcg_layout()
    coarse_n = sim.coarse_size() if sim.params.get("preconditioner", ipcsim.PRECOND_TWO_LEVEL) == ipcsim.PRECOND_TWO_LEVEL else 0
    b_launch, f_launch = pcg_work(work, sim, fp32, pcg["n"], coarse_n)
    alu_peak = peaks_dev["fp32_tflops"] if fp32 else peaks_dev["fp64_tflops"]
    t_mem = b_launch / (peaks["hbm_gbs"] * 1e9)
    t_alu = f_launch / (alu_peak * 1e12)
    kernel = "k_pcg32" if fp32 else "k_pcg"
    gbs = b_launch / (pcg_avg_ms / 1e3) / 1e9 if pcg["n"] else 0.0
    tfs = f_launch / (pcg_avg_ms / 1e3) / 1e12 if pcg["n"] else 0.0
    if t_alu > t_mem:
        bound = {"bound": "alu", "achieved": round(tfs, 5), "peak": round(alu_peak, 4), "unit": "TFLOP/s",
                 "frac": round(tfs / alu_peak, 5)}
    else:
        bound = {"bound": "hbm", "achieved": round(gbs, 2), "peak": peaks["hbm_gbs"], "unit": "GB/s",
                 "frac": round(gbs / peaks["hbm_gbs"], 5)}
    roofline = dict(bound, traffic=pcg_traffic(kernel, sc["name"] if not batched else f"batched{n_sc}"),
                    kernel=kernel,
                    peak_source=("FP64 FMA rate measured in this run (sim_device_peaks)" if bound["bound"] == "alu"
                                 and not fp32 else "FP32 FMA rate measured in this run (sim_device_peaks)"
                                 if bound["bound"] == "alu" else f"HBM copy bandwidth, {peak_src} (MEASURED_PEAKS.json)"),
                    hbm={"achieved_gbs": round(gbs, 2), "peak_gbs": peaks["hbm_gbs"],
                         "frac": round(gbs / peaks["hbm_gbs"], 5)},
                    alu={"achieved_tflops": round(tfs, 5), "peak_tflops": round(alu_peak, 4),
                         "frac": round(tfs / alu_peak, 5), "pipe": "fp32" if fp32 else "fp64"},
                    launch_ms=round(pcg_avg_ms, 5), algorithmic_bytes_per_launch=int(b_launch),
                    algorithmic_flops_per_launch=int(f_launch),
                    pcg_iterations_per_launch=round(work["pcg_iters"] / max(pcg["n"], 1), 1),
                    pcg_ctas=pcg_grid, operator_in_shared_memory=pcg_resident, dominant_stage=dom,
                    preconditioner="two-level" if coarse_n else "block Jacobi", coarse_unknowns=coarse_n,
                    stage_ms_per_step={k: round(v["ms"] / args.steps, 4) for k, v in prof.items() if v["n"]})
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the oracle advances one scene at a time: scene-steps/s of the first scene of a batch
        cpu = cpu_baseline(wl[0] if batched else sc, args.cpu_seconds, sum(s["newton_iters"] for s in stats) / len(stats))
    clocks = clk.summary()
    if rank == 0:
        newton = [s["newton_iters"] for s in stats]
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if precision == "fp64" else "f64+f32",
            "data": "synthetic",
            "config": workload_config(wl, args.workload, {
                "parallelism": (f"scene-shards{world}" if batched and world > 1 else f"replicas{world}"),
                "precision": precision,
                "preconditioner": args.preconditioner, "coarse_rebuild": args.coarse_rebuild,
                "value_counts": "scene-steps" if batched else "steps",
                "timed_steps": timed if args.sample == "consecutive" or len(timed) <= 40 else f"{timed[0]}..{timed[-1]}",
                "timed_sample": ("every step after the warm-up, each replayed from its saved state" if args.sample == "consecutive" else
                                 f"{len(timed)} steps spread over the {n_traj}-step trajectory, each replayed "
                                 "from its state saved in one untimed pass"),
                "pcg_threads_per_row": rowg, "pcg_blocks_per_sm": bps,
                "pcg_shape": "cached" if tuned_from_cache else (("autotuned over the sampled steps" if tune_replay else
                                                                  "autotuned on the first linear system")
                                                                 if tuned_from_cache is False else "default"),
                "pcg_shape_ms": [round(m, 2) for m in tune_ms] if tune_ms else None,
                "newton_iters_per_step": round(sum(newton) / len(newton), 2),
                "pcg_iters_per_step": round(sum(s["pcg_iters_total"] for s in stats) / len(stats), 1),
                "pcg_unconverged_solves": int(sum(s["pcg_unconverged"] for s in stats)),
                "pcg_two_level_fallbacks": int(sum(s["pcg_fallbacks"] for s in stats)),
                "active_pairs_max": max(s["n_pairs_max"] for s in stats)}),
            "roofline": roofline,
            "cpu_baseline": cpu,
            "adjoint": adjoint,
            "accuracy_gate": gate,
            "e2e": {"value": round(e2e_value, 3), "unit": UNIT, "h2d_bytes_per_step": 96 * sim.nkb,
                    "d2h_bytes_per_step": 24 * sim.nf},
            "gpu_launches": int(launches),
            "clocks": clocks,
            "device_peaks_tflops": {k: round(v, 4) for k, v in peaks_dev.items()},
        }
        print(json.dumps(line))
    sim.close()
    if world > 1:
        dist.destroy_process_group()


def run_material_id(args):
    """Differentiable material identification at full size (about 100k tets): a forward rollout of
    `--id-steps` steps with per-tet ln E and mu as parameters, the loss sum_t 1/2 |x_t - x*_t|^2 against a
    target trajectory simulated with hidden parameters, its backward through the implicit adjoint of every
    step (timed: adjoint ms/step), and the gradient against central differences of the GPU forward on 16
    random parameter directions over the first `--fd-steps` steps."""
    import numpy as np
    import torch
    from paper_2609_25653_b300 import autograd, ipcsim, scenes
    torch.cuda.set_device(0)
    n = args.id_steps
    sc = scenes.material_identification(0, n_steps=max(n, args.fd_steps) + 1)
    sim = ipcsim.Simulator(sc)
    z0, zd0 = sim.get_dofs()
    logE0 = torch.tensor(sc["fem_logE"], dtype=torch.float64)
    hidden = torch.tensor(sc["hidden_logE"], dtype=torch.float64)
    t0 = time.perf_counter()
    with torch.no_grad():
        target = [t.detach() for t in autograd.rollout(sim, hidden, sc["hidden_mu"], n, z0, zd0)]
    t_target = time.perf_counter() - t0

    def loss_of(traj):
        return sum(0.5 * torch.sum((x - t) ** 2) for x, t in zip(traj, target))

    logE = logE0.clone().requires_grad_(True)
    mu = torch.tensor(0.6, dtype=torch.float64, requires_grad=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    traj = autograd.rollout(sim, logE, mu, n, z0, zd0)
    L = loss_of(traj)
    torch.cuda.synchronize()
    t_fwd = time.perf_counter() - t0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    L.backward()
    e1.record()
    e1.synchronize()
    adj_ms = e0.elapsed_time(e1) / n
    # central differences over the first fd_steps steps, 16 random directions (ln E: 14, mu: 2), on a
    # simulator with tight Newton and PCG tolerances (the implicit function theorem assumes converged
    # steps, and the differences must resolve loss changes far below the default tolerances)
    m = args.fd_steps
    sim.close()
    sim = ipcsim.Simulator(sc, newton_tol=1e-10, pcg_rtol=1e-12, max_newton=300)
    with torch.no_grad():
        target = [t.detach() for t in autograd.rollout(sim, hidden, sc["hidden_mu"], m, z0, zd0)]

    def loss_short(le, mu_v):
        with torch.no_grad():
            tr = autograd.rollout(sim, le, mu_v, m, z0, zd0)
            return float(sum(0.5 * torch.sum((x - t) ** 2) for x, t in zip(tr, target[:m])))

    le = logE0.clone().requires_grad_(True)
    muv = torch.tensor(0.6, dtype=torch.float64, requires_grad=True)
    Ls = sum(0.5 * torch.sum((x - t) ** 2) for x, t in
                             zip(autograd.rollout(sim, le, muv, m, z0, zd0), target[:m]))
    Ls.backward()
    g_le, g_mu = le.grad.numpy(), float(muv.grad)
    r = np.random.default_rng(2)
    errs = []
    for k in range(16):
        if k < 14:
            d = r.normal(size=g_le.shape)
            d /= np.linalg.norm(d)
            h = 1e-4
            fd = (loss_short(logE0 + h * torch.as_tensor(d), 0.6) - loss_short(logE0 - h * torch.as_tensor(d), 0.6)) / (2 * h)
            ad = float(g_le @ d)
        else:
            h = 1e-5
            fd = (loss_short(logE0, 0.6 + h) - loss_short(logE0, 0.6 - h)) / (2 * h)
            ad = g_mu
        errs.append(abs(fd - ad) / max(abs(fd), 1e-300))
    line = {"workload": sc["name"], "fem_tets": len(sc["fem_tets"]), "steps": n, "precision": "fp64",
            "adjoint_ms_per_step": round(adj_ms, 3), "forward_ms_per_step": round(1e3 * t_fwd / n, 3),
            "target_forward_s": round(t_target, 2), "loss": float(L),
            "fd_check": {"directions": 16, "steps": m, "tolerances": "newton 1e-10, pcg 1e-12",
                         "max_rel_err": float(max(errs)),
                         "rel_errs": [float("%.3g" % e) for e in errs]},
            "grad_norm_logE": float(np.linalg.norm(logE.grad.numpy())), "grad_mu": float(mu.grad)}
    print(json.dumps(line))


def run_render(args):
    """Frames/s of the path tracer (640 x 360, 32 paths per pixel, 2 bounces, 8 shadow samples for Eq. 7)
    on the arm-gripper grasp after --warmup steps, timed with CUDA events over --steps frames."""
    import numpy as np
    import torch
    from paper_2609_25653_b300 import ipcsim, scenes
    torch.cuda.set_device(0)
    sc = scenes.arm_gripper_grasp(0)
    sim = ipcsim.Simulator(sc)
    for _ in range(max(args.warmup, 1)):
        sim.step()
    _, tris_s, _ = sim.surface()
    extra, tris, types, rgb, cam = scenes.render_setup(sc, tris_s, sim.nv)
    xv = torch.cat([sim.positions(), torch.as_tensor(extra, device="cuda")]).contiguous()
    r = ipcsim.Renderer(tris, types, rgb, xv.shape[0])
    out = r.render(xv, cam, spp=32, max_depth=2, n_shadow=8)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for k in range(args.steps):
        r.render(xv, cam, spp=32, max_depth=2, n_shadow=8, seed=k, out=out)
    e1.record()
    e1.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    img = out.cpu().numpy()
    if args.frame_out:
        np.save(args.frame_out, img)  # the last frame, (height, width, 3) linear RGB
    print(json.dumps({"workload": "render_" + sc["name"], "triangles": int(len(tris)), "width": cam[1],
                      "height": cam[2], "spp": 32, "max_depth": 2, "n_shadow": 8, "frames": args.steps,
                      "ms_per_frame": round(ms, 3), "fps": round(1e3 / ms, 2),
                      "mean_rgb": [float(v) for v in img.reshape(-1, 3).mean(0)],
                      "context": "paper: 24 FPS at 640x360, 32 SPP on one RTX 5090 (its own renderer)"}))


def shard_scenes(scenes_list, rank, world):
    """Scenes of rank `rank` out of `world` (round robin: r, r + N, ...); every rank keeps at least one."""
    mine = scenes_list[rank::world]
    return mine if mine else scenes_list[:1]


def _small_enough(S):
    return S.sv.size * len(S.tris) + len(S.edges) ** 2 / 2 < 3e7


def oracle_sampled_iteration_seconds(o, budget):
    """Seconds one oracle Newton iteration takes on this workload, from a measured sample.

    A Newton iteration of the oracle runs three brute-force pair sweeps (active
    set for the assembly, active set for the line-search energy, CCD), two
    elastic passes (with and without Hessians) and one sparse LU solve.  The
    elastic passes and the solve are timed in full; the pair sweeps are timed
    over the first k surface vertices (point-triangle) and the first m edges
    (edge-edge) and scaled by the fraction of pair tests they cover."""
    import ctypes as C
    import numpy as np
    import scipy.sparse.linalg as spla
    from oracle import ipc as orc
    S = o.S
    L = orc.lib()
    x = np.ascontiguousarray(S.positions(o.z).reshape(-1))
    t0 = time.perf_counter()
    Ec = C.c_double(0.0)
    g = np.zeros(3 * S.nv)
    Hv = np.zeros(len(S.tets) * 144)
    L.orc_elastic_all(len(S.tets), orc._i(S.tets), orc._d(S.B), orc._d(S.vol), orc._d(S.mu), orc._d(S.lam),
                      orc._d(x), 1, C.byref(Ec), orc._d(g), orc._d(Hv))
    t_el_h = time.perf_counter() - t0
    t0 = time.perf_counter()
    L.orc_elastic_all(len(S.tets), orc._i(S.tets), orc._d(S.B), orc._d(S.vol), orc._d(S.mu), orc._d(S.lam),
                      orc._d(x), 0, C.byref(Ec), orc._d(g), C.cast(0, orc.dp))
    t_el = time.perf_counter() - t0
    import scipy.sparse as sp
    H = sp.csr_matrix((Hv, (S.el_rows, S.el_cols)), shape=(3 * S.nv, 3 * S.nv))
    H = (S.M + S.dt ** 2 * (S.Jmap.T @ H @ S.Jmap)).tocsr()[:S.n_free, :S.n_free].tocsc()
    H = H + sp.identity(S.n_free, format="csc") * 1e-12
    t0 = time.perf_counter()
    spla.spsolve(H, np.ones(S.n_free))
    t_solve = time.perf_counter() - t0
    # pair sweeps over a prefix of the primitives
    per_sweep = max(0.5, (budget - t_el_h - t_el - t_solve) / 3)
    nsv, ne = len(S.sv), len(S.edges)
    k = max(1, min(nsv, int(nsv * 0.04)))
    m = max(2, min(ne, int(ne * 0.1)))
    sub = orc.OrcSurf(k, len(S.tris), 0, orc._i(S.sv), orc._i(S.tris), orc._i(S.edges), orc._i(S.vbody),
                      orc._i(S.bkind))
    rec = np.zeros((1 << 16, 8), np.int32)
    rs = np.zeros(1 << 16)
    t0 = time.perf_counter()
    L.orc_active_pairs(C.byref(sub), orc._d(x), S.sh, 1 << 16, orc._i(rec), orc._d(rs))
    t_pt = (time.perf_counter() - t0) * nsv / k
    sub = orc.OrcSurf(0, len(S.tris), m, orc._i(S.sv), orc._i(S.tris), orc._i(S.edges), orc._i(S.vbody),
                      orc._i(S.bkind))
    t0 = time.perf_counter()
    L.orc_active_pairs(C.byref(sub), orc._d(x), S.sh, 1 << 16, orc._i(rec), orc._d(rs))
    t_ee = (time.perf_counter() - t0) * (ne * (ne - 1)) / (m * (m - 1))
    t_sweep = t_pt + t_ee
    total = 3 * t_sweep + t_el_h + t_el + t_solve
    detail = (f"elastic+Hessian {t_el_h:.2f} s, elastic {t_el:.2f} s, sparse LU {t_solve:.2f} s measured in full; "
              f"pair sweep {t_sweep:.1f} s scaled from {k}/{nsv} surface vertices and {m}/{ne} edges")
    return total, detail


def cpu_baseline(sc, seconds, newton_per_step=None):
    """The oracle as it stands on a bounded sample of the same workload (its brute-force pair loops on all
    host cores, the rest on one)."""
    from oracle import ipc as orc
    o = orc.Oracle(sc)
    if _small_enough(o.S):
        t0 = time.perf_counter()
        n = 0
        while True:
            o.step()
            n += 1
            el = time.perf_counter() - t0
            if el > seconds or n >= sc["params"]["n_steps"]:
                break
        return {"value": round(n / el, 4), "unit": UNIT, "cores": orc.get_threads(), "kind": "oracle",
                "sample": (f"first {n} steps of the same workload ({el:.1f} s; brute-force pair loops on "
                           f"{orc.get_threads()} threads, element loops and scipy sparse LU on one)")}
    t_it, detail = oracle_sampled_iteration_seconds(o, seconds)
    nps = newton_per_step or 5.0
    return {"value": round(1.0 / (t_it * nps), 7), "unit": UNIT, "cores": orc.get_threads(), "kind": "oracle",
            "sample": (f"extrapolated: one oracle Newton iteration = {t_it:.1f} s ({detail}); "
                       f"x {nps:.1f} Newton iterations per step as measured on the GPU run")}


REDUCED = {"arm_gripper": "arm_gripper_grasp_reduced", "soft_cylinder": "soft_gripper_cylinder_reduced"}


def oracle_newton_per_step(workload, seconds):
    """Newton iterations per step of the oracle itself, measured over the first steps of the reduced
    version of the workload (the same ingredients at a resolution it steps in seconds)."""
    from oracle import ipc as orc
    from paper_2609_25653_b300 import scenes
    name = REDUCED.get(workload, "arm_gripper_grasp_reduced")
    o = orc.Oracle(getattr(scenes, name)(0))
    its, t0 = [], time.perf_counter()
    while time.perf_counter() - t0 < seconds and len(its) < 12:
        its.append(len(o.step()))
    return sum(its) / len(its), f"{len(its)} oracle steps of {name}"


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl = make_workload(args.workload)
    sc = wl[0] if isinstance(wl, list) else wl
    from oracle import ipc as orc
    o = orc.Oracle(sc)
    if _small_enough(o.S):
        for _ in range(min(args.warmup, 1)):
            o.step()
        t0 = time.perf_counter()
        n = 0
        budget = args.cpu_seconds * 4
        for _ in range(args.steps):
            o.step()
            n += 1
            if time.perf_counter() - t0 > budget:
                break
        el = time.perf_counter() - t0
        v = n / el
        sample = f"{n} timed steps after the warm-up, stopped at {budget:.0f} s"
        ms = 1e3 * el / n
    else:
        # each step: one bounded sample of an oracle Newton iteration on this workload (timed in full where
        # it is cheap, the pair sweeps over a prefix), x 5 Newton iterations per step; the median is kept
        for _ in range(min(args.warmup, 1)):
            oracle_sampled_iteration_seconds(o, args.cpu_seconds)
        t0 = time.perf_counter()
        its = []
        for _ in range(max(1, args.steps)):
            t_one, detail = oracle_sampled_iteration_seconds(o, args.cpu_seconds)
            its.append(t_one)
            if time.perf_counter() - t0 > 180.0:
                break
        t_it = float(sorted(its)[len(its) // 2])
        nps, nps_src = oracle_newton_per_step(args.workload, min(60.0, 4 * args.cpu_seconds))
        v = 1.0 / (t_it * nps)
        n = len(its)
        ms = 1e3 / v
        sample = (f"{n} sampled oracle Newton iterations, median {t_it:.1f} s (last: {detail}); "
                  f"x {nps:.2f} Newton iterations per step, measured by the oracle over {nps_src}")
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 7), "unit": UNIT, "n_gpus": args.gpus, "steps": n,
            "warmup": min(args.warmup, 1), "ms_per_step": round(ms, 2), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(wl, args.workload, {"parallelism": f"cpu-{orc.get_threads()}",
                                                          "reference_scene": sc["name"]}),
            "cpu_baseline": {"value": round(v, 7), "unit": UNIT, "cores": orc.get_threads(), "kind": "oracle",
                             "sample": sample + f"; brute-force pair loops on {orc.get_threads()} threads"},
            "e2e": {"value": round(v, 7), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="arm_gripper")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default PCG launch shape")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint ms/step measurement")
    ap.add_argument("--id-steps", type=int, default=100, help="material_id workload: rollout steps")
    ap.add_argument("--preconditioner", choices=["two-level", "block-jacobi"], default="two-level")
    ap.add_argument("--coarse-rebuild", type=int, default=0,
                    help="two-level: 0 rebuild every step, n keep up to n steps, -1 every Newton iteration")
    ap.add_argument("--gate", type=int, default=0,
                    help="batched workloads: compare the first N scenes with FP64 single-scene runs")
    ap.add_argument("--fd-steps", type=int, default=10, help="material_id workload: steps of the FD check")
    ap.add_argument("--frame-out", default=None, help="render workload: save the last frame (.npy) here")
    ap.add_argument("--sample", choices=["trajectory", "consecutive"], default="trajectory",
                    help="time K steps spread over the whole trajectory (default) or the K steps after the warm-up")
    ap.add_argument("--precision", choices=["fp64", "mixed"], default=None,
                    help="default: fp64 for single scenes, mixed (FP32 PCG, FP64 residuals) for batches")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "material_id":
        run_material_id(args)
    elif args.workload == "render":
        run_render(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
