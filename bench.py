#!/usr/bin/env python
"""Benchmark of the differentiable MAC-grid fluid step (arXiv 2503.00868, Sec. 3.4).

Metric: forward + adjoint cell-steps per second at 256^3. One benchmark step is
one pass of the whole hot path over one synthetic scene: a checkpointed rollout
of FRAMES steps (advection, body force, implicit viscosity, pressure projection),
the Eq. eq::optLoss loss on the surface band at the last frame, and the reverse
pass (segment recompute + adjoint steps) giving dL/du0 and dL/dnu.
cell-steps/s = nx * ny * nz * FRAMES / (time of the step).

Scene (stand-in for the paper's video-derived liquid blob): an ellipsoid of
liquid resting on the floor, 40 % occupancy, air elsewhere, box walls solid;
initial velocity = seeded N(0,1) noise blurred by a sigma = 3 cell Gaussian;
target = an independent blurred field (seed + 100); nu = 0.01, dt = 1/30,
dx = 1/256; both implicit solves by multigrid-preconditioned CG to relative
residual 1e-6 (--precond jacobi / mic0 for the others), pressure solves warm
started from the previous frame's pressure.

Besides the headline line's keys it reports, per kernel, the live mean duration,
the launches that did work and their estimated share of the step; a roofline for
the single kernel with the largest share and one for the level-0 multigrid
kernels together; the oracle on one host core and on all of them; the smaller
configurations (32^3 plain forward with MIC(0), 128^3 forward + adjoint over four
viscosities); and the projection comparison of the preconditioners at 256^3.

Usage: python bench.py [--gpus N --steps K --warmup W] [--impl reference]
Multi-GPU runs are independent replicas (one scene per rank, no collective on
the data path); the timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2503_00868_gb300.clocks import ClockSampler  # noqa: E402

FRAMES = 8
CHECKPOINT = 4
PROFILE_PERIOD = 8   # time every 8th CG iteration inside the timed region
METRIC = "fwd+adjoint cell-steps/s at 256^3"
UNIT = "cell-steps/s"

# ncu DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum,
# bytes) of the kernels, keyed by the profile name; each entry holds the hash of
# the files that define the kernel and the data layout it reads, and is reported
# only while those files are unchanged (capture commands in profiles/).
NCU_TRAFFIC = {
    # ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum on the benchmark's 256^3 blob with the
    # multigrid preconditioner (profiles/fwd_adjoint_256.md); DRAM writes still held dirty in L2
    # when the kernel ends are not counted
    "visc_spmv": {"bytes_per_launch": 342685440 + 134320896, "source": "5e31bb1c3ef8787b"},
    "visc_update": {"bytes_per_launch": 387683584 + 125340416, "source": "5e31bb1c3ef8787b"},
    # ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum -k regex:k_mg0_smooth2 on the
    # benchmark's 256^3 blob, one level-0 launch (profiles/mg0_kernels_256_ncu.md); the entry
    # names its own files: the V-cycle kernels and the mask layout they read
    "mg0_smooth2": {"bytes_per_launch": 50603776 + 3720704, "source": "4cfc780494228df8",
                    "files": ("fs_mg.cu", "fs_mask.cu")},
    # the same metrics -k regex:^k_mg0_smooth$ on a 256^3 blob projection with the multigrid
    # preconditioner: the last level-0 sweep of a pressure V-cycle, which forms r.z (the mean
    # of two launches; profiles/mg0_kernels_256_ncu.md); its files include the grid sums
    # the same metrics -k regex:k_spmv_list on that projection: the pressure operator apply over
    # the multigrid level-0 list of active quads (the mean of four launches; profiles/spmv_list_256_ncu.md)
    "pressure_spmv": {"bytes_per_launch": 85581312 + 35093888, "source": "83675cdd5bd4c57e",
                      "files": ("fs_pcg.cu", "fs_internal.cuh", "fs_mg.cu", "fs_mask.cu")},
    "mg0_smooth_z": {"bytes_per_launch": 83167232 + 5408384, "source": "5ebc55d1e28ef6ee",
                     "files": ("fs_mg.cu", "fs_internal.cuh", "fs_mask.cu")},
}
KERNEL_FILES = ("fs_stencil.cuh", "fs_tma.cuh", "fs_mask.cu")


def args_parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--frames", type=int, default=FRAMES)
    ap.add_argument("--precond", default="mg", choices=["jacobi", "mic0", "mg"])
    ap.add_argument("--cpu-sample-n", type=int, default=64)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the 32^3 plain-forward and 128^3 four-viscosity configurations")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the Jacobi / MIC(0) / learned projection comparison")
    ap.add_argument("--compare-n", type=int, default=256)
    ap.add_argument("--cold-start", action="store_true",
                    help="every pressure solve from q = 0 (default: warm start from the previous solve)")
    return ap.parse_args()


def source_hash(files=KERNEL_FILES):
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2503_00868_gb300", "csrc")
    for name in files:
        h.update(open(os.path.join(csrc, name), "rb").read())
    return h.hexdigest()[:16]


# profile entries that aggregate several kernels (a whole V-cycle, the coarse
# levels of one): reported, but not a kernel for the roofline
AGGREGATES = ("all_kernels", "mg_vcycle_p", "mg_vcycle_v", "mg_coarse")
# the level-0 multigrid kernels, reported together as one family
MG_LEVEL0 = ("mg0_smooth2", "mg0_residual", "mg0_restrict", "mg0_prolong", "mg0_smooth", "mg0_smooth_z")


def _entry(v):
    """(timed launches, total ms, bytes, all launches) from a profile value (the
    all-launch count defaults to the timed count)"""
    return (v[0], v[1], v[2], v[3] if len(v) > 3 else v[0])


def kernel_table(prof, step_ms, steps, hbm):
    """Per profile entry: timed launches, launches that did work, live mean, the
    estimated share of the step (mean x all launches / timed region) and, where
    algorithmic bytes are known, the achieved GB/s and its fraction of `hbm`."""
    out = {}
    for k, v in prof.items():
        launches, ms, by, alln = _entry(v)
        if k == "all_kernels" or not launches:
            continue
        mean_ms = ms / launches
        e = {"timed_launches": launches, "launches": alln, "mean_us": round(1e3 * mean_ms, 2),
             "est_share_of_step": round(mean_ms * alln / (step_ms * steps), 4)}
        if by > 0:
            gbs = (by / launches) / (mean_ms * 1e-3) / 1e9
            e["achieved_gbs"] = round(gbs, 1)
            e["frac_of_hbm"] = round(gbs / hbm, 3)
            e["algorithmic_bytes_per_launch"] = by / launches
        out[k] = e
    return out


def roofline_of(prof, peaks, src_hash, traffic_table=None):
    """The roofline object of the single kernel with the largest estimated share
    of the step among those that carry algorithmic bytes (the share is its mean
    duration times the launches that did work). prof maps a name to (timed
    launches, total ms, total algorithmic bytes[, all launches]). achieved = bytes
    per launch / mean launch time; the peak is the measured HBM copy bandwidth
    (the 6800 GB/s fallback without a measurement); the ncu traffic is reported
    only while the hash of the files that define the kernels matches its
    capture's."""
    traffic_table = NCU_TRAFFIC if traffic_table is None else traffic_table
    hbm = peaks["hbm_gbs"] if peaks else 6800.0
    cands = [(k, _entry(v)) for k, v in prof.items() if k not in AGGREGATES]
    top = max((kv for kv in cands if kv[1][2] > 0 and kv[1][0] > 0),
              key=lambda kv: kv[1][1] / kv[1][0] * kv[1][3], default=None)
    if top is None:
        return None
    name, (launches, ms, by, alln) = top
    achieved = (by / launches) / (ms / launches * 1e-3) / 1e9
    tr = traffic_table.get(name)
    want = source_hash(tr["files"]) if tr and "files" in tr else src_hash
    traffic = tr["bytes_per_launch"] if tr and tr.get("source") == want else None
    return {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": hbm, "unit": "GB/s",
            "frac": achieved / hbm, "traffic": traffic,
            "algorithmic_bytes_per_launch": by / launches, "launches": launches, "launches_all": alln,
            "avg_launch_us": 1e3 * ms / launches,
            "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if peaks else "fallback"}


def family_roofline(prof, peaks, names=MG_LEVEL0):
    """The level-0 multigrid kernels as one family: summed algorithmic bytes of
    their timed launches over their summed durations."""
    hbm = peaks["hbm_gbs"] if peaks else 6800.0
    got = [_entry(prof[k]) for k in names if k in prof and prof[k][0] > 0]
    if not got:
        return None
    by = sum(v[2] for v in got)
    ms = sum(v[1] for v in got)
    achieved = by / (ms * 1e-3) / 1e9
    return {"bound": "hbm", "kernels": [k for k in names if k in prof], "achieved": achieved, "peak": hbm,
            "unit": "GB/s", "frac": achieved / hbm,
            "note": "level 0 of the pressure V-cycle, timed kernel by kernel on the library stream"}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


def make_scene(n, seed):
    from paper_2503_00868_gb300 import workloads as W
    types, info = W.ellipsoid_blob(n, n, n, seed)
    u0 = W.blurred_noise_mac(n, n, n, seed)
    tgt = W.blurred_noise_mac(n, n, n, seed + 100)
    return types, u0, tgt, info


def params_for(n, precond, warm_start=1):
    from paper_2503_00868_gb300 import fluidstep as F
    return dict(dx=1.0 / n, dt=1.0 / 30.0, nu=0.01, g=(0.0, 0.0, 0.0), tol_p=1e-6, tol_v=1e-6,
                precond={"mic0": F.FS_PRECOND_MIC0, "mg": F.FS_PRECOND_MG}.get(precond, F.FS_PRECOND_JACOBI),
                check_every=16,
                maxit_p=20000, maxit_v=4000, warm_start=warm_start)


ORACLE_SAMPLE = ("FP64 oracle (plain C), fwd+adjoint of 1 frame of the same scene recipe at {n}^3: "
                 "MIC(0)-PCG pressure and Jacobi-PCG viscosity to 1e-6, loss at that frame")


def cpu_oracle_sample(n, frames=1, seed=0):
    """The FP64 oracle, as it stands, on a bounded sample of the workload: the
    same scene recipe at n^3, one forward step + loss + one adjoint step, with
    the oracle's fastest pressure preconditioner (MIC(0))."""
    import oracle as O
    types, u0, tgt, _ = make_scene(n, seed)
    kw = params_for(n, "jacobi")
    g = O.Grid(types, kw["dx"], kw["dt"], kw["nu"], g=kw["g"], tol_p=kw["tol_p"], tol_v=kw["tol_v"],
               precond=O.PC_MIC0)
    t0 = time.perf_counter()
    states = [u0]
    for _ in range(frames):
        states.append(O.step(g, states[-1])[0])
    loss, gbar = O.loss_grad(g, states[-1], tgt)
    for k in range(frames - 1, -1, -1):
        gbar, _ = O.adjoint_step(g, states[k], gbar)
    dt = time.perf_counter() - t0
    return n ** 3 * frames / dt, dt


def _oracle_worker(args):
    n, seed = args
    import oracle as O
    O.build()
    return cpu_oracle_sample(n, seed=seed)


def cpu_oracle_all_cores(n, cores=None):
    """The same oracle sample run as independent copies, one per host core (a
    process pool started with spawn): the host's whole-machine throughput on the
    sample, cell-steps/s summed over the copies."""
    import multiprocessing as mp
    cores = cores or os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(cores) as pool:
        res = pool.map(_oracle_worker, [(n, s) for s in range(cores)])
    wall = time.perf_counter() - t0
    return cores * n ** 3 / wall, cores, wall, res


def reference_config(a):
    """The configuration the reference arm actually runs: the oracle on a bounded
    sample of the benchmark's scene recipe."""
    n = a.cpu_sample_n
    return {"workload": ORACLE_SAMPLE.format(n=n) + f"; stands in for the {a.n}^3, {a.frames}-frame benchmark, "
                        "whose full size the oracle cannot finish in minutes",
            "grid": [n, n, n], "frames": 1, "precond": "mic0 (pressure), jacobi (viscosity)", "tol": 1e-6,
            "nu": 0.01, "dt": 1.0 / 30.0, "dtype": "f64", "cores": 1, "parallelism": "single"}


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle as O
    O.build()
    n = a.cpu_sample_n
    for _ in range(a.warmup):
        cpu_oracle_sample(n)
    vals, total = [], 0.0
    for _ in range(a.steps):
        v, dt = cpu_oracle_sample(n)
        vals.append(v)
        total += dt
    value = a.steps * n ** 3 / total
    sample = (ORACLE_SAMPLE.format(n=n) + ", one host core (iteration counts grow with n, so this overstates "
              "the oracle's throughput at 256^3)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * total / a.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": reference_config(a),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def workload_config(a):
    return {"workload": f"fwd+adjoint checkpointed rollout on a {a.n}^3 MAC grid: ellipsoid liquid blob "
                        f"(40% occupancy) on the floor, {a.frames} frames, checkpoint every {CHECKPOINT}, "
                        f"surface-band L2 loss at the last frame, gradients w.r.t. nu and u0",
            "grid": [a.n, a.n, a.n], "frames": a.frames, "checkpoint_every": CHECKPOINT,
            "precond": a.precond, "tol": 1e-6, "nu": 0.01, "dt": 1.0 / 30.0,
            "warm_start": not a.cold_start,
            "l2_between_steps": "inputs larger than L2 (working set > 1 GB per replica)",
            "parallelism": "replicas" if a.gpus > 1 else "single"}


def precond_compare(n, seeds=(0,)):
    """Projection of an unblurred N(0,1) MAC field (the stress right-hand side) on
    a union of 8 spheres at n^3, to relative residual 1e-6, with Jacobi, MIC(0),
    the multigrid V-cycle, the shipped learned network alone, and the network
    trained for the smoother role in front of one V-cycle (flexible CG; its layers
    on mma.sync and on tcgen05): device wall time of fs_project (CUDA events,
    after one warm-up solve), iterations, true residual, and the network's share."""
    import torch
    from paper_2503_00868_gb300 import fluidstep as F
    from paper_2503_00868_gb300 import train_precond as T
    from paper_2503_00868_gb300 import workloads as W
    out = {"workload": f"projection of a divergent N(0,1) MAC field on a union of 8 spheres at {n}^3, "
                       "tol 1e-6, maxit 20000", "rows": []}
    pcs = (("jacobi", F.FS_PRECOND_JACOBI), ("mic0", F.FS_PRECOND_MIC0), ("mg", F.FS_PRECOND_MG),
           ("learned", F.FS_PRECOND_LEARNED), ("learned_mg", F.FS_PRECOND_LEARNED_MG),
           ("learned_mg_tcgen05", F.FS_PRECOND_LEARNED_MG))
    for seed in seeds:
        types, info = W.sphere_union(n, n, n, seed)
        row = {"seed": seed, "occupancy": info["occupancy"]}
        for name, pc in pcs:
            g = F.Grid(n, n, n, dx=1.0 / n, tol_p=1e-6, maxit_p=20000, precond=pc)
            g.set_mask(types)
            if pc == F.FS_PRECOND_LEARNED:
                F.fs_net_load(g.ctx, T.default_weights())
            elif pc == F.FS_PRECOND_LEARNED_MG:
                F.fs_net_load(g.ctx, T.role_weights("net_mg"))
                F.fs_net_kernel(g.ctx, 1 if name.endswith("tcgen05") else 0)
            u0 = g.pack(W.random_mac(n, n, n, 500 + seed))
            ts = []
            for rep in range(2):
                u = F.Mac(*(t.clone() for t in u0))
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                rc, st = g.project(u)
                e1.record()
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            row[name] = {"ms": round(ts[-1], 3), "iters": st["iters_p"], "true_relres": st["true_relres_p"],
                         "fallbacks": st["fallbacks"], "restarts": st["restarts_p"], "status": rc}
            if pc in (F.FS_PRECOND_LEARNED, F.FS_PRECOND_LEARNED_MG):
                # the network's applications in a third, profiled solve (every one timed):
                # useful flops on the visited tiles over their time, against the bf16 peak
                g.profile(1)
                g.project(F.Mac(*(t.clone() for t in u0)))
                na = g.profile_read().get("net_apply")
                g.profile(0)
                if na and na[0]:
                    tfl = na[2] / (na[1] * 1e-3) / 1e12
                    peak = (measured_peaks() or {}).get("bf16_tflops", 1900.0)
                    row[name]["net"] = {"applies": na[0], "ms_per_apply": round(na[1] / na[0], 4),
                                        "useful_tflop_per_apply": na[2] / na[0] / 1e12, "achieved_tflops": tfl,
                                        "frac_of_bf16_peak": tfl / peak}
            g.close()
        # the recurrent convolutional solver with the shipped fitted kernel: a fixed
        # 100 sub-steps, so its true residual is reported rather than reached
        from paper_2503_00868_gb300 import train_percnn as TP
        g = F.Grid(n, n, n, dx=1.0 / n, pressure_solver=F.FS_SOLVER_PERCNN)
        g.set_mask(types)
        F.fs_percnn_load(g.ctx, TP.default_kernel(), 100)
        u0 = g.pack(W.random_mac(n, n, n, 500 + seed))
        for rep in range(2):
            u = F.Mac(*(t.clone() for t in u0))
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            rc, st = g.project(u)
            e1.record()
            torch.cuda.synchronize()
        row["percnn_k100"] = {"ms": round(e0.elapsed_time(e1), 3), "iters": st["iters_p"],
                              "true_relres": st["true_relres_p"], "status": rc}
        g.close()
        out["rows"].append(row)
    # the learned preconditioner in its V-cycle role against MIC(0)-PCG (the
    # network alone is the "learned" row)
    r0 = out["rows"][0]
    out["learned_vs_mic0"] = {"learned_row": "learned_mg", "learned_ms": r0["learned_mg"]["ms"],
                              "mic0_ms": r0["mic0"]["ms"],
                              "speedup": r0["mic0"]["ms"] / max(r0["learned_mg"]["ms"], 1e-9),
                              "learned_true_relres": r0["learned_mg"]["true_relres"],
                              "learned_fallbacks": r0["learned_mg"]["fallbacks"]}
    return out


def config_c1():
    """The plain forward configuration: 32^3, all cells liquid in a closed box,
    dx = 1/32, dt = 1/30, nu = 0.01, 10 steps from the blurred noise field,
    MIC(0)-PCG to 1e-6 (Jacobi-PCG for the viscosity). Device time of the 10
    steps after one untimed run."""
    import torch
    from paper_2503_00868_gb300 import fluidstep as F
    from paper_2503_00868_gb300 import workloads as W
    n, steps = 32, 10
    g = F.Grid(n, n, n, dx=1.0 / n, dt=1.0 / 30.0, nu=0.01, precond=F.FS_PRECOND_MIC0, tol_p=1e-6, tol_v=1e-6,
               maxit_p=20000, maxit_v=4000)
    g.set_mask(W.all_liquid(n, n, n))
    u0 = g.pack(W.blurred_noise_mac(n, n, n, 0))
    a, b = g.zeros(), g.zeros()
    sts = []
    for rep in range(2):
        for t, s0 in zip(a, u0):
            t.copy_(s0)
        sts.clear()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            rc, st = g.step(a, b)
            sts.append(st)
            a, b = b, a
        e1.record()
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    g.close()
    return {"workload": "plain forward, 32^3 closed box full of liquid, 10 steps, MIC(0)-PCG to 1e-6",
            "value": n ** 3 * steps / (ms * 1e-3), "unit": "cell-steps/s", "ms": round(ms, 3),
            "pressure_iters_mean": sum(x["iters_p"] for x in sts) / len(sts),
            "true_relres_p_max": max(x["true_relres_p"] for x in sts)}


def config_c2(nus=(1e-4, 1e-3, 1e-2, 1e-1), frames=24):
    """Forward + adjoint at 128^3: the ellipsoid blob (40 % occupancy), 24 frames,
    checkpoint every 4, the band loss at the last frame against an independent
    blurred target, gradients w.r.t. nu and u0, one run per viscosity (after an
    untimed one), with the benchmark's multigrid solves."""
    import torch
    from paper_2503_00868_gb300 import fluidstep as F
    from paper_2503_00868_gb300.rollout import rollout_loss
    n = 128
    types, u0_np, tgt_np, info = make_scene(n, 0)
    grid = F.Grid(n, n, n, **params_for(n, "mg", 1))
    grid.set_mask(types)
    u0, tgt = grid.pack(u0_np), grid.pack(tgt_np)
    rows, total_ms = [], 0.0
    for nu in nus:
        for rep in range(2):
            leaves = [t.detach().clone().requires_grad_(True) for t in u0]
            nu_t = torch.tensor(nu, dtype=torch.float32, requires_grad=True)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            loss = rollout_loss(grid, F.Mac(*leaves), nu_t, frames, {frames: tgt}, CHECKPOINT)
            loss.backward()
            e1.record()
            torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        total_ms += ms
        rows.append({"nu": nu, "ms": round(ms, 2), "cell_steps_per_s": n ** 3 * frames / (ms * 1e-3),
                     "loss": float(loss.detach()), "dL_dnu": float(nu_t.grad)})
    grid.close()
    return {"workload": f"fwd+adjoint, 128^3 ellipsoid blob ({info['occupancy']:.2f} occupancy), {frames} frames, "
                        "checkpoint 4, band loss at the last frame, multigrid PCG to 1e-6",
            "value": len(nus) * n ** 3 * frames / (total_ms * 1e-3), "unit": "cell-steps/s", "rows": rows}


def dist_env():
    """(world size, rank, local rank) from the torchrun environment (1, 0, 0 alone)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(x: float, world: int, device) -> float:
    """The largest x over the ranks of the process group: a job's time is its
    slowest rank's."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, steps: int, cells: int, frames: int, seconds: float) -> float:
    """Cell-steps per second of the whole job: every rank runs its own scene
    (weak scaling), and the job takes the slowest rank's time."""
    return world * steps * cells * frames / seconds


def main():
    a = args_parse()
    if a.impl == "reference":
        return run_reference(a)

    import torch
    import torch.distributed as dist

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2503_00868_gb300 import build as B
    from paper_2503_00868_gb300 import fluidstep as F
    from paper_2503_00868_gb300.rollout import rollout_loss
    B.build()
    F.load()

    n, frames = a.n, a.frames
    types, u0_np, tgt_np, info = make_scene(n, rank)
    grid = F.Grid(n, n, n, **params_for(n, a.precond, 0 if a.cold_start else 1))
    grid.set_mask(types)
    u0 = grid.pack(u0_np)
    tgt = grid.pack(tgt_np)
    nu_t = torch.tensor(0.01, dtype=torch.float32)
    stats = []

    def one_step(u0m, tgtm):
        leaves = [t.detach().requires_grad_(True) for t in u0m]
        nu = nu_t.detach().clone().requires_grad_(True)
        loss = rollout_loss(grid, F.Mac(*leaves), nu, frames, {frames: tgtm}, CHECKPOINT, stats=stats)
        loss.backward()
        return loss, nu.grad, leaves

    stream = torch.cuda.current_stream()
    for _ in range(max(a.warmup, 0)):
        one_step(u0, tgt)
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            dist.barrier()

    # ---- device-resident timing -------------------------------------------
    stats.clear()
    grid.profile(PROFILE_PERIOD)
    sampler = ClockSampler(local)
    sampler.start()
    barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(a.steps):
        loss, gnu, leaves = one_step(u0, tgt)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    elapsed = ev0.elapsed_time(ev1) / 1e3
    prof = grid.profile_read()
    grid.profile(0)
    elapsed = max_over_ranks(elapsed, world, "cuda")
    cells = n ** 3
    value = job_throughput(world, a.steps, cells, frames, elapsed)
    ms_per_step = 1e3 * elapsed / a.steps
    iters_p = [s[2]["iters_p"] for s in stats if s[0] == "fwd"]
    iters_v = [s[2]["iters_v"] for s in stats if s[0] == "fwd"]
    refines = [s[2]["restarts_p"] for s in stats]

    # ---- end to end through the public API with host buffers ---------------
    e2e = None
    if not a.no_e2e:
        host_u0 = [t.cpu().pin_memory() for t in u0]
        host_t = [t.cpu().pin_memory() for t in tgt]
        host_g = [torch.empty_like(t, device="cpu").pin_memory() for t in u0]
        hb = sum(t.numel() * 4 for t in host_u0) + sum(t.numel() * 4 for t in host_t)
        db = sum(t.numel() * 4 for t in host_g) + 16
        results = []
        barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(a.steps):
            du = F.Mac(*(h.to("cuda", non_blocking=True) for h in host_u0))
            dtg = F.Mac(*(h.to("cuda", non_blocking=True) for h in host_t))
            loss, gnu, leaves_e = one_step(du, dtg)
            # the step's results read back on the host: dL/du0, the loss and dL/dnu
            for h, t in zip(host_g, leaves_e):
                h.copy_(t.grad, non_blocking=True)
            results.append((float(loss.detach().cpu()), float(gnu.detach().cpu())))
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        t_e2e = max_over_ranks(e0.elapsed_time(e1) / 1e3, world, "cuda")
        e2e = {"value": job_throughput(world, a.steps, cells, frames, t_e2e), "unit": UNIT,
               "h2d_bytes_per_step": hb, "d2h_bytes_per_step": db}

    # ---- roofline of the dominant kernel -----------------------------------
    peaks = measured_peaks()
    hbm = peaks["hbm_gbs"] if peaks else 6800.0
    roofline = roofline_of(prof, peaks, source_hash())
    mg_family = family_roofline(prof, peaks)
    kernels = kernel_table(prof, ms_per_step, a.steps, hbm)
    gpu_launches = None
    if "all_kernels" in prof:
        gpu_launches = prof["all_kernels"][0]

    cpu = cpu_all = None
    if rank == 0 and world == 1 and not a.no_cpu:
        import oracle as O
        O.build()
        v, dt = cpu_oracle_sample(a.cpu_sample_n)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": ORACLE_SAMPLE.format(n=a.cpu_sample_n) + f", one host core ({dt:.1f} s; iteration "
                         "counts grow with n, so this overstates the oracle at 256^3)"}
        va, cores, wall, _ = cpu_oracle_all_cores(a.cpu_sample_n)
        cpu_all = {"value": va, "unit": UNIT, "cores": cores, "kind": "oracle",
                   "sample": f"{cores} independent copies of the one-core sample, one per host core, "
                             f"{wall:.1f} s wall"}

    configs = None
    if rank == 0 and world == 1 and not a.no_configs:
        configs = {"plain_forward_32": config_c1(), "fwd_adjoint_128_four_nu": config_c2()}

    compare = None
    if rank == 0 and not a.no_compare:
        compare = precond_compare(a.compare_n)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
                "warmup": a.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": workload_config(a),
                "clocks": clocks, "e2e": e2e, "gpu_launches": gpu_launches, "roofline": roofline,
                "roofline_mg_level0": mg_family, "cpu_baseline": cpu, "cpu_baseline_all_cores": cpu_all,
                "kernels": kernels, "occupancy": info["occupancy"],
                "pcg_iters_per_step": {"pressure_mean": sum(iters_p) / max(len(iters_p), 1),
                                       "viscosity_mean": sum(iters_v) / max(len(iters_v), 1),
                                       "pressure_refinements": sum(refines)},
                "loss": float(loss.detach()), "dL_dnu": float(gnu), "configs": configs,
                "precond_compare": compare}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    grid.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
