"""Benchmark of the entropic-MRT two-phase lattice Boltzmann time step.

Workload: D3Q27 drop impact on a thin film, 512x512x256 nodes, FP32 populations
in one A-A buffer (7.25 GB, far larger than the 129 MB L2, so no flush is
needed between steps), density ratio ~1000 (T/Tc = 0.59).  One benchmark step is
one lattice time step (its three kernels: moments and EOS, force and q, collide
and stream) over the whole domain.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  value = MLUPS (million lattice updates per second, whole
job); e2e = the same metric through the C ABI with host buffers (initial fields
copied in, K steps, density and velocity copied out); roofline = the
force+collide+stream kernel's algorithmic bytes per launch over its CUDA-event
duration, against the measured HBM copy bandwidth; cpu_baseline = the FP64
oracle on a bounded crop of the same workload on the host cores; serving (N = 1)
= p50/p99 latency and aggregate MLUPS of a 200-job continuous-batching run.

--impl reference times the FP64 CPU oracle (the reference implementation of
the method) on a bounded crop of the same workload; N > 1: rank 0 only.
--workload drop2d runs the D2Q9 drop impact (2048x1024) the same way.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PEAKS_FALLBACK = {"hbm_gbs": 6800.0}
E2E_REPEATS = 5  # end-to-end passes; the line reports the median (host copies on a
                 # shared host stall now and then: one or two slow passes do not set it)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except Exception:
        return PEAKS_FALLBACK, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
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

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        except Exception:
            pass
        finally:
            try:
                os.unlink(self.path)
            except Exception:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x, world):
    """Largest value over all ranks (the job's wall time is the slowest rank's)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(nodes_per_rank, steps, world, max_ms):
    """Weak scaling: every rank advances its own replica, so the job's updates are
    world x nodes x steps over the slowest rank's time."""
    return nodes_per_rank * steps * world / (max_ms * 1e-3) / 1e6


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------------------------
# CPU oracle on a bounded crop of the workload
# ---------------------------------------------------------------------------
CPU_CROP = (48, 64, 64)   # nz, ny, nx: 196,608 nodes
CPU_CROP_2D = (1, 384, 512)
CPU_SAMPLE_S = 10.0   # seconds of oracle work in the bench line's cpu_baseline
CPU_MAX_STEPS = 2000


def oracle_crop_state(wl, crop=CPU_CROP):
    """Oracle parameters and initial populations of a crop of the workload."""
    import oracle as O
    from oracle import thermo
    from paper_2201_12404_gb300 import workloads as WL
    rv, rl, _ = thermo.maxwell(wl.T_over_Tc, **WL.PAPER_EOS)
    nu_l, nu_v = WL.viscosities(wl, rv, rl)
    bc = [0] * 6
    if wl.walls_axis >= 0:
        bc[2 * wl.walls_axis] = bc[2 * wl.walls_axis + 1] = 1
    nz, ny, nx = crop
    p = O.make_params(wl.D, nx, ny, nz, T_over_Tc=wl.T_over_Tc, kappa=wl.kappa, nu_liquid=nu_l,
                      nu_vapour=nu_v, rho_liquid=rl, rho_vapour=rv, bc=bc, **WL.PAPER_EOS)
    rho, u = WL.initial_fields(wl, rv, rl, crop=crop)
    return p, O.init_physical(p, rho, u)


def crop_of(wl):
    """The oracle's crop of a workload: CPU_CROP (3-D) or CPU_CROP_2D, clipped to the
    domain (the 128x128 static drop is timed whole)."""
    crop = CPU_CROP if wl.D == 3 else CPU_CROP_2D
    return tuple(min(c, n) for c, n in zip(crop, (wl.nz, wl.ny, wl.nx)))


def lattice_of(wl):
    return "D3Q27" if wl.D == 3 else "D2Q9"


def oracle_sample(wl, target_s=CPU_SAMPLE_S, crop=None):
    """The oracle on a crop of the workload for about target_s seconds: one step sets
    the step count of the rest (at most CPU_MAX_STEPS), and every step is timed."""
    import oracle as O
    crop = crop or crop_of(wl)
    p, f = oracle_crop_state(wl, crop)
    nz, ny, nx = crop
    t0 = time.perf_counter()
    f, _g = O.run(p, f, 1)
    first = time.perf_counter() - t0
    steps = 1 + max(0, min(CPU_MAX_STEPS, int((target_s - first) / max(first, 1e-6))))
    if steps > 1:
        O.run(p, f, steps - 1)
    dt = time.perf_counter() - t0
    lups = nx * ny * nz * steps
    return {"value": lups / dt / 1e6, "unit": "MLUPS", "cores": O.num_threads(), "kind": "oracle",
            "sample": f"FP64 oracle, {steps} steps of a {nx}x{ny}x{nz} crop of the same {lattice_of(wl)} drop-on-film "
                      f"workload (same EOS, kappa, viscosities, walls), {dt:.1f} s"}


L2_BYTES = 129e6  # GB300 L2 (the device query below replaces it when available)


def l2_note(pop_bytes_total):
    """How the timed steps stand against L2: the populations of the default
    workload are far larger than L2, so consecutive steps cannot hit in it."""
    l2 = L2_BYTES
    try:
        import torch
        if torch.cuda.is_available():
            l2 = float(getattr(torch.cuda.get_device_properties(0), "L2_cache_size", l2) or l2)
    except Exception:
        pass
    if pop_bytes_total > 4 * l2:
        return f"inputs larger than L2 ({pop_bytes_total / 1e9:.2f} GB populations vs {l2 / 1e6:.0f} MB L2), no flush"
    return (f"populations ({pop_bytes_total / 1e6:.0f} MB) within a few times the {l2 / 1e6:.0f} MB L2: "
            f"L2-resident throughput, no flush")


def metric_and_config(args, wl, world):
    """Metric name and config of a benchmark line (shared by both arms)."""
    pop_bytes = {"fp64": 8, "fp32": 4, "fp16dev": 2}[args.precision]
    Q = 27 if wl.D == 3 else 9
    metric = f"{lattice_of(wl)} entropic-MRT MLUPS (whole time step, {args.precision.upper()} A-A)"
    config = {"workload": wl.name, "nodes": wl.N, "lattice": lattice_of(wl), "storage": f"{args.precision} A-A",
              "l2": l2_note(Q * pop_bytes * wl.N),
              "parallelism": f"replicas{world}" if world > 1 else "single GPU"}
    return metric, config


def run_reference(args):
    """The reference arm: the FP64 oracle as it stands, on the host cores, one
    oracle step of a bounded crop of the workload per benchmark step (rank 0 only)."""
    import oracle as O
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from paper_2201_12404_gb300 import workloads as WL
    wl = WL.by_name(args.workload)
    crop = crop_of(wl)
    p, f = oracle_crop_state(wl, crop)
    for _ in range(args.warmup):
        f, _g = O.run(p, f, 1)
    times = []
    for _ in range(max(1, args.steps)):
        t0 = time.perf_counter()
        f, _g = O.run(p, f, 1)
        times.append(time.perf_counter() - t0)
    nodes = crop[0] * crop[1] * crop[2]
    v = nodes * len(times) / sum(times) / 1e6
    metric, config = metric_and_config(args, wl, world)
    config["oracle_crop"] = f"{crop[2]}x{crop[1]}x{crop[0]}"
    sample = (f"FP64 oracle, {len(times)} steps of a {crop[2]}x{crop[1]}x{crop[0]} crop of the same "
              f"{lattice_of(wl)} drop-on-film workload, one per benchmark step, {sum(times):.1f} s")
    line = {"impl": "reference", "metric": metric, "value": v, "unit": "MLUPS",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config,
            "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": O.num_threads(), "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def recorded_traffic(key):
    """DRAM bytes per launch of a kernel from the committed ncu summary, or None
    when the kernel's source has changed since the counters were taken."""
    import hashlib
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))[key]
        h = hashlib.sha1()
        for f in rec["source_files"]:
            h.update(open(os.path.join(ROOT, f), "rb").read())
        return rec["bytes_per_launch"] if h.hexdigest() == rec["source_sha1"] else None
    except Exception:
        return None


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def algorithmic_bytes_k2(wl, pop_bytes, aux_bytes):
    """Force+collide+stream kernel: each population read once and written once;
    the node's D components of q and of the force F read once (the q halo re-reads
    are cache hits)."""
    Q = 27 if wl.D == 3 else 9
    return wl.N * (2 * Q * pop_bytes + 2 * wl.D * aux_bytes)


def serving_sample(n_jobs, scale=0.25, seed=None):
    """The served-job part of the metric: a run of the continuous-batching server
    (seeded Poisson arrivals offering 80% of 12 GLUPS of mixed D2Q9/D3Q27 jobs, FP32,
    1,000-10,000 steps per job scaled by `scale`, admission by footprint against half
    of the free HBM)."""
    import torch
    from paper_2201_12404_gb300 import inputs as I
    from paper_2201_12404_gb300 import serve as SV
    seed = I.SEED_BASE if seed is None else seed
    jobs = SV.random_jobs(n_jobs, seed, scale)
    rate = SV.rate_for_load(jobs)
    free, _ = torch.cuda.mem_get_info()
    rep = SV.serve(jobs, SV.poisson_arrivals(len(jobs), rate, seed), int(0.5 * free))
    return {"p50_latency_s": rep["p50_latency_s"], "p99_latency_s": rep["p99_latency_s"],
            "aggregate_mlups": rep["aggregate_mlups"], "jobs": rep["jobs"], "completed": rep["completed"],
            "failed": rep["failed"], "admitted_while_busy": rep["admissions_while_busy"], "wall_s": rep["wall_s"],
            "batch_builds": rep.get("batch_builds"),
            "what": f"{n_jobs} seeded Poisson arrivals (rate {rate:.2f}/s), half D2Q9 64^2-1024^2, half D3Q27 "
                    f"64^3-256^3, steps 1,000-10,000 x {scale} (that fraction of each job's steps), FP32"}


def algorithmic_bytes_k1(wl, pop_bytes, aux_bytes):
    """Passes 1 and 1b, timed together: pass 1 reads each population once, writes
    the (rho, psi) pair at every padded node (interior nodes and the ghosts imaging
    them) and the D momentum planes j at the interior; pass 1b reads the pairs once
    per padded node (halo re-reads are cache hits) and j once per interior node,
    writes q at every padded node and F over j at the interior."""
    Q = 27 if wl.D == 3 else 9
    px = (wl.nx + 4 + 3) // 4 * 4
    pn = px * (wl.ny + 4) * ((wl.nz + 4) if wl.D == 3 else 1)
    return wl.N * Q * pop_bytes + pn * (2 + 2 + wl.D) * aux_bytes + wl.N * 3 * wl.D * aux_bytes


def run_ours(args):
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2201_12404_gb300 import lbm
    from paper_2201_12404_gb300 import workloads as WL
    lbm.load()

    wl = WL.by_name(args.workload)
    rv, rl = WL.coexistence(wl)
    # a dedicated stream: the library launches on it and the timing events are recorded on it
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    prec = {"fp64": lbm.LBM_FP64, "fp32": lbm.LBM_FP32, "fp16dev": lbm.LBM_FP16DEV}[args.precision]
    pop_bytes = {"fp64": 8, "fp32": 4, "fp16dev": 2}[args.precision]
    p = WL.params(wl, prec, stream=stream.cuda_stream, rv=rv, rl=rl)
    rho0, u0 = WL.initial_fields(wl, rv, rl)

    dom = lbm.Domain(p)
    dom.lbm_init_fields(rho0, u0)
    dom.lbm_step(args.warmup)
    dom.lbm_synchronize()

    # ---- timed region: K steps, device-resident state
    barrier(world)
    torch.cuda.synchronize()
    dom.lbm_set_timing(True)
    launches0 = dom.lbm_launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(stream)
        dom.lbm_step(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
    launches = dom.lbm_launch_count() - launches0
    dom.lbm_synchronize()
    barrier(world)
    ms = e0.elapsed_time(e1)
    ms_max = max_over_ranks(ms, world)
    kms, kcnt = dom.lbm_kernel_times()
    dom.lbm_set_timing(False)
    clocks = clk.summary()
    mlups = whole_job_mlups(wl.N, args.steps, world, ms_max)

    # ---- end to end through the C ABI, host fields in the library's page-locked
    #      huge-page buffers (lbm_host_alloc): one for the 1 + D input fields, one for
    #      the 1 + D output fields
    nb = wl.N * 8
    h_in, h_out = lbm.HostBuffer((1 + wl.D) * nb), lbm.HostBuffer((1 + wl.D) * nb)
    for k, a in enumerate([rho0] + [u0[c] for c in range(wl.D)]):
        np.copyto(h_in.array(np.float64, wl.N, k * nb), np.ravel(a))
    in_ptrs = [h_in.ptr + k * nb for k in range(1 + wl.D)] + ([None] if wl.D == 2 else [])
    out_ptrs = [h_out.ptr + k * nb for k in range(1 + wl.D)] + ([None] if wl.D == 2 else [])
    o_rho = h_out.array(np.float64, wl.N, 0)
    # two untimed passes through the same two calls, so that the timed passes do not
    # pay for first use of the library's device memory pool or of the host buffers
    for _ in range(2):
        dom.lbm_init_fields_ptr(*in_ptrs)
        dom.lbm_read_macroscopic_ptr(*out_ptrs)
    # E2E_REPEATS timed passes, the median reported (single passes scattered by up to
    # 80% from run to run, all of it in the host copies)
    e2e_runs = []
    for _ in range(E2E_REPEATS):
        barrier(world)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        dom.lbm_init_fields_ptr(*in_ptrs)
        dom.lbm_step(args.steps)
        dom.lbm_read_macroscopic_ptr(*out_ptrs)
        e2e_runs.append(max_over_ranks(time.perf_counter() - t0, world))
        assert np.isfinite(o_rho).all(), "non-finite density after the e2e run"
    e2e_s = sorted(e2e_runs)[len(e2e_runs) // 2]
    e2e_mlups = wl.N * args.steps * world / e2e_s / 1e6
    dom.close()
    del o_rho
    h_in.close()
    h_out.close()

    if rank != 0:
        return 0
    peaks, peak_kind = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", PEAKS_FALLBACK["hbm_gbs"]))
    k2_ms = kms[1] / max(1, kcnt[1])
    k1_ms = kms[0] / max(1, kcnt[0])
    Q = 27 if wl.D == 3 else 9
    full_fp32 = args.precision == "fp32" and wl.N == 512 * 512 * 256
    k2_bytes = algorithmic_bytes_k2(wl, pop_bytes, 8 if pop_bytes == 8 else 4)
    if args.precision == "fp16dev":
        k2_bytes += wl.N * 8  # writer densities: one read (the neighbours' are cache hits), one write
    k1_bytes = algorithmic_bytes_k1(wl, pop_bytes, 8 if pop_bytes == 8 else 4)
    if args.precision == "fp16dev":
        k1_bytes += wl.N * 4  # writer densities read by the decode
    traffic = recorded_traffic("d3q27_fp32_collide_stream") if full_fp32 else None
    t_p1 = recorded_traffic("d3q27_fp32_moments_eos") if full_fp32 else None
    t_p1b = recorded_traffic("d3q27_fp32_qflux_tile") if full_fp32 else None
    traffic_k1 = t_p1 + t_p1b if t_p1 is not None and t_p1b is not None else None
    achieved = k2_bytes / (k2_ms * 1e-3) / 1e9
    step_achieved = (k1_bytes + k2_bytes) / ((k1_ms + k2_ms) * 1e-3) / 1e9
    both = traffic is not None and traffic_k1 is not None
    metric, config = metric_and_config(args, wl, world)
    line = {
        "metric": metric,
        "value": mlups, "unit": "MLUPS", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp64": "f64", "fp32": "f32", "fp16dev": "f16 storage, f32 arithmetic"}[args.precision],
        "data": "synthetic",
        "config": config,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": traffic, "peak_kind": peak_kind,
                     "kernel": "collide_stream (force + collide + stream)",
                     "algorithmic_bytes_per_launch": k2_bytes,
                     "kernel_ms": k2_ms},
        # the whole step, all its kernels together: their algorithmic bytes (and the
        # recorded DRAM bytes) over their summed CUDA-event times
        "step_roofline": {"kernels": "moments_eos + qflux_tile + collide_stream", "unit": "GB/s", "peak": hbm,
                          "achieved": step_achieved, "frac": step_achieved / hbm,
                          "algorithmic_bytes_per_step": k1_bytes + k2_bytes,
                          "traffic_per_step": (traffic + traffic_k1) if both else None,
                          "dram_frac": ((traffic + traffic_k1) / ((k1_ms + k2_ms) * 1e-3) / 1e9 / hbm)
                          if both else None,
                          "bytes_per_lup_floor": 2 * Q * pop_bytes,
                          "frac_of_floor": mlups / world * 1e6 * 2 * Q * pop_bytes / (hbm * 1e9),
                          "moments_eos_qflux_ms": k1_ms, "collide_stream_ms": k2_ms},
        "e2e": {"value": e2e_mlups, "unit": "MLUPS",
                "h2d_bytes_per_step": (1 + wl.D) * wl.N * 8 / args.steps,
                "d2h_bytes_per_step": (1 + wl.D) * wl.N * 8 / args.steps,
                "what": "lbm_init_fields from host arrays + K steps + lbm_read_macroscopic to host arrays, "
                        "the arrays in page-locked huge-page buffers of lbm_host_alloc; "
                        f"median of {E2E_REPEATS} passes", "passes_s": e2e_runs},
        "gpu_launches": launches,
        "clocks": clocks,
    }
    if world == 1 and args.serve_jobs > 0:
        line["serving"] = serving_sample(args.serve_jobs, args.serve_scale)
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_sample(wl)
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serve-jobs", type=int, default=200,
                    help="jobs of the served-latency sample added to the line at N = 1 (0: none)")
    ap.add_argument("--serve-scale", type=float, default=0.25,
                    help="fraction of each served job's 1,000-10,000 steps")
    ap.add_argument("--precision", choices=["fp32", "fp64", "fp16dev"], default="fp32",
                    help="population storage/arithmetic of the timed path (fp32 is the headline)")
    ap.add_argument("--workload", default="drop3d", choices=["drop3d", "drop3d-small", "drop2d", "static2d"],
                    help="drop3d (default, D3Q27 512x512x256), drop3d-small (256x256x128, the profiling "
                    "case), drop2d (D2Q9 2048x1024) or static2d (D2Q9 128x128 static drop, T/Tc = 0.8)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
