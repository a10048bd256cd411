#!/usr/bin/env python
"""Benchmark: complete hpG solves per second on one GB300 (per rank), FP32-inner
mixed precision (headline) and plain FP64, on the 32x32-cell, p = 8 radial
obstacle (66,049 u-dofs incl. boundary, 50,176 psi-dofs; 10 proximal steps).

One "step" = one complete hpG solve (all alpha_k subproblems, every Newton
step with its Schur/GMRES solve) from psi_0 = 0, with the problem data already
resident on the device.  The e2e figure goes through the C ABI with host
buffers: each step uploads phi at the Gauss points from host memory, solves,
and reads u_h and psi_h back.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  Multi-GPU: one independent replica per rank
(the solves do not shard), barrier + max over ranks.
"""
import os

# the oracle baseline runs single-threaded (SuperLU is sequential; BLAS pinned to 1 thread)
for _v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import argparse
import json
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "radial32"
METRIC = "solves/s (complete hpG solve at 1e-8 rel err vs FP64 oracle), mixed vs FP64; DoF*Krylov-its/s"


def rank_info():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        load = [s for s in sm if smax and s > 0.5 * max(smax)] or sm
        return {"sm_mhz": statistics.median(load) if load else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------ oracle leg
def oracle_sample(max_alpha_steps=1):
    """Time the CPU oracle on a bounded sample of the workload: its setup plus
    the first `max_alpha_steps` proximal subproblems; extrapolate linearly in
    Newton steps to one complete solve (Newton count of the full solve taken
    from the stored oracle run, else 34)."""
    from paper_2412_13733_gb300 import workloads as W
    from oracle.hpg import ObstacleOracle
    w = W.workload(WORKLOAD)
    golden = os.path.join(ROOT, "tests", "golden", f"{WORKLOAD}_oracle.npz")
    total_newton = int(np.load(golden)["newton"].sum()) if os.path.exists(golden) else 34
    t0 = time.perf_counter()
    o = ObstacleOracle(w["breakpoints"], w["p"], w["f"], w["phi"], w["g"], beta=w["beta"], lower=w["lower"])
    t_setup = time.perf_counter() - t0
    r = o.solve(w["alphas"][:max_alpha_steps], tol=w["tol"])
    t_newton = time.perf_counter() - t0 - t_setup
    done = sum(r["newton"])
    t_full = t_setup + t_newton * total_newton / max(done, 1)
    return dict(value=1.0 / t_full, seconds=time.perf_counter() - t0, newton_done=done, total_newton=total_newton,
                t_setup=t_setup, t_newton=t_newton)


def cpu_threads():
    return int(os.environ.get("OPENBLAS_NUM_THREADS", "1"))


def run_reference(args):
    rank, _, world = rank_info()
    if rank != 0:
        return 0
    for _ in range(args.warmup if args.warmup < 1 else 1):
        pass
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vals.append(oracle_sample()["value"])
    wall = time.perf_counter() - t0
    v = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * wall / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "radial obstacle 32x32 cells p=8 (66049 u-dofs, 50176 psi-dofs), 10 alpha steps",
                       "l2_flush": "n/a (CPU)"},
            "cpu_baseline": {"value": v, "unit": "solves/s", "cores": cpu_threads(), "kind": "oracle",
                             "sample": "oracle setup + first alpha subproblem per step, extrapolated in Newton steps"},
            "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ GPU legs
def algorithmic_work(P, w):
    """Per-launch algorithmic FLOPs / bytes of the kernel classes."""
    d = len(w["breakpoints"])
    n1 = [len(b) - 1 for b in w["breakpoints"]]
    n1 = [m * w["p"] - 1 for m in n1]
    Nu0 = P.n_u
    Npsi = P.n_psi
    n = w["p"] - 1
    Nc = P.cells
    nb = n ** d
    fdm_flops = sum(2.0 * n1[ax] * Nu0 * 2 for ax in range(d))       # d forward + d backward GEMM passes
    newton_bytes = 8.0 * (2 * (Nu0 + Npsi) + Npsi)                   # x in, y out, Gauss weights
    newton_flops = 2.0 * (3 * d * 3) * Nu0 + 2.0 * 16 * Npsi + 2.0 * 2 * d * n * Npsi
    factor_flops = Nc * (nb ** 3 / 3.0 + nb ** 3 / 3.0 + nb ** 3 / 3.0) * 2.0
    precond_bytes = Nc * nb * nb * 4.0                              # FP32 inverse blocks read once
    return dict(fdm=("alu", fdm_flops, "TFLOP/s"), newton_apply=("alu", newton_flops, "TFLOP/s"),
                factor=("alu", factor_flops, "TFLOP/s"), precond=("hbm", precond_bytes, "GB/s"),
                newton_apply_bytes=newton_bytes)


def alu_peak_tflops(kind, clock_mhz):
    """Derived ALU peaks (152 SMs): FP32 128 FMA/clk/SM, FP64 nominal 1.25 TFLOP/s at 2070 MHz."""
    if kind == "fp32":
        return 152 * 128 * 2 * clock_mhz * 1e6 / 1e12
    return 1.25 * clock_mhz / 2070.0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    rank, local_rank, world = rank_info()
    import torch
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    from paper_2412_13733_gb300 import hpg, workloads as W
    if not os.path.exists(hpg.LIB_PATH):
        from paper_2412_13733_gb300 import build
        build.build()

    def barrier():
        if dist is not None:
            dist.barrier()

    w = W.workload(WORKLOAD)
    stream = torch.cuda.current_stream()
    ctx = hpg.Context(local_rank, stream=stream.cuda_stream)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")   # 256 MB > 126 MB L2
    peaks, peak_src = load_peaks()

    def timed(P, steps, e2e=False, host_phi=None):
        times = []
        d2h = 0
        for _ in range(steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            if e2e:
                P.set_constraint_values(host_phi)
                P.solve()
                u = P.u()
                psi = P.psi()
                d2h = 8 * (P.n_u + P.n_psi)
            else:
                P.solve()
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        return times, d2h

    results = {}
    precisions = [("mixed", hpg.HPG_MIXED)] + ([] if args.no_fp64 else [("fp64", hpg.HPG_FP64)])
    clocks = None
    for name, prec in precisions:
        P = hpg.from_workload(ctx, w, hpg.default_params(precision=prec))
        for _ in range(args.warmup):
            P.solve()
        st = P.stats()
        sampler = ClockSampler(local_rank) if name == "mixed" else None
        if sampler:
            sampler.start()
        barrier()
        torch.cuda.synchronize()
        t_wall0 = time.perf_counter()
        times, _ = timed(P, args.steps)
        torch.cuda.synchronize()
        barrier()
        t_wall = time.perf_counter() - t_wall0
        if sampler:
            clocks = sampler.stop()
        st = P.stats()
        total_ms = sum(times)
        if dist is not None:
            t = torch.tensor([total_ms], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            total_ms = float(t.item())
        dofs = P.n_u + P.n_psi
        res = dict(value=world * args.steps / (total_ms / 1000.0), ms_per_step=total_ms / args.steps,
                   wall_s=t_wall, newton=st["newton_total"], krylov=st["krylov_total"],
                   refine=st["refine_total"], launches=st["kernel_launches"],
                   dof_krylov_per_s=world * dofs * st["krylov_total"] / (total_ms / args.steps / 1000.0))
        # e2e through the C ABI with host buffers
        host_phi = np.ascontiguousarray(w["phi"](P.quad_points()), dtype=np.float64)
        host_phi_pinned = torch.from_numpy(host_phi).pin_memory().numpy()
        times_e2e, d2h = timed(P, args.steps, e2e=True, host_phi=host_phi_pinned)
        st2 = P.stats()
        e2e_ms = sum(times_e2e)
        res["e2e"] = dict(value=world * args.steps / (e2e_ms / 1000.0), unit="solves/s",
                          h2d_bytes_per_step=int(st2["h2d_bytes"]), d2h_bytes_per_step=int(d2h))
        # per-kernel-class device time: a second pass of the same steps with event pairs
        prm = hpg.default_params(precision=prec, timing=1)
        prm.beta = w["beta"]
        P.set_params(prm)
        P.solve()
        P.reset_kernel_times()
        for _ in range(args.steps):
            flush.zero_()
            P.solve()
        torch.cuda.synchronize()
        res["kernels"] = P.kernel_times()
        res["work"] = algorithmic_work(P, w)
        results[name] = res
        P.free()

    mixed = results["mixed"]
    # dominant kernel of the headline (mixed) path
    kt = mixed["kernels"]
    dom = max(kt, key=lambda k: kt[k][0])
    clock_mhz = (clocks or {}).get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    work = mixed["work"]
    roof = None
    if dom in ("fdm", "factor", "newton_apply"):
        kind, flops, unit = work[dom]
        avg_ms = kt[dom][0] / max(kt[dom][1], 1)
        ach = flops / (avg_ms / 1000.0) / 1e12
        fp = "fp64" if dom == "newton_apply" else "fp32"
        peak = alu_peak_tflops(fp, peaks.get("sm_max_mhz", 2070.0))
        roof = {"kernel": dom, "bound": "alu", "achieved": ach, "peak": peak, "unit": unit, "frac": ach / peak,
                "traffic": None, "peak_source": f"derived {fp} ALU peak at {peaks.get('sm_max_mhz', 2070.0)} MHz"}
    elif dom == "precond":
        kind, byts, unit = work["precond"]
        avg_ms = kt[dom][0] / max(kt[dom][1], 1)
        ach = byts / (avg_ms / 1000.0) / 1e9
        roof = {"kernel": dom, "bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": ach / peaks["hbm_gbs"], "traffic": None, "peak_source": peak_src}
    else:
        avg_ms = kt[dom][0] / max(kt[dom][1], 1)
        roof = {"kernel": dom, "bound": "latency", "achieved": None, "peak": None, "unit": None, "frac": None,
                "traffic": None, "avg_launch_ms": avg_ms}
    # FP64 matrix-free Newton apply (the refinement residual kernel) against its own roofline
    na = kt.get("newton_apply", (0.0, 0))
    newton_roof = None
    if na[1] > 0:
        avg = na[0] / na[1] / 1000.0
        _, fl, _ = work["newton_apply"]
        t_alu = fl / (alu_peak_tflops("fp64", peaks.get("sm_max_mhz", 2070.0)) * 1e12)
        t_hbm = work["newton_apply_bytes"] / (peaks["hbm_gbs"] * 1e9)
        newton_roof = {"bound": "alu" if t_alu > t_hbm else "hbm", "roofline_us": max(t_alu, t_hbm) * 1e6,
                       "avg_us": avg * 1e6, "frac": max(t_alu, t_hbm) / avg}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        s = oracle_sample()
        cpu = {"value": s["value"], "unit": "solves/s", "cores": cpu_threads(), "kind": "oracle",
               "sample": (f"oracle setup + first alpha subproblem ({s['newton_done']} of {s['total_newton']} "
                          f"Newton steps, {s['seconds']:.1f} s), extrapolated linearly in Newton steps")}

    if rank == 0:
        line = {"metric": METRIC, "value": mixed["value"], "unit": "solves/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": mixed["ms_per_step"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
                "data": "synthetic (analytic radial obstacle; no dataset)",
                "config": {"workload": "radial obstacle 32x32 cells p=8 (66049 u-dofs, 50176 psi-dofs), "
                                       "10 alpha steps, Newton tol 1e-10",
                           "precision": "FP32 inner Schur/GMRES operator in FP64 iterative refinement",
                           "l2_flush": "256 MB buffer zeroed before every timed step",
                           "parallelism": f"replicas x{world}"},
                "dof_krylov_its_per_s": mixed["dof_krylov_per_s"],
                "fp64": {"value": results["fp64"]["value"], "ms_per_step": results["fp64"]["ms_per_step"],
                         "dof_krylov_its_per_s": results["fp64"]["dof_krylov_per_s"],
                         "e2e": results["fp64"]["e2e"], "newton": results["fp64"]["newton"],
                         "krylov": results["fp64"]["krylov"]} if "fp64" in results else None,
                "mixed_over_fp64": (mixed["value"] / results["fp64"]["value"]) if "fp64" in results else None,
                "newton": mixed["newton"], "krylov": mixed["krylov"], "refine_sweeps": mixed["refine"],
                "e2e": mixed["e2e"], "gpu_launches": int(mixed["launches"] * args.steps),
                "roofline": roof, "newton_apply_roofline": newton_roof,
                "kernel_ms_per_step": {k: v[0] / args.steps for k, v in kt.items()},
                "clocks": clocks, "cpu_baseline": cpu}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    ctx.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
