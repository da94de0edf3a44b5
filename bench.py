#!/usr/bin/env python
"""Benchmark: P_N solve time to relative residual 1e-6 on GB300, and the
operator's throughput against HBM.

Workload (one step = one whole solve): P5 (36 real SH coefficients per
location) on 64^3 cells, seeded 4-octave value-noise fBm extinction in
[0.5, 40], albedo 0.95, Henyey-Greenstein g = 0.3, point source at a seeded
voxel, vacuum boundary; FP32 GMRES inner solves with FP64 iterative
refinement (FP64 residual, inner products, Givens) to ||Q - A u|| / ||Q|| <=
1e-6, starting from u = 0.  Synthetic data, generated in pn_inputs.

Prints ONE JSON line (rank 0).  Under torchrun every rank solves its own
replica (seed = rank): the method has no data exchange between independent
problems, so there is no collective on the data path (weak scaling).

--impl reference times the FP64 CPU oracle (GMRES on its matrix-free
operator) on the same workload, on the host cores, as a bounded sample per
step extrapolated to a whole solve.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "P_N solve time to rel. residual 1e-6 (learned vs plain); apply GDOF/s vs HBM"
WORKLOAD = "P5 64^3 fBm sigma_t[0.5,40] albedo 0.95 g 0.3 point source, solve to rel. residual 1e-6 (plain)"
FALLBACK_HBM_GBS = 6800.0
L2_FLUSH_BYTES = 512 << 20

# DRAM traffic of the dominant kernel from one ncu capture of the current
# kernel (dram__bytes_read.sum + dram__bytes_write.sum over the algorithmic
# bytes of the same launches, in the committed ncu summaries), keyed by kernel and
# workload (the staged kernels run from five basis vectors on, the direct ones
# below: the ratio of the kernel that carries most of the bytes is used).
# Launches differ in the number of basis vectors, so the mean ratio is
# applied to this run's average algorithmic bytes per launch.  An entry is
# removed when its kernel changes (traffic is then reported as null).
NCU_TRAFFIC = {("k_mdot16_tma", "p5_64"): 1.076, ("k_maxpy16_tma", "p5_64"): 1.049}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--restart", type=int, default=12)
    ap.add_argument("--inner-tol", type=float, default=1e-2)
    ap.add_argument("--ortho", choices=["cgs2", "cgs1"], default="cgs1")
    ap.add_argument("--basis", choices=["f32", "f16"], default="f16",
                    help="element type of the stored Krylov basis of the inner FP32 GMRES (the other one is "
                         "timed too and reported under alt_basis)")
    ap.add_argument("--no-apply-scan", action="store_true", help="skip the separate operator throughput scan")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true", help="skip the CPU oracle timing")
    ap.add_argument("--no-config5", action="store_true", help="skip the P7 256^3 cloud solve within a budget")
    ap.add_argument("--config5-iters", type=int, default=300,
                    help="inner-iteration budget of the P7 256^3 cloud solve")
    ap.add_argument("--no-paper-cgls", action="store_true",
                    help="skip the GPU FP64 CGLS solve (the paper's method) of the same workload")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-vs-plain comparison")
    ap.add_argument("--apply-only", action="store_true",
                    help="time only the FP32 operator on the P_N cloud medium given by --apply-n / --apply-r")
    ap.add_argument("--access-probe", action="store_true",
                    help="bandwidth of a plain copy with the tiled operator's access pattern (P7 and P5 plane "
                         "counts at --apply-r^3) against tile shape and loads in flight, next to the operator")
    ap.add_argument("--threshold-sweep", action="store_true",
                    help="iterations / time to 1e-6 vs the sigma_t threshold on the 64^3 cloud medium")
    ap.add_argument("--checkerboard", action="store_true",
                    help="2D checkerboard (7 x 7 blocks, 71 x 71 cells): P1 and P5 solve time to 1e-10")
    ap.add_argument("--batched", action="store_true",
                    help="many-instance workload: batched solve of --batch-count systems vs one-by-one solves")
    ap.add_argument("--batch-count", type=int, default=64)
    ap.add_argument("--batch-restart", type=int, default=15, help="--batched: GMRES restart of both arms")
    ap.add_argument("--batch-seed", type=int, default=0)
    ap.add_argument("--batch-rmin", type=int, default=24)
    ap.add_argument("--batch-rmax", type=int, default=96)
    ap.add_argument("--network-only", action="store_true",
                    help="time the learned preconditioner's network (P3: 19 input, 16 output channels): forward at "
                         "64^3 and a training step (batch 8 at 32^3) with the tcgen05 and the mma.sync convolutions")
    ap.add_argument("--large-solve", action="store_true",
                    help="the P7 256^3 cloud (1.08 G unknowns) solved by FP16-basis refinement, capped at "
                         "--large-iters inner iterations: time per iteration and the residual reached")
    ap.add_argument("--large-iters", type=int, default=600)
    ap.add_argument("--large-sigma-min", type=float, default=0.1)
    ap.add_argument("--seed", type=int, default=0, help="medium seed offset (the medium of rank r is seed + r)")
    ap.add_argument("--stream-tma", type=int, default=3,
                    help="FP16-basis GMRES: bulk-copy staged multi-dot (bit 0) and multi-axpy (bit 1)")
    ap.add_argument("--no-pdl", action="store_true",
                    help="launch the Arnoldi-step kernels without programmatic dependent launch")
    ap.add_argument("--no-l2-resident", action="store_true",
                    help="do not keep the solver's FP32 step vectors resident in L2")
    ap.add_argument("--augment", type=int, default=4,
                    help="LGMRES: corrections of earlier restart cycles appended to each cycle (FP16 basis)")
    ap.add_argument("--apply-n", type=int, default=7)
    ap.add_argument("--apply-kernel", choices=["auto", "tma", "register"], default="auto",
                    help="main kernel of the tiled operator (auto: the autotuner's pick)")
    ap.add_argument("--apply-r", type=int, default=256)
    return ap.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [r.split(",") for r in self.file.read().strip().splitlines() if r.strip()]
        os.unlink(self.file.name)
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


def dist_init(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        dist.init_process_group(backend=backend)
    return rank, world, local


def max_over_ranks(v: float, world: int, device=None) -> float:
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ----------------------------------------------------------------------------
# CPU oracle timing (the reference arm and the cpu_baseline object): the
# paper's solver -- CG on the normal equations without forming A^T A
# (section "Results"; oracle.pn.cgls) -- on the oracle's explicitly assembled
# FP64 CSR matrix (section "Runtime"), its sparse products split into row
# blocks over all host cores.

def host_threads() -> int:
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:
        return max(1, os.cpu_count() or 1)


class ThreadedCSR:
    """y = A v and y = A^T v for a SciPy CSR matrix, the rows of A (and of
    A^T) split into one contiguous block per thread.  SciPy's sparse products
    release the GIL, so the blocks run on separate cores."""

    def __init__(self, A, threads: int):
        import numpy as np
        from concurrent.futures import ThreadPoolExecutor
        self.n = A.shape[0]
        self.threads = threads
        self.bounds = np.linspace(0, self.n, threads + 1).astype(np.int64)
        AT = A.T.tocsr()
        self.rows = [A[self.bounds[i]:self.bounds[i + 1]] for i in range(threads)]
        self.rows_t = [AT[self.bounds[i]:self.bounds[i + 1]] for i in range(threads)]
        self.pool = ThreadPoolExecutor(threads)

    def _prod(self, blocks, v):
        import numpy as np
        out = np.empty(self.n)

        def part(i):
            out[self.bounds[i]:self.bounds[i + 1]] = blocks[i] @ v
        list(self.pool.map(part, range(self.threads)))
        return out

    def matvec(self, v):
        return self._prod(self.rows, v)

    def rmatvec(self, v):
        return self._prod(self.rows_t, v)

    # the matrix interface oracle.pn.cgls uses: A @ v and A.T @ v
    def __matmul__(self, v):
        return self.matvec(v)

    @property
    def T(self):
        outer = self

        class _Transposed:
            def __matmul__(self, v):
                return outer.rmatvec(v)
        return _Transposed()

    def close(self):
        self.pool.shutdown()


def oracle_cgls_setup(seed: int):
    """The oracle's CSR of the bench workload (untimed setup) and its
    right-hand side, with a threaded product over all host cores."""
    import pn_inputs
    from oracle import pn as opn
    p = pn_inputs.p5_64_fbm(seed)
    S = opn.assemble(p.N, p.R, opn.Medium(p.sigma_t, p.albedo, p.g, p.Q00, p.sigma_t_min))
    return ThreadedCSR(S.A, host_threads()), S.b


def oracle_cgls_sample(op, b, iters: int):
    """Seconds of the oracle's CGLS set-up (initial residual and A^T r) and
    seconds per CGLS iteration, from one run of `iters` iterations."""
    from oracle import pn as opn
    t0 = time.perf_counter()
    opn.cgls(op, b, tol=1e-300, max_iter=0)
    t1 = time.perf_counter()
    opn.cgls(op, b, tol=1e-300, max_iter=iters)
    t2 = time.perf_counter()
    return t1 - t0, max((t2 - t1) - (t1 - t0), 0.0) / iters


def run_reference(args):
    rank, world, _ = dist_init(args)
    if rank != 0:
        return
    op, b = oracle_cgls_setup(0)
    times, walls = [], []
    t_setup = per_iter = 0.0
    for s in range(args.warmup + args.steps):
        w0 = time.perf_counter()
        t_setup, per_iter = oracle_cgls_sample(op, b, REF_SAMPLE_ITERS)
        w1 = time.perf_counter()
        if s >= args.warmup:
            times.append(t_setup + per_iter * REF_CGLS_ITERS)
            walls.append(w1 - w0)
    op.close()
    sec = statistics.mean(times)
    value = 1.0 / sec
    sample = (f"{REF_SAMPLE_ITERS} CGLS iterations (the paper's CG on the normal equations) per step on the "
              f"oracle's FP64 CSR of the full P5 64^3 problem, products split over {op.threads} host threads; "
              f"solve time extrapolated to the {REF_CGLS_ITERS} iterations the same method (FP64 CGLS) needs on "
              f"this workload on the GPU")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solve/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.mean(walls) * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "solver": "oracle CGLS FP64 (oracle.pn.cgls) on the assembled CSR"},
        "extrapolated": {"seconds_per_iteration": per_iter, "setup_seconds": t_setup, "iterations": REF_CGLS_ITERS,
                         "seconds_per_solve": sec, "ms_per_step_is": "wall time of the step's sample"},
        "cpu_baseline": {"value": value, "unit": "solve/s", "cores": op.threads, "kind": "oracle",
                         "cpu_count": os.cpu_count(), "sample": sample},
        "e2e": {"value": value, "unit": "solve/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


REF_SAMPLE_ITERS = 10
CPU_SAMPLE_ITERS = 20
# iterations FP64 CGLS needs to reach 1e-6 on the P5 64^3 workload (medium
# seed 0), measured by the bench's own `paper_cgls` run of the library's FP64
# CGLS on GB300 (the GPU arm reports the count it measured next to this one)
REF_CGLS_ITERS = 650


# ----------------------------------------------------------------------------
# GPU arm

def apply_scan(torch, System, pn_inputs, hbm_peak):
    """Separately timed FP32 operator throughput on two workloads."""
    out = {}
    for name, maker in (("P7 256^3 cloud (working set >> L2)", lambda: pn_inputs.p7_256_cloud(0)),
                        ("P5 64^3 fBm (working set ~ L2)", lambda: pn_inputs.p5_64_fbm(0))):
        p = maker()
        sysm = System(p.N, p.R, p.sigma_t, p.albedo, p.g, p.Q00, sigma_t_min=p.sigma_t_min)
        lay = sysm.layout
        tiling = sysm.tune_apply()
        x = torch.rand(lay.n_elems, dtype=torch.float32, device="cuda")
        ys = [torch.empty_like(x) for _ in range(2)]
        for i in range(3):
            sysm.apply(x, ys[i % 2])
        torch.cuda.synchronize()
        n = 20
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for i in range(n):
            sysm.apply(x, ys[i % 2])
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1) / n
        V = p.R ** 3
        bytes_alg = (2 * lay.n_active + 2 * V) * 4
        gbs = bytes_alg / (ms * 1e-3) / 1e9
        out[name] = {"ms": ms, "gdof_s": lay.n_active / (ms * 1e-3) / 1e9, "gb_s": gbs,
                     "frac_of_hbm": gbs / hbm_peak, "dof": lay.n_active, "bytes_per_apply": bytes_alg,
                     "ctas_per_sm": tiling["ctas_per_sm"], "kernel": tiling["kernel"],
                     "face_serial": tiling["face_serial"]}
        sysm.close()
        del x, ys
        torch.cuda.empty_cache()
    return out


def config5_run(torch, args):
    """The P7 256^3 cloud workload (1.08 G unknowns): thresholded fBm with
    sigma_t up to 100 and empty regions clamped to sigma_t_min = 0.1, albedo
    0.99, g 0.6, the single-scatter source of a seeded collimated beam.  FP64
    refinement around the bench's FP32 LGMRES(12, 4) with the FP16 basis,
    capped at --config5-iters inner iterations (it does not reach 1e-6 within
    any budget a bench run can afford): CUDA events around the solve; the
    residual reached and the time per inner iteration.  The committed network
    is trained for P3 (16 coefficients), so there is no learned arm here."""
    import pn_inputs
    from paper_1807_00410_gb300 import System
    from paper_1807_00410_gb300 import pn as ppn
    p, (axis, sign, radius, centre) = pn_inputs.p7_256_cloud_beam(0)
    st = torch.tensor(p.sigma_t, dtype=torch.float64, device="cuda")
    Q = ppn.single_scatter_beam(p.N, st, p.albedo, p.g, axis, sign, radius, centre)
    sysm = System(p.N, p.R, st, p.albedo, p.g, Q, sigma_t_min=p.sigma_t_min)
    del Q
    torch.cuda.empty_cache()
    tiling = sysm.tune_apply()
    sysm.set_pdl(not args.no_pdl)
    u = sysm.zeros(torch.float64)
    opts = dict(solver="ir", tol=1e-6, restart=args.restart, inner_tol=args.inner_tol, ortho="cgs1", basis="f16",
                augment=args.augment, check_every=5, raise_on_error=False)
    sysm.solve(u, **dict(opts, max_iter=20))  # workspace (untimed)
    u.zero_()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    s = sysm.solve(u, **dict(opts, max_iter=args.config5_iters))
    e1.record()
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    dof = sysm.layout.n_active
    out = {"workload": "P7 256^3 thresholded-fBm cloud (sigma_t up to 100, empty regions at sigma_t_min 0.1), "
                       f"albedo 0.99, g 0.6, collimated beam (axis {axis}, sign {sign}, radius {radius}) "
                       "single-scatter source; FP64 IR around FP32 LGMRES"
                       f"({args.restart}, {args.augment}), FP16 basis",
           "dof": dof, "iteration_budget": args.config5_iters, "ms": ms, "iterations": s["iterations"],
           "outer_iterations": s["outer_iterations"], "rel_residual": s["rel_residual"], "status": s["status"],
           "converged_to_1e-6": s["status"] == 0, "ms_per_iteration": ms / max(1, s["iterations"]),
           "gdof_iterations_per_s": dof * s["iterations"] / (ms * 1e-3) / 1e9,
           "apply_kernel": tiling["kernel"], "apply_ctas_per_sm": tiling["ctas_per_sm"],
           "learned": "not applicable: the committed network is trained for P3 (16 coefficients), this is P7"}
    sysm.close()
    del u, st
    torch.cuda.empty_cache()
    return out


LEARNED_WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_1807_00410_gb300", "weights",
                               "p3_unet_hard.npy")


def learned_compare(torch, args, seeds=(90000, 90001)):
    """Learned vs plain: held-out P3 64^3 fBm media (sigma_t in [0.5, 80],
    albedo 0.8..0.99, g 0..0.6, point source) solved to 1e-6 by FP64
    refinement around the bench's plain solver (LGMRES(restart, augment) with
    its basis) and around flexible GMRES(15) with the committed network
    (training: learned.py --loss hard); CUDA events around each solve, best of
    two."""
    import numpy as np

    from paper_1807_00410_gb300 import Net, System
    from paper_1807_00410_gb300 import learned as L
    K = 16
    net = Net(K + 3, K)
    net.set_params(np.load(LEARNED_WEIGHTS))
    rows = []
    for seed in seeds:
        st, albedo, g = L.medium(seed, 64)
        Q = np.zeros((64, 64, 64))
        Q[L.sources(seed, 64, 1)[0][1]] = float(64 ** 3)
        sysm = System(3, 64, st, albedo, g, Q)
        row = {"seed": seed}
        for mode in ("plain", "learned"):
            best = None
            for _ in range(2):
                u = sysm.zeros(torch.float64)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                if mode == "plain":
                    s = sysm.solve(u, solver="ir", tol=1e-6, restart=args.restart, ortho="cgs1", basis=args.basis,
                                   augment=args.augment if args.basis == "f16" else 0)
                else:
                    s = sysm.solve(u, solver="ir_fgmres", tol=1e-6, restart=15, ortho="cgs1", precond=net)
                e1.record()
                e1.synchronize()
                ms = e0.elapsed_time(e1)
                if best is None or ms < best["ms"]:
                    best = {"ms": ms, "iterations": s["iterations"], "rel_residual": s["rel_residual"],
                            "fallback": s["fallback"], "precond_applications": s["precond_applications"]}
            row[mode] = best
        rows.append(row)
        sysm.close()
    net.close()
    return {"workload": "P3 64^3 fBm sigma_t[0.5,80], held-out seeds, point source, to 1e-6",
            "plain": f"LGMRES({args.restart}, {args.augment if args.basis == 'f16' else 0}), {args.basis} basis",
            "learned": "flexible GMRES(15) with the network, FP32 basis",
            "plain_ms_mean": float(np.mean([r["plain"]["ms"] for r in rows])),
            "learned_ms_mean": float(np.mean([r["learned"]["ms"] for r in rows])), "rows": rows}


def run_ours(args):
    import torch

    import pn_inputs
    from paper_1807_00410_gb300 import System

    rank, world, local = dist_init(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    hbm_peak, peak_src = peaks()
    p = pn_inputs.p5_64_fbm(rank + args.seed)
    sysm = System(p.N, p.R, p.sigma_t, p.albedo, p.g, p.Q00, sigma_t_min=p.sigma_t_min)
    lay = sysm.layout
    tiling = sysm.tune_apply()  # the operator's kernel and z-chunking, picked by timing (setup, untimed)
    sysm.set_l2_residency(not args.no_l2_resident)
    sysm.set_stream_kernels(args.stream_tma)
    sysm.set_pdl(not args.no_pdl)
    if args.apply_kernel != "auto":
        sysm.set_apply_kernel(args.apply_kernel)
        tiling["kernel"] = sysm.apply_kernel
    u = sysm.zeros(torch.float64)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    opts = dict(solver="ir", tol=1e-6, restart=args.restart, inner_tol=args.inner_tol, max_iter=30000,
                check_every=8, ortho=args.ortho, basis=args.basis,
                augment=args.augment if args.basis == "f16" else 0)
    for _ in range(args.warmup):
        u.zero_()
        sysm.solve(u, **opts)
    torch.cuda.synchronize()
    barrier(world)
    sampler = ClockSampler(local)
    sampler.start()
    torch.cuda.synchronize()
    barrier(world)
    t_wall0 = time.perf_counter()
    step_ms, stats, prof, prof_ms = [], [], {}, []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # the timed solves (the value); then the same solves again with the
    # library's per-launch CUDA events on (the kernel breakdown and roofline),
    # so that the events' own cost stays out of the value
    for profiled in (False, True):
        for k in range(args.steps):
            flush.fill_(float(k))  # evict L2 between timed solves
            u.zero_()
            e0.record()
            st = sysm.solve(u, profile=profiled, **opts)
            e1.record()
            e1.synchronize()
            if not profiled:
                step_ms.append(e0.elapsed_time(e1))
                stats.append(st)
                continue
            prof_ms.append(e0.elapsed_time(e1))
            for kind, v in sysm.profile().items():
                agg = prof.setdefault(kind, {"ms": 0.0, "launches": 0, "bytes": 0.0})
                for key in agg:
                    agg[key] += v[key]
    # the same solves with the other basis element type, for comparison
    alt = "f32" if args.basis == "f16" else "f16"
    alt_opts = dict(opts, basis=alt, augment=0)  # augmentation needs the FP16 basis
    alt_ms, alt_st = [], None
    for k in range(args.steps):
        flush.fill_(float(k))
        u.zero_()
        e0.record()
        alt_st = sysm.solve(u, **alt_opts)
        e1.record()
        e1.synchronize()
        alt_ms.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    barrier(world)
    wall = time.perf_counter() - t_wall0
    clocks = sampler.stop()
    total_ms = max_over_ranks(sum(step_ms), world, dev)
    ms_per_step = total_ms / args.steps
    value = world * args.steps / (total_ms * 1e-3)

    # dominant kernel class and its roofline
    kinds = {k: v for k, v in prof.items() if k != "scalar" and v["launches"] > 0}
    dom = max(kinds, key=lambda k: kinds[k]["ms"])
    d = kinds[dom]
    achieved = d["bytes"] / (d["ms"] * 1e-3) / 1e9
    f16 = args.basis == "f16"
    op = "k_apply_tma" if tiling["kernel"] == "tma" else "k_apply_tiled"
    md = ("k_mdot16_tma" if args.stream_tma & 1 else "k_mdot16_givens") if f16 else "k_mdot_givens_f32"
    mx = ("k_maxpy16_tma" if args.stream_tma & 2 else "k_maxpy16") if f16 else "k_maxpy_f32"
    kernels = {"apply": op, "residual": op, "mdot": md, "maxpy": mx, "dot": "k_dot_f32", "vector": "vector updates"}
    kernel_names = {"apply": f"{op}<5, OP_APPLY> + k_face_x", "residual": f"{op}<5, OP_RESIDUAL> + k_face_x",
                    "mdot": f"{md} (fused CGS1 step{', FP16 basis' if f16 else ''})",
                    "maxpy": f"{mx} (multi-axpy) + update", "dot": "k_dot_f32", "vector": "vector updates"}
    ratio = NCU_TRAFFIC.get((kernels.get(dom, dom), "p5_64"))
    traffic = ratio * d["bytes"] / d["launches"] if ratio else None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "traffic": traffic, "kernel": kernel_names.get(dom, dom),
                "kind": dom, "launches_per_step": d["launches"] / args.steps,
                "avg_launch_us": d["ms"] * 1e3 / d["launches"],
                "bytes_per_launch": d["bytes"] / d["launches"], "peak_source": f"{peak_src} hbm_gbs",
                "share_of_step": d["ms"] / sum(prof_ms), "profiled_ms_per_step": sum(prof_ms) / len(prof_ms)}
    breakdown = {k: {"ms_per_step": v["ms"] / args.steps, "launches_per_step": v["launches"] / args.steps,
                     "gb_s": (v["bytes"] / (v["ms"] * 1e-3) / 1e9) if v["ms"] > 0 else 0.0}
                 for k, v in prof.items()}

    learned = None if (args.no_learned or rank != 0) else learned_compare(torch, args)

    # end-to-end through the public API with host buffers
    e2e = None
    if args.e2e_steps > 0:
        pin = lambda a: torch.from_numpy(a).pin_memory()  # noqa: E731
        st_h, q_h = pin(p.sigma_t), pin(p.Q00)
        out_h = torch.empty(lay.n_elems, dtype=torch.float64).pin_memory()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            s2 = System(p.N, p.R, st_h, p.albedo, p.g, q_h, sigma_t_min=p.sigma_t_min)
            u2 = s2.zeros(torch.float64)
            s2.solve(u2, **opts)
            out_h.copy_(u2)
            torch.cuda.synchronize()
            s2.close()
        t_e2e = time.perf_counter() - t0
        t_e2e = max_over_ranks(t_e2e, world, dev)
        e2e = {"value": world * args.e2e_steps / t_e2e, "unit": "solve/s",
               "h2d_bytes_per_step": int(st_h.numel() * 8 + q_h.numel() * 8),
               "d2h_bytes_per_step": int(out_h.numel() * 8), "steps": args.e2e_steps}

    scan = None
    if rank == 0 and not args.no_apply_scan:
        scan = apply_scan(torch, System, pn_inputs, hbm_peak)

    config5 = None
    if rank == 0 and not args.no_config5:
        config5 = config5_run(torch, args)

    # the paper's own solver on the GPU: FP64 CG on the normal equations
    # (CGLS, the library's FP64 operator) on the same medium, to the same target
    paper = None
    if rank == 0 and not args.no_paper_cgls:
        cg_opts = dict(solver="cgls", tol=1e-6, max_iter=200000, check_every=50)
        u64 = sysm.zeros(torch.float64)
        sysm.solve(u64, **dict(cg_opts, max_iter=20), raise_on_error=False)  # workspace, untimed
        u64.zero_()
        torch.cuda.synchronize()
        e0.record()
        cst = sysm.solve(u64, **cg_opts, raise_on_error=False)
        e1.record()
        e1.synchronize()
        paper = {"solver": "CGLS (CG on the normal equations, the paper's method), FP64 vectors and operator",
                 "ms": e0.elapsed_time(e1), "iterations": cst["iterations"], "rel_residual": cst["rel_residual"],
                 "status": cst["status"], "vs_plain_solve": e0.elapsed_time(e1) / ms_per_step}
        del u64

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the oracle's CGLS on its CSR over all host cores: a bounded sample of
        # iterations on the full problem, extrapolated to the iterations the
        # same method needed on the GPU in this run
        iters = paper["iterations"] if paper and paper["status"] == 0 else None
        op, bvec = oracle_cgls_setup(0)
        t_setup, per_iter = oracle_cgls_sample(op, bvec, CPU_SAMPLE_ITERS)
        op.close()
        cpu = {"unit": "solve/s", "cores": op.threads, "cpu_count": os.cpu_count(), "kind": "oracle",
               "method": "oracle.pn.cgls: CG on the normal equations (the paper's solver), FP64, assembled CSR, "
                         f"sparse products split over {op.threads} threads",
               "seconds_per_iteration": per_iter, "setup_seconds": t_setup}
        if iters:
            cpu_sec = t_setup + per_iter * iters
            cpu.update({"value": 1.0 / cpu_sec, "seconds_per_solve": cpu_sec, "iterations": iters,
                        "sample": f"{CPU_SAMPLE_ITERS} CGLS iterations on the full P5 64^3 problem, extrapolated "
                                  f"to the {iters} iterations FP64 CGLS needed on the GPU in this run"})
        else:
            cpu.update({"value": None, "sample": "no GPU CGLS iteration count in this run: not extrapolated"})

    sysm.close()
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "solve/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f16-basis+f32+f64" if args.basis == "f16" else "f32+f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "dof": lay.n_active,
                       "solver": (f"FP64 iterative refinement around FP32 LGMRES({args.restart}, {opts['augment']})"
                                  if opts["augment"] else
                                  f"FP64 iterative refinement around FP32 GMRES({args.restart})"),
                       "restart": args.restart,
                       "augment": opts["augment"], "ortho": args.ortho, "l2_resident": not args.no_l2_resident,
                       "pdl": not args.no_pdl,
                       "stream_tma": args.stream_tma,
                       "basis": args.basis, "apply_ctas_per_sm": tiling["ctas_per_sm"], "apply_kernel": tiling["kernel"],
                       "apply_face_serial": tiling["face_serial"],
                       "inner_tol": args.inner_tol, "check_every": opts["check_every"], "l2": "flushed between timed solves (512 MiB write)",
                       "replicas": f"one independent problem per GPU (medium seed = {args.seed} + rank)"},
            "solve": {"iterations": stats[-1]["iterations"], "outer_iterations": stats[-1]["outer_iterations"],
                      "rel_residual": stats[-1]["rel_residual"], "wall_s": wall},
            "roofline": roofline,
            "breakdown": breakdown,
            "alt_basis": {"basis": alt, "ms_per_step": sum(alt_ms) / len(alt_ms),
                          "iterations": alt_st["iterations"], "rel_residual": alt_st["rel_residual"]},
            "apply": scan,
            "learned": learned,
            "paper_cgls": paper,
            "config5": config5,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": int(sum(s["launches"] for s in stats)),
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_apply_only(args):
    """Operator throughput alone: W warm-up and K timed FP32 applies on the
    thresholded-fBm cloud medium at order --apply-n on --apply-r^3 cells."""
    import torch

    import pn_inputs
    from paper_1807_00410_gb300 import System
    torch.cuda.set_device(0)
    hbm_peak, peak_src = peaks()
    p = pn_inputs.cloud_point(args.apply_n, args.apply_r, 0)
    sysm = System(p.N, p.R, p.sigma_t, p.albedo, p.g, p.Q00, sigma_t_min=p.sigma_t_min)
    lay = sysm.layout
    tiling = sysm.tune_apply()
    if args.apply_kernel != "auto":
        sysm.set_apply_kernel(args.apply_kernel)
    g = torch.Generator(device="cuda").manual_seed(0)
    x = torch.rand(lay.n_elems, dtype=torch.float32, device="cuda", generator=g)
    ys = [torch.empty_like(x) for _ in range(2)]
    for i in range(args.warmup):
        sysm.apply(x, ys[i % 2])
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for i in range(args.steps):
        sysm.apply(x, ys[i % 2])
    e1.record()
    e1.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    V = p.R ** 3
    bytes_alg = (2 * lay.n_active + 2 * V) * 4
    gbs = bytes_alg / (ms * 1e-3) / 1e9
    print(json.dumps({"mode": "apply-only", "workload": f"P{p.N} {p.R}^3 cloud FP32 apply", "ms": ms,
                      "gdof_s": lay.n_active / (ms * 1e-3) / 1e9, "gb_s": gbs, "frac": gbs / hbm_peak,
                      "peak": hbm_peak, "peak_source": peak_src, "dof": lay.n_active,
                      "bytes_per_apply": bytes_alg, "ctas_per_sm": tiling["ctas_per_sm"],
                      "kernel": sysm.apply_kernel, "face_serial": sysm.apply_plan["face_serial"], "steps": args.steps,
                      "warmup": args.warmup}), flush=True)
    sysm.close()


def run_access_probe(args):
    """What DRAM delivers to the tiled operator's access pattern without its
    arithmetic (pn_access_probe): copies of 64 and 36 planes (P7, P5) of an
    --apply-r^3 grid by 512-thread CTAs marching column tiles through z, for
    tile shapes 32 x 4, 64 x 2, 128 x 1 and 1, 2, 4 z-slices of loads in flight
    per thread (32, 64, 128 KB per CTA at 64 planes), as fractions of the
    measured copy peak."""
    import torch

    from paper_1807_00410_gb300 import pn as ppn
    torch.cuda.set_device(0)
    hbm_peak, peak_src = peaks()
    rows = []
    for planes in (64, 36):
        for tile_x in (32, 64, 128):
            for slices in (1, 2, 4):
                gbs = ppn.access_probe(args.apply_r, planes, tile_x, slices)
                rows.append({"planes": planes, "tile": f"{tile_x}x{128 // tile_x}", "slices_in_flight": slices,
                             "kb_in_flight_per_cta": planes * slices // 2, "gb_s": round(gbs, 1),
                             "frac": round(gbs / hbm_peak, 4)})
    print(json.dumps({"mode": "access-probe", "R": args.apply_r, "peak": hbm_peak, "peak_source": peak_src,
                      "rows": rows}), flush=True)


def run_threshold_sweep(args):
    """Convergence against the extinction threshold (the paper clamps sigma_t
    from below because vacuum makes A singular, section "Nebulae"): IR solves
    of the thresholded-fBm cloud (54 % empty voxels) at each threshold."""
    import torch

    import pn_inputs
    from paper_1807_00410_gb300 import System
    torch.cuda.set_device(0)
    rows = []
    for N in (1, 5):
        for smin in (1.0, 0.3, 0.1, 0.03):
            p = pn_inputs.cloud_point(N, 64, 0, sigma_t_min=smin)
            sysm = System(p.N, p.R, p.sigma_t, p.albedo, p.g, p.Q00, sigma_t_min=smin)
            u = sysm.zeros(torch.float64)
            st = sysm.solve(u, solver="ir", tol=1e-6, restart=args.restart, ortho=args.ortho, max_iter=200000,
                            basis=args.basis, augment=args.augment if args.basis == "f16" else 0,
                            raise_on_error=False)
            rows.append({"N": N, "sigma_t_min": smin, "iterations": st["iterations"],
                         "outer": st["outer_iterations"], "seconds": st["seconds"],
                         "rel_residual": st["rel_residual"], "status": st["status"]})
            sysm.close()
    print(json.dumps({"mode": "threshold-sweep", "workload": "64^3 thresholded-fBm cloud, albedo 0.99, g 0.6, "
                      f"point source, FP32 LGMRES({args.restart}, {args.augment}) ({args.basis} basis) + FP64 IR "
                      "to 1e-6", "rows": rows}), flush=True)


def run_checkerboard(args):
    """The 2D checkerboard (section "2D checkerboard": 7 x 7 unit blocks at
    71 x 71 cells, absorbing blocks sigma_a = 10, scattering blocks sigma_s =
    1) through the 2D reduction: solve time to the paper's residual 1e-10 for
    P1 and P5 (FP32 GMRES inside FP64 refinement), CUDA events around the
    solve, best of --steps after --warmup solves."""
    import torch

    import pn_inputs
    from paper_1807_00410_gb300 import System
    torch.cuda.set_device(0)
    st, al, Q = pn_inputs.checkerboard_2d(71)
    rows = []
    for N in (1, 3, 5):
        sysm = System(N, 71, st, al, 0.0, Q, dims=2)
        times = []
        for it in range(args.warmup + args.steps):
            u = sysm.zeros(torch.float64)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            s = sysm.solve(u, solver="ir", tol=1e-10, restart=30, ortho=args.ortho, max_iter=500000,
                           max_outer=100)
            e1.record()
            e1.synchronize()
            if it >= args.warmup:
                times.append(e0.elapsed_time(e1))
        rows.append({"N": N, "dof": sysm.layout.n_active, "ms": min(times), "ms_median": statistics.median(times),
                     "iterations": s["iterations"], "outer": s["outer_iterations"],
                     "rel_residual": s["rel_residual"], "launches": s["launches"]})
        sysm.close()
    print(json.dumps({"mode": "checkerboard", "workload": "2D checkerboard, 7 x 7 unit blocks on 71 x 71 cells, "
                      "sigma_a 10 / sigma_s 1, unit source in the centre block, vacuum boundary; FP32 GMRES(30) "
                      "+ FP64 IR to 1e-10", "rows": rows}), flush=True)


def run_batched(args):
    """The many-instance workload (--batch-count systems, grids 24..96 cells
    per axis, orders {1, 3, 5}, fBm extinction in [0.1, 60], point or beam
    sources): wall time of one batched solve to 1e-6 (CUDA events around
    pn_batch_solve, best of --steps after --warmup), against the same systems
    solved one after another with pn_solve (FP32 GMRES + FP64 refinement, the
    same restart and tolerance)."""
    import numpy as np
    import torch

    import pn_inputs
    from paper_1807_00410_gb300 import Batch, System
    from paper_1807_00410_gb300 import pn as ppn
    torch.cuda.set_device(0)
    inst = pn_inputs.batch_instances(args.batch_count, args.batch_seed, r_lo=args.batch_rmin, r_hi=args.batch_rmax)
    systems = []
    for b in inst:
        st = torch.tensor(b.sigma_t, dtype=torch.float64, device="cuda")
        if b.source[0] == "point":
            Q = torch.zeros((b.R,) * 3, dtype=torch.float64, device="cuda")
            Q[b.source[1][0], b.source[1][1], b.source[1][2]] = float(b.R ** 3)
        else:
            _, axis, sign, radius, centre = b.source
            Q = ppn.single_scatter_beam(b.N, st, b.albedo, b.g, axis, sign, radius, centre)
        systems.append(System(b.N, b.R, st, b.albedo, b.g, Q))
    dof = sum(s.layout.n_active for s in systems)
    batch = Batch(systems, restart=args.batch_restart, tune=True)
    tiling = batch.tiling()

    def timed(fn):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        out = fn()
        e1.record()
        e1.synchronize()
        return e0.elapsed_time(e1), out

    times, stats = [], None
    for it in range(args.warmup + args.steps):
        us = [s.zeros(torch.float64) for s in systems]
        ms, stats = timed(lambda: batch.solve(us, tol=1e-6, max_iter=200000, raise_on_error=False))
        if it >= args.warmup:
            times.append(ms)
    its = [st["iterations"] for st in stats]
    ok = sum(1 for st in stats if st["status"] == 0)
    solo_min = 1 << 18  # the library's default: instances at least this large are solved by pn_solve
    n_solo = sum(1 for s in systems if s.layout.n_active >= solo_min)
    # the same batch with every instance in the batched launches (tiling
    # re-tuned for that set)
    batch.set_solo(0)
    batch.tune()
    all_times = []
    for it in range(1 + max(1, args.steps // 2)):
        us = [s.zeros(torch.float64) for s in systems]
        ms_all, _ = timed(lambda: batch.solve(us, tol=1e-6, max_iter=200000, raise_on_error=False))
        if it >= 1:
            all_times.append(ms_all)
    batch.set_solo(solo_min)

    def one_by_one():
        out = []
        for s in systems:
            u = s.zeros(torch.float64)
            out.append(s.solve(u, solver="ir", tol=1e-6, restart=args.batch_restart, ortho=args.ortho, max_iter=200000,
                               raise_on_error=False))
        return out
    seq_ms, seq_stats = timed(one_by_one)
    best = min(times)
    print(json.dumps({
        "mode": "batched", "workload": f"{len(systems)} instances (pn_inputs.batch_instances, seed "
        f"{args.batch_seed}): grids {args.batch_rmin}..{args.batch_rmax} per axis, N in {{1,3,5}}, fBm sigma_t in "
        f"[0.1, 60], albedo 0.7..0.99, "
        f"g 0..0.7, point or beam source; FP32 GMRES({args.batch_restart}) + FP64 IR to 1e-6",
        "instances": len(systems), "dof": dof, "ms": best, "ms_median": statistics.median(times),
        "solves_per_s": len(systems) / (best * 1e-3), "converged": ok,
        "iterations_max": max(its), "iterations_mean": float(np.mean(its)),
        "launches": stats[0]["launches"], "tiling": tiling,
        "one_by_one_ms": seq_ms, "one_by_one_converged": sum(1 for st in seq_stats if st["status"] == 0),
        "one_by_one_launches": int(sum(st["launches"] for st in seq_stats)),
        "speedup_vs_one_by_one": seq_ms / best, "solo_min_unknowns": solo_min, "solo_instances": n_solo,
        "all_batched_ms": min(all_times), "all_batched_speedup_vs_one_by_one": seq_ms / min(all_times),
        "steps": args.steps, "warmup": args.warmup}), flush=True)
    batch.close()
    for s in systems:
        s.close()


def run_network_only(args):
    """The network alone: W warm-up and K timed forwards (batch 1 at 64^3, the
    preconditioner's size) and training steps (batch 8 at 32^3: forward,
    backward, Adam), CUDA events, for each convolution kernel."""
    import torch

    from paper_1807_00410_gb300 import Net
    from paper_1807_00410_gb300 import learned as L
    torch.cuda.set_device(0)
    K = 16
    net = Net(K + 3, K)
    net.set_params(L.init_params(K + 3, K, seed=1))
    g = torch.Generator(device="cuda").manual_seed(0)
    out = {}
    for kern in ("tcgen05", "mma_sync"):
        net.set_conv_kernel(kern)
        row = {}
        for what, (B, R) in (("forward", (1, 64)), ("train_step", (8, 32))):
            x = torch.randn((B, R, R, R, K + 3), device="cuda", generator=g)
            t = torch.randn((B, R, R, R, K), device="cuda", generator=g)
            fn = (lambda: net.forward(x)) if what == "forward" else (lambda: net.train_step(x, t, 1e-4))
            for _ in range(args.warmup):
                fn()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(args.steps):
                fn()
            e1.record()
            e1.synchronize()
            row[what + "_ms"] = e0.elapsed_time(e1) / args.steps
        out[kern] = row
    net.take_error()
    net.close()
    print(json.dumps({"mode": "network-only", "network": "U-Net 4 levels, widths 16/32/48/64, c_in 19, c_out 16",
                      "forward": "batch 1 at 64^3", "train_step": "batch 8 at 32^3 (forward, backward, Adam)",
                      "kernels": out, "steps": args.steps, "warmup": args.warmup}), flush=True)


def run_large_solve(args):
    """Full-size solve on the P7 256^3 thresholded-fBm cloud (albedo 0.99,
    g 0.6, sigma_t_min --large-sigma-min, seeded point source): IR with the
    bench's FP32 solver (LGMRES(--restart, --augment), FP16-stored basis),
    capped at --large-iters inner iterations; CUDA events around the solve."""
    import torch

    import pn_inputs
    from paper_1807_00410_gb300 import System
    torch.cuda.set_device(0)
    hbm_peak, peak_src = peaks()
    p = pn_inputs.cloud_point(7, 256, 0, sigma_t_min=args.large_sigma_min)
    sysm = System(p.N, p.R, p.sigma_t, p.albedo, p.g, p.Q00, sigma_t_min=args.large_sigma_min)
    tiling = sysm.tune_apply()
    sysm.set_l2_residency(not args.no_l2_resident)
    sysm.set_stream_kernels(args.stream_tma)
    u = sysm.zeros(torch.float64)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    st = sysm.solve(u, solver="ir", tol=1e-6, restart=args.restart, ortho="cgs1", basis="f16",
                    augment=args.augment, max_iter=args.large_iters, raise_on_error=False)
    e1.record()
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    dof = sysm.layout.n_active
    print(json.dumps({"mode": "large-solve", "workload": f"P7 256^3 thresholded-fBm cloud, sigma_t_min "
                      f"{args.large_sigma_min}, albedo 0.99, g 0.6, point source; FP32 LGMRES({args.restart}, "
                      f"{args.augment}), FP16 basis, FP64 IR", "dof": dof, "ms": ms, "iterations": st["iterations"],
                      "outer_iterations": st["outer_iterations"], "rel_residual": st["rel_residual"],
                      "status": st["status"], "ms_per_iteration": ms / max(1, st["iterations"]),
                      "gdof_iterations_per_s": dof * st["iterations"] / (ms * 1e-3) / 1e9,
                      "apply_ctas_per_sm": tiling["ctas_per_sm"], "apply_kernel": tiling["kernel"]}), flush=True)
    sysm.close()


def main():
    args = parse()
    if args.network_only:
        run_network_only(args)
        return
    if args.large_solve:
        run_large_solve(args)
        return
    if args.batched:
        run_batched(args)
        return
    if args.checkerboard:
        run_checkerboard(args)
        return
    if args.threshold_sweep:
        run_threshold_sweep(args)
        return
    if args.apply_only:
        run_apply_only(args)
        return
    if args.access_probe:
        run_access_probe(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
