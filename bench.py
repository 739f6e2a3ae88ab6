#!/usr/bin/env python
"""Operator-apply throughput of the matrix-free tetrahedral Laplacian on GB300.

Workload (default): CG P3 Laplacian on the 64^3 Kuhn-split unit cube
(1,572,864 tets, 7,189,057 DoFs), interior vertices jittered by U[-0.2h, 0.2h]
(seed 0), Morton-ordered cells, u ~ U[-1, 1] (seed 1).  One step = one
operator application y = A u through the C ABI (fem_apply), inputs resident in
HBM; the L2 is flushed (a 256 MiB write) before every timed step, outside the
timed events.  `value` is the TF32 tensor-core apply in GDoF/s (DoFs / s,
Sec. 2.3); the FP64, FP32 and BF16 applies, the assembled CSR SpMV of the same
operator and the DG SIPG P2 apply on the 48^3 cube are reported under
`variants`.  `e2e` is the same apply through the host-buffer call
(fem_apply_host): every step copies its input from pinned host memory and its
result back inside the timed region, one call streaming all steps (copy in,
apply and copy out overlapped on three streams); `serial_value` makes one
blocking call per step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank runs the whole workload on its own GPU (replicas;
`value` = all ranks' DoFs / max time).
"""
from __future__ import annotations

import os

# every oracle process runs single-threaded (the multi-core baseline uses one process per core);
# pin BLAS pools before numpy loads
for _v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import argparse
import json
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "operator-apply GDoF/s (CG P3, DG P2) FP64 vs FP32-TC, % roofline, vs CSR SpMV"
UNIT = "GDoF/s"
L2_FLUSH_BYTES = 256 << 20
NOMINAL_FP64_TFLOPS = 1.25  # GB300 FP64 (no FP64 tensor path)


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return {"hbm_gbs": d["hbm_gbs"], "source": "measured", "sm_max_mhz": d.get("sm_max_mhz", 2070.0)}
    return {"hbm_gbs": 6800.0, "source": "fallback", "sm_max_mhz": 2070.0}


def profiled_traffic(kernel_sources, summary):
    """DRAM bytes per launch recorded by an ncu capture in profiles/<summary>, if that capture was taken of
    the current kernel sources (sha1 of the files concatenated in the given order), else None."""
    import hashlib

    path = os.path.join(ROOT, "profiles", summary)
    srcs = [os.path.join(ROOT, "paper_2509_10226_gb300", "csrc", k) for k in kernel_sources]
    if not (os.path.exists(path) and all(os.path.exists(p) for p in srcs)):
        return None
    h = hashlib.sha1()
    for p in srcs:
        with open(p, "rb") as f:
            h.update(f.read())
    digest = h.hexdigest()
    rec = {}
    with open(path) as f:
        for line in f:
            if ":" in line and line.strip().startswith("- "):
                k, v = line.strip()[2:].split(":", 1)
                v = v.strip()
                rec[k.strip()] = v.split("`")[1] if v.startswith("`") else v.split()[0] if v else v
    if rec.get("source_sha1") != digest:
        return None
    try:
        return float(rec["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def cg_bytes(C, N, nd, prec):
    """Algorithmic bytes of one CG apply: 4 nd index bytes + the 6-entry metric per cell, u read and y written
    once per DoF (8-byte FP64 or 4-byte FP32 values)."""
    vb = 8 if prec == "fp64" else 4
    return C * (4 * nd + 6 * vb) + 2 * vb * N


def cg_flops(C, nd, nq):
    """Flops per apply counted as in Eq. 6: 2 * (3 nq nd * 2) + (15*2 + 3) nq + nd per cell."""
    return C * (2 * (3 * nq * nd * 2) + 33 * nq + nd)


def cg_flops_executed(C, nd, nq):
    """Flops the SIMT apply executes per cell: per point 3 nd FMAs for the gradient and 3 nd for the
    integration, the symmetric metric (3 x (1 mul + 2 FMA)) and the weight (3 mul)."""
    return C * nq * (12 * nd + 18)


def dg_bytes(C, F_int, F_bnd, nd, prec):
    """DG: one 4-byte index and the metric per cell, u read and y written per DoF, per face 2 cell ids, a code
    word and 8 (interior) / 5 (boundary) geometry values."""
    vb = 8 if prec == "fp64" else 4
    return C * (4 + 6 * vb) + 2 * vb * C * nd + F_int * (12 + 8 * vb) + F_bnd * (8 + 5 * vb)


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons while the timed loops run."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap,utilization.gpu")

    def __init__(self, device_index):
        self.proc = None
        self.dev = device_index
        self.path = os.path.join("/tmp", f"tetmf_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.out,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.out.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 8:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        loaded = [r for r in rows if (num(r[7]) or 0) > 0] or rows
        sm = [num(r[0]) for r in loaded if num(r[0]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[3 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": num(rows[0][1]),
                "reasons": reasons, "samples": len(rows), "samples_under_load": len(loaded),
                "power_w_max": max((num(r[2]) or 0) for r in rows)}


def time_steps(torch, fn, steps, warmup, flush, stream, barrier):
    """Per-step device time (ms) with CUDA events on the launching stream; L2 flushed before every step."""
    for _ in range(warmup):
        flush()
        fn()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for i in range(steps):
        flush()
        ev[i][0].record(stream)
        fn()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


def replica_max(x, dist, device):
    """Max of a per-rank value over the replicas (the job's time is its slowest rank's); x itself
    when there is no process group.  Replicas run the whole workload each, so the job's throughput is
    world x units / replica_max(time)."""
    if dist is None:
        return x
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def tstat(ms):
    """Median and minimum of per-step times (ms), next to the mean each line reports."""
    return {"ms_median": float(np.median(ms)), "ms_min": float(np.min(ms))}


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the machine type)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform

    return platform.machine()


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _oracle_worker(conn):
    """One single-threaded oracle process: keeps a chunk of cells with its local numbering and applies
    the oracle to it on request."""
    from oracle import cg

    state = None
    while True:
        msg = conn.recv()
        if msg[0] == "setup":
            state = msg[1:]
            conn.send("ready")
        elif msg[0] == "run":
            xyz, cells, u, p, dofs = state
            t0 = time.perf_counter()
            y = cg.apply(xyz, cells, u, p, dofs=dofs)
            conn.send((y, time.perf_counter() - t0))
        else:
            conn.close()
            return


class OracleCores:
    """The FP64 oracle on every host core: the sample's cells are split into contiguous chunks, one
    single-threaded process per core applies the unchanged oracle (gather, element loop, scatter) to
    its chunk in the chunk's own numbering, and the parent adds the chunk results into the sample's
    vector (that sum is inside the timed region).  Processes are started with spawn."""

    def __init__(self, xyz, cells, u, p, dofs, cores):
        import multiprocessing as mp

        ctx = mp.get_context("spawn")
        self.cores = cores
        self.n = int(dofs.max()) + 1
        bounds = np.linspace(0, cells.shape[0], cores + 1).astype(np.int64)
        self.procs, self.conns, self.maps = [], [], []
        for k in range(cores):
            a, b = bounds[k], bounds[k + 1]
            uniq, local = np.unique(dofs[a:b], return_inverse=True)
            parent, child = ctx.Pipe()
            pr = ctx.Process(target=_oracle_worker, args=(child,), daemon=True)
            pr.start()
            parent.send(("setup", xyz, cells[a:b], u[uniq], p, local.reshape(b - a, -1)))
            self.procs.append(pr)
            self.conns.append(parent)
            self.maps.append(uniq)
        for c in self.conns:
            assert c.recv() == "ready"

    def apply(self):
        """One parallel oracle apply of the whole sample; returns (y, wall seconds)."""
        t0 = time.perf_counter()
        for c in self.conns:
            c.send(("run",))
        y = np.zeros(self.n)
        for c, m in zip(self.conns, self.maps):
            yk, _ = c.recv()
            y[m] += yk
        return y, time.perf_counter() - t0

    def close(self):
        for c in self.conns:
            c.send(("stop",))
        for pr in self.procs:
            pr.join(timeout=10)


def oracle_sample(xyz, cells, p, target_s):
    """A bounded sample of the workload for the oracle: the first S cells, S sized so that one
    single-core oracle apply takes about target_s seconds (calibrated on 2,048 cells)."""
    from oracle import cg, topology

    def numbered(S):
        sub = cells[:S]
        dofs, keys = topology.cg_numbering(sub, p)
        return sub, dofs, synth.uniform_vector(keys.shape[0], 1)

    sub, dofs, u = numbered(2048)
    t0 = time.perf_counter()
    cg.apply(xyz, sub, u, p, dofs=dofs)
    t = time.perf_counter() - t0
    S = int(min(cells.shape[0], max(2048, 2048 * target_s / max(t, 1e-6))))
    return numbered(S)


def oracle_cpu_baseline(xyz, cells, p, N, target_s=10.0):
    """The FP64 oracle on the host cores on a bounded sample of the same mesh: one single-core apply of
    the sample, then the same apply split over every core (best of two); throughputs scaled to
    whole-problem DoFs, (sample cells / s) x (N / C)."""
    from oracle import cg

    C = cells.shape[0]
    sub, dofs, u = oracle_sample(xyz, cells, p, target_s)
    S = sub.shape[0]
    t0 = time.perf_counter()
    y1 = cg.apply(xyz, sub, u, p, dofs=dofs)
    t1 = time.perf_counter() - t0
    cores = host_cores()
    pool = OracleCores(xyz, sub, u, p, dofs, cores)
    try:
        pool.apply()  # warm-up
        runs = [pool.apply() for _ in range(2)]
    finally:
        pool.close()
    yk, tk = min(runs, key=lambda r: r[1])
    agree = float(np.abs(yk - y1).max() / max(np.abs(y1).max(), 1e-300))
    scale = N / C / 1e9
    return {"value": S / tk * scale, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu_model": cpu_model(),
            "single_core_value": S / t1 * scale,
            "sample": f"oracle cg.apply (gather, element loop, scatter) on the first {S} of {C} cells: "
                      f"{t1:.1f} s on one core, {tk:.2f} s split over {cores} processes (one per core, "
                      f"chunk results summed; max rel. difference to the one-core result {agree:.1e}); "
                      f"scaled by N/C = {N / C:.4f} DoFs per cell"}


SOLVE_MODES_P3 = (("ir_tf32", "ir", "tf32", 0, 0), ("ir_bf16", "ir", "bf16", 0, 0),
                  ("ir_tf32x3", "ir", "tf32x3", 0, 0), ("ir_fp32", "ir", "fp32", 0, 0),
                  ("ir_pmg_tf32", "pmg", "tf32", 5, 20), ("ir_pmg_tf32x3", "pmg", "tf32x3", 3, 10),
                  ("pcg_fp64", "pcg", "fp32", 0, 0))


def time_solve_sweep(torch, FemSpace, device, degrees=(1, 2, 3, 4)):
    """Poisson solve -Laplace u = 1, homogeneous Dirichlet, CG P_p on the 48^3 cube (117,649 / 912,673 /
    3,048,625 / 7,189,057 DoFs for p = 1..4) to a relative residual of 1e-10: FP64 iterative refinement
    around the TF32 inner Jacobi-PCG and (p >= 2) around the p-multigrid cycle (the paper's 5 + 5
    Chebyshev steps, 20 coarse steps), against the all-FP64 Jacobi-PCG.  At p = 3 also BF16, 3xTF32 and
    FP32 inner solves and a lighter 3 + 3 cycle around 3xTF32.  Wall time of each solve, after short
    warm-up solves (which also build the p-hierarchy)."""
    xyz, cells = synth.kuhn_cube(48, jitter=0.2, seed=synth.SEEDS["jitter"])
    out = {"rtol": 1e-10}
    for p in degrees:
        sp = FemSpace(xyz, cells, kind="cg", degree=p, dirichlet=True, device=device)
        b = sp.rhs_const(1.0)
        if p == 3:
            modes = list(SOLVE_MODES_P3)
        else:
            modes = [("ir_tf32", "ir", "tf32", 0, 0)] + ([("ir_pmg_tf32", "pmg", "tf32", 5, 20)] if p >= 2 else []) + [
                ("pcg_fp64", "pcg", "fp32", 0, 0)]
        for _, mode, inner, deg, cs in modes[:-1]:
            sp.solve(b, mode=mode, inner_prec=inner, rtol=1e-3, raise_on_notconv=False, smoother_degree=deg,
                     coarse_steps=cs)
        row = {"n_dofs": sp.n_dofs}
        for name, mode, inner, deg, cs in modes:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, st = sp.solve(b, mode=mode, inner_prec=inner, rtol=1e-10, inner_rtol=1e-3, raise_on_notconv=False,
                             smoother_degree=deg, coarse_steps=cs)
            torch.cuda.synchronize()
            row[name] = {"seconds": time.perf_counter() - t0, "outer": st["outer"], "inner": st["inner"],
                         "rel_residual": st["rel_residual"], "converged": st["converged"]}
        best = min(row[n]["seconds"] for n in row if n.startswith("ir"))
        row["speedup_best_mixed_vs_fp64"] = row["pcg_fp64"]["seconds"] / best
        out[f"p{p}"] = row
        del sp, b
        torch.cuda.empty_cache()
    return out


def flat_summary(variants, fma_peaks):
    """The comparison the metric names, as flat keys (4 significant digits): GDoF/s of every apply of the
    CG P3 64^3 workload and of the DG P2 48^3 one, their relative l2 difference to the FP64 apply, the
    FP64 apply's fraction of the measured FP64 FMA peak, and the solve sweep's seconds."""
    def r(x):
        return None if x is None else float(f"{x:.4g}")

    out = {}
    for k in ("fp64", "fp32", "tf32", "bf16", "tf32x3", "csr_fp64", "csr_fp32", "dg_p2_48_fp64", "dg_p2_48_fp32",
              "dg_p2_48_tf32", "dg_p2_48_bf16", "modified_rule_tf32"):
        v = variants.get(k)
        if isinstance(v, dict) and "gdofs" in v:
            out[f"{k}_gdofs"] = r(v["gdofs"])
            if "rel_l2_vs_fp64" in v:
                out[f"{k}_rel_l2"] = r(v["rel_l2_vs_fp64"])
    if "frac_measured" in variants.get("fp64", {}):
        out["fp64_frac_of_measured_fp64_peak"] = r(variants["fp64"]["frac_measured"])
        out["fp64_frac_executed_flops"] = r(variants["fp64"]["frac_measured_executed"])
    if fma_peaks:
        out.update({f"peak_{k}_tflops_measured": r(v) for k, v in fma_peaks.items()})
    sw = variants.get("solve_sweep_48", {})
    for p in (1, 2, 3, 4):
        row = sw.get(f"p{p}")
        if row:
            out[f"solve_p{p}_48_s"] = {k: r(v["seconds"]) for k, v in row.items()
                                       if isinstance(v, dict) and k in ("ir_tf32", "ir_pmg_tf32", "pcg_fp64")}
    return out


def measure_fma_peaks(torch, stream):
    """FP64, FP32 and packed FP32x2 FMA throughput of this GPU (TFLOP/s) with the library's probe kernel:
    one warm-up launch, then the best of three launches of about 50 ms each, timed with CUDA events."""
    from paper_2509_10226_gb300.fem import fma_probe

    sink = torch.zeros(1, dtype=torch.float64, device="cuda")
    out = {}
    for kind, iters in (("fp64", 25_000), ("fp32", 1_600_000), ("fp32x2", 800_000)):
        fma_probe(kind, iters // 80 * 8, sink, stream)
        best = 0.0
        for _ in range(3):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fl = fma_probe(kind, iters, sink, stream)
            b.record(stream)
            b.synchronize()
            best = max(best, fl / (a.elapsed_time(b) * 1e-3) / 1e12)
        out[kind] = best
    return out


def run_reference(args):
    """--impl reference: the oracle on every host core, each step one parallel apply of a bounded sample
    of the workload (the first cells of the 64^3 mesh, sized for about 10 s of one core's work)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from oracle import cg

    xyz, cells = synth.kuhn_cube(64, jitter=0.2, seed=synth.SEEDS["jitter"])
    p = 3
    C = cells.shape[0]
    N = (3 * 64 + 1) ** 3
    sub, dofs, u = oracle_sample(xyz, cells, p, 10.0)
    S = sub.shape[0]
    t0 = time.perf_counter()
    cg.apply(xyz, sub, u, p, dofs=dofs)
    t1 = time.perf_counter() - t0
    cores = host_cores()
    pool = OracleCores(xyz, sub, u, p, dofs, cores)
    try:
        for _ in range(args.warmup):
            pool.apply()
        times = [pool.apply()[1] for _ in range(args.steps)]
    finally:
        pool.close()
    t = float(np.mean(times))
    scale = N / C / 1e9
    value = S / t * scale
    sample = (f"oracle cg.apply on the first {S} of {C} cells of the CG P3 64^3 workload per step, split over "
              f"{cores} processes (one per core, chunk results summed); scaled by N/C = {N / C:.4f} DoFs per cell")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "CG P3 Laplacian, 64^3 Kuhn cube (1,572,864 tets, 7,189,057 DoFs), "
                               "jitter 0.2h, FP64 oracle on a cell sample", "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu_model": cpu_model(),
                         "single_core_value": S / t1 * scale, "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=64, help="subcubes per direction of the CG workload")
    ap.add_argument("--no-variants", action="store_true", help="time the headline apply only")
    ap.add_argument("--no-dg", action="store_true")
    ap.add_argument("--no-reorder", action="store_true", help="skip the shuffled-mesh reordering ablation")
    ap.add_argument("--no-modified", action="store_true", help="skip the modified-integration variants")
    ap.add_argument("--no-colour", action="store_true", help="skip the colour-scatter ablation")
    ap.add_argument("--no-smoother", action="store_true", help="skip the Chebyshev smoother sweeps")
    ap.add_argument("--no-curved", action="store_true", help="skip the curved-cell variants")
    ap.add_argument("--no-vector", action="store_true", help="skip the vector-Laplacian variants")
    ap.add_argument("--no-transfer", action="store_true", help="skip the p-transfer variants")
    ap.add_argument("--no-csr", action="store_true")
    ap.add_argument("--no-solve", action="store_true")
    ap.add_argument("--no-solve-sweep", action="store_true",
                    help="time the 48^3 Dirichlet solve at p = 3 only (the default sweeps p = 1..4, about a minute)")
    ap.add_argument("--no-peaks", action="store_true", help="skip the FMA-throughput probe")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    def max_over_ranks(x):
        return replica_max(x, dist, "cuda")

    from paper_2509_10226_gb300.fem import FemSpace

    peaks = load_peaks()
    stream = torch.cuda.current_stream()
    flush_buf = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def flush():
        flush_buf.fill_(1.0)

    n = args.n
    p = 3
    t0 = time.perf_counter()
    xyz, cells = synth.kuhn_cube(n, jitter=0.2, seed=synth.SEEDS["jitter"])
    sp = FemSpace(xyz, cells, kind="cg", degree=p, device=local)
    setup_s = time.perf_counter() - t0
    C, N, nd, nq = sp.n_cells, sp.n_dofs, sp.dofs_per_cell, sp.n_qpoints
    u64 = torch.as_tensor(synth.uniform_vector(N, synth.SEEDS["u"]), device="cuda")
    u32 = u64.float()
    y64 = torch.empty_like(u64)
    y32 = torch.empty_like(u32)
    clocks = Clocks(local)
    clocks.start()

    # headline: TF32 tensor-core apply
    head = "tf32"
    ms = time_steps(torch, lambda: sp.apply(u32, prec=head, out=y32), args.steps, args.warmup, flush, stream,
                    barrier)
    t_head = max_over_ranks(float(np.mean(ms)))
    value = world * N / (t_head * 1e-3) / 1e9
    y_head = y32.double().clone()
    hb = cg_bytes(C, N, nd, head)
    achieved = hb / (t_head * 1e-3) / 1e9
    # the capture belongs to the kernel sources and to the tile lists' layout built in device.cu
    traffic = (profiled_traffic(["cg_tc.cu", "tc_ptx.cuh", "device.cu"], "k_cg_apply_tc.cg_p3_64.md")
               if n == 64 else None)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "traffic": traffic, "algorithmic_bytes": hb,
                "kernel": "fem_apply tf32 (zero-fill + k_cg_apply_tc_ws)",
                "peak_source": peaks["source"] + " hbm_gbs (burst copy)"}

    # end to end through the public host-buffer call (fem_apply_host): every step copies its own
    # input from pinned host memory to the device and its result back, inside the timed region.
    # Serial: one blocking call per step; streamed: one call for all steps, whose copies in, applies
    # and copies out overlap on three streams (inputs larger than L2, no flush between steps).
    u_hs = [torch.empty(N, dtype=torch.float32, pin_memory=True) for _ in range(2)]
    for t_ in u_hs:
        t_.copy_(u32.cpu())
    y_hs = [torch.empty(N, dtype=torch.float32, pin_memory=True) for _ in range(2)]
    sp.apply_host(u_hs, y_hs, prec=head)  # allocates the context's transfer slots and streams
    for _ in range(max(args.warmup - 1, 0)):
        sp.apply_host(u_hs[:1], y_hs[:1], prec=head)
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for k_ in range(args.steps):
        sp.apply_host(u_hs[k_ % 2:k_ % 2 + 1], y_hs[k_ % 2:k_ % 2 + 1], prec=head)
    t_serial = max_over_ranks((time.perf_counter() - t0) * 1e3 / args.steps)
    barrier()
    seq_u = [u_hs[k_ % 2] for k_ in range(args.steps)]
    seq_y = [y_hs[k_ % 2] for k_ in range(args.steps)]
    sp.apply_host(seq_u[:4], seq_y[:4], prec=head)
    barrier()
    t0 = time.perf_counter()
    sp.apply_host(seq_u, seq_y, prec=head)
    t_e2e = max_over_ranks((time.perf_counter() - t0) * 1e3 / args.steps)
    barrier()
    e2e_err = float(np.abs(y_hs[0].double().numpy() - y_head.cpu().numpy()).max() /
                    max(np.abs(y_head.cpu().numpy()).max(), 1e-300))
    e2e = {"value": world * N / (t_e2e * 1e-3) / 1e9, "unit": UNIT, "h2d_bytes_per_step": 4 * N,
           "d2h_bytes_per_step": 4 * N, "ms_per_step": t_e2e, "api": "fem_apply_host (three streams)",
           "serial_ms_per_step": t_serial, "serial_value": world * N / (t_serial * 1e-3) / 1e9,
           "max_rel_diff_vs_device_apply": e2e_err}

    fma_peaks = None if args.no_peaks else measure_fma_peaks(torch, stream)
    variants = {}
    ref64 = None
    if not args.no_variants:
        vsteps = max(5, min(args.steps, 30))
        ms64 = time_steps(torch, lambda: sp.apply(u64, prec="fp64", out=y64), vsteps, 2, flush, stream, barrier)
        ref64 = y64.clone()

        def rel(y):
            return float(torch.linalg.norm(y.double() - ref64) / torch.linalg.norm(ref64))

        t = float(np.mean(ms64))
        fl = cg_flops(C, nd, nq)
        fx = cg_flops_executed(C, nd, nq)
        variants["fp64"] = {**tstat(ms64), "gdofs": N / (t * 1e-3) / 1e9, "ms": t, "bound": "alu",
                            "achieved_tflops": fl / (t * 1e-3) / 1e12, "flops_counted": "Eq. 6",
                            "achieved_tflops_executed": fx / (t * 1e-3) / 1e12,
                            "flops_executed": "12 nd + 18 per point (the kernel's FMA chain)",
                            "peak_tflops_nominal": NOMINAL_FP64_TFLOPS,
                            "hbm_gbs": cg_bytes(C, N, nd, "fp64") / (t * 1e-3) / 1e9}
        if fma_peaks:
            variants["fp64"].update({"peak_tflops_measured": fma_peaks["fp64"],
                                     "frac_measured": fl / (t * 1e-3) / 1e12 / fma_peaks["fp64"],
                                     "frac_measured_executed": fx / (t * 1e-3) / 1e12 / fma_peaks["fp64"]})
        for prec in ("fp32", "bf16", "tf32x3"):
            msv = time_steps(torch, lambda: sp.apply(u32, prec=prec, out=y32), vsteps, 2, flush, stream, barrier)
            t = float(np.mean(msv))
            gbs = cg_bytes(C, N, nd, prec) / (t * 1e-3) / 1e9
            variants[prec] = {**tstat(msv), "gdofs": N / (t * 1e-3) / 1e9, "ms": t, "hbm_gbs": gbs,
                              "frac_hbm": gbs / peaks["hbm_gbs"], "rel_l2_vs_fp64": rel(y32)}
            if prec == "fp32":
                variants[prec].update({"bound": "alu", "achieved_tflops": fl / (t * 1e-3) / 1e12,
                                       "achieved_tflops_executed": fx / (t * 1e-3) / 1e12})
                if fma_peaks:
                    variants[prec].update({"peak_tflops_measured": fma_peaks["fp32"],
                                           "frac_measured_executed": fx / (t * 1e-3) / 1e12 / fma_peaks["fp32"]})
        variants["tf32"] = {**tstat(ms), "gdofs": value / world, "ms": t_head, "hbm_gbs": achieved,
                            "frac_hbm": achieved / peaks["hbm_gbs"], "rel_l2_vs_fp64": rel(y_head)}
        if not args.no_csr:
            try:
                t0 = time.perf_counter()
                nnz = sp.csr_build()
                build_s = time.perf_counter() - t0
                for prec, u_, y_ in (("fp64", u64, y64), ("fp32", u32, y32)):
                    msv = time_steps(torch, lambda: sp.csr_apply(u_, prec=prec, out=y_), vsteps, 2, flush, stream,
                                     barrier)
                    t = float(np.mean(msv))
                    vb = 8 if prec == "fp64" else 4
                    b = nnz * (4 + vb) + 8 * (N + 1) + 2 * vb * N
                    gbs = b / (t * 1e-3) / 1e9
                    variants[f"csr_{prec}"] = {**tstat(msv), "gdofs": N / (t * 1e-3) / 1e9, "ms": t, "nnz": nnz,
                                               "hbm_gbs": gbs, "frac_hbm": gbs / peaks["hbm_gbs"],
                                               "rel_l2_vs_fp64": rel(y_), "build_s": build_s}
            except Exception as e:  # noqa: BLE001
                variants["csr"] = {"unavailable": str(e).splitlines()[0]}
        if not args.no_reorder:
            # Sec. 2.5 ablation: the same cube with cells and vertices shuffled (generator order), applied
            # in that order and after the Morton renumbering
            try:
                xs, cs, _ = synth.shuffle_mesh(xyz, cells, seed=synth.SEEDS["shuffle"])
                for tag, ro in (("none", False), ("morton", True)):
                    ssp = FemSpace(xs, cs, kind="cg", degree=p, reorder=ro, device=local)
                    su = torch.as_tensor(synth.uniform_vector(ssp.n_dofs, synth.SEEDS["u"]), device="cuda",
                                         dtype=torch.float32)
                    sy = torch.empty_like(su)
                    for prec in ("tf32", "fp32"):
                        msv = time_steps(torch, lambda: ssp.apply(su, prec=prec, out=sy), vsteps, 2, flush, stream,
                                         barrier)
                        t = float(np.mean(msv))
                        variants[f"shuffled_reorder_{tag}_{prec}"] = {**tstat(msv), "gdofs": ssp.n_dofs / (t * 1e-3) / 1e9, "ms": t}
                    del ssp, su, sy
            except Exception as e:  # noqa: BLE001
                variants["shuffled_reorder"] = {"unavailable": str(e).splitlines()[0]}
        if not args.no_vector:
            # vector Laplacian, 3 components (Sec. 3.1): components-batched on the FMA units
            try:
                U64 = torch.stack([u64, u64.flip(0), -u64])
                U32 = U64.float()
                vec = {}
                for prec, U_ in (("fp64", U64), ("fp32", U32), ("tf32", U32)):
                    Y_ = torch.empty_like(U_)
                    msv = time_steps(torch, lambda: sp.apply_vector(U_, prec=prec, out=Y_),
                                     vsteps if prec != "fp64" else 3, 1, flush, stream, barrier)
                    t = float(np.mean(msv))
                    vec[prec] = {**tstat(msv), "gdofs": 3 * N / (t * 1e-3) / 1e9, "ms": t, "components": 3}
                variants["vector3_p3_64"] = vec
                del U64, U32
            except Exception as e:  # noqa: BLE001
                variants["vector3_p3_64"] = {"unavailable": str(e).splitlines()[0]}
        if not args.no_curved:
            # curved cells (second-order geometry, Sec. 3.2): a metric per quadrature point, 35 x 6
            # words per cell instead of 6 -- the memory-bound variant of the apply
            try:
                nodes = synth.curved_nodes(xyz, cells, 0.05)
                csp = FemSpace(xyz, cells, kind="cg", degree=p, device=local, cell_nodes=nodes)
                del nodes
                cur = {}
                yref = None
                for prec, u_, y_ in (("fp64", u64, y64), ("fp32", u32, y32), ("tf32", u32, y32), ("bf16", u32, y32)):
                    msv = time_steps(torch, lambda: csp.apply(u_, prec=prec, out=y_), vsteps if prec != "fp64" else 5,
                                     2, flush, stream, barrier)
                    t = float(np.mean(msv))
                    vb = 8 if prec == "fp64" else 4
                    b = C * (4 * nd + 6 * nq * vb) + 2 * vb * N
                    gbs = b / (t * 1e-3) / 1e9
                    if prec == "fp64":
                        yref = y64.clone()
                    relc = float(torch.linalg.norm(y_.double() - yref) / torch.linalg.norm(yref))
                    cur[prec] = {**tstat(msv), "gdofs": N / (t * 1e-3) / 1e9, "ms": t, "algorithmic_bytes": b,
                                 "hbm_gbs": gbs, "frac_hbm": gbs / peaks["hbm_gbs"], "rel_l2_vs_fp64": relc}
                variants["curved_p3_64"] = cur
                del csp
            except Exception as e:  # noqa: BLE001
                variants["curved_p3_64"] = {"unavailable": str(e).splitlines()[0]}
        if not args.no_smoother:
            # Chebyshev-Jacobi smoothing sweeps of degree 5 (the smoother of the paper's multigrid,
            # Sec. 4.1) with the tensor-core apply: one apply and one fused vector pass per step
            try:
                sm = {}
                for prec in ("tf32", "fp64"):
                    uu, xx = (u64, y64) if prec == "fp64" else (u32, y32)
                    dg_ = sp.diagonal(prec="fp64" if prec == "fp64" else "fp32")  # FP32 vectors for TF32
                    lam = 1.2 * sp.lambda_max(dg_, uu, iterations=20, prec=prec)
                    msv = time_steps(torch, lambda: sp.chebyshev(uu, xx, dg_, degree=5, lam_max=lam, prec=prec),
                                     vsteps if prec != "fp64" else 5, 2, flush, stream, barrier)
                    t = float(np.mean(msv))
                    sm[prec] = {**tstat(msv), "ms_per_sweep": t, "applies_per_sweep": 5,
                                "gdofs_per_apply": 5 * N / (t * 1e-3) / 1e9, "lambda_max": lam}
                variants["chebyshev_degree5"] = sm
            except Exception as e:  # noqa: BLE001
                variants["chebyshev_degree5"] = {"unavailable": str(e).splitlines()[0]}
        if not args.no_transfer:
            # p-transfer P3 -> P1 on the same mesh (the p-levels of the paper's multigrid, Sec. 4.1)
            try:
                from paper_2509_10226_gb300.fem import Transfer

                c1 = FemSpace(xyz, cells, kind="cg", degree=1, device=local)
                tr = Transfer(sp, c1)
                uc = torch.as_tensor(synth.uniform_vector(c1.n_dofs, synth.SEEDS["u"]), device="cuda",
                                     dtype=torch.float32)
                rc = torch.empty_like(uc)
                tv = {}
                for name, fn in (("prolongate", lambda: tr.prolongate(uc, prec="fp32", out=y32)),
                                 ("restrict", lambda: tr.restrict(u32, prec="fp32", out=rc))):
                    msv = time_steps(torch, fn, vsteps, 2, flush, stream, barrier)
                    t = float(np.mean(msv))
                    tv[name] = {**tstat(msv), "ms": t, "fine_gdofs": N / (t * 1e-3) / 1e9}
                variants["transfer_p3_p1_fp32"] = tv
                tr.close()
                del c1
            except Exception as e:  # noqa: BLE001
                variants["transfer_p3_p1_fp32"] = {"unavailable": str(e).splitlines()[0]}
        if not args.no_colour:
            # scatter ablation: cells ordered by colour, one launch per colour without atomics
            try:
                csp = FemSpace(xyz, cells, kind="cg", degree=p, device=local, scatter="colour")
                ncol = len(csp.colour_starts()) - 1
                for prec, u_, y_ in (("fp64", u64, y64), ("fp32", u32, y32)):
                    msv = time_steps(torch, lambda: csp.apply(u_, prec=prec, out=y_), vsteps, 2, flush, stream,
                                     barrier)
                    t = float(np.mean(msv))
                    variants[f"colour_scatter_{prec}"] = {**tstat(msv), "gdofs": N / (t * 1e-3) / 1e9, "ms": t,
                                                          "colours": ncol, "rel_l2_vs_fp64": rel(y_)}
                del csp
            except Exception as e:  # noqa: BLE001
                variants["colour_scatter"] = {"unavailable": str(e).splitlines()[0]}
        if not args.no_modified:
            # Sec. 3.3: cell rule exact to degree 2p - 2 (15 instead of 35 points at p = 3); with a
            # constant coefficient the operator is the same (the integrand has degree 2p - 2)
            try:
                msp = FemSpace(xyz, cells, kind="cg", degree=p, device=local, modified_rule=True)
                for prec, u_, y_ in (("fp64", u64, y64), ("fp32", u32, y32), ("tf32", u32, y32), ("bf16", u32, y32)):
                    msv = time_steps(torch, lambda: msp.apply(u_, prec=prec, out=y_), vsteps, 2, flush, stream,
                                     barrier)
                    t = float(np.mean(msv))
                    variants[f"modified_rule_{prec}"] = {**tstat(msv), "gdofs": N / (t * 1e-3) / 1e9, "ms": t,
                                                         "n_qpoints": msp.n_qpoints, "rel_l2_vs_fp64": rel(y_)}
                del msp
            except Exception as e:  # noqa: BLE001
                variants["modified_rule"] = {"unavailable": str(e).splitlines()[0]}
        if not args.no_dg:
            try:
                xd, cd = synth.kuhn_cube(48, jitter=0.2, seed=synth.SEEDS["jitter"])
                dsp = FemSpace(xd, cd, kind="dg", degree=2, device=local)
                du64 = torch.as_tensor(synth.uniform_vector(dsp.n_dofs, synth.SEEDS["u"]), device="cuda")
                du32 = du64.float()
                dy64 = torch.empty_like(du64)
                dy32 = torch.empty_like(du32)
                dytc = {q: torch.empty_like(du32) for q in ("tf32", "bf16")}
                for prec, u_, y_ in (("fp64", du64, dy64), ("fp32", du32, dy32), ("tf32", du32, dytc["tf32"]),
                                     ("bf16", du32, dytc["bf16"])):
                    msv = time_steps(torch, lambda: dsp.apply(u_, prec=prec, out=y_), vsteps, 2, flush, stream,
                                     barrier)
                    t = float(np.mean(msv))
                    b = dg_bytes(dsp.n_cells, dsp.n_interior_faces, dsp.n_boundary_faces, 10, prec)
                    variants[f"dg_p2_48_{prec}"] = {**tstat(msv), "gdofs": dsp.n_dofs / (t * 1e-3) / 1e9, "ms": t,
                                                    "n_dofs": dsp.n_dofs, "hbm_gbs": b / (t * 1e-3) / 1e9}
                for prec, y_ in (("fp32", dy32), ("tf32", dytc["tf32"]), ("bf16", dytc["bf16"])):
                    variants[f"dg_p2_48_{prec}"]["rel_l2_vs_fp64"] = float(
                        torch.linalg.norm(y_.double() - dy64) / torch.linalg.norm(dy64))
                del dsp
            except Exception as e:  # noqa: BLE001
                variants["dg_p2_48"] = {"unavailable": str(e).splitlines()[0]}
    if not args.no_variants and not args.no_solve:
        try:
            variants["solve_sweep_48"] = time_solve_sweep(torch, FemSpace, local,
                                                          (3,) if args.no_solve_sweep else (1, 2, 3, 4))
        except Exception as e:  # noqa: BLE001
            variants["solve_sweep_48"] = {"unavailable": str(e).splitlines()[0]}
    clk = clocks.stop()
    status = sp.device_status()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = oracle_cpu_baseline(xyz, cells, p, N)

    if rank == 0:
        # the bulky per-variant record first, on its own line; the result line last, short, with the
        # metric's comparison (FP64 vs the FP32 / tensor-core applies vs the CSR SpMV, DG P2, the solve
        # sweep) as flat keys at its end
        print(json.dumps({"variants": variants, "fma_peaks_tflops": fma_peaks}), flush=True)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_head, **tstat(ms), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "tf32", "data": "synthetic",
            "config": {"workload": f"CG P3 Laplacian, {n}^3 Kuhn cube ({C:,} tets, {N:,} DoFs), TF32 tensor cores",
                       "cells": C, "dofs": N, "degree": p, "quadrature": "Grundmann-Moeller s=3 (35 points)",
                       "parallelism": f"replicas x{world}", "l2": "flushed (256 MiB write) before every step",
                       "setup_s": round(setup_s, 2)},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": 2 * args.steps,
            "clocks": clk, "device_status": status, **flat_summary(variants, fma_peaks),
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
