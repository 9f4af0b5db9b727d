#!/usr/bin/env python3
"""Benchmark: symmetric SpMM GB/s inside LOBPCG on the n = 2M workload (one GB300).

One step = one LOBPCG iteration on the n = 2M matrix (~400 stored entries per
row, k = 16, nev = 8, float32, diagonal preconditioner): residual and
preconditioner, two Cholesky-QR passes, the SpMM H W, Gram matrices,
Rayleigh-Ritz and the update -- every row of the hot path -- with inputs
resident in HBM.  The matrix stream (~6.4 GB) is far larger than L2, so no
explicit flush is done.

value      : SpMM algorithmic bytes per step x steps / timed region (GB/s),
             algorithmic bytes = nnz (4 col + 4 val) + 8 (n + 1) + 2 n k 4.
lobpcg     : time-to-solution (nev pairs at relative residual 1e-6) of
             lobpcg_solve from a host X0, per preconditioner.
e2e        : the same metric through lobpcg_spmm_sym with pinned HOST X and Y
             (host->device copy of X and device->host copy of Y each step).
roofline   : the spmm_sym kernel alone, timed with CUDA events on its stream,
             against the measured HBM copy bandwidth.
cpu_baseline: the CPU oracle's SpMM on the host cores, on a bounded sample.
value_only_tiles: the SpMM and the diagonal solve with tile_format 1
             (complete tiles keep value words only), with GB/s on its own
             stream bytes -- reported beside the CSR-equivalent metric,
             never folded into it.
spmm_f64   : lobpcg_spmm_sym_f64 (float64 X and Y, products in compensated
             float32) on the same matrix, median of 5 launches.

--impl reference times the CPU oracle (the only reference there is: the
paper's code is not available) on the same metric.

Multi-GPU: the path does not shard here; N ranks run N independent replicas
(weak scaling), value = total bytes of all ranks / max time over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

WORKLOAD = "full_n2m"


def alg_bytes(n: int, nnz: int, k: int) -> int:
    return nnz * 8 + 8 * (n + 1) + 2 * n * k * 4


def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm_gbs": float(d["hbm_gbs"]), "sm_max_mhz": float(d.get("sm_max_mhz", 2070.0)),
                "bf16_tflops": float(d.get("bf16_tflops", 1900.0)), "source": "measured"}
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0, "bf16_tflops": 1900.0, "source": "fallback"}


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in ("spmm_sym.cu", "common.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2109_00485_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic(workload: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source; else None."""
    p = os.path.join(ROOT, "profiles", "spmm_sym_traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    e = d.get(workload)
    if not e or e.get("kernel_source_hash") != kernel_source_hash():
        return None
    return e.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"bench_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
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
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# Kernel launches of one LOBPCG iteration with a P block (from the ncu launch
# list of this bench, profiles/spmm_sym_full_n2m_ncu.md): first
# orthonormalisation pass (2 Gram, projection coefficients, Cholesky-QR
# factor, 2 combines); second pass (Gram, Omega, factor, coefficients,
# combine); SpMM; Gram, P scaling, Rayleigh-Ritz; the fused update with the
# next residual = 16.
LAUNCHES_PER_ITERATION = 16


def aggregate(total_ms: float, bytes_per_step: int, steps: int, world: int, device=None):
    """Max of the timed region over ranks and the whole-job value (GB/s):
    every rank runs its own replica, so the job moves world x bytes_per_step
    per step in the slowest rank's time."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return total_ms, bytes_per_step * steps * world / (total_ms / 1e3) / 1e9


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def cpu_baseline(A, k: int, max_seconds: float = 20.0) -> dict:
    """Time the CPU oracle's SpMM (Algorithm 2 plus its transposed loop, FP64
    arithmetic) on a leading principal sub-matrix of the workload sized to a
    bounded amount of work."""
    import oracle
    n = A.n
    # leading rows of a lower triangle form a valid smaller matrix
    target_nnz = min(A.nnz, 200_000_000)
    m = int(np.searchsorted(A.row_ptr, target_nnz))
    m = max(16, min(n, m))
    sub = synth.CSR(n=m, row_ptr=A.row_ptr[:m + 1], col=A.col[:A.row_ptr[m]], val=A.val[:A.row_ptr[m]])
    X = synth.normal_block(m, k, seed=4242)
    t0 = time.perf_counter()
    reps = 0
    while True:
        oracle.spmm_tri(sub, X)
        reps += 1
        if time.perf_counter() - t0 > max_seconds / 2 or reps >= 3:
            break
    dt = (time.perf_counter() - t0) / reps
    gbs = alg_bytes(m, sub.nnz, k) / dt / 1e9
    return {"value": round(gbs, 3), "unit": "GB/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"leading {m} rows ({sub.nnz} stored entries) of the n=2M matrix, k={k}, {reps} call(s), "
                      f"{dt:.2f} s per call; same algorithmic-byte formula as the GPU"}


def run_reference(args):
    world, rank, local = dist_setup()
    if rank != 0:
        return
    p = synth.WORKLOADS[args.workload]
    A = synth.tile_matrix(p["n"], p["nnz_per_row"], seed=p["seed"], fp32=True)
    k = p["k"]
    import oracle
    target_nnz = min(A.nnz, 100_000_000)
    m = max(16, min(A.n, int(np.searchsorted(A.row_ptr, target_nnz))))
    sub = synth.CSR(n=m, row_ptr=A.row_ptr[:m + 1], col=A.col[:A.row_ptr[m]], val=A.val[:A.row_ptr[m]])
    X = synth.normal_block(m, k, seed=4242)
    for _ in range(args.warmup):
        oracle.spmm_tri(sub, X)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.spmm_tri(sub, X)
    dt = time.perf_counter() - t0
    gbs = alg_bytes(m, sub.nnz, k) * args.steps / dt / 1e9
    line = {"metric": "symmetric SpMM GB/s", "value": round(gbs, 3), "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": args.workload, "n": A.n, "nnz": A.nnz, "k": k,
                       "sample_rows": m, "sample_nnz": sub.nnz},
            "cpu_baseline": {"value": round(gbs, 3), "unit": "GB/s", "cores": oracle.num_threads(),
                             "kind": "oracle", "sample": f"leading {m} rows ({sub.nnz} entries) per step"},
            "e2e": {"value": round(gbs, 3), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def fom_report(pkg, A, p, stream, sm_mhz: float) -> dict:
    """The FOM preconditioner (Section 3.3) on its own: one application to a
    seeded n x k block, 4 FOM steps, on 64-row tiles (k_fom_small) and on a
    seeded partition into 5..6000-row tiles (mostly k_fl_* segment kernels);
    CUDA events over 10 applications after 3 warm-ups.  The 64-row kernel is
    bound by FP32 arithmetic: its algorithmic FLOPs are the products
    2 * 64 * 64 * k per tile and step; the peak is 152 SMs x 128 FP32 lanes x
    2 FLOP x the SM clock."""
    import torch
    k = p["k"]
    R = torch.from_numpy(synth.normal_block(A.n, k, seed=41, fp32=True)).cuda()
    th = torch.linspace(-2.0, 30.0, k, dtype=torch.float64, device="cuda")
    tpv = synth.tile_partition(A.n, p["seed"])
    out = {}
    for label, tp in (("tiles64", None), ("variable", tpv)):
        h = pkg.from_csr(A, k=k, nev=p["nev"], precond="fom", fom_steps=4, fom_tile_ptr=tp, stream=stream)
        W = torch.empty_like(R)
        with torch.cuda.stream(stream):
            for _ in range(3):
                h.precond_apply(R, th, W, mode="fom")
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(10):
                h.precond_apply(R, th, W, mode="fom")
            e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 10
        h.destroy()
        d = {"ms": round(ms, 4), "steps": 4, "k": k}
        if tp is None:
            nt = (A.n + 63) // 64
            flops = nt * 4 * 2 * 64 * 64 * k
            peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12
            d.update({"kernel": "k_fom_small", "tiles": nt, "tflops": round(flops / (ms / 1e3) / 1e12, 2),
                      "peak_tflops_fp32_alu": round(peak, 1), "peak_clock_mhz": sm_mhz,
                      "frac": round(flops / (ms / 1e3) / 1e12 / peak, 4)})
        else:
            sizes = np.diff(tpv)
            d.update({"tiles": int(sizes.size), "tiles_over_64_rows": int((sizes > 64).sum()),
                      "rows_in_tiles_over_64": int(sizes[sizes > 64].sum()), "largest_tile": int(sizes.max()),
                      "median_tile": float(np.median(sizes))})
        out[label] = d
    return out


def golden_evals(workload: str):
    """The FP64 oracle's eigenvalues of this workload (tests/golden, written
    by tests/golden/make_full_n2m_oracle.py from the oracle alone), or None."""
    path = os.path.join(ROOT, "tests", "golden", f"{workload}_oracle_evals.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        g = json.load(f)
    return g if g.get("converged") else None


def eig_error(ev, gold) -> dict:
    """|theta - lambda| / max(|lambda|, 1e-3 ||H||_G) against the oracle run
    to 1e-10 (max over the nev pairs), and the largest absolute error."""
    lam = np.asarray(gold["evals"], dtype=np.float64)
    ev = np.asarray(ev, dtype=np.float64)[:lam.size]
    rel = np.abs(ev - lam) / np.maximum(np.abs(lam), 1e-3 * gold["gershgorin"])
    return {"max_rel": float(rel.max()), "max_abs": float(np.abs(ev - lam).max()),
            "oracle": f"FP64 LOBPCG to 1e-10, {gold['iters']} iterations (tests/golden)"}


def lobpcg_solves(pkg, A, p, stream, precs=("diag", "bjacobi", "fom", "fom_var", "mlp", "davidson_diag"),
                  repeats: int = 3, gold=None):
    """Time-to-solution (relative residual 1e-6, nev pairs) from a host X0,
    through lobpcg_solve; create (matrix tiling, preconditioner set-up) is
    timed separately.  The learned form ("mlp") is first trained on pairs
    harvested from 20 block-Jacobi iterations from the same X0 (about 1M
    pairs, 5 epochs, Adam lr 1e-3): its training time is reported on its own
    and added in.  "fom" runs 4 FOM steps per 64-row tile, "fom_var" the same
    on a seeded partition into 5..6000-row tiles (synth.tile_partition);
    "davidson_diag" is block Davidson (lobpcg_davidson, basis of 6 blocks)
    with the diagonal form on the same SpMM.  Each form solves `repeats`
    times from the same X0 on one handle (iteration counts vary from run to
    run: the float32 SpMM's order of additions is not fixed); the median run
    is reported with the spread of all runs.  X0 is resident in HBM when a
    timed solve starts and X stays there (the matrix too); one more solve
    from a host X0, returning X to the host, is reported as
    time_to_solution_host_s.  With the oracle's eigenvalues at hand, each
    form's eigenvalue error against them."""
    import torch
    out = {}
    X0 = synth.initial_guess(A, p["k"], seed=p["seed"] + synth.X0_SEED_OFFSET, fp32=True)
    with torch.cuda.stream(stream):
        X0d = torch.from_numpy(X0).cuda()
    torch.cuda.synchronize()
    for pc in precs:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        extra = {"fom_tile_ptr": synth.tile_partition(A.n, p["seed"])} if pc == "fom_var" else {}
        pcond = pc.replace("_var", "").replace("davidson_", "")
        h = pkg.from_csr(A, k=p["k"], nev=p["nev"], tol=1e-6, maxiter=1000, precond=pcond,
                         polish_fp64=1, stream=stream, seed=p["seed"], **extra)
        torch.cuda.synchronize()
        t_create = time.perf_counter() - t0
        train = None
        if pc == "mlp":
            t0 = time.perf_counter()
            hist, used = h.precond_train(X0, harvest_iters=20, n_pairs=1 << 20, epochs=5, lr=1e-3)
            train = {"train_s": round(time.perf_counter() - t0, 3), "pairs": int(used),
                     "held_out_mse": [round(float(v), 5) for v in hist]}
            train["apply"] = mlp_apply_report(h, A.n, p["k"], stream)
        def run_once(x0):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            try:
                X, ev, rs, st = h.davidson(x0) if pc.startswith("davidson") else h.solve(x0)
                ok = True
            except pkg.LobpcgError as e:
                X, ev, rs, st = e.result
                ok = False
            torch.cuda.synchronize()
            return (time.perf_counter() - t0, ev, rs, st, ok)
        runs = [run_once(X0d) for _ in range(max(1, repeats))]
        t_host = run_once(X0)[0]
        h.destroy()
        order = sorted(range(len(runs)), key=lambda i: runs[i][0])
        t_solve, ev, rs, st, ok = runs[order[len(order) // 2]]
        out[pc] = {"time_to_solution_s": round(t_solve, 3), "time_to_solution_host_s": round(t_host, 3),
                   "create_s": round(t_create, 3),
                   "iters": st["iters"], "iters_fp64": st["iters_fp64"], "converged": bool(ok and st["converged"]),
                   "max_resid": float(np.max(rs)), "evals": [float(v) for v in ev],
                   "runs": {"time_s": [round(r[0], 3) for r in runs], "iters": [r[3]["iters"] for r in runs],
                            "converged": [bool(r[4] and r[3]["converged"]) for r in runs]}}
        if gold is not None:
            out[pc]["eig_err_vs_oracle"] = eig_error(ev, gold)
        if train:
            out[pc]["training"] = train
            out[pc]["time_to_solution_with_training_s"] = round(t_solve + train["train_s"], 3)
    return out


def spmm_f64_report(pkg, A, p, stream, csr_bytes: int) -> dict:
    """The float64-vector SpMM (lobpcg_spmm_sym_f64: the refinement's
    explicit products, in compensated float32) on the same matrix: median
    of 5 launches, CUDA events, X seeded N(0, 1) in float64."""
    import torch
    n, k = A.n, p["k"]
    h = pkg.from_csr(A, k=k, nev=p["nev"], stream=stream)
    g = torch.Generator(device="cuda")
    g.manual_seed(p["seed"])
    with torch.cuda.stream(stream):
        X = torch.randn(n, k, device="cuda", dtype=torch.float64, generator=g)
        Y = torch.empty_like(X)
    for _ in range(2):
        h.spmm_sym_f64(X, Y)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
    for i in range(5):
        evs[i].record(stream)
        h.spmm_sym_f64(X, Y)
        evs[i + 1].record(stream)
    torch.cuda.synchronize()
    ms = statistics.median(evs[i].elapsed_time(evs[i + 1]) for i in range(5))
    h.destroy()
    # the float32 metric's bytes with X and Y in float64
    own = csr_bytes + 2 * n * k * 4
    return {"kernels": "k_split64, k_spmm_df_rows, k_spmm_df_cols (compensated float32)", "ms": round(ms, 3),
            "gbs_csr_equivalent_f64_vectors": round(own / (ms / 1e3) / 1e9, 1)}


def mlp_apply_report(h, n: int, k: int, stream) -> dict:
    """One learned-form application W = K_mlp^{-1} R on the n x k block
    (precond_apply, mode "mlp": the fused kernel), median of 5 launches timed
    with CUDA events on the handle's stream, R seeded N(0, 1).  Algorithmic
    FLOPs: 2 (129 256 + 256 64) per (64-row tile, column) pair, against the
    measured dense bf16 peak."""
    import torch
    pairs = (n + 63) // 64 * k
    with torch.cuda.stream(stream):
        g = torch.Generator(device="cuda").manual_seed(5)
        R = torch.randn(n, k, device="cuda", dtype=torch.float32, generator=g)
        W = torch.empty_like(R)
        th = torch.linspace(-1.0, 1.0, k, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    h.precond_apply(R, th, W, mode="mlp")
    ts = []
    for _ in range(5):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        h.precond_apply(R, th, W, mode="mlp")
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    ms = statistics.median(ts)
    tf = 2.0 * (129 * 256 + 256 * 64) * pairs / (ms / 1e3) / 1e12
    peak = measured_peaks()["bf16_tflops"]
    return {"kernel": "k_mlp_apply_fused", "pairs": int(pairs), "ms": round(ms, 4), "tflops": round(tf, 2),
            "frac_of_bf16_peak": round(tf / peak, 4)}


def mlp_kernels_report(pkg, stream, peak_tflops: float, rows: int = 500_000, batch: int = 4096) -> dict:
    """The learned preconditioner's network kernels, timed with CUDA events
    against the measured dense bf16 peak: the forward pass (129 -> 256 -> 64,
    bfloat16 tensor-core products, float32 accumulation) on `rows` inputs
    (one application at n = 2M, k = 16: 31,250 tiles x 16 columns), and the
    loss with its gradients (forward + backward) on one training batch of
    `batch` rows.  Algorithmic FLOPs: forward 2 B (129 256 + 256 64);
    gradients 3 x forward (the two weight gradients and the hidden layer's
    input gradient are each the size of a forward product)."""
    import torch
    A = synth.tile_matrix(256, 20, seed=7, fp32=True)
    h = pkg.from_csr(A, k=4, nev=1, precond="mlp", stream=stream, seed=7)
    g = torch.Generator(device="cpu").manual_seed(11)
    params = (torch.randn(49728, generator=g) * 0.05).numpy().astype(np.float32)
    h.mlp_set_params(params)
    with torch.cuda.stream(stream):
        Xin = torch.randn(rows, 129, device="cuda", dtype=torch.float32)
        Y = torch.empty(rows, 64, device="cuda", dtype=torch.float32)
        Xb = Xin[:batch].contiguous()
        T = torch.randn(batch, 64, device="cuda", dtype=torch.float32)
    torch.cuda.synchronize()

    def timed(fn, reps=5):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)
    f_ms = timed(lambda: h.mlp_forward(Xin, Y))
    g_ms = timed(lambda: h.mlp_grad(Xb, T))
    h.destroy()
    flop_row = 2.0 * (129 * 256 + 256 * 64)
    out = {"forward_rows": rows, "forward_ms": round(f_ms, 4), "grad_batch_rows": batch,
           "grad_ms": round(g_ms, 4),
           "forward_tflops": round(flop_row * rows / (f_ms / 1e3) / 1e12, 2),
           "grad_tflops": round(3 * flop_row * batch / (g_ms / 1e3) / 1e12, 2),
           "peak_bf16_tflops": peak_tflops, "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst)",
           "kernel": "k_gemm_bf16 (mma.sync m16n8k16 bf16, float32 accumulation)"}
    out["forward_frac"] = round(out["forward_tflops"] / peak_tflops, 4)
    out["grad_frac"] = round(out["grad_tflops"] / peak_tflops, 4)
    return out


def largest_report(pkg, stream, peak_gbs: float, workload: str = "largest_n8m") -> dict:
    """The largest workload (n = 8,000,000, ~250 stored entries per row, about
    2.0 G stored entries, k = 20, nev = 10): the SpMM kernel's time and
    fraction of the measured HBM peak, one LOBPCG iteration, and the
    time-to-1e-6 of the diagonal form and of the learned form (trained as in
    lobpcg_solves; a tile column whose correction is not finite or longer
    than the diagonal solve keeps the diagonal solve), one solve each.  The
    matrix is generated here (host), copied to the device once per form."""
    import torch
    p = synth.WORKLOADS[workload]
    t0 = time.perf_counter()
    A = synth.tile_matrix(p["n"], p["nnz_per_row"], seed=p["seed"], fp32=True)
    t_gen = time.perf_counter() - t0
    n, k, nnz = A.n, p["k"], A.nnz
    X0 = synth.initial_guess(A, k, seed=p["seed"] + synth.X0_SEED_OFFSET, fp32=True)
    out = {"workload": workload, "n": n, "nnz": int(nnz), "k": k, "nev": p["nev"],
           "generate_s": round(t_gen, 1)}
    for pc in ("diag", "mlp"):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h = pkg.from_csr(A, k=k, nev=p["nev"], tol=1e-6, maxiter=1000, precond=pc, polish_fp64=1,
                         stream=stream, seed=p["seed"])
        torch.cuda.synchronize()
        t_create = time.perf_counter() - t0
        if pc == "diag":
            with torch.cuda.stream(stream):
                X = torch.from_numpy(X0).cuda()
                Y = torch.empty_like(X)
            for _ in range(3):
                h.spmm_sym(X, Y)
            evs = [torch.cuda.Event(enable_timing=True) for _ in range(11)]
            for i in range(10):
                evs[i].record(stream)
                h.spmm_sym(X, Y)
                evs[i + 1].record(stream)
            torch.cuda.synchronize()
            ms = statistics.median(evs[i].elapsed_time(evs[i + 1]) for i in range(10))
            B = alg_bytes(n, nnz, k)
            out["spmm"] = {"kernel": f"k_spmm_sym_tiled<3, 20> (k={k})", "ms": round(ms, 4),
                           "alg_bytes_per_launch": int(B), "gbs": round(B / (ms / 1e3) / 1e9, 1),
                           "frac_of_peak": round(B / (ms / 1e3) / 1e9 / peak_gbs, 4), "traffic": None}
            h.iterate(3, X0=X)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            h.iterate(5)
            e1.record(stream)
            torch.cuda.synchronize()
            out["iteration_ms"] = round(e0.elapsed_time(e1) / 5, 3)
            del X, Y
        train = None
        if pc == "mlp":
            t0 = time.perf_counter()
            hist, used = h.precond_train(X0, harvest_iters=20, n_pairs=1 << 20, epochs=5, lr=1e-3)
            train = {"train_s": round(time.perf_counter() - t0, 3), "pairs": int(used)}
        with torch.cuda.stream(stream):
            X0d = torch.from_numpy(X0).cuda()   # resident in HBM when the timed solve starts
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        try:
            _, ev, rs, st = h.solve(X0d)
            ok = True
        except pkg.LobpcgError as e:
            _, ev, rs, st = e.result
            ok = False
        torch.cuda.synchronize()
        t_solve = time.perf_counter() - t0
        h.destroy()
        del X0d
        rec = {"time_to_solution_s": round(t_solve, 3), "create_s": round(t_create, 3), "iters": st["iters"],
               "iters_fp64": st["iters_fp64"], "converged": bool(ok and st["converged"]),
               "max_resid": float(np.max(rs)), "evals": [float(v) for v in ev]}
        if train:
            rec["training"] = train
            rec["time_to_solution_with_training_s"] = round(t_solve + train["train_s"], 3)
        out[pc] = rec
    if "diag" in out and "mlp" in out:
        a, b = np.array(out["diag"]["evals"]), np.array(out["mlp"]["evals"])
        out["forms_agree_max_rel"] = float(np.max(np.abs(a - b) / np.abs(a)))
    return out


def value_only_report(pkg, A, p, stream, spmm_csr_ms: float, peak_gbs: float) -> dict:
    """The SpMM and the diagonal-preconditioned solve with tile_format 1
    (complete 16x16 tiles and complete diagonal triangles keep value words
    only).  Reported beside, not in, the CSR-equivalent metric: its bytes are
    its own stream (values, the index words of incomplete tiles, chunk
    records, row-block table) plus X and Y."""
    import torch
    n, k = A.n, p["k"]
    h = pkg.from_csr(A, k=k, nev=p["nev"], tol=1e-6, maxiter=1000, precond="diag", polish_fp64=1,
                     stream=stream, seed=p["seed"], tile_format=1)
    info = h.info()
    R = info["row_blocks"]
    own = info["stream_bytes"] + 16 * info["chunks"] + 8 * (R + 1) + 2 * n * k * 4
    with torch.cuda.stream(stream):
        X = torch.randn(n, k, device="cuda", dtype=torch.float32)
        Y = torch.empty_like(X)
    for _ in range(3):
        h.spmm_sym(X, Y)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(21)]
    for i in range(20):
        evs[i].record(stream)
        h.spmm_sym(X, Y)
        evs[i + 1].record(stream)
    torch.cuda.synchronize()
    ms = statistics.median(evs[i].elapsed_time(evs[i + 1]) for i in range(20))
    X0 = synth.initial_guess(A, k, seed=p["seed"] + synth.X0_SEED_OFFSET, fp32=True)
    t0 = time.perf_counter()
    try:
        _, ev, rs, st = h.solve(X0)
        ok = True
    except pkg.LobpcgError as e:
        _, ev, rs, st = e.result
        ok = False
    t_solve = time.perf_counter() - t0
    h.destroy()
    gbs = own / (ms / 1e3) / 1e9
    return {"tile_format": 1, "spmm_ms": round(ms, 4), "bytes_per_launch": int(own),
            "stream_bytes": int(info["stream_bytes"]), "gbs_own_bytes": round(gbs, 1),
            "frac_of_peak": round(gbs / peak_gbs, 4), "speedup_vs_csr_equivalent": round(spmm_csr_ms / ms, 3),
            "lobpcg_diag": {"time_to_solution_s": round(t_solve, 3), "iters": st["iters"],
                            "iters_fp64": st["iters_fp64"], "converged": bool(ok and st["converged"]),
                            "max_resid": float(np.max(rs)), "evals": [float(v) for v in ev]}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(synth.WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-solves", action="store_true")
    ap.add_argument("--forms", default="diag,bjacobi,fom,fom_var,mlp,davidson_diag",
                    help="comma-separated solve forms of the lobpcg sub-record")
    ap.add_argument("--solve-repeats", type=int, default=3, help="solves per preconditioner form (median reported)")
    ap.add_argument("--no-largest", action="store_true", help="skip the n = 8M sub-record")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-value-only", action="store_true")
    ap.add_argument("--no-f64", action="store_true", help="skip the float64-vector SpMM sub-record")
    ap.add_argument("--fom-only", action="store_true",
                    help="only the FOM preconditioner report (fom_apply) on the workload; for profiling")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import paper_2109_00485_gb300 as pkg

    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pkg.load()

    p = synth.WORKLOADS[args.workload]
    tdt = {np.int64: torch.int64, np.int32: torch.int32, np.float32: torch.float32, np.float64: torch.float64}
    pinned = lambda shape, dt: torch.empty(shape, dtype=tdt[dt], pin_memory=True).numpy()
    A = synth.tile_matrix(p["n"], p["nnz_per_row"], seed=p["seed"], fp32=True, alloc=pinned)
    n, k, nnz = A.n, p["k"], A.nnz
    stream = torch.cuda.Stream(device=dev)
    if args.fom_only:
        if rank == 0:
            print(json.dumps({"workload": args.workload, "fom_apply": fom_report(pkg, A, p, stream,
                                                                                measured_peaks()["sm_max_mhz"])}))
        return
    h = pkg.from_csr(A, k=k, nev=p["nev"], tol=1e-6, maxiter=1000, precond="diag", stream=stream)
    X0 = synth.initial_guess(A, k, seed=p["seed"] + synth.X0_SEED_OFFSET, fp32=True)
    with torch.cuda.stream(stream):
        X0d = torch.from_numpy(X0).to(dev)
    torch.cuda.synchronize()
    info = h.info()
    B = alg_bytes(n, nnz, k)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    # warm-up: start a run from X0 and take W iterations
    h.iterate(max(args.warmup, 3), X0=X0d)
    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    theta, st = h.iterate(args.steps)          # the timed steps: K LOBPCG iterations
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier()
    total_ms, value = aggregate(e0.elapsed_time(e1), B, args.steps, world, dev)
    ms_step = total_ms / args.steps
    spmm_ms = st["spmm_ms"] / max(1, st["spmm_calls"])

    # e2e: the same metric through lobpcg_spmm_sym with pinned HOST X and Y
    Xh = torch.empty((n, k), dtype=torch.float32, pin_memory=True)
    Xh.copy_(torch.from_numpy(X0))
    Yh = torch.empty((n, k), dtype=torch.float32, pin_memory=True)
    h.spmm_sym_host(Xh, Yh)
    h.sync()
    barrier()
    t0 = time.perf_counter()
    e2e_steps = max(1, args.e2e_steps)
    for _ in range(e2e_steps):
        h.spmm_sym_host(Xh, Yh)
    h.sync()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    e2e = {"value": round(B * world / e2e_s / 1e9, 2), "unit": "GB/s",
           "h2d_bytes_per_step": n * k * 4, "d2h_bytes_per_step": n * k * 4,
           "call": "lobpcg_spmm_sym with pinned host X, Y"}
    h.destroy()

    peaks = measured_peaks()
    achieved = B / (spmm_ms / 1e3) / 1e9
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": round(achieved / peaks["hbm_gbs"], 4), "traffic": recorded_traffic(args.workload),
                "peak_source": f"{peaks['source']} (MEASURED_PEAKS.json hbm_gbs, burst copy)",
                "kernel": f"k_spmm_sym_tiled<{(k + 7) // 8}, {k if k in (8, 16, 20, 32) else 0}> (k={k})",
                "alg_bytes_per_launch": B,
                "kernel_ms": round(spmm_ms, 4)}

    solves = None
    if rank == 0 and not args.no_solves:
        forms = tuple(f for f in args.forms.split(",") if f)
        solves = lobpcg_solves(pkg, A, p, stream, precs=forms, repeats=args.solve_repeats,
                               gold=golden_evals(args.workload))
    fom = None
    if rank == 0 and not args.no_solves:
        fom = fom_report(pkg, A, p, stream, peaks["sm_max_mhz"])
    vonly = None
    if rank == 0 and not args.no_value_only and not args.no_solves:
        vonly = value_only_report(pkg, A, p, stream, spmm_ms, peaks["hbm_gbs"])
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(A, k)
    mlpk = None
    if rank == 0 and not args.no_solves:
        mlpk = mlp_kernels_report(pkg, stream, peaks["bf16_tflops"])
    f64 = None
    if rank == 0 and not args.no_f64:
        f64 = spmm_f64_report(pkg, A, p, stream, B)
    largest = None
    if rank == 0 and not args.no_largest and not args.no_solves and args.workload == WORKLOAD:
        del A   # the n = 2M matrix's pinned host copy
        largest = largest_report(pkg, stream, peaks["hbm_gbs"])

    if rank == 0:
        line = {"metric": "symmetric SpMM GB/s", "value": round(value, 2), "unit": "GB/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 4),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": args.workload, "n": n, "nnz": nnz, "k": k, "nev": p["nev"],
                           "step": "one LOBPCG iteration (residual+diag preconditioner, 2x CholQR, SpMM H W, "
                                   "Gram, Rayleigh-Ritz, update); value = SpMM algorithmic bytes per step / step time",
                           "structure": "16x16 dense tiles, 90% within 5% of the diagonal, 10% scattered",
                           "l2": "inputs (6.4 GB matrix stream) larger than L2; no flush",
                           "parallelism": "replicas" if world > 1 else "single"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
                "gpu_launches": LAUNCHES_PER_ITERATION * args.steps,
                "gflops_spmm": round(4.0 * k * nnz / (spmm_ms / 1e3) / 1e9, 1),
                "lobpcg": solves,
                "fom_apply": fom,
                "value_only_tiles": vonly,
                "mlp_kernels": mlpk,
                "spmm_f64": f64,
                "largest": largest,
                "layout": {"chunks": info["chunks"], "full_chunks": info["full_chunks"],
                           "padded_nnz": info["padded_nnz"], "warps": info["warps"]}}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
