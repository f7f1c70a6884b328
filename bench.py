"""Benchmark of the mArnoldi hot path on GB300: columns per second.

One step = one pass of the whole hot path over the workload: every column's
Krylov subspace, S-orthonormalisation, subspace eigensolve, the Fermi level by
bisection, and the density / energy-density columns written on H's pattern
(device buffers) with the band energy reduced.

Default workload: 4,096-atom random-packed amorphous carbon (M = 16,384), global
mode, nu = 30, all 16,384 columns, kT = 0.1 eV, 4 electrons per atom.  The
headline `value` is mixed precision; the FP64 path is timed beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl marnoldi|reference]

Under torchrun (N > 1) every rank solves its own copy of the workload
(independent problems, no collective on the data path); rank 0 prints the
whole-job rate from the slowest rank's time.  `--impl reference` times the CPU
oracle instead (rank 0 only).
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

KT = 0.1
REFERENCE_MU = 4.185   # Fermi level of the default workload (eV); the sampled oracle arm uses it fixed
METRIC = "mArnoldi columns/s"
UNIT = "columns/s"
L2_FLUSH_BYTES = 256 << 20
FP64_PEAK_NOTE = "152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz (nominal 1.25 TFLOP/s FP64)"
# (dram__bytes_read + dram__bytes_write) / algorithmic bytes of one captured
# Gram-Schmidt launch (ncu --set full, mixed precision, 608 columns, step n = 20,
# algorithmic 1.929072e9 B read + 0.039846e9 B written over the supports), per
# precision and launch shape (values per thread, threads) of the kernel that was
# captured; a shape without an entry reports no traffic.  An entry must be
# re-measured (or removed) whenever its kernel changes.
# gs_stream_kernel<256,16384,3,2> (shape 64 x 288, two CTAs per SM): (2.363514e9 + 0.038593e9)
# / 1.968918e9; above 1 by the re-reads of u, its lo word and w_n with every block that miss L2
# despite their evict-last hint (twice as many columns share L2 as with one CTA per SM).
# gs_stream_kernel<512,16384,4,1> (shape 32 x 544, one CTA per SM; chosen through a tune cache):
# (2.024088e9 + 0.038078e9) / 1.968918e9.
GS_DRAM_PER_ALGORITHMIC = {("mixed", (64, 288)): 1.2200, ("mixed", (32, 544)): 1.0474}
GS_DRAM_KERNEL = {(64, 288): "gs_stream_kernel<256,16384,3,2>", (32, 544): "gs_stream_kernel<512,16384,4,1>"}
# SHA-256 of the sources of each captured kernel; when they differ from the files
# on disk the capture no longer describes the kernel and no traffic is reported
_GS_STREAM_SOURCES = {
    "paper_1307_3218_gb300/csrc/gs_stream.cu": "340e6c10e95f7d1e86a82211f1ddcad5ee2a72a0f817bc552caa00582069825d",
    "paper_1307_3218_gb300/csrc/gs_common.cuh": "c17924ab36aeabf9b8ba5efafff26274875b1c7d799fc4bfb056719952d4d512"}
GS_DRAM_SOURCES = {(64, 288): _GS_STREAM_SOURCES, (32, 544): _GS_STREAM_SOURCES}


def capture_current(shape) -> bool:
    """True when the sources of the kernel whose DRAM ratio is recorded for `shape` are unchanged."""
    import hashlib
    want = GS_DRAM_SOURCES.get(shape)
    if not want:
        return False
    for rel, digest in want.items():
        try:
            if hashlib.sha256(open(os.path.join(ROOT, rel), "rb").read()).hexdigest() != digest:
                return False
        except OSError:
            return False
    return True


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="marnoldi", choices=["marnoldi", "reference"])
    p.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    p.add_argument("--nu", type=int, default=30)
    p.add_argument("--atoms", type=int, default=4096)
    p.add_argument("--columns", type=int, default=0, help="solve only the first N columns (0 = all)")
    p.add_argument("--no-fp64", action="store_true", help="skip the FP64 side measurement")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-extra", action="store_true",
                   help="skip the nu=100 and regional side measurements")
    p.add_argument("--no-serving", action="store_true", help="skip the request-server measurement")
    p.add_argument("--c4", action="store_true",
                   help="only the polymer-chain batching workload as configured (256 chains, 4..400 units)")
    p.add_argument("--c5", action="store_true",
                   help="only the Poisson serving workload as configured (1,000-200,000 atoms, a sweep of rates)")
    p.add_argument("--c5-window", type=float, default=30.0)
    p.add_argument("--c5-rates", default="1.0,0.5,0.25,0.125",
                   help="Poisson arrival rates (requests/s) of the --c5 sweep, highest first")
    p.add_argument("--chain", type=int, default=0,
                   help="only a per-kernel breakdown of one polymer chain of this many units in regional "
                        "mode (256-atom regions) at each nu of --chain-nu")
    p.add_argument("--chain-nu", default="100,300")
    p.add_argument("--mixed-vs-fp64", default="",
                   help="comma-separated nu list: mixed against FP64 on every column of the benchmark "
                        "structure (density statistics at the FP64 Fermi level) and exit")
    p.add_argument("--large-full", type=int, default=0,
                   help="only the paper-scale structure of this many atoms at nu = 100, every column, in "
                        "65,536-column batches, mixed and FP64 (e.g. 1048576)")
    p.add_argument("--large", type=int, default=0,
                   help="atoms of the paper-scale regional run (e.g. 1048576); 0 = skip")
    p.add_argument("--order-n", default="",
                   help="comma-separated atom counts for the order-N study (regional mode), e.g. "
                        "4096,16384,65536,262144; empty = skip")
    p.add_argument("--fixed-shapes", action="store_true",
                   help="fixed Gram-Schmidt launch-shape rule instead of the autotuner (use it under a "
                        "profiler: the tuner's CUDA-event timings are meaningless when every kernel is "
                        "serialised and replayed)")
    p.add_argument("--serve-requests", type=int, default=60)
    p.add_argument("--serve-workers", type=int, default=4)
    p.add_argument("--serve-budget-gb", type=float, default=64.0)
    p.add_argument("--cpu-seconds", type=float, default=15.0)
    p.add_argument("--region", type=int, default=0,
                   help="regional mode with this many atoms per region (0 = global mode)")
    return p.parse_args()


def workload(args):
    from tbsynth import amorphous_system
    t = amorphous_system(args.atoms, seed=0)
    cols = t.real_columns()
    if args.columns:
        cols = cols[:args.columns]
    return t, cols


def electrons(t, cols) -> float:
    """Target electron count of the solved columns: the structure's count scaled to the subset."""
    return float(t.n_electrons) * len(cols) / len(t.real_columns())


def workload_name(args, t, ncols):
    return (f"amorphous sp2-sp3 carbon {t.n_block_rows} atoms (M={t.M}, 3.0 g/cm^3, seed 0), "
            f"{mode_name(args)}, nu={args.nu}, {ncols} columns, kT={KT} eV, mu by bisection at 4 e/atom")


def mode_name(args) -> str:
    return f"regional mode ({args.region}-atom regions)" if args.region else "global mode"


# ------------------------------------------------------------------------ measurement helpers

def read_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi while the timed region runs."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.proc = None
        self.path = None
        self.dev = device_index

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
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
        rows = []
        for ln in open(self.path):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 7:
                continue
            try:
                rows.append((float(f[0]), float(f[1]), float(f[2]), f[3:7]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[3]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "power_w_max": max(r[2] for r in rows), "samples": len(rows), "reasons": reasons}


def gs_algorithmic(nu: int, m: int, vbytes: int, ncols: int):
    """Bytes the Gram-Schmidt step must stream and FP64 flops it must do (dense vectors).

    Step n (0-based) loads u (and its lo word in mixed precision) and w_n, reads
    w_i and S w_i of every stored vector i <= n once for the coefficients
    (a_i = w_i . u, b_i = S w_i . u, g_i = S w_i . w_n) and, for n < nu-1, w_i once
    more for the subtraction, and writes the new w.  Flops: three dots per entry
    and stored vector and one update (the last step: two dots).
    """
    vals = fmas = 0
    for n in range(nu):
        need_w = n + 1 < nu
        vals += (2 if vbytes == 4 else 1) + 1 + 2 * (n + 1) + ((n + 1) + 1 if need_w else 0)
        fmas += (4 if need_w else 2) * (n + 1)
    return vals * m * vbytes * ncols, 2.0 * fmas * m * ncols


def column_m_pad(m: int) -> int:
    """Padded vector length of the column-per-CTA kernels (256 or 1024 threads x a power of two <= 16)."""
    T = 256 if m <= 4096 else 1024
    v = 1
    while v < 16 and v * T < m:
        v *= 2
    return v * T


def support_counts(t, cols, nu: int, m_pad: int):
    """tcnt[c][L]: tiles of 8 atoms (32 vector entries) within L pattern hops of column c's atom.

    Basis vector w_i of column c vanishes outside the tiles with L <= i, S w_i and
    H w_i outside L <= i + 1 (breadth-first hop counts over the block pattern).
    """
    import scipy.sparse as sp
    from scipy.sparse.csgraph import shortest_path
    nbr = t.n_block_rows
    G = sp.csr_matrix((np.ones(len(t.col_idx)), t.col_idx, t.row_ptr), shape=(nbr, nbr))
    atoms, inv = np.unique(np.asarray(cols) // 4, return_inverse=True)
    ntile = m_pad // 32
    out = np.zeros((len(atoms), nu + 2), dtype=np.int64)
    for a0 in range(0, len(atoms), 512):
        D = shortest_path(G, unweighted=True, indices=atoms[a0:a0 + 512])
        D = np.where(np.isfinite(D), D, 1e9)
        if ntile * 8 > nbr:
            D = np.concatenate([D, np.full((D.shape[0], ntile * 8 - nbr), 1e9)], axis=1)
        th = D.reshape(D.shape[0], ntile, 8).min(axis=2)
        for L in range(nu + 2):
            out[a0:a0 + 512, L] = (th <= L).sum(axis=1)
    return out[inv]


def gs_algorithmic_support(nu: int, tcnt, vbytes: int):
    """Bytes and FP64 flops of the Gram-Schmidt steps over the basis vectors' supports.

    As gs_algorithmic, but every vector counts only the entries of its support
    tiles (32 entries per tile): u (and its lo word) and the new w within n + 1
    hops, w_n within n, the pair w_i, S w_i and the subtraction's w_i within
    i + 1.
    """
    E = 32.0 * np.asarray(tcnt).sum(axis=0)   # entries within L hops, summed over columns
    vals = fmas = 0.0
    for n in range(nu):
        need_w = n + 1 < nu
        s = sum(E[i + 1] for i in range(n + 1))
        vals += (2 if vbytes == 4 else 1) * E[n + 1] + E[n] + 2 * s
        fmas += 2 * s
        if need_w:
            vals += s + E[n + 1]
            fmas += 2 * s
    return vals * vbytes, 2.0 * fmas


def spmm_algorithmic(nu: int, m: int, nnzb: int, nbr: int, vbytes: int, ncols: int):
    """Per column and application: read x, write y (m values each); flops 2 * 16 nnzb."""
    apps = 2 * nu - 1
    return apps * 2 * m * vbytes * ncols, apps * 2.0 * 16 * nnzb * ncols


FP32_INST_PEAK = 152 * 128 * 2.07e9   # FP32 instructions/s: 152 SMs x 128 lanes x 2.07 GHz (nominal)
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def eig_flops(nu: int, rows: int) -> float:
    """FP64 flops of one subspace eigensolve (model), with rows = n_pat + 2 rows of R = [e_1; q; K_pat]:
    L^-1 H L^-T (4/3 nu^3: the full first product, the lower triangle of the second), Householder
    tridiagonalisation of a symmetric matrix (4/3 nu^3), R L^-T and R's reflections (3 rows nu^2),
    implicit QL with about nu^2 Givens rotations (20 nu^2) and their replay on R (6 rows nu^2)."""
    return 8.0 / 3.0 * nu ** 3 + 9.0 * rows * nu * nu + 20.0 * nu * nu


def eig_roofline(t, cols, nu: int, eig_stats, steps: int):
    """The eigensolver's FP64 rate over a timed region: model flops of every column (eig_flops with
    each column's pattern rows) / the summed CUDA-event time of its kernels, against the FP64 peak
    derived from the unit counts (GB300's FP64 pipe: 2 FMA per clock per SM)."""
    n_launch, ms = eig_stats
    if ms <= 0:
        return None
    blocks = np.diff(np.asarray(t.row_ptr))[np.asarray(cols) // 4]
    flops = float(sum(eig_flops(nu, 4 * int(b) + 2) for b in blocks)) * steps
    ach = flops / (ms / 1e3) / 1e12
    return {"kernel": "eigsub (tridiagonalisation, QL, replay)", "bound": "alu", "achieved": round(ach, 4),
            "peak": round(FP64_PEAK_TFLOPS, 3), "unit": "TFLOP/s", "frac": round(ach / FP64_PEAK_TFLOPS, 4),
            "peak_source": "derived: " + FP64_PEAK_NOTE, "launches": n_launch,
            "model": "per column 8/3 nu^3 + 9 r nu^2 + 20 nu^2 flops, r = pattern rows + 2 (about nu^2 "
                     "QL rotations)"}


def spmm_instructions_support(t, tcnt, nu: int, prec: int):
    """FP32 (mixed) or FP64 arithmetic instructions of the fused H and S products
    over the rows within the output support, summed over the columns and steps.

    Step n computes the rows of tiles within n + 1 hops (8 rows per tile, the
    structure's mean blocks per row); per block and column: 16 products of H,
    each an exact product, a fused lo product and a two-sum (11 FP32
    instructions; FP64: 1 FMA), plus 16 FMAs of S from step 1 on.
    """
    rows = 8.0 * np.asarray(tcnt).sum(axis=0)            # rows within L hops, summed over columns
    bpr = t.nnzb / t.n_block_rows
    h_inst = 11.0 if prec == 1 else 1.0
    total = 0.0
    for n in range(nu):
        total += rows[n + 1] * bpr * 16.0 * (h_inst + (1.0 if n > 0 else 0.0))
    return total


# ------------------------------------------------------------------------ GPU arm

def time_gpu(m, t, cols, args, prec, steps, warmup, dev, measure_clocks=False):
    import torch
    stream = torch.cuda.current_stream()
    ctx = m.setup_system(t, prec)
    rho = torch.empty(t.nnzb * 16, dtype=torch.float64, device=dev)
    rhoE = torch.empty_like(rho)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    colsel = None if len(cols) == t.M else cols

    ne = electrons(t, cols)

    def step():
        m.marnoldi_solve(ctx, colsel, args.nu, args.region, ne, KT)
        m.marnoldi_density_device(ctx, rho, rhoE)

    for _ in range(warmup):
        step()
        flush.fill_(1.0)
    torch.cuda.synchronize()
    m.marnoldi_set_profiling(ctx, True)
    m.marnoldi_kernel_stats(ctx, reset=True)
    clk = Clocks(dev.index if dev.index is not None else 0) if measure_clocks else None
    if clk:
        clk.start()
    times = []
    if torch.distributed.is_initialized():
        torch.distributed.barrier()
    torch.cuda.synchronize()
    for _ in range(steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        flush.fill_(float(len(times)))   # L2 flush between timed steps, outside the events
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    if torch.distributed.is_initialized():
        torch.distributed.barrier()
    clocks = clk.stop() if clk else None
    stats = m.marnoldi_kernel_stats(ctx)
    E, mu, N = m.marnoldi_energy(ctx)
    res = dict(times=times, stats=stats, E=E, mu=mu, N=N, clocks=clocks, ctx=ctx,
               gs_shape=tuple(m.marnoldi_gs_shape(ctx)))
    return res


def time_e2e(m, t, cols, args, prec, steps, warmup):
    """Through the public API with host buffers: upload, solve, density to host, energy."""
    import torch
    colsel = None if len(cols) == t.M else cols

    ne = electrons(t, cols)

    def step():
        ctx = m.setup_system(t, prec)
        m.marnoldi_solve(ctx, colsel, args.nu, args.region, ne, KT)
        rho, rhoE = m.marnoldi_density(ctx)
        E, mu, N = m.marnoldi_energy(ctx)
        m.marnoldi_destroy(ctx)
        return rho

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    ts = []
    for _ in range(steps):
        t0 = time.perf_counter()
        step()
        torch.cuda.synchronize()
        ts.append(time.perf_counter() - t0)
    h2d = (8 * (t.n_block_rows + 1) + 4 * t.nnzb + 2 * 128 * t.nnzb + 8 * t.M + 8 * t.nnzb
           + (2 * 128 * t.nnzb if prec == 1 else 0) + (0 if colsel is None else 8 * len(cols)))
    d2h = 2 * 128 * t.nnzb
    return statistics.mean(ts), h2d, d2h


def gpu_outputs(m, ctx, cols, nu, prec):
    """What the oracle checks compare: mu, the density arrays and the levels of a solved context."""
    rho, rhoE = m.marnoldi_density(ctx)
    E, mu, N = m.marnoldi_energy(ctx)
    _, eps, _ = m.marnoldi_column_stats(ctx)
    return dict(mu=mu, rho=rho, rhoE=rhoE, eps=eps, cols=np.asarray(cols), nu=nu, prec=prec)


# ------------------------------------------------------------------------ CPU oracle

def oracle_checks(t, checks, n_sample=48):
    """GPU results against the oracle on seeded columns of each measured configuration.

    The oracle recomputes the sampled columns at the GPU's mu; the maxima of the
    differences over those columns' pattern entries and levels are reported with
    the tolerance that applies (FP64: 1e-10 relative; mixed: 1e-5 on rho, 1e-4 eV
    on rho^E).
    """
    import oracle
    out = {}
    for label, g in checks.items():
        rng = np.random.default_rng(7)
        pick = np.sort(rng.choice(g["cols"].size, size=min(n_sample, g["cols"].size), replace=False))
        sample = g["cols"][pick]
        ref = oracle.solve(t, nu=g["nu"], kT=KT, mu_fixed=g["mu"], cols=sample)
        mask = ~np.isnan(ref.rho)
        drho = float(np.abs(g["rho"][mask] - ref.rho[mask]).max())
        drhoE = float(np.abs(g["rhoE"][mask] - ref.rhoE[mask]).max())
        deps = float(np.nanmax(np.abs(g["eps"][pick] - ref.cols.eps)))
        if g["prec"] == 0:
            tol = {"rho": 1e-10 * float(np.abs(ref.rho[mask]).max()),
                   "rhoE": 1e-10 * float(np.abs(ref.rhoE[mask]).max())}
        else:
            tol = {"rho": 1e-5, "rhoE": 1e-4}
        out[label] = {"columns": int(sample.size), "nu": g["nu"], "max_abs_drho": drho,
                      "max_abs_drhoE_eV": drhoE, "max_abs_deps_eV": deps, "tolerance": tol,
                      "within": bool(drho <= tol["rho"] and drhoE <= tol["rhoE"])}
    return out


def oracle_sample(t, args, budget_s, mu=None):
    """Time the oracle on a bounded seeded sample of columns (all host cores)."""
    import oracle
    rng = np.random.default_rng(1234)
    allc = t.real_columns()
    nth = oracle.threads()
    n = max(nth, 16)
    t0 = time.perf_counter()
    oracle.columns(t, rng.choice(allc, size=n, replace=False), args.nu)
    dt = time.perf_counter() - t0
    n2 = int(min(len(allc), max(n, budget_s / max(dt / n, 1e-6))))
    sample = np.sort(rng.choice(allc, size=n2, replace=False))
    t0 = time.perf_counter()
    c = oracle.columns(t, sample, args.nu)
    if mu is not None:
        oracle.density_rows(c, mu, KT)
    dt = time.perf_counter() - t0
    return dict(value=n2 / dt, cores=nth, n=n2, seconds=dt, cols=c, sample=sample)


# ------------------------------------------------------------------------ main

def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        return main_reference(args, world, rank)

    import torch
    import paper_1307_3218_gb300 as m
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if world > 1:
        torch.distributed.init_process_group("nccl", device_id=dev)
    m.load()
    m.marnoldi_set_autotune(0 if args.fixed_shapes else 1)
    if args.chain:
        print(json.dumps({"metric": "mArnoldi columns/s", "n_gpus": 1, "data": "synthetic",
                          "chain": chain_breakdown(m, args.chain, [int(x) for x in args.chain_nu.split(",")])}))
        return
    if args.mixed_vs_fp64:
        for nu in [int(x) for x in args.mixed_vs_fp64.split(",")]:
            print(json.dumps({"mixed_vs_fp64": mixed_vs_fp64(m, nu)}), flush=True)
        return
    if args.large_full:
        print(json.dumps({"metric": "mArnoldi columns/s", "n_gpus": 1, "data": "synthetic",
                          "large_full": large_full(m, args.large_full, 256, 65536)}))
        return
    if args.c4 or args.c5:
        # the configured batching / serving workloads alone (one JSON line of their own)
        prec = 1 if args.precision == "mixed" else 0
        budget = int(args.serve_budget_gb * 2**30)
        out = {"metric": "mArnoldi columns/s and serve p50/p99 ms", "n_gpus": 1, "data": "synthetic"}
        if args.c4:
            out["c4"] = serve_c4(m, args.serve_workers, budget, prec)
        if args.c5:
            out["c5"] = serve_c5(m, args.serve_workers, budget, prec, window_s=args.c5_window,
                                 rates=tuple(float(x) for x in args.c5_rates.split(",")))
        print(json.dumps(out))
        return
    t, cols = workload(args)
    ncols = len(cols)
    prec = 1 if args.precision == "mixed" else 0
    res = time_gpu(m, t, cols, args, prec, args.steps, args.warmup, dev, measure_clocks=(rank == 0))
    step_s = statistics.mean(res["times"]) / 1e3
    tmax = torch.tensor([step_s], dtype=torch.float64, device=dev)
    if world > 1:
        torch.distributed.all_reduce(tmax, op=torch.distributed.ReduceOp.MAX)
    step_s = float(tmax.item())
    value = world * ncols / step_s
    stats = res["stats"]
    launches = sum(v[0] for v in stats.values())
    peaks = read_peaks()

    # roofline of the dominant kernel over the timed region (vector length: M, or 4 n_reg)
    m_vec = 4 * args.region if args.region else t.M
    vb = 4 if prec == 1 else 8
    dom = max(stats, key=lambda k: stats[k][1])
    nlaunch, dom_ms = stats[dom]
    steps = args.steps
    tcnt = None if args.region else support_counts(t, cols, args.nu, column_m_pad(m_vec))
    if dom == "gs":
        by, fl = (gs_algorithmic_support(args.nu, tcnt, vb) if tcnt is not None
                  else gs_algorithmic(args.nu, m_vec, vb, ncols))
    elif dom in ("spmm_H", "spmm_S", "spmm_HS"):
        by, fl = spmm_algorithmic(args.nu, m_vec, t.nnzb, t.n_block_rows, vb, ncols)
        if dom != "spmm_HS":
            by, fl = by / 2, fl / 2
    else:
        by, fl = None, None
    if prec == 1 and by is not None:
        bound, ach, peak, unit = "hbm", by * steps / (dom_ms / 1e3) / 1e9, peaks.get("hbm_gbs", 6800.0), "GB/s"
        peak_src = "measured (MEASURED_PEAKS.json hbm_gbs)" if "hbm_gbs" in peaks else "fallback"
    elif by is not None:
        bound, ach, unit = "alu", fl * steps / (dom_ms / 1e3) / 1e12, "TFLOP/s"
        peak, peak_src = 152 * 2 * 2 * 2.07e9 / 1e12, "derived: " + FP64_PEAK_NOTE
    else:
        bound = ach = peak = unit = peak_src = None
    roof = None
    if ach is not None:
        # DRAM bytes per average launch: the ncu capture's DRAM/algorithmic ratio for
        # this kernel (a smaller case of the same kernel; bytes scale with columns and
        # stored vectors) times the algorithmic bytes per launch
        gs_shape = res.get("gs_shape")
        ratio = (GS_DRAM_PER_ALGORITHMIC.get((args.precision, gs_shape))
                 if dom == "gs" and not args.region and capture_current(gs_shape) else None)
        launches_per_step = nlaunch / steps
        traffic = round(ratio * by / launches_per_step) if ratio and by else None
        roof = {"kernel": dom, "bound": bound, "achieved": round(ach, 3), "peak": round(peak, 3),
                "unit": unit, "frac": round(ach / peak, 4), "traffic": traffic,
                "traffic_note": ("dram bytes per average launch = DRAM/algorithmic "
                                 f"{ratio} (ncu, {GS_DRAM_KERNEL.get(gs_shape)}, step n=20, 608 columns) "
                                 "x algorithmic bytes per launch") if traffic else None,
                "gs_shape": list(gs_shape) if gs_shape else None,
                "peak_source": peak_src, "launches": nlaunch, "avg_launch_ms": round(dom_ms / nlaunch, 4),
                "algorithmic_per_step": {"bytes": by, "flops": fl}}

    spmm_roof = None
    if tcnt is not None and stats.get("spmm_HS", (0, 0.0))[1] > 0:
        inst = spmm_instructions_support(t, tcnt, args.nu, prec) * steps
        ach_i = inst / (stats["spmm_HS"][1] / 1e3)
        pk = FP32_INST_PEAK if prec == 1 else FP32_INST_PEAK / 64.0
        spmm_roof = {"kernel": "spmm_HS", "bound": "alu", "achieved": round(ach_i / 1e12, 3), "peak": round(pk / 1e12, 3),
                     "unit": "T FP32 inst/s" if prec == 1 else "T FP64 inst/s", "frac": round(ach_i / pk, 4),
                     "peak_source": "nominal: 152 SMs x 128 FP32 lanes x 2.07 GHz (FP64: 1/64)",
                     "note": "H products error-free in FP32 (11 instructions each) over L2-resident "
                             "panels: bound by FP32 issue, not by HBM"}

    line = {
        "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(step_s * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if prec == 1 else "f64", "data": "synthetic",
        "config": {"workload": workload_name(args, t, ncols), "precision": args.precision,
                   "nu": args.nu, "columns": ncols, "atoms": t.n_block_rows, "M": t.M,
                   "nnzb": t.nnzb, "mode": mode_name(args),
                   "gs_shape_rule": "fixed" if args.fixed_shapes else "autotuned",
                   "l2": f"flushed between timed steps ({L2_FLUSH_BYTES >> 20} MB write)",
                   "parallelism": f"{world} independent replica(s)" if world > 1 else "1 GPU"},
        "roofline": roof,
        "spmm_roofline": spmm_roof,
        "eig_roofline": (eig_roofline(t, cols, args.nu, stats["eigsub"], steps)
                         if "eigsub" in stats and not args.region else None),
        "gpu_launches": int(launches),
        "kernel_ms_per_step": {k: round(v[1] / steps, 3) for k, v in stats.items() if v[0]},
        "clocks": res["clocks"],
        "result": {"E_band_eV": res["E"], "mu_eV": res["mu"], "N": res["N"]},
    }
    mu_gpu = res["mu"]
    checks = {"headline": gpu_outputs(m, res["ctx"], cols, args.nu, prec)}
    if not args.no_extra and len(cols) == len(t.real_columns()):
        # forces from the headline solve: density, derivative upload, one kernel, read-back
        from tbsynth import build_tb_derivatives
        dH, dS = build_tb_derivatives(t)
        m.marnoldi_forces(res["ctx"], dH, dS)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        F = m.marnoldi_forces(res["ctx"], dH, dS)
        line["forces"] = {"ms": round((time.perf_counter() - t0) * 1e3, 3),
                          "includes": "rho and rho^E on the device, dH/dS upload (host arrays), "
                                      "force kernel, read-back",
                          "max_abs_eV_per_A": round(float(np.abs(F).max()), 6),
                          "abs_sum_eV_per_A": float(np.abs(F.sum(axis=0)).max())}
    m.marnoldi_destroy(res["ctx"])

    if not args.no_fp64 and prec == 1:
        r64 = time_gpu(m, t, cols, args, 0, max(3, args.steps // 2), 3, dev)
        s64 = statistics.mean(r64["times"]) / 1e3
        st64 = r64["stats"]
        ms64 = st64["gs"][1]
        by64, fl64 = (gs_algorithmic_support(args.nu, tcnt, 8) if tcnt is not None
                      else gs_algorithmic(args.nu, m_vec, 8, ncols))
        ach64 = fl64 * max(3, args.steps // 2) / (ms64 / 1e3) / 1e12
        pk64 = 152 * 2 * 2 * 2.07e9 / 1e12
        line["fp64"] = {"value": round(world * ncols / s64, 2), "ms_per_step": round(s64 * 1e3, 3),
                        "kernel_ms_per_step": {k: round(v[1] / max(3, args.steps // 2), 3)
                                               for k, v in st64.items() if v[0]},
                        "gs_roofline": {"bound": "alu", "achieved": round(ach64, 3), "peak": round(pk64, 3),
                                         "unit": "TFLOP/s", "frac": round(ach64 / pk64, 4)},
                        "result": {"E_band_eV": r64["E"], "mu_eV": r64["mu"], "N": r64["N"]}}
        checks["fp64"] = gpu_outputs(m, r64["ctx"], cols, args.nu, 0)
        m.marnoldi_destroy(r64["ctx"])

    if not args.no_extra and not args.region and args.nu == 30:
        # the metric's second subspace dimension, and regional (order-N) mode,
        # on the same structure and precision
        import copy
        # nu = 100 in FP64 on every 4th column (a full FP64 nu = 100 step takes ~15 s)
        sub = cols[::4]
        for label, nu_x, reg_x, pr, cl in (("nu100", 100, 0, prec, cols),
                                           ("regional_256", 30, 256, prec, cols),
                                           ("nu100_fp64_quarter", 100, 0, 0, sub)):
            a2 = copy.copy(args)
            a2.nu, a2.region = nu_x, reg_x
            rx = time_gpu(m, t, cl, a2, pr, 3, 3, dev)
            sx = statistics.mean(rx["times"]) / 1e3
            line[label] = {"value": round(world * len(cl) / sx, 2), "unit": UNIT, "nu": nu_x,
                           "precision": "fp64" if pr == 0 else "mixed", "columns": len(cl),
                           "mode": mode_name(a2), "ms_per_step": round(sx * 1e3, 3),
                           "kernel_ms_per_step": {k: round(v[1] / 3, 3) for k, v in rx["stats"].items() if v[0]},
                           "result": {"E_band_eV": rx["E"], "mu_eV": rx["mu"], "N": rx["N"]}}
            if reg_x == 0:
                checks[label] = gpu_outputs(m, rx["ctx"], cl, nu_x, pr)
                if "eigsub" in rx["stats"]:
                    line[label]["eig_roofline"] = eig_roofline(t, cl, nu_x, rx["stats"]["eigsub"], 3)
            if label == "nu100" and pr == 1 and rx["stats"].get("gs", (0, 0.0))[1] > 0:
                # the Gram-Schmidt kernel's HBM fraction at nu = 100 (support bytes)
                tc100 = support_counts(t, cl, nu_x, column_m_pad(t.M))
                by100, _ = gs_algorithmic_support(nu_x, tc100, 4)
                gs_n, gs_ms = rx["stats"]["gs"]
                ach100 = by100 * 3 / (gs_ms / 1e3) / 1e9
                pk = peaks.get("hbm_gbs", 6800.0)
                r100 = (GS_DRAM_PER_ALGORITHMIC.get(("mixed", rx.get("gs_shape")))
                        if capture_current(rx.get("gs_shape")) else None)
                line[label]["roofline"] = {
                    "kernel": "gs", "bound": "hbm", "achieved": round(ach100, 3), "peak": round(pk, 3),
                    "unit": "GB/s", "frac": round(ach100 / pk, 4),
                    "traffic": round(r100 * by100 * 3 / gs_n) if r100 else None,
                    "traffic_note": (f"DRAM/algorithmic {r100} of the nu = 30 capture of the same kernel x "
                                     "algorithmic bytes per launch") if r100 else None,
                    "gs_shape": list(rx.get("gs_shape") or []), "launches": gs_n,
                    "avg_launch_ms": round(gs_ms / gs_n, 4)}
            m.marnoldi_destroy(rx["ctx"])

    if args.large and world == 1:
        line["large"] = large_structure(m, args.large, 256, 65536)

    if args.order_n and world == 1:
        sizes = [int(x) for x in args.order_n.split(",")]
        line["order_n"] = order_n(m, t, sizes, 256, prec)

    if not args.no_serving and world == 1:
        line["serving"] = serving(m, t, args.serve_requests, args.serve_workers,
                                  int(args.serve_budget_gb * 2**30), prec)

    if not args.no_e2e:
        e2e_s, h2d, d2h = time_e2e(m, t, cols, args, prec, max(3, args.steps // 2), 1)
        line["e2e"] = {"value": round(world * ncols / e2e_s, 2), "unit": UNIT,
                       "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                       "ms_per_step": round(e2e_s * 1e3, 3)}

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = oracle_sample(t, args, args.cpu_seconds, mu=mu_gpu)
        line["cpu_baseline"] = {"value": round(cb["value"], 3), "unit": UNIT, "cores": cb["cores"],
                                "kind": "oracle",
                                "sample": f"{cb['n']} seeded columns of the same workload (Krylov build, "
                                          f"eigensolve, weights, density columns at the GPU's mu), "
                                          f"{cb['seconds']:.1f} s",
                                "gpu_vs_oracle": oracle_checks(t, checks)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def order_n(m, t4096, sizes, n_reg: int, prec: int, nu: int = 30):
    """The method's order-N claim on one GPU, and the error of the regions.

    Time: regional solves (n_reg-atom regions, all real orbitals, mu by
    bisection, density on the device) of amorphous carbon of each size, one
    timed solve each after one untimed solve of the smallest.  Error: on the
    4,096-atom structure in FP64, regional solves at N_reg = 64 .. 1,024
    against the global-mode solve at the same nu (8, 16 and nu): band energy
    per atom, largest density-matrix entry difference and the Fermi level.
    """
    import torch
    from tbsynth import amorphous_system

    def solve(t, p, reg, nu_x):
        ctx = m.setup_system(t, p)
        rho = torch.empty(t.nnzb * 16, dtype=torch.float64, device="cuda")
        rhoE = torch.empty_like(rho)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        m.marnoldi_solve(ctx, None, nu_x, reg, float(t.n_electrons), KT)
        m.marnoldi_density_device(ctx, rho, rhoE)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        E, mu, N = m.marnoldi_energy(ctx)
        m.marnoldi_destroy(ctx)
        return dt, E, mu, rho

    out = {"time": [], "error": []}
    first = True
    for n in sizes:
        t = t4096 if n == t4096.n_block_rows else amorphous_system(n, seed=0)
        if first:
            solve(t, prec, n_reg, nu)
            first = False
        dt, E, mu, _ = solve(t, prec, n_reg, nu)
        ncols = int(t.real_columns().size)
        out["time"].append({"atoms": n, "columns": ncols, "seconds": round(dt, 3),
                            "columns_per_s": round(ncols / dt, 1), "E_band_per_atom_eV": E / n})
        del t
    for nu_e in (8, 16, nu):
        _, E0, mu0, rho0 = solve(t4096, 0, 0, nu_e)
        r0 = rho0.cpu().numpy()
        for reg in (64, 128, 256, 512, 1024):
            _, E, mu, rho = solve(t4096, 0, reg, nu_e)
            out["error"].append({"nu": nu_e, "region_atoms": reg,
                                 "dE_band_per_atom_eV": abs(E - E0) / t4096.n_block_rows,
                                 "max_abs_drho": float(np.abs(rho.cpu().numpy() - r0).max()),
                                 "dmu_eV": abs(mu - mu0)})
    out["setup"] = (f"amorphous carbon, seed 0, {n_reg}-atom regions, nu={nu}, "
                    f"{'mixed' if prec else 'fp64'} for the times; errors in FP64 against global mode "
                    f"at the same nu on {t4096.n_block_rows} atoms")
    return out


def large_structure(m, n_atoms: int, n_reg: int, batch: int):
    """The paper-scale configuration on one GPU: amorphous carbon of n_atoms
    atoms (1,048,576 by default) in regional mode (n_reg-atom regions).  Times
    (a) the whole structure at nu = 30 in mixed precision (every real orbital,
    mu by bisection, density on the device) and (b) one batch of `batch`
    columns (the first ones) at nu = 100 in mixed precision and in FP64 (mu
    fixed at the nu = 30 solve's level, so that only the batch is timed)."""
    import torch
    from tbsynth import amorphous_system
    t0 = time.perf_counter()
    t = amorphous_system(n_atoms, seed=0)
    gen_s = time.perf_counter() - t0
    out = {"atoms": n_atoms, "M": t.M, "nnzb": t.nnzb, "region_atoms": n_reg,
           "generation_s": round(gen_s, 1)}
    for prec in (1, 0):
        t0 = time.perf_counter()
        ctx = m.setup_system(t, prec)
        torch.cuda.synchronize()
        out[f"setup_s_{'mixed' if prec else 'fp64'}"] = round(time.perf_counter() - t0, 1)
        if prec == 1:
            rho = torch.empty(t.nnzb * 16, dtype=torch.float64, device="cuda")
            rhoE = torch.empty_like(rho)
            t0 = time.perf_counter()
            m.marnoldi_solve(ctx, None, 30, n_reg, float(t.n_electrons), KT)
            m.marnoldi_density_device(ctx, rho, rhoE)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            E, mu, N = m.marnoldi_energy(ctx)
            out["nu30_all_columns"] = {"columns": int(t.M), "seconds": round(dt, 2),
                                       "columns_per_s": round(t.M / dt, 1),
                                       "E_band_per_atom_eV": E / n_atoms, "mu_eV": mu}
            mu30 = mu
            del rho, rhoE
        cols = np.arange(batch, dtype=np.int64)
        m.marnoldi_solve(ctx, cols[:256], 100, n_reg, 0.0, KT, mu_fixed=mu30)   # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        m.marnoldi_solve(ctx, cols, 100, n_reg, 0.0, KT, mu_fixed=mu30)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        out[f"nu100_batch_{'mixed' if prec else 'fp64'}"] = {"columns": batch, "seconds": round(dt, 2),
                                                              "columns_per_s": round(batch / dt, 1)}
        m.marnoldi_destroy(ctx)
        torch.cuda.empty_cache()
    out["note"] = ("regional mode (the order-N form); the nu = 100 lines time one batch of the first "
                   f"{batch} columns at the nu = 30 Fermi level")
    return out


def mixed_vs_fp64(m, nu: int):
    """Every column of the benchmark structure (amorphous carbon, 4,096 atoms, global mode) at `nu`
    in mixed precision against the FP64 path, the mixed density evaluated at the FP64 Fermi level:
    energy and count differences and the distribution of |d rho| over all entries, with the
    worst entry's column and its levels nearest mu."""
    from tbsynth import config_c2
    t = config_c2(seed=0)
    ci = np.asarray(t.col_idx)
    blk_row = np.repeat(np.arange(t.n_block_rows), np.diff(np.asarray(t.row_ptr)))
    c = m.setup_system(t, 0)
    m.marnoldi_solve(c, None, nu, 0, t.n_electrons, KT)
    E64, mu64, N64 = m.marnoldi_energy(c)
    r64, rE64 = m.marnoldi_density(c)
    nue, eps64, _ = m.marnoldi_column_stats(c)
    m.marnoldi_destroy(c)
    c = m.setup_system(t, 1)
    m.marnoldi_solve(c, None, nu, 0, t.n_electrons, KT)
    E32, mu32, N32 = m.marnoldi_energy(c)
    m.marnoldi_fermi_at(c, mu64, KT)
    r32, rE32 = m.marnoldi_density(c)
    nue32, eps32, _ = m.marnoldi_column_stats(c)
    shape = m.marnoldi_gs_shape(c)
    m.marnoldi_destroy(c)
    d, dE = np.abs(r32 - r64).ravel(), np.abs(rE32 - rE64).ravel()
    k = int(d.argmax())
    blk, (a, b) = k // 16, divmod(k % 16, 4)
    col = 4 * int(ci[blk]) + b            # rho e_j fills column j of the block row
    lv = eps64[col][:nue[col]]
    near = np.argsort(np.abs(lv - mu64))[:3]
    shift = (float(np.abs(np.sort(eps32[col][:nue32[col]]) - np.sort(lv)).max())
             if nue32[col] == nue[col] else None)
    return {"nu": nu, "atoms": int(t.n_block_rows), "columns": int(t.M), "gs_shape": list(shape),
            "dE_band_per_atom_eV": abs(E32 - E64) / t.n_block_rows, "dN": abs(N32 - N64),
            "dmu_eV": abs(mu32 - mu64), "rho_entries": int(d.size), "max_drho": float(d.max()),
            "max_drhoE_eV": float(dE.max()), "drho_gt_1e-5": int((d > 1e-5).sum()),
            "drhoE_gt_1e-4": int((dE > 1e-4).sum()),
            "drho_p99_9": float(np.quantile(d, 0.999)), "drho_p99_99": float(np.quantile(d, 0.9999)),
            "worst": {"row_atom": int(blk_row[blk]), "column": col, "rho_fp64": float(r64.ravel()[k]),
                      "rho_mixed": float(r32.ravel()[k]),
                      "levels_nearest_mu_eV": [float(lv[q] - mu64) for q in near],
                      "max_level_shift_eV": shift}}


def chain_breakdown(m, units: int, nus, n_reg: int = 256, prec: int = 1):
    """One fluorene-like chain of `units` units in regional mode: every real orbital solved (mu by
    bisection, kT = 0.1 eV) once per nu after a warm-up, with the per-kernel CUDA-event times."""
    import torch
    from tbsynth import polymer_system
    t = polymer_system(units, seed=3, check_spd=False)
    out = {"units": units, "atoms": int(t.n_block_rows), "columns": int(t.real_columns().size),
           "region_atoms": n_reg, "precision": "mixed" if prec else "fp64"}
    for nu in nus:
        ctx = m.setup_system(t, prec)
        m.marnoldi_solve(ctx, t.real_columns()[:512], nu, n_reg, 0.0, KT, mu_fixed=-2.0)   # warm-up
        m.marnoldi_set_profiling(ctx, True)
        m.marnoldi_kernel_stats(ctx, reset=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        m.marnoldi_solve(ctx, None, nu, n_reg, float(t.n_electrons), KT)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        st = m.marnoldi_kernel_stats(ctx)
        out[f"nu{nu}"] = {"seconds": round(dt, 3), "columns_per_s": round(t.real_columns().size / dt, 1),
                          "kernel_ms": {k: round(v[1], 1) for k, v in st.items() if v[1] > 0}}
        m.marnoldi_destroy(ctx)
    return out


def large_full(m, n_atoms: int, n_reg: int, batch: int, n_sample: int = 32, fp64_batch: int = 32768):
    """The paper-scale configuration in full: every one of the 4 n_atoms columns of amorphous
    carbon at nu = 100 in regional mode (n_reg-atom regions), streamed through the solve in
    batches of `batch` columns, mu by bisection over all of them, densities on the device;
    mixed precision and FP64.  Per-kernel times (CUDA events) give each kernel's share and
    the Gram-Schmidt HBM fraction (dense-region bytes: every stored vector over the whole
    region, an upper bound of the supports) and the eigensolver's FP64 rate; a seeded sample
    of columns is recomputed by the regional oracle at the GPU's mu."""
    import torch
    import oracle
    from tbsynth import amorphous_system
    t0 = time.perf_counter()
    t = amorphous_system(n_atoms, seed=0)
    out = {"atoms": n_atoms, "M": t.M, "nnzb": t.nnzb, "region_atoms": n_reg, "nu": 100,
           "batch_columns": batch, "generation_s": round(time.perf_counter() - t0, 1)}
    peaks = read_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    nu, m_reg = 100, 4 * n_reg
    rng = np.random.default_rng(17)
    sample = np.sort(rng.choice(t.M, size=n_sample, replace=False))
    for prec in (1, 0):
        name = "mixed" if prec else "fp64"
        ctx = m.setup_system(t, prec)
        # FP64 vectors double the batch workspace; beside the per-column state of all
        # 4,194,304 columns (their pattern rows P_j: about 160 GB) half the batch fits
        b_prec = batch if prec else fp64_batch
        m.marnoldi_set_batch(ctx, b_prec)
        m.marnoldi_solve(ctx, np.arange(4096, dtype=np.int64), nu, n_reg, 0.0, KT, mu_fixed=4.0)  # warm-up
        m.marnoldi_set_profiling(ctx, True)
        m.marnoldi_kernel_stats(ctx, reset=True)
        rho = torch.empty(t.nnzb * 16, dtype=torch.float64, device="cuda")
        rhoE = torch.empty_like(rho)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        m.marnoldi_solve(ctx, None, nu, n_reg, float(t.n_electrons), KT)
        m.marnoldi_density_device(ctx, rho, rhoE)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        E, mu, N = m.marnoldi_energy(ctx)
        st = m.marnoldi_kernel_stats(ctx)
        nue, eps, w = m.marnoldi_column_stats(ctx)
        vb = 4 if prec else 8
        # Gram-Schmidt bytes over dense regions: per column and step n, u (and lo), w_n,
        # w_i and S w_i (i <= n), w_i again, the new w
        per_col = sum(((2 if prec else 1) + 1 + 2 * (n + 1) + (n + 1 if n < nu - 1 else 0) +
                       (1 if n < nu - 1 else 0)) * m_reg * vb for n in range(nu))
        gs_ms = st["gs"][1]
        eig_ms = st["eigsub"][1]
        eig_flop = (4.0 / 3.0 * nu ** 3 + 6.0 * nu * nu * (4 * 12 + 2)) * t.M
        rho_h = rho.cpu().numpy().reshape(-1, 4, 4)
        rhoE_h = rhoE.cpu().numpy().reshape(-1, 4, 4)
        ref = oracle.solve(t, nu=nu, kT=KT, mu_fixed=mu, cols=sample, region_atoms=n_reg)
        mask = ~np.isnan(ref.rho)
        drho = float(np.abs(rho_h[mask] - ref.rho[mask]).max())
        drhoE = float(np.abs(rhoE_h[mask] - ref.rhoE[mask]).max())
        out[name] = {"seconds": round(dt, 2), "columns_per_s": round(t.M / dt, 1), "batch_columns": b_prec,
                     "E_band_per_atom_eV": E / n_atoms, "mu_eV": mu, "N": N,
                     "kernel_ms": {k: round(v[1], 1) for k, v in st.items() if v[1] > 0},
                     "gs_hbm_frac_dense_bytes": round(per_col * t.M / (gs_ms / 1e3) / 1e9 / hbm, 3),
                     "eig_fp64_tflops": round(eig_flop / (eig_ms / 1e3) / 1e12, 3),
                     "oracle_sample": {"columns": int(sample.size), "max_abs_drho": drho,
                                       "max_abs_drhoE_eV": drhoE}}
        print(json.dumps({"partial": name, name: out[name]}), flush=True)
        m.marnoldi_destroy(ctx)
        del rho, rhoE
        torch.cuda.empty_cache()
    out["note"] = ("gs_hbm_frac_dense_bytes counts every stored vector over the whole region (an upper "
                   "bound of the bytes over the vectors' supports); eig_fp64_tflops counts the "
                   "tridiagonalisation (4/3 nu^3) and the rotations applied to 50 rows (6 nu^2 x 50)")
    return out


SERVE_SIZES = (256, 512, 1024, 2048, 4096)
SERVE_SIZE_P = (0.3, 0.3, 0.2, 0.15, 0.05)


def serving(m, t4096, requests: int, workers: int, budget: int, prec: int):
    """Whole calculations through the request server on a seeded trace.

    Structures of 256 to 4,096 atoms (amorphous carbon, the same recipe as
    the headline), nu = 30, or nu = 100 for a quarter of the requests of
    <= 1,024 atoms; the density matrices go back to the host.  Three passes:
    the whole trace submitted at once with one worker (requests one after
    another) and with `workers` (concurrent), then Poisson arrivals at 60 % of
    the concurrent pass's request rate, whose submit-to-result latencies give
    p50 / p99.
    """
    import torch
    from tbsynth import amorphous_system

    rng = np.random.default_rng(2024)
    pool = {n: (t4096 if n == t4096.n_block_rows else amorphous_system(n, seed=100 + n))
            for n in SERVE_SIZES}
    trace = []
    for _ in range(requests):
        n = int(rng.choice(SERVE_SIZES, p=SERVE_SIZE_P))
        nu = 100 if n <= 1024 and rng.random() < 0.25 else 30
        trace.append((n, nu))
    ncols_total = sum(pool[n].real_columns().size for n, _ in trace)
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    # every (size, nu) once before the timed passes: kernel loading and, with
    # the autotuner on, the one-time shape tuning of each key
    shapes = {}
    with m.Server(workers=1, hbm_budget_bytes=budget) as srv:
        for n, nu in sorted(set(trace)):
            srv.wait(srv.submit_system(pool[n], prec, nu, 0, pool[n].n_electrons, 0.1))
    for n, nu in sorted(set(trace)):
        ctx = m.setup_system(pool[n], prec)
        m.marnoldi_solve(ctx, pool[n].real_columns()[:1], nu, 0, 0.0, 0.1, mu_fixed=0.0)
        shapes[f"{n}_atoms_nu{nu}"] = "x".join(map(str, m.marnoldi_gs_shape(ctx)))
        m.marnoldi_destroy(ctx)

    def run(nworkers, gaps=None, group=16, reqs=None):
        reqs = [(pool[n], nu) for n, nu in trace] if reqs is None else reqs
        with m.Server(workers=nworkers, hbm_budget_bytes=budget) as srv:
            srv.set_group_limit(group)
            # warm the server's memory pool once
            srv.wait(srv.submit_system(pool[512], prec, 30, 0, pool[512].n_electrons, 0.1))
            ids, t0 = [], time.perf_counter()
            for k, (sysm, nu) in enumerate(reqs):
                if gaps is not None:
                    due = t0 + gaps[k]
                    while time.perf_counter() < due:
                        time.sleep(min(0.002, max(0.0, due - time.perf_counter())))
                ids.append(srv.submit_system(sysm, prec, nu, 0, sysm.n_electrons, 0.1))
            res = [srv.wait(i) for i in ids]
            st = srv.stats()
        first = min(r["t_submit"] for r in res)
        wall = max(r["t_end"] for r in res) - first
        lat = np.array([r["latency_s"] for r in res]) * 1e3
        return dict(wall=wall, lat=lat, stats=st)

    seq = run(1, group=1)
    burst = run(workers)
    rate = 0.6 * requests / burst["wall"]
    gaps = np.cumsum(rng.exponential(1.0 / rate, size=requests))
    gaps -= gaps[0]
    pois = run(workers, gaps)
    lat = pois["lat"]
    # many small molecules: 64-atom diamond cells (8 seeds), all at once, with
    # and without grouping queued requests into shared launches
    from tbsynth import config_c1
    cells = [config_c1(seed=s) for s in range(8)]
    small = [(cells[k % 8], 30) for k in range(128)]
    run(workers, group=16, reqs=small[:16])   # warm-up of this class
    solo = run(workers, group=1, reqs=small)
    grouped = run(workers, group=16, reqs=small)
    # the same two passes with each request's Krylov build as one CUDA graph
    os.environ["MARNOLDI_KRYLOV_GRAPH"] = "1"
    try:
        run(workers, group=16, reqs=small[:16])
        solo_g = run(workers, group=1, reqs=small)
        grouped_g = run(workers, group=16, reqs=small)
    finally:
        os.environ.pop("MARNOLDI_KRYLOV_GRAPH", None)
    ncols_small = sum(c.real_columns().size for c, _ in small)
    # uneven polymer chains: fluorene-like units (69 atoms each), lengths
    # log-uniform in 4..59 units (the global-mode limit of 4,096 atoms), nu 30
    # or 100, all submitted at once
    from tbsynth import polymer_system
    prng = np.random.default_rng(7)
    chains = []
    for q in range(24):
        units = int(round(np.exp(prng.uniform(np.log(4), np.log(59)))))
        chains.append((polymer_system(units, seed=q), 100 if prng.random() < 0.25 else 30))
    run(workers, group=16, reqs=chains[:2])   # warm-up
    poly = run(workers, group=16, reqs=chains)
    ncols_poly = sum(c.real_columns().size for c, _ in chains)
    out_poly = {"requests": len(chains), "units": [int(c.n_block_rows // 69) for c, _ in chains],
                "atoms_total": int(sum(c.n_block_rows for c, _ in chains)), "columns": int(ncols_poly),
                "columns_per_s": round(ncols_poly / poly["wall"], 1),
                "p50_ms": round(float(np.percentile(poly["lat"], 50)), 2),
                "p99_ms": round(float(np.percentile(poly["lat"], 99)), 2),
                "groups": poly["stats"]["groups"], "largest_group": poly["stats"]["largest_group"]}
    out_small = {"requests": len(small), "atoms": 64, "nu": 30, "columns": int(ncols_small),
                 "one_by_one": {"columns_per_s": round(ncols_small / solo["wall"], 1),
                                "p50_ms": round(float(np.percentile(solo["lat"], 50)), 2)},
                 "grouped": {"columns_per_s": round(ncols_small / grouped["wall"], 1),
                             "p50_ms": round(float(np.percentile(grouped["lat"], 50)), 2),
                             "groups": grouped["stats"]["groups"],
                             "largest_group": grouped["stats"]["largest_group"]},
                 "krylov_graph": {
                     "one_by_one": {"columns_per_s": round(ncols_small / solo_g["wall"], 1),
                                    "p50_ms": round(float(np.percentile(solo_g["lat"], 50)), 2)},
                     "grouped": {"columns_per_s": round(ncols_small / grouped_g["wall"], 1),
                                 "p50_ms": round(float(np.percentile(grouped_g["lat"], 50)), 2)}}}
    return {
        "small_molecules": out_small,
        "polymer_chains": out_poly,
        "trace": f"{requests} requests, atoms {list(SERVE_SIZES)} with p {list(SERVE_SIZE_P)}, "
                 f"nu 30 (nu 100 for 1/4 of those <= 1024 atoms), {'mixed' if prec else 'fp64'}, "
                 f"all real orbitals, density matrices returned to the host",
        "columns": int(ncols_total), "workers": workers, "hbm_budget_gb": round(budget / 2**30, 1),
        "gs_shapes": shapes,
        "sequential": {"wall_s": round(seq["wall"], 3), "columns_per_s": round(ncols_total / seq["wall"], 1)},
        "concurrent": {"wall_s": round(burst["wall"], 3),
                       "columns_per_s": round(ncols_total / burst["wall"], 1),
                       "peak_running": burst["stats"]["peak_running"],
                       "groups": burst["stats"]["groups"], "largest_group": burst["stats"]["largest_group"],
                       "peak_footprint_gb": round(burst["stats"]["peak_bytes"] / 2**30, 2)},
        "poisson": {"offered_requests_per_s": round(rate, 2), "groups": pois["stats"]["groups"],
                    "p50_ms": round(float(np.percentile(lat, 50)), 2),
                    "p99_ms": round(float(np.percentile(lat, 99)), 2),
                    "mean_ms": round(float(lat.mean()), 2), "max_ms": round(float(lat.max()), 2),
                    "columns_per_s": round(ncols_total / pois["wall"], 1)},
    }


def _served(results):
    """Wall time from the first submission to the last result (the server's clock) and the
    latencies (ms) of a set of served results."""
    first = min(r["t_submit"] for r in results)
    wall = max(r["t_end"] for r in results) - first
    lat = np.array([r["latency_s"] for r in results]) * 1e3
    return wall, lat


def serve_c4(m, workers: int, budget: int, prec: int = 1, n_chains: int = 256, seed: int = 4):
    """Uneven batching on the polymer workload as configured: n_chains fluorene-like chains
    (69 atoms per unit), unit counts log-uniform in 4..400 from `seed`, nu drawn from
    {30, 100, 300}, every real orbital, mu by bisection (kT = 0.1 eV), densities back to the
    host; chains of up to 59 units (4,073 atoms) in global mode, longer ones in regional mode
    (256-atom regions).  All submitted at once to the request server."""
    from tbsynth import polymer_system
    rng = np.random.default_rng(seed)
    units = np.rint(np.exp(rng.uniform(np.log(4), np.log(400), size=n_chains))).astype(int)
    nus = rng.choice([30, 100, 300], size=n_chains)
    t0 = time.perf_counter()
    chains = [polymer_system(int(u), seed=1000 + q, check_spd=False) for q, u in enumerate(units)]
    gen_s = time.perf_counter() - t0
    regions = [0 if u <= 59 else 256 for u in units]
    cols = [c.real_columns().size for c in chains]
    with m.Server(workers=workers, hbm_budget_bytes=budget) as srv:
        srv.set_group_limit(16)
        srv.wait(srv.submit_system(chains[0], prec, 30, regions[0], chains[0].n_electrons, 0.1))   # warm-up
        ids = [srv.submit_system(c, prec, int(nu), reg, c.n_electrons, 0.1)
               for c, nu, reg in zip(chains, nus, regions)]
        res = [srv.wait(i) for i in ids]
        st = srv.stats()
    wall, lat = _served(res)
    by_nu = {}
    for nu in (30, 100, 300):
        sel = [q for q in range(n_chains) if nus[q] == nu]
        by_nu[f"nu{nu}"] = {"chains": len(sel), "columns": int(sum(cols[q] for q in sel)),
                            "p50_ms": round(float(np.percentile(lat[sel], 50)), 1) if sel else None}
    return {"config": f"{n_chains} fluorene-like chains, units log-uniform 4..400 (seed {seed}), nu from "
                      "{30, 100, 300}, global mode up to 59 units, 256-atom regions above, "
                      f"{'mixed' if prec else 'fp64'}, kT 0.1 eV, densities to the host",
            "atoms_total": int(sum(c.n_block_rows for c in chains)), "columns": int(sum(cols)),
            "regional_chains": int(sum(1 for r in regions if r)), "generation_s": round(gen_s, 1),
            "wall_s": round(wall, 2), "columns_per_s": round(sum(cols) / wall, 1),
            "p50_ms": round(float(np.percentile(lat, 50)), 1), "p99_ms": round(float(np.percentile(lat, 99)), 1),
            "groups": st["groups"], "largest_group": st["largest_group"], "by_nu": by_nu}


def serve_c5(m, workers: int, budget: int, prec: int = 1, window_s: float = 30.0,
             rates=(1.0, 0.5, 0.25, 0.125), seed: int = 5, pool_sizes: int = 6, deadline_s: float = 600.0):
    """Serving as configured: Poisson arrivals of carbon or polymer structures (50/50) of
    1,000-200,000 atoms (log-uniform; drawn from a pool of `pool_sizes` log-spaced sizes per
    kind), each with its own nu in {30, 100} and kT in {0.05, 0.1, 0.2} eV; global mode up to
    4,096 atoms, 256-atom regions above.  For each arrival rate lambda (requests/s), `window_s`
    seconds of arrivals; reported: offered and served load (requests/s and columns/s) and the
    submit-to-result latency p50 / p99."""
    from tbsynth import amorphous_system, polymer_system
    rng = np.random.default_rng(seed)
    sizes = np.exp(np.linspace(np.log(1000), np.log(200000), pool_sizes))
    t0 = time.perf_counter()
    pool = {("carbon", q): amorphous_system(int(round(n)), seed=500 + q, check_spd=False)
            for q, n in enumerate(sizes)}
    pool.update({("polymer", q): polymer_system(max(15, int(round(n / 69))), seed=600 + q, check_spd=False)
                 for q, n in enumerate(sizes)})
    gen_s = time.perf_counter() - t0
    t_begin = time.perf_counter()
    print(json.dumps({"progress": "pool generated", "seconds": round(gen_s, 1)}), flush=True)
    out = {"config": f"Poisson arrivals, carbon or polymer 50/50, 1,000-200,000 atoms log-uniform "
                     f"(pool of {pool_sizes} sizes per kind), nu from {{30, 100}}, kT from {{0.05, 0.1, 0.2}} eV, "
                     f"global mode up to 4,096 atoms, 256-atom regions above, {'mixed' if prec else 'fp64'}, "
                     f"densities to the host, {window_s:g} s of arrivals per rate",
           "pool_atoms": {f"{k}_{q}": int(v.n_block_rows) for (k, q), v in pool.items()},
           "generation_s": round(gen_s, 1), "rates": []}
    with m.Server(workers=workers, hbm_budget_bytes=budget) as srv:
        srv.set_group_limit(16)
        # one solve of each class first (kernel loading, shape tuning): global and regional
        # mode at both nu, on the smallest structures of each mode
        small_global = min((v for v in pool.values() if v.n_block_rows <= 4096), key=lambda v: v.n_block_rows)
        small_reg = min((v for v in pool.values() if v.n_block_rows > 4096), key=lambda v: v.n_block_rows)
        for sysm, reg in ((small_global, 0), (small_reg, 256)):
            for nu in (30, 100):
                srv.wait(srv.submit_system(sysm, prec, nu, reg, sysm.n_electrons, 0.1))
        print(json.dumps({"progress": "warmed up", "seconds": round(time.perf_counter() - t_begin, 1)}),
              flush=True)
        for lam in rates:
            if time.perf_counter() - t_begin > deadline_s:
                break
            n_req = max(1, rng.poisson(lam * window_s))
            gaps = np.sort(rng.uniform(0.0, window_s, size=n_req))
            reqs = []
            for _ in range(n_req):
                kind = "carbon" if rng.random() < 0.5 else "polymer"
                n = np.exp(rng.uniform(np.log(1000), np.log(200000)))
                q = int(np.argmin(np.abs(np.log(sizes) - np.log(n))))
                reqs.append((pool[(kind, q)], int(rng.choice([30, 100])), float(rng.choice([0.05, 0.1, 0.2]))))
            ids, t_start = [], time.perf_counter()
            for g, (sysm, nu, kT) in zip(gaps, reqs):
                due = t_start + g
                while time.perf_counter() < due:
                    time.sleep(min(0.002, max(0.0, due - time.perf_counter())))
                reg = 0 if sysm.n_block_rows <= 4096 else 256
                ids.append(srv.submit_system(sysm, prec, nu, reg, sysm.n_electrons, kT))
            res = [srv.wait(i) for i in ids]
            wall, lat = _served(res)   # the server's clock: first submission to last result
            cols = sum(int(s.real_columns().size) for s, _, _ in reqs)
            out["rates"].append({
                "offered_requests_per_s": lam, "requests": n_req,
                "offered_columns_per_s": round(cols / window_s, 1),
                "served_requests_per_s": round(n_req / wall, 3), "served_columns_per_s": round(cols / wall, 1),
                "drained_s": round(wall, 1), "p50_ms": round(float(np.percentile(lat, 50)), 1),
                "p99_ms": round(float(np.percentile(lat, 99)), 1),
                "atoms": [int(sm.n_block_rows) for sm, _, _ in reqs], "nu": [nu for _, nu, _ in reqs],
                "latency_s": [round(float(x) / 1e3, 2) for x in lat]})
            print(json.dumps({"progress": "rate", **out["rates"][-1]}), flush=True)
        out["stats"] = {k: srv.stats()[k] for k in ("groups", "largest_group", "peak_running")}
    # sustainable: every request of the window served within 25 % past the window
    sustain = [r for r in out["rates"] if r["drained_s"] <= 1.25 * window_s]
    out["sustainable_requests_per_s"] = max((r["offered_requests_per_s"] for r in sustain), default=None)
    return out


def main_reference(args, world, rank):
    """The CPU oracle as the reference arm: each step a bounded sample of the workload."""
    if rank != 0:
        return
    import oracle
    t, cols = workload(args)
    oracle.build()
    nth = oracle.threads()
    rng = np.random.default_rng(99)
    # size a step to ~args.cpu_seconds / steps of CPU work
    probe = rng.choice(cols, size=max(nth, 16), replace=False)
    t0 = time.perf_counter()
    oracle.columns(t, probe, args.nu)
    per_col = (time.perf_counter() - t0) / probe.size
    per_step = int(max(nth, min(len(cols), (args.cpu_seconds / max(1, args.steps)) / per_col)))
    for _ in range(args.warmup):
        oracle.columns(t, rng.choice(cols, size=nth, replace=False), args.nu)
    ts = []
    for _ in range(args.steps):
        sample = rng.choice(cols, size=per_step, replace=False)
        t0 = time.perf_counter()
        c = oracle.columns(t, sample, args.nu)
        oracle.density_rows(c, REFERENCE_MU, KT)
        ts.append(time.perf_counter() - t0)
    v = per_step / statistics.mean(ts)
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 3), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(statistics.mean(ts) * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": workload_name(args, t, len(cols)), "nu": args.nu, "mode": mode_name(args)},
            "cpu_baseline": {"value": round(v, 3), "unit": UNIT, "cores": nth, "kind": "oracle",
                             "sample": f"{per_step} seeded columns per step (Krylov build, eigensolve, "
                                       f"weights, density columns at a fixed mu)"},
            "e2e": {"value": round(v, 3), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
