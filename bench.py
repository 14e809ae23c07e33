"""Benchmark: low-rank assembly + block-AMEn KKT solve on one GB300.

One step = the whole hot path on one synthetic workload: sampling of the
geometry weights, TT-SVD, batched univariate assembly (low-rank M, K and
load), then the KKT solve by block AMEn with FP64 iterative refinement to
a relative residual of 1e-6.  Default workload: the extruded quarter annulus,
degree 3, 64 elements per direction (65^3 interior unknowns per field),
TT tolerance 1e-6, beta = 1e-4, desired state exp(-|x - c|^2 / 0.1).

Usage:  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun every rank solves its own replica of the workload (the path
does not exchange data between GPUs); rank 0 prints one JSON line.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "KKT solve s to 1e-6 rel. residual; Kron/TT apply % of roofline, mixed vs FP64"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
# ALU peaks derived from unit counts and the maximum SM clock: 152 SMs, 2 FP64
# FMA and 128 FP32 FMA per SM per clock (2 flop per FMA); at 2070 MHz that is
# 1.26 and 80.6 TFLOP/s.  The library's own FMA micro-kernel
# (iga_measure_fma) is run in the same job and reported beside them.
SMS = 152
FP64_FMA_PER_SM_CLK = 2
FP32_FMA_PER_SM_CLK = 128


def alu_peak_tflops(arith, pk):
    mhz = float(pk.get("sm_max_mhz") or 2070.0)
    per = FP64_FMA_PER_SM_CLK if arith == "fp64" else FP32_FMA_PER_SM_CLK
    return SMS * per * 2.0 * mhz * 1e6 / 1e12


FP64_FMA_TFLOPS = alu_peak_tflops("fp64", {})
FP32_FMA_TFLOPS = alu_peak_tflops("fp32", {})
# DRAM bytes (read + write) per launch from one ncu capture of the kernel, as
# summarised under profiles/; an entry is dropped whenever its kernel changes
NCU_TRAFFIC = {}
# kernels that can dominate a step, with the arithmetic they run in
CANDIDATES = {
    "jacobi_eig_kernel": "fp64", "sample_weights_kernel": "fp64",
    "kkt_block_solve_kernel": "fp32", "kkt_block_factor_kernel": "fp32",
    "kkt_qd_solve_kernel": "fp32", "kkt_qd_factor_kernel": "fp32",
    "kron_rank1_kernel": "fp64",
    "qrcp_cluster_kernel": "fp64", "householder_qr_cluster_kernel": "fp64",
    "rank1_residual_kernel": "fp64", "gemm_tile_kernel": "fp64",
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--config", type=int, default=2)
    ap.add_argument("--precision", default="fp64", choices=["mixed", "fp64"])
    ap.add_argument("--weights", default="interp", choices=["interp", "sampled"],
                    help="weights interpolated in degree 2p+1 (the paper's route, Sec. 3) or "
                         "sampled on the Gauss grid")
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--roofline-kernel", default="auto",
                    help="kernel name for the roofline entry, or auto (largest device time)")
    ap.add_argument("--only", default=None,
                    choices=["ttm", "c5solve", "step", "parabolic", "kron32"],
                    help="ttm: only the tensor-core TT apply measurement (a profiling case); "
                         "c5solve: only the random-volume solve without full-size applies; "
                         "step: only the timed steps of the workload; "
                         "parabolic: only the parabolic solve on the workload's operators")
    ap.add_argument("--nt", type=int, default=10, help="time steps of the parabolic solve")
    ap.add_argument("--c5-tol", type=float, default=1e-4)
    ap.add_argument("--c5-trunc", type=float, default=1e-6)
    ap.add_argument("--c5-sweeps", type=int, default=4)
    ap.add_argument("--c5-state-weight", type=float, default=1000.0)
    ap.add_argument("--ttm-elements", type=int, default=512,
                    help="elements per direction of the --only ttm grid")
    ap.add_argument("--ttm-kinds", default="tf32,bf16", help="operand types of --only ttm")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def aggregate_ms(ms, dist):
    """Whole-job step time: the maximum over ranks (every rank solves its own replica)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return ms
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def peaks():
    try:
        with open(PEAKS_FILE) as f:
            p = json.load(f)
        return p, "measured"
    except Exception:
        return FALLBACK_PEAKS, "fallback"


def alu_roofline(kernel, p, peak_tflops, peak_kind):
    """Roofline object of one kernel against an arithmetic peak, from the
    library's live profile of one step (launches, ms, algorithmic bytes and
    flops summed over the launches); None when the kernel did not run."""
    try:
        if not p or p["launches"] <= 0 or p["ms"] <= 0:
            return None
        avg = p["ms"] / p["launches"]
        fl = p["flops"] / p["launches"]
        ach = fl / (avg * 1e-3) / 1e12
        return {"kernel": kernel, "bound": "alu", "achieved": ach, "peak": peak_tflops,
                "unit": "TFLOP/s", "frac": ach / peak_tflops, "peak_kind": peak_kind,
                "launches_per_step": p["launches"], "avg_us": avg * 1e3,
                "algorithmic_flops_per_launch": fl,
                "algorithmic_bytes_per_launch": p["bytes"] / p["launches"]}
    except (KeyError, TypeError, ZeroDivisionError):
        return None


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                 "-lms", "20"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        try:
            rows = [l.strip().split(",") for l in open(self.path) if l.strip()]
        except Exception:
            return out
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for k, nm in enumerate(names):
                    if r[5 + k].strip().lower() == "active":
                        reasons.add(nm)
            except Exception:
                pass
        if sm:
            out["sm_mhz"] = statistics.median(sm)
            out["sm_max_mhz"] = max(mx)
        out["reasons"] = sorted(reasons)
        out["samples"] = len(sm)
        try:
            os.unlink(self.path)
        except Exception:
            pass
        return out


# ------------------------------------------------------------------ CPU oracle leg

def _threads():
    cores = os.cpu_count() or 1
    try:
        import threadpoolctl
        info = threadpoolctl.threadpool_info()
        cores = max([i.get("num_threads", 1) for i in info] + [1])
    except Exception:
        pass
    return cores


class OracleLeg:
    """The oracle (oracle/) timed on the host cores on a bounded sample of the
    workload, and its solution for the per-field errors of the GPU result.

    Set-up (untimed, once): the oracle's full pipeline at full size -- the
    weights sampled on the whole Gauss grid, TT-SVD, univariate factors, the
    reduced-system CG solve to 1e-12 (oracle/solve.py).  One timed step:
      * sampling of the weights on a slab of 1/S of the Gauss planes along
        direction 3, scaled by S (the per-point work is identical);
      * TT-SVD of the eight sample tensors of that slab, scaled by S (the
        first unfolding dominates and its SVD cost is linear in its number of
        columns);
      * univariate factors and load vector at full size;
      * the reduced-system CG solve at full size to 1e-12.
    The value is the sum, in seconds per step of the GPU arm's metric.
    """

    def __init__(self, work, slab=16, route="sampled"):
        self.route = route
        if route == "interp":
            # the interpolation route is cheap enough to run in full every step
            self.work = work
            t0 = time.perf_counter()
            v, parts, sol = self._interp_pipeline()
            self.full = sol
            self.setup_s = time.perf_counter() - t0
            return
        import numpy as np
        from oracle.assemble import Discretisation, sample_weights
        self.work = work
        self.disc = Discretisation(work.space.degree, work.space.knots, work.space.nquad)
        from oracle.lowrank import weight_tts
        from oracle.solve import operators_from_tts, solve_kkt
        t0 = time.perf_counter()
        samples = sample_weights(work.geometry, self.disc)
        self.tts = weight_tts(work.geometry, self.disc, work.tol, work.target, samples=samples)
        Mt, Kt, diag, b = operators_from_tts(work.space, self.tts)
        y, u, lam, _ = solve_kkt(Mt, Kt, diag, b, work.beta, tol=1e-12)
        self.full = {"y": y, "u": u, "lam": lam}
        self.setup_s = time.perf_counter() - t0
        q3 = len(self.disc.x[2].ravel())
        self.S = max(1, q3 // slab)
        self.slab = q3 // self.S
        del samples
        self.np = np

    def _interp_pipeline(self):
        """The oracle's whole interpolated-weight pipeline at full size:
        (seconds, parts, solution)."""
        from oracle.assemble import Discretisation
        from oracle.interp import weight_tts_interp
        from oracle.solve import operators_from_tts, solve_kkt
        w = self.work
        t0 = time.perf_counter()
        disc = Discretisation(w.space.degree, w.space.knots, w.space.nquad)
        tts = weight_tts_interp(w.geometry, disc, w.tol, w.target)
        t1 = time.perf_counter()
        Mt, Kt, diag, b = operators_from_tts(w.space, tts)
        t2 = time.perf_counter()
        y, u, lam, _ = solve_kkt(Mt, Kt, diag, b, w.beta, tol=1e-12)
        t3 = time.perf_counter()
        parts = {"weights_s": t1 - t0, "univariate_s": t2 - t1, "solve_s": t3 - t2}
        return t3 - t0, parts, {"y": y, "u": u, "lam": lam}

    def step(self):
        """One timed step: (seconds scaled to the whole workload, parts)."""
        if self.route == "interp":
            v, parts, _ = self._interp_pipeline()
            return v, parts
        np = self.np
        from oracle.assemble import evaluate_target
        from oracle.geometry import grid_points, map_and_jacobian, weights_from_jacobian
        from oracle.lowrank import tt_svd
        from oracle.solve import operators_from_tts, solve_kkt
        w = self.work
        xs, gs = self.disc.gauss_grid()
        xs3 = [xs[0], xs[1], xs[2][:self.slab]]
        gs3 = [gs[0], gs[1], gs[2][:self.slab]]
        t0 = time.perf_counter()
        pts = grid_points(xs3)
        G, J = map_and_jacobian(w.geometry.kind, w.geometry.degree, w.geometry.knots,
                                w.geometry.homogeneous(), w.geometry.twist, pts)
        omega, Q, _ = weights_from_jacobian(J)
        shp = tuple(len(x) for x in xs3)
        g = np.einsum("a,b,c->abc", *gs3)
        om = omega.reshape(shp) * g
        Qg = Q.reshape(shp + (3, 3)) * g[..., None, None]
        f = evaluate_target(w.target, G).reshape(shp) * om
        t1 = time.perf_counter()
        qn = np.linalg.norm(Qg)
        tt_svd(om, w.tol)
        for k in range(3):
            for l in range(k, 3):
                tt_svd(np.ascontiguousarray(Qg[..., k, l]), w.tol, norm=qn)
        tt_svd(f, w.tol)
        t2 = time.perf_counter()
        Mt, Kt, diag, b = operators_from_tts(w.space, self.tts)
        t3 = time.perf_counter()
        solve_kkt(Mt, Kt, diag, b, w.beta, tol=1e-12)
        t4 = time.perf_counter()
        parts = {"sampling_s": (t1 - t0) * self.S, "tt_svd_s": (t2 - t1) * self.S,
                 "univariate_s": t3 - t2, "solve_s": t4 - t3}
        return sum(parts.values()), parts

    def describe(self):
        if self.route == "interp":
            return ("the oracle's whole pipeline at full size every step, no sampling or "
                    "scaling: weights at the Greville nodes of the degree-2p+1 space, TT-SVD, "
                    "collocation maps, univariate factors, load, reduced-system CG to 1e-12")
        return (f"oracle pipeline at full size in the set-up ({self.setup_s:.1f} s, untimed); per "
                f"step: weight sampling and TT-SVD on a slab of {self.slab} of "
                f"{self.slab * self.S} Gauss planes along direction 3, scaled x{self.S}; "
                f"univariate factors, load and reduced-system CG solve to 1e-12 at full size")


# ------------------------------------------------------------------ GPU leg

# TF32 dense tensor rate from the measured BF16 GEMM rate and the nominal
# ratio of the two (1.1 / 2.25 PFLOP/s dense per GB300)
TF32_PER_BF16 = 1.1 / 2.25
# TT ranks of the tensor-core apply measurement: the ranks of the sampled
# metric entries q_kl of the random-volume workload at TT tolerance 1e-8
# (36-38 on a 96^3 Gauss grid; omega has 33)
TTM_RANK = 37


def ttm_roofline(ctx, iga, torch, pk, pk_kind, reps=5, elements=512, kinds=("tf32", "bf16")):
    """The TT-matrix Kronecker apply on the tensor cores (TF32 and BF16
    operands) at the shape of the random-volume workload: degree 2, 512
    elements per direction (n = 512 interior functions per direction; a
    smaller `elements` gives the same shape on a smaller grid), one
    TT-matrix block of ranks (TTM_RANK, TTM_RANK) assembled from a seeded
    weight TT of those ranks on its Gauss grid.  Live CUDA-event timing of
    the fused kernel; algorithmic flops 2 (2p+1) N (R2 + R1 R2 + R1)."""
    import numpy as np
    from paper_1811_06797_gb300 import workloads as wl
    space = wl.uniform_space(2, elements)
    Q = elements * space.nquad
    R = TTM_RANK
    rng = np.random.default_rng(1811)
    cores = [rng.uniform(0.5, 1.5, (1, Q, R)), rng.standard_normal((R, Q, R)),
             rng.uniform(0.5, 1.5, (R, Q, 1))]
    tt = iga.iga_tt_from_cores(ctx, [torch.tensor(c, device="cuda") for c in cores])
    M, _ = iga.iga_ops_from_weights(ctx, space, [tt] + [None] * 6)
    N = int(np.prod(M.info()["n"]))
    x = torch.randn(N, device="cuda", dtype=torch.float32)
    y = torch.zeros(N, device="cuda", dtype=torch.float32)
    out = {}
    for kind in kinds:
        kw = {kind: True}
        iga.iga_kron_apply(ctx, M, 1.0, x, 0.0, y, **kw)
        torch.cuda.synchronize()
        ctx.profile_begin("ttm_tc_kernel")
        for _ in range(reps):
            iga.iga_kron_apply(ctx, M, 1.0, x, 0.0, y, **kw)
        p = ctx.profile_end()
        avg = p["ms"] / max(1, p["launches"])
        fl = p["flops"] / max(1, p["launches"])
        ach = fl / (avg * 1e-3) / 1e12
        peak = pk["bf16_tflops"] * (TF32_PER_BF16 if kind == "tf32" else 1.0)
        out[kind] = {"kernel": "ttm_tc_kernel", "bound": "tensor", "achieved": ach, "peak": peak,
                     "unit": "TFLOP/s", "frac": ach / peak,
                     "peak_kind": (f"{pk_kind} BF16 GEMM rate" +
                                   (" x 1.1/2.25 (nominal TF32/BF16)" if kind == "tf32" else "")),
                     "avg_ms": avg, "launches": p["launches"],
                     "algorithmic_flops_per_launch": fl,
                     "algorithmic_bytes_per_launch": p["bytes"] / max(1, p["launches"]),
                     "workload": f"random-volume shape, p=2, n={elements}^3, TT ranks ({R},{R})"}
    del M, tt, x, y
    torch.cuda.empty_cache()
    return out


def assembly_routes(assemble, work, torch, reps=3):
    """Median wall time of the low-rank assembly of the workload through both
    weight routes (interpolated in degree 2p+1, sampled on the Gauss grid)."""
    out = {}
    for route in ("interp", "sampled"):
        ts = []
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ops = assemble(work, route)
            torch.cuda.synchronize()
            ts.append((time.perf_counter() - t0) * 1e3)
            del ops
        out[route] = round(statistics.median(ts), 3)
    return out


def config5_assembly(ctx, iga, torch):
    """The random-volume workload (degree 2, 512 elements per direction, TT
    tolerance 1e-8) assembled through the paper's weight interpolation: wall
    time of iga_lowrank_assemble_interp (the weights at the 517^3 Greville
    nodes of the degree-5 interpolation space, TT-SVD, collocation solves,
    univariate assembly) and the ranks and bytes of the operators."""
    from paper_1811_06797_gb300 import workloads as wl
    work = wl.config(5)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    M, K, load = iga.iga_lowrank_assemble_interp(ctx, work.geometry, work.space, work.target,
                                                 work.tol)
    torch.cuda.synchronize()
    t = time.perf_counter() - t0
    out = {"workload": work.name, "route": "weights interpolated in degree 5 (Sec. 3)",
           "seconds": t}
    for name, op in (("M", M), ("K", K)):
        inf = op.info()
        out[name] = {"blocks": inf["nblocks"], "R_sum": list(inf["R"]), "bytes": inf["bytes"],
                     "block_ranks": [list(op.block_ranks(k)) for k in range(inf["nblocks"])]}
    del M, K, load
    torch.cuda.empty_cache()
    return out


def config5_solve(ctx, iga, torch, tol, trunc_tol, max_sweeps, state_weight=1.0, rows=512):
    """The random-volume KKT solve (degree 2, 512 elements per direction,
    beta 1e-6, 1.34e8 unknowns per field) without any full-size operator
    apply (IGA_RESID_LOCAL, the solution as the block TT), mixed precision
    (IGA_TF32: local contractions on the tensor cores, FP64 local refinement):
    wall time of the solve, its sweeps, ranks and projected residual, and the
    true relative residual estimated from `rows` uniformly sampled rows of
    the three KKT equations (iga_kkt_residual_rows)."""
    import numpy as np
    from paper_1811_06797_gb300 import workloads as wl
    work = wl.config(5)
    M, K, load = iga.iga_lowrank_assemble_interp(ctx, work.geometry, work.space, work.target,
                                                 work.tol)
    ni = M.info()["n"]
    N = int(np.prod(ni))
    bfull = torch.empty(ni, dtype=torch.float64, device="cuda")
    load.full(ctx, bfull)
    bnorm = float(bfull.norm())
    del bfull
    torch.cuda.empty_cache()
    rng = np.random.default_rng(5120)
    pts = np.stack([rng.integers(0, ni[d], rows) for d in range(3)], axis=1)
    out = {"workload": work.name, "unknowns_per_field": N, "beta": work.beta,
           "residual_mode": "projected residuals, Khatri-Rao sketches (IGA_RESID_LOCAL)",
           "tol_projected": tol, "trunc_tol": trunc_tol, "state_weight": state_weight}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ty, tu, tl, info = iga.iga_kkt_solve_amen_tt(ctx, M, K, load, work.beta, tol=tol,
                                                 precision=iga.IGA_TF32,
                                                 residual=iga.IGA_RESID_LOCAL,
                                                 max_sweeps=max_sweeps, trunc_tol=trunc_tol,
                                                 state_weight=state_weight)
    torch.cuda.synchronize()
    t = time.perf_counter() - t0
    res = iga.iga_kkt_residual_rows(ctx, M, K, work.beta, load, ty, tu, tl, pts)
    est = float(np.sqrt(N / rows * np.sum(res ** 2)) / bnorm)
    out["mixed"] = {"solve_s": t, "sweeps": info["sweeps"], "max_rank": info["max_rank"],
                    "local_iters": info["local_iters"],
                    "projected_residual": info["residual"], "converged": info["converged"],
                    "residual_estimate": est, "rows_sampled": rows,
                    "device_s_by_phase": {"local": info["t_local"], "move": info["t_move"]}}
    del ty, tu, tl
    # the tensor-core GEMMs of the local operator (right-interface products,
    # banded middle-core contraction, left-interface products) against the
    # TF32 rate, over the first two sweeps of the same solve (a separate run:
    # the per-launch events would slow the timed one)
    pk, pk_kind = peaks()
    ctx.profile_begin("tc_gemm_tf32_kernel")
    iga.iga_kkt_solve_amen_tt(ctx, M, K, load, work.beta, tol=tol, precision=iga.IGA_TF32,
                              residual=iga.IGA_RESID_LOCAL, max_sweeps=2, trunc_tol=trunc_tol,
                              state_weight=state_weight)
    p = ctx.profile_end()
    if p["launches"] > 0 and p["ms"] > 0:
        ach = p["flops"] / (p["ms"] * 1e-3) / 1e12
        peak = pk["bf16_tflops"] * TF32_PER_BF16
        out["local_contraction_roofline"] = {
            "kernel": "tc_gemm_tf32_kernel", "bound": "tensor", "achieved": ach, "peak": peak,
            "unit": "TFLOP/s", "frac": ach / peak, "launches": p["launches"],
            "device_ms": p["ms"], "algorithmic_flops": p["flops"],
            "peak_kind": f"{pk_kind} BF16 GEMM rate x 1.1/2.25 (nominal TF32/BF16)",
            "sample": "first two sweeps"}
    del M, K, load
    torch.cuda.empty_cache()
    return out


def kron_fp32_roofline(ctx, iga, torch, pk, pk_kind, reps=8):
    """The fused rank-1 Kronecker apply in FP32 storage (the bulk apply of
    the mixed path) at the twisted-annulus size of 256 elements per direction
    (degree 3, 257^3 = 1.7e7 points): the mass operator alone (one term, 8 B
    and 42 flop per point: HBM-bound) and the whole KKT operator (three
    inputs, three outputs, every term), each against the roofline that binds
    it.  L2 is flushed (256 MB write) before every launch; the launches are
    timed with CUDA events on the context stream."""
    import numpy as np
    from paper_1811_06797_gb300 import workloads as wl
    work = wl.config(3)
    M, K, _ = iga.iga_lowrank_assemble(ctx, work.geometry, work.space, work.target, work.tol)
    N = int(np.prod(M.info()["n"]))
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    g = torch.Generator(device="cuda").manual_seed(3)
    out = {"workload": work.name, "points": N, "l2": "flushed before every launch"}
    fp32_peak = alu_peak_tflops("fp32", pk)

    def measure(fn):
        fn()
        torch.cuda.synchronize()
        # the marching kernel takes the large FP32 applies; the tiled one the rest
        for kernel in ("kron_march_kernel", "kron_rank1_kernel"):
            ctx.profile_begin(kernel)
            for _ in range(reps):
                flush.zero_()
                fn()
            p = ctx.profile_end()
            torch.cuda.synchronize()
            if p["launches"] > 0:
                break
        avg = p["ms"] / p["launches"]
        by, fl = p["bytes"] / p["launches"], p["flops"] / p["launches"]
        t_hbm = by / (pk["hbm_gbs"] * 1e9)
        t_alu = fl / (fp32_peak * 1e12)
        if t_hbm >= t_alu:
            ach = by / (avg * 1e-3) / 1e9
            r = {"bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s",
                 "frac": ach / pk["hbm_gbs"], "peak_kind": pk_kind}
        else:
            ach = fl / (avg * 1e-3) / 1e12
            r = {"bound": "alu", "achieved": ach, "peak": fp32_peak, "unit": "TFLOP/s",
                 "frac": ach / fp32_peak,
                 "peak_kind": "FP32 FMA rate from unit counts and the maximum SM clock"}
        r.update({"kernel": kernel, "avg_us": avg * 1e3, "launches": p["launches"],
                  "algorithmic_bytes_per_launch": by, "algorithmic_flops_per_launch": fl})
        return r

    x = torch.randn(N, generator=g, device="cuda", dtype=torch.float32)
    y = torch.empty_like(x)
    out["mass_apply"] = measure(lambda: iga.iga_kron_apply(ctx, M, 1.0, x, 0.0, y))
    del x, y
    z = torch.randn(3 * N, generator=g, device="cuda", dtype=torch.float32)
    zo = torch.empty_like(z)
    out["kkt_apply"] = measure(lambda: iga.iga_kkt_apply(ctx, M, K, work.beta, z, zo))
    del z, zo, flush, M, K
    torch.cuda.empty_cache()
    return out


def parabolic_solve(ctx, iga, torch, work, M, K, load, nt=10, tol=1e-6, reps=2):
    """The parabolic KKT solve (Sec. 4 eq. KKTSystem, nt implicit Euler steps
    on [0, 1], tau = 1/nt; nt = 10 as in the paper's optimal-control runs) on
    the bench workload's operators: the desired state is the workload's
    target with the time profile g(t) = 1/2 + sin(pi t), b_k = tau g(t_k) b.
    Block AMEn on the space-time TT (the time index as a fourth core) in FP64
    and in mixed precision, each to the relative FP64 residual tol."""
    import numpy as np
    tau = 1.0 / nt
    N = int(np.prod(M.info()["n"]))
    b = torch.empty(N, dtype=torch.float64, device="cuda")
    load.full(ctx, b)
    g = torch.tensor([tau * (0.5 + np.sin(np.pi * tau * (k + 1))) for k in range(nt)],
                     dtype=torch.float64, device="cuda")
    B = (g[:, None] * b[None, :]).contiguous()
    y, u, lam = (torch.empty((nt, N), dtype=torch.float64, device="cuda") for _ in range(3))
    out = {"workload": work.name, "time_steps": nt, "tau": tau, "beta": work.beta,
           "unknowns_per_field": nt * N, "kkt_unknowns": 3 * nt * N, "residual_tol": tol}
    for name, prec in (("fp64", iga.IGA_FP64), ("mixed", iga.IGA_FP32)):
        ts = []
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            info = iga.iga_kkt_solve_parabolic(ctx, M, K, nt, tau, B, work.beta, y, u, lam,
                                               tol=tol, precision=prec)
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
        out[name] = {"solve_s": min(ts), "sweeps": info["sweeps"],
                     "refinements": info["refinements"], "max_rank": info["max_rank"],
                     "local_iters": info["local_iters"], "residual": info["residual"],
                     "converged": info["converged"],
                     "device_s_by_phase": {k[2:]: round(info[k], 6) for k in
                                           ("t_local", "t_residual", "t_move", "t_refine")}}
    del y, u, lam, B, b
    torch.cuda.empty_cache()
    return out


def rank_tables(ctx):
    """TT ranks of the seven sampled weights at the tolerances of the paper's
    rank tables (Sec. 6) on the two curved synthetic geometries, degree 2,
    64 elements per direction."""
    import math
    from paper_1811_06797_gb300 import report, workloads as wl
    out = {}
    space = wl.uniform_space(2, 64)
    for name, geo in (("twisted_annulus_p2_e64", wl.quarter_annulus(twist=math.pi / 4)),
                      ("random_volume_p2_e64", wl.random_volume())):
        tab = report.rank_table(ctx, geo, space, (1e-4, 1e-7, 1e-10))
        out[name] = {f"{t:g}": {w: (list(r) if r else None) for w, r in row.items()}
                     for t, row in tab.items()}
    return out


def field_errors(sol, ref):
    """Relative 2-norm and max-norm errors of (y, u, lam) against the oracle."""
    import numpy as np
    out = {}
    for name, a in zip(("y", "u", "lam"), sol):
        r = ref[name]
        out[name] = {"rel_2": float(np.linalg.norm(a - r) / np.linalg.norm(r)),
                     "rel_max": float(np.abs(a - r).max() / np.abs(r).max())}
    return out

def run_gpu(args, world, rank, local):
    import numpy as np
    import torch
    from paper_1811_06797_gb300 import build, iga, workloads as wl

    build.build()
    from paper_1811_06797_gb300 import report
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    work = wl.config(args.config)
    prec = iga.IGA_FP32 if args.precision == "mixed" else iga.IGA_FP64
    ctx = iga.Context()
    stream = torch.cuda.current_stream()
    l2flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    state = {}

    def assemble(w, route=None):
        route = route or args.weights
        if route == "interp":
            return iga.iga_lowrank_assemble_interp(ctx, w.geometry, w.space, w.target, w.tol)
        return iga.iga_lowrank_assemble(ctx, w.geometry, w.space, w.target, w.tol)

    def step():
        ea = torch.cuda.Event(enable_timing=True)
        ea.record(stream)
        M, K, load = assemble(work)
        eb = torch.cuda.Event(enable_timing=True)
        eb.record(stream)
        state["split"] = (ea, eb)
        if "y" not in state:
            N = int(np.prod(M.info()["n"]))
            state["N"] = N
            state["y"], state["u"], state["lam"] = (
                torch.empty(N, dtype=torch.float64, device="cuda") for _ in range(3))
        info = iga.iga_kkt_solve_amen(ctx, M, K, load, work.beta, state["y"], state["u"],
                                      state["lam"], tol=args.tol, precision=prec)
        state["info"] = info
        state["ops"] = (M, K, load)
        return info

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if not state["info"]["converged"]:
        raise RuntimeError(f"solve did not converge: {state['info']}")

    # dominant kernel: device time of each candidate over one (untimed) step
    shares = {}
    per_kernel = {}
    for k in CANDIDATES:
        ctx.profile_begin(k)
        step()
        p = ctx.profile_end()
        shares[k] = p["ms"]
        per_kernel[k] = p
    if args.roofline_kernel == "auto":
        args.roofline_kernel = max(shares, key=shares.get)

    # timed region (device time with CUDA events on the context stream)
    times = []
    asm_times = []
    launches0 = ctx.launches
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    ctx.profile_begin(args.roofline_kernel)
    with ClockSampler(torch.cuda.current_device()) as clk:
        for _ in range(args.steps):
            l2flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
            ea, eb = state["split"]
            asm_times.append(ea.elapsed_time(eb))
    prof = ctx.profile_end()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    launches = ctx.launches - launches0
    ms = aggregate_ms(sum(times) / len(times), dist)
    clocks = clk.summary()
    info = state["info"]
    if args.only == "step":
        # profiling case: the timed steps of the workload alone
        return {"metric": METRIC, "value": ms / 1e3, "unit": "s", "steps": args.steps,
                "warmup": args.warmup, "gpu_launches": launches // max(1, args.steps),
                "config": {"workload": work.name}, "only": "step"}, work, {}

    # the other precision path, same workload (solve only, assembly excluded)
    other = iga.IGA_FP32 if prec == iga.IGA_FP64 else iga.IGA_FP64
    M, K, load = state["ops"]
    iga.iga_kkt_solve_amen(ctx, M, K, load, work.beta, state["y"], state["u"], state["lam"],
                           tol=args.tol, precision=other)
    paths = {}
    solutions = {}
    # the two precisions with the default (pivoted) moves, and FP64 with the
    # SVD moves of the paper
    variants = [(prec, iga.IGA_TRUNC_PIVOTED), (other, iga.IGA_TRUNC_PIVOTED),
                (iga.IGA_FP64, iga.IGA_TRUNC_SVD)]
    for pr, tr in variants:
        ts = []
        for _ in range(max(2, args.steps)):
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            inf = iga.iga_kkt_solve_amen(ctx, M, K, load, work.beta, state["y"], state["u"],
                                         state["lam"], tol=args.tol, precision=pr, truncation=tr)
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        key = ("fp64" if pr == iga.IGA_FP64 else "mixed") + ("_svd_moves" if tr else "")
        paths[key] = {"solve_s": statistics.median(ts) / 1e3, "sweeps": inf["sweeps"],
                      "max_rank": inf["max_rank"], "local_iters": inf["local_iters"],
                      "residual": inf["residual"], "converged": inf["converged"]}
        solutions[key] = tuple(t.cpu().numpy().copy() for t in (state["y"], state["u"],
                                                                  state["lam"]))
    # restore the headline solution in y, u, lam
    iga.iga_kkt_solve_amen(ctx, M, K, load, work.beta, state["y"], state["u"], state["lam"],
                           tol=args.tol, precision=prec)

    # end to end through the public API with host buffers: the geometry and
    # discretisation arrays go host -> device inside the assembly call, the
    # solution (y, u, lambda) comes back into pinned host memory
    N = state["N"]
    host = torch.empty(3 * N, dtype=torch.float64, pin_memory=True)
    h2d = sum(a.nbytes for a in (*work.space.knots, *work.geometry.knots,
                                 work.geometry.homogeneous()))
    e2e_times = []
    for _ in range(max(2, args.steps // 2)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        step()
        host[:N].copy_(state["y"], non_blocking=True)
        host[N:2 * N].copy_(state["u"], non_blocking=True)
        host[2 * N:].copy_(state["lam"], non_blocking=True)
        torch.cuda.synchronize()
        e2e_times.append(time.perf_counter() - t0)
    e2e = statistics.median(e2e_times)

    pk, pk_kind = peaks()
    roof = None
    if prof["launches"] > 0 and prof["ms"] > 0:
        avg_ms = prof["ms"] / prof["launches"]
        by = prof["bytes"] / prof["launches"]
        fl = prof["flops"] / prof["launches"]
        arith = CANDIDATES.get(args.roofline_kernel, "fp64")
        if arith == "prec":
            arith = "fp64" if args.precision == "fp64" else "fp32"
        alu_peak = alu_peak_tflops(arith, pk)
        t_alu = fl / (alu_peak * 1e12)
        t_hbm = by / (pk["hbm_gbs"] * 1e9)
        if t_alu >= t_hbm:
            achieved = fl / (avg_ms * 1e-3) / 1e12
            roof = {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                    "frac": achieved / alu_peak,
                    "peak_kind": f"{arith.upper()} FMA rate from unit counts and the maximum "
                                 f"SM clock (CUDA cores)"}
        else:
            achieved = by / (avg_ms * 1e-3) / 1e9
            roof = {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                    "frac": achieved / pk["hbm_gbs"], "peak_kind": pk_kind}
        roof.update({"traffic": NCU_TRAFFIC.get(args.roofline_kernel), "kernel": args.roofline_kernel,
                     "launches": prof["launches"], "avg_us": avg_ms * 1e3,
                     "algorithmic_bytes_per_launch": by, "algorithmic_flops_per_launch": fl,
                     "device_ms_per_step_by_kernel": {k: round(v, 3) for k, v in shares.items()}})

    # the Kronecker apply (KKT residuals) against the FP64 rate: the metric's
    # second part, from the same untimed per-kernel step
    kron_roof = alu_roofline("kron_rank1_kernel", per_kernel.get("kron_rank1_kernel"),
                             alu_peak_tflops("fp64", pk),
                             "FP64 FMA rate from unit counts and the maximum SM clock")

    line = {
        "metric": METRIC,
        "value": ms / 1e3,
        "unit": "s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms,
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32+f64" if args.precision == "mixed" else "f64",
        "data": "synthetic",
        "config": {"workload": work.name, "unknowns_per_field": N, "kkt_unknowns": 3 * N,
                   "beta": work.beta, "tt_tol": work.tol, "residual_tol": args.tol,
                   "precision": args.precision,
                   "weights": ("interpolated in degree 2p+1 at the Greville nodes"
                               if args.weights == "interp" else "sampled on the Gauss grid"),
                   "l2": "flushed (256 MB write) before every step",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "solve": {**{k: info[k] for k in ("sweeps", "refinements", "max_rank", "local_iters",
                                          "residual")},
                  "device_s_by_phase": {k[2:]: round(info[k], 6) for k in
                                        ("t_local", "t_residual", "t_move", "t_refine")}},
        "step_split_ms": {"assembly": round(statistics.mean(asm_times), 3),
                          "solve": round(statistics.mean(times) - statistics.mean(asm_times), 3)},
        "paths": paths,
        "e2e": {"value": e2e, "unit": "s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(3 * N * 8)},
        "gpu_launches": int(launches),
        "gpu_launches_per_step": int(launches / max(1, args.steps)),
        "roofline": roof,
        "kron_roofline": kron_roof,
        "ttm_roofline": ttm_roofline(ctx, iga, torch, pk, pk_kind),
        "kron_fp32_roofline": kron_fp32_roofline(ctx, iga, torch, pk, pk_kind),
        "assembly_routes_ms": assembly_routes(assemble, work, torch),
        "rank_tables": rank_tables(ctx),
        "config5_assembly": config5_assembly(ctx, iga, torch),
        "config5_solve": config5_solve(ctx, iga, torch, args.c5_tol, args.c5_trunc,
                                       args.c5_sweeps, args.c5_state_weight),
        "parabolic_solve": parabolic_solve(ctx, iga, torch, work, *state["ops"], nt=args.nt),
        "storage": {work.name: report.storage(ctx, work.geometry, work.space, work.target,
                                              work.tol)},
        "alu_rates_measured_tflops": {"fp64": iga.iga_measure_fma(ctx, iga.IGA_FP64),
                                      "fp32": iga.iga_measure_fma(ctx, iga.IGA_FP32)},
        "clocks": clocks,
    }
    return line, work, solutions


def oracle_baseline(work, steps, route):
    """cpu_baseline: the oracle leg's set-up plus `steps` timed steps."""
    leg = OracleLeg(work, route=route)
    vals, parts = [], None
    for _ in range(max(1, steps)):
        v, parts = leg.step()
        vals.append(v)
    return leg, {"value": statistics.median(vals), "unit": "s", "cores": _threads(),
                 "kind": "oracle", "sample": leg.describe(),
                 "parts_s": {k: round(v, 3) for k, v in parts.items()},
                 "setup_s": round(leg.setup_s, 2)}


def run_reference(args):
    """The oracle timed as it stands on the host cores (no GPU): the set-up,
    W untimed and K timed steps of the bounded sample (OracleLeg)."""
    from paper_1811_06797_gb300 import workloads as wl
    work = wl.config(args.config)
    leg = OracleLeg(work, route=args.weights)
    for _ in range(args.warmup):
        leg.step()
    vals, parts = [], None
    for _ in range(args.steps):
        v, parts = leg.step()
        vals.append(v)
    v = statistics.median(vals)
    return {
        "metric": METRIC, "value": v, "unit": "s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": work.name,
                   "weights": "interpolated" if args.weights == "interp" else "sampled"},
        "impl": "reference",
        "cpu_baseline": {"kind": "oracle", "cores": _threads(), "sample": leg.describe(),
                         "value": v, "unit": "s",
                         "parts_s": {k: round(x, 3) for k, x in parts.items()}},
        "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    args = parse()
    world, rank, local = dist_env()
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)))
        return
    if args.only == "ttm":
        import torch
        from paper_1811_06797_gb300 import build, iga
        build.build()
        torch.cuda.set_device(local)
        pk, pk_kind = peaks()
        out = ttm_roofline(iga.Context(), iga, torch, pk, pk_kind, reps=args.steps,
                           elements=args.ttm_elements, kinds=tuple(args.ttm_kinds.split(",")))
        if rank == 0:
            print(json.dumps({"ttm_roofline": out}))
        return
    if args.only == "c5solve":
        import torch
        from paper_1811_06797_gb300 import build, iga
        build.build()
        torch.cuda.set_device(local)
        out = config5_solve(iga.Context(), iga, torch, args.c5_tol, args.c5_trunc, args.c5_sweeps,
                            args.c5_state_weight)
        if rank == 0:
            print(json.dumps({"config5_solve": out}))
        return
    if args.only == "kron32":
        import torch
        from paper_1811_06797_gb300 import build, iga
        build.build()
        torch.cuda.set_device(local)
        pk, pk_kind = peaks()
        out = kron_fp32_roofline(iga.Context(), iga, torch, pk, pk_kind)
        if rank == 0:
            print(json.dumps({"kron_fp32_roofline": out}))
        return
    if args.only == "parabolic":
        import torch
        from paper_1811_06797_gb300 import build, iga, workloads as wl
        build.build()
        torch.cuda.set_device(local)
        ctx = iga.Context()
        work = wl.config(args.config)
        M, K, load = iga.iga_lowrank_assemble_interp(ctx, work.geometry, work.space, work.target,
                                                     work.tol)
        out = parabolic_solve(ctx, iga, torch, work, M, K, load, nt=args.nt, tol=args.tol,
                              reps=max(1, args.steps))
        if rank == 0:
            print(json.dumps({"parabolic_solve": out}))
        return
    line, work, solutions = run_gpu(args, world, rank, local)
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline and args.only is None:
            try:
                leg, base = oracle_baseline(work, 2, args.weights)
                line["cpu_baseline"] = base
                # the error of every result against the oracle's solution
                line["oracle_errors"] = {k: field_errors(v, leg.full) for k, v in solutions.items()}
            except Exception as e:   # the baseline is reported, not required
                line["cpu_baseline"] = {"value": None, "unit": "s", "kind": "oracle",
                                        "cores": os.cpu_count(), "sample": f"failed: {e}"}
        print(json.dumps(line))


if __name__ == "__main__":
    main()
