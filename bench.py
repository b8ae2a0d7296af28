"""Benchmark of the matrix-free operator apply on one macro-tetrahedron at level 8.

Workload (synthetic, seeded): the reference macro-tetrahedron refined to
level 8 (2,862,209 P1 / 22,632,705 P2 points), variable coefficient
k(x) = 1 + 0.5 sin(2 pi x) sin(2 pi y) sin(2 pi z) at quadrature points
(4-point degree-2 rule for P1, 14-point rule for P2), zero Dirichlet
boundary, x ~ U[-1, 1] from seed 0, FP64 and FP32 applies.  One step applies
every leg once; each apply runs after an L2 flush (a 512 MB write), timed with
CUDA events on the launching stream.  Metric: updated (interior) DoFs per
second over the whole step, in MDoF/s.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun each rank runs an independent replica (the apply of one mesh
needs no data from other GPUs); value = DoFs of all ranks / max rank time.
"""
from __future__ import annotations

import argparse
import itertools
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "operator apply MDoF/s & % HBM roofline; FMG time-to-1e-10 residual, FP32-mixed vs FP64"
LEVEL = 8

# (name, degree, coefficient, quad_degree, dtype)
LEGS = [
    ("p1_sin3_f64", 1, ("sin3",), 2, "f64"),
    ("p1_sin3_f32", 1, ("sin3",), 2, "f32"),
    ("p2_sin3_f64", 2, ("sin3",), 4, "f64"),
    ("p2_sin3_f32", 2, ("sin3",), 4, "f32"),
]
# Algorithmic FLOPs per unit (point or micro-tet) of each apply variant.
def flops_per_unit(name: str, degree: int, nq: int):
    if name.startswith("p1_const"):
        return ("dof", 30.0)                       # 15-point stencil: 15 FMA per point
    if name.startswith("p1_sin3"):
        return ("tet", nq * 15.0 + 36.0)           # k at nq points (angle addition), kbar, 4x4 apply
    if name.startswith("p2_const"):
        return ("tet", 2.0 * 100)                  # 10x10 apply
    if name.startswith("p2_sin3"):
        return ("tet", 117.0 * nq)                 # fused quadrature: grad u, k, metric, test (per point)
    return ("dof", 0.0)


# FLOP (FMA = 2) per micro-tet and right-hand side of the epsilon kernels as formulated: the affine
# symmetric gradient of the three components (390: reference affine terms, J^-1 map, 24 entries),
# per quadrature point its value (36), the stress (6) and its moments (42), i.e. 84 x 14 points, the
# moments mapped back and tested (342), mu at the points shared by the right-hand sides (308 / 16);
# the adjoint forms the terms of u and g (780), per point both gradients, E(g) : E(u) / 2 and the
# ten basis moments (106 x 14), and sums over the right-hand sides by shuffles (40).
EPS_FLOP_PER_TET_RHS = {"apply": 390 + 84 * 14 + 342 + 19, "adjoint": 780 + 106 * 14 + 40}


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            p = json.load(f)
        return {"hbm_gbs": p["hbm_gbs"], "src": "measured"}
    return {"hbm_gbs": 6800.0, "src": "fallback"}


# FP64 / FP32 ALU peaks from unit counts: FMA per clock per SM (GB300: 2 FP64, 128 FP32; the
# FMA-chain probe paper_2404_08371_gb300/peaks.cu measures the per-clock rate) x 2 FLOP x SMs x the
# SM clock sampled by nvidia-smi during the timed region (the maximum clock if no sample was taken).
FMA_PER_CLK_SM = {"f64": 2, "f32": 128}


def alu_peak_tflops(dt: str, sms: int, sm_mhz: float) -> float:
    return FMA_PER_CLK_SM[dt] * 2.0 * sms * sm_mhz * 1e6 / 1e12


def load_traffic():
    """DRAM bytes per launch from an ncu capture (profiles/traffic.json), dropped when the kernel's
    sources changed after the capture (their sha256 no longer matches)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return {}
    with open(path) as f:
        table = json.load(f)
    out = {}
    for leg, rec in table.items():
        h = hashlib.sha256()
        try:
            for fn in rec["sources"]:
                with open(os.path.join(ROOT, fn), "rb") as f:
                    h.update(f.read())
        except OSError:
            continue
        if h.hexdigest() == rec["sources_sha256"]:
            out[leg] = rec
    return out


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.idx = device_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def host_cpu():
    """CPU model, logical CPU count and the CPUs this process may run on."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if model is None:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith(("model name", "cpu part")):
                        model = line.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    import platform
    return {"model": model or platform.processor() or platform.machine(), "machine": platform.machine(),
            "nproc": os.cpu_count(), "affinity": len(os.sched_getaffinity(0))}


CPU_LEGS = [("p1_sin3", 1, 7, 2), ("p2_sin3", 2, 6, 4)]   # (name, degree, level, quadrature degree)


def cpu_assemble():
    """The oracle's operators of the CPU sample: the reference macro, sin3 coefficient, Dirichlet,
    P1 at level 7 and P2 at level 6 (366,145 points each; the level-8 operators take minutes to
    assemble, beyond a bounded sample).  Returns [(name, level, interior dofs, CSR, x, seconds)]."""
    import workloads as W
    from oracle import assemble as OA, mesh as OM
    mm = OM.MacroMesh(*W.reference_tet())
    out = []
    for name, degree, level, qd in CPU_LEGS:
        t0 = time.perf_counter()
        S = OA.Space(mm, level, degree)
        A = OA.diffusion_matrix(S, ("sin3",), qd, "dirichlet")
        out.append((name, level, int(S.interior.sum()), A, W.uniform(S.ndof, seed=0), time.perf_counter() - t0))
    return out


def time_spmv(fn, min_s: float = 1.0) -> float:
    """Mean seconds of fn() over repetitions filling at least min_s (at least 3)."""
    fn()
    reps, t0 = 0, time.perf_counter()
    while reps < 3 or time.perf_counter() - t0 < min_s:
        fn()
        reps += 1
    return (time.perf_counter() - t0) / reps


def cpu_baseline():
    """The oracle as it stands on the host: element-by-element CSR assembly, then the sparse apply,
    (i) scipy on one thread, (ii) the oracle's OpenMP CSR product on every core, (iii) assembly
    timed apart; plus the oracle's FP64 FMG on the FMG workload's mesh at level 4."""
    from oracle import spmv
    host = host_cpu()
    threads = spmv.max_threads()
    res = {}
    dofs = t1 = tn = t_asm = 0.0
    for name, level, nint, A, x, ta in cpu_assemble():
        op = spmv.CsrSpmv(A)
        s1 = time_spmv(lambda: A @ x)
        sn = time_spmv(lambda: op(x, threads))
        res[name] = {"level": level, "dofs": nint, "spmv_1thread_mdofs": nint / s1 / 1e6,
                     "spmv_all_cores_mdofs": nint / sn / 1e6, "assembly_s": ta,
                     "assembly_plus_spmv_mdofs": nint / (ta + s1) / 1e6}
        dofs, t1, tn, t_asm = dofs + nint, t1 + s1, tn + sn, t_asm + ta
    # the oracle's FP64 FMG + V(2,2) on the FMG workload's mesh, at a level it finishes in seconds
    import workloads as W
    from oracle import mesh as OM, mg as OMG
    fl = 4
    t0 = time.perf_counter()
    H = OMG.Hierarchy(OM.MacroMesh(*W.cube6()), fl, 2, quad_degree=4)
    b = OMG.load_vector(H.spaces[fl], W.manufactured_f)
    t_setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    xf, cycles, hist = H.fmg(b, tol=1e-10)
    t_solve = time.perf_counter() - t0
    nint = int(H.spaces[fl].interior.sum())
    fmg = {"workload": "unit cube as 6 macros, level %d, P2 Poisson, FMG (coarse right-hand sides restricted) "
                       "+ V(2,2), tol 1e-10, FP64, one thread" % fl,
           "dofs": nint, "setup_s": t_setup, "solve_s": t_solve, "cycles": cycles,
           "rel_residual": float(hist[-1]), "l2_error": OMG.l2_error(H.spaces[fl], xf, W.manufactured_u),
           "mdofs_per_s": nint / t_solve / 1e6}
    return {"value": dofs / tn / 1e6, "unit": "MDoF/s", "cores": threads, "kind": "oracle",
            "sample": "reference macro, sin3 coefficient, Dirichlet: P1 at level 7 + P2 at level 6 (366,145 points "
                      "each, the level-8 workload's operators at 1/8 of its size), FP64 CSR product on %d OpenMP "
                      "threads (assembly timed separately: %.1f s)" % (threads, t_asm),
            "value_1thread": dofs / t1 / 1e6, "host": host, "legs": res, "fmg": fmg}


def run_fmg(hhg, torch, level: int, reps: int = 1):
    """FMG + V(2,2) Chebyshev solves of the manufactured Poisson problem, P2, unit cube as 6 macros.

    All-FP64 against FP32 cycles inside FP64 iterative refinement, to a relative residual of 1e-10.
    Times are CUDA-event device times of the solve (FMG + iterations); the hierarchy set-up of the
    first call is reported separately.  The discretisation error is also taken one level coarser.
    """
    import workloads as W
    v, t = W.cube6()
    out = {"workload": "unit cube as 6 macros, level %d, P2 Poisson, f = 3 pi^2 sin sin sin, FMG + V(2,2), "
                       "Chebyshev order 2, tol 1e-10" % level}
    errs = {}
    for lvl in (level - 1, level):
        mesh = hhg.Mesh(v, t, lvl)
        op = hhg.Operator(mesh, degree=2, coeff=("const", 1.0), bc="dirichlet", quad_degree=4)
        b = mesh.rhs_sin3_poisson(2)
        tot, inner = mesh.dof_count(2)
        for name, mixed in (("fp64", 0), ("mixed", 1)):
            x, st0 = op.mg_solve(b, torch.zeros_like(b), mixed=mixed)
            ms = []
            for _ in range(reps if lvl == level else 0):
                x, st = op.mg_solve(b, torch.zeros_like(b), mixed=mixed)
                ms.append(st["solve_ms"])
            e = mesh.l2_error_sin3(x, 2)
            errs[(name, lvl)] = e
            if lvl == level:
                out[name] = {"solve_ms": min(ms), "setup_ms": st0["setup_ms"], "iterations": st["iterations"],
                             "rel_residual": st["rel_residual"], "l2_error": e, "dofs": inner,
                             "mdofs_per_s": inner / (min(ms) * 1e-3) / 1e6}
        if lvl == level:
            # the same solves with the FP64 applies in double-float arithmetic (FP32 pairs), coarse
            # operators included: all cycles, and the FP64 residuals of the mixed solve
            opd = hhg.Operator(mesh, degree=2, coeff=("const", 1.0), bc="dirichlet", quad_degree=4)
            opd.set_fp64_arith("double_float")
            for name, mixed in (("fp64_double_float", 0), ("mixed_double_float", 1)):
                x, st0 = opd.mg_solve(b, torch.zeros_like(b), mixed=mixed)
                ms = []
                for _ in range(reps):
                    x, st = opd.mg_solve(b, torch.zeros_like(b), mixed=mixed)
                    ms.append(st["solve_ms"])
                out[name] = {"solve_ms": min(ms), "iterations": st["iterations"], "rel_residual": st["rel_residual"],
                             "l2_error": mesh.l2_error_sin3(x, 2)}
            del opd
        del op, mesh
    for name in ("fp64", "mixed"):
        out[name]["l2_error_ratio_vs_level_%d" % (level - 1)] = errs[(name, level - 1)] / errs[(name, level)]
    out["mixed_speedup"] = out["fp64"]["solve_ms"] / out["mixed"]["solve_ms"]
    return out


def aggregate_replicas(step_ms: float, dofs_step: float, device="cpu"):
    """Whole-job figures of independent per-rank replicas: (max step time over ranks in ms, sum of
    the ranks' DoFs per step, rate in MDoF/s = that sum / that max time)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([step_ms], dtype=torch.float64, device=device)
    d = torch.tensor([float(dofs_step)], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(d, op=dist.ReduceOp.SUM)
    ms, dofs = float(t.item()), float(d.item())
    return ms, dofs, dofs / (ms * 1e-3) / 1e6


def time_apply(torch, fn, flush, reps: int, warmup: int = 1):
    """Mean CUDA-event time (ms) of fn() on the current stream, L2 flushed before every call."""
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        fn()
    ms = []
    for _ in range(reps):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    return statistics.mean(ms)


def run_const_legs(hhg, torch, flush, peak_gbs: float, reps: int = 5):
    """Constant-coefficient applies on working sets larger than L2: P1 at level 9, P2 at level 8."""
    import workloads as W
    v, t = W.reference_tet()
    out = {}
    for name, level, degree in (("p1_const", 9, 1), ("p2_const", 8, 2)):
        mesh = hhg.Mesh(v, t, level)
        op = hhg.Operator(mesh, degree=degree, coeff=("const", 1.0), bc="dirichlet")
        tot, inner = mesh.dof_count(degree)
        variants = [("f64", torch.float64, "native"), ("f32", torch.float32, "native"),
                    ("df64", torch.float64, "double_float")]   # FP64 vectors, FP32-pair arithmetic
        for dt, tdt, arith in variants:
            op.set_fp64_arith(arith) if tdt == torch.float64 else None
            x = torch.from_numpy(W.uniform(mesh.vec_size(degree), seed=0)).to("cuda", tdt)
            y = torch.empty_like(x)
            ms = time_apply(torch, lambda: op.apply(x, out=y), flush, reps)
            nbytes = 2 * x.numel() * x.element_size()
            key = "%s_%s" % (name, dt)
            tr = load_traffic().get(key)
            out[key] = {"level": level, "ms": ms, "mdofs": inner / ms / 1e3, "gbs": nbytes / ms / 1e6,
                        "hbm_frac": nbytes / ms / 1e6 / peak_gbs, "bytes": nbytes,
                        "arith": {"f64": "fp64", "f32": "fp32", "df64": "double-float (FP32 pairs, 48-bit "
                                  "significands; FP64 input and output)"}[dt],
                        "traffic": tr["bytes_per_launch"] if tr else None}
            del x, y
        op.set_fp64_arith("native")
        del op, mesh
    return out


def run_eps(hhg, torch, flush, fp64_peak: float, level: int = 6, nrhs: int = 16, reps: int = 1):
    """P2 vector epsilon operator on the unit cube as 48 macros, mu = 10^(3(z-0.5)) as a P2 field,
    nrhs seeded right-hand sides in one launch (FP64), and its adjoint in mu."""
    import workloads as W
    v, t = W.cube48()
    mesh = hhg.Mesh(v, t, level)
    n = mesh.vec_size(2)
    # mu = 10^(3(z - 0.5)) at the packed points of every macro (a P2 field)
    xyz = mesh.coordinates(2)
    mu_t = torch.pow(10.0, 3.0 * (xyz[:, 2] - 0.5)).contiguous()
    op = hhg.Operator(mesh, kind="epsilon", degree=2, coeff=("field_p2", mu_t), bc="dirichlet", quad_degree=4)
    x = torch.empty(n * 3 * nrhs, dtype=torch.float64, device="cuda")
    for r in range(nrhs):
        x.view(n, 3, nrhs)[:, :, r] = torch.from_numpy(W.uniform(3 * n, seed=r)).to("cuda").view(n, 3)
    mesh.make_consistent(x, 2, per_point=3 * nrhs)
    y = torch.empty_like(x)
    tot, inner = mesh.dof_count(2)
    ms = time_apply(torch, lambda: op.apply(x, out=y, nrhs=nrhs), flush, reps)
    ms_adj = time_apply(torch, lambda: op.adjoint_coeff(x, y, nrhs=nrhs), flush, reps)
    ntet = len(t) * 8 ** level
    fl_apply = EPS_FLOP_PER_TET_RHS["apply"] * ntet * nrhs
    fl_adj = EPS_FLOP_PER_TET_RHS["adjoint"] * ntet * nrhs
    return {"workload": "unit cube as 48 macros, level %d, P2 vector epsilon, mu = 10^(3(z-0.5)) P2 field, "
                        "%d right-hand sides, FP64, Dirichlet" % (level, nrhs),
            "apply_ms": ms, "adjoint_ms": ms_adj, "mdofs": 3 * inner * nrhs / ms / 1e3,
            "adjoint_mdofs": 3 * inner * nrhs / ms_adj / 1e3, "micro_tets": ntet,
            "flop_per_tet_per_rhs": dict(EPS_FLOP_PER_TET_RHS),
            "apply_tflops": fl_apply / ms / 1e9, "apply_fp64_frac": fl_apply / ms / 1e9 / fp64_peak,
            "adjoint_tflops": fl_adj / ms_adj / 1e9, "adjoint_fp64_frac": fl_adj / ms_adj / 1e9 / fp64_peak,
            "fp64_peak_tflops": fp64_peak}


def run_adjoint(hhg, torch, flush, peak_gbs: float, level: int = 7, reps: int = 5):
    """The coefficient-inversion workload's kernels: reference macro at level 7, P1, k = exp(g) as a
    P1 nodal field (g the seeded sum of 8 Fourier modes, amplitude 0.5), u and g ~ U[-1, 1] (seeds 1
    and 2), Dirichlet; the adjoint dk_v = sum_T 1/4 g_T^T A0_T u_T (reads u and g, writes dk) and
    the apply of the same operator, FP64 and FP32."""
    import workloads as W
    v, t = W.reference_tet()
    mesh = hhg.Mesh(v, t, level)
    n = mesh.vec_size(1)
    xyz = mesh.coordinates(1).cpu().numpy()
    kval = np.exp(W.fourier_field(xyz, seed=0))
    tot, inner = mesh.dof_count(1)
    out = {"workload": "reference macro, level %d, P1, k = exp(g) P1 field (8 Fourier modes, amplitude 0.5), "
                       "Dirichlet: adjoint dL/dk and apply" % level}
    for dt, tdt in (("f64", torch.float64), ("f32", torch.float32)):
        k = torch.from_numpy(kval).to("cuda", tdt)
        op = hhg.Operator(mesh, degree=1, coeff=("field_p1", k), bc="dirichlet", quad_degree=2)
        u = torch.from_numpy(W.uniform(n, seed=1)).to("cuda", tdt)
        g = torch.from_numpy(W.uniform(n, seed=2)).to("cuda", tdt)
        dk = torch.empty_like(u)
        y = torch.empty_like(u)
        ms_adj = time_apply(torch, lambda: op.adjoint_coeff(u, g, out=dk), flush, reps)
        ms_app = time_apply(torch, lambda: op.apply(u, out=y), flush, reps)
        nbytes = 3 * n * u.element_size()          # read u and g, write dk
        out[dt] = {"adjoint_ms": ms_adj, "adjoint_mdofs": inner / ms_adj / 1e3, "adjoint_gbs": nbytes / ms_adj / 1e6,
                   "adjoint_hbm_frac": nbytes / ms_adj / 1e6 / peak_gbs, "apply_ms": ms_app,
                   "apply_mdofs": inner / ms_app / 1e3, "points": n}
        del op, k, u, g, dk, y
    return out


def run_n1(hhg, torch, flush, level: int = 7, reps: int = 3):
    """Nedelec curl-curl + mass (Eq. N1) on the 36-macro 3x2x1 cuboid (the paper's test domain) at
    level 7, alpha and beta P1 fields, FP64 and FP32, Dirichlet; MDoF/s counts interior edges."""
    import workloads as W
    v, t = W.cuboid36()
    mesh = hhg.Mesh(v, t, level)
    out = {"workload": "3x2x1 cuboid as 36 macros, level %d, N1 curl-curl + mass, alpha = 1 + x/3, "
                       "beta = 1 + z (P1 fields), Dirichlet" % level}
    xyz1 = mesh.coordinates(1)
    # interior edges: the distinct edge midpoints minus the boundary ones (from the degree-2 counts)
    tot2, int2 = mesh.dof_count(2)
    tot1, int1 = mesh.dof_count(1)
    n_edges_interior = int2 - int1
    for dt, tdt in (("f64", torch.float64), ("f32", torch.float32)):
        a = (1.0 + xyz1[:, 0] / 3.0).to(tdt).contiguous()
        b = (1.0 + xyz1[:, 2]).to(tdt).contiguous()
        op = hhg.CurlCurl(mesh, ("field_p1", a), ("field_p1", b), bc="dirichlet")
        x = torch.from_numpy(W.uniform(mesh.vec_size(2), seed=0)).to("cuda", tdt)
        y = torch.empty_like(x)
        ms = time_apply(torch, lambda: op.apply(x, out=y), flush, reps)
        out[dt] = {"ms": ms, "mdofs": n_edges_interior / ms / 1e3, "interior_edges": n_edges_interior}
        if dt == "f64":
            tr = load_traffic().get("n1_f64")
            out[dt]["traffic"] = tr["bytes_per_launch"] if tr else None
        # precomputed variant: the 21 entries per micro-tet stored once (set-up timed separately)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        op.store_element_matrices(tdt)
        e1.record()
        torch.cuda.synchronize()
        ms_st = time_apply(torch, lambda: op.apply(x, out=y), flush, reps)
        out[dt]["stored"] = {"ms": ms_st, "mdofs": n_edges_interior / ms_st / 1e3, "setup_ms": e0.elapsed_time(e1)}
        del op, x, y
    return out


def n1_interpolant(mesh, torch, E):
    """Packed Nedelec vector of the smooth field E (points (n, 3) -> (n, 3), torch): on every edge
    point of the doubled lattice E at the midpoint dotted with the physical edge vector along the
    macro's canonical lattice direction (midpoint rule; vertex points 0).  Synthetic input only."""
    import numpy as np
    N = 2 ** (mesh.level + 1)
    pts = []
    for k in range(N + 1):
        for j in range(N + 1 - k):
            for_i = np.arange(N - k - j + 1)
            pts.append(np.stack([for_i, np.full_like(for_i, j), np.full_like(for_i, k)], axis=1))
    pts = np.concatenate(pts)
    par = pts & 1
    d = par.copy()
    d[(par[:, 0] == 1) & (par[:, 1] == 1), 1] = -1
    sel = ((par[:, 0] == 1) | (par[:, 1] == 1)) & (par[:, 2] == 1) & ~((par[:, 0] == 1) & (par[:, 1] == 1))
    d[sel, 2] = -1
    edge = par.any(axis=1)

    def packed(q):
        i, j, k = q[:, 0], q[:, 1], q[:, 2]
        vk = lambda s: (s + 1) * (s + 2) * (s + 3) // 6
        m = N - k
        return vk(N) - vk(N - k) + j * (m + 1) - j * (j - 1) // 2 + i

    start, end = packed(np.where(edge[:, None], pts - d, pts)), packed(np.where(edge[:, None], pts + d, pts))
    V = len(pts)
    xyz = mesh.coordinates(2).view(-1, V, 3)
    s_t = torch.from_numpy(start).to(xyz.device)
    e_t = torch.from_numpy(end).to(xyz.device)
    vec = xyz[:, e_t] - xyz[:, s_t]                        # (macros, V, 3): zero at vertex points
    val = (E(xyz.reshape(-1, 3)).view(-1, V, 3) * vec).sum(dim=2)
    return val.reshape(-1).contiguous()


def run_n1_fmg(hhg, torch, level: int = 6):
    """FMG + V(2,2) with Hiptmair's hybrid smoother for the curl-curl + mass problem (Eq. N1,
    alpha = beta = 1) on the 36-macro 3x2x1 cuboid, all-FP64 against FP32 cycles inside FP64
    refinement, to a relative residual of 1e-10.  b = A u_I with u_I the Nedelec interpolant of
    E = (sin pi y sin pi z, sin pi x sin pi z, sin pi x sin pi y); times are CUDA-event device
    times of the solve (FMG + iterations), the hierarchy set-up reported apart."""
    import math
    import workloads as W
    v, t = W.cuboid36()
    mesh = hhg.Mesh(v, t, level)
    op = hhg.CurlCurl(mesh, ("const", 1.0), ("const", 1.0), bc="dirichlet")

    def E(p):
        s = torch.sin(math.pi * p)
        return torch.stack([s[:, 1] * s[:, 2], s[:, 0] * s[:, 2], s[:, 0] * s[:, 1]], dim=1)

    u = n1_interpolant(mesh, torch, E)
    b = op.apply(u)
    tot2, int2 = mesh.dof_count(2)
    tot1, int1 = mesh.dof_count(1)
    n_edges = int2 - int1
    out = {"workload": "3x2x1 cuboid as 36 macros, level %d, N1 curl-curl + mass (alpha = beta = 1), "
                       "b = A u_I, FMG + V(2,2) with the hybrid smoother, tol 1e-10" % level,
           "interior_edges": n_edges}
    for name, mixed in (("fp64", 0), ("mixed", 1)):
        x, st0 = op.mg_solve(b, torch.zeros_like(b), mixed=mixed)
        x, st = op.mg_solve(b, torch.zeros_like(b), mixed=mixed)
        err = ((x - u).abs().max() / u.abs().max()).item()
        out[name] = {"solve_ms": st["solve_ms"], "setup_ms": st0["setup_ms"], "iterations": st["iterations"],
                     "rel_residual": st["rel_residual"], "max_rel_diff_to_u_I": err,
                     "mdofs_per_s": n_edges / (st["solve_ms"] * 1e-3) / 1e6}
    out["mixed_speedup"] = out["fp64"]["solve_ms"] / out["mixed"]["solve_ms"]
    return out


def run_underint(hhg, torch, flush, level: int = 8, reps: int = 3):
    """P2 with the analytic coefficient under-integrated by the degree-2 (4-point) rule, the
    paper's under-integration variant (Section 6.7), reference macro at level 8."""
    import workloads as W
    v, t = W.reference_tet()
    mesh = hhg.Mesh(v, t, level)
    op = hhg.Operator(mesh, degree=2, coeff=("sin3",), bc="dirichlet", quad_degree=2)
    tot, inner = mesh.dof_count(2)
    out = {"workload": "reference macro, level %d, P2, sin3 coefficient at the 4-point degree-2 rule" % level}
    for dt, tdt in (("f64", torch.float64), ("f32", torch.float32)):
        x = torch.from_numpy(W.uniform(mesh.vec_size(2), seed=0)).to("cuda", tdt)
        y = torch.empty_like(x)
        ms = time_apply(torch, lambda: op.apply(x, out=y), flush, reps)
        out[dt] = {"ms": ms, "mdofs": inner / ms / 1e3}
        del x, y
    return out


def run_precomputed(hhg, torch, flush, level: int = 8, reps: int = 3):
    """The precomputed variant against the matrix-free apply: local matrices of the sin3 legs
    integrated once and stored (set-up timed separately), reference macro at level 8."""
    import workloads as W
    v, t = W.reference_tet()
    mesh = hhg.Mesh(v, t, level)
    out = {"workload": "reference macro, level %d, sin3 coefficient: stored local matrices vs matrix-free" % level}
    for deg, qd in ((2, 4), (1, 2)):
        tot, inner = mesh.dof_count(deg)
        for dt, tdt in (("f64", torch.float64), ("f32", torch.float32)):
            op = hhg.Operator(mesh, degree=deg, coeff=("sin3",), bc="dirichlet", quad_degree=qd)
            x = torch.from_numpy(W.uniform(mesh.vec_size(deg), seed=0)).to("cuda", tdt)
            y = torch.empty_like(x)
            free = time_apply(torch, lambda: op.apply(x, out=y), flush, reps)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            op.store_element_matrices(tdt)
            e1.record()
            torch.cuda.synchronize()
            setup = e0.elapsed_time(e1)
            stored = time_apply(torch, lambda: op.apply(x, out=y), flush, reps)
            nbytes = len(t) * 6 * (55 if deg == 2 else 1) * (2 ** level) * (2 ** level + 1) * (2 ** level + 2) // 6 * \
                (8 if dt == "f64" else 4)
            out["p%d_sin3_%s" % (deg, dt)] = {"matrix_free_ms": free, "stored_ms": stored, "setup_ms": setup,
                                              "stored_mdofs": inner / stored / 1e3, "stored_bytes": nbytes,
                                              "break_even_applies": setup / (free - stored) if free > stored else None}
            del op, x, y
            torch.cuda.empty_cache()
    return out


def run_reference(args):
    """The oracle as the reference arm: its operators assembled once (outside the steps, as the
    library's operators are created before its timed region), then every step applies each leg
    once with the oracle's OpenMP CSR product on all host cores.  Rank 0 only."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import spmv
    threads = spmv.max_threads()
    legs = [(nint, spmv.CsrSpmv(A), x) for _, _, nint, A, x, _ in cpu_assemble()]
    dofs = sum(nint for nint, _, _ in legs)
    times = []
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        for _, op, x in legs:
            op(x, threads)
        if s >= args.warmup:
            times.append(time.perf_counter() - t0)
    ms = 1e3 * statistics.mean(times)
    value = dofs / (ms * 1e-3) / 1e6
    sample = ("reference macro, sin3 coefficient, Dirichlet: P1 at level 7 + P2 at level 6 (366,145 points each, "
              "the level-8 workload's operators at 1/8 of its size), FP64 CSR product on %d OpenMP threads" % threads)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "MDoF/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "reference macro-tetrahedron, variable-coefficient P1/P2 diffusion (bounded "
                                   "sample of the level-8 workload: P1 level 7, P2 level 6)"},
            "cpu_baseline": {"kind": "oracle", "cores": threads, "sample": sample, "value": value, "unit": "MDoF/s",
                             "host": host_cpu()},
            "e2e": {"value": value, "unit": "MDoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="hhg", choices=["hhg", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fmg-level", type=int, default=7)
    ap.add_argument("--no-fmg", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the constant-coefficient and epsilon legs")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    import workloads as W
    import paper_2404_08371_gb300 as hhg
    from paper_2404_08371_gb300 import _lib

    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    v, t = W.reference_tet()
    mesh = hhg.Mesh(v, t, LEVEL)
    legs = []
    for leg in LEGS:
        name, degree, coeff, qd, dt = leg
        op = hhg.Operator(mesh, degree=degree, coeff=coeff, bc="dirichlet", quad_degree=qd)
        x0 = torch.empty(mesh.vec_size(degree), dtype=torch.float64, device=dev)
        x0.copy_(torch.from_numpy(W.uniform(mesh.vec_size(degree), seed=0)))
        x = x0 if dt == "f64" else x0.float()
        y = torch.empty_like(x)
        tot, inner = mesh.dof_count(degree)
        legs.append({"name": name, "op": op, "x": x, "y": y, "dofs": inner, "npts": x.numel(),
                     "esize": x.element_size(), "dt": dt, "degree": degree,
                     "nq": 4 if qd == 2 else 14, "ms": []})
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def run_step(record: bool):
        for L in legs:
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            L["op"].apply(L["x"], out=L["y"])
            e1.record(stream)
            if record:
                L["ev"].append((e0, e1))

    for L in legs:
        L["ev"] = []
    for _ in range(args.warmup):
        run_step(False)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for _ in range(args.steps):
        run_step(True)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    clk = clocks.stop()
    step_ms = 0.0
    for L in legs:
        L["ms"] = [a.elapsed_time(b) for a, b in L["ev"]]
        step_ms += sum(L["ms"]) / args.steps
    dofs_step = sum(L["dofs"] for L in legs)
    step_ms, dofs_all, value = aggregate_replicas(step_ms, dofs_step, dev)
    # the same rate over the FP64 legs alone and over the FP32 legs alone
    value_by_dt = {}
    for dt in ("f64", "f32"):
        sel = [L for L in legs if L["dt"] == dt]
        if sel:
            value_by_dt[dt] = aggregate_replicas(sum(sum(L["ms"]) / args.steps for L in sel),
                                                 sum(L["dofs"] for L in sel), dev)[2]

    # end to end through the C-ABI with host buffers: pinned H2D of x, apply, D2H of y
    h2d = d2h = 0
    for L in legs:
        L["hx"] = L["x"].cpu().pin_memory()
        L["hy"] = torch.empty_like(L["hx"]).pin_memory()
        h2d += L["hx"].numel() * L["esize"]
        d2h += L["hy"].numel() * L["esize"]
    # End to end: every step copies each leg's x from pinned host memory and its y back, through the
    # public apply.  Copies run on their own streams, ordered by events around each apply, so they
    # overlap the other legs' applies.  The leg order is the one with the shortest modelled step
    # (copies in order on one stream per direction at the rates measured here, applies in order).
    big = max(legs, key=lambda L: L["hx"].numel())
    nbig = big["hx"].numel() * big["esize"]

    def copy_ms(fn):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    h2d_rate = nbig / copy_ms(lambda: big["x"].copy_(big["hx"], non_blocking=True))   # bytes per ms
    d2h_rate = nbig / copy_ms(lambda: big["hy"].copy_(big["y"], non_blocking=True))

    def modelled_ms(order):
        th = tc = td = 0.0
        for L in order:
            th += L["hx"].numel() * L["esize"] / h2d_rate
            tc = max(tc, th) + statistics.mean(L["ms"])
            td = max(td, tc) + L["hy"].numel() * L["esize"] / d2h_rate
        return td

    order = list(min(itertools.permutations(legs), key=modelled_ms))
    comp = torch.cuda.current_stream()
    h2d_s, d2h_s = torch.cuda.Stream(), torch.cuda.Stream()
    e2e_ms, e2e_apply_ms = [], []
    for s in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ready = []
        with torch.cuda.stream(h2d_s):
            for L in order:
                L["x"].copy_(L["hx"], non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(h2d_s)
                ready.append(ev)
        spans = []
        for L, ev in zip(order, ready):
            comp.wait_event(ev)
            a0 = torch.cuda.Event(enable_timing=True)
            a0.record(comp)
            L["op"].apply(L["x"], out=L["y"])
            done = torch.cuda.Event(enable_timing=True)
            done.record(comp)
            spans.append((a0, done))
            d2h_s.wait_event(done)
            with torch.cuda.stream(d2h_s):
                L["hy"].copy_(L["y"], non_blocking=True)
        torch.cuda.synchronize()
        if s >= args.warmup:
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
            e2e_apply_ms.append(sum(a.elapsed_time(b) for a, b in spans))
    _, _, e2e_value = aggregate_replicas(statistics.mean(e2e_ms), dofs_step, dev)
    e2e_detail = {"order": [L["name"] for L in order], "h2d_gbs": h2d_rate / 1e6, "d2h_gbs": d2h_rate / 1e6,
                  "modelled_ms": modelled_ms(order), "measured_ms": statistics.mean(e2e_ms),
                  "applies_ms": statistics.mean(e2e_apply_ms)}

    peaks = load_peaks()
    traffic = load_traffic()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    run_mhz = clk.get("sm_mhz") or clk.get("sm_max_mhz") or 2070.0
    alu_peak = {dt: alu_peak_tflops(dt, sms, run_mhz) for dt in FMA_PER_CLK_SM}
    details = {}
    dom = None
    for L in legs:
        ms = statistics.mean(L["ms"])
        nbytes = 2 * L["npts"] * L["esize"]          # read x, write y (algorithmic minimum)
        unit, fpu = flops_per_unit(L["name"], L["degree"], L["nq"])
        ntets = 8 ** LEVEL
        flops = fpu * (L["dofs"] if unit == "dof" else ntets)
        d = {"ms": ms, "mdofs": L["dofs"] / (ms * 1e-3) / 1e6, "gbs": nbytes / (ms * 1e-3) / 1e9,
             "hbm_frac": nbytes / (ms * 1e-3) / 1e9 / peaks["hbm_gbs"],
             "tflops": flops / (ms * 1e-3) / 1e12,
             "alu_frac": flops / (ms * 1e-3) / 1e12 / alu_peak[L["dt"]],
             "dofs": L["dofs"], "bytes": nbytes, "flops": flops}
        details[L["name"]] = d
        if dom is None or ms > details[dom]["ms"]:
            dom = L["name"]
    D = details[dom]
    dom_leg = [L for L in legs if L["name"] == dom][0]
    if D["alu_frac"] > D["hbm_frac"]:
        roof = {"bound": "alu", "achieved": D["tflops"], "peak": alu_peak[dom_leg["dt"]], "unit": "TFLOP/s",
                "frac": D["alu_frac"],
                "peak_src": "unit-count %s peak: %d FMA/clock/SM x 2 FLOP x %d SMs x %.0f MHz (median SM clock "
                            "sampled during the timed region)" % (dom_leg["dt"], FMA_PER_CLK_SM[dom_leg["dt"]], sms,
                                                                  run_mhz)}
    else:
        roof = {"bound": "hbm", "achieved": D["gbs"], "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": D["hbm_frac"],
                "peak_src": peaks["src"] + " (burst copy)"}
    tr = traffic.get(dom)
    roof["traffic"] = tr["bytes_per_launch"] if tr else None
    roof["kernel"] = dom

    extra = {}
    for L in legs:
        L["x"] = L["y"] = L["hx"] = L["hy"] = None
    torch.cuda.empty_cache()
    if not args.no_extra:
        extra["const_legs"] = run_const_legs(hhg, torch, flush, peaks["hbm_gbs"])
        torch.cuda.empty_cache()
        extra["coefficient_adjoint"] = run_adjoint(hhg, torch, flush, peaks["hbm_gbs"])
        torch.cuda.empty_cache()
        extra["epsilon"] = run_eps(hhg, torch, flush, alu_peak["f64"])
        torch.cuda.empty_cache()
        extra["n1"] = run_n1(hhg, torch, flush)
        torch.cuda.empty_cache()
        extra["under_integration"] = run_underint(hhg, torch, flush)
        torch.cuda.empty_cache()
        extra["precomputed"] = run_precomputed(hhg, torch, flush)
        torch.cuda.empty_cache()
    fmg = None
    if not args.no_fmg:
        del flush
        torch.cuda.empty_cache()
        fmg = run_fmg(hhg, torch, args.fmg_level)
        torch.cuda.empty_cache()
        fmg["n1"] = run_n1_fmg(hhg, torch)
    cb = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = cpu_baseline()
    # per apply on a single macro: the marching kernel, plus the Dirichlet-row kernel on lattices
    # whose marching tiles add their shared j-faces atomically (at least 64 cubes per edge)
    launches = sum(2 if 2 ** LEVEL >= 64 else 1 for _ in legs) * args.steps
    line = {"metric": METRIC, "value": value, "value_f64_legs": value_by_dt.get("f64"),
            "value_f32_legs": value_by_dt.get("f32"), "unit": "MDoF/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "+".join(sorted({L["dt"] for L in legs})), "data": "synthetic",
            "config": {"workload": "reference macro-tetrahedron at level %d, legs: %s" % (
                LEVEL, ", ".join(L["name"] for L in legs)), "level": LEVEL, "bc": "dirichlet",
                "l2": "flushed before every apply (512 MB write)", "parallelism": "replicas" if world > 1 else "1gpu"},
            "legs": details, "roofline": roof,
            "e2e": {"value": e2e_value, "unit": "MDoF/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "e2e_detail": e2e_detail,
            "gpu_launches": launches, "clocks": clk, "wall_s_timed": wall}
    line.update(extra)
    if fmg is not None:
        line["fmg"] = fmg
    if cb is not None:
        line["cpu_baseline"] = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")}
        for k in ("value_1thread", "host", "legs", "fmg"):
            line["cpu_baseline"][k] = cb[k]
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
