"""Run a few applies of one operator configuration (for timing by hand or under a profiler).

    python -m paper_2404_08371_gb300.profile_apply --mesh reference_tet --level 9 --degree 1 \
        --coeff const --dtype f64 --reps 3

Prints the mean CUDA-event time per apply and the derived MDoF/s and GB/s
(read x + write y).  The L2 is flushed (512 MB write) before every apply.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--mesh", default="reference_tet")
    ap.add_argument("--level", type=int, default=8)
    ap.add_argument("--degree", type=int, default=1)
    ap.add_argument("--kind", default="diffusion")
    ap.add_argument("--coeff", default="const")
    ap.add_argument("--quad", type=int, default=0)
    ap.add_argument("--dtype", default="f64")
    ap.add_argument("--bc", default="dirichlet")
    ap.add_argument("--nrhs", type=int, default=1)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=1)
    ap.add_argument("--op", default="apply", choices=["apply", "adjoint", "diagonal", "mg"])
    ap.add_argument("--mixed", type=int, default=1, help="--op mg: FP32 cycles inside FP64 refinement (1) or all FP64 (0)")
    ap.add_argument("--fp64-arith", default="native", choices=["native", "double_float"],
                    help="arithmetic of FP64 applies (double_float: P1 and P2 constant coefficient)")
    args = ap.parse_args()

    import torch
    import workloads as W
    import paper_2404_08371_gb300 as hhg

    v, t = getattr(W, args.mesh)()
    mesh = hhg.Mesh(v, t, args.level)
    dt = torch.float64 if args.dtype == "f64" else torch.float32
    qd = args.quad or (2 if args.degree == 1 else 4)
    field = None
    if args.kind == "curlcurl":
        coeff = None
    elif args.coeff == "const":
        coeff = ("const", 1.0)
    elif args.coeff == "sin3":
        coeff = ("sin3",)
    else:
        kdeg = 1 if args.coeff == "field_p1" else 2
        field = torch.from_numpy(1.0 + 0.5 * W.uniform(mesh.vec_size(kdeg), seed=7)).to("cuda", dt)
        mesh.make_consistent(field, kdeg)
        coeff = (args.coeff, field)
    if args.kind == "curlcurl":
        if args.coeff == "field_p1":
            a = torch.from_numpy(1.0 + 0.5 * W.uniform(mesh.vec_size(1), seed=8)).to("cuda", dt)
            b = torch.from_numpy(1.0 + 0.5 * W.uniform(mesh.vec_size(1), seed=9)).to("cuda", dt)
            mesh.make_consistent(a, 1)
            mesh.make_consistent(b, 1)
            op = hhg.CurlCurl(mesh, ("field_p1", a), ("field_p1", b), bc=args.bc)
        else:
            op = hhg.CurlCurl(mesh, ("const", 1.0), ("const", 1.0), bc=args.bc)
        args.degree = 2
    else:
        op = hhg.Operator(mesh, kind=args.kind, degree=args.degree, coeff=coeff, bc=args.bc, quad_degree=qd)
        if args.fp64_arith != "native":
            op.set_fp64_arith(args.fp64_arith)
    ncomp = 3 if args.kind == "epsilon" else 1
    n = mesh.vec_size(args.degree) * ncomp * args.nrhs
    x = torch.from_numpy(W.uniform(n, seed=0)).to("cuda", dt)
    mesh.make_consistent(x, args.degree, per_point=ncomp * args.nrhs)
    g = torch.from_numpy(W.uniform(n, seed=1)).to("cuda", dt)
    mesh.make_consistent(g, args.degree, per_point=ncomp * args.nrhs)
    y = torch.empty_like(x)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    if args.op == "mg":
        # FMG + V(2,2) solve of the manufactured Poisson problem (the operator must be DIRICHLET diffusion)
        b = mesh.rhs_sin3_poisson(args.degree)
        for _ in range(args.warmup):
            op.mg_solve(b, torch.zeros_like(b), mixed=args.mixed)
        sts = [op.mg_solve(b, torch.zeros_like(b), mixed=args.mixed)[1] for _ in range(args.reps)]
        print(json.dumps({"config": vars(args), "solve_ms": [st["solve_ms"] for st in sts],
                          "iterations": sts[-1]["iterations"], "rel_residual": sts[-1]["rel_residual"]}))
        return

    def once():
        if args.op == "apply":
            op.apply(x, out=y, nrhs=args.nrhs)
        elif args.op == "adjoint":
            op.adjoint_coeff(u=x, g=g, nrhs=args.nrhs)
        else:
            op.diagonal(dt)

    for _ in range(args.warmup):
        once()
    ms = []
    for _ in range(args.reps):
        flush.fill_(0.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        once()
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    tot, inner = mesh.dof_count(args.degree)
    mean = sum(ms) / len(ms)
    nbytes = 2 * n * x.element_size()
    print(json.dumps({"config": vars(args), "ms": mean, "ms_all": ms, "mdofs": inner * ncomp * args.nrhs / mean / 1e3,
                      "gbs_rw": nbytes / mean / 1e6, "points": n, "interior_dofs": inner}))


if __name__ == "__main__":
    main()
