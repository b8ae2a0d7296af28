"""DRAM traffic per launch of the kernel each bench leg times, written to profiles/traffic.json.

    python -m paper_2404_08371_gb300.capture_traffic [--out PATH] [leg ...]

For every leg: the plain profile_apply command runs first and must exit 0; then ncu captures the
second launch of the leg's kernel (the first is the warm-up; profile_apply flushes L2 before it)
with three metrics (DRAM bytes read and written, duration), one pass, clocks left alone.  Each entry
carries the sha256 of the kernel's sources, so bench.py drops it once those sources change.
"""
from __future__ import annotations

import csv
import hashlib
import io
import json
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
OUT = os.path.join(ROOT, "profiles", "traffic.json")
MARCH = ["paper_2404_08371_gb300/csrc/march_kernel.cuh", "paper_2404_08371_gb300/csrc/hhg_internal.h",
         "paper_2404_08371_gb300/csrc/lattice.cuh"]
OPS = ["paper_2404_08371_gb300/csrc/ops.cu", "paper_2404_08371_gb300/csrc/hhg_internal.h",
       "paper_2404_08371_gb300/csrc/lattice.cuh"]

# leg: (kernel name pattern, launches per apply to sum, profile_apply arguments, sources, workload)
LEGS = {
    "p2_sin3_f64": ("march_kernel", 1, "--level 8 --degree 2 --coeff sin3 --dtype f64", MARCH, "reference macro, level 8"),
    "p1_sin3_f64": ("march_kernel", 1, "--level 8 --degree 1 --coeff sin3 --dtype f64", MARCH, "reference macro, level 8"),
    "p2_sin3_f32": ("march_kernel", 1, "--level 8 --degree 2 --coeff sin3 --dtype f32", MARCH, "reference macro, level 8"),
    "p1_sin3_f32": ("march_kernel", 1, "--level 8 --degree 1 --coeff sin3 --dtype f32", MARCH, "reference macro, level 8"),
    "p2_const_f64": ("p2_tile_kernel", 1, "--level 8 --degree 2 --coeff const --dtype f64", OPS, "reference macro, level 8"),
    "p2_const_f32": ("p2_quad_kernel", 1, "--level 8 --degree 2 --coeff const --dtype f32", OPS, "reference macro, level 8"),
    "p1_const_f64": ("p1_gather_kernel", 1, "--level 9 --degree 1 --coeff const --dtype f64", OPS,
                     "reference macro, level 9"),
    "p1_const_df64": ("split_double_kernel|p1_gather_df_kernel", 2,
                      "--level 9 --degree 1 --coeff const --dtype f64 --fp64-arith double_float", OPS,
                      "reference macro, level 9"),
    "p2_const_df64": ("split_double_kernel|p2_quad_kernel", 2,
                      "--level 8 --degree 2 --coeff const --dtype f64 --fp64-arith double_float", OPS,
                      "reference macro, level 8"),
    "p1_const_f32": ("p1_climb_f32_kernel", 1, "--level 9 --degree 1 --coeff const --dtype f32", OPS,
                     "reference macro, level 9"),
    "n1_f64": ("march_kernel", 1, "--mesh cuboid36 --level 7 --kind curlcurl --coeff field_p1 --dtype f64", MARCH,
               "3x2x1 cuboid as 36 macros, level 7"),
}


def sources_sha256(files) -> str:
    h = hashlib.sha256()
    for fn in files:
        with open(os.path.join(ROOT, fn), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def capture(leg: str) -> dict:
    pattern, launches, args, files, workload = LEGS[leg]
    cmd = [sys.executable, "-m", "paper_2404_08371_gb300.profile_apply", "--reps", "1", "--warmup", "1"] + args.split()
    subprocess.run(cmd, check=True, cwd=ROOT, capture_output=True)   # the plain run must exit 0 first
    log = os.path.join(ROOT, "gpurun_out", "traffic_%s.csv" % leg)
    os.makedirs(os.path.dirname(log), exist_ok=True)
    ncu = ["ncu", "--metrics", "dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum",
           "--clock-control", "none", "-s", str(launches), "-c", str(launches), "--csv", "-k",
           "regex:" + pattern, "--log-file", log] + cmd
    subprocess.run(ncu, check=True, cwd=ROOT, capture_output=True)
    text = open(log).read()
    rows = list(csv.reader(io.StringIO(text[text.index('"ID"'):])))
    head = rows[0]
    ki, mi, ui, vi = head.index("Kernel Name"), head.index("Metric Name"), head.index("Metric Unit"), head.index("Metric Value")
    scale = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "B": 1.0, "KB": 1e3, "MB": 1e6, "GB": 1e9,
             "nsecond": 1e-6, "usecond": 1e-3, "msecond": 1.0, "ns": 1e-6, "us": 1e-3, "ms": 1.0}
    tot = {"dram__bytes_read.sum": 0.0, "dram__bytes_write.sum": 0.0, "gpu__time_duration.sum": 0.0}
    names = []
    for r in rows[1:]:
        if r[mi] in tot:
            tot[r[mi]] += float(r[vi].replace(",", "")) * scale[r[ui]]
        if r[ki] not in names:
            names.append(r[ki])
    return {"bytes_per_launch": int(tot["dram__bytes_read.sum"] + tot["dram__bytes_write.sum"]),
            "read": int(tot["dram__bytes_read.sum"]), "write": int(tot["dram__bytes_write.sum"]),
            "ncu_ms": tot["gpu__time_duration.sum"], "kernel": " + ".join(n.split("(")[0] for n in names),
            "workload": workload, "sources": files, "sources_sha256": sources_sha256(files)}


def main(argv):
    out = OUT
    if argv[:1] == ["--out"]:
        out, argv = argv[1], argv[2:]
    table = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for leg in argv or list(LEGS):
        table[leg] = capture(leg)
        print(leg, json.dumps(table[leg]))
        with open(out, "w") as f:   # after every leg: a later failure keeps the earlier captures
            json.dump(table, f, indent=1)


if __name__ == "__main__":
    main(sys.argv[1:])
