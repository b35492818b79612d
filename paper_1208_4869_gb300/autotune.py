"""Measure launch choices on the GPU and write csrc/tune_table.h.

For every precision (complex64, complex128), method of the persistent
launch (BiCGSTAB, CGNR, QMR, COCG) and order n in a ladder of sizes, times a
fixed number of iterations (tol = 0) of one solve on the synthetic dense
system of the benchmark's recipe with each candidate:

  * the kernel-per-step loop (CCG_OPT_PERSISTENT = 0),
  * one persistent launch with 1, 2, or the occupancy limit of blocks per SM,

and keeps the fastest (the loop unless a persistent form beats it by the
margin below).  Adjacent sizes with the same choice merge into one entry of
the table (n <= nmax).  Both forms compute bitwise the same result, so the
table only moves time.

    python -m paper_1208_4869_gb300.autotune            # print the table
    python -m paper_1208_4869_gb300.autotune --write    # and regenerate tune_table.h
"""
import argparse
import json
import os
import statistics
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
TABLE = os.path.join(HERE, "csrc", "tune_table.h")

SIZES = [128, 256, 512, 1024, 2048, 4096, 8192]
METHODS = [("bicgstab", 0, False), ("cgnr", 1, False), ("qmr", 2, False), ("cocg", 3, True)]
CANDIDATES = [(0, 0), (1, 1), (1, 2), (1, 0)]   # (persistent, blocks per SM; 0 = occupancy limit)
MARGIN = 0.03       # a persistent form must be this much faster than the loop


def measure(ccg, torch, W, dtype, method, sym, n, iters, reps):
    A, y = W.dense_system(n, 3.0, 0)
    if sym:
        A = (A + A.T) / 2
    tdt = torch.complex128 if dtype == 1 else torch.complex64
    Ad = torch.from_numpy(A).cuda().to(tdt)
    yd = torch.from_numpy(y).cuda().to(tdt)
    out = {}
    for pers, blocks in CANDIDATES:
        h = ccg.Handle()
        h.set_option(ccg.OPT_PERSISTENT, pers)
        h.set_option(ccg.OPT_PK_BLOCKS, blocks)
        op = h.op_dense(Ad, symmetric=sym)
        xd = torch.zeros_like(yd)
        h.solve(method, op, yd, xd, tol=0.0, maxit=iters, want_hist=False, want_info=False)   # warm
        ts = []
        for _ in range(reps):
            xd.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            h.solve(method, op, yd, xd, tol=0.0, maxit=iters, want_hist=False, want_info=False)
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
        out[(pers, blocks)] = statistics.median(ts) / iters
        del op, h
    return out


def choose(times):
    loop = times[(0, 0)]
    best = min(((t, c) for c, t in times.items() if c[0] == 1), default=(None, None))
    if best[0] is not None and best[0] < (1.0 - MARGIN) * loop:
        return best[1]
    return (0, 0)


def table_text(entries, device):
    lines = ["// Launch choices measured on the GPU by paper_1208_4869_gb300/autotune.py",
             "// (rerun it with --write to regenerate this file; measured on %s)." % device,
             "// Each entry: for solves of precision `dtype` (CCG_C64 / CCG_C128) by",
             "// `method` on a dense operator of order n <= nmax (the first matching entry",
             "// wins), whether the solve runs as one persistent launch (1) or as the",
             "// kernel-per-step loop (0), and the persistent launch's blocks per SM (0:",
             "// the occupancy limit).",
             "#pragma once", "", "namespace ccg {", "",
             "struct TuneEntry {", "  int dtype, method;", "  long long nmax;", "  int persistent, pk_blocks;", "};",
             "", "static const TuneEntry kTune[] = {"]
    for e in entries:
        lines.append("    {%d, %d, %d, %d, %d},   // %s" % e)
    if not entries:
        lines.append("    {-1, -1, 0, 0, 0},")
    lines += ["};", "", "}  // namespace ccg", ""]
    return "\n".join(lines)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--write", action="store_true", help="regenerate csrc/tune_table.h")
    ap.add_argument("--out", default=None, help="write the table here instead of csrc/tune_table.h")
    ap.add_argument("--iters", type=int, default=30)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--sizes", default=",".join(map(str, SIZES)))
    a = ap.parse_args(argv)
    import torch
    sys.path.insert(0, os.path.dirname(HERE))
    from paper_1208_4869_gb300 import build as B
    B.build()
    from paper_1208_4869_gb300 import ccg
    from paper_1208_4869_gb300 import workloads as W
    sizes = [int(s) for s in a.sizes.split(",")]
    device = torch.cuda.get_device_name(0)
    entries = []
    for dtype, dname in ((0, "complex64"), (1, "complex128")):
        for mname, mcode, sym in METHODS:
            picks = []
            for n in sizes:
                times = measure(ccg, torch, W, dtype, mname, sym, n, a.iters, a.reps)
                c = choose(times)
                picks.append((n, c))
                print(json.dumps({"dtype": dname, "method": mname, "n": n, "choice": c,
                                  "us_per_iteration": {"%d/%d" % k: round(1e6 * v, 2) for k, v in times.items()}}),
                      flush=True)
            entries += merge(picks, dtype, mcode, "%s %s" % (dname, mname))
    text = table_text(entries, device)
    print(text)
    if a.write:
        with open(a.out or TABLE, "w") as fh:
            fh.write(text)
    return 0


def merge(picks, dtype, mcode, label):
    """Runs of equal choices over the size ladder as n <= nmax entries; the
    largest size's choice holds beyond the ladder."""
    out = []
    for i, (n, c) in enumerate(picks):
        last = i + 1 == len(picks)
        if last or picks[i + 1][1] != c:
            out.append((dtype, mcode, (1 << 62) if last else n, c[0], c[1],
                        "%s n <= %s" % (label, "any" if last else n)))
    return out


if __name__ == "__main__":
    sys.exit(main())
