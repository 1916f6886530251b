"""Per-cell work counters of the benchmark workloads, from the oracle (harness script, run by hand and by a test).

Prints, for each workload of ``bench.py``, the means over a random sample of cells (seed 7) of
  n_cert  planes the oracle examines before the security-radius stop (certified mode: every site
          closer than twice the cell's largest vertex distance, plus the box walls),
  verts   vertices of the final cell,
  faces   facets of the final cell,
the three numbers of the algorithmic work W = n_cert * verts * 6 + verts * 40 + faces * 30 flops that the
benchmark divides by the clipping kernel's time.  Nothing here reads the CUDA path.

    python tests/work_per_cell.py [workload ...] [--sample 2048]
"""
import argparse
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def counters(name, n_sample, seed=7):
    import bench
    import oracle

    x, desc = bench.workload(name)
    N = len(x)
    pick = np.sort(np.random.default_rng(seed).choice(N, min(n_sample, N), replace=False))
    if "set_off" in desc:
        off = desc["set_off"]
        sid = np.searchsorted(off, pick, side="right") - 1
        parts = []
        for s in np.unique(sid):
            xs = x[off[s]:off[s + 1]].astype(np.float64)
            parts.append(oracle.cells(xs, -1.0, 1.0, False, which=pick[sid == s] - off[s], mode="certified"))
        cat = lambda k: np.concatenate([p[k] for p in parts])  # noqa: E731
    else:
        o = oracle.cells(x.astype(np.float64), 0.0, desc["L"], True, which=pick, mode="certified")
        cat = lambda k: o[k]  # noqa: E731
    return dict(n_cert=float(cat("ntest").mean()), verts=float(cat("nvert").mean()),
                faces=float(cat("nface").mean()), sample=len(pick))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("workloads", nargs="*",
                    default=["uniform4096", "clustered64k", "clustered2M", "clustered16M", "halosets4096"])
    ap.add_argument("--sample", type=int, default=2048)
    args = ap.parse_args()
    for w in args.workloads:
        c = counters(w, args.sample)
        print('"%s": {"n_cert": %.2f, "verts": %.2f, "faces": %.2f},  # %d cells'
              % (w, c["n_cert"], c["verts"], c["faces"], c["sample"]))


if __name__ == "__main__":
    main()
