"""Writes sinkhorn_ball3d_n2e4_eps0.02_it20.json: the FP64 oracle's Sinkhorn
value after 20 iterations (Alg. 1 from u = v = 1, every product an exact
matrix-free sum, Eqs. (matexp)/(matexpt)) on n = m = 20000 points uniform in
the radius-0.2 ball in R^3 (seeds 1 and 2, the input generators of the
library's workloads), uniform weights, r = 2, eps = 0.02.

It calls only oracle/ and the input generators.  Run from the repository root:
    python tests/golden/make_sinkhorn_ball3d_n2e4.py
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import sinkhorn as osk                      # noqa: E402
from paper_2201_07524_gb300 import workloads as wl      # noqa: E402

N, D, EPS, R, ITERS, SEED_X, SEED_Y = 20000, 3, 0.02, 2.0, 20, 1, 2


def main():
    x = wl.uniform_ball(N, D, 0.2, SEED_X)
    y = wl.uniform_ball(N, D, 0.2, SEED_Y)
    a, b = wl.uniform_weights(N), wl.uniform_weights(N)
    t0 = time.time()
    out = osk.sinkhorn_matrix_free(x, a, y, b, EPS, R, ITERS)
    rec = {
        "what": "oracle.sinkhorn.sinkhorn_matrix_free after %d iterations from u = v = 1" % ITERS,
        "n": N, "m": N, "d": D, "eps": EPS, "r": R, "iters": ITERS,
        "points": "workloads.uniform_ball(n, 3, 0.2, seed), seeds %d (x) and %d (y)" % (SEED_X, SEED_Y),
        "weights": "uniform",
        "s": out["s"], "err_row": out["err_row"], "err_col": out["err_col"],
        "u_head": [float(v) for v in out["u"][:8]], "v_head": [float(v) for v in out["v"][:8]],
        "oracle_seconds": round(time.time() - t0, 1),
    }
    with open(os.path.join(HERE, "sinkhorn_ball3d_n2e4_eps0.02_it20.json"), "w") as f:
        json.dump(rec, f, indent=1)
        f.write("\n")
    print(json.dumps(rec))


if __name__ == "__main__":
    main()
