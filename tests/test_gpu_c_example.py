"""The C ABI from plain C: the example program (built next to the library)
solves a small problem with host buffers; its value matches the FP64 oracle's
on the same points (relative error <= 1e-5, the Sinkhorn-value target)."""
import os
import subprocess

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from oracle import sinkhorn as osk   # noqa: E402


def lcg_ball_points(state, n, d):
    """The example's generator: 64-bit LCG, top 53 bits as a uniform double,
    rejection in the cube [-0.2, 0.2]^d."""
    pts = np.zeros((n, d))
    for i in range(n):
        while True:
            r2 = 0.0
            for t in range(d):
                state = (state * 6364136223846793005 + 1442695040888963407) % (1 << 64)
                pts[i, t] = 0.4 * ((state >> 11) * (1.0 / 9007199254740992.0)) - 0.2
                r2 += pts[i, t] * pts[i, t]
            if r2 <= 0.04:
                break
    return pts, state


@pytest.mark.parametrize("d,n,m,eps", [(2, 700, 600, 0.05), (3, 900, 800, 0.02)])
def test_c_example_matches_oracle(d, n, m, eps):
    from paper_2201_07524_gb300 import build
    exe = build.build_example()
    out = subprocess.run([exe, str(d), str(n), str(m), str(eps), "30"], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    vals = dict(line.split() for line in out.stdout.strip().splitlines())
    x, state = lcg_ball_points(12345, n, d)
    y, _ = lcg_ball_points(state, m, d)
    ref = osk.sinkhorn_dense(x, np.full(n, 1.0 / n), y, np.full(m, 1.0 / m), eps, 2.0, 30)
    assert abs(float(vals["s"]) - ref["s"]) <= 1e-5 * abs(ref["s"])
    assert int(vals["iters"]) == 30
