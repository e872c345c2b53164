"""The Sinkhorn value at the headline workload's settings against the FP64
oracle (Alg. 3 result line; Alg. 1 with exact sums).

n = m = 20000 points uniform in the radius-0.2 ball in R^3, uniform weights,
r = 2, eps = 0.02, 20 iterations from u = v = 1, the library's default
parameters (N = 64, sigma = 2, m_w = 4, FP32 fast summation, FP64 updates):
the same settings as the 1e6-point benchmark at a size the oracle finishes.
The oracle's value is stored in tests/golden/ by a script that calls only
oracle/.  Both GPU methods -- the NFFT fast summation and the direct sums
(FP32 kernel values, FP64 across tiles) -- must match it to 1e-5 relative,
which makes the direct method a checked reference for the full-size
comparison the benchmark prints.
"""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2201_07524_gb300 import workloads as wl   # noqa: E402

sk = pytest.importorskip("paper_2201_07524_gb300.sk")

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "sinkhorn_ball3d_n2e4_eps0.02_it20.json")
TOL_S = 1e-5


@pytest.fixture(scope="module")
def golden():
    with open(GOLDEN) as f:
        return json.load(f)


@pytest.mark.parametrize("method", ["nfft", "direct"])
def test_value_at_2e4_matches_fp64_oracle(golden, method):
    g = golden
    x = wl.uniform_ball(g["n"], g["d"], 0.2, 1)
    y = wl.uniform_ball(g["m"], g["d"], 0.2, 2)
    a, b = wl.uniform_weights(g["n"]), wl.uniform_weights(g["m"])
    T = lambda z: torch.as_tensor(z, dtype=torch.float64, device="cuda")
    plan = sk.sk_init(T(x), T(a), T(y), T(b), g["eps"], g["r"], sk.sk_default_params())
    info = sk.sk_plan_info(plan)
    assert (info["N"], info["m_w"], info["precision"]) == (64, 4, sk.SK_FP32)
    if method == "direct":
        sk.sk_set_method(plan, sk.SK_METHOD_DIRECT)
    u = np.zeros(g["n"])
    v = np.zeros(g["m"])
    st, res = sk.sk_solve(plan, g["iters"], u_out=u, v_out=v)
    plan.close()
    rel = abs(res["s"] - g["s"]) / abs(g["s"])
    assert rel <= TOL_S, (method, res["s"], g["s"], rel)
    # the state itself: the first scaling values in caller order
    assert np.allclose(u[:8], g["u_head"], rtol=1e-4, atol=0)
    assert np.allclose(v[:8], g["v_head"], rtol=1e-4, atol=0)
    # the oracle's state is converged (row residual of Eq. (Error) ~1e-14 of
    # ||a||); the GPU state is too, to the precision of its FP32 sums
    assert g["err_row"] <= 1e-10 * np.linalg.norm(a)
    assert res["err_row"] <= 1e-5 * np.linalg.norm(a)
