"""The sharded product's entry points, sk_spectrum and sk_apply_spectrum, on
one GPU through the C ABI.

Two shard plans (alternate sources and targets of one problem, the shared
torus geometry) stand in for two ranks; their spectra are summed here where
the ranks would all-reduce them.  Checked: the sum of the shards' spectra
equals the unsharded plan's spectrum (linearity of the inner sum of
Eq. (fastsum)), and each shard's product from the summed spectrum meets the
fast-summation tolerance of the other parity tests against the oracle's exact
sums (E_fs <= 1e-6 FP64, <= 1e-5 FP32).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import sinkhorn as osk                    # noqa: E402
from paper_2201_07524_gb300 import workloads as wl   # noqa: E402

sk = pytest.importorskip("paper_2201_07524_gb300.sk")
shard = pytest.importorskip("paper_2201_07524_gb300.shard")

TOL_FS = {sk.SK_FP64: 1e-6, sk.SK_FP32: 1e-5}
TOL_SPEC = {sk.SK_FP64: 1e-12, sk.SK_FP32: 1e-6}


def cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


@pytest.mark.parametrize("precision", [sk.SK_FP32, sk.SK_FP64])
@pytest.mark.parametrize("d", [2, 3])
def test_shard_spectra_sum_to_the_unsharded_product(d, precision):
    x = wl.uniform_ball(2501, d, 0.2, 71)
    y = np.concatenate([wl.uniform_ball(1700, d, 0.2, 72), 0.05 + 0.01 * np.random.default_rng(73).standard_normal((300, d))])
    v = wl.positive_vector(len(y), 74)
    eps, world = 0.02, 2
    center, scale = shard.shared_geometry(cuda(x), cuda(y), 0.1)
    prm = shard.shard_params(center, scale, precision=precision)

    def plan(xs, ys):
        return sk.sk_init(cuda(xs), cuda(wl.uniform_weights(len(xs))), cuda(ys), cuda(wl.uniform_weights(len(ys))),
                          eps, 2.0, prm)

    full = plan(x, y)
    size = 2 * sk.spectrum_size(full)
    spec_full = torch.zeros(size, dtype=torch.float64, device="cuda")
    sk.sk_spectrum(full, sk.SK_SET_Y, cuda(v), spec_full)
    shards = [plan(x[r::world], y[r::world]) for r in range(world)]
    total = torch.zeros(size, dtype=torch.float64, device="cuda")
    for r, p in enumerate(shards):
        spec = torch.zeros(size, dtype=torch.float64, device="cuda")
        sk.sk_spectrum(p, sk.SK_SET_Y, cuda(v[r::world]), spec)
        total += spec                       # the all-reduce of the ranks
    err = (total - spec_full).abs().max().item() / np.sum(v)
    assert err <= TOL_SPEC[precision], err
    for r, p in enumerate(shards):
        t = torch.zeros(len(x[r::world]), dtype=torch.float64, device="cuda")
        sk.sk_apply_spectrum(p, sk.SK_SET_X, total, t)
        exact = osk.kernel_apply(x[r::world], y, v, eps, 2.0)
        e_fs = np.max(np.abs(t.cpu().numpy() - exact)) / np.max(exact)
        assert e_fs <= TOL_FS[precision], (r, e_fs)
    for p in shards + [full]:
        p.close()


def test_sharded_product_refuses_near_field_kernels():
    x = wl.uniform_ball(300, 3, 0.2, 75)
    y = wl.uniform_ball(200, 3, 0.2, 76)
    p = sk.sk_init(cuda(x), cuda(wl.uniform_weights(300)), cuda(y), cuda(wl.uniform_weights(200)), 0.02, 1.0,
                   sk.sk_default_params())
    spec = torch.zeros(2 * sk.spectrum_size(p), dtype=torch.float64, device="cuda")
    with pytest.raises(sk.SkError) as err:
        sk.sk_spectrum(p, sk.SK_SET_Y, cuda(np.ones(200)), spec)
    assert err.value.status == sk.SK_ERR_UNSUPPORTED
    p.close()
