"""Host side of the sharded product (paper_2201_07524_gb300/shard.py) on two
gloo ranks, without a GPU.

The linearity of the inner sum of Eq. (fastsum) is what the sharding rests
on: the spectrum of all sources is the sum of the shards' spectra.  Here each
rank's spectrum and outer sum are the oracle's exact trigonometric sums
(oracle.fastsum.adjoint_ndft / ndft with the oracle's b_k) in place of the
library's sk_spectrum / sk_apply_spectrum, so what is tested is the wiring:
the shared geometry, the all-reduce of the spectra, and that every rank's
values equal the unsharded Eq. (fastsum) at its own targets.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")

D, N, EPS, R, EPS_B, P = 2, 64, 0.05, 2.0, 0.1, 8


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _points():
    from paper_2201_07524_gb300 import workloads as wl
    x = wl.uniform_ball(401, D, 0.2, 61) + np.array([0.05, -0.02])
    y = wl.uniform_ball(303, D, 0.2, 62)
    v = wl.positive_vector(303, 63)
    return x, y, v


class _Shard:
    """A rank's shard in torus coordinates (the stand-in for its plan)."""

    def __init__(self, x, y, center, scale):
        from oracle import fastsum as ofs
        self.zx = ofs.torus_coordinates(x, center, scale)
        self.zy = ofs.torus_coordinates(y, center, scale)
        self.b = ofs.fourier_coefficients(N, D, EPS * scale ** R, R, 0.5 - EPS_B, P)


class _OracleOps:
    """The library's stage calls replaced by the oracle's exact sums; spectra
    over I_N as interleaved (re, im) doubles in a CPU tensor."""

    @staticmethod
    def spectrum_size(plan):
        return N ** D

    @staticmethod
    def spectrum(plan, which, w, spec):
        from oracle import fastsum as ofs
        from paper_2201_07524_gb300 import sk
        z = plan.zy if which == sk.SK_SET_Y else plan.zx
        h = ofs.adjoint_ndft(z, w.numpy(), N).reshape(-1)
        spec.copy_(torch.from_numpy(np.stack([h.real, h.imag], axis=-1).reshape(-1)))

    @staticmethod
    def apply(plan, which, spec, out):
        from oracle import fastsum as ofs
        from paper_2201_07524_gb300 import sk
        z = plan.zx if which == sk.SK_SET_X else plan.zy
        s = spec.numpy().reshape(-1, 2)
        h = (s[:, 0] + 1j * s[:, 1]).reshape((N,) * D)
        out.copy_(torch.from_numpy(ofs.ndft(z, plan.b * h, N).real))


def _rank(rank, world, port, results):
    import sys
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2201_07524_gb300 import shard
        x, y, v = _points()
        xs, ys, vs = x[rank::world], y[rank::world], v[rank::world]
        center, scale = shard.shared_geometry(torch.from_numpy(xs), torch.from_numpy(ys), EPS_B)
        plan = _Shard(xs, ys, center, scale)
        out = torch.zeros(len(xs), dtype=torch.float64)
        shard.sharded_kernel_apply(plan, torch.from_numpy(vs), out, ops=_OracleOps)
        results[rank] = (center, scale, out.numpy().tolist())
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_sum_spectra_into_the_unsharded_product():
    import torch.multiprocessing as mp
    from oracle import fastsum as ofs
    from oracle import sinkhorn as osk
    from paper_2201_07524_gb300 import build
    build.build()                      # shard.py loads the library (no GPU call is made)
    world, port = 2, _free_port()
    results = mp.get_context("spawn").Manager().dict()
    mp.start_processes(_rank, args=(world, port, results), nprocs=world, join=True, start_method="spawn")
    assert sorted(results.keys()) == [0, 1]
    x, y, v = _points()
    # the shared geometry is sk_init's automatic rule over the union of all points
    pts = np.concatenate([x, y])
    c = 0.5 * (pts.min(0) + pts.max(0))
    scale = (0.25 - 0.5 * EPS_B) / np.max(np.linalg.norm(pts - c, axis=1))
    for r in range(world):
        cr, sr, t = results[r]
        t = np.asarray(t)
        assert np.allclose(cr[:D], c, rtol=0, atol=1e-15) and cr[D:] == [0.0] * (3 - D)
        assert sr == pytest.approx(scale, rel=1e-14)
        # every rank: the unsharded Eq. (fastsum) over all sources at its own targets
        want = ofs.fastsum(x[r::world], y, v, EPS, R, N, list(c) + [0.0], scale, EPS_B, P)
        assert np.max(np.abs(t - want)) <= 1e-12 * np.max(np.abs(want))
        # and, within the kernel approximation, the exact product
        exact = osk.kernel_apply(x[r::world], y, v, EPS, R)
        assert np.max(np.abs(t - exact)) <= 1e-6 * np.max(exact)
