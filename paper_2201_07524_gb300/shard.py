"""One fast summation sharded over ranks (one GPU per rank, torch.distributed).

The inner sum of Eq. (fastsum) is linear in the sources: the spectrum of all
sources, spec_k = sum_j w_j exp(-2 pi i k.z_j), is the sum over shards of each
shard's spectrum.  So every rank holds a plan with its own shard of the
sources and of the targets, all plans share one torus geometry, and one
product K w is

    sk_spectrum (own sources)  ->  all-reduce (sum) of the (N+1)^d spectrum
    ->  sk_apply_spectrum (own targets)

with the all-reduce the only exchange.  This module holds the host side of
that: the shared geometry (the rule sk_init applies to a single plan, taken
over the union of all shards) and the product's orchestration.  Every step of
the summation runs in the library; the collectives are torch.distributed
(NCCL between GPUs, gloo on the CPU).
"""
from . import sk as _sk


def shared_geometry(x_local, y_local, eps_B=0.1, group=None):
    """Center and scale of the torus coordinates z = scale (x - center) + 1/2
    shared by all shards: center = midpoint of the bounding box of every
    rank's points, scale = (1/4 - eps_B/2) / R with R the largest distance of
    a point to the center (the automatic geometry of sk_init, over the union).
    x_local (n x d) and y_local (m x d) are float64 tensors; returns
    (center as a list of 3 floats, scale)."""
    import torch
    import torch.distributed as dist
    pts = torch.cat([x_local, y_local]).to(torch.float64)
    d = pts.shape[1]
    lo = pts.min(0).values.clone()
    hi = pts.max(0).values.clone()
    if dist.is_initialized():
        dist.all_reduce(lo, op=dist.ReduceOp.MIN, group=group)
        dist.all_reduce(hi, op=dist.ReduceOp.MAX, group=group)
    c = 0.5 * (lo + hi)
    r = torch.sqrt(((pts - c) ** 2).sum(1)).max().reshape(1).clone()
    if dist.is_initialized():
        dist.all_reduce(r, op=dist.ReduceOp.MAX, group=group)
    R = float(r.item())
    if not R > 0.0:
        R = 1.0
    center = [float(v) for v in c.tolist()] + [0.0] * (3 - d)
    return center, (0.25 - 0.5 * eps_B) / R


def shard_params(center, scale, **overrides):
    """sk_nfft_params for a shard's plan: the library defaults with the shared
    geometry fixed (user_geometry = 1) and the given overrides."""
    prm = _sk.sk_default_params(**overrides)
    prm.user_geometry = 1
    prm.scale = float(scale)
    for t in range(3):
        prm.center[t] = float(center[t])
    return prm


class LibraryOps:
    """The library's stage calls on device tensors (the production path)."""

    @staticmethod
    def spectrum_size(plan):
        return _sk.spectrum_size(plan)

    @staticmethod
    def spectrum(plan, which, w, spec):
        _sk.sk_spectrum(plan, which, w, spec)

    @staticmethod
    def apply(plan, which, spec, out):
        _sk.sk_apply_spectrum(plan, which, spec, out)


def sharded_kernel_apply(plan, w, out, transpose=False, group=None, ops=LibraryOps):
    """out = K w at this rank's targets, with the sources of K spread over the
    ranks of `group`: transpose = False gives (K v) at the shard's x-points
    from weights v on its y-points, transpose = True gives (K^T u) at its
    y-points from u on its x-points.  w and out are float64 tensors on the
    plan's device, in the shard's own point order.  One all-reduce of the
    (N+1)^d complex spectrum (2 (N+1)^d doubles) per product."""
    import torch
    import torch.distributed as dist
    src, dst = (_sk.SK_SET_X, _sk.SK_SET_Y) if transpose else (_sk.SK_SET_Y, _sk.SK_SET_X)
    spec = torch.empty(2 * ops.spectrum_size(plan), dtype=torch.float64, device=w.device)
    ops.spectrum(plan, src, w, spec)
    if dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(spec, op=dist.ReduceOp.SUM, group=group)
    ops.apply(plan, dst, spec, out)
    return out
