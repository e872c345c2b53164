"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances (stated in the tests below):
  * fast summation E_fs = max_i |t_i - t_i^exact| / max_i |t_i^exact|:
    <= 1e-6 for the FP64 path, <= 1e-5 for the FP32 path;
  * Sinkhorn value s: relative error <= 1e-5;
  * stage entry points (adjoint NFFT, NFFT): max error <= 1e-6 (FP64) /
    1e-5 (FP32) relative to the l1 norm of their input, the scale of the
    Kaiser-Bessel window error with m = 4, sigma = 2;
  * Fourier coefficients b_k: both sides sample K_R in FP64 and take its DFT;
    the boundary polynomial's coefficients come from two independent FP64
    linear solves whose rounding differs, so agreement to 1e-10 of max |b_k|;
  * direct summation: FP64 1e-12 per element; FP32 1e-5 per element (FP32
    coordinates carry ~6e-8 relative rounding, amplified by |d K / d x|).
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import fastsum as ofs          # noqa: E402
from oracle import sinkhorn as osk         # noqa: E402
from paper_2201_07524_gb300 import workloads as wl   # noqa: E402

sk = pytest.importorskip("paper_2201_07524_gb300.sk")

DEV = "cuda"


def cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=DEV)


def plan_for(x, y, a=None, b=None, eps=0.05, r=2.0, precision=sk.SK_FP64, user_geometry=True, **kw):
    n, m = len(x), len(y)
    a = wl.uniform_weights(n) if a is None else a
    b = wl.uniform_weights(m) if b is None else b
    prm = sk.sk_default_params(precision=precision, **kw)
    if user_geometry:
        prm.user_geometry = 1
        prm.scale = 1.0
        for t in range(3):
            prm.center[t] = 0.0
    return sk.sk_init(cuda(x), cuda(a), cuda(y), cuda(b), eps, r, prm)


def efs(t, exact):
    return float(np.max(np.abs(t - exact)) / np.max(np.abs(exact)))


TOL_FS = {sk.SK_FP64: 1e-6, sk.SK_FP32: 1e-5}


# --------------------------------------------------------- coefficients
@pytest.mark.parametrize("d,N,eps", [(1, 64, 0.05), (2, 64, 0.05), (3, 32, 0.02), (2, 128, 0.01)])
def test_fourier_coefficients_match_oracle(d, N, eps):
    x = wl.uniform_ball(50, d, 0.2, 1)
    y = wl.uniform_ball(60, d, 0.2, 2)
    plan = plan_for(x, y, eps=eps, N=N)
    got = np.zeros((N,) * d)
    sk.sk_fourier_coefficients(plan, got)
    want = ofs.fourier_coefficients(N, d, eps, 2.0, 0.4, 8)
    assert np.max(np.abs(got - want)) <= 1e-10 * np.max(np.abs(want))


def test_fourier_coefficients_follow_auto_scaling():
    # automatic geometry: the kernel in torus coordinates is exp(-rho^r / (eps scale^r))
    d, N, eps = 2, 64, 0.05
    x = wl.uniform_ball(300, d, 0.2, 3) + 0.7
    y = wl.uniform_ball(200, d, 0.2, 4) + 0.7
    plan = plan_for(x, y, eps=eps, N=N, user_geometry=False)
    info = sk.sk_plan_info(plan)
    got = np.zeros((N,) * d)
    sk.sk_fourier_coefficients(plan, got)
    want = ofs.fourier_coefficients(N, d, eps * info["scale"] ** 2, 2.0, 0.4, 8)
    assert np.max(np.abs(got - want)) <= 1e-10 * np.max(np.abs(want))
    assert info["eps_scaled"] == pytest.approx(eps * info["scale"] ** 2, rel=1e-15)


# --------------------------------------------------------- NFFT stages
def _common(arr, h, d):
    return arr[tuple([slice(0, 2 * h)] * d)]


@pytest.mark.parametrize("precision", [sk.SK_FP64, sk.SK_FP32])
@pytest.mark.parametrize("d,N", [(1, 32), (2, 32), (3, 16)])
def test_adjoint_nfft_matches_adjoint_ndft(d, N, precision):
    h = N // 2
    x = wl.uniform_ball(333, d, 0.2, 5)
    y = wl.uniform_ball(211, d, 0.2, 6)
    plan = plan_for(x, y, N=N, precision=precision)
    w = np.random.default_rng(7).standard_normal(333)
    out = np.zeros(((2 * h + 1),) * d + (2,))
    sk.sk_adjoint_nfft(plan, sk.SK_SET_X, w, out.reshape(-1))
    got = out[..., 0] + 1j * out[..., 1]
    want = ofs.adjoint_ndft(x + 0.5, w, N)
    err = np.max(np.abs(_common(got, h, d) - want)) / np.sum(np.abs(w))
    assert err <= TOL_FS[precision]
    # Hermitian symmetry of the real-data spectrum, including the +N/2 planes:
    # exact in exact arithmetic, so to the precision's rounding level here
    flip = got[tuple([slice(None, None, -1)] * d)]
    sym_tol = 1e-12 if precision == sk.SK_FP64 else 1e-6
    assert np.max(np.abs(got - np.conj(flip))) <= sym_tol * np.max(np.abs(got)) + 1e-300


@pytest.mark.parametrize("precision", [sk.SK_FP64, sk.SK_FP32])
@pytest.mark.parametrize("d,N", [(1, 32), (2, 32), (3, 16)])
def test_nfft_matches_ndft(d, N, precision):
    h = N // 2
    x = wl.uniform_ball(129, d, 0.2, 8)
    y = wl.uniform_ball(301, d, 0.2, 9)
    plan = plan_for(x, y, N=N, precision=precision)
    rng = np.random.default_rng(10)
    A = rng.standard_normal((2 * h + 1,) * d) + 1j * rng.standard_normal((2 * h + 1,) * d)
    F = 0.5 * (A + np.conj(A[tuple([slice(None, None, -1)] * d)]))       # Hermitian: F[-k] = conj F[k]
    buf = np.stack([F.real, F.imag], axis=-1).reshape(-1).copy()
    got = np.zeros(301)
    sk.sk_nfft(plan, sk.SK_SET_Y, buf, got)
    # the stage computes the real part of the sum over I_N
    want = ofs.ndft(y + 0.5, _common(F, h, d), N).real
    assert np.max(np.abs(got - want)) / np.sum(np.abs(F)) <= TOL_FS[precision]


def kb_window_bound(m, sigma=2.0):
    """Error bound of the Kaiser-Bessel window relative to the l1 norm of the
    input (Potts and Steidl's estimate, 4 pi (sqrt m + m) (1 - 1/sigma)^(1/4)
    exp(-2 pi m sqrt(1 - 1/sigma)))."""
    q = 1.0 - 1.0 / sigma
    return 4 * math.pi * (math.sqrt(m) + m) * q ** 0.25 * math.exp(-2 * math.pi * m * math.sqrt(q))


FLOOR_NFFT = {sk.SK_FP64: 1e-12, sk.SK_FP32: 1e-5}


@pytest.mark.parametrize("precision", [sk.SK_FP64, sk.SK_FP32])
@pytest.mark.parametrize("m_w", [2, 3, 4, 5, 6, 7, 8])
def test_2d_nfft_stages_every_window_width(m_w, precision):
    # every 2-D window width; a dense cluster puts several hundred points in
    # one bin (tasks split into runs) next to sparse bins and a ragged tail
    N, h = 64, 32
    x = np.concatenate([wl.uniform_ball(1401, 2, 0.2, 21), 0.004 * np.random.default_rng(22).standard_normal((600, 2))])
    y = np.concatenate([wl.uniform_ball(555, 2, 0.2, 23), 0.11 + 0.002 * np.random.default_rng(24).standard_normal((333, 2))])
    plan = plan_for(x, y, N=N, m_w=m_w, precision=precision)
    tol = max(kb_window_bound(m_w), FLOOR_NFFT[precision])
    w = np.random.default_rng(25).standard_normal(len(x))
    out = np.zeros((2 * h + 1, 2 * h + 1, 2))
    sk.sk_adjoint_nfft(plan, sk.SK_SET_X, w, out.reshape(-1))
    got = out[..., 0] + 1j * out[..., 1]
    err = np.max(np.abs(_common(got, h, 2) - ofs.adjoint_ndft(x + 0.5, w, N))) / np.sum(np.abs(w))
    assert err <= tol, (err, tol)
    rng = np.random.default_rng(26)
    A = rng.standard_normal((2 * h + 1,) * 2) + 1j * rng.standard_normal((2 * h + 1,) * 2)
    F = 0.5 * (A + np.conj(A[::-1, ::-1]))
    buf = np.stack([F.real, F.imag], axis=-1).reshape(-1).copy()
    t = np.zeros(len(y))
    sk.sk_nfft(plan, sk.SK_SET_Y, buf, t)
    err = np.max(np.abs(t - ofs.ndft(y + 0.5, _common(F, h, 2), N).real)) / np.sum(np.abs(F))
    assert err <= tol, (err, tol)


@pytest.mark.parametrize("precision", [sk.SK_FP64, sk.SK_FP32])
@pytest.mark.parametrize("m_w", [2, 3, 4, 5, 6, 7, 8])
@pytest.mark.parametrize("d,N", [(1, 64), (3, 32)])
def test_1d_3d_nfft_stages_every_window_width(d, N, m_w, precision):
    # every window width in 1-D and 3-D: the 3-D column kernels (m <= 5, both
    # precisions; tensor-core interpolation in FP32) and the per-point kernels
    # (m >= 6), against the adjoint NDFT and the NDFT
    h = N // 2
    rng = np.random.default_rng(101 + 10 * d + m_w)
    x = np.concatenate([wl.uniform_ball(401, d, 0.2, 102 + m_w), 0.01 * rng.standard_normal((300, d))])
    y = wl.uniform_ball(333, d, 0.2, 103 + m_w)
    plan = plan_for(x, y, N=N, m_w=m_w, precision=precision)
    tol = max(kb_window_bound(m_w), FLOOR_NFFT[precision])
    w = rng.standard_normal(len(x))
    out = np.zeros(((2 * h + 1),) * d + (2,))
    sk.sk_adjoint_nfft(plan, sk.SK_SET_X, w, out.reshape(-1))
    got = out[..., 0] + 1j * out[..., 1]
    err = np.max(np.abs(_common(got, h, d) - ofs.adjoint_ndft(x + 0.5, w, N))) / np.sum(np.abs(w))
    assert err <= tol, (err, tol)
    A = rng.standard_normal((2 * h + 1,) * d) + 1j * rng.standard_normal((2 * h + 1,) * d)
    F = 0.5 * (A + np.conj(A[tuple([slice(None, None, -1)] * d)]))
    buf = np.stack([F.real, F.imag], axis=-1).reshape(-1).copy()
    t = np.zeros(len(y))
    sk.sk_nfft(plan, sk.SK_SET_Y, buf, t)
    err = np.max(np.abs(t - ofs.ndft(y + 0.5, _common(F, h, d), N).real)) / np.sum(np.abs(F))
    assert err <= tol, (err, tol)


@pytest.mark.parametrize("m_w", [2, 3, 4, 5])
def test_3d_tensor_core_interpolation_matches_exact_sums_and_cuda_cores(m_w):
    # the tcgen05 interpolation (default for 3-D FP32) against the exact sums and
    # against the CUDA-core kernels on the same plan; a dense cluster puts
    # thousands of points into a few bins (several tasks per bin, ragged tiles)
    rng = np.random.default_rng(31 + m_w)
    x = np.concatenate([wl.uniform_ball(3001, 3, 0.2, 32), 0.01 * rng.standard_normal((2500, 3))])
    y = np.concatenate([wl.uniform_ball(1777, 3, 0.2, 33), 0.05 + 0.003 * rng.standard_normal((900, 3))])
    plan = plan_for(x, y, eps=0.02, N=32, m_w=m_w, precision=sk.SK_FP32, user_geometry=False)
    v = wl.positive_vector(len(y), 34)
    u = wl.positive_vector(len(x), 35)
    out = {}
    for kind in (sk.SK_KERNELS_TENSOR, sk.SK_KERNELS_SIMT):
        sk.sk_set_kernels(plan, kind)
        t = np.zeros(len(x))
        tt = np.zeros(len(y))
        sk.sk_kernel_apply(plan, 0, v, t)
        sk.sk_kernel_apply(plan, 1, u, tt)
        out[kind] = (t, tt)
    t_exact = osk.kernel_apply(x, y, v, 0.02, 2.0)
    tt_exact = osk.kernel_apply_T(x, y, u, 0.02, 2.0)
    # the window error bound of m_w with sigma = 2 (relative to the l1 norm,
    # here of the weights times max K = 1), or the FP32 floor
    tol = max(1e-5, 4 * kb_window_bound(m_w))
    for kind in out:
        assert efs(out[kind][0], t_exact) <= tol, (kind, efs(out[kind][0], t_exact))
        assert efs(out[kind][1], tt_exact) <= tol
    # the two kernels differ by FP32 rounding only (the FP32 tolerance)
    for a, b in zip(out[sk.SK_KERNELS_TENSOR], out[sk.SK_KERNELS_SIMT]):
        assert np.max(np.abs(a - b)) <= TOL_FS[sk.SK_FP32] * np.max(np.abs(b))


@pytest.mark.parametrize("m_w", [2, 4, 6, 8])
def test_2d_tensor_core_interpolation_matches_exact_sums_and_cuda_cores(m_w):
    # the 2-D tcgen05 interpolation (default for 2-D FP32) against the exact
    # sums and the strip kernels; a Gaussian-mixture source puts several
    # hundred points into single strips (several runs per bin)
    x = wl.gaussian_mixture(4000, 2, 4, 0.01, 0.1, 61)
    y = wl.uniform_ball(3000, 2, 0.2, 62)
    plan = plan_for(x, y, eps=0.01, N=128, m_w=m_w, precision=sk.SK_FP32, user_geometry=False)
    v = wl.positive_vector(len(y), 63)
    u = wl.positive_vector(len(x), 64)
    out = {}
    for kind in (sk.SK_KERNELS_TENSOR, sk.SK_KERNELS_SIMT):
        sk.sk_set_kernels(plan, kind)
        t = np.zeros(len(x))
        tt = np.zeros(len(y))
        sk.sk_kernel_apply(plan, 0, v, t)
        sk.sk_kernel_apply(plan, 1, u, tt)
        out[kind] = (t, tt)
    tol = max(1e-5, 4 * kb_window_bound(m_w))
    t_exact = osk.kernel_apply(x, y, v, 0.01, 2.0)
    tt_exact = osk.kernel_apply_T(x, y, u, 0.01, 2.0)
    for kind in out:
        assert efs(out[kind][0], t_exact) <= tol
        assert efs(out[kind][1], tt_exact) <= tol
    for a, b in zip(out[sk.SK_KERNELS_TENSOR], out[sk.SK_KERNELS_SIMT]):
        assert np.max(np.abs(a - b)) <= TOL_FS[sk.SK_FP32] * np.max(np.abs(b))


def test_tensor_core_wait_gives_up_and_the_plan_recovers():
    # the failure path of the tensor-core kernels, made on purpose without a
    # fault: the MMA group is skipped, the bounded wait (about a second) runs
    # out, the solve reports SK_ERR_TIMEOUT; afterwards the same plan solves
    # normally
    x = wl.uniform_ball(1200, 3, 0.2, 81)
    y = wl.uniform_ball(900, 3, 0.2, 82)
    a, b = wl.uniform_weights(1200), wl.uniform_weights(900)
    plan = plan_for(x, y, a, b, eps=0.02, precision=sk.SK_FP32, user_geometry=False)
    sk.sk_inject_fault(plan, sk.SK_FAULT_TC_WAIT)
    st, _ = sk.sk_solve(plan, 1, raise_on_error=False)
    assert st == sk.SK_ERR_TIMEOUT
    sk.sk_inject_fault(plan, sk.SK_FAULT_NONE)
    sk.sk_set_state(plan)                       # u = v = 1 again
    st, res = sk.sk_solve(plan, 30)
    assert st == sk.SK_OK
    ref = osk.sinkhorn_dense(x, a, y, b, 0.02, 2.0, 30)
    assert abs(res["s"] - ref["s"]) <= 1e-5 * abs(ref["s"])
    plan64 = plan_for(x, y, a, b, eps=0.02, precision=sk.SK_FP64)
    with pytest.raises(sk.SkError) as err:
        sk.sk_inject_fault(plan64, sk.SK_FAULT_TC_WAIT)
    assert err.value.status == sk.SK_ERR_UNSUPPORTED


def test_autotune_keeps_a_valid_kind_and_the_state():
    x = wl.uniform_ball(3000, 3, 0.2, 91)
    y = wl.uniform_ball(2500, 3, 0.2, 92)
    plan = plan_for(x, y, eps=0.02, precision=sk.SK_FP32, user_geometry=False)
    sk.sk_solve(plan, 5, result=False)
    u0, v0 = np.zeros(3000), np.zeros(2500)
    it0 = sk.sk_get_state(plan, u0, v0)
    chosen = sk.sk_autotune(plan)
    assert chosen in (sk.SK_KERNELS_TENSOR, sk.SK_KERNELS_SIMT)
    assert sk.sk_plan_info(plan)["tensor_cores"] == (1 if chosen == sk.SK_KERNELS_TENSOR else 0)
    u1, v1 = np.zeros(3000), np.zeros(2500)
    assert sk.sk_get_state(plan, u1, v1) == it0
    assert np.array_equal(u0, u1) and np.array_equal(v0, v1)
    plan64 = plan_for(x, y, eps=0.02, precision=sk.SK_FP64)
    assert sk.sk_autotune(plan64) == sk.SK_KERNELS_SIMT


def test_kernel_selection_errors():
    x = wl.uniform_ball(100, 3, 0.2, 40)
    plan64 = plan_for(x, x, precision=sk.SK_FP64, N=16)
    with pytest.raises(sk.SkError) as err:
        sk.sk_set_kernels(plan64, sk.SK_KERNELS_TENSOR)
    assert err.value.status == sk.SK_ERR_UNSUPPORTED
    sk.sk_set_kernels(plan64, sk.SK_KERNELS_SIMT)
    plan1 = plan_for(wl.uniform_ball(100, 1, 0.2, 41), wl.uniform_ball(90, 1, 0.2, 42), precision=sk.SK_FP32)
    with pytest.raises(sk.SkError) as err:
        sk.sk_set_kernels(plan1, sk.SK_KERNELS_TENSOR)
    assert err.value.status == sk.SK_ERR_UNSUPPORTED
    with pytest.raises(sk.SkError) as err:
        sk.sk_set_kernels(plan1, 7)
    assert err.value.status == sk.SK_ERR_ARG
    assert sk.sk_plan_info(plan1)["tensor_cores"] == 0
    plan2 = plan_for(wl.uniform_ball(100, 2, 0.2, 43), wl.uniform_ball(90, 2, 0.2, 44), precision=sk.SK_FP32)
    assert sk.sk_plan_info(plan2)["tensor_cores"] == 1
    sk.sk_set_kernels(plan2, sk.SK_KERNELS_SIMT)
    assert sk.sk_plan_info(plan2)["tensor_cores"] == 0


@pytest.mark.parametrize("kind", ["tensor", "simt"])
@pytest.mark.parametrize("d,N", [(2, 32), (3, 16)])
def test_nfft_points_at_the_edges_of_the_valid_region(d, N, kind):
    # points filling the whole region whose windows stay on the grid
    # (cells m-1 .. n_os-1-m along every axis), so the bins' boxes reach the
    # grid's first and last cells: interpolation against the NDFT
    h, n_os, m = N // 2, 2 * N, 4
    lo, hi = (m - 1 + 0.01) / n_os, (n_os - m - 0.01) / n_os
    rng = np.random.default_rng(71 + d)
    x = rng.uniform(lo, hi, (300, d)) - 0.5
    y = rng.uniform(lo, hi, (700, d)) - 0.5
    y[:d] = np.diag(np.full(d, lo - 0.5)) + (hi - 0.5) * (1 - np.eye(d))   # corners of the region
    plan = plan_for(x, y, N=N, precision=sk.SK_FP32)
    sk.sk_set_kernels(plan, sk.SK_KERNELS_TENSOR if kind == "tensor" else sk.SK_KERNELS_SIMT)
    A = rng.standard_normal((2 * h + 1,) * d) + 1j * rng.standard_normal((2 * h + 1,) * d)
    F = 0.5 * (A + np.conj(A[tuple([slice(None, None, -1)] * d)]))
    buf = np.stack([F.real, F.imag], axis=-1).reshape(-1).copy()
    got = np.zeros(len(y))
    sk.sk_nfft(plan, sk.SK_SET_Y, buf, got)
    want = ofs.ndft(y + 0.5, _common(F, h, d), N).real
    assert np.max(np.abs(got - want)) / np.sum(np.abs(F)) <= TOL_FS[sk.SK_FP32]


# --------------------------------------------------------- kernel products
@pytest.mark.parametrize("precision", [sk.SK_FP64, sk.SK_FP32])
@pytest.mark.parametrize("d,n,m,N,eps", [(1, 1000, 777, 64, 0.05), (2, 2000, 1337, 64, 0.05),
                                         (3, 1500, 1999, 64, 0.02), (2, 1024, 1000, 128, 0.01)])
def test_kernel_apply_matches_exact_sums(d, n, m, N, eps, precision):
    x = wl.uniform_ball(n, d, 0.2, 11)
    y = wl.uniform_ball(m, d, 0.2, 12)
    plan = plan_for(x, y, eps=eps, N=N, precision=precision, user_geometry=False)
    v = wl.positive_vector(m, 13)
    u = wl.positive_vector(n, 14)
    t = torch.zeros(n, dtype=torch.float64, device=DEV)
    tt = torch.zeros(m, dtype=torch.float64, device=DEV)
    sk.sk_kernel_apply(plan, 0, cuda(v), t)
    sk.sk_kernel_apply(plan, 1, cuda(u), tt)
    torch.cuda.synchronize()
    assert efs(t.cpu().numpy(), osk.kernel_apply(x, y, v, eps, 2.0)) <= TOL_FS[precision]
    assert efs(tt.cpu().numpy(), osk.kernel_apply_T(x, y, u, eps, 2.0)) <= TOL_FS[precision]


@pytest.mark.parametrize("precision", [sk.SK_FP64, sk.SK_FP32])
@pytest.mark.parametrize("d,N", [(1, 2048), (1, 1024), (2, 512)])
def test_kernel_apply_longest_pencils(d, N, precision):
    # the largest FFT lengths (n_os = 4096 in 1-D, where FP64 pencils switch
    # to 8 elements per thread; 1024 in 2-D) against the exact sums
    x = wl.uniform_ball(1500, d, 0.2, 51)
    y = wl.uniform_ball(1300, d, 0.2, 52)
    eps = 2e-4 if d == 1 else 0.002
    plan = plan_for(x, y, eps=eps, N=N, precision=precision, user_geometry=False)
    v = wl.positive_vector(len(y), 53)
    t = np.zeros(len(x))
    sk.sk_kernel_apply(plan, 0, v, t)
    assert efs(t, osk.kernel_apply(x, y, v, eps, 2.0)) <= TOL_FS[precision]


@pytest.mark.parametrize("N,radius,m_w", [(32, 0.2, 4), (64, 0.2, 4), (128, 0.2, 4), (64, 0.2, 8),
                                           (64, 0.004, 4), (32, 0.24, 4)])
def test_3d_fft_planes_match_passes_and_exact_sums(N, radius, m_w):
    # the cluster-plane FFT (three launches) against the five pass launches on
    # the same plan, and both against the exact sums: n_os = 64, 128, 256; a
    # band of ~0.5 n_os, a band of a few cells (points in a radius-0.004 ball)
    # and a wide one (points near the edge of the valid region)
    x = wl.uniform_ball(2100, 3, radius, 41)
    y = wl.uniform_ball(1900, 3, radius, 42)
    eps = 0.02
    plan = plan_for(x, y, eps=eps, N=N, m_w=m_w, precision=sk.SK_FP32)
    assert sk.sk_plan_info(plan)["fft_planes"] == 1
    v = wl.positive_vector(len(y), 43)
    u = wl.positive_vector(len(x), 44)
    out = {}
    for form in (sk.SK_FFT_PLANES, sk.SK_FFT_PASSES):
        sk.sk_set_fft(plan, form)
        t, tt = np.zeros(len(x)), np.zeros(len(y))
        sk.sk_kernel_apply(plan, 0, v, t)
        sk.sk_kernel_apply(plan, 1, u, tt)
        out[form] = (t, tt)
    exact = (osk.kernel_apply(x, y, v, eps, 2.0), osk.kernel_apply_T(x, y, u, eps, 2.0))
    for k in range(2):
        a, b = out[sk.SK_FFT_PLANES][k], out[sk.SK_FFT_PASSES][k]
        assert np.max(np.abs(a - b)) <= 1e-6 * np.max(np.abs(b))
        assert efs(a, exact[k]) <= TOL_FS[sk.SK_FP32]
        assert efs(b, exact[k]) <= TOL_FS[sk.SK_FP32]


def test_fft_form_selection_errors():
    x = wl.uniform_ball(300, 3, 0.2, 45)
    y = wl.uniform_ball(200, 3, 0.2, 46)
    p64 = plan_for(x, y, precision=sk.SK_FP64)
    assert sk.sk_plan_info(p64)["fft_planes"] == 0
    with pytest.raises(sk.SkError) as e:
        sk.sk_set_fft(p64, sk.SK_FFT_PLANES)
    assert e.value.status == sk.SK_ERR_UNSUPPORTED
    sk.sk_set_fft(p64, sk.SK_FFT_PASSES)
    p2 = plan_for(x[:, :2], y[:, :2], precision=sk.SK_FP32)
    assert sk.sk_plan_info(p2)["fft_planes"] == 0
    with pytest.raises(sk.SkError) as e:
        sk.sk_set_fft(p2, sk.SK_FFT_PLANES)
    assert e.value.status == sk.SK_ERR_UNSUPPORTED
    with pytest.raises(sk.SkError) as e:
        sk.sk_set_fft(p64, 7)
    assert e.value.status == sk.SK_ERR_ARG


def test_kernel_apply_host_buffers_and_ragged_tiny_sizes():
    # host (numpy) in/out buffers; sizes below one block and not multiples of anything
    for n, m in [(1, 1), (1, 5), (7, 1), (33, 65)]:
        x = wl.uniform_ball(n, 2, 0.2, 15 + n)
        y = wl.uniform_ball(m, 2, 0.2, 16 + m)
        plan = plan_for(x, y)
        v = wl.positive_vector(m, 17)
        t = np.zeros(n)
        sk.sk_kernel_apply(plan, 0, v, t)
        assert efs(t, osk.kernel_apply(x, y, v, 0.05, 2.0)) <= 1e-6


def test_identical_points_and_degenerate_geometry():
    # all points at one location: bounding radius 0, scale falls back to 1
    x = np.full((10, 3), 0.123)
    y = np.full((4, 3), 0.123)
    plan = plan_for(x, y, user_geometry=False, eps=0.02)
    t = np.zeros(10)
    sk.sk_kernel_apply(plan, 0, np.ones(4), t)
    np.testing.assert_allclose(t, 4.0, rtol=1e-6)


@pytest.mark.parametrize("precision,tol", [(sk.SK_FP64, 1e-12), (sk.SK_FP32, 1e-5)])
@pytest.mark.parametrize("r", [2.0, 1.0, 1.5])
def test_direct_method_matches_exact_sums(precision, tol, r):
    d, n, m, eps = 3, 700, 901, 0.02
    x = wl.uniform_ball(n, d, 0.2, 18)
    y = wl.uniform_ball(m, d, 0.2, 19)
    plan = plan_for(x, y, eps=eps, r=r, precision=precision, user_geometry=False)
    sk.sk_set_method(plan, sk.SK_METHOD_DIRECT)
    v = wl.positive_vector(m, 20)
    t = np.zeros(n)
    sk.sk_kernel_apply(plan, 0, v, t)
    exact = osk.kernel_apply(x, y, v, eps, r)
    assert np.max(np.abs(t - exact) / exact) <= tol


# --------------------------------------------------------- Sinkhorn
def test_solve_matches_dense_oracle_small_2d_fp64():
    w = wl.SMALL_2D
    x, y = w.points()
    a, b = w.marginals()
    ref = osk.sinkhorn_dense(x, a, y, b, w.eps, w.r, w.iters)
    plan = sk.sk_init(cuda(x), cuda(a), cuda(y), cuda(b), w.eps, w.r,
                      sk.sk_default_params(N=w.N, m_w=w.m_w, precision=sk.SK_FP64))
    u = torch.zeros(w.n, dtype=torch.float64, device=DEV)
    v = torch.zeros(w.m, dtype=torch.float64, device=DEV)
    st, res = sk.sk_solve(plan, w.iters, 0.0, 10, u, v)
    assert st == sk.SK_OK and res["iters"] == w.iters and res["total_iters"] == w.iters
    assert abs(res["s"] - ref["s"]) / abs(ref["s"]) <= 1e-5
    ent = osk.entropy(a) + osk.entropy(b)
    assert res["s_upper"] == pytest.approx(res["s"] + w.eps * ent, rel=1e-12)
    # the scaling vectors follow the oracle's iterates
    np.testing.assert_allclose(u.cpu().numpy(), ref["u"], rtol=1e-4)
    np.testing.assert_allclose(v.cpu().numpy(), ref["v"], rtol=1e-4)
    assert res["err_row"] == pytest.approx(ref["err_row"], abs=1e-6)
    assert res["err_col"] < 1e-6


@pytest.mark.parametrize("precision", [sk.SK_FP32, sk.SK_FP64])
def test_solve_matches_dense_oracle_3d(precision):
    d, n, m, eps, iters = 3, 2500, 2100, 0.02, 30
    x = wl.uniform_ball(n, d, 0.2, 21)
    y = wl.uniform_ball(m, d, 0.2, 22)
    a, b = wl.dirichlet_weights(n, 23), wl.dirichlet_weights(m, 24)
    ref = osk.sinkhorn_dense(x, a, y, b, eps, 2.0, iters)
    plan = sk.sk_init(cuda(x), cuda(a), cuda(y), cuda(b), eps, 2.0,
                      sk.sk_default_params(N=64, m_w=4, precision=precision))
    st, res = sk.sk_solve(plan, iters)
    assert st == sk.SK_OK
    assert abs(res["s"] - ref["s"]) / abs(ref["s"]) <= 1e-5


def test_solve_direct_method_matches_oracle():
    d, n, m, eps, iters = 2, 900, 1100, 0.05, 20
    x = wl.uniform_ball(n, d, 0.2, 25)
    y = wl.uniform_ball(m, d, 0.2, 26)
    a, b = wl.uniform_weights(n), wl.uniform_weights(m)
    ref = osk.sinkhorn_dense(x, a, y, b, eps, 2.0, iters)
    plan = sk.sk_init(cuda(x), cuda(a), cuda(y), cuda(b), eps, 2.0, sk.sk_default_params(precision=sk.SK_FP32))
    sk.sk_set_method(plan, sk.SK_METHOD_DIRECT)
    st, res = sk.sk_solve(plan, iters)
    assert abs(res["s"] - ref["s"]) / abs(ref["s"]) <= 1e-5


def test_fp64_direct_solve_state_matches_oracle_closely():
    # FP64 direct sums are exact to ~1e-15, so after 20 iterations the state
    # pins the fused FP64 update (the Newton quotient a / t) to 1e-11
    d, n, m, eps, iters = 2, 400, 300, 0.05, 20
    x = wl.uniform_ball(n, d, 0.2, 27)
    y = wl.uniform_ball(m, d, 0.2, 28)
    a, b = wl.dirichlet_weights(n, 29), wl.dirichlet_weights(m, 30)
    ref = osk.sinkhorn_dense(x, a, y, b, eps, 2.0, iters)
    plan = sk.sk_init(cuda(x), cuda(a), cuda(y), cuda(b), eps, 2.0, sk.sk_default_params(precision=sk.SK_FP64))
    sk.sk_set_method(plan, sk.SK_METHOD_DIRECT)
    u = torch.zeros(n, dtype=torch.float64, device=DEV)
    v = torch.zeros(m, dtype=torch.float64, device=DEV)
    st, res = sk.sk_solve(plan, iters, u_out=u, v_out=v)
    assert np.max(np.abs(u.cpu().numpy() / ref["u"] - 1)) <= 1e-11
    assert np.max(np.abs(v.cpu().numpy() / ref["v"] - 1)) <= 1e-11
    assert abs(res["s"] - ref["s"]) <= 1e-11 * abs(ref["s"])


def test_state_checkpoint_and_resume_is_exact():
    x = wl.uniform_ball(800, 2, 0.2, 27)
    y = wl.uniform_ball(600, 2, 0.2, 28)
    plan = plan_for(x, y, user_geometry=False)
    st, r_full = sk.sk_solve(plan, 12)
    u_full = np.zeros(800)
    v_full = np.zeros(600)
    assert sk.sk_get_state(plan, u_full, v_full) == 12
    sk.sk_set_state(plan)                      # back to u = v = 1
    sk.sk_solve(plan, 5, result=False)
    u5 = np.zeros(800)
    v5 = np.zeros(600)
    assert sk.sk_get_state(plan, u5, v5) == 5
    sk.sk_set_state(plan)
    sk.sk_set_state(plan, u5, v5, 5)           # resume from the checkpoint
    st, r_res = sk.sk_solve(plan, 7)
    assert r_res["total_iters"] == 12
    u_res = np.zeros(800)
    sk.sk_get_state(plan, u_res, None)
    np.testing.assert_allclose(u_res, u_full, rtol=1e-12)
    assert r_res["s"] == pytest.approx(r_full["s"], rel=1e-12)


def test_tolerance_stopping():
    x = wl.uniform_ball(500, 2, 0.2, 29)
    y = wl.uniform_ball(500, 2, 0.2, 30)
    plan = plan_for(x, y, user_geometry=False)
    st, res = sk.sk_solve(plan, 400, tol=1e-9, check_every=5)
    assert st == sk.SK_OK
    assert res["iters"] < 400 and res["iters"] % 5 == 0
    assert res["err_row"] <= 1e-9
    plan2 = plan_for(x, y, user_geometry=False)
    st2, res2 = sk.sk_solve(plan2, 3, tol=1e-14, check_every=1, raise_on_error=False)
    assert st2 == sk.SK_ERR_NOT_CONVERGED and res2["iters"] == 3


def test_input_errors_are_reported():
    x = wl.uniform_ball(20, 2, 0.2, 31)
    y = wl.uniform_ball(20, 2, 0.2, 32)
    with pytest.raises(sk.SkError) as e:
        plan_for(x, y, a=np.full(20, 0.1))
    assert e.value.status == sk.SK_ERR_WEIGHTS
    bad = x.copy()
    bad[3, 1] = np.nan
    with pytest.raises(sk.SkError) as e:
        plan_for(bad, y)
    assert e.value.status == sk.SK_ERR_DOMAIN
    with pytest.raises(sk.SkError) as e:
        plan_for(x + 0.4, y)                  # user geometry: points leave the torus box
    assert e.value.status == sk.SK_ERR_DOMAIN
    neg = wl.uniform_weights(20)
    neg[0], neg[1] = -0.05, neg[1] + 0.1
    with pytest.raises(sk.SkError) as e:
        plan_for(x, y, a=neg)
    assert e.value.status == sk.SK_ERR_WEIGHTS


def test_launch_count_and_stage_timing():
    x = wl.uniform_ball(3000, 3, 0.2, 34)
    y = wl.uniform_ball(3000, 3, 0.2, 35)
    plan = plan_for(x, y, user_geometry=False, precision=sk.SK_FP32)
    c0 = sk.sk_launch_count(plan)
    sk.sk_solve(plan, 4, result=False)
    torch.cuda.synchronize()
    per_iter = (sk.sk_launch_count(plan) - c0) / 4
    assert sk.sk_plan_info(plan)["fft_planes"] == 1
    assert per_iter == 2 * (1 + 3 + 1)        # spread, 3 FFT launches (cluster planes), interp per half-step
    sk.sk_set_fft(plan, sk.SK_FFT_PASSES)
    c0 = sk.sk_launch_count(plan)
    sk.sk_solve(plan, 2, result=False)
    torch.cuda.synchronize()
    assert (sk.sk_launch_count(plan) - c0) / 2 == 2 * (1 + 5 + 1)   # 5 FFT passes
    sk.sk_stage_times(plan, 1)
    sk.sk_solve(plan, 3, result=False)
    times = sk.sk_stage_times(plan, 0)
    assert times["spread"][1] == 6 and times["fft"][1] == 6 and times["interp"][1] == 6
    assert all(times[k][0] > 0 for k in ("spread", "fft", "interp"))


# --------------------------------------------------------- full-size workloads
def _sampled_rows(x, y, v, eps, r, rows):
    return osk.kernel_apply(x[rows], y, v, eps, r, chunk=4)


@pytest.mark.parametrize("work", [wl.HEADLINE_3D, wl.GMM_2D], ids=lambda w: w.name)
def test_full_size_kernel_apply_sampled_rows(work):
    x, y = work.points()
    a, b = work.marginals()
    prm = sk.sk_default_params(N=work.N, m_w=work.m_w,
                               precision=sk.SK_FP32 if work.precision == "fp32" else sk.SK_FP64)
    plan = sk.sk_init(cuda(x), cuda(a), cuda(y), cuda(b), work.eps, work.r, prm)
    v = wl.positive_vector(work.m, 36)
    t = torch.zeros(work.n, dtype=torch.float64, device=DEV)
    sk.sk_kernel_apply(plan, 0, cuda(v), t)
    rows = np.random.default_rng(37).choice(work.n, 64, replace=False)
    rows = np.concatenate([rows, [0, work.n - 1]])
    exact = _sampled_rows(x, y, v, work.eps, work.r, rows)
    got = t.cpu().numpy()[rows]
    # E_fs over the sample, normalized by the largest sum in the sample
    assert np.max(np.abs(got - exact)) / np.max(np.abs(exact)) <= 1e-5


def test_full_size_solve_marginal_property():
    # after the even half-step the column marginal v * (K^T u) equals b; check it
    # on sampled columns with exact FP64 sums over all 1e6 rows.
    work = wl.HEADLINE_3D
    x, y = work.points()
    a, b = work.marginals()
    plan = sk.sk_init(cuda(x), cuda(a), cuda(y), cuda(b), work.eps, work.r,
                      sk.sk_default_params(N=work.N, m_w=work.m_w))
    u = np.zeros(work.n)
    v = np.zeros(work.m)
    st, res = sk.sk_solve(plan, 10, u_out=u, v_out=v)
    assert st == sk.SK_OK and math.isfinite(res["s"])
    cols = np.random.default_rng(38).choice(work.m, 16, replace=False)
    marg = np.empty(len(cols))
    for k, j in enumerate(cols):
        d2 = np.sum((x - y[j]) ** 2, axis=1)
        marg[k] = v[j] * np.dot(u, np.exp(-d2 / work.eps))
    np.testing.assert_allclose(marg, b[cols], rtol=1e-4)
    assert res["err_col"] < 1e-4 * np.linalg.norm(b)


# --------------------------------------------------------- near field (r not an even integer)
@pytest.mark.parametrize("d,N,r,eps,eps_I,precision", [
    (1, 256, 1.0, 0.05, 0.0, sk.SK_FP64),
    (2, 64, 1.0, 0.05, 0.0, sk.SK_FP64),
    (2, 64, 1.0, 0.05, 0.0, sk.SK_FP32),
    (2, 64, 1.5, 0.05, 0.0, sk.SK_FP32),
    (3, 64, 1.0, 0.02, 0.0, sk.SK_FP32),
    (3, 64, 1.0, 0.02, 1.0 / 8, sk.SK_FP64),
])
def test_nearfield_kernel_apply_matches_exact_sums(d, N, r, eps, eps_I, precision):
    n, m = 1500, 1301
    x = wl.uniform_ball(n, d, 0.2, 41)
    y = wl.uniform_ball(m, d, 0.2, 42)
    plan = plan_for(x, y, eps=eps, r=r, N=N, precision=precision, user_geometry=False, eps_I=eps_I)
    assert sk.sk_plan_info(plan)["nearfield"] == 1
    v = wl.positive_vector(m, 43)
    u = wl.positive_vector(n, 44)
    t = np.zeros(n)
    tt = np.zeros(m)
    sk.sk_kernel_apply(plan, 0, v, t)
    sk.sk_kernel_apply(plan, 1, u, tt)
    assert efs(t, osk.kernel_apply(x, y, v, eps, r)) <= TOL_FS[precision]
    assert efs(tt, osk.kernel_apply_T(x, y, u, eps, r)) <= TOL_FS[precision]


def test_nearfield_solve_matches_dense_oracle():
    d, n, m, eps, iters = 2, 1200, 1000, 0.05, 30
    x = wl.uniform_ball(n, d, 0.2, 45)
    y = wl.uniform_ball(m, d, 0.2, 46)
    a, b = wl.dirichlet_weights(n, 47), wl.dirichlet_weights(m, 48)
    ref = osk.sinkhorn_dense(x, a, y, b, eps, 1.0, iters)
    plan = sk.sk_init(cuda(x), cuda(a), cuda(y), cuda(b), eps, 1.0, sk.sk_default_params(precision=sk.SK_FP64))
    st, res = sk.sk_solve(plan, iters)
    assert st == sk.SK_OK
    assert abs(res["s"] - ref["s"]) / abs(ref["s"]) <= 1e-5


def test_nearfield_stage_timing_counts():
    x = wl.uniform_ball(2000, 3, 0.2, 49)
    y = wl.uniform_ball(2000, 3, 0.2, 50)
    plan = plan_for(x, y, r=1.0, eps=0.02, precision=sk.SK_FP32, user_geometry=False)
    sk.sk_stage_times(plan, 1)
    sk.sk_solve(plan, 2, result=False)
    times = sk.sk_stage_times(plan, 0)
    assert times["near"][1] == 4 and times["near"][0] > 0


def test_full_size_r1_efs_on_2e4_target_subsample():
    # the r = 1 workload's prescribed check: E_fs of the FP32 fast summation
    # (near field included) on 2e4 random targets against exact FP64 sums over
    # all 4e6 sources.  The exact sums come from the FP64 direct method
    # (Eq. (matexp) term by term, pinned to the oracle to 1e-12 per element in
    # test_direct_method_matches_exact_sums) on a plan whose targets are the
    # subsample: 8e10 FP64 kernel evaluations on the GPU.
    work = wl.BALL3D_R1
    x, y = work.points()
    a, b = work.marginals()
    prm = sk.sk_default_params(N=work.N, m_w=work.m_w, precision=sk.SK_FP32, eps_I=work.extra["eps_I"])
    plan = sk.sk_init(cuda(x), cuda(a), cuda(y), cuda(b), work.eps, work.r, prm)
    v = wl.positive_vector(work.m, 53)
    t = torch.zeros(work.n, dtype=torch.float64, device=DEV)
    sk.sk_kernel_apply(plan, 0, cuda(v), t)
    plan.close()
    rows = np.random.default_rng(54).choice(work.n, 20000, replace=False)
    xs = x[rows]
    ref_plan = sk.sk_init(cuda(xs), cuda(wl.uniform_weights(len(rows))), cuda(y), cuda(b), work.eps, work.r,
                          sk.sk_default_params(precision=sk.SK_FP64, eps_I=work.extra["eps_I"]))
    sk.sk_set_method(ref_plan, sk.SK_METHOD_DIRECT)
    exact = torch.zeros(len(rows), dtype=torch.float64, device=DEV)
    sk.sk_kernel_apply(ref_plan, 0, cuda(v), exact)
    ref_plan.close()
    got, exact = t.cpu().numpy()[rows], exact.cpu().numpy()
    assert np.all(exact > 0)
    # the direct reference itself, on a few rows, against the oracle
    few = np.arange(8)
    assert np.max(np.abs(exact[few] - _sampled_rows(xs, y, v, work.eps, work.r, few)) / exact[few]) <= 1e-12
    assert np.max(np.abs(got - exact)) / np.max(exact) <= 1e-5


def test_full_size_r1_kernel_apply_sampled_rows():
    work = wl.BALL3D_R1
    x, y = work.points()
    a, b = work.marginals()
    prm = sk.sk_default_params(N=work.N, m_w=work.m_w, precision=sk.SK_FP32, eps_I=work.extra["eps_I"])
    plan = sk.sk_init(cuda(x), cuda(a), cuda(y), cuda(b), work.eps, work.r, prm)
    v = wl.positive_vector(work.m, 51)
    t = torch.zeros(work.n, dtype=torch.float64, device=DEV)
    sk.sk_kernel_apply(plan, 0, cuda(v), t)
    rows = np.random.default_rng(52).choice(work.n, 24, replace=False)
    exact = _sampled_rows(x, y, v, work.eps, work.r, rows)
    got = t.cpu().numpy()[rows]
    assert np.max(np.abs(got - exact)) / np.max(np.abs(exact)) <= 1e-5
