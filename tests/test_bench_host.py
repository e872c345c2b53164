"""Host logic of the multi-rank bench, run as two gloo ranks on the CPU: the
timed region is the maximum over ranks and the value counts every rank's
iterations; each rank gets its own problem."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist          # noqa: E402
import torch.multiprocessing as mp        # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [12.5, 20.0][rank]
    ms_max = bench.reduce_max_ms(ms, world)
    out[rank] = (ms_max, bench.whole_job_rate(ms_max, 100, world))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    assert out[0] == out[1]
    ms_max, rate = out[0]
    assert ms_max == 20.0
    assert rate == pytest.approx(2 * 100 / 0.020)


def test_single_rank_needs_no_collective():
    import bench
    assert bench.reduce_max_ms(7.0, 1) == 7.0
    assert bench.whole_job_rate(50.0, 10, 1) == pytest.approx(200.0)


def test_replica_problems_differ_by_rank():
    import bench
    from paper_2201_07524_gb300 import workloads as wl
    w0 = bench.replica_workload(wl.SMALL_2D, 0)
    w1 = bench.replica_workload(wl.SMALL_2D, 1)
    assert (w0.seed_x, w0.seed_y) == (wl.SMALL_2D.seed_x, wl.SMALL_2D.seed_y)
    assert w1.seed_x != w0.seed_x and w1.seed_y != w0.seed_y
    x0, _ = w0.points()
    x1, _ = w1.points()
    assert not (x0 == x1).all()


@pytest.mark.parametrize("name", ["GMM_2D", "BALL3D_R1", "HEADLINE_3D"])
def test_replica_keeps_every_workload_field(name):
    # a replica differs from its workload only in the seeds: the point source,
    # weights and extra parameters (the near-field radius) carry over
    import dataclasses
    import bench
    from paper_2201_07524_gb300 import workloads as wl
    w = getattr(wl, name)
    r = bench.replica_workload(w, 3)
    for f in dataclasses.fields(w):
        if f.name in ("seed_x", "seed_y"):
            assert getattr(r, f.name) == getattr(w, f.name) + 3000
        else:
            assert getattr(r, f.name) == getattr(w, f.name), f.name


def test_roofline_kernel_names_follow_dimension_and_kernel_kind():
    import bench
    from paper_2201_07524_gb300 import workloads as wl
    assert bench.kernel_name("interp", wl.HEADLINE_3D, 1) == "k_interp3_tc<8>"
    assert bench.kernel_name("interp", wl.HEADLINE_3D, 0) == "k_interp3_col<8, float>"
    assert bench.kernel_name("spread", wl.HEADLINE_3D, 1) == "k_spread3_col<8, float>"
    assert bench.kernel_name("interp", wl.GMM_2D, 1) == "k_interp2_tc<12>"
    assert bench.kernel_name("spread", wl.GMM_2D, 1) == "k_spread2_col<12, float>"
    assert bench.kernel_name("interp", wl.GMM_2D, 0) == "k_interp2_strip<12, float>"
    # every name the bench can look up is one the traffic record may hold
    import json
    import os
    rec = json.load(open(os.path.join(os.path.dirname(bench.__file__), "profiles", "traffic.json")))
    for stage, w in (("spread", wl.HEADLINE_3D), ("interp", wl.HEADLINE_3D), ("spread", wl.GMM_2D),
                     ("interp", wl.GMM_2D)):
        assert bench.kernel_name(stage, w, 1) in rec


def test_bench_workload_table():
    import bench
    from paper_2201_07524_gb300 import workloads as wl
    table = bench._workloads(wl)
    assert table["headline"] is wl.HEADLINE_3D
    assert table["gmm2d"].source == "gmm" and table["gmm2d"].weights == "dirichlet"
    assert table["r1"].r == 1.0 and table["r1"].extra["eps_I"] == 1.0 / 32
