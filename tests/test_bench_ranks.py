"""Multi-rank host logic of bench.py on CPU: two gloo ranks (replicas) agree
on the job time (max over ranks) and the whole-job throughput; the reference
arm does its work on rank 0 only."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms_local = [12.5, 30.0, 7.0, 21.0][rank]
        dist.barrier()
        ms = bench.max_over_ranks(ms_local, dist, device="cpu")
        value = bench.job_gbps(world, 1e9, ms)
        with open(os.path.join(out, f"r{rank}.txt"), "w") as f:
            f.write(f"{ms} {value}")
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
def test_max_over_ranks_and_job_value(tmp_path, world):
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    want_ms = max([12.5, 30.0, 7.0, 21.0][:world])
    for r in range(world):
        ms, value = map(float, (tmp_path / f"r{r}.txt").read_text().split())
        assert ms == want_ms
        assert value == pytest.approx(world * 1e9 / (want_ms * 1e-3) / 1e9)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25, None) == 3.25
    assert bench.job_gbps(1, 2e9, 1000.0) == pytest.approx(2.0)


def test_reference_arm_other_ranks_exit_without_work(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")

    class A:
        steps, warmup, gpus = 2, 3, 2
    assert bench.run_reference(A()) == 0
    assert capsys.readouterr().out == ""


def test_traffic_is_reported_only_for_the_captured_kernel(tmp_path):
    """The roofline's DRAM traffic comes from a committed ncu summary only when
    the summary names the exact kernel instance (arguments and source hash)."""
    import bench
    f = tmp_path / "t.md"
    f.write_text("text\nkernel: k_hvp<f32,512,RED1,MINB2>@0123456789\nbytes_per_launch: 123\n")
    assert bench.traffic_for(str(f), "k_hvp<f32,512,RED1,MINB2>@0123456789") == 123.0
    assert bench.traffic_for(str(f), "k_hvp<f32,512,RED1,MINB2>@9876543210") is None
    assert bench.traffic_for(str(f), "k_hvs<f32,RED1,TAB1,MINB3>@0123456789") is None
    assert bench.traffic_for(str(tmp_path / "missing.md"), "x") is None


def test_source_tag_tracks_the_kernel_sources():
    """One tag per translation unit: its own source and the shared headers and
    table builders; kernels in different files get different tags."""
    import importlib
    build = importlib.import_module("paper_2307_13222_gb300.build")
    t = build.source_tag("hv_phased.cu")
    assert len(t) == 10 and all(c in "0123456789abcdef" for c in t)
    assert t != build.source_tag("hv_tile.cu") and t == build.source_tag("hv_phased.cu")
    assert all(f in build.SOURCES or f.endswith(".cuh") for f in build.HV_COMMON)


def test_issue_roofline_matches_family_and_hash(tmp_path):
    import bench
    f = tmp_path / "p.md"
    f.write_text("text\nkernel: k_hvp<f32,512,RED0,MINB2>@0123456789\nwarp_inst_per_row: 29.0\n")
    r = bench.issue_roofline(str(f), "k_hvp<f32,512,RED1,MINB2>@0123456789", 1000000, 2.0, 100, 2000)
    # 1e6 rows x 29 / (100 SMs x 4 x 2e9 per s) = 0.03625 ms
    assert r is not None and abs(r["bound_ms"] - 0.03625) < 1e-12 and abs(r["frac"] - 0.018125) < 1e-12
    assert bench.issue_roofline(str(f), "k_hvp<f32,512,RED1,MINB2>@9876543210", 10, 1.0, 1, 1) is None
    assert bench.issue_roofline(str(f), "k_hvp<f64,1024,RED1,MINB1>@0123456789", 10, 1.0, 1, 1) is None


def test_parse_cpulist():
    import bench
    assert bench.parse_cpulist("0-3,8,10-11\n") == {0, 1, 2, 3, 8, 10, 11}
    assert bench.parse_cpulist("") is None


def test_traffic_for_same_family(tmp_path):
    import bench
    f = tmp_path / "t.md"
    f.write_text("kernel: k_tile<f32,RED0>x2@0123456789\nbytes_per_stage: 77\n")
    assert bench.traffic_for(str(f), "k_tile<f32,RED3>x2@0123456789", key="bytes_per_stage", same_family=True) == 77.0
    assert bench.traffic_for(str(f), "k_tile<f32,RED3>x2@9999999999", key="bytes_per_stage", same_family=True) is None
    assert bench.traffic_for(str(f), "k_tile<f32,RED3>x2@0123456789", key="bytes_per_stage") is None
