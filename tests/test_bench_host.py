"""Host-side pieces of bench.py: the multi-rank aggregation (replicas; run as
two gloo ranks on the CPU) and the clock-record parser."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    ms = 100.0 + 50.0 * rank  # rank 1 is the slow one
    bench.barrier(world)
    m = bench.reduce_max(ms, world)
    rate = bench.whole_job_rate(1000, world, m)
    with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as fh:
        fh.write(f"{m} {rate}")
    dist.destroy_process_group()


def test_two_rank_max_and_whole_job_rate(tmp_path):
    import torch.multiprocessing as mp

    port = _free_port()
    mp.spawn(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    for r in range(2):
        m, rate = map(float, open(tmp_path / f"r{r}.txt").read().split())
        assert m == 150.0
        assert rate == pytest.approx(2 * 1000 / 0.150)


def test_single_rank_is_identity():
    import bench

    assert bench.reduce_max(12.5, 1) == 12.5
    assert bench.whole_job_rate(10, 1, 1000.0) == pytest.approx(10.0)


def test_clock_parser_flags_only_active_reasons():
    import bench

    rows = [["0", "2070", "2070", "900.1", "0x0000000000000000", "Not Active", "Not Active", "Not Active", "Not Active"],
            ["0", "1950", "2070", "1390.0", "0x0000000000000004", "Not Active", "Not Active", "Not Active", "Active"],
            ["0", "2070", "2070", "1100.0", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"]]
    c = bench.parse_clock_rows(rows)
    assert c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap"] and c["samples"] == 3
    assert bench.parse_clock_rows([]) is None
