"""The multi-GPU form of the benchmark is weak scaling with no collective on
the data path: every rank runs its own mixture, and only the timing is
combined (max over ranks).  These world-size-2 gloo runs on the CPU cover
that host logic: the max-over-ranks reduction, the whole-job rate, the
per-rank seeds, and the reference arm's rank-0-only rule."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    local_ms = 100.0 + 50.0 * rank          # rank 1 is the slow one
    ms_max = bench._max_over_ranks(local_ms, dist)
    rate = bench.whole_job_rate(1e9, 10, ms_max, ws)
    ref = bench.run_reference(type("A", (), {"steps": 1, "warmup": 0})(), bench.CONFIGS[bench.WORKLOAD],
                              rank, ws) if rank != 0 else "rank0"
    with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as fh:
        fh.write(f"{ms_max} {rate} {bench.rank_seed(rank)} {ref is None}\n")
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_weak_scaling(tmp_path):
    ws = 2
    mp.start_processes(_worker, args=(ws, _free_port(), str(tmp_path)), nprocs=ws, start_method="spawn")
    rows = [open(tmp_path / f"r{r}.txt").read().split() for r in range(ws)]
    for r, (ms_max, rate, seed, ref_none) in enumerate(rows):
        assert float(ms_max) == 150.0                     # the slowest rank's time on every rank
        assert float(rate) == pytest.approx(ws * 1e9 * 10 / 0.150)
        assert int(seed) == r                             # independent mixtures
        if r != 0:
            assert ref_none == "True"                     # the reference arm runs on rank 0 only
    assert rows[0][2] != rows[1][2]
