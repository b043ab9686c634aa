"""The multi-rank path of bench.py on CPU: two gloo ranks, each an independent replica with its
own step time; the reported throughput uses the slowest rank's time and all ranks' steps."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    value, ms_max = bench.aggregate(1000.0 * (rank + 1), steps=3, world=world, device="cpu")
    out[rank] = (value, ms_max)
    dist.destroy_process_group()


def test_two_rank_aggregation():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        value, ms_max = res[rank]
        assert ms_max == 2000.0                      # slowest rank
        assert abs(value - world * 3 / 2.0) < 1e-12  # 6 steps in 2 s


def test_single_rank_aggregation():
    import bench
    value, ms_max = bench.aggregate(500.0, steps=4, world=1, device="cpu")
    assert ms_max == 500.0 and value == 8.0


def test_metric_names_the_workload_and_fourier_path_selection(monkeypatch):
    import bench
    assert bench._metric("plain-scale") == bench.METRIC
    assert "fourier-100k" in bench._metric("fourier-100k")
    assert "plain-scale" not in bench._metric("fourier-100k")
    monkeypatch.delenv("CMCS_DFT_FOURSTEP", raising=False)
    assert bench._single_cta_fft(8192) and bench._single_cta_fft(128)
    assert not bench._single_cta_fft(16384) and not bench._single_cta_fft(100000)
    assert not bench._single_cta_fft(2000)
    monkeypatch.setenv("CMCS_DFT_FOURSTEP", "1")
    assert not bench._single_cta_fft(8192)


def test_workload_subsets_for_the_bench():
    import bench
    wl = bench._workload("fourier-small", 0, tasks=2)
    assert wl.T == 2 and wl.mask.shape == (2, 256)
    wl = bench._workload("plain-small", 0, tasks=3)
    assert wl.T == 3


def test_split_problem_aggregation_counts_one_problem():
    """With the tasks of one problem split over the ranks, the whole job makes one EM
    iteration per step: value = steps / slowest rank's time."""
    import bench
    value, ms_max = bench.aggregate(500.0, steps=4, world=1, device="cpu", units=4)
    assert value == 8.0
    assert "tasks split over the GPUs" in bench._metric("plain-scale", sharded=True)
