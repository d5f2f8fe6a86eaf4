"""The multi-rank host logic of bench.py on CPU: two gloo ranks on
127.0.0.1 (the layout torchrun gives one node), checking the timing
collectives (barrier, the maximum of the ranks' times, the sum of their
throughputs), the whole-job rate, and that the reference arm runs on rank 0
only (the other ranks return without work)."""
import json
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out_dir):
    os.environ.update({"WORLD_SIZE": str(ws), "RANK": str(rank), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import bench
    R = bench.Ranks("gloo")
    res = {"ws": R.ws, "rank": R.rank, "local": R.local}
    R.barrier()
    # rank r took 10 + r ms over 4 steps: the job took the slowest rank's time
    res["max"] = R.max(10.0 + rank)
    res["sum"] = R.sum([1.0 + rank, 2.0 * rank])
    res["rate"] = bench.whole_job_rate(4096, R.ws, res["max"], 4)
    # the reference arm: rank 0 alone runs it; the others return at once
    if rank != 0:
        res["reference"] = bench.run_reference(None)
    R.close()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump(res, f)


def test_two_gloo_ranks(tmp_path):
    ws = 2
    mp.start_processes(_rank_main, args=(ws, _free_port(), str(tmp_path)), nprocs=ws,
                       join=True, start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(ws)]
    for r, d in enumerate(res):
        assert (d["ws"], d["rank"], d["local"]) == (2, r, r)
        assert d["max"] == 11.0
        assert d["sum"] == [3.0, 2.0]
        # 2 ranks x 4096 vectors per step, 11 ms over 4 steps
        assert d["rate"] == pytest.approx(2 * 4096 / (11.0 / 4 / 1e3))
    assert res[1]["reference"] is None


def test_single_rank_without_torchrun(monkeypatch):
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    sys.path.insert(0, ROOT)
    import bench
    R = bench.Ranks("gloo")
    assert (R.ws, R.rank, R.local) == (1, 0, 0) and R.dist is None
    assert R.max(3.5) == 3.5 and R.sum([1, 2]) == [1.0, 2.0]
    R.barrier()
    R.close()
    assert bench.whole_job_rate(4096, 1, 2.0, 1) == pytest.approx(4096 / 2e-3)
