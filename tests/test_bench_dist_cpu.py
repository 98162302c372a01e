"""The benchmark's multi-process host logic on the CPU: two ranks on the gloo
backend (rendezvous on 127.0.0.1) agree on the slowest rank's time and the
whole-job rate, and the reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    r, w, local = bench.dist_env()
    slowest = bench.max_over_ranks(1.5 + rank, w, device="cpu")     # rank r took 1.5 + r s
    rate = bench.whole_job_rate(1000, w, slowest)
    dist.barrier()
    dist.destroy_process_group()
    q.put((r, w, local, slowest, rate))


def test_two_gloo_ranks_agree_on_the_slowest_time_and_the_rate():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1] and all(o[1] == 2 for o in out)
    for r, w, local, slowest, rate in out:
        assert local == r
        assert slowest == 2.5                     # the max over the ranks' 1.5 and 2.5 s
        assert rate == pytest.approx(2 * 1000 / 2.5)


def test_one_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.0, 1) == 3.0
    assert bench.whole_job_rate(10, 1, 2.0) == 5.0


def test_reference_arm_is_rank_zero_only(monkeypatch, capsys):
    # under torchrun every rank but 0 exits 0 at once, with no output and no work
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = bench.argparse.Namespace(gpus=2, steps=1, warmup=3, impl="reference")
    assert bench.run_reference(args) == 0
    assert capsys.readouterr().out == ""


def test_oracle_baseline_over_all_host_cores():
    # the oracle's pass with its bosonic planes in a spawned process pool runs
    # (no GPU involved) and reports the workers it used
    sys.path.insert(0, ROOT)
    import bench
    from paper_1507_00895_gb300 import inputs as I
    w = I.workload("paper_u20", nk=4, n_w=8, m_max=2)
    r = bench.cpu_baseline(w)
    assert r["kind"] == "oracle" and r["value"] > 0
    a = r["all_cores"]
    assert "unavailable" not in a, a
    assert a["value"] > 0 and 1 <= a["cores"] <= min(os.cpu_count() or 1, w.n_bos)
