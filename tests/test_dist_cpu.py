"""Multi-rank plumbing of bench.py on CPU (gloo, world size 2): ranks build
independent replicas, so the only cross-rank steps are the barrier and the
max over ranks of the step time."""
import os
import socket

import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    r, local, ws, pg = bench.dist()
    assert (r, ws) == (rank, world)
    bench.barrier(pg)
    m = bench.max_over_ranks(pg, 10.0 + rank)
    out[rank] = m
    pg.destroy_process_group()


def test_two_rank_max_over_ranks():
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, _free_port(), out), nprocs=2, join=True)
    assert dict(out) == {0: 11.0, 1: 11.0}


REF_ARGS = ["--impl", "reference", "--workload", "small", "--steps", "2", "--warmup", "1",
            "--oracle-sample-log2", "15"]


def _check_reference_line(line, gpus):
    import json
    d = json.loads(line)
    assert d["impl"] == "reference" and d["n_gpus"] == gpus
    assert d["unit"] == "symbols/s" and d["higher_is_better"] is True and d["value"] > 0
    assert d["steps"] == 2 and d["warmup"] == 1 and d["dtype"] == "u8"
    assert "n=2^20" in d["metric"] and d["config"]["workload"].startswith("WT+WM, n=2^20")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == d["value"] and "2^15" in cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def _ref_worker(rank, world, port, out):
    import contextlib
    import io
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        rc = bench.main(REF_ARGS + ["--gpus", str(world)])
    out[rank] = (rc, buf.getvalue())


def test_reference_arm_one_rank(capsys):
    """--impl reference times the oracle on a bounded sample and prints one line with
    the keys the measurement contract asks for (no GPU involved)."""
    import bench
    assert bench.main(REF_ARGS + ["--gpus", "1"]) == 0
    lines = [x for x in capsys.readouterr().out.splitlines() if x.strip()]
    assert len(lines) == 1
    _check_reference_line(lines[0], 1)


def test_reference_arm_two_ranks():
    """Under two ranks rank 0 alone runs and prints; rank 1 exits 0 without work."""
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_ref_worker, args=(2, _free_port(), out), nprocs=2, join=True)
    rc0, text0 = out[0]
    rc1, text1 = out[1]
    assert rc0 == 0 and rc1 == 0 and text1.strip() == ""
    lines = [x for x in text0.splitlines() if x.strip()]
    assert len(lines) == 1
    _check_reference_line(lines[0], 2)
