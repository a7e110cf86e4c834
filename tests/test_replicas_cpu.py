"""The N > 1 path of bench.py on CPU: two spawned gloo ranks initialise the
process group from the torchrun environment, meet at the barrier, take the
maximum over ranks (the bench's timing rule), and run the reference arm,
which rank 0 alone executes and prints."""
import json
import os
import multiprocessing as mp
import socket

import pytest

from _replica_worker import replica


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_replicas():
    pytest.importorskip("torch")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=replica, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = []
    try:
        for _ in procs:
            res.append(q.get(timeout=240))
    finally:
        for p in procs:
            p.join(timeout=30)
            if p.is_alive():
                p.kill()
    res.sort(key=lambda d: d["rank"])
    assert [d["world"] for d in res] == [2, 2] and [d["backend"] for d in res] == ["gloo", "gloo"]
    assert [d["max"] for d in res] == [2.5, 2.5]
    line = json.loads(res[0]["ref_out"].strip())
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert res[1]["ref_out"] == ""


def test_reference_arm_prints_a_bounded_oracle_line():
    """bench.py --impl reference times bounded samples of the oracle's apply
    (a block of node rows per step when full applies would not fit) and prints
    one JSON line with the contract's keys."""
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "40",
                          "--warmup", "3", "--ref-seconds", "2"], capture_output=True, text=True, timeout=300,
                         cwd=root, env={**os.environ, "WORLD_SIZE": "1", "RANK": "0"})
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["steps"] == 40
    assert line["cpu_baseline"]["kind"] == "oracle" and "node rows" in line["cpu_baseline"]["sample"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["unit"] == "GDoF*modes/s"
