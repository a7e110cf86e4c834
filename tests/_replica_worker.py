"""Worker of the multi-process (gloo, CPU) tests of bench.py's replica path:
run as a spawned process with RANK / WORLD_SIZE / MASTER_* in the environment."""
import io
import json
import os
import sys
from contextlib import redirect_stdout


def replica(rank, world, port, out_q):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    import torch.distributed as dist
    w, r, _ = bench.dist_init()
    res = {"world": w, "rank": r, "backend": dist.get_backend()}
    bench.barrier(w)
    res["max"] = bench.max_over_ranks(1.5 + r, w)
    # the reference arm: rank 0 times the oracle and prints one line, the others print nothing
    import argparse
    args = argparse.Namespace(steps=1, warmup=0, ref_seconds=2.0)
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(args, w, r)
    res["ref_out"] = buf.getvalue()
    bench.barrier(w)
    dist.destroy_process_group()
    out_q.put(res)
