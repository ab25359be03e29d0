"""The N>1 path of bench.py on CPU: two gloo ranks.

Reactors are independent (Sec. 1, 4), so the multi-GPU form is weak scaling:
every rank integrates its own seeded batch and the only collective is the
max over ranks of the timed region.  Here two CPU processes stand in for two
GPUs; each integrates its shard with the oracle, and the test checks that the
shards are distinct and valid, that the job time is the slowest rank's, and
that the whole-job rate counts every rank's reactors.
"""
import os
import socket

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    from oracle import ORA_ROS4, OracleMech
    from synth.configs import CONFIGS, load_mechanism
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, _ = bench._rank_env()
    n = 4
    y, p = bench.rank_states("small", n, r)
    om = OracleMech(load_mechanism(CONFIGS["small"]["mech"]))
    yo, steps, st, _ = om.integrate(ORA_ROS4, p, y, 1e-6, rtol=1e-6, atol=1e-10)
    fake_elapsed = 1.0 + r  # rank 1 is the slower one
    job = bench.max_over_ranks(fake_elapsed, w)
    rate = bench.aggregate_rate(2.0 * n, w, job)
    np.savez(os.path.join(out_dir, f"rank{r}.npz"), y=y, yo=yo, st=st, job=job, rate=rate, world=w)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling(tmp_path):
    import torch.multiprocessing as mp
    pytest.importorskip("torch.distributed")
    from oracle.oracle import build_oracle
    build_oracle()  # once, before the ranks load it
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    r0 = np.load(tmp_path / "rank0.npz")
    r1 = np.load(tmp_path / "rank1.npz")
    assert int(r0["world"]) == int(r1["world"]) == 2
    # every rank has its own batch
    assert r0["y"].shape == r1["y"].shape
    assert not np.allclose(r0["y"], r1["y"])
    # each shard integrated without trouble
    assert (r0["st"] == 0).all() and (r1["st"] == 0).all()
    assert np.isfinite(r0["yo"]).all() and np.isfinite(r1["yo"]).all()
    # the job's time is the slowest rank's, identical on every rank
    assert float(r0["job"]) == float(r1["job"]) == 2.0
    # whole-job rate: both ranks' 2 x 4 integrations over the slowest time
    assert float(r0["rate"]) == pytest.approx(2 * 2.0 * 4 / 2.0)


def test_single_rank_needs_no_process_group():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.aggregate_rate(10.0, 1, 2.0) == 5.0
    y0, _ = bench.rank_states("small", 3, 0)
    y1, _ = bench.rank_states("small", 3, 1)
    assert not np.allclose(y0, y1)
