"""The N>1 path on CPU: two gloo ranks each simulate their own walker range
(no communication on the data path) and merge their FP64 partial sums in
rank order; the merged signal and moments equal a single-process run of all
walkers, and every walker's final state is the same as in that run.  The
oracle does the walking here (no GPU needed); the sharding and merge code is
the one bench.py uses."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _workload():
    import rms_inputs as ri
    return ri.workload("cylinder-32^3").with_(n_walkers=3001, n_steps=300, G=ri.pgse(0.1, 0.2, 1e-3, 300)[None, :],
                                              rec_steps=np.arange(50, 301, 50))


def _rank(rank, world, port, out_dir, weak):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from paper_2012_06478_gb300 import shard
    wl = _workload()
    b, e = shard.shard_range(rank, world, wl.n_walkers, weak=weak)
    r = oracle.run(wl, b, e, n_threads=2)
    S, asum = oracle.readout(r, wl)
    # the oracle normalises; its numerators are S * sum alpha (the library
    # returns them as such, rms_read_partials)
    v = shard.allreduce_partials(shard.pack_partials(S * asum, asum, r["moments"]))
    Sm, Mm, am = shard.unpack_partials(v, S.shape, r["moments"].shape)
    np.savez(os.path.join(out_dir, f"rank{rank}.npz"), S=Sm, M=Mm, a=am, i=r["i"], o=r["o"], b=b, e=e)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("weak", [False, True])
def test_two_gloo_ranks_merge_to_the_single_run(tmp_path, weak):
    import oracle
    oracle.build()
    world = 2
    mp.start_processes(_rank, args=(world, _port(), str(tmp_path), weak), nprocs=world, start_method="spawn")
    wl = _workload()
    total = world * wl.n_walkers if weak else wl.n_walkers
    ref = oracle.run(wl, 0, total, n_threads=4)
    S_ref, a_ref = oracle.readout(ref, wl)
    outs = [np.load(os.path.join(tmp_path, f"rank{r}.npz")) for r in range(world)]
    for o in outs:  # every rank holds the same merged result
        np.testing.assert_allclose(o["S"], S_ref, rtol=0, atol=1e-12)
        np.testing.assert_allclose(o["M"], ref["moments"], rtol=1e-12)
        assert abs(float(o["a"]) - a_ref) <= 1e-12 * a_ref
        b, e = int(o["b"]), int(o["e"])
        np.testing.assert_array_equal(o["i"], ref["i"][b:e])
        np.testing.assert_array_equal(o["o"], ref["o"][b:e])
    assert int(outs[0]["e"]) == int(outs[1]["b"])
