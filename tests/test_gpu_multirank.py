"""The N>1 path through the product: two processes share the one GPU, each
runs its half of the walkers of one simulation through the C ABI (global
walker ids keep the random streams), and the ranks exchange only the
library's unnormalised sums (rms_read_partials) over gloo, add them in rank
order and let the library normalise (rms_normalise_partials).  The merged
signal, moments and sum of alpha equal the single-process run of all
walkers to 1e-12.  The two processes never wait on each other on the GPU:
each runs its own kernels to completion; the exchange is on the host."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _workload():
    import rms_inputs as ri
    # the 32^3 cylinder case with a permeable membrane, T2 and an odd walker count
    wl = ri.workload("cylinder-32^3")
    return wl.with_(n_walkers=10_001, kappa=np.array([[0.0, 0.02], [0.02, 0.0]]), T2=np.array([80.0, 50.0]))


def _rank(rank, world, port, out_dir):
    import sys
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    import paper_2012_06478_gb300 as rms
    from paper_2012_06478_gb300 import shard
    wl = _workload()
    b, e = shard.shard_range(rank, world, wl.n_walkers)
    out = {}
    for name, prec in (("fp64", rms.RMS_FP64), ("fp32", rms.RMS_FP32)):
        g = rms.simulate(wl, prec, n_walkers=e - b, walker_begin=b)
        v = shard.allreduce_partials(shard.pack_partials(g["num"], g["alpha_sum"], g["moments"]))
        S, M, a = shard.unpack_partials(v, g["S"].shape, g["moments"].shape)
        out[f"S_{name}"], out[f"M_{name}"], out[f"a_{name}"] = S, M, a
    np.savez(os.path.join(out_dir, f"rank{rank}.npz"), b=b, e=e, **out)
    dist.barrier()
    dist.destroy_process_group()


def test_two_processes_on_one_gpu_merge_to_the_single_run(tmp_path):
    import torch
    assert torch.cuda.is_available()
    import paper_2012_06478_gb300 as rms
    world = 2
    mp.start_processes(_rank, args=(world, _port(), str(tmp_path)), nprocs=world, start_method="spawn")
    wl = _workload()
    outs = [np.load(os.path.join(tmp_path, f"rank{r}.npz")) for r in range(world)]
    assert int(outs[0]["b"]) == 0 and int(outs[0]["e"]) == int(outs[1]["b"]) and int(outs[1]["e"]) == wl.n_walkers
    for name, prec in (("fp64", rms.RMS_FP64), ("fp32", rms.RMS_FP32)):
        ref = rms.simulate(wl, prec)
        for o in outs:  # every rank holds the same merged result
            np.testing.assert_allclose(o[f"S_{name}"], ref["S"], rtol=0, atol=1e-12)
            np.testing.assert_allclose(o[f"M_{name}"], ref["moments"], rtol=1e-12)
            assert abs(float(o[f"a_{name}"]) - ref["alpha_sum"]) <= 1e-12 * ref["alpha_sum"]
        # the normalised read equals the library's division of its own partials
        np.testing.assert_array_equal(rms.rms_normalise_partials(ref["num"], ref["alpha_sum"]), ref["S"])
