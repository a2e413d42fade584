"""Morton re-bucketing of walkers (RMS_MORTON): before every step launch the
walkers are put in Morton order of their voxel in device memory.  A walker's
random streams follow its id, not its place in memory, so every trajectory
is unchanged bit for bit -- in both precision forms, under every
interaction, with absorbing membranes and spin concentrations -- and only the
order of the FP64 sums over walkers differs (signal and moment sums agree to
rounding).  The order itself is checked against the Morton codes of the
walkers' voxels at the start of the last launch."""
import numpy as np
import pytest

from conftest import make_workload
from test_gpu_parity import _rand_case, assert_moments_close, assert_signal_close, assert_walkers_equal

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rms():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2012_06478_gb300 as rms
    return rms


@pytest.fixture(scope="module")
def oracle():
    import oracle
    oracle.build()
    return oracle


WALKER_KEYS = ("i", "o", "i0", "o0", "c", "A", "phase", "hash")


def _same_walkers(a, b):
    for k in WALKER_KEYS:
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)


@pytest.mark.parametrize("case", [
    dict(seed=21),
    dict(seed=22, S=1, periodic=(0, 0, 0)),
    dict(seed=23, S=2, dead=[0, 0, 1, 0], W=3000),
    dict(seed=24, W=1, n_steps=50),
    dict(seed=25, shape=(1, 1, 1), L=1, W=700, S=1),
    dict(seed=26, shape=(33, 5, 300), W=2500, n_steps=200),
])
def test_bit_exact_with_the_oracle(rms, oracle, case):
    wl = _rand_case(**case)
    g = rms.simulate(wl, rms.RMS_FP64, hash_=True, steps_per_launch=29, walkers=True, morton=True)
    o = oracle.run(wl, 0, wl.n_walkers, hash_=True)
    assert o["err"] == 0
    S_o, asum_o = oracle.readout(o, wl)
    assert_walkers_equal(g, o)
    if wl.rec_steps.size:
        assert_moments_close(g["moments"], o["moments"])
    assert_signal_close(g["S"], S_o)
    assert abs(g["alpha_sum"] - asum_o) <= 1e-12 * asum_o
    assert np.array_equal(np.sort(g["slots"]), np.arange(wl.n_walkers))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("interaction,extras", [(0, False), (0, True), (1, True), (2, True)])
def test_same_walkers_as_without_reordering(rms, precision, interaction, extras):
    wl = _rand_case(31, W=4000, n_steps=240, shape=(12, 9, 10)).with_(interaction=interaction)
    if extras:
        R = np.full((wl.n_labels, wl.n_labels), 0.05)
        np.fill_diagonal(R, 0.0)
        wl = wl.with_(rho=R, conc=np.array([1.0, 0.7, 1.2, 0.9]))
    p = rms.RMS_FP64 if precision == "fp64" else rms.RMS_FP32
    a = rms.simulate(wl, p, hash_=True, counts=True, steps_per_launch=50, walkers=True)
    b = rms.simulate(wl, p, hash_=True, counts=True, steps_per_launch=50, walkers=True, morton=True)
    _same_walkers(a, b)
    np.testing.assert_array_equal(a["counts"], b["counts"])
    assert_signal_close(b["S"], a["S"])
    assert_moments_close(b["moments"], a["moments"])
    assert abs(b["alpha_sum"] - a["alpha_sum"]) <= 1e-12 * a["alpha_sum"]
    assert not np.array_equal(b["slots"], np.arange(wl.n_walkers))  # the order did change


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_axon_substrate_over_many_launches(rms, precision):
    """The benchmark's axon substrate, 3e4 walkers, 12 launches (12 re-orderings);
    the production kernel (no checksum) in both layouts."""
    import rms_inputs as ri
    wl = ri.workload("axons-200x200x400")
    n = 1200
    wl = wl.with_(n_walkers=30000, n_steps=n, G=ri.pgse(0.05, 0.15, wl.dt, n)[None, :],
                  rec_steps=np.arange(100, n + 1, 100))
    p = rms.RMS_FP64 if precision == "fp64" else rms.RMS_FP32
    a = rms.simulate(wl, p, steps_per_launch=100, walkers=True)
    b = rms.simulate(wl, p, steps_per_launch=100, walkers=True, morton=True)
    for k in ("i", "o", "i0", "o0", "c", "A", "phase"):
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)
    assert_signal_close(b["S"], a["S"])
    assert_moments_close(b["moments"], a["moments"])


def _morton_key(ix, iy, iz, shape_xyz):
    """Morton code of wrapped voxel coordinates, each shifted to at most 8 bits
    (the ordering RMS_MORTON documents)."""
    bits = int(max(shape_xyz) - 1).bit_length()
    s = max(0, bits - 8)
    key = np.zeros(ix.shape, np.uint64)
    for a, c in enumerate((ix, iy, iz)):
        c = (c.astype(np.int64) % shape_xyz[a]) >> s
        for bit in range(10):
            key |= ((c >> bit) & 1).astype(np.uint64) << np.uint64(3 * bit + a)
    return key


def test_slots_are_in_morton_order_of_the_last_launch_start(rms):
    lab = np.zeros((40, 70, 600), np.uint16)  # (z, y, x): x has 600 voxels -> coordinates shifted by 2
    lab[:, :, 300:] = 1
    def wl_of(n):
        return make_workload(lab, voxel_um=0.2, D=2.0, kappa=0.5, dt=5e-4, n_steps=n, n_walkers=6000, seed=9,
                             G=np.ones(n))

    wl = wl_of(90)
    spl = 30
    full = rms.simulate(wl, rms.RMS_FP64, steps_per_launch=spl, walkers=True, morton=True)
    # positions at the start of the last launch (step 60), from a run stopped there
    part = rms.simulate(wl, rms.RMS_FP64, steps_per_launch=spl, walkers=True, step_end=60)
    slots = full["slots"]
    assert np.array_equal(np.sort(slots), np.arange(wl.n_walkers))
    i = part["i"][slots]
    key = _morton_key(i[:, 0], i[:, 1], i[:, 2], (600, 70, 40))
    assert np.all(np.diff(key.astype(np.int64)) >= 0)
    # stable: walkers of one key keep the order of the previous layout, which
    # starts as walker order -- so the first launch's layout is sorted by
    # (key at step 0, walker id)
    one = rms.simulate(wl_of(30), rms.RMS_FP64, steps_per_launch=spl, walkers=True, morton=True)
    i0 = one["i0"]
    k0 = _morton_key(i0[:, 0], i0[:, 1], i0[:, 2], (600, 70, 40))
    np.testing.assert_array_equal(one["slots"], np.lexsort((np.arange(wl.n_walkers), k0)))


def test_resume_from_a_reordered_run(rms):
    wl = _rand_case(41, W=2500, n_steps=300)
    full = rms.simulate(wl, rms.RMS_FP64, hash_=True, walkers=True, steps_per_launch=40)
    part = rms.simulate(wl, rms.RMS_FP64, hash_=True, walkers=True, steps_per_launch=40, step_end=130, morton=True)
    st = {k: part[k] for k in WALKER_KEYS}
    st.update(moments=part["moments"], step=130)
    rest = rms.simulate(wl, rms.RMS_FP64, hash_=True, walkers=True, steps_per_launch=40, resume=st, morton=True)
    _same_walkers(rest, full)
    assert_moments_close(rest["moments"], full["moments"])
    assert_signal_close(rest["S"], full["S"])


def test_checked_mode_with_reordering(rms):
    wl = _rand_case(43, W=3000, n_steps=200)
    a = rms.simulate(wl, rms.RMS_FP32, checked=True, steps_per_launch=20, walkers=True, morton=True)
    b = rms.simulate(wl, rms.RMS_FP32, steps_per_launch=20, walkers=True)
    for k in ("i", "o", "c", "A", "phase"):
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)
