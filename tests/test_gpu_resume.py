"""Checkpoint and resume (rms_run_range): the random streams depend only on
(seed, walker, step), so a plain FP64 run stopped at any step, read back and
resumed reproduces the uninterrupted run -- walkers, checksums, moments and
signal -- bit for bit; the FP32 form agrees to rounding."""
import numpy as np
import pytest

from test_gpu_parity import _rand_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rms():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2012_06478_gb300 as rms
    return rms


def _state(res, step):
    st = {k: res[k] for k in ("i", "o", "i0", "o0", "c", "A", "phase", "hash")}
    st["moments"] = res["moments"]
    st["step"] = step
    return st


def _case(interaction, extras):
    wl = _rand_case(71, W=1500, n_steps=300).with_(interaction=interaction)
    if extras:
        R = np.full((wl.n_labels, wl.n_labels), 0.05)
        np.fill_diagonal(R, 0.0)
        wl = wl.with_(rho=R, conc=np.array([1.0, 0.7, 1.2, 0.9]))
    return wl


@pytest.mark.parametrize("interaction,extras", [(0, False), (0, True), (1, True), (2, True)])
def test_split_runs_are_bit_identical(rms, interaction, extras):
    wl = _case(interaction, extras)
    full = rms.simulate(wl, rms.RMS_FP64, hash_=True, walkers=True, steps_per_launch=41)
    for cuts in ((1,), (137,), (wl.n_steps - 1,), (60, 211)):
        res, step = None, 0
        for cut in cuts + (wl.n_steps,):
            res = rms.simulate(wl, rms.RMS_FP64, hash_=True, walkers=True, steps_per_launch=41,
                               resume=None if res is None else _state(res, step),
                               step_end=cut if cut < wl.n_steps else 0)
            step = cut
        for k in ("i", "o", "i0", "o0", "c", "A", "phase", "hash", "moments"):
            np.testing.assert_array_equal(res[k], full[k], err_msg=f"{k} {cuts}")
        np.testing.assert_array_equal(res["S"], full["S"])


def test_fp32_resume_agrees_to_rounding(rms):
    wl = _case(0, True)
    full = rms.simulate(wl, rms.RMS_FP32, walkers=True)
    part = rms.simulate(wl, rms.RMS_FP32, walkers=True, step_end=150)
    rest = rms.simulate(wl, rms.RMS_FP32, walkers=True, resume=_state(part, 150))
    same = np.all(rest["i"] == full["i"], axis=1).mean()
    assert same > 0.99, same
    assert np.abs(rest["S"] - full["S"]).max() < 1e-4


def test_bad_step_ranges_are_refused(rms):
    from paper_2012_06478_gb300 import _lib
    wl = _case(0, False)
    part = rms.simulate(wl, rms.RMS_FP64, walkers=True, step_end=100)
    for resume, step_end in ((_state(part, 100), 50), (None, wl.n_steps + 1), (_state(part, wl.n_steps + 1), 0)):
        with pytest.raises(rms.RmsError) as e:
            rms.simulate(wl, rms.RMS_FP64, resume=resume, step_end=step_end)
        assert e.value.status == _lib.RMS_E_INVALID_ARG
