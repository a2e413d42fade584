"""The machine peaks the rooflines divide by (include/rms_peaks.h), on the GPU:
each is a positive rate of the right order for one GB300, ordered the way
the memory hierarchy orders them (a volume that stays in L1 or L2 gathers
faster than one that has to come from HBM), and sizes outside the
documented range are refused before any device work."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rms():
    import torch
    assert torch.cuda.is_available()
    import paper_2012_06478_gb300 as rms
    return rms


def test_sm_count(rms):
    import torch
    assert rms.rms_device_sm_count() == torch.cuda.get_device_properties(0).multi_processor_count


def test_fp64_rates(rms):
    n = rms.rms_device_sm_count()
    clock = 2.1e9
    rates = {k: rms.rms_measure_peak(k, 0, 5.0, 2)[0]
             for k in (rms.RMS_PEAK_FP64_ADD, rms.RMS_PEAK_FP64_MUL, rms.RMS_PEAK_FP64_FMA)}
    for k, r in rates.items():
        # at least a quarter of an operation and at most 64 per SM per clock
        assert 0.25 * n * 1e9 < r < 64 * n * clock, (k, r)


def test_gather_rates_follow_the_memory_hierarchy(rms):
    l1 = rms.rms_measure_peak(rms.RMS_PEAK_GATHER, 1 << 16, 5.0, 2)[0]      # 128 KiB
    l2 = rms.rms_measure_peak(rms.RMS_PEAK_GATHER, 1 << 22, 5.0, 2)[0]      # 8 MiB
    hbm = rms.rms_measure_peak(rms.RMS_PEAK_GATHER, 1 << 29, 5.0, 2)[0]     # 1 GiB
    dep = rms.rms_measure_peak(rms.RMS_PEAK_GATHER_DEP, 1 << 22, 5.0, 2)[0]
    assert l1 > l2 > hbm > 1e9, (l1, l2, hbm)
    assert 0.2 * l2 < dep <= 1.5 * l2


def test_arguments_checked(rms):
    from paper_2012_06478_gb300 import _lib
    for kind, vol, ms, reps in ((7, 0, 5.0, 1), (rms.RMS_PEAK_GATHER, 1000, 5.0, 1),
                                (rms.RMS_PEAK_GATHER, 1 << 32, 5.0, 1), (rms.RMS_PEAK_FP64_ADD, 0, -1.0, 1),
                                (rms.RMS_PEAK_FP64_ADD, 0, 5.0, 0)):
        with pytest.raises(rms.RmsError) as e:
            rms.rms_measure_peak(kind, vol, ms, reps)
        assert e.value.status == _lib.RMS_E_INVALID_ARG
