"""The SFU-rate probe that bench.py uses for the synthesis roofline's sincos
bound: a plausible rate, stable between calls."""
from __future__ import annotations

import pytest

from paper_2310_09200_b300 import bipp_ss

pytestmark = pytest.mark.gpu


def test_sincos_rate_is_plausible_and_repeatable():
    import torch
    r1 = bipp_ss.bipp_ss_measure_sincos_rate(0, 3)
    r2 = bipp_ss.bipp_ss_measure_sincos_rate(0, 3)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    # one sine and one cosine per pair: between 1 and 64 pairs per SM per nanosecond-clock
    # (an SFU issues a handful of results per SM per clock; at 1-3 GHz that is 1e9-2e10 pairs/s per SM)
    assert 1e9 * sms < r1 < 2e10 * sms, r1
    assert abs(r1 - r2) <= 0.2 * max(r1, r2), (r1, r2)


def test_fma_rates_are_plausible():
    import torch
    f32, f64 = bipp_ss.bipp_ss_measure_fma_rates(0, 3)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    # FP32: 128 FMA lanes per SM at 1-3 GHz; FP64 is a small fraction of it on this part
    assert 2 * 64 * 1e9 * sms < f32 < 2 * 128 * 3.2e9 * sms, f32
    assert 0 < f64 < f32, (f64, f32)
