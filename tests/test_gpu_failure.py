"""Failure detection on the GPU without a GPU fault: the tensor-core synthesis
kernel's bounded waits (its mbarrier handoffs between the producer warps, the
MMA issuer and the bulk-copy warp) run out, the kernel leaves cleanly and the
host reads BIPP_ERR_DEVICE_TIMEOUT; the handle stays usable."""
import time

import numpy as np
import pytest

from paper_2310_09200_b300 import bipp_ss, inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["split_fp16", "split_bf16"])
def test_bounded_wait_expiry_reports_timeout_and_recovers(precision):
    """With the fault-injection switch on, the MMA issuer waits on a barrier
    phase that nothing completes: its wait runs out (~2 s), every other warp
    leaves its own wait, and the collect fails with DEVICE_TIMEOUT, the images
    unchanged. The second collect of a geometry is captured into CUDA graphs,
    so the failing and the recovering collects run the captured kernels; with
    the switch off the same handle images exactly as before."""
    inp = inputs.make_config(0, n_t=2, n_side=16)
    bounds = np.array([[200.0, np.inf], [50.0, 200.0], [-np.inf, 50.0]])
    with bipp_ss.StandardSynthesis(inp.pix, inp.wl, bounds, n_eig=inp.n_eig, precision=precision,
                                   autotune=0) as ss:
        ss.collect_batch(inp.st_xyz, inp.vis)
        first = ss.get()
        assert np.all(np.isfinite(first)) and np.any(first != 0.0)
        bipp_ss.bipp_ss_debug_fail_wait(ss.h, True)
        t0 = time.monotonic()
        with pytest.raises(bipp_ss.BippError) as e:
            ss.collect_batch(inp.st_xyz, inp.vis)
        waited = time.monotonic() - t0
        assert e.value.code == bipp_ss.BIPP_ERR_DEVICE_TIMEOUT
        assert waited < 60.0
        np.testing.assert_array_equal(ss.get(), first)
        bipp_ss.bipp_ss_debug_fail_wait(ss.h, False)
        ss.reset()
        ss.collect_batch(inp.st_xyz, inp.vis)
        np.testing.assert_allclose(ss.get(), first, rtol=1e-12, atol=0)


def test_fault_injection_switch_validates_its_argument():
    inp = inputs.make_config(0, n_t=1, n_side=8)
    b = np.array([[-np.inf, np.inf]])
    with bipp_ss.StandardSynthesis(inp.pix, inp.wl, b, n_eig=4, precision="split_fp16") as ss:
        rc = bipp_ss.load().bipp_ss_debug_fail_wait(ss.h, 2)
        assert rc == bipp_ss.BIPP_ERR_INVALID_ARG
