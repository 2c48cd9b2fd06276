"""Effect of the Gram matrix (App. A) on synthetic SKA-Low-like data: one
1000 Jy source observed by the 128 stations of the layout's core in one epoch,
imaged with all eigenpairs at 53 MHz and 89 MHz with the NUFFT (as App. A
does) twice: with the sinc Gram matrix (the least-squares image) and with
G = I (the back-projected image). Both match the oracle; their difference is
small (baselines >> wavelength) and larger at the lower frequency, where the
Gram matrix's off-diagonal terms are larger."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2310_09200_b300 import bipp_ss, inputs

pytestmark = pytest.mark.gpu


def _core(n=128):
    rng = np.random.default_rng(1001)
    p0 = inputs.layout_lognormal(512, 1000.0, 1.0, 20.0, 65000.0, 5.0, 35.0, rng)
    return p0[np.argsort(np.linalg.norm(p0[:, :2], axis=1))[:n]]


def test_gram_effect_appendix_a():
    p = _core()
    n = p.shape[0]
    b = np.array([[-np.inf, np.inf]])
    diff = {}
    for f_mhz, fov_deg in [(53.0, 1.16692), (89.0, 0.7002)]:
        wl = 299.792458 / f_mhz
        V = inputs.visibilities(p, wl, np.array([[0.0, 0.0, 1.0]]), np.array([1000.0]), None, None)
        pix = inputs.pixel_grid(49, fov_deg / 2)  # odd: the centre pixel is the source's direction
        imgs = {}
        for gi in (False, True):
            want, *_ = oracle.ss_step(pix, wl, b, n, p, V, gram_identity=gi)
            with bipp_ss.StandardSynthesis(pix, wl, b, n_eig=n, synthesis="nufft", nufft_eps=1e-6,
                                           gram_identity=gi) as ss:
                ss.collect_batch([p], [V])
                got = ss.get()
            err = np.linalg.norm(got - want) / np.linalg.norm(want)
            assert err <= 1e-4, (f_mhz, gi, err)
            assert np.argmax(got[:, 0]) == np.argmax(want[:, 0]) == 24 + 49 * 24  # peak at the source
            imgs[gi] = got
        diff[f_mhz] = np.linalg.norm(imgs[False] - imgs[True]) / np.linalg.norm(imgs[True])
    assert 0.0 < diff[89.0] < diff[53.0] < 0.05, diff
