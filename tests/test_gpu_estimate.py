"""The parameter-estimation pre-pass on the GPU (Sec. 2.6): N_eig from an
energy fraction and k-means level bounds from the GPU eigenvalues, against the
oracle's eigensolve and estimation."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from oracle import estimate as oest
from paper_2310_09200_b300 import bipp_ss, inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("eig_mode", ["jacobi64", "mixed"])
def test_prepass_energy_and_kmeans_match_oracle(eig_mode):
    inp = inputs.make_config(0, n_t=4)
    steps = [oracle.geneig(V, oracle.gram(p, inp.wl))[0] for p, V in zip(inp.st_xyz, inp.vis)]
    for f in (0.5, 0.9, 0.99):
        want = max(oest.energy_n_eig(mu, f) for mu in steps)
        assert bipp_ss.estimate_n_eig(inp.st_xyz, inp.vis, inp.wl, f, precision="fp64", eig_mode=eig_mode) == want
    pooled = np.concatenate([mu[: inp.n_eig] for mu in steps])
    bounds, pooled_gpu = bipp_ss.estimate_level_bounds(inp.st_xyz, inp.vis, inp.wl, inp.n_eig, 4, method="kmeans",
                                                       precision="fp64", eig_mode=eig_mode)
    np.testing.assert_allclose(pooled_gpu, pooled, rtol=1e-10)
    np.testing.assert_allclose(bounds, np.array(oest.kmeans_bounds(pooled, 4)), rtol=1e-9)
