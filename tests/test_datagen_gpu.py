"""The device-side served-solve recipe (datagen.spd_request_device), GPU.

The served benchmark generates its requests on the GPU with torch's seeded
generator; this checks that they are what the recipe states: G's singular
values are the geometric sequence from 1 to 1e-10 (so F = G G^T has
condition ~1e20), the dd planes are normalised, generation is reproducible,
and F formed by the oracle is positive definite in dd arithmetic (the
oracle's Cholesky succeeds).
"""
from __future__ import annotations

import numpy as np
import pytest

import datagen
import oracle

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n", [64, 200])
def test_device_requests_follow_the_recipe(cuda_lib, n):
    mp = cuda_lib
    (gh, gl), (bh, bl) = datagen.spd_request_device(1234, n)
    G = (mp.to_numpy(gh), mp.to_numpy(gl))
    B = (mp.to_numpy(bh), mp.to_numpy(bl))
    assert G[0].shape == (n, 2 * n) and B[0].shape == (n, 4)
    for h, l in (G, B):
        assert np.all(h + l == h)
        assert np.all(np.abs(l) <= np.spacing(np.abs(h)) / 2)
    assert np.abs(B[0]).max() <= 1.0
    s = np.linalg.svd(G[0], compute_uv=False)
    want = np.geomspace(1.0, 1e-10, n)
    assert np.max(np.abs(s - want) / want) < 1e-4          # cond(G) = 1e10, cond(F) = 1e20
    again = datagen.spd_request_device(1234, n)
    assert np.array_equal(mp.to_numpy(again[0][0]), G[0])
    # positive definite in dd: the oracle's F = G G^T and its Cholesky
    Fd = oracle.dd_syrk("U", "N", (1.0, 0.0), G, (0.0, 0.0),
                        (np.zeros((n, n), order="F"), np.zeros((n, n), order="F")))
    Fs = tuple(np.asfortranarray(np.triu(P) + np.triu(P, 1).T) for P in Fd)
    _, _, info = oracle.dd_potrf("U", Fs)
    assert info == 0
