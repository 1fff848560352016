"""The spectrum entry point that allocates no device memory.

Some callers cannot let a library allocate device memory during a call, e.g.
a service that has reserved all HBM up front for resident meshes and request
buffers.  ifilt_spectrum_noalloc keeps its scratch in a fixed array inside the
library; this test calls it through the C ABI twice in a row and checks each
result against ifilt_spectrum on the same filtered fields.  The file is named
to be collected last; it also passes alone in a fresh process.
"""

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_noalloc_spectrum_matches_ifilt_spectrum_twice(lib):
    import torch
    m = synth.icosphere(4, radius=6371.0, jitter=0.2, seed=71)
    m["ocean"] = synth.land_mask(m["coords"], 0.3, seed=72)
    h = lib.prepare_mesh(m, "vertex_scalar", max_order=2)
    rng = np.random.default_rng(8)
    ks = synth.log_wavenumbers(4000.0, 300.0, 7)
    f = torch.tensor(rng.normal(size=(3, 1, h.info["n_in"])), device="cuda")
    out, stats, st = lib.solve(h, f, ks, order=2, tol=1e-12)
    assert st == 0
    E, spec, kmid = lib.spectrum(h, out, ks)
    for _ in range(2):
        E2, spec2, kmid2 = lib.spectrum_noalloc(h, out, ks)
        assert np.allclose(E2, E, rtol=1e-13, atol=0)
        assert np.allclose(spec2, spec, rtol=1e-9, atol=1e-14 * np.abs(spec).max())
        assert np.allclose(kmid2, kmid, rtol=1e-15)
    # a different, smaller request reuses the same array without stale values
    E3, spec3, _ = lib.spectrum_noalloc(h, out[:1, :3], ks[:3])
    assert np.allclose(E3, E[:1, :3], rtol=1e-13)
    assert np.allclose(spec3, spec[:1, :2], rtol=1e-9, atol=1e-14 * np.abs(spec).max())
    h.release()


def test_noalloc_spectrum_rejects_oversized_requests(lib):
    import torch
    m = synth.icosphere(1, radius=6371.0, jitter=0.0)
    h = lib.prepare_mesh(m, "vertex_scalar", max_order=1)
    ks = np.geomspace(1e-3, 1.0, 40)
    filt = torch.zeros((13, 40, 1, h.info["n_out"]), dtype=torch.float64, device="cuda")
    with pytest.raises(lib.IfiltError) as e:
        lib.spectrum_noalloc(h, filt, ks)
    assert e.value.status == -1
    h.release()
