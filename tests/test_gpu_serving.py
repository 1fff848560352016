"""Serving: requests on resident meshes through the continuous-batching server.

A request's result must be the same (within the solve tolerance) when it runs
alone and when its columns share batches with other requests, and must match
the FP64 oracle.
"""

import time

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _sphere(level, seed):
    m = synth.icosphere(level, radius=6371.0, jitter=0.2, seed=seed)
    m["ocean"] = synth.land_mask(m["coords"], 0.3, seed=seed + 1)
    return m


def _wait_all(srv, ids, timeout_s=120):
    t0 = time.time()
    infos = {}
    for rid in ids:
        while True:
            state, info = srv.wait(rid, 200)
            if state >= 2:
                infos[rid] = info
                break
            assert time.time() - t0 < timeout_s, "request did not finish"
    return infos


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_request_same_alone_and_in_mix(lib):
    import torch
    m1, m2 = _sphere(4, 81), _sphere(3, 83)
    h1 = lib.prepare_mesh(m1, "vertex_scalar", max_order=2)
    h2 = lib.prepare_mesh(m2, "vertex_scalar", max_order=2)
    rng = np.random.default_rng(11)
    fa = torch.tensor(rng.normal(size=(2, 1, h1.info["n_in"])), device="cuda")
    fb = torch.tensor(rng.normal(size=(3, 1, h2.info["n_in"])), device="cuda")
    fc = torch.tensor(rng.normal(size=(1, 1, h1.info["n_in"])), device="cuda")
    ka = synth.log_wavenumbers(4000.0, 300.0, 5)
    kb = synth.log_wavenumbers(6000.0, 800.0, 7)
    kc = synth.log_wavenumbers(3000.0, 500.0, 3)
    opts = dict(order=2, tol=1e-10, precision=lib.PREC_FP32_IR)
    srv = lib.Server(max_lanes=16, check_every=8)
    try:
        a0 = srv.submit(h1, fa, ka, **opts)
        _wait_all(srv, [a0])
        alone, st_alone = srv.result(a0)
        ids = [srv.submit(h1, fc, kc, order=1, tol=1e-10, precision=lib.PREC_FP32_IR),
               srv.submit(h2, fb, kb, **opts),
               srv.submit(h1, fa, ka, **opts),
               srv.submit(h1, fc, kc, **opts)]
        infos = _wait_all(srv, ids)
        for rid in ids:
            assert infos[rid]["state"] == 2 and infos[rid]["status"] == 0, infos[rid]
            assert infos[rid]["t_submit"] <= infos[rid]["t_start"] <= infos[rid]["t_done"]
        outs = {rid: srv.result(rid) for rid in ids}
    finally:
        srv.close()
    mixed = outs[ids[2]][0].cpu().numpy()
    alone = alone.cpu().numpy()
    P = oracle.build_problem(m1, "vertex_scalar")
    for f in range(2):
        ref, _ = oracle.filter_field(P, fa[f].cpu().numpy(), ka, 2)
        for j in range(ka.size):
            assert _rel(mixed[f, j, 0], alone[f, j, 0]) <= 1e-6
            assert _rel(mixed[f, j, 0], ref[j, 0]) <= 1e-6
    # the other mesh's request against the oracle as well
    P2 = oracle.build_problem(m2, "vertex_scalar")
    ob = outs[ids[1]][0].cpu().numpy()
    ref, _ = oracle.filter_field(P2, fb[1].cpu().numpy(), kb, 2)
    for j in range(kb.size):
        assert _rel(ob[1, j, 0], ref[j, 0]) <= 1e-6
    h1.release()
    h2.release()


def test_multigrid_requests_in_the_mix(lib):
    """Multigrid and unpreconditioned requests on one mesh run in separate
    engines of the server and both match the oracle."""
    import torch
    m = _sphere(4, 87)
    h = lib.prepare_mesh(m, "vertex_scalar", max_order=2)
    rng = np.random.default_rng(13)
    f = torch.tensor(rng.normal(size=(2, 1, h.info["n_in"])), device="cuda")
    ks = synth.log_wavenumbers(5000.0, 300.0, 4)
    srv = lib.Server(max_lanes=32, check_every=8)
    try:
        ids = [srv.submit(h, f, ks, order=2, tol=1e-10, precision=lib.PREC_FP32_IR, precond=pc)
               for pc in (lib.PRECOND_MG, lib.PRECOND_NONE, lib.PRECOND_MG)]
        infos = _wait_all(srv, ids)
        outs = [srv.result(rid)[0].cpu().numpy() for rid in ids]
    finally:
        srv.close()
    for rid in ids:
        assert infos[rid]["state"] == 2 and infos[rid]["status"] == 0
    P = oracle.build_problem(m, "vertex_scalar")
    for fi in range(2):
        ref, _ = oracle.filter_field(P, f[fi].cpu().numpy(), ks, 2)
        for o in outs:
            for j in range(ks.size):
                assert _rel(o[fi, j, 0], ref[j, 0]) <= 1e-6
    h.release()


def test_small_memory_budget_still_completes(lib):
    """A budget that holds only a few lanes at a time: columns wait for memory
    and are admitted as others retire."""
    import torch
    m = _sphere(6, 85)
    h = lib.prepare_mesh(m, "vertex_scalar", max_order=1)
    n = h.info["n_rows"]
    rng = np.random.default_rng(12)
    f = torch.tensor(rng.normal(size=(2, 1, h.info["n_in"])), device="cuda")
    ks = synth.log_wavenumbers(5000.0, 500.0, 6)
    # fixed tables (~1.3 MB) plus about four lanes of tiles (24 B per row and
    # lane) and two right-hand sides (16 B per row each)
    budget = 2 * 1024 * 1024 + n * (24 * 4 + 16 * 2)
    srv = lib.Server(memory_budget=budget, max_lanes=64, check_every=8)
    try:
        rid = srv.submit(h, f, ks, order=1, tol=1e-10, precision=lib.PREC_FP32_IR)
        info = _wait_all(srv, [rid])[rid]
        assert info["state"] == 2 and info["status"] == 0
        out, _ = srv.result(rid)
    finally:
        srv.close()
    P = oracle.build_problem(m, "vertex_scalar")
    ref, _ = oracle.filter_field(P, f[0].cpu().numpy(), ks, 1)
    res = out.cpu().numpy()
    for j in range(ks.size):
        assert _rel(res[0, j, 0], ref[j, 0]) <= 1e-6
    h.release()
