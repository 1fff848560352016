"""Mesh cache files (no GPU): a prepared mesh written by ifilt_mesh_save and
read by ifilt_mesh_load_host is the same mesh bit for bit, and every kind of
bad file is refused with IFILT_ECACHE, including files whose checksum was
recomputed over arrays that would index out of range."""

import os
import struct

import numpy as np
import pytest

import synth

PLACEMENTS = ["vertex_scalar", "vertex_vector", "cell", "vertex_voronoi", "cell_circumcenter"]
EXPORTS = ["perm", "k_rowptr", "k_col", "k_val", "mass", "g2_rowptr", "g2_col", "g2_val"]
MG_EXPORTS = ["s_rowptr", "s_col", "s_val", "p_rowptr", "p_col", "p_val", "dk", "dm", "omega"]
HEADER = 8 + 4 + 4 + 8 + 8 + 8    # magic, format, revision, key, payload bytes, payload hash


@pytest.fixture(scope="module")
def api():
    from paper_2404_07398_gb300 import api as a
    if not os.path.exists(a.LIB_PATH):
        from paper_2404_07398_gb300 import build
        build.build()
    a.load()
    return a


def _mesh(level=3, seed=91):
    m = synth.icosphere(level, radius=6371.0, jitter=0.05, seed=seed)
    m["ocean"] = synth.land_mask(m["coords"], 0.3, seed=seed + 1, polar_cap_deg=8.0)
    return m


def _same_mesh(a, b, multigrid=True):
    ia, ib = dict(a.info), dict(b.info)
    assert ia == ib
    for w in EXPORTS:
        x, y = a.export(w), b.export(w)
        assert x.dtype == y.dtype and np.array_equal(x.view(np.uint8), y.view(np.uint8)), w
    if multigrid:
        ga, gb = a.multigrid(), b.multigrid()
        assert ga == gb
        for level in range(ga["levels"]):
            for w in MG_EXPORTS:
                x, y = a.multigrid_export(level, w), b.multigrid_export(level, w)
                assert np.array_equal(x.view(np.uint8), y.view(np.uint8)), (level, w)


@pytest.mark.parametrize("placement", PLACEMENTS)
def test_round_trip_is_bit_exact(api, tmp_path, placement):
    m = _mesh()
    h = api.prepare_mesh_host(m, placement, max_order=2)
    assert h.key == api.mesh_key(m, placement, max_order=2) != 0
    path = tmp_path / "m.ifmesh"
    h.save(path, multigrid=True)
    assert sorted(os.listdir(tmp_path)) == ["m.ifmesh"]      # no temporary left behind
    g = api.load_mesh_host(path, key=h.key)
    assert g.key == h.key
    _same_mesh(h, g)
    h.release()
    g.release()


def test_hierarchy_built_on_demand_after_load(api, tmp_path):
    m = _mesh(seed=93)
    h = api.prepare_mesh_host(m, "cell", max_order=1)
    h.save(tmp_path / "c.ifmesh")                            # without the hierarchy
    g = api.load_mesh_host(tmp_path / "c.ifmesh")
    _same_mesh(h, g)                                         # both build it now, deterministically
    assert os.path.getsize(tmp_path / "c.ifmesh") < _saved_size(api, h, tmp_path / "c2.ifmesh")


def _saved_size(api, h, path):
    h.save(path, multigrid=True)
    return os.path.getsize(path)


def test_key_tracks_every_input(api):
    m = _mesh(2, 95)
    base = api.mesh_key(m, "vertex_scalar")
    assert api.mesh_key(m, "vertex_scalar") == base
    variants = []
    c = dict(m)
    c["coords"] = m["coords"].copy()
    c["coords"][7, 1] = np.nextafter(c["coords"][7, 1], np.inf)
    variants.append(api.mesh_key(c, "vertex_scalar"))
    c = dict(m)
    c["tri"] = m["tri"][:, [1, 2, 0]].copy()                 # same triangles, other corner order
    variants.append(api.mesh_key(c, "vertex_scalar"))
    c = dict(m)
    c["ocean"] = m["ocean"].copy()
    c["ocean"][3] ^= 1
    variants.append(api.mesh_key(c, "vertex_scalar"))
    c = dict(m)
    c["ocean"] = None
    variants.append(api.mesh_key(c, "vertex_scalar"))
    variants.append(api.mesh_key(m, "vertex_voronoi"))
    variants.append(api.mesh_key(m, "vertex_scalar", max_order=1))
    variants.append(api.mesh_key(m, "vertex_scalar", reorder=2))
    variants.append(api.mesh_key(m, "vertex_scalar", ell_slice=32))
    variants.append(api.mesh_key(m, "cell"))
    variants.append(api.mesh_key(m, "cell", cell_A=1.5))
    assert base not in variants and len(set(variants)) == len(variants)
    # ocean flags are taken as 0/1: any nonzero byte is ocean
    c = dict(m)
    c["ocean"] = (m["ocean"].astype(np.uint8) * 7).astype(np.uint8)
    assert api.mesh_key(c, "vertex_scalar") == base


def _saved(api, tmp_path, placement="vertex_scalar", multigrid=False):
    m = _mesh(2, 97)
    h = api.prepare_mesh_host(m, placement, max_order=2)
    path = tmp_path / "x.ifmesh"
    h.save(path, multigrid=multigrid)
    return h, path, bytearray(path.read_bytes())


def _refused(api, path, key=0):
    with pytest.raises(api.IfiltError) as e:
        api.load_mesh_host(path, key)
    assert e.value.status == api.ECACHE
    return str(e.value)


def test_bad_files_are_refused(api, tmp_path):
    h, path, raw = _saved(api, tmp_path)
    _refused(api, tmp_path / "missing.ifmesh")
    assert "another mesh" in _refused(api, path, key=h.key ^ 1)
    api.load_mesh_host(path, key=h.key).release()
    bad = tmp_path / "bad.ifmesh"
    cases = {
        "magic": lambda b: b.__setitem__(0, ord("J")),
        "format": lambda b: b.__setitem__(8, 99),
        "revision": lambda b: b.__setitem__(12, 99),
        "payload byte": lambda b: b.__setitem__(HEADER + 100, b[HEADER + 100] ^ 0x10),
        "last byte": lambda b: b.__setitem__(len(b) - 1, b[-1] ^ 1),
    }
    for name, edit in cases.items():
        b = bytearray(raw)
        edit(b)
        bad.write_bytes(bytes(b))
        _refused(api, bad)
    for cut in (4, HEADER - 1, HEADER + 20, len(raw) // 2, len(raw) - 1):
        bad.write_bytes(bytes(raw[:cut]))
        _refused(api, bad)
    bad.write_bytes(bytes(raw) + b"\0")
    _refused(api, bad)
    # a header that claims a huge payload is refused before anything is allocated
    b = bytearray(raw)
    struct.pack_into("<Q", b, 24, 1 << 40)
    bad.write_bytes(bytes(b))
    assert "truncated" in _refused(api, bad)
    h.release()


# ---- a restatement of the file hash, so that forged files pass the checksum
M64 = (1 << 64) - 1


def _mix64(z):
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def _rotl(x, r):
    return ((x << r) | (x >> (64 - r))) & M64


def _hash64(data, seed=0):
    acc = [_mix64((seed + 0x9E3779B97F4A7C15 * (i + 1)) & M64) for i in range(4)]
    n = len(data)
    full = n - n % 32
    words = np.frombuffer(bytes(data[:full]), dtype="<u8").reshape(-1, 4)
    for blk in words:
        for i in range(4):
            acc[i] = _mix64(acc[i] ^ int(blk[i]))
    if n % 32:
        last = bytes(data[full:]) + b"\0" * (32 - n % 32)
        for i, w in enumerate(struct.unpack("<4Q", last)):
            acc[i] = _mix64(acc[i] ^ w)
    return _mix64(acc[0] ^ _rotl(acc[1], 16) ^ _rotl(acc[2], 32) ^ _rotl(acc[3], 48) ^ _mix64(n))


def _reseal(b):
    payload = bytes(b[HEADER:])
    struct.pack_into("<QQ", b, 24, len(payload), _hash64(payload))
    return b


def _offsets(b):
    """Byte offsets of the first arrays of a payload (see the file layout)."""
    o = HEADER
    ints = struct.unpack_from("<9i", b, o)
    o += 36 + 8                                             # header ints, multigrid strength
    n = ints[4]
    off = {}
    cnt = struct.unpack_from("<Q", b, o)[0]
    off["perm"] = o + 8
    o += 8 + 4 * cnt
    cnt = struct.unpack_from("<Q", b, o)[0]
    off["mass"] = o + 8
    o += 8 + 8 * cnt
    o += 8                                                  # K: n, nval
    cnt = struct.unpack_from("<Q", b, o)[0]
    off["k_rowptr"] = o + 8
    o += 8 + 8 * cnt
    off["k_col_count"] = o
    off["k_col"] = o + 8
    return n, off


def test_checksum_restatement_matches(api, tmp_path):
    _, path, raw = _saved(api, tmp_path)
    assert bytes(_reseal(bytearray(raw))) == bytes(raw)


def test_forged_arrays_are_refused(api, tmp_path):
    h, path, raw = _saved(api, tmp_path)
    n, off = _offsets(raw)
    bad = tmp_path / "forged.ifmesh"

    def forge(edit):
        b = bytearray(raw)
        edit(b)
        bad.write_bytes(bytes(_reseal(b)))
        return _refused(api, bad)

    assert "operator K" in forge(lambda b: struct.pack_into("<i", b, off["k_col"], n))         # column out of range
    assert "operator K" in forge(lambda b: struct.pack_into("<i", b, off["k_col"], -1))
    assert "operator K" in forge(lambda b: struct.pack_into("<q", b, off["k_rowptr"] + 8, 10 ** 9))
    p0, p1 = struct.unpack_from("<2i", raw, off["perm"])
    assert "permutation" in forge(lambda b: struct.pack_into("<i", b, off["perm"] + 4, p0))    # duplicate
    assert "lumped mass" in forge(lambda b: struct.pack_into("<d", b, off["mass"], float("nan")))
    # an array count that runs past the end of the file
    assert "past the end" in forge(lambda b: struct.pack_into("<Q", b, off["k_col_count"], 1 << 40))
    h.release()


def test_forged_hierarchy_is_refused(api, tmp_path):
    h, path, raw = _saved(api, tmp_path, "cell", multigrid=True)
    g = h.multigrid()
    # the coarsest level's diagonal is the last array of the file: make it NaN
    b = bytearray(raw)
    struct.pack_into("<d", b, len(b) - 8, float("nan"))
    bad = tmp_path / "forged.ifmesh"
    bad.write_bytes(bytes(_reseal(b)))
    assert "multigrid" in _refused(api, bad)
    assert g["levels"] >= 2
    h.release()


def test_prepare_mesh_cached(api, tmp_path):
    m = _mesh(3, 99)
    d = tmp_path / "cache"
    a, hit = api.prepare_mesh_cached(m, "cell", d, upload=False)
    assert not hit and len(os.listdir(d)) == 1
    b, hit = api.prepare_mesh_cached(m, "cell", d, upload=False)
    assert hit
    _same_mesh(a, b)
    # a damaged file is prepared again and replaced
    f = d / os.listdir(d)[0]
    raw = bytearray(f.read_bytes())
    raw[HEADER + 64] ^= 0xFF
    f.write_bytes(bytes(raw))
    c, hit = api.prepare_mesh_cached(m, "cell", d, upload=False)
    assert not hit
    _same_mesh(a, c)
    e, hit = api.prepare_mesh_cached(m, "cell", d, upload=False)
    assert hit
    for x in (a, b, c, e):
        x.release()


def test_bad_arguments(api, tmp_path):
    import ctypes
    lib = api.load()
    h = api.prepare_mesh_host(_mesh(1, 3), "vertex_scalar", max_order=1)
    assert lib.ifilt_mesh_save(h.handle, os.fsencode(tmp_path / "a"), 4) == -1
    assert lib.ifilt_mesh_save(None, os.fsencode(tmp_path / "a"), 0) == -1
    assert lib.ifilt_mesh_save(h.handle, None, 0) == -1
    assert lib.ifilt_mesh_save(h.handle, os.fsencode(tmp_path / "no" / "such" / "dir"), 0) == api.ECACHE
    out = ctypes.c_void_p()
    assert lib.ifilt_mesh_load_host(None, 0, ctypes.byref(out)) == -1
    assert lib.ifilt_mesh_key(None, None) == -1
    h.release()
