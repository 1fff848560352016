"""Python binding of libifilt (include/ifilt.h): argument marshalling only.

Every computation runs inside the compiled library; this module converts numpy
arrays and torch CUDA tensors to pointers, checks shapes and dtypes, and raises
IfiltError for a negative status.  There is no fallback: if the library is not
built, `load()` raises.
"""

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libifilt.so")

VERTEX_SCALAR, VERTEX_VECTOR, CELL, VERTEX_VORONOI, CELL_CIRCUMCENTER = 0, 1, 2, 3, 4
GEOM_PLANAR_PERIODIC, GEOM_PLANAR, GEOM_SPHERE = 0, 1, 2
PREC_FP64, PREC_FP32_IR, PREC_BF16_IR = 0, 1, 2
METHOD_PLAIN, METHOD_BATCHED = 0, 1
N2_AUTO, N2_REAL, N2_COMPLEX = 0, 1, 2
PRECOND_NONE, PRECOND_JACOBI, PRECOND_MG = 0, 1, 2
REORDER_NONE, REORDER_RCM, REORDER_HILBERT = 0, 1, 2
MG_V, MG_W12 = 0, 1
MG_MAX_LEVELS = 16
MAX_ORDER = 4
OK, NOT_CONVERGED = 0, 1
ECACHE = -6
SAVE_MULTIGRID = 1
EXPORT = dict(perm=0, k_rowptr=1, k_col=2, k_val=3, mass=4, g2_rowptr=5, g2_col=6, g2_val=7)
PLACEMENTS = {"vertex_scalar": VERTEX_SCALAR, "vertex_vector": VERTEX_VECTOR, "cell": CELL,
              "vertex_voronoi": VERTEX_VORONOI, "cell_circumcenter": CELL_CIRCUMCENTER}
GEOMS = {"planar_periodic": GEOM_PLANAR_PERIODIC, "planar": GEOM_PLANAR, "sphere": GEOM_SPHERE}


class IfiltError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"ifilt status {status}: {msg}")
        self.status = status


class MeshDesc(C.Structure):
    _fields_ = [("n_vert", C.c_int32), ("n_tri", C.c_int32), ("coords", C.c_void_p), ("tri", C.c_void_p),
                ("ocean", C.c_void_p), ("geometry", C.c_int32), ("period_x", C.c_double),
                ("period_y", C.c_double), ("radius", C.c_double), ("placement", C.c_int32),
                ("max_order", C.c_int32), ("reorder", C.c_int32), ("cell_A", C.c_double),
                ("ell_slice", C.c_int32), ("mg_strength", C.c_double)]


class SolveOpts(C.Structure):
    _fields_ = [("order", C.c_int32), ("tol", C.c_double), ("max_iter", C.c_int32), ("precision", C.c_int32),
                ("method", C.c_int32), ("n2_solver", C.c_int32), ("precond", C.c_int32),
                ("check_every", C.c_int32), ("inner_tol", C.c_double), ("max_lanes", C.c_int32),
                ("err_tol", C.c_double), ("mg_cycle", C.c_int32)]


class SolveItem(C.Structure):
    _fields_ = [("mesh", C.c_void_p), ("opts", SolveOpts), ("n_fields", C.c_int32), ("fields", C.c_void_p),
                ("n_k", C.c_int32), ("k", C.c_void_p), ("out", C.c_void_p), ("stats", C.c_void_p)]


class ColStats(C.Structure):
    _fields_ = [("iters", C.c_int32), ("refinements", C.c_int32), ("status", C.c_int32), ("pad", C.c_int32),
                ("rel_residual", C.c_double), ("err_bound", C.c_double)]


class MeshInfo(C.Structure):
    _fields_ = [("placement", C.c_int32), ("geometry", C.c_int32), ("max_order", C.c_int32),
                ("reorder", C.c_int32), ("n_rows", C.c_int32), ("n_in", C.c_int32), ("n_out", C.c_int32),
                ("n_comp", C.c_int32), ("nnz_k", C.c_int64), ("nnz_g2", C.c_int64), ("ell_slice", C.c_int32),
                ("ell_width_k", C.c_int32), ("ell_width_g2", C.c_int32), ("pad", C.c_int32),
                ("device_bytes", C.c_int64)]


class ServerOpts(C.Structure):
    _fields_ = [("memory_budget", C.c_int64), ("reserve", C.c_int64), ("max_lanes", C.c_int32),
                ("check_every", C.c_int32)]


class RequestInfo(C.Structure):
    _fields_ = [("state", C.c_int32), ("status", C.c_int32), ("columns", C.c_int32), ("columns_done", C.c_int32),
                ("t_submit", C.c_double), ("t_start", C.c_double), ("t_done", C.c_double)]


class KernelProfile(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("launches", C.c_int64), ("samples", C.c_int64),
                ("sampled_ms", C.c_double), ("bytes_per_launch", C.c_double)]


COL_STATS_DTYPE = np.dtype([("iters", np.int32), ("refinements", np.int32), ("status", np.int32),
                            ("pad", np.int32), ("rel_residual", np.float64), ("err_bound", np.float64)])

class MultigridInfo(C.Structure):
    _fields_ = [("n_levels", C.c_int32), ("rows", C.c_int32 * MG_MAX_LEVELS), ("nnz_s", C.c_int64 * MG_MAX_LEVELS),
                ("nnz_p", C.c_int64 * MG_MAX_LEVELS)]


MG_EXPORT = {"s_rowptr": 0, "s_col": 1, "s_val": 2, "p_rowptr": 3, "p_col": 4, "p_val": 5, "dk": 6, "dm": 7,
             "omega": 8}

# every symbol include/ifilt.h declares
SYMBOLS = ["ifilt_prepare_mesh", "ifilt_prepare_mesh_host", "ifilt_mesh_upload", "ifilt_release_mesh", "ifilt_mesh_info", "ifilt_mesh_export",
           "ifilt_mesh_multigrid", "ifilt_mesh_multigrid_export", "ifilt_mesh_export_gn", "ifilt_mesh_key",
           "ifilt_mesh_get_key",
           "ifilt_mesh_save", "ifilt_mesh_load_host", "ifilt_solve",
           "ifilt_solve_many", "ifilt_spectrum", "ifilt_spectrum_noalloc", "ifilt_solve_scratch_bytes", "ifilt_profile_enable", "ifilt_profile_read",
           "ifilt_profile_reset", "ifilt_last_error", "ifilt_version", "ifilt_server_create",
           "ifilt_server_submit", "ifilt_server_wait", "ifilt_server_forget", "ifilt_server_now",
           "ifilt_server_destroy"]

_lib = None


def load(path=None):
    """Load libifilt.so (once).  Raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"{p} is missing: build it with `python -m paper_2404_07398_gb300.build`")
    lib = C.CDLL(p)
    vp, i32, i64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    lib.ifilt_prepare_mesh.argtypes = [C.POINTER(MeshDesc), vp, C.POINTER(vp)]
    lib.ifilt_prepare_mesh.restype = i32
    lib.ifilt_prepare_mesh_host.argtypes = [C.POINTER(MeshDesc), C.POINTER(vp)]
    lib.ifilt_prepare_mesh_host.restype = i32
    lib.ifilt_mesh_upload.argtypes = [vp, vp]
    lib.ifilt_mesh_upload.restype = i32
    lib.ifilt_release_mesh.argtypes = [vp]
    lib.ifilt_release_mesh.restype = None
    lib.ifilt_mesh_info.argtypes = [vp, C.POINTER(MeshInfo)]
    lib.ifilt_mesh_info.restype = i32
    lib.ifilt_mesh_export.argtypes = [vp, i32, vp, C.c_size_t]
    lib.ifilt_mesh_export.restype = i32
    lib.ifilt_mesh_multigrid.argtypes = [vp, C.POINTER(MultigridInfo)]
    lib.ifilt_mesh_multigrid.restype = i32
    lib.ifilt_mesh_multigrid_export.argtypes = [vp, i32, i32, vp, C.c_size_t, C.POINTER(C.c_size_t)]
    lib.ifilt_mesh_multigrid_export.restype = i32
    lib.ifilt_mesh_export_gn.argtypes = [vp, i32, i32, vp, C.c_size_t, C.POINTER(C.c_size_t)]
    lib.ifilt_mesh_export_gn.restype = i32
    lib.ifilt_mesh_key.argtypes = [C.POINTER(MeshDesc), C.POINTER(C.c_uint64)]
    lib.ifilt_mesh_key.restype = i32
    lib.ifilt_mesh_get_key.argtypes = [vp, C.POINTER(C.c_uint64)]
    lib.ifilt_mesh_get_key.restype = i32
    lib.ifilt_mesh_save.argtypes = [vp, C.c_char_p, i32]
    lib.ifilt_mesh_save.restype = i32
    lib.ifilt_mesh_load_host.argtypes = [C.c_char_p, C.c_uint64, C.POINTER(vp)]
    lib.ifilt_mesh_load_host.restype = i32
    lib.ifilt_solve.argtypes = [vp, C.POINTER(SolveOpts), i32, vp, i32, vp, vp, vp, vp]
    lib.ifilt_solve.restype = i32
    lib.ifilt_solve_many.argtypes = [i32, C.POINTER(SolveItem), vp]
    lib.ifilt_solve_many.restype = i32
    lib.ifilt_spectrum.argtypes = [vp, i32, i32, vp, vp, vp, vp, vp, vp]
    lib.ifilt_spectrum.restype = i32
    lib.ifilt_spectrum_noalloc.argtypes = [vp, i32, i32, vp, vp, vp, vp, vp, vp]
    lib.ifilt_spectrum_noalloc.restype = i32
    lib.ifilt_solve_scratch_bytes.argtypes = [vp, C.POINTER(SolveOpts), i32, i32]
    lib.ifilt_solve_scratch_bytes.restype = C.c_size_t
    lib.ifilt_profile_enable.argtypes = [i32]
    lib.ifilt_profile_enable.restype = None
    lib.ifilt_profile_read.argtypes = [C.POINTER(KernelProfile), i32]
    lib.ifilt_profile_read.restype = i32
    lib.ifilt_profile_reset.argtypes = []
    lib.ifilt_profile_reset.restype = None
    lib.ifilt_last_error.argtypes = []
    lib.ifilt_last_error.restype = C.c_char_p
    lib.ifilt_version.argtypes = []
    lib.ifilt_version.restype = C.c_char_p
    lib.ifilt_server_create.argtypes = [C.POINTER(ServerOpts), C.POINTER(vp)]
    lib.ifilt_server_create.restype = i32
    lib.ifilt_server_submit.argtypes = [vp, vp, C.POINTER(SolveOpts), i32, vp, i32, vp, vp, vp, C.POINTER(i64)]
    lib.ifilt_server_submit.restype = i32
    lib.ifilt_server_wait.argtypes = [vp, i64, i32, C.POINTER(RequestInfo)]
    lib.ifilt_server_wait.restype = i32
    lib.ifilt_server_forget.argtypes = [vp, i64]
    lib.ifilt_server_forget.restype = i32
    lib.ifilt_server_now.argtypes = [vp]
    lib.ifilt_server_now.restype = dbl
    lib.ifilt_server_destroy.argtypes = [vp]
    lib.ifilt_server_destroy.restype = None
    _lib = lib
    return lib


def _check(st):
    if st < 0:
        raise IfiltError(st, load().ifilt_last_error().decode())
    return st


def _stream_ptr(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(a):
    """Pointer of a numpy array or torch tensor (contiguous)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return C.c_void_p(a.ctypes.data)
    assert a.is_contiguous()
    return C.c_void_p(a.data_ptr())


def _info(handle):
    info = MeshInfo()
    _check(load().ifilt_mesh_info(handle, C.byref(info)))
    return {f: getattr(info, f) for f, _ in MeshInfo._fields_ if f != "pad"}


class Mesh:
    """A prepared mesh (device-resident handle)."""

    def __init__(self, handle):
        self.handle = handle
        self.info = _info(handle)

    def upload(self, stream=None):
        _check(load().ifilt_mesh_upload(self.handle, _stream_ptr(stream)))
        self.info = _info(self.handle)   # device layout fields are known now

    def release(self):
        if self.handle:
            load().ifilt_release_mesh(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.release()
        except Exception:
            pass

    def export(self, what):
        key = EXPORT[what]
        n = self.info["n_rows"]
        nv = 2 if self.info["placement"] == VERTEX_VECTOR else 1
        sizes = {"perm": (n, np.int32), "k_rowptr": (n + 1, np.int64), "k_col": (self.info["nnz_k"], np.int32),
                 "k_val": (self.info["nnz_k"] * nv, np.float64), "mass": (n, np.float64),
                 "g2_rowptr": (n + 1 if self.info["nnz_g2"] else 0, np.int64),
                 "g2_col": (self.info["nnz_g2"], np.int32), "g2_val": (self.info["nnz_g2"] * nv, np.float64)}
        cnt, dt = sizes[what]
        out = np.zeros(max(int(cnt), 1), dtype=dt)
        _check(load().ifilt_mesh_export(self.handle, key, _ptr(out), out.nbytes))
        return out[:cnt]

    def export_gn(self, order, part):
        """G_n = K (M^-1 K)^(n-1) for 2 <= n <= max_order: part "rowptr", "col" or "val"."""
        p = {"rowptr": 0, "col": 1, "val": 2}[part]
        need = C.c_size_t(0)
        lib = load()
        _check(lib.ifilt_mesh_export_gn(self.handle, order, p, None, 0, C.byref(need)))
        dt = {0: np.int64, 1: np.int32, 2: np.float64}[p]
        out = np.zeros(max(need.value // np.dtype(dt).itemsize, 1), dtype=dt)
        _check(lib.ifilt_mesh_export_gn(self.handle, order, p, _ptr(out), out.nbytes, C.byref(need)))
        return out[: need.value // out.itemsize]

    @property
    def key(self):
        """Key of the descriptor the mesh was prepared from (see mesh_key)."""
        k = C.c_uint64(0)
        _check(load().ifilt_mesh_get_key(self.handle, C.byref(k)))
        return k.value

    def save(self, path, multigrid=False):
        """Write the host half (and the multigrid hierarchy) to a cache file."""
        _check(load().ifilt_mesh_save(self.handle, os.fsencode(path), SAVE_MULTIGRID if multigrid else 0))

    def multigrid(self):
        """Shape of the multigrid hierarchy (built on the host if needed)."""
        info = MultigridInfo()
        _check(load().ifilt_mesh_multigrid(self.handle, C.byref(info)))
        L = info.n_levels
        return {"levels": L, "rows": list(info.rows[:L]), "nnz_s": list(info.nnz_s[:L]),
                "nnz_p": list(info.nnz_p[:L])}

    def multigrid_export(self, level, what):
        """One array of multigrid level `level` (see MG_EXPORT)."""
        g = self.multigrid()
        n = g["rows"][level]
        blk = self.info["placement"] == VERTEX_VECTOR
        cap = {"s_rowptr": (n + 1, np.int64), "s_col": (g["nnz_s"][level], np.int32),
               "s_val": (g["nnz_s"][level] * (4 if blk else 2), np.float64), "p_rowptr": (n + 1, np.int64),
               "p_col": (g["nnz_p"][level], np.int32), "p_val": (g["nnz_p"][level] * (2 if blk else 1), np.float64),
               "dk": (n, np.float64), "dm": (n, np.float64), "omega": (2, np.float64)}
        cnt, dt = cap[what]
        out = np.zeros(max(int(cnt), 1), dtype=dt)
        wrote = C.c_size_t(0)
        _check(load().ifilt_mesh_multigrid_export(self.handle, level, MG_EXPORT[what], _ptr(out), out.nbytes,
                                                  C.byref(wrote)))
        return out[: wrote.value // out.itemsize]


def _desc(mesh, placement, max_order, reorder, cell_A, ell_slice, mg_strength=0.0):
    coords = np.ascontiguousarray(mesh["coords"], dtype=np.float64)
    tri = np.ascontiguousarray(mesh["tri"], dtype=np.int32)
    ocean = mesh.get("ocean")
    ocean = None if ocean is None else np.ascontiguousarray(ocean, dtype=np.uint8)
    d = MeshDesc(n_vert=coords.shape[0], n_tri=tri.shape[0], coords=coords.ctypes.data, tri=tri.ctypes.data,
                 ocean=None if ocean is None else ocean.ctypes.data, geometry=GEOMS[mesh["geom"]],
                 period_x=float(mesh.get("period_x", 0.0)), period_y=float(mesh.get("period_y", 0.0)),
                 radius=float(mesh.get("radius", 0.0)), placement=PLACEMENTS.get(placement, placement),
                 max_order=max_order, reorder=reorder, cell_A=float(cell_A), ell_slice=ell_slice,
                 mg_strength=float(mg_strength))
    return d, (coords, tri, ocean)   # keep the arrays alive with the descriptor


def prepare_mesh(mesh, placement, max_order=2, reorder=1, cell_A=0.0, ell_slice=0, stream=None, mg_strength=0.0):
    """`mesh` is a dict with coords [V][2|3], tri [T][3], geom, period_x, period_y,
    radius and optional ocean [V] (uint8).  Returns a device-resident Mesh."""
    d, keep = _desc(mesh, placement, max_order, reorder, cell_A, ell_slice, mg_strength)
    h = C.c_void_p()
    _check(load().ifilt_prepare_mesh(C.byref(d), _stream_ptr(stream), C.byref(h)))
    return Mesh(h)


def prepare_mesh_host(mesh, placement, max_order=2, reorder=1, cell_A=0.0, ell_slice=0, mg_strength=0.0):
    """Host half of the preparation (no GPU needed): the Mesh answers info and
    export; `upload()` makes it solvable."""
    d, keep = _desc(mesh, placement, max_order, reorder, cell_A, ell_slice, mg_strength)
    h = C.c_void_p()
    _check(load().ifilt_prepare_mesh_host(C.byref(d), C.byref(h)))
    return Mesh(h)


def mesh_key(mesh, placement, max_order=2, reorder=1, cell_A=0.0, ell_slice=0, mg_strength=0.0):
    """64-bit key of a mesh descriptor (names its cache file)."""
    d, keep = _desc(mesh, placement, max_order, reorder, cell_A, ell_slice, mg_strength)
    k = C.c_uint64(0)
    _check(load().ifilt_mesh_key(C.byref(d), C.byref(k)))
    return k.value


def load_mesh_host(path, key=0):
    """Read a cache file written by Mesh.save into a host-only Mesh; `key` != 0
    must match the key of the descriptor it was prepared from."""
    h = C.c_void_p()
    _check(load().ifilt_mesh_load_host(os.fsencode(path), key, C.byref(h)))
    return Mesh(h)


def prepare_mesh_cached(mesh, placement, cache_dir, max_order=2, reorder=1, cell_A=0.0, ell_slice=0,
                        multigrid=True, upload=True, stream=None, mg_strength=0.0):
    """prepare_mesh through a directory of cache files named by the descriptor
    key: load the file if it is there and valid, else prepare on the host and
    write it (with the multigrid hierarchy if `multigrid`).  Returns
    (Mesh, hit) with the mesh uploaded if `upload`."""
    key = mesh_key(mesh, placement, max_order, reorder, cell_A, ell_slice, mg_strength)
    path = os.path.join(cache_dir, f"{key:016x}.ifmesh")
    hit = False
    try:
        m = load_mesh_host(path, key)
        hit = True
    except IfiltError as e:
        if e.status != ECACHE:
            raise
        m = prepare_mesh_host(mesh, placement, max_order, reorder, cell_A, ell_slice, mg_strength)
        os.makedirs(cache_dir, exist_ok=True)
        m.save(path, multigrid=multigrid)
    if upload:
        m.upload(stream)
    return m, hit


def solve_opts(order=1, tol=1e-9, precision=PREC_FP64, method=METHOD_BATCHED, n2_solver=N2_AUTO, max_iter=0,
               precond=0, check_every=0, inner_tol=0.0, max_lanes=0, err_tol=0.0, mg_cycle=0):
    return SolveOpts(order=order, tol=tol, max_iter=max_iter, precision=precision, method=method,
                     n2_solver=n2_solver, precond=precond, check_every=check_every, inner_tol=inner_tol,
                     max_lanes=max_lanes, err_tol=err_tol, mg_cycle=mg_cycle)


def solve(mesh, fields, k, out=None, stream=None, **opts):
    """fields: torch CUDA float64 [F][n_comp][n_in]; k: 1-D array of wavenumbers.
    Returns (out [F][K][n_comp][n_out] float64 CUDA tensor, stats structured array, status)."""
    import torch
    lib = load()
    info = mesh.info
    assert fields.is_cuda and fields.dtype == torch.float64 and fields.is_contiguous()
    F = fields.shape[0]
    assert tuple(fields.shape[1:]) == (info["n_comp"], info["n_in"]), (fields.shape, info)
    kk = np.ascontiguousarray(k, dtype=np.float64).ravel()
    K = kk.size
    if out is None:
        out = torch.empty((F, K, info["n_comp"], info["n_out"]), dtype=torch.float64, device=fields.device)
    assert out.is_contiguous() and out.dtype == torch.float64
    nsys = 2 if info["placement"] == CELL else 1
    stats = np.zeros(F * K * nsys, dtype=COL_STATS_DTYPE)
    o = solve_opts(**opts)
    st = lib.ifilt_solve(mesh.handle, C.byref(o), F, _ptr(fields), K, _ptr(kk), _ptr(out), _ptr(stats),
                         _stream_ptr(stream))
    _check(st)
    return out, stats.reshape(F, K, nsys), st


def solve_many(jobs, stream=None):
    """Several solves at once; `jobs` is a list of (mesh, fields, k, out_or_None, opts-dict).
    Returns [(out, stats)] in order and the worst status."""
    import torch
    items = (SolveItem * len(jobs))()
    keep = []
    results = []
    for i, (mesh, fields, k, out, opts) in enumerate(jobs):
        info = mesh.info
        assert fields.is_cuda and fields.dtype == torch.float64 and fields.is_contiguous()
        F = fields.shape[0]
        assert tuple(fields.shape[1:]) == (info["n_comp"], info["n_in"])
        kk = np.ascontiguousarray(k, dtype=np.float64).ravel()
        if out is None:
            out = torch.empty((F, kk.size, info["n_comp"], info["n_out"]), dtype=torch.float64, device=fields.device)
        nsys = 2 if info["placement"] == CELL else 1
        stats = np.zeros(F * kk.size * nsys, dtype=COL_STATS_DTYPE)
        items[i].mesh = mesh.handle
        items[i].opts = solve_opts(**opts)
        items[i].n_fields = F
        items[i].fields = fields.data_ptr()
        items[i].n_k = kk.size
        items[i].k = kk.ctypes.data
        items[i].out = out.data_ptr()
        items[i].stats = stats.ctypes.data
        keep.append(kk)
        results.append((out, stats.reshape(F, kk.size, nsys)))
    st = load().ifilt_solve_many(len(jobs), items, _stream_ptr(stream))
    _check(st)
    return results, st


def _check_filtered(mesh, filtered, K):
    """The spectrum kernels read filtered[F][K][n_comp][n_out] as one block of
    float64 on the device: refuse any other shape, type or layout up front."""
    import torch
    info = mesh.info
    if not (isinstance(filtered, torch.Tensor) and filtered.is_cuda and filtered.dtype == torch.float64
            and filtered.is_contiguous() and filtered.dim() == 4):
        raise ValueError("filtered must be a contiguous CUDA float64 tensor [F][K][n_comp][n_out]")
    want = (K, info["n_comp"], info["n_out"])
    if tuple(filtered.shape[1:]) != want:
        raise ValueError(f"filtered has shape {tuple(filtered.shape)}, expected [F]{list(want)}")


def spectrum(mesh, filtered, k, stream=None):
    """filtered: CUDA float64 [F][K][n_comp][n_out] (as `solve` returns); k ascending.
    Returns (energy [F][K], spec [F][K-1], kmid [K-1]) as numpy arrays."""
    lib = load()
    kk = np.ascontiguousarray(k, dtype=np.float64).ravel()
    _check_filtered(mesh, filtered, kk.size)
    F, K = filtered.shape[0], kk.size
    energy = np.zeros((F, K))
    spec = np.zeros((F, max(K - 1, 1)))
    kmid = np.zeros(max(K - 1, 1))
    _check(lib.ifilt_spectrum(mesh.handle, F, K, _ptr(kk), _ptr(filtered), _ptr(energy), _ptr(spec),
                              _ptr(kmid), _stream_ptr(stream)))
    return energy, spec[:, :K - 1], kmid[:K - 1]


def spectrum_noalloc(mesh, filtered, k, stream=None):
    """As `spectrum`, through the entry point that takes no device memory from
    any allocator (its scratch is a fixed array inside the library)."""
    lib = load()
    kk = np.ascontiguousarray(k, dtype=np.float64).ravel()
    _check_filtered(mesh, filtered, kk.size)
    F, K = filtered.shape[0], kk.size
    energy = np.zeros((F, K))
    spec = np.zeros((F, max(K - 1, 1)))
    kmid = np.zeros(max(K - 1, 1))
    _check(lib.ifilt_spectrum_noalloc(mesh.handle, F, K, _ptr(kk), _ptr(filtered), _ptr(energy), _ptr(spec),
                                      _ptr(kmid), _stream_ptr(stream)))
    return energy, spec[:, :K - 1], kmid[:K - 1]


def scratch_bytes(mesh, F, K, **opts):
    o = solve_opts(**opts)
    return load().ifilt_solve_scratch_bytes(mesh.handle, C.byref(o), F, K)


def profile_enable(on=True):
    load().ifilt_profile_enable(1 if on else 0)


def profile_reset():
    load().ifilt_profile_reset()


def profile_read():
    lib = load()
    n = lib.ifilt_profile_read(None, 0)
    arr = (KernelProfile * max(n, 1))()
    lib.ifilt_profile_read(arr, n)
    return [dict(name=a.name.decode(), launches=a.launches, samples=a.samples, sampled_ms=a.sampled_ms,
                 bytes_per_launch=a.bytes_per_launch) for a in arr[:n]]


def version():
    return load().ifilt_version().decode()


class Server:
    """A serving loop over resident prepared meshes (continuous batching).

    submit() queues a request and returns its id; the caller keeps `fields`,
    `out` and `stats` alive until wait() reports it done."""

    def __init__(self, memory_budget=0, reserve=0, max_lanes=0, check_every=0):
        o = ServerOpts(memory_budget=memory_budget, reserve=reserve, max_lanes=max_lanes, check_every=check_every)
        h = C.c_void_p()
        _check(load().ifilt_server_create(C.byref(o), C.byref(h)))
        self.handle = h
        self._keep = {}

    def submit(self, mesh, fields, k, out=None, **opts):
        import torch
        info = mesh.info
        assert fields.is_cuda and fields.dtype == torch.float64 and fields.is_contiguous()
        F = fields.shape[0]
        kk = np.ascontiguousarray(k, dtype=np.float64).ravel()
        K = kk.size
        if out is None:
            out = torch.empty((F, K, info["n_comp"], info["n_out"]), dtype=torch.float64, device=fields.device)
        nsys = 2 if info["placement"] == CELL else 1
        stats = np.zeros(F * K * nsys, dtype=COL_STATS_DTYPE)
        o = solve_opts(**opts)
        rid = C.c_int64()
        _check(load().ifilt_server_submit(self.handle, mesh.handle, C.byref(o), F, _ptr(fields), K, _ptr(kk),
                                          _ptr(out), _ptr(stats), C.byref(rid)))
        self._keep[rid.value] = (fields, out, stats, mesh)
        return rid.value

    def wait(self, rid, timeout_ms=0):
        """Returns (state, info dict); state 2 = done, 3 = failed."""
        i = RequestInfo()
        _check(load().ifilt_server_wait(self.handle, rid, int(timeout_ms), C.byref(i)))
        d = {f: getattr(i, f) for f, _ in RequestInfo._fields_}
        return d["state"], d

    def result(self, rid):
        """(out, stats) of a finished request; forgets it."""
        fields, out, stats, mesh = self._keep.pop(rid)
        _check(load().ifilt_server_forget(self.handle, rid))
        nsys = 2 if mesh.info["placement"] == CELL else 1
        return out, stats.reshape(out.shape[0], out.shape[1], nsys)

    def now(self):
        return load().ifilt_server_now(self.handle)

    def close(self):
        if self.handle:
            load().ifilt_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
