"""Synthetic triangular meshes (seeded, deterministic).

Every mesh is returned as a dict with
  coords : float64 [V, 2] (planar) or [V, 3] (sphere, in the same length unit as `radius`)
  tri    : int32  [T, 3], counter-clockwise seen from outside / from +z
  geom   : "planar_periodic" | "sphere"
plus the geometry parameters (period_x, period_y or radius).
"""

import numpy as np


def periodic_split_square(nx, ny, h=1.0):
    """Doubly periodic regular grid of nx*ny squares, each bisected along the
    same diagonal (the construction of the paper's Fig. 2).

    Vertex (i, j) has id j*nx + i and sits at (i*h, j*h).  Square (i, j) with
    corners a=(i,j), b=(i+1,j), c=(i+1,j+1), d=(i,j+1) is split along a-c into
    the triangles (a, b, c) and (a, c, d).
    """
    i, j = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    i = i.ravel()
    j = j.ravel()
    coords = np.stack([i * h, j * h], axis=1).astype(np.float64)

    def vid(ii, jj):
        return (jj % ny) * nx + (ii % nx)

    a = vid(i, j)
    b = vid(i + 1, j)
    c = vid(i + 1, j + 1)
    d = vid(i, j + 1)
    t1 = np.stack([a, b, c], axis=1)
    t2 = np.stack([a, c, d], axis=1)
    tri = np.empty((2 * nx * ny, 3), dtype=np.int32)
    tri[0::2] = t1
    tri[1::2] = t2
    return dict(coords=coords, tri=tri, geom="planar_periodic",
                period_x=nx * h, period_y=ny * h, radius=0.0)


def periodic_equilateral(nx, ny, a=1.0):
    """Doubly periodic lattice of equilateral triangles with side a.

    Row j (ny even) holds nx vertices at x = (i + (j % 2)/2) * a, y = j*a*sqrt(3)/2;
    the periods are nx*a and ny*a*sqrt(3)/2, so the lattice tiles a rectangle.
    """
    if ny % 2:
        raise ValueError("ny must be even for a rectangular period")
    s3 = np.sqrt(3.0)
    i, j = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    i = i.ravel()
    j = j.ravel()
    coords = np.stack([(i + 0.5 * (j % 2)) * a, j * a * s3 / 2], axis=1)

    def vid(ii, jj):
        return (jj % ny) * nx + (ii % nx)

    tris = []
    for jj in range(ny):
        odd = jj % 2
        for ii in range(nx):
            # the two vertices of row jj+1 that sit half a side left/right of (ii, jj)
            v0, v1 = vid(ii, jj), vid(ii + 1, jj)
            u0, u1 = vid(ii - 1 + odd, jj + 1), vid(ii + odd, jj + 1)
            tris.append((v0, v1, u1))   # upward triangle
            tris.append((v0, u1, u0))   # downward triangle
    tri = np.asarray(tris, dtype=np.int32)
    return dict(coords=coords.astype(np.float64), tri=tri, geom="planar_periodic",
                period_x=nx * a, period_y=ny * a * s3 / 2, radius=0.0)


_PHI = (1.0 + 5.0 ** 0.5) / 2.0
_ICO_V = np.array([
    [-1, _PHI, 0], [1, _PHI, 0], [-1, -_PHI, 0], [1, -_PHI, 0],
    [0, -1, _PHI], [0, 1, _PHI], [0, -1, -_PHI], [0, 1, -_PHI],
    [_PHI, 0, -1], [_PHI, 0, 1], [-_PHI, 0, -1], [-_PHI, 0, 1],
], dtype=np.float64)
_ICO_F = np.array([
    [0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
    [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
    [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
    [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1],
], dtype=np.int64)


def _device(n):
    """Generator device: the GPU for big meshes when one is present."""
    import torch
    return "cuda" if (n > 2_000_000 and torch.cuda.is_available()) else "cpu"


def _subdivide(xyz, faces):
    """One 1-to-4 split of every face (torch tensors); midpoints projected to
    the unit sphere.  New vertices are appended in the order of their sorted
    edge key."""
    import torch
    nv = xyz.shape[0]
    a, b, c = faces[:, 0], faces[:, 1], faces[:, 2]
    lo = torch.stack([torch.minimum(a, b), torch.minimum(b, c), torch.minimum(c, a)])
    hi = torch.stack([torch.maximum(a, b), torch.maximum(b, c), torch.maximum(c, a)])
    key = (lo * nv + hi).reshape(-1)
    ukey, inv = torch.unique(key, sorted=True, return_inverse=True)
    inv = inv.reshape(3, -1)
    mid = xyz[ukey // nv] + xyz[ukey % nv]
    mid = mid / torch.linalg.norm(mid, dim=1, keepdim=True)
    new_xyz = torch.cat([xyz, mid], 0)
    mab, mbc, mca = inv[0] + nv, inv[1] + nv, inv[2] + nv
    f = torch.empty((faces.shape[0] * 4, 3), dtype=torch.int64, device=faces.device)
    f[0::4] = torch.stack([a, mab, mca], 1)
    f[1::4] = torch.stack([mab, b, mbc], 1)
    f[2::4] = torch.stack([mca, mbc, c], 1)
    f[3::4] = torch.stack([mab, mbc, mca], 1)
    return new_xyz, f


def _tangent_basis(n):
    """Orthonormal tangent vectors (e1, e2) at unit normals n (rows, torch)."""
    import torch
    ref = torch.zeros_like(n)
    ref[:, 2] = 1.0
    near_pole = n[:, 2].abs() > 0.9
    ref[near_pole] = torch.tensor([1.0, 0.0, 0.0], dtype=n.dtype, device=n.device)
    e1 = torch.linalg.cross(ref, n)
    e1 = e1 / torch.linalg.norm(e1, dim=1, keepdim=True)
    e2 = torch.linalg.cross(n, e1)
    return e1, e2


def icosphere(level, radius=6371.0, jitter=0.2, seed=11):
    """Icosahedral subdivision of the sphere: 10*4^level + 2 vertices,
    20*4^level triangles.  Each vertex is displaced tangentially, uniformly in
    a disc of radius `jitter` times the mean length of its edges, then put back
    on the sphere (seeded)."""
    import torch
    dev = _device(10 * 4 ** level + 2)
    xyz = torch.tensor(_ICO_V / np.linalg.norm(_ICO_V, axis=1, keepdims=True), device=dev)
    faces = torch.tensor(_ICO_F, device=dev)
    for _ in range(level):
        xyz, faces = _subdivide(xyz, faces)
    if jitter > 0:
        nv = xyz.shape[0]
        e = torch.cat([faces[:, [0, 1]], faces[:, [1, 2]], faces[:, [2, 0]]], 0)
        ln = torch.linalg.norm(xyz[e[:, 0]] - xyz[e[:, 1]], dim=1)
        acc = torch.zeros(nv, dtype=xyz.dtype, device=dev)
        cnt = torch.zeros(nv, dtype=xyz.dtype, device=dev)
        acc.index_add_(0, e[:, 0], ln)
        acc.index_add_(0, e[:, 1], ln)
        one = torch.ones_like(ln)
        cnt.index_add_(0, e[:, 0], one)
        cnt.index_add_(0, e[:, 1], one)
        hloc = acc / cnt
        rng = np.random.default_rng(seed)
        u1 = torch.tensor(rng.random(nv), device=dev)
        u2 = torch.tensor(rng.random(nv), device=dev)
        rad = jitter * hloc * torch.sqrt(u1)
        ang = 2.0 * np.pi * u2
        e1, e2 = _tangent_basis(xyz)
        xyz = xyz + (rad * torch.cos(ang))[:, None] * e1 + (rad * torch.sin(ang))[:, None] * e2
        xyz = xyz / torch.linalg.norm(xyz, dim=1, keepdim=True)
    coords = (xyz * radius).cpu().numpy().astype(np.float64)
    return dict(coords=coords, tri=faces.cpu().numpy().astype(np.int32),
                geom="sphere", period_x=0.0, period_y=0.0, radius=float(radius))


def land_mask(coords, frac_land=0.3, n_blobs=64, seed=12, polar_cap_deg=0.0):
    """Ocean mask (uint8, 1 = ocean) from a seeded sum of smooth Gaussian caps on
    the unit sphere, thresholded so that a fraction `frac_land` of the points is
    land.  With polar_cap_deg > 0 every point within that many degrees of a
    geographic pole is also land."""
    import torch
    dev = _device(coords.shape[0])
    x = torch.tensor(coords, device=dev)
    x = x / torch.linalg.norm(x, dim=1, keepdim=True)
    rng = np.random.default_rng(seed)
    c = rng.normal(size=(n_blobs, 3))
    c /= np.linalg.norm(c, axis=1, keepdims=True)
    sig = rng.uniform(0.15, 0.5, size=n_blobs)
    w = rng.uniform(0.5, 1.5, size=n_blobs)
    s = torch.zeros(x.shape[0], dtype=x.dtype, device=dev)
    ct = torch.tensor(c, device=dev)
    for b in range(n_blobs):
        d2 = 2.0 * (1.0 - x @ ct[b])
        s += w[b] * torch.exp(-d2 / (2.0 * sig[b] ** 2))
    s = s.cpu().numpy()
    thr = np.quantile(s, 1.0 - frac_land)
    land = s >= thr
    if polar_cap_deg > 0:
        z = x[:, 2].clamp(-1, 1).cpu().numpy()
        lat = np.degrees(np.arcsin(z))
        land |= np.abs(lat) >= 90.0 - polar_cap_deg
    return (~land).astype(np.uint8)


def triangle_centroids(mesh):
    """Centroids of the triangles (for fields that live on cells).  On the
    sphere the centroid is projected radially onto the sphere."""
    x = mesh["coords"]
    t = mesh["tri"]
    if mesh["geom"] == "sphere":
        c = (x[t[:, 0]] + x[t[:, 1]] + x[t[:, 2]]) / 3.0
        return c / np.linalg.norm(c, axis=1, keepdims=True) * mesh["radius"]
    # planar periodic: average with minimum-image offsets relative to vertex 0
    px, py = mesh["period_x"], mesh["period_y"]
    p0 = x[t[:, 0]]
    acc = p0.copy()
    for k in (1, 2):
        d = x[t[:, k]] - p0
        d[:, 0] -= px * np.round(d[:, 0] / px)
        d[:, 1] -= py * np.round(d[:, 1] / py)
        acc += p0 + d
    c = acc / 3.0
    c[:, 0] %= px
    c[:, 1] %= py
    return c
