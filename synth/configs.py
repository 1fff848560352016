"""Named synthetic workloads (meshes, masks, fields and wavenumbers).

Each recipe is seeded, so every caller that asks for the same workload gets the
same arrays.  `level` overrides the icosahedral subdivision level so that tests
can run the same recipe at a size the oracle finishes in seconds.

Workloads
---------
periodic32        : doubly periodic 32x32 split-square grid, unit spacing, scalar at
                    vertices, n = 1, one wavenumber k = 2*pi/8, k^-3 random field.
sphere            : icosahedral level 8 (655,362 vertices), 20 % jitter, 30 % land,
                    scalar at vertices, n = 2, 40 wavenumbers log-spaced between
                    2*pi/4000 km and 2*pi/10 km on a 6371 km sphere.
uv_batch          : icosahedral level 10 (10,485,762 vertices), 20 % jitter, 30 % land plus
                    polar caps, velocity components (u, v) on triangles, n = 2,
                    40 wavenumbers x 2 components; filtered with the vertex-vector
                    and the cell placements.
precision         : icosahedral level 9 (2,621,442 vertices), scalar at vertices, n = 2,
                    40 wavenumbers.
serving           : resident icosahedral meshes at levels 6, 8, 9, 10.
"""

import numpy as np

from .meshes import periodic_split_square, icosphere, land_mask, triangle_centroids
from .fields import grf_periodic, grf_sphere, log_wavenumbers

EARTH_RADIUS_KM = 6371.0

_SPHERE_SEEDS = {
    "sphere": dict(level=8, jitter=11, land=12, field=(13,)),
    "uv_batch": dict(level=10, jitter=21, land=22, field=(23, 24)),
    "precision": dict(level=9, jitter=31, land=32, field=(33,)),
}


def sphere_mesh(level, jitter_seed, land_seed, polar_cap_deg=0.0):
    m = icosphere(level, radius=EARTH_RADIUS_KM, jitter=0.2, seed=jitter_seed)
    m["ocean"] = land_mask(m["coords"], frac_land=0.3, n_blobs=64, seed=land_seed,
                           polar_cap_deg=polar_cap_deg)
    return m


def workload(name, level=None, n_k=None, n_fields=1):
    """Return a dict with keys mesh, fields, k, order, placements, on.

    fields : float64 [F][n_comp][P] with P = vertices ("on" == "vertex") or
             triangles ("on" == "cell").
    """
    if name == "periodic32":
        n = 32 if level is None else level
        m = periodic_split_square(n, n, 1.0)
        m["ocean"] = None
        f = np.stack([grf_periodic(n, n, 1.0, seed=1 + s) for s in range(n_fields)])[:, None, :]
        return dict(mesh=m, fields=f, k=np.array([2 * np.pi / 8.0]), order=1,
                    placements=("vertex_scalar",), on="vertex")
    if name not in _SPHERE_SEEDS:
        raise KeyError(name)
    s = _SPHERE_SEEDS[name]
    lev = s["level"] if level is None else level
    polar = 5.0 if name == "uv_batch" else 0.0
    m = sphere_mesh(lev, s["jitter"], s["land"], polar_cap_deg=polar)
    nk = 40 if n_k is None else n_k
    k = log_wavenumbers(4000.0, 10.0, nk)
    h = 7.5 * 2.0 ** (10 - lev)  # nominal edge length (km)
    kmax = 2 * np.pi / (2.0 * h)
    kmin = 2 * np.pi / 20000.0
    if name == "uv_batch":
        c = triangle_centroids(m)
        comps = [grf_sphere(c, seed=sd, k_min=kmin, k_max=kmax, n_features=256) for sd in s["field"]]
        f = np.stack(comps)[None, :, :]
        return dict(mesh=m, fields=f, k=k, order=2,
                    placements=("vertex_vector", "cell"), on="cell")
    fs = [grf_sphere(m["coords"], seed=s["field"][0] + 1000 * i, k_min=kmin, k_max=kmax,
                     n_features=512 if lev <= 8 else 256) for i in range(n_fields)]
    f = np.stack(fs)[:, None, :]
    return dict(mesh=m, fields=f, k=k, order=2, placements=("vertex_scalar",), on="vertex")
