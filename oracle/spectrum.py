"""Oracle: coarse-grained energy spectra from filtered fields.  Test infrastructure only.

The paper computes spectra from fields filtered at a sequence of scales
(Sect. 1, 4 and 5, following the coarse-graining approach it cites) but prints
no formula.  Reading used here:
  E(k)      = sum_i w_i * 1/2 * sum_comp phi_k(i)^2 / sum_i w_i
              over the unknowns i (w = A_v at vertices, A_c on cells);
  spec_j    = (E(k_{j+1}) - E(k_j)) / (k_{j+1} - k_j) at k_mid = sqrt(k_j k_{j+1}),
              k ascending.
E(k) grows with k (a larger k removes less), so spec_j >= 0.
Parity: pinned (Parseval on a periodic grid, tests).
"""

import numpy as np


def filtered_energy(filtered, out_ids, weights):
    """filtered [K][n_comp][n_out] -> E [K]."""
    f = np.asarray(filtered)[:, :, out_ids]
    e = 0.5 * np.sum(f * f, axis=1)          # [K][n]
    return (e @ weights) / np.sum(weights)


def spectrum(ks, E):
    ks = np.asarray(ks, dtype=np.float64)
    E = np.asarray(E, dtype=np.float64)
    o = np.argsort(ks, kind="stable")
    k = ks[o]
    e = E[..., o]
    kmid = np.sqrt(k[1:] * k[:-1])
    spec = (e[..., 1:] - e[..., :-1]) / (k[1:] - k[:-1])
    return kmid, spec
