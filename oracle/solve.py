"""Oracle: the filter equations and their conjugate-gradient solution.  Test infrastructure only.

For a wavenumber k (l = 1/k, Sect. 2.1) and order n the system matrix is
    S = M + (1/2) l^(2n) K (M^-1 K)^(n-1)
with M = diag(A) the lumped mass and K the l-free operator of the placement
(Sect. 2.1.1: n = 1 and n = 2 written out, "can be generalized").  Right-hand
sides and initial guesses per placement:
  vertex_scalar : b = M phi,           x0 = phi            (Sect. 2.1.1)
  vertex_vector : b = R u_c (2 comps), x0 = M^-1 b, unknowns (u block, v block)
                  coupled by T                              (Sect. 2.1.2)
  cell          : b = A_c u_c,         x0 = u_c, each component on its own (Eq. 6)
The solve follows Sect. 2.2.2: S x0 is subtracted first (residual form), then
conjugate gradients run on the remainder.  The result is the unique solution
of the SPD system; CG is only the means, so the oracle drives the true
residual as low as FP64 allows, and `filter_dense` re-solves tiny systems with
a dense LU as a second opinion.

Entries that are not unknowns (land) pass through unchanged for the vertex
scalar and cell placements; the vertex-vector output is zero there.

`residual_certificate` bounds the error of any candidate solution without
solving: S >= M (K is symmetric positive semidefinite for n = 1, and
K M^-1 K is for n = 2), hence ||x - x*||_M <= ||b - S x||_{M^-1}.
Parity: pinned (Fourier closed forms on periodic grids, dense solves, tests).
"""

from dataclasses import dataclass, field as dc_field

import numpy as np
import scipy.sparse as sp

from .operators import (scalar_vertex_operators, vector_vertex_operators, cell_operators,
                        voronoi_vertex_operators, circumcenter_cell_operators)


@dataclass
class Problem:
    placement: str
    K: sp.csr_matrix           # l-free operator of the unknowns, symmetric
    A: np.ndarray              # lumped mass of the unknowns
    n_in: int                  # entries per input component
    n_out: int                 # entries per output component
    n_comp: int
    out_ids: np.ndarray        # output index of each output unknown
    parts: dict = dc_field(default_factory=dict)

    def apply_S(self, x, ell, order):
        """S x = M x + (1/2) l^(2n) K (M^-1 K)^(n-1) x."""
        y = self.K @ x
        for _ in range(order - 1):
            y = self.K @ (y / self.A)
        return self.A * x + 0.5 * ell ** (2 * order) * y

    def systems(self, fld):
        """[(b, x0)] of the independent systems of one field [n_comp][n_in]."""
        if self.placement in ("vertex_scalar", "vertex_voronoi"):
            phi = fld[0][self.parts["vert_ids"]]
            return [(self.A * phi, phi.copy())]
        if self.placement == "vertex_vector":
            kc = self.parts["kept_tri"]
            R = self.parts["R"]
            b = np.concatenate([R @ fld[0][kc], R @ fld[1][kc]])
            return [(b, b / self.A)]
        if self.placement in ("cell", "cell_circumcenter"):
            ids = self.parts["cell_ids"]
            return [(self.A * fld[c][ids], fld[c][ids].copy()) for c in range(self.n_comp)]
        raise ValueError(self.placement)

    def output(self, fld, sols):
        """Assemble [n_comp][n_out] from the system solutions."""
        if self.placement in ("vertex_scalar", "vertex_voronoi"):
            out = np.array(fld, dtype=np.float64, copy=True)
            out[0][self.out_ids] = sols[0]
            return out
        if self.placement == "vertex_vector":
            n = self.out_ids.size
            out = np.zeros((2, self.n_out))
            out[0][self.out_ids] = sols[0][:n]
            out[1][self.out_ids] = sols[0][n:]
            return out
        out = np.array(fld, dtype=np.float64, copy=True)
        for c in range(self.n_comp):
            out[c][self.out_ids] = sols[c]
        return out

    def weights(self):
        """Area of each output unknown (A_v or A_c)."""
        if self.placement == "vertex_vector":
            return self.A[: self.out_ids.size]
        return self.A


def build_problem(mesh, placement, cell_A=None):
    V = mesh["coords"].shape[0]
    T = np.asarray(mesh["tri"]).shape[0]
    if placement == "vertex_scalar":
        o = scalar_vertex_operators(mesh)
        return Problem(placement, o["K"], o["A"], V, V, 1, o["vert_ids"], parts=o)
    if placement == "vertex_vector":
        o = vector_vertex_operators(mesh)
        K2 = sp.bmat([[o["Kt"], o["Tm"]], [-o["Tm"], o["Kt"]]]).tocsr()
        A2 = np.concatenate([o["A"], o["A"]])
        return Problem(placement, K2, A2, T, V, 2, o["vert_ids"], parts=o)
    if placement == "cell":
        o = cell_operators(mesh, cell_A)
        return Problem(placement, o["K"], o["A"], T, T, 2, o["cell_ids"], parts=o)
    if placement == "vertex_voronoi":
        o = voronoi_vertex_operators(mesh)
        return Problem(placement, o["K"], o["A"], V, V, 1, o["vert_ids"], parts=o)
    if placement == "cell_circumcenter":
        o = circumcenter_cell_operators(mesh)
        return Problem(placement, o["K"], o["A"], T, T, 1, o["cell_ids"], parts=o)
    raise ValueError(placement)


def cg(apply_A, b, x0, rtol, max_iter=200000, max_restarts=8):
    """Conjugate gradients (Hestenes-Stiefel) from x0 for SPD A.

    Stops when the TRUE residual ||b - A x|| <= rtol * ||b - A x0||; the
    recursive residual is trusted only until it reaches the target, then CG
    restarts from the current iterate (at most max_restarts times, and only
    while the true residual keeps falling).
    Returns (x, iterations, achieved true relative residual)."""
    x = np.array(x0, dtype=np.float64, copy=True)
    r = b - apply_A(x)
    r0 = np.linalg.norm(r)
    if r0 == 0.0:
        return x, 0, 0.0
    target = rtol * r0
    its = 0
    best = r0
    for _ in range(max_restarts + 1):
        p = r.copy()
        rr = r @ r
        while np.sqrt(rr) > target and its < max_iter:
            q = apply_A(p)
            alpha = rr / (p @ q)
            x += alpha * p
            r -= alpha * q
            rr_new = r @ r
            p = r + (rr_new / rr) * p
            rr = rr_new
            its += 1
        r = b - apply_A(x)
        true = np.linalg.norm(r)
        if true <= target or its >= max_iter or true >= 0.5 * best:
            best = min(best, true)
            break
        best = true
    return x, its, best / r0


def filter_field(problem, fld, ks, order, rtol=1e-14, max_iter=200000):
    """Filtered fields [K][n_comp][n_out] and per-(k, system) stats."""
    out = []
    stats = []
    for k in ks:
        ell = 1.0 / k
        sols = []
        for b, x0 in problem.systems(fld):
            x, its, rel = cg(lambda v: problem.apply_S(v, ell, order), b, x0, rtol, max_iter)
            sols.append(x)
            stats.append((k, its, rel))
        out.append(problem.output(fld, sols))
    return np.stack(out), stats


def dense_S(problem, ell, order):
    K = problem.K.toarray()
    G = K.copy()
    for _ in range(order - 1):
        G = K @ (G / problem.A[:, None])
    return np.diag(problem.A) + 0.5 * ell ** (2 * order) * G


def filter_dense(problem, fld, ks, order):
    """Same result as filter_field by a dense LU solve of S (small meshes only)."""
    out = []
    for k in ks:
        S = dense_S(problem, 1.0 / k, order)
        sols = [np.linalg.solve(S, b) for b, _ in problem.systems(fld)]
        out.append(problem.output(fld, sols))
    return np.stack(out)


def shifted_factors(order):
    """Partial fractions of the filter's response (Eq. 1 with gamma = 1/2):
    with x standing for l^2 times the discrete -Laplacian's eigenvalue,
        1 / (1 + x^n / 2) = sum_j (1/n) / (1 - x / r_j),   r_j^n = -2,
    r_j = 2^(1/n) exp(i pi (2j + 1) / n), j = 0 .. n-1 (the residue of the
    simple pole r_j is -r_j / n).  Each term is one solve with M + sigma_j K,
    sigma_j = -l^2 / r_j, on the pattern of K alone.  Returns the list of
    (sigma_j / l^2, 1/n) pairs."""
    n = int(order)
    out = []
    for j in range(n):
        r = 2.0 ** (1.0 / n) * np.exp(1j * np.pi * (2 * j + 1) / n)
        out.append((-1.0 / r, 1.0 / n))
    return out


def filter_shifted(problem, fld, ks, order):
    """The filtered fields as the sum over the partial fractions of
    `shifted_factors`: phi_l = sum_j (1/n) (M + sigma_j K)^-1 b, one sparse
    complex LU per term (small meshes; a second route to `filter_dense`)."""
    import scipy.sparse.linalg as spla
    K = problem.K.tocsc().astype(np.complex128)
    M = sp.diags(problem.A.astype(np.complex128)).tocsc()
    out = []
    for k in ks:
        ell2 = 1.0 / (k * k)
        sols = []
        for b, _ in problem.systems(fld):
            acc = np.zeros(b.shape, dtype=np.complex128)
            for sig, w in shifted_factors(order):
                acc += w * spla.spsolve((M + (sig * ell2) * K).tocsc(), b.astype(np.complex128))
            sols.append(acc.real.copy())
        out.append(problem.output(fld, sols))
    return np.stack(out)


def _candidates(problem, fld, filtered_k):
    """The unknowns of each system read back from an output block [n_comp][n_out]."""
    ids = problem.out_ids
    if problem.placement == "vertex_vector":
        return [np.concatenate([filtered_k[0][ids], filtered_k[1][ids]])]
    return [filtered_k[c][ids] for c in range(len(problem.systems(fld)))]


def relative_residual(problem, fld, filtered_k, k, order):
    """Per system, ||b - S x|| / ||b - S x0|| (2-norms) for the candidate x read
    from `filtered_k`: the quantity the paper's solver drives below its tolerance
    (Sect. 2.2.2, residual form with x0 as in `systems`)."""
    ell = 1.0 / k
    out = []
    for (b, x0), x in zip(problem.systems(fld), _candidates(problem, fld, filtered_k)):
        r0 = np.linalg.norm(b - problem.apply_S(x0, ell, order))
        r = np.linalg.norm(b - problem.apply_S(x, ell, order))
        out.append(r / r0 if r0 > 0 else r)
    return out


def refined_certificate(problem, fld, filtered_k, k, order, iters=50, stop=0.0):
    """As `residual_certificate`, sharpened by a correction the oracle computes
    itself.  For a candidate x with residual r = b - S x, let e~ be the result of
    `iters` conjugate-gradient steps on S e = r from e = 0.  Since
    x* - x = S^-1 r = e~ + S^-1 (r - S e~) and S >= M,
        ||x - x*||_M <= ||e~||_M + ||r - S e~||_{M^-1}.
    The first term is about the true error; the second is the part of the
    residual the steps did not resolve.  Where S is far above M (the short
    scales of a large-l system) the plain bound ||r||_{M^-1} overstates the
    error by up to the ratio of the two, and a few steps remove that part of r.
    iters = 0 gives the plain bound.  With stop > 0 the steps end early, once
    the recurrence's residual r - S e~ is at most stop ||x||_M in the M^-1 norm
    (the bound itself is always formed from r - S e~ recomputed).  Returns per
    system (bound, ||x||_M)."""
    ell = 1.0 / k
    apply = lambda v: problem.apply_S(v, ell, order)
    res = []
    syst = problem.systems(fld)
    for (b, _), x in zip(syst, _candidates(problem, fld, filtered_k)):
        r = b - apply(x)
        xn = np.sqrt(np.sum(problem.A * x * x))
        e = np.zeros_like(r)
        rr = r.copy()
        p = rr.copy()
        rho = rr @ rr
        for _ in range(iters):
            if rho == 0.0 or np.sqrt(np.sum(rr * rr / problem.A)) <= stop * xn:
                break
            q = apply(p)
            alpha = rho / (p @ q)
            e += alpha * p
            rr -= alpha * q
            rho_new = rr @ rr
            p = rr + (rho_new / rho) * p
            rho = rho_new
        left = r - apply(e)  # the unresolved residual, recomputed
        bound = np.sqrt(np.sum(problem.A * e * e)) + np.sqrt(np.sum(left * left / problem.A))
        res.append((bound, xn))
    return res


def lambda_max_minv_k(problem, iters=60, seed=0):
    """Power iteration for the largest eigenvalue of M^-1 K (the l-free
    operator's spectrum in the M inner product).  Power iteration approaches it
    from below, so the result never overstates it.  The condition number of S
    in the M-norm is then kappa(l) = 1 + 1/2 (l^2 lambda)^n for K symmetric
    positive semidefinite."""
    rng = np.random.default_rng(seed)
    x = rng.normal(size=problem.A.size)
    lam = 0.0
    for _ in range(iters):
        y = (problem.K @ x) / problem.A
        nrm = np.sqrt(np.sum(problem.A * y * y))
        if nrm == 0.0:
            return 0.0
        lam = np.sum(problem.A * x * y) / np.sum(problem.A * x * x)  # Rayleigh quotient in the M inner product
        x = y / nrm
    return float(lam)


def residual_certificate(problem, fld, filtered_k, k, order):
    """For one wavenumber: per system (||b - S x||_{M^-1}, ||x||_M) where x is the
    candidate solution read back from `filtered_k` [n_comp][n_out].  The first
    number bounds ||x - x*||_M."""
    ell = 1.0 / k
    res = []
    syst = problem.systems(fld)
    ids = problem.out_ids
    if problem.placement == "vertex_vector":
        xs = [np.concatenate([filtered_k[0][ids], filtered_k[1][ids]])]
    else:
        xs = [filtered_k[c][ids] for c in range(len(syst))]
    for (b, _), x in zip(syst, xs):
        r = b - problem.apply_S(x, ell, order)
        res.append((np.sqrt(np.sum(r * r / problem.A)), np.sqrt(np.sum(problem.A * x * x))))
    return res
