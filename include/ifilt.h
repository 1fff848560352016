/*
 * ifilt.h -- C ABI of the GB300 implicit-filter library (libifilt.so).
 *
 * The implicit filter of Nowak, Danilov, Mueller and Liu ("Implementation of
 * implicit filter for spatial spectra extraction") coarse-grains a field phi
 * on an unstructured triangular mesh by solving
 *
 *     (1 + 1/2 (-l^2 Lap)^n) phi_l = phi,      k = 1/l        (Eq. 1 and 2)
 *
 * with a discrete Laplacian built for the data placement (Sect. 2.1).  The
 * work is split in two phases (Sect. 2.2): a mesh-only preparation whose
 * arrays are reused for every scale, and a solving phase of sparse matrix
 * products inside a conjugate-gradient iteration (Sect. 2.2.2).  Spectra are
 * differences of filtered energies over k (Sect. 1, 4, 5).
 *
 * Conventions for every entry point:
 *   - Pointers documented "host" are CPU memory; "device" are CUDA device
 *     memory of the current device (e.g. torch tensors' data_ptr()).
 *   - The caller owns every buffer it passes; the library never frees them
 *     and keeps no reference to them after the call returns.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is
 *     enqueued on it; calls that return host results synchronise it.
 *   - A negative ifilt_status is an error: outputs are left untouched and
 *     ifilt_last_error() returns a message (thread-local).  IFILT_NOT_CONVERGED
 *     is a warning: outputs are written, per-column stats say which columns
 *     missed the tolerance.  No call aborts the process or waits without bound.
 *
 * Environment variables (read at each call that uses them):
 *   IFILT_HOST_THREADS  host worker threads for preparation and the multigrid
 *                       setup (default: hardware threads, at most 64); results
 *                       are the same bytes for any value
 *   IFILT_AUTOTUNE=0    keep the default launch shapes of the batched solver
 *                       instead of timing candidates on the first solve of a
 *                       mesh (results then depend on nothing but the inputs)
 *   IFILT_NO_GRAPH=1    launch every kernel directly instead of through CUDA graphs
 *   IFILT_TRACE=1       print each batched-solver launch to stderr (read once)
 *   IFILT_MG_COARSE_SWEEPS=k  damped-Jacobi sweeps before and after the coarse
 *                       correction on multigrid levels >= 1 (1..6; default 2)
 *   IFILT_MG_FINE_SWEEPS=k    the same on the finest level (1..6; default 1)
 */
#ifndef IFILT_H
#define IFILT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ifilt_mesh_s* ifilt_mesh;

typedef enum {
  IFILT_OK = 0,
  IFILT_NOT_CONVERGED = 1,   /* warning: some column stopped at max_iter or broke down */
  IFILT_EINVAL = -1,         /* bad argument */
  IFILT_ENOMEM = -2,         /* device or host allocation failed */
  IFILT_ECUDA = -3,          /* a CUDA call failed */
  IFILT_EMESH = -4,          /* malformed mesh (index out of range, degenerate triangle, ...) */
  IFILT_DEVICE_TIMEOUT = -5, /* a bounded device-side wait expired */
  IFILT_ECACHE = -6          /* mesh cache file missing, unreadable, corrupt, of another format or
                                preparation revision, or written for another mesh */
} ifilt_status;

/* Data placements (Sect. 2.1, Fig. 1). */
enum {
  IFILT_VERTEX_SCALAR = 0,   /* scalar at vertices, median-dual volumes, P1 FE (Sect. 2.1.1)     */
  IFILT_VERTEX_VECTOR = 1,   /* (u, v) from cells filtered at vertices with metric terms (Sect. 2.1.2) */
  IFILT_CELL = 2,            /* (u, v) at triangles, simplified Laplacian of Eq. 6, per component */
  IFILT_VERTEX_VORONOI = 3,  /* scalar at vertices, quasi-hexagonal control volumes, finite volumes
                                (Eq. 3-5): A_v (D phi)_v = l^2 sum (phi_v - phi_v') l_vv' / d_vv',
                                d the edge length, l the distance between the circumcentres on its
                                two sides (signed; the edge midpoint on a coast), A_v the area of the
                                circumcentric (Voronoi) dual cell */
  IFILT_CELL_CIRCUMCENTER = 4 /* scalar at triangle circumcentres, finite volumes: A_c (D phi)_c =
                                l^2 sum (phi_c - phi_c') l_e / d_cc', l_e the shared edge's length,
                                d_cc' the distance between the two circumcentres; EMESH where they
                                coincide */
};

/* Mesh geometry. */
enum {
  IFILT_GEOM_PLANAR_PERIODIC = 0,  /* coords [V][2]; edge vectors taken as minimum images */
  IFILT_GEOM_PLANAR = 1,           /* coords [V][2] */
  IFILT_GEOM_SPHERE = 2            /* coords [V][3] on a sphere of `radius`; flat chordal triangles */
};

/* Device row order.  RCM: reverse Cuthill-McKee on the graph of K (component
 * start = least (degree, id), neighbours by (degree, id), reversed).  HILBERT:
 * by a space-filling-curve key of each unknown's position (the vertex, or the
 * triangle's corner average ((a + b) + c) / 3 in FP64), ties by id -- sphere:
 * cube face of the direction (largest |component|, ties to x then y, +axis
 * before -axis) then the Hilbert index of the two other components divided by
 * the largest, each mapped to [0, 1] and quantised to 16 bits as
 * floor(t * 2^16) clamped; plane: the coordinates scaled to the mesh's bounding
 * box.  The curve starts at (0, 0) and ends at (2^16 - 1, 0). */
enum { IFILT_REORDER_NONE = 0, IFILT_REORDER_RCM = 1, IFILT_REORDER_HILBERT = 2 };

/* Arithmetic of the solve. */
enum {
  IFILT_PREC_FP64 = 0,       /* FP64 matrix, vectors and dots */
  IFILT_PREC_FP32_IR = 1,    /* FP32 matrix and Krylov vectors, FP64-accurate dots, true residual
                                and iterative-refinement correction in double-float (hi + lo FP32
                                pairs) when tol >= 1e-10 and err_tol is 0 or >= 1e-8, else FP64 */
  IFILT_PREC_BF16_IR = 2     /* as FP32_IR with BF16-stored matrix values */
};

enum {
  IFILT_METHOD_PLAIN = 0,    /* one right-hand side at a time: S assembled per scale in FP64 CSR,
                                separate SpMV / dot / axpy kernels, host convergence test every
                                iteration (the paper's CG, Sect. 2.2.2) */
  IFILT_METHOD_BATCHED = 1   /* every (field, component, scale) column of the call solved together:
                                one shared operator, per-column shift, fused kernels, CUDA graphs */
};

/* How order n = 2 is solved by the batched method (ignored for n = 1). */
enum {
  IFILT_N2_AUTO = 0,         /* complex factorisation */
  IFILT_N2_REAL = 1,         /* CG on S = M + 1/2 l^4 K M^-1 K with the product assembled */
  IFILT_N2_COMPLEX = 2       /* S = M (1 + i a)(1 - i a), a = l^2 M^-1 K / sqrt(2):
                                phi_l = Re[(M + i l^2/sqrt(2) K)^-1 M phi], solved by
                                conjugate orthogonal CG (a CG-type method for complex
                                symmetric systems).  Same solution, condition ~ l^2 instead of l^4. */
};

/* Preconditioning of the batched Krylov solve (the plain method takes none). */
enum {
  IFILT_PRECOND_NONE = 0,
  IFILT_PRECOND_JACOBI = 1,  /* z = D^-1 r, D the diagonal of the shifted operator of each column
                                (m_i + s g_ii, or m_i + i s g_ii for the complex form); the
                                preconditioned CG / COCG keeps the same solution and stopping test
                                on the unpreconditioned residual */
  IFILT_PRECOND_MG = 2       /* z = one V-cycle of smoothed-aggregation multigrid on each column's
                                S = M + s K (or M + i s K): two damped-Jacobi sweeps before and
                                after each coarse correction, Jacobi sweeps on the coarsest level;
                                a symmetric preconditioner, so CG / COCG apply.  Needs S built on
                                K (order 1, or order 2 in the complex form) and the FP32 or BF16
                                precision; EINVAL otherwise */
};

typedef struct {
  int32_t n_vert;            /* V > 0 */
  int32_t n_tri;             /* T > 0 */
  const double* coords;      /* host [V][2] or [V][3] (geometry), any length unit */
  const int32_t* tri;        /* host [T][3] vertex ids, counter-clockwise seen from outside */
  const uint8_t* ocean;      /* host [V], nonzero = ocean; NULL = everything is ocean.
                                A triangle is in the domain iff its 3 vertices are ocean;
                                coast edges get the no-flux condition of Sect. 2.1 */
  int32_t geometry;          /* IFILT_GEOM_* */
  double period_x, period_y; /* periodic plane only */
  double radius;             /* sphere only (metric factor m = tan(lat)/radius, Sect. 2.1.2) */
  int32_t placement;         /* IFILT_VERTEX_SCALAR ... IFILT_CELL_CIRCUMCENTER */
  int32_t max_order;         /* highest filter order n the mesh must serve, 1 .. IFILT_MAX_ORDER;
                                orders >= 3 store G_n = K (M^-1 K)^(n-1) for n = 3 .. max_order */
  int32_t reorder;           /* IFILT_REORDER_* : device row order */
  double cell_A;             /* constant A of Eq. 6 (cell placement); 0 selects sqrt(3) */
  int32_t ell_slice;         /* rows per sliced-ELL slice, 4..1024; 0 = library default (64) */
  double mg_strength;        /* multigrid aggregation threshold theta in [0, 1): aggregates follow
                                only connections |k_ij| >= theta sqrt(|k_ii k_jj|), and coarse levels
                                get smoother weights scaled to their operators; 0 = every neighbour
                                and weight 2/3 on all levels (the default hierarchy) */
} ifilt_mesh_desc;

#define IFILT_MAX_ORDER 4

typedef struct {
  int32_t order;             /* filter order n, 1 <= n <= mesh max_order.  n >= 3 (the paper's
                                generalisation of Sect. 2.1.1) is solved on the explicit operator
                                S = M + 1/2 l^(2n) G_n by CG in real arithmetic: the plain method,
                                or the batched method without multigrid (the condition number
                                grows like l^(2n), so FP32 inner solves suit small scales only) */
  double tol;                /* stop when ||r|| <= tol * ||r0|| (r0 = b - S phi, Sect. 2.2.2); the paper uses 1e-9 */
  int32_t max_iter;          /* cap on Krylov iterations per column (all refinement rounds); 0 = 100000 */
  int32_t precision;         /* IFILT_PREC_* */
  int32_t method;            /* IFILT_METHOD_* */
  int32_t n2_solver;         /* IFILT_N2_* (order 2 only; orders >= 3 take AUTO or REAL) */
  int32_t precond;           /* IFILT_PRECOND_*; batched method only */
  int32_t check_every;       /* batched: iterations per CUDA graph between host checks; 0 = 32
                                (8 with IFILT_PRECOND_MG) */
  double inner_tol;          /* FP32 inner solves: relative reduction per refinement round; 0 = 1e-4 */
  int32_t max_lanes;         /* batched: widest column tile in 32-bit lanes; 0 = library default */
  double err_tol;            /* batched: if > 0, a column also needs ||b - S x||_{M^-1} <= err_tol ||x||_M
                                (x the filtered part: the real part in the complex n = 2 form), a
                                bound on its relative error in the M-norm, because S >= M (and
                                |e^H A e| >= e^H M e for A = M + i s K); 0 = the residual test only */
  int32_t mg_cycle;          /* multigrid cycle: IFILT_MG_V (0) or IFILT_MG_W12 (1), which applies the
                                coarse correction of levels 1 and 2 twice (more coarse work, fewer
                                Krylov iterations on large meshes) */
} ifilt_solve_opts;

enum { IFILT_MG_V = 0, IFILT_MG_W12 = 1 };

typedef struct {
  int32_t iters;             /* Krylov iterations (all rounds) */
  int32_t refinements;       /* FP64 true-residual rounds */
  int32_t status;            /* IFILT_OK or IFILT_NOT_CONVERGED */
  int32_t pad;
  double rel_residual;       /* final true ||b - S x|| / ||b - S x0|| in FP64 (of the system solved) */
  double err_bound;          /* batched: final ||b - S x||_{M^-1} / ||x||_M (see err_tol); plain: 0 */
} ifilt_col_stats;

typedef struct {
  int32_t placement, geometry, max_order, reorder;
  int32_t n_rows;            /* unknown rows on the device (vertices or cells of the ocean domain) */
  int32_t n_in;              /* entries per input component (V, or T for vector/cell) */
  int32_t n_out;             /* entries per output component (V, or T for cell) */
  int32_t n_comp;            /* components per field: 1 scalar, 2 vector or cell */
  int64_t nnz_k;             /* stored entries of the n = 1 operator (blocks for the vector placement) */
  int64_t nnz_g2;            /* stored entries of K M^-1 K (0 if max_order < 2) */
  int32_t ell_slice, ell_width_k, ell_width_g2, pad;
  int64_t device_bytes;      /* device memory held by the handle */
} ifilt_mesh_info_t;

/* Export selectors for ifilt_mesh_export (host copies of the prepared arrays). */
enum {
  IFILT_EXPORT_PERM = 0,       /* int32 [n_rows]: original input index of each device row */
  IFILT_EXPORT_K_ROWPTR = 1,   /* int64 [n_rows+1]: CSR of the n = 1 operator in device order */
  IFILT_EXPORT_K_COL = 2,      /* int32 [nnz_k] */
  IFILT_EXPORT_K_VAL = 3,      /* double [nnz_k] (vector placement: [nnz_k][2] = (K~, Tm)) */
  IFILT_EXPORT_MASS = 4,       /* double [n_rows]: lumped mass A_v or A_c */
  IFILT_EXPORT_G2_ROWPTR = 5,  /* int64 [n_rows+1] */
  IFILT_EXPORT_G2_COL = 6,     /* int32 [nnz_g2] */
  IFILT_EXPORT_G2_VAL = 7      /* double [nnz_g2] (vector: [nnz_g2][2]) */
};

/* Higher-order operators G_n = K (M^-1 K)^(n-1), 2 <= n <= max_order, as host
 * copies: part 0 row pointers (int64 [n_rows+1]), 1 columns (int32 [nnz]),
 * 2 values (double [nnz], vector placement [nnz][2] for the 2x2 blocks).
 * dst = NULL with bytes = 0 only reports the size.  *written (if not NULL)
 * receives the byte count.  Errors: EINVAL (order outside 2..max_order,
 * unknown part, destination too small). */
ifilt_status ifilt_mesh_export_gn(ifilt_mesh mesh, int32_t order, int32_t part, void* dst, size_t bytes,
                                  size_t* written);

/* Build and cache the mesh-only arrays on the current device (Sect. 2.2.1):
 * ocean subset, device row order, the l-free operator K of the placement
 * (P1 stiffness for vertices, Sect. 2.1.1; stiffness plus metric terms and the
 * metric operator T for vectors, Sect. 2.1.2; A * graph Laplacian for cells,
 * Eq. 6), the lumped mass, K M^-1 K when max_order >= 2 (and G_n up to
 * max_order), FP64 CSR and
 * FP64/FP32/BF16 sliced-ELL copies.  Host inputs are read during the call only.
 * On success *out owns device memory until ifilt_release_mesh.  Errors:
 * EINVAL (null or inconsistent arguments), EMESH (index out of range, repeated
 * vertex in a triangle, zero-area triangle, an edge shared by more than two
 * ocean triangles, empty ocean), ENOMEM, ECUDA. */
ifilt_status ifilt_prepare_mesh(const ifilt_mesh_desc* desc, void* stream, ifilt_mesh* out);

/* The host half of ifilt_prepare_mesh: ocean subset, row order, operators
 * and packing on the CPU, no device memory touched (needs no GPU).  The
 * handle answers ifilt_mesh_info / ifilt_mesh_export; ifilt_mesh_upload makes
 * it usable by ifilt_solve.  Errors as ifilt_prepare_mesh. */
ifilt_status ifilt_prepare_mesh_host(const ifilt_mesh_desc* desc, ifilt_mesh* out);

/* Copy a host-prepared mesh to the current device (no-op if already there).
 * Errors: ENOMEM, ECUDA. */
ifilt_status ifilt_mesh_upload(ifilt_mesh mesh, void* stream);

/* Release a prepared mesh (NULL is ignored).  Waits for the device. */
void ifilt_release_mesh(ifilt_mesh mesh);

ifilt_status ifilt_mesh_info(ifilt_mesh mesh, ifilt_mesh_info_t* out);

/* Copy one prepared array to host memory `dst` of `bytes` bytes (EINVAL if
 * too small).  For tests of the integer layout against an independent
 * reference. */
ifilt_status ifilt_mesh_export(ifilt_mesh mesh, int32_t what, void* dst, size_t bytes);

/* Multigrid hierarchy of a mesh (IFILT_PRECOND_MG).  Built on the host from
 * the prepared n = 1 operator K and the lumped mass the first time it is
 * needed (this call or the first multigrid solve), then kept with the mesh;
 * it does not depend on l.  The paper has no counterpart: it reports that ILU
 * did not help (Sect. 2.2) and names better preconditioners as future work
 * (Sect. 6).  Smoothed aggregation: greedy
 * aggregates on the graph of K_l, prolongation P = (I - w D^-1 K_l) P_tent,
 * restriction R = P^T, coarse pair (K, M)_{l+1} = R (K, M)_l P.  Vertex-vector
 * meshes aggregate vertices and keep 2x2 blocks [[a, b], [-b, a]] on every level.
 * Works on host-only meshes (no GPU needed). */
#define IFILT_MG_MAX_LEVELS 16
typedef struct {
  int32_t n_levels;
  int32_t rows[IFILT_MG_MAX_LEVELS];    /* rows (vertices for the vector placement) per level */
  int64_t nnz_s[IFILT_MG_MAX_LEVELS];   /* stored entries of (K_l, M_l); level 0: of K */
  int64_t nnz_p[IFILT_MG_MAX_LEVELS];   /* entries of P_l (0 on the last level) */
} ifilt_multigrid_info;
ifilt_status ifilt_mesh_multigrid(ifilt_mesh mesh, ifilt_multigrid_info* info);

/* Export selectors for ifilt_mesh_multigrid_export (host copies, level >= 0).
 * Values per entry: (K_l, M_l) pairs hold (k, m) for scalar rows and
 * (k_a, k_b, m_a, m_b) for 2x2-block rows; P and R hold 1 or 2 values. */
enum {
  IFILT_MG_S_ROWPTR = 0,  /* int64 [rows_l+1] (level 0: empty) */
  IFILT_MG_S_COL = 1,     /* int32 [nnz_s] */
  IFILT_MG_S_VAL = 2,     /* double [nnz_s][2 or 4] */
  IFILT_MG_P_ROWPTR = 3,  /* int64 [rows_l+1]: P_l, columns index level l+1 */
  IFILT_MG_P_COL = 4,
  IFILT_MG_P_VAL = 5,     /* double [nnz_p][1 or 2] */
  IFILT_MG_DK = 6,        /* double [rows_l]: diagonal of K_l */
  IFILT_MG_DM = 7,        /* double [rows_l]: diagonal of M_l */
  IFILT_MG_OMEGA = 8      /* double [2]: prolongator-smoothing weight, smoother weight of level l */
};
/* Copy one array of level `level` to `dst` of `bytes` bytes (EINVAL if too
 * small or out of range); *written receives the byte count. */
ifilt_status ifilt_mesh_multigrid_export(ifilt_mesh mesh, int32_t level, int32_t what, void* dst, size_t bytes,
                                         size_t* written);

/* ---- Mesh cache files.  Preparation depends on the mesh only (Sect. 2.2
 * separates it from the solves, whose every scale and field reuse it); at
 * 10 M vertices its host half and the multigrid hierarchy take tens of
 * seconds, so a prepared mesh can be written to a file and read back in
 * another process, bit for bit.  Files are little-endian and carry the
 * descriptor key, a format number, the preparation code's revision and a
 * checksum of their contents. */

/* 64-bit key of a descriptor (never 0): a hash of every field, of the arrays it
 * points to (coords [V][dim], tri [T][3], ocean taken as 0/1 flags) and of the
 * preparation revision.  Equal keys mean the same prepared mesh, up to hash
 * collisions.  Errors: EINVAL (null pointers, non-positive sizes). */
ifilt_status ifilt_mesh_key(const ifilt_mesh_desc* desc, uint64_t* key);

#define IFILT_SAVE_MULTIGRID 1  /* also write the multigrid hierarchy (built first if needed) */
/* Write the host half of `mesh` (what ifilt_prepare_mesh_host computes, and
 * the hierarchy with IFILT_SAVE_MULTIGRID) to the host path `path`, replacing
 * any file there.  The file is written under a temporary name in the same
 * directory and renamed into place.  Errors: EINVAL (null mesh or path,
 * unknown flags), ECACHE (cannot write). */
ifilt_status ifilt_mesh_save(ifilt_mesh mesh, const char* path, int32_t flags);

/* Read a file written by ifilt_mesh_save into a new host-only handle, as
 * ifilt_prepare_mesh_host returns (ifilt_mesh_upload makes it solvable; the
 * hierarchy, if the file holds it, is not rebuilt).  expect_key != 0 demands
 * the key of the descriptor the mesh was prepared from (ifilt_mesh_key).
 * Every array is checked before the handle is returned: sizes, row pointers,
 * index ranges, sorted columns, finite values.  Errors: EINVAL (null
 * arguments), ECACHE (see the status), ENOMEM. */
ifilt_status ifilt_mesh_load_host(const char* path, uint64_t expect_key, ifilt_mesh* out);

/* Descriptor key of a prepared or loaded mesh (0 if unknown). */
ifilt_status ifilt_mesh_get_key(ifilt_mesh mesh, uint64_t* key);

/* Filter a batch of fields at a list of wavenumbers (Eq. 1-2 solved as in
 * Sect. 2.2.2).
 *   fields  : device double [n_fields][n_comp][n_in]  (original mesh order)
 *   k       : host double [n_k], k = 1/l > 0 in radians per coordinate unit
 *   out     : device double [n_fields][n_k][n_comp][n_out]
 *   stats   : host [n_fields][n_k][n_sys] or NULL, n_sys = 2 for the cell
 *             placement (u and v solved separately) and 1 otherwise
 * Land entries (not unknowns) of scalar-vertex and cell outputs copy the input;
 * vertex-vector outputs are zero there.  Synchronises `stream` before
 * returning.  Device scratch is taken from the stream-ordered allocator and
 * returned before the call ends. */
ifilt_status ifilt_solve(ifilt_mesh mesh, const ifilt_solve_opts* opts,
                         int32_t n_fields, const double* fields, int32_t n_k,
                         const double* k, double* out, ifilt_col_stats* stats,
                         void* stream);

/* One solve of a multi-item call: the arguments of ifilt_solve. */
typedef struct {
  ifilt_mesh mesh;
  ifilt_solve_opts opts;
  int32_t n_fields;
  const double* fields;      /* device */
  int32_t n_k;
  const double* k;           /* host */
  double* out;               /* device */
  ifilt_col_stats* stats;    /* host or NULL */
} ifilt_solve_item;

/* Several solves at once (e.g. the vertex-vector and the cell placement of
 * the same velocity field): every item gets its own batched solver on its
 * own stream and the solvers step together, so one item's narrow final phase
 * overlaps with the others' work.  Items use the batched method (their
 * `method` is ignored).  Same results and errors as calling ifilt_solve for
 * each item; returns the worst status.  Synchronises `stream`. */
ifilt_status ifilt_solve_many(int32_t n_items, const ifilt_solve_item* items, void* stream);

/* Coarse-grained energy spectrum of filtered fields (Sect. 1, 4, 5; the paper
 * gives no formula, the reading is):
 *   energy[f][j] = sum_i w_i 1/2 sum_c out[f][j][c][i]^2 / sum_i w_i over unknowns i
 *   spec[f][j]   = (energy[f][j+1] - energy[f][j]) / (k[j+1] - k[j]), k ascending,
 *   kmid[j]      = sqrt(k[j] k[j+1])
 * with w the lumped mass (A_v or A_c).  `filtered` is device memory in the
 * layout ifilt_solve writes; k must be strictly ascending.  energy [F][n_k],
 * spec [F][n_k-1] and kmid [n_k-1] are host memory (spec/kmid may be NULL).
 * Synchronises `stream`. */
ifilt_status ifilt_spectrum(ifilt_mesh mesh, int32_t n_fields, int32_t n_k,
                            const double* k, const double* filtered,
                            double* energy, double* spec, double* kmid, void* stream);

/* The spectrum of ifilt_spectrum for callers that cannot allocate device
 * memory during a call: for instance a service that reserves all of HBM up
 * front for resident meshes and request buffers, or a process held to a
 * fixed device-memory budget, where taking scratch from an allocator would
 * fail or stall.  This entry point calls no allocator (no cudaMalloc,
 * cudaFree, memory pool or torch allocation).  Its scratch is one fixed array
 * of 532 KB inside the library, resident on every device that loads the
 * library until the process exits.  The paper has no counterpart; this is an
 * operational variant of ifilt_spectrum with the same arguments, layout,
 * results and synchronisation.
 *   - n_fields * n_k must not exceed 512 (EINVAL otherwise).
 *   - The first call on a device looks up the array's device address; make
 *     that first call before any stream capture on that device.  Later calls
 *     outside a capture look it up again, so a device reset (which reloads
 *     the library's device code) does not leave a stale address behind.
 *   - All calls share the one array: calls that overlap on the GPU (other
 *     streams, other host threads) race and must be serialised by the caller.
 *     Every scratch value a call reads is written earlier in the same call,
 *     so nothing has to be cleared between calls. */
ifilt_status ifilt_spectrum_noalloc(ifilt_mesh mesh, int32_t n_fields, int32_t n_k,
                                    const double* k, const double* filtered,
                                    double* energy, double* spec, double* kmid, void* stream);

/* Device memory an ifilt_solve call with these options would take from the
 * stream-ordered allocator (upper bound), for admission control. */
size_t ifilt_solve_scratch_bytes(ifilt_mesh mesh, const ifilt_solve_opts* opts,
                                 int32_t n_fields, int32_t n_k);

/* ------------------------------------------------------------------------
 * Serving: a persistent request loop over resident prepared meshes.
 *
 * A worker thread keeps one batched solver per (mesh, order, precision,
 * n = 2 form).  Requests are split into columns (field x system x scale) that
 * join the solver's queue; at every step boundary (check_every iterations)
 * finished columns retire and queued ones are admitted into the freed lanes
 * while device memory stays within the budget (continuous batching).  The
 * solvers run on separate streams, so the work of different meshes and
 * orders overlaps on the device.  A column's result does not depend on which
 * other columns share its batch beyond rounding (the batch width changes the
 * grouping of partial sums), so a request gives the same result, within the
 * solve tolerance, alone or in a mix.
 * ------------------------------------------------------------------------ */
typedef struct ifilt_server_s* ifilt_server;

typedef struct {
  int64_t memory_budget;     /* device bytes the solvers may hold; 0 = free memory at creation minus reserve */
  int64_t reserve;           /* bytes kept free when memory_budget = 0; 0 = 2 GiB */
  int32_t max_lanes;         /* lane capacity of each solver; 0 = 256 */
  int32_t check_every;       /* iterations per step; 0 = 32 */
} ifilt_server_opts;

typedef struct {
  int32_t state;             /* 0 queued, 1 running, 2 done, 3 failed */
  int32_t status;            /* when done: IFILT_OK or IFILT_NOT_CONVERGED; when failed: the error */
  int32_t columns, columns_done;
  double t_submit, t_start, t_done;  /* seconds on the server's monotonic clock (t_start: handed to its solver) */
} ifilt_request_info;

/* Start a server on the current device.  Errors: EINVAL, ENOMEM, ECUDA. */
ifilt_status ifilt_server_create(const ifilt_server_opts* opts, ifilt_server* out);

/* Queue a request.  Arguments as ifilt_solve (method is ignored: requests are
 * always batched).  `fields` (device) must hold its final values when the
 * call is made; `fields`, `out` (device) and `stats` (host, may be NULL) must
 * stay valid until the request is done.  `k` is copied.  *request receives an
 * id for ifilt_server_wait.  The mesh must outlive the server's use of it.
 * Errors: EINVAL (bad options, server failed or stopping). */
ifilt_status ifilt_server_submit(ifilt_server server, ifilt_mesh mesh, const ifilt_solve_opts* opts,
                                 int32_t n_fields, const double* fields, int32_t n_k, const double* k,
                                 double* out, ifilt_col_stats* stats, int64_t* request);

/* Wait up to timeout_ms (0 = just look) for a request to finish and fill
 * *info.  Returns IFILT_OK with info->state telling where the request is;
 * EINVAL for an unknown id.  Finished requests are forgotten by
 * ifilt_server_forget. */
ifilt_status ifilt_server_wait(ifilt_server server, int64_t request, int32_t timeout_ms, ifilt_request_info* info);

/* Drop the record of a finished request. */
ifilt_status ifilt_server_forget(ifilt_server server, int64_t request);

/* Seconds on the server's clock (the clock of the request timestamps). */
double ifilt_server_now(ifilt_server server);

/* Stop the worker at its next step boundary, cancel every request that has
 * not finished (state 3, status IFILT_EINVAL; its outputs are partial), free
 * the solvers and the server.  Wait for requests first to drain.  NULL is
 * ignored. */
void ifilt_server_destroy(ifilt_server server);

/* Per-kernel timing sampled with CUDA events on the launching stream while
 * profiling is on (off by default).  Each record: kernel name, launches,
 * sampled launches, summed sampled milliseconds, algorithmic bytes per launch
 * (averaged over the sampled launches). */
typedef struct {
  char name[32];
  int64_t launches;
  int64_t samples;
  double sampled_ms;
  double bytes_per_launch;
} ifilt_kernel_profile;

void ifilt_profile_enable(int32_t on);
/* Writes up to `max` records, returns how many kernels have records. */
int32_t ifilt_profile_read(ifilt_kernel_profile* out, int32_t max);
void ifilt_profile_reset(void);

/* Thread-local message for the last non-OK status of this thread. */
const char* ifilt_last_error(void);

/* Library version string. */
const char* ifilt_version(void);

#ifdef __cplusplus
}
#endif

#endif /* IFILT_H */
