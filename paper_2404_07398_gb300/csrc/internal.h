// Internal declarations of libifilt (not part of the C ABI).
#pragma once

#include <array>
#include <cstdint>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include "../../include/ifilt.h"

namespace ifilt {

// ---------------------------------------------------------------- errors
struct Error {
  ifilt_status status;
  std::string msg;
};
[[noreturn]] void fail(ifilt_status st, const char* fmt, ...);
void set_last_error(const std::string& msg);

#define IFILT_CUDA(call)                                                          \
  do {                                                                            \
    cudaError_t e_ = (call);                                                      \
    if (e_ != cudaSuccess)                                                        \
      ::ifilt::fail(e_ == cudaErrorMemoryAllocation ? IFILT_ENOMEM : IFILT_ECUDA, \
                    "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),       \
                    __FILE__, __LINE__);                                          \
  } while (0)

// Wall-clock phases of preparation, printed to stderr when IFILT_TRACE_PREPARE=1.
struct PhaseClock {
  explicit PhaseClock(const char* what);
  void lap(const char* phase);
  const char* what;
  bool on;
  double t0;
};

// ---------------------------------------------------------------- host side
// Compressed sparse rows; `nval` doubles per entry (1 = scalar, 2 = block
// [[a, b], [-b, a]] stored as (a, b)).
struct HostCSR {
  int32_t n = 0;
  int32_t nval = 1;
  std::vector<int64_t> row_ptr;
  std::vector<int32_t> col;
  std::vector<double> val;
  int64_t nnz() const { return row_ptr.empty() ? 0 : row_ptr.back(); }
};

struct HostPrepared {
  uint64_t key = 0;               // ifilt_mesh_key of the descriptor it was prepared from
  double mg_strength = 0.0;       // multigrid aggregation threshold (ifilt_mesh_desc)
  int32_t placement = 0, geometry = 0, max_order = 1, reorder = 1;
  int32_t n_rows = 0, n_in = 0, n_out = 0, n_comp = 1;
  std::vector<int32_t> perm;      // device row -> original index (vertex or triangle)
  std::vector<double> mass;       // lumped mass per row
  HostCSR K;                      // n = 1 operator, l-free, device order, sorted columns
  HostCSR G2;                     // K M^-1 K (max_order >= 2)
  std::vector<HostCSR> Gn;        // G_n = G_(n-1) M^-1 K for n = 3 .. max_order (index n - 3)
  bool products_pending = false;  // G2, Gn not formed yet: the upload forms them on the device
  // vertex-vector right-hand side: b_i = sum over incident ocean triangles c of (A_c / 3) u_c
  std::vector<int64_t> proj_ptr;
  std::vector<int32_t> proj_cell;
  std::vector<double> proj_w;
};

// products = false leaves G2 and the higher orders to the upload (on the device)
HostPrepared prepare_host(const ifilt_mesh_desc& d, bool products = true);
// the products of prepare_host, formed on the host
void host_products(HostPrepared& hp);

// The complex-shift factorisation serves order 2 only (orders >= 3 run on G_n in real arithmetic).
inline bool complex_form(const ifilt_solve_opts& o) { return o.order == 2 && o.n2_solver != IFILT_N2_REAL; }

// ---------------------------------------------------------------- device side
// Sliced ELL: rows are cut into slices of `slice_h`; slice s holds its rows
// row-major with width slice_w[s] (a multiple of 4) starting at slice_off[s].
// Padding entries point at their own row with value 0.
struct DevEll {
  int32_t n = 0, slice_h = 0, n_slices = 0, nval = 1, max_width = 0;
  int64_t entries = 0;
  int64_t* slice_off = nullptr;
  int32_t* slice_w = nullptr;
  int32_t* col = nullptr;
  double* val64 = nullptr;
  float* val32 = nullptr;
  float* val32lo = nullptr;  // val64 - val32 rounded to float (double-float residual)
  __nv_bfloat16* val16 = nullptr;
  // per row: its entries rounded up to a multiple of 4, counted in fours (255: the
  // slice's full width); a gather stops there instead of at the slice's width
  uint8_t* rowq = nullptr;
};

// One level of the multigrid preconditioner on the device: the pair
// (K_l, M_l) as one ELL with both values per entry (level 0 uses the mesh's
// K and lumped mass instead), the prolongation P_l (rows of level l) and the
// restriction R_l = P_l^T (rows of level l+1), FP32 diagonals of K_l and M_l.
struct DevMgLevel {
  int32_t n = 0;
  DevEll S, P, R;
  float* dk32 = nullptr;
  float* dm32 = nullptr;
  double omega = 2.0 / 3.0;  // damped-Jacobi weight of the smoother on this level
};
struct MgHost;  // multigrid.h

struct DevCSR {
  int32_t n = 0;          // rows of the real (expanded) matrix
  int64_t nnz = 0;
  int64_t* row_ptr = nullptr;
  int32_t* col = nullptr;
  double* val = nullptr;
};

}  // namespace ifilt

struct ifilt_mesh_s {
  ifilt::HostPrepared host;
  int device = -1;               // -1 until uploaded
  int32_t slice_h = 0;
  int64_t bytes = 0;
  std::vector<void*> allocations;
  // device arrays
  int32_t* perm = nullptr;       // [n_rows]
  double* mass = nullptr;        // [n_rows]
  float* mass32 = nullptr;       // [n_rows] the same in FP32 (FP32 kernels)
  float* mass32lo = nullptr;     // [n_rows] mass - mass32 rounded to float (double-float residual)
  double* diag_k = nullptr;      // [n_rows] diagonal of K (K~ for vectors)
  double* diag_g2 = nullptr;     // [n_rows]
  float* diag_k32 = nullptr;     // [n_rows] FP32 copies (Jacobi preconditioning in FP32 kernels)
  float* diag_g2_32 = nullptr;   // [n_rows]
  int64_t* proj_ptr = nullptr;
  int32_t* proj_cell = nullptr;
  double* proj_w = nullptr;
  double* w_out = nullptr;       // [n_out] lumped mass of each output entry (0 where not an unknown)
  int32_t* inv_perm = nullptr;   // [n_out] device row of each output entry, -1 where not an unknown
  ifilt::DevEll ell_k, ell_g2;
  ifilt::DevCSR csr_k, csr_g2;   // real expanded CSR in FP64 (vector placement: interleaved u,v rows)
  // orders n >= 3 (index n - 3): G_n as ELL and CSR, its diagonal in FP64 and FP32
  std::vector<ifilt::DevEll> ell_gn;
  std::vector<ifilt::DevCSR> csr_gn;
  std::vector<double*> diag_gn;
  std::vector<float*> diag_gn32;
  // multigrid preconditioner, built on first use (host) and uploaded on first device use
  std::mutex mg_mu;
  std::shared_ptr<ifilt::MgHost> mg_host;
  std::vector<ifilt::DevMgLevel> mg_dev;
  // autotuned launch shapes of the batched solver, per engine kind and tile width
  std::mutex tune_mu;
  std::map<std::string, std::array<int, 6>> tune;
};

namespace ifilt {

// device upload (device_mesh.cu)
void upload_mesh(ifilt_mesh_s* m, int32_t slice_h, cudaStream_t st);
void free_mesh(ifilt_mesh_s* m);
// multigrid hierarchy of a mesh: built on the host once, uploaded once
const MgHost& multigrid_host(ifilt_mesh_s* m);
// mesh cache files (cache.cpp)
uint64_t mesh_key(const ifilt_mesh_desc& d);
void save_mesh(ifilt_mesh_s* m, const char* path, int32_t flags);
ifilt_mesh_s* load_mesh_host(const char* path, uint64_t expect_key);
const std::vector<DevMgLevel>& multigrid_device(ifilt_mesh_s* m, cudaStream_t st);

// solvers (solve_plain.cu, solve_batched.cu)
ifilt_status solve_plain(ifilt_mesh_s* m, const ifilt_solve_opts& o, int32_t F, const double* fields,
                         int32_t nk, const double* k, double* out, ifilt_col_stats* stats,
                         cudaStream_t st);
ifilt_status solve_batched(ifilt_mesh_s* m, const ifilt_solve_opts& o, int32_t F,
                           const double* fields, int32_t nk, const double* k, double* out,
                           ifilt_col_stats* stats, cudaStream_t st);
ifilt_status solve_many(int32_t n, const ifilt_solve_item* items, cudaStream_t st);
size_t batched_scratch_bytes(const ifilt_mesh_s* m, const ifilt_solve_opts& o, int32_t F, int32_t nk);
size_t plain_scratch_bytes(const ifilt_mesh_s* m, const ifilt_solve_opts& o);

// right-hand side and output maps (io.cu)
// b and x0 of one system in device order, layout [n_rows][nsub] (nsub = 2 for
// the vertex-vector placement, else 1).  `field` is one field [n_comp][n_in];
// `comp` selects the component for the cell placement.
void launch_rhs(ifilt_mesh_s* m, const double* field, int comp, double* b, double* x0, cudaStream_t st);
// out[c][o] for every output entry o of one system: the solution where o is an
// unknown, the input (scalar, cell) or 0 (vector) elsewhere.  x is [n_rows][nsub]
// with stride `ld` doubles between consecutive sub-values (1 for a packed system).
void launch_output_plain(ifilt_mesh_s* m, const double* x, const double* field, int comp,
                         double* out_sys, cudaStream_t st);

// ---------------------------------------------------------------- engines
// One column of work: a (field, system, wavenumber) solve.  `field` is the
// caller's device field [n_comp][n_in]; `out` the caller's device block
// [n_comp][n_out] of that (field, wavenumber); `stat` a host record or null.
struct ColumnJob {
  int64_t request = 0;
  const double* field = nullptr;
  int sys = 0;
  double k = 0.0;
  double* out = nullptr;
  ifilt_col_stats* stat = nullptr;
};

struct ColumnDone {
  int64_t request;
  int status;  // IFILT_OK or IFILT_NOT_CONVERGED
};

// A persistent batched solver for one mesh and one (order, precision, n = 2
// form): columns queue up, are admitted into free lanes of the tiles at step
// boundaries, iterate together, and retire (outputs written) when done.
// launch() enqueues one step on the engine's stream; settle() waits for it
// and retires finished columns.  Not thread-safe: one owner drives it.
class Engine {
 public:
  virtual ~Engine() = default;
  virtual void submit(const std::vector<ColumnJob>& jobs) = 0;
  virtual bool idle() const = 0;
  virtual void launch() = 0;
  virtual void settle(std::vector<ColumnDone>& done) = 0;
  virtual int64_t bytes_held() const = 0;   // device memory held now
  virtual void set_budget(int64_t budget) = 0;
  virtual int running() const = 0;          // columns in the tiles
  virtual int pending() const = 0;          // columns waiting for lanes
  virtual cudaStream_t stream() const = 0;
  // kernels launched so far and sampled kernel timings (profiling)
  virtual void report_profile() = 0;
};

// `budget` bounds the device memory the engine may take (0 = no bound).
Engine* make_engine(ifilt_mesh_s* m, const ifilt_solve_opts& o, cudaStream_t st, int64_t budget);

// spectrum (spectrum.cu)
// energy [F][nk], spec [F][nk-1], kmid [nk-1] written to device buffers;
// `partial` holds F*nk*nb doubles.
void spectrum_device(ifilt_mesh_s* m, int32_t F, int32_t nk, const double* k_dev, const double* filtered,
                     double* energy, double* spec, double* kmid, double* partial, int nb, cudaStream_t st);

// spectrum with its scratch in a fixed device array (noalloc.cu)
ifilt_status spectrum_noalloc(ifilt_mesh_s* m, int32_t F, int32_t K, const double* k, const double* filtered,
                              double* energy, double* spec, double* kmid, cudaStream_t st);

// profiling (abi.cpp): per-kernel launch counts and CUDA-event samples
bool profiling_on();
void profile_add(const char* name, int64_t launches, int64_t samples, double sampled_ms,
                 double bytes_per_launch);
// count kernel launches of this library (reported as "(all kernels)")
void profile_count(int64_t launches);

// stream-ordered scratch
void* scratch_alloc(size_t bytes, cudaStream_t st);
void scratch_free(void* p, cudaStream_t st);

}  // namespace ifilt
