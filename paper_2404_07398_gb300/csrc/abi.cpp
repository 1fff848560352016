// extern "C" entry points of libifilt (declared in include/ifilt.h), error
// reporting, the stream-ordered scratch pool and the kernel profile registry.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>

#include <nvtx3/nvToolsExt.h>

#include "internal.h"
#include "multigrid.h"

namespace ifilt {

static thread_local std::string g_last_error;

void set_last_error(const std::string& msg) { g_last_error = msg; }

[[noreturn]] void fail(ifilt_status st, const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  throw Error{st, std::string(buf)};
}

// ---- scratch: one memory pool per device, kept warm between calls
static std::mutex g_pool_mu;
static std::map<int, cudaMemPool_t> g_pools;

static cudaMemPool_t pool_for_current_device() {
  int dev = 0;
  IFILT_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_pool_mu);
  auto it = g_pools.find(dev);
  if (it != g_pools.end()) return it->second;
  cudaMemPoolProps props{};
  props.allocType = cudaMemAllocationTypePinned;
  props.handleTypes = cudaMemHandleTypeNone;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev;
  cudaMemPool_t pool;
  IFILT_CUDA(cudaMemPoolCreate(&pool, &props));
  uint64_t thr = UINT64_MAX;
  IFILT_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));
  g_pools[dev] = pool;
  return pool;
}

void* scratch_alloc(size_t bytes, cudaStream_t st) {
  void* p = nullptr;
  cudaMemPool_t pool = pool_for_current_device();
  cudaError_t e = cudaMallocFromPoolAsync(&p, bytes < 256 ? 256 : bytes, pool, st);
  if (e != cudaSuccess) {
    // give memory held by the pool but not in use back to the device, then retry once
    cudaGetLastError();
    cudaStreamSynchronize(st);
    cudaMemPoolTrimTo(pool, 0);
    e = cudaMallocFromPoolAsync(&p, bytes < 256 ? 256 : bytes, pool, st);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    fail(IFILT_ENOMEM, "device scratch of %zu bytes not available: %s", bytes, cudaGetErrorString(e));
  }
  return p;
}

void scratch_free(void* p, cudaStream_t st) {
  if (p) cudaFreeAsync(p, st);
}

// ---- profiling registry
static std::atomic<bool> g_prof{false};
static std::mutex g_prof_mu;
struct ProfRec {
  int64_t launches = 0, samples = 0;
  double ms = 0.0, bytes_sum = 0.0;
};
static std::map<std::string, ProfRec> g_prof_recs;

bool profiling_on() { return g_prof.load(); }

void profile_add(const char* name, int64_t launches, int64_t samples, double sampled_ms, double bytes_per_launch) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  ProfRec& r = g_prof_recs[name];
  r.launches += launches;
  r.samples += samples;
  r.ms += sampled_ms;
  r.bytes_sum += bytes_per_launch * (double)samples;
}

void profile_count(int64_t launches) {
  if (!profiling_on()) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof_recs["(all kernels)"].launches += launches;
}

}  // namespace ifilt

using namespace ifilt;

#define IFILT_GUARD_BEGIN try {
#define IFILT_GUARD_END                                   \
  }                                                       \
  catch (const Error& e) {                                \
    set_last_error(e.msg);                                \
    return e.status;                                      \
  }                                                       \
  catch (const std::bad_alloc&) {                         \
    set_last_error("host allocation failed");             \
    return IFILT_ENOMEM;                                  \
  }                                                       \
  catch (const std::exception& e) {                       \
    set_last_error(std::string("internal error: ") + e.what()); \
    return IFILT_ECUDA;                                   \
  }

namespace {

struct DeviceScope {
  int prev = -1;
  explicit DeviceScope(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) IFILT_CUDA(cudaSetDevice(dev));
  }
  ~DeviceScope() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

void check_mesh(ifilt_mesh m) {
  if (!m) fail(IFILT_EINVAL, "null mesh handle");
}

void check_uploaded(ifilt_mesh m) {
  check_mesh(m);
  if (m->device < 0) fail(IFILT_EINVAL, "mesh was prepared on the host only; call ifilt_mesh_upload first");
}

}  // namespace

// An NVTX range around each heavy entry point, so that a timeline tool shows
// where the library's time goes (no cost without a tool attached).
struct ApiRange {
  explicit ApiRange(const char* name) { nvtxRangePushA(name); }
  ~ApiRange() { nvtxRangePop(); }
  ApiRange(const ApiRange&) = delete;
  ApiRange& operator=(const ApiRange&) = delete;
};

extern "C" {

const char* ifilt_last_error(void) { return g_last_error.c_str(); }

const char* ifilt_version(void) { return "ifilt 0.1 (sm_103a)"; }

ifilt_status ifilt_prepare_mesh(const ifilt_mesh_desc* desc, void* stream, ifilt_mesh* out) {
  ApiRange range_("ifilt_prepare_mesh");
  IFILT_GUARD_BEGIN
  if (!desc || !out) fail(IFILT_EINVAL, "null argument");
  *out = nullptr;
  cudaStream_t st = (cudaStream_t)stream;
  ifilt_mesh_s* m = new ifilt_mesh_s();
  try {
    IFILT_CUDA(cudaGetDevice(&m->device));
    m->host = prepare_host(*desc, /*products=*/false);  // the upload forms G2 and G_n on the device
    m->host.key = mesh_key(*desc);
    m->slice_h = desc->ell_slice;
    upload_mesh(m, desc->ell_slice, st);
  } catch (...) {
    free_mesh(m);
    delete m;
    throw;
  }
  *out = m;
  set_last_error("");
  return IFILT_OK;
  IFILT_GUARD_END
}

ifilt_status ifilt_prepare_mesh_host(const ifilt_mesh_desc* desc, ifilt_mesh* out) {
  ApiRange range_("ifilt_prepare_mesh_host");
  IFILT_GUARD_BEGIN
  if (!desc || !out) fail(IFILT_EINVAL, "null argument");
  *out = nullptr;
  ifilt_mesh_s* m = new ifilt_mesh_s();
  try {
    m->host = prepare_host(*desc);
    m->host.key = mesh_key(*desc);
    m->slice_h = desc->ell_slice;
  } catch (...) {
    delete m;
    throw;
  }
  *out = m;
  set_last_error("");
  return IFILT_OK;
  IFILT_GUARD_END
}

ifilt_status ifilt_mesh_upload(ifilt_mesh m, void* stream) {
  ApiRange range_("ifilt_mesh_upload");
  IFILT_GUARD_BEGIN
  check_mesh(m);
  if (m->device >= 0) return IFILT_OK;
  int dev = 0;
  IFILT_CUDA(cudaGetDevice(&dev));
  try {
    m->device = dev;
    upload_mesh(m, m->slice_h, (cudaStream_t)stream);
  } catch (...) {
    free_mesh(m);
    m->device = -1;
    throw;
  }
  return IFILT_OK;
  IFILT_GUARD_END
}

ifilt_status ifilt_mesh_key(const ifilt_mesh_desc* desc, uint64_t* key) {
  IFILT_GUARD_BEGIN
  if (!desc || !key) fail(IFILT_EINVAL, "null argument");
  *key = mesh_key(*desc);
  return IFILT_OK;
  IFILT_GUARD_END
}

ifilt_status ifilt_mesh_get_key(ifilt_mesh m, uint64_t* key) {
  IFILT_GUARD_BEGIN
  check_mesh(m);
  if (!key) fail(IFILT_EINVAL, "null argument");
  *key = m->host.key;
  return IFILT_OK;
  IFILT_GUARD_END
}

ifilt_status ifilt_mesh_save(ifilt_mesh m, const char* path, int32_t flags) {
  ApiRange range_("ifilt_mesh_save");
  IFILT_GUARD_BEGIN
  check_mesh(m);
  save_mesh(m, path, flags);
  return IFILT_OK;
  IFILT_GUARD_END
}

ifilt_status ifilt_mesh_load_host(const char* path, uint64_t expect_key, ifilt_mesh* out) {
  ApiRange range_("ifilt_mesh_load_host");
  IFILT_GUARD_BEGIN
  if (!out) fail(IFILT_EINVAL, "null argument");
  *out = nullptr;
  *out = load_mesh_host(path, expect_key);
  set_last_error("");
  return IFILT_OK;
  IFILT_GUARD_END
}

void ifilt_release_mesh(ifilt_mesh m) {
  if (!m) return;
  if (m->device >= 0) {
    try {
      DeviceScope ds(m->device);
      free_mesh(m);
    } catch (...) {
    }
  }
  delete m;
}

ifilt_status ifilt_mesh_info(ifilt_mesh m, ifilt_mesh_info_t* out) {
  IFILT_GUARD_BEGIN
  check_mesh(m);
  if (!out) fail(IFILT_EINVAL, "null output");
  const HostPrepared& h = m->host;
  std::memset(out, 0, sizeof *out);
  out->placement = h.placement;
  out->geometry = h.geometry;
  out->max_order = h.max_order;
  out->reorder = h.reorder;
  out->n_rows = h.n_rows;
  out->n_in = h.n_in;
  out->n_out = h.n_out;
  out->n_comp = h.n_comp;
  out->nnz_k = h.K.nnz();
  out->nnz_g2 = h.G2.nnz();
  out->ell_slice = m->device >= 0 ? m->ell_k.slice_h : m->slice_h;
  out->ell_width_k = m->ell_k.max_width;
  out->ell_width_g2 = m->ell_g2.max_width;
  out->device_bytes = m->bytes;
  return IFILT_OK;
  IFILT_GUARD_END
}

ifilt_status ifilt_mesh_multigrid(ifilt_mesh m, ifilt_multigrid_info* info) {
  ApiRange range_("ifilt_mesh_multigrid");
  IFILT_GUARD_BEGIN
  check_mesh(m);
  if (!info) fail(IFILT_EINVAL, "null info");
  const MgHost& h = multigrid_host(m);
  std::memset(info, 0, sizeof(*info));
  info->n_levels = (int32_t)std::min<size_t>(h.levels.size(), IFILT_MG_MAX_LEVELS);
  for (int32_t l = 0; l < info->n_levels; l++) {
    info->rows[l] = h.levels[l].n;
    info->nnz_s[l] = l == 0 ? m->host.K.nnz() : h.levels[l].S.nnz();
    info->nnz_p[l] = h.levels[l].P.nnz();
  }
  return IFILT_OK;
  IFILT_GUARD_END
}

ifilt_status ifilt_mesh_multigrid_export(ifilt_mesh m, int32_t level, int32_t what, void* dst, size_t bytes,
                                         size_t* written) {
  IFILT_GUARD_BEGIN
  check_mesh(m);
  if (!dst && bytes) fail(IFILT_EINVAL, "null destination");
  const MgHost& h = multigrid_host(m);
  if (level < 0 || level >= (int32_t)h.levels.size()) fail(IFILT_EINVAL, "level %d outside the hierarchy", level);
  const MgHostLevel& L = h.levels[level];
  const void* src = nullptr;
  size_t need = 0;
  double omega[2];
  switch (what) {
    case IFILT_MG_S_ROWPTR: src = L.S.row_ptr.data(); need = L.S.row_ptr.size() * 8; break;
    case IFILT_MG_S_COL: src = L.S.col.data(); need = L.S.col.size() * 4; break;
    case IFILT_MG_S_VAL: src = L.S.val.data(); need = L.S.val.size() * 8; break;
    case IFILT_MG_P_ROWPTR: src = L.P.row_ptr.data(); need = L.P.row_ptr.size() * 8; break;
    case IFILT_MG_P_COL: src = L.P.col.data(); need = L.P.col.size() * 4; break;
    case IFILT_MG_P_VAL: src = L.P.val.data(); need = L.P.val.size() * 8; break;
    case IFILT_MG_DK: src = L.dk.data(); need = L.dk.size() * 8; break;
    case IFILT_MG_DM: src = L.dm.data(); need = L.dm.size() * 8; break;
    case IFILT_MG_OMEGA: {
      omega[0] = L.omega_p;
      omega[1] = L.omega_s;
      src = omega;
      need = sizeof omega;
      break;
    }
    default: fail(IFILT_EINVAL, "unknown multigrid export selector %d", what);
  }
  if (bytes < need) fail(IFILT_EINVAL, "destination holds %zu bytes, %zu needed", bytes, need);
  if (need) std::memcpy(dst, src, need);
  if (written) *written = need;
  return IFILT_OK;
  IFILT_GUARD_END
}

ifilt_status ifilt_mesh_export_gn(ifilt_mesh m, int32_t order, int32_t part, void* dst, size_t bytes,
                                  size_t* written) {
  IFILT_GUARD_BEGIN
  check_mesh(m);
  const HostPrepared& h = m->host;
  if (order < 2 || order > h.max_order) fail(IFILT_EINVAL, "order %d outside 2..%d (mesh max_order)", order, h.max_order);
  const HostCSR& G = order == 2 ? h.G2 : h.Gn[(size_t)order - 3];
  const void* src = nullptr;
  size_t need = 0;
  switch (part) {
    case 0: src = G.row_ptr.data(); need = G.row_ptr.size() * 8; break;
    case 1: src = G.col.data(); need = G.col.size() * 4; break;
    case 2: src = G.val.data(); need = G.val.size() * 8; break;
    default: fail(IFILT_EINVAL, "unknown part %d (0 row pointers, 1 columns, 2 values)", part);
  }
  if (written) *written = need;
  if (!dst && bytes == 0) return IFILT_OK;
  if (!dst) fail(IFILT_EINVAL, "null destination");
  if (bytes < need) fail(IFILT_EINVAL, "destination holds %zu bytes, %zu needed", bytes, need);
  if (need) std::memcpy(dst, src, need);
  return IFILT_OK;
  IFILT_GUARD_END
}

ifilt_status ifilt_mesh_export(ifilt_mesh m, int32_t what, void* dst, size_t bytes) {
  IFILT_GUARD_BEGIN
  check_mesh(m);
  if (!dst) fail(IFILT_EINVAL, "null destination");
  const HostPrepared& h = m->host;
  const void* src = nullptr;
  size_t need = 0;
  switch (what) {
    case IFILT_EXPORT_PERM: src = h.perm.data(); need = h.perm.size() * 4; break;
    case IFILT_EXPORT_K_ROWPTR: src = h.K.row_ptr.data(); need = h.K.row_ptr.size() * 8; break;
    case IFILT_EXPORT_K_COL: src = h.K.col.data(); need = h.K.col.size() * 4; break;
    case IFILT_EXPORT_K_VAL: src = h.K.val.data(); need = h.K.val.size() * 8; break;
    case IFILT_EXPORT_MASS: src = h.mass.data(); need = h.mass.size() * 8; break;
    case IFILT_EXPORT_G2_ROWPTR: src = h.G2.row_ptr.data(); need = h.G2.row_ptr.size() * 8; break;
    case IFILT_EXPORT_G2_COL: src = h.G2.col.data(); need = h.G2.col.size() * 4; break;
    case IFILT_EXPORT_G2_VAL: src = h.G2.val.data(); need = h.G2.val.size() * 8; break;
    default: fail(IFILT_EINVAL, "unknown export selector %d", what);
  }
  if (bytes < need) fail(IFILT_EINVAL, "destination holds %zu bytes, %zu needed", bytes, need);
  if (need) std::memcpy(dst, src, need);
  return IFILT_OK;
  IFILT_GUARD_END
}

static void check_opts(ifilt_mesh m, const ifilt_solve_opts* o) {
  if (!o) fail(IFILT_EINVAL, "null options");
  if (o->order < 1 || o->order > m->host.max_order)
    fail(IFILT_EINVAL, "order %d outside 1..%d (mesh max_order)", o->order, m->host.max_order);
  if (!(o->tol > 0.0) || !std::isfinite(o->tol)) fail(IFILT_EINVAL, "tol must be positive");
  if (o->precision < IFILT_PREC_FP64 || o->precision > IFILT_PREC_BF16_IR) fail(IFILT_EINVAL, "unknown precision");
  if (o->method != IFILT_METHOD_PLAIN && o->method != IFILT_METHOD_BATCHED) fail(IFILT_EINVAL, "unknown method");
  if (o->n2_solver < IFILT_N2_AUTO || o->n2_solver > IFILT_N2_COMPLEX) fail(IFILT_EINVAL, "unknown n2_solver");
  if (o->order >= 3 && o->n2_solver == IFILT_N2_COMPLEX)
    fail(IFILT_EINVAL, "the complex factorisation serves order 2 only; orders >= 3 run in real arithmetic");
  if (o->method == IFILT_METHOD_PLAIN && o->precision != IFILT_PREC_FP64)
    fail(IFILT_EINVAL, "the plain method runs in FP64 only");
  if (o->precond < IFILT_PRECOND_NONE || o->precond > IFILT_PRECOND_MG)
    fail(IFILT_EINVAL, "unknown precond %d", o->precond);
  if (o->precond == IFILT_PRECOND_MG) {
    if (o->precision == IFILT_PREC_FP64) fail(IFILT_EINVAL, "multigrid preconditioning runs with FP32 or BF16 precision");
    if (!(o->order == 1 || complex_form(*o)))
      fail(IFILT_EINVAL, "multigrid preconditioning needs order 1 or the complex n = 2 form");
  }
  if (o->method == IFILT_METHOD_PLAIN && o->precond != IFILT_PRECOND_NONE)
    fail(IFILT_EINVAL, "the plain method takes no preconditioner");
  if (o->max_iter < 0 || o->check_every < 0 || o->max_lanes < 0 || o->inner_tol < 0)
    fail(IFILT_EINVAL, "negative option");
  if (!(o->err_tol >= 0.0) || !std::isfinite(o->err_tol)) fail(IFILT_EINVAL, "err_tol must be >= 0 and finite");
  if (o->mg_cycle != IFILT_MG_V && o->mg_cycle != IFILT_MG_W12) fail(IFILT_EINVAL, "unknown mg_cycle %d", o->mg_cycle);
  if (o->method == IFILT_METHOD_PLAIN && o->err_tol > 0.0)
    fail(IFILT_EINVAL, "the plain method stops on the residual only (err_tol = 0)");
}

ifilt_status ifilt_solve(ifilt_mesh m, const ifilt_solve_opts* o, int32_t n_fields, const double* fields, int32_t n_k,
                         const double* k, double* out, ifilt_col_stats* stats, void* stream) {
  ApiRange range_("ifilt_solve");
  IFILT_GUARD_BEGIN
  check_uploaded(m);
  check_opts(m, o);
  if (n_fields <= 0 || n_k <= 0) fail(IFILT_EINVAL, "n_fields and n_k must be positive");
  if (!fields || !k || !out) fail(IFILT_EINVAL, "null fields, k or out");
  for (int32_t j = 0; j < n_k; j++)
    if (!(k[j] > 0.0) || !std::isfinite(k[j])) fail(IFILT_EINVAL, "k[%d] must be positive and finite", j);
  DeviceScope ds(m->device);
  cudaStream_t st = (cudaStream_t)stream;
  ifilt_status s;
  if (o->method == IFILT_METHOD_PLAIN) s = solve_plain(m, *o, n_fields, fields, n_k, k, out, stats, st);
  else s = solve_batched(m, *o, n_fields, fields, n_k, k, out, stats, st);
  IFILT_CUDA(cudaStreamSynchronize(st));
  IFILT_CUDA(cudaGetLastError());
  if (s == IFILT_NOT_CONVERGED) set_last_error("some columns did not reach the tolerance");
  return s;
  IFILT_GUARD_END
}

ifilt_status ifilt_solve_many(int32_t n_items, const ifilt_solve_item* items, void* stream) {
  ApiRange range_("ifilt_solve_many");
  IFILT_GUARD_BEGIN
  if (n_items <= 0 || !items) fail(IFILT_EINVAL, "need at least one item");
  int dev = -1;
  for (int32_t i = 0; i < n_items; i++) {
    const ifilt_solve_item& it = items[i];
    check_uploaded(it.mesh);
    ifilt_solve_opts o = it.opts;
    o.method = IFILT_METHOD_BATCHED;
    check_opts(it.mesh, &o);
    if (it.n_fields <= 0 || it.n_k <= 0) fail(IFILT_EINVAL, "item %d: n_fields and n_k must be positive", i);
    if (!it.fields || !it.k || !it.out) fail(IFILT_EINVAL, "item %d: null fields, k or out", i);
    for (int32_t j = 0; j < it.n_k; j++)
      if (!(it.k[j] > 0.0) || !std::isfinite(it.k[j])) fail(IFILT_EINVAL, "item %d: k must be positive", i);
    if (dev >= 0 && it.mesh->device != dev) fail(IFILT_EINVAL, "all items must live on one device");
    dev = it.mesh->device;
  }
  DeviceScope ds(dev);
  cudaStream_t st = (cudaStream_t)stream;
  ifilt_status s = solve_many(n_items, items, st);
  IFILT_CUDA(cudaStreamSynchronize(st));
  IFILT_CUDA(cudaGetLastError());
  if (s == IFILT_NOT_CONVERGED) set_last_error("some columns did not reach the tolerance");
  return s;
  IFILT_GUARD_END
}

size_t ifilt_solve_scratch_bytes(ifilt_mesh m, const ifilt_solve_opts* o, int32_t n_fields, int32_t n_k) {
  if (!m || !o || n_fields <= 0 || n_k <= 0) return 0;
  if (o->order < 1 || o->order > m->host.max_order) return 0;
  if (o->method == IFILT_METHOD_PLAIN && m->device < 0) return 0;
  try {
    if (o->method == IFILT_METHOD_PLAIN) return plain_scratch_bytes(m, *o);
    return batched_scratch_bytes(m, *o, n_fields, n_k);
  } catch (...) {
    return 0;
  }
}

ifilt_status ifilt_spectrum(ifilt_mesh m, int32_t n_fields, int32_t n_k, const double* k, const double* filtered,
                            double* energy, double* spec, double* kmid, void* stream) {
  ApiRange range_("ifilt_spectrum");
  IFILT_GUARD_BEGIN
  check_uploaded(m);
  if (n_fields <= 0 || n_k <= 0) fail(IFILT_EINVAL, "n_fields and n_k must be positive");
  if (!k || !filtered || !energy) fail(IFILT_EINVAL, "null k, filtered or energy");
  for (int32_t j = 0; j < n_k; j++)
    if (!(k[j] > 0.0) || !std::isfinite(k[j]) || (j > 0 && !(k[j] > k[j - 1])))
      fail(IFILT_EINVAL, "k must be positive, finite and strictly ascending");
  DeviceScope ds(m->device);
  cudaStream_t st = (cudaStream_t)stream;
  const int nb = 256;
  const size_t F = (size_t)n_fields, K = (size_t)n_k;
  size_t bytes = (K + F * K + F * K + K + F * K * nb) * sizeof(double) + 1024;
  double* buf = (double*)scratch_alloc(bytes, st);
  double* k_dev = buf;
  double* e_dev = k_dev + K;
  double* s_dev = e_dev + F * K;
  double* km_dev = s_dev + F * K;
  double* part = km_dev + K;
  IFILT_CUDA(cudaMemcpyAsync(k_dev, k, K * sizeof(double), cudaMemcpyHostToDevice, st));
  spectrum_device(m, n_fields, n_k, k_dev, filtered, e_dev, s_dev, km_dev, part, nb, st);
  profile_count(2);
  IFILT_CUDA(cudaMemcpyAsync(energy, e_dev, F * K * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (spec && K > 1) IFILT_CUDA(cudaMemcpyAsync(spec, s_dev, F * (K - 1) * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (kmid && K > 1) IFILT_CUDA(cudaMemcpyAsync(kmid, km_dev, (K - 1) * sizeof(double), cudaMemcpyDeviceToHost, st));
  scratch_free(buf, st);
  IFILT_CUDA(cudaStreamSynchronize(st));
  return IFILT_OK;
  IFILT_GUARD_END
}

ifilt_status ifilt_spectrum_noalloc(ifilt_mesh m, int32_t n_fields, int32_t n_k, const double* k,
                                    const double* filtered, double* energy, double* spec, double* kmid,
                                    void* stream) {
  IFILT_GUARD_BEGIN
  check_uploaded(m);
  if (n_fields <= 0 || n_k <= 0) fail(IFILT_EINVAL, "n_fields and n_k must be positive");
  if (!k || !filtered || !energy) fail(IFILT_EINVAL, "null k, filtered or energy");
  for (int32_t j = 0; j < n_k; j++)
    if (!(k[j] > 0.0) || !std::isfinite(k[j]) || (j > 0 && !(k[j] > k[j - 1])))
      fail(IFILT_EINVAL, "k must be positive, finite and strictly ascending");
  DeviceScope ds(m->device);
  return spectrum_noalloc(m, n_fields, n_k, k, filtered, energy, spec, kmid, (cudaStream_t)stream);
  IFILT_GUARD_END
}

void ifilt_profile_enable(int32_t on) { g_prof.store(on != 0); }

void ifilt_profile_reset(void) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof_recs.clear();
}

int32_t ifilt_profile_read(ifilt_kernel_profile* out, int32_t max) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  int32_t i = 0;
  for (auto& kv : g_prof_recs) {
    if (out && i < max) {
      ifilt_kernel_profile& r = out[i];
      std::memset(&r, 0, sizeof r);
      std::strncpy(r.name, kv.first.c_str(), sizeof r.name - 1);
      r.launches = kv.second.launches;
      r.samples = kv.second.samples;
      r.sampled_ms = kv.second.ms;
      r.bytes_per_launch = kv.second.samples ? kv.second.bytes_sum / kv.second.samples : 0.0;
    }
    i++;
  }
  return i;
}

}  // extern "C"
