// Upload of the prepared mesh arrays to the device (end of the preparation
// phase, Sect. 2.2.1): the operators are packed once into the layouts the
// solve kernels read and stay resident until the handle is released.
#include <algorithm>
#include <cstring>

#include "internal.h"
#include "multigrid.h"

namespace ifilt {
namespace {

template <typename T>
T* dev_copy(ifilt_mesh_s* m, const T* src, size_t count, cudaStream_t st) {
  if (count == 0) return nullptr;
  void* p = nullptr;
  IFILT_CUDA(cudaMalloc(&p, count * sizeof(T)));
  m->allocations.push_back(p);
  m->bytes += (int64_t)(count * sizeof(T));
  IFILT_CUDA(cudaMemcpyAsync(p, src, count * sizeof(T), cudaMemcpyHostToDevice, st));
  // keep host staging alive until the copy is done
  IFILT_CUDA(cudaStreamSynchronize(st));
  return static_cast<T*>(p);
}

// Sliced ELL from CSR; padding entries point at their own row with value 0.
// Every slice starts on an 8-entry boundary (so any run of slices can be
// bulk-copied with 16-byte aligned addresses and sizes for every value type).
// `ncols` >= 0 marks a rectangular matrix: its padding entries repeat the
// row's last column (0 for an empty row) so that they stay inside the source.
void build_ell(ifilt_mesh_s* m, const HostCSR& a, int32_t slice_h, DevEll& out, cudaStream_t st,
               int32_t ncols = -1) {
  const int32_t n = a.n, nv = a.nval;
  const int32_t ns = (n + slice_h - 1) / slice_h;
  std::vector<int64_t> off((size_t)ns + 1, 0);
  std::vector<int32_t> width(ns, 0);
  int32_t maxw = 0;
  for (int32_t s = 0; s < ns; s++) {
    int64_t w = 0;
    int32_t r1 = std::min(n, (s + 1) * slice_h);
    for (int32_t r = s * slice_h; r < r1; r++) w = std::max<int64_t>(w, a.row_ptr[r + 1] - a.row_ptr[r]);
    w = (w + 3) / 4 * 4;
    width[s] = (int32_t)w;
    maxw = std::max(maxw, (int32_t)w);
    off[s + 1] = (off[s] + (int64_t)(r1 - s * slice_h) * w + 7) / 8 * 8;
  }
  const int64_t E = off[ns];
  std::vector<int32_t> col((size_t)E);
  std::vector<double> v64((size_t)E * nv, 0.0);
  for (int32_t s = 0; s < ns; s++) {
    int32_t r1 = std::min(n, (s + 1) * slice_h);
    for (int32_t r = s * slice_h; r < r1; r++) {
      int64_t base = off[s] + (int64_t)(r - s * slice_h) * width[s];
      int64_t len = a.row_ptr[r + 1] - a.row_ptr[r];
      for (int64_t e = 0; e < width[s]; e++) {
        if (e < len) {
          col[base + e] = a.col[a.row_ptr[r] + e];
          for (int q = 0; q < nv; q++) v64[(size_t)(base + e) * nv + q] = a.val[(size_t)(a.row_ptr[r] + e) * nv + q];
        } else if (ncols < 0) {
          col[base + e] = r;
        } else {
          col[base + e] = len > 0 ? a.col[a.row_ptr[r] + len - 1] : 0;
        }
      }
    }
  }
  // every index the gather kernels will follow stays inside the source vector
  const int32_t limit = ncols < 0 ? n : ncols;
  for (int64_t e = 0; e < E; e++)
    if (col[e] < 0 || col[e] >= limit) fail(IFILT_EINVAL, "internal: ELL column %d outside 0..%d", col[e], limit - 1);
  std::vector<float> v32(v64.size()), v32lo(v64.size());
  std::vector<__nv_bfloat16> v16(v64.size());
  for (size_t i = 0; i < v64.size(); i++) {
    v32[i] = (float)v64[i];
    v32lo[i] = (float)(v64[i] - (double)v32[i]);
    v16[i] = __float2bfloat16_rn((float)v64[i]);
  }
  out.n = n;
  out.slice_h = slice_h;
  out.n_slices = ns;
  out.nval = nv;
  out.max_width = maxw;
  out.entries = E;
  out.slice_off = dev_copy(m, off.data(), off.size(), st);
  out.slice_w = dev_copy(m, width.data(), width.size(), st);
  out.col = dev_copy(m, col.data(), col.size(), st);
  out.val64 = dev_copy(m, v64.data(), v64.size(), st);
  out.val32 = dev_copy(m, v32.data(), v32.size(), st);
  out.val32lo = dev_copy(m, v32lo.data(), v32lo.size(), st);
  out.val16 = dev_copy(m, v16.data(), v16.size(), st);
}

// Real FP64 CSR; block matrices are expanded to interleaved rows (u_i at 2i, v_i at 2i+1):
// block (a, b) at (i, j) gives u_i: a u_j + b v_j and v_i: -b u_j + a v_j.
void build_csr(ifilt_mesh_s* m, const HostCSR& a, DevCSR& out, cudaStream_t st) {
  if (a.row_ptr.size() != (size_t)a.n + 1 || a.row_ptr[0] != 0 || a.row_ptr[a.n] != (int64_t)a.col.size())
    fail(IFILT_EINVAL, "internal: inconsistent CSR row pointers");
  for (int32_t c : a.col)
    if (c < 0 || c >= a.n) fail(IFILT_EINVAL, "internal: CSR column %d outside 0..%d", c, a.n - 1);
  if (a.nval == 1) {
    out.n = a.n;
    out.nnz = a.nnz();
    out.row_ptr = dev_copy(m, a.row_ptr.data(), a.row_ptr.size(), st);
    out.col = dev_copy(m, a.col.data(), a.col.size(), st);
    out.val = dev_copy(m, a.val.data(), a.val.size(), st);
    return;
  }
  const int32_t n = a.n;
  std::vector<int64_t> rp((size_t)2 * n + 1, 0);
  for (int32_t i = 0; i < n; i++) {
    int64_t len = 2 * (a.row_ptr[i + 1] - a.row_ptr[i]);
    rp[2 * i + 1] = rp[2 * i] + len;
    rp[2 * i + 2] = rp[2 * i + 1] + len;
  }
  std::vector<int32_t> col((size_t)rp.back());
  std::vector<double> val((size_t)rp.back());
  for (int32_t i = 0; i < n; i++) {
    int64_t ou = rp[2 * i], ov = rp[2 * i + 1];
    for (int64_t e = a.row_ptr[i]; e < a.row_ptr[i + 1]; e++) {
      int32_t j = a.col[e];
      double av = a.val[2 * e], bv = a.val[2 * e + 1];
      col[ou] = 2 * j;
      val[ou++] = av;
      col[ou] = 2 * j + 1;
      val[ou++] = bv;
      col[ov] = 2 * j;
      val[ov++] = -bv;
      col[ov] = 2 * j + 1;
      val[ov++] = av;
    }
  }
  out.n = 2 * n;
  out.nnz = rp.back();
  out.row_ptr = dev_copy(m, rp.data(), rp.size(), st);
  out.col = dev_copy(m, col.data(), col.size(), st);
  out.val = dev_copy(m, val.data(), val.size(), st);
}

std::vector<double> diagonal(const HostCSR& a) {
  std::vector<double> d(a.n, 0.0);
  for (int32_t r = 0; r < a.n; r++)
    for (int64_t e = a.row_ptr[r]; e < a.row_ptr[r + 1]; e++)
      if (a.col[e] == r) d[r] = a.val[(size_t)e * a.nval];
  return d;
}

}  // namespace

void upload_mesh(ifilt_mesh_s* m, int32_t slice_h, cudaStream_t st) {
  const HostPrepared& h = m->host;
  if (slice_h <= 0) slice_h = 64;
  if (slice_h < 4 || slice_h > 1024) fail(IFILT_EINVAL, "ell_slice must be between 4 and 1024 rows");
  PhaseClock clock("upload");
  m->perm = dev_copy(m, h.perm.data(), h.perm.size(), st);
  m->mass = dev_copy(m, h.mass.data(), h.mass.size(), st);
  std::vector<float> m32(h.mass.begin(), h.mass.end()), m32lo(h.mass.size());
  for (size_t i = 0; i < m32.size(); i++) m32lo[i] = (float)(h.mass[i] - (double)m32[i]);
  m->mass32 = dev_copy(m, m32.data(), m32.size(), st);
  m->mass32lo = dev_copy(m, m32lo.data(), m32lo.size(), st);
  std::vector<double> dk = diagonal(h.K);
  m->diag_k = dev_copy(m, dk.data(), dk.size(), st);
  std::vector<float> dk32(dk.begin(), dk.end());
  m->diag_k32 = dev_copy(m, dk32.data(), dk32.size(), st);
  build_ell(m, h.K, slice_h, m->ell_k, st);
  build_csr(m, h.K, m->csr_k, st);
  clock.lap("K");
  if (h.max_order >= 2) {
    std::vector<double> dg = diagonal(h.G2);
    m->diag_g2 = dev_copy(m, dg.data(), dg.size(), st);
    std::vector<float> dg32(dg.begin(), dg.end());
    m->diag_g2_32 = dev_copy(m, dg32.data(), dg32.size(), st);
    build_ell(m, h.G2, slice_h, m->ell_g2, st);
    build_csr(m, h.G2, m->csr_g2, st);
  }
  clock.lap("G2");
  m->ell_gn.assign(h.Gn.size(), DevEll{});
  m->csr_gn.assign(h.Gn.size(), DevCSR{});
  m->diag_gn.assign(h.Gn.size(), nullptr);
  m->diag_gn32.assign(h.Gn.size(), nullptr);
  for (size_t i = 0; i < h.Gn.size(); i++) {
    std::vector<double> dg = diagonal(h.Gn[i]);
    m->diag_gn[i] = dev_copy(m, dg.data(), dg.size(), st);
    std::vector<float> dg32(dg.begin(), dg.end());
    m->diag_gn32[i] = dev_copy(m, dg32.data(), dg32.size(), st);
    build_ell(m, h.Gn[i], slice_h, m->ell_gn[i], st);
    build_csr(m, h.Gn[i], m->csr_gn[i], st);
  }
  if (h.placement == IFILT_VERTEX_VECTOR) {
    m->proj_ptr = dev_copy(m, h.proj_ptr.data(), h.proj_ptr.size(), st);
    m->proj_cell = dev_copy(m, h.proj_cell.data(), h.proj_cell.size(), st);
    m->proj_w = dev_copy(m, h.proj_w.data(), h.proj_w.size(), st);
  }
  // weight of each output entry for the energy sums (0 where not an unknown)
  std::vector<double> w((size_t)h.n_out, 0.0);
  for (int32_t r = 0; r < h.n_rows; r++) w[h.perm[r]] = h.mass[r];
  m->w_out = dev_copy(m, w.data(), w.size(), st);
  std::vector<int32_t> ip((size_t)h.n_out, -1);
  for (int32_t r = 0; r < h.n_rows; r++) ip[h.perm[r]] = r;
  m->inv_perm = dev_copy(m, ip.data(), ip.size(), st);
}

const MgHost& multigrid_host(ifilt_mesh_s* m) {
  std::lock_guard<std::mutex> lk(m->mg_mu);
  if (!m->mg_host) {
    MgParams prm;
    prm.strength = m->host.mg_strength;
    m->mg_host = std::make_shared<MgHost>(build_multigrid(m->host, prm));
  }
  return *m->mg_host;
}

const std::vector<DevMgLevel>& multigrid_device(ifilt_mesh_s* m, cudaStream_t st) {
  const MgHost& h = multigrid_host(m);
  std::lock_guard<std::mutex> lk(m->mg_mu);
  if (!m->mg_dev.empty()) return m->mg_dev;
  if (m->device < 0) fail(IFILT_EINVAL, "mesh is not uploaded");
  // coarse levels are small and their rows wide: short slices keep a stage small
  constexpr int32_t kMgSlice = 16;
  std::vector<DevMgLevel> dev(h.levels.size());
  for (size_t l = 0; l < h.levels.size(); l++) {
    const MgHostLevel& L = h.levels[l];
    DevMgLevel& D = dev[l];
    D.n = L.n;
    D.omega = L.omega_s;
    if (l > 0) build_ell(m, L.S, kMgSlice, D.S, st);
    if (l + 1 < h.levels.size()) {
      build_ell(m, L.P, kMgSlice, D.P, st, h.levels[l + 1].n);
      build_ell(m, L.R, kMgSlice, D.R, st, L.n);
    }
    std::vector<float> dk(L.dk.begin(), L.dk.end()), dm(L.dm.begin(), L.dm.end());
    D.dk32 = dev_copy(m, dk.data(), dk.size(), st);
    D.dm32 = dev_copy(m, dm.data(), dm.size(), st);
  }
  m->mg_dev = std::move(dev);
  return m->mg_dev;
}

void free_mesh(ifilt_mesh_s* m) {
  cudaDeviceSynchronize();
  for (void* p : m->allocations) cudaFree(p);
  m->allocations.clear();
}

}  // namespace ifilt
