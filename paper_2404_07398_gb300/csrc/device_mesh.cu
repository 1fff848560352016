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

// A CSR's arrays on the device: row pointers, columns, nval values per entry.
struct RawCSR {
  int32_t n = 0, nval = 1;
  int64_t nnz = 0;
  int64_t* rp = nullptr;
  int32_t* col = nullptr;
  double* val = nullptr;
};

// Upload a host CSR as it is (one copy of each array), after checking its row
// pointers and that every column lies in 0 .. ncols-1.  `keep`: the arrays
// belong to the mesh (they serve as its FP64 CSR); otherwise the caller frees
// them with free_raw.
RawCSR upload_csr(ifilt_mesh_s* m, const HostCSR& a, int32_t ncols, bool keep, cudaStream_t st) {
  if (a.row_ptr.size() != (size_t)a.n + 1 || a.row_ptr[0] != 0 || a.row_ptr[a.n] != (int64_t)a.col.size() ||
      a.val.size() != a.col.size() * (size_t)a.nval)
    fail(IFILT_EINVAL, "internal: inconsistent CSR arrays");
  for (int32_t c : a.col)
    if (c < 0 || c >= ncols) fail(IFILT_EINVAL, "internal: CSR column %d outside 0..%d", c, ncols - 1);
  RawCSR r;
  r.n = a.n;
  r.nval = a.nval;
  r.nnz = a.nnz();
  if (keep) {
    r.rp = dev_copy(m, a.row_ptr.data(), a.row_ptr.size(), st);
    r.col = dev_copy(m, a.col.data(), a.col.size(), st);
    r.val = dev_copy(m, a.val.data(), a.val.size(), st);
  } else {
    auto tmp = [&](const void* src, size_t bytes) {
      void* p = nullptr;
      if (bytes == 0) return p;
      IFILT_CUDA(cudaMalloc(&p, bytes));
      IFILT_CUDA(cudaMemcpyAsync(p, src, bytes, cudaMemcpyHostToDevice, st));
      return p;
    };
    r.rp = (int64_t*)tmp(a.row_ptr.data(), a.row_ptr.size() * sizeof(int64_t));
    r.col = (int32_t*)tmp(a.col.data(), a.col.size() * sizeof(int32_t));
    r.val = (double*)tmp(a.val.data(), a.val.size() * sizeof(double));
    IFILT_CUDA(cudaStreamSynchronize(st));  // the host arrays may go once this returns
  }
  return r;
}
void free_raw(RawCSR& r) {
  cudaFree(r.rp);
  cudaFree(r.col);
  cudaFree(r.val);
  r = RawCSR{};
}

// width of every slice: its longest row, rounded up to a multiple of 4 entries
__global__ void ell_width_kernel(int32_t n, int32_t slice_h, int32_t ns, const int64_t* __restrict__ rp,
                                 int32_t* __restrict__ width) {
  for (int32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < ns; s += gridDim.x * blockDim.x) {
    const int32_t r1 = min(n, (s + 1) * slice_h);
    int64_t w = 0;
    for (int32_t r = s * slice_h; r < r1; r++) w = max(w, rp[r + 1] - rp[r]);
    width[s] = (int32_t)((w + 3) / 4 * 4);
  }
}

// One row of the sliced ELL per thread: its entries, then padding that points at
// the row itself with value 0 (square operators) or repeats the row's last
// column (rectangular ones, ncols >= 0: 0 for an empty row), with the FP64
// values' FP32, FP32-remainder and BF16 copies, and the row's length in fours
// (entries rounded up to 4; 255 for rows longer than 1020 entries, which then
// run to the slice's width).  A column outside the source vector raises *bad.
__global__ void ell_fill_kernel(int32_t n, int32_t slice_h, int nv, int32_t ncols, const int64_t* __restrict__ rp,
                                const int32_t* __restrict__ col, const double* __restrict__ val,
                                const int64_t* __restrict__ off, const int32_t* __restrict__ width,
                                int32_t* __restrict__ ecol, double* __restrict__ v64, float* __restrict__ v32,
                                float* __restrict__ v32lo, __nv_bfloat16* __restrict__ v16,
                                uint8_t* __restrict__ rowq, int* __restrict__ bad) {
  const int32_t limit = ncols < 0 ? n : ncols;
  for (int32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    const int32_t s = r / slice_h;
    const int32_t w = width[s];
    const int64_t base = off[s] + (int64_t)(r - s * slice_h) * w;
    const int64_t b0 = rp[r], len = rp[r + 1] - b0;
    rowq[r] = len > 4 * 254 ? (uint8_t)255 : (uint8_t)((len + 3) / 4);
    for (int64_t e = 0; e < w; e++) {
      int32_t c;
      if (e < len) c = col[b0 + e];
      else if (ncols < 0) c = r;
      else c = len > 0 ? col[b0 + len - 1] : 0;
      if (c < 0 || c >= limit) atomicExch(bad, 1);
      ecol[base + e] = c;
      for (int q = 0; q < nv; q++) {
        const double v = e < len ? val[(b0 + e) * nv + q] : 0.0;
        const float f = __double2float_rn(v);
        const int64_t i = (base + e) * nv + q;
        v64[i] = v;
        v32[i] = f;
        v32lo[i] = __double2float_rn(__dsub_rn(v, (double)f));
        v16[i] = __float2bfloat16_rn(f);
      }
    }
  }
}

template <typename T>
T* dev_alloc(ifilt_mesh_s* m, size_t count, cudaStream_t st) {
  if (count == 0) return nullptr;
  void* p = nullptr;
  IFILT_CUDA(cudaMalloc(&p, count * sizeof(T)));
  m->allocations.push_back(p);
  m->bytes += (int64_t)(count * sizeof(T));
  IFILT_CUDA(cudaMemsetAsync(p, 0, count * sizeof(T), st));
  return static_cast<T*>(p);
}

// Sliced ELL packed on the device from a device CSR: the same layout as a host
// packing would give (slices of slice_h rows, widths a multiple of 4, every
// slice starting on an 8-entry boundary so that any run of slices can be
// bulk-copied with 16-byte aligned addresses and sizes for every value type;
// the gap before a slice start holds column 0 and value 0).  `ncols` >= 0 marks
// a rectangular matrix (see ell_fill_kernel).
void pack_ell(ifilt_mesh_s* m, const RawCSR& a, int32_t slice_h, DevEll& out, cudaStream_t st,
              int32_t ncols = -1) {
  const int32_t n = a.n, nv = a.nval;
  const int32_t ns = (n + slice_h - 1) / slice_h;
  std::vector<int32_t> width(ns, 0);
  int32_t* dwidth = dev_alloc<int32_t>(m, (size_t)ns, st);
  const int block = 256;
  if (ns > 0) {
    const int g = (int)std::min<int64_t>((ns + block - 1) / block, 152LL * 16);
    ell_width_kernel<<<g, block, 0, st>>>(n, slice_h, ns, a.rp, dwidth);
    IFILT_CUDA(cudaGetLastError());
    IFILT_CUDA(cudaMemcpyAsync(width.data(), dwidth, (size_t)ns * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    IFILT_CUDA(cudaStreamSynchronize(st));
  }
  std::vector<int64_t> off((size_t)ns + 1, 0);
  int32_t maxw = 0;
  for (int32_t s = 0; s < ns; s++) {
    const int32_t rows = std::min(n, (s + 1) * slice_h) - s * slice_h;
    maxw = std::max(maxw, width[s]);
    off[s + 1] = (off[s] + (int64_t)rows * width[s] + 7) / 8 * 8;
  }
  const int64_t E = off[ns];
  out.n = n;
  out.slice_h = slice_h;
  out.n_slices = ns;
  out.nval = nv;
  out.max_width = maxw;
  out.entries = E;
  out.slice_w = dwidth;
  out.slice_off = dev_copy(m, off.data(), off.size(), st);
  out.col = dev_alloc<int32_t>(m, (size_t)E, st);
  out.val64 = dev_alloc<double>(m, (size_t)E * nv, st);
  out.val32 = dev_alloc<float>(m, (size_t)E * nv, st);
  out.val32lo = dev_alloc<float>(m, (size_t)E * nv, st);
  out.val16 = dev_alloc<__nv_bfloat16>(m, (size_t)E * nv, st);
  out.rowq = dev_alloc<uint8_t>(m, (size_t)ns * slice_h, st);  // whole slices: bulk-copied per tile
  int* bad = nullptr;
  IFILT_CUDA(cudaMalloc(&bad, sizeof(int)));
  IFILT_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), st));
  if (n > 0) {
    const int g = (int)std::min<int64_t>(((int64_t)n + block - 1) / block, 152LL * 32);
    ell_fill_kernel<<<g, block, 0, st>>>(n, slice_h, nv, ncols, a.rp, a.col, a.val, out.slice_off, dwidth, out.col,
                                         out.val64, out.val32, out.val32lo, out.val16, out.rowq, bad);
    IFILT_CUDA(cudaGetLastError());
  }
  int hbad = 0;
  IFILT_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
  IFILT_CUDA(cudaStreamSynchronize(st));
  cudaFree(bad);
  if (hbad) fail(IFILT_EINVAL, "internal: ELL column outside its source vector");
}

// block rows [[a, b], [-b, a]] as interleaved real rows (u_i at 2i, v_i at 2i+1):
// block (a, b) at (i, j) gives u_i: a u_j + b v_j and v_i: -b u_j + a v_j
__global__ void expand_blocks_kernel(int32_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                     const double* __restrict__ val, int64_t* __restrict__ rp2,
                                     int32_t* __restrict__ col2, double* __restrict__ val2) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int64_t b0 = rp[i], len = rp[i + 1] - b0;
    int64_t ou = 4 * b0, ov = 4 * b0 + 2 * len;
    rp2[2 * i] = ou;
    rp2[2 * i + 1] = ov;
    if (i + 1 == n) rp2[2 * n] = 4 * rp[n];
    for (int64_t e = b0; e < b0 + len; e++) {
      const int32_t j = col[e];
      const double av = val[2 * e], bv = val[2 * e + 1];
      col2[ou] = 2 * j;
      val2[ou++] = av;
      col2[ou] = 2 * j + 1;
      val2[ou++] = bv;
      col2[ov] = 2 * j;
      val2[ov++] = -bv;
      col2[ov] = 2 * j + 1;
      val2[ov++] = av;
    }
  }
}

// Real FP64 CSR of the plain path from a device CSR: shared as it is for scalar
// entries, expanded to interleaved real rows on the device for 2x2 blocks.
void csr_from_raw(ifilt_mesh_s* m, const RawCSR& a, DevCSR& out, cudaStream_t st) {
  if (a.nval == 1) {
    out.n = a.n;
    out.nnz = a.nnz;
    out.row_ptr = a.rp;
    out.col = a.col;
    out.val = a.val;
    return;
  }
  out.n = 2 * a.n;
  out.nnz = 4 * a.nnz;
  out.row_ptr = dev_alloc<int64_t>(m, (size_t)2 * a.n + 1, st);
  out.col = dev_alloc<int32_t>(m, (size_t)out.nnz, st);
  out.val = dev_alloc<double>(m, (size_t)out.nnz, st);
  if (a.n > 0) {
    const int block = 256;
    const int g = (int)std::min<int64_t>(((int64_t)a.n + block - 1) / block, 152LL * 32);
    expand_blocks_kernel<<<g, block, 0, st>>>(a.n, a.rp, a.col, a.val, out.row_ptr, out.col, out.val);
    IFILT_CUDA(cudaGetLastError());
  }
  IFILT_CUDA(cudaStreamSynchronize(st));
}

// Sliced ELL and FP64 CSR of a square operator: the CSR is uploaded once and
// both layouts are built from it on the device.
void build_operator(ifilt_mesh_s* m, const HostCSR& a, int32_t slice_h, DevEll& ell, DevCSR& csr, cudaStream_t st) {
  RawCSR raw = upload_csr(m, a, a.n, a.nval == 1, st);
  pack_ell(m, raw, slice_h, ell, st);
  csr_from_raw(m, raw, csr, st);
  if (a.nval != 1) free_raw(raw);
}

// Sliced ELL alone (multigrid operators), packed on the device
void build_ell(ifilt_mesh_s* m, const HostCSR& a, int32_t slice_h, DevEll& out, cudaStream_t st,
               int32_t ncols = -1) {
  RawCSR raw = upload_csr(m, a, ncols < 0 ? a.n : ncols, false, st);
  pack_ell(m, raw, slice_h, out, st, ncols);
  free_raw(raw);
}

// G = A M^-1 K with the structural product pattern, on the device (Sect. 2.1.1:
// K M^-1 K for n = 2, G_(n-1) M^-1 K for the higher orders).  Row i collects
// the candidate products (entry e of row i of A, entry f of row A.col[e] of K)
// in that order, sorts them stably by column and sums each column's run in
// that order: the same products, summed in the same order and with the same
// IEEE operations (no fused multiply-adds) as the host product, so both give
// the same bits.  One row per thread; a row with more than MAXC candidates
// raises *overflow (the caller then takes the host product).  Count pass
// (grp == nullptr): distinct columns per row into cnt.
template <int MAXC>
__global__ void product_kernel(int32_t n, int nv, const int64_t* __restrict__ arp, const int32_t* __restrict__ acol,
                               const double* __restrict__ aval, const int64_t* __restrict__ krp,
                               const int32_t* __restrict__ kcol, const double* __restrict__ kval,
                               const double* __restrict__ mass, const int64_t* __restrict__ grp,
                               int32_t* __restrict__ cnt, int32_t* __restrict__ gcol, double* __restrict__ gval,
                               int* __restrict__ overflow) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int32_t key[MAXC];
    uint16_t qa[MAXC], qk[MAXC];  // entry offsets inside row i of A and row j of K
    int m = 0;
    const int64_t a0 = arp[i], a1 = arp[i + 1];
    for (int64_t q = a0; q < a1; q++) {
      const int32_t j = acol[q];
      for (int64_t f = krp[j]; f < krp[j + 1]; f++) {
        if (m < MAXC) {
          key[m] = kcol[f];
          qa[m] = (uint16_t)(q - a0);
          qk[m] = (uint16_t)(f - krp[j]);
        }
        m++;
      }
    }
    if (m > MAXC || a1 - a0 > 65535) {
      atomicExch(overflow, 1);
      if (!grp) cnt[i] = 0;
      continue;
    }
    for (int t = 1; t < m; t++) {  // stable insertion sort by column
      const int32_t k = key[t];
      const uint16_t x = qa[t], y = qk[t];
      int u = t - 1;
      while (u >= 0 && key[u] > k) {
        key[u + 1] = key[u];
        qa[u + 1] = qa[u];
        qk[u + 1] = qk[u];
        u--;
      }
      key[u + 1] = k;
      qa[u + 1] = x;
      qk[u + 1] = y;
    }
    if (!grp) {
      int d = 0;
      for (int t = 0; t < m; t++) d += (t == 0 || key[t] != key[t - 1]) ? 1 : 0;
      cnt[i] = d;
      continue;
    }
    int64_t o = grp[i];
    for (int t = 0; t < m; o++) {
      const int32_t c = key[t];
      double s0 = 0.0, s1 = 0.0;
      for (; t < m && key[t] == c; t++) {
        const int64_t ee = a0 + qa[t];
        const int32_t j = acol[ee];
        const int64_t ff = krp[j] + qk[t];
        const double inv = __ddiv_rn(1.0, mass[j]);
        if (nv == 1) {
          s0 = __dadd_rn(s0, __dmul_rn(__dmul_rn(aval[ee], inv), kval[ff]));
        } else {  // blocks [[a, b], [-b, a]] multiply like a + i b
          const double x1 = __dmul_rn(aval[2 * ee], inv), y1 = __dmul_rn(aval[2 * ee + 1], inv);
          const double x2 = kval[2 * ff], y2 = kval[2 * ff + 1];
          s0 = __dadd_rn(s0, __dsub_rn(__dmul_rn(x1, x2), __dmul_rn(y1, y2)));
          s1 = __dadd_rn(s1, __dadd_rn(__dmul_rn(x1, y2), __dmul_rn(y1, x2)));
        }
      }
      gcol[o] = c;
      gval[o * nv] = s0;
      if (nv == 2) gval[o * nv + 1] = s1;
    }
  }
}

// The product on the device, as a mesh-owned RawCSR; false (nothing kept) when
// some row has more candidates than the kernel holds.
bool device_product(ifilt_mesh_s* m, const RawCSR& A, const RawCSR& K, const double* mass, RawCSR& G,
                    cudaStream_t st) {
  const int32_t n = A.n;
  const int nv = A.nval;
  const int block = 128;
  const int g = (int)std::max<int64_t>(1, std::min<int64_t>(((int64_t)n + block - 1) / block, 152LL * 64));
  int32_t* cnt = nullptr;
  int* overflow = nullptr;
  IFILT_CUDA(cudaMalloc(&cnt, (size_t)std::max(n, 1) * sizeof(int32_t)));
  IFILT_CUDA(cudaMalloc(&overflow, sizeof(int)));
  IFILT_CUDA(cudaMemsetAsync(overflow, 0, sizeof(int), st));
  // rows of K hold at most ~10 entries on these meshes: K M^-1 K rows take ~100 candidates,
  // the higher orders a few hundred
  const bool wide = A.nnz > 12LL * std::max(n, 1);
  auto launch = [&](const int64_t* grp, int32_t* gcol, double* gval) {
    if (wide)
      product_kernel<512><<<g, block, 0, st>>>(n, nv, A.rp, A.col, A.val, K.rp, K.col, K.val, mass, grp, cnt, gcol,
                                               gval, overflow);
    else
      product_kernel<128><<<g, block, 0, st>>>(n, nv, A.rp, A.col, A.val, K.rp, K.col, K.val, mass, grp, cnt, gcol,
                                               gval, overflow);
    IFILT_CUDA(cudaGetLastError());
  };
  launch(nullptr, nullptr, nullptr);
  std::vector<int32_t> hc((size_t)n);
  int hover = 0;
  IFILT_CUDA(cudaMemcpyAsync(hc.data(), cnt, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  IFILT_CUDA(cudaMemcpyAsync(&hover, overflow, sizeof(int), cudaMemcpyDeviceToHost, st));
  IFILT_CUDA(cudaStreamSynchronize(st));
  bool ok = hover == 0;
  if (ok) {
    std::vector<int64_t> rp((size_t)n + 1, 0);
    for (int32_t i = 0; i < n; i++) rp[i + 1] = rp[i] + hc[i];
    G.n = n;
    G.nval = nv;
    G.nnz = rp[n];
    G.rp = dev_copy(m, rp.data(), rp.size(), st);
    G.col = dev_alloc<int32_t>(m, (size_t)G.nnz, st);
    G.val = dev_alloc<double>(m, (size_t)G.nnz * nv, st);
    launch(G.rp, G.col, G.val);
    IFILT_CUDA(cudaStreamSynchronize(st));
  }
  cudaFree(cnt);
  cudaFree(overflow);
  return ok;
}

// host copy of a device CSR (for saving, exporting and checking)
HostCSR download_csr(const RawCSR& a, cudaStream_t st) {
  HostCSR h;
  h.n = a.n;
  h.nval = a.nval;
  h.row_ptr.resize((size_t)a.n + 1);
  h.col.resize((size_t)a.nnz);
  h.val.resize((size_t)a.nnz * a.nval);
  IFILT_CUDA(cudaMemcpyAsync(h.row_ptr.data(), a.rp, h.row_ptr.size() * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  if (a.nnz > 0) {
    IFILT_CUDA(cudaMemcpyAsync(h.col.data(), a.col, h.col.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    IFILT_CUDA(cudaMemcpyAsync(h.val.data(), a.val, h.val.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  }
  IFILT_CUDA(cudaStreamSynchronize(st));
  return h;
}

std::vector<double> diagonal(const HostCSR& a) {
  std::vector<double> d(a.n, 0.0);
  for (int32_t r = 0; r < a.n; r++)
    for (int64_t e = a.row_ptr[r]; e < a.row_ptr[r + 1]; e++)
      if (a.col[e] == r) d[r] = a.val[(size_t)e * a.nval];
  return d;
}

}  // namespace

// drop a mesh-owned allocation again (a device array only needed while uploading)
void release_owned(ifilt_mesh_s* m, void* p, int64_t bytes) {
  if (!p) return;
  auto it = std::find(m->allocations.begin(), m->allocations.end(), p);
  if (it != m->allocations.end()) {
    m->allocations.erase(it);
    m->bytes -= bytes;
  }
  cudaFree(p);
}

void upload_mesh(ifilt_mesh_s* m, int32_t slice_h, cudaStream_t st) {
  HostPrepared& h = m->host;
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
  // K: uploaded once; its sliced ELL and FP64 CSR are built from it on the device
  RawCSR rawK = upload_csr(m, h.K, h.K.n, h.K.nval == 1, st);
  pack_ell(m, rawK, slice_h, m->ell_k, st);
  csr_from_raw(m, rawK, m->csr_k, st);
  clock.lap("K");
  // G2 and the higher orders: formed on the device when the host left them
  // (the host copy is then read back for saving and exporting)
  std::vector<RawCSR> prods;
  if (h.products_pending) {
    bool ok = true;
    for (int n = 2; n <= h.max_order && ok; n++) {
      RawCSR G;
      ok = device_product(m, n == 2 ? rawK : prods.back(), rawK, m->mass, G, st);
      if (ok) prods.push_back(G);
    }
    if (ok) {
      h.G2 = download_csr(prods[0], st);
      h.Gn.clear();
      for (size_t i = 1; i < prods.size(); i++) h.Gn.push_back(download_csr(prods[i], st));
      h.products_pending = false;
    } else {  // a row wider than the device product holds: the host forms them
      for (RawCSR& G : prods) {
        release_owned(m, G.rp, (int64_t)(G.n + 1) * 8);
        release_owned(m, G.col, G.nnz * 4);
        release_owned(m, G.val, G.nnz * 8 * G.nval);
      }
      prods.clear();
      host_products(h);
    }
    clock.lap("device products");
  }
  auto operator_of = [&](size_t i, const HostCSR& hc, DevEll& ell, DevCSR& csr, double*& dg64, float*& dg32) {
    std::vector<double> dg = diagonal(hc);
    dg64 = dev_copy(m, dg.data(), dg.size(), st);
    std::vector<float> d32(dg.begin(), dg.end());
    dg32 = dev_copy(m, d32.data(), d32.size(), st);
    if (i < prods.size()) {  // from the device product: pack it where it is
      RawCSR& G = prods[i];
      pack_ell(m, G, slice_h, ell, st);
      csr_from_raw(m, G, csr, st);
      if (G.nval != 1) {  // expanded for the plain path: the block form is not kept
        release_owned(m, G.rp, (int64_t)(G.n + 1) * 8);
        release_owned(m, G.col, G.nnz * 4);
        release_owned(m, G.val, G.nnz * 8 * G.nval);
      }
    } else {
      build_operator(m, hc, slice_h, ell, csr, st);
    }
  };
  if (h.max_order >= 2) operator_of(0, h.G2, m->ell_g2, m->csr_g2, m->diag_g2, m->diag_g2_32);
  clock.lap("G2");
  m->ell_gn.assign(h.Gn.size(), DevEll{});
  m->csr_gn.assign(h.Gn.size(), DevCSR{});
  m->diag_gn.assign(h.Gn.size(), nullptr);
  m->diag_gn32.assign(h.Gn.size(), nullptr);
  for (size_t i = 0; i < h.Gn.size(); i++)
    operator_of(i + 1, h.Gn[i], m->ell_gn[i], m->csr_gn[i], m->diag_gn[i], m->diag_gn32[i]);
  if (rawK.nval != 1) free_raw(rawK);
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
