// Mesh cache files (ifilt_mesh_key / ifilt_mesh_save / ifilt_mesh_load_host).
//
// Preparation depends on the mesh only (Sect. 2.2 splits the work into a
// mesh-only phase whose arrays serve every scale and field, and the solves).
// At 10 M vertices it takes tens of seconds on the host (ocean subset, row
// order, operator assembly, K M^-1 K, and the multigrid hierarchy), so its
// result is kept across processes in one file per mesh.
//
// File layout (little-endian, the byte order of both hosts the library is
// built for):
//   "IFILTMC" 0 | u32 format | u32 prepare revision | u64 descriptor key
//   | u64 payload bytes | u64 payload hash | payload
// The payload is a sequence of fields: fixed-size scalars, and arrays as
// (u64 element count, raw elements).  Readers refuse a file whose magic,
// format, revision, length or hash differ, whose key is not the expected one,
// or whose arrays are inconsistent (sizes, row pointers, index ranges): the
// device code indexes with these arrays, so nothing unchecked reaches it.
// Writers write under a temporary name in the same directory and rename, so
// a concurrent reader sees the old file or the new one, never a partial one.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include <unistd.h>

#include "internal.h"
#include "multigrid.h"

namespace ifilt {

namespace {

constexpr char kMagic[8] = {'I', 'F', 'I', 'L', 'T', 'M', 'C', 0};
constexpr uint32_t kFormat = 3;
// Bumped whenever preparation or the multigrid construction changes what it
// produces, so that files written by an older library are prepared again.
constexpr uint32_t kPrepareRevision = 2;

// splitmix64 output function (Steele, Lea and Flood, OOPSLA 2014) as a mixer.
inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}
inline uint64_t rotl(uint64_t x, int r) { return (x << r) | (x >> (64 - r)); }

// A non-cryptographic 64-bit hash over a byte stream, independent of how the
// stream is chunked: four lanes absorb one 8-byte word each per 32-byte block
// (independent multiply chains, several GB/s), the tail is zero-padded, and the
// length is mixed into the digest.  It detects truncation and corruption; it
// is not a defence against a crafted file, which the structural checks are.
class Hash64 {
 public:
  explicit Hash64(uint64_t seed = 0) {
    for (int i = 0; i < 4; i++) acc_[i] = mix64(seed + 0x9e3779b97f4a7c15ULL * (uint64_t)(i + 1));
  }
  void update(const void* data, size_t n) {
    const uint8_t* p = static_cast<const uint8_t*>(data);
    total_ += n;
    if (nbuf_) {
      size_t take = std::min(n, sizeof buf_ - nbuf_);
      std::memcpy(buf_ + nbuf_, p, take);
      nbuf_ += take;
      p += take;
      n -= take;
      if (nbuf_ < sizeof buf_) return;
      block(buf_);
      nbuf_ = 0;
    }
    for (; n >= sizeof buf_; p += sizeof buf_, n -= sizeof buf_) block(p);
    std::memcpy(buf_, p, n);
    nbuf_ = n;
  }
  uint64_t digest() const {
    uint64_t a[4] = {acc_[0], acc_[1], acc_[2], acc_[3]};
    if (nbuf_) {
      uint8_t last[32] = {0};
      std::memcpy(last, buf_, nbuf_);
      absorb(a, last);
    }
    return mix64(a[0] ^ rotl(a[1], 16) ^ rotl(a[2], 32) ^ rotl(a[3], 48) ^ mix64(total_));
  }

 private:
  static void absorb(uint64_t* a, const uint8_t* b) {
    for (int i = 0; i < 4; i++) {
      uint64_t w;
      std::memcpy(&w, b + 8 * i, 8);
      a[i] = mix64(a[i] ^ w);
    }
  }
  void block(const uint8_t* b) { absorb(acc_, b); }
  uint64_t acc_[4];
  uint8_t buf_[32];
  size_t nbuf_ = 0;
  uint64_t total_ = 0;
};

struct File {
  FILE* f = nullptr;
  ~File() {
    if (f) std::fclose(f);
  }
};

class Writer {
 public:
  Writer(FILE* f) : f_(f) {}
  void raw(const void* p, size_t n) {
    if (n && std::fwrite(p, 1, n, f_) != n) fail(IFILT_ECACHE, "cache file write failed");
    h_.update(p, n);
    bytes_ += n;
  }
  template <typename T>
  void scalar(T v) {
    raw(&v, sizeof v);
  }
  template <typename T>
  void vec(const std::vector<T>& v) {
    scalar<uint64_t>(v.size());
    raw(v.data(), v.size() * sizeof(T));
  }
  void csr(const HostCSR& c) {
    scalar<int32_t>(c.n);
    scalar<int32_t>(c.nval);
    vec(c.row_ptr);
    vec(c.col);
    vec(c.val);
  }
  uint64_t bytes() const { return bytes_; }
  uint64_t digest() const { return h_.digest(); }

 private:
  FILE* f_;
  Hash64 h_;
  uint64_t bytes_ = 0;
};

class Reader {
 public:
  Reader(FILE* f, uint64_t payload) : f_(f), left_(payload) {}
  void raw(void* p, size_t n) {
    if (n > left_) fail(IFILT_ECACHE, "cache file is truncated or inconsistent");
    if (n && std::fread(p, 1, n, f_) != n) fail(IFILT_ECACHE, "cache file is truncated");
    h_.update(p, n);
    left_ -= n;
  }
  template <typename T>
  T scalar() {
    T v;
    raw(&v, sizeof v);
    return v;
  }
  template <typename T>
  void vec(std::vector<T>& v) {
    const uint64_t n = scalar<uint64_t>();
    if (n > left_ / sizeof(T)) fail(IFILT_ECACHE, "cache file array runs past the end of the file");
    v.resize(n);
    raw(v.data(), n * sizeof(T));
  }
  void csr(HostCSR& c) {
    c.n = scalar<int32_t>();
    c.nval = scalar<int32_t>();
    vec(c.row_ptr);
    vec(c.col);
    vec(c.val);
  }
  uint64_t left() const { return left_; }
  uint64_t digest() const { return h_.digest(); }

 private:
  FILE* f_;
  Hash64 h_;
  uint64_t left_;
};

[[noreturn]] void bad(const char* what) { fail(IFILT_ECACHE, "cache file holds an inconsistent %s", what); }

// rows x ncols CSR with `nval` values per entry, columns strictly increasing
// within each row and inside [0, ncols).
void check_csr(const HostCSR& c, int64_t rows, int64_t ncols, int32_t nval, const char* what) {
  if (c.n != rows || c.nval != nval || c.row_ptr.size() != (size_t)rows + 1 || c.row_ptr[0] != 0) bad(what);
  for (int64_t r = 0; r < rows; r++) {
    const int64_t a = c.row_ptr[r], b = c.row_ptr[r + 1];
    if (b < a || b > (int64_t)c.col.size()) bad(what);
    for (int64_t q = a; q < b; q++)
      if (c.col[q] < 0 || c.col[q] >= ncols || (q > a && c.col[q] <= c.col[q - 1])) bad(what);
  }
  if (c.row_ptr[rows] != (int64_t)c.col.size() || c.val.size() != c.col.size() * (size_t)nval) bad(what);
  for (double v : c.val)
    if (!std::isfinite(v)) bad(what);
}

void check_finite(const std::vector<double>& v, size_t n, const char* what) {
  if (v.size() != n) bad(what);
  for (double x : v)
    if (!std::isfinite(x)) bad(what);
}

void check_prepared(const HostPrepared& h) {
  if (h.placement < IFILT_VERTEX_SCALAR || h.placement > IFILT_CELL_CIRCUMCENTER ||
      h.geometry < IFILT_GEOM_PLANAR_PERIODIC || h.geometry > IFILT_GEOM_SPHERE || h.max_order < 1 ||
      h.max_order > IFILT_MAX_ORDER || h.reorder < IFILT_REORDER_NONE || h.reorder > IFILT_REORDER_HILBERT)
    bad("header");
  const bool vec = h.placement == IFILT_VERTEX_VECTOR;
  const int32_t n_comp = (h.placement == IFILT_VERTEX_VECTOR || h.placement == IFILT_CELL) ? 2 : 1;
  if (h.n_rows <= 0 || h.n_in <= 0 || h.n_out <= 0 || h.n_comp != n_comp || h.n_rows > h.n_out) bad("header");
  if (!vec && h.n_in != h.n_out) bad("header");
  if (h.perm.size() != (size_t)h.n_rows) bad("permutation");
  std::vector<uint8_t> seen((size_t)h.n_out, 0);
  for (int32_t p : h.perm) {
    if (p < 0 || p >= h.n_out || seen[(size_t)p]) bad("permutation");
    seen[(size_t)p] = 1;
  }
  check_finite(h.mass, (size_t)h.n_rows, "lumped mass");
  const int32_t nv = vec ? 2 : 1;
  check_csr(h.K, h.n_rows, h.n_rows, nv, "operator K");
  if (h.max_order >= 2) check_csr(h.G2, h.n_rows, h.n_rows, nv, "operator K M^-1 K");
  else if (h.G2.nnz() != 0 || !h.G2.col.empty()) bad("operator K M^-1 K");
  if (h.Gn.size() != (size_t)std::max(0, h.max_order - 2)) bad("higher-order operators");
  for (const HostCSR& G : h.Gn) check_csr(G, h.n_rows, h.n_rows, nv, "higher-order operator");
  if (vec) {
    if (h.proj_ptr.size() != (size_t)h.n_rows + 1 || h.proj_ptr[0] != 0) bad("projection");
    for (int32_t r = 0; r < h.n_rows; r++)
      if (h.proj_ptr[r + 1] < h.proj_ptr[r]) bad("projection");
    if ((size_t)h.proj_ptr.back() != h.proj_cell.size()) bad("projection");
    for (int32_t c : h.proj_cell)
      if (c < 0 || c >= h.n_in) bad("projection");
    check_finite(h.proj_w, h.proj_cell.size(), "projection");
  } else if (!h.proj_ptr.empty() || !h.proj_cell.empty() || !h.proj_w.empty()) {
    bad("projection");
  }
}

void check_multigrid(const MgHost& g, const HostPrepared& h) {
  const size_t L = g.levels.size();
  if (L == 0 || L > IFILT_MG_MAX_LEVELS || g.levels[0].n != h.n_rows) bad("multigrid hierarchy");
  const int32_t nv = h.placement == IFILT_VERTEX_VECTOR ? 2 : 1;
  for (size_t l = 0; l < L; l++) {
    const MgHostLevel& Lv = g.levels[l];
    if (Lv.n <= 0 || !std::isfinite(Lv.omega_p) || !(Lv.omega_s > 0.0 && Lv.omega_s <= 1.0)) bad("multigrid level");
    if (l == 0) {
      if (!Lv.S.row_ptr.empty() || !Lv.S.col.empty()) bad("multigrid level 0");
    } else {
      check_csr(Lv.S, Lv.n, Lv.n, 2 * nv, "multigrid level operator");
    }
    if (l + 1 < L) {
      const int32_t nc = g.levels[l + 1].n;
      check_csr(Lv.P, Lv.n, nc, nv, "multigrid prolongation");
      check_csr(Lv.R, nc, Lv.n, nv, "multigrid restriction");
    } else if (!Lv.P.col.empty() || !Lv.R.col.empty()) {
      bad("multigrid coarsest level");
    }
    check_finite(Lv.dk, (size_t)Lv.n, "multigrid diagonal");
    check_finite(Lv.dm, (size_t)Lv.n, "multigrid diagonal");
  }
}

}  // namespace

uint64_t mesh_key(const ifilt_mesh_desc& d) {
  if (d.n_vert <= 0 || d.n_tri <= 0 || !d.coords || !d.tri)
    fail(IFILT_EINVAL, "mesh needs n_vert > 0, n_tri > 0, coords and tri");
  Hash64 h(0x6966696c746d6b79ULL);
  const uint32_t rev[2] = {kFormat, kPrepareRevision};
  h.update(rev, sizeof rev);
  const int32_t ints[7] = {d.n_vert, d.n_tri, d.geometry, d.placement, d.max_order, d.reorder, d.ell_slice};
  h.update(ints, sizeof ints);
  const double dbl[5] = {d.period_x, d.period_y, d.radius, d.cell_A, d.mg_strength};
  h.update(dbl, sizeof dbl);
  const int dim = d.geometry == IFILT_GEOM_SPHERE ? 3 : 2;
  h.update(d.coords, sizeof(double) * (size_t)d.n_vert * dim);
  h.update(d.tri, sizeof(int32_t) * 3 * (size_t)d.n_tri);
  const uint8_t has_ocean = d.ocean ? 1 : 0;
  h.update(&has_ocean, 1);
  if (d.ocean) {
    // any nonzero byte is ocean: hash the 0/1 flags, in chunks
    uint8_t buf[4096];
    for (int64_t i = 0; i < d.n_vert; i += (int64_t)sizeof buf) {
      const int64_t n = std::min<int64_t>(sizeof buf, d.n_vert - i);
      for (int64_t j = 0; j < n; j++) buf[j] = d.ocean[i + j] ? 1 : 0;
      h.update(buf, (size_t)n);
    }
  }
  uint64_t k = h.digest();
  return k ? k : 1;  // 0 means "do not check" in ifilt_mesh_load_host
}

void save_mesh(ifilt_mesh_s* m, const char* path, int32_t flags) {
  if (!path || !*path) fail(IFILT_EINVAL, "null or empty path");
  if (flags & ~IFILT_SAVE_MULTIGRID) fail(IFILT_EINVAL, "unknown save flags %d", flags);
  std::shared_ptr<MgHost> mg;
  if (flags & IFILT_SAVE_MULTIGRID) {
    multigrid_host(m);
    std::lock_guard<std::mutex> lk(m->mg_mu);
    mg = m->mg_host;
  }
  const HostPrepared& h = m->host;
  static std::atomic<uint64_t> serial{0};
  const std::string tmp = std::string(path) + ".tmp." + std::to_string((long long)getpid()) + "." +
                          std::to_string((unsigned long long)serial.fetch_add(1));
  {
    File fl;
    fl.f = std::fopen(tmp.c_str(), "wb");
    if (!fl.f) fail(IFILT_ECACHE, "cannot create %s", tmp.c_str());
    try {
      std::fwrite(kMagic, 1, sizeof kMagic, fl.f);
      const uint32_t fr[2] = {kFormat, kPrepareRevision};
      std::fwrite(fr, sizeof fr, 1, fl.f);
      const uint64_t hdr[3] = {h.key, 0, 0};  // payload bytes and hash filled in below
      std::fwrite(hdr, sizeof hdr, 1, fl.f);
      Writer w(fl.f);
      const int32_t ints[9] = {h.placement, h.geometry, h.max_order, h.reorder, h.n_rows,
                               h.n_in,      h.n_out,    h.n_comp,    m->slice_h};
      w.raw(ints, sizeof ints);
      w.scalar<double>(h.mg_strength);
      w.vec(h.perm);
      w.vec(h.mass);
      w.csr(h.K);
      w.csr(h.G2);
      w.scalar<int32_t>((int32_t)h.Gn.size());
      for (const HostCSR& G : h.Gn) w.csr(G);
      w.vec(h.proj_ptr);
      w.vec(h.proj_cell);
      w.vec(h.proj_w);
      w.scalar<int32_t>(mg ? (int32_t)mg->levels.size() : 0);
      if (mg) {
        for (const MgHostLevel& L : mg->levels) {
          w.scalar<int32_t>(L.n);
          w.scalar<double>(L.omega_p);
          w.scalar<double>(L.omega_s);
          w.csr(L.S);
          w.csr(L.P);
          w.csr(L.R);
          w.vec(L.dk);
          w.vec(L.dm);
        }
      }
      const uint64_t tail[2] = {w.bytes(), w.digest()};
      if (std::fseek(fl.f, (long)(sizeof kMagic + sizeof fr + sizeof(uint64_t)), SEEK_SET) != 0 ||
          std::fwrite(tail, sizeof tail, 1, fl.f) != 1 || std::fflush(fl.f) != 0)
        fail(IFILT_ECACHE, "cache file write failed");
      FILE* f = fl.f;
      fl.f = nullptr;
      if (std::fclose(f) != 0) fail(IFILT_ECACHE, "cache file write failed");
    } catch (...) {
      if (fl.f) {
        std::fclose(fl.f);
        fl.f = nullptr;
      }
      std::remove(tmp.c_str());
      throw;
    }
  }
  if (std::rename(tmp.c_str(), path) != 0) {
    std::remove(tmp.c_str());
    fail(IFILT_ECACHE, "cannot move the cache file into place at %s", path);
  }
}

ifilt_mesh_s* load_mesh_host(const char* path, uint64_t expect_key) {
  if (!path || !*path) fail(IFILT_EINVAL, "null or empty path");
  File fl;
  fl.f = std::fopen(path, "rb");
  if (!fl.f) fail(IFILT_ECACHE, "cannot open cache file %s", path);
  char magic[8];
  uint32_t fr[2];
  uint64_t hdr[3];
  if (std::fread(magic, 1, sizeof magic, fl.f) != sizeof magic || std::memcmp(magic, kMagic, sizeof magic) != 0)
    fail(IFILT_ECACHE, "%s is not an ifilt cache file", path);
  if (std::fread(fr, sizeof fr, 1, fl.f) != 1 || std::fread(hdr, sizeof hdr, 1, fl.f) != 1)
    fail(IFILT_ECACHE, "cache file %s is truncated", path);
  if (fr[0] != kFormat || fr[1] != kPrepareRevision)
    fail(IFILT_ECACHE, "cache file %s has format %u revision %u; this library writes %u / %u", path, fr[0], fr[1],
         kFormat, kPrepareRevision);
  if (expect_key && hdr[0] != expect_key) fail(IFILT_ECACHE, "cache file %s was written for another mesh", path);
  {
    // the payload length must be what the file holds (no allocation beyond the file's size)
    const long here = std::ftell(fl.f);
    if (here < 0 || std::fseek(fl.f, 0, SEEK_END) != 0) fail(IFILT_ECACHE, "cannot size cache file %s", path);
    const long end = std::ftell(fl.f);
    if (end < 0 || std::fseek(fl.f, here, SEEK_SET) != 0) fail(IFILT_ECACHE, "cannot size cache file %s", path);
    if ((uint64_t)(end - here) != hdr[1]) fail(IFILT_ECACHE, "cache file %s is truncated or has trailing bytes", path);
  }
  std::unique_ptr<ifilt_mesh_s> m(new ifilt_mesh_s());
  HostPrepared& h = m->host;
  h.key = hdr[0];
  Reader r(fl.f, hdr[1]);
  int32_t ints[9];
  r.raw(ints, sizeof ints);
  h.placement = ints[0];
  h.geometry = ints[1];
  h.max_order = ints[2];
  h.reorder = ints[3];
  h.n_rows = ints[4];
  h.n_in = ints[5];
  h.n_out = ints[6];
  h.n_comp = ints[7];
  m->slice_h = ints[8];
  h.mg_strength = r.scalar<double>();
  if (!(h.mg_strength >= 0.0 && h.mg_strength < 1.0)) bad("multigrid strength");
  r.vec(h.perm);
  r.vec(h.mass);
  r.csr(h.K);
  r.csr(h.G2);
  const int32_t n_gn = r.scalar<int32_t>();
  if (n_gn < 0 || n_gn > IFILT_MAX_ORDER - 2) bad("higher-order operator count");
  h.Gn.resize((size_t)n_gn);
  for (HostCSR& G : h.Gn) r.csr(G);
  r.vec(h.proj_ptr);
  r.vec(h.proj_cell);
  r.vec(h.proj_w);
  const int32_t levels = r.scalar<int32_t>();
  if (levels < 0 || levels > IFILT_MG_MAX_LEVELS) bad("multigrid level count");
  std::shared_ptr<MgHost> mg;
  if (levels) {
    mg = std::make_shared<MgHost>();
    mg->levels.resize((size_t)levels);
    for (MgHostLevel& L : mg->levels) {
      L.n = r.scalar<int32_t>();
      L.omega_p = r.scalar<double>();
      L.omega_s = r.scalar<double>();
      r.csr(L.S);
      r.csr(L.P);
      r.csr(L.R);
      r.vec(L.dk);
      r.vec(L.dm);
    }
  }
  if (r.left() != 0) fail(IFILT_ECACHE, "cache file %s is longer than its header says", path);
  char extra;
  if (std::fread(&extra, 1, 1, fl.f) != 0) fail(IFILT_ECACHE, "cache file %s has trailing bytes", path);
  if (r.digest() != hdr[2]) fail(IFILT_ECACHE, "cache file %s fails its checksum", path);
  if (m->slice_h != 0 && (m->slice_h < 4 || m->slice_h > 1024)) bad("slice height");
  check_prepared(h);
  if (mg) {
    check_multigrid(*mg, h);
    m->mg_host = mg;
  }
  return m.release();
}

}  // namespace ifilt
