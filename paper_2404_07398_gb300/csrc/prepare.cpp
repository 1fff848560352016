// Host side of the preparation phase (Sect. 2.2.1 of the paper): everything
// that depends on the mesh only and is reused for every scale and field.
//
//   1. ocean subset: a triangle is in the domain iff its three vertices are
//      ocean; coast edges carry the no-flux condition of Sect. 2.1 by simply
//      having no neighbour across them;
//   2. device row order: reverse Cuthill-McKee on the graph of the n = 1
//      operator (least (degree, id) start per component, children by
//      (degree, id), sequence reversed) so that gathered neighbour rows of a
//      sparse product sit close together in memory;
//   3. the l-free operator K of the placement and the lumped mass:
//        vertex scalar: K_ab = int grad N_a . grad N_b = -1/2 cot(opposite angle)
//                       summed over the two triangles of edge ab, A_v = sum A_c/3
//                       (Sect. 2.1.1);
//        vertex vector: blocks [[K~, Tm], [-Tm, K~]], K~ = stiffness + (R^-2 + m^2)
//                       x consistent P1 mass, Tm_ab = int m (-N_b d_x N_a + N_a d_x N_b),
//                       m = tan(lat)/R per triangle (Sect. 2.1.2);
//        cell:          A * graph Laplacian of edge-adjacent triangles, A_c (Eq. 6);
//   4. G2 = K M^-1 K for order n = 2 (Sect. 2.1.1).
// Everything is FP64 here; device copies are cast once at upload.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <numeric>

#include "host_parallel.h"
#include "internal.h"

namespace ifilt {
namespace {

struct V3 {
  double x, y, z;
};
inline V3 sub(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
inline V3 add(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
inline V3 scale(V3 a, double s) { return {a.x * s, a.y * s, a.z * s}; }
inline double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline V3 cross(V3 a, V3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
inline double norm(V3 a) { return std::sqrt(dot(a, a)); }

struct Geometry {
  const double* xy;
  int geom;
  double px, py, radius;
  V3 pos(int v) const {
    if (geom == IFILT_GEOM_SPHERE) return {xy[3 * (int64_t)v], xy[3 * (int64_t)v + 1], xy[3 * (int64_t)v + 2]};
    return {xy[2 * (int64_t)v], xy[2 * (int64_t)v + 1], 0.0};
  }
  // x_b - x_a, minimum image on the periodic plane
  V3 edge(int a, int b) const {
    V3 d = sub(pos(b), pos(a));
    if (geom == IFILT_GEOM_PLANAR_PERIODIC) {
      d.x -= px * std::nearbyint(d.x / px);
      d.y -= py * std::nearbyint(d.y / py);
    }
    return d;
  }
};

// Compressed adjacency (no self loops), rows sorted ascending.
struct Graph {
  int32_t n = 0;
  std::vector<int64_t> ptr;
  std::vector<int32_t> adj;
};

// counting-sort based CSR "item -> list" builder
void bucket(int32_t n, const std::vector<int32_t>& key, std::vector<int64_t>& ptr,
            std::vector<int32_t>& idx) {
  ptr.assign((size_t)n + 1, 0);
  for (int32_t k : key) ptr[(size_t)k + 1]++;
  for (int32_t i = 0; i < n; i++) ptr[i + 1] += ptr[i];
  idx.resize(key.size());
  std::vector<int64_t> fill(ptr.begin(), ptr.end() - 1);
  for (size_t i = 0; i < key.size(); i++) idx[fill[key[i]]++] = (int32_t)i;
}

// Index of grid cell (x, y), 0 <= x, y < 2^bits, along the Hilbert curve that
// starts at (0, 0) and ends at (2^bits - 1, 0).  Top bit first: the quadrant
// gives two bits of the index (lower-left 0, upper-left 1, upper-right 2,
// lower-right 3), then the coordinates inside the quadrant are mapped into the
// sub-curve's own frame (the lower quadrants are transposed, the lower-right
// one also reflected) and the next bit is read.
uint64_t hilbert_index(uint32_t x, uint32_t y, int bits) {
  uint64_t d = 0;
  for (int b = bits - 1; b >= 0; b--) {
    const uint32_t s = 1u << b;
    const uint32_t rx = (x >> b) & 1u, ry = (y >> b) & 1u;
    d += (uint64_t)s * s * ((3u * rx) ^ ry);
    x &= s - 1;
    y &= s - 1;
    if (ry == 0) {
      if (rx == 1) {
        x = s - 1 - x;
        y = s - 1 - y;
      }
      std::swap(x, y);
    }
  }
  return d;
}

constexpr int kCurveBits = 16;

inline uint32_t quantise(double t) {  // t in [0, 1] -> 0 .. 2^bits - 1
  const double q = std::floor(t * (double)(1u << kCurveBits));
  if (!(q > 0.0)) return 0;
  if (q >= (double)((1u << kCurveBits) - 1)) return (1u << kCurveBits) - 1;
  return (uint32_t)q;
}

// Space-filling-curve key of a point.  Sphere: the cube face of the direction
// (largest |component|, ties to x then y; +axis before -axis) and the two other
// components divided by the largest, each in [-1, 1]; plane: the coordinates
// scaled to the mesh's bounding box.
uint64_t curve_key(const double* p, bool sphere, const double* lo, const double* span) {
  if (sphere) {
    const double ax = std::fabs(p[0]), ay = std::fabs(p[1]), az = std::fabs(p[2]);
    int face;
    double u, v, m;
    if (ax >= ay && ax >= az) {
      face = p[0] >= 0.0 ? 0 : 1;
      m = ax;
      u = p[1];
      v = p[2];
    } else if (ay >= az) {
      face = p[1] >= 0.0 ? 2 : 3;
      m = ay;
      u = p[0];
      v = p[2];
    } else {
      face = p[2] >= 0.0 ? 4 : 5;
      m = az;
      u = p[0];
      v = p[1];
    }
    const uint32_t iu = quantise((u / m + 1.0) * 0.5), iv = quantise((v / m + 1.0) * 0.5);
    return ((uint64_t)face << (2 * kCurveBits)) | hilbert_index(iu, iv, kCurveBits);
  }
  const uint32_t ix = quantise((p[0] - lo[0]) / span[0]), iy = quantise((p[1] - lo[1]) / span[1]);
  return hilbert_index(ix, iy, kCurveBits);
}

std::vector<int32_t> reverse_cuthill_mckee(const Graph& g) {
  const int32_t n = g.n;
  std::vector<int32_t> deg(n);
  int32_t maxdeg = 0;
  for (int32_t v = 0; v < n; v++) {
    deg[v] = (int32_t)(g.ptr[v + 1] - g.ptr[v]);
    maxdeg = std::max(maxdeg, deg[v]);
  }
  // vertices by (degree, id): counting sort on degree, stable in id
  std::vector<int64_t> cnt((size_t)maxdeg + 2, 0);
  for (int32_t v = 0; v < n; v++) cnt[deg[v] + 1]++;
  for (int32_t d = 0; d <= maxdeg; d++) cnt[d + 1] += cnt[d];
  std::vector<int32_t> by_key(n);
  for (int32_t v = 0; v < n; v++) by_key[cnt[deg[v]]++] = v;

  std::vector<uint8_t> seen(n, 0);
  std::vector<int32_t> seq;
  seq.reserve(n);
  std::vector<int32_t> fresh;
  size_t scan = 0, head = 0;
  while ((int32_t)seq.size() < n) {
    while (seen[by_key[scan]]) scan++;
    int32_t s = by_key[scan];
    seen[s] = 1;
    seq.push_back(s);
    while (head < seq.size()) {
      int32_t u = seq[head++];
      fresh.clear();
      for (int64_t e = g.ptr[u]; e < g.ptr[u + 1]; e++) {
        int32_t w = g.adj[e];
        if (!seen[w]) {
          seen[w] = 1;
          fresh.push_back(w);
        }
      }
      std::sort(fresh.begin(), fresh.end(), [&](int32_t a, int32_t b) {
        return deg[a] != deg[b] ? deg[a] < deg[b] : a < b;
      });
      seq.insert(seq.end(), fresh.begin(), fresh.end());
    }
  }
  std::reverse(seq.begin(), seq.end());
  return seq;
}

// Position of column c in row r of a CSR with sorted columns.
// Circumcentre of a (flat) triangle tv, as a vector from its vertex `from`
// (edge vectors are minimum images on periodic planes):  with e1, e2 the edges
// from `from`, n = e1 x e2, it is (|e1|^2 e2 x n + |e2|^2 n x e1) / (2 |n|^2).
inline V3 circumcentre_from(const Geometry& geo, const int32_t* tv, int from) {
  int o[2], k = 0;
  for (int i = 0; i < 3; i++)
    if (tv[i] != from) o[k++] = tv[i];
  const V3 e1 = geo.edge(from, o[0]), e2 = geo.edge(from, o[1]);
  const V3 n = cross(e1, e2);
  const double n2 = dot(n, n);
  return scale(add(scale(cross(e2, n), dot(e1, e1)), scale(cross(n, e1), dot(e2, e2))), 0.5 / n2);
}

inline int64_t find_entry(const HostCSR& a, int32_t r, int32_t c) {
  const int32_t* b = a.col.data() + a.row_ptr[r];
  const int32_t* e = a.col.data() + a.row_ptr[r + 1];
  const int32_t* p = std::lower_bound(b, e, c);
  return (p != e && *p == c) ? (int64_t)(p - a.col.data()) : -1;
}

// CSR pattern in device order from a compact-id graph and the permutation.
HostCSR pattern_from_graph(const Graph& g, const std::vector<int32_t>& order,
                           const std::vector<int32_t>& rank, int nval) {
  HostCSR a;
  a.n = g.n;
  a.nval = nval;
  a.row_ptr.assign((size_t)g.n + 1, 0);
  for (int32_t r = 0; r < g.n; r++) {
    int32_t c = order[r];
    a.row_ptr[r + 1] = a.row_ptr[r] + (g.ptr[c + 1] - g.ptr[c]) + 1;
  }
  a.col.resize(a.row_ptr.back());
  for (int32_t r = 0; r < g.n; r++) {
    int32_t c = order[r];
    int32_t* out = a.col.data() + a.row_ptr[r];
    int k = 0;
    out[k++] = r;
    for (int64_t e = g.ptr[c]; e < g.ptr[c + 1]; e++) out[k++] = rank[g.adj[e]];
    std::sort(out, out + k);
  }
  a.val.assign((size_t)a.col.size() * nval, 0.0);
  return a;
}

// G = A M^-1 K with the structural product pattern (explicit zeros kept):
// K M^-1 K for order 2 (A = K), and G_n = G_(n-1) M^-1 K for higher orders.
// Rows are independent: each gathers its candidate products in the order
// (entry e of row i of A, entry f of row A.col[e] of K), sorts them stably by column and
// sums each column's run in that order, so every value is the same sum, in the
// same order, whatever the number of threads.  Two passes: row sizes from the
// columns alone, then columns and sums written in place.
HostCSR product_amk(const HostCSR& A, const HostCSR& K, const std::vector<double>& mass) {
  const int32_t n = K.n;
  const int nv = K.nval;
  HostCSR G;
  G.n = n;
  G.nval = nv;
  G.row_ptr.assign((size_t)n + 1, 0);
  struct Cand {
    int32_t k;
    int64_t e, f;
  };
  const int nt = host_threads();
  std::vector<std::vector<Cand>> scratch((size_t)nt);
  std::vector<std::vector<int32_t>> cscratch((size_t)nt);
  constexpr int64_t kRows = 4096;
  parallel_range(n, kRows, [&](int64_t b, int64_t e, int w) {
    std::vector<int32_t>& c = cscratch[(size_t)w];
    for (int64_t i = b; i < e; i++) {
      c.clear();
      for (int64_t q = A.row_ptr[i]; q < A.row_ptr[i + 1]; q++) {
        const int32_t j = A.col[q];
        c.insert(c.end(), K.col.begin() + K.row_ptr[j], K.col.begin() + K.row_ptr[j + 1]);
      }
      stable_sort_small(c.data(), (int64_t)c.size(), [](int32_t x, int32_t y) { return x < y; });
      int64_t cnt = 0;
      for (size_t t = 0; t < c.size(); t++) cnt += (t == 0 || c[t] != c[t - 1]) ? 1 : 0;
      G.row_ptr[i + 1] = cnt;
    }
  });
  for (int32_t i = 0; i < n; i++) G.row_ptr[i + 1] += G.row_ptr[i];
  G.col.resize(G.row_ptr.back());
  G.val.resize((size_t)G.row_ptr.back() * nv);
  parallel_range(n, kRows, [&](int64_t b, int64_t e, int w) {
    std::vector<Cand>& c = scratch[(size_t)w];
    for (int64_t i = b; i < e; i++) {
      c.clear();
      for (int64_t q = A.row_ptr[i]; q < A.row_ptr[i + 1]; q++) {
        const int32_t j = A.col[q];
        for (int64_t f = K.row_ptr[j]; f < K.row_ptr[j + 1]; f++) c.push_back(Cand{K.col[f], q, f});
      }
      stable_sort_small(c.data(), (int64_t)c.size(), [](const Cand& x, const Cand& y) { return x.k < y.k; });
      int64_t o = G.row_ptr[i];
      for (size_t t = 0; t < c.size(); o++) {
        const int32_t col = c[t].k;
        double s0 = 0.0, s1 = 0.0;
        for (; t < c.size() && c[t].k == col; t++) {
          const int64_t ee = c[t].e, ff = c[t].f;
          const double inv = 1.0 / mass[A.col[ee]];
          if (nv == 1) {
            s0 += A.val[ee] * inv * K.val[ff];
          } else {
            // blocks [[a, b], [-b, a]] multiply like a + i b
            const double a1 = A.val[2 * ee] * inv, b1 = A.val[2 * ee + 1] * inv;
            const double a2 = K.val[2 * ff], b2 = K.val[2 * ff + 1];
            s0 += a1 * a2 - b1 * b2;
            s1 += a1 * b2 + b1 * a2;
          }
        }
        G.col[o] = col;
        G.val[(size_t)o * nv] = s0;
        if (nv == 2) G.val[(size_t)o * nv + 1] = s1;
      }
    }
  });
  return G;
}

}  // namespace

static double wall_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}
PhaseClock::PhaseClock(const char* w) : what(w), t0(wall_ms()) {
  const char* e = getenv("IFILT_TRACE_PREPARE");
  on = e && e[0] == '1';
}
void PhaseClock::lap(const char* phase) {
  if (!on) return;
  const double t = wall_ms();
  fprintf(stderr, "ifilt %s: %-24s %9.1f ms\n", what, phase, t - t0);
  t0 = t;
}

void host_products(HostPrepared& hp) {
  hp.G2 = HostCSR{};
  hp.Gn.clear();
  if (hp.max_order >= 2) hp.G2 = product_amk(hp.K, hp.K, hp.mass);
  for (int n = 3; n <= hp.max_order; n++) hp.Gn.push_back(product_amk(n == 3 ? hp.G2 : hp.Gn.back(), hp.K, hp.mass));
  hp.products_pending = false;
}

HostPrepared prepare_host(const ifilt_mesh_desc& d, bool products) {
  if (d.n_vert <= 0 || d.n_tri <= 0 || !d.coords || !d.tri)
    fail(IFILT_EINVAL, "mesh needs n_vert > 0, n_tri > 0, coords and tri");
  if (d.placement < IFILT_VERTEX_SCALAR || d.placement > IFILT_CELL_CIRCUMCENTER)
    fail(IFILT_EINVAL, "unknown placement %d", d.placement);
  if (d.geometry < IFILT_GEOM_PLANAR_PERIODIC || d.geometry > IFILT_GEOM_SPHERE) fail(IFILT_EINVAL, "unknown geometry %d", d.geometry);
  if (d.max_order < 1 || d.max_order > IFILT_MAX_ORDER) fail(IFILT_EINVAL, "max_order must be 1 .. %d", IFILT_MAX_ORDER);
  if (d.geometry == IFILT_GEOM_PLANAR_PERIODIC && !(d.period_x > 0 && d.period_y > 0))
    fail(IFILT_EINVAL, "periodic geometry needs positive periods");
  if (d.geometry == IFILT_GEOM_SPHERE && !(d.radius > 0)) fail(IFILT_EINVAL, "sphere needs radius > 0");
  if (d.reorder < IFILT_REORDER_NONE || d.reorder > IFILT_REORDER_HILBERT) fail(IFILT_EINVAL, "unknown reorder %d", d.reorder);
  if (!(d.mg_strength >= 0.0 && d.mg_strength < 1.0)) fail(IFILT_EINVAL, "mg_strength must be in [0, 1)");

  const int32_t V = d.n_vert, T = d.n_tri;
  const int32_t* tri = d.tri;
  const int dim = d.geometry == IFILT_GEOM_SPHERE ? 3 : 2;
  for (int64_t i = 0; i < (int64_t)V * dim; i++)
    if (!std::isfinite(d.coords[i])) fail(IFILT_EMESH, "coordinate %lld is not finite", (long long)i);
  for (int32_t t = 0; t < T; t++) {
    int a = tri[3 * (int64_t)t], b = tri[3 * (int64_t)t + 1], c = tri[3 * (int64_t)t + 2];
    if (a < 0 || b < 0 || c < 0 || a >= V || b >= V || c >= V)
      fail(IFILT_EMESH, "triangle %d has a vertex index out of range", t);
    if (a == b || b == c || a == c) fail(IFILT_EMESH, "triangle %d repeats a vertex", t);
  }
  Geometry geo{d.coords, d.geometry, d.period_x, d.period_y, d.radius};
  PhaseClock clock("prepare");

  HostPrepared hp;
  hp.placement = d.placement;
  hp.geometry = d.geometry;
  hp.max_order = d.max_order;
  hp.reorder = d.reorder;
  hp.mg_strength = d.mg_strength;

  // ---- 1. ocean subset
  std::vector<int32_t> kept;  // original ids of kept triangles, ascending
  kept.reserve(T);
  for (int32_t t = 0; t < T; t++) {
    bool k = true;
    if (d.ocean)
      k = d.ocean[tri[3 * (int64_t)t]] && d.ocean[tri[3 * (int64_t)t + 1]] && d.ocean[tri[3 * (int64_t)t + 2]];
    if (k) kept.push_back(t);
  }
  if (kept.empty()) fail(IFILT_EMESH, "no ocean triangle");
  const int32_t Tk = (int32_t)kept.size();
  std::vector<double> area(Tk);
  for (int32_t c = 0; c < Tk; c++) {
    const int32_t* tv = tri + 3 * (int64_t)kept[c];
    V3 e1 = geo.edge(tv[0], tv[1]), e2 = geo.edge(tv[0], tv[2]);
    area[c] = 0.5 * norm(cross(e1, e2));
    if (!(area[c] > 0.0)) fail(IFILT_EMESH, "triangle %d has zero area", kept[c]);
  }
  // vertex compaction (ascending original id)
  std::vector<int32_t> vid(V, -1), verts;
  for (int32_t c = 0; c < Tk; c++)
    for (int q = 0; q < 3; q++) vid[tri[3 * (int64_t)kept[c] + q]] = 0;
  for (int32_t v = 0; v < V; v++)
    if (vid[v] == 0) {
      vid[v] = (int32_t)verts.size();
      verts.push_back(v);
    }
  const int32_t Nv = (int32_t)verts.size();
  // incidence: compact vertex -> kept triangles (compact triangle ids)
  std::vector<int32_t> inc_key((size_t)Tk * 3);
  for (int32_t c = 0; c < Tk; c++)
    for (int q = 0; q < 3; q++) inc_key[3 * (size_t)c + q] = vid[tri[3 * (int64_t)kept[c] + q]];
  std::vector<int64_t> inc_ptr;
  std::vector<int32_t> inc_idx;  // -> 3*c + corner
  bucket(Nv, inc_key, inc_ptr, inc_idx);
  auto corner_v = [&](int32_t c, int q) { return vid[tri[3 * (int64_t)kept[c] + q]]; };

  clock.lap("ocean subset");
  // ---- graph of the n = 1 operator (compact ids)
  Graph g;
  const bool cells = d.placement == IFILT_CELL || d.placement == IFILT_CELL_CIRCUMCENTER;
  if (!cells) {
    g.n = Nv;
    g.ptr.assign((size_t)Nv + 1, 0);
    std::vector<int32_t> tmp;
    std::vector<std::vector<int32_t>> rows;  // built row by row
    g.adj.reserve((size_t)Nv * 7);
    for (int32_t v = 0; v < Nv; v++) {
      tmp.clear();
      for (int64_t e = inc_ptr[v]; e < inc_ptr[v + 1]; e++) {
        int32_t c = inc_idx[e] / 3;
        for (int q = 0; q < 3; q++) {
          int32_t w = corner_v(c, q);
          if (w != v) tmp.push_back(w);
        }
      }
      std::sort(tmp.begin(), tmp.end());
      tmp.erase(std::unique(tmp.begin(), tmp.end()), tmp.end());
      g.adj.insert(g.adj.end(), tmp.begin(), tmp.end());
      g.ptr[v + 1] = (int64_t)g.adj.size();
    }
  } else {
    g.n = Tk;
    g.ptr.assign((size_t)Tk + 1, 0);
    g.adj.reserve((size_t)Tk * 3);
    std::vector<int32_t> tmp;
    for (int32_t c = 0; c < Tk; c++) {
      tmp.clear();
      for (int q = 0; q < 3; q++) {
        int32_t a = corner_v(c, q), b = corner_v(c, (q + 1) % 3);
        int found = 0;
        // triangles incident to a that also contain b
        for (int64_t e = inc_ptr[a]; e < inc_ptr[a + 1]; e++) {
          int32_t c2 = inc_idx[e] / 3;
          if (c2 == c) continue;
          if (corner_v(c2, 0) == b || corner_v(c2, 1) == b || corner_v(c2, 2) == b) {
            tmp.push_back(c2);
            found++;
          }
        }
        if (found > 1) fail(IFILT_EMESH, "an edge of triangle %d is shared by more than two ocean triangles", kept[c]);
      }
      std::sort(tmp.begin(), tmp.end());
      tmp.erase(std::unique(tmp.begin(), tmp.end()), tmp.end());
      g.adj.insert(g.adj.end(), tmp.begin(), tmp.end());
      g.ptr[c + 1] = (int64_t)g.adj.size();
    }
  }
  const int32_t N = g.n;

  clock.lap("graph");
  // ---- 2. device order
  std::vector<int32_t> order(N), rank(N);
  if (d.reorder == IFILT_REORDER_RCM) {
    order = reverse_cuthill_mckee(g);
  } else if (d.reorder == IFILT_REORDER_HILBERT) {
    // positions: the vertex, or the triangle's corner average ((a + b) + c) / 3
    const bool sphere = d.geometry == IFILT_GEOM_SPHERE;
    double lo[2] = {0, 0}, span[2] = {1, 1};
    if (!sphere) {
      double hi[2] = {d.coords[0], d.coords[1]};
      lo[0] = d.coords[0];
      lo[1] = d.coords[1];
      for (int32_t v = 0; v < V; v++)
        for (int k = 0; k < 2; k++) {
          lo[k] = std::min(lo[k], d.coords[2 * (int64_t)v + k]);
          hi[k] = std::max(hi[k], d.coords[2 * (int64_t)v + k]);
        }
      for (int k = 0; k < 2; k++) span[k] = hi[k] > lo[k] ? hi[k] - lo[k] : 1.0;
    }
    std::vector<std::pair<uint64_t, int32_t>> key(N);
    for (int32_t i = 0; i < N; i++) {
      double pos[3];
      if (cells) {
        const int32_t* tv = tri + 3 * (int64_t)kept[i];
        for (int k = 0; k < dim; k++)
          pos[k] = ((d.coords[dim * (int64_t)tv[0] + k] + d.coords[dim * (int64_t)tv[1] + k]) +
                    d.coords[dim * (int64_t)tv[2] + k]) / 3.0;
      } else {
        for (int k = 0; k < dim; k++) pos[k] = d.coords[dim * (int64_t)verts[i] + k];
      }
      key[i] = {curve_key(pos, sphere, lo, span), i};
    }
    std::sort(key.begin(), key.end());
    for (int32_t r = 0; r < N; r++) order[r] = key[r].second;
  } else {
    std::iota(order.begin(), order.end(), 0);
  }
  for (int32_t r = 0; r < N; r++) rank[order[r]] = r;

  hp.n_rows = N;
  hp.perm.resize(N);
  for (int32_t r = 0; r < N; r++) hp.perm[r] = cells ? kept[order[r]] : verts[order[r]];
  const bool scalar_in = d.placement == IFILT_VERTEX_SCALAR || d.placement == IFILT_VERTEX_VORONOI ||
                         d.placement == IFILT_CELL_CIRCUMCENTER;
  hp.n_comp = scalar_in ? 1 : 2;
  hp.n_in = (d.placement == IFILT_VERTEX_SCALAR || d.placement == IFILT_VERTEX_VORONOI) ? V : T;
  hp.n_out = cells ? T : V;

  clock.lap("device order");
  // ---- 3. operator and mass in device order
  const int nval = d.placement == IFILT_VERTEX_VECTOR ? 2 : 1;
  hp.K = pattern_from_graph(g, order, rank, nval);
  HostCSR& K = hp.K;
  hp.mass.assign(N, 0.0);
  if (d.placement == IFILT_CELL_CIRCUMCENTER) {
    // flux weight of a shared edge: its length over the distance between the two circumcentres,
    // both circumcentres taken relative to the edge's first vertex (minimum-image edges)
    for (int32_t r = 0; r < N; r++) hp.mass[r] = area[order[r]];
    std::vector<double> offd(K.col.size(), 0.0);
    for (int32_t r = 0; r < N; r++) {
      const int32_t c = order[r];
      const int32_t* tv = tri + 3 * (int64_t)kept[c];
      for (int64_t q = K.row_ptr[r]; q < K.row_ptr[r + 1]; q++) {
        const int32_t r2 = K.col[q];
        if (r2 == r) continue;
        const int32_t* tw = tri + 3 * (int64_t)kept[order[r2]];
        // shared edge (a, b)
        int a = -1, b = -1;
        for (int i = 0; i < 3; i++)
          for (int j = 0; j < 3; j++)
            if (tv[i] == tw[j]) {
              if (a < 0) a = tv[i];
              else b = tv[i];
            }
        if (a < 0 || b < 0) fail(IFILT_EMESH, "neighbouring triangles %d and %d share no edge", kept[c], kept[order[r2]]);
        const V3 oc = circumcentre_from(geo, tv, a), oc2 = circumcentre_from(geo, tw, a);
        const double le = norm(geo.edge(a, b)), dcc = norm(sub(oc, oc2));
        if (!(dcc > 1e-12 * le)) fail(IFILT_EMESH, "triangles %d and %d have coincident circumcentres", kept[c],
                                      kept[order[r2]]);
        offd[q] = -le / dcc;
      }
    }
    for (int32_t r = 0; r < N; r++) {
      double sdiag = 0.0;
      int64_t pd = -1;
      for (int64_t q = K.row_ptr[r]; q < K.row_ptr[r + 1]; q++) {
        if (K.col[q] == r) pd = q;
        else sdiag -= offd[q];
      }
      for (int64_t q = K.row_ptr[r]; q < K.row_ptr[r + 1]; q++) K.val[q] = q == pd ? sdiag : offd[q];
    }
  } else if (cells) {
    const double Ac = d.cell_A > 0 ? d.cell_A : std::sqrt(3.0);
    for (int32_t r = 0; r < N; r++) {
      int64_t b = K.row_ptr[r], e = K.row_ptr[r + 1];
      for (int64_t q = b; q < e; q++) K.val[q] = (K.col[q] == r) ? Ac * (double)(e - b - 1) : -Ac;
      hp.mass[r] = area[order[r]];
    }
  } else if (d.placement == IFILT_VERTEX_VORONOI) {
    // per triangle and edge: h = signed distance from the circumcentre to the edge midpoint,
    // positive toward the opposite corner; the edge's flux weight gains h / d (l_vv' is the sum of
    // the h of its triangles) and each end's dual cell the kite area d h / 4
    std::vector<double> offd(K.col.size(), 0.0);
    for (int32_t c = 0; c < Tk; c++) {
      const int32_t* tv = tri + 3 * (int64_t)kept[c];
      int32_t rr[3] = {rank[vid[tv[0]]], rank[vid[tv[1]]], rank[vid[tv[2]]]};
      const V3 o = circumcentre_from(geo, tv, tv[0]);  // relative to corner 0
      for (int k = 0; k < 3; k++) {
        const int a = (k + 1) % 3, b = (k + 2) % 3;
        const V3 pa = geo.edge(tv[0], tv[a]), pb = geo.edge(tv[0], tv[b]), pk = geo.edge(tv[0], tv[k]);
        const V3 e = sub(pb, pa);
        const double de = norm(e);
        const V3 mid = scale(add(pa, pb), 0.5);
        const V3 t = scale(e, 1.0 / de);
        V3 toward = sub(pk, mid);
        toward = sub(toward, scale(t, dot(toward, t)));
        const V3 u = scale(toward, 1.0 / norm(toward));
        const double h = dot(sub(o, mid), u);
        offd[find_entry(K, rr[a], rr[b])] -= h / de;
        offd[find_entry(K, rr[b], rr[a])] -= h / de;
        hp.mass[rr[a]] += 0.25 * de * h;
        hp.mass[rr[b]] += 0.25 * de * h;
      }
    }
    for (int32_t r = 0; r < N; r++) {
      double sdiag = 0.0;
      int64_t pd = -1;
      for (int64_t q = K.row_ptr[r]; q < K.row_ptr[r + 1]; q++) {
        if (K.col[q] == r) pd = q;
        else sdiag -= offd[q];
      }
      for (int64_t q = K.row_ptr[r]; q < K.row_ptr[r + 1]; q++) K.val[q] = q == pd ? sdiag : offd[q];
    }
    for (int32_t r = 0; r < N; r++)
      if (!(hp.mass[r] > 0.0)) fail(IFILT_EMESH, "vertex %d has a non-positive circumcentric dual area", hp.perm[r]);
  } else {
    const bool vec = d.placement == IFILT_VERTEX_VECTOR;
    const bool sphere = d.geometry == IFILT_GEOM_SPHERE;
    const double inv_r2 = sphere ? 1.0 / (d.radius * d.radius) : 0.0;
    const size_t nnz = K.col.size();
    // Two phases so that rows can be assembled in parallel with the serial
    // sums: (a) per triangle, its cotangent weights (and for vectors the metric
    // factor and zonal derivatives of the basis functions); (b) per row, the
    // contributions of the row's triangles in increasing triangle order (the
    // incidence lists are ascending), which is the order a triangle-by-triangle
    // scatter would add them in.
    std::vector<double> tw((size_t)Tk * 3), tcoef, tmet, tdx;
    if (vec) {
      tcoef.resize(Tk);
      tmet.resize(Tk);
      tdx.resize((size_t)Tk * 3);
    }
    parallel_range(Tk, 4096, [&](int64_t cb, int64_t ce, int) {
      for (int64_t c = cb; c < ce; c++) {
        const int32_t* tv = tri + 3 * (int64_t)kept[c];
        // stiffness: corner k receives nothing, its opposite edge (a, b) gets -1/2 cot
        for (int k = 0; k < 3; k++) {
          const int a = (k + 1) % 3, b = (k + 2) % 3;
          const V3 u = geo.edge(tv[k], tv[a]), v = geo.edge(tv[k], tv[b]);
          tw[3 * (size_t)c + k] = -0.5 * dot(u, v) / norm(cross(u, v));
        }
        if (vec) {
          // metric factor m = tan(lat)/R and zonal unit vector at the centroid direction
          double m = 0.0;
          V3 east{1.0, 0.0, 0.0};
          if (sphere) {
            V3 cdir = add(add(geo.pos(tv[0]), geo.pos(tv[1])), geo.pos(tv[2]));
            cdir = scale(cdir, 1.0 / norm(cdir));
            const double lat = std::asin(std::max(-1.0, std::min(1.0, cdir.z)));
            m = std::tan(lat) / d.radius;
            const double h = std::sqrt(cdir.x * cdir.x + cdir.y * cdir.y);
            east = {-cdir.y / h, cdir.x / h, 0.0};
          }
          // P1 gradients on the flat triangle: grad N_k = n x (x_{k+2} - x_{k+1}) / (2A)
          const V3 e1 = geo.edge(tv[0], tv[1]), e2 = geo.edge(tv[0], tv[2]);
          V3 nrm = cross(e1, e2);
          const double twoA = norm(nrm);
          nrm = scale(nrm, 1.0 / twoA);
          for (int k = 0; k < 3; k++) {
            const V3 eab = geo.edge(tv[(k + 1) % 3], tv[(k + 2) % 3]);
            tdx[3 * (size_t)c + k] = dot(scale(cross(nrm, eab), 1.0 / twoA), east);
          }
          tcoef[c] = inv_r2 + m * m;
          tmet[c] = m;
        }
      }
    });
    std::vector<double> stiff(nnz, 0.0), mmass, tm;
    if (vec) {
      mmass.assign(nnz, 0.0);
      tm.assign(nnz, 0.0);
    }
    parallel_range(N, 4096, [&](int64_t rb, int64_t re, int) {
      for (int64_t r = rb; r < re; r++) {
        const int32_t v = order[r];
        for (int64_t e = inc_ptr[v]; e < inc_ptr[v + 1]; e++) {
          const int32_t c = inc_idx[e] / 3, a = inc_idx[e] % 3;
          const int32_t* tv = tri + 3 * (int64_t)kept[c];
          const double A = area[c];
          hp.mass[r] += A / 3.0;
          for (int b = 0; b < 3; b++) {
            const int64_t p = find_entry(K, (int32_t)r, rank[vid[tv[b]]]);
            if (b != a) stiff[p] += tw[3 * (size_t)c + (3 - a - b)];
            if (vec) {
              // consistent P1 mass: A/6 on the diagonal, A/12 off it
              mmass[p] += tcoef[c] * (a == b ? A / 6.0 : A / 12.0);
              // int N = A/3; m and d_x N are constant on the triangle
              if (a != b) tm[p] += tmet[c] * (A / 3.0) * (tdx[3 * (size_t)c + b] - tdx[3 * (size_t)c + a]);
            }
          }
        }
        // diagonal stiffness: minus the off-diagonal row sum (basis functions sum to one)
        double sum = 0.0;
        int64_t pd = -1;
        for (int64_t q = K.row_ptr[r]; q < K.row_ptr[r + 1]; q++) {
          if (K.col[q] == r) pd = q;
          else sum += stiff[q];
        }
        stiff[pd] = -sum;
        for (int64_t q = K.row_ptr[r]; q < K.row_ptr[r + 1]; q++) {
          if (vec) {
            K.val[2 * q] = stiff[q] + mmass[q];
            K.val[2 * q + 1] = tm[q];
          } else {
            K.val[q] = stiff[q];
          }
        }
      }
    });
  }
  if (d.placement == IFILT_VERTEX_VECTOR) {
    // Projection of cell velocities to vertices: R_vc = A_c / 3 (Sect. 2.1.2)
    hp.proj_ptr.assign((size_t)N + 1, 0);
    for (int32_t r = 0; r < N; r++) {
      int32_t v = order[r];
      hp.proj_ptr[r + 1] = hp.proj_ptr[r] + (inc_ptr[v + 1] - inc_ptr[v]);
    }
    hp.proj_cell.resize(hp.proj_ptr.back());
    hp.proj_w.resize(hp.proj_ptr.back());
    for (int32_t r = 0; r < N; r++) {
      int32_t v = order[r];
      int64_t o = hp.proj_ptr[r];
      for (int64_t e = inc_ptr[v]; e < inc_ptr[v + 1]; e++, o++) {
        int32_t c = inc_idx[e] / 3;
        hp.proj_cell[o] = kept[c];
        hp.proj_w[o] = area[c] / 3.0;
      }
    }
  }
  clock.lap("operator and mass");
  // ---- 4. order-2 and higher products (on the device at upload when products = false)
  if (products) host_products(hp);
  else hp.products_pending = d.max_order >= 2;
  clock.lap("products");
  return hp;
}

}  // namespace ifilt
