// Smoothed-aggregation multigrid hierarchy for the batched solver's
// preconditioner (host side, built once per mesh; independent of l).
//
// The operators of a column are S = M + s K (real) or S = M + i s K (complex
// form of n = 2); every level keeps the pair (K_l, M_l) on one sparsity
// pattern so that the per-column shift is applied on the device exactly as
// on the finest level.  Construction per level:
//   aggregates   greedy on the graph of K_l: a node whose neighbours are all
//                free roots an aggregate of itself and its neighbours; left
//                nodes join a neighbouring aggregate, isolated ones form their own
//   tentative P  one 1 per row, in the column of the row's aggregate (the
//                near-null space of K is the constant)
//   smoothing    P = (I - w D^-1 K) P_tent, D = diag K, w = 4 / (3 lambda_max(D^-1 K))
//   coarse pair  (K, M)_{l+1} = R (K, M)_l P with R = P^T
// The vertex-vector operator is a matrix of 2x2 blocks [[a, b], [-b, a]];
// such blocks multiply like the complex numbers a + ib and transpose like
// their conjugates, so the same code runs on complex values for it.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdint>
#include <vector>

#include "host_parallel.h"
#include "internal.h"
#include "multigrid.h"

namespace ifilt {
namespace {

using cplx = std::complex<double>;

inline double re(double v) { return v; }
inline double re(const cplx& v) { return v.real(); }
inline double conj_of(double v) { return v; }
inline cplx conj_of(const cplx& v) { return std::conj(v); }
inline double mag(double v) { return std::fabs(v); }
inline double mag(const cplx& v) { return std::abs(v); }

template <typename V>
struct Csr {
  int32_t n = 0, m = 0;  // rows, columns
  std::vector<int64_t> ptr;
  std::vector<int32_t> col;
  std::vector<V> val;
};

// values of a level operator: the l-free part and the mass part
template <typename V>
struct Pair {
  V k{}, m{};
  Pair& operator+=(const Pair& o) {
    k += o.k;
    m += o.m;
    return *this;
  }
};
template <typename V>
Pair<V> scale(const Pair<V>& a, const V& s) {
  return {a.k * s, a.m * s};
}
template <typename V>
Pair<V> scale(const V& s, const Pair<V>& a) {
  return {s * a.k, s * a.m};
}
template <typename V>
V scale(const V& a, const V& s) {
  return a * s;
}

constexpr int64_t kRowChunk = 4096;  // rows per parallel chunk (fixed: results do not depend on threads)

// Builds a CSR row by row, in parallel.  gather(i, cand) appends row i's
// contributions (column, value) in their summation order; each column's
// contributions are summed from zero in that order (a stable sort by column
// keeps it), columns come out ascending, and keep(sum) decides whether the
// entry is stored.  Two passes over the rows: sizes, then contents written in
// place.  When every entry is kept, `columns(i, cols)` (if given) lists row i's
// columns, with repeats, for the first pass without forming the values.
template <typename V, typename Gather, typename Keep, typename Columns>
Csr<V> build_rows(int32_t n, int32_t m, Gather gather, Keep keep, Columns columns) {
  constexpr bool kCountCols = !std::is_same<Columns, std::nullptr_t>::value;
  Csr<V> C;
  C.n = n;
  C.m = m;
  C.ptr.assign((size_t)n + 1, 0);
  using Cand = std::pair<int32_t, V>;
  const int nt = host_threads();
  std::vector<std::vector<Cand>> scratch((size_t)nt);
  std::vector<std::vector<int32_t>> cscratch((size_t)nt);
  auto sorted_row = [&](int32_t i, std::vector<Cand>& c) {
    c.clear();
    gather(i, c);
    stable_sort_small(c.data(), (int64_t)c.size(), [](const Cand& a, const Cand& b) { return a.first < b.first; });
  };
  parallel_range(n, kRowChunk, [&](int64_t b, int64_t e, int w) {
    for (int64_t i = b; i < e; i++) {
      int64_t cnt = 0;
      if constexpr (kCountCols) {
        std::vector<int32_t>& c = cscratch[(size_t)w];
        c.clear();
        columns((int32_t)i, c);
        stable_sort_small(c.data(), (int64_t)c.size(), [](int32_t x, int32_t y) { return x < y; });
        for (size_t t = 0; t < c.size(); t++) cnt += (t == 0 || c[t] != c[t - 1]) ? 1 : 0;
      } else {
        std::vector<Cand>& c = scratch[(size_t)w];
        sorted_row((int32_t)i, c);
        for (size_t t = 0; t < c.size();) {
          const int32_t col = c[t].first;
          V acc{};
          for (; t < c.size() && c[t].first == col; t++) acc += c[t].second;
          cnt += keep(acc) ? 1 : 0;
        }
      }
      C.ptr[i + 1] = cnt;
    }
  });
  for (int32_t i = 0; i < n; i++) C.ptr[i + 1] += C.ptr[i];
  C.col.resize((size_t)C.ptr[n]);
  C.val.resize((size_t)C.ptr[n]);
  parallel_range(n, kRowChunk, [&](int64_t b, int64_t e, int w) {
    std::vector<Cand>& c = scratch[(size_t)w];
    for (int64_t i = b; i < e; i++) {
      sorted_row((int32_t)i, c);
      int64_t o = C.ptr[i];
      for (size_t t = 0; t < c.size();) {
        const int32_t col = c[t].first;
        V acc{};
        for (; t < c.size() && c[t].first == col; t++) acc += c[t].second;
        if (keep(acc)) {
          C.col[o] = col;
          C.val[o] = acc;
          o++;
        }
      }
    }
  });
  return C;
}
template <typename V, typename Gather, typename Keep>
Csr<V> build_rows(int32_t n, int32_t m, Gather gather, Keep keep) {
  return build_rows<V>(n, m, gather, keep, nullptr);
}

// C = A B (Gustavson order: row i of C sums A(i, k) B(k, :) over k ascending;
// every structural entry is kept)
template <typename VA, typename VB, typename VC>
Csr<VC> multiply(const Csr<VA>& A, const Csr<VB>& B) {
  return build_rows<VC>(
      A.n, B.m,
      [&](int32_t i, std::vector<std::pair<int32_t, VC>>& c) {
        for (int64_t e = A.ptr[i]; e < A.ptr[i + 1]; e++) {
          const int32_t k = A.col[e];
          for (int64_t f = B.ptr[k]; f < B.ptr[k + 1]; f++) c.emplace_back(B.col[f], scale(A.val[e], B.val[f]));
        }
      },
      [](const VC&) { return true; },
      [&](int32_t i, std::vector<int32_t>& c) {
        for (int64_t e = A.ptr[i]; e < A.ptr[i + 1]; e++) {
          const int32_t k = A.col[e];
          c.insert(c.end(), B.col.begin() + B.ptr[k], B.col.begin() + B.ptr[k + 1]);
        }
      });
}

// R = P^T with conjugated values
template <typename V>
Csr<V> transpose(const Csr<V>& P) {
  Csr<V> R;
  R.n = P.m;
  R.m = P.n;
  R.ptr.assign((size_t)P.m + 1, 0);
  for (int32_t c : P.col) R.ptr[c + 1]++;
  for (int32_t i = 0; i < P.m; i++) R.ptr[i + 1] += R.ptr[i];
  R.col.resize(P.col.size());
  R.val.resize(P.val.size());
  std::vector<int64_t> fill(R.ptr.begin(), R.ptr.end() - 1);
  for (int32_t i = 0; i < P.n; i++)
    for (int64_t e = P.ptr[i]; e < P.ptr[i + 1]; e++) {
      const int64_t at = fill[P.col[e]]++;
      R.col[at] = i;
      R.val[at] = conj_of(P.val[e]);
    }
  return R;
}

// Greedy aggregation on the pattern of A (diagonal ignored), following only strong
// connections |a_ij| >= theta sqrt(|a_ii a_jj|) (theta = 0: every stored neighbour):
// a node whose strong neighbours are all free roots an aggregate of itself and them;
// left nodes join the aggregate of a strong neighbour; the rest form their own.
template <typename V>
std::vector<int32_t> aggregate(const Csr<V>& A, double theta, int32_t& n_agg) {
  const int32_t n = A.n;
  std::vector<double> d((size_t)n, 0.0);
  if (theta > 0.0)
    for (int32_t i = 0; i < n; i++)
      for (int64_t e = A.ptr[i]; e < A.ptr[i + 1]; e++)
        if (A.col[e] == i) d[i] = mag(A.val[e]);
  auto strong = [&](int32_t i, int64_t e) {
    const int32_t j = A.col[e];
    if (j == i) return false;
    return theta <= 0.0 || mag(A.val[e]) >= theta * std::sqrt(d[i] * d[j]);
  };
  std::vector<int32_t> agg((size_t)n, -1);
  int32_t na = 0;
  for (int32_t i = 0; i < n; i++) {
    if (agg[i] >= 0) continue;
    bool free_nb = true;
    for (int64_t e = A.ptr[i]; e < A.ptr[i + 1] && free_nb; e++)
      if (strong(i, e) && agg[A.col[e]] >= 0) free_nb = false;
    if (!free_nb) continue;
    for (int64_t e = A.ptr[i]; e < A.ptr[i + 1]; e++)
      if (strong(i, e)) agg[A.col[e]] = na;
    agg[i] = na++;
  }
  for (int32_t i = 0; i < n; i++) {
    if (agg[i] >= 0) continue;
    for (int64_t e = A.ptr[i]; e < A.ptr[i + 1]; e++)
      if (strong(i, e) && agg[A.col[e]] >= 0 && agg[A.col[e]] < na) {
        agg[i] = agg[A.col[e]];
        break;
      }
  }
  // nodes with no aggregated strong neighbour (e.g. isolated rows) form their own
  for (int32_t i = 0; i < n; i++)
    if (agg[i] < 0) agg[i] = na++;
  n_agg = na;
  return agg;
}

// largest eigenvalue of D^-1 K by power iteration (D^-1 K is similar to a
// Hermitian positive semidefinite matrix, so the iteration converges to it)
template <typename V>
double lambda_max(const Csr<V>& K, const std::vector<double>& dinv) {
  const int32_t n = K.n;
  std::vector<V> x((size_t)n), y((size_t)n);
  uint64_t s = 0x9E3779B97F4A7C15ull;
  for (int32_t i = 0; i < n; i++) {
    s = s * 6364136223846793005ull + 1442695040888963407ull;
    x[i] = V(0.5 + (double)(s >> 11) * (1.0 / 9007199254740992.0));
  }
  constexpr int64_t kChunk = 16384;
  const int64_t nc = ((int64_t)n + kChunk - 1) / kChunk;
  std::vector<double> px((size_t)nc), py((size_t)nc);
  double lam = 0.0;
  for (int it = 0; it < 40; it++) {
    parallel_range(n, kChunk, [&](int64_t b, int64_t e, int) {
      double sx = 0.0, sy = 0.0;
      for (int64_t i = b; i < e; i++) {
        V t{};
        for (int64_t q = K.ptr[i]; q < K.ptr[i + 1]; q++) t += K.val[q] * x[K.col[q]];
        y[i] = t * dinv[i];
        sx += std::norm(cplx(x[i]));
        sy += std::norm(cplx(y[i]));
      }
      px[(size_t)(b / kChunk)] = sx;
      py[(size_t)(b / kChunk)] = sy;
    });
    double nx = 0.0, ny = 0.0;  // chunk partials added in chunk order
    for (int64_t c = 0; c < nc; c++) {
      nx += px[(size_t)c];
      ny += py[(size_t)c];
    }
    if (nx == 0.0 || ny == 0.0) return 1.0;
    lam = std::sqrt(ny / nx);
    const double inv = 1.0 / std::sqrt(ny);
    parallel_range(n, kChunk, [&](int64_t b, int64_t e, int) {
      for (int64_t i = b; i < e; i++) x[i] = y[i] * inv;
    });
  }
  return lam > 0.0 ? lam : 1.0;
}

template <typename V>
Csr<V> from_host(const HostCSR& a) {
  Csr<V> c;
  c.n = c.m = a.n;
  c.ptr = a.row_ptr;
  c.col = a.col;
  c.val.resize(a.col.size());
  parallel_range((int64_t)a.col.size(), 1 << 20, [&](int64_t b, int64_t e, int) {
    for (int64_t q = b; q < e; q++) {
      if constexpr (std::is_same<V, cplx>::value) c.val[q] = cplx(a.val[2 * q], a.val[2 * q + 1]);
      else c.val[q] = a.val[q];
    }
  });
  return c;
}

template <typename V>
constexpr int nval_of() {
  return std::is_same<V, cplx>::value ? 2 : 1;
}
template <typename V>
void put(double* out, const V& v) {
  if constexpr (std::is_same<V, cplx>::value) {
    out[0] = v.real();
    out[1] = v.imag();
  } else {
    out[0] = v;
  }
}

template <typename V>
HostCSR to_host(const Csr<V>& c) {
  HostCSR h;
  h.n = c.n;
  h.nval = nval_of<V>();
  h.row_ptr = c.ptr;
  h.col = c.col;
  h.val.resize(c.val.size() * h.nval);
  const int nv = h.nval;
  parallel_range((int64_t)c.val.size(), 1 << 20, [&](int64_t b, int64_t e, int) {
    for (int64_t q = b; q < e; q++) put(h.val.data() + q * nv, c.val[q]);
  });
  return h;
}
template <typename V>
HostCSR to_host(const Csr<Pair<V>>& c) {
  HostCSR h;
  h.n = c.n;
  h.nval = 2 * nval_of<V>();
  h.row_ptr = c.ptr;
  h.col = c.col;
  h.val.resize(c.val.size() * h.nval);
  const int nv = h.nval, half = nval_of<V>();
  parallel_range((int64_t)c.val.size(), 1 << 20, [&](int64_t b, int64_t e, int) {
    for (int64_t q = b; q < e; q++) {
      put(h.val.data() + q * nv, c.val[q].k);
      put(h.val.data() + q * nv + half, c.val[q].m);
    }
  });
  return h;
}

template <typename V>
MgHost build(const HostPrepared& hp, const MgParams& prm) {
  MgHost out;
  // level 0: (K, M) with M the lumped mass on the diagonal
  const Csr<V> K0 = from_host<V>(hp.K);
  // (K, M) on K's pattern; a row without a stored diagonal gets one
  Csr<Pair<V>> S = build_rows<Pair<V>>(
      K0.n, K0.n,
      [&](int32_t i, std::vector<std::pair<int32_t, Pair<V>>>& c) {
        bool has_diag = false;
        for (int64_t e = K0.ptr[i]; e < K0.ptr[i + 1]; e++) {
          has_diag |= K0.col[e] == i;
          c.emplace_back(K0.col[e], Pair<V>{K0.val[e], K0.col[e] == i ? V(hp.mass[i]) : V{}});
        }
        if (!has_diag) c.emplace_back(i, Pair<V>{V{}, V(hp.mass[i])});
      },
      [](const Pair<V>&) { return true; });
  for (int level = 0;; level++) {
    MgHostLevel L;
    L.n = S.n;
    L.dk.assign((size_t)S.n, 0.0);
    L.dm.assign((size_t)S.n, 0.0);
    parallel_range(S.n, kRowChunk, [&](int64_t b, int64_t e, int) {
      for (int64_t i = b; i < e; i++)
        for (int64_t q = S.ptr[i]; q < S.ptr[i + 1]; q++)
          if (S.col[q] == i) {
            L.dk[i] = re(S.val[q].k);
            L.dm[i] = re(S.val[q].m);
          }
    });
    if (level > 0) L.S = to_host(S);
    if (level > 0 && prm.strength > 0.0) {
      // smoother weight scaled to this level's pair: the Galerkin mass is not diagonal
      Csr<V> Kl, Ml;
      Kl.n = Kl.m = Ml.n = Ml.m = S.n;
      Kl.ptr = Ml.ptr = S.ptr;
      Kl.col = Ml.col = S.col;
      Kl.val.resize(S.val.size());
      Ml.val.resize(S.val.size());
      for (size_t q = 0; q < S.val.size(); q++) {
        Kl.val[q] = S.val[q].k;
        Ml.val[q] = S.val[q].m;
      }
      std::vector<double> ik((size_t)S.n), im((size_t)S.n);
      for (int32_t i = 0; i < S.n; i++) {
        ik[i] = L.dk[i] > 0.0 ? 1.0 / L.dk[i] : 0.0;
        im[i] = L.dm[i] > 0.0 ? 1.0 / L.dm[i] : 0.0;
      }
      const double lam = std::max(lambda_max(Kl, ik), lambda_max(Ml, im));
      L.omega_s = std::min(2.0 / 3.0, (4.0 / 3.0) / lam);
    }
    const bool last = S.n <= prm.coarsest_rows || level + 1 >= prm.max_levels;
    if (!last) {
      // K_l alone, for the aggregation graph and the prolongator smoothing
      Csr<V> K;
      K.n = K.m = S.n;
      K.ptr = S.ptr;
      K.col = S.col;
      K.val.resize(S.val.size());
      parallel_range((int64_t)S.val.size(), 1 << 20, [&](int64_t b, int64_t e, int) {
        for (int64_t q = b; q < e; q++) K.val[q] = S.val[q].k;
      });
      int32_t na = 0;
      const std::vector<int32_t> agg = aggregate(K, prm.strength, na);
      if (na > 0 && (double)na <= prm.min_ratio * (double)S.n) {
        std::vector<double> dinv((size_t)S.n, 0.0);
        for (int32_t i = 0; i < S.n; i++) dinv[i] = L.dk[i] > 0.0 ? 1.0 / L.dk[i] : 0.0;
        const double w = (4.0 / 3.0) / lambda_max(K, dinv);
        // P = P_tent - w D^-1 K P_tent, row by row; exact zeros are dropped
        const Csr<V> P = build_rows<V>(
            S.n, na,
            [&](int32_t i, std::vector<std::pair<int32_t, V>>& c) {
              c.emplace_back(agg[i], V(1.0));
              for (int64_t e = K.ptr[i]; e < K.ptr[i + 1]; e++)
                c.emplace_back(agg[K.col[e]], K.val[e] * (-w * dinv[i]));
            },
            [](const V& v) { return mag(v) != 0.0; });
        const Csr<V> R = transpose(P);
        const Csr<Pair<V>> SP = multiply<Pair<V>, V, Pair<V>>(S, P);
        Csr<Pair<V>> Sc = multiply<V, Pair<V>, Pair<V>>(R, SP);
        L.P = to_host(P);
        L.R = to_host(R);
        L.omega_p = w;
        out.levels.push_back(std::move(L));
        S = std::move(Sc);
        continue;
      }
    }
    out.levels.push_back(std::move(L));
    break;
  }
  return out;
}

}  // namespace

MgHost build_multigrid(const HostPrepared& h, const MgParams& prm) {
  if (h.placement == IFILT_VERTEX_VECTOR) return build<cplx>(h, prm);
  return build<double>(h, prm);
}

}  // namespace ifilt
