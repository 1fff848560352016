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

// C = A B (Gustavson, columns of each row in increasing order)
template <typename VA, typename VB, typename VC>
Csr<VC> multiply(const Csr<VA>& A, const Csr<VB>& B) {
  Csr<VC> C;
  C.n = A.n;
  C.m = B.m;
  C.ptr.assign((size_t)A.n + 1, 0);
  std::vector<int32_t> mark((size_t)B.m, -1);
  std::vector<VC> acc((size_t)B.m);
  std::vector<int32_t> cols;
  for (int32_t i = 0; i < A.n; i++) {
    cols.clear();
    for (int64_t e = A.ptr[i]; e < A.ptr[i + 1]; e++) {
      const int32_t k = A.col[e];
      for (int64_t f = B.ptr[k]; f < B.ptr[k + 1]; f++) {
        const int32_t j = B.col[f];
        if (mark[j] != i) {
          mark[j] = i;
          acc[j] = VC{};
          cols.push_back(j);
        }
        acc[j] += scale(A.val[e], B.val[f]);
      }
    }
    std::sort(cols.begin(), cols.end());
    for (int32_t j : cols) {
      C.col.push_back(j);
      C.val.push_back(acc[j]);
    }
    C.ptr[i + 1] = (int64_t)C.col.size();
  }
  return C;
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

// greedy aggregation on the pattern of A (diagonal ignored)
template <typename V>
std::vector<int32_t> aggregate(const Csr<V>& A, int32_t& n_agg) {
  const int32_t n = A.n;
  std::vector<int32_t> agg((size_t)n, -1);
  int32_t na = 0;
  for (int32_t i = 0; i < n; i++) {
    if (agg[i] >= 0) continue;
    bool free_nb = true;
    for (int64_t e = A.ptr[i]; e < A.ptr[i + 1] && free_nb; e++)
      if (agg[A.col[e]] >= 0) free_nb = false;
    if (!free_nb) continue;
    for (int64_t e = A.ptr[i]; e < A.ptr[i + 1]; e++) agg[A.col[e]] = na;
    agg[i] = na++;
  }
  for (int32_t i = 0; i < n; i++) {
    if (agg[i] >= 0) continue;
    for (int64_t e = A.ptr[i]; e < A.ptr[i + 1]; e++)
      if (A.col[e] != i && agg[A.col[e]] >= 0 && agg[A.col[e]] < na) {
        agg[i] = agg[A.col[e]];
        break;
      }
  }
  // nodes with no aggregated neighbour (e.g. isolated rows) form their own
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
  double lam = 0.0;
  for (int it = 0; it < 40; it++) {
    double nx = 0.0, ny = 0.0;
    for (int32_t i = 0; i < n; i++) {
      V t{};
      for (int64_t e = K.ptr[i]; e < K.ptr[i + 1]; e++) t += K.val[e] * x[K.col[e]];
      y[i] = t * dinv[i];
      nx += std::norm(cplx(x[i]));
      ny += std::norm(cplx(y[i]));
    }
    if (nx == 0.0 || ny == 0.0) return 1.0;
    lam = std::sqrt(ny / nx);
    const double inv = 1.0 / std::sqrt(ny);
    for (int32_t i = 0; i < n; i++) x[i] = y[i] * inv;
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
  for (size_t e = 0; e < a.col.size(); e++) {
    if constexpr (std::is_same<V, cplx>::value) c.val[e] = cplx(a.val[2 * e], a.val[2 * e + 1]);
    else c.val[e] = a.val[e];
  }
  return c;
}

template <typename V>
constexpr int nval_of() {
  return std::is_same<V, cplx>::value ? 2 : 1;
}
template <typename V>
void put(std::vector<double>& out, const V& v) {
  if constexpr (std::is_same<V, cplx>::value) {
    out.push_back(v.real());
    out.push_back(v.imag());
  } else {
    out.push_back(v);
  }
}

template <typename V>
HostCSR to_host(const Csr<V>& c) {
  HostCSR h;
  h.n = c.n;
  h.nval = nval_of<V>();
  h.row_ptr = c.ptr;
  h.col = c.col;
  h.val.reserve(c.val.size() * h.nval);
  for (const V& v : c.val) put(h.val, v);
  return h;
}
template <typename V>
HostCSR to_host(const Csr<Pair<V>>& c) {
  HostCSR h;
  h.n = c.n;
  h.nval = 2 * nval_of<V>();
  h.row_ptr = c.ptr;
  h.col = c.col;
  h.val.reserve(c.val.size() * h.nval);
  for (const auto& v : c.val) {
    put(h.val, v.k);
    put(h.val, v.m);
  }
  return h;
}

template <typename V>
MgHost build(const HostPrepared& hp, const MgParams& prm) {
  MgHost out;
  // level 0: (K, M) with M the lumped mass on the diagonal
  const Csr<V> K0 = from_host<V>(hp.K);
  Csr<Pair<V>> S;
  S.n = S.m = K0.n;
  S.ptr.assign((size_t)K0.n + 1, 0);
  for (int32_t i = 0; i < K0.n; i++) {
    bool has_diag = false;
    for (int64_t e = K0.ptr[i]; e < K0.ptr[i + 1]; e++) has_diag |= K0.col[e] == i;
    bool placed = has_diag;
    for (int64_t e = K0.ptr[i]; e < K0.ptr[i + 1]; e++) {
      if (!placed && K0.col[e] > i) {  // a row without a stored diagonal gets one
        S.col.push_back(i);
        S.val.push_back(Pair<V>{V{}, V(hp.mass[i])});
        placed = true;
      }
      S.col.push_back(K0.col[e]);
      S.val.push_back(Pair<V>{K0.val[e], K0.col[e] == i ? V(hp.mass[i]) : V{}});
    }
    if (!placed) {
      S.col.push_back(i);
      S.val.push_back(Pair<V>{V{}, V(hp.mass[i])});
    }
    S.ptr[i + 1] = (int64_t)S.col.size();
  }
  for (int level = 0;; level++) {
    MgHostLevel L;
    L.n = S.n;
    L.dk.assign((size_t)S.n, 0.0);
    L.dm.assign((size_t)S.n, 0.0);
    for (int32_t i = 0; i < S.n; i++)
      for (int64_t e = S.ptr[i]; e < S.ptr[i + 1]; e++)
        if (S.col[e] == i) {
          L.dk[i] = re(S.val[e].k);
          L.dm[i] = re(S.val[e].m);
        }
    if (level > 0) L.S = to_host(S);
    const bool last = S.n <= prm.coarsest_rows || level + 1 >= prm.max_levels;
    if (!last) {
      // K_l alone, for the aggregation graph and the prolongator smoothing
      Csr<V> K;
      K.n = K.m = S.n;
      K.ptr = S.ptr;
      K.col = S.col;
      K.val.resize(S.val.size());
      for (size_t e = 0; e < S.val.size(); e++) K.val[e] = S.val[e].k;
      int32_t na = 0;
      const std::vector<int32_t> agg = aggregate(K, na);
      if (na > 0 && (double)na <= prm.min_ratio * (double)S.n) {
        std::vector<double> dinv((size_t)S.n, 0.0);
        for (int32_t i = 0; i < S.n; i++) dinv[i] = L.dk[i] > 0.0 ? 1.0 / L.dk[i] : 0.0;
        const double w = (4.0 / 3.0) / lambda_max(K, dinv);
        // P = P_tent - w D^-1 K P_tent, row by row
        Csr<V> P;
        P.n = S.n;
        P.m = na;
        P.ptr.assign((size_t)S.n + 1, 0);
        std::vector<int32_t> mark((size_t)na, -1);
        std::vector<V> acc((size_t)na);
        std::vector<int32_t> cols;
        for (int32_t i = 0; i < S.n; i++) {
          cols.clear();
          auto add = [&](int32_t a, const V& v) {
            if (mark[a] != i) {
              mark[a] = i;
              acc[a] = V{};
              cols.push_back(a);
            }
            acc[a] += v;
          };
          add(agg[i], V(1.0));
          for (int64_t e = K.ptr[i]; e < K.ptr[i + 1]; e++) add(agg[K.col[e]], K.val[e] * (-w * dinv[i]));
          std::sort(cols.begin(), cols.end());
          for (int32_t a : cols)
            if (mag(acc[a]) != 0.0) {
              P.col.push_back(a);
              P.val.push_back(acc[a]);
            }
          P.ptr[i + 1] = (int64_t)P.col.size();
        }
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
