// Batched path: every (field, component, scale) column of a call is solved
// together.  The paper solves one right-hand side per scale (Sect. 2.2.2); here
// the l-free operator is shared by all columns and only the shift differs:
//
//   n = 1 :  S_j = M + c_j K,            c_j = l_j^2 / 2          (Sect. 2.1.1)
//   n = 2 :  S_j = M + c_j K M^-1 K,     c_j = l_j^4 / 2          (real form), or
//            S_j = M + i b_j K,          b_j = l_j^2 / sqrt(2),   phi_l = Re x
//            (complex form: M + 1/2 l^4 K M^-1 K = (M + i b K) M^-1 (M - i b K), and the
//            real part of the first factor's solve is the filtered field)
//
// Vectors live in node-major tiles X[row][sub][lane] (sub = u, v for the
// vertex-vector placement), so one gathered neighbour row feeds every column
// with 16-byte loads.  One CG (or conjugate-orthogonal CG for complex
// symmetric S_j) iteration is five launches:
//   spmm       q = S p,  partial <p, q>           (sliced ELL, FP64 per-column sums)
//   finish_a   alpha = rho / <p, q>               (fixed-order reduction of the partials)
//   update     x += alpha p, r -= alpha q, partial <r, r>, ||r||^2
//   finish_b   beta, convergence mask
//   direction  p = r + beta p
// captured m at a time in a CUDA graph; the host reads the masks between graphs.
// Precision pattern: FP32 (or FP64) matrix and Krylov vectors with FP64 dot
// accumulation; every refinement round recomputes the true residual
// b - S x in FP64 from an FP64 solution and restarts the inner solve on it.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <mutex>
#include <type_traits>
#include <vector>

#include "common.cuh"

namespace ifilt {

int grid_for(const void* kernel, int block, size_t smem, long long work_items) {
  int dev = 0, sms = kNumSMs, occ = 1;
  IFILT_CUDA(cudaGetDevice(&dev));
  IFILT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  IFILT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, block, smem));
  if (occ < 1) fail(IFILT_ECUDA, "kernel cannot be resident with %d threads and %zu bytes of shared memory", block, smem);
  long long g = (long long)sms * occ;
  long long need = (work_items + block - 1) / block;
  if (need < 1) need = 1;
  return (int)std::min(g, need);
}

namespace {

constexpr int kBlock = 256;

template <typename T>
struct alignas(16) Pack {
  static constexpr int N = 16 / sizeof(T);
  T v[N];
};

template <typename T>
__device__ __forceinline__ Pack<T> ldp(const T* p) {
  Pack<T> r;
  *reinterpret_cast<uint4*>(&r) = __ldg(reinterpret_cast<const uint4*>(p));
  return r;
}
template <typename T>
__device__ __forceinline__ Pack<T> ldv(const T* p) {  // plain load (data written by this kernel's stream)
  Pack<T> r;
  *reinterpret_cast<uint4*>(&r) = *reinterpret_cast<const uint4*>(p);
  return r;
}
template <typename T>
__device__ __forceinline__ void stp(T* p, const Pack<T>& v) {
  *reinterpret_cast<uint4*>(p) = *reinterpret_cast<const uint4*>(&v);
}

// Fused multiply-add in the precision of T.  (A bare fma() on floats can bind
// to the double overload and run on the FP64 pipe.)
__device__ __forceinline__ float madd(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double madd(double a, double b, double c) { return __fma_rn(a, b, c); }

// Per-thread dot-product accumulator.  For FP32 vectors the FP64 unit of
// GB300 is far too slow to take one operation per element, so partial sums
// are carried as an unevaluated pair (s, c) on the FP32 pipes: each product
// a*b is split exactly into p + e by an FMA, p is added to s with a two-sum,
// and every rounding error goes into c (the compensated dot product of Ogita,
// Rump and Oishi, 2005).  Its error is about u|sum| + (m u)^2 sum|terms| for a
// chain of m terms, so chains are kept short: `flush` moves the pair into an
// FP64 sum every few rows, which costs one FP64 add per lane and flush.
// Explicit _rn intrinsics keep the compiler from contracting the error terms.
template <typename T>
struct DotAcc {
  double d = 0.0;
  __device__ __forceinline__ void add(T a, T b) { d = __fma_rn((double)a, (double)b, d); }
  __device__ __forceinline__ void add_sum(T x) { d += (double)x; }
  __device__ __forceinline__ void flush() {}
  __device__ __forceinline__ void spill(double& slot) {
    slot += d;
    d = 0.0;
  }
  __device__ __forceinline__ double get() const { return d; }
};
template <>
struct DotAcc<float> {
  float s = 0.f, c = 0.f;
  double d = 0.0;
  __device__ __forceinline__ void add(float a, float b) {
    const float p = __fmul_rn(a, b);
    const float e = __fmaf_rn(a, b, -p);
    const float t = __fadd_rn(s, p);
    const float z = __fsub_rn(t, s);
    const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));
    s = t;
    c = __fadd_rn(c, __fadd_rn(err, e));
  }
  // x is a row's few terms already summed in FP32: a two-sum only
  __device__ __forceinline__ void add_sum(float x) {
    const float t = __fadd_rn(s, x);
    const float z = __fsub_rn(t, s);
    c = __fadd_rn(c, __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(x, z)));
    s = t;
  }
  __device__ __forceinline__ void flush() {
    d += (double)s + (double)c;
    s = 0.f;
    c = 0.f;
  }
  // flush into an FP64 slot kept elsewhere (shared memory), freeing d's registers
  __device__ __forceinline__ void spill(double& slot) {
    slot += (double)s + (double)c;
    s = 0.f;
    c = 0.f;
  }
  __device__ __forceinline__ double get() const { return d + ((double)s + (double)c); }
};
constexpr int kFlushRows = 64;  // rows per compensated chain

// Jacobi step z = D^-1 r on VEC lanes of one row, D the diagonal of the
// shifted operator: m + s g for real columns, m + i s g for complex ones
// (lanes in (re, im) pairs); m, g the row's mass and diagonal of G.
template <typename T, bool CPLX, int VEC>
__device__ __forceinline__ void jacobi(T m, T g, const T* sh, const T* rv, T* z) {
  if constexpr (CPLX) {
#pragma unroll
    for (int v = 0; v < VEC; v += 2) {
      const T bg = sh[v] * g;
      const T inv = (T)1 / madd(m, m, bg * bg);
      z[v] = madd(rv[v], m, rv[v + 1] * bg) * inv;
      z[v + 1] = madd(rv[v + 1], m, -(rv[v] * bg)) * inv;
    }
  } else {
#pragma unroll
    for (int v = 0; v < VEC; v++) z[v] = rv[v] / madd(sh[v], g, m);
  }
}

// The multigrid smoother's damped-Jacobi step: the same z = D^-1 r, with the
// reciprocal of each diagonal entry taken by the fast hardware approximation
// in single precision (a relative error of a few ulp).  The smoother only has
// to be one fixed diagonal operator, applied alike before and after the coarse
// correction (which keeps the V-cycle symmetric); an IEEE division per lane was
// a large share of the sweep's instructions.  The Jacobi preconditioner of the
// Krylov solve keeps the exact division (jacobi above).
template <typename T, bool CPLX, int VEC>
__device__ __forceinline__ void smooth_jacobi(T m, T g, const T* sh, const T* rv, T* z) {
  if constexpr (sizeof(T) == 4) {
    if constexpr (CPLX) {
#pragma unroll
      for (int v = 0; v < VEC; v += 2) {
        const T bg = sh[v] * g;
        const T inv = __fdividef(1.0f, madd(m, m, bg * bg));
        z[v] = madd(rv[v], m, rv[v + 1] * bg) * inv;
        z[v + 1] = madd(rv[v + 1], m, -(rv[v] * bg)) * inv;
      }
    } else {
#pragma unroll
      for (int v = 0; v < VEC; v++) z[v] = rv[v] * __fdividef(1.0f, madd(sh[v], g, m));
    }
  } else {
    jacobi<T, CPLX, VEC>(m, g, sh, rv, z);
  }
}

// 4 consecutive ELL entries' values (NV per entry) converted to AT.
template <typename MV, int NV, typename AT>
__device__ __forceinline__ void load_vals(const MV* __restrict__ p, AT* out) {
  if constexpr (sizeof(MV) * 4 * NV == 8) {
    uint2 u = __ldg(reinterpret_cast<const uint2*>(p));
    const MV* m = reinterpret_cast<const MV*>(&u);
#pragma unroll
    for (int t = 0; t < 4 * NV; t++) out[t] = (AT)to_f(m[t]);
  } else {
    constexpr int CH = sizeof(MV) * 4 * NV / 16;
#pragma unroll
    for (int c = 0; c < CH; c++) {
      uint4 u = __ldg(reinterpret_cast<const uint4*>(p) + c);
      const MV* m = reinterpret_cast<const MV*>(&u);
#pragma unroll
      for (int t = 0; t < 16 / (int)sizeof(MV); t++) {
        if constexpr (sizeof(MV) == 2) out[c * 8 + t] = (AT)to_f(m[t]);
        else out[c * (16 / sizeof(MV)) + t] = (AT)m[t];
      }
    }
  }
}

// Per-column solver state (device arrays, one entry per column unless noted).
struct Cols {
  double* shift;    // c_j (real) or b_j (complex)
  double* rho;      // [2n] <r, r> (re, im)
  double* alpha;    // [2n]
  double* beta;     // [2n]
  double* rn2;      // ||r||^2 of the inner recursion
  double* target2;  // inner stop threshold on ||r||^2
  double* r0n2;     // ||b - S x0||^2 (FP64), < 0 until the first residual round
  double* tol2;     // tol^2 * r0n2
  double* rel;      // last true relative residual
  double* err;      // last certified relative error bound ||r||_{M^-1} / ||x||_M
  int* active;      // inner recursion running
  int* done;        // column finished (converged, capped or broken down)
  int* iters;
  int* rounds;
  int* status;      // 0 ok, 1 not converged, 2 breakdown
  int* refresh;     // column waits for its FP64 true residual / next refinement round
  int* round_it0;   // iteration count when the current inner round started
  int* round_cap;   // iterations allowed in the current inner round
  int* restart;     // multigrid: the next direction restarts (beta = 0)
  int* live;        // [4] number of active columns, columns to refresh, columns not done; device error flag
};

struct Params {
  int32_t n;        // rows
  int W;            // lanes per sub-row
  int ncols;        // columns (incl. padding)
  int pstride;      // doubles per block in `partial`
  int maxit;
  double tol2_rel;  // tol^2
  double err2;      // err_tol^2 (0: no error test)
  double inner2;    // inner_tol^2 (0: run to the outer tolerance)
  int mg;           // multigrid-preconditioned iteration order
  int spt;          // ELL slices per SpMM tile
  int wmax;         // widest ELL slice
  int stage_e;      // ELL entries one SpMM stage buffer holds
  int rn_slot;      // real columns: ||r||^2 has slots of its own in the update partials (Jacobi)
};

// ------------------------------------------------------------------ kernels

template <typename T, typename MV>
__device__ __forceinline__ T cvt(MV v) {
  if constexpr (sizeof(MV) == 2) return (T)__bfloat162float(v);
  else return (T)v;
}

// Epilogues of the gather kernel.  CG: q = M p + s (G p) with <p, q>.  The
// multigrid operations on a level operator S = M + s K (M the lumped mass on
// the finest level, a sparse matrix on the coarser ones):
//   SMOOTH    out = x + w D^-1 (rhs - S x)   (damped Jacobi; optionally <rhs, out>)
//   RESID     out = rhs - S x
//   RESTRICT  out = R t                      (gather of the finer level)
//   PROLONG   out = y + P x_c                (gather of the coarser level)
constexpr int kEpiCG = 0, kEpiSmooth = 1, kEpiResid = 2, kEpiRestrict = 3, kEpiProlong = 4;

template <typename T, typename TR, typename TS>
struct MgArgs {
  const T* dk;    // diagonal of K_l (SMOOTH)
  const TR* rhs;  // right-hand side of the level (SMOOTH, RESID)
  const TS* own;  // y of PROLONG
  T omega;        // Jacobi weight (SMOOTH)
};



// VEC lanes of a vector stored as TS (FP64 or FP32), moved as one load or store
// of VEC * sizeof(TS) bytes (16 or 32) and converted to or from the arithmetic
// type T.
template <typename TS, int VEC>
struct Lanes {
  static constexpr int B = VEC * (int)sizeof(TS);
  static_assert(B == 16 || B == 32, "a lane group moves 16 or 32 bytes");
  uint32_t w[B / 4];
};
template <bool NC, typename TS, int VEC>
__device__ __forceinline__ Lanes<TS, VEC> lanes_ld(const TS* p) {
  Lanes<TS, VEC> r;
#pragma unroll
  for (int c = 0; c < Lanes<TS, VEC>::B / 16; c++) {
    const uint4 u = NC ? __ldg(reinterpret_cast<const uint4*>(p) + c) : reinterpret_cast<const uint4*>(p)[c];
    r.w[4 * c] = u.x, r.w[4 * c + 1] = u.y, r.w[4 * c + 2] = u.z, r.w[4 * c + 3] = u.w;
  }
  return r;
}
template <typename TS, int VEC>
__device__ __forceinline__ void lanes_st(TS* p, const Lanes<TS, VEC>& r) {
#pragma unroll
  for (int c = 0; c < Lanes<TS, VEC>::B / 16; c++)
    reinterpret_cast<uint4*>(p)[c] = make_uint4(r.w[4 * c], r.w[4 * c + 1], r.w[4 * c + 2], r.w[4 * c + 3]);
}
template <typename T, typename TS, int VEC>
__device__ __forceinline__ void lanes_get(const Lanes<TS, VEC>& r, T* v) {
  if constexpr (sizeof(TS) == 4) {
#pragma unroll
    for (int i = 0; i < VEC; i++) v[i] = (T)__uint_as_float(r.w[i]);
  } else {
#pragma unroll
    for (int i = 0; i < VEC; i++) v[i] = (T)__hiloint2double((int)r.w[2 * i + 1], (int)r.w[2 * i]);
  }
}
template <typename T, typename TS, int VEC>
__device__ __forceinline__ Lanes<TS, VEC> lanes_put(const T* v) {
  Lanes<TS, VEC> r;
  if constexpr (sizeof(TS) == 4) {
#pragma unroll
    for (int i = 0; i < VEC; i++) r.w[i] = __float_as_uint((float)v[i]);
  } else {
#pragma unroll
    for (int i = 0; i < VEC; i++) {
      r.w[2 * i] = (uint32_t)__double2loint((double)v[i]);
      r.w[2 * i + 1] = (uint32_t)__double2hiint((double)v[i]);
    }
  }
  return r;
}

// q = M p + shift * acc for one row (all sub-rows), and the row's share of
// <p, q>: the row's few terms are summed in FP32, then added to the
// compensated per-thread accumulator.
template <typename T, typename TS, int VEC, bool CPLX, bool BLK>
__device__ __forceinline__ void spmm_epilogue(int64_t r, int64_t rowW, int W, int l0, const T mr,
                                              const T* sh, T (*acc)[VEC], T (*pr)[VEC],
                                              TS* __restrict__ q, DotAcc<T>* dacc) {
  constexpr int NS = BLK ? 2 : 1;
  T rowdot[VEC];
#pragma unroll
  for (int v = 0; v < VEC; v++) rowdot[v] = (T)0;
#pragma unroll
  for (int b = 0; b < NS; b++) {
    const int64_t off = r * rowW + (int64_t)b * W + l0;
    T qo[VEC];
    if constexpr (CPLX) {
#pragma unroll
      for (int v = 0; v < VEC; v += 2) {
        const T pre = pr[b][v], pim = pr[b][v + 1];
        const T qre = mr * pre - sh[v] * acc[b][v + 1];
        const T qim = mr * pim + sh[v] * acc[b][v];
        qo[v] = qre;
        qo[v + 1] = qim;
        rowdot[v] = madd(pre, qre, madd(-pim, qim, rowdot[v]));
        rowdot[v + 1] = madd(pre, qim, madd(pim, qre, rowdot[v + 1]));
      }
    } else {
#pragma unroll
      for (int v = 0; v < VEC; v++) {
        const T qv = mr * pr[b][v] + sh[v] * acc[b][v];
        qo[v] = qv;
        if constexpr (NS == 1) dacc[v].add(pr[b][v], qv);  // a single exact product
        else rowdot[v] = madd(pr[b][v], qv, rowdot[v]);
      }
    }
    lanes_st<TS, VEC>(q + off, lanes_put<T, TS, VEC>(qo));
  }
  if constexpr (CPLX || NS > 1) {
#pragma unroll
    for (int v = 0; v < VEC; v++) dacc[v].add_sum(rowdot[v]);
  }
}

// Multigrid epilogue for one row: acc holds the K part of the gather (or the
// whole gather for RESTRICT / PROLONG), accm the M part on coarse levels
// (NSET = 2); own is x_r (SMOOTH, RESID) or y_r (PROLONG); mdiag is the
// diagonal of M_l (the lumped mass on the finest level).
template <typename T, typename TS, int VEC, bool CPLX, bool BLK, int EPI, int NSET>
__device__ __forceinline__ void mg_epilogue(int64_t r, int64_t rowW, int W, int l0, const T mr, const T gr,
                                            T (*rh)[VEC], const T* sh, T (*acc)[VEC], T (*accm)[VEC],
                                            T (*own)[VEC], const T omega, TS* __restrict__ out, DotAcc<T>* dacc,
                                            bool dot) {
  constexpr int NS = BLK ? 2 : 1;
  T rowdot[VEC];
#pragma unroll
  for (int v = 0; v < VEC; v++) rowdot[v] = (T)0;
#pragma unroll
  for (int b = 0; b < NS; b++) {
    const int64_t off = r * rowW + (int64_t)b * W + l0;
    T o[VEC];
    if constexpr (EPI == kEpiRestrict) {
#pragma unroll
      for (int v = 0; v < VEC; v++) o[v] = acc[b][v];
    } else if constexpr (EPI == kEpiProlong) {
#pragma unroll
      for (int v = 0; v < VEC; v++) o[v] = own[b][v] + acc[b][v];
    } else {
      T res[VEC];
#pragma unroll
      for (int v = 0; v < VEC; v++) {
        const T mx = NSET == 2 ? accm[b][v] : mr * own[b][v];
        T sx;
        if constexpr (CPLX) sx = (v & 1) ? mx + sh[v] * acc[b][v - 1] : mx - sh[v] * acc[b][v + 1];
        else sx = madd(sh[v], acc[b][v], mx);
        res[v] = rh[b][v] - sx;
      }
      if constexpr (EPI == kEpiResid) {
#pragma unroll
        for (int v = 0; v < VEC; v++) o[v] = res[v];
      } else {
        T z[VEC];
        smooth_jacobi<T, CPLX, VEC>(mr, gr, sh, res, z);
#pragma unroll
        for (int v = 0; v < VEC; v++) o[v] = madd(omega, z[v], own[b][v]);
        if (dot) {
          if constexpr (CPLX) {
#pragma unroll
            for (int v = 0; v < VEC; v += 2) {
              rowdot[v] = madd(rh[b][v], o[v], madd(-rh[b][v + 1], o[v + 1], rowdot[v]));
              rowdot[v + 1] = madd(rh[b][v], o[v + 1], madd(rh[b][v + 1], o[v], rowdot[v + 1]));
            }
          } else {
#pragma unroll
            for (int v = 0; v < VEC; v++) rowdot[v] = madd(rh[b][v], o[v], rowdot[v]);
          }
        }
      }
    }
    lanes_st<TS, VEC>(out + off, lanes_put<T, TS, VEC>(o));
  }
  if constexpr (EPI == kEpiSmooth) {
    if (dot) {
#pragma unroll
      for (int v = 0; v < VEC; v++) dacc[v].add_sum(rowdot[v]);
    }
  }
}

#ifndef IFILT_SPMM_MINB_BLK
#define IFILT_SPMM_MINB_BLK 3  // resident blocks per SM asked of the compiler for 2x2-block FP32 SpMM
#endif
#ifndef IFILT_SPMM_MINB
#define IFILT_SPMM_MINB 3      // resident blocks per SM asked of the compiler for the other SpMM instances
#endif
#ifndef IFILT_MG_MINB_BLK
#define IFILT_MG_MINB_BLK 2    // resident blocks per SM asked for the 2x2-block multigrid sweeps and residuals
#endif
#ifndef IFILT_MG_EB_COARSE
#define IFILT_MG_EB_COARSE 4     // gathered entries in flight per row on the Galerkin levels (scalar rows)
#endif
#ifndef IFILT_MG_MINB_XFER
#define IFILT_MG_MINB_XFER 4     // resident blocks per SM asked for the scalar-row restrictions and prolongations
#endif
#ifndef IFILT_MG_MINB_CRESID
#define IFILT_MG_MINB_CRESID 3   // ... for the coarse levels' residuals (scalar rows; 4 was slower)
#endif
#ifndef IFILT_MG_MINB_CSMOOTH
#define IFILT_MG_MINB_CSMOOTH 3  // ... for the coarse levels' sweeps (scalar rows; 4 spills and was slower)
#endif
#ifndef IFILT_SPMM_EB_BLK
#define IFILT_SPMM_EB_BLK 4    // gathered entries in flight per row for 2x2-block FP32 SpMM
#endif
constexpr int kMaxSpt = 64;            // sliced-ELL slices staged per tile
constexpr int kStageBytes = 24 * 1024;  // one of the two stage buffers, when it holds several slices
constexpr int kStageMax = 96 * 1024;    // one of the two stage buffers holding a single slice
constexpr int kTilePasses = 8;          // rows per tile ~ this many passes of the block's row groups

// Bulk (TMA engine) copies of a tile's ELL entries into shared memory,
// completed on an mbarrier.  Both addresses and the size are multiples of 16
// bytes: slices start on 8-entry boundaries and hold a multiple of 4 entries
// per row, and the buffers are 16-byte aligned.
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void async_proxy_fence() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_to_smem(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for phase `parity` of `bar` for at most ~1 s of SM clock; false on expiry.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_test(bar, parity))
    if (clock64() - t0 > 2000000000LL) return false;
  return true;
}

// q = M p + shift * (G p) for every lane, with the per-block partials of <p, q>
// (or a multigrid operation, EPI).  Work is cut into tiles of `spt` ELL slices.
// A tile's column indices and values are bulk-copied into one of two
// shared-memory buffers while the block works on the previous tile, so a row
// waits on one round of global loads: its own row of p and all gathered
// neighbour rows (EB entries at a time) are issued before any of them is used.
// Vectors are stored as TS (the right-hand side of a multigrid level as TRS,
// the output as TO) and computed in T; a thread owns VEC consecutive lanes of
// a row.
template <typename T, typename MV, typename TS, typename TRS, typename TO, int VEC, bool CPLX, bool BLK, int EB,
          int MINB, int EPI = kEpiCG, int NSET = 1>
__global__ void __launch_bounds__(kBlock, MINB) spmm_kernel(EllView<MV> A, Params P, int n_slices, const TS* __restrict__ p,
                                                         TO* __restrict__ q, const T* __restrict__ mass,
                                                         Cols C, double* __restrict__ partial, MgArgs<T, TRS, TS> mg) {
  if (*C.live == 0) return;
  constexpr int NS = BLK ? 2 : 1;
  constexpr int NV = (BLK ? 2 : 1) * NSET;  // values per ELL entry
  constexpr int NB = BLK ? 2 : 1;           // values of one operator per entry
  const bool dot = EPI == kEpiCG || (EPI == kEpiSmooth && partial != nullptr);
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ int s_w[2][kMaxSpt], s_o[2][kMaxSpt];
  __shared__ __align__(8) uint64_t bar[2];
  const int W = P.W;
  const int TPR = W / VEC;
  const int RPP = kBlock / TPR;
  const int H = A.slice_h;
  const int spt = P.spt;
  const int TR = spt * H;
  double* sred = reinterpret_cast<double*>(smraw);
  const size_t colb = ((size_t)P.stage_e * 4 + 15) / 16 * 16;
  const size_t valb = ((size_t)P.stage_e * NV * sizeof(MV) + 15) / 16 * 16;
  // row lengths (A.rowq) only where rows are uneven: the Galerkin levels' (K, M) pairs and
  // the restrictions; the other instances run every row to its slice's width
  constexpr bool kRowq = NSET == 2 || EPI == kEpiRestrict;
  const size_t qb = kRowq ? ((size_t)P.spt * A.slice_h + 15) / 16 * 16 : 0;
  unsigned char* const sbase = smraw + (size_t)RPP * W * sizeof(double);
  auto stage_col = [&](int b) { return reinterpret_cast<int*>(sbase + b * (colb + valb + qb)); };
  auto stage_val = [&](int b) { return reinterpret_cast<MV*>(sbase + b * (colb + valb + qb) + colb); };
  auto stage_q = [&](int b) { return reinterpret_cast<const uint8_t*>(sbase + b * (colb + valb + qb) + colb + valb); };
  const int tr = threadIdx.x / TPR, g = threadIdx.x - tr * TPR;
  const int l0 = g * VEC;
  const bool on = tr < RPP && tr < TR;
  const int ntiles = (n_slices + spt - 1) / spt;
  if (on) {
#pragma unroll
    for (int v = 0; v < VEC; v++) sred[tr * W + l0 + v] = 0.0;  // FP64 dot slots, one per thread and lane
  }

  auto issue = [&](int tile, int b) {  // one thread
    const int s0 = tile * spt, s1 = min(s0 + spt, n_slices);
    const int64_t ob = A.slice_off[s0], oe = A.slice_off[s1];
    const uint32_t ne = (uint32_t)(oe - ob);
    const uint32_t bc = ne * 4u, bv = ne * (uint32_t)(NV * sizeof(MV));
    // row lengths: whole slices of the per-row array (allocated for every slice's rows,
    // so a multiple of 64 bytes from a 64-byte boundary)
    const uint32_t bq = kRowq && A.rowq ? (uint32_t)((s1 - s0) * A.slice_h) : 0u;
    async_proxy_fence();  // earlier generic reads of the buffer come first
    mbar_expect(&bar[b], bc + bv + bq);  // with no bytes the phase completes here
    if (ne > 0) {
      bulk_to_smem(stage_col(b), A.col + ob, bc, &bar[b]);
      bulk_to_smem(stage_val(b), A.val + ob * NV, bv, &bar[b]);
    }
    if (bq > 0) bulk_to_smem(const_cast<uint8_t*>(stage_q(b)), A.rowq + (int64_t)s0 * A.slice_h, bq, &bar[b]);
  };
  if (threadIdx.x == 0) {
    mbar_init(&bar[0]);
    mbar_init(&bar[1]);
    async_proxy_fence();
  }
  __syncthreads();
  if ((int)blockIdx.x < ntiles) {
    const int s0 = blockIdx.x * spt, cnt = min(s0 + spt, n_slices) - s0;
    if (threadIdx.x == 0) issue(blockIdx.x, 0);
    if ((int)threadIdx.x < cnt) {
      s_w[0][threadIdx.x] = A.slice_w[s0 + threadIdx.x];
      s_o[0][threadIdx.x] = (int)(A.slice_off[s0 + threadIdx.x] - A.slice_off[s0]);
    }
  }
  __syncthreads();

  DotAcc<T> dacc[VEC];
  T sh[VEC];
#pragma unroll
  for (int v = 0; v < VEC; v++) sh[v] = on ? (T)C.shift[CPLX ? (l0 + v) >> 1 : l0 + v] : (T)0;
  const int64_t rowW = (int64_t)NS * W;
  int chain = 0;
  unsigned inflight = (int)blockIdx.x < ntiles ? 1u : 0u;  // bit b: a copy into buffer b is outstanding
  int it = 0;
  bool failed = false;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, it++) {
    const int b = it & 1;
    const int next = tile + gridDim.x;
    int nw = 0, no = 0, ncnt = 0;
    if (next < ntiles) {
      if (threadIdx.x == 0) issue(next, b ^ 1);
      inflight |= 1u << (b ^ 1);
      const int s0 = next * spt;
      ncnt = min(s0 + spt, n_slices) - s0;
      if ((int)threadIdx.x < ncnt) {  // consumed after this tile's rows
        nw = A.slice_w[s0 + threadIdx.x];
        no = (int)(A.slice_off[s0 + threadIdx.x] - A.slice_off[s0]);
      }
    }
    bool late = false;
    if (threadIdx.x == 0) late = !mbar_wait_bounded(&bar[b], (uint32_t)((it >> 1) & 1));
    if (__syncthreads_or(late)) {
      failed = true;
      break;
    }
    inflight &= ~(1u << b);
    const int* scol = stage_col(b);
    const MV* sval = stage_val(b);
    const int64_t r0 = (int64_t)tile * spt * H;
    const int rows = (int)min((int64_t)TR, (int64_t)P.n - r0);

    if (on) {
      for (int lr = tr; lr < rows; lr += RPP) {
        const int64_t r = r0 + lr;
        const int sl = lr / H;
        const int w = s_w[b][sl];
        const int eb = s_o[b][sl] + (lr - sl * H) * w;
        // the row's own length (a multiple of 4 entries, at most the slice's width), staged
        // with the tile: the slice's padding past it is skipped
        int rq = 255;
        if constexpr (kRowq) {
          if (A.rowq) rq = (int)stage_q(b)[lr];
        }
        const int wr = (kRowq && rq != 255) ? min(w, 4 * rq) : w;
        Lanes<TS, VEC> pr[NS];
        if constexpr (EPI == kEpiProlong) {
#pragma unroll
          for (int s = 0; s < NS; s++) pr[s] = lanes_ld<false, TS, VEC>(mg.own + r * rowW + (int64_t)s * W + l0);
        } else if constexpr (EPI != kEpiRestrict) {
#pragma unroll
          for (int s = 0; s < NS; s++) pr[s] = lanes_ld<true, TS, VEC>(p + r * rowW + (int64_t)s * W + l0);
        }
        // the row's own operands are loaded with its gathers: one round of global loads per row
        T mrow = (T)0, grow = (T)0;
        Lanes<TRS, VEC> rrow[NS];
        if constexpr (EPI == kEpiCG || EPI == kEpiSmooth || EPI == kEpiResid) mrow = mass[r];
        if constexpr (EPI == kEpiSmooth) grow = mg.dk[r];
        if constexpr (EPI == kEpiSmooth || EPI == kEpiResid) {
#pragma unroll
          for (int s = 0; s < NS; s++) rrow[s] = lanes_ld<false, TRS, VEC>(mg.rhs + r * rowW + (int64_t)s * W + l0);
        }
        T acc[NS][VEC], accm[NS][VEC];
#pragma unroll
        for (int s = 0; s < NS; s++)
#pragma unroll
          for (int v = 0; v < VEC; v++) acc[s][v] = accm[s][v] = (T)0;
        // EB entries at a time (a multiple of 4 entries, or 2 for a 2-entry batch:
        // rows hold a multiple of 4 entries, so a batch never runs past the row)
        for (int e = 0; e < w; e += EB) {
          if constexpr (kRowq) {
            if (e > 0 && e >= wr) break;
          }
          Lanes<TS, VEC> nb[EB][NS];
#pragma unroll
          for (int h = 0; h < EB; h += 4) {
            if (h == 0 || e + h < wr) {
              int cc[4];
              if constexpr (EB >= 4) {
                const int4 c4 = *reinterpret_cast<const int4*>(scol + eb + e + h);
                cc[0] = c4.x, cc[1] = c4.y, cc[2] = c4.z, cc[3] = c4.w;
              } else {
                const int2 c2 = *reinterpret_cast<const int2*>(scol + eb + e);
                cc[0] = c2.x, cc[1] = c2.y, cc[2] = cc[3] = 0;
              }
#pragma unroll
              for (int t = 0; t < (EB >= 4 ? 4 : EB); t++)
#pragma unroll
                for (int s = 0; s < NS; s++)
                  nb[h + t][s] = lanes_ld<true, TS, VEC>(p + (int64_t)cc[t] * rowW + (int64_t)s * W + l0);
            }
          }
#pragma unroll
          for (int h = 0; h < EB; h += 4) {
            if (h == 0 || e + h < wr) {
              const MV* vv = sval + (size_t)(eb + e + h) * NV;
#pragma unroll
              for (int t = 0; t < (EB >= 4 ? 4 : EB); t++) {
                T xu[VEC], xw[VEC];
                lanes_get<T, TS, VEC>(nb[h + t][0], xu);
                if constexpr (BLK) {
                  lanes_get<T, TS, VEC>(nb[h + t][1], xw);
                  const T a = cvt<T>(vv[NV * t]), bb = cvt<T>(vv[NV * t + 1]);
#pragma unroll
                  for (int v = 0; v < VEC; v++) {
                    acc[0][v] = madd(a, xu[v], madd(bb, xw[v], acc[0][v]));
                    acc[1][v] = madd(a, xw[v], madd(-bb, xu[v], acc[1][v]));
                  }
                  if constexpr (NSET == 2) {
                    const T am = cvt<T>(vv[NV * t + NB]), bm = cvt<T>(vv[NV * t + NB + 1]);
#pragma unroll
                    for (int v = 0; v < VEC; v++) {
                      accm[0][v] = madd(am, xu[v], madd(bm, xw[v], accm[0][v]));
                      accm[1][v] = madd(am, xw[v], madd(-bm, xu[v], accm[1][v]));
                    }
                  }
                } else {
                  const T a = cvt<T>(vv[NV * t]);
#pragma unroll
                  for (int v = 0; v < VEC; v++) acc[0][v] = madd(a, xu[v], acc[0][v]);
                  if constexpr (NSET == 2) {
                    const T am = cvt<T>(vv[NV * t + NB]);
#pragma unroll
                    for (int v = 0; v < VEC; v++) accm[0][v] = madd(am, xu[v], accm[0][v]);
                  }
                }
              }
            }
          }
        }
        if (++chain == kFlushRows) {
          chain = 0;
          if (dot) {
#pragma unroll
            for (int v = 0; v < VEC; v++) dacc[v].spill(sred[tr * W + l0 + v]);
          }
        }
        T own[NS][VEC], rh[NS][VEC];
        if constexpr (EPI != kEpiRestrict) {
#pragma unroll
          for (int s = 0; s < NS; s++) lanes_get<T, TS, VEC>(pr[s], own[s]);
        }
        if constexpr (EPI == kEpiSmooth || EPI == kEpiResid) {
#pragma unroll
          for (int s = 0; s < NS; s++) lanes_get<T, TRS, VEC>(rrow[s], rh[s]);
        }
        if constexpr (EPI == kEpiCG) spmm_epilogue<T, TO, VEC, CPLX, BLK>(r, rowW, W, l0, mrow, sh, acc, own, q, dacc);
        else
          mg_epilogue<T, TO, VEC, CPLX, BLK, EPI, NSET>(r, rowW, W, l0, mrow, grow, rh, sh, acc, accm, own, mg.omega,
                                                         q, dacc, dot);
      }
    }
    if ((int)threadIdx.x < ncnt) {
      s_w[b ^ 1][threadIdx.x] = nw;
      s_o[b ^ 1][threadIdx.x] = no;
    }
    __syncthreads();  // the buffer is free for the tile after next; the next tile's layout is visible
  }
  if (failed) {
    // leave no bulk copy writing into this block's shared memory after it exits
    if (threadIdx.x == 0) {
      const int b0 = it & 1, b1 = b0 ^ 1;
      if (inflight & (1u << b0)) (void)mbar_wait_bounded(&bar[b0], (uint32_t)((it >> 1) & 1));
      if (inflight & (1u << b1)) (void)mbar_wait_bounded(&bar[b1], (uint32_t)(((it + 1) >> 1) & 1));
      atomicExch(C.live + 3, 1);
    }
    return;
  }
  if (!dot) return;
  if (on) {
#pragma unroll
    for (int v = 0; v < VEC; v++) dacc[v].spill(sred[tr * W + l0 + v]);
  }
  __syncthreads();
  const int rg = min(RPP, TR);
  for (int l = threadIdx.x; l < W; l += kBlock) {
    double s = 0.0;
    for (int t = 0; t < rg; t++) s += sred[t * W + l];
    partial[(int64_t)blockIdx.x * P.pstride + l] = s;
  }
}

// x += alpha p ; r -= alpha q ; partial <r, z> (slots [0, W): lane-wise for real,
// (re, im) pairs for complex; z = r, or D^-1 r under Jacobi preconditioning)
// and ||r||^2 (slots W + column) where <r, z> is not it: complex columns, and
// real columns under Jacobi preconditioning.  With MGJ it also writes the
// multigrid's first fine-level sweep for the next iteration, zj = omega D^-1 r
// (D = mass + shift * K diagonal, gdiag), as mg_jacobi_kernel would from the
// stored r: one pass over r fewer per iteration.
template <typename T, bool CPLX, bool BLK, bool PRE, bool MGJ = false>
__global__ void __launch_bounds__(kBlock, BLK ? 3 : 4) update_kernel(Params P, T* __restrict__ x, const T* __restrict__ p,
                                                        T* __restrict__ r, const T* __restrict__ q, Cols C,
                                                        double* __restrict__ partial, const T* __restrict__ mass,
                                                        const T* __restrict__ gdiag, T* __restrict__ zj, T omega) {
  if (*C.live == 0) return;
  constexpr int VEC = Pack<T>::N;
  constexpr int NS = BLK ? 2 : 1;
  extern __shared__ double sm[];
  const int W = P.W;
  const int NSL = CPLX ? W + W / 2 : (PRE ? 2 * W : W);  // slots
  const int TPR = W / VEC;
  const int RPP = kBlock / TPR;
  const int tr = threadIdx.x / TPR, g = threadIdx.x - tr * TPR;
  const int l0 = g * VEC;
  constexpr int ND2 = CPLX ? (VEC / 2 > 0 ? VEC / 2 : 1) : (PRE ? VEC : 1);
  DotAcc<T> d1[VEC], d2[ND2];
  if (tr < RPP) {
    T a[VEC], sh[VEC];
#pragma unroll
    for (int v = 0; v < VEC; v++) {
      if constexpr (CPLX) a[v] = (T)C.alpha[(l0 & ~1) + v];  // lanes (re, im) of one column
      else a[v] = (T)C.alpha[2 * (l0 + v)];
      sh[v] = (PRE || MGJ) ? (T)C.shift[CPLX ? (l0 + v) >> 1 : l0 + v] : (T)0;
    }
    const int64_t rowW = (int64_t)NS * W;
    int chain = 0;
    for (int64_t row = (int64_t)blockIdx.x * RPP + tr; row < P.n; row += (int64_t)gridDim.x * RPP) {
      if (++chain == kFlushRows) {
        chain = 0;
#pragma unroll
        for (int v = 0; v < VEC; v++) d1[v].flush();
#pragma unroll
        for (int v = 0; v < ND2; v++) d2[v].flush();
      }
      const T mr = (PRE || MGJ) ? mass[row] : (T)0, gr = (PRE || MGJ) ? gdiag[row] : (T)0;
#pragma unroll
      for (int b = 0; b < NS; b++) {
        const int64_t off = row * rowW + (int64_t)b * W + l0;
        Pack<T> xv = ldv(x + off), rv = ldv(r + off);
        const Pack<T> pv = ldp(p + off), qv = ldp(q + off);
        if constexpr (CPLX) {
#pragma unroll
          for (int v = 0; v < VEC; v += 2) {
            const T are = a[v], aim = a[v + 1];
            xv.v[v] += are * pv.v[v] - aim * pv.v[v + 1];
            xv.v[v + 1] += are * pv.v[v + 1] + aim * pv.v[v];
            rv.v[v] -= are * qv.v[v] - aim * qv.v[v + 1];
            rv.v[v + 1] -= are * qv.v[v + 1] + aim * qv.v[v];
          }
        } else {
#pragma unroll
          for (int v = 0; v < VEC; v++) {
            xv.v[v] = madd(a[v], pv.v[v], xv.v[v]);
            rv.v[v] = madd(-a[v], qv.v[v], rv.v[v]);
          }
        }
        // rho = <r, z> with z = r, or z = D^-1 r under Jacobi preconditioning
        T zv[VEC];
        if constexpr (PRE) jacobi<T, CPLX, VEC>(mr, gr, sh, rv.v, zv);
        else {
#pragma unroll
          for (int v = 0; v < VEC; v++) zv[v] = rv.v[v];
        }
        if constexpr (CPLX) {
#pragma unroll
          for (int v = 0; v < VEC; v += 2) {
            const T rre = rv.v[v], rim = rv.v[v + 1];
            d1[v].add_sum(madd(rre, zv[v], -rim * zv[v + 1]));
            d1[v + 1].add_sum(madd(rre, zv[v + 1], rim * zv[v]));
            d2[v / 2].add_sum(madd(rre, rre, rim * rim));
          }
        } else {
#pragma unroll
          for (int v = 0; v < VEC; v++) {
            d1[v].add(rv.v[v], zv[v]);
            if constexpr (PRE) d2[v].add(rv.v[v], rv.v[v]);
          }
        }
        stp(x + off, xv);
        stp(r + off, rv);
        if constexpr (MGJ) {
          Pack<T> zo;
          smooth_jacobi<T, CPLX, VEC>(mr, gr, sh, rv.v, zo.v);
#pragma unroll
          for (int v = 0; v < VEC; v++) zo.v[v] *= omega;
          stp(zj + off, zo);
        }
      }
    }
#pragma unroll
    for (int v = 0; v < VEC; v++) sm[tr * NSL + l0 + v] = d1[v].get();
    if constexpr (CPLX) {
#pragma unroll
      for (int v = 0; v < VEC / 2; v++) sm[tr * NSL + W + l0 / 2 + v] = d2[v].get();
    } else if constexpr (PRE) {
#pragma unroll
      for (int v = 0; v < VEC; v++) sm[tr * NSL + W + l0 + v] = d2[v].get();
    }
  }
  __syncthreads();
  for (int l = threadIdx.x; l < NSL; l += kBlock) {
    double s = 0.0;
    for (int t = 0; t < RPP; t++) s += sm[t * NSL + l];
    partial[(int64_t)blockIdx.x * P.pstride + l] = s;
  }
}

// p = r + beta p (r: the residual, or the preconditioned z stored as TZ)
template <typename T, typename TZ, bool CPLX, bool BLK, bool PRE>
__global__ void __launch_bounds__(kBlock) direction_kernel(Params P, T* __restrict__ p, const TZ* __restrict__ r,
                                                           Cols C, const T* __restrict__ mass,
                                                           const T* __restrict__ gdiag) {
  if (*C.live == 0) return;
  constexpr int VEC = Pack<T>::N;
  constexpr int NS = BLK ? 2 : 1;
  const int W = P.W;
  const int TPR = W / VEC;
  const int RPP = kBlock / TPR;
  const int tr = threadIdx.x / TPR, g = threadIdx.x - tr * TPR;
  if (tr >= RPP) return;
  const int l0 = g * VEC;
  T bt[VEC], sh[VEC];
#pragma unroll
  for (int v = 0; v < VEC; v++) {
    if constexpr (CPLX) bt[v] = (T)C.beta[(l0 & ~1) + v];
    else bt[v] = (T)C.beta[2 * (l0 + v)];
    sh[v] = PRE ? (T)C.shift[CPLX ? (l0 + v) >> 1 : l0 + v] : (T)0;
  }
  const int64_t rowW = (int64_t)NS * W;
  for (int64_t row = (int64_t)blockIdx.x * RPP + tr; row < P.n; row += (int64_t)gridDim.x * RPP) {
    const T mr = PRE ? mass[row] : (T)0, gr = PRE ? gdiag[row] : (T)0;
#pragma unroll
    for (int b = 0; b < NS; b++) {
      const int64_t off = row * rowW + (int64_t)b * W + l0;
      Pack<T> pv = ldv(p + off);
      Pack<T> rv;
      lanes_get<T, TZ, VEC>(lanes_ld<false, TZ, VEC>(r + off), rv.v);
      if constexpr (PRE) {  // p = D^-1 r + beta p
        T zv[VEC];
        jacobi<T, CPLX, VEC>(mr, gr, sh, rv.v, zv);
#pragma unroll
        for (int v = 0; v < VEC; v++) rv.v[v] = zv[v];
      }
      if constexpr (CPLX) {
#pragma unroll
        for (int v = 0; v < VEC; v += 2) {
          const T pre = pv.v[v], pim = pv.v[v + 1];
          pv.v[v] = rv.v[v] + bt[v] * pre - bt[v + 1] * pim;
          pv.v[v + 1] = rv.v[v + 1] + bt[v] * pim + bt[v + 1] * pre;
        }
      } else {
#pragma unroll
        for (int v = 0; v < VEC; v++) pv.v[v] = madd(bt[v], pv.v[v], rv.v[v]);
      }
      stp(p + off, pv);
    }
  }
}

__device__ __forceinline__ void cdiv(double ar, double ai, double br, double bi, double& cr, double& ci) {
  const double den = br * br + bi * bi;
  cr = (ar * br + ai * bi) / den;
  ci = (ai * br - ar * bi) / den;
}

// Fixed-order reduction of one slot over the blocks: thread (x, y) sums blocks
// y, y + 8, ...; the eight partial sums are then added in order y = 0..7.
__device__ __forceinline__ double reduce_slot(const double* __restrict__ partial, int nb, int pstride, int slot,
                                              double (*buf)[33]) {
  const int x = threadIdx.x, y = threadIdx.y;
  double s = 0.0;
  if (slot >= 0)
    for (int b = y; b < nb; b += 8) s += partial[(int64_t)b * pstride + slot];
  buf[y][x] = s;
  __syncthreads();
  double t = 0.0;
  if (y == 0)
    for (int k = 0; k < 8; k++) t += buf[k][x];
  __syncthreads();
  return t;
}

template <bool CPLX>
__global__ void finish_alpha_kernel(Params P, int nb, const double* __restrict__ partial, Cols C) {
  __shared__ double buf[8][33];
  const int col = blockIdx.x * 32 + threadIdx.x;
  const bool ok = col < P.ncols;
  const double sre = reduce_slot(partial, nb, P.pstride, ok ? (CPLX ? 2 * col : col) : -1, buf);
  const double sim = CPLX ? reduce_slot(partial, nb, P.pstride, ok ? 2 * col + 1 : -1, buf) : 0.0;
  if (threadIdx.y != 0 || !ok) return;
  double ar = 0.0, ai = 0.0;
  if (C.active[col]) {
    const double rr = C.rho[2 * col], ri = C.rho[2 * col + 1];
    if (!(isfinite(sre) && isfinite(sim)) || (sre == 0.0 && sim == 0.0)) {
      C.active[col] = 0;
      C.done[col] = 1;
      C.status[col] = 2;
      atomicSub(C.live, 1);
    } else if (CPLX) {
      cdiv(rr, ri, sre, sim, ar, ai);
    } else {
      ar = rr / sre;
    }
  }
  C.alpha[2 * col] = ar;
  C.alpha[2 * col + 1] = ai;
}

template <bool CPLX>
__global__ void finish_beta_kernel(Params P, int nb, const double* __restrict__ partial, Cols C) {
  __shared__ double buf[8][33];
  const int col = blockIdx.x * 32 + threadIdx.x;
  const bool ok = col < P.ncols;
  const double rre = reduce_slot(partial, nb, P.pstride, ok ? (CPLX ? 2 * col : col) : -1, buf);
  const double rim = CPLX ? reduce_slot(partial, nb, P.pstride, ok ? 2 * col + 1 : -1, buf) : 0.0;
  // ||r||^2: its own slot for complex columns and under Jacobi preconditioning, <r, r> otherwise
  const double n2 = (CPLX || P.rn_slot) ? reduce_slot(partial, nb, P.pstride, ok ? P.W + col : -1, buf) : rre;
  if (threadIdx.y != 0 || !ok) return;
  double br = 0.0, bi = 0.0;
  if (C.active[col]) {
    if (!P.mg) {  // multigrid: rho and beta come from <r, z> (finish_rho_kernel)
      const double orr = C.rho[2 * col], ori = C.rho[2 * col + 1];
      if (CPLX) cdiv(rre, rim, orr, ori, br, bi);
      else br = rre / orr;
      C.rho[2 * col] = rre;
      C.rho[2 * col + 1] = rim;
    }
    C.rn2[col] = n2;
    const int it = ++C.iters[col];
    bool stop = false;
    if (!(isfinite(n2) && isfinite(br) && isfinite(bi))) {  // (br, bi stay 0 under multigrid)
      C.status[col] = 2;
      C.done[col] = 1;
      stop = true;
    } else if (n2 <= C.target2[col]) {
      stop = true;
    } else if (it >= P.maxit || it - C.round_it0[col] >= C.round_cap[col]) {
      // iteration cap, or an inner round that stalls: end the round so that a
      // fresh FP64 residual restarts it
      stop = true;
    }
    if (stop) {
      C.active[col] = 0;
      atomicSub(C.live, 1);
      br = bi = 0.0;
    }
  }
  C.beta[2 * col] = br;
  C.beta[2 * col + 1] = bi;
}

// Residual form of the solve (Sect. 2.2.2): the unfiltered field x0 is kept
// apart and the engines solve S delta = r0 = b - S x0, the filtered field being
// x0 + delta.  The true residual of a refinement round is then r0 - S delta,
// whose rounding error is relative to ||S delta|| ~ ||r0|| rather than to
// ||b|| (at small scales ||r0|| is orders of magnitude below ||b||, and b - S x
// could not be driven to the paper's relative tolerance in FP64).  Each source
// (field, system) keeps, in one buffer of 3 [n][NS] FP64 blocks and one FP32
// block:
//   e0 = b - M x0   (exact up to one rounding; 0 up to rounding for b = M x0)
//   x0
//   g0 = G x0       (the operator without its shift, shared by all scales)
//   x0 rounded to float (the double-float engines' norm of the solution)
// so that r0 = e0 - shift g0 (real columns) or e0 - i shift g0 (complex ones).
template <bool BLK>
__global__ void __launch_bounds__(256) source_kernel(EllView<double> A, int32_t n, const double* __restrict__ mass,
                                                     double* __restrict__ buf) {
  constexpr int NS = BLK ? 2 : 1;
  const int64_t bs = (int64_t)n * NS;
  double* e0 = buf;
  const double* x0 = buf + bs;
  double* g0 = buf + 2 * bs;
  float* x0f = reinterpret_cast<float*>(buf + 3 * bs);
  for (int32_t row = blockIdx.x * blockDim.x + threadIdx.x; row < n; row += gridDim.x * blockDim.x) {
    const int s = row / A.slice_h;
    const int w = A.slice_w[s];
    const int64_t base = A.slice_off[s] + (int64_t)(row - s * A.slice_h) * w;
    double acc[NS];
#pragma unroll
    for (int b = 0; b < NS; b++) acc[b] = 0.0;
    for (int e = 0; e < w; e++) {
      const int64_t c = A.col[base + e];
      if constexpr (BLK) {
        const double a = A.val[(base + e) * 2], bb = A.val[(base + e) * 2 + 1];
        const double xu = x0[c * 2], xw = x0[c * 2 + 1];
        acc[0] = __fma_rn(a, xu, __fma_rn(bb, xw, acc[0]));
        acc[1] = __fma_rn(a, xw, __fma_rn(-bb, xu, acc[1]));
      } else {
        acc[0] = __fma_rn(A.val[base + e], x0[c], acc[0]);
      }
    }
    const double mr = mass[row];
#pragma unroll
    for (int b = 0; b < NS; b++) {
      const int64_t i = (int64_t)row * NS + b;
      g0[i] = acc[b];
      x0f[i] = (float)x0[i];
      e0[i] = __fma_rn(-mr, x0[i], e0[i]);
    }
  }
}

// delta = 0 on the lanes of newly admitted columns (FP64 and double-float
// lanes alike: both are 8 bytes of zeros)
template <bool CPLX>
__global__ void init_lanes_kernel(Params P, int NS, const int* __restrict__ fresh, double* __restrict__ x64) {
  const int64_t total = (int64_t)P.n * NS * P.W;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int l = (int)(i % P.W);
    if (fresh[CPLX ? l >> 1 : l]) x64[i] = 0.0;
  }
}

// FP64 true residual r64 = r0 - S delta (delta in x64); starts an inner round:
// r = p = (T) r64, d = 0.
// Slots: [0, W) <r, r> of the rounded residual (lane-wise / (re, im) pairs),
//        [W, W + ncols) ||r64||^2.
template <typename T, bool CPLX, bool BLK>
__global__ void __launch_bounds__(kBlock) residual_kernel(EllView<double> A, Params P,
                                                          const double* __restrict__ x64,
                                                          const double* const* __restrict__ bptr,
                                                          const int* __restrict__ lane_src,
                                                          const double* __restrict__ mass, Cols C,
                                                          T* __restrict__ r, T* __restrict__ d, T* __restrict__ p,
                                                          double* __restrict__ partial,
                                                          const double* __restrict__ gdiag) {
  constexpr int VEC = Pack<T>::N;
  constexpr int NS = BLK ? 2 : 1;
  constexpr int NV = BLK ? 2 : 1;
  constexpr int DP = VEC / 2;  // double packs per thread
  if (C.live[1] == 0) return;   // no column waits for a refinement round
  extern __shared__ double sm[];
  const int W = P.W;
  const int ncolsW = CPLX ? W / 2 : W;
  const int NSL = W + 3 * ncolsW;  // <r, z> lanes, then per column ||r||^2, ||r||^2_{M^-1}, ||x||^2_M
  const int TPR = W / VEC;
  const int RPP = kBlock / TPR;
  const int tr = threadIdx.x / TPR, g = threadIdx.x - tr * TPR;
  const int l0 = g * VEC;
  double d1[VEC], d2[VEC], e2[VEC], x2[VEC];
#pragma unroll
  for (int v = 0; v < VEC; v++) d1[v] = d2[v] = e2[v] = x2[v] = 0.0;
  // Lanes of columns that are not being refreshed keep their inner state; a
  // thread none of whose columns is refreshed skips its loads altogether, so
  // the traffic follows the number of refreshed columns.
  bool mine[VEC];
  bool any = false, all = true;
#pragma unroll
  for (int v = 0; v < VEC; v++) {
    mine[v] = C.refresh[CPLX ? (l0 + v) >> 1 : l0 + v] != 0;
    any |= mine[v];
    all &= mine[v];
  }
  if (tr < RPP && any) {
    double sh[VEC];
    int src[VEC];
#pragma unroll
    for (int v = 0; v < VEC; v++) {
      sh[v] = C.shift[CPLX ? (l0 + v) >> 1 : l0 + v];
      src[v] = lane_src[l0 + v];
    }
    const int64_t rowW = (int64_t)NS * W;
    const int64_t sstride = (int64_t)P.n * NS;  // blocks of a source buffer
    for (int64_t row = (int64_t)blockIdx.x * RPP + tr; row < P.n; row += (int64_t)gridDim.x * RPP) {
      const int s = (int)(row / A.slice_h);
      const int w = A.slice_w[s];
      const int64_t base = A.slice_off[s] + (row - (int64_t)s * A.slice_h) * w;
      double acc[NS][VEC];
#pragma unroll
      for (int b = 0; b < NS; b++)
#pragma unroll
        for (int v = 0; v < VEC; v++) acc[b][v] = 0.0;
      for (int e = 0; e < w; e++) {
        const int c = A.col[base + e];
        const double* xs = x64 + (int64_t)c * rowW + l0;
        double xu[VEC], xw[VEC];
#pragma unroll
        for (int k = 0; k < DP; k++) {
          Pack<double> t = ldp(xs + 2 * k);
          xu[2 * k] = t.v[0];
          xu[2 * k + 1] = t.v[1];
          if constexpr (BLK) {
            Pack<double> t2 = ldp(xs + W + 2 * k);
            xw[2 * k] = t2.v[0];
            xw[2 * k + 1] = t2.v[1];
          }
        }
        if constexpr (BLK) {
          const double a = A.val[(base + e) * 2], bb = A.val[(base + e) * 2 + 1];
#pragma unroll
          for (int v = 0; v < VEC; v++) {
            acc[0][v] += a * xu[v] + bb * xw[v];
            acc[1][v] += -bb * xu[v] + a * xw[v];
          }
        } else {
          const double a = A.val[base + e];
#pragma unroll
          for (int v = 0; v < VEC; v++) acc[0][v] += a * xu[v];
        }
        (void)NV;
      }
      const double mr = mass[row];
      const double gr = gdiag ? gdiag[row] : 0.0;
#pragma unroll
      for (int b = 0; b < NS; b++) {
        const int64_t off = row * rowW + (int64_t)b * W + l0;
        double xo[VEC];
#pragma unroll
        for (int k = 0; k < DP; k++) {
          Pack<double> t = ldp(x64 + off + 2 * k);
          xo[2 * k] = t.v[0];
          xo[2 * k + 1] = t.v[1];
        }
        // r (rounded to T), the restarted direction p = z (z = r, or D^-1 r
        // under Jacobi preconditioning) and rho = <r, z>
        Pack<T> ro, po, zo;
#pragma unroll
        for (int v = 0; v < VEC; v++) zo.v[v] = (T)0;
        if constexpr (CPLX) {
#pragma unroll
          for (int v = 0; v < VEC; v += 2) {
            double e0 = 0.0, g0 = 0.0, x0 = 0.0;
            if (mine[v]) {  // a retired column's source may be gone
              const double* sb = bptr[src[v]] + row * NS + b;
              e0 = sb[0];
              x0 = sb[sstride];
              g0 = sb[2 * sstride];
            }
            // r0 = e0 - i shift g0, minus S delta = (m + i shift G) delta
            const double r_re = e0 - (mr * xo[v] - sh[v] * acc[b][v + 1]);
            const double r_im = -(sh[v] * g0) - (mr * xo[v + 1] + sh[v] * acc[b][v]);
            const T tre = (T)r_re, tim = (T)r_im;
            T zre = tre, zim = tim;
            if (gdiag) {
              const double bg = sh[v] * gr;
              const double inv = 1.0 / (mr * mr + bg * bg);
              zre = (T)((r_re * mr + r_im * bg) * inv);
              zim = (T)((r_im * mr - r_re * bg) * inv);
            }
            ro.v[v] = tre;
            ro.v[v + 1] = tim;
            po.v[v] = zre;
            po.v[v + 1] = zim;
            d1[v] += (double)tre * zre - (double)tim * zim;
            d1[v + 1] += (double)tre * zim + (double)tim * zre;
            d2[v / 2] += r_re * r_re + r_im * r_im;
            e2[v / 2] += (r_re * r_re + r_im * r_im) / mr;
            const double xr = x0 + xo[v];  // the filtered field is the real part
            x2[v / 2] += mr * xr * xr;
          }
        } else {
#pragma unroll
          for (int v = 0; v < VEC; v++) {
            double e0 = 0.0, g0 = 0.0, x0 = 0.0;
            if (mine[v]) {
              const double* sb = bptr[src[v]] + row * NS + b;
              e0 = sb[0];
              x0 = sb[sstride];
              g0 = sb[2 * sstride];
            }
            const double rv = __fma_rn(-sh[v], g0, e0) - (mr * xo[v] + sh[v] * acc[b][v]);
            const T t = (T)rv;
            const T z = gdiag ? (T)(rv / (mr + sh[v] * gr)) : t;
            ro.v[v] = t;
            po.v[v] = z;
            d1[v] += (double)t * z;
            d2[v] += rv * rv;
            e2[v] += rv * rv / mr;
            const double xr = x0 + xo[v];
            x2[v] += mr * xr * xr;
          }
        }
        if (all) {
          stp(r + off, ro);
          stp(p + off, po);
          stp(d + off, zo);
        } else {
#pragma unroll
          for (int v = 0; v < VEC; v++)
            if (mine[v]) {
              r[off + v] = ro.v[v];
              p[off + v] = po.v[v];
              d[off + v] = (T)0;
            }
        }
      }
    }
  }
  if (tr < RPP) {
#pragma unroll
    for (int v = 0; v < VEC; v++) sm[tr * NSL + l0 + v] = d1[v];
    if constexpr (CPLX) {
#pragma unroll
      for (int v = 0; v < VEC / 2; v++) {
        sm[tr * NSL + W + l0 / 2 + v] = d2[v];
        sm[tr * NSL + W + ncolsW + l0 / 2 + v] = e2[v];
        sm[tr * NSL + W + 2 * ncolsW + l0 / 2 + v] = x2[v];
      }
    } else {
#pragma unroll
      for (int v = 0; v < VEC; v++) {
        sm[tr * NSL + W + l0 + v] = d2[v];
        sm[tr * NSL + W + ncolsW + l0 + v] = e2[v];
        sm[tr * NSL + W + 2 * ncolsW + l0 + v] = x2[v];
      }
    }
  }
  __syncthreads();
  for (int l = threadIdx.x; l < NSL; l += kBlock) {
    double s = 0.0;
    for (int t = 0; t < RPP; t++) s += sm[t * NSL + l];
    partial[(int64_t)blockIdx.x * P.pstride + l] = s;
  }
}

template <bool CPLX>
__global__ void finish_residual_kernel(Params P, int nb, const double* __restrict__ partial, Cols C) {
  if (C.live[1] == 0) return;
  __shared__ double buf[8][33];
  const int col = blockIdx.x * 32 + threadIdx.x;
  const bool ok = col < P.ncols;
  const double rre = reduce_slot(partial, nb, P.pstride, ok ? (CPLX ? 2 * col : col) : -1, buf);
  const double rim = CPLX ? reduce_slot(partial, nb, P.pstride, ok ? 2 * col + 1 : -1, buf) : 0.0;
  const double n2 = reduce_slot(partial, nb, P.pstride, ok ? P.W + col : -1, buf);
  const int ncolsW = CPLX ? P.W / 2 : P.W;
  const double e2 = reduce_slot(partial, nb, P.pstride, ok ? P.W + ncolsW + col : -1, buf);
  const double x2 = reduce_slot(partial, nb, P.pstride, ok ? P.W + 2 * ncolsW + col : -1, buf);
  if (threadIdx.y != 0 || !ok) return;
  if (!C.refresh[col]) return;
  C.refresh[col] = 0;
  if (C.r0n2[col] < 0.0) {
    C.r0n2[col] = n2;
    C.tol2[col] = P.tol2_rel * n2;
  }
  const double r0 = C.r0n2[col];
  const double rel_prev = C.rel[col];  // at the end of the previous round (1 after the first residual)
  C.rel[col] = r0 > 0.0 ? sqrt(n2 / r0) : 0.0;
  C.err[col] = x2 > 0.0 ? sqrt(e2 / x2) : (e2 > 0.0 ? INFINITY : 0.0);
  // error test: ||r||^2_{M^-1} <= err_tol^2 ||x||^2_M; its equivalent in ||r||^2
  // (at the current ratio of the two norms) bounds the inner target below
  const bool err_ok = !(P.err2 > 0.0) || e2 <= P.err2 * x2;
  const double tol2_eff = (P.err2 > 0.0 && e2 > 0.0) ? fmin(C.tol2[col], P.err2 * x2 * (n2 / e2)) : C.tol2[col];
  if (C.active[col]) {  // inner round stopped by its iteration cap
    C.active[col] = 0;
    atomicSub(C.live, 1);
  }
  if (C.done[col]) return;
  if ((!(n2 > C.tol2[col]) && err_ok) || r0 == 0.0) {
    C.done[col] = 1;
    return;
  }
  if (!isfinite(n2)) {
    C.done[col] = 1;
    C.status[col] = 2;
    return;
  }
  if (C.iters[col] >= P.maxit) {
    C.done[col] = 1;
    C.status[col] = 1;
    return;
  }
  if (C.rounds[col] >= 1 && !(C.rel[col] < rel_prev)) {
    // a whole round left the true residual where it was: it sits at its
    // rounding floor (or the inner solve diverges), and more rounds cannot help
    C.done[col] = 1;
    C.status[col] = 1;
    return;
  }
  C.rho[2 * col] = rre;
  C.rho[2 * col + 1] = rim;
  C.rn2[col] = n2;
  C.target2[col] = fmax(P.inner2 * n2, 0.25 * tol2_eff);
  // later rounds get twice the length of the first (at least 256 iterations)
  if (C.rounds[col] == 1) C.round_cap[col] = max(256, 2 * (C.iters[col] - C.round_it0[col]));
  else if (C.rounds[col] == 0) C.round_cap[col] = P.maxit;
  C.round_it0[col] = C.iters[col];
  C.rounds[col]++;
  C.active[col] = 1;
  C.restart[col] = P.mg;
  atomicAdd(C.live, 1);
}

// Multigrid order: beta = <r, z>_new / <r, z>_old from the partials of the
// last smoothing sweep (z the V-cycle of r); beta = 0 on a restarted column.
template <bool CPLX>
__global__ void finish_rho_kernel(Params P, int nb, const double* __restrict__ partial, Cols C) {
  __shared__ double buf[8][33];
  const int col = blockIdx.x * 32 + threadIdx.x;
  const bool ok = col < P.ncols;
  const double zre = reduce_slot(partial, nb, P.pstride, ok ? (CPLX ? 2 * col : col) : -1, buf);
  const double zim = CPLX ? reduce_slot(partial, nb, P.pstride, ok ? 2 * col + 1 : -1, buf) : 0.0;
  if (threadIdx.y != 0 || !ok) return;
  double br = 0.0, bi = 0.0;
  if (C.active[col]) {
    if (!(isfinite(zre) && isfinite(zim)) || (zre == 0.0 && zim == 0.0)) {
      C.active[col] = 0;
      C.done[col] = 1;
      C.status[col] = 2;
      atomicSub(C.live, 1);
    } else {
      if (C.restart[col]) {
        C.restart[col] = 0;
      } else {
        const double orr = C.rho[2 * col], ori = C.rho[2 * col + 1];
        if (CPLX) cdiv(zre, zim, orr, ori, br, bi);
        else br = zre / orr;
      }
      C.rho[2 * col] = zre;
      C.rho[2 * col + 1] = zim;
    }
  }
  C.beta[2 * col] = br;
  C.beta[2 * col + 1] = bi;
}

// x = w D^-1 rhs on a multigrid level (the first smoothing sweep from zero);
// rhs stored as TR, x as TS, VEC lanes per thread
template <typename T, typename TR, typename TS, int VEC, bool CPLX, bool BLK>
__global__ void __launch_bounds__(kBlock) mg_jacobi_kernel(Params P, const TR* __restrict__ rhs, TS* __restrict__ x,
                                                           const T* __restrict__ mdiag, const T* __restrict__ kdiag,
                                                           Cols C, T omega) {
  if (*C.live == 0) return;
  constexpr int NS = BLK ? 2 : 1;
  const int W = P.W;
  const int TPR = W / VEC;
  const int RPP = kBlock / TPR;
  const int tr = threadIdx.x / TPR, g = threadIdx.x - tr * TPR;
  if (tr >= RPP) return;
  const int l0 = g * VEC;
  T sh[VEC];
#pragma unroll
  for (int v = 0; v < VEC; v++) sh[v] = (T)C.shift[CPLX ? (l0 + v) >> 1 : l0 + v];
  const int64_t rowW = (int64_t)NS * W;
  for (int64_t row = (int64_t)blockIdx.x * RPP + tr; row < P.n; row += (int64_t)gridDim.x * RPP) {
    const T mr = mdiag[row], kr = kdiag[row];
#pragma unroll
    for (int b = 0; b < NS; b++) {
      const int64_t off = row * rowW + (int64_t)b * W + l0;
      T rv[VEC];
      lanes_get<T, TR, VEC>(lanes_ld<false, TR, VEC>(rhs + off), rv);
      T z[VEC];
      smooth_jacobi<T, CPLX, VEC>(mr, kr, sh, rv, z);
#pragma unroll
      for (int v = 0; v < VEC; v++) z[v] *= omega;
      lanes_st<TS, VEC>(x + off, lanes_put<T, TS, VEC>(z));
    }
  }
}

// x64 += d on the lanes of refreshed columns
template <typename T, bool CPLX>
__global__ void accumulate_kernel(int64_t total, int W, const int* __restrict__ refresh, double* __restrict__ x64,
                                  const T* __restrict__ d, const int* __restrict__ live) {
  if (live[1] == 0) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int l = (int)(i % W);
    if (refresh[CPLX ? l >> 1 : l]) x64[i] += (double)d[i];
  }
}

// Flags every column whose inner solve has ended but which is not done for
// a refinement round, and counts active / to-refresh / unfinished columns.
__global__ void scan_kernel(int ncols, Cols C) {
  __shared__ int cnt[3];
  if (threadIdx.x < 3) cnt[threadIdx.x] = 0;
  __syncthreads();
  for (int c = threadIdx.x; c < ncols; c += blockDim.x) {
    const int a = C.active[c], dn = C.done[c];
    const int rf = (!a && !dn) ? 1 : 0;
    C.refresh[c] = rf;
    if (a) atomicAdd(&cnt[0], 1);
    if (rf) atomicAdd(&cnt[1], 1);
    if (!dn) atomicAdd(&cnt[2], 1);
  }
  __syncthreads();
  if (threadIdx.x < 3) C.live[threadIdx.x] = cnt[threadIdx.x];
}

// dst[row][l'] = src[row][map[l']] (0 where map < 0): narrows the lane tiles
// to the columns that are still running.
template <typename T>
__global__ void gather_lanes_kernel(int64_t rows, int Wold, int Wnew, const int* __restrict__ map,
                                    const T* __restrict__ src, T* __restrict__ dst) {
  const int64_t total = rows * Wnew;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = i / Wnew;
    const int l = (int)(i - row * Wnew);
    const int mo = map[l];
    dst[i] = mo >= 0 ? src[row * Wold + mo] : (T)0;
  }
}

// The filtered field x0 + delta (real part) of every column flagged in `emit`,
// written to its caller block out[comp][o] in original mesh order; land
// entries copy the input (scalar, cell) or are zero (vector).
template <bool CPLX, bool BLK, bool DFX>
__global__ void output_kernel(Params P, int32_t n_out, const int32_t* __restrict__ inv,
                              const double* __restrict__ x64, const double* const* __restrict__ bptr,
                              const int* __restrict__ lane_src, double* const* __restrict__ col_out,
                              const double* const* __restrict__ col_in, const int* __restrict__ emit) {
  constexpr int NS = BLK ? 2 : 1;
  const int col = blockIdx.y;
  if (!emit[col]) return;
  double* out = col_out[col];
  const double* in = col_in[col];
  const int lane = CPLX ? 2 * col : col;
  const double* x0 = bptr[lane_src[lane]] + (int64_t)P.n * NS;
  for (int32_t o = blockIdx.x * blockDim.x + threadIdx.x; o < n_out; o += gridDim.x * blockDim.x) {
    const int32_t r = inv[o];
#pragma unroll
    for (int b = 0; b < NS; b++) {
      double v;
      if (r >= 0) {
        const int64_t i = ((int64_t)r * NS + b) * P.W + lane;
        double dv;
        if constexpr (DFX) {  // double-float pair (FP32 engines)
          const float2 h = reinterpret_cast<const float2*>(x64)[i];
          dv = (double)h.x + (double)h.y;
        } else {
          dv = x64[i];
        }
        v = x0[(int64_t)r * NS + b] + dv;
      }
      else v = BLK ? 0.0 : in[o];
      out[(int64_t)b * n_out + o] = v;
    }
  }
}


// ------------------------------------------------------------ double-float
// The FP32 engines keep the refined solution x and the right-hand sides as
// unevaluated pairs hi + lo of floats (about 48 significant bits) and compute
// the true residual with them on the FP32 pipes: products split exactly with an
// FMA, sums by two-sum (Dekker; Knuth).  GB300's FP64 rate is a small fraction
// of its FP32 rate, and this residual is recomputed for every refinement round.
struct DF {
  float hi, lo;
};
__device__ __forceinline__ DF df_from(double v) {
  const float h = (float)v;
  return {h, (float)(v - (double)h)};
}
__device__ __forceinline__ double df_to(DF a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ DF df_norm(float s, float e) {  // |e| small relative to s
  const float t = __fadd_rn(s, e);
  return {t, __fsub_rn(e, __fsub_rn(t, s))};
}
__device__ __forceinline__ DF df_add(DF a, DF b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float z = __fsub_rn(s, a.hi);
  const float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, z)), __fsub_rn(b.hi, z));
  return df_norm(s, __fadd_rn(err, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ DF df_neg(DF a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ DF df_mul(DF a, DF b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_norm(p, e);
}
__device__ __forceinline__ DF df_add_f(DF a, float b) { return df_add(a, DF{b, 0.f}); }

template <bool CPLX>
__global__ void accumulate_df_kernel(int64_t total, int W, const int* __restrict__ refresh, DF* __restrict__ x,
                                     const float* __restrict__ d, const int* __restrict__ live) {
  if (live[1] == 0) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int l = (int)(i % W);
    if (refresh[CPLX ? l >> 1 : l]) x[i] = df_add_f(x[i], d[i]);
  }
}
// a block of a source buffer (double) rewritten in place as double-float pairs
__global__ void to_df_kernel(int64_t n, double* __restrict__ v) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const DF a = df_from(v[i]);
    reinterpret_cast<DF*>(v)[i] = a;
  }
}

// The refinement residual of the FP32 engines, as residual_kernel computes it
// in FP64 but in double-float arithmetic: r = r0 - (M delta + shift * (G delta))
// with r0 = e0 - shift g0 from the column's source, the operator values split
// hi + lo (val32 and val32lo), the lumped mass likewise, delta, e0 and g0 as
// pairs.  Writes r (rounded to float), the restarted p (= r, or
// D^-1 r with Jacobi) and d = 0 on the refreshed lanes, and per-block partials
// of <r, z>, ||r||^2, ||r||^2_{M^-1} and ||x||^2_M (compensated FP32 sums of
// the rounded values, flushed to FP64).
template <bool CPLX, bool BLK>
__global__ void __launch_bounds__(kBlock, 2) residual_df_kernel(EllView<float> A, const float* __restrict__ vlo, Params P,
                                                               const DF* __restrict__ x, const DF* const* __restrict__ bptr,
                                                               const int* __restrict__ lane_src,
                                                               const float* __restrict__ mhi, const float* __restrict__ mlo,
                                                               Cols C, float* __restrict__ r, float* __restrict__ d,
                                                               float* __restrict__ p, double* __restrict__ partial,
                                                               const float* __restrict__ gdiag) {
  constexpr int VEC = Pack<float>::N;
  static_assert(VEC == 4, "the double-float residual moves 4 lanes of (hi, lo) pairs per thread");
  constexpr int NS = BLK ? 2 : 1;
  constexpr int NV = BLK ? 2 : 1;
  if (C.live[1] == 0) return;
  extern __shared__ __align__(16) double sm[];
  __shared__ int s_w[2][kMaxSpt], s_o[2][kMaxSpt];
  __shared__ __align__(8) uint64_t bar[2];
  const int W = P.W;
  const int ncolsW = CPLX ? W / 2 : W;
  const int NSL = W + 3 * ncolsW;
  const int TPR = W / VEC;
  const int RPP = kBlock / TPR;
  const int tr = threadIdx.x / TPR, g = threadIdx.x - tr * TPR;
  const int l0 = g * VEC;
  // Tiles of `spt` ELL slices: their column indices and the operator's hi and lo values are
  // bulk-copied into one of two shared-memory buffers while the block works on the previous
  // tile, as in spmm_kernel, so a row waits only on its gathered rows and its own operands.
  const int H = A.slice_h;
  const int spt = P.spt;
  const int TR = spt * H;
  const int n_slices = (int)((P.n + H - 1) / H);
  const int ntiles = (n_slices + spt - 1) / spt;
  unsigned char* const sbase =
      reinterpret_cast<unsigned char*>(sm) + ((size_t)RPP * NSL * sizeof(double) + 15) / 16 * 16;
  const size_t colb = ((size_t)P.stage_e * 4 + 15) / 16 * 16;
  const size_t valb = ((size_t)P.stage_e * NV * sizeof(float) + 15) / 16 * 16;
  auto stage_col = [&](int b) { return reinterpret_cast<int*>(sbase + b * (colb + 2 * valb)); };
  auto stage_hi = [&](int b) { return reinterpret_cast<float*>(sbase + b * (colb + 2 * valb) + colb); };
  auto stage_lo = [&](int b) { return reinterpret_cast<float*>(sbase + b * (colb + 2 * valb) + colb + valb); };
  auto issue = [&](int tile, int b) {  // one thread
    const int s0 = tile * spt, s1 = min(s0 + spt, n_slices);
    const int64_t ob = A.slice_off[s0], oe = A.slice_off[s1];
    const uint32_t ne = (uint32_t)(oe - ob);
    const uint32_t bc = ne * 4u, bv = ne * (uint32_t)(NV * sizeof(float));
    async_proxy_fence();  // earlier generic reads of the buffer come first
    mbar_expect(&bar[b], bc + 2 * bv);
    if (ne > 0) {
      bulk_to_smem(stage_col(b), A.col + ob, bc, &bar[b]);
      bulk_to_smem(stage_hi(b), A.val + ob * NV, bv, &bar[b]);
      bulk_to_smem(stage_lo(b), vlo + ob * NV, bv, &bar[b]);
    }
  };
  if (threadIdx.x == 0) {
    mbar_init(&bar[0]);
    mbar_init(&bar[1]);
    async_proxy_fence();
  }
  __syncthreads();
  if ((int)blockIdx.x < ntiles) {
    const int s0 = blockIdx.x * spt, cnt = min(s0 + spt, n_slices) - s0;
    if (threadIdx.x == 0) issue(blockIdx.x, 0);
    if ((int)threadIdx.x < cnt) {
      s_w[0][threadIdx.x] = A.slice_w[s0 + threadIdx.x];
      s_o[0][threadIdx.x] = (int)(A.slice_off[s0 + threadIdx.x] - A.slice_off[s0]);
    }
  }
  __syncthreads();
  DotAcc<float> d1[VEC], d2[VEC], e2[VEC], x2[VEC];
  bool mine[VEC];
  bool any = false, all = true;
#pragma unroll
  for (int v = 0; v < VEC; v++) {
    mine[v] = tr < RPP && C.refresh[CPLX ? (l0 + v) >> 1 : l0 + v] != 0;
    any |= mine[v];
    all &= mine[v];
  }
  const bool work = tr < RPP && any;
  DF sh[VEC];
  int src[VEC];
  float shf[VEC];
#pragma unroll
  for (int v = 0; v < VEC; v++) {
    const double s = work ? C.shift[CPLX ? (l0 + v) >> 1 : l0 + v] : 0.0;
    sh[v] = df_from(s);
    shf[v] = (float)s;
    src[v] = work ? lane_src[l0 + v] : 0;
  }
  const int64_t rowW = (int64_t)NS * W;
  const int64_t sstride = (int64_t)P.n * NS;  // blocks of a source buffer
  int chain = 0;
  unsigned inflight = (int)blockIdx.x < ntiles ? 1u : 0u;  // bit b: a copy into buffer b is outstanding
  int it = 0;
  bool failed = false;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, it++) {
    const int buf = it & 1;
    const int next = tile + gridDim.x;
    int nw = 0, no = 0, ncnt = 0;
    if (next < ntiles) {
      if (threadIdx.x == 0) issue(next, buf ^ 1);
      inflight |= 1u << (buf ^ 1);
      const int s0 = next * spt;
      ncnt = min(s0 + spt, n_slices) - s0;
      if ((int)threadIdx.x < ncnt) {  // consumed after this tile's rows
        nw = A.slice_w[s0 + threadIdx.x];
        no = (int)(A.slice_off[s0 + threadIdx.x] - A.slice_off[s0]);
      }
    }
    bool late = false;
    if (threadIdx.x == 0) late = !mbar_wait_bounded(&bar[buf], (uint32_t)((it >> 1) & 1));
    if (__syncthreads_or(late)) {
      failed = true;
      break;
    }
    inflight &= ~(1u << buf);
    const int* scol = stage_col(buf);
    const float* shi = stage_hi(buf);
    const float* slo = stage_lo(buf);
    const int64_t r0 = (int64_t)tile * TR;
    const int rows = (int)min((int64_t)TR, P.n - r0);
    if (work) {
      for (int lr = tr; lr < rows; lr += RPP) {
        const int64_t row = r0 + lr;
        const int sl = lr / H;
        const int w = s_w[buf][sl];
        const int eb = s_o[buf][sl] + (lr - sl * H) * w;
        DF acc[NS][VEC];
  #pragma unroll
        for (int b = 0; b < NS; b++)
  #pragma unroll
          for (int v = 0; v < VEC; v++) acc[b][v] = DF{0.f, 0.f};
        // The row's source values (e0, g0, x0 of each refreshed column): loaded
        // before its gathers, so that both wait out one memory latency together,
        // where the registers allow it (scalar rows); after them for 2x2 blocks.
        constexpr int SV = CPLX ? VEC / 2 : VEC;  // source values per sub-row: one per column
        constexpr bool HOIST = !BLK;
        DF se0[NS][SV], sg0[NS][SV];
        float sx0[NS][SV];
        auto load_sources = [&]() {
  #pragma unroll
          for (int b = 0; b < NS; b++)
  #pragma unroll
            for (int c = 0; c < SV; c++) {
              const int v = CPLX ? 2 * c : c;
              se0[b][c] = sg0[b][c] = DF{0.f, 0.f};
              sx0[b][c] = 0.f;
              if (mine[v]) {  // a retired column's source may be gone
                const DF* sb = bptr[src[v]] + row * NS + b;
                se0[b][c] = sb[0];
                sg0[b][c] = sb[2 * sstride];
                sx0[b][c] = reinterpret_cast<const float*>(bptr[src[v]] + 3 * sstride)[row * NS + b];
              }
            }
        };
        if constexpr (HOIST) load_sources();
        // EBR entries at a time: their column indices in one load, then all their
        // gathered rows, then the arithmetic (one round of dependent loads per batch).
        // Rows hold a multiple of 4 entries and start 4-aligned, so the index and
        // value loads are aligned vector loads.
        constexpr int EBR = BLK ? 2 : 4;
        for (int e = 0; e < w; e += EBR) {
          int cc[EBR];
          if constexpr (EBR == 4) {
            const int4 c4 = *reinterpret_cast<const int4*>(scol + eb + e);
            cc[0] = c4.x, cc[1] = c4.y, cc[2] = c4.z, cc[3] = c4.w;
          } else {
            const int2 c2 = *reinterpret_cast<const int2*>(scol + eb + e);
            cc[0] = c2.x, cc[1] = c2.y;
          }
          float4 xv[EBR][NS][2];  // 4 lanes of (hi, lo) pairs per entry and sub-row
  #pragma unroll
          for (int t = 0; t < EBR; t++)
  #pragma unroll
            for (int b = 0; b < NS; b++) {
              const float4* xp = reinterpret_cast<const float4*>(x + (int64_t)cc[t] * rowW + (int64_t)b * W + l0);
              xv[t][b][0] = __ldg(xp);
              xv[t][b][1] = __ldg(xp + 1);
            }
          const float4 vh = *reinterpret_cast<const float4*>(shi + (eb + e) * NV);
          const float4 vl = *reinterpret_cast<const float4*>(slo + (eb + e) * NV);
          const float hv[4] = {vh.x, vh.y, vh.z, vh.w}, lv[4] = {vl.x, vl.y, vl.z, vl.w};
  #pragma unroll
          for (int t = 0; t < EBR; t++) {
            DF xu[VEC], xw[VEC];
  #pragma unroll
            for (int b = 0; b < NS; b++) {
              DF* d = b == 0 ? xu : xw;
              d[0] = DF{xv[t][b][0].x, xv[t][b][0].y};
              d[1] = DF{xv[t][b][0].z, xv[t][b][0].w};
              d[2] = DF{xv[t][b][1].x, xv[t][b][1].y};
              d[3] = DF{xv[t][b][1].z, xv[t][b][1].w};
            }
            if constexpr (BLK) {
              const DF a{hv[2 * t], lv[2 * t]};
              const DF bb{hv[2 * t + 1], lv[2 * t + 1]};
  #pragma unroll
              for (int v = 0; v < VEC; v++) {
                acc[0][v] = df_add(acc[0][v], df_add(df_mul(a, xu[v]), df_mul(bb, xw[v])));
                acc[1][v] = df_add(acc[1][v], df_add(df_mul(a, xw[v]), df_neg(df_mul(bb, xu[v]))));
              }
            } else {
              const DF a{hv[t], lv[t]};
  #pragma unroll
              for (int v = 0; v < VEC; v++) acc[0][v] = df_add(acc[0][v], df_mul(a, xu[v]));
            }
          }
        }
        if constexpr (!HOIST) load_sources();
        const DF mr{mhi[row], mlo[row]};
        const float mrf = mhi[row];
        const float imrf = 1.0f / mrf;  // once per row: the M^-1-norm terms of its lanes
        const float gr = gdiag ? gdiag[row] : 0.f;
        if (++chain == kFlushRows) {
          chain = 0;
  #pragma unroll
          for (int v = 0; v < VEC; v++) {
            d1[v].flush();
            d2[v].flush();
            e2[v].flush();
            x2[v].flush();
          }
        }
  #pragma unroll
        for (int b = 0; b < NS; b++) {
          const int64_t off = row * rowW + (int64_t)b * W + l0;
          DF xo[VEC];
          {
            const float4* xp = reinterpret_cast<const float4*>(x + off);
            const float4 a = __ldg(xp), c = __ldg(xp + 1);
            xo[0] = DF{a.x, a.y}, xo[1] = DF{a.z, a.w}, xo[2] = DF{c.x, c.y}, xo[3] = DF{c.z, c.w};
          }
          Pack<float> ro, po, zo;
  #pragma unroll
          for (int v = 0; v < VEC; v++) zo.v[v] = 0.f;
          if constexpr (CPLX) {
  #pragma unroll
            for (int v = 0; v < VEC; v += 2) {
              const DF e0 = se0[b][v / 2], g0 = sg0[b][v / 2];
              const float x0 = sx0[b][v / 2];
              // r_re = e0 - (m d_re - s acc_im),  r_im = -s g0 - (m d_im + s acc_re)
              const DF q_re = df_add(df_mul(mr, xo[v]), df_neg(df_mul(sh[v], acc[b][v + 1])));
              const DF q_im = df_add(df_mul(mr, xo[v + 1]), df_mul(sh[v], acc[b][v]));
              const DF rre = df_add(e0, df_neg(q_re));
              const DF rim = df_neg(df_add(df_mul(sh[v], g0), q_im));
              const float tre = rre.hi + rre.lo, tim = rim.hi + rim.lo;
              float zre = tre, zim = tim;
              if (gdiag) {
                const float bg = shf[v] * gr;
                const float inv = 1.f / __fmaf_rn(mrf, mrf, bg * bg);
                zre = __fmaf_rn(tre, mrf, tim * bg) * inv;
                zim = __fmaf_rn(tim, mrf, -(tre * bg)) * inv;
              }
              ro.v[v] = tre;
              ro.v[v + 1] = tim;
              po.v[v] = zre;
              po.v[v + 1] = zim;
              d1[v].add_sum(__fmaf_rn(tre, zre, -(tim * zim)));
              d1[v + 1].add_sum(__fmaf_rn(tre, zim, tim * zre));
              const float nn = __fmaf_rn(tre, tre, tim * tim);
              d2[v / 2].add_sum(nn);
              e2[v / 2].add_sum(nn * imrf);
              const float xr = x0 + xo[v].hi;
              x2[v / 2].add_sum(mrf * xr * xr);  // the filtered field is the real part
            }
          } else {
  #pragma unroll
            for (int v = 0; v < VEC; v++) {
              const DF e0 = se0[b][v], g0 = sg0[b][v];
              const float x0 = sx0[b][v];
              const DF q = df_add(df_mul(mr, xo[v]), df_mul(sh[v], acc[b][v]));
              const DF rv = df_add(df_add(e0, df_neg(df_mul(sh[v], g0))), df_neg(q));
              const float t = rv.hi + rv.lo;
              const float z = gdiag ? t / __fmaf_rn(shf[v], gr, mrf) : t;
              ro.v[v] = t;
              po.v[v] = z;
              d1[v].add(t, z);
              d2[v].add(t, t);
              e2[v].add_sum(t * t * imrf);
              const float xr = x0 + xo[v].hi;
              x2[v].add_sum(mrf * xr * xr);
            }
          }
          if (all) {
            stp(r + off, ro);
            stp(p + off, po);
            stp(d + off, zo);
          } else {
  #pragma unroll
            for (int v = 0; v < VEC; v++)
              if (mine[v]) {
                r[off + v] = ro.v[v];
                p[off + v] = po.v[v];
                d[off + v] = 0.f;
              }
          }
        }
      }
    }
    if ((int)threadIdx.x < ncnt) {
      s_w[buf ^ 1][threadIdx.x] = nw;
      s_o[buf ^ 1][threadIdx.x] = no;
    }
    __syncthreads();  // the buffer is free for the tile after next; the next tile's layout is visible
  }
  if (failed) {
    // leave no bulk copy writing into this block's shared memory after it exits
    if (threadIdx.x == 0) {
      const int b0 = it & 1, b1 = b0 ^ 1;
      if (inflight & (1u << b0)) (void)mbar_wait_bounded(&bar[b0], (uint32_t)((it >> 1) & 1));
      if (inflight & (1u << b1)) (void)mbar_wait_bounded(&bar[b1], (uint32_t)(((it + 1) >> 1) & 1));
      atomicExch(C.live + 3, 1);
    }
    return;
  }
  if (tr < RPP) {
#pragma unroll
    for (int v = 0; v < VEC; v++) sm[tr * NSL + l0 + v] = d1[v].get();
    if constexpr (CPLX) {
#pragma unroll
      for (int v = 0; v < VEC / 2; v++) {
        sm[tr * NSL + W + l0 / 2 + v] = d2[v].get();
        sm[tr * NSL + W + ncolsW + l0 / 2 + v] = e2[v].get();
        sm[tr * NSL + W + 2 * ncolsW + l0 / 2 + v] = x2[v].get();
      }
    } else {
#pragma unroll
      for (int v = 0; v < VEC; v++) {
        sm[tr * NSL + W + l0 + v] = d2[v].get();
        sm[tr * NSL + W + ncolsW + l0 + v] = e2[v].get();
        sm[tr * NSL + W + 2 * ncolsW + l0 + v] = x2[v].get();
      }
    }
  }
  __syncthreads();
  for (int l = threadIdx.x; l < NSL; l += kBlock) {
    double s = 0.0;
    for (int t = 0; t < RPP; t++) s += sm[t * NSL + l];
    partial[(int64_t)blockIdx.x * P.pstride + l] = s;
  }
}

// ------------------------------------------------------------------ host side

// Error of the launch just made (or a stale one left by an earlier call), with
// the launch geometry in the message.
void launch_check(const char* what, int blocks, size_t smem, int W) {
  static const bool trace = [] {
    const char* t = getenv("IFILT_TRACE");
    return t && t[0] == '1';
  }();
  if (trace) fprintf(stderr, "ifilt trace: %s blocks=%d W=%d pending=%s\n", what, blocks, W,
                     cudaGetErrorString(cudaPeekAtLastError()));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    fail(e == cudaErrorMemoryAllocation ? IFILT_ENOMEM : IFILT_ECUDA, "%s launch (blocks=%d, smem=%zu, W=%d): %s",
         what, blocks, smem, W, cudaGetErrorString(e));
}

// Lane tiles of an engine: [row][sub][lane] arrays, reallocated when columns
// are admitted or retired.
template <typename T>
struct Tiles {
  int W = 0;
  T *d = nullptr, *r = nullptr, *p = nullptr, *q = nullptr;
  double* x64 = nullptr;
  void* base = nullptr;
  int64_t bytes = 0;
};

template <typename T>
Tiles<T> alloc_tiles(int64_t n, int NS, int W, cudaStream_t st) {
  Tiles<T> t;
  t.W = W;
  const size_t vb = ((size_t)n * NS * W * sizeof(T) + 255) / 256 * 256;
  const size_t xb = ((size_t)n * NS * W * sizeof(double) + 255) / 256 * 256;
  t.bytes = (int64_t)(4 * vb + xb);
  char* b = (char*)scratch_alloc(4 * vb + xb, st);
  t.base = b;
  t.d = (T*)b;
  t.r = (T*)(b + vb);
  t.p = (T*)(b + 2 * vb);
  t.q = (T*)(b + 3 * vb);
  t.x64 = (double*)(b + 4 * vb);
  return t;
}

// Host copy of the per-column state, for retiring and re-packing columns.
struct HostCols {
  std::vector<double> shift, rho, alpha, beta, rn2, target2, r0n2, tol2, rel, err;
  std::vector<int> active, done, iters, rounds, status, refresh, round_it0, round_cap, restart;
  void resize(int n) {
    for (auto* v : {&shift, &rn2, &target2, &r0n2, &tol2, &rel, &err}) v->assign(n, 0.0);
    for (auto* v : {&rho, &alpha, &beta}) v->assign(2 * n, 0.0);
    for (auto* v : {&active, &done, &iters, &rounds, &status, &refresh, &round_it0, &round_cap, &restart})
      v->assign(n, 0);
  }
  // entry j of this <- entry c of h
  void take(int j, const HostCols& h, int c) {
    shift[j] = h.shift[c];
    for (int t = 0; t < 2; t++) {
      rho[2 * j + t] = h.rho[2 * c + t];
      alpha[2 * j + t] = h.alpha[2 * c + t];
      beta[2 * j + t] = h.beta[2 * c + t];
    }
    rn2[j] = h.rn2[c];
    target2[j] = h.target2[c];
    r0n2[j] = h.r0n2[c];
    tol2[j] = h.tol2[c];
    rel[j] = h.rel[c];
    err[j] = h.err[c];
    active[j] = h.active[c];
    done[j] = h.done[c];
    iters[j] = h.iters[c];
    rounds[j] = h.rounds[c];
    status[j] = h.status[c];
    refresh[j] = h.refresh[c];
    round_it0[j] = h.round_it0[c];
    round_cap[j] = h.round_cap[c];
    restart[j] = h.restart[c];
  }
};

void cols_download(const Cols& C, HostCols& H, int n, cudaStream_t st) {
  H.resize(n);
  auto dn = [&](void* dst, const void* src, size_t b) {
    IFILT_CUDA(cudaMemcpyAsync(dst, src, b, cudaMemcpyDeviceToHost, st));
  };
  dn(H.shift.data(), C.shift, n * 8);
  dn(H.rho.data(), C.rho, 2 * n * 8);
  dn(H.alpha.data(), C.alpha, 2 * n * 8);
  dn(H.beta.data(), C.beta, 2 * n * 8);
  dn(H.rn2.data(), C.rn2, n * 8);
  dn(H.target2.data(), C.target2, n * 8);
  dn(H.r0n2.data(), C.r0n2, n * 8);
  dn(H.tol2.data(), C.tol2, n * 8);
  dn(H.rel.data(), C.rel, n * 8);
  dn(H.err.data(), C.err, n * 8);
  dn(H.active.data(), C.active, n * 4);
  dn(H.done.data(), C.done, n * 4);
  dn(H.iters.data(), C.iters, n * 4);
  dn(H.rounds.data(), C.rounds, n * 4);
  dn(H.status.data(), C.status, n * 4);
  dn(H.refresh.data(), C.refresh, n * 4);
  dn(H.round_it0.data(), C.round_it0, n * 4);
  dn(H.round_cap.data(), C.round_cap, n * 4);
  dn(H.restart.data(), C.restart, n * 4);
  IFILT_CUDA(cudaStreamSynchronize(st));
}

void cols_upload(const Cols& C, const HostCols& H, int n, cudaStream_t st) {
  auto up = [&](void* dst, const void* src, size_t b) {
    IFILT_CUDA(cudaMemcpyAsync(dst, src, b, cudaMemcpyHostToDevice, st));
  };
  up(C.shift, H.shift.data(), n * 8);
  up(C.rho, H.rho.data(), 2 * n * 8);
  up(C.alpha, H.alpha.data(), 2 * n * 8);
  up(C.beta, H.beta.data(), 2 * n * 8);
  up(C.rn2, H.rn2.data(), n * 8);
  up(C.target2, H.target2.data(), n * 8);
  up(C.r0n2, H.r0n2.data(), n * 8);
  up(C.tol2, H.tol2.data(), n * 8);
  up(C.rel, H.rel.data(), n * 8);
  up(C.err, H.err.data(), n * 8);
  up(C.active, H.active.data(), n * 4);
  up(C.done, H.done.data(), n * 4);
  up(C.iters, H.iters.data(), n * 4);
  up(C.rounds, H.rounds.data(), n * 4);
  up(C.status, H.status.data(), n * 4);
  up(C.refresh, H.refresh.data(), n * 4);
  up(C.round_it0, H.round_it0.data(), n * 4);
  up(C.round_cap, H.round_cap.data(), n * 4);
  up(C.restart, H.restart.data(), n * 4);
  IFILT_CUDA(cudaStreamSynchronize(st));  // the host vectors must outlive the copies
}

// T: arithmetic and Krylov-vector type; MV: stored operator values; TM: stored
// multigrid work vectors (T in every engine the library builds; FP16 and BF16
// storage were measured and dropped).
template <typename T, typename MV, typename TM, bool CPLX, bool BLK>
class EngineT final : public Engine {
  static constexpr int VEC = Pack<T>::N;
  static constexpr int VM = 16 / (int)sizeof(TM);  // lanes per thread in the multigrid kernels (16-byte loads)
  static constexpr int NS = BLK ? 2 : 1;
  static constexpr int LPC = CPLX ? 2 : 1;  // lanes per column
  static constexpr int NVAL = BLK ? 2 : 1;

  struct Source {
    const double* field = nullptr;
    int sys = 0;
    double* buf = nullptr;  // e0, x0, g0 [n][NS] (FP64 or double-float pairs), x0 as float [n][NS]
    int refs = 0;
  };
  struct Slot {
    ColumnJob job;
    int src = -1;
    bool retired = false;
  };

 public:
  EngineT(ifilt_mesh_s* m, const ifilt_solve_opts& o, cudaStream_t st, int64_t budget)
      : m_(m), o_(o), st_(st), budget_(budget) {
    const HostPrepared& h = m->host;
    n_ = h.n_rows;
    // the operator G of S = M + shift G: K for order 1 and the complex n = 2 form, K M^-1 K for the
    // real n = 2 form, G_n for the orders above
    op_ = CPLX ? 1 : o.order;
    if (op_ >= 3 && (size_t)(op_ - 3) >= m->ell_gn.size()) fail(IFILT_EINVAL, "mesh holds no order-%d operator", op_);
    E_ = op_ == 1 ? &m->ell_k : (op_ == 2 ? &m->ell_g2 : &m->ell_gn[(size_t)op_ - 3]);
    A_ = ell_view<MV>(*E_);
    A64_ = ell_view<double>(*E_);
    A_.rowq = A64_.rowq = nullptr;  // the Krylov product runs every row to its slice's width
    int lanes = o.max_lanes > 0 ? o.max_lanes : 256;
    lanes = std::min(lanes, kBlock * VEC) / 4 * 4;
    if (lanes < 4) fail(IFILT_EINVAL, "max_lanes must allow at least 4 lanes");
    wcap_ = lanes;
    ncap_ = wcap_ / LPC;
    entry_bytes_ = 4 + NVAL * sizeof(MV);
    if (stage_bytes(1) > (size_t)kStageMax)
      fail(IFILT_EINVAL, "ELL slice of %d rows x %d entries exceeds the shared-memory stage", E_->slice_h,
           E_->max_width);
    int dev = 0;
    IFILT_CUDA(cudaGetDevice(&dev));
    IFILT_CUDA(cudaDeviceGetAttribute(&n_sms_, cudaDevAttrMultiProcessorCount, dev));
    nb_max_ = n_sms_ * (2048 / kBlock);
    IFILT_CUDA(cudaFuncSetAttribute((const void*)spmm_fn(), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)(kBlock * VEC * sizeof(double) +
                                          2 * std::max(stage_bytes(1), (size_t)kStageBytes))));
    if constexpr (sizeof(T) == 4)
      IFILT_CUDA(cudaFuncSetAttribute((const void*)residual_df_kernel<CPLX, BLK>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)(smem_of(wcap_ > 0 ? wcap_ : 4, 8, 4) + 16 +
                                            2 * std::max(res_stage_bytes(1), (size_t)kStageBytes))));
    // fixed part: partial sums, column state, tables
    size_t total = (size_t)nb_max_ * 8 * wcap_ * 8 + (size_t)ncap_ * (8 * 18 + 4 * 12 + 4 * 8) +
                   (size_t)wcap_ * 8 + 64 * 256;
    char* cur = (char*)scratch_alloc(total, st_);
    fixed_ = cur;
    fixed_bytes_ = (int64_t)total;
    auto take = [&](size_t bytes) {
      char* p = cur;
      cur += (bytes + 255) / 256 * 256;
      return (void*)p;
    };
    partial_ = (double*)take((size_t)nb_max_ * 4 * wcap_ * 8);
    partial2_ = (double*)take((size_t)nb_max_ * 4 * wcap_ * 8);
    C_.shift = (double*)take(ncap_ * 8);
    C_.rho = (double*)take(2 * ncap_ * 8);
    C_.alpha = (double*)take(2 * ncap_ * 8);
    C_.beta = (double*)take(2 * ncap_ * 8);
    C_.rn2 = (double*)take(ncap_ * 8);
    C_.target2 = (double*)take(ncap_ * 8);
    C_.r0n2 = (double*)take(ncap_ * 8);
    C_.tol2 = (double*)take(ncap_ * 8);
    C_.rel = (double*)take(ncap_ * 8);
    C_.err = (double*)take(ncap_ * 8);
    C_.active = (int*)take(ncap_ * 4);
    C_.done = (int*)take(ncap_ * 4);
    C_.iters = (int*)take(ncap_ * 4);
    C_.rounds = (int*)take(ncap_ * 4);
    C_.status = (int*)take(ncap_ * 4);
    C_.refresh = (int*)take(ncap_ * 4);
    C_.round_it0 = (int*)take(ncap_ * 4);
    C_.round_cap = (int*)take(ncap_ * 4);
    C_.restart = (int*)take(ncap_ * 4);
    C_.live = (int*)take(4 * 4);
    tune_live_ = (int*)take(4 * 4);
    lane_src_ = (int*)take(wcap_ * 4);
    lane_map_ = (int*)take(wcap_ * 4);
    flags_ = (int*)take(ncap_ * 4);
    bptr_ = (const double**)take(ncap_ * 8);
    col_out_ = (double**)take(ncap_ * 8);
    col_in_ = (const double**)take(ncap_ * 8);
    IFILT_CUDA(cudaMemsetAsync(C_.live, 0, 16, st_));
    {
      const int one[4] = {1, 0, 0, 0};
      IFILT_CUDA(cudaMemcpyAsync(tune_live_, one, sizeof one, cudaMemcpyHostToDevice, st_));
      IFILT_CUDA(cudaStreamSynchronize(st_));
    }
    IFILT_CUDA(cudaMallocHost(&h_cnt_, 8 * sizeof(int)));
    P_.n = (int32_t)n_;
    P_.maxit = o.max_iter > 0 ? o.max_iter : 100000;
    P_.tol2_rel = o.tol * o.tol;
    P_.err2 = o.err_tol * o.err_tol;
    const double itol = (sizeof(T) == 8) ? 0.0 : (o.inner_tol > 0 ? o.inner_tol : 1e-4);
    P_.inner2 = itol * itol;
    P_.wmax = E_->max_width;
    // iterations per step: a multigrid iteration costs several plain ones and
    // its rounds are short, so its columns are checked more often
    m_it_ = o.check_every > 0 ? o.check_every : (o.precond == IFILT_PRECOND_MG ? 8 : 32);
    const char* ng = getenv("IFILT_NO_GRAPH");
    use_graph_ = !(ng && ng[0] == '1');
    // experiment knob: damped-Jacobi sweeps before and after the coarse correction on levels >= 1
    if (const char* cs = getenv("IFILT_MG_COARSE_SWEEPS")) mg_nu_c_ = std::max(1, std::min(6, atoi(cs)));
    if (const char* fs = getenv("IFILT_MG_FINE_SWEEPS")) mg_nu_f_ = std::max(1, std::min(6, atoi(fs)));
    // double-float refinement residual on the FP32 engines, unless a tolerance asks for more than its
    // about 48 bits carry on hard columns; then FP64, as on the FP64 engine
    df_ = sizeof(T) == 4 && o.tol >= kDfMinTol && (!(o.err_tol > 0.0) || o.err_tol >= kDfMinErrTol);
    if (o.precond == IFILT_PRECOND_MG) mg_setup();
    P_.mg = mg_on_ ? 1 : 0;
    P_.rn_slot = (!CPLX && o.precond == IFILT_PRECOND_JACOBI) ? 1 : 0;
    prof_ = profiling_on();
  }

  ~EngineT() override {
    cudaStreamSynchronize(st_);
    if (exec_) cudaGraphExecDestroy(exec_);
    if (graph_) cudaGraphDestroy(graph_);
    for (auto& s : src_)
      if (s.buf) scratch_free(s.buf, st_);
    if (tl_.base) scratch_free(tl_.base, st_);
    if (mg_base_) scratch_free(mg_base_, st_);
    if (fixed_) scratch_free(fixed_, st_);
    if (h_cnt_) cudaFreeHost(h_cnt_);
    for (auto& e : pev_)
      if (e) cudaEventDestroy(e);
    cudaStreamSynchronize(st_);
  }

  void submit(const std::vector<ColumnJob>& jobs) override {
    for (const auto& j : jobs) pend_.push_back(j);
  }
  bool idle() const override { return live_columns() == 0 && pend_.empty(); }
  int64_t bytes_held() const override {
    int64_t b = fixed_bytes_ + tl_.bytes + mg_bytes_;
    for (auto& s : src_)
      if (s.buf) b += src_bytes();
    return b;
  }
  int running() const override { return live_columns(); }
  void set_budget(int64_t budget) override { budget_ = budget; }
  int pending() const override { return (int)pend_.size(); }
  cudaStream_t stream() const override { return st_; }

 private:
  int live_columns() const {
    int c = 0;
    for (auto& s : cur_)
      if (s.src >= 0 && !s.retired) c++;
    return c;
  }
  // lanes of a tile: a multiple of the lanes one thread moves (4, or VM in the multigrid kernels)
  int lanes_for(int ncol) const {
    const int g = mg_on_ ? std::max(4, VM) : 4;
    return (ncol * LPC + g - 1) / g * g;
  }
  size_t smem_of(int W, int slots2, int vec = VEC) const {
    return (size_t)(kBlock / (W / vec)) * (size_t)W * slots2 / 2 * sizeof(double);
  }
  // SpMM instance: gathers issued EB entries at a time (4 when no row holds
  // more, as for the cell operator); FP32 2x2 blocks trade occupancy for more
  // loads in flight per thread.
  using SpmmFn = void (*)(EllView<MV>, Params, int, const T*, T*, const T*, Cols, double*, MgArgs<T, T, T>);
  static constexpr int kMinB = (BLK && sizeof(T) == 4) ? IFILT_SPMM_MINB_BLK : IFILT_SPMM_MINB;
  SpmmFn spmm_fn() const {
    if constexpr (sizeof(T) == 8) return spmm_kernel<T, MV, T, T, T, VEC, CPLX, BLK, 4, kMinB>;
    else if constexpr (BLK) return spmm_kernel<T, MV, T, T, T, VEC, CPLX, BLK, IFILT_SPMM_EB_BLK, kMinB>;
    else
      return E_->max_width <= 4 ? spmm_kernel<T, MV, T, T, T, VEC, CPLX, BLK, 4, kMinB>
                                : spmm_kernel<T, MV, T, T, T, VEC, CPLX, BLK, 8, kMinB>;
  }
  // ELL entries of a stage buffer holding `spt` slices (each slice starts on an
  // 8-entry boundary, so a slice spans at most 7 entries more than it holds)
  int64_t stage_entries(int spt) const { return (int64_t)spt * ((int64_t)E_->slice_h * E_->max_width + 8); }
  size_t stage_bytes(int spt) const {
    const int64_t e = stage_entries(spt);
    return (size_t)((e * 4 + 15) / 16 * 16 + (e * NVAL * (int64_t)sizeof(MV) + 15) / 16 * 16 +
                    ((int64_t)spt * E_->slice_h + 15) / 16 * 16);
  }
  int spmm_spt(int W) const {
    const int RPP = kBlock / (W / VEC);
    int spt = std::max(1, (RPP * tp_cg_ + E_->slice_h - 1) / E_->slice_h);
    while (spt > 1 && stage_bytes(spt) > (size_t)kStageBytes) spt--;
    // keep several tiles per resident block so that the grid ends evenly
    const long long want = (long long)n_sms_ * kMinB * 8;
    while (spt > 1 && (E_->n_slices + spt - 1) / spt < want) spt--;
    return std::min(spt, kMaxSpt);
  }
  size_t spmm_smem(int W) const { return smem_of(W, 2) + 2 * stage_bytes(spmm_spt(W)); }
  // the double-float residual's stage: column indices and the operator's hi and lo values
  size_t res_stage_bytes(int spt) const {
    const int64_t e = stage_entries(spt);
    return (size_t)((e * 4 + 15) / 16 * 16 + 2 * ((e * NVAL * 4 + 15) / 16 * 16));
  }
  int res_spt(int W) const {
    const int RPP = kBlock / (W / 4);
    int spt = std::max(1, (RPP * kTilePasses + E_->slice_h - 1) / E_->slice_h);
    while (spt > 1 && res_stage_bytes(spt) > (size_t)kStageBytes) spt--;
    const long long want = (long long)n_sms_ * 2 * 8;  // several tiles per resident block
    while (spt > 1 && (E_->n_slices + spt - 1) / spt < want) spt--;
    return std::min(spt, kMaxSpt);
  }
  int blocks_for(int W) const {
    const long long ntiles = (E_->n_slices + spmm_spt(W) - 1) / spmm_spt(W);
    int nb = std::min(nb_max_, grid_for((const void*)spmm_fn(), kBlock, spmm_smem(W), ntiles * kBlock));
    if (bpsm_cg_ > 0) nb = std::min(nb, n_sms_ * bpsm_cg_);
    return nb;
  }
  size_t src_bytes() const { return (size_t)n_ * NS * (3 * sizeof(double) + sizeof(float)); }
  const T* mass_t() const {
    if constexpr (sizeof(T) == 4) return m_->mass32;
    else return m_->mass;
  }
  // diagonal of G for Jacobi preconditioning (nullptr: none)
  const double* gdiag64() const {
    if (o_.precond != IFILT_PRECOND_JACOBI) return nullptr;
    return op_ == 1 ? m_->diag_k : (op_ == 2 ? m_->diag_g2 : m_->diag_gn[(size_t)op_ - 3]);
  }
  const T* gdiag_t() const {
    if (o_.precond != IFILT_PRECOND_JACOBI) return nullptr;
    if constexpr (sizeof(T) == 4)
      return op_ == 1 ? m_->diag_k32 : (op_ == 2 ? m_->diag_g2_32 : m_->diag_gn32[(size_t)op_ - 3]);
    else return gdiag64();
  }
  int64_t tile_bytes(int W) const {
    return (int64_t)n_ * NS * W * (4 * sizeof(T) + sizeof(double)) + mg_tile_bytes(W);
  }
  double shift_of(double k) const {
    const double ell = 1.0 / k;
    if (o_.order == 1) return 0.5 * ell * ell;
    if (CPLX) return ell * ell / std::sqrt(2.0);
    if (o_.order == 2) return 0.5 * ell * ell * ell * ell;
    double l2n = 1.0;  // l^(2n)
    for (int i = 0; i < o_.order; i++) l2n *= ell * ell;
    return 0.5 * l2n;
  }

  // source slot (b, x0) of a (field, system), built on first use
  int source_for(const ColumnJob& j) {
    for (int s = 0; s < (int)src_.size(); s++)
      if (src_[s].buf && src_[s].field == j.field && src_[s].sys == j.sys) {
        src_[s].refs++;
        return s;
      }
    int s = -1;
    for (int t = 0; t < (int)src_.size(); t++)
      if (!src_[t].buf) s = t;
    if (s < 0) {
      if ((int)src_.size() >= ncap_) fail(IFILT_ECUDA, "source table full");
      src_.emplace_back();
      s = (int)src_.size() - 1;
    }
    Source& q = src_[s];
    q.field = j.field;
    q.sys = j.sys;
    q.buf = (double*)scratch_alloc(src_bytes(), st_);
    q.refs = 1;
    launch_rhs(m_, j.field, j.sys, q.buf, q.buf + (size_t)n_ * NS, st_);
    {  // e0 = b - M x0, g0 = G x0 and x0 as float: the residual form's fixed part
      const int g = grid_for((const void*)source_kernel<BLK>, 256, 0, n_);
      source_kernel<BLK><<<g, 256, 0, st_>>>(A64_, (int32_t)n_, m_->mass, q.buf);
      launch_check("source", g, 0, 0);
      other_launches_++;
    }
    if (df_) {  // e0 and g0 as double-float pairs for the double-float residual
      const int g = grid_for((const void*)to_df_kernel, kBlock, 0, n_ * NS);
      to_df_kernel<<<g, kBlock, 0, st_>>>(n_ * NS, q.buf);
      to_df_kernel<<<g, kBlock, 0, st_>>>(n_ * NS, q.buf + (size_t)2 * n_ * NS);
      other_launches_ += 2;
    }
    other_launches_++;
    return s;
  }
  void release_source(int s) {
    if (s < 0) return;
    if (--src_[s].refs == 0) {
      scratch_free(src_[s].buf, st_);
      src_[s].buf = nullptr;
      src_[s].field = nullptr;
    }
  }

  // one step: refinement prologue, m iterations, counters to the host
  void enqueue_step(bool check) {
    const int W = P_.W;
    const size_t sm2 = spmm_smem(W), sm3 = smem_of(W, 4), sm4 = smem_of(W, 8);
    const int fg = (P_.ncols + 31) / 32;
    const dim3 fb(32, 8);
    evf_ = check ? cudaEventRecordDefault : cudaEventRecordExternal;
    auto chk = [&](const char* what) {
      if (!check) return;
      cudaError_t e = cudaGetLastError();
      if (e == cudaSuccess) e = cudaStreamSynchronize(st_);
      if (e != cudaSuccess) fail(IFILT_ECUDA, "%s (W=%d, blocks=%d): %s", what, W, nb_, cudaGetErrorString(e));
    };
    // algorithmic bytes: one tile vector, the operator's entries, one per-row scalar array
    const double vb = (double)n_ * NS * W * sizeof(T);
    const double ell_b = (double)E_->entries * (4.0 + E_->nval * sizeof(MV));
    const double rows_t = (double)n_ * sizeof(T);
    const int ga = grid_for((const void*)accumulate_kernel<T, CPLX>, kBlock, 0, n_ * NS * W);
    marks_.clear();
    pmark_open();
    scan_kernel<<<1, 256, 0, st_>>>(P_.ncols, C_);
    chk("scan");
    pmark(kCatFinish, 0.0);
    // refreshed-column count of this step, for the bytes of its refinement kernels
    IFILT_CUDA(cudaMemcpyAsync(h_cnt_ + 4, C_.live, 4 * sizeof(int), cudaMemcpyDeviceToHost, st_));
    bool done_acc = false;
    if constexpr (sizeof(T) == 4) {
      if (df_) {
        accumulate_df_kernel<CPLX><<<ga, kBlock, 0, st_>>>(n_ * NS * W, W, C_.refresh,
                                                          reinterpret_cast<DF*>(tl_.x64), tl_.d, C_.live);
        done_acc = true;
      }
    }
    if (!done_acc)
      accumulate_kernel<T, CPLX><<<ga, kBlock, 0, st_>>>(n_ * NS * W, W, C_.refresh, tl_.x64, tl_.d, C_.live);
    chk("accumulate");
    pmark(kCatAccumulate, 0.0);  // bytes follow the refreshed lanes (settle)
    int nbr = nb_;
    bool done_res = false;
    if constexpr (sizeof(T) == 4) {
      if (df_) {
        Params Qr = P_;
        Qr.spt = res_spt(W);
        Qr.stage_e = (int)stage_entries(Qr.spt);
        const size_t smr = sm4 + 16 + 2 * res_stage_bytes(Qr.spt);
        const long long rtiles = (E_->n_slices + Qr.spt - 1) / Qr.spt;
        const int nr = std::min(nb_max_, grid_for((const void*)residual_df_kernel<CPLX, BLK>, kBlock, smr,
                                                  rtiles * kBlock));
        nbr = nr;
        done_res = true;
        residual_df_kernel<CPLX, BLK><<<nr, kBlock, smr, st_>>>(
            ell_view<float>(*E_), E_->val32lo, Qr, reinterpret_cast<const DF*>(tl_.x64),
            reinterpret_cast<const DF* const*>(bptr_), lane_src_, m_->mass32, m_->mass32lo, C_, tl_.r, tl_.d, tl_.p,
            partial_, gdiag_t());
      }
    }
    if (!done_res)
      residual_kernel<T, CPLX, BLK><<<nb_, kBlock, sm4, st_>>>(A64_, P_, tl_.x64, bptr_, lane_src_, m_->mass, C_,
                                                              tl_.r, tl_.d, tl_.p, partial_, gdiag64());
    chk("residual");
    pmark(kCatResidual, 0.0);  // bytes follow the refreshed lanes (settle)
    finish_residual_kernel<CPLX><<<fg, fb, 0, st_>>>(P_, nbr, partial_, C_);
    chk("finish_residual");
    scan_kernel<<<1, 256, 0, st_>>>(P_.ncols, C_);
    pmark(kCatFinish, 0.0);
    const double pre_b = gdiag_t() ? 2.0 * rows_t : 0.0;
    for (int it = 0; it < m_it_; it++) {
      if (mg_on_) {
        // preconditioned order: z = V(r), beta from <r, z>, p = z + beta p, then q = S p ...
        // z = V(r) into q (free until the SpMM below); after the first iteration of the step the
        // update kernel has already written the finest level's first sweep
        vcycle(0, tl_.r, tl_.q, it > 0);
        const T* z = tl_.q;
        chk("vcycle");
        finish_rho_kernel<CPLX><<<fg, fb, 0, st_>>>(P_, nbz_, partial2_, C_);
        chk("finish_rho");
        pmark(kCatFinish, 0.0);
        direction_kernel<T, T, CPLX, BLK, false><<<nbd_, kBlock, 0, st_>>>(P_, tl_.p, z, C_, mass_t(), nullptr);
        chk("direction");
        pmark(kCatDirection, 3.0 * vb);
      }
      spmm_fn()<<<nb_, kBlock, sm2, st_>>>(A_, P_, E_->n_slices, tl_.p, tl_.q, mass_t(), C_, partial_,
                                            MgArgs<T, T, T>{});
      chk("spmm");
      pmark(kCatSpmm, 2.0 * vb + ell_b + rows_t);
      finish_alpha_kernel<CPLX><<<fg, fb, 0, st_>>>(P_, nb_, partial_, C_);
      chk("finish_alpha");
      pmark(kCatFinish, 0.0);
      bool mgj = false;  // this update also writes the next iteration's first fine sweep
      if constexpr (sizeof(T) == 4) mgj = mg_on_ && it + 1 < m_it_;
      if (gdiag_t())
        update_kernel<T, CPLX, BLK, true><<<nbu_, kBlock, sm3, st_>>>(P_, tl_.d, tl_.p, tl_.r, tl_.q, C_, partial_,
                                                                    mass_t(), gdiag_t(), nullptr, (T)0);
      else if (mgj) {
        if constexpr (sizeof(T) == 4)
          update_kernel<T, CPLX, BLK, false, true><<<nbu_, kBlock, sm3, st_>>>(
              P_, tl_.d, tl_.p, tl_.r, tl_.q, C_, partial_, mass_t(), m_->diag_k32, mgb_[0].a, (T)(*mgl_)[0].omega);
      } else
        update_kernel<T, CPLX, BLK, false><<<nbu_, kBlock, sm3, st_>>>(P_, tl_.d, tl_.p, tl_.r, tl_.q, C_,
                                                                     partial_, mass_t(), nullptr, nullptr, (T)0);
      chk("update");
      pmark(kCatUpdate, 6.0 * vb + pre_b + (mgj ? vb + 2.0 * rows_t : 0.0));
      finish_beta_kernel<CPLX><<<fg, fb, 0, st_>>>(P_, nbu_, partial_, C_);
      chk("finish_beta");
      pmark(kCatFinish, 0.0);
      if (mg_on_) continue;
      if (gdiag_t())
        direction_kernel<T, T, CPLX, BLK, true><<<nbd_, kBlock, 0, st_>>>(P_, tl_.p, tl_.r, C_, mass_t(), gdiag_t());
      else
        direction_kernel<T, T, CPLX, BLK, false><<<nbd_, kBlock, 0, st_>>>(P_, tl_.p, tl_.r, C_, mass_t(), nullptr);
      chk("direction");
      pmark(kCatDirection, 3.0 * vb + pre_b);
    }
    scan_kernel<<<1, 256, 0, st_>>>(P_.ncols, C_);
    pmark(kCatFinish, 0.0);
    marking_ = false;
    IFILT_CUDA(cudaMemcpyAsync(h_cnt_, C_.live, 4 * sizeof(int), cudaMemcpyDeviceToHost, st_));
  }
  // (with multigrid the updates of all but the last iteration replace the next cycle's first fine sweep)
  int launches_per_step() const {
    return 7 + 5 * m_it_ + (mg_on_ ? m_it_ * (mg_launches() + 1) - (m_it_ - 1) : 0);
  }

  void capture() {
    if (exec_) cudaGraphExecDestroy(exec_);
    if (graph_) cudaGraphDestroy(graph_);
    exec_ = nullptr;
    graph_ = nullptr;
    autotune();
    nb_ = blocks_for(P_.W);
    // the streaming kernels get their own grids: as many resident blocks as fit
    const long long rows_threads = (long long)n_ * (P_.W / VEC);
    const bool pre = gdiag_t() != nullptr;
    nbu_ = std::min(nb_max_, grid_for(pre ? (const void*)update_kernel<T, CPLX, BLK, true>
                                          : (const void*)update_kernel<T, CPLX, BLK, false>,
                                      kBlock, smem_of(P_.W, 4), rows_threads));
    nbd_ = std::min(nb_max_, grid_for(pre ? (const void*)direction_kernel<T, T, CPLX, BLK, true>
                                          : (const void*)direction_kernel<T, T, CPLX, BLK, false>,
                                      kBlock, 0, rows_threads));
    launch_check("before capture", nb_, 0, P_.W);
    if (!use_graph_) return;
    IFILT_CUDA(cudaStreamBeginCapture(st_, cudaStreamCaptureModeThreadLocal));
    enqueue_step(false);
    cudaError_t cap = cudaStreamEndCapture(st_, &graph_);
    if (cap != cudaSuccess) fail(IFILT_ECUDA, "graph capture failed: %s", cudaGetErrorString(cap));
    launch_check("capture", nb_, 0, P_.W);
    IFILT_CUDA(cudaGraphInstantiate(&exec_, graph_, 0));
  }

  void set_width(int W) {
    P_.W = W;
    P_.ncols = W / LPC;
    P_.pstride = 4 * W;
    P_.spt = W > 0 ? spmm_spt(W) : 1;
    P_.stage_e = (int)stage_entries(P_.spt);
  }

  void release_tiles() {
    if (exec_) cudaGraphExecDestroy(exec_);
    if (graph_) cudaGraphDestroy(graph_);
    exec_ = nullptr;
    graph_ = nullptr;
    if (tl_.base) scratch_free(tl_.base, st_);
    tl_ = Tiles<T>{};
    mg_free();
    cur_.clear();
    set_width(0);
  }

  // Keep the running columns, admit queued ones into the free lanes (within
  // the lane capacity and the memory budget) and re-pack the tiles.
  void relayout() {
    const int nc_old = P_.ncols;
    HostCols Hold;
    if (nc_old > 0) cols_download(C_, Hold, nc_old, st_);
    std::vector<int> keep;
    for (int c = 0; c < (int)cur_.size(); c++)
      if (cur_[c].src >= 0 && !cur_[c].retired) keep.push_back(c);
    std::vector<ColumnJob> adm;
    int64_t held = bytes_held();
    int64_t new_src = 0;
    while ((int)(keep.size() + adm.size()) < ncap_ && !pend_.empty()) {
      const int Wtry = lanes_for((int)(keep.size() + adm.size()) + 1);
      const int64_t need = held + tile_bytes(Wtry) + new_src + (int64_t)src_bytes();
      if (budget_ > 0 && need > budget_ && !(keep.empty() && adm.empty())) break;
      adm.push_back(pend_.front());
      pend_.pop_front();
      new_src += (int64_t)src_bytes();
    }
    // the tiles: when the device cannot hold them, admit fewer columns
    Tiles<T> tn;
    while (true) {
      const int nr = (int)(keep.size() + adm.size());
      if (nr == 0) {
        release_tiles();
        return;
      }
      try {
        tn = alloc_tiles<T>(n_, NS, lanes_for(nr), st_);
        break;
      } catch (const Error& e) {
        if (e.status != IFILT_ENOMEM) throw;
        if (adm.empty()) {
          if (tl_.base) return;  // cannot narrow now: keep the tiles, finished lanes stay idle
          throw;
        }
        const size_t back = (adm.size() + 1) / 2;
        for (size_t i = 0; i < back; i++) {
          pend_.push_front(adm.back());
          adm.pop_back();
        }
      }
    }
    const int nreal = (int)(keep.size() + adm.size());
    const int Wn = lanes_for(nreal);
    const int ncn = Wn / LPC;
    HostCols Hn;
    Hn.resize(ncn);
    std::vector<Slot> ncur(ncn);
    std::vector<int> map(Wn, -1), fresh(ncn, 0);
    for (int j = 0; j < (int)keep.size(); j++) {
      const int c = keep[j];
      ncur[j] = cur_[c];
      Hn.take(j, Hold, c);
      for (int t = 0; t < LPC; t++) map[j * LPC + t] = c * LPC + t;
    }
    for (int i = 0; i < (int)adm.size(); i++) {
      const int j = (int)keep.size() + i;
      ncur[j].job = adm[i];
      ncur[j].src = source_for(adm[i]);
      Hn.shift[j] = shift_of(adm[i].k);
      Hn.r0n2[j] = -1.0;
      fresh[j] = 1;
    }
    for (int j = nreal; j < ncn; j++) Hn.done[j] = 1;
    const int64_t rows = n_ * NS;
    if (tl_.base && !keep.empty()) {
      IFILT_CUDA(cudaMemcpyAsync(lane_map_, map.data(), Wn * 4, cudaMemcpyHostToDevice, st_));
      const int g = grid_for((const void*)gather_lanes_kernel<T>, kBlock, 0, rows * Wn);
      gather_lanes_kernel<T><<<g, kBlock, 0, st_>>>(rows, P_.W, Wn, lane_map_, tl_.d, tn.d);
      gather_lanes_kernel<T><<<g, kBlock, 0, st_>>>(rows, P_.W, Wn, lane_map_, tl_.r, tn.r);
      gather_lanes_kernel<T><<<g, kBlock, 0, st_>>>(rows, P_.W, Wn, lane_map_, tl_.p, tn.p);
      gather_lanes_kernel<double><<<g, kBlock, 0, st_>>>(rows, P_.W, Wn, lane_map_, tl_.x64, tn.x64);
      other_launches_ += 4;
      launch_check("gather", g, 0, Wn);
      IFILT_CUDA(cudaStreamSynchronize(st_));  // lane_map_ is rewritten below
    } else {
      IFILT_CUDA(cudaMemsetAsync(tn.d, 0, (size_t)rows * Wn * sizeof(T), st_));
    }
    if (tl_.base) scratch_free(tl_.base, st_);
    tl_ = tn;
    cur_ = ncur;
    set_width(Wn);
    if (mg_on_) mg_alloc(Wn);
    upload_tables();
    cols_upload(C_, Hn, ncn, st_);
    IFILT_CUDA(cudaMemcpyAsync(flags_, fresh.data(), ncn * 4, cudaMemcpyHostToDevice, st_));
    const int g = grid_for((const void*)init_lanes_kernel<CPLX>, kBlock, 0, rows * Wn);
    init_lanes_kernel<CPLX><<<g, kBlock, 0, st_>>>(P_, NS, flags_, tl_.x64);
    other_launches_++;
    launch_check("init lanes", g, 0, Wn);
    IFILT_CUDA(cudaStreamSynchronize(st_));
    capture();
  }

  void upload_tables() {
    const HostPrepared& h = m_->host;
    const int W = P_.W, nc = P_.ncols;
    const double* any_b = nullptr;
    for (auto& s : src_)
      if (s.buf) {
        any_b = s.buf;
        break;
      }
    std::vector<const double*> bp(ncap_, any_b), ci(ncap_, nullptr);
    std::vector<double*> co(ncap_, nullptr);
    for (int s = 0; s < (int)src_.size(); s++)
      if (src_[s].buf) bp[s] = src_[s].buf;
    std::vector<int> ls(W, 0);
    for (int c = 0; c < nc; c++) {
      const Slot& sl = cur_[c];
      if (sl.src < 0) continue;
      for (int t = 0; t < LPC; t++) ls[c * LPC + t] = sl.src;
      const int comp = h.placement == IFILT_CELL ? sl.job.sys : 0;
      co[c] = sl.job.out + (int64_t)comp * h.n_out;
      ci[c] = BLK ? nullptr : sl.job.field + (int64_t)comp * h.n_in;
    }
    IFILT_CUDA(cudaMemcpyAsync(lane_src_, ls.data(), W * 4, cudaMemcpyHostToDevice, st_));
    IFILT_CUDA(cudaMemcpyAsync(bptr_, bp.data(), ncap_ * 8, cudaMemcpyHostToDevice, st_));
    IFILT_CUDA(cudaMemcpyAsync(col_out_, co.data(), ncap_ * 8, cudaMemcpyHostToDevice, st_));
    IFILT_CUDA(cudaMemcpyAsync(col_in_, ci.data(), ncap_ * 8, cudaMemcpyHostToDevice, st_));
    IFILT_CUDA(cudaStreamSynchronize(st_));
  }

  // write outputs and stats of finished columns, free their lanes' sources
  void retire(const HostCols& H, std::vector<ColumnDone>& done) {
    const HostPrepared& h = m_->host;
    const int nc = P_.ncols;
    std::vector<int> emit(nc, 0);
    bool any = false;
    for (int c = 0; c < nc; c++) {
      Slot& sl = cur_[c];
      if (sl.src < 0 || sl.retired || !H.done[c]) continue;
      emit[c] = 1;
      any = true;
    }
    if (!any) return;
    IFILT_CUDA(cudaMemcpyAsync(flags_, emit.data(), nc * 4, cudaMemcpyHostToDevice, st_));
    dim3 og((unsigned)std::min<long long>((h.n_out + kBlock - 1) / kBlock, 1024), (unsigned)nc);
    if (df_)
      output_kernel<CPLX, BLK, true><<<og, kBlock, 0, st_>>>(P_, h.n_out, m_->inv_perm, tl_.x64, bptr_, lane_src_,
                                                             col_out_, col_in_, flags_);
    else
      output_kernel<CPLX, BLK, false><<<og, kBlock, 0, st_>>>(P_, h.n_out, m_->inv_perm, tl_.x64, bptr_, lane_src_,
                                                              col_out_, col_in_, flags_);
    other_launches_++;
    launch_check("output", (int)og.x, 0, P_.W);
    IFILT_CUDA(cudaStreamSynchronize(st_));
    for (int c = 0; c < nc; c++) {
      if (!emit[c]) continue;
      Slot& sl = cur_[c];
      const bool err_bad = o_.err_tol > 0.0 && !(H.err[c] <= o_.err_tol);
      const int status = (H.status[c] != 0 || H.rel[c] > o_.tol || err_bad) ? IFILT_NOT_CONVERGED : IFILT_OK;
      if (sl.job.stat) {
        sl.job.stat->iters = H.iters[c];
        sl.job.stat->refinements = H.rounds[c];
        sl.job.stat->status = status;
        sl.job.stat->pad = 0;
        sl.job.stat->rel_residual = H.rel[c];
        sl.job.stat->err_bound = H.err[c];
      }
      done.push_back({sl.job.request, status});
      sl.retired = true;
      release_source(sl.src);
    }
  }

 public:
  void launch() override {
    if (launched_) return;
    if (live_columns() == 0) {
      if (pend_.empty()) return;
      relayout();
      if (P_.W == 0) return;
    }
    if (use_graph_) IFILT_CUDA(cudaGraphLaunch(exec_, st_));
    else enqueue_step(true);
    steps_++;
    launched_ = true;
  }

  void settle(std::vector<ColumnDone>& done) override {
    if (!launched_) return;
    IFILT_CUDA(cudaStreamSynchronize(st_));
    launched_ = false;
    const int live = h_cnt_[0], notdone = h_cnt_[2];
    (void)live;
    if (h_cnt_[3])
      fail(IFILT_DEVICE_TIMEOUT,
           "a stage copy of the SpMM, a multigrid gather or the refinement residual did not complete in its wait limit");
    if (prof_) account_step();
    const int lc = live_columns();
    if (notdone < lc) {
      HostCols H;
      cols_download(C_, H, P_.ncols, st_);
      retire(H, done);
    }
    const int run = live_columns();
    bool want = false;
    if (run < lc && run * 5 <= P_.ncols * 3) want = true;                      // narrow the tiles
    if (!pend_.empty() && ncap_ - run >= std::max(1, ncap_ / 4)) want = true;  // room for queued columns
    if (!pend_.empty() && run == 0) want = true;
    if (run == 0 && pend_.empty()) {
      release_tiles();
      return;
    }
    if (want) relayout();
  }

  void report_profile() override {
    profile_count(other_launches_ + steps_ * launches_per_step());
    other_launches_ = 0;
    if (prof_) {
      char eng[16];
      snprintf(eng, sizeof eng, "%s%s_%s", CPLX ? "c" : "r", BLK ? "b" : "s", sizeof(T) == 8 ? "f64" : "f32");
      for (int c = 0; c < kCatN; c++) {
        if (cat_n_[c] == 0) continue;
        char nm[48];
        snprintf(nm, sizeof nm, "%s_%s", kCatName[c], eng);
        profile_add(nm, cat_n_[c], cat_n_[c], cat_ms_[c], cat_bytes_[c] / (double)cat_n_[c]);
      }
      if (graph_n_ > 0) {  // every step's graph from its first to its last event (spans all categories)
        char nm[48];
        snprintf(nm, sizeof nm, "(steps)_%s", eng);
        profile_add(nm, graph_n_, graph_n_, graph_ms_, 0.0);
      }
    }
    for (int c = 0; c < kCatN; c++) cat_ms_[c] = cat_bytes_[c] = 0.0, cat_n_[c] = 0;
    graph_ms_ = 0.0;
    graph_n_ = 0;
    steps_ = 0;
  }

 private:
  ifilt_mesh_s* m_;
  ifilt_solve_opts o_;
  cudaStream_t st_;
  int64_t budget_;
  const DevEll* E_ = nullptr;
  int op_ = 1;  // which operator E_ holds: 1 = K, 2 = K M^-1 K, n = G_n
  EllView<MV> A_{};
  EllView<double> A64_{};
  int64_t n_ = 0;
  int wcap_ = 0, ncap_ = 0, nb_max_ = 0, n_sms_ = kNumSMs, nb_ = 1, nbu_ = 1, nbd_ = 1;
  size_t entry_bytes_ = 0;
  Params P_{};
  Cols C_{};
  void* fixed_ = nullptr;
  int64_t fixed_bytes_ = 0;
  double* partial_ = nullptr;
  int* lane_src_ = nullptr;
  int* lane_map_ = nullptr;
  int* flags_ = nullptr;
  const double** bptr_ = nullptr;
  double** col_out_ = nullptr;
  const double** col_in_ = nullptr;
  int* h_cnt_ = nullptr;
  Tiles<T> tl_{};
  std::vector<Slot> cur_;
  std::deque<ColumnJob> pend_;
  std::vector<Source> src_;
  cudaGraph_t graph_ = nullptr;
  cudaGraphExec_t exec_ = nullptr;
  int m_it_ = 32;
  bool use_graph_ = true, launched_ = false, prof_ = false;
  int mg_nu_c_ = 2;  // smoothing sweeps before and after the coarse correction on levels >= 1
  int mg_nu_f_ = 1;  // the same on the finest level: one sweep each side (more iterations, cheaper cycles)
  // ------------------------------------------------------------ autotuning
  // Launch shape of the gather kernels (rows per tile, blocks per SM), chosen
  // per engine kind and tile-width bucket by timing the candidates on the live
  // tiles at the first capture, and kept with the mesh for later engines.
  // The timed launches write only outputs the next iteration recomputes (q,
  // partial sums, multigrid scratch) and see a "live" flag forced to 1.
  int tp_cg_ = kTilePasses, bpsm_cg_ = 0;  // bpsm 0: occupancy
  // multigrid gathers: [0] the finest level (and its transfers), [1] the coarser levels
  int tp_mg_[2] = {kTilePasses, kTilePasses}, bpsm_mg_[2] = {0, 0};

  Cols mg_cols_{};
  int* tune_live_ = nullptr;
  std::string tune_key(int W) const {
    int wb = 4;
    while (wb < W) wb <<= 1;
    char b[96];
    snprintf(b, sizeof b, "T%d/V%d/c%d/b%d/mg%d/E%d/W%d", (int)sizeof(T), (int)sizeof(MV), (int)CPLX, (int)BLK,
             mg_on_ ? 1 : 0, op_, wb);
    return b;
  }
  void autotune() {
    mg_cols_ = C_;
    const int W = P_.W;
    if (W <= 0) return;
    const char* env = getenv("IFILT_AUTOTUNE");
    if (env && env[0] == '0') return;
    const std::string key = tune_key(W);
    {
      std::lock_guard<std::mutex> lk(m_->tune_mu);
      auto it = m_->tune.find(key);
      if (it != m_->tune.end()) {
        tp_cg_ = it->second[0];
        bpsm_cg_ = it->second[1];
        tp_mg_[0] = it->second[2];
        bpsm_mg_[0] = it->second[3];
        tp_mg_[1] = it->second[4];
        bpsm_mg_[1] = it->second[5];
        set_width(W);
        return;
      }
    }
    Cols Ct = C_;
    Ct.live = tune_live_;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    IFILT_CUDA(cudaEventCreate(&e0));
    IFILT_CUDA(cudaEventCreate(&e1));
    auto timeit = [&](auto&& launch) {
      launch();  // warm
      IFILT_CUDA(cudaEventRecord(e0, st_));
      for (int i = 0; i < 3; i++) launch();
      IFILT_CUDA(cudaEventRecord(e1, st_));
      IFILT_CUDA(cudaEventSynchronize(e1));
      float ms = 0.f;
      IFILT_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      launch_check("autotune", 0, 0, W);
      return ms;
    };
    const int tps[4] = {4, 8, 16, 32};
    int occ = 1;
    float best = 1e30f;
    int btp = kTilePasses, bb = 0;
    for (int tp : tps) {
      tp_cg_ = tp;
      bpsm_cg_ = 0;
      set_width(W);
      IFILT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, (const void*)spmm_fn(), kBlock, spmm_smem(W)));
      for (int bps : {0, occ - 1}) {  // all resident blocks, or one fewer per SM
        if (bps == occ - 1 && bps < 1) continue;
        bpsm_cg_ = bps;
        const int nb = blocks_for(W);
        const size_t sm = spmm_smem(W);
        const float ms = timeit([&] {
          spmm_fn()<<<nb, kBlock, sm, st_>>>(A_, P_, E_->n_slices, tl_.p, tl_.q, mass_t(), Ct, partial_,
                                             MgArgs<T, T, T>{});
        });
        if (ms < best) {
          best = ms;
          btp = tp;
          bb = bps;
        }
      }
    }
    tp_cg_ = btp;
    bpsm_cg_ = bb;
    if (mg_on_) {
      // the finest level's sweep sets the shape of the finest level's gathers; the first coarse
      // level's sweep (a wider, uneven operator with a (K, M) pair per entry) that of the coarser ones
      mg_cols_ = Ct;
      const int groups = mgl_->size() > 1 ? 2 : 1;
      for (int grp = 0; grp < groups; grp++) {
        best = 1e30f;
        btp = kTilePasses;
        bb = 0;
        const void* rhs = grp == 0 ? (const void*)tl_.r : (const void*)mgb_[1].r;
        for (int tp : tps) {
          for (int bps : {0, 2}) {
            tp_mg_[grp] = tp;
            bpsm_mg_[grp] = bps;
            const float ms = timeit([&] { mg_smooth((size_t)grp, mgb_[grp].a, mgb_[grp].b, rhs, nullptr); });
            if (ms < best) {
              best = ms;
              btp = tp;
              bb = bps;
            }
          }
        }
        tp_mg_[grp] = btp;
        bpsm_mg_[grp] = bb;
      }
      if (groups == 1) tp_mg_[1] = tp_mg_[0], bpsm_mg_[1] = bpsm_mg_[0];
      mg_cols_ = C_;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    set_width(W);
    std::lock_guard<std::mutex> lk(m_->tune_mu);
    m_->tune[key] = {tp_cg_, bpsm_cg_, tp_mg_[0], bpsm_mg_[0], tp_mg_[1], bpsm_mg_[1]};
  }
  // ------------------------------------------------------------ multigrid
  static constexpr int kMgMinB = 3;
  static constexpr int kMgCoarseSweeps = 4;  // Jacobi sweeps on the coarsest level
  static constexpr double kMgOmega = 2.0 / 3.0;
  struct MgBuf {
    TM* r = nullptr;  // right-hand side of the level (levels >= 1)
    TM* a = nullptr;
    TM* b = nullptr;
  };
  bool mg_on_ = false;
  const std::vector<DevMgLevel>* mgl_ = nullptr;
  std::vector<MgBuf> mgb_;
  void* mg_base_ = nullptr;
  int64_t mg_bytes_ = 0;
  double* partial2_ = nullptr;
  int nbz_ = 1;  // blocks of the last level-0 smoothing sweep (partials of <r, z>)

  // Resident blocks per SM asked of the compiler, per gather kind: the scalar-row transfers fit
  // 64 registers without spills (4 blocks: prolongation 4.6 -> 3.8 ms, restriction from the
  // finest level 2.6 -> 2.1 ms at level 10); the 2x2-block sweeps and residuals hold the row's
  // right-hand side too (fewer blocks, no spills)
  template <int EPI, int NSET>
  static constexpr int mg_minb() {
    if constexpr (!BLK && (EPI == kEpiRestrict || EPI == kEpiProlong)) return IFILT_MG_MINB_XFER;
    if constexpr (BLK && (EPI == kEpiSmooth || EPI == kEpiResid)) return IFILT_MG_MINB_BLK;
    if constexpr (NSET == 2 && EPI == kEpiResid) return IFILT_MG_MINB_CRESID;
    if constexpr (NSET == 2 && EPI == kEpiSmooth) return IFILT_MG_MINB_CSMOOTH;
    return kMgMinB;
  }
  // right-hand side type of a gather: the Krylov residual (T) for the sweeps and
  // residuals of the finest level (NSET = 1), a multigrid vector (TM) otherwise
  template <int EPI, int NSET>
  using MgTR = std::conditional_t<NSET == 1 && (EPI == kEpiSmooth || EPI == kEpiResid), T, TM>;
  // entries gathered per batch: 2x2 blocks of two sub-rows take 2 at a time when a thread moves 8
  // lanes (register room), else 4
  static constexpr int kMgEB = (BLK && VM > 4) ? 2 : 4;
  // ... and on the Galerkin levels of scalar rows (a (K, M) pair per entry, 12-16 entries a row)
  template <int NSET>
  static constexpr int mg_eb() { return (NSET == 2 && !BLK && VM == 4) ? IFILT_MG_EB_COARSE : kMgEB; }
  // output type of a gather: TM, or T for the last sweep of the finest level, whose
  // result z = V(r) enters the Krylov recursion (<r, z> and p = z + beta p): it is
  // kept unrounded so that the preconditioner stays the same symmetric operator
  // from one iteration to the next
  template <int EPI, int NSET, bool FINAL>
  using MgTO = std::conditional_t<FINAL, T, TM>;
  template <int EPI, int NSET, bool FINAL = false>
  static const void* mg_fn() {
    return (const void*)spmm_kernel<T, T, TM, MgTR<EPI, NSET>, MgTO<EPI, NSET, FINAL>, VM, CPLX, BLK, mg_eb<NSET>(),
                                    mg_minb<EPI, NSET>(), EPI, NSET>;
  }
  static int64_t stage_entries_of(const DevEll& E, int spt) {
    return (int64_t)spt * ((int64_t)E.slice_h * E.max_width + 8);
  }
  static size_t stage_bytes_of(const DevEll& E, int spt, int vbytes) {
    const int64_t e = stage_entries_of(E, spt);
    return (size_t)((e * 4 + 15) / 16 * 16 + (e * vbytes + 15) / 16 * 16 + ((int64_t)spt * E.slice_h + 15) / 16 * 16);
  }
  int spt_of(const DevEll& E, int W, int vbytes, int minb, int tp) const {
    const int RPP = kBlock / (W / VM);
    int spt = std::max(1, (RPP * tp + E.slice_h - 1) / E.slice_h);
    // two stage buffers per block, small enough that `minb` blocks fit an SM's shared memory
    const size_t cap = std::min<size_t>((size_t)kStageBytes,
                                        ((size_t)227 * 1024 / (size_t)minb - smem_of(W, 2, VM) - 2048) / 2);
    while (spt > 1 && stage_bytes_of(E, spt, vbytes) > cap) spt--;
    const long long want = (long long)n_sms_ * minb * 8;
    while (spt > 1 && (E.n_slices + spt - 1) / spt < want) spt--;
    return std::min(spt, kMaxSpt);
  }

  void mg_setup() {
    if (sizeof(T) != 4) fail(IFILT_EINVAL, "multigrid preconditioning runs with FP32 or BF16 precision");
    if (E_ != &m_->ell_k) fail(IFILT_EINVAL, "multigrid preconditioning needs order 1 or the complex n = 2 form");
    mgl_ = &multigrid_device(m_, st_);
    const int vb1 = NVAL * (int)sizeof(T), vb2 = 2 * vb1;
    for (size_t l = 0; l < mgl_->size(); l++) {
      const DevMgLevel& L = (*mgl_)[l];
      const DevEll* ells[3] = {&L.S, &L.P, &L.R};
      for (int i = 0; i < 3; i++)
        if (ells[i]->n > 0 && stage_bytes_of(*ells[i], 1, i == 0 ? vb2 : vb1) > (size_t)kStageMax)
          fail(IFILT_EINVAL, "multigrid level %zu: ELL slice exceeds the shared-memory stage", l);
    }
    if constexpr (sizeof(T) == 4) {
      const int smax = (int)(kBlock * VM * sizeof(double) + 2 * kStageMax);
      const void* fns[] = {mg_fn<kEpiSmooth, 1>(), mg_fn<kEpiSmooth, 2>(), mg_fn<kEpiResid, 1>(),
                           mg_fn<kEpiResid, 2>(), mg_fn<kEpiRestrict, 1>(), mg_fn<kEpiProlong, 1>(),
                           mg_fn<kEpiSmooth, 1, true>()};
      for (const void* f : fns)
        IFILT_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smax));
      mg_on_ = true;
    }
  }
  int64_t mg_tile_bytes(int W) const {
    if (!mg_on_) return 0;
    int64_t b = 0;
    for (size_t l = 0; l < mgl_->size(); l++) {
      const int64_t rows = l == 0 ? n_ : (*mgl_)[l].n;
      const int64_t vb = (rows * NS * W * (int64_t)sizeof(TM) + 255) / 256 * 256;
      b += (l == 0 ? 2 : 3) * vb;
    }
    return b;
  }
  void mg_free() {
    if (mg_base_) scratch_free(mg_base_, st_);
    mg_base_ = nullptr;
    mg_bytes_ = 0;
    mgb_.clear();
  }
  void mg_alloc(int W) {
    mg_free();
    mg_bytes_ = mg_tile_bytes(W);
    char* p = (char*)scratch_alloc((size_t)mg_bytes_, st_);
    mg_base_ = p;
    mgb_.resize(mgl_->size());
    for (size_t l = 0; l < mgl_->size(); l++) {
      const int64_t rows = l == 0 ? n_ : (*mgl_)[l].n;
      const int64_t vb = (rows * NS * W * (int64_t)sizeof(TM) + 255) / 256 * 256;
      if (l > 0) {
        mgb_[l].r = (TM*)p;
        p += vb;
      }
      mgb_[l].a = (TM*)p;
      p += vb;
      mgb_[l].b = (TM*)p;
      p += vb;
    }
  }

  // one gather-kernel launch on a multigrid operator; returns its block count
  // level l: the level whose rows the operation writes (restriction and prolongation: the finer one)
  template <int EPI, int NSET, bool FINAL = false>
  int mg_gather(size_t l, const DevEll& E, const TM* src, void* out, const T* mdiag, const T* kd, const void* rhs,
                const TM* own, double* partial, double omega = kMgOmega) {
    const int W = P_.W;
    const int vbytes = NVAL * NSET * (int)sizeof(T);
    Params Q = P_;
    Q.n = E.n;
    const int grp = l == 0 ? 0 : 1;
    Q.spt = spt_of(E, W, vbytes, mg_minb<EPI, NSET>(), tp_mg_[grp]);
    Q.stage_e = (int)stage_entries_of(E, Q.spt);
    const size_t smem = smem_of(W, 2, VM) + 2 * stage_bytes_of(E, Q.spt, vbytes);
    const long long ntiles = (E.n_slices + Q.spt - 1) / Q.spt;
    int blocks = std::min(nb_max_, grid_for(mg_fn<EPI, NSET, FINAL>(), kBlock, smem, ntiles * kBlock));
    if (bpsm_mg_[grp] > 0) blocks = std::min(blocks, n_sms_ * bpsm_mg_[grp]);
    using TR = MgTR<EPI, NSET>;
    using TO = MgTO<EPI, NSET, FINAL>;
    MgArgs<T, TR, TM> args{kd, static_cast<const TR*>(rhs), own, (T)omega};
    // row lengths only where rows are uneven (Galerkin levels, transfers): the finest
    // level's rows fill their slices almost exactly
    EllView<T> V = ell_view<T>(E);
    if (&E == &m_->ell_k) V.rowq = nullptr;
    spmm_kernel<T, T, TM, TR, TO, VM, CPLX, BLK, mg_eb<NSET>(), mg_minb<EPI, NSET>(), EPI, NSET><<<blocks, kBlock, smem, st_>>>(
        V, Q, E.n_slices, src, static_cast<TO*>(out), mdiag, mg_cols_, partial, args);
    return blocks;
  }
  // S_l-operations: level 0 uses the mesh's K and lumped mass, coarser levels their (K, M) pair
  // (FP32 engines only: the FP64 engine refuses multigrid in mg_setup).  Each records its
  // category and algorithmic bytes for the profile.
  int64_t mg_rows(size_t l) const { return l == 0 ? n_ : (int64_t)(*mgl_)[l].n; }
  double mg_vb(size_t l) const { return (double)mg_rows(l) * NS * P_.W * sizeof(TM); }
  // a level's right-hand side: the Krylov residual on level 0, a multigrid vector below
  double mg_vb_rhs(size_t l) const { return l == 0 ? (double)n_ * NS * P_.W * sizeof(T) : mg_vb(l); }
  double mg_ell_b(const DevEll& E, int nset) const {
    return (double)E.entries * (4.0 + (double)nset * NVAL * sizeof(T));
  }
  // final: the last sweep of the finest level, writing z = V(r) in T into `out`
  int mg_smooth(size_t l, const TM* x, void* out, const void* rhs, double* partial, bool final = false) {
    if constexpr (sizeof(T) == 4) {
      const DevMgLevel& L = (*mgl_)[l];
      int nb;
      if (final)
        nb = mg_gather<kEpiSmooth, 1, true>(l, m_->ell_k, x, out, mass_t(), m_->diag_k32, rhs, nullptr, partial,
                                            L.omega);
      else if (l == 0)
        nb = mg_gather<kEpiSmooth, 1>(l, m_->ell_k, x, out, mass_t(), m_->diag_k32, rhs, nullptr, partial, L.omega);
      else
        nb = mg_gather<kEpiSmooth, 2>(l, L.S, x, out, L.dm32, L.dk32, rhs, nullptr, partial, L.omega);
      const DevEll& S = l == 0 ? m_->ell_k : L.S;
      const double out_b = final ? (double)n_ * NS * P_.W * sizeof(T) : mg_vb(l);
      pmark(lcat(l, kCatMgSmooth0),
            mg_vb(l) + out_b + mg_vb_rhs(l) + mg_ell_b(S, l == 0 ? 1 : 2) + 2.0 * mg_rows(l) * sizeof(T));
      return nb;
    } else {
      return 0;
    }
  }
  void mg_resid(size_t l, const TM* x, TM* out, const void* rhs) {
    if constexpr (sizeof(T) == 4) {
      if (l == 0) mg_gather<kEpiResid, 1>(l, m_->ell_k, x, out, mass_t(), nullptr, rhs, nullptr, nullptr);
      else mg_gather<kEpiResid, 2>(l, (*mgl_)[l].S, x, out, (*mgl_)[l].dm32, nullptr, rhs, nullptr, nullptr);
      const DevEll& S = l == 0 ? m_->ell_k : (*mgl_)[l].S;
      pmark(lcat(l, kCatMgResid0),
            2.0 * mg_vb(l) + mg_vb_rhs(l) + mg_ell_b(S, l == 0 ? 1 : 2) + (double)mg_rows(l) * sizeof(T));
    }
  }
  void mg_transfer(size_t l, bool restrict_, const TM* src, TM* out, const TM* own) {
    if constexpr (sizeof(T) == 4) {
      const DevMgLevel& L = (*mgl_)[l];
      if (restrict_) {
        mg_gather<kEpiRestrict, 1>(l, L.R, src, out, nullptr, nullptr, nullptr, nullptr, nullptr);
        pmark(lcat(l, kCatMgRestrict0), mg_vb(l) + mg_vb(l + 1) + mg_ell_b(L.R, 1));
      } else {
        mg_gather<kEpiProlong, 1>(l, L.P, src, out, nullptr, nullptr, nullptr, own, nullptr);
        pmark(lcat(l, kCatMgProlong0), 2.0 * mg_vb(l) + mg_vb(l + 1) + mg_ell_b(L.P, 1));
      }
    }
  }
  void mg_jacobi(size_t l, const void* rhs, TM* out) {
    if constexpr (sizeof(T) == 4) {
      const int32_t rows = (int32_t)mg_rows(l);
      const T* md = l == 0 ? mass_t() : (*mgl_)[l].dm32;
      const T* kd = l == 0 ? m_->diag_k32 : (*mgl_)[l].dk32;
      Params Q = P_;
      Q.n = rows;
      const T om = (T)(*mgl_)[l].omega;
      const long long work = (long long)rows * (P_.W / VM);
      if (l == 0) {
        const int g = std::min(nb_max_, grid_for((const void*)mg_jacobi_kernel<T, T, TM, VM, CPLX, BLK>, kBlock, 0, work));
        mg_jacobi_kernel<T, T, TM, VM, CPLX, BLK><<<g, kBlock, 0, st_>>>(Q, static_cast<const T*>(rhs), out, md, kd,
                                                                        C_, om);
      } else {
        const int g = std::min(nb_max_, grid_for((const void*)mg_jacobi_kernel<T, TM, TM, VM, CPLX, BLK>, kBlock, 0, work));
        mg_jacobi_kernel<T, TM, TM, VM, CPLX, BLK><<<g, kBlock, 0, st_>>>(Q, static_cast<const TM*>(rhs), out, md,
                                                                         kd, C_, om);
      }
      pmark(lcat(l, kCatMgJacobi0), mg_vb(l) + mg_vb_rhs(l) + 2.0 * rows * sizeof(T));
    }
  }
  // One V-cycle on level l for the right-hand side rhs: nu damped-Jacobi
  // sweeps (1 on the finest level, 2 below it, unless IFILT_MG_FINE_SWEEPS /
  // IFILT_MG_COARSE_SWEEPS say otherwise), coarse correction, nu sweeps (Jacobi
  // sweeps only on the last level).  Returns the buffer holding the result.  On level 0 the last sweep
  // writes the result z in T into zout and leaves the partials of <rhs, z> in
  // partial2_.
  TM* vcycle(size_t l, const void* rhs, T* zout = nullptr, bool first_done = false) {
    MgBuf& B = mgb_[l];
    const bool last = l + 1 == mgl_->size();
    if (!first_done) mg_jacobi(l, rhs, B.a);  // else B.a holds it already (level 0, from the update)
    if (last) {
      TM* x = B.a;
      TM* y = B.b;
      for (int s = 1; s < kMgCoarseSweeps; s++) {
        const bool fin = l == 0 && s + 1 == kMgCoarseSweeps;
        const int nb = mg_smooth(l, x, fin ? (void*)zout : (void*)y, rhs, fin ? partial2_ : nullptr, fin);
        if (l == 0) nbz_ = nb;
        std::swap(x, y);
      }
      return x;
    }
    // the first pre-smoothing sweep is the Jacobi step above (from x = 0); then nu - 1 more
    TM* x = B.a;
    TM* t = B.b;
    for (int s = 1; s < mg_nu(l); s++) {
      mg_smooth(l, x, t, rhs, nullptr);
      std::swap(x, t);
    }
    // coarse correction(s): x <- x + P V_{l+1}(R (rhs - S x)), twice on levels 1 and 2 of a W12 cycle
    for (int rep = 0; rep < mg_reps(l); rep++) {
      mg_resid(l, x, t, rhs);
      mg_transfer(l, true, t, mgb_[l + 1].r, nullptr);
      const TM* xc = vcycle(l + 1, mgb_[l + 1].r);
      mg_transfer(l, false, xc, t, x);
      std::swap(x, t);
    }
    // nu post-smoothing sweeps with the same damped Jacobi operator (a symmetric cycle); the last
    // writes the result (on level 0: z in T, with the partials of <rhs, z>)
    for (int s = 1; s < mg_nu(l); s++) {
      mg_smooth(l, x, t, rhs, nullptr);
      std::swap(x, t);
    }
    const int nb = mg_smooth(l, x, l == 0 ? (void*)zout : (void*)t, rhs, l == 0 ? partial2_ : nullptr, l == 0);
    if (l == 0) nbz_ = nb;
    return t;
  }
  int mg_nu(size_t l) const { return l == 0 ? mg_nu_f_ : mg_nu_c_; }
  int mg_reps(size_t l) const { return (o_.mg_cycle == IFILT_MG_W12 && (l == 1 || l == 2)) ? 2 : 1; }
  // visits of each level in one cycle
  std::vector<int> mg_visits() const {
    std::vector<int> v(mgl_->size(), 0);
    v[0] = 1;
    for (size_t l = 0; l + 1 < v.size(); l++) v[l + 1] = v[l] * mg_reps(l);
    return v;
  }
  int mg_launches() const {
    if (!mg_on_) return 0;
    const std::vector<int> v = mg_visits();
    int n = 0;
    for (size_t l = 0; l < v.size(); l++)
      n += v[l] * (l + 1 == v.size() ? kMgCoarseSweeps : 2 * mg_nu(l) + 3 * mg_reps(l));
    return n;
  }
  static constexpr double kDfMinTol = 1e-10, kDfMinErrTol = 1e-8;
  bool df_ = false;  // refined solution, right-hand sides and true residual as double-float pairs
  // ------------------------------------------------------------ profiling
  // With profiling on, an event is recorded after every launch of a step (in
  // the captured graph: external event-record nodes), so the device time of
  // every launch is measured and the launches of a step account for all of its
  // time from the first event to the last.  Each launch carries a category and
  // its algorithmic bytes (every vector it reads or writes counted once, the
  // operator entries and per-row scalars it reads).  A launch that found no
  // work (its kernel returns at once when no column runs) counts its time but
  // no bytes.
  enum Cat {
    kCatSpmm, kCatUpdate, kCatDirection, kCatFinish, kCatResidual, kCatAccumulate,
    kCatMgJacobi0, kCatMgSmooth0, kCatMgResid0, kCatMgRestrict0, kCatMgProlong0,
    kCatMgJacobi1, kCatMgSmooth1, kCatMgResid1, kCatMgRestrict1, kCatMgProlong1,
    kCatMgJacobiC, kCatMgSmoothC, kCatMgResidC, kCatMgRestrictC, kCatMgProlongC, kCatN
  };
  static constexpr int kCatMgKinds = kCatMgJacobi1 - kCatMgJacobi0;
  // a multigrid launch's category on level l: the finest level, the first
  // coarse level (the largest), or the coarser ones together
  static Cat lcat(size_t l, Cat fine) { return (Cat)(fine + kCatMgKinds * (int)(l < 2 ? l : 2)); }
  static constexpr const char* kCatName[kCatN] = {
      "spmm", "update", "direction", "finish", "residual", "accumulate",
      "mgjacobi0", "mgsmooth0", "mgresid0", "mgrestrict0", "mgprolong0",
      "mgjacobi1", "mgsmooth1", "mgresid1", "mgrestrict1", "mgprolong1",
      "mgjacobic", "mgsmoothc", "mgresidc", "mgrestrictc", "mgprolongc"};
  struct Mark {
    int cat;
    double bytes;
  };
  std::vector<Mark> marks_;
  std::vector<cudaEvent_t> pev_;
  unsigned evf_ = cudaEventRecordDefault;
  double cat_ms_[kCatN] = {}, cat_bytes_[kCatN] = {};
  int64_t cat_n_[kCatN] = {};
  double graph_ms_ = 0.0;
  int64_t graph_n_ = 0, steps_ = 0, other_launches_ = 0;
  cudaEvent_t pev(size_t i) {
    while (pev_.size() <= i) {
      cudaEvent_t e = nullptr;
      IFILT_CUDA(cudaEventCreate(&e));
      pev_.push_back(e);
    }
    return pev_[i];
  }
  bool marking_ = false;  // inside enqueue_step (autotuning launches are not marked)
  void pmark_open() {
    marking_ = prof_;
    if (marking_) IFILT_CUDA(cudaEventRecordWithFlags(pev(0), st_, evf_));
  }
  void pmark(int cat, double bytes) {
    if (!marking_) return;
    IFILT_CUDA(cudaEventRecordWithFlags(pev(marks_.size() + 1), st_, evf_));
    marks_.push_back({cat, bytes});
  }
  // after a step: the time of every launch into its category
  void account_step() {
    if (marks_.empty()) return;
    // lanes of the columns refreshed this step (counts copied after the step's first scan)
    const double wr = (double)h_cnt_[5] * LPC;
    const double s = sizeof(T);
    const double src_b = (double)n_ * NS * (3 * 8 + 4) * std::min<double>((double)src_.size(), h_cnt_[5]);
    const double res_ell = df_ ? (double)E_->entries * (4.0 + 2 * 4.0 * E_->nval)
                               : (double)E_->entries * (4.0 + 8.0 * E_->nval);
    const double rows = (double)n_ * NS;
    float total = 0.f;
    IFILT_CUDA(cudaEventElapsedTime(&total, pev_[0], pev_[marks_.size()]));
    graph_ms_ += total;
    graph_n_++;
    for (size_t i = 0; i < marks_.size(); i++) {
      float ms = 0.f;
      IFILT_CUDA(cudaEventElapsedTime(&ms, pev_[i], pev_[i + 1]));
      const Mark& mk = marks_[i];
      double b = mk.bytes;
      if (mk.cat == kCatResidual) b = wr > 0 ? rows * wr * (8.0 + 3.0 * s) + res_ell + 8.0 * n_ + src_b : 0.0;
      if (mk.cat == kCatAccumulate) b = rows * wr * (16.0 + s);
      // a launch that returned at once (no column running) moves nothing
      if (b > 0.0 && ms < 0.004f && b > 4e7) b = 0.0;
      cat_ms_[mk.cat] += ms;
      cat_bytes_[mk.cat] += b;
      cat_n_[mk.cat]++;
    }
  }
};

template <typename T, typename MV, typename TM>
Engine* make_kind(ifilt_mesh_s* m, const ifilt_solve_opts& o, cudaStream_t st, int64_t budget, bool cplx, bool blk) {
  if (cplx) {
    if (blk) return new EngineT<T, MV, TM, true, true>(m, o, st, budget);
    return new EngineT<T, MV, TM, true, false>(m, o, st, budget);
  }
  if (blk) return new EngineT<T, MV, TM, false, true>(m, o, st, budget);
  return new EngineT<T, MV, TM, false, false>(m, o, st, budget);
}

}  // namespace

Engine* make_engine(ifilt_mesh_s* m, const ifilt_solve_opts& o, cudaStream_t st, int64_t budget) {
  const bool cplx = complex_form(o);
  const bool blk = m->host.placement == IFILT_VERTEX_VECTOR;
  if (o.precision == IFILT_PREC_FP64) return make_kind<double, double, double>(m, o, st, budget, cplx, blk);
  if (o.precision == IFILT_PREC_BF16_IR) return make_kind<float, __nv_bfloat16, float>(m, o, st, budget, cplx, blk);
  return make_kind<float, float, float>(m, o, st, budget, cplx, blk);
}

size_t batched_scratch_bytes(const ifilt_mesh_s* m, const ifilt_solve_opts& o, int32_t F, int32_t nk) {
  const HostPrepared& h = m->host;
  const bool cplx = complex_form(o);
  const int nsys = h.placement == IFILT_CELL ? 2 : 1;
  const int ns = h.placement == IFILT_VERTEX_VECTOR ? 2 : 1;
  const int vec = o.precision == IFILT_PREC_FP64 ? 2 : 4;
  const int cap = std::min(o.max_lanes > 0 ? o.max_lanes : 256, kBlock * vec) / 4 * 4;
  const int lanes = (int)std::min<long long>((long long)F * nsys * nk * (cplx ? 2 : 1), cap);
  const int W = (lanes + 3) / 4 * 4;
  const size_t tb = o.precision == IFILT_PREC_FP64 ? 8 : 4;
  const size_t n = (size_t)h.n_rows;
  const size_t cols = (size_t)W / (cplx ? 2 : 1);
  const size_t srcs = std::min<size_t>((size_t)F * nsys, cols) * n * ns * (3 * 8 + 4);  // e0, x0, g0, x0 float
  // multigrid: two fine scratch vectors and three per coarser level (coarsening >= 1.25x per level)
  const size_t mg = o.precond == IFILT_PRECOND_MG ? n * ns * W * tb * (2 + 3 * 4) : 0;
  // tiles twice (old and new during a re-pack), sources, partial sums and tables
  return 2 * n * ns * W * (4 * tb + 8) + mg + srcs + (size_t)152 * 8 * 8 * W * 8 + (1 << 20);
}

namespace {
std::vector<ColumnJob> jobs_of(const ifilt_solve_item& it) {
  const HostPrepared& h = it.mesh->host;
  const int nsys = h.placement == IFILT_CELL ? 2 : 1;
  std::vector<ColumnJob> jobs;
  jobs.reserve((size_t)it.n_fields * nsys * it.n_k);
  for (int f = 0; f < it.n_fields; f++)
    for (int s = 0; s < nsys; s++)
      for (int j = 0; j < it.n_k; j++) {
        ColumnJob c;
        c.field = it.fields + (int64_t)f * h.n_comp * h.n_in;
        c.sys = s;
        c.k = it.k[j];
        c.out = it.out + ((int64_t)f * it.n_k + j) * h.n_comp * h.n_out;
        c.stat = it.stats ? &it.stats[((int64_t)f * it.n_k + j) * nsys + s] : nullptr;
        jobs.push_back(c);
      }
  // the largest scales (slowest columns) are admitted first
  std::stable_sort(jobs.begin(), jobs.end(), [](const ColumnJob& a, const ColumnJob& b) { return a.k < b.k; });
  return jobs;
}
}  // namespace

ifilt_status solve_many(int32_t n, const ifilt_solve_item* items, cudaStream_t st) {
  std::vector<cudaStream_t> ws(n, nullptr);
  std::vector<Engine*> eng(n, nullptr);
  cudaEvent_t ev = nullptr;
  ifilt_status result = IFILT_OK;
  auto cleanup = [&]() {
    for (int i = 0; i < n; i++) {
      delete eng[i];
      eng[i] = nullptr;
      if (ws[i]) {
        cudaStreamSynchronize(ws[i]);
        cudaStreamDestroy(ws[i]);
        ws[i] = nullptr;
      }
    }
    if (ev) cudaEventDestroy(ev);
    ev = nullptr;
  };
  try {
    // CUDA graphs cannot be captured on the legacy default stream, so every
    // engine runs on a private stream ordered after the caller's work.
    IFILT_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    IFILT_CUDA(cudaEventRecord(ev, st));
    for (int i = 0; i < n; i++) {
      IFILT_CUDA(cudaStreamCreateWithFlags(&ws[i], cudaStreamNonBlocking));
      IFILT_CUDA(cudaStreamWaitEvent(ws[i], ev, 0));
      ifilt_solve_opts o = items[i].opts;
      o.method = IFILT_METHOD_BATCHED;
      eng[i] = make_engine(items[i].mesh, o, ws[i], 0);
      eng[i]->submit(jobs_of(items[i]));
    }
    std::vector<ColumnDone> done;
    while (true) {
      bool any = false;
      for (int i = 0; i < n; i++)
        if (!eng[i]->idle()) {
          eng[i]->launch();
          any = true;
        }
      if (!any) break;
      for (int i = 0; i < n; i++) eng[i]->settle(done);
    }
    for (auto& d : done)
      if (d.status != IFILT_OK) result = IFILT_NOT_CONVERGED;
    for (int i = 0; i < n; i++) {
      eng[i]->report_profile();
      IFILT_CUDA(cudaEventRecord(ev, ws[i]));
      IFILT_CUDA(cudaStreamWaitEvent(st, ev, 0));
    }
  } catch (...) {
    cleanup();
    throw;
  }
  cleanup();
  return result;
}

ifilt_status solve_batched(ifilt_mesh_s* m, const ifilt_solve_opts& o, int32_t F, const double* fields, int32_t nk,
                           const double* k, double* out, ifilt_col_stats* stats, cudaStream_t st) {
  ifilt_solve_item it{};
  it.mesh = m;
  it.opts = o;
  it.n_fields = F;
  it.fields = fields;
  it.n_k = nk;
  it.k = k;
  it.out = out;
  it.stats = stats;
  return solve_many(1, &it, st);
}

}  // namespace ifilt
