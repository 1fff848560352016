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
#include <mutex>
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
  int* active;      // inner recursion running
  int* done;        // column finished (converged, capped or broken down)
  int* iters;
  int* rounds;
  int* status;      // 0 ok, 1 not converged, 2 breakdown
  int* refresh;     // column waits for its FP64 true residual / next refinement round
  int* live;        // [3] number of active columns, columns to refresh, columns not done
};

struct Params {
  int32_t n;        // rows
  int W;            // lanes per sub-row
  int ncols;        // columns (incl. padding)
  int pstride;      // doubles per block in `partial`
  int maxit;
  double tol2_rel;  // tol^2
  double inner2;    // inner_tol^2 (0: run to the outer tolerance)
};

// ------------------------------------------------------------------ kernels

template <typename T, typename MV, bool CPLX, bool BLK>
__global__ void __launch_bounds__(kBlock) spmm_kernel(EllView<MV> A, Params P, const T* __restrict__ p,
                                                      T* __restrict__ q, const double* __restrict__ mass,
                                                      Cols C, double* __restrict__ partial) {
  if (*C.live == 0) return;
  constexpr int VEC = Pack<T>::N;
  constexpr int NS = BLK ? 2 : 1;
  constexpr int NV = BLK ? 2 : 1;
  extern __shared__ double sm[];
  const int W = P.W;
  const int TPR = W / VEC;
  const int RPP = kBlock / TPR;
  const int tr = threadIdx.x / TPR, g = threadIdx.x - tr * TPR;
  const int l0 = g * VEC;
  double dacc[VEC];
#pragma unroll
  for (int v = 0; v < VEC; v++) dacc[v] = 0.0;
  if (tr < RPP) {
    T sh[VEC];
#pragma unroll
    for (int v = 0; v < VEC; v++) sh[v] = (T)C.shift[CPLX ? (l0 + v) >> 1 : l0 + v];
    const int64_t rowW = (int64_t)NS * W;
    for (int64_t r = (int64_t)blockIdx.x * RPP + tr; r < P.n; r += (int64_t)gridDim.x * RPP) {
      const int s = (int)(r / A.slice_h);
      const int w = A.slice_w[s];
      const int64_t base = A.slice_off[s] + (r - (int64_t)s * A.slice_h) * w;
      T acc[NS][VEC];
#pragma unroll
      for (int b = 0; b < NS; b++)
#pragma unroll
        for (int v = 0; v < VEC; v++) acc[b][v] = (T)0;
      for (int e = 0; e < w; e += 4) {
        const int4 c4 = __ldg(reinterpret_cast<const int4*>(A.col + base + e));
        T vals[4 * NV];
        load_vals<MV, NV, T>(A.val + (base + e) * NV, vals);
        const int cc[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
        for (int t = 0; t < 4; t++) {
          const T* src = p + (int64_t)cc[t] * rowW + l0;
          Pack<T> pu = ldp(src);
          if constexpr (BLK) {
            Pack<T> pv = ldp(src + W);
            const T a = vals[2 * t], bb = vals[2 * t + 1];
#pragma unroll
            for (int v = 0; v < VEC; v++) {
              acc[0][v] = fma(a, pu.v[v], fma(bb, pv.v[v], acc[0][v]));
              acc[1][v] = fma(a, pv.v[v], fma(-bb, pu.v[v], acc[1][v]));
            }
          } else {
            const T a = vals[t];
#pragma unroll
            for (int v = 0; v < VEC; v++) acc[0][v] = fma(a, pu.v[v], acc[0][v]);
          }
        }
      }
      const T mr = (T)mass[r];
#pragma unroll
      for (int b = 0; b < NS; b++) {
        const int64_t off = r * rowW + (int64_t)b * W + l0;
        const Pack<T> pr = ldp(p + off);
        Pack<T> qo;
        if constexpr (CPLX) {
#pragma unroll
          for (int v = 0; v < VEC; v += 2) {
            const T pre = pr.v[v], pim = pr.v[v + 1];
            const T qre = mr * pre - sh[v] * acc[b][v + 1];
            const T qim = mr * pim + sh[v] * acc[b][v];
            qo.v[v] = qre;
            qo.v[v + 1] = qim;
            dacc[v] += (double)pre * qre - (double)pim * qim;
            dacc[v + 1] += (double)pre * qim + (double)pim * qre;
          }
        } else {
#pragma unroll
          for (int v = 0; v < VEC; v++) {
            const T qv = mr * pr.v[v] + sh[v] * acc[b][v];
            qo.v[v] = qv;
            dacc[v] += (double)pr.v[v] * qv;
          }
        }
        stp(q + off, qo);
      }
    }
#pragma unroll
    for (int v = 0; v < VEC; v++) sm[tr * W + l0 + v] = dacc[v];
  }
  __syncthreads();
  for (int l = threadIdx.x; l < W; l += kBlock) {
    double s = 0.0;
    for (int t = 0; t < RPP; t++) s += sm[t * W + l];
    partial[(int64_t)blockIdx.x * P.pstride + l] = s;
  }
}

// x += alpha p ; r -= alpha q ; partial <r, r> (slots [0, W): lane-wise for real,
// (re, im) pairs for complex) and ||r||^2 (complex only, slots W + column).
template <typename T, bool CPLX, bool BLK>
__global__ void __launch_bounds__(kBlock) update_kernel(Params P, T* __restrict__ x, const T* __restrict__ p,
                                                        T* __restrict__ r, const T* __restrict__ q, Cols C,
                                                        double* __restrict__ partial) {
  if (*C.live == 0) return;
  constexpr int VEC = Pack<T>::N;
  constexpr int NS = BLK ? 2 : 1;
  extern __shared__ double sm[];
  const int W = P.W;
  const int NSL = CPLX ? W + W / 2 : W;  // slots
  const int TPR = W / VEC;
  const int RPP = kBlock / TPR;
  const int tr = threadIdx.x / TPR, g = threadIdx.x - tr * TPR;
  const int l0 = g * VEC;
  double d1[VEC], d2[VEC / 2 > 0 ? VEC / 2 : 1];
#pragma unroll
  for (int v = 0; v < VEC; v++) d1[v] = 0.0;
#pragma unroll
  for (int v = 0; v < (VEC / 2 > 0 ? VEC / 2 : 1); v++) d2[v] = 0.0;
  if (tr < RPP) {
    T a[VEC];
#pragma unroll
    for (int v = 0; v < VEC; v++) {
      if constexpr (CPLX) a[v] = (T)C.alpha[(l0 & ~1) + v];  // lanes (re, im) of one column
      else a[v] = (T)C.alpha[2 * (l0 + v)];
    }
    const int64_t rowW = (int64_t)NS * W;
    for (int64_t row = (int64_t)blockIdx.x * RPP + tr; row < P.n; row += (int64_t)gridDim.x * RPP) {
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
            const double rre = rv.v[v], rim = rv.v[v + 1];
            d1[v] += rre * rre - rim * rim;
            d1[v + 1] += 2.0 * rre * rim;
            d2[v / 2] += rre * rre + rim * rim;
          }
        } else {
#pragma unroll
          for (int v = 0; v < VEC; v++) {
            xv.v[v] = fma(a[v], pv.v[v], xv.v[v]);
            rv.v[v] = fma(-a[v], qv.v[v], rv.v[v]);
            d1[v] += (double)rv.v[v] * rv.v[v];
          }
        }
        stp(x + off, xv);
        stp(r + off, rv);
      }
    }
#pragma unroll
    for (int v = 0; v < VEC; v++) sm[tr * NSL + l0 + v] = d1[v];
    if constexpr (CPLX) {
#pragma unroll
      for (int v = 0; v < VEC / 2; v++) sm[tr * NSL + W + l0 / 2 + v] = d2[v];
    }
  }
  __syncthreads();
  for (int l = threadIdx.x; l < NSL; l += kBlock) {
    double s = 0.0;
    for (int t = 0; t < RPP; t++) s += sm[t * NSL + l];
    partial[(int64_t)blockIdx.x * P.pstride + l] = s;
  }
}

// p = r + beta p
template <typename T, bool CPLX, bool BLK>
__global__ void __launch_bounds__(kBlock) direction_kernel(Params P, T* __restrict__ p, const T* __restrict__ r,
                                                           Cols C) {
  if (*C.live == 0) return;
  constexpr int VEC = Pack<T>::N;
  constexpr int NS = BLK ? 2 : 1;
  const int W = P.W;
  const int TPR = W / VEC;
  const int RPP = kBlock / TPR;
  const int tr = threadIdx.x / TPR, g = threadIdx.x - tr * TPR;
  if (tr >= RPP) return;
  const int l0 = g * VEC;
  T bt[VEC];
#pragma unroll
  for (int v = 0; v < VEC; v++) {
    if constexpr (CPLX) bt[v] = (T)C.beta[(l0 & ~1) + v];
    else bt[v] = (T)C.beta[2 * (l0 + v)];
  }
  const int64_t rowW = (int64_t)NS * W;
  for (int64_t row = (int64_t)blockIdx.x * RPP + tr; row < P.n; row += (int64_t)gridDim.x * RPP) {
#pragma unroll
    for (int b = 0; b < NS; b++) {
      const int64_t off = row * rowW + (int64_t)b * W + l0;
      Pack<T> pv = ldv(p + off);
      const Pack<T> rv = ldv(r + off);
      if constexpr (CPLX) {
#pragma unroll
        for (int v = 0; v < VEC; v += 2) {
          const T pre = pv.v[v], pim = pv.v[v + 1];
          pv.v[v] = rv.v[v] + bt[v] * pre - bt[v + 1] * pim;
          pv.v[v + 1] = rv.v[v + 1] + bt[v] * pim + bt[v + 1] * pre;
        }
      } else {
#pragma unroll
        for (int v = 0; v < VEC; v++) pv.v[v] = fma(bt[v], pv.v[v], rv.v[v]);
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
  const double n2 = CPLX ? reduce_slot(partial, nb, P.pstride, ok ? P.W + col : -1, buf) : rre;
  if (threadIdx.y != 0 || !ok) return;
  double br = 0.0, bi = 0.0;
  if (C.active[col]) {
    const double orr = C.rho[2 * col], ori = C.rho[2 * col + 1];
    if (CPLX) cdiv(rre, rim, orr, ori, br, bi);
    else br = rre / orr;
    C.rho[2 * col] = rre;
    C.rho[2 * col + 1] = rim;
    C.rn2[col] = n2;
    const int it = ++C.iters[col];
    bool stop = false;
    if (!(isfinite(n2) && isfinite(br) && isfinite(bi))) {
      C.status[col] = 2;
      C.done[col] = 1;
      stop = true;
    } else if (n2 <= C.target2[col]) {
      stop = true;
    } else if (it >= P.maxit) {
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

// x64 = x0 (real lanes; imaginary lanes 0)
template <bool CPLX, bool BLK>
__global__ void init_x_kernel(Params P, const double* __restrict__ x0src, const int* __restrict__ lane_src,
                              double* __restrict__ x64) {
  constexpr int NS = BLK ? 2 : 1;
  const int64_t total = (int64_t)P.n * NS * P.W;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int l = (int)(i % P.W);
    const int64_t rs = i / P.W;  // row * NS + sub
    double v = 0.0;
    if (!(CPLX && (l & 1))) v = x0src[(int64_t)lane_src[l] * P.n * NS + rs];
    x64[i] = v;
  }
}

// FP64 true residual r64 = b - S x64; starts an inner round: r = p = (T) r64, d = 0.
// Slots: [0, W) <r, r> of the rounded residual (lane-wise / (re, im) pairs),
//        [W, W + ncols) ||r64||^2.
template <typename T, bool CPLX, bool BLK>
__global__ void __launch_bounds__(kBlock) residual_kernel(EllView<double> A, Params P,
                                                          const double* __restrict__ x64,
                                                          const double* __restrict__ bsrc,
                                                          const int* __restrict__ lane_src,
                                                          const double* __restrict__ mass, Cols C,
                                                          T* __restrict__ r, T* __restrict__ d, T* __restrict__ p,
                                                          double* __restrict__ partial) {
  constexpr int VEC = Pack<T>::N;
  constexpr int NS = BLK ? 2 : 1;
  constexpr int NV = BLK ? 2 : 1;
  constexpr int DP = VEC / 2;  // double packs per thread
  extern __shared__ double sm[];
  const int W = P.W;
  const int ncolsW = CPLX ? W / 2 : W;
  const int NSL = W + ncolsW;
  const int TPR = W / VEC;
  const int RPP = kBlock / TPR;
  const int tr = threadIdx.x / TPR, g = threadIdx.x - tr * TPR;
  const int l0 = g * VEC;
  double d1[VEC], d2[VEC];
#pragma unroll
  for (int v = 0; v < VEC; v++) d1[v] = d2[v] = 0.0;
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
        Pack<T> ro, zo;
#pragma unroll
        for (int v = 0; v < VEC; v++) zo.v[v] = (T)0;
        if constexpr (CPLX) {
#pragma unroll
          for (int v = 0; v < VEC; v += 2) {
            const double bre = bsrc[(int64_t)src[v] * P.n * NS + row * NS + b];
            const double r_re = bre - (mr * xo[v] - sh[v] * acc[b][v + 1]);
            const double r_im = -(mr * xo[v + 1] + sh[v] * acc[b][v]);
            const T tre = (T)r_re, tim = (T)r_im;
            ro.v[v] = tre;
            ro.v[v + 1] = tim;
            d1[v] += (double)tre * tre - (double)tim * tim;
            d1[v + 1] += 2.0 * (double)tre * tim;
            d2[v / 2] += r_re * r_re + r_im * r_im;
          }
        } else {
#pragma unroll
          for (int v = 0; v < VEC; v++) {
            const double bv = bsrc[(int64_t)src[v] * P.n * NS + row * NS + b];
            const double rv = bv - (mr * xo[v] + sh[v] * acc[b][v]);
            const T t = (T)rv;
            ro.v[v] = t;
            d1[v] += (double)t * t;
            d2[v] += rv * rv;
          }
        }
        if (all) {
          stp(r + off, ro);
          stp(p + off, ro);
          stp(d + off, zo);
        } else {
#pragma unroll
          for (int v = 0; v < VEC; v++)
            if (mine[v]) {
              r[off + v] = ro.v[v];
              p[off + v] = ro.v[v];
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
      for (int v = 0; v < VEC / 2; v++) sm[tr * NSL + W + l0 / 2 + v] = d2[v];
    } else {
#pragma unroll
      for (int v = 0; v < VEC; v++) sm[tr * NSL + W + l0 + v] = d2[v];
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
  __shared__ double buf[8][33];
  const int col = blockIdx.x * 32 + threadIdx.x;
  const bool ok = col < P.ncols;
  const double rre = reduce_slot(partial, nb, P.pstride, ok ? (CPLX ? 2 * col : col) : -1, buf);
  const double rim = CPLX ? reduce_slot(partial, nb, P.pstride, ok ? 2 * col + 1 : -1, buf) : 0.0;
  const double n2 = reduce_slot(partial, nb, P.pstride, ok ? P.W + col : -1, buf);
  if (threadIdx.y != 0 || !ok) return;
  if (!C.refresh[col]) return;
  C.refresh[col] = 0;
  if (C.r0n2[col] < 0.0) {
    C.r0n2[col] = n2;
    C.tol2[col] = P.tol2_rel * n2;
  }
  const double r0 = C.r0n2[col];
  C.rel[col] = r0 > 0.0 ? sqrt(n2 / r0) : 0.0;
  if (C.active[col]) {  // inner round stopped by its iteration cap
    C.active[col] = 0;
    atomicSub(C.live, 1);
  }
  if (C.done[col]) return;
  if (!(n2 > C.tol2[col]) || r0 == 0.0) {
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
  C.rho[2 * col] = rre;
  C.rho[2 * col + 1] = rim;
  C.rn2[col] = n2;
  C.target2[col] = fmax(P.inner2 * n2, 0.25 * C.tol2[col]);
  C.rounds[col]++;
  C.active[col] = 1;
  atomicAdd(C.live, 1);
}

// x64 += d on the lanes of refreshed columns
template <typename T, bool CPLX>
__global__ void accumulate_kernel(int64_t total, int W, const int* __restrict__ refresh, double* __restrict__ x64,
                                  const T* __restrict__ d) {
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

// out[f][k][comp][o] from the FP64 solution (real part); land entries copy the
// input (scalar, cell) or are zero (vector).
template <bool CPLX, bool BLK>
__global__ void output_kernel(Params P, int32_t n_out, const int32_t* __restrict__ inv,
                              const double* __restrict__ x64, const double* __restrict__ fields,
                              const int64_t* __restrict__ col_out, const int64_t* __restrict__ col_in,
                              double* __restrict__ out) {
  constexpr int NS = BLK ? 2 : 1;
  const int col = blockIdx.y;
  const int64_t obase = col_out[col];
  if (obase < 0) return;
  const int64_t ibase = col_in[col];
  const int lane = CPLX ? 2 * col : col;
  for (int32_t o = blockIdx.x * blockDim.x + threadIdx.x; o < n_out; o += gridDim.x * blockDim.x) {
    const int32_t r = inv[o];
#pragma unroll
    for (int b = 0; b < NS; b++) {
      double v;
      if (r >= 0) v = x64[((int64_t)r * NS + b) * P.W + lane];
      else v = BLK ? 0.0 : fields[ibase + o];
      out[obase * 1 + (int64_t)b * n_out + o] = v;
    }
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

struct Variant {
  bool cplx, blk;
  int prec;  // 0 fp64, 1 fp32, 2 bf16-valued fp32
};

template <typename T>
size_t vec_bytes(int64_t n, int ns, int W) {
  return (size_t)n * ns * W * sizeof(T);
}

struct ColumnSpec {
  int f, sys, kj, src;
  double shift;
};

// Lane tiles of one batch: [row][sub][lane] arrays, reallocated narrower when
// finished columns are retired.
template <typename T>
struct Tiles {
  int W = 0;
  T *d = nullptr, *r = nullptr, *p = nullptr, *q = nullptr;
  double* x64 = nullptr;
  void* base = nullptr;
};

template <typename T>
Tiles<T> alloc_tiles(int64_t n, int NS, int W, cudaStream_t st) {
  Tiles<T> t;
  t.W = W;
  const size_t vb = ((size_t)n * NS * W * sizeof(T) + 255) / 256 * 256;
  const size_t xb = ((size_t)n * NS * W * sizeof(double) + 255) / 256 * 256;
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
  std::vector<double> shift, rho, alpha, beta, rn2, target2, r0n2, tol2, rel;
  std::vector<int> active, done, iters, rounds, status, refresh;
  void resize(int n) {
    for (auto* v : {&shift, &rn2, &target2, &r0n2, &tol2, &rel}) v->assign(n, 0.0);
    for (auto* v : {&rho, &alpha, &beta}) v->assign(2 * n, 0.0);
    for (auto* v : {&active, &done, &iters, &rounds, &status, &refresh}) v->assign(n, 0);
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
  dn(H.active.data(), C.active, n * 4);
  dn(H.done.data(), C.done, n * 4);
  dn(H.iters.data(), C.iters, n * 4);
  dn(H.rounds.data(), C.rounds, n * 4);
  dn(H.status.data(), C.status, n * 4);
  dn(H.refresh.data(), C.refresh, n * 4);
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
  up(C.active, H.active.data(), n * 4);
  up(C.done, H.done.data(), n * 4);
  up(C.iters, H.iters.data(), n * 4);
  up(C.rounds, H.rounds.data(), n * 4);
  up(C.status, H.status.data(), n * 4);
  up(C.refresh, H.refresh.data(), n * 4);
  // the host vectors must outlive the copies
  IFILT_CUDA(cudaStreamSynchronize(st));
}

// Host record of every column of the batch (index into the batch's spec list).
struct ColResult {
  int iters = 0, rounds = 0, status = 0, done = 0;
  double rel = 0.0;
};

template <typename T, typename MV, bool CPLX, bool BLK>
ifilt_status run_batch(ifilt_mesh_s* m, const ifilt_solve_opts& o, const std::vector<ColumnSpec>& cols,
                       int nsrc_total, const double* bsrc_all, const double* x0src_all, const double* fields,
                       int32_t nk, double* out, ifilt_col_stats* stats, cudaStream_t st) {
  (void)nsrc_total;
  const HostPrepared& h = m->host;
  constexpr int VEC = Pack<T>::N;
  constexpr int NS = BLK ? 2 : 1;
  const int lpc = CPLX ? 2 : 1;  // lanes per column
  const int nreal = (int)cols.size();
  auto lanes_for = [&](int ncol) { return (ncol * lpc + 3) / 4 * 4; };
  const int Wmax = lanes_for(nreal);
  if (Wmax / VEC > kBlock) fail(IFILT_EINVAL, "batch too wide (%d lanes)", Wmax);
  const int ncmax = Wmax / lpc;
  const int64_t n = h.n_rows;
  const bool use_g2 = (o.order >= 2) && !CPLX;
  const DevEll& E = use_g2 ? m->ell_g2 : m->ell_k;
  const EllView<MV> A = ell_view<MV>(E);
  const EllView<double> A64 = ell_view<double>(E);

  std::vector<int> src_ids;
  for (auto& c : cols)
    if (std::find(src_ids.begin(), src_ids.end(), c.src) == src_ids.end()) src_ids.push_back(c.src);
  const int nsrc = (int)src_ids.size();

  auto smem_of = [&](int W, int slots_per_lane2) {  // slots per row-pass in units of W/2
    return (size_t)(kBlock / (W / VEC)) * (size_t)W * slots_per_lane2 / 2 * sizeof(double);
  };
  auto blocks_for = [&](int W) {
    return grid_for((const void*)spmm_kernel<T, MV, CPLX, BLK>, kBlock, smem_of(W, 2), n * (long long)(W / VEC));
  };
  const int nb_max = blocks_for(Wmax);

  // fixed scratch: sources, reduction partials, column state, tables
  const size_t sb = (size_t)nsrc * n * NS * sizeof(double);
  size_t total = 2 * sb + (size_t)nb_max * 2 * Wmax * 8 + (size_t)ncmax * (8 * 16 + 4 * 8) + (size_t)Wmax * 8 +
                 64 * 256;
  char* base = (char*)scratch_alloc(total, st);
  char* cur = base;
  auto take = [&](size_t bytes) {
    char* p = cur;
    cur += (bytes + 255) / 256 * 256;
    return (void*)p;
  };
  double* bs = (double*)take(sb);
  double* x0s = (double*)take(sb);
  double* partial = (double*)take((size_t)nb_max * 2 * Wmax * 8);
  Cols C{};
  C.shift = (double*)take(ncmax * 8);
  C.rho = (double*)take(2 * ncmax * 8);
  C.alpha = (double*)take(2 * ncmax * 8);
  C.beta = (double*)take(2 * ncmax * 8);
  C.rn2 = (double*)take(ncmax * 8);
  C.target2 = (double*)take(ncmax * 8);
  C.r0n2 = (double*)take(ncmax * 8);
  C.tol2 = (double*)take(ncmax * 8);
  C.rel = (double*)take(ncmax * 8);
  C.active = (int*)take(ncmax * 4);
  C.done = (int*)take(ncmax * 4);
  C.iters = (int*)take(ncmax * 4);
  C.rounds = (int*)take(ncmax * 4);
  C.status = (int*)take(ncmax * 4);
  C.refresh = (int*)take(ncmax * 4);
  C.live = (int*)take(4 * 4);
  int* lane_src = (int*)take(Wmax * 4);
  int* lane_map = (int*)take(Wmax * 4);
  int64_t* col_out = (int64_t*)take(ncmax * 8);
  int64_t* col_in = (int64_t*)take(ncmax * 8);
  for (int s = 0; s < nsrc; s++) {
    IFILT_CUDA(cudaMemcpyAsync(bs + (size_t)s * n * NS, bsrc_all + (size_t)src_ids[s] * n * NS,
                               n * NS * sizeof(double), cudaMemcpyDeviceToDevice, st));
    IFILT_CUDA(cudaMemcpyAsync(x0s + (size_t)s * n * NS, x0src_all + (size_t)src_ids[s] * n * NS,
                               n * NS * sizeof(double), cudaMemcpyDeviceToDevice, st));
  }

  // current column set: batch-spec index of each column (-1 = padding)
  std::vector<int> curcols(nreal);
  for (int c = 0; c < nreal; c++) curcols[c] = c;
  std::vector<ColResult> res(nreal);
  std::vector<int> lsrc_h;
  std::vector<int64_t> cout_h, cin_h;
  auto upload_tables = [&](int W) {
    const int nc = W / lpc;
    lsrc_h.assign(W, 0);
    cout_h.assign(nc, -1);
    cin_h.assign(nc, 0);
    for (int c = 0; c < nc; c++) {
      const int id = c < (int)curcols.size() ? curcols[c] : -1;
      if (id < 0) continue;
      const ColumnSpec& cs = cols[id];
      const int s = (int)(std::find(src_ids.begin(), src_ids.end(), cs.src) - src_ids.begin());
      for (int t = 0; t < lpc; t++) lsrc_h[c * lpc + t] = s;
      const int comp = h.placement == IFILT_CELL ? cs.sys : 0;
      cout_h[c] = (((int64_t)cs.f * nk + cs.kj) * h.n_comp + comp) * h.n_out;
      cin_h[c] = ((int64_t)cs.f * h.n_comp + comp) * h.n_in;
    }
    IFILT_CUDA(cudaMemcpyAsync(lane_src, lsrc_h.data(), W * 4, cudaMemcpyHostToDevice, st));
    IFILT_CUDA(cudaMemcpyAsync(col_out, cout_h.data(), nc * 8, cudaMemcpyHostToDevice, st));
    IFILT_CUDA(cudaMemcpyAsync(col_in, cin_h.data(), nc * 8, cudaMemcpyHostToDevice, st));
    IFILT_CUDA(cudaStreamSynchronize(st));
  };

  // initial column state: every real column asks for its first true residual
  HostCols H;
  H.resize(ncmax);
  for (int c = 0; c < ncmax; c++) {
    if (c < nreal) {
      H.shift[c] = cols[c].shift;
      H.r0n2[c] = -1.0;
      H.refresh[c] = 1;
    } else {
      H.done[c] = 1;
    }
  }
  cols_upload(C, H, ncmax, st);
  upload_tables(Wmax);

  Params P{};
  P.n = (int32_t)n;
  P.maxit = o.max_iter > 0 ? o.max_iter : 100000;
  P.tol2_rel = o.tol * o.tol;
  const double itol = (sizeof(T) == 8) ? 0.0 : (o.inner_tol > 0 ? o.inner_tol : 1e-4);
  P.inner2 = itol * itol;
  Tiles<T> tl = alloc_tiles<T>(n, NS, Wmax, st);
  auto set_width = [&](int W) {
    P.W = W;
    P.ncols = W / lpc;
    P.pstride = 2 * W;
  };
  set_width(Wmax);
  IFILT_CUDA(cudaMemsetAsync(tl.d, 0, (size_t)n * NS * Wmax * sizeof(T), st));
  {
    const int g = grid_for((const void*)init_x_kernel<CPLX, BLK>, kBlock, 0, n * NS * Wmax);
    launch_check("before init", 0, 0, Wmax);
    (void)0;
    init_x_kernel<CPLX, BLK><<<g, kBlock, 0, st>>>(P, x0s, lane_src, tl.x64);
    launch_check("init", g, 0, Wmax);
  }

  const int m_it = o.check_every > 0 ? o.check_every : 32;
  const bool prof = profiling_on();
  cudaEvent_t ev[6] = {};
  if (prof)
    for (auto& e : ev) IFILT_CUDA(cudaEventCreate(&e));
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int nb = nb_max;
  // IFILT_NO_GRAPH=1 launches every iteration directly and checks each launch
  // (debugging aid); otherwise m iterations are captured once per tile width.
  const char* ng = getenv("IFILT_NO_GRAPH");
  const bool use_graph = !(ng && ng[0] == '1');
  auto enqueue_iters = [&](bool check) {
    const int W = P.W;
    const size_t sm2 = smem_of(W, 2), sm3 = smem_of(W, 3);
    const int fin_grid = (P.ncols + 31) / 32;
    const dim3 fin_block(32, 8);
    auto chk = [&](const char* what) {
      if (!check) return;
      cudaError_t e = cudaGetLastError();
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess)
        fail(IFILT_ECUDA, "%s (W=%d, blocks=%d, smem=%zu/%zu): %s", what, W, nb, sm2, sm3, cudaGetErrorString(e));
    };
    // Inside a stream capture an event record is only a dependency marker
    // unless it is recorded as an external event node.
    const unsigned evflags = check ? cudaEventRecordDefault : cudaEventRecordExternal;
    auto rec = [&](cudaEvent_t e) { IFILT_CUDA(cudaEventRecordWithFlags(e, st, evflags)); };
    for (int it = 0; it < m_it; it++) {
      if (prof && it == 0) rec(ev[0]);
      spmm_kernel<T, MV, CPLX, BLK><<<nb, kBlock, sm2, st>>>(A, P, tl.p, tl.q, m->mass, C, partial);
      chk("spmm");
      if (prof && it == 0) rec(ev[1]);
      finish_alpha_kernel<CPLX><<<fin_grid, fin_block, 0, st>>>(P, nb, partial, C);
      chk("finish_alpha");
      if (prof && it == 0) rec(ev[2]);
      update_kernel<T, CPLX, BLK><<<nb, kBlock, sm3, st>>>(P, tl.d, tl.p, tl.r, tl.q, C, partial);
      chk("update");
      if (prof && it == 0) rec(ev[3]);
      finish_beta_kernel<CPLX><<<fin_grid, fin_block, 0, st>>>(P, nb, partial, C);
      chk("finish_beta");
      if (prof && it == 0) rec(ev[4]);
      direction_kernel<T, CPLX, BLK><<<nb, kBlock, 0, st>>>(P, tl.p, tl.r, C);
      chk("direction");
      if (prof && it == 0) rec(ev[5]);
    }
  };
  auto capture = [&]() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    exec = nullptr;
    graph = nullptr;
    nb = blocks_for(P.W);
    IFILT_CUDA(cudaGetLastError());
    if (!use_graph) return;
    IFILT_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    enqueue_iters(false);
    cudaError_t cap = cudaStreamEndCapture(st, &graph);
    if (cap != cudaSuccess) fail(IFILT_ECUDA, "graph capture failed: %s", cudaGetErrorString(cap));
    launch_check("capture", nb, 0, P.W);
    IFILT_CUDA(cudaGraphInstantiate(&exec, graph, 0));
    launch_check("instantiate", nb, 0, P.W);
  };
  // writes the outputs of the current columns for which `sel` holds
  auto emit = [&](const std::vector<int>& sel) {
    const int nc = P.ncols;
    std::vector<int64_t> co(nc, -1);
    for (int c = 0; c < nc && c < (int)curcols.size(); c++)
      if (curcols[c] >= 0 && sel[c]) co[c] = cout_h[c];
    IFILT_CUDA(cudaMemcpyAsync(col_out, co.data(), nc * 8, cudaMemcpyHostToDevice, st));
    dim3 og((unsigned)std::min<long long>((h.n_out + kBlock - 1) / kBlock, 1024), (unsigned)nc);
    output_kernel<CPLX, BLK><<<og, kBlock, 0, st>>>(P, h.n_out, m->inv_perm, tl.x64, fields, col_out, col_in, out);
    IFILT_CUDA(cudaGetLastError());
    IFILT_CUDA(cudaStreamSynchronize(st));
  };
  auto record = [&](const HostCols& Hc, int c) {
    const int id = curcols[c];
    if (id < 0) return;
    ColResult& r = res[id];
    r.iters = Hc.iters[c];
    r.rounds = Hc.rounds[c];
    r.status = Hc.status[c];
    r.done = Hc.done[c];
    r.rel = Hc.rel[c];
  };
  // Retire finished columns and narrow the tiles to the ones still running.
  auto compact = [&]() {
    const int nc = P.ncols, Wold = P.W;
    cols_download(C, H, nc, st);
    std::vector<int> keep, sel(nc, 0);
    for (int c = 0; c < nc; c++) {
      if (c >= (int)curcols.size() || curcols[c] < 0) continue;
      if (H.done[c]) {
        sel[c] = 1;
        record(H, c);
      } else {
        keep.push_back(c);
      }
    }
    emit(sel);
    const int Wn = lanes_for((int)keep.size());
    const int ncn = Wn / lpc;
    std::vector<int> map(Wn, -1);
    HostCols Hn;
    Hn.resize(ncn);
    std::vector<int> ncur(ncn, -1);
    for (int j = 0; j < ncn; j++) {
      if (j >= (int)keep.size()) {
        Hn.done[j] = 1;
        continue;
      }
      const int c = keep[j];
      ncur[j] = curcols[c];
      for (int t = 0; t < lpc; t++) map[j * lpc + t] = c * lpc + t;
      Hn.shift[j] = H.shift[c];
      for (int t = 0; t < 2; t++) {
        Hn.rho[2 * j + t] = H.rho[2 * c + t];
        Hn.alpha[2 * j + t] = H.alpha[2 * c + t];
        Hn.beta[2 * j + t] = H.beta[2 * c + t];
      }
      Hn.rn2[j] = H.rn2[c];
      Hn.target2[j] = H.target2[c];
      Hn.r0n2[j] = H.r0n2[c];
      Hn.tol2[j] = H.tol2[c];
      Hn.rel[j] = H.rel[c];
      Hn.active[j] = H.active[c];
      Hn.done[j] = H.done[c];
      Hn.iters[j] = H.iters[c];
      Hn.rounds[j] = H.rounds[c];
      Hn.status[j] = H.status[c];
      Hn.refresh[j] = H.refresh[c];
    }
    IFILT_CUDA(cudaMemcpyAsync(lane_map, map.data(), Wn * 4, cudaMemcpyHostToDevice, st));
    Tiles<T> tn = alloc_tiles<T>(n, NS, Wn, st);
    const int64_t rows = n * NS;
    const int g = grid_for((const void*)gather_lanes_kernel<T>, kBlock, 0, rows * Wn);
    gather_lanes_kernel<T><<<g, kBlock, 0, st>>>(rows, Wold, Wn, lane_map, tl.d, tn.d);
    gather_lanes_kernel<T><<<g, kBlock, 0, st>>>(rows, Wold, Wn, lane_map, tl.r, tn.r);
    gather_lanes_kernel<T><<<g, kBlock, 0, st>>>(rows, Wold, Wn, lane_map, tl.p, tn.p);
    gather_lanes_kernel<double><<<g, kBlock, 0, st>>>(rows, Wold, Wn, lane_map, tl.x64, tn.x64);
    IFILT_CUDA(cudaGetLastError());
    scratch_free(tl.base, st);
    tl = tn;
    curcols = ncur;
    set_width(Wn);
    cols_upload(C, Hn, ncn, st);
    upload_tables(Wn);
    capture();
  };

  capture();
  int* h_flags = nullptr;
  IFILT_CUDA(cudaMallocHost(&h_flags, sizeof(int) * 4));
  launch_check("pinned flags", 0, 0, P.W);
  auto scan = [&]() {
    launch_check("before scan", 0, 0, P.W);
    scan_kernel<<<1, 256, 0, st>>>(P.ncols, C);
    launch_check("scan", 1, 0, P.W);
    IFILT_CUDA(cudaMemcpyAsync(h_flags, C.live, 3 * sizeof(int), cudaMemcpyDeviceToHost, st));
    IFILT_CUDA(cudaStreamSynchronize(st));
  };
  double t_spmm = 0, t_upd = 0, t_dir = 0, b_spmm = 0, b_upd = 0, b_dir = 0;
  int64_t samples = 0, graph_launches = 0, other_launches = 2;
  const double mbytes = (double)E.entries * (4.0 + E.nval * sizeof(MV)) + (double)n * 8.0;
  const int64_t guard = (int64_t)(P.maxit / m_it + 2) * 8 + 64;
  ifilt_status result = IFILT_OK;
  for (int64_t loop = 0;; loop++) {
    if (loop > guard) {
      result = IFILT_NOT_CONVERGED;
      break;
    }
    scan();
    other_launches++;
    if (h_flags[2] == 0) break;  // every column finished
    if (h_flags[1] > 0) {        // FP64 true residual and a new inner round for finished inner solves
      const int W = P.W;
      const int ga = grid_for((const void*)accumulate_kernel<T, CPLX>, kBlock, 0, n * NS * W);
      launch_check("before refinement", 0, 0, 0);
      accumulate_kernel<T, CPLX><<<ga, kBlock, 0, st>>>(n * NS * W, W, C.refresh, tl.x64, tl.d);
      launch_check("accumulate", ga, 0, W);
      residual_kernel<T, CPLX, BLK><<<nb, kBlock, smem_of(W, 4), st>>>(A64, P, tl.x64, bs, lane_src, m->mass, C,
                                                                      tl.r, tl.d, tl.p, partial);
      launch_check("residual", nb, smem_of(W, 4), W);
      finish_residual_kernel<CPLX><<<(P.ncols + 31) / 32, dim3(32, 8), 0, st>>>(P, nb, partial, C);
      launch_check("finish_residual", (P.ncols + 31) / 32, 0, W);
      other_launches += 3;
      scan();
      other_launches++;
      if (h_flags[2] == 0) break;
    }
    const int running = h_flags[2];
    if (lanes_for(running) < P.W && running * 5 <= P.ncols * 3) {
      compact();
      launch_check("compact", 0, 0, P.W);
    }
    if (h_flags[0] == 0) continue;
    if (use_graph) IFILT_CUDA(cudaGraphLaunch(exec, st));
    else enqueue_iters(true);
    graph_launches++;
    IFILT_CUDA(cudaStreamSynchronize(st));
    launch_check("graph", nb, 0, P.W);

    if (prof) {
      float a = 0, b = 0, c = 0;
      IFILT_CUDA(cudaEventElapsedTime(&a, ev[0], ev[1]));
      IFILT_CUDA(cudaEventElapsedTime(&b, ev[2], ev[3]));
      IFILT_CUDA(cudaEventElapsedTime(&c, ev[4], ev[5]));
      {
        const double vb = (double)n * NS * P.W * sizeof(T);
        t_spmm += a;
        t_upd += b;
        t_dir += c;
        b_spmm += 2.0 * vb + mbytes;
        b_upd += 6.0 * vb;
        b_dir += 3.0 * vb;
        samples++;
      }
    }
  }
  // outputs and stats of the columns still in the tiles
  {
    const int nc = P.ncols;
    cols_download(C, H, nc, st);
    std::vector<int> sel(nc, 1);
    for (int c = 0; c < nc; c++)
      if (c < (int)curcols.size()) record(H, c);
    emit(sel);
  }
  profile_count(other_launches + graph_launches * m_it * 5);
  const int nsys = h.placement == IFILT_CELL ? 2 : 1;
  for (int id = 0; id < nreal; id++) {
    const ColumnSpec& cs = cols[id];
    const ColResult& r = res[id];
    const int status = (r.status != 0 || !r.done || r.rel > o.tol) ? IFILT_NOT_CONVERGED : IFILT_OK;
    if (status != IFILT_OK) result = IFILT_NOT_CONVERGED;
    if (stats) {
      ifilt_col_stats& s = stats[((int64_t)cs.f * nk + cs.kj) * nsys + cs.sys];
      s.iters = r.iters;
      s.refinements = r.rounds;
      s.status = status;
      s.pad = 0;
      s.rel_residual = r.rel;
    }
  }
  if (prof) {
    const int64_t launches = graph_launches * m_it;
    const char* k1 = CPLX ? "c" : "r";
    const char* k2 = BLK ? "b" : "s";
    const char* k3 = sizeof(T) == 8 ? "f64" : "f32";
    char nm[32];
    if (samples > 0) {
      snprintf(nm, sizeof nm, "spmm_%s%s_%s", k1, k2, k3);
      profile_add(nm, launches, samples, t_spmm, b_spmm / samples);
      snprintf(nm, sizeof nm, "update_%s%s_%s", k1, k2, k3);
      profile_add(nm, launches, samples, t_upd, b_upd / samples);
      snprintf(nm, sizeof nm, "direction_%s%s_%s", k1, k2, k3);
      profile_add(nm, launches, samples, t_dir, b_dir / samples);
    }
    for (auto& e : ev) cudaEventDestroy(e);
  }
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  cudaFreeHost(h_flags);
  scratch_free(tl.base, st);
  scratch_free(base, st);
  return result;
}

using BatchFn = ifilt_status (*)(ifilt_mesh_s*, const ifilt_solve_opts&, const std::vector<ColumnSpec>&, int,
                                 const double*, const double*, const double*, int32_t, double*, ifilt_col_stats*,
                                 cudaStream_t);

template <typename T, typename MV>
BatchFn pick_kind(bool cplx, bool blk) {
  if (cplx) return blk ? run_batch<T, MV, true, true> : run_batch<T, MV, true, false>;
  return blk ? run_batch<T, MV, false, true> : run_batch<T, MV, false, false>;
}

BatchFn pick(int prec, bool cplx, bool blk) {
  if (prec == IFILT_PREC_FP64) return pick_kind<double, double>(cplx, blk);
  if (prec == IFILT_PREC_BF16_IR) return pick_kind<float, __nv_bfloat16>(cplx, blk);
  return pick_kind<float, float>(cplx, blk);
}

}  // namespace

size_t batched_scratch_bytes(const ifilt_mesh_s* m, const ifilt_solve_opts& o, int32_t F, int32_t nk) {
  const HostPrepared& h = m->host;
  const bool cplx = o.order >= 2 && o.n2_solver != IFILT_N2_REAL;
  const int nsys = h.placement == IFILT_CELL ? 2 : 1;
  const int ns = h.placement == IFILT_VERTEX_VECTOR ? 2 : 1;
  const int lanes = (int)std::min<long long>((long long)F * nsys * nk * (cplx ? 2 : 1),
                                             o.max_lanes > 0 ? o.max_lanes : 256);
  const int W = (lanes + 3) / 4 * 4;
  const size_t tb = o.precision == IFILT_PREC_FP64 ? 8 : 4;
  const size_t n = (size_t)h.n_rows;
  size_t srcs = (size_t)F * nsys * n * ns * 8 * 2;
  return 4 * n * ns * W * tb + n * ns * W * 8 + 2 * srcs + (size_t)152 * 16 * 2 * W * 8 + (1 << 20);
}

ifilt_status solve_batched(ifilt_mesh_s* m, const ifilt_solve_opts& o, int32_t F, const double* fields, int32_t nk,
                           const double* k, double* out, ifilt_col_stats* stats, cudaStream_t st) {
  const HostPrepared& h = m->host;
  const bool cplx = o.order >= 2 && o.n2_solver != IFILT_N2_REAL;
  const bool blk = h.placement == IFILT_VERTEX_VECTOR;
  const int nsys = h.placement == IFILT_CELL ? 2 : 1;
  const int NS = blk ? 2 : 1;
  const int64_t n = h.n_rows;
  const int nsrc = F * nsys;

  // right-hand sides and initial guesses of every (field, system), device order
  double* srcbuf = (double*)scratch_alloc((size_t)2 * nsrc * n * NS * sizeof(double) + 512, st);
  double* bsrc = srcbuf;
  double* x0src = srcbuf + (size_t)nsrc * n * NS;
  for (int f = 0; f < F; f++)
    for (int s = 0; s < nsys; s++) {
      const int id = f * nsys + s;
      launch_rhs(m, fields + (int64_t)f * h.n_comp * h.n_in, s, bsrc + (size_t)id * n * NS,
                 x0src + (size_t)id * n * NS, st);
      profile_count(1);
    }

  std::vector<ColumnSpec> all;
  for (int f = 0; f < F; f++)
    for (int s = 0; s < nsys; s++)
      for (int j = 0; j < nk; j++) {
        const double ell = 1.0 / k[j];
        double shift;
        if (o.order == 1) shift = 0.5 * ell * ell;
        else if (cplx) shift = ell * ell / std::sqrt(2.0);
        else shift = 0.5 * ell * ell * ell * ell;
        all.push_back({f, s, j, f * nsys + s, shift});
      }
  const int lanes_per_col = cplx ? 2 : 1;
  int max_lanes = o.max_lanes > 0 ? o.max_lanes : 256;
  const int vecw = o.precision == IFILT_PREC_FP64 ? 2 : 4;
  max_lanes = std::min(max_lanes, kBlock * vecw);
  const int per_batch = std::max(1, max_lanes / lanes_per_col);
  BatchFn fn = pick(o.precision, cplx, blk);
  ifilt_status result = IFILT_OK;
  // CUDA graphs cannot be captured on the legacy default stream, so the
  // iterations run on a private stream ordered after the caller's work.
  cudaStream_t ws = nullptr;
  cudaEvent_t ev = nullptr;
  IFILT_CUDA(cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking));
  IFILT_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  IFILT_CUDA(cudaEventRecord(ev, st));
  IFILT_CUDA(cudaStreamWaitEvent(ws, ev, 0));
  try {
    for (size_t b0 = 0; b0 < all.size(); b0 += per_batch) {
      std::vector<ColumnSpec> part(all.begin() + b0, all.begin() + std::min(all.size(), b0 + per_batch));
      ifilt_status s = fn(m, o, part, nsrc, bsrc, x0src, fields, nk, out, stats, ws);
      if (s != IFILT_OK) result = s;
    }
  } catch (...) {
    cudaStreamSynchronize(ws);
    cudaStreamDestroy(ws);
    cudaEventDestroy(ev);
    throw;
  }
  IFILT_CUDA(cudaEventRecord(ev, ws));
  IFILT_CUDA(cudaStreamWaitEvent(st, ev, 0));
  cudaStreamDestroy(ws);
  cudaEventDestroy(ev);
  scratch_free(srcbuf, st);
  return result;
}

}  // namespace ifilt
