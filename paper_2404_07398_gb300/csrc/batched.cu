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
#include <cstring>
#include <mutex>
#include <vector>

#include "common.cuh"

namespace ifilt {

int grid_for(const void* kernel, int block, size_t smem, long long work_items) {
  int dev = 0, sms = kNumSMs, occ = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, block, smem);
  if (occ < 1) occ = 1;
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
  int* live;        // [1] number of active columns
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
  if (tr < RPP) {
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
        stp(r + off, ro);
        stp(p + off, ro);
        stp(d + off, zo);
      }
    }
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

// x64 += d
template <typename T>
__global__ void accumulate_kernel(int64_t total, double* __restrict__ x64, const T* __restrict__ d) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
    x64[i] += (double)d[i];
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

template <typename T, typename MV, bool CPLX, bool BLK>
ifilt_status run_batch(ifilt_mesh_s* m, const ifilt_solve_opts& o, const std::vector<ColumnSpec>& cols,
                       int nsrc_total, const double* bsrc_all, const double* x0src_all, const double* fields,
                       int32_t nk, double* out, ifilt_col_stats* stats, cudaStream_t st) {
  (void)nsrc_total;
  const HostPrepared& h = m->host;
  constexpr int VEC = Pack<T>::N;
  constexpr int NS = BLK ? 2 : 1;
  const int lanes_per_col = CPLX ? 2 : 1;
  const int ncols_real = (int)cols.size();
  int W = ncols_real * lanes_per_col;
  W = (W + 3) / 4 * 4;
  if (W / VEC > kBlock) fail(IFILT_EINVAL, "batch too wide (%d lanes)", W);
  const int ncols = W / lanes_per_col;
  const int64_t n = h.n_rows;
  const bool use_g2 = (o.order >= 2) && !CPLX;
  const DevEll& E = use_g2 ? m->ell_g2 : m->ell_k;
  EllView<MV> A = ell_view<MV>(E);
  EllView<double> A64 = ell_view<double>(E);

  // sources used by this batch: compact them
  std::vector<int> src_ids;
  for (auto& c : cols)
    if (std::find(src_ids.begin(), src_ids.end(), c.src) == src_ids.end()) src_ids.push_back(c.src);
  const int nsrc = (int)src_ids.size();

  // launch geometry
  const size_t smem_spmm = (size_t)(kBlock / (W / VEC)) * W * sizeof(double);
  const size_t smem_upd = (size_t)(kBlock / (W / VEC)) * (W + W / 2) * sizeof(double);
  const size_t smem_res = (size_t)(kBlock / (W / VEC)) * 2 * W * sizeof(double);
  const long long rows_work = n * (long long)(W / VEC);
  const int nb = grid_for((const void*)spmm_kernel<T, MV, CPLX, BLK>, kBlock, smem_spmm, rows_work);
  const int pstride = 2 * W;

  // scratch
  const size_t vb = vec_bytes<T>(n, NS, W);
  const size_t xb = (size_t)n * NS * W * sizeof(double);
  const size_t sb = (size_t)nsrc * n * NS * sizeof(double);
  size_t total = 4 * vb + xb + 2 * sb + (size_t)nb * pstride * 8 + (size_t)ncols * (8 * 16 + 4 * 8) +
                 (size_t)W * 4 + 64 * 256;
  char* base = (char*)scratch_alloc(total, st);
  char* cur = base;
  auto take = [&](size_t bytes) {
    char* p = cur;
    cur += (bytes + 255) / 256 * 256;
    return (void*)p;
  };
  T* d = (T*)take(vb);
  T* r = (T*)take(vb);
  T* p = (T*)take(vb);
  T* q = (T*)take(vb);
  double* x64 = (double*)take(xb);
  double* bs = (double*)take(sb);
  double* x0s = (double*)take(sb);
  double* partial = (double*)take((size_t)nb * pstride * 8);
  Cols C{};
  C.shift = (double*)take(ncols * 8);
  C.rho = (double*)take(2 * ncols * 8);
  C.alpha = (double*)take(2 * ncols * 8);
  C.beta = (double*)take(2 * ncols * 8);
  C.rn2 = (double*)take(ncols * 8);
  C.target2 = (double*)take(ncols * 8);
  C.r0n2 = (double*)take(ncols * 8);
  C.tol2 = (double*)take(ncols * 8);
  C.rel = (double*)take(ncols * 8);
  C.active = (int*)take(ncols * 4);
  C.done = (int*)take(ncols * 4);
  C.iters = (int*)take(ncols * 4);
  C.rounds = (int*)take(ncols * 4);
  C.status = (int*)take(ncols * 4);
  C.live = (int*)take(4);
  int* lane_src = (int*)take(W * 4);
  int64_t* col_out = (int64_t*)take(ncols * 8);
  int64_t* col_in = (int64_t*)take(ncols * 8);

  // host-side column tables
  std::vector<double> shift(ncols, 0.0), neg(ncols, -1.0), zeros(2 * ncols, 0.0);
  std::vector<int> done(ncols, 0), izero(ncols, 0), lsrc(W, 0);
  std::vector<int64_t> cout_(ncols, -1), cin(ncols, 0);
  for (int c = 0; c < ncols; c++) {
    if (c < ncols_real) {
      const ColumnSpec& cs = cols[c];
      shift[c] = cs.shift;
      int s = (int)(std::find(src_ids.begin(), src_ids.end(), cs.src) - src_ids.begin());
      for (int t = 0; t < lanes_per_col; t++) lsrc[c * lanes_per_col + t] = s;
      const int comp = h.placement == IFILT_CELL ? cs.sys : 0;
      cout_[c] = (((int64_t)cs.f * nk + cs.kj) * h.n_comp + comp) * h.n_out;
      cin[c] = ((int64_t)cs.f * h.n_comp + comp) * h.n_in;
    } else {
      done[c] = 1;
    }
  }
  auto up = [&](void* dst, const void* src, size_t bytes) {
    IFILT_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st));
  };
  up(C.shift, shift.data(), ncols * 8);
  up(C.r0n2, neg.data(), ncols * 8);
  up(C.rho, zeros.data(), 2 * ncols * 8);
  up(C.alpha, zeros.data(), 2 * ncols * 8);
  up(C.beta, zeros.data(), 2 * ncols * 8);
  up(C.done, done.data(), ncols * 4);
  up(C.active, izero.data(), ncols * 4);
  up(C.iters, izero.data(), ncols * 4);
  up(C.rounds, izero.data(), ncols * 4);
  up(C.status, izero.data(), ncols * 4);
  up(C.live, izero.data(), 4);
  up(lane_src, lsrc.data(), W * 4);
  up(col_out, cout_.data(), ncols * 8);
  up(col_in, cin.data(), ncols * 8);
  for (int s = 0; s < nsrc; s++) {
    IFILT_CUDA(cudaMemcpyAsync(bs + (size_t)s * n * NS, bsrc_all + (size_t)src_ids[s] * n * NS,
                               n * NS * sizeof(double), cudaMemcpyDeviceToDevice, st));
    IFILT_CUDA(cudaMemcpyAsync(x0s + (size_t)s * n * NS, x0src_all + (size_t)src_ids[s] * n * NS,
                               n * NS * sizeof(double), cudaMemcpyDeviceToDevice, st));
  }

  Params P{};
  P.n = (int32_t)n;
  P.W = W;
  P.ncols = ncols;
  P.pstride = pstride;
  P.maxit = o.max_iter > 0 ? o.max_iter : 100000;
  P.tol2_rel = o.tol * o.tol;
  const double itol = (sizeof(T) == 8) ? 0.0 : (o.inner_tol > 0 ? o.inner_tol : 1e-4);
  P.inner2 = itol * itol;

  const int fin_grid = (ncols + 31) / 32;
  const dim3 fin_block(32, 8);
  const int ew_grid = grid_for((const void*)accumulate_kernel<T>, kBlock, 0, n * NS * W);

  init_x_kernel<CPLX, BLK><<<ew_grid, kBlock, 0, st>>>(P, x0s, lane_src, x64);
  IFILT_CUDA(cudaGetLastError());

  // capture m iterations in a graph
  const int m_it = o.check_every > 0 ? o.check_every : 32;
  const bool prof = profiling_on();
  cudaEvent_t ev[6] = {};
  if (prof)
    for (auto& e : ev) IFILT_CUDA(cudaEventCreate(&e));
  IFILT_CUDA(cudaFuncSetAttribute(spmm_kernel<T, MV, CPLX, BLK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem_spmm));
  IFILT_CUDA(cudaFuncSetAttribute(update_kernel<T, CPLX, BLK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem_upd));
  IFILT_CUDA(cudaFuncSetAttribute(residual_kernel<T, CPLX, BLK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem_res));
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  IFILT_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  for (int it = 0; it < m_it; it++) {
    if (prof && it == 0) cudaEventRecord(ev[0], st);
    spmm_kernel<T, MV, CPLX, BLK><<<nb, kBlock, smem_spmm, st>>>(A, P, p, q, m->mass, C, partial);
    if (prof && it == 0) cudaEventRecord(ev[1], st);
    finish_alpha_kernel<CPLX><<<fin_grid, fin_block, 0, st>>>(P, nb, partial, C);
    if (prof && it == 0) cudaEventRecord(ev[2], st);
    update_kernel<T, CPLX, BLK><<<nb, kBlock, smem_upd, st>>>(P, d, p, r, q, C, partial);
    if (prof && it == 0) cudaEventRecord(ev[3], st);
    finish_beta_kernel<CPLX><<<fin_grid, fin_block, 0, st>>>(P, nb, partial, C);
    if (prof && it == 0) cudaEventRecord(ev[4], st);
    direction_kernel<T, CPLX, BLK><<<nb, kBlock, 0, st>>>(P, p, r, C);
    if (prof && it == 0) cudaEventRecord(ev[5], st);
  }
  cudaError_t cap = cudaStreamEndCapture(st, &graph);
  if (cap != cudaSuccess) fail(IFILT_ECUDA, "graph capture failed: %s", cudaGetErrorString(cap));
  IFILT_CUDA(cudaGraphInstantiate(&exec, graph, 0));

  int* h_flags = nullptr;
  IFILT_CUDA(cudaMallocHost(&h_flags, sizeof(int) * (2 * ncols + 1)));
  double t_spmm = 0, t_upd = 0, t_dir = 0;
  int64_t samples = 0, graph_launches = 0;
  const int max_rounds = 64;
  const int round_cap = std::max(P.maxit, 1);
  for (int round = 0; round < max_rounds; round++) {
    residual_kernel<T, CPLX, BLK><<<nb, kBlock, smem_res, st>>>(A64, P, x64, bs, lane_src, m->mass, C, r, d, p,
                                                               partial);
    finish_residual_kernel<CPLX><<<fin_grid, fin_block, 0, st>>>(P, nb, partial, C);
    IFILT_CUDA(cudaGetLastError());
    IFILT_CUDA(cudaMemcpyAsync(h_flags, C.live, sizeof(int), cudaMemcpyDeviceToHost, st));
    IFILT_CUDA(cudaStreamSynchronize(st));
    if (h_flags[0] == 0) break;
    int inner = 0;
    while (true) {
      IFILT_CUDA(cudaGraphLaunch(exec, st));
      graph_launches++;
      IFILT_CUDA(cudaMemcpyAsync(h_flags, C.live, sizeof(int), cudaMemcpyDeviceToHost, st));
      IFILT_CUDA(cudaStreamSynchronize(st));
      if (prof) {
        float a = 0, b = 0, c = 0;
        if (cudaEventElapsedTime(&a, ev[0], ev[1]) == cudaSuccess &&
            cudaEventElapsedTime(&b, ev[2], ev[3]) == cudaSuccess &&
            cudaEventElapsedTime(&c, ev[4], ev[5]) == cudaSuccess && h_flags[0] > 0) {
          t_spmm += a;
          t_upd += b;
          t_dir += c;
          samples++;
        }
      }
      inner += m_it;
      if (h_flags[0] == 0 || inner >= round_cap) break;
    }
    accumulate_kernel<T><<<ew_grid, kBlock, 0, st>>>(n * NS * W, x64, d);
  }
  // results
  {
    dim3 og((unsigned)std::min<long long>((h.n_out + kBlock - 1) / kBlock, 1024), (unsigned)ncols);
    output_kernel<CPLX, BLK><<<og, kBlock, 0, st>>>(P, h.n_out, m->inv_perm, x64, fields, col_out, col_in, out);
    IFILT_CUDA(cudaGetLastError());
  }
  std::vector<int> it_h(ncols), rd_h(ncols), stt_h(ncols), done_h(ncols);
  std::vector<double> rel_h(ncols);
  IFILT_CUDA(cudaMemcpyAsync(it_h.data(), C.iters, ncols * 4, cudaMemcpyDeviceToHost, st));
  IFILT_CUDA(cudaMemcpyAsync(rd_h.data(), C.rounds, ncols * 4, cudaMemcpyDeviceToHost, st));
  IFILT_CUDA(cudaMemcpyAsync(stt_h.data(), C.status, ncols * 4, cudaMemcpyDeviceToHost, st));
  IFILT_CUDA(cudaMemcpyAsync(done_h.data(), C.done, ncols * 4, cudaMemcpyDeviceToHost, st));
  IFILT_CUDA(cudaMemcpyAsync(rel_h.data(), C.rel, ncols * 8, cudaMemcpyDeviceToHost, st));
  IFILT_CUDA(cudaStreamSynchronize(st));

  ifilt_status result = IFILT_OK;
  const int nsys = h.placement == IFILT_CELL ? 2 : 1;
  for (int c = 0; c < ncols_real; c++) {
    const ColumnSpec& cs = cols[c];
    int status = stt_h[c] != 0 || !done_h[c] || rel_h[c] > o.tol ? IFILT_NOT_CONVERGED : IFILT_OK;
    if (status != IFILT_OK) result = IFILT_NOT_CONVERGED;
    if (stats) {
      ifilt_col_stats& s = stats[((int64_t)cs.f * nk + cs.kj) * nsys + cs.sys];
      s.iters = it_h[c];
      s.refinements = rd_h[c];
      s.status = status;
      s.pad = 0;
      s.rel_residual = rel_h[c];
    }
  }
  if (prof) {
    const double vbytes = (double)n * NS * W * sizeof(T);
    const double mbytes = (double)E.entries * (4.0 + E.nval * sizeof(MV)) + (double)n * 8.0;
    const int64_t launches = graph_launches * m_it;
    char nm[32];
    snprintf(nm, sizeof nm, "spmm_%s%s_%s", CPLX ? "c" : "r", BLK ? "b" : "s", sizeof(T) == 8 ? "f64" : "f32");
    profile_add(nm, launches, samples, t_spmm, 2.0 * vbytes + mbytes);
    snprintf(nm, sizeof nm, "update_%s%s_%s", CPLX ? "c" : "r", BLK ? "b" : "s", sizeof(T) == 8 ? "f64" : "f32");
    profile_add(nm, launches, samples, t_upd, 6.0 * vbytes);
    snprintf(nm, sizeof nm, "direction_%s%s_%s", CPLX ? "c" : "r", BLK ? "b" : "s", sizeof(T) == 8 ? "f64" : "f32");
    profile_add(nm, launches, samples, t_dir, 3.0 * vbytes);
    for (auto& e : ev) cudaEventDestroy(e);
  }
  cudaGraphExecDestroy(exec);
  cudaGraphDestroy(graph);
  cudaFreeHost(h_flags);
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
