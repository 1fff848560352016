// Plain path: one right-hand side at a time in FP64, the way the paper's
// CuPy implementation proceeds (Sect. 2.2.2): for every scale the system
// matrix S = M + 1/2 l^(2n) K (M^-1 K)^(n-1) is assembled explicitly as CSR,
// S x0 is subtracted from the right-hand side (r0 = b - S x0), conjugate
// gradients solve S delta = r0 from delta = 0 with one sparse matrix-vector
// product, separate dot and axpy kernels and a host-side convergence test per
// iteration, and the filtered field is x0 + delta.  This is the baseline the
// batched path is measured against.
//
// Convergence is judged as on the batched path: when the recursive residual
// reaches tol ||r0||, the true residual r0 - S delta is recomputed in FP64; the
// column is converged when that is within tol ||r0||, and otherwise CG restarts
// from it while each restart lowers it (IFILT_NOT_CONVERGED when it stops
// falling or the iteration cap is reached).
#include <algorithm>
#include <cmath>

#include "common.cuh"

namespace ifilt {
namespace {

constexpr int kBlock = 256;

__global__ void assemble_s_kernel(int32_t n, int nsub, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                  const double* __restrict__ gval, const double* __restrict__ mass, double c,
                                  double* __restrict__ sval) {
  for (int32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    const double mr = mass[r / nsub];
    for (int64_t e = rp[r]; e < rp[r + 1]; e++) sval[e] = c * gval[e] + (col[e] == r ? mr : 0.0);
  }
}

// y = A x, TPR threads per row, shuffle reduction within the row group.
template <int TPR>
__global__ void spmv_csr_kernel(int32_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                const double* __restrict__ val, const double* __restrict__ x,
                                double* __restrict__ y) {
  // The loop runs the same number of times in every lane of a warp (rows are
  // taken a warp's worth at a time), so the shuffles below see all 32 lanes.
  const int lane = threadIdx.x % TPR;
  constexpr int RPW = 32 / TPR;  // rows per warp step
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
  const int64_t nwarps = (int64_t)gridDim.x * blockDim.x / 32;
  const int sub = (threadIdx.x % 32) / TPR;
  for (int64_t r0 = warp * RPW; r0 < n; r0 += nwarps * RPW) {
    const int64_t r = r0 + sub;
    double s = 0.0;
    if (r < n)
      for (int64_t e = rp[r] + lane; e < rp[r + 1]; e += TPR) s += val[e] * x[col[e]];
#pragma unroll
    for (int o = TPR / 2; o > 0; o /= 2) s += __shfl_down_sync(0xffffffffu, s, o, TPR);
    if (lane == 0 && r < n) y[r] = s;
  }
}

__global__ void dot_partial_kernel(int32_t n, const double* __restrict__ a, const double* __restrict__ b,
                                   double* __restrict__ partial) {
  __shared__ double sm[kBlock / 32];
  double s = 0.0;
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) s += a[i] * b[i];
#pragma unroll
  for (int o = 16; o > 0; o /= 2) s += __shfl_down_sync(0xffffffffu, s, o);
  if (threadIdx.x % 32 == 0) sm[threadIdx.x / 32] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kBlock / 32; w++) t += sm[w];
    partial[blockIdx.x] = t;
  }
}

__global__ void dot_final_kernel(int nb, const double* __restrict__ partial, double* __restrict__ out) {
  __shared__ double sm[kBlock];
  double s = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) s += partial[i];
  sm[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o /= 2) {
    if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sm[0];
}

// Device scalars of the CG recurrence.
struct Scalars {
  double rho, rho_new, pq;
};

// r = b - y (and p = r when p is given); r may alias b
__global__ void sub_kernel(int32_t n, const double* b, const double* __restrict__ y, double* r,
                           double* __restrict__ p) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double v = b[i] - y[i];
    r[i] = v;
    if (p) p[i] = v;
  }
}

// start of the residual-form solve: r = p = r0, delta = 0
__global__ void start_kernel(int32_t n, const double* __restrict__ r0, double* __restrict__ r,
                             double* __restrict__ p, double* __restrict__ d) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    r[i] = r0[i];
    p[i] = r0[i];
    d[i] = 0.0;
  }
}

// x += d (the filtered field x0 + delta)
__global__ void add_kernel(int32_t n, const double* __restrict__ d, double* __restrict__ x) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) x[i] += d[i];
}

// x += alpha p  with alpha = rho / pq
__global__ void axpy_x_kernel(int32_t n, const Scalars* __restrict__ s, const double* __restrict__ p,
                              double* __restrict__ x) {
  const double alpha = s->rho / s->pq;
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) x[i] += alpha * p[i];
}

// r -= alpha q
__global__ void axpy_r_kernel(int32_t n, const Scalars* __restrict__ s, const double* __restrict__ q,
                              double* __restrict__ r) {
  const double alpha = s->rho / s->pq;
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) r[i] -= alpha * q[i];
}

// p = r + beta p with beta = rho_new / rho; then rho <- rho_new (one thread, after the sweep it reads)
__global__ void xpay_kernel(int32_t n, const Scalars* __restrict__ s, const double* __restrict__ r,
                            double* __restrict__ p) {
  const double beta = s->rho_new / s->rho;
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = r[i] + beta * p[i];
}

__global__ void roll_rho_kernel(Scalars* s) { s->rho = s->rho_new; }

struct PlainWork {
  double *sval, *x, *b, *r, *p, *q, *d, *partial;
  Scalars* sc;
  double* host;  // pinned [1]
};

}  // namespace

// the explicit operator of order n: K, K M^-1 K or G_n
static const DevCSR& order_csr(const ifilt_mesh_s* m, int order) {
  if (order == 1) return m->csr_k;
  if (order == 2) return m->csr_g2;
  if ((size_t)(order - 3) >= m->csr_gn.size()) fail(IFILT_EINVAL, "mesh holds no order-%d operator", order);
  return m->csr_gn[(size_t)order - 3];
}

size_t plain_scratch_bytes(const ifilt_mesh_s* m, const ifilt_solve_opts& o) {
  const DevCSR& G = order_csr(m, o.order);
  size_t n = (size_t)G.n;
  return (size_t)G.nnz * 8 + 7 * n * 8 + 4096 * 8 + 2048;
}

ifilt_status solve_plain(ifilt_mesh_s* m, const ifilt_solve_opts& o, int32_t F, const double* fields, int32_t nk,
                         const double* k, double* out, ifilt_col_stats* stats, cudaStream_t st) {
  const HostPrepared& h = m->host;
  const DevCSR& G = order_csr(m, o.order);
  const int32_t n = G.n;  // real unknowns
  const int nsub = h.placement == IFILT_VERTEX_VECTOR ? 2 : 1;
  const int nsys = h.placement == IFILT_CELL ? 2 : 1;
  const int max_iter = o.max_iter > 0 ? o.max_iter : 100000;
  const int grid = (int)std::min<long long>((n + kBlock - 1) / kBlock, 152LL * 8);
  const int nb = grid;

  PlainWork w{};
  char* base = (char*)scratch_alloc(plain_scratch_bytes(m, o), st);
  char* cur = base;
  auto take = [&](size_t bytes) {
    char* p = cur;
    cur += (bytes + 255) / 256 * 256;
    return p;
  };
  w.sval = (double*)take((size_t)G.nnz * 8);
  w.x = (double*)take((size_t)n * 8);
  w.b = (double*)take((size_t)n * 8);
  w.r = (double*)take((size_t)n * 8);
  w.p = (double*)take((size_t)n * 8);
  w.q = (double*)take((size_t)n * 8);
  w.d = (double*)take((size_t)n * 8);
  w.partial = (double*)take(4096 * 8);
  w.sc = (Scalars*)take(sizeof(Scalars));
  IFILT_CUDA(cudaMallocHost(&w.host, sizeof(double) * 2));

  const double avg = (double)G.nnz / std::max(1, n);
  auto spmv = [&](const double* x, double* y) {
    if (avg <= 8) spmv_csr_kernel<4><<<grid * 2, kBlock, 0, st>>>(n, G.row_ptr, G.col, w.sval, x, y);
    else if (avg <= 24) spmv_csr_kernel<8><<<grid * 2, kBlock, 0, st>>>(n, G.row_ptr, G.col, w.sval, x, y);
    else spmv_csr_kernel<16><<<grid * 2, kBlock, 0, st>>>(n, G.row_ptr, G.col, w.sval, x, y);
  };
  auto dot = [&](const double* a, const double* b, double* dst) {
    dot_partial_kernel<<<nb, kBlock, 0, st>>>(n, a, b, w.partial);
    dot_final_kernel<<<1, kBlock, 0, st>>>(nb, w.partial, dst);
  };
  auto fetch = [&](const double* dev) {
    IFILT_CUDA(cudaMemcpyAsync(w.host, dev, sizeof(double), cudaMemcpyDeviceToHost, st));
    IFILT_CUDA(cudaStreamSynchronize(st));
    return w.host[0];
  };

  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  const bool prof = profiling_on();
  if (prof) {
    IFILT_CUDA(cudaEventCreate(&ev0));
    IFILT_CUDA(cudaEventCreate(&ev1));
  }
  double spmv_ms = 0.0;
  int64_t spmv_samples = 0, spmv_launches = 0;
  // algorithmic bytes of one CSR SpMV: values + column indices + row pointers,
  // one read of x per stored entry's column is counted once per row (x fits L2),
  // plus x read and y written once.
  const double spmv_bytes = (double)G.nnz * 12.0 + (double)(n + 1) * 8.0 + 2.0 * n * 8.0;

  ifilt_status result = IFILT_OK;
  const int64_t out_sys_stride = (int64_t)h.n_out;
  for (int32_t f = 0; f < F; f++) {
    const double* field = fields + (int64_t)f * h.n_comp * h.n_in;
    for (int sys = 0; sys < nsys; sys++) {
      for (int32_t j = 0; j < nk; j++) {
        const double ell = 1.0 / k[j];
        const double c = 0.5 * std::pow(ell, 2.0 * o.order);
        assemble_s_kernel<<<grid, kBlock, 0, st>>>(n, nsub, G.row_ptr, G.col, G.val, m->mass, c, w.sval);
        launch_rhs(m, field, sys, w.b, w.x, st);  // b and x0
        spmv(w.x, w.q);
        sub_kernel<<<grid, kBlock, 0, st>>>(n, w.b, w.q, w.b, nullptr);  // r0 = b - S x0, in place of b
        start_kernel<<<grid, kBlock, 0, st>>>(n, w.b, w.r, w.p, w.d);
        dot(w.r, w.r, &w.sc->rho);
        int64_t launches = 7;
        const double rho0 = fetch(&w.sc->rho);
        const double target = o.tol * std::sqrt(rho0);
        double rho = rho0;
        double best = std::sqrt(rho0);  // smallest true residual so far
        double rt = best;
        int it = 0, rounds = 0;
        bool broke = false, ok = rho0 == 0.0;
        while (!ok) {
          while (std::sqrt(rho) > target && it < max_iter) {
            if (prof && (it % 16) == 0) IFILT_CUDA(cudaEventRecord(ev0, st));
            spmv(w.p, w.q);
            if (prof && (it % 16) == 0) {
              IFILT_CUDA(cudaEventRecord(ev1, st));
            }
            dot(w.p, w.q, &w.sc->pq);
            axpy_x_kernel<<<grid, kBlock, 0, st>>>(n, w.sc, w.p, w.d);
            axpy_r_kernel<<<grid, kBlock, 0, st>>>(n, w.sc, w.q, w.r);
            dot(w.r, w.r, &w.sc->rho_new);
            const double rn = fetch(&w.sc->rho_new);
            if (prof && (it % 16) == 0) {
              float ms = 0.f;
              IFILT_CUDA(cudaEventElapsedTime(&ms, ev0, ev1));
              spmv_ms += ms;
              spmv_samples++;
            }
            spmv_launches++;
            it++;
            launches += 7;
            if (!std::isfinite(rn)) {
              broke = true;
              break;
            }
            xpay_kernel<<<grid, kBlock, 0, st>>>(n, w.sc, w.r, w.p);
            roll_rho_kernel<<<1, 1, 0, st>>>(w.sc);
            launches += 2;
            rho = rn;
          }
          if (broke) break;
          // true residual r0 - S delta in FP64; a restart continues from it (p = r)
          spmv(w.d, w.q);
          sub_kernel<<<grid, kBlock, 0, st>>>(n, w.b, w.q, w.r, w.p);
          dot(w.r, w.r, &w.sc->rho);
          launches += 4;
          rounds++;
          const double tr2 = fetch(&w.sc->rho);
          rt = std::sqrt(tr2);
          if (!std::isfinite(rt)) {
            broke = true;
            break;
          }
          if (rt <= target) {
            ok = true;
            break;
          }
          if (it >= max_iter || !(rt < best)) break;  // capped, or stopped falling
          best = rt;
          rho = tr2;
        }
        const double rel = rho0 > 0 ? rt / std::sqrt(rho0) : 0.0;
        if (!ok) result = IFILT_NOT_CONVERGED;
        add_kernel<<<grid, kBlock, 0, st>>>(n, w.d, w.x);
        double* out_sys = out + (((int64_t)f * nk + j) * h.n_comp + sys) * out_sys_stride;
        launch_output_plain(m, w.x, field, sys, out_sys, st);
        profile_count(launches + 2);  // setup, iterations, true residuals, output
        if (stats) {
          ifilt_col_stats& s = stats[((int64_t)f * nk + j) * nsys + sys];
          s.iters = it;
          s.refinements = rounds;
          s.status = ok ? IFILT_OK : IFILT_NOT_CONVERGED;
          s.pad = 0;
          s.rel_residual = rel;
          s.err_bound = 0.0;
        }
      }
    }
  }
  IFILT_CUDA(cudaStreamSynchronize(st));
  if (prof) {
    profile_add("plain_spmv_csr_fp64", spmv_launches, spmv_samples, spmv_ms, spmv_bytes);
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
  }
  cudaFreeHost(w.host);
  scratch_free(base, st);
  return result;
}

}  // namespace ifilt
