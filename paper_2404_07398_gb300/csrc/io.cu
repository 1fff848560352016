// Right-hand sides, initial guesses and output maps of the filter systems.
//
//   vertex scalar : b = M phi,  x0 = phi                           (Sect. 2.1.1)
//   vertex vector : b = R u_c with R_vc = A_c / 3, x0 = M^-1 b      (Sect. 2.1.2)
//   cell          : b = A_c u_c, x0 = u_c, one component at a time  (Eq. 6)
// The initial guess is the unfiltered field, so the Krylov solve works on the
// remainder b - S x0 (the residual form of Sect. 2.2.2).
#include "common.cuh"

namespace ifilt {
namespace {

__global__ void rhs_scalar_kernel(int32_t n, const int32_t* __restrict__ perm, const double* __restrict__ mass,
                                  const double* __restrict__ field, double* __restrict__ b,
                                  double* __restrict__ x0) {
  for (int32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    double v = field[perm[r]];
    x0[r] = v;
    b[r] = mass[r] * v;
  }
}

__global__ void rhs_vector_kernel(int32_t n, const int64_t* __restrict__ pp, const int32_t* __restrict__ pc,
                                  const double* __restrict__ pw, const double* __restrict__ mass,
                                  const double* __restrict__ u, const double* __restrict__ v,
                                  double* __restrict__ b, double* __restrict__ x0) {
  for (int32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    double bu = 0.0, bv = 0.0;
    for (int64_t e = pp[r]; e < pp[r + 1]; e++) {
      int32_t c = pc[e];
      bu += pw[e] * u[c];
      bv += pw[e] * v[c];
    }
    b[2 * r] = bu;
    b[2 * r + 1] = bv;
    x0[2 * r] = bu / mass[r];
    x0[2 * r + 1] = bv / mass[r];
  }
}

__global__ void output_kernel(int32_t n_out, int nsub, int vector_placement, const int32_t* __restrict__ inv,
                              const double* __restrict__ x, const double* __restrict__ field,
                              double* __restrict__ out, int64_t comp_stride) {
  for (int32_t o = blockIdx.x * blockDim.x + threadIdx.x; o < n_out; o += gridDim.x * blockDim.x) {
    int32_t r = inv[o];
    for (int s = 0; s < nsub; s++) {
      double val;
      if (r >= 0) val = x[(int64_t)r * nsub + s];
      else val = vector_placement ? 0.0 : field[o];
      out[s * comp_stride + o] = val;
    }
  }
}

}  // namespace

void launch_rhs(ifilt_mesh_s* m, const double* field, int comp, double* b, double* x0, cudaStream_t st) {
  const HostPrepared& h = m->host;
  const int32_t n = h.n_rows;
  const int block = 256;
  const int grid = (int)std::min<long long>((n + block - 1) / block, 152LL * 16);
  if (h.placement == IFILT_VERTEX_VECTOR) {
    rhs_vector_kernel<<<grid, block, 0, st>>>(n, m->proj_ptr, m->proj_cell, m->proj_w, m->mass, field,
                                              field + h.n_in, b, x0);
  } else {
    const double* f = field + (int64_t)comp * h.n_in;
    rhs_scalar_kernel<<<grid, block, 0, st>>>(n, m->perm, m->mass, f, b, x0);
  }
  IFILT_CUDA(cudaGetLastError());
}

void launch_output_plain(ifilt_mesh_s* m, const double* x, const double* field, int comp, double* out_sys,
                         cudaStream_t st) {
  const HostPrepared& h = m->host;
  const int block = 256;
  const int grid = (int)std::min<long long>((h.n_out + block - 1) / block, 152LL * 16);
  const bool vec = h.placement == IFILT_VERTEX_VECTOR;
  const double* f = vec ? nullptr : field + (int64_t)comp * h.n_in;
  output_kernel<<<grid, block, 0, st>>>(h.n_out, vec ? 2 : 1, vec ? 1 : 0, m->inv_perm, x, f, out_sys,
                                        (int64_t)h.n_out);
  IFILT_CUDA(cudaGetLastError());
}

}  // namespace ifilt
