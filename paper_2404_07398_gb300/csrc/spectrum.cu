// Coarse-grained energy spectrum from filtered fields.  The paper computes
// spectra from fields filtered over a sequence of scales (Sect. 1, 4, 5) and
// prints no formula; the reading implemented here:
//   E_f(k_j) = sum_o w_o 1/2 sum_c phi_{f,j,c}(o)^2 / sum_o w_o   (w = lumped mass, 0 on land)
//   spec_f,j = (E_f(k_{j+1}) - E_f(k_j)) / (k_{j+1} - k_j),   kmid_j = sqrt(k_j k_{j+1})
#include <cmath>

#include "common.cuh"

namespace ifilt {
namespace {

constexpr int kBlock = 256;

// partial[fk][b] = sum over the block's share of o of w_o * 1/2 sum_c x^2
__global__ void energy_partial_kernel(int32_t n_out, int ncomp, const double* __restrict__ w,
                                      const double* __restrict__ x, double* __restrict__ partial) {
  __shared__ double sm[kBlock / 32];
  const int fk = blockIdx.y;
  const double* xf = x + (int64_t)fk * ncomp * n_out;
  double s = 0.0;
  for (int32_t o = blockIdx.x * blockDim.x + threadIdx.x; o < n_out; o += gridDim.x * blockDim.x) {
    const double wo = w[o];
    double e = 0.0;
    for (int c = 0; c < ncomp; c++) {
      const double v = xf[(int64_t)c * n_out + o];
      e += v * v;
    }
    s += wo * 0.5 * e;
  }
#pragma unroll
  for (int o = 16; o > 0; o /= 2) s += __shfl_down_sync(0xffffffffu, s, o);
  if (threadIdx.x % 32 == 0) sm[threadIdx.x / 32] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < kBlock / 32; i++) t += sm[i];
    partial[(int64_t)fk * gridDim.x + blockIdx.x] = t;
  }
}

// One block per field: energies of its n_k scales, then the differences.
__global__ void spectrum_final_kernel(int nb, int nk, double inv_wsum, const double* __restrict__ partial,
                                      const double* __restrict__ k, double* __restrict__ energy,
                                      double* __restrict__ spec, double* __restrict__ kmid) {
  const int f = blockIdx.x;
  for (int j = threadIdx.x; j < nk; j += blockDim.x) {
    const double* p = partial + ((int64_t)f * nk + j) * nb;
    double s = 0.0;
    for (int b = 0; b < nb; b++) s += p[b];
    energy[f * nk + j] = s * inv_wsum;
  }
  __syncthreads();
  for (int j = threadIdx.x; j + 1 < nk; j += blockDim.x) {
    const double dk = k[j + 1] - k[j];
    spec[f * (nk - 1) + j] = (energy[f * nk + j + 1] - energy[f * nk + j]) / dk;
    if (f == 0) kmid[j] = sqrt(k[j] * k[j + 1]);
  }
}

}  // namespace

// energy/spec/kmid are device buffers here; the ABI copies them to the host.
void spectrum_device(ifilt_mesh_s* m, int32_t F, int32_t nk, const double* k_dev, const double* filtered,
                     double* energy, double* spec, double* kmid, double* partial, int nb, cudaStream_t st) {
  const HostPrepared& h = m->host;
  double wsum = 0.0;
  for (double a : h.mass) wsum += a;
  dim3 grid((unsigned)nb, (unsigned)(F * nk));
  energy_partial_kernel<<<grid, kBlock, 0, st>>>(h.n_out, h.n_comp, m->w_out, filtered, partial);
  spectrum_final_kernel<<<F, 64, 0, st>>>(nb, nk, 1.0 / wsum, partial, k_dev, energy, spec, kmid);
  IFILT_CUDA(cudaGetLastError());
}

}  // namespace ifilt
