// Device helpers shared by the solve kernels.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include "internal.h"

namespace ifilt {

constexpr int kNumSMs = 152;          // GB300: 2 dies x 76 SMs (queried at run time where it matters)

template <typename T>
__device__ __forceinline__ double to_d(T v) { return (double)v; }
template <>
__device__ __forceinline__ double to_d<__nv_bfloat16>(__nv_bfloat16 v) { return (double)__bfloat162float(v); }

template <typename T>
__device__ __forceinline__ float to_f(T v) { return (float)v; }
template <>
__device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

// Read-only view of a sliced ELL operator with value storage MV.
template <typename MV>
struct EllView {
  const int64_t* __restrict__ slice_off;
  const int32_t* __restrict__ slice_w;
  const int32_t* __restrict__ col;
  const MV* __restrict__ val;
  int32_t slice_h;
  const uint8_t* __restrict__ rowq;  // per-row length in fours (see DevEll), or null
};

template <typename MV>
inline EllView<MV> ell_view(const DevEll& e);
template <>
inline EllView<double> ell_view<double>(const DevEll& e) { return {e.slice_off, e.slice_w, e.col, e.val64, e.slice_h, e.rowq}; }
template <>
inline EllView<float> ell_view<float>(const DevEll& e) { return {e.slice_off, e.slice_w, e.col, e.val32, e.slice_h, e.rowq}; }
template <>
inline EllView<__nv_bfloat16> ell_view<__nv_bfloat16>(const DevEll& e) { return {e.slice_off, e.slice_w, e.col, e.val16, e.slice_h, e.rowq}; }

// Grid size for a bandwidth-bound kernel: whole waves of resident CTAs.
int grid_for(const void* kernel, int block, size_t smem, long long work_items);

}  // namespace ifilt
