// Shared device helpers for libdeblur (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda/atomic>
#include <stdint.h>

namespace db {

// ---- storage / accumulation types -----------------------------------------
// Storage T in {double, float, __nv_bfloat16}; arithmetic Acc is double for
// double storage and float otherwise. Reductions (norms, dot products) are
// always finished in double. X is the type of the outer iterate x^(k) and of
// the LSQR correction delta: the accumulating quantities, which stay in Acc
// when T is bfloat16 (its 8-bit significand would otherwise cap the
// reconstruction at ~4e-3 relative, whatever the solver does).
template <typename T> struct Traits { using Acc = float; using X = float; };
template <> struct Traits<double> { using Acc = double; using X = double; };

__device__ __forceinline__ float to_acc(float v) { return v; }
__device__ __forceinline__ double to_acc(double v) { return v; }
__device__ __forceinline__ float to_acc(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename T> __device__ __forceinline__ T from_acc(float v);
template <> __device__ __forceinline__ float from_acc<float>(float v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 from_acc<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
template <typename T> __device__ __forceinline__ T from_acc_d(double v);
template <> __device__ __forceinline__ double from_acc_d<double>(double v) { return v; }

template <typename T, typename A> __device__ __forceinline__ T store_cast(A v);
template <> __device__ __forceinline__ double store_cast<double, double>(double v) { return v; }
template <> __device__ __forceinline__ float store_cast<float, float>(float v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 store_cast<__nv_bfloat16, float>(float v) { return __float2bfloat16_rn(v); }

// i mod m for a power-of-two m (every image side in this library is one),
// correct for negative i.
__device__ __forceinline__ int wrap(int i, int m) { return i & (m - 1); }

// ---- reductions -------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum of NV doubles per thread; result valid in all threads.
// `scratch` needs NV * 32 doubles of shared memory.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* scratch) {
  const int lane = threadIdx.x & 31, wid = (threadIdx.x + threadIdx.y * blockDim.x) >> 5;
  const int nw = (blockDim.x * blockDim.y) >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = warp_sum(v[k]);
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) scratch[k * 32 + wid] = v[k];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double s = (lane < nw) ? scratch[k * 32 + lane] : 0.0;
    v[k] = warp_sum(s);
  }
  __syncthreads();
}

// Compensated (error-free TwoSum) warp reduction of float partials: returns
// hi + lo in double on every lane. Keeps the sum to about twice float
// precision without FP64 arithmetic, whose rate is a small fraction of FP32
// on this part.
__device__ __forceinline__ double warp_sum_comp(float v) {
  float s = v, c = 0.f;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float s2 = __shfl_xor_sync(0xffffffffu, s, o);
    const float c2 = __shfl_xor_sync(0xffffffffu, c, o);
    const float t = s + s2;
    const float bp = t - s;
    const float e = (s - (t - bp)) + (s2 - bp);
    c = c + c2 + e;
    s = t;
  }
  return (double)s + (double)c;
}
__device__ __forceinline__ double warp_sum_comp(double v) { return warp_sum(v); }

// Double-float arithmetic on the FP32 pipe: (hi, lo) += (xh, xl) with the
// rounding error of hi + xh recovered exactly (TwoSum) and carried in lo.
__device__ __forceinline__ void df_add(float& hi, float& lo, float xh, float xl) {
  const float s = hi + xh;
  const float bp = s - hi;
  const float e = (hi - (s - bp)) + (xh - bp);
  lo = lo + xl + e;
  hi = s;
}

// (hi, lo) += a * b with the product entered exactly: its rounding error is
// recovered with one FMA and carried in lo.
__device__ __forceinline__ void df_fma(float& hi, float& lo, float a, float b) {
  const float p = a * b;
  df_add(hi, lo, p, fmaf(a, b, -p));
}

// (hi, lo) += p[0], p[1], ..., p[n-1] in that order, the loads issued in
// batches of 8 (L1 bypassed: the partials were written by other blocks), so
// the chain waits for one memory round trip per batch, not per element.
__device__ __forceinline__ void df_sum_loads(const float2* p, int n, float& hi, float& lo) {
  int c = 0;
  for (; c + 8 <= n; c += 8) {
    float2 q[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) q[k] = __ldcg(p + c + k);
#pragma unroll
    for (int k = 0; k < 8; ++k) df_add(hi, lo, q[k].x, q[k].y);
  }
  for (; c < n; ++c) {
    const float2 v = __ldcg(p + c);
    df_add(hi, lo, v.x, v.y);
  }
}

// Warp sum of double-float pairs (hi, lo) with a fixed xor butterfly; every
// lane ends with the same total.
__device__ __forceinline__ float2 warp_df_pair(float hi, float lo) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float h2 = __shfl_xor_sync(0xffffffffu, hi, o);
    const float l2 = __shfl_xor_sync(0xffffffffu, lo, o);
    df_add(hi, lo, h2, l2);
  }
  return make_float2(hi, lo);
}

// Block sum of NV per-thread partials (float or double); the result (double)
// is valid in thread (0,0) only. `scratch` needs NV * 32 doubles. The warp
// totals are combined by warp 0 with a fixed butterfly (no serial chain of
// double additions).
template <int NV, typename A>
__device__ __forceinline__ void block_sum_to0(const A (&v)[NV], double (&out)[NV], double* scratch) {
  const int tid = threadIdx.x + threadIdx.y * blockDim.x;
  const int lane = tid & 31, wid = tid >> 5;
  const int nw = (blockDim.x * blockDim.y) >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    const double w = warp_sum_comp(v[k]);
    if (lane == 0) scratch[k * 32 + wid] = w;
  }
  __syncthreads();
  if (wid == 0) {
    double s[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) s[k] = lane < nw ? scratch[k * 32 + lane] : 0.0;
#pragma unroll
    for (int k = 0; k < NV; ++k) s[k] = warp_sum(s[k]);
#pragma unroll
    for (int k = 0; k < NV; ++k) out[k] = s[k];
  }
  __syncthreads();
}

// ---- timing / bounded waits ------------------------------------------------
__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// State of the grid-wide phase barrier of the persistent LSQR launch
// (lsqr_phase_arrive / lsqr_wait_release): an arrival counter that only
// grows, the generation published by the block that arrived last, a
// timeout flag every waiting block checks, and that block's decision.
struct GridBarrier {
  unsigned int count;
  unsigned int gen;
  int error;      // 0 ok, 1 timeout
  int decision;   // written by the last block to arrive, read by all after release
};


}  // namespace db
