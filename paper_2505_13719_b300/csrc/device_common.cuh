// Device helpers shared by the kernels: 16-byte vector access to factor rows,
// group shuffles and the deterministic block -> grid reduction.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace hallar {

constexpr int kBlock = 256;  // threads per block of every row kernel

// 16-byte vectors of the factor element type -------------------------------
template <class T> struct V16;
template <> struct V16<double> {
  using type = double2;
  static constexpr int N = 2;
  __device__ static inline void unpack(const double2& v, double* o) { o[0] = v.x; o[1] = v.y; }
  __device__ static inline double2 pack(const double* o) { return make_double2(o[0], o[1]); }
};
template <> struct V16<float> {
  using type = float4;
  static constexpr int N = 4;
  __device__ static inline void unpack(const float4& v, float* o) {
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
  }
  __device__ static inline float4 pack(const float* o) { return make_float4(o[0], o[1], o[2], o[3]); }
};

template <class T>
__device__ inline void load_chunk(const T* __restrict__ base, int64_t off, T* o) {
  using VT = typename V16<T>::type;
  VT v = __ldg(reinterpret_cast<const VT*>(base + off));
  V16<T>::unpack(v, o);
}
template <class T>
__device__ inline void load_chunk_l2(const T* __restrict__ base, int64_t off, T* o) {
  // gathered neighbour rows: served from L2, no L1 allocation
  using VT = typename V16<T>::type;
  VT v = __ldcg(reinterpret_cast<const VT*>(base + off));
  V16<T>::unpack(v, o);
}
template <class T>
__device__ inline void store_chunk(T* base, int64_t off, const T* o) {
  using VT = typename V16<T>::type;
  *reinterpret_cast<VT*>(base + off) = V16<T>::pack(o);
}

// typed arithmetic: the explicit intrinsics keep float operations in float
// (an unqualified fma or fabs on floats can resolve to the double overload
// and round-trip through the FP64 pipe)
__device__ __forceinline__ float tfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double tfma(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float tabs(float a) { return fabsf(a); }
__device__ __forceinline__ double tabs(double a) { return ::fabs(a); }

// per-thread accumulation in the factor precision --------------------------
// double adds directly.  float uses Neumaier's compensated summation (1974):
// on B300 every double instruction (conversions included) occupies the FP64
// pipe for many cycles, so the float form keeps its per-row sums in float
// and carries the rounding error of each addition in a second float; the
// partial becomes a double only once per thread.
template <class T> struct Acc;
template <> struct Acc<double> {
  double s = 0.0;
  __device__ inline void add(double x) { s += x; }
  __device__ inline double value() const { return s; }
};
template <> struct Acc<float> {
  float s = 0.0f, c = 0.0f;
  __device__ inline void add(float x) {
    const float t = s + x;
    c += (fabsf(s) >= fabsf(x)) ? (s - t) + x : (x - t) + s;
    s = t;
  }
  __device__ inline double value() const { return (double)s + (double)c; }
};

// sum over the G lanes of a group (G a power of two, groups aligned) -------
template <int G, class T>
__device__ inline T group_sum(T v, unsigned mask) {
#pragma unroll
  for (int off = G / 2; off > 0; off >>= 1) v += __shfl_xor_sync(mask, v, off, G);
  return v;
}
// value v of lane t of the group (G = 1: the thread's own value, no shuffle)
template <int G, class V>
__device__ __forceinline__ V group_bcast(V v, int t, unsigned mask) {
  if constexpr (G == 1) {
    return v;
  } else {
    return __shfl_sync(mask, v, t, G);
  }
}
template <int G>
__device__ inline unsigned group_mask() {
  if (G == 32) return 0xffffffffu;
  unsigned lane = threadIdx.x & 31u;
  unsigned base = lane & ~(unsigned)(G - 1);
  return ((1u << (G & 31)) - 1u) << base;
}

// deterministic reduction of NS doubles over the grid ------------------------
// Every block reduces its threads' values (fixed tree), writes one partial
// per scalar, and the last block to finish sums the partials in block order
// (fixed assignment of blocks to threads, then the same fixed tree), writes
// out[0..NS) and re-arms the counter.  Results do not depend on scheduling.
template <int NS>
__device__ inline void block_sum(double (&v)[NS], double (*sh)[kBlock / 32]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    double x = v[s];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
    if (lane == 0) sh[s][warp] = x;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      double x = 0.0;
      for (int w = 0; w < kBlock / 32; ++w) x += sh[s][w];
      v[s] = x;
    }
  }
  __syncthreads();
}

template <int NS>
__device__ inline void grid_reduce(double (&v)[NS], double* __restrict__ partials,
                                   unsigned* counter, double* out) {
  __shared__ double sh[NS][kBlock / 32];
  __shared__ bool am_last;
  block_sum<NS>(v, sh);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int s = 0; s < NS; ++s) partials[(size_t)blockIdx.x * NS + s] = v[s];
    __threadfence();
    unsigned prev = atomicAdd(counter, 1u);
    am_last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (!am_last) return;
  __threadfence();
  double acc[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) acc[s] = 0.0;
  for (unsigned b = threadIdx.x; b < gridDim.x; b += kBlock) {
#pragma unroll
    for (int s = 0; s < NS; ++s) acc[s] += __ldcg(&partials[(size_t)b * NS + s]);
  }
  block_sum<NS>(acc, sh);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int s = 0; s < NS; ++s) out[s] = acc[s];
    *counter = 0u;
  }
}

// grid reduction of per-thread accumulators: the warp stage runs in the
// accumulator's own precision (float pairs combined with TwoSum for the
// compensated float form), so each warp converts to double once; the block
// and grid stages are grid_reduce's.
__device__ inline void acc_combine(Acc<double>& a, double s, double) { a.s += s; }
__device__ inline void acc_combine(Acc<float>& a, float s, float c) {
  const float t = a.s + s;
  const float bb = t - a.s;
  const float err = (a.s - (t - bb)) + (s - bb);
  a.s = t;
  a.c += c + err;
}
__device__ inline double acc_c(const Acc<double>&) { return 0.0; }
__device__ inline float acc_c(const Acc<float>& a) { return a.c; }

template <class T, int NS>
__device__ inline void grid_reduce_acc(Acc<T> (&acc)[NS], double* __restrict__ partials,
                                       unsigned* counter, double* out) {
  __shared__ double shw[NS][kBlock / 32];
  __shared__ bool am_last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    T cs = (T)acc_c(acc[s]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const T os = __shfl_xor_sync(0xffffffffu, acc[s].s, off);
      const T oc = __shfl_xor_sync(0xffffffffu, cs, off);
      Acc<T> tmp = acc[s];
      acc_combine(tmp, os, oc);
      acc[s] = tmp;
      cs = (T)acc_c(acc[s]);
    }
    if (lane == 0) shw[s][warp] = acc[s].value();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      double x = 0.0;
      for (int w = 0; w < kBlock / 32; ++w) x += shw[s][w];
      partials[(size_t)blockIdx.x * NS + s] = x;
    }
    __threadfence();
    am_last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!am_last) return;
  __threadfence();
  double tot[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) tot[s] = 0.0;
  for (unsigned b = threadIdx.x; b < gridDim.x; b += kBlock) {
#pragma unroll
    for (int s = 0; s < NS; ++s) tot[s] += __ldcg(&partials[(size_t)b * NS + s]);
  }
  __shared__ double sh2[NS][kBlock / 32];
  block_sum<NS>(tot, sh2);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int s = 0; s < NS; ++s) out[s] = tot[s];
    *counter = 0u;
  }
}

}  // namespace hallar
