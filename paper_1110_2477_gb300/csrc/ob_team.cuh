// ob_team.cuh -- portable helpers shared by the kernels: order-preserving
// integer keys for doubles and the warp team used by the level passes.
#pragma once
#include <stdint.h>
#include <string.h>

#if defined(__CUDACC__)
#define OB_HD __host__ __device__ __forceinline__
#else
#define OB_HD inline
#endif

namespace obk {

OB_HD long long dbits(double x) {
#if defined(__CUDA_ARCH__)
  return __double_as_longlong(x);
#else
  long long b;
  memcpy(&b, &x, 8);
  return b;
#endif
}

OB_HD double bitsd(long long b) {
#if defined(__CUDA_ARCH__)
  return __longlong_as_double(b);
#else
  double x;
  memcpy(&x, &b, 8);
  return x;
#endif
}

// Order-preserving key: for finite doubles a < b  <=>  okey(a) < okey(b), and
// -0.0 and +0.0 share a key.  On GB300 every FP64 instruction (compare and
// min included) issues on the narrow FP64 pipe, while 64-bit integer compares
// run on the integer ALUs, so all decisions below are made on keys.
OB_HD long long okey(double x) {
  long long b = dbits(x);
  if (b == (long long)0x8000000000000000ULL) b = 0;
  return b ^ ((b >> 63) & 0x7FFFFFFFFFFFFFFFLL);
}

OB_HD double unkey(long long k) { return bitsd(k ^ ((k >> 63) & 0x7FFFFFFFFFFFFFFFLL)); }

OB_HD bool klt(double a, double b) { return okey(a) < okey(b); }
OB_HD bool kle(double a, double b) { return okey(a) <= okey(b); }
OB_HD bool keq(double a, double b) { return okey(a) == okey(b); }
OB_HD bool same_bits(double a, double b) { return dbits(a) == dbits(b); }
OB_HD long long kmin(long long a, long long b) { return a < b ? a : b; }

OB_HD int popc32(unsigned x) {
#if defined(__CUDA_ARCH__)
  return __popc(x);
#else
  return __builtin_popcount(x);
#endif
}

#if defined(__CUDACC__)
// A warp working on one option.  All 32 lanes call every team operation.
struct WarpTeam {
  static constexpr int W = 32;
  __device__ __forceinline__ int lane() const { return threadIdx.x & 31; }
  __device__ __forceinline__ void sync() const { __syncwarp(); }
  __device__ __forceinline__ unsigned ballot(bool p) const { return __ballot_sync(0xffffffffu, p); }
  template <class T>
  __device__ __forceinline__ T shfl(T v, int src) const { return __shfl_sync(0xffffffffu, v, src); }
  template <class T>
  __device__ __forceinline__ T shfl_up(T v, int d) const { return __shfl_up_sync(0xffffffffu, v, d); }
  template <class T>
  __device__ __forceinline__ T shfl_down(T v, int d) const {
    return __shfl_down_sync(0xffffffffu, v, d);
  }
};
#endif

}  // namespace obk
