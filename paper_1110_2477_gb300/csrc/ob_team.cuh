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
// Team operations used by the level passes.  Every thread of the team calls
// each operation (uniform control flow); lane() runs over 0..W-1.
//   prev(v, c)           value of lane-1 (lane 0 gets c)
//   prev_last(v, c, l)   prev(v, c), and l = value of lane W-1
//   count_le(v, q)       number of lanes with v <= q, for v nondecreasing in lane
//   count(p), any(p)     number of lanes with p / whether any lane has p
//   excl_sum(v, tot)     exclusive prefix sum over lanes, tot = the sum
//   seg_min(v, h, c)     inclusive min-scan over lanes restarted at heads h,
//                        continuing the previous tile's c (updated to the last lane)

// One warp.
struct WarpTeam {
  static constexpr int W = 32;
  __device__ __forceinline__ int lane() const { return threadIdx.x & 31; }
  __device__ __forceinline__ void sync() const { __syncwarp(); }
  template <class T>
  __device__ __forceinline__ T bcast0(T v) const { return __shfl_sync(0xffffffffu, v, 0); }
  template <class T>
  __device__ __forceinline__ T prev(T v, T carry) const {
    T r = __shfl_up_sync(0xffffffffu, v, 1);
    return lane() == 0 ? carry : r;
  }
  template <class T>
  __device__ __forceinline__ T prev_last(T v, T carry, T& last) const {
    last = __shfl_sync(0xffffffffu, v, 31);
    return prev(v, carry);
  }
  __device__ __forceinline__ int count_le(int v, int q) const {
    int pos = 0;  // binary search over the lanes' (sorted) values
    for (int step = 16; step >= 1; step >>= 1) {
      const int x = __shfl_sync(0xffffffffu, v, pos + step - 1);
      if (x <= q) pos += step;
    }
    const int x = __shfl_sync(0xffffffffu, v, 31);
    if (pos == 31 && x <= q) pos = 32;
    return pos;
  }
  __device__ __forceinline__ int count(bool p) const { return __popc(__ballot_sync(0xffffffffu, p)); }
  __device__ __forceinline__ bool any(bool p) const { return __ballot_sync(0xffffffffu, p) != 0u; }
  __device__ __forceinline__ int excl_sum(int v, int& total) const {
    const int l = lane();
    int x = v;
    for (int d = 1; d < 32; d <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, d);
      if (l >= d) x += y;
    }
    total = __shfl_sync(0xffffffffu, x, 31);
    return x - v;
  }
  __device__ __forceinline__ long long seg_min(long long v, bool head, long long& carry) const {
    const int l = lane();
    int fl = head ? 1 : 0;
    for (int d = 1; d < 32; d <<= 1) {
      const long long vu = __shfl_up_sync(0xffffffffu, v, d);
      const int fu = __shfl_up_sync(0xffffffffu, fl, d);
      if (l >= d) {
        if (!fl) v = kmin(v, vu);
        fl |= fu;
      }
    }
    if (!fl) v = kmin(v, carry);
    carry = __shfl_sync(0xffffffffu, v, 31);
    return v;
  }
  // seg_min that also carries the index of the minimum
  __device__ __forceinline__ void seg_argmin(long long& v, int& ix, bool head, long long& cv,
                                             int& ci) const {
    const int l = lane();
    int fl = head ? 1 : 0;
    for (int d = 1; d < 32; d <<= 1) {
      const long long vu = __shfl_up_sync(0xffffffffu, v, d);
      const int iu = __shfl_up_sync(0xffffffffu, ix, d);
      const int fu = __shfl_up_sync(0xffffffffu, fl, d);
      if (l >= d) {
        if (!fl && vu < v) { v = vu; ix = iu; }
        fl |= fu;
      }
    }
    if (!fl && cv < v) { v = cv; ix = ci; }
    cv = __shfl_sync(0xffffffffu, v, 31);
    ci = __shfl_sync(0xffffffffu, ix, 31);
  }
  __device__ __forceinline__ double sum(double v) const {
    for (int d = 16; d >= 1; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
    return v;
  }
};

template <class T>
__device__ __forceinline__ long long to_ll(T v);
template <>
__device__ __forceinline__ long long to_ll<int>(int v) { return (long long)v; }
template <>
__device__ __forceinline__ long long to_ll<long long>(long long v) { return v; }
template <>
__device__ __forceinline__ long long to_ll<double>(double v) { return __double_as_longlong(v); }
template <class T>
__device__ __forceinline__ T from_ll(long long v);
template <>
__device__ __forceinline__ int from_ll<int>(long long v) { return (int)v; }
template <>
__device__ __forceinline__ long long from_ll<long long>(long long v) { return v; }
template <>
__device__ __forceinline__ double from_ll<double>(long long v) { return __longlong_as_double(v); }

// All threads of one CTA (NW warps, W = 32 NW lanes) working on one option.
// Exchanges go through a shared-memory buffer of BUF slots.
template <int NW>
struct BlockTeam {
  static constexpr int W = 32 * NW;
  static constexpr int BUF = W + 4 * NW + 8;
  long long* buf;
  __device__ __forceinline__ int lane() const { return threadIdx.x; }
  __device__ __forceinline__ void sync() const { __syncthreads(); }
  template <class T>
  __device__ __forceinline__ T bcast0(T v) const {
    if (threadIdx.x == 0) buf[W] = to_ll(v);
    __syncthreads();
    const T r = from_ll<T>(buf[W]);
    __syncthreads();
    return r;
  }
  template <class T>
  __device__ __forceinline__ T prev(T v, T carry) const {
    buf[threadIdx.x] = to_ll(v);
    __syncthreads();
    const T r = threadIdx.x ? from_ll<T>(buf[threadIdx.x - 1]) : carry;
    __syncthreads();
    return r;
  }
  template <class T>
  __device__ __forceinline__ T prev_last(T v, T carry, T& last) const {
    buf[threadIdx.x] = to_ll(v);
    __syncthreads();
    const T r = threadIdx.x ? from_ll<T>(buf[threadIdx.x - 1]) : carry;
    last = from_ll<T>(buf[W - 1]);
    __syncthreads();
    return r;
  }
  __device__ __forceinline__ int count_le(int v, int q) const {
    buf[threadIdx.x] = v;
    __syncthreads();
    int lo = 0, hi = W;  // first slot with value > q
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if ((int)buf[mid] <= q) lo = mid + 1; else hi = mid;
    }
    __syncthreads();
    return lo;
  }
  __device__ __forceinline__ int count(bool p) const { return __syncthreads_count(p ? 1 : 0); }
  __device__ __forceinline__ bool any(bool p) const { return __syncthreads_or(p ? 1 : 0) != 0; }
  __device__ __forceinline__ int excl_sum(int v, int& total) const {
    const int l = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
    for (int d = 1; d < 32; d <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, d);
      if (l >= d) x += y;
    }
    if (l == 31) buf[W + w] = x;
    __syncthreads();
    int off = 0, tot = 0;
    for (int k = 0; k < NW; ++k) {
      const int c = (int)buf[W + k];
      if (k < w) off += c;
      tot += c;
    }
    __syncthreads();
    total = tot;
    return off + x - v;
  }
  __device__ __forceinline__ long long seg_min(long long v, bool head, long long& carry) const {
    const int l = threadIdx.x & 31, w = threadIdx.x >> 5;
    int fl = head ? 1 : 0;
    for (int d = 1; d < 32; d <<= 1) {
      const long long vu = __shfl_up_sync(0xffffffffu, v, d);
      const int fu = __shfl_up_sync(0xffffffffu, fl, d);
      if (l >= d) {
        if (!fl) v = kmin(v, vu);
        fl |= fu;
      }
    }
    if (l == 31) {
      buf[W + 2 * w] = v;
      buf[W + 2 * w + 1] = fl;
    }
    __syncthreads();
    if (!fl) {  // no head in this warp up to here: continue from earlier warps, then the carry
      bool stop = false;
      for (int k = w - 1; k >= 0 && !stop; --k) {
        v = kmin(v, buf[W + 2 * k]);
        stop = buf[W + 2 * k + 1] != 0;
      }
      if (!stop) v = kmin(v, carry);
    }
    if (threadIdx.x == W - 1) buf[W + 2 * NW] = v;
    __syncthreads();
    carry = buf[W + 2 * NW];
    __syncthreads();
    return v;
  }
  __device__ __forceinline__ void seg_argmin(long long& v, int& ix, bool head, long long& cv,
                                             int& ci) const {
    const int l = threadIdx.x & 31, w = threadIdx.x >> 5;
    int fl = head ? 1 : 0;
    for (int d = 1; d < 32; d <<= 1) {
      const long long vu = __shfl_up_sync(0xffffffffu, v, d);
      const int iu = __shfl_up_sync(0xffffffffu, ix, d);
      const int fu = __shfl_up_sync(0xffffffffu, fl, d);
      if (l >= d) {
        if (!fl && vu < v) { v = vu; ix = iu; }
        fl |= fu;
      }
    }
    if (l == 31) {
      buf[W + 3 * w] = v;
      buf[W + 3 * w + 1] = ix;
      buf[W + 3 * w + 2] = fl;
    }
    __syncthreads();
    if (!fl) {
      bool stop = false;
      for (int k = w - 1; k >= 0 && !stop; --k) {
        if (buf[W + 3 * k] < v) { v = buf[W + 3 * k]; ix = (int)buf[W + 3 * k + 1]; }
        stop = buf[W + 3 * k + 2] != 0;
      }
      if (!stop && cv < v) { v = cv; ix = ci; }
    }
    if (threadIdx.x == W - 1) { buf[W + 3 * NW] = v; buf[W + 3 * NW + 1] = ix; }
    __syncthreads();
    cv = buf[W + 3 * NW];
    ci = (int)buf[W + 3 * NW + 1];
    __syncthreads();
  }
  __device__ __forceinline__ double sum(double v) const {
    for (int d = 16; d >= 1; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
    if ((threadIdx.x & 31) == 0) buf[W + (threadIdx.x >> 5)] = __double_as_longlong(v);
    __syncthreads();
    double t = 0.0;
    for (int k = 0; k < NW; ++k) t += __longlong_as_double(buf[W + k]);
    __syncthreads();
    return t;
  }
};
#endif

}  // namespace obk
