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
constexpr long long KMAXLL = 0x7fffffffffffffffLL;

// smallest power of two >= w
OB_HD constexpr int pow2_ceil(int w) {
  int p = 1;
  while (p < w) p <<= 1;
  return p;
}

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
  // counts of lanes with v <= q1 and v <= q2 (v nondecreasing in lane)
  __device__ __forceinline__ void count_le2(int v, int q1, int q2, int& c1, int& c2) const {
    c1 = count_le(v, q1);
    c2 = __popc(__ballot_sync(0xffffffffu, v <= q2));  // q2 is the same on all lanes
  }
  // values of lanes l-1 and l-2 (carries for lanes 0 and 1) and of lanes W-1 and W-2
  template <class T>
  __device__ __forceinline__ void look2(T v, T c1, T c2, T& m1, T& m2, T& l1, T& l2) const {
    const int l = lane();
    const T a = __shfl_up_sync(0xffffffffu, v, 1), b = __shfl_up_sync(0xffffffffu, v, 2);
    m1 = (l >= 1) ? a : c1;
    m2 = (l >= 2) ? b : (l == 1 ? c1 : c2);
    l1 = __shfl_sync(0xffffffffu, v, 31);
    l2 = __shfl_sync(0xffffffffu, v, 30);
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

// Barrier b (1..15) for the n threads of a sub-team of a CTA, and its reductions.
__device__ __forceinline__ void bar_sync(int b, int n) {
  asm volatile("bar.sync %0, %1;" ::"r"(b), "r"(n) : "memory");
}
__device__ __forceinline__ int bar_popc(int b, int n, bool p) {
  int r;
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.ne.s32 q, %1, 0;\n\tbar.red.popc.u32 %0, %2, %3, q;\n\t}"
      : "=r"(r)
      : "r"(p ? 1 : 0), "r"(b), "r"(n)
      : "memory");
  return r;
}

// The threads of one CTA (NW warps, W = 32 NW lanes) working on one option; SUB: the
// team is the W threads from thread `base` on, one of several teams of the CTA, and
// meets at barrier `bar` instead of the CTA's.
// Exchanges go through shared memory, two halves used alternately, so that one
// barrier per exchange suffices: a half is rewritten only after the next
// exchange's barrier, which every thread reaches after its reads of that half.
template <int NW, bool SUB = false>
struct BlockTeam {
  static constexpr int W = 32 * NW;
  static constexpr int HALF = W + 4 * NW + 8;
  static constexpr int BUF = 2 * HALF;
  long long* buf;
  int base = 0;  // SUB: first thread of the team
  int bar = 0;   // SUB: its barrier
  mutable int par = 0;
  __device__ __forceinline__ long long* half() const {
    long long* h = buf + par * HALF;
    par ^= 1;
    return h;
  }
  __device__ __forceinline__ int lane() const { return SUB ? (int)threadIdx.x - base : (int)threadIdx.x; }
  __device__ __forceinline__ void sync() const {
    if (SUB) bar_sync(bar, W);
    else __syncthreads();
  }
  template <class T>
  __device__ __forceinline__ T bcast0(T v) const {
    long long* h = half();
    if (lane() == 0) h[0] = to_ll(v);
    sync();
    return from_ll<T>(h[0]);
  }
  template <class T>
  __device__ __forceinline__ T prev(T v, T carry) const {
    long long* h = half();
    h[lane()] = to_ll(v);
    sync();
    return lane() ? from_ll<T>(h[lane() - 1]) : carry;
  }
  template <class T>
  __device__ __forceinline__ T prev_last(T v, T carry, T& last) const {
    long long* h = half();
    h[lane()] = to_ll(v);
    sync();
    last = from_ll<T>(h[W - 1]);
    return lane() ? from_ll<T>(h[lane() - 1]) : carry;
  }
  template <class T>
  __device__ __forceinline__ void look2(T v, T c1, T c2, T& m1, T& m2, T& l1, T& l2) const {
    long long* h = half();
    const int l = lane();
    h[l] = to_ll(v);
    sync();
    m1 = (l >= 1) ? from_ll<T>(h[l - 1]) : c1;
    m2 = (l >= 2) ? from_ll<T>(h[l - 2]) : (l == 1 ? c1 : c2);
    l1 = from_ll<T>(h[W - 1]);
    l2 = from_ll<T>(h[W - 2]);
  }
  __device__ __forceinline__ int count_le(int v, int q) const {
    int c1, c2;
    count_le2(v, q, q, c1, c2);
    return c1;
  }
  __device__ __forceinline__ void count_le2(int v, int q1, int q2, int& c1, int& c2) const {
    long long* h = half();
    h[lane()] = v;
    sync();
    // first slots with value > q1 and > q2: both searches advance together over the
    // next power of two P >= W (slots past W read as +infinity)
    constexpr int P = pow2_ceil(W);
    int lo1 = 0, lo2 = 0;
    for (int step = P >> 1; step >= 1; step >>= 1) {
      const int i1 = lo1 + step - 1, i2 = lo2 + step - 1;
      if (i1 < W && (int)h[i1] <= q1) lo1 += step;
      if (i2 < W && (int)h[i2] <= q2) lo2 += step;
    }
    if (P == W) {
      if (lo1 == W - 1 && (int)h[W - 1] <= q1) lo1 = W;
      if (lo2 == W - 1 && (int)h[W - 1] <= q2) lo2 = W;
    }
    c1 = lo1;
    c2 = lo2;
  }
  __device__ __forceinline__ int count(bool p) const { return (SUB ? bar_popc(bar, W, p) : __syncthreads_count(p ? 1 : 0)); }
  __device__ __forceinline__ bool any(bool p) const { return (SUB ? bar_popc(bar, W, p) : __syncthreads_or(p ? 1 : 0)) != 0; }
  __device__ __forceinline__ int excl_sum(int v, int& total) const {
    long long* h = half();
    const int l = lane() & 31, w = lane() >> 5;
    int x = v;
    for (int d = 1; d < 32; d <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, d);
      if (l >= d) x += y;
    }
    if (l == 31) h[W + w] = x;
    sync();
    // across warps: lane k of every warp takes warp k's total and the warp scans them with
    // shuffles; warp w's offset is the inclusive sum of warps 0..w-1
    int c = (l < NW) ? (int)h[W + l] : 0;
    for (int d = 1; d < NW; d <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, c, d);
      if (l >= d) c += y;
    }
    const int before = __shfl_sync(0xffffffffu, c, (w + 31) & 31);
    total = __shfl_sync(0xffffffffu, c, NW - 1);
    return (w ? before : 0) + x - v;
  }
  __device__ __forceinline__ long long seg_min(long long v, bool head, long long& carry) const {
    long long* h = half();
    const int l = lane() & 31, w = lane() >> 5;
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
      h[W + 2 * w] = v;
      h[W + 2 * w + 1] = fl;
    }
    sync();
    // across warps: lane k of every warp takes warp k's record and the warp runs the
    // segmented scan over lanes 0..NW-1 with shuffles; acc_k = head in warp k ? its value :
    // min(acc_{k-1}, its value), acc_{-1} = carry
    long long rv = KMAXLL;
    int rf = 0;
    if (l < NW) {
      rv = h[W + 2 * l];
      rf = (int)h[W + 2 * l + 1];
    }
    if (l == 0 && !rf) rv = kmin(rv, carry);
    for (int d = 1; d < NW; d <<= 1) {
      const long long vu = __shfl_up_sync(0xffffffffu, rv, d);
      const int fu = __shfl_up_sync(0xffffffffu, rf, d);
      if (l >= d) {
        if (!rf) rv = kmin(rv, vu);
        rf |= fu;
      }
    }
    const long long before = __shfl_sync(0xffffffffu, rv, (w + 31) & 31);  // acc_{w-1}
    if (!fl) v = kmin(v, w ? before : carry);
    carry = __shfl_sync(0xffffffffu, rv, NW - 1);
    return v;
  }
  __device__ __forceinline__ void seg_argmin(long long& v, int& ix, bool head, long long& cv,
                                             int& ci) const {
    long long* h = half();
    const int l = lane() & 31, w = lane() >> 5;
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
      h[W + 3 * w] = v;
      h[W + 3 * w + 1] = ix;
      h[W + 3 * w + 2] = fl;
    }
    sync();
    // across warps as in seg_min, carrying the index; among equal minima the latest wins
    long long rv = KMAXLL;
    int ri = 0, rf = 0;
    if (l < NW) {
      rv = h[W + 3 * l];
      ri = (int)h[W + 3 * l + 1];
      rf = (int)h[W + 3 * l + 2];
    }
    if (l == 0 && !rf && cv < rv) { rv = cv; ri = ci; }
    for (int d = 1; d < NW; d <<= 1) {
      const long long vu = __shfl_up_sync(0xffffffffu, rv, d);
      const int iu = __shfl_up_sync(0xffffffffu, ri, d);
      const int fu = __shfl_up_sync(0xffffffffu, rf, d);
      if (l >= d) {
        if (!rf && vu < rv) { rv = vu; ri = iu; }
        rf |= fu;
      }
    }
    const int src = (w + 31) & 31;
    const long long bv = w ? __shfl_sync(0xffffffffu, rv, src) : cv;
    const int bi = w ? __shfl_sync(0xffffffffu, ri, src) : ci;
    if (!fl && bv < v) { v = bv; ix = bi; }
    cv = __shfl_sync(0xffffffffu, rv, NW - 1);
    ci = __shfl_sync(0xffffffffu, ri, NW - 1);
  }
  __device__ __forceinline__ double sum(double v) const {
    long long* h = half();
    for (int d = 16; d >= 1; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
    if ((lane() & 31) == 0) h[W + (lane() >> 5)] = __double_as_longlong(v);
    sync();
    double t = 0.0;
    for (int k = 0; k < NW; ++k) t += __longlong_as_double(h[W + k]);
    return t;
  }
};
#endif

}  // namespace obk
