// Device helpers shared by the YLT kernels: exact 128-bit fixed-point sums and the aggregate
// terms applied to them.
#pragma once

#include "ara_internal.cuh"

namespace ara {

constexpr unsigned FULL = 0xffffffffu;

// Retention/limit clamp C(x; R, L) = min(max(x - R, 0), L), evaluated in the same order of
// IEEE operations as the FP64 reference so that results agree bit for bit.
__device__ __forceinline__ double clamp_terms(double x, double R, double L) {
  double ex = __dsub_rn(x, R);
  if (ex < 0.0) ex = 0.0;
  if (ex > L) ex = L;
  return ex;
}

// Exact binary32 -> binary64 widening with integer instructions only (FP64 conversions issue at
// a small fraction of the integer rate on this GPU).  From the IEEE 754 formats: binary32 has an
// 8-bit exponent biased by 127 and a 23-bit fraction, binary64 an 11-bit exponent biased by 1023
// and a 52-bit fraction.  A normal value keeps its significand (fraction << 29) and moves its
// exponent by 1023 - 127 = 896; a subnormal f * 2^-149 with its leading bit at position p becomes
// the normal 2^(p-149) * (f / 2^p); zeros keep their sign; infinities and NaNs map to the
// all-ones exponent with the fraction shifted along.
__device__ __forceinline__ double widen_f32(float x) {
  const uint32_t b = __float_as_uint(x);
  const uint64_t sign = (uint64_t)(b >> 31) << 63;
  const uint32_t ex = (b >> 23) & 0xffu;
  const uint32_t fr = b & 0x7fffffu;
  uint64_t bits;
  if (ex == 0xffu) {
    bits = sign | (0x7ffull << 52) | ((uint64_t)fr << 29);
  } else if (ex != 0u) {
    bits = sign | ((uint64_t)(ex + 896u) << 52) | ((uint64_t)fr << 29);
  } else if (fr == 0u) {
    bits = sign;
  } else {
    const int p = 31 - __clz((int)fr);
    bits = sign | ((uint64_t)(p + 1023 - 149) << 52) | (((uint64_t)fr << (52 - p)) & ((1ull << 52) - 1));
  }
  return __longlong_as_double((long long)bits);
}
__device__ __forceinline__ double to_f64(float x) { return widen_f32(x); }
__device__ __forceinline__ double to_f64(double x) { return x; }

// The same terms with the two clamps done on the bit patterns (only the subtraction is FP64):
// for ex >= +0 and L >= +0 the IEEE order is the integer order of the bit patterns, and a
// negative ex (sign bit set) becomes +0.  The result can differ from clamp_terms only in the
// sign of a zero (ex = -0, or L = -0), which no sum of such terms can see.  Requires finite x
// and R (no NaN).
__device__ __forceinline__ double clamp_terms_bits(double x, double R, double L) {
  const long long b = __double_as_longlong(__dsub_rn(x, R));
  const long long lb = __double_as_longlong(L);
  long long r = b < 0 ? 0 : b;
  r = r > lb ? lb : r;
  return __longlong_as_double(r);
}

struct U128 {
  uint64_t lo, hi;
};

__device__ __forceinline__ void add_u64(U128& a, uint64_t v) {
  asm("add.cc.u64 %0, %0, %2;\n\taddc.u64 %1, %1, 0;" : "+l"(a.lo), "+l"(a.hi) : "l"(v));
}
__device__ __forceinline__ void add_u128(U128& a, uint64_t lo, uint64_t hi) {
  asm("add.cc.u64 %0, %0, %2;\n\taddc.u64 %1, %1, %3;" : "+l"(a.lo), "+l"(a.hi) : "l"(lo), "l"(hi));
}
__device__ __forceinline__ bool le_u128(uint64_t alo, uint64_t ahi, uint64_t blo, uint64_t bhi) {
  return ahi < bhi || (ahi == bhi && alo <= blo);
}

template <typename Acc> struct AccOps;
template <> struct AccOps<U128> {
  static __device__ __forceinline__ U128 zero() { return U128{0ull, 0ull}; }
  static __device__ __forceinline__ void add(U128& a, uint64_t v) { add_u64(a, v); }
  static __device__ __forceinline__ U128 warp_sum(U128 a) {
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      const uint64_t l = __shfl_xor_sync(FULL, a.lo, o), h = __shfl_xor_sync(FULL, a.hi, o);
      add_u128(a, l, h);
    }
    return a;
  }
  static __device__ __forceinline__ U128 shfl(U128 a, int src) {
    return U128{__shfl_sync(FULL, a.lo, src), __shfl_sync(FULL, a.hi, src)};
  }
  // Aggregate terms on the exact fixed-point sum; only the result is rounded to double.
  static __device__ __forceinline__ double finish(U128 S, const LayerConst& lc, uint8_t& reg) {
    if (le_u128(S.lo, S.hi, lc.agg_ret_lo, lc.agg_ret_hi)) { reg = 0; return 0.0; }
    U128 d = S;
    asm("sub.cc.u64 %0, %0, %2;\n\tsubc.u64 %1, %1, %3;" : "+l"(d.lo), "+l"(d.hi)
        : "l"(lc.agg_ret_lo), "l"(lc.agg_ret_hi));
    if (le_u128(lc.agg_lim_lo, lc.agg_lim_hi, d.lo, d.hi)) {
      reg = (d.lo == lc.agg_lim_lo && d.hi == lc.agg_lim_hi) ? 0 : 2;
      return lc.agg_lim;
    }
    reg = 1;
    const double v = __dadd_rn(__dmul_rn(__ull2double_rn(d.hi), 18446744073709551616.0),
                               __ull2double_rn(d.lo));
    return __dmul_rn(v, lc.inv_scale);
  }
};
template <> struct AccOps<double> {
  static __device__ __forceinline__ double zero() { return 0.0; }
  static __device__ __forceinline__ void add(double& a, uint64_t v) {
    a = __dadd_rn(a, __longlong_as_double((long long)v));
  }
  static __device__ __forceinline__ double warp_sum(double a) {
#pragma unroll
    for (int o = 16; o; o >>= 1) a = __dadd_rn(a, __shfl_xor_sync(FULL, a, o));
    return a;
  }
  static __device__ __forceinline__ double shfl(double a, int src) { return __shfl_sync(FULL, a, src); }
  static __device__ __forceinline__ double finish(double S, const LayerConst& lc, uint8_t& reg) {
    const double ex = __dsub_rn(S, lc.agg_ret);
    reg = (ex > 0.0 && ex < lc.agg_lim) ? 1 : (ex > lc.agg_lim ? 2 : 0);
    return clamp_terms(S, lc.agg_ret, lc.agg_lim);
  }
};


// Occurrence basis (OEP): the largest occurrence loss of the trial instead of the sum; the
// aggregate terms do not apply.  The fixed-point maximum is exact; only the result is rounded.
struct OepMax {
  uint64_t v;
};
template <> struct AccOps<OepMax> {
  static __device__ __forceinline__ OepMax zero() { return OepMax{0ull}; }
  static __device__ __forceinline__ void add(OepMax& a, uint64_t v) { a.v = a.v > v ? a.v : v; }
  static __device__ __forceinline__ OepMax warp_sum(OepMax a) {
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      const uint64_t b = __shfl_xor_sync(FULL, a.v, o);
      a.v = a.v > b ? a.v : b;
    }
    return a;
  }
  static __device__ __forceinline__ OepMax shfl(OepMax a, int src) { return OepMax{__shfl_sync(FULL, a.v, src)}; }
  static __device__ __forceinline__ double finish(OepMax S, const LayerConst& lc, uint8_t& reg) {
    reg = 0;
    return __dmul_rn(__ull2double_rn(S.v), lc.inv_scale);
  }
};

// Per-lane partial of the current trial in the bulk stream (LaneOps<Acc>::T), reduced over the
// warp into an Acc at the trial's end.
//
// For exact sums the partial is two 64-bit sums of the low and high 32-bit halves of the table
// values, each added with one wide multiply-add (the FMA pipe; no carry chain per value).  A
// chunk that lies inside one trial first sums its K values in 64 bits (K <= 512 values of
// < 2^55 cannot overflow) and adds that sum once.
//
// At the trial's end the lane partial P = lo + hi * 2^32 is split into three 27-bit limbs;
// each limb is summed over the warp by one redux.sync (32 limbs of < 2^27 sum below 2^32) and
// the three sums are recombined into 128 bits.  This needs P < 2^81.  The stream kernel takes a
// warp's event range only below 2^31 - 512 events, so a lane holds fewer than 2^26 values of any
// trial (at most 8 per 256-event chunk, 16 per 512-event chunk, plus one head and one tail
// value), each below 2^55.
template <typename Acc> struct LaneOps;
template <> struct LaneOps<U128> {
  struct T {
    uint64_t lo, hi;
  };
  static __device__ __forceinline__ T zero() { return T{0ull, 0ull}; }
  static __device__ __forceinline__ void add(T& a, uint64_t v) {
    asm("mad.wide.u32 %0, %1, 1, %0;" : "+l"(a.lo) : "r"((uint32_t)v));
    asm("mad.wide.u32 %0, %1, 1, %0;" : "+l"(a.hi) : "r"((uint32_t)(v >> 32)));
  }
  template <int K>
  static __device__ __forceinline__ void add_all(T& a, const uint64_t (&v)[K]) {
    static_assert(K <= 512, "a 64-bit sum holds at most 512 values below 2^55");
    uint64_t s = 0;
#pragma unroll
    for (int i = 0; i < K; ++i) s += v[i];
    add(a, s);
  }
  static __device__ __forceinline__ U128 reduce(T a) {
    const uint64_t p0 = a.lo + (a.hi << 32);                               // bits 0..63 of P
    const uint32_t p1 = (uint32_t)(a.hi >> 32) + (p0 < a.lo ? 1u : 0u);    // bits 64..80
    constexpr uint32_t M = (1u << 27) - 1u;
    const uint32_t s0 = __reduce_add_sync(FULL, (uint32_t)p0 & M);
    const uint32_t s1 = __reduce_add_sync(FULL, (uint32_t)(p0 >> 27) & M);
    const uint32_t s2 = __reduce_add_sync(FULL, (uint32_t)(p0 >> 54) | (p1 << 10));
    U128 r{(uint64_t)s0, 0ull};
    add_u128(r, (uint64_t)s1 << 27, 0ull);
    add_u128(r, (uint64_t)s2 << 54, (uint64_t)(s2 >> 10));
    return r;
  }
};
template <> struct LaneOps<double> {
  using T = double;
  static __device__ __forceinline__ T zero() { return 0.0; }
  static __device__ __forceinline__ void add(T& a, uint64_t v) { AccOps<double>::add(a, v); }
  template <int K>
  static __device__ __forceinline__ void add_all(T& a, const uint64_t (&v)[K]) {
#pragma unroll
    for (int i = 0; i < K; ++i) add(a, v[i]);
  }
  static __device__ __forceinline__ double reduce(T a) { return AccOps<double>::warp_sum(a); }
};
template <> struct LaneOps<OepMax> {
  using T = OepMax;
  static __device__ __forceinline__ T zero() { return OepMax{0ull}; }
  static __device__ __forceinline__ void add(T& a, uint64_t v) { AccOps<OepMax>::add(a, v); }
  template <int K>
  static __device__ __forceinline__ void add_all(T& a, const uint64_t (&v)[K]) {
#pragma unroll
    for (int i = 0; i < K; ++i) add(a, v[i]);
  }
  static __device__ __forceinline__ OepMax reduce(T a) { return AccOps<OepMax>::warp_sum(a); }
};

}  // namespace ara
