// Device-side building blocks shared by the ihsbin kernels.
//
//  * dd   : a float-float ("double-float") value hi + lo built from error-free
//           transformations -- Knuth's TwoSum, Dekker's FastTwoSum and the
//           FMA-based exact product (Dekker, Numer. Math. 18, 1971).  It carries
//           about 44-48 significant bits at FP32-pipe throughput, which on
//           GB300 is several times the FP64 rate.
//  * Mode : compile-time precision policies.  F64 = IEEE double everywhere;
//           DD = float-float for every accuracy-critical contraction.
//  * Philox4x32-10 (Salmon et al., SC'11) counter-based generator for the
//           sketch draws.  Stream layout: key = (seed lo32, seed hi32),
//           counter = (index lo32, index hi32, stream, 0).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

namespace ihsbin {

// ----------------------------------------------------------------- status word
// Device kernels never trap: they record the first fault in a status word the
// host reads at the next synchronisation point.
enum DevStatus : int { DEV_OK = 0, DEV_NOT_SPD = 4, DEV_NAN = 11, DEV_BOUNDS = 12, DEV_TIMEOUT = 13 };

__device__ __forceinline__ void dev_fail(int* status, int code) {
  if (status) atomicCAS(status, 0, code);
}

// ------------------------------------------------------------------ float-float
struct dd {
  float hi, lo;
};

__device__ __forceinline__ dd two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ dd fast_two_sum(float a, float b) {  // requires |a| >= |b| or a == 0
  float s = __fadd_rn(a, b);
  float e = __fsub_rn(b, __fsub_rn(s, a));
  return {s, e};
}
__device__ __forceinline__ dd two_prod(float a, float b) {
  float p = __fmul_rn(a, b);
  float e = __fmaf_rn(a, b, -p);
  return {p, e};
}
__device__ __forceinline__ dd dd_from_double(double x) {
  float h = __double2float_rn(x);
  float l = __double2float_rn(x - (double)h);
  return {h, l};
}
__device__ __forceinline__ double dd_to_double(dd a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ dd dd_renorm(dd a) { return fast_two_sum(a.hi, a.lo); }
__device__ __forceinline__ dd dd_neg(dd a) { return {-a.hi, -a.lo}; }

__device__ __forceinline__ dd dd_add(dd a, dd b) {
  dd s = two_sum(a.hi, b.hi);
  dd t = two_sum(a.lo, b.lo);
  s.lo = __fadd_rn(s.lo, t.hi);
  s = fast_two_sum(s.hi, s.lo);
  s.lo = __fadd_rn(s.lo, t.lo);
  return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ dd dd_sub(dd a, dd b) { return dd_add(a, dd_neg(b)); }
// An int64 as a float-float value with 32-bit conversions only (64-bit integer <-> float
// conversions run on the FP64 pipe): x = a 2^48 + b 2^32 + c 2^16 + d with a signed and b, c, d
// in [0, 2^16), every part exact in FP32; each pair adds exactly (TwoSum), the two pairs with a
// float-float addition (relative error about 2^-48).
__device__ __forceinline__ dd ll_to_dd(long long x) {
  const unsigned long long u = (unsigned long long)x;
  const int a = (int)(x >> 48);
  const unsigned b = (unsigned)(u >> 32) & 0xffffu, c = (unsigned)(u >> 16) & 0xffffu, d = (unsigned)u & 0xffffu;
  return dd_add(two_sum((float)a * 281474976710656.f, (float)b * 4294967296.f),
                two_sum((float)c * 65536.f, (float)d));
}
// x 2^k, exact unless the result leaves the normal range (then as ldexpf)
__device__ __forceinline__ float scale_pow2(float x, int k) {
  return (k >= -126 && k <= 127) ? x * __int_as_float((k + 127) << 23) : ldexpf(x, k);
}

// Exact-slice products (tc_loop.cu) leave, per output entry, the exact integers
//   hi = acc_0 2^24 + acc_1 2^16 + acc_2 2^8 + acc_3,  lo = acc_4 2^16 + acc_5 2^8 + acc_6
// of the weight accumulators; the entry is 2^(e_row + e_col - 38) hi + 2^(e_row + e_col - 62) lo.
// Sum of the n exact int64 partials of the k-splits at off, off + stride, ... (two arrays): the
// loads go out four splits at a time, so a consumer waits for one memory round trip per four
// splits instead of one per split, with few registers held (bandwidth-bound consumers keep
// their occupancy).  Integer addition is exact, so the order does not matter.
__device__ __forceinline__ void oz_sum_splits(const long long* __restrict__ a, const long long* __restrict__ b, int n,
                                              int64_t stride, int64_t off, long long& sa, long long& sb) {
  sa = 0;
  sb = 0;
  for (int s0 = 0; s0 < n; s0 += 4) {
    long long va[4], vb[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const bool in = s0 + q < n;
      va[q] = in ? __ldg(a + (int64_t)(s0 + q) * stride + off) : 0LL;
      vb[q] = in ? __ldg(b + (int64_t)(s0 + q) * stride + off) : 0LL;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      sa += va[q];
      sb += vb[q];
    }
  }
}
constexpr int OZ_EXP_NONFINITE = 1 << 20;  // row/column exponent marking an Inf/NaN entry
__device__ __forceinline__ dd oz_join(long long hi, long long lo, int erow, int ecol) {
  if (erow == OZ_EXP_NONFINITE || ecol == OZ_EXP_NONFINITE) return dd{__int_as_float(0x7fc00000), 0.f};
  const int sc = erow + ecol;
  const dd yh = ll_to_dd(hi), yl = ll_to_dd(lo);
  return dd_add(dd{scale_pow2(yh.hi, sc - 38), scale_pow2(yh.lo, sc - 38)},
                dd{scale_pow2(yl.hi, sc - 62), scale_pow2(yl.lo, sc - 62)});
}
__device__ __forceinline__ dd dd_mul(dd a, dd b) {
  dd p = two_prod(a.hi, b.hi);
  p.lo = __fmaf_rn(a.hi, b.lo, p.lo);
  p.lo = __fmaf_rn(a.lo, b.hi, p.lo);
  return fast_two_sum(p.hi, p.lo);
}
// Quotient by one Newton correction of the FP32 quotient: q1 = a.hi / b.hi,
// r = a - q1 b (float-float), q = q1 + r.hi / b.hi.
__device__ __forceinline__ dd dd_div(dd a, dd b) {
  float q1 = __fdiv_rn(a.hi, b.hi);
  dd r = dd_sub(a, dd_mul({q1, 0.f}, b));
  float q2 = __fdiv_rn(r.hi, b.hi);
  return fast_two_sum(q1, q2);
}
// Square root by one Newton correction of sqrtf: s = sqrt(a.hi), r = a - s^2, x = s + r / (2 s).
__device__ __forceinline__ dd dd_sqrt(dd a) {
  if (a.hi <= 0.f) return {0.f, 0.f};
  float s = __fsqrt_rn(a.hi);
  dd r = dd_sub(a, two_prod(s, s));
  float c = __fdiv_rn(r.hi, 2.f * s);
  return fast_two_sum(s, c);
}

// ------------------------------------------------------------------ precision modes
// A matrix held "in compute precision" is a pair of raw pointers: F64 uses p0
// as double*; DD uses p0 (hi) and p1 (lo) as float*.
struct CBuf {
  void* p0 = nullptr;
  void* p1 = nullptr;
};

struct F64 {
  using V = double;
  static constexpr int id = 0;
  __device__ __forceinline__ static V zero() { return 0.0; }
  __device__ __forceinline__ static V ld(const CBuf& b, int64_t i) { return ((const double*)b.p0)[i]; }
  __device__ __forceinline__ static void st(const CBuf& b, int64_t i, V v) { ((double*)b.p0)[i] = v; }
  __device__ __forceinline__ static V add(V a, V b) { return a + b; }
  __device__ __forceinline__ static V sub(V a, V b) { return a - b; }
  __device__ __forceinline__ static V mul(V a, V b) { return a * b; }
  __device__ __forceinline__ static V div(V a, V b) { return a / b; }
  __device__ __forceinline__ static V sqrt_(V a) { return ::sqrt(a); }
  __device__ __forceinline__ static V from_d(double x) { return x; }
  __device__ __forceinline__ static double to_d(V v) { return v; }
  __device__ __forceinline__ static V renorm(V v) { return v; }
  __device__ __forceinline__ static V neg_(V v) { return -v; }
  __device__ __forceinline__ static void mac(V& acc, V a, V b) { acc = fma(a, b, acc); }
  __device__ __forceinline__ static void mac(V& acc, float a, float b) {
    acc = fma((double)a, (double)b, acc);
  }
};

struct DD {
  using V = dd;
  static constexpr int id = 1;
  __device__ __forceinline__ static V zero() { return {0.f, 0.f}; }
  __device__ __forceinline__ static V ld(const CBuf& b, int64_t i) {
    return {((const float*)b.p0)[i], ((const float*)b.p1)[i]};
  }
  __device__ __forceinline__ static void st(const CBuf& b, int64_t i, V v) {
    ((float*)b.p0)[i] = v.hi;
    ((float*)b.p1)[i] = v.lo;
  }
  __device__ __forceinline__ static V add(V a, V b) { return dd_add(a, b); }
  __device__ __forceinline__ static V sub(V a, V b) { return dd_sub(a, b); }
  __device__ __forceinline__ static V mul(V a, V b) { return dd_mul(a, b); }
  __device__ __forceinline__ static V div(V a, V b) { return dd_div(a, b); }
  __device__ __forceinline__ static V sqrt_(V a) { return dd_sqrt(a); }
  __device__ __forceinline__ static V from_d(double x) { return dd_from_double(x); }
  __device__ __forceinline__ static double to_d(V v) { return dd_to_double(v); }
  __device__ __forceinline__ static V renorm(V v) { return dd_renorm(v); }
  __device__ __forceinline__ static V neg_(V v) { return dd_neg(v); }
  // acc += a * b with both operands float-float: the exact product of the high
  // parts plus the two cross terms, added to the accumulator by TwoSum; the
  // low word is left unnormalised (callers renormalise every few steps).
  __device__ __forceinline__ static void mac(V& acc, V a, V b) {
    dd p = two_prod(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.lo, p.lo);
    e = __fmaf_rn(a.lo, b.hi, e);
    dd s = two_sum(acc.hi, p.hi);
    acc.hi = s.hi;
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(s.lo, e));
  }
  // one exact float operand (FP32/BF16 data) times a float-float value
  __device__ __forceinline__ static void mac(V& acc, float a, V b) {
    dd p = two_prod(a, b.hi);
    float e = __fmaf_rn(a, b.lo, p.lo);
    dd s = two_sum(acc.hi, p.hi);
    acc.hi = s.hi;
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(s.lo, e));
  }
  __device__ __forceinline__ static void mac(V& acc, V a, float b) { mac(acc, b, a); }
  // both operands exact floats (e.g. FP32 or BF16 data): the product is exact.
  __device__ __forceinline__ static void mac(V& acc, float a, float b) {
    dd p = two_prod(a, b);
    dd s = two_sum(acc.hi, p.hi);
    acc.hi = s.hi;
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(s.lo, p.lo));
  }
};

// ------------------------------------------------------------------ Philox4x32-10
struct u32x4 {
  uint32_t x, y, z, w;
};

__host__ __device__ __forceinline__ void mulhilo32(uint32_t a, uint32_t b, uint32_t& hi, uint32_t& lo) {
  uint64_t p = (uint64_t)a * (uint64_t)b;
  hi = (uint32_t)(p >> 32);
  lo = (uint32_t)p;
}

__host__ __device__ __forceinline__ u32x4 philox4x32_10(u32x4 c, uint32_t k0, uint32_t k1) {
  const uint32_t MA = 0xD2511F53u, MB = 0xCD9E8D57u;
  const uint32_t WA = 0x9E3779B9u, WB = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += WA;
      k1 += WB;
    }
    uint32_t h0, l0, h1, l1;
    mulhilo32(MA, c.x, h0, l0);
    mulhilo32(MB, c.z, h1, l1);
    c = {h1 ^ c.y ^ k0, l1, h0 ^ c.w ^ k1, l0};
  }
  return c;
}

__host__ __device__ __forceinline__ u32x4 rng_draw(uint64_t seed, uint32_t stream, uint64_t index) {
  return philox4x32_10({(uint32_t)index, (uint32_t)(index >> 32), stream, 0u}, (uint32_t)seed,
                       (uint32_t)(seed >> 32));
}

enum RngStream : uint32_t {
  STREAM_COUNTSKETCH = 3,
  STREAM_GAUSSIAN = 5,
  STREAM_SRHT_SIGN = 6,
  STREAM_SRHT_KEY = 7
};

// Programmatic dependent launch.  A kernel launched with programmatic stream serialization may
// start while its predecessor in the stream still runs: pdl_wait() returns once the predecessor
// has completed and its memory is visible (immediately when there is none), so it must come
// before the first access to anything the predecessor may read or write.  pdl_trigger() lets
// the successor start launching (its prologue then overlaps the rest of this kernel).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Launch with programmatic stream serialization (the kernel must call pdl_wait first).
template <typename... P, typename... A>
inline cudaError_t launch_pdl(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              A&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<P>(args)...);
}

// Launch as clusters of `cl` CTAs along x (grid.x a multiple of cl), with programmatic stream
// serialization (the kernel must call pdl_wait first).
template <typename... P, typename... A>
inline cudaError_t launch_pdl_cluster(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem, int cl,
                                      cudaStream_t st, A&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  attr[1].id = cudaLaunchAttributeClusterDimension;
  attr[1].val.clusterDim.x = (unsigned)cl;
  attr[1].val.clusterDim.y = 1;
  attr[1].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<P>(args)...);
}

// ------------------------------------------------------------------ element loads
__device__ __forceinline__ float bf16_to_f(uint16_t b) {
  return __uint_as_float(((uint32_t)b) << 16);
}

// Read element i of a raw array of the given storage type, widened exactly.
enum ElemType : int { ELEM_F64 = 0, ELEM_F32 = 1, ELEM_BF16 = 2 };

__device__ __forceinline__ double load_elem_d(const void* p, int et, int64_t i) {
  if (et == ELEM_F64) return ((const double*)p)[i];
  if (et == ELEM_F32) return (double)((const float*)p)[i];
  return (double)bf16_to_f(((const uint16_t*)p)[i]);
}

}  // namespace ihsbin
