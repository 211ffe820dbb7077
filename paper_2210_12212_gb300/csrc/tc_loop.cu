// The two products of every step of the basis recursion (Algorithm 2) in the
// float-float compute mode, on the 5th-generation tensor cores:
//   Y   = A_hat^T A_hat U   (the Gram times the old columns of all live intervals)
//   Z_l = P_l R_l           (interval l's preconditioner times its right-hand sides)
// by the exact-slice method of the Gram kernel (tc_gram.cu), now on both operands:
//  * A operand (the Gram, or P_l; fixed during the recursion): row i scaled by
//    2^(7 - ea_i), ea_i the exponent of its largest magnitude, and cut into
//    OZ_S = 6 integer slices exact in BF16; done once per build;
//  * B operand (the columns of U or R; new every step): column j scaled by
//    2^(7 - eb_j) and cut the same way, every step;
//  * C_ij = 2^(ea_i + eb_j - 14) sum_{s + t <= 6} 2^(-8(s+t)) sum_k a_s(i,k) b_t(k,j).
// The 26 slice pairs of one k-block accumulate by weight w = s + t into seven
// Tensor Memory accumulators.  Between two drains an accumulator receives at most
// 6 pairs x 128 k integer products of magnitude <= 2^14 (|sum| < 2^24: exact in
// its FP32 accumulator); drained chunks add exactly in int32, the weights are
// joined exactly in int64 and written per k-split; the recursion's update kernels
// add the splits exactly and convert to float-float with the row/column exponents.
// Slicing: each entry is rounded to an integer V in units of 2^(e - 47) (|V| <= 2^47,
// e the exponent of its row's / column's largest magnitude) and written as six
// balanced base-256 digits.  Combination: the seven weights are joined exactly in
// int64 (two Horner groups); the conversion to float-float uses FP32 operations only.
// Accuracy: every operand entry is held to 2^-47 of its row's (column's) largest
// magnitude and the dropped pairs weigh at most 2^-52 of the leading product, the
// accuracy class of the float-float contraction these products replace.  A product may
// keep fewer pairs, s + t <= wmax (the residual form's P_l r: its errors are corrected by
// the later steps of the recursion); it then reads only the slices 0 .. wmax of each
// block, and with wmax <= 3 it runs on 128 x 64 tiles (four accumulators of 64 columns fit
// the Tensor Memory twice).
//
// Kernel roles (persistent: one CTA per SM walks the work items, a work item being a
// 128-row tile x NT-column tile x group x k-range): warp 0 (one lane) streams each
// k-block's A slices (up to 48 KiB) and B slices with two bulk copies into a ring of
// stages; warp 1 owns the Tensor Memory and one lane issues one MMA per A slice and
// K = 16 step (M = 128, N = the stacked B slices it meets); the epilogue warps, each
// warpgroup on its own columns, drain finished accumulators into int32 while the MMAs of
// the next chunk (of this or the next item) run into the other buffer, and write either
// the exact int64 partials or, for a product with one k-split, the joined float-float
// value itself.  All waits are bounded in time (DEV_TIMEOUT in the status word).
#include <algorithm>
#include <cfloat>

#include "common.cuh"
#include "internal.h"
#include "tc.cuh"

#include <cooperative_groups.h>
namespace cg = cooperative_groups;

namespace ihsbin {
namespace {

#define CK(x)                              \
  do {                                     \
    cudaError_t e__ = (x);                 \
    if (e__ != cudaSuccess) return e__;    \
  } while (0)

constexpr int OZ_S = 6;              // slices per operand entry
constexpr int OZ_W = 6;              // kept pairs: s + t <= OZ_W
constexpr int OZ_NW = OZ_W + 1;      // weights 0 .. OZ_W
constexpr int OZ_BK = 32;            // k per block
constexpr int OZ_ABLK = 128 * OZ_BK; // A block: 128 rows x 32 k (8 KiB)
constexpr int OZ_CHUNK = 4;          // k-blocks between drains (6 x 128 x 2^14 < 2^24)
constexpr int OZ_KB_MAX = 512;       // k-blocks per CTA (int32 sums: 6 x 16384 x 2^14 < 2^31)
constexpr int OZ_NONFINITE = OZ_EXP_NONFINITE;

// NT = 16 / 32: every weight 0..6 (seven accumulators per buffer).  NT = 64 ("wide"): products
// that keep only the pairs s + t <= 3 (the residual form's P_l r), four accumulators of 64
// columns per buffer, and a stage holding the four slices those pairs read.
template <int NT>
struct OzCfg {
  static constexpr bool WIDE = NT == 64;
  static constexpr int WMAX = WIDE ? 3 : OZ_W;          // largest pair weight the layout holds
  static constexpr int BBLK = NT * OZ_BK;               // B block: NT rows x 32 k
  static constexpr int A_BYTES = (WMAX + 1 < OZ_S ? WMAX + 1 : OZ_S) * OZ_ABLK * 2;  // 48 / 32 KiB
  static constexpr int B_BYTES = (WMAX + 1 < OZ_S ? WMAX + 1 : OZ_S) * BBLK * 2;     // 6 / 12 / 16 KiB
  // plus one all-zero slice where the s = 0 MMA reaches weight 6 (see the MMA issue)
  static constexpr int B_SLOT = B_BYTES + (WIDE ? 0 : BBLK * 2);
  static constexpr int STAGE = A_BYTES + B_SLOT;
  static constexpr int STAGES = NT == 32 ? 3 : 4;
  static constexpr int SMEM = STAGES * STAGE;              // 220 / 186 / 192 KiB
  static constexpr int EPI_WARPS = NT == 16 ? 4 : 8;
  static constexpr int THREADS = 64 + 32 * EPI_WARPS;
  static constexpr int COLS = NT == 16 ? 256 : 512;     // two buffers of (WMAX + 1) NT accumulator columns
  // an epilogue warpgroup drains every weight (WPG) of EC of the tile's columns
  static constexpr int WPG = WMAX + 1;
  static constexpr int EC = NT / (EPI_WARPS / 4);
};

struct OzArgs {
  const __nv_bfloat16* As;
  int64_t a_gstride;     // elements per A group (0: one A shared by every group)
  const int* a_perm;     // group -> A group (nullptr: identity)
  const int* ea;
  int64_t ea_gstride;
  const __nv_bfloat16* Bs;
  int64_t b_gstride;
  const int* eb;
  int64_t eb_gstride;
  int KB;                // k-blocks of the contraction
  int MT, NTL;           // row tiles, column tiles per group
  int64_t M, N;          // valid rows, valid columns per group
  int groups, ksplit, kbper;
  int tri;               // OZ_TRI_* flags: zero blocks of triangular operands skipped per tile
  int sym;               // 1: only tiles that touch i <= j (symmetric result)
  // pair mode: group 2q takes A group q of As (a_perm), group 2q + 1 takes A group q of As2
  // (a_perm2); both multiply B group q
  int pair;
  const __nv_bfloat16* As2;
  const int* a_perm2;
  long long* ohi;        // exact partials (weights 0..3 / 4..6), entry ((s * groups + g) * N + j) * M + i
  long long* olo;
  int* status;
  int wmax;              // slice pairs kept: s + t <= wmax (<= OZ_W); the others weigh below 2^(-8 (wmax + 1))
  int epi;               // OZ_EPI_*: exact partials, or the joined float-float value written into out
  CBuf out;
  int64_t out_ld, out_gs, out_r0, out_c0;
};

// The float-float epilogue of a product with one k-split: C_ij = hi 2^(ea_i + eb_j - 38) +
// lo 2^(ea_i + eb_j - 62) (oz_join), written as OzGemm's epi mode says.
__device__ __forceinline__ void oz_epilogue_dd(const OzArgs& a, int g, int ag, int bg, int64_t i, int64_t j,
                                               long long hi, long long lo) {
  if (a.epi != OZ_EPI_STORE_NEG && i > j) return;  // symmetric results: the entries i <= j
  const dd v = oz_join(hi, lo, a.ea[(int64_t)ag * a.ea_gstride + i], a.eb[(int64_t)bg * a.eb_gstride + j]);
  const int64_t base = (int64_t)g * a.out_gs;
  if (a.epi == OZ_EPI_STORE_NEG) {
    DD::st(a.out, base + (a.out_r0 + i) * a.out_ld + a.out_c0 + j, dd_neg(v));
  } else {
    DD::st(a.out, base + j * a.out_ld + i, v);
    DD::st(a.out, base + i * a.out_ld + j, v);
  }
}

// Persistent: CTA b takes work items b, b + gridDim.x, ...; item = ((g * ksplit + sp) * MT + mt) * NTL + nt
// (column tiles fastest, so CTAs running at the same time share the A rows in L2).  The stage ring
// and the two Tensor Memory buffers run on counters that continue across items.
template <int NT>
__global__ void __launch_bounds__(OzCfg<NT>::THREADS, 1) k_oz_mma(OzArgs a) {
  using C = OzCfg<NT>;
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t full[C::STAGES], empty[C::STAGES], tfull[2], tempty[2], done;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int items = a.NTL * a.MT * a.groups * a.ksplit;

  struct Item {
    int nt, mt, g, sp, ag, bg, kb0, nkb;
    bool skip, a2;
  };
  auto decode = [&](int item) {
    Item w;
    w.nt = item % a.NTL;
    int r = item / a.NTL;
    w.mt = r % a.MT;
    r /= a.MT;
    w.sp = r % a.ksplit;
    w.g = r / a.ksplit;
    w.a2 = a.pair && (w.g & 1);
    w.bg = a.pair ? (w.g >> 1) : w.g;
    const int* pm = w.a2 ? a.a_perm2 : a.a_perm;
    w.ag = pm ? pm[w.bg] : w.bg;
    w.kb0 = w.sp * a.kbper;
    int kb1 = min(a.KB, w.kb0 + a.kbper);
    if (a.tri & OZ_TRI_GE_ROW) w.kb0 = max(w.kb0, (w.mt * 128) / OZ_BK);         // k >= the tile's first row
    if (a.tri & OZ_TRI_GE_COL) w.kb0 = max(w.kb0, (w.nt * NT) / OZ_BK);          // k >= its first column
    if (a.tri & OZ_TRI_LE_ROW) kb1 = min(kb1, (w.mt * 128 + 127) / OZ_BK + 1);   // k <= its last row
    w.skip = a.sym && w.mt * 128 > w.nt * NT + NT - 1;                          // entirely below the diagonal
    w.nkb = w.skip ? 0 : max(0, kb1 - w.kb0);
    return w;
  };

  if (warp == 1) tc::tmem_alloc(tc::smem_addr(&tmem_base), C::COLS);
  if (tid == 0) {
    for (int i = 0; i < C::STAGES; ++i) {
      tc::bar_init(tc::smem_addr(&full[i]), 1);
      tc::bar_init(tc::smem_addr(&empty[i]), 1);
    }
    for (int i = 0; i < 2; ++i) {
      tc::bar_init(tc::smem_addr(&tfull[i]), 1);
      tc::bar_init(tc::smem_addr(&tempty[i]), C::EPI_WARPS);
    }
    tc::bar_init(tc::smem_addr(&done), 1);
    abort_flag = 0;
    tc::bar_init_fence();
  }
  // the seventh B slice of every stage stays zero (the copies fill slices 0..5 only)
  if constexpr (!C::WIDE)
    for (int st = 0; st < C::STAGES; ++st)
      for (int x = tid; x < C::BBLK * 2 / 16; x += C::THREADS)
        reinterpret_cast<uint4*>(smem + st * C::STAGE + C::A_BYTES + C::B_BYTES)[x] = make_uint4(0, 0, 0, 0);
  tc::fence_proxy_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  // launched with programmatic serialization: everything above overlapped the predecessor
  pdl_wait();
  pdl_trigger();
  const uint32_t tmem = tmem_base;
  volatile int* abort_v = &abort_flag;

  if (warp == 0) {
    if (lane == 0) {  // producer
      // only the slices 0 .. wmax of either operand meet a kept pair: a prefix of each block
      const int nsl = min(a.wmax, OZ_S - 1) + 1;
      const uint32_t a_bytes = (uint32_t)nsl * OZ_ABLK * 2, b_bytes = (uint32_t)nsl * C::BBLK * 2;
      uint32_t q = 0;
      bool ok = true;
      for (int item = blockIdx.x; item < items && ok; item += gridDim.x) {
        const Item w = decode(item);
        const __nv_bfloat16* gA =
            (w.a2 ? a.As2 : a.As) + (int64_t)w.ag * a.a_gstride + ((int64_t)w.mt * a.KB + w.kb0) * (OZ_S * OZ_ABLK);
        const __nv_bfloat16* gB =
            a.Bs + (int64_t)w.bg * a.b_gstride + ((int64_t)w.nt * a.KB + w.kb0) * (OZ_S * C::BBLK);
        for (int it = 0; it < w.nkb; ++it, ++q) {
          const uint32_t st = q % C::STAGES, rnd = q / C::STAGES;
          if (rnd > 0 && !tc::bar_wait(tc::smem_addr(&empty[st]), (rnd - 1) & 1)) {
            dev_fail(a.status, DEV_TIMEOUT);
            *abort_v = 1;
          }
          if (*abort_v) {
            ok = false;
            break;
          }
          const uint32_t sa = tc::smem_addr(smem + st * C::STAGE), fb = tc::smem_addr(&full[st]);
          tc::bar_arrive_tx(fb, a_bytes + b_bytes);
          tc::bulk_load(sa, gA + (int64_t)it * (OZ_S * OZ_ABLK), a_bytes, fb);
          tc::bulk_load(sa + C::A_BYTES, gB + (int64_t)it * (OZ_S * C::BBLK), b_bytes, fb);
        }
      }
      // the copies of the last stages land before the CTA may leave
      for (uint32_t qq = q > (uint32_t)C::STAGES ? q - C::STAGES : 0; qq < q; ++qq)
        tc::bar_wait(tc::smem_addr(&full[qq % C::STAGES]), (qq / C::STAGES) & 1);
    }
  } else if (warp == 1) {
    if (lane == 0) {  // MMA issuer
      uint32_t q = 0, cc = 0;
      bool ok = true;
      for (int item = blockIdx.x; item < items && ok; item += gridDim.x) {
        const Item w = decode(item);
        const int nch = (w.nkb + OZ_CHUNK - 1) / OZ_CHUNK;
        for (int c = 0; c < nch && ok; ++c, ++cc) {
          const int h = cc & 1;
          if (cc >= 2 && !tc::bar_wait(tc::smem_addr(&tempty[h]), ((cc >> 1) - 1) & 1)) {
            dev_fail(a.status, DEV_TIMEOUT);
            *abort_v = 1;
            ok = false;
            break;
          }
          tc::fence_after_sync();
          const uint32_t dbase = tmem + (uint32_t)(h * (C::COLS / 2));
          const int i0 = c * OZ_CHUNK, i1 = min(w.nkb, i0 + OZ_CHUNK);
          for (int it = i0; it < i1; ++it, ++q) {
            const uint32_t st = q % C::STAGES, rnd = q / C::STAGES;
            if (!tc::bar_wait(tc::smem_addr(&full[st]), rnd & 1) || *abort_v) {
              dev_fail(a.status, DEV_TIMEOUT);
              *abort_v = 1;
              ok = false;
              break;
            }
            tc::fence_after_sync();
            const uint32_t sa = tc::smem_addr(smem + st * C::STAGE), sb = sa + C::A_BYTES;
            const uint64_t da0 = tc::smem_desc(sa, 128, 512), db0 = tc::smem_desc(sb, 128, 512);
            // One MMA per A slice s: a_s times the B slices b_0 .. b_{6-s} stacked as (7 - s) NT rows
            // (slice 6 is the zero slice), written from Tensor Memory column s NT on, so the block of
            // b_t lands in the accumulator of weight s + t.  The s = 0 MMA spans all seven weights and
            // opens a chunk by overwriting them.
#pragma unroll
            for (int ks = 0; ks < OZ_BK / 16; ++ks)
#pragma unroll
              for (int s = 0; s < OZ_S; ++s) {
                if (s > a.wmax) break;  // uniform
                const bool first = it == i0 && ks == 0 && s == 0;
                // descriptor start-address field: byte offset / 16 (no carry: shared addresses < 2^18)
                tc::mma_bf16(dbase + (uint32_t)(s * NT), da0 + (uint64_t)((s * (OZ_ABLK * 2) + ks * 256) >> 4),
                             db0 + (uint64_t)((ks * 256) >> 4), tc::idesc_bf16(128, (a.wmax + 1 - s) * NT),
                             first ? 0u : 1u);
              }
            tc::commit(tc::smem_addr(&empty[st]));
          }
          if (ok) tc::commit(tc::smem_addr(&tfull[h]));
        }
      }
      tc::commit(tc::smem_addr(&done));
      tc::bar_wait(tc::smem_addr(&done), 0);
    }
  } else {  // epilogue warps: warpgroup qg drains weights [w0, w0 + WPG) of columns [c0, c0 + EC)
    const int qg = (warp - 2) >> 2, lq = warp & 3;
    const int w0 = 0;
    const int c0 = qg * C::EC;
    const int r = lq * 32 + lane;  // Tensor Memory lane = row of the tile
    uint32_t cc = 0;
    for (int item = blockIdx.x; item < items; item += gridDim.x) {
      const Item w = decode(item);
      const int nch = (w.nkb + OZ_CHUNK - 1) / OZ_CHUNK;
      int acc[C::WPG * C::EC];
#pragma unroll
      for (int x = 0; x < C::WPG * C::EC; ++x) acc[x] = 0;
      for (int c = 0; c < nch; ++c, ++cc) {
        const int h = cc & 1;
        if (!tc::bar_wait(tc::smem_addr(&tfull[h]), (cc >> 1) & 1) || *abort_v) {
          if (lane == 0) dev_fail(a.status, DEV_TIMEOUT);
          *abort_v = 1;
          break;
        }
        tc::fence_after_sync();
#pragma unroll
        for (int wi = 0; wi < C::WPG; ++wi) {
          if (w0 + wi > a.wmax) continue;  // warp-uniform; weights above wmax stay zero
          const uint32_t ta =
              tmem + ((uint32_t)(lq * 32) << 16) + (uint32_t)(h * (C::COLS / 2) + (w0 + wi) * NT + c0);
          if constexpr (C::EC == 16) {
            uint32_t v[16];
            tc::tmem_ld16(ta, v);
            tc::tmem_ld_wait();
#pragma unroll
            for (int j = 0; j < 16; ++j) acc[wi * C::EC + j] += __float2int_rn(__uint_as_float(v[j]));
          } else {
            uint32_t v[32];
            tc::tmem_ld32(ta, v);
            tc::tmem_ld_wait();
#pragma unroll
            for (int j = 0; j < 32; ++j) acc[wi * C::EC + j] += __float2int_rn(__uint_as_float(v[j]));
          }
        }
        tc::fence_before_sync();
        __syncwarp();
        if (lane == 0) tc::bar_arrive(tc::smem_addr(&tempty[h]));
      }
      // every epilogue warp reaches this barrier; after it they agree on aborting
      tc::named_sync(1, 32 * C::EPI_WARPS);
      if (*abort_v) break;
      // The weights joined exactly in int64 (|acc_w| < 2^31):
      //   hi = acc_0 2^24 + acc_1 2^16 + acc_2 2^8 + acc_3,  lo = acc_4 2^16 + acc_5 2^8 + acc_6;
      // either written per k-split for the consumer to add and convert at full occupancy, or (one
      // k-split) converted here and written into the float-float result.
      const int64_t i = (int64_t)w.mt * 128 + r;
      constexpr int E = C::EC;
      if (i < a.M && !w.skip) {
#pragma unroll
        for (int j = 0; j < E; ++j) {
          const int64_t jj = (int64_t)w.nt * NT + c0 + j;
          if (jj >= a.N) break;
          const long long hi =
              (((long long)acc[j] * 256 + acc[E + j]) * 256 + acc[2 * E + j]) * 256 + acc[3 * E + j];
          long long lo = 0;
          if constexpr (C::WPG == OZ_NW) lo = ((long long)acc[4 * E + j] * 256 + acc[5 * E + j]) * 256 + acc[6 * E + j];
          if (a.epi == OZ_EPI_PARTIALS) {
            const int64_t o = (((int64_t)w.sp * a.groups + w.g) * a.N + jj) * a.M + i;
            a.ohi[o] = hi;
            if constexpr (!C::WIDE) a.olo[o] = lo;  // (weights 0..3 only: no lo partial, its consumer reads none)
          } else {
            oz_epilogue_dd(a, w.g, w.ag, w.bg, i, jj, hi, lo);
          }
        }
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 1) tc::tmem_dealloc(tmem, C::COLS);
}

// Block-wide maximum of a non-negative float (blockDim.x = 128).
__device__ __forceinline__ float block_max128(float v, float* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  return fmaxf(fmaxf(red[0], red[1]), fmaxf(red[2], red[3]));
}

// Exponent e with |x| < 2^e for the row / column maximum m (its high words: a
// normalised float-float value never exceeds the float below 2^e plus half its ulp).
__device__ __forceinline__ int oz_exp(float m) {
  if (!(m <= 3.402823466e38f)) return OZ_NONFINITE;  // Inf or NaN
  int e = 0;
  if (m > 0.f) frexpf(m, &e);
  return e;
}

// Nearest integer (ties to even) of a float of magnitude < 2^48 with 32-bit conversions only (64-bit
// float <-> integer conversions run on the FP64 pipe): r = rint(x) is integer-valued, and
// r = a 2^24 + b exactly with a = trunc(r 2^-24) (|a| < 2^24) and |b| < 2^24, both exact in FP32.
__device__ __forceinline__ long long round_to_ll(float x) {
  const float r = rintf(x);
  const float a = truncf(r * 5.9604644775390625e-8f);  // r 2^-24, exact
  const float b = fmaf(-a, 16777216.f, r);              // r - a 2^24, exact
  return ((long long)__float2int_rz(a) << 24) + (long long)__float2int_rz(b);
}

// v = hi + lo scaled by 2^(47 - e) to the nearest integer V (|V| <= 2^47, error <= 1 unit,
// i.e. 2^-47 of 2^e), then V = sum_t a_t 2^(8 (5 - t)) in balanced base-256 digits |a_t| <= 128.
__device__ __forceinline__ void store_digits(const float (&hi)[8], const float (&lo)[8], int e, bool live,
                                             __nv_bfloat16* dst, int64_t tstride) {
  long long V[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) V[q] = live ? round_to_ll(ldexpf(hi[q], 47 - e)) + round_to_ll(ldexpf(lo[q], 47 - e)) : 0ll;
  int dg[OZ_S][8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    long long x = V[q];
#pragma unroll
    for (int t = OZ_S - 1; t >= 1; --t) {
      int d = (int)(x & 255);
      d -= d > 128 ? 256 : 0;
      dg[t][q] = d;
      x = (x - d) >> 8;  // exact: x - d is a multiple of 256
    }
    dg[0][q] = (int)x;
  }
#pragma unroll
  for (int t = 0; t < OZ_S; ++t) {
    __align__(16) __nv_bfloat16 h[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) h[q] = __float2bfloat16_rn((float)dg[t][q]);  // |digit| <= 128: exact
    *reinterpret_cast<uint4*>(dst + t * tstride) = *reinterpret_cast<const uint4*>(h);
  }
}

// A operand: the rows of D x D row-major float-float matrices (group stride gs), one
// CTA of 128 threads per row.  Block (g, mt, kb, s) of `out` holds slice s of rows
// 128 mt .. +127, k = 32 kb .. +31; element (r, kk) at byte (r/8)*512 + (kk/8)*128 + (r%8)*16 + (kk%8)*2.
__global__ void __launch_bounds__(128) k_oz_slice_rows(CBuf X, int64_t D, int64_t gs, int MT, int KB,
                                                       __nv_bfloat16* out, int* ea) {
  pdl_wait();  // launched with programmatic serialization
  pdl_trigger();
  __shared__ float red[4];
  const int64_t i = blockIdx.x;
  const int g = blockIdx.y;
  const float* xh = (const float*)X.p0 + (int64_t)g * gs + i * D;
  const float* xl = (const float*)X.p1 + (int64_t)g * gs + i * D;
  float m = 0.f;
  if (i < D)
    for (int64_t k = threadIdx.x; k < D; k += 128) {
      const float a = fabsf(xh[k]);
      m = (a <= 3.402823466e38f) ? fmaxf(m, a) : __int_as_float(0x7f800000);  // Inf / NaN mark the row
    }
  m = block_max128(m, red);
  const int e = oz_exp(m);
  const bool live = i < D && e != OZ_NONFINITE;
  if (threadIdx.x == 0) ea[(int64_t)g * MT * 128 + i] = e;
  const int mt = (int)(i >> 7), r = (int)(i & 127);
  for (int c = threadIdx.x; c < KB * 4; c += 128) {
    const int kb = c >> 2, kc = c & 3;
    float h[8], l[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int64_t k = (int64_t)c * 8 + q;
      h[q] = (live && k < D) ? xh[k] : 0.f;
      l[q] = (live && k < D) ? xl[k] : 0.f;
    }
    store_digits(h, l, e, live, out + ((((int64_t)g * MT + mt) * KB + kb) * OZ_S) * OZ_ABLK +
                                   ((r >> 3) * 512 + kc * 128 + (r & 7) * 16) / 2, OZ_ABLK);
  }
}

// B operand: columns of column-major float-float panels (a column is contiguous over its D
// entries).  Column cl < ncolg of group g is source column cg = g * ncolg + cl, stored at
// (perm ? perm[cg / cpg] : cg / cpg) * gs + (cg % cpg) * D.  One CTA of 128 threads per
// column (padded to NTL * NT per group).  Block (g, nt, kb, t) holds NT columns x 32 k.
__global__ void __launch_bounds__(128) k_oz_slice_cols(CBuf X, int64_t D, int64_t ncolg, int NT, int NTL, int64_t cpg,
                                                       int64_t gs, const int* perm, int KB, __nv_bfloat16* out,
                                                       int* eb) {
  __shared__ float red[4];
  const int64_t c = blockIdx.x;
  const int64_t per = (int64_t)NTL * NT;
  const int g = (int)(c / per);
  const int64_t cl = c - g * per;
  const bool valid = cl < ncolg;
  int64_t base = 0;
  if (valid) {
    const int64_t cg = (int64_t)g * ncolg + cl;
    const int64_t grp = cg / cpg;
    base = (perm ? (int64_t)perm[grp] : grp) * gs + (cg - grp * cpg) * D;
  }
  const float* xh = (const float*)X.p0 + base;
  const float* xl = (const float*)X.p1 + base;
  float m = 0.f;
  if (valid)
    for (int64_t k = threadIdx.x; k < D; k += 128) {
      const float a = fabsf(xh[k]);
      m = (a <= 3.402823466e38f) ? fmaxf(m, a) : __int_as_float(0x7f800000);
    }
  m = block_max128(m, red);
  const int e = oz_exp(m);
  const bool live = valid && e != OZ_NONFINITE;
  if (threadIdx.x == 0) eb[c] = e;
  const int ntile = (int)(cl / NT), nl = (int)(cl - (int64_t)ntile * NT);
  const int64_t bblk = (int64_t)NT * OZ_BK;
  for (int ch = threadIdx.x; ch < KB * 4; ch += 128) {
    const int kb = ch >> 2, kc = ch & 3;
    float h[8], l[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int64_t k = (int64_t)ch * 8 + q;
      h[q] = (live && k < D) ? xh[k] : 0.f;
      l[q] = (live && k < D) ? xl[k] : 0.f;
    }
    store_digits(h, l, e, live, out + ((((int64_t)g * NTL + ntile) * KB + kb) * OZ_S) * bblk +
                                   ((nl >> 3) * 512 + kc * 128 + (nl & 7) * 16) / 2, bblk);
  }
}

// Vectors = the columns of row-major float-float matrices (group stride gs, row stride ld), K rows
// each: CTA (32 x 32 threads) per 32 columns; a column's maximum from its 32 threads, then thread
// (x, y) cuts rows 8c .. 8c+7 (c = y, y + 32, ...) of column x (loads coalesced across x).
// Layout as k_oz_slice_cols with tile height TH.
__global__ void __launch_bounds__(1024) k_oz_slice_matcols(CBuf X, int64_t ld, int64_t K, int64_t nvec, int64_t gs,
                                                          int TH, int NTL, int KB, __nv_bfloat16* out, int* e) {
  pdl_wait();  // launched with programmatic serialization
  pdl_trigger();
  __shared__ float red[32][33];
  __shared__ int ex[32];
  const int x = threadIdx.x, y = threadIdx.y, g = blockIdx.y, ny = blockDim.y;  // 32 columns x ny row lanes
  const int64_t v = (int64_t)blockIdx.x * 32 + x;
  const bool valid = v < nvec;
  const float* xh = (const float*)X.p0 + (int64_t)g * gs;
  const float* xl = (const float*)X.p1 + (int64_t)g * gs;
  float m = 0.f;
  if (valid)
    for (int64_t k = y; k < K; k += ny) {
      const float a = fabsf(xh[k * ld + v]);
      m = (a <= 3.402823466e38f) ? fmaxf(m, a) : __int_as_float(0x7f800000);
    }
  red[y][x] = m;
  __syncthreads();
  if (y == 0) {
    float mm = red[0][x];
    for (int q = 1; q < ny; ++q) mm = fmaxf(mm, red[q][x]);
    ex[x] = oz_exp(mm);
    if (v < (int64_t)NTL * TH) e[(int64_t)g * NTL * TH + v] = ex[x];
  }
  __syncthreads();
  if (v >= (int64_t)NTL * TH) return;
  const int ev = ex[x];
  const bool live = valid && ev != OZ_NONFINITE;
  const int tile = (int)(v / TH), nl = (int)(v - (int64_t)tile * TH);
  const int64_t bblk = (int64_t)TH * OZ_BK;
  for (int c = y; c < KB * 4; c += ny) {
    const int kb = c >> 2, kc = c & 3;
    float h[8], l[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int64_t k = (int64_t)c * 8 + q;
      h[q] = (live && k < K) ? xh[k * ld + v] : 0.f;
      l[q] = (live && k < K) ? xl[k * ld + v] : 0.f;
    }
    store_digits(h, l, ev, live, out + ((((int64_t)g * NTL + tile) * KB + kb) * OZ_S) * bblk +
                                    ((nl >> 3) * 512 + kc * 128 + (nl & 7) * 16) / 2, bblk);
  }
}

// Vectors with contiguous entries: vector v < nvec of group g starts at g * gs + off + v * vstride
// and has K entries.  One CTA of 128 threads per vector (padded to NTL * TH per group); layout as
// k_oz_slice_cols with tile height TH.
__global__ void __launch_bounds__(128) k_oz_slice_vecs(CBuf X, int64_t gs, int64_t off, int64_t vstride, int64_t K,
                                                       int64_t nvec, int TH, int NTL, int KB, __nv_bfloat16* out,
                                                       int* e) {
  pdl_wait();  // launched with programmatic serialization
  pdl_trigger();
  __shared__ float red[4];
  const int64_t v = blockIdx.x;
  const int g = blockIdx.y;
  const bool valid = v < nvec;
  const int64_t base = (int64_t)g * gs + off + (valid ? v : 0) * vstride;
  const float* xh = (const float*)X.p0 + base;
  const float* xl = (const float*)X.p1 + base;
  float m = 0.f;
  if (valid)
    for (int64_t k = threadIdx.x; k < K; k += 128) {
      const float a = fabsf(xh[k]);
      m = (a <= 3.402823466e38f) ? fmaxf(m, a) : __int_as_float(0x7f800000);
    }
  m = block_max128(m, red);
  const int ev = oz_exp(m);
  const bool live = valid && ev != OZ_NONFINITE;
  if (threadIdx.x == 0) e[(int64_t)g * NTL * TH + v] = ev;
  const int tile = (int)(v / TH), nl = (int)(v - (int64_t)tile * TH);
  const int64_t bblk = (int64_t)TH * OZ_BK;
  for (int c = threadIdx.x; c < KB * 4; c += 128) {
    const int kb = c >> 2, kc = c & 3;
    float h[8], l[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int64_t k = (int64_t)c * 8 + q;
      h[q] = (live && k < K) ? xh[k] : 0.f;
      l[q] = (live && k < K) ? xl[k] : 0.f;
    }
    store_digits(h, l, ev, live, out + ((((int64_t)g * NTL + tile) * KB + kb) * OZ_S) * bblk +
                                    ((nl >> 3) * 512 + kc * 128 + (nl & 7) * 16) / 2, bblk);
  }
}

// Rows of a row-major data matrix (element type ET, row stride ld), K entries each: the A operand of
// a product with the data.  FP32 / BF16 entries are their own high word (low word 0); an FP64 entry
// is split into its nearest float and the float of the remainder.  One CTA of 128 threads per row
// (padded to NTL * TH); layout as k_oz_slice_cols with tile height TH.
template <int ET>
__device__ __forceinline__ void data_hl(const void* X, int64_t i, float& h, float& l) {
  if (ET == ELEM_F64) {
    const double x = ((const double*)X)[i];
    h = (float)x;
    l = (float)(x - (double)h);
  } else if (ET == ELEM_F32) {
    h = ((const float*)X)[i];
    l = 0.f;
  } else {
    h = __uint_as_float((uint32_t)((const uint16_t*)X)[i] << 16);
    l = 0.f;
  }
}
template <int ET>
__global__ void __launch_bounds__(128) k_oz_slice_data_rows(const void* X, int64_t ld, int64_t K, int64_t nvec, int TH,
                                                            int NTL, int KB, __nv_bfloat16* out, int* e) {
  __shared__ float red[4];
  const int64_t v = blockIdx.x;
  const bool valid = v < nvec;
  const int64_t base = (valid ? v : 0) * ld;
  float m = 0.f;
  if (valid)
    for (int64_t k = threadIdx.x; k < K; k += 128) {
      float h, l;
      data_hl<ET>(X, base + k, h, l);
      const float a = fabsf(h);
      m = (a <= 3.402823466e38f) ? fmaxf(m, a) : __int_as_float(0x7f800000);
    }
  m = block_max128(m, red);
  const int ev = oz_exp(m);
  const bool live = valid && ev != OZ_NONFINITE;
  if (threadIdx.x == 0) e[v] = ev;
  const int tile = (int)(v / TH), nl = (int)(v - (int64_t)tile * TH);
  const int64_t bblk = (int64_t)TH * OZ_BK;
  for (int c = threadIdx.x; c < KB * 4; c += 128) {
    const int kb = c >> 2, kc = c & 3;
    float h[8], l[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int64_t k = (int64_t)c * 8 + q;
      h[q] = l[q] = 0.f;
      if (live && k < K) data_hl<ET>(X, base + k, h[q], l[q]);
    }
    store_digits(h, l, ev, live, out + (((int64_t)tile * KB + kb) * OZ_S) * bblk +
                                    ((nl >> 3) * 512 + kc * 128 + (nl & 7) * 16) / 2, bblk);
  }
}

// As k_oz_slice_vecs for short vectors (K <= 256: at most 32 chunks of 8 entries): one warp per
// vector, four vectors per CTA, the largest magnitude by a warp reduction.  Same digits and
// exponents as the one-CTA-per-vector kernel.
__global__ void __launch_bounds__(128) k_oz_slice_vecs_warp(CBuf X, int64_t gs, int64_t off, int64_t vstride,
                                                            int64_t K, int64_t nvec, int TH, int NTL, int KB,
                                                            __nv_bfloat16* out, int* e) {
  pdl_wait();  // launched with programmatic serialization
  pdl_trigger();
  const int lane = threadIdx.x & 31;
  const int64_t v = (int64_t)blockIdx.x * 4 + (threadIdx.x >> 5);
  const int g = blockIdx.y;
  if (v >= (int64_t)NTL * TH) return;  // whole warps only
  const bool valid = v < nvec;
  const int64_t base = (int64_t)g * gs + off + (valid ? v : 0) * vstride;
  const float* xh = (const float*)X.p0 + base;
  const float* xl = (const float*)X.p1 + base;
  const int c = lane;                  // this lane's chunk of 8 entries
  const bool has = c < KB * 4;
  float h[8], l[8];
  float m = 0.f;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int64_t k = (int64_t)c * 8 + q;
    const bool in = valid && has && k < K;
    h[q] = in ? xh[k] : 0.f;
    l[q] = in ? xl[k] : 0.f;
    const float a = fabsf(h[q]);
    m = (a <= 3.402823466e38f) ? fmaxf(m, a) : __int_as_float(0x7f800000);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  const int ev = oz_exp(m);
  const bool live = valid && ev != OZ_NONFINITE;
  if (lane == 0) e[(int64_t)g * NTL * TH + v] = ev;
  if (!has) return;
  const int tile = (int)(v / TH), nl = (int)(v - (int64_t)tile * TH);
  const int64_t bblk = (int64_t)TH * OZ_BK;
  const int kb = c >> 2, kc = c & 3;
  store_digits(h, l, ev, live, out + ((((int64_t)g * NTL + tile) * KB + kb) * OZ_S) * bblk +
                                  ((nl >> 3) * 512 + kc * 128 + (nl & 7) * 16) / 2, bblk);
}

// ---- The recursion's per-column kernels (right-hand sides, updates) with the next product's
// slicing fused.  A column of D rows is handled by a cluster of CL <= 8 CTAs: CTA r of the cluster
// owns the whole k-blocks [r KBC, (r + 1) KBC) of 32 rows (KBC = ceil(KB / CL)), one row per
// thread, so the loads of a row's split partials all go out together and a column spreads over
// CL SMs.  The column's largest magnitude (its slicing exponent) is reduced across the cluster
// through distributed shared memory; each CTA then cuts its own k-blocks.
constexpr int OZ_COL_THREADS_MAX = 512;

struct ColPart {
  int64_t c;       // column (cluster) index
  int64_t r0, r1;  // rows [r0, r1) of this CTA
  int rank, CL;
};

__device__ __forceinline__ ColPart col_part(int64_t D, int KBC) {
  cg::cluster_group cl = cg::this_cluster();
  ColPart p;
  p.rank = (int)cl.block_rank();
  p.CL = (int)cl.num_blocks();
  p.c = blockIdx.x / p.CL;
  p.r0 = (int64_t)p.rank * KBC * OZ_BK;
  p.r1 = min(D, p.r0 + (int64_t)KBC * OZ_BK);
  if (p.r1 < p.r0) p.r1 = p.r0;
  return p;
}

// Sum of n exact int64 split partials of up to two entries (offsets o1, o2; the second only when
// two is true): eight splits of every array per round, all loads of a round issued together.
// b == nullptr: the products wrote no lo partials (weights 0..3 only), which count as zero.
__device__ __forceinline__ void oz_sum_splits2(const long long* __restrict__ a, const long long* __restrict__ b, int n,
                                               int64_t stride, int64_t o1, int64_t o2, bool two, long long& s1a,
                                               long long& s1b, long long& s2a, long long& s2b) {
  s1a = s1b = s2a = s2b = 0;
  for (int s0 = 0; s0 < n; s0 += 8) {
    long long v1a[8], v1b[8], v2a[8], v2b[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const bool in = s0 + q < n;
      const int64_t so = (int64_t)(s0 + q) * stride;
      v1a[q] = in ? __ldg(a + so + o1) : 0LL;
      v1b[q] = (in && b) ? __ldg(b + so + o1) : 0LL;
      v2a[q] = (in && two) ? __ldg(a + so + o2) : 0LL;
      v2b[q] = (in && two && b) ? __ldg(b + so + o2) : 0LL;
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      s1a += v1a[q];
      s1b += v1b[q];
      s2a += v2a[q];
      s2b += v2b[q];
    }
  }
}

// Cut this CTA's k-blocks of column c (its rows held in hi / lo from offset 0) into the
// tile-height-NT layout (column c, tile c / NT) with the cluster-wide exponent, written to e[c].
__device__ void cluster_slice_column(const float* hi, const float* lo, const ColPart& p, int64_t D, int64_t c, int NT,
                                     int KB, int KBC, float* red, float* smax, __nv_bfloat16* out, int* e) {
  const int nrow = (int)(p.r1 - p.r0);
  float m = 0.f;
  for (int k = threadIdx.x; k < nrow; k += blockDim.x) {
    const float a = fabsf(hi[k]);
    m = (a <= 3.402823466e38f) ? fmaxf(m, a) : __int_as_float(0x7f800000);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    float b = red[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) b = fmaxf(b, red[w]);
    *smax = b;
  }
  cg::cluster_group cl = cg::this_cluster();
  cl.sync();
  float gm = 0.f;
  for (int r = 0; r < p.CL; ++r) gm = fmaxf(gm, *cl.map_shared_rank(smax, r));
  cl.sync();  // every CTA has read the others' maxima before any leaves
  const int ev = oz_exp(gm);
  const bool live = ev != OZ_NONFINITE;
  if (p.rank == 0 && threadIdx.x == 0) e[c] = ev;
  const int tile = (int)(c / NT), nl = (int)(c - (int64_t)tile * NT);
  const int64_t bblk = (int64_t)NT * OZ_BK;
  for (int ch = threadIdx.x; ch < KBC * 4; ch += blockDim.x) {
    const int kb = p.rank * KBC + (ch >> 2), kc = ch & 3;
    if (kb >= KB) continue;
    float h[8], l[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int k = ch * 8 + q;  // row p.r0 + k
      const bool in = live && p.r0 + k < D;
      h[q] = in ? hi[k] : 0.f;
      l[q] = in ? lo[k] : 0.f;
    }
    store_digits(h, l, ev, live, out + (((int64_t)tile * KB + kb) * OZ_S) * bblk +
                                   ((nl >> 3) * 512 + kc * 128 + (nl & 7) * 16) / 2, bblk);
  }
}

// The recursion's right-hand sides R (as k_make_R_oz) with their slicing fused: one cluster per
// column of R, padded to NTL x NT per live interval.  In the residual form U holds the partial
// sums v_j and Cr the right-hand side c: R is then minus the residual,
//   R_j = tau (G v_j + lam0 v_j) + lam0 v_{j-1} - [j = 0] c.
__global__ void __launch_bounds__(OZ_COL_THREADS_MAX, 2) k_make_R_oz_slice(const long long* Yhi, const long long* Ylo,
                                                            int ny, int64_t ny_stride, const int* eg, const int* eu,
                                                            CBuf U, int64_t nold, int64_t nnew, int64_t D, int64_t K,
                                                            int inew, const int* perm, const double* tau,
                                                            const double* lam0, int64_t gs, int NT, int NTL, int KB,
                                                            int KBC, __nv_bfloat16* Rs, int* er, CBuf Cr) {
  extern __shared__ float colbuf[];  // hi[KBC 32], lo[KBC 32]
  __shared__ float red[OZ_COL_THREADS_MAX / 32];
  __shared__ float smax;
  pdl_wait();
  pdl_trigger();
  const ColPart pt = col_part(D, KBC);
  float* bh = colbuf;
  float* bl = colbuf + KBC * OZ_BK;
  const int64_t per = (int64_t)NTL * NT;
  const int g = (int)(pt.c / per);
  const int64_t col = pt.c - g * per;
  const bool valid = col < nnew;
  if (valid) {
    const int l = perm[g];
    const int64_t j = col / K;
    const dd lm = dd_from_double(lam0[l]), tl = dd_from_double(tau[l]);
    for (int64_t k = pt.r0 + threadIdx.x; k < pt.r1; k += blockDim.x) {
      const int64_t o = (int64_t)l * gs + col * D + k;
      dd r;
      if (j == inew) {
        r = dd_mul(lm, DD::ld(U, o - K * D));
      } else {
        const int64_t cc = (int64_t)g * nold + col, yo = cc * D + k;
        long long h, w, h2, w2;
        oz_sum_splits2(Yhi, Ylo, ny, ny_stride, yo, yo, false, h, w, h2, w2);
        // ny = 0: no product (the residual form's first step, v = 0): R = -c
        const dd y = ny > 0 ? oz_join(h, w, eg[k], eu[cc]) : DD::zero();
        r = dd_mul(tl, dd_add(y, dd_mul(lm, DD::ld(U, o))));
        if (j > 0) r = dd_add(r, dd_mul(lm, DD::ld(U, o - K * D)));
        else if (Cr.p0) r = dd_sub(r, DD::ld(Cr, col * D + k));  // residual form: minus c in the j = 0 term
      }
      bh[k - pt.r0] = r.hi;
      bl[k - pt.r0] = r.lo;
    }
  } else {
    for (int64_t k = pt.r0 + threadIdx.x; k < pt.r1; k += blockDim.x) bh[k - pt.r0] = bl[k - pt.r0] = 0.f;
  }
  __syncthreads();
  // group g's tiles start at tile g * NTL
  cluster_slice_column(bh, bl, pt, D, (int64_t)g * per + col, NT, KB, KBC, red, &smax, Rs, er);
}

// The update of the recursion (as k_update_oz) with the next step's slicing of the new columns
// fused: one cluster per new column (g, col); for an interval still live at the next step, the
// new u is cut into the next step's concatenated-column layout (column g * ncol + col, tile NTn).
// Residual form (resid != 0): Ut holds the partial sums v, updated in place, and v is cut.
__global__ void __launch_bounds__(OZ_COL_THREADS_MAX, 2) k_update_oz_slice(const long long* Zhi, const long long* Zlo,
                                                            int S, const int* ep, int64_t ep_gs, const int* er,
                                                            int64_t er_gs, int live, int64_t ncol, int64_t D, int64_t K,
                                                            int i, CBuf Uin, CBuf Uout, CBuf Ut, const int* perm,
                                                            int64_t gs, int live_next, int NTn, int KB, int KBC,
                                                            __nv_bfloat16* Us, int* eu, int resid) {
  extern __shared__ float colbuf[];
  __shared__ float red[OZ_COL_THREADS_MAX / 32];
  __shared__ float smax;
  pdl_wait();
  pdl_trigger();
  const ColPart pt = col_part(D, KBC);
  float* bh = colbuf;
  float* bl = colbuf + KBC * OZ_BK;
  const int g = (int)(pt.c / ncol);
  const int64_t col = pt.c - (int64_t)g * ncol;
  const int l = perm[g];
  const int64_t j = col / K, ss = (int64_t)live * ncol * D;
  const int ec = er[(int64_t)g * er_gs + col];
  for (int64_t row = pt.r0 + threadIdx.x; row < pt.r1; row += blockDim.x) {
    const int64_t zo = ((int64_t)g * ncol + col) * D + row;
    long long h, w, h2, w2;
    oz_sum_splits2(Zhi, Zlo, S, ss, zo, zo, false, h, w, h2, w2);
    const dd z = oz_join(h, w, ep[(int64_t)l * ep_gs + row], ec);
    const int64_t o = (int64_t)l * gs + col * D + row;
    dd u;
    if (resid) {  // v_j <- v_j - P_l R_j, in place (a new term's v is still zero)
      u = dd_sub(DD::ld(Ut, o), z);
      DD::st(Ut, o, u);
    } else {
      u = dd_sub((j < i) ? DD::ld(Uin, o) : DD::zero(), z);
      DD::st(Uout, o, u);
      DD::st(Ut, o, dd_add(DD::ld(Ut, o), u));
    }
    bh[row - pt.r0] = u.hi;
    bl[row - pt.r0] = u.lo;
  }
  if (g >= live_next) return;  // uniform over the cluster
  __syncthreads();
  cluster_slice_column(bh, bl, pt, D, (int64_t)g * ncol + col, NTn, KB, KBC, red, &smax, Us, eu);
}

// The recursion in the two-product form (intervals with M_q = P_l (G + lam0_l I) formed):
//   u_{i+1,j} = u_{i,j} - tau_l M_q u_{i,j} - lam0_l P_l u_{i,j-1}   (no second term for j = 0),
// the same polynomial as R = tau (G u_j + lam0 u_j) + lam0 u_{j-1}, u_j <- u_j - P_l R, with
// both products taken over the step's old columns in one launch (pair mode: group 2q holds
// M_q U_q, group 2q + 1 holds P_l U_q).  One cluster per column (q, col) of the ncol columns of
// each live interval (every column exists: the basis is truncated to ncol = jmax K columns);
// the new column is cut into the next step's slices (tile height 16, column q ncol + col).
__global__ void __launch_bounds__(OZ_COL_THREADS_MAX) k_update_mw_slice(const long long* Phi, const long long* Plo,
                                                            int S, const int* em, const int* ep, int64_t e_gs, int live,
                                                            int64_t ncol, int64_t D, int64_t K, CBuf Uin, CBuf Uout,
                                                            CBuf Ut, const int* perm, const double* tau,
                                                            const double* lam0, int64_t gs, const int* eu_in,
                                                            int live_next, int KB, int KBC, __nv_bfloat16* Us,
                                                            int* eu) {
  extern __shared__ float colbuf[];
  __shared__ float red[OZ_COL_THREADS_MAX / 32];
  __shared__ float smax;
  pdl_wait();
  pdl_trigger();
  const ColPart pt = col_part(D, KBC);
  float* bh = colbuf;
  float* bl = colbuf + KBC * OZ_BK;
  const int q = (int)(pt.c / ncol);
  const int64_t col = pt.c - (int64_t)q * ncol;
  const int l = perm[q];
  const bool has_w = col >= K;  // j >= 1
  const int64_t ss = 2 * (int64_t)live * ncol * D;                  // stride of the k-splits
  const int64_t zo = ((int64_t)(2 * q) * ncol + col) * D;            // M_q u_j
  const int64_t wo = ((int64_t)(2 * q + 1) * ncol + col - K) * D;    // P_l u_{j-1}
  const int ez = eu_in[(int64_t)q * ncol + col];
  const int ew = has_w ? eu_in[(int64_t)q * ncol + col - K] : 0;
  const dd tl = dd_from_double(tau[l]), lm = dd_from_double(lam0[l]);
  for (int64_t row = pt.r0 + threadIdx.x; row < pt.r1; row += blockDim.x) {
    long long zh, zl, wh, wl;
    oz_sum_splits2(Phi, Plo, S, ss, zo + row, wo + row, has_w, zh, zl, wh, wl);
    dd t = dd_mul(tl, oz_join(zh, zl, em[(int64_t)q * e_gs + row], ez));
    if (has_w) t = dd_add(t, dd_mul(lm, oz_join(wh, wl, ep[(int64_t)l * e_gs + row], ew)));
    const int64_t o = (int64_t)l * gs + col * D + row;
    const dd u = dd_sub(DD::ld(Uin, o), t);
    DD::st(Uout, o, u);
    DD::st(Ut, o, dd_add(DD::ld(Ut, o), u));
    bh[row - pt.r0] = u.hi;
    bl[row - pt.r0] = u.lo;
  }
  if (q >= live_next) return;  // uniform over the cluster
  __syncthreads();
  cluster_slice_column(bh, bl, pt, D, (int64_t)q * ncol + col, 16, KB, KBC, red, &smax, Us, eu);
}

// M_q = P_l (G + lam0_l I), l = perm[q], from the exact partials of G P_l (A = the rows of G,
// B = the columns of P_l; P_l and G are symmetric, so entry (i, j) of G P_l is entry (j, i) of
// P_l G): M_q[j][i] = (G P_l)[i][j] + lam0_l P_l[j][i], row-major, float-float.
__global__ void k_oz_make_M(const long long* hi, const long long* lo, int S, int64_t D, int T, const int* eg,
                            const int* epc, int64_t epc_gs, const int* perm, const double* lam0, CBuf P, CBuf M) {
  pdl_wait();  // launched with programmatic serialization
  pdl_trigger();
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)T * D * D) return;
  const int64_t q = e / (D * D), r = e - q * D * D, j = r / D, i = r - j * D;
  long long h = 0, w = 0;
  for (int s = 0; s < S; ++s) {
    h += hi[(int64_t)s * T * D * D + e];
    w += lo[(int64_t)s * T * D * D + e];
  }
  const int l = perm[q];
  const dd v = oz_join(h, w, eg[i], epc[q * epc_gs + j]);
  DD::st(M, e, dd_add(v, dd_mul(dd_from_double(lam0[l]), DD::ld(P, (int64_t)l * D * D + r))));
}

inline int oz_kb(int64_t D) { return (int)((D + OZ_BK - 1) / OZ_BK); }
inline int oz_mt(int64_t D) { return (int)((D + 127) / 128); }

int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      n = 148;
  }
  return n;
}

template <int NT>
cudaError_t launch_oz(const OzArgs& a, cudaStream_t st) {
  using C = OzCfg<NT>;
  CK(cudaFuncSetAttribute(k_oz_mma<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM));
  const int64_t items = (int64_t)a.NTL * a.MT * a.groups * a.ksplit;
  const unsigned grid = (unsigned)std::min<int64_t>(items, sm_count());  // one CTA per SM (shared memory)
  return launch_pdl(k_oz_mma<NT>, dim3(grid), dim3(C::THREADS), C::SMEM, st, a);
}

}  // namespace

// ---------------------------------------------------------------- host interface
int oz_tile_n(int64_t ncolg, int wmax) { return ncolg <= 16 ? 16 : (ncolg <= 32 || wmax > OzCfg<64>::WMAX) ? 32 : 64; }

size_t oz_rows_elems(int64_t D) { return (size_t)oz_mt(D) * oz_kb(D) * OZ_S * OZ_ABLK; }
size_t oz_rows_exps(int64_t D) { return (size_t)oz_mt(D) * 128; }
size_t oz_cols_elems(int64_t D, int64_t ncolg, int NT) {
  return (size_t)((ncolg + NT - 1) / NT) * oz_kb(D) * OZ_S * NT * OZ_BK;
}
size_t oz_cols_exps(int64_t ncolg, int NT) { return (size_t)((ncolg + NT - 1) / NT) * NT; }

cudaError_t oz_slice_rows(CBuf X, int64_t D, int groups, int64_t gs, __nv_bfloat16* out, int* ea, cudaStream_t st) {
  dim3 grid((unsigned)(oz_mt(D) * 128), (unsigned)groups);
  return launch_pdl(k_oz_slice_rows, grid, dim3(128), 0, st, X, D, gs, oz_mt(D), oz_kb(D), out, ea);
}

cudaError_t oz_slice_cols(CBuf X, int64_t D, int ngroups, int64_t ncolg, int NT, int64_t cpg, int64_t gs,
                          const int* perm, __nv_bfloat16* out, int* eb, cudaStream_t st) {
  const int NTL = (int)((ncolg + NT - 1) / NT);
  const int64_t cols = (int64_t)ngroups * NTL * NT;
  k_oz_slice_cols<<<(unsigned)cols, 128, 0, st>>>(X, D, ncolg, NT, NTL, cpg, gs, perm, oz_kb(D), out, eb);
  return cudaGetLastError();
}

int oz_pick_split(int64_t D, int64_t ncolg, int groups, int NT, int cap) {
  const int KB = oz_kb(D);
  const int64_t ctas = (int64_t)oz_mt(D) * ((ncolg + NT - 1) / NT) * groups;
  int s = (int)std::max<int64_t>(1, (sm_count() + ctas - 1) / ctas);  // about one work item per SM
  s = std::min(s, std::max(1, KB / OZ_CHUNK));            // at least one drain chunk per split
  s = std::max(s, (KB + OZ_KB_MAX - 1) / OZ_KB_MAX);     // int32 bound per CTA
  s = std::min(s, cap);
  const int kbper = (KB + s - 1) / s;
  return (KB + kbper - 1) / kbper;                        // every split non-empty
}

cudaError_t oz_gemm(const OzGemm& q, cudaStream_t st) {
  OzArgs a{};
  const int KB = (int)((q.K + OZ_BK - 1) / OZ_BK), MT = (int)((q.M + 127) / 128);
  const int NTL = (int)((q.N + q.NT - 1) / q.NT);
  if (q.NT != 16 && q.NT != 32 && !(q.NT == 64 && q.wmax <= OzCfg<64>::WMAX)) return cudaErrorInvalidValue;
  a.As = q.As;
  a.a_gstride = q.a_shared ? 0 : (int64_t)oz_vec_elems(q.M, q.K, 128);
  a.a_perm = q.a_perm;
  a.ea = q.ea;
  a.ea_gstride = q.a_shared ? 0 : (int64_t)oz_vec_exps(q.M, 128);
  a.Bs = q.Bs;
  a.b_gstride = q.b_shared ? 0 : (int64_t)oz_vec_elems(q.N, q.K, q.NT);
  a.eb = q.eb;
  a.eb_gstride = (int64_t)oz_vec_exps(q.N, q.NT);
  a.KB = KB;
  a.MT = MT;
  a.NTL = NTL;
  a.M = q.M;
  a.N = q.N;
  a.groups = q.groups;
  a.kbper = (KB + q.ksplit - 1) / q.ksplit;
  a.ksplit = (KB + a.kbper - 1) / a.kbper;
  if (a.ksplit != q.ksplit || a.kbper > OZ_KB_MAX) return cudaErrorInvalidValue;
  a.tri = q.tri;
  a.sym = q.sym;
  a.pair = q.pair;
  a.As2 = q.As2;
  a.a_perm2 = q.a_perm2;
  if (q.pair && (q.groups & 1)) return cudaErrorInvalidValue;
  a.ohi = q.ohi;
  a.olo = q.olo;
  a.status = q.status;
  if (q.wmax < 1 || q.wmax > OZ_W) return cudaErrorInvalidValue;
  a.wmax = q.wmax;
  if (q.epi != OZ_EPI_PARTIALS && (a.ksplit != 1 || q.pair || !q.ea || !q.eb || !q.out.p0)) return cudaErrorInvalidValue;
  a.epi = q.epi;
  a.out = q.out;
  a.out_ld = q.out_ld;
  a.out_gs = q.out_gs;
  a.out_r0 = q.out_r0;
  a.out_c0 = q.out_c0;
  return q.NT == 16 ? launch_oz<16>(a, st) : q.NT == 32 ? launch_oz<32>(a, st) : launch_oz<64>(a, st);
}

cudaError_t oz_product(const __nv_bfloat16* As, const int* ea, const int* a_perm, bool a_shared,
                       const __nv_bfloat16* Bs, const int* eb, int64_t D, int64_t ncolg, int groups, int NT,
                       int ksplit, long long* ohi, long long* olo, int* status, cudaStream_t st, int wmax) {
  OzGemm q;
  q.wmax = wmax;
  q.As = As; q.ea = ea; q.a_perm = a_perm; q.a_shared = a_shared;
  q.Bs = Bs; q.eb = eb;
  q.M = D; q.N = ncolg; q.K = D; q.groups = groups; q.NT = NT; q.ksplit = ksplit;
  q.ohi = ohi; q.olo = olo; q.status = status;
  return oz_gemm(q, st);
}

cudaError_t oz_slice_vecs(CBuf X, int64_t gs, int64_t off, int64_t vstride, int64_t K, int64_t nvec, int groups,
                          int TH, __nv_bfloat16* out, int* e, cudaStream_t st) {
  const int NTL = (int)((nvec + TH - 1) / TH);
  const int KB = (int)((K + OZ_BK - 1) / OZ_BK);
  if (KB * 4 <= 32) {
    dim3 grid((unsigned)((NTL * TH + 3) / 4), (unsigned)groups);
    return launch_pdl(k_oz_slice_vecs_warp, grid, dim3(128), 0, st, X, gs, off, vstride, K, nvec, TH, NTL, KB, out, e);
  }
  dim3 grid((unsigned)(NTL * TH), (unsigned)groups);
  return launch_pdl(k_oz_slice_vecs, grid, dim3(128), 0, st, X, gs, off, vstride, K, nvec, TH, NTL, KB, out, e);
}

int oz_pick_split_mnk(int64_t M, int64_t N, int64_t K, int groups, int NT, int cap) {
  const int KB = (int)((K + OZ_BK - 1) / OZ_BK);
  const int64_t ctas = ((M + 127) / 128) * ((N + NT - 1) / NT) * groups;
  int s = (int)std::max<int64_t>(1, (sm_count() + ctas - 1) / ctas);
  s = std::min(s, std::max(1, KB / OZ_CHUNK));
  s = std::max(s, (KB + OZ_KB_MAX - 1) / OZ_KB_MAX);
  s = std::min(s, cap);
  const int kbper = (KB + s - 1) / s;
  return (KB + kbper - 1) / kbper;
}

bool oz_fused_ok(int64_t D) { return (size_t)D * 8 <= 160 * 1024; }

// Cluster geometry of the per-column kernels: CL <= 8 CTAs per column, KBC k-blocks of 32 rows
// per CTA, one row per thread (up to 512 threads), the CTA's rows in shared memory.
struct ColGeom {
  int KB, CL, KBC, threads;
  size_t smem;
};
inline ColGeom col_geom(int64_t D, int CL) {
  ColGeom g;
  g.KB = oz_kb(D);
  g.CL = std::min(CL, std::max(1, g.KB));
  g.KBC = (g.KB + g.CL - 1) / g.CL;
  g.threads = std::min(g.KBC * OZ_BK, OZ_COL_THREADS_MAX);
  g.smem = (size_t)g.KBC * OZ_BK * 2 * sizeof(float);
  return g;
}

// Cluster sizes the autotuner tries for a per-column launch (every one gives the same values):
// 8, 4, 2, 1 CTAs per column, as far as the column has k-blocks.
inline int col_cands(int64_t D, int* c) {
  const int KB = oz_kb(D);
  int n = 0;
  for (int cl = 8; cl >= 1; cl /= 2)
    if (cl <= KB || cl == 1) c[n++] = cl;
  return n;
}

cudaError_t oz_make_R_slice(const long long* Yhi, const long long* Ylo, int ny, int64_t ny_stride, const int* eg,
                            const int* eu, CBuf U, int live, int64_t nold, int64_t nnew, int64_t D, int64_t K, int inew,
                            const int* perm, const double* tau, const double* lam0, int64_t gs, int NT,
                            __nv_bfloat16* Rs, int* er, CBuf c, cudaStream_t st) {
  const int NTL = (int)((nnew + NT - 1) / NT);
  int cands[4];
  const int nc = col_cands(D, cands);
  TuneLaunch t = tune_begin(tune_key(TUNE_COL_R, D, shape_class((int64_t)live * NTL * NT), 0), "col_R_cluster",
                            cands, nc, st);
  const ColGeom cg_ = col_geom(D, t.value);
  if (cg_.smem > 48 * 1024)
    CK(cudaFuncSetAttribute(k_make_R_oz_slice, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cg_.smem));
  const cudaError_t e =
      launch_pdl_cluster(k_make_R_oz_slice, dim3((unsigned)((int64_t)live * NTL * NT * cg_.CL)), dim3(cg_.threads),
                         cg_.smem, cg_.CL, st, Yhi, Ylo, ny, ny_stride, eg, eu, U, nold, nnew, D, K, inew, perm, tau,
                         lam0, gs, NT, NTL, cg_.KB, cg_.KBC, Rs, er, c);
  tune_end(t, st);
  return e;
}

cudaError_t oz_update_slice(const long long* Zhi, const long long* Zlo, int S, const int* ep, int64_t ep_gs,
                            const int* er, int64_t er_gs, int live, int64_t ncol, int64_t D, int64_t K, int i, CBuf Uin,
                            CBuf Uout, CBuf Ut, const int* perm, int64_t gs, int live_next, int NTn, __nv_bfloat16* Us,
                            int* eu, int resid, cudaStream_t st) {
  int cands[4];
  const int nc = col_cands(D, cands);
  TuneLaunch t = tune_begin(tune_key(TUNE_COL_UPDATE, D, shape_class((int64_t)live * ncol), 0), "col_update_cluster",
                            cands, nc, st);
  const ColGeom cg_ = col_geom(D, t.value);
  if (cg_.smem > 48 * 1024)
    CK(cudaFuncSetAttribute(k_update_oz_slice, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cg_.smem));
  const cudaError_t e =
      launch_pdl_cluster(k_update_oz_slice, dim3((unsigned)((int64_t)live * ncol * cg_.CL)), dim3(cg_.threads),
                         cg_.smem, cg_.CL, st, Zhi, Zlo, S, ep, ep_gs, er, er_gs, live, ncol, D, K, i, Uin, Uout, Ut,
                         perm, gs, live_next, NTn, cg_.KB, cg_.KBC, Us, eu, resid);
  tune_end(t, st);
  return e;
}

cudaError_t oz_update_mw_slice(const long long* Phi, const long long* Plo, int S, const int* em, const int* ep,
                               int live, int64_t ncol, int64_t D, int64_t K, CBuf Uin, CBuf Uout, CBuf Ut,
                               const int* perm, const double* tau, const double* lam0, int64_t gs, const int* eu_in,
                               int live_next, __nv_bfloat16* Us, int* eu, cudaStream_t st) {
  int cands[4];
  const int nc = col_cands(D, cands);
  TuneLaunch t = tune_begin(tune_key(TUNE_COL_MW, D, shape_class((int64_t)live * ncol), 0), "col_mw_cluster", cands,
                            nc, st);
  const ColGeom cg_ = col_geom(D, t.value);
  if (cg_.smem > 48 * 1024)
    CK(cudaFuncSetAttribute(k_update_mw_slice, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cg_.smem));
  const cudaError_t e =
      launch_pdl_cluster(k_update_mw_slice, dim3((unsigned)((int64_t)live * ncol * cg_.CL)), dim3(cg_.threads),
                         cg_.smem, cg_.CL, st, Phi, Plo, S, em, ep, (int64_t)oz_rows_exps(D), live, ncol, D, K, Uin,
                         Uout, Ut, perm, tau, lam0, gs, eu_in, live_next, cg_.KB, cg_.KBC, Us, eu);
  tune_end(t, st);
  return e;
}

cudaError_t oz_make_M(const long long* hi, const long long* lo, int S, int64_t D, int T, const int* eg, const int* epc,
                      int64_t epc_gs, const int* perm, const double* lam0, CBuf P, CBuf M, cudaStream_t st) {
  const int64_t n = (int64_t)T * D * D;
  return launch_pdl(k_oz_make_M, dim3((unsigned)((n + 255) / 256)), dim3(256), 0, st, hi, lo, S, D, T, eg, epc, epc_gs,
                    perm, lam0, P, M);
}

cudaError_t oz_slice_data_rows(const void* X, int elem, int64_t ld, int64_t K, int64_t nvec, int TH,
                               __nv_bfloat16* out, int* e, cudaStream_t st) {
  const int NTL = (int)((nvec + TH - 1) / TH);
  const unsigned grid = (unsigned)(NTL * TH);
  const int KB = (int)((K + OZ_BK - 1) / OZ_BK);
  if (elem == ELEM_F64) k_oz_slice_data_rows<ELEM_F64><<<grid, 128, 0, st>>>(X, ld, K, nvec, TH, NTL, KB, out, e);
  else if (elem == ELEM_F32) k_oz_slice_data_rows<ELEM_F32><<<grid, 128, 0, st>>>(X, ld, K, nvec, TH, NTL, KB, out, e);
  else k_oz_slice_data_rows<ELEM_BF16><<<grid, 128, 0, st>>>(X, ld, K, nvec, TH, NTL, KB, out, e);
  return cudaGetLastError();
}

size_t oz_vec_elems(int64_t nvec, int64_t K, int TH) {
  return (size_t)((nvec + TH - 1) / TH) * ((K + OZ_BK - 1) / OZ_BK) * OZ_S * TH * OZ_BK;
}
size_t oz_vec_exps(int64_t nvec, int TH) { return (size_t)((nvec + TH - 1) / TH) * TH; }

cudaError_t oz_slice_matcols(CBuf X, int64_t ld, int64_t K, int64_t nvec, int groups, int64_t gs, int TH,
                             __nv_bfloat16* out, int* e, cudaStream_t st) {
  const int NTL = (int)((nvec + TH - 1) / TH);
  dim3 grid((unsigned)((NTL * TH + 31) / 32), (unsigned)groups), blk(32, 32);
  return launch_pdl(k_oz_slice_matcols, grid, blk, 0, st, X, ld, K, nvec, gs, TH, NTL, (int)((K + OZ_BK - 1) / OZ_BK), out,
                    e);
}

uint64_t loop_slices_bytes(int64_t D, int L, int64_t ncol_max) {
  const uint64_t bcols = (uint64_t)L * (uint64_t)(ncol_max + 32);  // one step's columns, padded per group
  return (uint64_t)(L + 1) * (oz_rows_elems(D) * 2 + oz_rows_exps(D) * 4) +
         bcols * (uint64_t)oz_kb(D) * OZ_S * OZ_BK * 2 + bcols * 4;
}

double oz_pair_flops(int64_t M, int64_t N, int64_t K, int wmax) {
  int pairs = 0;
  for (int s = 0; s < OZ_S; ++s)
    for (int t = 0; t < OZ_S; ++t) pairs += s + t <= wmax;
  return 2.0 * pairs * (double)M * (double)N * (double)K;
}

}  // namespace ihsbin
