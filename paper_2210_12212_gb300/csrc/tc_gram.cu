// Step a3 (the Gram G = A_hat^T A_hat of the Gram product mode) for dense FP32 /
// BF16 data on the 5th-generation tensor cores, with an exactly rounded-once
// FP64 result.
//
// Method (error-free splitting of the data, as in Ozaki-style exact products):
//  * each column j is scaled by the power of two 2^(7 - e_j), e_j the exponent of
//    its largest magnitude, so that every scaled entry v satisfies |v| < 2^7;
//  * v is cut into `ns` integer slices a_0 + a_1 2^-8 + a_2 2^-16 + ...,
//    |a_t| <= 128, every one exact in BF16 (8 significant bits);
//  * G_ij = 2^(e_i + e_j - 14) sum_{s,t} 2^(-8(s+t)) sum_k a_s(k,i) a_t(k,j).
//    Every product a_s a_t is an integer of magnitude <= 2^14, so a tensor-core
//    sum of 512 of them (|sum| <= 2^23) is exact in its FP32 accumulator; each
//    such chunk is drained from Tensor Memory into int32 registers, and a work
//    item covers at most 65536 rows (|int32 sum| <= 2^30);
//  * a combine pass adds the integer tiles of all slice pairs in FP64 from the
//    smallest weight up and applies the power-of-two scales.
// For FP32 data six slices represent every entry within a factor 2^-17 of its
// column's maximum exactly (smaller entries to 2^-41 of that maximum), and
// pairs with s + t <= 6 are kept (the rest weigh below 2^-56 of the leading
// term), so the result agrees with the exact Gram to about FP64 rounding.
// Symmetry: the pair (s, t), s < t, is computed for all tile pairs (I, J) and
// enters G_IJ and G_JI; the pair (s, s) only for I <= J.
//
// Tensor-core kernel (one CTA per 128 x 128 output tile, pair and row range):
//  * slices are written by the slicing kernel directly in the shared-memory
//    image the MMA reads (K-major 8 x 16-byte core matrices, 128 rows x 64 k
//    per 16 KiB block), so one pipeline stage is two 16 KiB bulk copies;
//  * warp 0 (one lane) issues the bulk copies into a 6-stage ring; warp 1
//    owns the Tensor Memory (256 columns: two 128-column FP32 accumulators)
//    and one lane issues tcgen05.mma (M = N = 128, K = 16; 4 per stage);
//  * warps 2..5 drain a finished accumulator (tcgen05.ld) into int32 while the
//    MMAs of the next chunk run into the other one;
//  * every wait is bounded in time: a pipeline that cannot progress records
//    DEV_TIMEOUT in the status word, lets its copies and MMAs land, frees its
//    Tensor Memory and returns.
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "tc.cuh"

namespace ihsbin {
namespace {

#define CK(x)                              \
  do {                                     \
    cudaError_t e__ = (x);                 \
    if (e__ != cudaSuccess) return e__;    \
  } while (0)

constexpr int SL_BLOCK_ELEMS = 8192;     // 128 rows x 64 k (BF16)
constexpr int SL_CHUNK = 8;              // K-blocks per exact Tensor Memory chunk (512 k)
constexpr int SL_KB_MAX = 1024;          // K-blocks per work item (65536 k)
constexpr int SL_MAX_PAIRS = 36;
constexpr int SL_NONFINITE = 1 << 20;    // column exponent marking a column holding Inf/NaN

struct SlicePlan {
  int ns, np, T, RB, KB, nsplit, kbper, D;  // RB: 128-column blocks per slice of the A-side buffer (its stride)
  int rect;   // 1: C = X^T Y of two sliced operands (all tiles of every pair); 0: the symmetric Gram X^T X
  int nw;     // 128-column blocks per result tile (1 or 2)
  int TJ;     // result column tiles (each nw blocks wide)
  int RBb;    // 128-column blocks per slice of the B-side buffer (TJ nw: padded with zero blocks)
  int8_t ps[SL_MAX_PAIRS], pt[SL_MAX_PAIRS];
  int base[SL_MAX_PAIRS + 1];  // first tile of each pair; base[np] = tiles of all pairs (items = tiles x nsplit)
};

// sum over I' < I of floor(I' / nw): the tiles a symmetric pair skips before row tile I
__host__ __device__ __forceinline__ int diag_skip(int I, int nw) {
  if (nw == 1) return I * (I - 1) / 2;
  const int a = I / 2;
  return a * (a - 1) + (I & 1) * a;
}
// index of result tile (I, Jw) (Jw in nw-wide column tiles) within its pair
__host__ __device__ __forceinline__ int tile_index(bool diag_pair, int TJ, int nw, int I, int Jw) {
  return diag_pair ? I * TJ - diag_skip(I, nw) + (Jw - I / nw) : I * TJ + Jw;
}

__device__ __forceinline__ int col_exp(unsigned mbits) {
  if (mbits >= 0x7f800000u) return SL_NONFINITE;
  if (mbits == 0u) return 0;
  int e;
  frexpf(__uint_as_float(mbits), &e);  // max |a| = f 2^e with f in [0.5, 1)
  return e;
}

template <int ET>
__device__ __forceinline__ float load_f(const void* X, int64_t i) {
  if (ET == ELEM_F32) return ((const float*)X)[i];
  return __uint_as_float((uint32_t)((const uint16_t*)X)[i] << 16);
}

// cmax[j] = bits of max_k |A[k][j]| (Inf bits when the column holds Inf or NaN)
template <int ET>
__global__ void k_col_absmax(const void* A, int64_t ld, int64_t N, int64_t D, unsigned* cmax) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= D) return;
  float m = 0.f;
  bool bad = false;
  for (int64_t k = blockIdx.y; k < N; k += gridDim.y) {
    float a;
    if (ET == ELEM_F64) {
      const double x = fabs(((const double*)A)[k * ld + j]);
      bad |= !(x <= 1.0e38);
      a = __double2float_ru(x);  // rounded up: every |entry| stays below 2^e of the float maximum
    } else {
      a = fabsf(load_f<ET>(A, k * ld + j));
    }
    bad |= !(a <= 3.402823466e38f);
    m = fmaxf(m, a);
  }
  atomicMax(&cmax[j], bad ? 0x7f800000u : __float_as_uint(m));
}

// Thread (j, k8): rows 8 k8 .. 8 k8 + 7 of column j -> one 16-byte run per slice.
// Block (t, rb, kb) of S holds slice t of columns 128 rb .. +127, rows 64 kb .. +63,
// element (r, kk) at byte (r/8)*1024 + (kk/8)*128 + (r%8)*16 + (kk%8)*2.
template <int ET>
__global__ void k_slice(const void* A, int64_t ld, int64_t N, int64_t D, const unsigned* cmax, int ns, int RB,
                        int KB, __nv_bfloat16* S) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= (int64_t)RB * 128) return;
  int e = j < D ? col_exp(cmax[j]) : 0;
  const bool live = j < D && e != SL_NONFINITE;
  if (!live) e = 0;
  const int r = (int)(j & 127), rb = (int)(j >> 7);
  if (ET == ELEM_F64) {  // FP64 data: the digits in double arithmetic (53-bit entries, up to 7 slices)
    for (int64_t k8 = blockIdx.y; k8 < (int64_t)KB * 8; k8 += gridDim.y) {
      double v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int64_t k = k8 * 8 + q;
        v[q] = (live && k < N) ? ldexp(((const double*)A)[k * ld + j], 7 - e) : 0.0;  // exact, |v| < 2^7
      }
      const int64_t kb = k8 >> 3, kc = k8 & 7;
      const int64_t off = ((r >> 3) * 1024 + kc * 128 + (r & 7) * 16) / 2;
      for (int t = 0; t < ns; ++t) {
        __align__(16) __nv_bfloat16 h[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const double a = rint(v[q]);
          h[q] = __float2bfloat16_rn((float)a);
          v[q] = (v[q] - a) * 256.0;
        }
        *reinterpret_cast<uint4*>(S + (((int64_t)t * RB + rb) * KB + kb) * SL_BLOCK_ELEMS + off) =
            *reinterpret_cast<const uint4*>(h);
      }
    }
    return;
  }
  for (int64_t k8 = blockIdx.y; k8 < (int64_t)KB * 8; k8 += gridDim.y) {
    float v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int64_t k = k8 * 8 + q;
      v[q] = (live && k < N) ? ldexpf(load_f<ET>(A, k * ld + j), 7 - e) : 0.f;  // exact, |v| < 2^7
    }
    const int64_t kb = k8 >> 3, kc = k8 & 7;
    const int64_t off = ((r >> 3) * 1024 + kc * 128 + (r & 7) * 16) / 2;
    for (int t = 0; t < ns; ++t) {
      __align__(16) __nv_bfloat16 h[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const float a = rintf(v[q]);  // |a| <= 128: exact in BF16
        h[q] = __float2bfloat16_rn(a);
        v[q] = (v[q] - a) * 256.f;    // exact: |v - a| <= 1/2
      }
      *reinterpret_cast<uint4*>(S + (((int64_t)t * RB + rb) * KB + kb) * SL_BLOCK_ELEMS + off) =
          *reinterpret_cast<const uint4*>(h);
    }
  }
}

// Work item of the slice products: pair p = (s, t), tile (I, J) with J counted in NW-block-wide
// column tiles, row split q.  item = q * tiles + (tile of pair p): the row split outermost, so that
// the CTAs running together work on one row range and share its slice blocks in L2.
struct SlItem {
  int s, t, I, J, q;
};
__device__ __forceinline__ SlItem sl_decode(const SlicePlan& pl, int item) {
  SlItem w;
  const int tiles_all = pl.base[pl.np];
  w.q = item / tiles_all;
  const int r = item - w.q * tiles_all;
  int p = 0;
  while (p + 1 < pl.np && pl.base[p + 1] <= r) ++p;
  w.s = pl.ps[p];
  w.t = pl.pt[p];
  const int tile = r - pl.base[p];
  if (!pl.rect && w.s == w.t) {  // symmetric pair: only tiles reaching the upper triangle
    int I = 0, rest = tile;
    while (rest >= pl.TJ - I / pl.nw) {
      rest -= pl.TJ - I / pl.nw;
      ++I;
    }
    w.I = I;
    w.J = I / pl.nw + rest;
  } else {
    w.I = tile / pl.TJ;
    w.J = tile - w.I * pl.TJ;
  }
  return w;
}

// One CTA per work item: a 128 x (128 NW) tile of one slice pair over one row range.  NW = 2 halves
// the shared-memory traffic per MMA flop (the A block serves a 256-wide B operand).
template <int NW>
struct SlCfg {
  static constexpr int STAGES = NW == 1 ? 6 : 4;
  static constexpr int STAGE = (1 + NW) * SL_BLOCK_ELEMS * 2;  // A block + NW B blocks
  static constexpr int SMEM = STAGES * STAGE;                   // 192 KiB
  static constexpr int EPI = 4 * NW;                            // epilogue warps (128 columns each)
  static constexpr int THREADS = 64 + 32 * EPI;
  static constexpr int COLS = 256 * NW;                         // two 128 x 128 NW accumulators
};

template <int NW>
__global__ void __launch_bounds__(SlCfg<NW>::THREADS, 1)
    k_gram_slices_tc(const __nv_bfloat16* __restrict__ S, const __nv_bfloat16* __restrict__ SB, SlicePlan pl,
                     int* __restrict__ out, int* status, int item0) {
  using C = SlCfg<NW>;
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t full[C::STAGES], empty[C::STAGES], tfull[2], tempty[2], drained;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  const int item = item0 + blockIdx.x;
  const SlItem w = sl_decode(pl, item);
  const int kb0 = w.q * pl.kbper, kb1 = min(pl.KB, kb0 + pl.kbper);
  const int nkb = kb1 - kb0, nch = (nkb + SL_CHUNK - 1) / SL_CHUNK;

  if (warp == 1) tc::tmem_alloc(tc::smem_addr(&tmem_base), C::COLS);
  if (tid == 0) {
    for (int i = 0; i < C::STAGES; ++i) {
      tc::bar_init(tc::smem_addr(&full[i]), 1);
      tc::bar_init(tc::smem_addr(&empty[i]), 1);
    }
    for (int i = 0; i < 2; ++i) {
      tc::bar_init(tc::smem_addr(&tfull[i]), 1);
      tc::bar_init(tc::smem_addr(&tempty[i]), C::EPI);
    }
    tc::bar_init(tc::smem_addr(&drained), 1);
    abort_flag = 0;
    tc::bar_init_fence();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_base;
  const __nv_bfloat16* gA = S + (((int64_t)w.s * pl.RB + w.I) * pl.KB + kb0) * SL_BLOCK_ELEMS;
  const __nv_bfloat16* gB = SB + (((int64_t)w.t * pl.RBb + (int64_t)w.J * NW) * pl.KB + kb0) * SL_BLOCK_ELEMS;
  const int64_t bstep = (int64_t)pl.KB * SL_BLOCK_ELEMS;  // next 128-column block of B
  volatile int* abort_v = &abort_flag;

  if (warp == 0) {
    if (lane == 0) {  // producer: bulk copies into the stage ring
      int issued = 0;
      for (int it = 0; it < nkb; ++it) {
        const int st = it % C::STAGES, rnd = it / C::STAGES;
        if (rnd > 0 && !tc::bar_wait(tc::smem_addr(&empty[st]), (rnd - 1) & 1)) {
          dev_fail(status, DEV_TIMEOUT);
          *abort_v = 1;
          break;
        }
        if (*abort_v) break;
        const uint32_t sa = tc::smem_addr(smem + st * C::STAGE), fb = tc::smem_addr(&full[st]);
        tc::bar_arrive_tx(fb, C::STAGE);
        tc::bulk_load(sa, gA + (int64_t)it * SL_BLOCK_ELEMS, SL_BLOCK_ELEMS * 2, fb);
#pragma unroll
        for (int b = 0; b < NW; ++b)  // the B blocks land adjacent: one 128 NW-row operand
          tc::bulk_load(sa + (1 + b) * SL_BLOCK_ELEMS * 2, gB + b * bstep + (int64_t)it * SL_BLOCK_ELEMS,
                        SL_BLOCK_ELEMS * 2, fb);
        issued = it + 1;
      }
      // the copies of the last stages land before the CTA may leave
      for (int it = issued > C::STAGES ? issued - C::STAGES : 0; it < issued; ++it)
        tc::bar_wait(tc::smem_addr(&full[it % C::STAGES]), (it / C::STAGES) & 1);
    }
  } else if (warp == 1) {
    if (lane == 0) {  // MMA issuer
      constexpr uint32_t idesc = tc::idesc_bf16(128, 128 * NW);
      bool ok = true;
      for (int c = 0; c < nch && ok; ++c) {
        const int h = c & 1;
        if (c >= 2 && !tc::bar_wait(tc::smem_addr(&tempty[h]), ((c >> 1) - 1) & 1)) {
          dev_fail(status, DEV_TIMEOUT);
          *abort_v = 1;
          break;
        }
        tc::fence_after_sync();
        const uint32_t d = tmem + (uint32_t)(h * 128 * NW);
        const int i0 = c * SL_CHUNK, i1 = min(nkb, i0 + SL_CHUNK);
        for (int it = i0; it < i1; ++it) {
          const int st = it % C::STAGES, rnd = it / C::STAGES;
          if (!tc::bar_wait(tc::smem_addr(&full[st]), rnd & 1) || *abort_v) {
            dev_fail(status, DEV_TIMEOUT);
            *abort_v = 1;
            ok = false;
            break;
          }
          tc::fence_after_sync();
          const uint32_t sa = tc::smem_addr(smem + st * C::STAGE);
#pragma unroll
          for (int ks = 0; ks < 4; ++ks)  // K = 16 per MMA: two core matrices (256 bytes) along K
            tc::mma_bf16(d, tc::smem_desc(sa + ks * 256, 128, 1024),
                         tc::smem_desc(sa + SL_BLOCK_ELEMS * 2 + ks * 256, 128, 1024), idesc,
                         (it > i0 || ks > 0) ? 1u : 0u);
          tc::commit(tc::smem_addr(&empty[st]));
        }
        if (ok) tc::commit(tc::smem_addr(&tfull[h]));
      }
      tc::commit(tc::smem_addr(&drained));  // every MMA of this CTA has completed
      tc::bar_wait(tc::smem_addr(&drained), 0);
    }
  } else {  // epilogue: lanes 32 (warp % 4) .. +31 are this thread's rows; warp group cg its 128 columns
    const int qd = warp & 3, cg = (warp - 2) >> 2;
    int acc[128];
#pragma unroll
    for (int c = 0; c < 128; ++c) acc[c] = 0;
    bool ok = true;
    for (int c = 0; c < nch; ++c) {
      const int h = c & 1;
      if (!tc::bar_wait(tc::smem_addr(&tfull[h]), (c >> 1) & 1) || *abort_v) {
        if (lane == 0) dev_fail(status, DEV_TIMEOUT);
        *abort_v = 1;
        ok = false;
        break;
      }
      tc::fence_after_sync();
#pragma unroll
      for (int cc = 0; cc < 128; cc += 32) {
        uint32_t r[32];
        tc::tmem_ld32(tmem + ((uint32_t)(qd * 32) << 16) + (uint32_t)(h * 128 * NW + cg * 128 + cc), r);
        tc::tmem_ld_wait();
#pragma unroll
        for (int x = 0; x < 32; ++x) acc[cc + x] += __float2int_rn(__uint_as_float(r[x]));  // integer-valued
      }
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tc::bar_arrive(tc::smem_addr(&tempty[h]));
    }
    if (ok) {  // tile stored column-major: out[item][col][row], 128 NW columns
      int* o = out + (int64_t)item * (16384 * NW) + (int64_t)cg * 16384 + qd * 32 + lane;
#pragma unroll
      for (int c = 0; c < 128; ++c) o[c * 128] = acc[c];
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 1) tc::tmem_dealloc(tmem, C::COLS);
}

// G[i][j] = G[j][i] for i <= j from the integer tiles (pairs ordered by weight, largest first)
template <class Mode>
__global__ void k_gram_combine(const int* __restrict__ out, SlicePlan pl, const unsigned* __restrict__ cmax, CBuf G) {
  const int64_t D = pl.D;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= D) return;
  const int I = (int)(i >> 7), ri = (int)(i & 127);
  const int ei = col_exp(cmax[i]);
  for (int64_t j = i + blockIdx.y; j < D; j += gridDim.y) {
    if (j < i) continue;
    const int J = (int)(j >> 7), rj = (int)(j & 127);
    const int ej = col_exp(cmax[j]);
    double g;
    if (ei == SL_NONFINITE || ej == SL_NONFINITE) {
      g = __longlong_as_double(0x7ff8000000000000ll);
    } else {
      double sum = 0.0;
      int w = pl.ps[0] + pl.pt[0];
      long long v = 0;
      for (int p = 0; p < pl.np; ++p) {
        const int s = pl.ps[p], t = pl.pt[p];
        if (s + t != w) {
          sum += ldexp((double)v, -8 * w);
          v = 0;
          w = s + t;
        }
        // tile (I, J / nw), column (J % nw) 128 + rj; tiles hold 16384 nw integers
        const int64_t ts = (int64_t)16384 * pl.nw;
        const int a = pl.base[p] + tile_index(s == t, pl.TJ, pl.nw, I, J / pl.nw);
        const int ca = (J % pl.nw) * 128 + rj;
        for (int q = 0; q < pl.nsplit; ++q) v += out[((int64_t)q * pl.base[pl.np] + a) * ts + ca * 128 + ri];
        if (s != t) {
          const int b = pl.base[p] + tile_index(false, pl.TJ, pl.nw, J, I / pl.nw);
          const int cb = (I % pl.nw) * 128 + ri;
          for (int q = 0; q < pl.nsplit; ++q) v += out[((int64_t)q * pl.base[pl.np] + b) * ts + cb * 128 + rj];
        }
      }
      sum += ldexp((double)v, -8 * w);
      g = ldexp(sum, ei + ej - 14);
    }
    Mode::st(G, i * D + j, Mode::from_d(g));
    Mode::st(G, j * D + i, Mode::from_d(g));
  }
}

SlicePlan make_slice_plan(int64_t N, int64_t D, int ns, int wmax) {
  SlicePlan pl{};
  pl.ns = ns;
  pl.D = (int)D;
  pl.T = (int)((D + 127) / 128);
  pl.nw = pl.T >= 2 ? 2 : 1;                 // 256-wide tiles once there are two column blocks
  pl.TJ = (pl.T + pl.nw - 1) / pl.nw;
  pl.RB = pl.RBb = pl.TJ * pl.nw;           // one buffer for both sides, padded with zero blocks
  pl.rect = 0;
  pl.KB = (int)((N + 63) / 64);
  // pairs s <= t, s + t <= wmax, ordered by weight (largest s + t first)
  pl.np = 0;
  for (int w = std::min(wmax, 2 * ns - 2); w >= 0; --w)
    for (int s = 0; s <= w / 2; ++s) {
      const int t = w - s;
      if (t >= ns) continue;
      pl.ps[pl.np] = (int8_t)s;
      pl.pt[pl.np] = (int8_t)t;
      ++pl.np;
    }
  auto pair_tiles = [&](int p) {
    return pl.ps[p] == pl.pt[p] ? (int64_t)pl.T * pl.TJ - diag_skip(pl.T, pl.nw) : (int64_t)pl.T * pl.TJ;
  };
  int64_t tiles = 0;
  for (int p = 0; p < pl.np; ++p) tiles += pair_tiles(p);
  // split the rows so that every item stays within SL_KB_MAX K-blocks and the GPU gets >= 2 waves
  int nsplit = (pl.KB + SL_KB_MAX - 1) / SL_KB_MAX;
  const int64_t want = (2 * 152 + tiles - 1) / tiles;
  nsplit = (int)std::max<int64_t>(nsplit, std::min<int64_t>(want, std::max(1, pl.KB / 16)));
  pl.kbper = (pl.KB + nsplit - 1) / nsplit;
  pl.nsplit = (pl.KB + pl.kbper - 1) / pl.kbper;
  int64_t b = 0;
  for (int p = 0; p < pl.np; ++p) {
    pl.base[p] = (int)b;
    b += pair_tiles(p);
  }
  pl.base[pl.np] = (int)b;
  return pl;
}

// Launch items [i0, i0 + n) of a slice-product plan (tile width pl.nw blocks).
cudaError_t launch_slices(const SlicePlan& pl, const __nv_bfloat16* S, const __nv_bfloat16* SB, int* out, int* status,
                          int i0, int n, cudaStream_t st) {
  if (pl.nw == 2) {
    CK(cudaFuncSetAttribute(k_gram_slices_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, SlCfg<2>::SMEM));
    k_gram_slices_tc<2><<<(unsigned)n, SlCfg<2>::THREADS, SlCfg<2>::SMEM, st>>>(S, SB, pl, out, status, i0);
  } else {
    CK(cudaFuncSetAttribute(k_gram_slices_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, SlCfg<1>::SMEM));
    k_gram_slices_tc<1><<<(unsigned)n, SlCfg<1>::THREADS, SlCfg<1>::SMEM, st>>>(S, SB, pl, out, status, i0);
  }
  return cudaGetLastError();
}

// C = X^T Y for X (N x D, nsa slices per entry) and Y (N x K, nsb slices per entry): every tile of
// every pair (s, t), s < nsa, t < nsb, s + t <= wmax, pairs ordered by weight (largest first).
SlicePlan make_rect_plan(int64_t N, int64_t D, int nsa, int a_stride, int64_t K, int nsb, int wmax) {
  SlicePlan pl{};
  pl.ns = nsa;
  pl.D = (int)D;
  pl.RB = a_stride;                          // the A side is the Gram's slice buffer
  pl.T = (int)((D + 127) / 128);
  const int kb = (int)((K + 127) / 128);
  pl.nw = kb >= 2 ? 2 : 1;
  pl.TJ = (kb + pl.nw - 1) / pl.nw;
  pl.RBb = pl.TJ * pl.nw;
  pl.rect = 1;
  pl.KB = (int)((N + 63) / 64);
  pl.np = 0;
  for (int w = std::min(wmax, nsa + nsb - 2); w >= 0; --w)
    for (int a = 0; a <= w; ++a) {
      const int b = w - a;
      if (a >= nsa || b >= nsb) continue;
      pl.ps[pl.np] = (int8_t)a;
      pl.pt[pl.np] = (int8_t)b;
      ++pl.np;
    }
  const int64_t tiles = (int64_t)pl.np * pl.T * pl.TJ;
  int nsplit = (pl.KB + SL_KB_MAX - 1) / SL_KB_MAX;
  const int64_t want = (2 * 152 + tiles - 1) / tiles;
  nsplit = (int)std::max<int64_t>(nsplit, std::min<int64_t>(want, std::max(1, pl.KB / 16)));
  pl.kbper = (pl.KB + nsplit - 1) / nsplit;
  pl.nsplit = (pl.KB + pl.kbper - 1) / pl.kbper;
  for (int q = 0; q <= pl.np; ++q) pl.base[q] = q * pl.T * pl.TJ;
  return pl;
}

// c[r][i] (column-major, D x K) = sum over pairs of the integer tiles of X^T Y, scaled by the column
// exponents of X (i) and Y (r); weights added from the smallest up, as in the Gram's combine.
template <class Mode>
__global__ void k_rect_combine(const int* __restrict__ out, SlicePlan pl, const unsigned* __restrict__ cmaxa,
                               const unsigned* __restrict__ cmaxb, int64_t K, CBuf c) {
  const int64_t D = pl.D;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= D) return;
  const int I = (int)(i >> 7), ri = (int)(i & 127);
  const int ei = col_exp(cmaxa[i]);
  for (int64_t r = blockIdx.y; r < K; r += gridDim.y) {
    const int J = (int)(r >> 7), rj = (int)(r & 127);
    const int ej = col_exp(cmaxb[r]);
    double g;
    if (ei == SL_NONFINITE || ej == SL_NONFINITE) {
      g = __longlong_as_double(0x7ff8000000000000ll);
    } else {
      double sum = 0.0;
      int w = pl.ps[0] + pl.pt[0];
      long long v = 0;
      for (int p = 0; p < pl.np; ++p) {
        if (pl.ps[p] + pl.pt[p] != w) {
          sum += ldexp((double)v, -8 * w);
          v = 0;
          w = pl.ps[p] + pl.pt[p];
        }
        const int a = pl.base[p] + I * pl.TJ + J / pl.nw;
        const int ca = (J % pl.nw) * 128 + rj;
        const int64_t ts = (int64_t)16384 * pl.nw;
        for (int q = 0; q < pl.nsplit; ++q) v += out[((int64_t)q * pl.base[pl.np] + a) * ts + ca * 128 + ri];
      }
      sum += ldexp((double)v, -8 * w);
      g = ldexp(sum, ei + ej - 14);
    }
    Mode::st(c, r * D + i, Mode::from_d(g));
  }
}

// G = X^T X for X (N x D, row-major, row stride ld, element type ET) into `G` (Mode precision):
// ns slices per entry, pairs s + t <= wmax.  With Y != nullptr (N x K FP64, row stride K) also
// c = X^T Y (column-major D x K, Mode precision) from the same slices of X and nsy slices of Y.
template <class Mode, int ET>
cudaError_t gram_slices_typed(ihsbin_problem* p, const void* X, int64_t ld, int64_t N, int64_t D, int ns, int wmax,
                              CBuf G, int cat_slice, int cat_tc, int cat_combine, cudaStream_t st, int max_ctas = 0,
                              const double* Y = nullptr, int64_t K = 0, int nsy = 0, CBuf c = CBuf{}) {
  struct {
    const void* A;
    int64_t ld;
  } A{X, ld};
  const SlicePlan pl = make_slice_plan(N, D, ns, wmax);
  const int items = pl.base[pl.np] * pl.nsplit;
  unsigned* cmax = nullptr;
  __nv_bfloat16* S = nullptr;
  int* out = nullptr;
  CK(prob_alloc(p, (size_t)D * sizeof(unsigned), (void**)&cmax, SCOPE_SCRATCH));
  CK(prob_alloc(p, (size_t)pl.ns * pl.RB * pl.KB * SL_BLOCK_ELEMS * 2, (void**)&S, SCOPE_SCRATCH));
  CK(prob_alloc(p, (size_t)items * 16384 * pl.nw * sizeof(int), (void**)&out, SCOPE_SCRATCH));
  CK(cudaMemsetAsync(cmax, 0, (size_t)D * sizeof(unsigned), st));
  const size_t es = ET == ELEM_F64 ? 8 : ET == ELEM_F32 ? 4 : 2;
  {
    KTimer kt(p, cat_slice, st, 0, (double)N * D * es);
    const unsigned gy = (unsigned)std::min<int64_t>(std::max<int64_t>(1, N / 64), 1024);
    k_col_absmax<ET><<<dim3((unsigned)((D + 127) / 128), gy), 128, 0, st>>>(A.A, A.ld, N, D, cmax);
    CK(cudaGetLastError());
  }
  {
    KTimer kt(p, cat_slice, st, 0, (double)N * D * es + (double)pl.ns * pl.RB * pl.KB * SL_BLOCK_ELEMS * 2);
    const unsigned gy = (unsigned)std::min<int64_t>((int64_t)pl.KB * 8, 32768);
    k_slice<ET><<<dim3((unsigned)pl.RB, gy), 128, 0, st>>>(A.A, A.ld, N, D, cmax, pl.ns, pl.RB, pl.KB, S);
    CK(cudaGetLastError());
  }
  {
    // the method's work: the symmetric Gram, N D (D + 1) flops, one read of X at its storage width;
    // executed: the BF16 slice products (unpadded, 2 N per output entry and pair) and slice images
    const double mfl = (double)N * D * (D + 1.0), mby = (double)N * D * es;
    double fl = 0;
    for (int q = 0; q < pl.np; ++q) fl += 2.0 * N * (pl.ps[q] == pl.pt[q] ? D * (D + 1) / 2.0 : (double)D * D);
    const double by = (double)pl.ns * pl.RB * pl.KB * SL_BLOCK_ELEMS * 2 + (double)items * 65536 * pl.nw;
    // max_ctas > 0: launches of at most max_ctas CTAs (one wave each), so that the SMs beyond them
    // stay free for work on other streams
    const int chunk = max_ctas > 0 ? std::min(items, max_ctas) : items;
    for (int i0 = 0; i0 < items; i0 += chunk) {
      const int n = std::min(chunk, items - i0);
      KTimer kt(p, cat_tc, st, mfl * n / items, mby * n / items, fl * n / items, by * n / items);
      CK(launch_slices(pl, S, S, out, p->status, i0, n, st));
    }
  }
  {
    KTimer kt(p, cat_combine, st, 0, (double)items * 65536 * pl.nw + (double)D * D * 8);
    const unsigned gy = (unsigned)std::min<int64_t>(std::max<int64_t>(1, D), 1024);
    k_gram_combine<Mode><<<dim3((unsigned)((D + 127) / 128), gy), 128, 0, st>>>(out, pl, cmax, G);
    CK(cudaGetLastError());
  }
  if (!Y) return cudaSuccess;
  // the right-hand side X^T Y from the same slices of X (step a3)
  const SlicePlan pr = make_rect_plan(N, D, ns, pl.RB, K, nsy, kGramMaxWeight);
  const int itr = pr.base[pr.np] * pr.nsplit;
  unsigned* cmaxy = nullptr;
  __nv_bfloat16* SY = nullptr;
  int* outy = nullptr;
  CK(prob_alloc(p, (size_t)K * sizeof(unsigned), (void**)&cmaxy, SCOPE_SCRATCH));
  CK(prob_alloc(p, (size_t)nsy * pr.RBb * pr.KB * SL_BLOCK_ELEMS * 2, (void**)&SY, SCOPE_SCRATCH));
  CK(prob_alloc(p, (size_t)itr * 16384 * pr.nw * sizeof(int), (void**)&outy, SCOPE_SCRATCH));
  CK(cudaMemsetAsync(cmaxy, 0, (size_t)K * sizeof(unsigned), st));
  {
    KTimer kt(p, K_RHS, st, 0, (double)N * K * 8 * 2 + (double)nsy * pr.RBb * pr.KB * SL_BLOCK_ELEMS * 2);
    const unsigned gy = (unsigned)std::min<int64_t>(std::max<int64_t>(1, N / 64), 1024);
    k_col_absmax<ELEM_F64><<<dim3((unsigned)pr.RBb, gy), 128, 0, st>>>(Y, K, N, K, cmaxy);
    CK(cudaGetLastError());
    const unsigned gy2 = (unsigned)std::min<int64_t>((int64_t)pr.KB * 8, 32768);
    k_slice<ELEM_F64><<<dim3((unsigned)pr.RBb, gy2), 128, 0, st>>>(Y, K, N, K, cmaxy, nsy, pr.RBb, pr.KB, SY);
    CK(cudaGetLastError());
  }
  {
    double fl = 2.0 * pr.np * N * D * K;
    const double by = ((double)pl.ns * pl.RB + (double)nsy * pr.RBb) * pr.KB * SL_BLOCK_ELEMS * 2 +
                      (double)itr * 65536 * pr.nw;
    const int chunk = max_ctas > 0 ? std::min(itr, max_ctas) : itr;
    for (int i0 = 0; i0 < itr; i0 += chunk) {
      const int n = std::min(chunk, itr - i0);
      // the method's work: 2 N D K flops, one read of X and of Y
      KTimer kt(p, K_RHS, st, 2.0 * N * D * K * n / itr, ((double)N * D * es + (double)N * K * 8) * n / itr,
                fl * n / itr, by * n / itr);
      CK(launch_slices(pr, S, SY, outy, p->status, i0, n, st));
    }
  }
  {
    KTimer kt(p, K_RHS, st, 0, (double)itr * 65536 * pr.nw + (double)D * K * 8);
    const unsigned gy = (unsigned)std::min<int64_t>(std::max<int64_t>(1, K), 1024);
    k_rect_combine<Mode><<<dim3((unsigned)((D + 127) / 128), gy), 128, 0, st>>>(outy, pr, cmax, cmaxy, K, c);
    CK(cudaGetLastError());
  }
  return cudaSuccess;
}

}  // namespace

cudaError_t gram_dense_slices(ihsbin_problem* p, int compute, cudaStream_t st, int reserve_sms, CBuf* rhs) {
  const Tall& A = p->A;
  const int et = A.elem;
  const int cs = K_GRAM_SLICE, ct = K_GRAM_TC, cc = K_GRAM_COMBINE;
  int mc = 0;
  if (reserve_sms > 0) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
      mc = std::max(1, sms - reserve_sms);
  }
  const int ns = gram_slices_for(et, p->tf32);
  const double* Y = rhs ? p->B : nullptr;
  const int64_t K = rhs ? p->K : 0;
  const CBuf c = rhs ? *rhs : CBuf{};
  if (compute == IHSBIN_COMPUTE_F64)
    return et == ELEM_F32
               ? gram_slices_typed<F64, ELEM_F32>(p, A.A, A.ld, A.N, A.D, ns, kGramMaxWeight, p->G, cs, ct, cc, st, mc,
                                                  Y, K, kRhsSlices, c)
               : gram_slices_typed<F64, ELEM_BF16>(p, A.A, A.ld, A.N, A.D, ns, kGramMaxWeight, p->G, cs, ct, cc, st, mc,
                                                   Y, K, kRhsSlices, c);
  return et == ELEM_F32
             ? gram_slices_typed<DD, ELEM_F32>(p, A.A, A.ld, A.N, A.D, ns, kGramMaxWeight, p->G, cs, ct, cc, st, mc, Y,
                                               K, kRhsSlices, c)
             : gram_slices_typed<DD, ELEM_BF16>(p, A.A, A.ld, A.N, A.D, ns, kGramMaxWeight, p->G, cs, ct, cc, st, mc, Y,
                                                K, kRhsSlices, c);
}

// G_S = (S A_hat)^T (S A_hat) of the FP64 sketch: seven slices (55 bits) and pairs s + t <= 7, so
// every entry of S A_hat within 2^-48 of its column's largest magnitude is exact and the result
// matches the exact Gram to about FP64 rounding.
cudaError_t sketch_gram_slices(ihsbin_problem* p, cudaStream_t st) {
  return gram_slices_typed<F64, ELEM_F64>(p, p->SA, p->A.D, p->sk.m, p->A.D, 7, 7, CBuf{p->GS, nullptr},
                                          K_SKETCH_GRAM, K_SKETCH_GRAM, K_SKETCH_GRAM, st);
}

uint64_t gram_slices_scratch_bytes(int64_t N, int64_t D) {
  const SlicePlan pl = make_slice_plan(N, D, kGramSlices, kGramMaxWeight);  // the FP32 count bounds the BF16 one
  return (uint64_t)pl.ns * pl.RB * pl.KB * SL_BLOCK_ELEMS * 2 + (uint64_t)pl.base[pl.np] * pl.nsplit * 65536 + (uint64_t)D * 4;
}

}  // namespace ihsbin
