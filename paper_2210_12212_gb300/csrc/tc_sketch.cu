// Step a1 for the Gaussian sketch with BF16 entries of BF16 data: S A_hat on the
// 5th-generation tensor cores (tcgen05), S drawn once per call and never per tile.
//
// Section 3 lists the Gaussian sketch first: S_ij = z_ij / sqrt(m) with z_ij ~ N(0, 1).
// With BF16 entries each z_ij / sqrt(m) (FP64) is rounded to FP32 and then to BF16 (to
// nearest, ties to even).  A product of two BF16 numbers is exact in FP32, so S A_hat is
// a plain BF16 contraction accumulated in FP32 -- the sketch arithmetic of the precision
// form (BF16 data, FP32 accumulation).
//
// Draws (k_gauss_draw).  z = sqrt(-2 ln u0) cos(2 pi u1) on the Philox words (w0, w1) of
// counter i N + j (stream 5), u = (w + 1/2) 2^-32.  The kernel evaluates it in FP32:
//  * ln u0 as logf(u0) for u0 < 1/2 and as log1pf(-(1 - u0)) above, both arguments formed
//    from the integer word with one rounding;
//  * cos(2 pi u1) by an exact quadrant reduction on the integer word, then sinpif on an
//    argument in (0, 1/2] (so the result keeps its relative accuracy near the zeros);
//  * with CUDA's documented bounds (logf, log1pf, sinpif: 1 ulp; sqrtf correctly rounded)
//    the FP32 value t of z / sqrt(m) is within 10 FP32 ulps of the FP32 rounding of the FP64
//    value.  Its BF16 rounding is therefore the same unless the low 16 bits of t lie within
//    24 ulps of the rounding midpoint 0x8000 (probability 49/65536).  Those entries go to a
//    fix-up list and are redrawn in FP64 exactly as the FP64 definition reads
//    (k_gauss_fixup), so every BF16 entry equals the one the FP64 computation rounds to.
// The draws are written in the shared-memory image the MMA reads: blocks of 128 rows x 64 k
// (16 KiB), element (r, k) at byte (r/8)*1024 + (k/8)*128 + (r%8)*16 + (k%8)*2 (K-major
// 8 x 16-byte core matrices, no swizzle).  A_hat is laid out the same way by columns
// (k_sketch_bimg: blocks of 256 columns x 64 rows, 32 KiB), through shared memory.
//
// Contraction (k_sketch_mma, persistent, one CTA per SM).  Work item = 128-row tile of S x
// 256-column tile of A_hat x k-split.  Warp 0 (one lane) streams each k-block with two bulk
// copies (16 + 32 KiB) into a 4-stage ring; warp 1 owns 512 Tensor Memory columns (two
// 128 x 256 FP32 accumulators) and one lane issues four tcgen05.mma (M = 128, N = 256,
// K = 16) per stage; warps 2..5 drain a finished accumulator (tcgen05.ld) into FP32 partial
// sums [split][column][row] while the next item accumulates into the other buffer.
// k_sketch_reduce adds the splits in FP64 in a fixed order into S A_hat.  Every wait is
// bounded in time (DEV_TIMEOUT in the status word; the pipeline drains and returns).
//
// Accuracy: the products are exact; the only rounding is the FP32 accumulation of at most
// kbper * 64 products per output entry and split, then one FP64 addition per split.
#include <algorithm>
#include <cmath>

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

constexpr int SK_BK = 64;                       // k per block
constexpr int SK_ABLK = 128 * SK_BK;            // S block: 128 rows x 64 k (16 KiB)
constexpr int SK_BBLK = 256 * SK_BK;            // A_hat block: 256 columns x 64 k (32 KiB)
constexpr int SK_STAGES = 4;
constexpr int SK_STAGE = (SK_ABLK + SK_BBLK) * 2;  // 48 KiB
constexpr int SK_SMEM = SK_STAGES * SK_STAGE;      // 192 KiB
constexpr int SK_THREADS = 192;
constexpr int SK_TMEM_COLS = 512;               // two 128 x 256 FP32 accumulators
constexpr int SK_MARGIN = 24;                   // fall-back window around a BF16 midpoint (FP32 ulps)
constexpr int SK_FIXBUF = 3072;                 // per-block staging of fall-back entries (24 KiB: a draw CTA fits beside a Gram CTA)
constexpr int SK_DRAW_THREADS = 256;

// A window [i0, i0 + rows) x [j0, j0 + cols) of the m x N sketch, drawn into image blocks.
struct DrawWin {
  int64_t m, N;
  int64_t i0, j0, rows, cols;
  int RB, KB;                    // image blocks: RB row tiles x KB k-blocks
  uint64_t seed;
  float ism;                     // FP32(1 / sqrt(m))
  double sqrt_m;                 // sqrt(m) in FP64
  uint16_t* img;                 // [RB][KB][8192] BF16 bits
  unsigned long long* fix;       // fall-back list: image element indices
  unsigned* fix_count;
  unsigned fix_cap;
};

__device__ __forceinline__ uint16_t bf16_rne(float f) {
  const uint32_t b = __float_as_uint(f);
  return (uint16_t)((b + 0x7FFFu + ((b >> 16) & 1u)) >> 16);
}

// z in FP32 from the two Philox words (see the file comment for the error bound).
__device__ __forceinline__ float gauss_f32(uint32_t w0, uint32_t w1) {
  float l;
  if (w0 < 0x80000000u) l = logf(__uint2float_rn(2u * w0 + 1u) * 0x1p-33f);      // u0 = (2 w0 + 1) 2^-33
  else l = log1pf(-(__uint2float_rn(2u * ~w0 + 1u) * 0x1p-33f));                   // 1 - u0 = (2 ~w0 + 1) 2^-33
  const float r = sqrtf(-2.f * l);
  // cos(2 pi u1) = cos(qd pi/2 + theta), theta = 2 pi (g + 1/2) 2^-32 in (0, pi/2)
  const uint32_t g = w1 & 0x3FFFFFFFu, qd = w1 >> 30;
  const uint32_t a = (qd & 1u) ? 2u * g + 1u            // sin(theta)  = sinpi((2g + 1) 2^-32)
                               : 0x7FFFFFFFu - 2u * g;  // cos(theta)  = sinpi((2^31 - 2g - 1) 2^-32)
  const float s = sinpif(__uint2float_rn(a) * 0x1p-32f);
  const float z = r * s;
  return (qd == 1u || qd == 2u) ? -z : z;
}

// The FP64 definition, rounded FP64 -> FP32 -> BF16.
__device__ __forceinline__ uint16_t gauss_bf16_f64(uint32_t w0, uint32_t w1, double sqrt_m) {
  const double u0 = ((double)w0 + 0.5) * 0x1p-32, u1 = ((double)w1 + 0.5) * 0x1p-32;
  const double z = sqrt(-2.0 * log(u0)) * cos(2.0 * 3.141592653589793 * u1);
  return bf16_rne(__double2float_rn(z / sqrt_m));
}

// image element index -> (row, column) of the window
__device__ __forceinline__ void img_decode(uint64_t e, int KB, int64_t& li, int64_t& lj) {
  const uint64_t G = e >> 3;
  const int q = (int)(e & 7);
  const uint64_t b = G >> 10;
  const int g = (int)(G & 1023);
  const int64_t rb = (int64_t)(b / (uint64_t)KB), kb = (int64_t)(b % (uint64_t)KB);
  li = rb * 128 + (((g >> 6) << 3) | (g & 7));
  lj = kb * 64 + (((g >> 3) & 7) << 3) + q;
}

// One thread per 16-byte granule (8 consecutive k of one row); consecutive threads write
// consecutive granules.  Grid-stride with block-uniform trip counts (the fall-back entries are
// staged in shared memory and flushed with one global atomic per flush).
__global__ void __launch_bounds__(SK_DRAW_THREADS) k_gauss_draw(DrawWin w) {
  __shared__ unsigned long long sbuf[SK_FIXBUF];
  __shared__ unsigned scount, sbase;
  if (threadIdx.x == 0) scount = 0;
  __syncthreads();
  const int64_t total = (int64_t)w.RB * w.KB * 1024;
  const int64_t stride = (int64_t)gridDim.x * SK_DRAW_THREADS;
  for (int64_t base = (int64_t)blockIdx.x * SK_DRAW_THREADS; base < total; base += stride) {
    const int64_t G = base + threadIdx.x;
    if (G < total) {
      const int64_t b = G >> 10;
      const int g = (int)(G & 1023);
      const int64_t rb = b / w.KB, kb = b - rb * w.KB;
      const int64_t li = rb * 128 + (((g >> 6) << 3) | (g & 7));
      const int64_t lj = kb * 64 + (((g >> 3) & 7) << 3);
      __align__(16) uint16_t h[8];
      const uint64_t c0 = (uint64_t)(w.i0 + li) * (uint64_t)w.N + (uint64_t)(w.j0 + lj);
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        h[q] = 0;
        if (li < w.rows && lj + q < w.cols) {
          const u32x4 x = rng_draw(w.seed, STREAM_GAUSSIAN, c0 + (uint64_t)q);
          const float t = gauss_f32(x.x, x.y) * w.ism;
          const int d = (int)(__float_as_uint(t) & 0xFFFFu) - 0x8000;
          h[q] = bf16_rne(t);
          if (d <= SK_MARGIN && d >= -SK_MARGIN) {
            const unsigned s = atomicAdd(&scount, 1u);
            sbuf[s] = ((unsigned long long)G << 3) | (unsigned long long)q;
          }
        }
      }
      *reinterpret_cast<uint4*>(w.img + (G << 3)) = *reinterpret_cast<const uint4*>(h);
    }
    __syncthreads();
    // block-uniform: flush when another iteration could overflow the buffer, or at the end
    if (scount > (unsigned)(SK_FIXBUF - 8 * SK_DRAW_THREADS) || base + stride >= total) {
      if (threadIdx.x == 0) sbase = scount ? atomicAdd(w.fix_count, scount) : 0u;
      __syncthreads();
      for (unsigned x = threadIdx.x; x < scount; x += SK_DRAW_THREADS)
        if ((unsigned long long)sbase + x < w.fix_cap) w.fix[sbase + x] = sbuf[x];
      __syncthreads();
      if (threadIdx.x == 0) scount = 0;
      __syncthreads();
    }
  }
}

// The listed entries redrawn in FP64 (full warps: the FP64 pipe's cost is per instruction).
__global__ void k_gauss_fixup(DrawWin w) {
  const unsigned n = min(*w.fix_count, w.fix_cap);
  for (unsigned x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x) {
    const unsigned long long e = w.fix[x];
    int64_t li, lj;
    img_decode(e, w.KB, li, lj);
    const u32x4 v = rng_draw(w.seed, STREAM_GAUSSIAN, (uint64_t)(w.i0 + li) * (uint64_t)w.N + (uint64_t)(w.j0 + lj));
    w.img[e] = gauss_bf16_f64(v.x, v.y, w.sqrt_m);
  }
}

// Only when the list overflowed: every entry of the window near a midpoint redrawn in FP64.
__global__ void k_gauss_redo(DrawWin w) {
  if (*w.fix_count <= w.fix_cap) return;
  const int64_t total = (int64_t)w.RB * w.KB * 8192;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t li, lj;
    img_decode((uint64_t)e, w.KB, li, lj);
    if (li >= w.rows || lj >= w.cols) continue;
    const u32x4 v = rng_draw(w.seed, STREAM_GAUSSIAN, (uint64_t)(w.i0 + li) * (uint64_t)w.N + (uint64_t)(w.j0 + lj));
    const float t = gauss_f32(v.x, v.y) * w.ism;
    const int d = (int)(__float_as_uint(t) & 0xFFFFu) - 0x8000;
    if (d <= SK_MARGIN && d >= -SK_MARGIN) w.img[e] = gauss_bf16_f64(v.x, v.y, w.sqrt_m);
  }
}

// Image -> row-major window (for the entries export).
__global__ void k_img_unpack(const uint16_t* img, int KB, int64_t rows, int64_t cols, uint16_t* out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= rows * cols) return;
  const int64_t i = e / cols, j = e % cols;
  const int64_t rb = i >> 7, kb = j >> 6;
  const int r = (int)(i & 127), k = (int)(j & 63);
  out[e] = img[(rb * KB + kb) * SK_ABLK + (r >> 3) * 512 + (k >> 3) * 64 + (r & 7) * 8 + (k & 7)];
}

// A_hat rows [j0, j0 + 64 KB) as B-operand blocks [cb][kb] of 256 columns x 64 rows: one CTA per
// block, a 64 x 256 tile through shared memory (4-byte words, rows padded to 129 words so the
// column reads are free of bank conflicts).
__global__ void __launch_bounds__(256) k_sketch_bimg(const uint16_t* A, int64_t ld, int64_t N, int64_t D, int64_t j0,
                                                      int KB, uint16_t* img) {
  __shared__ uint32_t t[64][129];
  const int64_t kb = blockIdx.x, cb = blockIdx.y;
  for (int x = threadIdx.x; x < 64 * 128; x += 256) {
    const int row = x >> 7, wc = x & 127;
    const int64_t k = j0 + kb * 64 + row, c = cb * 256 + 2 * wc;
    uint32_t v = 0;
    if (k < N) {
      const uint16_t* src = A + k * ld + c;
      const uint32_t lo = c < D ? src[0] : 0u, hi = c + 1 < D ? src[1] : 0u;
      v = lo | (hi << 16);
    }
    t[row][wc] = v;
  }
  __syncthreads();
  uint16_t* dst = img + (cb * KB + kb) * SK_BBLK;
  for (int g = threadIdx.x; g < 2048; g += 256) {
    const int c = ((g >> 6) << 3) | (g & 7), k8 = ((g >> 3) & 7) << 3;
    __align__(16) uint16_t h[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) h[q] = (uint16_t)(t[k8 + q][c >> 1] >> ((c & 1) * 16));
    *reinterpret_cast<uint4*>(dst + g * 8) = *reinterpret_cast<const uint4*>(h);
  }
}

struct SkArgs {
  const __nv_bfloat16* S;   // [RB][KB] blocks of 128 x 64
  const __nv_bfloat16* Bm;  // [CB][KB] blocks of 256 x 64
  int RB, CB, KB, nsplit, kbper;
  int64_t Mp, Dp;           // padded rows / columns of the partial sums
  float* part;              // [split][column][row]
  int* status;
};

// Persistent: CTA b takes items b, b + gridDim.x, ...; item = (sp * RB + rb) * CB + cb (column tiles
// fastest, so CTAs running together share S blocks in L2).  Ring and accumulator counters run on
// across items.
__global__ void __launch_bounds__(SK_THREADS, 1) k_sketch_mma(SkArgs a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t full[SK_STAGES], empty[SK_STAGES], tfull[2], tempty[2], done;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int items = a.RB * a.CB * a.nsplit;
  struct Item {
    int cb, rb, sp, kb0, nkb;
  };
  auto decode = [&](int item) {
    Item w;
    w.cb = item % a.CB;
    const int r = item / a.CB;
    w.rb = r % a.RB;
    w.sp = r / a.RB;
    w.kb0 = w.sp * a.kbper;
    w.nkb = max(0, min(a.KB, w.kb0 + a.kbper) - w.kb0);
    return w;
  };

  if (warp == 1) tc::tmem_alloc(tc::smem_addr(&tmem_base), SK_TMEM_COLS);
  if (tid == 0) {
    for (int i = 0; i < SK_STAGES; ++i) {
      tc::bar_init(tc::smem_addr(&full[i]), 1);
      tc::bar_init(tc::smem_addr(&empty[i]), 1);
    }
    for (int i = 0; i < 2; ++i) {
      tc::bar_init(tc::smem_addr(&tfull[i]), 1);
      tc::bar_init(tc::smem_addr(&tempty[i]), 4);
    }
    tc::bar_init(tc::smem_addr(&done), 1);
    abort_flag = 0;
    tc::bar_init_fence();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_base;
  volatile int* abort_v = &abort_flag;

  if (warp == 0) {
    if (lane == 0) {  // producer
      uint32_t q = 0;
      bool ok = true;
      for (int item = blockIdx.x; item < items && ok; item += gridDim.x) {
        const Item w = decode(item);
        const __nv_bfloat16* gA = a.S + ((int64_t)w.rb * a.KB + w.kb0) * SK_ABLK;
        const __nv_bfloat16* gB = a.Bm + ((int64_t)w.cb * a.KB + w.kb0) * SK_BBLK;
        for (int it = 0; it < w.nkb; ++it, ++q) {
          const uint32_t st = q % SK_STAGES, rnd = q / SK_STAGES;
          if (rnd > 0 && !tc::bar_wait(tc::smem_addr(&empty[st]), (rnd - 1) & 1)) {
            dev_fail(a.status, DEV_TIMEOUT);
            *abort_v = 1;
          }
          if (*abort_v) {
            ok = false;
            break;
          }
          const uint32_t sa = tc::smem_addr(smem + st * SK_STAGE), fb = tc::smem_addr(&full[st]);
          tc::bar_arrive_tx(fb, SK_STAGE);
          tc::bulk_load(sa, gA + (int64_t)it * SK_ABLK, SK_ABLK * 2, fb);
          tc::bulk_load(sa + SK_ABLK * 2, gB + (int64_t)it * SK_BBLK, SK_BBLK * 2, fb);
        }
      }
      // the copies of the last stages land before the CTA may leave
      for (uint32_t qq = q > (uint32_t)SK_STAGES ? q - SK_STAGES : 0; qq < q; ++qq)
        tc::bar_wait(tc::smem_addr(&full[qq % SK_STAGES]), (qq / SK_STAGES) & 1);
    }
  } else if (warp == 1) {
    if (lane == 0) {  // MMA issuer
      constexpr uint32_t idesc = tc::idesc_bf16(128, 256);
      uint32_t q = 0, cc = 0;
      bool ok = true;
      for (int item = blockIdx.x; item < items && ok; item += gridDim.x, ++cc) {
        const Item w = decode(item);
        const int h = cc & 1;
        if (cc >= 2 && !tc::bar_wait(tc::smem_addr(&tempty[h]), ((cc >> 1) - 1) & 1)) {
          dev_fail(a.status, DEV_TIMEOUT);
          *abort_v = 1;
          break;
        }
        tc::fence_after_sync();
        const uint32_t d = tmem + (uint32_t)(h * 256);
        for (int it = 0; it < w.nkb; ++it, ++q) {
          const uint32_t st = q % SK_STAGES, rnd = q / SK_STAGES;
          if (!tc::bar_wait(tc::smem_addr(&full[st]), rnd & 1) || *abort_v) {
            dev_fail(a.status, DEV_TIMEOUT);
            *abort_v = 1;
            ok = false;
            break;
          }
          tc::fence_after_sync();
          const uint32_t sa = tc::smem_addr(smem + st * SK_STAGE), sb = sa + SK_ABLK * 2;
#pragma unroll
          for (int ks = 0; ks < SK_BK / 16; ++ks)  // K = 16 per MMA: two core matrices (256 bytes) along K
            tc::mma_bf16(d, tc::smem_desc(sa + ks * 256, 128, 1024), tc::smem_desc(sb + ks * 256, 128, 1024), idesc,
                         (it > 0 || ks > 0) ? 1u : 0u);
          tc::commit(tc::smem_addr(&empty[st]));
        }
        if (ok) tc::commit(tc::smem_addr(&tfull[h]));
      }
      tc::commit(tc::smem_addr(&done));  // every MMA of this CTA has completed
      tc::bar_wait(tc::smem_addr(&done), 0);
    }
  } else {  // warps 2..5: Tensor Memory lanes 32 (warp % 4) .. +31 are this thread's rows
    const int qd = warp & 3;
    const int r = qd * 32 + lane;
    uint32_t cc = 0;
    for (int item = blockIdx.x; item < items; item += gridDim.x, ++cc) {
      const Item w = decode(item);
      const int h = cc & 1;
      if (!tc::bar_wait(tc::smem_addr(&tfull[h]), (cc >> 1) & 1) || *abort_v) {
        if (lane == 0) dev_fail(a.status, DEV_TIMEOUT);
        *abort_v = 1;
        break;
      }
      tc::fence_after_sync();
      float* o = a.part + ((int64_t)w.sp * a.Dp + (int64_t)w.cb * 256) * a.Mp + (int64_t)w.rb * 128 + r;
      const bool empty_item = w.nkb == 0;  // no MMA ran into this accumulator: its sums are zero
#pragma unroll 1
      for (int c = 0; c < 256; c += 32) {
        uint32_t v[32];
        tc::tmem_ld32(tmem + ((uint32_t)(qd * 32) << 16) + (uint32_t)(h * 256 + c), v);
        tc::tmem_ld_wait();
#pragma unroll
        for (int x = 0; x < 32; ++x) o[(int64_t)(c + x) * a.Mp] = empty_item ? 0.f : __uint_as_float(v[x]);
      }
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tc::bar_arrive(tc::smem_addr(&tempty[h]));
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 1) tc::tmem_dealloc(tmem, SK_TMEM_COLS);
}

// SA[i][j] += sum over splits of part[q][j][i], in FP64 in split order; 32 x 32 tiles through
// shared memory (reads coalesced along i, writes along j).
__global__ void k_sketch_reduce(const float* __restrict__ part, int nq, int64_t Mp, int64_t Dp, int64_t m, int64_t D,
                                double* __restrict__ SA) {
  __shared__ double t[32][33];
  const int64_t i0 = (int64_t)blockIdx.x * 32, j0 = (int64_t)blockIdx.y * 32;
  for (int jj = threadIdx.y; jj < 32; jj += 8) {
    const int64_t j = j0 + jj, i = i0 + threadIdx.x;
    double s = 0.0;
    for (int q = 0; q < nq; ++q) s += (double)part[((int64_t)q * Dp + j) * Mp + i];
    t[jj][threadIdx.x] = s;
  }
  __syncthreads();
  for (int ii = threadIdx.y; ii < 32; ii += 8) {
    const int64_t i = i0 + ii, j = j0 + threadIdx.x;
    if (i < m && j < D) SA[i * D + j] += t[threadIdx.x][ii];
  }
}

int sm_count() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 148;
  return std::max(1, sms);
}

// k-split of a chunk of KB k-blocks over `tiles` output tiles: the fewest splits that minimise
// the per-SM critical path (waves x (k-blocks per item + a fixed per-item cost)).
void pick_split(int64_t tiles, int KB, int sms, int* nsplit, int* kbper) {
  int64_t best = -1;
  *nsplit = 1;
  *kbper = KB;
  for (int ns = 1; ns <= std::min(64, KB); ++ns) {
    const int kp = (KB + ns - 1) / ns;
    const int nsr = (KB + kp - 1) / kp;
    const int64_t items = tiles * nsr;
    const int64_t waves = (items + sms - 1) / sms;
    const int64_t cost = waves * (kp + 8);
    if (best < 0 || cost < best) {
      best = cost;
      *nsplit = nsr;
      *kbper = kp;
    }
  }
}

DrawWin make_win(ihsbin_problem* p, int64_t i0, int64_t rows, int64_t j0, int64_t cols, uint16_t* img,
                 unsigned long long* fix, unsigned* fix_count, unsigned fix_cap) {
  DrawWin w{};
  w.m = p->sk.m;
  w.N = p->A.N;
  w.i0 = i0;
  w.j0 = j0;
  w.rows = rows;
  w.cols = cols;
  w.RB = (int)((rows + 127) / 128);
  w.KB = (int)((cols + 63) / 64);
  w.seed = p->sk.seed;
  w.sqrt_m = std::sqrt((double)p->sk.m);
  w.ism = (float)(1.0 / w.sqrt_m);
  w.img = img;
  w.fix = fix;
  w.fix_count = fix_count;
  w.fix_cap = fix_cap;
  return w;
}

unsigned fix_capacity(int64_t entries) {
  return (unsigned)std::min<int64_t>(std::max<int64_t>(1 << 20, entries / 256), 1u << 30);
}

// Draw the window (FP32 draws, fall-back list, FP64 redraws) into w.img.
cudaError_t draw_window(ihsbin_problem* p, const DrawWin& w, cudaStream_t st) {
  const int sms = sm_count();
  const int64_t granules = (int64_t)w.RB * w.KB * 1024;
  CK(cudaMemsetAsync(w.fix_count, 0, sizeof(unsigned), st));
  {
    KTimer kt(p, K_SKETCH_DRAW, st, 0, (double)granules * 16);
    const int64_t blocks = std::min<int64_t>((granules + SK_DRAW_THREADS - 1) / SK_DRAW_THREADS, (int64_t)sms * 8);
    k_gauss_draw<<<(unsigned)std::max<int64_t>(1, blocks), SK_DRAW_THREADS, 0, st>>>(w);
    CK(cudaGetLastError());
    k_gauss_fixup<<<(unsigned)(sms * 4), 256, 0, st>>>(w);
    CK(cudaGetLastError());
    k_gauss_redo<<<(unsigned)(sms * 4), 256, 0, st>>>(w);
    CK(cudaGetLastError());
  }
  return cudaSuccess;
}

}  // namespace

bool sketch_gaussian_tc_ok(const ihsbin_problem* p) {
  return p->A.layout == IHSBIN_DENSE_ROWMAJOR && p->A.elem == ELEM_BF16 && p->sk.entries == IHSBIN_BF16;
}

cudaError_t sketch_gaussian_tc(ihsbin_problem* p, cudaStream_t st) {
  const Tall& A = p->A;
  const int64_t m = p->sk.m, N = A.N, D = A.D;
  const int RB = (int)((m + 127) / 128), CB = (int)((D + 255) / 256);
  const int64_t Mp = (int64_t)RB * 128, Dp = (int64_t)CB * 256;
  const int64_t KBt = (N + 63) / 64;
  const int sms = sm_count();
  // k-chunks: the S image of one chunk stays within 4 GiB
  const int64_t kb_chunk = std::max<int64_t>(1, std::min<int64_t>(KBt, (4ll << 30) / (Mp * SK_BK * 2)));
  int ns_max = 1, kp = 1;
  for (int64_t kb0 = 0; kb0 < KBt; kb0 += kb_chunk) {
    int ns;
    pick_split((int64_t)RB * CB, (int)std::min(kb_chunk, KBt - kb0), sms, &ns, &kp);
    ns_max = std::max(ns_max, ns);
  }
  uint16_t *Simg = nullptr, *Bimg = nullptr;
  float* part = nullptr;
  unsigned long long* fix = nullptr;
  unsigned* fix_count = nullptr;
  const unsigned cap = fix_capacity(Mp * kb_chunk * SK_BK);
  CK(prob_alloc(p, (size_t)Mp * kb_chunk * SK_BK * 2, (void**)&Simg, SCOPE_SCRATCH));
  CK(prob_alloc(p, (size_t)Dp * kb_chunk * SK_BK * 2, (void**)&Bimg, SCOPE_SCRATCH));
  CK(prob_alloc(p, (size_t)ns_max * Dp * Mp * sizeof(float), (void**)&part, SCOPE_SCRATCH));
  CK(prob_alloc(p, (size_t)cap * sizeof(unsigned long long), (void**)&fix, SCOPE_SCRATCH));
  CK(prob_alloc(p, sizeof(unsigned), (void**)&fix_count, SCOPE_SCRATCH));
  CK(cudaMemsetAsync(p->SA, 0, (size_t)m * D * sizeof(double), st));
  CK(cudaFuncSetAttribute(k_sketch_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, SK_SMEM));
  for (int64_t kb0 = 0; kb0 < KBt; kb0 += kb_chunk) {
    const int KB = (int)std::min(kb_chunk, KBt - kb0);
    const int64_t j0 = kb0 * SK_BK, nc = std::min<int64_t>(N - j0, (int64_t)KB * SK_BK);
    const DrawWin w = make_win(p, 0, m, j0, nc, Simg, fix, fix_count, cap);
    CK(draw_window(p, w, st));
    {
      KTimer kt(p, K_SKETCH_IMAGE, st, 0, (double)nc * D * 2 + (double)Dp * KB * SK_BK * 2);
      k_sketch_bimg<<<dim3((unsigned)KB, (unsigned)CB), 256, 0, st>>>((const uint16_t*)A.A, A.ld, N, D, j0, KB, Bimg);
      CK(cudaGetLastError());
    }
    int nsplit, kbper;
    pick_split((int64_t)RB * CB, KB, sms, &nsplit, &kbper);
    {
      SkArgs a{};
      a.S = (const __nv_bfloat16*)Simg;
      a.Bm = (const __nv_bfloat16*)Bimg;
      a.RB = RB;
      a.CB = CB;
      a.KB = KB;
      a.nsplit = nsplit;
      a.kbper = kbper;
      a.Mp = Mp;
      a.Dp = Dp;
      a.part = part;
      a.status = p->status;
      const int items = RB * CB * nsplit;
      // algorithmic work: 2 m D N_chunk flops; bytes: one read of S and of A_hat (BF16), FP32 partials
      KTimer kt(p, K_SKETCH_TC, st, 2.0 * m * D * nc, (double)m * nc * 2 + (double)nc * D * 2);
      k_sketch_mma<<<(unsigned)std::min(items, sms), SK_THREADS, SK_SMEM, st>>>(a);
      CK(cudaGetLastError());
    }
    {
      KTimer kt(p, K_SKETCH_REDUCE, st, 0, (double)nsplit * Dp * Mp * 4 + (double)m * D * 16);
      k_sketch_reduce<<<dim3((unsigned)(Mp / 32), (unsigned)(Dp / 32)), dim3(32, 8), 0, st>>>(part, nsplit, Mp, Dp, m,
                                                                                               D, p->SA);
      CK(cudaGetLastError());
    }
  }
  return cudaSuccess;
}

cudaError_t gaussian_entries_bf16(ihsbin_problem* p, int64_t i0, int64_t rows, int64_t j0, int64_t cols,
                                  uint16_t* out_dev, cudaStream_t st) {
  const int64_t RB = (rows + 127) / 128, KB = (cols + 63) / 64;
  uint16_t* img = nullptr;
  unsigned long long* fix = nullptr;
  unsigned* fix_count = nullptr;
  const unsigned cap = fix_capacity(RB * 128 * KB * 64);
  CK(prob_alloc(p, (size_t)RB * KB * SK_ABLK * 2, (void**)&img, SCOPE_SCRATCH));
  CK(prob_alloc(p, (size_t)cap * sizeof(unsigned long long), (void**)&fix, SCOPE_SCRATCH));
  CK(prob_alloc(p, sizeof(unsigned), (void**)&fix_count, SCOPE_SCRATCH));
  const DrawWin w = make_win(p, i0, rows, j0, cols, img, fix, fix_count, cap);
  CK(draw_window(p, w, st));
  const int64_t n = rows * cols;
  k_img_unpack<<<(unsigned)std::max<int64_t>(1, (n + 255) / 256), 256, 0, st>>>(img, (int)KB, rows, cols, out_dev);
  return cudaGetLastError();
}

}  // namespace ihsbin
