// Generic tiled contraction  C_g(i, j) = sum_k A_g(i, k) * B_g(k, j)  on the FP32/FP64 pipes.
//
// Operands come from loader functors (so the sketch draws, the shifted basis
// columns of the IHS-BIN recursion, transposed views, ... are formed while the
// tile is staged) and results go to an epilogue functor (so updates such as
// u_j <- u_j - P r_j and utilde_j += u_j are fused).  blockIdx.z indexes a
// group (an interval of the lambda split, or a batch entry); all groups share
// the same M, N, K.
//
// Loader contract:  using T = element type (float, double or dd);
//   static constexpr bool k_contig  -- consecutive k are adjacent in memory;
//   __device__ T operator()(int g, int64_t row, int64_t col) const  (in range only).
// Epilogue contract: __device__ void operator()(int g, int s, int64_t i, int64_t j, Mode::V acc) const,
// where s is the split index when the K range is split over `ksplit` CTAs
// (each split's epilogue then writes a partial sum that a later pass reduces).
#pragma once
#include "common.cuh"

namespace ihsbin {

template <class T>
__device__ __forceinline__ T zero_of();
template <>
__device__ __forceinline__ float zero_of<float>() { return 0.f; }
template <>
__device__ __forceinline__ double zero_of<double>() { return 0.0; }
template <>
__device__ __forceinline__ dd zero_of<dd>() { return {0.f, 0.f}; }

struct GemmShape {
  int64_t M, N, K;
  int tri;         // 0: full; 1: only tiles touching i <= j; 2: only tiles touching i >= j
  int ksplit = 1;  // K range split over this many CTAs (partial sums per split)
  int kdiag = 0;   // 1: operands vanish for k < max(row, col) (triangular factors): skip that range
};

// Split factor that brings a grid of `ctas` CTAs to about `target` CTAs, with
// at least `min_tiles` BK-tiles of K per split.
inline int pick_split(int64_t ctas, int64_t K, int BK, int64_t target = 4 * 152, int min_tiles = 4,
                      int cap = 64) {
  if (ctas >= target) return 1;
  int64_t s = (target + ctas - 1) / ctas;
  int64_t smax = K / ((int64_t)BK * min_tiles);
  if (s > smax) s = smax;
  if (s > cap) s = cap;
  return s < 1 ? 1 : (int)s;
}

template <class Mode, int BM, int BN, int BK, int TM, int TN, class LA, class LB, class EP>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
    gemm_kernel(GemmShape sh, LA la, LB lb, EP ep) {
  using V = typename Mode::V;
  using TA = typename LA::T;
  using TB = typename LB::T;
  constexpr int NT = (BM / TM) * (BN / TN);
  constexpr int RY = BM / TM, RX = BN / TN;
  static_assert((BM * BK) % NT == 0 && (BK * BN) % NT == 0, "tile/thread mismatch");
  constexpr int LA_PER = BM * BK / NT;
  constexpr int LB_PER = BK * BN / NT;
  pdl_wait();  // launched with programmatic serialization (launch_gemm)
  pdl_trigger();

  const int g = blockIdx.z / sh.ksplit;
  const int sp = blockIdx.z % sh.ksplit;
  const int64_t i0 = (int64_t)blockIdx.y * BM;
  const int64_t j0 = (int64_t)blockIdx.x * BN;
  if (i0 >= sh.M || j0 >= sh.N) return;
  if (sh.tri == 1 && i0 > j0 + BN - 1) return;
  if (sh.tri == 2 && j0 > i0 + BM - 1) return;

  __shared__ TA As[BK][BM + 1];
  __shared__ TB Bs[BK][BN + 1];

  const int tid = threadIdx.x;
  const int tx = tid % RX, ty = tid / RX;

  V acc[TM][TN];
#pragma unroll
  for (int a = 0; a < TM; ++a)
#pragma unroll
    for (int b = 0; b < TN; ++b) acc[a][b] = Mode::zero();

  TA ra[LA_PER];
  TB rb[LB_PER];

  // this CTA's share of the K range
  const int64_t kc = ((sh.K + sh.ksplit - 1) / sh.ksplit + BK - 1) / BK * BK;
  int64_t kbeg = (int64_t)sp * kc;
  const int64_t kend = (kbeg + kc < sh.K) ? kbeg + kc : sh.K;
  if (sh.kdiag) {
    const int64_t kd = ((i0 > j0 ? i0 : j0) / BK) * BK;
    if (kd > kbeg) kbeg = kd;
  }
  auto load_tiles = [&](int64_t k0) {
#pragma unroll
    for (int q = 0; q < LA_PER; ++q) {
      int e = tid + q * NT;
      int r, c;
      if (LA::k_contig) { r = e / BK; c = e % BK; } else { c = e / BM; r = e % BM; }
      int64_t gi = i0 + r, gk = k0 + c;
      ra[q] = (gi < sh.M && gk < kend) ? la(g, gi, gk) : zero_of<TA>();
    }
#pragma unroll
    for (int q = 0; q < LB_PER; ++q) {
      int e = tid + q * NT;
      int r, c;  // r: k index, c: column
      if (LB::k_contig) { c = e / BK; r = e % BK; } else { r = e / BN; c = e % BN; }
      int64_t gk = k0 + r, gj = j0 + c;
      rb[q] = (gk < kend && gj < sh.N) ? lb(g, gk, gj) : zero_of<TB>();
    }
  };
  auto store_tiles = [&]() {
#pragma unroll
    for (int q = 0; q < LA_PER; ++q) {
      int e = tid + q * NT;
      int r, c;
      if (LA::k_contig) { r = e / BK; c = e % BK; } else { c = e / BM; r = e % BM; }
      As[c][r] = ra[q];
    }
#pragma unroll
    for (int q = 0; q < LB_PER; ++q) {
      int e = tid + q * NT;
      int r, c;
      if (LB::k_contig) { c = e / BK; r = e % BK; } else { r = e / BN; c = e % BN; }
      Bs[r][c] = rb[q];
    }
  };

  const int64_t ntiles = kend > kbeg ? (kend - kbeg + BK - 1) / BK : 0;
  load_tiles(kbeg);
  for (int64_t kt = 0; kt < ntiles; ++kt) {
    store_tiles();
    __syncthreads();
    if (kt + 1 < ntiles) load_tiles(kbeg + (kt + 1) * BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      TA av[TM];
      TB bv[TN];
#pragma unroll
      for (int a = 0; a < TM; ++a) av[a] = As[kk][ty + a * RY];
#pragma unroll
      for (int b = 0; b < TN; ++b) bv[b] = Bs[kk][tx + b * RX];
#pragma unroll
      for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int b = 0; b < TN; ++b) Mode::mac(acc[a][b], av[a], bv[b]);
    }
    __syncthreads();
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
      for (int b = 0; b < TN; ++b) acc[a][b] = Mode::renorm(acc[a][b]);
  }

#pragma unroll
  for (int a = 0; a < TM; ++a) {
    int64_t gi = i0 + ty + a * RY;
    if (gi >= sh.M) continue;
#pragma unroll
    for (int b = 0; b < TN; ++b) {
      int64_t gj = j0 + tx + b * RX;
      if (gj < sh.N) ep(g, sp, gi, gj, acc[a][b]);
    }
  }
}

template <class Mode, int BM, int BN, int BK, int TM, int TN, class LA, class LB, class EP>
inline cudaError_t launch_gemm(GemmShape sh, int groups, LA la, LB lb, EP ep, cudaStream_t st) {
  if (sh.M <= 0 || sh.N <= 0 || groups <= 0) return cudaSuccess;
  dim3 grid((unsigned)((sh.N + BN - 1) / BN), (unsigned)((sh.M + BM - 1) / BM), (unsigned)(groups * sh.ksplit));
  return launch_pdl(gemm_kernel<Mode, BM, BN, BK, TM, TN, LA, LB, EP>, grid, dim3((BM / TM) * (BN / TN)), 0, st, sh, la,
                    lb, ep);
}

}  // namespace ihsbin
