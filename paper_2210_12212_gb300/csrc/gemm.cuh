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
// Epilogue contract: __device__ void operator()(int g, int64_t i, int64_t j, Mode::V acc) const.
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
  int tri;  // 0: full; 1: only tiles touching i <= j; 2: only tiles touching i >= j
};

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

  const int g = blockIdx.z;
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

  auto load_tiles = [&](int64_t k0) {
#pragma unroll
    for (int q = 0; q < LA_PER; ++q) {
      int e = tid + q * NT;
      int r, c;
      if (LA::k_contig) { r = e / BK; c = e % BK; } else { c = e / BM; r = e % BM; }
      int64_t gi = i0 + r, gk = k0 + c;
      ra[q] = (gi < sh.M && gk < sh.K) ? la(g, gi, gk) : zero_of<TA>();
    }
#pragma unroll
    for (int q = 0; q < LB_PER; ++q) {
      int e = tid + q * NT;
      int r, c;  // r: k index, c: column
      if (LB::k_contig) { c = e / BK; r = e % BK; } else { r = e / BN; c = e % BN; }
      int64_t gk = k0 + r, gj = j0 + c;
      rb[q] = (gk < sh.K && gj < sh.N) ? lb(g, gk, gj) : zero_of<TB>();
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

  const int64_t ntiles = (sh.K + BK - 1) / BK;
  load_tiles(0);
  for (int64_t kt = 0; kt < ntiles; ++kt) {
    store_tiles();
    __syncthreads();
    if (kt + 1 < ntiles) load_tiles((kt + 1) * BK);
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
      if (gj < sh.N) ep(g, gi, gj, acc[a][b]);
    }
  }
}

template <class Mode, int BM, int BN, int BK, int TM, int TN, class LA, class LB, class EP>
inline cudaError_t launch_gemm(GemmShape sh, int groups, LA la, LB lb, EP ep, cudaStream_t st) {
  if (sh.M <= 0 || sh.N <= 0 || groups <= 0) return cudaSuccess;
  dim3 grid((unsigned)((sh.N + BN - 1) / BN), (unsigned)((sh.M + BM - 1) / BM), (unsigned)groups);
  gemm_kernel<Mode, BM, BN, BK, TM, TN, LA, LB, EP><<<grid, (BM / TM) * (BN / TN), 0, st>>>(sh, la, lb, ep);
  return cudaGetLastError();
}

}  // namespace ihsbin
