// Kernels and launchers of the IHS-BIN hot path (sm_103a).
//
//  a1  sketch        Gaussian (Philox draws + contraction), SRHT (two-level
//                    shared-memory Walsh-Hadamard + row selection), CountSketch/SJLT
//  a2  factor        Gram of S A_hat, batched blocked Cholesky of G_S + lam0_l I for
//                    all intervals at once, explicit inverse P_l = L^-T L^-1
//  a3  rhs           c = A_hat^T B (dual: c = B), u_00 = P_l c
//  a4  basis loop    Proposition 1 / Algorithm 2 recursion, all live intervals per launch
//  a5  dual map      W_l = A_hat utilde_l
//  a6  path eval     X(:, :, t) = tau_l sum_j theta_t^j utilde_j (FP64 coefficients)
#include <algorithm>
#include <cmath>
#include <vector>

#include "gemm.cuh"
#include "internal.h"

namespace ihsbin {

#define CK(x)                              \
  do {                                     \
    cudaError_t e_ = (x);                  \
    if (e_ != cudaSuccess) return e_;      \
  } while (0)

static inline unsigned nblocks(int64_t n, int b) { return (unsigned)std::max<int64_t>(1, (n + b - 1) / b); }

// =============================================================== utilities
__global__ void k_convert_f64(const void* src, int elem, int64_t rows, int64_t cols, int64_t ld, double* dst) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows * cols) return;
  int64_t r = i / cols, c = i % cols;
  dst[i] = load_elem_d(src, elem, r * ld + c);
}

// TF32 by the tensor cores' own conversion (cvt.rna: to nearest, ties away from zero)
__global__ void k_round_tf32(const float* src, int64_t ld, int64_t rows, int64_t cols, float* dst) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= rows * cols) return;
  const int64_t r = e / cols, c = e - r * cols;
  uint32_t t;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(t) : "f"(src[r * ld + c]));
  dst[e] = __uint_as_float(t);
}

cudaError_t launch_round_tf32(const float* src, int64_t ld, int64_t rows, int64_t cols, float* dst, cudaStream_t st) {
  if (rows * cols == 0) return cudaSuccess;
  k_round_tf32<<<nblocks(rows * cols, 256), 256, 0, st>>>(src, ld, rows, cols, dst);
  return cudaGetLastError();
}

cudaError_t launch_convert_to_f64(const void* src, int elem, int64_t rows, int64_t cols, int64_t ld,
                                  double* dst, cudaStream_t st) {
  if (rows * cols == 0) return cudaSuccess;
  k_convert_f64<<<nblocks(rows * cols, 256), 256, 0, st>>>(src, elem, rows, cols, ld, dst);
  return cudaGetLastError();
}

template <class E>
__global__ void k_transpose(const E* src, int64_t rows, int64_t cols, int64_t ld, E* dst) {
  __shared__ E t[32][33];
  int64_t c0 = (int64_t)blockIdx.x * 32, r0 = (int64_t)blockIdx.y * 32;
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    int64_t r = r0 + y, c = c0 + threadIdx.x;
    if (r < rows && c < cols) t[y][threadIdx.x] = src[r * ld + c];
  }
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    int64_t c = c0 + y, r = r0 + threadIdx.x;
    if (r < rows && c < cols) dst[c * rows + r] = t[threadIdx.x][y];
  }
}

cudaError_t launch_transpose_dense(const void* src, int elem, int64_t rows, int64_t cols, int64_t ld,
                                   void* dst, cudaStream_t st) {
  dim3 grid(nblocks(cols, 32), nblocks(rows, 32)), blk(32, 8);
  if (elem == ELEM_F64)
    k_transpose<double><<<grid, blk, 0, st>>>((const double*)src, rows, cols, ld, (double*)dst);
  else if (elem == ELEM_F32)
    k_transpose<float><<<grid, blk, 0, st>>>((const float*)src, rows, cols, ld, (float*)dst);
  else
    k_transpose<uint16_t><<<grid, blk, 0, st>>>((const uint16_t*)src, rows, cols, ld, (uint16_t*)dst);
  return cudaGetLastError();
}

// ============================================================ loaders (gemm)
// Raw data element as a contraction operand.  F64 mode widens to double; DD
// mode keeps FP32/BF16 data as exact floats and splits FP64 data into dd.
template <class Mode, int ET>
struct ElemOp;
template <int ET>
struct ElemOp<F64, ET> {
  using T = double;
  __device__ __forceinline__ static T get(const void* p, int64_t i) { return load_elem_d(p, ET, i); }
};
template <>
struct ElemOp<DD, ELEM_F32> {
  using T = float;
  __device__ __forceinline__ static T get(const void* p, int64_t i) { return ((const float*)p)[i]; }
};
template <>
struct ElemOp<DD, ELEM_BF16> {
  using T = float;
  __device__ __forceinline__ static T get(const void* p, int64_t i) { return bf16_to_f(((const uint16_t*)p)[i]); }
};
template <>
struct ElemOp<DD, ELEM_F64> {
  using T = dd;
  __device__ __forceinline__ static T get(const void* p, int64_t i) { return dd_from_double(((const double*)p)[i]); }
};

// X (rows x cols, row stride ld) read as X^T: operand (i, k) = X[k, i]   (A side, i = column of X)
template <class Mode, int ET>
struct LdTrans {
  using T = typename ElemOp<Mode, ET>::T;
  static constexpr bool k_contig = false;
  const void* X;
  int64_t ld;
  __device__ __forceinline__ T operator()(int, int64_t i, int64_t k) const { return ElemOp<Mode, ET>::get(X, k * ld + i); }
};
// X read as-is on the B side: operand (k, j) = X[k, j]
template <class Mode, int ET>
struct LdRowB {
  using T = typename ElemOp<Mode, ET>::T;
  static constexpr bool k_contig = false;
  const void* X;
  int64_t ld;
  __device__ __forceinline__ T operator()(int, int64_t k, int64_t j) const { return ElemOp<Mode, ET>::get(X, k * ld + j); }
};
// X read as-is on the A side: operand (i, k) = X[i, k]   (row-major, k contiguous)
template <class Mode, int ET>
struct LdRowA {
  using T = typename ElemOp<Mode, ET>::T;
  static constexpr bool k_contig = true;
  const void* X;
  int64_t ld;
  int64_t gstride;  // per-group offset in elements
  __device__ __forceinline__ T operator()(int g, int64_t i, int64_t k) const {
    return ElemOp<Mode, ET>::get(X, g * gstride + i * ld + k);
  }
};
// compute-precision square matrix (row-major), one per group (stride gs) or shared (gs = 0)
template <class Mode>
struct LdCMatA {
  using T = typename Mode::V;
  static constexpr bool k_contig = true;
  CBuf M;
  int64_t D, gs;
  const int* perm;  // group -> matrix index (nullptr = identity)
  __device__ __forceinline__ T operator()(int g, int64_t i, int64_t k) const {
    int64_t gi = perm ? perm[g] : g;
    return Mode::ld(M, gi * gs + i * D + k);
  }
};
// compute-precision column-major panel (column j contiguous over k), per group stride gs
template <class Mode>
struct LdCColB {
  using T = typename Mode::V;
  static constexpr bool k_contig = true;
  CBuf M;
  int64_t D, gs;
  const int* perm;
  __device__ __forceinline__ T operator()(int g, int64_t k, int64_t j) const {
    int64_t gi = perm ? perm[g] : g;
    return Mode::ld(M, gi * gs + j * D + k);
  }
};

// the old columns of every live interval side by side: column c -> (group c / ncol, column c % ncol)
template <class Mode>
struct LdUcat {
  using T = typename Mode::V;
  static constexpr bool k_contig = true;
  CBuf U;
  int64_t D, gs, ncol;
  const int* perm;
  __device__ __forceinline__ T operator()(int, int64_t k, int64_t c) const {
    const int64_t g = c / ncol, col = c - g * ncol;
    return Mode::ld(U, (int64_t)perm[g] * gs + col * D + k);
  }
};

// ============================================================ epilogues
template <class Mode>
struct EpStoreSym {  // symmetric result: write (i, j) and (j, i) into a D x D matrix (group stride gs)
  CBuf M;
  int64_t D, gs;
  __device__ __forceinline__ void operator()(int g, int, int64_t i, int64_t j, typename Mode::V a) const {
    if (i > j) return;
    Mode::st(M, g * gs + i * D + j, a);
    Mode::st(M, g * gs + j * D + i, a);
  }
};
struct EpStoreSymF64 {  // symmetric result into an FP64 matrix
  double* M;
  int64_t D;
  template <class V>
  __device__ __forceinline__ void operator()(int, int, int64_t i, int64_t j, V a) const;
};
template <>
__device__ __forceinline__ void EpStoreSymF64::operator()<double>(int, int, int64_t i, int64_t j, double a) const {
  if (i > j) return;
  M[i * D + j] = a;
  M[j * D + i] = a;
}
template <>
__device__ __forceinline__ void EpStoreSymF64::operator()<dd>(int, int, int64_t i, int64_t j, dd a) const {
  if (i > j) return;
  double v = dd_to_double(a);
  M[i * D + j] = v;
  M[j * D + i] = v;
}
struct EpStoreF64 {  // plain store into an FP64 row-major matrix with row stride ld (group stride gs)
  double* M;
  int64_t ld, gs;
  __device__ __forceinline__ void operator()(int g, int, int64_t i, int64_t j, double a) const { M[g * gs + i * ld + j] = a; }
};
template <class Mode>
struct EpStoreColMajor {  // result (i, j) -> M[g*gs + j*D + i]
  CBuf M;
  int64_t D, gs;
  const int* perm;
  __device__ __forceinline__ void operator()(int g, int, int64_t i, int64_t j, typename Mode::V a) const {
    int64_t gi = perm ? perm[g] : g;
    Mode::st(M, gi * gs + j * D + i, a);
  }
};

// split-K partial sums: buf[((s * G + g) * N + j) * M + i]
template <class Mode>
struct EpPartial {
  CBuf buf;
  int64_t M, N, G;
  __device__ __forceinline__ void operator()(int g, int s, int64_t i, int64_t j, typename Mode::V a) const {
    Mode::st(buf, (((int64_t)s * G + g) * N + j) * M + i, Mode::renorm(a));
  }
};

// symmetric D x D result from S partials of the upper triangle
template <class Mode>
__global__ void k_reduce_sym(CBuf part, int S, int64_t D, CBuf out) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= D * D) return;
  int64_t i = e / D, j = e % D;
  if (i > j) return;
  typename Mode::V v = Mode::ld(part, j * D + i);
#pragma unroll 4
  for (int s = 1; s < S; ++s) v = Mode::add(v, Mode::ld(part, ((int64_t)s * D + j) * D + i));
  Mode::st(out, i * D + j, v);
  Mode::st(out, j * D + i, v);
}

// column-major M x N result (one group) from S partials
template <class Mode>
__global__ void k_reduce_cols(CBuf part, int S, int64_t M, int64_t N, CBuf out) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= M * N) return;
  typename Mode::V v = Mode::ld(part, e);
#pragma unroll 4
  for (int s = 1; s < S; ++s) v = Mode::add(v, Mode::ld(part, (int64_t)s * M * N + e));
  Mode::st(out, e, v);
}

// Tile shape by the column count N (small N: narrow tiles, so that the
// padded columns do not multiply the work).
template <class Mode, class LA, class LB, class EP>
static cudaError_t launch_gemm_n(GemmShape sh, int groups, LA la, LB lb, EP ep, cudaStream_t st) {
  if (sh.N <= 8) return launch_gemm<Mode, 64, 8, 32, 2, 1>(sh, groups, la, lb, ep, st);
  if (sh.N <= 16) return launch_gemm<Mode, 64, 16, 16, 4, 1>(sh, groups, la, lb, ep, st);
  return launch_gemm<Mode, 64, 32, 16, 4, 2>(sh, groups, la, lb, ep, st);
}
static inline int tile_n(int64_t N) { return N <= 8 ? 8 : N <= 16 ? 16 : 32; }
static inline int tile_k(int64_t N) { return N <= 8 ? 32 : 16; }

// =============================================================== a1: sketches
// Gaussian entries S[i][j] = z_ij / sqrt(m), z by Box-Muller on (w0, w1) of
// draw(seed, stream 5, i * N + j); written for a block of columns [j0, j0 + nc).
__global__ void k_gauss_fill(double* S, int64_t m, int64_t N, int64_t j0, int64_t nc, uint64_t seed, double inv_sqrt_m) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m * nc) return;
  int64_t i = e / nc, jj = e % nc;
  u32x4 w = rng_draw(seed, STREAM_GAUSSIAN, (uint64_t)i * (uint64_t)N + (uint64_t)(j0 + jj));
  double u0 = ((double)w.x + 0.5) * 2.3283064365386963e-10;
  double u1 = ((double)w.y + 0.5) * 2.3283064365386963e-10;
  double z = sqrt(-2.0 * log(u0)) * cospi(2.0 * u1);
  S[e] = z * inv_sqrt_m;
}

// The same entries rounded to BF16 (FP64 -> FP32 -> BF16, round to nearest even), stored as floats.
__global__ void k_gauss_fill_bf16(float* S, int64_t m, int64_t N, int64_t j0, int64_t nc, uint64_t seed,
                                  double inv_sqrt_m) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m * nc) return;
  int64_t i = e / nc, jj = e % nc;
  u32x4 w = rng_draw(seed, STREAM_GAUSSIAN, (uint64_t)i * (uint64_t)N + (uint64_t)(j0 + jj));
  double u0 = ((double)w.x + 0.5) * 2.3283064365386963e-10;
  double u1 = ((double)w.y + 0.5) * 2.3283064365386963e-10;
  double z = sqrt(-2.0 * log(u0)) * cospi(2.0 * u1);
  float f = __double2float_rn(z * inv_sqrt_m);
  uint32_t b = __float_as_uint(f);
  b = (b + 0x7FFFu + ((b >> 16) & 1u)) & 0xFFFF0000u;
  S[e] = __uint_as_float(b);
}
struct LdGaussSf {  // float S block (m x nc) as the A operand (exact floats)
  using T = float;
  static constexpr bool k_contig = true;
  const float* S;
  int64_t nc;
  __device__ __forceinline__ T operator()(int, int64_t i, int64_t k) const { return S[i * nc + k]; }
};

template <class Mode>
struct LdGaussS {  // S block (m x nc, row-major FP64) as the A operand
  using T = typename Mode::V;
  static constexpr bool k_contig = true;
  const double* S;
  int64_t nc;
  __device__ __forceinline__ T operator()(int, int64_t i, int64_t k) const { return Mode::from_d(S[i * nc + k]); }
};
template <class Mode, int ET>
struct LdRowsB {  // rows [r0, r0 + nc) of A_hat as the B operand (k = row, j = column)
  using T = typename ElemOp<Mode, ET>::T;
  static constexpr bool k_contig = false;
  const void* X;
  int64_t ld, r0;
  __device__ __forceinline__ T operator()(int, int64_t k, int64_t j) const { return ElemOp<Mode, ET>::get(X, (r0 + k) * ld + j); }
};
struct EpAccumF64 {  // SA[i][j] += acc (FP64; each element owned by one thread per launch)
  double* M;
  int64_t ld;
  template <class V>
  __device__ __forceinline__ void operator()(int, int, int64_t i, int64_t j, V a) const;
};
template <>
__device__ __forceinline__ void EpAccumF64::operator()<double>(int, int, int64_t i, int64_t j, double a) const { M[i * ld + j] += a; }
template <>
__device__ __forceinline__ void EpAccumF64::operator()<dd>(int, int, int64_t i, int64_t j, dd a) const {
  M[i * ld + j] += dd_to_double(a);
}

template <class Mode, int ET>
static cudaError_t gauss_apply(ihsbin_problem* p, double* Sbuf, int64_t chunk, cudaStream_t st) {
  const Tall& A = p->A;
  const int64_t m = p->sk.m, N = A.N, D = A.D;
  const double ism = 1.0 / std::sqrt((double)m);
  for (int64_t j0 = 0; j0 < N; j0 += chunk) {
    int64_t nc = std::min(chunk, N - j0);
    {
      KTimer kt(p, K_SKETCH_DRAW, st, 0, (double)m * nc * 8);
      k_gauss_fill<<<nblocks(m * nc, 256), 256, 0, st>>>(Sbuf, m, N, j0, nc, p->sk.seed, ism);
    }
    CK(cudaGetLastError());
    GemmShape sh{m, D, nc, 0};
    KTimer kt(p, K_SKETCH_APPLY, st, 2.0 * m * D * nc, (double)nc * D * (ET == ELEM_F64 ? 8 : ET == ELEM_F32 ? 4 : 2));
    CK((launch_gemm<Mode, 64, 64, 16, 4, 4>(sh, 1, LdGaussS<Mode>{Sbuf, nc},
                                            LdRowsB<Mode, ET>{A.A, A.ld, j0}, EpAccumF64{p->SA, D}, st)));
  }
  return cudaSuccess;
}

// BF16 entries with FP32/BF16 data: exact float x float products accumulated in float-float
template <int ET>
static cudaError_t gauss_apply_bf16(ihsbin_problem* p, float* Sbuf, int64_t chunk, cudaStream_t st) {
  const Tall& A = p->A;
  const int64_t m = p->sk.m, N = A.N, D = A.D;
  const double ism = 1.0 / std::sqrt((double)m);
  for (int64_t j0 = 0; j0 < N; j0 += chunk) {
    int64_t nc = std::min(chunk, N - j0);
    {
      KTimer kt(p, K_SKETCH_DRAW, st, 0, (double)m * nc * 4);
      k_gauss_fill_bf16<<<nblocks(m * nc, 256), 256, 0, st>>>(Sbuf, m, N, j0, nc, p->sk.seed, ism);
    }
    CK(cudaGetLastError());
    GemmShape sh{m, D, nc, 0};
    KTimer kt(p, K_SKETCH_APPLY, st, 2.0 * m * D * nc, (double)nc * D * (ET == ELEM_F32 ? 4 : 2));
    CK((launch_gemm<DD, 64, 64, 16, 4, 4>(sh, 1, LdGaussSf{Sbuf, nc}, LdRowsB<DD, ET>{A.A, A.ld, j0},
                                          EpAccumF64{p->SA, D}, st)));
  }
  return cudaSuccess;
}

cudaError_t sketch_gaussian(ihsbin_problem* p, cudaStream_t st) {
  const Tall& A = p->A;
  if (A.layout != IHSBIN_DENSE_ROWMAJOR) return cudaErrorNotSupported;
  if (p->sk.apply != IHSBIN_APPLY_FMA && sketch_gaussian_tc_ok(p)) return sketch_gaussian_tc(p, st);
  if (p->sk.entries == IHSBIN_BF16 && A.elem != ELEM_F64) {
    const int64_t m = p->sk.m, N = A.N;
    int64_t chunk = std::max<int64_t>(16, std::min<int64_t>(N, (int64_t)((256ll << 20) / (4 * m))));
    float* Sbuf = nullptr;
    CK(ihsbin::prob_alloc(p, (size_t)m * chunk * sizeof(float), (void**)&Sbuf, SCOPE_SCRATCH));
    CK(cudaMemsetAsync(p->SA, 0, (size_t)m * A.D * sizeof(double), st));
    if (A.elem == ELEM_F32) return gauss_apply_bf16<ELEM_F32>(p, Sbuf, chunk, st);
    return gauss_apply_bf16<ELEM_BF16>(p, Sbuf, chunk, st);
  }
  const int64_t m = p->sk.m, N = A.N;
  int64_t chunk = std::max<int64_t>(16, std::min<int64_t>(N, (int64_t)((256ll << 20) / (8 * m))));
  double* Sbuf = nullptr;
  CK(ihsbin::prob_alloc(p, (size_t)m * chunk * sizeof(double), (void**)&Sbuf, SCOPE_SCRATCH));
  CK(cudaMemsetAsync(p->SA, 0, (size_t)m * A.D * sizeof(double), st));
  // the sketch is applied in FP64 arithmetic in both compute modes
  if (A.elem == ELEM_F64) return gauss_apply<F64, ELEM_F64>(p, Sbuf, chunk, st);
  if (A.elem == ELEM_F32) return gauss_apply<F64, ELEM_F32>(p, Sbuf, chunk, st);
  return gauss_apply<F64, ELEM_BF16>(p, Sbuf, chunk, st);
}

// ---- CountSketch / SJLT: row of S and sign for every (input row i, block t)
__global__ void k_cs_map(int64_t N, int s, int64_t mb, uint64_t seed, int64_t* idx, int8_t* sign) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N * s) return;
  int t = (int)(e % s);
  u32x4 w = rng_draw(seed, STREAM_COUNTSKETCH, (uint64_t)e);
  int64_t bucket = (int64_t)(((uint64_t)w.x * (uint64_t)mb) >> 32);
  idx[e] = (int64_t)t * mb + bucket;
  sign[e] = (w.y & 1u) ? (int8_t)-1 : (int8_t)1;
}
// dense rows: SA[idx[i*s+t], :] += sign * A[i, :] / sqrt(s)   (FP64 atomics); one CTA per row
__global__ void k_cs_dense(const void* A, int elem, int64_t N, int64_t D, int64_t ld, int s, const int64_t* idx,
                           const int8_t* sign, double scale, double* SA) {
  for (int64_t i = blockIdx.x; i < N; i += gridDim.x) {
    for (int64_t c = threadIdx.x; c < D; c += blockDim.x) {
      double v = load_elem_d(A, elem, i * ld + c) * scale;
      for (int t = 0; t < s; ++t) atomicAdd(&SA[idx[i * s + t] * D + c], sign[i * s + t] * v);
    }
  }
}
// CSR rows: one warp per row
__global__ void k_cs_csr(const int64_t* rp, const int32_t* ci, const void* val, int elem, int64_t N, int64_t D,
                         int s, const int64_t* idx, const int8_t* sign, double scale, double* SA) {
  int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
  int lane = threadIdx.x & 31;
  if (row >= N) return;
  for (int64_t e = rp[row] + lane; e < rp[row + 1]; e += 32) {
    double v = load_elem_d(val, elem, e) * scale;
    int64_t c = ci[e];
    for (int t = 0; t < s; ++t) atomicAdd(&SA[idx[row * s + t] * D + c], sign[row * s + t] * v);
  }
}

cudaError_t sketch_countsketch(ihsbin_problem* p, cudaStream_t st) {
  const Tall& A = p->A;
  const int64_t m = p->sk.m, N = A.N, D = A.D;
  const int s = p->sk.s;
  {
    KTimer kt(p, K_SKETCH_DRAW, st, 0, (double)N * s * 9);
    k_cs_map<<<nblocks(N * s, 256), 256, 0, st>>>(N, s, m / s, p->sk.seed, p->sk_idx, p->sk_sign);
  }
  CK(cudaGetLastError());
  CK(cudaMemsetAsync(p->SA, 0, (size_t)m * D * sizeof(double), st));
  const double scale = 1.0 / std::sqrt((double)s);
  const double es = A.elem == ELEM_F64 ? 8 : A.elem == ELEM_F32 ? 4 : 2;
  KTimer kt(p, K_SKETCH_APPLY, st, 2.0 * s * (A.layout == IHSBIN_CSR ? (double)A.nnz : (double)N * D),
            A.layout == IHSBIN_CSR ? A.nnz * (es + 4) + 8.0 * (N + 1) : (double)N * D * es);
  if (A.layout == IHSBIN_DENSE_ROWMAJOR) {
    k_cs_dense<<<(unsigned)std::min<int64_t>(N, 1 << 20), 256, 0, st>>>(A.A, A.elem, N, D, A.ld, s, p->sk_idx, p->sk_sign, scale, p->SA);
  } else {
    k_cs_csr<<<nblocks(N * 32, 256), 256, 0, st>>>(A.rp, A.ci, A.val, A.elem, N, D, s, p->sk_idx, p->sk_sign,
                                                   scale, p->SA);
  }
  return cudaGetLastError();
}

// ---- SRHT
__global__ void k_srht_draws(int64_t Np, uint64_t seed, uint64_t* key, int8_t* sign) {
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= Np) return;
  u32x4 a = rng_draw(seed, STREAM_SRHT_SIGN, (uint64_t)r);
  sign[r] = (a.x & 1u) ? (int8_t)-1 : (int8_t)1;
  u32x4 b = rng_draw(seed, STREAM_SRHT_KEY, (uint64_t)r);
  key[r] = ((uint64_t)b.y << 32) | (uint64_t)b.x;
}

// Select the m smallest keys (ties to the lower index) by an 8-pass MSB radix
// select in one CTA, then list the kept rows in ascending order and record
// each row's rank (rowmap[r] = rank or -1).
__global__ void __launch_bounds__(1024) k_srht_select(const uint64_t* key, int64_t Np, int64_t m, int64_t* sel,
                                                      int* rowmap) {
  __shared__ unsigned int hist[256];
  __shared__ uint64_t s_prefix;
  __shared__ int64_t s_need;
  __shared__ int64_t warp_sums[32];
  __shared__ int64_t s_base;
  const int tid = threadIdx.x;
  if (tid == 0) {
    s_prefix = 0;
    s_need = m;
  }
  __syncthreads();
  uint64_t mask = 0;
  for (int pass = 7; pass >= 0; --pass) {
    for (int b = tid; b < 256; b += blockDim.x) hist[b] = 0;
    __syncthreads();
    const uint64_t prefix = s_prefix;
    for (int64_t r = tid; r < Np; r += blockDim.x) {
      uint64_t k = key[r];
      if ((k & mask) == prefix) atomicAdd(&hist[(k >> (8 * pass)) & 0xFF], 1u);
    }
    __syncthreads();
    if (tid == 0) {
      int64_t need = s_need;
      int b = 0;
      for (; b < 256; ++b) {
        if ((int64_t)hist[b] >= need) break;
        need -= hist[b];
      }
      if (b > 255) b = 255;
      s_need = need;
      s_prefix = prefix | ((uint64_t)b << (8 * pass));
    }
    mask |= (uint64_t)0xFF << (8 * pass);
    __syncthreads();
  }
  const uint64_t thr = s_prefix;  // the m-th smallest key; s_need copies of it are kept
  const int64_t need_eq = s_need;
  // scan in index order: keep key < thr, and the first need_eq rows with key == thr
  if (tid == 0) s_base = 0;
  __syncthreads();
  int64_t eq_seen_before = 0;
  for (int64_t base = 0; base < Np; base += blockDim.x) {
    int64_t r = base + tid;
    int flag_lt = 0, flag_eq = 0;
    if (r < Np) {
      uint64_t k = key[r];
      flag_lt = k < thr;
      flag_eq = k == thr;
    }
    // block-wide exclusive scan of flag_eq then of keep
    int lane = tid & 31, wid = tid >> 5;
    int v = flag_eq;
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += y;
    }
    if (lane == 31) warp_sums[wid] = v;
    __syncthreads();
    if (wid == 0) {
      int64_t w = (lane < (int)(blockDim.x / 32)) ? warp_sums[lane] : 0;
      for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += y;
      }
      warp_sums[lane] = w;
    }
    __syncthreads();
    int64_t eq_rank = eq_seen_before + (v - flag_eq) + (wid > 0 ? warp_sums[wid - 1] : 0);
    int64_t eq_total = warp_sums[blockDim.x / 32 - 1];
    __syncthreads();
    int keep = flag_lt || (flag_eq && eq_rank < need_eq);
    v = keep;
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += y;
    }
    if (lane == 31) warp_sums[wid] = v;
    __syncthreads();
    if (wid == 0) {
      int64_t w = (lane < (int)(blockDim.x / 32)) ? warp_sums[lane] : 0;
      for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += y;
      }
      warp_sums[lane] = w;
    }
    __syncthreads();
    int64_t pos = s_base + (v - keep) + (wid > 0 ? warp_sums[wid - 1] : 0);
    if (r < Np) {
      if (keep && pos < m) {
        sel[pos] = r;
        rowmap[r] = (int)pos;
      } else {
        rowmap[r] = -1;
      }
    }
    int64_t tot = warp_sums[blockDim.x / 32 - 1];
    __syncthreads();
    if (tid == 0) s_base += tot;
    eq_seen_before += eq_total;
    __syncthreads();
  }
}

// One level of the Walsh-Hadamard transform along rows: butterflies over the
// address bits [b0, b0 + q) of the row index, for a tile of w columns.  The
// first level reads A_hat (applying the signs D and the zero padding); the
// last level writes only the kept rows, scaled by 1/sqrt(m), into SA.
// The Hadamard transform runs on exact integers: each column c of D A is converted once to
// int64 fixed point, v = round(a 2^k_c), with k_c chosen from the column's largest magnitude so
// that |v| < 2^(61 - pbits); the pbits butterfly stages can then at most double it pbits times,
// and every addition is exact (no FP64 arithmetic, a slow pipe here).  The only rounding is the
// conversion, at 2^-(62 - pbits) of the column's maximum; the kept rows are converted back
// to FP64 and scaled by 2^-k_c / sqrt(m).
constexpr int FWHT_NONFINITE = -(1 << 30);  // k_c of a column holding an Inf or NaN

// cmax[c] = bits of max_r |A[r][c]| as FP64 (non-negative doubles order like their bit patterns;
// a NaN is larger than every finite value and Inf).  cmax must be zero on entry.
__global__ void k_fwht_colmax(const void* A, int elem, int64_t N, int64_t D, int64_t ld, int64_t rows_per_block,
                              unsigned long long* cmax) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= D) return;
  const int64_t r0 = (int64_t)blockIdx.y * rows_per_block;
  const int64_t r1 = r0 + rows_per_block < N ? r0 + rows_per_block : N;
  unsigned long long m = 0;
  if (elem == ELEM_F64) {
    const unsigned long long* a = (const unsigned long long*)A;
    for (int64_t r = r0; r < r1; ++r) {
      const unsigned long long b = a[r * ld + c] & 0x7fffffffffffffffull;
      m = b > m ? b : m;
    }
  } else {
    unsigned mf = 0;
    for (int64_t r = r0; r < r1; ++r) {
      const unsigned b = (elem == ELEM_F32 ? __float_as_uint(((const float*)A)[r * ld + c])
                                           : ((unsigned)((const uint16_t*)A)[r * ld + c]) << 16) & 0x7fffffffu;
      mf = b > mf ? b : mf;
    }
    m = (unsigned long long)__double_as_longlong((double)__uint_as_float(mf));
  }
  if (m) atomicMax(cmax + c, m);
}

// k_c from the column maximum: |a| <= cmax < 2^e, so |a 2^k| < 2^(61 - pbits) with k = 61 - pbits - e.
__global__ void k_fwht_shift(const unsigned long long* cmax, int64_t D, int pbits, int* kc) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= D) return;
  const unsigned long long b = cmax[c];
  const int E = (int)((b >> 52) & 0x7ff);
  int k;
  if (E == 0x7ff) k = FWHT_NONFINITE;
  else if (b == 0) k = 0;
  else k = 61 - pbits - (E == 0 ? -1022 : E - 1022);
  kc[c] = k;
}

// round(x 2^k) for a finite FP32 x with |x 2^k| < 2^62 (ties away from zero), integer operations only
__device__ __forceinline__ long long f32_to_fixed(float x, int k) {
  const unsigned u = __float_as_uint(x);
  const int ex = (int)((u >> 23) & 0xff);
  if (ex == 0xff) return 0;
  const unsigned long long mant = ex ? ((u & 0x7fffffu) | 0x800000u) : (u & 0x7fffffu);
  const int sh = (ex ? ex - 150 : -149) + k;  // |x| 2^k = mant 2^sh
  unsigned long long mag;
  if (sh >= 0) mag = mant << sh;
  else if (sh > -63) mag = (mant + (1ull << (-sh - 1))) >> (-sh);
  else mag = 0;
  return (u >> 31) ? -(long long)mag : (long long)mag;
}

__device__ __forceinline__ long long load_fixed(const void* A, int elem, int64_t i, int k) {
  if (k == FWHT_NONFINITE) return 0;
  if (elem == ELEM_F32) return f32_to_fixed(((const float*)A)[i], k);
  if (elem == ELEM_BF16) return f32_to_fixed(bf16_to_f(((const uint16_t*)A)[i]), k);
  const double x = ((const double*)A)[i];
  return isfinite(x) ? __double2ll_rn(ldexp(x, k)) : 0;
}

// One level of the transform over the q address bits [b0, b0 + q) of the padded rows: a CTA holds
// the G = 2^q rows of one group (the other bits fixed) for w columns in shared memory and applies
// the q butterfly stages, two at a time (radix 4) and a last single stage when q is odd.  The
// first level reads D A (rows >= N are zero), the last writes the kept rows of S A.
__global__ void k_fwht_level(const void* A, int elem, int64_t N, int64_t D, int64_t ld, const int8_t* dsign,
                             const long long* Yin, long long* Yout, int64_t Np, int b0, int q, int w, bool first,
                             bool last, const int* rowmap, const int* kc, double scale, double* SA) {
  extern __shared__ long long smi[];
  const int G = 1 << q;
  const int64_t grp = blockIdx.y;   // group id: the bits outside [b0, b0+q)
  const int64_t c0 = (int64_t)blockIdx.x * w;
  const int64_t lowmask = ((int64_t)1 << b0) - 1;
  const int64_t base = (grp & lowmask) | ((grp >> b0) << (b0 + q));
  (void)Np;
  auto row_of = [&](int t) -> int64_t { return base | ((int64_t)t << b0); };
  for (int e = threadIdx.x; e < G * w; e += blockDim.x) {
    const int t = e / w, cc = e % w;
    const int64_t r = row_of(t), c = c0 + cc;
    long long v = 0;
    if (c < D) {
      if (first) {
        if (r < N) {
          v = load_fixed(A, elem, r * ld + c, kc[c]);
          if (dsign[r] < 0) v = -v;
        }
      } else {
        v = Yin[r * D + c];
      }
    }
    smi[t * w + cc] = v;
  }
  __syncthreads();
  int h = 1;
  for (; 4 * h <= G; h <<= 2) {  // stages h and 2h together
    for (int e = threadIdx.x; e < (G / 4) * w; e += blockDim.x) {
      const int gi = e / w, cc = e % w;
      const int i0 = (gi & (h - 1)) | ((gi & ~(h - 1)) << 2);
      long long* x = smi + cc;
      const long long x0 = x[i0 * w], x1 = x[(i0 + h) * w], x2 = x[(i0 + 2 * h) * w], x3 = x[(i0 + 3 * h) * w];
      const long long y0 = x0 + x1, y1 = x0 - x1, y2 = x2 + x3, y3 = x2 - x3;
      x[i0 * w] = y0 + y2;
      x[(i0 + h) * w] = y1 + y3;
      x[(i0 + 2 * h) * w] = y0 - y2;
      x[(i0 + 3 * h) * w] = y1 - y3;
    }
    __syncthreads();
  }
  if (h < G) {  // q odd: the last stage alone
    for (int e = threadIdx.x; e < (G / 2) * w; e += blockDim.x) {
      const int pr = e / w, cc = e % w;
      const int lo = (pr / h) * (2 * h) + (pr % h), hi = lo + h;
      const long long a = smi[lo * w + cc], b = smi[hi * w + cc];
      smi[lo * w + cc] = a + b;
      smi[hi * w + cc] = a - b;
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < G * w; e += blockDim.x) {
    const int t = e / w, cc = e % w;
    const int64_t r = row_of(t), c = c0 + cc;
    if (c >= D) continue;
    if (last) {
      const int k = rowmap[r];
      if (k >= 0) {
        const int sh = kc[c];
        SA[(int64_t)k * D + c] = sh == FWHT_NONFINITE ? __longlong_as_double(0x7ff8000000000000ll)
                                                      : ldexp((double)smi[t * w + cc], -sh) * scale;
      }
    } else {
      Yout[r * D + c] = smi[t * w + cc];
    }
  }
}

cudaError_t sketch_srht(ihsbin_problem* p, cudaStream_t st) {
  const Tall& A = p->A;
  if (A.layout != IHSBIN_DENSE_ROWMAJOR) return cudaErrorNotSupported;
  const int64_t N = A.N, D = A.D, m = p->sk.m;
  int pbits = 0;
  while (((int64_t)1 << pbits) < N) ++pbits;
  const int64_t Np = (int64_t)1 << pbits;
  uint64_t* keys = nullptr;
  int* rowmap = nullptr;
  CK(prob_alloc(p, Np * sizeof(uint64_t), (void**)&keys, SCOPE_SCRATCH));
  CK(prob_alloc(p, Np * sizeof(int), (void**)&rowmap, SCOPE_SCRATCH));
  {
    KTimer kt(p, K_SKETCH_DRAW, st, 0, (double)Np * 9);
    k_srht_draws<<<nblocks(Np, 256), 256, 0, st>>>(Np, p->sk.seed, keys, p->sk_sign);
  }
  CK(cudaGetLastError());
  {
    KTimer kt(p, K_SKETCH_DRAW, st, 0, (double)Np * 12 + m * 8);
    k_srht_select<<<1, 1024, 0, st>>>(keys, Np, m, p->sk_idx, rowmap);
  }
  CK(cudaGetLastError());
  const double scale = 1.0 / std::sqrt((double)m);
  // column scales of the fixed-point transform
  unsigned long long* cmax = nullptr;
  int* kc = nullptr;
  CK(prob_alloc(p, D * sizeof(unsigned long long), (void**)&cmax, SCOPE_SCRATCH));
  CK(prob_alloc(p, D * sizeof(int), (void**)&kc, SCOPE_SCRATCH));
  CK(cudaMemsetAsync(cmax, 0, D * sizeof(unsigned long long), st));
  {
    const double es = A.elem == ELEM_F64 ? 8 : A.elem == ELEM_F32 ? 4 : 2;
    KTimer kt(p, K_SKETCH_APPLY, st, 0, (double)N * D * es);
    const int64_t rpb = 256;
    dim3 grid(nblocks(D, 128), (unsigned)((N + rpb - 1) / rpb));
    k_fwht_colmax<<<grid, 128, 0, st>>>(A.A, A.elem, N, D, A.ld, rpb, cmax);
  }
  CK(cudaGetLastError());
  {
    KTimer kt(p, K_SKETCH_APPLY, st, 0, (double)D * 12);
    k_fwht_shift<<<nblocks(D, 256), 256, 0, st>>>(cmax, D, pbits, kc);
  }
  CK(cudaGetLastError());
  // split the pbits address bits into levels of at most 12 bits
  std::vector<std::pair<int, int>> levels;
  if (pbits == 0) levels.push_back({0, 0});
  int nlev = (pbits + 11) / 12;
  if (nlev == 0) nlev = 1;
  int done = 0;
  for (int l = 0; l < nlev && pbits > 0; ++l) {
    int q = (pbits - done + (nlev - l) - 1) / (nlev - l);
    levels.push_back({done, q});
    done += q;
  }
  long long* Y0 = nullptr;
  long long* Y1 = nullptr;
  if (levels.size() > 1) {
    CK(prob_alloc(p, Np * D * sizeof(long long), (void**)&Y0, SCOPE_SCRATCH));
    if (levels.size() > 2) CK(prob_alloc(p, Np * D * sizeof(long long), (void**)&Y1, SCOPE_SCRATCH));
  }
  const long long* yin = nullptr;
  long long* yout = Y0;
  for (size_t l = 0; l < levels.size(); ++l) {
    int b0 = levels[l].first, q = levels[l].second;
    int G = 1 << q;
    int w = std::max(1, std::min(32, 6144 / G));
    size_t smem = (size_t)G * w * sizeof(long long);
    dim3 grid(nblocks(D, w), (unsigned)(Np >> q));
    bool first = (l == 0), last = (l + 1 == levels.size());
    if (smem > 48 * 1024)
      CK(cudaFuncSetAttribute(k_fwht_level, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const double es = A.elem == ELEM_F64 ? 8 : A.elem == ELEM_F32 ? 4 : 2;
    const double rd = first ? (double)N * D * es : (double)Np * D * 8;
    const double wr = last ? (double)m * D * 8 : (double)Np * D * 8;
    KTimer kt(p, K_SKETCH_APPLY, st, (double)Np * D * q, rd + wr);
    k_fwht_level<<<grid, 256, smem, st>>>(A.A, A.elem, N, D, A.ld, p->sk_sign, yin, yout, Np, b0, q, w, first, last,
                                           rowmap, kc, scale, p->SA);
    CK(cudaGetLastError());
    yin = yout;
    yout = (yout == Y0) ? Y1 : Y0;
  }
  return cudaSuccess;
}

// G_S = (S A_hat)^T (S A_hat) in FP64 (the sketched Hessian without the shift).
// The sketched Gram G_S = (S A_hat)^T (S A_hat): on the tensor cores from exact slices of the FP64
// sketch (tc_gram.cu).
cudaError_t sketch_gram(ihsbin_problem* p, cudaStream_t st) { return sketch_gram_slices(p, st); }

// ======================================================= a2: factor and inverse
// H_l = G_S + lam0_l I in compute precision, for every interval l.
template <class Mode>
__global__ void k_shift_copy(const double* GS, int64_t D, const double* lam0, CBuf H) {
  int l = blockIdx.y;
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= D * D) return;
  int64_t i = e / D, j = e % D;
  double v = GS[e];
  typename Mode::V x = Mode::from_d(v);
  if (i == j) x = Mode::add(x, Mode::from_d(lam0[l]));
  Mode::st(H, (int64_t)l * D * D + e, x);
}

constexpr int NB = 32;

// Factor the diagonal block kb of every interval in place (unblocked, column by column) and store
// the inverse of the resulting lower-triangular block (NB x NB, one CTA per interval).
// The block is held in registers: warp w owns rows w, w + 8, w + 16,
// w + 24 and lane c column c.  Column j of a step is published through shared memory (double
// buffered, so one barrier per step), and every thread forms the pivot's square root and
// reciprocal itself, so no thread waits on another's scalar work.  The inverse X = L^-1 is a
// column sweep in the same layout: row k of X divided by L_kk, then subtracted from the rows
// below with L's column k.
template <class Mode>
__global__ void __launch_bounds__(256) k_potrf_diag_reg(CBuf H, int64_t D, int kb, CBuf dinv, int* status) {
  pdl_wait();  // launched with programmatic serialization
  pdl_trigger();
  using V = typename Mode::V;
  const int l = blockIdx.x;
  const int64_t off = (int64_t)l * D * D;
  const int64_t r0 = (int64_t)kb * NB;
  const int nb = (D - r0 < NB) ? (int)(D - r0) : NB;
  const int w = threadIdx.x >> 5, c = threadIdx.x & 31;
  __shared__ V col[2][NB];   // column j of L (step j)
  __shared__ V xrow[2][NB];  // row k of X (inverse step k)
  __shared__ V rdiag[NB];    // 1 / L_kk
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  V a[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i = w + 8 * q;
    a[q] = (i < nb && c < nb) ? Mode::ld(H, off + (r0 + i) * D + r0 + c) : (i == c ? Mode::from_d(1.0) : Mode::zero());
  }
  // Cholesky: column j
  for (int j = 0; j < NB; ++j) {
    V* cj = col[j & 1];
    if (c == j) {
#pragma unroll
      for (int q = 0; q < 4; ++q) cj[w + 8 * q] = a[q];
    }
    __syncthreads();
    V piv = cj[j];
    if (!(Mode::to_d(piv) > 0.0)) {
      if (threadIdx.x == 0 && j < nb) bad = (Mode::to_d(piv) != Mode::to_d(piv)) ? DEV_NAN : DEV_NOT_SPD;
      piv = Mode::from_d(1.0);
    }
    const V d = Mode::sqrt_(piv);
    const V rinv = Mode::div(Mode::from_d(1.0), d);
    if (threadIdx.x == 0) rdiag[j] = rinv;
    const V lc = Mode::mul(cj[c], rinv);  // L[c][j] for c > j
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = w + 8 * q;
      if (c == j) {
        a[q] = i > j ? Mode::mul(a[q], rinv) : (i == j ? d : a[q]);
      } else if (c > j && i >= c) {
        a[q] = Mode::sub(a[q], Mode::mul(Mode::mul(cj[i], rinv), lc));
      }
    }
  }
  // X = L^-1 (column sweep), X lower triangular; x starts as the identity
  V x[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) x[q] = (w + 8 * q == c) ? Mode::from_d(1.0) : Mode::zero();
  __syncthreads();  // rdiag complete
  for (int k = 0; k < NB; ++k) {
    V* xr = xrow[k & 1];
    V* lk = col[k & 1];
    if (w == (k & 7)) xr[c] = Mode::mul(x[k >> 3], rdiag[k]);  // row k of X, final
    if (c == k) {
#pragma unroll
      for (int q = 0; q < 4; ++q) lk[w + 8 * q] = a[q];           // column k of L
    }
    __syncthreads();
    const V xk = xr[c];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = w + 8 * q;
      if (i == k) x[q] = xk;
      else if (i > k) x[q] = Mode::sub(x[q], Mode::mul(lk[i], xk));
    }
  }
  const int64_t dbase = ((int64_t)l * ((D + NB - 1) / NB) + kb) * NB * NB;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i = w + 8 * q;
    const bool in = i < nb && c < nb;
    if (in) Mode::st(H, off + (r0 + i) * D + r0 + c, c <= i ? a[q] : Mode::zero());
    Mode::st(dinv, dbase + i * NB + c, (in && c <= i) ? x[q] : Mode::zero());
  }
  if (threadIdx.x == 0 && bad) dev_fail(status, bad);
}

// panel rows below the diagonal block: L[i, kb] = H[i, kb] * Linv_kk^T  (in place)
template <class Mode>
struct LdPanel {
  using T = typename Mode::V;
  static constexpr bool k_contig = true;
  CBuf H;
  int64_t D, r0, c0;
  __device__ __forceinline__ T operator()(int g, int64_t i, int64_t k) const {
    return Mode::ld(H, (int64_t)g * D * D + (r0 + i) * D + c0 + k);
  }
};
template <class Mode>
struct LdDinvT {  // operand (k, j) = Linv_kk[j][k]
  using T = typename Mode::V;
  static constexpr bool k_contig = true;
  CBuf dinv;
  int64_t nblk;
  int kb;
  __device__ __forceinline__ T operator()(int g, int64_t k, int64_t j) const {
    return Mode::ld(dinv, ((int64_t)g * nblk + kb) * NB * NB + j * NB + k);
  }
};
template <class Mode>
struct EpPanel {
  CBuf H;
  int64_t D, r0, c0;
  __device__ __forceinline__ void operator()(int g, int, int64_t i, int64_t j, typename Mode::V a) const {
    Mode::st(H, (int64_t)g * D * D + (r0 + i) * D + c0 + j, a);
  }
};
template <class Mode>
struct LdPanelT {  // operand (k, j) = L[r0 + j][c0 + k]
  using T = typename Mode::V;
  static constexpr bool k_contig = true;
  CBuf H;
  int64_t D, r0, c0;
  __device__ __forceinline__ T operator()(int g, int64_t k, int64_t j) const {
    return Mode::ld(H, (int64_t)g * D * D + (r0 + j) * D + c0 + k);
  }
};
template <class Mode>
struct EpTrailing {  // H[r0+i][r0+j] -= acc on the lower triangle
  CBuf H;
  int64_t D, r0;
  __device__ __forceinline__ void operator()(int g, int, int64_t i, int64_t j, typename Mode::V a) const {
    if (j > i) return;
    int64_t o = (int64_t)g * D * D + (r0 + i) * D + r0 + j;
    Mode::st(H, o, Mode::sub(Mode::ld(H, o), a));
  }
};

// ---- W = L^-1 by recursive doubling of the inverted diagonal blocks:
//   inv([A 0; B C]) = [A^-1 0; -C^-1 (B A^-1)  C^-1]
// Level s (block size s = 32, 64, ...): for every pair of s-blocks starting at r0 = 2 s p, the
// off-diagonal block W[r0+s:r0+2s, r0:r0+s] = -W_C (L_B W_A).  Groups are (interval, pair).
template <class Mode>
__global__ void k_wdiag(CBuf dinv, int64_t D, CBuf Wm) {  // W <- block diagonal of the 32x32 inverses, 0 elsewhere
  const int l = blockIdx.y;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= D * D) return;
  const int64_t i = e / D, j = e % D, nblk = (D + NB - 1) / NB;
  typename Mode::V v = Mode::zero();
  if (i / NB == j / NB) v = Mode::ld(dinv, ((int64_t)l * nblk + i / NB) * NB * NB + (i % NB) * NB + (j % NB));
  Mode::st(Wm, (int64_t)l * D * D + e, v);
}
template <class Mode>
struct LdPairB {  // operand (i, k) = L[r0 + s + i][r0 + k]  (the lower-left block B of the pair)
  using T = typename Mode::V;
  static constexpr bool k_contig = true;
  CBuf H;
  int64_t D, s;
  int npairs;
  __device__ __forceinline__ T operator()(int g, int64_t i, int64_t k) const {
    const int64_t l = g / npairs, r0 = 2 * s * (g % npairs);
    const int64_t r = r0 + s + i;
    return r < D ? Mode::ld(H, l * D * D + r * D + r0 + k) : Mode::zero();
  }
};
template <class Mode>
struct LdPairWA {  // operand (k, j) = W[r0 + k][r0 + j]  (the inverted upper-left block)
  using T = typename Mode::V;
  static constexpr bool k_contig = false;
  CBuf Wm;
  int64_t D, s;
  int npairs;
  __device__ __forceinline__ T operator()(int g, int64_t k, int64_t j) const {
    const int64_t l = g / npairs, r0 = 2 * s * (g % npairs);
    const int64_t r = r0 + k, c = r0 + j;
    return (r < D && c < D) ? Mode::ld(Wm, l * D * D + r * D + c) : Mode::zero();
  }
};
template <class Mode>
struct EpPairT {  // T[g][i][j] (s x s scratch per group)
  CBuf Tm;
  int64_t s;
  __device__ __forceinline__ void operator()(int g, int, int64_t i, int64_t j, typename Mode::V a) const {
    Mode::st(Tm, ((int64_t)g * s + i) * s + j, Mode::renorm(a));
  }
};
template <class Mode>
struct LdPairWC {  // operand (i, k) = W[r0 + s + i][r0 + s + k]  (the inverted lower-right block)
  using T = typename Mode::V;
  static constexpr bool k_contig = true;
  CBuf Wm;
  int64_t D, s;
  int npairs;
  __device__ __forceinline__ T operator()(int g, int64_t i, int64_t k) const {
    const int64_t l = g / npairs, r0 = 2 * s * (g % npairs);
    const int64_t r = r0 + s + i, c = r0 + s + k;
    return (r < D && c < D) ? Mode::ld(Wm, l * D * D + r * D + c) : Mode::zero();
  }
};
template <class Mode>
struct LdPairT {  // operand (k, j) = T[g][k][j]
  using T = typename Mode::V;
  static constexpr bool k_contig = false;
  CBuf Tm;
  int64_t s;
  __device__ __forceinline__ T operator()(int g, int64_t k, int64_t j) const {
    return Mode::ld(Tm, ((int64_t)g * s + k) * s + j);
  }
};
template <class Mode>
struct EpPairOff {  // W[r0 + s + i][r0 + j] = -acc
  CBuf Wm;
  int64_t D, s;
  int npairs;
  __device__ __forceinline__ void operator()(int g, int, int64_t i, int64_t j, typename Mode::V a) const {
    const int64_t l = g / npairs, r0 = 2 * s * (g % npairs);
    const int64_t r = r0 + s + i;
    if (r < D) Mode::st(Wm, l * D * D + r * D + r0 + j, Mode::neg_(Mode::renorm(a)));
  }
};

template <class Mode>
static cudaError_t trtri_doubling(ihsbin_problem* p, CBuf H, CBuf dinv, CBuf Wm, CBuf Tm, int L, int64_t smax,
                                  cudaStream_t st) {
  const int64_t D = p->A.D;
  {
    KTimer kt(p, K_TRTRI, st, 0, (double)L * D * D * 8);
    k_wdiag<Mode><<<dim3(nblocks(D * D, 256), L), 256, 0, st>>>(dinv, D, Wm);
    CK(cudaGetLastError());
  }
  for (int64_t s = NB; s < D && s < smax; s *= 2) {
    const int npairs = (int)((D + 2 * s - 1) / (2 * s));
    // pairs whose lower block starts beyond D contribute nothing (loaders return zeros, stores are skipped)
    const int groups = npairs * L;
    GemmShape s1{s, s, s, 0};
    {
      KTimer kt(p, K_TRTRI, st, 2.0 * groups * s * s * s / 2, (double)groups * s * s * 8 * 3);
      CK((launch_gemm<Mode, 64, 64, 16, 4, 4>(s1, groups, LdPairB<Mode>{H, D, s, npairs},
                                              LdPairWA<Mode>{Wm, D, s, npairs}, EpPairT<Mode>{Tm, s}, st)));
    }
    {
      KTimer kt(p, K_TRTRI, st, 2.0 * groups * s * s * s / 2, (double)groups * s * s * 8 * 3);
      CK((launch_gemm<Mode, 64, 64, 16, 4, 4>(s1, groups, LdPairWC<Mode>{Wm, D, s, npairs},
                                              LdPairT<Mode>{Tm, s}, EpPairOff<Mode>{Wm, D, s, npairs}, st)));
    }
  }
  return cudaSuccess;
}

template <class Mode>
struct LdWT {  // operand (i, k) = W[k][i] (zero above the diagonal)
  using T = typename Mode::V;
  static constexpr bool k_contig = false;
  CBuf Wm;
  int64_t D;
  __device__ __forceinline__ T operator()(int g, int64_t i, int64_t k) const {
    return Mode::ld(Wm, (int64_t)g * D * D + k * D + i);
  }
};
template <class Mode>
struct LdW {  // operand (k, j) = W[k][j]
  using T = typename Mode::V;
  static constexpr bool k_contig = false;
  CBuf Wm;
  int64_t D;
  __device__ __forceinline__ T operator()(int g, int64_t k, int64_t j) const {
    return Mode::ld(Wm, (int64_t)g * D * D + k * D + j);
  }
};

// ---- W = L^-1 with the tensor cores: doubling on CUDA cores up to the 128 x 128 diagonal blocks,
// then the block columns J (128 wide) from right to left, with R the rows below J:
//   W_RJ = -W_RR (L_RJ W_JJ),
// W_RR being complete when J is reached.  T = L_RJ W_JJ is a float-float contraction; W_RR T is
// an exact-slice product (rows of W_RR against the columns of T), W_RR lower triangular.
template <class Mode>
struct LdBlockB {  // operand (k, j) = M[g][r0 + k][c0 + j]
  using T = typename Mode::V;
  static constexpr bool k_contig = false;
  CBuf M;
  int64_t D, r0, c0;
  __device__ __forceinline__ T operator()(int g, int64_t k, int64_t j) const {
    return Mode::ld(M, (int64_t)g * D * D + (r0 + k) * D + c0 + j);
  }
};
template <class Mode>
struct EpStoreRowMajor {  // out[g * gs + i * ld + j]
  CBuf M;
  int64_t ld, gs;
  __device__ __forceinline__ void operator()(int g, int, int64_t i, int64_t j, typename Mode::V a) const {
    Mode::st(M, (int64_t)g * gs + i * ld + j, Mode::renorm(a));
  }
};
// W[g][R0 + i][J0 + j] = -(W_RR T)_ij from the exact split partials (M = |R| rows, N = 128 columns)
__global__ void k_oz_store_wblock(const long long* hi, const long long* lo, int S, int64_t M, int64_t N, int L,
                                  const int* ex, int64_t exg, const int* ey, int64_t eyg, int64_t D, int64_t R0,
                                  int64_t J0, CBuf W) {
  pdl_wait();  // launched with programmatic serialization
  pdl_trigger();
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)L * M * N) return;
  const int64_t i = e % M, j = (e / M) % N, g = e / (M * N);
  long long h = 0, w = 0;
  for (int s = 0; s < S; ++s) {
    h += hi[(int64_t)s * L * M * N + e];
    w += lo[(int64_t)s * L * M * N + e];
  }
  const dd v = oz_join(h, w, ex[g * exg + i], ey[g * eyg + j]);
  DD::st(W, g * D * D + (R0 + i) * D + J0 + j, dd_neg(v));
}

static cudaError_t trtri_sweep_slices(ihsbin_problem* p, CBuf H, CBuf Wm, cudaStream_t st) {
  const int64_t D = p->A.D, B = 128;
  const int L = p->plan.L;
  const int nbk = (int)((D + B - 1) / B);
  if (nbk < 2) return cudaSuccess;
  const int64_t nRmax = D - B;
  size_t hmax = 1;  // the largest split partials of any step
  for (int j = nbk - 2; j >= 0; --j) {
    const int64_t nR = D - (int64_t)(j + 1) * B;
    hmax = std::max(hmax, (size_t)oz_pick_split_mnk(nR, B, nR, L, 32, 16) * L * nR * B);
  }
  cudaError_t err = cudaSuccess;
  CBuf T = alloc_cbuf(p, IHSBIN_COMPUTE_F32X2, (size_t)L * nRmax * B, SCOPE_SCRATCH, &err);
  CK(err);
  __nv_bfloat16 *Xs = nullptr, *Ys = nullptr;
  int *ex = nullptr, *ey = nullptr;
  long long *hi = nullptr, *lo = nullptr;
  CK(prob_alloc(p, oz_vec_elems(nRmax, nRmax, 128) * 2 * L, (void**)&Xs, SCOPE_SCRATCH));
  CK(prob_alloc(p, oz_vec_exps(nRmax, 128) * 4 * L, (void**)&ex, SCOPE_SCRATCH));
  CK(prob_alloc(p, oz_vec_elems(B, nRmax, 32) * 2 * L, (void**)&Ys, SCOPE_SCRATCH));
  CK(prob_alloc(p, oz_vec_exps(B, 32) * 4 * L, (void**)&ey, SCOPE_SCRATCH));
  CK(prob_alloc(p, hmax * 8, (void**)&hi, SCOPE_SCRATCH));
  CK(prob_alloc(p, hmax * 8, (void**)&lo, SCOPE_SCRATCH));
  for (int j = nbk - 2; j >= 0; --j) {
    const int64_t J0 = (int64_t)j * B, R0 = J0 + B, nR = D - R0;
    {
      KTimer kt(p, K_TRTRI, st, 2.0 * L * nR * B * B, (double)L * (nR * B + B * B + nR * B) * 8);
      CK((launch_gemm<DD, 64, 64, 16, 4, 4>(GemmShape{nR, B, B, 0}, L, LdPanel<DD>{H, D, R0, J0},
                                            LdBlockB<DD>{Wm, D, J0, J0}, EpStoreRowMajor<DD>{T, B, nR * B}, st)));
    }
    {
      KTimer kt(p, K_INVERSE_SLICE, st, 0, (double)L * (nR * nR + nR * B) * 20);
      CK(oz_slice_vecs(Wm, D * D, R0 * D + R0, D, nR, nR, L, 128, Xs, ex, st));
      CK(oz_slice_matcols(T, B, nR, B, L, nR * B, 32, Ys, ey, st));
    }
    const int S = oz_pick_split_mnk(nR, B, nR, L, 32, 16);
    {
      OzGemm q;
      q.wmax = p->plan.slice_w;
      q.As = Xs; q.ea = ex; q.Bs = Ys; q.eb = ey;
      q.M = nR; q.N = B; q.K = nR; q.groups = L; q.NT = 32; q.ksplit = S;
      q.tri = OZ_TRI_LE_ROW;
      q.ohi = hi; q.olo = lo; q.status = p->status;
      if (S == 1) {  // W[R0 + i][J0 + j] = -(W_RR T)_ij written by the kernel's epilogue
        q.epi = OZ_EPI_STORE_NEG; q.out = Wm; q.out_ld = D; q.out_gs = D * D; q.out_r0 = R0; q.out_c0 = J0;
      }
      KTimer kt(p, K_TRTRI_TC, st, 2.0 * L * (nR * (nR + 1.0) / 2.0) * B, (double)L * (nR * nR / 2.0 + 2.0 * nR * B) * 8,
                oz_pair_flops(1, 1, 1, p->plan.slice_w) * L * (nR * (nR + 1.0) / 2.0) * B,
                (double)L * (oz_vec_elems(nR, nR, 128) + oz_vec_elems(B, nR, 32)) * 2 + 16.0 * S * L * nR * B);
      CK(oz_gemm(q, st));
    }
    if (S > 1) {
      KTimer kt(p, K_INVERSE_SLICE, st, 0, (double)L * nR * B * (16.0 * S + 8));
      CK(launch_pdl(k_oz_store_wblock, dim3(nblocks((int64_t)L * nR * B, 256)), dim3(256), 0, st, hi, lo, S, nR, B, L,
                    ex, (int64_t)oz_vec_exps(nR, 128), ey, (int64_t)oz_vec_exps(B, 32), D, R0, J0, Wm));
    }
  }
  return cudaSuccess;
}

// ---- Two-level Cholesky: within a 128-wide panel the 32-wide steps update only the panel's
// columns; at the panel's end the trailing matrix takes the delayed rank-128 update
//   H[c1:, c1:] -= L_p L_p^T,  L_p = L[c1:, c0:c1],
// as an exact-slice product on the tensor cores (symmetric: tiles touching i <= j).  Its exact
// partials are subtracted by a separate pass at full occupancy: a read-modify-write of H in the
// product's epilogue (8 warps per SM) took longer than the product itself.
__global__ void k_oz_sub_sym(const long long* hi, const long long* lo, int S, int64_t M, int L, const int* ea,
                             int64_t eag, const int* eb, int64_t ebg, int64_t D, int64_t c1, CBuf H) {
  pdl_wait();  // launched with programmatic serialization
  pdl_trigger();
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)L * M * M) return;
  const int64_t i = e % M, j = (e / M) % M, g = e / (M * M);
  if (i > j) return;
  long long h = 0, w = 0;
  for (int s = 0; s < S; ++s) {
    h += hi[(int64_t)s * L * M * M + e];
    w += lo[(int64_t)s * L * M * M + e];
  }
  const dd v = oz_join(h, w, ea[g * eag + i], eb[g * ebg + j]);
  const int64_t o = g * D * D + (c1 + j) * D + c1 + i;  // the lower-triangle entry (c1 + j, c1 + i)
  DD::st(H, o, dd_sub(DD::ld(H, o), v));
}

struct PanelUpdate {
  __nv_bfloat16 *Xs = nullptr, *Ys = nullptr;
  int *ea = nullptr, *eb = nullptr;
  long long *hi = nullptr, *lo = nullptr;
};
static cudaError_t panel_update_alloc(ihsbin_problem* p, PanelUpdate& u) {
  const int64_t D = p->A.D, M = D > 128 ? D - 128 : 1;
  const int L = p->plan.L;
  CK(prob_alloc(p, oz_vec_elems(M, 128, 128) * 2 * L, (void**)&u.Xs, SCOPE_SCRATCH));
  CK(prob_alloc(p, oz_vec_exps(M, 128) * 4 * L, (void**)&u.ea, SCOPE_SCRATCH));
  CK(prob_alloc(p, oz_vec_elems(M, 128, 32) * 2 * L, (void**)&u.Ys, SCOPE_SCRATCH));
  CK(prob_alloc(p, oz_vec_exps(M, 32) * 4 * L, (void**)&u.eb, SCOPE_SCRATCH));
  CK(prob_alloc(p, (size_t)L * M * M * 8, (void**)&u.hi, SCOPE_SCRATCH));
  CK(prob_alloc(p, (size_t)L * M * M * 8, (void**)&u.lo, SCOPE_SCRATCH));
  return cudaSuccess;
}
static cudaError_t panel_update(ihsbin_problem* p, CBuf H, const PanelUpdate& u, int64_t c0, int64_t c1,
                                cudaStream_t st) {
  const int64_t D = p->A.D, M = D - c1, w = c1 - c0;
  const int L = p->plan.L;
  {
    KTimer kt(p, K_INVERSE_SLICE, st, 0, (double)L * M * w * 8 * 2 + (double)L * (oz_vec_elems(M, w, 128) + oz_vec_elems(M, w, 32)) * 2);
    CK(oz_slice_vecs(H, D * D, c1 * D + c0, D, w, M, L, 128, u.Xs, u.ea, st));
    CK(oz_slice_vecs(H, D * D, c1 * D + c0, D, w, M, L, 32, u.Ys, u.eb, st));
  }
  {
    OzGemm q;
    q.wmax = p->plan.slice_w;
    q.As = u.Xs; q.ea = u.ea; q.Bs = u.Ys; q.eb = u.eb;
    q.M = M; q.N = M; q.K = w; q.groups = L; q.NT = 32; q.ksplit = 1; q.sym = 1;
    q.ohi = u.hi; q.olo = u.lo; q.status = p->status;
    KTimer kt(p, K_SYRK_TC, st, 2.0 * L * (M * (M + 1.0) / 2.0) * w, (double)L * (M * w + M * (M + 1.0) / 2.0) * 8,
              oz_pair_flops(1, 1, 1, p->plan.slice_w) * L * (M * (M + 1.0) / 2.0) * w,
              (double)L * (oz_vec_elems(M, w, 128) + oz_vec_elems(M, w, 32)) * 2 + 16.0 * L * M * M);
    CK(oz_gemm(q, st));
  }
  KTimer kt(p, K_INVERSE_SLICE, st, 0, (double)L * M * M * (16.0 + 16.0));
  return launch_pdl(k_oz_sub_sym, dim3(nblocks((int64_t)L * M * M, 256)), dim3(256), 0, st, u.hi, u.lo, 1, M, L, u.ea,
                    (int64_t)oz_vec_exps(M, 128), u.eb, (int64_t)oz_vec_exps(M, 32), D, c1, H);
}

// P_l = W_l^T W_l on the tensor cores: X = Y = W_l^T (vectors = the columns of W_l), k >= max(i, j)
static cudaError_t inverse_slices(ihsbin_problem* p, CBuf Wm, cudaStream_t st) {
  const int64_t D = p->A.D;
  const int L = p->plan.L;
  __nv_bfloat16 *As = nullptr, *Bs = nullptr;
  int *ea = nullptr, *eb = nullptr;
  CK(prob_alloc(p, oz_vec_elems(D, D, 128) * 2 * L, (void**)&As, SCOPE_SCRATCH));
  CK(prob_alloc(p, oz_vec_exps(D, 128) * 4 * L, (void**)&ea, SCOPE_SCRATCH));
  CK(prob_alloc(p, oz_vec_elems(D, D, 32) * 2 * L, (void**)&Bs, SCOPE_SCRATCH));
  CK(prob_alloc(p, oz_vec_exps(D, 32) * 4 * L, (void**)&eb, SCOPE_SCRATCH));
  {
    KTimer kt(p, K_INVERSE_SLICE, st, 0, (double)L * D * D * 8 * 2 + (double)L * (oz_vec_elems(D, D, 128) + oz_vec_elems(D, D, 32)) * 2);
    CK(oz_slice_matcols(Wm, D, D, D, L, D * D, 128, As, ea, st));
    CK(oz_slice_matcols(Wm, D, D, D, L, D * D, 32, Bs, eb, st));
  }
  OzGemm q;
  q.wmax = p->plan.slice_w;
  q.As = As; q.ea = ea; q.Bs = Bs; q.eb = eb;
  q.M = D; q.N = D; q.K = D; q.groups = L; q.NT = 32; q.ksplit = 1;
  q.tri = OZ_TRI_GE_ROW | OZ_TRI_GE_COL;
  q.sym = 1;
  q.status = p->status;
  // P_l[i][j] = P_l[j][i] written by the kernel's epilogue
  q.epi = OZ_EPI_STORE_SYM; q.out = p->Pinv; q.out_ld = D; q.out_gs = D * D;
  KTimer kt(p, K_INVERSE_TC, st, (double)L * D * (D + 1.0) * (D + 2.0) / 3.0, (double)L * D * D * 8,
            oz_pair_flops(1, 1, 1, p->plan.slice_w) / 2.0 * L * D * (D + 1.0) * (D + 2.0) / 3.0,
            (double)L * (oz_vec_elems(D, D, 128) + oz_vec_elems(D, D, 32)) * 2 + (double)L * D * D * 16);
  return oz_gemm(q, st);
}

template <class Mode>
static cudaError_t factor_and_invert(ihsbin_problem* p, CBuf H, CBuf Wm, CBuf dinv, const double* lam0_dev,
                                     cudaStream_t st) {
  const int64_t D = p->A.D;
  const int L = p->plan.L;
  const int64_t nblk = (D + NB - 1) / NB;
  const double cs = Mode::id == 0 ? 8 : 8;  // bytes per compute-precision element (double or two floats)
  {
    KTimer kt(p, K_FACTOR_SHIFT, st, 0, (double)D * D * (8 + cs * L));
    k_shift_copy<Mode><<<dim3(nblocks(D * D, 256), L), 256, 0, st>>>(p->GS, D, lam0_dev, H);
  }
  CK(cudaGetLastError());
  const bool two_level = Mode::id == 1 && p->plan.factor == IHSBIN_FACTOR_SLICES && D > 128;
  PanelUpdate pu;
  if (two_level) CK(panel_update_alloc(p, pu));
  for (int kb = 0; kb < nblk; ++kb) {
    {
      KTimer kt(p, K_FACTOR_POTRF, st, (double)L * NB * NB * NB * 2.0 / 3.0, (double)L * NB * NB * cs * 3);
      CK(launch_pdl(k_potrf_diag_reg<Mode>, dim3(L), dim3(256), 0, st, H, D, kb, dinv, p->status));
    }
    CK(cudaGetLastError());
    const int64_t r0 = (int64_t)(kb + 1) * NB;
    if (r0 >= D) break;
    const int64_t rem = D - r0;
    const int64_t c0 = (int64_t)kb * NB;
    GemmShape sp{rem, NB, NB, 0};
    {
      KTimer kt(p, K_FACTOR_TRSM, st, 2.0 * L * rem * NB * NB, (double)L * rem * NB * cs * 2);
      CK((launch_gemm<Mode, 64, 32, 16, 4, 2>(sp, L, LdPanel<Mode>{H, D, r0, c0}, LdDinvT<Mode>{dinv, nblk, kb},
                                              EpPanel<Mode>{H, D, r0, c0}, st)));
    }
    // two-level: the 32-wide step updates only the columns of its 128-wide panel
    const int64_t pend = two_level ? std::min<int64_t>(D, (int64_t)(kb / 4 + 1) * 128) : D;
    const int64_t wcols = pend - r0;
    if (wcols > 0) {
      GemmShape su{rem, wcols, NB, 2};
      KTimer kt(p, K_FACTOR_SYRK, st, (double)L * wcols * (2.0 * rem - wcols + 1) * NB, (double)L * rem * wcols * cs);
      CK((launch_gemm<Mode, 64, 64, 16, 4, 4>(su, L, LdPanel<Mode>{H, D, r0, c0}, LdPanelT<Mode>{H, D, r0, c0},
                                              EpTrailing<Mode>{H, D, r0}, st)));
    }
    if (two_level && (kb % 4 == 3 || kb == nblk - 1) && pend < D)
      CK(panel_update(p, H, pu, (int64_t)(kb / 4) * 128, pend, st));
  }
  {
    cudaError_t err = cudaSuccess;
    size_t tmax = 1;  // the largest per-level scratch: (pairs x s x s) per interval
    for (int64_t sz = NB; sz < D; sz *= 2) tmax = std::max(tmax, (size_t)((D + 2 * sz - 1) / (2 * sz)) * sz * sz);
    CBuf Tm = alloc_cbuf(p, Mode::id == 0 ? IHSBIN_COMPUTE_F64 : IHSBIN_COMPUTE_F32X2, (size_t)L * tmax,
                         SCOPE_SCRATCH, &err);
    CK(err);
    const bool sweep = Mode::id == 1 && p->plan.factor == IHSBIN_FACTOR_SLICES;
    CK(trtri_doubling<Mode>(p, H, dinv, Wm, Tm, L, sweep ? 128 : D, st));
    if (sweep) CK(trtri_sweep_slices(p, H, Wm, st));
  }
  // P_l = W^T W  (W lower triangular: the sum starts at k = max(i, j))
  if (Mode::id == 1 && p->plan.factor == IHSBIN_FACTOR_SLICES) return inverse_slices(p, Wm, st);
  GemmShape sh{D, D, D, 1};
  sh.kdiag = 1;
  KTimer kt(p, K_INVERSE, st, (double)L * D * (D + 1) * (D + 2) / 3.0, (double)L * D * D * cs * 2);
  return launch_gemm<Mode, 64, 64, 16, 4, 4>(sh, L, LdWT<Mode>{Wm, D}, LdW<Mode>{Wm, D},
                                             EpStoreSym<Mode>{p->Pinv, D, D * D}, st);
}

// tr(P_l) for every interval (one CTA each), for the effective dimension of the sketch
template <class Mode>
__global__ void k_trace(CBuf Pm, int64_t D, double* out) {
  __shared__ double part[256];
  const int l = blockIdx.x;
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < D; i += blockDim.x) s += Mode::to_d(Mode::ld(Pm, (int64_t)l * D * D + i * D + i));
  part[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[l] = part[0];
}

// ============================================================ a3: Gram and rhs
template <class Mode, int ET>
static cudaError_t gram_dense(ihsbin_problem* p, cudaStream_t st) {
  const Tall& A = p->A;
  const int64_t D = A.D, tm = (D + 63) / 64;
  GemmShape sh{D, D, A.N, 1};
  sh.ksplit = pick_split(tm * (tm + 1) / 2, A.N, 16);
  KTimer kt(p, K_GRAM, st, (double)A.N * D * (D + 1), (double)A.N * D * (ET == ELEM_F64 ? 8 : ET == ELEM_F32 ? 4 : 2));
  if (sh.ksplit == 1)
    return launch_gemm<Mode, 64, 64, 16, 4, 4>(sh, 1, LdTrans<Mode, ET>{A.A, A.ld}, LdRowB<Mode, ET>{A.A, A.ld},
                                               EpStoreSym<Mode>{p->G, D, 0}, st);
  cudaError_t err = cudaSuccess;
  CBuf part = alloc_cbuf(p, Mode::id == 0 ? IHSBIN_COMPUTE_F64 : IHSBIN_COMPUTE_F32X2, (size_t)sh.ksplit * D * D,
                         SCOPE_SCRATCH, &err);
  CK(err);
  CK((launch_gemm<Mode, 64, 64, 16, 4, 4>(sh, 1, LdTrans<Mode, ET>{A.A, A.ld}, LdRowB<Mode, ET>{A.A, A.ld},
                                          EpPartial<Mode>{part, D, D, 1}, st)));
  k_reduce_sym<Mode><<<nblocks(D * D, 256), 256, 0, st>>>(part, sh.ksplit, D, p->G);
  return cudaGetLastError();
}

template <class Mode>
struct LdBcol {  // B (n x K, FP64 row-major) as the B operand: (k, j) = B[k][j]
  using T = typename Mode::V;
  static constexpr bool k_contig = false;
  const double* B;
  int64_t K;
  __device__ __forceinline__ T operator()(int, int64_t k, int64_t j) const { return Mode::from_d(B[k * K + j]); }
};

template <class Mode>
__global__ void k_copy_B_colmajor(const double* B, int64_t n, int64_t K, CBuf c) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * K) return;
  int64_t i = e / K, r = e % K;
  Mode::st(c, r * n + i, Mode::from_d(B[e]));
}

template <class Mode, int ET>
static cudaError_t rhs_dense(ihsbin_problem* p, CBuf c, cudaStream_t st) {
  const Tall& A = p->A;
  const int64_t D = A.D, K = p->K;
  GemmShape sh{D, K, A.N, 0};
  sh.ksplit = pick_split(((D + 63) / 64) * ((K + tile_n(K) - 1) / tile_n(K)), A.N, tile_k(K));
  KTimer kt(p, K_RHS, st, 2.0 * A.N * D * K, (double)A.N * D * (ET == ELEM_F64 ? 8 : ET == ELEM_F32 ? 4 : 2));
  if (sh.ksplit == 1)
    return launch_gemm_n<Mode>(sh, 1, LdTrans<Mode, ET>{A.A, A.ld}, LdBcol<Mode>{p->B, K},
                               EpStoreColMajor<Mode>{c, D, 0, nullptr}, st);
  cudaError_t err = cudaSuccess;
  CBuf part = alloc_cbuf(p, Mode::id == 0 ? IHSBIN_COMPUTE_F64 : IHSBIN_COMPUTE_F32X2, (size_t)sh.ksplit * D * K,
                         SCOPE_SCRATCH, &err);
  CK(err);
  CK((launch_gemm_n<Mode>(sh, 1, LdTrans<Mode, ET>{A.A, A.ld}, LdBcol<Mode>{p->B, K}, EpPartial<Mode>{part, D, K, 1},
                          st)));
  k_reduce_cols<Mode><<<nblocks(D * K, 256), 256, 0, st>>>(part, sh.ksplit, D, K, c);
  return cudaGetLastError();
}

// ===================================================== a4: the basis recursion
// Per-interval state: U (ping-pong), Ut (the accumulated basis), Y = A^T A U;
// column (j, r) of interval l lives at offset (l * jc * K + j * K + r) * D.
template <class Mode>
struct EpInit {  // u_00 = P c: write U0 and Ut
  CBuf U, Ut;
  int64_t D, gs;
  const int* perm;
  __device__ __forceinline__ void operator()(int g, int, int64_t i, int64_t j, typename Mode::V a) const {
    int64_t o = (int64_t)perm[g] * gs + j * D + i;
    a = Mode::renorm(a);
    Mode::st(U, o, a);
    Mode::st(Ut, o, a);
  }
};

// B operand of the preconditioner product: column (j, r) of
//   R = tau (Y_j + lam0 u_j) + lam0 u_{j-1}   (j < i; no shift term for j = 0)
//   R = lam0 u_{i-1}                          (j = i, the new column)
template <class Mode>
struct LdR {
  using T = typename Mode::V;
  static constexpr bool k_contig = true;
  CBuf U, Y;
  int64_t D, K, gs, ys;   // ys: per-group stride of Y; the ny splits of Y are ny_stride apart
  int i;
  const int* perm;
  const double* tau;
  const double* lam0;
  int ny;
  int64_t ny_stride;
  __device__ __forceinline__ T operator()(int g, int64_t k, int64_t col) const {
    const int l = perm[g];
    const int64_t j = col / K;
    const int64_t o = (int64_t)l * gs + col * D + k;
    const T lm = Mode::from_d(lam0[l]);
    if (j == i) return Mode::mul(lm, Mode::ld(U, o - K * D));
    T u = Mode::ld(U, o);
    const int64_t yo = (int64_t)g * ys + col * D + k;
    T y = Mode::ld(Y, yo);
#pragma unroll 4
    for (int s = 1; s < ny; ++s) y = Mode::add(y, Mode::ld(Y, s * ny_stride + yo));
    T r = Mode::mul(Mode::from_d(tau[l]), Mode::add(y, Mode::mul(lm, u)));
    if (j > 0) r = Mode::add(r, Mode::mul(lm, Mode::ld(U, o - K * D)));
    return r;
  }
};
template <class Mode>
struct EpUpdate {  // u_j <- u_j - P R_j (new column: u_i = -P R_i); utilde_j += u_j
  CBuf Uin, Uout, Ut;
  int64_t D, K, gs;
  int i;
  const int* perm;
  __device__ __forceinline__ void operator()(int g, int, int64_t row, int64_t col, typename Mode::V a) const {
    const int64_t o = (int64_t)perm[g] * gs + col * D + row;
    const int64_t j = col / K;
    typename Mode::V u = (j < i) ? Mode::ld(Uin, o) : Mode::zero();
    u = Mode::sub(u, Mode::renorm(a));
    Mode::st(Uout, o, u);
    Mode::st(Ut, o, Mode::add(Mode::ld(Ut, o), u));
  }
};
// The preconditioner's right-hand sides of one step, once per element:
//   R_j = tau (sum_s Y_s,j + lam0 u_j) + lam0 u_{j-1}   (j < i; no shift term for j = 0)
//   R_i = lam0 u_{i-1}                                 (the new column, when i < jmax)
template <class Mode>
__global__ void k_make_R(CBuf Y, int ny, int64_t ny_stride, CBuf U, int live, int64_t nold, int64_t nnew, int64_t D,
                         int64_t K, int inew, const int* perm, const double* tau, const double* lam0, int64_t gs,
                         CBuf R) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)live * nnew * D) return;
  const int g = (int)(e / (nnew * D));
  const int64_t col = (e / D) % nnew, k = e % D;
  const int l = perm[g];
  const int64_t j = col / K;
  const int64_t o = (int64_t)l * gs + col * D + k;
  const typename Mode::V lm = Mode::from_d(lam0[l]);
  typename Mode::V r;
  if (j == inew) {
    r = Mode::mul(lm, Mode::ld(U, o - K * D));
  } else {
    const int64_t yo = ((int64_t)g * nold + col) * D + k;
    typename Mode::V y = Mode::ld(Y, yo);
#pragma unroll 4
    for (int s = 1; s < ny; ++s) y = Mode::add(y, Mode::ld(Y, s * ny_stride + yo));
    r = Mode::mul(Mode::from_d(tau[l]), Mode::add(y, Mode::mul(lm, Mode::ld(U, o))));
    if (j > 0) r = Mode::add(r, Mode::mul(lm, Mode::ld(U, o - K * D)));
  }
  Mode::st(R, e, r);
}

// u_j <- u_j - sum_s Z_s (new column: -sum_s Z_s); utilde_j += u_j, from split partials of P R
template <class Mode>
__global__ void k_update(CBuf Z, int S, int live, int64_t ncol, int64_t D, int64_t K, int i, CBuf Uin, CBuf Uout,
                         CBuf Ut, const int* perm, int64_t gs) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)live * ncol * D) return;
  const int g = (int)(e / (ncol * D));
  const int64_t col = (e / D) % ncol, row = e % D;
  const int64_t zo = ((int64_t)g * ncol + col) * D + row;
  typename Mode::V z = Mode::ld(Z, zo);
#pragma unroll 4
  for (int s = 1; s < S; ++s) z = Mode::add(z, Mode::ld(Z, (int64_t)s * live * ncol * D + zo));
  const int64_t o = (int64_t)perm[g] * gs + col * D + row;
  const int64_t j = col / K;
  typename Mode::V u = (j < i) ? Mode::ld(Uin, o) : Mode::zero();
  u = Mode::sub(u, z);
  Mode::st(Uout, o, u);
  Mode::st(Ut, o, Mode::add(Mode::ld(Ut, o), u));
}

// The same two kernels when the products ran on the tensor cores (tc_loop.cu): a product entry
// is the sum over the k-splits of two exact int64 partials, joined into float-float with its
// row exponent (G, or P_l) and column exponent (U, or R) -- oz_join in common.cuh.
__global__ void k_make_R_oz(const long long* Yhi, const long long* Ylo, int ny, int64_t ny_stride, const int* eg,
                            const int* eu, CBuf U, int live, int64_t nold, int64_t nnew, int64_t D, int64_t K, int inew,
                            const int* perm, const double* tau, const double* lam0, int64_t gs, CBuf R) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)live * nnew * D) return;
  const int g = (int)(e / (nnew * D));
  const int64_t col = (e / D) % nnew, k = e % D;
  const int l = perm[g];
  const int64_t j = col / K;
  const int64_t o = (int64_t)l * gs + col * D + k;
  const dd lm = dd_from_double(lam0[l]);
  dd r;
  if (j == inew) {
    r = dd_mul(lm, DD::ld(U, o - K * D));
  } else {
    const int64_t c = (int64_t)g * nold + col, yo = c * D + k;
    long long h = Yhi[yo], lo = Ylo[yo];
    for (int s = 1; s < ny; ++s) {
      h += Yhi[s * ny_stride + yo];
      lo += Ylo[s * ny_stride + yo];
    }
    const dd y = oz_join(h, lo, eg[k], eu[c]);
    r = dd_mul(dd_from_double(tau[l]), dd_add(y, dd_mul(lm, DD::ld(U, o))));
    if (j > 0) r = dd_add(r, dd_mul(lm, DD::ld(U, o - K * D)));
  }
  DD::st(R, e, r);
}
__global__ void k_update_oz(const long long* Zhi, const long long* Zlo, int S, const int* ep, int64_t ep_gs,
                            const int* er, int64_t er_gs, int live, int64_t ncol, int64_t D, int64_t K, int i,
                            CBuf Uin, CBuf Uout, CBuf Ut, const int* perm, int64_t gs) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)live * ncol * D) return;
  const int g = (int)(e / (ncol * D));
  const int64_t col = (e / D) % ncol, row = e % D;
  const int64_t zo = ((int64_t)g * ncol + col) * D + row, ss = (int64_t)live * ncol * D;
  long long h = Zhi[zo], lo = Zlo[zo];
  for (int s = 1; s < S; ++s) {
    h += Zhi[s * ss + zo];
    lo += Zlo[s * ss + zo];
  }
  const dd z = oz_join(h, lo, ep[(int64_t)perm[g] * ep_gs + row], er[(int64_t)g * er_gs + col]);
  const int64_t o = (int64_t)perm[g] * gs + col * D + row;
  const int64_t j = col / K;
  dd u = (j < i) ? DD::ld(Uin, o) : DD::zero();
  u = dd_sub(u, z);
  DD::st(Uout, o, u);
  DD::st(Ut, o, dd_add(DD::ld(Ut, o), u));
}

// Y = A^T A U for the Gram product: the B operand is U (column j, contiguous over k)
template <class Mode>
struct EpY {
  CBuf Y;
  int64_t D, ys;
  __device__ __forceinline__ void operator()(int g, int, int64_t i, int64_t col, typename Mode::V a) const {
    Mode::st(Y, (int64_t)g * ys + col * D + i, Mode::renorm(a));
  }
};

// A-space product, first half: W = A_hat U  (N x ncol per live interval)
template <class Mode, int ET>
struct LdAhatRow {  // operand (i, k) = A_hat[i][k]
  using T = typename ElemOp<Mode, ET>::T;
  static constexpr bool k_contig = true;
  const void* A;
  int64_t ld;
  __device__ __forceinline__ T operator()(int, int64_t i, int64_t k) const { return ElemOp<Mode, ET>::get(A, i * ld + k); }
};
template <class Mode>
struct LdWcol {  // operand (k, j) = Wtmp[g][j][k] (column-major, N rows)
  using T = typename Mode::V;
  static constexpr bool k_contig = true;
  CBuf Wt;
  int64_t N, ws;
  __device__ __forceinline__ T operator()(int g, int64_t k, int64_t j) const { return Mode::ld(Wt, (int64_t)g * ws + j * N + k); }
};

constexpr int SPLIT_MAX = 16;

// Tensor-core operands of the recursion's products (exact slices, tc_loop.cu)
struct OzLoop {
  bool on = false;
  const __nv_bfloat16* Gs = nullptr;  // the Gram, rows sliced (Gram product mode)
  const int* eg = nullptr;
  const __nv_bfloat16* Ps = nullptr;  // P_l of every interval, rows sliced
  const int* ep = nullptr;
  __nv_bfloat16* Bs = nullptr;        // the step's B operand, columns sliced
  int* eb = nullptr;                  // its column exponents (the step's U columns)
  int* er = nullptr;                  // column exponents of R (fused path)
  long long *Yhi = nullptr, *Ylo = nullptr, *Zhi = nullptr, *Zlo = nullptr;  // exact split partials
  // two-product form of the recursion (from step mform_from on): M_q = P_l (G + lam0_l I) for the
  // intervals order[0 .. Tm-1], rows sliced; column exponents alternate between eb and eb2
  int mform_from = 0;
  const __nv_bfloat16* Ms = nullptr;
  const int* em = nullptr;
  int* eb2 = nullptr;
  // residual form (fused path only): U aliases Ut, which holds the partial sums v; c enters the
  // j = 0 residual; P_l R keeps the slice pairs s + t <= pw
  bool resid = false;
  int pw = 6;
};

// tr(G_S) in FP64 (one CTA of 256 threads), for the residual form's pair-weight rule
__global__ void k_diag_sum(const double* M, int64_t D, double* out) {
  __shared__ double part[256];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < D; i += blockDim.x) s += M[i * D + i];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = part[0];
}

cudaError_t gs_trace_launch(ihsbin_problem* p, double* out, cudaStream_t st) {
  k_diag_sum<<<1, 256, 0, st>>>(p->GS, p->A.D, out);
  return cudaGetLastError();
}

// The residual form's default pair weight for P_l r.  Dropping the pairs s + t > w makes each
// application of P_l wrong by about eps_w = 2^(-8(w+1)) of |P_l| |r| (relative to the row and
// column maxima), i.e. by up to kappa eps_w relative, kappa <= 1 + tr(G_S) / lam0 bounding the
// conditioning of the shifted sketched Hessian.  Two conditions on w:
//  (1) the iteration map I - tau P_l (G + lam0 I) changes by at most sqrt(D) kappa eps_w <= 2^-5,
//      so it keeps its contraction;
//  (2) the error carried to the end is no larger than the increment form's own: there step i's
//      error is damped by the later steps to about rate^(k-1-i) of it while |r_i| falls like
//      rate^i, so the k steps leave about g kappa eps_w of x, g = max_l k_l rate_l^(k_l - 1), with
//      rate Theorem 4's bound max(|1 - tau e_min|, |1 - tau e_max|) over the interval's spectrum
//      bounds e = rho2 (lo + s) / (lam0 + s) .. rho1 (hi + s) / (lam0 + s); the increment form keeps
//      every step's rounding of 2^-47 kappa (the slices hold each entry to 2^-47 of its row's
//      maximum), about k_max kappa 2^-47 in all.  So g eps_w <= k_max 2^-47.
// Returns the smallest such w in 2..5, or 6 when none qualifies.
static int precond_weight_rule(int64_t D, double trGS, const Plan& pl) {
  double lmin = pl.lam0[0], g = 0.0;
  for (int l = 0; l < pl.L; ++l) {
    lmin = std::min(lmin, pl.lam0[l]);
    const double s2 = pl.sigma_d2, lo = pl.edges[l], hi = pl.edges[l + 1];
    const double emin = pl.rho2[l] * (lo + s2) / (pl.lam0[l] + s2), emax = pl.rho1[l] * (hi + s2) / (pl.lam0[l] + s2);
    const double rate = std::max(std::fabs(1.0 - pl.tau[l] * emin), std::fabs(1.0 - pl.tau[l] * emax));
    g = std::max(g, pl.k[l] * std::pow(rate, pl.k[l] - 1));
  }
  const double kappa = 1.0 + trGS / lmin;
  for (int w = 2; w < 6; ++w) {
    const double ew = std::ldexp(1.0, -8 * (w + 1));
    if (std::sqrt((double)D) * kappa * ew <= std::ldexp(1.0, -5) && g * ew <= pl.kmax * std::ldexp(1.0, -47)) return w;
  }
  return 6;
}

template <class Mode, int ET>
static cudaError_t basis_loop(ihsbin_problem* p, CBuf c, CBuf U0, CBuf U1, CBuf Y, CBuf Z, CBuf R, CBuf Wtmp,
                              const int* perm_dev,
                              const double* tau_dev, const double* lam0_dev, const std::vector<int>& order,
                              const OzLoop& oz, cudaStream_t st) {
  const Tall& A = p->A;
  const int64_t D = A.D, K = p->K;
  const Plan& pl = p->plan;
  const int64_t gs = (int64_t)pl.jc * K * D;  // per-interval stride of U / Ut
  const int L = pl.L;
  const int pw = oz.resid ? oz.pw : pl.slice_w;  // pair weight of the P_l R products
  if (oz.resid) {
    // v_0 = P_l c as a step of the residual form from v = 0 (R = -c, no product with G): the
    // tensor-core P_l r with pw's pairs, whose error the later steps remove like any other's;
    // the update cuts v_0 for the first G v
    int live0 = 0;
    while (live0 < L && pl.k[order[live0]] > 0) ++live0;
    const int live1 = pl.kmax > 1 ? [&] { int n = 0; while (n < L && pl.k[order[n]] > 1) ++n; return n; }() : 0;
    const int NT = oz_tile_n(K, pw);
    {
      KTimer kt(p, K_LOOP_P, st, 0, (double)live0 * K * D * (16.0 + 12));
      CK(oz_make_R_slice(oz.Yhi, oz.Ylo, 0, 0, oz.eg, oz.eb, p->Ut, live0, 0, K, D, K, -1, perm_dev, tau_dev,
                         lam0_dev, gs, NT, oz.Bs, oz.er, c, st));
    }
    const int ks = oz_pick_split(D, K, live0, NT, SPLIT_MAX);
    {
      const double fsl = (std::min(pw, 5) + 1) / 6.0;
      KTimer kt(p, K_LOOP_P_TC, st, 2.0 * D * D * K * live0, (double)live0 * D * D * 8 + 16.0 * D * K * live0,
                oz_pair_flops(D, K, D, pw) * live0,
                (double)live0 * (oz_rows_elems(D) * 2 + oz_cols_elems(D, K, NT) * 2) * fsl + 16.0 * ks * D * K * live0);
      CK(oz_product(oz.Ps, oz.ep, perm_dev, false, oz.Bs, oz.er, D, K, live0, NT, ks, oz.Zhi, oz.Zlo, p->status, st,
                    pw));
    }
    {
      KTimer kt(p, K_LOOP_P, st, 0, (double)live0 * K * D * (16.0 * ks + 24 + 12));
      CK(oz_update_slice(oz.Zhi, NT == 64 ? nullptr : oz.Zlo, ks, oz.ep, (int64_t)oz_rows_exps(D), oz.er,
                         (int64_t)oz_cols_exps(K, NT), live0, K, D, K, 0, U0, U1, p->Ut, perm_dev, gs, live1,
                         oz_tile_n((int64_t)K * std::max(live1, 1)), oz.Bs, oz.eb, 1, st));
    }
  } else {
    // u_00 = P_l c for every interval
    GemmShape sh{D, K, D, 0};
    KTimer kt(p, K_LOOP_P, st, 2.0 * D * D * K * L, (double)L * D * D * 8);
    CK((launch_gemm_n<Mode>(sh, L, LdCMatA<Mode>{p->Pinv, D, D * D, perm_dev},
                                            LdCColB<Mode>{c, D, 0, nullptr}, EpInit<Mode>{U0, p->Ut, D, gs, perm_dev},
                                            st)));
  }
  CBuf Uin = U0, Uout = U1;
  const int J = pl.jmax > 0 ? pl.jmax : (1 << 30);
  for (int i = 1; i < pl.kmax; ++i) {
    int live = 0;
    while (live < L && pl.k[order[live]] > i) ++live;
    if (live == 0) break;
    const int64_t nold = (int64_t)std::min(i, J) * K;
    const int64_t nnew = (int64_t)std::min(i + 1, J) * K;
    const int64_t ys = nold * D;
    const int64_t mt = (D + 63) / 64;
    int live_next = 0;
    if (i + 1 < pl.kmax)
      while (live_next < L && pl.k[order[live_next]] > i + 1) ++live_next;
    if (oz.mform_from > 0 && i >= oz.mform_from) {
      // two-product form: [M_q U_q, P_l U_q] for every live interval in one launch, then the update
      // (ncol = nold = nnew = jmax K columns, tile height 16)
      const int64_t ncol = nold;
      const int ks = oz_pick_split(D, ncol, 2 * live, 16, SPLIT_MAX);
      const int parity = (i - oz.mform_from) & 1;
      int* eu_in = parity ? oz.eb2 : oz.eb;
      int* eu_out = parity ? oz.eb : oz.eb2;
      {
        OzGemm q;
        q.wmax = p->plan.slice_w;
        q.As = oz.Ms; q.As2 = oz.Ps; q.a_perm2 = perm_dev; q.pair = 1;
        q.Bs = oz.Bs;
        q.M = D; q.N = ncol; q.K = D; q.groups = 2 * live; q.NT = 16; q.ksplit = ks;
        q.ohi = oz.Zhi; q.olo = oz.Zlo; q.status = p->status;
        // the method's step: G U (G read once) and P_l R (each live P_l once); M_l is the implementation's
        KTimer kt(p, K_LOOP_P_TC, st, 4.0 * D * D * ncol * live, (double)(live + 1) * D * D * 8 + 16.0 * D * ncol * live,
                  2.0 * oz_pair_flops(D, ncol, D, pl.slice_w) * live,
                  (double)2 * live * (oz_rows_elems(D) * 2 + oz_cols_elems(D, ncol, 16) * 2) + 32.0 * ks * D * ncol * live);
        CK(oz_gemm(q, st));
      }
      {
        KTimer kt(p, K_LOOP_P, st, 0, (double)live * ncol * D * (32.0 * ks + 24 + 12));
        CK(oz_update_mw_slice(oz.Zhi, oz.Zlo, ks, oz.em, oz.ep, live, ncol, D, K, Uin, Uout, p->Ut, perm_dev, tau_dev,
                              lam0_dev, gs, eu_in, live_next, oz.Bs, eu_out, st));
      }
      std::swap(Uin, Uout);
      continue;
    }
    int ny = 1;
    const bool fused = oz.on && pl.product == IHSBIN_PRODUCT_GRAM && oz_fused_ok(D);
    if (pl.product == IHSBIN_PRODUCT_GRAM && oz.on) {
      // G times the concatenated old columns of every live interval, on the tensor cores (with the
      // fused path the previous step's update already sliced them)
      const int64_t ncat = nold * live;
      const int NT = oz_tile_n(ncat);
      if (!fused || (i == 1 && !oz.resid)) {  // (the residual form's first update cut v_0)
        KTimer kt(p, K_LOOP_SLICE, st, 0, 8.0 * D * ncat + 12.0 * D * ncat);
        CK(oz_slice_cols(Uin, D, 1, ncat, NT, nold, gs, perm_dev, oz.Bs, oz.eb, st));
      }
      ny = oz_pick_split(D, ncat, 1, NT, SPLIT_MAX);
      KTimer kt(p, K_LOOP_Y_TC, st, 2.0 * D * D * ncat, (double)D * D * 8 + 16.0 * D * ncat, oz_pair_flops(D, ncat, D, pl.slice_w),
                (double)oz_rows_elems(D) * 2 + (double)oz_cols_elems(D, ncat, NT) * 2 + 16.0 * ny * D * ncat);
      CK(oz_product(oz.Gs, oz.eg, nullptr, true, oz.Bs, oz.eb, D, ncat, 1, NT, ny, oz.Yhi, oz.Ylo, p->status, st,
                    pl.slice_w));
    } else if (pl.product == IHSBIN_PRODUCT_GRAM) {
      // every live interval multiplies the same G: one contraction over their concatenated columns
      const int64_t ncat = nold * live;
      GemmShape sh{D, ncat, D, 0};
      KTimer kt(p, K_LOOP_Y, st, 2.0 * D * D * ncat, (double)D * D * 8 + 16.0 * D * ncat);
      if (ncat > 32) {
        sh.ksplit = ny = std::min(pick_split(mt * ((ncat + 63) / 64), D, 16), SPLIT_MAX);
        CK((launch_gemm<Mode, 64, 64, 16, 4, 4>(sh, 1, LdCMatA<Mode>{p->G, D, 0, nullptr},
                                                LdUcat<Mode>{Uin, D, gs, nold, perm_dev},
                                                EpPartial<Mode>{Y, D, ncat, 1}, st)));
      } else {
        sh.ksplit = ny = std::min(pick_split(mt * ((ncat + tile_n(ncat) - 1) / tile_n(ncat)), D, tile_k(ncat)),
                                  SPLIT_MAX);
        CK((launch_gemm_n<Mode>(sh, 1, LdCMatA<Mode>{p->G, D, 0, nullptr}, LdUcat<Mode>{Uin, D, gs, nold, perm_dev},
                                EpPartial<Mode>{Y, D, ncat, 1}, st)));
      }
    } else {
      // W = A_hat U (N x nold), then Y = A_hat^T W
      const int64_t N = A.N;
      const double esz = ET == ELEM_F64 ? 8 : ET == ELEM_F32 ? 4 : 2;
      KTimer kt(p, K_LOOP_Y, st, 4.0 * N * D * nold * live, 2.0 * N * D * esz * live);
      GemmShape s1{N, nold, D, 0};
      CK((launch_gemm<Mode, 64, 32, 16, 4, 2>(s1, live, LdAhatRow<Mode, ET>{A.A, A.ld},
                                              LdCColB<Mode>{Uin, D, gs, perm_dev},
                                              EpStoreColMajor<Mode>{Wtmp, N, nold * N, nullptr}, st)));
      GemmShape s2{D, nold, N, 0};
      CK((launch_gemm<Mode, 64, 32, 16, 4, 2>(s2, live, LdTrans<Mode, ET>{A.A, A.ld},
                                              LdWcol<Mode>{Wtmp, N, nold * N}, EpY<Mode>{Y, D, ys}, st)));
    }
    GemmShape sp{D, nnew, D, 0};
    const int inew = (i < J) ? i : -1;
    sp.ksplit = std::min(pick_split(mt * ((nnew + tile_n(nnew) - 1) / tile_n(nnew)) * live, D, tile_k(nnew)),
                         SPLIT_MAX);
    if (fused) {
      KTimer kt(p, K_LOOP_P, st, 0, (double)live * nnew * D * (16.0 * ny + 24 + 12));
      CK(oz_make_R_slice(oz.Yhi, oz.Ylo, ny, (int64_t)live * ys, oz.eg, oz.eb, Uin, live, nold, nnew, D, K, inew,
                         perm_dev, tau_dev, lam0_dev, gs, oz_tile_n(nnew, pw), oz.Bs, oz.er, oz.resid ? c : CBuf{}, st));
    } else if (oz.on && pl.product == IHSBIN_PRODUCT_GRAM) {
      KTimer kt(p, K_LOOP_P, st, 0, (double)live * nnew * D * (16.0 * ny + 24));
      k_make_R_oz<<<nblocks((int64_t)live * nnew * D, 256), 256, 0, st>>>(
          oz.Yhi, oz.Ylo, ny, (int64_t)live * ys, oz.eg, oz.eb, Uin, live, nold, nnew, D, K, inew, perm_dev, tau_dev,
          lam0_dev, gs, R);
      CK(cudaGetLastError());
    } else {
      KTimer kt(p, K_LOOP_P, st, 0, (double)live * nnew * D * 8 * (ny + 3));
      k_make_R<Mode><<<nblocks((int64_t)live * nnew * D, 256), 256, 0, st>>>(
          Y, ny, (int64_t)live * ys, Uin, live, nold, nnew, D, K, inew, perm_dev, tau_dev, lam0_dev, gs, R);
      CK(cudaGetLastError());
    }
    if (oz.on) {
      // P_l R_l of every live interval, on the tensor cores
      const int NT = oz_tile_n(nnew, pw);
      int* erv = fused ? oz.er : oz.eb;  // column exponents of R
      if (!fused) {
        KTimer kt(p, K_LOOP_SLICE, st, 0, 20.0 * D * nnew * live);
        CK(oz_slice_cols(R, D, live, nnew, NT, nnew, nnew * D, nullptr, oz.Bs, oz.eb, st));
      }
      const int ks = oz_pick_split(D, nnew, live, NT, SPLIT_MAX);
      {
        // the residual form's P_l R keeps the pairs s + t <= pw and reads only the slices 0 .. pw
        const double fsl = (std::min(pw, 5) + 1) / 6.0;
        KTimer kt(p, K_LOOP_P_TC, st, 2.0 * D * D * nnew * live, (double)live * D * D * 8 + 16.0 * D * nnew * live,
                  oz_pair_flops(D, nnew, D, pw) * live,
                  (double)live * (oz_rows_elems(D) * 2 + oz_cols_elems(D, nnew, NT) * 2) * fsl + 16.0 * ks * D * nnew * live);
        CK(oz_product(oz.Ps, oz.ep, perm_dev, false, oz.Bs, erv, D, nnew, live, NT, ks, oz.Zhi, oz.Zlo, p->status,
                      st, pw));
      }
      if (fused) {
        // the intervals still running at the next step take their new columns' slices now
        // (tile height 16 when the next step takes the two-product form)
        const int NTn = (live_next > 0 && !(oz.mform_from > 0 && i + 1 >= oz.mform_from)) ? oz_tile_n(nnew * live_next)
                                                                                       : 16;
        KTimer kt(p, K_LOOP_P, st, 0, (double)live * nnew * D * (16.0 * ks + 24 + 12));
        CK(oz_update_slice(oz.Zhi, NT == 64 ? nullptr : oz.Zlo, ks, oz.ep, (int64_t)oz_rows_exps(D), oz.er,
                           (int64_t)oz_cols_exps(nnew, NT),
                           live, nnew, D, K, i, Uin, Uout, p->Ut, perm_dev, gs, live_next, NTn, oz.Bs, oz.eb,
                           oz.resid ? 1 : 0, st));
      } else {
        KTimer kt(p, K_LOOP_P, st, 0, (double)live * nnew * D * (16.0 * ks + 24));
        k_update_oz<<<nblocks((int64_t)live * nnew * D, 256), 256, 0, st>>>(
            oz.Zhi, oz.Zlo, ks, oz.ep, (int64_t)oz_rows_exps(D), oz.eb, (int64_t)oz_cols_exps(nnew, NT), live, nnew, D,
            K, i, Uin, Uout, p->Ut, perm_dev, gs);
        CK(cudaGetLastError());
      }
      std::swap(Uin, Uout);
      continue;
    }
    const LdCColB<Mode> ldr{R, D, nnew * D, nullptr};
    {
      KTimer kt(p, K_LOOP_P, st, 2.0 * D * D * nnew * live, (double)live * D * D * 8 + 32.0 * D * nnew * live);
      if (sp.ksplit == 1) {
        CK((launch_gemm_n<Mode>(sp, live, LdCMatA<Mode>{p->Pinv, D, D * D, perm_dev}, ldr,
                                EpUpdate<Mode>{Uin, Uout, p->Ut, D, K, gs, i, perm_dev}, st)));
      } else {
        CK((launch_gemm_n<Mode>(sp, live, LdCMatA<Mode>{p->Pinv, D, D * D, perm_dev}, ldr,
                                EpPartial<Mode>{Z, D, nnew, live}, st)));
      }
    }
    if (sp.ksplit > 1) {
      KTimer kt(p, K_LOOP_P, st, 0, (double)live * nnew * D * 8 * (sp.ksplit + 3));
      k_update<Mode><<<nblocks((int64_t)live * nnew * D, 256), 256, 0, st>>>(Z, sp.ksplit, live, nnew, D, K, i, Uin,
                                                                            Uout, p->Ut, perm_dev, gs);
      CK(cudaGetLastError());
    }
    std::swap(Uin, Uout);
  }
  return cudaSuccess;
}

// ===================================================== a6: path evaluation
// coefficient table coef[t][j] = tau_l theta_t^j (FP64), interval per lambda
// (the table is also written as float-float hi/lo when ch is not null, so that the evaluation's
// inner loop does no FP64 conversion)
__global__ void k_eval_coef(const double* lam, int64_t T, const double* edges, int L, const double* tau,
                            const double* lam0, const int* jcount, int jc, int* tint, double* coef, float* ch,
                            float* cl) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= T) return;
  double x = lam[t];
  // half-open [edge_l, edge_{l+1}), last interval closed
  int lo = 0, hi = L;  // find the largest l with edges[l] <= x
  while (hi - lo > 1) {
    int mid = (lo + hi) / 2;
    if (edges[mid] <= x) lo = mid; else hi = mid;
  }
  int l = lo;
  tint[t] = l;
  double th = tau[l] * (x - lam0[l]) / lam0[l];
  double cf = tau[l];
  for (int j = 0; j < jc; ++j) {
    const double v = (j < jcount[l]) ? cf : 0.0;
    coef[t * jc + j] = v;
    if (ch) {
      const float h = (float)v;
      ch[t * jc + j] = h;
      cl[t * jc + j] = (float)(v - (double)h);
    }
    cf *= th;
  }
}

// X[t][i][r] = sum_j coef[t][j] * B_l[j][r][i]   (B = utilde, or its primal image for the dual).
// Chunks of up to EVAL_TB lambdas of one interval: each basis entry is read once per chunk (not
// once per lambda) and applied to every lambda of the chunk.
constexpr int EVAL_TB = 16;
template <class Mode>
__global__ void k_eval_chunks(CBuf Bm, int64_t rows, int64_t K, int jc, int64_t gs, const int* chunk_l,
                              const int* chunk_t0, const int* chunk_n, const int* torder, CBuf coef,
                              const int* jcount, void* X, int x_elem) {
  const int c = blockIdx.y;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= rows * K) return;
  // X[t][i][r] is row-major with r fastest: for several right-hand sides consecutive threads take
  // consecutive r, so that the writes (the dominant traffic) coalesce; for K < 4, consecutive i
  const bool rfast = K >= 4;
  const int64_t r = rfast ? e % K : e / rows, i = rfast ? e / K : e % rows;
  const int l = chunk_l[c], nq = chunk_n[c], t0 = chunk_t0[c];
  const int jn = jcount[l];
  int tq[EVAL_TB];
  typename Mode::V acc[EVAL_TB];
#pragma unroll
  for (int q = 0; q < EVAL_TB; ++q) {
    tq[q] = q < nq ? torder[t0 + q] : 0;
    acc[q] = Mode::zero();
  }
  for (int j = 0; j < jn; ++j) {
    const typename Mode::V b = Mode::ld(Bm, (int64_t)l * gs + ((int64_t)j * K + r) * rows + i);
#pragma unroll
    for (int q = 0; q < EVAL_TB; ++q)
      if (q < nq) acc[q] = Mode::add(acc[q], Mode::mul(Mode::ld(coef, (int64_t)tq[q] * jc + j), b));
  }
#pragma unroll
  for (int q = 0; q < EVAL_TB; ++q) {
    if (q >= nq) break;
    const int64_t o = (int64_t)tq[q] * rows * K + i * K + r;
    const double v = Mode::to_d(acc[q]);
    if (x_elem == ELEM_F64) ((double*)X)[o] = v;
    else ((float*)X)[o] = (float)v;
  }
}

// ============================================================ orchestration
cudaError_t ensure_streams(ihsbin_problem* p) {
  // Stream priorities: the factorization's chain of small dependent launches is the critical
  // path, so its CTAs are scheduled first whenever SMs free up; the Gram's long tensor-core CTAs
  // (lowest priority) fill the rest.
  int prio_lo = 0, prio_hi = 0;
  CK(cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi));
  if (!p->side) CK(cudaStreamCreateWithPriority(&p->side, cudaStreamNonBlocking, prio_lo));
  if (!p->fac) CK(cudaStreamCreateWithPriority(&p->fac, cudaStreamNonBlocking, prio_hi));
  return cudaSuccess;
}

// ihsbin_sketch starts the Gram of A and A^T b (which do not depend on the sketch) on the side
// stream when the next build will most likely take them: dense FP32/BF16/TF32 data with the
// right-hand side formed from the Gram's slices (K >= 32, not the dual), the float-float compute
// mode with the sliced Gram (the defaults; or the last build's mode), and per-launch timing off
// (its events are read at the call's own synchronisation).  The draws of the sketch, an ALU load,
// then run beside the Gram's tensor-core work, and the build's factorization beside the rest.
bool pre_gram_eligible(const ihsbin_problem* p) {
  const Tall& A = p->A;
  return !p->timing && !p->pre_off && A.layout == IHSBIN_DENSE_ROWMAJOR && A.elem != ELEM_F64 && !p->dual &&
         p->K >= 32 &&
         (p->last_compute < 0 || (p->last_compute == IHSBIN_COMPUTE_F32X2 && p->last_gram == IHSBIN_GRAM_SLICES));
}

cudaError_t pre_gram_launch(ihsbin_problem* p) {
  CK(ensure_streams(p));
  cudaStream_t s2 = p->side;
  const int64_t D = p->A.D, K = p->K;
  for (auto& e : p->pre_ev)
    if (!e) CK(cudaEventCreate(&e));
  CK(cudaEventRecord(p->pre_ev[0], s2));
  // the SMs the Gram's launches leave free for the sketch and then the factorization beside it,
  // tuned on the time from here to the build's join (tune_end there)
  static const int cands[] = {40, 24, 64, 0};
  p->pre_tune = new TuneLaunch(
      tune_begin(tune_key(TUNE_PRE_RESERVE, D, shape_class(p->A.N), K), "pre_gram_reserve_sms", cands, 4, s2));
  cudaError_t err = cudaSuccess;
  p->G_pre = alloc_cbuf(p, IHSBIN_COMPUTE_F32X2, (size_t)D * D, SCOPE_PRE, &err);
  p->c_pre = alloc_cbuf(p, IHSBIN_COMPUTE_F32X2, (size_t)D * K, SCOPE_PRE, &err);
  CK(err);
  const CBuf G_keep = p->G;
  p->G = p->G_pre;
  err = gram_dense_slices(p, IHSBIN_COMPUTE_F32X2, s2, p->pre_tune->value, &p->c_pre);
  p->G = G_keep;
  CK(err);
  CK(cudaEventRecord(p->pre_ev[1], s2));
  p->gram_pre = true;
  return cudaSuccess;
}

template <class Mode, int ET>
static cudaError_t build_typed(ihsbin_problem* p, cudaStream_t st, cudaEvent_t* ev) {
  const Tall& A = p->A;
  const int64_t D = A.D, K = p->K;
  Plan& pl = p->plan;
  const int L = pl.L;
  const int cm = pl.compute;
  cudaError_t err = cudaSuccess;
  auto cb = [&](size_t elems) { return alloc_cbuf(p, cm, elems, SCOPE_SCRATCH, &err); };

  // plan arrays on the device
  std::vector<int> order(L);
  for (int l = 0; l < L; ++l) order[l] = l;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return pl.k[a] > pl.k[b]; });
  double* tau_dev = nullptr;
  double* lam0_dev = nullptr;
  int* perm_dev = nullptr;
  CK(prob_alloc(p, L * sizeof(double), (void**)&tau_dev, SCOPE_SCRATCH));
  CK(prob_alloc(p, L * sizeof(double), (void**)&lam0_dev, SCOPE_SCRATCH));
  CK(prob_alloc(p, L * sizeof(int), (void**)&perm_dev, SCOPE_SCRATCH));
  CK(cudaMemcpyAsync(tau_dev, pl.tau.data(), L * sizeof(double), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(lam0_dev, pl.lam0.data(), L * sizeof(double), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(perm_dev, order.data(), L * sizeof(int), cudaMemcpyHostToDevice, st));

  // the recursion's form (resolved after the factorization, when the plan is final): the residual
  // form is possible where the fused tensor-core recursion runs; every other configuration carries
  // the increments of Algorithm 2 as printed.
  const bool oz_on = Mode::id == 1 && pl.loop == IHSBIN_LOOP_SLICES;
  const bool resid_ok = oz_on && pl.product == IHSBIN_PRODUCT_GRAM && oz_fused_ok(D) && pl.form != IHSBIN_FORM_INCREMENT;
  const double trGS = p->trGS;  // tr(G_S), read by the sketch call

  // SMs the Gram's tensor-core launches leave to the factorization running beside them: chosen by
  // the autotuner per shape class, timing the whole fork-join region of both streams
  const bool tune_reserve =
      pl.product == IHSBIN_PRODUCT_GRAM && A.layout != IHSBIN_CSR && pl.gram == IHSBIN_GRAM_SLICES && !p->pre_taken;
  TuneLaunch rtune{};
  int gram_reserve = 0;
  if (tune_reserve) {
    static const int cands[] = {40, 0, 24, 64};
    rtune = tune_begin(tune_key(TUNE_GRAM_RESERVE, D, shape_class(A.N), L), "gram_reserve_sms", cands, 4, st);
    gram_reserve = rtune.value;
  }
  // a3: Gram (product mode GRAM) and right-hand side.  They do not depend on a2 (the factors of
  // the sketched Hessian), so they run on the problem's side stream, forked here and joined
  // before the recursion: their tensor-core work fills the SMs that the factorization's small
  // launches leave idle.  Allocations in this section are ordered on the side stream.
  CK(ensure_streams(p));
  cudaStream_t s2 = p->side;
  const bool csr = A.layout == IHSBIN_CSR;
  CBuf c{};
  if (p->pre_taken) {
    // the Gram of A and A^T b were started by ihsbin_sketch on the side stream (joined below)
    c = p->c_pre;
    CK(cudaEventRecord(ev[5], st));
  } else {
    CK(cudaEventRecord(ev[5], st));
    CK(cudaStreamWaitEvent(s2, ev[5], 0));
    CallStream side_alloc(s2);
    c = cb((size_t)D * K);
    CK(err);
    // dense data with the sliced Gram: the right-hand side comes from the same slices of A_hat
    // (K >= 32: the product's 128-column tiles of B are at least a quarter full)
    const bool rhs_fused =
        pl.product == IHSBIN_PRODUCT_GRAM && !csr && !p->dual && pl.gram == IHSBIN_GRAM_SLICES && K >= 32;
    if (pl.product == IHSBIN_PRODUCT_GRAM) {
      p->G = alloc_cbuf(p, cm, (size_t)D * D, SCOPE_BASIS, &err);
      CK(err);
      if (csr) CK(csr_gram(p, cm, s2));
      else if (pl.gram == IHSBIN_GRAM_SLICES) CK(gram_dense_slices(p, cm, s2, gram_reserve, rhs_fused ? &c : nullptr));
      else CK((gram_dense<Mode, ET>(p, s2)));
    }
    if (rhs_fused) {
      // c was formed with the Gram
    } else if (csr && !p->dual) {
      CK(csr_rhs(p, cm, c, s2));
    } else if (p->dual) {
      KTimer kt(p, K_RHS, s2, 0, (double)D * K * 16);
      k_copy_B_colmajor<Mode><<<nblocks(D * K, 256), 256, 0, s2>>>(p->B, D, K, c);
      CK(cudaGetLastError());
    } else {
      CK((rhs_dense<Mode, ET>(p, c, s2)));
    }
    CK(cudaEventRecord(ev[2], s2));
  }

  // a2: factor + inverse of the shifted sketched Hessians, on the problem's second internal
  // stream (forked with the Gram's, joined before the recursion).  Allocations in this section
  // are ordered on that stream.
  cudaStream_t sf = p->fac;
  CK(cudaStreamWaitEvent(sf, ev[5], 0));
  {
    CallStream fac_alloc(sf);
    CK(cudaEventRecord(ev[0], sf));
    p->Pinv = alloc_cbuf(p, cm, (size_t)L * D * D, SCOPE_BASIS, &err);
    CK(err);
    CBuf H = cb((size_t)L * D * D);
    CBuf Wm = cb((size_t)L * D * D);
    const int64_t nblk = (D + NB - 1) / NB;
    CBuf dinv = cb((size_t)L * nblk * NB * NB);
    CK(err);
    CK(factor_and_invert<Mode>(p, H, Wm, dinv, lam0_dev, sf));
    if (pl.auto_rho) {
      double* tr_dev = nullptr;
      CK(prob_alloc(p, L * sizeof(double), (void**)&tr_dev, SCOPE_SCRATCH));
      k_trace<Mode><<<L, 256, 0, sf>>>(p->Pinv, D, tr_dev);
      CK(cudaGetLastError());
      std::vector<double> trP(L);
      CK(cudaMemcpyAsync(trP.data(), tr_dev, L * sizeof(double), cudaMemcpyDeviceToHost, sf));
      CK(cudaStreamSynchronize(sf));
      finalize_plan(p, trP.data());
      CK(cudaMemcpyAsync(tau_dev, pl.tau.data(), L * sizeof(double), cudaMemcpyHostToDevice, sf));
      std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return pl.k[a] > pl.k[b]; });
      CK(cudaMemcpyAsync(perm_dev, order.data(), L * sizeof(int), cudaMemcpyHostToDevice, sf));
    }
    CK(cudaEventRecord(ev[1], sf));
  }

  // join both forks before the recursion
  CK(cudaStreamWaitEvent(st, ev[1], 0));
  CK(cudaStreamWaitEvent(st, p->pre_taken ? p->pre_ev[1] : ev[2], 0));
  CK(cudaEventRecord(ev[6], st));
  if (tune_reserve) tune_end(rtune, st);
  if (p->pre_taken && p->pre_tune) {
    tune_end(*p->pre_tune, st);
    delete p->pre_tune;
    p->pre_tune = nullptr;
  }

  // a4: the recursion, in the residual form when it is possible and asked for (RESIDUAL, or an
  // explicit precond_weight) or when AUTO's pair weight is at most 4
  int pw = pl.slice_w;
  bool resid = false;
  if (resid_ok) {
    pw = pl.precond_req > 0 ? pl.precond_req : precond_weight_rule(D, trGS, pl);
    // AUTO: from weight 5 on the products save little (21 of 26 pairs) and the increment form's
    // two-product steps at the end of the longest intervals are faster
    resid = pl.form == IHSBIN_FORM_RESIDUAL || pl.precond_req > 0 || pw <= 4;
  }
  pl.form_run = resid ? IHSBIN_FORM_RESIDUAL : IHSBIN_FORM_INCREMENT;
  pl.precond_w = resid ? pw : pl.slice_w;
  const size_t per = (size_t)pl.jc * K * D;
  p->Ut = alloc_cbuf(p, cm, per * L, SCOPE_BASIS, &err);
  CK(err);
  // the residual form keeps only the partial sums (in Ut); the increment form ping-pongs U0 / U1
  CBuf U0 = resid ? p->Ut : cb(per * L), U1 = resid ? p->Ut : cb(per * L);
  const int64_t ncol_max = (int64_t)pl.jc * K;
  // the tensor-core products leave exact int64 partials instead of float-float ones
  CBuf Y = cb((oz_on && pl.product == IHSBIN_PRODUCT_GRAM) ? 1 : (size_t)SPLIT_MAX * ncol_max * D * L);
  CBuf Z = cb(oz_on ? 1 : (size_t)SPLIT_MAX * ncol_max * D * L);
  CBuf R = cb((size_t)ncol_max * D * L);
  CBuf Wtmp{};
  if (pl.product == IHSBIN_PRODUCT_ASPACE) Wtmp = cb((size_t)ncol_max * A.N * L);
  CK(err);
  if (!resid) {
    CK(cudaMemsetAsync(U0.p0, 0, per * L * (cm == IHSBIN_COMPUTE_F64 ? 8 : 4), st));
    if (U0.p1) CK(cudaMemsetAsync(U0.p1, 0, per * L * 4, st));
  }
  CK(cudaMemsetAsync(p->Ut.p0, 0, per * L * (cm == IHSBIN_COMPUTE_F64 ? 8 : 4), st));
  if (p->Ut.p1) CK(cudaMemsetAsync(p->Ut.p1, 0, per * L * 4, st));
  OzLoop oz;
  if (oz_on) {
    oz.on = true;
    const int64_t bcols = (int64_t)L * (ncol_max + 64);  // columns padded to the tile width (<= 64)
    __nv_bfloat16 *Ps = nullptr, *Bs = nullptr;
    int *ep = nullptr, *eb = nullptr;
    CK(prob_alloc(p, oz_rows_elems(D) * 2 * L, (void**)&Ps, SCOPE_SCRATCH));
    CK(prob_alloc(p, oz_rows_exps(D) * 4 * L, (void**)&ep, SCOPE_SCRATCH));
    CK(prob_alloc(p, (size_t)bcols * ((D + 31) / 32) * 6 * 32 * 2, (void**)&Bs, SCOPE_SCRATCH));
    CK(prob_alloc(p, (size_t)bcols * 4, (void**)&eb, SCOPE_SCRATCH));
    CK(prob_alloc(p, (size_t)bcols * 4, (void**)&oz.er, SCOPE_SCRATCH));
    // The two-product form of the recursion (basis_loop) for the longest intervals: from the first
    // step at or after the truncation (all intervals then hold jmax K columns, a multiple of the
    // tile height 16) at which at most MFORM_LIVE intervals are still running.  It spends one D^3
    // product per interval on M_q = P_l (G + lam0_l I) and saves two of the four launches of every
    // later step.
    // (Not in the residual form: there M_l v would carry the residual, so both of its products
    // would need every pair, while the residual form's P_l r needs few.)
    constexpr int MFORM_LIVE = 6;
    int mform_from = 0, Tm = 0;
    if (!resid && pl.product == IHSBIN_PRODUCT_GRAM && oz_fused_ok(D) && pl.jmax > 0 &&
        ((int64_t)pl.jmax * K) % 16 == 0) {
      for (int i = std::max(pl.jmax, 2); i < pl.kmax; ++i) {
        int live = 0;
        while (live < L && pl.k[order[live]] > i) ++live;
        if (live == 0) break;
        if (live <= MFORM_LIVE) {
          mform_from = i;
          Tm = live;
          break;
        }
      }
    }
    // the largest split partials of any step, replaying the recursion's (live, columns, splits)
    size_t ymax = 1, zmax = 1;
    if (resid)  // the residual form's first step: P_l (-c) for every interval
      zmax = (size_t)oz_pick_split(D, K, L, oz_tile_n(K, pw), SPLIT_MAX) * L * K * D;
    {
      const int J = pl.jmax > 0 ? pl.jmax : (1 << 30);
      for (int i = 1; i < pl.kmax; ++i) {
        int live = 0;
        while (live < L && pl.k[order[live]] > i) ++live;
        if (live == 0) break;
        const int64_t nold = (int64_t)std::min(i, J) * K, nnew = (int64_t)std::min(i + 1, J) * K;
        if (mform_from > 0 && i >= mform_from) {
          zmax = std::max(zmax, (size_t)oz_pick_split(D, nold, 2 * live, 16, SPLIT_MAX) * 2 * live * nold * D);
          continue;
        }
        const int64_t ncat = nold * live;
        if (pl.product == IHSBIN_PRODUCT_GRAM)
          ymax = std::max(ymax, (size_t)oz_pick_split(D, ncat, 1, oz_tile_n(ncat), SPLIT_MAX) * ncat * D);
        zmax = std::max(zmax, (size_t)oz_pick_split(D, nnew, live, oz_tile_n(nnew, resid ? pw : pl.slice_w), SPLIT_MAX) *
                                  live * nnew * D);
      }
    }
    CK(prob_alloc(p, ymax * 8, (void**)&oz.Yhi, SCOPE_SCRATCH));
    CK(prob_alloc(p, ymax * 8, (void**)&oz.Ylo, SCOPE_SCRATCH));
    CK(prob_alloc(p, zmax * 8, (void**)&oz.Zhi, SCOPE_SCRATCH));
    CK(prob_alloc(p, zmax * 8, (void**)&oz.Zlo, SCOPE_SCRATCH));
    {
      KTimer kt(p, K_LOOP_SLICE, st, 0, (double)L * D * D * 16 + (double)L * oz_rows_elems(D) * 2);
      CK(oz_slice_rows(p->Pinv, D, L, D * D, Ps, ep, st));
    }
    if (pl.product == IHSBIN_PRODUCT_GRAM) {
      __nv_bfloat16* Gs = nullptr;
      int* eg = nullptr;
      CK(prob_alloc(p, oz_rows_elems(D) * 2, (void**)&Gs, SCOPE_SCRATCH));
      CK(prob_alloc(p, oz_rows_exps(D) * 4, (void**)&eg, SCOPE_SCRATCH));
      KTimer kt(p, K_LOOP_SLICE, st, 0, (double)D * D * 16 + (double)oz_rows_elems(D) * 2);
      CK(oz_slice_rows(p->G, D, 1, 0, Gs, eg, st));
      oz.Gs = Gs;
      oz.eg = eg;
    }
    oz.Ps = Ps;
    oz.ep = ep;
    oz.Bs = Bs;
    oz.eb = eb;
    oz.resid = resid;
    oz.pw = pl.precond_w;
    if (mform_from > 0) {
      // M_q = P_l G + lam0_l P_l for l = order[q], q < Tm: the exact-slice product G P_l (A = the
      // rows of G, shared; B = the columns of P_l), joined with lam0_l P_l, then cut by rows
      __nv_bfloat16 *Pc = nullptr, *Ms = nullptr;
      int *epc = nullptr, *em = nullptr;
      long long *mh = nullptr, *ml = nullptr;
      const size_t vcol = oz_vec_elems(D, D, 32), vexp = oz_vec_exps(D, 32);
      const int ks = oz_pick_split_mnk(D, D, D, Tm, 32, SPLIT_MAX);
      CK(prob_alloc(p, vcol * 2 * Tm, (void**)&Pc, SCOPE_SCRATCH));
      CK(prob_alloc(p, vexp * 4 * Tm, (void**)&epc, SCOPE_SCRATCH));
      CK(prob_alloc(p, (size_t)ks * Tm * D * D * 8, (void**)&mh, SCOPE_SCRATCH));
      CK(prob_alloc(p, (size_t)ks * Tm * D * D * 8, (void**)&ml, SCOPE_SCRATCH));
      CK(prob_alloc(p, oz_rows_elems(D) * 2 * Tm, (void**)&Ms, SCOPE_SCRATCH));
      CK(prob_alloc(p, oz_rows_exps(D) * 4 * Tm, (void**)&em, SCOPE_SCRATCH));
      CK(prob_alloc(p, (size_t)bcols * 4, (void**)&oz.eb2, SCOPE_SCRATCH));
      CBuf Mb = alloc_cbuf(p, IHSBIN_COMPUTE_F32X2, (size_t)Tm * D * D, SCOPE_SCRATCH, &err);
      CK(err);
      {
        KTimer kt(p, K_INVERSE_SLICE, st, 0, (double)Tm * D * D * 8 + (double)Tm * vcol * 2);
        CK(oz_slice_cols(p->Pinv, D, Tm, D, 32, D, D * D, perm_dev, Pc, epc, st));
      }
      {
        OzGemm q;
        q.wmax = p->plan.slice_w;
        q.As = oz.Gs; q.a_shared = true; q.Bs = Pc;
        q.M = D; q.N = D; q.K = D; q.groups = Tm; q.NT = 32; q.ksplit = ks;
        q.ohi = mh; q.olo = ml; q.status = p->status;
        KTimer kt(p, K_INVERSE_TC, st, 2.0 * D * D * D * Tm, (double)(1 + 2 * Tm) * D * D * 8, oz_pair_flops(D, D, D, pl.slice_w) * Tm,
                  (double)oz_rows_elems(D) * 2 + (double)Tm * vcol * 2 + 16.0 * ks * Tm * D * D);
        CK(oz_gemm(q, st));
      }
      {
        KTimer kt(p, K_INVERSE_SLICE, st, 0, (double)Tm * D * D * (16.0 * ks + 16));
        CK(oz_make_M(mh, ml, ks, D, Tm, oz.eg, epc, (int64_t)vexp, perm_dev, lam0_dev, p->Pinv, Mb, st));
      }
      {
        KTimer kt(p, K_INVERSE_SLICE, st, 0, (double)Tm * D * D * 8 + (double)Tm * oz_rows_elems(D) * 2);
        CK(oz_slice_rows(Mb, D, Tm, D * D, Ms, em, st));
      }
      oz.Ms = Ms;
      oz.em = em;
      oz.mform_from = mform_from;
    }
  }
  CK((basis_loop<Mode, ET>(p, c, U0, U1, Y, Z, R, Wtmp, perm_dev, tau_dev, lam0_dev, order, oz, st)));

  // a5: primal image of the dual basis, W_l = A_hat utilde_l (N x jc K)
  if (p->dual && csr) {
    p->W = alloc_cbuf(p, cm, (size_t)L * pl.jc * K * A.N, SCOPE_BASIS, &err);
    CK(err);
    CK(csr_dual_map(p, cm, (int64_t)pl.jc * K, st));
  } else if (p->dual) {
    const int64_t N = A.N;
    p->W = alloc_cbuf(p, cm, (size_t)L * pl.jc * K * N, SCOPE_BASIS, &err);
    CK(err);
    GemmShape sh{N, (int64_t)pl.jc * K, D, 0};
    KTimer kt(p, K_DUAL_MAP, st, 2.0 * N * D * pl.jc * K * L, (double)N * D * (ET == ELEM_F64 ? 8 : ET == ELEM_F32 ? 4 : 2) * L);
    CK((launch_gemm<Mode, 64, 32, 16, 4, 2>(sh, L, LdAhatRow<Mode, ET>{A.A, A.ld}, LdCColB<Mode>{p->Ut, D, (int64_t)per, nullptr},
                                            EpStoreColMajor<Mode>{p->W, N, (int64_t)pl.jc * K * N, nullptr}, st)));
  }
  CK(cudaEventRecord(ev[3], st));
  return cudaSuccess;
}

// ============================================= adaptive sketch dimension (Section 5.1, Algorithm 4)
// Newton-sketch steps on f(x) = 1/2 x^T (G + lam I) x - c^T x (G = A_hat^T A_hat, D x K iterate,
// column-major) in the compute mode's arithmetic; the host takes the Armijo and doubling decisions
// from the two inner products each step leaves in FP64.

// part[b] = sum over block b's entries of a_e b_e (each product rounded to FP64); fixed tree order
template <class Mode>
__global__ void __launch_bounds__(256) k_dot_partial(CBuf a, CBuf b, int64_t n, double* part) {
  __shared__ double red[8];
  double v = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * 256 + threadIdx.x; e < n; e += (int64_t)gridDim.x * 256)
    v += Mode::to_d(Mode::mul(Mode::ld(a, e), Mode::ld(b, e)));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += red[w];
    part[blockIdx.x] = s;
  }
}
__global__ void k_sum_parts(const double* part, int nb, double* out) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += part[b];
    *out = s;
  }
}
// y += alpha x (alpha an FP64 scalar), or y = alpha x when assign
template <class Mode>
__global__ void k_axpy(CBuf x, double alpha, CBuf y, int64_t n, int assign) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const typename Mode::V t = Mode::mul(Mode::from_d(alpha), Mode::ld(x, e));
  Mode::st(y, e, assign ? t : Mode::add(Mode::ld(y, e), t));
}
template <class Mode>
__global__ void k_to_rowmajor_f64(CBuf x, int64_t D, int64_t K, double* out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // over D x K, row-major output
  if (e >= D * K) return;
  const int64_t i = e / K, r = e - i * K;
  out[e] = Mode::to_d(Mode::ld(x, r * D + i));
}

constexpr int DOT_BLOCKS = 256;

template <class Mode>
static cudaError_t dot_into(CBuf a, CBuf b, int64_t n, double* part, double* out, cudaStream_t st) {
  const int nb = (int)std::min<int64_t>(DOT_BLOCKS, nblocks(n, 256));
  k_dot_partial<Mode><<<nb, 256, 0, st>>>(a, b, n, part);
  CK(cudaGetLastError());
  k_sum_parts<<<1, 32, 0, st>>>(part, nb, out);
  return cudaGetLastError();
}
template <class Mode>
static cudaError_t sym_apply(CBuf M, CBuf X, int64_t D, int64_t K, CBuf Y, cudaStream_t st) {
  GemmShape sh{D, K, D, 0};
  return launch_gemm<Mode, 64, 32, 16, 4, 2>(sh, 1, LdCMatA<Mode>{M, D, 0, nullptr}, LdCColB<Mode>{X, D, 0, nullptr},
                                             EpStoreColMajor<Mode>{Y, D, 0, nullptr}, st);
}

template <class Mode, int ET>
static cudaError_t adaptive_setup_typed(ihsbin_problem* p, AdaptiveBufs& b, cudaStream_t st) {
  const Tall& A = p->A;
  const int64_t D = A.D, K = p->K;
  const int cm = p->plan.compute;
  p->G = b.G;
  if (A.layout == IHSBIN_CSR) CK(csr_gram(p, cm, st));
  else if (p->plan.gram == IHSBIN_GRAM_SLICES) CK(gram_dense_slices(p, cm, st));
  else CK((gram_dense<Mode, ET>(p, st)));
  if (A.layout == IHSBIN_CSR && !p->dual) {
    CK(csr_rhs(p, cm, b.c, st));
  } else if (p->dual) {
    KTimer kt(p, K_RHS, st, 0, (double)D * K * 16);
    k_copy_B_colmajor<Mode><<<nblocks(D * K, 256), 256, 0, st>>>(p->B, D, K, b.c);
    CK(cudaGetLastError());
  } else {
    CK((rhs_dense<Mode, ET>(p, b.c, st)));
  }
  p->G = CBuf{};
  // x = 0, g = grad f(0) = -c
  KTimer kt(p, K_ADAPTIVE, st, 0, 24.0 * D * K);
  k_axpy<Mode><<<nblocks(D * K, 256), 256, 0, st>>>(b.c, 0.0, b.x, D * K, 1);
  k_axpy<Mode><<<nblocks(D * K, 256), 256, 0, st>>>(b.c, -1.0, b.g, D * K, 1);
  return cudaGetLastError();
}

template <class Mode>
static cudaError_t adaptive_precond_typed(ihsbin_problem* p, AdaptiveBufs& b, cudaStream_t st) {
  const int64_t D = p->A.D;
  cudaError_t err = cudaSuccess;
  const int cm = p->plan.compute;
  CBuf H = alloc_cbuf(p, cm, (size_t)D * D, SCOPE_SCRATCH, &err);
  CBuf Wm = alloc_cbuf(p, cm, (size_t)D * D, SCOPE_SCRATCH, &err);
  const int64_t nblk = (D + NB - 1) / NB;
  CBuf dinv = alloc_cbuf(p, cm, (size_t)nblk * NB * NB, SCOPE_SCRATCH, &err);
  CK(err);
  p->Pinv = b.P;
  err = factor_and_invert<Mode>(p, H, Wm, dinv, b.lam_dev, st);
  p->Pinv = CBuf{};
  return err;
}

template <class Mode>
static cudaError_t adaptive_direction_typed(ihsbin_problem* p, AdaptiveBufs& b, cudaStream_t st) {
  const int64_t D = p->A.D, K = p->K;
  KTimer kt(p, K_ADAPTIVE, st, 2.0 * D * D * K + 2.0 * D * K, 8.0 * D * D + 24.0 * D * K);
  CK(sym_apply<Mode>(b.P, b.g, D, K, b.d, st));
  return dot_into<Mode>(b.d, b.g, D * K, b.part, b.dots, st);
}

template <class Mode>
static cudaError_t adaptive_curvature_typed(ihsbin_problem* p, AdaptiveBufs& b, double lam, cudaStream_t st) {
  const int64_t D = p->A.D, K = p->K;
  KTimer kt(p, K_ADAPTIVE, st, 2.0 * D * D * K + 4.0 * D * K, 8.0 * D * D + 40.0 * D * K);
  CK(sym_apply<Mode>(b.G, b.d, D, K, b.hd, st));
  k_axpy<Mode><<<nblocks(D * K, 256), 256, 0, st>>>(b.d, lam, b.hd, D * K, 0);
  CK(cudaGetLastError());
  return dot_into<Mode>(b.d, b.hd, D * K, b.part, b.dots + 1, st);
}

template <class Mode>
static cudaError_t adaptive_step_typed(ihsbin_problem* p, AdaptiveBufs& b, double t, cudaStream_t st) {
  const int64_t D = p->A.D, K = p->K;
  KTimer kt(p, K_ADAPTIVE, st, 4.0 * D * K, 48.0 * D * K);
  k_axpy<Mode><<<nblocks(D * K, 256), 256, 0, st>>>(b.d, -t, b.x, D * K, 0);
  k_axpy<Mode><<<nblocks(D * K, 256), 256, 0, st>>>(b.hd, -t, b.g, D * K, 0);
  return cudaGetLastError();
}

cudaError_t adaptive_setup(ihsbin_problem* p, AdaptiveBufs& b, cudaStream_t st) {
  const int et = p->A.elem;
  if (p->plan.compute == IHSBIN_COMPUTE_F64) {
    if (et == ELEM_F64) return adaptive_setup_typed<F64, ELEM_F64>(p, b, st);
    if (et == ELEM_F32) return adaptive_setup_typed<F64, ELEM_F32>(p, b, st);
    return adaptive_setup_typed<F64, ELEM_BF16>(p, b, st);
  }
  if (et == ELEM_F64) return adaptive_setup_typed<DD, ELEM_F64>(p, b, st);
  if (et == ELEM_F32) return adaptive_setup_typed<DD, ELEM_F32>(p, b, st);
  return adaptive_setup_typed<DD, ELEM_BF16>(p, b, st);
}
cudaError_t adaptive_precond(ihsbin_problem* p, AdaptiveBufs& b, cudaStream_t st) {
  return p->plan.compute == IHSBIN_COMPUTE_F64 ? adaptive_precond_typed<F64>(p, b, st)
                                               : adaptive_precond_typed<DD>(p, b, st);
}
cudaError_t adaptive_direction(ihsbin_problem* p, AdaptiveBufs& b, cudaStream_t st) {
  return p->plan.compute == IHSBIN_COMPUTE_F64 ? adaptive_direction_typed<F64>(p, b, st)
                                               : adaptive_direction_typed<DD>(p, b, st);
}
cudaError_t adaptive_curvature(ihsbin_problem* p, AdaptiveBufs& b, double lam, cudaStream_t st) {
  return p->plan.compute == IHSBIN_COMPUTE_F64 ? adaptive_curvature_typed<F64>(p, b, lam, st)
                                               : adaptive_curvature_typed<DD>(p, b, lam, st);
}
cudaError_t adaptive_step(ihsbin_problem* p, AdaptiveBufs& b, double t, cudaStream_t st) {
  return p->plan.compute == IHSBIN_COMPUTE_F64 ? adaptive_step_typed<F64>(p, b, t, st)
                                               : adaptive_step_typed<DD>(p, b, t, st);
}
cudaError_t adaptive_export_x(ihsbin_problem* p, AdaptiveBufs& b, double* out_dev, cudaStream_t st) {
  const int64_t D = p->A.D, K = p->K;
  if (p->plan.compute == IHSBIN_COMPUTE_F64)
    k_to_rowmajor_f64<F64><<<nblocks(D * K, 256), 256, 0, st>>>(b.x, D, K, out_dev);
  else
    k_to_rowmajor_f64<DD><<<nblocks(D * K, 256), 256, 0, st>>>(b.x, D, K, out_dev);
  return cudaGetLastError();
}

cudaError_t build_basis_device(ihsbin_problem* p, cudaStream_t st, cudaEvent_t* ev) {
  const int cm = p->plan.compute, et = p->A.elem;
  if (p->A.layout == IHSBIN_CSR && p->plan.product != IHSBIN_PRODUCT_GRAM) return cudaErrorNotSupported;
  if (cm == IHSBIN_COMPUTE_F64) {
    if (et == ELEM_F64) return build_typed<F64, ELEM_F64>(p, st, ev);
    if (et == ELEM_F32) return build_typed<F64, ELEM_F32>(p, st, ev);
    return build_typed<F64, ELEM_BF16>(p, st, ev);
  }
  if (et == ELEM_F64) return build_typed<DD, ELEM_F64>(p, st, ev);
  if (et == ELEM_F32) return build_typed<DD, ELEM_F32>(p, st, ev);
  return build_typed<DD, ELEM_BF16>(p, st, ev);
}

// The lambdas grouped by interval (the interval rule of k_eval_coef) into chunks of <= EVAL_TB, as one
// device array [order T][chunk interval][chunk start][chunk count].
static cudaError_t lambda_chunks(ihsbin_problem* p, const double* lam_host, int64_t T, int** dev_out, int* nch_out,
                                 cudaStream_t st) {
  const Plan& pl = p->plan;
  const int L = pl.L;
  std::vector<std::vector<int>> by(L);
  for (int64_t t = 0; t < T; ++t) {
    int lo = 0, hi = L;
    while (hi - lo > 1) {
      const int mid = (lo + hi) / 2;
      if (pl.edges[mid] <= lam_host[t]) lo = mid; else hi = mid;
    }
    by[lo].push_back((int)t);
  }
  std::vector<int> torder, cl, ct0, cn;
  for (int l = 0; l < L; ++l)
    for (size_t a = 0; a < by[l].size(); a += EVAL_TB) {
      cl.push_back(l);
      ct0.push_back((int)torder.size());
      cn.push_back((int)std::min<size_t>(EVAL_TB, by[l].size() - a));
      for (size_t b = a; b < std::min(by[l].size(), a + EVAL_TB); ++b) torder.push_back(by[l][b]);
    }
  const int nch = (int)cl.size();
  int* dev = nullptr;
  CK(prob_alloc(p, (T + 3 * (size_t)nch) * sizeof(int), (void**)&dev, SCOPE_SCRATCH));
  std::vector<int> pack(torder);
  pack.insert(pack.end(), cl.begin(), cl.end());
  pack.insert(pack.end(), ct0.begin(), ct0.end());
  pack.insert(pack.end(), cn.begin(), cn.end());
  // from pageable memory: the call returns once `pack` is staged, so it may go out of scope
  CK(cudaMemcpyAsync(dev, pack.data(), pack.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  *dev_out = dev;
  *nch_out = nch;
  return cudaSuccess;
}

// The coefficient table coef[t][j] = tau_l theta_t^j, in FP64 and in compute precision.
template <class Mode>
static cudaError_t coef_table(ihsbin_problem* p, const double* lam_dev, int64_t T, CBuf* coefc, int** jcount_out,
                              cudaStream_t st) {
  const Plan& pl = p->plan;
  const int L = pl.L, jc = pl.jc;
  double *edges = nullptr, *tau = nullptr, *lam0 = nullptr, *coef = nullptr;
  int *jcount = nullptr, *tint = nullptr;
  CK(prob_alloc(p, (L + 1) * sizeof(double), (void**)&edges, SCOPE_SCRATCH));
  CK(prob_alloc(p, L * sizeof(double), (void**)&tau, SCOPE_SCRATCH));
  CK(prob_alloc(p, L * sizeof(double), (void**)&lam0, SCOPE_SCRATCH));
  CK(prob_alloc(p, L * sizeof(int), (void**)&jcount, SCOPE_SCRATCH));
  CK(prob_alloc(p, T * sizeof(int), (void**)&tint, SCOPE_SCRATCH));
  CK(prob_alloc(p, (size_t)T * jc * sizeof(double), (void**)&coef, SCOPE_SCRATCH));
  *coefc = CBuf{coef, nullptr};
  if (Mode::id == 1) {
    CK(prob_alloc(p, (size_t)T * jc * sizeof(float), &coefc->p0, SCOPE_SCRATCH));
    CK(prob_alloc(p, (size_t)T * jc * sizeof(float), &coefc->p1, SCOPE_SCRATCH));
  }
  CK(cudaMemcpyAsync(edges, pl.edges.data(), (L + 1) * sizeof(double), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(tau, pl.tau.data(), L * sizeof(double), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(lam0, pl.lam0.data(), L * sizeof(double), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(jcount, pl.jcount.data(), L * sizeof(int), cudaMemcpyHostToDevice, st));
  *jcount_out = jcount;
  KTimer kt(p, K_EVAL_COEF, st, 0, (double)T * jc * 8);
  k_eval_coef<<<nblocks(T, 128), 128, 0, st>>>(lam_dev, T, edges, L, tau, lam0, jcount, jc, tint, coef,
                                               Mode::id == 1 ? (float*)coefc->p0 : nullptr,
                                               Mode::id == 1 ? (float*)coefc->p1 : nullptr);
  return cudaGetLastError();
}

template <class Mode>
static cudaError_t eval_typed(ihsbin_problem* p, const double* lam_host, const double* lam_dev, int64_t T, void* X,
                              int x_elem, cudaStream_t st) {
  const int jc = p->plan.jc;
  CBuf coefc;
  int* jcount = nullptr;
  CK(coef_table<Mode>(p, lam_dev, T, &coefc, &jcount, st));
  const int64_t K = p->K;
  const int64_t rows = p->dual ? p->A.N : p->A.D;
  const CBuf Bm = p->dual ? p->W : p->Ut;
  const int64_t gs = (int64_t)jc * K * rows;
  int* dev = nullptr;
  int nch = 0;
  CK(lambda_chunks(p, lam_host, T, &dev, &nch, st));
  dim3 grid(nblocks(rows * K, 256), (unsigned)nch);
  KTimer kt(p, K_EVAL, st, 2.0 * T * rows * K * jc, (double)T * rows * K * (x_elem == ELEM_F64 ? 8 : 4));
  k_eval_chunks<Mode><<<grid, 256, 0, st>>>(Bm, rows, K, jc, gs, dev + T, dev + T + nch, dev + T + 2 * nch, dev, coefc,
                                            jcount, X, x_elem);
  return cudaGetLastError();
}

// ============================================= losses along the path (Section 6.1), without X
// For a chunk of lambdas of interval l: ssq[pos][boff + block] = sum over the block's entries (i, r) of
// (sum_j coef[t][j] V_l[j][r][i] - target[i][r])^2  (target null: plain squares), pos = the lambda's
// position in the chunk order; the residual in compute precision, its square summed in FP64.
template <class Mode>
__global__ void __launch_bounds__(256) k_resid_ssq_chunks(CBuf Vm, int64_t rows, int64_t K, int jc, int64_t gs,
                                                          const int* chunk_l, const int* chunk_t0, const int* chunk_n,
                                                          const int* torder, CBuf coef, const int* jcount,
                                                          const double* target, double* ssq, int64_t nbt,
                                                          int64_t boff) {
  __shared__ double red[EVAL_TB][8];
  const int c = blockIdx.y;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool in = e < rows * K;
  const int64_t r = in ? e / rows : 0, i = in ? e % rows : 0;
  const int l = chunk_l[c], nq = chunk_n[c], t0 = chunk_t0[c];
  const int jn = jcount[l];
  int tq[EVAL_TB];
  typename Mode::V acc[EVAL_TB];
#pragma unroll
  for (int q = 0; q < EVAL_TB; ++q) {
    tq[q] = q < nq ? torder[t0 + q] : 0;
    acc[q] = Mode::zero();
  }
  if (in)
    for (int j = 0; j < jn; ++j) {
      const typename Mode::V b = Mode::ld(Vm, (int64_t)l * gs + ((int64_t)j * K + r) * rows + i);
#pragma unroll
      for (int q = 0; q < EVAL_TB; ++q)
        if (q < nq) acc[q] = Mode::add(acc[q], Mode::mul(Mode::ld(coef, (int64_t)tq[q] * jc + j), b));
    }
  const typename Mode::V tg = (in && target) ? Mode::from_d(target[i * K + r]) : Mode::zero();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int q = 0; q < EVAL_TB; ++q) {
    double v = 0.0;
    if (in && q < nq) {
      v = Mode::to_d(Mode::sub(acc[q], tg));
      v *= v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[q][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x < nq) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += red[threadIdx.x][w];
    ssq[(int64_t)(t0 + threadIdx.x) * nbt + boff + blockIdx.x] = s;
  }
}
// out[t] = 1/2 sum_b ssq[pos][b] (+ 1/2 lambda_t sum_b xsq[pos][b]); fixed summation order
__global__ void k_loss_reduce(const double* ssq, const double* xsq, int64_t nb, int64_t nbx, const int* torder,
                              int64_t T, const double* lam, double* out) {
  const int64_t pos = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (pos >= T) return;
  double s = 0.0;
  for (int64_t b = 0; b < nb; ++b) s += ssq[pos * nb + b];
  const int t = torder[pos];
  double v = 0.5 * s;
  if (xsq) {
    double x = 0.0;
    for (int64_t b = 0; b < nbx; ++b) x += xsq[pos * nbx + b];
    v += 0.5 * lam[t] * x;
  }
  out[t] = v;
}
// V[j][i] = the float-float value of the exact partials of (row i, column j), summed over S splits
__global__ void k_oz_join_cols(const long long* hi, const long long* lo, int S, int64_t M, int64_t N, const int* ea,
                               const int* eb, CBuf V) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= M * N) return;
  const int64_t i = e % M, j = e / M;
  long long h = 0, w = 0;
  for (int s = 0; s < S; ++s) {
    h += hi[(int64_t)s * M * N + e];
    w += lo[(int64_t)s * M * N + e];
  }
  DD::st(V, e, oz_join(h, w, ea[i], eb[j]));
}

// The matrix of one loss term, by rows: dense row-major (rows of M), the transposed view of a dense
// row-major M (its columns), or CSR.  target: rows x K row-major FP64 (null: no target).
struct LossSrc {
  int kind = 0;  // 0 dense rows, 1 dense columns, 2 CSR
  const void* M = nullptr;
  int elem = ELEM_F64;
  int64_t ld = 0;
  const int64_t* rp = nullptr;
  const int32_t* ci = nullptr;
  const void* val = nullptr;
  int64_t rows = 0;
  const double* target = nullptr;
};
struct LossCtx {
  CBuf PB;  // the primal basis: ncols columns of length d
  int64_t d = 0, ncols = 0;
  CBuf coefc;
  const int* jcount = nullptr;
  const int* chunks = nullptr;
  int nch = 0;
  int64_t T = 0;
  // exact-slice images: the basis cut once (tile height 32)
  __nv_bfloat16* Bs = nullptr;
  int* eb = nullptr;
  CBuf PBT;  // transposed basis for CSR rows
};

constexpr size_t LOSS_CHUNK_BYTES = size_t(2) << 30;  // scratch for one block of rows
constexpr int64_t LOSS_CHUNK_ROWS = 32768;             // and at most this many rows

// V = M0 PB on the CUDA cores: M0's rows (or, trans, its columns) x the basis columns, column-major
template <class Mode, int ET>
static cudaError_t image_fma(const GemmShape& sh, const void* M0, int64_t ld, bool trans, CBuf PB, int64_t d, CBuf V,
                             cudaStream_t st) {
  const EpStoreColMajor<Mode> ep{V, sh.M, 0, nullptr};
  const LdCColB<Mode> lb{PB, d, 0, nullptr};
  if (trans) return launch_gemm<Mode, 64, 32, 16, 4, 2>(sh, 1, LdTrans<Mode, ET>{M0, ld}, lb, ep, st);
  return launch_gemm<Mode, 64, 32, 16, 4, 2>(sh, 1, LdAhatRow<Mode, ET>{M0, ld}, lb, ep, st);
}

static size_t elem_bytes(int elem) { return elem == ELEM_F64 ? 8 : elem == ELEM_F32 ? 4 : 2; }

// sum of squared residuals of every lambda over the rows of `s` into ssq (T x nbt, positions in the
// chunk order); rows taken in blocks so that the images fit LOSS_CHUNK_BYTES
template <class Mode>
static cudaError_t loss_term(ihsbin_problem* p, const LossSrc& s, LossCtx& c, double** ssq_out, int64_t* nbt_out,
                             cudaStream_t st) {
  const int64_t K = p->K, d = c.d, nc = c.ncols;
  const int jc = p->plan.jc;
  const int cm = Mode::id == 0 ? IHSBIN_COMPUTE_F64 : IHSBIN_COMPUTE_F32X2;
  const bool tc = Mode::id == 1 && p->plan.loop == IHSBIN_LOOP_SLICES && s.kind == 0;
  const int64_t dpad = (d + 31) / 32 * 32;
  int S0 = tc ? oz_pick_split_mnk(std::min<int64_t>(s.rows, 1 << 16), nc, d, 1, 32, 16) : 0;
  const size_t per_row = (size_t)8 * nc + (tc ? (size_t)16 * S0 * nc + (size_t)12 * dpad + 4 : 0);
  int64_t nr = std::max<int64_t>(128, (int64_t)(LOSS_CHUNK_BYTES / per_row) / 128 * 128);
  nr = std::min(std::min(nr, LOSS_CHUNK_ROWS), s.rows);
  const int64_t nblk_rows = (s.rows + nr - 1) / nr;
  const int64_t last = s.rows - (nblk_rows - 1) * nr;
  int64_t nbt = 0;
  for (int64_t b = 0; b < nblk_rows; ++b) nbt += nblocks((b + 1 < nblk_rows ? nr : last) * K, 256);
  double* ssq = nullptr;
  CK(prob_alloc(p, (size_t)c.T * nbt * sizeof(double), (void**)&ssq, SCOPE_SCRATCH));
  cudaError_t err = cudaSuccess;
  CBuf V = alloc_cbuf(p, cm, (size_t)nr * nc, SCOPE_SCRATCH, &err);
  CK(err);
  __nv_bfloat16* As = nullptr;
  int* ea = nullptr;
  long long *hi = nullptr, *lo = nullptr;
  int Smax = 1;
  if (tc) {
    Smax = std::max(oz_pick_split_mnk(nr, nc, d, 1, 32, 16), oz_pick_split_mnk(last, nc, d, 1, 32, 16));
    CK(prob_alloc(p, oz_vec_elems(nr, d, 128) * 2, (void**)&As, SCOPE_SCRATCH));
    CK(prob_alloc(p, oz_vec_exps(nr, 128) * 4, (void**)&ea, SCOPE_SCRATCH));
    CK(prob_alloc(p, (size_t)Smax * nr * nc * 8, (void**)&hi, SCOPE_SCRATCH));
    CK(prob_alloc(p, (size_t)Smax * nr * nc * 8, (void**)&lo, SCOPE_SCRATCH));
  }
  const size_t es = elem_bytes(s.elem);
  int64_t boff = 0;
  for (int64_t b = 0; b < nblk_rows; ++b) {
    const int64_t r0 = b * nr, rows = b + 1 < nblk_rows ? nr : last;
    if (s.kind == 2) {
      CK(csr_basis_image(p, cm, s.rp + r0, s.ci, s.val, rows, c.PBT, nc, V, st));
    } else if (tc) {
      const char* M0 = (const char*)s.M + (size_t)r0 * s.ld * es;
      {
        KTimer kt(p, K_LOSS_SLICE, st, 0, (double)rows * d * es + (double)oz_vec_elems(rows, d, 128) * 2);
        CK(oz_slice_data_rows(M0, s.elem, s.ld, d, rows, 128, As, ea, st));
      }
      const int S = oz_pick_split_mnk(rows, nc, d, 1, 32, 16);
      {
        OzGemm q;
        q.As = As; q.ea = ea; q.Bs = c.Bs; q.eb = c.eb;
        q.M = rows; q.N = nc; q.K = d; q.groups = 1; q.NT = 32; q.ksplit = S;
        q.ohi = hi; q.olo = lo; q.status = p->status;
        KTimer kt(p, K_LOSS_TC, st, 2.0 * rows * nc * d, (double)rows * d * es + 8.0 * nc * d + 8.0 * rows * nc,
                  oz_pair_flops(rows, nc, d),
                  (double)oz_vec_elems(rows, d, 128) * 2 + (double)oz_vec_elems(nc, d, 32) * 2 + 16.0 * S * rows * nc);
        CK(oz_gemm(q, st));
      }
      KTimer kt(p, K_LOSS_SLICE, st, 0, 16.0 * S * rows * nc + 8.0 * rows * nc);
      k_oz_join_cols<<<nblocks(rows * nc, 256), 256, 0, st>>>(hi, lo, S, rows, nc, ea, c.eb, V);
      CK(cudaGetLastError());
    } else {
      GemmShape sh{rows, nc, d, 0};
      KTimer kt(p, K_LOSS_IMAGE, st, 2.0 * rows * nc * d, (double)rows * d * es + 8.0 * rows * nc);
      const char* M0 = (const char*)s.M + (size_t)r0 * (s.kind == 0 ? s.ld : 1) * es;
      if (s.elem == ELEM_F64) CK((image_fma<Mode, ELEM_F64>(sh, M0, s.ld, s.kind == 1, c.PB, d, V, st)));
      else if (s.elem == ELEM_F32) CK((image_fma<Mode, ELEM_F32>(sh, M0, s.ld, s.kind == 1, c.PB, d, V, st)));
      else CK((image_fma<Mode, ELEM_BF16>(sh, M0, s.ld, s.kind == 1, c.PB, d, V, st)));
    }
    const int64_t nb = nblocks(rows * K, 256);
    KTimer kt(p, K_LOSS_RESID, st, 2.0 * c.T * rows * K * jc, (double)rows * K * jc * 8 * c.nch + 8.0 * rows * K);
    k_resid_ssq_chunks<Mode><<<dim3((unsigned)nb, (unsigned)c.nch), 256, 0, st>>>(
        V, rows, K, jc, (int64_t)jc * K * rows, c.chunks + c.T, c.chunks + c.T + c.nch, c.chunks + c.T + 2 * c.nch,
        c.chunks, c.coefc, c.jcount, s.target ? s.target + r0 * K : nullptr, ssq, nbt, boff);
    CK(cudaGetLastError());
    boff += nb;
  }
  *ssq_out = ssq;
  *nbt_out = nbt;
  return cudaSuccess;
}

template <class Mode>
static cudaError_t losses_typed(ihsbin_problem* p, const double* lam_host, const double* lam_dev, int64_t T,
                                const void* At, int at_elem, int64_t at_ld, int64_t n_test, const double* Bt,
                                double* train_out, double* test_out, cudaStream_t st) {
  const Plan& pl = p->plan;
  const int64_t K = p->K, d = p->d;
  const int cm = Mode::id == 0 ? IHSBIN_COMPUTE_F64 : IHSBIN_COMPUTE_F32X2;
  LossCtx c;
  c.PB = p->dual ? p->W : p->Ut;  // (L x jc x K) columns of length d
  c.d = d;
  c.ncols = (int64_t)pl.L * pl.jc * K;
  c.T = T;
  CK(coef_table<Mode>(p, lam_dev, T, &c.coefc, (int**)&c.jcount, st));
  int* chunks = nullptr;
  CK(lambda_chunks(p, lam_host, T, &chunks, &c.nch, st));
  c.chunks = chunks;
  const Tall& A = p->A;
  LossSrc tr;  // the training rows: A itself (A_hat over-determined, A_hat^T for the dual)
  tr.rows = p->n;
  tr.target = p->B;
  if (A.layout == IHSBIN_CSR) {
    tr.kind = 2;
    tr.rp = p->dual ? A.rpT : A.rp;
    tr.ci = p->dual ? A.ciT : A.ci;
    tr.val = p->dual ? A.valT : A.val;
    tr.elem = A.elem;
  } else {
    tr.kind = p->dual ? 1 : 0;
    tr.M = A.A;
    tr.elem = A.elem;
    tr.ld = A.ld;
  }
  LossSrc te;
  te.kind = 0;
  te.M = At;
  te.elem = at_elem;
  te.ld = at_ld;
  te.rows = n_test;
  te.target = Bt;
  const bool slices = Mode::id == 1 && pl.loop == IHSBIN_LOOP_SLICES &&
                      ((train_out && tr.kind == 0) || (test_out && te.kind == 0));
  if (slices) {
    CK(prob_alloc(p, oz_vec_elems(c.ncols, d, 32) * 2, (void**)&c.Bs, SCOPE_SCRATCH));
    CK(prob_alloc(p, oz_vec_exps(c.ncols, 32) * 4, (void**)&c.eb, SCOPE_SCRATCH));
    KTimer kt(p, K_LOSS_SLICE, st, 0, 8.0 * c.ncols * d + (double)oz_vec_elems(c.ncols, d, 32) * 2);
    CK(oz_slice_vecs(c.PB, 0, 0, d, d, c.ncols, 1, 32, c.Bs, c.eb, st));
  }
  if (train_out && tr.kind == 2) {
    cudaError_t err = cudaSuccess;
    c.PBT = alloc_cbuf(p, cm, (size_t)c.ncols * d, SCOPE_SCRATCH, &err);
    CK(err);
    CK(basis_transpose(p, cm, c.PB, d, c.ncols, c.PBT, st));
  }
  if (train_out) {
    // ||x(lambda)||^2 from the basis itself, then the residuals against B
    double *xsq = nullptr, *ssq = nullptr;
    int64_t nbx = nblocks(d * K, 256), nbt = 0;
    CK(prob_alloc(p, (size_t)T * nbx * sizeof(double), (void**)&xsq, SCOPE_SCRATCH));
    {
      KTimer kt(p, K_LOSS_RESID, st, 2.0 * T * d * K * pl.jc, (double)d * K * pl.jc * 8 * c.nch);
      k_resid_ssq_chunks<Mode><<<dim3((unsigned)nbx, (unsigned)c.nch), 256, 0, st>>>(
          c.PB, d, K, pl.jc, (int64_t)pl.jc * K * d, chunks + T, chunks + T + c.nch, chunks + T + 2 * c.nch, chunks,
          c.coefc, c.jcount, nullptr, xsq, nbx, 0);
      CK(cudaGetLastError());
    }
    CK(loss_term<Mode>(p, tr, c, &ssq, &nbt, st));
    KTimer kt(p, K_LOSS_RESID, st, 0, 8.0 * T * (nbt + nbx));
    k_loss_reduce<<<nblocks(T, 128), 128, 0, st>>>(ssq, xsq, nbt, nbx, chunks, T, lam_dev, train_out);
    CK(cudaGetLastError());
  }
  if (test_out) {
    double* ssq = nullptr;
    int64_t nbt = 0;
    CK(loss_term<Mode>(p, te, c, &ssq, &nbt, st));
    KTimer kt(p, K_LOSS_RESID, st, 0, 8.0 * T * nbt);
    k_loss_reduce<<<nblocks(T, 128), 128, 0, st>>>(ssq, nullptr, nbt, 0, chunks, T, lam_dev, test_out);
    CK(cudaGetLastError());
  }
  return cudaSuccess;
}

cudaError_t losses_device(ihsbin_problem* p, const double* lam_host, const double* lam_dev, int64_t T, const void* At,
                          int at_elem, int64_t at_ld, int64_t n_test, const double* Bt, double* train_out,
                          double* test_out, cudaStream_t st) {
  if (p->plan.compute == IHSBIN_COMPUTE_F64)
    return losses_typed<F64>(p, lam_host, lam_dev, T, At, at_elem, at_ld, n_test, Bt, train_out, test_out, st);
  return losses_typed<DD>(p, lam_host, lam_dev, T, At, at_elem, at_ld, n_test, Bt, train_out, test_out, st);
}

cudaError_t eval_device(ihsbin_problem* p, const double* lam_host, const double* lam_dev, int64_t T, void* X,
                        int x_elem, cudaStream_t st) {
  if (p->plan.compute == IHSBIN_COMPUTE_F64) return eval_typed<F64>(p, lam_host, lam_dev, T, X, x_elem, st);
  return eval_typed<DD>(p, lam_host, lam_dev, T, X, x_elem, st);
}


}  // namespace ihsbin
