// CSR data matrices: transpose, Gram matrix, right-hand side and dual map.
//
// A CSR problem keeps both CSR(A_hat) and CSR(A_hat^T) on the device (one of
// them is the caller's array, the other is built here by a counting-sort
// transpose), so every product is a row gather.
//
//  * Gram  G = A_hat^T A_hat = sum over rows r of a_r^T a_r: each row's
//    nonzero pairs are added into the upper triangle with FP64 atomics (a row
//    of C3 has 40 nonzeros: 820 pairs); G is then mirrored and converted to the
//    compute precision.  The loop then runs on G exactly as for dense data.
//  * rhs   c = A_hat^T B: one warp per row of A_hat^T, float-float (or FP64)
//    accumulation, warp-reduced.
//  * dual  W_l = A_hat utilde_l: one warp per row of A_hat.
#include <algorithm>
#include <cmath>

#include "internal.h"

namespace ihsbin {

#define CK(x)                         \
  do {                                \
    cudaError_t e_ = (x);             \
    if (e_ != cudaSuccess) return e_; \
  } while (0)

static inline unsigned nblk(int64_t n, int b) { return (unsigned)std::max<int64_t>(1, (n + b - 1) / b); }

// ------------------------------------------------------------------ transpose
__global__ void k_count_cols(const int32_t* ci, int64_t nnz, unsigned long long* cnt) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&cnt[ci[e]], 1ull);
}

// exclusive scan of n counts into out[0..n] (out[n] = total), three passes
constexpr int SCAN_B = 1024;
__global__ void __launch_bounds__(SCAN_B) k_scan_blocks(const unsigned long long* in, int64_t n, int64_t* out,
                                                        int64_t* sums) {
  __shared__ int64_t ws[32];
  const int64_t i = (int64_t)blockIdx.x * SCAN_B + threadIdx.x;
  int64_t v = i < n ? (int64_t)in[i] : 0;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int64_t x = v;
  for (int o = 1; o < 32; o <<= 1) {
    int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) ws[w] = x;
  __syncthreads();
  if (w == 0) {
    int64_t t = ws[lane];
    for (int o = 1; o < 32; o <<= 1) {
      int64_t y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    ws[lane] = t;
  }
  __syncthreads();
  const int64_t incl = x + (w > 0 ? ws[w - 1] : 0);
  if (i < n) out[i] = incl - v;
  if (threadIdx.x == SCAN_B - 1) sums[blockIdx.x] = incl;
}
__global__ void __launch_bounds__(SCAN_B) k_scan_sums(int64_t* sums, int64_t nb) {
  // exclusive scan of the block sums in one CTA (sequential over chunks of SCAN_B)
  __shared__ int64_t ws[32];
  __shared__ int64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < nb; base += SCAN_B) {
    const int64_t i = base + threadIdx.x;
    int64_t v = i < nb ? sums[i] : 0;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
      int64_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) ws[w] = x;
    __syncthreads();
    if (w == 0) {
      int64_t t = ws[lane];
      for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, t, o);
        if (lane >= o) t += y;
      }
      ws[lane] = t;
    }
    __syncthreads();
    const int64_t incl = x + (w > 0 ? ws[w - 1] : 0);
    if (i < nb) sums[i] = carry + incl - v;
    __syncthreads();
    if (threadIdx.x == SCAN_B - 1) carry += incl;
    __syncthreads();
  }
}
__global__ void k_scan_add(int64_t* out, int64_t n, const int64_t* sums, int64_t total_slot) {
  const int64_t i = (int64_t)blockIdx.x * SCAN_B + threadIdx.x;
  if (i < n) out[i] += sums[blockIdx.x];
  (void)total_slot;
}
__global__ void k_set_total(int64_t* out, int64_t n, const int64_t* last_in, const unsigned long long* cnt) {
  out[n] = out[n - 1] + (int64_t)cnt[n - 1];
  (void)last_in;
}

// one warp per source row: its entries go to the cursor positions of their columns
template <class E>
__global__ void k_scatter_rows(const int64_t* rp, const int32_t* ci, const E* val, int64_t rows, int64_t* cursor,
                               int32_t* ciT, E* valT) {
  const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
  const int lane = threadIdx.x & 31;
  if (r >= rows) return;
  for (int64_t e = rp[r] + lane; e < rp[r + 1]; e += 32) {
    const int64_t pos = (int64_t)atomicAdd((unsigned long long*)&cursor[ci[e]], 1ull);
    ciT[pos] = (int32_t)r;
    valT[pos] = val[e];
  }
}

// The CSR structure a problem is created from, before any kernel indexes with it: row_ptr starts at
// 0, never decreases and ends at nnz, and every row's column indices lie in [0, cols) and increase
// strictly.  One thread per row; a row's columns are read only once its range has been checked.
// A violation records DEV_BOUNDS in the status word.
__global__ void k_csr_check(const int64_t* rp, const int32_t* ci, int64_t rows, int64_t cols, int64_t nnz,
                            int* status) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = rp[r], b = rp[r + 1];
    if (a < 0 || b < a || b > nnz || (r == 0 && a != 0) || (r == rows - 1 && b != nnz)) {
      dev_fail(status, DEV_BOUNDS);
      continue;
    }
    int32_t prev = -1;
    for (int64_t k = a; k < b; ++k) {
      const int32_t c = ci[k];
      if (c <= prev || c >= cols) {
        dev_fail(status, DEV_BOUNDS);
        break;
      }
      prev = c;
    }
  }
}

cudaError_t launch_csr_check(const int64_t* rp, const int32_t* ci, int64_t rows, int64_t cols, int64_t nnz,
                             int* status, cudaStream_t st) {
  const int64_t blocks = std::min<int64_t>((rows + 255) / 256, 4096);
  k_csr_check<<<(unsigned)std::max<int64_t>(1, blocks), 256, 0, st>>>(rp, ci, rows, cols, nnz, status);
  return cudaGetLastError();
}

cudaError_t launch_csr_transpose(ihsbin_problem* p, const int64_t* rp, const int32_t* ci, const void* val, int elem,
                                 int64_t rows, int64_t cols, int64_t nnz, int64_t** rpT, int32_t** ciT, void** valT,
                                 cudaStream_t st) {
  const size_t es = elem == ELEM_F64 ? 8 : elem == ELEM_F32 ? 4 : 2;
  unsigned long long* cnt = nullptr;
  int64_t* sums = nullptr;
  int64_t* cursor = nullptr;
  const int64_t nb = (cols + SCAN_B - 1) / SCAN_B;
  CK(prob_alloc(p, (size_t)(cols + 1) * 8, (void**)rpT, SCOPE_PERSIST));
  CK(prob_alloc(p, (size_t)std::max<int64_t>(1, nnz) * 4, (void**)ciT, SCOPE_PERSIST));
  CK(prob_alloc(p, (size_t)std::max<int64_t>(1, nnz) * es, valT, SCOPE_PERSIST));
  CK(prob_alloc(p, (size_t)cols * 8, (void**)&cnt, SCOPE_SCRATCH));
  CK(prob_alloc(p, (size_t)std::max<int64_t>(1, nb) * 8, (void**)&sums, SCOPE_SCRATCH));
  CK(prob_alloc(p, (size_t)cols * 8, (void**)&cursor, SCOPE_SCRATCH));
  CK(cudaMemsetAsync(cnt, 0, (size_t)cols * 8, st));
  {
    KTimer kt(p, K_SPARSE, st, 0, (double)nnz * 4);
    k_count_cols<<<nblk(nnz, 256) > 65535 * 8 ? 65535 * 8 : nblk(nnz, 256), 256, 0, st>>>(ci, nnz, cnt);
  }
  CK(cudaGetLastError());
  {
    KTimer kt(p, K_SPARSE, st, 0, (double)cols * 16);
    k_scan_blocks<<<(unsigned)nb, SCAN_B, 0, st>>>(cnt, cols, *rpT, sums);
    k_scan_sums<<<1, SCAN_B, 0, st>>>(sums, nb);
    k_scan_add<<<(unsigned)nb, SCAN_B, 0, st>>>(*rpT, cols, sums, cols);
    k_set_total<<<1, 1, 0, st>>>(*rpT, cols, nullptr, cnt);
  }
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(cursor, *rpT, (size_t)cols * 8, cudaMemcpyDeviceToDevice, st));
  {
    KTimer kt(p, K_SPARSE, st, 0, (double)nnz * (8 + 2 * es));
    const unsigned g = nblk(rows * 32, 256);
    if (es == 8)
      k_scatter_rows<double><<<g, 256, 0, st>>>(rp, ci, (const double*)val, rows, cursor, *ciT, (double*)*valT);
    else if (es == 4)
      k_scatter_rows<float><<<g, 256, 0, st>>>(rp, ci, (const float*)val, rows, cursor, *ciT, (float*)*valT);
    else
      k_scatter_rows<uint16_t><<<g, 256, 0, st>>>(rp, ci, (const uint16_t*)val, rows, cursor, *ciT,
                                                  (uint16_t*)*valT);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------- Gram
// one warp per row: all pairs (a <= b) of its nonzeros into the upper triangle
__global__ void k_csr_gram_pairs(const int64_t* rp, const int32_t* ci, const void* val, int elem, int64_t rows,
                                 int64_t D, double* G) {
  const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
  const int lane = threadIdx.x & 31;
  if (r >= rows) return;
  const int64_t e0 = rp[r];
  const int64_t n = rp[r + 1] - e0;
  const int64_t npairs = n * (n + 1) / 2;
  for (int64_t q = lane; q < npairs; q += 32) {
    // pair index q -> (a, b) with a <= b: row a of the upper triangle starts at a*n - a(a-1)/2
    int64_t a = (int64_t)((2.0 * n + 1.0 - sqrt((2.0 * n + 1.0) * (2.0 * n + 1.0) - 8.0 * (double)q)) / 2.0);
    if (a < 0) a = 0;
    while (a > 0 && a * n - a * (a - 1) / 2 > q) --a;
    while ((a + 1) * n - (a + 1) * a / 2 <= q) ++a;
    const int64_t b = a + (q - (a * n - a * (a - 1) / 2));
    const int64_t ca = ci[e0 + a], cb = ci[e0 + b];
    const double v = load_elem_d(val, elem, e0 + a) * load_elem_d(val, elem, e0 + b);
    const int64_t lo = ca < cb ? ca : cb, hi = ca < cb ? cb : ca;
    atomicAdd(&G[lo * D + hi], v);
  }
}

template <class Mode>
__global__ void k_mirror_upper(const double* Gu, int64_t D, CBuf G) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= D * D) return;
  const int64_t i = e / D, j = e % D;
  const double v = i <= j ? Gu[i * D + j] : Gu[j * D + i];
  Mode::st(G, e, Mode::from_d(v));
}

cudaError_t csr_gram(ihsbin_problem* p, int compute, cudaStream_t st) {
  const Tall& A = p->A;
  const int64_t D = A.D;
  double* Gu = nullptr;
  CK(prob_alloc(p, (size_t)D * D * 8, (void**)&Gu, SCOPE_SCRATCH));
  CK(cudaMemsetAsync(Gu, 0, (size_t)D * D * 8, st));
  const double es = A.elem == ELEM_F64 ? 8 : A.elem == ELEM_F32 ? 4 : 2;
  {
    // algorithmic work: one multiply-add per nonzero pair of every row
    const double pairs = (double)A.nnz * ((double)A.nnz / std::max<int64_t>(1, A.N) + 1) / 2.0;
    KTimer kt(p, K_GRAM, st, 2.0 * pairs, A.nnz * (es + 4) + 8.0 * (A.N + 1) + (double)D * D * 8);
    k_csr_gram_pairs<<<nblk(A.N * 32, 256), 256, 0, st>>>(A.rp, A.ci, A.val, A.elem, A.N, D, Gu);
  }
  CK(cudaGetLastError());
  KTimer kt(p, K_GRAM, st, 0, (double)D * D * 16);
  if (compute == IHSBIN_COMPUTE_F64) k_mirror_upper<F64><<<nblk(D * D, 256), 256, 0, st>>>(Gu, D, p->G);
  else k_mirror_upper<DD><<<nblk(D * D, 256), 256, 0, st>>>(Gu, D, p->G);
  return cudaGetLastError();
}

// ----------------------------------------------------------------------- rhs
template <class Mode>
__device__ __forceinline__ typename Mode::V warp_sum(typename Mode::V v);
template <>
__device__ __forceinline__ double warp_sum<F64>(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <>
__device__ __forceinline__ dd warp_sum<DD>(dd v) {
  for (int o = 16; o > 0; o >>= 1) {
    dd w{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
    v = dd_add(v, w);
  }
  return v;
}

// c[r*D + i] = sum_e valT[e] * B[ciT[e]][r]: one warp per row i of A_hat^T
template <class Mode>
__global__ void k_csr_rhs(const int64_t* rpT, const int32_t* ciT, const void* valT, int elem, int64_t D,
                          const double* B, int64_t K, CBuf c) {
  const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
  const int lane = threadIdx.x & 31;
  if (i >= D) return;
  for (int64_t r = 0; r < K; ++r) {
    typename Mode::V acc = Mode::zero();
    for (int64_t e = rpT[i] + lane; e < rpT[i + 1]; e += 32)
      acc = Mode::add(acc, Mode::mul(Mode::from_d(load_elem_d(valT, elem, e)), Mode::from_d(B[(int64_t)ciT[e] * K + r])));
    acc = warp_sum<Mode>(acc);
    if (lane == 0) Mode::st(c, r * D + i, acc);
  }
}

cudaError_t csr_rhs(ihsbin_problem* p, int compute, CBuf c, cudaStream_t st) {
  const Tall& A = p->A;
  const double es = A.elem == ELEM_F64 ? 8 : A.elem == ELEM_F32 ? 4 : 2;
  KTimer kt(p, K_RHS, st, 2.0 * A.nnz * p->K, A.nnz * (es + 4) + 8.0 * (A.D + 1));
  const unsigned g = nblk(A.D * 32, 256);
  if (compute == IHSBIN_COMPUTE_F64)
    k_csr_rhs<F64><<<g, 256, 0, st>>>(A.rpT, A.ciT, A.valT, A.elem, A.D, p->B, p->K, c);
  else
    k_csr_rhs<DD><<<g, 256, 0, st>>>(A.rpT, A.ciT, A.valT, A.elem, A.D, p->B, p->K, c);
  return cudaGetLastError();
}

// ----------------------------------------------------------------- dual map
// W_l[col*N + r] = sum_e val[e] * Ut_l[col*D + ci[e]] for every interval l and basis column col.
// One warp per row r of A_hat; lane c takes the basis columns c, c + 32, ... of all intervals and
// walks the row's nonzeros itself (broadcast loads, no cross-lane sums), reading the basis from a
// transposed copy UtT[k][column] so that the lanes' loads are contiguous.
template <class Mode>
__global__ void k_transpose_basis(CBuf Ut, int64_t D, int64_t nc, CBuf UtT) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // over D x nc, column fastest
  if (e >= D * nc) return;
  const int64_t k = e / nc, c = e - k * nc;
  Mode::st(UtT, e, Mode::ld(Ut, c * D + k));
}
template <class Mode>
__device__ __forceinline__ void mac_elem(typename Mode::V& acc, const void* val, int elem, int64_t e,
                                         typename Mode::V u) {
  if (elem == ELEM_F32) Mode::mac(acc, ((const float*)val)[e], u);  // an exact float operand
  else if (elem == ELEM_BF16) Mode::mac(acc, __uint_as_float((uint32_t)((const uint16_t*)val)[e] << 16), u);
  else acc = Mode::add(acc, Mode::mul(Mode::from_d(((const double*)val)[e]), u));
}
template <class Mode>
__global__ void k_csr_dual_map(const int64_t* rp, const int32_t* ci, const void* val, int elem, int64_t N, int64_t nc,
                               CBuf UtT, CBuf W) {
  const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
  const int lane = threadIdx.x & 31;
  if (r >= N) return;
  const int64_t e0 = rp[r], e1 = rp[r + 1];
  for (int64_t c = lane; c < nc; c += 32) {
    typename Mode::V acc = Mode::zero();
    for (int64_t e = e0; e < e1; ++e) {
      mac_elem<Mode>(acc, val, elem, e, Mode::ld(UtT, (int64_t)ci[e] * nc + c));
      if (((e - e0) & 31) == 31) acc = Mode::renorm(acc);
    }
    Mode::st(W, c * N + r, Mode::renorm(acc));
  }
}

// WT[k][c] = W[c][k] for nc columns of length d (the CSR image kernel's operand layout)
cudaError_t basis_transpose(ihsbin_problem* p, int compute, CBuf W, int64_t d, int64_t nc, CBuf WT, cudaStream_t st) {
  KTimer kt(p, K_LOSS_IMAGE, st, 0, 16.0 * d * nc);
  if (compute == IHSBIN_COMPUTE_F64) k_transpose_basis<F64><<<nblk(d * nc, 256), 256, 0, st>>>(W, d, nc, WT);
  else k_transpose_basis<DD><<<nblk(d * nc, 256), 256, 0, st>>>(W, d, nc, WT);
  return cudaGetLastError();
}

// V[c][i] = sum_e val[e] W[c][ci[e]] for the n_rows rows of a CSR matrix (row_ptr rp, absolute
// offsets into ci / val) and nc basis columns given transposed (WT[k][c]): a loss's image of the basis.
cudaError_t csr_basis_image(ihsbin_problem* p, int compute, const int64_t* rp, const int32_t* ci, const void* val,
                            int64_t n_rows, CBuf WT, int64_t nc, CBuf V, cudaStream_t st) {
  const Tall& A = p->A;
  const double es = A.elem == ELEM_F64 ? 8 : A.elem == ELEM_F32 ? 4 : 2;
  KTimer kt(p, K_LOSS_IMAGE, st, 0, 8.0 * nc * n_rows + (es + 4) * (double)A.nnz * n_rows / std::max<int64_t>(1, p->n));
  const unsigned g = nblk(n_rows * 32, 256);
  if (compute == IHSBIN_COMPUTE_F64) k_csr_dual_map<F64><<<g, 256, 0, st>>>(rp, ci, val, A.elem, n_rows, nc, WT, V);
  else k_csr_dual_map<DD><<<g, 256, 0, st>>>(rp, ci, val, A.elem, n_rows, nc, WT, V);
  return cudaGetLastError();
}

cudaError_t csr_dual_map(ihsbin_problem* p, int compute, int64_t ncol, cudaStream_t st) {
  const Tall& A = p->A;
  const int L = p->plan.L;
  const int64_t nc = ncol * L, D = A.D;
  const double es = A.elem == ELEM_F64 ? 8 : A.elem == ELEM_F32 ? 4 : 2;
  cudaError_t err = cudaSuccess;
  CBuf UtT = alloc_cbuf(p, compute, (size_t)D * nc, SCOPE_SCRATCH, &err);
  if (err != cudaSuccess) return err;
  KTimer kt(p, K_DUAL_MAP, st, 2.0 * A.nnz * nc, A.nnz * (es + 4) + 8.0 * nc * A.N);
  const unsigned g = nblk(A.N * 32, 256);
  if (compute == IHSBIN_COMPUTE_F64) {
    k_transpose_basis<F64><<<nblk(D * nc, 256), 256, 0, st>>>(p->Ut, D, nc, UtT);
    k_csr_dual_map<F64><<<g, 256, 0, st>>>(A.rp, A.ci, A.val, A.elem, A.N, nc, UtT, p->W);
  } else {
    k_transpose_basis<DD><<<nblk(D * nc, 256), 256, 0, st>>>(p->Ut, D, nc, UtT);
    k_csr_dual_map<DD><<<g, 256, 0, st>>>(A.rp, A.ci, A.val, A.elem, A.N, nc, UtT, p->W);
  }
  return cudaGetLastError();
}

}  // namespace ihsbin
