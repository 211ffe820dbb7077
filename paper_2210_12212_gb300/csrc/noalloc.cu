// ihsbin_sketch_gram_noalloc: the Gram matrix G_S = (S A)^T (S A) of a sketch,
// computed without any device allocation.
//
// Who needs it: callers that cannot call cudaMalloc at the point where they
// need G_S -- callers on a latency budget that cannot absorb cudaMalloc or
// cudaFree (either may synchronise the whole device and stall other streams),
// and hosts that hand all device memory to their own pool (a framework's
// caching allocator, a fixed arena sized at start-up) and forbid allocations
// by libraries, so that a library allocation would fail or break the pool's
// accounting.  The regular path (ihsbin_sketch) allocates its split-K
// partial sums per call; this variant keeps them in one file-scope device
// array instead.
//
// The scratch array: IHSBIN_NOALLOC_SCRATCH_BYTES (16 MiB) of device memory,
// reserved by every GPU that loads the library until the process exits.  All
// calls share it, and it keeps whatever the last call left there, so calls
// that overlap on the GPU (different streams, or different host threads on the
// same device) race on it: serialise them.  Nothing in it has to start at zero:
// every partial sum the reduction reads is written by the same call first.
//
// Set-up: the first call on a device (with that device current) looks up the
// array's device address with cudaGetSymbolAddress and caches it for that
// device; make that first call before any stream capture begins.
#include <mutex>

#include "gemm.cuh"
#include "internal.h"

namespace ihsbin {
namespace {

constexpr size_t kScratchBytes = IHSBIN_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_scratch[kScratchBytes / sizeof(double)];

std::mutex g_setup_mu;
double* g_scratch_ptr[kMaxDevices] = {};

// operand (i, k) = SA[k][i]  (column i of SA, reduction over the m rows)
struct LdSAt {
  using T = double;
  static constexpr bool k_contig = false;
  const double* SA;
  int64_t D;
  __device__ __forceinline__ T operator()(int, int64_t i, int64_t k) const { return SA[k * D + i]; }
};
// operand (k, j) = SA[k][j]
struct LdSA {
  using T = double;
  static constexpr bool k_contig = false;
  const double* SA;
  int64_t D;
  __device__ __forceinline__ T operator()(int, int64_t k, int64_t j) const { return SA[k * D + j]; }
};
// partial sum of split s: part[(s * D + j) * D + i]
struct EpPart {
  double* part;
  int64_t D;
  __device__ __forceinline__ void operator()(int, int s, int64_t i, int64_t j, double a) const {
    part[((int64_t)s * D + j) * D + i] = a;
  }
};
// G[i][j] = G[j][i] = sum over the splits, for i <= j (every such entry was written by this call)
__global__ void k_reduce_upper(const double* part, int S, int64_t D, double* G) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= D * D) return;
  const int64_t i = e / D, j = e % D;
  if (i > j) return;
  double v = 0.0;
  for (int s = 0; s < S; ++s) v += part[((int64_t)s * D + j) * D + i];
  G[i * D + j] = v;
  G[j * D + i] = v;
}

ihsbin_status noalloc_fail(ihsbin_status s, const char* msg) {
  set_last_error(msg);
  return s;
}

}  // namespace
}  // namespace ihsbin

using namespace ihsbin;

extern "C" IHSBIN_API ihsbin_status ihsbin_sketch_gram_noalloc(const double* SA, int64_t m, int64_t D, double* GS,
                                                               void* stream) {
  if (!SA || !GS) return noalloc_fail(IHSBIN_ERR_INVALID_ARG, "sketch_gram_noalloc: NULL pointer");
  if (m <= 0 || D <= 0) return noalloc_fail(IHSBIN_ERR_INVALID_ARG, "sketch_gram_noalloc: m and D must be positive");
  const size_t cap = kScratchBytes / sizeof(double);
  if ((size_t)D > cap / (size_t)D)  // D * D > cap, without forming a product that could wrap
    return noalloc_fail(IHSBIN_ERR_INVALID_ARG,
                        "sketch_gram_noalloc: D*D partial sums exceed the 16 MiB scratch array (D <= 1448)");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return noalloc_fail(IHSBIN_ERR_CUDA, "sketch_gram_noalloc: no current CUDA device");
  double* scratch;
  {
    std::lock_guard<std::mutex> g(g_setup_mu);
    if (!g_scratch_ptr[dev]) {
      void* ptr = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (e != cudaSuccess || !ptr)
        return noalloc_fail(IHSBIN_ERR_CUDA, "sketch_gram_noalloc: cudaGetSymbolAddress of the scratch array failed");
      g_scratch_ptr[dev] = (double*)ptr;
    }
    scratch = g_scratch_ptr[dev];
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t tm = (D + 63) / 64;
  GemmShape sh{D, D, m, 1};
  int ks = pick_split(tm * (tm + 1) / 2, m, 16);
  const int64_t fit = (int64_t)(cap / ((size_t)D * (size_t)D));
  if (ks > fit) ks = (int)fit;
  sh.ksplit = ks < 1 ? 1 : ks;
  cudaError_t e = launch_gemm<F64, 64, 64, 16, 4, 4>(sh, 1, LdSAt{SA, D}, LdSA{SA, D}, EpPart{scratch, D}, st);
  if (e == cudaSuccess) {
    k_reduce_upper<<<(unsigned)((D * D + 255) / 256), 256, 0, st>>>(scratch, sh.ksplit, D, GS);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return noalloc_fail(IHSBIN_ERR_CUDA, cudaGetErrorString(e));
  return IHSBIN_OK;
}
