// oci_noalloc.cu -- convergence norm ||a - b||_2 that allocates nothing.
//
// Some callers cannot allocate device memory at the moment they need the norm:
// code running inside a caching allocator's callback, a real-time loop whose
// memory is budgeted once at start-up, or an application whose device memory is
// owned by another framework.  For them this file keeps the per-block partial
// sums in a fixed file-scope device array instead of memory from cudaMalloc.
//
// Scratch: kNoallocMaxBlocks FP64 partials (128 KiB), one per block of
// kNoallocChunk elements, so n is limited to kNoallocMaxBlocks * kNoallocChunk
// = 33,554,432 elements.  Every GPU that loads the library holds the array until
// the process exits.  Each call writes every slot it reads, so nothing has to
// be cleared between calls; calls that overlap on the GPU (different streams,
// same device) share the array and race.
//
// In host code the array's name does not denote a device address; its device
// address is obtained once per device with cudaGetSymbolAddress (on the first
// call made with that device current) and passed to the kernels.  The cached
// address belongs to the device's primary context: after cudaDeviceReset the
// entry point must not be called again in that process.
#include <math.h>

#include <mutex>

#include "oci_internal.h"

namespace oci {
namespace {

constexpr int kNoallocChunk = 2048;       // elements summed by one block
constexpr int kNoallocThreads = 256;
constexpr int kNoallocMaxBlocks = 16384;  // 128 KiB of partials
constexpr int kNoallocMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_partials[kNoallocMaxBlocks];

// Block i sums (a-b)^2 over elements [i*chunk, min(n, (i+1)*chunk)) in a fixed order.
__global__ void __launch_bounds__(kNoallocThreads) k_noalloc_partials(const double *__restrict__ a,
                                                                      const double *__restrict__ b, long long n,
                                                                      double *__restrict__ partials) {
  __shared__ double red[kNoallocThreads / 32];
  const long long base = (long long)blockIdx.x * kNoallocChunk;
  double s = 0.0;
  for (int k = threadIdx.x; k < kNoallocChunk; k += kNoallocThreads) {
    const long long i = base + k;
    if (i < n) {
      const double d = a[i] - b[i];
      s = fma(d, d, s);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kNoallocThreads / 32; w++) t += red[w];
    partials[blockIdx.x] = t;
  }
}

// One block: fixed-order sum of the nb partials, then the square root.
__global__ void __launch_bounds__(512) k_noalloc_final(const double *__restrict__ partials, int nb,
                                                       double *__restrict__ out) {
  __shared__ double sh[512];
  double s = 0.0;
  for (int i = threadIdx.x; i < nb; i += 512) s += partials[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = 256; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sqrt(sh[0]);
}

std::mutex g_noalloc_mu;
double *g_noalloc_ptr[kNoallocMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (set up once).
int noalloc_scratch(double **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kNoallocMaxDevices) return set_error("device index beyond the supported range"), OCI_E_INVAL;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    double *p = nullptr;
    e = cudaGetSymbolAddress((void **)&p, g_noalloc_partials);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(norm scratch)");
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return OCI_OK;
}

}  // namespace
}  // namespace oci

extern "C" int oci_diff_norm_noalloc(const double *a, const double *b, int64_t n, double *e_out, void *stream) {
  using namespace oci;
  if (!a || !b || !e_out) return set_error("a, b and e_out must be device pointers"), OCI_E_INVAL;
  if (n < 0) return set_error("n must be >= 0"), OCI_E_INVAL;
  const long long max_n = (long long)kNoallocMaxBlocks * kNoallocChunk;
  if (n > max_n) return set_error("n exceeds the 33,554,432 elements the fixed scratch array covers"), OCI_E_INVAL;
  double *scratch = nullptr;
  int rc = noalloc_scratch(&scratch);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const int nb = (int)((n + kNoallocChunk - 1) / kNoallocChunk);
  if (nb > 0) k_noalloc_partials<<<nb, kNoallocThreads, 0, st>>>(a, b, (long long)n, scratch);
  k_noalloc_final<<<1, 512, 0, st>>>(scratch, nb, e_out);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "oci_diff_norm_noalloc launch");
  return OCI_OK;
}
