// QTT mat-vec for callers that cannot allocate device memory.
//
// qtt_apply_f32_noalloc() computes y = A x like qtt_apply(), but needs no
// context and never allocates: its two intermediate buffers live in the
// file-scope device array below, which every GPU that loads this library holds
// until the process exits.  Code running where cudaMalloc is not available or
// not allowed (inside a host callback, a plugin of a host application that owns
// the device memory pool, or a caller that has to run with a fixed device
// footprint) can still apply a QTT matrix, passing only its own input and output
// buffers.
#include <mutex>

#include "internal.cuh"
#include "qtt_dev.cuh"

namespace qp {
namespace {

// Two buffers of QTT_NOALLOC_MAX_VALUES floats each (2 x 16 MiB).
constexpr long long kNoallocValues = QTT_NOALLOC_MAX_VALUES;
static __device__ __align__(256) float g_qtt_noalloc_scratch[2 * kNoallocValues];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
float* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the static scratch for the current device, looked up once
// per device (the array's host-side name is only a stand-in, never a pointer).
int noalloc_scratch(float** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return QP_CUDA_ERROR;
  if (dev < 0 || dev >= kMaxDevices) return QP_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_qtt_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return QP_CUDA_ERROR;
    }
    g_scratch_ptr[dev] = static_cast<float*>(p);
  }
  *out = g_scratch_ptr[dev];
  return QP_OK;
}

__global__ void k_qtt_step_noalloc(QttDev q, int k, const float* in, float* out, long long items) {
  const long long gsz = (long long)gridDim.x * blockDim.x;
  for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < items; it += gsz)
    qtt_step_any<float, float, float>(q, k, in, out, it);
}

}  // namespace
}  // namespace qp

extern "C" int qtt_apply_f32_noalloc(int d, const int* ranks_host, const float* cores, const float* x, float* y,
                                     void* cuda_stream) {
  using namespace qp;
  if (d < 1 || d > 40 || !ranks_host || !cores || !x || !y || x == y) return QP_INVALID_ARG;
  if (ranks_host[0] != 1 || ranks_host[d] != 1) return QP_INVALID_ARG;
  QttDev q;
  q.d = d;
  q.rmax = 1;
  long long off = 0;
  for (int k = 0; k <= d; ++k) {
    if (ranks_host[k] < 1) return QP_INVALID_ARG;
    q.ranks[k] = ranks_host[k];
    if (ranks_host[k] > q.rmax) q.rmax = ranks_host[k];
    q.off[k] = off;
    if (k < d) off += (long long)ranks_host[k] * 4 * ranks_host[k + 1];
  }
  q.cores = cores;
  const long long N = 1LL << d;
  // every intermediate Z_k holds r_{k-1} * 2^d values; both buffers must fit
  if ((long long)q.rmax * N > kNoallocValues) return QP_INVALID_ARG;
  float* scratch = nullptr;
  int rc = noalloc_scratch(&scratch);
  if (rc != QP_OK) return rc;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return QP_CUDA_ERROR;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return QP_CUDA_ERROR;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  float* w0 = scratch;
  float* w1 = scratch + kNoallocValues;
  const long long items = N >> 1;
  long long blocks = (items + 255) / 256;
  if (blocks > (long long)sms * 16) blocks = (long long)sms * 16;
  if (blocks < 1) blocks = 1;
  const float* in = x;
  for (int k = d; k >= 1; --k) {
    float* out = (k == 1) ? y : (((d - k) & 1) ? w1 : w0);
    // cudaLaunchKernel returns this launch's own status: an earlier error of the
    // caller is neither reported as ours nor cleared
    void* args[] = {&q, &k, (void*)&in, &out, (void*)&items};
    if (cudaLaunchKernel((const void*)k_qtt_step_noalloc, dim3((unsigned)blocks), dim3(256), args, 0, st) !=
        cudaSuccess)
      return QP_CUDA_ERROR;
    in = out;
  }
  return QP_OK;
}
