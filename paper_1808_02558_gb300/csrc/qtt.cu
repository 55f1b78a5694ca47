// QTT matrices: storage, mat-vec (Sec. 3.2), and the C-ABI glue for rounding,
// compression and inversion (implemented in qtt_linalg.cu).
#include <cstring>

#include "internal.cuh"
#include "qtt_dev.cuh"

namespace qp {
namespace {

constexpr int QTT_GCAP = 4 * 16 * 16;  // staged core values (ranks up to 16)

template <class TV, class TA, class TC>
__global__ void k_qtt_step(QttDev q, int k, const TV* in, TV* out, long long items) {
  __shared__ TA gc[QTT_GCAP];
  qtt_step_grid<TV, TA, TC>(q, k, in, out, items, gc, QTT_GCAP);
}

__global__ void k_to_f32(const double* __restrict__ a, float* __restrict__ b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}
__global__ void k_to_bf16(const double* __restrict__ a, __nv_bfloat16* __restrict__ b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    b[i] = __float2bfloat16_rn((float)a[i]);
}

}  // namespace

qp_qtt* qtt_alloc(qp_ctx* c, int d, const std::vector<int>& ranks) {
  QP_REQUIRE(d >= 1 && d <= 64, QP_INVALID_ARG, "QTT: d must be in [1, 64]");
  QP_REQUIRE((int)ranks.size() == d + 1 && ranks[0] == 1 && ranks[d] == 1, QP_INVALID_ARG,
             "QTT: ranks must have d+1 entries with r_0 = r_d = 1");
  qp_qtt* A = new qp_qtt();
  A->ctx = c;
  A->d = d;
  A->ranks = ranks;
  A->offset.assign(d + 1, 0);
  long long off = 0;
  for (int k = 0; k < d; ++k) {
    if (ranks[k] < 1 || ranks[k + 1] < 1) {
      delete A;
      throw Error{QP_INVALID_ARG, "QTT: ranks must be >= 1"};
    }
    A->offset[k] = off;
    off += (long long)ranks[k] * 4 * ranks[k + 1];
  }
  A->offset[d] = off;
  A->nvals = off;
  cudaError_t e = cudaMalloc(&A->cores, (size_t)off * sizeof(double));
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete A;
    throw Error{QP_OOM, "QTT: core allocation failed"};
  }
  return A;
}

static void qtt_release(qp_qtt* A) {
  if (!A) return;
  if (A->cores) cudaFree(A->cores);
  if (A->cores32) cudaFree(A->cores32);
  if (A->cores16) cudaFree(A->cores16);
  delete A;
}

void qtt_prepare_copies(qp_ctx* c, qp_qtt* A, qp_dtype dt) {
  if (dt == QP_F32 && !A->cores32) {
    QP_CUDA(cudaMalloc(&A->cores32, (size_t)A->nvals * sizeof(float)));
    k_to_f32<<<c->num_sms * 4, 256, 0, c->stream>>>(A->cores, A->cores32, A->nvals);
    QP_CUDA(cudaGetLastError());
  }
  if (dt == QP_BF16 && !A->cores16) {
    QP_CUDA(cudaMalloc(&A->cores16, (size_t)A->nvals * sizeof(__nv_bfloat16)));
    k_to_bf16<<<c->num_sms * 4, 256, 0, c->stream>>>(A->cores, A->cores16, A->nvals);
    QP_CUDA(cudaGetLastError());
  }
}

static QttDev dev_view(qp_qtt* A, const void* cores) {
  QttDev q;
  q.d = A->d;
  q.rmax = 1;
  for (int k = 0; k <= A->d; ++k) {
    q.ranks[k] = A->ranks[k];
    q.off[k] = A->offset[k];
    if (A->ranks[k] > q.rmax) q.rmax = A->ranks[k];
  }
  q.cores = cores;
  return q;
}

// y = A x: d launches of the column step, ping-ponging between two work buffers.
void launch_qtt_apply(qp_ctx* c, qp_qtt* A, const void* x, void* y, qp_dtype cdt, qp_dtype vdt) {
  QP_REQUIRE(vdt == QP_F64 || vdt == QP_F32, QP_INVALID_ARG, "qtt_apply: vector dtype must be F64 or F32");
  QP_REQUIRE(!(vdt == QP_F64 && cdt != QP_F64), QP_INVALID_ARG, "qtt_apply: F64 vectors need F64 cores");
  QP_REQUIRE(cdt == QP_F64 || cdt == QP_F32 || cdt == QP_BF16, QP_INVALID_ARG, "qtt_apply: bad core dtype");
  qtt_prepare_copies(c, A, cdt);
  const void* cores = cdt == QP_F64 ? (const void*)A->cores
                                    : (cdt == QP_F32 ? (const void*)A->cores32 : (const void*)A->cores16);
  QttDev q = dev_view(A, cores);
  const long long N = 1LL << A->d;
  const size_t es = vdt == QP_F64 ? sizeof(double) : sizeof(float);
  void* w0 = c->scratch[5].ensure((size_t)N * q.rmax * es);
  void* w1 = c->scratch[6].ensure((size_t)N * q.rmax * es);
  const long long items = N >> 1;
  // two columns per thread
  long long want = (items + 511) / 512;
  if (want > (long long)c->num_sms * 16) want = (long long)c->num_sms * 16;
  const int grid = (int)(want < 1 ? 1 : want);
  const void* in = x;
  for (int k = A->d; k >= 1; --k) {
    void* out = (k == 1) ? y : (((A->d - k) & 1) ? w1 : w0);
    if (vdt == QP_F64) {
      k_qtt_step<double, double, double><<<grid, 256, 0, c->stream>>>(q, k, static_cast<const double*>(in),
                                                                       static_cast<double*>(out), items);
    } else if (cdt == QP_F32) {
      k_qtt_step<float, float, float><<<grid, 256, 0, c->stream>>>(q, k, static_cast<const float*>(in),
                                                                   static_cast<float*>(out), items);
    } else if (cdt == QP_BF16) {
      k_qtt_step<float, float, __nv_bfloat16><<<grid, 256, 0, c->stream>>>(q, k, static_cast<const float*>(in),
                                                                           static_cast<float*>(out), items);
    } else {
      k_qtt_step<float, float, double><<<grid, 256, 0, c->stream>>>(q, k, static_cast<const float*>(in),
                                                                    static_cast<float*>(out), items);
    }
    QP_CUDA(cudaGetLastError());
    in = out;
  }
}

}  // namespace qp

using namespace qp;

extern "C" {

int qtt_from_host(qp_ctx_t c, int d, const int* ranks_host, const double* cores_host, qtt_t* out) {
  if (!c || !ranks_host || !cores_host || !out) return QP_INVALID_ARG;
  try {
    QP_CUDA(cudaSetDevice(c->device));
    std::vector<int> r(ranks_host, ranks_host + d + 1);
    qp_qtt* A = qtt_alloc(c, d, r);
    cudaError_t e = cudaMemcpy(A->cores, cores_host, (size_t)A->nvals * sizeof(double), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      qtt_release(A);
      throw Error{QP_CUDA_ERROR, std::string("qtt_from_host: ") + cudaGetErrorString(e)};
    }
    *out = A;
  } catch (const Error& e) {
    set_error(c, e);
    return e.code;
  }
  return QP_OK;
}

int qtt_free(qp_ctx_t c, qtt_t A) {
  if (!c || !A) return QP_INVALID_ARG;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  qtt_release(A);
  return QP_OK;
}

int qtt_get_dims(qtt_t A, int* d, long long* nvals) {
  if (!A) return QP_INVALID_ARG;
  if (d) *d = A->d;
  if (nvals) *nvals = A->nvals;
  return QP_OK;
}

int qtt_get_ranks(qtt_t A, int* ranks) {
  if (!A || !ranks) return QP_INVALID_ARG;
  for (int k = 0; k <= A->d; ++k) ranks[k] = A->ranks[k];
  return QP_OK;
}

int qtt_copy_cores_to_host(qtt_t A, double* out) {
  if (!A || !out) return QP_INVALID_ARG;
  qp_ctx* c = A->ctx;
  cudaSetDevice(c->device);
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return QP_CUDA_ERROR;
  if (cudaMemcpy(out, A->cores, (size_t)A->nvals * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
    return QP_CUDA_ERROR;
  return QP_OK;
}

int qtt_apply(qp_ctx_t c, qtt_t A, const void* x, void* y, qp_dtype cdt, qp_dtype vdt) {
  if (!c || !A || !x || !y || x == y) return QP_INVALID_ARG;
  try {
    QP_CUDA(cudaSetDevice(c->device));
    launch_qtt_apply(c, A, x, y, cdt, vdt);
  } catch (const Error& e) {
    set_error(c, e);
    return e.code;
  }
  return QP_OK;
}

}  // extern "C"
