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

constexpr int QTT_GQ = 2 * 12 * 12;  // staged quads of a fused pass (ranks up to 12)

// Two blocks of 256 threads per SM (128 registers): the fused pass is limited by
// FP32 issue and latency at rank 10, and the second block hides more of it.
template <class TV, class TA, class TC>
__global__ void __launch_bounds__(256, 2) k_qtt_step2(QttDev q, int k, const TV* in, TV* out, int bound) {
  __shared__ Quad<TA> gq[QTT_GQ];
  qtt_step2_grid<TV, TA, TC>(q, k, in, out, gq, bound);
}

template <class TV, class TA, class TC>
void launch_step(qp_ctx* c, const QttDev& q, int k, const void* in, void* out, int bound, long long N) {
  const TV* i = static_cast<const TV*>(in);
  TV* o = static_cast<TV*>(out);
  if (bound) {
    // one wave of the two resident blocks per SM: each block stages its two cores
    // once and its threads stride over several column items
    long long want = ((N >> 2) + 255) / 256;
    if (want > (long long)c->num_sms * 2) want = (long long)c->num_sms * 2;
    k_qtt_step2<TV, TA, TC><<<(int)(want < 1 ? 1 : want), 256, 0, c->stream>>>(q, k, i, o, bound);
  } else {
    const long long items = N >> 1;
    long long want = (items + 511) / 512;  // two columns per thread
    if (want > (long long)c->num_sms * 16) want = (long long)c->num_sms * 16;
    k_qtt_step<TV, TA, TC><<<(int)(want < 1 ? 1 : want), 256, 0, c->stream>>>(q, k, i, o, items);
  }
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

// y = A x: one launch per pass (two cores per pass where the ranks allow, else
// one), ping-ponging between two work buffers.
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
  const void* in = x;
  int pass = 0;
  // tensor-core steps for the dense cores (FP32 vectors, BF16 or F32 cores);
  // when every core that fits goes there, no two cores are fused into one pass
  const bool tc_ok = vdt == QP_F32 && cdt != QP_F64;
  const bool tc_all = tc_ok && c->qtt_tc_mode == 2 && A->d >= 8;
  bool used_tc = false;
  for (int k = A->d; k >= 1; ++pass) {
    const bool tcs = tc_ok && qtt_tc_eligible(c, q, k, cdt);
    const int bound = (vdt == QP_F64 || tcs || tc_all) ? 0 : qtt_fuse_bound<float>(q, k, QTT_GQ);
    const int next = bound ? k - 2 : k - 1;
    void* out = (next == 0) ? y : ((pass & 1) ? w1 : w0);
    if (tcs) {
      if (!used_tc) QP_CUDA(cudaMemsetAsync(qtt_tc_flag(c), 0, sizeof(int), c->stream));
      used_tc = true;
      launch_qtt_step_tc(c, q, k, static_cast<const float*>(in), static_cast<float*>(out), cdt);
    } else if (vdt == QP_F64) launch_step<double, double, double>(c, q, k, in, out, bound, N);
    else if (cdt == QP_F32) launch_step<float, float, float>(c, q, k, in, out, bound, N);
    else if (cdt == QP_BF16) launch_step<float, float, __nv_bfloat16>(c, q, k, in, out, bound, N);
    else launch_step<float, float, double>(c, q, k, in, out, bound, N);
    QP_CUDA(cudaGetLastError());
    in = out;
    k = next;
  }
  if (used_tc) {
    int h = 0;
    QP_CUDA(cudaMemcpyAsync(&h, qtt_tc_flag(c), sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    QP_CUDA(cudaStreamSynchronize(c->stream));
    QP_REQUIRE(h == 0, QP_TIMEOUT, "qtt_apply: a tensor-core step's wait expired");
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
