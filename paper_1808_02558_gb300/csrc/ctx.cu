// Context, buffers and status handling of the C ABI.
#include <cstring>

#include "internal.cuh"

namespace qp {

void* Buf::ensure(size_t bytes) {
  if (bytes <= cap && p) return p;
  if (p) cudaFree(p);
  p = nullptr;
  cap = 0;
  size_t want = bytes < 256 ? 256 : bytes;
  cudaError_t e = cudaMalloc(&p, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
    throw Error{QP_OOM, std::string("cudaMalloc(") + std::to_string(want) + "): " + cudaGetErrorString(e)};
  }
  cap = want;
  return p;
}

void Buf::release() {
  if (p) cudaFree(p);
  p = nullptr;
  cap = 0;
}

void set_error(qp_ctx* c, const Error& e) {
  if (c) c->last_error = e.msg;
}

void sync(qp_ctx* c) { QP_CUDA(cudaStreamSynchronize(c->stream)); }

SysView<double> view64(qp_ctx* c, bool with_H) {
  SysView<double> v;
  v.M = c->M;
  v.Nc = c->Nc;
  v.slots = c->slots;
  v.P = c->P;
  v.ca = c->ca.as<int>();
  v.cb = c->cb.as<int>();
  v.rec = c->rec64.as<double>();
  v.inv_m = c->inv_m.as<double>();
  v.inv_I = c->inv_I.as<double>();
  v.bptr = c->bptr.as<int>();
  v.inc = c->inc.as<int>();
  v.H = with_H ? c->H.as<double>() : nullptr;
  v.w = c->wbody.as<double>();
  return v;
}

SysView<float> view32(qp_ctx* c, bool with_H) {
  SysView<float> v;
  v.M = c->M;
  v.Nc = c->Nc;
  v.slots = c->slots;
  v.P = c->P;
  v.ca = c->ca.as<int>();
  v.cb = c->cb.as<int>();
  v.rec = c->rec32.as<float>();
  v.inv_m = c->inv_m32.as<float>();
  v.inv_I = c->inv_I32.as<float>();
  v.bptr = c->bptr.as<int>();
  v.inc = c->inc.as<int>();
  v.H = with_H ? c->H32.as<float>() : nullptr;
  v.w = c->wbody32.as<float>();
  return v;
}

}  // namespace qp

using namespace qp;

extern "C" {

const char* qp_status_string(int s) {
  switch (s) {
    case QP_OK: return "QP_OK";
    case QP_INVALID_ARG: return "QP_INVALID_ARG";
    case QP_OOM: return "QP_OOM";
    case QP_CUDA_ERROR: return "QP_CUDA_ERROR";
    case QP_NOT_CONVERGED: return "QP_NOT_CONVERGED";
    case QP_BREAKDOWN: return "QP_BREAKDOWN";
    case QP_LINESEARCH_FAIL: return "QP_LINESEARCH_FAIL";
    case QP_TIMEOUT: return "QP_TIMEOUT";
    case QP_NOT_READY: return "QP_NOT_READY";
    default: return "QP_UNKNOWN";
  }
}

int qp_create(qp_ctx_t* out, int device, void* stream) {
  if (!out) return QP_INVALID_ARG;
  *out = nullptr;
  qp_ctx* c = new qp_ctx();
  try {
    QP_CUDA(cudaSetDevice(device));
    c->device = device;
    c->stream = static_cast<cudaStream_t>(stream);
    QP_CUDA(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device));
    c->ctl.ensure(sizeof(DevCtl));
    QP_CUDA(cudaMemsetAsync(c->ctl.p, 0, sizeof(DevCtl), c->stream));
    QP_CUDA(cudaMallocHost(&c->ctl_host, sizeof(DevCtl)));
    QP_CUDA(cudaEventCreate(&c->ev0));
    QP_CUDA(cudaEventCreate(&c->ev1));
    QP_CUDA(cudaStreamSynchronize(c->stream));
  } catch (const Error& e) {
    delete c;
    return e.code;
  }
  *out = c;
  return QP_OK;
}

int qp_destroy(qp_ctx_t c) {
  if (!c) return QP_INVALID_ARG;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  Buf* bufs[] = {&c->ca, &c->cb, &c->phi, &c->frame, &c->point, &c->arm_a, &c->arm_b, &c->key, &c->r,
                 &c->rec64, &c->rec32, &c->inv_m, &c->inv_I, &c->inv_m32, &c->inv_I32,
                 &c->bptr, &c->inc, &c->wbody, &c->wbody32, &c->H, &c->H32, &c->dinv, &c->dinv32,
                 &c->partial, &c->ctl, &c->part_nb, &c->part_bodies, &c->part_cl, &c->fused_pool, &c->batch64, &c->batch32,
                 &c->batch_table, &c->mp_act, &c->mp_w, &c->mp_grad, &c->mp_sum};
  for (Buf* b : bufs) b->release();
  for (auto& b : c->v64) b.release();
  for (auto& b : c->v32) b.release();
  for (auto& b : c->scratch) b.release();
  for (auto& b : c->la) b.release();
  for (auto& b : c->dm) b.release();
  if (c->last_inv) qtt_free(c, c->last_inv);
  if (c->ctl_host) cudaFreeHost(c->ctl_host);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  delete c;
  return QP_OK;
}

int qp_last_error(qp_ctx_t c, char* buf, int len) {
  if (!c || !buf || len <= 0) return QP_INVALID_ARG;
  std::strncpy(buf, c->last_error.c_str(), (size_t)len - 1);
  buf[len - 1] = 0;
  return QP_OK;
}

}  // extern "C"
