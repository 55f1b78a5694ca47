// Internal declarations shared by the translation units of the library.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/qttpdip.h"

namespace qp {

// ---------------------------------------------------------------- errors
struct Error {
  int code;
  std::string msg;
};

#define QP_CUDA(call)                                                              \
  do {                                                                             \
    cudaError_t e__ = (call);                                                      \
    if (e__ != cudaSuccess)                                                        \
      throw ::qp::Error{QP_CUDA_ERROR, std::string(#call) + ": " + cudaGetErrorString(e__)}; \
  } while (0)

#define QP_REQUIRE(cond, code, what)                                               \
  do {                                                                             \
    if (!(cond)) throw ::qp::Error{(code), std::string(what)};                     \
  } while (0)

// ---------------------------------------------------------------- buffers
// Grow-only device buffer; contents are not preserved when it grows.
struct Buf {
  void* p = nullptr;
  size_t cap = 0;
  void* ensure(size_t bytes);
  void release();
  template <class T> T* as() const { return static_cast<T*>(p); }
};

// Device-side control block of the persistent kernels.
struct DevCtl {
  unsigned int bar_count;  // grid barrier: arrivals so far (monotonic within a launch)
  unsigned int pad0_[31];  // keeps the polled counter on its own cache line
  int err;                 // 0 or a QP_* code set by a device-side failure
  int iters;               // Krylov iterations
  int outer;               // refinement steps
  int halvings;
  double scal[16];         // scalars handed between kernels (eta, t, s, norms, ...)
};

enum Scal { S_ETA = 0, S_T, S_RDUAL, S_RT, S_S, S_RELRES, S_BNORM, S_SMAX, S_RCENT };

struct QTTCore;

}  // namespace qp

struct qp_qtt {
  qp_ctx* ctx = nullptr;
  int d = 0;
  std::vector<int> ranks;          // d+1
  std::vector<long long> offset;   // d+1, value offsets of each core
  long long nvals = 0;
  double* cores = nullptr;         // FP64 master copy (device)
  float* cores32 = nullptr;        // FP32 apply copy (device, lazily made)
  __nv_bfloat16* cores16 = nullptr;// BF16 apply copy (device, lazily made)
  int scaled = 0;                  // 1: approximates D^-1/2 S D^-1/2 (or its inverse), D = diag(S)
};

struct qp_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int num_sms = 0;
  std::string last_error;

  // scene / contact sizes
  int M = 0, Nc = 0, L = 0, slots = 3;
  long long P = 0;
  double mu = 0.5, dt = 1e-3;
  bool have_contacts = false;

  // contact arrays (FP64 master + FP32 copies for the mixed-precision path)
  qp::Buf ca, cb, phi, frame, point, arm_a, arm_b, key, r, cplane;
  qp::Buf rec64, rec32;  // [Nc][16] contact records: n t1 t2 ra rb pad
  // body arrays
  qp::Buf inv_m, inv_I, inv_m32, inv_I32, bptr, inc;
  // operator work
  qp::Buf wbody, wbody32, H, H32, dinv, dinv32;
  // Krylov / PDIP vectors (P doubles / floats each)
  qp::Buf v64[8], v32[8];
  qp::Buf partial;     // per-block partial sums
  qp::Buf ctl;         // DevCtl
  qp::Buf scratch[8];  // assembly / QTT scratch
  qp::Buf la[6];       // one-block linear algebra workspaces (A, V, Vs, w, tmp, misc)
  qp::Buf dm[16];      // QTT inverse workspaces
  qp::DevCtl* ctl_host = nullptr;  // pinned mirror

  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  qp_qtt* last_inv = nullptr;  // last QTT inverse built by pdip_step (warm start of the next)
  // contact partition of the fused Krylov kernel (one contiguous chunk per block)
  int part_G = 0, part_chunk = 0, part_maxb = 0, part_nbmax = 0;
  qp::Buf part_nb, part_bodies, part_cl;
  // contact partition of the standalone fused apply (newton_apply)
  int apart_G = 0, apart_chunk = 0, apart_maxb = 0, apart_nbmax = 0;
  qp::Buf apart_nb, apart_bodies, apart_cl;
  qp::Buf fused_pool;
  qp::Buf mp_act, mp_w, mp_grad, mp_sum;  // learned warm start: activations, BF16 weights, scratch
  qp::Buf batch64, batch32, batch_table;  // batched solves: per-scene vectors; table (first context)
  qp::Buf batch_qw, tune_buf;  // batched QTT work buffers; tile-shape probe data
  qp::Buf tc_err;  // error flag of the tensor-core QTT step
  int qtt_tc_mode = 1;  // tensor-core QTT steps: 0 never, 1 dense cores, 2 every core that fits
};

namespace qp {

inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

// Device views of the Schur operator for precision T.
template <class T>
struct SysView {
  int M, Nc, slots;
  long long P;
  const int* ca;
  const int* cb;
  const T* rec;    // [Nc][16] contact records: n(3) t1(3) t2(3) ra(3) rb(3) 0
  const T* inv_m;  // [M]
  const T* inv_I;  // [M]
  const int* bptr; // [M+1]
  const int* inc;  // [2Nc] (contact << 1) | side, side 1 = body b
  const T* H;      // [6][Nc] packed 3x3 blocks (00 01 02 11 12 22) or null
  T* w;            // [M][8] body scratch: M^-1 (force, torque), 2 pad
};

SysView<double> view64(qp_ctx* c, bool with_H);
SysView<float> view32(qp_ctx* c, bool with_H);

void set_error(qp_ctx* c, const Error& e);
void sync(qp_ctx* c);

// kernels launched from several translation units
void launch_schur_blocks(qp_ctx* c, const double* gamma, const double* lambda);
void launch_apply64(qp_ctx* c, const double* x, double* y, bool with_H);
void launch_apply32(qp_ctx* c, const float* x, float* y, bool with_H);
void launch_qtt_apply(qp_ctx* c, qp_qtt* A, const void* x, void* y, qp_dtype core_dt, qp_dtype vec_dt);
// tensor-core QTT step (qtt_tc.cu): FP32 vectors, cores with r_{k-1}, r_k <= 64;
// in the automatic mode only BF16 cores with r_{k-1} r_k >= QTT_TC_MIN_RR
struct QttDev;
constexpr int QTT_TC_MIN_RR = 512;
bool qtt_tc_eligible(const qp_ctx* c, const QttDev& q, int k, qp_dtype core_dt);
void launch_qtt_step_tc(qp_ctx* c, const QttDev& q, int k, const float* in, float* out, qp_dtype core_dt);
int* qtt_tc_flag(qp_ctx* c);
void qtt_prepare_copies(qp_ctx* c, qp_qtt* A, qp_dtype core_dt);
qp_qtt* qtt_alloc(qp_ctx* c, int d, const std::vector<int>& ranks);
size_t qtt_work_bytes(qp_qtt* A, qp_dtype core_dt);
qp_qtt* compress_impl(qp_ctx* c, bool with_H, double eps, int rmax, const double* rowscale);
void launch_rowscale(qp_ctx* c, double* rowscale);

}  // namespace qp
