// Learned warm start (an extension, not in the paper): a message-passing
// network over the contact graph predicts the impulses that start the PDIP.
// Contacts are the nodes; a message goes from a contact to each of its dynamic
// bodies and back (m_b = sum of h_c over the body's contacts, s_c = m_a + m_b).
//   h0 = relu(W0 x + b0), hl = relu(Wl [h(l-1); s(h(l-1))] + bl) (l = 1..3),
//   o = Wo h3 + bo,  with x the 8 scaled contact features (n, Phi/dt, the
// relative velocity in the contact frame, mu).  Parameters are BF16-rounded
// for the passes (FP32 master kept by the caller), activations and sums FP32.
#include <cuda_bf16.h>

#include "internal.cuh"

namespace qp {
namespace {

constexpr int MF = 8, MW = 64, MO = 3, ML = 3;
constexpr int OFF_W0 = 0, OFF_B0 = MW * MF;
constexpr int LAYER = MW * 2 * MW + MW;
constexpr int OFF_L = OFF_B0 + MW;                // layer l: W at OFF_L + l*LAYER, b after W
constexpr int OFF_WO = OFF_L + ML * LAYER, OFF_BO = OFF_WO + MO * MW;
constexpr int NPAR = OFF_BO + MO;
static_assert(NPAR == QP_MPNN_NPARAM, "parameter layout");

struct Scale {
  float s[MF];
};

__global__ void k_mp_round(const float* __restrict__ p, __nv_bfloat16* __restrict__ q, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) q[i] = __float2bfloat16_rn(p[i]);
}

__device__ __forceinline__ float pb(const __nv_bfloat16* p, int i) { return __bfloat162float(p[i]); }

__global__ void k_mp_features(int Nc, int slots, const double* __restrict__ phi, const double* __restrict__ frame,
                              const double* __restrict__ r, double dt, double mu, Scale sc, float* __restrict__ X) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < Nc; c += gridDim.x * blockDim.x) {
    const double pd = phi[c] / dt;
    const long long row = (long long)slots * c;
    float x[MF];
    x[0] = (float)frame[c];
    x[1] = (float)frame[(size_t)Nc + c];
    x[2] = (float)frame[2 * (size_t)Nc + c];
    x[3] = (float)pd;
    x[4] = (float)(r[row] - pd);
    x[5] = (float)r[row + 1];
    x[6] = (float)r[row + 2];
    x[7] = (float)mu;
    for (int k = 0; k < MF; ++k) X[(size_t)c * MF + k] = x[k] * sc.s[k];
  }
}

// Y[c][j] = act(b[j] + sum_k W[j][k] Xa[c][k] + sum_k W[j][Ka + k] Xb[c][k])
__global__ void k_mp_dense(int Nc, const float* __restrict__ Xa, int Ka, const float* __restrict__ Xb, int Kb,
                           const __nv_bfloat16* __restrict__ Wt, const __nv_bfloat16* __restrict__ bias, int J,
                           int relu, float* __restrict__ Y) {
  const long long n = (long long)Nc * J;
  const int K = Ka + Kb;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i / J), j = (int)(i - (long long)c * J);
    float acc = pb(bias, j);
    const __nv_bfloat16* w = Wt + (size_t)j * K;
    for (int k = 0; k < Ka; ++k) acc = fmaf(pb(w, k), Xa[(size_t)c * Ka + k], acc);
    for (int k = 0; k < Kb; ++k) acc = fmaf(pb(w, Ka + k), Xb[(size_t)c * Kb + k], acc);
    Y[i] = relu ? fmaxf(acc, 0.f) : acc;
  }
}

// Mb[b][f] = sum over the incidences of body b of H[contact][f]
__global__ void k_mp_bodysum(int M, const int* __restrict__ bptr, const int* __restrict__ inc,
                             const float* __restrict__ H, float* __restrict__ Mb) {
  const long long n = (long long)M * MW;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(i / MW), f = (int)(i - (long long)b * MW);
    float s = 0.f;
    for (int k = bptr[b]; k < bptr[b + 1]; ++k) s += H[(size_t)(inc[k] >> 1) * MW + f];
    Mb[i] = s;
  }
}

// S[c][f] (+)= Mb[a][f] (dynamic a) + Mb[b][f]
__global__ void k_mp_gather(int Nc, int M, const int* __restrict__ ca, const int* __restrict__ cb,
                            const float* __restrict__ Mb, float* __restrict__ S, int accumulate) {
  const long long n = (long long)Nc * MW;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i / MW), f = (int)(i - (long long)c * MW);
    const int a = ca[c], b = cb[c];
    float s = (a < M ? Mb[(size_t)a * MW + f] : 0.f) + Mb[(size_t)b * MW + f];
    S[i] = accumulate ? S[i] + s : s;
  }
}

// dO = 2 (O - Y) / (3 Nc); e[i] = (O - Y)^2
__global__ void k_mp_loss(int n, const float* __restrict__ O, const float* __restrict__ Yt, float* __restrict__ dO,
                          double* __restrict__ e) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float d = O[i] - Yt[i];
    dO[i] = 2.f * d / (float)n;
    e[i] = (double)d * (double)d;
  }
}

__global__ void k_mp_sum(int n, const double* __restrict__ e, double* __restrict__ out) {
  __shared__ double sm[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += e[i];
  sm[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) sm[threadIdx.x] += sm[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sm[0];
}

// dZ = dY where the layer's output is positive (ReLU), in place
__global__ void k_mp_relu_bwd(long long n, const float* __restrict__ Y, float* __restrict__ dY) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    if (!(Y[i] > 0.f)) dY[i] = 0.f;
}

// dXa[c][k] = sum_j W[j][k] dZ[c][j]; dXb[c][k] = sum_j W[j][Ka+k] dZ[c][j]
__global__ void k_mp_dense_bwd_x(int Nc, const float* __restrict__ dZ, int J, const __nv_bfloat16* __restrict__ Wt,
                                 int Ka, int Kb, float* __restrict__ dXa, float* __restrict__ dXb) {
  const int K = Ka + Kb;
  const long long n = (long long)Nc * K;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i / K), k = (int)(i - (long long)c * K);
    float s = 0.f;
    for (int j = 0; j < J; ++j) s = fmaf(pb(Wt, j * K + k), dZ[(size_t)c * J + j], s);
    if (k < Ka) dXa[(size_t)c * Ka + k] = s;
    else dXb[(size_t)c * Kb + (k - Ka)] = s;
  }
}

// gW[j][k] = sum_c dZ[c][j] X[c][k] (X = [Xa, Xb]); gb[j] = sum_c dZ[c][j]
__global__ void k_mp_dense_bwd_w(int Nc, const float* __restrict__ dZ, int J, const float* __restrict__ Xa, int Ka,
                                 const float* __restrict__ Xb, int Kb, float* __restrict__ gW, float* __restrict__ gb) {
  const int K = Ka + Kb;
  const int n = J * (K + 1);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int j = i / (K + 1), k = i - j * (K + 1);
    double s = 0.0;  // FP64: one long sum per weight, exact enough for the oracle comparison
    if (k == K) {
      for (int c = 0; c < Nc; ++c) s += dZ[(size_t)c * J + j];
      gb[j] = (float)s;
    } else {
      for (int c = 0; c < Nc; ++c) {
        const float x = k < Ka ? Xa[(size_t)c * Ka + k] : Xb[(size_t)c * Kb + (k - Ka)];
        s += (double)(dZ[(size_t)c * J + j] * x);
      }
      gW[j * K + k] = (float)s;
    }
  }
}

__global__ void k_mp_adam(int n, float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                          const float* __restrict__ g, float lr, float b1, float b2, float eps, float c1, float c2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// gamma = out_scale * o moved into the cone's interior; lambda = -1/f; dummies 0
__global__ void k_mp_warm(int Nc, int slots, long long P, const float* __restrict__ O, double out_scale, double mu,
                          double gn_min, double shrink, double* __restrict__ gamma, double* __restrict__ lambda) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P; i += (long long)gridDim.x * blockDim.x) {
    const long long c = i / slots;
    const int u = (int)(i - c * slots);
    if (c >= Nc || u >= 3) {
      gamma[i] = 0.0;
      continue;
    }
    double gn = fmax(out_scale * (double)O[3 * c], gn_min);
    double t1 = out_scale * (double)O[3 * c + 1], t2 = out_scale * (double)O[3 * c + 2];
    const double nt = hypot(t1, t2), cap = shrink * mu * gn;
    if (nt > cap) {
      t1 *= cap / nt;
      t2 *= cap / nt;
    }
    gamma[i] = u == 0 ? gn : (u == 1 ? t1 : t2);
    if (u == 0) {
      lambda[c] = -1.0 / (0.5 * (t1 * t1 + t2 * t2 - mu * mu * gn * gn));
      lambda[Nc + c] = 1.0 / gn;
    }
  }
}

inline int blocks_for(long long n, int per = 256, int cap = 152 * 32) {
  long long b = (n + per - 1) / per;
  if (b > cap) b = cap;
  return (int)(b < 1 ? 1 : b);
}

struct Net {
  float* X0;
  float* H[ML + 1];
  float* S[ML];
  float* Mb;
  float* O;
  __nv_bfloat16* pw;
};

// workspace: activations of one pass (kept for the backward pass) + scratch
Net workspace(qp_ctx* c) {
  const size_t Nc = (size_t)(c->Nc > 0 ? c->Nc : 1), M = (size_t)(c->M > 0 ? c->M : 1);
  const size_t nf = Nc * MF + (ML + 1) * Nc * MW + ML * Nc * MW + M * MW + Nc * MO + 64;
  float* w = static_cast<float*>(c->mp_act.ensure(nf * sizeof(float)));
  Net n;
  n.X0 = w;
  w += Nc * MF;
  for (int l = 0; l <= ML; ++l, w += Nc * MW) n.H[l] = w;
  for (int l = 0; l < ML; ++l, w += Nc * MW) n.S[l] = w;
  n.Mb = w;
  w += M * MW;
  n.O = w;
  n.pw = static_cast<__nv_bfloat16*>(c->mp_w.ensure((size_t)NPAR * sizeof(__nv_bfloat16)));
  return n;
}

void forward(qp_ctx* c, const float* params, const float* scale_host, float* out, Net& n) {
  cudaStream_t st = c->stream;
  const int Nc = c->Nc, M = c->M;
  k_mp_round<<<blocks_for(NPAR), 256, 0, st>>>(params, n.pw, NPAR);
  Scale sc;
  for (int k = 0; k < MF; ++k) sc.s[k] = scale_host[k];
  if (Nc > 0) {
    k_mp_features<<<blocks_for(Nc), 256, 0, st>>>(Nc, c->slots, c->phi.as<double>(), c->frame.as<double>(),
                                                 c->r.as<double>(), c->dt, c->mu, sc, n.X0);
    k_mp_dense<<<blocks_for((long long)Nc * MW), 256, 0, st>>>(Nc, n.X0, MF, nullptr, 0, n.pw + OFF_W0, n.pw + OFF_B0,
                                                              MW, 1, n.H[0]);
    for (int l = 0; l < ML; ++l) {
      k_mp_bodysum<<<blocks_for((long long)M * MW), 256, 0, st>>>(M, c->bptr.as<int>(), c->inc.as<int>(), n.H[l], n.Mb);
      k_mp_gather<<<blocks_for((long long)Nc * MW), 256, 0, st>>>(Nc, M, c->ca.as<int>(), c->cb.as<int>(), n.Mb,
                                                                 n.S[l], 0);
      const __nv_bfloat16* W = n.pw + OFF_L + l * LAYER;
      k_mp_dense<<<blocks_for((long long)Nc * MW), 256, 0, st>>>(Nc, n.H[l], MW, n.S[l], MW, W, W + MW * 2 * MW, MW, 1,
                                                                n.H[l + 1]);
    }
    k_mp_dense<<<blocks_for((long long)Nc * MO), 256, 0, st>>>(Nc, n.H[ML], MW, nullptr, 0, n.pw + OFF_WO,
                                                              n.pw + OFF_BO, MO, 0, out);
  }
  QP_CUDA(cudaGetLastError());
}

}  // namespace
}  // namespace qp

using namespace qp;

#define MP_BEGIN(c)               \
  if (!(c)) return QP_INVALID_ARG; \
  try {                           \
    QP_CUDA(cudaSetDevice((c)->device));
#define MP_END(c)                 \
  }                               \
  catch (const Error& e) {        \
    set_error((c), e);            \
    return e.code;                \
  }                               \
  return QP_OK;

extern "C" {

int mpnn_forward(qp_ctx_t c, const float* params, const float* feat_scale, float* out) {
  MP_BEGIN(c)
  QP_REQUIRE(c->have_contacts, QP_NOT_READY, "mpnn_forward: call ccp_assemble first");
  QP_REQUIRE(params && feat_scale && (out || c->Nc == 0), QP_INVALID_ARG, "mpnn_forward: null argument");
  Net n = workspace(c);
  forward(c, params, feat_scale, out, n);
  MP_END(c)
}

int mpnn_grad(qp_ctx_t c, const float* params, const float* feat_scale, const float* target, float* grad,
              double* loss) {
  MP_BEGIN(c)
  QP_REQUIRE(c->have_contacts, QP_NOT_READY, "mpnn_grad: call ccp_assemble first");
  QP_REQUIRE(params && feat_scale && grad && target, QP_INVALID_ARG, "mpnn_grad: null argument");
  QP_REQUIRE(c->Nc > 0, QP_INVALID_ARG, "mpnn_grad: no contacts to fit");
  QP_REQUIRE(grad != params, QP_INVALID_ARG, "mpnn_grad: grad aliases params");
  Net n = workspace(c);
  const int Nc = c->Nc, M = c->M;
  cudaStream_t st = c->stream;
  forward(c, params, feat_scale, n.O, n);
  // scratch: per-entry errors (double) [3Nc], dO [3Nc], three [Nc][64] buffers
  const size_t nb = (size_t)3 * Nc * sizeof(double) + (size_t)3 * Nc * sizeof(float) + 3 * (size_t)Nc * MW * 4 + 256;
  char* s = static_cast<char*>(c->mp_grad.ensure(nb));
  double* err = reinterpret_cast<double*>(s);
  float* dO = reinterpret_cast<float*>(err + 3 * (size_t)Nc);
  float* A = dO + 3 * (size_t)Nc + 4;
  float* B = A + (size_t)Nc * MW;
  float* Cs = B + (size_t)Nc * MW;
  float* dM = n.Mb;  // the forward pass is done with it
  double* lsum = static_cast<double*>(c->mp_sum.ensure(sizeof(double)));
  const long long nh = (long long)Nc * MW;
  k_mp_loss<<<blocks_for(3LL * Nc), 256, 0, st>>>(3 * Nc, n.O, target, dO, err);
  k_mp_sum<<<1, 256, 0, st>>>(3 * Nc, err, lsum);
  // head: o = Wo h3 + bo
  k_mp_dense_bwd_w<<<blocks_for(MO * (MW + 1)), 256, 0, st>>>(Nc, dO, MO, n.H[ML], MW, nullptr, 0, grad + OFF_WO,
                                                             grad + OFF_BO);
  k_mp_dense_bwd_x<<<blocks_for(nh), 256, 0, st>>>(Nc, dO, MO, n.pw + OFF_WO, MW, 0, A, nullptr);
  for (int l = ML - 1; l >= 0; --l) {
    // layer l: H[l+1] = relu(W [H[l]; S[l]] + b); A holds d/dH[l+1]
    const __nv_bfloat16* W = n.pw + OFF_L + l * LAYER;
    float* gW = grad + OFF_L + l * LAYER;
    k_mp_relu_bwd<<<blocks_for(nh), 256, 0, st>>>(nh, n.H[l + 1], A);
    k_mp_dense_bwd_w<<<blocks_for(MW * (2 * MW + 1)), 256, 0, st>>>(Nc, A, MW, n.H[l], MW, n.S[l], MW, gW,
                                                                    gW + MW * 2 * MW);
    k_mp_dense_bwd_x<<<blocks_for((long long)Nc * 2 * MW), 256, 0, st>>>(Nc, A, MW, W, MW, MW, B, Cs);
    // S[l] = gather(bodysum(H[l])): its adjoint is the same pair of sums
    k_mp_bodysum<<<blocks_for((long long)M * MW), 256, 0, st>>>(M, c->bptr.as<int>(), c->inc.as<int>(), Cs, dM);
    k_mp_gather<<<blocks_for(nh), 256, 0, st>>>(Nc, M, c->ca.as<int>(), c->cb.as<int>(), dM, B, 1);
    float* t = A;
    A = B;
    B = t;
  }
  // input layer: H[0] = relu(W0 X0 + b0)
  k_mp_relu_bwd<<<blocks_for(nh), 256, 0, st>>>(nh, n.H[0], A);
  k_mp_dense_bwd_w<<<blocks_for(MW * (MF + 1)), 256, 0, st>>>(Nc, A, MW, n.X0, MF, nullptr, 0, grad + OFF_W0,
                                                             grad + OFF_B0);
  QP_CUDA(cudaGetLastError());
  if (loss) {
    double h = 0.0;
    QP_CUDA(cudaMemcpyAsync(&h, lsum, sizeof(double), cudaMemcpyDeviceToHost, st));
    QP_CUDA(cudaStreamSynchronize(st));
    *loss = h / (3.0 * Nc);
  }
  MP_END(c)
}

int mpnn_adam(qp_ctx_t c, float* params, float* m, float* v, const float* grad, int step, double lr, double beta1,
              double beta2, double eps) {
  MP_BEGIN(c)
  QP_REQUIRE(params && m && v && grad && step >= 1 && lr > 0 && beta1 >= 0 && beta1 < 1 && beta2 >= 0 && beta2 < 1 &&
                 eps > 0,
             QP_INVALID_ARG, "mpnn_adam: bad argument");
  const float c1 = (float)(1.0 - pow(beta1, step)), c2 = (float)(1.0 - pow(beta2, step));
  k_mp_adam<<<blocks_for(NPAR), 256, 0, c->stream>>>(NPAR, params, m, v, grad, (float)lr, (float)beta1, (float)beta2,
                                                     (float)eps, c1, c2);
  QP_CUDA(cudaGetLastError());
  MP_END(c)
}

int mpnn_warm_start(qp_ctx_t c, qp_state* st, const float* out, double out_scale, double gn_min, double shrink) {
  MP_BEGIN(c)
  QP_REQUIRE(c->have_contacts, QP_NOT_READY, "mpnn_warm_start: call ccp_assemble first");
  QP_REQUIRE(st && st->gamma && st->lambda && (out || c->Nc == 0), QP_INVALID_ARG, "mpnn_warm_start: null argument");
  QP_REQUIRE(out_scale > 0 && gn_min > 0 && shrink > 0 && shrink <= 1, QP_INVALID_ARG,
             "mpnn_warm_start: need out_scale > 0, gn_min > 0, 0 < shrink <= 1");
  k_mp_warm<<<blocks_for(c->P), 256, 0, c->stream>>>(c->Nc, c->slots, c->P, out, out_scale, c->mu, gn_min, shrink,
                                                     st->gamma, st->lambda);
  QP_CUDA(cudaGetLastError());
  st->t = 1.0;
  MP_END(c)
}

}  // extern "C"
