// Learned warm start (an extension, not in the paper): a message-passing
// network over the contact graph predicts the impulses that start the PDIP.
// Contacts are the nodes; a message goes from a contact to each of its dynamic
// bodies and back (m_b = sum of h_c over the body's contacts, s_c = m_a + m_b).
//   h0 = relu(W0 x + b0), hl = relu(Wl [h(l-1); s(h(l-1))] + bl) (l = 1..3),
//   o = Wo h3 + bo,  with x the 8 scaled contact features (n, Phi/dt, the
// relative velocity in the contact frame, mu).  Parameters are BF16-rounded
// for the passes (FP32 master kept by the caller), activations and sums FP32.
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "internal.cuh"
#include "tc.cuh"

namespace qp {

// The driver's tensor-map encoder, looked up once (shared with qtt_tc.cu).
PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  QP_REQUIRE(fn != nullptr, QP_CUDA_ERROR, "cuTensorMapEncodeTiled is not available");
  return fn;
}

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

// ---------------------------------------------------------------- tensor-core rows GEMM
// OUT[r][n] = sum_k A[r][k] B[n][k] on the tensor cores (tcgen05, kind::tf32),
// 128 rows per tile, persistent blocks of 128 threads.  A is FP32, read by TMA
// from up to two row-major sources of 64 columns (kb0 blocks of 32 columns from
// the first, the rest from the second: the concatenation [h; s] of a layer);
// B comes from the BF16 weights, staged once per block as FP32 (exact in TF32).
// Products are FP32-accurate: A = A_hi + A_lo, A_hi = A with its 13 low mantissa
// bits cleared (exact in TF32), A_lo = A - A_hi (exact in FP32, within 2^-11 of
// its own size after the MMA's TF32 conversion), two MMAs per K step, so the
// error is about 2^-21 |A| |B| per term.  The accumulator (128 lanes x N FP32
// columns) lives in tensor memory; each warp reads its 32 rows back.
// EPI 0: Y0[r][n] = relu(acc + bias[n]) (N = 64).  EPI 1: Y0[r][n] = acc for
// n < 64, Y1[r][n - 64] = acc for n >= 64 (N = 128).
constexpr long long TC_BUDGET = 2000000000LL;  // clock ticks (~1 s) per wait

template <int N, int KB, int EPI>
__global__ void __launch_bounds__(128, 1)
    k_tc_rows(const __grid_constant__ CUtensorMap mA0, const __grid_constant__ CUtensorMap mA1, int kb0, int rows,
              const __nv_bfloat16* __restrict__ W, int ldw, int wtrans, const __nv_bfloat16* __restrict__ bias,
              float* __restrict__ Y0, float* __restrict__ Y1, int* __restrict__ err) {
  using namespace tc;
  constexpr int A_BLK = 128 * 128;  // bytes of a 128-row x 32-column block
  constexpr int B_BLK = N * 128;
  constexpr int A_BYTES = KB * A_BLK, B_BYTES = KB * B_BLK;
  // shared memory: B, two A stages (the next tile's copy overlaps this tile's work), A_lo
  extern __shared__ __align__(1024) unsigned char tc_raw[];
  unsigned char* base = tc_raw + ((1024u - (smem_addr(tc_raw) & 1023u)) & 1023u);
  unsigned char* sB = base;
  unsigned char* const sA0 = base + B_BYTES;  // stage s at sA0 + s A_BYTES
  unsigned char* sL = base + B_BYTES + 2 * A_BYTES;
  __shared__ uint64_t bar_tma[2], bar_mma;
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ntiles = (rows + 127) / 128;
  auto issue = [&](int t, int st) {  // thread 0: the A tile of row block t into stage st
    mbar_arrive_expect_tx(&bar_tma[st], A_BYTES);
    for (int j = 0; j < KB; ++j) {
      if (j < kb0) tma_load_2d(sA0 + st * A_BYTES + j * A_BLK, &mA0, &bar_tma[st], 32 * j, t * 128);
      else tma_load_2d(sA0 + st * A_BYTES + j * A_BLK, &mA1, &bar_tma[st], 32 * (j - kb0), t * 128);
    }
  };
  if (tid == 0) {
    mbar_init(&bar_tma[0], 1);
    mbar_init(&bar_tma[1], 1);
    mbar_init(&bar_mma, 1);
    fence_mbar_init();
  }
  if (warp == 0) {
    tmem_alloc(&tmem_base, N);
    tmem_relinquish();
  }
  // B(n, k) = W[n ldw + k] (or W[k ldw + n]) into the swizzled K-major layout
  for (int i = tid; i < N * KB * 32; i += blockDim.x) {
    const int n = i / (KB * 32), k = i - n * (KB * 32);
    const float w = __bfloat162float(wtrans ? W[(size_t)k * ldw + n] : W[(size_t)n * ldw + k]);
    const int kk = k & 31;
    *reinterpret_cast<float*>(sB + (k >> 5) * B_BLK + n * 128 + (((kk >> 2) ^ (n & 7)) << 4) + ((kk & 3) << 2)) = w;
  }
  fence_async_shared();
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if (tid == 0 && (int)blockIdx.x < ntiles) issue(blockIdx.x, 0);
  const uint32_t tmem = tmem_base;
  constexpr uint32_t idesc = idesc_tf32(128, N);
  uint32_t ph_tma = 0u, ph_mma = 0u;  // bit s: parity of stage s's next phase
  int fail = 0;      // 1: a wait expired
  int inflight = 0;  // stages with a copy issued and not yet waited for (bit mask)
  if ((int)blockIdx.x < ntiles) inflight = 1;
  int st = 0;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x, st ^= 1) {
    const int r0 = t * 128;
    if (!mbar_wait(&bar_tma[st], (ph_tma >> st) & 1u, TC_BUDGET)) fail = 1;
    if (__syncthreads_or(fail)) {
      fail = 1;
      break;
    }
    ph_tma ^= 1u << st;
    inflight &= ~(1 << st);
    // the other stage is free (its tile's MMAs completed): start the next copy now
    const int tn = t + gridDim.x;
    if (tn < ntiles) {
      if (tid == 0) issue(tn, st ^ 1);
      inflight |= 1 << (st ^ 1);
    }
    // A_hi in place, A_lo beside it (same swizzled positions)
    float4* a4 = reinterpret_cast<float4*>(sA0 + st * A_BYTES);
    float4* l4 = reinterpret_cast<float4*>(sL);
    for (int i = tid; i < A_BYTES / 16; i += blockDim.x) {
      const float4 a = a4[i];
      float4 h;
      h.x = __uint_as_float(__float_as_uint(a.x) & 0xFFFFE000u);
      h.y = __uint_as_float(__float_as_uint(a.y) & 0xFFFFE000u);
      h.z = __uint_as_float(__float_as_uint(a.z) & 0xFFFFE000u);
      h.w = __uint_as_float(__float_as_uint(a.w) & 0xFFFFE000u);
      a4[i] = h;
      l4[i] = make_float4(a.x - h.x, a.y - h.y, a.z - h.z, a.w - h.w);
    }
    fence_async_shared();
    __syncthreads();
    if (tid == 0) {
      fence_after_sync();
      const uint32_t ah = smem_addr(sA0 + st * A_BYTES), al = smem_addr(sL), bb = smem_addr(sB);
      for (int kk = 0; kk < 4 * KB; ++kk) {
        const uint32_t ao = (kk >> 2) * A_BLK + (kk & 3) * 32, bo = (kk >> 2) * B_BLK + (kk & 3) * 32;
        const uint64_t bd = desc_k_sw128(bb + bo);
        mma_tf32(tmem, desc_k_sw128(ah + ao), bd, idesc, kk > 0 ? 1u : 0u);
        mma_tf32(tmem, desc_k_sw128(al + ao), bd, idesc, 1u);
      }
      mma_commit(&bar_mma);
    }
    if (!mbar_wait(&bar_mma, ph_mma, TC_BUDGET)) fail = 1;
    if (__syncthreads_or(fail)) {
      fail = 1;
      break;
    }
    ph_mma ^= 1u;
    fence_after_sync();
    const int r = r0 + warp * 32 + lane;
    const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll
    for (int c0 = 0; c0 < N; c0 += 32) {
      float v[32];
      tmem_ld32(tl + (uint32_t)c0, v);
      if (r < rows) {
        if constexpr (EPI == 0) {
          float4* o = reinterpret_cast<float4*>(Y0 + (size_t)r * 64 + c0);
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            float4 w;
            w.x = fmaxf(v[4 * q] + __bfloat162float(bias[c0 + 4 * q]), 0.f);
            w.y = fmaxf(v[4 * q + 1] + __bfloat162float(bias[c0 + 4 * q + 1]), 0.f);
            w.z = fmaxf(v[4 * q + 2] + __bfloat162float(bias[c0 + 4 * q + 2]), 0.f);
            w.w = fmaxf(v[4 * q + 3] + __bfloat162float(bias[c0 + 4 * q + 3]), 0.f);
            o[q] = w;
          }
        } else {
          float* dst = c0 < 64 ? Y0 + (size_t)r * 64 + c0 : Y1 + (size_t)r * 64 + (c0 - 64);
          float4* o = reinterpret_cast<float4*>(dst);
#pragma unroll
          for (int q = 0; q < 8; ++q) o[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        }
      }
    }
    fence_before_sync();
    __syncthreads();
  }
  if (fail) {
    // let copies and MMAs of the failed step finish (bounded) before the
    // block's shared and tensor memory go away
    for (int k = 0; k < 2; ++k)
      if (inflight & (1 << k)) mbar_wait(&bar_tma[k], (ph_tma >> k) & 1u, TC_BUDGET);
    mbar_wait(&bar_mma, ph_mma, TC_BUDGET);
    if (tid == 0) atomicExch(err, 1);
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if (warp == 0) tmem_dealloc(tmem, N);
}

// Weight gradient in two deterministic passes: block g sums its chunk of rows,
// part[g][j (K + 1) + k] = sum_c dZ[c][j] X[c][k] (k < K) and sum_c dZ[c][j]
// (k = K), staging 32 rows of dZ and X = [Xa, Xb] in shared memory at a time;
// then the partials are added in block order in FP64.
template <int J, int K, int PER>
__global__ void __launch_bounds__(256) k_wgrad_part(int Nc, int chunk, const float* __restrict__ dZ,
                                                    const float* __restrict__ Xa, int Ka, const float* __restrict__ Xb,
                                                    float* __restrict__ part) {
  static_assert(PER * 256 >= J * (K + 1), "outputs per thread");
  __shared__ float sz[32][J];
  __shared__ float sx[32][K + 1];
  const int c0 = blockIdx.x * chunk, c1 = min(Nc, c0 + chunk);
  float acc[PER];
#pragma unroll
  for (int i = 0; i < PER; ++i) acc[i] = 0.f;
  for (int r0 = c0; r0 < c1; r0 += 32) {
    const int nr = min(32, c1 - r0);
    for (int i = threadIdx.x; i < 32 * J; i += blockDim.x) {
      const int r = i / J, j = i - r * J;
      sz[r][j] = r < nr ? dZ[(size_t)(r0 + r) * J + j] : 0.f;
    }
    for (int i = threadIdx.x; i < 32 * K; i += blockDim.x) {
      const int r = i / K, k = i - r * K;
      float x = 0.f;
      if (r < nr) x = k < Ka ? Xa[(size_t)(r0 + r) * Ka + k] : Xb[(size_t)(r0 + r) * (K - Ka) + (k - Ka)];
      sx[r][k] = x;
    }
    for (int r = threadIdx.x; r < 32; r += blockDim.x) sx[r][K] = 1.f;
    __syncthreads();
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int o = threadIdx.x + i * 256;
      if (o < J * (K + 1)) {
        const int j = o / (K + 1), k = o - j * (K + 1);
        float s = acc[i];
#pragma unroll 8
        for (int r = 0; r < 32; ++r) s = fmaf(sz[r][j], sx[r][k], s);
        acc[i] = s;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int o = threadIdx.x + i * 256;
    if (o < J * (K + 1)) part[(size_t)blockIdx.x * J * (K + 1) + o] = acc[i];
  }
}

// gW[j K + k] = sum_g part[g][j (K+1) + k], gb[j] = sum_g part[g][j (K+1) + K]
__global__ void k_wgrad_sum(int nparts, int J, int K, const float* __restrict__ part, float* __restrict__ gW,
                            float* __restrict__ gb) {
  const int n = J * (K + 1);
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < n; o += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int g = 0; g < nparts; ++g) s += (double)part[(size_t)g * n + o];
    const int j = o / (K + 1), k = o - j * (K + 1);
    if (k == K) gb[j] = (float)s;
    else gW[j * K + k] = (float)s;
  }
}

inline int blocks_for(long long n, int per = 256, int cap = 152 * 32) {
  long long b = (n + per - 1) / per;
  if (b > cap) b = cap;
  return (int)(b < 1 ? 1 : b);
}

// ---- host side of the tensor-core GEMM

// Row-major FP32 matrix [rows][64], boxes of 128 rows x 32 columns (128 bytes
// wide, the 128-byte swizzle); rows past the end read as zeros.
CUtensorMap rows64_map(const float* base, int rows) {
  QP_REQUIRE((reinterpret_cast<uintptr_t>(base) & 15u) == 0, QP_CUDA_ERROR, "tensor map base not 16-byte aligned");
  CUtensorMap m;
  const cuuint64_t gdim[2] = {64, (cuuint64_t)rows};
  const cuuint64_t gstride[1] = {64 * sizeof(float)};
  const cuuint32_t box[2] = {32, 128};
  const cuuint32_t es[2] = {1, 1};
  const CUresult r = tmap_encoder()(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), gdim, gstride,
                                    box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  QP_REQUIRE(r == CUDA_SUCCESS, QP_CUDA_ERROR, "cuTensorMapEncodeTiled failed");
  return m;
}

int* tc_flag(qp_ctx* c) {
  char* p = static_cast<char*>(c->mp_sum.ensure(64));
  return reinterpret_cast<int*>(p + 32);
}

template <int N, int KB, int EPI>
void launch_tc_rows(qp_ctx* c, const float* A0, const float* A1, int kb0, int rows, const __nv_bfloat16* W, int ldw,
                    int wtrans, const __nv_bfloat16* bias, float* Y0, float* Y1) {
  if (rows <= 0) return;
  const CUtensorMap m0 = rows64_map(A0, rows);
  const CUtensorMap m1 = rows64_map(A1 ? A1 : A0, rows);
  auto k = k_tc_rows<N, KB, EPI>;
  const int smem = KB * N * 128 + 3 * KB * 128 * 128 + 1024;  // B, two A stages, A_lo, alignment
  QP_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  const int grid = std::min((rows + 127) / 128, c->num_sms);
  k<<<grid, 128, smem, c->stream>>>(m0, m1, kb0, rows, W, ldw, wtrans, bias, Y0, Y1, tc_flag(c));
  QP_CUDA(cudaGetLastError());
}

// Weight and bias gradient of a dense layer (dZ [Nc][J], X = [Xa (Ka) | Xb (K - Ka)]).
template <int J, int K>
void launch_wgrad(qp_ctx* c, const float* dZ, const float* Xa, int Ka, const float* Xb, float* part, float* gW,
                  float* gb) {
  constexpr int PER = (J * (K + 1) + 255) / 256;
  const int Nc = c->Nc, chunk = 256;
  const int nparts = (Nc + chunk - 1) / chunk;
  k_wgrad_part<J, K, PER><<<nparts, 256, 0, c->stream>>>(Nc, chunk, dZ, Xa, Ka, Xb, part);
  k_wgrad_sum<<<(J * (K + 1) + 255) / 256, 256, 0, c->stream>>>(nparts, J, K, part, gW, gb);
  QP_CUDA(cudaGetLastError());
}

void check_tc_flag(qp_ctx* c) {
  int h = 0;
  QP_CUDA(cudaMemcpyAsync(&h, tc_flag(c), sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  QP_CUDA(cudaStreamSynchronize(c->stream));
  QP_REQUIRE(h == 0, QP_TIMEOUT, "tensor-core GEMM: a wait expired");
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
  QP_CUDA(cudaMemsetAsync(tc_flag(c), 0, sizeof(int), st));
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
      // H[l+1] = relu(W [H[l]; S[l]] + b): Nc x 128 by 128 x 64 on the tensor cores
      launch_tc_rows<MW, 4, 0>(c, n.H[l], n.S[l], 2, Nc, W, 2 * MW, 0, W + MW * 2 * MW, n.H[l + 1], nullptr);
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
  check_tc_flag(c);
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
  // (every buffer starts on a 256-byte boundary: the tensor-core GEMM reads A by TMA)
  auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t nparts = ((size_t)Nc + 255) / 256;
  const size_t o_dO = up((size_t)3 * Nc * sizeof(double)), o_A = o_dO + up((size_t)3 * Nc * sizeof(float));
  const size_t o_B = o_A + up((size_t)Nc * MW * 4), o_C = o_B + up((size_t)Nc * MW * 4);
  const size_t o_P = o_C + up((size_t)Nc * MW * 4);
  const size_t nb = o_P + nparts * MW * (2 * MW + 1) * sizeof(float);
  char* s = static_cast<char*>(c->mp_grad.ensure(nb));
  double* err = reinterpret_cast<double*>(s);
  float* dO = reinterpret_cast<float*>(s + o_dO);
  float* A = reinterpret_cast<float*>(s + o_A);
  float* B = reinterpret_cast<float*>(s + o_B);
  float* Cs = reinterpret_cast<float*>(s + o_C);
  float* part = reinterpret_cast<float*>(s + o_P);
  float* dM = n.Mb;  // the forward pass is done with it
  double* lsum = static_cast<double*>(c->mp_sum.ensure(64));  // the GEMM flag shares this buffer
  const long long nh = (long long)Nc * MW;
  k_mp_loss<<<blocks_for(3LL * Nc), 256, 0, st>>>(3 * Nc, n.O, target, dO, err);
  k_mp_sum<<<1, 256, 0, st>>>(3 * Nc, err, lsum);
  // head: o = Wo h3 + bo
  launch_wgrad<MO, MW>(c, dO, n.H[ML], MW, nullptr, part, grad + OFF_WO, grad + OFF_BO);
  k_mp_dense_bwd_x<<<blocks_for(nh), 256, 0, st>>>(Nc, dO, MO, n.pw + OFF_WO, MW, 0, A, nullptr);
  for (int l = ML - 1; l >= 0; --l) {
    // layer l: H[l+1] = relu(W [H[l]; S[l]] + b); A holds d/dH[l+1]
    const __nv_bfloat16* W = n.pw + OFF_L + l * LAYER;
    float* gW = grad + OFF_L + l * LAYER;
    k_mp_relu_bwd<<<blocks_for(nh), 256, 0, st>>>(nh, n.H[l + 1], A);
    launch_wgrad<MW, 2 * MW>(c, A, n.H[l], MW, n.S[l], part, gW, gW + MW * 2 * MW);
    // [dH[l], dS[l]] = dZ W: Nc x 64 by 64 x 128 on the tensor cores (B(n, j) = W[j][n])
    launch_tc_rows<2 * MW, 2, 1>(c, A, nullptr, 2, Nc, W, 2 * MW, 1, nullptr, B, Cs);
    // S[l] = gather(bodysum(H[l])): its adjoint is the same pair of sums
    k_mp_bodysum<<<blocks_for((long long)M * MW), 256, 0, st>>>(M, c->bptr.as<int>(), c->inc.as<int>(), Cs, dM);
    k_mp_gather<<<blocks_for(nh), 256, 0, st>>>(Nc, M, c->ca.as<int>(), c->cb.as<int>(), dM, B, 1);
    float* t = A;
    A = B;
    B = t;
  }
  // input layer: H[0] = relu(W0 X0 + b0)
  k_mp_relu_bwd<<<blocks_for(nh), 256, 0, st>>>(nh, n.H[0], A);
  launch_wgrad<MW, MF>(c, A, n.X0, MF, nullptr, part, grad + OFF_W0, grad + OFF_B0);
  QP_CUDA(cudaGetLastError());
  check_tc_flag(c);
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
