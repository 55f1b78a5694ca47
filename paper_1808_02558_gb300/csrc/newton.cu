// Newton-step operator and solvers of the PDIP iteration (Sec. 2.4, 3.3).
//
//  * Fused Schur apply y = S x, S = N + blockdiag(H_c), N = D^T M^-1 D (Eq. Ndef)
//    applied in factored form: a body pass gathers w_b = M_b^-1 sum_c D_cb x_c
//    over the body's contacts (CSR, fixed order, no atomics), then a contact
//    pass projects y_c = D_cb^T w_b + D_ca^T w_a + H_c x_c with the 3x3 frame and
//    block held in registers.
//  * Schur blocks H_c and the Newton right-hand side (Sec. 3.3 Schur
//    complement of Eq. qp_Newton_system).
//  * Preconditioned CG with Jacobi or QTT preconditioner as ONE persistent
//    cooperative kernel: every phase is a grid-stride loop separated by a
//    bounded grid barrier; FP64 outer iterative refinement around an inner
//    PCG in FP64 or FP32.
//  * PDIP pre-step (gap, t, residual norms, blocks, rhs, Jacobi diagonal) and
//    post-step (dlambda, ratio test, backtracking, update) as cooperative kernels.
#include <cooperative_groups.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <cmath>
#include <vector>

#include <type_traits>

#include "internal.cuh"
#include "qtt_dev.cuh"

namespace cg = cooperative_groups;

namespace qp {
namespace {

constexpr int NT = 512;               // threads per block of the cooperative kernels
constexpr int NT_FUSED = 512;         // threads per block of the fused pipelined kernel
constexpr int FUSED_MAX_CHUNK = 512;  // contacts per block up to which the fused kernel is used
constexpr int NWMAX = 32;             // warps per block at most
constexpr int NRED = 16;              // reduction slots per block
constexpr long long BARRIER_BUDGET = 4000000000LL;  // clock64 ticks (~2 s) per barrier wait

// ------------------------------------------------------------------ barrier
// Grid barrier with a bounded wait: on expiry it records QP_TIMEOUT in ctl->err
// and returns false; callers leave the kernel.  A block that finds the error
// flag set while it waits also returns false.
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void red_release_add(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Counter barrier: after a __syncthreads (which orders the writes of the whole
// block before thread 0's release), thread 0 of every block adds 1 to
// ctl->bar_count and polls it with acquire loads until it reaches
// generation x nblocks; a second __syncthreads hands the acquired state to the
// rest of the block.  The counter starts at 0 (the control block is cleared
// before every launch) and each block counts its generations in shared memory
// (every cooperative kernel calls barrier_init first).  One poller per block
// on one word keeps the polling traffic low.
__shared__ unsigned g_bar_gen;

__device__ __forceinline__ void barrier_init() {
  if (threadIdx.x == 0) g_bar_gen = 0;
  __syncthreads();
}

// Thread 0 only: arrive and wait (bounded).  Returns false on timeout or when
// another block has recorded an error.
__device__ __forceinline__ bool barrier_arrive_wait(DevCtl* ctl, unsigned nblocks, long long budget) {
  const unsigned gen = g_bar_gen + 1u;
  g_bar_gen = gen;
  red_release_add(&ctl->bar_count, 1u);
  const unsigned target = gen * nblocks;
  if ((int)(ld_acquire(&ctl->bar_count) - target) >= 0) return true;
  const long long t0 = clock64();
  for (;;) {
    if ((int)(ld_acquire(&ctl->bar_count) - target) >= 0) return true;
    if (*(volatile int*)&ctl->err) return false;
    if (clock64() - t0 > budget) {
      atomicCAS(&ctl->err, 0, QP_TIMEOUT);
      return false;
    }
  }
}

__device__ bool grid_barrier(DevCtl* ctl, unsigned nblocks, long long budget = BARRIER_BUDGET) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) ok = barrier_arrive_wait(ctl, nblocks, budget) ? 1 : 0;
  __syncthreads();
  return ok != 0;
}

template <class V>
__device__ __forceinline__ V warp_sum(V v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_min(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block-reduce n values (sum) and store them as this block's partials.  The
// per-thread and per-warp sums are taken in the accumulator type V, the
// cross-warp sum and the stored partial in the reduction type R: float in
// the FP32 inner solves, double elsewhere.  FP64 arithmetic is a narrow,
// long-latency pipe on this part, so FP64 sums are kept to short trees in one
// warp.  A float partial of slot s sits in the first half of double slot s.
template <class R>
__device__ __forceinline__ R* partial_slot(double* partial, int b, int slot) {
  return reinterpret_cast<R*>(partial + (size_t)b * NRED + slot);
}
template <class R>
__device__ __forceinline__ R load_partial(const double* partial, int b, int slot) {
  return *reinterpret_cast<volatile const R*>(partial + (size_t)b * NRED + slot);
}

template <int N, class V, class R = double>
__device__ void block_partials(V (&v)[N], double* partial, int slot0, bool is_min = false) {
  __shared__ R sm[N][NWMAX];
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int k = 0; k < N; ++k) {
    if (is_min) {
      const double x = warp_min((double)v[k]);
      if (lane == 0) sm[k][threadIdx.x >> 5] = (R)x;
    } else {
      const V x = warp_sum(v[k]);
      if (lane == 0) sm[k][threadIdx.x >> 5] = (R)x;
    }
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    for (int k = 0; k < N; ++k) {
      R x;
      if (is_min) {
        x = lane < nw ? sm[k][lane] : R(1e300);
        x = (R)warp_min((double)x);
      } else {
        x = lane < nw ? sm[k][lane] : R(0);
        x = warp_sum(x);
      }
      if (lane == 0) *partial_slot<R>(partial, blockIdx.x, slot0 + k) = x;
    }
  }
  __syncthreads();
}

// Sum (or min) of one partial slot over all blocks, same value in every block
// (warp 0 reduces, in a fixed order).
__device__ double grid_total(const double* partial, int slot, bool is_min = false) {
  __shared__ double res;
  if (threadIdx.x < 32) {
    double x = is_min ? 1e300 : 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += 32) {
      const double y = *(volatile const double*)&partial[(size_t)b * NRED + slot];
      x = is_min ? fmin(x, y) : x + y;
    }
    x = is_min ? warp_min(x) : warp_sum(x);
    if (threadIdx.x == 0) res = x;
  }
  __syncthreads();
  const double out = res;
  __syncthreads();
  return out;
}

// Grid barrier that also forms the totals of K consecutive partial slots
// (written by block_partials before the barrier).  Warp 0 adds the blocks'
// partials in a fixed order, so all blocks obtain bit-identical totals; then
// thread 0 runs `scal` on the totals (the scalar recurrences of a Krylov
// method, written to shared memory), so that FP64 scalar work is done once per
// block rather than by every thread.  Shared results are visible to the whole
// block when this returns and stay valid until the next barrier call.
struct NoScal {
  template <class R>
  __device__ void operator()(const R*) const {}
};

template <int K, class R = double, class F = NoScal>
__device__ bool grid_barrier_total(DevCtl* ctl, unsigned nblocks, const double* partial, int slot, R (&out)[K],
                                   F scal = F(), long long budget = BARRIER_BUDGET) {
  __shared__ R res[K];
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) ok = barrier_arrive_wait(ctl, nblocks, budget) ? 1 : 0;
  __syncthreads();
  const bool good = ok != 0;
  if (threadIdx.x < 32) {
    R x[K];
    for (int k = 0; k < K; ++k) x[k] = R(0);
    if (good)
      for (unsigned b = threadIdx.x; b < nblocks; b += 32)
        for (int k = 0; k < K; ++k) x[k] += load_partial<R>(partial, b, slot + k);
    for (int k = 0; k < K; ++k) x[k] = warp_sum(x[k]);
    if (threadIdx.x == 0) {
      for (int k = 0; k < K; ++k) res[k] = x[k];
      if (good) scal(res);
    }
  }
  __syncthreads();
  for (int k = 0; k < K; ++k) out[k] = res[k];
  return good;
}

// ------------------------------------------------------------------ operator
// Contact record c (16 values): n(3) t1(3) t2(3) ra(3) rb(3) 0.  Body
// intermediate w_b (8 values): M^-1 force (3), I^-1 torque (3), 2 pad.
__device__ __forceinline__ void load_rec(const float* rec, int c, float (&v)[16]) {
  const float4* p = reinterpret_cast<const float4*>(rec + (size_t)c * 16);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    float4 q = __ldg(p + k);
    v[4 * k] = q.x;
    v[4 * k + 1] = q.y;
    v[4 * k + 2] = q.z;
    v[4 * k + 3] = q.w;
  }
}
__device__ __forceinline__ void load_rec(const double* rec, int c, double (&v)[16]) {
  const double2* p = reinterpret_cast<const double2*>(rec + (size_t)c * 16);
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    double2 q = __ldg(p + k);
    v[2 * k] = q.x;
    v[2 * k + 1] = q.y;
  }
}
__device__ __forceinline__ void load_w(const float* w, int b, float (&v)[6]) {
  const float4* p = reinterpret_cast<const float4*>(w + (size_t)b * 8);
  float4 a = p[0], q = p[1];
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = q.x; v[5] = q.y;
}
__device__ __forceinline__ void load_w(const double* w, int b, double (&v)[6]) {
  const double2* p = reinterpret_cast<const double2*>(w + (size_t)b * 8);
  double2 a = p[0], q = p[1], r = p[2];
  v[0] = a.x; v[1] = a.y; v[2] = q.x; v[3] = q.y; v[4] = r.x; v[5] = r.y;
}
__device__ __forceinline__ void store_w(float* w, int b, const float (&v)[6]) {
  float4* p = reinterpret_cast<float4*>(w + (size_t)b * 8);
  p[0] = make_float4(v[0], v[1], v[2], v[3]);
  p[1] = make_float4(v[4], v[5], 0.f, 0.f);
}
__device__ __forceinline__ void store_w(double* w, int b, const double (&v)[6]) {
  double2* p = reinterpret_cast<double2*>(w + (size_t)b * 8);
  p[0] = make_double2(v[0], v[1]);
  p[1] = make_double2(v[2], v[3]);
  p[2] = make_double2(v[4], v[5]);
}

// Operand of the gather: x itself (beta == 0 and xprev == null) or the search
// direction z + beta * xprev formed on the fly.
template <class T>
struct Operand {
  const T* z;
  const T* prev;
  T beta;
  __device__ __forceinline__ T operator()(long long i) const {
    return prev ? z[i] + beta * prev[i] : z[i];
  }
};

// Accumulate D_cb^T-weighted force and torque of up to NB incidences (codes
// 2c + side, -1 = none); all record and operand loads are issued before use.
template <int NB, class T, class X>
__device__ __forceinline__ void gather_batch(const SysView<T>& s, const X& x, const int (&code)[NB], T& F0, T& F1,
                                             T& F2, T& Q0, T& Q1, T& Q2) {
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    if (code[j] < 0) continue;
    const int c = code[j] >> 1;
    const long long row = (long long)s.slots * c;
    T R[16];
    load_rec(s.rec, c, R);
    const T x0 = x(row), x1 = x(row + 1), x2 = x(row + 2);
    T f0 = R[0] * x0 + R[3] * x1 + R[6] * x2;
    T f1 = R[1] * x0 + R[4] * x1 + R[7] * x2;
    T f2 = R[2] * x0 + R[5] * x1 + R[8] * x2;
    const bool side_b = (code[j] & 1) != 0;
    const T a0 = side_b ? R[12] : R[9], a1 = side_b ? R[13] : R[10], a2 = side_b ? R[14] : R[11];
    const T sg = side_b ? T(1) : T(-1);
    f0 *= sg;
    f1 *= sg;
    f2 *= sg;
    F0 += f0;
    F1 += f1;
    F2 += f2;
    Q0 += a1 * f2 - a2 * f1;
    Q1 += a2 * f0 - a0 * f2;
    Q2 += a0 * f1 - a1 * f0;
  }
}

template <class T>
constexpr int gather_nb() {
  return sizeof(T) == 8 ? 2 : 4;  // batch size within the register budget
}

// w_b = M_b^-1 sum_{c in b} D_cb x_c   (force and torque of body b).
// Incidences are taken in batches (4 in FP32, 2 in FP64): their codes first,
// then all record and operand loads of the batch, so they are in flight together.
template <class T, class X, int NB = gather_nb<T>()>
__device__ __forceinline__ void body_gather_vals(const SysView<T>& s, const X& x, int b, T (&v)[6]) {
  T F0 = 0, F1 = 0, F2 = 0, Q0 = 0, Q1 = 0, Q2 = 0;
  const int e = __ldg(s.bptr + b + 1);
  for (int k0 = __ldg(s.bptr + b); k0 < e; k0 += NB) {
    int code[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j) code[j] = (k0 + j < e) ? __ldg(s.inc + k0 + j) : -1;
    gather_batch<NB>(s, x, code, F0, F1, F2, Q0, Q1, Q2);
  }
  const T im = __ldg(s.inv_m + b), iI = __ldg(s.inv_I + b);
  v[0] = im * F0;
  v[1] = im * F1;
  v[2] = im * F2;
  v[3] = iI * Q0;
  v[4] = iI * Q1;
  v[5] = iI * Q2;
}
template <class T, class X, int NB = gather_nb<T>()>
__device__ __forceinline__ void body_gather(const SysView<T>& s, const X& x, int b) {
  T v[6];
  body_gather_vals<T, X, NB>(s, x, b, v);
  store_w(s.w, b, v);
}

// Per-block work ranges and per-thread gather plan of a persistent Krylov
// kernel, kept in shared memory for the whole launch.  Block g owns a
// contiguous range of bodies holding an equal share (1/G) of the incidences,
// and an equal contiguous share of the contacts, so that every SM gets the
// same work in each operator pass.  Thread t of the block keeps the incidence
// codes of its first body (up to PLAN_INC of them) and the body pairs of its
// first PLAN_CON contacts, which removes the CSR and body-index loads, and
// the load-to-load dependence they create, from every operator application.
constexpr int PLAN_INC = 12;
constexpr int PLAN_CON = 3;
struct GatherPlan {
  int code[PLAN_INC][NT];
  int n[NT];                 // incidences of the thread's first body (0: none)
  int off[NT];               // its first incidence, counted from the block's first
  int ca[PLAN_CON][NT];
  int cb[PLAN_CON][NT];
  int b0, b1;                // bodies [b0, b1) of this block
  int c0, c1;                // contacts [c0, c1) of this block
  int base;                  // the block's first incidence (CSR position)
  int ncache;                // incidences whose geometry is cached (0: no cache)
  const float4* cache;       // [ncache][3] sign-folded frame and arm per incidence
};

// first body whose incidence range ends above k (bptr is nondecreasing)
__device__ __forceinline__ int body_at_incidence(const int* bptr, int M, long long k) {
  int lo = 0, hi = M;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if ((long long)__ldg(bptr + mid + 1) <= k) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

template <class T>
__device__ void plan_fill(const SysView<T>& s, GatherPlan& pl) {
  const int t = threadIdx.x;
  const long long G = gridDim.x, g = blockIdx.x;
  if (t == 0) {
    const long long ninc = s.M > 0 ? (long long)__ldg(s.bptr + s.M) : 0;
    pl.b0 = g == 0 ? 0 : body_at_incidence(s.bptr, s.M, ninc * g / G);
    pl.b1 = g == G - 1 ? s.M : body_at_incidence(s.bptr, s.M, ninc * (g + 1) / G);
    pl.c0 = (int)(s.Nc * g / G);
    pl.c1 = (int)(s.Nc * (g + 1) / G);
  }
  __syncthreads();
  if (t == 0) {
    pl.base = s.M > 0 ? __ldg(s.bptr + pl.b0) : 0;
    pl.ncache = 0;
    pl.cache = nullptr;
  }
  __syncthreads();
  int n = 0, off = 0;
  const int b = pl.b0 + t;
  if (b < pl.b1) {
    const int k0 = __ldg(s.bptr + b);
    n = __ldg(s.bptr + b + 1) - k0;
    off = k0 - pl.base;
    for (int j = 0; j < PLAN_INC && j < n; ++j) pl.code[j][t] = __ldg(s.inc + k0 + j);
  }
  pl.n[t] = n;
  pl.off[t] = off;
#pragma unroll
  for (int k = 0; k < PLAN_CON; ++k) {
    const int c = pl.c0 + t + k * (int)blockDim.x;
    pl.ca[k][t] = c < pl.c1 ? __ldg(s.ca + c) : 0;
    pl.cb[k][t] = c < pl.c1 ? __ldg(s.cb + c) : 0;
  }
  __syncthreads();
}

// Cache in shared memory, for the whole launch, the geometry the body gather
// needs from each incidence of the block's bodies (the first `cap` of them):
// the contact frame with the side's sign folded in, and the side's arm,
//   q[0] = s (n.x n.y n.z t1.x), q[1] = s (t1.y t1.z t2.x t2.y),
//   q[2] = (s t2.z, arm.x, arm.y, arm.z),  s = +1 for body b, -1 for body a,
// so that f = [q] x and the torque is arm x f.  Record loads were the largest
// part of the gather's time.
__device__ void plan_fill_cache(const SysView<float>& s, GatherPlan& pl, float4* cache, int cap) {
  const int nb = pl.b1 > pl.b0 ? __ldg(s.bptr + pl.b1) - pl.base : 0;
  const int nc = nb < cap ? nb : cap;
  for (int k = threadIdx.x; k < nc; k += blockDim.x) {
    const int code = __ldg(s.inc + pl.base + k);
    const int c = code >> 1;
    const bool side_b = (code & 1) != 0;
    float R[16];
    load_rec(s.rec, c, R);
    const float sg = side_b ? 1.f : -1.f;
    const float a0 = side_b ? R[12] : R[9], a1 = side_b ? R[13] : R[10], a2 = side_b ? R[14] : R[11];
    cache[3 * k] = make_float4(sg * R[0], sg * R[1], sg * R[2], sg * R[3]);
    cache[3 * k + 1] = make_float4(sg * R[4], sg * R[5], sg * R[6], sg * R[7]);
    cache[3 * k + 2] = make_float4(sg * R[8], a0, a1, a2);
  }
  if (threadIdx.x == 0) {
    pl.ncache = nc;
    pl.cache = cache;
  }
  __syncthreads();
}

// body_gather for the thread's planned body with the cached geometry: per
// incidence three shared-memory loads and the operand's rows.
template <class X>
__device__ __forceinline__ void body_gather_cached(const SysView<float>& s, const X& x, const GatherPlan& pl, int b) {
  const int t = threadIdx.x;
  const int n = pl.n[t], off = pl.off[t];
  float F0 = 0, F1 = 0, F2 = 0, Q0 = 0, Q1 = 0, Q2 = 0;
  const float im = __ldg(s.inv_m + b), iI = __ldg(s.inv_I + b);
  constexpr int NB = 4;
#pragma unroll
  for (int k0 = 0; k0 < PLAN_INC; k0 += NB) {
    if (k0 < n) {
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        if (k0 + j < n) {
          const int code = pl.code[k0 + j][t];
          const int k = off + k0 + j;
          const long long row = (long long)s.slots * (code >> 1);
          const float x0 = x(row), x1 = x(row + 1), x2 = x(row + 2);
          float f0, f1, f2, a0, a1, a2;
          if (k < pl.ncache) {
            const float4 q0 = pl.cache[3 * k], q1 = pl.cache[3 * k + 1], q2 = pl.cache[3 * k + 2];
            f0 = q0.x * x0 + q0.w * x1 + q1.z * x2;
            f1 = q0.y * x0 + q1.x * x1 + q1.w * x2;
            f2 = q0.z * x0 + q1.y * x1 + q2.x * x2;
            a0 = q2.y;
            a1 = q2.z;
            a2 = q2.w;
          } else {
            float R[16];
            load_rec(s.rec, code >> 1, R);
            const bool side_b = (code & 1) != 0;
            const float sg = side_b ? 1.f : -1.f;
            f0 = sg * (R[0] * x0 + R[3] * x1 + R[6] * x2);
            f1 = sg * (R[1] * x0 + R[4] * x1 + R[7] * x2);
            f2 = sg * (R[2] * x0 + R[5] * x1 + R[8] * x2);
            a0 = side_b ? R[12] : R[9];
            a1 = side_b ? R[13] : R[10];
            a2 = side_b ? R[14] : R[11];
          }
          F0 += f0;
          F1 += f1;
          F2 += f2;
          Q0 += a1 * f2 - a2 * f1;
          Q1 += a2 * f0 - a0 * f2;
          Q2 += a0 * f1 - a1 * f0;
        }
      }
    }
  }
  if (n > PLAN_INC) {
    const int b0 = __ldg(s.bptr + b);
    for (int k0 = b0 + PLAN_INC; k0 < b0 + n; k0 += NB) {
      int code[NB];
#pragma unroll
      for (int j = 0; j < NB; ++j) code[j] = (k0 + j < b0 + n) ? __ldg(s.inc + k0 + j) : -1;
      gather_batch<NB>(s, x, code, F0, F1, F2, Q0, Q1, Q2);
    }
  }
  float v[6] = {im * F0, im * F1, im * F2, iI * Q0, iI * Q1, iI * Q2};
  store_w(s.w, b, v);
}

// body_gather for the thread's planned body b (= b0 + threadIdx.x).
template <class T, class X, int NB = gather_nb<T>()>
__device__ __forceinline__ void body_gather_planned(const SysView<T>& s, const X& x, const GatherPlan& pl, int b) {
  const int t = threadIdx.x;
  const int n = pl.n[t];
  T F0 = 0, F1 = 0, F2 = 0, Q0 = 0, Q1 = 0, Q2 = 0;
  const T im = __ldg(s.inv_m + b), iI = __ldg(s.inv_I + b);
#pragma unroll
  for (int k0 = 0; k0 < PLAN_INC; k0 += NB) {
    if (k0 < n) {
      int code[NB];
#pragma unroll
      for (int j = 0; j < NB; ++j) code[j] = (k0 + j < n) ? pl.code[k0 + j][t] : -1;
      gather_batch<NB>(s, x, code, F0, F1, F2, Q0, Q1, Q2);
    }
  }
  if (n > PLAN_INC) {
    const int b0 = __ldg(s.bptr + b);
    for (int k0 = b0 + PLAN_INC; k0 < b0 + n; k0 += NB) {
      int code[NB];
#pragma unroll
      for (int j = 0; j < NB; ++j) code[j] = (k0 + j < b0 + n) ? __ldg(s.inc + k0 + j) : -1;
      gather_batch<NB>(s, x, code, F0, F1, F2, Q0, Q1, Q2);
    }
  }
  T v[6] = {im * F0, im * F1, im * F2, iI * Q0, iI * Q1, iI * Q2};
  store_w(s.w, b, v);
}

// y_c = U^T [(v_b + w_b x rb) - (v_a + w_a x ra)] + H_c x_c ; returns x_c . y_c.
// If xout is set, the operand value of row i is also stored there (the
// materialised search direction).
template <class T, class X>
__device__ __forceinline__ T contact_apply_ab(const SysView<T>& s, const X& x, T* y, int c, int a, int b,
                                              T* xout = nullptr) {
  const long long n = s.Nc;
  T R[16];
  load_rec(s.rec, c, R);
  T wb[6];
  load_w(s.w, b, wb);
  T d0 = wb[0] + (wb[4] * R[14] - wb[5] * R[13]);
  T d1 = wb[1] + (wb[5] * R[12] - wb[3] * R[14]);
  T d2 = wb[2] + (wb[3] * R[13] - wb[4] * R[12]);
  if (a < s.M) {
    T wa[6];
    load_w(s.w, a, wa);
    d0 -= wa[0] + (wa[4] * R[11] - wa[5] * R[10]);
    d1 -= wa[1] + (wa[5] * R[9] - wa[3] * R[11]);
    d2 -= wa[2] + (wa[3] * R[10] - wa[4] * R[9]);
  }
  const long long row = (long long)s.slots * c;
  const T x0 = x(row), x1 = x(row + 1), x2 = x(row + 2);
  T y0 = R[0] * d0 + R[1] * d1 + R[2] * d2;
  T y1 = R[3] * d0 + R[4] * d1 + R[5] * d2;
  T y2 = R[6] * d0 + R[7] * d1 + R[8] * d2;
  if (s.H) {
    const T* H = s.H;
    T h00 = __ldg(H + c), h01 = __ldg(H + n + c), h02 = __ldg(H + 2 * n + c);
    T h11 = __ldg(H + 3 * n + c), h12 = __ldg(H + 4 * n + c), h22 = __ldg(H + 5 * n + c);
    y0 += h00 * x0 + h01 * x1 + h02 * x2;
    y1 += h01 * x0 + h11 * x1 + h12 * x2;
    y2 += h02 * x0 + h12 * x1 + h22 * x2;
  }
  y[row] = y0;
  y[row + 1] = y1;
  y[row + 2] = y2;
  T dot = x0 * y0 + x1 * y1 + x2 * y2;
  if (xout) {
    xout[row] = x0;
    xout[row + 1] = x1;
    xout[row + 2] = x2;
  }
  if (s.slots == 4) {
    const T x3 = x(row + 3);
    y[row + 3] = x3;
    if (xout) xout[row + 3] = x3;
    dot += x3 * x3;
  }
  return dot;
}

template <class T, class X>
__device__ __forceinline__ T contact_apply(const SysView<T>& s, const X& x, T* y, int c, T* xout = nullptr) {
  return contact_apply_ab(s, x, y, c, __ldg(s.ca + c), __ldg(s.cb + c), xout);
}

// Operator passes of a persistent kernel with a gather plan: w for the
// block's bodies, then y for the block's contacts (returns the thread's share
// of x . y).
template <class T, class X, int NB = gather_nb<T>()>
__device__ __forceinline__ void gather_all(const SysView<T>& s, const X& x, const GatherPlan& pl) {
  const int b = pl.b0 + threadIdx.x;
  if constexpr (sizeof(T) == 4) {
    if (pl.cache) {
      if (b < pl.b1) body_gather_cached(s, x, pl, b);
      for (int bd = b + blockDim.x; bd < pl.b1; bd += blockDim.x) body_gather<T, X, NB>(s, x, bd);
      return;
    }
  }
  if (b < pl.b1) body_gather_planned<T, X, NB>(s, x, pl, b);
  for (int bd = b + blockDim.x; bd < pl.b1; bd += blockDim.x) body_gather<T, X, NB>(s, x, bd);
}
template <class T, class X>
__device__ __forceinline__ T apply_all(const SysView<T>& s, const X& x, T* y, const GatherPlan& pl, T* xout) {
  T acc = 0;
  const int c = pl.c0 + threadIdx.x;
#pragma unroll
  for (int k = 0; k < PLAN_CON; ++k) {
    const int ck = c + k * (int)blockDim.x;
    if (ck < pl.c1) acc += contact_apply_ab(s, x, y, ck, pl.ca[k][threadIdx.x], pl.cb[k][threadIdx.x], xout);
  }
  for (int ck = c + PLAN_CON * (int)blockDim.x; ck < pl.c1; ck += blockDim.x) acc += contact_apply(s, x, y, ck, xout);
  return acc;
}

template <class T>
__device__ __forceinline__ Operand<T> plain(const T* x) {
  return Operand<T>{x, nullptr, T(0)};
}

// Standalone body gather with L lanes per body, one body per lane group (no
// grid-stride loop, so every lane reaches the shuffles): lane j takes the
// body's incidences j, j + L, ... two at a time, the L partial force and
// torque sums are combined by butterfly shuffles within the aligned group, and
// lane 0 scales and stores w_b.  A thread per body leaves too few loads in
// flight when the caches are cold (64 k bodies on 152 SMs); four lanes per body
// measured faster than one or eight on the 40^3 pile (FP32 apply 27 -> 23 us).
#ifndef QP_APPLY_LANES
#define QP_APPLY_LANES 4
#endif
template <class T, int L>
__global__ void k_body_gather_lanes(SysView<T> s, const T* x) {
  static_assert(L >= 1 && L <= 32 && (L & (L - 1)) == 0, "lanes: a power of two up to 32");
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long b = t / L;
  const int lane = (int)(t & (L - 1));
  T F0 = 0, F1 = 0, F2 = 0, Q0 = 0, Q1 = 0, Q2 = 0;
  if (b < s.M) {
    const int e = __ldg(s.bptr + b + 1);
    for (int k = __ldg(s.bptr + b) + lane; k < e; k += 2 * L) {
      const int code[2] = {__ldg(s.inc + k), k + L < e ? __ldg(s.inc + k + L) : -1};
      gather_batch<2>(s, plain(x), code, F0, F1, F2, Q0, Q1, Q2);
    }
  }
#pragma unroll
  for (int o = L / 2; o > 0; o >>= 1) {
    F0 += __shfl_xor_sync(0xffffffffu, F0, o);
    F1 += __shfl_xor_sync(0xffffffffu, F1, o);
    F2 += __shfl_xor_sync(0xffffffffu, F2, o);
    Q0 += __shfl_xor_sync(0xffffffffu, Q0, o);
    Q1 += __shfl_xor_sync(0xffffffffu, Q1, o);
    Q2 += __shfl_xor_sync(0xffffffffu, Q2, o);
  }
  if (b < s.M && lane == 0) {
    const T im = __ldg(s.inv_m + b), iI = __ldg(s.inv_I + b);
    T v[6] = {im * F0, im * F1, im * F2, iI * Q0, iI * Q1, iI * Q2};
    store_w(s.w, b, v);
  }
}

template <class T>
__global__ void k_contact_apply(SysView<T> s, const T* x, T* y) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < s.Nc; c += gridDim.x * blockDim.x)
    contact_apply(s, plain(x), y, c);
  // dummy tail rows: identity
  const long long tail0 = (long long)s.slots * s.Nc;
  for (long long i = tail0 + blockIdx.x * (long long)blockDim.x + threadIdx.x; i < s.P;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = x[i];
}

// ------------------------------------------------------------------ PDIP pieces
struct PdipView {
  int Nc, slots;
  double mu;
  double* gamma;   // [P]
  double* lambda;  // [2Nc]
};

// H_c = l_c diag(-mu^2,1,1) + (l_c/(-f_c)) g g^T + (l'_c/gn) e1 e1^T, g = grad f_c
__device__ __forceinline__ void schur_block(double mu, double gn, double g1, double g2, double lc, double ln,
                                            double h[6]) {
  double fc = 0.5 * (g1 * g1 + g2 * g2 - mu * mu * gn * gn);
  double q0 = -mu * mu * gn, q1 = g1, q2 = g2;
  double sc = lc / (-fc);
  h[0] = -mu * mu * lc + sc * q0 * q0 + ln / gn;
  h[1] = sc * q0 * q1;
  h[2] = sc * q0 * q2;
  h[3] = lc + sc * q1 * q1;
  h[4] = sc * q1 * q2;
  h[5] = lc + sc * q2 * q2;
}

__global__ void k_schur_blocks(PdipView v, double* __restrict__ H, float* __restrict__ H32) {
  const int n = v.Nc;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
    const long long row = (long long)v.slots * c;
    double h[6];
    schur_block(v.mu, v.gamma[row], v.gamma[row + 1], v.gamma[row + 2], v.lambda[c], v.lambda[n + c], h);
    for (int k = 0; k < 6; ++k) {
      H[(size_t)k * n + c] = h[k];
      H32[(size_t)k * n + c] = (float)h[k];
    }
  }
}

// Contact pass of the standalone FP64 apply with the Schur block of each
// contact formed in registers from (gamma_c, lambda_c) (none when gamma is
// null): y_c = U_c^T (w terms) + H_c x_c; dummy rows copy x.
__global__ void k_contact_apply_h(SysView<double> s, const double* __restrict__ x, double* __restrict__ y,
                                  const double* __restrict__ gamma, const double* __restrict__ lambda, double mu) {
  const int n = s.Nc;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
    const long long row = (long long)s.slots * c;
    contact_apply(s, plain(x), y, c);
    if (gamma) {
      double h[6];
      schur_block(mu, gamma[row], gamma[row + 1], gamma[row + 2], lambda[c], lambda[n + c], h);
      const double x0 = x[row], x1 = x[row + 1], x2 = x[row + 2];
      y[row] += h[0] * x0 + h[1] * x1 + h[2] * x2;
      y[row + 1] += h[1] * x0 + h[3] * x1 + h[4] * x2;
      y[row + 2] += h[2] * x0 + h[4] * x1 + h[5] * x2;
    }
  }
  const long long tail0 = (long long)s.slots * n;
  for (long long i = tail0 + blockIdx.x * (long long)blockDim.x + threadIdx.x; i < s.P;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = x[i];
}

// Diagonal entry (c, u) of N = D^T M^-1 D: sum over the contact's dynamic
// bodies of 1/m + (rho x U_u)^T I^-1 (rho x U_u).
__device__ __forceinline__ double diag_entry(const SysView<double>& s, int c, int u) {
  double R[16];
  load_rec(s.rec, c, R);
  const double U0 = R[3 * u], U1 = R[3 * u + 1], U2 = R[3 * u + 2];
  const int a = s.ca[c], b = s.cb[c];
  double t0 = R[13] * U2 - R[14] * U1, t1 = R[14] * U0 - R[12] * U2, t2 = R[12] * U1 - R[13] * U0;
  double v = s.inv_m[b] + s.inv_I[b] * (t0 * t0 + t1 * t1 + t2 * t2);
  if (a < s.M) {
    t0 = R[10] * U2 - R[11] * U1;
    t1 = R[11] * U0 - R[9] * U2;
    t2 = R[9] * U1 - R[10] * U0;
    v += s.inv_m[a] + s.inv_I[a] * (t0 * t0 + t1 * t1 + t2 * t2);
  }
  return v;
}

// ------------------------------------------------------------------ PCG kernel
struct PcgArgs {
  SysView<double> s64;
  SysView<float> s32;
  int nrow;                 // slots * Nc
  long long P;
  const double* rhs;        // [P]
  double* x;                // [P] solution (FP64)
  double* r64;              // [P] outer residual
  double* q64;              // [P]
  // inner vectors, type T (double or float), each [P]
  void* b;
  void* e;
  void* r;
  void* z;
  void* p;
  void* q;
  const void* dinv;         // Jacobi diagonal inverse (type T)
  int use_qtt;
  int qtt_scaled;           // preconditioner is D^-1/2 X D^-1/2 (X approximates the scaled inverse)
  QttDev qtt;
  void* qw0;                // QTT work buffers (type T), rmax * P each
  void* qw1;
  void* xb;                 // BiCGSTAB vectors (type T), 5 * P
  int krylov;               // QP_CG or QP_BICGSTAB
  int direct;               // QTT direct mode: the inner solve is one application of X
  int reliable;             // FP32 Jacobi-CG with reliable updates instead of restarted refinement
  int rec_cache;            // incidences of a block whose gather geometry is cached in shared memory (0: none)
  double tol, inner_tol;
  int maxit, max_outer;
  DevCtl* ctl;
  double* partial;
};

template <class T>
__device__ __forceinline__ const SysView<T>& sys_of(const PcgArgs& a);
template <>
__device__ __forceinline__ const SysView<double>& sys_of<double>(const PcgArgs& a) { return a.s64; }
template <>
__device__ __forceinline__ const SysView<float>& sys_of<float>(const PcgArgs& a) { return a.s32; }

// z = X r through the QTT cores (d grid-synchronised steps).  For a Jacobi-
// scaled preconditioner z = D^-1/2 X D^-1/2 r, the scalings taken from the
// Jacobi diagonal inverse (sqrt(dinv) = D^-1/2).
template <class T, class TC>
__device__ bool qtt_precond(const PcgArgs& A, const T* r, T* z) {
  const QttDev& q = A.qtt;
  const long long items = A.P >> 1;
  const long long gsz = (long long)gridDim.x * blockDim.x;
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const T* dinv = static_cast<const T*>(A.dinv);
  const T* in = r;
  if (A.qtt_scaled) {
    // the last core's step reads this buffer and writes qw0; qw1 is free until the next step
    T* tmp = static_cast<T*>(A.qw1);
    for (long long i = tid; i < A.P; i += gsz) tmp[i] = i < A.nrow ? sqrt(dinv[i]) * r[i] : T(0);
    if (!grid_barrier(A.ctl, gridDim.x)) return false;
    in = tmp;
  }
  // one grid-synchronised pass per two cores where the ranks allow (else one)
  constexpr int GQ = 2 * 12 * 12;
  __shared__ Quad<T> gq[GQ];
  T* gc = reinterpret_cast<T*>(gq);  // single-core staging (4 * 16 * 16 values fit in GQ quads)
  int pass = 0;
  for (int k = q.d; k >= 1; ++pass) {
    const int bound = qtt_fuse_bound<T>(q, k, GQ);
    const int next = bound ? k - 2 : k - 1;
    T* out = (next == 0) ? z : static_cast<T*>((pass & 1) ? A.qw1 : A.qw0);
    if (bound) qtt_step2_grid<T, T, TC>(q, k, in, out, gq, bound);
    else qtt_step_grid<T, T, TC>(q, k, in, out, items, gc, 4 * GQ);
    if (!grid_barrier(A.ctl, gridDim.x)) return false;
    in = out;
    k = next;
  }
  if (A.qtt_scaled) {
    for (long long i = tid; i < A.nrow; i += gsz) z[i] *= sqrt(dinv[i]);
    if (!grid_barrier(A.ctl, gridDim.x)) return false;
  }
  return true;
}

// Inner PCG on S_T e = b (x0 = 0) to ||b - S e|| <= tol ||b||.  Returns
// 0 converged, 1 cap reached, 2 breakdown, -1 barrier failure.
//
// Three grid barriers per iteration: the search direction p_k = z + beta p_{k-1}
// is never materialised before the operator: the body gather forms it on the
// fly from (z, p_{k-1}), and the contact pass stores it into the other p buffer
// while it computes q = S p_k.
// TC = void instantiates the Jacobi-only solver: no QTT code, fewer registers.
template <class TC>
constexpr bool kQtt = !std::is_void_v<TC>;

template <class T, class TC>
__device__ __forceinline__ bool qtt_precond_if(const PcgArgs& A, const T* in, T* out) {
  if constexpr (kQtt<TC>) return qtt_precond<T, TC>(A, in, out);
  else return false;
}

template <class T, class TC>
__device__ int inner_pcg(const PcgArgs& A, const GatherPlan& pl, double tol, int maxit, int& iters) {
  const SysView<T>& s = sys_of<T>(A);
  T* b = static_cast<T*>(A.b);
  T* e = static_cast<T*>(A.e);
  T* r = static_cast<T*>(A.r);
  T* z = static_cast<T*>(A.z);
  T* pa = static_cast<T*>(A.p);
  T* pb = static_cast<T*>(A.q) + A.P;  // second search-direction buffer
  T* q = static_cast<T*>(A.q);
  const T* dinv = static_cast<const T*>(A.dinv);
  const long long gsz = (long long)gridDim.x * blockDim.x;
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int nrow = A.nrow;
  const unsigned nb = gridDim.x;

  // setup: e = 0, r = b, z = M^-1 r
  T acc[2] = {};
  for (long long i = tid; i < nrow; i += gsz) {
    T bi = b[i];
    e[i] = 0;
    r[i] = bi;
    acc[0] += bi * bi;
    if (!(kQtt<TC> && A.use_qtt)) {
      T zi = dinv[i] * bi;
      z[i] = zi;
      acc[1] += bi * zi;
    }
  }
  // reductions and scalar recurrences in T (float in the FP32 inner solve)
  block_partials<2, T, T>(acc, A.partial, 0);
  T t0[2];
  if (!grid_barrier_total<2, T>(A.ctl, nb, A.partial, 0, t0)) return -1;
  const T bb = t0[0];
  T rz = t0[1];
  if (bb == T(0)) return 0;
  if ((kQtt<TC> && A.use_qtt)) {
    if (!qtt_precond_if<T, TC>(A, r, z)) return -1;
    T a1[1] = {};
    for (long long i = tid; i < nrow; i += gsz) a1[0] += r[i] * z[i];
    block_partials<1, T, T>(a1, A.partial, 1);
    T t1[1];
    if (!grid_barrier_total<1, T>(A.ctl, nb, A.partial, 1, t1)) return -1;
    rz = t1[0];
  }
  const T stop = (T)(tol * tol) * bb;
  T* pold = pa;   // p_{k-1} (unused while beta == 0)
  T* pnew = pb;   // p_k, written by the contact pass
  T beta = 0;
  for (int it = 0; it < maxit; ++it) {
    if (!(rz > T(0))) return 2;
    const Operand<T> dir{z, it == 0 ? nullptr : pold, beta};
    // q = S p_k
    gather_all(s, dir, pl);
    if (!grid_barrier(A.ctl, nb)) return -1;
    T a2[1] = {apply_all(s, dir, q, pl, pnew)};
    block_partials<1, T, T>(a2, A.partial, 2);
    T t2[1];
    __shared__ T s_alpha;
    if (!grid_barrier_total<1, T>(A.ctl, nb, A.partial, 2, t2,
                                  [&](const T* t) { s_alpha = t[0] > T(0) ? rz / t[0] : T(0); }))
      return -1;
    const T pq = t2[0];
    if (!(pq > T(0))) return 2;
    const T alpha = s_alpha;
    T a3[2] = {};
    bool updated = false;
    if constexpr (sizeof(T) == 4) {
      if (!(kQtt<TC> && A.use_qtt)) {
        // FP32 Jacobi: four rows per thread with float4 loads and stores (all
        // buffers are allocated with P >= round_up(nrow, 4) values, 16-byte aligned)
        const long long n4 = nrow >> 2;
        const float4* P4 = reinterpret_cast<const float4*>(pnew);
        const float4* Q4 = reinterpret_cast<const float4*>(q);
        const float4* D4 = reinterpret_cast<const float4*>(dinv);
        float4* E4 = reinterpret_cast<float4*>(e);
        float4* R4 = reinterpret_cast<float4*>(r);
        float4* Z4 = reinterpret_cast<float4*>(z);
        const float al = (float)alpha;
        // the block's equal share of the float4 rows; two float4 per thread
        // and pass, all loads of the pass before any store
        const long long u0 = n4 * blockIdx.x / gridDim.x, u1 = n4 * (blockIdx.x + 1) / gridDim.x;
        const long long bs = blockDim.x;
        for (long long i0 = u0 + threadIdx.x; i0 < u1; i0 += 2 * bs) {
          float4 pv[2], qv[2], dv[2], ev[2], rv[2];
#pragma unroll
          for (int j = 0; j < 2; ++j) {
            const long long i = i0 + j * bs;
            if (i < u1) {
              pv[j] = P4[i];
              qv[j] = Q4[i];
              dv[j] = D4[i];
              ev[j] = E4[i];
              rv[j] = R4[i];
            }
          }
#pragma unroll
          for (int j = 0; j < 2; ++j) {
            const long long i = i0 + j * bs;
            if (i >= u1) break;
            float4 e4 = ev[j], r4 = rv[j];
            e4.x += al * pv[j].x; e4.y += al * pv[j].y; e4.z += al * pv[j].z; e4.w += al * pv[j].w;
            r4.x -= al * qv[j].x; r4.y -= al * qv[j].y; r4.z -= al * qv[j].z; r4.w -= al * qv[j].w;
            const float4 z4 = make_float4(dv[j].x * r4.x, dv[j].y * r4.y, dv[j].z * r4.z, dv[j].w * r4.w);
            E4[i] = e4;
            R4[i] = r4;
            Z4[i] = z4;
            a3[0] += r4.x * r4.x + r4.y * r4.y + r4.z * r4.z + r4.w * r4.w;
            a3[1] += r4.x * z4.x + r4.y * z4.y + r4.z * z4.z + r4.w * z4.w;
          }
        }
        for (long long i = (n4 << 2) + tid; i < nrow; i += gsz) {
          e[i] += (T)alpha * pnew[i];
          const T ri = r[i] - (T)alpha * q[i];
          r[i] = ri;
          const T zi = dinv[i] * ri;
          z[i] = zi;
          a3[0] += ri * ri;
          a3[1] += ri * zi;
        }
        updated = true;
      }
    }
    if (!updated) {
    // several rows per thread and pass: every load of the batch before any store
    constexpr int RB = sizeof(T) == 8 ? 2 : 4;
    for (long long i0 = tid; i0 < nrow; i0 += RB * gsz) {
      T pv[RB], ev[RB], rv[RB], qv[RB], dv[RB];
#pragma unroll
      for (int j = 0; j < RB; ++j) {
        const long long i = i0 + j * gsz;
        const bool in = i < nrow;
        pv[j] = in ? pnew[i] : T(0);
        ev[j] = in ? e[i] : T(0);
        rv[j] = in ? r[i] : T(0);
        qv[j] = in ? q[i] : T(0);
        dv[j] = in ? dinv[i] : T(0);
      }
#pragma unroll
      for (int j = 0; j < RB; ++j) {
        const long long i = i0 + j * gsz;
        if (i >= nrow) break;
        e[i] = ev[j] + (T)alpha * pv[j];
        const T ri = rv[j] - (T)alpha * qv[j];
        r[i] = ri;
        a3[0] += ri * ri;
        if (!(kQtt<TC> && A.use_qtt)) {
          const T zi = dv[j] * ri;
          z[i] = zi;
          a3[1] += ri * zi;
        }
      }
    }
    }
    block_partials<2, T, T>(a3, A.partial, 3);
    T t3[2];
    __shared__ T s_beta;
    if (!grid_barrier_total<2, T>(A.ctl, nb, A.partial, 3, t3, [&](const T* t) { s_beta = t[1] / rz; }))
      return -1;
    ++iters;
    const T rr = t3[0];
    T rz_new;
    if (rr <= stop) return 0;
    if ((kQtt<TC> && A.use_qtt)) {
      if (!qtt_precond_if<T, TC>(A, r, z)) return -1;
      T a4[1] = {};
      for (long long i = tid; i < nrow; i += gsz) a4[0] += r[i] * z[i];
      block_partials<1, T, T>(a4, A.partial, 5);
      T t4[1];
      if (!grid_barrier_total<1, T>(A.ctl, nb, A.partial, 5, t4, [&](const T* t) { s_beta = t[0] / rz; }))
        return -1;
      rz_new = t4[0];
    } else {
      rz_new = t3[1];
    }
    beta = s_beta;
    rz = rz_new;
    T* t = pold;
    pold = pnew;
    pnew = t;
  }
  return 1;
}

// Mixed-precision Jacobi-PCG with reliable updates (residual replacement; van
// der Vorst and Ye, SIAM J. Sci. Comput. 22 (2000); its mixed-precision use in
// Clark et al., Comput. Phys. Commun. 181 (2010)).  The FP32 CG recursion runs
// without restarts on S e = r, r = (rhs - S x) / scale.  Whenever its
// recurrence residual has fallen by inner_tol since the last replacement (or
// says the target is reached), the FP32 increment is added to the FP64
// solution x, the true residual rhs - S x is formed in FP64 and replaces the
// FP32 residual (rescaled to unit norm), and the search direction is kept:
// with r and z in the new units, p_old in the old ones,
//   p = z + beta p_old,  beta = (r.z)_new / (r.z)_old * (scale_new / scale_old).
// An outer restart per refinement would discard the Krylov space each time.
// Returns 0 converged (true FP64 residual <= tol ||rhs||), 1 cap reached,
// 2 breakdown, -1 barrier failure; `repl` counts FP64 residual evaluations.
__device__ int pcg_reliable(const PcgArgs& A, const GatherPlan& pl, double bnorm, int& iters, int& repl,
                            double& rel) {
  using T = float;
  const SysView<T>& s = A.s32;
  const SysView<double>& s64 = A.s64;
  T* e = static_cast<T*>(A.e);
  T* r = static_cast<T*>(A.r);
  T* z = static_cast<T*>(A.z);
  T* q = static_cast<T*>(A.q);
  T* pold = static_cast<T*>(A.p);        // p_{k-1}
  T* pnew = static_cast<T*>(A.q) + A.P;  // p_k, written by the contact pass
  const T* dinv = static_cast<const T*>(A.dinv);
  const long long gsz = (long long)gridDim.x * blockDim.x;
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int nrow = A.nrow;
  const unsigned nb = gridDim.x;
  const double target = A.tol * bnorm;
  double scale = bnorm;
  T a0[1] = {};
  for (long long i = tid; i < nrow; i += gsz) {
    const T ri = (T)(A.rhs[i] / scale);
    r[i] = ri;
    e[i] = 0;
    const T zi = dinv[i] * ri;
    z[i] = zi;
    a0[0] += ri * zi;
  }
  block_partials<1, T, T>(a0, A.partial, 0);
  T t0[1];
  if (!grid_barrier_total<1, T>(A.ctl, nb, A.partial, 0, t0)) return -1;
  T rz = t0[0];
  const T drop2 = (T)(A.inner_tol * A.inner_tol);
  T beta = 0;
  bool first = true;
  // x += scale e (FP64); r64 = rhs - S x; r = r64 / ||r64||, e = 0, z = M^-1 r.
  // Returns 0 converged, 1 cap, -1 barrier failure, 3 continue (rz_out = r.z).
  auto replace = [&](T& rz_out) -> int {
    for (long long i = tid; i < nrow; i += gsz) A.x[i] += scale * (double)e[i];
    if (!grid_barrier(A.ctl, nb)) return -1;
    gather_all(s64, plain<double>(A.x), pl);
    if (!grid_barrier(A.ctl, nb)) return -1;
    apply_all(s64, plain<double>(A.x), A.q64, pl, (double*)nullptr);
    if (!grid_barrier(A.ctl, nb)) return -1;
    double r2[1] = {0.0};
    for (long long i = tid; i < nrow; i += gsz) {
      const double ri = A.rhs[i] - A.q64[i];
      A.r64[i] = ri;
      r2[0] += ri * ri;
    }
    block_partials<1>(r2, A.partial, 7);
    if (!grid_barrier(A.ctl, nb)) return -1;
    const double rn = sqrt(grid_total(A.partial, 7));
    ++repl;
    rel = rn / bnorm;
    if (rel <= A.tol) return 0;
    if (iters >= A.maxit || repl >= A.max_outer) return 1;
    T a4[1] = {};
    for (long long i = tid; i < nrow; i += gsz) {
      const T ri = (T)(A.r64[i] / rn);
      r[i] = ri;
      e[i] = 0;
      const T zi = dinv[i] * ri;
      z[i] = zi;
      a4[0] += ri * zi;
    }
    block_partials<1, T, T>(a4, A.partial, 5);
    T t4[1];
    if (!grid_barrier_total<1, T>(A.ctl, nb, A.partial, 5, t4)) return -1;
    rz_out = t4[0];
    beta = (T)((double)t4[0] / (double)rz * (rn / scale));  // the kept direction in the new units
    scale = rn;
    return 3;
  };
  for (;;) {
    if (iters >= A.maxit) return 1;
    bool broke = !(rz > T(0));
    T al = 0;
    if (!broke) {
      const Operand<T> dir{z, first ? nullptr : pold, beta};
      // q = S p_k (p_k formed on the fly, stored by the contact pass)
      gather_all(s, dir, pl);
      if (!grid_barrier(A.ctl, nb)) return -1;
      T a2[1] = {apply_all(s, dir, q, pl, pnew)};
      block_partials<1, T, T>(a2, A.partial, 2);
      T t2[1];
      __shared__ T s_alpha_r;
      if (!grid_barrier_total<1, T>(A.ctl, nb, A.partial, 2, t2,
                                    [&](const T* t) { s_alpha_r = t[0] > T(0) ? rz / t[0] : T(0); }))
        return -1;
      broke = !(t2[0] > T(0));
      al = s_alpha_r;
    }
    if (broke) {
      // breakdown at the FP32 rounding level: restart the direction from the
      // true residual (a breakdown before any progress is reported)
      if (iters == 0) return 2;
      T rzr;
      const int st = replace(rzr);
      if (st != 3) return st;
      rz = rzr;
      beta = 0;
      first = true;
      continue;
    }
    // e += alpha p, r -= alpha q, z = M^-1 r: four rows per thread (float4),
    // each block on an equal share, all loads of a pass before any store
    T a3[2] = {};
    {
      const long long n4 = nrow >> 2;
      const float4* P4 = reinterpret_cast<const float4*>(pnew);
      const float4* Q4 = reinterpret_cast<const float4*>(q);
      const float4* D4 = reinterpret_cast<const float4*>(dinv);
      float4* E4 = reinterpret_cast<float4*>(e);
      float4* R4 = reinterpret_cast<float4*>(r);
      float4* Z4 = reinterpret_cast<float4*>(z);
      const long long u0 = n4 * blockIdx.x / gridDim.x, u1 = n4 * (blockIdx.x + 1) / gridDim.x;
      const long long bs = blockDim.x;
      for (long long i0 = u0 + threadIdx.x; i0 < u1; i0 += 2 * bs) {
        float4 pv[2], qv[2], dv[2], ev[2], rv[2];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const long long i = i0 + j * bs;
          if (i < u1) {
            pv[j] = P4[i];
            qv[j] = Q4[i];
            dv[j] = D4[i];
            ev[j] = E4[i];
            rv[j] = R4[i];
          }
        }
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const long long i = i0 + j * bs;
          if (i >= u1) break;
          float4 e4 = ev[j], r4 = rv[j];
          e4.x += al * pv[j].x; e4.y += al * pv[j].y; e4.z += al * pv[j].z; e4.w += al * pv[j].w;
          r4.x -= al * qv[j].x; r4.y -= al * qv[j].y; r4.z -= al * qv[j].z; r4.w -= al * qv[j].w;
          const float4 z4 = make_float4(dv[j].x * r4.x, dv[j].y * r4.y, dv[j].z * r4.z, dv[j].w * r4.w);
          E4[i] = e4;
          R4[i] = r4;
          Z4[i] = z4;
          a3[0] += r4.x * r4.x + r4.y * r4.y + r4.z * r4.z + r4.w * r4.w;
          a3[1] += r4.x * z4.x + r4.y * z4.y + r4.z * z4.z + r4.w * z4.w;
        }
      }
      for (long long i = (n4 << 2) + tid; i < nrow; i += gsz) {
        e[i] += al * pnew[i];
        const T ri = r[i] - al * q[i];
        r[i] = ri;
        const T zi = dinv[i] * ri;
        z[i] = zi;
        a3[0] += ri * ri;
        a3[1] += ri * zi;
      }
    }
    block_partials<2, T, T>(a3, A.partial, 3);
    T t3[2];
    if (!grid_barrier_total<2, T>(A.ctl, nb, A.partial, 3, t3)) return -1;
    ++iters;
    first = false;
    const T rr = t3[0];
    T rz_new = t3[1];
    const bool reached = (double)rr * scale * scale <= target * target;
    if (rr <= drop2 || reached || iters >= A.maxit) {
      const int st = replace(rz_new);
      if (st != 3) return st;
    } else {
      beta = rz_new / rz;
    }
    rz = rz_new;
    T* t = pold;
    pold = pnew;
    pnew = t;
  }
}

// y = S x for the operator of precision T (two grid-synchronised phases).
template <class T>
__device__ bool op_apply(const PcgArgs& A, const SysView<T>& s, const T* x, T* y) {
  const long long gsz = (long long)gridDim.x * blockDim.x;
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  for (int bd = (int)tid; bd < s.M; bd += (int)gsz) body_gather(s, plain(x), bd);
  if (!grid_barrier(A.ctl, gridDim.x)) return false;
  for (int c = (int)tid; c < s.Nc; c += (int)gsz) contact_apply(s, plain(x), y, c);
  return grid_barrier(A.ctl, gridDim.x);
}

// out = M^-1 in: Jacobi or the QTT approximate inverse.
template <class T, class TC>
__device__ bool prec_apply(const PcgArgs& A, const T* in, T* out) {
  if ((kQtt<TC> && A.use_qtt)) return qtt_precond_if<T, TC>(A, in, out);
  const long long gsz = (long long)gridDim.x * blockDim.x;
  const T* dinv = static_cast<const T*>(A.dinv);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < A.nrow; i += gsz) out[i] = dinv[i] * in[i];
  return grid_barrier(A.ctl, gridDim.x);
}

// Right-preconditioned BiCGSTAB (van der Vorst, SIAM J. Sci. Stat. Comput. 13
// (1992)) on S_T e = b, e0 = 0: the Krylov method of the paper's Sec. 4.2.
// Returns 0 converged, 1 cap, 2 breakdown, -1 barrier failure.
template <class T, class TC>
__device__ int inner_bicgstab(const PcgArgs& A, double tol, int maxit, int& iters) {
  const SysView<T>& s = sys_of<T>(A);
  const long long P = A.P;
  T* b = static_cast<T*>(A.b);
  T* x = static_cast<T*>(A.e);
  T* r = static_cast<T*>(A.r);
  T* p = static_cast<T*>(A.p);
  T* z = static_cast<T*>(A.z);
  T* xb = static_cast<T*>(A.xb);
  T* rh = xb;
  T* v = xb + P;
  T* y = xb + 2 * P;
  T* sv = xb + 3 * P;
  T* t = xb + 4 * P;
  const long long gsz = (long long)gridDim.x * blockDim.x;
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int nrow = A.nrow;
  const unsigned nb = gridDim.x;
  T a0[1] = {};
  for (long long i = tid; i < P; i += gsz) {
    if (i < nrow) {
      const T bi = b[i];
      x[i] = 0;
      r[i] = bi;
      rh[i] = bi;
      v[i] = 0;
      a0[0] += bi * bi;
    }
    p[i] = 0;   // the QTT preconditioner reads whole padded vectors
    sv[i] = 0;
  }
  block_partials<1>(a0, A.partial, 8);
  if (!grid_barrier(A.ctl, nb)) return -1;
  const double bb = grid_total(A.partial, 8);
  if (bb == 0.0) return 0;
  const double stop = tol * tol * bb;
  double rho = 1.0, alpha = 1.0, omega = 1.0, rho1 = bb;
  for (int it = 0; it < maxit; ++it) {
    if (rho1 == 0.0 || omega == 0.0) return 2;
    const double beta = (rho1 / rho) * (alpha / omega);
    rho = rho1;
    for (long long i = tid; i < nrow; i += gsz) p[i] = r[i] + (T)beta * (p[i] - (T)omega * v[i]);
    if (!grid_barrier(A.ctl, nb)) return -1;
    if (!prec_apply<T, TC>(A, p, y)) return -1;
    if (!op_apply<T>(A, s, y, v)) return -1;
    T a1[1] = {};
    for (long long i = tid; i < nrow; i += gsz) a1[0] += rh[i] * v[i];
    block_partials<1>(a1, A.partial, 9);
    if (!grid_barrier(A.ctl, nb)) return -1;
    const double rv = grid_total(A.partial, 9);
    if (rv == 0.0) return 2;
    alpha = rho / rv;
    T a2[1] = {};
    for (long long i = tid; i < nrow; i += gsz) {
      x[i] += (T)alpha * y[i];
      const T si = r[i] - (T)alpha * v[i];
      sv[i] = si;
      a2[0] += si * si;
    }
    block_partials<1>(a2, A.partial, 10);
    if (!grid_barrier(A.ctl, nb)) return -1;
    if (grid_total(A.partial, 10) <= stop) {
      ++iters;
      return 0;
    }
    if (!prec_apply<T, TC>(A, sv, z)) return -1;
    if (!op_apply<T>(A, s, z, t)) return -1;
    T a3[2] = {};
    for (long long i = tid; i < nrow; i += gsz) {
      a3[0] += t[i] * sv[i];
      a3[1] += t[i] * t[i];
    }
    block_partials<2>(a3, A.partial, 11);
    if (!grid_barrier(A.ctl, nb)) return -1;
    const double ts = grid_total(A.partial, 11), tt = grid_total(A.partial, 12);
    if (!(tt > 0.0)) return 2;
    omega = ts / tt;
    T a4[2] = {};
    for (long long i = tid; i < nrow; i += gsz) {
      x[i] += (T)omega * z[i];
      const T ri = sv[i] - (T)omega * t[i];
      r[i] = ri;
      a4[0] += rh[i] * ri;
      a4[1] += ri * ri;
    }
    block_partials<2>(a4, A.partial, 13);
    if (!grid_barrier(A.ctl, nb)) return -1;
    ++iters;
    rho1 = grid_total(A.partial, 13);
    if (grid_total(A.partial, 14) <= stop) return 0;
  }
  return 1;
}

// FP64 outer refinement: r64 = rhs - S x; inner solve on r64/||r64||; x += ...
template <class T, class TC>
__global__ void __launch_bounds__(NT, 1) k_pcg(PcgArgs A) {
  __shared__ GatherPlan pl;
  extern __shared__ float4 rec_cache[];
  barrier_init();
  plan_fill(A.s64, pl);
  if constexpr (sizeof(T) == 4) {
    if (A.rec_cache > 0) plan_fill_cache(A.s32, pl, rec_cache, A.rec_cache);
  }
  const long long gsz = (long long)gridDim.x * blockDim.x;
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const unsigned nb = gridDim.x;
  const SysView<double>& s64 = A.s64;
  T* b = static_cast<T*>(A.b);
  const T* e = static_cast<const T*>(A.e);
  double a0[1] = {0.0};
  for (long long i = tid; i < A.P; i += gsz) {
    A.x[i] = 0.0;
    if (i < A.nrow) a0[0] += A.rhs[i] * A.rhs[i];
  }
  // the QTT preconditioner reads the whole padded vector: keep its tail zero
  for (long long i = A.nrow + tid; i < A.P; i += gsz) {
    static_cast<T*>(A.r)[i] = 0;
    static_cast<T*>(A.z)[i] = 0;
    b[i] = 0;
  }
  block_partials<1>(a0, A.partial, 6);
  if (!grid_barrier(A.ctl, nb)) return;
  const double bnorm = sqrt(grid_total(A.partial, 6));
  int iters = 0, status = 0, outer = 0;
  double rel = 0.0;
  bool reliable = false;
  if constexpr (sizeof(T) == 4 && !kQtt<TC>) reliable = A.reliable != 0;
  if (bnorm == 0.0) {
    status = 0;
  } else if (reliable) {
    if constexpr (sizeof(T) == 4 && !kQtt<TC>) {
      const int st = pcg_reliable(A, pl, bnorm, iters, outer, rel);
      if (st < 0) return;
      status = st == 0 ? 0 : (st == 2 && iters == 0 ? 2 : 1);
    }
  } else {
    for (outer = 0;; ++outer) {
      // r64 = rhs - S x
      double rr[1] = {0.0};
      if (outer == 0) {
        for (long long i = tid; i < A.nrow; i += gsz) {
          A.r64[i] = A.rhs[i];
          rr[0] += A.rhs[i] * A.rhs[i];
        }
      } else {
        gather_all(s64, plain<double>(A.x), pl);
        if (!grid_barrier(A.ctl, nb)) return;
        apply_all(s64, plain<double>(A.x), A.q64, pl, (double*)nullptr);
        if (!grid_barrier(A.ctl, nb)) return;
        for (long long i = tid; i < A.nrow; i += gsz) {
          double ri = A.rhs[i] - A.q64[i];
          A.r64[i] = ri;
          rr[0] += ri * ri;
        }
      }
      block_partials<1>(rr, A.partial, 7);
      if (!grid_barrier(A.ctl, nb)) return;
      const double rn = sqrt(grid_total(A.partial, 7));
      rel = rn / bnorm;
      if (rel <= A.tol) {
        status = 0;
        break;
      }
      if (outer >= A.max_outer || iters >= A.maxit) {
        status = 1;
        break;
      }
      const double inv = 1.0 / rn;
      for (long long i = tid; i < A.nrow; i += gsz) b[i] = (T)(A.r64[i] * inv);
      if (!grid_barrier(A.ctl, nb)) return;
      int st;
      if (A.direct) {
        // refinement with the approximate inverse: e = X b
        if (!qtt_precond_if<T, TC>(A, b, static_cast<T*>(A.e))) return;
        ++iters;
        st = 0;
      } else if (A.krylov == QP_BICGSTAB) st = inner_bicgstab<T, TC>(A, A.inner_tol, A.maxit - iters, iters);
      else st = inner_pcg<T, TC>(A, pl, A.inner_tol, A.maxit - iters, iters);
      if (st < 0) return;
      for (long long i = tid; i < A.nrow; i += gsz) A.x[i] += rn * (double)e[i];
      if (!grid_barrier(A.ctl, nb)) return;
      if (st == 2 && iters == 0) {
        status = 2;
        break;
      }
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    A.ctl->iters = iters;
    A.ctl->outer = outer;
    A.ctl->scal[S_RELRES] = rel;
    A.ctl->scal[S_BNORM] = bnorm;
    A.ctl->halvings = status;
  }
}

// ------------------------------------------------------------------ batched scenes
// Many independent Newton solves in one launch.  The launch is made of clusters
// of two thread blocks, each cluster running one job: either one large scene
// split over both blocks (rows, contacts and bodies interleaved in slices of
// one block's width; hardware cluster barriers between phases; sums reduced
// through distributed shared memory) or up to two small scenes, one per block,
// with block-level synchronisation only.  Each scene's job builds the Schur
// blocks and the Jacobi diagonal and runs the FP32 inner PCG inside the FP64
// refinement.  Jobs start in decreasing cost, so the longest start first.
struct BatchScene {
  SysView<double> s64;   // H = the scene's FP64 block buffer (written here)
  SysView<float> s32;
  double* H64;
  float* H32;
  double* dinv64;
  float* dinv32;
  const double* gamma;   // null: S = N
  const double* lambda;
  double mu;
  const double* rhs;
  double* dx;
  double* r64;           // [P] FP64 residual
  double* q64;           // [P]
  float* v32;            // 7 [P] FP32 vectors: b, e, r, z, p, p', q
  long long P;
  int nrow;
  const QttDev* qtt;     // the scene's QTT preconditioner (device copy), or null: Jacobi
  float* qw;             // QTT work: two [P * rmax] FP32 buffers
  int qtt_scaled;        // X approximates the inverse of D^-1/2 S D^-1/2
  int qtt_bf16;          // cores in BF16 (else FP32)
};

struct BatchOut {
  int iters, outer, status, fallback;  // fallback: the QTT preconditioner broke down, Jacobi finished
  double rel;
};

// The threads working on one scene: one block, or both blocks of the cluster.
// T is the thread's index among them and NT their number; ph counts the sums,
// so that consecutive sums use alternate result slots.
struct Grp {
  int T, NT;
  bool split;
  unsigned ph;
};

__device__ __forceinline__ void grp_sync(const Grp& g) {
  if (g.split) cg::this_cluster().sync();
  else __syncthreads();
}

// Sum over the group, identical in every thread: per-warp sums, then warp 0 of
// each block; with two blocks both read the two block totals (rank 0 first)
// from distributed shared memory after one cluster barrier.  The per-warp
// partials are reused only after this call's barrier; the block totals
// alternate between two slots, so a sum never overwrites a total that the other
// block may still be reading.
template <int NTB, class V, int K>
__device__ __forceinline__ void group_sum(V (&v)[K], Grp& g) {
  __shared__ V sm[K][NTB / 32];
  __shared__ V tot[2][K];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int slot = g.ph & 1;
  ++g.ph;
  for (int k = 0; k < K; ++k) {
    const V x = warp_sum(v[k]);
    if (lane == 0) sm[k][wid] = x;
  }
  __syncthreads();
  if (wid == 0) {
    for (int k = 0; k < K; ++k) {
      V x = lane < NTB / 32 ? sm[k][lane] : V(0);
      x = warp_sum(x);
      if (lane == 0) tot[slot][k] = x;
    }
  }
  if (g.split) {
    cg::cluster_group cl = cg::this_cluster();
    cl.sync();
    const V* t0 = cl.map_shared_rank(&tot[slot][0], 0);
    const V* t1 = cl.map_shared_rank(&tot[slot][0], 1);
    for (int k = 0; k < K; ++k) v[k] = t0[k] + t1[k];
  } else {
    __syncthreads();
    for (int k = 0; k < K; ++k) v[k] = tot[slot][k];
  }
}

// FP32 inner PCG of one scene on S e = b.  Returns 0 converged, 1 cap,
// 2 breakdown; every thread of the group takes the same branch (the sums are
// identical).
template <int NTB>
__device__ int block_inner_pcg(const BatchScene& S, float tol, int maxit, int& iters, Grp& g) {
  const SysView<float>& s = S.s32;
  const int nrow = S.nrow, t = g.T, NT = g.NT;
  const long long P = S.P;
  float* b = S.v32;
  float* e = b + P;
  float* r = e + P;
  float* z = r + P;
  float* pa = z + P;
  float* pb = pa + P;
  float* q = pb + P;
  const float* dinv = S.dinv32;
  float a0[2] = {0.f, 0.f};
  for (int i = t; i < nrow; i += NT) {
    const float bi = b[i];
    e[i] = 0.f;
    r[i] = bi;
    const float zi = dinv[i] * bi;
    z[i] = zi;
    a0[0] += bi * bi;
    a0[1] += bi * zi;
  }
  group_sum<NTB>(a0, g);
  const float bb = a0[0];
  float rz = a0[1];
  if (bb == 0.f) return 0;
  const float stop = tol * tol * bb;
  float* pold = pa;
  float* pnew = pb;
  float beta = 0.f;
  for (int it = 0; it < maxit; ++it) {
    if (!(rz > 0.f)) return 2;
    const Operand<float> dir{z, it == 0 ? nullptr : pold, beta};
    for (int bd = t; bd < s.M; bd += NT) body_gather(s, dir, bd);
    grp_sync(g);
    float a1[1] = {0.f};
    for (int c = t; c < s.Nc; c += NT) a1[0] += contact_apply(s, dir, q, c, pnew);
    group_sum<NTB>(a1, g);
    const float pq = a1[0];
    if (!(pq > 0.f)) return 2;
    const float alpha = rz / pq;
    float a2[2] = {0.f, 0.f};
    // four rows per thread and pass, every load of the pass before any store
    for (int i0 = t; i0 < nrow; i0 += 4 * NT) {
      float pv[4], ev[4], rv[4], qv[4], dv[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int i = i0 + j * NT;
        const bool in = i < nrow;
        pv[j] = in ? pnew[i] : 0.f;
        ev[j] = in ? e[i] : 0.f;
        rv[j] = in ? r[i] : 0.f;
        qv[j] = in ? q[i] : 0.f;
        dv[j] = in ? dinv[i] : 0.f;
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int i = i0 + j * NT;
        if (i >= nrow) break;
        e[i] = ev[j] + alpha * pv[j];
        const float ri = rv[j] - alpha * qv[j];
        r[i] = ri;
        const float zi = dv[j] * ri;
        z[i] = zi;
        a2[0] += ri * ri;
        a2[1] += ri * zi;
      }
    }
    group_sum<NTB>(a2, g);
    ++iters;
    if (a2[0] <= stop) return 0;
    beta = a2[1] / rz;
    rz = a2[1];
    float* tmp = pold;
    pold = pnew;
    pnew = tmp;
  }
  return 1;
}

// z = X r through a QTT preconditioner by the threads of one group (one core
// per pass, group-synchronised), z = D^-1/2 X D^-1/2 r when X approximates the
// inverse of the Jacobi-scaled matrix (Sec. 3.2 mat-vec, as qtt_precond does it
// for the whole grid).  Tile shape per core, by the class of its input rank
// r_k (<= 4, <= 8, <= 16): bit c of tilemask set = two column items per thread
// sharing the core staged in shared memory (r_{k-1} r_k <= 256); clear, or a
// rank above 16 = one item per thread, its inputs in registers.  Rows of r
// from nrow on must be zero.
template <int NTB, class TC>
__device__ void group_qtt_apply(const QttDev& q, int scaled, const float* dinv, int nrow, long long P, float* qw,
                                const float* r, float* z, Grp& g, unsigned tilemask) {
  __shared__ float gc[4 * 16 * 16];
  const int t = g.T, NT = g.NT;
  const long long items = P >> 1;
  float* w0 = qw;
  float* w1 = qw + (size_t)P * q.rmax;
  const float* in = r;
  if (scaled) {
    for (long long i = t; i < P; i += NT) w1[i] = i < nrow ? sqrtf(dinv[i]) * r[i] : 0.f;
    grp_sync(g);
    in = w1;  // read by the first pass only, which writes w0
  }
  int pass = 0;
  for (int k = q.d; k >= 1; --k, ++pass) {
    float* out = k == 1 ? z : ((pass & 1) ? w1 : w0);
    const int r0 = q.ranks[k - 1], r1 = q.ranks[k];
    const int cls = r1 <= 4 ? 0 : (r1 <= 8 ? 1 : (r1 <= 16 ? 2 : 3));
    if (cls < 3 && ((tilemask >> cls) & 1u) && r0 * r1 <= 256) {
      if (cls == 0) qtt_step_block<4, float, float, TC>(q, k, in, out, items, gc, t, NT);
      else if (cls == 1) qtt_step_block<8, float, float, TC>(q, k, in, out, items, gc, t, NT);
      else qtt_step_block<16, float, float, TC>(q, k, in, out, items, gc, t, NT);
    } else {
      for (long long it = t; it < items; it += NT) qtt_step_any<float, float, TC>(q, k, in, out, it);
    }
    grp_sync(g);
    in = out;
  }
  if (scaled) {
    for (long long i = t; i < nrow; i += NT) z[i] *= sqrtf(dinv[i]);
    grp_sync(g);
  }
}

// The FP32 inner PCG of block_inner_pcg with the scene's QTT preconditioner:
// after each update of r the whole group applies z = M^-1 r, then r.z is summed.
template <int NTB, class TC>
__device__ int block_inner_pcg_qtt(const BatchScene& S, float tol, int maxit, int& iters, Grp& g, unsigned tilemask) {
  const SysView<float>& s = S.s32;
  const int nrow = S.nrow, t = g.T, NT = g.NT;
  const long long P = S.P;
  float* b = S.v32;
  float* e = b + P;
  float* r = e + P;
  float* z = r + P;
  float* pa = z + P;
  float* pb = pa + P;
  float* q = pb + P;
  float a0[1] = {0.f};
  for (long long i = t; i < P; i += NT) {
    const float bi = i < nrow ? b[i] : 0.f;
    e[i] = 0.f;
    r[i] = bi;
    a0[0] += bi * bi;
  }
  group_sum<NTB>(a0, g);
  const float bb = a0[0];
  if (bb == 0.f) return 0;
  const float stop = tol * tol * bb;
  group_qtt_apply<NTB, TC>(*S.qtt, S.qtt_scaled, S.dinv32, nrow, P, S.qw, r, z, g, tilemask);
  float a1[1] = {0.f};
  for (int i = t; i < nrow; i += NT) a1[0] += r[i] * z[i];
  group_sum<NTB>(a1, g);
  float rz = a1[0];
  float* pold = pa;
  float* pnew = pb;
  float beta = 0.f;
  for (int it = 0; it < maxit; ++it) {
    if (!(rz > 0.f)) return 2;
    const Operand<float> dir{z, it == 0 ? nullptr : pold, beta};
    for (int bd = t; bd < s.M; bd += NT) body_gather(s, dir, bd);
    grp_sync(g);
    float a2[1] = {0.f};
    for (int c = t; c < s.Nc; c += NT) a2[0] += contact_apply(s, dir, q, c, pnew);
    group_sum<NTB>(a2, g);
    const float pq = a2[0];
    if (!(pq > 0.f)) return 2;
    const float alpha = rz / pq;
    float a3[1] = {0.f};
    for (int i = t; i < nrow; i += NT) {
      e[i] += alpha * pnew[i];
      const float ri = r[i] - alpha * q[i];
      r[i] = ri;
      a3[0] += ri * ri;
    }
    group_sum<NTB>(a3, g);
    ++iters;
    if (a3[0] <= stop) return 0;
    group_qtt_apply<NTB, TC>(*S.qtt, S.qtt_scaled, S.dinv32, nrow, P, S.qw, r, z, g, tilemask);
    float a4[1] = {0.f};
    for (int i = t; i < nrow; i += NT) a4[0] += r[i] * z[i];
    group_sum<NTB>(a4, g);
    beta = a4[0] / rz;
    rz = a4[0];
    float* tmp = pold;
    pold = pnew;
    pnew = tmp;
  }
  return 1;
}

// Tile-shape probe of the autotuner: one block applies a QTT `reps` times with
// the given tile mask (the batched kernel runs one scene per block).
template <int NTB>
__global__ void __launch_bounds__(NTB) k_qtt_tile_probe(QttDev q, const float* x, float* y, float* qw, unsigned tilemask,
                                                        int reps) {
  Grp g;
  g.T = threadIdx.x;
  g.NT = NTB;
  g.split = false;
  g.ph = 0;
  const long long P = 1LL << q.d;
  for (int i = 0; i < reps; ++i) group_qtt_apply<NTB, float>(q, 0, nullptr, (int)P, P, qw, x, y, g, tilemask);
}

// One job per cluster: jobs[j] = (scene, -2) runs that scene on both blocks;
// (a, b) runs scene a on block rank 0 and scene b (b >= 0) on rank 1.
// QTT = true adds the per-scene QTT preconditioner (scenes with S.qtt set; the
// others keep Jacobi); QTT = false is the Jacobi-only kernel.
template <int NTB, bool QTT>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(NTB)
    k_pcg_batched(const BatchScene* __restrict__ tab, const int2* __restrict__ jobs, double tol, double inner_tol,
                  int maxit, int max_outer, BatchOut* __restrict__ out, unsigned tilemask) {
  const int rank = (int)cg::this_cluster().block_rank();
  const int2 job = jobs[blockIdx.x >> 1];
  Grp g;
  g.split = job.y == -2;
  g.ph = 0;
  const int sid = g.split ? job.x : (rank == 0 ? job.x : job.y);
  if (sid < 0) return;  // the second block of a job with one small scene
  g.T = g.split ? rank * NTB + (int)threadIdx.x : (int)threadIdx.x;
  g.NT = g.split ? 2 * NTB : NTB;
  const BatchScene S = tab[sid];
  const int t = g.T, NT = g.NT;
  const int n = S.s64.Nc;
  // Schur blocks (zero without a state) and the Jacobi diagonal
  for (int c = t; c < n; c += NT) {
    double h[6] = {0, 0, 0, 0, 0, 0};
    if (S.gamma) {
      const long long row = (long long)S.s64.slots * c;
      schur_block(S.mu, S.gamma[row], S.gamma[row + 1], S.gamma[row + 2], S.lambda[c], S.lambda[n + c], h);
    }
    for (int k = 0; k < 6; ++k) {
      S.H64[(size_t)k * n + c] = h[k];
      S.H32[(size_t)k * n + c] = (float)h[k];
    }
  }
  grp_sync(g);
  for (long long i = t; i < S.P; i += NT) {
    const long long c = i / S.s64.slots;
    const int u = (int)(i - c * S.s64.slots);
    double v = 1.0;
    if (c < n && u < 3) v = diag_entry(S.s64, (int)c, u) + S.H64[(u == 0 ? 0 : (u == 1 ? 3 : 5)) * (long long)n + c];
    S.dinv64[i] = 1.0 / v;
    S.dinv32[i] = (float)(1.0 / v);
    S.dx[i] = 0.0;
  }
  double bn[1] = {0.0};
  for (int i = t; i < S.nrow; i += NT) bn[0] += S.rhs[i] * S.rhs[i];
  group_sum<NTB>(bn, g);
  const double bnorm = sqrt(bn[0]);
  int iters = 0, outer = 0, status = 0, fell_back = 0;
  double rel = 0.0;
  if (bnorm > 0.0) {
    for (outer = 0;; ++outer) {
      double rr[1] = {0.0};
      if (outer == 0) {
        for (int i = t; i < S.nrow; i += NT) {
          S.r64[i] = S.rhs[i];
          rr[0] += S.rhs[i] * S.rhs[i];
        }
      } else {
        for (int bd = t; bd < S.s64.M; bd += NT) body_gather(S.s64, plain<double>(S.dx), bd);
        grp_sync(g);
        for (int c = t; c < n; c += NT) contact_apply(S.s64, plain<double>(S.dx), S.q64, c);
        grp_sync(g);
        for (int i = t; i < S.nrow; i += NT) {
          const double ri = S.rhs[i] - S.q64[i];
          S.r64[i] = ri;
          rr[0] += ri * ri;
        }
      }
      group_sum<NTB>(rr, g);
      const double rn = sqrt(rr[0]);
      rel = rn / bnorm;
      if (rel <= tol) break;
      if (outer >= max_outer || iters >= maxit) {
        status = 1;
        break;
      }
      const double inv = 1.0 / rn;
      for (int i = t; i < S.nrow; i += NT) S.v32[i] = (float)(S.r64[i] * inv);
      grp_sync(g);
      const int before = iters;
      int st;
      if constexpr (QTT) {
        if (S.qtt && !fell_back) {
          st = S.qtt_bf16 ? block_inner_pcg_qtt<NTB, __nv_bfloat16>(S, (float)inner_tol, maxit - iters, iters, g, tilemask)
                          : block_inner_pcg_qtt<NTB, float>(S, (float)inner_tol, maxit - iters, iters, g, tilemask);
          // a truncated QTT inverse need not be definite: on a breakdown the
          // scene continues with the Jacobi preconditioner (as newton_solve does)
          if (st == 2) {
            fell_back = 1;
            st = block_inner_pcg<NTB>(S, (float)inner_tol, maxit - iters, iters, g);
          }
        } else {
          st = block_inner_pcg<NTB>(S, (float)inner_tol, maxit - iters, iters, g);
        }
      } else {
        st = block_inner_pcg<NTB>(S, (float)inner_tol, maxit - iters, iters, g);
      }
      const float* e = S.v32 + S.P;
      for (int i = t; i < S.nrow; i += NT) S.dx[i] += rn * (double)e[i];
      grp_sync(g);
      if (st == 2 && iters == before) {
        status = 2;
        break;
      }
    }
  }
  if (t == 0) {
    out[sid].iters = iters;
    out[sid].outer = outer;
    out[sid].status = status;
    out[sid].fallback = fell_back;
    out[sid].rel = rel;
  }
  // a block's shared memory must outlive the other block's last read of it
  if (g.split) cg::this_cluster().sync();
}

// ------------------------------------------------------------------ fused pipelined PCG
// Contact partition: block g owns contacts [g*chunk, (g+1)*chunk) (Morton order,
// so a chunk is spatially compact) and gathers every body its contacts touch
// into shared memory; bodies on chunk borders are gathered by each block that
// needs them.  A matrix-vector product then needs no grid barrier.
struct Part {
  int chunk;
  int maxb;
  const int* nb;      // [G] bodies per block
  const int* bodies;  // [G][maxb] global body ids
  const int* cl;      // [2 Nc] local index of body a, body b (-1: static floor)
};

__global__ void k_partition(int Nc, int M, int chunk, int maxb, const int* __restrict__ ca,
                            const int* __restrict__ cb, int* __restrict__ nb, int* __restrict__ bodies,
                            int* __restrict__ cl) {
  extern __shared__ int sb[];
  const int g = blockIdx.x;
  const int c0 = g * chunk, c1 = min(Nc, c0 + chunk);
  const int nref = 2 * max(0, c1 - c0);
  int n2 = 1;
  while (n2 < nref) n2 <<= 1;
  for (int i = threadIdx.x; i < n2; i += blockDim.x) {
    int v = 0x7fffffff;
    if (i < nref) {
      const int c = c0 + (i >> 1);
      const int body = (i & 1) ? cb[c] : ca[c];
      if (body < M) v = body;
    }
    sb[i] = v;
  }
  __syncthreads();
  // bitonic sort
  for (int k = 2; k <= n2; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < n2; i += blockDim.x) {
        const int l = i ^ j;
        if (l > i) {
          const bool up = (i & k) == 0;
          const int a = sb[i], b = sb[l];
          if ((a > b) == up) {
            sb[i] = b;
            sb[l] = a;
          }
        }
      }
      __syncthreads();
    }
  // unique (serial compaction by thread 0: at most a few thousand entries)
  __shared__ int cnt;
  if (threadIdx.x == 0) {
    int k = 0;
    for (int i = 0; i < n2; ++i) {
      const int v = sb[i];
      if (v == 0x7fffffff) break;
      if (k == 0 || sb[k - 1] != v) sb[k++] = v;
    }
    cnt = k;
    nb[g] = k;
  }
  __syncthreads();
  const int nbk = cnt;
  for (int i = threadIdx.x; i < nbk; i += blockDim.x) bodies[(long long)g * maxb + i] = sb[i];
  for (int c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
    for (int side = 0; side < 2; ++side) {
      const int body = side ? cb[c] : ca[c];
      int idx = -1;
      if (body < M) {
        int lo = 0, hi = nbk - 1;
        while (lo <= hi) {
          const int mid = (lo + hi) >> 1;
          const int v = sb[mid];
          if (v == body) {
            idx = mid;
            break;
          }
          if (v < body) lo = mid + 1;
          else hi = mid - 1;
        }
      }
      cl[2 * c + side] = idx;
    }
  }
}

// Per-row records of the pipelined solver (8 values of type T each):
//   pipe  record: w[2], n[2], z[2] (ping-pong pairs), M^-1 (Jacobi), 0
//   state record: e, r, u, p, q, s, b, 0
// One or two vector loads fetch everything a row needs.
template <class T>
__device__ __forceinline__ void load8(const T* p, T (&v)[8]) {
  if constexpr (sizeof(T) == 4) {
    const float4* q = reinterpret_cast<const float4*>(p);
    float4 a = q[0], b = q[1];
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
  } else {
    const double2* q = reinterpret_cast<const double2*>(p);
    double2 a = q[0], b = q[1], c = q[2], d = q[3];
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y; v[4] = c.x; v[5] = c.y; v[6] = d.x; v[7] = d.y;
  }
}
template <class T>
__device__ __forceinline__ void store8(T* p, const T (&v)[8]) {
  if constexpr (sizeof(T) == 4) {
    float4* q = reinterpret_cast<float4*>(p);
    q[0] = make_float4(v[0], v[1], v[2], v[3]);
    q[1] = make_float4(v[4], v[5], v[6], v[7]);
  } else {
    double2* q = reinterpret_cast<double2*>(p);
    q[0] = make_double2(v[0], v[1]);
    q[1] = make_double2(v[2], v[3]);
    q[2] = make_double2(v[4], v[5]);
    q[3] = make_double2(v[6], v[7]);
  }
}

// operand M^-1 b for the first product (b from the state record)
template <class T>
struct OpRhs {
  const T* pr;
  const T* sr;
  __device__ __forceinline__ T operator()(long long i) const { return pr[i * 8 + 6] * sr[i * 8 + 6]; }
};
// operand M^-1 w (w = w[slot] of the pipe record)
template <class T>
struct OpW {
  const T* pr;
  int slot;
  __device__ __forceinline__ T operator()(long long i) const { return pr[i * 8 + 6] * pr[i * 8 + slot]; }
};
// operand M^-1 w_next, w_next = w[cur] - alpha (n[cur] + beta z[nxt]), all from one record load
template <class T>
struct OpPipe {
  const T* pr;
  int cur;
  T alpha, beta;
  __device__ __forceinline__ T operator()(long long i) const {
    T v[8];
    load8(pr + i * 8, v);
    const T w = cur ? v[1] : v[0];
    const T nn = cur ? v[3] : v[2];
    const T z = cur ? v[4] : v[5];
    return v[6] * (w - alpha * (nn + beta * z));
  }
};

// Plain FP64 operand (outer residual).
template <class T>
struct PlainOp {
  const T* x;
  __device__ __forceinline__ T operator()(long long i) const { return x[i]; }
};

// y = S x for the rows of this block's contacts; x is evaluated through `op`;
// row i of y is stored at y[i * ys].
template <class T, class X>
__device__ void fused_apply(const SysView<T>& s, const Part& pt, const X& op, T* y, int ys, T* wl) {
  const int g = blockIdx.x;
  const int nbk = pt.nb[g];
  for (int lb = threadIdx.x; lb < nbk; lb += blockDim.x) {
    const int b = pt.bodies[(long long)g * pt.maxb + lb];
    T F0 = 0, F1 = 0, F2 = 0, Q0 = 0, Q1 = 0, Q2 = 0;
    const int e = __ldg(s.bptr + b + 1);
#pragma unroll 2
    for (int k = __ldg(s.bptr + b); k < e; ++k) {
      const int code = __ldg(s.inc + k);
      const int c = code >> 1;
      const long long row = (long long)s.slots * c;
      T R[16];
      load_rec(s.rec, c, R);
      const T x0 = op(row), x1 = op(row + 1), x2 = op(row + 2);
      T f0 = R[0] * x0 + R[3] * x1 + R[6] * x2;
      T f1 = R[1] * x0 + R[4] * x1 + R[7] * x2;
      T f2 = R[2] * x0 + R[5] * x1 + R[8] * x2;
      const bool sb = (code & 1) != 0;
      const T a0 = sb ? R[12] : R[9], a1 = sb ? R[13] : R[10], a2 = sb ? R[14] : R[11];
      const T sg = sb ? T(1) : T(-1);
      f0 *= sg;
      f1 *= sg;
      f2 *= sg;
      F0 += f0;
      F1 += f1;
      F2 += f2;
      Q0 += a1 * f2 - a2 * f1;
      Q1 += a2 * f0 - a0 * f2;
      Q2 += a0 * f1 - a1 * f0;
    }
    const T im = __ldg(s.inv_m + b), iI = __ldg(s.inv_I + b);
    T* o = wl + (long long)lb * 8;
    o[0] = im * F0;
    o[1] = im * F1;
    o[2] = im * F2;
    o[3] = iI * Q0;
    o[4] = iI * Q1;
    o[5] = iI * Q2;
  }
  __syncthreads();
  const int c0 = g * pt.chunk, c1 = min(s.Nc, c0 + pt.chunk);
  const long long n = s.Nc;
  for (int c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
    T R[16];
    load_rec(s.rec, c, R);
    const int la = pt.cl[2 * c], lb = pt.cl[2 * c + 1];
    const T* wb = wl + (long long)lb * 8;
    T d0 = wb[0] + (wb[4] * R[14] - wb[5] * R[13]);
    T d1 = wb[1] + (wb[5] * R[12] - wb[3] * R[14]);
    T d2 = wb[2] + (wb[3] * R[13] - wb[4] * R[12]);
    if (la >= 0) {
      const T* wa = wl + (long long)la * 8;
      d0 -= wa[0] + (wa[4] * R[11] - wa[5] * R[10]);
      d1 -= wa[1] + (wa[5] * R[9] - wa[3] * R[11]);
      d2 -= wa[2] + (wa[3] * R[10] - wa[4] * R[9]);
    }
    const long long row = (long long)s.slots * c;
    const T x0 = op(row), x1 = op(row + 1), x2 = op(row + 2);
    T y0 = R[0] * d0 + R[1] * d1 + R[2] * d2;
    T y1 = R[3] * d0 + R[4] * d1 + R[5] * d2;
    T y2 = R[6] * d0 + R[7] * d1 + R[8] * d2;
    if (s.H) {
      const T* H = s.H;
      T h00 = __ldg(H + c), h01 = __ldg(H + n + c), h02 = __ldg(H + 2 * n + c);
      T h11 = __ldg(H + 3 * n + c), h12 = __ldg(H + 4 * n + c), h22 = __ldg(H + 5 * n + c);
      y0 += h00 * x0 + h01 * x1 + h02 * x2;
      y1 += h01 * x0 + h11 * x1 + h12 * x2;
      y2 += h02 * x0 + h12 * x1 + h22 * x2;
    }
    y[row * ys] = y0;
    y[(row + 1) * ys] = y1;
    y[(row + 2) * ys] = y2;
    if (s.slots == 4) y[(row + 3) * ys] = op(row + 3);
  }
  __syncthreads();
}

// y = S x (or N x without a state) in a single launch, the standalone form of
// the fused operator (Eq. Ndef plus the Schur blocks of Sec. 3.3).  Block g
// owns contacts [g chunk, (g+1) chunk) of the Morton order and the bodies they
// touch (the partition of the pipelined solver): phase 1 forms w_b = M^-1 D_b x
// for those bodies in shared memory (all incidences of each body, L lanes per
// body, combined by shuffles; a border body is formed by every block that needs
// it); phase 2 applies each contact's rows, with its 3x3 block H_c formed in
// registers from (gamma_c, lambda_c) and never stored.  In FP32 the cone
// function f_c (a difference of squares near the cone) is taken in FP64, the
// rest of the block in FP32.  Dummy rows copy x.
template <class T>
__device__ __forceinline__ void schur_block_t(double mu, double gn, double g1, double g2, double lc, double ln,
                                              T (&h)[6]) {
  if constexpr (sizeof(T) == 8) {
    schur_block(mu, gn, g1, g2, lc, ln, h);
  } else {
    const double fc = 0.5 * (g1 * g1 + g2 * g2 - mu * mu * gn * gn);
    const float m2 = (float)(mu * mu);
    const float q0 = -m2 * (float)gn, q1 = (float)g1, q2 = (float)g2;
    const float l = (float)lc;
    const float sc = l / (float)(-fc);
    h[0] = -m2 * l + sc * q0 * q0 + (float)ln / (float)gn;
    h[1] = sc * q0 * q1;
    h[2] = sc * q0 * q2;
    h[3] = l + sc * q1 * q1;
    h[4] = sc * q1 * q2;
    h[5] = l + sc * q2 * q2;
  }
}

template <class T, bool WITH_H, int L>
__global__ void __launch_bounds__(256) k_apply_one(SysView<T> s, Part pt, const T* __restrict__ x,
                                                   T* __restrict__ y, const double* __restrict__ gamma,
                                                   const double* __restrict__ lambda, double mu) {
  static_assert(L >= 1 && L <= 32 && (L & (L - 1)) == 0, "lanes: a power of two up to 32");
  extern __shared__ __align__(16) unsigned char apply_smem[];
  T* wl = reinterpret_cast<T*>(apply_smem);
  const int g = blockIdx.x;
  const int nbk = pt.nb[g];
  const int per = blockDim.x / L;
  const int lane = threadIdx.x & (L - 1);
  const int* bl = pt.bodies + (long long)g * pt.maxb;
  // phase 1: the loop bound is uniform over the block, so every lane reaches the shuffles
  for (int b0 = 0; b0 < nbk; b0 += per) {
    const int lb = b0 + (int)threadIdx.x / L;
    T F0 = 0, F1 = 0, F2 = 0, Q0 = 0, Q1 = 0, Q2 = 0;
    int b = 0;
    if (lb < nbk) {
      b = bl[lb];
      const int e = __ldg(s.bptr + b + 1);
      for (int k = __ldg(s.bptr + b) + lane; k < e; k += 2 * L) {
        const int code[2] = {__ldg(s.inc + k), k + L < e ? __ldg(s.inc + k + L) : -1};
        gather_batch<2>(s, plain(x), code, F0, F1, F2, Q0, Q1, Q2);
      }
    }
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1) {
      F0 += __shfl_xor_sync(0xffffffffu, F0, o);
      F1 += __shfl_xor_sync(0xffffffffu, F1, o);
      F2 += __shfl_xor_sync(0xffffffffu, F2, o);
      Q0 += __shfl_xor_sync(0xffffffffu, Q0, o);
      Q1 += __shfl_xor_sync(0xffffffffu, Q1, o);
      Q2 += __shfl_xor_sync(0xffffffffu, Q2, o);
    }
    if (lb < nbk && lane == 0) {
      const T im = __ldg(s.inv_m + b), iI = __ldg(s.inv_I + b);
      T* o = wl + (long long)lb * 8;
      o[0] = im * F0;
      o[1] = im * F1;
      o[2] = im * F2;
      o[3] = iI * Q0;
      o[4] = iI * Q1;
      o[5] = iI * Q2;
    }
  }
  __syncthreads();
  // phase 2: the block's contacts
  const int n = s.Nc;
  const int c0 = g * pt.chunk, c1 = min(n, c0 + pt.chunk);
  for (int c = c0 + (int)threadIdx.x; c < c1; c += blockDim.x) {
    T R[16];
    load_rec(s.rec, c, R);
    const int la = pt.cl[2 * c], lb = pt.cl[2 * c + 1];
    const T* wb = wl + (long long)lb * 8;
    T d0 = wb[0] + (wb[4] * R[14] - wb[5] * R[13]);
    T d1 = wb[1] + (wb[5] * R[12] - wb[3] * R[14]);
    T d2 = wb[2] + (wb[3] * R[13] - wb[4] * R[12]);
    if (la >= 0) {
      const T* wa = wl + (long long)la * 8;
      d0 -= wa[0] + (wa[4] * R[11] - wa[5] * R[10]);
      d1 -= wa[1] + (wa[5] * R[9] - wa[3] * R[11]);
      d2 -= wa[2] + (wa[3] * R[10] - wa[4] * R[9]);
    }
    const long long row = (long long)s.slots * c;
    const T x0 = x[row], x1 = x[row + 1], x2 = x[row + 2];
    T y0 = R[0] * d0 + R[1] * d1 + R[2] * d2;
    T y1 = R[3] * d0 + R[4] * d1 + R[5] * d2;
    T y2 = R[6] * d0 + R[7] * d1 + R[8] * d2;
    if constexpr (WITH_H) {
      T h[6];
      schur_block_t<T>(mu, gamma[row], gamma[row + 1], gamma[row + 2], lambda[c], lambda[n + c], h);
      y0 += h[0] * x0 + h[1] * x1 + h[2] * x2;
      y1 += h[1] * x0 + h[3] * x1 + h[4] * x2;
      y2 += h[2] * x0 + h[4] * x1 + h[5] * x2;
    }
    y[row] = y0;
    y[row + 1] = y1;
    y[row + 2] = y2;
    if (s.slots == 4) y[row + 3] = x[row + 3];
  }
  const long long tail0 = (long long)s.slots * n;
  for (long long i = tail0 + blockIdx.x * (long long)blockDim.x + threadIdx.x; i < s.P;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = x[i];
}

struct FusedArgs {
  SysView<double> s64;
  SysView<float> s32;
  Part pt;
  int nrow;
  long long P;
  const double* rhs;
  double* x;
  double* r64;
  double* q64;
  void* pool;          // 13 vectors of type T, P each
  const void* dinv;
  double tol, inner_tol;
  int maxit, max_outer;
  DevCtl* ctl;
  double* partial;
};

template <class T>
__device__ __forceinline__ const SysView<T>& fsys(const FusedArgs& a);
template <>
__device__ __forceinline__ const SysView<double>& fsys<double>(const FusedArgs& a) { return a.s64; }
template <>
__device__ __forceinline__ const SysView<float>& fsys<float>(const FusedArgs& a) { return a.s32; }


// Pipelined Jacobi-PCG (Ghysels and Vanroose, Parallel Computing 40 (2014),
// Alg. 3) on S_T e = b, x0 = 0, b in the state records.  One grid barrier per
// iteration: it publishes the new n, w, z and completes the reduction of
// (r,u), (w,u), (r,r).  Returns 0 converged, 1 cap, 2 breakdown, -1 barrier failure.
template <class T>
__device__ int inner_pcg_fused(const FusedArgs& A, double tol, int maxit, int& iters, T* wl) {
  const SysView<T>& s = fsys<T>(A);
  T* pool = static_cast<T*>(A.pool);
  T* pr = pool;                  // pipe records   [P][8]
  T* sr = pool + 8 * A.P;        // state records  [P][8]
  const unsigned nb = gridDim.x;
  const int g = blockIdx.x;
  const int c0 = g * A.pt.chunk, c1 = min(s.Nc, c0 + A.pt.chunk);
  const long long r0 = (long long)s.slots * c0, r1 = (long long)s.slots * c1;
  // phase I: e = 0, r = b, u = M^-1 b, p = q = s = 0, z = 0; w0 = S u -> pipe n[1]
  // (stored in the n slot of the other parity, moved to w[0] below)
  T acc[3] = {};
  for (long long i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
    const T bi = sr[i * 8 + 6];
    T pv[8];
    load8(pr + i * 8, pv);
    const T ui = pv[6] * bi;
    const T ns[8] = {T(0), bi, ui, T(0), T(0), T(0), bi, T(0)};
    store8(sr + i * 8, ns);
    pr[i * 8 + 4] = T(0);
    pr[i * 8 + 5] = T(0);
    acc[0] += bi * ui;
    acc[1] += bi * bi;
  }
  // w0 = S M^-1 b into the n[1] slot of each row (no one reads n[1] in this phase)
  fused_apply(s, A.pt, OpRhs<T>{pr, sr}, pr + 3, 8, wl);
  // reductions and scalar recurrences in T (float in the FP32 inner solve)
  block_partials<3, T, T>(acc, A.partial, 0);
  T tot[3];
  if (!grid_barrier_total<3, T>(A.ctl, nb, A.partial, 0, tot)) return -1;
  T gamma = tot[0];
  const T bb = tot[1];
  if (bb == T(0)) return 0;
  // phase 0: w[0] <- n[1] (own rows); n0 = S M^-1 w0 into n[0]; delta0 = (w0, u0)
  T acc1[3] = {};
  for (long long i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
    const T w0 = pr[i * 8 + 3];
    pr[i * 8 + 0] = w0;
    acc1[0] += w0 * sr[i * 8 + 2];
  }
  __syncthreads();
  // other blocks read w0 of our rows through n[1]: use that slot as the operand
  fused_apply(s, A.pt, OpW<T>{pr, 3}, pr + 2, 8, wl);
  block_partials<3, T, T>(acc1, A.partial, 3);
  if (!grid_barrier_total<3, T>(A.ctl, nb, A.partial, 3, tot)) return -1;
  const T delta = tot[0];
  if (!(gamma > T(0)) || !(delta > T(0))) return 2;
  T alpha = gamma / delta, beta = 0;
  const T stop = (T)(tol * tol) * bb;
  int cur = 0;  // w[cur] = w_i, n[cur] = n_i, z[cur ^ 1] = z_{i-1}
  for (int it = 0; it < maxit; ++it) {
    const T a = alpha, bt = beta;
    const int nxt = cur ^ 1;
    T d3[3] = {};
#pragma unroll 2
    for (long long i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
      T pv[8], st[8];
      load8(pr + i * 8, pv);
      load8(sr + i * 8, st);
      const T wi = cur ? pv[1] : pv[0];
      const T ni = cur ? pv[3] : pv[2];
      const T zp = cur ? pv[4] : pv[5];
      const T mi = pv[6] * wi;
      const T zi = ni + bt * zp;
      const T qi = mi + bt * st[4];
      const T si = wi + bt * st[5];
      const T pi = st[2] + bt * st[3];
      const T ei = st[0] + a * pi;
      const T ri = st[1] - a * si;
      const T ui = st[2] - a * qi;
      const T wn = wi - a * zi;
      pr[i * 8 + nxt] = wn;        // w[nxt]
      pr[i * 8 + 4 + cur] = zi;    // z[cur]
      const T ns[8] = {ei, ri, ui, pi, qi, si, st[6], T(0)};
      store8(sr + i * 8, ns);
      d3[0] += ri * ui;
      d3[1] += wn * ui;
      d3[2] += ri * ri;
    }
    // n_{i+1} = S M^-1 w_{i+1}, w_{i+1} formed on the fly from (w_i, n_i, z_{i-1})
    fused_apply(s, A.pt, OpPipe<T>{pr, cur, a, bt}, pr + 2 + nxt, 8, wl);
    // one barrier per iteration: alternate the partial-sum slots so that a block
    // already in the next iteration never overwrites sums still being read
    const int sl = 6 + 3 * (it & 1);
    block_partials<3, T, T>(d3, A.partial, sl);
    // thread 0: next (alpha, beta) and the exit code (-2: continue)
    __shared__ T s_ab[2];
    __shared__ int s_exit;
    if (!grid_barrier_total<3, T>(A.ctl, nb, A.partial, sl, tot, [&](const T* t) {
          const T gnew = t[0], dnew = t[1], rr = t[2];
          int ex = -2;
          T al = alpha, be = beta;
          if (rr <= stop) ex = 0;
          else if (!(gnew > T(0))) ex = 2;
          else {
            be = gnew / gamma;
            const T den = dnew - be * gnew / alpha;
            if (!(den > T(0))) ex = 2;
            else al = gnew / den;
          }
          s_ab[0] = al;
          s_ab[1] = be;
          s_exit = ex;
        }))
      return -1;
    ++iters;
    if (s_exit != -2) return s_exit;
    alpha = s_ab[0];
    beta = s_ab[1];
    gamma = tot[0];
    cur = nxt;
  }
  return 1;
}

template <class T>
__global__ void __launch_bounds__(NT_FUSED, 1) k_pcg_fused(FusedArgs A) {
  barrier_init();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const long long gsz = (long long)gridDim.x * blockDim.x;
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const unsigned nb = gridDim.x;
  const SysView<double>& s64 = A.s64;
  T* pool = static_cast<T*>(A.pool);
  T* pr = pool;
  T* sr = pool + 8 * A.P;
  const T* dinv = static_cast<const T*>(A.dinv);
  double a0[1] = {0.0};
  for (long long i = tid; i < A.P; i += gsz) {
    A.x[i] = 0.0;
    if (i < A.nrow) {
      a0[0] += A.rhs[i] * A.rhs[i];
      pr[i * 8 + 6] = dinv[i];
    }
  }
  block_partials<1>(a0, A.partial, 12);
  if (!grid_barrier(A.ctl, nb)) return;
  const double bnorm = sqrt(grid_total(A.partial, 12));
  int iters = 0, status = 0, outer = 0;
  double rel = 0.0;
  const int g = blockIdx.x;
  const int c0 = g * A.pt.chunk, c1 = min(s64.Nc, c0 + A.pt.chunk);
  const long long r0 = (long long)s64.slots * c0, r1 = (long long)s64.slots * c1;
  if (bnorm > 0.0) {
    for (outer = 0;; ++outer) {
      double rr[1] = {0.0};
      if (outer == 0) {
        for (long long i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
          A.r64[i] = A.rhs[i];
          rr[0] += A.rhs[i] * A.rhs[i];
        }
      } else {
        fused_apply(s64, A.pt, PlainOp<double>{A.x}, A.q64, 1, reinterpret_cast<double*>(smem_raw));
        for (long long i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
          const double ri = A.rhs[i] - A.q64[i];
          A.r64[i] = ri;
          rr[0] += ri * ri;
        }
      }
      block_partials<1>(rr, A.partial, 13);
      if (!grid_barrier(A.ctl, nb)) return;
      const double rn = sqrt(grid_total(A.partial, 13));
      rel = rn / bnorm;
      if (rel <= A.tol) {
        status = 0;
        break;
      }
      if (outer >= A.max_outer || iters >= A.maxit) {
        status = 1;
        break;
      }
      const double inv = 1.0 / rn;
      for (long long i = r0 + threadIdx.x; i < r1; i += blockDim.x) sr[i * 8 + 6] = (T)(A.r64[i] * inv);
      if (!grid_barrier(A.ctl, nb)) return;
      const int before = iters;
      const int st = inner_pcg_fused<T>(A, A.inner_tol, A.maxit - iters, iters, reinterpret_cast<T*>(smem_raw));
      if (st < 0) return;
      for (long long i = r0 + threadIdx.x; i < r1; i += blockDim.x) A.x[i] += rn * (double)sr[i * 8];
      if (!grid_barrier(A.ctl, nb)) return;
      // a pipelined-CG breakdown after some progress (loss of orthogonality near
      // the attainable accuracy) restarts from the true residual; a breakdown
      // without progress is reported
      if (st == 2 && iters == before) {
        status = 2;
        break;
      }
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    A.ctl->iters = iters;
    A.ctl->outer = outer;
    A.ctl->scal[S_RELRES] = rel;
    A.ctl->scal[S_BNORM] = bnorm;
    A.ctl->halvings = status;
  }
}

// Jacobi diagonal of S: diag(N) + diag(H); dummy rows 1.
__global__ void k_diag(SysView<double> s, const double* __restrict__ H, double* __restrict__ d64,
                       float* __restrict__ d32, long long P) {
  const long long n = s.Nc;
  const long long gsz = (long long)gridDim.x * blockDim.x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P; i += gsz) {
    long long c = i / s.slots;
    int u = (int)(i - c * s.slots);
    double v = 1.0;
    if (c < n && u < 3) {
      v = diag_entry(s, (int)c, u);
      if (H) v += H[(u == 0 ? 0 : (u == 1 ? 3 : 5)) * n + c];
    }
    d64[i] = 1.0 / v;
    d32[i] = (float)(1.0 / v);
  }
}

__global__ void k_sqrt_into(const double* __restrict__ dinv, double* __restrict__ out, long long P) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P; i += (long long)gridDim.x * blockDim.x)
    out[i] = sqrt(dinv[i]);
}

// ------------------------------------------------------------------ PDIP kernels
struct PdipArgs {
  SysView<double> s;
  int Nc, slots;
  long long P;
  double mu, nu, alpha, beta, step_frac;
  int max_halvings;
  double* gamma;
  double* lambda;
  const double* r;       // [P]
  double* Ng;            // [P] N gamma
  double* rhs;           // [P]
  double* dg;            // [P] Newton direction
  double* NDg;           // [P] N dg
  double* dlam;          // [2Nc]
  double* H;
  float* H32;
  DevCtl* ctl;
  double* partial;
};

// gap, t, residual norms, Schur blocks and Newton rhs at (gamma, lambda).
// mode 0: full pre-step; mode 1: only eta and ||r_dual|| (measurement).
__global__ void __launch_bounds__(NT, 1) k_pdip_pre(PdipArgs A, int mode) {
  barrier_init();
  const long long gsz = (long long)gridDim.x * blockDim.x;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned nb = gridDim.x;
  const int n = A.Nc;
  SysView<double> s = A.s;
  s.H = nullptr;
  // N gamma
  for (int b = tid; b < s.M; b += (int)gsz) body_gather(s, plain<double>(A.gamma), b);
  if (!grid_barrier(A.ctl, nb)) return;
  double acc[1] = {0.0};
  for (int c = tid; c < n; c += (int)gsz) {
    contact_apply(s, plain<double>(A.gamma), A.Ng, c);
    const long long row = (long long)A.slots * c;
    double gn = A.gamma[row], g1 = A.gamma[row + 1], g2 = A.gamma[row + 2];
    double fc = 0.5 * (g1 * g1 + g2 * g2 - A.mu * A.mu * gn * gn);
    acc[0] += -(fc * A.lambda[c] + (-gn) * A.lambda[n + c]);
  }
  block_partials<1>(acc, A.partial, 0);
  if (!grid_barrier(A.ctl, nb)) return;
  const double eta = grid_total(A.partial, 0);
  const double t = A.nu * 2.0 * n / eta;
  double nr[2] = {0.0, 0.0};
  for (int c = tid; c < n; c += (int)gsz) {
    const long long row = (long long)A.slots * c;
    double gn = A.gamma[row], g1 = A.gamma[row + 1], g2 = A.gamma[row + 2];
    double lc = A.lambda[c], ln = A.lambda[n + c];
    double mu2 = A.mu * A.mu;
    double fc = 0.5 * (g1 * g1 + g2 * g2 - mu2 * gn * gn);
    double q0 = -mu2 * gn;
    double u0 = A.Ng[row] + A.r[row], u1 = A.Ng[row + 1] + A.r[row + 1], u2 = A.Ng[row + 2] + A.r[row + 2];
    double rd0 = u0 + lc * q0 - ln, rd1 = u1 + lc * g1, rd2 = u2 + lc * g2;
    double rc0 = -lc * fc - 1.0 / t, rc1 = -ln * (-gn) - 1.0 / t;
    nr[0] += rd0 * rd0 + rd1 * rd1 + rd2 * rd2;
    nr[1] += rc0 * rc0 + rc1 * rc1;
    if (mode == 0) {
      double h[6];
      schur_block(A.mu, gn, g1, g2, lc, ln, h);
      for (int k = 0; k < 6; ++k) {
        A.H[(size_t)k * n + c] = h[k];
        A.H32[(size_t)k * n + c] = (float)h[k];
      }
      // rhs = -(N gamma + r) + (1/t) (g/f_c + e1/gn)
      A.rhs[row] = -u0 + (q0 / fc + 1.0 / gn) / t;
      A.rhs[row + 1] = -u1 + (g1 / fc) / t;
      A.rhs[row + 2] = -u2 + (g2 / fc) / t;
      if (A.slots == 4) A.rhs[row + 3] = 0.0;
    }
  }
  block_partials<2>(nr, A.partial, 1);
  if (!grid_barrier(A.ctl, nb)) return;
  const double rd2 = grid_total(A.partial, 1), rc2 = grid_total(A.partial, 2);
  if (mode == 0) {
    for (long long i = (long long)A.slots * n + tid; i < A.P; i += gsz) A.rhs[i] = 0.0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    A.ctl->scal[S_ETA] = eta;
    A.ctl->scal[S_T] = t;
    A.ctl->scal[S_RDUAL] = sqrt(rd2);
    A.ctl->scal[S_RT] = sqrt(rd2 + rc2);
  }
}

// dlambda, ratio test, backtracking (feasibility, then sufficient decrease of
// ||r_t||), update.  Every block evaluates the same reduced scalars, so all
// blocks take the same branches.
__global__ void __launch_bounds__(NT, 1) k_pdip_post(PdipArgs A) {
  barrier_init();
  const long long gsz = (long long)gridDim.x * blockDim.x;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned nb = gridDim.x;
  const int n = A.Nc;
  const double t = A.ctl->scal[S_T];
  const double rt0 = A.ctl->scal[S_RT];
  const double mu2 = A.mu * A.mu;
  SysView<double> s = A.s;
  s.H = nullptr;
  // N dg
  for (int b = tid; b < s.M; b += (int)gsz) body_gather(s, plain<double>(A.dg), b);
  if (!grid_barrier(A.ctl, nb)) return;
  double mn[1] = {1e300};
  for (int c = tid; c < n; c += (int)gsz) {
    contact_apply(s, plain<double>(A.dg), A.NDg, c);
    const long long row = (long long)A.slots * c;
    double gn = A.gamma[row], g1 = A.gamma[row + 1], g2 = A.gamma[row + 2];
    double d0 = A.dg[row], d1 = A.dg[row + 1], d2 = A.dg[row + 2];
    double lc = A.lambda[c], ln = A.lambda[n + c];
    double fc = 0.5 * (g1 * g1 + g2 * g2 - mu2 * gn * gn), fn = -gn;
    double gdc = -mu2 * gn * d0 + g1 * d1 + g2 * d2, gdn = -d0;
    double dlc = -lc - 1.0 / (t * fc) - (lc / fc) * gdc;
    double dln = -ln - 1.0 / (t * fn) - (ln / fn) * gdn;
    A.dlam[c] = dlc;
    A.dlam[n + c] = dln;
    if (dlc < 0.0) mn[0] = fmin(mn[0], -lc / dlc);
    if (dln < 0.0) mn[0] = fmin(mn[0], -ln / dln);
  }
  block_partials<1>(mn, A.partial, 0, true);
  if (!grid_barrier(A.ctl, nb)) return;
  double smax = fmin(1.0, grid_total(A.partial, 0, true));
  double sstep = A.step_frac * smax;
  int halv = 0;
  int status = 0;
  // feasibility: all f(gamma + s dg) < 0
  for (;;) {
    double bad[1] = {0.0};
    for (int c = tid; c < n; c += (int)gsz) {
      const long long row = (long long)A.slots * c;
      double gn = A.gamma[row] + sstep * A.dg[row];
      double g1 = A.gamma[row + 1] + sstep * A.dg[row + 1];
      double g2 = A.gamma[row + 2] + sstep * A.dg[row + 2];
      double fc = 0.5 * (g1 * g1 + g2 * g2 - mu2 * gn * gn);
      if (fc >= 0.0 || -gn >= 0.0) bad[0] += 1.0;
    }
    block_partials<1>(bad, A.partial, 1 + (halv & 1));
    if (!grid_barrier(A.ctl, nb)) return;
    if (grid_total(A.partial, 1 + (halv & 1)) == 0.0) break;
    sstep *= A.beta;
    if (++halv > A.max_halvings) {
      status = QP_LINESEARCH_FAIL;
      break;
    }
  }
  // sufficient decrease of ||r_t|| at fixed t
  while (status == 0) {
    double nr[1] = {0.0};
    for (int c = tid; c < n; c += (int)gsz) {
      const long long row = (long long)A.slots * c;
      double gn = A.gamma[row] + sstep * A.dg[row];
      double g1 = A.gamma[row + 1] + sstep * A.dg[row + 1];
      double g2 = A.gamma[row + 2] + sstep * A.dg[row + 2];
      double lc = A.lambda[c] + sstep * A.dlam[c];
      double ln = A.lambda[n + c] + sstep * A.dlam[n + c];
      double fc = 0.5 * (g1 * g1 + g2 * g2 - mu2 * gn * gn);
      double u0 = A.Ng[row] + sstep * A.NDg[row] + A.r[row];
      double u1 = A.Ng[row + 1] + sstep * A.NDg[row + 1] + A.r[row + 1];
      double u2 = A.Ng[row + 2] + sstep * A.NDg[row + 2] + A.r[row + 2];
      double rd0 = u0 + lc * (-mu2 * gn) - ln, rd1 = u1 + lc * g1, rd2 = u2 + lc * g2;
      double rc0 = -lc * fc - 1.0 / t, rc1 = -ln * (-gn) - 1.0 / t;
      nr[0] += rd0 * rd0 + rd1 * rd1 + rd2 * rd2 + rc0 * rc0 + rc1 * rc1;
    }
    block_partials<1>(nr, A.partial, 3 + (halv & 1));
    if (!grid_barrier(A.ctl, nb)) return;
    if (sqrt(grid_total(A.partial, 3 + (halv & 1))) <= (1.0 - A.alpha * sstep) * rt0) break;
    sstep *= A.beta;
    if (++halv > A.max_halvings) {
      status = QP_LINESEARCH_FAIL;
      break;
    }
  }
  if (status == 0) {
    for (int c = tid; c < n; c += (int)gsz) {
      const long long row = (long long)A.slots * c;
      for (int u = 0; u < 3; ++u) A.gamma[row + u] += sstep * A.dg[row + u];
      A.lambda[c] += sstep * A.dlam[c];
      A.lambda[n + c] += sstep * A.dlam[n + c];
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    A.ctl->scal[S_S] = sstep;
    A.ctl->scal[S_SMAX] = smax;
    A.ctl->halvings = halv;
    A.ctl->iters = status;
  }
}

__global__ void k_pdip_init(int Nc, int slots, long long P, double mu, double gn0, double* gamma, double* lambda) {
  const long long gsz = (long long)gridDim.x * blockDim.x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P; i += gsz) {
    long long c = i / slots;
    int u = (int)(i - c * slots);
    gamma[i] = (c < Nc && u == 0) ? gn0 : 0.0;
    if (i < Nc) {
      // f_c = -mu^2 gn0^2 / 2, f_{Nc+c} = -gn0; lambda = -1/f
      lambda[i] = 2.0 / (mu * mu * gn0 * gn0);
      lambda[Nc + i] = 1.0 / gn0;
    }
  }
}

// Time step (Sec. 2.3, Eqs. force_balance_disc, particle_evolution_disc):
// v' = (v + dt g) + M^-1 D gamma, omega' = omega + I^-1 (D gamma)_torque,
// x' = x + dt v'.  SoA [3][M] in and out; one thread per body reads its inputs
// before it writes, so outputs may alias inputs.
__global__ void k_advance(SysView<double> s, const double* __restrict__ gamma, const double* pos,
                          const double* vel, const double* omega, double dt, double gx, double gy, double gz,
                          double* pos_o, double* vel_o, double* om_o) {
  const int M = s.M;
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < M; b += gridDim.x * blockDim.x) {
    double w[6];
    body_gather_vals(s, plain<double>(gamma), b, w);
    const double v0 = (vel[b] + dt * gx) + w[0];
    const double v1 = (vel[M + b] + dt * gy) + w[1];
    const double v2 = (vel[2 * M + b] + dt * gz) + w[2];
    const double o0 = omega[b] + w[3], o1 = omega[M + b] + w[4], o2 = omega[2 * M + b] + w[5];
    const double x0 = pos[b] + dt * v0, x1 = pos[M + b] + dt * v1, x2 = pos[2 * M + b] + dt * v2;
    vel_o[b] = v0;
    vel_o[M + b] = v1;
    vel_o[2 * M + b] = v2;
    om_o[b] = o0;
    om_o[M + b] = o1;
    om_o[2 * M + b] = o2;
    pos_o[b] = x0;
    pos_o[M + b] = x1;
    pos_o[2 * M + b] = x2;
  }
}

// Bounded-wait self-test: block `absent` never arrives at the grid barrier, so
// every other block's wait runs out after `budget` clock ticks and records
// QP_TIMEOUT (absent < 0: all arrive, no error).  Nothing hangs either way.
__global__ void k_barrier_probe(DevCtl* ctl, long long budget, int absent) {
  barrier_init();
  if ((int)blockIdx.x == absent) return;
  grid_barrier(ctl, gridDim.x, budget);
}

template <class K>
int coop_grid(qp_ctx* c, K kernel) {
  int per_sm = 0;
  QP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, NT, 0));
  QP_REQUIRE(per_sm > 0, QP_CUDA_ERROR, "cooperative kernel does not fit on an SM");
  if (per_sm > 2) per_sm = 2;
  QP_REQUIRE(per_sm * c->num_sms <= 4096, QP_INVALID_ARG, "grid larger than the partial-sum array");
  return per_sm * c->num_sms;
}

template <class K, class Arg>
void coop_launch(qp_ctx* c, K kernel, int grid, Arg& a) {
  void* args[] = {&a};
  QP_CUDA(cudaLaunchCooperativeKernel((const void*)kernel, dim3(grid), dim3(NT), args, 0, c->stream));
}

template <class K, class Arg>
void coop_launch2(qp_ctx* c, K kernel, int grid, Arg& a, int& mode) {
  void* args[] = {&a, &mode};
  QP_CUDA(cudaLaunchCooperativeKernel((const void*)kernel, dim3(grid), dim3(NT), args, 0, c->stream));
}

}  // namespace

// ---------------------------------------------------------------- host side
void launch_schur_blocks(qp_ctx* c, const double* gamma, const double* lambda) {
  if (c->Nc == 0) return;
  PdipView v{c->Nc, c->slots, c->mu, const_cast<double*>(gamma), const_cast<double*>(lambda)};
  k_schur_blocks<<<ceil_div(c->Nc, 256), 256, 0, c->stream>>>(v, c->H.as<double>(), c->H32.as<float>());
  QP_CUDA(cudaGetLastError());
}

// rowscale[i] = diag(S)_i^-1/2 for the current Schur blocks (dummy rows: 1).
void launch_rowscale(qp_ctx* c, double* rowscale) {
  SysView<double> s64 = view64(c, true);
  k_diag<<<c->num_sms * 4, 256, 0, c->stream>>>(s64, c->H.as<double>(), c->dinv.as<double>(), c->dinv32.as<float>(),
                                                c->P);
  k_sqrt_into<<<c->num_sms * 4, 256, 0, c->stream>>>(c->dinv.as<double>(), rowscale, c->P);
  QP_CUDA(cudaGetLastError());
}

void launch_apply64(qp_ctx* c, const double* x, double* y, bool with_H) {
  SysView<double> s = view64(c, with_H);
  int g = c->num_sms * 8;
  if (c->M > 0)
    k_body_gather_lanes<double, QP_APPLY_LANES><<<ceil_div((long long)c->M * QP_APPLY_LANES, 256), 256, 0, c->stream>>>(s, x);
  k_contact_apply<double><<<g, 256, 0, c->stream>>>(s, x, y);
  QP_CUDA(cudaGetLastError());
}

void launch_apply32(qp_ctx* c, const float* x, float* y, bool with_H) {
  SysView<float> s = view32(c, with_H);
  int g = c->num_sms * 8;
  if (c->M > 0)
    k_body_gather_lanes<float, QP_APPLY_LANES><<<ceil_div((long long)c->M * QP_APPLY_LANES, 256), 256, 0, c->stream>>>(s, x);
  k_contact_apply<float><<<g, 256, 0, c->stream>>>(s, x, y);
  QP_CUDA(cudaGetLastError());
}

static void reset_ctl(qp_ctx* c) {
  QP_CUDA(cudaMemsetAsync(c->ctl.p, 0, sizeof(DevCtl), c->stream));
}

static DevCtl read_ctl(qp_ctx* c) {
  QP_CUDA(cudaMemcpyAsync(c->ctl_host, c->ctl.p, sizeof(DevCtl), cudaMemcpyDeviceToHost, c->stream));
  QP_CUDA(cudaStreamSynchronize(c->stream));
  return *c->ctl_host;
}

static PdipArgs pdip_args(qp_ctx* c, const qp_state* st) {
  PdipArgs A;
  A.s = view64(c, false);
  A.Nc = c->Nc;
  A.slots = c->slots;
  A.P = c->P;
  A.mu = c->mu;
  A.nu = 10.0;
  A.alpha = 0.01;
  A.beta = 0.5;
  A.step_frac = 0.99;
  A.max_halvings = 60;
  A.gamma = st->gamma;
  A.lambda = st->lambda;
  A.r = c->r.as<double>();
  const size_t P = (size_t)c->P;
  A.Ng = static_cast<double*>(c->v64[0].ensure(P * sizeof(double)));
  A.rhs = static_cast<double*>(c->v64[1].ensure(P * sizeof(double)));
  A.dg = static_cast<double*>(c->v64[2].ensure(P * sizeof(double)));
  A.NDg = static_cast<double*>(c->v64[3].ensure(P * sizeof(double)));
  A.dlam = static_cast<double*>(c->v64[4].ensure(2 * (size_t)(c->Nc > 0 ? c->Nc : 1) * sizeof(double)));
  A.H = c->H.as<double>();
  A.H32 = c->H32.as<float>();
  A.ctl = c->ctl.as<DevCtl>();
  A.partial = c->partial.as<double>();
  return A;
}

static void ensure_partial(qp_ctx* c) {
  c->partial.ensure((size_t)c->num_sms * 8 * NRED * sizeof(double));
}

static void check_ready(qp_ctx* c, const qp_state* st) {
  QP_REQUIRE(c->have_contacts, QP_NOT_READY, "no contacts: call ccp_assemble first");
  if (st) QP_REQUIRE(st->gamma && st->lambda, QP_INVALID_ARG, "state with null gamma/lambda");
}

static void pdip_pre(qp_ctx* c, qp_state* st, int mode, const qp_pdip_opts* o) {
  ensure_partial(c);
  PdipArgs A = pdip_args(c, st);
  if (o) {
    A.nu = o->nu;
  }
  int grid = coop_grid(c, k_pdip_pre);
  reset_ctl(c);
  coop_launch2(c, k_pdip_pre, grid, A, mode);
}

// Contact partition into G chunks (one per block) with each block's body set.
static void build_partition(qp_ctx* c, int G, qp::Buf& b_nb, qp::Buf& b_bodies, qp::Buf& b_cl, int& chunk_out,
                            int& maxb_out, int& nbmax_out) {
  const int Nc = c->Nc;
  const int chunk = std::max(1, (Nc + G - 1) / G);
  QP_REQUIRE(chunk <= 16384, QP_INVALID_ARG, "too many contacts per block for the fused operator");
  int n2 = 1;
  while (n2 < 2 * chunk) n2 <<= 1;
  const int maxb = 2 * chunk;
  int* nb = static_cast<int*>(b_nb.ensure((size_t)G * sizeof(int)));
  int* bodies = static_cast<int*>(b_bodies.ensure((size_t)G * maxb * sizeof(int)));
  int* cl = static_cast<int*>(b_cl.ensure(2 * (size_t)std::max(Nc, 1) * sizeof(int)));
  const size_t smem = (size_t)n2 * sizeof(int);
  QP_CUDA(cudaFuncSetAttribute(k_partition, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_partition<<<G, 1024, smem, c->stream>>>(Nc, c->M, chunk, maxb, c->ca.as<int>(), c->cb.as<int>(), nb, bodies, cl);
  QP_CUDA(cudaGetLastError());
  std::vector<int> h(G);
  QP_CUDA(cudaMemcpyAsync(h.data(), nb, (size_t)G * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  QP_CUDA(cudaStreamSynchronize(c->stream));
  int mx = 1;
  for (int v : h) mx = std::max(mx, v);
  chunk_out = chunk;
  maxb_out = maxb;
  nbmax_out = mx;
}

static void ensure_partition(qp_ctx* c, int G) {
  if (c->part_G == G) return;
  build_partition(c, G, c->part_nb, c->part_bodies, c->part_cl, c->part_chunk, c->part_maxb, c->part_nbmax);
  c->part_G = G;
}

// Partition of the standalone fused apply: chunks of about 256 contacts, the
// block count a multiple of the SM count; cached per contact set.
static Part apply_partition(qp_ctx* c) {
  const int want = std::max(1, (c->Nc + 255) / 256);
  const int G = ((want + c->num_sms - 1) / c->num_sms) * c->num_sms;
  if (c->apart_G != G) {
    build_partition(c, G, c->apart_nb, c->apart_bodies, c->apart_cl, c->apart_chunk, c->apart_maxb,
                    c->apart_nbmax);
    c->apart_G = G;
  }
  return Part{c->apart_chunk, c->apart_maxb, c->apart_nb.as<int>(), c->apart_bodies.as<int>(), c->apart_cl.as<int>()};
}

template <class T>
static void launch_apply_one(qp_ctx* c, const SysView<T>& s, const T* x, T* y, const qp_state* st) {
  if (c->Nc == 0) {
    // no contacts: every row is a dummy row
    QP_CUDA(cudaMemcpyAsync(y, x, (size_t)c->P * sizeof(T), cudaMemcpyDeviceToDevice, c->stream));
    return;
  }
  const Part pt = apply_partition(c);
  const size_t smem = (size_t)c->apart_nbmax * 8 * sizeof(T);
  const int G = c->apart_G;
  if (st) {
    auto k = k_apply_one<T, true, 4>;
    QP_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k<<<G, 256, smem, c->stream>>>(s, pt, x, y, st->gamma, st->lambda, c->mu);
  } else {
    auto k = k_apply_one<T, false, 4>;
    QP_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k<<<G, 256, smem, c->stream>>>(s, pt, x, y, nullptr, nullptr, c->mu);
  }
  QP_CUDA(cudaGetLastError());
}

template <class T>
static void launch_fused(qp_ctx* c, FusedArgs& A) {
  auto k = k_pcg_fused<T>;
  const size_t smem = (size_t)c->part_nbmax * 8 * sizeof(double);
  QP_REQUIRE(smem <= 200 * 1024, QP_INVALID_ARG, "fused Krylov kernel: body set of a block exceeds shared memory");
  QP_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  QP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, NT_FUSED, smem));
  QP_REQUIRE(per_sm >= 1, QP_CUDA_ERROR, "fused Krylov kernel does not fit on an SM");
  const int G = c->part_G;
  QP_REQUIRE(G <= per_sm * c->num_sms, QP_CUDA_ERROR, "fused Krylov grid exceeds co-resident blocks");
  void* args[] = {&A};
  QP_CUDA(cudaLaunchCooperativeKernel((const void*)k, dim3(G), dim3(NT_FUSED), args, smem, c->stream));
}

static void solve_fused(qp_ctx* c, const double* rhs, double* dx, const qp_solve_opts* o, bool mixed) {
  // one block per SM: the partition is built for that grid
  const int G = c->num_sms;
  ensure_partition(c, G);
  const size_t P = (size_t)c->P;
  const size_t es = mixed ? sizeof(float) : sizeof(double);
  FusedArgs A;
  A.s64 = view64(c, true);
  A.s32 = view32(c, true);
  A.pt.chunk = c->part_chunk;
  A.pt.maxb = c->part_maxb;
  A.pt.nb = c->part_nb.as<int>();
  A.pt.bodies = c->part_bodies.as<int>();
  A.pt.cl = c->part_cl.as<int>();
  A.nrow = c->slots * c->Nc;
  A.P = c->P;
  A.rhs = rhs;
  A.x = dx;
  A.r64 = static_cast<double*>(c->v64[5].ensure(P * sizeof(double)));
  A.q64 = static_cast<double*>(c->v64[6].ensure(P * sizeof(double)));
  // pipe + state records in a buffer of their own: the classic solver that may
  // run after a failed fused solve holds pointers into v32 / scratch, which a
  // reallocation here would invalidate
  A.pool = c->fused_pool.ensure(16 * P * es);
  A.dinv = mixed ? (const void*)c->dinv32.p : (const void*)c->dinv.p;
  A.tol = o->tol;
  A.inner_tol = mixed ? (o->inner_tol > 0 ? o->inner_tol : 1e-4) : (o->inner_tol > 0 ? o->inner_tol : o->tol);
  A.maxit = o->maxit;
  A.max_outer = o->max_outer > 0 ? o->max_outer : (mixed ? 50 : 20);
  A.ctl = c->ctl.as<DevCtl>();
  A.partial = c->partial.as<double>();
  reset_ctl(c);
  QP_CUDA(cudaEventRecord(c->ev0, c->stream));
  if (mixed) launch_fused<float>(c, A);
  else launch_fused<double>(c, A);
}

// solve S dx = rhs with the current H blocks (already built for st)
static qp_solve_stats solve_once(qp_ctx* c, const double* rhs, double* dx, const qp_solve_opts* o) {
  ensure_partial(c);
  QP_REQUIRE(o, QP_INVALID_ARG, "newton_solve: null options");
  QP_REQUIRE(o->tol > 0 && o->maxit > 0, QP_INVALID_ARG, "newton_solve: tol > 0 and maxit > 0 required");
  const bool mixed = o->mixed != 0;
  QP_REQUIRE(o->precond == QP_JACOBI_PCG || o->precond == QP_QTT_PCG || o->precond == QP_QTT_DIRECT,
             QP_INVALID_ARG, "newton_solve: unknown preconditioner");
  const bool use_qtt = o->precond == QP_QTT_PCG || o->precond == QP_QTT_DIRECT;
  QP_REQUIRE(!use_qtt || o->X, QP_INVALID_ARG, "newton_solve: QTT preconditioner requires X");
  const size_t P = (size_t)c->P;
  PcgArgs A;
  A.s64 = view64(c, true);
  A.s32 = view32(c, true);
  A.nrow = c->slots * c->Nc;
  A.P = c->P;
  A.rhs = rhs;
  A.x = dx;
  A.r64 = static_cast<double*>(c->v64[5].ensure(P * sizeof(double)));
  A.q64 = static_cast<double*>(c->v64[6].ensure(P * sizeof(double)));
  const size_t es = mixed ? sizeof(float) : sizeof(double);
  // inner vectors: for FP64 reuse slots 7 and scratch; keep distinct buffers
  A.b = (mixed ? c->v32[0] : c->scratch[0]).ensure(P * es);
  A.e = (mixed ? c->v32[1] : c->scratch[1]).ensure(P * es);
  A.r = (mixed ? c->v32[2] : c->scratch[2]).ensure(P * es);
  A.z = (mixed ? c->v32[3] : c->scratch[3]).ensure(P * es);
  A.p = (mixed ? c->v32[4] : c->scratch[4]).ensure(P * es);
  A.q = (mixed ? c->v32[5] : c->v64[7]).ensure(2 * P * es);  // q and the second search direction
  A.dinv = mixed ? (const void*)c->dinv32.p : (const void*)c->dinv.p;
  A.use_qtt = use_qtt ? 1 : 0;
  A.qtt_scaled = (use_qtt && o->X->scaled) ? 1 : 0;
  A.qw0 = A.qw1 = nullptr;
  A.krylov = o->krylov == QP_BICGSTAB ? QP_BICGSTAB : QP_CG;
  A.direct = o->precond == QP_QTT_DIRECT ? 1 : 0;
  A.reliable = (mixed && !use_qtt && A.krylov == QP_CG && !A.direct) ? 1 : 0;
  A.rec_cache = 0;
  A.xb = A.krylov == QP_BICGSTAB ? c->dm[12].ensure(5 * P * es) : nullptr;
  qp_dtype cdt = QP_F64;
  if (use_qtt) {
    qp_qtt* X = o->X;
    QP_REQUIRE(X->d == c->L, QP_INVALID_ARG, "newton_solve: preconditioner size does not match 2^L");
    QP_REQUIRE(X->d <= 64, QP_INVALID_ARG, "QTT with more than 64 cores");
    cdt = mixed ? (o->core_dtype == QP_BF16 ? QP_BF16 : QP_F32) : QP_F64;
    qtt_prepare_copies(c, X, cdt);
    A.qtt.d = X->d;
    int rmax = 1;
    for (int k = 0; k <= X->d; ++k) {
      A.qtt.ranks[k] = X->ranks[k];
      A.qtt.off[k] = X->offset[k];
      if (X->ranks[k] > rmax) rmax = X->ranks[k];
    }
    A.qtt.rmax = rmax;
    A.qtt.cores = cdt == QP_F64 ? (const void*)X->cores : (cdt == QP_F32 ? (const void*)X->cores32 : (const void*)X->cores16);
    A.qw0 = (mixed ? c->v32[6] : c->scratch[5]).ensure(P * es * rmax);
    A.qw1 = (mixed ? c->v32[7] : c->scratch[6]).ensure(P * es * rmax);
  }
  A.tol = o->tol;
  A.inner_tol = mixed ? (o->inner_tol > 0 ? o->inner_tol : 1e-4) : (o->inner_tol > 0 ? o->inner_tol : o->tol);
  A.maxit = o->maxit;
  A.max_outer = o->max_outer > 0 ? o->max_outer : (A.direct ? 100 : (mixed ? 50 : 5));
  A.ctl = c->ctl.as<DevCtl>();
  A.partial = c->partial.as<double>();

  // Jacobi diagonal from the current blocks
  SysView<double> s64 = view64(c, true);
  k_diag<<<c->num_sms * 4, 256, 0, c->stream>>>(s64, c->H.as<double>(), c->dinv.as<double>(), c->dinv32.as<float>(),
                                                c->P);
  QP_CUDA(cudaGetLastError());
  // Jacobi preconditioner: pipelined CG with the fused operator (one grid
  // barrier per iteration) on small systems, classic CG otherwise; a failed
  // pipelined solve (its recurrence residual can drift from the true one at
  // tight FP64 tolerances) is redone with classic CG.
  bool done = false;
  // The fused kernel removes two of the three grid barriers of an iteration but
  // gathers border bodies redundantly and forms its operand on the fly; that
  // pays off while iterations are barrier-bound (few contacts per block).
  // Pipelined CG reaches a lower attainable accuracy than classic CG (its
  // recurrences propagate local rounding errors; Cools et al., SIAM J. Matrix
  // Anal. Appl. 39 (2018)): at FP64 tolerances below 1e-9 its recurrence
  // residual drifts from the true one and the refinement restarts it, so those
  // solves take the classic kernel.
  const bool fused = !use_qtt && A.krylov == QP_CG && (c->Nc + c->num_sms - 1) / c->num_sms <= FUSED_MAX_CHUNK &&
                     (mixed || o->tol >= 1e-9);
  if (fused) {
    solve_fused(c, rhs, dx, o, mixed);
    QP_CUDA(cudaMemcpyAsync(c->ctl_host, c->ctl.p, sizeof(DevCtl), cudaMemcpyDeviceToHost, c->stream));
    QP_CUDA(cudaStreamSynchronize(c->stream));
    done = c->ctl_host->err == 0 && c->ctl_host->halvings == 0;
  }
  if (!done) {
    reset_ctl(c);
    QP_CUDA(cudaEventRecord(c->ev0, c->stream));
    if (mixed && use_qtt) {
      if (cdt == QP_BF16) {
        auto k = k_pcg<float, __nv_bfloat16>;
        coop_launch(c, k, coop_grid(c, k), A);
      } else {
        auto k = k_pcg<float, float>;
        coop_launch(c, k, coop_grid(c, k), A);
      }
    } else if (mixed) {
      auto k = k_pcg<float, void>;
      // geometry cache of the body gather: as many incidences as the shared
      // memory left by the kernel's static arrays holds (48 bytes each)
      static int cap_of[64];  // per device; 0: not yet measured, else 1 + capacity
      int& slot = cap_of[c->device & 63];
      int cap = slot - 1;
      if (slot == 0) {
        cudaFuncAttributes fa;
        QP_CUDA(cudaFuncGetAttributes(&fa, k));
        int optin = 0;
        QP_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device));
        const long long room = (long long)optin - (long long)fa.sharedSizeBytes - 1024;
        cap = room > 0 ? (int)std::min<long long>(room / (3 * (long long)sizeof(float4)), 4096) : 0;
        if (cap > 0)
          QP_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       cap * 3 * (int)sizeof(float4)));
        slot = cap + 1;
      }
      // only as much as a block needs (its share of the incidences), so that the
      // rest of the unified L1 / shared memory stays L1 cache
      const long long need = 2LL * c->Nc / c->num_sms + 64;
      A.rec_cache = (int)std::min<long long>(cap, need);
      const size_t smem = (size_t)A.rec_cache * 3 * sizeof(float4);
      int per_sm = 0;
      QP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, NT, smem));
      QP_REQUIRE(per_sm > 0, QP_CUDA_ERROR, "cooperative kernel does not fit on an SM");
      void* args[] = {&A};
      QP_CUDA(cudaLaunchCooperativeKernel((const void*)k, dim3(c->num_sms * (per_sm > 2 ? 2 : per_sm)), dim3(NT),
                                          args, smem, c->stream));
    } else if (use_qtt) {
      auto k = k_pcg<double, double>;
      coop_launch(c, k, coop_grid(c, k), A);
    } else {
      auto k = k_pcg<double, void>;
      coop_launch(c, k, coop_grid(c, k), A);
    }
  }
  QP_CUDA(cudaEventRecord(c->ev1, c->stream));
  DevCtl h = read_ctl(c);
  qp_solve_stats out;
  float ms = 0;
  QP_CUDA(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
  out.ms = ms;
  out.iters = h.iters;
  out.outer = h.outer;
  out.rel_res = h.scal[S_RELRES];
  if (h.err) out.status = h.err;
  else if (h.halvings == 2) out.status = QP_BREAKDOWN;
  else if (h.halvings == 1) out.status = QP_NOT_CONVERGED;
  else out.status = QP_OK;
  out.fallback = 0;
  return out;
}

// A QTT-preconditioned solve that breaks down (the rank-truncated inverse need
// not be definite), or a QTT direct solve whose refinement does not converge,
// is redone with the Jacobi preconditioner on the device (stats.fallback = 1).
static qp_solve_stats solve(qp_ctx* c, const double* rhs, double* dx, const qp_solve_opts* o) {
  qp_solve_stats st = solve_once(c, rhs, dx, o);
  if ((o->precond == QP_QTT_PCG || o->precond == QP_QTT_DIRECT) &&
      (st.status == QP_BREAKDOWN || st.status == QP_NOT_CONVERGED)) {
    qp_solve_opts j = *o;
    j.precond = QP_JACOBI_PCG;
    j.X = nullptr;
    qp_solve_stats s2 = solve_once(c, rhs, dx, &j);
    s2.iters += st.iters;
    s2.ms += st.ms;
    s2.fallback = 1;
    return s2;
  }
  return st;
}

// Batched solve: build the scene table, group the scenes into cluster jobs
// (large scenes split over two blocks, small ones paired), launch one cluster
// per job (block size given or measured), read the per-scene results.
template <bool QTT>
static void launch_batched_t(qp_ctx* c0, int nt, int grid, const BatchScene* tab, const int2* jobs, double tol,
                             double itol, int maxit, int mo, BatchOut* out, unsigned tm) {
  switch (nt) {
    case 128: k_pcg_batched<128, QTT><<<grid, 128, 0, c0->stream>>>(tab, jobs, tol, itol, maxit, mo, out, tm); break;
    case 256: k_pcg_batched<256, QTT><<<grid, 256, 0, c0->stream>>>(tab, jobs, tol, itol, maxit, mo, out, tm); break;
    case 512: k_pcg_batched<512, QTT><<<grid, 512, 0, c0->stream>>>(tab, jobs, tol, itol, maxit, mo, out, tm); break;
    default: k_pcg_batched<1024, QTT><<<grid, 1024, 0, c0->stream>>>(tab, jobs, tol, itol, maxit, mo, out, tm); break;
  }
}

static void launch_batched(qp_ctx* c0, int nt, int njobs, const BatchScene* tab, const int2* jobs,
                           const qp_batch_opts* o, BatchOut* out, bool qtt, unsigned tilemask) {
  const double itol = o->inner_tol > 0 ? o->inner_tol : 1e-3;
  const int mo = o->max_outer > 0 ? o->max_outer : 50;
  const int grid = 2 * njobs;
  if (qtt) launch_batched_t<true>(c0, nt, grid, tab, jobs, o->tol, itol, o->maxit, mo, out, tilemask);
  else launch_batched_t<false>(c0, nt, grid, tab, jobs, o->tol, itol, o->maxit, mo, out, tilemask);
  QP_CUDA(cudaGetLastError());
}

// Measured tile shapes of the batched QTT apply, per (device, block size): for
// each input-rank class (<= 4, <= 8, <= 16) one block applies a d = 14 QTT of
// that interior rank with one and with two column items per thread (4 applies
// each, timed with events after a warm-up), and the faster shape sets the bit.
static std::mutex g_tile_mu;
static std::map<std::pair<int, int>, unsigned> g_tiles;

template <int NTB>
static float time_tile_probe(qp_ctx* c, const QttDev& q, const float* x, float* y, float* qw, unsigned tm) {
  k_qtt_tile_probe<NTB><<<1, NTB, 0, c->stream>>>(q, x, y, qw, tm, 1);
  QP_CUDA(cudaEventRecord(c->ev0, c->stream));
  k_qtt_tile_probe<NTB><<<1, NTB, 0, c->stream>>>(q, x, y, qw, tm, 4);
  QP_CUDA(cudaEventRecord(c->ev1, c->stream));
  QP_CUDA(cudaEventSynchronize(c->ev1));
  QP_CUDA(cudaGetLastError());
  float ms = 0.f;
  QP_CUDA(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
  return ms;
}

static unsigned batch_tile_mask(qp_ctx* c, int nt) {
  const auto key = std::make_pair(c->device, nt);
  {
    std::lock_guard<std::mutex> lock(g_tile_mu);
    auto it = g_tiles.find(key);
    if (it != g_tiles.end()) return it->second;
  }
  constexpr int d = 14;
  const long long P = 1LL << d;
  unsigned mask = 0;
  for (int cls = 0; cls < 3; ++cls) {
    const int R = 4 << cls;
    QttDev q;
    q.d = d;
    q.rmax = R;
    long long off = 0;
    for (int k = 0; k <= d; ++k) {
      q.ranks[k] = (k == 0 || k == d) ? 1 : R;
      q.off[k] = off;
      if (k < d) off += (long long)((k == 0) ? 1 : R) * 4 * ((k + 1 == d) ? 1 : R);
    }
    // deterministic core values of unit scale (any finite values time the same)
    std::vector<float> hc((size_t)off);
    for (size_t i = 0; i < hc.size(); ++i) hc[i] = (float)(((i * 2654435761u) % 1000u) / 1000.0 - 0.5);
    char* buf = static_cast<char*>(c->tune_buf.ensure(sizeof(float) * ((size_t)off + 2 * (size_t)P + 2 * (size_t)P * R)));
    float* cores = reinterpret_cast<float*>(buf);
    float* x = cores + off;
    float* y = x + P;
    float* qw = y + P;
    QP_CUDA(cudaMemcpyAsync(cores, hc.data(), sizeof(float) * (size_t)off, cudaMemcpyHostToDevice, c->stream));
    QP_CUDA(cudaMemsetAsync(x, 0, sizeof(float) * (size_t)P, c->stream));
    q.cores = cores;
    float t1 = 0.f, t2 = 0.f;
    const unsigned bit = 1u << cls;
    switch (nt) {
      case 128: t1 = time_tile_probe<128>(c, q, x, y, qw, 0u); t2 = time_tile_probe<128>(c, q, x, y, qw, bit); break;
      case 256: t1 = time_tile_probe<256>(c, q, x, y, qw, 0u); t2 = time_tile_probe<256>(c, q, x, y, qw, bit); break;
      case 512: t1 = time_tile_probe<512>(c, q, x, y, qw, 0u); t2 = time_tile_probe<512>(c, q, x, y, qw, bit); break;
      default: t1 = time_tile_probe<1024>(c, q, x, y, qw, 0u); t2 = time_tile_probe<1024>(c, q, x, y, qw, bit); break;
    }
    if (t2 < t1) mask |= bit;
  }
  std::lock_guard<std::mutex> lock(g_tile_mu);
  g_tiles[key] = mask;
  return mask;
}

// Cluster jobs from per-scene costs: with split = 0 a scene whose cost exceeds
// an even share of the SMs (total / SM count) runs on both blocks of a
// cluster, split = 2 splits every scene, split = 1 none.  The remaining scenes
// are paired in decreasing cost (neighbours, so the two blocks of a cluster
// finish together).  Jobs are ordered by decreasing time estimate: half the
// cost for a split scene, the larger cost for a pair.
static std::vector<int2> batch_jobs(const std::vector<long long>& cost, int num_sms, int split) {
  const int n = (int)cost.size();
  std::vector<int> ord(n);
  for (int i = 0; i < n; ++i) ord[i] = i;
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  long long total = 0;
  for (long long w : cost) total += w;
  const double share = (double)total / (num_sms > 0 ? num_sms : 1);
  std::vector<std::pair<double, int2>> jobs;
  int pending = -1;
  for (int i : ord) {
    const bool big = split == 2 || (split == 0 && (double)cost[i] > share);
    if (big) {
      jobs.push_back({0.5 * (double)cost[i], make_int2(i, -2)});
    } else if (pending < 0) {
      pending = i;
    } else {
      jobs.push_back({(double)cost[pending], make_int2(pending, i)});
      pending = -1;
    }
  }
  if (pending >= 0) jobs.push_back({(double)cost[pending], make_int2(pending, -1)});
  std::stable_sort(jobs.begin(), jobs.end(),
                   [](const std::pair<double, int2>& a, const std::pair<double, int2>& b) { return a.first > b.first; });
  std::vector<int2> out(jobs.size());
  for (size_t j = 0; j < jobs.size(); ++j) out[j] = jobs[j].second;
  return out;
}

// measured block size per (device, batch size class)
static std::mutex g_tune_mu;
static std::map<std::pair<int, long long>, int> g_tune;

static int batched_solve(int n, const qp_ctx_t* ctxs, const qp_state* const* st, const double* const* rhs,
                         double* const* dx, const qp_batch_opts* o, qp_solve_stats* stats, int* used) {
  qp_ctx* c0 = ctxs[0];
  std::vector<BatchScene> tab(n);
  std::vector<long long> cost(n);
  long long work = 0;
  for (int i = 0; i < n; ++i) {
    qp_ctx* c = ctxs[i];
    QP_REQUIRE(c, QP_INVALID_ARG, "newton_solve_batched: null context");
    QP_REQUIRE(c->device == c0->device, QP_INVALID_ARG, "newton_solve_batched: contexts on different devices");
    QP_REQUIRE(c->have_contacts, QP_NOT_READY, "newton_solve_batched: a context has no contacts");
    QP_REQUIRE(rhs[i] && dx[i] && rhs[i] != dx[i], QP_INVALID_ARG, "newton_solve_batched: null or aliased vectors");
    if (st && st[i]) QP_REQUIRE(st[i]->gamma && st[i]->lambda, QP_INVALID_ARG, "newton_solve_batched: bad state");
    BatchScene& b = tab[i];
    b.s64 = view64(c, true);
    b.s32 = view32(c, true);
    b.H64 = c->H.as<double>();
    b.H32 = c->H32.as<float>();
    b.dinv64 = c->dinv.as<double>();
    b.dinv32 = c->dinv32.as<float>();
    b.gamma = (st && st[i]) ? st[i]->gamma : nullptr;
    b.lambda = (st && st[i]) ? st[i]->lambda : nullptr;
    b.mu = c->mu;
    b.rhs = rhs[i];
    b.dx = dx[i];
    const size_t P = (size_t)c->P;
    double* w64 = static_cast<double*>(c->batch64.ensure(2 * P * sizeof(double)));
    b.r64 = w64;
    b.q64 = w64 + P;
    b.v32 = static_cast<float*>(c->batch32.ensure(7 * P * sizeof(float)));
    b.P = c->P;
    b.nrow = c->slots * c->Nc;
    cost[i] = (long long)c->P + c->Nc;
    work += c->P;
  }
  QP_REQUIRE(o->split >= 0 && o->split <= 2, QP_INVALID_ARG, "newton_solve_batched: split must be 0, 1 or 2");
  QP_REQUIRE(o->qtt_tile >= 0 && o->qtt_tile <= 2, QP_INVALID_ARG, "newton_solve_batched: qtt_tile must be 0, 1 or 2");
  // per-scene QTT preconditioners (FP32 or BF16 copies of the cores)
  const qp_dtype cdt = o->core_dtype == QP_BF16 ? QP_BF16 : QP_F32;
  std::vector<QttDev> qdev;
  std::vector<int> qidx(n, -1);
  for (int i = 0; o->precond && i < n; ++i) {
    qp_qtt* X = o->precond[i];
    if (!X) continue;
    qp_ctx* c = ctxs[i];
    QP_REQUIRE(X->d == c->L && X->d <= 64, QP_INVALID_ARG, "newton_solve_batched: preconditioner size does not match 2^L");
    qtt_prepare_copies(c, X, cdt);
    QttDev q;
    q.d = X->d;
    q.rmax = 1;
    for (int k = 0; k <= X->d; ++k) {
      q.ranks[k] = X->ranks[k];
      q.off[k] = X->offset[k];
      if (X->ranks[k] > q.rmax) q.rmax = X->ranks[k];
    }
    q.cores = cdt == QP_BF16 ? (const void*)X->cores16 : (const void*)X->cores32;
    BatchScene& b = tab[i];
    b.qw = static_cast<float*>(c->batch_qw.ensure(2 * (size_t)c->P * q.rmax * sizeof(float)));
    b.qtt_scaled = X->scaled;
    b.qtt_bf16 = cdt == QP_BF16 ? 1 : 0;
    qidx[i] = (int)qdev.size();
    qdev.push_back(q);
  }
  const bool use_qtt = !qdev.empty();
  const std::vector<int2> jobs = batch_jobs(cost, c0->num_sms, o->split);
  const int nj = (int)jobs.size();
  // table, jobs, outputs and QTT views in one device buffer of ctxs[0]
  auto up = [](size_t b) { return ((b + 255) / 256) * 256; };
  const size_t tb = sizeof(BatchScene) * n, ob = sizeof(int2) * n, rb = sizeof(BatchOut) * n;
  const size_t qb = sizeof(QttDev) * qdev.size();
  char* buf = static_cast<char*>(c0->batch_table.ensure(up(tb) + up(ob) + up(rb) + qb + 256));
  BatchScene* dtab = reinterpret_cast<BatchScene*>(buf);
  int2* djobs = reinterpret_cast<int2*>(buf + up(tb));
  BatchOut* dout = reinterpret_cast<BatchOut*>(buf + up(tb) + up(ob));
  QttDev* dq = reinterpret_cast<QttDev*>(buf + up(tb) + up(ob) + up(rb));
  for (int i = 0; i < n; ++i) tab[i].qtt = qidx[i] >= 0 ? dq + qidx[i] : nullptr;
  // the other contexts' pending work (assembly, states) comes first
  for (int i = 0; i < n; ++i)
    if (ctxs[i] != c0) {
      QP_CUDA(cudaEventRecord(ctxs[i]->ev0, ctxs[i]->stream));
      QP_CUDA(cudaStreamWaitEvent(c0->stream, ctxs[i]->ev0, 0));
    }
  QP_CUDA(cudaMemcpyAsync(dtab, tab.data(), tb, cudaMemcpyHostToDevice, c0->stream));
  QP_CUDA(cudaMemcpyAsync(djobs, jobs.data(), sizeof(int2) * nj, cudaMemcpyHostToDevice, c0->stream));
  if (use_qtt) QP_CUDA(cudaMemcpyAsync(dq, qdev.data(), qb, cudaMemcpyHostToDevice, c0->stream));
  auto tiles_for = [&](int threads) -> unsigned {
    if (!use_qtt) return 0u;
    if (o->qtt_tile == 1) return 0u;
    if (o->qtt_tile == 2) return 7u;
    return batch_tile_mask(c0, threads);
  };
  int nt = o->block_threads;
  QP_REQUIRE(nt == 0 || nt == 128 || nt == 256 || nt == 512 || nt == 1024, QP_INVALID_ARG,
             "newton_solve_batched: block_threads must be 0, 128, 256, 512 or 1024");
  if (nt == 0) {
    long long cls = 1;
    while (cls < work / n) cls <<= 1;
    const auto key = std::make_pair(c0->device, ((cls * 4096 + (n < 4096 ? n / 64 : 64)) * 4 + o->split) * 2 +
                                                    (use_qtt ? 1 : 0));
    {
      std::lock_guard<std::mutex> lock(g_tune_mu);
      auto it = g_tune.find(key);
      if (it != g_tune.end()) nt = it->second;
    }
    if (nt == 0) {
      float best = 1e30f;
      for (int cand : {256, 512, 1024}) {
        const unsigned tm = tiles_for(cand);
        QP_CUDA(cudaEventRecord(c0->ev0, c0->stream));
        launch_batched(c0, cand, nj, dtab, djobs, o, dout, use_qtt, tm);
        QP_CUDA(cudaEventRecord(c0->ev1, c0->stream));
        QP_CUDA(cudaEventSynchronize(c0->ev1));
        float ms = 0;
        QP_CUDA(cudaEventElapsedTime(&ms, c0->ev0, c0->ev1));
        if (ms < best) {
          best = ms;
          nt = cand;
        }
      }
      std::lock_guard<std::mutex> lock(g_tune_mu);
      g_tune[key] = nt;
    }
  }
  const unsigned tm = tiles_for(nt);
  QP_CUDA(cudaEventRecord(c0->ev0, c0->stream));
  launch_batched(c0, nt, nj, dtab, djobs, o, dout, use_qtt, tm);
  QP_CUDA(cudaEventRecord(c0->ev1, c0->stream));
  std::vector<BatchOut> res(n);
  QP_CUDA(cudaMemcpyAsync(res.data(), dout, rb, cudaMemcpyDeviceToHost, c0->stream));
  QP_CUDA(cudaStreamSynchronize(c0->stream));
  float ms = 0;
  QP_CUDA(cudaEventElapsedTime(&ms, c0->ev0, c0->ev1));
  // later work on the other contexts waits for the batch
  for (int i = 0; i < n; ++i)
    if (ctxs[i] != c0) QP_CUDA(cudaStreamWaitEvent(ctxs[i]->stream, c0->ev1, 0));
  int rc = QP_OK;
  for (int i = 0; i < n; ++i) {
    const int code = res[i].status == 0 ? QP_OK : (res[i].status == 2 ? QP_BREAKDOWN : QP_NOT_CONVERGED);
    if (stats) {
      stats[i].status = code;
      stats[i].iters = res[i].iters;
      stats[i].outer = res[i].outer;
      stats[i].rel_res = res[i].rel;
      stats[i].ms = ms;
      stats[i].fallback = res[i].fallback;
    }
    if (rc == QP_OK && code != QP_OK) rc = code;
  }
  if (used) *used = nt;
  return rc;
}

}  // namespace qp

using namespace qp;

#define API_BEGIN(c)            \
  if (!(c)) return QP_INVALID_ARG; \
  try {                         \
    QP_CUDA(cudaSetDevice((c)->device));
#define API_END(c)               \
  }                              \
  catch (const qp::Error& e) {   \
    qp::set_error((c), e);       \
    return e.code;               \
  }                              \
  return QP_OK;

extern "C" {

int pdip_init(qp_ctx_t c, qp_state* st, double gn0) {
  API_BEGIN(c)
  check_ready(c, st);
  QP_REQUIRE(gn0 > 0, QP_INVALID_ARG, "pdip_init: gn0 must be > 0");
  k_pdip_init<<<c->num_sms * 4, 256, 0, c->stream>>>(c->Nc, c->slots, c->P, c->mu, gn0, st->gamma, st->lambda);
  QP_CUDA(cudaGetLastError());
  st->t = 1.0;
  API_END(c)
}

int ccp_advance(qp_ctx_t c, const qp_scene* sc, const qp_state* st, double* pos_out, double* vel_out,
                double* omega_out) {
  API_BEGIN(c)
  QP_REQUIRE(st, QP_INVALID_ARG, "ccp_advance: null state");
  check_ready(c, st);
  QP_REQUIRE(sc && sc->pos && sc->vel && sc->omega && pos_out && vel_out && omega_out, QP_INVALID_ARG,
             "ccp_advance: null scene array");
  QP_REQUIRE(sc->M == c->M, QP_INVALID_ARG, "ccp_advance: scene is not the one of the current contact set");
  if (c->M > 0) {
    SysView<double> s = view64(c, false);
    int grid = (c->M + 255) / 256;
    if (grid > c->num_sms * 8) grid = c->num_sms * 8;
    k_advance<<<grid, 256, 0, c->stream>>>(s, st->gamma, sc->pos, sc->vel, sc->omega, sc->dt, sc->gravity[0],
                                           sc->gravity[1], sc->gravity[2], pos_out, vel_out, omega_out);
    QP_CUDA(cudaGetLastError());
  }
  API_END(c)
}

int newton_apply(qp_ctx_t c, const qp_state* st, const void* x, void* y, qp_dtype dt) {
  API_BEGIN(c)
  check_ready(c, st);
  QP_REQUIRE(x && y && x != y, QP_INVALID_ARG, "newton_apply: null or aliased vectors");
  QP_REQUIRE(dt == QP_F64 || dt == QP_F32, QP_INVALID_ARG, "newton_apply: dtype must be QP_F64 or QP_F32");
  if (st) QP_REQUIRE(st->gamma && st->lambda, QP_INVALID_ARG, "newton_apply: state with null gamma/lambda");
  if (dt == QP_F64) {
    // FP64: two launches (the body gather once per body, then the contacts with
    // their Schur blocks formed in registers); the one-launch form gathers the
    // border bodies of every block again, which costs more on the narrow FP64 pipe
    const SysView<double> s64 = view64(c, false);
    if (c->M > 0)
      k_body_gather_lanes<double, QP_APPLY_LANES><<<ceil_div((long long)c->M * QP_APPLY_LANES, 256), 256, 0,
                                                   c->stream>>>(s64, static_cast<const double*>(x));
    k_contact_apply_h<<<c->num_sms * 8, 256, 0, c->stream>>>(s64, static_cast<const double*>(x), static_cast<double*>(y),
                                                             st ? st->gamma : nullptr, st ? st->lambda : nullptr, c->mu);
    QP_CUDA(cudaGetLastError());
  } else {
    // FP32: one launch, the body intermediates in shared memory, the Schur blocks in registers
    launch_apply_one<float>(c, view32(c, false), static_cast<const float*>(x), static_cast<float*>(y), st);
  }
  API_END(c)
}

int newton_rhs(qp_ctx_t c, const qp_state* st, double* rhs) {
  API_BEGIN(c)
  check_ready(c, st);
  QP_REQUIRE(st && rhs, QP_INVALID_ARG, "newton_rhs: null state or rhs");
  pdip_pre(c, const_cast<qp_state*>(st), 0, nullptr);
  QP_CUDA(cudaMemcpyAsync(rhs, c->v64[1].p, (size_t)c->P * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  DevCtl h = read_ctl(c);
  QP_REQUIRE(h.err == 0, h.err, "newton_rhs: device wait expired");
  const_cast<qp_state*>(st)->t = h.scal[S_T];
  API_END(c)
}

int newton_solve(qp_ctx_t c, const qp_state* st, const double* rhs, double* dx, const qp_solve_opts* o,
                 qp_solve_stats* stats) {
  API_BEGIN(c)
  check_ready(c, st);
  QP_REQUIRE(rhs && dx && rhs != dx, QP_INVALID_ARG, "newton_solve: null or aliased vectors");
  if (st) launch_schur_blocks(c, st->gamma, st->lambda);
  else QP_CUDA(cudaMemsetAsync(c->H.p, 0, 6 * (size_t)(c->Nc > 0 ? c->Nc : 1) * sizeof(double), c->stream));
  if (!st) QP_CUDA(cudaMemsetAsync(c->H32.p, 0, 6 * (size_t)(c->Nc > 0 ? c->Nc : 1) * sizeof(float), c->stream));
  qp_solve_stats s = solve(c, rhs, dx, o);
  if (stats) *stats = s;
  if (s.status == QP_TIMEOUT) throw Error{QP_TIMEOUT, "newton_solve: device barrier wait expired"};
  return s.status;
  API_END(c)
}

int newton_batch_plan(int n, const long long* cost_host, int num_sms, int split, int* jobs_host, int* njobs) {
  if (n < 0 || (n > 0 && (!cost_host || !jobs_host)) || !njobs || split < 0 || split > 2) return QP_INVALID_ARG;
  for (int i = 0; i < n; ++i)
    if (cost_host[i] < 0) return QP_INVALID_ARG;
  const std::vector<int2> jobs = batch_jobs(std::vector<long long>(cost_host, cost_host + n), num_sms, split);
  for (size_t j = 0; j < jobs.size(); ++j) {
    jobs_host[2 * j] = jobs[j].x;
    jobs_host[2 * j + 1] = jobs[j].y;
  }
  *njobs = (int)jobs.size();
  return QP_OK;
}

int newton_solve_batched(int n, const qp_ctx_t* ctxs, const qp_state* const* st, const double* const* rhs,
                         double* const* dx, const qp_batch_opts* o, qp_solve_stats* stats, int* used) {
  if (n < 1 || !ctxs || !ctxs[0] || !rhs || !dx || !o) return QP_INVALID_ARG;
  qp_ctx* c = ctxs[0];
  API_BEGIN(c)
  QP_REQUIRE(o->tol > 0 && o->maxit > 0, QP_INVALID_ARG, "newton_solve_batched: tol > 0 and maxit > 0 required");
  return batched_solve(n, ctxs, st, rhs, dx, o, stats, used);
  API_END(c)
}

int newton_batch_qtt_tiles(qp_ctx_t c, int block_threads, int* tiles) {
  if (!c || !tiles) return QP_INVALID_ARG;
  API_BEGIN(c)
  QP_REQUIRE(block_threads == 128 || block_threads == 256 || block_threads == 512 || block_threads == 1024,
             QP_INVALID_ARG, "newton_batch_qtt_tiles: block_threads must be 128, 256, 512 or 1024");
  QP_CUDA(cudaSetDevice(c->device));
  const unsigned m = batch_tile_mask(c, block_threads);
  for (int k = 0; k < 3; ++k) tiles[k] = ((m >> k) & 1u) ? 2 : 1;
  tiles[3] = 1;
  API_END(c)
}

int qp_selftest_barrier(qp_ctx_t c, long long budget, int absent_block, int* device_status) {
  API_BEGIN(c)
  QP_REQUIRE(budget > 0 && budget <= BARRIER_BUDGET && device_status, QP_INVALID_ARG,
             "qp_selftest_barrier: need 0 < budget <= the default budget and a status pointer");
  QP_REQUIRE(absent_block < c->num_sms, QP_INVALID_ARG, "qp_selftest_barrier: absent block out of range");
  ensure_partial(c);
  reset_ctl(c);
  DevCtl* ctl = c->ctl.as<DevCtl>();
  void* args[] = {&ctl, &budget, &absent_block};
  QP_CUDA(cudaLaunchCooperativeKernel((const void*)k_barrier_probe, dim3(c->num_sms), dim3(128), args, 0, c->stream));
  DevCtl h = read_ctl(c);
  *device_status = h.err;
  API_END(c)
}

int pdip_measure(qp_ctx_t c, const qp_state* st, double* eta, double* rdual) {
  API_BEGIN(c)
  check_ready(c, st);
  pdip_pre(c, const_cast<qp_state*>(st), 1, nullptr);
  DevCtl h = read_ctl(c);
  QP_REQUIRE(h.err == 0, h.err, "pdip_measure: device wait expired");
  if (eta) *eta = h.scal[S_ETA];
  if (rdual) *rdual = h.scal[S_RDUAL];
  API_END(c)
}

int pdip_step(qp_ctx_t c, qp_state* st, const qp_pdip_opts* o, qp_pdip_stats* stats) {
  API_BEGIN(c)
  check_ready(c, st);
  QP_REQUIRE(o, QP_INVALID_ARG, "pdip_step: null options");
  qp_pdip_stats out{};
  pdip_pre(c, st, 0, o);
  DevCtl h = read_ctl(c);
  QP_REQUIRE(h.err == 0, h.err, "pdip_step: device wait expired (pre)");
  out.eta = h.scal[S_ETA];
  out.t = h.scal[S_T];
  out.r_dual = h.scal[S_RDUAL];
  out.r_t = h.scal[S_RT];
  st->t = out.t;
  qp_solve_opts so = o->solve;
  if (o->qtt_refresh && so.precond == QP_QTT_PCG) {
    // compress S_k and invert it, warm-started from the previous inverse
    // (Sec. 3.3: S_{k+1} = S_k + L_k with L_k block diagonal)
    QP_CUDA(cudaEventRecord(c->ev0, c->stream));
    // compress the Jacobi-scaled Schur matrix D^-1/2 S D^-1/2 (unit diagonal, dummy
    // rows included), so that relative TT accuracy is not dominated by a few rows
    double* rs = static_cast<double*>(c->dm[13].ensure((size_t)c->P * sizeof(double)));
    launch_rowscale(c, rs);
    qtt_t S = compress_impl(c, true, o->qtt_eps, o->qtt_rmax, rs);
    int rc = QP_OK;
    qtt_t warm = so.X ? so.X : c->last_inv;
    if (warm && warm->d != S->d) warm = nullptr;
    qtt_t X = nullptr;
    rc = qtt_inverse(c, S, o->qtt_eps, o->qtt_rmax, warm ? 2 : 4, warm, &X);
    qtt_free(c, S);
    if (rc != QP_OK) throw Error{rc, "pdip_step: qtt_inverse failed: " + c->last_error};
    if (c->last_inv) qtt_free(c, c->last_inv);
    c->last_inv = X;
    QP_CUDA(cudaEventRecord(c->ev1, c->stream));
    QP_CUDA(cudaEventSynchronize(c->ev1));
    float ms = 0;
    QP_CUDA(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
    out.ms_refresh = ms;
    so.X = X;
  } else if (so.precond == QP_QTT_PCG && !so.X) {
    // no refresh and no X: reuse the inverse of the context's last refresh
    QP_REQUIRE(c->last_inv && c->last_inv->d == c->L, QP_INVALID_ARG,
               "pdip_step: QTT preconditioner without X, and no refreshed inverse of this size to reuse");
    so.X = c->last_inv;
  }
  PdipArgs A = pdip_args(c, st);
  A.nu = o->nu;
  A.alpha = o->alpha;
  A.beta = o->beta;
  A.step_frac = o->step_frac;
  A.max_halvings = o->max_halvings;
  // H blocks were built by the pre-step
  out.solve = solve(c, A.rhs, A.dg, &so);
  if (out.solve.status == QP_TIMEOUT) throw Error{QP_TIMEOUT, "pdip_step: Krylov barrier wait expired"};
  // keep t in the control block for the post-step
  reset_ctl(c);
  QP_CUDA(cudaMemcpyAsync(&c->ctl.as<DevCtl>()->scal[S_T], &out.t, sizeof(double), cudaMemcpyHostToDevice,
                          c->stream));
  QP_CUDA(cudaMemcpyAsync(&c->ctl.as<DevCtl>()->scal[S_RT], &out.r_t, sizeof(double), cudaMemcpyHostToDevice,
                          c->stream));
  int grid = coop_grid(c, k_pdip_post);
  coop_launch(c, k_pdip_post, grid, A);
  h = read_ctl(c);
  QP_REQUIRE(h.err == 0, h.err, "pdip_step: device wait expired (post)");
  out.s = h.scal[S_S];
  out.halvings = h.halvings;
  out.status = h.iters != 0 ? h.iters : out.solve.status;
  if (stats) *stats = out;
  return out.status;
  API_END(c)
}

int pdip_solve(qp_ctx_t c, qp_state* st, const qp_pdip_opts* o, double gap_tol, double dual_tol, int max_iter,
               qp_pdip_stats* stats, int* iters) {
  if (!c || !st || !o || max_iter < 0 || !(gap_tol >= 0.0) || !(dual_tol >= 0.0)) return QP_INVALID_ARG;
  qp_pdip_stats last{};
  int k = 0, rc = QP_OK;
  for (;; ++k) {
    double eta = 0.0, rd = 0.0;
    rc = pdip_measure(c, st, &eta, &rd);
    if (rc != QP_OK) break;
    last.eta = eta;
    last.r_dual = rd;
    if (eta <= gap_tol && rd <= dual_tol) break;
    if (k == max_iter) {
      rc = QP_NOT_CONVERGED;
      break;
    }
    rc = pdip_step(c, st, o, &last);
    if (rc != QP_OK && rc != QP_NOT_CONVERGED) {
      ++k;
      break;
    }
    rc = QP_OK;
  }
  last.status = rc;
  if (stats) *stats = last;
  if (iters) *iters = k;
  return rc;
}

}  // extern "C"
