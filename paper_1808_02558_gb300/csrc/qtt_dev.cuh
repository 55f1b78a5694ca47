// Device-side QTT mat-vec step (Sec. 3.2: contract one core at a time), shared
// by the standalone qtt_apply kernels and the persistent PCG preconditioner.
//
// Layout of the intermediate after contracting cores k+1..d (1-based k):
//   Z_{k+1}[J][b][I]   J = (j_1..j_k) (k bits), b < r_k, I = (i_{k+1}..i_d)
// flattened as ((J * r_k) + b) * 2^(d-k) + I.  Z_{d+1} = x (r_d = 1) and
// Z_1 = y (r_0 = 1).  Step k maps Z_{k+1} to Z_k:
//   Z_k[J'][a][i*2^(d-k) + I] = sum_{j,b} G_k(a, i, j, b) Z_{k+1}[2J'+j][b][I].
// One work item is a column (J', I); it produces the 2 r_{k-1} outputs of that
// column from the 2 r_k inputs, so every input value is read once.
#pragma once

#include <cuda_bf16.h>

namespace qp {

template <class TC> __device__ __forceinline__ float core_f(const TC* p, long long i);
template <> __device__ __forceinline__ float core_f<float>(const float* p, long long i) { return __ldg(p + i); }
template <> __device__ __forceinline__ float core_f<__nv_bfloat16>(const __nv_bfloat16* p, long long i) {
  return __bfloat162float(p[i]);
}

struct QttDev {
  int d;
  int rmax;
  int ranks[65];            // r_0..r_d
  long long off[65];        // value offset of each core
  const void* cores;        // typed by the caller: double / float / bf16
};

constexpr int QTT_MAX_IN = 128;  // 2 * max rank handled by the register path

// Column-per-thread step for small ranks (2 r_k <= QTT_MAX_IN inputs held in
// registers is not possible for runtime sizes, so inputs are re-read from L1).
// TV: vector type, TA: accumulation type, TC: core type.
template <class TV, class TA, class TC>
__device__ __forceinline__ void qtt_step_item(const QttDev& q, int k, const TV* in, TV* out, long long item) {
  // k is 1-based core index
  const int d = q.d;
  const int r0 = q.ranks[k - 1], r1 = q.ranks[k];
  const int lowbits = d - k;                      // bits of I
  const long long nI = 1LL << lowbits;
  const long long I = item & (nI - 1);
  const long long Jp = item >> lowbits;           // J' (k-1 bits)
  const TC* G = static_cast<const TC*>(q.cores) + q.off[k - 1];
  const TV* in0 = in + ((2 * Jp) * r1) * nI + I;       // j = 0
  const TV* in1 = in + ((2 * Jp + 1) * r1) * nI + I;   // j = 1
  TV* o = out + (Jp * r0) * (2 * nI) + I;
  for (int a = 0; a < r0; ++a) {
    TA acc0 = 0, acc1 = 0;  // i = 0, 1
    const TC* Ga = G + (long long)a * 4 * r1;       // G(a, i, j, b) at ((a*2+i)*2+j)*r1+b
    for (int b = 0; b < r1; ++b) {
      TA v0 = (TA)in0[(long long)b * nI];
      TA v1 = (TA)in1[(long long)b * nI];
      TA g00, g01, g10, g11;
      if constexpr (sizeof(TC) == 8) {
        g00 = (TA)Ga[b];
        g01 = (TA)Ga[r1 + b];
        g10 = (TA)Ga[2 * r1 + b];
        g11 = (TA)Ga[3 * r1 + b];
      } else {
        g00 = (TA)core_f<TC>(Ga, b);
        g01 = (TA)core_f<TC>(Ga, r1 + b);
        g10 = (TA)core_f<TC>(Ga, 2 * r1 + b);
        g11 = (TA)core_f<TC>(Ga, 3 * r1 + b);
      }
      acc0 += g00 * v0 + g01 * v1;
      acc1 += g10 * v0 + g11 * v1;
    }
    o[(long long)a * 2 * nI] = (TV)acc0;
    o[(long long)a * 2 * nI + nI] = (TV)acc1;
  }
}

// Same step with the 2 r_k inputs of the column held in registers (r_k <= R):
// each input is loaded once, each core value once per output row.
template <int R, class TV, class TA, class TC>
__device__ __forceinline__ void qtt_step_item_reg(const QttDev& q, int k, const TV* in, TV* out, long long item) {
  const int d = q.d;
  const int r0 = q.ranks[k - 1], r1 = q.ranks[k];
  const int lowbits = d - k;
  const long long nI = 1LL << lowbits;
  const long long I = item & (nI - 1);
  const long long Jp = item >> lowbits;
  const TC* G = static_cast<const TC*>(q.cores) + q.off[k - 1];
  const TV* in0 = in + ((2 * Jp) * r1) * nI + I;
  const TV* in1 = in + ((2 * Jp + 1) * r1) * nI + I;
  TA v0[R], v1[R];
#pragma unroll
  for (int b = 0; b < R; ++b) {
    v0[b] = b < r1 ? (TA)in0[(long long)b * nI] : TA(0);
    v1[b] = b < r1 ? (TA)in1[(long long)b * nI] : TA(0);
  }
  TV* o = out + (Jp * r0) * (2 * nI) + I;
  for (int a = 0; a < r0; ++a) {
    const TC* Ga = G + (long long)a * 4 * r1;
    TA acc0 = 0, acc1 = 0;
#pragma unroll
    for (int b = 0; b < R; ++b) {
      if (b < r1) {
        TA g00, g01, g10, g11;
        if constexpr (sizeof(TC) == 8) {
          g00 = (TA)__ldg(Ga + b);
          g01 = (TA)__ldg(Ga + r1 + b);
          g10 = (TA)__ldg(Ga + 2 * r1 + b);
          g11 = (TA)__ldg(Ga + 3 * r1 + b);
        } else {
          g00 = (TA)core_f<TC>(Ga, b);
          g01 = (TA)core_f<TC>(Ga, r1 + b);
          g10 = (TA)core_f<TC>(Ga, 2 * r1 + b);
          g11 = (TA)core_f<TC>(Ga, 3 * r1 + b);
        }
        acc0 += g00 * v0[b] + g01 * v1[b];
        acc1 += g10 * v0[b] + g11 * v1[b];
      }
    }
    o[(long long)a * 2 * nI] = (TV)acc0;
    o[(long long)a * 2 * nI + nI] = (TV)acc1;
  }
}

// Dispatch on the input rank of core k.
template <class TV, class TA, class TC>
__device__ __forceinline__ void qtt_step_any(const QttDev& q, int k, const TV* in, TV* out, long long item) {
  const int r1 = q.ranks[k];
  if (r1 <= 4) qtt_step_item_reg<4, TV, TA, TC>(q, k, in, out, item);
  else if (r1 <= 8) qtt_step_item_reg<8, TV, TA, TC>(q, k, in, out, item);
  else if (r1 <= 16) qtt_step_item_reg<16, TV, TA, TC>(q, k, in, out, item);
  else if (r1 <= 32) qtt_step_item_reg<32, TV, TA, TC>(q, k, in, out, item);
  else qtt_step_item<TV, TA, TC>(q, k, in, out, item);
}

// Block-level step: the core (converted to TA) is staged in shared memory once
// per block, and each thread computes two columns (items it and it + stride),
// so every core value read from shared memory feeds two columns.  All threads of
// the block must call it (it synchronises).  gc: shared buffer of at least
// r_{k-1} * 4 * r_k values.  Requires r_k <= R.
template <int R, class TV, class TA, class TC>
__device__ __forceinline__ void qtt_step_block(const QttDev& q, int k, const TV* in, TV* out, long long items,
                                               TA* gc, long long first, long long stride) {
  const int d = q.d;
  const int r0 = q.ranks[k - 1], r1 = q.ranks[k];
  const TC* G = static_cast<const TC*>(q.cores) + q.off[k - 1];
  const int ncore = r0 * 4 * r1;
  for (int i = threadIdx.x; i < ncore; i += blockDim.x) {
    if constexpr (sizeof(TC) == 8) gc[i] = (TA)G[i];
    else gc[i] = (TA)core_f<TC>(G, i);
  }
  __syncthreads();
  const int lowbits = d - k;
  const long long nI = 1LL << lowbits;
  for (long long it = first; it < items; it += 2 * stride) {
    const long long it2 = it + stride;
    const bool two = it2 < items;
    TA v0[R], v1[R], u0[R], u1[R];
    const long long I = it & (nI - 1), Jp = it >> lowbits;
    const long long I2 = it2 & (nI - 1), Jp2 = it2 >> lowbits;
    const TV* a0 = in + ((2 * Jp) * r1) * nI + I;
    const TV* a1 = in + ((2 * Jp + 1) * r1) * nI + I;
    const TV* b0 = in + ((2 * Jp2) * r1) * nI + I2;
    const TV* b1 = in + ((2 * Jp2 + 1) * r1) * nI + I2;
#pragma unroll
    for (int b = 0; b < R; ++b) {
      const bool ok = b < r1;
      v0[b] = ok ? (TA)a0[(long long)b * nI] : TA(0);
      v1[b] = ok ? (TA)a1[(long long)b * nI] : TA(0);
      u0[b] = (ok && two) ? (TA)b0[(long long)b * nI] : TA(0);
      u1[b] = (ok && two) ? (TA)b1[(long long)b * nI] : TA(0);
    }
    TV* o = out + (Jp * r0) * (2 * nI) + I;
    TV* o2 = out + (Jp2 * r0) * (2 * nI) + I2;
    for (int a = 0; a < r0; ++a) {
      const TA* Ga = gc + a * 4 * r1;
      TA p0 = 0, p1 = 0, q0 = 0, q1 = 0;
#pragma unroll
      for (int b = 0; b < R; ++b) {
        if (b < r1) {
          const TA g00 = Ga[b], g01 = Ga[r1 + b], g10 = Ga[2 * r1 + b], g11 = Ga[3 * r1 + b];
          p0 += g00 * v0[b] + g01 * v1[b];
          p1 += g10 * v0[b] + g11 * v1[b];
          q0 += g00 * u0[b] + g01 * u1[b];
          q1 += g10 * u0[b] + g11 * u1[b];
        }
      }
      o[(long long)a * 2 * nI] = (TV)p0;
      o[(long long)a * 2 * nI + nI] = (TV)p1;
      if (two) {
        o2[(long long)a * 2 * nI] = (TV)q0;
        o2[(long long)a * 2 * nI + nI] = (TV)q1;
      }
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------- two cores per pass
// Steps k and k-1 fused: a column (J'', I), J'' = (j_1..j_{k-2}), I =
// (i_{k+1}..i_d), reads the 4 r_k inputs Z_{k+1}[4J''+2j_{k-1}+j_k][b][I],
// forms the 4 r_{k-1} values of Z_k in registers and writes the 4 r_{k-2}
// outputs Z_{k-1}[J''][c][(2 i_{k-1} + i_k) 2^(d-k) + I].  Each pass moves
// (r_k + r_{k-2}) N values instead of (r_k + 2 r_{k-1} + r_{k-2}) N.
// Both cores are staged in shared memory as one 4-vector (i, j) per rank pair:
// gk[a r_k + b] = G_k(a, ., ., b), gm[c r_{k-1} + a] = G_{k-1}(c, ., ., a).
template <class TA>
struct Quad {
  TA v[4];
};
template <>
struct Quad<float> {
  float4 q;
};
template <class TA>
__device__ __forceinline__ void quad_get(const Quad<TA>& g, TA& g00, TA& g01, TA& g10, TA& g11) {
  g00 = g.v[0]; g01 = g.v[1]; g10 = g.v[2]; g11 = g.v[3];
}
__device__ __forceinline__ void quad_get(const Quad<float>& g, float& g00, float& g01, float& g10, float& g11) {
  const float4 q = g.q;
  g00 = q.x; g01 = q.y; g10 = q.z; g11 = q.w;
}
template <class TA>
__device__ __forceinline__ void quad_set(Quad<TA>& g, TA g00, TA g01, TA g10, TA g11) {
  g.v[0] = g00; g.v[1] = g01; g.v[2] = g10; g.v[3] = g11;
}
__device__ __forceinline__ void quad_set(Quad<float>& g, float g00, float g01, float g10, float g11) {
  g.q = make_float4(g00, g01, g10, g11);
}

template <class TA, class TC>
__device__ __forceinline__ TA core_ta(const TC* G, long long i) {
  if constexpr (sizeof(TC) == 8) return (TA)G[i];
  else return (TA)core_f<TC>(G, i);
}

// Stage core kk (1-based) as quads: out[a * rin + b] = G_kk(a, ., ., b).
template <class TA, class TC>
__device__ __forceinline__ void stage_quads(const QttDev& q, int kk, Quad<TA>* out) {
  const int ro = q.ranks[kk - 1], ri = q.ranks[kk];
  const TC* G = static_cast<const TC*>(q.cores) + q.off[kk - 1];
  for (int t = threadIdx.x; t < ro * ri; t += blockDim.x) {
    const int a = t / ri, b = t - a * ri;
    const long long base = (long long)a * 4 * ri + b;
    quad_set(out[t], core_ta<TA, TC>(G, base), core_ta<TA, TC>(G, base + ri), core_ta<TA, TC>(G, base + 2 * ri),
             core_ta<TA, TC>(G, base + 3 * ri));
  }
}

// Requires r_k, r_{k-1} <= R and r_{k-1} r_k + r_{k-2} r_{k-1} <= gcap quads.
// All threads of the block call it (it synchronises).
template <int R, class TV, class TA, class TC>
__device__ __forceinline__ void qtt_step2_block(const QttDev& q, int k, const TV* in, TV* out, Quad<TA>* gq,
                                                long long first, long long stride) {
  const int d = q.d;
  const int r2 = q.ranks[k - 2], r0 = q.ranks[k - 1], r1 = q.ranks[k];
  Quad<TA>* gk = gq;
  Quad<TA>* gm = gq + r0 * r1;
  stage_quads<TA, TC>(q, k, gk);
  stage_quads<TA, TC>(q, k - 1, gm);
  __syncthreads();
  const int lowbits = d - k;
  const long long nI = 1LL << lowbits;
  const long long cols = 1LL << (d - 2);
  for (long long it = first; it < cols; it += stride) {
    const long long I = it & (nI - 1), J = it >> lowbits;
    // inputs v[2 j_{k-1} + j_k][b]
    TA v[4][R];
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) {
      const TV* src = in + ((4 * J + jj) * r1) * nI + I;
#pragma unroll
      for (int b = 0; b < R; ++b) v[jj][b] = b < r1 ? (TA)src[(long long)b * nI] : TA(0);
    }
    // step k: t[j_{k-1}][i_k][a]
    TA t[2][2][R];
#pragma unroll
    for (int a = 0; a < R; ++a) {
      TA s00 = 0, s01 = 0, s10 = 0, s11 = 0;  // [j_{k-1}][i_k]
      if (a < r0) {
#pragma unroll
        for (int b = 0; b < R; ++b) {
          if (b < r1) {
            TA g00, g01, g10, g11;  // G_k(a, i, j, b)
            quad_get(gk[a * r1 + b], g00, g01, g10, g11);
            s00 += g00 * v[0][b] + g01 * v[1][b];
            s01 += g10 * v[0][b] + g11 * v[1][b];
            s10 += g00 * v[2][b] + g01 * v[3][b];
            s11 += g10 * v[2][b] + g11 * v[3][b];
          }
        }
      }
      t[0][0][a] = s00;
      t[0][1][a] = s01;
      t[1][0][a] = s10;
      t[1][1][a] = s11;
    }
    // step k-1: outputs [c][2 i_{k-1} + i_k]
    TV* o = out + (J * r2) * (4 * nI) + I;
    for (int c = 0; c < r2; ++c) {
      TA y00 = 0, y01 = 0, y10 = 0, y11 = 0;  // [i_{k-1}][i_k]
#pragma unroll
      for (int a = 0; a < R; ++a) {
        if (a < r0) {
          TA g00, g01, g10, g11;  // G_{k-1}(c, i, j, a)
          quad_get(gm[c * r0 + a], g00, g01, g10, g11);
          y00 += g00 * t[0][0][a] + g01 * t[1][0][a];
          y01 += g00 * t[0][1][a] + g01 * t[1][1][a];
          y10 += g10 * t[0][0][a] + g11 * t[1][0][a];
          y11 += g10 * t[0][1][a] + g11 * t[1][1][a];
        }
      }
      TV* oc = o + (long long)c * 4 * nI;
      oc[0] = (TV)y00;
      oc[nI] = (TV)y01;
      oc[2 * nI] = (TV)y10;
      oc[3 * nI] = (TV)y11;
    }
  }
  __syncthreads();
}

// Rank bound of the fused pass for cores k, k-1 (0: not fusable).  Only FP32
// accumulation is fused: FP64 intermediates of rank 12 do not fit the registers.
template <class TA>
__host__ __device__ __forceinline__ int qtt_fuse_bound(const QttDev& q, int k, int gcap_quads) {
  if (sizeof(TA) != 4 || k < 2) return 0;
  const int r2 = q.ranks[k - 2], r0 = q.ranks[k - 1], r1 = q.ranks[k];
  if (r0 * r1 + r2 * r0 > gcap_quads) return 0;
  const int r = r0 > r1 ? r0 : r1;
  if (r <= 4) return 4;
  if (r <= 8) return 8;
  if (r <= 10) return 10;  // the paper's operating rank
  if (r <= 12) return 12;
  return 0;
}

// Grid-stride fused pass with the block dispatch on the rank bound.
template <class TV, class TA, class TC>
__device__ __forceinline__ void qtt_step2_grid(const QttDev& q, int k, const TV* in, TV* out, Quad<TA>* gq,
                                               int bound) {
  const long long first = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long stride = (long long)gridDim.x * blockDim.x;
  if constexpr (sizeof(TA) == 4) {
    if (bound == 4) qtt_step2_block<4, TV, TA, TC>(q, k, in, out, gq, first, stride);
    else if (bound == 8) qtt_step2_block<8, TV, TA, TC>(q, k, in, out, gq, first, stride);
    else if (bound == 10) qtt_step2_block<10, TV, TA, TC>(q, k, in, out, gq, first, stride);
    else qtt_step2_block<12, TV, TA, TC>(q, k, in, out, gq, first, stride);
  }
}

// Block-level dispatch on the input rank; falls back to the per-item step
// (cores read from global memory) for ranks above 32 or cores larger than gcap.
template <class TV, class TA, class TC>
__device__ __forceinline__ void qtt_step_grid(const QttDev& q, int k, const TV* in, TV* out, long long items,
                                              TA* gc, int gcap) {
  const int r0 = q.ranks[k - 1], r1 = q.ranks[k];
  const long long first = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long stride = (long long)gridDim.x * blockDim.x;
  if (r0 * 4 * r1 <= gcap) {
    if (r1 <= 8) return qtt_step_block<8, TV, TA, TC>(q, k, in, out, items, gc, first, stride);
    if (r1 <= 16) return qtt_step_block<16, TV, TA, TC>(q, k, in, out, items, gc, first, stride);
  }
  for (long long it = first; it < items; it += stride) qtt_step_any<TV, TA, TC>(q, k, in, out, it);
}

}  // namespace qp
