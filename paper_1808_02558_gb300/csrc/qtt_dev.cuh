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

}  // namespace qp
