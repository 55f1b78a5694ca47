// Tensor-core step of the QTT mat-vec (Sec. 3.2: the product is formed one core
// at a time) for cores whose ranks on both sides are at most 64.
//
// With the intermediate layout of qtt_dev.cuh, contracting core k (ranks
// r0 = r_{k-1}, r1 = r_k, nI = 2^(d-k)) is, for every column item g = (J', I),
//   out[(J' 2 r0 + m) nI + I] = sum_kk G[m][kk] in[(2 J' r1 + kk) nI + I],
// with m = 2a + i < 2 r0 and kk = j r1 + b < 2 r1, G[m][kk] = G_k(a, i, j, b):
// the stored core already is this (2 r0) x (2 r1) matrix, row-major.  So the
// step is the product D = A B^T with A = G (2 r0 rows, zero-padded to 128) and
// B = a tile of NT consecutive items (rows) by their 2 r1 inputs (K, zero-padded
// to whole 32-column chunks) -- a dense contraction once r0 r1 is large.
//
// The tensor cores multiply TF32 values (FP32 with 10 mantissa bits).  BF16
// cores are exact in TF32.  The FP32 vector values are split x = x_hi + x_lo,
// x_hi the TF32 part, and D = G x_hi + G x_lo: each product is then good to
// about 2^-21.  FP32 cores are split the same way and G_lo x_hi is added
// (G_lo x_lo lies below FP32 rounding).  The accumulator itself rounds less
// carefully than an FP32 FMA chain: measured against FP64, a whole apply ends
// about 3e-6 (BF16 cores, d = 8) to 1.2e-5 (FP32 cores, d = 12) of the largest
// entry off, against about 4e-7 for the CUDA-core steps -- far below TF32's
// 2^-11 and below the BF16 cores' own 2^-9.
//
// One block per SM walks over its tiles with four kinds of warps linked by
// mbarriers, so that copies, splits, products and stores of successive tiles
// overlap:
//   warp 0     the bulk copy (TMA) of a tile's raw inputs, the box [NT/bi][2 r1][bi]
//              of the input seen as (Jp, kk, I), up to two tiles ahead;
//   warps 2-9  split each raw input into its TF32 part and remainder and write
//              both into one of two B buffers in the K-major 128-byte-swizzled
//              operand layout of tc.cuh (the next tile's split overlaps this
//              tile's products);
//   warp 1     one lane issues the products into one of four tensor-memory
//              accumulators, the core (A, TF32) read from tensor memory, where
//              the drain warps put it at the start;
//   warps 10-13 read an accumulator back (one lane quarter each), turn each
//              32 x 32 block around in shared memory and store rows of 32
//              consecutive items.
// Every wait is bounded: on expiry a warp records the failure in `err` and
// leaves its loop; the others then run out of time on their own waits; copies
// and products in flight are waited for (bounded) before the tensor memory is
// freed and the block exits.
#include "internal.cuh"
#include "qtt_dev.cuh"
#include "tc.cuh"

namespace qp {
namespace {

constexpr long long QTC_BUDGET = 2000000000LL;  // clock ticks (~1 s) per wait
constexpr int QTC_THREADS = 448;                 // 14 warps: copy, MMA, 8 split, 4 drain
constexpr int QTC_NSPLIT = 256;                  // threads of the split warps
constexpr int QTC_DRAIN0 = 10;                   // first drain warp
constexpr int QTC_T_BYTES = 32 * 32 * 4;         // per drain warp: a 32 x 32 block on its way out
constexpr int QTC_NACC = 4;                      // tensor-memory accumulators
constexpr int QTC_NRAW = 2;                      // raw input stages
constexpr int QTC_NB = 2;                        // B operand buffers (hi and lo each)
constexpr int QTC_TMEM_COLS = 512;               // accumulators, then A (and A_lo) at 128 columns each
// shared memory: the raw stages of NT x 128 floats, the B buffers (B_hi and B_lo,
// four 32-column chunks each), the drain warps' blocks, 1 KB alignment slack
constexpr int qtc_smem(int nt) {
  return QTC_NRAW * nt * 128 * 4 + QTC_NB * 8 * nt * 128 + 4 * QTC_T_BYTES + 1024;
}

__device__ __forceinline__ float tf32_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

template <class TC>
__device__ __forceinline__ float core_val(const TC* G, long long i) {
  if constexpr (sizeof(TC) == 2) return __bfloat162float(G[i]);
  else return G[i];
}

template <int NT, bool SPLIT_A, class TC>
__global__ void __launch_bounds__(QTC_THREADS, 1)
    k_qtt_tc(const __grid_constant__ CUtensorMap mIn, const TC* __restrict__ G, int r0, int r1, int lowbits, int bi,
             long long items, float* __restrict__ out, int* __restrict__ err) {
  using namespace tc;
  const int lbi = __ffs(bi) - 1;  // bi = 2^lbi items of one J' per box row
  constexpr int B_BLK = NT * 128;  // one 32-column chunk of B
  constexpr int RAW = NT * 128;    // floats of one raw stage (K up to 128)
  extern __shared__ __align__(1024) unsigned char qtc_raw[];
  unsigned char* base = qtc_raw + ((1024u - (smem_addr(qtc_raw) & 1023u)) & 1023u);
  float* sRaw = reinterpret_cast<float*>(base);
  unsigned char* sB0 = reinterpret_cast<unsigned char*>(sRaw + QTC_NRAW * RAW);  // buffer b: hi at sB0 + 8 b B_BLK
  float* sT = reinterpret_cast<float*>(sB0 + QTC_NB * 8 * B_BLK);                  // lo 4 B_BLK after hi
  __shared__ uint64_t raw_full[QTC_NRAW], raw_empty[QTC_NRAW], b_full[QTC_NB], b_empty[QTC_NB], acc_full[QTC_NACC],
      acc_empty[QTC_NACC];
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int M2 = 2 * r0, K2 = 2 * r1;
  const int KQ = ((K2 + 31) >> 5) * 8;  // 4-column groups in whole chunks
  const int KS = (K2 + 7) >> 3;         // products of K = 8
  const long long nI = 1LL << lowbits;
  const long long ntiles = items / NT;
  const int nloc = blockIdx.x < ntiles ? (int)((ntiles - 1 - blockIdx.x) / gridDim.x) + 1 : 0;

  if (tid == 0) {
    for (int s = 0; s < QTC_NRAW; ++s) {
      mbar_init(&raw_full[s], 1);
      mbar_init(&raw_empty[s], QTC_NSPLIT);
    }
    for (int b = 0; b < QTC_NB; ++b) {
      mbar_init(&b_full[b], QTC_NSPLIT);
      mbar_init(&b_empty[b], 1);
    }
    for (int a = 0; a < QTC_NACC; ++a) {
      mbar_init(&acc_full[a], 1);
      mbar_init(&acc_empty[a], 128);
    }
    fence_mbar_init();
  }
  if (warp == 1) {
    tmem_alloc(&tmem_base, QTC_TMEM_COLS);
    tmem_relinquish();
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = tmem_base;
  const uint32_t acol = QTC_NACC * NT;  // A_hi at acol, A_lo at acol + 128
  if (warp >= QTC_DRAIN0) {
    // A = the core into tensor memory: lane m holds row m, zero-padded to 128
    // rows and whole 32-column chunks
    const int m = (warp & 3) * 32 + lane;
    for (int c0 = 0; c0 < K2; c0 += 32) {
      float h[32], l[32];
#pragma unroll
      for (int e = 0; e < 32; ++e) {
        const int kk = c0 + e;
        const float v = (m < M2 && kk < K2) ? core_val<TC>(G, (long long)m * K2 + kk) : 0.f;
        h[e] = tf32_hi(v);
        l[e] = v - h[e];
      }
      const uint32_t ta = tmem + ((uint32_t)((warp & 3) * 32) << 16) + acol + (uint32_t)c0;
      tmem_st32(ta, h);
      if constexpr (SPLIT_A) tmem_st32(ta + 128u, l);
    }
    tmem_wait_st();
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();

  if (warp == 0) {
    // ---- bulk copies of the raw inputs
    int issued = 0;
    for (int i = 0; i < nloc; ++i) {
      const int s = i % QTC_NRAW;
      bool ok = mbar_wait(&raw_empty[s], ((i / QTC_NRAW) & 1) ^ 1, QTC_BUDGET);
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) {
        if (lane == 0) atomicExch(err, 1);
        break;
      }
      if (lane == 0) {
        const long long g0 = ((long long)blockIdx.x + (long long)i * gridDim.x) * NT;
        mbar_arrive_expect_tx(&raw_full[s], (uint32_t)(NT * K2 * 4));
        tma_load_3d(sRaw + s * RAW, &mIn, &raw_full[s], (int)(g0 & (nI - 1)), 0, (int)(g0 >> lowbits));
      }
      __syncwarp();
      issued = i + 1;
    }
    // copies in flight complete before the block's shared memory goes away
    for (int i = issued - QTC_NRAW < 0 ? 0 : issued - QTC_NRAW; i < issued; ++i)
      mbar_wait(&raw_full[i % QTC_NRAW], (i / QTC_NRAW) & 1, QTC_BUDGET);
  } else if (warp == 1) {
    // ---- products: D[a] = A B_hi^T + A B_lo^T (+ A_lo B_hi^T)
    constexpr uint32_t idesc = idesc_tf32(128, NT);
    int committed = 0;
    for (int i = 0; i < nloc; ++i) {
      const int a = i % QTC_NACC, b = i % QTC_NB;
      bool ok = mbar_wait(&b_full[b], (i / QTC_NB) & 1, QTC_BUDGET) &&
                mbar_wait(&acc_empty[a], ((i / QTC_NACC) & 1) ^ 1, QTC_BUDGET);
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) {
        if (lane == 0) atomicExch(err, 1);
        break;
      }
      fence_after_sync();
      if (lane == 0) {
        const uint32_t d = tmem + (uint32_t)(a * NT);
        const uint32_t bb = smem_addr(sB0 + b * 8 * B_BLK), bl = bb + 4 * B_BLK;
        for (int s = 0; s < KS; ++s) {
          const uint32_t ah = tmem + acol + (uint32_t)(8 * s), bo = (s >> 2) * B_BLK + (s & 3) * 32;
          const uint64_t bd = desc_k_sw128(bb + bo);
          mma_tf32_ts(d, ah, bd, idesc, s > 0 ? 1u : 0u);
          mma_tf32_ts(d, ah, desc_k_sw128(bl + bo), idesc, 1u);
          if constexpr (SPLIT_A) mma_tf32_ts(d, ah + 128u, bd, idesc, 1u);
        }
        mma_commit(&b_empty[b]);   // buffer b may be rewritten once these products are done
        mma_commit(&acc_full[a]);  // and the accumulator read
      }
      __syncwarp();
      committed = i + 1;
    }
    for (int i = committed - QTC_NB < 0 ? 0 : committed - QTC_NB; i < committed; ++i)
      mbar_wait(&b_empty[i % QTC_NB], (i / QTC_NB) & 1, QTC_BUDGET);
  } else if (warp < QTC_DRAIN0) {
    // ---- split: raw stage -> B_hi, B_lo (items on consecutive threads)
    const int ct = tid - 64;
    for (int i = 0; i < nloc; ++i) {
      const int s = i % QTC_NRAW, b = i % QTC_NB;
      const bool ok = mbar_wait(&raw_full[s], (i / QTC_NRAW) & 1, QTC_BUDGET) &&
                      mbar_wait(&b_empty[b], ((i / QTC_NB) & 1) ^ 1, QTC_BUDGET);
      if (!ok) {
        atomicExch(err, 1);
        break;
      }
      const float* raw = sRaw + s * RAW;
      unsigned char* sB = sB0 + b * 8 * B_BLK;
      unsigned char* sBl = sB + 4 * B_BLK;
#pragma unroll 4
      for (int unit = ct; unit < NT * KQ; unit += QTC_NSPLIT) {
        const int n = unit & (NT - 1), q = unit / NT;
        const int jj = n >> lbi, ii = n & (bi - 1);
        const float* src = raw + jj * (K2 * bi) + ii;
        float x[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int kk = 4 * q + e;
          x[e] = kk < K2 ? src[kk * bi] : 0.f;
        }
        const int off = (q >> 3) * B_BLK + n * 128 + (((q & 7) ^ (n & 7)) << 4);
        const float4 h = make_float4(tf32_hi(x[0]), tf32_hi(x[1]), tf32_hi(x[2]), tf32_hi(x[3]));
        *reinterpret_cast<float4*>(sB + off) = h;
        *reinterpret_cast<float4*>(sBl + off) = make_float4(x[0] - h.x, x[1] - h.y, x[2] - h.z, x[3] - h.w);
      }
      fence_async_shared();
      mbar_arrive(&b_full[b]);
      mbar_arrive(&raw_empty[s]);
    }
  } else {
    // ---- drain: accumulator -> out, 32 x 32 blocks turned around in shared
    // memory (column index XOR row: no bank conflicts either way)
    const int quarter = warp & 3;
    const int mbase = quarter * 32;
    const int rows = M2 - mbase < 32 ? M2 - mbase : 32;  // <= 0: padding rows only
    float* st = sT + (warp - QTC_DRAIN0) * (QTC_T_BYTES / 4);
    for (int i = 0; i < nloc; ++i) {
      const int a = i % QTC_NACC;
      const bool ok = mbar_wait(&acc_full[a], (i / QTC_NACC) & 1, QTC_BUDGET);
      if (__any_sync(0xffffffffu, !ok)) {
        if (lane == 0) atomicExch(err, 1);
        break;
      }
      fence_after_sync();
      if (rows > 0) {
        const long long t = (long long)blockIdx.x + (long long)i * gridDim.x;
#pragma unroll
        for (int c0 = 0; c0 < NT; c0 += 32) {
          float v[32];
          tmem_ld32(tmem + ((uint32_t)mbase << 16) + (uint32_t)(a * NT + c0), v);
#pragma unroll
          for (int e = 0; e < 32; ++e) st[lane * 32 + (e ^ lane)] = v[e];
          __syncwarp();
          const long long g = t * NT + c0 + lane;
          const long long Jp = g >> lowbits, I = g & (nI - 1);
          float* o = out + (Jp * M2 + mbase) * nI + I;
#pragma unroll 4
          for (int r = 0; r < rows; ++r) o[(long long)r * nI] = st[r * 32 + (lane ^ r)];
          __syncwarp();
        }
      }
      fence_before_sync();
      mbar_arrive(&acc_empty[a]);
    }
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if (warp == 1) tmem_dealloc(tmem, QTC_TMEM_COLS);
}

// The input of the step seen as a 3-D tensor (I: nI, kk: 2 r1, Jp: 2^(k-1)),
// boxes of (bi, 2 r1, NT / bi) with bi = min(nI, NT).
CUtensorMap step_map(const float* in, int lowbits, int r1, int njp, int bi, int nt) {
  QP_REQUIRE((reinterpret_cast<uintptr_t>(in) & 15u) == 0, QP_CUDA_ERROR, "tensor map base not 16-byte aligned");
  CUtensorMap m;
  const cuuint64_t nI = 1ull << lowbits;
  const cuuint64_t gdim[3] = {nI, (cuuint64_t)(2 * r1), (cuuint64_t)njp};
  const cuuint64_t gstride[2] = {nI * sizeof(float), nI * 2 * r1 * sizeof(float)};
  const cuuint32_t box[3] = {(cuuint32_t)bi, (cuuint32_t)(2 * r1), (cuuint32_t)(nt / bi)};
  const cuuint32_t es[3] = {1, 1, 1};
  const CUresult r = tmap_encoder()(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(in), gdim, gstride,
                                    box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  QP_REQUIRE(r == CUDA_SUCCESS, QP_CUDA_ERROR, "cuTensorMapEncodeTiled failed (QTT step)");
  return m;
}

template <int NT, bool SPLIT_A, class TC>
void launch_tc(qp_ctx* c, const QttDev& q, int k, const TC* G, const float* in, float* out) {
  const int r0 = q.ranks[k - 1], r1 = q.ranks[k];
  const int lowbits = q.d - k;
  const long long items = 1LL << (q.d - 1);
  const int bi = (1 << lowbits) < NT ? (1 << lowbits) : NT;
  const CUtensorMap m = step_map(in, lowbits, r1, 1 << (k - 1), bi, NT);
  auto kern = k_qtt_tc<NT, SPLIT_A, TC>;
  constexpr int smem = qtc_smem(NT);
  QP_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  const long long ntiles = items / NT;
  const int grid = (int)std::min<long long>(ntiles, c->num_sms);
  kern<<<grid, QTC_THREADS, smem, c->stream>>>(m, G, r0, r1, lowbits, bi, items, out, qtt_tc_flag(c));
  QP_CUDA(cudaGetLastError());
}

}  // namespace

int* qtt_tc_flag(qp_ctx* c) { return static_cast<int*>(c->tc_err.ensure(64)); }

bool qtt_tc_eligible(const qp_ctx* c, const QttDev& q, int k, qp_dtype cdt) {
  // a tile holds 64 (BF16 cores) or 32 (F32 cores) of the 2^(d-1) items; the
  // bulk copy's innermost extent 2^(d-k) must span at least 16 bytes
  if (c->qtt_tc_mode == 0 || q.d < 8 || q.d - k < 2) return false;
  if (cdt != QP_BF16 && cdt != QP_F32) return false;
  const int r0 = q.ranks[k - 1], r1 = q.ranks[k];
  if (r0 > 64 || r1 > 64) return false;
  if (c->qtt_tc_mode == 2) return true;
  // automatic: BF16 cores only (their rounding, 2^-9, dominates the tensor
  // cores' accumulation error), and only where the contraction is dense
  return cdt == QP_BF16 && r0 * r1 >= QTT_TC_MIN_RR;
}

void launch_qtt_step_tc(qp_ctx* c, const QttDev& q, int k, const float* in, float* out, qp_dtype cdt) {
  if (cdt == QP_BF16) {
    const auto* G = static_cast<const __nv_bfloat16*>(q.cores) + q.off[k - 1];
    launch_tc<64, false, __nv_bfloat16>(c, q, k, G, in, out);
  } else {
    QP_REQUIRE(cdt == QP_F32, QP_INVALID_ARG, "tensor-core QTT step: cores must be BF16 or F32");
    const auto* G = static_cast<const float*>(q.cores) + q.off[k - 1];
    launch_tc<32, true, float>(c, q, k, G, in, out);
  }
}

}  // namespace qp

extern "C" int qtt_set_tensor_cores(qp_ctx_t c, int mode) {
  if (!c || mode < 0 || mode > 2) return QP_INVALID_ARG;
  c->qtt_tc_mode = mode;
  return QP_OK;
}
