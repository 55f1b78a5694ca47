// Warm start of the PDIP of a new time step from the previous step's impulses
// (Sec. 3.3: most contacts persist from one step to the next).
#include <cub/cub.cuh>

#include "internal.cuh"

namespace qp {
namespace {

// Key of a contact: (a, b), with a static plane's body M replaced by M + its
// plane index (floor 0, wall w: 1 + w), so a sphere's floor and wall contacts
// differ; without plane indices (plane == nullptr) the pair alone.
__device__ __forceinline__ unsigned long long pair_key(int a, int b, const int* plane, int i, int M) {
  if (plane) {
    const int w = __ldg(plane + i);
    if (w >= 0) a = M + w;
  }
  return ((unsigned long long)(unsigned)a << 32) | (unsigned)b;
}

__global__ void k_prev_keys(int n, int M, const int* __restrict__ a, const int* __restrict__ b,
                            const int* __restrict__ plane, unsigned long long* __restrict__ key,
                            int* __restrict__ idx) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    key[i] = pair_key(__ldg(a + i), __ldg(b + i), plane, i, M);
    idx[i] = i;
  }
}

// One thread per padded row; the row of slot 0 of a contact also writes its
// two multipliers.  A contact whose pair was in the previous set takes that
// impulse moved into its cone's interior (gamma_n >= gn0, |gamma_t| <=
// shrink mu gamma_n); a new contact takes (gn0, 0, 0); lambda = -1/f.
__global__ void k_pdip_warm(int Nc, int M, int slots, long long P, double mu, double gn0, double shrink,
                            const int* __restrict__ ca, const int* __restrict__ cb, const int* __restrict__ cplane,
                            const unsigned long long* __restrict__ skey, const int* __restrict__ sidx, int nprev,
                            int pslots, const double* __restrict__ pgamma, double* __restrict__ gamma,
                            double* __restrict__ lambda) {
  const long long gsz = (long long)gridDim.x * blockDim.x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P; i += gsz) {
    const long long c = i / slots;
    const int u = (int)(i - c * slots);
    if (c >= Nc || u >= 3) {
      gamma[i] = 0.0;
      continue;
    }
    const unsigned long long k = pair_key(__ldg(ca + c), __ldg(cb + c), cplane, (int)c, M);
    int lo = 0, hi = nprev;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (__ldg(skey + mid) < k) lo = mid + 1;
      else hi = mid;
    }
    double gn = gn0, t1 = 0.0, t2 = 0.0;
    if (lo < nprev && __ldg(skey + lo) == k) {
      const long long j = __ldg(sidx + lo);
      gn = fmax(__ldg(pgamma + pslots * j), gn0);
      t1 = __ldg(pgamma + pslots * j + 1);
      t2 = __ldg(pgamma + pslots * j + 2);
      const double nt = hypot(t1, t2);
      const double cap = shrink * mu * gn;
      if (nt > cap) {
        t1 *= cap / nt;
        t2 *= cap / nt;
      }
    }
    gamma[i] = u == 0 ? gn : (u == 1 ? t1 : t2);
    if (u == 0) {
      const double f = 0.5 * (t1 * t1 + t2 * t2 - mu * mu * gn * gn);
      lambda[c] = -1.0 / f;
      lambda[Nc + c] = 1.0 / gn;
    }
  }
}

}  // namespace
}  // namespace qp

using namespace qp;

extern "C" int pdip_init_warm(qp_ctx_t c, qp_state* st, const qp_prev_contacts* prev, double gn0, double shrink) {
  if (!c) return QP_INVALID_ARG;
  try {
    QP_CUDA(cudaSetDevice(c->device));
    QP_REQUIRE(c->have_contacts, QP_NOT_READY, "no contacts: call ccp_assemble first");
    QP_REQUIRE(st && st->gamma && st->lambda, QP_INVALID_ARG, "pdip_init_warm: null state");
    QP_REQUIRE(prev && prev->Nc >= 0, QP_INVALID_ARG, "pdip_init_warm: null previous contact set");
    QP_REQUIRE(prev->Nc == 0 || (prev->body_a && prev->body_b && prev->gamma), QP_INVALID_ARG,
               "pdip_init_warm: null previous arrays");
    QP_REQUIRE(prev->slots == 3 || prev->slots == 4, QP_INVALID_ARG, "pdip_init_warm: slots must be 3 or 4");
    QP_REQUIRE(gn0 > 0 && shrink > 0 && shrink <= 1, QP_INVALID_ARG, "pdip_init_warm: need gn0 > 0, 0 < shrink <= 1");
    const int n = prev->Nc;
    const size_t nn = (size_t)(n > 0 ? n : 1);
    // previous pairs sorted by key, with their indices (scratch buffers of the step)
    auto* key = static_cast<unsigned long long*>(c->dm[14].ensure(4 * nn * sizeof(unsigned long long)));
    unsigned long long* skey = key + nn;
    int* idx = reinterpret_cast<int*>(key + 2 * nn);
    int* sidx = idx + nn;
    if (n > 0) {
      k_prev_keys<<<(n + 255) / 256, 256, 0, c->stream>>>(n, c->M, prev->body_a, prev->body_b, prev->plane, key,
                                                          idx);
      QP_CUDA(cudaGetLastError());
      size_t tmp_bytes = 0;
      QP_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, key, skey, idx, sidx, n, 0, 64, c->stream));
      void* tmp = c->dm[15].ensure(tmp_bytes > 0 ? tmp_bytes : 1);
      QP_CUDA(cub::DeviceRadixSort::SortPairs(tmp, tmp_bytes, key, skey, idx, sidx, n, 0, 64, c->stream));
    }
    int grid = (int)((c->P + 255) / 256);
    if (grid > c->num_sms * 8) grid = c->num_sms * 8;
    // plane indices take part in the keys on both sides, or on neither
    k_pdip_warm<<<grid, 256, 0, c->stream>>>(c->Nc, c->M, c->slots, c->P, c->mu, gn0, shrink, c->ca.as<int>(),
                                             c->cb.as<int>(), prev->plane ? c->cplane.as<int>() : nullptr, skey, sidx,
                                             n, prev->slots, prev->gamma, st->gamma, st->lambda);
    QP_CUDA(cudaGetLastError());
    st->t = 1.0;
  } catch (const Error& e) {
    set_error(c, e);
    return e.code;
  }
  return QP_OK;
}
