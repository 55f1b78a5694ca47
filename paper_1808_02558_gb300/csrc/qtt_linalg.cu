// TT rounding (Sec. 3.1 truncation rule, Oseledets 2011 rounding) and the QTT
// compression of the Schur matrix (Sec. 3.2 tensorisation, Alg. 1 TT-SVD).
//
// Small dense linear algebra runs in FP64 inside one thread block (la_dev.cuh): symmetric
// eigendecompositions by cyclic Jacobi with round-robin (parallel) rotation
// order (Golub and Van Loan, Matrix Computations, Sec. 8.5), and the SVD of a
// tall matrix C through the eigenpairs of its Gram matrix C^T C.
//
// Compression exploits the sparsity of S: the TT-SVD is swept right to left, so
// the rows of each unfolding are the nonzero matrix blocks of one level of the
// binary row/column trees and the columns are (mode digit, rank index); zero
// rows of the dense unfolding never appear.  The result is the TT-SVD of the
// index-reversed tensor, i.e. Alg. 1 applied from the last core to the first.
#include <cub/cub.cuh>

#include <algorithm>
#include <cmath>

#include "internal.cuh"
#include "la_dev.cuh"

namespace qp {
namespace {

constexpr int LT = 1024;  // threads of the one-block kernels

using dla::trunc_rank;

__device__ inline double cta_sum(double v) { return dla::block_sum(v); }

// dynamic shared memory of the one-block kernels (the eigensolver's staging area)
extern __shared__ double la_smem[];

__device__ inline void cta_syev(double* A, double* V, double* Vs, double* w, int n) {
  dla::syev(A, V, Vs, w, n, la_smem);
}

// ---------------------------------------------------------------- rounding
struct RoundArgs {
  int d;
  double eps;
  int rmax;
  int* ranks;      // [d+1], in/out
  long long cap;   // values per core slot
  double* cores;   // [d][cap]
  double* A;       // n x n workspaces
  double* V;
  double* Vs;
  double* w;
  double* tmp;     // cap values
  double* norm_out;
};

// Below eps = 1e-7 the SVDs are one-sided Jacobi on the cores themselves (the
// Gram route resolves singular values only down to about 1e-8 sigma_max);
// above, the Gram matrices and the shared eigensolver, which are faster at
// large ranks on the narrow FP64 pipe.
__global__ void __launch_bounds__(LT) k_tt_round(RoundArgs a) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int d = a.d;
  __shared__ int sh_r;
  const bool accurate = a.eps < 1e-7;
  int* ord = reinterpret_cast<int*>(a.A);  // order of the singular values (accurate path)
  // right-to-left orthogonalisation: core_k = R Q with orthonormal rows of Q
  for (int k = d - 1; k >= 1; --k) {
    const int rk = a.ranks[k], rn = a.ranks[k + 1], rp = a.ranks[k - 1];
    double* B = a.cores + (long long)k * a.cap;         // rk x 4rn
    double* Cp = a.cores + (long long)(k - 1) * a.cap;  // (rp*4) x rk
    const int nc = 4 * rn;
    if (accurate) {
      // rows of B made orthogonal: B = Vr (Sigma Q); Q's rows are the normalised
      // rows, Vr Sigma moves into core_{k-1}; rows at FP64 rounding are dropped
      dla::osj(B, rk, nc, nc, 1, a.V);
      dla::osj_norms(B, rk, nc, nc, 1, a.w, ord);
      if (tid == 0) {
        const double smax = a.w[ord[0]];
        int r = 0;
        while (r < rk && a.w[ord[r]] > 1e-15 * smax && a.w[ord[r]] > 0.0) ++r;
        sh_r = r < 1 ? 1 : r;
      }
      __syncthreads();
      const int r = sh_r;
      for (int i = tid; i < r * nc; i += nt) {
        const int x = i / nc, cc = i - x * nc;
        const double sg = a.w[ord[x]];
        a.tmp[i] = sg > 0.0 ? B[ord[x] * nc + cc] / sg : 0.0;
      }
      __syncthreads();
      for (int i = tid; i < r * nc; i += nt) B[i] = a.tmp[i];
      __syncthreads();
      const int mrow = rp * 4;
      for (int i = tid; i < mrow * r; i += nt) {
        const int x = i / r, y = i - x * r;
        double sm = 0.0;
        for (int z = 0; z < rk; ++z) sm += Cp[x * rk + z] * a.V[z * rk + ord[y]];
        a.tmp[i] = sm * a.w[ord[y]];
      }
      __syncthreads();
      for (int i = tid; i < mrow * r; i += nt) Cp[i] = a.tmp[i];
      if (tid == 0) a.ranks[k] = r;
      __syncthreads();
      continue;
    }
    for (int i = tid; i < rk * rk; i += nt) {
      int x = i / rk, y = i - x * rk;
      double s = 0.0;
      for (int c = 0; c < nc; ++c) s += B[x * nc + c] * B[y * nc + c];
      a.A[i] = s;
    }
    __syncthreads();
    cta_syev(a.A, a.V, a.Vs, a.w, rk);
    if (tid == 0) {
      double lmax = fmax(a.w[0], 0.0);
      int r = 0;
      while (r < rk && a.w[r] > 1e-20 * lmax && a.w[r] > 0.0) ++r;  // sigma > 1e-10 sigma_max
      sh_r = r < 1 ? 1 : r;
    }
    __syncthreads();
    const int r = sh_r;
    // Q = diag(lambda^-1/2) Vs^T B   (r x nc)
    for (int i = tid; i < r * nc; i += nt) {
      int x = i / nc, c = i - x * nc;
      double lam = a.w[x];
      double s = 0.0;
      for (int y = 0; y < rk; ++y) s += a.Vs[y * rk + x] * B[y * nc + c];
      a.tmp[i] = lam > 0.0 ? s / sqrt(lam) : 0.0;
    }
    __syncthreads();
    for (int i = tid; i < r * nc; i += nt) B[i] = a.tmp[i];
    __syncthreads();
    // core_{k-1} <- core_{k-1} * Vs diag(lambda^1/2)   ((rp*4) x r)
    const int mrow = rp * 4;
    for (int i = tid; i < mrow * r; i += nt) {
      int x = i / r, y = i - x * r;
      double s = 0.0;
      for (int z = 0; z < rk; ++z) s += Cp[x * rk + z] * a.Vs[z * rk + y];
      a.tmp[i] = s * sqrt(fmax(a.w[y], 0.0));
    }
    __syncthreads();
    for (int i = tid; i < mrow * r; i += nt) Cp[i] = a.tmp[i];
    if (tid == 0) a.ranks[k] = r;
    __syncthreads();
  }
  // Frobenius norm of the (now right-orthogonal) TT = norm of core 0
  double nn = 0.0;
  {
    const int n0 = 4 * a.ranks[1];
    for (int i = tid; i < n0; i += nt) nn += a.cores[i] * a.cores[i];
  }
  nn = sqrt(cta_sum(nn));
  if (tid == 0 && a.norm_out) *a.norm_out = nn;
  const double delta = a.eps * nn / sqrt((double)(d > 1 ? d - 1 : 1));
  // left-to-right truncated SVD
  for (int k = 0; k < d - 1; ++k) {
    const int rk = a.ranks[k], rn = a.ranks[k + 1], r2 = a.ranks[k + 2];
    double* C = a.cores + (long long)k * a.cap;            // (rk*4) x rn
    double* Cn = a.cores + (long long)(k + 1) * a.cap;     // rn x 4 r2
    const int mrow = rk * 4;
    if (accurate) {
      // columns of C made orthogonal: C = (U Sigma) Vr^T; core_k <- U[:, :r],
      // core_{k+1} <- Sigma Vr[:, :r]^T core_{k+1}, r by the truncation rule on sigma^2
      dla::osj(C, rn, mrow, 1, rn, a.V);
      dla::osj_norms(C, rn, mrow, 1, rn, a.Vs, ord);
      for (int i = tid; i < rn; i += nt) a.w[i] = a.Vs[ord[i]] * a.Vs[ord[i]];
      __syncthreads();
      if (tid == 0) sh_r = trunc_rank(a.w, rn, delta, a.rmax);
      __syncthreads();
      const int r = sh_r;
      for (int i = tid; i < mrow * r; i += nt) {
        const int x = i / r, y = i - x * r;
        const double sg = a.Vs[ord[y]];
        a.tmp[i] = sg > 0.0 ? C[x * rn + ord[y]] / sg : 0.0;
      }
      __syncthreads();
      for (int i = tid; i < mrow * r; i += nt) C[i] = a.tmp[i];
      __syncthreads();
      const int nc = 4 * r2;
      for (int i = tid; i < r * nc; i += nt) {
        const int x = i / nc, cc = i - x * nc;
        double sm = 0.0;
        for (int z = 0; z < rn; ++z) sm += a.V[z * rn + ord[x]] * Cn[z * nc + cc];
        a.tmp[i] = sm * a.Vs[ord[x]];
      }
      __syncthreads();
      for (int i = tid; i < r * nc; i += nt) Cn[i] = a.tmp[i];
      if (tid == 0) a.ranks[k + 1] = r;
      __syncthreads();
      continue;
    }
    for (int i = tid; i < rn * rn; i += nt) {
      int x = i / rn, y = i - x * rn;
      double s = 0.0;
      for (int z = 0; z < mrow; ++z) s += C[z * rn + x] * C[z * rn + y];
      a.A[i] = s;
    }
    __syncthreads();
    cta_syev(a.A, a.V, a.Vs, a.w, rn);
    if (tid == 0) sh_r = trunc_rank(a.w, rn, delta, a.rmax);
    __syncthreads();
    const int r = sh_r;
    // core_k <- C Vs[:, :r] diag(1/sigma)
    for (int i = tid; i < mrow * r; i += nt) {
      int x = i / r, y = i - x * r;
      double s = 0.0;
      for (int z = 0; z < rn; ++z) s += C[x * rn + z] * a.Vs[z * rn + y];
      double sig = sqrt(fmax(a.w[y], 0.0));
      a.tmp[i] = sig > 0.0 ? s / sig : 0.0;
    }
    __syncthreads();
    for (int i = tid; i < mrow * r; i += nt) C[i] = a.tmp[i];
    __syncthreads();
    // core_{k+1} <- diag(sigma) Vs[:, :r]^T core_{k+1}
    const int nc = 4 * r2;
    for (int i = tid; i < r * nc; i += nt) {
      int x = i / nc, c = i - x * nc;
      double s = 0.0;
      for (int z = 0; z < rn; ++z) s += a.Vs[z * rn + x] * Cn[z * nc + c];
      a.tmp[i] = s * sqrt(fmax(a.w[x], 0.0));
    }
    __syncthreads();
    for (int i = tid; i < r * nc; i += nt) Cn[i] = a.tmp[i];
    if (tid == 0) a.ranks[k + 1] = r;
    __syncthreads();
  }
}

// ---------------------------------------------------------------- compression
// Entry (i, j) -> tensor key: base-4 digits b_k = 2 i_k + j_k, most significant first,
// i.e. bit 2m+1 = bit m of i and bit 2m = bit m of j.
__device__ __forceinline__ unsigned long long qtt_key(unsigned long long i, unsigned long long j, int d) {
  unsigned long long k = 0;
  for (int m = 0; m < d; ++m) k |= (((i >> m) & 1ull) << (2 * m + 1)) | (((j >> m) & 1ull) << (2 * m));
  return k;
}

__global__ void k_pair_count(int M, const int* __restrict__ bptr, int* __restrict__ cnt) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b > M) return;
  if (b == M) {
    cnt[b] = 0;
    return;
  }
  int dg = bptr[b + 1] - bptr[b];
  cnt[b] = dg * (dg - 1);
}

// 3x3 block of D_c1b^T M_b^-1 D_c2b for contacts c1, c2 incident to body b.
__device__ __forceinline__ void body_block(const double* R1, int side1, const double* R2, int side2, double im,
                                           double iI, double out[9]) {
  const double s = (side1 ? 1.0 : -1.0) * (side2 ? 1.0 : -1.0);
  const double* a1 = side1 ? R1 + 12 : R1 + 9;
  const double* a2 = side2 ? R2 + 12 : R2 + 9;
  for (int u = 0; u < 3; ++u) {
    const double* U1 = R1 + 3 * u;
    double t1[3] = {a1[1] * U1[2] - a1[2] * U1[1], a1[2] * U1[0] - a1[0] * U1[2], a1[0] * U1[1] - a1[1] * U1[0]};
    for (int v = 0; v < 3; ++v) {
      const double* U2 = R2 + 3 * v;
      double t2[3] = {a2[1] * U2[2] - a2[2] * U2[1], a2[2] * U2[0] - a2[0] * U2[2], a2[0] * U2[1] - a2[1] * U2[0]};
      out[3 * u + v] = s * (im * (U1[0] * U2[0] + U1[1] * U2[1] + U1[2] * U2[2]) +
                            iI * (t1[0] * t2[0] + t1[1] * t2[1] + t1[2] * t2[2]));
    }
  }
}

struct EntryArgs {
  int M, Nc, slots, d;
  long long P;
  const double* rec;  // [Nc][16] FP64 records
  const int* ca;
  const int* cb;
  const double* inv_m;
  const double* inv_I;
  const int* bptr;
  const int* inc;
  const double* H;    // [6][Nc] or null
  const int* off;     // [M+1] offsets of off-diagonal blocks (per body)
  const double* rs;   // [P] row scaling (entry (i,j) is multiplied by rs[i] rs[j]) or null
  unsigned long long* key;
  double* val;
};

__device__ __forceinline__ double escale(const EntryArgs& e, long long i, long long j) {
  return e.rs ? e.rs[i] * e.rs[j] : 1.0;
}

__global__ void k_entries_offdiag(EntryArgs e) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= e.M) return;
  const int s = e.bptr[b], t = e.bptr[b + 1];
  long long o = 9LL * e.off[b];
  const double im = e.inv_m[b], iI = e.inv_I[b];
  for (int k1 = s; k1 < t; ++k1) {
    const int c1 = e.inc[k1] >> 1, s1 = e.inc[k1] & 1;
    const double* R1 = e.rec + (size_t)c1 * 16;
    for (int k2 = s; k2 < t; ++k2) {
      if (k2 == k1) continue;
      const int c2 = e.inc[k2] >> 1, s2 = e.inc[k2] & 1;
      double blk[9];
      body_block(R1, s1, e.rec + (size_t)c2 * 16, s2, im, iI, blk);
      for (int u = 0; u < 3; ++u)
        for (int v = 0; v < 3; ++v) {
          const long long ri = (long long)e.slots * c1 + u, ci = (long long)e.slots * c2 + v;
          e.key[o] = qtt_key((unsigned long long)ri, (unsigned long long)ci, e.d);
          e.val[o] = blk[3 * u + v] * escale(e, ri, ci);
          ++o;
        }
    }
  }
}

__global__ void k_entries_diag(EntryArgs e, long long base) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= e.Nc) return;
  const double* R = e.rec + (size_t)c * 16;
  const int a = e.ca[c], b = e.cb[c];
  double blk[9], tmp[9];
  body_block(R, 1, R, 1, e.inv_m[b], e.inv_I[b], blk);
  if (a < e.M) {
    body_block(R, 0, R, 0, e.inv_m[a], e.inv_I[a], tmp);
    for (int k = 0; k < 9; ++k) blk[k] += tmp[k];
  }
  if (e.H) {
    const long long n = e.Nc;
    double h[6] = {e.H[c], e.H[n + c], e.H[2 * n + c], e.H[3 * n + c], e.H[4 * n + c], e.H[5 * n + c]};
    const int map[9] = {0, 1, 2, 1, 3, 4, 2, 4, 5};
    for (int k = 0; k < 9; ++k) blk[k] += h[map[k]];
  }
  const int per = e.slots == 4 ? 10 : 9;
  long long o = base + (long long)per * c;
  for (int u = 0; u < 3; ++u)
    for (int v = 0; v < 3; ++v) {
      const long long ri = (long long)e.slots * c + u, ci = (long long)e.slots * c + v;
      e.key[o] = qtt_key((unsigned long long)ri, (unsigned long long)ci, e.d);
      e.val[o] = blk[3 * u + v] * escale(e, ri, ci);
      ++o;
    }
  if (e.slots == 4) {
    e.key[o] = qtt_key(4ull * c + 3, 4ull * c + 3, e.d);
    e.val[o] = escale(e, 4LL * c + 3, 4LL * c + 3);
  }
}

__global__ void k_entries_tail(EntryArgs e, long long base) {
  const long long t0 = (long long)e.slots * e.Nc;
  for (long long i = t0 + blockIdx.x * (long long)blockDim.x + threadIdx.x; i < e.P;
       i += (long long)gridDim.x * blockDim.x) {
    e.key[base + i - t0] = qtt_key((unsigned long long)i, (unsigned long long)i, e.d);
    e.val[base + i - t0] = escale(e, i, i);
  }
}

__global__ void k_parent_flags(long long n, const unsigned long long* __restrict__ key, int* __restrict__ flag) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    flag[i] = (i == 0 || (key[i] >> 2) != (key[i - 1] >> 2)) ? 1 : 0;
}

// M[pid, child*r + a] = W[i, a];  parent key list
__global__ void k_scatter_rows(long long n, int r, const unsigned long long* __restrict__ key,
                               const int* __restrict__ pid, const double* __restrict__ W, double* __restrict__ Mx,
                               unsigned long long* __restrict__ pkey) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int p = pid[i] - 1;
    const int ch = (int)(key[i] & 3ull);
    for (int a = 0; a < r; ++a) Mx[(long long)p * 4 * r + ch * r + a] = W[i * r + a];
    if (i == 0 || (key[i] >> 2) != (key[i - 1] >> 2)) pkey[p] = key[i] >> 2;
  }
}

// Partial Gram matrices of row chunks: part[chunk][x][y] = sum_rows M[row][x] M[row][y]
__global__ void k_gram_partial(long long rows, int n, const double* __restrict__ Mx, double* __restrict__ part,
                               long long chunk) {
  const long long r0 = blockIdx.x * chunk;
  const long long r1 = min(rows, r0 + chunk);
  double* out = part + (long long)blockIdx.x * n * n;
  for (int xy = threadIdx.x; xy < n * n; xy += blockDim.x) {
    const int x = xy / n, y = xy - x * n;
    double s = 0.0;
    for (long long r = r0; r < r1; ++r) s += Mx[r * n + x] * Mx[r * n + y];
    out[xy] = s;
  }
}

// The same partial Gram matrices for n = 4 r <= 64, register-tiled: the block
// stages GR_ROWS rows of its chunk in shared memory, thread t owns the 4 x 4
// tile (tx, ty), tx <= ty, of the upper triangle in row group g (groups take
// every G-th staged row, so all 256 threads work at small n); the groups' tiles
// are then added in group order into the block's partial (both triangles).
// Partials are summed in block order by k_gram_reduce: the result does not
// depend on scheduling.  Dynamic shared memory: GR_SMEM bytes.
constexpr int GR_ROWS = 64;
constexpr int GR_SMEM = 60 * 1024;  // >= GR_ROWS * 64 doubles and >= G n^2 doubles for every n = 4 r <= 64
__global__ void __launch_bounds__(256) k_gram_tiled(long long rows, int n, const double* __restrict__ Mx,
                                                    double* __restrict__ part, long long chunk) {
  extern __shared__ double gr_sm[];
  const int T = n >> 2, ntiles = T * (T + 1) / 2;
  const int G = 256 / ntiles;  // row groups (>= 1 for n <= 64)
  const int tid = threadIdx.x, g = tid / ntiles, tile = tid - g * ntiles;
  const bool active = g < G;
  int tx = 0, ty = 0;
  if (active) {
    int rem = tile;
    while (rem > ty) {
      rem -= ty + 1;
      ++ty;
    }
    tx = rem;  // 0 <= tx <= ty
  }
  double acc[4][4] = {};
  const long long r0 = blockIdx.x * chunk;
  const long long r1 = min(rows, r0 + chunk);
  for (long long base = r0; base < r1; base += GR_ROWS) {
    const int nr = (int)min((long long)GR_ROWS, r1 - base);
    __syncthreads();
    for (int i = tid; i < nr * n; i += 256) gr_sm[i] = Mx[base * n + i];
    __syncthreads();
    if (active) {
      for (int rr = g; rr < nr; rr += G) {
        const double* row = gr_sm + rr * n;
        double a[4], b[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          a[i] = row[4 * tx + i];
          b[i] = row[4 * ty + i];
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
      }
    }
  }
  __syncthreads();
  const int nn = n * n;
  if (active) {
    double* red = gr_sm + g * nn;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int x = 4 * tx + i, y = 4 * ty + j;
        red[x * n + y] = acc[i][j];
        red[y * n + x] = acc[i][j];
      }
  }
  __syncthreads();
  double* out = part + (long long)blockIdx.x * nn;
  for (int xy = tid; xy < nn; xy += 256) {
    double v = 0.0;
    for (int q = 0; q < G; ++q) v += gr_sm[q * nn + xy];
    out[xy] = v;
  }
}

__global__ void k_gram_reduce(int nparts, int n, const double* __restrict__ part, double* __restrict__ G) {
  for (int xy = blockIdx.x * blockDim.x + threadIdx.x; xy < n * n; xy += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int p = 0; p < nparts; ++p) s += part[(long long)p * n * n + xy];
    G[xy] = s;
  }
}

struct EigArgs {
  double* A;
  double* V;
  double* Vs;
  double* w;
  int n;
  double delta;
  int rmax;
  int* rank_out;
};

__global__ void __launch_bounds__(LT) k_eig_trunc(EigArgs e) {
  cta_syev(e.A, e.V, e.Vs, e.w, e.n);
  if (threadIdx.x == 0) *e.rank_out = trunc_rank(e.w, e.n, e.delta, e.rmax);
}

// ---------------------------------------------------------------- multi-block Jacobi
// Gram matrices of order n > SYEV_SMEM_N (ranks above 16) do not fit in one
// block's shared memory, and one block rotating them in global memory spends
// most of its time waiting on L2.  Their rotation rounds spread over a
// cooperative grid: in round r every block forms the round's rotations from A
// (the same values in every block), the rows of B = J^T A are written from A,
// a grid barrier, then A = B J and V = V J, a grid barrier.  B is a second
// buffer so that no block rotates rows of A that another block is still
// reading for its rotations.  The sweeps, the convergence test and the sorted
// output are those of the one-block solver; every wait is bounded (QP_TIMEOUT).
struct EigCoopArgs {
  double* A;
  double* B;
  double* V;
  double* Vs;
  double* w;
  int n;
  double delta;
  int rmax;
  int* rank_out;
  DevCtl* ctl;
  double* part;  // 2 per block
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_add_u32(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Counter barrier over the cooperative grid (the counter starts at 0); thread
// 0 of each block counts the generations in `gen`.  False on timeout or when
// another block has recorded an error.
__device__ bool coop_barrier(DevCtl* ctl, unsigned& gen) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    gen += 1u;
    red_release_add_u32(&ctl->bar_count, 1u);
    const unsigned target = gen * gridDim.x;
    const long long t0 = clock64();
    ok = 1;
    while ((int)(ld_acquire_u32(&ctl->bar_count) - target) < 0) {
      if (*(volatile int*)&ctl->err) {
        ok = 0;
        break;
      }
      if (clock64() - t0 > 4000000000LL) {
        atomicCAS(&ctl->err, 0, QP_TIMEOUT);
        ok = 0;
        break;
      }
    }
  }
  __syncthreads();
  return ok != 0;
}

__global__ void __launch_bounds__(256) k_eig_coop(EigCoopArgs e) {
  __shared__ double rc[256], rs[256];
  __shared__ int rp[256], rq[256];
  __shared__ int s_done;
  unsigned gen = 0;
  const int n = e.n;
  const long long nn = (long long)n * n;
  const long long gsz = (long long)gridDim.x * blockDim.x;
  const long long gtid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  double* A = e.A;
  double* B = e.B;
  double* V = e.V;
  for (long long i = gtid; i < nn; i += gsz) V[i] = (i / n == i % n) ? 1.0 : 0.0;
  const int m = n + (n & 1), npairs = m / 2;
  bool good = coop_barrier(e.ctl, gen);
  for (int sweep = 0; good && sweep < 40 && n > 1; ++sweep) {
    double off = 0.0, on = 0.0;
    for (long long i = gtid; i < nn; i += gsz) {
      const double a = A[i];
      if (i / n == i % n) on += a * a;
      else off += a * a;
    }
    off = dla::block_sum(off);
    on = dla::block_sum(on);
    if (threadIdx.x == 0) {
      e.part[2 * blockIdx.x] = off;
      e.part[2 * blockIdx.x + 1] = on;
    }
    if (!(good = coop_barrier(e.ctl, gen))) break;
    if (threadIdx.x == 0) {
      double so = 0.0, sn = 0.0;
      for (unsigned b = 0; b < gridDim.x; ++b) {
        so += *(volatile double*)&e.part[2 * b];
        sn += *(volatile double*)&e.part[2 * b + 1];
      }
      s_done = (so <= 1e-30 * sn) || (sn == 0.0);
    }
    __syncthreads();
    if (s_done) break;
    for (int r = 0; r < m - 1 && good; ++r) {
      for (int i = threadIdx.x; i < npairs; i += blockDim.x) {
        int p, q;
        dla::rr_pair(m, r, i, p, q);
        double c = 1.0, s = 0.0;
        if (q < n) {
          const double apq = A[p * n + q];
          const double app = A[p * n + p], aqq = A[q * n + q];
          if (apq != 0.0 && fabs(apq) > 1e-300) {
            const double tau = (aqq - app) / (2.0 * apq);
            const double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + t * t);
            s = t * c;
          }
        }
        rp[i] = p;
        rq[i] = q;
        rc[i] = c;
        rs[i] = s;
      }
      __syncthreads();
      // B = J^T A: rows p, q of each pair (an unpaired row is copied)
      for (long long idx = gtid; idx < (long long)npairs * n; idx += gsz) {
        const int i = (int)(idx / n), j = (int)(idx - (long long)i * n);
        const int p = rp[i], q = rq[i];
        if (q >= n) {
          B[p * n + j] = A[p * n + j];
          continue;
        }
        const double c = rc[i], s = rs[i];
        const double a = A[p * n + j], b = A[q * n + j];
        B[p * n + j] = c * a - s * b;
        B[q * n + j] = s * a + c * b;
      }
      if (!(good = coop_barrier(e.ctl, gen))) break;
      // A = B J and V = V J: columns p, q of each pair
      for (long long idx = gtid; idx < (long long)npairs * n; idx += gsz) {
        const int i = (int)(idx / n), j = (int)(idx - (long long)i * n);
        const int p = rp[i], q = rq[i];
        if (q >= n) {
          A[j * n + p] = B[j * n + p];
          continue;
        }
        const double c = rc[i], s = rs[i];
        double a = B[j * n + p], b = B[j * n + q];
        A[j * n + p] = c * a - s * b;
        A[j * n + q] = s * a + c * b;
        a = V[j * n + p];
        b = V[j * n + q];
        V[j * n + p] = c * a - s * b;
        V[j * n + q] = s * a + c * b;
      }
      good = coop_barrier(e.ctl, gen);
    }
  }
  if (!good) return;
  // eigenvalues in descending order (ties by index), eigenvectors as columns
  for (long long i = gtid; i < n; i += gsz) {
    const double di = A[i * n + i];
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      const double dj = A[(long long)j * n + j];
      if (dj > di || (dj == di && j < i)) ++rank;
    }
    e.w[rank] = di;
    for (int row = 0; row < n; ++row) e.Vs[(long long)row * n + rank] = V[(long long)row * n + i];
  }
  if (!coop_barrier(e.ctl, gen)) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) *e.rank_out = trunc_rank(e.w, n, e.delta, e.rmax);
}

// core_k(a, b, al) = Vs[(b*r + al), a]  for a < rnew
__global__ void k_core_from_V(int n, int r, int rnew, const double* __restrict__ Vs, double* __restrict__ core) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < rnew * n; i += gridDim.x * blockDim.x) {
    const int a = i / n, col = i - a * n;  // col = b*r + al
    core[i] = Vs[col * n + a];
  }
}

// Wn[row][a] = sum_x M[row][x] Vs[x][a]
__global__ void k_project(long long rows, int n, int rnew, const double* __restrict__ Mx,
                          const double* __restrict__ Vs, double* __restrict__ Wn) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < rows * rnew;
       i += (long long)gridDim.x * blockDim.x) {
    const long long row = i / rnew;
    const int a = (int)(i - row * rnew);
    double s = 0.0;
    for (int x = 0; x < n; ++x) s += Mx[row * n + x] * Vs[x * n + a];
    Wn[i] = s;
  }
}

// last core: core_1(0, b_1, al) = W[row with key b_1][al]
__global__ void k_first_core(long long rows, int r, const unsigned long long* __restrict__ key,
                             const double* __restrict__ W, double* __restrict__ core) {
  for (int i = threadIdx.x; i < 4 * r; i += blockDim.x) core[i] = 0.0;
  __syncthreads();
  for (int i = threadIdx.x; i < rows * r; i += blockDim.x) {
    const int row = i / r, a = i - row * r;
    core[(int)key[row] * r + a] = W[i];
  }
}

__global__ void k_sumsq(long long n, const double* __restrict__ v, double* out) {
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    s += v[i] * v[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __shared__ double sm[32];
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sm[w];
    out[blockIdx.x] = t;
  }
}

}  // namespace

// Workspace for the one-block linear algebra: three n x n matrices, n values, tmp.
struct LaWork {
  Buf &A, &V, &Vs, &w, &tmp, &misc;
};

static LaWork la(qp_ctx* c) { return LaWork{c->la[0], c->la[1], c->la[2], c->la[3], c->la[4], c->la[5]}; }

qp_qtt* tt_round_impl(qp_ctx* c, const qp_qtt* A, double eps, int rmax) {
  QP_REQUIRE(eps >= 0, QP_INVALID_ARG, "qtt_round: eps must be >= 0");
  QP_REQUIRE(rmax >= 1, QP_INVALID_ARG, "qtt_round: rmax must be >= 1");
  const int d = A->d;
  long long cap = 1;
  int nmax = 1;
  for (int k = 0; k < d; ++k) {
    cap = std::max(cap, A->offset[k + 1] - A->offset[k]);
    nmax = std::max(nmax, A->ranks[k]);
  }
  nmax = std::max(nmax, A->ranks[d]);
  QP_REQUIRE(nmax <= 512, QP_INVALID_ARG, "qtt_round: ranks above 512 are not supported");
  LaWork w = la(c);
  double* cores = static_cast<double*>(w.misc.ensure((size_t)d * cap * sizeof(double) + (d + 1) * sizeof(int) + 64));
  int* ranks = reinterpret_cast<int*>(cores + (size_t)d * cap);
  const size_t n2 = (size_t)nmax * nmax * sizeof(double);
  RoundArgs a;
  a.d = d;
  a.eps = eps;
  a.rmax = rmax;
  a.ranks = ranks;
  a.cap = cap;
  a.cores = cores;
  a.A = static_cast<double*>(w.A.ensure(n2));
  a.V = static_cast<double*>(w.V.ensure(n2));
  a.Vs = static_cast<double*>(w.Vs.ensure(n2));
  a.w = static_cast<double*>(w.w.ensure((size_t)nmax * sizeof(double) + 64));
  a.tmp = static_cast<double*>(w.tmp.ensure((size_t)cap * sizeof(double)));
  a.norm_out = nullptr;
  for (int k = 0; k < d; ++k)
    QP_CUDA(cudaMemcpyAsync(cores + (size_t)k * cap, A->cores + A->offset[k],
                            (A->offset[k + 1] - A->offset[k]) * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  QP_CUDA(cudaMemcpyAsync(ranks, A->ranks.data(), (d + 1) * sizeof(int), cudaMemcpyHostToDevice, c->stream));
  QP_CUDA(cudaFuncSetAttribute(k_tt_round, cudaFuncAttributeMaxDynamicSharedMemorySize, dla::SYEV_SMEM_BYTES));
  k_tt_round<<<1, LT, dla::SYEV_SMEM_BYTES, c->stream>>>(a);
  QP_CUDA(cudaGetLastError());
  std::vector<int> r(d + 1);
  QP_CUDA(cudaMemcpyAsync(r.data(), ranks, (d + 1) * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  QP_CUDA(cudaStreamSynchronize(c->stream));
  qp_qtt* out = qtt_alloc(c, d, r);
  out->scaled = A->scaled;
  for (int k = 0; k < d; ++k)
    QP_CUDA(cudaMemcpyAsync(out->cores + out->offset[k], cores + (size_t)k * cap,
                            (out->offset[k + 1] - out->offset[k]) * sizeof(double), cudaMemcpyDeviceToDevice,
                            c->stream));
  QP_CUDA(cudaStreamSynchronize(c->stream));
  return out;
}

// Right-to-left sparse TT-SVD of the padded Schur matrix (or N when H == null).
qp_qtt* compress_impl(qp_ctx* c, bool with_H, double eps, int rmax, const double* rowscale) {
  QP_REQUIRE(c->have_contacts, QP_NOT_READY, "qtt_compress: no contacts");
  QP_REQUIRE(eps >= 0 && rmax >= 1, QP_INVALID_ARG, "qtt_compress: eps >= 0 and rmax >= 1 required");
  if (rmax > 128) rmax = 128;  // unfoldings have 4 r columns; the one-block eigensolver takes n <= 512
  cudaStream_t st = c->stream;
  const int d = c->L, M = c->M, Nc = c->Nc, slots = c->slots;
  const long long P = c->P;
  LaWork w = la(c);
  // 1. offsets of off-diagonal blocks
  Buf& b_cnt = c->scratch[0];
  int* cnt = static_cast<int*>(b_cnt.ensure(sizeof(int) * (2 * (size_t)M + 4)));
  int* off = cnt + M + 1;
  k_pair_count<<<ceil_div(M + 1, 256), 256, 0, st>>>(M, c->bptr.as<int>(), cnt);
  size_t tb = 0;
  cub::DeviceScan::ExclusiveSum(nullptr, tb, cnt, off, M + 1, st);
  void* tmp = c->scratch[1].ensure(tb);
  QP_CUDA(cub::DeviceScan::ExclusiveSum(tmp, tb, cnt, off, M + 1, st));
  int noff = 0;
  QP_CUDA(cudaMemcpyAsync(&noff, off + M, sizeof(int), cudaMemcpyDeviceToHost, st));
  QP_CUDA(cudaStreamSynchronize(st));
  const long long per = slots == 4 ? 10 : 9;
  const long long nent = 9LL * noff + per * Nc + (P - (long long)slots * Nc);
  // 2. entries (key, value), sorted by key
  unsigned long long* key = static_cast<unsigned long long*>(c->scratch[2].ensure(2 * nent * sizeof(unsigned long long)));
  unsigned long long* key_s = key + nent;
  double* val = static_cast<double*>(c->scratch[3].ensure(2 * nent * sizeof(double)));
  double* val_s = val + nent;
  EntryArgs e;
  e.M = M;
  e.Nc = Nc;
  e.slots = slots;
  e.d = d;
  e.P = P;
  e.rec = c->rec64.as<double>();
  e.ca = c->ca.as<int>();
  e.cb = c->cb.as<int>();
  e.inv_m = c->inv_m.as<double>();
  e.inv_I = c->inv_I.as<double>();
  e.bptr = c->bptr.as<int>();
  e.inc = c->inc.as<int>();
  e.H = with_H ? c->H.as<double>() : nullptr;
  e.off = off;
  e.rs = rowscale;
  e.key = key;
  e.val = val;
  if (M > 0) k_entries_offdiag<<<ceil_div(M, 128), 128, 0, st>>>(e);
  if (Nc > 0) k_entries_diag<<<ceil_div(Nc, 128), 128, 0, st>>>(e, 9LL * noff);
  k_entries_tail<<<c->num_sms * 4, 256, 0, st>>>(e, 9LL * noff + per * Nc);
  QP_CUDA(cudaGetLastError());
  tb = 0;
  cub::DeviceRadixSort::SortPairs(nullptr, tb, key, key_s, val, val_s, nent, 0, 2 * d, st);
  tmp = c->scratch[1].ensure(tb);
  QP_CUDA(cub::DeviceRadixSort::SortPairs(tmp, tb, key, key_s, val, val_s, nent, 0, 2 * d, st));
  // 3. ||S||_F and delta
  // [0, 256): norm partials; 512: rank; [1024, 1024 + 2 x blocks): eigensolver partials
  double* part = static_cast<double*>(w.tmp.ensure((1024 + 4096) * sizeof(double)));
  k_sumsq<<<256, 256, 0, st>>>(nent, val_s, part);
  std::vector<double> hp(256);
  QP_CUDA(cudaMemcpyAsync(hp.data(), part, 256 * sizeof(double), cudaMemcpyDeviceToHost, st));
  QP_CUDA(cudaStreamSynchronize(st));
  double nrm2 = 0.0;
  for (double v : hp) nrm2 += v;
  const double delta = eps * std::sqrt(nrm2) / std::sqrt((double)std::max(d - 1, 1));
  // 4. sweep right to left
  std::vector<int> ranks(d + 1, 1);
  qp_qtt* out = nullptr;
  // cores are produced last-to-first; keep them in device scratch until ranks are known
  std::vector<Buf*> core_bufs;
  std::vector<Buf> cb_store(d);
  long long rows = nent;
  int r = 1;
  unsigned long long* K = key_s;
  unsigned long long* Kalt = key;
  double* W = val_s;
  Buf& b_flag = c->scratch[4];
  Buf& b_M = c->scratch[5];
  Buf& b_W = c->scratch[6];
  Buf& b_part = c->scratch[7];
  for (int k = d; k >= 2; --k) {
    int* flag = static_cast<int*>(b_flag.ensure(2 * rows * sizeof(int) + 64));
    int* pid = flag + rows;
    k_parent_flags<<<c->num_sms * 8, 256, 0, st>>>(rows, K, flag);
    tb = 0;
    cub::DeviceScan::InclusiveSum(nullptr, tb, flag, pid, rows, st);
    tmp = c->scratch[1].ensure(tb);
    QP_CUDA(cub::DeviceScan::InclusiveSum(tmp, tb, flag, pid, rows, st));
    int npar = 0;
    QP_CUDA(cudaMemcpyAsync(&npar, pid + rows - 1, sizeof(int), cudaMemcpyDeviceToHost, st));
    QP_CUDA(cudaStreamSynchronize(st));
    const int n = 4 * r;
    double* Mx = static_cast<double*>(b_M.ensure((size_t)npar * n * sizeof(double)));
    QP_CUDA(cudaMemsetAsync(Mx, 0, (size_t)npar * n * sizeof(double), st));
    k_scatter_rows<<<c->num_sms * 8, 256, 0, st>>>(rows, r, K, pid, W, Mx, Kalt);
    // Gram: register-tiled partials for n <= 64, one entry per thread above
    double* G = static_cast<double*>(w.A.ensure((size_t)n * n * sizeof(double)));
    if (n <= 64) {
      const int nparts = (int)std::min<long long>(2 * c->num_sms, std::max<long long>(1, npar / 256));
      const long long chunk = (npar + nparts - 1) / nparts;
      double* gp = static_cast<double*>(b_part.ensure((size_t)nparts * n * n * sizeof(double)));
      QP_CUDA(cudaFuncSetAttribute(k_gram_tiled, cudaFuncAttributeMaxDynamicSharedMemorySize, GR_SMEM));
      k_gram_tiled<<<nparts, 256, GR_SMEM, st>>>(npar, n, Mx, gp, chunk);
      k_gram_reduce<<<ceil_div((long long)n * n, 256), 256, 0, st>>>(nparts, n, gp, G);
    } else {
      const int nparts = (int)std::min<long long>(256, std::max<long long>(1, npar / 64));
      const long long chunk = (npar + nparts - 1) / nparts;
      double* gp = static_cast<double*>(b_part.ensure((size_t)nparts * n * n * sizeof(double)));
      k_gram_partial<<<nparts, 256, 0, st>>>(npar, n, Mx, gp, chunk);
      k_gram_reduce<<<ceil_div((long long)n * n, 256), 256, 0, st>>>(nparts, n, gp, G);
    }
    EigArgs ea;
    ea.A = G;
    ea.V = static_cast<double*>(w.V.ensure((size_t)n * n * sizeof(double)));
    ea.Vs = static_cast<double*>(w.Vs.ensure((size_t)n * n * sizeof(double)));
    ea.w = static_cast<double*>(w.w.ensure((size_t)n * sizeof(double) + 64));
    ea.n = n;
    ea.delta = delta;
    ea.rmax = rmax;
    int* rk_dev = reinterpret_cast<int*>(static_cast<double*>(w.tmp.p) + 512);
    ea.rank_out = rk_dev;
    if (n <= dla::SYEV_SMEM_N) {
      QP_CUDA(cudaFuncSetAttribute(k_eig_trunc, cudaFuncAttributeMaxDynamicSharedMemorySize, dla::SYEV_SMEM_BYTES));
      k_eig_trunc<<<1, LT, dla::SYEV_SMEM_BYTES, st>>>(ea);
      QP_CUDA(cudaGetLastError());
    } else {
      // larger Gram matrices: the rotation rounds on a cooperative grid
      EigCoopArgs ec{G, static_cast<double*>(w.misc.ensure((size_t)n * n * sizeof(double))), ea.V, ea.Vs, ea.w, n,
                     delta, rmax, rk_dev, c->ctl.as<DevCtl>(),
                     static_cast<double*>(w.tmp.p) + 1024};
      QP_CUDA(cudaMemsetAsync(c->ctl.p, 0, sizeof(DevCtl), st));
      int per_sm = 0;
      QP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_eig_coop, 256, 0));
      const int grid = std::min(c->num_sms * std::max(per_sm, 1), std::max(1, (n / 2) * n / 256));
      void* args[] = {&ec};
      QP_CUDA(cudaLaunchCooperativeKernel((const void*)k_eig_coop, dim3(grid), dim3(256), args, 0, st));
      DevCtl hc;
      QP_CUDA(cudaMemcpyAsync(&hc, c->ctl.p, sizeof(DevCtl), cudaMemcpyDeviceToHost, st));
      QP_CUDA(cudaStreamSynchronize(st));
      QP_REQUIRE(hc.err == 0, QP_TIMEOUT, "qtt_compress: eigensolver grid barrier wait expired");
    }
    int rnew = 1;
    QP_CUDA(cudaMemcpyAsync(&rnew, rk_dev, sizeof(int), cudaMemcpyDeviceToHost, st));
    QP_CUDA(cudaStreamSynchronize(st));
    rnew = std::min(rnew, npar);  // rank cannot exceed the number of nonzero rows
    if (rnew < 1) rnew = 1;
    ranks[k - 1] = rnew;
    // core k (1-based) -> index k-1: shape (rnew, 4, r)
    double* core = static_cast<double*>(cb_store[k - 1].ensure((size_t)rnew * n * sizeof(double)));
    k_core_from_V<<<ceil_div((long long)rnew * n, 256), 256, 0, st>>>(n, r, rnew, ea.Vs, core);
    double* Wn = static_cast<double*>(b_W.ensure((size_t)npar * rnew * sizeof(double)));
    k_project<<<c->num_sms * 8, 256, 0, st>>>(npar, n, rnew, Mx, ea.Vs, Wn);
    QP_CUDA(cudaGetLastError());
    // next level: rows = parents
    rows = npar;
    r = rnew;
    std::swap(K, Kalt);
    // W must not alias the next level's M: copy into the value scratch
    double* Wkeep = static_cast<double*>(c->scratch[3].ensure((size_t)rows * r * sizeof(double) * 2));
    QP_CUDA(cudaMemcpyAsync(Wkeep, Wn, (size_t)rows * r * sizeof(double), cudaMemcpyDeviceToDevice, st));
    W = Wkeep;
    // keys: K now points to the parent keys written by k_scatter_rows into Kalt (swapped)
  }
  // first core (k = 1): rows <= 4 with keys b_1
  QP_REQUIRE(rows <= 4, QP_CUDA_ERROR, "qtt_compress: inconsistent top level");
  double* core0 = static_cast<double*>(cb_store[0].ensure((size_t)4 * r * sizeof(double)));
  k_first_core<<<1, 256, 0, st>>>(rows, r, K, W, core0);
  QP_CUDA(cudaGetLastError());
  out = qtt_alloc(c, d, ranks);
  for (int k = 0; k < d; ++k)
    QP_CUDA(cudaMemcpyAsync(out->cores + out->offset[k], cb_store[k].p,
                            (out->offset[k + 1] - out->offset[k]) * sizeof(double), cudaMemcpyDeviceToDevice, st));
  QP_CUDA(cudaStreamSynchronize(st));
  for (auto& b : cb_store) b.release();
  out->scaled = rowscale ? 1 : 0;
  return out;
}

}  // namespace qp

using namespace qp;

extern "C" {

int qtt_round(qp_ctx_t c, qtt_t A, double eps, int rmax, qtt_t* out) {
  if (!c || !A || !out) return QP_INVALID_ARG;
  try {
    QP_CUDA(cudaSetDevice(c->device));
    *out = tt_round_impl(c, A, eps, rmax);
  } catch (const Error& e) {
    set_error(c, e);
    return e.code;
  }
  return QP_OK;
}

int qtt_compress(qp_ctx_t c, const qp_state* st, double eps, int rmax, qtt_t* out) {
  if (!c || !out) return QP_INVALID_ARG;
  try {
    QP_CUDA(cudaSetDevice(c->device));
    if (st) {
      QP_REQUIRE(st->gamma && st->lambda, QP_INVALID_ARG, "qtt_compress: state with null gamma/lambda");
      launch_schur_blocks(c, st->gamma, st->lambda);
    }
    *out = compress_impl(c, st != nullptr, eps, rmax, nullptr);
  } catch (const Error& e) {
    set_error(c, e);
    return e.code;
  }
  return QP_OK;
}


}  // extern "C"
