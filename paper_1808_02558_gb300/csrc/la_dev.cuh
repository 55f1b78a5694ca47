// Small dense FP64 linear algebra inside one thread block, shared by the QTT
// compression, rounding and inversion: a block sum, and the symmetric
// eigendecomposition by cyclic Jacobi with round-robin (parallel) rotation
// order (Golub and Van Loan, Matrix Computations, Sec. 8.5), eigenvalues in
// descending order, and the truncation rank of Sec. 3.1.
//
// GB300's FP64 pipe is narrow and an L2 round trip costs hundreds of cycles,
// so a matrix of order n <= SYEV_SMEM_N is copied into shared memory (the
// calling kernel launches with SYEV_SMEM_BYTES of dynamic shared memory) and
// every rotation round works there; larger matrices are rotated in place in
// global memory.
#pragma once

namespace qp {
namespace dla {

constexpr int SYEV_SMEM_N = 64;
constexpr int SYEV_SMEM_BYTES = 2 * SYEV_SMEM_N * SYEV_SMEM_N * (int)sizeof(double);

__device__ inline double block_sum(double v) {
  __shared__ double sm[32];
  __shared__ double res;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double x = (threadIdx.x < (blockDim.x >> 5)) ? sm[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (threadIdx.x == 0) res = x;
  }
  __syncthreads();
  double out = res;
  __syncthreads();
  return out;
}

// Round-robin pairing of m (even) players: round r, pair i.
__device__ __forceinline__ void rr_pair(int m, int r, int i, int& p, int& q) {
  if (i == 0) {
    p = m - 1;
    q = r;
  } else {
    p = (r + i) % (m - 1);
    q = (r - i + (m - 1)) % (m - 1);
  }
  if (p > q) {
    const int t = p;
    p = q;
    q = t;
  }
}

// Rotation (c, s) annihilating a_pq of the 2 x 2 block [[a_pp, a_pq], [a_pq,
// a_qq]] (a_pq != 0).  precise: the angle in FP64.  Otherwise the angle comes
// from FP32 arithmetic on the block scaled by a power of two (FP64 division and
// square root are long dependent sequences on GB300's narrow FP64 pipe), and
// (c, s) is made a rotation to FP64 rounding by two Newton steps towards
// c^2 + s^2 = 1: the rotation stays exactly orthogonal and only its angle
// carries the FP32 error, which the next sweep removes (the sweeps switch to
// precise angles once the off-diagonal part is small).
__device__ __forceinline__ void jacobi_rotation(double app, double aqq, double apq, bool precise, double& c,
                                                double& s) {
  if (!precise) {
    const double num = aqq - app, den = 2.0 * apq;
    int e;
    frexp(fmax(fabs(num), fabs(den)), &e);
    const float nf = (float)ldexp(num, -e), df = (float)ldexp(den, -e);
    if (df != 0.0f && isfinite(nf / df)) {
      const float tau = nf / df;
      // large |tau|: t = 1 / (2 tau) to FP32 rounding (tau^2 would overflow)
      const float t = fabsf(tau) > 1e18f ? 0.5f / tau
                                         : (tau >= 0.0f ? 1.0f : -1.0f) / (fabsf(tau) + sqrtf(1.0f + tau * tau));
      const float cf = rsqrtf(1.0f + t * t);
      double cc = (double)cf, ss = (double)(t * cf);
      for (int it = 0; it < 2; ++it) {
        const double f = 1.5 - 0.5 * (cc * cc + ss * ss);
        cc *= f;
        ss *= f;
      }
      c = cc;
      s = ss;
      return;
    }
  }
  const double tau = (aqq - app) / (2.0 * apq);
  const double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
  c = 1.0 / sqrt(1.0 + t * t);
  s = t * c;
}

// Jacobi sweeps on A (n x n, row-major, destroyed); V accumulates the
// rotations (starts as I).  A and V may live in shared or global memory.
__device__ inline void jacobi_sweeps(double* A, double* V, int n) {
  __shared__ double rc[256], rs[256];
  __shared__ int rp[256], rq[256];
  __shared__ int done, precise;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int i = tid; i < n * n; i += nt) V[i] = (i / n == i % n) ? 1.0 : 0.0;
  __syncthreads();
  const int m = n + (n & 1);
  const int npairs = m / 2;
  for (int sweep = 0; sweep < 40 && n > 1; ++sweep) {
    double off = 0.0, on = 0.0;
    for (int i = tid; i < n * n; i += nt) {
      const double a = A[i];
      if (i / n == i % n) on += a * a;
      else off += a * a;
    }
    off = block_sum(off);
    on = block_sum(on);
    if (tid == 0) {
      done = (off <= 1e-30 * on) || (on == 0.0);
      precise = off <= 1e-16 * on;  // off-diagonal below 1e-8 of the diagonal: FP64 angles
    }
    __syncthreads();
    if (done) break;
    const bool prec = precise != 0;
    for (int r = 0; r < m - 1; ++r) {
      for (int i = tid; i < npairs; i += nt) {
        int p, q;
        rr_pair(m, r, i, p, q);
        double c = 1.0, s = 0.0;
        if (q < n) {
          const double apq = A[p * n + q];
          const double app = A[p * n + p], aqq = A[q * n + q];
          if (apq != 0.0 && fabs(apq) > 1e-300) jacobi_rotation(app, aqq, apq, prec, c, s);
        }
        rp[i] = p;
        rq[i] = q;
        rc[i] = c;
        rs[i] = s;
      }
      __syncthreads();
      // A <- J^T A J in one pass: J is block diagonal in the pairs, so the 2 x 2
      // block of rows (p_i, q_i) and columns (p_j, q_j) becomes J_i^T A_ij J_j;
      // A stays symmetric, so a thread forms block (i, j), i <= j, and writes its
      // transpose into block (j, i) as well (a missing q of the odd pair is left
      // out); V <- V J for one row and pair per thread
      const int nblk = npairs * (npairs + 1) / 2;
      for (int idx = tid; idx < nblk + npairs * n; idx += nt) {
        if (idx < nblk) {
          // block index -> (i, j), i <= j: row i holds npairs - i blocks
          int i = 0, rem = idx;
          while (rem >= npairs - i) {
            rem -= npairs - i;
            ++i;
          }
          const int j = i + rem;
          const int p = rp[i], q = rq[i], p2 = rp[j], q2 = rq[j];
          const double ci = rc[i], si = rs[i], cj = rc[j], sj = rs[j];
          if (si == 0.0 && sj == 0.0) continue;
          const bool hq = q < n, hq2 = q2 < n;
          const double a00 = A[p * n + p2], a01 = hq2 ? A[p * n + q2] : 0.0;
          const double a10 = hq ? A[q * n + p2] : 0.0, a11 = (hq && hq2) ? A[q * n + q2] : 0.0;
          // rows: (J_i^T A): row p <- c a_p - s a_q, row q <- s a_p + c a_q
          const double b00 = ci * a00 - si * a10, b01 = ci * a01 - si * a11;
          const double b10 = si * a00 + ci * a10, b11 = si * a01 + ci * a11;
          // columns: (. J_j): col p2 <- c b_p2 - s b_q2, col q2 <- s b_p2 + c b_q2
          const double c00 = cj * b00 - sj * b01, c01 = sj * b00 + cj * b01;
          const double c10 = cj * b10 - sj * b11, c11 = sj * b10 + cj * b11;
          A[p * n + p2] = c00;
          if (hq2) A[p * n + q2] = c01;
          if (hq) A[q * n + p2] = c10;
          if (hq && hq2) A[q * n + q2] = c11;
          if (i != j) {  // the mirrored block (j, i)
            A[p2 * n + p] = c00;
            if (hq2) A[q2 * n + p] = c01;
            if (hq) A[p2 * n + q] = c10;
            if (hq && hq2) A[q2 * n + q] = c11;
          }
        } else {
          const int u = idx - nblk, i = u / n, j = u - i * n;
          const int p = rp[i], q = rq[i];
          if (q >= n || rs[i] == 0.0) continue;
          const double c = rc[i], s = rs[i];
          const double a = V[j * n + p], b = V[j * n + q];
          V[j * n + p] = c * a - s * b;
          V[j * n + q] = s * a + c * b;
        }
      }
      __syncthreads();
    }
  }
}

// Eigendecomposition of the symmetric n x n matrix A (row-major, destroyed):
// w[0..n) the eigenvalues in descending order (ties by index), Vs the
// eigenvectors as columns (row-major n x n); V is workspace n x n.  `smem`
// points at SYEV_SMEM_BYTES of the block's dynamic shared memory, or is null.
__device__ inline void syev(double* A, double* V, double* Vs, double* w, int n, double* smem) {
  const int tid = threadIdx.x, nt = blockDim.x;
  double* a = A;
  double* v = V;
  if (smem && n <= SYEV_SMEM_N) {
    a = smem;
    v = smem + n * n;
    for (int i = tid; i < n * n; i += nt) a[i] = A[i];
    __syncthreads();
  }
  jacobi_sweeps(a, v, n);
  for (int i = tid; i < n; i += nt) {
    const double di = a[i * n + i];
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      const double dj = a[j * n + j];
      if (dj > di || (dj == di && j < i)) ++rank;
    }
    w[rank] = di;
    for (int row = 0; row < n; ++row) Vs[row * n + rank] = v[row * n + i];
  }
  __syncthreads();
}

// One-sided (Hestenes) Jacobi: the k vectors of length L, element e of vector
// i at X[i sv + e se], are made mutually orthogonal by plane rotations applied
// to the vectors themselves (no Gram matrix, so singular values down to FP64
// rounding of the largest are resolved; Demmel and Veselic, SIAM J. Matrix
// Anal. Appl. 13 (1992)).  Vr (k x k, row-major) accumulates the rotations:
// with the vectors as columns, X_new = X_old Vr.  A warp handles one pair of a
// round-robin round; sweeps stop when no pair had |x_p.x_q| above
// sqrt(L) eps sqrt(|x_p|^2 |x_q|^2).
__device__ inline void osj(double* X, int k, int L, long long sv, long long se, double* Vr) {
  __shared__ int s_rot;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  for (int i = tid; i < k * k; i += nt) Vr[i] = (i / k == i % k) ? 1.0 : 0.0;
  const double tol = sqrt((double)L) * 2.2e-16;
  const int m = k + (k & 1), npairs = m / 2;
  __syncthreads();
  for (int sweep = 0; sweep < 60 && k > 1; ++sweep) {
    if (tid == 0) s_rot = 0;
    __syncthreads();
    for (int r = 0; r < m - 1; ++r) {
      for (int i = warp; i < npairs; i += nw) {
        int p, q;
        rr_pair(m, r, i, p, q);
        if (q >= k) continue;
        double al = 0.0, be = 0.0, ga = 0.0;
        for (int e = lane; e < L; e += 32) {
          const double xp = X[p * sv + e * se], xq = X[q * sv + e * se];
          al += xp * xp;
          be += xq * xq;
          ga += xp * xq;
        }
        for (int o = 16; o > 0; o >>= 1) {
          al += __shfl_xor_sync(0xffffffffu, al, o);
          be += __shfl_xor_sync(0xffffffffu, be, o);
          ga += __shfl_xor_sync(0xffffffffu, ga, o);
        }
        if (fabs(ga) > 1e-300 && fabs(ga) > tol * sqrt(al * be)) {
          const double zeta = (be - al) / (2.0 * ga);
          const double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
          const double c = 1.0 / sqrt(1.0 + t * t), sn = t * c;
          for (int e = lane; e < L; e += 32) {
            const double xp = X[p * sv + e * se], xq = X[q * sv + e * se];
            X[p * sv + e * se] = c * xp - sn * xq;
            X[q * sv + e * se] = sn * xp + c * xq;
          }
          for (int j = lane; j < k; j += 32) {
            const double vp = Vr[j * k + p], vq = Vr[j * k + q];
            Vr[j * k + p] = c * vp - sn * vq;
            Vr[j * k + q] = sn * vp + c * vq;
          }
          if (lane == 0) s_rot = 1;
        }
      }
      __syncthreads();
    }
    const int any = s_rot;
    __syncthreads();
    if (!any) break;
  }
}

// Norms of the k vectors of X (as in osj) into sig, and ord[j] = the index of
// the j-th largest (ties by index).
__device__ inline void osj_norms(const double* X, int k, int L, long long sv, long long se, double* sig, int* ord) {
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int i = tid; i < k; i += nt) {
    double s = 0.0;
    for (int e = 0; e < L; ++e) s += X[i * sv + e * se] * X[i * sv + e * se];
    sig[i] = sqrt(s);
  }
  __syncthreads();
  for (int i = tid; i < k; i += nt) {
    int rank = 0;
    for (int j = 0; j < k; ++j)
      if (sig[j] > sig[i] || (sig[j] == sig[i] && j < i)) ++rank;
    ord[rank] = i;
  }
  __syncthreads();
}

// Smallest r with sqrt(sum_{l >= r} lambda_l) <= delta, 1 <= r <= min(rmax, n)
// (eigenvalues of a Gram matrix, descending: the squared singular values).
__device__ inline int trunc_rank(const double* lam, int n, double delta, int rmax) {
  double tail = 0.0;
  int r = n;
  for (int k = n - 1; k >= 1; --k) {
    tail += fmax(lam[k], 0.0);
    if (sqrt(tail) <= delta) r = k;
    else break;
  }
  if (r > rmax) r = rmax;
  if (r < 1) r = 1;
  return r;
}

}  // namespace dla
}  // namespace qp
