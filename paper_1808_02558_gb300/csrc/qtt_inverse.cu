// QTT approximate inverse (Sec. 3.2 "TT inversion", Sec. 3.3 inverse update).
//
// X ~ S^-1 is sought in QTT format by minimising, one pair of neighbouring
// cores at a time, the residual of S X = I projected on the frame of the other
// cores (two-site alternating linear scheme: the "ALS with rank increase" the
// paper refers to, in its DMRG form).  The operator acting on X is S on the row
// index only, so the local operator of cores (k, k+1) is
//   y(b,i1,j1,i2,j2,c) = sum PhiL(b,s0,b') S_k(s0,i1,l1,s1) S_k+1(s1,i2,l2,s2)
//                             PhiR(c,s2,c') w(b',l1,j1,l2,j2,c'),
// the local right-hand side is PsiL(b) [i1=j1] [i2=j2] PsiR(c), and the local
// system is solved by BiCGSTAB (the compressed S need not be exactly symmetric
// or definite).  The solved supercore is split by a truncated SVD (rank chosen
// with the TT truncation rule), which is where ranks grow or shrink.
//
// Everything runs in one thread block: local solves and contractions in FP32,
// the SVD splits through FP64 Gram eigenpairs.
#include <algorithm>
#include <cmath>

#include "internal.cuh"
#include "la_dev.cuh"

namespace qp {
namespace {

constexpr int DT = 1024;

__device__ inline double blk_sum(double v) { return dla::block_sum(v); }

extern __shared__ double la_smem[];

__device__ inline void blk_syev(double* A, double* V, double* Vs, double* w, int n) {
  dla::syev(A, V, Vs, w, n, la_smem);
}

struct DmrgArgs {
  int d, sweeps, rmax, local_maxit;
  double eps, local_tol;
  // operator S (FP32 cores), ranks s[0..d], offsets
  const float* S;
  const int* sr;
  const long long* soff;
  int smax;
  // unknown X: FP32 cores in slots of `xcap` values, ranks xr[0..d] (in/out)
  float* X;
  int* xr;
  long long xcap;
  // interfaces: PhiL[t], PhiR[t] slots of `phicap` values; PsiL/PsiR slots of rmax
  float* PhiL;
  float* PhiR;
  long long phicap;
  float* PsiL;
  float* PsiR;
  // local work (wcap values each): W, b, BiCGSTAB vectors, contraction temporaries (tcap)
  float* W;
  float* B;
  float* v[6];
  long long wcap;
  float* T1;
  float* T2;
  float* T3;
  long long tcap;
  // FP64 split workspace
  double* G;
  double* V;
  double* Vs;
  double* ev;
  double* norms;  // diagnostics: [0] last local residual, [1] max local iterations
};

__device__ __forceinline__ const float* Score(const DmrgArgs& a, int k) { return a.S + a.soff[k]; }
__device__ __forceinline__ float* Xcore(const DmrgArgs& a, int k) { return a.X + (long long)k * a.xcap; }
__device__ __forceinline__ float* PL(const DmrgArgs& a, int t) { return a.PhiL + (long long)t * a.phicap; }
__device__ __forceinline__ float* PR(const DmrgArgs& a, int t) { return a.PhiR + (long long)t * a.phicap; }

// y = A_loc w for the pair (k, k+1); rl = xr[k], rr = xr[k+2]
__device__ void local_apply(const DmrgArgs& a, int k, int rl, int rr, const float* w, float* y) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int sl = a.sr[k], sm = a.sr[k + 1], sr = a.sr[k + 2];
  const float* pl = PL(a, k);
  const float* pr = PR(a, k + 2);
  const float* S0 = Score(a, k);
  const float* S1 = Score(a, k + 1);
  // T1[s0][b][q][c'] = sum_b' PhiL(b, s0, b') w[b'][q][c']
  const long long n1 = (long long)sl * rl * 16 * rr;
  for (long long i = tid; i < n1; i += nt) {
    long long t = i;
    const int cp = (int)(t % rr); t /= rr;
    const int q = (int)(t % 16); t /= 16;
    const int b = (int)(t % rl); t /= rl;
    const int s0 = (int)t;
    float s = 0.f;
    for (int bp = 0; bp < rl; ++bp) s += pl[(b * sl + s0) * rl + bp] * w[((long long)bp * 16 + q) * rr + cp];
    a.T1[i] = s;
  }
  __syncthreads();
  // T2[b][s1][q'][c'] = sum_{s0,l1} S_k(s0,i1,l1,s1) T1[s0][b][(l1,j1,l2,j2)][c'],  q' = (i1,j1,l2,j2)
  const long long n2 = (long long)rl * sm * 16 * rr;
  for (long long i = tid; i < n2; i += nt) {
    long long t = i;
    const int cp = (int)(t % rr); t /= rr;
    const int q = (int)(t % 16); t /= 16;
    const int s1 = (int)(t % sm); t /= sm;
    const int b = (int)t;
    const int i1 = q >> 3, rest = q & 7;
    float s = 0.f;
    for (int s0 = 0; s0 < sl; ++s0)
      for (int l1 = 0; l1 < 2; ++l1)
        s += S0[((s0 * 2 + i1) * 2 + l1) * sm + s1] * a.T1[(((long long)s0 * rl + b) * 16 + (l1 << 3 | rest)) * rr + cp];
    a.T2[i] = s;
  }
  __syncthreads();
  // T3[b][q''][s2][c'] = sum_{s1,l2} S_k+1(s1,i2,l2,s2) T2[b][s1][(i1,j1,l2,j2)][c'],  q'' = (i1,j1,i2,j2)
  const long long n3 = (long long)rl * 16 * sr * rr;
  for (long long i = tid; i < n3; i += nt) {
    long long t = i;
    const int cp = (int)(t % rr); t /= rr;
    const int s2 = (int)(t % sr); t /= sr;
    const int q = (int)(t % 16); t /= 16;
    const int b = (int)t;
    const int i2 = (q >> 1) & 1, j2 = q & 1, hi = q & 12;
    float s = 0.f;
    for (int s1 = 0; s1 < sm; ++s1)
      for (int l2 = 0; l2 < 2; ++l2)
        s += S1[((s1 * 2 + i2) * 2 + l2) * sr + s2] * a.T2[(((long long)b * sm + s1) * 16 + (hi | (l2 << 1) | j2)) * rr + cp];
    a.T3[i] = s;
  }
  __syncthreads();
  // y[b][q''][c] = sum_{s2,c'} PhiR(c, s2, c') T3[b][q''][s2][c']
  const long long n4 = (long long)rl * 16 * rr;
  for (long long i = tid; i < n4; i += nt) {
    long long t = i;
    const int c = (int)(t % rr); t /= rr;
    const int q = (int)(t % 16); t /= 16;
    const int b = (int)t;
    float s = 0.f;
    for (int s2 = 0; s2 < sr; ++s2)
      for (int cp = 0; cp < rr; ++cp)
        s += pr[(c * sr + s2) * rr + cp] * a.T3[(((long long)b * 16 + q) * sr + s2) * rr + cp];
    y[i] = s;
  }
  __syncthreads();
}

__device__ double dotf(const float* x, const float* y, long long n) {
  double s = 0.0;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) s += (double)x[i] * (double)y[i];
  return blk_sum(s);
}

// BiCGSTAB on A_loc x = b, x holds the warm start.  Returns the relative residual.
__device__ double local_solve(const DmrgArgs& a, int k, int rl, int rr, float* x, const float* b, int& its) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const long long n = (long long)rl * 16 * rr;
  float *r = a.v[0], *rh = a.v[1], *p = a.v[2], *v = a.v[3], *s = a.v[4], *t = a.v[5];
  local_apply(a, k, rl, rr, x, v);
  for (long long i = tid; i < n; i += nt) {
    float ri = b[i] - v[i];
    r[i] = ri;
    rh[i] = ri;
    p[i] = 0.f;
    v[i] = 0.f;
  }
  __syncthreads();
  const double bn = sqrt(dotf(b, b, n));
  double rn = sqrt(dotf(r, r, n));
  its = 0;
  if (bn == 0.0) return 0.0;
  double rho = 1.0, alpha = 1.0, omega = 1.0;
  while (its < a.local_maxit && rn > a.local_tol * bn) {
    const double rho1 = dotf(rh, r, n);
    if (rho1 == 0.0 || omega == 0.0) break;
    const double beta = (rho1 / rho) * (alpha / omega);
    rho = rho1;
    for (long long i = tid; i < n; i += nt) p[i] = r[i] + (float)beta * (p[i] - (float)omega * v[i]);
    __syncthreads();
    local_apply(a, k, rl, rr, p, v);
    const double rv = dotf(rh, v, n);
    if (rv == 0.0) break;
    alpha = rho / rv;
    for (long long i = tid; i < n; i += nt) s[i] = r[i] - (float)alpha * v[i];
    __syncthreads();
    local_apply(a, k, rl, rr, s, t);
    const double tt = dotf(t, t, n);
    omega = tt > 0.0 ? dotf(t, s, n) / tt : 0.0;
    for (long long i = tid; i < n; i += nt) {
      x[i] += (float)alpha * p[i] + (float)omega * s[i];
      r[i] = s[i] - (float)omega * t[i];
    }
    __syncthreads();
    rn = sqrt(dotf(r, r, n));
    ++its;
  }
  return rn / bn;
}

__device__ inline int trunc_rank2(const double* lam, int n, double delta, int rmax) {
  return dla::trunc_rank(lam, n, delta, rmax);
}

// PhiL[k+1], PsiL[k+1] from PhiL[k], PsiL[k] and core X_k (rank rl x 4 x rn)
__device__ void left_update(const DmrgArgs& a, int k) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int rl = a.xr[k], rn = a.xr[k + 1], sl = a.sr[k], sn = a.sr[k + 1];
  const float* X = Xcore(a, k);
  const float* S = Score(a, k);
  const float* pl = PL(a, k);
  float* out = PL(a, k + 1);
  // U1[a][s0][l][j][b'] = sum_a' PhiL(a,s0,a') X(a',l,j,b')
  const long long n1 = (long long)rl * sl * 4 * rn;
  for (long long i = tid; i < n1; i += nt) {
    long long t = i;
    const int bp = (int)(t % rn); t /= rn;
    const int lj = (int)(t % 4); t /= 4;
    const int s0 = (int)(t % sl); t /= sl;
    const int al = (int)t;
    float s = 0.f;
    for (int ap = 0; ap < rl; ++ap) s += pl[(al * sl + s0) * rl + ap] * X[((long long)ap * 4 + lj) * rn + bp];
    a.T1[i] = s;
  }
  __syncthreads();
  // U2[a][i][j][s][b'] = sum_{s0,l} S(s0,i,l,s) U1[a][s0][l][j][b']
  const long long n2 = (long long)rl * 4 * sn * rn;
  for (long long i = tid; i < n2; i += nt) {
    long long t = i;
    const int bp = (int)(t % rn); t /= rn;
    const int s = (int)(t % sn); t /= sn;
    const int ij = (int)(t % 4); t /= 4;
    const int al = (int)t;
    const int ii = ij >> 1, j = ij & 1;
    float acc = 0.f;
    for (int s0 = 0; s0 < sl; ++s0)
      for (int l = 0; l < 2; ++l)
        acc += S[((s0 * 2 + ii) * 2 + l) * sn + s] * a.T1[(((long long)al * sl + s0) * 4 + (l * 2 + j)) * rn + bp];
    a.T2[i] = acc;
  }
  __syncthreads();
  // PhiL[k+1](b, s, b') = sum_{a,i,j} X(a,i,j,b) U2[a][i][j][s][b']
  const long long n3 = (long long)rn * sn * rn;
  for (long long i = tid; i < n3; i += nt) {
    long long t = i;
    const int bp = (int)(t % rn); t /= rn;
    const int s = (int)(t % sn); t /= sn;
    const int b = (int)t;
    float acc = 0.f;
    for (int al = 0; al < rl; ++al)
      for (int ij = 0; ij < 4; ++ij)
        acc += X[((long long)al * 4 + ij) * rn + b] * a.T2[(((long long)al * 4 + ij) * sn + s) * rn + bp];
    out[i] = acc;
  }
  // PsiL[k+1](b) = sum_{a,i} X(a,i,i,b) PsiL[k](a)
  for (int b = tid; b < rn; b += nt) {
    float acc = 0.f;
    for (int al = 0; al < rl; ++al)
      acc += (X[((long long)al * 4 + 0) * rn + b] + X[((long long)al * 4 + 3) * rn + b]) * a.PsiL[k * a.rmax + al];
    a.PsiL[(k + 1) * a.rmax + b] = acc;
  }
  __syncthreads();
}

// PhiR[k], PsiR[k] from PhiR[k+1], PsiR[k+1] and core X_k (rank rl x 4 x rn)
__device__ void right_update(const DmrgArgs& a, int k) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int rl = a.xr[k], rn = a.xr[k + 1], sl = a.sr[k], sn = a.sr[k + 1];
  const float* X = Xcore(a, k);
  const float* S = Score(a, k);
  const float* pr = PR(a, k + 1);
  float* out = PR(a, k);
  // V1[a'][l][j][s2][b] = sum_b' X(a',l,j,b') PhiR(b, s2, b')
  const long long n1 = (long long)rl * 4 * sn * rn;
  for (long long i = tid; i < n1; i += nt) {
    long long t = i;
    const int b = (int)(t % rn); t /= rn;
    const int s2 = (int)(t % sn); t /= sn;
    const int lj = (int)(t % 4); t /= 4;
    const int ap = (int)t;
    float s = 0.f;
    for (int bp = 0; bp < rn; ++bp) s += X[((long long)ap * 4 + lj) * rn + bp] * pr[(b * sn + s2) * rn + bp];
    a.T1[i] = s;
  }
  __syncthreads();
  // V2[a'][s][i][j][b] = sum_{l,s2} S(s,i,l,s2) V1[a'][l][j][s2][b]
  const long long n2 = (long long)rl * sl * 4 * rn;
  for (long long i = tid; i < n2; i += nt) {
    long long t = i;
    const int b = (int)(t % rn); t /= rn;
    const int ij = (int)(t % 4); t /= 4;
    const int s = (int)(t % sl); t /= sl;
    const int ap = (int)t;
    const int ii = ij >> 1, j = ij & 1;
    float acc = 0.f;
    for (int l = 0; l < 2; ++l)
      for (int s2 = 0; s2 < sn; ++s2)
        acc += S[((s * 2 + ii) * 2 + l) * sn + s2] * a.T1[(((long long)ap * 4 + (l * 2 + j)) * sn + s2) * rn + b];
    a.T2[i] = acc;
  }
  __syncthreads();
  // PhiR[k](a, s, a') = sum_{i,j,b} X(a,i,j,b) V2[a'][s][i][j][b]
  const long long n3 = (long long)rl * sl * rl;
  for (long long i = tid; i < n3; i += nt) {
    long long t = i;
    const int ap = (int)(t % rl); t /= rl;
    const int s = (int)(t % sl); t /= sl;
    const int al = (int)t;
    float acc = 0.f;
    for (int ij = 0; ij < 4; ++ij)
      for (int b = 0; b < rn; ++b)
        acc += X[((long long)al * 4 + ij) * rn + b] * a.T2[(((long long)ap * sl + s) * 4 + ij) * rn + b];
    out[i] = acc;
  }
  for (int al = tid; al < rl; al += nt) {
    float acc = 0.f;
    for (int b = 0; b < rn; ++b)
      acc += (X[((long long)al * 4 + 0) * rn + b] + X[((long long)al * 4 + 3) * rn + b]) * a.PsiR[(k + 1) * a.rmax + b];
    a.PsiR[k * a.rmax + al] = acc;
  }
  __syncthreads();
}

// Solve the pair (k, k+1) and split it; dir = -1 (sweep to the left: X_{k+1}
// right-orthonormal) or +1 (sweep to the right: X_k left-orthonormal).
__device__ void solve_pair(const DmrgArgs& a, int k, int dir) {
  const int tid = threadIdx.x, nt = blockDim.x;
  __shared__ int sh_r;
  const int rl = a.xr[k], rm = a.xr[k + 1], rr = a.xr[k + 2];
  const float* X0 = Xcore(a, k);
  const float* X1 = Xcore(a, k + 1);
  const long long n = (long long)rl * 16 * rr;
  // W[b][(i1 j1 i2 j2)][c] = sum_m X0(b,i1,j1,m) X1(m,i2,j2,c)
  for (long long i = tid; i < n; i += nt) {
    long long t = i;
    const int c = (int)(t % rr); t /= rr;
    const int q = (int)(t % 16); t /= 16;
    const int b = (int)t;
    float s = 0.f;
    for (int m = 0; m < rm; ++m) s += X0[((long long)b * 4 + (q >> 2)) * rm + m] * X1[((long long)m * 4 + (q & 3)) * rr + c];
    a.W[i] = s;
  }
  // local right-hand side
  for (long long i = tid; i < n; i += nt) {
    long long t = i;
    const int c = (int)(t % rr); t /= rr;
    const int q = (int)(t % 16); t /= 16;
    const int b = (int)t;
    const bool diag = ((q >> 3) == ((q >> 2) & 1)) && (((q >> 1) & 1) == (q & 1));
    a.B[i] = diag ? a.PsiL[k * a.rmax + b] * a.PsiR[(k + 2) * a.rmax + c] : 0.f;
  }
  __syncthreads();
  int its = 0;
  double res = local_solve(a, k, rl, rr, a.W, a.B, its);
  if (tid == 0) {
    a.norms[0] = res;
    a.norms[1] = fmax(a.norms[1], (double)its);
  }
  // split W (rows (b,i1,j1): 4rl, cols (i2,j2,c): 4rr) by a truncated SVD
  const int m1 = 4 * rl, m2 = 4 * rr;
  const bool rows_small = m1 <= m2;
  const int ng = rows_small ? m1 : m2;
  for (int i = tid; i < ng * ng; i += nt) {
    const int x = i / ng, y = i - x * ng;
    double s = 0.0;
    if (rows_small) {
      for (int cidx = 0; cidx < m2; ++cidx) s += (double)a.W[(long long)x * m2 + cidx] * (double)a.W[(long long)y * m2 + cidx];
    } else {
      for (int ridx = 0; ridx < m1; ++ridx) s += (double)a.W[(long long)ridx * m2 + x] * (double)a.W[(long long)ridx * m2 + y];
    }
    a.G[i] = s;
  }
  __syncthreads();
  double fro = 0.0;
  for (int i = tid; i < ng; i += nt) fro += a.G[i * ng + i];
  fro = sqrt(blk_sum(fro));
  blk_syev(a.G, a.V, a.Vs, a.ev, ng);
  if (tid == 0) {
    int r = trunc_rank2(a.ev, ng, a.eps * fro / sqrt((double)(a.d > 1 ? a.d - 1 : 1)), a.rmax);
    int lim = m1 < m2 ? m1 : m2;
    sh_r = r > lim ? lim : r;
  }
  __syncthreads();
  const int r = sh_r;
  float* N0 = Xcore(a, k);
  float* N1 = Xcore(a, k + 1);
  // singular vectors: small side directly from Vs, other side by projection
  // U (m1 x r), V (m2 x r); W = U diag(sig) V^T
  // dir = +1: X_k = U, X_{k+1} = diag(sig) V^T ; dir = -1: X_k = U diag(sig), X_{k+1} = V^T
  if (rows_small) {
    // U = Vs[:, :r];  sig V^T = U^T W
    for (long long i = tid; i < (long long)m1 * r; i += nt) {
      const int x = (int)(i / r), y = (int)(i - (long long)x * r);
      const double sig = sqrt(fmax(a.ev[y], 0.0));
      a.T1[i] = (float)(dir > 0 ? a.Vs[x * ng + y] : a.Vs[x * ng + y] * sig);
    }
    for (long long i = tid; i < (long long)r * m2; i += nt) {
      const int y = (int)(i / m2), cidx = (int)(i - (long long)y * m2);
      double s = 0.0;
      for (int x = 0; x < m1; ++x) s += a.Vs[x * ng + y] * (double)a.W[(long long)x * m2 + cidx];
      const double sig = sqrt(fmax(a.ev[y], 0.0));
      a.T2[i] = (float)(dir > 0 ? s : (sig > 0.0 ? s / sig : 0.0));
    }
  } else {
    // V = Vs[:, :r];  U sig = W V
    for (long long i = tid; i < (long long)r * m2; i += nt) {
      const int y = (int)(i / m2), cidx = (int)(i - (long long)y * m2);
      const double sig = sqrt(fmax(a.ev[y], 0.0));
      a.T2[i] = (float)(dir > 0 ? a.Vs[cidx * ng + y] * sig : a.Vs[cidx * ng + y]);
    }
    for (long long i = tid; i < (long long)m1 * r; i += nt) {
      const int x = (int)(i / r), y = (int)(i - (long long)x * r);
      double s = 0.0;
      for (int cidx = 0; cidx < m2; ++cidx) s += (double)a.W[(long long)x * m2 + cidx] * a.Vs[cidx * ng + y];
      const double sig = sqrt(fmax(a.ev[y], 0.0));
      a.T1[i] = (float)(dir > 0 ? (sig > 0.0 ? s / sig : 0.0) : s);
    }
  }
  __syncthreads();
  for (long long i = tid; i < (long long)m1 * r; i += nt) N0[i] = a.T1[i];     // (rl,4) x r
  for (long long i = tid; i < (long long)r * m2; i += nt) N1[i] = a.T2[i];     // r x (4,rr)
  if (tid == 0) a.xr[k + 1] = r;
  __syncthreads();
  if (dir > 0) left_update(a, k);
  else right_update(a, k + 1);
}

__global__ void __launch_bounds__(DT) k_dmrg(DmrgArgs a) {
  const int d = a.d;
  // boundary interfaces of a rank-1 frame
  if (threadIdx.x == 0) {
    PL(a, 0)[0] = 1.f;
    PR(a, d)[0] = 1.f;
    a.PsiL[0] = 1.f;
    a.PsiR[d * a.rmax] = 1.f;
    a.norms[0] = 0.0;
    a.norms[1] = 0.0;
  }
  __syncthreads();
  // X arrives left-orthogonal in cores 0..d-2: build the left interfaces
  for (int k = 0; k < d - 1; ++k) left_update(a, k);
  for (int sw = 0; sw < a.sweeps; ++sw) {
    for (int k = d - 2; k >= 0; --k) solve_pair(a, k, -1);
    for (int k = 0; k <= d - 2; ++k) solve_pair(a, k, +1);
  }
}

__global__ void k_f64_to_f32(const double* __restrict__ a, float* __restrict__ b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}
__global__ void k_f32_to_f64(const float* __restrict__ a, double* __restrict__ b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    b[i] = (double)a[i];
}

// C = A + B^T or a scaled copy: block cores (Sec. 3.1 TT sum); transpose swaps i, j.
__global__ void k_sum_core(int k, int d, const double* __restrict__ A, int ra0, int ra1, const double* __restrict__ Bc,
                           int rb0, int rb1, int transB, double sa, double sb, double* __restrict__ C) {
  const int c0 = (k == 0) ? 1 : ra0 + rb0;
  const int c1 = (k == d - 1) ? 1 : ra1 + rb1;
  const int n = c0 * 4 * c1;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int b = i % c1, m = (i / c1) % 4, a = i / (4 * c1);
    double v = 0.0;
    // block of A: rows [0, ra0) (or 0 at k = 0), cols [0, ra1) (or 0 at k = d-1)
    const int aa = a, ab = b;
    const bool inA = (k == 0 ? aa == 0 : aa < ra0) && (k == d - 1 ? ab == 0 : ab < ra1);
    if (inA) v += (k == 0 ? sa : 1.0) * A[((long long)aa * 4 + m) * ra1 + ab];
    const int ba = (k == 0) ? 0 : a - ra0;
    const int bb = (k == d - 1) ? 0 : b - ra1;
    const bool inB = (k == 0 ? true : (a >= ra0)) && (k == d - 1 ? true : (b >= ra1)) && ba >= 0 && bb >= 0 &&
                     ba < rb0 && bb < rb1;
    if (inB) {
      const int mm = transB ? ((m & 1) << 1 | (m >> 1)) : m;
      v += (k == 0 ? sb : 1.0) * Bc[((long long)ba * 4 + mm) * rb1 + bb];
    }
    C[i] = v;
  }
}

}  // namespace

qp_qtt* tt_round_impl(qp_ctx* c, const qp_qtt* A, double eps, int rmax);

// 0.5 (A + A^T), rounded
static qp_qtt* symmetrize(qp_ctx* c, qp_qtt* A, double eps, int rmax) {
  const int d = A->d;
  std::vector<int> r(d + 1, 1);
  for (int k = 1; k < d; ++k) r[k] = 2 * A->ranks[k];
  qp_qtt* S = qtt_alloc(c, d, r);
  for (int k = 0; k < d; ++k) {
    k_sum_core<<<64, 256, 0, c->stream>>>(k, d, A->cores + A->offset[k], A->ranks[k], A->ranks[k + 1],
                                          A->cores + A->offset[k], A->ranks[k], A->ranks[k + 1], 1, 0.5, 0.5,
                                          S->cores + S->offset[k]);
  }
  QP_CUDA(cudaGetLastError());
  qp_qtt* R = nullptr;
  try {
    R = tt_round_impl(c, S, eps, rmax);
  } catch (...) {
    cudaFree(S->cores);
    delete S;
    throw;
  }
  cudaFree(S->cores);
  delete S;
  return R;
}

qp_qtt* inverse_impl(qp_ctx* c, qp_qtt* S, double eps, int rmax, int sweeps, qp_qtt* warm) {
  const int d = S->d;
  QP_REQUIRE(d >= 2, QP_INVALID_ARG, "qtt_inverse: d >= 2 required");
  QP_REQUIRE(eps > 0 && rmax >= 1 && sweeps >= 1, QP_INVALID_ARG, "qtt_inverse: eps > 0, rmax >= 1, sweeps >= 1");
  if (rmax > 64) rmax = 64;
  if (warm) QP_REQUIRE(warm->d == d, QP_INVALID_ARG, "qtt_inverse: warm start has a different d");
  cudaStream_t st = c->stream;
  qtt_prepare_copies(c, S, QP_F32);
  int smax = 1;
  for (int k = 0; k <= d; ++k) smax = std::max(smax, S->ranks[k]);
  // initial X, left-orthogonal: rounded warm start, or the scaled identity
  qp_qtt* X0 = nullptr;
  std::vector<int> xr(d + 1, 1);
  if (warm) {
    X0 = tt_round_impl(c, warm, 1e-7, rmax);
    xr = X0->ranks;
  } else {
    // trace of S: host-side chain of the 2x2 traces of each core
    std::vector<double> h(S->nvals);
    QP_CUDA(cudaMemcpyAsync(h.data(), S->cores, S->nvals * sizeof(double), cudaMemcpyDeviceToHost, st));
    QP_CUDA(cudaStreamSynchronize(st));
    std::vector<double> v(1, 1.0);
    for (int k = 0; k < d; ++k) {
      const int r0 = S->ranks[k], r1 = S->ranks[k + 1];
      std::vector<double> nv(r1, 0.0);
      const double* G = h.data() + S->offset[k];
      for (int a = 0; a < r0; ++a)
        for (int b = 0; b < r1; ++b) nv[b] += v[a] * (G[(a * 4 + 0) * r1 + b] + G[(a * 4 + 3) * r1 + b]);
      v.swap(nv);
    }
    const double N = std::ldexp(1.0, d);
    const double tr = v[0];
    QP_REQUIRE(tr > 0, QP_INVALID_ARG, "qtt_inverse: trace of S is not positive");
    X0 = qtt_alloc(c, d, xr);
    std::vector<double> core(4);
    for (int k = 0; k < d; ++k) {
      const double sc = (k < d - 1) ? 1.0 / std::sqrt(2.0) : (N / tr) * std::pow(2.0, 0.5 * (d - 1));
      core = {sc, 0.0, 0.0, sc};
      QP_CUDA(cudaMemcpyAsync(X0->cores + X0->offset[k], core.data(), 4 * sizeof(double), cudaMemcpyHostToDevice, st));
      QP_CUDA(cudaStreamSynchronize(st));
    }
  }
  // workspaces
  const long long R = rmax;
  const long long xcap = R * 4 * R;
  const long long phicap = R * smax * R;
  const long long wcap = R * 16 * R;
  const long long tcap = (long long)smax * R * 16 * R;
  float* X = static_cast<float*>(c->dm[0].ensure((size_t)d * xcap * sizeof(float)));
  float* PhiL = static_cast<float*>(c->dm[1].ensure((size_t)(d + 1) * phicap * sizeof(float)));
  float* PhiR = static_cast<float*>(c->dm[2].ensure((size_t)(d + 1) * phicap * sizeof(float)));
  float* Psi = static_cast<float*>(c->dm[3].ensure((size_t)2 * (d + 1) * R * sizeof(float)));
  float* Wb = static_cast<float*>(c->dm[4].ensure((size_t)8 * wcap * sizeof(float)));
  float* Tb = static_cast<float*>(c->dm[5].ensure((size_t)3 * tcap * sizeof(float)));
  const long long gcap = 4 * R * 4 * R;
  double* Gb = static_cast<double*>(c->dm[6].ensure((size_t)(3 * gcap + 4 * R + 16) * sizeof(double)));
  int* xr_dev = static_cast<int*>(c->dm[7].ensure((size_t)(d + 1) * (sizeof(int) + sizeof(long long)) * 2 + 64));
  int* sr_dev = xr_dev + (d + 1);
  long long* soff_dev = reinterpret_cast<long long*>(c->dm[8].ensure((size_t)(d + 1) * sizeof(long long)));
  QP_CUDA(cudaMemsetAsync(Psi, 0, (size_t)2 * (d + 1) * R * sizeof(float), st));
  for (int k = 0; k < d; ++k) {
    const long long nv = X0->offset[k + 1] - X0->offset[k];
    k_f64_to_f32<<<32, 256, 0, st>>>(X0->cores + X0->offset[k], X + k * xcap, nv);
  }
  QP_CUDA(cudaMemcpyAsync(xr_dev, xr.data(), (d + 1) * sizeof(int), cudaMemcpyHostToDevice, st));
  QP_CUDA(cudaMemcpyAsync(sr_dev, S->ranks.data(), (d + 1) * sizeof(int), cudaMemcpyHostToDevice, st));
  QP_CUDA(cudaMemcpyAsync(soff_dev, S->offset.data(), (d + 1) * sizeof(long long), cudaMemcpyHostToDevice, st));
  DmrgArgs a;
  a.d = d;
  a.sweeps = sweeps;
  a.rmax = rmax;
  a.local_maxit = 60;
  a.eps = eps;
  a.local_tol = std::max(1e-5, 0.1 * eps);
  a.S = S->cores32;
  a.sr = sr_dev;
  a.soff = soff_dev;
  a.smax = smax;
  a.X = X;
  a.xr = xr_dev;
  a.xcap = xcap;
  a.PhiL = PhiL;
  a.PhiR = PhiR;
  a.phicap = phicap;
  a.PsiL = Psi;
  a.PsiR = Psi + (d + 1) * R;
  a.W = Wb;
  a.B = Wb + wcap;
  for (int i = 0; i < 6; ++i) a.v[i] = Wb + (2 + i) * wcap;
  a.wcap = wcap;
  a.T1 = Tb;
  a.T2 = Tb + tcap;
  a.T3 = Tb + 2 * tcap;
  a.tcap = tcap;
  a.G = Gb;
  a.V = Gb + gcap;
  a.Vs = Gb + 2 * gcap;
  a.ev = Gb + 3 * gcap;
  a.norms = Gb + 3 * gcap + 4 * R;
  QP_CUDA(cudaFuncSetAttribute(k_dmrg, cudaFuncAttributeMaxDynamicSharedMemorySize, dla::SYEV_SMEM_BYTES));
  k_dmrg<<<1, DT, dla::SYEV_SMEM_BYTES, st>>>(a);
  QP_CUDA(cudaGetLastError());
  std::vector<int> ro(d + 1);
  QP_CUDA(cudaMemcpyAsync(ro.data(), xr_dev, (d + 1) * sizeof(int), cudaMemcpyDeviceToHost, st));
  QP_CUDA(cudaStreamSynchronize(st));
  cudaFree(X0->cores);
  if (X0->cores32) cudaFree(X0->cores32);
  delete X0;
  qp_qtt* Xr = qtt_alloc(c, d, ro);
  for (int k = 0; k < d; ++k)
    k_f32_to_f64<<<32, 256, 0, st>>>(X + k * xcap, Xr->cores + Xr->offset[k], Xr->offset[k + 1] - Xr->offset[k]);
  QP_CUDA(cudaGetLastError());
  qp_qtt* out = nullptr;
  try {
    out = symmetrize(c, Xr, eps, rmax);
  } catch (...) {
    cudaFree(Xr->cores);
    delete Xr;
    throw;
  }
  cudaFree(Xr->cores);
  delete Xr;
  out->scaled = S->scaled;
  return out;
}

}  // namespace qp

using namespace qp;

extern "C" int qtt_inverse(qp_ctx_t c, qtt_t S, double eps, int rmax, int sweeps, qtt_t warm, qtt_t* out) {
  if (!c || !S || !out) return QP_INVALID_ARG;
  try {
    QP_CUDA(cudaSetDevice(c->device));
    *out = inverse_impl(c, S, eps, rmax, sweeps, warm);
  } catch (const Error& e) {
    set_error(c, e);
    return e.code;
  }
  return QP_OK;
}
