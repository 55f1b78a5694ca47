// Contact assembly (Sec. 2.2-2.3, 3.3): active set, frames, Morton order,
// body->contact incidence and the vector r of Eq. rdef.
//
// Integer results (the pair list and its order) are bit-exact with any IEEE
// double evaluation that uses the same operation order, so every floating-point
// step that feeds a decision or a key is written with round-to-nearest
// intrinsics (no FMA contraction): the pair test d^2 <= (r_a + r_b + delta)^2
// with d^2 = (dx*dx + dy*dy) + dz*dz, the gap, the normal, the contact point and
// its quantisation.
#include <cub/cub.cuh>

#include "internal.cuh"

namespace qp {
namespace {

constexpr int MORTON_BITS = 21;

__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double ddiv(double a, double b) { return __ddiv_rn(a, b); }

struct Box {
  double lo[3], hi[3], rmax;
};

// Bounding box of n points (SoA [3][n]) and, when r is given, the largest r:
// block g reduces a grid-stride share into part[g][7] = (lo xyz, hi xyz, rmax);
// k_box_final combines the partials.  min/max are exact, so the result does
// not depend on the split.
constexpr int BOX_BLOCKS = 128;

__global__ void k_box_partial(int n, const double* __restrict__ p, const double* __restrict__ r,
                              double* __restrict__ part) {
  __shared__ double sm[7][32];
  double v[7] = {1e300, 1e300, 1e300, -1e300, -1e300, -1e300, 0.0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    for (int a = 0; a < 3; ++a) {
      const double x = p[(size_t)a * n + i];
      v[a] = fmin(v[a], x);
      v[3 + a] = fmax(v[3 + a], x);
    }
    if (r) v[6] = fmax(v[6], r[i]);
  }
  for (int k = 0; k < 7; ++k) {
    double x = v[k];
    for (int o = 16; o > 0; o >>= 1) {
      const double y = __shfl_xor_sync(0xffffffffu, x, o);
      x = (k < 3) ? fmin(x, y) : fmax(x, y);
    }
    if ((threadIdx.x & 31) == 0) sm[k][threadIdx.x >> 5] = x;
  }
  __syncthreads();
  if (threadIdx.x < 7) {
    const int k = threadIdx.x, nw = blockDim.x >> 5;
    double x = sm[k][0];
    for (int w = 1; w < nw; ++w) x = (k < 3) ? fmin(x, sm[k][w]) : fmax(x, sm[k][w]);
    part[(size_t)blockIdx.x * 7 + k] = x;
  }
}

__global__ void k_box_final(int G, const double* __restrict__ part, double* __restrict__ out, int nout) {
  // one warp per value: each lane folds a strided share of the partials, then
  // the warp combines the lanes
  const int k = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (k >= nout) return;
  double x = k < 3 ? 1e300 : (k < 6 ? -1e300 : 0.0);
  for (int g = lane; g < G; g += 32) {
    const double y = part[(size_t)g * 7 + k];
    x = (k < 3) ? fmin(x, y) : fmax(x, y);
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double y = __shfl_xor_sync(0xffffffffu, x, o);
    x = (k < 3) ? fmin(x, y) : fmax(x, y);
  }
  if (lane == 0) out[k] = x;
}

struct Grid {
  double lo[3];
  double h;
  int n[3];
};

__device__ __forceinline__ int cell_coord(double x, double lo, double h, int n) {
  int c = (int)floor((x - lo) / h);
  return c < 0 ? 0 : (c >= n ? n - 1 : c);
}

__global__ void k_cell_ids(int M, const double* __restrict__ pos, Grid g, unsigned* __restrict__ cell,
                           int* __restrict__ body) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  int cx = cell_coord(pos[i], g.lo[0], g.h, g.n[0]);
  int cy = cell_coord(pos[(size_t)M + i], g.lo[1], g.h, g.n[1]);
  int cz = cell_coord(pos[2 * (size_t)M + i], g.lo[2], g.h, g.n[2]);
  cell[i] = (unsigned)(cx + g.n[0] * (cy + g.n[1] * cz));
  body[i] = i;
}

__global__ void k_cell_ranges(int M, const unsigned* __restrict__ sorted_cell, int* __restrict__ start,
                              int* __restrict__ end) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  unsigned c = sorted_cell[i];
  if (i == 0 || sorted_cell[i - 1] != c) start[c] = i;
  if (i == M - 1 || sorted_cell[i + 1] != c) end[c] = i + 1;
}

__device__ __forceinline__ bool pair_active(const double* __restrict__ pos, const double* __restrict__ rad, int M,
                                            int a, int b, double delta) {
  double dx = dsub(pos[b], pos[a]);
  double dy = dsub(pos[(size_t)M + b], pos[(size_t)M + a]);
  double dz = dsub(pos[2 * (size_t)M + b], pos[2 * (size_t)M + a]);
  double d2 = dadd(dadd(dmul(dx, dx), dmul(dy, dy)), dmul(dz, dz));
  double s = dadd(dadd(rad[a], rad[b]), delta);
  return d2 <= dmul(s, s);
}

// FP32 copies of the centres relative to the grid origin (the FP64 difference
// rounded once) and the radii, for the conservative pre-test of k_pairs.
__global__ void k_pos32(int M, const double* __restrict__ pos, const double* __restrict__ rad, Grid g,
                        float4* __restrict__ p32) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M; i += gridDim.x * blockDim.x)
    p32[i] = make_float4((float)(pos[i] - g.lo[0]), (float)(pos[(size_t)M + i] - g.lo[1]),
                         (float)(pos[2 * (size_t)M + i] - g.lo[2]), (float)rad[i]);
}

// Side walls of a boxed scene: static planes x_axis = off with the box on the
// side of sign (+1 / -1).
struct Walls {
  int n;
  int axis[4];
  int sign[4];
  double off[4];
};

__device__ __forceinline__ double wall_gap(const double* pos, const double* rad, int M, int b, const Walls& wl,
                                           int w) {
  const double x = pos[(size_t)wl.axis[w] * M + b];
  return wl.sign[w] > 0 ? dsub(dsub(x, wl.off[w]), rad[b]) : dsub(dsub(wl.off[w], x), rad[b]);
}

// Count (write == nullptr) or write the contacts of body a: partners b > a in
// the 27 neighbouring cells, then the floor, then the side walls (a wall's raw
// first body is M + 1 + w until the contacts are ordered; then it is M).  Written pairs of one body are in
// arbitrary order; the global order is fixed afterwards by sorting.
// Each candidate is first tested in FP32 against an envelope widened by a bound
// on the FP32 rounding (err: 4 x the largest coordinate error, plus a relative
// 1e-5): only candidates that pass it take the exact FP64 test, so the pair list
// is the exact one while most FP64 work (a narrow pipe on this part) is skipped.
__global__ void k_pairs(int M, const double* __restrict__ pos, const double* __restrict__ rad, Grid g,
                        const int* __restrict__ cstart, const int* __restrict__ cend,
                        const int* __restrict__ sbody, double delta, double floor_z, Walls wl,
                        int* __restrict__ count, const int* __restrict__ offset, int* __restrict__ wa,
                        int* __restrict__ wb, const float4* __restrict__ p32, float err) {
  int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= M) return;
  const float4 pa = p32[a];
  const float dl = (float)delta;
  int cx = cell_coord(pos[a], g.lo[0], g.h, g.n[0]);
  int cy = cell_coord(pos[(size_t)M + a], g.lo[1], g.h, g.n[1]);
  int cz = cell_coord(pos[2 * (size_t)M + a], g.lo[2], g.h, g.n[2]);
  int k = 0;
  int base = offset ? offset[a] : 0;
  for (int dz = -1; dz <= 1; ++dz) {
    int z = cz + dz;
    if (z < 0 || z >= g.n[2]) continue;
    for (int dy = -1; dy <= 1; ++dy) {
      int y = cy + dy;
      if (y < 0 || y >= g.n[1]) continue;
      for (int dx = -1; dx <= 1; ++dx) {
        int x = cx + dx;
        if (x < 0 || x >= g.n[0]) continue;
        unsigned cell = (unsigned)(x + g.n[0] * (y + g.n[1] * z));
        int s = cstart[cell];
        if (s < 0) continue;
        int e = cend[cell];
        for (int j = s; j < e; ++j) {
          int b = sbody[j];
          if (b <= a) continue;
          const float4 pb = p32[b];
          const float ex = pb.x - pa.x, ey = pb.y - pa.y, ez = pb.z - pa.z;
          const float lim = (pa.w + pb.w + dl) + err;
          if (ex * ex + ey * ey + ez * ez > lim * lim * 1.00001f) continue;
          if (pair_active(pos, rad, M, a, b, delta)) {
            if (wa) {
              wa[base + k] = a;
              wb[base + k] = b;
            }
            ++k;
          }
        }
      }
    }
  }
  double phi_f = dsub(dsub(pos[2 * (size_t)M + a], floor_z), rad[a]);
  if (phi_f <= delta) {
    if (wa) {
      wa[base + k] = M;  // static floor is body a
      wb[base + k] = a;
    }
    ++k;
  }
  for (int w = 0; w < wl.n; ++w) {
    if (wall_gap(pos, rad, M, a, wl, w) <= delta) {
      if (wa) {
        wa[base + k] = M + 1 + w;
        wb[base + k] = a;
      }
      ++k;
    }
  }
  if (count) count[a] = k;
}

// Gap, normal and contact point of every raw contact, plus the (a, b) sort key.
__global__ void k_geom_raw(int n, int M, const double* __restrict__ pos, const double* __restrict__ rad,
                           double floor_z, Walls wl, const int* __restrict__ wa, const int* __restrict__ wb,
                           double* __restrict__ phi, double* __restrict__ nrm, double* __restrict__ pt,
                           unsigned long long* __restrict__ abkey, int* __restrict__ idx) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int a = wa[i], b = wb[i];
  double ph, nx, ny, nz, px, py, pz;
  if (a == M) {
    double zb = pos[2 * (size_t)M + b];
    ph = dsub(dsub(zb, floor_z), rad[b]);
    nx = 0.0;
    ny = 0.0;
    nz = 1.0;
    px = pos[b];
    py = pos[(size_t)M + b];
    pz = dadd(floor_z, dmul(ph, 0.5));
  } else if (a > M) {
    // side wall w: normal sign e_axis, point offset + sign Phi/2 on that axis
    const int w = a - M - 1, ax = wl.axis[w];
    ph = wall_gap(pos, rad, M, b, wl, w);
    const double sn = wl.sign[w] > 0 ? 1.0 : -1.0;
    const double hp = dmul(ph, 0.5);
    const double pw = dadd(wl.off[w], wl.sign[w] > 0 ? hp : -hp);
    nx = ax == 0 ? sn : 0.0;
    ny = ax == 1 ? sn : 0.0;
    nz = ax == 2 ? sn : 0.0;
    px = ax == 0 ? pw : pos[b];
    py = ax == 1 ? pw : pos[(size_t)M + b];
    pz = ax == 2 ? pw : pos[2 * (size_t)M + b];
  } else {
    double xa = pos[a], ya = pos[(size_t)M + a], za = pos[2 * (size_t)M + a];
    double dx = dsub(pos[b], xa);
    double dy = dsub(pos[(size_t)M + b], ya);
    double dz = dsub(pos[2 * (size_t)M + b], za);
    double d = __dsqrt_rn(dadd(dadd(dmul(dx, dx), dmul(dy, dy)), dmul(dz, dz)));
    ph = dsub(d, dadd(rad[a], rad[b]));
    nx = ddiv(dx, d);
    ny = ddiv(dy, d);
    nz = ddiv(dz, d);
    double h = dadd(rad[a], dmul(ph, 0.5));
    px = dadd(xa, dmul(nx, h));
    py = dadd(ya, dmul(ny, h));
    pz = dadd(za, dmul(nz, h));
  }
  phi[i] = ph;
  nrm[i] = nx;
  nrm[(size_t)n + i] = ny;
  nrm[2 * (size_t)n + i] = nz;
  pt[i] = px;
  pt[(size_t)n + i] = py;
  pt[2 * (size_t)n + i] = pz;
  abkey[i] = (unsigned long long)a * (unsigned long long)(M + 1) + (unsigned long long)b;
  idx[i] = i;
}

__device__ __forceinline__ unsigned long long spread3(unsigned long long v) {
  unsigned long long out = 0;
  for (int k = 0; k < MORTON_BITS; ++k) out |= ((v >> k) & 1ull) << (3 * k);
  return out;
}

// Morton key of the contact point quantised over the point bounding box.  The
// permutation of the first (a, b) sort is applied on the fly.
__global__ void k_morton(int n, const double* __restrict__ pt, const double* __restrict__ box,
                         const int* __restrict__ perm, unsigned long long* __restrict__ key) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int j = perm[i];
  unsigned long long q[3];
  const unsigned long long top = (1ull << MORTON_BITS) - 1ull;
  for (int a = 0; a < 3; ++a) {
    double lo = box[a], ext = dsub(box[3 + a], box[a]);
    q[a] = 0;
    if (ext > 0.0) {
      double v = floor(dmul(ddiv(dsub(pt[(size_t)a * n + j], lo), ext), (double)(1 << MORTON_BITS)));
      unsigned long long qi = (unsigned long long)v;
      q[a] = qi > top ? top : qi;
    }
  }
  key[i] = spread3(q[0]) | (spread3(q[1]) << 1) | (spread3(q[2]) << 2);
}

// Final contact arrays in hierarchy order: frames, arms, FP32 copies.
__global__ void k_gather(int n, int M, const int* __restrict__ perm2, const int* __restrict__ perm1,
                         const int* __restrict__ wa, const int* __restrict__ wb, const double* __restrict__ phi_raw,
                         const double* __restrict__ nrm_raw, const double* __restrict__ pt_raw,
                         const double* __restrict__ pos, int* __restrict__ ca, int* __restrict__ cb,
                         int* __restrict__ cplane,
                         double* __restrict__ phi, double* __restrict__ frame, double* __restrict__ point,
                         double* __restrict__ arm_a, double* __restrict__ arm_b, double* __restrict__ rec64,
                         float* __restrict__ rec32) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  int j = perm1[perm2[c]];
  int a = wa[j], b = wb[j];
  cplane[c] = a >= M ? a - M : -1;  // which plane, before it is folded into body M
  if (a > M) a = M;                 // every static plane (floor or wall) is body M
  ca[c] = a;
  cb[c] = b;
  phi[c] = phi_raw[j];
  double nx = nrm_raw[j], ny = nrm_raw[(size_t)n + j], nz = nrm_raw[2 * (size_t)n + j];
  double p[3] = {pt_raw[j], pt_raw[(size_t)n + j], pt_raw[2 * (size_t)n + j]};
  // tangent frame: e = axis minimising |n_e| (lowest index on ties)
  double ax = fabs(nx), ay = fabs(ny), az = fabs(nz);
  int e = (ay < ax) ? 1 : 0;
  double best = (e == 1) ? ay : ax;
  if (az < best) e = 2;
  double c0, c1, c2;
  if (e == 0) {
    c0 = 0.0; c1 = nz; c2 = -ny;
  } else if (e == 1) {
    c0 = -nz; c1 = 0.0; c2 = nx;
  } else {
    c0 = ny; c1 = -nx; c2 = 0.0;
  }
  double Ln = __dsqrt_rn(dadd(dadd(dmul(c0, c0), dmul(c1, c1)), dmul(c2, c2)));
  double t1x = ddiv(c0, Ln), t1y = ddiv(c1, Ln), t1z = ddiv(c2, Ln);
  double t2x = dsub(dmul(ny, t1z), dmul(nz, t1y));
  double t2y = dsub(dmul(nz, t1x), dmul(nx, t1z));
  double t2z = dsub(dmul(nx, t1y), dmul(ny, t1x));
  double F[9] = {nx, ny, nz, t1x, t1y, t1z, t2x, t2y, t2z};
  double* R = rec64 + (size_t)c * 16;
  float* R32 = rec32 + (size_t)c * 16;
  for (int k = 0; k < 9; ++k) {
    frame[(size_t)k * n + c] = F[k];
    R[k] = F[k];
    R32[k] = (float)F[k];
  }
  R[15] = 0.0;
  R32[15] = 0.0f;
  for (int k = 0; k < 3; ++k) {
    point[(size_t)k * n + c] = p[k];
    double xa = (a == M) ? 0.0 : pos[(size_t)k * M + a];
    double va = (a == M) ? 0.0 : dsub(p[k], xa);
    double vb = dsub(p[k], pos[(size_t)k * M + b]);
    arm_a[(size_t)k * n + c] = va;
    arm_b[(size_t)k * n + c] = vb;
    R[9 + k] = va;
    R[12 + k] = vb;
    R32[9 + k] = (float)va;
    R32[12 + k] = (float)vb;
  }
}

__global__ void k_inc_count(int n, int M, const int* __restrict__ ca, const int* __restrict__ cb, int* cnt) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  if (ca[c] < M) atomicAdd(&cnt[ca[c]], 1);
  atomicAdd(&cnt[cb[c]], 1);
}

__global__ void k_inc_fill(int n, int M, const int* __restrict__ ca, const int* __restrict__ cb,
                           const int* __restrict__ bptr, int* cursor, int* __restrict__ inc) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  int a = ca[c], b = cb[c];
  if (a < M) inc[bptr[a] + atomicAdd(&cursor[a], 1)] = (c << 1);
  inc[bptr[b] + atomicAdd(&cursor[b], 1)] = (c << 1) | 1;
}

// Sort each body's incidence list by contact index (deterministic sum order).
__global__ void k_inc_sort(int M, const int* __restrict__ bptr, int* __restrict__ inc) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= M) return;
  int s = bptr[b], e = bptr[b + 1];
  for (int i = s + 1; i < e; ++i) {
    int v = inc[i];
    int j = i - 1;
    while (j >= s && inc[j] > v) {
      inc[j + 1] = inc[j];
      --j;
    }
    inc[j + 1] = v;
  }
}

// r = b + D^T (v + dt g, omega) with b_c = (Phi_c/dt, 0, 0)  (Eq. rdef).
__global__ void k_rvec(int n, int M, int slots, const int* __restrict__ ca, const int* __restrict__ cb,
                       const double* __restrict__ phi, const double* __restrict__ frame,
                       const double* __restrict__ arm_a, const double* __restrict__ arm_b,
                       const double* __restrict__ vel, const double* __restrict__ omg, double gx, double gy,
                       double gz, double dt, double* __restrict__ r) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  int a = ca[c], b = cb[c];
  double g[3] = {gx, gy, gz};
  double dv[3];
  double rb[3], ra[3], wb[3], wa[3];
  for (int k = 0; k < 3; ++k) {
    rb[k] = arm_b[(size_t)k * n + c];
    ra[k] = arm_a[(size_t)k * n + c];
    wb[k] = omg[(size_t)k * M + b];
    wa[k] = (a == M) ? 0.0 : omg[(size_t)k * M + a];
  }
  double cbx = wb[1] * rb[2] - wb[2] * rb[1], cby = wb[2] * rb[0] - wb[0] * rb[2], cbz = wb[0] * rb[1] - wb[1] * rb[0];
  double cax = wa[1] * ra[2] - wa[2] * ra[1], cay = wa[2] * ra[0] - wa[0] * ra[2], caz = wa[0] * ra[1] - wa[1] * ra[0];
  double crb[3] = {cbx, cby, cbz}, cra[3] = {cax, cay, caz};
  for (int k = 0; k < 3; ++k) {
    double vb = vel[(size_t)k * M + b] + dt * g[k] + crb[k];
    double va = (a == M) ? 0.0 : vel[(size_t)k * M + a] + dt * g[k] + cra[k];
    dv[k] = vb - va;
  }
  for (int u = 0; u < 3; ++u) {
    const double* F = frame + (size_t)(3 * u) * n;
    double s = F[c] * dv[0] + F[(size_t)n + c] * dv[1] + F[2 * (size_t)n + c] * dv[2];
    if (u == 0) s += phi[c] / dt;
    r[(size_t)slots * c + u] = s;
  }
}

__global__ void k_body_copy(int M, const double* __restrict__ im, const double* __restrict__ iI,
                            double* __restrict__ im64, double* __restrict__ iI64, float* __restrict__ im32,
                            float* __restrict__ iI32) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  im64[i] = im[i];
  iI64[i] = iI[i];
  im32[i] = (float)im[i];
  iI32[i] = (float)iI[i];
}

}  // namespace

static void assemble(qp_ctx* c, const qp_scene* s, qp_contacts* out) {
  QP_REQUIRE(s && out, QP_INVALID_ARG, "ccp_assemble: null scene or output");
  QP_REQUIRE(s->M >= 1, QP_INVALID_ARG, "ccp_assemble: M must be >= 1");
  QP_REQUIRE(s->slots == 3 || s->slots == 4, QP_INVALID_ARG, "ccp_assemble: slots must be 3 or 4");
  QP_REQUIRE(s->dt > 0 && s->delta >= 0, QP_INVALID_ARG, "ccp_assemble: dt > 0 and delta >= 0 required");
  QP_REQUIRE(s->pos && s->vel && s->omega && s->radius && s->inv_mass && s->inv_inertia, QP_INVALID_ARG,
             "ccp_assemble: null scene array");
  QP_REQUIRE(s->nwalls >= 0 && s->nwalls <= 4, QP_INVALID_ARG, "ccp_assemble: nwalls must be 0..4");
  Walls wl{};
  wl.n = s->nwalls;
  for (int w = 0; w < s->nwalls; ++w) {
    QP_REQUIRE(s->wall_axis[w] >= 0 && s->wall_axis[w] <= 2 && (s->wall_sign[w] == 1 || s->wall_sign[w] == -1),
               QP_INVALID_ARG, "ccp_assemble: wall axis must be 0..2 and sign +-1");
    wl.axis[w] = s->wall_axis[w];
    wl.sign[w] = s->wall_sign[w];
    wl.off[w] = s->wall_offset[w];
  }
  QP_CUDA(cudaSetDevice(c->device));
  cudaStream_t st = c->stream;
  const int M = s->M;
  const int TB = 256;

  // 1. bounding box and uniform grid (cell >= 2 r_max + delta)
  // scratch[0]: body box (Box), point box (6 doubles) at +64, block partials at +256
  char* sb = static_cast<char*>(c->scratch[0].ensure(256 + (size_t)BOX_BLOCKS * 7 * sizeof(double)));
  Box* dbox = reinterpret_cast<Box*>(sb);
  double* bpart = reinterpret_cast<double*>(sb + 256);
  {
    const int G = std::max(1, std::min(BOX_BLOCKS, ceil_div(M, 256)));
    k_box_partial<<<G, 256, 0, st>>>(M, s->pos, s->radius, bpart);
    k_box_final<<<1, 7 * 32, 0, st>>>(G, bpart, reinterpret_cast<double*>(dbox), 7);
  }
  QP_CUDA(cudaGetLastError());
  Box box;
  QP_CUDA(cudaMemcpyAsync(&box, dbox, sizeof(Box), cudaMemcpyDeviceToHost, st));
  QP_CUDA(cudaStreamSynchronize(st));
  Grid g;
  g.h = (2.0 * box.rmax + s->delta) * (1.0 + 1e-6) + 1e-12;
  long long ncell;
  for (;;) {
    ncell = 1;
    for (int a = 0; a < 3; ++a) {
      g.lo[a] = box.lo[a];
      g.n[a] = (int)floor((box.hi[a] - box.lo[a]) / g.h) + 1;
      ncell *= g.n[a];
    }
    if (ncell <= 8LL * M + 64) break;
    g.h *= 1.5;
  }

  // 2. bodies sorted by cell
  unsigned* cell = static_cast<unsigned*>(c->scratch[1].ensure(sizeof(unsigned) * 2 * (size_t)M));
  unsigned* cell_s = cell + M;
  int* body = static_cast<int*>(c->scratch[2].ensure(sizeof(int) * 2 * (size_t)M));
  int* body_s = body + M;
  k_cell_ids<<<ceil_div(M, TB), TB, 0, st>>>(M, s->pos, g, cell, body);
  size_t tmp_bytes = 0;
  cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, cell, cell_s, body, body_s, M, 0, 32, st);
  void* tmp = c->scratch[3].ensure(tmp_bytes);
  QP_CUDA(cub::DeviceRadixSort::SortPairs(tmp, tmp_bytes, cell, cell_s, body, body_s, M, 0, 32, st));
  int* cstart = static_cast<int*>(c->scratch[4].ensure(sizeof(int) * 2 * (size_t)ncell));
  int* cend = cstart + ncell;
  QP_CUDA(cudaMemsetAsync(cstart, 0xff, sizeof(int) * (size_t)ncell, st));
  k_cell_ranges<<<ceil_div(M, TB), TB, 0, st>>>(M, cell_s, cstart, cend);

  // 3. count, scan, write pairs
  int* count = static_cast<int*>(c->scratch[5].ensure(sizeof(int) * (2 * (size_t)M + 2) + 16 * (size_t)M + 64));
  int* offset = count + M + 1;
  float4* p32 = reinterpret_cast<float4*>(count + ((2 * (size_t)M + 2 + 3) & ~(size_t)3));
  // rounding bound of the FP32 pre-test: each coordinate (relative to the grid
  // origin, at most the box extent E) is off by at most E 2^-24, and the
  // radii and delta by a relative 2^-24; a difference is then off by at most
  // 2 E 2^-24 per axis, the distance by sqrt(3) of that
  double ext = 0.0;
  for (int a2 = 0; a2 < 3; ++a2) ext = std::max(ext, box.hi[a2] - box.lo[a2]);
  const float perr = (float)(4.0 * (ext + 2.0 * box.rmax + s->delta + 1.0) * 6.0e-8) + 1e-30f;
  k_pos32<<<ceil_div(M, TB), TB, 0, st>>>(M, s->pos, s->radius, g, p32);
  k_pairs<<<ceil_div(M, TB), TB, 0, st>>>(M, s->pos, s->radius, g, cstart, cend, body_s, s->delta, s->floor_z, wl,
                                          count, nullptr, nullptr, nullptr, p32, perr);
  QP_CUDA(cudaGetLastError());
  tmp_bytes = 0;
  cub::DeviceScan::ExclusiveSum(nullptr, tmp_bytes, count, offset, M + 1, st);
  tmp = c->scratch[3].ensure(tmp_bytes);
  QP_CUDA(cudaMemsetAsync(count + M, 0, sizeof(int), st));
  QP_CUDA(cub::DeviceScan::ExclusiveSum(tmp, tmp_bytes, count, offset, M + 1, st));
  int Nc = 0;
  QP_CUDA(cudaMemcpyAsync(&Nc, offset + M, sizeof(int), cudaMemcpyDeviceToHost, st));
  QP_CUDA(cudaStreamSynchronize(st));

  const int slots = s->slots;
  long long rows = (long long)slots * Nc;
  if (rows < 1) rows = 1;
  int L = 1;
  while ((1LL << L) < rows) ++L;
  const long long P = 1LL << L;

  c->M = M;
  c->Nc = Nc;
  c->L = L;
  c->P = P;
  c->slots = slots;
  c->mu = s->mu;
  c->dt = s->dt;
  const size_t n = (size_t)(Nc > 0 ? Nc : 1);

  // raw contact arrays live in scratch 6/7
  char* raw = static_cast<char*>(c->scratch[6].ensure(n * (2 * sizeof(int) + 7 * sizeof(double)) + 256));
  int* wa = reinterpret_cast<int*>(raw);
  int* wb = wa + n;
  double* phi_raw = reinterpret_cast<double*>(wb + n);  // 2n ints: 8-byte aligned
  double* nrm_raw = phi_raw + n;
  double* pt_raw = nrm_raw + 3 * n;
  char* keys = static_cast<char*>(c->scratch[7].ensure(n * (4 * sizeof(unsigned long long) + 4 * sizeof(int)) + 256));
  unsigned long long* k1 = reinterpret_cast<unsigned long long*>(keys);
  unsigned long long* k1s = k1 + n;
  unsigned long long* k2 = k1s + n;
  unsigned long long* k2s = k2 + n;
  int* i0 = reinterpret_cast<int*>(k2s + n);
  int* i1 = i0 + n;
  int* i2 = i1 + n;
  int* i3 = i2 + n;

  // final arrays
  c->ca.ensure(n * sizeof(int));
  c->cb.ensure(n * sizeof(int));
  c->cplane.ensure(n * sizeof(int));
  c->phi.ensure(n * sizeof(double));
  c->frame.ensure(9 * n * sizeof(double));
  c->point.ensure(3 * n * sizeof(double));
  c->arm_a.ensure(3 * n * sizeof(double));
  c->arm_b.ensure(3 * n * sizeof(double));
  c->key.ensure(n * sizeof(unsigned long long));
  c->r.ensure((size_t)P * sizeof(double));
  c->rec64.ensure(16 * n * sizeof(double));
  c->rec32.ensure(16 * n * sizeof(float));
  c->inv_m.ensure((size_t)M * sizeof(double));
  c->inv_I.ensure((size_t)M * sizeof(double));
  c->inv_m32.ensure((size_t)M * sizeof(float));
  c->inv_I32.ensure((size_t)M * sizeof(float));
  c->bptr.ensure(((size_t)M + 1) * sizeof(int));
  c->inc.ensure(2 * n * sizeof(int));
  c->wbody.ensure(8 * (size_t)M * sizeof(double));
  c->wbody32.ensure(8 * (size_t)M * sizeof(float));
  c->H.ensure(6 * n * sizeof(double));
  c->H32.ensure(6 * n * sizeof(float));
  c->dinv.ensure((size_t)P * sizeof(double));
  c->dinv32.ensure((size_t)P * sizeof(float));
  QP_CUDA(cudaMemsetAsync(c->r.p, 0, (size_t)P * sizeof(double), st));

  k_body_copy<<<ceil_div(M, TB), TB, 0, st>>>(M, s->inv_mass, s->inv_inertia, c->inv_m.as<double>(),
                                              c->inv_I.as<double>(), c->inv_m32.as<float>(), c->inv_I32.as<float>());
  int* bptr = c->bptr.as<int>();
  if (Nc > 0) {
    k_pairs<<<ceil_div(M, TB), TB, 0, st>>>(M, s->pos, s->radius, g, cstart, cend, body_s, s->delta, s->floor_z, wl,
                                            nullptr, offset, wa, wb, p32, perr);
    k_geom_raw<<<ceil_div(Nc, TB), TB, 0, st>>>(Nc, M, s->pos, s->radius, s->floor_z, wl, wa, wb, phi_raw, nrm_raw,
                                                pt_raw, k1, i0);
    QP_CUDA(cudaGetLastError());
    // 4. order: sort by (a, b), then stable sort by Morton key -> (key, a, b)
    int abbits = 1;
    // raw first bodies reach M + 4 (walls): keys below (M + 5)(M + 1)
    while (abbits < 64 && (1ull << abbits) <= (unsigned long long)(M + 5) * (unsigned long long)(M + 1)) ++abbits;
    tmp_bytes = 0;
    cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, k1, k1s, i0, i1, Nc, 0, abbits, st);
    size_t t2 = 0;
    cub::DeviceRadixSort::SortPairs(nullptr, t2, k2, k2s, i2, i3, Nc, 0, 3 * MORTON_BITS, st);
    tmp = c->scratch[3].ensure(tmp_bytes > t2 ? tmp_bytes : t2);
    QP_CUDA(cub::DeviceRadixSort::SortPairs(tmp, tmp_bytes, k1, k1s, i0, i1, Nc, 0, abbits, st));
    double* pbox = reinterpret_cast<double*>(static_cast<char*>(c->scratch[0].p) + 64);
    {
      double* ppart = reinterpret_cast<double*>(static_cast<char*>(c->scratch[0].p) + 256);
      const int G = std::max(1, std::min(BOX_BLOCKS, ceil_div(Nc, 256)));
      k_box_partial<<<G, 256, 0, st>>>(Nc, pt_raw, nullptr, ppart);
      k_box_final<<<1, 6 * 32, 0, st>>>(G, ppart, pbox, 6);
    }
    k_morton<<<ceil_div(Nc, TB), TB, 0, st>>>(Nc, pt_raw, pbox, i1, k2);
    // i2 = identity positions into the (a,b)-sorted list (i0 still holds 0..Nc-1)
    QP_CUDA(cudaMemcpyAsync(i2, i0, sizeof(int) * (size_t)Nc, cudaMemcpyDeviceToDevice, st));
    tmp_bytes = t2;
    QP_CUDA(cub::DeviceRadixSort::SortPairs(tmp, tmp_bytes, k2, k2s, i2, i3, Nc, 0, 3 * MORTON_BITS, st));
    // 5. gather final arrays (contact c <- raw i1[i3[c]])
    k_gather<<<ceil_div(Nc, TB), TB, 0, st>>>(Nc, M, i3, i1, wa, wb, phi_raw, nrm_raw, pt_raw, s->pos,
                                              c->ca.as<int>(), c->cb.as<int>(), c->cplane.as<int>(),
                                              c->phi.as<double>(),
                                              c->frame.as<double>(), c->point.as<double>(), c->arm_a.as<double>(),
                                              c->arm_b.as<double>(), c->rec64.as<double>(),
                                              c->rec32.as<float>());
    QP_CUDA(cudaMemcpyAsync(c->key.p, k2s, sizeof(unsigned long long) * (size_t)Nc, cudaMemcpyDeviceToDevice, st));
    QP_CUDA(cudaGetLastError());
  }
  // 6. body -> contact incidence (CSR, per-body lists sorted by contact)
  int* cnt = count;  // reuse: M+1 ints
  QP_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * ((size_t)M + 1), st));
  if (Nc > 0) k_inc_count<<<ceil_div(Nc, TB), TB, 0, st>>>(Nc, M, c->ca.as<int>(), c->cb.as<int>(), cnt);
  tmp_bytes = 0;
  cub::DeviceScan::ExclusiveSum(nullptr, tmp_bytes, cnt, bptr, M + 1, st);
  tmp = c->scratch[3].ensure(tmp_bytes);
  QP_CUDA(cub::DeviceScan::ExclusiveSum(tmp, tmp_bytes, cnt, bptr, M + 1, st));
  if (Nc > 0) {
    QP_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * ((size_t)M + 1), st));
    k_inc_fill<<<ceil_div(Nc, TB), TB, 0, st>>>(Nc, M, c->ca.as<int>(), c->cb.as<int>(), bptr, cnt,
                                                c->inc.as<int>());
    k_inc_sort<<<ceil_div(M, TB), TB, 0, st>>>(M, bptr, c->inc.as<int>());
    // 7. r (Eq. rdef)
    k_rvec<<<ceil_div(Nc, TB), TB, 0, st>>>(Nc, M, slots, c->ca.as<int>(), c->cb.as<int>(), c->phi.as<double>(),
                                            c->frame.as<double>(), c->arm_a.as<double>(), c->arm_b.as<double>(),
                                            s->vel, s->omega, s->gravity[0], s->gravity[1], s->gravity[2], s->dt,
                                            c->r.as<double>());
  }
  QP_CUDA(cudaGetLastError());
  QP_CUDA(cudaStreamSynchronize(st));
  c->have_contacts = true;
  c->part_G = 0;  // the Krylov partition follows the contact set
  c->apart_G = 0;  // and so does the fused apply's

  out->M = M;
  out->Nc = Nc;
  out->L = L;
  out->slots = slots;
  out->P = P;
  out->body_a = c->ca.as<int>();
  out->body_b = c->cb.as<int>();
  out->phi = c->phi.as<double>();
  out->frame = c->frame.as<double>();
  out->point = c->point.as<double>();
  out->arm_a = c->arm_a.as<double>();
  out->arm_b = c->arm_b.as<double>();
  out->key = c->key.as<unsigned long long>();
  out->r = c->r.as<double>();
  out->plane = c->cplane.as<int>();
}

}  // namespace qp

extern "C" int ccp_assemble(qp_ctx_t c, const qp_scene* s, qp_contacts* out) {
  if (!c) return QP_INVALID_ARG;
  try {
    qp::assemble(c, s, out);
    return QP_OK;
  } catch (const qp::Error& e) {
    qp::set_error(c, e);
    return e.code;
  }
}
