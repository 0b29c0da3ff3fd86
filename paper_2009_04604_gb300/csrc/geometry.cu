// geometry.cu -- link-geometry kernels: node flags, boundary records, q and u_w
// from analytic shapes, computed on the device (lbm_build_geometry).
//
// q of a wall link (x_F, i) is the smallest t in (0,1] at which the segment
// x_F - t c_i enters a shape (the normalised wall distance along the link,
// Sec. II.B). u_w is the rigid-body velocity v + om x (x_W - c) at the wall point
// x_W = x_F - q c_i (Sec. II.E). This file is compiled with -fmad=false. The
// solid tests then round exactly like the plain FP64 definition, so the flags
// are reproducible bit for bit.
//
// A thin shell (LBM_SHAPE_SHELL) makes no node solid: a link between two fluid
// nodes on different sides of it (one strictly inside |x - c| < r0, one not) is
// a wall link of both nodes, with q measured from each end. The records mark
// those links (Rec::shell) and the nodes carry F_SHELL; the inner side's links
// get the force tag TAG_INNER.
//
// Candidate shapes of a node come from a uniform cell list. Each cell lists, in
// increasing shape index, every shape whose bounding box padded by 2 lattice
// units overlaps the cell. Unbounded shapes (sphere-outside, strip) sit in every
// cell.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "lbm.h"
#include "geometry.hpp"
#include "kernels.cuh"
#include "launch.hpp"
#include "sim.hpp"

namespace lbm {

struct GeoShape {
  int type, tag;
  double c[3], r[3], nrm[3];
  double off, width, period;
  double v[3], om[3], v1[3], om1[3];
  double ca, sa;  // ellipsoid: cos and sin of its rotation about the z axis
};

// rotation of a shape about z, as its cosine and sine
__host__ __device__ inline void set_rotation(GeoShape &s, double ang) {
  s.ca = cos(ang);
  s.sa = sin(ang);
}

struct GeoView {
  View v;
  int D;
  const uint8_t *base;     // [N] caller's node kinds (unpadded) or null
  const double *base_u;    // [N*3] or null
  const GeoShape *shapes;
  const int *cell_start;   // [ncell + 1]
  const int *cell_items;
  int cs, cnx, cny, cnz;   // cell size and counts
  uint32_t *err;           // set to 1 when a fluid node lies exactly on a thin shell
};

__device__ __forceinline__ int cell_of(const GeoView &g, int x, int y, int z) {
  const int a = min(x / g.cs, g.cnx - 1), b = min(y / g.cs, g.cny - 1), c = min(z / g.cs, g.cnz - 1);
  return (c * g.cny + b) * g.cnx + a;
}

// point inside the solid of the shape (ties count as solid)
__device__ bool shape_solid(const GeoShape &s, int D, double x0, double x1, double x2) {
  const double d0 = x0 - s.c[0], d1 = x1 - s.c[1], d2 = D == 3 ? x2 - s.c[2] : 0.0;
  switch (s.type) {
    case LBM_SHAPE_SPHERE: return d0 * d0 + d1 * d1 + d2 * d2 <= s.r[0] * s.r[0];
    case LBM_SHAPE_SPHERE_OUT: return d0 * d0 + d1 * d1 + d2 * d2 >= s.r[0] * s.r[0];
    case LBM_SHAPE_ELLIPSOID: {
      // the offset in the body frame: turned by -ang about z
      const double b0 = s.ca * d0 + s.sa * d1, b1 = s.ca * d1 - s.sa * d0;
      const double t0 = b0 / s.r[0], t1 = b1 / s.r[1], t2 = D == 3 ? d2 / s.r[2] : 0.0;
      return t0 * t0 + t1 * t1 + t2 * t2 <= 1.0;
    }
    case LBM_SHAPE_STRIP: {
      double w = s.nrm[0] * x0 + s.nrm[1] * x1 + (D == 3 ? s.nrm[2] * x2 : 0.0) - s.off;
      if (s.period > 0.0) w = w - s.period * floor(w / s.period + 0.5);
      return fabs(w) >= 0.5 * s.width;
    }
  }
  return false;
}

// strictly inside a thin shell
__device__ __forceinline__ bool shell_inside(const GeoShape &s, int D, double x0, double x1, double x2) {
  const double d0 = x0 - s.c[0], d1 = x1 - s.c[1], d2 = D == 3 ? x2 - s.c[2] : 0.0;
  return d0 * d0 + d1 * d1 + d2 * d2 < s.r[0] * s.r[0];
}

// smallest t in (0,1] with x - t e on the shape boundary, entering the solid (any
// crossing for a thin shell); -1 if none. Quadratic roots in the cancellation-free form.
__device__ double shape_cross(const GeoShape &s, int D, const double x[3], const int ci[3]) {
  double d[3], e[3];
  for (int a = 0; a < 3; ++a) {
    d[a] = a < D ? x[a] - s.c[a] : 0.0;
    e[a] = a < D ? (double)ci[a] : 0.0;
  }
  if (s.type == LBM_SHAPE_STRIP) {
    double w = s.nrm[0] * x[0] + s.nrm[1] * x[1] + (D == 3 ? s.nrm[2] * x[2] : 0.0) - s.off;
    if (s.period > 0.0) w = w - s.period * floor(w / s.period + 0.5);
    const double a = s.nrm[0] * e[0] + s.nrm[1] * e[1] + s.nrm[2] * e[2];
    const double h = 0.5 * s.width;
    double t;
    if (a > 0.0) t = (w + h) / a;
    else if (a < 0.0) t = (w - h) / a;
    else return -1.0;
    return (t > 0.0 && t <= 1.0) ? t : -1.0;
  }
  double R2 = 1.0;
  if (s.type == LBM_SHAPE_ELLIPSOID) {
    // offset and link direction in the body frame, scaled to the unit sphere
    const double d0 = s.ca * d[0] + s.sa * d[1], d1 = s.ca * d[1] - s.sa * d[0];
    const double e0 = s.ca * e[0] + s.sa * e[1], e1 = s.ca * e[1] - s.sa * e[0];
    d[0] = d0; d[1] = d1; e[0] = e0; e[1] = e1;
    for (int a = 0; a < D; ++a) { d[a] = d[a] / s.r[a]; e[a] = e[a] / s.r[a]; }
  } else {
    R2 = s.r[0] * s.r[0];
  }
  const double A = e[0] * e[0] + e[1] * e[1] + e[2] * e[2];
  const double B = d[0] * e[0] + d[1] * e[1] + d[2] * e[2];
  const double C = d[0] * d[0] + d[1] * d[1] + d[2] * d[2] - R2;
  const double disc = B * B - A * C;
  if (disc < 0.0) return -1.0;
  const double sq = sqrt(disc);
  double t;
  if (s.type == LBM_SHAPE_SHELL) {
    // both roots (B -/+ sq) / A; the smaller one when it lies in (0,1]
    const double qq = B >= 0.0 ? B + sq : B - sq;
    const double ta = qq != 0.0 ? C / qq : -1.0, tb = qq / A;
    const double lo = fmin(ta, tb), hi = fmax(ta, tb);
    t = (lo > 0.0 && lo <= 1.0) ? lo : hi;
  } else if (s.type != LBM_SHAPE_SPHERE_OUT) {
    if (C <= 0.0 || B <= 0.0) return -1.0;
    t = C / (B + sq);
  } else {
    if (C >= 0.0) return -1.0;
    t = (B >= 0.0) ? (B + sq) / A : C / (B - sq);
  }
  return (t > 0.0 && t <= 1.0) ? t : -1.0;
}

template <class L>
__device__ __forceinline__ void dir(int i, int c[3]) { c[0] = L::cx(i); c[1] = L::cy(i); c[2] = L::cz(i); }

// Links of the fluid node n = (x, y, z) that cross a thin shell to a fluid node
// (bit i: towards n - c_i). flags: kinds in the low two bits.
template <class L>
__device__ uint32_t shell_links(const GeoView &g, const uint8_t *flags, long long n, const Nbr &nb,
                                int x, int y, int z) {
  const int cell = cell_of(g, x, y, z);
  uint32_t m = 0;
  for (int j = g.cell_start[cell]; j < g.cell_start[cell + 1]; ++j) {
    const GeoShape &s = g.shapes[g.cell_items[j]];
    if (s.type != LBM_SHAPE_SHELL) continue;
    const bool in = shell_inside(s, g.D, (double)x, (double)y, (double)z);
#pragma unroll 1
    for (int i = 0; i < L::Q; ++i) {
      int c[3];
      dir<L>(i, c);
      if (c[0] == 0 && c[1] == 0 && c[2] == 0) continue;
      if ((flags[n + nb.at(-c[0], -c[1], -c[2])] & 3) != K_FLUID) continue;
      if (shell_inside(s, g.D, (double)(x - c[0]), (double)(y - c[1]), (double)(z - c[2])) != in)
        m |= 1u << i;
    }
  }
  return m;
}

// 1. node kinds: the caller's base flags, turned SOLID inside any shape
__global__ void k_geo_flags(const GeoView g, uint8_t *__restrict__ flags) {
  const View &v = g.v;
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= v.np) return;
  const int x = (int)(n % v.nxp), y = (int)((n / v.nxp) % v.ny), z = (int)(n / ((long long)v.nxp * v.ny));
  if (x >= v.nx) { flags[n] = K_PAD; return; }
  const long long hn = ((long long)z * v.ny + y) * v.nx + x;
  uint8_t k = g.base ? g.base[hn] : (uint8_t)K_FLUID;
  if (k == K_FLUID) {
    const int cell = cell_of(g, x, y, z);
    for (int j = g.cell_start[cell]; j < g.cell_start[cell + 1]; ++j)
      if (shape_solid(g.shapes[g.cell_items[j]], g.D, (double)x, (double)y, (double)z)) { k = K_SOLID; break; }
    if (k == K_FLUID)
      for (int j = g.cell_start[cell]; j < g.cell_start[cell + 1]; ++j) {
        const GeoShape &s = g.shapes[g.cell_items[j]];
        if (s.type != LBM_SHAPE_SHELL) continue;
        const double d0 = x - s.c[0], d1 = y - s.c[1], d2 = g.D == 3 ? z - s.c[2] : 0.0;
        if (d0 * d0 + d1 * d1 + d2 * d2 == s.r[0] * s.r[0]) *g.err = 1u;
      }
  }
  flags[n] = k;
}

// 2. cut/open masks, boundary bit, and per-chunk counts of records and wall links
template <class L>
__global__ void k_geo_count(const GeoView g, uint8_t *__restrict__ flags, uint32_t *__restrict__ crec,
                            uint32_t *__restrict__ clink) {
  const View &v = g.v;
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= v.np) return;  // np is a multiple of 32: whole warps leave together
  const int x = (int)(n % v.nxp), y = (int)((n / v.nxp) % v.ny), z = (int)(n / ((long long)v.nxp * v.ny));
  uint32_t cut = 0, open = 0, shell = 0;
  const uint8_t k = flags[n] & 3;
  if (k == K_FLUID) {
    Nbr nb;
    nb.init(v, x, y, z);
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
      if (L::cx(i) == 0 && L::cy(i) == 0 && L::cz(i) == 0) continue;
      const uint8_t km = flags[n + nb.at(-L::cx(i), -L::cy(i), -L::cz(i))] & 3;
      if (km == K_SOLID) cut |= 1u << i;
      else if (km == K_OPEN) open |= 1u << i;
    }
    shell = shell_links<L>(g, flags, n, nb, x, y, z);
    cut |= shell;
  }
  const bool isb = (cut | open) != 0;
  const uint32_t bal = __ballot_sync(0xffffffffu, isb);
  uint32_t nl = __popc(cut);
  for (int o = 16; o > 0; o >>= 1) nl += __shfl_down_sync(0xffffffffu, nl, o);
  if ((threadIdx.x & 31) == 0) {
    crec[n >> 5] = __popc(bal);
    clink[n >> 5] = nl;
  }
  __syncwarp();
  if (isb) flags[n] = k | F_BOUNDARY | (shell ? F_SHELL : 0);
}

// Planes of a non-fluid node whose slot receives a value written ahead: bit i when
// the node n + c_i is fluid (its link i is a wall or open link, and the step
// writes its incoming population into slot (i, n)). Fluid and padding nodes get 0.
template <class L>
__global__ void k_geo_amask(const View v, uint32_t *__restrict__ amask) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= v.np) return;
  const int x = (int)(n % v.nxp), y = (int)((n / v.nxp) % v.ny), z = (int)(n / ((long long)v.nxp * v.ny));
  uint32_t m = 0;
  if (x < v.nx && (v.flags[n] & 3) != K_FLUID) {
    Nbr nb;
    nb.init(v, x, y, z);
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
      if (L::cx(i) == 0 && L::cy(i) == 0 && L::cz(i) == 0) continue;
      if ((v.flags[n + nb.at(L::cx(i), L::cy(i), L::cz(i))] & 3) == K_FLUID) m |= 1u << i;
    }
  }
  amask[n] = m;
}

// 3. exclusive scan of per-chunk counts (three launches: blocks, block totals, add)
__global__ void k_scan_block(uint32_t *__restrict__ a, long long n, uint32_t *__restrict__ tot) {
  __shared__ uint32_t ws[32];
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t x = i < n ? a[i] : 0u;
  uint32_t s = x;  // inclusive warp scan
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) >= o) s += y;
  }
  if ((threadIdx.x & 31) == 31) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    uint32_t t = ws[threadIdx.x];
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
      if (threadIdx.x >= o) t += y;
    }
    ws[threadIdx.x] = t;
  }
  __syncthreads();
  const uint32_t warp_off = (threadIdx.x >> 5) ? ws[(threadIdx.x >> 5) - 1] : 0u;
  if (i < n) a[i] = warp_off + s - x;
  if (threadIdx.x == blockDim.x - 1) tot[blockIdx.x] = warp_off + s;
}

__global__ void k_scan_totals(uint32_t *__restrict__ tot, long long nblk, uint32_t *__restrict__ total) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  uint32_t run = 0;
  for (long long b = 0; b < nblk; ++b) {
    const uint32_t t = tot[b];
    tot[b] = run;
    run += t;
  }
  *total = run;
}

__global__ void k_scan_add(uint32_t *__restrict__ a, long long n, const uint32_t *__restrict__ tot) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] += tot[blockIdx.x];
}

// 4. records and per-link q, u_w(t), u_w(t+1), tag
template <class L, typename LT>
__global__ void k_geo_fill(const GeoView g, const uint32_t *__restrict__ cbase,
                           const uint32_t *__restrict__ lbase, Rec *__restrict__ rec,
                           uint32_t *__restrict__ rnode, LT *__restrict__ lq, LT *__restrict__ luw,
                           LT *__restrict__ luw1, uint8_t *__restrict__ ltag) {
  const View &v = g.v;
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= v.np) return;  // whole warps
  const int x = (int)(n % v.nxp), y = (int)((n / v.nxp) % v.ny), z = (int)(n / ((long long)v.nxp * v.ny));
  const uint8_t fl = v.flags[n];
  const bool isb = (fl & F_BOUNDARY) != 0;
  const uint32_t bal = __ballot_sync(0xffffffffu, isb);
  Nbr nb;
  nb.init(v, x, y, z);
  Rec r = {0u, 0u, 0u, 0u, 0u};
  if (isb) {
    r.shell = (fl & F_SHELL) ? shell_links<L>(g, v.flags, n, nb, x, y, z) : 0u;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
      if (L::cx(i) == 0 && L::cy(i) == 0 && L::cz(i) == 0) continue;
      const uint8_t km = v.flags[n + nb.at(-L::cx(i), -L::cy(i), -L::cz(i))] & 3;
      if (km == K_SOLID || (r.shell & (1u << i))) r.cut |= 1u << i;
      else if (km == K_OPEN) r.open |= 1u << i;
      else continue;
      // the second node must be fluid and on this node's side of any shell
      if ((v.flags[n + nb.at(L::cx(i), L::cy(i), L::cz(i))] & 3) == K_FLUID && !((r.shell >> opp<L>(i)) & 1u))
        r.ffok |= 1u << i;
    }
  }
  // exclusive warp scan of the wall-link counts gives this node's first link
  const uint32_t cnt = __popc(r.cut);
  uint32_t s = cnt;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) >= o) s += t;
  }
  if (!isb) return;
  const uint32_t lt = (1u << (threadIdx.x & 31)) - 1u;
  const uint32_t rid = cbase[n >> 5] + __popc(bal & lt);
  r.link0 = lbase[n >> 5] + s - cnt;
  rnode[rid] = (uint32_t)n;
  bool moving_node = false;
  const double X[3] = {(double)x, (double)y, (double)z};
  const int cell = cell_of(g, x, y, z);
  uint32_t li = r.link0;
  for (int i = 0; i < L::Q; ++i) {
    if (!(r.cut & (1u << i))) continue;
    int c[3];
    dir<L>(i, c);
    const long long m = n + nb.at(-c[0], -c[1], -c[2]);
    double qq = 0.5, u0[3] = {0.0, 0.0, 0.0}, u1[3] = {0.0, 0.0, 0.0};
    int tg = 0;
    const bool across = (r.shell >> i) & 1u;
    // the neighbour's kind in the caller's base flags decides who cut the link
    const int mx = (int)(m % v.nxp), my = (int)((m / v.nxp) % v.ny), mz = (int)(m / ((long long)v.nxp * v.ny));
    const long long hm = ((long long)mz * v.ny + my) * v.nx + mx;
    const uint8_t bk = g.base ? g.base[hm] : (uint8_t)K_FLUID;
    if (bk != K_FLUID && !across) {
      if (g.base_u && bk == K_SOLID)
        for (int a = 0; a < 3; ++a) { u0[a] = g.base_u[hm * 3 + a]; u1[a] = u0[a]; }
    } else {
      double best = 2.0;
      int kb = -1;
      for (int j = g.cell_start[cell]; j < g.cell_start[cell + 1]; ++j) {
        const int k = g.cell_items[j];
        const double t = shape_cross(g.shapes[k], g.D, X, c);
        if (t > 0.0 && t < best) { best = t; kb = k; }
      }
      // the first shell (in shape order) whose sides the link joins
      int ks = -1;
      if (across)
        for (int j = g.cell_start[cell]; j < g.cell_start[cell + 1] && ks < 0; ++j) {
          const GeoShape &s = g.shapes[g.cell_items[j]];
          if (s.type == LBM_SHAPE_SHELL &&
              shell_inside(s, g.D, X[0], X[1], X[2]) != shell_inside(s, g.D, X[0] - c[0], X[1] - c[1], X[2] - c[2]))
            ks = g.cell_items[j];
        }
      if (kb < 0) {
        // no root (rounding at a tangent): the wall sits on the far node
        best = 1.0;
        for (int j = g.cell_start[cell]; j < g.cell_start[cell + 1]; ++j) {
          const int k = g.cell_items[j];
          if (shape_solid(g.shapes[k], g.D, X[0] - c[0], X[1] - c[1], X[2] - c[2]) || k == ks) { kb = k; break; }
        }
      }
      qq = best;
      if (kb >= 0) {
        const GeoShape &sh = g.shapes[kb];
        double rr[3];
        for (int a = 0; a < 3; ++a) rr[a] = a < g.D ? X[a] - qq * c[a] - sh.c[a] : 0.0;
        u0[0] = sh.v[0] + sh.om[1] * rr[2] - sh.om[2] * rr[1];
        u0[1] = sh.v[1] + sh.om[2] * rr[0] - sh.om[0] * rr[2];
        u0[2] = sh.v[2] + sh.om[0] * rr[1] - sh.om[1] * rr[0];
        u1[0] = sh.v1[0] + sh.om1[1] * rr[2] - sh.om1[2] * rr[1];
        u1[1] = sh.v1[1] + sh.om1[2] * rr[0] - sh.om1[0] * rr[2];
        u1[2] = sh.v1[2] + sh.om1[0] * rr[1] - sh.om1[1] * rr[0];
        if (g.D == 2) { u0[2] = 0.0; u1[2] = 0.0; }
        const bool inner = ks >= 0 && shell_inside(g.shapes[ks], g.D, X[0], X[1], X[2]);
        tg = inner ? TAG_INNER : sh.tag;
      }
    }
    if (u0[0] != 0.0 || u0[1] != 0.0 || u0[2] != 0.0 || u1[0] != 0.0 || u1[1] != 0.0 || u1[2] != 0.0)
      moving_node = true;
    lq[li] = (LT)qq;
    ltag[li] = (uint8_t)tg;
    if (luw) for (int a = 0; a < 3; ++a) { luw[3 * li + a] = (LT)u0[a]; luw1[3 * li + a] = (LT)u1[a]; }
    ++li;
  }
  if (moving_node) r.open |= REC_MOVING;
  rec[rid] = r;
}

cudaError_t launch_amask(int lattice, const View &v, uint32_t *amask, cudaStream_t s) {
  const unsigned blocks = (unsigned)((v.np + 255) / 256);
  if (lattice == 0) k_geo_amask<D2Q9><<<blocks, 256, 0, s>>>(v, amask);
  else if (lattice == 1) k_geo_amask<D3Q19><<<blocks, 256, 0, s>>>(v, amask);
  else k_geo_amask<D3Q27><<<blocks, 256, 0, s>>>(v, amask);
  return cudaGetLastError();
}

}  // namespace lbm

using namespace lbm;

void exclusive_scan(uint32_t *a, long long n, uint32_t *tot, uint32_t *total, cudaStream_t st);

#define GEO_CUDA(call)                                                                          \
  do {                                                                                          \
    cudaError_t e_ = (call);                                                                    \
    if (e_ != cudaSuccess) {                                                                    \
      rc = lbm_fail(h, e_ == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA,            \
                    std::string(#call) + ": " + cudaGetErrorString(e_));                        \
      goto done;                                                                                \
    }                                                                                           \
  } while (0)

#define LBM_CUDA_GEO(h, call)                                                                   \
  do {                                                                                          \
    cudaError_t e_ = (call);                                                                    \
    if (e_ != cudaSuccess)                                                                      \
      return lbm_fail((h), e_ == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA,        \
                      std::string(#call) + ": " + cudaGetErrorString(e_));                      \
  } while (0)

static void shape_box(const lbm_shape &s, int D, double lo[3], double hi[3], bool &bounded) {
  bounded = s.type == LBM_SHAPE_SPHERE || s.type == LBM_SHAPE_ELLIPSOID || s.type == LBM_SHAPE_SHELL;
  for (int a = 0; a < 3; ++a) {
    // a rotated ellipsoid stays inside max(r[0], r[1]) in x and y
    const double rxy = s.r[0] > s.r[1] ? s.r[0] : s.r[1];
    const double r = s.type == LBM_SHAPE_ELLIPSOID ? (a < 2 && s.ang != 0.0 ? rxy : s.r[a]) : s.r[0];
    lo[a] = (a < D) ? s.c[a] - r - 2.0 : -1e300;
    hi[a] = (a < D) ? s.c[a] + r + 2.0 : 1e300;
  }
}

void exclusive_scan(uint32_t *a, long long n, uint32_t *tot, uint32_t *total, cudaStream_t st) {
  const long long nblk = (n + 1023) / 1024;
  k_scan_block<<<(unsigned)nblk, 1024, 0, st>>>(a, n, tot);
  k_scan_totals<<<1, 1, 0, st>>>(tot, nblk, total);
  k_scan_add<<<(unsigned)nblk, 1024, 0, st>>>(a, n, tot);
}

extern "C" int lbm_build_geometry(lbm_handle h, const uint8_t *base, const double *base_u,
                                  const lbm_shape *shapes, int nshapes) {
  if (!h) return lbm_fail(nullptr, LBM_ERR_ARG, "null handle");
  if (nshapes < 0 || nshapes > 65536 || (nshapes > 0 && !shapes))
    return lbm_fail(h, LBM_ERR_ARG, "bad shape list");
  const int D = h->lattice == LBM_D2Q9 ? 2 : 3;
  for (int k = 0; k < nshapes; ++k) {
    const lbm_shape &s = shapes[k];
    if (s.type < LBM_SHAPE_SPHERE || s.type > LBM_SHAPE_SHELL) return lbm_fail(h, LBM_ERR_ARG, "unknown shape type");
    if (s.type == LBM_SHAPE_SHELL && !(s.r[0] >= 1.0))
      return lbm_fail(h, LBM_ERR_ARG, "a thin shell's radius must be at least 1");
    if (s.tag < 0 || s.tag > 7) return lbm_fail(h, LBM_ERR_ARG, "shape tags must be 0..7");
    if (s.type == LBM_SHAPE_ELLIPSOID)
      for (int a = 0; a < D; ++a) if (!(s.r[a] > 0.0)) return lbm_fail(h, LBM_ERR_ARG, "ellipsoid axes must be positive");
    if (s.type == LBM_SHAPE_STRIP && !(s.width > 0.0)) return lbm_fail(h, LBM_ERR_ARG, "strip width must be positive");
  }
  if (base)
    for (long long n = 0; n < h->N; ++n)
      if (base[n] > LBM_OPEN) return lbm_fail(h, LBM_ERR_ARG, "base flags must be 0, 1 or 2");

  // ---- cell list on the host
  const int cs = 8;
  const int cnx = (h->nx + cs - 1) / cs, cny = (h->ny + cs - 1) / cs, cnz = (h->nz + cs - 1) / cs;
  const long long ncell = (long long)cnx * cny * cnz;
  std::vector<std::vector<int>> lists(ncell);
  for (int k = 0; k < nshapes; ++k) {
    double lo[3], hi[3];
    bool bounded;
    shape_box(shapes[k], D, lo, hi, bounded);
    int a0[3], a1[3];
    const int cn[3] = {cnx, cny, cnz};
    for (int a = 0; a < 3; ++a) {
      if (!bounded || a >= D) { a0[a] = 0; a1[a] = cn[a] - 1; continue; }
      a0[a] = std::max(0, (int)std::floor(lo[a] / cs));
      a1[a] = std::min(cn[a] - 1, (int)std::floor(hi[a] / cs));
    }
    for (int cz = a0[2]; cz <= a1[2]; ++cz)
      for (int cy = a0[1]; cy <= a1[1]; ++cy)
        for (int cx = a0[0]; cx <= a1[0]; ++cx) lists[((long long)cz * cny + cy) * cnx + cx].push_back(k);
  }
  std::vector<int> cstart(ncell + 1, 0), items;
  for (long long c = 0; c < ncell; ++c) {
    cstart[c] = (int)items.size();
    items.insert(items.end(), lists[c].begin(), lists[c].end());
  }
  cstart[ncell] = (int)items.size();
  bool moving = false;
  std::vector<GeoShape> gs(nshapes);
  for (int k = 0; k < nshapes; ++k) {
    const lbm_shape &s = shapes[k];
    GeoShape &o = gs[k];
    o.type = s.type; o.tag = s.tag;
    for (int a = 0; a < 3; ++a) {
      o.c[a] = s.c[a]; o.r[a] = s.r[a]; o.nrm[a] = s.nrm[a];
      o.v[a] = s.v[a]; o.om[a] = s.om[a]; o.v1[a] = s.v1[a]; o.om1[a] = s.om1[a];
      if (s.v[a] != 0.0 || s.om[a] != 0.0 || s.v1[a] != 0.0 || s.om1[a] != 0.0) moving = true;
    }
    o.off = s.off; o.width = s.width; o.period = s.period;
    set_rotation(o, s.type == LBM_SHAPE_ELLIPSOID ? s.ang : 0.0);
  }
  if (base && base_u)
    for (long long n = 0; n < h->N && !moving; ++n)
      if (base[n] == LBM_SOLID && (base_u[3 * n] != 0.0 || base_u[3 * n + 1] != 0.0 || base_u[3 * n + 2] != 0.0))
        moving = true;

  int rc = LBM_OK;
  uint8_t *d_base = nullptr;
  double *d_base_u = nullptr;
  GeoShape *d_shapes = nullptr;
  int *d_cstart = nullptr, *d_items = nullptr;
  uint32_t *crec = nullptr, *clink = nullptr, *tot = nullptr, *totals = nullptr;
  uint32_t htot[3] = {0u, 0u, 0u};
  bool has_shell = false;
  for (int k = 0; k < nshapes; ++k) has_shell = has_shell || shapes[k].type == LBM_SHAPE_SHELL;
  const long long nchunk = h->np / 32;
  const long long nblk = (nchunk + 1023) / 1024;
  GeoView g;
  cudaStream_t st = h->stream;
  ++h->version;
  h->free_moving_body();
  h->drop_graphs();
  h->free_geometry();
  h->tiles_bx = h->tiles_by = 0;
  h->geom_ok = false;
  if (base) {
    GEO_CUDA(cudaMalloc(&d_base, h->N));
    GEO_CUDA(cudaMemcpyAsync(d_base, base, h->N, cudaMemcpyHostToDevice, st));
  }
  if (base && base_u) {
    GEO_CUDA(cudaMalloc(&d_base_u, h->N * 3 * sizeof(double)));
    GEO_CUDA(cudaMemcpyAsync(d_base_u, base_u, h->N * 3 * sizeof(double), cudaMemcpyHostToDevice, st));
  }
  GEO_CUDA(cudaMalloc(&d_shapes, std::max(1, nshapes) * sizeof(GeoShape)));
  if (nshapes) GEO_CUDA(cudaMemcpyAsync(d_shapes, gs.data(), nshapes * sizeof(GeoShape), cudaMemcpyHostToDevice, st));
  GEO_CUDA(cudaMalloc(&d_cstart, (ncell + 1) * sizeof(int)));
  GEO_CUDA(cudaMemcpyAsync(d_cstart, cstart.data(), (ncell + 1) * sizeof(int), cudaMemcpyHostToDevice, st));
  GEO_CUDA(cudaMalloc(&d_items, std::max<size_t>(1, items.size()) * sizeof(int)));
  if (!items.empty())
    GEO_CUDA(cudaMemcpyAsync(d_items, items.data(), items.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  GEO_CUDA(cudaMalloc(&crec, (nchunk + 1) * sizeof(uint32_t)));
  GEO_CUDA(cudaMalloc(&clink, (nchunk + 1) * sizeof(uint32_t)));
  GEO_CUDA(cudaMalloc(&tot, (nblk + 1) * sizeof(uint32_t)));
  GEO_CUDA(cudaMalloc(&totals, 3 * sizeof(uint32_t)));
  GEO_CUDA(cudaMemsetAsync(totals, 0, 3 * sizeof(uint32_t), st));

  g.v = h->view();
  g.D = D;
  g.base = d_base;
  g.base_u = d_base_u;
  g.shapes = d_shapes;
  g.cell_start = d_cstart;
  g.cell_items = d_items;
  g.cs = cs; g.cnx = cnx; g.cny = cny; g.cnz = cnz;
  g.err = totals + 2;
  {
    const unsigned blocks = (unsigned)((h->np + 255) / 256);
    k_geo_flags<<<blocks, 256, 0, st>>>(g, h->flags);
    if (h->lattice == LBM_D2Q9) k_geo_count<D2Q9><<<blocks, 256, 0, st>>>(g, h->flags, crec, clink);
    else if (h->lattice == LBM_D3Q19) k_geo_count<D3Q19><<<blocks, 256, 0, st>>>(g, h->flags, crec, clink);
    else k_geo_count<D3Q27><<<blocks, 256, 0, st>>>(g, h->flags, crec, clink);
    GEO_CUDA(cudaGetLastError());
    exclusive_scan(crec, nchunk, tot, totals, st);
    exclusive_scan(clink, nchunk, tot, totals + 1, st);
    GEO_CUDA(cudaGetLastError());
    GEO_CUDA(cudaMemcpyAsync(htot, totals, 3 * sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    GEO_CUDA(cudaStreamSynchronize(st));
    if (htot[2]) {
      rc = lbm_fail(h, LBM_ERR_ARG, "a fluid node lies exactly on a thin shell");
      goto done;
    }
    // cbase: records before each chunk, plus the total at the end
    GEO_CUDA(cudaMemcpyAsync(h->cbase, crec, nchunk * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st));
    GEO_CUDA(cudaMemcpyAsync(h->cbase + nchunk, &totals[0], sizeof(uint32_t), cudaMemcpyDeviceToDevice, st));
    h->nb = htot[0];
    h->nl = htot[1];
    h->has_uw = moving ? 1 : 0;
    h->has_shell = has_shell ? 1 : 0;
    const size_t ls = h->link_size();
    if (h->nb) {
      GEO_CUDA(cudaMalloc(&h->rec, h->nb * sizeof(Rec)));
      GEO_CUDA(cudaMalloc(&h->rnode, h->nb * sizeof(uint32_t)));
    }
    if (h->nl) {
      GEO_CUDA(cudaMalloc(&h->lq, h->nl * ls));
      GEO_CUDA(cudaMalloc(&h->ltag, h->nl));
      if (moving) {
        GEO_CUDA(cudaMalloc(&h->luw, h->nl * 3 * ls));
        GEO_CUDA(cudaMalloc(&h->luw1, h->nl * 3 * ls));
      }
    }
    g.v = h->view();
    if (h->nb) {
      if (h->lattice == LBM_D2Q9) {
        if (ls == 8) k_geo_fill<D2Q9, double><<<blocks, 256, 0, st>>>(g, crec, clink, h->rec, h->rnode, (double *)h->lq, (double *)h->luw, (double *)h->luw1, h->ltag);
        else k_geo_fill<D2Q9, float><<<blocks, 256, 0, st>>>(g, crec, clink, h->rec, h->rnode, (float *)h->lq, (float *)h->luw, (float *)h->luw1, h->ltag);
      } else if (h->lattice == LBM_D3Q19) {
        if (ls == 8) k_geo_fill<D3Q19, double><<<blocks, 256, 0, st>>>(g, crec, clink, h->rec, h->rnode, (double *)h->lq, (double *)h->luw, (double *)h->luw1, h->ltag);
        else k_geo_fill<D3Q19, float><<<blocks, 256, 0, st>>>(g, crec, clink, h->rec, h->rnode, (float *)h->lq, (float *)h->luw, (float *)h->luw1, h->ltag);
      } else {
        if (ls == 8) k_geo_fill<D3Q27, double><<<blocks, 256, 0, st>>>(g, crec, clink, h->rec, h->rnode, (double *)h->lq, (double *)h->luw, (double *)h->luw1, h->ltag);
        else k_geo_fill<D3Q27, float><<<blocks, 256, 0, st>>>(g, crec, clink, h->rec, h->rnode, (float *)h->lq, (float *)h->luw, (float *)h->luw1, h->ltag);
      }
      GEO_CUDA(cudaGetLastError());
    }
    // fluid node count
    {
      std::vector<uint8_t> fl(h->np);
      GEO_CUDA(cudaMemcpyAsync(fl.data(), h->flags, h->np, cudaMemcpyDeviceToHost, st));
      GEO_CUDA(cudaStreamSynchronize(st));
      long long nf = 0;
      for (long long n = 0; n < h->np; ++n) nf += (fl[n] & 3) == K_FLUID;
      h->nfluid = nf;
    }
    rc = h->finish_geometry();
    if (rc) goto done;
    h->geom_ok = true;
  }
done:
  cudaStreamSynchronize(st);
  cudaFree(d_base); cudaFree(d_base_u); cudaFree(d_shapes); cudaFree(d_cstart); cudaFree(d_items);
  cudaFree(crec); cudaFree(clink); cudaFree(tot); cudaFree(totals);
  return rc;
}

// ====================================================================== moving body
// A rigid body on a prescribed trajectory (Sec. II.E: wall velocity at the link's
// wall point). After every step t -> t+1, inside the fixed region box that covers
// the body's whole trajectory:
//  1. k_move_update: node kinds for the pose at t+1. A node that turns fluid
//     (solid at t, fluid at t+1) is refilled with f^eq(rho0, u_body(x)). Its
//     gather slots are written in the buffer the next step reads. The paper
//     refills by local iterations (App. D); the equilibrium refill is this
//     library's simpler choice.
//  2. k_move_count, scan, k_move_fill: the boundary records of the region's
//     fluid nodes, with q and u_w at t+1 and u_w at t+2, in region order.
//  3. k_move_advance: the pose index moves on.
// Everything stays on the device, so the step loop remains one CUDA graph.
namespace lbm {

struct MoveGeo {
  View v;
  int D;
  const GeoShape *shape;   // the body at unit pose: centre and velocities come from traj
  const double *traj;      // [ntraj][9]
  int ntraj;
  const int *step;         // current pose index
  const double *state;     // free body: [angle, omega, centre, inertia] (null: traj)
  int ox, oy, oz, rx, ry, rz;
  long long rsize;
};

__device__ __forceinline__ GeoShape body_at(const MoveGeo &g, int k) {
  GeoShape s = *g.shape;
  if (g.state) {
    // free rotation about z through the fixed centre; the wall velocity at t+1 is
    // taken as the current one (the torque of the next step is not known yet)
    const double ang = g.state[0], om = g.state[1];
    for (int a = 0; a < 3; ++a) {
      s.c[a] = g.state[2 + a];
      s.v[a] = s.v1[a] = 0.0;
      s.om[a] = s.om1[a] = a == 2 ? om : 0.0;
    }
    set_rotation(s, ang);
    return s;
  }
  const double *p = g.traj + 9LL * (k % g.ntraj);
  const double *p1 = g.traj + 9LL * ((k + 1) % g.ntraj);
  for (int a = 0; a < 3; ++a) {
    s.c[a] = p[a]; s.v[a] = p[3 + a]; s.om[a] = p[6 + a];
    s.v1[a] = p1[3 + a]; s.om1[a] = p1[6 + a];
  }
  return s;
}

__device__ __forceinline__ void region_xyz(const MoveGeo &g, long long r, int &x, int &y, int &z) {
  x = g.ox + (int)(r % g.rx);
  y = g.oy + (int)((r / g.rx) % g.ry);
  z = g.oz + (int)(r / ((long long)g.rx * g.ry));
}

template <class L, typename S, typename M>
__global__ void k_move_update(const MoveGeo g, int koff, int refill, uint8_t *__restrict__ flags,
                              S *__restrict__ fout) {
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= g.rsize) return;
  int x, y, z;
  region_xyz(g, r, x, y, z);
  const View &v = g.v;
  const int n = (z * v.ny + y) * v.nxp + x;
  const GeoShape b = body_at(g, *g.step + koff);
  const uint8_t old = flags[n] & 3;
  const uint8_t now = shape_solid(b, g.D, (double)x, (double)y, (double)z) ? K_SOLID : K_FLUID;
  if (refill && old != K_FLUID && now == K_FLUID) {
    // u_body at the node at the new pose: v + om x (x - c)
    const double rx_ = x - b.c[0], ry_ = y - b.c[1], rz_ = g.D == 3 ? z - b.c[2] : 0.0;
    double u[3] = {b.v[0] + b.om[1] * rz_ - b.om[2] * ry_, b.v[1] + b.om[2] * rx_ - b.om[0] * rz_,
                   b.v[2] + b.om[0] * ry_ - b.om[1] * rx_};
    if (g.D == 2) u[2] = 0.0;
    const M ux = M(u[0]), uy = M(u[1]), uz = M(u[2]);
    const M usq = ux * ux + uy * uy + uz * uz;
    Nbr nb;
    nb.init(v, x, y, z);
#pragma unroll
    for (int i = 0; i < L::Q; ++i)
      fout[(long long)i * v.np + n + nb.at(-L::cx(i), -L::cy(i), -L::cz(i))] =
          to_store<S, M>(feq_s<L, M>(i, M(0), M(v.rho0), ux, uy, uz, usq));
  }
  flags[n] = now | F_KEEP;  // the lattice tiles never store into the region's non-fluid slots
}

// Local iteration refill (LIR), in three launches so that the neighbours' kinds
// at t are still in `flags` while fresh nodes are refilled:
//  1. k_move_kinds: the region's kinds at the new pose into nkind;
//  2. k_move_lir: every fresh node (not fluid at t, fluid at t+1) keeps the
//     values streamed to it from upstream nodes that were fluid at t (already in
//     its gather slots: those nodes' own post-collision stores), and finds the
//     others by `iters` local iterations of collide-and-bounce-back: start from
//     f^eq_i(rho0, u_b); collide at the node's density and the body velocity u_b
//     (the step's collision, with the body force); set each unknown f_i to the
//     node's post-collision f*_ibar plus 2 w_i rho c_i.u_b / c_s^2. The results
//     go into the gather slots of the unknown directions, which belong to nodes
//     that were the body's at t (never stored into by the lattice tiles);
//  3. k_move_commit: the new kinds into flags.
// The paper applies its modified LIR before the global collide and stream (App.
// D); here it runs at the end of step t, which comes to the same: before the
// collide and stream of step t+1.
template <class L>
__global__ void k_move_kinds(const MoveGeo g, int koff, uint8_t *__restrict__ nkind) {
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= g.rsize) return;
  int x, y, z;
  region_xyz(g, r, x, y, z);
  const GeoShape b = body_at(g, *g.step + koff);
  nkind[r] = shape_solid(b, g.D, (double)x, (double)y, (double)z) ? K_SOLID : K_FLUID;
}

template <class L, typename S, typename M>
__global__ void k_move_lir(const MoveGeo g, int koff, int iters, const uint8_t *__restrict__ flags,
                           const uint8_t *__restrict__ nkind, S *__restrict__ fout) {
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= g.rsize) return;
  int x, y, z;
  region_xyz(g, r, x, y, z);
  const View &v = g.v;
  const int n = (z * v.ny + y) * v.nxp + x;
  if ((flags[n] & 3) == K_FLUID || nkind[r] != K_FLUID) return;  // not a fresh node
  const GeoShape b = body_at(g, *g.step + koff);
  const double rx_ = x - b.c[0], ry_ = y - b.c[1], rz_ = g.D == 3 ? z - b.c[2] : 0.0;
  double ub[3] = {b.v[0] + b.om[1] * rz_ - b.om[2] * ry_, b.v[1] + b.om[2] * rx_ - b.om[0] * rz_,
                  b.v[2] + b.om[0] * ry_ - b.om[1] * rx_};
  if (g.D == 2) ub[2] = 0.0;
  using X = Ex<M>;
  const Par<M> P(v);
  const M ux = M(ub[0]), uy = M(ub[1]), uz = M(ub[2]);
  const M usq = X::fma(uz, uz, X::fma(uy, uy, X::mul(ux, ux)));
  Nbr nb;
  nb.init(v, x, y, z);
  M f[L::Q];
  uint32_t unknown = 0;
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    const int off = nb.at(-L::cx(i), -L::cy(i), -L::cz(i));
    if ((flags[n + off] & 3) == K_FLUID) {
      f[i] = to_math<S, M>(fout[(long long)i * v.np + n + off]);
    } else {
      unknown |= 1u << i;
      f[i] = feq_r<L, M>(i, M(0), P.rho0, ux, uy, uz, usq);
    }
  }
  for (int k = 0; k < iters; ++k) {
    Macro<L, M> m;
    M d = M(0);
#pragma unroll
    for (int i = 0; i < L::Q; ++i) d = X::add(d, f[i]);
    m.drho = d;
    m.rho = X::add(P.rho0, d);
    m.ux = ux; m.uy = uy; m.uz = uz; m.usq = usq;
    M post[L::Q];
#pragma unroll
    for (int i = 0; i < L::Q; ++i) post[i] = post_r<L, M>(v, P, i, f[i], f[opp<L>(i)], m);
#pragma unroll
    for (int i = 0; i < L::Q; ++i)
      if ((unknown >> i) & 1u) {
        const M me = X::mul(X::mul(X::mul(M(6), M(weight<L>(i))), m.rho), cdot_r<L, M>(i, ux, uy, uz));
        f[i] = X::add(post[opp<L>(i)], me);
      }
  }
#pragma unroll
  for (int i = 0; i < L::Q; ++i)
    if ((unknown >> i) & 1u)
      fout[(long long)i * v.np + n + nb.at(-L::cx(i), -L::cy(i), -L::cz(i))] = to_store<S, M>(f[i]);
}

__global__ void k_move_commit(const MoveGeo g, const uint8_t *__restrict__ nkind, uint8_t *__restrict__ flags) {
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= g.rsize) return;
  int x, y, z;
  region_xyz(g, r, x, y, z);
  const View &v = g.v;
  flags[(z * v.ny + y) * v.nxp + x] = nkind[r] | F_KEEP;
}

// per 32-node region chunk: records and wall links (the region's fluid nodes whose
// upstream neighbours are solid)
template <class L>
__global__ void k_move_count(const MoveGeo g, const uint8_t *__restrict__ flags, uint32_t *__restrict__ crec,
                             uint32_t *__restrict__ clink, long long rpad) {
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rpad) return;  // rpad is a multiple of 32: whole warps
  uint32_t cut = 0;
  if (r < g.rsize) {
    int x, y, z;
    region_xyz(g, r, x, y, z);
    const View &v = g.v;
    const int n = (z * v.ny + y) * v.nxp + x;
    if ((flags[n] & 3) == K_FLUID) {
      Nbr nb;
      nb.init(v, x, y, z);
#pragma unroll
      for (int i = 0; i < L::Q; ++i) {
        if (L::cx(i) == 0 && L::cy(i) == 0 && L::cz(i) == 0) continue;
        if ((flags[n + nb.at(-L::cx(i), -L::cy(i), -L::cz(i))] & 3) == K_SOLID) cut |= 1u << i;
      }
    }
  }
  const uint32_t bal = __ballot_sync(0xffffffffu, cut != 0);
  uint32_t nl = __popc(cut);
  for (int o = 16; o > 0; o >>= 1) nl += __shfl_down_sync(0xffffffffu, nl, o);
  if ((threadIdx.x & 31) == 0) {
    crec[r >> 5] = __popc(bal);
    clink[r >> 5] = nl;
  }
}

template <class L, typename LT>
__global__ void k_move_fill(const MoveGeo g, int koff, const uint8_t *__restrict__ flags,
                            const uint32_t *__restrict__ cbase, const uint32_t *__restrict__ lbase,
                            long long rpad, Rec *__restrict__ rec, uint32_t *__restrict__ rnode,
                            LT *__restrict__ lq, LT *__restrict__ luw, LT *__restrict__ luw1,
                            uint8_t *__restrict__ ltag) {
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rpad) return;
  const View &v = g.v;
  int x = 0, y = 0, z = 0, n = 0;
  Rec rc = {0u, 0u, 0u, 0u, 0u};
  Nbr nb;
  if (r < g.rsize) {
    region_xyz(g, r, x, y, z);
    n = (z * v.ny + y) * v.nxp + x;
    if ((flags[n] & 3) == K_FLUID) {
      nb.init(v, x, y, z);
#pragma unroll
      for (int i = 0; i < L::Q; ++i) {
        if (L::cx(i) == 0 && L::cy(i) == 0 && L::cz(i) == 0) continue;
        if ((flags[n + nb.at(-L::cx(i), -L::cy(i), -L::cz(i))] & 3) == K_SOLID) rc.cut |= 1u << i;
      }
    }
  }
  const uint32_t bal = __ballot_sync(0xffffffffu, rc.cut != 0);
  const uint32_t cnt = __popc(rc.cut);
  uint32_t s = cnt;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) >= o) s += t;
  }
  if (!rc.cut) return;
  const uint32_t lt = (1u << (threadIdx.x & 31)) - 1u;
  const uint32_t rid = cbase[r >> 5] + __popc(bal & lt);
  rc.link0 = lbase[r >> 5] + s - cnt;
  const GeoShape b = body_at(g, *g.step + koff);
  const double X[3] = {(double)x, (double)y, (double)z};
  bool moving = false;
  uint32_t li = rc.link0;
  for (int i = 0; i < L::Q; ++i) {
    if (!(rc.cut & (1u << i))) continue;
    const int c[3] = {L::cx(i), L::cy(i), L::cz(i)};
    double qq = shape_cross(b, g.D, X, c);
    if (qq <= 0.0) qq = 1.0;  // rounding at a tangent: the wall sits on the solid node
    double rr[3];
    for (int a = 0; a < 3; ++a) rr[a] = a < g.D ? X[a] - qq * c[a] - b.c[a] : 0.0;
    double u0[3] = {b.v[0] + b.om[1] * rr[2] - b.om[2] * rr[1], b.v[1] + b.om[2] * rr[0] - b.om[0] * rr[2],
                    b.v[2] + b.om[0] * rr[1] - b.om[1] * rr[0]};
    double u1[3] = {b.v1[0] + b.om1[1] * rr[2] - b.om1[2] * rr[1], b.v1[1] + b.om1[2] * rr[0] - b.om1[0] * rr[2],
                    b.v1[2] + b.om1[0] * rr[1] - b.om1[1] * rr[0]};
    if (g.D == 2) { u0[2] = 0.0; u1[2] = 0.0; }
    for (int a = 0; a < 3; ++a) {
      if (u0[a] != 0.0 || u1[a] != 0.0) moving = true;
      luw[3 * li + a] = (LT)u0[a];
      luw1[3 * li + a] = (LT)u1[a];
    }
    lq[li] = (LT)qq;
    ltag[li] = (uint8_t)b.tag;
    ++li;
  }
  if (moving) rc.open |= REC_MOVING;
  rec[rid] = rc;
  rnode[rid] = (uint32_t)n;
}

__global__ void k_move_advance(int *step) { *step += 1; }

// Free body: the torque of the step just taken (sum of the per-block partials, z
// component, in a fixed order) turns the body about z: omega += T / I, then
// angle += omega (semi-implicit Euler, unit time step). History entry `*step`
// records angle, omega and torque. One warp.
__global__ void k_body_rotate(const double *__restrict__ tpart, long long nblk, double *__restrict__ state,
                              double *__restrict__ hist, int cap, const int *__restrict__ step) {
  const int lane = threadIdx.x;
  double t = 0.0;
  for (long long b = lane; b < nblk; b += 32) t += tpart[b * 3 + 2];
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if (lane == 0) {
    const double om = state[1] + t / state[5];
    const double ang = state[0] + om;
    state[0] = ang;
    state[1] = om;
    if (cap > 0) {
      const long long k = *step % cap;
      hist[3 * k] = ang;
      hist[3 * k + 1] = om;
      hist[3 * k + 2] = t;
    }
  }
}

template <class Fn>
static cudaError_t move_dispatch(int lattice, int dtype, Fn &&fn) {
  if (lattice == 0) {
    switch (dtype) {
      case 0: return fn.template operator()<D2Q9, double, double>();
      case 1: return fn.template operator()<D2Q9, float, float>();
      case 2: return fn.template operator()<D2Q9, __half, float>();
      default: return fn.template operator()<D2Q9, __nv_bfloat16, float>();
    }
  }
  if (lattice == 2) {
    switch (dtype) {
      case 0: return fn.template operator()<D3Q27, double, double>();
      case 1: return fn.template operator()<D3Q27, float, float>();
      case 2: return fn.template operator()<D3Q27, __half, float>();
      default: return fn.template operator()<D3Q27, __nv_bfloat16, float>();
    }
  }
  switch (dtype) {
    case 0: return fn.template operator()<D3Q19, double, double>();
    case 1: return fn.template operator()<D3Q19, float, float>();
    case 2: return fn.template operator()<D3Q19, __half, float>();
    default: return fn.template operator()<D3Q19, __nv_bfloat16, float>();
  }
}

// Body geometry of pose (*step + koff) into record set `set`; refill fresh nodes in fout.
static cudaError_t move_geometry(lbm_sim *h, int koff, int refill, void *fout, int set) {
  MovingBody &mb = h->mb;
  MoveGeo g;
  g.v = h->view();
  g.D = h->lattice == LBM_D2Q9 ? 2 : 3;
  g.shape = static_cast<const GeoShape *>(mb.shape);
  g.traj = mb.traj;
  g.ntraj = mb.ntraj;
  g.step = mb.step;
  g.state = mb.free_rot ? mb.state : nullptr;
  g.ox = mb.ox; g.oy = mb.oy; g.oz = mb.oz; g.rx = mb.rx; g.ry = mb.ry; g.rz = mb.rz;
  g.rsize = mb.rsize;
  cudaStream_t st = h->stream;
  const unsigned blocks = (unsigned)((mb.rpad + 255) / 256);
  const long long nchunk = mb.rpad / 32;
  return move_dispatch(h->lattice, h->dtype, [&]<class L, typename S, typename M>() {
    if (refill && mb.refill_mode == LBM_REFILL_LIR) {
      k_move_kinds<L><<<blocks, 256, 0, st>>>(g, koff, mb.nkind);
      k_move_lir<L, S, M><<<blocks, 256, 0, st>>>(g, koff, mb.refill_iters, h->flags, mb.nkind,
                                                  static_cast<S *>(fout));
      k_move_commit<<<blocks, 256, 0, st>>>(g, mb.nkind, h->flags);
    } else {
      k_move_update<L, S, M><<<blocks, 256, 0, st>>>(g, koff, refill, h->flags, static_cast<S *>(fout));
    }
    k_move_count<L><<<blocks, 256, 0, st>>>(g, h->flags, mb.crec, mb.clink, mb.rpad);
    exclusive_scan(mb.crec, nchunk, mb.tot, reinterpret_cast<uint32_t *>(mb.count[set]), st);
    exclusive_scan(mb.clink, nchunk, mb.tot, mb.totals, st);
    k_move_fill<L, M><<<blocks, 256, 0, st>>>(g, koff, h->flags, mb.crec, mb.clink, mb.rpad, mb.rec[set],
                                              mb.rnode[set], static_cast<M *>(mb.lq[set]),
                                              static_cast<M *>(mb.luw[set]), static_cast<M *>(mb.luw1[set]),
                                              mb.ltag[set]);
    return cudaGetLastError();
  });
}

}  // namespace lbm

int lbm_sim::move_after_step(void *fout, int set) {
  // The body's momentum exchange of the step just taken (its records are set ^ 1).
  // It is taken before the refill, which may overwrite the outgoing populations
  // f*_ibar(x_F, t) of links whose solid node turns fluid.
  const int s = set ^ 1;
  const RecSet rs{mb.rec[s], mb.rnode[s], mb.lq[s], mb.luw[s], mb.luw1[s], mb.ltag[s]};
  Launch lf;
  lf.grid = dim3((unsigned)mb.nfpart);
  lf.block = dim3(256);
  lf.stream = stream;
  cudaError_t e = launch_force(lattice, dtype, view(), fout, nullptr, rs, 0, mb.count[s], -1, mb.fpart, lf,
                               mb.free_rot ? mb.tpart : nullptr, mb.centre[0], mb.centre[1], mb.centre[2]);
  if (e == cudaSuccess && mb.free_rot) {
    k_body_rotate<<<1, 32, 0, stream>>>(mb.tpart, mb.nfpart, mb.state, mb.hist, mb.hist_cap, mb.step);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = move_geometry(this, 1, 1, fout, set);
  if (e == cudaSuccess) {
    k_move_advance<<<1, 1, 0, stream>>>(mb.step);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return lbm_fail(this, LBM_ERR_CUDA, std::string("moving body: ") + cudaGetErrorString(e));
  return LBM_OK;
}

int lbm_sim::move_rebuild(long long pose) {
  const int k = (int)pose;
  LBM_CUDA_GEO(this, cudaMemcpyAsync(mb.step, &k, sizeof(int), cudaMemcpyHostToDevice, stream));
  cudaError_t e = move_geometry(this, 0, 0, f[cur], cur);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return lbm_fail(this, LBM_ERR_CUDA, std::string("moving body: ") + cudaGetErrorString(e));
  return LBM_OK;
}

void lbm_sim::free_moving_body() {
  if (!mb.on && !mb.traj) return;
  cudaStreamSynchronize(stream);
  cudaFree(mb.shape); cudaFree(mb.traj); cudaFree(mb.step); cudaFree(mb.fpart);
  cudaFree(mb.state); cudaFree(mb.tpart); cudaFree(mb.hist); cudaFree(mb.nkind);
  cudaFree(mb.crec); cudaFree(mb.clink); cudaFree(mb.tot); cudaFree(mb.totals);
  for (int k = 0; k < 2; ++k) {
    cudaFree(mb.rec[k]); cudaFree(mb.rnode[k]); cudaFree(mb.lq[k]); cudaFree(mb.luw[k]); cudaFree(mb.luw1[k]);
    cudaFree(mb.ltag[k]); cudaFree(mb.count[k]);
  }
  mb = MovingBody();
  tiles_bx = tiles_by = 0;
  drop_graphs();
}

// Region, buffers and first geometry of a moving body (prescribed trajectory,
// or free rotation when free_state is not null). lo/hi: the box the body's
// centre covers; ext: the body's half-extent along each axis.
static int setup_body(lbm_handle h, const lbm_shape *body, const double lo[3], const double hi[3],
                      const double ext[3], const double *traj, int ntraj, int t0, const double *free_state,
                      int history) {
  const int D = h->lattice == LBM_D2Q9 ? 2 : 3;
  // region: the box widened by the body and two links
  const int dims[3] = {h->nx, h->ny, h->nz};
  int o[3], e[3];
  for (int a = 0; a < 3; ++a) {
    if (a >= D) { o[a] = 0; e[a] = 1; continue; }
    o[a] = (int)std::floor(lo[a] - ext[a] - 2.0);
    const int hi_i = (int)std::ceil(hi[a] + ext[a] + 2.0);
    e[a] = hi_i - o[a] + 1;
    if (o[a] < 1 || hi_i > dims[a] - 2)
      return lbm_fail(h, LBM_ERR_ARG, "the moving body's region must stay one node inside the lattice");
  }
  // static kinds in the region, widened by one node, must all be fluid
  {
    std::vector<uint8_t> fl(h->np);
    LBM_CUDA_GEO(h, cudaMemcpyAsync(fl.data(), h->flags, h->np, cudaMemcpyDeviceToHost, h->stream));
    LBM_CUDA_GEO(h, cudaStreamSynchronize(h->stream));
    for (int z = (D == 3 ? o[2] - 1 : 0); z < (D == 3 ? o[2] + e[2] + 1 : 1); ++z)
      for (int y = o[1] - 1; y < o[1] + e[1] + 1; ++y)
        for (int x = o[0] - 1; x < o[0] + e[0] + 1; ++x)
          if ((fl[((long long)z * h->ny + y) * h->nxp + x] & 3) != K_FLUID)
            return lbm_fail(h, LBM_ERR_ARG, "the moving body's region overlaps static solid or open nodes");
  }
  h->free_moving_body();
  MovingBody &mb = h->mb;
  mb.ox = o[0]; mb.oy = o[1]; mb.oz = o[2]; mb.rx = e[0]; mb.ry = e[1]; mb.rz = e[2];
  mb.rsize = (long long)e[0] * e[1] * e[2];
  mb.rpad = (mb.rsize + 31) / 32 * 32;
  mb.ntraj = ntraj;
  mb.cap_rec = mb.rsize;
  mb.cap_link = mb.rsize * (h->Q - 1);
  mb.tag = body->tag;
  mb.nfpart = (mb.cap_rec + 255) / 256;
  GeoShape gs;
  std::memset(&gs, 0, sizeof(gs));
  gs.type = body->type;
  gs.tag = body->tag;
  for (int a = 0; a < 3; ++a) gs.r[a] = body->r[a];
  set_rotation(gs, body->type == LBM_SHAPE_ELLIPSOID ? body->ang : 0.0);
  const size_t ls = h->link_size();
  const long long nchunk = mb.rpad / 32;
  LBM_CUDA_GEO(h, cudaMalloc(&mb.shape, sizeof(GeoShape)));
  LBM_CUDA_GEO(h, cudaMalloc(&mb.traj, sizeof(double) * 9 * ntraj));
  LBM_CUDA_GEO(h, cudaMalloc(&mb.step, sizeof(int)));
  LBM_CUDA_GEO(h, cudaMalloc(&mb.fpart, sizeof(double) * 3 * mb.nfpart));
  LBM_CUDA_GEO(h, cudaMemsetAsync(mb.fpart, 0, sizeof(double) * 3 * mb.nfpart, h->stream));
  LBM_CUDA_GEO(h, cudaMalloc(&mb.crec, sizeof(uint32_t) * (nchunk + 1)));
  LBM_CUDA_GEO(h, cudaMalloc(&mb.clink, sizeof(uint32_t) * (nchunk + 1)));
  LBM_CUDA_GEO(h, cudaMalloc(&mb.tot, sizeof(uint32_t) * ((nchunk + 1023) / 1024 + 1)));
  LBM_CUDA_GEO(h, cudaMalloc(&mb.totals, sizeof(uint32_t) * 2));
  LBM_CUDA_GEO(h, cudaMalloc(&mb.nkind, mb.rpad));
  mb.refill_mode = h->refill_mode;
  mb.refill_iters = h->refill_iters;
  for (int k = 0; k < 2; ++k) {
    LBM_CUDA_GEO(h, cudaMalloc(&mb.rec[k], sizeof(Rec) * mb.cap_rec));
    LBM_CUDA_GEO(h, cudaMalloc(&mb.rnode[k], sizeof(uint32_t) * mb.cap_rec));
    LBM_CUDA_GEO(h, cudaMalloc(&mb.lq[k], ls * mb.cap_link));
    LBM_CUDA_GEO(h, cudaMalloc(&mb.luw[k], 3 * ls * mb.cap_link));
    LBM_CUDA_GEO(h, cudaMalloc(&mb.luw1[k], 3 * ls * mb.cap_link));
    LBM_CUDA_GEO(h, cudaMalloc(&mb.ltag[k], mb.cap_link));
    LBM_CUDA_GEO(h, cudaMalloc(&mb.count[k], sizeof(int)));
    LBM_CUDA_GEO(h, cudaMemsetAsync(mb.count[k], 0, sizeof(int), h->stream));
  }
  LBM_CUDA_GEO(h, cudaMemcpyAsync(mb.shape, &gs, sizeof(GeoShape), cudaMemcpyHostToDevice, h->stream));
  LBM_CUDA_GEO(h, cudaMemcpyAsync(mb.traj, traj, sizeof(double) * 9 * ntraj, cudaMemcpyHostToDevice, h->stream));
  LBM_CUDA_GEO(h, cudaMemcpyAsync(mb.step, &t0, sizeof(int), cudaMemcpyHostToDevice, h->stream));
  unsigned long long hh = 0xcbf29ce484222325ULL;  // identity of the body for lbm_save / lbm_load
  {
    const unsigned char *pb = reinterpret_cast<const unsigned char *>(&gs);
    for (size_t k = 0; k < sizeof(GeoShape); ++k) hh = (hh ^ pb[k]) * 0x100000001b3ULL;
    const unsigned char *pt = reinterpret_cast<const unsigned char *>(traj);
    for (size_t k = 0; k < sizeof(double) * 9 * (size_t)ntraj; ++k) hh = (hh ^ pt[k]) * 0x100000001b3ULL;
  }
  if (free_state) {
    mb.free_rot = true;
    for (int a = 0; a < 3; ++a) mb.centre[a] = free_state[2 + a];
    mb.hist_cap = history;
    LBM_CUDA_GEO(h, cudaMalloc(&mb.state, sizeof(double) * 6));
    LBM_CUDA_GEO(h, cudaMemcpyAsync(mb.state, free_state, sizeof(double) * 6, cudaMemcpyHostToDevice, h->stream));
    LBM_CUDA_GEO(h, cudaMalloc(&mb.tpart, sizeof(double) * 3 * mb.nfpart));
    LBM_CUDA_GEO(h, cudaMemsetAsync(mb.tpart, 0, sizeof(double) * 3 * mb.nfpart, h->stream));
    LBM_CUDA_GEO(h, cudaMalloc(&mb.hist, sizeof(double) * 3 * std::max(1, history)));
    LBM_CUDA_GEO(h, cudaMemsetAsync(mb.hist, 0, sizeof(double) * 3 * std::max(1, history), h->stream));
    const unsigned char *pf = reinterpret_cast<const unsigned char *>(free_state + 2);  // centre, inertia
    for (size_t k = 0; k < sizeof(double) * 4; ++k) hh = (hh ^ pf[k]) * 0x100000001b3ULL;
  }
  mb.hash = hh;
  mb.on = true;
  ++h->version;
  h->tiles_bx = h->tiles_by = 0;
  h->drop_graphs();
  // geometry of the first pose for the next step (no refill: the state is set
  // afterwards or was set on the static geometry)
  cudaError_t err = move_geometry(h, 0, 0, h->f[h->cur], h->cur);
  if (err == cudaSuccess) err = cudaStreamSynchronize(h->stream);
  if (err != cudaSuccess) return lbm_fail(h, LBM_ERR_CUDA, std::string("moving body: ") + cudaGetErrorString(err));
  // fluid node count of the current geometry
  std::vector<uint8_t> fl(h->np);
  LBM_CUDA_GEO(h, cudaMemcpy(fl.data(), h->flags, h->np, cudaMemcpyDeviceToHost));
  long long nf = 0;
  for (long long n = 0; n < h->np; ++n) nf += (fl[n] & 3) == K_FLUID;
  h->nfluid = nf;
  return LBM_OK;
}

static int check_body(lbm_handle h, const lbm_shape *body) {
  if (!h->geom_ok) return lbm_fail(h, LBM_ERR_STATE, "build the static geometry first");
  if (h->has_shell) return lbm_fail(h, LBM_ERR_ARG, "a moving body cannot share a geometry with thin shells");
  if (body->type != LBM_SHAPE_SPHERE && body->type != LBM_SHAPE_ELLIPSOID)
    return lbm_fail(h, LBM_ERR_ARG, "a moving body is a sphere or an ellipsoid");
  if (body->tag < 0 || body->tag > 7) return lbm_fail(h, LBM_ERR_ARG, "tags must be 0..7");
  if (h->bc == LBM_BC_BFL) return lbm_fail(h, LBM_ERR_ARG, "BFL cannot be used with a moving body");
  return LBM_OK;
}

extern "C" int lbm_set_moving_body(lbm_handle h, const lbm_shape *body, const double *traj, int ntraj, int t0) {
  if (!h || !body || !traj) return lbm_fail(h, LBM_ERR_ARG, "null argument");
  int rc = check_body(h, body);
  if (rc) return rc;
  if (ntraj < 2 || t0 < 0) return lbm_fail(h, LBM_ERR_ARG, "the trajectory needs at least two poses");
  double ext[3];
  const double rxy = std::max(body->r[0], body->r[1]);
  for (int a = 0; a < 3; ++a)
    ext[a] = body->type == LBM_SHAPE_ELLIPSOID ? (a < 2 && body->ang != 0.0 ? rxy : body->r[a]) : body->r[0];
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int k = 0; k < ntraj; ++k)
    for (int a = 0; a < 3; ++a) {
      lo[a] = std::min(lo[a], traj[9 * k + a]);
      hi[a] = std::max(hi[a], traj[9 * k + a]);
    }
  return setup_body(h, body, lo, hi, ext, traj, ntraj, t0, nullptr, 0);
}

extern "C" int lbm_set_free_body(lbm_handle h, const lbm_shape *body, double inertia, int history) {
  if (!h || !body) return lbm_fail(h, LBM_ERR_ARG, "null argument");
  int rc = check_body(h, body);
  if (rc) return rc;
  if (!(inertia > 0.0) || !std::isfinite(inertia)) return lbm_fail(h, LBM_ERR_ARG, "the inertia must be positive");
  if (history < 0) return lbm_fail(h, LBM_ERR_ARG, "negative history length");
  // the body turns about z through its centre: it sweeps a disc of its largest
  // in-plane semi-axis (a sphere: its radius)
  const double rxy = body->type == LBM_SHAPE_ELLIPSOID ? std::max(body->r[0], body->r[1]) : body->r[0];
  const double ext[3] = {rxy, rxy, body->type == LBM_SHAPE_ELLIPSOID ? body->r[2] : body->r[0]};
  const double traj[18] = {body->c[0], body->c[1], body->c[2], 0, 0, 0, 0, 0, 0,
                           body->c[0], body->c[1], body->c[2], 0, 0, 0, 0, 0, 0};
  const double state[6] = {body->type == LBM_SHAPE_ELLIPSOID ? body->ang : 0.0, body->om[2],
                           body->c[0], body->c[1], body->c[2], inertia};
  return setup_body(h, body, body->c, body->c, ext, traj, 2, 0, state, history);
}

extern "C" int lbm_get_body_history(lbm_handle h, double *out, int64_t *n) {
  if (!h || !n) return lbm_fail(h, LBM_ERR_ARG, "null argument");
  if (!h->mb.on || !h->mb.free_rot) return lbm_fail(h, LBM_ERR_STATE, "no free body");
  MovingBody &mb = h->mb;
  int steps = 0;
  LBM_CUDA_GEO(h, cudaStreamSynchronize(h->stream));
  LBM_CUDA_GEO(h, cudaMemcpy(&steps, mb.step, sizeof(int), cudaMemcpyDeviceToHost));
  const long long avail = std::min<long long>(steps, mb.hist_cap);
  if (!out) { *n = avail; return LBM_OK; }
  const long long want = std::min<long long>(*n, avail);
  std::vector<double> all((size_t)3 * std::max(1, mb.hist_cap));
  LBM_CUDA_GEO(h, cudaMemcpy(all.data(), mb.hist, sizeof(double) * 3 * mb.hist_cap, cudaMemcpyDeviceToHost));
  // the last `want` entries in step order: step k sits at k % cap
  for (long long j = 0; j < want; ++j) {
    const long long k = (steps - want + j) % mb.hist_cap;
    for (int c = 0; c < 3; ++c) out[3 * j + c] = all[3 * k + c];
  }
  *n = want;
  return LBM_OK;
}

extern "C" int lbm_set_refill(lbm_handle h, int mode, int iterations) {
  if (!h) return lbm_fail(nullptr, LBM_ERR_ARG, "null handle");
  if (mode != LBM_REFILL_EQUILIBRIUM && mode != LBM_REFILL_LIR) return lbm_fail(h, LBM_ERR_ARG, "unknown refill");
  if (iterations < 0 || iterations > 100000) return lbm_fail(h, LBM_ERR_ARG, "iterations must be 0..100000");
  h->refill_mode = mode;
  h->refill_iters = iterations;
  h->mb.refill_mode = mode;
  h->mb.refill_iters = iterations;
  h->drop_graphs();
  return LBM_OK;
}
