// lattice.cuh -- velocity sets, storage conversions and the shared kernel view
// of a simulation (device side of liblbm).
//
// Directions are ordered lexicographically by (c_z, c_y, c_x). With that order the
// opposite of direction i is Q-1-i and the rest population sits in the middle.
// Weights are the standard Gauss-Hermite weights of the D2Q9 / D3Q19 sets
// (Sec. II.A, c_s^2 = 1/3): 4/9, 1/9, 1/36 and 1/3, 1/18, 1/36.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace lbm {

struct D2Q9 {
  static constexpr int Q = 9;
  static constexpr int D = 2;
  __host__ __device__ static constexpr int cx(int i) { return i % 3 - 1; }
  __host__ __device__ static constexpr int cy(int i) { return i / 3 - 1; }
  __host__ __device__ static constexpr int cz(int) { return 0; }
};

struct D3Q19 {
  static constexpr int Q = 19;
  static constexpr int D = 3;
  // (cx, cy, cz) for i = 0..18, lexicographic in (cz, cy, cx):
  //  z=-1: (0,-1) (-1,0) (0,0) (1,0) (0,1)
  //  z= 0: (-1,-1) (0,-1) (1,-1) (-1,0) (0,0) (1,0) (-1,1) (0,1) (1,1)
  //  z=+1: (0,-1) (-1,0) (0,0) (1,0) (0,1)
  __host__ __device__ static constexpr int cz(int i) { return i < 5 ? -1 : (i < 14 ? 0 : 1); }
  __host__ __device__ static constexpr int cx(int i) {
    return (i < 5 || i >= 14) ? ((i % 9 == 1 || i == 15) ? -1 : ((i == 3 || i == 17) ? 1 : 0))
                              : ((i - 5) % 3 - 1);
  }
  __host__ __device__ static constexpr int cy(int i) {
    return (i < 5 || i >= 14) ? ((i == 0 || i == 14) ? -1 : ((i == 4 || i == 18) ? 1 : 0))
                              : ((i - 5) / 3 - 1);
  }
};

template <class L>
__host__ __device__ constexpr int c2(int i) {
  return L::cx(i) * L::cx(i) + L::cy(i) * L::cy(i) + L::cz(i) * L::cz(i);
}

// Gauss-Hermite weight of direction i, from |c_i|^2.
template <class L>
__host__ __device__ constexpr double weight(int i) {
  return L::Q == 9 ? (c2<L>(i) == 0 ? 4.0 / 9.0 : (c2<L>(i) == 1 ? 1.0 / 9.0 : 1.0 / 36.0))
                   : (c2<L>(i) == 0 ? 1.0 / 3.0 : (c2<L>(i) == 1 ? 1.0 / 18.0 : 1.0 / 36.0));
}

template <class L>
__host__ __device__ constexpr int opp(int i) { return L::Q - 1 - i; }

// ---- storage <-> math conversions (round to nearest even on store) ----
template <typename S, typename M> __device__ __forceinline__ M to_math(S v);
template <> __device__ __forceinline__ double to_math<double, double>(double v) { return v; }
template <> __device__ __forceinline__ float to_math<float, float>(float v) { return v; }
template <> __device__ __forceinline__ float to_math<__half, float>(__half v) { return __half2float(v); }
template <> __device__ __forceinline__ float to_math<__nv_bfloat16, float>(__nv_bfloat16 v) {
  return __bfloat162float(v);
}

template <typename S, typename M> __device__ __forceinline__ S to_store(M v);
template <> __device__ __forceinline__ double to_store<double, double>(double v) { return v; }
template <> __device__ __forceinline__ float to_store<float, float>(float v) { return v; }
template <> __device__ __forceinline__ __half to_store<__half, float>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 to_store<__nv_bfloat16, float>(float v) {
  return __float2bfloat16_rn(v);
}

// Node flag byte: low two bits are the kind, bit 2 marks a fluid node with at
// least one wall or open link (a boundary node with a record).
enum : uint8_t { K_FLUID = 0, K_SOLID = 1, K_OPEN = 2, K_PAD = 3, F_BOUNDARY = 4 };

// Boundary record of one boundary node (records are sorted by node index).
struct Rec {
  uint32_t cut;   // bit i: link i is a wall link (node n - c_i is SOLID)
  uint32_t open;  // bit i: link i is an open link (node n - c_i is OPEN)
  uint32_t ffok;  // bit i: the second node along the link, n + c_i, is fluid (BFL)
  uint32_t link0; // index of the first wall link of this node in the link arrays
};

// Kernel view of one simulation (passed by value).
struct View {
  int nx, ny, nz, nxp;       // extents; nxp = padded row length (multiple of 32)
  long long np;              // elements per population plane = nxp*ny*nz
  int xshift;                // sheared x-periodicity
  int bc;                    // boundary rule
  double omega, rho0, qcut;  // 1/tau, reference density, ELIBB-FQ cutoff
  double F[3];               // body-force density
  int has_force, has_uw;
  const uint8_t *flags;      // [np]
  const uint32_t *cbase;     // [np/32] records before each 32-node chunk
  const Rec *rec;            // [nb]
  const uint32_t *rnode;     // [nb] padded node index of each record
  const void *lq;            // [nl] q of each wall link (math type)
  const void *luw, *luw1;    // [nl*3] wall velocity at t, t+1 (math type) or null
  const uint8_t *ltag;       // [nl] force tag of each wall link
};

// Relative element offsets of the 27 neighbours (dx, dy, dz in {-1,0,1}) of a node,
// with periodic wrap and the sheared x-wrap: oxy[a][b] covers x and y for
// dx = a-1, dy = b-1; oz[c] covers z for dz = c-1.
struct Nbr {
  int oxy[3][3];
  long long oz[3];

  __device__ __forceinline__ void init(const View &v, int x, int y, int z) {
    const int xs[3] = {x == 0 ? v.nx - 1 : x - 1, x, x == v.nx - 1 ? 0 : x + 1};
    // crossing x = 0 downwards lands on x = nx-1 of the row y + xshift; crossing
    // x = nx-1 upwards lands on x = 0 of the row y - xshift
    const int ysh[3] = {x == 0 ? v.xshift : 0, 0, x == v.nx - 1 ? -v.xshift : 0};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        int yy = y + (b - 1) + ysh[a];
        if (v.xshift != 0) {
          yy %= v.ny;
          if (yy < 0) yy += v.ny;
        } else {
          yy = yy < 0 ? yy + v.ny : (yy >= v.ny ? yy - v.ny : yy);
        }
        oxy[a][b] = (yy - y) * v.nxp + (xs[a] - x);
      }
    }
    const long long plane = (long long)v.nxp * v.ny;
    const int zm = z == 0 ? v.nz - 1 : z - 1, zp = z == v.nz - 1 ? 0 : z + 1;
    oz[0] = (long long)(zm - z) * plane;
    oz[1] = 0;
    oz[2] = (long long)(zp - z) * plane;
  }
  // offset of the node n + (dx, dy, dz)
  __device__ __forceinline__ long long at(int dx, int dy, int dz) const {
    return (long long)oxy[dx + 1][dy + 1] + oz[dz + 1];
  }
};

}  // namespace lbm
