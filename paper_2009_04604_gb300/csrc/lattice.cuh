// lattice.cuh -- velocity sets, storage conversions and the shared kernel view
// of a simulation (device side of liblbm).
//
// Directions are ordered lexicographically by (c_z, c_y, c_x). With that order the
// opposite of direction i is Q-1-i and the rest population sits in the middle.
// Weights are the standard Gauss-Hermite weights of the D2Q9 / D3Q19 / D3Q27 sets
// (Sec. II.A, c_s^2 = 1/3): 4/9, 1/9, 1/36; 1/3, 1/18, 1/36; 8/27, 2/27, 1/54, 1/216.
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

// all 27 velocities with components in {-1, 0, 1} (the lattice of the paper's 3-D
// cylindrical Couette runs): i = 9 (c_z + 1) + 3 (c_y + 1) + (c_x + 1)
struct D3Q27 {
  static constexpr int Q = 27;
  static constexpr int D = 3;
  __host__ __device__ static constexpr int cx(int i) { return i % 3 - 1; }
  __host__ __device__ static constexpr int cy(int i) { return (i / 3) % 3 - 1; }
  __host__ __device__ static constexpr int cz(int i) { return i / 9 - 1; }
};

template <class L>
__host__ __device__ constexpr int c2(int i) {
  return L::cx(i) * L::cx(i) + L::cy(i) * L::cy(i) + L::cz(i) * L::cz(i);
}

// Gauss-Hermite weight of direction i, from |c_i|^2.
template <class L>
__host__ __device__ constexpr double weight(int i) {
  return L::Q == 9    ? (c2<L>(i) == 0 ? 4.0 / 9.0 : (c2<L>(i) == 1 ? 1.0 / 9.0 : 1.0 / 36.0))
         : L::Q == 19 ? (c2<L>(i) == 0 ? 1.0 / 3.0 : (c2<L>(i) == 1 ? 1.0 / 18.0 : 1.0 / 36.0))
                      : (c2<L>(i) == 0 ? 8.0 / 27.0
                                       : (c2<L>(i) == 1 ? 2.0 / 27.0 : (c2<L>(i) == 2 ? 1.0 / 54.0 : 1.0 / 216.0)));
}

template <class L>
__host__ __device__ constexpr int opp(int i) { return L::Q - 1 - i; }

// Threads per block whose boundary work the step kernels stage in static shared
// memory: 256, or 128 where Q x 256 values of the math type would pass the 48 KB
// static limit (FP64 on D3Q27). Launches are limited to that many threads.
template <class L, typename M>
__host__ __device__ constexpr int stage_threads() {
  return L::Q * 256 * (int)sizeof(M) <= 48 * 1024 ? 256 : 128;
}

// Run-time direction index: the velocity components packed as 2-bit fields
// (component + 1) in 64-bit constants, and the weight in the math type. These
// keep a rolled loop over links free of lookup chains and of FP64 arithmetic.
template <class L>
__host__ __device__ constexpr unsigned long long pack_c(int comp) {
  unsigned long long p = 0;
  for (int i = 0; i < L::Q; ++i) {
    const int c = comp == 0 ? L::cx(i) : (comp == 1 ? L::cy(i) : L::cz(i));
    p |= (unsigned long long)(c + 1) << (2 * i);
  }
  return p;
}
template <class L>
__device__ __forceinline__ int dcx(int i) { return (int)((pack_c<L>(0) >> (2 * i)) & 3ull) - 1; }
template <class L>
__device__ __forceinline__ int dcy(int i) { return (int)((pack_c<L>(1) >> (2 * i)) & 3ull) - 1; }
template <class L>
__device__ __forceinline__ int dcz(int i) { return (int)((pack_c<L>(2) >> (2 * i)) & 3ull) - 1; }
template <class L, typename M>
__device__ __forceinline__ M dweight(int i) {
  const int a = dcx<L>(i), b = dcy<L>(i), c = dcz<L>(i);
  const int k = a * a + b * b + c * c;
  constexpr M w0 = M(weight<L>(L::Q / 2));  // rest
  constexpr M w1 = M(L::Q == 9 ? 1.0 / 9.0 : (L::Q == 19 ? 1.0 / 18.0 : 2.0 / 27.0));
  constexpr M w2 = M(L::Q == 27 ? 1.0 / 54.0 : 1.0 / 36.0);
  if constexpr (L::Q == 27) {  // corners only on D3Q27
    constexpr M w3 = M(1.0 / 216.0);
    return k == 0 ? w0 : (k == 1 ? w1 : (k == 2 ? w2 : w3));
  } else {
    return k == 0 ? w0 : (k == 1 ? w1 : w2);
  }
}

// ---- storage <-> math conversions (round to nearest even on store) ----
// FP16 storage holds the shifted value times 2^14. The factor is a power of two,
// so scaling is exact in FP32 and the rounding to FP16 is the same relative
// rounding as without it. What it changes is the range: FP16 turns subnormal
// below 6.1e-5, and the shifted populations of slow flows (f~ ~ w rho c.u) and a
// weak body force's increments (~ w 3 c.F, about 1.7e-7 at |F| = 1e-6) lie far
// below that, where subnormal spacing (6e-8) would swallow them. Scaled, values
// down to 3.7e-9 stay normal, and |f~| up to 3.99 still fits. BF16 has the FP32
// exponent range and needs no scaling.
constexpr float kF16Scale = 16384.0f;
constexpr float kF16Unscale = 1.0f / 16384.0f;
template <typename S, typename M> __device__ __forceinline__ M to_math(S v);
template <> __device__ __forceinline__ double to_math<double, double>(double v) { return v; }
template <> __device__ __forceinline__ float to_math<float, float>(float v) { return v; }
template <> __device__ __forceinline__ float to_math<__half, float>(__half v) {
  return __half2float(v) * kF16Unscale;
}
template <> __device__ __forceinline__ float to_math<__nv_bfloat16, float>(__nv_bfloat16 v) {
  return __bfloat162float(v);
}

template <typename S, typename M> __device__ __forceinline__ S to_store(M v);
template <> __device__ __forceinline__ double to_store<double, double>(double v) { return v; }
template <> __device__ __forceinline__ float to_store<float, float>(float v) { return v; }
template <> __device__ __forceinline__ __half to_store<__half, float>(float v) {
  return __float2half_rn(v * kF16Scale);
}
template <> __device__ __forceinline__ __nv_bfloat16 to_store<__nv_bfloat16, float>(float v) {
  return __float2bfloat16_rn(v);
}

// Node flag byte: low two bits are the kind, bit 2 marks a fluid node with at
// least one wall or open link (a boundary node with a record), bit 3 a fluid node
// with a link across a thin shell (its boundary tile, not a lattice tile, relaxes
// and stores it).
// Bit 4 marks the nodes of a moving body's region: the lattice tiles never store
// into a non-fluid node's slots there (values are written ahead into them, and
// which ones changes every step).
enum : uint8_t { K_FLUID = 0, K_SOLID = 1, K_OPEN = 2, K_PAD = 3, F_BOUNDARY = 4, F_SHELL = 8, F_KEEP = 16 };
// Flag bits a lattice tile tests: it relaxes the node only when they are all zero.
constexpr uint8_t K_LATTICE_MASK = 3 | F_SHELL;
// Force tag of the links on the inner side of a thin shell: no force is counted there.
constexpr uint8_t TAG_INNER = 0xFF;

// Boundary record of one boundary node (records are sorted by node index).
constexpr uint32_t REC_MOVING = 1u << 31;  // in Rec::open: the node has moving wall links
struct Rec {
  uint32_t cut;   // bit i: link i is a wall link (node n - c_i is SOLID, or across a thin shell)
  uint32_t open;  // bit i: link i is an open link (node n - c_i is OPEN); bit 31: REC_MOVING
  uint32_t ffok;  // bit i: the second node along the link, n + c_i, is fluid and on this side (BFL)
  uint32_t link0; // index of the first wall link of this node in the link arrays
  uint32_t shell; // bit i: link i crosses a thin shell to the fluid node n - c_i (also in cut)
};

// One set of boundary records and their per-link data (math type).
struct RecSet {
  const Rec *rec;         // [count] records, sorted by node (static) or region index (moving body)
  const uint32_t *rnode;  // [count] padded node index of each record
  const void *lq;         // [links] q of each wall link
  const void *luw, *luw1; // [links*3] wall velocity at t, t+1, or null
  const uint8_t *ltag;    // [links] force tag of each wall link
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
  int trt;                   // 1: TRT collision, odd parts relax with omega_m
  int wall_neq;              // 0: non-equilibrium bounce-back, 1: regularized wall estimate
  double omega_m;            // TRT omega- (Eq. magic-parameter); equals omega under BGK
  // the same scalars in FP32, so that FP32 kernels convert nothing on the
  // (slow) FP64 pipe: omega, rho0, qcut, F, omega_m
  float omega_f, rho0_f, qcut_f, F_f[3], omega_m_f;
  // rho0 and F in the units of the stored values (times 2^14 for FP16 storage)
  float rho0_u, F_u[3];
  const uint8_t *flags;      // [np]
  // [np] for a non-fluid node, bit i: slot (i, n) receives a boundary value written
  // ahead by the fluid node n + c_i (the other planes take the lattice tile's store)
  const uint32_t *amask;
  const uint32_t *cbase;     // [np/32] records before each 32-node chunk
  const Rec *rec;            // [nb]
  const uint32_t *rnode;     // [nb] padded node index of each record
  long long nb;              // number of boundary records
  const int2 *tiles;         // step-kernel block table (see k_step)
  int gx;                    // lattice tiles per row of tiles (nxp / block x)
  uint32_t gx_m, gx_s;       // t / gx = (t gx_m) >> gx_s for 0 <= t < 2^31 (tile_coords)
  uint32_t nxp_m, nxp_s;     // n / nxp, the same way (node_coords)
  uint32_t pl_m, pl_s;       // n / (nxp ny), the same way
  // per-direction element offsets, computed on the host so that the kernels use
  // them as constant operands: soff[i] = i np (plane i), loff[i] = i np - (c_ix +
  // c_iy nxp + c_iz nxp ny) (the source of population i at an interior node)
  int soff[27], loff[27];
  int ntiles, tpb_tiles;     // table length; consecutive table entries per block
  const int2 *btiles;        // split step (variants 9, 10): the boundary entries, apart from v.tiles
  // moving body: records of the nodes of its region, rebuilt every step
  RecSet dyn;
  const int *dyn_count;      // device: number of records in dyn (null: no moving body)
  int *err;                  // device error word (bounded waits that ran out set bit 0)
  long long wait_limit;      // polls before a first wait of the TMA-staged step counts as hung
  unsigned long long *dbg;   // LBM_DEBUG builds: first out-of-range population index (kernels.cuh LD_POP)
  long long dbg_limit;       // LBM_DEBUG builds: population indices at or above it count as out of range

  __host__ __device__ RecSet stat() const { return RecSet{rec, rnode, lq, luw, luw1, ltag}; }
  const void *lq;            // [nl] q of each wall link (math type)
  const void *luw, *luw1;    // [nl*3] wall velocity at t, t+1 (math type) or null
  const uint8_t *ltag;       // [nl] force tag of each wall link
};

// Scalar parameters in the math type of a kernel. stored_units: rho0 and F in the
// units of the stored values (Units<S> below) instead of lattice units.
template <typename M> struct Par;
template <> struct Par<double> {
  double omega, rho0, qcut, F[3], omega_m;
  __device__ __forceinline__ explicit Par(const View &v, bool = false)
      : omega(v.omega), rho0(v.rho0), qcut(v.qcut), F{v.F[0], v.F[1], v.F[2]}, omega_m(v.omega_m) {}
};
template <> struct Par<float> {
  float omega, rho0, qcut, F[3], omega_m;
  __device__ __forceinline__ explicit Par(const View &v, bool stored_units = false)
      : omega(v.omega_f), rho0(stored_units ? v.rho0_u : v.rho0_f), qcut(v.qcut_f),
        F{stored_units ? v.F_u[0] : v.F_f[0], stored_units ? v.F_u[1] : v.F_f[1],
          stored_units ? v.F_u[2] : v.F_f[2]},
        omega_m(v.omega_m_f) {}
};

// The lattice tiles compute in the units of the stored values. For FP16 storage
// these are the shifted populations times 2^14. With rho0 and the body force
// scaled by the same power of two (Par with stored_units), every operation of
// the moments and the relaxation scales exactly: the results are the lattice-unit
// computation's times 2^14, bit for bit (FP32 neither overflows nor turns
// subnormal at these magnitudes), and no population is multiplied on load or
// store. The boundary tiles work in lattice units through to_math / to_store.
template <typename S> struct Units {
  static constexpr bool kStored = false;
  template <typename M> __device__ static __forceinline__ M load(S v) { return to_math<S, M>(v); }
  template <typename M> __device__ static __forceinline__ S store(M v) { return to_store<S, M>(v); }
};
template <> struct Units<__half> {
  static constexpr bool kStored = true;
  template <typename M> __device__ static __forceinline__ M load(__half v) { return __half2float(v); }
  template <typename M> __device__ static __forceinline__ __half store(M v) { return __float2half_rn(v); }
};

// Relative element offsets of the 27 neighbours (dx, dy, dz in {-1,0,1}) of a node,
// with periodic wrap and the sheared x-wrap: oxy[a][b] covers x and y for
// dx = a-1, dy = b-1; oz[c] covers z for dz = c-1.
struct Nbr {
  int oxy[3][3];
  int oz[3];  // 32-bit: a simulation keeps Q x padded nodes below 2^31

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
    const int plane = v.nxp * v.ny;
    const int zm = z == 0 ? v.nz - 1 : z - 1, zp = z == v.nz - 1 ? 0 : z + 1;
    oz[0] = (zm - z) * plane;
    oz[1] = 0;
    oz[2] = (zp - z) * plane;
  }
  // offset of the node n + (dx, dy, dz)
  __device__ __forceinline__ int at(int dx, int dy, int dz) const {
    return oxy[dx + 1][dy + 1] + oz[dz + 1];
  }
};

}  // namespace lbm
