// kernels.cuh -- device code of the fused lattice Boltzmann step and its companions.
//
// Layout: populations are stored structure-of-arrays, plane i of buffer f holds
// f[i][z][y][x] with rows padded to nxp (a multiple of 32). Values are shifted,
// f~_i = f_i - w_i rho0, so the reduced-precision formats spend their bits on
// the deviation from rest.
//
// Pull scheme with two buffers (A-B): the thread of node x reads f_i(x,t) from
// slot fin[i][x - c_i] (Eq. LBE: exact on-grid streaming), relaxes with BGK
// (Eq. LB-BGK, equilibrium Eq. Eq2ndOrder, Guo forcing), and writes f*_i(x,t) to
// fout[i][x].
//
// Single-node boundary rule, written ahead. Let link i of a boundary node x_F be
// cut, so x_F - c_i is not fluid. The thread of x_F evaluates the unknown incoming
// population f_i(x_F, t+1) from its own registers alone (Sec. II.C-II.E: f*_ibar(x_F),
// f*_i(x_F), rho_F, u_F, f^neq_ibar(x_F) and the wall data q, u_w). It stores the
// value in slot fout[i][x_F - c_i], the slot its own gather reads at t+1. The
// non-fluid node x_F - c_i never writes, and only x_F reads that slot, so there is
// no race and no second pass. This is the locality the paper argues for in its
// conclusions.
//
// BFL needs f*_ibar(x_FF, t) at x_FF = x_F + c_i, which another thread produces
// in the same step. The thread therefore writes ahead the part it knows,
// 2q g + (1-2q) ME. At t+1 the gather adds (1-2q) f*_ibar(x_FF, t), a value it
// has just loaded as its own population ibar. So BFL costs no extra load.
#pragma once

#include "lattice.cuh"

namespace lbm {

enum { BC_ELIBB_F = 0, BC_ELIBB_FQ = 1, BC_BFL = 2, BC_HWBB = 3 };

// ---------------------------------------------------------------- gather
template <class L, typename S, typename M>
__device__ __forceinline__ void gather(const View &v, const S *__restrict__ fin, long long n,
                                       const Nbr &nb, M (&f)[L::Q]) {
#pragma unroll
  for (int i = 0; i < L::Q; ++i)
    f[i] = to_math<S, M>(__ldg(fin + (long long)i * v.np + n + nb.at(-L::cx(i), -L::cy(i), -L::cz(i))));
}

// BFL, q < 1/2: complete the written-ahead part with (1-2q) f*_ibar(x_FF, t),
// which the gather of direction ibar has just read from x_F - c_ibar = x_FF.
template <class L, typename M>
__device__ __forceinline__ void bfl_complete(const View &v, const Rec &r, M (&f)[L::Q]) {
  const M *lq = static_cast<const M *>(v.lq);
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    const uint32_t bit = 1u << i;
    if (r.cut & r.ffok & bit) {
      const M q = lq[r.link0 + __popc(r.cut & (bit - 1u))];
      if (q < M(0.5)) f[i] += (M(1) - M(2) * q) * f[opp<L>(i)];
    }
  }
}

// Record of a boundary node. bal is the warp ballot of the boundary flag, taken by
// a warp that covers 32 consecutive nodes of one row (one 32-node chunk).
__device__ __forceinline__ const Rec *record_of(const View &v, long long n, uint32_t bal) {
  const uint32_t lt = (1u << (threadIdx.x & 31)) - 1u;
  return v.rec + v.cbase[n >> 5] + __popc(bal & lt);
}

// ---------------------------------------------------------------- moments, equilibrium
template <class L, typename M>
struct Macro {
  M drho, rho, ux, uy, uz, usq;
};

template <class L, typename M>
__device__ __forceinline__ Macro<L, M> moments(const View &v, const M (&f)[L::Q]) {
  M d = M(0), jx = M(0), jy = M(0), jz = M(0);
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    d += f[i];
    if (L::cx(i) > 0) jx += f[i]; else if (L::cx(i) < 0) jx -= f[i];
    if (L::cy(i) > 0) jy += f[i]; else if (L::cy(i) < 0) jy -= f[i];
    if (L::cz(i) > 0) jz += f[i]; else if (L::cz(i) < 0) jz -= f[i];
  }
  Macro<L, M> m;
  m.drho = d;
  m.rho = M(v.rho0) + d;
  const M inv = M(1) / m.rho;
  if (v.has_force) {  // Guo: u = (sum c f + F/2) / rho
    jx += M(0.5 * v.F[0]);
    jy += M(0.5 * v.F[1]);
    jz += M(0.5 * v.F[2]);
  }
  m.ux = jx * inv;
  m.uy = jy * inv;
  m.uz = jz * inv;
  m.usq = m.ux * m.ux + m.uy * m.uy + m.uz * m.uz;
  return m;
}

// shifted equilibrium f^eq_i(rho, u) - w_i rho0 = w_i [drho + rho (3 cu + 9/2 cu^2 - 3/2 u^2)]
template <class L, typename M>
__device__ __forceinline__ M feq_s(int i, M drho, M rho, M ux, M uy, M uz, M usq) {
  const M cu = M(L::cx(i)) * ux + M(L::cy(i)) * uy + M(L::cz(i)) * uz;
  return M(weight<L>(i)) * (drho + rho * (M(3) * cu + M(4.5) * cu * cu - M(1.5) * usq));
}

// Guo source (1 - omega/2) w_i [3 (c_i - u).F + 9 (c_i.u)(c_i.F)]
template <class L, typename M>
__device__ __forceinline__ M guo(const View &v, int i, const Macro<L, M> &m) {
  const M Fx = M(v.F[0]), Fy = M(v.F[1]), Fz = M(v.F[2]);
  const M cu = M(L::cx(i)) * m.ux + M(L::cy(i)) * m.uy + M(L::cz(i)) * m.uz;
  const M cF = M(L::cx(i)) * Fx + M(L::cy(i)) * Fy + M(L::cz(i)) * Fz;
  const M uF = m.ux * Fx + m.uy * Fy + m.uz * Fz;
  return (M(1) - M(0.5 * v.omega)) * M(weight<L>(i)) * (M(3) * (cF - uF) + M(9) * cu * cF);
}

// post-collision shifted population f*_i = f_i + omega (f^eq_i - f_i) + S_i
template <class L, typename M>
__device__ __forceinline__ M post(const View &v, int i, const M fi, const Macro<L, M> &m) {
  M r = fi + M(v.omega) * (feq_s<L, M>(i, m.drho, m.rho, m.ux, m.uy, m.uz, m.usq) - fi);
  if (v.has_force) r += guo<L, M>(v, i, m);
  return r;
}

// ---------------------------------------------------------------- boundary rule
// Unknown incoming population f_i(x_F, t+1) (shifted) of every wall or open link.
// Points on the link, by the s coordinate of Eq. x_to_s_helper:
//   f0 = f~_i^{t+1}(x_W) = f^eq_i(rho_F, u_w(t+1)) + f^neq_ibar(x_F)            s = 0
//   g  = f*_ibar(x_F) + ME, ME = 2 w_i rho_F c_i.u_w / c_s^2 (Eq. ME-solid-to-fluid)  s = 1-q
//   f1 = f~*_i(x_W) = f^eq_i(rho_F, u_w(t)) + (1 - omega) f^neq_ibar(x_F)          s = 1
//   h  = f*_i(x_F)                                                                 s = 1+q
// Weights: Lagrange weights (Eq. poli_coeff) at s_ref = q, in closed form.
template <class L, typename S, typename M>
__device__ __forceinline__ void boundary(const View &v, const Rec &r, const M (&f)[L::Q],
                                         const Macro<L, M> &m, long long n, const Nbr &nb,
                                         S *__restrict__ fout) {
  const M *lq = static_cast<const M *>(v.lq);
  const M *luw = static_cast<const M *>(v.luw);
  const M *luw1 = static_cast<const M *>(v.luw1);
  const M om = M(v.omega);
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    const uint32_t bit = 1u << i;
    if (!((r.cut | r.open) & bit)) continue;
    const int ib = opp<L>(i);
    const M fneq_ib = f[ib] - feq_s<L, M>(ib, m.drho, m.rho, m.ux, m.uy, m.uz, m.usq);
    M val;
    if (r.open & bit) {
      // single-node pressure outlet: f^eq_i(rho0, u_F) + f^neq_ibar(x_F)
      val = feq_s<L, M>(i, M(0), M(v.rho0), m.ux, m.uy, m.uz, m.usq) + fneq_ib;
    } else {
      const uint32_t li = r.link0 + __popc(r.cut & (bit - 1u));
      const M q = lq[li];
      M wx = M(0), wy = M(0), wz = M(0), vx = M(0), vy = M(0), vz = M(0);
      if (v.has_uw) {
        wx = luw[3 * li]; wy = luw[3 * li + 1]; wz = luw[3 * li + 2];
        vx = luw1[3 * li]; vy = luw1[3 * li + 1]; vz = luw1[3 * li + 2];
      }
      const M cu0 = M(L::cx(i)) * wx + M(L::cy(i)) * wy + M(L::cz(i)) * wz;
      const M me = M(6.0 * weight<L>(i)) * m.rho * cu0;
      const M g = post<L, M>(v, ib, f[ib], m) + me;
      if (v.bc == BC_HWBB) {
        val = g;
      } else if (v.bc == BC_BFL) {
        if (q < M(0.5)) {
          val = (r.ffok & bit) ? M(2) * q * g + (M(1) - M(2) * q) * me : g;
        } else {
          const M h = post<L, M>(v, i, f[i], m);
          val = (g + (M(2) * q - M(1)) * h) / (M(2) * q);
        }
      } else {
        const M u0sq = wx * wx + wy * wy + wz * wz;
        const M u1sq = vx * vx + vy * vy + vz * vz;
        const M f1 = feq_s<L, M>(i, m.drho, m.rho, wx, wy, wz, u0sq) + (M(1) - om) * fneq_ib;
        if (q < M(0.5)) {
          const M f0 = feq_s<L, M>(i, m.drho, m.rho, vx, vy, vz, u1sq) + fneq_ib;
          if (v.bc == BC_ELIBB_FQ && q >= M(v.qcut))
            val = (M(1) - M(2) * q) * f0 + g + (M(2) * q - M(1)) * f1;
          else
            val = ((M(1) - M(2) * q) * f0 + q * g) / (M(1) - q);
        } else {
          if (v.bc == BC_ELIBB_FQ) {
            const M h = post<L, M>(v, i, f[i], m);
            const M a = M(2) * q - M(1);
            val = ((M(1) - q) * g + M(2) * a * f1 + a * (q - M(1)) * h) / (M(2) * q * q);
          } else {
            val = ((M(1) - q) * g + (M(2) * q - M(1)) * f1) / q;
          }
        }
      }
    }
    fout[(long long)i * v.np + n + nb.at(-L::cx(i), -L::cy(i), -L::cz(i))] = to_store<S, M>(val);
  }
}

// ---------------------------------------------------------------- the fused step
// One thread per node. blockDim.x is a multiple of 32 and divides nxp, so every
// warp covers one aligned 32-node chunk of one row.
template <class L, typename S, typename M>
__global__ void __launch_bounds__(256) k_step(const View v, const S *__restrict__ fin,
                                              S *__restrict__ fout) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (y >= v.ny) return;  // uniform across the warp
  const long long n = ((long long)z * v.ny + y) * v.nxp + x;
  const uint8_t fl = v.flags[n];
  const uint32_t bal = __ballot_sync(0xffffffffu, fl & F_BOUNDARY);
  if ((fl & 3) != K_FLUID) return;
  Nbr nb;
  nb.init(v, x, y, z);
  M f[L::Q];
  gather<L, S, M>(v, fin, n, nb, f);
  const bool isb = fl & F_BOUNDARY;
  Rec r = {0u, 0u, 0u, 0u};
  if (isb) {
    r = *record_of(v, n, bal);
    if (v.bc == BC_BFL) bfl_complete<L, M>(v, r, f);
  }
  const Macro<L, M> m = moments<L, M>(v, f);
#pragma unroll
  for (int i = 0; i < L::Q; ++i)
    fout[(long long)i * v.np + n] = to_store<S, M>(post<L, M>(v, i, f[i], m));
  if (isb) boundary<L, S, M>(v, r, f, m, n, nb, fout);
}

// ---------------------------------------------------------------- state set-up and read-out
// f_i(x) = f^eq_i(rho, u) on every fluid node, written to the slot its gather reads.
template <class L, typename S, typename M>
__global__ void k_init(const View v, S *__restrict__ fout, double rho, double ux, double uy,
                       double uz) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (y >= v.ny) return;
  const long long n = ((long long)z * v.ny + y) * v.nxp + x;
  if ((v.flags[n] & 3) != K_FLUID) return;
  Nbr nb;
  nb.init(v, x, y, z);
  const M usq = M(ux * ux + uy * uy + uz * uz);
#pragma unroll
  for (int i = 0; i < L::Q; ++i)
    fout[(long long)i * v.np + n + nb.at(-L::cx(i), -L::cy(i), -L::cz(i))] = to_store<S, M>(
        feq_s<L, M>(i, M(rho - v.rho0), M(rho), M(ux), M(uy), M(uz), usq));
}

// Host-layout FP64 populations fh[(x + nx*(y + ny*z))*Q + i] -> slots (unshifted in, shifted stored).
template <class L, typename S, typename M>
__global__ void k_set_pop(const View v, S *__restrict__ fout, const double *__restrict__ fh) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (y >= v.ny || x >= v.nx) return;
  const long long n = ((long long)z * v.ny + y) * v.nxp + x;
  if ((v.flags[n] & 3) != K_FLUID) return;
  const long long hn = ((long long)z * v.ny + y) * v.nx + x;
  Nbr nb;
  nb.init(v, x, y, z);
#pragma unroll
  for (int i = 0; i < L::Q; ++i)
    fout[(long long)i * v.np + n + nb.at(-L::cx(i), -L::cy(i), -L::cz(i))] =
        to_store<S, M>(M(fh[hn * L::Q + i] - weight<L>(i) * v.rho0));
}

// Pre-collision populations (gathered, BFL-completed), macroscopic fields, and the
// per-block FP64 partial of the mass. Any output pointer may be null.
template <class L, typename S, typename M>
__global__ void __launch_bounds__(256) k_read(const View v, const S *__restrict__ fin,
                                              double *__restrict__ fh, double *__restrict__ rho_out,
                                              double *__restrict__ u_out, double *__restrict__ mass_part) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  double mloc = 0.0;
  if (y < v.ny) {
    const long long n = ((long long)z * v.ny + y) * v.nxp + x;
    const uint8_t fl = v.flags[n];
    const uint32_t bal = __ballot_sync(0xffffffffu, fl & F_BOUNDARY);
    const long long hn = ((long long)z * v.ny + y) * v.nx + x;
    if ((fl & 3) == K_FLUID) {
      Nbr nb;
      nb.init(v, x, y, z);
      M f[L::Q];
      gather<L, S, M>(v, fin, n, nb, f);
      if ((fl & F_BOUNDARY) && v.bc == BC_BFL) bfl_complete<L, M>(v, *record_of(v, n, bal), f);
      double d = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
#pragma unroll
      for (int i = 0; i < L::Q; ++i) {
        const double fi = (double)f[i];
        d += fi;
        jx += L::cx(i) * fi;
        jy += L::cy(i) * fi;
        jz += L::cz(i) * fi;
        if (fh) fh[hn * L::Q + i] = fi + weight<L>(i) * v.rho0;
      }
      const double r = v.rho0 + d;
      mloc = r;
      if (rho_out) rho_out[hn] = r;
      if (u_out) {
        const double hx = v.has_force ? 0.5 * v.F[0] : 0.0, hy = v.has_force ? 0.5 * v.F[1] : 0.0,
                     hz = v.has_force ? 0.5 * v.F[2] : 0.0;
        u_out[hn * 3 + 0] = (jx + hx) / r;
        u_out[hn * 3 + 1] = (jy + hy) / r;
        u_out[hn * 3 + 2] = (jz + hz) / r;
      }
    } else if (x < v.nx) {
      if (fh)
        for (int i = 0; i < L::Q; ++i) fh[hn * L::Q + i] = 0.0;
      if (rho_out) rho_out[hn] = 0.0;
      if (u_out) u_out[hn * 3] = u_out[hn * 3 + 1] = u_out[hn * 3 + 2] = 0.0;
    }
  }
  if (mass_part) {
    // fixed-order block sum: warp shuffles, then warp 0 over the warp sums
    __shared__ double sm[32];
    for (int o = 16; o > 0; o >>= 1) mloc += __shfl_down_sync(0xffffffffu, mloc, o);
    const int t = threadIdx.y * blockDim.x + threadIdx.x;
    const int nw = (blockDim.x * blockDim.y) >> 5;
    if ((t & 31) == 0) sm[t >> 5] = mloc;
    __syncthreads();
    if (t < 32) {
      double s = t < nw ? sm[t] : 0.0;
      for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
      if (t == 0)
        mass_part[((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = s;
    }
  }
}

// Momentum-exchange force (Sec. II.F, Eq. force-boundary-node) of the last step,
// one thread per boundary record, links of one tag (tag < 0: all). It reads the
// buffer just written: f*_ibar(x_F, t) from the node's own slot and
// f_i(x_F, t+1) from the written-ahead slot (BFL-completed). Writes a per-block
// FP64 partial (3 doubles).
template <class L, typename S, typename M>
__global__ void __launch_bounds__(256) k_force(const View v, const S *__restrict__ cur, long long nb_,
                                               int tag, double *__restrict__ part) {
  const long long rid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double fx = 0.0, fy = 0.0, fz = 0.0;
  if (rid < nb_) {
    const Rec r = v.rec[rid];
    const long long n = v.rnode[rid];
    const int x = (int)(n % v.nxp);
    const int y = (int)((n / v.nxp) % v.ny);
    const int z = (int)(n / ((long long)v.nxp * v.ny));
    Nbr nb;
    nb.init(v, x, y, z);
    const M *lq = static_cast<const M *>(v.lq);
    const M *luw = static_cast<const M *>(v.luw);
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
      const uint32_t bit = 1u << i;
      if (!(r.cut & bit)) continue;
      const uint32_t li = r.link0 + __popc(r.cut & (bit - 1u));
      if (tag >= 0 && v.ltag[li] != tag) continue;
      const int ib = opp<L>(i);
      const double w = weight<L>(i);
      const double fpost_ib = (double)to_math<S, M>(cur[(long long)ib * v.np + n]) + w * v.rho0;
      double fnew = (double)to_math<S, M>(cur[(long long)i * v.np + n + nb.at(-L::cx(i), -L::cy(i), -L::cz(i))]);
      if (v.bc == BC_BFL && (r.ffok & bit)) {
        const M q = lq[li];
        if (q < M(0.5))
          fnew += (double)((M(1) - M(2) * q) *
                           to_math<S, M>(cur[(long long)ib * v.np + n + nb.at(L::cx(i), L::cy(i), L::cz(i))]));
      }
      fnew += w * v.rho0;
      double wx = 0.0, wy = 0.0, wz = 0.0;
      if (v.has_uw) { wx = (double)luw[3 * li]; wy = (double)luw[3 * li + 1]; wz = (double)luw[3 * li + 2]; }
      fx += (-L::cx(i) - wx) * fpost_ib - (L::cx(i) - wx) * fnew;
      fy += (-L::cy(i) - wy) * fpost_ib - (L::cy(i) - wy) * fnew;
      fz += (-L::cz(i) - wz) * fpost_ib - (L::cz(i) - wz) * fnew;
    }
  }
  __shared__ double sm[3][8];
  for (int o = 16; o > 0; o >>= 1) {
    fx += __shfl_down_sync(0xffffffffu, fx, o);
    fy += __shfl_down_sync(0xffffffffu, fy, o);
    fz += __shfl_down_sync(0xffffffffu, fz, o);
  }
  const int t = threadIdx.x;
  if ((t & 31) == 0) { sm[0][t >> 5] = fx; sm[1][t >> 5] = fy; sm[2][t >> 5] = fz; }
  __syncthreads();
  if (t < 3) {
    double s = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += sm[t][k];
    part[(long long)blockIdx.x * 3 + t] = s;
  }
}

// Fixed-order sum of per-block partials: out[c] = sum_b part[b*ncomp + c]. One block.
__global__ void k_reduce_final(const double *__restrict__ part, long long nblocks, int ncomp,
                               double *__restrict__ out);

}  // namespace lbm
