// step.cuh -- launch of the fused step kernel for one (lattice, storage type).
//
// The step kernel has many instantiations (register budget, node pairs, force
// path, the TMA-staged kernel). They are compiled in one translation unit per
// (lattice, storage type), step_inst.cu built once for each pair, so that the
// build runs them in parallel. kernels.cu dispatches to the explicit
// instantiations of launch_step_ls and prepare_step_tma_ls.
#pragma once

#include "kernels.cuh"
#include "launch.hpp"

namespace lbm {

// Compile-time physics (PH_FORCE, PH_TRT) of a view.
inline int phys_of(const View &v) { return (v.has_force ? PH_FORCE : 0) | (v.trt ? PH_TRT : 0); }

// The step grid is 1-D, one block per entry of the tile table (l.grid.x entries).
template <class L, typename S, typename M, int MINB, bool PAIR = false, int MAXT = 256>
cudaError_t step_variant(const View &v, const void *fin, void *fout, const Launch &l) {
  const S *a = static_cast<const S *>(fin);
  S *b = static_cast<S *>(fout);
  switch (phys_of(v)) {
    case PH_FORCE: k_step<L, S, M, MINB, PH_FORCE, PAIR, MAXT><<<l.grid, l.block, 0, l.stream>>>(v, a, b); break;
    case PH_TRT: k_step<L, S, M, MINB, PH_TRT, PAIR, MAXT><<<l.grid, l.block, 0, l.stream>>>(v, a, b); break;
    case PH_FORCE | PH_TRT:
      k_step<L, S, M, MINB, PH_FORCE | PH_TRT, PAIR, MAXT><<<l.grid, l.block, 0, l.stream>>>(v, a, b);
      break;
    default: k_step<L, S, M, MINB, 0, PAIR, MAXT><<<l.grid, l.block, 0, l.stream>>>(v, a, b); break;
  }
  return cudaGetLastError();
}

// The split step (variants 9, 10): the boundary kernel on lb.stream, then the
// lattice kernel on l.stream. The caller orders the two streams around the pair.
template <class L, typename S, typename M, int MINB>
cudaError_t split_variant(const View &v, const void *fin, void *fout, const Launch &l, const Launch *lb) {
  const S *a = static_cast<const S *>(fin);
  S *b = static_cast<S *>(fout);
  if (lb != nullptr && lb->grid.x > 0) {
    k_boundary<L, S, M><<<lb->grid, lb->block, 0, lb->stream>>>(v, a, b);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  switch (phys_of(v)) {
    case PH_FORCE: k_lattice<L, S, M, MINB, PH_FORCE><<<l.grid, l.block, 0, l.stream>>>(v, a, b); break;
    case PH_TRT: k_lattice<L, S, M, MINB, PH_TRT><<<l.grid, l.block, 0, l.stream>>>(v, a, b); break;
    case PH_FORCE | PH_TRT: k_lattice<L, S, M, MINB, PH_FORCE | PH_TRT><<<l.grid, l.block, 0, l.stream>>>(v, a, b); break;
    default: k_lattice<L, S, M, MINB, 0><<<l.grid, l.block, 0, l.stream>>>(v, a, b); break;
  }
  return cudaGetLastError();
}

// Shared-memory bytes of one stage of the TMA-staged step: the rows of every
// population plane with a 16-byte halo on each side, the flag rows, and at least
// the boundary tiles' staging array.
template <class L, typename S, typename M>
int tma_stage_bytes(int bx, int by) {
  const int halo = 16 / (int)sizeof(S);
  const int pops = L::Q * by * (bx + 2 * halo) * (int)sizeof(S);
  const int need = pops + bx * by;
  const int stagebnd = L::Q * 256 * (int)sizeof(M);
  const int b = need > stagebnd ? need : stagebnd;
  return (b + 127) / 128 * 128;
}

// Two persistent blocks per SM, each with as many stages as half of the shared
// memory allows (at most 16): the copies in flight, not registers, then set the
// memory-level parallelism.
inline int tma_stages(int stage_bytes, int optin) {
  int k = (optin / 2 - 128) / stage_bytes;
  return k > 16 ? 16 : k;
}

template <class L, typename S, typename M, int PHYS>
cudaError_t tma_prepare(int bx, int by, long long ntiles, int *blocks, int *smem) {
  const int sb = tma_stage_bytes<L, S, M>(bx, by);
  int dev0 = 0, optin = 0;
  cudaError_t e0 = cudaGetDevice(&dev0);
  if (e0 == cudaSuccess) e0 = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev0);
  if (e0 != cudaSuccess) return e0;
  const int stages = tma_stages(sb, optin);
  if (stages < 2) return cudaErrorInvalidConfiguration;
  *smem = 128 + stages * sb;
  auto kern = k_step_tma<L, S, M, PHYS>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, *smem);
  if (e != cudaSuccess) return e;
  int dev = 0, nsm = 0, per = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, bx * by, *smem);
  if (e != cudaSuccess) return e;
  if (per < 1) return cudaErrorInvalidConfiguration;
  long long b = (long long)nsm * per;
  if (b > ntiles) b = ntiles;
  *blocks = (int)(b < 1 ? 1 : b);
  return cudaSuccess;
}

template <class L, typename S, typename M, int PHYS>
cudaError_t tma_launch(const View &v, const void *fin, void *fout, const Launch &l) {
  const int sb = tma_stage_bytes<L, S, M>(l.block.x, l.block.y);
  const int stages = (l.smem - 128) / sb;
  k_step_tma<L, S, M, PHYS><<<l.grid, l.block, l.smem, l.stream>>>(
      v, static_cast<const S *>(fin), static_cast<S *>(fout), stages, sb);
  return cudaGetLastError();
}

// Storage type S of lattice L: M is the arithmetic type (FP64 for FP64 storage).
template <typename S> struct MathOf { using T = float; };
template <> struct MathOf<double> { using T = double; };

template <class L, typename S>
cudaError_t launch_step_ls(int variant, const View &v, const void *fin, void *fout, const Launch &l,
                           const Launch *lb) {
  using M = typename MathOf<S>::T;
  if constexpr (sizeof(M) == 8) {
    return step_variant<L, S, M, 1>(v, fin, fout, l);  // FP64: one register budget
  } else {
    if (variant == 9) return split_variant<L, S, M, 6>(v, fin, fout, l, lb);
    if (variant == 10) return split_variant<L, S, M, 5>(v, fin, fout, l, lb);
    if (variant == 11) return step_variant<L, S, M, 5>(v, fin, fout, l);
    if (variant == 12) return step_variant<L, S, M, 6>(v, fin, fout, l);
    if (variant == 4) {
      switch (phys_of(v)) {
        case PH_FORCE: return tma_launch<L, S, M, PH_FORCE>(v, fin, fout, l);
        case PH_TRT: return tma_launch<L, S, M, PH_TRT>(v, fin, fout, l);
        case PH_FORCE | PH_TRT: return tma_launch<L, S, M, PH_FORCE | PH_TRT>(v, fin, fout, l);
        default: return tma_launch<L, S, M, 0>(v, fin, fout, l);
      }
    }
    switch (variant) {
      case 1: return step_variant<L, S, M, 2>(v, fin, fout, l);
      case 2: return step_variant<L, S, M, 3>(v, fin, fout, l);
      case 3: return step_variant<L, S, M, 4>(v, fin, fout, l);
      case 5: return step_variant<L, S, M, 1, true>(v, fin, fout, l);
      case 6: return step_variant<L, S, M, 2, true>(v, fin, fout, l);
      case 7: return step_variant<L, S, M, 3, true>(v, fin, fout, l);
      case 8: return step_variant<L, S, M, 7, true, 128>(v, fin, fout, l);
      default: return step_variant<L, S, M, 1>(v, fin, fout, l);
    }
  }
}

template <class L, typename S>
cudaError_t prepare_step_tma_ls(int phys, int bx, int by, long long ntiles, int *blocks, int *smem) {
  using M = typename MathOf<S>::T;
  if constexpr (sizeof(M) == 8) {
    return cudaErrorInvalidValue;  // FP64 has no TMA-staged variant
  } else {
    switch (phys) {
      case PH_FORCE: return tma_prepare<L, S, M, PH_FORCE>(bx, by, ntiles, blocks, smem);
      case PH_TRT: return tma_prepare<L, S, M, PH_TRT>(bx, by, ntiles, blocks, smem);
      case PH_FORCE | PH_TRT: return tma_prepare<L, S, M, PH_FORCE | PH_TRT>(bx, by, ntiles, blocks, smem);
      default: return tma_prepare<L, S, M, 0>(bx, by, ntiles, blocks, smem);
    }
  }
}

#define LBM_STEP_INSTANCES(X) \
  X(D2Q9, double) X(D2Q9, float) X(D2Q9, __half) X(D2Q9, __nv_bfloat16) \
  X(D3Q19, double) X(D3Q19, float) X(D3Q19, __half) X(D3Q19, __nv_bfloat16) \
  X(D3Q27, double) X(D3Q27, float) X(D3Q27, __half) X(D3Q27, __nv_bfloat16)

#define LBM_STEP_DECLARE(Lat, Sto)                                                                  \
  extern template cudaError_t launch_step_ls<Lat, Sto>(int, const View &, const void *, void *,    \
                                                       const Launch &, const Launch *);           \
  extern template cudaError_t prepare_step_tma_ls<Lat, Sto>(int, int, int, long long, int *, int *);

}  // namespace lbm
