// kernels.cu -- instantiation and dispatch of the lattice Boltzmann kernels.
#include "kernels.cuh"
#include "launch.hpp"

namespace lbm {

__global__ void k_reduce_final(const double *__restrict__ part, long long nblocks, int ncomp,
                               double *__restrict__ out) {
  // thread t sums partials t, t + 1024, ... of each component in order, then a
  // fixed tree over the 1024 thread sums
  __shared__ double sm[1024];
  for (int c = 0; c < ncomp; ++c) {
    double s = 0.0;
    for (long long b = threadIdx.x; b < nblocks; b += blockDim.x) s += part[b * ncomp + c];
    sm[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if ((int)threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[c] = sm[0];
    __syncthreads();
  }
}

cudaError_t launch_reduce_final(const double *part, long long nblocks, int ncomp, double *out,
                                cudaStream_t s) {
  k_reduce_final<<<1, 1024, 0, s>>>(part, nblocks, ncomp, out);
  return cudaGetLastError();
}

// Calls F.template operator()<L, S, M>() for the (lattice, dtype) pair.
template <class Fn>
static cudaError_t dispatch(int lattice, int dtype, Fn &&fn) {
  if (lattice == 0) {
    switch (dtype) {
      case 0: return fn.template operator()<D2Q9, double, double>();
      case 1: return fn.template operator()<D2Q9, float, float>();
      case 2: return fn.template operator()<D2Q9, __half, float>();
      case 3: return fn.template operator()<D2Q9, __nv_bfloat16, float>();
    }
  } else if (lattice == 1) {
    switch (dtype) {
      case 0: return fn.template operator()<D3Q19, double, double>();
      case 1: return fn.template operator()<D3Q19, float, float>();
      case 2: return fn.template operator()<D3Q19, __half, float>();
      case 3: return fn.template operator()<D3Q19, __nv_bfloat16, float>();
    }
  }
  return cudaErrorInvalidValue;
}

// The step grid is 1-D, one block per entry of the tile table (l.grid.x entries).
template <class L, typename S, typename M, int MINB, bool PAIR = false>
static cudaError_t step_variant(const View &v, const void *fin, void *fout, const Launch &l) {
  if (v.has_force)
    k_step<L, S, M, MINB, true, PAIR><<<l.grid, l.block, 0, l.stream>>>(v, static_cast<const S *>(fin),
                                                                        static_cast<S *>(fout));
  else
    k_step<L, S, M, MINB, false, PAIR><<<l.grid, l.block, 0, l.stream>>>(v, static_cast<const S *>(fin),
                                                                         static_cast<S *>(fout));
  return cudaGetLastError();
}

// Shared-memory bytes of one stage of the TMA-staged step: the rows of every
// population plane with a 16-byte halo on each side, the flag rows, and at least
// the boundary tiles' staging array.
template <class L, typename S, typename M>
static int tma_stage_bytes(int bx, int by) {
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
static int tma_stages(int stage_bytes, int optin) {
  int k = (optin / 2 - 128) / stage_bytes;
  return k > 16 ? 16 : k;
}

template <class L, typename S, typename M, bool FORCE>
static cudaError_t tma_prepare(int bx, int by, long long ntiles, int *blocks, int *smem) {
  const int sb = tma_stage_bytes<L, S, M>(bx, by);
  int dev0 = 0, optin = 0;
  cudaError_t e0 = cudaGetDevice(&dev0);
  if (e0 == cudaSuccess) e0 = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev0);
  if (e0 != cudaSuccess) return e0;
  const int stages = tma_stages(sb, optin);
  if (stages < 2) return cudaErrorInvalidConfiguration;
  *smem = 128 + stages * sb;
  auto kern = k_step_tma<L, S, M, FORCE>;
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

cudaError_t prepare_step_tma(int lattice, int dtype, int has_force, int bx, int by, long long ntiles,
                             int *blocks, int *smem) {
  return dispatch(lattice, dtype, [&]<class L, typename S, typename M>() {
    if constexpr (sizeof(M) == 8) {
      return cudaErrorInvalidValue;  // FP64 has no TMA-staged variant
    } else {
      return has_force ? tma_prepare<L, S, M, true>(bx, by, ntiles, blocks, smem)
                       : tma_prepare<L, S, M, false>(bx, by, ntiles, blocks, smem);
    }
  });
}

template <class L, typename S, typename M, bool FORCE>
static cudaError_t tma_launch(const View &v, const void *fin, void *fout, const Launch &l) {
  const int sb = tma_stage_bytes<L, S, M>(l.block.x, l.block.y);
  const int stages = (l.smem - 128) / sb;
  k_step_tma<L, S, M, FORCE><<<l.grid, l.block, l.smem, l.stream>>>(
      v, static_cast<const S *>(fin), static_cast<S *>(fout), stages, sb);
  return cudaGetLastError();
}

cudaError_t launch_step(int lattice, int dtype, int variant, const View &v, const void *fin,
                        void *fout, const Launch &l) {
  return dispatch(lattice, dtype, [&]<class L, typename S, typename M>() {
    if constexpr (sizeof(M) == 8) {
      return step_variant<L, S, M, 1>(v, fin, fout, l);  // FP64: one register budget
    } else {
      if (variant == 4)
        return v.has_force ? tma_launch<L, S, M, true>(v, fin, fout, l) : tma_launch<L, S, M, false>(v, fin, fout, l);
      switch (variant) {
        case 1: return step_variant<L, S, M, 2>(v, fin, fout, l);
        case 2: return step_variant<L, S, M, 3>(v, fin, fout, l);
        case 3: return step_variant<L, S, M, 4>(v, fin, fout, l);
        case 5: return step_variant<L, S, M, 1, true>(v, fin, fout, l);
        case 6: return step_variant<L, S, M, 2, true>(v, fin, fout, l);
        case 7: return step_variant<L, S, M, 3, true>(v, fin, fout, l);
        default: return step_variant<L, S, M, 1>(v, fin, fout, l);
      }
    }
  });
}

cudaError_t launch_init(int lattice, int dtype, const View &v, void *fout, double rho, double ux,
                        double uy, double uz, const Launch &l) {
  return dispatch(lattice, dtype, [&]<class L, typename S, typename M>() {
    k_init<L, S, M><<<l.grid, l.block, 0, l.stream>>>(v, static_cast<S *>(fout), rho, ux, uy, uz);
    return cudaGetLastError();
  });
}

cudaError_t launch_set_pop(int lattice, int dtype, const View &v, void *fout, const double *fh,
                           const Launch &l) {
  return dispatch(lattice, dtype, [&]<class L, typename S, typename M>() {
    k_set_pop<L, S, M><<<l.grid, l.block, 0, l.stream>>>(v, static_cast<S *>(fout), fh);
    return cudaGetLastError();
  });
}

cudaError_t launch_read(int lattice, int dtype, const View &v, const void *fin, double *fh,
                        double *rho, double *u, double *mass_part, const Launch &l) {
  return dispatch(lattice, dtype, [&]<class L, typename S, typename M>() {
    k_read<L, S, M><<<l.grid, l.block, 0, l.stream>>>(v, static_cast<const S *>(fin), fh, rho, u,
                                                      mass_part);
    return cudaGetLastError();
  });
}

cudaError_t launch_force(int lattice, int dtype, const View &v, const void *cur, const RecSet &rs,
                         long long nrec, const int *nrec_dev, int tag, double *part, const Launch &l) {
  return dispatch(lattice, dtype, [&]<class L, typename S, typename M>() {
    k_force<L, S, M><<<l.grid, l.block, 0, l.stream>>>(v, static_cast<const S *>(cur), rs, nrec, nrec_dev,
                                                       tag, part);
    return cudaGetLastError();
  });
}

}  // namespace lbm
