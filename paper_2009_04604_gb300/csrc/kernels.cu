// kernels.cu -- instantiation and dispatch of the lattice Boltzmann kernels.
#include "step.cuh"

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
  } else if (lattice == 2) {
    switch (dtype) {
      case 0: return fn.template operator()<D3Q27, double, double>();
      case 1: return fn.template operator()<D3Q27, float, float>();
      case 2: return fn.template operator()<D3Q27, __half, float>();
      case 3: return fn.template operator()<D3Q27, __nv_bfloat16, float>();
    }
  }
  return cudaErrorInvalidValue;
}

LBM_STEP_INSTANCES(LBM_STEP_DECLARE)

cudaError_t prepare_step_tma(int lattice, int dtype, int phys, int bx, int by, long long ntiles,
                             int *blocks, int *smem) {
  return dispatch(lattice, dtype, [&]<class L, typename S, typename M>() {
    return prepare_step_tma_ls<L, S>(phys, bx, by, ntiles, blocks, smem);
  });
}

cudaError_t launch_step(int lattice, int dtype, int variant, const View &v, const void *fin,
                        void *fout, const Launch &l, const Launch *lb) {
  return dispatch(lattice, dtype, [&]<class L, typename S, typename M>() {
    return launch_step_ls<L, S>(variant, v, fin, fout, l, lb);
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

cudaError_t launch_force(int lattice, int dtype, const View &v, const void *cur, const void *prev,
                         const RecSet &rs, long long nrec, const int *nrec_dev, int tag, double *part,
                         const Launch &l, double *tpart, double cx, double cy, double cz) {
  return dispatch(lattice, dtype, [&]<class L, typename S, typename M>() {
    k_force<L, S, M><<<l.grid, l.block, 0, l.stream>>>(v, static_cast<const S *>(cur),
                                                       static_cast<const S *>(prev), rs, nrec,
                                                       nrec_dev, tag, part, tpart, cx, cy, cz);
    return cudaGetLastError();
  });
}

}  // namespace lbm
