// launch.hpp -- host-side entry points of the kernels (one per kernel family),
// dispatched on lattice and storage type.
#pragma once

#include <cuda_runtime.h>

#include "lattice.cuh"

namespace lbm {

struct Launch {
  dim3 grid, block;
  cudaStream_t stream;
  int smem = 0;  // dynamic shared memory (TMA-staged step)
};

// Sets the shared-memory limit of the TMA-staged step kernel for this launch shape
// and returns its persistent grid (SMs x resident blocks, at most ntiles) and its
// dynamic shared memory. Call outside stream capture.
// phys: PH_FORCE | PH_TRT bits of the view (see phys_of).
cudaError_t prepare_step_tma(int lattice, int dtype, int phys, int bx, int by, long long ntiles,
                             int *blocks, int *smem);

// lattice: 0 D2Q9, 1 D3Q19, 2 D3Q27; dtype: 0 F64, 1 F32, 2 F16, 3 BF16
// variant: register budget of the step kernel, at least variant+1 resident
// 256-thread blocks per SM (0..3), 4: the TMA-staged persistent kernel, 5..7:
// two nodes per thread with at least 1..3 resident blocks per SM, 8: two nodes
// per thread in 128-thread blocks, 9 and 10: the split step, whose lattice kernel
// keeps at least 6 or 5 resident 256-thread blocks per SM and whose boundary
// kernel runs with the launch lb, 11 and 12: the combined kernel with at least 5
// or 6 resident 256-thread blocks per SM (FP32/FP16/BF16). FP64 has a single
// variant.
cudaError_t launch_step(int lattice, int dtype, int variant, const View &v, const void *fin,
                        void *fout, const Launch &l, const Launch *lb = nullptr);
cudaError_t launch_init(int lattice, int dtype, const View &v, void *fout, double rho, double ux,
                        double uy, double uz, const Launch &l);
cudaError_t launch_set_pop(int lattice, int dtype, const View &v, void *fout, const double *fh,
                           const Launch &l);
cudaError_t launch_read(int lattice, int dtype, const View &v, const void *fin, double *fh,
                        double *rho, double *u, double *mass_part, const Launch &l);
// Momentum-exchange partials over the records rs: nrec of them, or *nrec_dev
// (device) when nrec_dev is not null; the grid must cover the largest count.
// cur is the state the last step wrote, prev the state it read (used for the
// links across thin shells; may be null when rs has none).
// With tpart, also the torque about (cx, cy, cz) of every link force, taken at the
// link's wall point x_F - q c_i (3 doubles per block).
cudaError_t launch_force(int lattice, int dtype, const View &v, const void *cur, const void *prev,
                         const RecSet &rs, long long nrec, const int *nrec_dev, int tag, double *part,
                         const Launch &l, double *tpart = nullptr, double cx = 0.0, double cy = 0.0,
                         double cz = 0.0);
// amask[n] of every padded node (View::amask) from the node kinds in v.flags
// (geometry.cu).
cudaError_t launch_amask(int lattice, const View &v, uint32_t *amask, cudaStream_t s);
cudaError_t launch_reduce_final(const double *part, long long nblocks, int ncomp, double *out,
                                cudaStream_t s);

}  // namespace lbm
