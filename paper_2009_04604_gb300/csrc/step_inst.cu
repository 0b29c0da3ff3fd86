// step_inst.cu -- explicit instantiation of the fused step for one lattice and
// storage type. The build compiles this file once per pair, with
// -DLBM_STEP_LATTICE=<D2Q9|D3Q19|D3Q27> -DLBM_STEP_STORE=<double|float|__half|__nv_bfloat16>;
// without them it defines nothing.
#include "step.cuh"

#if defined(LBM_STEP_LATTICE) && defined(LBM_STEP_STORE)
namespace lbm {
template cudaError_t launch_step_ls<LBM_STEP_LATTICE, LBM_STEP_STORE>(int, const View &, const void *, void *,
                                                                     const Launch &, const Launch *);
template cudaError_t prepare_step_tma_ls<LBM_STEP_LATTICE, LBM_STEP_STORE>(int, int, int, long long, int *,
                                                                          int *);
}  // namespace lbm
#endif
