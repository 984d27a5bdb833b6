// pic_particles_o5.cu -- the per-particle kernels with the alternating-order
// form factor l_a = 2 1/2 (Sec. 4.5; process_item<..., ORD = 5> in
// pic_particles.cuh), any tile geometry, both precisions and all three modes.
// Kept in their own translation unit so that they compile beside the
// l_a = 1 1/2 kernels.
#include "pic_particles.cuh"

namespace pic {

template <int DIM, typename R>
static cudaError_t launch_mode5(int mode, cudaStream_t st, int max_items, size_t smem, const PartArgs<R> &a)
{
    switch (mode) {
    case 0: return launch_t<DIM, R, 0, GeoDyn, 5>(st, max_items, smem, a);
    case 1: return launch_t<DIM, R, 1, GeoDyn, 5>(st, max_items, smem, a);
    default: return launch_t<DIM, R, 2, GeoDyn, 5>(st, max_items, smem, a);
    }
}

cudaError_t launch_particles_o5(int dims, int prec, int mode, cudaStream_t st, int max_items, size_t smem,
                                const WorkItem *items, const int *n_items, const RunDev *runs, const GroupDev *groups,
                                const PoolBuf &P, void *const E[3], void *const B[3], void *const J[3],
                                int *old_cell, void *const old_off[3], int halo, int *err)
{
    if (prec == 0) {
        auto a = make_args<double>(items, n_items, runs, groups, P, E, B, J, old_cell, old_off, halo, err);
        return dims == 3 ? launch_mode5<3, double>(mode, st, max_items, smem, a)
                         : launch_mode5<2, double>(mode, st, max_items, smem, a);
    }
    auto a = make_args<float>(items, n_items, runs, groups, P, E, B, J, old_cell, old_off, halo, err);
    return dims == 3 ? launch_mode5<3, float>(mode, st, max_items, smem, a)
                     : launch_mode5<2, float>(mode, st, max_items, smem, a);
}

template <int DIM, typename R>
static cudaError_t set_limit5(int mode, size_t bytes)
{
    const int b = (int)bytes;
    switch (mode) {
    case 0: return cudaFuncSetAttribute(k_particles<DIM, R, 0, GeoDyn, 5>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    case 1: return cudaFuncSetAttribute(k_particles<DIM, R, 1, GeoDyn, 5>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    default: return cudaFuncSetAttribute(k_particles<DIM, R, 2, GeoDyn, 5>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    }
}

cudaError_t particles_o5_set_smem_limit(int dims, int prec, int mode, size_t bytes)
{
    if (dims == 3) return prec == 0 ? set_limit5<3, double>(mode, bytes) : set_limit5<3, float>(mode, bytes);
    return prec == 0 ? set_limit5<2, double>(mode, bytes) : set_limit5<2, float>(mode, bytes);
}

}  // namespace pic
