// pic_particles_o5.cu -- the per-particle kernels with the alternating-order
// form factor l_a = 2 1/2 (Sec. 4.5; process_item<..., ORD = 5> in
// pic_particles.cuh), any tile geometry, both precisions and all three modes.
// Kept in their own translation unit so that they compile beside the
// l_a = 1 1/2 kernels.
#include "pic_particles.cuh"

namespace pic {

cudaError_t launch_particles_o5(int dims, int prec, int mode, cudaStream_t st, int max_items, size_t smem,
                                const WorkItem *items, const int *n_items, const RunDev *runs, const GroupDev *groups,
                                const PoolBuf &P, void *const E[3], void *const B[3], void *const J[3],
                                int *old_cell, void *const old_off[3], int halo, int *err)
{
    return launch_particles_ord_t<5>(dims, prec, mode, st, max_items, smem, items, n_items, runs, groups, P, E, B, J,
                                      old_cell, old_off, halo, err);
}

cudaError_t particles_o5_set_smem_limit(int dims, int prec, int mode, size_t bytes)
{
    return particles_ord_set_smem_limit_t<5>(dims, prec, mode, bytes);
}

}  // namespace pic
