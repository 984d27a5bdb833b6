// pic_particles_w1.cu -- the per-particle kernels of the comparison scheme of
// Eq. wrong1 (Sec. 5: the uniform-order l = 2 interpolation of the fields with
// the l_a = 1 1/2 charge and current; process_item<..., ORD = 4> in
// pic_particles.cuh), any tile geometry, both precisions and all three modes,
// in their own translation unit.
#include "pic_particles.cuh"

namespace pic {

cudaError_t launch_particles_w1(int dims, int prec, int mode, cudaStream_t st, int max_items, size_t smem,
                                const WorkItem *items, const int *n_items, const RunDev *runs, const GroupDev *groups,
                                const PoolBuf &P, void *const E[3], void *const B[3], void *const J[3],
                                int *old_cell, void *const old_off[3], int halo, int *err)
{
    return launch_particles_ord_t<4>(dims, prec, mode, st, max_items, smem, items, n_items, runs, groups, P, E, B, J,
                                      old_cell, old_off, halo, err);
}

cudaError_t particles_w1_set_smem_limit(int dims, int prec, int mode, size_t bytes)
{
    return particles_ord_set_smem_limit_t<4>(dims, prec, mode, bytes);
}

}  // namespace pic
