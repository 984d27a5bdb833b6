// pic_particles_o5.cu -- the per-particle kernels with the alternating-order
// form factor l_a = 2 1/2 (Sec. 4.5; process_item<..., ORD = 5> in
// pic_particles.cuh), any tile geometry, both precisions and all three modes,
// and the FP32 fused kernel for the fixed 4x4x4 tile.
// Kept in their own translation unit so that they compile beside the
// l_a = 1 1/2 kernels.
#include "pic_particles.cuh"

namespace pic {

// The FP32 fused kernel compiled for the 3D 4x4x4 tile with halo 1 (its pitches
// from the tile layout choice), the tile that suits l_a = 2 1/2 best: every
// shared-memory offset of its gather and deposit is an immediate.
using Geo5_444 = GeoFix<4, 4, 4, 1, 12, 12>;

cudaError_t launch_particles_o5(int dims, int prec, int mode, cudaStream_t st, int max_items, size_t smem,
                                const WorkItem *items, const int *n_items, const RunDev *runs, const GroupDev *groups,
                                const PoolBuf &P, void *const E[3], void *const B[3], void *const J[3],
                                int *old_cell, void *const old_off[3], int halo, int *err, const int tile[3], int p0,
                                int p1)
{
    if (dims == 3 && prec != 0 && mode == 0 && tile[0] == Geo5_444::T0 && tile[1] == Geo5_444::T1 &&
        tile[2] == Geo5_444::T2 && halo == Geo5_444::G && p0 == Geo5_444::P0 && p1 == Geo5_444::P1) {
        auto a = make_args<float>(items, n_items, runs, groups, P, E, B, J, old_cell, old_off, halo, err);
        return launch_t<3, float, 0, Geo5_444, 5>(st, max_items, smem, a);
    }
    return launch_particles_ord_t<5>(dims, prec, mode, st, max_items, smem, items, n_items, runs, groups, P, E, B, J,
                                      old_cell, old_off, halo, err);
}

cudaError_t particles_o5_set_smem_limit(int dims, int prec, int mode, size_t bytes)
{
    if (dims == 3 && prec != 0 && mode == 0) {
        const cudaError_t e = cudaFuncSetAttribute(k_particles<3, float, 0, Geo5_444, 5>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (e != cudaSuccess) return e;
    }
    return particles_ord_set_smem_limit_t<5>(dims, prec, mode, bytes);
}

}  // namespace pic
