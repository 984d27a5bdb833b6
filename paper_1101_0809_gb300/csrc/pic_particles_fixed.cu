// pic_particles_fixed.cu -- the FP32 fused particle kernel and the persistent
// batch step compiled for fixed tile geometries (GeoFix in pic_particles.cuh):
// the 3D 8x4x4 tile and the 2D 16x16 and 8x8 tiles, each with halo 1, and the
// 3D 4x4x4 tile with halo 2 (the laser slab at a long sort interval), with the
// pitches the grid's layout choice gives them.  With the geometry known at
// compile time every shared-memory offset of the gather and the deposit is an
// immediate of the load or atomic instruction.  Any other geometry runs the
// GeoDyn kernels of pic_particles.cu; the arithmetic is the same.
#include "pic_particles.cuh"

namespace pic {

using Geo3_844 = GeoFix<8, 4, 4, 1, 14, 12>;
using Geo3_444h2 = GeoFix<4, 4, 4, 2, 12, 12>;
using Geo2_16 = GeoFix<16, 16, 1, 1, 22, 22>;
using Geo2_8 = GeoFix<8, 8, 1, 1, 20, 14>;

template <class GEO>
static bool matches(int dims, const int tile[3], int halo, int p0, int p1)
{
    return tile[0] == GEO::T0 && tile[1] == GEO::T1 && (dims == 2 ? 1 : tile[2]) == GEO::T2 && halo == GEO::G &&
           p0 == GEO::P0 && p1 == GEO::P1;
}

bool launch_particles_fixed(int dims, cudaStream_t st, int max_items, size_t smem, const PartArgs<float> &a,
                            const int tile[3], int halo, int p0, int p1, cudaError_t *err)
{
    if (dims == 3 && matches<Geo3_844>(3, tile, halo, p0, p1)) {
        *err = launch_t<3, float, 0, Geo3_844>(st, max_items, smem, a);
        return true;
    }
    if (dims == 3 && matches<Geo3_444h2>(3, tile, halo, p0, p1)) {
        *err = launch_t<3, float, 0, Geo3_444h2>(st, max_items, smem, a);
        return true;
    }
    if (dims == 2 && matches<Geo2_16>(2, tile, halo, p0, p1)) {
        *err = launch_t<2, float, 0, Geo2_16>(st, max_items, smem, a);
        return true;
    }
    if (dims == 2 && matches<Geo2_8>(2, tile, halo, p0, p1)) {
        *err = launch_t<2, float, 0, Geo2_8>(st, max_items, smem, a);
        return true;
    }
    return false;
}

bool launch_persistent_fixed(int dims, cudaStream_t st, size_t smem, int nruns, const long long *run_cell_base,
                             const PartArgs<float> &a, int *grid_blocks, int launch, const int tile[3], int halo,
                             int p0, int p1, long long *ant_n, int antennas, cudaError_t *err)
{
    if (dims == 2 && matches<Geo2_16>(2, tile, halo, p0, p1)) {
        *err = persistent_t<2, float, Geo2_16>(st, smem, nruns, run_cell_base, a, grid_blocks, launch, ant_n,
                                                antennas);
        return true;
    }
    if (dims == 2 && matches<Geo2_8>(2, tile, halo, p0, p1)) {
        *err = persistent_t<2, float, Geo2_8>(st, smem, nruns, run_cell_base, a, grid_blocks, launch, ant_n,
                                               antennas);
        return true;
    }
    return false;
}

cudaError_t fixed_set_smem_limit(int dims, size_t bytes)
{
    const int b = (int)bytes;
    if (dims == 3) {
        const cudaError_t e3 = set_limit_fused<3, float, Geo3_844>(b);
        if (e3 != cudaSuccess) return e3;
        return set_limit_fused<3, float, Geo3_444h2>(b);
    }
    cudaError_t e = set_limit_fused<2, float, Geo2_16>(b);
    if (e != cudaSuccess) return e;
    return set_limit_fused<2, float, Geo2_8>(b);
}

}  // namespace pic
