// pic_particles.cu -- launchers of the per-particle kernels (pic_particles.cuh)
// with the tile geometry read at run time, the shared-memory sizing, and the
// particle loader and pool copy.
#include "pic_particles.cuh"

namespace pic {

template <int DIM, typename R>
static cudaError_t launch_mode(int mode, cudaStream_t st, int max_items, size_t smem, const PartArgs<R> &a)
{
    switch (mode) {
    case 0: return launch_t<DIM, R, 0>(st, max_items, smem, a);
    case 1: return launch_t<DIM, R, 1>(st, max_items, smem, a);
    default: return launch_t<DIM, R, 2>(st, max_items, smem, a);
    }
}

size_t particles_smem_bytes(int dims, int prec, int mode, int tx, int ty, int tz, int halo, int p0, int p1,
                            int order2)
{
    (void)tx;   // the x and y extents enter through the pitches (p0, p1 cover the widest tile)
    (void)ty;
    const size_t es = prec == 0 ? sizeof(double) : sizeof(float);
    // l_a = 2 1/2 reaches one cell further in both tiles; the gather of
    // Eq. wrong1 (order2 = 4) in the field tile only
    const int fext = order2 == 3 ? 0 : 1, jext = order2 == 5 ? 1 : 0;
    const long long fe = (long long)p0 * p1 * (dims == 3 ? tz + 2 * (halo + 1 + fext) : 1);
    const long long je = (long long)p0 * p1 * (dims == 3 ? tz + 2 * (halo + 2 + jext) : 1);
    size_t b = 0;
    if (mode != 2) b += 6 * fe * es;
    // current tile (+ per-cell counts in FP32), the warps' deposit queues and one count per warp
    if (mode != 1)
        b += (prec == 0 ? 24 : 28) * je + (size_t)(kThreads / 32) * (kQueueCap * (kQueueVals * es + sizeof(int)) + sizeof(int));
    return b;
}

template <int DIM, typename R>
static cudaError_t set_limit_t(int mode, size_t bytes)
{
    const int b = (int)bytes;
    switch (mode) {
    case 0: return set_limit_fused<DIM, R, GeoDyn>(b);
    case 1: return cudaFuncSetAttribute(k_particles<DIM, R, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    default: return cudaFuncSetAttribute(k_particles<DIM, R, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    }
}

cudaError_t particles_set_smem_limit(int dims, int prec, int mode, size_t bytes, int order2)
{
    if (order2 == 5) return particles_o5_set_smem_limit(dims, prec, mode, bytes);
    if (order2 == 4) return particles_w1_set_smem_limit(dims, prec, mode, bytes);
    if (prec != 0 && mode == 0) {
        const cudaError_t e = fixed_set_smem_limit(dims, bytes);
        if (e != cudaSuccess) return e;
    }
    if (dims == 3) return prec == 0 ? set_limit_t<3, double>(mode, bytes) : set_limit_t<3, float>(mode, bytes);
    return prec == 0 ? set_limit_t<2, double>(mode, bytes) : set_limit_t<2, float>(mode, bytes);
}


cudaError_t launch_particles(int dims, int prec, int mode, cudaStream_t st, const WorkItem *items,
                             const int *n_items, int max_items, const RunDev *runs, const GroupDev *groups,
                             const PoolBuf &P, void *const E[3], void *const B[3], void *const J[3],
                             int *old_cell, void *const old_off[3], int halo, int max_tile_x, int max_tile_y,
                             int max_tile_z, int *err, int p0, int p1, int order2, const PoolBuf *src,
                             const unsigned *perm)
{
    if (perm && (mode != 0 || order2 != 3)) return cudaErrorInvalidValue;   // read through perm: fused l_a = 1 1/2 only
    const size_t smem =
        particles_smem_bytes(dims, prec, mode, max_tile_x, max_tile_y, max_tile_z, halo, p0, p1, order2);
    if (order2 == 5) {
        const int tile[3] = {max_tile_x, max_tile_y, max_tile_z};
        return launch_particles_o5(dims, prec, mode, st, max_items, smem, items, n_items, runs, groups, P, E, B, J,
                                   old_cell, old_off, halo, err, tile, p0, p1);
    }
    if (order2 == 4)
        return launch_particles_w1(dims, prec, mode, st, max_items, smem, items, n_items, runs, groups, P, E, B, J,
                                   old_cell, old_off, halo, err);
    if (prec == 0) {
        auto a = make_args<double>(items, n_items, runs, groups, P, E, B, J, old_cell, old_off, halo, err, src, perm);
        return dims == 3 ? launch_mode<3, double>(mode, st, max_items, smem, a)
                         : launch_mode<2, double>(mode, st, max_items, smem, a);
    }
    auto a = make_args<float>(items, n_items, runs, groups, P, E, B, J, old_cell, old_off, halo, err, src, perm);
    if (mode == 0) {
        const int tile[3] = {max_tile_x, max_tile_y, max_tile_z};
        cudaError_t e = cudaSuccess;
        if (launch_particles_fixed(dims, st, max_items, smem, a, tile, halo, p0, p1, &e)) return e;
    }
    return dims == 3 ? launch_mode<3, float>(mode, st, max_items, smem, a)
                     : launch_mode<2, float>(mode, st, max_items, smem, a);
}

cudaError_t launch_step_persistent(int dims, int prec, cudaStream_t st, const WorkItem *items, const int *n_items,
                                   const RunDev *runs, const GroupDev *groups, const PoolBuf &P, void *const E[3],
                                   void *const B[3], void *const J[3], int halo, int tx, int ty, int tz, int *err,
                                   int nruns, const long long *run_cell_base, int *grid_blocks, int launch, int p0,
                                   int p1, long long *ant_n, int antennas, const PoolBuf *src, const unsigned *perm)
{
    void *none[3] = {nullptr, nullptr, nullptr};
    const size_t smem = particles_smem_bytes(dims, prec, 0, tx, ty, tz, halo, p0, p1);
    if (prec == 0) {
        auto a = make_args<double>(items, n_items, runs, groups, P, E, B, J, nullptr, none, halo, err, src, perm);
        return dims == 3 ? persistent_t<3, double>(st, smem, nruns, run_cell_base, a, grid_blocks, launch, ant_n, antennas)
                         : persistent_t<2, double>(st, smem, nruns, run_cell_base, a, grid_blocks, launch, ant_n, antennas);
    }
    auto a = make_args<float>(items, n_items, runs, groups, P, E, B, J, nullptr, none, halo, err, src, perm);
    const int tile[3] = {tx, ty, tz};
    cudaError_t e = cudaSuccess;
    if (launch_persistent_fixed(dims, st, smem, nruns, run_cell_base, a, grid_blocks, launch, tile, halo, p0, p1,
                                ant_n, antennas, &e))
        return e;
    return dims == 3 ? persistent_t<3, float>(st, smem, nruns, run_cell_base, a, grid_blocks, launch, ant_n, antennas)
                     : persistent_t<2, float>(st, smem, nruns, run_cell_base, a, grid_blocks, launch, ant_n, antennas);
}

// ---------------------------------------------------------------------------
// Loader: absolute normalized FP64 positions -> (cell, offset) of the pool's
// precision, periodic wrap into [0, N); an offset that rounds to 1 moves to the
// next cell with offset 0.  Momenta are converted; id = index in the call.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void k_load(long long n, const double *x0, const double *x1, const double *x2, const double *w0,
                       const double *w1, const double *w2, int dims, int nx, int ny, int nz, int *cell,
                       R *off0, R *off1, R *off2, R *wo0, R *wo1, R *wo2, int *id, long long base)
{
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= n) return;
    const double *xs[3] = {x0, x1, x2};
    R *offs[3] = {off0, off1, off2};
    const int nn[3] = {nx, ny, nz};
    int ci[3] = {0, 0, 0};
    for (int a = 0; a < dims; ++a) {
        const double N = (double)nn[a];
        double x = xs[a][p];
        x -= N * floor(x / N);
        if (x >= N) x -= N;
        if (x < 0.0) x = 0.0;
        double fl = floor(x);
        int c = (int)fl;
        if (c >= nn[a]) c = nn[a] - 1;
        R o = (R)(x - (double)c);
        if (o >= R(1)) {
            o = R(0);
            c = c + 1 == nn[a] ? 0 : c + 1;
        }
        ci[a] = c;
        offs[a][base + p] = o;
    }
    cell[base + p] = ci[0] + nx * (ci[1] + ny * ci[2]);
    wo0[base + p] = (R)w0[p];
    wo1[base + p] = (R)w1[p];
    wo2[base + p] = (R)w2[p];
    id[base + p] = (int)p;
}

cudaError_t launch_load(int prec, cudaStream_t st, long long n, const double *x0, const double *x1,
                        const double *x2, const double *w0, const double *w1, const double *w2, int dims, int nx,
                        int ny, int nz, const PoolBuf &P, long long base)
{
    if (n <= 0) return cudaSuccess;
    const int nt = 256;
    const long long nb = (n + nt - 1) / nt;
    if (prec == 0) {
        k_load<double><<<(unsigned)nb, nt, 0, st>>>(n, x0, x1, dims == 3 ? x2 : x0, w0, w1, w2, dims, nx, ny, nz,
                                                    P.cell, (double *)P.off[0], (double *)P.off[1],
                                                    dims == 3 ? (double *)P.off[2] : (double *)P.off[0],
                                                    (double *)P.w[0], (double *)P.w[1], (double *)P.w[2], P.id, base);
    } else {
        k_load<float><<<(unsigned)nb, nt, 0, st>>>(n, x0, x1, dims == 3 ? x2 : x0, w0, w1, w2, dims, nx, ny, nz,
                                                   P.cell, (float *)P.off[0], (float *)P.off[1],
                                                   dims == 3 ? (float *)P.off[2] : (float *)P.off[0],
                                                   (float *)P.w[0], (float *)P.w[1], (float *)P.w[2], P.id, base);
    }
    return cudaGetLastError();
}

// Device-to-device copy of a range of pool entries (used when the pool is re-laid out).
template <typename R>
__global__ void k_copy_pool(long long n, const int *sc, const R *so0, const R *so1, const R *so2, const R *sw0,
                            const R *sw1, const R *sw2, const int *sid, int *dc, R *do0, R *do1, R *do2, R *dw0,
                            R *dw1, R *dw2, int *did)
{
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= n) return;
    dc[p] = sc[p];
    do0[p] = so0[p];
    do1[p] = so1[p];
    if (do2) do2[p] = so2[p];
    dw0[p] = sw0[p];
    dw1[p] = sw1[p];
    dw2[p] = sw2[p];
    did[p] = sid[p];
}

cudaError_t launch_copy_pool(int prec, cudaStream_t st, const PoolBuf &src, long long sb, const PoolBuf &dst,
                             long long db, long long n)
{
    if (n <= 0) return cudaSuccess;
    const int nt = 256;
    const unsigned nb = (unsigned)((n + nt - 1) / nt);
    if (prec == 0) {
        auto S = [&](void *p) { return p ? (double *)p + sb : nullptr; };
        auto D = [&](void *p) { return p ? (double *)p + db : nullptr; };
        k_copy_pool<double><<<nb, nt, 0, st>>>(n, src.cell + sb, S(src.off[0]), S(src.off[1]), S(src.off[2]),
                                               S(src.w[0]), S(src.w[1]), S(src.w[2]), src.id + sb, dst.cell + db,
                                               D(dst.off[0]), D(dst.off[1]), D(dst.off[2]), D(dst.w[0]),
                                               D(dst.w[1]), D(dst.w[2]), dst.id + db);
    } else {
        auto S = [&](void *p) { return p ? (float *)p + sb : nullptr; };
        auto D = [&](void *p) { return p ? (float *)p + db : nullptr; };
        k_copy_pool<float><<<nb, nt, 0, st>>>(n, src.cell + sb, S(src.off[0]), S(src.off[1]), S(src.off[2]),
                                              S(src.w[0]), S(src.w[1]), S(src.w[2]), src.id + sb, dst.cell + db,
                                              D(dst.off[0]), D(dst.off[1]), D(dst.off[2]), D(dst.w[0]),
                                              D(dst.w[1]), D(dst.w[2]), dst.id + db);
    }
    return cudaGetLastError();
}

}  // namespace pic
