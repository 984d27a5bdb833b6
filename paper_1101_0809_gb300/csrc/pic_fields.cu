// pic_fields.cu -- Yee field updates of the Appendix (Eqs. updateB, escheme),
// one thread per cell, x-fastest so that warps read and write coalesced rows.
// Runs of a batch are blockIdx.y; blocks past a run's last cell return.  The
// per-cell arithmetic is in pic_device.cuh (shared with the persistent kernel).
#include "pic_internal.h"

namespace pic {

template <int DIM, typename R>
__global__ void k_yee_b_half(const RunDev *runs, Fields<R> F, int zero_j, const long long *ant_n)
{
    const RunDev &rn = runs[blockIdx.y];
    const long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (l >= (long long)rn.n[0] * rn.n[1] * rn.n[2]) return;
    yee_b_half_cell<DIM, R>(rn, F, l, zero_j, ant_n[blockIdx.y]);
}

template <int DIM, typename R>
__global__ void k_yee_e(const RunDev *runs, Fields<R> F, const long long *ant_n)
{
    const RunDev &rn = runs[blockIdx.y];
    const long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (l >= (long long)rn.n[0] * rn.n[1] * rn.n[2]) return;
    yee_e_cell<DIM, R>(rn, F, l, ant_n[blockIdx.y]);
}

// Advances every run's antenna clock by one E step.
__global__ void k_antenna_tick(long long *ant_n, int nruns)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < nruns) ant_n[r] += 1;
}

cudaError_t launch_antenna_tick(cudaStream_t st, long long *ant_n, int nruns)
{
    k_antenna_tick<<<(nruns + 255) / 256, 256, 0, st>>>(ant_n, nruns);
    return cudaGetLastError();
}

template <int DIM, typename R>
static cudaError_t launch_yee_t(int which, int zero_j, cudaStream_t st, const RunDev *runs, int nruns,
                                long long max_cells, void *const E[3], void *const B[3], void *const J[3],
                                const long long *ant_n)
{
    Fields<R> F;
    for (int c = 0; c < 3; ++c) {
        F.E[c] = static_cast<R *>(E[c]);
        F.B[c] = static_cast<R *>(B[c]);
        F.J[c] = static_cast<R *>(J[c]);
    }
    const int nt = 256;
    dim3 grid((unsigned)((max_cells + nt - 1) / nt), (unsigned)nruns);
    if (which == 1)
        k_yee_b_half<DIM, R><<<grid, nt, 0, st>>>(runs, F, zero_j, ant_n);
    else
        k_yee_e<DIM, R><<<grid, nt, 0, st>>>(runs, F, ant_n);
    return cudaGetLastError();
}

cudaError_t launch_yee(int prec, int which, int zero_j, cudaStream_t st, const RunDev *runs, int nruns,
                       long long max_cells, void *const E[3], void *const B[3], void *const J[3], int dims,
                       const long long *ant_n)
{
    if (dims == 3)
        return prec == 0 ? launch_yee_t<3, double>(which, zero_j, st, runs, nruns, max_cells, E, B, J, ant_n)
                         : launch_yee_t<3, float>(which, zero_j, st, runs, nruns, max_cells, E, B, J, ant_n);
    return prec == 0 ? launch_yee_t<2, double>(which, zero_j, st, runs, nruns, max_cells, E, B, J, ant_n)
                     : launch_yee_t<2, float>(which, zero_j, st, runs, nruns, max_cells, E, B, J, ant_n);
}

}  // namespace pic
