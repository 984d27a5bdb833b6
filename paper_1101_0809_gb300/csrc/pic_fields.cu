// pic_fields.cu -- Yee field updates of the Appendix (Eqs. updateB, escheme),
// one thread per cell, x-fastest so that warps read and write coalesced rows.
// Runs of a batch are blockIdx.y; blocks past a run's last cell return.
#include "pic_internal.h"

namespace pic {

// B half step (Eq. updateB, completed cyclically):
//   Bx[i,j,k] -= (c_y/2)(Ez[i,j,k]-Ez[i,j-1,k]) - (c_z/2)(Ey[i,j,k]-Ey[i,j,k-1])
//   By[i,j,k] -= (c_z/2)(Ex[i,j,k]-Ex[i,j,k-1]) - (c_x/2)(Ez[i,j,k]-Ez[i-1,j,k])
//   Bz[i,j,k] -= (c_x/2)(Ey[i,j,k]-Ey[i-1,j,k]) - (c_y/2)(Ex[i,j,k]-Ex[i,j-1,k])
// With zero_j the same pass clears J for the coming deposit.
template <int DIM, typename R>
__global__ void k_yee_b_half(const RunDev *runs, Fields<R> F, int zero_j)
{
    const RunDev rn = runs[blockIdx.y];
    const int nx = rn.n[0], ny = rn.n[1], nz = rn.n[2];
    const long long ncell = (long long)nx * ny * nz;
    const long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (l >= ncell) return;
    const int i = (int)(l % nx);
    const long long r = l / nx;
    const int j = (int)(r % ny);
    const int k = (int)(r / ny);
    const long long p = rn.cell_base + l;
    const long long pim = p + (i == 0 ? nx - 1 : -1);
    const long long pjm = p + (long long)nx * (j == 0 ? ny - 1 : -1);
    const R hx = R(0.5 * rn.cN[0]), hy = R(0.5 * rn.cN[1]);
    const R ex = F.E[0][p], ey = F.E[1][p], ez = F.E[2][p];
    R bx = F.B[0][p] - hy * (ez - F.E[2][pjm]);
    R by = F.B[1][p] + hx * (ez - F.E[2][pim]);
    R bz = F.B[2][p] - hx * (ey - F.E[1][pim]) + hy * (ex - F.E[0][pjm]);
    if (DIM == 3) {
        const long long pkm = p + (long long)nx * ny * (k == 0 ? nz - 1 : -1);
        const R hz = R(0.5 * rn.cN[2]);
        bx += hz * (ey - F.E[1][pkm]);
        by -= hz * (ex - F.E[0][pkm]);
    }
    F.B[0][p] = bx;
    F.B[1][p] = by;
    F.B[2][p] = bz;
    if (zero_j) {
        F.J[0][p] = R(0);
        F.J[1][p] = R(0);
        F.J[2][p] = R(0);
    }
}

// E full step (Eq. escheme, completed cyclically):
//   Ex += -4 pi dt Jx + c_y(Bz[i,j+1,k]-Bz[i,j,k]) - c_z(By[i,j,k+1]-By[i,j,k])
//   Ey += -4 pi dt Jy + c_z(Bx[i,j,k+1]-Bx[i,j,k]) - c_x(Bz[i+1,j,k]-Bz[i,j,k])
//   Ez += -4 pi dt Jz + c_x(By[i+1,j,k]-By[i,j,k]) - c_y(Bx[i,j+1,k]-Bx[i,j,k])
template <int DIM, typename R>
__global__ void k_yee_e(const RunDev *runs, Fields<R> F)
{
    const RunDev rn = runs[blockIdx.y];
    const int nx = rn.n[0], ny = rn.n[1], nz = rn.n[2];
    const long long ncell = (long long)nx * ny * nz;
    const long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (l >= ncell) return;
    const int i = (int)(l % nx);
    const long long r = l / nx;
    const int j = (int)(r % ny);
    const int k = (int)(r / ny);
    const long long p = rn.cell_base + l;
    const long long pip = p + (i == nx - 1 ? -(nx - 1) : 1);
    const long long pjp = p + (long long)nx * (j == ny - 1 ? -(ny - 1) : 1);
    const R cx = R(rn.cN[0]), cy = R(rn.cN[1]);
    const R fp = R(4.0 * 3.14159265358979323846 * rn.dt);
    const R bx = F.B[0][p], by = F.B[1][p], bz = F.B[2][p];
    R ex = F.E[0][p] - fp * F.J[0][p] + cy * (F.B[2][pjp] - bz);
    R ey = F.E[1][p] - fp * F.J[1][p] - cx * (F.B[2][pip] - bz);
    R ez = F.E[2][p] - fp * F.J[2][p] + cx * (F.B[1][pip] - by) - cy * (F.B[0][pjp] - bx);
    if (DIM == 3) {
        const long long pkp = p + (long long)nx * ny * (k == nz - 1 ? -(nz - 1) : 1);
        const R cz = R(rn.cN[2]);
        ex -= cz * (F.B[1][pkp] - by);
        ey += cz * (F.B[0][pkp] - bx);
    }
    F.E[0][p] = ex;
    F.E[1][p] = ey;
    F.E[2][p] = ez;
}

template <int DIM, typename R>
static cudaError_t launch_yee_t(int which, int zero_j, cudaStream_t st, const RunDev *runs, int nruns,
                                long long max_cells, void *const E[3], void *const B[3], void *const J[3])
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
        k_yee_b_half<DIM, R><<<grid, nt, 0, st>>>(runs, F, zero_j);
    else
        k_yee_e<DIM, R><<<grid, nt, 0, st>>>(runs, F);
    return cudaGetLastError();
}

cudaError_t launch_yee(int prec, int which, int zero_j, cudaStream_t st, const RunDev *runs, int nruns,
                       long long max_cells, void *const E[3], void *const B[3], void *const J[3], int dims)
{
    if (dims == 3)
        return prec == 0 ? launch_yee_t<3, double>(which, zero_j, st, runs, nruns, max_cells, E, B, J)
                         : launch_yee_t<3, float>(which, zero_j, st, runs, nruns, max_cells, E, B, J);
    return prec == 0 ? launch_yee_t<2, double>(which, zero_j, st, runs, nruns, max_cells, E, B, J)
                     : launch_yee_t<2, float>(which, zero_j, st, runs, nruns, max_cells, E, B, J);
}

}  // namespace pic
