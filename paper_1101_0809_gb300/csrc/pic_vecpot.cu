// pic_vecpot.cu -- the vector-potential formulation (Sec. 4.2): A on the E
// points, advanced by Eq. dadt (A^{n+1/2} = A^{n-1/2} - c dt E^n, launched with
// the E step, before E changes), B = curl_h A (Eq. viaA, grid form), and the
// generalized momentum sum_p m_p w_p + (q_p/c) A(x_p - (dt/2) u_p) of the
// particles, with A interpolated by the weights alpha of E of the grid's
// interpolation at the time-centred position.
#include "pic_internal.h"

namespace pic {

template <typename R>
__global__ void k_update_A(const RunDev *runs, R *A0, R *A1, R *A2, const R *E0, const R *E1, const R *E2)
{
    const RunDev &rn = runs[blockIdx.y];
    const long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (l >= (long long)rn.n[0] * rn.n[1] * rn.n[2]) return;
    const long long p = rn.cell_base + l;
    const R cdt = (R)(rn.c * rn.dt);
    A0[p] -= cdt * E0[p];
    A1[p] -= cdt * E1[p];
    A2[p] -= cdt * E2[p];
}

// Bx[i,j,k] = (Az[i,j,k] - Az[i,j-1,k])/dy - (Ay[i,j,k] - Ay[i,j,k-1])/dz, cyclically.
template <int DIM, typename R>
__global__ void k_curl_A(const RunDev *runs, const R *A0, const R *A1, const R *A2, R *B0, R *B1, R *B2)
{
    const RunDev &rn = runs[blockIdx.y];
    const int nx = rn.n[0], ny = rn.n[1], nz = rn.n[2];
    const long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (l >= (long long)nx * ny * nz) return;
    const int i = (int)(l % nx);
    const long long r = l / nx;
    const int j = (int)(r % ny), k = (int)(r / ny);
    const long long p = rn.cell_base + l;
    const long long pim = p + (i == 0 ? nx - 1 : -1);
    const long long pjm = p + (long long)nx * (j == 0 ? ny - 1 : -1);
    const double idx = 1.0 / rn.d[0], idy = 1.0 / rn.d[1];
    double bx = ((double)A2[p] - A2[pjm]) * idy;
    double by = -((double)A2[p] - A2[pim]) * idx;
    double bz = ((double)A1[p] - A1[pim]) * idx - ((double)A0[p] - A0[pjm]) * idy;
    if (DIM == 3) {
        const long long pkm = p + (long long)nx * ny * (k == 0 ? nz - 1 : -1);
        const double idz = 1.0 / rn.d[2];
        bx -= ((double)A1[p] - A1[pkm]) * idz;
        by += ((double)A0[p] - A0[pkm]) * idz;
    }
    B0[p] = (R)bx;
    B1[p] = (R)by;
    B2[p] = (R)bz;
}

// A at offsets -2..2 from an index (x: i, y: nx j, z: nx ny k, run-local),
// read as double; B reads as zero, so that the gathers return A's alpha sum.
template <typename R>
struct AReader {
    const R *A[3];
    long long xi[5], yj[5], zk[5];
    __device__ __forceinline__ double e(int a, int dx, int dy, int dz) const
    {
        return (double)A[a][xi[dx + 2] + yj[dy + 2] + zk[dz + 2]];
    }
    __device__ __forceinline__ double b(int, int, int, int) const { return 0.0; }
};

template <int DIM, typename R, int ORD>
__global__ void __launch_bounds__(256) k_gen_momentum(int run, long long total, const long long *group_base,
                                                      int ngroups, const GroupDev *groups, const RunDev *runs,
                                                      Pool<R> P, const R *A0, const R *A1, const R *A2, double *out)
{
    double acc[3] = {0.0, 0.0, 0.0};
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < total; p += stride) {
        int lo = 0, hi = ngroups;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (group_base[mid] <= p) lo = mid; else hi = mid;
        }
        const GroupDev gr = groups[lo];
        if (gr.run != run) continue;
        const RunDev &rn = runs[run];
        const int n3[3] = {rn.n[0], rn.n[1], rn.n[2]};
        const int c = P.cell[p];
        int ci[3] = {c % n3[0], (c / n3[0]) % n3[1], DIM == 3 ? c / (n3[0] * n3[1]) : 0};
        const double w[3] = {(double)P.w[0][p], (double)P.w[1][p], (double)P.w[2][p]};
        const double gam = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2] + rn.c * rn.c);
        double x[3] = {0.5, 0.5, 0.5};
        for (int a = 0; a < DIM; ++a) {
            // the time-centred position x^n - (dt/2) u^{n-1/2}: less than half a cell away
            x[a] = (double)P.off[a][p] - 0.5 * rn.cN[a] * w[a] / gam;
            if (x[a] < 0.0) { x[a] += 1.0; ci[a] = ci[a] == 0 ? n3[a] - 1 : ci[a] - 1; }
            else if (x[a] >= 1.0) { x[a] -= 1.0; ci[a] = ci[a] == n3[a] - 1 ? 0 : ci[a] + 1; }
        }
        // the base index of the weights (the cell, or for l_a = 2 1/2 the nearest integer)
        int ib[3] = {ci[0], ci[1], ci[2]};
        double d5[3] = {0.5, 0.5, 0.5};
        if (ORD == 5)
            for (int a = 0; a < DIM; ++a) ib[a] += split5(x[a], d5[a]);
        AReader<R> rd;
        rd.A[0] = A0; rd.A[1] = A1; rd.A[2] = A2;
        for (int q = 0; q < 5; ++q) {
            // ib - 2 + q lies in [-2, n + 2]: one wrap suffices on these grids (n >= 4)
            rd.xi[q] = rn.cell_base + wrapi(ib[0] - 2 + q, n3[0]);
            rd.yj[q] = (long long)n3[0] * wrapi(ib[1] - 2 + q, n3[1]);
            rd.zk[q] = DIM == 3 ? (long long)n3[0] * n3[1] * wrapi(ib[2] - 2 + q, n3[2]) : 0;
        }
        double Ap[3], Bp[3];
        if (ORD == 5) {
            double wt[21];
            form_factor5(d5[0], wt, wt + 3);
            form_factor5(d5[1], wt + 7, wt + 10);
            form_factor5(d5[2], wt + 14, wt + 17);
            gather5<DIM>(rd, wt, wt + 3, wt + 7, wt + 10, wt + 14, wt + 17, Ap, Bp);
        } else {
            double f[3][2], S[3][3];
            for (int a = 0; a < 3; ++a) {
                if (a < DIM) {
                    form_factor(x[a], f[a], S[a]);
                } else {
                    f[a][0] = 1.0; f[a][1] = 0.0; S[a][0] = 0.0; S[a][1] = 1.0; S[a][2] = 0.0;
                }
            }
            if (ORD == 4)
                gather_w1<DIM>(rd, S[0], S[1], S[2], Ap, Bp);
            else
                gather<DIM>(rd, f[0], S[0], f[1], S[1], f[2], S[2], Ap, Bp);
        }
        for (int a = 0; a < 3; ++a) acc[a] += gr.mp * w[a] + gr.qp / rn.c * Ap[a];
    }
    for (int a = 0; a < 3; ++a) {
        double v = acc[a];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) atomicAdd(&out[a], v);
    }
}

template <typename R>
static cudaError_t vp_fields_t(int which, int dims, cudaStream_t st, const RunDev *runs, int nruns,
                               long long max_cells, void *const A[3], void *const F[3])
{
    const int nt = 256;
    dim3 grid((unsigned)((max_cells + nt - 1) / nt), (unsigned)nruns);
    R *a[3], *f[3];
    for (int c = 0; c < 3; ++c) { a[c] = (R *)A[c]; f[c] = (R *)F[c]; }
    if (which == 0)
        k_update_A<R><<<grid, nt, 0, st>>>(runs, a[0], a[1], a[2], f[0], f[1], f[2]);
    else if (dims == 3)
        k_curl_A<3, R><<<grid, nt, 0, st>>>(runs, a[0], a[1], a[2], f[0], f[1], f[2]);
    else
        k_curl_A<2, R><<<grid, nt, 0, st>>>(runs, a[0], a[1], a[2], f[0], f[1], f[2]);
    return cudaGetLastError();
}

cudaError_t launch_update_A(int prec, cudaStream_t st, const RunDev *runs, int nruns, long long max_cells,
                            void *const A[3], void *const E[3])
{
    return prec == 0 ? vp_fields_t<double>(0, 0, st, runs, nruns, max_cells, A, E)
                     : vp_fields_t<float>(0, 0, st, runs, nruns, max_cells, A, E);
}

cudaError_t launch_curl_A(int dims, int prec, cudaStream_t st, const RunDev *runs, int nruns, long long max_cells,
                          void *const A[3], void *const B[3])
{
    return prec == 0 ? vp_fields_t<double>(1, dims, st, runs, nruns, max_cells, A, B)
                     : vp_fields_t<float>(1, dims, st, runs, nruns, max_cells, A, B);
}

template <int DIM, typename R>
static cudaError_t gm_t(int order2, cudaStream_t st, int run, long long total, const long long *gbase, int ngroups,
                        const GroupDev *groups, const RunDev *runs, const PoolBuf &PB, void *const A[3], double *out)
{
    Pool<R> P;
    P.cell = PB.cell;
    P.id = PB.id;
    for (int c = 0; c < 3; ++c) {
        P.off[c] = (R *)PB.off[c];
        P.w[c] = (R *)PB.w[c];
    }
    const R *a0 = (const R *)A[0], *a1 = (const R *)A[1], *a2 = (const R *)A[2];
    cudaError_t e = cudaMemsetAsync(out, 0, 3 * sizeof(double), st);
    if (e != cudaSuccess || total <= 0) return e;
    const int blocks = (int)((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096);
    if (order2 == 5)
        k_gen_momentum<DIM, R, 5><<<blocks, 256, 0, st>>>(run, total, gbase, ngroups, groups, runs, P, a0, a1, a2, out);
    else if (order2 == 4)
        k_gen_momentum<DIM, R, 4><<<blocks, 256, 0, st>>>(run, total, gbase, ngroups, groups, runs, P, a0, a1, a2, out);
    else
        k_gen_momentum<DIM, R, 3><<<blocks, 256, 0, st>>>(run, total, gbase, ngroups, groups, runs, P, a0, a1, a2, out);
    return cudaGetLastError();
}

cudaError_t launch_gen_momentum(int dims, int prec, int order2, cudaStream_t st, int run, long long total,
                                const long long *gbase, int ngroups, const GroupDev *groups, const RunDev *runs,
                                const PoolBuf &P, void *const A[3], double *out)
{
    if (dims == 3)
        return prec == 0 ? gm_t<3, double>(order2, st, run, total, gbase, ngroups, groups, runs, P, A, out)
                         : gm_t<3, float>(order2, st, run, total, gbase, ngroups, groups, runs, P, A, out);
    return prec == 0 ? gm_t<2, double>(order2, st, run, total, gbase, ngroups, groups, runs, P, A, out)
                     : gm_t<2, float>(order2, st, run, total, gbase, ngroups, groups, runs, P, A, out);
}

}  // namespace pic
