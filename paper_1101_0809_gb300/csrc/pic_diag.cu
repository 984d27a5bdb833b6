// pic_diag.cu -- FP64 diagnostics of one run at time level n (state E^n,
// B^{n-1/2}, x^n, w^{n-1/2}), whatever the precision of the state:
//   rho^n from the stored positions (Eq. rho), the Gauss residual
//   r = div_h E - 4 pi rho (Eq. chargelaw, Poisson form of Sec. 2) against a
//   stored reference, the energy integral of Sec. 4.1 (kinetic part without
//   rest mass, B^n = B^{n-1/2} - (1/2) c curl_h E^n), and the momentum sum.
// Sums are per-block tree reductions written to fixed slots and reduced by one
// block in slot order.
#include "pic_internal.h"

namespace pic {

constexpr int kDiagThreads = 256;
constexpr int kPartVals = 8;   // values per partial slot
constexpr double kPi = 3.14159265358979323846;

template <typename R>
struct ConvReader {   // reads the state's precision, returns double, periodic indices
    const R *E[3];
    const R *B[3];
    long long xi[4], yj[4], zk[4];
    __device__ __forceinline__ long long at(int dx, int dy, int dz) const { return xi[dx + 1] + yj[dy + 1] + zk[dz + 1]; }
    __device__ __forceinline__ double e(int a, int dx, int dy, int dz) const { return (double)E[a][at(dx, dy, dz)]; }
    __device__ __forceinline__ double b(int a, int dx, int dy, int dz) const { return (double)B[a][at(dx, dy, dz)]; }
};

template <typename R>
struct ConvReader5 {   // the same with offsets -2..2 (l_a = 2 1/2, relative to the base index)
    const R *E[3];
    const R *B[3];
    long long xi[5], yj[5], zk[5];
    __device__ __forceinline__ long long at(int dx, int dy, int dz) const { return xi[dx + 2] + yj[dy + 2] + zk[dz + 2]; }
    __device__ __forceinline__ double e(int a, int dx, int dy, int dz) const { return (double)E[a][at(dx, dy, dz)]; }
    __device__ __forceinline__ double b(int a, int dx, int dy, int dz) const { return (double)B[a][at(dx, dy, dz)]; }
};

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_max(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

// Block reduction of kPartVals values (sums, except slot `max_slot` which is a max).
__device__ void block_reduce_store(double v[kPartVals], int max_slot, double *out)
{
    __shared__ double sh[kDiagThreads / 32][kPartVals];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < kPartVals; ++q) {
        const double r = q == max_slot ? warp_max(v[q]) : warp_sum(v[q]);
        if (lane == 0) sh[warp][q] = r;
    }
    __syncthreads();
    if (threadIdx.x < kPartVals) {
        const int q = threadIdx.x;
        double acc = sh[0][q];
        for (int w = 1; w < kDiagThreads / 32; ++w) acc = q == max_slot ? fmax(acc, sh[w][q]) : acc + sh[w][q];
        out[q] = acc;
    }
}

// Particles: rho deposit (atomics) and kinetic / momentum / half-step sums.
// Partial slots: 0 kinetic, 1-3 momentum, 4 half-step correction, 5 count.
// ORD = 3: l_a = 1 1/2 (rho over the 3 cells per axis around the cell);
// ORD = 5: l_a = 2 1/2 (rho over the 4 cells ib-2 .. ib+1 of the base index);
// ORD = 4: the comparison scheme of Eq. wrong1 (rho of l_a = 1 1/2, its own gather).
template <int DIM, typename R, int ORD = 3>
__global__ void __launch_bounds__(kDiagThreads) k_diag_particles(int run, long long total, const long long *group_base,
                                                                 int ngroups, const GroupDev *groups, const RunDev *runs,
                                                                 Pool<R> P, Fields<R> F, double *rho, double *partials)
{
    double v[kPartVals] = {0, 0, 0, 0, 0, 0, 0, 0};
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < total; p += stride) {
        int lo = 0, hi = ngroups;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (group_base[mid] <= p) lo = mid; else hi = mid;
        }
        const GroupDev g = groups[lo];
        if (g.run != run) continue;
        const RunDev rn = runs[g.run];
        const int nx = rn.n[0], ny = rn.n[1], nz = rn.n[2];
        const int c = P.cell[p];
        const int i = c % nx, rest = c / nx, j = rest % ny, k = DIM == 3 ? rest / ny : 0;
        const double qV = g.qp / rn.V;
        double Ep[3], Bp[3];
        if constexpr (ORD == 5) {
            double e3[3] = {0.5, 0.5, 0.5}, w[21];
            int u3[3] = {0, 0, 0};
            for (int ax = 0; ax < DIM; ++ax) u3[ax] = split5((double)P.off[ax][p], e3[ax]);
            form_factor5(e3[0], w, w + 3);
            form_factor5(e3[1], w + 7, w + 10);
            form_factor5(e3[2], w + 14, w + 17);
            const int ib = i + u3[0], jb = j + u3[1], kb = k + u3[2];
            const int nzw = DIM == 3 ? 4 : 1;
            for (int dz = 0; dz < nzw; ++dz)
                for (int dy = 0; dy < 4; ++dy)
                    for (int dx = 0; dx < 4; ++dx) {
                        const long long idx =
                            rn.cell_base + wrapi(ib + dx - 2, nx) +
                            (long long)nx * (wrapi(jb + dy - 2, ny) + (long long)ny * (DIM == 3 ? wrapi(kb + dz - 2, nz) : 0));
                        atomicAdd(&rho[idx], qV * w[3 + dx] * w[10 + dy] * (DIM == 3 ? w[17 + dz] : 1.0));
                    }
            ConvReader5<R> rd;
            for (int q = 0; q < 3; ++q) { rd.E[q] = F.E[q]; rd.B[q] = F.B[q]; }
            for (int q = 0; q < 5; ++q) {
                rd.xi[q] = rn.cell_base + wrapi(ib - 2 + q, nx);
                rd.yj[q] = (long long)nx * wrapi(jb - 2 + q, ny);
                rd.zk[q] = DIM == 3 ? (long long)nx * ny * wrapi(kb - 2 + q, nz) : 0;
            }
            gather5<DIM>(rd, w, w + 3, w + 7, w + 10, w + 14, w + 17, Ep, Bp);
        } else {
            double fx[2], Sx[3], fy[2], Sy[3], fz[2], Sz[3];
            form_factor((double)P.off[0][p], fx, Sx);
            form_factor((double)P.off[1][p], fy, Sy);
            if (DIM == 3) {
                form_factor((double)P.off[2][p], fz, Sz);
            } else {
                fz[0] = 1; fz[1] = 0; Sz[0] = 0; Sz[1] = 1; Sz[2] = 0;
            }
            const int kz0 = DIM == 3 ? -1 : 0, kz1 = DIM == 3 ? 1 : 0;
            for (int dz = kz0; dz <= kz1; ++dz)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        const long long idx = rn.cell_base + wrapi(i + dx, nx) +
                                              (long long)nx * (wrapi(j + dy, ny) + (long long)ny * (DIM == 3 ? wrapi(k + dz, nz) : 0));
                        atomicAdd(&rho[idx], qV * Sx[dx + 1] * Sy[dy + 1] * Sz[dz + 1]);
                    }
            ConvReader<R> rd;
            for (int q = 0; q < 3; ++q) { rd.E[q] = F.E[q]; rd.B[q] = F.B[q]; }
            for (int q = 0; q < 4; ++q) {
                rd.xi[q] = rn.cell_base + wrapi(i - 1 + q, nx);
                rd.yj[q] = (long long)nx * wrapi(j - 1 + q, ny);
                rd.zk[q] = DIM == 3 ? (long long)nx * ny * wrapi(k - 1 + q, nz) : 0;
            }
            if constexpr (ORD == 4)
                gather_w1<DIM>(rd, Sx, Sy, Sz, Ep, Bp);
            else
                gather<DIM>(rd, fx, Sx, fy, Sy, fz, Sz, Ep, Bp);
        }
        const double w0 = (double)P.w[0][p], w1 = (double)P.w[1][p], w2 = (double)P.w[2][p];
        const double gam = sqrt(w0 * w0 + w1 * w1 + w2 * w2 + rn.c * rn.c);
        v[0] += g.mp * rn.c * (gam - rn.c);
        v[1] += g.mp * w0;
        v[2] += g.mp * w1;
        v[3] += g.mp * w2;
        v[4] += 0.5 * g.qp * rn.dt * rn.c * (w0 * Ep[0] + w1 * Ep[1] + w2 * Ep[2]) / gam;
        v[5] += 1.0;
    }
    block_reduce_store(v, -1, partials + (long long)blockIdx.x * kPartVals);
}

// FP32 state: the same particle sums over the tile-sorted work items.  A block
// stages the item's E tile (halo + 1) in shared memory and accumulates rho on a
// shared tile in integer fixed point (the current tile's scheme of the
// particle kernels, scale rscale per group), then adds it to the FP64 rho.  The
// per-particle terms are FP32 (kinetic energy in the cancellation-free form
// m c w^2 / (gamma + c)), every sum FP64.  Particles more than `halo` cells
// outside their tile read E and add rho on the global arrays.  Blocks take
// items round-robin, so the partial slot of a block sums a fixed set of items.
struct ZeroB {   // gather reader for E only: B reads as 0
    const float *E[3];
    int base, s1, s2;
    __device__ __forceinline__ float e(int a, int dx, int dy, int dz) const { return E[a][base + dx + s1 * dy + s2 * dz]; }
    __device__ __forceinline__ float b(int, int, int, int) const { return 0.0f; }
};
struct GlobalZeroB {
    const float *E[3];
    long long xi[4], yj[4], zk[4];
    __device__ __forceinline__ float e(int a, int dx, int dy, int dz) const { return E[a][xi[dx + 1] + yj[dy + 1] + zk[dz + 1]]; }
    __device__ __forceinline__ float b(int, int, int, int) const { return 0.0f; }
};
struct GlobalZeroB5 {   // offsets -2..2 from the l_a = 2 1/2 base index
    const float *E[3];
    long long xi[5], yj[5], zk[5];
    __device__ __forceinline__ float e(int a, int dx, int dy, int dz) const { return E[a][xi[dx + 2] + yj[dy + 2] + zk[dz + 2]]; }
    __device__ __forceinline__ float b(int, int, int, int) const { return 0.0f; }
};

// ORD = 5 (l_a = 2 1/2): E and rho tiles with a halo of (halo + 2) cells, the
// 4-cell cubic weights around the base index.  ORD = 4 (Eq. wrong1): the same
// halo for its gather, the l_a = 1 1/2 charge.
template <int DIM, int ORD = 3>
__global__ void __launch_bounds__(kDiagThreads, 2) k_diag_items(int run, const WorkItem *items, const int *n_items,
                                                             const GroupDev *groups, const RunDev *runs, Pool<float> P,
                                                             Fields<float> F, int halo, double *rho, double *partials)
{
    extern __shared__ __align__(16) unsigned char dsm[];
    double v[kPartVals] = {0, 0, 0, 0, 0, 0, 0, 0};
    const int ni = *n_items;
    const RunDev &rn = runs[run];
    const int G = halo;
    const int nx = rn.n[0], ny = rn.n[1], nz = rn.n[2];
    const int T0 = rn.tile[0], T1 = rn.tile[1], T2 = DIM == 3 ? rn.tile[2] : 1;
    const int P0 = rn.pitch[0], P1 = rn.pitch[1];
    constexpr int FH = ORD == 3 ? 1 : 2;   // tile halo beyond G
    const int fe0 = T0 + 2 * (G + FH), fe1 = T1 + 2 * (G + FH), fe2 = DIM == 3 ? T2 + 2 * (G + FH) : 1;
    const int nf = P0 * P1 * fe2;
    float *sE[3];
    for (int c = 0; c < 3; ++c) sE[c] = reinterpret_cast<float *>(dsm) + c * nf;
    int *rh = reinterpret_cast<int *>(dsm) + 3 * nf;
    int *rl = rh + nf;
    const long long cb = rn.cell_base;
    const float cl = rn.cf, c2 = cl * cl;
    for (int item = blockIdx.x; item < ni; item += gridDim.x) {
        const WorkItem it = items[item];
        const GroupDev &gr = groups[it.group];
        if (gr.run != run) continue;   // the same for the whole block
        const int tx = it.tile % rn.ntile[0];
        const int ty = (it.tile / rn.ntile[0]) % rn.ntile[1];
        const int tz = DIM == 3 ? it.tile / (rn.ntile[0] * rn.ntile[1]) : 0;
        const int ox = tx * T0, oy = ty * T1, oz = tz * T2;
        for (int l = threadIdx.x; l < nf; l += blockDim.x) {
            const int lx = l % P0, r = l / P0, ly = r % P1, lz = r / P1;
            rh[l] = 0;
            rl[l] = 0;
            if (lx >= fe0 || ly >= fe1) continue;   // pitch padding
            const int gx = wrapi(ox - G - FH + lx, nx);
            const int gy = wrapi(oy - G - FH + ly, ny);
            const int gz = DIM == 3 ? wrapi(oz - G - FH + lz, nz) : 0;
            const long long gi = cb + gx + (long long)nx * (gy + (long long)ny * gz);
            for (int c = 0; c < 3; ++c) sE[c][l] = F.E[c][gi];
        }
        __syncthreads();
        const float qV = (float)(gr.qp / rn.V);
        const float kq = qV * gr.rscale;
        const float mp = (float)gr.mp;
        const float hqdt = (float)(0.5 * gr.qp * rn.dt * rn.c);
        FixedAcc acc;
        acc.hi[0] = rh;
        acc.lo[0] = rl;
        acc.s1 = P0;
        acc.s2 = P0 * P1;
        // the item's share of this thread (at most particles per item / threads
        // values) is summed in FP32 with Kahan compensation, then added in FP64
        float ks[5] = {0, 0, 0, 0, 0}, kc[5] = {0, 0, 0, 0, 0};
        int count = 0;
        auto kahan = [&](int q, float x) {
            const float y = x - kc[q];
            const float t = ks[q] + y;
            kc[q] = (t - ks[q]) - y;
            ks[q] = t;
        };
        for (long long p = it.begin + threadIdx.x; p < it.end; p += blockDim.x) {
            const int c0 = P.cell[p];
            const int rest = divu31(c0, rn.div_nx);
            const int i = c0 - rest * nx;
            const int k = DIM == 3 ? divu31(rest, rn.div_ny) : 0;
            const int j = rest - k * ny;
            int li = i - ox, lj = j - oy, lk = k - oz;
            if (li >= T0 + G) li -= nx; if (li < -G) li += nx;
            if (lj >= T1 + G) lj -= ny; if (lj < -G) lj += ny;
            if (DIM == 3) { if (lk >= T2 + G) lk -= nz; if (lk < -G) lk += nz; }
            const bool inr = li >= -G && li < T0 + G && lj >= -G && lj < T1 + G && (DIM == 2 || (lk >= -G && lk < T2 + G));
            float Ep[3], Bp[3];
            if constexpr (ORD == 5) {
                float e3[3] = {0.5f, 0.5f, 0.5f}, w[21];
                int u3[3] = {0, 0, 0};
                u3[0] = split5(P.off[0][p], e3[0]);
                u3[1] = split5(P.off[1][p], e3[1]);
                if (DIM == 3) u3[2] = split5(P.off[2][p], e3[2]);
                form_factor5(e3[0], w, w + 3);
                form_factor5(e3[1], w + 7, w + 10);
                form_factor5(e3[2], w + 14, w + 17);
                const int nzw = DIM == 3 ? 4 : 1;
                if (inr) {
                    ZeroB rd;
                    for (int c = 0; c < 3; ++c) rd.E[c] = sE[c];
                    rd.base = (li + u3[0] + G + FH) +
                              P0 * ((lj + u3[1] + G + FH) + (DIM == 3 ? P1 * (lk + u3[2] + G + FH) : 0));
                    rd.s1 = P0;
                    rd.s2 = P0 * P1;
                    gather5<DIM>(rd, w, w + 3, w + 7, w + 10, w + 14, w + 17, Ep, Bp);
                    acc.base = rd.base;
#pragma unroll
                    for (int dz = 0; dz < nzw; ++dz)
#pragma unroll
                        for (int dy = 0; dy < 4; ++dy) {
                            const float t = w[10 + dy] * (DIM == 3 ? w[17 + dz] : 1.0f);
#pragma unroll
                            for (int dx = 0; dx < 4; ++dx)
                                acc.add(0, dx - 2, dy - 2, DIM == 3 ? dz - 2 : 0, kq * w[3 + dx], t);
                        }
                } else {
                    const int ib = i + u3[0], jb = j + u3[1], kb = k + u3[2];
                    GlobalZeroB5 rd;
                    for (int c = 0; c < 3; ++c) rd.E[c] = F.E[c];
                    for (int q = 0; q < 5; ++q) {
                        rd.xi[q] = cb + wrapi(ib - 2 + q, nx);
                        rd.yj[q] = (long long)nx * wrapi(jb - 2 + q, ny);
                        rd.zk[q] = DIM == 3 ? (long long)nx * ny * wrapi(kb - 2 + q, nz) : 0;
                    }
                    gather5<DIM>(rd, w, w + 3, w + 7, w + 10, w + 14, w + 17, Ep, Bp);
                    for (int dz = 0; dz < nzw; ++dz)
                        for (int dy = 0; dy < 4; ++dy)
                            for (int dx = 0; dx < 4; ++dx)
                                atomicAdd(&rho[rd.xi[dx] + rd.yj[dy] + rd.zk[DIM == 3 ? dz : 2]],
                                          (double)qV * w[3 + dx] * w[10 + dy] * (DIM == 3 ? w[17 + dz] : 1.0f));
                }
            } else {
                float fx[2], Sx[3], fy[2], Sy[3], fz[2], Sz[3];
                form_factor(P.off[0][p], fx, Sx);
                form_factor(P.off[1][p], fy, Sy);
                if (DIM == 3) {
                    form_factor(P.off[2][p], fz, Sz);
                } else {
                    fz[0] = 1.0f; fz[1] = 0.0f; Sz[0] = 0.0f; Sz[1] = 1.0f; Sz[2] = 0.0f;
                }
                if (inr) {
                    ZeroB rd;
                    for (int c = 0; c < 3; ++c) rd.E[c] = sE[c];
                    rd.base = (li + G + FH) + P0 * ((lj + G + FH) + (DIM == 3 ? P1 * (lk + G + FH) : 0));
                    rd.s1 = P0;
                    rd.s2 = P0 * P1;
                    if constexpr (ORD == 4)
                        gather_w1<DIM>(rd, Sx, Sy, Sz, Ep, Bp);
                    else
                        gather<DIM>(rd, fx, Sx, fy, Sy, fz, Sz, Ep, Bp);
                    acc.base = rd.base;
                    const int kz0 = DIM == 3 ? -1 : 0, kz1 = DIM == 3 ? 1 : 0;
#pragma unroll
                    for (int dz = kz0; dz <= kz1; ++dz)
#pragma unroll
                        for (int dy = -1; dy <= 1; ++dy) {
                            const float t = Sy[dy + 1] * Sz[dz + 1];
#pragma unroll
                            for (int dx = -1; dx <= 1; ++dx) acc.add(0, dx, dy, dz, kq * Sx[dx + 1], t);
                        }
                } else {
                    GlobalZeroB rd;
                    for (int c = 0; c < 3; ++c) rd.E[c] = F.E[c];
                    for (int q = 0; q < 4; ++q) {
                        rd.xi[q] = cb + wrapi(i - 1 + q, nx);
                        rd.yj[q] = (long long)nx * wrapi(j - 1 + q, ny);
                        rd.zk[q] = DIM == 3 ? (long long)nx * ny * wrapi(k - 1 + q, nz) : 0;
                    }
                    if constexpr (ORD == 4)
                        gather_w1<DIM>(rd, Sx, Sy, Sz, Ep, Bp);
                    else
                        gather<DIM>(rd, fx, Sx, fy, Sy, fz, Sz, Ep, Bp);
                    const int kz0 = DIM == 3 ? -1 : 0, kz1 = DIM == 3 ? 1 : 0;
                    for (int dz = kz0; dz <= kz1; ++dz)
                        for (int dy = -1; dy <= 1; ++dy)
                            for (int dx = -1; dx <= 1; ++dx)
                                atomicAdd(&rho[rd.xi[dx + 1] + rd.yj[dy + 1] + rd.zk[dz + 1]],
                                          (double)qV * Sx[dx + 1] * Sy[dy + 1] * Sz[dz + 1]);
                }
            }
            const float w0 = P.w[0][p], w1 = P.w[1][p], w2 = P.w[2][p];
            const float ww = w0 * w0 + w1 * w1 + w2 * w2;
            const float gam = sqrtf(ww + c2);
            kahan(0, mp * cl * ww / (gam + cl));
            kahan(1, mp * w0);
            kahan(2, mp * w1);
            kahan(3, mp * w2);
            kahan(4, hqdt * (w0 * Ep[0] + w1 * Ep[1] + w2 * Ep[2]) / gam);
            ++count;
        }
        for (int q = 0; q < 5; ++q) v[q] += (double)ks[q] - (double)kc[q];
        v[5] += (double)count;
        __syncthreads();
        const double rinv = gr.rinv;
        for (int l = threadIdx.x; l < nf; l += blockDim.x) {
            const int h = rh[l], lo = rl[l];
            if ((h | lo) == 0) continue;
            const int lx = l % P0, r = l / P0, ly = r % P1, lz = r / P1;
            const int gx = wrapi(ox - G - FH + lx, nx);
            const int gy = wrapi(oy - G - FH + ly, ny);
            const int gz = DIM == 3 ? wrapi(oz - G - FH + lz, nz) : 0;
            atomicAdd(&rho[cb + gx + (long long)nx * (gy + (long long)ny * gz)], ((double)h * 65536.0 + (double)lo) * rinv);
        }
        __syncthreads();
    }
    block_reduce_store(v, -1, partials + (long long)blockIdx.x * kPartVals);
}

// Cells: residual against the reference, charge, field energies.
// Partial slots: 0 max |r - r_ref|, 1 sum (r - r_ref)^2, 2 charge, 3 sum E^2, 4 sum B^2.
template <int DIM, typename R>
__global__ void __launch_bounds__(kDiagThreads) k_diag_cells(const RunDev *runs, int run, Fields<R> F, const double *rho,
                                                             double *ref, int set_ref, double *partials)
{
    double v[kPartVals] = {0, 0, 0, 0, 0, 0, 0, 0};
    const RunDev rn = runs[run];
    const int nx = rn.n[0], ny = rn.n[1], nz = rn.n[2];
    const long long ncell = (long long)nx * ny * nz;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const double hx = 0.5 * rn.cN[0], hy = 0.5 * rn.cN[1], hz = 0.5 * rn.cN[2];
    for (long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x; l < ncell; l += stride) {
        const int i = (int)(l % nx);
        const long long r = l / nx;
        const int j = (int)(r % ny), k = (int)(r / ny);
        const long long p = rn.cell_base + l;
        const long long pip = p + (i == nx - 1 ? -(nx - 1) : 1), pim = p + (i == 0 ? nx - 1 : -1);
        const long long pjp = p + (long long)nx * (j == ny - 1 ? -(ny - 1) : 1);
        const long long pjm = p + (long long)nx * (j == 0 ? ny - 1 : -1);
        const double ex = F.E[0][p], ey = F.E[1][p], ez = F.E[2][p];
        double div = ((double)F.E[0][pip] - ex) / rn.d[0] + ((double)F.E[1][pjp] - ey) / rn.d[1];
        double bx = (double)F.B[0][p] - hy * (ez - (double)F.E[2][pjm]);
        double by = (double)F.B[1][p] + hx * (ez - (double)F.E[2][pim]);
        double bz = (double)F.B[2][p] - hx * (ey - (double)F.E[1][pim]) + hy * (ex - (double)F.E[0][pjm]);
        if (DIM == 3) {
            const long long pkp = p + (long long)nx * ny * (k == nz - 1 ? -(nz - 1) : 1);
            const long long pkm = p + (long long)nx * ny * (k == 0 ? nz - 1 : -1);
            div += ((double)F.E[2][pkp] - ez) / rn.d[2];
            bx += hz * (ey - (double)F.E[1][pkm]);
            by -= hz * (ex - (double)F.E[0][pkm]);
        }
        const double rt = rho[p] + rn.rho_bg;
        const double res = div - 4.0 * kPi * rt;
        if (set_ref) ref[p] = res;
        const double dr = res - ref[p];
        v[0] = fmax(v[0], fabs(dr));
        v[1] += dr * dr;
        v[2] += rt * rn.V;
        v[3] += ex * ex + ey * ey + ez * ez;
        v[4] += bx * bx + by * by + bz * bz;
    }
    block_reduce_store(v, 0, partials + (long long)blockIdx.x * kPartVals);
}

// One block: fixed-order reduction of the partial slots into result[0..11]:
// kinetic, field_E, field_B, half_step_corr, total, px, py, pz, charge,
// resid_max, resid_rms, n_particles.  Thread t sums the slots of blocks t,
// t + kFinalThreads, ... in order, then a pairwise tree in shared memory
// combines the threads' sums: the order is fixed, so the result is the same
// on every call.
constexpr int kFinalThreads = 256;
__global__ void __launch_bounds__(kFinalThreads) k_diag_final(const double *pp, int np, const double *pc, int nc,
                                                             const RunDev *runs, int run, double *result)
{
    __shared__ double sp[kPartVals][kFinalThreads];
    __shared__ double sc[kPartVals][kFinalThreads];
    const int t = threadIdx.x;
    double s[kPartVals] = {0, 0, 0, 0, 0, 0, 0, 0};
    double c[kPartVals] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int b = t; b < np; b += kFinalThreads)
        for (int q = 0; q < kPartVals; ++q) s[q] += pp[(long long)b * kPartVals + q];
    for (int b = t; b < nc; b += kFinalThreads) {
        c[0] = fmax(c[0], pc[(long long)b * kPartVals + 0]);
        for (int q = 1; q < kPartVals; ++q) c[q] += pc[(long long)b * kPartVals + q];
    }
    for (int q = 0; q < kPartVals; ++q) {
        sp[q][t] = s[q];
        sc[q][t] = c[q];
    }
    __syncthreads();
    for (int h = kFinalThreads / 2; h > 0; h >>= 1) {
        if (t < h) {
            for (int q = 0; q < kPartVals; ++q) {
                sp[q][t] += sp[q][t + h];
                sc[q][t] = q == 0 ? fmax(sc[q][t], sc[q][t + h]) : sc[q][t] + sc[q][t + h];
            }
        }
        __syncthreads();
    }
    if (t == 0) {
        const RunDev rn = runs[run];
        const double ncell = (double)rn.n[0] * rn.n[1] * rn.n[2];
        const double fe = rn.V / (8.0 * kPi);
        double acc[12];
        acc[0] = sp[0][0];
        acc[1] = fe * sc[3][0];
        acc[2] = fe * sc[4][0];
        acc[3] = sp[4][0];
        acc[4] = acc[0] + acc[1] + acc[2] + acc[3];
        acc[5] = sp[1][0];
        acc[6] = sp[2][0];
        acc[7] = sp[3][0];
        acc[8] = sc[2][0];
        acc[9] = sc[0][0];
        acc[10] = sqrt(sc[1][0] / ncell);
        acc[11] = sp[5][0];
        for (int q = 0; q < 12; ++q) result[q] = acc[q];
    }
}

template <int DIM, typename R, int ORD>
static cudaError_t diag_t(cudaStream_t st, const RunDev *runs, int run,
                          const GroupDev *groups, const long long *group_base, int ngroups, long long total,
                          const PoolBuf &P, void *const E[3], void *const B[3], DiagScratch &scr, int set_ref,
                          int np_blocks, int nc_blocks, int *launches, const WorkItem *items, const int *n_items,
                          int halo, size_t items_smem)
{
    Pool<R> pool;
    pool.cell = P.cell;
    pool.id = P.id;
    Fields<R> F;
    for (int c = 0; c < 3; ++c) {
        pool.off[c] = (R *)P.off[c];
        pool.w[c] = (R *)P.w[c];
        F.E[c] = (R *)E[c];
        F.B[c] = (R *)B[c];
        F.J[c] = nullptr;
    }
    int np_items = np_blocks;   // blocks of the particle pass (partial slots filled)
    if (sizeof(R) == 4 && items) {
        Pool<float> pf;
        Fields<float> ff;
        pf.cell = P.cell;
        pf.id = P.id;
        for (int c = 0; c < 3; ++c) {
            pf.off[c] = (float *)P.off[c];
            pf.w[c] = (float *)P.w[c];
            ff.E[c] = (float *)E[c];
            ff.B[c] = (float *)B[c];
            ff.J[c] = nullptr;
        }
        // one wave of resident blocks, each looping over the items: no partial last wave
        int dev = 0, sms = 0, per_sm = 0;
        cudaError_t e;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_diag_items<DIM, ORD>, kDiagThreads,
                                                               items_smem)) != cudaSuccess)
            return e;
        if (per_sm > 0 && sms * per_sm < np_blocks) np_items = sms * per_sm;
        k_diag_items<DIM, ORD><<<np_items, kDiagThreads, items_smem, st>>>(run, items, n_items, groups, runs, pf, ff,
                                                                          halo, scr.rho, scr.partials);
    } else {
        k_diag_particles<DIM, R, ORD><<<np_blocks, kDiagThreads, 0, st>>>(run, total, group_base, ngroups, groups, runs,
                                                                     pool, F, scr.rho, scr.partials);
    }
    k_diag_cells<DIM, R><<<nc_blocks, kDiagThreads, 0, st>>>(runs, run, F, scr.rho, scr.resid_ref, set_ref,
                                                             scr.partials + (long long)np_blocks * kPartVals);
    k_diag_final<<<1, kFinalThreads, 0, st>>>(scr.partials, np_items, scr.partials + (long long)np_blocks * kPartVals,
                                              nc_blocks, runs, run, scr.result);
    *launches += 3;
    return cudaGetLastError();
}

template <int ORD>
static cudaError_t diag_run_o(int dims, int prec, cudaStream_t st, const RunDev *runs, int run,
                              const GroupDev *groups, const long long *group_base, int ngroups, long long total,
                              const PoolBuf &P, void *const E[3], void *const B[3], DiagScratch &scr, int set_ref,
                              int np_blocks, int nc_blocks, int *launches, const WorkItem *items, const int *n_items,
                              int halo, size_t items_smem)
{
    if (dims == 3)
        return prec == 0 ? diag_t<3, double, ORD>(st, runs, run, groups, group_base, ngroups, total, P, E,
                                                  B, scr, set_ref, np_blocks, nc_blocks, launches, nullptr, nullptr,
                                                  halo, 0)
                         : diag_t<3, float, ORD>(st, runs, run, groups, group_base, ngroups, total, P, E,
                                                 B, scr, set_ref, np_blocks, nc_blocks, launches, items, n_items,
                                                 halo, items_smem);
    return prec == 0 ? diag_t<2, double, ORD>(st, runs, run, groups, group_base, ngroups, total, P, E, B,
                                              scr, set_ref, np_blocks, nc_blocks, launches, nullptr, nullptr, halo, 0)
                     : diag_t<2, float, ORD>(st, runs, run, groups, group_base, ngroups, total, P, E, B,
                                             scr, set_ref, np_blocks, nc_blocks, launches, items, n_items, halo,
                                             items_smem);
}

cudaError_t launch_diagnostics_run(int dims, int prec, cudaStream_t st, const RunDev *runs, int run,
                                   long long run_cells, long long cell_base, const GroupDev *groups,
                                   const long long *group_base, int ngroups, long long total, const PoolBuf &P,
                                   void *const E[3], void *const B[3], DiagScratch &scr, int set_ref,
                                   int np_blocks, int nc_blocks, int *launches, const WorkItem *items,
                                   const int *n_items, int halo, const int tile[3], const int pitch[2], int order2)
{
    cudaError_t e = cudaMemsetAsync(scr.rho + cell_base, 0, sizeof(double) * run_cells, st);
    if (e != cudaSuccess) return e;
    const size_t items_smem = diag_items_smem_bytes(dims, tile, halo, pitch, order2);
    if (order2 == 5)
        return diag_run_o<5>(dims, prec, st, runs, run, groups, group_base, ngroups, total, P, E, B, scr,
                             set_ref, np_blocks, nc_blocks, launches, items, n_items, halo, items_smem);
    if (order2 == 4)
        return diag_run_o<4>(dims, prec, st, runs, run, groups, group_base, ngroups, total, P, E, B, scr,
                             set_ref, np_blocks, nc_blocks, launches, items, n_items, halo, items_smem);
    return diag_run_o<3>(dims, prec, st, runs, run, groups, group_base, ngroups, total, P, E, B, scr,
                         set_ref, np_blocks, nc_blocks, launches, items, n_items, halo, items_smem);
}

size_t diag_items_smem_bytes(int dims, const int tile[3], int halo, const int pitch[2], int order2)
{
    const int fh = order2 == 3 ? 1 : 2;
    const long long fe2 = dims == 3 ? tile[2] + 2 * (halo + fh) : 1;
    return (size_t)5 * pitch[0] * pitch[1] * fe2 * sizeof(float);
}

cudaError_t diag_set_smem_limit(int dims, size_t bytes, int order2)
{
    const int b = (int)bytes;
    if (order2 == 5)
        return dims == 3 ? cudaFuncSetAttribute(k_diag_items<3, 5>, cudaFuncAttributeMaxDynamicSharedMemorySize, b)
                         : cudaFuncSetAttribute(k_diag_items<2, 5>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    if (order2 == 4)
        return dims == 3 ? cudaFuncSetAttribute(k_diag_items<3, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, b)
                         : cudaFuncSetAttribute(k_diag_items<2, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    return dims == 3 ? cudaFuncSetAttribute(k_diag_items<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, b)
                     : cudaFuncSetAttribute(k_diag_items<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
}

}  // namespace pic
