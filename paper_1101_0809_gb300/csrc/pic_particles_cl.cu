// pic_particles_cl.cu -- the FP32 fused particle step (Appendix step 2:
// alternating-order gather of Eqs. alphax and betax, the push of Eq. 1, the
// move of Eq. coordscheme and the virtual-path current of Eq. current) for the
// 3D 8x4x4 tile with halo 1, over the cell-lane particle order.
//
// Order (PIC_SORT_CELL_LANES, written by the tile sort): inside a tile the 128
// cells are given lanes 0..127 by descending particle count (ties by the cell's
// index in the tile), and the r-th particle of the cell of lane l (its input
// order among the cell's particles) sits at tile_start + P(r) + l, where
// P(r) = sum_l' min(count_l', r).  Lane l of the kernel's 128-thread block
// therefore walks the particles of one cell, and the 32 lanes of a warp read
// 32 consecutive slots at every step of their walk.
//
// Per lane, the cell is fixed, so two things are done once per lane instead of
// once per particle:
//  - Gather.  Inside a cell each interpolated field component is a polynomial
//    in the particle's offsets (dx, dy, dz): of degree 1 along an axis where
//    the component takes the point values f = (1-d, d) and of degree 2 where it
//    takes the cell integrals S = ((1-d)^2/2, 3/4-(1/2-d)^2, d^2/2) (Sec. 4.5).
//    The lane turns the component's 12 or 18 grid values into the monomial
//    coefficients of that polynomial and evaluates it for every particle by
//    Horner's rule: 84 fused multiply-adds for E and B, no loads.
//  - Deposit.  A particle that stays in its cell along every axis deposits
//    Eq. current on the fixed 54-word stencil of its cell.  The lane sums those
//    contributions in registers (FP32, in the walk order) and adds the 54 sums
//    to the block's exact fixed-point current tile once, at the end of the walk.
// A particle that changes cell deposits on its wider window through the
// per-warp queue (as in k_particles); one that has left the lane's cell since
// the last sort (drift) is put on the tile's drift list and takes the general
// path after the walk: gather from the shared field tile (or the global arrays
// past the halo), push, move and deposit of that particle alone.  Nothing is
// dropped and the arithmetic of every particle is that of the step.
#include "pic_particles.cuh"

namespace pic {

namespace {

constexpr int kT0 = 8, kT1 = 4, kT2 = 4, kG = 1;
constexpr int kCells = kT0 * kT1 * kT2;          // 128: one thread per cell
constexpr int kWarps = kCells / 32;
// shared tiles, unpadded: E and B with a halo of G + 1 = 2 cells, the current
// with G + 2 = 3 (a particle's window reaches two cells from its cell)
constexpr int kFE0 = kT0 + 2 * (kG + 1), kFE1 = kT1 + 2 * (kG + 1), kFE2 = kT2 + 2 * (kG + 1);
constexpr int kJE0 = kT0 + 2 * (kG + 2), kJE1 = kT1 + 2 * (kG + 2), kJE2 = kT2 + 2 * (kG + 2);
constexpr int kNF = kFE0 * kFE1 * kFE2;          // field tile words per component
constexpr int kNJ = kJE0 * kJE1 * kJE2;          // current tile words per component
constexpr int kFS1 = kFE0, kFS2 = kFE0 * kFE1;   // strides of the field tile
constexpr int kJS1 = kJE0, kJS2 = kJE0 * kJE1;   // strides of the current tile

struct ClArgs {
    const long long *tile_start;
    const unsigned char *lane_cell;   // [tile * 128 + lane]: the lane's cell, lx + 8 (ly + 4 lz)
    const int *lane_count;            // [tile * 128 + lane]: its particle count, descending in lane
    int *drift;                       // pool-sized: the drift list of a tile at [tile_start, ...)
    const GroupDev *groups;
    int ngroups;
    const RunDev *runs;
    Pool<float> P;
    Fields<float> F;
    int lg_ppb;                       // log2 of the particles per block the groups' scales assume
    int *err;
};

// Monomial coefficients of one field component inside a cell.  NX, NY, NZ are
// 2 along an axis where the component takes f (grid points 0, 1 of the cell)
// and 3 where it takes S (points -1, 0, 1).  Per axis, the weighted sum of the
// grid values v is v0 + d (v1 - v0) for f, and
// (v0 + v1)/2 + d (v1 - v0) + d^2 (v0/2 - v1 + v2/2) for S; applying these maps
// along x, y and z gives c[i][j][k], the coefficient of dx^i dy^j dz^k.
template <int N>
__device__ __forceinline__ void to_monomials(float &a, float &b, float &c)
{
    if (N == 2) {
        b = b - a;
    } else {
        const float c0 = 0.5f * (a + b), c1 = b - a, c2 = fmaf(0.5f, a + c, -b);
        a = c0;
        b = c1;
        c = c2;
    }
}

template <int NX, int NY, int NZ>
__device__ __forceinline__ void poly_coeffs(const float *f, float *c)
{
    constexpr int sx = NX == 3 ? -1 : 0, sy = NY == 3 ? -1 : 0, sz = NZ == 3 ? -1 : 0;
    float v[NX][NY][NZ];
#pragma unroll
    for (int a = 0; a < NX; ++a)
#pragma unroll
        for (int b = 0; b < NY; ++b)
#pragma unroll
            for (int k = 0; k < NZ; ++k) v[a][b][k] = f[(a + sx) + kFS1 * (b + sy) + kFS2 * (k + sz)];
    float dummy = 0.f;
#pragma unroll
    for (int b = 0; b < NY; ++b)
#pragma unroll
        for (int k = 0; k < NZ; ++k) to_monomials<NX>(v[0][b][k], v[1][b][k], NX == 3 ? v[NX - 1][b][k] : dummy);
#pragma unroll
    for (int a = 0; a < NX; ++a)
#pragma unroll
        for (int k = 0; k < NZ; ++k) to_monomials<NY>(v[a][0][k], v[a][1][k], NY == 3 ? v[a][NY - 1][k] : dummy);
#pragma unroll
    for (int a = 0; a < NX; ++a)
#pragma unroll
        for (int b = 0; b < NY; ++b) to_monomials<NZ>(v[a][b][0], v[a][b][1], NZ == 3 ? v[a][b][NZ - 1] : dummy);
#pragma unroll
    for (int a = 0; a < NX; ++a)
#pragma unroll
        for (int b = 0; b < NY; ++b)
#pragma unroll
            for (int k = 0; k < NZ; ++k) c[(a * NY + b) * NZ + k] = v[a][b][k];
}

template <int NX, int NY, int NZ>
__device__ __forceinline__ float poly_eval(const float *c, float dx, float dy, float dz)
{
    float r[NX];
#pragma unroll
    for (int a = 0; a < NX; ++a) {
        float s[NY];
#pragma unroll
        for (int b = 0; b < NY; ++b) {
            float h = c[(a * NY + b) * NZ + NZ - 1];
#pragma unroll
            for (int k = NZ - 2; k >= 0; --k) h = fmaf(h, dz, c[(a * NY + b) * NZ + k]);
            s[b] = h;
        }
        float h = s[NY - 1];
#pragma unroll
        for (int b = NY - 2; b >= 0; --b) h = fmaf(h, dy, s[b]);
        r[a] = h;
    }
    float e = r[NX - 1];
#pragma unroll
    for (int a = NX - 2; a >= 0; --a) e = fmaf(e, dx, r[a]);
    return e;
}

// The push of the Appendix (Eq. 1) in FP32 with the hardware reciprocal square
// root and a fast reciprocal: e = (q dt/2m) E; w~ = w + e;
// b = (q dt/2m) B / sqrt(w~^2 + c^2); w_n = w~ + w~ x b;
// w' = w~ + e + 2 (w_n x b)/(1 + b^2).
__device__ __forceinline__ void boris_f32(float w[3], const float Ep[3], const float Bp[3], float hq, float c2)
{
    const float e0 = hq * Ep[0], e1 = hq * Ep[1], e2 = hq * Ep[2];
    const float t0 = w[0] + e0, t1 = w[1] + e1, t2 = w[2] + e2;
    const float s = hq * rsqrtf(fmaf(t0, t0, fmaf(t1, t1, fmaf(t2, t2, c2))));
    const float b0 = s * Bp[0], b1 = s * Bp[1], b2 = s * Bp[2];
    const float n0 = t0 + (t1 * b2 - t2 * b1);
    const float n1 = t1 + (t2 * b0 - t0 * b2);
    const float n2 = t2 + (t0 * b1 - t1 * b0);
    const float f = __fdividef(2.0f, 1.0f + fmaf(b0, b0, fmaf(b1, b1, b2 * b2)));
    w[0] = t0 + e0 + f * (n1 * b2 - n2 * b1);
    w[1] = t1 + e1 + f * (n2 * b0 - n0 * b2);
    w[2] = t2 + e2 + f * (n0 * b1 - n1 * b0);
}

// Eq. current's window of an axis along which the particle stayed in its cell
// (offsets d0 -> d1, cells -1..1): Pp = dF(x^{n+1}) + dF(x^n) and
// Pm = dF(x^{n+1}) - dF(x^n) of the l_a = 1 1/2 cell integrals, and the face
// sums D0 = Pm0, D1 = Pm0 + Pm1 = -Pm2.  Pp0 = ((1-d0)^2 + (1-d1)^2)/2,
// Pp2 = (d0^2 + d1^2)/2, Pp1 = 2 - Pp0 - Pp2 (the cell integrals sum to one);
// Pm in the factored form of the differences with h = (d1 - d0)/2 and
// s = d0 + d1: Pm0 = h (s - 2), Pm2 = h s, Pm1 = -(Pm0 + Pm2), which is exactly
// zero for a particle at rest.
struct StillWin {
    float pp[3], pm[3], d[2];
};
__device__ __forceinline__ void still_window(float d0, float d1, StillWin &a)
{
    const float e0 = 1.0f - d0, e1 = 1.0f - d1;
    a.pp[0] = 0.5f * fmaf(e0, e0, e1 * e1);
    a.pp[2] = 0.5f * fmaf(d0, d0, d1 * d1);
    a.pp[1] = (2.0f - a.pp[0]) - a.pp[2];
    const float h = 0.5f * (d1 - d0), sm = d0 + d1;
    a.pm[0] = h * (sm - 2.0f);
    a.pm[2] = h * sm;
    a.pm[1] = -(a.pm[0] + a.pm[2]);
    a.d[0] = a.pm[0];
    a.d[1] = -a.pm[2];
}

// Deposits the queue entries [first, first + 32) of a warp whose lanes have
// `on` (old offsets, new offsets, and (base << 8) | shifts + 1 per entry) into
// the shared fixed-point current tile, Eq. current on each entry's window.
// Out of line: it is called from three places and its fully unrolled window
// is the largest code of the kernel.
__device__ __noinline__ void drain_queue(const float *qv, const int *qs, int first, bool on, int *jh0, int *jh1,
                                         int *jh2, int *jl0, int *jl1, int *jl2, float k0, float k1, float k2)
{
    const int slot = first + (threadIdx.x & 31);
    float d0 = 0.f, d1 = 0.f, d2 = 0.f, f0 = 0.f, f1 = 0.f, f2 = 0.f;
    int code = 1 | (1 << 2) | (1 << 4);
    if (on) {
        d0 = qv[0 * kQueueCap + slot];
        d1 = qv[1 * kQueueCap + slot];
        d2 = qv[2 * kQueueCap + slot];
        f0 = qv[3 * kQueueCap + slot];
        f1 = qv[4 * kQueueCap + slot];
        f2 = qv[5 * kQueueCap + slot];
        code = qs[slot];
    }
    const int q0 = (code & 3) - 1, q1 = ((code >> 2) & 3) - 1, q2 = ((code >> 4) & 3) - 1;
    const int full = (__any_sync(0xffffffffu, q0 != 0) ? 1 : 0) | (__any_sync(0xffffffffu, q1 != 0) ? 2 : 0) |
                     (__any_sync(0xffffffffu, q2 != 0) ? 4 : 0);
    if (on) {
        AxisWin<float> X, Y, Z;
        axis_window(d0, f0, q0, X);
        axis_window(d1, f1, q1, Y);
        axis_window(d2, f2, q2, Z);
        FixedAcc acc;
        acc.hi[0] = jh0; acc.hi[1] = jh1; acc.hi[2] = jh2;
        acc.lo[0] = jl0; acc.lo[1] = jl1; acc.lo[2] = jl2;
        acc.base = code >> 8;
        acc.s1 = kJS1;
        acc.s2 = kJS2;
        const float kf[3] = {k0, k1, k2};
        deposit<3>(acc, X, Y, Z, kf, 0.f, full);
    }
}

// Fixed-point split of a lane's summed contribution kp * t for the current
// tile: hi = rint(kp t / 2^16) and lo = rint(kp t - 2^16 hi), with the product
// formed exactly inside the fused multiply-add.  Unlike FixedAcc (whose single
// contributions stay below 2^38 and can use the magic-number rounding), a sum
// over a cell's particles may reach the tile's bound of 2^46, so the rounding
// to integers is done by conversion instructions.
__device__ __forceinline__ void add_sum(int *hi, int *lo, int idx, float kp, float t)
{
    const float hf = rintf((kp * (1.0f / 65536.0f)) * t);
    const float lf = fmaf(kp, t, -65536.0f * hf);
    atomicAdd(hi + idx, __float2int_rn(hf));
    atomicAdd(lo + idx, __float2int_rn(lf));
}

__global__ void __launch_bounds__(kCells, 3) k_particles_cl(const ClArgs A)
{
    const int t = blockIdx.x;
    const long long b0 = A.tile_start[t], e0 = A.tile_start[t + 1];
    if (e0 <= b0) return;
    int lo = 0, hi = A.ngroups;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (A.groups[mid].tile_base <= t) lo = mid; else hi = mid;
    }
    const GroupDev gr = A.groups[lo];
    const RunDev rn = A.runs[gr.run];
    const int lt = t - gr.tile_base;
    const int ox = (lt % rn.ntile[0]) * kT0;
    const int oy = ((lt / rn.ntile[0]) % rn.ntile[1]) * kT1;
    const int oz = (lt / (rn.ntile[0] * rn.ntile[1])) * kT2;
    const int nx = rn.n[0], ny = rn.n[1], nz = rn.n[2];
    const long long cb = rn.cell_base;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    float *sE[3], *sB[3];
    int *sJh[3], *sJl[3];
    {
        float *f = reinterpret_cast<float *>(g_smem);
        int *j = reinterpret_cast<int *>(g_smem + 6 * (size_t)kNF * sizeof(float));
        for (int c = 0; c < 3; ++c) {
            sE[c] = f + c * kNF;
            sB[c] = f + (3 + c) * kNF;
            sJh[c] = j + c * kNJ;
            sJl[c] = j + (3 + c) * kNJ;
        }
    }
    unsigned char *after = g_smem + 6 * (size_t)kNF * sizeof(float) + 6 * (size_t)kNJ * sizeof(int);
    float *qv = reinterpret_cast<float *>(after) + warp * kQueueCap * kQueueVals;
    int *qs = reinterpret_cast<int *>(after + (size_t)kWarps * kQueueCap * kQueueVals * sizeof(float)) +
              warp * kQueueCap;
    int *s_cnt = reinterpret_cast<int *>(after + (size_t)kWarps * kQueueCap * (kQueueVals * sizeof(float) +
                                                                                  sizeof(int)));
    int *s_ndrift = s_cnt + kCells;

    // stage E and B of the tile with a halo of 2 cells; clear the current tile
    for (int l = tid; l < kNF; l += kCells) {
        const int lx = l % kFE0, r = l / kFE0, ly = r % kFE1, lz = r / kFE1;
        const int gx = wrapi(ox - 2 + lx, nx), gy = wrapi(oy - 2 + ly, ny), gz = wrapi(oz - 2 + lz, nz);
        const long long gi = cb + gx + (long long)nx * (gy + (long long)ny * gz);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            sE[c][l] = A.F.E[c][gi];
            sB[c][l] = A.F.B[c][gi];
        }
    }
    for (int l = tid; l < 6 * kNJ; l += kCells) sJh[0][l] = 0;
    const int my_cnt = A.lane_count[(long long)t * kCells + tid];
    s_cnt[tid] = my_cnt;
    if (tid == 0) *s_ndrift = 0;
    __syncthreads();

    // this tile's scale of the fixed-point current: the groups' scales assume
    // at most 2^lg_ppb particles per block; a fuller tile takes 2^-k of it so
    // that the tile's sums keep within 2^46 (exact powers of two)
    int k = 0;
    while ((e0 - b0) > (1LL << (A.lg_ppb + k))) ++k;
    const float tscale = ldexpf(1.0f, -k);
    const float kfs[3] = {gr.kfsf[0] * tscale, gr.kfsf[1] * tscale, gr.kfsf[2] * tscale};
    const float jinv = gr.jinv / tscale;
    const float hq = gr.hqf, cl = rn.cf, c2 = cl * cl;
    const float cN0 = rn.cNf[0], cN1 = rn.cNf[1], cN2 = rn.cNf[2];

    // ---- the lane's cell -------------------------------------------------------
    const int lc = A.lane_cell[(long long)t * kCells + tid];
    const int lx = lc % kT0, ly = (lc / kT0) % kT1, lz = lc / (kT0 * kT1);
    const int gi = ox + lx, gj = oy + ly, gk = oz + lz;      // inside the grid when my_cnt > 0
    const int cellG = gi + nx * (gj + ny * gk);
    const int fbase = (lx + 2) + kFS1 * ((ly + 2) + kFE1 * (lz + 2));
    const int jbase = (lx + 3) + kJS1 * ((ly + 3) + kJE1 * (lz + 3));

    float cex[18], cey[18], cez[18], cbx[12], cby[12], cbz[12];
    poly_coeffs<2, 3, 3>(sE[0] + fbase, cex);
    poly_coeffs<3, 2, 3>(sE[1] + fbase, cey);
    poly_coeffs<3, 3, 2>(sE[2] + fbase, cez);
    poly_coeffs<3, 2, 2>(sB[0] + fbase, cbx);
    poly_coeffs<2, 3, 2>(sB[1] + fbase, cby);
    poly_coeffs<2, 2, 3>(sB[2] + fbase, cbz);

    // Current sums of the particles that stay in the cell, as moments.  Per axis
    // (offsets d0 -> d1, h = d1 - d0, s = d0 + d1, A = d0^2 + d1^2) the window of
    // Eq. current is linear in a few monomials: Pp = u1 + s us + A uA,
    // Pm = h us + h s uA and the face sums D = h a0 + h s a1, with the fixed
    // vectors u1 = (1, 1, 0), us = (-1, 1, 0), uA = (1/2, -1, 1/2) over the cells
    // -1..1 and a0 = (-1, 0), a1 = (1/2, -1/2) over the faces 0, 1.  So the
    // lane sums, per particle, products of those monomials: mt[i][j][k] for the
    // Pm Pm D terms (shared by the three components), and mx (D_x Pp_y Pp_z),
    // my, mz; the 54 stencil words follow from them once, at the flush.
    float mt[2][2][2], mx[2][3][3], my[2][3][3], mz[2][3][3];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                mx[i][j][k] = 0.f;
                my[i][j][k] = 0.f;
                mz[i][j][k] = 0.f;
                if (j < 2 && k < 2) mt[i][j][k] = 0.f;
            }

    int qn = 0;   // entries in this warp's deposit queue (warp-uniform)
    auto drain = [&](int first, bool on) {
        drain_queue(qv, qs, first, on, sJh[0], sJh[1], sJh[2], sJl[0], sJl[1], sJl[2], kfs[0], kfs[1], kfs[2]);
    };
    // queues a particle that changed cell (warp-uniform call)
    auto enqueue = [&](bool enq, float a0, float a1, float a2, float n0, float n1, float n2, int base, int s0,
                       int s1, int s2) {
        const unsigned qm = __ballot_sync(0xffffffffu, enq);
        if (enq) {
            const int slot = qn + __popc(qm & ((1u << lane) - 1u));
            qv[0 * kQueueCap + slot] = a0;
            qv[1 * kQueueCap + slot] = a1;
            qv[2 * kQueueCap + slot] = a2;
            qv[3 * kQueueCap + slot] = n0;
            qv[4 * kQueueCap + slot] = n1;
            qv[5 * kQueueCap + slot] = n2;
            qs[slot] = (base << 8) | (s0 + 1) | ((s1 + 1) << 2) | ((s2 + 1) << 4);
        }
        qn += __popc(qm);
        if (qn >= 32) {
            __syncwarp();
            qn -= 32;
            drain(qn, true);
            __syncwarp();
        }
    };

    // ---- the walk: lane tid takes the r-th particle of its cell ----------------
    const int wmax = s_cnt[warp * 32];    // counts descend with the lane
    int act = 0;                          // lanes of the tile with more than r particles
    {
        int a = 0, b = kCells;            // first lane with count 0
        while (a < b) {
            const int m = (a + b) >> 1;
            if (s_cnt[m] > 0) a = m + 1; else b = m;
        }
        act = a;
    }
    long long prow = 0;                   // P(r)
    // the state of the lane's next particle, loaded one row ahead of its use
    int fc = -1;
    float fo0 = 0.f, fo1 = 0.f, fo2 = 0.f, fw0 = 0.f, fw1 = 0.f, fw2 = 0.f;
    auto fetch = [&](long long q, bool on) {
        if (on) {
            fc = A.P.cell[q];
            fo0 = A.P.off[0][q];
            fo1 = A.P.off[1][q];
            fo2 = A.P.off[2][q];
            fw0 = A.P.w[0][q];
            fw1 = A.P.w[1][q];
            fw2 = A.P.w[2][q];
        }
    };
    fetch(b0 + tid, my_cnt > 0);
    for (int r = 0; r < wmax; ++r) {
        const bool on = r < my_cnt;
        const long long p = b0 + prow + tid;
        const int cell0 = fc;
        const float o0 = fo0, o1 = fo1, o2 = fo2;
        float w[3] = {fw0, fw1, fw2};
        // the next row of the walk, and its loads
        prow += act;
        while (act > 0 && s_cnt[act - 1] <= r + 1) --act;
        fetch(b0 + prow + tid, r + 1 < my_cnt);
        const bool mine = on && cell0 == cellG;
        const unsigned dm = __ballot_sync(0xffffffffu, on && !mine);
        if (dm) {   // a particle that left the lane's cell since the sort: to the drift list
            int base = 0;
            if (lane == 0) base = atomicAdd(s_ndrift, __popc(dm));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (on && !mine) A.drift[b0 + base + __popc(dm & ((1u << lane) - 1u))] = (int)(p - b0);
        }
        bool enq = false;
        float n0 = o0, n1 = o1, n2 = o2;
        int s0 = 0, s1 = 0, s2 = 0;
        if (mine) {
            float Ep[3], Bp[3];
            Ep[0] = poly_eval<2, 3, 3>(cex, o0, o1, o2);
            Ep[1] = poly_eval<3, 2, 3>(cey, o0, o1, o2);
            Ep[2] = poly_eval<3, 3, 2>(cez, o0, o1, o2);
            Bp[0] = poly_eval<3, 2, 2>(cbx, o0, o1, o2);
            Bp[1] = poly_eval<2, 3, 2>(cby, o0, o1, o2);
            Bp[2] = poly_eval<2, 2, 3>(cbz, o0, o1, o2);
            boris_f32(w, Ep, Bp, hq, c2);
            if (!finite3(w[0], w[1], w[2])) {
                atomicOr(A.err, ERR_NONFINITE);   // the particle keeps x^n and adds no current
            } else {
                const float ig = rsqrtf(fmaf(w[0], w[0], fmaf(w[1], w[1], fmaf(w[2], w[2], c2))));
                s0 = renormalize(o0, w[0] * ig * cN0, n0);
                s1 = renormalize(o1, w[1] * ig * cN1, n1);
                s2 = renormalize(o2, w[2] * ig * cN2, n2);
                const int i1 = wrapi(gi + s0, nx), j1 = wrapi(gj + s1, ny), k1 = wrapi(gk + s2, nz);
                A.P.cell[p] = i1 + nx * (j1 + ny * k1);
                A.P.off[0][p] = n0;
                A.P.off[1][p] = n1;
                A.P.off[2][p] = n2;
                A.P.w[0][p] = w[0];
                A.P.w[1][p] = w[1];
                A.P.w[2][p] = w[2];
                if ((s0 | s1 | s2) == 0) {
                    // the fixed stencil (Eq. current with three-cell windows), as moments
                    float al[3][2], sv[3], av[3];
                    {
                        const float d0[3] = {o0, o1, o2}, d1[3] = {n0, n1, n2};
#pragma unroll
                        for (int x = 0; x < 3; ++x) {
                            const float h = d1[x] - d0[x];
                            sv[x] = d0[x] + d1[x];
                            av[x] = fmaf(d0[x], d0[x], d1[x] * d1[x]);
                            al[x][0] = h;
                            al[x][1] = h * sv[x];
                        }
                    }
#pragma unroll
                    for (int i = 0; i < 2; ++i)
#pragma unroll
                        for (int j = 0; j < 2; ++j) {
                            const float xy = al[0][i] * al[1][j];
#pragma unroll
                            for (int k = 0; k < 2; ++k) mt[i][j][k] = fmaf(xy, al[2][k], mt[i][j][k]);
                        }
                    // products of the Pp monomials (1, s, A) of two axes
                    auto pp2 = [&](int u, int v, float m[3][3]) {
                        const float bu[3] = {1.0f, sv[u], av[u]}, bv[3] = {1.0f, sv[v], av[v]};
#pragma unroll
                        for (int j = 0; j < 3; ++j)
#pragma unroll
                            for (int k = 0; k < 3; ++k) m[j][k] = bu[j] * bv[k];
                    };
                    float pyz[3][3], pxz[3][3], pxy[3][3];
                    pp2(1, 2, pyz);
                    pp2(0, 2, pxz);
                    pp2(0, 1, pxy);
#pragma unroll
                    for (int i = 0; i < 2; ++i)
#pragma unroll
                        for (int j = 0; j < 3; ++j)
#pragma unroll
                            for (int k = 0; k < 3; ++k) {
                                mx[i][j][k] = fmaf(al[0][i], pyz[j][k], mx[i][j][k]);
                                my[i][j][k] = fmaf(al[1][i], pxz[j][k], my[i][j][k]);
                                mz[i][j][k] = fmaf(al[2][i], pxy[j][k], mz[i][j][k]);
                            }
                } else {
                    enq = true;
                }
            }
        }
        enqueue(enq, o0, o1, o2, n0, n1, n2, jbase, s0, s1, s2);
    }

    // ---- the lane's sums into the current tile ---------------------------------
    // N[i][j][k] = M[i][j][k] plus, where both cell factors are Pm monomials,
    // a third of the shared triple moment; then the monomial vectors are laid
    // on the faces (a0, a1) and cells (u1, us, uA) of the stencil.
    if (my_cnt > 0) {
        const float third = 1.0f / 3.0f;
        auto words = [&](const float m[2][3][3], int comp) {
            float nm[2][3][3];
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j)
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        float t = m[i][j][k];
                        if (j > 0 && k > 0) {
                            const float tri = comp == 0 ? mt[i][j - 1][k - 1]
                                                        : (comp == 1 ? mt[j - 1][i][k - 1] : mt[j - 1][k - 1][i]);
                            t = fmaf(third, tri, t);
                        }
                        nm[i][j][k] = t;
                    }
            // monomials -> cells along k, then j; -> faces along i
            float cj[2][3][3];
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    const float a = nm[i][j][0], b = nm[i][j][1], c = nm[i][j][2];
                    nm[i][j][0] = fmaf(0.5f, c, a - b);
                    nm[i][j][1] = (a + b) - c;
                    nm[i][j][2] = 0.5f * c;
                }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const float a = nm[i][0][k], b = nm[i][1][k], c = nm[i][2][k];
                    cj[i][0][k] = fmaf(0.5f, c, a - b);
                    cj[i][1][k] = (a + b) - c;
                    cj[i][2][k] = 0.5f * c;
                }
#pragma unroll
            for (int j = 0; j < 3; ++j)
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const float a = cj[0][j][k], b = cj[1][j][k];
                    const float f0 = fmaf(0.5f, b, -a), f1 = -0.5f * b;
                    // component comp: the face axis is comp; j and k run over the
                    // other two axes in increasing order
                    const int dj = j - 1, dk = k - 1;
                    int i0, i1;
                    if (comp == 0) {
                        i0 = jbase + kJS1 * dj + kJS2 * dk;
                        i1 = i0 + 1;
                    } else if (comp == 1) {
                        i0 = jbase + dj + kJS2 * dk;
                        i1 = i0 + kJS1;
                    } else {
                        i0 = jbase + dj + kJS1 * dk;
                        i1 = i0 + kJS2;
                    }
                    add_sum(sJh[comp], sJl[comp], i0, kfs[comp], f0);
                    add_sum(sJh[comp], sJl[comp], i1, kfs[comp], f1);
                }
        };
        words(mx, 0);
        words(my, 1);
        words(mz, 2);
    }
    __syncthreads();   // the drift list is complete

    // ---- drifted particles: the general path, one per thread ------------------
    const int ndrift = *s_ndrift;
    unsigned ran_past = 0;   // particles past the tile's halo (the sort policy's measure)
    for (int d0 = warp * 32; d0 < ndrift; d0 += kCells) {
        const int dk = d0 + lane;
        const bool valid = dk < ndrift;
        bool inr = false, enq = false;
        int s0 = 0, s1 = 0, s2 = 0, base = 0;
        float o0 = 0.f, o1 = 0.f, o2 = 0.f, n0 = 0.f, n1 = 0.f, n2 = 0.f;
        if (valid) {
            const long long p = b0 + A.drift[b0 + dk];
            const int cell0 = A.P.cell[p];
            o0 = A.P.off[0][p];
            o1 = A.P.off[1][p];
            o2 = A.P.off[2][p];
            float w[3] = {A.P.w[0][p], A.P.w[1][p], A.P.w[2][p]};
            const int rest = divu31(cell0, rn.div_nx);
            const int i = cell0 - rest * nx;
            const int kk = divu31(rest, rn.div_ny);
            const int j = rest - kk * ny;
            const int li = local_coord(i, ox, kT0, kG, nx);
            const int lj = local_coord(j, oy, kT1, kG, ny);
            const int lk = local_coord(kk, oz, kT2, kG, nz);
            inr = li >= -kG && li < kT0 + kG && lj >= -kG && lj < kT1 + kG && lk >= -kG && lk < kT2 + kG;
            float fx[2], Sx[3], fy[2], Sy[3], fz[2], Sz[3];
            form_factor(o0, fx, Sx);
            form_factor(o1, fy, Sy);
            form_factor(o2, fz, Sz);
            float Ep[3], Bp[3];
            if (inr) {
                SmemReader<float> rd;
                for (int c = 0; c < 3; ++c) { rd.E[c] = sE[c]; rd.B[c] = sB[c]; }
                rd.base = (li + 2) + kFS1 * ((lj + 2) + kFE1 * (lk + 2));
                rd.s1 = kFS1;
                rd.s2 = kFS2;
                gather<3>(rd, fx, Sx, fy, Sy, fz, Sz, Ep, Bp);
            } else {
                float w6[15] = {fx[0], fx[1], Sx[0], Sx[1], Sx[2], fy[0], fy[1], Sy[0], Sy[1], Sy[2],
                                fz[0], fz[1], Sz[0], Sz[1], Sz[2]};
                gather_global<3, float>(A.F, cb, i, j, kk, nx, ny, nz, w6, Ep, Bp);
            }
            boris_f32(w, Ep, Bp, hq, c2);
            if (!finite3(w[0], w[1], w[2])) {
                atomicOr(A.err, ERR_NONFINITE);
            } else {
                const float ig = rsqrtf(fmaf(w[0], w[0], fmaf(w[1], w[1], fmaf(w[2], w[2], c2))));
                s0 = renormalize(o0, w[0] * ig * cN0, n0);
                s1 = renormalize(o1, w[1] * ig * cN1, n1);
                s2 = renormalize(o2, w[2] * ig * cN2, n2);
                const int i1 = wrapi(i + s0, nx), j1 = wrapi(j + s1, ny), k1 = wrapi(kk + s2, nz);
                A.P.cell[p] = i1 + nx * (j1 + ny * k1);
                A.P.off[0][p] = n0;
                A.P.off[1][p] = n1;
                A.P.off[2][p] = n2;
                A.P.w[0][p] = w[0];
                A.P.w[1][p] = w[1];
                A.P.w[2][p] = w[2];
                if (inr) {
                    base = (li + 3) + kJS1 * ((lj + 3) + kJE1 * (lk + 3));
                    enq = true;   // any window, through the queue
                } else {
                    AxisWin<float> win[3];
                    axis_window(o0, n0, s0, win[0]);
                    axis_window(o1, n1, s1, win[1]);
                    axis_window(o2, n2, s2, win[2]);
                    const float kf[3] = {gr.kff[0], gr.kff[1], gr.kff[2]};
                    deposit_global<3, float>(A.F, cb, i, j, kk, nx, ny, nz, win, kf, 0.f,
                                             (s0 != 0 ? 1 : 0) | (s1 != 0 ? 2 : 0) | (s2 != 0 ? 4 : 0));
                }
            }
        }
        const unsigned pm = __ballot_sync(0xffffffffu, valid && !inr);
        if (lane == 0) ran_past += __popc(pm);
        enqueue(enq, o0, o1, o2, n0, n1, n2, base, s0, s1, s2);
    }
    if (qn > 0) {
        __syncwarp();
        drain(0, lane < qn);
    }
    if (lane == 0 && ran_past) atomicAdd(reinterpret_cast<unsigned *>(A.err) + 1, ran_past);

    // ---- the current tile into J ---------------------------------------------
    __syncthreads();
    for (int l = tid; l < kNJ; l += kCells) {
        const int jx = l % kJE0, r = l / kJE0, jy = r % kJE1, jz = r / kJE1;
        const int gx = wrapi(ox - 3 + jx, nx), gy = wrapi(oy - 3 + jy, ny), gz = wrapi(oz - 3 + jz, nz);
        const long long gidx = cb + gx + (long long)nx * (gy + (long long)ny * gz);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const int h = sJh[c][l], q = sJl[c][l];
            if ((h | q) != 0) atomicAdd(&A.F.J[c][gidx], fmaf((float)h, 65536.0f, (float)q) * jinv);
        }
    }
}

}  // namespace

size_t particles_cl_smem_bytes()
{
    return 6 * (size_t)kNF * sizeof(float) + 6 * (size_t)kNJ * sizeof(int) +
           (size_t)kWarps * kQueueCap * (kQueueVals * sizeof(float) + sizeof(int)) + (kCells + 1) * sizeof(int);
}

cudaError_t particles_cl_set_smem_limit()
{
    return cudaFuncSetAttribute(k_particles_cl, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)particles_cl_smem_bytes());
}

bool particles_cl_applies(int dims, int prec, int order2, const int tile[3], int halo)
{
    return dims == 3 && prec != 0 && order2 == 3 && tile[0] == kT0 && tile[1] == kT1 && tile[2] == kT2 &&
           halo == kG;
}

cudaError_t launch_particles_cl(cudaStream_t st, int total_tiles, const long long *tile_start,
                                const unsigned char *lane_cell, const int *lane_count, int *drift,
                                const GroupDev *groups, int ngroups, const RunDev *runs, const PoolBuf &P,
                                void *const E[3], void *const B[3], void *const J[3], int ppb, int *err)
{
    if (total_tiles <= 0) return cudaSuccess;
    ClArgs a;
    a.tile_start = tile_start;
    a.lane_cell = lane_cell;
    a.lane_count = lane_count;
    a.drift = drift;
    a.groups = groups;
    a.ngroups = ngroups;
    a.runs = runs;
    a.P.cell = P.cell;
    a.P.id = P.id;
    for (int c = 0; c < 3; ++c) {
        a.P.off[c] = static_cast<float *>(P.off[c]);
        a.P.w[c] = static_cast<float *>(P.w[c]);
        a.F.E[c] = static_cast<float *>(E[c]);
        a.F.B[c] = static_cast<float *>(B[c]);
        a.F.J[c] = static_cast<float *>(J[c]);
    }
    int lg = 0;
    while ((1 << lg) < ppb) ++lg;
    a.lg_ppb = lg;
    a.err = err;
    k_particles_cl<<<(unsigned)total_tiles, kCells, particles_cl_smem_bytes(), st>>>(a);
    return cudaGetLastError();
}

}  // namespace pic
