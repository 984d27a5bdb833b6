// pic_adjoint.cu -- discrete adjoint of one time step (reverse mode of the step
// of the paper's Appendix), for gradients of a loss of the final state with
// respect to the initial positions and momenta.
//
// Forward step at level n: B1 = B - (1/2) C_B E; per particle: gather E and B1
// at x^n, push, move, deposit J; B2 = B1 - (1/2) C_B E; E' = E - 4 pi dt J + C_E B2.
// Reverse: transpose of the E step (lamJ = -4 pi dt lamE, lamB += C_E^T lamE),
// of the second B half step (lamE += (-(1/2) C_B)^T lamB), of every particle
// (gather of lamJ over the particle's current window, hand-derived reverse of the
// deposit, move and push, scatter of the gather's transpose into lamE and lamB1),
// and of the first B half step.  The particle's intermediate quantities are
// recomputed from the state at level n, in the same arithmetic as the forward
// kernel (including the offset renormalization).  The particle adjoints are
// indexed by group base + particle id, i.e. in each species' load order.
// The particle part runs over the last tile sort's work items with the item's
// E, B1 and lambda_J in shared memory (k_particles_adj_tiled), or untiled over
// the pool with every read global (k_particles_adj); the arithmetic is the same.
#include "pic_particles.cuh"

namespace pic {

template <typename R>
struct AdjArgs {
    const RunDev *runs;
    const GroupDev *groups;
    const long long *group_base;
    int ngroups;
    long long total;
    Pool<R> P;
    const R *E[3];
    const R *B1[3];
    const R *lamJ[3];
    R *lamE[3];
    R *lamB1[3];
    R *lamx[3];
    R *lamw[3];
    // FP32 tiled form: largest |lambda| of a gathered field value seen by the
    // previous launch (bits of a non-negative float; 0: none yet) and the word
    // this launch records its own into
    const unsigned *lam_prev;
    unsigned *lam_cur;
};

template <typename R>
__device__ __forceinline__ void form_factor_d(R d, R df[2], R dS[3])
{
    df[0] = R(-1);
    df[1] = R(1);
    dS[0] = d - R(1);
    dS[1] = R(1) - R(2) * d;
    dS[2] = d;
}

// Placed old/new weights of one axis on the deposit's 4-cell window (same
// placement as axis_window) and their derivatives with respect to the old and
// new offsets.
template <typename R>
struct AxisWinAdj {
    R o[4], n[4], dO[4], dN[4];
};

template <typename R>
__device__ __forceinline__ void axis_window_adj(R d0, R d1, int s, AxisWinAdj<R> &a)
{
    R f[2], S0[3], S1[3], df[2], dS0[3], dS1[3];
    form_factor(d0, f, S0);
    form_factor(d1, f, S1);
    form_factor_d(d0, df, dS0);
    form_factor_d(d1, df, dS1);
    const bool neg = s < 0, pos = s > 0;
    a.o[0] = neg ? R(0) : S0[0];  a.dO[0] = neg ? R(0) : dS0[0];
    a.o[1] = neg ? S0[0] : S0[1]; a.dO[1] = neg ? dS0[0] : dS0[1];
    a.o[2] = neg ? S0[1] : S0[2]; a.dO[2] = neg ? dS0[1] : dS0[2];
    a.o[3] = neg ? S0[2] : R(0);  a.dO[3] = neg ? dS0[2] : R(0);
    a.n[0] = pos ? R(0) : S1[0];  a.dN[0] = pos ? R(0) : dS1[0];
    a.n[1] = pos ? S1[0] : S1[1]; a.dN[1] = pos ? dS1[0] : dS1[1];
    a.n[2] = pos ? S1[1] : S1[2]; a.dN[2] = pos ? dS1[1] : dS1[2];
    a.n[3] = pos ? S1[2] : R(0);  a.dN[3] = pos ? dS1[2] : R(0);
}

// Wrapped run-local offsets of the cells -2..2 around a particle's old cell
// per axis (x: i, y: nx j, z: nx ny k; a run has fewer than 2^31 cells) and the
// run's first cell.  They index the scatter into lambda_E and lambda_B on every
// path, and every read on the global-memory path.
struct AdjWrap {
    long long cb;
    int x[5], y[5], z[5];
    __device__ __forceinline__ long long at(int dx, int dy, int dz) const
    {
        return cb + (long long)(x[dx + 2] + y[dy + 2] + z[dz + 2]);
    }
};

template <int DIM>
__device__ __forceinline__ void adj_wrap(AdjWrap &w, const RunDev &rn, int i, int j, int k)
{
    const int nx = rn.n[0], ny = rn.n[1], nz = rn.n[2];
    w.cb = rn.cell_base;
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        w.x[q] = wrapi(i - 2 + q, nx);
        w.y[q] = nx * wrapi(j - 2 + q, ny);
        w.z[q] = DIM == 3 ? nx * ny * wrapi(k - 2 + q, nz) : 0;
    }
}

// Readers of the particle adjoint: E and B1 at offsets -1..1 and lambda_J at
// offsets -2..2 from the particle's old cell, from the periodic global arrays
// or from a work item's shared-memory tiles.
template <typename R>
struct AdjGlobalRd {
    static constexpr bool kFixed = false;
    const R *E[3];
    const R *B[3];
    const R *LJ[3];
    R *LE[3];
    R *LB[3];
    const AdjWrap *w;
    __device__ __forceinline__ R e(int c, int dx, int dy, int dz) const { return E[c][w->at(dx, dy, dz)]; }
    __device__ __forceinline__ R b(int c, int dx, int dy, int dz) const { return B[c][w->at(dx, dy, dz)]; }
    __device__ __forceinline__ R lj(int c, int dx, int dy, int dz) const { return LJ[c][w->at(dx, dy, dz)]; }
    // transposed gather: one global reduction per tap
    __device__ __forceinline__ void scatter(int fld, int c, int dx, int dy, int dz, R v) const
    {
        atomicAdd(&(fld == 0 ? LE[c] : LB[c])[w->at(dx, dy, dz)], v);
    }
};

template <typename R>
struct AdjSmemRd {
    static constexpr bool kFixed = false;
    const R *E[3];
    const R *B[3];
    const R *LJ[3];
    R *LE[3];
    R *LB[3];
    int fb, jb, s1, s2;   // the old cell in the field tile and in the lambda_J tile; y and z strides
    __device__ __forceinline__ R e(int c, int dx, int dy, int dz) const { return E[c][fb + dx + s1 * dy + s2 * dz]; }
    __device__ __forceinline__ R b(int c, int dx, int dy, int dz) const { return B[c][fb + dx + s1 * dy + s2 * dz]; }
    __device__ __forceinline__ R lj(int c, int dx, int dy, int dz) const
    {
        return LJ[c][jb + dx + s1 * dy + s2 * dz];
    }
    // transposed gather into the block's lambda_E / lambda_B tiles (same layout
    // as the field tile), added to the global arrays once per block
    __device__ __forceinline__ void scatter(int fld, int c, int dx, int dy, int dz, R v) const
    {
        atomicAdd(&(fld == 0 ? LE[c] : LB[c])[fb + dx + s1 * dy + s2 * dz], v);
    }
};

// Six-component fixed-point accumulator for the adjoint's lambda_E and lambda_B
// tiles (the FixedAcc split, components 0..5).
struct FixedAcc6 {
    int *hi[6];
    int *lo[6];
    int base, s1, s2;
    __device__ __forceinline__ void add(int a, int dx, int dy, int dz, float kp, float t) const
    {
        const float magic = 12582912.0f;   // 1.5 * 2^23
        const float th = fmaf(kp * (1.0f / 65536.0f), t, magic);   // magic + hi
        const float ch = fmaf(th, -65536.0f, magic * 65537.0f);      // magic - hi * 2^16, exact
        const float tl = fmaf(kp, t, ch);                            // magic + lo, one rounding
        const int idx = base + dx + s1 * dy + s2 * dz;
        atomicAdd(&hi[a][idx], __float_as_int(th) - (int)kFixBias);
        atomicAdd(&lo[a][idx], __float_as_int(tl) - (int)kFixBias);
    }
};

// FP32 tiles with the transposed gather in exact fixed point: the block's
// lambda_E / lambda_B tiles are pairs of int32 words (FixedAcc), the scale a
// power of two chosen from the largest |lambda| of the previous launch with a
// margin, so that every contribution of a particle whose lambdas stay below
// `bound` keeps within the fixed-point range.  A particle above it (the first
// launch, or a sudden growth) scatters into the global arrays instead.
struct AdjSmemRdFixed {
    static constexpr bool kFixed = true;
    const float *E[3];
    const float *B[3];
    const float *LJ[3];
    FixedAcc6 acc;       // base set per particle to its field-tile cell
    float kp;            // the fixed-point scale
    float bound;         // largest |lambda| kept in the tiles
    int fb, jb, s1, s2;
    __device__ __forceinline__ float e(int c, int dx, int dy, int dz) const { return E[c][fb + dx + s1 * dy + s2 * dz]; }
    __device__ __forceinline__ float b(int c, int dx, int dy, int dz) const { return B[c][fb + dx + s1 * dy + s2 * dz]; }
    __device__ __forceinline__ float lj(int c, int dx, int dy, int dz) const
    {
        return LJ[c][jb + dx + s1 * dy + s2 * dz];
    }
    // fld 0: lambda_E (components 0..2 of the accumulator), 1: lambda_B (3..5)
    __device__ __forceinline__ void scatter(int fld, int c, int dx, int dy, int dz, float v) const
    {
        acc.add(fld * 3 + c, dx, dy, dz, kp, v);
    }
};


// Reverse of one particle's step: from lambda_x, lambda_w at level n+1 (index
// L) to level n, adding the transposed gather into lambda_E and lambda_B1.
// The transposed gather of one particle into the global lambda_E and
// lambda_B1 arrays (the fixed-point tiles' fallback for a particle whose
// lambdas exceed the tiles' bound): weights f, S per axis, old cell (i, j, k).
template <int DIM, typename R>
__device__ __noinline__ void adj_scatter_global(const AdjArgs<R> &a, const RunDev &rn, int i, int j, int k,
                                                const R *f, const R *S, const R *lEp, const R *lBp)
{
    AdjWrap w;
    adj_wrap<DIM>(w, rn, i, j, k);
    for (int fld = 0; fld < 2; ++fld)
        for (int c = 0; c < 3; ++c) {
            const bool intx = (fld == 0) == (c == 0), inty = (fld == 0) == (c == 1), intz = (fld == 0) == (c == 2);
            const int cx = intx ? 2 : 3, cy = inty ? 2 : 3, cz = DIM == 3 ? (intz ? 2 : 3) : 1;
            const int ox = intx ? 0 : -1, oy = inty ? 0 : -1, oz = DIM == 3 ? (intz ? 0 : -1) : 0;
            const R lam = fld == 0 ? lEp[c] : lBp[c];
            R *dst = fld == 0 ? a.lamE[c] : a.lamB1[c];
            for (int sz = 0; sz < cz; ++sz)
                for (int sy = 0; sy < cy; ++sy)
                    for (int sx = 0; sx < cx; ++sx) {
                        const R vx = intx ? f[0 * 2 + sx] : S[0 * 3 + sx];
                        const R vy = inty ? f[1 * 2 + sy] : S[1 * 3 + sy];
                        const R vz = DIM == 3 ? (intz ? f[2 * 2 + sz] : S[2 * 3 + sz]) : R(1);
                        atomicAdd(&dst[w.at(ox + sx, oy + sy, DIM == 3 ? oz + sz : 0)], vx * vy * vz * lam);
                    }
        }
}

template <int DIM, typename R, class Rd>
__device__ __forceinline__ void adj_particle(const AdjArgs<R> &a, const GroupDev &gr, const RunDev &rn, long long p,
                                             long long L, const Rd &rd, int ci = 0, int cj = 0, int ck = 0,
                                             float *lam_seen = nullptr)
{
    constexpr bool F32 = sizeof(R) == 4;
    const R third = R(1) / R(3);
    // the particle's adjoints at level n+1, loaded first so that their latency
    // overlaps the recomputation
    R lx1[3], lw1[3];
    #pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        lx1[ax] = ax < DIM ? a.lamx[ax][L] : R(0);
        lw1[ax] = a.lamw[ax][L];
    }
    R o[3] = {a.P.off[0][p], a.P.off[1][p], DIM == 3 ? a.P.off[2][p] : R(0)};
    const R w0[3] = {a.P.w[0][p], a.P.w[1][p], a.P.w[2][p]};
    // ---- recompute the forward quantities ------------------------------------
    R f[3][2], S[3][3], df[3][2], dS[3][3];
    #pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        if (ax == 2 && DIM == 2) {
            f[2][0] = R(1); f[2][1] = R(0); S[2][0] = R(0); S[2][1] = R(1); S[2][2] = R(0);
            df[2][0] = df[2][1] = R(0); dS[2][0] = dS[2][1] = dS[2][2] = R(0);
            continue;
        }
        form_factor(o[ax], f[ax], S[ax]);
        form_factor_d(o[ax], df[ax], dS[ax]);
    }
    // alternating-order gather (Eqs. alphax, betax), the forward kernel's sums
    R Ep[3], Bp[3];
    gather<DIM>(rd, f[0], S[0], f[1], S[1], f[2], S[2], Ep, Bp);
    // group and run constants prepared on the host (no FP64 arithmetic in FP32)
    const R hq = F32 ? R(gr.hqf) : R(gr.hq);
    const R cl = F32 ? R(rn.cf) : R(rn.c), c2 = cl * cl;
    const R cN[3] = {F32 ? R(rn.cNf[0]) : R(rn.cN[0]), F32 ? R(rn.cNf[1]) : R(rn.cN[1]),
                     F32 ? R(rn.cNf[2]) : R(rn.cN[2])};
    R w1[3] = {w0[0], w0[1], w0[2]};
    boris(w1, Ep, Bp, hq, c2);
    const R ig = rsqrt_r(w1[0] * w1[0] + w1[1] * w1[1] + w1[2] * w1[2] + c2);   // as the forward kernels
    R n1[3] = {o[0], o[1], o[2]};
    int sh[3] = {0, 0, 0};
    #pragma unroll
    for (int ax = 0; ax < DIM; ++ax) sh[ax] = renormalize(o[ax], w1[ax] * ig * cN[ax], n1[ax]);
    const R uz = cl * w1[2] * ig;
    // ---- reverse of the deposit ----------------------------------------------
    AxisWin<R> W[3];
    AxisWinAdj<R> WA[3];
    #pragma unroll
    for (int ax = 0; ax < DIM; ++ax) {
        axis_window(o[ax], n1[ax], sh[ax], W[ax]);
        axis_window_adj(o[ax], n1[ax], sh[ax], WA[ax]);
    }
    R lPp[3][4] = {{0}}, lPm[3][4] = {{0}}, lD[3][3] = {{0}};
    R luz = 0;
    if (DIM == 3) {
        #pragma unroll
        for (int cmp = 0; cmp < 3; ++cmp) {
            const int b = (cmp + 1) % 3, cc = (cmp + 2) % 3;
            const R ka = F32 ? R(gr.kff[cmp]) : R(gr.kf[cmp]);
            #pragma unroll
            for (int wc = 0; wc < 4; ++wc)
                #pragma unroll
                for (int wb = 0; wb < 4; ++wb) {
                    const R T = W[b].Pp[wb] * W[cc].Pp[wc] + W[b].Pm[wb] * W[cc].Pm[wc] * third;
                    #pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        int off[3];
                        off[cmp] = W[cmp].lo + 1 + q;
                        off[b] = W[b].lo + wb;
                        off[cc] = W[cc].lo + wc;
                        const R G = rd.lj(cmp, off[0], off[1], off[2]) * ka;
                        lD[cmp][q] += G * T;
                        lPp[b][wb] += G * W[cmp].D[q] * W[cc].Pp[wc];
                        lPp[cc][wc] += G * W[cmp].D[q] * W[b].Pp[wb];
                        lPm[b][wb] += G * W[cmp].D[q] * W[cc].Pm[wc] * third;
                        lPm[cc][wc] += G * W[cmp].D[q] * W[b].Pm[wb] * third;
                    }
                }
        }
    } else {
        const R kx = F32 ? R(gr.kff[0]) : R(gr.kf[0]);
        const R ky = F32 ? R(gr.kff[1]) : R(gr.kf[1]);
        const R kz = F32 ? R(gr.kff[2]) : R(gr.kf[2]);
        #pragma unroll
        for (int wy = 0; wy < 4; ++wy)
            #pragma unroll
            for (int q = 0; q < 3; ++q) {
                const R G = rd.lj(0, W[0].lo + 1 + q, W[1].lo + wy, 0) * kx;
                lD[0][q] += G * W[1].Pp[wy];
                lPp[1][wy] += G * W[0].D[q];
            }
        #pragma unroll
        for (int wx = 0; wx < 4; ++wx)
            #pragma unroll
            for (int q = 0; q < 3; ++q) {
                const R G = rd.lj(1, W[0].lo + wx, W[1].lo + 1 + q, 0) * ky;
                lD[1][q] += G * W[0].Pp[wx];
                lPp[0][wx] += G * W[1].D[q];
            }
        #pragma unroll
        for (int wy = 0; wy < 4; ++wy)
            #pragma unroll
            for (int wx = 0; wx < 4; ++wx) {
                const R G = rd.lj(2, W[0].lo + wx, W[1].lo + wy, 0) * kz;
                luz += G * (W[0].Pp[wx] * W[1].Pp[wy] + W[0].Pm[wx] * W[1].Pm[wy] * third);
                lPp[0][wx] += G * uz * W[1].Pp[wy];
                lPp[1][wy] += G * uz * W[0].Pp[wx];
                lPm[0][wx] += G * uz * W[1].Pm[wy] * third;
                lPm[1][wy] += G * uz * W[0].Pm[wx] * third;
            }
    }
    R lx0[3] = {R(0), R(0), R(0)};
    #pragma unroll
    for (int ax = 0; ax < DIM; ++ax) {
        // D[q] = sum_{w <= q} Pm[w]
        lPm[ax][0] += lD[ax][0] + lD[ax][1] + lD[ax][2];
        lPm[ax][1] += lD[ax][1] + lD[ax][2];
        lPm[ax][2] += lD[ax][2];
        R ln = 0, lo2 = 0;
        #pragma unroll
        for (int w4 = 0; w4 < 4; ++w4) {
            ln += (lPp[ax][w4] + lPm[ax][w4]) * WA[ax].dN[w4];
            lo2 += (lPp[ax][w4] - lPm[ax][w4]) * WA[ax].dO[w4];
        }
        lx1[ax] += ln;
        lx0[ax] += lo2 + lx1[ax];   // x^{n+1} = x^n + delta
    }
    // ---- reverse of the move: delta_a = cN_a w1_a / gamma1, u_z = c w1_z / gamma1
    const R ig3 = ig * ig * ig;
    #pragma unroll
    for (int bb = 0; bb < 3; ++bb) {
        R acc = 0;
        #pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            const R jac = (ax == bb ? ig : R(0)) - w1[ax] * w1[bb] * ig3;
            if (ax < DIM) acc += lx1[ax] * cN[ax] * jac;
            if (ax == 2 && DIM == 2) acc += luz * cl * jac;
        }
        lw1[bb] += acc;
    }
    // ---- reverse of the push (Appendix): t = w + e, b = s B, n = t + t x b,
    // F = 2/(1 + b.b), w1 = t + e + F (n x b)
    R lEp[3], lBp[3], lw0[3];
    {
        R e[3], t[3], b[3], nn3[3], m[3];
        #pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            e[ax] = hq * Ep[ax];
            t[ax] = w0[ax] + e[ax];
        }
        const R gt = sqrt(t[0] * t[0] + t[1] * t[1] + t[2] * t[2] + c2);
        const R s = hq / gt;
        #pragma unroll
        for (int ax = 0; ax < 3; ++ax) b[ax] = s * Bp[ax];
        nn3[0] = t[0] + (t[1] * b[2] - t[2] * b[1]);
        nn3[1] = t[1] + (t[2] * b[0] - t[0] * b[2]);
        nn3[2] = t[2] + (t[0] * b[1] - t[1] * b[0]);
        const R b2 = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
        const R Fq = R(2) / (R(1) + b2);
        m[0] = nn3[1] * b[2] - nn3[2] * b[1];
        m[1] = nn3[2] * b[0] - nn3[0] * b[2];
        m[2] = nn3[0] * b[1] - nn3[1] * b[0];
        R lt[3], le[3], lm[3], ln3[3], lb[3];
        R lF = 0;
        #pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            lt[ax] = lw1[ax];
            le[ax] = lw1[ax];
            lm[ax] = Fq * lw1[ax];
            lF += lw1[ax] * m[ax];
        }
        // m = n x b: ln = b x lm, lb = lm x n
        ln3[0] = b[1] * lm[2] - b[2] * lm[1];
        ln3[1] = b[2] * lm[0] - b[0] * lm[2];
        ln3[2] = b[0] * lm[1] - b[1] * lm[0];
        lb[0] = lm[1] * nn3[2] - lm[2] * nn3[1];
        lb[1] = lm[2] * nn3[0] - lm[0] * nn3[2];
        lb[2] = lm[0] * nn3[1] - lm[1] * nn3[0];
        const R lb2 = lF * (-R(2) / ((R(1) + b2) * (R(1) + b2)));
        #pragma unroll
        for (int ax = 0; ax < 3; ++ax) lb[ax] += R(2) * b[ax] * lb2;
        // n = t + t x b: lt += ln + b x ln, lb += ln x t
        lt[0] += ln3[0] + (b[1] * ln3[2] - b[2] * ln3[1]);
        lt[1] += ln3[1] + (b[2] * ln3[0] - b[0] * ln3[2]);
        lt[2] += ln3[2] + (b[0] * ln3[1] - b[1] * ln3[0]);
        lb[0] += ln3[1] * t[2] - ln3[2] * t[1];
        lb[1] += ln3[2] * t[0] - ln3[0] * t[2];
        lb[2] += ln3[0] * t[1] - ln3[1] * t[0];
        R ls = 0;
        #pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            ls += lb[ax] * Bp[ax];
            lBp[ax] = s * lb[ax];
        }
        const R lgt = -ls * hq / (gt * gt);
        #pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            lt[ax] += lgt * t[ax] / gt;
            lw0[ax] = lt[ax];
            lEp[ax] = hq * (le[ax] + lt[ax]);
        }
    }
    // ---- reverse of the gather: scatter into lamE, lamB1; derivatives of the
    // weights into lx0
    bool big = false;   // (fixed-point tiles) the particle's lambdas exceed their bound
    if constexpr (Rd::kFixed) {
        float mx = 0.f;
        #pragma unroll
        for (int c = 0; c < 3; ++c) {
            big = big || !(fabsf(lEp[c]) <= rd.bound) || !(fabsf(lBp[c]) <= rd.bound);
            mx = fmaxf(mx, fmaxf(fabsf(lEp[c]), fabsf(lBp[c])));
        }
        *lam_seen = fmaxf(*lam_seen, mx);
        if (big) {
            R fw[6], Sw[9];
            #pragma unroll
            for (int ax = 0; ax < 3; ++ax) {
                fw[2 * ax] = f[ax][0];
                fw[2 * ax + 1] = f[ax][1];
                Sw[3 * ax] = S[ax][0];
                Sw[3 * ax + 1] = S[ax][1];
                Sw[3 * ax + 2] = S[ax][2];
            }
            adj_scatter_global<DIM, R>(a, rn, ci, cj, ck, fw, Sw, lEp, lBp);
        }
    }
    #pragma unroll
    for (int fld = 0; fld < 2; ++fld)
        #pragma unroll
        for (int c = 0; c < 3; ++c) {
            const bool intx = (fld == 0) == (c == 0), inty = (fld == 0) == (c == 1), intz = (fld == 0) == (c == 2);
            const int cx = intx ? 2 : 3, cy = inty ? 2 : 3, cz = DIM == 3 ? (intz ? 2 : 3) : 1;
            const int ox = intx ? 0 : -1, oy = inty ? 0 : -1, oz = DIM == 3 ? (intz ? 0 : -1) : 0;
            const R lam = fld == 0 ? lEp[c] : lBp[c];
            #pragma unroll
            for (int sz = 0; sz < cz; ++sz)
                #pragma unroll
                for (int sy = 0; sy < cy; ++sy)
                    #pragma unroll
                    for (int sx = 0; sx < cx; ++sx) {
                        const int dx = ox + sx, dy = oy + sy, dz = DIM == 3 ? oz + sz : 0;
                        const R vx = intx ? f[0][sx] : S[0][sx], ddx = intx ? df[0][sx] : dS[0][sx];
                        const R vy = inty ? f[1][sy] : S[1][sy], ddy = inty ? df[1][sy] : dS[1][sy];
                        const R vz = DIM == 3 ? (intz ? f[2][sz] : S[2][sz]) : R(1);
                        const R ddz = DIM == 3 ? (intz ? df[2][sz] : dS[2][sz]) : R(0);
                        if (!big) rd.scatter(fld, c, dx, dy, dz, vx * vy * vz * lam);
                        const R fl = (fld == 0 ? rd.e(c, dx, dy, dz) : rd.b(c, dx, dy, dz)) * lam;
                        lx0[0] += ddx * vy * vz * fl;
                        lx0[1] += vx * ddy * vz * fl;
                        lx0[2] += vx * vy * ddz * fl;
                    }
        }
    #pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        if (ax < DIM) a.lamx[ax][L] = lx0[ax];
        a.lamw[ax][L] = lw0[ax];
    }
}

template <int DIM>
__device__ __forceinline__ void split_cell(const RunDev &rn, int cell, int &i, int &j, int &k)
{
    const int rest = divu31(cell, rn.div_nx);
    i = cell - rest * rn.n[0];
    k = DIM == 3 ? divu31(rest, rn.div_ny) : 0;
    j = rest - k * rn.n[1];
}

// A particle on the periodic global arrays (the untiled kernel, and particles
// that drifted past their tile's halo since the last sort).  The wrapped
// offsets are indexed at run time here, so they live in local memory.
template <int DIM, typename R>
__device__ __forceinline__ void adj_particle_global_body(const AdjArgs<R> &a, const GroupDev &gr, const RunDev &rn,
                                                         long long p, long long L, int i, int j, int k)
{
    AdjWrap wr;
    adj_wrap<DIM>(wr, rn, i, j, k);
    AdjGlobalRd<R> rd;
    for (int c = 0; c < 3; ++c) {
        rd.E[c] = a.E[c];
        rd.B[c] = a.B1[c];
        rd.LJ[c] = a.lamJ[c];
        rd.LE[c] = a.lamE[c];
        rd.LB[c] = a.lamB1[c];
    }
    rd.w = &wr;
    adj_particle<DIM, R>(a, gr, rn, p, L, rd);
}

// Untiled form: one thread per particle in pool order, all reads global.
template <int DIM, typename R>
__global__ void __launch_bounds__(256) k_particles_adj(const AdjArgs<R> a)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < a.total; p += stride) {
        int lo = 0, hi = a.ngroups;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (a.group_base[mid] <= p) lo = mid; else hi = mid;
        }
        const GroupDev &gr = a.groups[lo];
        const RunDev &rn = a.runs[gr.run];
        int i, j, k;
        split_cell<DIM>(rn, a.P.cell[p], i, j, k);
        adj_particle_global_body<DIM, R>(a, gr, rn, p, gr.base + a.P.id[p], i, j, k);
    }
}

// Tiled form over the last sort's work items: `nsplit` blocks share one item,
// each stages the item's E and B1 with a halo of (halo + 1) cells and lambda_J
// with a halo of (halo + 2) cells in shared memory, in the particle kernels'
// tile pitches, then takes every nsplit-th round of 256 particles of the item.
// Reads come from the tiles; the transposed gather adds into the block's
// lambda_E / lambda_B tiles, flushed to the global arrays once per block.  In
// FP32 those tiles hold exact fixed-point sums (integer atomics, at a scale set
// from the previous launch's largest lambda; AdjSmemRdFixed); in FP64 they are
// float tiles.  A particle that drifted past the tile's halo takes the
// global-memory form.
template <int DIM, typename R>
__global__ void __launch_bounds__(kThreads, sizeof(R) == 4 ? 2 : 1) k_particles_adj_tiled(const AdjArgs<R> a, const WorkItem *items,
                                                                  const int *n_items, int halo, int nsplit)
{
    constexpr bool FIX = sizeof(R) == 4;
    const int item = blockIdx.x / nsplit, part = blockIdx.x - item * nsplit;
    if (item >= *n_items) return;
    const WorkItem it = items[item];
    const GroupDev gr = a.groups[it.group];
    const RunDev rn = a.runs[gr.run];
    const int G = halo;
    const int nx = rn.n[0], ny = rn.n[1], nz = rn.n[2];
    const int T0 = rn.tile[0], T1 = rn.tile[1], T2 = DIM == 3 ? rn.tile[2] : 1;
    const int tx = it.tile % rn.ntile[0];
    const int ty = (it.tile / rn.ntile[0]) % rn.ntile[1];
    const int tz = DIM == 3 ? it.tile / (rn.ntile[0] * rn.ntile[1]) : 0;
    const int ox = tx * T0, oy = ty * T1, oz = tz * T2;
    const int fe0 = T0 + 2 * G + 2, fe1 = T1 + 2 * G + 2, fe2 = DIM == 3 ? T2 + 2 * G + 2 : 1;
    const int je0 = T0 + 2 * G + 4, je1 = T1 + 2 * G + 4, je2 = DIM == 3 ? T2 + 2 * G + 4 : 1;
    const int P0 = rn.pitch[0], P1 = rn.pitch[1];   // >= je0, je1
    const int nf = P0 * P1 * fe2, nj = P0 * P1 * je2;
    const long long cb = rn.cell_base;
    R *sE[3], *sB[3], *sL[3], *sLE[3], *sLB[3];
    int *sH[6], *sLo[6];   // FP32: hi and lo words of lambda_E (0..2) and lambda_B (3..5)
    {
        // FP64: E, B1, lambda_E, lambda_B1 (12 tiles of nf), lambda_J (3 of nj);
        // FP32: E, B1 (6 of nf), the int hi/lo words (12 of nf), lambda_J
        R *s = reinterpret_cast<R *>(g_smem);
        int *q = reinterpret_cast<int *>(s + 6 * nf);
        for (int c = 0; c < 3; ++c) {
            sE[c] = s + c * nf;
            sB[c] = s + (3 + c) * nf;
            sLE[c] = s + (6 + c) * nf;
            sLB[c] = s + (9 + c) * nf;
            sL[c] = s + (FIX ? 18 : 12) * nf + c * nj;
        }
        for (int c = 0; c < 6; ++c) {
            sH[c] = q + c * nf;
            sLo[c] = q + (6 + c) * nf;
        }
    }
    for (int l = threadIdx.x; l < nf; l += blockDim.x) {
        if constexpr (FIX) {
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                sH[c][l] = 0;
                sLo[c][l] = 0;
            }
        } else {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                sLE[c][l] = R(0);
                sLB[c][l] = R(0);
            }
        }
        const int lx = l % P0, r = l / P0, ly = r % P1, lz = r / P1;
        if (lx >= fe0 || ly >= fe1) continue;   // pitch padding
        const int gx = wrapi(ox - G - 1 + lx, nx);
        const int gy = wrapi(oy - G - 1 + ly, ny);
        const int gz = DIM == 3 ? wrapi(oz - G - 1 + lz, nz) : 0;
        const long long gi = cb + gx + (long long)nx * (gy + (long long)ny * gz);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            sE[c][l] = a.E[c][gi];
            sB[c][l] = a.B1[c][gi];
        }
    }
    for (int l = threadIdx.x; l < nj; l += blockDim.x) {
        const int lx = l % P0, r = l / P0, ly = r % P1, lz = r / P1;
        if (lx >= je0 || ly >= je1) continue;
        const int gx = wrapi(ox - G - 2 + lx, nx);
        const int gy = wrapi(oy - G - 2 + ly, ny);
        const int gz = DIM == 3 ? wrapi(oz - G - 2 + lz, nz) : 0;
        const long long gi = cb + gx + (long long)nx * (gy + (long long)ny * gz);
#pragma unroll
        for (int c = 0; c < 3; ++c) sL[c][l] = a.lamJ[c][gi];
    }
    // FP32: the fixed-point scale, 2^(33 - ceil(log2 bound)) for lambdas up to
    // bound = 256 x the previous launch's largest (a work item holds at most
    // 8192 particles, so every word's sum stays within 2^46); none yet: every
    // particle scatters into the global arrays
    float bound = -1.f, kp = 1.f;
    if (FIX) {
        const float prev = __uint_as_float(*a.lam_prev);
        if (prev > 0.f && prev < 1e30f) {
            bound = 256.f * prev;
            int e2 = 0;
            frexpf(bound, &e2);   // bound <= 2^e2
            kp = ldexpf(1.0f, 33 - e2);
        }
    }
    __syncthreads();
    float lam_seen = 0.f;
    const long long step = (long long)nsplit * blockDim.x;
    for (long long p = it.begin + (long long)part * blockDim.x + threadIdx.x; p < it.end; p += step) {
        const long long L = gr.base + a.P.id[p];
        int i, j, k;
        split_cell<DIM>(rn, a.P.cell[p], i, j, k);
        const int li = local_coord(i, ox, T0, G, nx);
        const int lj = local_coord(j, oy, T1, G, ny);
        const int lk = DIM == 3 ? local_coord(k, oz, T2, G, nz) : 0;
        const bool inr =
            li >= -G && li < T0 + G && lj >= -G && lj < T1 + G && (DIM == 2 || (lk >= -G && lk < T2 + G));
        if (inr) {
            const int fb = (li + G + 1) + P0 * ((lj + G + 1) + (DIM == 3 ? P1 * (lk + G + 1) : 0));
            const int jb = (li + G + 2) + P0 * ((lj + G + 2) + (DIM == 3 ? P1 * (lk + G + 2) : 0));
            if constexpr (FIX) {
                AdjSmemRdFixed rd;
                for (int c = 0; c < 3; ++c) {
                    rd.E[c] = reinterpret_cast<const float *>(sE[c]);
                    rd.B[c] = reinterpret_cast<const float *>(sB[c]);
                    rd.LJ[c] = reinterpret_cast<const float *>(sL[c]);
                }
                for (int c = 0; c < 6; ++c) {
                    rd.acc.hi[c] = sH[c];
                    rd.acc.lo[c] = sLo[c];
                }
                rd.acc.base = fb;
                rd.acc.s1 = P0;
                rd.acc.s2 = P0 * P1;
                rd.kp = kp;
                rd.bound = bound;
                rd.s1 = P0;
                rd.s2 = P0 * P1;
                rd.fb = fb;
                rd.jb = jb;
                adj_particle<DIM, R>(a, gr, rn, p, L, rd, i, j, k, &lam_seen);
            } else {
                AdjSmemRd<R> rd;
                for (int c = 0; c < 3; ++c) {
                    rd.E[c] = sE[c];
                    rd.B[c] = sB[c];
                    rd.LJ[c] = sL[c];
                    rd.LE[c] = sLE[c];
                    rd.LB[c] = sLB[c];
                }
                rd.s1 = P0;
                rd.s2 = P0 * P1;
                rd.fb = fb;
                rd.jb = jb;
                adj_particle<DIM, R>(a, gr, rn, p, L, rd);
            }
        } else {
            adj_particle_global_body<DIM, R>(a, gr, rn, p, L, i, j, k);
        }
    }
    if (FIX) {   // the launch's largest lambda, for the next launch's scale
        unsigned m = __float_as_uint(lam_seen);
        for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
        if ((threadIdx.x & 31) == 0 && m != 0u) atomicMax(a.lam_cur, m);
    }
    // the block's lambda_E / lambda_B tiles into the global arrays
    __syncthreads();
    const float inv = 1.0f / kp;
    for (int l = threadIdx.x; l < nf; l += blockDim.x) {
        const int lx = l % P0, r = l / P0, ly = r % P1, lz = r / P1;
        if (lx >= fe0 || ly >= fe1) continue;
        const int gx = wrapi(ox - G - 1 + lx, nx);
        const int gy = wrapi(oy - G - 1 + ly, ny);
        const int gz = DIM == 3 ? wrapi(oz - G - 1 + lz, nz) : 0;
        const long long gi = cb + gx + (long long)nx * (gy + (long long)ny * gz);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            if constexpr (FIX) {
                const int he = sH[c][l], le = sLo[c][l], hb = sH[3 + c][l], lb = sLo[3 + c][l];
                if ((he | le) != 0) atomicAdd(&a.lamE[c][gi], (R)(fmaf((float)he, 65536.0f, (float)le) * inv));
                if ((hb | lb) != 0) atomicAdd(&a.lamB1[c][gi], (R)(fmaf((float)hb, 65536.0f, (float)lb) * inv));
            } else {
                const R ve = sLE[c][l], vb = sLB[c][l];
                if (ve != R(0)) atomicAdd(&a.lamE[c][gi], ve);
                if (vb != R(0)) atomicAdd(&a.lamB1[c][gi], vb);
            }
        }
    }
}

// Transpose of the E step at one cell: lamJ = -4 pi dt lamE; lamB += C_E^T lamE,
// i.e. lamBx += c_y(lamEz[p] - lamEz[j-1]) - c_z(lamEy[p] - lamEy[k-1]) and cyclically.
template <int DIM, typename R>
__global__ void k_adj_yee_e(const RunDev *runs, const R *lamE0, const R *lamE1, const R *lamE2, R *lB0, R *lB1,
                            R *lB2, R *lJ0, R *lJ1, R *lJ2)
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
    const R cx = R(rn.cN[0]), cy = R(rn.cN[1]);
    const R fp = R(4.0 * 3.14159265358979323846 * rn.dt);
    lJ0[p] = -fp * lamE0[p];
    lJ1[p] = -fp * lamE1[p];
    lJ2[p] = -fp * lamE2[p];
    R bx = cy * (lamE2[p] - lamE2[pjm]);
    R by = -cx * (lamE2[p] - lamE2[pim]);
    R bz = cx * (lamE1[p] - lamE1[pim]) - cy * (lamE0[p] - lamE0[pjm]);
    if (DIM == 3) {
        const long long pkm = p + (long long)nx * ny * (k == 0 ? nz - 1 : -1);
        const R cz = R(rn.cN[2]);
        bx -= cz * (lamE1[p] - lamE1[pkm]);
        by += cz * (lamE0[p] - lamE0[pkm]);
    }
    lB0[p] += bx;
    lB1[p] += by;
    lB2[p] += bz;
}

// Transpose of the B half step at one cell: lamE += (-(1/2) C_B)^T lamB, i.e.
// lamEx += -(1/2)[c_y(lamBz[j+1] - lamBz[p]) - c_z(lamBy[k+1] - lamBy[p])] and cyclically.
template <int DIM, typename R>
__global__ void k_adj_yee_b(const RunDev *runs, const R *lB0, const R *lB1, const R *lB2, R *lE0, R *lE1, R *lE2)
{
    const RunDev &rn = runs[blockIdx.y];
    const int nx = rn.n[0], ny = rn.n[1], nz = rn.n[2];
    const long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (l >= (long long)nx * ny * nz) return;
    const int i = (int)(l % nx);
    const long long r = l / nx;
    const int j = (int)(r % ny), k = (int)(r / ny);
    const long long p = rn.cell_base + l;
    const long long pip = p + (i == nx - 1 ? -(nx - 1) : 1);
    const long long pjp = p + (long long)nx * (j == ny - 1 ? -(ny - 1) : 1);
    const R hx = R(0.5 * rn.cN[0]), hy = R(0.5 * rn.cN[1]);
    R ex = -hy * (lB2[pjp] - lB2[p]);
    R ey = hx * (lB2[pip] - lB2[p]);
    R ez = -hx * (lB1[pip] - lB1[p]) + hy * (lB0[pjp] - lB0[p]);
    if (DIM == 3) {
        const long long pkp = p + (long long)nx * ny * (k == nz - 1 ? -(nz - 1) : 1);
        const R hz = R(0.5 * rn.cN[2]);
        ex += hz * (lB1[pkp] - lB1[p]);
        ey -= hz * (lB0[pkp] - lB0[p]);
    }
    lE0[p] += ex;
    lE1[p] += ey;
    lE2[p] += ez;
}

template <int DIM, typename R>
static cudaError_t adj_yee_t(int which, cudaStream_t st, const RunDev *runs, int nruns, long long max_cells,
                             void *const lamE[3], void *const lamB[3], void *const lamJ[3])
{
    const int nt = 256;
    dim3 grid((unsigned)((max_cells + nt - 1) / nt), (unsigned)nruns);
    R *e[3], *b[3], *j[3];
    for (int c = 0; c < 3; ++c) {
        e[c] = (R *)lamE[c];
        b[c] = (R *)lamB[c];
        j[c] = lamJ ? (R *)lamJ[c] : nullptr;
    }
    if (which == 2)
        k_adj_yee_e<DIM, R><<<grid, nt, 0, st>>>(runs, e[0], e[1], e[2], b[0], b[1], b[2], j[0], j[1], j[2]);
    else
        k_adj_yee_b<DIM, R><<<grid, nt, 0, st>>>(runs, b[0], b[1], b[2], e[0], e[1], e[2]);
    return cudaGetLastError();
}

cudaError_t launch_adj_yee(int dims, int prec, int which, cudaStream_t st, const RunDev *runs, int nruns,
                           long long max_cells, void *const lamE[3], void *const lamB[3], void *const lamJ[3])
{
    if (dims == 3)
        return prec == 0 ? adj_yee_t<3, double>(which, st, runs, nruns, max_cells, lamE, lamB, lamJ)
                         : adj_yee_t<3, float>(which, st, runs, nruns, max_cells, lamE, lamB, lamJ);
    return prec == 0 ? adj_yee_t<2, double>(which, st, runs, nruns, max_cells, lamE, lamB, lamJ)
                     : adj_yee_t<2, float>(which, st, runs, nruns, max_cells, lamE, lamB, lamJ);
}

template <int DIM, typename R>
static cudaError_t adj_part_t(cudaStream_t st, const AdjLaunch &lc, const PoolBuf &P, void *const E[3],
                              void *const B1[3], void *const lamJ[3], void *const lamE[3], void *const lamB1[3],
                              void *const lamx[3], void *const lamw[3])
{
    AdjArgs<R> a;
    a.runs = lc.runs;
    a.groups = lc.groups;
    a.group_base = lc.group_base;
    a.ngroups = lc.ngroups;
    a.total = lc.total;
    a.P.cell = P.cell;
    a.P.id = P.id;
    for (int c = 0; c < 3; ++c) {
        a.P.off[c] = (R *)P.off[c];
        a.P.w[c] = (R *)P.w[c];
        a.E[c] = (const R *)E[c];
        a.B1[c] = (const R *)B1[c];
        a.lamJ[c] = (const R *)lamJ[c];
        a.lamE[c] = (R *)lamE[c];
        a.lamB1[c] = (R *)lamB1[c];
        a.lamx[c] = (R *)lamx[c];
        a.lamw[c] = (R *)lamw[c];
    }
    a.lam_prev = lc.lam_prev;
    a.lam_cur = lc.lam_cur;
    if (lc.total <= 0) return cudaSuccess;
    if (lc.items && lc.max_items > 0) {
        // blocks per work item: about 512 particles or more per block on average
        long long ns = lc.total / ((long long)lc.max_items * 512);
        const int nsplit = (int)(ns < 1 ? 1 : ns > 8 ? 8 : ns);
        const size_t smem = adjoint_smem_bytes(DIM, sizeof(R) == 8 ? 0 : 1, lc.tile, lc.halo, lc.pitch);
        k_particles_adj_tiled<DIM, R><<<(unsigned)((long long)lc.max_items * nsplit), kThreads, smem, st>>>(
            a, lc.items, lc.n_items, lc.halo, nsplit);
        return cudaGetLastError();
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long blocks = (lc.total + 255) / 256;
    if (blocks > 16LL * sms) blocks = 16LL * sms;
    k_particles_adj<DIM, R><<<(unsigned)blocks, 256, 0, st>>>(a);
    return cudaGetLastError();
}

size_t adjoint_smem_bytes(int dims, int prec, const int tile[3], int halo, const int pitch[2])
{
    const size_t fe2 = dims == 3 ? (size_t)tile[2] + 2 * halo + 2 : 1;
    const size_t je2 = dims == 3 ? (size_t)tile[2] + 2 * halo + 4 : 1;
    const size_t plane = (size_t)pitch[0] * pitch[1];
    // FP64: E, B1, lambda_E, lambda_B1 (12 tiles) and lambda_J; FP32: E, B1,
    // the hi and lo words of lambda_E and lambda_B1 (12 int tiles) and lambda_J
    return prec == 0 ? (12 * plane * fe2 + 3 * plane * je2) * sizeof(double)
                     : (18 * plane * fe2 + 3 * plane * je2) * sizeof(float);
}

cudaError_t adjoint_set_smem_limit(int dims, int prec, size_t bytes)
{
    const int b = (int)bytes;
    if (dims == 3)
        return prec == 0
                   ? cudaFuncSetAttribute(k_particles_adj_tiled<3, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, b)
                   : cudaFuncSetAttribute(k_particles_adj_tiled<3, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    return prec == 0
               ? cudaFuncSetAttribute(k_particles_adj_tiled<2, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, b)
               : cudaFuncSetAttribute(k_particles_adj_tiled<2, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
}

cudaError_t launch_particles_adj(int dims, int prec, cudaStream_t st, const AdjLaunch &lc, const PoolBuf &P,
                                 void *const E[3], void *const B1[3], void *const lamJ[3], void *const lamE[3],
                                 void *const lamB1[3], void *const lamx[3], void *const lamw[3])
{
    if (dims == 3)
        return prec == 0 ? adj_part_t<3, double>(st, lc, P, E, B1, lamJ, lamE, lamB1, lamx, lamw)
                         : adj_part_t<3, float>(st, lc, P, E, B1, lamJ, lamE, lamB1, lamx, lamw);
    return prec == 0 ? adj_part_t<2, double>(st, lc, P, E, B1, lamJ, lamE, lamB1, lamx, lamw)
                     : adj_part_t<2, float>(st, lc, P, E, B1, lamJ, lamE, lamB1, lamx, lamw);
}

}  // namespace pic
