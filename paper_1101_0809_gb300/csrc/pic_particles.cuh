// pic_particles.cuh -- per-particle kernels of the charge-conserving PIC step
// (Sokolov, arXiv:1101.0809, Appendix step 2): alternating-order gather, push,
// move and virtual-path deposit, run over tile-sorted particles.
//
// One thread block takes one work item: a contiguous range of particles that
// the last sort put in one tile.  The block stages E and B of the tile plus a
// halo of (halo + 1) cells in shared memory, and a current tile with a halo of
// (halo + 2) cells.  Each thread streams particles (coalesced SoA loads),
// gathers from shared memory, pushes, renormalizes offset and cell, writes the
// particle back and scatters its face currents into the shared current tile
// with shared-memory atomics: 54 (3D) or 21 (2D) for a particle that kept its
// cell, at once; up to 144 or 40 for one that changed cell, through its warp's
// queue, drained 32 particles at a time.  A particle that has drifted
// more than `halo` cells outside the tile since the last sort takes the same
// arithmetic on the global arrays instead (periodic indices, global atomics).
// At the end the block adds its current tile to the global J with atomics.
#pragma once

#include <cooperative_groups.h>

#include "pic_internal.h"

namespace cg = cooperative_groups;

namespace pic {

template <typename R>
struct PartArgs {
    const WorkItem *items;
    const int *n_items;
    const RunDev *runs;
    const GroupDev *groups;
    Pool<R> P;
    // MODE 0 right after a sort: the particles are read from S, particle p of
    // the new order at S[perm[p]], and written to P; otherwise S = P, perm null
    Pool<R> S;
    const unsigned *perm;
    Fields<R> F;
    int *old_cell;
    R *old_off[3];
    int halo;
    int *err;   // err[0]: error word; err[1]: particles that ran past their tile's halo (counted by MODES 0, 1)
};

extern __shared__ __align__(16) unsigned char g_smem[];

// Tile geometry of the particle kernels: extents T0 x T1 x T2, halo G and the
// shared tiles' x and y pitches P0, P1.  GeoDyn reads them from the run and the
// launch; a GeoFix kernel has them as constants, so that every shared-memory
// offset of the gather and the deposit is an immediate.  The host launches a
// GeoFix kernel only when the grid's geometry equals it (pic_particles_fixed.cu).
struct GeoDyn {
    static constexpr bool dyn = true;
    static constexpr int T0 = 0, T1 = 0, T2 = 0, G = 0, P0 = 0, P1 = 0;
};
template <int t0, int t1, int t2, int g, int p0, int p1>
struct GeoFix {
    static constexpr bool dyn = false;
    static constexpr int T0 = t0, T1 = t1, T2 = t2, G = g, P0 = p0, P1 = p1;
};


// Per-warp deposit queue of particles that changed cell: capacity (a warp adds
// at most 32 entries to fewer than 32) and the values kept per entry (old and
// new offsets, u_z in 2D) besides one packed int (tile base << 8 | shifts + 1).
constexpr int kQueueCap = 64;
constexpr int kQueueVals = 7;

__device__ __forceinline__ bool finite3(float a, float b, float c) { return isfinite(a) && isfinite(b) && isfinite(c); }
__device__ __forceinline__ bool finite3(double a, double b, double c) { return isfinite(a) && isfinite(b) && isfinite(c); }

// Tile-local coordinate of global index i for a tile starting at o with extent T:
// the periodic image in [-G, T+G) if there is one (the grid is wider than the
// staged region, so at most one image lies there), else a value outside it.
__device__ __forceinline__ int local_coord(int i, int o, int T, int G, int n)
{
    int l = i - o;
    if (l >= T + G) l -= n;
    if (l < -G) l += n;
    return l;
}

// Rare path: a particle more than `halo` cells outside its tile since the
// last sort.  Same arithmetic on the periodic global arrays; kept out of line
// so that it does not raise the register count of the tiled path.
template <int DIM, typename R>
__device__ __noinline__ void gather_global(const Fields<R> &F, long long cb, int i, int j, int k, int nx, int ny,
                                           int nz, const R *w6, R *Ep, R *Bp)
{
    GlobalReader<R> rd;
    for (int c = 0; c < 3; ++c) { rd.E[c] = F.E[c]; rd.B[c] = F.B[c]; }
    for (int q = 0; q < 4; ++q) {
        rd.xi[q] = cb + wrapi(i - 1 + q, nx);
        rd.yj[q] = (long long)nx * wrapi(j - 1 + q, ny);
        rd.zk[q] = DIM == 3 ? (long long)nx * ny * wrapi(k - 1 + q, nz) : 0;
    }
    R fx[2] = {w6[0], w6[1]}, fy[2] = {w6[5], w6[6]}, fz[2] = {w6[10], w6[11]};
    R Sx[3] = {w6[2], w6[3], w6[4]}, Sy[3] = {w6[7], w6[8], w6[9]}, Sz[3] = {w6[12], w6[13], w6[14]};
    gather<DIM>(rd, fx, Sx, fy, Sy, fz, Sz, Ep, Bp);
}

// full: bit a set when the particle changed cell along axis a (its window
// there has four cells and three faces; along the other axes the fourth cell
// and the third face carry nothing and are skipped, as on the tiled path)
template <int DIM, typename R>
__device__ __noinline__ void deposit_global(const Fields<R> &F, long long cb, int i, int j, int k, int nx, int ny,
                                            int nz, const AxisWin<R> *win, const R *kf, R uz, int full)
{
    const AxisWin<R> X = win[0], Y = win[1], Z = win[2];
    GlobalAcc<R, 4> acc;
    for (int c = 0; c < 3; ++c) acc.J[c] = F.J[c];
    acc.set(cb, i, j, k, nx, ny, nz, X.lo, Y.lo, Z.lo, DIM == 3);
    deposit<DIM>(acc, X, Y, Z, kf, uz, full);
}

// The same for l_a = 2 1/2; (i, j, k) is the particle's base index.
template <int DIM, typename R>
__device__ __noinline__ void gather_global5(const Fields<R> &F, long long cb, int i, int j, int k, int nx, int ny,
                                            int nz, const R *w, R *Ep, R *Bp)
{
    GlobalReader5<R> rd;
    for (int c = 0; c < 3; ++c) { rd.E[c] = F.E[c]; rd.B[c] = F.B[c]; }
    for (int q = 0; q < 5; ++q) {
        rd.xi[q] = cb + wrapi(i - 2 + q, nx);
        rd.yj[q] = (long long)nx * wrapi(j - 2 + q, ny);
        rd.zk[q] = DIM == 3 ? (long long)nx * ny * wrapi(k - 2 + q, nz) : 0;
    }
    // w: f (3) and S (4) per axis
    gather5<DIM>(rd, w, w + 3, w + 7, w + 10, w + 14, w + 17, Ep, Bp);
}

template <int DIM, typename R>
__device__ __noinline__ void deposit_global5(const Fields<R> &F, long long cb, int i, int j, int k, int nx, int ny,
                                             int nz, const AxisWin5<R> *win, const R *kf, R uz, int full)
{
    const AxisWin5<R> X = win[0], Y = win[1], Z = win[2];
    GlobalAcc<R, 5> acc;
    for (int c = 0; c < 3; ++c) acc.J[c] = F.J[c];
    acc.set(cb, i, j, k, nx, ny, nz, X.lo, Y.lo, Z.lo, DIM == 3);
    deposit5<DIM>(acc, X, Y, Z, kf, uz, full);
}

// The comparison scheme of Eq. wrong1 on the global arrays; (i, j, k) is the cell.
template <int DIM, typename R>
__device__ __noinline__ void gather_global_w1(const Fields<R> &F, long long cb, int i, int j, int k, int nx, int ny,
                                              int nz, const R *S, R *Ep, R *Bp)
{
    GlobalReader5<R> rd;
    for (int c = 0; c < 3; ++c) { rd.E[c] = F.E[c]; rd.B[c] = F.B[c]; }
    for (int q = 0; q < 5; ++q) {
        rd.xi[q] = cb + wrapi(i - 2 + q, nx);
        rd.yj[q] = (long long)nx * wrapi(j - 2 + q, ny);
        rd.zk[q] = DIM == 3 ? (long long)nx * ny * wrapi(k - 2 + q, nz) : 0;
    }
    gather_w1<DIM>(rd, S, S + 3, S + 6, Ep, Bp);
}

// MODE 0: fused gather + push + move + deposit (pic_step).
// MODE 1: gather + push + move, keeping x^n (pic_gather_push).
// MODE 2: deposit from the kept x^n and the current x^{n+1} (pic_deposit_current).
// Shared memory: E and B tiles (6 * nf values of R) for MODES 0, 1; the current
// tile for MODES 0, 2: in FP32 two int32 fixed-point words per value, in FP64
// one double -- 24 * nj bytes either way.
// ORD = 3 is l_a = 1 1/2, ORD = 5 is l_a = 2 1/2 (Sec. 4.5): its stencil
// reaches one cell further, so the field tile has a halo of (halo + 2) cells
// and the current tile one of (halo + 3), and every particle deposits through
// the bias-removing accumulator (the per-cell counts serve the l_a = 1 1/2
// stencil only).  ORD = 4 is the comparison scheme of Eq. wrong1: its gather
// reaches the integer points -1..2 (field tile halo (halo + 2)); its charge and
// current are those of l_a = 1 1/2.
template <int DIM, typename R, int MODE, class GEO, int ORD = 3, bool PERM = false>
__device__ __forceinline__ void process_item(const PartArgs<R> &a, int item)
{
    // MODE 0 right after a sort whose arrays have not moved: the state comes
    // from a.S through a.perm, and the stepped particle goes to its new slot
    constexpr bool RP = PERM && MODE == 0;
    constexpr bool FIX = sizeof(R) == 4;
    const WorkItem it = a.items[item];
    const GroupDev gr = a.groups[it.group];
    const RunDev rn = a.runs[gr.run];
    const int G = GEO::dyn ? a.halo : GEO::G;
    const int nx = rn.n[0], ny = rn.n[1], nz = rn.n[2];
    const int T0 = GEO::dyn ? rn.tile[0] : GEO::T0, T1 = GEO::dyn ? rn.tile[1] : GEO::T1;
    const int T2 = DIM == 3 ? (GEO::dyn ? rn.tile[2] : GEO::T2) : 1;
    const int tx = it.tile % rn.ntile[0];
    const int ty = (it.tile / rn.ntile[0]) % rn.ntile[1];
    const int tz = DIM == 3 ? it.tile / (rn.ntile[0] * rn.ntile[1]) : 0;
    const int ox = tx * T0, oy = ty * T1, oz = tz * T2;
    constexpr int FH = ORD == 3 ? 1 : 2, JH = ORD == 5 ? 3 : 2;   // field and current halo beyond G
    const int fe0 = T0 + 2 * (G + FH), fe1 = T1 + 2 * (G + FH), fe2 = DIM == 3 ? T2 + 2 * (G + FH) : 1;
    const int je0 = T0 + 2 * (G + JH), je1 = T1 + 2 * (G + JH), je2 = DIM == 3 ? T2 + 2 * (G + JH) : 1;
    // the field tile is stored with the current tile's x and y pitches, so that
    // a particle's field and current bases differ by a constant and one bank
    // order of the particles (set by the tile sort) serves both
    const int P0 = GEO::dyn ? rn.pitch[0] : GEO::P0;   // >= je0 (see the tile layout choice)
    const int P1 = GEO::dyn ? rn.pitch[1] : GEO::P1;   // >= je1
    const int nf = P0 * P1 * fe2, nj = P0 * P1 * je2;
    // l_a = 2 1/2, FP32: particles whose base index stayed add raw words and the
    // bias comes off at the flush, which sums 64 counts per word of the current
    // tile.  That pays when the item has at least about 2/3 of a particle per
    // word (each such particle saves two integer subtractions on each of its
    // 144 contributions); sparser items take the bias off per contribution.
    // The choice is uniform over the block.
    const bool fix5 = FIX && ORD == 5 && (it.end - it.begin) * 3 >= 2LL * nj;
    constexpr bool NEED_F = MODE != 2;
    constexpr bool NEED_J = MODE != 1;
    const long long cb = rn.cell_base;

    R *sE[3], *sB[3];
    R *sJ[3];          // FP64 current tile
    int *sJh[3], *sJl[3];   // FP32 fixed-point current tile
    int *scnt = nullptr;    // FP32: particles that stayed in their cell, per base cell
    {
        unsigned char *sp = g_smem;
        if (NEED_F) {
            R *f = reinterpret_cast<R *>(sp);
            for (int c = 0; c < 3; ++c) { sE[c] = f + c * nf; sB[c] = f + (3 + c) * nf; }
            sp += 6 * (size_t)nf * sizeof(R);
        }
        if (NEED_J) {
            for (int c = 0; c < 3; ++c) {
                sJ[c] = reinterpret_cast<R *>(sp) + c * nj;
                sJh[c] = reinterpret_cast<int *>(sp) + c * nj;
                sJl[c] = reinterpret_cast<int *>(sp) + (3 + c) * nj;
            }
            if (FIX) scnt = reinterpret_cast<int *>(sp) + 6 * nj;
        }
    }

    if (NEED_F) {
        for (int l = threadIdx.x; l < nf; l += blockDim.x) {
            const int lx = l % P0, r = l / P0, ly = r % P1, lz = r / P1;
            if (lx >= fe0 || ly >= fe1) continue;   // pitch padding
            const int gx = wrapi(ox - G - FH + lx, nx);
            const int gy = wrapi(oy - G - FH + ly, ny);
            const int gz = DIM == 3 ? wrapi(oz - G - FH + lz, nz) : 0;
            const long long gi = cb + gx + (long long)nx * (gy + (long long)ny * gz);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                sE[c][l] = a.F.E[c][gi];
                sB[c][l] = a.F.B[c][gi];
            }
        }
    }
    if (NEED_J) {
        int *z = sJh[0];   // 24 * nj bytes = 6 * nj words in both precisions, + nj counts in FP32
        for (int l = threadIdx.x; l < (FIX ? 7 : 6) * nj; l += blockDim.x) z[l] = 0;
    }
    __syncthreads();

    // constants of the group and run, prepared on the host (no FP64 arithmetic
    // runs in the FP32 kernels)
    R hq, cl, cN0, cN1, cN2;
    R kf[3], kfs[3];   // kfs: prefactors with the fixed-point scale of the FP32 current tile folded in
    if constexpr (FIX) {
        hq = gr.hqf;
        cl = rn.cf;
        cN0 = rn.cNf[0]; cN1 = rn.cNf[1]; cN2 = rn.cNf[2];
        for (int c = 0; c < 3; ++c) { kf[c] = gr.kff[c]; kfs[c] = gr.kfsf[c]; }
    } else {
        hq = gr.hq;
        cl = rn.c;
        cN0 = rn.cN[0]; cN1 = rn.cN[1]; cN2 = rn.cN[2];
        for (int c = 0; c < 3; ++c) { kf[c] = gr.kf[c]; kfs[c] = gr.kf[c]; }
    }
    const R c2 = cl * cl;

    // Deposit queue of this warp (MODES 0, 2).  A particle that stayed in its
    // cell along every axis deposits at once with three-cell windows (54
    // contributions in 3D, 21 in 2D), where its lane's bank is the one the tile
    // sort gave it.  A particle that changed cell needs four-cell windows along
    // the axes it crossed; it is queued and deposited later together with 31
    // other such particles, so that the wider windows are paid only by warps
    // of moved particles.  The integer current sums do not depend on the order.
    // The warps' queues lie one after another (values, then codes), followed by
    // one count per warp for the merged drain at the end of the item.
    R *qv0 = nullptr, *qv = nullptr;
    int *qs0 = nullptr, *qs = nullptr, *qcnt = nullptr;
    if (NEED_J) {
        unsigned char *qb = g_smem + (NEED_F ? 6 * (size_t)nf * sizeof(R) : 0) + (FIX ? 28 : 24) * (size_t)nj;
        const int warp = threadIdx.x >> 5;
        qv0 = reinterpret_cast<R *>(qb);
        qs0 = reinterpret_cast<int *>(qb + (size_t)(kThreads / 32) * kQueueCap * kQueueVals * sizeof(R));
        qcnt = qs0 + (kThreads / 32) * kQueueCap;
        qv = qv0 + (size_t)warp * kQueueCap * kQueueVals;
        qs = qs0 + warp * kQueueCap;
    }
    const int lane = threadIdx.x & 31;
    int qn = 0;   // entries in this warp's queue (warp-uniform)


    auto deposit_local = [&](int base, const AxisWin<R> &X, const AxisWin<R> &Y, const AxisWin<R> &Z, R uz,
                             int full) {
        if constexpr (FIX) {
            FixedAcc acc;   // bias taken off per contribution (variable stencil)
            for (int c = 0; c < 3; ++c) { acc.hi[c] = sJh[c]; acc.lo[c] = sJl[c]; }
            acc.base = base;
            acc.s1 = P0;
            acc.s2 = P0 * P1;
            deposit<DIM>(acc, X, Y, Z, kfs, uz, full);
        } else {
            SmemAcc<R> acc;
            for (int c = 0; c < 3; ++c) acc.J[c] = sJ[c];
            acc.base = base;
            acc.s1 = P0;
            acc.s2 = P0 * P1;
            deposit<DIM>(acc, X, Y, Z, kf, uz, full);
        }
    };
    auto deposit_local5 = [&](int base, const AxisWin5<R> &X, const AxisWin5<R> &Y, const AxisWin5<R> &Z, R uz,
                              int full) {
        if constexpr (FIX) {
            FixedAcc acc;
            for (int c = 0; c < 3; ++c) { acc.hi[c] = sJh[c]; acc.lo[c] = sJl[c]; }
            acc.base = base;
            acc.s1 = P0;
            acc.s2 = P0 * P1;
            deposit5<DIM>(acc, X, Y, Z, kfs, uz, full);
        } else {
            SmemAcc<R> acc;
            for (int c = 0; c < 3; ++c) acc.J[c] = sJ[c];
            acc.base = base;
            acc.s1 = P0;
            acc.s2 = P0 * P1;
            deposit5<DIM>(acc, X, Y, Z, kf, uz, full);
        }
    };
    // deposits, on each lane with `on`, entry `slot` of the queue whose values
    // and codes start at sv and ss (a whole warp calls it)
    auto drain = [&](const R *sv, const int *ss, int slot, bool on) {
        R d0 = R(0), d1 = R(0), d2 = R(0), e0 = R(0), e1 = R(0), e2 = R(0), u = R(0);
        int code = 1 | (1 << 2) | (1 << 4);
        if (on) {
            d0 = sv[0 * kQueueCap + slot];
            d1 = sv[1 * kQueueCap + slot];
            e0 = sv[3 * kQueueCap + slot];
            e1 = sv[4 * kQueueCap + slot];
            if (DIM == 3) {
                d2 = sv[2 * kQueueCap + slot];
                e2 = sv[5 * kQueueCap + slot];
            } else {
                u = sv[6 * kQueueCap + slot];
            }
            code = ss[slot];
        }
        const int q0 = (code & 3) - 1, q1 = ((code >> 2) & 3) - 1, q2 = ((code >> 4) & 3) - 1;
        const int full = (__any_sync(0xffffffffu, q0 != 0) ? 1 : 0) | (__any_sync(0xffffffffu, q1 != 0) ? 2 : 0) |
                         (DIM == 3 && __any_sync(0xffffffffu, q2 != 0) ? 4 : 0);
        if (on) {
            if constexpr (ORD == 5) {   // the entries hold the l_a = 2 1/2 d values
                AxisWin5<R> X, Y, Z;
                axis_window5(d0, e0, q0, X);
                axis_window5(d1, e1, q1, Y);
                if (DIM == 3) axis_window5(d2, e2, q2, Z); else Z = X;
                deposit_local5(code >> 8, X, Y, Z, u, full);
            } else {
                AxisWin<R> X, Y, Z;
                axis_window(d0, e0, q0, X);
                axis_window(d1, e1, q1, Y);
                if (DIM == 3) axis_window(d2, e2, q2, Z); else Z = X;
                deposit_local(code >> 8, X, Y, Z, u, full);
            }
        }
    };

    // warps run whole rounds of 32 consecutive particles (the last one partial)
    // RP: the permutation index of the lane's next particle is read one round ahead
    unsigned sp_next = 0;
    if (RP && it.begin + threadIdx.x < it.end) sp_next = a.perm[it.begin + threadIdx.x];
    for (long long pw = it.begin + (threadIdx.x & ~31); pw < it.end; pw += blockDim.x) {
        const long long p = pw + lane;
        const bool valid = p < it.end;
        unsigned sp_cur = 0;
        if (RP) {
            sp_cur = sp_next;
            if (p + blockDim.x < it.end) sp_next = a.perm[p + blockDim.x];
        }
        bool live = false;   // the particle moves and deposits this step
        bool inr = false;
        int i = 0, j = 0, k = 0, li = 0, lj = 0, lk = 0;
        R o0 = R(0), o1 = R(0), o2 = R(0), n0 = R(0), n1 = R(0), n2 = R(0), uz = R(0);
        int s0 = 0, s1 = 0, s2 = 0;
        if (valid) {
            // ---- the particle's state at x^n (old) -------------------------------
            const long long sp = RP ? (long long)sp_cur : p;   // where the state is read
            const Pool<R> &src = RP ? a.S : a.P;
            const int cell0 = MODE == 2 ? a.old_cell[p] : src.cell[sp];
            o0 = MODE == 2 ? a.old_off[0][p] : src.off[0][sp];
            o1 = MODE == 2 ? a.old_off[1][p] : src.off[1][sp];
            o2 = DIM == 3 ? (MODE == 2 ? a.old_off[2][p] : src.off[2][sp]) : R(0);
            R w[3] = {R(0), R(0), R(0)};
            if (MODE != 2 || DIM == 2) {
                w[0] = src.w[0][sp];
                w[1] = src.w[1][sp];
                w[2] = src.w[2][sp];
            }

            const int rest = divu31(cell0, rn.div_nx);
            i = cell0 - rest * nx;
            if (DIM == 3) {
                k = divu31(rest, rn.div_ny);
                j = rest - k * ny;
            } else {
                j = rest;
            }
            li = local_coord(i, ox, T0, G, nx);
            lj = local_coord(j, oy, T1, G, ny);
            lk = DIM == 3 ? local_coord(k, oz, T2, G, nz) : 0;
            inr = li >= -G && li < T0 + G && lj >= -G && lj < T1 + G && (DIM == 2 || (lk >= -G && lk < T2 + G));

            n0 = o0; n1 = o1; n2 = o2;
            live = true;
            if (MODE != 2) {
                R Ep[3], Bp[3];
                if constexpr (ORD == 5) {
                    R e0, e1, e2 = R(0.5);
                    const int u0 = split5(o0, e0), u1 = split5(o1, e1), u2 = DIM == 3 ? split5(o2, e2) : 0;
                    R w[21];   // f (3) and S (4) along x, y, z
                    form_factor5(e0, w, w + 3);
                    form_factor5(e1, w + 7, w + 10);
                    form_factor5(e2, w + 14, w + 17);
                    if (inr) {
                        SmemReader<R> rd;
                        for (int c = 0; c < 3; ++c) { rd.E[c] = sE[c]; rd.B[c] = sB[c]; }
                        rd.base = (li + u0 + G + FH) +
                                  P0 * ((lj + u1 + G + FH) + (DIM == 3 ? P1 * (lk + u2 + G + FH) : 0));
                        rd.s1 = P0;
                        rd.s2 = P0 * P1;
                        gather5<DIM>(rd, w, w + 3, w + 7, w + 10, w + 14, w + 17, Ep, Bp);
                    } else {
                        gather_global5<DIM, R>(a.F, cb, i + u0, j + u1, k + u2, nx, ny, nz, w, Ep, Bp);
                    }
                } else if constexpr (ORD == 4) {
                    R f[2], S[9] = {R(0), R(1), R(0), R(0), R(1), R(0), R(0), R(1), R(0)};   // S along x, y, z
                    form_factor(o0, f, S);
                    form_factor(o1, f, S + 3);
                    if (DIM == 3) form_factor(o2, f, S + 6);
                    if (inr) {
                        SmemReader<R> rd;
                        for (int c = 0; c < 3; ++c) { rd.E[c] = sE[c]; rd.B[c] = sB[c]; }
                        rd.base = (li + G + FH) + P0 * ((lj + G + FH) + (DIM == 3 ? P1 * (lk + G + FH) : 0));
                        rd.s1 = P0;
                        rd.s2 = P0 * P1;
                        gather_w1<DIM>(rd, S, S + 3, S + 6, Ep, Bp);
                    } else {
                        gather_global_w1<DIM, R>(a.F, cb, i, j, k, nx, ny, nz, S, Ep, Bp);
                    }
                } else {
                    R fx[2], Sx[3], fy[2], Sy[3], fz[2], Sz[3];
                    form_factor(o0, fx, Sx);
                    form_factor(o1, fy, Sy);
                    if (DIM == 3) {
                        form_factor(o2, fz, Sz);
                    } else {
                        fz[0] = R(1); fz[1] = R(0);
                        Sz[0] = R(0); Sz[1] = R(1); Sz[2] = R(0);
                    }
                    if (inr) {
                        SmemReader<R> rd;
                        for (int c = 0; c < 3; ++c) { rd.E[c] = sE[c]; rd.B[c] = sB[c]; }
                        rd.base = (li + G + 1) + P0 * ((lj + G + 1) + (DIM == 3 ? P1 * (lk + G + 1) : 0));
                        rd.s1 = P0;
                        rd.s2 = P0 * P1;
                        gather<DIM>(rd, fx, Sx, fy, Sy, fz, Sz, Ep, Bp);
                    } else {
                        R w6[15] = {fx[0], fx[1], Sx[0], Sx[1], Sx[2], fy[0], fy[1], Sy[0], Sy[1], Sy[2],
                                    fz[0], fz[1], Sz[0], Sz[1], Sz[2]};
                        gather_global<DIM, R>(a.F, cb, i, j, k, nx, ny, nz, w6, Ep, Bp);
                    }
                }
                boris(w, Ep, Bp, hq, c2);
                if (!finite3(w[0], w[1], w[2])) {
                    atomicOr(a.err, ERR_NONFINITE);
                    live = false;   // the particle keeps x^n and contributes no current
                    if (RP) {   // ... in its slot of the new order, with the momentum it reached
                        a.P.id[p] = a.S.id[sp];
                        a.P.cell[p] = cell0;
                        a.P.off[0][p] = o0;
                        a.P.off[1][p] = o1;
                        if (DIM == 3) a.P.off[2][p] = o2;
                        for (int c = 0; c < 3; ++c) a.P.w[c][p] = w[c];
                    }
                } else {
                    const R ig = rsqrt_r(w[0] * w[0] + w[1] * w[1] + w[2] * w[2] + c2);
                    s0 = renormalize(o0, w[0] * ig * cN0, n0);
                    s1 = renormalize(o1, w[1] * ig * cN1, n1);
                    if (DIM == 3) s2 = renormalize(o2, w[2] * ig * cN2, n2);
                    uz = cl * w[2] * ig;
                    const int i1 = wrapi(i + s0, nx), j1 = wrapi(j + s1, ny), k1 = DIM == 3 ? wrapi(k + s2, nz) : 0;
                    const int cell1 = i1 + nx * (j1 + ny * k1);
                    if (MODE == 1) {
                        a.old_cell[p] = cell0;
                        a.old_off[0][p] = o0;
                        a.old_off[1][p] = o1;
                        if (DIM == 3) a.old_off[2][p] = o2;
                    }
                    if (RP) a.P.id[p] = a.S.id[sp];   // the id moves with the particle
                    a.P.cell[p] = cell1;
                    a.P.off[0][p] = n0;
                    a.P.off[1][p] = n1;
                    if (DIM == 3) a.P.off[2][p] = n2;
                    a.P.w[0][p] = w[0];
                    a.P.w[1][p] = w[1];
                    a.P.w[2][p] = w[2];
                }
            } else {
                // deposit-only: x^{n+1} is the stored state, the shift follows from the cells
                const int cell1 = a.P.cell[p];
                n0 = a.P.off[0][p];
                n1 = a.P.off[1][p];
                if (DIM == 3) n2 = a.P.off[2][p];
                const int r1 = divu31(cell1, rn.div_nx);
                const int i1 = cell1 - r1 * nx;
                const int k1 = DIM == 3 ? divu31(r1, rn.div_ny) : 0;
                const int j1 = r1 - k1 * ny;
                s0 = i1 - i; if (s0 > 1) s0 -= nx; if (s0 < -1) s0 += nx;
                s1 = j1 - j; if (s1 > 1) s1 -= ny; if (s1 < -1) s1 += ny;
                if (DIM == 3) { s2 = k1 - k; if (s2 > 1) s2 -= nz; if (s2 < -1) s2 += nz; }
                if (DIM == 2) {
                    const R ig = rsqrt_r(w[0] * w[0] + w[1] * w[1] + w[2] * w[2] + c2);
                    uz = cl * w[2] * ig;
                }
            }
        }
        if (MODE != 2) {   // particles on the global path: the sort policy's measure of drift
            const unsigned dm = __ballot_sync(0xffffffffu, valid && !inr);
            if (lane == 0 && dm != 0u) atomicAdd(reinterpret_cast<unsigned *>(a.err) + 1, (unsigned)__popc(dm));
        }
        if (MODE == 1) continue;

        // ---- virtual-path current (Eq. current) -------------------------------
        // The windows take the d values and shifts of the base index: for
        // l_a = 1 1/2 the offsets and cell shifts themselves; for l_a = 2 1/2 the
        // base index is cell + (offset >= 1/2), so it moves with the cell shift
        // and the half-offset flags.
        int q0 = s0, q1 = s1, q2 = s2;
        R a0 = o0, a1 = o1, a2 = o2, b0 = n0, b1 = n1, b2 = n2;
        int ub0 = 0, ub1 = 0, ub2 = 0;   // old base index - old cell
        if constexpr (ORD == 5) {
            ub0 = split5(o0, a0);
            ub1 = split5(o1, a1);
            const int v0 = split5(n0, b0), v1 = split5(n1, b1);
            q0 = s0 + v0 - ub0;
            q1 = s1 + v1 - ub1;
            if (DIM == 3) {
                ub2 = split5(o2, a2);
                q2 = s2 + split5(n2, b2) - ub2;
            }
        }
        const bool moved = (q0 | q1 | q2) != 0;
        const int base = (li + ub0 + G + JH) +
                         P0 * ((lj + ub1 + G + JH) + (DIM == 3 ? P1 * (lk + ub2 + G + JH) : 0));
        if (live && inr && !moved) {
            if constexpr (ORD == 5) {
                AxisWin5<R> X, Y, Z;
                axis_window5(a0, b0, 0, X);
                axis_window5(a1, b1, 0, Y);
                if (DIM == 3) axis_window5(a2, b2, 0, Z); else Z = X;
                if (fix5) {
                    // fixed stencil: the bias comes off once per word at the flush
                    FixedAccT<false> acc;
                    for (int c = 0; c < 3; ++c) { acc.hi[c] = sJh[c]; acc.lo[c] = sJl[c]; }
                    acc.base = base;
                    acc.s1 = P0;
                    acc.s2 = P0 * P1;
                    deposit5<DIM>(acc, X, Y, Z, kfs, uz, 0);
                    atomicAdd(&scnt[base], 1);
                } else {
                    deposit_local5(base, X, Y, Z, uz, 0);
                }
            } else {
                AxisWin<R> X, Y, Z;
                axis_window_still(o0, n0, X);
                axis_window_still(o1, n1, Y);
                if (DIM == 3) axis_window_still(o2, n2, Z); else Z = X;
                if constexpr (FIX) {
                    // fixed stencil: the bias comes off once per word at the flush
                    FixedAccT<false> acc;
                    for (int c = 0; c < 3; ++c) { acc.hi[c] = sJh[c]; acc.lo[c] = sJl[c]; }
                    acc.base = base;
                    acc.s1 = P0;
                    acc.s2 = P0 * P1;
                    deposit<DIM>(acc, X, Y, Z, kfs, uz, 0);
                    atomicAdd(&scnt[base], 1);
                } else {
                    deposit_local(base, X, Y, Z, uz, 0);
                }
            }
        } else if (live && !inr) {
            if constexpr (ORD == 5) {
                AxisWin5<R> win[3];
                axis_window5(a0, b0, q0, win[0]);
                axis_window5(a1, b1, q1, win[1]);
                if (DIM == 3) axis_window5(a2, b2, q2, win[2]); else win[2] = win[0];
                deposit_global5<DIM, R>(a.F, cb, i + ub0, j + ub1, k + ub2, nx, ny, nz, win, kf, uz,
                                        (q0 != 0 ? 1 : 0) | (q1 != 0 ? 2 : 0) | (q2 != 0 ? 4 : 0));
            } else {
                AxisWin<R> win[3];
                axis_window(o0, n0, s0, win[0]);
                axis_window(o1, n1, s1, win[1]);
                if (DIM == 3) axis_window(o2, n2, s2, win[2]); else win[2] = win[0];
                deposit_global<DIM, R>(a.F, cb, i, j, k, nx, ny, nz, win, kf, uz,
                                       (s0 != 0 ? 1 : 0) | (s1 != 0 ? 2 : 0) | (s2 != 0 ? 4 : 0));
            }
        }
        const bool enq = live && inr && moved;
        const unsigned qm = __ballot_sync(0xffffffffu, enq);
        if (enq) {
            const int slot = qn + __popc(qm & ((1u << lane) - 1u));
            qv[0 * kQueueCap + slot] = a0;
            qv[1 * kQueueCap + slot] = a1;
            qv[3 * kQueueCap + slot] = b0;
            qv[4 * kQueueCap + slot] = b1;
            if (DIM == 3) {
                qv[2 * kQueueCap + slot] = a2;
                qv[5 * kQueueCap + slot] = b2;
            } else {
                qv[6 * kQueueCap + slot] = uz;
            }
            qs[slot] = (base << 8) | (q0 + 1) | ((q1 + 1) << 2) | ((q2 + 1) << 4);
        }
        qn += __popc(qm);
        if (qn >= 32) {   // warp-uniform
            __syncwarp();
            qn -= 32;
            drain(qv, qs, qn + lane, true);
            __syncwarp();   // the drained slots are free again
        }
    }
    if (NEED_J) {
        // The entries left in the warps' queues (fewer than 32 each) are drained
        // together: merged entry m is slot m - (entries of the warps before) of
        // its warp's queue, and warp w deposits the merged entries
        // [32w, 32w + 32), [32w + 256, ...).  A block then runs about one
        // partly filled drain per item instead of one per warp.
        if (lane == 0) qcnt[threadIdx.x >> 5] = qn;
        __syncthreads();
        int tot = 0;
#pragma unroll
        for (int w = 0; w < kThreads / 32; ++w) tot += qcnt[w];
        for (int m0 = threadIdx.x & ~31; m0 < tot; m0 += blockDim.x) {   // uniform over the warp
            int src = 0, slot = m0 + lane;
#pragma unroll
            for (int w = 0; w < kThreads / 32 - 1; ++w) {
                const int c = qcnt[src];
                if (slot >= c) {
                    slot -= c;
                    ++src;
                }
            }
            const bool on = m0 + lane < tot;
            drain(qv0 + (size_t)(on ? src : 0) * kQueueCap * kQueueVals, qs0 + (on ? src : 0) * kQueueCap,
                  on ? slot : 0, on);
        }
        __syncthreads();
        const float jinv = gr.jinv;
        for (int l = threadIdx.x; l < nj; l += blockDim.x) {
            const int lx = l % P0, r = l / P0, ly = r % P1, lz = r / P1;
            if (lx >= je0 || ly >= je1) continue;   // pitch padding
            const int gx = wrapi(ox - G - JH + lx, nx);
            const int gy = wrapi(oy - G - JH + ly, ny);
            const int gz = DIM == 3 ? wrapi(oz - G - JH + lz, nz) : 0;
            const long long gi = cb + gx + (long long)nx * (gy + (long long)ny * gz);
            // FP32: contributions of particles that stayed in their cell, per
            // component: the stencil of such a particle with base b covers the
            // cells b + (dx, dy, dz) with dx in {0, 1} and dy, dz in {-1, 0, 1}
            // for J^x (faces 0, 1; cells -1..1), likewise for J^y and J^z, so a
            // cell l received sum_{b in l - stencil} cnt[b] of them
            unsigned nst[3] = {0u, 0u, 0u};
            if (fix5) {
                // l_a = 2 1/2: the stencil of base b covers b + (dx, dy, dz) with
                // dx in {-1, 0, 1} (faces) and dy, dz in {-2, ..., 1} (cells) for
                // J^x, likewise for J^y and J^z; so the bases of word l are
                // l + o, o in {-1, ..., 2} per axis, without the o_a = 2 plane for
                // J^a.  A base is the local cell (in [-G, T + G)) plus the
                // half-offset flag (0 or 1) plus G + JH, so bases lie in
                // [JH, T + 2G + JH] = [JH, je - JH] along each axis: only those
                // indices are read, which keeps every read in the tile.
                bool vx[4], vy[4], vz[4];
#pragma unroll
                for (int o = 0; o < 4; ++o) {
                    vx[o] = lx + o - 1 >= JH && lx + o - 1 <= je0 - JH;
                    vy[o] = ly + o - 1 >= JH && ly + o - 1 <= je1 - JH;
                    vz[o] = DIM == 3 ? (lz + o - 1 >= JH && lz + o - 1 <= je2 - JH) : o == 1;
                }
                unsigned tot = 0, px = 0, py = 0, pz = 0;   // all, and the o = 2 planes
#pragma unroll
                for (int oz = -1; oz <= (DIM == 3 ? 2 : -1); ++oz)
#pragma unroll
                    for (int oy = -1; oy <= 2; ++oy)
#pragma unroll
                        for (int ox = -1; ox <= 2; ++ox) {
                            const int dz = DIM == 3 ? oz : 0;
                            if (!(vx[ox + 1] && vy[oy + 1] && vz[dz + 1])) continue;
                            const unsigned v = (unsigned)scnt[l + ox + P0 * (oy + P1 * dz)];
                            tot += v;
                            if (ox == 2) px += v;
                            if (oy == 2) py += v;
                            if (DIM == 3 && oz == 2) pz += v;
                        }
                nst[0] = tot - px;
                nst[1] = tot - py;
                nst[2] = tot - pz;
            }
            if constexpr (FIX && ORD != 5) {
                if (lx >= 1 && lx < je0 - 1 && ly >= 1 && ly < je1 - 1 && (DIM == 2 || (lz >= 1 && lz < je2 - 1))) {
                    if (DIM == 3) {
                        unsigned tot = 0, px = 0, py = 0, pz = 0;   // all 27, and the +1 planes
#pragma unroll
                        for (int oz = -1; oz <= 1; ++oz)
#pragma unroll
                            for (int oy = -1; oy <= 1; ++oy)
#pragma unroll
                                for (int ox = -1; ox <= 1; ++ox) {
                                    const unsigned v = (unsigned)scnt[l + ox + P0 * (oy + P1 * oz)];
                                    tot += v;
                                    if (ox == 1) px += v;
                                    if (oy == 1) py += v;
                                    if (oz == 1) pz += v;
                                }
                        nst[0] = tot - px;
                        nst[1] = tot - py;
                        nst[2] = tot - pz;
                    } else {
                        unsigned tot = 0, px = 0, py = 0;
#pragma unroll
                        for (int oy = -1; oy <= 1; ++oy)
#pragma unroll
                            for (int ox = -1; ox <= 1; ++ox) {
                                const unsigned v = (unsigned)scnt[l + ox + P0 * oy];
                                tot += v;
                                if (ox == 1) px += v;
                                if (oy == 1) py += v;
                            }
                        nst[0] = tot - px;
                        nst[1] = tot - py;
                        nst[2] = tot;
                    }
                }
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                if constexpr (FIX) {
                    const unsigned off = nst[c] * kFixBias;
                    const int h = (int)((unsigned)sJh[c][l] - off), lo = (int)((unsigned)sJl[c][l] - off);
                    if ((h | lo) != 0)
                        atomicAdd(&a.F.J[c][gi], (R)(fmaf((float)h, 65536.0f, (float)lo) * jinv));
                } else {
                    const R v = sJ[c][l];
                    if (v != R(0)) atomicAdd(&a.F.J[c][gi], v);
                }
            }
        }
    }
    __syncthreads();   // the shared tiles are free for the block's next item
}

template <int DIM, typename R, int MODE, class GEO = GeoDyn, int ORD = 3, bool PERM = false>
__global__ void __launch_bounds__(kThreads) k_particles(const PartArgs<R> a)
{
    if ((int)blockIdx.x >= *a.n_items) return;
    process_item<DIM, R, MODE, GEO, ORD, PERM>(a, blockIdx.x);
}

// Run of a batch that owns concatenated cell l (run_cell_base has nruns + 1 entries).
__device__ __forceinline__ int find_run(const long long *run_cell_base, int nruns, long long l)
{
    int lo = 0, hi = nruns;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (run_cell_base[mid] <= l) lo = mid; else hi = mid;
    }
    return lo;
}

// One whole step of every run of a batch in one cooperative launch: B half
// step (+ J clear) over all cells, grid barrier, the fused particle work items,
// grid barrier, B half step, grid barrier, E full step.  The grid is sized so
// that all blocks are resident (cooperative launch), which the barriers need.
// PERM: the step right after a sort that left the arrays in place; the work
// items read the particles through the permutation (as k_particles does).
template <int DIM, typename R, class GEO = GeoDyn, bool PERM = false>
__global__ void __launch_bounds__(kThreads) k_step_persistent(const PartArgs<R> a, int nruns,
                                                              const long long *run_cell_base, long long *ant_n,
                                                              int antennas)
{
    cg::grid_group grid = cg::this_grid();
    const long long total = run_cell_base[nruns];
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    for (long long l = t0; l < total; l += stride) {
        const int r = find_run(run_cell_base, nruns, l);
        yee_b_half_cell<DIM, R>(a.runs[r], a.F, l - run_cell_base[r], 1, ant_n[r]);
    }
    grid.sync();
    const int ni = *a.n_items;
    for (int it = blockIdx.x; it < ni; it += gridDim.x) process_item<DIM, R, 0, GEO, 3, PERM>(a, it);
    grid.sync();
    for (long long l = t0; l < total; l += stride) {
        const int r = find_run(run_cell_base, nruns, l);
        yee_b_half_cell<DIM, R>(a.runs[r], a.F, l - run_cell_base[r], 0, ant_n[r]);
    }
    grid.sync();
    for (long long l = t0; l < total; l += stride) {
        const int r = find_run(run_cell_base, nruns, l);
        yee_e_cell<DIM, R>(a.runs[r], a.F, l - run_cell_base[r], ant_n[r]);
    }
    if (antennas) {   // the antenna clocks advance once every block has read them
        grid.sync();
        if (blockIdx.x == 0)
            for (int r = threadIdx.x; r < nruns; r += blockDim.x) ant_n[r] += 1;
    }
}

template <int DIM, typename R, int MODE, class GEO = GeoDyn, int ORD = 3>
static cudaError_t launch_t(cudaStream_t st, int max_items, size_t smem, const PartArgs<R> &a)
{
    if (max_items <= 0) return cudaSuccess;
    if constexpr (MODE == 0 && ORD == 3) {
        if (a.perm) {   // right after a sort: the kernel that reads through the permutation
            k_particles<DIM, R, 0, GEO, 3, true><<<max_items, kThreads, smem, st>>>(a);
            return cudaGetLastError();
        }
    }
    k_particles<DIM, R, MODE, GEO, ORD><<<max_items, kThreads, smem, st>>>(a);
    return cudaGetLastError();
}

// The shared-memory limit of the fused kernel of a geometry, both variants.
template <int DIM, typename R, class GEO>
static cudaError_t set_limit_fused(int bytes)
{
    cudaError_t e = cudaFuncSetAttribute(k_particles<DIM, R, 0, GEO>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_particles<DIM, R, 0, GEO, 3, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                bytes);
}

template <int DIM, typename R, class GEO = GeoDyn>
static cudaError_t persistent_t(cudaStream_t st, size_t smem, int nruns, const long long *run_cell_base,
                                PartArgs<R> a, int *grid_blocks, int launch, long long *ant_n, int antennas)
{
    auto fn0 = k_step_persistent<DIM, R, GEO, false>;
    auto fn1 = k_step_persistent<DIM, R, GEO, true>;
    auto fn = a.perm ? fn1 : fn0;
    cudaError_t e;
    if (*grid_blocks <= 0) {
        // first use (outside any stream capture): shared-memory limit and grid
        // size, the same for both variants (all blocks of either must be resident)
        int dev = 0, sms = 0, per = 1 << 30;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        for (auto f : {fn0, fn1}) {
            e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            int pf = 0;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pf, f, kThreads, smem);
            if (e != cudaSuccess) return e;
            per = std::min(per, pf);
        }
        if (per <= 0) return cudaErrorInvalidConfiguration;
        *grid_blocks = sms * per;
    }
    if (!launch) return cudaSuccess;
    void *args[] = {(void *)&a, (void *)&nruns, (void *)&run_cell_base, (void *)&ant_n, (void *)&antennas};
    return cudaLaunchCooperativeKernel((const void *)fn, dim3(*grid_blocks), dim3(kThreads), args, smem, st);
}

// Kernel arguments from the host-side buffers.
template <typename R>
inline PartArgs<R> make_args(const WorkItem *items, const int *n_items, const RunDev *runs, const GroupDev *groups,
                             const PoolBuf &P, void *const E[3], void *const B[3], void *const J[3], int *old_cell,
                             void *const old_off[3], int halo, int *err, const PoolBuf *S = nullptr,
                             const unsigned *perm = nullptr)
{
    PartArgs<R> a;
    a.items = items;
    a.n_items = n_items;
    a.runs = runs;
    a.groups = groups;
    a.P.cell = P.cell;
    a.P.id = P.id;
    const PoolBuf &Q = S ? *S : P;
    a.S.cell = Q.cell;
    a.S.id = Q.id;
    a.perm = S ? perm : nullptr;
    for (int c = 0; c < 3; ++c) {
        a.S.off[c] = static_cast<R *>(Q.off[c]);
        a.S.w[c] = static_cast<R *>(Q.w[c]);
        a.P.off[c] = static_cast<R *>(P.off[c]);
        a.P.w[c] = static_cast<R *>(P.w[c]);
        a.F.E[c] = static_cast<R *>(E[c]);
        a.F.B[c] = static_cast<R *>(B[c]);
        a.F.J[c] = static_cast<R *>(J[c]);
        a.old_off[c] = static_cast<R *>(old_off[c]);
    }
    a.old_cell = old_cell;
    a.halo = halo;
    a.err = err;
    return a;
}

// Kernels with a fixed tile geometry (pic_particles_fixed.cu), FP32 fused step
// and persistent batch step.  Each returns false, without launching, when no
// fixed kernel has the grid's geometry.
bool launch_particles_fixed(int dims, cudaStream_t st, int max_items, size_t smem, const PartArgs<float> &a,
                            const int tile[3], int halo, int p0, int p1, cudaError_t *err);
bool launch_persistent_fixed(int dims, cudaStream_t st, size_t smem, int nruns, const long long *run_cell_base,
                             const PartArgs<float> &a, int *grid_blocks, int launch, const int tile[3], int halo,
                             int p0, int p1, long long *ant_n, int antennas, cudaError_t *err);
cudaError_t fixed_set_smem_limit(int dims, size_t bytes);

// Launch and shared-memory limit of the kernels of another stencil (ORD = 5:
// l_a = 2 1/2 in pic_particles_o5.cu; ORD = 4: Eq. wrong1 in pic_particles_w1.cu),
// any tile geometry, both precisions, all three modes.
template <int DIM, typename R, int ORD>
static cudaError_t launch_mode_ord(int mode, cudaStream_t st, int max_items, size_t smem, const PartArgs<R> &a)
{
    switch (mode) {
    case 0: return launch_t<DIM, R, 0, GeoDyn, ORD>(st, max_items, smem, a);
    case 1: return launch_t<DIM, R, 1, GeoDyn, ORD>(st, max_items, smem, a);
    default: return launch_t<DIM, R, 2, GeoDyn, ORD>(st, max_items, smem, a);
    }
}

template <int ORD>
static cudaError_t launch_particles_ord_t(int dims, int prec, int mode, cudaStream_t st, int max_items, size_t smem,
                                          const WorkItem *items, const int *n_items, const RunDev *runs,
                                          const GroupDev *groups, const PoolBuf &P, void *const E[3],
                                          void *const B[3], void *const J[3], int *old_cell, void *const old_off[3],
                                          int halo, int *err)
{
    if (prec == 0) {
        auto a = make_args<double>(items, n_items, runs, groups, P, E, B, J, old_cell, old_off, halo, err);
        return dims == 3 ? launch_mode_ord<3, double, ORD>(mode, st, max_items, smem, a)
                         : launch_mode_ord<2, double, ORD>(mode, st, max_items, smem, a);
    }
    auto a = make_args<float>(items, n_items, runs, groups, P, E, B, J, old_cell, old_off, halo, err);
    return dims == 3 ? launch_mode_ord<3, float, ORD>(mode, st, max_items, smem, a)
                     : launch_mode_ord<2, float, ORD>(mode, st, max_items, smem, a);
}

template <int DIM, typename R, int ORD>
static cudaError_t set_limit_ord(int mode, size_t bytes)
{
    const int b = (int)bytes;
    switch (mode) {
    case 0: return cudaFuncSetAttribute(k_particles<DIM, R, 0, GeoDyn, ORD>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    case 1: return cudaFuncSetAttribute(k_particles<DIM, R, 1, GeoDyn, ORD>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    default: return cudaFuncSetAttribute(k_particles<DIM, R, 2, GeoDyn, ORD>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    }
}

template <int ORD>
static cudaError_t particles_ord_set_smem_limit_t(int dims, int prec, int mode, size_t bytes)
{
    if (dims == 3)
        return prec == 0 ? set_limit_ord<3, double, ORD>(mode, bytes) : set_limit_ord<3, float, ORD>(mode, bytes);
    return prec == 0 ? set_limit_ord<2, double, ORD>(mode, bytes) : set_limit_ord<2, float, ORD>(mode, bytes);
}

cudaError_t launch_particles_o5(int dims, int prec, int mode, cudaStream_t st, int max_items, size_t smem,
                                const WorkItem *items, const int *n_items, const RunDev *runs, const GroupDev *groups,
                                const PoolBuf &P, void *const E[3], void *const B[3], void *const J[3],
                                int *old_cell, void *const old_off[3], int halo, int *err, const int tile[3], int p0,
                                int p1);
cudaError_t particles_o5_set_smem_limit(int dims, int prec, int mode, size_t bytes);
cudaError_t launch_particles_w1(int dims, int prec, int mode, cudaStream_t st, int max_items, size_t smem,
                                const WorkItem *items, const int *n_items, const RunDev *runs, const GroupDev *groups,
                                const PoolBuf &P, void *const E[3], void *const B[3], void *const J[3],
                                int *old_cell, void *const old_off[3], int halo, int *err);
cudaError_t particles_w1_set_smem_limit(int dims, int prec, int mode, size_t bytes);

}  // namespace pic
