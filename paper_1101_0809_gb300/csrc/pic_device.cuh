// pic_device.cuh -- device-side data structures and per-particle arithmetic of
// the charge-conserving PIC step (Sokolov, arXiv:1101.0809), shared by the
// particle kernels.  Everything here is templated on the dimension (2 = 2D3V
// with an ignorable z, 3 = 3D3V) and on the real type R (float or double).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace pic {

// ---------------------------------------------------------------------------
// Device-side descriptors.  A batch holds one or more independent runs; each
// (run, species) pair is a "group" owning a contiguous range of the particle
// pool.  Tiles of all groups share one global numbering (group tile_base + the
// tile's linear index inside its run) that is the sort key.
// ---------------------------------------------------------------------------
// Division of a non-negative int below 2^31 by a fixed divisor d >= 1 as a
// multiply and shift (Granlund and Montgomery, "Division by invariant integers
// using multiplication", 1994, Thm. 4.2): with L = 31 + ceil(log2 d) and
// m = ceil(2^L / d) (at most 2^32), floor(n / d) = (n * m) >> L exactly, and
// n * m < 2^63.
struct DivU31 {
    unsigned long long m;
    int L;
};
inline DivU31 make_divu31(int d)
{
    int c = 0;
    while ((1LL << c) < (long long)d) ++c;
    const int L = 31 + c;
    DivU31 v;
    v.m = (unsigned long long)(((unsigned __int128)1 << L) + (unsigned)d - 1) / (unsigned)d;
    v.L = L;
    return v;
}
__device__ __forceinline__ int divu31(int n, const DivU31 &v)
{
    return (int)(((unsigned long long)(unsigned)n * v.m) >> v.L);
}

struct RunDev {
    int n[3];             // cells per axis (n[2] = 1 in 2D)
    int tile[3];          // tile extents (tile[2] = 1 in 2D)
    int ntile[3];         // tiles per axis, ceil(n/tile)
    int pitch[2];         // x and y pitch of the shared-memory field and current tiles
    long long cell_base;  // first cell of this run in the concatenated field arrays
    double cN[3];         // Courant numbers c*dt/d_a
    double dt, c;
    double d[3];
    double V;             // cell volume (dx*dy in 2D)
    double rho_bg;        // uniform background charge density
    // plane-wave antenna (include/pic.h): pol 0 none, 1 E_y/B_z, 2 E_z/B_y;
    // the total field starts at the B node x = ant_i0
    int ant_pol, ant_i0;
    double ant_E0, ant_omega, ant_ramp;
    double fpdt;            // 4 pi dt
    float fpdtf;            // 4 pi dt in FP32
    DivU31 div_nx, div_ny;  // division by n[0] and n[1]
    DivU31 div_t[3];        // division by the tile extents
    float cf, cNf[3];     // c and the Courant numbers in FP32
};

struct GroupDev {
    int run;
    int tile_base;        // global tile id of this group's tile 0
    long long base, n;    // particle range [base, base+n) in the pool
    double qm;            // q/m
    double qp;            // macro charge q_p = weight*q
    double mp;            // macro mass m_p = weight*m
    float jscale;         // fixed-point scale of the FP32 shared current tile (a power of two)
    float jinv;           // 1 / jscale
    // push and deposit prefactors of the group in its run, from the host:
    // hq = (1/2)(q/m) dt; kf[a] = -(1/4)(d_a/dt) q_p/V in 3D, and in 2D
    // kf[0,1] = -(1/2)(d_a/dt) q_p/V, kf[2] = (1/4) q_p/V (see deposit)
    double hq, kf[3];
    float hqf, kff[3], kfsf[3];   // FP32: the same, and kf * jscale
    float rscale, rinv;   // fixed-point scale of the FP32 diagnostics' shared charge tile, 1/rscale
};

struct WorkItem {
    int group;
    int tile;             // tile index inside the run
    long long begin, end; // particle range of this item
};

template <typename R>
struct Pool {
    int *cell;
    R *off[3];
    R *w[3];
    int *id;
};

template <typename R>
struct Fields {
    R *E[3];
    R *B[3];
    R *J[3];
};

enum : int { ERR_NONFINITE = 1 };

__device__ __forceinline__ int wrapi(int i, int n)
{
    return i < 0 ? i + n : (i >= n ? i - n : i);
}

// ---------------------------------------------------------------------------
// Alternating-order form factor l_a = 1 1/2 (Sec. 4.5): with d the in-cell
// offset of the particle, the lower-order point values at the integer points
// i, i+1 are f = (1-d, d), and the cell integrals at the half-integer points
// i-1/2, i+1/2, i+3/2 (centres of cells i-1, i, i+1) are
// S = ((1-d)^2/2, 3/4 - (1/2-d)^2, d^2/2).
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ void form_factor(R d, R f[2], R S[3])
{
    const R h = R(0.5);
    const R e = R(1) - d;
    const R m = h - d;
    f[0] = e;
    f[1] = d;
    S[0] = h * e * e;
    S[1] = R(0.75) - m * m;
    S[2] = h * d * d;
}

// ---------------------------------------------------------------------------
// Field readers.  Offsets (dx, dy, dz) are relative to the particle's cell.
// ---------------------------------------------------------------------------
template <typename R>
struct SmemReader {          // E/B tile with halo in shared memory
    const R *E[3];
    const R *B[3];
    int base, s1, s2;        // index of the particle cell, strides in y and z
    __device__ __forceinline__ R e(int a, int dx, int dy, int dz) const { return E[a][base + dx + s1 * dy + s2 * dz]; }
    __device__ __forceinline__ R b(int a, int dx, int dy, int dz) const { return B[a][base + dx + s1 * dy + s2 * dz]; }
};

template <typename R>
struct GlobalReader {        // periodic global arrays (particles outside their tile's halo)
    const R *E[3];
    const R *B[3];
    long long xi[4], yj[4], zk[4];   // wrapped offsets for relative -1..2 per axis
    __device__ __forceinline__ long long at(int dx, int dy, int dz) const { return xi[dx + 1] + yj[dy + 1] + zk[dz + 1]; }
    __device__ __forceinline__ R e(int a, int dx, int dy, int dz) const { return E[a][at(dx, dy, dz)]; }
    __device__ __forceinline__ R b(int a, int dx, int dy, int dz) const { return B[a][at(dx, dy, dz)]; }
};

// ---------------------------------------------------------------------------
// Gather (Sec. 2 interpolation sums with alpha of Eq. alphax and beta of
// Eq. betax).  Along its own axis an E component uses f, along the others S;
// a B component uses S along its own axis and f along the others.  2D drops
// every z factor (it sums to one).
// ---------------------------------------------------------------------------
template <int DIM, typename R, class Rd>
__device__ __forceinline__ void gather(const Rd &rd, const R fx[2], const R Sx[3], const R fy[2], const R Sy[3],
                                       const R fz[2], const R Sz[3], R Ep[3], R Bp[3])
{
    if (DIM == 3) {
        R ex = 0, ey = 0, ez = 0, bx = 0, by = 0, bz = 0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                const R wyz = Sy[b] * Sz[c];
                ex += wyz * (fx[0] * rd.e(0, 0, b - 1, c - 1) + fx[1] * rd.e(0, 1, b - 1, c - 1));
            }
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                const R wyz = fy[b] * Sz[c];
                ey += wyz * (Sx[0] * rd.e(1, -1, b, c - 1) + Sx[1] * rd.e(1, 0, b, c - 1) + Sx[2] * rd.e(1, 1, b, c - 1));
                const R wyz2 = fy[b] * (c < 2 ? fz[c] : R(0));
                if (c < 2)
                    bx += wyz2 * (Sx[0] * rd.b(0, -1, b, c) + Sx[1] * rd.b(0, 0, b, c) + Sx[2] * rd.b(0, 1, b, c));
            }
        }
#pragma unroll
        for (int c = 0; c < 2; ++c) {
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                const R wyz = Sy[b] * fz[c];
                ez += wyz * (Sx[0] * rd.e(2, -1, b - 1, c) + Sx[1] * rd.e(2, 0, b - 1, c) + Sx[2] * rd.e(2, 1, b - 1, c));
                by += wyz * (fx[0] * rd.b(1, 0, b - 1, c) + fx[1] * rd.b(1, 1, b - 1, c));
            }
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                const R wyz = fy[b] * Sz[c];
                bz += wyz * (fx[0] * rd.b(2, 0, b, c - 1) + fx[1] * rd.b(2, 1, b, c - 1));
            }
        }
        Ep[0] = ex; Ep[1] = ey; Ep[2] = ez;
        Bp[0] = bx; Bp[1] = by; Bp[2] = bz;
    } else {
        R ex = 0, ey = 0, ez = 0, bx = 0, by = 0, bz = 0;
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            ex += Sy[b] * (fx[0] * rd.e(0, 0, b - 1, 0) + fx[1] * rd.e(0, 1, b - 1, 0));
            ez += Sy[b] * (Sx[0] * rd.e(2, -1, b - 1, 0) + Sx[1] * rd.e(2, 0, b - 1, 0) + Sx[2] * rd.e(2, 1, b - 1, 0));
            by += Sy[b] * (fx[0] * rd.b(1, 0, b - 1, 0) + fx[1] * rd.b(1, 1, b - 1, 0));
        }
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            ey += fy[b] * (Sx[0] * rd.e(1, -1, b, 0) + Sx[1] * rd.e(1, 0, b, 0) + Sx[2] * rd.e(1, 1, b, 0));
            bx += fy[b] * (Sx[0] * rd.b(0, -1, b, 0) + Sx[1] * rd.b(0, 0, b, 0) + Sx[2] * rd.b(0, 1, b, 0));
            bz += fy[b] * (fx[0] * rd.b(2, 0, b, 0) + fx[1] * rd.b(2, 1, b, 0));
        }
        Ep[0] = ex; Ep[1] = ey; Ep[2] = ez;
        Bp[0] = bx; Bp[1] = by; Bp[2] = bz;
    }
}

// ---------------------------------------------------------------------------
// Relativistic push of the Appendix (Eq. 1): e = (q dt/2m) E; w~ = w + e;
// b = (q dt/2m) B / sqrt(w~^2 + c^2); w_n = w~ + w~ x b;
// w' = w~ + e + 2 (w_n x b)/(1 + b^2).   hq = q dt/(2m).
// ---------------------------------------------------------------------------
// The reciprocal of sqrt(x) and the quotient 2/(1 + b^2): correctly rounded in
// FP64; in FP32 the hardware reciprocal square root and a fast reciprocal, whose
// few-ulp errors lie far below the FP32 form's tolerance and replace the
// longer IEEE division and square-root sequences.
__device__ __forceinline__ double rsqrt_r(double x) { return 1.0 / sqrt(x); }
__device__ __forceinline__ float rsqrt_r(float x) { return rsqrtf(x); }
__device__ __forceinline__ double div_sqrt(double a, double x) { return a / sqrt(x); }
__device__ __forceinline__ float div_sqrt(float a, float x) { return a * rsqrtf(x); }
__device__ __forceinline__ double two_over(double x) { return 2.0 / x; }
__device__ __forceinline__ float two_over(float x) { return __fdividef(2.0f, x); }

template <typename R>
__device__ __forceinline__ void boris(R w[3], const R Ep[3], const R Bp[3], R hq, R c2)
{
    const R e0 = hq * Ep[0], e1 = hq * Ep[1], e2 = hq * Ep[2];
    const R t0 = w[0] + e0, t1 = w[1] + e1, t2 = w[2] + e2;
    const R s = div_sqrt(hq, t0 * t0 + t1 * t1 + t2 * t2 + c2);
    const R b0 = s * Bp[0], b1 = s * Bp[1], b2 = s * Bp[2];
    const R n0 = t0 + (t1 * b2 - t2 * b1);
    const R n1 = t1 + (t2 * b0 - t0 * b2);
    const R n2 = t2 + (t0 * b1 - t1 * b0);
    const R f = two_over(R(1) + b0 * b0 + b1 * b1 + b2 * b2);
    w[0] = t0 + e0 + f * (n1 * b2 - n2 * b1);
    w[1] = t1 + e1 + f * (n2 * b0 - n0 * b2);
    w[2] = t2 + e2 + f * (n0 * b1 - n1 * b0);
}

// ---------------------------------------------------------------------------
// Offset-to-cell renormalization after a move by delta (|delta| < 1): returns
// the cell shift k and the new offset o' in [0, 1) with cell + o' = old cell +
// o + delta.  The float version forms o + delta - k with two error-free
// TwoSum steps (Knuth) and rounds once, so o' is the float nearest to the exact
// value, as a double-precision renormalization followed by one rounding would
// give, without a single double-precision instruction.  An offset that rounds
// to 1 moves to the next cell with offset 0.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int renormalize(float o, float delta, float &out)
{
    const float s = __fadd_rn(o, delta);
    const float bv = __fsub_rn(s, o);
    const float err1 = __fadd_rn(__fsub_rn(o, __fsub_rn(s, bv)), __fsub_rn(delta, bv));
    const float k = floorf(s);
    const float t = __fsub_rn(s, k);
    const float bt = __fsub_rn(t, s);
    const float err2 = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bt)), __fsub_rn(-k, bt));
    float r = __fadd_rn(t, __fadd_rn(err1, err2));
    int ki = (int)k;
    if (r < 0.f) {
        ki -= 1;
        r = __fadd_rn(r, 1.0f);
    }
    if (r >= 1.f) {
        ki += 1;
        r = __fsub_rn(r, 1.0f);
    }
    out = r;
    return ki;
}

__device__ __forceinline__ int renormalize(double o, double delta, double &out)
{
    const double s = o + delta;
    const double k = floor(s);
    double r = s - k;
    int ki = (int)k;
    if (r >= 1.0) {
        ki += 1;
        r -= 1.0;
    }
    out = r;
    return ki;
}

// ---------------------------------------------------------------------------
// Virtual-path current (Sec. 3.2, Eq. current; Appendix step 2d).  Per axis,
// with the old cloud on cells -1..1 around the old cell and the new one on
// s-1..s+1 (s in {-1,0,1} the cell shift), the window is four cells starting at
// lo = -1 + min(s, 0).  Pp = dF(x^{n+1}) + dF(x^n) and Pm = dF(x^{n+1}) - dF(x^n)
// per window cell, and D[q] = F_f(x^{n+1}) - F_f(x^n) = sum_{w <= q} Pm[w] at the
// face f = lo + q + 1 (q = 0..2; the face after the window has D = 0).
// ---------------------------------------------------------------------------
template <typename R>
struct AxisWin {
    R Pp[4], Pm[4], D[3];
    int lo;
};

// Pm = dF(x^{n+1}) - dF(x^n) on the cells -1..1 of a particle that stayed in
// its cell along this axis (offsets d0 -> d1), in the factored form of the
// differences of the l_a = 1 1/2 weights,
//   (1-d1)^2/2 - (1-d0)^2/2 = -(1/2) dl (2 - d0 - d1),
//   (1/2-d0)^2 - (1/2-d1)^2 =  dl (1 - d0 - d1),
//   d1^2/2 - d0^2/2          =  (1/2) dl (d0 + d1),       dl = d1 - d0,
// which vanishes exactly for a particle at rest and keeps its relative accuracy
// for small displacements (the plain differences cancel).
template <typename R>
__device__ __forceinline__ void still_pm(R d0, R d1, R pm[3])
{
    const R dl = d1 - d0;
    const R sm = d0 + d1;
    pm[0] = R(-0.5) * dl * (R(2) - sm);
    pm[1] = dl * (R(1) - sm);
    pm[2] = R(0.5) * dl * sm;
}

template <typename R>
__device__ __forceinline__ void axis_window(R d0, R d1, int s, AxisWin<R> &a)
{
    R f0[2], S0[3], f1[2], S1[3];
    form_factor(d0, f0, S0);
    form_factor(d1, f1, S1);
    const bool neg = s < 0, pos = s > 0;
    const R o0 = neg ? R(0) : S0[0];
    const R o1 = neg ? S0[0] : S0[1];
    const R o2 = neg ? S0[1] : S0[2];
    const R o3 = neg ? S0[2] : R(0);
    const R n0 = pos ? R(0) : S1[0];
    const R n1 = pos ? S1[0] : S1[1];
    const R n2 = pos ? S1[1] : S1[2];
    const R n3 = pos ? S1[2] : R(0);
    a.Pp[0] = n0 + o0; a.Pm[0] = n0 - o0;
    a.Pp[1] = n1 + o1; a.Pm[1] = n1 - o1;
    a.Pp[2] = n2 + o2; a.Pm[2] = n2 - o2;
    a.Pp[3] = n3 + o3; a.Pm[3] = n3 - o3;
    if (s == 0) {   // no shift along this axis: the factored differences
        R pm[3];
        still_pm(d0, d1, pm);
        a.Pm[0] = pm[0];
        a.Pm[1] = pm[1];
        a.Pm[2] = pm[2];
    }
    a.D[0] = a.Pm[0];
    a.D[1] = a.D[0] + a.Pm[1];
    a.D[2] = a.D[1] + a.Pm[2];
    a.lo = neg ? -2 : -1;
}

// The window of a particle that stayed in its cell along this axis (s = 0):
// cells -1..1 of the old cell, interior faces 0 and 1.  The fourth cell and the
// third face carry nothing (zero weight; the closure sum of Pm), and a
// deposit called with the axis' `full` bit clear never reads them.
template <typename R>
__device__ __forceinline__ void axis_window_still(R d0, R d1, AxisWin<R> &a)
{
    // Pp = S(d1) + S(d0): Pp0 = ((1-d0)^2 + (1-d1)^2)/2, Pp2 = (d0^2 + d1^2)/2 and
    // Pp1 = 2 - Pp0 - Pp2 (the cell integrals sum to one); Pm in the factored
    // form of still_pm with h = (d1 - d0)/2 and s = d0 + d1: Pm0 = h (s - 2),
    // Pm2 = h s, Pm1 = -(Pm0 + Pm2); the face sums D0 = Pm0, D1 = -Pm2.
    const R e0 = R(1) - d0, e1 = R(1) - d1;
    a.Pp[0] = R(0.5) * (e0 * e0 + e1 * e1);
    a.Pp[2] = R(0.5) * (d0 * d0 + d1 * d1);
    a.Pp[1] = (R(2) - a.Pp[0]) - a.Pp[2];
    a.Pp[3] = R(0);
    const R h = R(0.5) * (d1 - d0), sm = d0 + d1;
    a.Pm[0] = h * (sm - R(2));
    a.Pm[2] = h * sm;
    a.Pm[1] = -(a.Pm[0] + a.Pm[2]);
    a.Pm[3] = R(0);
    a.D[0] = a.Pm[0];
    a.D[1] = -a.Pm[2];
    a.D[2] = R(0);
    a.lo = -1;
}

// Current accumulators; offsets are relative to the particle's OLD cell.
template <typename R>
struct SmemAcc {
    R *J[3];
    int base, s1, s2;
    // adds kp * t
    __device__ __forceinline__ void add(int a, int dx, int dy, int dz, R kp, R t) const
    {
        atomicAdd(&J[a][base + dx + s1 * dy + s2 * dz], kp * t);
    }
};

// FP32 form: the shared current tile accumulates in integer fixed point.
// Shared-memory float atomics run as compare-and-swap loops on this GPU while
// 32-bit integer atomics are native.  A contribution is the product kp*t, where
// the caller's prefactor kp carries a power-of-two scale: q = kp*t (|q| <= 2^33
// for every possible contribution; the host sets the scale).  It is split into
// hi = rint(q/2^16) and lo = rint(q - hi*2^16) (|lo| <= 2^15), both taken from
// the 1.5*2^23 magic-number addition, with the product formed inside the fused
// multiply-adds: magic + hi = fma(kp/2^16, t, magic), then the exact constant
// magic - hi*2^16 = fma(magic + hi, -2^16, magic*(2^16 + 1)) (at most 18
// significant bits), and magic + lo = fma(kp, t, magic - hi*2^16), rounded once
// to an integer because it lies in [2^23, 2^24).  The two integer sums are exact and stay below 2^31 for up to
// 2^13 particles per block; the block converts hi*2^16 + lo back once.
// The words added are the bit patterns of magic + hi and magic + lo, i.e.
// kFixBias + hi and kFixBias + lo.  With SUB the bias is taken off before each
// atomic; without it the block takes N * kFixBias off each word once before the
// flush, N being the number of contributions the word received (known for the
// fixed stencil of a particle that stayed in its cell; integer sums wrap
// modulo 2^32, so the order does not matter).
constexpr unsigned kFixBias = 0x4B400000u;
template <bool SUB>
struct FixedAccT {
    int *hi[3];
    int *lo[3];
    int base, s1, s2;
    __device__ __forceinline__ void add(int a, int dx, int dy, int dz, float kp, float t) const
    {
        const float magic = 12582912.0f;   // 1.5 * 2^23
        const float th = fmaf(kp * (1.0f / 65536.0f), t, magic);   // magic + hi
        const float ch = fmaf(th, -65536.0f, magic * 65537.0f);      // magic - hi * 2^16, exact
        const float tl = fmaf(kp, t, ch);                            // magic + lo, one rounding
        const int idx = base + dx + s1 * dy + s2 * dz;
        atomicAdd(&hi[a][idx], SUB ? __float_as_int(th) - (int)kFixBias : __float_as_int(th));
        atomicAdd(&lo[a][idx], SUB ? __float_as_int(tl) - (int)kFixBias : __float_as_int(tl));
    }
};
using FixedAcc = FixedAccT<true>;

// Current accumulator on the periodic global arrays for one particle's windows:
// the wrapped offsets of the window's NW cells along each axis (from lo) are
// formed once, so that a contribution costs one index sum and one atomic.
template <typename R, int NW>
struct GlobalAcc {
    R *J[3];
    long long xw[NW], yw[NW], zw[NW];
    int lox, loy, loz;
    __device__ __forceinline__ void set(long long cb, int i, int j, int k, int nx, int ny, int nz, int lx, int ly,
                                        int lz, bool three)
    {
        lox = lx;
        loy = ly;
        loz = three ? lz : 0;
#pragma unroll
        for (int m = 0; m < NW; ++m) {
            xw[m] = cb + wrapi(i + lox + m, nx);
            yw[m] = (long long)nx * wrapi(j + loy + m, ny);
            zw[m] = three ? (long long)nx * ny * wrapi(k + loz + m, nz) : 0;
        }
    }
    __device__ __forceinline__ void add(int a, int dx, int dy, int dz, R kp, R t) const
    {
        atomicAdd(&J[a][xw[dx - lox] + yw[dy - loy] + zw[dz - loz]], kp * t);
    }
};

// Deposit one particle.  kf[a] = -(1/4)(d_a/dt) q_p/V in 3D and -(1/2)(d_a/dt) q_p/V
// (a = x, y) with kf[2] = (1/4) q_p/V in 2D (reading of Eq. current summed
// over the ignorable z: xi^x = -(1/2)(dx/dt) D_x Pp_y, xi^z = (1/4) u_z [Pp Pp + Pm Pm/3]).
// Bit a of `full` is clear when no particle handled by the warp changed cell
// along axis a: then every window's fourth cell along a carries zero weight and
// its third face only the closure sum of Pm (zero up to rounding; the window
// of an unshifted particle has two interior faces), and those contributions are
// skipped.  The flag is warp-uniform, so the skip is a uniform branch.
template <int DIM, typename R, class Acc>
__device__ __forceinline__ void deposit(const Acc &acc, const AxisWin<R> &X, const AxisWin<R> &Y, const AxisWin<R> &Z,
                                        const R kf[3], R uz, int full)
{
    const R third = R(1) / R(3);
    const bool fx = full & 1, fy = full & 2, fz = full & 4;
    if (DIM == 3) {
#pragma unroll
        for (int wz = 0; wz < 4; ++wz) {
            if (wz == 3 && !fz) continue;
#pragma unroll
            for (int wy = 0; wy < 4; ++wy) {
                if (wy == 3 && !fy) continue;
                const R T = Y.Pp[wy] * Z.Pp[wz] + third * Y.Pm[wy] * Z.Pm[wz];
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    if (q == 2 && !fx) continue;
                    acc.add(0, X.lo + 1 + q, Y.lo + wy, Z.lo + wz, kf[0] * X.D[q], T);
                }
            }
        }
#pragma unroll
        for (int wz = 0; wz < 4; ++wz) {
            if (wz == 3 && !fz) continue;
#pragma unroll
            for (int wx = 0; wx < 4; ++wx) {
                if (wx == 3 && !fx) continue;
                const R T = X.Pp[wx] * Z.Pp[wz] + third * X.Pm[wx] * Z.Pm[wz];
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    if (q == 2 && !fy) continue;
                    acc.add(1, X.lo + wx, Y.lo + 1 + q, Z.lo + wz, kf[1] * Y.D[q], T);
                }
            }
        }
#pragma unroll
        for (int wy = 0; wy < 4; ++wy) {
            if (wy == 3 && !fy) continue;
#pragma unroll
            for (int wx = 0; wx < 4; ++wx) {
                if (wx == 3 && !fx) continue;
                const R T = X.Pp[wx] * Y.Pp[wy] + third * X.Pm[wx] * Y.Pm[wy];
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    if (q == 2 && !fz) continue;
                    acc.add(2, X.lo + wx, Y.lo + wy, Z.lo + 1 + q, kf[2] * Z.D[q], T);
                }
            }
        }
    } else {
#pragma unroll
        for (int wy = 0; wy < 4; ++wy) {
            if (wy == 3 && !fy) continue;
            const R t = kf[0] * Y.Pp[wy];
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                if (q == 2 && !fx) continue;
                acc.add(0, X.lo + 1 + q, Y.lo + wy, 0, t, X.D[q]);
            }
        }
#pragma unroll
        for (int wx = 0; wx < 4; ++wx) {
            if (wx == 3 && !fx) continue;
            const R t = kf[1] * X.Pp[wx];
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                if (q == 2 && !fy) continue;
                acc.add(1, X.lo + wx, Y.lo + 1 + q, 0, t, Y.D[q]);
            }
        }
        const R kz = kf[2] * uz;
#pragma unroll
        for (int wy = 0; wy < 4; ++wy) {
            if (wy == 3 && !fy) continue;
#pragma unroll
            for (int wx = 0; wx < 4; ++wx) {
                if (wx == 3 && !fx) continue;
                const R T = X.Pp[wx] * Y.Pp[wy] + third * X.Pm[wx] * Y.Pm[wy];
                acc.add(2, X.lo + wx, Y.lo + wy, 0, kz, T);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Alternating-order form factor l_a = 2 1/2 (Sec. 4.5).  The base index is
// ib = int(x_p + 1/2) with d = x_p + 1/2 - ib; the point values f = f^(2) at
// the integer points ib-1, ib, ib+1 are ((1-d)^2/2, 3/4 - (1/2-d)^2, d^2/2) and
// the cell integrals S = f^(3) over the cells ib-2 .. ib+1 (centres
// ib-3/2 .. ib+3/2) are the cubic B-spline values
//   ((1-d)^3/6, (4 - 6d^2 + 3d^3)/6, (1 + 3d + 3d^2 - 3d^3)/6, d^3/6),
// the second and third being the paper's (2-d)^3/6 - 2(1-d)^3/3 and
// (1+d)^3/6 - 2d^3/3 multiplied out.  From the stored (cell, offset o):
// ib = cell + (o >= 1/2), d = o + 1/2 - (o >= 1/2).
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ int split5(R o, R &d)
{
    const int up = o >= R(0.5) ? 1 : 0;
    d = up ? o - R(0.5) : o + R(0.5);
    return up;
}

template <typename R>
__device__ __forceinline__ void form_factor5(R d, R f[3], R S[4])
{
    const R h = R(0.5), s6 = R(1) / R(6);
    const R e = R(1) - d, m = h - d, d2 = d * d;
    f[0] = h * e * e;
    f[1] = R(0.75) - m * m;
    f[2] = h * d2;
    S[0] = s6 * e * e * e;
    S[1] = s6 * (R(4) + d2 * (R(3) * d - R(6)));
    S[2] = s6 * (R(1) + R(3) * d * (R(1) + d - d2));
    S[3] = s6 * d2 * d;
}

// Gather with l_a = 2 1/2 (Eqs. alphax, betax with f^(2) and f^(3)); reader
// offsets are relative to the base index ib: f index a sits at a - 1, S index
// b at b - 2.  2D drops every z factor.
template <int DIM, typename R, class Rd>
__device__ __forceinline__ void gather5(const Rd &rd, const R fx[3], const R Sx[4], const R fy[3], const R Sy[4],
                                        const R fz[3], const R Sz[4], R Ep[3], R Bp[3])
{
    constexpr int NZS = DIM == 3 ? 4 : 1, NZF = DIM == 3 ? 3 : 1;
    R ex = 0, ey = 0, ez = 0, bx = 0, by = 0, bz = 0;
    // The z planes are a loop, not unrolled: unrolled, the 252 taps of the
    // 3D gather need more than the 128 registers of two blocks per SM and spill.
#pragma unroll 1
    for (int c = 0; c < NZS; ++c) {   // S along z: E^x, E^y, B^z
        const R wz = DIM == 3 ? (c == 0 ? Sz[0] : c == 1 ? Sz[1] : c == 2 ? Sz[2] : Sz[3]) : R(1);
        const int oz = DIM == 3 ? c - 2 : 0;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const R t = fx[0] * rd.e(0, -1, b - 2, oz) + fx[1] * rd.e(0, 0, b - 2, oz) + fx[2] * rd.e(0, 1, b - 2, oz);
            ex += Sy[b] * wz * t;
        }
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const R t = Sx[0] * rd.e(1, -2, b - 1, oz) + Sx[1] * rd.e(1, -1, b - 1, oz) +
                        Sx[2] * rd.e(1, 0, b - 1, oz) + Sx[3] * rd.e(1, 1, b - 1, oz);
            ey += fy[b] * wz * t;
            const R u = fx[0] * rd.b(2, -1, b - 1, oz) + fx[1] * rd.b(2, 0, b - 1, oz) + fx[2] * rd.b(2, 1, b - 1, oz);
            bz += fy[b] * wz * u;
        }
    }
#pragma unroll 1
    for (int c = 0; c < NZF; ++c) {   // f along z: E^z, B^x, B^y
        const R wz = DIM == 3 ? (c == 0 ? fz[0] : c == 1 ? fz[1] : fz[2]) : R(1);
        const int oz = DIM == 3 ? c - 1 : 0;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const R t = Sx[0] * rd.e(2, -2, b - 2, oz) + Sx[1] * rd.e(2, -1, b - 2, oz) +
                        Sx[2] * rd.e(2, 0, b - 2, oz) + Sx[3] * rd.e(2, 1, b - 2, oz);
            ez += Sy[b] * wz * t;
            const R u = fx[0] * rd.b(1, -1, b - 2, oz) + fx[1] * rd.b(1, 0, b - 2, oz) + fx[2] * rd.b(1, 1, b - 2, oz);
            by += Sy[b] * wz * u;
        }
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const R t = Sx[0] * rd.b(0, -2, b - 1, oz) + Sx[1] * rd.b(0, -1, b - 1, oz) +
                        Sx[2] * rd.b(0, 0, b - 1, oz) + Sx[3] * rd.b(0, 1, b - 1, oz);
            bx += fy[b] * wz * t;
        }
    }
    Ep[0] = ex; Ep[1] = ey; Ep[2] = ez;
    Bp[0] = bx; Bp[1] = by; Bp[2] = bz;
}

// Gather of the comparison scheme of Eq. wrong1 (Sec. 5, the "conventional"
// uniform-order l = 2 interpolation): the l_a = 1 1/2 cell integrals S at the
// cells -1..1 of the particle's cell, and at the integer points -1..2 the mean
// of the two neighbouring cell integrals, g = (S0/2, (S0+S1)/2, (S1+S2)/2, S2/2).
// Reader offsets are relative to the cell.  2D drops every z factor.
template <typename R>
__device__ __forceinline__ void wrong1_points(const R S[3], R g[4])
{
    const R h = R(0.5);
    g[0] = h * S[0];
    g[1] = h * (S[0] + S[1]);
    g[2] = h * (S[1] + S[2]);
    g[3] = h * S[2];
}

template <int DIM, typename R, class Rd>
__device__ __forceinline__ void gather_w1(const Rd &rd, const R Sx[3], const R Sy[3], const R Sz[3], R Ep[3],
                                          R Bp[3])
{
    R gx[4], gy[4], gz[4];
    wrong1_points(Sx, gx);
    wrong1_points(Sy, gy);
    wrong1_points(Sz, gz);
    constexpr int NZS = DIM == 3 ? 3 : 1, NZG = DIM == 3 ? 4 : 1;
    R ex = 0, ey = 0, ez = 0, bx = 0, by = 0, bz = 0;
    // The z planes are a loop, not unrolled: unrolled, the 132 taps of the
    // 3D gather need more than the 128 registers of two blocks per SM and spill.
#pragma unroll 1
    for (int c = 0; c < NZS; ++c) {   // S along z: E^x, E^y, B^z
        const R wz = DIM == 3 ? (c == 0 ? Sz[0] : c == 1 ? Sz[1] : Sz[2]) : R(1);
        const int oz = DIM == 3 ? c - 1 : 0;
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const R t = gx[0] * rd.e(0, -1, b - 1, oz) + gx[1] * rd.e(0, 0, b - 1, oz) +
                        gx[2] * rd.e(0, 1, b - 1, oz) + gx[3] * rd.e(0, 2, b - 1, oz);
            ex += Sy[b] * wz * t;
        }
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const R t = Sx[0] * rd.e(1, -1, b - 1, oz) + Sx[1] * rd.e(1, 0, b - 1, oz) + Sx[2] * rd.e(1, 1, b - 1, oz);
            ey += gy[b] * wz * t;
            const R u = gx[0] * rd.b(2, -1, b - 1, oz) + gx[1] * rd.b(2, 0, b - 1, oz) +
                        gx[2] * rd.b(2, 1, b - 1, oz) + gx[3] * rd.b(2, 2, b - 1, oz);
            bz += gy[b] * wz * u;
        }
    }
#pragma unroll 1
    for (int c = 0; c < NZG; ++c) {   // g along z: E^z, B^x, B^y
        const R wz = DIM == 3 ? (c == 0 ? gz[0] : c == 1 ? gz[1] : c == 2 ? gz[2] : gz[3]) : R(1);
        const int oz = DIM == 3 ? c - 1 : 0;
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const R t = Sx[0] * rd.e(2, -1, b - 1, oz) + Sx[1] * rd.e(2, 0, b - 1, oz) + Sx[2] * rd.e(2, 1, b - 1, oz);
            ez += Sy[b] * wz * t;
            const R u = gx[0] * rd.b(1, -1, b - 1, oz) + gx[1] * rd.b(1, 0, b - 1, oz) +
                        gx[2] * rd.b(1, 1, b - 1, oz) + gx[3] * rd.b(1, 2, b - 1, oz);
            by += Sy[b] * wz * u;
        }
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const R t = Sx[0] * rd.b(0, -1, b - 1, oz) + Sx[1] * rd.b(0, 0, b - 1, oz) + Sx[2] * rd.b(0, 1, b - 1, oz);
            bx += gy[b] * wz * t;
        }
    }
    Ep[0] = ex; Ep[1] = ey; Ep[2] = ez;
    Bp[0] = bx; Bp[1] = by; Bp[2] = bz;
}

template <typename R>
struct GlobalReader5 {       // periodic global arrays, offsets -2..2 from the base index
    const R *E[3];
    const R *B[3];
    long long xi[5], yj[5], zk[5];
    __device__ __forceinline__ long long at(int dx, int dy, int dz) const { return xi[dx + 2] + yj[dy + 2] + zk[dz + 2]; }
    __device__ __forceinline__ R e(int a, int dx, int dy, int dz) const { return E[a][at(dx, dy, dz)]; }
    __device__ __forceinline__ R b(int a, int dx, int dy, int dz) const { return B[a][at(dx, dy, dz)]; }
};

// Deposit window of one axis with l_a = 2 1/2: the cells lo .. lo+4 relative to
// the old base index (lo = -2, or -3 when the base index moved down), the old
// and new cell integrals laid on it, Pp/Pm = new +- old, and the partial sums
// D[q] = sum_{w <= q} Pm[w] at the faces lo+q+1 (q = 0..3; the face after the
// last cell carries the closure sum only).
template <typename R>
struct AxisWin5 {
    R Pp[5], Pm[5], D[4];
    int lo;
};

template <typename R>
__device__ __forceinline__ void axis_window5(R d0, R d1, int s, AxisWin5<R> &a)
{
    R f0[3], S0[4], f1[3], S1[4];
    form_factor5(d0, f0, S0);
    form_factor5(d1, f1, S1);
    const bool neg = s < 0, pos = s > 0;
    R o[5], n[5];
#pragma unroll
    for (int w = 0; w < 5; ++w) {
        o[w] = neg ? (w == 0 ? R(0) : S0[w - 1]) : (w == 4 ? R(0) : S0[w]);
        n[w] = pos ? (w == 0 ? R(0) : S1[w - 1]) : (w == 4 ? R(0) : S1[w]);
    }
#pragma unroll
    for (int w = 0; w < 5; ++w) {
        a.Pp[w] = n[w] + o[w];
        a.Pm[w] = n[w] - o[w];
    }
    a.D[0] = a.Pm[0];
#pragma unroll
    for (int q = 1; q < 4; ++q) a.D[q] = a.D[q - 1] + a.Pm[q];
    a.lo = neg ? -3 : -2;
}

// Deposit of one particle with l_a = 2 1/2 (Eq. current on the 5-cell windows;
// the prefactors kf as for deposit()).  Bit a of `full` clear: no particle of
// the warp moved its base index along a, so the fifth window cell and the
// fourth face (the closure) are skipped.
template <int DIM, typename R, class Acc>
__device__ __forceinline__ void deposit5(const Acc &acc, const AxisWin5<R> &X, const AxisWin5<R> &Y,
                                         const AxisWin5<R> &Z, const R kf[3], R uz, int full)
{
    const R third = R(1) / R(3);
    const bool fx = full & 1, fy = full & 2, fz = full & 4;
    if (DIM == 3) {
#pragma unroll
        for (int wz = 0; wz < 5; ++wz) {
            if (wz == 4 && !fz) continue;
#pragma unroll
            for (int wy = 0; wy < 5; ++wy) {
                if (wy == 4 && !fy) continue;
                const R T = Y.Pp[wy] * Z.Pp[wz] + third * Y.Pm[wy] * Z.Pm[wz];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (q == 3 && !fx) continue;
                    acc.add(0, X.lo + 1 + q, Y.lo + wy, Z.lo + wz, kf[0] * X.D[q], T);
                }
            }
        }
#pragma unroll
        for (int wz = 0; wz < 5; ++wz) {
            if (wz == 4 && !fz) continue;
#pragma unroll
            for (int wx = 0; wx < 5; ++wx) {
                if (wx == 4 && !fx) continue;
                const R T = X.Pp[wx] * Z.Pp[wz] + third * X.Pm[wx] * Z.Pm[wz];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (q == 3 && !fy) continue;
                    acc.add(1, X.lo + wx, Y.lo + 1 + q, Z.lo + wz, kf[1] * Y.D[q], T);
                }
            }
        }
#pragma unroll
        for (int wy = 0; wy < 5; ++wy) {
            if (wy == 4 && !fy) continue;
#pragma unroll
            for (int wx = 0; wx < 5; ++wx) {
                if (wx == 4 && !fx) continue;
                const R T = X.Pp[wx] * Y.Pp[wy] + third * X.Pm[wx] * Y.Pm[wy];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (q == 3 && !fz) continue;
                    acc.add(2, X.lo + wx, Y.lo + wy, Z.lo + 1 + q, kf[2] * Z.D[q], T);
                }
            }
        }
    } else {
#pragma unroll
        for (int wy = 0; wy < 5; ++wy) {
            if (wy == 4 && !fy) continue;
            const R t = kf[0] * Y.Pp[wy];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (q == 3 && !fx) continue;
                acc.add(0, X.lo + 1 + q, Y.lo + wy, 0, t, X.D[q]);
            }
        }
#pragma unroll
        for (int wx = 0; wx < 5; ++wx) {
            if (wx == 4 && !fx) continue;
            const R t = kf[1] * X.Pp[wx];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (q == 3 && !fy) continue;
                acc.add(1, X.lo + wx, Y.lo + 1 + q, 0, t, Y.D[q]);
            }
        }
        const R kz = kf[2] * uz;
#pragma unroll
        for (int wy = 0; wy < 5; ++wy) {
            if (wy == 4 && !fy) continue;
#pragma unroll
            for (int wx = 0; wx < 5; ++wx) {
                if (wx == 4 && !fx) continue;
                const R T = X.Pp[wx] * Y.Pp[wy] + third * X.Pm[wx] * Y.Pm[wy];
                acc.add(2, X.lo + wx, Y.lo + wy, 0, kz, T);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Yee updates of one cell l of run rn (Appendix, Eqs. updateB and escheme,
// completed cyclically; in 2D every z difference vanishes).
//   B half step:  Bx[i,j,k] -= (c_y/2)(Ez[i,j,k]-Ez[i,j-1,k]) - (c_z/2)(Ey[i,j,k]-Ey[i,j,k-1])
//                 By[i,j,k] -= (c_z/2)(Ex[i,j,k]-Ex[i,j,k-1]) - (c_x/2)(Ez[i,j,k]-Ez[i-1,j,k])
//                 Bz[i,j,k] -= (c_x/2)(Ey[i,j,k]-Ey[i-1,j,k]) - (c_y/2)(Ex[i,j,k]-Ex[i,j-1,k])
//   E full step:  Ex += -4 pi dt Jx + c_y(Bz[i,j+1,k]-Bz[i,j,k]) - c_z(By[i,j,k+1]-By[i,j,k])
//                 Ey += -4 pi dt Jy + c_z(Bx[i,j,k+1]-Bx[i,j,k]) - c_x(Bz[i+1,j,k]-Bz[i,j,k])
//                 Ez += -4 pi dt Jz + c_x(By[i+1,j,k]-By[i,j,k]) - c_y(Bx[i,j+1,k]-Bx[i,j,k])
// With zero_j the B pass also clears J for the coming deposit.
// ---------------------------------------------------------------------------
// The antenna's incident field at x (cell units) and time t (include/pic.h).
__device__ __forceinline__ double antenna_field(const RunDev &rn, double x, double t)
{
    const double tau = t - (x - rn.ant_i0) * rn.d[0] / rn.c;
    if (tau <= 0.0) return 0.0;
    double g = 1.0;
    if (tau < rn.ant_ramp) {
        const double s = sin(1.5707963267948966 * tau / rn.ant_ramp);
        g = s * s;
    }
    return rn.ant_E0 * g * sin(rn.ant_omega * tau);
}

// ant_n: the antenna clock of the run (E steps since the antenna was set).
template <int DIM, typename R>
__device__ __forceinline__ void yee_b_half_cell(const RunDev &rn, const Fields<R> &F, long long l, int zero_j,
                                                long long ant_n)
{
    const int nx = rn.n[0], ny = rn.n[1], nz = rn.n[2];
    const int i = (int)(l % nx);
    const long long r = l / nx;
    const int j = (int)(r % ny);
    const int k = (int)(r / ny);
    const long long p = rn.cell_base + l;
    const long long pim = p + (i == 0 ? nx - 1 : -1);
    const long long pjm = p + (long long)nx * (j == 0 ? ny - 1 : -1);
    const bool f32 = sizeof(R) == 4;
    const R hx = f32 ? R(0.5f * rn.cNf[0]) : R(0.5 * rn.cN[0]), hy = f32 ? R(0.5f * rn.cNf[1]) : R(0.5 * rn.cN[1]);
    const R ex = F.E[0][p], ey = F.E[1][p], ez = F.E[2][p];
    R bx = F.B[0][p] - hy * (ez - F.E[2][pjm]);
    R by = F.B[1][p] + hx * (ez - F.E[2][pim]);
    R bz = F.B[2][p] - hx * (ey - F.E[1][pim]) + hy * (ex - F.E[0][pjm]);
    if (DIM == 3) {
        const long long pkm = p + (long long)nx * ny * (k == 0 ? nz - 1 : -1);
        const R hz = f32 ? R(0.5f * rn.cNf[2]) : R(0.5 * rn.cN[2]);
        bx += hz * (ey - F.E[1][pkm]);
        by -= hz * (ex - F.E[0][pkm]);
    }
    if (rn.ant_pol != 0 && i == rn.ant_i0) {
        // the scattered-field E node at x = i0 - 1/2 lacks the incident wave
        const R a = R(0.5 * rn.cN[0] * antenna_field(rn, rn.ant_i0 - 0.5, ant_n * rn.dt));
        if (rn.ant_pol == 1) bz += a; else by -= a;
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

template <int DIM, typename R>
__device__ __forceinline__ void yee_e_cell(const RunDev &rn, const Fields<R> &F, long long l, long long ant_n)
{
    const int nx = rn.n[0], ny = rn.n[1], nz = rn.n[2];
    const int i = (int)(l % nx);
    const long long r = l / nx;
    const int j = (int)(r % ny);
    const int k = (int)(r / ny);
    const long long p = rn.cell_base + l;
    const long long pip = p + (i == nx - 1 ? -(nx - 1) : 1);
    const long long pjp = p + (long long)nx * (j == ny - 1 ? -(ny - 1) : 1);
    const bool f32 = sizeof(R) == 4;
    const R cx = f32 ? R(rn.cNf[0]) : R(rn.cN[0]), cy = f32 ? R(rn.cNf[1]) : R(rn.cN[1]);
    const R fp = f32 ? R(rn.fpdtf) : R(rn.fpdt);
    const R bx = F.B[0][p], by = F.B[1][p], bz = F.B[2][p];
    R ex = F.E[0][p] - fp * F.J[0][p] + cy * (F.B[2][pjp] - bz);
    R ey = F.E[1][p] - fp * F.J[1][p] - cx * (F.B[2][pip] - bz);
    R ez = F.E[2][p] - fp * F.J[2][p] + cx * (F.B[1][pip] - by) - cy * (F.B[0][pjp] - bx);
    if (DIM == 3) {
        const long long pkp = p + (long long)nx * ny * (k == nz - 1 ? -(nz - 1) : 1);
        const R cz = f32 ? R(rn.cNf[2]) : R(rn.cN[2]);
        ex -= cz * (F.B[1][pkp] - by);
        ey += cz * (F.B[0][pkp] - bx);
    }
    if (rn.ant_pol != 0 && i == rn.ant_i0 - 1) {
        // the scattered-field E node at x = i0 - 1/2 sees the total-field B node at
        // x = i0, whose incident part (B_z = E_inc, B_y = -E_inc) comes off
        const R a = R(rn.cN[0] * antenna_field(rn, rn.ant_i0, (ant_n + 0.5) * rn.dt));
        if (rn.ant_pol == 1) ey += a; else ez += a;
    }
    F.E[0][p] = ex;
    F.E[1][p] = ey;
    F.E[2][p] = ez;
}

}  // namespace pic
