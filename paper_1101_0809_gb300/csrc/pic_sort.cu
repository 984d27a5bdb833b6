// pic_sort.cu -- stable counting sort of the particle pool by tile, and the
// work list of the particle kernels.
//
// The key of a particle is its global tile id: the tile_base of its group
// (run, species) plus the linear index of the tile holding its cell,
// (k/Tz * nty + j/Ty) * ntx + i/Tx.  The sort is a least-significant-digit
// radix sort with 8-bit digits; every pass is a stable counting sort: per
// chunk of 4096 keys a digit histogram, one exclusive scan over all
// (digit, chunk) counts in digit-major order, then a scatter in which every key
// lands at its digit's chunk offset plus its rank among equal digits earlier in
// the chunk (warp match + per-warp counts), so equal keys keep their order.
// The permutation then moves every particle array once.
#include <algorithm>

#include "pic_internal.h"

namespace pic {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kChunk = kSortThreads * kSortItems;   // keys per chunk
constexpr int kScanItems = 8;
constexpr int kScanSeg = kSortThreads * kScanItems; // elements per scan block

// ---------------------------------------------------------------------------
// Exclusive scan of unsigned counts: per-block sums, one block scanning the
// sums, then every block scanning its segment with its offset.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned block_exclusive_scan(unsigned v, unsigned *warp_tot, unsigned &total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        unsigned t = lane < nw ? warp_tot[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < nw) warp_tot[lane] = t;   // inclusive warp prefix
    }
    __syncthreads();
    const unsigned before = warp == 0 ? 0u : warp_tot[warp - 1];
    total = warp_tot[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before + x - v;
}

__device__ __forceinline__ void scan_sums(const unsigned *in, long long n, unsigned *sums)
{
    __shared__ unsigned wt[32];
    const long long base = blockIdx.x * (long long)kScanSeg + threadIdx.x * kScanItems;
    unsigned s = 0;
#pragma unroll
    for (int q = 0; q < kScanItems; ++q)
        if (base + q < n) s += in[base + q];
    unsigned total;
    block_exclusive_scan(s, wt, total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__device__ __forceinline__ void scan_single(unsigned *a, long long n)
{
    __shared__ unsigned wt[32];
    unsigned carry = 0;
    for (long long seg = 0; seg < n; seg += kScanSeg) {
        const long long base = seg + threadIdx.x * kScanItems;
        unsigned v[kScanItems];
        unsigned s = 0;
#pragma unroll
        for (int q = 0; q < kScanItems; ++q) {
            v[q] = base + q < n ? a[base + q] : 0u;
            s += v[q];
        }
        unsigned total;
        unsigned run = carry + block_exclusive_scan(s, wt, total);
#pragma unroll
        for (int q = 0; q < kScanItems; ++q) {
            if (base + q < n) a[base + q] = run;
            run += v[q];
        }
        carry += total;
    }
}

__device__ __forceinline__ void scan_apply(unsigned *a, long long n, const unsigned *sums)
{
    __shared__ unsigned wt[32];
    const long long base = blockIdx.x * (long long)kScanSeg + threadIdx.x * kScanItems;
    unsigned v[kScanItems];
    unsigned s = 0;
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) {
        v[q] = base + q < n ? a[base + q] : 0u;
        s += v[q];
    }
    unsigned total;
    unsigned run = sums[blockIdx.x] + block_exclusive_scan(s, wt, total);
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) {
        if (base + q < n) a[base + q] = run;
        run += v[q];
    }
}

__global__ void k_scan_sums(const unsigned *in, long long n, unsigned *sums) { scan_sums(in, n, sums); }
__global__ void k_scan_single(unsigned *a, long long n) { scan_single(a, n); }
__global__ void k_scan_apply(unsigned *a, long long n, const unsigned *sums) { scan_apply(a, n, sums); }

// The same over a count held on the device (*n_dev); blocks past it return.
__global__ void k_scan_sums_dev(const unsigned *in, const unsigned *n_dev, unsigned *sums)
{
    const long long n = *n_dev;
    if (blockIdx.x * (long long)kScanSeg >= n) return;
    scan_sums(in, n, sums);
}

__global__ void k_scan_single_dev(unsigned *a, const unsigned *n_dev, int per)   // ceil(*n_dev / per) entries
{
    scan_single(a, ((long long)*n_dev + per - 1) / per);
}

__global__ void k_scan_apply_dev(unsigned *a, const unsigned *n_dev, const unsigned *sums)
{
    const long long n = *n_dev;
    if (blockIdx.x * (long long)kScanSeg >= n) return;
    scan_apply(a, n, sums);
}

static cudaError_t exclusive_scan(unsigned *a, long long n, unsigned *sums, cudaStream_t st, int *launches)
{
    if (n <= 0) return cudaSuccess;
    const long long nb = (n + kScanSeg - 1) / kScanSeg;
    if (nb == 1) {
        k_scan_single<<<1, kSortThreads, 0, st>>>(a, n);
        *launches += 1;
        return cudaGetLastError();
    }
    k_scan_sums<<<(unsigned)nb, kSortThreads, 0, st>>>(a, n, sums);
    k_scan_single<<<1, kSortThreads, 0, st>>>(sums, nb);
    k_scan_apply<<<(unsigned)nb, kSortThreads, 0, st>>>(a, n, sums);
    *launches += 3;
    return cudaGetLastError();
}

// Exclusive scan of the first *n_dev of at most n_max entries.
static cudaError_t exclusive_scan_dev(unsigned *a, long long n_max, const unsigned *n_dev, unsigned *sums,
                                      cudaStream_t st, int *launches)
{
    if (n_max <= 0) return cudaSuccess;
    const long long nb = (n_max + kScanSeg - 1) / kScanSeg;
    if (nb == 1) {
        k_scan_single_dev<<<1, kSortThreads, 0, st>>>(a, n_dev, 1);
        *launches += 1;
        return cudaGetLastError();
    }
    k_scan_sums_dev<<<(unsigned)nb, kSortThreads, 0, st>>>(a, n_dev, sums);
    k_scan_single_dev<<<1, kSortThreads, 0, st>>>(sums, n_dev, kScanSeg);
    k_scan_apply_dev<<<(unsigned)nb, kSortThreads, 0, st>>>(a, n_dev, sums);
    *launches += 3;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Keys: global tile id of every particle; vals: its index.
// ---------------------------------------------------------------------------
__global__ void k_keys(long long total, const int *cell, const long long *group_base, int ngroups,
                       const GroupDev *groups, const RunDev *runs, unsigned *keys, unsigned *vals)
{
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= total) return;
    int lo = 0, hi = ngroups;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (group_base[mid] <= p) lo = mid; else hi = mid;
    }
    const RunDev &r = runs[groups[lo].run];
    const int c = cell[p];
    const int rest = divu31(c, r.div_nx);
    const int i = c - rest * r.n[0];
    const int k = divu31(rest, r.div_ny);
    const int j = rest - k * r.n[1];
    const int t = (divu31(k, r.div_t[2]) * r.ntile[1] + divu31(j, r.div_t[1])) * r.ntile[0] + divu31(i, r.div_t[0]);
    keys[p] = (unsigned)(groups[lo].tile_base + t);
    vals[p] = (unsigned)p;
}

__device__ __forceinline__ void upsweep(const unsigned *keys, long long n, int shift, unsigned *hist, long long nchunks)
{
    __shared__ unsigned h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const long long base = blockIdx.x * (long long)kChunk;
#pragma unroll 4
    for (int r = 0; r < kSortItems; ++r) {
        const long long idx = base + r * kSortThreads + threadIdx.x;
        if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[threadIdx.x * nchunks + blockIdx.x] = h[threadIdx.x];
}

__global__ void k_upsweep(const unsigned *keys, long long n, int shift, unsigned *hist, long long nchunks)
{
    upsweep(keys, n, shift, hist, nchunks);
}

// The same over a key count held on the device, at most cap (the keys buffers'
// length): only its chunks take part, and the histogram is laid out for them
// (hist_n = 256 x their number, written by k_hist_count).
__global__ void k_hist_count(const unsigned *n_dev, long long cap, unsigned *hist_n)
{
    const long long n = min((long long)*n_dev, cap);
    *hist_n = (unsigned)(256 * ((n + kChunk - 1) / kChunk));
}

__global__ void k_upsweep_dev(const unsigned *keys, const unsigned *n_dev, long long cap, int shift, unsigned *hist,
                              const unsigned *hist_n)
{
    const long long nch = *hist_n / 256;
    if (blockIdx.x >= nch) return;
    upsweep(keys, min((long long)*n_dev, cap), shift, hist, nch);
}

__device__ __forceinline__ void downsweep(const unsigned *keys, const unsigned *vals, long long n, int shift,
                                          const unsigned *hist, long long nchunks, unsigned *keys_out,
                                          unsigned *vals_out)
{
    __shared__ unsigned off[256];
    __shared__ unsigned tot[256];
    __shared__ unsigned wh[kSortThreads / 32][256];
    __shared__ unsigned pre[kSortThreads / 32][256];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    off[tid] = hist[tid * nchunks + blockIdx.x];
    tot[tid] = 0;
#pragma unroll
    for (int w = 0; w < kSortThreads / 32; ++w) wh[w][tid] = 0;
    __syncthreads();
    const long long base = blockIdx.x * (long long)kChunk;
    const unsigned lt = (1u << lane) - 1u;
    for (int r = 0; r < kSortItems; ++r) {
        const long long idx = base + r * kSortThreads + tid;
        const bool valid = idx < n;
        const unsigned key = valid ? keys[idx] : 0u;
        const unsigned val = valid ? vals[idx] : 0u;
        const unsigned d = valid ? ((key >> shift) & 255u) : 256u;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const unsigned rank = __popc(peers & lt);
        if (valid && (__ffs(peers) - 1) == lane) wh[warp][d] = __popc(peers);
        __syncthreads();
        {
            unsigned run = tot[tid];
#pragma unroll
            for (int w = 0; w < kSortThreads / 32; ++w) {
                const unsigned c = wh[w][tid];
                pre[w][tid] = run;
                run += c;
                wh[w][tid] = 0;
            }
            tot[tid] = run;
        }
        __syncthreads();
        if (valid) {
            const unsigned dst = off[d] + pre[warp][d] + rank;
            keys_out[dst] = key;
            vals_out[dst] = val;
        }
    }
}

__global__ void __launch_bounds__(kSortThreads) k_downsweep(const unsigned *keys, const unsigned *vals, long long n,
                                                            int shift, const unsigned *hist, long long nchunks,
                                                            unsigned *keys_out, unsigned *vals_out)
{
    downsweep(keys, vals, n, shift, hist, nchunks, keys_out, vals_out);
}

__global__ void __launch_bounds__(kSortThreads) k_downsweep_dev(const unsigned *keys, const unsigned *vals,
                                                                const unsigned *n_dev, long long cap, int shift,
                                                                const unsigned *hist, const unsigned *hist_n,
                                                                unsigned *keys_out, unsigned *vals_out)
{
    const long long nch = *hist_n / 256;
    if (blockIdx.x >= nch) return;
    downsweep(keys, vals, min((long long)*n_dev, cap), shift, hist, nch, keys_out, vals_out);
}

// Bank interleave inside every tile.  The particle kernels stage the tile's
// current in shared memory with x pitch P0 and y pitch P1 (rn.pitch);
// a particle's accesses are its cell's base address plus offsets common to all
// particles, so the 32 lanes of a warp hit 32 distinct banks when their cells'
// base addresses are distinct modulo 32.  Within each tile this kernel keeps the
// stable tile order per bank b = base(cell) mod 32 and interleaves the banks:
// the r-th particle (r = its rank among the tile's particles of bank b) goes to
// slot S(r) + #{b' < b : cnt[b'] > r}, with S(r) = sum_b' min(cnt[b'], r).  The
// key order (by tile) is unchanged; only the order inside a tile changes.
// With half != 0 (l_a = 2 1/2) the accesses are relative to the base index
// cell + (offset >= 1/2) per axis, so that index takes the cell's place; the
// offsets are FP64 (prec 0) or FP32.
__global__ void __launch_bounds__(kSortThreads) k_bank_order(const long long *tile_start, const unsigned *vals_in,
                                                             unsigned *vals_out, const int *cell, const GroupDev *groups,
                                                             int ngroups, const RunDev *runs, int halo, int dims,
                                                             int half, int prec, const void *off0, const void *off1,
                                                             const void *off2)
{
    constexpr int kRankTab = 1024;   // ranks with a precomputed slot table
    __shared__ unsigned cnt[32];
    __shared__ unsigned tot[32];
    __shared__ unsigned wh[kSortThreads / 32][32];
    __shared__ unsigned pre[kSortThreads / 32][32];
    __shared__ unsigned gmask[kRankTab];   // banks b with cnt[b] > r
    __shared__ unsigned gS[kRankTab];      // S(r)
    __shared__ unsigned ntab;
    const int t = blockIdx.x;
    const long long b0 = tile_start[t], e0 = tile_start[t + 1];
    if (e0 - b0 <= 1) {
        if (threadIdx.x == 0 && e0 > b0) vals_out[b0] = vals_in[b0];
        return;
    }
    int lo = 0, hi = ngroups;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (groups[mid].tile_base <= t) lo = mid; else hi = mid;
    }
    const RunDev &rn = runs[groups[lo].run];
    const int lt = t - groups[lo].tile_base;
    const int tx = lt % rn.ntile[0], ty = (lt / rn.ntile[0]) % rn.ntile[1], tz = lt / (rn.ntile[0] * rn.ntile[1]);
    const int ox = tx * rn.tile[0], oy = ty * rn.tile[1], oz = tz * rn.tile[2];
    const int P0 = rn.pitch[0], P1 = rn.pitch[1];
    const int nx = rn.n[0], ny = rn.n[1];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    auto bank_of = [&](unsigned v) -> unsigned {
        const int c = cell[v];
        const int r = divu31(c, rn.div_nx);
        const int i = c - r * nx;
        const int k = dims == 3 ? divu31(r, rn.div_ny) : 0;
        const int j = r - k * ny;
        int u0 = 0, u1 = 0, u2 = 0;
        if (half) {
            auto up = [&](const void *o) -> int {
                return prec == 0 ? (static_cast<const double *>(o)[v] >= 0.5 ? 1 : 0)
                                 : (static_cast<const float *>(o)[v] >= 0.5f ? 1 : 0);
            };
            u0 = up(off0);
            u1 = up(off1);
            if (dims == 3) u2 = up(off2);
        }
        const int base = (i + u0 - ox + halo + 2) +
                         P0 * ((j + u1 - oy + halo + 2) + (dims == 3 ? P1 * (k + u2 - oz + halo + 2) : 0));
        return (unsigned)base & 31u;
    };
    if (tid < 32) {
        cnt[tid] = 0;
        tot[tid] = 0;
    }
    if (tid < kSortThreads / 32 * 32) wh[tid >> 5][tid & 31] = 0;
    __syncthreads();
    for (long long o = b0 + tid; o < e0; o += kSortThreads) atomicAdd(&cnt[bank_of(vals_in[o])], 1u);
    __syncthreads();
    // slot tables for ranks below min(max cnt, kRankTab): the mask of banks that
    // still have a particle of rank r, and S(r) = sum_b min(cnt[b], r), the
    // number of slots taken by lower ranks
    if (warp == 0) {
        unsigned m = cnt[lane];
        for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) ntab = m < (unsigned)kRankTab ? m : (unsigned)kRankTab;
    }
    __syncthreads();
    const unsigned nt = ntab;
    for (unsigned r = tid; r < nt; r += kSortThreads) {
        unsigned m = 0;
        for (int b = 0; b < 32; ++b) m |= (cnt[b] > r ? 1u : 0u) << b;
        gmask[r] = m;
    }
    __syncthreads();
    if (warp == 0) {
        unsigned run = 0;
        for (unsigned r0 = 0; r0 < nt; r0 += 32) {
            const unsigned r = r0 + lane;
            const unsigned g = r < nt ? __popc(gmask[r]) : 0u;
            unsigned inc = g;
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned y = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += y;
            }
            if (r < nt) gS[r] = run + inc - g;
            run += __shfl_sync(0xffffffffu, inc, 31);
        }
    }
    __syncthreads();
    const unsigned ltm = (1u << lane) - 1u;
    for (long long r0 = b0; r0 < e0; r0 += kSortThreads) {
        const long long o = r0 + tid;
        const bool valid = o < e0;
        const unsigned v = valid ? vals_in[o] : 0u;
        const unsigned bk = valid ? bank_of(v) : 32u;
        const unsigned peers = __match_any_sync(0xffffffffu, bk);
        const unsigned rk = __popc(peers & ltm);
        if (valid && (__ffs(peers) - 1) == lane) wh[warp][bk] = __popc(peers);
        __syncthreads();
        if (tid < 32) {
            unsigned run = tot[tid];
            for (int w = 0; w < kSortThreads / 32; ++w) {
                const unsigned c = wh[w][tid];
                pre[w][tid] = run;
                run += c;
                wh[w][tid] = 0;
            }
            tot[tid] = run;
        }
        __syncthreads();
        if (valid) {
            const unsigned rank = pre[warp][bk] + rk;   // rank among the tile's particles of bank bk
            unsigned S = 0, below = 0;
            if (rank < nt) {
                S = gS[rank];
                below = __popc(gmask[rank] & ((1u << bk) - 1u));
            } else {
                for (int b = 0; b < 32; ++b) {
                    const unsigned cb = cnt[b];
                    S += cb < rank ? cb : rank;
                    if (b < (int)bk && cb > rank) ++below;
                }
            }
            vals_out[b0 + S + below] = v;
        }
    }
}

// ---------------------------------------------------------------------------
// Cell-lane order inside a tile (PIC_SORT_CELL_LANES; tiles of at most 128
// cells).  The tile's cells are ranked by descending particle count, ties by
// their index c = lx + Tx (ly + Ty lz) in the tile: cell c gets lane L(c).  The
// particle of rank r among its cell's particles (input order) goes to slot
// P(r) + L(c) of the tile, P(r) = sum over the tile's cells of min(count, r):
// the slots of rank r follow those of all lower ranks, and within a rank the
// cells that still have particles come in lane order.  Per tile the kernel also
// writes, for every lane, its cell (lane_cell) and count (lane_count).
// ---------------------------------------------------------------------------
constexpr int kLaneCells = 128;
__global__ void __launch_bounds__(kSortThreads) k_cell_lane_order(const long long *tile_start, const unsigned *vals_in,
                                                                  unsigned *vals_out, const int *cell,
                                                                  const GroupDev *groups, int ngroups,
                                                                  const RunDev *runs, unsigned char *lane_cell,
                                                                  int *lane_count)
{
    constexpr int kRankTab = 1024;   // ranks with a precomputed P(r)
    constexpr int kW = kSortThreads / 32;
    __shared__ unsigned cnt[kLaneCells];
    __shared__ unsigned lane_of[kLaneCells];
    __shared__ unsigned scnt[kLaneCells];   // counts by lane (descending)
    __shared__ unsigned run[kLaneCells];    // particles of each cell in earlier chunks
    __shared__ unsigned wh[kW][kLaneCells];
    __shared__ unsigned pre[kW][kLaneCells];
    __shared__ unsigned ptab[kRankTab];
    const int t = blockIdx.x;
    const long long b0 = tile_start[t], e0 = tile_start[t + 1];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int lo = 0, hi = ngroups;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (groups[mid].tile_base <= t) lo = mid; else hi = mid;
    }
    const RunDev &rn = runs[groups[lo].run];
    const int lt = t - groups[lo].tile_base;
    const int T0 = rn.tile[0], T1 = rn.tile[1];
    const int ox = (lt % rn.ntile[0]) * T0, oy = ((lt / rn.ntile[0]) % rn.ntile[1]) * T1;
    const int oz = (lt / (rn.ntile[0] * rn.ntile[1])) * rn.tile[2];
    const int nx = rn.n[0], ny = rn.n[1];
    auto local_cell = [&](unsigned v) -> unsigned {
        const int c = cell[v];
        const int r = divu31(c, rn.div_nx);
        const int i = c - r * nx;
        const int k = divu31(r, rn.div_ny);
        const int j = r - k * ny;
        return (unsigned)((i - ox) + T0 * ((j - oy) + T1 * (k - oz)));
    };
    for (int c = tid; c < kLaneCells; c += kSortThreads) {
        cnt[c] = 0;
        run[c] = 0;
    }
    for (int q = tid; q < kW * kLaneCells; q += kSortThreads) (&wh[0][0])[q] = 0;
    __syncthreads();
    for (long long o = b0 + tid; o < e0; o += kSortThreads) atomicAdd(&cnt[local_cell(vals_in[o])], 1u);
    __syncthreads();
    for (int c = tid; c < kLaneCells; c += kSortThreads) {
        const unsigned mc = cnt[c];
        unsigned r = 0;
        for (int d = 0; d < kLaneCells; ++d) {
            const unsigned md = cnt[d];
            r += (md > mc || (md == mc && d < c)) ? 1u : 0u;
        }
        lane_of[c] = r;
        scnt[r] = mc;
        lane_cell[(long long)t * kLaneCells + r] = (unsigned char)c;
        lane_count[(long long)t * kLaneCells + r] = (int)mc;
    }
    __syncthreads();
    const unsigned maxc = scnt[0];
    const unsigned nt = maxc < (unsigned)kRankTab ? maxc : (unsigned)kRankTab;
    for (unsigned r = tid; r < nt; r += kSortThreads) {
        unsigned s = 0;
        for (int l = 0; l < kLaneCells; ++l) s += min(scnt[l], r);
        ptab[r] = s;
    }
    __syncthreads();
    const unsigned ltm = (1u << lane) - 1u;
    for (long long r0 = b0; r0 < e0; r0 += kSortThreads) {
        const long long o = r0 + tid;
        const bool valid = o < e0;
        const unsigned v = valid ? vals_in[o] : 0u;
        const unsigned lc = valid ? local_cell(v) : (unsigned)kLaneCells;
        const unsigned peers = __match_any_sync(0xffffffffu, lc);
        const unsigned rk = __popc(peers & ltm);
        if (valid && (__ffs(peers) - 1) == lane) wh[warp][lc] = __popc(peers);
        __syncthreads();
        for (int c = tid; c < kLaneCells; c += kSortThreads) {
            unsigned acc = run[c];
            for (int w = 0; w < kW; ++w) {
                const unsigned x = wh[w][c];
                pre[w][c] = acc;
                acc += x;
                wh[w][c] = 0;
            }
            run[c] = acc;
        }
        __syncthreads();
        if (valid) {
            const unsigned rank = pre[warp][lc] + rk;   // rank among the cell's particles
            unsigned P = 0;
            if (rank < nt) {
                P = ptab[rank];
            } else {
                for (int l = 0; l < kLaneCells; ++l) P += min(scnt[l], rank);
            }
            vals_out[b0 + P + lane_of[lc]] = v;
        }
    }
}

// ---------------------------------------------------------------------------
// Re-sort from the previous sort's tile segments.  Between sorts the particle
// kernels update the particles in place, so the pool still consists of the
// segments of the last sort: segment t = [tile_start[t], tile_start[t+1]) holds
// the particles that were in tile t then.  The segments are contiguous and in
// increasing order, so a particle's segment order is its input order, and the
// particles with new key t in input order are: the movers into t (particles
// whose tile changed) from segments before t, the particles of segment t that
// are still in tile t, and the movers into t from segments after t.  A first
// pass classifies every particle (mover, or its bank in its tile); only the
// movers need a global sort: they are listed in input order with their new keys
// (k_resort_movers) and sorted stably by key with the radix passes over a count
// held on the device.  One block per new tile then merges them with the
// stayers and takes the order inside the tile (banked or stable) as
// k_bank_order does, and the arrays move in one gather (k_permute4).  The
// permutation is the full sort's, bit for bit.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int group_of_tile(int t, const GroupDev *groups, int ngroups)
{
    int lo = 0, hi = ngroups;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (groups[mid].tile_base <= t) lo = mid; else hi = mid;
    }
    return lo;
}

// A tile of one run: its origin and extents, and the run's cell decomposition.
struct TileBox {
    const RunDev *rn;
    int ox, oy, oz;
    __device__ TileBox(const RunDev &r, int lt) : rn(&r)
    {
        ox = (lt % r.ntile[0]) * r.tile[0];
        oy = ((lt / r.ntile[0]) % r.ntile[1]) * r.tile[1];
        oz = (lt / (r.ntile[0] * r.ntile[1])) * r.tile[2];
    }
    __device__ __forceinline__ void ijk(int c, int &i, int &j, int &k) const
    {
        const int rest = divu31(c, rn->div_nx);
        i = c - rest * rn->n[0];
        k = divu31(rest, rn->div_ny);
        j = rest - k * rn->n[1];
    }
    __device__ __forceinline__ bool holds(int i, int j, int k) const
    {
        return (unsigned)(i - ox) < (unsigned)rn->tile[0] && (unsigned)(j - oy) < (unsigned)rn->tile[1] &&
               (unsigned)(k - oz) < (unsigned)rn->tile[2];
    }
    __device__ __forceinline__ int tile_of(int i, int j, int k) const
    {
        return (divu31(k, rn->div_t[2]) * rn->ntile[1] + divu31(j, rn->div_t[1])) * rn->ntile[0] +
               divu31(i, rn->div_t[0]);
    }
};

// Segments are clamped to [0, total): a snapshot's segments are trusted like
// its work items, and the clamps and the guarded writes below keep every
// access inside the buffers whatever they hold.
__device__ __forceinline__ long long seg_at(const long long *ts, int t, long long total)
{
    const long long v = ts[t];
    return v < 0 ? 0 : (v > total ? total : v);
}

// Class of a particle in its old segment: kMover if its tile changed, else its
// shared-memory bank in the tile (banked order, as in k_bank_order) or 0.
constexpr unsigned kMover = 32;

struct BankRule {
    int banked, half, halo, dims, P0, P1, prec;
    const void *off[3];
    // the bank of particle v with cell (i, j, k) in the tile at (ox, oy, oz)
    __device__ __forceinline__ unsigned bank(const TileBox &box, unsigned v, int i, int j, int k) const
    {
        if (!banked) return 0u;
        int u0 = 0, u1 = 0, u2 = 0;
        if (half) {
            auto up = [&](const void *o) -> int {
                return prec == 0 ? (static_cast<const double *>(o)[v] >= 0.5 ? 1 : 0)
                                 : (static_cast<const float *>(o)[v] >= 0.5f ? 1 : 0);
            };
            u0 = up(off[0]);
            u1 = up(off[1]);
            if (dims == 3) u2 = up(off[2]);
        }
        const int base = (i + u0 - box.ox + halo + 2) +
                         P0 * ((j + u1 - box.oy + halo + 2) + (dims == 3 ? P1 * (k + u2 - box.oz + halo + 2) : 0));
        return (unsigned)base & 31u;
    }
};

// Per old segment t: the class of every particle (cls), the number of movers
// (mcnt, and their total) and of stayers; block total_tiles writes the zero
// counts after the last tile (for the exclusive scans).  Every thread loads
// kResortU cells before it classifies them, so that enough loads are in flight.
constexpr int kResortU = 16;
__global__ void __launch_bounds__(kSortThreads) k_resort_classify(const long long *ots, long long total,
                                                                  int total_tiles, const int *cell,
                                                                  const GroupDev *groups, int ngroups,
                                                                  const RunDev *runs, BankRule rule,
                                                                  unsigned char *cls, unsigned *mcnt, unsigned *stay,
                                                                  unsigned *m_total)
{
    __shared__ unsigned ws[kSortThreads / 32];
    const int t = blockIdx.x;
    if (t == total_tiles) {
        if (threadIdx.x == 0) {
            mcnt[t] = 0;
            stay[t] = 0;
        }
        return;
    }
    const long long sb = seg_at(ots, t, total), se = max(sb, seg_at(ots, t + 1, total));
    const int gi = group_of_tile(t, groups, ngroups);
    const RunDev &rn = runs[groups[gi].run];
    const TileBox box(rn, t - groups[gi].tile_base);
    BankRule r = rule;
    r.P0 = rn.pitch[0];
    r.P1 = rn.pitch[1];
    unsigned m = 0;
    for (long long c0 = sb; c0 < se; c0 += kSortThreads * kResortU) {
        int cv[kResortU];
#pragma unroll
        for (int u = 0; u < kResortU; ++u) {
            const long long p = c0 + u * kSortThreads + threadIdx.x;
            cv[u] = p < se ? cell[p] : -1;
        }
#pragma unroll
        for (int u = 0; u < kResortU; ++u)
            if (cv[u] >= 0) {
                const long long p = c0 + u * kSortThreads + threadIdx.x;
                int i, j, k;
                box.ijk(cv[u], i, j, k);
                unsigned c = kMover;
                if (box.holds(i, j, k)) c = r.bank(box, (unsigned)p, i, j, k);
                else ++m;
                cls[p] = (unsigned char)c;
            }
    }
    for (int o = 16; o > 0; o >>= 1) m += __shfl_xor_sync(0xffffffffu, m, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned s = 0;
        for (int w = 0; w < kSortThreads / 32; ++w) s += ws[w];
        mcnt[t] = s;
        stay[t] = (unsigned)(se - sb) - s;
        if (s) atomicAdd(m_total, s);
    }
}

// Per old segment t: its movers in input order at moff[t] (exclusive scan of the
// counts), with their new keys.  A batch is kResortU chunks of kSortThreads
// particles; the movers of (chunk, warp) follow those of the earlier pairs, in
// one scan over the batch's counts.
__global__ void __launch_bounds__(kSortThreads) k_resort_movers(const long long *ots, long long total,
                                                                const unsigned *moff, const unsigned char *cls,
                                                                const int *cell, const GroupDev *groups, int ngroups,
                                                                const RunDev *runs, int total_tiles, unsigned *mkeys,
                                                                unsigned *mvals)
{
    constexpr int W = kSortThreads / 32;
    constexpr int NC = kResortU * W;   // (chunk, warp) pairs of a batch
    static_assert(NC % 32 == 0, "pairs per lane");
    __shared__ unsigned wt[NC];        // movers per pair, then their exclusive prefix
    __shared__ unsigned wtot;
    const int t = blockIdx.x;
    if (moff[t + 1] == moff[t]) return;   // no movers
    const long long sb = seg_at(ots, t, total), se = max(sb, seg_at(ots, t + 1, total));
    const int gi = group_of_tile(t, groups, ngroups);
    const int tb = groups[gi].tile_base;
    const TileBox box(runs[groups[gi].run], t - tb);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned ltm = (1u << lane) - 1u;
    unsigned run = moff[t];
    for (long long c0 = sb; c0 < se; c0 += kSortThreads * kResortU) {
        unsigned char c8[kResortU];
#pragma unroll
        for (int u = 0; u < kResortU; ++u) {
            const long long p = c0 + u * kSortThreads + threadIdx.x;
            c8[u] = p < se ? cls[p] : 0;
        }
        int cv[kResortU];   // the movers' cells, all requested before any is used
#pragma unroll
        for (int u = 0; u < kResortU; ++u) {
            const long long p = c0 + u * kSortThreads + threadIdx.x;
            cv[u] = c8[u] == kMover ? cell[p] : -1;
        }
        unsigned bal[kResortU];
#pragma unroll
        for (int u = 0; u < kResortU; ++u) {
            bal[u] = __ballot_sync(0xffffffffu, cv[u] >= 0);
            if (lane == 0) wt[u * W + warp] = __popc(bal[u]);
        }
        __syncthreads();
        if (warp == 0) {   // exclusive scan of the NC counts, NC / 32 consecutive ones per lane
            constexpr int PL = NC / 32;
            unsigned x[PL], s = 0;
#pragma unroll
            for (int q = 0; q < PL; ++q) {
                x[q] = wt[lane * PL + q];
                s += x[q];
            }
            unsigned inc = s;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned y = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += y;
            }
            unsigned acc = inc - s;
#pragma unroll
            for (int q = 0; q < PL; ++q) {
                wt[lane * PL + q] = acc;
                acc += x[q];
            }
            if (lane == 31) wtot = inc;
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < kResortU; ++u)
            if (cv[u] >= 0) {
                int i, j, k;
                box.ijk(cv[u], i, j, k);
                const unsigned kk = (unsigned)(tb + box.tile_of(i, j, k));
                const unsigned dst = run + wt[u * W + warp] + __popc(bal[u] & ltm);
                if (dst < total && kk < (unsigned)total_tiles) {
                    mkeys[dst] = kk;
                    mvals[dst] = (unsigned)(c0 + u * kSortThreads + threadIdx.x);
                }
            }
        run += wtot;
        __syncthreads();   // wt is rewritten by the next batch
    }
}

// Over the movers sorted by key (keys sk, indices sv, *n_dev of them): mstart[t]
// = the first with key >= t, for t in [0, total_tiles], and aft[t] = the first
// of key t whose index is at or past segment t's start (movers from later
// segments); aft stays 0xffffffff for a tile without such movers.
__global__ void k_resort_bounds(const unsigned *sk, const unsigned *sv, const unsigned *n_dev, long long cap,
                                int total_tiles, const long long *ots, unsigned *mstart, unsigned *aft)
{
    const long long n = min((long long)*n_dev, cap);
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o <= n; o += stride) {
        if (o == n) {   // the tiles after the last mover's key (all of them without movers)
            for (long long t = n ? (long long)sk[n - 1] + 1 : 0; t <= total_tiles; ++t) mstart[t] = (unsigned)n;
            continue;
        }
        const long long k = sk[o];
        const long long kp = o == 0 ? -1 : (long long)sk[o - 1];
        for (long long t = kp + 1; t <= k; ++t) mstart[t] = (unsigned)o;
        const bool late = (long long)sv[o] >= ots[k];
        const bool late_prev = o > 0 && kp == k && (long long)sv[o - 1] >= ots[k];
        if (late && !late_prev) aft[k] = (unsigned)o;
    }
}

// New counts (over total_tiles + 1 entries): stayers plus movers in; mbef[t] =
// the movers into t from earlier segments.
__global__ void k_resort_newcnt(int n, unsigned *stay, const unsigned *mstart, const unsigned *aft, unsigned *mbef)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const unsigned movin = t + 1 < n ? mstart[t + 1] - mstart[t] : 0u;
    stay[t] += movin;
    mbef[t] = aft[t] == 0xffffffffu ? movin : aft[t] - mstart[t];
}

__global__ void k_resort_tile_start(int n, const unsigned *nst, long long *tile_start)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) tile_start[t] = nst[t];
}

constexpr int kMoverCache = 1024;   // movers of a tile whose index and bank k_resort_order keeps in shared memory
constexpr int kClassCache = 8192;   // class bytes of a segment that k_resort_order keeps in shared memory

// One block per new tile t: the particles of t in input order are walked twice
// by the block's warps, each warp over a contiguous share of the sequence
// [movers from earlier segments | segment t | movers from later segments]:
// first counting per bank (shared atomics), then ranking (the lanes of the
// same bank found by five ballots), which gives every particle its slot in the
// tile's new range (banked or stable order): perm[new_start + slot] = index.
// The stayers' banks come from their class bytes; the movers' indices and
// banks are read once into shared memory.
__global__ void __launch_bounds__(kSortThreads) k_resort_order(const long long *ots, long long total,
                                                               const unsigned *nst, const unsigned *mstart,
                                                               const unsigned *mbef, const unsigned *mvals,
                                                               const unsigned char *cls, const int *cell,
                                                               const GroupDev *groups, int ngroups,
                                                               const RunDev *runs, BankRule rule, unsigned *perm)
{
    constexpr int kRankTab = 1024;   // ranks with a precomputed slot table
    constexpr int W = kSortThreads / 32;
    __shared__ unsigned cw[W][32];   // per warp and bank: count (first walk), then running rank
    __shared__ unsigned pre[W][32];  // per warp and bank: particles of the bank in earlier warps' shares
    __shared__ unsigned cnt[32];
    __shared__ unsigned gmask[kRankTab];   // banks b with cnt[b] > r
    __shared__ unsigned gS[kRankTab];      // S(r) = sum_b min(cnt[b], r)
    __shared__ unsigned ntab;
    __shared__ unsigned mv_v[kMoverCache];   // the first movers into the tile: pool index and bank
    __shared__ unsigned char mv_b[kMoverCache];
    __shared__ unsigned cls_w[kClassCache / 4 + 2];   // the segment's class bytes, from the 4-byte word of sb
    const int t = blockIdx.x;
    const unsigned nb = nst[t], ne = nst[t + 1];
    if (ne <= nb || (long long)ne > total) return;
    const unsigned nT = ne - nb;
    const long long sb = seg_at(ots, t, total), se = max(sb, seg_at(ots, t + 1, total));
    const unsigned seglen = (unsigned)(se - sb);
    const unsigned mb = min(mstart[t], (unsigned)total), me = max(mb, min(mstart[t + 1], (unsigned)total));
    const unsigned nbef = min(mbef[t], me - mb);
    const int gi = group_of_tile(t, groups, ngroups);
    const RunDev &rn = runs[groups[gi].run];
    const TileBox box(rn, t - groups[gi].tile_base);
    BankRule r = rule;
    r.P0 = rn.pitch[0];
    r.P1 = rn.pitch[1];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned ltm = (1u << lane) - 1u;
    auto mover_bank = [&](unsigned v) -> unsigned {
        int i, j, k;
        box.ijk(cell[v], i, j, k);
        return r.bank(box, v, i, j, k);
    };
    cw[warp][lane] = 0;
    const unsigned nmov = me - mb, ncached = min(nmov, (unsigned)kMoverCache);
    // the segment's class bytes as whole words (the pool is allocated in 4-element groups)
    const long long w0 = sb >> 2;
    const unsigned nw = (unsigned)(((se + 3) >> 2) - w0), nwc = min(nw, (unsigned)(kClassCache / 4 + 2));
    const unsigned *clsw = reinterpret_cast<const unsigned *>(cls);
    for (unsigned q = tid; q < nwc; q += kSortThreads) cls_w[q] = clsw[w0 + q];
    for (unsigned q = tid; q < ncached; q += kSortThreads) {
        const unsigned v = mvals[mb + q];
        mv_v[q] = v;
        mv_b[q] = (long long)v < total ? (unsigned char)mover_bank(v) : (unsigned char)kMover;
    }
    __syncthreads();
    const unsigned char *cls_s = reinterpret_cast<const unsigned char *>(cls_w);
    const unsigned cls_off = (unsigned)(sb - (w0 << 2)), cls_n = nwc * 4;   // byte of sb, bytes cached
    const unsigned nseq = nmov + seglen;
    const unsigned share = ((nseq + W - 1) / W + 31) & ~31u;
    const unsigned k0 = min(nseq, warp * share), k1 = min(nseq, k0 + share);
    // the k-th particle of the sequence: its index v and class (kMover: not in the tile)
    // a mover of the tile: its index v and bank
    auto fetch_mover = [&](unsigned jm, unsigned &v) -> unsigned {
        if (jm < ncached) {
            v = mv_v[jm];
            return mv_b[jm];
        }
        v = mvals[mb + jm];
        return (long long)v < total ? mover_bank(v) : kMover;
    };
    // the warp's share of the sequence, in order, 32 positions per round; each
    // of the three ranges has its own loop, so that a round never mixes them.
    // body(b, v): b the particle's bank (kMover: no particle of tile t), v its index
    auto walk = [&](auto &&body) {
        const unsigned a1 = min(k1, nbef), a2 = min(k1, nbef + seglen);
        for (unsigned q0 = k0; q0 < a1; q0 += 32) {   // movers from earlier segments
            const unsigned k = q0 + lane;
            unsigned v = 0;
            const unsigned b = k < a1 ? fetch_mover(k, v) : kMover;
            body(b, v);
        }
        for (unsigned q0 = max(k0, nbef); q0 < a2; q0 += 32) {   // segment t: its stayers
            const unsigned k = q0 + lane;
            unsigned v = 0, b = kMover;
            if (k < a2) {
                const unsigned q = cls_off + (k - nbef);
                v = (unsigned)sb + (k - nbef);
                b = q < cls_n ? cls_s[q] : cls[v];
            }
            body(b, v);
        }
        for (unsigned q0 = max(k0, nbef + seglen); q0 < k1; q0 += 32) {   // movers from later segments
            const unsigned k = q0 + lane;
            unsigned v = 0;
            const unsigned b = k < k1 ? fetch_mover(k - seglen, v) : kMover;
            body(b, v);
        }
    };
    walk([&](unsigned b, unsigned) {
        if (b != kMover) atomicAdd(&cw[warp][b], 1u);
    });
    __syncthreads();
    if (warp == 0) {
        unsigned run = 0;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            const unsigned c = cw[w][lane];
            pre[w][lane] = run;
            run += c;
            cw[w][lane] = 0;
        }
        cnt[lane] = run;
        unsigned m = run;
        for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) ntab = m < (unsigned)kRankTab ? m : (unsigned)kRankTab;
    }
    __syncthreads();
    const bool banked = r.banked != 0;
    const unsigned nt = banked ? ntab : 0u;
    for (unsigned rr = tid; rr < nt; rr += kSortThreads) {
        unsigned m = 0;
        for (int b = 0; b < 32; ++b) m |= (cnt[b] > rr ? 1u : 0u) << b;
        gmask[rr] = m;
    }
    __syncthreads();
    if (warp == 0 && nt) {
        unsigned run = 0;
        for (unsigned r0 = 0; r0 < nt; r0 += 32) {
            const unsigned rr = r0 + lane;
            const unsigned g = rr < nt ? __popc(gmask[rr]) : 0u;
            unsigned inc = g;
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned y = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += y;
            }
            if (rr < nt) gS[rr] = run + inc - g;
            run += __shfl_sync(0xffffffffu, inc, 31);
        }
    }
    __syncthreads();
    walk([&](unsigned b, unsigned v) {
        const bool ok = b != kMover;
        unsigned peers = __ballot_sync(0xffffffffu, ok);   // lanes of the same bank
#pragma unroll
        for (int bit = 0; bit < 5; ++bit) {
            const unsigned m = __ballot_sync(0xffffffffu, (b >> bit) & 1u);
            peers &= ((b >> bit) & 1u) ? m : ~m;
        }
        const unsigned before = ok ? cw[warp][b] : 0u;
        __syncwarp();
        if (ok && (__ffs(peers) - 1) == lane) cw[warp][b] = before + __popc(peers);
        __syncwarp();
        if (!ok) return;
        const unsigned rank = pre[warp][b] + before + __popc(peers & ltm);   // among the tile's bank b
        unsigned slot;
        if (!banked) {
            slot = rank;
        } else if (rank < nt) {
            slot = gS[rank] + __popc(gmask[rank] & ((1u << b) - 1u));
        } else {
            unsigned S = 0, below = 0;
            for (int bb = 0; bb < 32; ++bb) {
                const unsigned cb = cnt[bb];
                S += cb < rank ? cb : rank;
                if (bb < (int)b && cb > rank) ++below;
            }
            slot = S + below;
        }
        if (slot < nT) perm[nb + slot] = v;
    });
}

// Permute every particle array, dst[o] = src[perm[o]], four slots per thread:
// one 16-byte read of perm, four gathers per array in flight together, 16-byte
// writes.
template <typename T>
__device__ __forceinline__ void gather4(const T *__restrict__ src, T *__restrict__ dst, long long o, uint4 p)
{
    const T a = __ldg(src + p.x), b = __ldg(src + p.y), c = __ldg(src + p.z), d = __ldg(src + p.w);
    if (sizeof(T) == 4) {
        float4 v;
        v.x = __int_as_float((int)*reinterpret_cast<const unsigned *>(&a));
        v.y = __int_as_float((int)*reinterpret_cast<const unsigned *>(&b));
        v.z = __int_as_float((int)*reinterpret_cast<const unsigned *>(&c));
        v.w = __int_as_float((int)*reinterpret_cast<const unsigned *>(&d));
        *reinterpret_cast<float4 *>(dst + o) = v;
    } else {
        double2 v0, v1;
        v0.x = __longlong_as_double((long long)*reinterpret_cast<const unsigned long long *>(&a));
        v0.y = __longlong_as_double((long long)*reinterpret_cast<const unsigned long long *>(&b));
        v1.x = __longlong_as_double((long long)*reinterpret_cast<const unsigned long long *>(&c));
        v1.y = __longlong_as_double((long long)*reinterpret_cast<const unsigned long long *>(&d));
        reinterpret_cast<double2 *>(dst + o)[0] = v0;
        reinterpret_cast<double2 *>(dst + o)[1] = v1;
    }
}

template <typename R, int DIM>
__global__ void __launch_bounds__(256) k_permute4(long long n, const unsigned *__restrict__ perm, Pool<R> src,
                                                  Pool<R> dst)
{
    const long long o = (blockIdx.x * (long long)blockDim.x + threadIdx.x) * 4;
    if (o >= n) return;
    if (o + 4 <= n) {
        const uint4 p = *reinterpret_cast<const uint4 *>(perm + o);
        gather4(src.cell, dst.cell, o, p);
        gather4(src.off[0], dst.off[0], o, p);
        gather4(src.off[1], dst.off[1], o, p);
        if (DIM == 3) gather4(src.off[2], dst.off[2], o, p);
        gather4(src.w[0], dst.w[0], o, p);
        gather4(src.w[1], dst.w[1], o, p);
        gather4(src.w[2], dst.w[2], o, p);
        gather4(src.id, dst.id, o, p);
        return;
    }
    for (long long q = o; q < n; ++q) {
        const unsigned s = perm[q];
        dst.cell[q] = src.cell[s];
        dst.off[0][q] = src.off[0][s];
        dst.off[1][q] = src.off[1][s];
        if (DIM == 3) dst.off[2][q] = src.off[2][s];
        dst.w[0][q] = src.w[0][s];
        dst.w[1][q] = src.w[1][s];
        dst.w[2][q] = src.w[2][s];
        dst.id[q] = src.id[s];
    }
}

// tile_start[t] = first sorted position with key >= t, for t in [0, total_tiles].
__global__ void k_tile_start(const unsigned *keys, long long n, int total_tiles, long long *tile_start)
{
    const long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (o >= n) return;
    const long long k = keys[o];
    const long long kp = o == 0 ? -1 : (long long)keys[o - 1];
    for (long long t = kp + 1; t <= k; ++t) tile_start[t] = o;
    if (o == n - 1)
        for (long long t = k + 1; t <= total_tiles; ++t) tile_start[t] = n;
}

__global__ void k_item_counts(const long long *tile_start, int total_tiles, int ppi, unsigned *counts)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total_tiles) return;
    const long long c = tile_start[t + 1] - tile_start[t];
    counts[t] = (unsigned)((c + ppi - 1) / ppi);
}

__global__ void k_items(const long long *tile_start, const unsigned *scan, int total_tiles, int ppi,
                        const GroupDev *groups, int ngroups, WorkItem *items, int *n_items)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total_tiles) return;
    const long long b = tile_start[t], e = tile_start[t + 1];
    const int cnt = (int)((e - b + ppi - 1) / ppi);
    int lo = 0, hi = ngroups;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (groups[mid].tile_base <= t) lo = mid; else hi = mid;
    }
    const unsigned s = scan[t];
    for (int q = 0; q < cnt; ++q) {
        WorkItem w;
        w.group = lo;
        w.tile = t - groups[lo].tile_base;
        w.begin = b + (long long)q * ppi;
        w.end = w.begin + ppi < e ? w.begin + ppi : e;
        items[s + q] = w;
    }
    if (t == total_tiles - 1) *n_items = (int)(s + cnt);
}

template <typename R, int DIM>
static cudaError_t permute4_launch(cudaStream_t st, long long total, const PoolBuf &src, const PoolBuf &dst,
                                   const unsigned *perm)
{
    Pool<R> s, d;
    s.cell = src.cell; s.id = src.id; d.cell = dst.cell; d.id = dst.id;
    for (int c = 0; c < 3; ++c) {
        s.off[c] = (R *)src.off[c]; s.w[c] = (R *)src.w[c];
        d.off[c] = (R *)dst.off[c]; d.w[c] = (R *)dst.w[c];
    }
    const long long nq = (total + 3) / 4;
    k_permute4<R, DIM><<<(unsigned)((nq + 255) / 256), 256, 0, st>>>(total, perm, s, d);
    return cudaGetLastError();
}

static cudaError_t launch_permute4(int prec, int dims, cudaStream_t st, long long total, const PoolBuf &src,
                                   const PoolBuf &dst, const unsigned *perm)
{
    if (prec == 0)
        return dims == 3 ? permute4_launch<double, 3>(st, total, src, dst, perm)
                         : permute4_launch<double, 2>(st, total, src, dst, perm);
    return dims == 3 ? permute4_launch<float, 3>(st, total, src, dst, perm)
                     : permute4_launch<float, 2>(st, total, src, dst, perm);
}

static cudaError_t permute_and_build(int prec, int dims, cudaStream_t st, long long total, const PoolBuf &src,
                                     const PoolBuf &dst, const unsigned *perm, const GroupDev *groups, int ngroups,
                                     int total_tiles, SortScratch &scr, const long long *tile_start,
                                     unsigned *item_scan, WorkItem *items, int *n_items, int particles_per_item,
                                     int *launches);

cudaError_t sort_and_build_items(int prec, int dims, cudaStream_t st, long long total, const PoolBuf &src,
                                 const PoolBuf &dst, const GroupDev *groups, const long long *group_base_dev,
                                 int ngroups, const RunDev *runs, int total_tiles, SortScratch &scr,
                                 long long *tile_start, unsigned *item_scan, WorkItem *items, int *n_items,
                                 int particles_per_item, int halo, int banked, int half, int *launches,
                                 unsigned char *lane_cell, int *lane_count, int resort, const unsigned **perm_out)
{
    if (lane_cell) perm_out = nullptr;
    cudaError_t e;
    if (total <= 0 || ngroups <= 0) {
        e = cudaMemsetAsync(n_items, 0, sizeof(int), st);
        if (e != cudaSuccess) return e;
        return cudaMemsetAsync(tile_start, 0, sizeof(long long) * (total_tiles + 1), st);
    }
    const int nt = 256;
    const unsigned nbp = (unsigned)((total + nt - 1) / nt);
    int nbits = 1;
    while ((1ll << nbits) < (long long)total_tiles) ++nbits;
    const long long nchunks = (total + kChunk - 1) / kChunk;
    int cur = 0;
    if (resort && !lane_cell) {
        // tile_start holds the previous sort's segments of this pool
        const int ntp = total_tiles + 1;
        // per tile: movers out (then their offsets), stayers (then the new starts), the
        // sorted movers' starts, and the movers in from earlier segments
        unsigned *mcnt = scr.tcnt[0], *stay = scr.tcnt[1], *mstart = scr.tcnt[2], *mbef = scr.tcnt[3];
        unsigned *aft = scr.tcnt[4];   // first mover of each tile from a later segment
        if ((e = cudaMemsetAsync(scr.m_total, 0, sizeof(unsigned), st)) != cudaSuccess) return e;
        BankRule rule;
        rule.banked = banked;
        rule.half = half;
        rule.halo = halo;
        rule.dims = dims;
        rule.P0 = rule.P1 = 0;
        rule.prec = prec;
        for (int c = 0; c < 3; ++c) rule.off[c] = src.off[c];
        k_resort_classify<<<(unsigned)ntp, kSortThreads, 0, st>>>(tile_start, total, total_tiles, src.cell, groups,
                                                                  ngroups, runs, rule, scr.cls, mcnt, stay,
                                                                  scr.m_total);
        *launches += 1;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = exclusive_scan(mcnt, ntp, scr.block_sums, st, launches)) != cudaSuccess) return e;
        k_resort_movers<<<(unsigned)total_tiles, kSortThreads, 0, st>>>(tile_start, total, mcnt, scr.cls, src.cell,
                                                                        groups, ngroups, runs, total_tiles,
                                                                        scr.keys[0], scr.vals[0]);
        *launches += 1;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        unsigned *hist_n = scr.m_total + 1;
        k_hist_count<<<1, 1, 0, st>>>(scr.m_total, total, hist_n);
        *launches += 1;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        for (int shift = 0; shift < nbits; shift += 8) {
            k_upsweep_dev<<<(unsigned)nchunks, kSortThreads, 0, st>>>(scr.keys[cur], scr.m_total, total, shift,
                                                                      scr.hist, hist_n);
            *launches += 1;
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            if ((e = exclusive_scan_dev(scr.hist, 256 * nchunks, hist_n, scr.block_sums, st, launches)) != cudaSuccess)
                return e;
            k_downsweep_dev<<<(unsigned)nchunks, kSortThreads, 0, st>>>(scr.keys[cur], scr.vals[cur], scr.m_total,
                                                                        total, shift, scr.hist, hist_n,
                                                                        scr.keys[1 - cur], scr.vals[1 - cur]);
            *launches += 1;
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            cur = 1 - cur;
        }
        const unsigned nbt = (unsigned)((ntp + nt - 1) / nt);
        if ((e = cudaMemsetAsync(aft, 0xff, sizeof(unsigned) * ntp, st)) != cudaSuccess) return e;
        k_resort_bounds<<<(unsigned)std::min<long long>((total + nt) / nt, 4096), nt, 0, st>>>(scr.keys[cur],
                                                                                              scr.vals[cur],
                                                                                              scr.m_total, total,
                                                                                              total_tiles, tile_start,
                                                                                              mstart, aft);
        *launches += 1;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        k_resort_newcnt<<<nbt, nt, 0, st>>>(ntp, stay, mstart, aft, mbef);
        *launches += 1;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = exclusive_scan(stay, ntp, scr.block_sums, st, launches)) != cudaSuccess) return e;
        k_resort_order<<<(unsigned)total_tiles, kSortThreads, 0, st>>>(tile_start, total, stay, mstart, mbef,
                                                                       scr.vals[cur], scr.cls, src.cell, groups,
                                                                       ngroups, runs, rule, scr.vals[1 - cur]);
        *launches += 1;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if (perm_out) {
            *perm_out = scr.vals[1 - cur];
        } else {
            if ((e = launch_permute4(prec, dims, st, total, src, dst, scr.vals[1 - cur])) != cudaSuccess) return e;
            *launches += 1;
        }
        k_resort_tile_start<<<nbt, nt, 0, st>>>(ntp, stay, tile_start);
        *launches += 1;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        return build_items(st, tile_start, total_tiles, particles_per_item, groups, ngroups, scr, item_scan, items,
                           n_items, launches);
    }
    k_keys<<<nbp, nt, 0, st>>>(total, src.cell, group_base_dev, ngroups, groups, runs, scr.keys[0], scr.vals[0]);
    *launches += 1;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;

    for (int shift = 0; shift < nbits; shift += 8) {
        k_upsweep<<<(unsigned)nchunks, kSortThreads, 0, st>>>(scr.keys[cur], total, shift, scr.hist, nchunks);
        *launches += 1;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = exclusive_scan(scr.hist, 256 * nchunks, scr.block_sums, st, launches)) != cudaSuccess) return e;
        k_downsweep<<<(unsigned)nchunks, kSortThreads, 0, st>>>(scr.keys[cur], scr.vals[cur], total, shift,
                                                                scr.hist, nchunks, scr.keys[1 - cur],
                                                                scr.vals[1 - cur]);
        *launches += 1;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        cur = 1 - cur;
    }

    // tile starts, then the bank interleave inside every tile (into the other value buffer)
    k_tile_start<<<nbp, nt, 0, st>>>(scr.keys[cur], total, total_tiles, tile_start);
    *launches += 1;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (lane_cell && lane_count) {
        k_cell_lane_order<<<(unsigned)total_tiles, kSortThreads, 0, st>>>(tile_start, scr.vals[cur], scr.vals[1 - cur],
                                                                        src.cell, groups, ngroups, runs, lane_cell,
                                                                        lane_count);
        *launches += 1;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        cur = 1 - cur;
    } else if (banked) {
        k_bank_order<<<(unsigned)total_tiles, kSortThreads, 0, st>>>(tile_start, scr.vals[cur], scr.vals[1 - cur],
                                                                   src.cell, groups, ngroups, runs, halo, dims, half,
                                                                   prec, src.off[0], src.off[1], src.off[2]);
        *launches += 1;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        cur = 1 - cur;
    }
    if (perm_out) {
        *perm_out = scr.vals[cur];
        return build_items(st, tile_start, total_tiles, particles_per_item, groups, ngroups, scr, item_scan, items,
                           n_items, launches);
    }
    return permute_and_build(prec, dims, st, total, src, dst, scr.vals[cur], groups, ngroups, total_tiles, scr,
                             tile_start, item_scan, items, n_items, particles_per_item, launches);
}

cudaError_t launch_permute(int prec, int dims, cudaStream_t st, long long total, const PoolBuf &src,
                           const PoolBuf &dst, const unsigned *perm)
{
    return total > 0 ? launch_permute4(prec, dims, st, total, src, dst, perm) : cudaSuccess;
}

static cudaError_t permute_and_build(int prec, int dims, cudaStream_t st, long long total, const PoolBuf &src,
                                     const PoolBuf &dst, const unsigned *perm, const GroupDev *groups, int ngroups,
                                     int total_tiles, SortScratch &scr, const long long *tile_start,
                                     unsigned *item_scan, WorkItem *items, int *n_items, int particles_per_item,
                                     int *launches)
{
    cudaError_t e = launch_permute4(prec, dims, st, total, src, dst, perm);
    *launches += 1;
    if (e != cudaSuccess) return e;
    return build_items(st, tile_start, total_tiles, particles_per_item, groups, ngroups, scr, item_scan, items, n_items,
                       launches);
}

cudaError_t build_items(cudaStream_t st, const long long *tile_start, int total_tiles, int particles_per_item,
                        const GroupDev *groups, int ngroups, SortScratch &scr, unsigned *item_scan, WorkItem *items,
                        int *n_items, int *launches)
{
    cudaError_t e;
    const int nt = 256;
    const unsigned nbt = (unsigned)((total_tiles + nt - 1) / nt);
    k_item_counts<<<nbt, nt, 0, st>>>(tile_start, total_tiles, particles_per_item, item_scan);
    *launches += 1;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = exclusive_scan(item_scan, total_tiles, scr.block_sums, st, launches)) != cudaSuccess) return e;
    k_items<<<nbt, nt, 0, st>>>(tile_start, item_scan, total_tiles, particles_per_item, groups, ngroups, items,
                                n_items);
    *launches += 1;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Stable radix sort of (key, value) pairs in caller-provided scratch, and the
// tile starts of the sorted keys.  Used by the allocation-free sort entry point;
// the same kernels as sort_and_build_items.
// ---------------------------------------------------------------------------
cudaError_t radix_sort_pairs(cudaStream_t st, long long n, int nbits, unsigned *const keys[2], unsigned *const vals[2],
                             unsigned *hist, unsigned *block_sums, int *cur_out)
{
    cudaError_t e;
    int launches = 0;
    const long long nchunks = (n + kChunk - 1) / kChunk;
    int cur = 0;
    for (int shift = 0; shift < nbits; shift += 8) {
        k_upsweep<<<(unsigned)nchunks, kSortThreads, 0, st>>>(keys[cur], n, shift, hist, nchunks);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = exclusive_scan(hist, 256 * nchunks, block_sums, st, &launches)) != cudaSuccess) return e;
        k_downsweep<<<(unsigned)nchunks, kSortThreads, 0, st>>>(keys[cur], vals[cur], n, shift, hist, nchunks,
                                                                keys[1 - cur], vals[1 - cur]);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        cur = 1 - cur;
    }
    *cur_out = cur;
    return cudaSuccess;
}

cudaError_t launch_tile_start(cudaStream_t st, const unsigned *sorted_keys, long long n, int total_tiles,
                              long long *tile_start)
{
    const int nt = 256;
    k_tile_start<<<(unsigned)((n + nt - 1) / nt), nt, 0, st>>>(sorted_keys, n, total_tiles, tile_start);
    return cudaGetLastError();
}

}  // namespace pic
