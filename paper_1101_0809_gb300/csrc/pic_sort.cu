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

__global__ void k_scan_sums(const unsigned *in, long long n, unsigned *sums)
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

__global__ void k_scan_single(unsigned *a, long long n)
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

__global__ void k_scan_apply(unsigned *a, long long n, const unsigned *sums)
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

__global__ void k_upsweep(const unsigned *keys, long long n, int shift, unsigned *hist, long long nchunks)
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

__global__ void __launch_bounds__(kSortThreads) k_downsweep(const unsigned *keys, const unsigned *vals, long long n,
                                                            int shift, const unsigned *hist, long long nchunks,
                                                            unsigned *keys_out, unsigned *vals_out)
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

// Permute every particle array: dst[o] = src[perm[o]].
template <typename R, int DIM>
__global__ void k_permute(long long n, const unsigned *perm, Pool<R> src, Pool<R> dst)
{
    const long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (o >= n) return;
    const unsigned s = perm[o];
    dst.cell[o] = src.cell[s];
    dst.off[0][o] = src.off[0][s];
    dst.off[1][o] = src.off[1][s];
    if (DIM == 3) dst.off[2][o] = src.off[2][s];
    dst.w[0][o] = src.w[0][s];
    dst.w[1][o] = src.w[1][s];
    dst.w[2][o] = src.w[2][s];
    dst.id[o] = src.id[s];
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

cudaError_t sort_and_build_items(int prec, int dims, cudaStream_t st, long long total, const PoolBuf &src,
                                 const PoolBuf &dst, const GroupDev *groups, const long long *group_base_dev,
                                 int ngroups, const RunDev *runs, int total_tiles, SortScratch &scr,
                                 long long *tile_start, unsigned *item_scan, WorkItem *items, int *n_items,
                                 int particles_per_item, int halo, int banked, int half, int *launches,
                                 unsigned char *lane_cell, int *lane_count)
{
    cudaError_t e;
    if (total <= 0 || ngroups <= 0) {
        e = cudaMemsetAsync(n_items, 0, sizeof(int), st);
        if (e != cudaSuccess) return e;
        return cudaMemsetAsync(tile_start, 0, sizeof(long long) * (total_tiles + 1), st);
    }
    const int nt = 256;
    const unsigned nbp = (unsigned)((total + nt - 1) / nt);
    k_keys<<<nbp, nt, 0, st>>>(total, src.cell, group_base_dev, ngroups, groups, runs, scr.keys[0], scr.vals[0]);
    *launches += 1;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;

    int nbits = 1;
    while ((1ll << nbits) < (long long)total_tiles) ++nbits;
    const long long nchunks = (total + kChunk - 1) / kChunk;
    int cur = 0;
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

    if (prec == 0) {
        Pool<double> s, d;
        s.cell = src.cell; s.id = src.id; d.cell = dst.cell; d.id = dst.id;
        for (int c = 0; c < 3; ++c) {
            s.off[c] = (double *)src.off[c]; s.w[c] = (double *)src.w[c];
            d.off[c] = (double *)dst.off[c]; d.w[c] = (double *)dst.w[c];
        }
        if (dims == 3) k_permute<double, 3><<<nbp, nt, 0, st>>>(total, scr.vals[cur], s, d);
        else k_permute<double, 2><<<nbp, nt, 0, st>>>(total, scr.vals[cur], s, d);
    } else {
        Pool<float> s, d;
        s.cell = src.cell; s.id = src.id; d.cell = dst.cell; d.id = dst.id;
        for (int c = 0; c < 3; ++c) {
            s.off[c] = (float *)src.off[c]; s.w[c] = (float *)src.w[c];
            d.off[c] = (float *)dst.off[c]; d.w[c] = (float *)dst.w[c];
        }
        if (dims == 3) k_permute<float, 3><<<nbp, nt, 0, st>>>(total, scr.vals[cur], s, d);
        else k_permute<float, 2><<<nbp, nt, 0, st>>>(total, scr.vals[cur], s, d);
    }
    *launches += 1;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;

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
