// pic_api.cu -- the C ABI of libpic (include/pic.h): argument checks, device
// memory, stream ordering, and the order of the step of the paper's Appendix.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <cstddef>
#include <algorithm>
#include <array>
#include <atomic>
#include <string>
#include <new>

#include "../../include/pic.h"
#include "pic_internal.h"

using namespace pic;

namespace {

thread_local char t_err[512] = "";

int fail(int code, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(t_err, sizeof(t_err), fmt, ap);
    va_end(ap);
    return code;
}

int cuda_fail(cudaError_t e, const char *what)
{
    cudaGetLastError();   // clear a non-sticky error
    return fail(e == cudaErrorMemoryAllocation ? PIC_ERR_OOM : PIC_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call, what)                                  \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

constexpr int kDiagBlocks = 1024;

// Device-to-device copy of up to kCopySegs segments in one launch (blockIdx.y
// = segment), plus optionally a small block of bytes passed by value (a
// snapshot header, written in stream order without a host copy).  Segments
// whose source and destination agree modulo 16 bytes move as 16-byte words
// between byte-wise heads and tails; others move byte-wise.
constexpr int kCopySegs = 16;
struct CopyList {
    const unsigned char *src[kCopySegs];
    unsigned char *dst[kCopySegs];
    long long bytes[kCopySegs];
    int n;
    int inl_bytes;                 // 0..64 bytes of `inl` to write to inl_dst
    unsigned char *inl_dst;
    unsigned char inl[64];
};

__global__ void k_copy_segments(const CopyList L)
{
    const int sg = blockIdx.y;
    const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long stride = (long long)gridDim.x * blockDim.x;
    if (sg == L.n) {
        if (t0 < L.inl_bytes) L.inl_dst[t0] = L.inl[t0];
        return;
    }
    const unsigned char *src = L.src[sg];
    unsigned char *dst = L.dst[sg];
    const long long nb = L.bytes[sg];
    const unsigned long long sa = (unsigned long long)src, da = (unsigned long long)dst;
    if (((sa ^ da) & 15ull) == 0) {
        long long head = (long long)((16ull - (sa & 15ull)) & 15ull);
        if (head > nb) head = nb;
        const long long n16 = (nb - head) >> 4;
        if (t0 < head) dst[t0] = src[t0];
        const uint4 *s4 = reinterpret_cast<const uint4 *>(src + head);
        uint4 *d4 = reinterpret_cast<uint4 *>(dst + head);
        for (long long i = t0; i < n16; i += stride) d4[i] = s4[i];
        for (long long i = head + (n16 << 4) + t0; i < nb; i += stride) dst[i] = src[i];
    } else {
        for (long long i = t0; i < nb; i += stride) dst[i] = src[i];
    }
}

// Collects copies and issues them: device-to-device ones as k_copy_segments
// launches, the others (host memory on one side) as cudaMemcpyAsync.
struct Copier {
    cudaStream_t st;
    cudaMemcpyKind kind;
    CopyList L;
    long long maxb = 0;
    int launches = 0;
    Copier(cudaStream_t s, cudaMemcpyKind k) : st(s), kind(k)
    {
        memset(&L, 0, sizeof(L));
    }
    cudaError_t flush()
    {
        if (L.n == 0 && L.inl_bytes == 0) return cudaSuccess;
        const long long per = 256LL * 16 * 4;   // bytes per thread block and pass
        long long bx = (maxb + per - 1) / per;
        if (bx < 1) bx = 1;
        if (bx > 2048) bx = 2048;
        k_copy_segments<<<dim3((unsigned)bx, (unsigned)(L.n + (L.inl_bytes ? 1 : 0))), 256, 0, st>>>(L);
        ++launches;
        const cudaError_t e = cudaGetLastError();
        memset(&L, 0, sizeof(L));
        maxb = 0;
        return e;
    }
    cudaError_t add(void *dst, const void *src, size_t bytes)
    {
        if (bytes == 0) return cudaSuccess;
        if (kind != cudaMemcpyDeviceToDevice) return cudaMemcpyAsync(dst, src, bytes, kind, st);
        if (L.n == kCopySegs) {
            const cudaError_t e = flush();
            if (e != cudaSuccess) return e;
        }
        L.src[L.n] = (const unsigned char *)src;
        L.dst[L.n] = (unsigned char *)dst;
        L.bytes[L.n] = (long long)bytes;
        ++L.n;
        if ((long long)bytes > maxb) maxb = (long long)bytes;
        return cudaSuccess;
    }
    void inline_bytes(void *dst, const void *src, int bytes)
    {
        L.inl_bytes = bytes;
        L.inl_dst = (unsigned char *)dst;
        memcpy(L.inl, src, (size_t)bytes);
    }
};

size_t elem(const pic_grid *g) { return g->prec == PIC_FP64 ? sizeof(double) : sizeof(float); }

// Allocation-failure injection (pic_inject_alloc_failure): the number of device
// allocations still to succeed before one fails; -1 when disarmed.
std::atomic<long long> g_alloc_fail_in{-1};

bool injected_alloc_failure()
{
    long long n = g_alloc_fail_in.load();
    while (n >= 0) {
        if (g_alloc_fail_in.compare_exchange_weak(n, n - 1)) return n == 0;
    }
    return false;
}

template <typename T>
cudaError_t dalloc(T **p, size_t count)
{
    *p = nullptr;
    if (count == 0) return cudaSuccess;
    if (injected_alloc_failure()) return cudaErrorMemoryAllocation;
    return cudaMalloc((void **)p, count * sizeof(T));
}

cudaError_t dalloc_bytes(void **p, size_t bytes)
{
    *p = nullptr;
    if (bytes == 0) return cudaSuccess;
    if (injected_alloc_failure()) return cudaErrorMemoryAllocation;
    return cudaMalloc(p, bytes);
}

void dfree(void *p)
{
    if (p) cudaFree(p);
}

void free_pool(PoolBuf &P)
{
    dfree(P.cell);
    dfree(P.id);
    for (int c = 0; c < 3; ++c) {
        dfree(P.off[c]);
        dfree(P.w[c]);
    }
    P = PoolBuf();
}

cudaError_t alloc_pool(pic_grid *g, PoolBuf &P, long long n)
{
    P = PoolBuf();
    cudaError_t e;
    n = (n + 3) & ~3LL;   // whole 16-byte groups: the re-sort copies segments rounded out to them
    if ((e = dalloc(&P.cell, n)) != cudaSuccess) return e;
    if ((e = dalloc(&P.id, n)) != cudaSuccess) return e;
    for (int c = 0; c < 3; ++c) {
        if (c < g->dims && (e = dalloc_bytes(&P.off[c], n * elem(g))) != cudaSuccess) return e;
        if ((e = dalloc_bytes(&P.w[c], n * elem(g))) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

void free_sort(pic_grid *g)
{
    for (int b = 0; b < 2; ++b) {
        dfree(g->sort.keys[b]);
        dfree(g->sort.vals[b]);
    }
    dfree(g->sort.hist);
    dfree(g->sort.block_sums);
    for (int c = 0; c < 5; ++c) dfree(g->sort.tcnt[c]);
    dfree(g->sort.m_total);
    dfree(g->sort.cls);
    g->sort = SortScratch();
    g->tiles_valid = false;
    dfree(g->tile_start);
    dfree(g->item_scan);
    dfree(g->items);
    dfree(g->lane_cell);
    dfree(g->lane_count);
    dfree(g->drift);
    g->tile_start = nullptr;
    g->item_scan = nullptr;
    g->items = nullptr;
    g->lane_cell = nullptr;
    g->lane_count = nullptr;
    g->drift = nullptr;
}

int launch_count_add(pic_grid *g, int n)
{
    g->launches += n;
    return n;
}

cudaEvent_t prof_event(pic_grid *g)
{
    if (!g->prof_free.empty()) {
        cudaEvent_t e = g->prof_free.back();
        g->prof_free.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

// Records an event pair around one launch group when profiling is on.
struct ProfScope {
    pic_grid *g;
    int cat;
    cudaEvent_t a = nullptr, b = nullptr;
    ProfScope(pic_grid *g_, int cat_) : g(g_), cat(cat_)
    {
        if (!g->profiling) return;
        a = prof_event(g);
        b = prof_event(g);
        if (a && b) cudaEventRecord(a, g->stream);
    }
    ~ProfScope()
    {
        if (!a || !b) return;
        cudaEventRecord(b, g->stream);
        g->prof_marks.push_back({cat, {a, b}});
    }
};

void prof_clear(pic_grid *g)
{
    for (auto &m : g->prof_marks) {
        g->prof_free.push_back(m.second.first);
        g->prof_free.push_back(m.second.second);
    }
    g->prof_marks.clear();
}

void graph_drop(pic_grid *g)
{
    if (g->graph_exec) cudaGraphExecDestroy(g->graph_exec);
    g->graph_exec = nullptr;
    g->graph_valid = false;
}

// (Re)allocate everything whose size depends on the particle count.
int size_particle_buffers(pic_grid *g, long long total)
{
    free_sort(g);
    dfree(g->old_cell);
    g->old_cell = nullptr;
    for (int c = 0; c < 3; ++c) {
        dfree(g->old_off[c]);
        g->old_off[c] = nullptr;
    }
    const long long nchunks = (total + 4095) / 4096;
    const long long hist = 256 * std::max(1LL, nchunks);
    const long long sums = std::max<long long>((hist + 2047) / 2048, (g->total_tiles + 2047) / 2048) + 1;
    for (int b = 0; b < 2; ++b) {
        CK(dalloc(&g->sort.keys[b], std::max(1LL, total)), "sort keys");
        CK(dalloc(&g->sort.vals[b], std::max(1LL, total)), "sort values");
    }
    CK(dalloc(&g->sort.hist, hist), "sort histogram");
    CK(dalloc(&g->sort.block_sums, sums), "scan sums");
    for (int c = 0; c < 5; ++c) CK(dalloc(&g->sort.tcnt[c], (size_t)g->total_tiles + 1), "re-sort counts");
    CK(dalloc(&g->sort.m_total, 2), "re-sort mover count");   // movers, then their histogram length
    CK(dalloc(&g->sort.cls, (std::max(1LL, total) + 3) & ~3LL), "re-sort classes");   // whole 4-byte words
    g->sort.capacity = total;
    g->sort.hist_capacity = hist;
    g->sort.sums_capacity = sums;
    CK(dalloc(&g->tile_start, (size_t)g->total_tiles + 1), "tile starts");
    CK(dalloc(&g->item_scan, (size_t)g->total_tiles + 1), "item scan");
    g->max_items = g->total_tiles + (int)((total + g->ppi - 1) / g->ppi) + 1;
    CK(dalloc(&g->items, (size_t)g->max_items), "work items");
    if (g->sort_order == PIC_SORT_CELL_LANES) {
        CK(dalloc(&g->lane_cell, (size_t)std::max(1, g->total_tiles) * 128), "lane cells");
        CK(dalloc(&g->lane_count, (size_t)std::max(1, g->total_tiles) * 128), "lane counts");
        CK(dalloc(&g->drift, std::max(1LL, total)), "drift lists");
    }
    CK(dalloc(&g->old_cell, std::max(1LL, total)), "saved cells");
    for (int c = 0; c < g->dims; ++c) CK(dalloc_bytes(&g->old_off[c], std::max(1LL, total) * elem(g)), "saved offsets");
    return PIC_OK;
}

int upload_groups(pic_grid *g)
{
    g->tiles_valid = false;   // the next sort starts from the keys alone
    dfree(g->d_groups);
    dfree(g->d_group_base);
    g->d_groups = nullptr;
    g->d_group_base = nullptr;
    const int ng = (int)g->groups.size();
    std::vector<GroupDev> gd(std::max(1, ng));
    std::vector<long long> base(ng + 1, 0);
    int tb = 0;
    long long pb = 0;
    for (int q = 0; q < ng; ++q) {
        HostGroup &h = g->groups[q];
        const RunDev &rn = g->runs[h.run].dev;
        h.tile_base = tb;
        h.ntiles = rn.ntile[0] * rn.ntile[1] * rn.ntile[2];
        h.base = pb;
        tb += h.ntiles;
        pb += h.n;
        gd[q].run = h.run;
        gd[q].tile_base = h.tile_base;
        gd[q].base = h.base;
        gd[q].n = h.n;
        gd[q].qm = h.q / h.m;
        gd[q].qp = h.q * h.weight;
        gd[q].mp = h.m * h.weight;
        // bound on |contribution| of one particle to one face (|D| <= 1,
        // |P+| <= 2, |P-| <= 1, |u_z| <= c), then the power-of-two scale that
        // maps it to 2^R with R = 46 - log2(particles per block) (see FixedAcc)
        const double qV = std::fabs(gd[q].qp) / rn.V;
        double bound;
        if (g->dims == 3) {
            bound = 0.25 * std::max(rn.d[0], std::max(rn.d[1], rn.d[2])) / rn.dt * qV * (4.0 + 4.0 / 3.0);
        } else {
            bound = std::max(0.5 * std::max(rn.d[0], rn.d[1]) / rn.dt * qV * 2.0, 0.25 * qV * rn.c * (4.0 + 4.0 / 3.0));
        }
        int lg = 0;
        while ((1LL << lg) < (long long)g->ppi) ++lg;
        const int R = 46 - lg;
        const int e = bound > 0.0 ? R - (int)std::ceil(std::log2(bound)) : 0;
        gd[q].jscale = (float)std::ldexp(1.0, e);
        gd[q].jinv = (float)std::ldexp(1.0, -e);
        // charge of one particle on one cell: (q_p/V) Sx Sy Sz <= q_p/V
        const int er = qV > 0.0 ? R - (int)std::ceil(std::log2(qV)) : 0;
        gd[q].rscale = (float)std::ldexp(1.0, er);
        gd[q].rinv = (float)std::ldexp(1.0, -er);
        gd[q].hq = 0.5 * gd[q].qm * rn.dt;
        if (g->dims == 3) {
            for (int a = 0; a < 3; ++a) gd[q].kf[a] = -0.25 * rn.d[a] / rn.dt * gd[q].qp / rn.V;
        } else {
            gd[q].kf[0] = -0.5 * rn.d[0] / rn.dt * gd[q].qp / rn.V;
            gd[q].kf[1] = -0.5 * rn.d[1] / rn.dt * gd[q].qp / rn.V;
            gd[q].kf[2] = 0.25 * gd[q].qp / rn.V;
        }
        gd[q].hqf = (float)gd[q].hq;
        for (int a = 0; a < 3; ++a) {
            gd[q].kff[a] = (float)gd[q].kf[a];
            gd[q].kfsf[a] = gd[q].kff[a] * gd[q].jscale;
        }
        base[q] = h.base;
    }
    base[ng] = pb;
    g->total_tiles = tb;
    CK(dalloc(&g->d_groups, gd.size()), "groups");
    CK(cudaMemcpy(g->d_groups, gd.data(), sizeof(GroupDev) * gd.size(), cudaMemcpyHostToDevice), "groups upload");
    CK(dalloc(&g->d_group_base, base.size()), "group bases");
    CK(cudaMemcpy(g->d_group_base, base.data(), sizeof(long long) * base.size(), cudaMemcpyHostToDevice),
       "group bases upload");
    return PIC_OK;
}

// Applies a sort that pic_step left pending (the arrays in the old order and
// the permutation in the sort scratch): used when no fused particle launch
// follows to apply it.
static int settle(pic_grid *g)
{
    if (!g->pending_perm) return PIC_OK;
    cudaError_t e = launch_permute(g->prec, g->dims, g->stream, g->total, g->pool, g->pool_alt, g->pending_perm);
    launch_count_add(g, 1);
    g->pending_perm = nullptr;
    if (e != cudaSuccess) return cuda_fail(e, "permutation");
    std::swap(g->pool, g->pool_alt);
    return PIC_OK;
}

int do_sort(pic_grid *g, bool defer = false)
{
    int rc = settle(g);
    if (rc != PIC_OK) return rc;
    if (g->total <= 0 || g->groups.empty() || !g->tile_start) {   // nothing to sort
        g->steps_since_sort = 0;
        g->have_old = false;
        return PIC_OK;
    }
    ProfScope ps(g, PIC_PROF_SORT);
    int nl = 0;
    const unsigned *perm = nullptr;
    cudaError_t e = sort_and_build_items(g->prec, g->dims, g->stream, g->total, g->pool, g->pool_alt, g->d_groups,
                                         g->d_group_base, (int)g->groups.size(), g->d_runs, g->total_tiles, g->sort,
                                         g->tile_start, g->item_scan, g->items, g->n_items, g->ppi,
                                         g->halo + (g->order2 == 5 ? 1 : 0),   // the current tile's bank base
                                         g->sort_order == PIC_SORT_BANKED ? 1 : 0, g->order2 == 5 ? 1 : 0, &nl,
                                         g->sort_order == PIC_SORT_CELL_LANES ? g->lane_cell : nullptr,
                                         g->sort_order == PIC_SORT_CELL_LANES ? g->lane_count : nullptr,
                                         g->tiles_valid && g->sort_order != PIC_SORT_CELL_LANES ? 1 : 0,
                                         defer ? &perm : nullptr);
    launch_count_add(g, nl);
    g->tiles_valid = false;
    if (e != cudaSuccess) return cuda_fail(e, "tile sort");
    g->tiles_valid = true;
    if (perm) g->pending_perm = perm;   // the next fused particle launch moves the arrays
    else if (g->total > 0 && !g->groups.empty()) std::swap(g->pool, g->pool_alt);
    if (!g->capturing) graph_drop(g);   // a captured graph assumes its own buffer parity
    g->steps_since_sort = 0;
    g->have_old = false;
    return PIC_OK;
}

// The fused step of a grid in the cell-lane order whose geometry the cell-lane
// kernel is built for.
static bool uses_cell_lanes(const pic_grid *g)
{
    return g->sort_order == PIC_SORT_CELL_LANES &&
           particles_cl_applies(g->dims, g->prec, g->order2, g->tile, g->halo);
}

int launch_part(pic_grid *g, int mode)
{
    ProfScope ps(g, PIC_PROF_PARTICLES);
    if (mode == 0 && uses_cell_lanes(g)) {
        cudaError_t e = launch_particles_cl(g->stream, g->total_tiles, g->tile_start, g->lane_cell, g->lane_count,
                                            g->drift, g->d_groups, (int)g->groups.size(), g->d_runs, g->pool, g->E,
                                            g->B, g->J, g->ppi, g->d_err);
        launch_count_add(g, g->total_tiles > 0 ? 1 : 0);
        if (e != cudaSuccess) return cuda_fail(e, "particle kernel");
        return PIC_OK;
    }
    if (g->pending_perm && (mode != 0 || g->order2 != 3)) {
        const int rc = settle(g);
        if (rc != PIC_OK) return rc;
    }
    const unsigned *perm = g->pending_perm;
    // after a deferred sort: read the old order through the permutation, write the new one
    cudaError_t e = launch_particles(g->dims, g->prec, mode, g->stream, g->items, g->n_items, g->max_items, g->d_runs,
                                     g->d_groups, perm ? g->pool_alt : g->pool, g->E, g->B, g->J, g->old_cell,
                                     g->old_off, g->halo, g->tile[0], g->tile[1], g->tile[2], g->d_err, g->pitch[0],
                                     g->pitch[1], g->order2, perm ? &g->pool : nullptr, perm);
    launch_count_add(g, g->max_items > 0 ? 1 : 0);
    if (perm) {
        g->pending_perm = nullptr;
        std::swap(g->pool, g->pool_alt);
    }
    if (e != cudaSuccess) return cuda_fail(e, "particle kernel");
    return PIC_OK;
}

int launch_fields(pic_grid *g, int which, int zero_j)
{
    long long maxc = 0;
    for (auto &r : g->runs) maxc = std::max(maxc, (long long)r.dev.n[0] * r.dev.n[1] * r.dev.n[2]);
    ProfScope ps(g, which == PIC_B_HALF ? PIC_PROF_YEE_B : PIC_PROF_YEE_E);
    cudaError_t e;
    if (which == PIC_E_FULL && g->vecpot) {   // Eq. dadt with E^n, before the E step changes it
        e = launch_update_A(g->prec, g->stream, g->d_runs, (int)g->runs.size(), maxc, g->d_A, g->E);
        launch_count_add(g, 1);
        if (e != cudaSuccess) return cuda_fail(e, "vector potential");
    }
    e = launch_yee(g->prec, which, zero_j, g->stream, g->d_runs, (int)g->runs.size(), maxc, g->E, g->B, g->J,
                   g->dims, g->d_ant_n);
    launch_count_add(g, 1);
    if (e != cudaSuccess) return cuda_fail(e, "Yee kernel");
    if (which == PIC_E_FULL && g->antennas > 0) {   // the E step ends a step of the antenna clock
        e = launch_antenna_tick(g->stream, g->d_ant_n, (int)g->runs.size());
        launch_count_add(g, 1);
        if (e != cudaSuccess) return cuda_fail(e, "antenna clock");
    }
    return PIC_OK;
}

// Pitches of the shared-memory tiles: the smallest x pitch >= Tx + 2h + 4 and
// y pitch >= Ty + 2h + 4 (up to 32) that spread the tile's cells most evenly over
// the 32 shared-memory banks (so that the banked sort order keeps whole rounds
// of 32 distinct banks), preferring layouts that leave room for two blocks per
// SM.  In 2D only the x pitch matters.
static void choose_pitch(pic_grid *g)
{
    // h: the current tile's halo beyond the first two cells (one more for l_a = 2 1/2)
    const int h = g->halo + (g->order2 == 5 ? 1 : 0), T0 = g->tile[0], T1 = g->tile[1],
              T2 = g->dims == 3 ? g->tile[2] : 1;
    const int je0 = T0 + 2 * h + 4, je1 = T1 + 2 * h + 4;
    long long best_key = -1;
    for (int p0 = je0; p0 <= std::max(je0, 32); ++p0) {
        for (int p1 = je1; p1 <= (g->dims == 3 ? std::max(je1, 32) : je1); ++p1) {
            int cnt[32] = {0};
            for (int k = 0; k < T2; ++k)
                for (int j = 0; j < T1; ++j)
                    for (int i = 0; i < T0; ++i) {
                        const int base = (i + h + 2) + p0 * ((j + h + 2) + (g->dims == 3 ? p1 * (k + h + 2) : 0));
                        ++cnt[base & 31];
                    }
            int mn = cnt[0], mx = cnt[0];
            for (int b = 1; b < 32; ++b) {
                mn = std::min(mn, cnt[b]);
                mx = std::max(mx, cnt[b]);
            }
            const long long smem =
                (long long)particles_smem_bytes(g->dims, g->prec, 0, T0, T1, T2, g->halo, p0, p1, g->order2);
            const long long two = smem <= 113 * 1024 ? 0 : 1;
            const long long key = ((long long)(mx - mn) << 40) | (two << 39) | smem;
            if (best_key < 0 || key < best_key) {
                best_key = key;
                g->pitch[0] = p0;
                g->pitch[1] = p1;
            }
        }
    }
}

// Validates one run descriptor.  The first run of a batch fixes the settings
// every run shares (dims, precision, tile, halo, sort interval, block size,
// stream); later runs must agree on dims and precision.
int check_run(const pic_grid_desc *d, pic_grid *g, RunDev &rd, bool first)
{
    if (!d) return fail(PIC_ERR_INVALID_ARG, "null descriptor");
    if (d->dims != 2 && d->dims != 3) return fail(PIC_ERR_INVALID_ARG, "dims must be 2 or 3 (got %d)", d->dims);
    if (d->nx <= 0 || d->ny <= 0 || d->nz <= 0) return fail(PIC_ERR_INVALID_ARG, "cell counts must be positive");
    if (d->dims == 2 && d->nz != 1) return fail(PIC_ERR_INVALID_ARG, "nz must be 1 for a 2D grid");
    if (d->precision != PIC_FP64 && d->precision != PIC_FP32) return fail(PIC_ERR_INVALID_ARG, "bad precision");
    if (d->order2 != 3 && d->order2 != 4 && d->order2 != 5 && d->order2 != 0)
        return fail(PIC_ERR_INVALID_ARG, "order2 must be 3 (l_a = 1 1/2), 5 (l_a = 2 1/2) or 4 (Eq. wrong1)");
    const int order2 = d->order2 == 0 ? 3 : d->order2;
    if (!first && (d->dims != g->dims || d->precision != g->prec || order2 != g->order2))
        return fail(PIC_ERR_INVALID_ARG, "all runs of a batch need the same dims, precision and order");
    const double dd[3] = {d->dx, d->dy, d->dims == 3 ? d->dz : 1.0};
    for (int a = 0; a < 3; ++a)
        if (!(dd[a] > 0.0) || !std::isfinite(dd[a])) return fail(PIC_ERR_INVALID_ARG, "cell sizes must be positive");
    if (!(d->dt > 0.0) || !(d->c > 0.0) || !std::isfinite(d->dt) || !std::isfinite(d->c))
        return fail(PIC_ERR_INVALID_ARG, "dt and c must be positive");
    double s = 0.0;
    for (int a = 0; a < d->dims; ++a) {
        const double cN = d->c * d->dt / dd[a];
        if (cN >= 1.0) return fail(PIC_ERR_CFL, "Courant number c*dt/d = %g >= 1 on axis %d", cN, a);
        s += 1.0 / (dd[a] * dd[a]);
    }
    if (d->c * d->dt * std::sqrt(s) >= 1.0) return fail(PIC_ERR_CFL, "Yee stability limit c*dt*sqrt(sum 1/d^2) >= 1");
    if (first) {
        g->dims = d->dims;
        g->prec = d->precision;
        g->order2 = order2;
        // the FP64 particle adjoint is bound by the FP64 pipe; per-block tile
        // staging costs it more than the global reads it saves
        g->adj_tiled = g->prec == PIC_FP32 ? 1 : 0;
        g->halo = d->halo < 0 ? 1 : d->halo;
        if (g->halo > 2) return fail(PIC_ERR_INVALID_ARG, "halo must be 0..2");
        g->sort_interval = d->sort_interval > 0 ? d->sort_interval : 10;
        g->ppi = d->particles_per_block > 0 ? d->particles_per_block : 8192;
        if (g->ppi > 8192) return fail(PIC_ERR_INVALID_ARG, "particles_per_block must be <= 8192");
        if (g->ppi % 32 != 0) return fail(PIC_ERR_INVALID_ARG, "particles_per_block must be a multiple of 32");
        if (d->sort_order != PIC_SORT_AUTO && d->sort_order != PIC_SORT_BANKED && d->sort_order != PIC_SORT_STABLE &&
            d->sort_order != PIC_SORT_CELL_LANES)
            return fail(PIC_ERR_INVALID_ARG,
                        "sort_order must be PIC_SORT_AUTO, PIC_SORT_STABLE, PIC_SORT_BANKED or PIC_SORT_CELL_LANES");
        g->sort_order = d->sort_order;
        for (int a = 0; a < 3; ++a) g->tile[a] = d->tile[a] > 0 ? d->tile[a] : (d->dims == 3 ? 8 : 16);
        if (d->dims == 2) g->tile[2] = 1;
    }
    const int n[3] = {d->nx, d->ny, d->nz};
    int t[3];
    for (int a = 0; a < 3; ++a) t[a] = std::min(g->tile[a], n[a]);
    if (first)
        for (int a = 0; a < 3; ++a) g->tile[a] = t[a];
    const int staged = 2 * (g->halo + (g->order2 == 5 ? 3 : 2));   // the current tile's halo, both sides
    for (int a = 0; a < d->dims; ++a) {
        if (n[a] < t[a] + staged)
            return fail(PIC_ERR_INVALID_ARG,
                        "axis %d has %d cells; the tile (%d) plus its staged halo (%d) must fit in the grid", a, n[a],
                        t[a], staged);
    }
    if (first) {
        choose_pitch(g);
        if (g->sort_order == PIC_SORT_AUTO) g->sort_order = PIC_SORT_BANKED;
        if (g->sort_order == PIC_SORT_CELL_LANES && g->tile[0] * g->tile[1] * g->tile[2] > 128)
            return fail(PIC_ERR_INVALID_ARG, "the cell-lane order needs tiles of at most 128 cells (tile %dx%dx%d)",
                        g->tile[0], g->tile[1], g->tile[2]);
    }
    memset(&rd, 0, sizeof(rd));
    rd.pitch[0] = g->pitch[0];
    rd.pitch[1] = g->pitch[1];
    for (int a = 0; a < 3; ++a) {
        rd.n[a] = n[a];
        rd.tile[a] = t[a];
        rd.ntile[a] = (n[a] + t[a] - 1) / t[a];
        rd.d[a] = dd[a];
        rd.cN[a] = d->c * d->dt / dd[a];
    }
    if (d->dims == 2) rd.cN[2] = 0.0;
    rd.dt = d->dt;
    rd.c = d->c;
    rd.V = d->dims == 3 ? dd[0] * dd[1] * dd[2] : dd[0] * dd[1];
    rd.rho_bg = d->rho_bg;
    rd.cell_base = 0;
    rd.fpdt = 4.0 * 3.14159265358979323846 * rd.dt;
    rd.fpdtf = (float)rd.fpdt;
    rd.div_nx = make_divu31(n[0]);
    rd.div_ny = make_divu31(n[1]);
    for (int a = 0; a < 3; ++a) rd.div_t[a] = make_divu31(t[a]);
    rd.cf = (float)rd.c;
    for (int a = 0; a < 3; ++a) rd.cNf[a] = (float)rd.cN[a];
    return PIC_OK;
}

void destroy_grid(pic_grid *g)
{
    if (!g) return;
    cudaStreamSynchronize(g->stream);   // work still in flight may use the buffers freed below
    for (int c = 0; c < 3; ++c) {
        dfree(g->E[c]);
        dfree(g->B[c]);
        dfree(g->J[c]);
        dfree(g->old_off[c]);
    }
    dfree(g->old_cell);
    dfree(g->d_runs);
    dfree(g->d_groups);
    dfree(g->d_group_base);
    free_pool(g->pool);
    free_pool(g->pool_alt);
    free_sort(g);
    dfree(g->n_items);
    dfree(g->diag.rho);
    dfree(g->diag.resid_ref);
    dfree(g->diag.partials);
    dfree(g->diag.result);
    dfree(g->d_err);
    dfree(g->stage);
    dfree(g->d_run_cell_base);
    dfree(g->d_ant_n);
    if (g->h_drift) cudaFreeHost(g->h_drift);
    if (g->h_hdr) cudaFreeHost(g->h_hdr);
    for (auto &ev : g->ad_ev)
        if (ev) cudaEventDestroy(ev);
    for (int c = 0; c < 3; ++c) {
        dfree(g->adj_B1[c]);
        dfree(g->d_A[c]);
        if (c == 0) dfree(g->d_gm);
        dfree(g->adj_lamJ[c]);
    }
    dfree(g->adj_lam);
    graph_drop(g);
    prof_clear(g);
    for (auto e : g->prof_free) cudaEventDestroy(e);
    delete g;
}

}  // namespace

namespace pic {
// Sets the message returned by pic_last_error (for entry points in other files).
void set_last_error(const char *msg) { snprintf(t_err, sizeof(t_err), "%s", msg); }
}  // namespace pic

extern "C" {

const char *pic_last_error(void) { return t_err; }

int pic_inject_alloc_failure(long long after)
{
    g_alloc_fail_in.store(after < 0 ? -1 : after);
    return PIC_OK;
}

int pic_create_batch(const pic_grid_desc *descs, int nruns, pic_grid **out)
{
    if (!out) return fail(PIC_ERR_INVALID_ARG, "null output pointer");
    *out = nullptr;
    if (!descs) return fail(PIC_ERR_INVALID_ARG, "null descriptor");
    if (nruns <= 0 || nruns > 65535) return fail(PIC_ERR_INVALID_ARG, "run count must be 1..65535");
    pic_grid *g = new (std::nothrow) pic_grid();
    if (!g) return fail(PIC_ERR_OOM, "host allocation failed");
    std::vector<long long> base(nruns + 1, 0);
    for (int r = 0; r < nruns; ++r) {
        RunDev rd;
        int rc = check_run(&descs[r], g, rd, r == 0);
        if (rc != PIC_OK) {
            delete g;
            return rc;
        }
        rd.cell_base = base[r];
        base[r + 1] = base[r] + (long long)rd.n[0] * rd.n[1] * rd.n[2];
        HostRun hr;
        hr.dev = rd;
        hr.dims = g->dims;
        g->runs.push_back(hr);
    }
    g->stream = (cudaStream_t)descs[0].cuda_stream;
    g->total_cells = base[nruns];
    g->have_ref.assign(nruns, 0);
    auto bail = [&](cudaError_t e, const char *what) {
        int r = cuda_fail(e, what);
        destroy_grid(g);
        return r;
    };
    cudaError_t e;
    for (int c = 0; c < 3; ++c) {
        if ((e = dalloc_bytes(&g->E[c], g->total_cells * elem(g))) != cudaSuccess) return bail(e, "E");
        if ((e = dalloc_bytes(&g->B[c], g->total_cells * elem(g))) != cudaSuccess) return bail(e, "B");
        if ((e = dalloc_bytes(&g->J[c], g->total_cells * elem(g))) != cudaSuccess) return bail(e, "J");
        if ((e = cudaMemsetAsync(g->E[c], 0, g->total_cells * elem(g), g->stream)) != cudaSuccess) return bail(e, "E");
        if ((e = cudaMemsetAsync(g->B[c], 0, g->total_cells * elem(g), g->stream)) != cudaSuccess) return bail(e, "B");
        if ((e = cudaMemsetAsync(g->J[c], 0, g->total_cells * elem(g), g->stream)) != cudaSuccess) return bail(e, "J");
    }
    std::vector<RunDev> rds;
    for (auto &r : g->runs) rds.push_back(r.dev);
    if ((e = dalloc(&g->d_runs, rds.size())) != cudaSuccess) return bail(e, "runs");
    if ((e = cudaMemcpy(g->d_runs, rds.data(), sizeof(RunDev) * rds.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
        return bail(e, "runs");
    if ((e = dalloc(&g->d_run_cell_base, base.size())) != cudaSuccess) return bail(e, "run bases");
    if ((e = cudaMemcpy(g->d_run_cell_base, base.data(), sizeof(long long) * base.size(), cudaMemcpyHostToDevice)) !=
        cudaSuccess)
        return bail(e, "run bases");
    if ((e = dalloc(&g->d_ant_n, g->runs.size())) != cudaSuccess) return bail(e, "antenna clocks");
    if ((e = cudaMemset(g->d_ant_n, 0, sizeof(long long) * g->runs.size())) != cudaSuccess)
        return bail(e, "antenna clocks");
    if ((e = dalloc(&g->d_err, 2)) != cudaSuccess) return bail(e, "error word");
    if ((e = cudaMemset(g->d_err, 0, 2 * sizeof(int))) != cudaSuccess) return bail(e, "error word");
    if ((e = cudaHostAlloc((void **)&g->h_drift, sizeof(unsigned), cudaHostAllocDefault)) != cudaSuccess)
        return bail(e, "drift count");
    if ((e = dalloc(&g->n_items, 1)) != cudaSuccess) return bail(e, "item count");
    if ((e = cudaMemset(g->n_items, 0, sizeof(int))) != cudaSuccess) return bail(e, "item count");
    if ((e = dalloc(&g->diag.rho, g->total_cells)) != cudaSuccess) return bail(e, "rho");
    if ((e = dalloc(&g->diag.resid_ref, g->total_cells)) != cudaSuccess) return bail(e, "residual reference");
    if ((e = dalloc(&g->diag.partials, (size_t)2 * kDiagBlocks * 8)) != cudaSuccess) return bail(e, "partials");
    if ((e = dalloc(&g->diag.result, (size_t)kDiagResults)) != cudaSuccess) return bail(e, "diag result");
    // shared memory of the particle kernels
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    for (int mode = 0; mode < 3; ++mode) {
        const size_t b = particles_smem_bytes(g->dims, g->prec, mode, g->tile[0], g->tile[1], g->tile[2], g->halo,
                                              g->pitch[0], g->pitch[1], g->order2);
        if ((long long)b > optin) {
            destroy_grid(g);
            return fail(PIC_ERR_INVALID_ARG, "tile %dx%dx%d with halo %d needs %zu B of shared memory (> %d)",
                        descs[0].tile[0], descs[0].tile[1], descs[0].tile[2], descs[0].halo, b, optin);
        }
        if ((e = particles_set_smem_limit(g->dims, g->prec, mode, b, g->order2)) != cudaSuccess)
            return bail(e, "smem limit");
    }
    if (uses_cell_lanes(g) && (e = particles_cl_set_smem_limit()) != cudaSuccess) return bail(e, "smem limit");
    {
        // the tiled particle adjoint where its tiles fit in shared memory
        const size_t ab = adjoint_smem_bytes(g->dims, g->prec, g->tile, g->halo, g->pitch);
        g->adj_fits = (long long)ab <= optin && g->order2 == 3 ? 1 : 0;
        if (g->adj_fits && (e = adjoint_set_smem_limit(g->dims, g->prec, ab)) != cudaSuccess)
            return bail(e, "smem limit");
    }
    if (g->prec == PIC_FP32 &&
        (e = diag_set_smem_limit(g->dims, diag_items_smem_bytes(g->dims, g->tile, g->halo, g->pitch, g->order2),
                                 g->order2)) != cudaSuccess)
        return bail(e, "smem limit");
    if ((e = cudaStreamSynchronize(g->stream)) != cudaSuccess) return bail(e, "create");
    *out = g;
    return PIC_OK;
}

int pic_create_grid(const pic_grid_desc *desc, pic_grid **out)
{
    return pic_create_batch(desc, 1, out);
}

int pic_num_runs(pic_grid *g) { return g ? (int)g->runs.size() : 0; }

int pic_tile_layout(pic_grid *g, int out[6])
{
    if (!g || !out) return fail(PIC_ERR_INVALID_ARG, "null argument");
    out[0] = g->tile[0];
    out[1] = g->tile[1];
    out[2] = g->tile[2];
    out[3] = g->halo;
    out[4] = g->pitch[0];
    out[5] = g->pitch[1];
    return PIC_OK;
}

int pic_destroy(pic_grid *g)
{
    destroy_grid(g);
    return PIC_OK;
}

long long pic_kernel_launches(pic_grid *g) { return g ? g->launches : 0; }

static cudaMemcpyKind kind_in(int on_device) { return on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice; }
static cudaMemcpyKind kind_out(int on_device) { return on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost; }

static int check_run_index(pic_grid *g, int run)
{
    if (!g) return fail(PIC_ERR_INVALID_ARG, "null grid");
    if (run < 0 || run >= (int)g->runs.size()) return fail(PIC_ERR_INVALID_ARG, "run %d is not in the batch", run);
    return PIC_OK;
}

int pic_set_sort_policy(pic_grid *g, int adaptive)
{
    if (!g) return fail(PIC_ERR_INVALID_ARG, "null grid");
    g->adaptive_sort = adaptive ? 1 : 0;
    g->sort_due = false;
    g->ad_excess = 0.f;
    g->ad_sort = -1.f;
    g->ad_limit = 0;
    g->ad_clean = 0;
    g->ad_backoff = 2;
    g->ad_drifted = false;
    return PIC_OK;
}

int pic_set_antenna(pic_grid *g, int run, const pic_antenna_desc *a)
{
    int rc = check_run_index(g, run);
    if (rc != PIC_OK) return rc;
    RunDev &rd = g->runs[run].dev;
    const int was = rd.ant_pol != 0;
    if (a) {
        if (a->polarization != PIC_POL_Y && a->polarization != PIC_POL_Z)
            return fail(PIC_ERR_INVALID_ARG, "antenna polarization must be PIC_POL_Y or PIC_POL_Z");
        if (a->plane < 1 || a->plane >= rd.n[0])
            return fail(PIC_ERR_INVALID_ARG, "antenna plane %d outside 1..nx-1 (nx = %d)", a->plane, rd.n[0]);
        if (!std::isfinite(a->amplitude) || !std::isfinite(a->omega) || !std::isfinite(a->ramp) || a->ramp < 0.0 ||
            a->start < 0)
            return fail(PIC_ERR_INVALID_ARG, "antenna amplitude, frequency and ramp must be finite, ramp and start >= 0");
        rd.ant_pol = a->polarization;
        rd.ant_i0 = a->plane;
        rd.ant_E0 = a->amplitude;
        rd.ant_omega = a->omega;
        rd.ant_ramp = a->ramp;
    } else {
        rd.ant_pol = 0;
    }
    g->antennas += (rd.ant_pol != 0) - was;
    CK(cudaMemcpyAsync(g->d_runs + run, &rd, sizeof(RunDev), cudaMemcpyHostToDevice, g->stream), "antenna");
    const long long start = a ? a->start : 0;
    CK(cudaMemcpyAsync(g->d_ant_n + run, &start, sizeof(long long), cudaMemcpyHostToDevice, g->stream),
       "antenna clock");
    CK(cudaStreamSynchronize(g->stream), "antenna");
    if (!g->capturing) graph_drop(g);   // the graph's step has one launch more or less
    return PIC_OK;
}

static long long run_cells(const pic_grid *g, int run)
{
    const RunDev &r = g->runs[run].dev;
    return (long long)r.n[0] * r.n[1] * r.n[2];
}

int pic_set_fields_run(pic_grid *g, int run, const void *const E[3], const void *const B[3], int on_device)
{
    int rc = check_run_index(g, run);
    if (rc != PIC_OK) return rc;
    if (!E || !B) return fail(PIC_ERR_INVALID_ARG, "null argument");
    const size_t es = elem(g), bytes = run_cells(g, run) * es, off = g->runs[run].dev.cell_base * es;
    for (int c = 0; c < 3; ++c) {
        if (!E[c] || !B[c]) return fail(PIC_ERR_INVALID_ARG, "null field component");
        CK(cudaMemcpyAsync((char *)g->E[c] + off, E[c], bytes, kind_in(on_device), g->stream), "set E");
        CK(cudaMemcpyAsync((char *)g->B[c] + off, B[c], bytes, kind_in(on_device), g->stream), "set B");
    }
    if (!on_device) CK(cudaStreamSynchronize(g->stream), "set fields");
    g->have_ref[run] = 0;
    return PIC_OK;
}

int pic_set_fields(pic_grid *g, const void *const E[3], const void *const B[3], int on_device)
{
    return pic_set_fields_run(g, 0, E, B, on_device);
}

int pic_get_fields_run(pic_grid *g, int run, void *E[3], void *B[3], void *J[3], int on_device)
{
    int rc = check_run_index(g, run);
    if (rc != PIC_OK) return rc;
    const size_t es = elem(g), bytes = run_cells(g, run) * es, off = g->runs[run].dev.cell_base * es;
    for (int c = 0; c < 3; ++c) {
        if (E && E[c]) CK(cudaMemcpyAsync(E[c], (char *)g->E[c] + off, bytes, kind_out(on_device), g->stream), "get E");
        if (B && B[c]) CK(cudaMemcpyAsync(B[c], (char *)g->B[c] + off, bytes, kind_out(on_device), g->stream), "get B");
        if (J && J[c]) CK(cudaMemcpyAsync(J[c], (char *)g->J[c] + off, bytes, kind_out(on_device), g->stream), "get J");
    }
    if (!on_device) CK(cudaStreamSynchronize(g->stream), "get fields");
    return PIC_OK;
}

int pic_get_fields(pic_grid *g, void *E[3], void *B[3], void *J[3], int on_device)
{
    return pic_get_fields_run(g, 0, E, B, J, on_device);
}

// Frees every particle buffer and leaves the grid with its fields and no
// particles (the state of a new grid's particles).
static void drop_particles(pic_grid *g)
{
    cudaStreamSynchronize(g->stream);
    free_pool(g->pool);
    free_pool(g->pool_alt);
    free_sort(g);
    dfree(g->old_cell);
    g->old_cell = nullptr;
    for (int c = 0; c < 3; ++c) {
        dfree(g->old_off[c]);
        g->old_off[c] = nullptr;
    }
    g->groups.clear();
    g->total = 0;
    g->have_old = false;
    g->max_items = 0;
    cudaMemsetAsync(g->n_items, 0, sizeof(int), g->stream);
    upload_groups(g);
    graph_drop(g);
}

static bool group_before(int run_a, int sp_a, int run_b, int sp_b)
{
    return run_a < run_b || (run_a == run_b && sp_a < sp_b);
}

struct LoadReq {
    int run, species;
    pic_species_desc sp;
    long long n;
    const double *x[3];
    const double *w[3];
};

// Loads (replaces) several (run, species) groups with one pool re-layout and
// one sort.  Host arrays are staged in one device buffer first.
static int load_many(pic_grid *g, std::vector<LoadReq> &reqs, int on_device)
{
    for (auto &q : reqs) {
        int rc0 = check_run_index(g, q.run);
        if (rc0 != PIC_OK) return rc0;
        if (q.species < 0 || q.species >= kMaxSpecies)
            return fail(PIC_ERR_INVALID_ARG, "species must be 0..%d", kMaxSpecies - 1);
        if (q.n < 0 || q.n > 2000000000LL) return fail(PIC_ERR_INVALID_ARG, "particle count out of range");
        if (!(q.sp.m > 0.0) || !std::isfinite(q.sp.q) || !std::isfinite(q.sp.weight))
            return fail(PIC_ERR_INVALID_ARG, "species needs m > 0 and finite q, weight");
        if (q.n > 0)
            for (int a = 0; a < 3; ++a)
                if ((a < g->dims && !q.x[a]) || !q.w[a]) return fail(PIC_ERR_INVALID_ARG, "null particle component");
        for (auto &o : reqs)
            if (&o != &q && o.run == q.run && o.species == q.species)
                return fail(PIC_ERR_INVALID_ARG, "species %d of run %d appears twice", q.species, q.run);
    }
    CK(cudaStreamSynchronize(g->stream), "load: prior work");
    // device pointers of every request's x and w (staged if on the host)
    std::vector<std::array<const double *, 6>> src(reqs.size());
    long long need = 0;
    for (auto &q : reqs) need += 6 * q.n;
    if (!on_device && g->stage_n < need) {
        dfree(g->stage);
        g->stage = nullptr;
        g->stage_n = 0;
        CK(dalloc(&g->stage, (size_t)need), "load staging");
        g->stage_n = need;
    }
    long long so = 0;
    for (size_t r = 0; r < reqs.size(); ++r) {
        const LoadReq &q = reqs[r];
        for (int a = 0; a < 3; ++a) {
            src[r][a] = nullptr;
            src[r][3 + a] = nullptr;
        }
        if (q.n == 0) continue;
        for (int a = 0; a < 3; ++a) {
            if (on_device) {
                src[r][a] = a < g->dims ? q.x[a] : q.x[0];
                src[r][3 + a] = q.w[a];
            } else {
                if (a < g->dims)
                    CK(cudaMemcpyAsync(g->stage + so + a * q.n, q.x[a], sizeof(double) * q.n, cudaMemcpyHostToDevice,
                                       g->stream),
                       "stage x");
                CK(cudaMemcpyAsync(g->stage + so + (3 + a) * q.n, q.w[a], sizeof(double) * q.n,
                                   cudaMemcpyHostToDevice, g->stream),
                   "stage w");
                src[r][a] = g->stage + so + (a < g->dims ? a : 0) * q.n;
                src[r][3 + a] = g->stage + so + (3 + a) * q.n;
            }
        }
        so += 6 * q.n;
    }
    auto convert = [&](size_t r, const PoolBuf &P, long long base) -> cudaError_t {
        const LoadReq &q = reqs[r];
        if (q.n == 0) return cudaSuccess;
        const RunDev &rn = g->runs[q.run].dev;
        launch_count_add(g, 1);
        return launch_load(g->prec, g->stream, q.n, src[r][0], src[r][1], src[r][2], src[r][3], src[r][4], src[r][5],
                           g->dims, rn.n[0], rn.n[1], rn.n[2], P, base);
    };
    // every request matches a loaded group of the same size: convert in place
    bool in_place = true;
    std::vector<HostGroup *> match(reqs.size(), nullptr);
    for (size_t r = 0; r < reqs.size(); ++r) {
        for (auto &h : g->groups)
            if (h.run == reqs[r].run && h.species == reqs[r].species && h.n == reqs[r].n) match[r] = &h;
        if (!match[r]) in_place = false;
    }
    if (in_place) {
        for (size_t r = 0; r < reqs.size(); ++r) {
            match[r]->q = reqs[r].sp.q;
            match[r]->m = reqs[r].sp.m;
            match[r]->weight = reqs[r].sp.weight;
        }
        int rc = upload_groups(g);
        if (rc != PIC_OK) return rc;
        for (size_t r = 0; r < reqs.size(); ++r) CK(convert(r, g->pool, match[r]->base), "particle load");
        rc = do_sort(g);
        if (rc != PIC_OK) return rc;
        for (auto &q : reqs) g->have_ref[q.run] = 0;
        if (!on_device) CK(cudaStreamSynchronize(g->stream), "load");
        return PIC_OK;
    }
    // new layout: all (run, species) groups ordered by run then species
    std::vector<HostGroup> old = g->groups;
    std::vector<HostGroup> ng;
    for (auto &h : old) {
        bool replaced = false;
        for (auto &q : reqs)
            if (q.run == h.run && q.species == h.species) replaced = true;
        if (!replaced) ng.push_back(h);
    }
    for (auto &q : reqs) {
        HostGroup nh{};
        nh.run = q.run;
        nh.species = q.species;
        nh.q = q.sp.q;
        nh.m = q.sp.m;
        nh.weight = q.sp.weight;
        nh.n = q.n;
        nh.base = -1;   // marks a new group
        ng.push_back(nh);
    }
    std::stable_sort(ng.begin(), ng.end(), [](const HostGroup &x, const HostGroup &y) {
        return group_before(x.run, x.species, y.run, y.species);
    });
    long long total = 0;
    for (auto &h : ng) total += h.n;
    graph_drop(g);
    PoolBuf np, na;
    cudaError_t e = alloc_pool(g, np, total);
    if (e == cudaSuccess) e = alloc_pool(g, na, total);
    if (e != cudaSuccess) {
        free_pool(np);
        free_pool(na);
        return cuda_fail(e, "particle pool");
    }
    long long pb = 0;
    for (auto &h : ng) {
        if (e != cudaSuccess) break;
        if (h.base >= 0) {   // an old group keeps its data
            if (h.n > 0) {
                e = launch_copy_pool(g->prec, g->stream, g->pool, h.base, np, pb, h.n);
                launch_count_add(g, 1);
            }
        } else {
            for (size_t r = 0; r < reqs.size(); ++r)
                if (reqs[r].run == h.run && reqs[r].species == h.species) e = convert(r, np, pb);
        }
        h.base = pb;
        pb += h.n;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) {
        free_pool(np);
        free_pool(na);
        return cuda_fail(e, "particle load");
    }
    free_pool(g->pool);
    free_pool(g->pool_alt);
    g->pool = np;
    g->pool_alt = na;
    g->groups = ng;
    g->total = total;
    int rc = upload_groups(g);
    if (rc == PIC_OK) rc = size_particle_buffers(g, total);
    if (rc != PIC_OK) {
        // the new layout could not get its buffers: the grid keeps its fields
        // and no particles, and stays usable (a later load starts afresh)
        const std::string msg = pic_last_error();
        drop_particles(g);
        set_last_error((msg + "; the grid's particles were dropped").c_str());
        return rc;
    }
    rc = do_sort(g);
    if (rc != PIC_OK) return rc;
    for (auto &q : reqs) g->have_ref[q.run] = 0;
    CK(cudaStreamSynchronize(g->stream), "load: sort");
    return PIC_OK;
}

int pic_load_particles_run(pic_grid *g, int run, int species, const pic_species_desc *sp, long long n,
                           const double *const x[3], const double *const w[3], int on_device)
{
    if (!g || !sp) return fail(PIC_ERR_INVALID_ARG, "null argument");
    if (n > 0 && (!x || !w)) return fail(PIC_ERR_INVALID_ARG, "null particle arrays");
    std::vector<LoadReq> reqs(1);
    reqs[0].run = run;
    reqs[0].species = species;
    reqs[0].sp = *sp;
    reqs[0].n = n;
    for (int a = 0; a < 3; ++a) {
        reqs[0].x[a] = n > 0 ? x[a] : nullptr;
        reqs[0].w[a] = n > 0 ? w[a] : nullptr;
    }
    return load_many(g, reqs, on_device);
}

int pic_load_particles_runs(pic_grid *g, int count, const int *runs, int species, const pic_species_desc *sp,
                            const long long *n, const double *const *x, const double *const *w, int on_device)
{
    if (!g || !runs || !sp || !n || !x || !w) return fail(PIC_ERR_INVALID_ARG, "null argument");
    if (count <= 0) return fail(PIC_ERR_INVALID_ARG, "count must be positive");
    std::vector<LoadReq> reqs(count);
    for (int r = 0; r < count; ++r) {
        reqs[r].run = runs[r];
        reqs[r].species = species;
        reqs[r].sp = sp[r];
        reqs[r].n = n[r];
        for (int a = 0; a < 3; ++a) {
            reqs[r].x[a] = x[3 * r + a];
            reqs[r].w[a] = w[3 * r + a];
        }
    }
    return load_many(g, reqs, on_device);
}

int pic_load_particles(pic_grid *g, int species, const pic_species_desc *sp, long long n, const double *const x[3],
                       const double *const w[3], int on_device)
{
    return pic_load_particles_run(g, 0, species, sp, n, x, w, on_device);
}

long long pic_num_particles_run(pic_grid *g, int run, int species)
{
    if (!g) return 0;
    for (auto &h : g->groups)
        if (h.run == run && h.species == species) return h.n;
    return 0;
}

long long pic_num_particles(pic_grid *g, int species) { return pic_num_particles_run(g, 0, species); }

int pic_get_particles_run(pic_grid *g, int run, int species, int *cell, void *offset[3], void *w[3], int *id,
                          int on_device)
{
    int rc = check_run_index(g, run);
    if (rc != PIC_OK) return rc;
    const HostGroup *h = nullptr;
    for (auto &q : g->groups)
        if (q.run == run && q.species == species) h = &q;
    if (!h) return fail(PIC_ERR_INVALID_ARG, "species %d of run %d is not loaded", species, run);
    if (h->n == 0) return PIC_OK;
    const cudaMemcpyKind k = kind_out(on_device);
    const size_t es = elem(g);
    if (cell) CK(cudaMemcpyAsync(cell, g->pool.cell + h->base, sizeof(int) * h->n, k, g->stream), "get cells");
    if (id) CK(cudaMemcpyAsync(id, g->pool.id + h->base, sizeof(int) * h->n, k, g->stream), "get ids");
    for (int a = 0; a < 3; ++a) {
        if (offset && offset[a] && a < g->dims)
            CK(cudaMemcpyAsync(offset[a], (char *)g->pool.off[a] + h->base * es, es * h->n, k, g->stream), "get offsets");
        if (w && w[a]) CK(cudaMemcpyAsync(w[a], (char *)g->pool.w[a] + h->base * es, es * h->n, k, g->stream), "get momenta");
    }
    if (!on_device) CK(cudaStreamSynchronize(g->stream), "get particles");
    return PIC_OK;
}

int pic_get_particles(pic_grid *g, int species, int *cell, void *offset[3], void *w[3], int *id, int on_device)
{
    return pic_get_particles_run(g, 0, species, cell, offset, w, id, on_device);
}

int pic_gather_push(pic_grid *g)
{
    if (!g) return fail(PIC_ERR_INVALID_ARG, "null grid");
    if (g->total == 0) return PIC_OK;
    int rc = launch_part(g, 1);
    if (rc == PIC_OK) g->have_old = true;
    return rc;
}

int pic_deposit_current(pic_grid *g)
{
    if (!g) return fail(PIC_ERR_INVALID_ARG, "null grid");
    for (int c = 0; c < 3; ++c) CK(cudaMemsetAsync(g->J[c], 0, g->total_cells * elem(g), g->stream), "zero J");
    if (g->total == 0) return PIC_OK;
    if (!g->have_old) return fail(PIC_ERR_STATE, "pic_deposit_current needs a preceding pic_gather_push");
    return launch_part(g, 2);
}

int pic_yee_update(pic_grid *g, int which)
{
    if (!g) return fail(PIC_ERR_INVALID_ARG, "null grid");
    if (which != PIC_B_HALF && which != PIC_E_FULL) return fail(PIC_ERR_INVALID_ARG, "which must be PIC_B_HALF or PIC_E_FULL");
    return launch_fields(g, which, 0);
}

int pic_sort(pic_grid *g)
{
    if (!g) return fail(PIC_ERR_INVALID_ARG, "null grid");
    return do_sort(g);
}

int pic_step(pic_grid *g, int nsteps)
{
    if (!g) return fail(PIC_ERR_INVALID_ARG, "null grid");
    if (nsteps < 0) return fail(PIC_ERR_INVALID_ARG, "negative step count");
    const bool measure = g->adaptive_sort && g->total > 0;
    if (measure && !g->ad_ev[0])
        for (auto &ev : g->ad_ev) CK(cudaEventCreate(&ev), "sort policy events");
    for (int s = 0; s < nsteps; ++s) {
        int rc;
        bool timed_sort = false;
        const int limit = measure && g->ad_limit > 0 ? std::min(g->ad_limit, g->sort_interval) : g->sort_interval;
        if (measure && g->steps_since_sort >= limit && !g->sort_due && g->steps_since_sort > 0) {
            // a cycle that reached the learned interval without drift: after
            // ad_backoff of them, try one step longer
            if (!g->ad_drifted && ++g->ad_clean >= g->ad_backoff && limit < g->sort_interval) {
                g->ad_limit = limit + 1;
                g->ad_clean = 0;
            }
        }
        if (g->steps_since_sort >= limit || g->sort_due) {
            if (measure) CK(cudaEventRecord(g->ad_ev[2], g->stream), "sort policy events");
            // the arrays move inside this step's particle launch, unless the sort
            // policy times the sort or another kernel (cell lanes, l_a = 2 1/2,
            // Eq. wrong1) takes the step
            const bool defer = !measure && g->order2 == 3 && !uses_cell_lanes(g) && g->total > 0;
            if ((rc = do_sort(g, defer)) != PIC_OK) return rc;
            if (measure) CK(cudaEventRecord(g->ad_ev[3], g->stream), "sort policy events");
            timed_sort = measure;
        }
        const bool sorted = g->steps_since_sort == 0;
        g->sort_due = false;
        if (measure) CK(cudaMemsetAsync(g->d_err + 1, 0, sizeof(int), g->stream), "drift count");
        if ((rc = launch_fields(g, PIC_B_HALF, 1)) != PIC_OK) {
            settle(g);
            return rc;
        }
        if (measure) CK(cudaEventRecord(g->ad_ev[0], g->stream), "sort policy events");
        if (g->total > 0 && (rc = launch_part(g, 0)) != PIC_OK) return rc;
        if (measure) CK(cudaEventRecord(g->ad_ev[1], g->stream), "sort policy events");
        if ((rc = launch_fields(g, PIC_B_HALF, 0)) != PIC_OK) return rc;
        if ((rc = launch_fields(g, PIC_E_FULL, 0)) != PIC_OK) return rc;
        g->steps_since_sort += 1;
        g->have_old = false;
        if (measure) {
            // Particles past their tile's halo take the global-memory path; the
            // slowdown they cause since the last sort is summed, and the next
            // step sorts once it exceeds what a sort costs.
            CK(cudaMemcpyAsync(g->h_drift, g->d_err + 1, sizeof(unsigned), cudaMemcpyDeviceToHost, g->stream),
               "drift count");
            CK(cudaStreamSynchronize(g->stream), "sort policy");
            float tp = 0.f;
            CK(cudaEventElapsedTime(&tp, g->ad_ev[0], g->ad_ev[1]), "sort policy events");
            if (sorted) {
                if (timed_sort) CK(cudaEventElapsedTime(&g->ad_sort, g->ad_ev[2], g->ad_ev[3]), "sort policy events");
                g->ad_base = tp;
                g->ad_excess = 0.f;
                g->ad_drifted = false;
            }
            float last = 0.f;
            if (*g->h_drift > 0u) g->ad_drifted = true;
            if (!sorted && *g->h_drift > 0u) {
                last = std::max(0.f, tp - g->ad_base);
                g->ad_excess += last;
            }
            // the next step will cost at least as much extra as this one did
            const float cost = g->ad_sort > 0.f ? g->ad_sort : g->ad_base;
            g->sort_due = g->ad_excess + last > cost;
            if (g->sort_due) {
                // drift got costly after steps_since_sort steps: from now on sort
                // one step earlier; a failed attempt at a longer interval doubles
                // the clean cycles needed before the next attempt
                const int learned = std::max(1, g->steps_since_sort - 1);
                if (g->ad_limit > 0 && learned < g->ad_limit) g->ad_backoff = std::min(64, 2 * g->ad_backoff);
                g->ad_limit = learned;
                g->ad_clean = 0;
            }
        }
    }
    return PIC_OK;
}

// One step of every run in one cooperative launch (plus the sort launches
// every sort_interval steps).  As in pic_step, a sort leaves the arrays in
// place and the step's launch reads the particles through its permutation,
// writing them to the other buffer in the new order.
static int persistent_step(pic_grid *g)
{
    int rc;
    if (g->steps_since_sort >= g->sort_interval &&
        (rc = do_sort(g, g->order2 == 3 && !uses_cell_lanes(g) && g->total > 0)) != PIC_OK)
        return rc;
    ProfScope ps(g, PIC_PROF_PARTICLES);
    const unsigned *perm = g->pending_perm;
    cudaError_t e = launch_step_persistent(g->dims, g->prec, g->stream, g->items, g->n_items, g->d_runs, g->d_groups,
                                           perm ? g->pool_alt : g->pool, g->E, g->B, g->J, g->halo, g->tile[0],
                                           g->tile[1], g->tile[2], g->d_err, (int)g->runs.size(),
                                           g->d_run_cell_base, &g->persist_blocks, 1, g->pitch[0], g->pitch[1],
                                           g->d_ant_n, g->antennas, perm ? &g->pool : nullptr, perm);
    launch_count_add(g, 1);
    if (perm) {
        g->pending_perm = nullptr;
        std::swap(g->pool, g->pool_alt);
    }
    if (e != cudaSuccess) return cuda_fail(e, "persistent step");
    g->steps_since_sort += 1;
    g->have_old = false;
    return PIC_OK;
}

int pic_step_persistent(pic_grid *g, int nsteps)
{
    if (!g) return fail(PIC_ERR_INVALID_ARG, "null grid");
    if (nsteps < 0) return fail(PIC_ERR_INVALID_ARG, "negative step count");
    if (g->order2 != 3) return fail(PIC_ERR_INVALID_ARG, "the persistent batch step is built for l_a = 1 1/2");
    if (g->vecpot) return fail(PIC_ERR_INVALID_ARG, "the vector potential is advanced by pic_step and pic_yee_update");
    if (g->total == 0) return pic_step(g, nsteps);
    for (int s = 0; s < nsteps; ++s) {
        int rc = persistent_step(g);
        if (rc != PIC_OK) return rc;
    }
    return PIC_OK;
}

// Captures 2 * sort_interval persistent steps, starting with a sort, into a
// CUDA graph.  Two sorts bring the double-buffered pool back to the buffer it
// started in, so the graph can be replayed as often as needed.
static int capture_graph(pic_grid *g)
{
    graph_drop(g);
    if (g->persist_blocks <= 0) {
        cudaError_t ep = launch_step_persistent(g->dims, g->prec, g->stream, g->items, g->n_items, g->d_runs,
                                                g->d_groups, g->pool, g->E, g->B, g->J, g->halo, g->tile[0],
                                                g->tile[1], g->tile[2], g->d_err, (int)g->runs.size(),
                                                g->d_run_cell_base, &g->persist_blocks, 0, g->pitch[0], g->pitch[1],
                                                g->d_ant_n, g->antennas);
        if (ep != cudaSuccess) return cuda_fail(ep, "persistent kernel set-up");
    }
    const bool prof = g->profiling;
    g->profiling = false;
    g->capturing = true;
    const long long l0 = g->launches;
    cudaError_t e = cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeThreadLocal);
    int rc = PIC_OK;
    if (e == cudaSuccess) {
        for (int s = 0; s < 2 * g->sort_interval && rc == PIC_OK; ++s) rc = persistent_step(g);
        cudaGraph_t graph = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(g->stream, &graph);
        if (rc == PIC_OK && e2 == cudaSuccess) {
            e = cudaGraphInstantiate(&g->graph_exec, graph, 0);
            if (e == cudaSuccess) g->graph_valid = true;
        } else if (e2 != cudaSuccess) {
            e = e2;
        }
        if (graph) cudaGraphDestroy(graph);
    }
    g->graph_launches = g->launches - l0;
    g->launches = l0;
    g->profiling = prof;
    g->capturing = false;
    if (rc != PIC_OK) return rc;
    if (e != cudaSuccess) return cuda_fail(e, "graph capture");
    return PIC_OK;
}

int pic_step_graph(pic_grid *g, int nsteps)
{
    if (!g) return fail(PIC_ERR_INVALID_ARG, "null grid");
    if (nsteps < 0) return fail(PIC_ERR_INVALID_ARG, "negative step count");
    if (g->order2 != 3) return fail(PIC_ERR_INVALID_ARG, "the persistent batch step is built for l_a = 1 1/2");
    if (g->vecpot) return fail(PIC_ERR_INVALID_ARG, "the vector potential is advanced by pic_step and pic_yee_update");
    if (!g->stream) return fail(PIC_ERR_INVALID_ARG, "graph replay needs a non-default stream");
    if (g->total == 0) return pic_step(g, nsteps);
    const int span = 2 * g->sort_interval;
    while (nsteps > 0) {
        if (g->steps_since_sort >= g->sort_interval && nsteps >= span) {
            if (!g->graph_valid) {
                const long long since = g->steps_since_sort;
                int rc = capture_graph(g);
                if (rc != PIC_OK) return rc;
                if (g->steps_since_sort != since) return fail(PIC_ERR_STATE, "graph capture changed the sort phase");
            }
            ProfScope ps(g, PIC_PROF_PARTICLES);
            CK(cudaGraphLaunch(g->graph_exec, g->stream), "graph launch");
            g->launches += g->graph_launches;
            nsteps -= span;
            continue;
        }
        int rc = persistent_step(g);
        if (rc != PIC_OK) return rc;
        nsteps -= 1;
    }
    return PIC_OK;
}

int pic_profile(pic_grid *g, int enable)
{
    if (!g) return fail(PIC_ERR_INVALID_ARG, "null grid");
    if (enable) prof_clear(g);
    g->profiling = enable != 0;
    return PIC_OK;
}

int pic_profile_read(pic_grid *g, double ms[PIC_PROF_N], long long count[PIC_PROF_N])
{
    if (!g || !ms || !count) return fail(PIC_ERR_INVALID_ARG, "null argument");
    CK(cudaStreamSynchronize(g->stream), "profile sync");
    for (int c = 0; c < PIC_PROF_N; ++c) {
        ms[c] = 0.0;
        count[c] = 0;
    }
    for (auto &m : g->prof_marks) {
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, m.second.first, m.second.second), "event time");
        ms[m.first] += t;
        count[m.first] += 1;
    }
    return PIC_OK;
}

int pic_sync(pic_grid *g)
{
    if (!g) return fail(PIC_ERR_INVALID_ARG, "null grid");
    CK(cudaStreamSynchronize(g->stream), "sync");
    int err = 0;
    CK(cudaMemcpy(&err, g->d_err, sizeof(int), cudaMemcpyDeviceToHost), "error word");
    if (err & ERR_NONFINITE) return fail(PIC_ERR_NONFINITE, "a particle momentum became non-finite");
    return PIC_OK;
}

int pic_diagnostics_run(pic_grid *g, int run, pic_diag *out)
{
    int rc = check_run_index(g, run);
    if (rc != PIC_OK) return rc;
    if (!out) return fail(PIC_ERR_INVALID_ARG, "null argument");
    memset(out, 0, sizeof(*out));
    int nl = 0;
    const RunDev &rn = g->runs[run].dev;
    cudaError_t e = launch_diagnostics_run(g->dims, g->prec, g->stream, g->d_runs, run,
                                           (long long)rn.n[0] * rn.n[1] * rn.n[2], rn.cell_base, g->d_groups,
                                           g->d_group_base, (int)g->groups.size(), g->total, g->pool, g->E, g->B,
                                           g->diag, g->have_ref[run] ? 0 : 1, kDiagBlocks, kDiagBlocks, &nl,
                                           g->items, g->n_items, g->halo, g->tile, g->pitch, g->order2);
    launch_count_add(g, nl);
    if (e != cudaSuccess) return cuda_fail(e, "diagnostics");
    double r[kDiagResults];
    CK(cudaMemcpyAsync(r, g->diag.result, sizeof(r), cudaMemcpyDeviceToHost, g->stream), "diagnostics copy");
    int err = 0;
    CK(cudaMemcpyAsync(&err, g->d_err, sizeof(int), cudaMemcpyDeviceToHost, g->stream), "error word");
    CK(cudaStreamSynchronize(g->stream), "diagnostics");
    g->have_ref[run] = 1;
    out->kinetic = r[0];
    out->field_E = r[1];
    out->field_B = r[2];
    out->half_step_corr = r[3];
    out->total = r[4];
    out->momentum[0] = r[5];
    out->momentum[1] = r[6];
    out->momentum[2] = r[7];
    out->total_charge = r[8];
    out->gauss_resid_max = r[9];
    out->gauss_resid_rms = r[10];
    out->n_particles = (long long)llround(r[11]);
    out->error_word = err;
    if (err & ERR_NONFINITE) return fail(PIC_ERR_NONFINITE, "a particle momentum became non-finite");
    return PIC_OK;
}

int pic_diagnostics(pic_grid *g, pic_diag *out) { return pic_diagnostics_run(g, 0, out); }

// ---- vector potential ------------------------------------------------------------
int pic_set_vector_potential(pic_grid *g, const void *const A[3], int on_device, int set_B)
{
    if (!g) return fail(PIC_ERR_INVALID_ARG, "null grid");
    if (!A) {   // stop tracking
        for (int c = 0; c < 3; ++c) { dfree(g->d_A[c]); g->d_A[c] = nullptr; }
        g->vecpot = 0;
        return PIC_OK;
    }
    for (int c = 0; c < 3; ++c)
        if (!A[c]) return fail(PIC_ERR_INVALID_ARG, "null vector potential component");
    const size_t bytes = g->total_cells * elem(g);
    for (int c = 0; c < 3; ++c)
        if (!g->d_A[c]) CK(dalloc_bytes(&g->d_A[c], bytes), "vector potential");
    if (!g->d_gm) CK(dalloc(&g->d_gm, 3), "generalized momentum");
    for (int c = 0; c < 3; ++c) CK(cudaMemcpyAsync(g->d_A[c], A[c], bytes, kind_in(on_device), g->stream), "set A");
    g->vecpot = 1;
    if (set_B) {
        long long maxc = 0;
        for (auto &r : g->runs) maxc = std::max(maxc, (long long)r.dev.n[0] * r.dev.n[1] * r.dev.n[2]);
        CK(launch_curl_A(g->dims, g->prec, g->stream, g->d_runs, (int)g->runs.size(), maxc, g->d_A, g->B), "curl A");
        launch_count_add(g, 1);
    }
    if (!on_device) CK(cudaStreamSynchronize(g->stream), "set A");
    return PIC_OK;
}

int pic_get_vector_potential(pic_grid *g, void *A[3], int on_device)
{
    if (!g || !A) return fail(PIC_ERR_INVALID_ARG, "null argument");
    if (!g->vecpot) return fail(PIC_ERR_STATE, "no vector potential is tracked (pic_set_vector_potential)");
    const size_t bytes = g->total_cells * elem(g);
    for (int c = 0; c < 3; ++c)
        if (A[c]) CK(cudaMemcpyAsync(A[c], g->d_A[c], bytes, kind_out(on_device), g->stream), "get A");
    if (!on_device) CK(cudaStreamSynchronize(g->stream), "get A");
    return PIC_OK;
}

int pic_generalized_momentum_run(pic_grid *g, int run, double P[3])
{
    int rc = check_run_index(g, run);
    if (rc != PIC_OK) return rc;
    if (!P) return fail(PIC_ERR_INVALID_ARG, "null argument");
    if (!g->vecpot) return fail(PIC_ERR_STATE, "no vector potential is tracked (pic_set_vector_potential)");
    CK(launch_gen_momentum(g->dims, g->prec, g->order2, g->stream, run, g->total, g->d_group_base,
                           (int)g->groups.size(), g->d_groups, g->d_runs, g->pool, g->d_A, g->d_gm),
       "generalized momentum");
    launch_count_add(g, 1);
    CK(cudaMemcpyAsync(P, g->d_gm, 3 * sizeof(double), cudaMemcpyDeviceToHost, g->stream), "generalized momentum");
    CK(cudaStreamSynchronize(g->stream), "generalized momentum");
    return PIC_OK;
}

int pic_generalized_momentum(pic_grid *g, double P[3]) { return pic_generalized_momentum_run(g, 0, P); }

// ---- state snapshots -----------------------------------------------------------
struct StateHeader {
    char magic[4];            // "PICS"
    int version;              // 4
    int dims, prec, ngroups, steps_since_sort;
    long long total, total_cells;
    long long total_tiles;    // tile starts of the particle order follow the fields
    long long nruns;          // one antenna clock per run at the end
    int lanes;                // 1: the cell-lane tables of the particle order follow the antenna clocks
    unsigned checksum;        // FNV-1a of the bytes before this field
};
static_assert(sizeof(StateHeader) == 64, "snapshot header");

// Snapshot layout: the header, then each array at the next multiple of 16 bytes.
static long long seg16(long long b) { return (b + 15) & ~15LL; }

static unsigned fnv1a(const void *p, size_t n)
{
    const unsigned char *b = (const unsigned char *)p;
    unsigned h = 2166136261u;
    for (size_t i = 0; i < n; ++i) {
        h ^= b[i];
        h *= 16777619u;
    }
    return h;
}

static void fill_header(const pic_grid *g, StateHeader &h)
{
    memset(&h, 0, sizeof(h));
    memcpy(h.magic, "PICS", 4);
    h.version = 4;
    h.dims = g->dims;
    h.prec = g->prec;
    h.ngroups = (int)g->groups.size();
    h.steps_since_sort = g->steps_since_sort;
    h.total = g->total;
    h.total_cells = g->total_cells;
    h.total_tiles = g->total_tiles;
    h.nruns = (long long)g->runs.size();
    h.lanes = g->sort_order == PIC_SORT_CELL_LANES ? 1 : 0;
    h.checksum = fnv1a(&h, offsetof(StateHeader, checksum));
}

long long pic_state_bytes(pic_grid *g)
{
    if (!g) return 0;
    const long long es = (long long)elem(g);
    return (long long)sizeof(StateHeader) + 2 * seg16(4 * g->total) + (g->dims + 3) * seg16(es * g->total) +
           6 * seg16(es * g->total_cells) + seg16(8 * (g->total_tiles + 1)) + seg16(8 * (long long)g->runs.size()) +
           (g->sort_order == PIC_SORT_CELL_LANES ? seg16(128LL * g->total_tiles) + seg16(512LL * g->total_tiles) : 0);
}

// The (device array, bytes) list of a snapshot, in its order after the header.
constexpr int kStateSegs = 18;
static int state_segments(pic_grid *g, void *arr[kStateSegs], size_t bytes[kStateSegs])
{
    const size_t es = elem(g);
    int n = 0;
    auto seg = [&](void *p, size_t b) { arr[n] = p; bytes[n] = b; ++n; };
    seg(g->pool.cell, sizeof(int) * g->total);
    seg(g->pool.id, sizeof(int) * g->total);
    for (int a = 0; a < g->dims; ++a) seg(g->pool.off[a], es * g->total);
    for (int a = 0; a < 3; ++a) seg(g->pool.w[a], es * g->total);
    for (int a = 0; a < 3; ++a) seg(g->E[a], es * g->total_cells);
    for (int a = 0; a < 3; ++a) seg(g->B[a], es * g->total_cells);
    seg(g->tile_start, sizeof(long long) * (g->total_tiles + 1));
    seg(g->d_ant_n, sizeof(long long) * g->runs.size());
    if (g->sort_order == PIC_SORT_CELL_LANES) {
        seg(g->lane_cell, 128 * (size_t)g->total_tiles);
        seg(g->lane_count, 512 * (size_t)g->total_tiles);
    }
    return n;
}

// Enqueues a snapshot of the grid's state into dst on the grid's stream: one
// copy kernel for a device snapshot, one copy per array for a host one.
static int save_body(pic_grid *g, void *dst, int on_device)
{
    StateHeader h;
    fill_header(g, h);
    char *o = (char *)dst;
    Copier cp(g->stream, kind_out(on_device));
    if (on_device) cp.inline_bytes(o, &h, (int)sizeof(h));
    else memcpy(o, &h, sizeof(h));
    o += sizeof(h);
    void *arr[kStateSegs];
    size_t bytes[kStateSegs];
    const int n = state_segments(g, arr, bytes);
    for (int q = 0; q < n; ++q) {
        CK(cp.add(o, arr[q], bytes[q]), "state save");
        o += seg16((long long)bytes[q]);
    }
    CK(cp.flush(), "state save");
    launch_count_add(g, cp.launches);
    return PIC_OK;
}

static int check_header(const pic_grid *g, const StateHeader &h)
{
    if (memcmp(h.magic, "PICS", 4) != 0 || h.version != 4 || h.checksum != fnv1a(&h, offsetof(StateHeader, checksum)))
        return fail(PIC_ERR_INVALID_ARG, "not a libpic state snapshot (bad magic, version or header checksum)");
    if (h.dims != g->dims || h.prec != g->prec || h.total != g->total || h.total_cells != g->total_cells ||
        h.ngroups != (int)g->groups.size() || h.total_tiles != g->total_tiles || h.nruns != (long long)g->runs.size() ||
        h.lanes != (g->sort_order == PIC_SORT_CELL_LANES ? 1 : 0))
        return fail(PIC_ERR_INVALID_ARG, "state snapshot does not match this grid's layout");
    return PIC_OK;
}

// Enqueues the restore of a snapshot whose header h has been checked.
static int restore_body(pic_grid *g, const void *src, int on_device, const StateHeader &h)
{
    const char *o = (const char *)src + sizeof(h);
    Copier cp(g->stream, kind_in(on_device));
    void *arr[kStateSegs];
    size_t bytes[kStateSegs];
    const int n = state_segments(g, arr, bytes);
    for (int q = 0; q < n; ++q) {
        CK(cp.add(arr[q], o, bytes[q]), "state restore");
        o += seg16((long long)bytes[q]);
    }
    CK(cp.flush(), "state restore");
    launch_count_add(g, cp.launches);
    // the particles are in the order of the sort before the save: its tile
    // starts give the work items back, and the sort schedule continues
    if (g->total > 0 && !g->groups.empty()) {
        int nl = 0;
        cudaError_t e = build_items(g->stream, g->tile_start, g->total_tiles, g->ppi, g->d_groups,
                                    (int)g->groups.size(), g->sort, g->item_scan, g->items, g->n_items, &nl);
        launch_count_add(g, nl);
        if (e != cudaSuccess) return cuda_fail(e, "work items");
    }
    g->steps_since_sort = h.steps_since_sort;
    g->have_old = false;
    g->tiles_valid = g->total > 0 && !g->groups.empty();   // the saved segments describe the saved pool
    if (!g->capturing) graph_drop(g);
    for (auto &r : g->have_ref) r = 0;
    return PIC_OK;
}

int pic_state_save(pic_grid *g, void *dst, int on_device)
{
    if (!g || !dst) return fail(PIC_ERR_INVALID_ARG, "null argument");
    const int rc = save_body(g, dst, on_device);
    if (rc != PIC_OK) return rc;
    CK(cudaStreamSynchronize(g->stream), "state save");
    return PIC_OK;
}

// Reads and checks a snapshot's header, then enqueues the restore; waits for
// the copies only if wait is set.
static int state_restore(pic_grid *g, const void *src, int on_device, bool wait)
{
    if (!g || !src) return fail(PIC_ERR_INVALID_ARG, "null argument");
    StateHeader h;
    if (on_device) {
        // a device snapshot may still be in flight on the grid's stream
        CK(cudaMemcpyAsync(&h, src, sizeof(h), cudaMemcpyDeviceToHost, g->stream), "state header");
        CK(cudaStreamSynchronize(g->stream), "state header");
    } else {
        memcpy(&h, src, sizeof(h));
    }
    int rc = check_header(g, h);
    if (rc == PIC_OK) rc = restore_body(g, src, on_device, h);
    if (rc != PIC_OK) return rc;
    if (wait) CK(cudaStreamSynchronize(g->stream), "state restore");
    return PIC_OK;
}

int pic_state_restore(pic_grid *g, const void *src, int on_device)
{
    return state_restore(g, src, on_device, true);
}

int pic_state_restore_async(pic_grid *g, const void *src, int on_device)
{
    return state_restore(g, src, on_device, false);
}

int pic_step_saving(pic_grid *g, int nsteps, void *const *states)
{
    if (!g || (nsteps > 0 && !states)) return fail(PIC_ERR_INVALID_ARG, "null argument");
    if (nsteps < 0) return fail(PIC_ERR_INVALID_ARG, "negative step count");
    for (int s = 0; s < nsteps; ++s)
        if (!states[s]) return fail(PIC_ERR_INVALID_ARG, "null state buffer %d", s);
    for (int s = 0; s < nsteps; ++s) {
        int rc = save_body(g, states[s], 1);
        if (rc == PIC_OK) rc = pic_step(g, 1);
        if (rc != PIC_OK) return rc;
    }
    return PIC_OK;
}

// ---- adjoint ---------------------------------------------------------------------
static int adj_scratch(pic_grid *g)
{
    if (g->adj_B1[0] && g->adj_lam) return PIC_OK;
    for (int c = 0; c < 3; ++c) {
        if (!g->adj_B1[c]) CK(dalloc_bytes(&g->adj_B1[c], g->total_cells * elem(g)), "adjoint scratch");
        if (!g->adj_lamJ[c]) CK(dalloc_bytes(&g->adj_lamJ[c], g->total_cells * elem(g)), "adjoint scratch");
    }
    if (!g->adj_lam) {
        CK(dalloc(&g->adj_lam, 2), "adjoint scratch");
        CK(cudaMemsetAsync(g->adj_lam, 0, 2 * sizeof(unsigned), g->stream), "adjoint scratch");
        g->adj_lam_cur = 0;
    }
    return PIC_OK;
}

static long long max_run_cells(const pic_grid *g)
{
    long long m = 0;
    for (auto &r : g->runs) m = std::max(m, (long long)r.dev.n[0] * r.dev.n[1] * r.dev.n[2]);
    return m;
}

int pic_set_adjoint_tiled(pic_grid *g, int tiled)
{
    if (!g) return fail(PIC_ERR_INVALID_ARG, "null grid");
    g->adj_tiled = tiled ? 1 : 0;
    return PIC_OK;
}

int pic_adjoint_yee_half_B(pic_grid *g, void *const lamB[3], void *lamE[3])
{
    if (!g || !lamB || !lamE) return fail(PIC_ERR_INVALID_ARG, "null argument");
    CK(launch_adj_yee(g->dims, g->prec, 1, g->stream, g->d_runs, (int)g->runs.size(), max_run_cells(g), lamE, lamB,
                      nullptr),
       "adjoint B half step");
    launch_count_add(g, 1);
    return PIC_OK;
}

int pic_adjoint_step(pic_grid *g, void *lamE[3], void *lamB[3], void *lamx[3], void *lamw[3])
{
    if (!g || !lamE || !lamB || !lamx || !lamw) return fail(PIC_ERR_INVALID_ARG, "null argument");
    if (g->order2 != 3) return fail(PIC_ERR_INVALID_ARG, "the discrete adjoint is built for l_a = 1 1/2");
    for (int c = 0; c < 3; ++c)
        if (!lamE[c] || !lamB[c] || !lamw[c] || (c < g->dims && !lamx[c]))
            return fail(PIC_ERR_INVALID_ARG, "null adjoint component");
    int rc = adj_scratch(g);
    if (rc != PIC_OK) return rc;
    const size_t fb = g->total_cells * elem(g);
    const long long mc = max_run_cells(g);
    const int nr = (int)g->runs.size();
    // B^n = B^{n-1/2} - (1/2) C_B E^n into scratch (the state is not modified)
    Copier cp(g->stream, cudaMemcpyDeviceToDevice);
    for (int c = 0; c < 3; ++c) CK(cp.add(g->adj_B1[c], g->B[c], fb), "B1");
    CK(cp.flush(), "B1");
    CK(launch_yee(g->prec, PIC_B_HALF, 0, g->stream, g->d_runs, nr, mc, g->E, g->adj_B1, g->J, g->dims, g->d_ant_n),
       "B1");
    // (E step)^T, (second B half step)^T
    CK(launch_adj_yee(g->dims, g->prec, 2, g->stream, g->d_runs, nr, mc, lamE, lamB, g->adj_lamJ), "adjoint E step");
    CK(launch_adj_yee(g->dims, g->prec, 1, g->stream, g->d_runs, nr, mc, lamE, lamB, nullptr), "adjoint B half step");
    // particles^T: the transposed gather of B^n adds to lamB, which from here on
    // is the adjoint of B^n (the first B half step's output)
    AdjLaunch lc;
    lc.runs = g->d_runs;
    lc.groups = g->d_groups;
    lc.group_base = g->d_group_base;
    lc.ngroups = (int)g->groups.size();
    lc.total = g->total;
    lc.items = g->adj_tiled && g->adj_fits ? g->items : nullptr;
    lc.n_items = g->n_items;
    lc.max_items = g->max_items;
    lc.halo = g->halo;
    for (int a = 0; a < 3; ++a) lc.tile[a] = g->tile[a];
    lc.pitch[0] = g->pitch[0];
    lc.pitch[1] = g->pitch[1];
    // the FP32 tiled form's lagged scale: the launch reads the largest lambda
    // recorded by the previous one and records its own into the other word
    unsigned *cur = g->adj_lam + g->adj_lam_cur;
    lc.lam_prev = g->adj_lam + (1 - g->adj_lam_cur);
    lc.lam_cur = cur;
    CK(cudaMemsetAsync(cur, 0, sizeof(unsigned), g->stream), "adjoint scale");
    CK(launch_particles_adj(g->dims, g->prec, g->stream, lc, g->pool, g->E, g->adj_B1, g->adj_lamJ, lamE, lamB,
                            lamx, lamw),
       "adjoint particles");
    if (lc.items) g->adj_lam_cur = 1 - g->adj_lam_cur;
    // (first B half step)^T: lamB becomes the adjoint of B^{n-1/2}, unchanged
    CK(launch_adj_yee(g->dims, g->prec, 1, g->stream, g->d_runs, nr, mc, lamE, lamB, nullptr),
       "adjoint B half step");
    launch_count_add(g, 6);
    return PIC_OK;
}

int pic_adjoint_steps(pic_grid *g, void *const *states, int nstates, void *lamE[3], void *lamB[3], void *lamx[3],
                      void *lamw[3])
{
    if (!g || (nstates > 0 && !states)) return fail(PIC_ERR_INVALID_ARG, "null argument");
    if (nstates < 0) return fail(PIC_ERR_INVALID_ARG, "negative state count");
    if (g->order2 != 3) return fail(PIC_ERR_INVALID_ARG, "the discrete adjoint is built for l_a = 1 1/2");
    if (nstates == 0) return PIC_OK;
    for (int s = 0; s < nstates; ++s)
        if (!states[s]) return fail(PIC_ERR_INVALID_ARG, "null state buffer %d", s);
    // every header in one pass: the only host synchronization of the call
    if ((size_t)nstates > g->h_hdr_cap) {
        if (g->h_hdr) cudaFreeHost(g->h_hdr);
        g->h_hdr = nullptr;
        g->h_hdr_cap = 0;
        CK(cudaHostAlloc(&g->h_hdr, sizeof(StateHeader) * (size_t)nstates, cudaHostAllocDefault), "state headers");
        g->h_hdr_cap = (size_t)nstates;
    }
    StateHeader *hh = (StateHeader *)g->h_hdr;
    for (int s = 0; s < nstates; ++s)
        CK(cudaMemcpyAsync(&hh[s], states[s], sizeof(StateHeader), cudaMemcpyDeviceToHost, g->stream), "state header");
    CK(cudaStreamSynchronize(g->stream), "state headers");
    for (int s = 0; s < nstates; ++s) {
        const int rc = check_header(g, hh[s]);
        if (rc != PIC_OK) return rc;
    }
    for (int s = nstates - 1; s >= 0; --s) {
        int rc = restore_body(g, states[s], 1, hh[s]);
        if (rc == PIC_OK) rc = pic_adjoint_step(g, lamE, lamB, lamx, lamw);
        if (rc != PIC_OK) return rc;
    }
    return PIC_OK;
}

}  // extern "C"
