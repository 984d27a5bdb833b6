// pic_noalloc.cu -- pic_tile_sort_perm_noalloc: the stable tile sort of
// pic_sort, as a permutation, for callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc: code that runs inside a memory budget
// owned by another runtime (a framework's caching allocator, a simulation
// coupler that pre-reserves the whole GPU), or code on a path where an
// allocation would synchronize the device.  For them this entry point keeps
// its scratch in one file-scope device array of fixed size instead of asking
// for memory.  Every GPU that loads libpic holds that array until the process
// exits.
#include <cstdio>
#include <mutex>

#include "../../include/pic.h"
#include "pic_internal.h"

namespace {

constexpr long long kMaxN = PIC_NOALLOC_MAX_PARTICLES;
constexpr long long kChunkKeys = 4096;                                  // keys per radix chunk
constexpr long long kMaxChunks = (kMaxN + kChunkKeys - 1) / kChunkKeys;
constexpr long long kHistWords = 256 * kMaxChunks;
constexpr long long kSumWords = (kHistWords + 2047) / 2048 + 1;
// layout, in 32-bit words: keys[0], keys[1], vals[0], vals[1], hist, block sums
constexpr long long kScratchWords = 4 * kMaxN + kHistWords + kSumWords;

// The scratch.  In host code this name is only a stand-in for the device
// array: its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned g_sort_scratch[kScratchWords];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned *g_scratch_ptr[kMaxDevices] = {};

int fail(int code, const char *m)
{
    pic::set_last_error(m);
    return code;
}

// Device address of the scratch on the current device, looked up once per device.
cudaError_t scratch_address(unsigned **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_sort_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = static_cast<unsigned *>(p);
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

__global__ void k_tile_keys(long long n, const int *cell, int nx, int ny, int tx, int ty, int tz, int ntx, int nty,
                            unsigned *keys, unsigned *vals)
{
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int c = cell[p];
    const int i = c % nx, r = c / nx, j = r % ny, k = r / ny;
    keys[p] = (unsigned)(((k / tz) * nty + j / ty) * ntx + i / tx);
    vals[p] = (unsigned)p;
}

__global__ void k_check_cells(long long n, const int *cell, long long ncells, int *bad)
{
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p < n && (cell[p] < 0 || cell[p] >= ncells)) atomicOr(bad, 1);
}

__global__ void k_copy_perm(long long n, const unsigned *vals, int *perm)
{
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p < n) perm[p] = (int)vals[p];
}

}  // namespace

extern "C" int pic_tile_sort_perm_noalloc(const int *cell, long long n, int dims, const int ncell[3],
                                          const int tile[3], int *perm, long long *tile_start, void *cuda_stream)
{
    if (!ncell || !tile) return fail(PIC_ERR_INVALID_ARG, "null size arrays");
    if (dims != 2 && dims != 3) return fail(PIC_ERR_INVALID_ARG, "dims must be 2 or 3");
    if (n < 0 || n > kMaxN) {
        char m[160];
        snprintf(m, sizeof(m), "n = %lld is outside 0..%lld, the fixed scratch of the no-allocation sort", n, kMaxN);
        return fail(PIC_ERR_INVALID_ARG, m);
    }
    if (n > 0 && (!cell || !perm)) return fail(PIC_ERR_INVALID_ARG, "null cell or perm pointer");
    int nn[3], tt[3], nt[3];
    for (int a = 0; a < 3; ++a) {
        nn[a] = (a == 2 && dims == 2) ? 1 : ncell[a];
        tt[a] = (a == 2 && dims == 2) ? 1 : tile[a];
        if (nn[a] <= 0 || tt[a] <= 0) return fail(PIC_ERR_INVALID_ARG, "cell counts and tiles must be positive");
        nt[a] = (nn[a] + tt[a] - 1) / tt[a];
    }
    const long long ntiles = (long long)nt[0] * nt[1] * nt[2];
    if (ntiles > (1LL << 24)) return fail(PIC_ERR_INVALID_ARG, "more than 2^24 tiles");
    cudaStream_t st = (cudaStream_t)cuda_stream;

    unsigned *s = nullptr;
    cudaError_t e = scratch_address(&s);
    if (e != cudaSuccess) return fail(PIC_ERR_CUDA, "cudaGetSymbolAddress of the sort scratch failed");
    if (n == 0) {
        if (tile_start && cudaMemsetAsync(tile_start, 0, sizeof(long long) * (ntiles + 1), st) != cudaSuccess)
            return fail(PIC_ERR_CUDA, "clearing tile_start failed");
        return PIC_OK;
    }
    unsigned *keys[2] = {s, s + kMaxN};
    unsigned *vals[2] = {s + 2 * kMaxN, s + 3 * kMaxN};
    unsigned *hist = s + 4 * kMaxN;
    unsigned *sums = hist + kHistWords;
    // the last word of the scratch doubles as the invalid-cell flag (cleared here)
    int *bad = reinterpret_cast<int *>(sums + kSumWords - 1);
    const int nthr = 256;
    const unsigned nb = (unsigned)((n + nthr - 1) / nthr);
    if (cudaMemsetAsync(bad, 0, sizeof(int), st) != cudaSuccess) return fail(PIC_ERR_CUDA, "flag clear failed");
    k_check_cells<<<nb, nthr, 0, st>>>(n, cell, (long long)nn[0] * nn[1] * nn[2], bad);
    int hbad = 0;
    if (cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return fail(PIC_ERR_CUDA, "cell check failed");
    if (hbad) return fail(PIC_ERR_INVALID_ARG, "a cell index is outside the grid");
    k_tile_keys<<<nb, nthr, 0, st>>>(n, cell, nn[0], nn[1], tt[0], tt[1], tt[2], nt[0], nt[1], keys[0], vals[0]);
    if (cudaGetLastError() != cudaSuccess) return fail(PIC_ERR_CUDA, "key kernel launch failed");
    int nbits = 1;
    while ((1LL << nbits) < ntiles) ++nbits;
    int cur = 0;
    if (pic::radix_sort_pairs(st, n, nbits, keys, vals, hist, sums, &cur) != cudaSuccess)
        return fail(PIC_ERR_CUDA, "radix sort launch failed");
    k_copy_perm<<<nb, nthr, 0, st>>>(n, vals[cur], perm);
    if (cudaGetLastError() != cudaSuccess) return fail(PIC_ERR_CUDA, "permutation copy failed");
    if (tile_start && pic::launch_tile_start(st, keys[cur], n, (int)ntiles, tile_start) != cudaSuccess)
        return fail(PIC_ERR_CUDA, "tile start launch failed");
    return PIC_OK;
}
