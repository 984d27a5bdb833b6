// pic_internal.h -- host-side state of a libpic grid and the kernel launchers
// each translation unit provides.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "pic_device.cuh"

struct pic_grid;

namespace pic {

constexpr int kMaxSpecies = 32;
constexpr int kThreads = 256;      // threads per block of the particle kernels

struct HostRun {
    RunDev dev;                    // copy of the device descriptor
    int dims;
};

struct HostGroup {
    int run, species;
    double q, m, weight;
    long long base, n;
    int tile_base, ntiles;
};

// Device buffers of a particle pool (one of two, swapped by the sort).
struct PoolBuf {
    int *cell = nullptr;
    void *off[3] = {nullptr, nullptr, nullptr};
    void *w[3] = {nullptr, nullptr, nullptr};
    int *id = nullptr;
};

// Launch helpers implemented in the .cu files.  All enqueue on `st` and return
// a cudaError_t from the launch.
cudaError_t launch_particles(int dims, int prec, int mode, cudaStream_t st, const WorkItem *items,
                             const int *n_items, int max_items, const RunDev *runs, const GroupDev *groups,
                             const PoolBuf &P, void *const E[3], void *const B[3], void *const J[3],
                             int *old_cell, void *const old_off[3], int halo, int max_tile_x,
                             int max_tile_y, int max_tile_z, int *err, int p0, int p1, int order2 = 3,
                             const PoolBuf *src = nullptr, const unsigned *perm = nullptr);
// With perm (mode 0, l_a = 1 1/2): the pool was just sorted but not yet
// permuted; particle p of the new order is read from src at perm[p] and
// written, stepped, to P.
// order2 = 3: l_a = 1 1/2; 5: l_a = 2 1/2 (tiles one cell wider on every side).
size_t particles_smem_bytes(int dims, int prec, int mode, int tx, int ty, int tz, int halo, int p0, int p1,
                            int order2 = 3);
// One cooperative launch per step over every run (see k_step_persistent);
// *grid_blocks = 0 asks for the occupancy-derived grid and returns it; launch = 0
// only prepares (attributes and grid size), which must happen outside a capture.
cudaError_t launch_step_persistent(int dims, int prec, cudaStream_t st, const WorkItem *items, const int *n_items,
                                   const RunDev *runs, const GroupDev *groups, const PoolBuf &P, void *const E[3],
                                   void *const B[3], void *const J[3], int halo, int tx, int ty, int tz, int *err,
                                   int nruns, const long long *run_cell_base, int *grid_blocks, int launch, int p0,
                                   int p1, long long *ant_n, int antennas, const PoolBuf *src = nullptr,
                                   const unsigned *perm = nullptr);
cudaError_t particles_set_smem_limit(int dims, int prec, int mode, size_t bytes, int order2 = 3);

cudaError_t launch_load(int prec, cudaStream_t st, long long n, const double *x0, const double *x1,
                        const double *x2, const double *w0, const double *w1, const double *w2,
                        int dims, int nx, int ny, int nz, const PoolBuf &P, long long base);

cudaError_t launch_yee(int prec, int which, int zero_j, cudaStream_t st, const RunDev *runs, int nruns,
                       long long max_cells, void *const E[3], void *const B[3], void *const J[3], int dims,
                       const long long *ant_n);
// Advances every run's antenna clock (E steps since its antenna was set) by one.
cudaError_t launch_antenna_tick(cudaStream_t st, long long *ant_n, int nruns);

cudaError_t launch_copy_pool(int prec, cudaStream_t st, const PoolBuf &src, long long src_base,
                             const PoolBuf &dst, long long dst_base, long long n);

// Sort: computes keys, sorts them stably, permutes the pool from `src` into
// `dst`, fills tile_start[0..total_tiles] and the work items.
struct SortScratch {
    unsigned *keys[2] = {nullptr, nullptr};
    unsigned *vals[2] = {nullptr, nullptr};
    unsigned *hist = nullptr;      // 256 * max_chunks
    unsigned *block_sums = nullptr;
    unsigned *tcnt[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};   // re-sort: per-tile counts (total_tiles + 1 each)
    unsigned *m_total = nullptr;                       // re-sort: number of movers, histogram length
    unsigned char *cls = nullptr;                      // re-sort: class of every particle (capacity)
    long long capacity = 0;
    long long hist_capacity = 0;
    long long sums_capacity = 0;
};

cudaError_t sort_and_build_items(int prec, int dims, cudaStream_t st, long long total, const PoolBuf &src,
                                 const PoolBuf &dst, const GroupDev *groups, const long long *group_base_dev,
                                 int ngroups, const RunDev *runs, int total_tiles, SortScratch &scr,
                                 long long *tile_start, unsigned *item_scan, WorkItem *items, int *n_items,
                                 int particles_per_item, int halo, int banked, int half, int *launches,
                                 unsigned char *lane_cell = nullptr, int *lane_count = nullptr, int resort = 0,
                                 const unsigned **perm_out = nullptr);
// With lane_cell and lane_count (total_tiles * 128 entries each) the order
// inside a tile is the cell-lane order (PIC_SORT_CELL_LANES) instead of the
// banked or stable one, and the two tables receive every tile's lane cells
// and counts.  With resort (banked or stable order only), tile_start on entry
// holds the segments of the previous sort of this same pool and group layout,
// and only the particles whose tile changed are sorted globally; the result is
// the same.  With perm_out (not for the cell-lane order) the particle arrays
// are not moved: *perm_out receives the permutation (dst[o] = src[perm[o]], in
// the sort scratch, valid until the next sort) for the caller to apply.
cudaError_t launch_permute(int prec, int dims, cudaStream_t st, long long total, const PoolBuf &src,
                           const PoolBuf &dst, const unsigned *perm);

// The FP32 fused step over the cell-lane order (pic_particles_cl.cu): 3D,
// l_a = 1 1/2, 8x4x4 tiles with halo 1; one block of 128
// threads per tile.  drift is pool-sized scratch.  ppb: the particles per block
// the groups' fixed-point scales were set for.
bool particles_cl_applies(int dims, int prec, int order2, const int tile[3], int halo);
size_t particles_cl_smem_bytes();
cudaError_t particles_cl_set_smem_limit();
cudaError_t launch_particles_cl(cudaStream_t st, int total_tiles, const long long *tile_start,
                                const unsigned char *lane_cell, const int *lane_count, int *drift,
                                const GroupDev *groups, int ngroups, const RunDev *runs, const PoolBuf &P,
                                void *const E[3], void *const B[3], void *const J[3], int ppb, int *err);
// Work items (ranges of at most particles_per_item particles of one tile) from
// the tile starts of the current particle order.
cudaError_t build_items(cudaStream_t st, const long long *tile_start, int total_tiles, int particles_per_item,
                        const GroupDev *groups, int ngroups, SortScratch &scr, unsigned *item_scan, WorkItem *items,
                        int *n_items, int *launches);

cudaError_t radix_sort_pairs(cudaStream_t st, long long n, int nbits, unsigned *const keys[2], unsigned *const vals[2],
                             unsigned *hist, unsigned *block_sums, int *cur_out);
cudaError_t launch_tile_start(cudaStream_t st, const unsigned *sorted_keys, long long n, int total_tiles,
                              long long *tile_start);

// Diagnostics: accumulates into out (13 doubles) on the device.
struct DiagScratch {
    double *rho = nullptr;
    double *resid_ref = nullptr;
    double *partials = nullptr;    // per block partial sums, 8 values per block
    double *result = nullptr;      // kDiagResults reduced values
};

cudaError_t launch_diagnostics_run(int dims, int prec, cudaStream_t st, const RunDev *runs, int run,
                                   long long run_cells, long long cell_base, const GroupDev *groups,
                                   const long long *group_base, int ngroups, long long total, const PoolBuf &P,
                                   void *const E[3], void *const B[3], DiagScratch &scr, int set_ref,
                                   int np_blocks, int nc_blocks, int *launches, const WorkItem *items,
                                   const int *n_items, int halo, const int tile[3], const int pitch[2],
                                   int order2 = 3);
size_t diag_items_smem_bytes(int dims, const int tile[3], int halo, const int pitch[2], int order2 = 3);
cudaError_t diag_set_smem_limit(int dims, size_t bytes, int order2 = 3);
constexpr int kDiagResults = 12;

void set_last_error(const char *msg);

// Adjoint kernels (pic_adjoint.cu).  which = 2: transpose of the E step
// (lamJ = -4 pi dt lamE, lamB += C_E^T lamE); which = 1: transpose of the B half
// step (lamE += (-(1/2) C_B)^T lamB).
cudaError_t launch_adj_yee(int dims, int prec, int which, cudaStream_t st, const RunDev *runs, int nruns,
                           long long max_cells, void *const lamE[3], void *const lamB[3], void *const lamJ[3]);
// Particle part of the adjoint.  With work items (items != nullptr) the tiled
// kernel runs over them (shared-memory tiles in the particle kernels' pitches);
// without, the untiled kernel runs over the pool in group order.
struct AdjLaunch {
    const RunDev *runs;
    const GroupDev *groups;
    const long long *group_base;
    int ngroups;
    long long total;
    const WorkItem *items;
    const int *n_items;
    int max_items;
    int halo;
    int tile[3];
    int pitch[2];
    const unsigned *lam_prev = nullptr;   // FP32 tiled form: previous launch's largest |lambda| (float bits)
    unsigned *lam_cur = nullptr;          // this launch's
};
cudaError_t launch_particles_adj(int dims, int prec, cudaStream_t st, const AdjLaunch &lc, const PoolBuf &P,
                                 void *const E[3], void *const B1[3], void *const lamJ[3], void *const lamE[3],
                                 void *const lamB1[3], void *const lamx[3], void *const lamw[3]);
size_t adjoint_smem_bytes(int dims, int prec, const int tile[3], int halo, const int pitch[2]);

// Vector-potential formulation (pic_vecpot.cu): A -= c dt E (Eq. dadt), B = curl_h A
// (Eq. viaA), and the generalized momentum of one run's particles into out[3].
cudaError_t launch_update_A(int prec, cudaStream_t st, const RunDev *runs, int nruns, long long max_cells,
                            void *const A[3], void *const E[3]);
cudaError_t launch_curl_A(int dims, int prec, cudaStream_t st, const RunDev *runs, int nruns, long long max_cells,
                          void *const A[3], void *const B[3]);
cudaError_t launch_gen_momentum(int dims, int prec, int order2, cudaStream_t st, int run, long long total,
                                const long long *gbase, int ngroups, const GroupDev *groups, const RunDev *runs,
                                const PoolBuf &P, void *const A[3], double *out);
cudaError_t adjoint_set_smem_limit(int dims, int prec, size_t bytes);

}  // namespace pic

struct pic_grid {
    int dims = 3, prec = 0;
    int halo = 1, sort_interval = 10, ppi = 8192, sort_order = 0;   // sort_order: the resolved PIC_SORT_*
    int tile[3] = {8, 8, 8};
    int pitch[2] = {0, 0};   // x, y pitch of the shared tiles (chosen at create)
    cudaStream_t stream = nullptr;

    std::vector<pic::HostRun> runs;
    pic::RunDev *d_runs = nullptr;
    long long total_cells = 0;

    // fields, concatenated over runs
    void *E[3] = {nullptr, nullptr, nullptr};
    void *B[3] = {nullptr, nullptr, nullptr};
    void *J[3] = {nullptr, nullptr, nullptr};

    // species / groups
    std::vector<pic::HostGroup> groups;
    pic::GroupDev *d_groups = nullptr;
    long long *d_group_base = nullptr;
    int total_tiles = 0;

    // particle pool (double-buffered by the sort)
    pic::PoolBuf pool, pool_alt;
    long long total = 0, capacity = 0;

    // saved x^n for the unfused deposit
    int *old_cell = nullptr;
    void *old_off[3] = {nullptr, nullptr, nullptr};
    bool have_old = false;

    // sort products
    pic::SortScratch sort;
    unsigned char *lane_cell = nullptr;   // cell-lane order: per tile and lane, the lane's cell ...
    int *lane_count = nullptr;            // ... and its particle count (total_tiles * 128 each)
    int *drift = nullptr;                 // cell-lane kernel: drift lists, pool-sized
    long long *tile_start = nullptr;
    bool tiles_valid = false;       // tile_start holds the segments of the last sort of the current pool
    const unsigned *pending_perm = nullptr;   // sorted, not yet permuted: pool holds the old order (pic_step only)
    unsigned *item_scan = nullptr;
    pic::WorkItem *items = nullptr;
    long long *d_ant_n = nullptr;   // antenna clock per run (device)
    unsigned *h_drift = nullptr;    // pinned host copy of the drift count (d_err[1])
    void *h_hdr = nullptr;          // pinned host copies of snapshot headers (pic_adjoint_steps)
    size_t h_hdr_cap = 0;
    int order2 = 3;                 // twice the alternating order: 3 (l_a = 1 1/2) or 5 (l_a = 2 1/2)
    int adj_fits = 1;               // the tiled adjoint's shared memory fits the device
    int adj_tiled = 1;              // adjoint particle kernel over work items with shared-memory tiles (FP32 default)
    int adaptive_sort = 0;          // sort when the particle kernel's accumulated slowdown exceeds a sort
    bool sort_due = false;
    cudaEvent_t ad_ev[4] = {nullptr, nullptr, nullptr, nullptr};   // particle kernel, sort
    float ad_base = 0.f, ad_excess = 0.f, ad_sort = -1.f;          // ms
    int ad_limit = 0, ad_clean = 0, ad_backoff = 2;                // learned interval (steps)
    bool ad_drifted = false;                                       // drift seen since the last sort
    int antennas = 0;               // number of runs with an antenna
    int *n_items = nullptr;
    int max_items = 0;
    int steps_since_sort = 0;

    // diagnostics (residual reference per run)
    pic::DiagScratch diag;
    std::vector<char> have_ref;

    // batches: first cell of every run, nruns + 1 entries on the device
    long long *d_run_cell_base = nullptr;

    // one-launch-per-step persistent kernel and its CUDA graph (2 sort intervals of steps)
    int persist_blocks = 0;
    cudaGraphExec_t graph_exec = nullptr;
    bool graph_valid = false;
    bool capturing = false;
    long long graph_launches = 0;

    int *d_err = nullptr;
    long long launches = 0;

    // launch-group timing (pic_profile)
    bool profiling = false;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> prof_marks;
    std::vector<cudaEvent_t> prof_free;

    // vector potential A at the E points (pic_set_vector_potential), advanced with the E step
    void *d_A[3] = {nullptr, nullptr, nullptr};
    int vecpot = 0;
    double *d_gm = nullptr;          // generalized momentum result (3 doubles)
    // adjoint scratch: B^n, lamJ (field-sized, allocated on first use)
    void *adj_B1[3] = {nullptr, nullptr, nullptr};
    void *adj_lamJ[3] = {nullptr, nullptr, nullptr};
    unsigned *adj_lam = nullptr;     // two words: largest |lambda| of the last tiled adjoint launches (FP32)
    int adj_lam_cur = 0;             // which of them the next launch records into

    // staging for host-pointer particle loads (grown, never shrunk)
    double *stage = nullptr;
    long long stage_n = 0;
};
