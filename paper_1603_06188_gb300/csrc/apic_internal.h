// apic_internal.h -- declarations shared by the library's translation units (host side),
// and the launch helper of the step's kernel chain.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <utility>

#define APIC_BLOCK_EDGE 4
#define APIC_ERRBIT_RANGE 1u     // a particle's stencil left the grid (clamped)
#define APIC_ERRBIT_TIMEOUT 2u   // a bounded mbarrier wait ran out
#define APIC_ERRBIT_CAPACITY 4u  // tile list overflow
#define APIC_ERRBIT_NONFINITE 8u // a non-finite value in uploaded state
#define APIC_DEFAULT_WAIT_LIMIT (1u << 22)

// particle state lanes per copy: A V Ba Bb Fa Fb Fc Ta Tb M (layout in apic_device.cuh)
#define APIC_STATE_LANES 10

namespace apic {

// Type-erased description of one simulation's device buffers, handed to the launchers.
struct Buffers {
    // particle state: two copies (ping-pong), 7 arrays each, element size per precision
    void* st[2][APIC_STATE_LANES];
    uint32_t* knext;             // keys of the current particle order (input of the sort)
    uint32_t* kA; uint32_t* kB;  // radix ping-pong keys
    uint32_t* vA; uint32_t* vB;  // radix ping-pong values (particle indices)
    uint32_t* radix_counts;      // 256 * radix tiles
    // incremental sort: moved keys / indices (radix ping-pong), moved indices in index order,
    // per-chunk moved offsets, control words + digit counts, epoch-stamped look-back words
    uint32_t* mk[2]; uint32_t* mv[2];
    uint32_t* midx;
    uint32_t* choff;
    uint32_t* mcnt;              // moved count per chunk
    uint32_t* mbits;             // moved flags of the incremental sort, 1 bit per key
    uint32_t* mctl;              // [1] moved count, [2..5] pass tile counters
    uint32_t* mhist;             // [kMhistCopies][4][256] digit counts of the moved keys (follows mctl)
    unsigned long long* lbs;     // 256 * (radix tiles + 1)
    uint32_t* scan_part;         // partial sums of the device scan
    uint32_t* tiles;             // tile start offsets (+ end sentinel)
    uint32_t* chunk_cnt;         // per-chunk tile counts (scanned in place)
    uint32_t* ntiles;            // device counter: number of tiles
    uint32_t* tile_ctr;          // work counters: [0] P2G, [1] G2P (zeroed with each tile list), [2] sort tiles
    void* acc;                   // accumulation grid (4 lanes per node)
    void* vel;                   // velocity grid (4 lanes per node)
    void* acc2;                  // FLIP only: PIC momentum without the force (4 lanes per node)
    void* vdel;                  // FLIP only: the grid change (v~ - v, m) (4 lanes per node)
    void* vel1;                  // lambda = 1 / midpoint: the grid velocity before the update (v, m)
    void* sdv; void* su; void* sr; void* sp; void* ss; void* sdu;   // midpoint solve vectors (4 lanes per node)
    uint32_t* flags;             // active node blocks
    double* mom_part;            // per-CTA momentum partials
    double* mom_out;             // 6 doubles
    double* amom_part;           // the same two for apic_momentum_async, which runs on a
    double* amom_out;            // stream of its own
    uint32_t* err;               // latched error bits
    uint32_t* fallbacks;         // FP64 polar fallbacks
    void* dt_word;               // the current time step (one real) of adaptive stepping
    uint32_t* smax_word;         // max over particles of the Sec. 4.3 speed, FP32 bits (G2P)
    double* elapsed;             // simulated time of an adaptive run
    double* staging;             // FP64 staging for upload / download
    size_t staging_doubles;
};

struct HostCfg {
    int dim, order, precision, transfer;
    int res[3];
    int nb[3];
    double dx, origin[3], dt, gravity[3];
    int boundary, wall, model;
    int mat;                     // 1: per-particle parameters (lane M: mu, lam, m_p, V_p), else the config's
    int adaptive;                // 1: kernels read the time step from Buffers::dt_word
    double flip_alpha;           // transfer 2: weight of the FLIP update
    double mu, lam, mass, vol;
    int tile;                    // particles per tile (power of two)
    int p2g_kernel;              // 1: component-split (3-D), 2: cell-parallel
    int p2g_group;               // lanes per base cell of the cell-parallel P2G (2 or 4)
    int p2g_group_auto;          // 1: p2g_group follows the density after each upload
    int key_bits;
    int nblocks;
    int64_t capacity;
    unsigned wait_limit;         // polls of G2P's first bounded wait (APIC_DEFAULT_WAIT_LIMIT)
    int integrator;              // 0: lambda = 0 (symplectic Euler), 1: explicit lambda = 1, 2: implicit midpoint
    int newton_max, cg_max;      // midpoint: iteration caps
    double solve_tol;            // midpoint: Newton and CG tolerance
};

// per-simulation view of the sort buffers, for the batched sort (apic_sort.cu)
struct SortDesc {
    const uint32_t* knext;
    uint32_t* kb[2];
    uint32_t* vb[2];
    uint32_t n;       // particles
    uint32_t ntl;     // radix tiles
    uint32_t pbase;   // particles of the simulations before this one
    uint32_t rbase;   // radix tiles of the simulations before this one
    uint32_t cbase;   // tile-list chunks of the simulations before this one
    uint32_t nch;     // tile-list chunks
    // the member's incremental-sort buffers (Buffers of the same names)
    uint32_t* mk[2];
    uint32_t* mv[2];
    uint32_t* midx;
    uint32_t* choff;
    uint32_t* mcnt;
    uint32_t* mctl;   // + 16: digit counts
    unsigned long long* lbs;
};

// sort / tiles (apic_sort.cu)
int radix_tiles(int64_t n);
// words of the incremental sort's moved-key bitmap for n keys
size_t moved_bitmap_words(int64_t n);
// kernels launched by radix_sort, resort, build_tiles, and by batch_resort plus
// batch_build_tiles together (for the launch counters)
int radix_sort_kernels(int key_bits);
int resort_kernels(int64_t n, int key_bits);
int build_tiles_kernels(int64_t n, int tile);
int batch_sort_and_tiles_kernels(int passes);
size_t scan_partials_needed(int64_t n);
// sorts knext (values = identity) into (*keys_out, *vals_out); returns the CUDA error
// copies of the incremental sort's digit histogram (chunk t adds to copy t % kMhistCopies;
// batched members use copy 0 only)
constexpr int kMhistCopies = 16;
constexpr size_t kMsortCtlBytes = 64 + (size_t)kMhistCopies * 4 * 256 * 4;   // mctl words + mhist
// Incremental stable sort of knext given the previous sorted keys pk, valid when the
// particles are stored in that previous order; writes keys / permutation to kout / vout.
cudaError_t resort(const Buffers& b, int64_t n, int key_bits, const uint32_t* pk, uint32_t* kout, uint32_t* vout,
                   uint32_t* epoch, int sms, cudaStream_t s);
cudaError_t radix_sort(const Buffers& b, int64_t n, int key_bits, cudaStream_t s,
                       uint32_t** keys_out, uint32_t** vals_out);
cudaError_t build_tiles(const Buffers& b, const uint32_t* skeys, int64_t n, int dim, int tile,
                        int64_t max_tiles, cudaStream_t s);
cudaError_t exclusive_scan(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* part,
                           uint32_t* total, cudaStream_t s);
// incremental stable sort of every member's knext into kb[kpar] / vb[kpar]; members with
// bsorted[s] = 0 are sorted in full; bctl = [epoch, pass tile counters x4] on the device
cudaError_t batch_resort(const SortDesc* sd, const uint32_t* rt_sim, uint32_t total_rtiles, int nsims, int passes,
                         int kpar, const uint32_t* bsorted, uint32_t* bctl, uint32_t* err, int sms, cudaStream_t s);
cudaError_t batch_build_tiles(const SortDesc* sd, const uint32_t* ch_sim, uint32_t total_chunks, int dim, int tile,
                              int kpar, uint32_t* cnt, uint32_t* part, uint32_t* ntiles, int64_t max_tiles,
                              uint32_t* tile_sim, uint32_t* tile_start, uint32_t* err, uint32_t* tile_ctr,
                              cudaStream_t s);

// transfer kernels (apic_transfer_f32.cu / apic_transfer_f64.cu): one set per real type
struct Launch {
    int sms;          // multiprocessors
    int p2g_grid;     // persistent grid sizes
    int g2p_grid;
    int mom_parts;    // CTAs of the momentum reduction
    int p2g_cells;    // 1 if the cell-parallel P2G kernel serves this (dim, order)
};

#define APIC_DECLARE_PRECISION(SFX)                                                                          \
    cudaError_t keys_##SFX(const HostCfg& c, const Buffers& b, int cur, int64_t n, cudaStream_t s);           \
    cudaError_t p2g_##SFX(const HostCfg& c, const Buffers& b, int cur, const uint32_t* skeys,                 \
                          const uint32_t* perm, int64_t n, const Launch& L, cudaStream_t s);                   \
    cudaError_t grid_update_##SFX(const HostCfg& c, const Buffers& b, const Launch& L, cudaStream_t s);       \
    cudaError_t g2p_##SFX(const HostCfg& c, const Buffers& b, int cur, const uint32_t* skeys,                 \
                          const uint32_t* perm, int64_t n, const Launch& L, cudaStream_t s);                   \
    cudaError_t upload_##SFX(const HostCfg& c, const Buffers& b, int cur, int64_t n, const double* x,         \
                             const double* v, const double* B, const double* F, cudaStream_t s, int64_t k0,   \
                             int64_t k1);                                                                      \
    cudaError_t inverse_ids_##SFX(const HostCfg& c, const Buffers& b, int cur, int64_t n, uint32_t* inv,       \
                                  cudaStream_t s);                                                             \
    cudaError_t download_ids_##SFX(const HostCfg& c, const Buffers& b, int cur, int64_t n, const uint32_t* inv,\
                                   int64_t id0, int64_t id1, double* x, double* v, double* B, double* F,       \
                                   cudaStream_t s);                                                            \
    cudaError_t download_##SFX(const HostCfg& c, const Buffers& b, int cur, int64_t n, double* x, double* v,  \
                               double* B, double* F, int32_t* cell, double* off, cudaStream_t s);              \
    cudaError_t momentum_##SFX(const HostCfg& c, const Buffers& b, int cur, int64_t n, int where,             \
                               int grid_phase, const Launch& L, cudaStream_t s);                               \
    cudaError_t grid_dense_##SFX(const HostCfg& c, const Buffers& b, int which, double* m, double* mv,        \
                                 cudaStream_t s);                                                               \
    cudaError_t occupancy_##SFX(const HostCfg& c, int* p2g_per_sm, int* g2p_per_sm);                         \
    cudaError_t cfl_##SFX(const HostCfg& c, const Buffers& b, int cur, int64_t n, const Launch& L, cudaStream_t s); \
    cudaError_t set_params_##SFX(const HostCfg& c, const Buffers& b, int cur, int64_t n, const double* E,        \
                                 const double* nu, const double* mass, const double* vol, int keep,             \
                                 cudaStream_t s);                                                                 \
    cudaError_t adapt_dt_##SFX(const HostCfg& c, const Buffers& b, double nu, double dt_max, int first,         \
                               cudaStream_t s);                                                                 \
    cudaError_t grid_update_lambda1_##SFX(const HostCfg& c, const Buffers& b, int cur, const uint32_t* skeys,   \
                                          const uint32_t* perm, int64_t n, const Launch& L, cudaStream_t s);    \
    cudaError_t g2p_lambda1_##SFX(const HostCfg& c, const Buffers& b, int cur, const uint32_t* perm, int64_t n,  \
                                  const Launch& L, cudaStream_t s);                                              \
    cudaError_t grid_update_midpoint_##SFX(const HostCfg& c, const Buffers& b, int cur, const uint32_t* skeys,  \
                                           const uint32_t* perm, int64_t n, const Launch& L, cudaStream_t s,     \
                                           double* stats, int64_t* kernels);

#define APIC_DECLARE_BATCH(SFX)                                                                              \
    size_t batch_desc_bytes_##SFX();                                                                          \
    void batch_make_desc_##SFX(const HostCfg& c, const Buffers& b, int cur, int64_t n, void* out);            \
    cudaError_t batch_setup_##SFX(int dim, int order, int group, int* p2g_per_sm, int* g2p_per_sm);           \
    cudaError_t batch_p2g_##SFX(int dim, int order, int group, void* descs, const uint32_t* tile_sim,         \
                                const uint32_t* tile_start, const uint32_t* ntiles, uint32_t* ctr, int kpar,  \
                                int grid, cudaStream_t s);                                                     \
    cudaError_t batch_grid_##SFX(int dim, void* descs, const uint32_t* bbase, int nsims, uint32_t total_blocks, \
                                 int grid, cudaStream_t s);                                                    \
    cudaError_t batch_g2p_##SFX(int dim, int order, int ext, void* descs, const uint32_t* tile_sim,           \
                                const uint32_t* tile_start, const uint32_t* ntiles, uint32_t* ctr, int kpar,  \
                                int grid, cudaStream_t s);                                                     \
    cudaError_t batch_finish_##SFX(void* descs, int nsims, uint32_t* bsorted, cudaStream_t s);                                   \
    int batch_desc_cur_offset_##SFX();

APIC_DECLARE_PRECISION(f32)
APIC_DECLARE_PRECISION(f64)
APIC_DECLARE_BATCH(f32)
APIC_DECLARE_BATCH(f64)

// Programmatic dependent launch for the kernels of a step, which run back to back on one
// stream (sort passes, tile list, P2G, grid update, G2P): such a kernel is launched while the
// one before it drains, so its launch and the ramp of its CTAs overlap the previous kernel's
// tail.  Every kernel launched this way calls pdl_wait() before its first access to global
// memory: it returns once the previous kernel has completed and its writes are visible (so
// each kernel also completes after all earlier ones, and stream order holds for every
// buffer).  pdl_trigger() lets the next kernel launch once every CTA of this one is running.
// Without the launch attribute both are no-ops.
#ifdef __CUDACC__
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... P, typename... A>
inline cudaError_t launch_pdl(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, A&&... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<A>(args)...);
}
#endif

}  // namespace apic
