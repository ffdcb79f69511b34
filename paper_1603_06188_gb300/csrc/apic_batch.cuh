// apic_batch.cuh -- batched form of the step: many independent simulations (same dim,
// B-spline order and precision; their own grids, sizes and material constants) advanced
// together, one persistent launch per phase.  Work items carry their simulation's index;
// each CTA loads that simulation's descriptor (constants and buffer pointers) and runs the
// same per-tile code as a single simulation.  Included after apic_transfer.cuh.
#pragma once

#include <stddef.h>

#include "apic_transfer.cuh"

namespace apic {

template <typename R> struct SimDesc {
    DevCfg<R> c;
    PState<R> st[2];        // the two copies of the particle state
    uint32_t* knext;        // keys of the current order (sort input)
    uint32_t* kb[2];        // radix ping-pong keys
    uint32_t* vb[2];        // radix ping-pong indices
    R* acc;
    R* vel;
    uint32_t* flags;
    uint32_t* err;
    uint32_t* fallbacks;
    int cur;                // copy holding the particles; flipped on the device after each step
    int pad_;
};

template <typename R> SimDesc<R> make_desc(const HostCfg& h, const Buffers& b, int cur, int64_t n)
{
    SimDesc<R> d;
    d.c = HostToDev<R>::make(h, n);
    d.st[0] = state_of<R>(b, 0);
    d.st[1] = state_of<R>(b, 1);
    d.knext = b.knext;
    d.kb[0] = b.kA;
    d.kb[1] = b.kB;
    d.vb[0] = b.vA;
    d.vb[1] = b.vB;
    d.acc = (R*)b.acc;
    d.vel = (R*)b.vel;
    d.flags = b.flags;
    d.err = b.err;
    d.fallbacks = b.fallbacks;
    d.cur = cur;
    d.pad_ = 0;
    return d;
}

// copy a descriptor into shared memory with the whole CTA (caller synchronises)
template <typename R> __device__ __forceinline__ void load_desc(SimDesc<R>* dst, const SimDesc<R>* src, int nthreads)
{
    static_assert(sizeof(SimDesc<R>) % 4 == 0, "descriptor is copied as 32-bit words");
    const uint32_t* s = reinterpret_cast<const uint32_t*>(src);
    uint32_t* d = reinterpret_cast<uint32_t*>(dst);
    for (int i = threadIdx.x; i < (int)(sizeof(SimDesc<R>) / 4); i += nthreads) d[i] = s[i];
}

// end of a simulation's tile: the next tile of the same simulation starts it, else its n
__device__ __forceinline__ uint32_t tile_end(const uint32_t* tile_sim, const uint32_t* tile_start, int t, int ntiles,
                                             uint32_t sim, uint32_t n)
{
    return (t + 1 < ntiles && tile_sim[t + 1] == sim) ? tile_start[t + 1] : n;
}

template <int D, int ORDER, typename R, int G>
__global__ void __launch_bounds__(128, (cells_ctas_per_sm<D, ORDER>())) kb_p2g_cells(SimDesc<R>* __restrict__ descs,
                                                       const uint32_t* __restrict__ tile_sim,
                                                       const uint32_t* __restrict__ tile_start,
                                                       const uint32_t* __restrict__ ntiles_p,
                                                       uint32_t* __restrict__ tile_ctr, int kpar)
{
    constexpr int NC = (D == 3) ? 64 : 16;
    extern __shared__ __align__(32) unsigned char p2g_smem[];
    R* cellsum = reinterpret_cast<R*>(p2g_smem);
    R* pslots = reinterpret_cast<R*>(p2g_smem + (p2g_cellsum_bytes<D, ORDER, R>() + 31) / 32 * 32);
    __shared__ uint32_t cbeg[NC], cend[NC];
    __shared__ int s_tile, s_cell;
    __shared__ __align__(16) SimDesc<R> sd;
    const int ntiles = (int)*ntiles_p;
    for (;;) {
        if (threadIdx.x == 0) {
            s_tile = (int)atomicAdd(tile_ctr, 1u);
            s_cell = 0;
        }
        for (int i = threadIdx.x; i < NC; i += 128) { cbeg[i] = 0u; cend[i] = 0u; }
        __syncthreads();
        const int t = s_tile;
        if (t >= ntiles) break;
        const uint32_t sim = tile_sim[t];
        load_desc<R>(&sd, descs + sim, 128);
        __syncthreads();
        const uint32_t start = tile_start[t];
        const uint32_t end = tile_end(tile_sim, tile_start, t, ntiles, sim, (uint32_t)sd.c.n);
        p2g_cells_tile<D, ORDER, R, G>(sd.st[sd.cur], sd.vb[kpar], sd.kb[kpar] + start, start, end, sd.acc, sd.flags, sd.c,
                                       sd.err, sd.fallbacks, cellsum, cbeg, cend, &s_cell, pslots);
    }
}

// the component-split P2G of k_p2g_split over the batch's tiles (3-D)
template <int ORDER, typename R>
__global__ void __launch_bounds__(SplitShape<ORDER>::NT, (split_ctas_per_sm<ORDER, R>()))
    kb_p2g_split(SimDesc<R>* __restrict__ descs, const uint32_t* __restrict__ tile_sim,
                 const uint32_t* __restrict__ tile_start, const uint32_t* __restrict__ ntiles_p,
                 uint32_t* __restrict__ tile_ctr, int kpar)
{
    constexpr int NT = SplitShape<ORDER>::NT;
    extern __shared__ __align__(32) unsigned char p2g_smem[];
    R* cellsum = reinterpret_cast<R*>(p2g_smem);
    R* pslots = reinterpret_cast<R*>(p2g_smem + (p2g_cellsum_bytes<3, ORDER, R>() + 31) / 32 * 32);
    __shared__ uint32_t cbeg[64], cend[64];
    __shared__ int s_tile;
    __shared__ __align__(16) SimDesc<R> sd;
    const int ntiles = (int)*ntiles_p;
    int next = 0;
    if (threadIdx.x == 0) next = (int)atomicAdd(tile_ctr, 1u);
    for (;;) {
        if (threadIdx.x == 0) s_tile = next;
        if (threadIdx.x < 64) { cbeg[threadIdx.x] = 0u; cend[threadIdx.x] = 0u; }
        __syncthreads();
        const int t = s_tile;
        if (t >= ntiles) break;
        if (threadIdx.x == 0) next = (int)atomicAdd(tile_ctr, 1u);
        const uint32_t sim = tile_sim[t];
        load_desc<R>(&sd, descs + sim, NT);
        __syncthreads();
        const uint32_t start = tile_start[t];
        const uint32_t end = tile_end(tile_sim, tile_start, t, ntiles, sim, (uint32_t)sd.c.n);
        p2g_split_tile<ORDER, R>(sd.st[sd.cur], sd.vb[kpar], sd.kb[kpar], start, end, sd.acc, sd.flags, sd.c, sd.err,
                                 cellsum, cbeg, cend, pslots);
    }
}

template <int D, int ORDER, typename R, bool EXT>
__global__ void __launch_bounds__(G2P_THREADS, 4) kb_g2p(SimDesc<R>* __restrict__ descs, const uint32_t* __restrict__ tile_sim,
                                              const uint32_t* __restrict__ tile_start,
                                              const uint32_t* __restrict__ ntiles_p, uint32_t* __restrict__ tile_ctr,
                                              int kpar)
{
    constexpr int BN = (D == 3) ? 64 : 16;
    constexpr int NB = 1 << D;
    __shared__ __align__(128) R sv[2][NB][BN][4];
    __shared__ __align__(16) R stage[g2p_staged<R>() ? 2 * G2P_THREADS * kG2PSlot : 1];
    __shared__ __align__(8) uint64_t mbar[2];
    // s_t[b]: the tile staged in buffer b (written and read as in k_g2p)
    __shared__ int s_ok, s_t[2];
    __shared__ __align__(16) SimDesc<R> sd;
    unsigned phase[2] = {0u, 0u};
    const int ntiles = (int)*ntiles_p;
    // the grid-block copies of tile t (its simulation read from global): thread 0 in the
    // block layout, warp 0 in the dense one
    constexpr bool DENSE = g2p_dense<ORDER>();
    const int lane = threadIdx.x & 31;
    auto issue = [&](int t, int b) {
        const SimDesc<R>& d = descs[tile_sim[t]];
        const uint32_t blk = d.kb[kpar][tile_start[t]] >> (2 * D);
        if (DENSE) g2p_issue_dense<D, R>(d.vel, blk, d.c.nb, sv[b], &mbar[b], lane);
        else g2p_issue<D, R>(d.vel, blk, d.c.nb, sv[b], &mbar[b]);
    };
    if (threadIdx.x < 32) {
        int t0 = 0;
        if (lane == 0) {
            mbar_init(&mbar[0], 1);
            mbar_init(&mbar[1], 1);
            t0 = (int)atomicAdd(tile_ctr + 1, 1u);
            s_t[0] = t0;
            if (!DENSE && t0 < ntiles) issue(t0, 0);
        }
        if (DENSE) {
            t0 = __shfl_sync(FULLMASK, t0, 0);
            if (t0 < ntiles) issue(t0, 0);
        }
    }
    __syncthreads();
    for (int buf = 0;; buf ^= 1) {
        const int t = s_t[buf];
        if (t >= ntiles) break;
        const uint32_t sim = tile_sim[t];
        load_desc<R>(&sd, descs + sim, G2P_THREADS);
        if (threadIdx.x < 32) {
            int t1 = 0;
            if (lane == 0) {
                t1 = (int)atomicAdd(tile_ctr + 1, 1u);
                s_t[buf ^ 1] = t1;
                if (!DENSE && t1 < ntiles) issue(t1, buf ^ 1);
            }
            if (DENSE) {
                t1 = __shfl_sync(FULLMASK, t1, 0);
                if (t1 < ntiles) issue(t1, buf ^ 1);
            }
            if (lane == 0) {
                const bool ok = g2p_wait(&mbar[buf], phase[buf], descs[sim].err, descs[sim].c.wait_limit);   // sd is not complete before the barrier
                if (!ok && t1 < ntiles) mbar_wait_bounded(&mbar[buf ^ 1], phase[buf ^ 1], 1u << 22);   // drain before leaving
                s_ok = ok ? 1 : 0;
            }
        }
        __syncthreads();
        if (!s_ok) return;
        const uint32_t start = tile_start[t];
        const uint32_t end = tile_end(tile_sim, tile_start, t, ntiles, sim, (uint32_t)sd.c.n);
        float smax_unused = 0.0f;   // members are stepped at their fixed dt
        g2p_compute<D, ORDER, R, EXT, G2P_THREADS>(sd.st[sd.cur], sd.st[sd.cur ^ 1], sd.vb[kpar], sd.kb[kpar], start, end, sd.knext, sd.c,
                                 sd.err, sd.fallbacks, sv[buf], smax_unused, nullptr, stage);
        __syncthreads();
        phase[buf] ^= 1u;
    }
}

// one warp per node block of any member; bbase[s] = first global block of simulation s
template <int D, typename R>
__global__ void __launch_bounds__(TPB) kb_grid_update(SimDesc<R>* __restrict__ descs, const uint32_t* __restrict__ bbase,
                                                      int nsims, uint32_t total_blocks)
{
    // a warp takes 32 consecutive blocks: each lane finds its block's simulation and flag,
    // then the warp updates the flagged ones (most blocks of sparse grids are not)
    const int lane = threadIdx.x & 31;
    const uint32_t gw = (blockIdx.x * TPB + threadIdx.x) >> 5;
    const uint32_t nw = (gridDim.x * TPB) >> 5;
    for (uint32_t g0 = gw * 32u; g0 < total_blocks; g0 += nw * 32u) {
        const uint32_t gb = g0 + (uint32_t)lane;
        int sim = 0;
        bool on = false;
        if (gb < total_blocks) {
            int lo = 0, hi = nsims - 1;   // last s with bbase[s] <= gb
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (bbase[mid] <= gb) lo = mid;
                else hi = mid - 1;
            }
            sim = lo;
            on = descs[sim].flags[gb - bbase[sim]] != 0u;
        }
        unsigned todo = __ballot_sync(FULLMASK, on);
        while (todo) {
            const int src = __ffs(todo) - 1;
            todo &= todo - 1u;
            const int s2 = __shfl_sync(FULLMASK, sim, src);
            const SimDesc<R>& d = descs[s2];
            grid_update_block<D, R>(d.acc, d.vel, d.flags, d.c, (int)(g0 + (uint32_t)src - bbase[s2]), lane, nullptr,
                                    nullptr, true);
        }
    }
}

// end of a batched step: flip each member's state parity; G2P has stored its particles in
// sorted order, so the next sort may be incremental
template <typename R> __global__ void kb_finish(SimDesc<R>* __restrict__ descs, int nsims, uint32_t* bsorted)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < nsims) {
        descs[s].cur ^= 1;
        bsorted[s] = 1u;
    }
}

template <typename R> struct BatchImpl {
    template <int D, int O, int G> static cudaError_t setup_one(int* p2g_per_sm, int* g2p_per_sm)
    {
        const int smem = (int)p2g_cells_smem<D, O, R>();
        cudaError_t e = cudaFuncSetAttribute(kb_p2g_cells<D, O, R, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(p2g_per_sm, kb_p2g_cells<D, O, R, G>, 128, smem);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(g2p_per_sm, kb_g2p<D, O, R, false>, G2P_THREADS, 0);
        return e;
    }
    template <int O> static cudaError_t setup_split(int* p2g_per_sm, int* g2p_per_sm)
    {
        const int smem = (int)p2g_split_smem<O, R>();
        cudaError_t e = cudaFuncSetAttribute(kb_p2g_split<O, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(p2g_per_sm, kb_p2g_split<O, R>, SplitShape<O>::NT, smem);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(g2p_per_sm, kb_g2p<3, O, R, false>, G2P_THREADS, 0);
        return e;
    }
    // lane groups of 1, 2, 4 or 8 per base cell (fewer lanes suit fewer particles per cell), or
    // the component-split kernel (group 16, 3-D)
    template <int D, int O> static cudaError_t setup_dg(int group, int* p, int* g)
    {
        if (D == 3 && group == 16) return setup_split<O>(p, g);
        if (group == 8) return setup_one<D, O, 8>(p, g);
        if (group == 2) return setup_one<D, O, 2>(p, g);
        if (group == 1) return setup_one<D, O, 1>(p, g);
        return setup_one<D, O, 4>(p, g);
    }
    static cudaError_t setup(int dim, int order, int group, int* p2g_per_sm, int* g2p_per_sm)
    {
        if (dim == 3 && order == 2) return setup_dg<3, 2>(group, p2g_per_sm, g2p_per_sm);
        if (dim == 2 && order == 2) return setup_dg<2, 2>(group, p2g_per_sm, g2p_per_sm);
        if (dim == 2 && order == 3) return setup_dg<2, 3>(group, p2g_per_sm, g2p_per_sm);
        if (dim == 3 && order == 3) return setup_dg<3, 3>(group, p2g_per_sm, g2p_per_sm);
        return cudaErrorInvalidValue;
    }
    template <int D, int O, int G>
    static void p2g_one(void* descs, const uint32_t* ts, const uint32_t* tst, const uint32_t* nt, uint32_t* ctr, int kpar,
                        int grid, cudaStream_t s)
    {
        kb_p2g_cells<D, O, R, G><<<grid, 128, p2g_cells_smem<D, O, R>(), s>>>((SimDesc<R>*)descs, ts, tst, nt, ctr, kpar);
    }
    template <int D, int O>
    static void p2g_dg(int group, void* descs, const uint32_t* ts, const uint32_t* tst, const uint32_t* nt,
                       uint32_t* ctr, int kpar, int grid, cudaStream_t s)
    {
        if (D == 3 && group == 16)
            kb_p2g_split<O, R><<<grid, SplitShape<O>::NT, p2g_split_smem<O, R>(), s>>>((SimDesc<R>*)descs, ts, tst, nt,
                                                                                      ctr, kpar);
        else if (group == 8) p2g_one<D, O, 8>(descs, ts, tst, nt, ctr, kpar, grid, s);
        else if (group == 2) p2g_one<D, O, 2>(descs, ts, tst, nt, ctr, kpar, grid, s);
        else if (group == 1) p2g_one<D, O, 1>(descs, ts, tst, nt, ctr, kpar, grid, s);
        else p2g_one<D, O, 4>(descs, ts, tst, nt, ctr, kpar, grid, s);
    }
    static cudaError_t p2g(int dim, int order, int group, void* descs, const uint32_t* ts, const uint32_t* tst,
                           const uint32_t* nt, uint32_t* ctr, int kpar, int grid, cudaStream_t s)
    {
        if (dim == 3 && order == 2) p2g_dg<3, 2>(group, descs, ts, tst, nt, ctr, kpar, grid, s);
        else if (dim == 2 && order == 2) p2g_dg<2, 2>(group, descs, ts, tst, nt, ctr, kpar, grid, s);
        else if (dim == 2 && order == 3) p2g_dg<2, 3>(group, descs, ts, tst, nt, ctr, kpar, grid, s);
        else if (dim == 3 && order == 3) p2g_dg<3, 3>(group, descs, ts, tst, nt, ctr, kpar, grid, s);
        else return cudaErrorInvalidValue;
        return cudaGetLastError();
    }
    static cudaError_t grid(int dim, void* descs, const uint32_t* bbase, int nsims, uint32_t total_blocks, int grid,
                            cudaStream_t s)
    {
        if (dim == 3) kb_grid_update<3, R><<<grid, TPB, 0, s>>>((SimDesc<R>*)descs, bbase, nsims, total_blocks);
        else kb_grid_update<2, R><<<grid, TPB, 0, s>>>((SimDesc<R>*)descs, bbase, nsims, total_blocks);
        return cudaGetLastError();
    }
    template <int D, int O>
    static void g2p_one(int ext, SimDesc<R>* d, const uint32_t* ts, const uint32_t* tst, const uint32_t* nt,
                        uint32_t* ctr, int kpar, int grid, cudaStream_t s)
    {
        if (ext) kb_g2p<D, O, R, true><<<grid, G2P_THREADS, 0, s>>>(d, ts, tst, nt, ctr, kpar);
        else kb_g2p<D, O, R, false><<<grid, G2P_THREADS, 0, s>>>(d, ts, tst, nt, ctr, kpar);
    }
    static cudaError_t g2p(int dim, int order, int ext, void* descs, const uint32_t* ts, const uint32_t* tst,
                           const uint32_t* nt, uint32_t* ctr, int kpar, int grid, cudaStream_t s)
    {
        SimDesc<R>* d = (SimDesc<R>*)descs;
        if (dim == 3 && order == 2) g2p_one<3, 2>(ext, d, ts, tst, nt, ctr, kpar, grid, s);
        else if (dim == 2 && order == 2) g2p_one<2, 2>(ext, d, ts, tst, nt, ctr, kpar, grid, s);
        else if (dim == 2 && order == 3) g2p_one<2, 3>(ext, d, ts, tst, nt, ctr, kpar, grid, s);
        else if (dim == 3 && order == 3) g2p_one<3, 3>(ext, d, ts, tst, nt, ctr, kpar, grid, s);
        else return cudaErrorInvalidValue;
        return cudaGetLastError();
    }
    static cudaError_t finish(void* descs, int nsims, uint32_t* bsorted, cudaStream_t s)
    {
        kb_finish<R><<<(nsims + 255) / 256, 256, 0, s>>>((SimDesc<R>*)descs, nsims, bsorted);
        return cudaGetLastError();
    }
};

#define APIC_DEFINE_BATCH(R, SFX)                                                                              \
    size_t batch_desc_bytes_##SFX() { return sizeof(SimDesc<R>); }                                            \
    void batch_make_desc_##SFX(const HostCfg& c, const Buffers& b, int cur, int64_t n, void* out)             \
    {                                                                                                          \
        *reinterpret_cast<SimDesc<R>*>(out) = make_desc<R>(c, b, cur, n);                                      \
    }                                                                                                          \
    cudaError_t batch_setup_##SFX(int dim, int order, int group, int* p, int* g)                              \
    {                                                                                                          \
        return BatchImpl<R>::setup(dim, order, group, p, g);                                                   \
    }                                                                                                          \
    cudaError_t batch_p2g_##SFX(int dim, int order, int group, void* descs, const uint32_t* ts,              \
                                const uint32_t* tst, const uint32_t* nt, uint32_t* ctr, int kpar, int grid,    \
                                cudaStream_t s)                                                                \
    {                                                                                                          \
        return BatchImpl<R>::p2g(dim, order, group, descs, ts, tst, nt, ctr, kpar, grid, s);                   \
    }                                                                                                          \
    cudaError_t batch_grid_##SFX(int dim, void* descs, const uint32_t* bbase, int nsims, uint32_t tb, int grid, \
                                 cudaStream_t s)                                                               \
    {                                                                                                          \
        return BatchImpl<R>::grid(dim, descs, bbase, nsims, tb, grid, s);                                      \
    }                                                                                                          \
    cudaError_t batch_g2p_##SFX(int dim, int order, int ext, void* descs, const uint32_t* ts,                \
                                const uint32_t* tst, const uint32_t* nt, uint32_t* ctr, int kpar, int grid,    \
                                cudaStream_t s)                                                                \
    {                                                                                                          \
        return BatchImpl<R>::g2p(dim, order, ext, descs, ts, tst, nt, ctr, kpar, grid, s);                     \
    }                                                                                                          \
    cudaError_t batch_finish_##SFX(void* descs, int nsims, uint32_t* bsorted, cudaStream_t s)                 \
    {                                                                                                          \
        return BatchImpl<R>::finish(descs, nsims, bsorted, s);                                                 \
    }                                                                                                          \
    int batch_desc_cur_offset_##SFX() { return (int)offsetof(SimDesc<R>, cur); }

}  // namespace apic
