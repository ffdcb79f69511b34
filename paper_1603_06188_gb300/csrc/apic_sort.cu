// apic_sort.cu -- stable LSD radix sort of particle cell keys, a device-wide exclusive
// scan, and the tile list that P2G / G2P walk.  The sort is what lets P2G accumulate a
// grid block's particles in shared memory (the key is the particle's stencil-base block
// followed by the base node inside the block), so its order is part of the contract:
// stable, ties kept in current index order.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "apic.h"
#include "apic_internal.h"

namespace apic {

namespace {

constexpr int RT = 256;              // radix threads per CTA
constexpr int RI = 8;                // keys per thread
constexpr int RTILE = RT * RI;       // keys per radix tile
constexpr int RW = RT / 32;          // warps per CTA
constexpr int SCH = 4096;            // elements per scan chunk (256 threads x 16)
constexpr unsigned FULL = 0xffffffffu;
// up to this many chunks, a chunk's offset is a block reduction over the earlier chunks'
// counts (one kernel); above it, a device-wide scan computes the offsets first
constexpr int kReduceChunks = 4096;

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Per-tile digit histogram.  Warp w of tile lt owns keys [lt*RTILE + w*256, +256), walked in
// rounds of 32 (the same order the scatter uses).  Same-digit lanes are merged with
// match.any so the shared-memory counter sees one add per distinct digit.
__device__ __forceinline__ void radix_hist_tile(const uint32_t* __restrict__ keys, int64_t n, int64_t lt, int shift,
                                                uint32_t* h)
{
    h[threadIdx.x] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t base = lt * RTILE + w * (RI * 32);
#pragma unroll
    for (int r = 0; r < RI; ++r) {
        const int64_t idx = base + r * 32 + lane;
        const bool valid = idx < n;
        const unsigned d = valid ? (keys[idx] >> shift) & 255u : 256u;
        const unsigned peers = __match_any_sync(FULL, d);
        if (valid && lane == __ffs(peers) - 1) atomicAdd(&h[d], (uint32_t)__popc(peers));
    }
    __syncthreads();
}

__global__ void __launch_bounds__(RT) k_radix_hist(const uint32_t* __restrict__ keys, int64_t n, int shift,
                                                   int ntiles, uint32_t* __restrict__ counts)
{
    __shared__ uint32_t h[256];
    radix_hist_tile(keys, n, blockIdx.x, shift, h);
    counts[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter: rank = (global start of this digit in this tile) + (same digit in earlier
// warps of the tile) + (same digit earlier in this warp).  goff[d] (shared) holds the first
// output slot of digit d for this tile.
__device__ __forceinline__ void radix_scatter_tile(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                                                   uint32_t* __restrict__ kout, uint32_t* __restrict__ vout, int64_t n,
                                                   int64_t lt, int shift, const uint32_t* goff, uint32_t (*wc)[256])
{
    for (int i = threadIdx.x; i < RW * 256; i += RT) (&wc[0][0])[i] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t base = lt * RTILE + w * (RI * 32);
    uint32_t key[RI], val[RI], lr[RI];
    unsigned dig[RI];
#pragma unroll
    for (int r = 0; r < RI; ++r) {
        const int64_t idx = base + r * 32 + lane;
        const bool valid = idx < n;
        key[r] = valid ? kin[idx] : 0u;
        val[r] = valid ? (vin ? vin[idx] : (uint32_t)idx) : 0u;
        const unsigned d = valid ? (key[r] >> shift) & 255u : 256u;
        dig[r] = d;
        const unsigned peers = __match_any_sync(FULL, d);
        const unsigned before = (unsigned)__popc(peers & lanemask_lt());
        const uint32_t cnt = valid ? wc[w][d] : 0u;
        __syncwarp();
        lr[r] = cnt + before;
        if (valid && lane == __ffs(peers) - 1) wc[w][d] = cnt + (uint32_t)__popc(peers);
        __syncwarp();
    }
    __syncthreads();
    {
        uint32_t run = 0;
        for (int ww = 0; ww < RW; ++ww) {
            const uint32_t c = wc[ww][threadIdx.x];
            wc[ww][threadIdx.x] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RI; ++r) {
        const int64_t idx = base + r * 32 + lane;
        if (idx < n) {
            const unsigned d = dig[r];
            const uint32_t pos = goff[d] + wc[w][d] + lr[r];
            kout[pos] = key[r];
            vout[pos] = val[r];
        }
    }
}

__global__ void __launch_bounds__(RT) k_radix_scatter(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                                                      uint32_t* __restrict__ kout, uint32_t* __restrict__ vout, int64_t n,
                                                      int shift, int ntiles, const uint32_t* __restrict__ offsets)
{
    __shared__ uint32_t wc[RW][256];
    __shared__ uint32_t goff[256];
    goff[threadIdx.x] = offsets[(int64_t)threadIdx.x * ntiles + blockIdx.x];
    radix_scatter_tile(kin, vin, kout, vout, n, blockIdx.x, shift, goff, wc);
}

// ---------------------------------------------------------------- exclusive scan
__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v, int lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(FULL, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// exclusive scan of one value per thread over a 256-thread CTA; returns the CTA total
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t& excl)
{
    __shared__ uint32_t ws[8];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t inc = warp_incl_scan(v, lane);
    if (lane == 31) ws[w] = inc;
    __syncthreads();
    if (w == 0) {
        uint32_t t = lane < 8 ? ws[lane] : 0u;
        t = warp_incl_scan(t, lane);
        if (lane < 8) ws[lane] = t;
    }
    __syncthreads();
    excl = inc - v + (w > 0 ? ws[w - 1] : 0u);
    const uint32_t total = ws[7];
    __syncthreads();
    return total;
}

__global__ void __launch_bounds__(256) k_scan_reduce(const uint32_t* __restrict__ in, int64_t n, uint32_t* __restrict__ part)
{
    pdl_wait();
    pdl_trigger();
    const int64_t base = (int64_t)blockIdx.x * SCH + threadIdx.x * 16;
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < 16; ++i)
        if (base + i < n) s += in[base + i];
    uint32_t ex;
    const uint32_t tot = block_excl_scan(s, ex);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(256) k_scan_top(uint32_t* __restrict__ part, int64_t np, uint32_t* __restrict__ total)
{
    pdl_wait();
    pdl_trigger();
    uint32_t carry = 0;
    for (int64_t b = 0; b < np; b += 256) {
        const int64_t i = b + threadIdx.x;
        const uint32_t v = i < np ? part[i] : 0u;
        uint32_t ex;
        const uint32_t tot = block_excl_scan(v, ex);
        if (i < np) part[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0 && total) *total = carry;
}

__global__ void __launch_bounds__(256) k_scan_down(const uint32_t* in, uint32_t* out, int64_t n,
                                                   const uint32_t* __restrict__ part)
{
    pdl_wait();
    pdl_trigger();
    const int64_t base = (int64_t)blockIdx.x * SCH + threadIdx.x * 16;
    uint32_t v[16];
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        v[i] = (base + i < n) ? in[base + i] : 0u;
        s += v[i];
    }
    uint32_t ex;
    block_excl_scan(s, ex);
    uint32_t run = part[blockIdx.x] + ex;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        if (base + i < n) out[base + i] = run;
        run += v[i];
    }
}

// ---------------------------------------------------------------- tiles
// A tile is a maximal run of sorted particles with the same node block inside one aligned
// chunk of `tile` particles; a new tile starts at every chunk start and every block change.
// Tile heads of chunk [cs, cs + tile), tile <= 4096: thread t of the 256 takes the kpt =
// tile / 256 consecutive keys from cs + kpt t (four 16-byte loads for a full aligned chunk of
// 4096) plus the key before them, so the chunk costs about one memory latency; bit i of the
// result flags a head at cs + kpt t + i.
__device__ __forceinline__ unsigned chunk_head_bits(const uint32_t* __restrict__ skeys, int64_t n, int sh, int tile,
                                                    int64_t cs)
{
    const int kpt = tile >> 8;
    const int64_t ce = cs + tile < n ? cs + tile : n;
    const int64_t k0 = cs + (int64_t)threadIdx.x * kpt;
    uint32_t key[16];
    if (kpt == 16 && k0 + 16 <= ce && ((reinterpret_cast<uintptr_t>(skeys + k0) & 15u) == 0u)) {
        const uint4* q = reinterpret_cast<const uint4*>(skeys + k0);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint4 v = __ldg(q + j);
            key[4 * j + 0] = v.x;
            key[4 * j + 1] = v.y;
            key[4 * j + 2] = v.z;
            key[4 * j + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int i = 0; i < 16; ++i) key[i] = (i < kpt && k0 + i < ce) ? skeys[k0 + i] : 0u;
    }
    const uint32_t prev = (k0 > cs && k0 < ce) ? skeys[k0 - 1] : 0u;
    unsigned bits = 0u;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const uint32_t pk = i == 0 ? prev : key[i - 1];
        if (i < kpt && k0 + i < ce && (k0 + i == cs || (key[i] >> sh) != (pk >> sh))) bits |= 1u << i;
    }
    return bits;
}

// number of heads of the chunk (whole block of 256)
__device__ __forceinline__ uint32_t count_heads(const uint32_t* __restrict__ skeys, int64_t n, int sh, int tile,
                                                int64_t cs)
{
    uint32_t ex;
    return block_excl_scan((uint32_t)__popc(chunk_head_bits(skeys, n, sh, tile, cs)), ex);
}

// writes, in index order, every head of the chunk through emit(position, k) (whole block of
// 256): one block scan of the per-thread head counts gives each thread its first position
template <class Emit>
__device__ __forceinline__ void write_heads(const uint32_t* __restrict__ skeys, int64_t n, int sh, int tile, int64_t cs,
                                            uint32_t pos0, Emit emit)
{
    const unsigned bits = chunk_head_bits(skeys, n, sh, tile, cs);
    uint32_t ex;
    block_excl_scan((uint32_t)__popc(bits), ex);
    const int64_t k0 = cs + (int64_t)threadIdx.x * (tile >> 8);
#pragma unroll
    for (int i = 0; i < 16; ++i)
        if ((bits >> i) & 1u) emit(pos0 + ex + (uint32_t)__popc(bits & ((1u << i) - 1u)), k0 + i);
}

__global__ void __launch_bounds__(256) k_tile_count(const uint32_t* __restrict__ skeys, int64_t n, int sh, int tile,
                                                    uint32_t* __restrict__ cnt)
{
    pdl_wait();
    pdl_trigger();
    const uint32_t tot = count_heads(skeys, n, sh, tile, (int64_t)blockIdx.x * tile);
    if (threadIdx.x == 0) cnt[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(256) k_tile_write(const uint32_t* __restrict__ skeys, int64_t n, int sh, int tile,
                                                    const uint32_t* __restrict__ off, uint32_t* __restrict__ ntiles,
                                                    int64_t max_tiles, uint32_t* __restrict__ tiles, int nchunks,
                                                    uint32_t* __restrict__ err, uint32_t* __restrict__ tile_ctr,
                                                    const uint32_t* __restrict__ cnt)
{
    pdl_wait();
    pdl_trigger();
    // with cnt given, off[] and ntiles are computed here: chunk t's offset is the sum of the
    // counts of chunks 0..t-1 (a block reduction, used while the chunks are few)
    __shared__ uint32_t s_off;
    if (blockIdx.x == 0 && threadIdx.x < 2) tile_ctr[threadIdx.x] = 0u;
    if (cnt) {
        uint32_t part = 0;
        for (uint32_t i = threadIdx.x; i < blockIdx.x; i += 256) part += cnt[i];
        uint32_t ex;
        const uint32_t o = block_excl_scan(part, ex);
        if (threadIdx.x == 0) {
            s_off = o;
            if ((int)blockIdx.x == nchunks - 1) *ntiles = o + cnt[blockIdx.x];
        }
    } else if (threadIdx.x == 0) {
        s_off = off[blockIdx.x];
    }
    __syncthreads();
    const int64_t cs = (int64_t)blockIdx.x * tile;
    write_heads(skeys, n, sh, tile, cs, s_off, [&](uint32_t pos, int64_t k) {
        if ((int64_t)pos < max_tiles) tiles[pos] = (uint32_t)k;
    });
    if ((int)blockIdx.x == nchunks - 1 && threadIdx.x == 0) {
        const uint32_t nt = cnt ? s_off + cnt[blockIdx.x] : *ntiles;
        if ((int64_t)nt < max_tiles) tiles[nt] = (uint32_t)n;
        else atomicOr(err, APIC_ERRBIT_CAPACITY);
    }
}

// ---------------------------------------------------------------- one-sweep passes
// All digit histograms in one read of the keys, then one kernel per pass: a tile ranks its
// keys as in radix_scatter_tile, publishes its per-digit counts, and finds the counts of
// all earlier tiles by looking back over their published words (decoupled look-back:
// a word holds a flag -- tile aggregate, or inclusive prefix -- and a 30-bit count).
// Tiles take their index from a counter, so every earlier tile is already resident and
// the look-back always ends; each wait is still bounded and latches APIC_ERRBIT_TIMEOUT.
constexpr uint32_t LB_AGG = 1u << 30;
constexpr uint32_t LB_INC = 2u << 30;
constexpr uint32_t LB_VAL = (1u << 30) - 1u;

__global__ void __launch_bounds__(256) k_onesweep_hist(const uint32_t* __restrict__ keys, int64_t n, int passes,
                                                       uint32_t* __restrict__ ghist)
{
    __shared__ uint32_t h[4][256];
    for (int i = threadIdx.x; i < 4 * 256; i += 256) (&h[0][0])[i] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    for (int64_t base = (int64_t)blockIdx.x * 256; base < n; base += (int64_t)gridDim.x * 256) {
        const int64_t k = base + threadIdx.x;
        const bool valid = k < n;
        const uint32_t key = valid ? keys[k] : 0u;
        for (int p = 0; p < passes; ++p) {
            const unsigned d = valid ? (key >> (8 * p)) & 255u : 256u;
            const unsigned peers = __match_any_sync(0xffffffffu, d);
            if (valid && lane == __ffs(peers) - 1) atomicAdd(&h[p][d], (uint32_t)__popc(peers));
        }
    }
    __syncthreads();
    for (int p = 0; p < passes; ++p)
        if (h[p][threadIdx.x]) atomicAdd(&ghist[p * 256 + threadIdx.x], h[p][threadIdx.x]);
}

// exclusive scan of each pass's 256-bin histogram, in place (one CTA)
__global__ void __launch_bounds__(256) k_onesweep_digits(uint32_t* __restrict__ ghist, int passes)
{
    for (int p = 0; p < passes; ++p) {
        const uint32_t v = ghist[p * 256 + threadIdx.x];
        uint32_t ex;
        block_excl_scan(v, ex);
        ghist[p * 256 + threadIdx.x] = ex;
    }
}

__device__ __forceinline__ uint32_t ld_volatile(const uint32_t* p)
{
    uint32_t v;
    asm volatile("ld.volatile.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_volatile(uint32_t* p, uint32_t v)
{
    asm volatile("st.volatile.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__global__ void __launch_bounds__(RT) k_onesweep_pass(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                                                      uint32_t* __restrict__ kout, uint32_t* __restrict__ vout, int64_t n,
                                                      int shift, const uint32_t* __restrict__ dstart,
                                                      uint32_t* __restrict__ status, uint32_t* __restrict__ tile_ctr,
                                                      uint32_t* __restrict__ err)
{
    __shared__ uint32_t wc[RW][256];
    __shared__ uint32_t goff[256];
    __shared__ uint32_t s_t;
    if (threadIdx.x == 0) s_t = atomicAdd(tile_ctr, 1u);
    for (int i = threadIdx.x; i < RW * 256; i += RT) (&wc[0][0])[i] = 0;
    __syncthreads();
    const uint32_t t = s_t;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t base = (int64_t)t * RTILE + w * (RI * 32);
    uint32_t key[RI], val[RI], lr[RI];
    unsigned dig[RI];
#pragma unroll
    for (int r = 0; r < RI; ++r) {
        const int64_t idx = base + r * 32 + lane;
        const bool valid = idx < n;
        key[r] = valid ? kin[idx] : 0u;
        val[r] = valid ? (vin ? vin[idx] : (uint32_t)idx) : 0u;
        const unsigned d = valid ? (key[r] >> shift) & 255u : 256u;
        dig[r] = d;
        const unsigned peers = __match_any_sync(FULL, d);
        const unsigned before = (unsigned)__popc(peers & lanemask_lt());
        const uint32_t cnt = valid ? wc[w][d] : 0u;
        __syncwarp();
        lr[r] = cnt + before;
        if (valid && lane == __ffs(peers) - 1) wc[w][d] = cnt + (uint32_t)__popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // thread d: tile count of digit d, warp bases, then the look-back for digit d
    {
        const int d = threadIdx.x;
        uint32_t run = 0;
        for (int ww = 0; ww < RW; ++ww) {
            const uint32_t c = wc[ww][d];
            wc[ww][d] = run;
            run += c;
        }
        uint32_t* my = status + (size_t)t * 256 + d;
        if (t == 0) {
            st_volatile(my, LB_INC | run);
            goff[d] = dstart[d];
        } else {
            st_volatile(my, LB_AGG | run);
            uint32_t excl = 0;
            int64_t j = (int64_t)t - 1;
            uint32_t spins = 0;
            while (j >= 0) {
                const uint32_t v = ld_volatile(status + (size_t)j * 256 + d);
                const uint32_t f = v & ~LB_VAL;
                if (f == 0u) {
                    if (++spins > (1u << 22)) {   // bounded: a predecessor never published
                        atomicOr(err, APIC_ERRBIT_TIMEOUT);
                        break;
                    }
                    __nanosleep(32);
                    continue;
                }
                excl += v & LB_VAL;
                if (f == LB_INC) break;
                --j;
            }
            st_volatile(my, LB_INC | (excl + run));
            goff[d] = dstart[d] + excl;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RI; ++r) {
        const int64_t idx = base + r * 32 + lane;
        if (idx < n) {
            const unsigned d = dig[r];
            const uint32_t pos = goff[d] + wc[w][d] + lr[r];
            kout[pos] = key[r];
            vout[pos] = val[r];
        }
    }
}

// ---------------------------------------------------------------- incremental sort
// Between steps the particles are stored in the previous sorted order (G2P writes particle
// k of that order at k), so with P = the previous sorted keys, the particles whose key did
// not change, U = {k : knext[k] == P[k]}, are already in (key, k) order.  Only the moved
// ones, M, are sorted -- stably, from index order, so by (key, k) -- and the two sorted
// sequences are merged by (key, k): the result is the stable order of all keys, the same
// permutation the full sort gives.
//   k_moved_count    counts M per chunk and M's digits for every pass
//   k_moved_compact  compacts M in index order (chunk offsets by reduction) and stores m
//   k_msort_pass  one LSD pass over M (m read on the device; tiles taken from a counter)
//   k_merge       U element k goes to (k - #M before k) + #M below (key, k); M element j to
//                 j + #U below (key, idx), counted by the chunk of P whose key range holds it
// Look-back words are 64-bit: (epoch << 32) | flag | count, with a fresh epoch for every
// use, so a word left from an earlier use reads as unpublished and nothing is cleared.
constexpr unsigned long long LB64_AGG = 1ull << 30;
constexpr unsigned long long LB64_INC = 2ull << 30;
constexpr unsigned long long LB64_VAL = (1ull << 30) - 1ull;
constexpr int MCTL_M = 1, MCTL_PASS = 2;   // mctl word indices (+ pass)

__device__ __forceinline__ unsigned long long ld_volatile64(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.volatile.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_volatile64(unsigned long long* p, unsigned long long v)
{
    asm volatile("st.volatile.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// decoupled look-back over 64-bit epoch words: publishes `run` for slot `my` of tile t (stride
// between tiles `stride`), returns the exclusive prefix of the earlier tiles
__device__ __forceinline__ uint32_t lookback64(unsigned long long* words, uint32_t t, size_t stride, uint32_t run,
                                               uint32_t epoch, uint32_t* err)
{
    const unsigned long long tag = (unsigned long long)epoch << 32;
    unsigned long long* my = words + (size_t)t * stride;
    if (t == 0) {
        st_volatile64(my, tag | LB64_INC | run);
        return 0u;
    }
    st_volatile64(my, tag | LB64_AGG | run);
    uint32_t excl = 0;
    int64_t j = (int64_t)t - 1;
    uint32_t spins = 0;
    while (j >= 0) {
        const unsigned long long v = ld_volatile64(words + (size_t)j * stride);
        if ((v >> 32) != (unsigned long long)epoch) {
            if (++spins > (1u << 22)) {   // bounded: a predecessor never published
                atomicOr(err, APIC_ERRBIT_TIMEOUT);
                break;
            }
            __nanosleep(32);
            continue;
        }
        excl += (uint32_t)(v & LB64_VAL);
        if ((v & ~(LB64_VAL | (0xffffffffull << 32))) == LB64_INC) break;
        --j;
    }
    st_volatile64(my, tag | LB64_INC | (excl + run));
    return excl;
}

// zeroes the incremental sort's control words and digit counts (a kernel rather than a memset,
// so that the step's chain of dependent launches is not broken)
__global__ void __launch_bounds__(256) k_msort_reset(uint32_t* __restrict__ mctl, int words)
{
    pdl_wait();
    pdl_trigger();
    for (int i = blockIdx.x * 256 + threadIdx.x; i < words; i += gridDim.x * 256) mctl[i] = 0u;
}

// moved keys of chunk t (RTILE consecutive indices, thread-major rounds): count per chunk and
// the digit counts of every pass.  All keys of the thread are loaded before any is counted
// (the shared-memory atomics would otherwise hold back the later loads), and the digit counts
// go to copy t % kMhistCopies of the histogram: the high digits of the moved keys are nearly
// all alike, and one global counter per digit would take every chunk's add in turn.
// The moved flags also go to a bitmap (word blockIdx.x * RTILE / 32 + r * RW + w holds the
// flags of round r of warp w, bit = lane), so that the compaction and the merge read 1 bit
// per key instead of both keys.
__global__ void __launch_bounds__(RT) k_moved_count(const uint32_t* __restrict__ knext, const uint32_t* __restrict__ pk,
                                                    int64_t n, uint32_t* __restrict__ cnt, uint32_t* __restrict__ mhist,
                                                    int passes, uint32_t* __restrict__ mbits)
{
    pdl_wait();
    pdl_trigger();
    __shared__ uint32_t h[4][256];
    for (int i = threadIdx.x; i < 4 * 256; i += RT) (&h[0][0])[i] = 0u;
    const int64_t base = (int64_t)blockIdx.x * RTILE;
    uint32_t kn[RI], kp[RI];
#pragma unroll
    for (int r = 0; r < RI; ++r) {
        const int64_t k = base + r * RT + threadIdx.x;
        kn[r] = k < n ? knext[k] : 0u;
        kp[r] = k < n ? pk[k] : 0u;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int r = 0; r < RI; ++r) {
        const unsigned bal = __ballot_sync(FULL, kn[r] != kp[r]);
        if (lane == 0) mbits[(size_t)blockIdx.x * (RTILE / 32) + r * RW + w] = bal;
    }
    uint32_t c = 0;
#pragma unroll
    for (int r = 0; r < RI; ++r) {
        if (kn[r] != kp[r]) {
            ++c;
            for (int p = 0; p < passes; ++p) atomicAdd(&h[p][(kn[r] >> (8 * p)) & 255u], 1u);
        }
    }
    uint32_t ex;
    const uint32_t total = block_excl_scan(c, ex);
    if (threadIdx.x == 0) cnt[blockIdx.x] = total;
    uint32_t* hc = mhist + (size_t)(blockIdx.x % kMhistCopies) * (4 * 256);
    for (int i = threadIdx.x; i < passes * 256; i += RT) {
        const uint32_t v = (&h[0][0])[i];
        if (v) atomicAdd(hc + i, v);
    }
}

// compaction of the moved keys in index order; chunk t's offset is off[t] (a device scan) or,
// with off null, the sum of the counts of chunks 0..t-1 (a block reduction, used while the
// chunks are few), the last chunk stores m
__global__ void __launch_bounds__(RT) k_moved_compact(const uint32_t* __restrict__ knext, const uint32_t* __restrict__ pk,
                                                      int64_t n, const uint32_t* __restrict__ cnt,
                                                      const uint32_t* __restrict__ off, int nchunks,
                                                      uint32_t* __restrict__ ctl, uint32_t* __restrict__ mk,
                                                      uint32_t* __restrict__ mv,
                                                      uint32_t* __restrict__ choff, uint32_t* __restrict__ err,
                                                      const uint32_t* __restrict__ mbits)
{
    pdl_wait();
    pdl_trigger();
    __shared__ uint32_t wc[RI][RW];
    const uint32_t t = blockIdx.x;
    uint32_t excl;
    if (off) {
        excl = off[t];
    } else {
        uint32_t part = 0;
        for (uint32_t i = threadIdx.x; i < t; i += RT) part += cnt[i];
        uint32_t ex;
        excl = block_excl_scan(part, ex);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t base = (int64_t)t * RTILE;
    uint32_t key[RI];
    unsigned bal[RI];
#pragma unroll
    for (int r = 0; r < RI; ++r) {
        const int64_t k = base + r * RT + threadIdx.x;
        bal[r] = mbits[(size_t)t * (RTILE / 32) + r * RW + w];
        const bool moved = (bal[r] >> lane) & 1u;
        key[r] = moved ? knext[k] : 0u;
        if (lane == 0) wc[r][w] = (uint32_t)__popc(bal[r]);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t run = excl;
        for (int r = 0; r < RI; ++r)
            for (int ww = 0; ww < RW; ++ww) {
                const uint32_t c = wc[r][ww];
                wc[r][ww] = run;
                run += c;
            }
        choff[t] = excl;
        if ((int)t == nchunks - 1) {
            // counts that add up to more than n keys cannot come from knext: the range
            // error is raised and nothing is sorted
            if (run > (uint32_t)n) atomicOr(err, APIC_ERRBIT_RANGE);
            ctl[MCTL_M] = run <= (uint32_t)n ? run : 0u;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RI; ++r) {
        if (bal[r] & (1u << lane)) {
            const int64_t k = base + r * RT + threadIdx.x;
            const uint32_t p = wc[r][w] + (uint32_t)__popc(bal[r] & lanemask_lt());
            if (p < (uint32_t)n) {
                mk[p] = key[r];
                mv[p] = (uint32_t)k;
            } else {
                atomicOr(err, APIC_ERRBIT_RANGE);
            }
        }
    }
}

__global__ void __launch_bounds__(RT) k_msort_pass(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                                                   uint32_t* __restrict__ kout, uint32_t* __restrict__ vout,
                                                   uint32_t* __restrict__ ctl, int pass, const uint32_t* __restrict__ hist,
                                                   unsigned long long* lbs, uint32_t epoch, uint32_t* err)
{
    pdl_wait();
    pdl_trigger();
    __shared__ uint32_t wc[RW][256];
    __shared__ uint32_t goff[256];
    __shared__ uint32_t dst0[256];
    __shared__ uint32_t s_t;
    const uint32_t m = ctl[MCTL_M];
    const uint32_t nt = (m + RTILE - 1) / RTILE;
    if (blockIdx.x >= nt) return;
    {
        uint32_t hv = 0, ex;   // the digit's count, summed over the histogram's copies
#pragma unroll
        for (int cp = 0; cp < kMhistCopies; ++cp) hv += hist[cp * (4 * 256) + threadIdx.x];
        block_excl_scan(hv, ex);
        dst0[threadIdx.x] = ex;
    }
    const int shift = 8 * pass;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (;;) {
        if (threadIdx.x == 0) s_t = atomicAdd(ctl + MCTL_PASS + pass, 1u);
        for (int i = threadIdx.x; i < RW * 256; i += RT) (&wc[0][0])[i] = 0u;
        __syncthreads();
        const uint32_t t = s_t;
        if (t >= nt) break;
        const int64_t base = (int64_t)t * RTILE + w * (RI * 32);
        uint32_t key[RI], val[RI], lr[RI];
        unsigned dig[RI];
#pragma unroll
        for (int r = 0; r < RI; ++r) {
            const int64_t idx = base + r * 32 + lane;
            const bool valid = idx < (int64_t)m;
            key[r] = valid ? kin[idx] : 0u;
            val[r] = valid ? vin[idx] : 0u;
            const unsigned d = valid ? (key[r] >> shift) & 255u : 256u;
            dig[r] = d;
            const unsigned peers = __match_any_sync(FULL, d);
            const unsigned before = (unsigned)__popc(peers & lanemask_lt());
            const uint32_t cnt = valid ? wc[w][d] : 0u;
            __syncwarp();
            lr[r] = cnt + before;
            if (valid && lane == __ffs(peers) - 1) wc[w][d] = cnt + (uint32_t)__popc(peers);
            __syncwarp();
        }
        __syncthreads();
        {
            const int d = threadIdx.x;
            uint32_t run = 0;
            for (int ww = 0; ww < RW; ++ww) {
                const uint32_t c = wc[ww][d];
                wc[ww][d] = run;
                run += c;
            }
            goff[d] = dst0[d] + lookback64(lbs + d, t, 256, run, epoch, err);
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < RI; ++r) {
            const int64_t idx = base + r * 32 + lane;
            if (idx < (int64_t)m) {
                const unsigned d = dig[r];
                const uint32_t pos = goff[d] + wc[w][d] + lr[r];
                if (pos < m) {
                    kout[pos] = key[r];
                    vout[pos] = val[r];
                } else {
                    atomicOr(err, APIC_ERRBIT_RANGE);   // inconsistent counts: never write past m
                }
            }
        }
        __syncthreads();
    }
}

// number of (msk[j], msv[j]) in [lo, hi) below (key, idx); the sequence is sorted by (key, index)
__device__ __forceinline__ uint32_t below_m(const uint32_t* msk, const uint32_t* msv, uint32_t lo, uint32_t hi,
                                            uint32_t key, uint32_t idx)
{
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        const uint32_t a = msk[mid];
        if (a < key || (a == key && msv[mid] < idx)) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// moved keys of a chunk's key range staged in shared memory for the merge's searches
constexpr uint32_t MERGE_MCAP = 2048;

// Chunk t of P (indices [base, end)) owns the moved keys M[j] with j in [s_lo, s_nx): those at
// or above (P[base], base) and below the next chunk's first (P[end], end) (chunk 0 also the
// ones below its first key).  Its unmoved keys u get c_u = #M below (P[k], k) by a search of
// that range (staged in shared memory) and go to (k - #moved before k) + c_u.  A moved key
// M[j] of the range lies above every unmoved key of the earlier chunks and below every one of
// the later chunks, and above the chunk's own unmoved u exactly when c_u <= j; so it goes to
// j + #unmoved before the chunk + #{u : c_u <= j}, counted by a search of the c_u (kept in
// order in shared memory).
__global__ void __launch_bounds__(RT) k_merge(const uint32_t* __restrict__ knext, const uint32_t* __restrict__ pk,
                                              int64_t n, const uint32_t* __restrict__ choff,
                                              const uint32_t* __restrict__ msk, const uint32_t* __restrict__ msv,
                                              const uint32_t* __restrict__ ctl, int nchunks,
                                              uint32_t* __restrict__ kout, uint32_t* __restrict__ vout, uint32_t* err,
                                              const uint32_t* __restrict__ mbits)
{
    pdl_wait();
    pdl_trigger();
    __shared__ uint32_t wc[RI][RW];
    __shared__ uint32_t s_lo, s_nx, s_nm;
    __shared__ uint32_t sk[MERGE_MCAP], sv[MERGE_MCAP];
    __shared__ uint32_t cu[RTILE];
    const uint32_t m = ctl[MCTL_M];
    const uint32_t t = blockIdx.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t base = (int64_t)t * RTILE;
    const int64_t end = base + RTILE < n ? base + RTILE : n;
    // the two bounds of the chunk's range, by two warps at once
    if (threadIdx.x == 0) s_lo = below_m(msk, msv, 0u, m, pk[base], (uint32_t)base);
    if (threadIdx.x == 32) s_nx = end < n ? below_m(msk, msv, 0u, m, pk[end], (uint32_t)end) : m;
    unsigned bal[RI];
#pragma unroll
    for (int r = 0; r < RI; ++r) {
        bal[r] = mbits[(size_t)t * (RTILE / 32) + r * RW + w];
        if (lane == 0) wc[r][w] = (uint32_t)__popc(bal[r]);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t run = choff[t];
        for (int r = 0; r < RI; ++r)
            for (int ww = 0; ww < RW; ++ww) {
                const uint32_t c = wc[r][ww];
                wc[r][ww] = run;
                run += c;
            }
        s_nm = run - choff[t];
    }
    const uint32_t lo = s_lo, hi = s_nx > s_lo ? s_nx : s_lo;
    const bool staged = hi - lo <= MERGE_MCAP;
    if (staged)
        for (uint32_t j = lo + threadIdx.x; j < hi; j += RT) {
            sk[j - lo] = msk[j];
            sv[j - lo] = msv[j];
        }
    __syncthreads();
    const uint32_t uoff = (uint32_t)base - choff[t];   // unmoved keys before the chunk
#pragma unroll
    for (int r = 0; r < RI; ++r) {
        const int64_t k = base + r * RT + threadIdx.x;
        if (k < n && !(bal[r] & (1u << lane))) {
            const uint32_t before = wc[r][w] + (uint32_t)__popc(bal[r] & lanemask_lt());
            const uint32_t key = pk[k];
            const uint32_t c = staged ? lo + below_m(sk, sv, 0u, hi - lo, key, (uint32_t)k)
                                      : below_m(msk, msv, lo, hi, key, (uint32_t)k);
            const uint32_t u = (uint32_t)k - before;
            if (u - uoff < (uint32_t)RTILE) cu[u - uoff] = c;
            const uint32_t pos = u + c;
            if (pos < (uint32_t)n) {
                kout[pos] = key;
                vout[pos] = (uint32_t)k;
            } else {
                atomicOr(err, APIC_ERRBIT_RANGE);
            }
        }
    }
    __syncthreads();
    const uint32_t len = (uint32_t)(end - base);
    if (s_nm > len) {   // moved counts that do not fit the chunk: report, place nothing more
        if (threadIdx.x == 0) atomicOr(err, APIC_ERRBIT_RANGE);
        return;
    }
    const uint32_t nu = len - s_nm;
    for (uint32_t j = (t == 0 ? 0u : lo) + threadIdx.x; j < hi; j += RT) {
        uint32_t a = 0, b = nu;
        while (a < b) {
            const uint32_t mid = (a + b) >> 1;
            if (cu[mid] <= j) a = mid + 1;
            else b = mid;
        }
        const bool in = staged && j >= lo;
        const uint32_t pos = j + uoff + a;
        if (pos < (uint32_t)n) {
            kout[pos] = in ? sk[j - lo] : msk[j];
            vout[pos] = in ? sv[j - lo] : msv[j];
        } else {
            atomicOr(err, APIC_ERRBIT_RANGE);
        }
    }
}

// ---------------------------------------------------------------- batched forms
// Work item -> simulation tables (rt_sim per radix tile, ch_sim per chunk) are built on the
// host when membership changes.

// ---------------------------------------------------------------- batched incremental sort
// The incremental sort above, per member of a batch.  A member whose particles are not yet
// in its previous sorted order (bsorted[s] = 0: new in the batch) counts every key as
// changed, which makes the same kernels a full stable sort of it.  The previous sorted keys
// P are copied from kb[kpar] to kb[kpar ^ 1] while the changed keys are counted, so the
// output stays in kb[kpar] / vb[kpar], where the batched P2G and G2P read it.  The look-back
// epoch and the pass tile counters are device words (bctl: [0] epoch, [1 + p] pass p's
// counter), advanced on the device, so a captured step graph replays correctly.

__global__ void __launch_bounds__(256) kb_rs_init(const SortDesc* __restrict__ sd, uint32_t* __restrict__ bctl)
{
    // one CTA per member: clear its control words and digit counts
    uint32_t* ctl = sd[blockIdx.x].mctl;
    for (int i = threadIdx.x; i < 16 + 4 * 256; i += 256) ctl[i] = 0u;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        bctl[0] += 8u;
        bctl[1] = bctl[2] = bctl[3] = bctl[4] = 0u;
    }
}

__global__ void __launch_bounds__(RT) kb_moved_count(const SortDesc* __restrict__ sd, const uint32_t* __restrict__ rt_sim,
                                                     const uint32_t* __restrict__ bsorted, int kpar, int passes)
{
    __shared__ uint32_t h[4][256];
    for (int i = threadIdx.x; i < 4 * 256; i += RT) (&h[0][0])[i] = 0u;
    __syncthreads();
    const uint32_t sim = rt_sim[blockIdx.x];
    const SortDesc& d = sd[sim];
    const int64_t lt = (int64_t)blockIdx.x - d.rbase;
    const int64_t n = d.n;
    const int64_t base = lt * RTILE;
    const uint32_t* P = bsorted[sim] ? d.kb[kpar] : nullptr;
    uint32_t* Pc = d.kb[kpar ^ 1];
    // every key of the thread is loaded before any is counted (as in k_moved_count)
    uint32_t kn[RI], kp[RI];
#pragma unroll
    for (int r = 0; r < RI; ++r) {
        const int64_t k = base + r * RT + threadIdx.x;
        kn[r] = k < n ? d.knext[k] : 0u;
        kp[r] = (k < n && P) ? P[k] : 0u;
    }
    uint32_t c = 0;
#pragma unroll
    for (int r = 0; r < RI; ++r) {
        const int64_t k = base + r * RT + threadIdx.x;
        if (k < n) {
            if (P) Pc[k] = kp[r];
            if (!P || kn[r] != kp[r]) {
                ++c;
                for (int p = 0; p < passes; ++p) atomicAdd(&h[p][(kn[r] >> (8 * p)) & 255u], 1u);
            }
        }
    }
    uint32_t ex;
    const uint32_t total = block_excl_scan(c, ex);
    if (threadIdx.x == 0) d.mcnt[lt] = total;
    uint32_t* mh = d.mctl + 16;
    for (int i = threadIdx.x; i < passes * 256; i += RT) {
        const uint32_t v = (&h[0][0])[i];
        if (v) atomicAdd(mh + i, v);
    }
}

__global__ void __launch_bounds__(RT) kb_moved_compact(const SortDesc* __restrict__ sd, const uint32_t* __restrict__ rt_sim,
                                                       const uint32_t* __restrict__ bsorted, int kpar)
{
    __shared__ uint32_t wc[RI][RW];
    const uint32_t sim = rt_sim[blockIdx.x];
    const SortDesc& d = sd[sim];
    const uint32_t t = blockIdx.x - d.rbase;
    const int64_t n = d.n;
    const uint32_t* P = bsorted[sim] ? d.kb[kpar ^ 1] : nullptr;   // the copy of the previous keys
    uint32_t part = 0;
    for (uint32_t i = threadIdx.x; i < t; i += RT) part += d.mcnt[i];
    uint32_t ex;
    const uint32_t excl = block_excl_scan(part, ex);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t base = (int64_t)t * RTILE;
    uint32_t key[RI];
    unsigned bal[RI];
#pragma unroll
    for (int r = 0; r < RI; ++r) {
        const int64_t k = base + r * RT + threadIdx.x;
        const bool moved = k < n && (!P || d.knext[k] != P[k]);
        key[r] = moved ? d.knext[k] : 0u;
        bal[r] = __ballot_sync(FULL, moved);
        if (lane == 0) wc[r][w] = (uint32_t)__popc(bal[r]);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t run = excl;
        for (int r = 0; r < RI; ++r)
            for (int ww = 0; ww < RW; ++ww) {
                const uint32_t cc = wc[r][ww];
                wc[r][ww] = run;
                run += cc;
            }
        d.choff[t] = excl;
        if (t + 1 == d.ntl) d.mctl[MCTL_M] = run;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RI; ++r) {
        if (bal[r] & (1u << lane)) {
            const int64_t k = base + r * RT + threadIdx.x;
            const uint32_t p = wc[r][w] + (uint32_t)__popc(bal[r] & lanemask_lt());
            d.mk[0][p] = key[r];
            d.mv[0][p] = (uint32_t)k;
            d.midx[p] = (uint32_t)k;
        }
    }
}

// one LSD pass over every member's changed keys; tiles are numbered across members and
// taken from a counter, each tile's look-back stops at its member's first tile
__global__ void __launch_bounds__(RT) kb_msort_pass(const SortDesc* __restrict__ sd, int nsims, int pass,
                                                    uint32_t* __restrict__ bctl, uint32_t* err)
{
    extern __shared__ uint32_t pre[];      // [nsims + 1]: first tile of each member
    __shared__ uint32_t wc[RW][256];
    __shared__ uint32_t goff[256];
    __shared__ uint32_t dst0[256];
    __shared__ uint32_t s_t;
    uint32_t carry = 0;
    for (int b0 = 0; b0 < nsims; b0 += RT) {
        const int i = b0 + threadIdx.x;
        const uint32_t v = i < nsims ? (sd[i].mctl[MCTL_M] + RTILE - 1) / RTILE : 0u;
        uint32_t ex;
        const uint32_t tot = block_excl_scan(v, ex);
        if (i < nsims) pre[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) pre[nsims] = carry;
    __syncthreads();
    const uint32_t total = pre[nsims];
    if (blockIdx.x >= total) return;
    const uint32_t epoch = bctl[0] + (uint32_t)pass;
    const int shift = 8 * pass;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int cur = -1;
    for (;;) {
        if (threadIdx.x == 0) s_t = atomicAdd(bctl + 1 + pass, 1u);
        for (int i = threadIdx.x; i < RW * 256; i += RT) (&wc[0][0])[i] = 0u;
        __syncthreads();
        const uint32_t t = s_t;
        if (t >= total) break;
        int lo = 0, hi = nsims - 1;   // last member with pre <= t
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (pre[mid] <= t) lo = mid;
            else hi = mid - 1;
        }
        const SortDesc& d = sd[lo];
        if (lo != cur) {   // uniform: the member's digit starts of this pass
            uint32_t ex;
            block_excl_scan(d.mctl[16 + pass * 256 + threadIdx.x], ex);
            dst0[threadIdx.x] = ex;
            cur = lo;
        }
        const uint32_t m = d.mctl[MCTL_M];
        const uint32_t lt = t - pre[lo];
        const uint32_t* kin = d.mk[pass & 1];
        const uint32_t* vin = d.mv[pass & 1];
        uint32_t* kout = d.mk[(pass + 1) & 1];
        uint32_t* vout = d.mv[(pass + 1) & 1];
        const int64_t base = (int64_t)lt * RTILE + w * (RI * 32);
        uint32_t key[RI], val[RI], lr[RI];
        unsigned dig[RI];
#pragma unroll
        for (int r = 0; r < RI; ++r) {
            const int64_t idx = base + r * 32 + lane;
            const bool valid = idx < (int64_t)m;
            key[r] = valid ? kin[idx] : 0u;
            val[r] = valid ? vin[idx] : 0u;
            const unsigned dg = valid ? (key[r] >> shift) & 255u : 256u;
            dig[r] = dg;
            const unsigned peers = __match_any_sync(FULL, dg);
            const unsigned before = (unsigned)__popc(peers & lanemask_lt());
            const uint32_t cnt = valid ? wc[w][dg] : 0u;
            __syncwarp();
            lr[r] = cnt + before;
            if (valid && lane == __ffs(peers) - 1) wc[w][dg] = cnt + (uint32_t)__popc(peers);
            __syncwarp();
        }
        __syncthreads();
        {
            const int dg = threadIdx.x;
            uint32_t run = 0;
            for (int ww = 0; ww < RW; ++ww) {
                const uint32_t c = wc[ww][dg];
                wc[ww][dg] = run;
                run += c;
            }
            goff[dg] = dst0[dg] + lookback64(d.lbs + dg, lt, 256, run, epoch, err);
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < RI; ++r) {
            const int64_t idx = base + r * 32 + lane;
            if (idx < (int64_t)m) {
                const unsigned dg = dig[r];
                const uint32_t pos = goff[dg] + wc[w][dg] + lr[r];
                if (pos < m) {
                    kout[pos] = key[r];
                    vout[pos] = val[r];
                } else {
                    atomicOr(err, APIC_ERRBIT_RANGE);
                }
            }
        }
        __syncthreads();
    }
}

// unchanged keys of every member chunk into place (members not yet sorted have none)
__global__ void __launch_bounds__(RT) kb_merge_u(const SortDesc* __restrict__ sd, const uint32_t* __restrict__ rt_sim,
                                                 const uint32_t* __restrict__ bsorted, int kpar, int passes,
                                                 uint32_t* err)
{
    __shared__ uint32_t wc[RI][RW];
    __shared__ uint32_t s_lo, s_hi;
    const uint32_t sim = rt_sim[blockIdx.x];
    if (!bsorted[sim]) return;
    const SortDesc& d = sd[sim];
    const uint32_t t = blockIdx.x - d.rbase;
    const int64_t n = d.n;
    const uint32_t* pk = d.kb[kpar ^ 1];
    const uint32_t* msk = d.mk[passes & 1];
    const uint32_t* msv = d.mv[passes & 1];
    const uint32_t m = d.mctl[MCTL_M];
    uint32_t* kout = d.kb[kpar];
    uint32_t* vout = d.vb[kpar];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t base = (int64_t)t * RTILE;
    const int64_t kl = (base + RTILE < n ? base + RTILE : n) - 1;
    if (threadIdx.x == 0) {
        s_lo = below_m(msk, msv, 0u, m, pk[base], (uint32_t)base);
        s_hi = below_m(msk, msv, s_lo, m, pk[kl], (uint32_t)kl + 1u);
    }
    unsigned bal[RI];
#pragma unroll
    for (int r = 0; r < RI; ++r) {
        const int64_t k = base + r * RT + threadIdx.x;
        const bool moved = k < n && d.knext[k] != pk[k];
        bal[r] = __ballot_sync(FULL, moved);
        if (lane == 0) wc[r][w] = (uint32_t)__popc(bal[r]);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t run = d.choff[t];
        for (int r = 0; r < RI; ++r)
            for (int ww = 0; ww < RW; ++ww) {
                const uint32_t c = wc[r][ww];
                wc[r][ww] = run;
                run += c;
            }
    }
    __syncthreads();
    const uint32_t lo = s_lo, hi = s_hi;
#pragma unroll
    for (int r = 0; r < RI; ++r) {
        const int64_t k = base + r * RT + threadIdx.x;
        if (k < n && !(bal[r] & (1u << lane))) {
            const uint32_t before = wc[r][w] + (uint32_t)__popc(bal[r] & lanemask_lt());
            const uint32_t key = pk[k];
            const uint32_t pos = (uint32_t)k - before + below_m(msk, msv, lo, hi, key, (uint32_t)k);
            if (pos < (uint32_t)n) {
                kout[pos] = key;
                vout[pos] = (uint32_t)k;
            } else {
                atomicOr(err, APIC_ERRBIT_RANGE);
            }
        }
    }
}

// changed keys of member blockIdx.y into place
__global__ void __launch_bounds__(RT) kb_merge_m(const SortDesc* __restrict__ sd, const uint32_t* __restrict__ bsorted,
                                                 int kpar, int passes, uint32_t* err)
{
    const uint32_t sim = blockIdx.y;
    const SortDesc& d = sd[sim];
    const bool sorted = bsorted[sim] != 0u;
    const uint32_t n = d.n, m = d.mctl[MCTL_M];
    const uint32_t* pk = d.kb[kpar ^ 1];
    const uint32_t* msk = d.mk[passes & 1];
    const uint32_t* msv = d.mv[passes & 1];
    uint32_t* kout = d.kb[kpar];
    uint32_t* vout = d.vb[kpar];
    for (uint32_t j = blockIdx.x * RT + threadIdx.x; j < m; j += gridDim.x * RT) {
        const uint32_t key = msk[j], idx = msv[j];
        uint32_t pos = j;
        if (sorted) {
            uint32_t lo = 0, hi = n;   // K = #k with (P[k], k) below (key, idx)
            while (lo < hi) {
                const uint32_t mid = (lo + hi) >> 1;
                const uint32_t a = pk[mid];
                if (a < key || (a == key && mid < idx)) lo = mid + 1;
                else hi = mid;
            }
            uint32_t a = 0, b = m;     // changed indices below K
            while (a < b) {
                const uint32_t mid = (a + b) >> 1;
                if (d.midx[mid] < lo) a = mid + 1;
                else b = mid;
            }
            pos = j + lo - a;
        }
        if (pos < n) {
            kout[pos] = key;
            vout[pos] = idx;
        } else {
            atomicOr(err, APIC_ERRBIT_RANGE);
        }
    }
}

__global__ void __launch_bounds__(256) kb_tile_count(const SortDesc* __restrict__ sd, const uint32_t* __restrict__ ch_sim,
                                                     int sh, int tile, int kpar, uint32_t* __restrict__ cnt)
{
    const SortDesc& d = sd[ch_sim[blockIdx.x]];
    const int64_t lc = (int64_t)blockIdx.x - d.cbase;
    const uint32_t tot = count_heads(d.kb[kpar], d.n, sh, tile, lc * tile);
    if (threadIdx.x == 0) cnt[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(256) kb_tile_write(const SortDesc* __restrict__ sd, const uint32_t* __restrict__ ch_sim,
                                                     int sh, int tile, int kpar, const uint32_t* __restrict__ off,
                                                     int64_t max_tiles, uint32_t* __restrict__ tile_sim,
                                                     uint32_t* __restrict__ tile_start, uint32_t* __restrict__ err,
                                                     uint32_t* __restrict__ tile_ctr)
{
    if (blockIdx.x == 0 && threadIdx.x < 2) tile_ctr[threadIdx.x] = 0u;
    const uint32_t sim = ch_sim[blockIdx.x];
    const SortDesc& d = sd[sim];
    const int64_t cs = ((int64_t)blockIdx.x - d.cbase) * tile;
    write_heads(d.kb[kpar], d.n, sh, tile, cs, off[blockIdx.x], [&](uint32_t pos, int64_t k) {
        if ((int64_t)pos < max_tiles) {
            tile_sim[pos] = sim;
            tile_start[pos] = (uint32_t)k;
        } else {
            atomicOr(err, APIC_ERRBIT_CAPACITY);
        }
    });
}

}  // namespace

int radix_tiles(int64_t n) { return (int)((n + RTILE - 1) / RTILE); }
size_t moved_bitmap_words(int64_t n) { return (size_t)radix_tiles(n) * (RTILE / 32); }

// kernels the routines below launch (memsets not counted), for the launch counters
int radix_sort_kernels(int key_bits) { return 2 + (key_bits + 7) / 8; }
int resort_kernels(int64_t n, int key_bits)
{
    if (n <= 0) return 0;
    return 4 + (key_bits + 7) / 8 + (radix_tiles(n) > kReduceChunks ? 3 : 0);
}
int build_tiles_kernels(int64_t n, int tile) { return (n + tile - 1) / tile <= kReduceChunks ? 2 : 5; }
int batch_sort_and_tiles_kernels(int passes) { return (5 + passes) + 5; }

size_t scan_partials_needed(int64_t n)
{
    const int64_t m = 256 * (int64_t)radix_tiles(n) + 1;
    const int64_t mm = m > n ? m : n;
    return (size_t)((mm + SCH - 1) / SCH + 1);
}

cudaError_t exclusive_scan(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* part, uint32_t* total,
                           cudaStream_t s)
{
    if (n <= 0) {
        if (total) return cudaMemsetAsync(total, 0, sizeof(uint32_t), s);
        return cudaSuccess;
    }
    const int64_t np = (n + SCH - 1) / SCH;
    cudaError_t e = launch_pdl(k_scan_reduce, dim3((unsigned)np), dim3(256), 0, s, in, n, part);
    if (e == cudaSuccess) e = launch_pdl(k_scan_top, dim3(1), dim3(256), 0, s, part, np, total);
    if (e == cudaSuccess) e = launch_pdl(k_scan_down, dim3((unsigned)np), dim3(256), 0, s, in, out, n, part);
    return e;
}

cudaError_t radix_sort(const Buffers& b, int64_t n, int key_bits, cudaStream_t s, uint32_t** keys_out,
                       uint32_t** vals_out)
{
    const int nt = radix_tiles(n);
    const int passes = (key_bits + 7) / 8;
    const uint32_t* kin = b.knext;
    const uint32_t* vin = nullptr;
    uint32_t* kb[2] = {b.kA, b.kB};
    uint32_t* vb[2] = {b.vA, b.vB};
    // one-sweep form: digit histograms of every pass in one read, then one kernel per pass
    // (scratch: radix_counts holds [passes][256] digit starts, then the look-back words)
    uint32_t* dstart = b.radix_counts;
    uint32_t* status = b.radix_counts + 4 * 256;
    cudaError_t e = cudaMemsetAsync(dstart, 0, sizeof(uint32_t) * 256 * passes, s);
    if (e != cudaSuccess) return e;
    int grid = nt < 1024 ? nt : 1024;
    k_onesweep_hist<<<grid > 0 ? grid : 1, 256, 0, s>>>(b.knext, n, passes, dstart);
    k_onesweep_digits<<<1, 256, 0, s>>>(dstart, passes);
    for (int p = 0; p < passes; ++p) {
        e = cudaMemsetAsync(status, 0, sizeof(uint32_t) * 256 * (size_t)nt, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(b.tile_ctr + 2, 0, sizeof(uint32_t), s);
        if (e != cudaSuccess) return e;
        k_onesweep_pass<<<nt, RT, 0, s>>>(kin, vin, kb[p & 1], vb[p & 1], n, 8 * p, dstart + 256 * p, status,
                                          b.tile_ctr + 2, b.err);
        kin = kb[p & 1];
        vin = vb[p & 1];
    }
    *keys_out = const_cast<uint32_t*>(kin);
    *vals_out = const_cast<uint32_t*>(vin);
    return cudaGetLastError();
}

cudaError_t resort(const Buffers& b, int64_t n, int key_bits, const uint32_t* pk, uint32_t* kout, uint32_t* vout,
                   uint32_t* epoch, int sms, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const int nchunks = radix_tiles(n);
    const int passes = (key_bits + 7) / 8;
    cudaError_t e;
    if (*epoch == 0u || *epoch > 0xfffffff0u) {   // first use, or the epoch is about to wrap
        e = cudaMemsetAsync(b.lbs, 0, sizeof(unsigned long long) * 256 * ((size_t)nchunks + 1), s);
        if (e != cudaSuccess) return e;
        *epoch = 1u;
    }
    // counters, m, digit counts
    static_assert(kMsortCtlBytes % 4 == 0, "the control block is zeroed as 32-bit words");
    e = launch_pdl(k_msort_reset, dim3(16), dim3(256), 0, s, b.mctl, (int)(kMsortCtlBytes / 4));
    if (e == cudaSuccess)
        e = launch_pdl(k_moved_count, dim3(nchunks), dim3(RT), 0, s, b.knext, pk, n, b.mcnt, b.mhist, passes, b.mbits);
    if (e != cudaSuccess) return e;
    const uint32_t* off = nullptr;
    if (nchunks > kReduceChunks) {   // many chunks: offsets by the device scan instead
        e = exclusive_scan(b.mcnt, b.choff, nchunks, b.scan_part, nullptr, s);
        if (e != cudaSuccess) return e;
        off = b.choff;
    }
    e = launch_pdl(k_moved_compact, dim3(nchunks), dim3(RT), 0, s, b.knext, pk, n, b.mcnt, off, nchunks, b.mctl,
                   b.mk[0], b.mv[0], b.choff, b.err, b.mbits);
    const int grid = nchunks < sms * 8 ? nchunks : sms * 8;
    for (int p = 0; p < passes && e == cudaSuccess; ++p)
        e = launch_pdl(k_msort_pass, dim3(grid), dim3(RT), 0, s, b.mk[p & 1], b.mv[p & 1], b.mk[(p + 1) & 1],
                       b.mv[(p + 1) & 1], b.mctl, p, b.mhist + 256 * p, b.lbs, (*epoch)++, b.err);
    if (e == cudaSuccess)
        e = launch_pdl(k_merge, dim3(nchunks), dim3(RT), 0, s, b.knext, pk, n, b.choff, b.mk[passes & 1],
                       b.mv[passes & 1], b.mctl, nchunks, kout, vout, b.err, b.mbits);
    return e;
}

cudaError_t batch_resort(const SortDesc* sd, const uint32_t* rt_sim, uint32_t total_rtiles, int nsims, int passes,
                         int kpar, const uint32_t* bsorted, uint32_t* bctl, uint32_t* err, int sms, cudaStream_t s)
{
    if (total_rtiles == 0 || nsims == 0) return cudaSuccess;
    if (nsims > 12000) return cudaErrorInvalidValue;   // grid y and the per-member prefix in shared memory
    kb_rs_init<<<nsims, 256, 0, s>>>(sd, bctl);
    kb_moved_count<<<total_rtiles, RT, 0, s>>>(sd, rt_sim, bsorted, kpar, passes);
    kb_moved_compact<<<total_rtiles, RT, 0, s>>>(sd, rt_sim, bsorted, kpar);
    const int grid = (int)total_rtiles < sms * 8 ? (int)total_rtiles : sms * 8;
    const size_t smem = sizeof(uint32_t) * ((size_t)nsims + 1);
    for (int p = 0; p < passes; ++p) kb_msort_pass<<<grid, RT, smem, s>>>(sd, nsims, p, bctl, err);
    kb_merge_u<<<total_rtiles, RT, 0, s>>>(sd, rt_sim, bsorted, kpar, passes, err);
    kb_merge_m<<<dim3(8, (unsigned)nsims), RT, 0, s>>>(sd, bsorted, kpar, passes, err);
    return cudaGetLastError();
}

cudaError_t batch_build_tiles(const SortDesc* sd, const uint32_t* ch_sim, uint32_t total_chunks, int dim, int tile,
                              int kpar, uint32_t* cnt, uint32_t* part, uint32_t* ntiles, int64_t max_tiles,
                              uint32_t* tile_sim, uint32_t* tile_start, uint32_t* err, uint32_t* tile_ctr, cudaStream_t s)
{
    const int sh = 2 * dim;
    kb_tile_count<<<total_chunks, 256, 0, s>>>(sd, ch_sim, sh, tile, kpar, cnt);
    cudaError_t e = exclusive_scan(cnt, cnt, total_chunks, part, ntiles, s);
    if (e != cudaSuccess) return e;
    kb_tile_write<<<total_chunks, 256, 0, s>>>(sd, ch_sim, sh, tile, kpar, cnt, max_tiles, tile_sim, tile_start, err,
                                               tile_ctr);
    return cudaGetLastError();
}

cudaError_t build_tiles(const Buffers& b, const uint32_t* skeys, int64_t n, int dim, int tile, int64_t max_tiles,
                        cudaStream_t s)
{
    const int64_t nchunks = (n + tile - 1) / tile;
    const int sh = 2 * dim;
    cudaError_t e = launch_pdl(k_tile_count, dim3((unsigned)nchunks), dim3(256), 0, s, skeys, n, sh, tile, b.chunk_cnt);
    if (e != cudaSuccess) return e;
    if (nchunks <= kReduceChunks)
        return launch_pdl(k_tile_write, dim3((unsigned)nchunks), dim3(256), 0, s, skeys, n, sh, tile, nullptr, b.ntiles,
                          max_tiles, b.tiles, (int)nchunks, b.err, b.tile_ctr, b.chunk_cnt);
    e = exclusive_scan(b.chunk_cnt, b.chunk_cnt, nchunks, b.scan_part, b.ntiles, s);
    if (e != cudaSuccess) return e;
    return launch_pdl(k_tile_write, dim3((unsigned)nchunks), dim3(256), 0, s, skeys, n, sh, tile, b.chunk_cnt, b.ntiles,
                      max_tiles, b.tiles, (int)nchunks, b.err, b.tile_ctr, nullptr);
}

}  // namespace apic

// ---------------------------------------------------------------- sort without allocation
// apic_sort_keys_noalloc: a plain LSD radix sort (per 8-bit digit: a histogram pass, a
// device-wide exclusive scan and a stable scatter), with all scratch in one static device array.
namespace apic {
namespace {

constexpr int64_t kNoAllocMaxKeys = APIC_SORT_NOALLOC_MAX_KEYS;
constexpr int64_t kNoAllocTiles = (kNoAllocMaxKeys + RTILE - 1) / RTILE;
constexpr int64_t kNoAllocParts = (256 * kNoAllocTiles + 1 + SCH - 1) / SCH + 1;
// words: ping-pong keys, ping-pong indices, digit counts, scan partials
constexpr int64_t kNoAllocWords = 2 * kNoAllocMaxKeys + 256 * kNoAllocTiles + kNoAllocParts;

static __device__ __align__(256) uint32_t g_sort_scratch[kNoAllocWords];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
uint32_t* g_scratch_ptr[kMaxDevices] = {};

// device address of g_sort_scratch on the current device (looked up once per device)
cudaError_t noalloc_scratch(uint32_t** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_sort_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = static_cast<uint32_t*>(p);
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace apic

namespace {
// [a, a + n) and [b, b + n) share a word
bool overlaps(const uint32_t* a, const uint32_t* b, int64_t n)
{
    const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b, len = (uintptr_t)n * sizeof(uint32_t);
    return x < y + len && y < x + len;
}
}  // namespace

extern "C" apic_status apic_sort_keys_noalloc(const uint32_t* keys, int64_t n, int key_bits, uint32_t* sorted_keys,
                                              uint32_t* perm, void* stream)
{
    using namespace apic;
    if (n < 0 || key_bits < 1 || key_bits > 32) return APIC_ERR_ARG;
    if (n > kNoAllocMaxKeys) return APIC_ERR_OOM;
    if (n == 0) return APIC_OK;
    if (!keys || !sorted_keys || !perm) return APIC_ERR_ARG;
    // a pass reads keys while other CTAs already write its output: the buffers must be apart
    if (overlaps(keys, sorted_keys, n) || overlaps(keys, perm, n) || overlaps(sorted_keys, perm, n))
        return APIC_ERR_ARG;
    // an error left pending by earlier work on this thread is not this call's: leave it
    // in place for its owner and launch nothing
    if (cudaPeekAtLastError() != cudaSuccess) return APIC_ERR_CUDA;
    uint32_t* scratch = nullptr;
    if (noalloc_scratch(&scratch) != cudaSuccess) return APIC_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t* tmp_keys = scratch;
    uint32_t* tmp_vals = tmp_keys + kNoAllocMaxKeys;
    uint32_t* counts = tmp_vals + kNoAllocMaxKeys;
    uint32_t* part = counts + 256 * kNoAllocTiles;
    const int nt = radix_tiles(n);
    const int passes = (key_bits + 7) / 8;
    const uint32_t* kin = keys;
    const uint32_t* vin = nullptr;   // identity indices on the first pass
    for (int p = 0; p < passes; ++p) {
        // the last pass lands in the caller's outputs; earlier ones alternate with scratch
        const bool to_out = ((passes - 1 - p) % 2) == 0;
        uint32_t* kout = to_out ? sorted_keys : tmp_keys;
        uint32_t* vout = to_out ? perm : tmp_vals;
        const int shift = 8 * p;
        k_radix_hist<<<nt, RT, 0, s>>>(kin, n, shift, nt, counts);
        if (cudaGetLastError() != cudaSuccess) return APIC_ERR_CUDA;
        if (exclusive_scan(counts, counts, 256 * (int64_t)nt, part, nullptr, s) != cudaSuccess) return APIC_ERR_CUDA;
        k_radix_scatter<<<nt, RT, 0, s>>>(kin, vin, kout, vout, n, shift, nt, counts);
        if (cudaGetLastError() != cudaSuccess) return APIC_ERR_CUDA;
        kin = kout;
        vin = vout;
    }
    return APIC_OK;
}
