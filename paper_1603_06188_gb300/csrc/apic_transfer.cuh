// apic_transfer.cuh -- the per-step kernels of the APIC / explicit MPM method
// (arXiv:1603.06188), templated on dimension D, B-spline order and real type R:
//   k_keys         cell keys of the current particle order
//   k_p2g_cells    Sec. 3.2 transfer to grid + Sec. 3.3 force, per-cell register sums and a
//                  deterministic gather per node block
//   k_grid_update  Sec. 3.3 explicit (lambda = 0) grid update
//   k_g2p          Sec. 3.4 transfer to particles (lambda = 0 form of Sec. 5.7), grid blocks
//                  staged in shared memory by bulk asynchronous copies (TMA engine)
//   k_mom_*        Sec. 3.1 / 5.3 total momentum, FP64 accumulation
// plus upload / download / dense-grid conversion kernels.  Included by apic_transfer_f32.cu
// and apic_transfer_f64.cu, which instantiate it for one real type each.
#pragma once

#include <algorithm>

#include "apic_device.cuh"

namespace apic {

constexpr unsigned FULLMASK = 0xffffffffu;
constexpr int TPB = 256;

template <typename R> struct HostToDev {
    static DevCfg<R> make(const HostCfg& h, int64_t n)
    {
        DevCfg<R> c;
        for (int a = 0; a < 3; ++a) {
            c.res[a] = h.res[a];
            c.nb[a] = h.nb[a];
            c.origin[a] = (R)h.origin[a];
            c.gravity[a] = (R)h.gravity[a];
        }
        c.dx = (R)h.dx;
        c.inv_dx = (R)(1.0 / h.dx);
        c.dt = (R)h.dt;
        c.boundary = h.boundary;
        c.wall = h.wall;
        c.model = h.model;
        c.mat = h.mat;
        c.transfer = h.transfer;
        c.mu = (R)h.mu;
        c.lam = (R)h.lam;
        c.mass = (R)h.mass;
        c.vol = (R)h.vol;
        const double kappa = h.order == 2 ? 0.25 : 1.0 / 3.0;
        c.inv_kdx = (R)(1.0 / (kappa * h.dx));
        c.n = (int)n;
        c.nblocks = h.nblocks;
        c.dtp = nullptr;
        c.smax = nullptr;
        c.cfl_coef = (R)(6.0 * sqrt((double)h.dim) / h.dx);
        c.flip_alpha = (R)h.flip_alpha;
        c.wait_limit = h.wait_limit;
        return c;
    }
    // the per-simulation words of adaptive stepping: the time step and the fused speed
    // maximum (plain steps use neither)
    static DevCfg<R> make(const HostCfg& h, const Buffers& b, int64_t n)
    {
        DevCfg<R> c = make(h, n);
        c.dtp = h.adaptive ? (const R*)b.dt_word : nullptr;
        c.smax = h.adaptive ? b.smax_word : nullptr;
        return c;
    }
};

template <typename R> PState<R> state_of(const Buffers& b, int which)
{
    PState<R> s;
    s.A = (V4<R>*)b.st[which][0];
    s.V = (V4<R>*)b.st[which][1];
    s.Ba = (V4<R>*)b.st[which][2];
    s.Bb = (V4<R>*)b.st[which][3];
    s.Fa = (V4<R>*)b.st[which][4];
    s.Fb = (V4<R>*)b.st[which][5];
    s.Fc = (V2<R>*)b.st[which][6];
    s.Ta = (V4<R>*)b.st[which][7];
    s.Tb = (V2<R>*)b.st[which][8];
    s.M = (V4<R>*)b.st[which][9];
    return s;
}

// ---------------------------------------------------------------- stencil base + key
// Per-axis base node (clamped into the grid; a clamp latches APIC_ERRBIT_RANGE), its
// fractional position fx = u - base and the 1-D weights.
template <int D, int ORDER, typename R>
__device__ __forceinline__ bool particle_stencil(const R* o, const int* cell, const DevCfg<R>& c, int* base, R* fx,
                                                 R (*w)[ORDER + 1], R (*dw)[ORDER + 1])
{
    bool ok = true;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        axis_weights<ORDER, R>(o[a], cell[a], base[a], fx[a], w[a], dw[a]);
        if (base[a] < 0 || base[a] + ORDER > c.res[a] - 1) {
            ok = false;
            base[a] = base[a] < 0 ? 0 : c.res[a] - 1 - ORDER;
        }
    }
    return ok;
}

template <int D, int ORDER, typename R>
__device__ __forceinline__ uint32_t key_of(const R* o, const int* cell, const DevCfg<R>& c, uint32_t* err)
{
    int base[D];
    bool ok = true;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        int b = (ORDER == 2) ? (o[a] >= R(0.5) ? cell[a] : cell[a] - 1) : cell[a] - 1;
        if (b < 0 || b + ORDER > c.res[a] - 1) {
            ok = false;
            b = b < 0 ? 0 : c.res[a] - 1 - ORDER;
        }
        base[a] = b;
    }
    if (!ok) set_err(err, APIC_ERRBIT_RANGE);
    if (D == 3) {
        const uint32_t blk = ((uint32_t)(base[2] >> 2) * c.nb[1] + (uint32_t)(base[1] >> 2)) * c.nb[0] + (uint32_t)(base[0] >> 2);
        const uint32_t in = ((uint32_t)(base[2] & 3) << 4) | ((uint32_t)(base[1] & 3) << 2) | (uint32_t)(base[0] & 3);
        return (blk << 6) | in;
    }
    const uint32_t blk = (uint32_t)(base[1] >> 2) * c.nb[0] + (uint32_t)(base[0] >> 2);
    return (blk << 4) | ((uint32_t)(base[1] & 3) << 2) | (uint32_t)(base[0] & 3);
}

template <int D, typename R> __device__ __forceinline__ void block_coords(uint32_t blk, const DevCfg<R>& c, int* b)
{
    b[0] = (int)(blk % (uint32_t)c.nb[0]);
    if (D == 3) {
        b[1] = (int)((blk / (uint32_t)c.nb[0]) % (uint32_t)c.nb[1]);
        b[2] = (int)(blk / ((uint32_t)c.nb[0] * (uint32_t)c.nb[1]));
    } else {
        b[1] = (int)(blk / (uint32_t)c.nb[0]);
    }
}

template <int D, int ORDER, typename R>
__global__ void __launch_bounds__(TPB) k_keys(PState<R> st, DevCfg<R> c, uint32_t* __restrict__ keys, uint32_t* err)
{
    const int k = blockIdx.x * TPB + threadIdx.x;
    if (k >= c.n) return;
    Particle<D, R> p;
    load_x<D, R>(st, k, p);
    keys[k] = key_of<D, ORDER, R>(p.o, p.cell, c, err);
}

// ---------------------------------------------------------------- asynchronous particle staging
// A particle's packed state copied global -> shared with cp.async (16-byte pieces; the 8-byte
// Fc group of the FP32 layout with an 8-byte copy), so loads of the next particles overlap
// the arithmetic of the current one without holding them in registers.
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void cp_async16(void* dst, const void* src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// slot of packed state, in units of R: 3-D A V Ba Bb Ta Tb (m_p V_p) = 24, 2-D A V Ba Tb (m_p V_p)
// = 16; the last two words hold the particle's mass and volume when parameters per particle
// are set
template <int D> __host__ __device__ constexpr int slot_words() { return D == 3 ? 24 : 16; }
template <int D> __host__ __device__ constexpr int slot_mass_word() { return D == 3 ? 22 : 14; }

// the (m_p, V_p) half of a particle's parameter lane
template <typename R> __device__ __forceinline__ const V2<R>* mass_half(const PState<R>& s, uint32_t q)
{
    return reinterpret_cast<const V2<R>*>(s.M + q) + 1;
}

template <typename R> __device__ __forceinline__ void cp_group4(R* dst, const V4<R>* src)
{
    if (sizeof(R) == 4) {
        cp_async16(dst, src);
    } else {
        cp_async16(dst, src);
        cp_async16(dst + 2, reinterpret_cast<const R*>(src) + 2);
    }
}
template <typename R> __device__ __forceinline__ void cp_group2(R* dst, const V2<R>* src)
{
    if (sizeof(R) == 4) cp_async8(dst, src);
    else cp_async16(dst, src);
}

// what P2G reads of particle q: position, v, B, (with a stress model) tau and (with
// parameters per particle) its mass
template <int D, typename R>
__device__ __forceinline__ void stage_particle(R* slot, const PState<R>& s, uint32_t q, bool with_tau, bool mat)
{
    if (mat) cp_group2<R>(slot + slot_mass_word<D>(), mass_half(s, q));
    cp_group4<R>(slot + 0, s.A + q);
    cp_group4<R>(slot + 4, s.V + q);
    cp_group4<R>(slot + 8, s.Ba + q);
    if (D == 3) {
        cp_group4<R>(slot + 12, s.Bb + q);
        if (with_tau) {
            cp_group4<R>(slot + 16, s.Ta + q);
            cp_group2<R>(slot + 20, s.Tb + q);
        }
    } else {
        if (with_tau) cp_group2<R>(slot + 12, s.Tb + q);
    }
}

template <int D, typename R>
__device__ __forceinline__ void read_staged(const R* slot, Particle<D, R>& p, bool with_tau, bool mat)
{
    if (mat) p.pm = slot[slot_mass_word<D>()];
    const V4<R> a = *reinterpret_cast<const V4<R>*>(slot + 0);
    const V4<R> v = *reinterpret_cast<const V4<R>*>(slot + 4);
    const V4<R> ba = *reinterpret_cast<const V4<R>*>(slot + 8);
    if (D == 3) {
        const V4<R> bb = *reinterpret_cast<const V4<R>*>(slot + 12);
        p.o[0] = a.x; p.o[1] = a.y; p.o[2] = a.z;
        unpack_cell<D>(r2u(a.w), p.cell);
        p.v[0] = v.x; p.v[1] = v.y; p.v[2] = v.z;
        p.B[0] = v.w; p.B[1] = ba.x; p.B[2] = ba.y; p.B[3] = ba.z; p.B[4] = ba.w;
        p.B[5] = bb.x; p.B[6] = bb.y; p.B[7] = bb.z; p.B[8] = bb.w;
        if (with_tau) {
            const V4<R> ta = *reinterpret_cast<const V4<R>*>(slot + 16);
            const V2<R> tb = *reinterpret_cast<const V2<R>*>(slot + 20);
            p.tau[0] = ta.x; p.tau[1] = ta.y; p.tau[2] = ta.z; p.tau[3] = ta.w;
            p.tau[4] = tb.x; p.tau[5] = tb.y;
        }
    } else {
        p.o[0] = a.x; p.o[1] = a.y;
        unpack_cell<D>(r2u(a.z), p.cell);
        p.id = r2u(a.w);
        p.v[0] = v.x; p.v[1] = v.y;
        p.B[0] = v.z; p.B[1] = v.w; p.B[2] = ba.x; p.B[3] = ba.y;
        if (with_tau) {
            const V2<R> tb = *reinterpret_cast<const V2<R>*>(slot + 12);
            p.tau[0] = ba.z; p.tau[1] = ba.w; p.tau[2] = tb.x;
        }
    }
}

// staging depth (particles in flight per lane) of the cell-parallel P2G
template <typename R> __host__ __device__ constexpr int p2g_slots() { return 2; }

// the per-cell stencil sums of a tile, one row per base cell: rows are padded by 16 bytes
// when their length in 4-byte words is a multiple of 8, so that the rows read by 8 lanes at
// once (consecutive cells, the same stencil entry) start in different bank groups
template <int D, int ORDER, typename R> __host__ __device__ constexpr int p2g_cell_stride()
{
    constexpr int nval = ((D == 3) ? (ORDER + 1) * (ORDER + 1) * (ORDER + 1) : (ORDER + 1) * (ORDER + 1)) * (D + 1);
    constexpr int words = nval * (int)(sizeof(R) / 4);
    return (words % 8 == 0) ? nval + 16 / (int)sizeof(R) : nval;
}
template <int D, int ORDER, typename R> __host__ __device__ constexpr size_t p2g_cellsum_bytes()
{
    return (size_t)((D == 3) ? 64 : 16) * p2g_cell_stride<D, ORDER, R>() * sizeof(R);
}
// dynamic shared memory of the cell-parallel P2G: per-cell sums, then the staging slots
template <int D, int ORDER, typename R> __host__ __device__ constexpr size_t p2g_cells_smem()
{
    return (p2g_cellsum_bytes<D, ORDER, R>() + 31) / 32 * 32 + (size_t)p2g_slots<R>() * 128 * slot_words<D>() * sizeof(R);
}
// FP32 single-simulation P2G copies the next tile's keys (up to 4096) into shared memory
template <typename R> __host__ __device__ constexpr bool p2g_key_prefetch() { return sizeof(R) == 4; }
template <int D, int ORDER, typename R> __host__ __device__ constexpr size_t p2g_cells_launch_smem()
{
    return p2g_cells_smem<D, ORDER, R>() + (p2g_key_prefetch<R>() ? (size_t)4096 * 4 : 0);
}

// ---------------------------------------------------------------- P2G, cell-parallel
// Butterfly reduce-scatter of N register values over a group of lanes: at distance H the
// lane with bit H set keeps the upper half of its values and receives its partner's upper
// half, the other keeps the lower half; after log2(G) steps each lane holds the group's
// full sums of about N/G of the values.  (off, cnt) track which original indices a lane's
// first positions hold.
template <typename R, int N, int H>
__device__ __forceinline__ void bfly_step(R* cur, unsigned mask, bool upper)
{
    constexpr int HALF = (N + 1) / 2;
#pragma unroll
    for (int i = 0; i < HALF; ++i) {
        const R lo = cur[i];
        const R hi = (i + HALF < N) ? cur[i + HALF] : R(0);
        const R send = upper ? lo : hi;
        const R keep = upper ? hi : lo;
        cur[i] = keep + __shfl_xor_sync(mask, send, H);
    }
}

template <typename R, int N, int G> struct ReduceScatter {
    static constexpr int FINAL = ReduceScatter<R, (N + 1) / 2, G / 2>::FINAL;
    static __device__ __forceinline__ void run(R* cur, unsigned mask, int lig, int& off, int& cnt)
    {
        constexpr int H = G / 2;
        constexpr int HALF = (N + 1) / 2;
        const bool upper = (lig & H) != 0;
        bfly_step<R, N, H>(cur, mask, upper);
        if (upper) {
            off += HALF;
            cnt = cnt > HALF ? cnt - HALF : 0;
        } else {
            cnt = cnt < HALF ? cnt : HALF;
        }
        ReduceScatter<R, HALF, G / 2>::run(cur, mask, lig, off, cnt);
    }
};
template <typename R, int N> struct ReduceScatter<R, N, 1> {
    static constexpr int FINAL = N;
    static __device__ __forceinline__ void run(R*, unsigned, int, int&, int&) {}
};

// One CTA takes tiles from a shared counter.  In a tile (sorted particles of one node
// block) every in-block base cell's particles are a contiguous run; a group of G lanes
// takes cells from a shared-memory counter, each lane summing the full (ORDER+1)^D-node
// stencil of its particles in registers (lanes stride the run by G, so a group's loads
// are contiguous).  The group's sums are combined by the butterfly reduce-scatter and
// stored (plain stores, no atomics) as that cell's stencil sums; then every tile node
// gathers, in a fixed order, the sums of the cells whose stencils cover it, and adds the
// result to the global grid.  Contributions as in k_p2g.
// runs of equal base cell inside a tile (sorted keys of one node block): cbeg / cend per
// in-block cell (whole CTA of nt threads; the caller synchronises afterwards)
template <int D>
__device__ __forceinline__ void tile_cell_runs(const uint32_t* __restrict__ tk, uint32_t start, uint32_t end,
                                               uint32_t* cbeg, uint32_t* cend, int nt)
{
    constexpr int NC = (D == 3) ? 64 : 16;
    // U keys per thread and their neighbours are requested before any is used, so a tile
    // waits for one load latency instead of one per key
    constexpr int U = 8;
    for (uint32_t k0 = start; k0 < end; k0 += (uint32_t)nt * U) {
        uint32_t kc[U], kp[U], kn[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t k = k0 + threadIdx.x + (uint32_t)(u * nt);
            kc[u] = kp[u] = kn[u] = 0u;
            if (k < end) {
                kc[u] = tk[k - start];
                if (k > start) kp[u] = tk[k - start - 1];
                if (k + 1 < end) kn[u] = tk[k - start + 1];
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t k = k0 + threadIdx.x + (uint32_t)(u * nt);
            if (k < end) {
                const uint32_t cl = kc[u] & (NC - 1);
                if (k == start || (kp[u] & (NC - 1)) != cl) cbeg[cl] = k;
                if (k + 1 == end || (kn[u] & (NC - 1)) != cl) cend[cl] = k + 1;
            }
        }
    }
}

// The tile's occupied base cells as a bit mask, written to occ[0..1] by two whole warps (a
// cell test is then a shift instead of two shared-memory loads; most tests of a sparse tile
// fail).  The caller synchronises before reading it.
template <int D>
__device__ __forceinline__ void tile_occupancy(const uint32_t* cbeg, const uint32_t* cend, uint32_t* occ)
{
    if (threadIdx.x < 64) {
        const bool o = threadIdx.x < ((D == 3) ? 64 : 16) && cbeg[threadIdx.x] < cend[threadIdx.x];
        const unsigned bits = __ballot_sync(0xffffffffu, o);
        if ((threadIdx.x & 31) == 0) occ[threadIdx.x >> 5] = bits;
    }
}

// The tile's nodes from the per-cell stencil sums cellsum[cell][node j][lane v]: node n
// collects, in a fixed order, the sums of the occupied cells n - (a, b, c) whose stencils
// cover it, and adds them to the global grid once; then the 2^D node blocks the tile
// reaches are flagged active.  Whole CTA of nt threads, after a barrier that follows the
// sums.
template <int D, int ORDER, typename R>
__device__ __forceinline__ void tile_flush_nodes(const R* cellsum, uint64_t occ, const int* bo, uint32_t blk,
                                                 R* __restrict__ acc, uint32_t* __restrict__ flags,
                                                 const DevCfg<R>& c, int nt)
{
    constexpr int K = ORDER + 1;
    constexpr int TE = 4 + ORDER;
    constexpr int TN = (D == 3) ? TE * TE * TE : TE * TE;
    constexpr int NS = (D == 3) ? K * K * K : K * K;
    constexpr int NV = D + 1;
    // Cell n - (a, b, c) is linear index L - dj with L = n0 + 4 n1 + 16 n2 and dj = a + 4 b +
    // 16 c.  Per node the occupancy word is shifted so that the cell of stencil offset j sits
    // at the fixed bit DM - dj, and masked with the offsets whose cell lies in the block
    // (built from per-axis masks: bit K-1-a set when 0 <= n - a <= 3), so each of the NS
    // candidates costs one constant bit test.
    constexpr int DM = (K - 1) * ((D == 3) ? 21 : 5);
    constexpr unsigned KM = (1u << K) - 1u;
    // reversed valid-offset masks of the TE node positions of an axis, K bits each
    constexpr unsigned long long RA = [] {
        unsigned long long r = 0;
        for (int n = 0; n < TE; ++n) {
            unsigned m = 0;
            for (int a = 0; a < K; ++a)
                if (n - a >= 0 && n - a <= 3) m |= 1u << (K - 1 - a);
            r |= (unsigned long long)m << (K * n);
        }
        return r;
    }();
    for (int i = threadIdx.x; i < TN; i += nt) {
        const int n0 = i % TE, n1 = (i / TE) % TE, n2 = (D == 3) ? i / (TE * TE) : 0;
        const int L = n0 + 4 * n1 + 16 * n2;
        uint64_t t = (L >= DM) ? (occ >> (L - DM)) : (occ << (DM - L));
        {
            const uint64_t ra = (RA >> (K * n0)) & KM;
            const unsigned rb = (unsigned)(RA >> (K * n1)) & KM;
            uint64_t y = 0;
#pragma unroll
            for (int b = 0; b < K; ++b)
                if ((rb >> b) & 1u) y |= ra << (4 * b);
            if (D == 3) {
                const unsigned rc = (unsigned)(RA >> (K * n2)) & KM;
                uint64_t z = 0;
#pragma unroll
                for (int c3 = 0; c3 < K; ++c3)
                    if ((rc >> c3) & 1u) z |= y << (16 * c3);
                t &= z;
            } else {
                t &= y;
            }
        }
        const int cl0 = L;
        R sum[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) sum[v] = R(0);
#pragma unroll
        for (int j = 0; j < NS; ++j) {
            const int ia = j % K, ib = (j / K) % K, ic = j / (K * K);
            const int dj = ia + 4 * ib + 16 * ic;
            if (!((t >> (DM - dj)) & 1ull)) continue;
            const R* src = cellsum + (size_t)(cl0 - dj) * p2g_cell_stride<D, ORDER, R>() + j * NV;
#pragma unroll
            for (int v = 0; v < NV; ++v) sum[v] += src[v];
        }
        if (sum[D] == R(0)) continue;
        int g[3];
        g[0] = bo[0] + n0;
        g[1] = bo[1] + n1;
        g[2] = bo[2] + n2;
        const uint32_t ni = node_index<D>(g, c.nb);
        R* gdst = acc + 4 * (size_t)ni;
#pragma unroll
        for (int a = 0; a < D; ++a) atomicAdd(gdst + a, sum[a]);
        atomicAdd(gdst + 3, sum[D]);
    }
    if (threadIdx.x < (1 << D)) {
        int bb[3];
        block_coords<D, R>(blk, c, bb);
        bool in = true;
#pragma unroll
        for (int a = 0; a < D; ++a) {
            bb[a] += (threadIdx.x >> a) & 1;
            if (bb[a] >= c.nb[a]) in = false;
        }
        if (in) {
            const uint32_t b2 = (D == 3) ? ((uint32_t)bb[2] * c.nb[1] + bb[1]) * c.nb[0] + bb[0]
                                         : (uint32_t)bb[1] * c.nb[0] + bb[0];
            flags[b2] = 1u;
        }
    }
}

// occupancy, then the nodes (whole CTA, after a barrier that follows the sums)
template <int D, int ORDER, typename R>
__device__ __forceinline__ void tile_flush(const R* cellsum, const uint32_t* cbeg, const uint32_t* cend, const int* bo,
                                           uint32_t blk, R* __restrict__ acc, uint32_t* __restrict__ flags,
                                           const DevCfg<R>& c, int nt)
{
    __shared__ uint32_t s_occ[2];
    tile_occupancy<D>(cbeg, cend, s_occ);
    __syncthreads();
    const uint64_t occ = (uint64_t)s_occ[0] | ((uint64_t)s_occ[1] << 32);
    tile_flush_nodes<D, ORDER, R>(cellsum, occ, bo, blk, acc, flags, c, nt);
}

// two FP32 fused multiply-adds in one packed instruction (c0 += a0 b0, c1 += a1 b1), each
// rounded as a scalar fmaf; the FP64 form is two scalar fmas
template <typename R> __device__ __forceinline__ void fma_pair(R& c0, R& c1, R a0, R a1, R b0, R b1)
{
    c0 = fma(a0, b0, c0);
    c1 = fma(a1, b1, c1);
}
template <> __device__ __forceinline__ void fma_pair<float>(float& c0, float& c1, float a0, float a1, float b0, float b1)
{
    asm("{\n\t.reg .b64 pa, pb, pc;\n\tmov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\tmov.b64 pc, {%0, %1};\n\t"
        "fma.rn.f32x2 pc, pa, pb, pc;\n\tmov.b64 {%0, %1}, pc;\n\t}"
        : "+f"(c0), "+f"(c1)
        : "f"(a0), "f"(a1), "f"(b0), "f"(b1));
}

// two FP32 products in one packed instruction (d0 = a0 b0, d1 = a1 b1), each rounded as a
// scalar multiply; the FP64 form is two scalar products
template <typename R> __device__ __forceinline__ void mul_pair(R& d0, R& d1, R a0, R a1, R b0, R b1)
{
    d0 = a0 * b0;
    d1 = a1 * b1;
}
template <> __device__ __forceinline__ void mul_pair<float>(float& d0, float& d1, float a0, float a1, float b0, float b1)
{
    asm("{\n\t.reg .b64 pa, pb, pd;\n\tmov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
        "mul.rn.f32x2 pd, pa, pb;\n\tmov.b64 {%0, %1}, pd;\n\t}"
        : "=f"(d0), "=f"(d1)
        : "f"(a0), "f"(a1), "f"(b0), "f"(b1));
}

// One particle's stencil sums added to a lane's registers cur (the z-slab SLAB of the
// stencil for 3-D cubic).  A lane past its cell's run (live false) carries a neutral
// particle: an in-cell position and zero state, so its weights are finite and it adds
// zeros.  A particle outside the tile's reach sets the range error and adds nothing.
template <int D, int ORDER, typename R, int KZ, int SLAB>
__device__ __forceinline__ void p2g_cells_particle(Particle<D, R>& p, bool live, const int* lb, const int* bo,
                                                   const DevCfg<R>& c, uint32_t* err, R m, R sC, R dt_dx,
                                                   bool with_tau, R* cur)
{
    constexpr int K = ORDER + 1;
    constexpr int NV = D + 1;
    if (!live) {   // neutral: zero state (the weights below are those of an in-cell point)
#pragma unroll
        for (int a = 0; a < D; ++a) p.v[a] = R(0);
#pragma unroll
        for (int i = 0; i < D * D; ++i) p.B[i] = R(0);
#pragma unroll
        for (int i = 0; i < ((D == 3) ? 6 : 3); ++i) p.tau[i] = R(0);
    }
    // The stencil base of the lane's cell is known (bo + lb), so only the particle's distance
    // from it is needed: fx = o + (cell - base), with cell - base = 1 - [o >= 1/2] (quadratic)
    // or 1 (cubic) exactly when the particle's own base is that node (as axis_weights
    // decides); a particle outside its run's cell is reported and adds nothing
    R w[D][K], dw[D][K], fx[D];
    bool ok = true;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        const int d = p.cell[a] - (bo[a] + lb[a]);
        ok = ok && (d == ((ORDER == 2) ? (p.o[a] >= R(0.5) ? 0 : 1) : 1));
        fx[a] = live ? p.o[a] + R(d) : ((ORDER == 2) ? R(1) : R(1.5));
        axis_weights_fx<ORDER, R>(fx[a], w[a], dw[a]);
    }
    if (live && !ok) {
        set_err(err, APIC_ERRBIT_RANGE);
        live = false;
    }
    const R ml = live ? m : R(0);
    R mv[D], mC[D * D], T[D * D];   // T = -dt/dx tau
#pragma unroll
    for (int a = 0; a < D; ++a) mv[a] = ml * p.v[a];
#pragma unroll
    for (int i = 0; i < D * D; ++i) mC[i] = (live ? sC : R(0)) * p.B[i];
    if (with_tau) {
        R tau[D * D];
        tau_full<D, R>(p.tau, tau);
#pragma unroll
        for (int i = 0; i < D * D; ++i) T[i] = (live ? -dt_dx : R(0)) * tau[i];
    } else {
#pragma unroll
        for (int i = 0; i < D * D; ++i) T[i] = R(0);
    }
    // The weights are tensor products, so the contributions separate axis by axis
    // (r = node - fx in grid units, T = -dt/dx tau, mC = m B D^{-1} dx):
    //   dp_c(i,j,k) = w0_i P_c(j,k) + E_c(i) S(j,k),       mass = w0_i m S(j,k)
    //   P_c(j,k) = w1_j Q_c(k) + H_c(j) w2_k,              S(j,k) = w1_j w2_k
    //   Q_c(k) = m v_c w2_k + mC_c2 (r w)2_k + T_c2 dw2_k
    //   H_c(j) = mC_c1 (r w)1_j + T_c1 dw1_j,  E_c(i) = mC_c0 (r w)0_i + T_c0 dw0_i
    // which is w m (v + C (x_i - x_p)) - dt tau grad w summed in fewer operations; the
    // factors are formed two at a time in packed pairs (components 0 and 1 together, and
    // component 2 of E with that of H)
    if (D == 3) {
        R E[3][K], H[3][K], mw0[K];
#pragma unroll
        for (int i = 0; i < K; ++i) mw0[i] = ml * w[0][i];
#pragma unroll
        for (int i = 0; i < K; ++i) {
            const R rw0 = (R(i) - fx[0]) * w[0][i], rw1 = (R(i) - fx[1]) * w[1][i];
            mul_pair<R>(E[0][i], E[1][i], mC[0], mC[3], rw0, rw0);
            fma_pair<R>(E[0][i], E[1][i], T[0], T[3], dw[0][i], dw[0][i]);
            mul_pair<R>(H[0][i], H[1][i], mC[1], mC[4], rw1, rw1);
            fma_pair<R>(H[0][i], H[1][i], T[1], T[4], dw[1][i], dw[1][i]);
            mul_pair<R>(E[2][i], H[2][i], mC[6], mC[7], rw0, rw1);
            fma_pair<R>(E[2][i], H[2][i], T[6], T[7], dw[0][i], dw[1][i]);
        }
#pragma unroll
        for (int icl = 0; icl < KZ; ++icl) {
            const int ic = SLAB * KZ + icl;
            const R w2 = w[2][ic], dw2 = dw[2][ic], rw2 = (R(ic) - fx[2]) * w2;
            R Q[3];
            mul_pair<R>(Q[0], Q[1], mv[0], mv[1], w2, w2);
            fma_pair<R>(Q[0], Q[1], mC[2], mC[5], rw2, rw2);
            fma_pair<R>(Q[0], Q[1], T[2], T[5], dw2, dw2);
            Q[2] = fma(T[8], dw2, fma(mC[8], rw2, mv[2] * w2));
#pragma unroll
            for (int ib = 0; ib < K; ++ib) {
                const R w1 = w[1][ib];
                R P[3], S;
                mul_pair<R>(P[0], P[1], w1, w1, Q[0], Q[1]);
                fma_pair<R>(P[0], P[1], H[0][ib], H[1][ib], w2, w2);
                mul_pair<R>(P[2], S, w1, w1, Q[2], w2);
                P[2] = fma(H[2][ib], w2, P[2]);
#pragma unroll
                for (int ia = 0; ia < K; ++ia) {
                    const int j = ia + K * ib + K * K * icl;
                    // (c0, c1) and (c2, mass) as packed pairs
                    fma_pair<R>(cur[j * NV + 0], cur[j * NV + 1], E[0][ia], E[1][ia], S, S);
                    fma_pair<R>(cur[j * NV + 0], cur[j * NV + 1], w[0][ia], w[0][ia], P[0], P[1]);
                    cur[j * NV + 2] += E[2][ia] * S;
                    fma_pair<R>(cur[j * NV + 2], cur[j * NV + 3], w[0][ia], mw0[ia], P[2], S);
                }
            }
        }
    } else {
        R E[2][K];
#pragma unroll
        for (int i = 0; i < K; ++i) {
            const R rw0 = (R(i) - fx[0]) * w[0][i];
#pragma unroll
            for (int cc = 0; cc < 2; ++cc) E[cc][i] = mC[cc * 2 + 0] * rw0 + T[cc * 2 + 0] * dw[0][i];
        }
#pragma unroll
        for (int ib = 0; ib < K; ++ib) {
            const R w1 = w[1][ib], rw1 = (R(ib) - fx[1]) * w1, mw1 = ml * w1;
            R Q[2];
#pragma unroll
            for (int cc = 0; cc < 2; ++cc) Q[cc] = mv[cc] * w1 + mC[cc * 2 + 1] * rw1 + T[cc * 2 + 1] * dw[1][ib];
#pragma unroll
            for (int ia = 0; ia < K; ++ia) {
                const int j = ia + K * ib;
#pragma unroll
                for (int cc = 0; cc < 2; ++cc) cur[j * NV + cc] += w[0][ia] * Q[cc] + E[cc][ia] * w1;
                cur[j * NV + 2] += w[0][ia] * mw1;
            }
        }
    }
}

// One tile of the cell-parallel P2G (whole CTA, NT = 128 threads).  On entry the CTA is
// converged; cbeg / cend hold zeros and *s_cell = 0 (set by the caller before its last
// barrier).  Leaves the smem free for the next tile after its final barrier.
template <int D, int ORDER, typename R, int G>
__device__ __forceinline__ void p2g_cells_tile(const PState<R>& st, const uint32_t* __restrict__ perm,
                                               const uint32_t* tk, uint32_t start, uint32_t end,
                                               R* __restrict__ acc, uint32_t* __restrict__ flags, const DevCfg<R>& c,
                                               uint32_t* err, uint32_t* fallbacks, R* cellsum, uint32_t* cbeg,
                                               uint32_t* cend, int* s_cell, R* pslots,
                                               const uint32_t* pf_src = nullptr, uint32_t pf_n = 0u,
                                               uint32_t* pf_dst = nullptr)
{
    constexpr int NT = 128;
    constexpr int K = ORDER + 1;
    constexpr int NS = (D == 3) ? K * K * K : K * K;
    constexpr int NV = D + 1;
    constexpr int NVAL = NS * NV;
    constexpr int NC = (D == 3) ? 64 : 16;      // base cells of a node block
    // 3-D cubic: the 64-node stencil is summed in two z-halves (128 register sums each)
    constexpr int ZS = (D == 3 && ORDER == 3) ? 2 : 1;
    constexpr int KZ = (D == 3) ? K / ZS : 1;
    constexpr int NVS = NVAL / ZS;
    const int lane = threadIdx.x & 31;
    const int lig = threadIdx.x % G;
    const R dt_dx = step_dt(c) * c.inv_dx;
    const R m = c.mass;
    const R sC = (c.transfer == 0) ? m * c.inv_kdx : R(0);
    const bool with_tau = c.model != 0;
    const bool mat = c.mat != 0;
    const uint32_t blk = tk[0] >> (2 * D);
    int bo[3] = {0, 0, 0};
    block_coords<D, R>(blk, c, bo);
#pragma unroll
    for (int a = 0; a < D; ++a) bo[a] *= 4;
        tile_cell_runs<D>(tk, start, end, cbeg, cend, NT);
        __syncthreads();
        // the tile's keys are read: the next tile's may be copied over them while it runs
        if (pf_n > 0u) {
            for (uint32_t i = threadIdx.x; i < pf_n; i += NT) cp_async4(pf_dst + i, pf_src + i);
            cp_async_commit();
        }
        // A warp takes GPW cells at once (one per lane group) and runs a warp-uniform number
        // of iterations -- the longest run among them -- so all lanes follow one instruction
        // stream; lanes past their run carry a neutral particle that adds zeros.  (Groups
        // taking cells on their own fall out of step once the run lengths differ, and the
        // warp then executes them one after another.)
        constexpr int GPW = 32 / G;
        const int gw = lane / G;
        for (;;) {
            int cb = 0;
            if (lane == 0) cb = atomicAdd(s_cell, GPW);
            cb = __shfl_sync(FULLMASK, cb, 0);
            if (cb >= NC) break;
            const int cell = cb + gw;
            const bool has = cell < NC;
            const uint32_t kb = has ? cbeg[cell] : 0u, ke = has ? cend[cell] : 0u;
            const int lb[3] = {cell & 3, (cell >> 2) & 3, (D == 3) ? ((cell >> 4) & 3) : 0};
            const uint32_t mine = (ke > kb + (uint32_t)lig) ? (ke - kb - (uint32_t)lig + G - 1) / G : 0u;
            const uint32_t iters = __reduce_max_sync(FULLMASK, mine);
            if (iters == 0u) continue;
#pragma unroll 1
            for (int slab = 0; slab < ZS; ++slab) {
            R cur[NVS];
#pragma unroll
            for (int i = 0; i < NVS; ++i) cur[i] = R(0);
            // this lane's particles kb + lig + i G are staged NSL ahead through shared memory
            constexpr int NSL = p2g_slots<R>();
            constexpr int SW = slot_words<D>();
#pragma unroll
            for (int i = 0; i < NSL; ++i) {
                const uint32_t kk = kb + lig + (uint32_t)(i * G);
                if (kk < ke) stage_particle<D, R>(pslots + (size_t)(i * NT + threadIdx.x) * SW, st, perm[kk], with_tau, mat);
                cp_async_commit();
            }
            // the permutation entry of the particle staged next is read one iteration early,
            // so the copy's address is ready when the copy is issued
            uint32_t qn = 0u;
            {
                const uint32_t kn = kb + lig + (uint32_t)(NSL * G);
                if (kn < ke) qn = perm[kn];
            }
#pragma unroll 1
            for (uint32_t it = 0; it < iters; ++it) {
                const uint32_t k = kb + lig + it * G;
                bool live = k < ke;
                cp_async_wait<NSL - 1>();
                R* slot = pslots + (size_t)((it % NSL) * NT + threadIdx.x) * SW;
                Particle<D, R> p;
                read_staged<D, R>(slot, p, with_tau, mat);
                {
                    const uint32_t kn = k + (uint32_t)(NSL * G);
                    if (kn < ke) stage_particle<D, R>(slot, st, qn, with_tau, mat);
                    cp_async_commit();
                    const uint32_t kq = kn + (uint32_t)G;
                    if (kq < ke) qn = perm[kq];
                }
                // the particle's own mass when parameters per particle are set
                const R mp = mat ? p.pm : m;
                const R sCp = mat ? ((c.transfer == 0) ? mp * c.inv_kdx : R(0)) : sC;
                if (ZS == 1 || slab == 0)
                    p2g_cells_particle<D, ORDER, R, KZ, 0>(p, live, lb, bo, c, err, mp, sCp, dt_dx, with_tau, cur);
                else
                    p2g_cells_particle<D, ORDER, R, KZ, ZS - 1>(p, live, lb, bo, c, err, mp, sCp, dt_dx, with_tau, cur);
            }
            cp_async_wait<0>();
            int off = 0, cnt = NVS;
            ReduceScatter<R, NVS, G>::run(cur, FULLMASK, lig, off, cnt);
            constexpr int FIN = ReduceScatter<R, NVS, G>::FINAL;
            if (has) {
                R* dst = cellsum + (size_t)cell * p2g_cell_stride<D, ORDER, R>() + (size_t)slab * NVS + off;
#pragma unroll
                for (int i = 0; i < FIN; ++i)
                    if (i < cnt) dst[i] = cur[i];
            }
            }   // slab
        }
        __syncthreads();
        tile_flush<D, ORDER, R>(cellsum, cbeg, cend, bo, blk, acc, flags, c, NT);
    __syncthreads();
}

// CTAs per SM of the cell-parallel P2G: three for 3-D quadratic (a 168-register cap that its
// 108 accumulators fit without spilling), else two
template <int D, int ORDER> __host__ __device__ constexpr int cells_ctas_per_sm() { return (D == 3 && ORDER == 2) ? 3 : 2; }

template <int D, int ORDER, typename R, int G>
__global__ void __launch_bounds__(128, (cells_ctas_per_sm<D, ORDER>())) k_p2g_cells(PState<R> st, const uint32_t* __restrict__ perm,
                                                      const uint32_t* __restrict__ skeys,
                                                      const uint32_t* __restrict__ tiles,
                                                      const uint32_t* __restrict__ ntiles_p,
                                                      uint32_t* __restrict__ tile_ctr, R* __restrict__ acc,
                                                      uint32_t* __restrict__ flags, DevCfg<R> c, uint32_t* err,
                                                      uint32_t* fallbacks)
{
    pdl_wait();
    pdl_trigger();
    constexpr int NC = (D == 3) ? 64 : 16;
    extern __shared__ __align__(32) unsigned char p2g_smem[];
    R* cellsum = reinterpret_cast<R*>(p2g_smem);   // [NC][cell stride]
    R* pslots = reinterpret_cast<R*>(p2g_smem + (p2g_cellsum_bytes<D, ORDER, R>() + 31) / 32 * 32);
    __shared__ uint32_t cbeg[NC], cend[NC];
    __shared__ int s_tile, s_cell, s_next;
    const int ntiles = (int)*ntiles_p;
    if constexpr (p2g_key_prefetch<R>()) {
        // The keys of the next tile are copied into shared memory while the current tile
        // runs (its index is taken one tile ahead), so a tile starts without waiting for its
        // key loads.
        uint32_t* kbuf = reinterpret_cast<uint32_t*>(p2g_smem + p2g_cells_smem<D, ORDER, R>());
        if (threadIdx.x == 0) {
            s_tile = (int)atomicAdd(tile_ctr, 1u);
            s_next = (int)atomicAdd(tile_ctr, 1u);
        }
        __syncthreads();
        int t = s_tile;
        if (t < ntiles) {
            const uint32_t b0 = tiles[t], b1 = tiles[t + 1];
            for (uint32_t k = b0 + threadIdx.x; k < b1; k += 128u) cp_async4(kbuf + (k - b0), skeys + k);
            cp_async_commit();
        }
        while (t < ntiles) {
            const uint32_t b0 = tiles[t], b1 = tiles[t + 1];
            const int tn = s_next;
            uint32_t nb0 = 0u, nb1 = 0u;
            if (tn < ntiles) {
                nb0 = tiles[tn];
                nb1 = tiles[tn + 1];
            }
            for (int i = threadIdx.x; i < NC; i += 128) { cbeg[i] = 0u; cend[i] = 0u; }
            if (threadIdx.x == 0) s_cell = 0;
            cp_async_wait<0>();
            __syncthreads();   // this tile's keys have landed; s_next has been read by all
            if (threadIdx.x == 0) s_next = (int)atomicAdd(tile_ctr, 1u);   // read after the tile's barriers
            p2g_cells_tile<D, ORDER, R, G>(st, perm, kbuf, b0, b1, acc, flags, c, err, fallbacks, cellsum, cbeg,
                                           cend, &s_cell, pslots, skeys + nb0, nb1 - nb0, kbuf);
            t = tn;
        }
        cp_async_wait<0>();
    } else {
        for (;;) {
            if (threadIdx.x == 0) {
                s_tile = (int)atomicAdd(tile_ctr, 1u);
                s_cell = 0;
            }
            for (int i = threadIdx.x; i < NC; i += 128) { cbeg[i] = 0u; cend[i] = 0u; }
            __syncthreads();
            const int t = s_tile;
            if (t >= ntiles) break;
            p2g_cells_tile<D, ORDER, R, G>(st, perm, skeys + tiles[t], tiles[t], tiles[t + 1], acc, flags, c, err,
                                           fallbacks, cellsum, cbeg, cend, &s_cell, pslots);
        }
    }
}


// ---------------------------------------------------------------- P2G, component-split (3-D)
// A group of lanes per base cell of the tile's node block, all groups at once (64 groups per
// CTA), each walking its cell's run of sorted particles.  The lanes of a group split what a
// single lane would accumulate: lane bit 0 picks the pair of sums (momentum components 0 and
// 1, or component 2 and the mass) and, for cubic B-splines, lane bit 1 picks the z-half of
// the 4^3-node stencil.  A lane then holds 2 sums per node of 27 (quadratic) or 32 (cubic)
// nodes, half the registers of a lane that holds all four, so twice the warps fit on an SM;
// each lane repeats only the per-axis weights.  The mass rides as a fourth "component" whose
// velocity is 1 and whose affine and stress rows are zero, so every lane runs the same code.
// The group's lanes share each particle's staging slot (each copies part of it), so a group
// reads a particle once.  No reduction across lanes is needed: each lane stores its sums of
// its cell, and the node gather of the cell-parallel kernel adds them up.
template <int ORDER> struct SplitShape {
    static constexpr int K = ORDER + 1;
    static constexpr int ZS = ORDER == 3 ? 2 : 1;   // z-halves of the stencil
    static constexpr int KZ = K / ZS;               // z nodes per lane
    static constexpr int LPC = 2 * ZS;              // lanes per cell
    static constexpr int NT = 64 * LPC;             // threads per CTA: a lane group per base cell
    static constexpr int NSL = 3;                   // staging slots per group
};
template <int ORDER, typename R> __host__ __device__ constexpr int split_ctas_per_sm()
{
    return sizeof(R) == 4 ? (ORDER == 2 ? 4 : 2) : (ORDER == 2 ? 2 : 1);
}
template <int ORDER, typename R> __host__ __device__ constexpr size_t p2g_split_smem()
{
    return (p2g_cellsum_bytes<3, ORDER, R>() + 31) / 32 * 32 +
           (size_t)64 * SplitShape<ORDER>::NSL * slot_words<3>() * sizeof(R);
}

// lane r of a group copies the groups g = r, r + LPC, ... of particle q's packed state (A V Ba
// Bb Ta Tb, then the (m_p, V_p) half of M when parameters per particle are set) into the
// group's slot
template <int LPC, typename R>
__device__ __forceinline__ void stage_part(R* slot, const PState<R>& s, uint32_t q, int r, bool mat)
{
#pragma unroll
    for (int g = 0; g < 7; ++g) {
        if (g % LPC != r) continue;
        if (g == 6 && mat) cp_group2<R>(slot + slot_mass_word<3>(), mass_half(s, q));
        if (g == 0) cp_group4<R>(slot + 0, s.A + q);
        if (g == 1) cp_group4<R>(slot + 4, s.V + q);
        if (g == 2) cp_group4<R>(slot + 8, s.Ba + q);
        if (g == 3) cp_group4<R>(slot + 12, s.Bb + q);
        if (g == 4) cp_group4<R>(slot + 16, s.Ta + q);
        if (g == 5) cp_group2<R>(slot + 20, s.Tb + q);
    }
}

// One particle's two sums per node of the lane's stencil part added into accA / accB.
// h: 0 = momentum components (0, 1), 1 = (component 2, mass); zs: the lane's z-half.
template <int ORDER, typename R>
__device__ __forceinline__ void p2g_split_particle(const R* slot, bool live, int h, int zs, const int* lb, const int* bo,
                                                   const DevCfg<R>& c, uint32_t* err, R m, R sC, R dt_dx,
                                                   bool with_tau, R* accA, R* accB)
{
    using S = SplitShape<ORDER>;
    constexpr int K = S::K;
    constexpr int KZ = S::KZ;
    const V4<R> a = *reinterpret_cast<const V4<R>*>(slot + 0);
    const V4<R> v = *reinterpret_cast<const V4<R>*>(slot + 4);
    const V4<R> ba = *reinterpret_cast<const V4<R>*>(slot + 8);
    const V4<R> bb = *reinterpret_cast<const V4<R>*>(slot + 12);
    R o[3] = {a.x, a.y, a.z};
    int cell[3];
    unpack_cell<3>(r2u(a.w), cell);
    if (!live) {   // neutral: an in-cell position (finite weights) and zero weight of the state
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            o[d] = R(0.5);
            cell[d] = bo[d] + lb[d] + (ORDER == 3 ? 1 : 0);
        }
    }
    int base[3];
    R w[3][K], dw[3][K], fx[3];
    bool ok = particle_stencil<3, ORDER, R>(o, cell, c, base, fx, w, dw);
#pragma unroll
    for (int d = 0; d < 3; ++d)
        if (base[d] - bo[d] != lb[d]) ok = false;
    if (live && !ok) {
        set_err(err, APIC_ERRBIT_RANGE);
        live = false;
    }
    // the lane's two rows: velocity, B row (affine), tau row (stress); the mass row is (1, 0, 0).
    // A neutral lane's slot may hold anything (even NaN), so its rows are selected to zero
    // rather than scaled by zero.
    const bool hi = h != 0;
    const bool tau_on = live && with_tau;
    const R mvA = live ? m * (hi ? v.z : v.x) : R(0);
    const R mvB = live ? (hi ? m : m * v.y) : R(0);
    R CA[3], CB[3], TA[3], TB[3];
    CA[0] = live ? sC * (hi ? bb.y : v.w) : R(0);
    CA[1] = live ? sC * (hi ? bb.z : ba.x) : R(0);
    CA[2] = live ? sC * (hi ? bb.w : ba.y) : R(0);
    CB[0] = (live && !hi) ? sC * ba.z : R(0);
    CB[1] = (live && !hi) ? sC * ba.w : R(0);
    CB[2] = (live && !hi) ? sC * bb.x : R(0);
    {
        const V4<R> ta = *reinterpret_cast<const V4<R>*>(slot + 16);   // t00 t11 t22 t01
        const V2<R> tb = *reinterpret_cast<const V2<R>*>(slot + 20);   // t02 t12
        // T = -dt/dx tau (the sign folded in, so every factor below is a sum of products)
        TA[0] = tau_on ? -dt_dx * (hi ? tb.x : ta.x) : R(0);
        TA[1] = tau_on ? -dt_dx * (hi ? tb.y : ta.w) : R(0);
        TA[2] = tau_on ? -dt_dx * (hi ? ta.z : tb.x) : R(0);
        TB[0] = (tau_on && !hi) ? -dt_dx * ta.w : R(0);
        TB[1] = (tau_on && !hi) ? -dt_dx * ta.y : R(0);
        TB[2] = (tau_on && !hi) ? -dt_dx * tb.y : R(0);
    }
    // separable sums as in the cell-parallel kernel, for the lane's two rows and z-half
    //   sum_c(i,j,k) = w0_i P_c(j,k) + E_c(i) S(j,k),  S = w1_j w2_k
    //   P_c(j,k) = w1_j Q_c(k) + H_c(j) w2_k,  Q_c(k) = mv_c w2_k + C_c2 (r w)2_k + T_c2 dw2_k
    //   H_c(j) = C_c1 (r w)1_j + T_c1 dw1_j,    E_c(i) = C_c0 (r w)0_i + T_c0 dw0_i
    // the two rows' factors formed together in packed pairs
    R EA[K], EB[K], HA[K], HB[K];
#pragma unroll
    for (int i = 0; i < K; ++i) {
        const R rw0 = (R(i) - fx[0]) * w[0][i], rw1 = (R(i) - fx[1]) * w[1][i];
        mul_pair<R>(EA[i], EB[i], CA[0], CB[0], rw0, rw0);
        fma_pair<R>(EA[i], EB[i], TA[0], TB[0], dw[0][i], dw[0][i]);
        mul_pair<R>(HA[i], HB[i], CA[1], CB[1], rw1, rw1);
        fma_pair<R>(HA[i], HB[i], TA[1], TB[1], dw[1][i], dw[1][i]);
    }
#pragma unroll
    for (int icl = 0; icl < KZ; ++icl) {
        // the lane's z node: icl, or KZ + icl in the upper half (a select, so the weights
        // stay in registers)
        const R w2 = (ORDER == 3 && zs) ? w[2][(KZ + icl) % K] : w[2][icl];
        const R dw2 = (ORDER == 3 && zs) ? dw[2][(KZ + icl) % K] : dw[2][icl];
        const R z = (ORDER == 3 && zs) ? R(KZ + icl) : R(icl);
        const R rw2 = (z - fx[2]) * w2;
        R QA, QB;
        mul_pair<R>(QA, QB, mvA, mvB, w2, w2);
        fma_pair<R>(QA, QB, CA[2], CB[2], rw2, rw2);
        fma_pair<R>(QA, QB, TA[2], TB[2], dw2, dw2);
#pragma unroll
        for (int ib = 0; ib < K; ++ib) {
            const R w1 = w[1][ib];
            const R S = w1 * w2;
            R PA, PB;
            mul_pair<R>(PA, PB, w1, w1, QA, QB);
            fma_pair<R>(PA, PB, HA[ib], HB[ib], w2, w2);
#pragma unroll
            for (int ia = 0; ia < K; ++ia) {
                const int j = ia + K * ib + K * K * icl;
                fma_pair<R>(accA[j], accB[j], w[0][ia], w[0][ia], PA, PB);
                fma_pair<R>(accA[j], accB[j], EA[ia], EB[ia], S, S);
            }
        }
    }
}

// One tile (the sorted particles of one node block) by the whole CTA.  On entry the CTA is
// converged and cbeg / cend hold zeros.  Leaves the shared memory free after its final barrier.
template <int ORDER, typename R>
__device__ __forceinline__ void p2g_split_tile(const PState<R>& st, const uint32_t* __restrict__ perm,
                                               const uint32_t* __restrict__ skeys, uint32_t start, uint32_t end,
                                               R* __restrict__ acc, uint32_t* __restrict__ flags, const DevCfg<R>& c,
                                               uint32_t* err, R* cellsum, uint32_t* cbeg, uint32_t* cend, R* pslots)
{
    using S = SplitShape<ORDER>;
    constexpr int K = S::K;
    constexpr int KZ = S::KZ;
    constexpr int LPC = S::LPC;
    constexpr int NT = S::NT;
    constexpr int NSL = S::NSL;
    constexpr int SW = slot_words<3>();
    // lane group grp takes base cell grp of the block, so a warp's cells are neighbours in the
    // sorted order (its staging reads stay close together; spreading a warp's cells over the
    // whole block balanced the warps of partly filled blocks but cost more lane-iterations
    // than it saved in barrier waits)
    const int grp = threadIdx.x / LPC;
    const int cell = grp;
    const int r = threadIdx.x % LPC;
    const int h = r & 1;
    const int zs = (ORDER == 3) ? (r >> 1) : 0;
    const R dt_dx = step_dt(c) * c.inv_dx;
    const R m = c.mass;
    const R sC = (c.transfer == 0) ? m * c.inv_kdx : R(0);
    const bool with_tau = c.model != 0;
    const bool mat = c.mat != 0;
    const uint32_t blk = skeys[start] >> 6;
    int bo[3] = {0, 0, 0};
    block_coords<3, R>(blk, c, bo);
#pragma unroll
    for (int d = 0; d < 3; ++d) bo[d] *= 4;
    tile_cell_runs<3>(skeys + start, start, end, cbeg, cend, NT);
    __syncthreads();
    const uint32_t kb = cbeg[cell], ke = cend[cell];
    const int lb[3] = {cell & 3, (cell >> 2) & 3, (cell >> 4) & 3};
    const uint32_t run = ke - kb;
    // warp-uniform trip count (the longest run among the warp's cells): all lanes follow one
    // instruction stream; lanes past their run carry a neutral particle that adds zeros
    const uint32_t iters = __reduce_max_sync(FULLMASK, run);
    if (iters > 0u) {
        R accA[K * K * KZ], accB[K * K * KZ];
#pragma unroll
        for (int i = 0; i < K * K * KZ; ++i) { accA[i] = R(0); accB[i] = R(0); }
        R* gslots = pslots + (size_t)grp * NSL * SW;
        // particles 0 .. NSL-2 of the run first; particle it + NSL - 1 goes into the slot read
        // in the previous iteration (every lane of the warp has passed this iteration's
        // barrier after reading it)
#pragma unroll
        for (int i = 0; i < NSL - 1; ++i) {
            if ((uint32_t)i < run) stage_part<LPC, R>(gslots + i * SW, st, perm[kb + i], r, mat);
            cp_async_commit();
        }
        uint32_t qn = ((uint32_t)(NSL - 1) < run) ? perm[kb + NSL - 1] : 0u;
#pragma unroll 1
        for (uint32_t it = 0; it < iters; ++it) {
            cp_async_wait<NSL - 2>();
            __syncwarp();
            {
                const uint32_t nx = it + NSL - 1;
                if (nx < run) stage_part<LPC, R>(gslots + (nx % NSL) * SW, st, qn, r, mat);
                cp_async_commit();
                if (nx + 1 < run) qn = perm[kb + nx + 1];
            }
            // the particle's own mass when parameters per particle are set
            const R* sl = gslots + (it % NSL) * SW;
            const R mp = mat ? sl[slot_mass_word<3>()] : m;
            const R sCp = mat ? ((c.transfer == 0) ? mp * c.inv_kdx : R(0)) : sC;
            p2g_split_particle<ORDER, R>(sl, it < run, h, zs, lb, bo, c, err, mp, sCp, dt_dx, with_tau, accA, accB);
        }
        cp_async_wait<0>();
        if (run > 0u) {
            R* dst = cellsum + (size_t)cell * p2g_cell_stride<3, ORDER, R>() + 2 * h;
#pragma unroll
            for (int icl = 0; icl < KZ; ++icl)
#pragma unroll
                for (int ib = 0; ib < K; ++ib)
#pragma unroll
                    for (int ia = 0; ia < K; ++ia) {
                        const int jl = ia + K * ib + K * K * icl;
                        const int j = ia + K * ib + K * K * (zs * KZ + icl);
                        *reinterpret_cast<V2<R>*>(dst + 4 * j) = V2<R>{accA[jl], accB[jl]};
                    }
        }
    }
    __syncthreads();
    tile_flush<3, ORDER, R>(cellsum, cbeg, cend, bo, blk, acc, flags, c, NT);
    __syncthreads();
}

template <int ORDER, typename R>
__global__ void __launch_bounds__(SplitShape<ORDER>::NT, (split_ctas_per_sm<ORDER, R>()))
    k_p2g_split(PState<R> st, const uint32_t* __restrict__ perm, const uint32_t* __restrict__ skeys,
                const uint32_t* __restrict__ tiles, const uint32_t* __restrict__ ntiles_p,
                uint32_t* __restrict__ tile_ctr, R* __restrict__ acc, uint32_t* __restrict__ flags, DevCfg<R> c,
                uint32_t* err)
{
    pdl_wait();
    pdl_trigger();
    extern __shared__ __align__(32) unsigned char p2g_smem[];
    R* cellsum = reinterpret_cast<R*>(p2g_smem);   // [64][cell stride]
    R* pslots = reinterpret_cast<R*>(p2g_smem + (p2g_cellsum_bytes<3, ORDER, R>() + 31) / 32 * 32);
    __shared__ uint32_t cbeg[64], cend[64];
    __shared__ int s_tile;
    const int ntiles = (int)*ntiles_p;
    // the next tile's index is requested when a tile starts, so its latency passes during the
    // tile; thread 0 publishes it after the tile's last barrier
    int next = 0;
    if (threadIdx.x == 0) next = (int)atomicAdd(tile_ctr, 1u);
    for (;;) {
        if (threadIdx.x == 0) s_tile = next;
        if (threadIdx.x < 64) { cbeg[threadIdx.x] = 0u; cend[threadIdx.x] = 0u; }
        __syncthreads();
        const int t = s_tile;
        if (t >= ntiles) break;
        if (threadIdx.x == 0) next = (int)atomicAdd(tile_ctr, 1u);
        p2g_split_tile<ORDER, R>(st, perm, skeys, tiles[t], tiles[t + 1], acc, flags, c, err, cellsum, cbeg, cend,
                                 pslots);
    }
}

// ---------------------------------------------------------------- grid update (Sec. 3.3)
// One warp per active node block: v~ = ((m v) + dt f) / m + dt g, sticky walls, v~ = 0 where
// m = 0; writes (v~, m) to the velocity grid and clears the accumulation grid and flag.
// one node block of the grid update, by one warp
template <int D, typename R>
__device__ __forceinline__ void grid_update_block(R* __restrict__ acc, R* __restrict__ vel,
                                                  uint32_t* __restrict__ flags, const DevCfg<R>& c, int b, int lane,
                                                  R* __restrict__ acc2 = nullptr, R* __restrict__ vdel = nullptr,
                                                  bool known_active = false)
{
    constexpr int BN = (D == 3) ? 64 : 16;
    if (!known_active && flags[b] == 0u) return;
    int bc[3] = {0, 0, 0};
    block_coords<D, R>((uint32_t)b, c, bc);
    // the lane's nodes lane + 32 q, all loaded before any is written
    constexpr int PER = (BN + 31) / 32;
    V4<R> av[PER];
#pragma unroll
    for (int q = 0; q < PER; ++q)
        if (lane + 32 * q < BN) av[q] = *reinterpret_cast<const V4<R>*>(acc + 4 * ((size_t)b * BN + lane + 32 * q));
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int i = lane + 32 * q;
        if (i >= BN) continue;
        const size_t node = (size_t)b * BN + i;
        const V4<R> a = av[q];
        int g[3];
        g[0] = bc[0] * 4 + (i & 3);
        g[1] = bc[1] * 4 + ((i >> 2) & 3);
        g[2] = (D == 3) ? bc[2] * 4 + (i >> 4) : 0;
        const R m = a.w;
        R v[3] = {R(0), R(0), R(0)};
        if (m > R(0)) {
            const R inv = R(1) / m;
            const R dt = step_dt(c);
            v[0] = a.x * inv + dt * c.gravity[0];
            v[1] = a.y * inv + dt * c.gravity[1];
            if (D == 3) v[2] = a.z * inv + dt * c.gravity[2];
            if (c.boundary == 1) {           // sticky: the whole velocity
                bool wall = false;
#pragma unroll
                for (int d = 0; d < D; ++d)
                    if (g[d] < c.wall || g[d] >= c.res[d] - c.wall) wall = true;
                if (wall) v[0] = v[1] = v[2] = R(0);
            } else if (c.boundary == 2) {    // slip: the component normal to each wall
#pragma unroll
                for (int d = 0; d < D; ++d)
                    if (g[d] < c.wall || g[d] >= c.res[d] - c.wall) v[d] = R(0);
            }
        }
        *reinterpret_cast<V4<R>*>(vel + 4 * node) = V4<R>{v[0], v[1], v[2], m};
        *reinterpret_cast<V4<R>*>(acc + 4 * node) = V4<R>{R(0), R(0), R(0), R(0)};
        if (acc2) {   // FLIP: the change v~ - v against the velocity before the update
            const V4<R> a2 = *reinterpret_cast<const V4<R>*>(acc2 + 4 * node);
            R dv[3] = {R(0), R(0), R(0)};
            if (m > R(0)) {
                const R inv = R(1) / m;
                dv[0] = v[0] - a2.x * inv;
                dv[1] = v[1] - a2.y * inv;
                if (D == 3) dv[2] = v[2] - a2.z * inv;
            }
            *reinterpret_cast<V4<R>*>(vdel + 4 * node) = V4<R>{dv[0], dv[1], dv[2], m};
            *reinterpret_cast<V4<R>*>(acc2 + 4 * node) = V4<R>{R(0), R(0), R(0), R(0)};
        }
    }
    __syncwarp();
    if (lane == 0) flags[b] = 0u;
}

template <int D, typename R>
__global__ void __launch_bounds__(TPB) k_grid_update(R* __restrict__ acc, R* __restrict__ vel,
                                                     uint32_t* __restrict__ flags, DevCfg<R> c, R* acc2, R* vdel)
{
    pdl_wait();
    pdl_trigger();
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * TPB + threadIdx.x) >> 5;
    const int nw = (gridDim.x * TPB) >> 5;
    if (c.smax && blockIdx.x == 0 && threadIdx.x == 0) *c.smax = 0u;   // G2P, next, max-reduces into it
    // the warp's blocks b0 + j nw, 32 at a time: their flags in one load (lane j), then the
    // active ones one after another
    for (int b0 = gw; b0 < c.nblocks; b0 += 32 * nw) {
        const int bj = b0 + lane * nw;
        unsigned act = __ballot_sync(FULLMASK, bj < c.nblocks && flags[bj] != 0u);
        while (act) {
            const int j = __ffs(act) - 1;
            act &= act - 1u;
            grid_update_block<D, R>(acc, vel, flags, c, b0 + j * nw, lane, acc2, vdel, true);
        }
    }
}

// ---------------------------------------------------------------- mbarrier + bulk copy
__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0u;
}
// bounded wait: gives up after `limit` polls (each poll may suspend the thread briefly)
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity, unsigned limit)
{
    for (unsigned i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// ---------------------------------------------------------------- G2P (Sec. 3.4, 5.7)
// Per tile, the 2^D node blocks its particles' stencils can reach are brought into shared
// memory with bulk asynchronous copies completing on an mbarrier; each particle then
// gathers v_p = sum w v~, B_p = sum w v~ (x_i - x_p)^T, grad v = sum v~ grad w^T, updates
// F_p <- (I + dt grad v) F_p and x_p <- x_p + dt v_p, and is written at its sorted slot
// together with its next cell key.
// G2P works tile by tile with two staging buffers: while a tile's particles are processed,
// the 2^D grid blocks of the next tile are already in flight (bulk copies completing on that
// buffer's mbarrier), so the copy latency is hidden behind arithmetic.

// thread 0: start the bulk copies of the 2^D velocity blocks around node block `blk`
template <int D, typename R>
__device__ __forceinline__ void g2p_issue(const R* __restrict__ vel, uint32_t blk, const int* nb,
                                          R (*sv)[(D == 3) ? 64 : 16][4], uint64_t* mbar)
{
    constexpr int BN = (D == 3) ? 64 : 16;
    constexpr int NB = 1 << D;
    int bc[3];
    bc[0] = (int)(blk % (uint32_t)nb[0]);
    if (D == 3) {
        bc[1] = (int)((blk / (uint32_t)nb[0]) % (uint32_t)nb[1]);
        bc[2] = (int)(blk / ((uint32_t)nb[0] * (uint32_t)nb[1]));
    } else {
        bc[1] = (int)(blk / (uint32_t)nb[0]);
        bc[2] = 0;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    unsigned nblk = 0;
    bool inb[NB];
#pragma unroll
    for (int q = 0; q < NB; ++q) {
        inb[q] = true;
#pragma unroll
        for (int a = 0; a < D; ++a)
            if (bc[a] + ((q >> a) & 1) >= nb[a]) inb[q] = false;
        nblk += inb[q] ? 1u : 0u;
    }
    const unsigned bytes = (unsigned)(BN * 4 * sizeof(R));
    mbar_expect_tx(mbar, nblk * bytes);
#pragma unroll
    for (int q = 0; q < NB; ++q) {
        if (!inb[q]) continue;
        const int bb[3] = {bc[0] + (q & 1), bc[1] + ((q >> 1) & 1), (D == 3) ? bc[2] + ((q >> 2) & 1) : 0};
        const uint32_t b2 = (D == 3) ? ((uint32_t)bb[2] * nb[1] + bb[1]) * nb[0] + bb[0] : (uint32_t)bb[1] * nb[0] + bb[0];
        bulk_copy_g2s(&sv[q][0][0], vel + (size_t)b2 * BN * 4, bytes, mbar);
    }
}

// 3-D cubic G2P stages the dense 8^3 node array around the tile (node (x, y, z) at x + 8 y +
// 64 z), so a stencil node's offset is a per-particle base plus a constant; the 2^D blocks'
// rows of 4 nodes (contiguous in both layouts) are copied by the lanes of warp 0, after lane
// 0 has set the byte count the buffer's mbarrier expects.  (Quadratic G2P keeps the block
// layout: there the dense one raised its registers past the cap.)
template <int ORDER> __host__ __device__ constexpr bool g2p_dense() { return ORDER == 3; }

template <int D, typename R>
__device__ __noinline__ void g2p_issue_dense(const R* __restrict__ vel, uint32_t blk, const int* nb,
                                             R (*sv)[(D == 3) ? 64 : 16][4], uint64_t* mbar, int lane)
{
    constexpr int BN = (D == 3) ? 64 : 16;
    constexpr int NB = 1 << D;
    constexpr int ROWS = BN / 4;
    int bc[3];
    bc[0] = (int)(blk % (uint32_t)nb[0]);
    if (D == 3) {
        bc[1] = (int)((blk / (uint32_t)nb[0]) % (uint32_t)nb[1]);
        bc[2] = (int)(blk / ((uint32_t)nb[0] * (uint32_t)nb[1]));
    } else {
        bc[1] = (int)(blk / (uint32_t)nb[0]);
        bc[2] = 0;
    }
    unsigned nblk = 0;
    bool inb[NB];
#pragma unroll
    for (int q = 0; q < NB; ++q) {
        inb[q] = true;
#pragma unroll
        for (int a = 0; a < D; ++a)
            if (bc[a] + ((q >> a) & 1) >= nb[a]) inb[q] = false;
        nblk += inb[q] ? 1u : 0u;
    }
    if (lane == 0) mbar_expect_tx(mbar, nblk * (unsigned)(BN * 4 * sizeof(R)));
    __syncwarp();
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    R* dense = &sv[0][0][0];
    const unsigned row_bytes = (unsigned)(4 * 4 * sizeof(R));
    for (int rr = lane; rr < NB * ROWS; rr += 32) {
        const int q = rr / ROWS, r = rr % ROWS;
        if (!inb[q]) continue;
        const int bb[3] = {bc[0] + (q & 1), bc[1] + ((q >> 1) & 1), (D == 3) ? bc[2] + ((q >> 2) & 1) : 0};
        const uint32_t b2 = (D == 3) ? ((uint32_t)bb[2] * nb[1] + bb[1]) * nb[0] + bb[0] : (uint32_t)bb[1] * nb[0] + bb[0];
        const int q0 = 4 * (q & 1) + 32 * ((q >> 1) & 1) + ((D == 3) ? 256 * ((q >> 2) & 1) : 0);
        const int y = r & 3, z = r >> 2;
        bulk_copy_g2s(dense + 4 * (q0 + 8 * y + 64 * z), vel + ((size_t)b2 * BN + 4 * r) * 4, row_bytes, mbar);
    }
}

// thread 0: wait (at most `limit` polls) for a buffer's copies; false on timeout, after a
// second bounded wait that lets the copies in flight land before the CTA leaves
__device__ __forceinline__ bool g2p_wait(uint64_t* mbar, unsigned parity, uint32_t* err, unsigned limit)
{
    if (mbar_wait_bounded(mbar, parity, limit)) return true;
    set_err(err, APIC_ERRBIT_TIMEOUT);
    mbar_wait_bounded(mbar, parity, 1u << 22);   // let the copies in flight land before leaving
    return false;
}

// G2P's read-ahead of the next particle's x and F goes through shared memory in FP32 (a slot
// of 16 words per thread and buffer: A, Fa, Fb, Fc), not registers: the kernel works at its
// register cap, and the 16 registers a staged particle would hold are worth more there.
template <typename R> __host__ __device__ constexpr bool g2p_staged() { return sizeof(R) == 4; }
constexpr int kG2PSlot = 16;
template <int D, typename R>
__device__ __forceinline__ void stage_xF(R* slot, const PState<R>& s, uint32_t q)
{
    cp_async16(slot + 0, s.A + q);
    cp_async16(slot + 4, s.Fa + q);
    if (D == 3) {
        cp_async16(slot + 8, s.Fb + q);
        cp_async8(slot + 12, s.Fc + q);
    }
}
template <int D, typename R>
__device__ __forceinline__ void read_xF(const R* slot, Particle<D, R>& p)
{
    const V4<R> a = *reinterpret_cast<const V4<R>*>(slot + 0);
    const V4<R> fa = *reinterpret_cast<const V4<R>*>(slot + 4);
    if (D == 3) {
        const V4<R> fb = *reinterpret_cast<const V4<R>*>(slot + 8);
        const V2<R> fc = *reinterpret_cast<const V2<R>*>(slot + 12);
        p.o[0] = a.x; p.o[1] = a.y; p.o[2] = a.z;
        unpack_cell<D>(r2u(a.w), p.cell);
        p.F[0] = fa.x; p.F[1] = fa.y; p.F[2] = fa.z; p.F[3] = fa.w;
        p.F[4] = fb.x; p.F[5] = fb.y; p.F[6] = fb.z; p.F[7] = fb.w;
        p.F[8] = fc.x; p.id = r2u(fc.y);
    } else {
        p.o[0] = a.x; p.o[1] = a.y;
        unpack_cell<D>(r2u(a.z), p.cell);
        p.id = r2u(a.w);
        p.F[0] = fa.x; p.F[1] = fa.y; p.F[2] = fa.z; p.F[3] = fa.w;
    }
}

// the particles of one tile, with its grid blocks already in sv (whole CTA)
// EXT: the material lane, the fused speed maximum and the FLIP update may be in use (else
// compiled out)
template <int D, int ORDER, typename R, bool EXT, int NTH = TPB>
__device__ __forceinline__ void g2p_compute(const PState<R>& in, const PState<R>& out, const uint32_t* __restrict__ perm,
                                            const uint32_t* __restrict__ skeys, uint32_t start, uint32_t end,
                                            uint32_t* __restrict__ knext, const DevCfg<R>& c, uint32_t* err,
                                            uint32_t* fallbacks, const R (*sv)[(D == 3) ? 64 : 16][4],
                                            float& smax_l, const R* __restrict__ vdel, R* stage)
{
    constexpr int K = ORDER + 1;
    constexpr bool STG = g2p_staged<R>();
    const R dt_dx = step_dt(c) * c.inv_dx;
    const uint32_t blk = skeys[start] >> (2 * D);
    int bc[3] = {0, 0, 0};
    block_coords<D, R>(blk, c, bc);
    // the next round's particle is requested before the current one is processed
    // (and the permutation entry of the one after it, so that load's address is ready)
    Particle<D, R> nxt;
    R* const slot0 = STG ? stage + (size_t)threadIdx.x * kG2PSlot : nullptr;
    R* const slot1 = STG ? stage + (size_t)(NTH + threadIdx.x) * kG2PSlot : nullptr;
    if (start + threadIdx.x < end) {
        const uint32_t q0 = perm[start + threadIdx.x];
        if (STG) stage_xF<D, R>(slot0, in, q0);
        else load_xF<D, R>(in, q0, nxt);
        if (EXT && c.mat) load_mat<D, R>(in, q0, nxt);
        if (EXT && c.transfer == 2) load_v<D, R>(in, q0, nxt);
    }
    if (STG) cp_async_commit();
    uint32_t qn = (start + threadIdx.x + NTH < end) ? perm[start + threadIdx.x + NTH] : 0u;
    for (uint32_t k0 = start; k0 < end; k0 += NTH) {
        const uint32_t k = k0 + threadIdx.x;
        if (k >= end) continue;
        Particle<D, R> p = nxt;
        if (STG) {   // this particle from its slot, the next one's copies into the other
            const bool odd = (((k0 - start) / NTH) & 1u) != 0u;
            R* cur = odd ? slot1 : slot0;
            cp_async_wait<0>();
            read_xF<D, R>(cur, p);
            if (k + NTH < end) stage_xF<D, R>(odd ? slot0 : slot1, in, qn);
            cp_async_commit();
        }
        if (k + NTH < end) {
            if (!STG) load_xF<D, R>(in, qn, nxt);
            if (EXT && c.mat) load_mat<D, R>(in, qn, nxt);
            if (EXT && c.transfer == 2) load_v<D, R>(in, qn, nxt);
        }
        if (k + 2 * NTH < end) qn = perm[k + 2 * NTH];
        int base[D], lb[D];
        R w[D][K], dw[D][K], fx[D];
        bool ok = particle_stencil<D, ORDER, R>(p.o, p.cell, c, base, fx, w, dw);
#pragma unroll
        for (int a = 0; a < D; ++a) {
            lb[a] = base[a] - 4 * bc[a];
            if (lb[a] < 0 || lb[a] > 3) { ok = false; lb[a] = 0; }
        }
        if (!ok) set_err(err, APIC_ERRBIT_RANGE);
        // Separable gather: the weights are tensor products, so the sums over the
        // stencil are taken axis by axis (innermost axis first) instead of node by node:
        //   vp   = sum_i w v~                  = sum_a wx R_a
        //   G    = sum_i v~ grad^w^T           (columns: dwx R_a, wx S_a, wx T_a)
        //   Bh   = sum_i w v~ r^T, r^ = node - fx (columns: rx wx R_a, wx Y_a, wx Zc_a)
        // with per-(a,b) sums over c and per-a sums over b.
        R vp[D], Bh[D * D], G[D * D];
#pragma unroll
        for (int a = 0; a < D; ++a) vp[a] = R(0);
#pragma unroll
        for (int i = 0; i < D * D; ++i) { Bh[i] = R(0); G[i] = R(0); }
        // node (i, j, k) of the stencil sits in staged block qb = (L0>>2) | (L1>>2)<<1 | (L2>>2)<<2
        // at in-block index (L0&3) | (L1&3)<<2 | (L2&3)<<4 (L = lb + stencil index); its offset
        // in the staging buffer is a sum of per-axis terms, taken once per particle
        constexpr int BNN = (D == 3) ? 64 : 16;
        constexpr bool DENSE = g2p_dense<ORDER>();
        int ox[D][K];
#pragma unroll
        for (int a = 0; a < D; ++a)
#pragma unroll
            for (int i = 0; i < K; ++i) {
                const int L = lb[a] + i;
                // dense 8^D layout: node lb + (i, j, k) at a per-particle base plus a constant
                ox[a][i] = DENSE ? 4 * i * (1 << (3 * a)) : 4 * ((L >> 2) * (BNN << a) + (L & 3) * (1 << (2 * a)));
            }
        const R* svf = &sv[0][0][0] + (DENSE ? 4 * (lb[0] + 8 * lb[1] + ((D == 3) ? 64 * lb[2] : 0)) : 0);
        R rw[D][K];   // (node - fx) * w per axis
#pragma unroll
        for (int a = 0; a < D; ++a)
#pragma unroll
            for (int j = 0; j < K; ++j) rw[a][j] = (R(j) - fx[a]) * w[a][j];
#pragma unroll
        for (int ia = 0; ia < K; ++ia) {
            R Ra[D], Sa[D], Ta[D], Ya[D], Za[D];
#pragma unroll
            for (int a = 0; a < D; ++a) { Ra[a] = Sa[a] = Ta[a] = Ya[a] = Za[a] = R(0); }
#pragma unroll
            for (int ib = 0; ib < K; ++ib) {
                const int o01 = ox[0][ia] + ox[1][ib];
                if (D == 3) {
                    R P[3] = {R(0), R(0), R(0)}, Q[3] = {R(0), R(0), R(0)}, Z[3] = {R(0), R(0), R(0)};
#pragma unroll
                    for (int ic = 0; ic < K; ++ic) {
                        const V4<R> nv = *reinterpret_cast<const V4<R>*>(svf + o01 + ox[D - 1][ic]);
                        const R vt[3] = {nv.x, nv.y, nv.z};
                        // components (0, 1) as packed pairs, component 2 of P and Q as one more
                        fma_pair<R>(P[0], P[1], w[2][ic], w[2][ic], vt[0], vt[1]);
                        fma_pair<R>(Q[0], Q[1], dw[2][ic], dw[2][ic], vt[0], vt[1]);
                        fma_pair<R>(Z[0], Z[1], rw[2][ic], rw[2][ic], vt[0], vt[1]);
                        fma_pair<R>(P[2], Q[2], w[2][ic], dw[2][ic], vt[2], vt[2]);
                        Z[2] += rw[2][ic] * vt[2];
                    }
                    fma_pair<R>(Ra[0], Ra[1], w[1][ib], w[1][ib], P[0], P[1]);
                    fma_pair<R>(Sa[0], Sa[1], dw[1][ib], dw[1][ib], P[0], P[1]);
                    fma_pair<R>(Ta[0], Ta[1], w[1][ib], w[1][ib], Q[0], Q[1]);
                    fma_pair<R>(Ya[0], Ya[1], rw[1][ib], rw[1][ib], P[0], P[1]);
                    fma_pair<R>(Za[0], Za[1], w[1][ib], w[1][ib], Z[0], Z[1]);
                    fma_pair<R>(Ra[2], Sa[2], w[1][ib], dw[1][ib], P[2], P[2]);
                    fma_pair<R>(Ta[2], Za[2], w[1][ib], w[1][ib], Q[2], Z[2]);
                    Ya[2] += rw[1][ib] * P[2];
                } else {
                    const V4<R> nv = *reinterpret_cast<const V4<R>*>(svf + o01);
                    const R vt[2] = {nv.x, nv.y};
#pragma unroll
                    for (int a = 0; a < 2; ++a) {
                        Ra[a] += w[1][ib] * vt[a];
                        Sa[a] += dw[1][ib] * vt[a];
                        Ya[a] += rw[1][ib] * vt[a];
                    }
                }
            }
#pragma unroll
            for (int a = 0; a < D; ++a) {
                vp[a] += w[0][ia] * Ra[a];
                G[a * D + 0] += dw[0][ia] * Ra[a];
                G[a * D + 1] += w[0][ia] * Sa[a];
                Bh[a * D + 0] += rw[0][ia] * Ra[a];
                Bh[a * D + 1] += w[0][ia] * Ya[a];
                if (D == 3) {
                    G[a * D + 2] += w[0][ia] * Ta[a];
                    Bh[a * D + 2] += w[0][ia] * Za[a];
                }
            }
        }
        // F <- (I + dt grad v) F with grad v = G / dx
        R Fn[D * D];
#pragma unroll
        for (int a = 0; a < D; ++a)
#pragma unroll
            for (int b = 0; b < D; ++b) {
                R s = p.F[a * D + b];
#pragma unroll
                for (int kk = 0; kk < D; ++kk) s += dt_dx * G[a * D + kk] * p.F[kk * D + b];
                Fn[a * D + b] = s;
            }
#pragma unroll
        for (int i = 0; i < D * D; ++i) {
            p.F[i] = Fn[i];
            p.B[i] = (c.transfer == 0) ? c.dx * Bh[i] : R(0);
        }
        R vnew[D];
#pragma unroll
        for (int a = 0; a < D; ++a) vnew[a] = vp[a];
        if (EXT && c.transfer == 2) {
            // FLIP (Sec. 1): the particle's own velocity plus the interpolated grid change
            // v~_i - v_i, blended with the PIC velocity by flip_alpha
            R dv[3] = {R(0), R(0), R(0)};
#pragma unroll
            for (int ia = 0; ia < K; ++ia)
#pragma unroll
                for (int ib = 0; ib < K; ++ib)
#pragma unroll
                    for (int ic = 0; ic < ((D == 3) ? K : 1); ++ic) {
                        int g[3] = {base[0] + ia, base[1] + ib, (D == 3) ? base[D - 1] + ic : 0};
                        const V4<R> d4 = ld4(reinterpret_cast<const V4<R>*>(vdel) + node_index<D>(g, c.nb));
                        const R wt = w[0][ia] * w[1][ib] * ((D == 3) ? w[D - 1][ic] : R(1));
                        dv[0] += wt * d4.x;
                        dv[1] += wt * d4.y;
                        dv[2] += wt * d4.z;
                    }
#pragma unroll
            for (int a = 0; a < D; ++a) vnew[a] = c.flip_alpha * (p.v[a] + dv[a]) + (R(1) - c.flip_alpha) * vp[a];
        }
#pragma unroll
        for (int a = 0; a < D; ++a) {
            p.v[a] = vnew[a];
            R o = p.o[a] + dt_dx * vp[a];
            const R fl = floor(o);
            o -= fl;
            int cl = p.cell[a] + (int)fl;
            if (o >= R(1)) { o -= R(1); cl += 1; }
            if (cl < 0) { cl = 0; o = R(0); set_err(err, APIC_ERRBIT_RANGE); }
            if (cl > c.res[a] - 1) { cl = c.res[a] - 1; o = R(0); set_err(err, APIC_ERRBIT_RANGE); }
            p.o[a] = o;
            p.cell[a] = cl;
        }
        // the Sec. 4.3 speed of the new state, |v_p| + 6 sqrt(d)/dx |B_p|_F, for the next step's bound
        if (EXT && c.smax) {
            R vv = R(0), bb = R(0);
#pragma unroll
            for (int a = 0; a < D; ++a) vv += p.v[a] * p.v[a];
#pragma unroll
            for (int i = 0; i < D * D; ++i) bb += p.B[i] * p.B[i];
            smax_l = fmaxf(smax_l, (float)(sqrt(vv) + c.cfl_coef * sqrt(bb)));
        }
        // the stress of the new F_p, for the next P2G
        if (c.model != 0)
            stress_sym<D, R>(c.model, p.F, (EXT && c.mat) ? p.mu : c.mu, (EXT && c.mat) ? p.lam : c.lam,
                             (EXT && c.mat) ? p.pv : c.vol, p.tau, fallbacks);
        store_all<D, R>(out, k, p, c.model != 0, EXT && c.mat != 0);
        knext[k] = key_of<D, ORDER, R>(p.o, p.cell, c, err);
    }
}

// G2P runs in 128-thread CTAs (four per SM): a tile's particles then take more rounds per
// thread and fewer threads idle at the per-tile barriers (0.226 vs 0.238 ms with 256 on the
// 128^3 cube; batches of small tiles gain more)
constexpr int G2P_THREADS = 128;

// G2P work items.  The CTAs take items in order, so the last ones decide when the kernel ends:
// for quadratic splines each of the last kG2PTailTiles x (CTAs) tiles is cut into
// g2p_pieces() consecutive particle ranges (each staging the tile's grid blocks again), so
// the CTAs finish close together (cube: G2P 0.1918 -> 0.1884 ms).  Cubic G2P stages a dense
// 8^3 array per item, which costs more than the shorter tail saves, so its items are the
// tiles.  Item i -> [lo, hi); false past the last item.  A piece of a tile shorter than the
// piece count may be empty (lo == hi); the claim skips those.
constexpr int kG2PTailTiles = 3;
template <int ORDER> __host__ __device__ constexpr int g2p_pieces() { return ORDER == 2 ? 2 : 1; }
template <int P>
__device__ __forceinline__ bool g2p_item(const uint32_t* __restrict__ tiles, int ntiles, int i, uint32_t& lo,
                                         uint32_t& hi)
{
    if constexpr (P == 1) {
        if (i >= ntiles) return false;
        lo = tiles[i];
        hi = tiles[i + 1];
        return true;
    }
    const int tail = (int)gridDim.x * kG2PTailTiles;
    const int t0 = ntiles > tail ? ntiles - tail : 0;
    if (i < t0) {
        lo = tiles[i];
        hi = tiles[i + 1];
        return true;
    }
    const int t = t0 + (i - t0) / P;
    if (t >= ntiles) return false;
    const uint32_t a = tiles[t], len = tiles[t + 1] - a, piece = (uint32_t)((i - t0) % P);
    lo = a + len * piece / P;
    hi = a + len * (piece + 1) / P;
    return true;
}
// lane 0: the next non-empty item (valid = false when there is none)
template <int P>
__device__ __forceinline__ bool g2p_claim(const uint32_t* __restrict__ tiles, int ntiles, uint32_t* ctr, uint32_t& lo,
                                          uint32_t& hi)
{
    for (;;) {
        const int i = (int)atomicAdd(ctr, 1u);
        if (!g2p_item<P>(tiles, ntiles, i, lo, hi)) return false;
        if (hi > lo) return true;
    }
}

template <int D, int ORDER, typename R, bool EXT>
__global__ void __launch_bounds__(G2P_THREADS, 4) k_g2p(PState<R> in, PState<R> out, const uint32_t* __restrict__ perm,
                                             const uint32_t* __restrict__ skeys, const uint32_t* __restrict__ tiles,
                                             const uint32_t* __restrict__ ntiles_p, uint32_t* __restrict__ tile_ctr,
                                             const R* __restrict__ vel, uint32_t* __restrict__ knext, DevCfg<R> c,
                                             uint32_t* err, uint32_t* fallbacks, const R* __restrict__ vdel)
{
    pdl_wait();
    pdl_trigger();
    constexpr int BN = (D == 3) ? 64 : 16;
    constexpr int NB = 1 << D;
    __shared__ __align__(128) R sv[2][NB][BN][4];
    __shared__ __align__(16) R stage[g2p_staged<R>() ? 2 * G2P_THREADS * kG2PSlot : 1];
    __shared__ __align__(8) uint64_t mbar[2];
    // s_v[b], s_lo[b], s_hi[b]: whether buffer b holds an item, and its particle range (the
    // grid blocks of its tile are staged in buffer b).  Thread 0 writes entry b ^ 1 before the
    // first barrier of an iteration; every thread reads entry b at the top of the iteration,
    // after the previous iteration's closing barrier, and the entry is not written again
    // until the next iteration has passed that same barrier.
    __shared__ int s_ok, s_v[2];
    __shared__ uint32_t s_lo[2], s_hi[2];
    unsigned phase[2] = {0u, 0u};
    float smax_l = 0.0f;
    const int ntiles = (int)*ntiles_p;
    constexpr bool DENSE = g2p_dense<ORDER>();
    const int lane = threadIdx.x & 31;
    if (threadIdx.x < 32) {
        int v0 = 0;
        uint32_t lo = 0u, hi = 0u;
        if (lane == 0) {
            mbar_init(&mbar[0], 1);
            mbar_init(&mbar[1], 1);
            v0 = g2p_claim<g2p_pieces<ORDER>()>(tiles, ntiles, tile_ctr + 1, lo, hi) ? 1 : 0;
            s_v[0] = v0;
            s_lo[0] = lo;
            s_hi[0] = hi;
            if (!DENSE && v0) g2p_issue<D, R>(vel, skeys[lo] >> (2 * D), c.nb, sv[0], &mbar[0]);
        }
        if (DENSE) {
            v0 = __shfl_sync(FULLMASK, v0, 0);
            lo = __shfl_sync(FULLMASK, lo, 0);
            if (v0) g2p_issue_dense<D, R>(vel, skeys[lo] >> (2 * D), c.nb, sv[0], &mbar[0], lane);
        }
    }
    __syncthreads();
    for (int buf = 0;; buf ^= 1) {
        if (!s_v[buf]) break;
        if (threadIdx.x < 32) {
            int v1 = 0;
            uint32_t lo = 0u, hi = 0u;
            if (lane == 0) {
                v1 = g2p_claim<g2p_pieces<ORDER>()>(tiles, ntiles, tile_ctr + 1, lo, hi) ? 1 : 0;
                s_v[buf ^ 1] = v1;
                s_lo[buf ^ 1] = lo;
                s_hi[buf ^ 1] = hi;
                if (!DENSE && v1) g2p_issue<D, R>(vel, skeys[lo] >> (2 * D), c.nb, sv[buf ^ 1], &mbar[buf ^ 1]);
            }
            if (DENSE) {
                v1 = __shfl_sync(FULLMASK, v1, 0);
                lo = __shfl_sync(FULLMASK, lo, 0);
                if (v1) g2p_issue_dense<D, R>(vel, skeys[lo] >> (2 * D), c.nb, sv[buf ^ 1], &mbar[buf ^ 1], lane);
            }
            if (lane == 0) {
                const bool ok = g2p_wait(&mbar[buf], phase[buf], err, c.wait_limit);
                if (!ok && v1) mbar_wait_bounded(&mbar[buf ^ 1], phase[buf ^ 1], 1u << 22);   // drain before leaving
                s_ok = ok ? 1 : 0;
            }
        }
        __syncthreads();
        if (!s_ok) return;
        g2p_compute<D, ORDER, R, EXT, G2P_THREADS>(in, out, perm, skeys, s_lo[buf], s_hi[buf], knext, c, err, fallbacks,
                                                   sv[buf], smax_l, vdel, stage);
        __syncthreads();
        phase[buf] ^= 1u;
    }
    // the CTA's speed maximum (non-negative floats order like their bit patterns)
    if (EXT && c.smax) {
        const unsigned mx = __reduce_max_sync(FULLMASK, __float_as_uint(smax_l));
        if ((threadIdx.x & 31) == 0 && mx) atomicMax(c.smax, mx);
    }
    // no copy is issued for a claim past the last item; nothing is left in flight
}

// ---------------------------------------------------------------- momentum (FP64)
__device__ __forceinline__ double warp_sum_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(FULLMASK, v, o);
    return v;
}

// writes 6 partial sums (p, l) of this CTA to part[blockIdx.x*6 ...] in a fixed order
__device__ __forceinline__ void block_sum6(double* a, double* part)
{
    __shared__ double s[6][TPB / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        const double v = warp_sum_d(a[i]);
        if (lane == 0) s[i][w] = v;
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        double t = 0.0;
        for (int ww = 0; ww < TPB / 32; ++ww) t += s[threadIdx.x][ww];
        part[(size_t)blockIdx.x * 6 + threadIdx.x] = t;
    }
}

// Exact FP32 building blocks of the FP32 momentum sums: a running sum hi + lo that takes an
// FP32 term with no error beyond the rounding of lo (Knuth's TwoSum puts the rounding error
// of hi + x into lo), and the product of two FP32 numbers as p + e exactly (e by one fused
// multiply-add).  With an FP32 state every term of the momentum is such a product or value,
// so the sums carry about 48 bits, and the FP32 pipe does what FP64 arithmetic per particle
// would otherwise do at a small fraction of its rate.
struct SumF {
    float hi, lo;
};
__device__ __forceinline__ void sumf_add(SumF& a, float x)
{
    const float s = __fadd_rn(a.hi, x);
    const float bp = __fsub_rn(s, a.hi);
    const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bp)), __fsub_rn(x, bp));
    a.hi = s;
    a.lo = __fadd_rn(a.lo, e);
}
__device__ __forceinline__ void sumf_add_prod(SumF& a, float x, float y)
{
    const float p = __fmul_rn(x, y);
    const float e = __fmaf_rn(x, y, -p);   // x y = p + e exactly
    sumf_add(a, p);
    a.lo = __fadd_rn(a.lo, e);             // |e| <= ulp(p) / 2: lo's own rounding covers it
}
__device__ __forceinline__ double sumf_value(const SumF& a) { return (double)a.hi + (double)a.lo; }

template <int D, typename R>
__global__ void __launch_bounds__(TPB) k_mom_particles(PState<R> st, DevCfg<R> c, double mass_cfg, double dx,
                                                       double o0, double o1, double o2, double* part)
{
    double a[6] = {0, 0, 0, 0, 0, 0};
    const double org[3] = {o0, o1, o2};
    if (sizeof(R) == 4 && !c.mat) {
        // FP32 state, one mass: with x = org + dx (cell + o),
        //   p = m sum v,  l = m (org x sum v + dx sum (cell + o) x v + sum B^T : eps)
        // every term of the three sums an FP32 value or an exact product of two
        SumF sv[3] = {}, sx[3] = {}, sb[3] = {};
        for (int k = blockIdx.x * TPB + threadIdx.x; k < c.n; k += gridDim.x * TPB) {
            Particle<D, R> p;
            load_x<D, R>(st, k, p);
            load_vB<D, R>(st, k, p);
            float cf[3] = {0.0f, 0.0f, 0.0f}, of[3] = {0.0f, 0.0f, 0.0f}, vf[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
            for (int d = 0; d < D; ++d) {
                cf[d] = (float)p.cell[d];   // exact: a cell index is far below 2^24
                of[d] = (float)p.o[d];
                vf[d] = (float)p.v[d];
                sumf_add(sv[d], vf[d]);
            }
            // (cell + o) x v, component q = (a b): t_a v_b - t_b v_a
#pragma unroll
            for (int q = 0; q < ((D == 3) ? 3 : 1); ++q) {
                const int ia = (D == 3) ? (q + 1) % 3 : 0, ib = (D == 3) ? (q + 2) % 3 : 1;
                const int out = (D == 3) ? q : 0;
                sumf_add_prod(sx[out], cf[ia], vf[ib]);
                sumf_add_prod(sx[out], of[ia], vf[ib]);
                sumf_add_prod(sx[out], -cf[ib], vf[ia]);
                sumf_add_prod(sx[out], -of[ib], vf[ia]);
            }
            if (c.transfer == 0) {   // (B_p)^T : eps of Sec. 5.3
                if (D == 3) {
                    sumf_add(sb[0], (float)p.B[7]);
                    sumf_add(sb[0], -(float)p.B[5]);
                    sumf_add(sb[1], (float)p.B[2]);
                    sumf_add(sb[1], -(float)p.B[6]);
                    sumf_add(sb[2], (float)p.B[3]);
                    sumf_add(sb[2], -(float)p.B[1]);
                } else {
                    sumf_add(sb[0], (float)p.B[2]);
                    sumf_add(sb[0], -(float)p.B[1]);
                }
            }
        }
        double v[3], x[3], b[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            v[d] = sumf_value(sv[d]);
            x[d] = sumf_value(sx[d]);
            b[d] = sumf_value(sb[d]);
        }
#pragma unroll
        for (int d = 0; d < D; ++d) a[d] = mass_cfg * v[d];
        if (D == 3) {
            a[3] = mass_cfg * (org[1] * v[2] - org[2] * v[1] + dx * x[0] + b[0]);
            a[4] = mass_cfg * (org[2] * v[0] - org[0] * v[2] + dx * x[1] + b[1]);
            a[5] = mass_cfg * (org[0] * v[1] - org[1] * v[0] + dx * x[2] + b[2]);
        } else {
            a[3] = mass_cfg * (org[0] * v[1] - org[1] * v[0] + dx * x[0] + b[0]);
        }
        block_sum6(a, part);
        return;
    }
    // FP64 state or a mass per particle: every particle's terms in FP64 from its state
    // widened exactly (the position as origin + (cell + offset) dx, so the offset keeps its
    // full precision), sums in FP64
    for (int k = blockIdx.x * TPB + threadIdx.x; k < c.n; k += gridDim.x * TPB) {
        Particle<D, R> p;
        load_x<D, R>(st, k, p);
        load_vB<D, R>(st, k, p);
        const double mass = c.mat ? (double)ld4(st.M + k).z : mass_cfg;
        double x[3] = {0.0, 0.0, 0.0}, v[3] = {0.0, 0.0, 0.0};
#pragma unroll
        for (int d = 0; d < D; ++d) {
            x[d] = org[d] + ((double)p.cell[d] + (double)p.o[d]) * dx;
            v[d] = mass * (double)p.v[d];
            a[d] += v[d];
        }
        if (D == 3) {
            double l[3] = {x[1] * v[2] - x[2] * v[1], x[2] * v[0] - x[0] * v[2], x[0] * v[1] - x[1] * v[0]};
            if (c.transfer == 0) {   // m_p (B_p)^T : eps of Sec. 5.3
                l[0] += mass * ((double)p.B[7] - (double)p.B[5]);
                l[1] += mass * ((double)p.B[2] - (double)p.B[6]);
                l[2] += mass * ((double)p.B[3] - (double)p.B[1]);
            }
            a[3] += l[0];
            a[4] += l[1];
            a[5] += l[2];
        } else {
            double l = x[0] * v[1] - x[1] * v[0];
            if (c.transfer == 0) l += mass * ((double)p.B[2] - (double)p.B[1]);
            a[3] += l;
        }
    }
    block_sum6(a, part);
}

// which = 0: accumulation grid (lanes 0..D-1 = momentum); 1: velocity grid (m v~)
template <int D, typename R>
__global__ void __launch_bounds__(TPB) k_mom_grid(const R* __restrict__ grid, int which, DevCfg<R> c, double dx,
                                                  double o0, double o1, double o2, double* part)
{
    constexpr int BN = (D == 3) ? 64 : 16;
    double a[6] = {0, 0, 0, 0, 0, 0};
    const double org[3] = {o0, o1, o2};
    const int64_t total = (int64_t)c.nblocks * BN;
    for (int64_t node = (int64_t)blockIdx.x * TPB + threadIdx.x; node < total; node += (int64_t)gridDim.x * TPB) {
        const int b = (int)(node / BN), i = (int)(node % BN);
        int bc[3] = {0, 0, 0};
        block_coords<D, R>((uint32_t)b, c, bc);
        int g[3] = {bc[0] * 4 + (i & 3), bc[1] * 4 + ((i >> 2) & 3), (D == 3) ? bc[2] * 4 + (i >> 4) : 0};
        const R* q = grid + 4 * node;
        const double m = (double)q[3];
        if (m == 0.0) continue;
        double x[3] = {0, 0, 0}, mv[3] = {0, 0, 0};
#pragma unroll
        for (int d = 0; d < D; ++d) {
            x[d] = org[d] + (double)g[d] * dx;
            mv[d] = which == 0 ? (double)q[d] : m * (double)q[d];
            a[d] += mv[d];
        }
        if (D == 3) {
            a[3] += x[1] * mv[2] - x[2] * mv[1];
            a[4] += x[2] * mv[0] - x[0] * mv[2];
            a[5] += x[0] * mv[1] - x[1] * mv[0];
        } else {
            a[3] += x[0] * mv[1] - x[1] * mv[0];
        }
    }
    block_sum6(a, part);
}

template <typename R>
__global__ void __launch_bounds__(TPB) k_mom_final(const double* __restrict__ part, int np, double* __restrict__ out)
{
    __shared__ double s[6][TPB];
    for (int i = 0; i < 6; ++i) {
        double t = 0.0;
        for (int b = threadIdx.x; b < np; b += TPB) t += part[(size_t)b * 6 + i];
        s[i][threadIdx.x] = t;
    }
    __syncthreads();
    for (int st = TPB / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st)
            for (int i = 0; i < 6; ++i) s[i][threadIdx.x] += s[i][threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x < 6) out[threadIdx.x] = s[threadIdx.x][0];
}

// Sec. 4.3: per-CTA max of |v_p| + (6 sqrt(d) / dx) |B_p|_F into part[blockIdx.x * 6]
template <int D, typename R>
__global__ void __launch_bounds__(TPB) k_cfl_particles(PState<R> st, DevCfg<R> c, double coef, double* part)
{
    __shared__ double s[TPB / 32];
    double mx = 0.0;
    for (int k = blockIdx.x * TPB + threadIdx.x; k < c.n; k += gridDim.x * TPB) {
        Particle<D, R> p;
        load_vB<D, R>(st, k, p);
        double sv = 0.0, sb = 0.0;
#pragma unroll
        for (int a = 0; a < D; ++a) sv += (double)p.v[a] * (double)p.v[a];
#pragma unroll
        for (int i = 0; i < D * D; ++i) sb += (double)p.B[i] * (double)p.B[i];
        mx = fmax(mx, sqrt(sv) + coef * sqrt(sb));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_down_sync(FULLMASK, mx, o));
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < TPB / 32; ++w) t = fmax(t, s[w]);
        part[(size_t)blockIdx.x * 6] = t;
    }
}

template <typename R>
__global__ void __launch_bounds__(TPB) k_max_final(const double* __restrict__ part, int np, double* __restrict__ out)
{
    __shared__ double s[TPB];
    double t = 0.0;
    for (int b = threadIdx.x; b < np; b += TPB) t = fmax(t, part[(size_t)b * 6]);
    s[threadIdx.x] = t;
    __syncthreads();
    for (int st = TPB / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) s[threadIdx.x] = fmax(s[threadIdx.x], s[threadIdx.x + st]);
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = s[0];
}

// ---------------------------------------------------------------- upload / download
template <int D, typename R>
__global__ void __launch_bounds__(TPB) k_upload(PState<R> st, DevCfg<R> c, double dx, double o0, double o1, double o2,
                                                const double* __restrict__ x, const double* __restrict__ v,
                                                const double* __restrict__ B, const double* __restrict__ F,
                                                uint32_t* err, uint32_t* fallbacks, int64_t k0, int64_t k1)
{
    // particles [k0, k1) of the upload (a host upload runs in pieces, each after its copies)
    const int64_t k = k0 + (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (k >= k1) return;
    const double org[3] = {o0, o1, o2};
    Particle<D, R> p;
    p.id = (uint32_t)k;
    // a non-finite input value is reported (the particle is stored with zeros in its place)
    bool finite = true;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        finite &= isfinite(x[(size_t)k * D + a]);
        if (v) finite &= isfinite(v[(size_t)k * D + a]);
    }
#pragma unroll
    for (int i = 0; i < D * D; ++i) {
        if (B) finite &= isfinite(B[(size_t)k * D * D + i]);
        if (F) finite &= isfinite(F[(size_t)k * D * D + i]);
    }
    if (!finite) {
        set_err(err, APIC_ERRBIT_NONFINITE);
        x = nullptr;
        v = nullptr;
        B = nullptr;
        F = nullptr;
    }
#pragma unroll
    for (int a = 0; a < D; ++a) {
        const double u = x ? (x[(size_t)k * D + a] - org[a]) / dx : 0.0;
        double cl = floor(u);
        R o = (R)(u - cl);
        if (o >= R(1)) { o = R(0); cl += 1.0; }
        int ci = (int)cl;
        if (!(cl >= 0.0) || cl > (double)(c.res[a] - 1)) {
            set_err(err, APIC_ERRBIT_RANGE);
            ci = cl < 0.0 ? 0 : c.res[a] - 1;
            o = R(0);
        }
        p.o[a] = o;
        p.cell[a] = ci;
        p.v[a] = v ? (R)v[(size_t)k * D + a] : R(0);
    }
#pragma unroll
    for (int i = 0; i < D * D; ++i) {
        p.B[i] = B ? (R)B[(size_t)k * D * D + i] : R(0);
        p.F[i] = F ? (R)F[(size_t)k * D * D + i] : ((i % (D + 1)) == 0 ? R(1) : R(0));
    }
    if (c.model != 0) stress_sym<D, R>(c.model, p.F, c.mu, c.lam, c.vol, p.tau, fallbacks);
    store_all<D, R>(st, k, p, c.model != 0);
}

// a material per particle: Lame parameters from (E, nu) given in upload order (index = id),
// stored in lane M of the particle wherever it now sits, and its stress recomputed
template <int D, typename R>
__global__ void __launch_bounds__(TPB) k_set_params(PState<R> st, DevCfg<R> c, const double* __restrict__ E,
                                                    const double* __restrict__ nu, const double* __restrict__ mass,
                                                    const double* __restrict__ vol, int keep, uint32_t* fallbacks,
                                                    uint32_t* err)
{
    const int k = blockIdx.x * TPB + threadIdx.x;
    if (k >= c.n) return;
    Particle<D, R> p;
    load_xF<D, R>(st, k, p);
    load_vB<D, R>(st, k, p);
    if (p.id >= (uint32_t)c.n) {   // an id is an upload index; anything else is not valid state
        set_err(err, APIC_ERRBIT_RANGE);
        return;
    }
    // what is not given keeps the particle's earlier value (keep) or the configuration's
    if (keep) {
        load_mat<D, R>(st, k, p);
    } else {
        p.mu = c.mu;
        p.lam = c.lam;
        p.pm = c.mass;
        p.pv = c.vol;
    }
    if (E) {
        const double e = E[p.id], v = nu[p.id];
        p.mu = (R)(e / (2.0 * (1.0 + v)));
        p.lam = (R)(e * v / ((1.0 + v) * (1.0 - 2.0 * v)));
    }
    if (mass) {
        p.pm = (R)mass[p.id];
        p.pv = (R)vol[p.id];
    }
    if (c.model != 0) stress_sym<D, R>(c.model, p.F, p.mu, p.lam, p.pv, p.tau, fallbacks);
    store_all<D, R>(st, k, p, c.model != 0, true);
}

// adaptive time step (Sec. 4.3): dt = min(dt_max, nu dx / speed), speed = the FP64 reduction
// of the current state (first) or the maximum G2P reduced into smax (after a step, whose dt
// is first added to the elapsed time); one thread
template <typename R>
__global__ void k_adapt_dt(R* dtw, const uint32_t* smax, const double* speed64, double* elapsed, double dx,
                           double nu, double dt_max, int first)
{
    if (first) *elapsed = 0.0;
    else *elapsed += (double)*dtw;
    const double sp = first ? speed64[0] : (double)__uint_as_float(*smax);
    const double dt = sp > 0.0 ? fmin(dt_max, nu * dx / sp) : dt_max;
    *dtw = (R)dt;
}

// inv[id] = the storage slot of the particle uploaded at index id (inv filled with ~0 first);
// an id out of range is not valid state and is reported
template <int D, typename R>
__global__ void __launch_bounds__(TPB) k_inverse_ids(PState<R> st, DevCfg<R> c, uint32_t* __restrict__ inv,
                                                     uint32_t* err)
{
    const int k = blockIdx.x * TPB + threadIdx.x;
    if (k >= c.n) return;
    const uint32_t id = (D == 3) ? r2u(ld2(st.Fc + k).y) : r2u(ld4(st.A + k).w);
    if (id >= (uint32_t)c.n) {
        set_err(err, APIC_ERRBIT_RANGE);
        return;
    }
    inv[id] = (uint32_t)k;
}

// the particles uploaded at indices [id0, id1), read through inv and written in upload order
// (a host download gathers in pieces so that each piece's copies can start early)
template <int D, typename R>
__global__ void __launch_bounds__(TPB) k_download_ids(PState<R> st, DevCfg<R> c, double dx, double o0, double o1,
                                                      double o2, const uint32_t* __restrict__ inv, int64_t id0,
                                                      int64_t id1, double* __restrict__ x, double* __restrict__ v,
                                                      double* __restrict__ B, double* __restrict__ F, uint32_t* err)
{
    const int64_t id = id0 + (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (id >= id1) return;
    const uint32_t k = inv[id];
    if (k >= (uint32_t)c.n) {   // no particle carries this id: not valid state
        set_err(err, APIC_ERRBIT_RANGE);
        return;
    }
    const double org[3] = {o0, o1, o2};
    Particle<D, R> p;
    load_xF<D, R>(st, k, p);
    load_vB<D, R>(st, k, p);
#pragma unroll
    for (int a = 0; a < D; ++a) {
        if (x) x[id * D + a] = org[a] + ((double)p.cell[a] + (double)p.o[a]) * dx;
        if (v) v[id * D + a] = (double)p.v[a];
    }
#pragma unroll
    for (int i = 0; i < D * D; ++i) {
        if (B) B[id * D * D + i] = (double)p.B[i];
        if (F) F[id * D * D + i] = (double)p.F[i];
    }
}

template <int D, typename R>
__global__ void __launch_bounds__(TPB) k_download(PState<R> st, DevCfg<R> c, double dx, double o0, double o1, double o2,
                                                  double* __restrict__ x, double* __restrict__ v, double* __restrict__ B,
                                                  double* __restrict__ F, int32_t* __restrict__ cell,
                                                  double* __restrict__ off, uint32_t* err)
{
    const int k = blockIdx.x * TPB + threadIdx.x;
    if (k >= c.n) return;
    const double org[3] = {o0, o1, o2};
    Particle<D, R> p;
    load_xF<D, R>(st, k, p);
    load_vB<D, R>(st, k, p);
    const size_t id = p.id;
    if (id >= (size_t)c.n) {   // not valid state (e.g. a step whose G2P gave up): write nothing
        set_err(err, APIC_ERRBIT_RANGE);
        return;
    }
#pragma unroll
    for (int a = 0; a < D; ++a) {
        if (x) x[id * D + a] = org[a] + ((double)p.cell[a] + (double)p.o[a]) * dx;
        if (v) v[id * D + a] = (double)p.v[a];
        if (cell) cell[id * D + a] = p.cell[a];
        if (off) off[id * D + a] = (double)p.o[a];
    }
#pragma unroll
    for (int i = 0; i < D * D; ++i) {
        if (B) B[id * D * D + i] = (double)p.B[i];
        if (F) F[id * D * D + i] = (double)p.F[i];
    }
}

template <int D, typename R>
__global__ void __launch_bounds__(TPB) k_grid_dense(const R* __restrict__ grid, int which, DevCfg<R> c,
                                                    double* __restrict__ m, double* __restrict__ mv)
{
    const int64_t nn = (int64_t)c.res[0] * c.res[1] * (D == 3 ? c.res[2] : 1);
    for (int64_t idx = (int64_t)blockIdx.x * TPB + threadIdx.x; idx < nn; idx += (int64_t)gridDim.x * TPB) {
        int g[3];
        int64_t r = idx;
        g[0] = (int)(r % c.res[0]); r /= c.res[0];
        g[1] = (int)(r % c.res[1]); r /= c.res[1];
        g[2] = (D == 3) ? (int)r : 0;
        const uint32_t ni = node_index<D>(g, c.nb);
        const R* q = grid + 4 * (size_t)ni;
        m[idx] = (double)q[3];
        for (int a = 0; a < D; ++a) mv[idx * D + a] = (double)q[a];
        (void)which;
    }
}

}  // namespace apic

#include "apic_lambda1.cuh"
#include "apic_implicit.cuh"

namespace apic {

// ---------------------------------------------------------------- launchers
inline unsigned blocks_for(int64_t n) { return (unsigned)((n + TPB - 1) / TPB); }

#define APIC_DISPATCH(c, KERNEL_CALL)                                                  \
    do {                                                                               \
        if ((c).dim == 3 && (c).order == 2) { constexpr int D = 3, O = 2; KERNEL_CALL; } \
        else if ((c).dim == 3 && (c).order == 3) { constexpr int D = 3, O = 3; KERNEL_CALL; } \
        else if ((c).dim == 2 && (c).order == 2) { constexpr int D = 2, O = 2; KERNEL_CALL; } \
        else { constexpr int D = 2, O = 3; KERNEL_CALL; }                              \
    } while (0)

template <typename R> struct Impl {
    static cudaError_t keys(const HostCfg& h, const Buffers& b, int cur, int64_t n, cudaStream_t s)
    {
        if (n == 0) return cudaSuccess;
        DevCfg<R> c = HostToDev<R>::make(h, n);
        PState<R> st = state_of<R>(b, cur);
        APIC_DISPATCH(h, (k_keys<D, O, R><<<blocks_for(n), TPB, 0, s>>>(st, c, b.knext, b.err)));
        return cudaGetLastError();
    }
    static cudaError_t p2g(const HostCfg& h, const Buffers& b, int cur, const uint32_t* sk, const uint32_t* perm,
                           int64_t n, const Launch& L, cudaStream_t s)
    {
        if (n == 0) return cudaSuccess;
        DevCfg<R> c0 = HostToDev<R>::make(h, b, n);
        // lambda = 1 and the midpoint rule transfer mass and momentum alone: their force is taken
        // after the grid velocity v_i
        if (h.integrator != 0) c0.model = 0;
        PState<R> st = state_of<R>(b, cur);
        auto launch = [&](const DevCfg<R>& c, R* acc) {
        cudaError_t e = cudaSuccess;
        if (h.dim == 3 && h.p2g_kernel == 1) {
            if (h.order == 2)
                e = launch_pdl(k_p2g_split<2, R>, dim3(L.p2g_grid), dim3(SplitShape<2>::NT), p2g_split_smem<2, R>(), s,
                               st, perm, sk, b.tiles, b.ntiles, b.tile_ctr, acc, b.flags, c, b.err);
            else
                e = launch_pdl(k_p2g_split<3, R>, dim3(L.p2g_grid), dim3(SplitShape<3>::NT), p2g_split_smem<3, R>(), s,
                               st, perm, sk, b.tiles, b.ntiles, b.tile_ctr, acc, b.flags, c, b.err);
        } else if (h.p2g_group == 2)
            APIC_DISPATCH(h, (e = launch_pdl(k_p2g_cells<D, O, R, 2>, dim3(L.p2g_grid), dim3(128),
                                             p2g_cells_launch_smem<D, O, R>(), s, st, perm, sk, b.tiles, b.ntiles,
                                             b.tile_ctr, acc, b.flags, c, b.err, b.fallbacks)));
        else
            APIC_DISPATCH(h, (e = launch_pdl(k_p2g_cells<D, O, R, 4>, dim3(L.p2g_grid), dim3(128),
                                             p2g_cells_launch_smem<D, O, R>(), s, st, perm, sk, b.tiles, b.ntiles,
                                             b.tile_ctr, acc, b.flags, c, b.err, b.fallbacks)));
        return e;
        };
        cudaError_t e = launch(c0, (R*)b.acc);
        if (e == cudaSuccess && h.transfer == 2) {
            // FLIP keeps the grid velocity before the update: a second pass sums the PIC
            // momentum alone (no stress, no affine term) into acc2
            DevCfg<R> c2 = c0;
            c2.model = 0;
            c2.transfer = 1;
            e = cudaMemsetAsync(b.tile_ctr, 0, sizeof(uint32_t), s);
            if (e == cudaSuccess) e = launch(c2, (R*)b.acc2);
        }
        return e;
    }
    static cudaError_t grid_update(const HostCfg& h, const Buffers& b, const Launch& L, cudaStream_t s)
    {
        DevCfg<R> c = HostToDev<R>::make(h, b, 0);
        const int grid = L.sms * 8;
        if (h.dim == 3)
            return launch_pdl(k_grid_update<3, R>, dim3(grid), dim3(TPB), 0, s, (R*)b.acc, (R*)b.vel, b.flags, c,
                              (R*)b.acc2, (R*)b.vdel);
        return launch_pdl(k_grid_update<2, R>, dim3(grid), dim3(TPB), 0, s, (R*)b.acc, (R*)b.vel, b.flags, c,
                          (R*)b.acc2, (R*)b.vdel);
    }
    static cudaError_t g2p(const HostCfg& h, const Buffers& b, int cur, const uint32_t* sk, const uint32_t* perm,
                           int64_t n, const Launch& L, cudaStream_t s)
    {
        if (n == 0) return cudaSuccess;
        DevCfg<R> c = HostToDev<R>::make(h, b, n);
        PState<R> in = state_of<R>(b, cur), out = state_of<R>(b, cur ^ 1);
        cudaError_t e = cudaSuccess;
        if (h.mat || h.adaptive || h.transfer == 2)
            APIC_DISPATCH(h, (e = launch_pdl(k_g2p<D, O, R, true>, dim3(L.g2p_grid), dim3(G2P_THREADS), 0, s, in, out,
                                             perm, sk, b.tiles, b.ntiles, b.tile_ctr, (const R*)b.vel, b.knext, c,
                                             b.err, b.fallbacks, (const R*)b.vdel)));
        else
            APIC_DISPATCH(h, (e = launch_pdl(k_g2p<D, O, R, false>, dim3(L.g2p_grid), dim3(G2P_THREADS), 0, s, in, out,
                                             perm, sk, b.tiles, b.ntiles, b.tile_ctr, (const R*)b.vel, b.knext, c,
                                             b.err, b.fallbacks, nullptr)));
        return e;
    }
    // the grid phase of the lambda = 1 member: grid velocity, the force at F^{n+1}, the update
    static cudaError_t grid_update_lambda1(const HostCfg& h, const Buffers& b, int cur, const uint32_t* sk,
                                           const uint32_t* perm, int64_t n, const Launch& L, cudaStream_t s)
    {
        DevCfg<R> c = HostToDev<R>::make(h, b, n);
        const int grid = L.sms * 8;
        if (h.dim == 3) k_grid_velocity<3, R><<<grid, TPB, 0, s>>>((R*)b.acc, (R*)b.vel1, b.flags, c);
        else k_grid_velocity<2, R><<<grid, TPB, 0, s>>>((R*)b.acc, (R*)b.vel1, b.flags, c);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess && h.model != 0 && n > 0) {
            e = cudaMemsetAsync(b.tile_ctr + 3, 0, sizeof(uint32_t), s);
            PState<R> st = state_of<R>(b, cur);
            if (e == cudaSuccess)
                APIC_DISPATCH(h, (k_force_lambda1<D, O, R><<<L.sms * 4, 128, 0, s>>>(
                                     st, perm, sk, b.tiles, b.ntiles, b.tile_ctr + 3, (const R*)b.vel1, (R*)b.acc, c,
                                     b.err, b.fallbacks)));
            if (e == cudaSuccess) e = cudaGetLastError();
        }
        if (e == cudaSuccess) {
            if (h.dim == 3) k_grid_update_lambda1<3, R><<<grid, TPB, 0, s>>>((R*)b.acc, (R*)b.vel, (const R*)b.vel1, b.flags, c);
            else k_grid_update_lambda1<2, R><<<grid, TPB, 0, s>>>((R*)b.acc, (R*)b.vel, (const R*)b.vel1, b.flags, c);
            e = cudaGetLastError();
        }
        return e;
    }
    static cudaError_t g2p_lambda1(const HostCfg& h, const Buffers& b, int cur, const uint32_t* perm, int64_t n,
                                   const Launch& L, cudaStream_t s)
    {
        if (n == 0) return cudaSuccess;
        DevCfg<R> c = HostToDev<R>::make(h, b, n);
        PState<R> in = state_of<R>(b, cur), out = state_of<R>(b, cur ^ 1);
        const unsigned grid = (unsigned)std::min<int64_t>((n + 127) / 128, (int64_t)L.sms * 16);
        const R* ugrid = (const R*)(h.integrator == 2 ? b.su : b.vel1);   // midpoint: u = (v + v~) / 2
        APIC_DISPATCH(h, (k_g2p_general<D, O, R><<<grid, 128, 0, s>>>(in, out, perm, (const R*)b.vel, ugrid,
                                                                       b.knext, c, b.err)));
        return cudaGetLastError();
    }
    // <., .>_M partials of one solve step (per CTA) summed into mom_out[0] and read back
    static cudaError_t read_dot(const Buffers& b, int parts, cudaStream_t s, double* out)
    {
        k_sum_partials<R><<<1, TPB, 0, s>>>(b.mom_part, parts, b.mom_out);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(out, b.mom_out, sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        return e;
    }
    // The grid phase of the implicit midpoint rule: v_i = (m v)_i / m_i, Newton on dv with CG in
    // the mass inner product for each system (Algorithm 1), then v~ = v + dv and the displacement
    // velocity u = (v + v~) / 2 for G2P.  The scalars of each iteration are read back to the host,
    // which takes the decisions of the algorithm.  stats: [0] Newton iterations, [1] CG
    // iterations, [2] the last Newton residual relative to |v|_M (as doubles).
    static cudaError_t grid_update_midpoint(const HostCfg& h, const Buffers& b, int cur, const uint32_t* sk,
                                            const uint32_t* perm, int64_t n, const Launch& L, cudaStream_t s,
                                            double* stats, int64_t* kernels)
    {
        DevCfg<R> c = HostToDev<R>::make(h, b, n);
        const int ggrid = L.sms * 8;
        const int parts = L.mom_parts;
        const double dt = h.dt;
        SolveVecs sv{b.vel1, b.sdv, b.su, b.sr, b.sp, b.ss, b.sdu, b.acc, b.vel};
        stats[0] = stats[1] = stats[2] = 0.0;
        cudaError_t e = cudaSuccess;
        auto step = [&](int op, double a) {
            if (e != cudaSuccess) return;
            if (h.dim == 3) k_solve_step<3, R><<<parts, TPB, 0, s>>>(sv, b.flags, c, op, a, b.mom_part);
            else k_solve_step<2, R><<<parts, TPB, 0, s>>>(sv, b.flags, c, op, a, b.mom_part);
            e = cudaGetLastError();
            *kernels += 1;
        };
        auto force = [&](bool diff) {
            if (e != cudaSuccess || h.model == 0 || n == 0) return;
            e = cudaMemsetAsync(b.tile_ctr + 3, 0, sizeof(uint32_t), s);
            PState<R> st = state_of<R>(b, cur);
            if (e != cudaSuccess) return;
            if (diff)
                APIC_DISPATCH(h, (k_force_diff<D, O, R><<<L.sms * 4, 128, 0, s>>>(st, perm, sk, b.tiles, b.ntiles,
                                     b.tile_ctr + 3, (const R*)b.su, (const R*)b.sp, (R*)b.acc, R(1), c, b.err,
                                     b.fallbacks)));
            else
                APIC_DISPATCH(h, (k_force_lambda1<D, O, R><<<L.sms * 4, 128, 0, s>>>(st, perm, sk, b.tiles, b.ntiles,
                                     b.tile_ctr + 3, (const R*)b.su, (R*)b.acc, c, b.err, b.fallbacks)));
            e = cudaGetLastError();
            *kernels += 1;
        };
        if (h.dim == 3) k_grid_velocity<3, R><<<ggrid, TPB, 0, s>>>((R*)b.acc, (R*)b.vel1, b.flags, c);
        else k_grid_velocity<2, R><<<ggrid, TPB, 0, s>>>((R*)b.acc, (R*)b.vel1, b.flags, c);
        e = cudaGetLastError();
        *kernels += 1;
        // dv = 0 and |v|_M (from u = v / 2 + dv / 4 with dv = 0: |v|_M^2 = 4 <u, u>_M, taken with
        // op 1 on a zero force: r = -dv = 0 is not it, so use the velocity itself)
        const size_t gbytes = (size_t)h.nblocks * (h.dim == 3 ? 64 : 16) * 4 * sizeof(R);
        if (e == cudaSuccess) e = cudaMemsetAsync(b.sdv, 0, gbytes, s);
        double vnorm2 = 0.0;
        if (e == cudaSuccess) {
            if (h.dim == 3) k_solve_step<3, R><<<parts, TPB, 0, s>>>(SolveVecs{b.vel1, b.sdv, b.su, b.sr, b.sp, b.ss, b.sdu, b.vel1, b.vel},
                                                                       b.flags, c, 7, 0.0, b.mom_part);
            else k_solve_step<2, R><<<parts, TPB, 0, s>>>(SolveVecs{b.vel1, b.sdv, b.su, b.sr, b.sp, b.ss, b.sdu, b.vel1, b.vel},
                                                            b.flags, c, 7, 0.0, b.mom_part);
            e = cudaGetLastError();
            *kernels += 1;
        }
        if (e == cudaSuccess) e = read_dot(b, parts, s, &vnorm2);
        const double vnorm = sqrt(vnorm2) > 1e-300 ? sqrt(vnorm2) : 1e-300;
        for (int it = 0; it < h.newton_max && e == cudaSuccess; ++it) {
            step(0, 0.0);                       // u = v / 2 + dv / 4
            force(false);                       // acc = dt f at x + dt u
            double rr = 0.0;
            step(1, 0.0);                       // r = dt f / m - dv, p = r, du = 0
            if (e == cudaSuccess) e = read_dot(b, parts, s, &rr);
            const double rn0 = sqrt(rr);
            stats[2] = rn0 / vnorm;
            if (e != cudaSuccess || rn0 <= h.solve_tol * vnorm) break;
            stats[0] += 1.0;
            double gamma = rr;
            for (int k = 0; k < h.cg_max && gamma > 0.0 && e == cudaSuccess; ++k) {
                force(true);                    // acc = df/dx~ p
                double ps = 0.0;
                step(2, 0.0);                   // s = p - dt^2/4 acc / m
                if (e == cudaSuccess) e = read_dot(b, parts, s, &ps);
                if (e != cudaSuccess || !(ps > 0.0)) break;
                const double alpha = gamma / ps;
                double kappa = 0.0;
                step(3, alpha);                 // du += alpha p, r -= alpha s
                if (e == cudaSuccess) e = read_dot(b, parts, s, &kappa);
                stats[1] += 1.0;
                if (e != cudaSuccess || sqrt(kappa) <= h.solve_tol * rn0) break;
                step(4, kappa / gamma);         // p = r + beta p
                gamma = kappa;
            }
            step(5, 0.0);                       // dv += du
        }
        step(6, 0.0);                           // v~ = v + dv, u = (v + v~) / 2
        if (e == cudaSuccess) {
            k_clear_flags<R><<<ggrid, TPB, 0, s>>>(b.flags, h.nblocks);
            e = cudaGetLastError();
            *kernels += 1;
        }
        (void)dt;
        return e;
    }
    static cudaError_t adapt_dt(const HostCfg& h, const Buffers& b, double nu, double dt_max, int first, cudaStream_t s)
    {
        k_adapt_dt<R><<<1, 1, 0, s>>>((R*)b.dt_word, b.smax_word, b.mom_out, b.elapsed, h.dx, nu, dt_max, first);
        return cudaGetLastError();
    }
    static cudaError_t set_params(const HostCfg& h, const Buffers& b, int cur, int64_t n, const double* E,
                                  const double* nu, const double* mass, const double* vol, int keep, cudaStream_t s)
    {
        if (n == 0) return cudaSuccess;
        DevCfg<R> c = HostToDev<R>::make(h, n);
        PState<R> st = state_of<R>(b, cur);
        if (h.dim == 3) k_set_params<3, R><<<blocks_for(n), TPB, 0, s>>>(st, c, E, nu, mass, vol, keep, b.fallbacks, b.err);
        else k_set_params<2, R><<<blocks_for(n), TPB, 0, s>>>(st, c, E, nu, mass, vol, keep, b.fallbacks, b.err);
        return cudaGetLastError();
    }
    static cudaError_t upload(const HostCfg& h, const Buffers& b, int cur, int64_t n, const double* x,
                              const double* v, const double* B, const double* F, cudaStream_t s, int64_t k0,
                              int64_t k1)
    {
        if (k1 <= k0) return cudaSuccess;
        DevCfg<R> c = HostToDev<R>::make(h, n);
        PState<R> st = state_of<R>(b, cur);
        const int g = blocks_for(k1 - k0);
        if (h.dim == 3)
            k_upload<3, R><<<g, TPB, 0, s>>>(st, c, h.dx, h.origin[0], h.origin[1], h.origin[2], x, v, B, F, b.err, b.fallbacks, k0, k1);
        else
            k_upload<2, R><<<g, TPB, 0, s>>>(st, c, h.dx, h.origin[0], h.origin[1], h.origin[2], x, v, B, F, b.err, b.fallbacks, k0, k1);
        return cudaGetLastError();
    }
    static cudaError_t inverse_ids(const HostCfg& h, const Buffers& b, int cur, int64_t n, uint32_t* inv,
                                   cudaStream_t s)
    {
        if (n == 0) return cudaSuccess;
        DevCfg<R> c = HostToDev<R>::make(h, n);
        PState<R> st = state_of<R>(b, cur);
        cudaError_t e = cudaMemsetAsync(inv, 0xff, sizeof(uint32_t) * (size_t)n, s);
        if (e != cudaSuccess) return e;
        if (h.dim == 3) k_inverse_ids<3, R><<<blocks_for(n), TPB, 0, s>>>(st, c, inv, b.err);
        else k_inverse_ids<2, R><<<blocks_for(n), TPB, 0, s>>>(st, c, inv, b.err);
        return cudaGetLastError();
    }
    static cudaError_t download_ids(const HostCfg& h, const Buffers& b, int cur, int64_t n, const uint32_t* inv,
                                    int64_t id0, int64_t id1, double* x, double* v, double* B, double* F,
                                    cudaStream_t s)
    {
        if (id1 <= id0) return cudaSuccess;
        DevCfg<R> c = HostToDev<R>::make(h, n);
        PState<R> st = state_of<R>(b, cur);
        const int g = blocks_for(id1 - id0);
        if (h.dim == 3)
            k_download_ids<3, R><<<g, TPB, 0, s>>>(st, c, h.dx, h.origin[0], h.origin[1], h.origin[2], inv, id0, id1, x, v, B, F, b.err);
        else
            k_download_ids<2, R><<<g, TPB, 0, s>>>(st, c, h.dx, h.origin[0], h.origin[1], h.origin[2], inv, id0, id1, x, v, B, F, b.err);
        return cudaGetLastError();
    }
    static cudaError_t download(const HostCfg& h, const Buffers& b, int cur, int64_t n, double* x, double* v,
                                double* B, double* F, int32_t* cell, double* off, cudaStream_t s)
    {
        if (n == 0) return cudaSuccess;
        DevCfg<R> c = HostToDev<R>::make(h, n);
        PState<R> st = state_of<R>(b, cur);
        if (h.dim == 3)
            k_download<3, R><<<blocks_for(n), TPB, 0, s>>>(st, c, h.dx, h.origin[0], h.origin[1], h.origin[2], x, v, B, F, cell, off, b.err);
        else
            k_download<2, R><<<blocks_for(n), TPB, 0, s>>>(st, c, h.dx, h.origin[0], h.origin[1], h.origin[2], x, v, B, F, cell, off, b.err);
        return cudaGetLastError();
    }
    static cudaError_t momentum(const HostCfg& h, const Buffers& b, int cur, int64_t n, int where, int grid_phase,
                                const Launch& L, cudaStream_t s)
    {
        const int nparts = L.mom_parts;
        DevCfg<R> c = HostToDev<R>::make(h, n);
        if (where == 0) {
            PState<R> st = state_of<R>(b, cur);
            if (h.dim == 3)
                k_mom_particles<3, R><<<nparts, TPB, 0, s>>>(st, c, h.mass, h.dx, h.origin[0], h.origin[1], h.origin[2], b.mom_part);
            else
                k_mom_particles<2, R><<<nparts, TPB, 0, s>>>(st, c, h.mass, h.dx, h.origin[0], h.origin[1], h.origin[2], b.mom_part);
        } else {
            const R* g = (const R*)(grid_phase == 0 ? b.acc : b.vel);
            if (h.dim == 3)
                k_mom_grid<3, R><<<nparts, TPB, 0, s>>>(g, grid_phase, c, h.dx, h.origin[0], h.origin[1], h.origin[2], b.mom_part);
            else
                k_mom_grid<2, R><<<nparts, TPB, 0, s>>>(g, grid_phase, c, h.dx, h.origin[0], h.origin[1], h.origin[2], b.mom_part);
        }
        k_mom_final<R><<<1, TPB, 0, s>>>(b.mom_part, nparts, b.mom_out);
        return cudaGetLastError();
    }
    static cudaError_t cfl(const HostCfg& h, const Buffers& b, int cur, int64_t n, const Launch& L, cudaStream_t s)
    {
        DevCfg<R> c = HostToDev<R>::make(h, n);
        PState<R> st = state_of<R>(b, cur);
        const double coef = 6.0 * sqrt((double)h.dim) / h.dx;   // (kappa / k) dx of Sec. 4.3, both splines
        if (h.dim == 3) k_cfl_particles<3, R><<<L.mom_parts, TPB, 0, s>>>(st, c, coef, b.mom_part);
        else k_cfl_particles<2, R><<<L.mom_parts, TPB, 0, s>>>(st, c, coef, b.mom_part);
        k_max_final<R><<<1, TPB, 0, s>>>(b.mom_part, L.mom_parts, b.mom_out);
        return cudaGetLastError();
    }
    static cudaError_t grid_dense(const HostCfg& h, const Buffers& b, int which, double* m, double* mv, cudaStream_t s)
    {
        DevCfg<R> c = HostToDev<R>::make(h, 0);
        const R* g = (const R*)(which == 0 ? b.acc : b.vel);
        if (h.dim == 3) k_grid_dense<3, R><<<1024, TPB, 0, s>>>(g, which, c, m, mv);
        else k_grid_dense<2, R><<<1024, TPB, 0, s>>>(g, which, c, m, mv);
        return cudaGetLastError();
    }
    static cudaError_t occupancy(const HostCfg& h, int* p2g_per_sm, int* g2p_per_sm)
    {
        cudaError_t e = cudaSuccess;
        APIC_DISPATCH(h, {
            if (D == 3 && h.p2g_kernel == 1) {
                constexpr int O3 = O;
                e = cudaFuncSetAttribute(k_p2g_split<O3, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)p2g_split_smem<O3, R>());
                if (e == cudaSuccess)
                    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(p2g_per_sm, k_p2g_split<O3, R>,
                                                                      SplitShape<O3>::NT, p2g_split_smem<O3, R>());
            } else {
                // both lane groups are set up: the group can change at the next upload
                e = cudaFuncSetAttribute(k_p2g_cells<D, O, R, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)p2g_cells_launch_smem<D, O, R>());
                if (e == cudaSuccess)
                    e = cudaFuncSetAttribute(k_p2g_cells<D, O, R, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)p2g_cells_launch_smem<D, O, R>());
                int per2 = 0;
                if (e == cudaSuccess)
                    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per2, k_p2g_cells<D, O, R, 2>, 128,
                                                                      p2g_cells_launch_smem<D, O, R>());
                if (e == cudaSuccess)
                    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(p2g_per_sm, k_p2g_cells<D, O, R, 4>, 128,
                                                                      p2g_cells_launch_smem<D, O, R>());
                if (e == cudaSuccess && per2 < *p2g_per_sm) *p2g_per_sm = per2;
            }
            if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(g2p_per_sm, k_g2p<D, O, R, false>, G2P_THREADS, 0);
        });
        return e;
    }
};

#define APIC_DEFINE_PRECISION(R, SFX)                                                                         \
    cudaError_t keys_##SFX(const HostCfg& c, const Buffers& b, int cur, int64_t n, cudaStream_t s)             \
    {                                                                                                           \
        return Impl<R>::keys(c, b, cur, n, s);                                                                  \
    }                                                                                                           \
    cudaError_t p2g_##SFX(const HostCfg& c, const Buffers& b, int cur, const uint32_t* skeys,                  \
                          const uint32_t* perm, int64_t n, const Launch& L, cudaStream_t s)                     \
    {                                                                                                           \
        return Impl<R>::p2g(c, b, cur, skeys, perm, n, L, s);                                                   \
    }                                                                                                           \
    cudaError_t grid_update_##SFX(const HostCfg& c, const Buffers& b, const Launch& L, cudaStream_t s)         \
    {                                                                                                           \
        return Impl<R>::grid_update(c, b, L, s);                                                                \
    }                                                                                                           \
    cudaError_t g2p_##SFX(const HostCfg& c, const Buffers& b, int cur, const uint32_t* skeys,                  \
                          const uint32_t* perm, int64_t n, const Launch& L, cudaStream_t s)                     \
    {                                                                                                           \
        return Impl<R>::g2p(c, b, cur, skeys, perm, n, L, s);                                                   \
    }                                                                                                           \
    cudaError_t adapt_dt_##SFX(const HostCfg& c, const Buffers& b, double nu, double dt_max, int first,        \
                               cudaStream_t s)                                                                  \
    {                                                                                                           \
        return Impl<R>::adapt_dt(c, b, nu, dt_max, first, s);                                                   \
    }                                                                                                           \
    cudaError_t grid_update_lambda1_##SFX(const HostCfg& c, const Buffers& b, int cur, const uint32_t* skeys,  \
                                          const uint32_t* perm, int64_t n, const Launch& L, cudaStream_t s)     \
    {                                                                                                           \
        return Impl<R>::grid_update_lambda1(c, b, cur, skeys, perm, n, L, s);                                   \
    }                                                                                                           \
    cudaError_t g2p_lambda1_##SFX(const HostCfg& c, const Buffers& b, int cur, const uint32_t* perm, int64_t n, \
                                  const Launch& L, cudaStream_t s)                                              \
    {                                                                                                           \
        return Impl<R>::g2p_lambda1(c, b, cur, perm, n, L, s);                                                  \
    }                                                                                                           \
    cudaError_t grid_update_midpoint_##SFX(const HostCfg& c, const Buffers& b, int cur, const uint32_t* skeys, \
                                           const uint32_t* perm, int64_t n, const Launch& L, cudaStream_t s,    \
                                           double* stats, int64_t* kernels)                                     \
    {                                                                                                           \
        return Impl<R>::grid_update_midpoint(c, b, cur, skeys, perm, n, L, s, stats, kernels);                  \
    }                                                                                                           \
    cudaError_t set_params_##SFX(const HostCfg& c, const Buffers& b, int cur, int64_t n, const double* E,      \
                                 const double* nu, const double* mass, const double* vol, int keep,           \
                                 cudaStream_t s)                                                               \
    {                                                                                                           \
        return Impl<R>::set_params(c, b, cur, n, E, nu, mass, vol, keep, s);                                    \
    }                                                                                                           \
    cudaError_t upload_##SFX(const HostCfg& c, const Buffers& b, int cur, int64_t n, const double* x,          \
                             const double* v, const double* B, const double* F, cudaStream_t s, int64_t k0,     \
                             int64_t k1)                                                                        \
    {                                                                                                           \
        return Impl<R>::upload(c, b, cur, n, x, v, B, F, s, k0, k1);                                            \
    }                                                                                                           \
    cudaError_t inverse_ids_##SFX(const HostCfg& c, const Buffers& b, int cur, int64_t n, uint32_t* inv,        \
                                  cudaStream_t s)                                                               \
    {                                                                                                           \
        return Impl<R>::inverse_ids(c, b, cur, n, inv, s);                                                      \
    }                                                                                                           \
    cudaError_t download_ids_##SFX(const HostCfg& c, const Buffers& b, int cur, int64_t n, const uint32_t* inv, \
                                   int64_t id0, int64_t id1, double* x, double* v, double* B, double* F,        \
                                   cudaStream_t s)                                                              \
    {                                                                                                           \
        return Impl<R>::download_ids(c, b, cur, n, inv, id0, id1, x, v, B, F, s);                               \
    }                                                                                                           \
    cudaError_t download_##SFX(const HostCfg& c, const Buffers& b, int cur, int64_t n, double* x, double* v,   \
                               double* B, double* F, int32_t* cell, double* off, cudaStream_t s)                \
    {                                                                                                           \
        return Impl<R>::download(c, b, cur, n, x, v, B, F, cell, off, s);                                       \
    }                                                                                                           \
    cudaError_t momentum_##SFX(const HostCfg& c, const Buffers& b, int cur, int64_t n, int where,              \
                               int grid_phase, const Launch& L, cudaStream_t s)                                 \
    {                                                                                                           \
        return Impl<R>::momentum(c, b, cur, n, where, grid_phase, L, s);                                        \
    }                                                                                                           \
    cudaError_t grid_dense_##SFX(const HostCfg& c, const Buffers& b, int which, double* m, double* mv,         \
                                 cudaStream_t s)                                                                \
    {                                                                                                           \
        return Impl<R>::grid_dense(c, b, which, m, mv, s);                                                      \
    }                                                                                                           \
    cudaError_t cfl_##SFX(const HostCfg& c, const Buffers& b, int cur, int64_t n, const Launch& L, cudaStream_t s) \
    {                                                                                                           \
        return Impl<R>::cfl(c, b, cur, n, L, s);                                                                \
    }                                                                                                           \
    cudaError_t occupancy_##SFX(const HostCfg& c, int* p2g_per_sm, int* g2p_per_sm)                            \
    {                                                                                                           \
        return Impl<R>::occupancy(c, p2g_per_sm, g2p_per_sm);                                                   \
    }

}  // namespace apic
