// apic_abi.cu -- the C ABI declared in include/apic.h: argument checking, workspace
// carving, call sequencing and error reporting.  Every step of the method runs in the
// kernels of apic_sort.cu and apic_transfer_*.cu; this file only launches them.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <chrono>
#include <cmath>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "apic.h"
#include "apic_internal.h"

using namespace apic;

constexpr int kCopyEvents = 18;   // pieces of a host transfer (at most 16) and two more

struct apic_sim {
    apic_batch* batch;     // the batch this simulation belongs to, if any
    HostCfg c;
    Buffers b;
    Launch L;
    cudaStream_t stream;
    int device;
    int cur;               // which state copy holds the particles
    int64_t n;
    bool keys_valid;       // knext matches the particles in `cur`
    int phase;             // 0 idle, 1 after p2g, 2 after grid update
    uint32_t* skeys;       // last sort's keys / permutation (device)
    uint32_t* perm;
    bool order_sorted;     // the particles are stored in the order of skeys (after G2P)
    bool group_pending;    // p2g_group is chosen after the next full sort (auto, new upload)
    uint32_t epoch;        // look-back epoch of the incremental sort (0: words not cleared yet)
    int64_t max_tiles;
    std::string err;
    int64_t launches;      // kernels launched since creation
    double solve_stats[3]; // the last midpoint solve: Newton and CG iterations, final residual
    // host uploads and downloads in pieces: copies on their own stream, ordered against the
    // simulation's stream by events, so a piece's copies overlap the kernel of another
    cudaStream_t cstream;
    cudaEvent_t cev[kCopyEvents];
    bool copy_ready;
    // apic_momentum_async: reads on their own stream, after an event of the simulation's
    // stream; mdone[c] marks the last read of state copy c, which a later write of that copy
    // waits for (mpending[c] while such a wait is still owed)
    cudaStream_t mstream;
    cudaEvent_t mready, mdone[2];
    bool mom_ready;
    bool mpending[2];
    // per-phase timing
    bool prof_on;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used;
    struct Rec { int phase; cudaEvent_t a, b; int64_t kernels; };
    std::vector<Rec> recs;
};

namespace {

constexpr int64_t kMaxParticles = (int64_t)1 << 30;
constexpr int kMomParts = 1024;

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

int ceil_log2(int64_t v)
{
    int b = 0;
    while (((int64_t)1 << b) < v) ++b;
    return b;
}

apic_status fill_cfg(const apic_config* in, int64_t max_particles, HostCfg* c, std::string* why)
{
    if (!in) { *why = "config is NULL"; return APIC_ERR_ARG; }
    if (in->dim != 2 && in->dim != 3) { *why = "dim must be 2 or 3"; return APIC_ERR_ARG; }
    if (in->order == 1) { *why = "multilinear weights are not supported: the B_p transfer is unstable for them (Sec. 5.9)"; return APIC_ERR_UNSUPPORTED; }
    if (in->order != 2 && in->order != 3) { *why = "order must be 2 (quadratic) or 3 (cubic)"; return APIC_ERR_UNSUPPORTED; }
    if (in->precision != 32 && in->precision != 64) { *why = "precision must be 32 or 64"; return APIC_ERR_ARG; }
    if (in->transfer != APIC_TRANSFER_APIC && in->transfer != APIC_TRANSFER_PIC && in->transfer != APIC_TRANSFER_FLIP) { *why = "unknown transfer"; return APIC_ERR_ARG; }
    if (in->transfer == APIC_TRANSFER_FLIP && !(in->flip_alpha >= 0.0 && in->flip_alpha <= 1.0)) { *why = "flip_alpha must be in [0, 1]"; return APIC_ERR_ARG; }
    if (in->boundary < APIC_BOUNDARY_NONE || in->boundary > APIC_BOUNDARY_SLIP) { *why = "unknown boundary"; return APIC_ERR_UNSUPPORTED; }
    if (in->model < APIC_MODEL_NONE || in->model > APIC_MODEL_NEOHOOKEAN) { *why = "unknown constitutive model"; return APIC_ERR_UNSUPPORTED; }
    if (!(in->dx > 0.0)) { *why = "dx must be positive"; return APIC_ERR_ARG; }
    if (max_particles < 0 || max_particles > kMaxParticles) { *why = "max_particles out of range"; return APIC_ERR_ARG; }
    if (in->wall < 0) { *why = "wall must be >= 0"; return APIC_ERR_ARG; }
    const int maxres = in->dim == 3 ? 1024 : 32768;
    for (int a = 0; a < in->dim; ++a)
        if (in->res[a] < in->order + 2 || in->res[a] > maxres) { *why = "grid resolution out of range"; return APIC_ERR_ARG; }
    int tile = in->tile_particles == 0 ? 4096 : in->tile_particles;
    if (tile < 256 || tile > 4096 || (tile & (tile - 1))) { *why = "tile_particles must be a power of two in [256, 4096]"; return APIC_ERR_ARG; }
    memset(c, 0, sizeof(*c));
    c->dim = in->dim;
    c->order = in->order;
    c->precision = in->precision;
    c->transfer = in->transfer;
    c->flip_alpha = in->transfer == APIC_TRANSFER_FLIP ? in->flip_alpha : 0.0;
    c->nblocks = 1;
    for (int a = 0; a < 3; ++a) {
        c->res[a] = a < in->dim ? in->res[a] : 1;
        c->nb[a] = a < in->dim ? (in->res[a] + APIC_BLOCK_EDGE - 1) / APIC_BLOCK_EDGE : 1;
        c->nblocks *= c->nb[a];
        c->origin[a] = in->origin[a];
        c->gravity[a] = in->gravity[a];
    }
    c->dx = in->dx;
    c->dt = in->dt;
    c->boundary = in->boundary;
    c->wall = in->wall;
    c->model = in->model;
    c->mat = 0;
    c->adaptive = 0;
    if (in->model != APIC_MODEL_NONE) {
        if (!(in->E > 0.0) || !(in->nu > -1.0 && in->nu < 0.5)) { *why = "E must be > 0 and -1 < nu < 0.5"; return APIC_ERR_ARG; }
        c->mu = in->E / (2.0 * (1.0 + in->nu));
        c->lam = in->E * in->nu / ((1.0 + in->nu) * (1.0 - 2.0 * in->nu));
    }
    c->mass = in->particle_mass;
    c->vol = in->particle_volume;
    c->tile = tile;
    if (in->p2g_kernel < 0 || in->p2g_kernel > 2) { *why = "p2g_kernel must be 0, 1 or 2"; return APIC_ERR_ARG; }
    if (in->p2g_kernel == 1 && in->dim != 3) { *why = "the component-split P2G kernel is 3-D only"; return APIC_ERR_ARG; }
    // default: the cell-parallel kernel (the faster of the two on the 128^3 quadratic cube and
    // the 256^3 cubic spheres)
    c->p2g_kernel = in->p2g_kernel != 0 ? in->p2g_kernel : 2;
    if (in->p2g_group != 0 && in->p2g_group != 2 && in->p2g_group != 4) { *why = "p2g_group must be 0, 2 or 4"; return APIC_ERR_ARG; }
    c->p2g_group = in->p2g_group != 0 ? in->p2g_group : 4;
    c->p2g_group_auto = in->p2g_group == 0;
    c->key_bits = 2 * in->dim + ceil_log2(c->nblocks);
    if (c->key_bits > 32) { *why = "grid too large for 32-bit cell keys"; return APIC_ERR_UNSUPPORTED; }
    c->capacity = max_particles;
    c->wait_limit = APIC_DEFAULT_WAIT_LIMIT;
    if (in->integrator < APIC_INTEGRATOR_LAMBDA0 || in->integrator > APIC_INTEGRATOR_MIDPOINT) {
        *why = "integrator must be APIC_INTEGRATOR_LAMBDA0, _LAMBDA1 or _MIDPOINT";
        return APIC_ERR_ARG;
    }
    if (in->integrator != APIC_INTEGRATOR_LAMBDA0 && in->transfer == APIC_TRANSFER_FLIP) {
        *why = "the lambda = 1 and midpoint members are built for the APIC and PIC transfers";
        return APIC_ERR_UNSUPPORTED;
    }
    if (in->integrator == APIC_INTEGRATOR_MIDPOINT) {
        if (in->boundary != APIC_BOUNDARY_NONE || in->gravity[0] != 0.0 || in->gravity[1] != 0.0 ||
            (in->dim == 3 && in->gravity[2] != 0.0)) {
            *why = "the midpoint solve has neither gravity nor walls (the paper's solve has none)";
            return APIC_ERR_UNSUPPORTED;
        }
        if (in->newton_max < 0 || in->cg_max < 0 || in->solve_tol < 0.0) {
            *why = "newton_max, cg_max and solve_tol must be >= 0";
            return APIC_ERR_ARG;
        }
    }
    c->integrator = in->integrator;
    c->newton_max = in->newton_max > 0 ? in->newton_max : 20;
    c->cg_max = in->cg_max > 0 ? in->cg_max : 200;
    c->solve_tol = in->solve_tol > 0.0 ? in->solve_tol : (in->precision == 32 ? 1e-6 : 1e-12);
    return APIC_OK;
}

struct Carve {
    size_t cur = 0;
    size_t take(size_t bytes)
    {
        size_t o = cur;
        cur = align_up(cur + (bytes ? bytes : 1), 256);
        return o;
    }
};

// offsets of every buffer inside the workspace (relative to its base)
struct Layout {
    size_t st[2][APIC_STATE_LANES];
    size_t mk[2], mv[2], midx, choff, mcnt, mbits, mctl, lbs, step_words, acc2, vdel, vel1, solve[6];
    size_t knext, kA, kB, vA, vB, radix_counts, scan_part, tiles, chunk_cnt, ntiles, tile_ctr;
    size_t acc, vel, flags, mom_part, mom_out, amom_part, amom_out, err, fallbacks, staging;
    size_t staging_doubles;
    int64_t max_tiles;
    size_t total;
};

Layout layout_of(const HostCfg& c)
{
    Layout L;
    Carve cv;
    const int64_t n = c.capacity > 0 ? c.capacity : 1;
    const size_t R = c.precision == 32 ? 4 : 8;
    for (int s = 0; s < 2; ++s) {
        // lanes A V Ba Bb Fa Fb (4 reals), Fc (2), Ta (4), Tb (2), M (4: mu, lambda, m_p, V_p);
        // 2-D keeps A V Ba Fa Tb M
        static const int width[APIC_STATE_LANES] = {4, 4, 4, 4, 4, 4, 2, 4, 2, 4};
        static const bool used2d[APIC_STATE_LANES] = {true, true, true, false, true, false, false, false, true, true};
        for (int i = 0; i < APIC_STATE_LANES; ++i)
            L.st[s][i] = cv.take((c.dim == 3 || used2d[i]) ? (size_t)n * width[i] * R : 0);
    }
    L.knext = cv.take((size_t)n * 4);
    L.kA = cv.take((size_t)n * 4);
    L.kB = cv.take((size_t)n * 4);
    L.vA = cv.take((size_t)n * 4);
    L.vB = cv.take((size_t)n * 4);
    L.radix_counts = cv.take((size_t)256 * (radix_tiles(n) + 4) * 4);
    for (int i = 0; i < 2; ++i) {
        L.mk[i] = cv.take((size_t)n * 4);
        L.mv[i] = cv.take((size_t)n * 4);
    }
    L.midx = cv.take((size_t)n * 4);
    L.choff = cv.take(((size_t)radix_tiles(n) + 1) * 4);
    L.mcnt = cv.take(((size_t)radix_tiles(n) + 1) * 4);
    L.mbits = cv.take(moved_bitmap_words(n) * 4);
    L.mctl = cv.take(kMsortCtlBytes);
    L.lbs = cv.take((size_t)256 * ((size_t)radix_tiles(n) + 1) * 8);
    const int64_t nchunks = (n + c.tile - 1) / c.tile;
    L.scan_part = cv.take(scan_partials_needed(n > nchunks ? n : nchunks) * 4);
    L.max_tiles = nchunks + (n < c.nblocks ? n : c.nblocks) + 2;
    L.tiles = cv.take((size_t)(L.max_tiles + 1) * 4);
    L.chunk_cnt = cv.take((size_t)(nchunks + 1) * 4);
    L.ntiles = cv.take(4);
    L.tile_ctr = cv.take(16);
    const size_t bn = c.dim == 3 ? 64 : 16;
    L.acc = cv.take((size_t)c.nblocks * bn * 4 * R);
    L.vel = cv.take((size_t)c.nblocks * bn * 4 * R);
    // FLIP: PIC momentum without the force, and the grid change v~ - v (4 lanes per node each)
    const size_t flip_bytes = c.transfer == APIC_TRANSFER_FLIP ? (size_t)c.nblocks * bn * 4 * R : 0;
    L.acc2 = cv.take(flip_bytes);
    L.vdel = cv.take(flip_bytes);
    // lambda = 1 and the midpoint rule: the grid velocity before the update (4 lanes per node);
    // the midpoint solve: its six grid vectors
    const size_t gv_bytes = (size_t)c.nblocks * bn * 4 * R;
    L.vel1 = cv.take(c.integrator != APIC_INTEGRATOR_LAMBDA0 ? gv_bytes : 0);
    for (int i = 0; i < 6; ++i) L.solve[i] = cv.take(c.integrator == APIC_INTEGRATOR_MIDPOINT ? gv_bytes : 0);
    L.flags = cv.take((size_t)c.nblocks * 4);
    L.mom_part = cv.take((size_t)kMomParts * 6 * 8);
    L.mom_out = cv.take(6 * 8);
    L.amom_part = cv.take((size_t)kMomParts * 6 * 8);
    L.amom_out = cv.take(6 * 8);
    L.err = cv.take(4);
    L.fallbacks = cv.take(4);
    L.step_words = cv.take(32);   // dt word (8), speed maximum (4), elapsed time (8 at +16)
    const int d = c.dim;
    size_t nn = 1;
    for (int a = 0; a < d; ++a) nn *= (size_t)c.res[a];
    size_t sd = (size_t)n * (2 * d + 2 * d * d);
    const size_t grid_need = nn * (1 + d);
    if (grid_need > sd) sd = grid_need;
    L.staging_doubles = sd;
    L.staging = cv.take(sd * 8);
    L.total = cv.cur;
    return L;
}

apic_status fail(apic_sim* s, apic_status st, const std::string& why)
{
    if (s) s->err = why;
    return st;
}

apic_status cuda_fail(apic_sim* s, cudaError_t e, const char* where)
{
    return fail(s, APIC_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(expr, where)                                   \
    do {                                                  \
        cudaError_t e_ = (expr);                          \
        if (e_ != cudaSuccess) return cuda_fail(s, e_, where); \
    } while (0)

// read and clear the latched device error word (synchronises the stream); *bits (may be
// NULL) receives the bits that were set
apic_status check_device(apic_sim* s, uint32_t* bits = nullptr)
{
    uint32_t e = 0;
    if (bits) *bits = 0;
    CK(cudaMemcpyAsync(&e, s->b.err, 4, cudaMemcpyDeviceToHost, s->stream), "read error word");
    CK(cudaStreamSynchronize(s->stream), "synchronize");
    if (e == 0) return APIC_OK;
    if (bits) *bits = e;
    CK(cudaMemsetAsync(s->b.err, 0, 4, s->stream), "clear error word");
    CK(cudaStreamSynchronize(s->stream), "synchronize");
    if (e & APIC_ERRBIT_TIMEOUT) return fail(s, APIC_ERR_TIMEOUT, "a bounded device wait (bulk copy completion) ran out");
    if (e & APIC_ERRBIT_CAPACITY) return fail(s, APIC_ERR_OOM, "tile list capacity exceeded");
    if (e & APIC_ERRBIT_NONFINITE) return fail(s, APIC_ERR_NUMERIC, "a non-finite value (NaN or Inf) in the uploaded state");
    return fail(s, APIC_ERR_NUMERIC, "a particle's stencil left the grid; it was clamped to the boundary");
}

cudaEvent_t take_event(apic_sim* s)
{
    if (s->ev_used == s->ev_pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        s->ev_pool.push_back(e);
    }
    return s->ev_pool[s->ev_used++];
}

// records events around one phase when profiling is on; counts launched kernels always
struct PhaseScope {
    apic_sim* s;
    int phase;
    int64_t kernels;
    cudaEvent_t a = nullptr;
    PhaseScope(apic_sim* s_, int phase_, int64_t kernels_) : s(s_), phase(phase_), kernels(kernels_)
    {
        if (s->prof_on && (a = take_event(s)) != nullptr) cudaEventRecord(a, s->stream);
    }
    ~PhaseScope()
    {
        s->launches += kernels;
        if (a) {
            cudaEvent_t b = take_event(s);
            if (b) {
                cudaEventRecord(b, s->stream);
                s->recs.push_back({phase, a, b, kernels});
            }
        }
    }
};

apic_status batch_sync_member(apic_sim* s);

#define IN_BATCH_GUARD(s)                                                                       \
    do {                                                                                        \
        if ((s)->batch) return fail((s), APIC_ERR_ARG, "the simulation is a member of a batch"); \
    } while (0)

#define DISPATCH(s, fn, ...) ((s)->c.precision == 32 ? fn##_f32(__VA_ARGS__) : fn##_f64(__VA_ARGS__))

// the copy stream and events of a simulation's host transfers, made on first use
cudaError_t ensure_copy_stream(apic_sim* s)
{
    if (s->copy_ready) return cudaSuccess;
    cudaError_t e = cudaStreamCreateWithFlags(&s->cstream, cudaStreamNonBlocking);
    int made = 0;
    for (; e == cudaSuccess && made < kCopyEvents; ++made)
        e = cudaEventCreateWithFlags(&s->cev[made], cudaEventDisableTiming);
    if (e != cudaSuccess) {
        for (int i = 0; i < made; ++i) cudaEventDestroy(s->cev[i]);
        if (s->cstream) cudaStreamDestroy(s->cstream);
        s->cstream = nullptr;
        return e;
    }
    s->copy_ready = true;
    return cudaSuccess;
}

// the stream and events of apic_momentum_async, made on first use
cudaError_t ensure_mom_stream(apic_sim* s)
{
    if (s->mom_ready) return cudaSuccess;
    cudaError_t e = cudaStreamCreateWithFlags(&s->mstream, cudaStreamNonBlocking);
    cudaEvent_t* ev[3] = {&s->mready, &s->mdone[0], &s->mdone[1]};
    int made = 0;
    for (; e == cudaSuccess && made < 3; ++made) e = cudaEventCreateWithFlags(ev[made], cudaEventDisableTiming);
    if (e != cudaSuccess) {
        for (int i = 0; i < made; ++i) cudaEventDestroy(*ev[i]);
        if (s->mstream) cudaStreamDestroy(s->mstream);
        s->mstream = nullptr;
        return e;
    }
    s->mom_ready = true;
    return cudaSuccess;
}

// before work that overwrites state copy `copy` (-1: both): the simulation's stream waits
// for the asynchronous momentum reads of it that are still owed
cudaError_t mom_fence(apic_sim* s, int copy)
{
    for (int c = 0; c < 2; ++c) {
        if ((copy >= 0 && copy != c) || !s->mpending[c]) continue;
        const cudaError_t e = cudaStreamWaitEvent(s->stream, s->mdone[c], 0);
        if (e != cudaSuccess) return e;
        s->mpending[c] = false;
    }
    return cudaSuccess;
}

// pieces of a host transfer of n particles: about half a million particles each, at most 16
int copy_pieces(int64_t n)
{
    const int64_t p = (n + (int64_t)(1 << 19) - 1) >> 19;
    return (int)(p < 1 ? 1 : (p > 16 ? 16 : p));
}

}  // namespace

extern "C" {

apic_status apic_workspace_size(const apic_config* cfg, int64_t max_particles, size_t* bytes)
{
    if (!bytes) return APIC_ERR_ARG;
    HostCfg c;
    std::string why;
    apic_status st = fill_cfg(cfg, max_particles, &c, &why);
    if (st != APIC_OK) return st;
    *bytes = layout_of(c).total;
    return APIC_OK;
}

apic_status apic_create(const apic_config* cfg, int64_t max_particles, void* workspace, size_t workspace_bytes,
                        void* stream, apic_sim** out)
{
    if (!out) return APIC_ERR_ARG;
    *out = nullptr;
    HostCfg c;
    std::string why;
    apic_status st = fill_cfg(cfg, max_particles, &c, &why);
    if (st != APIC_OK) return st;
    if (!workspace || ((uintptr_t)workspace & 255)) return APIC_ERR_ARG;
    Layout L = layout_of(c);
    if (workspace_bytes < L.total) return APIC_ERR_OOM;
    apic_sim* s = new (std::nothrow) apic_sim();
    if (!s) return APIC_ERR_OOM;
    s->batch = nullptr;
    s->c = c;
    s->stream = (cudaStream_t)stream;
    s->cur = 0;
    s->n = 0;
    s->keys_valid = false;
    s->phase = 0;
    s->skeys = s->perm = nullptr;
    s->order_sorted = false;
    s->group_pending = false;
    s->epoch = 0;
    s->max_tiles = L.max_tiles;
    s->launches = 0;
    s->prof_on = false;
    s->ev_used = 0;
    char* base = (char*)workspace;
    for (int a = 0; a < 2; ++a)
        for (int i = 0; i < APIC_STATE_LANES; ++i) s->b.st[a][i] = base + L.st[a][i];
    s->b.knext = (uint32_t*)(base + L.knext);
    s->b.kA = (uint32_t*)(base + L.kA);
    s->b.kB = (uint32_t*)(base + L.kB);
    s->b.vA = (uint32_t*)(base + L.vA);
    s->b.vB = (uint32_t*)(base + L.vB);
    s->b.radix_counts = (uint32_t*)(base + L.radix_counts);
    for (int i = 0; i < 2; ++i) {
        s->b.mk[i] = (uint32_t*)(base + L.mk[i]);
        s->b.mv[i] = (uint32_t*)(base + L.mv[i]);
    }
    s->b.midx = (uint32_t*)(base + L.midx);
    s->b.choff = (uint32_t*)(base + L.choff);
    s->b.mcnt = (uint32_t*)(base + L.mcnt);
    s->b.mbits = (uint32_t*)(base + L.mbits);
    s->b.mctl = (uint32_t*)(base + L.mctl);
    s->b.mhist = s->b.mctl + 16;
    s->b.lbs = (unsigned long long*)(base + L.lbs);
    s->b.scan_part = (uint32_t*)(base + L.scan_part);
    s->b.tiles = (uint32_t*)(base + L.tiles);
    s->b.chunk_cnt = (uint32_t*)(base + L.chunk_cnt);
    s->b.ntiles = (uint32_t*)(base + L.ntiles);
    s->b.tile_ctr = (uint32_t*)(base + L.tile_ctr);
    s->b.acc = base + L.acc;
    s->b.vel = base + L.vel;
    s->b.acc2 = c.transfer == APIC_TRANSFER_FLIP ? base + L.acc2 : nullptr;
    s->b.vdel = c.transfer == APIC_TRANSFER_FLIP ? base + L.vdel : nullptr;
    s->b.vel1 = c.integrator != APIC_INTEGRATOR_LAMBDA0 ? base + L.vel1 : nullptr;
    {
        const bool mid = c.integrator == APIC_INTEGRATOR_MIDPOINT;
        void** sv[6] = {&s->b.sdv, &s->b.su, &s->b.sr, &s->b.sp, &s->b.ss, &s->b.sdu};
        for (int i = 0; i < 6; ++i) *sv[i] = mid ? base + L.solve[i] : nullptr;
    }
    s->solve_stats[0] = s->solve_stats[1] = s->solve_stats[2] = 0.0;
    s->b.flags = (uint32_t*)(base + L.flags);
    s->b.mom_part = (double*)(base + L.mom_part);
    s->b.mom_out = (double*)(base + L.mom_out);
    s->b.amom_part = (double*)(base + L.amom_part);
    s->b.amom_out = (double*)(base + L.amom_out);
    s->b.err = (uint32_t*)(base + L.err);
    s->b.fallbacks = (uint32_t*)(base + L.fallbacks);
    s->b.dt_word = base + L.step_words;
    s->b.smax_word = (uint32_t*)(base + L.step_words + 8);
    s->b.elapsed = (double*)(base + L.step_words + 16);
    s->b.staging = (double*)(base + L.staging);
    s->b.staging_doubles = L.staging_doubles;
    cudaError_t e = cudaGetDevice(&s->device);
    int sms = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device);
    int p2g_per = 1, g2p_per = 1;
    if (e == cudaSuccess) e = c.precision == 32 ? occupancy_f32(c, &p2g_per, &g2p_per) : occupancy_f64(c, &p2g_per, &g2p_per);
    if (e != cudaSuccess) {
        delete s;
        return APIC_ERR_CUDA;
    }
    s->L.sms = sms;
    s->L.p2g_grid = sms * (p2g_per > 0 ? p2g_per : 1);
    s->L.p2g_cells = 1;
    s->L.g2p_grid = sms * (g2p_per > 0 ? g2p_per : 1);
    s->L.mom_parts = kMomParts;
    const size_t bn = c.dim == 3 ? 64 : 16;
    const size_t gbytes = (size_t)c.nblocks * bn * 4 * (c.precision == 32 ? 4 : 8);
    e = cudaMemsetAsync(s->b.acc, 0, gbytes, s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->b.vel, 0, gbytes, s->stream);
    if (e == cudaSuccess && s->b.acc2) e = cudaMemsetAsync(s->b.acc2, 0, gbytes, s->stream);
    if (e == cudaSuccess && s->b.vdel) e = cudaMemsetAsync(s->b.vdel, 0, gbytes, s->stream);
    if (e == cudaSuccess && s->b.vel1) e = cudaMemsetAsync(s->b.vel1, 0, gbytes, s->stream);
    if (c.integrator == APIC_INTEGRATOR_MIDPOINT) {
        void* sv[6] = {s->b.sdv, s->b.su, s->b.sr, s->b.sp, s->b.ss, s->b.sdu};
        for (int i = 0; i < 6 && e == cudaSuccess; ++i) e = cudaMemsetAsync(sv[i], 0, gbytes, s->stream);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(s->b.flags, 0, (size_t)c.nblocks * 4, s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->b.err, 0, 4, s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->b.dt_word, 0, 32, s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->b.fallbacks, 0, 4, s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->b.ntiles, 0, 4, s->stream);
    if (e != cudaSuccess) {
        delete s;
        return APIC_ERR_CUDA;
    }
    *out = s;
    return APIC_OK;
}

apic_status apic_destroy(apic_sim* s)
{
    if (!s) return APIC_ERR_ARG;
    if (s->batch) apic_batch_remove(s->batch, s);
    cudaError_t e = cudaStreamSynchronize(s->stream);
    for (cudaEvent_t ev : s->ev_pool) cudaEventDestroy(ev);
    if (s->copy_ready) {
        cudaStreamSynchronize(s->cstream);
        for (cudaEvent_t ev : s->cev) cudaEventDestroy(ev);
        cudaStreamDestroy(s->cstream);
    }
    if (s->mom_ready) {
        cudaStreamSynchronize(s->mstream);
        cudaEventDestroy(s->mready);
        cudaEventDestroy(s->mdone[0]);
        cudaEventDestroy(s->mdone[1]);
        cudaStreamDestroy(s->mstream);
    }
    delete s;
    return e == cudaSuccess ? APIC_OK : APIC_ERR_CUDA;
}

apic_status apic_upload(apic_sim* s, int64_t n, const double* x, const double* v, const double* B, const double* F,
                        int on_device)
{
    if (!s) return APIC_ERR_ARG;
    IN_BATCH_GUARD(s);
    if (n < 0) return fail(s, APIC_ERR_ARG, "n < 0");
    if (n > s->c.capacity) return fail(s, APIC_ERR_OOM, "n exceeds the particle capacity given to apic_create");
    if (n > 0 && !x) return fail(s, APIC_ERR_ARG, "positions are required");
    CK(cudaSetDevice(s->device), "cudaSetDevice");
    CK(mom_fence(s, -1), "wait for momentum reads");
    const int d = s->c.dim;
    s->n = n;
    s->cur = 0;
    s->keys_valid = false;
    s->phase = 0;
    s->skeys = s->perm = nullptr;
    s->order_sorted = false;
    s->group_pending = s->c.p2g_group_auto != 0;   // the new particle set's density decides
    s->c.mat = 0;   // a new particle set: materials come from the configuration until set again
    if (on_device || n == 0) {
        CK(DISPATCH(s, upload, s->c, s->b, s->cur, n, x, v, B, F, s->stream, (int64_t)0, n), "upload kernel");
    } else {
        // host input: in pieces, each piece's copies on the copy stream and its kernel on the
        // simulation's stream after them, so copies and kernels overlap; the copy stream
        // first waits for the simulation's earlier work (it may still read the staging buffer)
        CK(ensure_copy_stream(s), "copy stream");
        double* sx = s->b.staging;
        double* sv = sx + n * d;
        double* sB = sv + n * d;
        double* sF = sB + n * d * d;
        const int pieces = copy_pieces(n);
        CK(cudaEventRecord(s->cev[kCopyEvents - 1], s->stream), "event");
        CK(cudaStreamWaitEvent(s->cstream, s->cev[kCopyEvents - 1], 0), "stream wait");
        for (int p = 0; p < pieces; ++p) {
            const int64_t k0 = n * p / pieces, k1 = n * (p + 1) / pieces, m = k1 - k0;
            CK(cudaMemcpyAsync(sx + k0 * d, x + k0 * d, sizeof(double) * m * d, cudaMemcpyHostToDevice, s->cstream),
               "upload x");
            if (v)
                CK(cudaMemcpyAsync(sv + k0 * d, v + k0 * d, sizeof(double) * m * d, cudaMemcpyHostToDevice,
                                   s->cstream), "upload v");
            if (B)
                CK(cudaMemcpyAsync(sB + k0 * d * d, B + k0 * d * d, sizeof(double) * m * d * d,
                                   cudaMemcpyHostToDevice, s->cstream), "upload B");
            if (F)
                CK(cudaMemcpyAsync(sF + k0 * d * d, F + k0 * d * d, sizeof(double) * m * d * d,
                                   cudaMemcpyHostToDevice, s->cstream), "upload F");
            CK(cudaEventRecord(s->cev[p], s->cstream), "event");
            CK(cudaStreamWaitEvent(s->stream, s->cev[p], 0), "stream wait");
            CK(DISPATCH(s, upload, s->c, s->b, s->cur, n, sx, v ? sv : nullptr, B ? sB : nullptr, F ? sF : nullptr,
                        s->stream, k0, k1), "upload kernel");
        }
    }
    if (!on_device) {
        uint32_t bits = 0;
        apic_status st = check_device(s, &bits);
        if (bits & APIC_ERRBIT_NONFINITE) s->n = 0;   // a rejected upload leaves no particles
        return st;
    }
    return APIC_OK;
}

apic_status apic_upload_materials(apic_sim* s, int64_t n, const double* E, const double* nu, int on_device)
{
    if (!s) return APIC_ERR_ARG;
    IN_BATCH_GUARD(s);
    if (s->phase != 0) return fail(s, APIC_ERR_ARG, "apic_upload_materials between apic_p2g and apic_g2p");
    if (n != s->n) return fail(s, APIC_ERR_ARG, "n must equal the particle count of the last apic_upload");
    if (n > 0 && (!E || !nu)) return fail(s, APIC_ERR_ARG, "E and nu are required");
    CK(cudaSetDevice(s->device), "cudaSetDevice");
    CK(mom_fence(s, -1), "wait for momentum reads");
    const int keep = s->c.mat;
    if (n == 0) {
        s->c.mat = 1;
        return APIC_OK;
    }
    const double *dE = E, *dnu = nu;
    if (!on_device) {
        for (int64_t i = 0; i < n; ++i)
            if (!(E[i] > 0.0) || !(nu[i] > -1.0 && nu[i] < 0.5))
                return fail(s, APIC_ERR_ARG, "each E must be > 0 and each nu in (-1, 0.5)");
        double* sE = s->b.staging;
        double* snu = sE + n;
        CK(cudaMemcpyAsync(sE, E, sizeof(double) * n, cudaMemcpyHostToDevice, s->stream), "upload E");
        CK(cudaMemcpyAsync(snu, nu, sizeof(double) * n, cudaMemcpyHostToDevice, s->stream), "upload nu");
        dE = sE;
        dnu = snu;
    }
    s->c.mat = 1;
    CK(DISPATCH(s, set_params, s->c, s->b, s->cur, n, dE, dnu, nullptr, nullptr, keep, s->stream), "materials kernel");
    s->launches += 1;
    if (!on_device) return check_device(s);
    return APIC_OK;
}

apic_status apic_upload_mass_volume(apic_sim* s, int64_t n, const double* mass, const double* vol, int on_device)
{
    if (!s) return APIC_ERR_ARG;
    IN_BATCH_GUARD(s);
    if (s->phase != 0) return fail(s, APIC_ERR_ARG, "apic_upload_mass_volume between apic_p2g and apic_g2p");
    if (n != s->n) return fail(s, APIC_ERR_ARG, "n must equal the particle count of the last apic_upload");
    if (n > 0 && (!mass || !vol)) return fail(s, APIC_ERR_ARG, "mass and vol are required");
    CK(cudaSetDevice(s->device), "cudaSetDevice");
    CK(mom_fence(s, -1), "wait for momentum reads");
    const int keep = s->c.mat;
    if (n == 0) {
        s->c.mat = 1;
        return APIC_OK;
    }
    const double *dm = mass, *dv = vol;
    if (!on_device) {
        for (int64_t i = 0; i < n; ++i)
            if (!(mass[i] > 0.0) || !(vol[i] > 0.0) || !std::isfinite(mass[i]) || !std::isfinite(vol[i]))
                return fail(s, APIC_ERR_ARG, "each mass and each volume must be finite and > 0");
        double* sm = s->b.staging;
        double* sv = sm + n;
        CK(cudaMemcpyAsync(sm, mass, sizeof(double) * n, cudaMemcpyHostToDevice, s->stream), "upload mass");
        CK(cudaMemcpyAsync(sv, vol, sizeof(double) * n, cudaMemcpyHostToDevice, s->stream), "upload vol");
        dm = sm;
        dv = sv;
    }
    s->c.mat = 1;
    CK(DISPATCH(s, set_params, s->c, s->b, s->cur, n, nullptr, nullptr, dm, dv, keep, s->stream), "mass kernel");
    s->launches += 1;
    if (!on_device) return check_device(s);
    return APIC_OK;
}

apic_status apic_download(apic_sim* s, double* x, double* v, double* B, double* F, int on_device)
{
    if (!s) return APIC_ERR_ARG;
    if (s->batch) {
        apic_status bst = batch_sync_member(s);
        if (bst != APIC_OK) return bst;
    }
    CK(cudaSetDevice(s->device), "cudaSetDevice");
    const int64_t n = s->n;
    const int d = s->c.dim;
    if (n == 0) return check_device(s);
    if (on_device) {
        CK(DISPATCH(s, download, s->c, s->b, s->cur, n, x, v, B, F, nullptr, nullptr, s->stream), "download kernel");
        return check_device(s);
    }
    // host output: the particles are gathered in upload order piece by piece (through the
    // inverse of their id lane, kept in the sort's moved-index scratch, free between steps),
    // and each piece's copies start on the copy stream as soon as its kernel is done
    CK(ensure_copy_stream(s), "copy stream");
    double* sx = s->b.staging;
    double* sv = sx + n * d;
    double* sB = sv + n * d;
    double* sF = sB + n * d * d;
    uint32_t* inv = s->b.midx;
    CK(DISPATCH(s, inverse_ids, s->c, s->b, s->cur, n, inv, s->stream), "id inverse kernel");
    const int pieces = copy_pieces(n);
    for (int p = 0; p < pieces; ++p) {
        const int64_t k0 = n * p / pieces, k1 = n * (p + 1) / pieces, m = k1 - k0;
        CK(DISPATCH(s, download_ids, s->c, s->b, s->cur, n, inv, k0, k1, x ? sx : nullptr, v ? sv : nullptr,
                    B ? sB : nullptr, F ? sF : nullptr, s->stream),
           "download kernel");
        CK(cudaEventRecord(s->cev[p], s->stream), "event");
        CK(cudaStreamWaitEvent(s->cstream, s->cev[p], 0), "stream wait");
        if (x)
            CK(cudaMemcpyAsync(x + k0 * d, sx + k0 * d, sizeof(double) * m * d, cudaMemcpyDeviceToHost, s->cstream),
               "download x");
        if (v)
            CK(cudaMemcpyAsync(v + k0 * d, sv + k0 * d, sizeof(double) * m * d, cudaMemcpyDeviceToHost, s->cstream),
               "download v");
        if (B)
            CK(cudaMemcpyAsync(B + k0 * d * d, sB + k0 * d * d, sizeof(double) * m * d * d, cudaMemcpyDeviceToHost,
                               s->cstream), "download B");
        if (F)
            CK(cudaMemcpyAsync(F + k0 * d * d, sF + k0 * d * d, sizeof(double) * m * d * d, cudaMemcpyDeviceToHost,
                               s->cstream), "download F");
    }
    // later work on the simulation's stream (and the synchronisation below) waits for the copies
    CK(cudaEventRecord(s->cev[kCopyEvents - 2], s->cstream), "event");
    CK(cudaStreamWaitEvent(s->stream, s->cev[kCopyEvents - 2], 0), "stream wait");
    return check_device(s);
}

apic_status apic_download_positions(apic_sim* s, int32_t* cell, double* offset)
{
    if (!s || !cell || !offset) return APIC_ERR_ARG;
    if (s->batch) {
        apic_status bst = batch_sync_member(s);
        if (bst != APIC_OK) return bst;
    }
    CK(cudaSetDevice(s->device), "cudaSetDevice");
    const int64_t n = s->n;
    const int d = s->c.dim;
    if (n == 0) return check_device(s);
    double* so = s->b.staging;
    int32_t* sc = (int32_t*)(so + n * d);
    CK(DISPATCH(s, download, s->c, s->b, s->cur, n, nullptr, nullptr, nullptr, nullptr, sc, so, s->stream),
       "download kernel");
    CK(cudaMemcpyAsync(offset, so, sizeof(double) * n * d, cudaMemcpyDeviceToHost, s->stream), "download offsets");
    CK(cudaMemcpyAsync(cell, sc, sizeof(int32_t) * n * d, cudaMemcpyDeviceToHost, s->stream), "download cells");
    return check_device(s);
}

apic_status apic_p2g(apic_sim* s)
{
    if (!s) return APIC_ERR_ARG;
    IN_BATCH_GUARD(s);
    if (s->phase != 0) return fail(s, APIC_ERR_ARG, "apic_p2g called twice without apic_grid_update / apic_g2p");
    CK(cudaSetDevice(s->device), "cudaSetDevice");
    const int64_t n = s->n;
    if (n == 0) {
        s->phase = 1;
        return APIC_OK;
    }
    if (!s->keys_valid) {
        PhaseScope ps(s, APIC_PHASE_KEYS, 1);
        CK(DISPATCH(s, keys, s->c, s->b, s->cur, n, s->stream), "keys kernel");
    }
    if (s->keys_valid && s->order_sorted && s->skeys) {
        // particles are stored in the previous sorted order: sort only the moved keys
        PhaseScope ps(s, APIC_PHASE_SORT, resort_kernels(n, s->c.key_bits));
        uint32_t* kout = s->skeys == s->b.kA ? s->b.kB : s->b.kA;
        uint32_t* vout = s->skeys == s->b.kA ? s->b.vB : s->b.vA;
        CK(resort(s->b, n, s->c.key_bits, s->skeys, kout, vout, &s->epoch, s->L.sms, s->stream), "incremental sort");
        s->skeys = kout;
        s->perm = vout;
    } else {
        PhaseScope ps(s, APIC_PHASE_SORT, radix_sort_kernels(s->c.key_bits));
        CK(radix_sort(s->b, n, s->c.key_bits, s->stream, &s->skeys, &s->perm), "radix sort");
    }
    {
        PhaseScope ps(s, APIC_PHASE_TILES, build_tiles_kernels(n, s->c.tile));
        CK(build_tiles(s->b, s->skeys, n, s->c.dim, s->c.tile, s->max_tiles, s->stream), "tile list");
    }
    if (s->group_pending && s->c.p2g_kernel == 2) {
        // particles per occupied base cell, from the tile count (a node block of 4^d cells
        // holds one tile up to tile_particles particles): fewer than 16 take groups of 2
        uint32_t nt = 0;
        CK(cudaMemcpyAsync(&nt, s->b.ntiles, sizeof(nt), cudaMemcpyDeviceToHost, s->stream), "read tile count");
        CK(cudaStreamSynchronize(s->stream), "synchronize");
        const double cells = (double)(nt ? nt : 1u) * (s->c.dim == 3 ? 64.0 : 16.0);
        s->c.p2g_group = (double)n / cells < 16.0 ? 2 : 4;
        s->group_pending = false;
    }
    {
        PhaseScope ps(s, APIC_PHASE_P2G, s->c.transfer == 2 ? 2 : 1);   // FLIP: a second pass
        CK(DISPATCH(s, p2g, s->c, s->b, s->cur, s->skeys, s->perm, n, s->L, s->stream), "p2g kernel");
    }
    s->phase = 1;
    return APIC_OK;
}

apic_status apic_grid_update(apic_sim* s)
{
    if (!s) return APIC_ERR_ARG;
    IN_BATCH_GUARD(s);
    if (s->phase != 1) return fail(s, APIC_ERR_ARG, "apic_grid_update must follow apic_p2g");
    CK(cudaSetDevice(s->device), "cudaSetDevice");
    if (s->c.integrator == APIC_INTEGRATOR_MIDPOINT) {
        int64_t kernels = 0;
        cudaError_t e = DISPATCH(s, grid_update_midpoint, s->c, s->b, s->cur, s->skeys, s->perm, s->n, s->L, s->stream,
                                 s->solve_stats, &kernels);
        PhaseScope ps(s, APIC_PHASE_GRID, kernels);
        CK(e, "midpoint grid solve");
    } else if (s->c.integrator == APIC_INTEGRATOR_LAMBDA1) {
        PhaseScope ps(s, APIC_PHASE_GRID, (s->c.model != 0 && s->n > 0) ? 3 : 2);
        CK(DISPATCH(s, grid_update_lambda1, s->c, s->b, s->cur, s->skeys, s->perm, s->n, s->L, s->stream),
           "lambda = 1 grid kernels");
    } else {
        PhaseScope ps(s, APIC_PHASE_GRID, 1);
        CK(DISPATCH(s, grid_update, s->c, s->b, s->L, s->stream), "grid update kernel");
    }
    s->phase = 2;
    return APIC_OK;
}

apic_status apic_g2p(apic_sim* s)
{
    if (!s) return APIC_ERR_ARG;
    IN_BATCH_GUARD(s);
    if (s->phase != 2) return fail(s, APIC_ERR_ARG, "apic_g2p must follow apic_grid_update");
    CK(cudaSetDevice(s->device), "cudaSetDevice");
    CK(mom_fence(s, s->cur ^ 1), "wait for momentum reads");   // G2P writes the other copy
    if (s->n > 0) {
        {
            PhaseScope ps(s, APIC_PHASE_G2P, 1);
            if (s->c.integrator != APIC_INTEGRATOR_LAMBDA0)
                CK(DISPATCH(s, g2p_lambda1, s->c, s->b, s->cur, s->perm, s->n, s->L, s->stream), "general g2p kernel");
            else
                CK(DISPATCH(s, g2p, s->c, s->b, s->cur, s->skeys, s->perm, s->n, s->L, s->stream), "g2p kernel");
        }
        s->cur ^= 1;
        s->keys_valid = true;
        s->order_sorted = true;   // G2P wrote particle k of the sorted order at k
    }
    s->phase = 0;
    return APIC_OK;
}

apic_status apic_step(apic_sim* s, int nsteps)
{
    if (!s || nsteps < 0) return APIC_ERR_ARG;
    IN_BATCH_GUARD(s);
    for (int i = 0; i < nsteps; ++i) {
        apic_status st = apic_p2g(s);
        if (st == APIC_OK) st = apic_grid_update(s);
        if (st == APIC_OK) st = apic_g2p(s);
        if (st != APIC_OK) return st;
    }
    return APIC_OK;
}

apic_status apic_step_adaptive(apic_sim* s, int nsteps, double nu, double dt_max, double* elapsed)
{
    if (!s || nsteps < 0 || !(nu > 0.0) || !(dt_max > 0.0)) return APIC_ERR_ARG;
    IN_BATCH_GUARD(s);
    if (s->phase != 0) return fail(s, APIC_ERR_ARG, "apic_step_adaptive between apic_p2g and apic_g2p");
    if (s->c.integrator != APIC_INTEGRATOR_LAMBDA0)
        return fail(s, APIC_ERR_UNSUPPORTED, "adaptive steps are built for the lambda = 0 integrator");
    CK(cudaSetDevice(s->device), "cudaSetDevice");
    if (elapsed) *elapsed = 0.0;
    if (s->n == 0 || nsteps == 0) return APIC_OK;
    // first time step from the FP64 speed maximum of the current state
    CK(DISPATCH(s, cfl, s->c, s->b, s->cur, s->n, s->L, s->stream), "cfl kernel");
    CK(DISPATCH(s, adapt_dt, s->c, s->b, nu, dt_max, 1, s->stream), "time step kernel");
    s->launches += 3;
    s->c.adaptive = 1;
    apic_status st = APIC_OK;
    for (int i = 0; i < nsteps && st == APIC_OK; ++i) {
        st = apic_p2g(s);
        if (st == APIC_OK) st = apic_grid_update(s);
        if (st == APIC_OK) st = apic_g2p(s);
        if (st == APIC_OK) {
            // adds this step's dt to the elapsed time, takes the next from G2P's speed maximum
            cudaError_t e = s->c.precision == 32 ? adapt_dt_f32(s->c, s->b, nu, dt_max, 0, s->stream)
                                                 : adapt_dt_f64(s->c, s->b, nu, dt_max, 0, s->stream);
            if (e != cudaSuccess) st = cuda_fail(s, e, "time step kernel");
            s->launches += 1;
        }
    }
    s->c.adaptive = 0;
    if (st != APIC_OK) return st;
    if (elapsed) {
        CK(cudaMemcpyAsync(elapsed, s->b.elapsed, sizeof(double), cudaMemcpyDeviceToHost, s->stream), "read time");
        return check_device(s);
    }
    return APIC_OK;
}

apic_status apic_momentum(apic_sim* s, int where, double p[3], double l[3])
{
    if (!s || !p || !l) return APIC_ERR_ARG;
    if (s->batch) {
        apic_status bst = batch_sync_member(s);
        if (bst != APIC_OK) return bst;
    }
    CK(cudaSetDevice(s->device), "cudaSetDevice");
    int grid_phase = 0;
    if (where == APIC_WHERE_GRID) {
        if (s->phase == 1) grid_phase = 0;
        else if (s->phase == 2) grid_phase = 1;
        else return fail(s, APIC_ERR_ARG, "grid momentum needs apic_p2g (or apic_grid_update) first");
    } else if (where != APIC_WHERE_PARTICLES) {
        return fail(s, APIC_ERR_ARG, "where must be APIC_WHERE_PARTICLES or APIC_WHERE_GRID");
    }
    CK(DISPATCH(s, momentum, s->c, s->b, s->cur, s->n, where, grid_phase, s->L, s->stream), "momentum kernel");
    double h[6];
    CK(cudaMemcpyAsync(h, s->b.mom_out, sizeof(h), cudaMemcpyDeviceToHost, s->stream), "read momentum");
    apic_status st = check_device(s);
    for (int i = 0; i < 3; ++i) {
        p[i] = h[i];
        l[i] = h[3 + i];
    }
    if (s->c.dim == 2) {
        p[2] = 0.0;
        l[1] = l[2] = 0.0;
    }
    return st;
}

apic_status apic_momentum_async(apic_sim* s, double* out)
{
    if (!s || !out) return APIC_ERR_ARG;
    if (s->batch) return fail(s, APIC_ERR_ARG, "asynchronous momentum reads are for simulations outside a batch");
    CK(cudaSetDevice(s->device), "cudaSetDevice");
    CK(ensure_mom_stream(s), "momentum stream");
    CK(cudaEventRecord(s->mready, s->stream), "record event");
    CK(cudaStreamWaitEvent(s->mstream, s->mready, 0), "stream wait");
    Buffers ab = s->b;   // the reduction's own scratch, so it may overlap the calls that follow
    ab.mom_part = s->b.amom_part;
    ab.mom_out = s->b.amom_out;
    CK(DISPATCH(s, momentum, s->c, ab, s->cur, s->n, (int)APIC_WHERE_PARTICLES, 0, s->L, s->mstream), "momentum kernel");
    s->launches += 2;
    CK(cudaMemcpyAsync(out, s->b.amom_out, 6 * sizeof(double), cudaMemcpyDefault, s->mstream), "read momentum");
    CK(cudaEventRecord(s->mdone[s->cur], s->mstream), "record event");
    s->mpending[s->cur] = true;
    return APIC_OK;
}

apic_status apic_momentum_wait(apic_sim* s)
{
    if (!s) return APIC_ERR_ARG;
    if (!s->mom_ready) return APIC_OK;
    CK(cudaSetDevice(s->device), "cudaSetDevice");
    CK(cudaStreamSynchronize(s->mstream), "wait for momentum reads");
    return APIC_OK;
}

apic_status apic_cfl(apic_sim* s, double* max_speed)
{
    if (!s || !max_speed) return APIC_ERR_ARG;
    if (s->batch) {
        apic_status bst = batch_sync_member(s);
        if (bst != APIC_OK) return bst;
    }
    CK(cudaSetDevice(s->device), "cudaSetDevice");
    *max_speed = 0.0;
    if (s->n == 0) return APIC_OK;
    CK(DISPATCH(s, cfl, s->c, s->b, s->cur, s->n, s->L, s->stream), "cfl kernel");
    s->launches += 2;
    CK(cudaMemcpyAsync(max_speed, s->b.mom_out, sizeof(double), cudaMemcpyDeviceToHost, s->stream), "read cfl");
    return check_device(s);
}

apic_status apic_grid_download(apic_sim* s, int which, double* m, double* mv)
{
    if (!s || !m || !mv) return APIC_ERR_ARG;
    if (which == APIC_GRID_MOMENTUM && s->phase != 1) return fail(s, APIC_ERR_ARG, "grid momentum exists only after apic_p2g");
    if (which == APIC_GRID_VELOCITY && s->phase != 2) return fail(s, APIC_ERR_ARG, "grid velocity exists only after apic_grid_update");
    if (which != APIC_GRID_MOMENTUM && which != APIC_GRID_VELOCITY) return fail(s, APIC_ERR_ARG, "bad `which`");
    CK(cudaSetDevice(s->device), "cudaSetDevice");
    const int d = s->c.dim;
    size_t nn = 1;
    for (int a = 0; a < d; ++a) nn *= (size_t)s->c.res[a];
    double* sm = s->b.staging;
    double* smv = sm + nn;
    CK(DISPATCH(s, grid_dense, s->c, s->b, which, sm, smv, s->stream), "grid download kernel");
    CK(cudaMemcpyAsync(m, sm, sizeof(double) * nn, cudaMemcpyDeviceToHost, s->stream), "download grid mass");
    CK(cudaMemcpyAsync(mv, smv, sizeof(double) * nn * d, cudaMemcpyDeviceToHost, s->stream), "download grid vector");
    return check_device(s);
}

apic_status apic_keys_download(apic_sim* s, uint32_t* keys, uint32_t* perm)
{
    if (!s || !keys || !perm) return APIC_ERR_ARG;
    if (s->n > 0 && !s->skeys) return fail(s, APIC_ERR_ARG, "no sort has run since the last upload");
    CK(cudaSetDevice(s->device), "cudaSetDevice");
    if (s->n > 0) {
        CK(cudaMemcpyAsync(keys, s->skeys, 4 * s->n, cudaMemcpyDeviceToHost, s->stream), "download keys");
        CK(cudaMemcpyAsync(perm, s->perm, 4 * s->n, cudaMemcpyDeviceToHost, s->stream), "download perm");
    }
    return check_device(s);
}

apic_status apic_grid_occupancy(apic_sim* s, uint8_t* out, int64_t n_blocks)
{
    if (!s || !out) return APIC_ERR_ARG;
    if (n_blocks != s->c.nblocks) return fail(s, APIC_ERR_ARG, "n_blocks does not match the grid's block count");
    if (s->phase != 1) return fail(s, APIC_ERR_ARG, "occupancy exists only between apic_p2g and apic_grid_update");
    CK(cudaSetDevice(s->device), "cudaSetDevice");
    uint32_t* tmp = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)n_blocks);
    if (!tmp) return fail(s, APIC_ERR_OOM, "host allocation failed");
    cudaError_t e = cudaMemcpyAsync(tmp, s->b.flags, sizeof(uint32_t) * (size_t)n_blocks, cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e == cudaSuccess)
        for (int64_t i = 0; i < n_blocks; ++i) out[i] = tmp[i] ? 1 : 0;
    free(tmp);
    if (e != cudaSuccess) return cuda_fail(s, e, "download occupancy");
    return check_device(s);
}

apic_status apic_stats(apic_sim* s, int64_t out[5])
{
    if (!s || !out) return APIC_ERR_ARG;
    CK(cudaSetDevice(s->device), "cudaSetDevice");
    uint32_t nt = 0, fb = 0;
    CK(cudaMemcpyAsync(&nt, s->b.ntiles, 4, cudaMemcpyDeviceToHost, s->stream), "read tile count");
    CK(cudaMemcpyAsync(&fb, s->b.fallbacks, 4, cudaMemcpyDeviceToHost, s->stream), "read fallback count");
    CK(cudaStreamSynchronize(s->stream), "synchronize");
    out[0] = s->n;
    out[1] = s->c.nblocks;
    out[2] = nt;
    out[3] = fb;
    out[4] = s->launches;
    return APIC_OK;
}

apic_status apic_profile(apic_sim* s, int enable)
{
    if (!s) return APIC_ERR_ARG;
    s->prof_on = enable != 0;
    if (enable) {
        s->recs.clear();
        s->ev_used = 0;
    }
    return APIC_OK;
}

apic_status apic_profile_read(apic_sim* s, double ms[APIC_NPHASE], int64_t launches[APIC_NPHASE])
{
    if (!s || !ms || !launches) return APIC_ERR_ARG;
    CK(cudaSetDevice(s->device), "cudaSetDevice");
    CK(cudaStreamSynchronize(s->stream), "synchronize");
    for (int i = 0; i < APIC_NPHASE; ++i) {
        ms[i] = 0.0;
        launches[i] = 0;
    }
    for (const auto& r : s->recs) {
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, r.a, r.b), "event elapsed time");
        ms[r.phase] += t;
        launches[r.phase] += r.kernels;
    }
    return APIC_OK;
}

apic_status apic_solve_stats(apic_sim* s, double out[3])
{
    if (!s || !out) return APIC_ERR_ARG;
    for (int i = 0; i < 3; ++i) out[i] = s->solve_stats[i];
    return APIC_OK;
}

apic_status apic_set_wait_limit(apic_sim* s, unsigned polls)
{
    if (!s) return APIC_ERR_ARG;
    if (s->batch) return fail(s, APIC_ERR_ARG, "the simulation is a member of a batch");
    s->c.wait_limit = polls;
    return APIC_OK;
}

const char* apic_last_error(apic_sim* s)
{
    if (!s) return "NULL simulation";
    return s->err.c_str();
}

}  // extern "C"

// ====================================================================== batched stepping
struct apic_batch {
    int dim, order, precision;
    int max_sims;
    int64_t max_particles, max_blocks;
    int tile, group;
    bool use_graph;
    cudaStream_t stream;
    int device;
    int sms;
    // workspace
    void* descs;
    SortDesc* sortdescs;
    uint32_t *rt_sim, *ch_sim, *bbase, *scan_part, *chunk_cnt, *tile_sim, *tile_start, *ntiles, *tile_ctr, *err,
        *bsorted, *bctl;
    int64_t max_rtiles, max_chunks, max_tiles;
    size_t desc_bytes;
    // membership
    std::vector<apic_sim*> members;
    std::vector<apic_sim*> uploaded;   // simulations whose descriptors are on the device, in order
    bool dirty;
    uint32_t total_rtiles, total_chunks, total_blocks;
    int64_t total_particles;
    int passes;
    int p2g_grid, g2p_grid, grid_grid;
    int64_t steps, launches;
    // graph
    cudaGraphExec_t gexec;
    bool graph_valid;
    std::string err_msg;
    // serving ledger: steps left and device footprint of the members admitted with
    // apic_batch_admit (members added with apic_batch_add have no entry)
    struct Ledger { int steps_left; int64_t footprint; };
    std::map<apic_sim*, Ledger> ledger;
    int64_t resident_bytes;
};

namespace {

constexpr int kBatchTiles[3] = {1024, 2048, 4096};

struct BatchLayout {
    size_t descs, sortdescs, rt_sim, ch_sim, bbase, scan_part, chunk_cnt, tile_sim, tile_start, ntiles, tile_ctr,
        err, bsorted, bctl, total;
    int64_t max_rtiles, max_chunks, max_tiles;
};

BatchLayout batch_layout(const apic_batch_config* c)
{
    BatchLayout L;
    Carve cv;
    const size_t db = c->precision == 32 ? batch_desc_bytes_f32() : batch_desc_bytes_f64();
    L.max_rtiles = c->max_particles / 2048 + c->max_sims + 1;
    L.max_chunks = c->max_particles / 1024 + c->max_sims + 1;
    L.max_tiles = L.max_chunks + (c->max_particles < c->max_blocks ? c->max_particles : c->max_blocks) + 2;
    L.descs = cv.take((size_t)c->max_sims * db);
    L.sortdescs = cv.take((size_t)c->max_sims * sizeof(SortDesc));
    L.rt_sim = cv.take((size_t)L.max_rtiles * 4);
    L.ch_sim = cv.take((size_t)L.max_chunks * 4);
    L.bbase = cv.take((size_t)(c->max_sims + 1) * 4);
    const int64_t scan_n = L.max_chunks;
    L.scan_part = cv.take(((size_t)(scan_n + 4095) / 4096 + 2) * 4);
    L.chunk_cnt = cv.take((size_t)L.max_chunks * 4);
    L.tile_sim = cv.take((size_t)L.max_tiles * 4);
    L.tile_start = cv.take((size_t)L.max_tiles * 4);
    L.ntiles = cv.take(4);
    L.tile_ctr = cv.take(16);
    L.err = cv.take(4);
    L.bsorted = cv.take((size_t)c->max_sims * 4);   // member stored in its previous sorted order
    L.bctl = cv.take(32);                            // sort epoch, pass tile counters
    L.total = cv.cur;
    return L;
}

apic_status batch_fail(apic_batch* b, apic_status st, const std::string& why)
{
    if (b) b->err_msg = why;
    return st;
}

#define BCK(expr, where)                                                                     \
    do {                                                                                     \
        cudaError_t e_ = (expr);                                                             \
        if (e_ != cudaSuccess) return batch_fail(b, APIC_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// Copy the device-side state parity back into the host structs of the simulations whose
// descriptors are on the device (the member list as of the last rebuild -- members added
// since then have no descriptor yet and keep their host value).
apic_status batch_pull_cur(apic_batch* b)
{
    const size_t n = b->uploaded.size();
    if (n == 0) return APIC_OK;
    std::vector<unsigned char> h(n * b->desc_bytes);
    BCK(cudaMemcpyAsync(h.data(), b->descs, h.size(), cudaMemcpyDeviceToHost, b->stream), "read descriptors");
    BCK(cudaStreamSynchronize(b->stream), "synchronize");
    const int off = b->precision == 32 ? batch_desc_cur_offset_f32() : batch_desc_cur_offset_f64();
    for (size_t i = 0; i < n; ++i) {
        int cur;
        memcpy(&cur, h.data() + i * b->desc_bytes + off, sizeof(int));
        if (!b->uploaded[i]) continue;
        if (cur != 0 && cur != 1) return batch_fail(b, APIC_ERR_CUDA, "corrupt state parity in a batch descriptor");
        b->uploaded[i]->cur = cur;
    }
    return APIC_OK;
}

apic_status batch_rebuild(apic_batch* b)
{
    {
        apic_status st = batch_pull_cur(b);   // parity of the previous descriptors first
        if (st != APIC_OK) return st;
    }
    const size_t S = b->members.size();
    std::vector<unsigned char> descs(S * b->desc_bytes);
    std::vector<SortDesc> sds(S);
    std::vector<uint32_t> rt, ch, bb(S + 1, 0);
    uint32_t pbase = 0, rbase = 0, cbase = 0, blocks = 0;
    int maxbits = 1;
    for (size_t i = 0; i < S; ++i) {
        apic_sim* m = b->members[i];
        if (b->precision == 32) batch_make_desc_f32(m->c, m->b, m->cur, m->n, descs.data() + i * b->desc_bytes);
        else batch_make_desc_f64(m->c, m->b, m->cur, m->n, descs.data() + i * b->desc_bytes);
        SortDesc& d = sds[i];
        d.knext = m->b.knext;
        d.kb[0] = m->b.kA;
        d.kb[1] = m->b.kB;
        d.vb[0] = m->b.vA;
        d.vb[1] = m->b.vB;
        for (int q = 0; q < 2; ++q) {
            d.mk[q] = m->b.mk[q];
            d.mv[q] = m->b.mv[q];
        }
        d.midx = m->b.midx;
        d.choff = m->b.choff;
        d.mcnt = m->b.mcnt;
        d.mctl = m->b.mctl;
        d.lbs = m->b.lbs;
        d.n = (uint32_t)m->n;
        d.ntl = (uint32_t)radix_tiles(m->n);
        d.nch = (uint32_t)((m->n + b->tile - 1) / b->tile);
        d.pbase = pbase;
        d.rbase = rbase;
        d.cbase = cbase;
        for (uint32_t t = 0; t < d.ntl; ++t) rt.push_back((uint32_t)i);
        for (uint32_t t = 0; t < d.nch; ++t) ch.push_back((uint32_t)i);
        bb[i] = blocks;
        pbase += d.n;
        rbase += d.ntl;
        cbase += d.nch;
        blocks += (uint32_t)m->c.nblocks;
        if (m->c.key_bits > maxbits) maxbits = m->c.key_bits;
    }
    bb[S] = blocks;
    if ((int64_t)rt.size() > b->max_rtiles || (int64_t)ch.size() > b->max_chunks)
        return batch_fail(b, APIC_ERR_OOM, "batch work-list capacity exceeded");
    b->total_rtiles = rbase;
    b->total_chunks = cbase;
    b->total_blocks = blocks;
    b->total_particles = pbase;
    b->passes = (maxbits + 7) / 8;
    if (S > 0) {
        BCK(cudaMemcpyAsync(b->descs, descs.data(), descs.size(), cudaMemcpyHostToDevice, b->stream), "upload descriptors");
        BCK(cudaMemcpyAsync(b->sortdescs, sds.data(), sds.size() * sizeof(SortDesc), cudaMemcpyHostToDevice, b->stream), "upload sort descriptors");
        if (!rt.empty()) BCK(cudaMemcpyAsync(b->rt_sim, rt.data(), rt.size() * 4, cudaMemcpyHostToDevice, b->stream), "upload tables");
        if (!ch.empty()) BCK(cudaMemcpyAsync(b->ch_sim, ch.data(), ch.size() * 4, cudaMemcpyHostToDevice, b->stream), "upload tables");
        BCK(cudaMemcpyAsync(b->bbase, bb.data(), bb.size() * 4, cudaMemcpyHostToDevice, b->stream), "upload tables");
        // after a membership change every member takes one full sort (its keys' home buffer
        // follows the pass count, which the new members may change)
        BCK(cudaMemsetAsync(b->bsorted, 0, S * sizeof(uint32_t), b->stream), "clear sorted flags");
        BCK(cudaStreamSynchronize(b->stream), "synchronize");   // host vectors die at return
    }
    int p2g_per = 1, g2p_per = 1;
    cudaError_t e = b->precision == 32 ? batch_setup_f32(b->dim, b->order, b->group, &p2g_per, &g2p_per)
                                       : batch_setup_f64(b->dim, b->order, b->group, &p2g_per, &g2p_per);
    BCK(e, "batch kernel setup");
    b->p2g_grid = b->sms * (p2g_per > 0 ? p2g_per : 1);
    b->g2p_grid = b->sms * (g2p_per > 0 ? g2p_per : 1);
    b->grid_grid = b->sms * 8;
    if (b->graph_valid) {
        cudaGraphExecDestroy(b->gexec);
        b->graph_valid = false;
    }
    b->uploaded = b->members;
    b->dirty = false;
    return APIC_OK;
}

// the kernels of one batched step
cudaError_t batch_enqueue(apic_batch* b)
{
    const int kpar = (b->passes - 1) & 1;
    const int S = (int)b->members.size();
    cudaError_t e = batch_resort(b->sortdescs, b->rt_sim, b->total_rtiles, S, b->passes, kpar, b->bsorted, b->bctl,
                                 b->err, b->sms, b->stream);
    if (e == cudaSuccess)
        e = batch_build_tiles(b->sortdescs, b->ch_sim, b->total_chunks, b->dim, b->tile, kpar, b->chunk_cnt, b->scan_part,
                              b->ntiles, b->max_tiles, b->tile_sim, b->tile_start, b->err, b->tile_ctr, b->stream);
    if (e == cudaSuccess)
        e = b->precision == 32 ? batch_p2g_f32(b->dim, b->order, b->group, b->descs, b->tile_sim, b->tile_start, b->ntiles,
                                               b->tile_ctr, kpar, b->p2g_grid, b->stream)
                               : batch_p2g_f64(b->dim, b->order, b->group, b->descs, b->tile_sim, b->tile_start, b->ntiles,
                                               b->tile_ctr, kpar, b->p2g_grid, b->stream);
    if (e == cudaSuccess)
        e = b->precision == 32 ? batch_grid_f32(b->dim, b->descs, b->bbase, S, b->total_blocks, b->grid_grid, b->stream)
                               : batch_grid_f64(b->dim, b->descs, b->bbase, S, b->total_blocks, b->grid_grid, b->stream);
    int ext = 0;   // some member carries a material per particle
    for (apic_sim* m : b->members) ext |= m->c.mat;
    if (e == cudaSuccess)
        e = b->precision == 32 ? batch_g2p_f32(b->dim, b->order, ext, b->descs, b->tile_sim, b->tile_start, b->ntiles,
                                               b->tile_ctr, kpar, b->g2p_grid, b->stream)
                               : batch_g2p_f64(b->dim, b->order, ext, b->descs, b->tile_sim, b->tile_start, b->ntiles,
                                               b->tile_ctr, kpar, b->g2p_grid, b->stream);
    if (e == cudaSuccess)
        e = b->precision == 32 ? batch_finish_f32(b->descs, S, b->bsorted, b->stream)
                               : batch_finish_f64(b->descs, S, b->bsorted, b->stream);
    return e;
}

// sort and tile list, then P2G, grid update, G2P and the parity flip
int64_t batch_kernels_per_step(const apic_batch* b) { return batch_sort_and_tiles_kernels(b->passes) + 4; }

apic_status batch_run(apic_batch* b, int n)
{
    if (b->dirty) {
        apic_status st = batch_rebuild(b);
        if (st != APIC_OK) return st;
    }
    if (b->members.empty()) return APIC_OK;
    BCK(cudaSetDevice(b->device), "cudaSetDevice");
    for (int i = 0; i < n; ++i) {
        if (b->use_graph && b->stream) {
            if (!b->graph_valid) {
                cudaGraph_t g;
                BCK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
                cudaError_t e = batch_enqueue(b);
                cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
                BCK(e, "capture step");
                BCK(e2, "end capture");
                e = cudaGraphInstantiate(&b->gexec, g, 0);
                cudaGraphDestroy(g);
                BCK(e, "instantiate graph");
                b->graph_valid = true;
            }
            BCK(cudaGraphLaunch(b->gexec, b->stream), "graph launch");
        } else {
            BCK(batch_enqueue(b), "batched step");
        }
        b->steps += 1;
        b->launches += batch_kernels_per_step(b);
    }
    return APIC_OK;
}

// (dim, order, precision, log2 of particles) -> (tile, group)
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int>, std::pair<int, int>> g_tune_cache;

apic_status batch_sync_member(apic_sim* s)
{
    apic_batch* b = s->batch;
    apic_status st = batch_pull_cur(b);
    if (st != APIC_OK) return fail(s, st, b->err_msg);
    s->keys_valid = b->steps > 0 ? true : s->keys_valid;
    return APIC_OK;
}

}  // namespace

extern "C" {

apic_status apic_batch_workspace_size(const apic_batch_config* c, size_t* bytes)
{
    if (!c || !bytes) return APIC_ERR_ARG;
    if (c->max_sims <= 0 || c->max_sims > 12000 || c->max_particles <= 0 || c->max_blocks <= 0) return APIC_ERR_ARG;
    if (c->precision != 32 && c->precision != 64) return APIC_ERR_ARG;
    *bytes = batch_layout(c).total;
    return APIC_OK;
}

apic_status apic_batch_create(const apic_batch_config* c, void* workspace, size_t workspace_bytes, void* stream,
                              apic_batch** out)
{
    if (!c || !out) return APIC_ERR_ARG;
    *out = nullptr;
    if ((c->dim != 2 && c->dim != 3) || (c->order != 2 && c->order != 3)) return APIC_ERR_ARG;
    if (c->precision != 32 && c->precision != 64) return APIC_ERR_ARG;
    if (c->max_sims <= 0 || c->max_sims > 12000 || c->max_particles <= 0 || c->max_blocks <= 0) return APIC_ERR_ARG;
    const int tile = c->tile_particles == 0 ? 4096 : c->tile_particles;
    if (tile != 1024 && tile != 2048 && tile != 4096) return APIC_ERR_ARG;
    const int group = c->group == 0 ? (c->dim == 3 ? APIC_BATCH_SPLIT : 8) : c->group;
    if (group != 1 && group != 2 && group != 4 && group != 8 && group != APIC_BATCH_SPLIT) return APIC_ERR_ARG;
    if (group == APIC_BATCH_SPLIT && c->dim != 3) return APIC_ERR_ARG;
    if (!workspace || ((uintptr_t)workspace & 255)) return APIC_ERR_ARG;
    BatchLayout L = batch_layout(c);
    if (workspace_bytes < L.total) return APIC_ERR_OOM;
    apic_batch* b = new (std::nothrow) apic_batch();
    if (!b) return APIC_ERR_OOM;
    b->dim = c->dim;
    b->order = c->order;
    b->precision = c->precision;
    b->max_sims = c->max_sims;
    b->max_particles = c->max_particles;
    b->max_blocks = c->max_blocks;
    b->tile = tile;
    b->group = group;
    b->use_graph = c->use_graph != 0;
    b->stream = (cudaStream_t)stream;
    char* base = (char*)workspace;
    b->descs = base + L.descs;
    b->sortdescs = (SortDesc*)(base + L.sortdescs);
    b->rt_sim = (uint32_t*)(base + L.rt_sim);
    b->ch_sim = (uint32_t*)(base + L.ch_sim);
    b->bbase = (uint32_t*)(base + L.bbase);

    b->scan_part = (uint32_t*)(base + L.scan_part);
    b->chunk_cnt = (uint32_t*)(base + L.chunk_cnt);
    b->tile_sim = (uint32_t*)(base + L.tile_sim);
    b->tile_start = (uint32_t*)(base + L.tile_start);
    b->ntiles = (uint32_t*)(base + L.ntiles);
    b->tile_ctr = (uint32_t*)(base + L.tile_ctr);
    b->err = (uint32_t*)(base + L.err);
    b->bsorted = (uint32_t*)(base + L.bsorted);
    b->bctl = (uint32_t*)(base + L.bctl);
    b->max_rtiles = L.max_rtiles;
    b->max_chunks = L.max_chunks;
    b->max_tiles = L.max_tiles;
    b->desc_bytes = c->precision == 32 ? batch_desc_bytes_f32() : batch_desc_bytes_f64();
    b->dirty = true;
    b->total_rtiles = b->total_chunks = b->total_blocks = 0;
    b->total_particles = 0;
    b->passes = 1;
    b->steps = b->launches = 0;
    b->graph_valid = false;
    b->resident_bytes = 0;
    cudaError_t e = cudaGetDevice(&b->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->err, 0, 4, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->ntiles, 0, 4, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->bctl, 0, 32, b->stream);
    if (e != cudaSuccess) {
        delete b;
        return APIC_ERR_CUDA;
    }
    *out = b;
    return APIC_OK;
}

apic_status apic_batch_destroy(apic_batch* b)
{
    if (!b) return APIC_ERR_ARG;
    while (!b->members.empty()) apic_batch_remove(b, b->members.back());
    if (b->graph_valid) cudaGraphExecDestroy(b->gexec);
    cudaStreamSynchronize(b->stream);
    delete b;
    return APIC_OK;
}

apic_status apic_batch_add(apic_batch* b, apic_sim* s)
{
    if (!b || !s) return APIC_ERR_ARG;
    if (s->batch) return batch_fail(b, APIC_ERR_ARG, "the simulation is already a member of a batch");
    if (s->c.dim != b->dim || s->c.order != b->order || s->c.precision != b->precision)
        return batch_fail(b, APIC_ERR_ARG, "dim, order and precision must match the batch");
    if (s->n <= 0) return batch_fail(b, APIC_ERR_ARG, "the simulation has no particles");
    if (s->phase != 0) return batch_fail(b, APIC_ERR_ARG, "the simulation is in the middle of a step");
    if (s->c.transfer == APIC_TRANSFER_FLIP)
        return batch_fail(b, APIC_ERR_UNSUPPORTED, "FLIP simulations are stepped on their own, not in batches");
    if (s->c.integrator != APIC_INTEGRATOR_LAMBDA0)
        return batch_fail(b, APIC_ERR_UNSUPPORTED, "lambda = 1 and midpoint simulations are stepped on their own, not in batches");
    if ((int)b->members.size() >= b->max_sims) return batch_fail(b, APIC_ERR_OOM, "batch member capacity reached");
    int64_t parts = 0, blocks = 0;
    for (apic_sim* m : b->members) {
        parts += m->n;
        blocks += m->c.nblocks;
    }
    if (parts + s->n > b->max_particles) return batch_fail(b, APIC_ERR_OOM, "batch particle capacity reached");
    if (blocks + s->c.nblocks > b->max_blocks) return batch_fail(b, APIC_ERR_OOM, "batch block capacity reached");
    BCK(cudaSetDevice(b->device), "cudaSetDevice");
    apic_status st = batch_pull_cur(b);   // keep the members' parity before the descriptors are rebuilt
    if (st != APIC_OK) return st;
    if (!s->keys_valid) {
        cudaError_t e = s->c.precision == 32 ? keys_f32(s->c, s->b, s->cur, s->n, s->stream)
                                             : keys_f64(s->c, s->b, s->cur, s->n, s->stream);
        BCK(e, "keys kernel");
        s->keys_valid = true;
        s->launches += 1;
    }
    BCK(mom_fence(s, -1), "wait for momentum reads");   // batch kernels will write the state
    // look-back words of the batch's sort epochs start clear
    BCK(cudaMemsetAsync(s->b.lbs, 0, sizeof(unsigned long long) * 256 * ((size_t)radix_tiles(s->c.capacity) + 1),
                        s->stream), "clear look-back words");
    BCK(cudaStreamSynchronize(s->stream), "synchronize member stream");
    s->order_sorted = false;
    s->batch = b;
    b->members.push_back(s);
    b->dirty = true;
    return APIC_OK;
}

apic_status apic_batch_remove(apic_batch* b, apic_sim* s)
{
    if (!b || !s || s->batch != b) return APIC_ERR_ARG;
    apic_status st = batch_pull_cur(b);
    if (st != APIC_OK) return st;
    for (size_t i = 0; i < b->members.size(); ++i)
        if (b->members[i] == s) {
            b->members.erase(b->members.begin() + (long)i);
            break;
        }
    // its descriptor stays on the device until the next rebuild, but its parity is now
    // owned by the host again: forget it so no later pull overwrites it
    for (size_t i = 0; i < b->uploaded.size(); ++i)
        if (b->uploaded[i] == s) b->uploaded[i] = nullptr;
    s->batch = nullptr;
    s->phase = 0;
    if (b->steps > 0) {
        const int kpar = (b->passes - 1) & 1;
        s->skeys = kpar ? s->b.kB : s->b.kA;
        s->perm = kpar ? s->b.vB : s->b.vA;
        s->keys_valid = true;
        s->order_sorted = true;   // batched G2P also stores particle k of the sorted order at k
    }
    s->epoch = 0;   // its look-back words hold batch epochs: the next single sort clears them
    auto it = b->ledger.find(s);
    if (it != b->ledger.end()) {
        b->resident_bytes -= it->second.footprint;
        b->ledger.erase(it);
    }
    b->dirty = true;
    return APIC_OK;
}

apic_status apic_batch_admit(apic_batch* b, apic_sim* s, int steps, int64_t footprint_bytes, int64_t budget_bytes)
{
    if (!b || !s || steps <= 0 || footprint_bytes < 0 || budget_bytes < 0) return APIC_ERR_ARG;
    if (b->resident_bytes + footprint_bytes > budget_bytes)
        return batch_fail(b, APIC_ERR_OOM, "the simulation's footprint does not fit the memory budget now");
    apic_status st = apic_batch_add(b, s);
    if (st != APIC_OK) return st;
    b->ledger[s] = {steps, footprint_bytes};
    b->resident_bytes += footprint_bytes;
    return APIC_OK;
}

apic_status apic_batch_run(apic_batch* b, int max_steps, apic_sim** finished, int max_finished, int* n_finished,
                           int* steps_done)
{
    if (!b || max_steps <= 0 || !n_finished) return APIC_ERR_ARG;
    *n_finished = 0;
    if (steps_done) *steps_done = 0;
    if (!b->ledger.empty() && (!finished || max_finished < (int)b->ledger.size()))
        return batch_fail(b, APIC_ERR_ARG, "`finished` needs room for every admitted member");
    if (b->members.empty()) return APIC_OK;
    int k = max_steps;
    for (const auto& e : b->ledger) k = e.second.steps_left < k ? e.second.steps_left : k;
    apic_status st = batch_run(b, k);
    if (st != APIC_OK) return st;
    if (steps_done) *steps_done = k;
    std::vector<apic_sim*> done;
    for (auto& e : b->ledger) {
        e.second.steps_left -= k;
        if (e.second.steps_left == 0) done.push_back(e.first);
    }
    // retire in membership order, so the report does not depend on pointer values
    std::vector<apic_sim*> order;
    for (apic_sim* m : b->members)
        for (apic_sim* d : done)
            if (d == m) order.push_back(m);
    for (apic_sim* m : order) {
        st = apic_batch_remove(b, m);
        if (st != APIC_OK) return st;
        finished[(*n_finished)++] = m;
    }
    return APIC_OK;
}

apic_status apic_batch_resident_bytes(apic_batch* b, int64_t* bytes)
{
    if (!b || !bytes) return APIC_ERR_ARG;
    *bytes = b->resident_bytes;
    return APIC_OK;
}

apic_status apic_batch_step(apic_batch* b, int n)
{
    if (!b || n < 0) return APIC_ERR_ARG;
    return batch_run(b, n);
}

apic_status apic_batch_set_tuning(apic_batch* b, int tile, int group)
{
    if (!b) return APIC_ERR_ARG;
    if (tile != 0 && tile != 1024 && tile != 2048 && tile != 4096) return APIC_ERR_ARG;
    if (group != 0 && group != 1 && group != 2 && group != 4 && group != 8 && group != APIC_BATCH_SPLIT) return APIC_ERR_ARG;
    if (group == APIC_BATCH_SPLIT && b->dim != 3) return APIC_ERR_ARG;
    if (tile) b->tile = tile;
    if (group) b->group = group;
    b->dirty = true;
    return APIC_OK;
}

apic_status apic_batch_autotune(apic_batch* b, int steps, int force, int* tile_out, int* group_out)
{
    if (!b || steps <= 0) return APIC_ERR_ARG;
    int64_t parts = 0;
    for (apic_sim* m : b->members) parts += m->n;
    int bucket = 0;
    while (((int64_t)1 << bucket) < parts) ++bucket;
    const auto key = std::make_tuple(b->dim, b->order, b->precision, bucket);
    if (!force) {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            apic_batch_set_tuning(b, it->second.first, it->second.second);
            if (tile_out) *tile_out = b->tile;
            if (group_out) *group_out = b->group;
            return APIC_OK;
        }
    }
    if (b->members.empty()) return APIC_OK;
    cudaEvent_t e0, e1;
    BCK(cudaEventCreate(&e0), "event");
    BCK(cudaEventCreate(&e1), "event");
    float best = 1e30f;
    int bt = b->tile, bg = b->group;
    const int groups[5] = {1, 2, 4, 8, APIC_BATCH_SPLIT};
    for (int tile : kBatchTiles)
        for (int group : groups) {
            if (group == APIC_BATCH_SPLIT && b->dim != 3) continue;
            apic_batch_set_tuning(b, tile, group);
            apic_status st = batch_run(b, 1);   // warm-up (and graph capture)
            if (st != APIC_OK) return st;
            BCK(cudaEventRecord(e0, b->stream), "event record");
            st = batch_run(b, steps);
            if (st != APIC_OK) return st;
            BCK(cudaEventRecord(e1, b->stream), "event record");
            BCK(cudaEventSynchronize(e1), "event sync");
            float ms = 0.f;
            BCK(cudaEventElapsedTime(&ms, e0, e1), "elapsed");
            if (ms < best) {
                best = ms;
                bt = tile;
                bg = group;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    apic_batch_set_tuning(b, bt, bg);
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune_cache[key] = std::make_pair(bt, bg);
    }
    if (tile_out) *tile_out = bt;
    if (group_out) *group_out = bg;
    return APIC_OK;
}

apic_status apic_batch_stats(apic_batch* b, int64_t out[5])
{
    if (!b || !out) return APIC_ERR_ARG;
    uint32_t nt = 0, e = 0;
    BCK(cudaMemcpyAsync(&nt, b->ntiles, 4, cudaMemcpyDeviceToHost, b->stream), "read tile count");
    BCK(cudaMemcpyAsync(&e, b->err, 4, cudaMemcpyDeviceToHost, b->stream), "read error word");
    BCK(cudaStreamSynchronize(b->stream), "synchronize");
    int64_t parts = 0;
    for (apic_sim* m : b->members) parts += m->n;
    out[0] = (int64_t)b->members.size();
    out[1] = parts;
    out[2] = b->steps;
    out[3] = b->launches;
    out[4] = nt;
    if (e & APIC_ERRBIT_TIMEOUT) return batch_fail(b, APIC_ERR_TIMEOUT, "a bounded device wait (sort look-back) ran out");
    if (e) return batch_fail(b, APIC_ERR_OOM, "batch tile capacity exceeded");
    return APIC_OK;
}

const char* apic_batch_last_error(apic_batch* b)
{
    if (!b) return "NULL batch";
    return b->err_msg.c_str();
}

}  // extern "C"
