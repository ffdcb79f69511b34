// apic_abi.cu -- the C ABI declared in include/apic.h: argument checking, workspace
// carving, call sequencing and error reporting.  Every step of the method runs in the
// kernels of apic_sort.cu and apic_transfer_*.cu; this file only launches them.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <string>
#include <vector>

#include "apic.h"
#include "apic_internal.h"

using namespace apic;

struct apic_sim {
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
    int64_t max_tiles;
    std::string err;
    int64_t launches;      // kernels launched since creation
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
    if (in->transfer != APIC_TRANSFER_APIC && in->transfer != APIC_TRANSFER_PIC) { *why = "unknown transfer"; return APIC_ERR_ARG; }
    if (in->boundary != APIC_BOUNDARY_NONE && in->boundary != APIC_BOUNDARY_STICKY) { *why = "unknown boundary"; return APIC_ERR_UNSUPPORTED; }
    if (in->model != APIC_MODEL_NONE && in->model != APIC_MODEL_FIXED_COROTATED) { *why = "unknown constitutive model"; return APIC_ERR_UNSUPPORTED; }
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
    if (in->model == APIC_MODEL_FIXED_COROTATED) {
        if (!(in->E > 0.0) || !(in->nu > -1.0 && in->nu < 0.5)) { *why = "E must be > 0 and -1 < nu < 0.5"; return APIC_ERR_ARG; }
        c->mu = in->E / (2.0 * (1.0 + in->nu));
        c->lam = in->E * in->nu / ((1.0 + in->nu) * (1.0 - 2.0 * in->nu));
    }
    c->mass = in->particle_mass;
    c->vol = in->particle_volume;
    c->tile = tile;
    if (in->p2g_kernel < 0 || in->p2g_kernel > 3) { *why = "p2g_kernel must be 0, 1, 2 or 3"; return APIC_ERR_ARG; }
    c->p2g_kernel = in->p2g_kernel == 0 ? 1 : in->p2g_kernel;
    if (c->p2g_kernel == 2 && in->dim == 3 && in->order == 3) { *why = "the cell-parallel P2G does not cover 3-D cubic"; return APIC_ERR_UNSUPPORTED; }
    c->key_bits = 2 * in->dim + ceil_log2(c->nblocks);
    if (c->key_bits > 32) { *why = "grid too large for 32-bit cell keys"; return APIC_ERR_UNSUPPORTED; }
    c->capacity = max_particles;
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
    size_t st[2][7];
    size_t knext, kA, kB, vA, vB, radix_counts, scan_part, tiles, chunk_cnt, ntiles, tile_ctr;
    size_t acc, vel, flags, mom_part, mom_out, err, fallbacks, staging;
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
        for (int i = 0; i < 6; ++i) L.st[s][i] = cv.take((size_t)n * 4 * R);
        L.st[s][6] = cv.take((size_t)n * 2 * R);
    }
    L.knext = cv.take((size_t)n * 4);
    L.kA = cv.take((size_t)n * 4);
    L.kB = cv.take((size_t)n * 4);
    L.vA = cv.take((size_t)n * 4);
    L.vB = cv.take((size_t)n * 4);
    L.radix_counts = cv.take((size_t)256 * radix_tiles(n) * 4);
    const int64_t nchunks = (n + c.tile - 1) / c.tile;
    L.scan_part = cv.take(scan_partials_needed(n > nchunks ? n : nchunks) * 4);
    L.max_tiles = nchunks + (n < c.nblocks ? n : c.nblocks) + 2;
    L.tiles = cv.take((size_t)(L.max_tiles + 1) * 4);
    L.chunk_cnt = cv.take((size_t)(nchunks + 1) * 4);
    L.ntiles = cv.take(4);
    L.tile_ctr = cv.take(8);
    const size_t bn = c.dim == 3 ? 64 : 16;
    L.acc = cv.take((size_t)c.nblocks * bn * 4 * R);
    L.vel = cv.take((size_t)c.nblocks * bn * 4 * R);
    L.flags = cv.take((size_t)c.nblocks * 4);
    L.mom_part = cv.take((size_t)kMomParts * 6 * 8);
    L.mom_out = cv.take(6 * 8);
    L.err = cv.take(4);
    L.fallbacks = cv.take(4);
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

// read and clear the latched device error word (synchronises the stream)
apic_status check_device(apic_sim* s)
{
    uint32_t e = 0;
    CK(cudaMemcpyAsync(&e, s->b.err, 4, cudaMemcpyDeviceToHost, s->stream), "read error word");
    CK(cudaStreamSynchronize(s->stream), "synchronize");
    if (e == 0) return APIC_OK;
    CK(cudaMemsetAsync(s->b.err, 0, 4, s->stream), "clear error word");
    CK(cudaStreamSynchronize(s->stream), "synchronize");
    if (e & APIC_ERRBIT_TIMEOUT) return fail(s, APIC_ERR_TIMEOUT, "a bounded device wait (bulk copy completion) ran out");
    if (e & APIC_ERRBIT_CAPACITY) return fail(s, APIC_ERR_OOM, "tile list capacity exceeded");
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

#define DISPATCH(s, fn, ...) ((s)->c.precision == 32 ? fn##_f32(__VA_ARGS__) : fn##_f64(__VA_ARGS__))

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
    s->c = c;
    s->stream = (cudaStream_t)stream;
    s->cur = 0;
    s->n = 0;
    s->keys_valid = false;
    s->phase = 0;
    s->skeys = s->perm = nullptr;
    s->max_tiles = L.max_tiles;
    s->launches = 0;
    s->prof_on = false;
    s->ev_used = 0;
    char* base = (char*)workspace;
    for (int a = 0; a < 2; ++a)
        for (int i = 0; i < 7; ++i) s->b.st[a][i] = base + L.st[a][i];
    s->b.knext = (uint32_t*)(base + L.knext);
    s->b.kA = (uint32_t*)(base + L.kA);
    s->b.kB = (uint32_t*)(base + L.kB);
    s->b.vA = (uint32_t*)(base + L.vA);
    s->b.vB = (uint32_t*)(base + L.vB);
    s->b.radix_counts = (uint32_t*)(base + L.radix_counts);
    s->b.scan_part = (uint32_t*)(base + L.scan_part);
    s->b.tiles = (uint32_t*)(base + L.tiles);
    s->b.chunk_cnt = (uint32_t*)(base + L.chunk_cnt);
    s->b.ntiles = (uint32_t*)(base + L.ntiles);
    s->b.tile_ctr = (uint32_t*)(base + L.tile_ctr);
    s->b.acc = base + L.acc;
    s->b.vel = base + L.vel;
    s->b.flags = (uint32_t*)(base + L.flags);
    s->b.mom_part = (double*)(base + L.mom_part);
    s->b.mom_out = (double*)(base + L.mom_out);
    s->b.err = (uint32_t*)(base + L.err);
    s->b.fallbacks = (uint32_t*)(base + L.fallbacks);
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
    s->L.p2g_cells = c.p2g_kernel == 2;
    s->L.g2p_grid = sms * (g2p_per > 0 ? g2p_per : 1);
    s->L.mom_parts = kMomParts;
    const size_t bn = c.dim == 3 ? 64 : 16;
    const size_t gbytes = (size_t)c.nblocks * bn * 4 * (c.precision == 32 ? 4 : 8);
    e = cudaMemsetAsync(s->b.acc, 0, gbytes, s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->b.vel, 0, gbytes, s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->b.flags, 0, (size_t)c.nblocks * 4, s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->b.err, 0, 4, s->stream);
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
    cudaError_t e = cudaStreamSynchronize(s->stream);
    for (cudaEvent_t ev : s->ev_pool) cudaEventDestroy(ev);
    delete s;
    return e == cudaSuccess ? APIC_OK : APIC_ERR_CUDA;
}

apic_status apic_upload(apic_sim* s, int64_t n, const double* x, const double* v, const double* B, const double* F,
                        int on_device)
{
    if (!s) return APIC_ERR_ARG;
    if (n < 0) return fail(s, APIC_ERR_ARG, "n < 0");
    if (n > s->c.capacity) return fail(s, APIC_ERR_OOM, "n exceeds the particle capacity given to apic_create");
    if (n > 0 && !x) return fail(s, APIC_ERR_ARG, "positions are required");
    CK(cudaSetDevice(s->device), "cudaSetDevice");
    const int d = s->c.dim;
    const double *dx_ = x, *dv = v, *dB = B, *dF = F;
    if (!on_device && n > 0) {
        double* st = s->b.staging;
        double* sx = st;
        double* sv = sx + n * d;
        double* sB = sv + n * d;
        double* sF = sB + n * d * d;
        CK(cudaMemcpyAsync(sx, x, sizeof(double) * n * d, cudaMemcpyHostToDevice, s->stream), "upload x");
        if (v) CK(cudaMemcpyAsync(sv, v, sizeof(double) * n * d, cudaMemcpyHostToDevice, s->stream), "upload v");
        if (B) CK(cudaMemcpyAsync(sB, B, sizeof(double) * n * d * d, cudaMemcpyHostToDevice, s->stream), "upload B");
        if (F) CK(cudaMemcpyAsync(sF, F, sizeof(double) * n * d * d, cudaMemcpyHostToDevice, s->stream), "upload F");
        dx_ = sx;
        dv = v ? sv : nullptr;
        dB = B ? sB : nullptr;
        dF = F ? sF : nullptr;
    }
    s->n = n;
    s->cur = 0;
    s->keys_valid = false;
    s->phase = 0;
    s->skeys = s->perm = nullptr;
    CK(DISPATCH(s, upload, s->c, s->b, s->cur, n, dx_, dv, dB, dF, s->stream), "upload kernel");
    if (!on_device) return check_device(s);
    return APIC_OK;
}

apic_status apic_download(apic_sim* s, double* x, double* v, double* B, double* F, int on_device)
{
    if (!s) return APIC_ERR_ARG;
    CK(cudaSetDevice(s->device), "cudaSetDevice");
    const int64_t n = s->n;
    const int d = s->c.dim;
    if (n == 0) return check_device(s);
    if (on_device) {
        CK(DISPATCH(s, download, s->c, s->b, s->cur, n, x, v, B, F, nullptr, nullptr, s->stream), "download kernel");
        return check_device(s);
    }
    double* sx = s->b.staging;
    double* sv = sx + n * d;
    double* sB = sv + n * d;
    double* sF = sB + n * d * d;
    CK(DISPATCH(s, download, s->c, s->b, s->cur, n, x ? sx : nullptr, v ? sv : nullptr, B ? sB : nullptr,
                F ? sF : nullptr, nullptr, nullptr, s->stream),
       "download kernel");
    if (x) CK(cudaMemcpyAsync(x, sx, sizeof(double) * n * d, cudaMemcpyDeviceToHost, s->stream), "download x");
    if (v) CK(cudaMemcpyAsync(v, sv, sizeof(double) * n * d, cudaMemcpyDeviceToHost, s->stream), "download v");
    if (B) CK(cudaMemcpyAsync(B, sB, sizeof(double) * n * d * d, cudaMemcpyDeviceToHost, s->stream), "download B");
    if (F) CK(cudaMemcpyAsync(F, sF, sizeof(double) * n * d * d, cudaMemcpyDeviceToHost, s->stream), "download F");
    return check_device(s);
}

apic_status apic_download_positions(apic_sim* s, int32_t* cell, double* offset)
{
    if (!s || !cell || !offset) return APIC_ERR_ARG;
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
    {
        PhaseScope ps(s, APIC_PHASE_SORT, 5 * ((s->c.key_bits + 7) / 8));
        CK(radix_sort(s->b, n, s->c.key_bits, s->stream, &s->skeys, &s->perm), "radix sort");
    }
    {
        PhaseScope ps(s, APIC_PHASE_TILES, 5);
        CK(build_tiles(s->b, s->skeys, n, s->c.dim, s->c.tile, s->max_tiles, s->stream), "tile list");
    }
    {
        PhaseScope ps(s, APIC_PHASE_P2G, 1);
        CK(DISPATCH(s, p2g, s->c, s->b, s->cur, s->skeys, s->perm, n, s->L, s->stream), "p2g kernel");
    }
    s->phase = 1;
    return APIC_OK;
}

apic_status apic_grid_update(apic_sim* s)
{
    if (!s) return APIC_ERR_ARG;
    if (s->phase != 1) return fail(s, APIC_ERR_ARG, "apic_grid_update must follow apic_p2g");
    CK(cudaSetDevice(s->device), "cudaSetDevice");
    {
        PhaseScope ps(s, APIC_PHASE_GRID, 1);
        CK(DISPATCH(s, grid_update, s->c, s->b, s->L, s->stream), "grid update kernel");
    }
    s->phase = 2;
    return APIC_OK;
}

apic_status apic_g2p(apic_sim* s)
{
    if (!s) return APIC_ERR_ARG;
    if (s->phase != 2) return fail(s, APIC_ERR_ARG, "apic_g2p must follow apic_grid_update");
    CK(cudaSetDevice(s->device), "cudaSetDevice");
    if (s->n > 0) {
        {
            PhaseScope ps(s, APIC_PHASE_G2P, 1);
            CK(DISPATCH(s, g2p, s->c, s->b, s->cur, s->skeys, s->perm, s->n, s->L, s->stream), "g2p kernel");
        }
        s->cur ^= 1;
        s->keys_valid = true;
    }
    s->phase = 0;
    return APIC_OK;
}

apic_status apic_step(apic_sim* s, int nsteps)
{
    if (!s || nsteps < 0) return APIC_ERR_ARG;
    for (int i = 0; i < nsteps; ++i) {
        apic_status st = apic_p2g(s);
        if (st == APIC_OK) st = apic_grid_update(s);
        if (st == APIC_OK) st = apic_g2p(s);
        if (st != APIC_OK) return st;
    }
    return APIC_OK;
}

apic_status apic_momentum(apic_sim* s, int where, double p[3], double l[3])
{
    if (!s || !p || !l) return APIC_ERR_ARG;
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

const char* apic_last_error(apic_sim* s)
{
    if (!s) return "NULL simulation";
    return s->err.c_str();
}

}  // extern "C"
