// apic_lambda1.cuh -- the explicit member lambda = 1 of the integrator family of Sec. 3.3
// (arXiv:1603.06188).  The step differs from the lambda = 0 one in where the force is taken
// and how the particles move:
//   P2G of mass and momentum alone (Sec. 3.2), v_i = (m v)_i / m_i          k_grid_velocity
//   x~_i = x_i + dt v_i, so F_p^{n+1} = (I + dt sum_i v_i (grad w_ip)^T) F_p^n,
//   f_i = -sum_p V_p P(F_p^{n+1}) (F_p^n)^T grad w_ip                        k_force_lambda1
//   v~_i = v_i + dt f_i / m_i (+ dt g, walls)                                 k_grid_update_lambda1
//   the general transfer to particles of Sec. 3.4 at lambda = 1               k_g2p_general
// The velocity grid before the update (v_i) lives in its own array (vel1), the updated one
// (v~_i) in the usual velocity grid, so G2P gathers both.  The force matrix
// A_p = V_p P(F^{n+1}) (F^n)^T is not symmetric; it is formed and scattered in the same
// kernel, tile by tile, so it is never stored.  Included by apic_transfer.cuh.
#pragma once

namespace apic {

// first Piola-Kirchhoff stress P(F) of the model: fixed-corotated
// P = 2 mu (F - R) + lam (J - 1) cof(F), Neo-Hookean P = mu (F - cof(F) / J) + lam log(J) cof(F) / J,
// with cof(F) = J F^{-T}; R from the same polar routes as the symmetric stress of lambda = 0
template <int D, typename R>
__device__ __forceinline__ void stress_first_pk(int model, const R* F, R mu, R lam, R* P, unsigned* fallbacks)
{
    R C[D * D];
    R J;
    if (D == 3) {
        C[0] = F[4] * F[8] - F[5] * F[7];
        C[1] = F[5] * F[6] - F[3] * F[8];
        C[2] = F[3] * F[7] - F[4] * F[6];
        C[3] = F[2] * F[7] - F[1] * F[8];
        C[4] = F[0] * F[8] - F[2] * F[6];
        C[5] = F[1] * F[6] - F[0] * F[7];
        C[6] = F[1] * F[5] - F[2] * F[4];
        C[7] = F[2] * F[3] - F[0] * F[5];
        C[8] = F[0] * F[4] - F[1] * F[3];
        J = F[0] * C[0] + F[1] * C[1] + F[2] * C[2];
    } else {
        C[0] = F[3];
        C[1] = -F[2];
        C[2] = -F[1];
        C[3] = F[0];
        J = F[0] * F[3] - F[1] * F[2];
    }
    if (model == 2) {
        const R inv = R(1) / J, lg = lam * log(J) * inv;
#pragma unroll
        for (int i = 0; i < D * D; ++i) P[i] = mu * (F[i] - C[i] * inv) + lg * C[i];
        return;
    }
    R Rot[D * D];
    if (D == 2) {
        const R a = F[0] + F[3], b = F[2] - F[1];
        const R r2 = a * a + b * b;
        R c = R(1), s = R(0);
        if (r2 > R(0)) {
            const R inv = rsqrt_t<R>(r2);
            c = a * inv;
            s = b * inv;
        }
        Rot[0] = c; Rot[1] = -s; Rot[2] = s; Rot[3] = c;
    } else if (!polar_newton3<R>(F, Rot)) {
        R gap = R(1);
        polar3<R>(F, Rot, &gap);
        if (sizeof(R) == 4 && (polar_residual<R>(F, Rot) > R(2e-5) || inverted_unresolved<R>(F, gap))) {
            double Fd[9], Rd[9];
            for (int i = 0; i < 9; ++i) Fd[i] = (double)F[i];
            polar3<double>(Fd, Rd);
            for (int i = 0; i < 9; ++i) Rot[i] = (R)Rd[i];
            if (fallbacks) atomicAdd(fallbacks, 1u);
        }
    }
    const R iso = lam * (J - R(1));
#pragma unroll
    for (int i = 0; i < D * D; ++i) P[i] = R(2) * mu * (F[i] - Rot[i]) + iso * C[i];
}

// velocity v~ of grid node g after the boundary rule (not in the paper): sticky walls zero the
// whole velocity, slip walls its component normal to each wall the node is in
template <int D, typename R> __device__ __forceinline__ void apply_walls(const int* g, const DevCfg<R>& c, R* v)
{
    if (c.boundary == 1) {
        bool wall = false;
#pragma unroll
        for (int d = 0; d < D; ++d)
            if (g[d] < c.wall || g[d] >= c.res[d] - c.wall) wall = true;
        if (wall) v[0] = v[1] = v[2] = R(0);
    } else if (c.boundary == 2) {
#pragma unroll
        for (int d = 0; d < D; ++d)
            if (g[d] < c.wall || g[d] >= c.res[d] - c.wall) v[d] = R(0);
    }
}

// v_i = (m v)_i / m_i into vel1 (v, m), for every node of an active block; the accumulation
// grid is cleared for the force and the flags are kept.  One warp per block.
template <int D, typename R>
__global__ void __launch_bounds__(TPB) k_grid_velocity(R* __restrict__ acc, R* __restrict__ vel1,
                                                       const uint32_t* __restrict__ flags, DevCfg<R> c)
{
    constexpr int BN = (D == 3) ? 64 : 16;
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * TPB + threadIdx.x) >> 5;
    const int nw = (gridDim.x * TPB) >> 5;
    for (int b = gw; b < c.nblocks; b += nw) {
        if (flags[b] == 0u) continue;
        for (int i = lane; i < BN; i += 32) {
            const size_t node = (size_t)b * BN + i;
            const V4<R> a = *reinterpret_cast<const V4<R>*>(acc + 4 * node);
            V4<R> o = {R(0), R(0), R(0), a.w};
            if (a.w > R(0)) {
                const R inv = R(1) / a.w;
                o.x = a.x * inv;
                o.y = a.y * inv;
                o.z = a.z * inv;
            }
            *reinterpret_cast<V4<R>*>(vel1 + 4 * node) = o;
            *reinterpret_cast<V4<R>*>(acc + 4 * node) = V4<R>{R(0), R(0), R(0), R(0)};
        }
    }
}

// The force of Sec. 3.3 at a displaced grid x~_i = x_i + dt u_i, tile by tile (a tile = sorted
// particles of one node block): each particle gathers grad u = sum_i u_i (grad w_ip)^T from
// ugrid, forms F^ = (I + dt grad u) F^n, P(F^) and A = V_p P(F^) (F^n)^T, and adds
// -dt A grad w_ip into a shared-memory tile of the (4 + ORDER)^D nodes its block's particles
// reach; the tile is added to the accumulation grid once.  u = v_i gives the member
// lambda = 1 (F^ = F^{n+1}); u = v_i / 2 + dv_i / 4 the implicit midpoint rule's force at
// F^{n+1/2}.  Persistent CTAs take tiles from ctr.
template <int D, int ORDER, typename R>
__global__ void __launch_bounds__(128) k_force_lambda1(PState<R> st, const uint32_t* __restrict__ perm,
                                                       const uint32_t* __restrict__ skeys,
                                                       const uint32_t* __restrict__ tiles,
                                                       const uint32_t* __restrict__ ntiles_p, uint32_t* __restrict__ ctr,
                                                       const R* __restrict__ ugrid, R* __restrict__ acc, DevCfg<R> c,
                                                       uint32_t* err, uint32_t* fallbacks)
{
    constexpr int K = ORDER + 1;
    constexpr int TE = 4 + ORDER;
    constexpr int TN = (D == 3) ? TE * TE * TE : TE * TE;
    __shared__ R sf[D][TN];
    __shared__ int s_tile;
    const int ntiles = (int)*ntiles_p;
    const R dt_dx = step_dt(c) * c.inv_dx;
    for (;;) {
        if (threadIdx.x == 0) s_tile = (int)atomicAdd(ctr, 1u);
        for (int i = threadIdx.x; i < D * TN; i += 128) (&sf[0][0])[i] = R(0);
        __syncthreads();
        const int t = s_tile;
        if (t >= ntiles) break;
        const uint32_t start = tiles[t], end = tiles[t + 1];
        const uint32_t blk = skeys[start] >> (2 * D);
        int bo[3] = {0, 0, 0};
        block_coords<D, R>(blk, c, bo);
#pragma unroll
        for (int a = 0; a < D; ++a) bo[a] *= 4;
        // warp-uniform rounds: a lane past the tile's end takes the tile's first particle and
        // adds nothing, so that every lane takes part in the warp's shuffles below
        for (uint32_t k0 = start; k0 < end; k0 += 128) {
            const uint32_t k = k0 + threadIdx.x;
            const bool live = k < end;
            Particle<D, R> p;
            const uint32_t q = perm[live ? k : start];
            load_xF<D, R>(st, q, p);
            if (c.mat) load_mat<D, R>(st, q, p);
            int base[D], lb[3] = {0, 0, 0};
            R w[D][K], dw[D][K], fx[D];
            bool ok = particle_stencil<D, ORDER, R>(p.o, p.cell, c, base, fx, w, dw);
#pragma unroll
            for (int a = 0; a < D; ++a) {
                lb[a] = base[a] - bo[a];
                if (lb[a] < 0 || lb[a] > 3) {
                    ok = false;
                    lb[a] = 0;
                }
            }
            if (live && !ok) set_err(err, APIC_ERRBIT_RANGE);
            const bool add = live && ok;
            // grad v in grid units: G_ab = sum_i v_ia (d w / d x^_b)
            R G[D * D];
#pragma unroll
            for (int i = 0; i < D * D; ++i) G[i] = R(0);
#pragma unroll
            for (int j = 0; j < ((D == 3) ? K * K * K : K * K); ++j) {
                const int ia = j % K, ib = (j / K) % K, ic = (D == 3) ? j / (K * K) : 0;
                const int g[3] = {base[0] + ia, base[1] + ib, (D == 3) ? base[D - 1] + ic : 0};
                const V4<R> vv = ld4(reinterpret_cast<const V4<R>*>(ugrid) + node_index<D>(g, c.nb));
                const R vi[3] = {vv.x, vv.y, vv.z};
                R gw[3];
                if (D == 3) {
                    gw[0] = dw[0][ia] * w[1][ib] * w[D - 1][ic];
                    gw[1] = w[0][ia] * dw[1][ib] * w[D - 1][ic];
                    gw[2] = w[0][ia] * w[1][ib] * dw[D - 1][ic];
                } else {
                    gw[0] = dw[0][ia] * w[1][ib];
                    gw[1] = w[0][ia] * dw[1][ib];
                }
#pragma unroll
                for (int a = 0; a < D; ++a)
#pragma unroll
                    for (int b2 = 0; b2 < D; ++b2) G[a * D + b2] += vi[a] * gw[b2];
            }
            // F^ = (I + dt grad v) F^n and A = V P(F^) (F^n)^T
            R Fh[D * D], P[D * D], A[D * D];
#pragma unroll
            for (int a = 0; a < D; ++a)
#pragma unroll
                for (int b2 = 0; b2 < D; ++b2) {
                    R s = p.F[a * D + b2];
#pragma unroll
                    for (int kk = 0; kk < D; ++kk) s += dt_dx * G[a * D + kk] * p.F[kk * D + b2];
                    Fh[a * D + b2] = s;
                }
            stress_first_pk<D, R>(c.model, Fh, c.mat ? p.mu : c.mu, c.mat ? p.lam : c.lam, P, fallbacks);
#pragma unroll
            for (int a = 0; a < D; ++a)
#pragma unroll
                for (int b2 = 0; b2 < D; ++b2) {
                    R s = R(0);
#pragma unroll
                    for (int kk = 0; kk < D; ++kk) s += P[a * D + kk] * p.F[b2 * D + kk];
                    A[a * D + b2] = add ? (c.mat ? p.pv : c.vol) * s : R(0);
                }
            // dt f_i = -dt A grad w / dx into the tile.  The warp's particles are consecutive in
            // the sorted order, so lanes with the same base cell form runs of lanes: each value is
            // summed over its run (a segmented suffix sum by shuffles) and the run's first lane
            // adds it, one shared-memory add per run instead of one per particle.  Every shuffle
            // is executed by all 32 lanes (none sits behind a lane-dependent condition).
            const int ck = add ? (lb[0] | (lb[1] << 2) | (lb[2] << 4)) : -1;
            const int lane = threadIdx.x & 31;
            bool same[5];
#pragma unroll
            for (int s5 = 0; s5 < 5; ++s5) {
                const int cn = __shfl_down_sync(FULLMASK, ck, 1 << s5);
                same[s5] = lane + (1 << s5) < 32 && cn == ck;
            }
            const int cprev = __shfl_up_sync(FULLMASK, ck, 1);
            const bool head = add && (lane == 0 || cprev != ck);
#pragma unroll
            for (int j = 0; j < ((D == 3) ? K * K * K : K * K); ++j) {
                const int ia = j % K, ib = (j / K) % K, ic = (D == 3) ? j / (K * K) : 0;
                R gw[3];
                if (D == 3) {
                    gw[0] = dw[0][ia] * w[1][ib] * w[D - 1][ic];
                    gw[1] = w[0][ia] * dw[1][ib] * w[D - 1][ic];
                    gw[2] = w[0][ia] * w[1][ib] * dw[D - 1][ic];
                } else {
                    gw[0] = dw[0][ia] * w[1][ib];
                    gw[1] = w[0][ia] * dw[1][ib];
                }
                const int li = (lb[0] + ia) + TE * ((lb[1] + ib) + ((D == 3) ? TE * (lb[2] + ic) : 0));
#pragma unroll
                for (int a = 0; a < D; ++a) {
                    R s = R(0);
#pragma unroll
                    for (int b2 = 0; b2 < D; ++b2) s += A[a * D + b2] * gw[b2];
                    s *= -dt_dx;
#pragma unroll
                    for (int s5 = 0; s5 < 5; ++s5) {
                        const R u = __shfl_down_sync(FULLMASK, s, 1 << s5);
                        if (same[s5]) s += u;
                    }
                    if (head) atomicAdd(&sf[a][li], s);
                }
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < TN; i += 128) {
            bool any = false;
#pragma unroll
            for (int a = 0; a < D; ++a) any |= sf[a][i] != R(0);
            if (!any) continue;   // only nodes some particle reached, all inside the grid
            const int g[3] = {bo[0] + i % TE, bo[1] + (i / TE) % TE, (D == 3) ? bo[2] + i / (TE * TE) : 0};
            R* dst = acc + 4 * (size_t)node_index<D>(g, c.nb);
#pragma unroll
            for (int a = 0; a < D; ++a) atomicAdd(dst + a, sf[a][i]);
        }
        __syncthreads();
    }
}

// v~_i = v_i + (dt f_i) / m_i + dt g, then the walls, into the velocity grid (v~, m); clears
// the accumulation grid and the block flags.  One warp per block.
template <int D, typename R>
__global__ void __launch_bounds__(TPB) k_grid_update_lambda1(R* __restrict__ acc, R* __restrict__ vel,
                                                             const R* __restrict__ vel1, uint32_t* __restrict__ flags,
                                                             DevCfg<R> c)
{
    constexpr int BN = (D == 3) ? 64 : 16;
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * TPB + threadIdx.x) >> 5;
    const int nw = (gridDim.x * TPB) >> 5;
    const R dt = step_dt(c);
    for (int b = gw; b < c.nblocks; b += nw) {
        if (flags[b] == 0u) continue;
        int bc[3] = {0, 0, 0};
        block_coords<D, R>((uint32_t)b, c, bc);
        for (int i = lane; i < BN; i += 32) {
            const size_t node = (size_t)b * BN + i;
            const V4<R> f = *reinterpret_cast<const V4<R>*>(acc + 4 * node);
            const V4<R> v1 = *reinterpret_cast<const V4<R>*>(vel1 + 4 * node);
            const R m = v1.w;
            R v[3] = {R(0), R(0), R(0)};
            if (m > R(0)) {
                const R inv = R(1) / m;
                v[0] = v1.x + f.x * inv + dt * c.gravity[0];
                v[1] = v1.y + f.y * inv + dt * c.gravity[1];
                if (D == 3) v[2] = v1.z + f.z * inv + dt * c.gravity[2];
                const int g[3] = {bc[0] * 4 + (i & 3), bc[1] * 4 + ((i >> 2) & 3), (D == 3) ? bc[2] * 4 + (i >> 4) : 0};
                apply_walls<D, R>(g, c, v);
            }
            *reinterpret_cast<V4<R>*>(vel + 4 * node) = V4<R>{v[0], v[1], v[2], m};
            *reinterpret_cast<V4<R>*>(acc + 4 * node) = V4<R>{R(0), R(0), R(0), R(0)};
        }
        __syncwarp();
        if (lane == 0) flags[b] = 0u;
    }
}

// The general transfer to particles of Sec. 3.4, with the nodes moved to x~_i = x_i + dt u_i,
// u_i = lambda v_i + (1 - lambda) v~_i (ugrid: v_i for lambda = 1, (v_i + v~_i) / 2 for the
// midpoint rule):
//   v_p = sum_i w v~_i,  x_p^{n+1} = sum_i w x~_i = x_p + dt ubar_p,  ubar_p = sum_i w u_i,
//   F_p^{n+1} = (I + dt sum_i u_i (grad w)^T) F_p^n,
//   B_p = 1/2 sum_i w (v~_i (x_i - x_p + x~_i - x_p^{n+1})^T + (x_i - x_p - x~_i + x_p^{n+1}) v~_i^T)
//       = sum_i w v~_i (x_i - x_p)^T + dt/2 (sum_i w (v~_i u_i^T - u_i v~_i^T) - (v_p ubar_p^T - ubar_p v_p^T))
// (the last line is the same sum with x~_i - x_p^{n+1} = x_i - x_p + dt (u_i - ubar_p) put in),
// B_p = 0 for PIC.  Particle k of the sorted order is read through the permutation and written
// at k, with its next cell key.
template <int D, int ORDER, typename R>
__global__ void __launch_bounds__(128) k_g2p_general(PState<R> in, PState<R> out, const uint32_t* __restrict__ perm,
                                                     const R* __restrict__ vel, const R* __restrict__ ugrid,
                                                     uint32_t* __restrict__ knext, DevCfg<R> c, uint32_t* err)
{
    constexpr int K = ORDER + 1;
    const R dt = step_dt(c);
    const R dt_dx = dt * c.inv_dx;
    for (int k = blockIdx.x * 128 + threadIdx.x; k < c.n; k += gridDim.x * 128) {
        Particle<D, R> p;
        const uint32_t q = perm[k];
        load_xF<D, R>(in, q, p);
        if (c.mat) load_mat<D, R>(in, q, p);
        int base[D];
        R w[D][K], dw[D][K], fx[D];
        if (!particle_stencil<D, ORDER, R>(p.o, p.cell, c, base, fx, w, dw)) set_err(err, APIC_ERRBIT_RANGE);
        R vn[3] = {R(0), R(0), R(0)}, vb[3] = {R(0), R(0), R(0)};
        R Bh[D * D], Kx[D * D], G[D * D];
#pragma unroll
        for (int i = 0; i < D * D; ++i) { Bh[i] = R(0); Kx[i] = R(0); G[i] = R(0); }
#pragma unroll
        for (int j = 0; j < ((D == 3) ? K * K * K : K * K); ++j) {
            const int ia = j % K, ib = (j / K) % K, ic = (D == 3) ? j / (K * K) : 0;
            const int g[3] = {base[0] + ia, base[1] + ib, (D == 3) ? base[D - 1] + ic : 0};
            const uint32_t ni = node_index<D>(g, c.nb);
            const V4<R> t4 = ld4(reinterpret_cast<const V4<R>*>(vel) + ni);
            const V4<R> v4 = ld4(reinterpret_cast<const V4<R>*>(ugrid) + ni);
            const R vt[3] = {t4.x, t4.y, t4.z}, v1[3] = {v4.x, v4.y, v4.z};
            const R wt = (D == 3) ? w[0][ia] * w[1][ib] * w[D - 1][ic] : w[0][ia] * w[1][ib];
            R gw[3], rh[3];
            if (D == 3) {
                gw[0] = dw[0][ia] * w[1][ib] * w[D - 1][ic];
                gw[1] = w[0][ia] * dw[1][ib] * w[D - 1][ic];
                gw[2] = w[0][ia] * w[1][ib] * dw[D - 1][ic];
            } else {
                gw[0] = dw[0][ia] * w[1][ib];
                gw[1] = w[0][ia] * dw[1][ib];
            }
            rh[0] = R(ia) - fx[0];
            rh[1] = R(ib) - fx[1];
            rh[2] = (D == 3) ? R(ic) - fx[D - 1] : R(0);
#pragma unroll
            for (int a = 0; a < D; ++a) {
                vn[a] += wt * vt[a];
                vb[a] += wt * v1[a];
#pragma unroll
                for (int b2 = 0; b2 < D; ++b2) {
                    Bh[a * D + b2] += wt * vt[a] * rh[b2];
                    Kx[a * D + b2] += wt * (vt[a] * v1[b2] - v1[a] * vt[b2]);
                    G[a * D + b2] += v1[a] * gw[b2];
                }
            }
        }
        // F <- (I + dt grad u) F with the displacement velocities
        R Fn[D * D];
#pragma unroll
        for (int a = 0; a < D; ++a)
#pragma unroll
            for (int b2 = 0; b2 < D; ++b2) {
                R s = p.F[a * D + b2];
#pragma unroll
                for (int kk = 0; kk < D; ++kk) s += dt_dx * G[a * D + kk] * p.F[kk * D + b2];
                Fn[a * D + b2] = s;
            }
#pragma unroll
        for (int a = 0; a < D; ++a)
#pragma unroll
            for (int b2 = 0; b2 < D; ++b2) {
                const int i = a * D + b2;
                p.F[i] = Fn[i];
                p.B[i] = (c.transfer == 0)
                             ? c.dx * Bh[i] + R(0.5) * dt * (Kx[i] - (vn[a] * vb[b2] - vb[a] * vn[b2]))
                             : R(0);
            }
#pragma unroll
        for (int a = 0; a < D; ++a) {
            p.v[a] = vn[a];
            R o = p.o[a] + dt_dx * vb[a];
            const R fl = floor(o);
            o -= fl;
            int cl = p.cell[a] + (int)fl;
            if (o >= R(1)) { o -= R(1); cl += 1; }
            if (cl < 0) { cl = 0; o = R(0); set_err(err, APIC_ERRBIT_RANGE); }
            if (cl > c.res[a] - 1) { cl = c.res[a] - 1; o = R(0); set_err(err, APIC_ERRBIT_RANGE); }
            p.o[a] = o;
            p.cell[a] = cl;
        }
        store_all<D, R>(out, k, p, false, c.mat != 0);
        knext[k] = key_of<D, ORDER, R>(p.o, p.cell, c, err);
    }
}

}  // namespace apic
