// apic_implicit.cuh -- the implicit midpoint rule (lambda = 1/2) of Sec. 3.3 as Sec. 4.1-4.2 solve
// it (arXiv:1603.06188): after P2G of mass and momentum and v_i = (m v)_i / m_i, Newton
// iterations on the grid velocity change dv = v~ - v for
//     m_i dv_i = dt f_i(x~),   x~_i = x_i + dt (v_i / 2 + dv_i / 4)
// (the force at F^{n+1/2}, the family's F^{n+lambda}), each Newton system solved by conjugate
// gradients in the mass inner product <u, w>_M = sum_i m_i u_i . w_i (Algorithm 1) on its
// velocity-like form (I - dt^2/4 M^{-1} df/dx~) du = dt M^{-1} f - dv; then v~ = v + dv and the
// general transfer to particles with u_i = (v_i + v~_i) / 2.  The force reuses the lambda = 1
// kernel (k_force_lambda1 with the displacement velocity u); this file adds the force-derivative
// product of Sec. 3.3 and the grid vector steps of the solve.  Every grid vector keeps the node
// layout of the velocity grid (4 lanes per node, lane 3 unused or the mass); only nodes with
// mass carry unknowns.  Included by apic_transfer.cuh after apic_lambda1.cuh.
#pragma once

namespace apic {

// 3x3 inverse through the cofactors (the caller keeps det away from zero)
template <typename R> __device__ __forceinline__ void inverse3(const R* M, R* Mi)
{
    R C[9];
    C[0] = M[4] * M[8] - M[5] * M[7];
    C[1] = M[5] * M[6] - M[3] * M[8];
    C[2] = M[3] * M[7] - M[4] * M[6];
    C[3] = M[2] * M[7] - M[1] * M[8];
    C[4] = M[0] * M[8] - M[2] * M[6];
    C[5] = M[1] * M[6] - M[0] * M[7];
    C[6] = M[1] * M[5] - M[2] * M[4];
    C[7] = M[2] * M[3] - M[0] * M[5];
    C[8] = M[0] * M[4] - M[1] * M[3];
    const R inv = R(1) / (M[0] * C[0] + M[1] * C[1] + M[2] * C[2]);
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) Mi[a * 3 + b] = C[b * 3 + a] * inv;
}

// dP = dP/dF (F) : dF of the models of stress_first_pk.
// Neo-Hookean: dP = mu dF + (mu - lam log J) F^-T dF^T F^-T + lam (F^-T : dF) F^-T.
// Fixed-corotated: dP = 2 mu (dF - dR) + lam (cof(F) : dF) cof(F) + lam (J - 1) d cof(F), with
// d cof(F) = (cof(F) : dF) F^-T - J F^-T dF^T F^-T and the rotation's variation dR = R W, W skew,
// from F = R S: W S + S W = R^T dF - dF^T R (in 3-D W = [w]x with (tr(S) I - S) w = k, k the axial
// vector of the right side; in 2-D W has the angle k / tr(S)).
template <int D, typename R>
__device__ __forceinline__ void stress_diff(int model, const R* F, const R* dF, R mu, R lam, R* dP, unsigned* fallbacks)
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
    // FiT = F^-T = C / J;  T = F^-T dF^T F^-T;  cdf = C : dF
    R FiT[D * D], T[D * D];
    R cdf = R(0);
#pragma unroll
    for (int i = 0; i < D * D; ++i) {
        FiT[i] = C[i] / J;
        cdf += C[i] * dF[i];
    }
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) {
            R s = R(0);
#pragma unroll
            for (int k = 0; k < D; ++k)
#pragma unroll
                for (int l = 0; l < D; ++l) s += FiT[a * D + k] * dF[l * D + k] * FiT[l * D + b];
            T[a * D + b] = s;
        }
    if (model == 2) {
        const R tr = cdf / J;
        const R cT = mu - lam * log(J);
#pragma unroll
        for (int i = 0; i < D * D; ++i) dP[i] = mu * dF[i] + cT * T[i] + lam * tr * FiT[i];
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
    // S = R^T F, K = R^T dF - dF^T R
    R S[D * D], K[D * D];
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) {
            R s = R(0), k = R(0);
#pragma unroll
            for (int m = 0; m < D; ++m) {
                s += Rot[m * D + a] * F[m * D + b];
                k += Rot[m * D + a] * dF[m * D + b] - dF[m * D + a] * Rot[m * D + b];
            }
            S[a * D + b] = s;
            K[a * D + b] = k;
        }
    R W[D * D];
    if (D == 3) {
        const R kv[3] = {K[7], K[2], K[3]};   // axial vector of K: (K21, K02, K10)
        const R tr = S[0] + S[4] + S[8];
        R M[9], Mi[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) M[i] = -S[i];
        M[0] += tr;
        M[4] += tr;
        M[8] += tr;
        inverse3<R>(M, Mi);
        R w[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) w[a] = Mi[a * 3 + 0] * kv[0] + Mi[a * 3 + 1] * kv[1] + Mi[a * 3 + 2] * kv[2];
        W[0] = R(0);  W[1] = -w[2]; W[2] = w[1];
        W[3] = w[2];  W[4] = R(0);  W[5] = -w[0];
        W[6] = -w[1]; W[7] = w[0];  W[8] = R(0);
    } else {
        const R t = K[2] / (S[0] + S[3]);
        W[0] = R(0); W[1] = -t; W[2] = t; W[3] = R(0);
    }
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) {
            R dR = R(0);
#pragma unroll
            for (int m = 0; m < D; ++m) dR += Rot[a * D + m] * W[m * D + b];
            const int i = a * D + b;
            const R dcof = cdf * FiT[i] - J * T[i];
            dP[i] = R(2) * mu * (dF[i] - dR) + lam * cdf * C[i] + lam * (J - R(1)) * dcof;
        }
}

// The force-derivative product of Sec. 3.3 at the displaced grid x~ = x + dt u:
//   df_i = sum_j (d f_i / d x~_j) p_j = -sum_p V_p A_p (F_p^n)^T grad w_ip,
//   A_p = dP/dF(F^_p) : ((sum_j p_j (grad w_jp)^T) F_p^n),  F^_p = (I + dt sum_j u_j grad w_jp^T) F_p^n,
// added (times `scale`) into the accumulation grid; tiles and shared-memory node tile as in
// k_force_lambda1.
template <int D, int ORDER, typename R>
__global__ void __launch_bounds__(128) k_force_diff(PState<R> st, const uint32_t* __restrict__ perm,
                                                    const uint32_t* __restrict__ skeys,
                                                    const uint32_t* __restrict__ tiles,
                                                    const uint32_t* __restrict__ ntiles_p, uint32_t* __restrict__ ctr,
                                                    const R* __restrict__ ugrid, const R* __restrict__ pgrid,
                                                    R* __restrict__ acc, R scale, DevCfg<R> c, uint32_t* err,
                                                    uint32_t* fallbacks)
{
    constexpr int K = ORDER + 1;
    constexpr int TE = 4 + ORDER;
    constexpr int TN = (D == 3) ? TE * TE * TE : TE * TE;
    constexpr int NS = (D == 3) ? K * K * K : K * K;
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
        for (uint32_t k = start + threadIdx.x; k < end; k += 128) {
            Particle<D, R> p;
            const uint32_t q = perm[k];
            load_xF<D, R>(st, q, p);
            if (c.mat) load_mat<D, R>(st, q, p);
            int base[D], lb[3] = {0, 0, 0};
            R w[D][K], dw[D][K], fx[D];
            bool ok = particle_stencil<D, ORDER, R>(p.o, p.cell, c, base, fx, w, dw);
#pragma unroll
            for (int a = 0; a < D; ++a) {
                lb[a] = base[a] - bo[a];
                if (lb[a] < 0 || lb[a] > 3) ok = false;
            }
            if (!ok) {
                set_err(err, APIC_ERRBIT_RANGE);
                continue;
            }
            // grad u and grad p in grid units
            R Gu[D * D], Gp[D * D];
#pragma unroll
            for (int i = 0; i < D * D; ++i) { Gu[i] = R(0); Gp[i] = R(0); }
#pragma unroll 1
            for (int j = 0; j < NS; ++j) {
                const int ia = j % K, ib = (j / K) % K, ic = (D == 3) ? j / (K * K) : 0;
                const int g[3] = {base[0] + ia, base[1] + ib, (D == 3) ? base[D - 1] + ic : 0};
                const uint32_t ni = node_index<D>(g, c.nb);
                const V4<R> uu = ld4(reinterpret_cast<const V4<R>*>(ugrid) + ni);
                const V4<R> pp = ld4(reinterpret_cast<const V4<R>*>(pgrid) + ni);
                const R ui[3] = {uu.x, uu.y, uu.z}, pi[3] = {pp.x, pp.y, pp.z};
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
                    for (int b2 = 0; b2 < D; ++b2) {
                        Gu[a * D + b2] += ui[a] * gw[b2];
                        Gp[a * D + b2] += pi[a] * gw[b2];
                    }
            }
            // F^ = (I + dt grad u) F^n, dF = (grad p) F^n (world units: grad w = grad^ w / dx)
            R Fh[D * D], dF[D * D], dP[D * D], A[D * D];
#pragma unroll
            for (int a = 0; a < D; ++a)
#pragma unroll
                for (int b2 = 0; b2 < D; ++b2) {
                    R s = p.F[a * D + b2], sd = R(0);
#pragma unroll
                    for (int kk = 0; kk < D; ++kk) {
                        s += dt_dx * Gu[a * D + kk] * p.F[kk * D + b2];
                        sd += c.inv_dx * Gp[a * D + kk] * p.F[kk * D + b2];
                    }
                    Fh[a * D + b2] = s;
                    dF[a * D + b2] = sd;
                }
            stress_diff<D, R>(c.model, Fh, dF, c.mat ? p.mu : c.mu, c.mat ? p.lam : c.lam, dP, fallbacks);
#pragma unroll
            for (int a = 0; a < D; ++a)
#pragma unroll
                for (int b2 = 0; b2 < D; ++b2) {
                    R s = R(0);
#pragma unroll
                    for (int kk = 0; kk < D; ++kk) s += dP[a * D + kk] * p.F[b2 * D + kk];
                    A[a * D + b2] = (c.mat ? p.pv : c.vol) * s;
                }
            // scale * (-A grad w), grad w = grad^ w / dx
            const R sc = -scale * c.inv_dx;
#pragma unroll 1
            for (int j = 0; j < NS; ++j) {
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
                    atomicAdd(&sf[a][li], sc * s);
                }
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < TN; i += 128) {
            bool any = false;
#pragma unroll
            for (int a = 0; a < D; ++a) any |= sf[a][i] != R(0);
            if (!any) continue;
            const int g[3] = {bo[0] + i % TE, bo[1] + (i / TE) % TE, (D == 3) ? bo[2] + i / (TE * TE) : 0};
            R* dst = acc + 4 * (size_t)node_index<D>(g, c.nb);
#pragma unroll
            for (int a = 0; a < D; ++a) atomicAdd(dst + a, sf[a][i]);
        }
        __syncthreads();
    }
}

// The grid vector steps of the solve, one kernel per step, each over the nodes of the active
// blocks (the mass is lane 3 of vel1, the grid velocity v_i before the solve).  Where a step
// takes a mass inner product its per-CTA FP64 partial goes to part[blockIdx.x].
//   op 0  u  = v / 2 + dv / 4                                   (displacement velocity)
//   op 1  r  = acc / m - dv,  p = r,  du = 0,  acc = 0;  <r, r>   (acc holds dt f)
//   op 2  s  = p - (dt^2 / 4) acc / m,  acc = 0;  <p, s>          (acc holds df/dx~ p)
//   op 3  du += a p,  r -= a s;  <r, r>
//   op 4  p  = r + a p
//   op 5  dv += du
//   op 6  v~ = v + dv into vel (with the mass), u = (v + v~) / 2
//   op 7  <v, v>_M (acc = vel1 here)
struct SolveVecs {
    void* vel1; void* dv; void* u; void* r; void* p; void* s; void* du; void* acc; void* vel;
};

template <int D, typename R>
__global__ void __launch_bounds__(TPB) k_solve_step(SolveVecs sv, uint32_t* __restrict__ flags, DevCfg<R> c, int op,
                                                    double a, double* __restrict__ part)
{
    constexpr int BN = (D == 3) ? 64 : 16;
    const R* v1 = (const R*)sv.vel1;
    R* dv = (R*)sv.dv;
    R* u = (R*)sv.u;
    R* r = (R*)sv.r;
    R* p = (R*)sv.p;
    R* s = (R*)sv.s;
    R* du = (R*)sv.du;
    R* acc = (R*)sv.acc;
    R* vel = (R*)sv.vel;
    const R dt = step_dt(c);
    const R ar = (R)a;
    double dot = 0.0;
    const int64_t total = (int64_t)c.nblocks * BN;
    for (int64_t node = (int64_t)blockIdx.x * TPB + threadIdx.x; node < total; node += (int64_t)gridDim.x * TPB) {
        const int b = (int)(node / BN);
        if (flags[b] == 0u) continue;
        const size_t o = 4 * (size_t)node;
        const R m = v1[o + 3];
        const bool live = m > R(0);
        for (int d = 0; d < D; ++d) {
            const size_t i = o + d;
            switch (op) {
            case 0: u[i] = live ? R(0.5) * v1[i] + R(0.25) * dv[i] : R(0); break;
            case 1: {
                const R ri = live ? acc[i] / m - dv[i] : R(0);
                r[i] = ri;
                p[i] = ri;
                du[i] = R(0);
                acc[i] = R(0);
                dot += (double)m * (double)ri * (double)ri;
                break;
            }
            case 2: {
                const R si = live ? p[i] - R(0.25) * dt * dt * acc[i] / m : R(0);
                s[i] = si;
                acc[i] = R(0);
                dot += (double)m * (double)p[i] * (double)si;
                break;
            }
            case 3: {
                du[i] += ar * p[i];
                const R ri = r[i] - ar * s[i];
                r[i] = ri;
                dot += (double)m * (double)ri * (double)ri;
                break;
            }
            case 4: p[i] = r[i] + ar * p[i]; break;
            case 5: dv[i] += du[i]; break;
            case 6: {
                const R vt = live ? v1[i] + dv[i] : R(0);
                vel[i] = vt;
                u[i] = live ? R(0.5) * (v1[i] + vt) : R(0);
                break;
            }
            case 7: dot += (double)m * (double)v1[i] * (double)v1[i]; break;
            default: break;
            }
        }
        if (op == 6) {
            vel[o + 3] = m;
            if (D == 2) vel[o + 2] = R(0);
        }
    }
    if (op == 6) return;
    // per-CTA FP64 partial in a fixed order
    __shared__ double sp[TPB / 32];
    for (int off = 16; off > 0; off >>= 1) dot += __shfl_down_sync(FULLMASK, dot, off);
    if ((threadIdx.x & 31) == 0) sp[threadIdx.x >> 5] = dot;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < TPB / 32; ++w) t += sp[w];
        part[blockIdx.x] = t;
    }
}

// flags cleared after the solve (the next P2G sets them again); one instance per real type
template <typename R> __global__ void __launch_bounds__(TPB) k_clear_flags(uint32_t* flags, int nblocks)
{
    for (int b = blockIdx.x * TPB + threadIdx.x; b < nblocks; b += gridDim.x * TPB) flags[b] = 0u;
}

// sum of np FP64 partials into out[0] (fixed order); one instance per real type
template <typename R>
__global__ void __launch_bounds__(TPB) k_sum_partials(const double* __restrict__ part, int np, double* __restrict__ out)
{
    __shared__ double s[TPB];
    double t = 0.0;
    for (int i = threadIdx.x; i < np; i += TPB) t += part[i];
    s[threadIdx.x] = t;
    __syncthreads();
    for (int st = TPB / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) s[threadIdx.x] += s[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = s[0];
}

}  // namespace apic
