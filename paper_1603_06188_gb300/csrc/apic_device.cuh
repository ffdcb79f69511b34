// apic_device.cuh -- device-side building blocks of the APIC / explicit MPM step
// (arXiv:1603.06188): state layout, B-spline weights (Sec. 3.5), 3x3 polar decomposition
// for the fixed-corotated stress, and small helpers.  Included by the kernel files only.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "apic_internal.h"

namespace apic {

// ---------------------------------------------------------------- packed state lanes
// Particle state is a structure of arrays of 16-byte (FP32) / 32-byte (FP64) groups so
// each group moves with one 128-bit load or store (two for FP64):
//   3-D: A  = (o0, o1, o2, cell)   V  = (v0, v1, v2, B00)
//        Ba = (B01, B02, B10, B11) Bb = (B12, B20, B21, B22)
//        Fa = (F00, F01, F02, F10) Fb = (F11, F12, F20, F21)   Fc = (F22, id)
//        Ta = (t00, t11, t22, t01) Tb = (t02, t12)
//   2-D: A  = (o0, o1, cell, id)   V  = (v0, v1, B00, B01)
//        Ba = (B10, B11, t00, t11) Fa = (F00, F01, F10, F11)   Tb = (t01, -)
//   both: M = (mu, lam), the particle's Lame parameters, kept only once a material per
//        particle is set (otherwise the configuration's mu, lam hold for every particle)
// o = offset in [0,1) inside integer cell `cell` (packed per axis), id = upload index,
// t = the symmetric stress tau_p = V_p P(F_p) F_p^T of the current F_p (Sec. 3.3 force).
// tau is written wherever F_p is (upload, G2P), so P2G reads position, v, B and tau --
// never F -- and the polar decomposition runs once per particle and step, in G2P.
template <typename R> struct alignas(4 * sizeof(R)) V4 { R x, y, z, w; };
template <typename R> struct alignas(2 * sizeof(R)) V2 { R x, y; };

template <typename R> struct PState {
    V4<R>* A; V4<R>* V; V4<R>* Ba; V4<R>* Bb; V4<R>* Fa; V4<R>* Fb; V2<R>* Fc; V4<R>* Ta; V2<R>* Tb; V4<R>* M;
};

__device__ __forceinline__ V4<float> ld4(const V4<float>* p)
{
    float4 t = __ldg(reinterpret_cast<const float4*>(p));
    return {t.x, t.y, t.z, t.w};
}
__device__ __forceinline__ V4<double> ld4(const V4<double>* p)
{
    const double2* q = reinterpret_cast<const double2*>(p);
    double2 a = __ldg(q), b = __ldg(q + 1);
    return {a.x, a.y, b.x, b.y};
}
__device__ __forceinline__ V2<float> ld2(const V2<float>* p)
{
    float2 t = __ldg(reinterpret_cast<const float2*>(p));
    return {t.x, t.y};
}
__device__ __forceinline__ V2<double> ld2(const V2<double>* p)
{
    double2 t = __ldg(reinterpret_cast<const double2*>(p));
    return {t.x, t.y};
}
__device__ __forceinline__ void st4(V4<float>* p, V4<float> v)
{
    *reinterpret_cast<float4*>(p) = make_float4(v.x, v.y, v.z, v.w);
}
__device__ __forceinline__ void st4(V4<double>* p, V4<double> v)
{
    double2* q = reinterpret_cast<double2*>(p);
    q[0] = make_double2(v.x, v.y);
    q[1] = make_double2(v.z, v.w);
}
__device__ __forceinline__ void st2(V2<float>* p, V2<float> v) { *reinterpret_cast<float2*>(p) = make_float2(v.x, v.y); }
__device__ __forceinline__ void st2(V2<double>* p, V2<double> v) { *reinterpret_cast<double2*>(p) = make_double2(v.x, v.y); }

// integer payloads (cell, id) ride in a float / double lane as raw bits
__device__ __forceinline__ float u2r(uint32_t u, float) { return __uint_as_float(u); }
__device__ __forceinline__ double u2r(uint32_t u, double) { return __longlong_as_double((long long)u); }
__device__ __forceinline__ uint32_t r2u(float r) { return __float_as_uint(r); }
__device__ __forceinline__ uint32_t r2u(double r) { return (uint32_t)__double_as_longlong(r); }

// cell index packing: 10 bits per axis in 3-D, 15 bits per axis in 2-D
template <int D> __device__ __forceinline__ uint32_t pack_cell(const int* c)
{
    if (D == 3) return (uint32_t)c[0] | ((uint32_t)c[1] << 10) | ((uint32_t)c[2] << 20);
    return (uint32_t)c[0] | ((uint32_t)c[1] << 15);
}
template <int D> __device__ __forceinline__ void unpack_cell(uint32_t u, int* c)
{
    if (D == 3) { c[0] = u & 1023; c[1] = (u >> 10) & 1023; c[2] = (u >> 20) & 1023; }
    else { c[0] = u & 32767; c[1] = (u >> 15) & 32767; }
}

template <int D, typename R> struct Particle {
    R o[D];
    int cell[D];
    uint32_t id;
    R v[D];
    R B[D * D];
    R F[D * D];
    R tau[(D == 3) ? 6 : 3];   // 3-D: t00 t11 t22 t01 t02 t12; 2-D: t00 t11 t01
    R mu, lam;                 // Lame parameters, when parameters per particle are set
    R pm, pv;                  // mass m_p and volume V_p, likewise
};

// full D x D matrix (row-major) of a symmetric stress held as its independent entries
template <int D, typename R> __device__ __forceinline__ void tau_full(const R* t, R* T)
{
    if (D == 3) {
        T[0] = t[0]; T[4] = t[1]; T[8] = t[2];
        T[1] = T[3] = t[3];
        T[2] = T[6] = t[4];
        T[5] = T[7] = t[5];
    } else {
        T[0] = t[0]; T[3] = t[1];
        T[1] = T[2] = t[2];
    }
}

// position (offset, cell; + id in 2-D): what the key and P2G need
template <int D, typename R>
__device__ __forceinline__ void load_x(const PState<R>& s, uint32_t k, Particle<D, R>& p)
{
    const V4<R> a = ld4(s.A + k);
    if (D == 3) {
        p.o[0] = a.x; p.o[1] = a.y; p.o[2] = a.z;
        unpack_cell<D>(r2u(a.w), p.cell);
    } else {
        p.o[0] = a.x; p.o[1] = a.y;
        unpack_cell<D>(r2u(a.z), p.cell);
        p.id = r2u(a.w);
    }
}

// position (offset, cell) and F (+ id): what G2P needs
template <int D, typename R>
__device__ __forceinline__ void load_xF(const PState<R>& s, uint32_t k, Particle<D, R>& p)
{
    V4<R> a = ld4(s.A + k);
    V4<R> fa = ld4(s.Fa + k);
    if (D == 3) {
        p.o[0] = a.x; p.o[1] = a.y; p.o[2] = a.z;
        unpack_cell<D>(r2u(a.w), p.cell);
        V4<R> fb = ld4(s.Fb + k);
        V2<R> fc = ld2(s.Fc + k);
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

template <int D, typename R>
__device__ __forceinline__ void load_vB(const PState<R>& s, uint32_t k, Particle<D, R>& p)
{
    V4<R> v = ld4(s.V + k);
    V4<R> ba = ld4(s.Ba + k);
    if (D == 3) {
        V4<R> bb = ld4(s.Bb + k);
        p.v[0] = v.x; p.v[1] = v.y; p.v[2] = v.z;
        p.B[0] = v.w; p.B[1] = ba.x; p.B[2] = ba.y; p.B[3] = ba.z; p.B[4] = ba.w;
        p.B[5] = bb.x; p.B[6] = bb.y; p.B[7] = bb.z; p.B[8] = bb.w;
    } else {
        p.v[0] = v.x; p.v[1] = v.y;
        p.B[0] = v.z; p.B[1] = v.w; p.B[2] = ba.x; p.B[3] = ba.y;
    }
}

// the stress of the particle (what P2G needs besides position, v and B)
template <int D, typename R>
__device__ __forceinline__ void load_tau(const PState<R>& s, uint32_t k, Particle<D, R>& p)
{
    if (D == 3) {
        const V4<R> ta = ld4(s.Ta + k);
        const V2<R> tb = ld2(s.Tb + k);
        p.tau[0] = ta.x; p.tau[1] = ta.y; p.tau[2] = ta.z; p.tau[3] = ta.w;
        p.tau[4] = tb.x; p.tau[5] = tb.y;
    } else {
        const V4<R> ba = ld4(s.Ba + k);
        const V2<R> tb = ld2(s.Tb + k);
        p.tau[0] = ba.z; p.tau[1] = ba.w; p.tau[2] = tb.x;
    }
}

// the velocity alone (what the FLIP update adds to)
template <int D, typename R>
__device__ __forceinline__ void load_v(const PState<R>& s, uint32_t k, Particle<D, R>& p)
{
    const V4<R> v = ld4(s.V + k);
    p.v[0] = v.x;
    p.v[1] = v.y;
    if (D == 3) p.v[D - 1] = v.z;
}

template <int D, typename R>
__device__ __forceinline__ void load_mat(const PState<R>& s, uint32_t k, Particle<D, R>& p)
{
    const V4<R> m = ld4(s.M + k);
    p.mu = m.x;
    p.lam = m.y;
    p.pm = m.z;
    p.pv = m.w;
}

// every lane of the particle; the stress lanes only when `with_tau` (a model is set), the
// material lane only when `with_mat` (a material per particle is set)
template <int D, typename R>
__device__ __forceinline__ void store_all(const PState<R>& s, uint32_t k, const Particle<D, R>& p, bool with_tau,
                                          bool with_mat = false)
{
    const R z = R(0);
    if (with_mat) st4(s.M + k, V4<R>{p.mu, p.lam, p.pm, p.pv});
    if (D == 3) {
        st4(s.A + k, V4<R>{p.o[0], p.o[1], p.o[2], u2r(pack_cell<D>(p.cell), z)});
        st4(s.V + k, V4<R>{p.v[0], p.v[1], p.v[2], p.B[0]});
        st4(s.Ba + k, V4<R>{p.B[1], p.B[2], p.B[3], p.B[4]});
        st4(s.Bb + k, V4<R>{p.B[5], p.B[6], p.B[7], p.B[8]});
        st4(s.Fa + k, V4<R>{p.F[0], p.F[1], p.F[2], p.F[3]});
        st4(s.Fb + k, V4<R>{p.F[4], p.F[5], p.F[6], p.F[7]});
        st2(s.Fc + k, V2<R>{p.F[8], u2r(p.id, z)});
        if (with_tau) {
            st4(s.Ta + k, V4<R>{p.tau[0], p.tau[1], p.tau[2], p.tau[3]});
            st2(s.Tb + k, V2<R>{p.tau[4], p.tau[5]});
        }
    } else {
        st4(s.A + k, V4<R>{p.o[0], p.o[1], u2r(pack_cell<D>(p.cell), z), u2r(p.id, z)});
        st4(s.V + k, V4<R>{p.v[0], p.v[1], p.B[0], p.B[1]});
        st4(s.Ba + k, V4<R>{p.B[2], p.B[3], with_tau ? p.tau[0] : z, with_tau ? p.tau[1] : z});
        st4(s.Fa + k, V4<R>{p.F[0], p.F[1], p.F[2], p.F[3]});
        if (with_tau) st2(s.Tb + k, V2<R>{p.tau[2], z});
    }
}

// ---------------------------------------------------------------- device config
template <typename R> struct DevCfg {
    int res[3];
    int nb[3];           // node blocks per axis
    R dx, inv_dx;
    R origin[3];
    R dt;
    R gravity[3];
    int boundary, wall, model, transfer;
    int mat;             // 1: per-particle parameters in lane M (mu, lam, m_p, V_p)
    R mu, lam;
    R mass, vol;
    R inv_kdx;           // 1 / (kappa dx): B_p D_p^{-1} (x_i - x_p) = (B_p / (kappa dx)) r^, r^ = (x_i - x_p)/dx
    int n;               // particles
    int nblocks;         // node blocks
    const R* dtp;        // when set, the time step is read here (adaptive stepping), else dt
    uint32_t* smax;      // when set, G2P max-reduces the Sec. 4.3 particle speed here (FP32 bits)
    R cfl_coef;          // 6 sqrt(d) / dx of the Sec. 4.3 speed |v| + 6 sqrt(d)/dx |B|_F
    R flip_alpha;        // transfer 2: weight of the FLIP update
    unsigned wait_limit; // polls of G2P's first wait for its staged grid blocks before it gives up
};

// the step's time step: fixed, or the adaptive one on the device
template <typename R> __device__ __forceinline__ R step_dt(const DevCfg<R>& c) { return c.dtp ? *c.dtp : c.dt; }

// ---------------------------------------------------------------- stencil (Sec. 3.5)
// Base node and 1-D weights / derivatives in grid units for one axis.  u = cell + o.
//   quadratic: base = floor(u - 1/2) -> cell - 1 + [o >= 1/2], fx = u - base in [1/2, 3/2)
//   cubic:     base = floor(u) - 1   -> cell - 1,               fx = u - base in [1, 2)
// w[a] = N(fx - a), dw[a] = N'(fx - a) (derivative in grid units; divide by dx for x).
template <int ORDER, typename R>
__device__ __forceinline__ void axis_weights(R o, int cell, int& base, R& fx, R* w, R* dw)
{
    if (ORDER == 2) {
        const bool hi = o >= R(0.5);
        base = hi ? cell : cell - 1;
        fx = hi ? o : o + R(1);
        const R t0 = R(1.5) - fx, t1 = fx - R(1), t2 = fx - R(0.5);
        w[0] = R(0.5) * t0 * t0;
        w[1] = R(0.75) - t1 * t1;
        w[2] = R(0.5) * t2 * t2;
        dw[0] = -t0;
        dw[1] = R(-2) * t1;
        dw[2] = t2;
    } else {
        base = cell - 1;
        fx = o + R(1);
        const R a0 = R(2) - fx;          // |t| for node 0 (t = fx)       in (0,1]
        const R a1 = fx - R(1);          // |t| for node 1 (t = fx - 1)   in [0,1)
        const R a2 = R(2) - fx;          // |t| for node 2 (t = fx - 2)   in (0,1]
        const R a3 = fx - R(1);          // 2 - |t| for node 3 (|t| = 3 - fx in (1,2])
        w[0] = a0 * a0 * a0 * (R(1) / R(6));
        w[1] = R(0.5) * a1 * a1 * a1 - a1 * a1 + R(2) / R(3);
        w[2] = R(0.5) * a2 * a2 * a2 - a2 * a2 + R(2) / R(3);
        w[3] = a3 * a3 * a3 * (R(1) / R(6));
        dw[0] = R(-0.5) * a0 * a0;
        dw[1] = R(1.5) * a1 * a1 - R(2) * a1;
        dw[2] = -(R(1.5) * a2 * a2 - R(2) * a2);
        dw[3] = R(0.5) * a3 * a3;
    }
}

// The 1-D weights and derivatives from the distance fx to the base node alone (as
// axis_weights, for a caller that knows the base)
template <int ORDER, typename R> __device__ __forceinline__ void axis_weights_fx(R fx, R* w, R* dw)
{
    if (ORDER == 2) {
        const R t0 = R(1.5) - fx, t1 = fx - R(1), t2 = fx - R(0.5);
        w[0] = R(0.5) * t0 * t0;
        w[1] = R(0.75) - t1 * t1;
        w[2] = R(0.5) * t2 * t2;
        dw[0] = -t0;
        dw[1] = R(-2) * t1;
        dw[2] = t2;
    } else {
        const R a0 = R(2) - fx, a1 = fx - R(1), a2 = R(2) - fx, a3 = fx - R(1);
        w[0] = a0 * a0 * a0 * (R(1) / R(6));
        w[1] = R(0.5) * a1 * a1 * a1 - a1 * a1 + R(2) / R(3);
        w[2] = R(0.5) * a2 * a2 * a2 - a2 * a2 + R(2) / R(3);
        w[3] = a3 * a3 * a3 * (R(1) / R(6));
        dw[0] = R(-0.5) * a0 * a0;
        dw[1] = R(1.5) * a1 * a1 - R(2) * a1;
        dw[2] = -(R(1.5) * a2 * a2 - R(2) * a2);
        dw[3] = R(0.5) * a3 * a3;
    }
}

// ---------------------------------------------------------------- small matrices
template <typename R> __device__ __forceinline__ R det3(const R* A)
{
    return A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
           A[2] * (A[3] * A[7] - A[4] * A[6]);
}

// Rotation R of the polar decomposition F = R S (det R = +1), 3-D.  Method: cyclic
// Jacobi eigen-decomposition of the symmetric F^T F (Golub & Van Loan, Sec. 8.5) gives V
// and sigma^2; the columns of F V, ordered by decreasing norm, are orthonormalised
// (Gram-Schmidt, third column as the cross product so det U = +1), and R = U V^T.
// This is the structure of McAdams et al. 2011 ("Computing the SVD of 3x3 matrices with
// minimal branching"), written here with exact rotations instead of its approximate ones.
template <typename R> __device__ __forceinline__ R rsqrt_t(R x);
template <> __device__ __forceinline__ float rsqrt_t<float>(float x) { return rsqrtf(x); }
template <> __device__ __forceinline__ double rsqrt_t<double>(double x) { return rsqrt(x); }

template <typename R>
__device__ __forceinline__ void jacobi_rot(R* S, R* V, int p, int q, int r)
{
    // S symmetric 3x3 (row-major, full), zero S_pq with J = [c s; -s c] in plane (p,q)
    const R spq = S[p * 3 + q];
    if (spq == R(0)) return;
    const R tau = (S[q * 3 + q] - S[p * 3 + p]) / (R(2) * spq);
    const R t = (tau >= R(0) ? R(1) : R(-1)) / (fabs(tau) + sqrt(R(1) + tau * tau));
    const R c = rsqrt_t<R>(R(1) + t * t), s = t * c;
    const R spp = S[p * 3 + p], sqq = S[q * 3 + q];
    const R srp = S[r * 3 + p], srq = S[r * 3 + q];
    S[p * 3 + p] = spp - t * spq;
    S[q * 3 + q] = sqq + t * spq;
    S[p * 3 + q] = S[q * 3 + p] = R(0);
    const R nrp = c * srp - s * srq, nrq = s * srp + c * srq;
    S[r * 3 + p] = S[p * 3 + r] = nrp;
    S[r * 3 + q] = S[q * 3 + r] = nrq;
    for (int i = 0; i < 3; ++i) {
        const R vp = V[i * 3 + p], vq = V[i * 3 + q];
        V[i * 3 + p] = c * vp - s * vq;
        V[i * 3 + q] = s * vp + c * vq;
    }
}

// gap (may be NULL): (sigma_2^2 - sigma_3^2) / sigma_1^2 of the two smallest singular values,
// which decides how well the rotation of an inverted F is resolved
template <typename R>
__device__ __forceinline__ void polar3(const R* F, R* Rot, R* gap = nullptr)
{
    R S[9], V[9] = {R(1), R(0), R(0), R(0), R(1), R(0), R(0), R(0), R(1)};
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            S[a * 3 + b] = F[0 * 3 + a] * F[0 * 3 + b] + F[1 * 3 + a] * F[1 * 3 + b] + F[2 * 3 + a] * F[2 * 3 + b];
#pragma unroll 1
    for (int sweep = 0; sweep < 6; ++sweep) {
        const R off = fabs(S[1]) + fabs(S[2]) + fabs(S[5]);
        const R diag = fabs(S[0]) + fabs(S[4]) + fabs(S[8]);
        // stop once the off-diagonal part is at the rounding level of the type: further
        // rotations cannot change R beyond rounding (FP32: ~4 eps, FP64: ~1e-16)
        if (off <= diag * (sizeof(R) == 4 ? R(5e-7) : R(1e-16))) break;
        jacobi_rot(S, V, 0, 1, 2);
        jacobi_rot(S, V, 0, 2, 1);
        jacobi_rot(S, V, 1, 2, 0);
    }
    // B = F V; order columns by decreasing norm (swap V columns alongside)
    R Bm[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            Bm[i * 3 + j] = F[i * 3 + 0] * V[0 * 3 + j] + F[i * 3 + 1] * V[1 * 3 + j] + F[i * 3 + 2] * V[2 * 3 + j];
    R nrm[3];
    for (int j = 0; j < 3; ++j) nrm[j] = Bm[j] * Bm[j] + Bm[3 + j] * Bm[3 + j] + Bm[6 + j] * Bm[6 + j];
    auto swapc = [&](int a, int b) {
        for (int i = 0; i < 3; ++i) {
            R t = Bm[i * 3 + a]; Bm[i * 3 + a] = Bm[i * 3 + b]; Bm[i * 3 + b] = t;
            t = V[i * 3 + a]; V[i * 3 + a] = V[i * 3 + b]; V[i * 3 + b] = t;
        }
        R t = nrm[a]; nrm[a] = nrm[b]; nrm[b] = t;
    };
    if (nrm[1] > nrm[0]) swapc(0, 1);
    if (nrm[2] > nrm[0]) swapc(0, 2);
    if (nrm[2] > nrm[1]) swapc(1, 2);
    if (gap) *gap = nrm[0] > R(0) ? (nrm[1] - nrm[2]) / nrm[0] : R(0);
    if (det3(V) < R(0))
        for (int i = 0; i < 3; ++i) V[i * 3 + 2] = -V[i * 3 + 2];
    // U by Gram-Schmidt; degenerate columns completed from the coordinate axes
    R u0[3], u1[3], u2[3];
    R n0 = nrm[0];
    if (n0 > R(0)) {
        const R inv = rsqrt_t<R>(n0);
        for (int i = 0; i < 3; ++i) u0[i] = Bm[i * 3 + 0] * inv;
    } else {
        u0[0] = R(1); u0[1] = R(0); u0[2] = R(0);
    }
    R d01 = u0[0] * Bm[1] + u0[1] * Bm[4] + u0[2] * Bm[7];
    for (int i = 0; i < 3; ++i) u1[i] = Bm[i * 3 + 1] - d01 * u0[i];
    R n1 = u1[0] * u1[0] + u1[1] * u1[1] + u1[2] * u1[2];
    if (!(n1 > n0 * (sizeof(R) == 4 ? R(1e-12) : R(1e-28)))) {
        // pick the axis least aligned with u0 and orthogonalise it
        int ax = (fabs(u0[0]) < fabs(u0[1])) ? (fabs(u0[0]) < fabs(u0[2]) ? 0 : 2) : (fabs(u0[1]) < fabs(u0[2]) ? 1 : 2);
        for (int i = 0; i < 3; ++i) u1[i] = (i == ax ? R(1) : R(0)) - u0[ax] * u0[i];
        n1 = u1[0] * u1[0] + u1[1] * u1[1] + u1[2] * u1[2];
    }
    const R inv1 = rsqrt_t<R>(n1);
    for (int i = 0; i < 3; ++i) u1[i] *= inv1;
    u2[0] = u0[1] * u1[2] - u0[2] * u1[1];
    u2[1] = u0[2] * u1[0] - u0[0] * u1[2];
    u2[2] = u0[0] * u1[1] - u0[1] * u1[0];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            Rot[a * 3 + b] = u0[a] * V[b * 3 + 0] + u1[a] * V[b * 3 + 1] + u2[a] * V[b * 3 + 2];
}

// residual of a polar rotation: asymmetry of R^T F relative to |F| (R is orthonormal by
// construction, so a wrong R shows up as a non-symmetric stretch R^T F)
template <typename R>
__device__ __forceinline__ R polar_residual(const R* F, const R* Rot)
{
    R fmax = R(0);
#pragma unroll
    for (int i = 0; i < 9; ++i) fmax = fmax > fabs(F[i]) ? fmax : fabs(F[i]);
    R asym = R(0);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = a + 1; b < 3; ++b) {
            const R sab = Rot[0 * 3 + a] * F[0 * 3 + b] + Rot[1 * 3 + a] * F[1 * 3 + b] + Rot[2 * 3 + a] * F[2 * 3 + b];
            const R sba = Rot[0 * 3 + b] * F[0 * 3 + a] + Rot[1 * 3 + b] * F[1 * 3 + a] + Rot[2 * 3 + b] * F[2 * 3 + a];
            asym += fabs(sab - sba);
        }
    return asym / (fmax > R(0) ? fmax : R(1));
}

template <typename R> __device__ __forceinline__ R rcbrt_t(R x);
template <> __device__ __forceinline__ float rcbrt_t<float>(float x) { return rcbrtf(x); }
template <> __device__ __forceinline__ double rcbrt_t<double>(double x) { return rcbrt(x); }

// Rotation of the polar decomposition F = R S by the scaled Newton iteration
//   X <- (g X + X^{-T} / g) / 2,   g = |det X|^{-1/3},   X^{-T} = cof(X) / det X
// (Higham 1986, "Computing the polar decomposition -- with applications", with the
// determinant scaling; the scaling is dropped once the step is small, where the plain
// iteration converges quadratically).  A step below 2e-4 (FP32) / 1e-8 (FP64) means the
// next one would be below rounding, so the iterate is returned.  Returns false, leaving
// Rot unset, when det F <= 0 (the orthogonal factor is then not the det R = +1 rotation)
// or without convergence in 12 steps; the caller then takes the Jacobi route.
template <typename R>
__device__ __forceinline__ bool polar_newton3(const R* F, R* Rot)
{
    R X[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) X[i] = F[i];
    const R tol = sizeof(R) == 4 ? R(2e-4) : R(1e-8);
    // the scaling factor (det^(-1/3)) speeds up iterates far from orthogonal; near a rotation
    // (det F within 5 % of 1) the plain iteration already converges quadratically
    bool scale = fabs(det3<R>(F) - R(1)) > R(0.05);
#pragma unroll 1
    for (int it = 0; it < 12; ++it) {
        R C[9];
        C[0] = X[4] * X[8] - X[5] * X[7];
        C[1] = X[5] * X[6] - X[3] * X[8];
        C[2] = X[3] * X[7] - X[4] * X[6];
        C[3] = X[2] * X[7] - X[1] * X[8];
        C[4] = X[0] * X[8] - X[2] * X[6];
        C[5] = X[1] * X[6] - X[0] * X[7];
        C[6] = X[1] * X[5] - X[2] * X[4];
        C[7] = X[2] * X[3] - X[0] * X[5];
        C[8] = X[0] * X[4] - X[1] * X[3];
        const R det = X[0] * C[0] + X[1] * C[1] + X[2] * C[2];
        if (!(det > R(0))) return false;
        const R g = scale ? rcbrt_t<R>(det) : R(1);
        const R a = R(0.5) * g, b = R(0.5) / (g * det);
        R d = R(0);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const R xn = a * X[i] + b * C[i];
            d = fmax(d, fabs(xn - X[i]));
            X[i] = xn;
        }
        if (d <= tol) {
#pragma unroll
            for (int i = 0; i < 9; ++i) Rot[i] = X[i];
            return true;
        }
        scale = d > R(1e-2);
    }
    return false;
}

// For an inverted F (det F <= 0) the rotation's sign convention puts the negative singular
// value last; the rotation in the plane of the two smallest singular values is then
// determined only to eps / gap (it is not corrected through U = F V as for det F > 0), and
// the residual of polar_residual does not see it (the two eigenvalues of R^T F in that plane
// nearly cancel).  Below gap = 1/8 the FP32 rotation can be off by more than ~1e-6, so it is
// recomputed in FP64: the "nearly coincident singular values" case of the FP64 fallback.
template <typename R> __device__ __forceinline__ bool inverted_unresolved(const R* F, R gap)
{
    return gap < R(0.125) && det3<R>(F) <= R(0);
}

// Kirchhoff-type stress tau = V_p P(F) F^T, which is symmetric for both models, returned
// as its independent entries (3-D: t00 t11 t22 t01 t02 t12; 2-D: t00 t11 t01).
// Fixed-corotated: P = 2 mu (F - R) + lam (J - 1) J F^{-T}
//   =>  P F^T = 2 mu (F - R) F^T + lam (J - 1) J I, off-diagonal entries symmetrised.
// FP32: a rotation from the Jacobi route is recomputed in FP64 when it fails its residual
// check (nearly coincident singular values of F at FP32 resolution, or near-singular F);
// each fallback is counted.
template <int D, typename R>
__device__ __forceinline__ void stress_sym_fcr(const R* F, R mu, R lam, R vol, R* t, unsigned* fallbacks)
{
    R Rot[D * D];
    R J;
    if (D == 2) {
        R a = F[0] + F[3], b = F[2] - F[1];
        R r2 = a * a + b * b;
        R c = R(1), s = R(0);
        if (r2 > R(0)) { R inv = rsqrt_t<R>(r2); c = a * inv; s = b * inv; }
        Rot[0] = c; Rot[1] = -s; Rot[2] = s; Rot[3] = c;
        J = F[0] * F[3] - F[1] * F[2];
    } else {
        // a converged Newton iterate is the orthogonal polar factor to working precision; the
        // Jacobi route (det F <= 0, or no convergence) is checked and redone in FP64 if needed
        if (!polar_newton3<R>(F, Rot)) {
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
        J = det3<R>(F);
    }
    const R c2 = R(2) * mu * vol;
    const R iso = vol * lam * (J - R(1)) * J;
    auto s = [&](int a, int b) {
        R x = R(0);
#pragma unroll
        for (int k = 0; k < D; ++k) x += (F[a * D + k] - Rot[a * D + k]) * F[b * D + k];
        return x;
    };
    if (D == 3) {
        t[0] = c2 * s(0, 0) + iso;
        t[1] = c2 * s(1, 1) + iso;
        t[2] = c2 * s(2, 2) + iso;
        t[3] = R(0.5) * c2 * (s(0, 1) + s(1, 0));
        t[4] = R(0.5) * c2 * (s(0, 2) + s(2, 0));
        t[5] = R(0.5) * c2 * (s(1, 2) + s(2, 1));
    } else {
        t[0] = c2 * s(0, 0) + iso;
        t[1] = c2 * s(1, 1) + iso;
        t[2] = R(0.5) * c2 * (s(0, 1) + s(1, 0));
    }
}

// Neo-Hookean: P = mu (F - F^{-T}) + lam log(J) F^{-T}  =>  tau = V (mu (F F^T - I) + lam log(J) I)
template <int D, typename R>
__device__ __forceinline__ void stress_sym_nh(const R* F, R mu, R lam, R vol, R* t)
{
    const R J = (D == 3) ? det3<R>(F) : F[0] * F[3] - F[1] * F[2];
    const R iso = vol * (lam * log(J) - mu);
    const R cm = vol * mu;
    auto ff = [&](int a, int b) {
        R x = R(0);
#pragma unroll
        for (int k = 0; k < D; ++k) x += F[a * D + k] * F[b * D + k];
        return x;
    };
    if (D == 3) {
        t[0] = cm * ff(0, 0) + iso;
        t[1] = cm * ff(1, 1) + iso;
        t[2] = cm * ff(2, 2) + iso;
        t[3] = cm * ff(0, 1);
        t[4] = cm * ff(0, 2);
        t[5] = cm * ff(1, 2);
    } else {
        t[0] = cm * ff(0, 0) + iso;
        t[1] = cm * ff(1, 1) + iso;
        t[2] = cm * ff(0, 1);
    }
}

// model 1: fixed-corotated, model 2: Neo-Hookean (model 0 has no stress and never calls this)
template <int D, typename R>
__device__ __forceinline__ void stress_sym(int model, const R* F, R mu, R lam, R vol, R* t, unsigned* fallbacks)
{
    if (model == 2) stress_sym_nh<D, R>(F, mu, lam, vol, t);
    else stress_sym_fcr<D, R>(F, mu, lam, vol, t, fallbacks);
}

// ---------------------------------------------------------------- misc
__device__ __forceinline__ void set_err(uint32_t* err, uint32_t bit) { atomicOr(err, bit); }

// block-major node index of global node coordinates g (block edge 4)
template <int D> __device__ __forceinline__ uint32_t node_index(const int* g, const int* nb)
{
    if (D == 3) {
        const uint32_t blk = ((uint32_t)(g[2] >> 2) * nb[1] + (uint32_t)(g[1] >> 2)) * nb[0] + (uint32_t)(g[0] >> 2);
        return (blk << 6) | ((uint32_t)(g[2] & 3) << 4) | ((uint32_t)(g[1] & 3) << 2) | (uint32_t)(g[0] & 3);
    }
    const uint32_t blk = (uint32_t)(g[1] >> 2) * nb[0] + (uint32_t)(g[0] >> 2);
    return (blk << 4) | ((uint32_t)(g[1] & 3) << 2) | (uint32_t)(g[0] & 3);
}

}  // namespace apic
