/*
 * apic_oracle.c -- plain, slow FP64 CPU oracle for the APIC / explicit MPM step of
 * Jiang, Schroeder & Teran, "An angular momentum conserving Affine-Particle-In-Cell
 * method" (arXiv:1603.06188).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the checker the CUDA path is compared
 * against.  Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * may load it.  It shares no code, header, table or constant with the CUDA library.
 *
 * Everything is written as the paper states it: dense grid arrays, loops over every
 * particle and every node of its stencil, no blocking, fusion or reordering.
 *
 * Conventions
 *   - d = dim (2 or 3).  Vectors are d doubles, matrices d*d doubles row-major
 *     (M[a*d+b] = M_ab).
 *   - Grid node i = (i0,i1[,i2]) sits at x_i = origin + i*dx, 0 <= i_a < res[a].
 *     Linear node index: i0 + res0*(i1 + res1*i2).
 *   - w_ip = N((x_p - x_i)/dx) as a tensor product of 1-D cardinal B-splines
 *     (Sec. 3.5); grad w_ip is the gradient with respect to x_p, which is what
 *     makes sum_i x_i (grad w_ip)^T = I (Sec. 3.5).
 *   - Integrator family parameter lambda (Sec. 3.3).  or_p2g evaluates forces for the
 *     explicit member lambda = 0 (F^{n+lambda} = F^n); or_force_at and or_step_lambda1
 *     evaluate them for the other explicit member, lambda = 1 (F^{n+lambda} = F^{n+1});
 *     or_step_midpoint takes the implicit midpoint rule, lambda = 1/2 (Sec. 4.1-4.2), with
 *     Newton on the grid velocity change and mass-inner-product conjugate gradients
 *     (Algorithm 1) on the force-derivative product.
 *
 * Readings of the paper taken here (each is listed with its reason in the design notes):
 *   - force sign: f_i = -sum_p V_p P(F_p^n) (F_p^n)^T grad w_ip, i.e. f = -dPhi/dx~
 *     (the printed force equation of Sec. 3.3 drops the minus sign);
 *   - kernel N: quadratic / cubic cardinal B-splines (never written out in the paper);
 *   - stencil base: floor(x/dx - 1/2) (quadratic), floor(x/dx) - 1 (cubic);
 *   - constitutive model: fixed-corotated, P = 2 mu (F - R) + lam (J - 1) J F^{-T};
 *   - Neo-Hookean (named, not written out, by the paper's experiments):
 *     Psi = mu/2 (tr(F^T F) - d) - mu log J + lam/2 (log J)^2,
 *     P = mu (F - F^{-T}) + lam log(J) F^{-T};
 *   - gravity and walls are not in the paper; they are applied in the grid update after
 *     the force, gravity only where m_i > 0.  Sticky walls zero v~ on wall nodes; slip
 *     walls zero only the component of v~ normal to each wall the node lies in.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int dim;            /* 2 or 3 */
    int order;          /* 2 = quadratic, 3 = cubic B-spline */
    int transfer;       /* 0 = APIC, 1 = PIC (C_p = 0, no B on the way back), 2 = PIC/FLIP blend */
    int res[3];         /* grid nodes per axis */
    double dx;
    double origin[3];
    double dt;
    double gravity[3];
    int boundary;       /* 0 = none, 1 = sticky walls, 2 = slip walls */
    int wall;           /* wall thickness in nodes */
    int model;          /* 0 = none (transfer only), 1 = fixed-corotated, 2 = Neo-Hookean */
    double mu, lam;     /* Lame parameters */
    double lambda_t;    /* integrator family parameter lambda of Sec. 3.3 */
    double flip_alpha;  /* transfer 2: weight of the FLIP update in a PIC/FLIP blend (1 = FLIP) */
} or_cfg;

/* ------------------------------------------------------------------ */
/* Sec. 3.5: 1-D cardinal B-splines and their derivatives.            */
/* ------------------------------------------------------------------ */
double or_N(int order, double t)
{
    double a = fabs(t);
    if (order == 2) {
        if (a < 0.5) return 0.75 - a * a;
        if (a < 1.5) return 0.5 * (1.5 - a) * (1.5 - a);
        return 0.0;
    }
    if (order == 3) {
        if (a < 1.0) return 0.5 * a * a * a - a * a + 2.0 / 3.0;
        if (a < 2.0) return (2.0 - a) * (2.0 - a) * (2.0 - a) / 6.0;
        return 0.0;
    }
    return 0.0;
}

double or_dN(int order, double t)
{
    double a = fabs(t), s = (t < 0.0) ? -1.0 : 1.0;
    if (order == 2) {
        if (a < 0.5) return -2.0 * t;
        if (a < 1.5) return -s * (1.5 - a);
        return 0.0;
    }
    if (order == 3) {
        if (a < 1.0) return s * (1.5 * a * a - 2.0 * a);
        if (a < 2.0) return -s * 0.5 * (2.0 - a) * (2.0 - a);
        return 0.0;
    }
    return 0.0;
}

static int stencil_width(const or_cfg* c) { return c->order + 1; }
static int stencil_count(const or_cfg* c)
{
    int K = stencil_width(c), n = 1;
    for (int a = 0; a < c->dim; ++a) n *= K;
    return n;
}
static int64_t node_count(const or_cfg* c)
{
    int64_t n = 1;
    for (int a = 0; a < c->dim; ++a) n *= c->res[a];
    return n;
}
static int64_t node_index(const or_cfg* c, const int* i)
{
    int64_t idx = 0;
    for (int a = c->dim - 1; a >= 0; --a) idx = idx * c->res[a] + i[a];
    return idx;
}

/*
 * Stencil of one particle (Sec. 3.5): base node, the (order+1)^d weights w_ip and
 * gradients grad w_ip.  Stencil node j has per-axis offset a_k = (j / K^k) % K from
 * the base.  Returns 0, or -1 if any stencil node falls outside the grid.
 */
int or_stencil(const or_cfg* c, const double* xp, int* base, double* w, double* dw)
{
    const int d = c->dim, K = stencil_width(c);
    double w1[3][4], d1[3][4];
    int rc = 0;
    for (int a = 0; a < d; ++a) {
        double u = (xp[a] - c->origin[a]) / c->dx;
        base[a] = (c->order == 2) ? (int)floor(u - 0.5) : (int)floor(u) - 1;
        if (base[a] < 0 || base[a] + c->order > c->res[a] - 1) rc = -1;
        for (int k = 0; k < K; ++k) {
            double t = u - (double)(base[a] + k);
            w1[a][k] = or_N(c->order, t);
            d1[a][k] = or_dN(c->order, t) / c->dx;
        }
    }
    const int ns = stencil_count(c);
    for (int j = 0; j < ns; ++j) {
        int off[3] = {0, 0, 0}, r = j;
        for (int a = 0; a < d; ++a) { off[a] = r % K; r /= K; }
        double ww = 1.0;
        for (int a = 0; a < d; ++a) ww *= w1[a][off[a]];
        w[j] = ww;
        for (int g = 0; g < d; ++g) {
            double gg = 1.0;
            for (int a = 0; a < d; ++a) gg *= (a == g) ? d1[a][off[a]] : w1[a][off[a]];
            dw[j * d + g] = gg;
        }
    }
    return rc;
}

/* Brute force: w_ip and grad w_ip for EVERY node of the grid (definition in Sec. 3.5). */
void or_weights_all(const or_cfg* c, const double* xp, double* w_all, double* dw_all)
{
    const int d = c->dim;
    const int64_t nn = node_count(c);
    for (int64_t idx = 0; idx < nn; ++idx) {
        int i[3] = {0, 0, 0};
        int64_t r = idx;
        for (int a = 0; a < d; ++a) { i[a] = (int)(r % c->res[a]); r /= c->res[a]; }
        double t[3];
        for (int a = 0; a < d; ++a) t[a] = (xp[a] - (c->origin[a] + i[a] * c->dx)) / c->dx;
        double ww = 1.0;
        for (int a = 0; a < d; ++a) ww *= or_N(c->order, t[a]);
        w_all[idx] = ww;
        for (int g = 0; g < d; ++g) {
            double gg = 1.0;
            for (int a = 0; a < d; ++a)
                gg *= (a == g) ? or_dN(c->order, t[a]) / c->dx : or_N(c->order, t[a]);
            dw_all[idx * d + g] = gg;
        }
    }
}

static void stencil_node(const or_cfg* c, const int* base, int j, int* i, double* xi)
{
    const int K = stencil_width(c);
    int r = j;
    for (int a = 0; a < c->dim; ++a) {
        i[a] = base[a] + r % K;
        r /= K;
        xi[a] = c->origin[a] + i[a] * c->dx;
    }
}

/* ------------------------------------------------------------------ */
/* Small dense linear algebra (d = 2 or 3).                            */
/* ------------------------------------------------------------------ */
static double det_d(int d, const double* A)
{
    if (d == 2) return A[0] * A[3] - A[1] * A[2];
    return A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
           A[2] * (A[3] * A[7] - A[4] * A[6]);
}

/* cofactor matrix: cof(A) = det(A) A^{-T} */
static void cofactor_d(int d, const double* A, double* C)
{
    if (d == 2) {
        C[0] = A[3]; C[1] = -A[2]; C[2] = -A[1]; C[3] = A[0];
        return;
    }
    C[0] = A[4] * A[8] - A[5] * A[7];
    C[1] = A[5] * A[6] - A[3] * A[8];
    C[2] = A[3] * A[7] - A[4] * A[6];
    C[3] = A[2] * A[7] - A[1] * A[8];
    C[4] = A[0] * A[8] - A[2] * A[6];
    C[5] = A[1] * A[6] - A[0] * A[7];
    C[6] = A[1] * A[5] - A[2] * A[4];
    C[7] = A[2] * A[3] - A[0] * A[5];
    C[8] = A[0] * A[4] - A[1] * A[3];
}

static void inverse_d(int d, const double* A, double* Ai)
{
    double C[9];
    cofactor_d(d, A, C);
    double det = det_d(d, A);
    for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b) Ai[a * d + b] = C[b * d + a] / det;
}

static void matmul_d(int d, const double* A, const double* B, double* C)
{
    for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b) {
            double s = 0.0;
            for (int k = 0; k < d; ++k) s += A[a * d + k] * B[k * d + b];
            C[a * d + b] = s;
        }
}

/*
 * Singular value decomposition F = U diag(sigma) V^T by one-sided (Hestenes) Jacobi:
 * plane rotations applied to the columns of F until they are mutually orthogonal.
 * Returned with det U = det V = +1; when det F < 0 the smallest singular value is
 * made negative.  Columns of U belonging to zero singular values are completed to an
 * orthonormal basis.
 */
void or_svd(int d, const double* F, double* U, double* sigma, double* V)
{
    double A[9];
    memcpy(A, F, sizeof(double) * d * d);
    for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b) V[a * d + b] = (a == b) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < d - 1; ++p)
            for (int q = p + 1; q < d; ++q) {
                double al = 0.0, be = 0.0, ga = 0.0;
                for (int i = 0; i < d; ++i) {
                    al += A[i * d + p] * A[i * d + p];
                    be += A[i * d + q] * A[i * d + q];
                    ga += A[i * d + p] * A[i * d + q];
                }
                if (ga == 0.0) continue;
                double rel = fabs(ga) / sqrt(al * be);
                if (rel > off) off = rel;
                if (rel < 1e-17) continue;
                double zeta = (be - al) / (2.0 * ga);
                double t = ((zeta >= 0.0) ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                double cs = 1.0 / sqrt(1.0 + t * t), sn = cs * t;
                for (int i = 0; i < d; ++i) {
                    double ap = A[i * d + p], aq = A[i * d + q];
                    A[i * d + p] = cs * ap - sn * aq;
                    A[i * d + q] = sn * ap + cs * aq;
                    double vp = V[i * d + p], vq = V[i * d + q];
                    V[i * d + p] = cs * vp - sn * vq;
                    V[i * d + q] = sn * vp + cs * vq;
                }
            }
        if (off < 1e-15) break;
    }
    /* column norms are the singular values; sort descending (permuting U and V alike) */
    double s[3];
    for (int j = 0; j < d; ++j) {
        double nrm = 0.0;
        for (int i = 0; i < d; ++i) nrm += A[i * d + j] * A[i * d + j];
        s[j] = sqrt(nrm);
    }
    for (int a = 0; a < d; ++a)
        for (int b = a + 1; b < d; ++b)
            if (s[b] > s[a]) {
                double tmp = s[a]; s[a] = s[b]; s[b] = tmp;
                for (int i = 0; i < d; ++i) {
                    tmp = A[i * d + a]; A[i * d + a] = A[i * d + b]; A[i * d + b] = tmp;
                    tmp = V[i * d + a]; V[i * d + a] = V[i * d + b]; V[i * d + b] = tmp;
                }
            }
    double smax = s[0] > 0.0 ? s[0] : 1.0;
    int have[3] = {0, 0, 0};
    for (int j = 0; j < d; ++j) {
        if (s[j] > 1e-14 * smax) {
            for (int i = 0; i < d; ++i) U[i * d + j] = A[i * d + j] / s[j];
            have[j] = 1;
        }
    }
    /* complete missing columns of U (rank-deficient F) */
    for (int j = 0; j < d; ++j) {
        if (have[j]) continue;
        if (d == 2) {
            int o = 1 - j;
            if (have[o]) { U[0 * 2 + j] = -U[1 * 2 + o]; U[1 * 2 + j] = U[0 * 2 + o]; }
            else { U[0 * 2 + j] = (j == 0); U[1 * 2 + j] = (j == 1); }
        } else {
            /* Gram-Schmidt against the columns already present, starting from the axes */
            for (int e = 0; e < 3; ++e) {
                double cnd[3] = {0, 0, 0};
                cnd[e] = 1.0;
                for (int k = 0; k < 3; ++k) {
                    if (!have[k]) continue;
                    double dot = 0.0;
                    for (int i = 0; i < 3; ++i) dot += cnd[i] * U[i * 3 + k];
                    for (int i = 0; i < 3; ++i) cnd[i] -= dot * U[i * 3 + k];
                }
                double nrm = sqrt(cnd[0] * cnd[0] + cnd[1] * cnd[1] + cnd[2] * cnd[2]);
                if (nrm > 0.5) {
                    for (int i = 0; i < 3; ++i) U[i * 3 + j] = cnd[i] / nrm;
                    break;
                }
            }
        }
        have[j] = 1;
    }
    /* make V a rotation (flip a column of U and V together), then U */
    if (det_d(d, V) < 0.0) {
        for (int i = 0; i < d; ++i) { V[i * d + d - 1] = -V[i * d + d - 1]; U[i * d + d - 1] = -U[i * d + d - 1]; }
    }
    if (det_d(d, U) < 0.0) {
        for (int i = 0; i < d; ++i) U[i * d + d - 1] = -U[i * d + d - 1];
        s[d - 1] = -s[d - 1];
    }
    for (int j = 0; j < d; ++j) sigma[j] = s[j];
}

/* Rotation part of the polar decomposition, R = U V^T with det R = +1. */
void or_polar(int d, const double* F, double* R)
{
    double U[9], s[3], V[9];
    or_svd(d, F, U, s, V);
    for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b) {
            double acc = 0.0;
            for (int k = 0; k < d; ++k) acc += U[a * d + k] * V[b * d + k];
            R[a * d + b] = acc;
        }
}

/*
 * Fixed-corotated energy density and first Piola-Kirchhoff stress (Sec. 3.1 defines
 * P = dPsi/dF; the paper says the particular model does not matter, Sec. 3.3):
 *   Psi = mu |F - R|_F^2 + lam/2 (J - 1)^2,   P = 2 mu (F - R) + lam (J - 1) J F^{-T}.
 */
double or_psi_fcr(int d, double mu, double lam, const double* F)
{
    double R[9];
    or_polar(d, F, R);
    double s = 0.0;
    for (int k = 0; k < d * d; ++k) s += (F[k] - R[k]) * (F[k] - R[k]);
    double J = det_d(d, F);
    return mu * s + 0.5 * lam * (J - 1.0) * (J - 1.0);
}

void or_stress_fcr(int d, double mu, double lam, const double* F, double* P)
{
    double R[9], C[9];
    or_polar(d, F, R);
    cofactor_d(d, F, C);
    double J = det_d(d, F);
    for (int k = 0; k < d * d; ++k) P[k] = 2.0 * mu * (F[k] - R[k]) + lam * (J - 1.0) * C[k];
}

/* Neo-Hookean energy density and stress (see the header comment). */
double or_psi_nh(int d, double mu, double lam, const double* F)
{
    double s = 0.0;
    for (int k = 0; k < d * d; ++k) s += F[k] * F[k];
    double lj = log(det_d(d, F));
    return 0.5 * mu * (s - d) - mu * lj + 0.5 * lam * lj * lj;
}

void or_stress_nh(int d, double mu, double lam, const double* F, double* P)
{
    double C[9];
    cofactor_d(d, F, C);              /* J F^{-T} */
    double J = det_d(d, F);
    double lj = log(J);
    for (int k = 0; k < d * d; ++k) P[k] = mu * (F[k] - C[k] / J) + lam * lj * C[k] / J;
}

/*
 * Directional derivatives of the stresses, dP = dP/dF : dF, which the force-derivative
 * product of Sec. 3.3 needs.
 * Fixed-corotated: dP = 2 mu (dF - dR) + lam (cof F : dF) cof F + lam (J - 1) d(cof F), where
 *   d(cof F) = (cof F : dF) F^{-T} - J F^{-T} dF^T F^{-T}   (cof F = J F^{-T}, d log J = F^{-T} : dF),
 *   dR = R W, and W (skew) solves S W + W S = R^T dF - dF^T R for F = R S (S = R^T F symmetric).
 *   In 3-D, with W = [w]x and R^T dF - dF^T R = [k]x, that is (tr(S) I - S) w = k; in 2-D,
 *   W = [[0, -t], [t, 0]] with t = k / tr(S).
 * Neo-Hookean: dP = mu dF + (mu - lam log J) F^{-T} dF^T F^{-T} + lam (F^{-T} : dF) F^{-T}.
 */
static void fit_dft_fit(int d, const double* FiT, const double* dF, double* T)
{
    /* T = F^{-T} dF^T F^{-T} */
    double A[9];
    for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b) {
            double s = 0.0;
            for (int k = 0; k < d; ++k) s += FiT[a * d + k] * dF[b * d + k];
            A[a * d + b] = s;
        }
    matmul_d(d, A, FiT, T);
}

void or_dstress_fcr(int d, double mu, double lam, const double* F, const double* dF, double* dP)
{
    double R[9], S[9], K[9], W[9], dR[9], C[9], FiT[9], T[9];
    or_polar(d, F, R);
    for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b) {
            double s = 0.0, k = 0.0;
            for (int m = 0; m < d; ++m) {
                s += R[m * d + a] * F[m * d + b];
                k += R[m * d + a] * dF[m * d + b] - dF[m * d + a] * R[m * d + b];
            }
            S[a * d + b] = s;
            K[a * d + b] = k;
        }
    if (d == 3) {
        const double kv[3] = {K[7], K[2], K[3]};   /* (K21, K02, K10) */
        const double tr = S[0] + S[4] + S[8];
        double M[9], Mi[9], w[3];
        for (int k = 0; k < 9; ++k) M[k] = -S[k];
        M[0] += tr; M[4] += tr; M[8] += tr;
        inverse_d(3, M, Mi);
        for (int a = 0; a < 3; ++a) w[a] = Mi[a * 3 + 0] * kv[0] + Mi[a * 3 + 1] * kv[1] + Mi[a * 3 + 2] * kv[2];
        W[0] = 0.0;   W[1] = -w[2]; W[2] = w[1];
        W[3] = w[2];  W[4] = 0.0;   W[5] = -w[0];
        W[6] = -w[1]; W[7] = w[0];  W[8] = 0.0;
    } else {
        const double t = K[2] / (S[0] + S[3]);   /* K10 / tr(S) */
        W[0] = 0.0; W[1] = -t; W[2] = t; W[3] = 0.0;
    }
    matmul_d(d, R, W, dR);
    cofactor_d(d, F, C);
    const double J = det_d(d, F);
    double cdf = 0.0;
    for (int k = 0; k < d * d; ++k) {
        FiT[k] = C[k] / J;
        cdf += C[k] * dF[k];
    }
    fit_dft_fit(d, FiT, dF, T);
    for (int k = 0; k < d * d; ++k) {
        const double dcof = cdf * FiT[k] - J * T[k];
        dP[k] = 2.0 * mu * (dF[k] - dR[k]) + lam * cdf * C[k] + lam * (J - 1.0) * dcof;
    }
}

void or_dstress_nh(int d, double mu, double lam, const double* F, const double* dF, double* dP)
{
    double C[9], FiT[9], T[9];
    cofactor_d(d, F, C);
    const double J = det_d(d, F);
    const double lj = log(J);
    double tr = 0.0;
    for (int k = 0; k < d * d; ++k) {
        FiT[k] = C[k] / J;
        tr += FiT[k] * dF[k];
    }
    fit_dft_fit(d, FiT, dF, T);
    for (int k = 0; k < d * d; ++k) dP[k] = mu * dF[k] + (mu - lam * lj) * T[k] + lam * tr * FiT[k];
}

static void dstress_with(const or_cfg* c, const double* F, const double* dF, double* dP)
{
    if (c->model == 2) or_dstress_nh(c->dim, c->mu, c->lam, F, dF, dP);
    else or_dstress_fcr(c->dim, c->mu, c->lam, F, dF, dP);
}

static void stress_with(const or_cfg* c, double mu, double lam, const double* F, double* P)
{
    if (c->model == 2) or_stress_nh(c->dim, mu, lam, F, P);
    else or_stress_fcr(c->dim, mu, lam, F, P);
}

static double psi_of(const or_cfg* c, const double* F)
{
    if (c->model == 2) return or_psi_nh(c->dim, c->mu, c->lam, F);
    return or_psi_fcr(c->dim, c->mu, c->lam, F);
}

/* ------------------------------------------------------------------ */
/* Sec. 3.2: transfer to grid.                                         */
/* ------------------------------------------------------------------ */
/*
 * m_i = sum_p m_p w_ip
 * D_p = sum_i w_ip (x_i - x_p)(x_i - x_p)^T          (computed by summation)
 * m_i v_i = sum_p w_ip m_p (v_p + B_p D_p^{-1} (x_i - x_p))   (APIC)
 * m_i v_i = sum_p w_ip m_p v_p                                (PIC, Sec. 1 eq. 1)
 * f_i = -sum_p V_p P(F_p) F_p^T grad w_ip   (Sec. 3.3, lambda = 0, sign reading above)
 * Grid arrays are accumulated into (callers zero them first).  Returns the number of
 * particles whose stencil left the grid (those are skipped).
 * Per-particle Lame parameters mu_p, lam_p (a material per particle) replace c->mu, c->lam
 * when given (or_p2g_mat); or_p2g uses the configuration's.
 */
int64_t or_p2g_mat(const or_cfg* c, int64_t n, const double* x, const double* v, const double* B,
                   const double* F, const double* mass, const double* vol, const double* mu_p,
                   const double* lam_p, double* gm, double* gmv, double* gf)
{
    const int d = c->dim, ns = stencil_count(c);
    int64_t bad = 0;
    double w[64], dw[192];
    for (int64_t p = 0; p < n; ++p) {
        const double* xp = x + p * d;
        int base[3];
        if (or_stencil(c, xp, base, w, dw) != 0) { ++bad; continue; }
        double D[9] = {0}, Dinv[9], Cp[9] = {0};
        for (int j = 0; j < ns; ++j) {
            int i[3]; double xi[3], r[3];
            stencil_node(c, base, j, i, xi);
            for (int a = 0; a < d; ++a) r[a] = xi[a] - xp[a];
            for (int a = 0; a < d; ++a)
                for (int b = 0; b < d; ++b) D[a * d + b] += w[j] * r[a] * r[b];
        }
        if (c->transfer == 0) {
            inverse_d(d, D, Dinv);
            matmul_d(d, B + p * d * d, Dinv, Cp);
        }
        double tau[9] = {0};
        if (c->model != 0) {
            double P[9];
            stress_with(c, mu_p ? mu_p[p] : c->mu, lam_p ? lam_p[p] : c->lam, F + p * d * d, P);
            /* tau = V_p P F^T */
            const double* Fp = F + p * d * d;
            for (int a = 0; a < d; ++a)
                for (int b = 0; b < d; ++b) {
                    double s = 0.0;
                    for (int k = 0; k < d; ++k) s += P[a * d + k] * Fp[b * d + k];
                    tau[a * d + b] = vol[p] * s;
                }
        }
        for (int j = 0; j < ns; ++j) {
            int i[3]; double xi[3], r[3];
            stencil_node(c, base, j, i, xi);
            for (int a = 0; a < d; ++a) r[a] = xi[a] - xp[a];
            int64_t ni = node_index(c, i);
            gm[ni] += w[j] * mass[p];
            for (int a = 0; a < d; ++a) {
                double vel = v[p * d + a];
                for (int b = 0; b < d; ++b) vel += Cp[a * d + b] * r[b];
                gmv[ni * d + a] += w[j] * mass[p] * vel;
                if (c->model != 0) {
                    double s = 0.0;
                    for (int b = 0; b < d; ++b) s += tau[a * d + b] * dw[j * d + b];
                    gf[ni * d + a] -= s;
                }
            }
        }
    }
    return bad;
}

int64_t or_p2g(const or_cfg* c, int64_t n, const double* x, const double* v, const double* B,
               const double* F, const double* mass, const double* vol, double* gm, double* gmv,
               double* gf)
{
    return or_p2g_mat(c, n, x, v, B, F, mass, vol, NULL, NULL, gm, gmv, gf);
}

/* ------------------------------------------------------------------ */
/* Sec. 3.3: grid evolution, explicit member lambda = 0.               */
/* ------------------------------------------------------------------ */
/*
 * v_i = (m v)_i / m_i,  v~_i = v_i + dt f_i / m_i (+ dt g, sticky walls; not in paper).
 * Nodes with m_i = 0 get v_i = v~_i = 0.
 */
void or_grid_update(const or_cfg* c, const double* gm, const double* gmv, const double* gf,
                    double* gv, double* gvt)
{
    const int d = c->dim;
    const int64_t nn = node_count(c);
    for (int64_t idx = 0; idx < nn; ++idx) {
        int i[3] = {0, 0, 0};
        int64_t r = idx;
        for (int a = 0; a < d; ++a) { i[a] = (int)(r % c->res[a]); r /= c->res[a]; }
        if (gm[idx] <= 0.0) {
            for (int a = 0; a < d; ++a) { gv[idx * d + a] = 0.0; gvt[idx * d + a] = 0.0; }
            continue;
        }
        int wall = 0, inwall[3] = {0, 0, 0};
        for (int a = 0; a < d; ++a)
            if (i[a] < c->wall || i[a] >= c->res[a] - c->wall) { wall = 1; inwall[a] = 1; }
        for (int a = 0; a < d; ++a) {
            double vi = gmv[idx * d + a] / gm[idx];
            double vt = vi + c->dt * gf[idx * d + a] / gm[idx] + c->dt * c->gravity[a];
            gv[idx * d + a] = vi;
            if (c->boundary == 1 && wall) vt = 0.0;          /* sticky: the whole velocity */
            if (c->boundary == 2 && inwall[a]) vt = 0.0;     /* slip: the normal component */
            gvt[idx * d + a] = vt;
        }
    }
}

/* ------------------------------------------------------------------ */
/* Sec. 3.4: transfer to particles, general form.                      */
/* ------------------------------------------------------------------ */
/*
 * x~_i = x_i + dt (lambda v_i + (1 - lambda) v~_i)
 * v_p^{n+1} = sum_i w_ip v~_i
 * x_p^{n+1} = sum_i w_ip x~_i
 * B_p^{n+1} = 1/2 sum_i w_ip ( v~_i (x_i - x_p + x~_i - x_p^{n+1})^T
 *                              + (x_i - x_p - x~_i + x_p^{n+1}) v~_i^T )   (APIC)
 * B_p^{n+1} = 0                                                            (PIC)
 * F_p^{n+1} = (I + sum_i (x~_i - x_i) (grad w_ip)^T) F_p^n
 * FLIP (Sec. 1): the particle-to-grid transfer is PIC's, and the velocity is incremented by
 * the interpolated grid change, v_p + sum_i w_ip (v~_i - v_i); transfer 2 blends it with the
 * PIC velocity: v_p^{n+1} = alpha (v_p + sum_i w (v~_i - v_i)) + (1 - alpha) sum_i w v~_i,
 * B_p^{n+1} = 0 (v holds the particles' velocities on entry).
 * x, F updated in place; v, B written.  Returns the number of skipped particles.
 */
int64_t or_g2p(const or_cfg* c, int64_t n, double* x, double* v, double* B, double* F,
               const double* gv, const double* gvt)
{
    const int d = c->dim, ns = stencil_count(c);
    const double lt = c->lambda_t;
    int64_t bad = 0;
    double w[64], dw[192];
    for (int64_t p = 0; p < n; ++p) {
        double* xp = x + p * d;
        int base[3];
        if (or_stencil(c, xp, base, w, dw) != 0) { ++bad; continue; }
        double xn[3] = {0, 0, 0}, vn[3] = {0, 0, 0}, dv[3] = {0, 0, 0}, G[9] = {0};
        for (int j = 0; j < ns; ++j) {
            int i[3]; double xi[3];
            stencil_node(c, base, j, i, xi);
            int64_t ni = node_index(c, i);
            for (int a = 0; a < d; ++a) {
                double xt = xi[a] + c->dt * (lt * gv[ni * d + a] + (1.0 - lt) * gvt[ni * d + a]);
                xn[a] += w[j] * xt;
                vn[a] += w[j] * gvt[ni * d + a];
                dv[a] += w[j] * (gvt[ni * d + a] - gv[ni * d + a]);
                for (int b = 0; b < d; ++b) G[a * d + b] += (xt - xi[a]) * dw[j * d + b];
            }
        }
        if (c->transfer == 2)
            for (int a = 0; a < d; ++a)
                vn[a] = c->flip_alpha * (v[p * d + a] + dv[a]) + (1.0 - c->flip_alpha) * vn[a];
        double Bn[9] = {0};
        if (c->transfer == 0) {
            for (int j = 0; j < ns; ++j) {
                int i[3]; double xi[3], xt[3], vt[3];
                stencil_node(c, base, j, i, xi);
                int64_t ni = node_index(c, i);
                for (int a = 0; a < d; ++a) {
                    vt[a] = gvt[ni * d + a];
                    xt[a] = xi[a] + c->dt * (lt * gv[ni * d + a] + (1.0 - lt) * vt[a]);
                }
                for (int a = 0; a < d; ++a)
                    for (int b = 0; b < d; ++b) {
                        double t1 = vt[a] * (xi[b] - xp[b] + xt[b] - xn[b]);
                        double t2 = (xi[a] - xp[a] - xt[a] + xn[a]) * vt[b];
                        Bn[a * d + b] += 0.5 * w[j] * (t1 + t2);
                    }
            }
        }
        double Fo[9], M[9];
        memcpy(Fo, F + p * d * d, sizeof(double) * d * d);
        for (int a = 0; a < d; ++a)
            for (int b = 0; b < d; ++b) M[a * d + b] = (a == b ? 1.0 : 0.0) + G[a * d + b];
        matmul_d(d, M, Fo, F + p * d * d);
        for (int a = 0; a < d; ++a) { xp[a] = xn[a]; v[p * d + a] = vn[a]; }
        memcpy(B + p * d * d, Bn, sizeof(double) * d * d);
    }
    return bad;
}

/*
 * The lambda = 0 form the general transfer reduces to (Sec. 5.7):
 *   v_p = sum_i w_ip v~_i,  B_p = sum_i w_ip v~_i (x_i - x_p)^T,
 *   x_p^{n+1} = x_p + dt v_p^{n+1},  F_p^{n+1} = (I + dt sum_i v~_i (grad w_ip)^T) F_p.
 */
int64_t or_g2p_lambda0(const or_cfg* c, int64_t n, double* x, double* v, double* B, double* F,
                       const double* gvt)
{
    const int d = c->dim, ns = stencil_count(c);
    int64_t bad = 0;
    double w[64], dw[192];
    for (int64_t p = 0; p < n; ++p) {
        double* xp = x + p * d;
        int base[3];
        if (or_stencil(c, xp, base, w, dw) != 0) { ++bad; continue; }
        double vn[3] = {0, 0, 0}, Bn[9] = {0}, G[9] = {0};
        for (int j = 0; j < ns; ++j) {
            int i[3]; double xi[3];
            stencil_node(c, base, j, i, xi);
            int64_t ni = node_index(c, i);
            for (int a = 0; a < d; ++a) {
                double vt = gvt[ni * d + a];
                vn[a] += w[j] * vt;
                for (int b = 0; b < d; ++b) {
                    if (c->transfer == 0) Bn[a * d + b] += w[j] * vt * (xi[b] - xp[b]);
                    G[a * d + b] += vt * dw[j * d + b];
                }
            }
        }
        double Fo[9], M[9];
        memcpy(Fo, F + p * d * d, sizeof(double) * d * d);
        for (int a = 0; a < d; ++a)
            for (int b = 0; b < d; ++b) M[a * d + b] = (a == b ? 1.0 : 0.0) + c->dt * G[a * d + b];
        matmul_d(d, M, Fo, F + p * d * d);
        for (int a = 0; a < d; ++a) { v[p * d + a] = vn[a]; xp[a] += c->dt * vn[a]; }
        memcpy(B + p * d * d, Bn, sizeof(double) * d * d);
    }
    return bad;
}

/* ------------------------------------------------------------------ */
/* Potential energy Phi(x~) = sum_p V_p Psi(F^_p(x~)) (Sec. 3.3), for the  */
/* finite-difference check of the force.  dxg holds x~_i - x_i per node. */
/* ------------------------------------------------------------------ */
double or_potential(const or_cfg* c, int64_t n, const double* x, const double* F,
                    const double* vol, const double* dxg)
{
    const int d = c->dim, ns = stencil_count(c);
    double w[64], dw[192], phi = 0.0;
    for (int64_t p = 0; p < n; ++p) {
        int base[3];
        if (or_stencil(c, x + p * d, base, w, dw) != 0) continue;
        double M[9], Fh[9];
        for (int a = 0; a < d; ++a)
            for (int b = 0; b < d; ++b) M[a * d + b] = (a == b) ? 1.0 : 0.0;
        for (int j = 0; j < ns; ++j) {
            int i[3]; double xi[3];
            stencil_node(c, base, j, i, xi);
            int64_t ni = node_index(c, i);
            for (int a = 0; a < d; ++a)
                for (int b = 0; b < d; ++b) M[a * d + b] += dxg[ni * d + a] * dw[j * d + b];
        }
        matmul_d(d, M, F + p * d * d, Fh);
        phi += vol[p] * psi_of(c, Fh);
    }
    return phi;
}

/* ------------------------------------------------------------------ */
/* Sec. 3.3: force at a displaced grid, and the explicit member        */
/* lambda = 1.                                                          */
/* ------------------------------------------------------------------ */
/*
 * f_i = -sum_p V_p P(F^_p) (F_p^n)^T grad w_ip,  F^_p = (I + sum_i dxg_i (grad w_ip)^T) F_p^n,
 * with dxg_i = x~_i - x_i per node: the force of Sec. 3.3 with F^{n+lambda} = F^_p (sign
 * reading above).  It is -dPhi/dx~ for Phi(x~) = sum_p V_p Psi(F^_p(x~)) (or_potential).
 * dxg = 0 gives or_p2g's force (lambda = 0); dxg_i = dt v_i gives the member lambda = 1.
 * gf is accumulated into (callers zero it).  Returns the number of skipped particles.
 */
int64_t or_force_at(const or_cfg* c, int64_t n, const double* x, const double* F, const double* vol,
                    const double* dxg, double* gf)
{
    const int d = c->dim, ns = stencil_count(c);
    int64_t bad = 0;
    double w[64], dw[192];
    if (c->model == 0) return 0;
    for (int64_t p = 0; p < n; ++p) {
        int base[3];
        if (or_stencil(c, x + p * d, base, w, dw) != 0) { ++bad; continue; }
        const double* Fp = F + p * d * d;
        double M[9], Fh[9], P[9], A[9];
        for (int a = 0; a < d; ++a)
            for (int b = 0; b < d; ++b) M[a * d + b] = (a == b) ? 1.0 : 0.0;
        for (int j = 0; j < ns; ++j) {
            int i[3]; double xi[3];
            stencil_node(c, base, j, i, xi);
            int64_t ni = node_index(c, i);
            for (int a = 0; a < d; ++a)
                for (int b = 0; b < d; ++b) M[a * d + b] += dxg[ni * d + a] * dw[j * d + b];
        }
        matmul_d(d, M, Fp, Fh);
        stress_with(c, c->mu, c->lam, Fh, P);
        /* A = V_p P(F^) (F^n)^T */
        for (int a = 0; a < d; ++a)
            for (int b = 0; b < d; ++b) {
                double s = 0.0;
                for (int k = 0; k < d; ++k) s += P[a * d + k] * Fp[b * d + k];
                A[a * d + b] = vol[p] * s;
            }
        for (int j = 0; j < ns; ++j) {
            int i[3]; double xi[3];
            stencil_node(c, base, j, i, xi);
            int64_t ni = node_index(c, i);
            for (int a = 0; a < d; ++a) {
                double s = 0.0;
                for (int b = 0; b < d; ++b) s += A[a * d + b] * dw[j * d + b];
                gf[ni * d + a] -= s;
            }
        }
    }
    return bad;
}

/*
 * One explicit step of the member lambda = 1 of Sec. 3.3, in the paper's order:
 *   P2G of mass and momentum (Sec. 3.2), v_i = (m v)_i / m_i;
 *   x~_i = x_i + dt v_i (lambda = 1), so F_p^{n+1} = (I + dt sum_i v_i (grad w_ip)^T) F_p^n
 *   and the force f_i = -sum_p V_p P(F_p^{n+1}) (F_p^n)^T grad w_ip;
 *   v~_i = v_i + dt f_i / m_i (with gravity and walls as in or_grid_update);
 *   the general transfer to particles (Sec. 3.4) with lambda = 1.
 * Returns the number of skipped particles (-1 when memory runs out).
 */
int64_t or_step_lambda1(const or_cfg* c, int64_t n, double* x, double* v, double* B, double* F,
                        const double* mass, const double* vol)
{
    const int d = c->dim;
    const int64_t nn = node_count(c);
    double* gm = (double*)calloc((size_t)nn, sizeof(double));
    double* gmv = (double*)calloc((size_t)nn * d, sizeof(double));
    double* gf = (double*)calloc((size_t)nn * d, sizeof(double));
    double* gv = (double*)calloc((size_t)nn * d, sizeof(double));
    double* gvt = (double*)calloc((size_t)nn * d, sizeof(double));
    double* dxg = (double*)calloc((size_t)nn * d, sizeof(double));
    int64_t bad = -1;
    if (gm && gmv && gf && gv && gvt && dxg) {
        or_cfg c1 = *c;
        c1.lambda_t = 1.0;
        or_cfg c0 = c1;
        c0.model = 0;                                   /* mass and momentum only */
        bad = or_p2g(&c0, n, x, v, B, F, mass, vol, gm, gmv, gf);
        or_grid_update(&c1, gm, gmv, gf, gv, gvt);      /* gv = v_i (gf is zero here) */
        for (int64_t k = 0; k < nn * d; ++k) dxg[k] = c->dt * gv[k];
        bad += or_force_at(&c1, n, x, F, vol, dxg, gf);
        or_grid_update(&c1, gm, gmv, gf, gv, gvt);
        bad += or_g2p(&c1, n, x, v, B, F, gv, gvt);
    }
    free(gm); free(gmv); free(gf); free(gv); free(gvt); free(dxg);
    return bad;
}

/*
 * Force-derivative product of Sec. 3.3 at a displaced grid (F^_p as in or_force_at):
 *   A_p = dP/dF(F^_p) : ((sum_j du_j (grad w_jp)^T) F_p^n),
 *   df_i = -sum_p V_p A_p (F_p^n)^T grad w_ip  = sum_j (d f_i / d x~_j) du_j.
 * gdf is accumulated into (callers zero it).  Returns the number of skipped particles.
 */
int64_t or_force_diff_at(const or_cfg* c, int64_t n, const double* x, const double* F, const double* vol,
                         const double* dxg, const double* du, double* gdf)
{
    const int d = c->dim, ns = stencil_count(c);
    int64_t bad = 0;
    double w[64], dw[192];
    if (c->model == 0) return 0;
    for (int64_t p = 0; p < n; ++p) {
        int base[3];
        if (or_stencil(c, x + p * d, base, w, dw) != 0) { ++bad; continue; }
        const double* Fp = F + p * d * d;
        double M[9], D[9], Fh[9], dFh[9], dP[9], A[9];
        for (int a = 0; a < d; ++a)
            for (int b = 0; b < d; ++b) { M[a * d + b] = (a == b) ? 1.0 : 0.0; D[a * d + b] = 0.0; }
        for (int j = 0; j < ns; ++j) {
            int i[3]; double xi[3];
            stencil_node(c, base, j, i, xi);
            int64_t ni = node_index(c, i);
            for (int a = 0; a < d; ++a)
                for (int b = 0; b < d; ++b) {
                    M[a * d + b] += dxg[ni * d + a] * dw[j * d + b];
                    D[a * d + b] += du[ni * d + a] * dw[j * d + b];
                }
        }
        matmul_d(d, M, Fp, Fh);
        matmul_d(d, D, Fp, dFh);
        dstress_with(c, Fh, dFh, dP);
        for (int a = 0; a < d; ++a)
            for (int b = 0; b < d; ++b) {
                double s = 0.0;
                for (int k = 0; k < d; ++k) s += dP[a * d + k] * Fp[b * d + k];
                A[a * d + b] = vol[p] * s;
            }
        for (int j = 0; j < ns; ++j) {
            int i[3]; double xi[3];
            stencil_node(c, base, j, i, xi);
            int64_t ni = node_index(c, i);
            for (int a = 0; a < d; ++a) {
                double s = 0.0;
                for (int b = 0; b < d; ++b) s += A[a * d + b] * dw[j * d + b];
                gdf[ni * d + a] -= s;
            }
        }
    }
    return bad;
}

/* <u, v>_M = sum_i m_i u_i . v_i over the nodes with mass */
static double dot_m(int64_t nn, int d, const double* gm, const double* u, const double* v)
{
    double s = 0.0;
    for (int64_t i = 0; i < nn; ++i)
        if (gm[i] > 0.0)
            for (int a = 0; a < d; ++a) s += gm[i] * u[i * d + a] * v[i * d + a];
    return s;
}

/*
 * The grid solve of the implicit midpoint rule (lambda = 1/2), as Sec. 4.1-4.2 do it:
 * Newton iterations on dv = v~ - v for  m_i dv_i = dt f_i(x_i + dt/2 v_i + dt/4 dv_i)
 * (F^{n+1/2} is F^ of or_force_at at the displacement dt/2 v + dt/4 dv), the gradient of the
 * objective being g_i = m_i/4 dv_i - dt/4 f_i; each Newton system (M/4 - dt^2/16 df/dx) du = -g
 * solved by conjugate gradients (Algorithm 1) on its velocity-like form
 * (I - dt^2/4 M^{-1} df/dx) du = -4 M^{-1} g with the mass inner product <u, v> = u^T M v,
 * from du = 0.  Only nodes with mass carry unknowns (dv = 0 elsewhere).  newton, cg:
 * iteration caps; the Newton loop ends when |4 M^{-1} g|_M <= tol max(|v|_M, tiny), a CG
 * solve when |r|_M <= tol |r_0|_M.  gv: v_i; dv: in (start) and out.  Returns the Newton
 * iterations taken, or -1 when memory runs out.
 */
int or_midpoint_solve(const or_cfg* c, int64_t n, const double* x, const double* F, const double* vol,
                      const double* gm, const double* gv, int newton, int cg, double tol, double* dv)
{
    const int d = c->dim;
    const int64_t nn = node_count(c), nv = nn * d;
    double* dxg = (double*)calloc((size_t)nv, sizeof(double));
    double* f = (double*)calloc((size_t)nv, sizeof(double));
    double* r = (double*)calloc((size_t)nv, sizeof(double));
    double* pd = (double*)calloc((size_t)nv, sizeof(double));
    double* sv = (double*)calloc((size_t)nv, sizeof(double));
    double* du = (double*)calloc((size_t)nv, sizeof(double));
    int it = -1;
    if (dxg && f && r && pd && sv && du) {
        const double vnorm = sqrt(dot_m(nn, d, gm, gv, gv));
        const double dt = c->dt;
        for (it = 0; it < newton; ++it) {
            for (int64_t k = 0; k < nv; ++k) { dxg[k] = 0.5 * dt * gv[k] + 0.25 * dt * dv[k]; f[k] = 0.0; }
            or_force_at(c, n, x, F, vol, dxg, f);
            /* r = -4 M^{-1} g = dt M^{-1} f - dv */
            for (int64_t i = 0; i < nn; ++i)
                for (int a = 0; a < d; ++a)
                    r[i * d + a] = gm[i] > 0.0 ? dt * f[i * d + a] / gm[i] - dv[i * d + a] : 0.0;
            const double rn0 = sqrt(dot_m(nn, d, gm, r, r));
            if (rn0 <= tol * (vnorm > 1e-300 ? vnorm : 1e-300)) break;
            /* Algorithm 1 on A2 du = r, du = 0 */
            for (int64_t k = 0; k < nv; ++k) { du[k] = 0.0; pd[k] = r[k]; }
            double gamma = rn0 * rn0;
            for (int k = 0; k < cg && gamma > 0.0; ++k) {
                for (int64_t q = 0; q < nv; ++q) sv[q] = 0.0;
                or_force_diff_at(c, n, x, F, vol, dxg, pd, sv);            /* df/dx p */
                for (int64_t i = 0; i < nn; ++i)
                    for (int a = 0; a < d; ++a) {
                        const int64_t q = i * d + a;
                        sv[q] = gm[i] > 0.0 ? pd[q] - 0.25 * dt * dt * sv[q] / gm[i] : 0.0;   /* s = A2 p */
                    }
                const double ps = dot_m(nn, d, gm, pd, sv);
                if (!(ps > 0.0)) break;
                const double alpha = gamma / ps;
                for (int64_t q = 0; q < nv; ++q) { du[q] += alpha * pd[q]; r[q] -= alpha * sv[q]; }
                const double kappa = dot_m(nn, d, gm, r, r);
                if (sqrt(kappa) <= tol * rn0) break;
                const double beta = kappa / gamma;
                for (int64_t q = 0; q < nv; ++q) pd[q] = r[q] + beta * pd[q];
                gamma = kappa;
            }
            for (int64_t q = 0; q < nv; ++q) dv[q] += du[q];
        }
    }
    free(dxg); free(f); free(r); free(pd); free(sv); free(du);
    return it;
}

/*
 * One step of the implicit midpoint rule: P2G of mass and momentum, v_i = (m v)_i / m_i,
 * the grid solve above from dv = 0, v~ = v + dv, and the general transfer to particles with
 * lambda = 1/2.  Gravity and walls are not applied (neither is in the paper).  Returns the
 * number of skipped particles (-1 when memory runs out).
 */
int64_t or_step_midpoint(const or_cfg* c, int64_t n, double* x, double* v, double* B, double* F,
                         const double* mass, const double* vol, int newton, int cg, double tol)
{
    const int d = c->dim;
    const int64_t nn = node_count(c), nv = nn * d;
    double* gm = (double*)calloc((size_t)nn, sizeof(double));
    double* gmv = (double*)calloc((size_t)nv, sizeof(double));
    double* gv = (double*)calloc((size_t)nv, sizeof(double));
    double* gvt = (double*)calloc((size_t)nv, sizeof(double));
    double* dv = (double*)calloc((size_t)nv, sizeof(double));
    double* f = (double*)calloc((size_t)nv, sizeof(double));
    int64_t bad = -1;
    if (gm && gmv && gv && gvt && dv && f) {
        or_cfg ch = *c;
        ch.lambda_t = 0.5;
        ch.boundary = 0;
        for (int a = 0; a < 3; ++a) ch.gravity[a] = 0.0;
        or_cfg c0 = ch;
        c0.model = 0;                                   /* mass and momentum only */
        bad = or_p2g(&c0, n, x, v, B, F, mass, vol, gm, gmv, f);
        for (int64_t i = 0; i < nn; ++i)
            for (int a = 0; a < d; ++a) gv[i * d + a] = gm[i] > 0.0 ? gmv[i * d + a] / gm[i] : 0.0;
        if (or_midpoint_solve(&ch, n, x, F, vol, gm, gv, newton, cg, tol, dv) < 0) bad = -1;
        for (int64_t q = 0; q < nv; ++q) gvt[q] = gv[q] + dv[q];
        if (bad >= 0) bad += or_g2p(&ch, n, x, v, B, F, gv, gvt);
    }
    free(gm); free(gmv); free(gv); free(gvt); free(dv); free(f);
    return bad;
}

/* ------------------------------------------------------------------ */
/* Sec. 3.1 / 5.3: total linear and angular momentum.                  */
/* ------------------------------------------------------------------ */
/*
 * Particles: p = sum m_p v_p;  l = sum x_p x m_p v_p + m_p (B_p)^T : eps
 * ((B^T):eps = (B_21 - B_12, B_02 - B_20, B_10 - B_01); in 2-D only the z entry).
 * In 2-D, l[0] holds the scalar z component and l[1] = l[2] = 0.
 */
void or_momentum_particles(const or_cfg* c, int64_t n, const double* x, const double* v,
                           const double* B, const double* mass, double* p, double* l)
{
    const int d = c->dim;
    for (int a = 0; a < 3; ++a) { p[a] = 0.0; l[a] = 0.0; }
    for (int64_t q = 0; q < n; ++q) {
        const double* xp = x + q * d;
        const double* vp = v + q * d;
        const double* Bp = B + q * d * d;
        double m = mass[q];
        for (int a = 0; a < d; ++a) p[a] += m * vp[a];
        if (d == 2) {
            l[0] += m * (xp[0] * vp[1] - xp[1] * vp[0]);
            if (c->transfer == 0) l[0] += m * (Bp[2] - Bp[1]);
        } else {
            l[0] += m * (xp[1] * vp[2] - xp[2] * vp[1]);
            l[1] += m * (xp[2] * vp[0] - xp[0] * vp[2]);
            l[2] += m * (xp[0] * vp[1] - xp[1] * vp[0]);
            if (c->transfer == 0) {
                l[0] += m * (Bp[7] - Bp[5]);
                l[1] += m * (Bp[2] - Bp[6]);
                l[2] += m * (Bp[3] - Bp[1]);
            }
        }
    }
}

/* Grid: p = sum_i (m v)_i,  l = sum_i x_i x (m v)_i (Sec. 5.1 / 5.3). */
void or_momentum_grid(const or_cfg* c, const double* gmv, double* p, double* l)
{
    const int d = c->dim;
    const int64_t nn = node_count(c);
    for (int a = 0; a < 3; ++a) { p[a] = 0.0; l[a] = 0.0; }
    for (int64_t idx = 0; idx < nn; ++idx) {
        int i[3] = {0, 0, 0};
        int64_t r = idx;
        double xi[3];
        for (int a = 0; a < d; ++a) {
            i[a] = (int)(r % c->res[a]); r /= c->res[a];
            xi[a] = c->origin[a] + i[a] * c->dx;
        }
        const double* q = gmv + idx * d;
        for (int a = 0; a < d; ++a) p[a] += q[a];
        if (d == 2) {
            l[0] += xi[0] * q[1] - xi[1] * q[0];
        } else {
            l[0] += xi[1] * q[2] - xi[2] * q[1];
            l[1] += xi[2] * q[0] - xi[0] * q[2];
            l[2] += xi[0] * q[1] - xi[1] * q[0];
        }
    }
}

/* ------------------------------------------------------------------ */
/* Sec. 4.3: time-step bound dt <= nu dx / max_p (|v_p| + (kappa/k) dx |B_p|_F), where    */
/* |x_i - x_p| <= kappa dx over the stencil and D_p = k I.                              */
/* ------------------------------------------------------------------ */
double or_cfl_speed(const or_cfg* c, int64_t n, const double* v, const double* B)
{
    const int d = c->dim;
    const double kappa = (c->order == 2 ? 1.5 : 2.0) * sqrt((double)d);
    const double k = (c->order == 2 ? 0.25 : 1.0 / 3.0) * c->dx * c->dx;
    const double coef = kappa * c->dx / k;      /* (kappa / k) dx */
    double mx = 0.0;
    for (int64_t p = 0; p < n; ++p) {
        double sv = 0.0, sb = 0.0;
        for (int a = 0; a < d; ++a) sv += v[p * d + a] * v[p * d + a];
        for (int a = 0; a < d * d; ++a) sb += B[p * d * d + a] * B[p * d * d + a];
        double s = sqrt(sv) + coef * sqrt(sb);
        if (s > mx) mx = s;
    }
    return mx;
}

/* ------------------------------------------------------------------ */
/* Cell keys and the stable sort by key.                                */
/* ------------------------------------------------------------------ */
/*
 * Key of a particle given as integer cell index plus offset in [0,1) per axis:
 * the stencil base node b (quadratic: cell - 1 if offset < 1/2 else cell;
 * cubic: cell - 1), then block = b / E (E = block edge, a power of two),
 * in-block cell = b mod E, key = linear(block) << (d log2 E) | linear(in-block),
 * both linearised with axis 0 fastest.  Blocks per axis = ceil(res / E).
 */
void or_keys(const or_cfg* c, int block_edge, int64_t n, const int32_t* cell, const double* off,
             uint32_t* keys)
{
    const int d = c->dim;
    int lg = 0;
    while ((1 << lg) < block_edge) ++lg;
    for (int64_t p = 0; p < n; ++p) {
        uint32_t blk = 0, in = 0, mult_b = 1, mult_i = 1;
        for (int a = 0; a < d; ++a) {
            int b = cell[p * d + a] - 1;
            if (c->order == 2 && off[p * d + a] >= 0.5) b = cell[p * d + a];
            int nb = (c->res[a] + block_edge - 1) / block_edge;
            blk += (uint32_t)(b / block_edge) * mult_b;
            in += (uint32_t)(b % block_edge) * mult_i;
            mult_b *= (uint32_t)nb;
            mult_i *= (uint32_t)block_edge;
        }
        keys[p] = (blk << (d * lg)) | in;
    }
}

typedef struct { uint32_t key; int64_t idx; } key_idx;
static int cmp_key_idx(const void* a, const void* b)
{
    const key_idx* x = (const key_idx*)a;
    const key_idx* y = (const key_idx*)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    if (x->idx != y->idx) return x->idx < y->idx ? -1 : 1;
    return 0;
}

/* Stable sort: order by (key, original index); perm[k] = index of the k-th particle. */
void or_stable_sort(int64_t n, const uint32_t* keys, int64_t* perm)
{
    key_idx* t = (key_idx*)malloc(sizeof(key_idx) * (n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) { t[i].key = keys[i]; t[i].idx = i; }
    qsort(t, (size_t)n, sizeof(key_idx), cmp_key_idx);
    for (int64_t i = 0; i < n; ++i) perm[i] = t[i].idx;
    free(t);
}

/* ------------------------------------------------------------------ */
/* One whole explicit step: P2G, grid update, G2P (general form).       */
/* ------------------------------------------------------------------ */
int64_t or_step_mat(const or_cfg* c, int64_t n, double* x, double* v, double* B, double* F,
                    const double* mass, const double* vol, const double* mu_p, const double* lam_p)
{
    const int d = c->dim;
    const int64_t nn = node_count(c);
    double* gm = (double*)calloc((size_t)nn, sizeof(double));
    double* gmv = (double*)calloc((size_t)nn * d, sizeof(double));
    double* gf = (double*)calloc((size_t)nn * d, sizeof(double));
    double* gv = (double*)calloc((size_t)nn * d, sizeof(double));
    double* gvt = (double*)calloc((size_t)nn * d, sizeof(double));
    int64_t bad = -1;
    if (gm && gmv && gf && gv && gvt) {
        bad = or_p2g_mat(c, n, x, v, B, F, mass, vol, mu_p, lam_p, gm, gmv, gf);
        or_grid_update(c, gm, gmv, gf, gv, gvt);
        bad += or_g2p(c, n, x, v, B, F, gv, gvt);
    }
    free(gm); free(gmv); free(gf); free(gv); free(gvt);
    return bad;
}

int64_t or_step(const or_cfg* c, int64_t n, double* x, double* v, double* B, double* F,
                const double* mass, const double* vol)
{
    return or_step_mat(c, n, x, v, B, F, mass, vol, NULL, NULL);
}
