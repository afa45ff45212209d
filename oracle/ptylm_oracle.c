/*
 * ptylm_oracle.c -- plain FP64 CPU oracle for the matrix-free Levenberg-Marquardt
 * ptychography method of arXiv 2103.01767 ("A matrix-free Levenberg-Marquardt
 * algorithm for efficient ptychographic phase retrieval").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct reference that
 * the CUDA library is checked against.  It shares no code, header, table or helper
 * with the CUDA path.  Only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark may load it; the product path never does.
 *
 * Every function restates one step of the paper in the paper's order:
 *   exit wave            psi_k = diag(P) S_k O                        (Sec. 2, Eq. exit_wave)
 *   far field            psihat_k = F psi_k, h_k = |psihat_k|^2 + b_k  (Sec. 2, Eq. expected_count)
 *   magnitude            zeta = h^(1/2)                                 (Sec. 4.1, Eq. magnitude)
 *   error metric         l_p = zeta^2 - y log zeta^2, l_g = (zeta-sqrt y)^2/2
 *                                                                      (Sec. 4.1, Eq. ell_magnitude)
 *   Jacobian             J = diag(psihat/zeta) F^* diag(P^*) S_k  (real-coordinate form of
 *                                                                      App. B, Eq. jac_ampl)
 *   GGN-vector product   J^T (Hess_zeta l) J v + lambda D v           (App. A, Eq. ggn_magnitude_appendix_2)
 *   GGN diagonal         (1/(4M)) sum_k tr(Hess_k l) Dg(S_k^T |P|^2 S_k)  (App. B, Eq. ggn_diag_mat)
 *   truncated CG + LM    Algorithm 1 with the stopping rule Eqs. lma_termination_magnitude/eta
 *
 * Conventions (readings of the paper where it is silent):
 *   - F is the orthonormal 2D DFT, forward sign -1 (App. B's [C_k]_11 = trace/M needs a
 *     unitary F).
 *   - Vectors over C^n stand for real coordinates [Re; Im] (Sec. 3); the inner product is
 *     Re sum conj(a) b and gradients are d/dRe + i d/dIm (twice the Wirtinger form of App. B).
 *   - Poisson curvature is the exact second derivative of l_p as written: 2 + 2 y / zeta^2.
 *   - eta = min(beta, sqrt(||grad f||)) (the printed J * grad l has no matching shape).
 *   - predicted reduction = -(g^T d + d^T G d / 2), evaluated with the CG residual.
 *   - a rejected step (rho <= rho_min) multiplies mu by kappa and re-solves.
 *   - lambda = mu ||grad_zeta l||^nu when D = I, lambda = mu when D = Dg(G).
 *
 * Parity pins: each function is checked in the CPU test-suite against invariants that
 * hold independently of this code (adjoint identity, finite differences, Parseval,
 * direct DFT, dense brute force on tiny sizes, zero loss/gradient at a noiseless truth);
 * Algorithm 1 against a dense restatement step for step (error metric, gain ratio, mu,
 * iterate) with its CG run to convergence; truncated CG against the forcing bound with
 * the dense G, and the forcing term eta of Algorithm 1 through its CG iteration counts.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double _Complex dc;

typedef struct {
    int ny, nx;      /* object rows, columns */
    int my, mx;      /* probe / detector rows, columns */
    int K;           /* number of scan positions */
    int loss;        /* 0 = Gaussian (amplitude) metric, 1 = Poisson metric */
    double b;        /* incoherent background per detector pixel (> 0) */
} orc_geom;

#define ORC_PI 3.14159265358979323846264338327950288

/* ------------------------------------------------------------------------------------
 * Discrete Fourier transforms.  Orthonormal: X[u] = M^{-1/2} sum_m x[m] e^{sign 2 pi i u.m/M}.
 * ------------------------------------------------------------------------------------ */

/* Direct O(M^2) 2D DFT, the textbook definition.  sign = -1 forward, +1 inverse. */
void orc_dft2(const dc* x, dc* X, int my, int mx, int sign)
{
    const double scale = 1.0 / sqrt((double)my * (double)mx);
    for (int uy = 0; uy < my; ++uy)
        for (int ux = 0; ux < mx; ++ux) {
            dc acc = 0.0;
            for (int yy = 0; yy < my; ++yy)
                for (int xx = 0; xx < mx; ++xx) {
                    double ph = 2.0 * ORC_PI *
                        ((double)((long)uy * yy % my) / my + (double)((long)ux * xx % mx) / mx);
                    acc += x[yy * mx + xx] * cexp(I * (double)sign * ph);
                }
            X[uy * mx + ux] = acc * scale;
        }
}

static int is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

/* Iterative radix-2 Cooley-Tukey on a strided 1D sequence (unnormalised). */
static void fft1d(dc* a, int n, int stride, int sign, dc* tmp)
{
    for (int i = 0; i < n; ++i) tmp[i] = a[(long)i * stride];
    /* bit-reversal permutation */
    for (int i = 1, j = 0; i < n; ++i) {
        int bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) { dc t = tmp[i]; tmp[i] = tmp[j]; tmp[j] = t; }
    }
    for (int len = 2; len <= n; len <<= 1) {
        for (int i = 0; i < n; i += len)
            for (int k = 0; k < len / 2; ++k) {
                dc w = cexp(I * (double)sign * 2.0 * ORC_PI * (double)k / (double)len);
                dc u = tmp[i + k], v = tmp[i + k + len / 2] * w;
                tmp[i + k] = u + v;
                tmp[i + k + len / 2] = u - v;
            }
    }
    for (int i = 0; i < n; ++i) a[(long)i * stride] = tmp[i];
}

/* In-place orthonormal 2D FFT (rows, then columns).  Requires power-of-two sides. */
int orc_fft2(dc* x, int my, int mx, int sign)
{
    if (!is_pow2(my) || !is_pow2(mx)) return 1;
    int nmax = my > mx ? my : mx;
    dc* tmp = (dc*)malloc(sizeof(dc) * nmax);
    for (int r = 0; r < my; ++r) fft1d(x + (long)r * mx, mx, 1, sign, tmp);
    for (int c = 0; c < mx; ++c) fft1d(x + c, my, mx, sign, tmp);
    free(tmp);
    const double scale = 1.0 / sqrt((double)my * (double)mx);
    for (long i = 0; i < (long)my * mx; ++i) x[i] *= scale;
    return 0;
}

/* The transform the model uses: direct DFT on tiny grids, FFT otherwise. */
static void transform(dc* x, int my, int mx, int sign, dc* scratch)
{
    if ((long)my * mx <= 256 || !is_pow2(my) || !is_pow2(mx)) {
        orc_dft2(x, scratch, my, mx, sign);
        memcpy(x, scratch, sizeof(dc) * (size_t)my * mx);
    } else {
        orc_fft2(x, my, mx, sign);
    }
}

/* ------------------------------------------------------------------------------------
 * Forward model, Sec. 2: psi_k = diag(P) S_k O  (Eq. exit_wave),
 * psihat_k = F psi_k, h_k = |psihat_k|^2 + b  (Eq. expected_count).
 * ------------------------------------------------------------------------------------ */

/* S_k O: the M-pixel patch of O whose top-left corner is (pos[2k], pos[2k+1]). */
static void gather_patch(const orc_geom* g, const dc* O, const int32_t* pos, int k, dc* out)
{
    int r0 = pos[2 * k], c0 = pos[2 * k + 1];
    for (int yy = 0; yy < g->my; ++yy)
        for (int xx = 0; xx < g->mx; ++xx)
            out[yy * g->mx + xx] = O[(long)(r0 + yy) * g->nx + (c0 + xx)];
}

/* psihat_k (length M) for position k. */
static void exit_wave_far_field(const orc_geom* g, const dc* O, const dc* P, const int32_t* pos,
                                int k, dc* psihat, dc* scratch)
{
    const int M = g->my * g->mx;
    gather_patch(g, O, pos, k, psihat);
    for (int m = 0; m < M; ++m) psihat[m] *= P[m];
    transform(psihat, g->my, g->mx, -1, scratch);
}

/* Public: psihat [K][M] and h [K][M]. */
void orc_forward(const orc_geom* g, const dc* O, const dc* P, const int32_t* pos,
                 dc* psihat_out, double* h_out)
{
    const int M = g->my * g->mx;
#pragma omp parallel
    {
        dc* scratch = (dc*)malloc(sizeof(dc) * M);
#pragma omp for schedule(static)
        for (int k = 0; k < g->K; ++k) {
            dc* ph = psihat_out + (long)k * M;
            exit_wave_far_field(g, O, P, pos, k, ph, scratch);
            for (int m = 0; m < M; ++m) {
                double a = cabs(ph[m]);
                h_out[(long)k * M + m] = a * a + g->b;
            }
        }
        free(scratch);
    }
}

/* ------------------------------------------------------------------------------------
 * Error metric, Sec. 4.1 Eq. ell_magnitude, and its derivatives with respect to zeta.
 *   Gaussian: l = (zeta - sqrt y)^2 / 2,  dl = zeta - sqrt y,  d2l = 1
 *   Poisson:  l = zeta^2 - y log zeta^2,  dl = 2 zeta - 2 y / zeta,  d2l = 2 + 2 y / zeta^2
 * (0 log 0 taken as 0.)
 * ------------------------------------------------------------------------------------ */
static double ell(int loss, double zeta, double y)
{
    if (loss == 0) {
        double d = zeta - sqrt(y);
        return 0.5 * d * d;
    }
    double h = zeta * zeta;
    return h - (y > 0.0 ? y * log(h) : 0.0);
}

static double dell(int loss, double zeta, double y)
{
    return loss == 0 ? zeta - sqrt(y) : 2.0 * zeta - 2.0 * y / zeta;
}

static double d2ell(int loss, double zeta, double y)
{
    return loss == 0 ? 1.0 : 2.0 + 2.0 * y / (zeta * zeta);
}

/* Public per-element derivative table (used by tests to pin the closed forms). */
void orc_ell_terms(int loss, long n, const double* zeta, const double* y,
                   double* l, double* dl, double* d2l)
{
    for (long i = 0; i < n; ++i) {
        if (l) l[i] = ell(loss, zeta[i], y[i]);
        if (dl) dl[i] = dell(loss, zeta[i], y[i]);
        if (d2l) d2l[i] = d2ell(loss, zeta[i], y[i]);
    }
}

/* f = sum_k sum_m l(zeta_km, y_km)  (Eq. error_metric_magnitude).
 * Also returns ||grad_zeta l||^2 (needed for lambda in Algorithm 1). */
double orc_loss(const orc_geom* g, const dc* O, const dc* P, const int32_t* pos, const double* y,
                double* dl_norm2_out)
{
    const int M = g->my * g->mx;
    double* per_k = (double*)calloc((size_t)g->K * 2, sizeof(double));
#pragma omp parallel
    {
        dc* ph = (dc*)malloc(sizeof(dc) * M);
        dc* scratch = (dc*)malloc(sizeof(dc) * M);
#pragma omp for schedule(static)
        for (int k = 0; k < g->K; ++k) {
            exit_wave_far_field(g, O, P, pos, k, ph, scratch);
            double s = 0.0, s2 = 0.0;
            for (int m = 0; m < M; ++m) {
                double a = cabs(ph[m]);
                double zeta = sqrt(a * a + g->b);
                double yy = y[(long)k * M + m];
                s += ell(g->loss, zeta, yy);
                double d = dell(g->loss, zeta, yy);
                s2 += d * d;
            }
            per_k[2 * k] = s;
            per_k[2 * k + 1] = s2;
        }
        free(ph);
        free(scratch);
    }
    double f = 0.0, n2 = 0.0;
    for (int k = 0; k < g->K; ++k) { f += per_k[2 * k]; n2 += per_k[2 * k + 1]; }
    free(per_k);
    if (dl_norm2_out) *dl_norm2_out = n2;
    return f;
}

/* ------------------------------------------------------------------------------------
 * Jacobian products (real coordinates), from App. B Eq. jac_ampl:
 *   J v  = Re( conj(psihat) . F( P . S_k vO  +  vP . S_k O ) ) / zeta
 *   J^T w = ( sum_k S_k^T [ conj(P) . F^H(psihat w / zeta) ],
 *             sum_k        conj(S_k O) . F^H(psihat w / zeta) )
 * vP / outP may be NULL (object-only problem).
 * ------------------------------------------------------------------------------------ */
void orc_jvp(const orc_geom* g, const dc* O, const dc* P, const int32_t* pos,
             const dc* vO, const dc* vP, double* out)
{
    const int M = g->my * g->mx;
#pragma omp parallel
    {
        dc* ph = (dc*)malloc(sizeof(dc) * M);
        dc* dv = (dc*)malloc(sizeof(dc) * M);
        dc* ok = (dc*)malloc(sizeof(dc) * M);
        dc* scratch = (dc*)malloc(sizeof(dc) * M);
#pragma omp for schedule(static)
        for (int k = 0; k < g->K; ++k) {
            exit_wave_far_field(g, O, P, pos, k, ph, scratch);
            gather_patch(g, vO, pos, k, dv);
            for (int m = 0; m < M; ++m) dv[m] *= P[m];
            if (vP) {
                gather_patch(g, O, pos, k, ok);
                for (int m = 0; m < M; ++m) dv[m] += vP[m] * ok[m];
            }
            transform(dv, g->my, g->mx, -1, scratch);
            for (int m = 0; m < M; ++m) {
                double a = cabs(ph[m]);
                double zeta = sqrt(a * a + g->b);
                out[(long)k * M + m] = creal(conj(ph[m]) * dv[m]) / zeta;
            }
        }
        free(ph); free(dv); free(ok); free(scratch);
    }
}

/* chi_k = F^H(psihat_k w_k / zeta_k) for every k, stored [K][M]. */
static void adjoint_waves(const orc_geom* g, const dc* O, const dc* P, const int32_t* pos,
                          const double* w, dc* chi)
{
    const int M = g->my * g->mx;
#pragma omp parallel
    {
        dc* scratch = (dc*)malloc(sizeof(dc) * M);
#pragma omp for schedule(static)
        for (int k = 0; k < g->K; ++k) {
            dc* c = chi + (long)k * M;
            exit_wave_far_field(g, O, P, pos, k, c, scratch);
            for (int m = 0; m < M; ++m) {
                double a = cabs(c[m]);
                double zeta = sqrt(a * a + g->b);
                c[m] = c[m] * (w[(long)k * M + m] / zeta);
            }
            transform(c, g->my, g->mx, +1, scratch);
        }
        free(scratch);
    }
}

/* Sum over k of S_k^T(conj(P) chi_k) and of conj(S_k O) chi_k, in position order. */
static void adjoint_scatter(const orc_geom* g, const dc* O, const dc* P, const int32_t* pos,
                            const dc* chi, dc* outO, dc* outP)
{
    const int M = g->my * g->mx;
    const long N = (long)g->ny * g->nx;
    if (outO) for (long n = 0; n < N; ++n) outO[n] = 0.0;
    if (outP) for (int m = 0; m < M; ++m) outP[m] = 0.0;
    for (int k = 0; k < g->K; ++k) {
        int r0 = pos[2 * k], c0 = pos[2 * k + 1];
        const dc* c = chi + (long)k * M;
        for (int yy = 0; yy < g->my; ++yy)
            for (int xx = 0; xx < g->mx; ++xx) {
                int m = yy * g->mx + xx;
                long n = (long)(r0 + yy) * g->nx + (c0 + xx);
                if (outO) outO[n] += conj(P[m]) * c[m];
                if (outP) outP[m] += conj(O[n]) * c[m];
            }
    }
}

void orc_jtvp(const orc_geom* g, const dc* O, const dc* P, const int32_t* pos,
              const double* w, dc* outO, dc* outP)
{
    const int M = g->my * g->mx;
    dc* chi = (dc*)malloc(sizeof(dc) * (size_t)g->K * M);
    adjoint_waves(g, O, P, pos, w, chi);
    adjoint_scatter(g, O, P, pos, chi, outO, outP);
    free(chi);
}

/* grad f = J^T grad_zeta l  (App. A step 1). */
void orc_gradient(const orc_geom* g, const dc* O, const dc* P, const int32_t* pos,
                  const double* y, dc* gO, dc* gP)
{
    const int M = g->my * g->mx;
    const long KM = (long)g->K * M;
    dc* ph = (dc*)malloc(sizeof(dc) * KM);
    double* h = (double*)malloc(sizeof(double) * KM);
    double* w = (double*)malloc(sizeof(double) * KM);
    orc_forward(g, O, P, pos, ph, h);
    for (long j = 0; j < KM; ++j) w[j] = dell(g->loss, sqrt(h[j]), y[j]);
    orc_jtvp(g, O, P, pos, w, gO, gP);
    free(ph); free(h); free(w);
}

/* GGN.v + lambda D v = J^T( Hess_zeta l . (J v) ) + lambda D v
 * (App. A steps 2-4, Eq. ggn_magnitude_appendix_2, with the closed-form diagonal Hessian
 * of step 3(ii)).  D_O / D_P NULL means the identity. */
void orc_ggn_matvec(const orc_geom* g, const dc* O, const dc* P, const int32_t* pos,
                    const double* y, const dc* vO, const dc* vP, double lambda,
                    const double* D_O, const double* D_P, dc* outO, dc* outP)
{
    const int M = g->my * g->mx;
    const long KM = (long)g->K * M;
    const long N = (long)g->ny * g->nx;
    double* jv = (double*)malloc(sizeof(double) * KM);
    dc* ph = (dc*)malloc(sizeof(dc) * KM);
    double* h = (double*)malloc(sizeof(double) * KM);
    orc_jvp(g, O, P, pos, vO, vP, jv);                       /* step 2: J v            */
    orc_forward(g, O, P, pos, ph, h);
    for (long j = 0; j < KM; ++j)                            /* step 3: Hess_zeta l . Jv */
        jv[j] *= d2ell(g->loss, sqrt(h[j]), y[j]);
    orc_jtvp(g, O, P, pos, jv, outO, vP ? outP : NULL);      /* step 4: J^T(...)       */
    for (long n = 0; n < N; ++n) outO[n] += lambda * (D_O ? D_O[n] : 1.0) * vO[n];
    if (vP && outP)
        for (int m = 0; m < M; ++m) outP[m] += lambda * (D_P ? D_P[m] : 1.0) * vP[m];
    free(jv); free(ph); free(h);
}

/* ------------------------------------------------------------------------------------
 * Diagonal of the GGN in real coordinates, App. B Eqs. ggn_diag_elem_final / ggn_diag_mat
 * / ggn_joint_diag, converted from the Wirtinger block 1/(4M) to real coordinates:
 *   D_O[n] = (1/(2M)) sum_{k: n in patch k} |P[n - r_k]|^2 tr_k
 *   D_P[m] = (1/(2M)) sum_k |O[r_k + m]|^2 tr_k,      tr_k = sum_m Hess_zeta l_km
 * (the paper's h ~ |psihat|^2 approximation).  Values below floor_rel * max are raised to
 * that floor so unilluminated pixels stay invertible.
 * ------------------------------------------------------------------------------------ */
void orc_ggn_diag(const orc_geom* g, const dc* O, const dc* P, const int32_t* pos,
                  const double* y, double floor_rel, double* D_O, double* D_P)
{
    const int M = g->my * g->mx;
    const long N = (long)g->ny * g->nx;
    const long KM = (long)g->K * M;
    dc* ph = (dc*)malloc(sizeof(dc) * KM);
    double* h = (double*)malloc(sizeof(double) * KM);
    double* tr = (double*)calloc((size_t)g->K, sizeof(double));
    orc_forward(g, O, P, pos, ph, h);
    for (int k = 0; k < g->K; ++k)
        for (int m = 0; m < M; ++m)
            tr[k] += d2ell(g->loss, sqrt(h[(long)k * M + m]), y[(long)k * M + m]);
    if (D_O) for (long n = 0; n < N; ++n) D_O[n] = 0.0;
    if (D_P) for (int m = 0; m < M; ++m) D_P[m] = 0.0;
    for (int k = 0; k < g->K; ++k) {
        int r0 = pos[2 * k], c0 = pos[2 * k + 1];
        for (int yy = 0; yy < g->my; ++yy)
            for (int xx = 0; xx < g->mx; ++xx) {
                int m = yy * g->mx + xx;
                long n = (long)(r0 + yy) * g->nx + (c0 + xx);
                double pa = cabs(P[m]), oa = cabs(O[n]);
                if (D_O) D_O[n] += pa * pa * tr[k] / (2.0 * M);
                if (D_P) D_P[m] += oa * oa * tr[k] / (2.0 * M);
            }
    }
    if (floor_rel > 0.0) {
        double mo = 0.0, mp = 0.0;
        if (D_O) for (long n = 0; n < N; ++n) mo = fmax(mo, D_O[n]);
        if (D_P) for (int m = 0; m < M; ++m) mp = fmax(mp, D_P[m]);
        if (D_O) for (long n = 0; n < N; ++n) D_O[n] = fmax(D_O[n], floor_rel * mo);
        if (D_P) for (int m = 0; m < M; ++m) D_P[m] = fmax(D_P[m], floor_rel * mp);
    }
    free(ph); free(h); free(tr);
}

/* ------------------------------------------------------------------------------------
 * Real-coordinate vector helpers on C^n storage.
 * ------------------------------------------------------------------------------------ */
static double rdot(const dc* a, const dc* b, long n)
{
    double s = 0.0;
    for (long i = 0; i < n; ++i) s += creal(a[i]) * creal(b[i]) + cimag(a[i]) * cimag(b[i]);
    return s;
}

/* ------------------------------------------------------------------------------------
 * Truncated CG for (G + lambda I) x = -g, stopped by Eq. lma_termination_magnitude:
 *   || (G + lambda I) x + g || <= eta ||g||.
 * Object-only (SPR) system, D = I.  x holds the warm start on entry and the step on exit;
 * r_out receives the final CG residual r = -g - (G + lambda I) x.  Returns the number of
 * CG iterations (matrix-vector products after the initial residual).
 * ------------------------------------------------------------------------------------ */
int orc_cg(const orc_geom* g, const dc* O, const dc* P, const int32_t* pos, const double* y,
           const dc* grad, double lambda, double eta, int max_iter, dc* x, dc* r_out,
           int* converged_out)
{
    const long N = (long)g->ny * g->nx;
    dc* r = r_out;
    dc* p = (dc*)malloc(sizeof(dc) * N);
    dc* q = (dc*)malloc(sizeof(dc) * N);
    /* r0 = -g - A x0 */
    orc_ggn_matvec(g, O, P, pos, y, x, NULL, lambda, NULL, NULL, q, NULL);
    for (long i = 0; i < N; ++i) r[i] = -grad[i] - q[i];
    double gnorm = sqrt(rdot(grad, grad, N));
    double tol = eta * gnorm;
    double rr = rdot(r, r, N);
    for (long i = 0; i < N; ++i) p[i] = r[i];
    int it = 0, conv = 0;
    while (1) {
        if (sqrt(rr) <= tol) { conv = 1; break; }
        if (it >= max_iter) break;
        orc_ggn_matvec(g, O, P, pos, y, p, NULL, lambda, NULL, NULL, q, NULL);
        double pq = rdot(p, q, N);
        if (!(pq > 0.0)) break;
        double alpha = rr / pq;
        for (long i = 0; i < N; ++i) { x[i] += alpha * p[i]; r[i] -= alpha * q[i]; }
        double rr_new = rdot(r, r, N);
        double beta = rr_new / rr;
        rr = rr_new;
        for (long i = 0; i < N; ++i) p[i] = r[i] + beta * p[i];
        ++it;
    }
    if (converged_out) *converged_out = conv;
    free(p); free(q);
    return it;
}

/* ------------------------------------------------------------------------------------
 * Object error after global-phase alignment over an illumination mask:
 *   eps = min_phi || e^{i phi} O - O_ref || / || O_ref ||,  closed form phi = arg <O, O_ref>.
 * mask[n] != 0 selects the pixels compared.
 * ------------------------------------------------------------------------------------ */
double orc_object_error(long N, const dc* O, const dc* O_ref, const unsigned char* mask)
{
    dc c = 0.0;
    double nref = 0.0, no = 0.0;
    for (long n = 0; n < N; ++n) {
        if (mask && !mask[n]) continue;
        c += conj(O[n]) * O_ref[n];
        nref += creal(O_ref[n] * conj(O_ref[n]));
        no += creal(O[n] * conj(O[n]));
    }
    double ac = cabs(c);
    /* || e^{i phi} O - O_ref ||^2 = ||O||^2 + ||O_ref||^2 - 2 |<O, O_ref>| */
    double e2 = no + nref - 2.0 * ac;
    if (e2 < 0.0) e2 = 0.0;
    return sqrt(e2 / nref);
}

/* ------------------------------------------------------------------------------------
 * Truncated LM, Algorithm 1 (Sec. 4.2), object-only problem with D = I.
 * Parameters follow Sec. 5: mu0 = 1e-5, mu_min = 1e-8, nu = 1, rho_min = 1e-4, kappa = 4;
 * beta = 0.1 (Gaussian) or 0.9 (Poisson).  Per outer iteration the history arrays receive
 * f, ||g||, mu, number of CG iterations, accepted flag and (if O_ref) the object error.
 * Returns 0 on normal termination, 6 if mu overflowed (stalled).  state (may be NULL): the
 * run starts from it (outer iteration state->t, mu, warm start delta; history entries and
 * max_outer count from there) and receives the state after the last outer iteration run.
 * ------------------------------------------------------------------------------------ */
typedef struct {
    double mu0, mu_min, kappa, nu, rho_min, beta, mu_max;
    int max_outer, max_cg;
    double target_err;   /* stop once the object error <= target_err (if O_ref given; 0: no target) */
} orc_lm_params;

/* Resumable state of Algorithm 1 (Sec. 4.2) between calls: the outer iterations completed
 * so far (t; the App. E surrogate level s_t is a function of t), the damping multiplier mu,
 * and the last CG solution delta, the warm start of the next inner solve (Sec. 4.2, "warm
 * start"), [N] (object only) or [L] (joint state).  With the iterate z itself this is all
 * Algorithm 1 carries from one outer iteration to the next, so a run split in two with the
 * state handed over computes exactly the same iterates as one uninterrupted run. */
typedef struct {
    int t;
    double mu;
    dc* delta;
} orc_lm_state;

int orc_lm_solve(const orc_geom* g, dc* O, const dc* P, const int32_t* pos, const double* y,
                 const orc_lm_params* prm, const dc* O_ref, const unsigned char* mask,
                 int* n_outer_out, int* cg_total_out,
                 double* hist_f, double* hist_gnorm, double* hist_mu, int* hist_cg,
                 double* hist_err, double* hist_rho, int hist_len, orc_lm_state* state)
{
    const long N = (long)g->ny * g->nx;
    dc* grad = (dc*)malloc(sizeof(dc) * N);
    dc* delta = (dc*)calloc((size_t)N, sizeof(dc));
    dc* r = (dc*)malloc(sizeof(dc) * N);
    dc* trial = (dc*)malloc(sizeof(dc) * N);
    double mu = prm->mu0;
    int cg_total = 0, status = 0, t = 0;
    const int t0 = state ? state->t : 0;   /* history entries are counted from t0 */
    if (state) {
        mu = state->mu;
        if (state->delta) memcpy(delta, state->delta, sizeof(dc) * N);
    }
    for (t = t0; t < t0 + prm->max_outer; ++t) {
        const int h = t - t0;
        double dl2 = 0.0;
        double f = orc_loss(g, O, P, pos, y, &dl2);
        orc_gradient(g, O, P, pos, y, grad, NULL);
        double gnorm = sqrt(rdot(grad, grad, N));
        double eta = fmin(prm->beta, sqrt(gnorm));
        double rho = 0.0;
        int cg_this = 0;
        if (hist_f && h < hist_len) hist_f[h] = f;
        if (hist_gnorm && h < hist_len) hist_gnorm[h] = gnorm;
        while (!(rho > prm->rho_min)) {
            double lambda = mu * pow(sqrt(dl2), prm->nu);
            int conv = 0;
            cg_this += orc_cg(g, O, P, pos, y, grad, lambda, eta, prm->max_cg, delta, r, &conv);
            for (long n = 0; n < N; ++n) trial[n] = O[n] + delta[n];
            double f_trial = orc_loss(g, trial, P, pos, y, NULL);
            double dfa = f - f_trial;
            /* predicted reduction -(g.d + d.G.d/2) = d.(lambda d - g)/2 + d.r/2 */
            double dfp = 0.5 * (lambda * rdot(delta, delta, N) - rdot(delta, grad, N)) +
                         0.5 * rdot(delta, r, N);
            rho = dfa / dfp;
            if (!(dfp > 0.0)) rho = -1.0;
            if (rho > 0.75) {
                mu = fmax(mu / prm->kappa, prm->mu_min);
            } else if (rho > 0.25) {
                /* mu unchanged */
            } else {
                mu = prm->kappa * mu;
            }
            if (rho > prm->rho_min) {
                for (long n = 0; n < N; ++n) O[n] = trial[n];
            } else if (mu > prm->mu_max) {
                status = 6;
                break;
            }
        }
        cg_total += cg_this;
        if (hist_mu && h < hist_len) hist_mu[h] = mu;
        if (hist_cg && h < hist_len) hist_cg[h] = cg_this;
        if (hist_rho && h < hist_len) hist_rho[h] = rho;   /* gain ratio of the step that ended it */
        if (status) { ++t; break; }
        if (O_ref) {
            double e = orc_object_error(N, O, O_ref, mask);
            if (hist_err && h < hist_len) hist_err[h] = e;
            if (prm->target_err > 0.0 && e <= prm->target_err) { ++t; break; }
        }
    }
    if (n_outer_out) *n_outer_out = t - t0;
    if (cg_total_out) *cg_total_out = cg_total;
    if (state) {
        state->t = t;
        state->mu = mu;
        if (state->delta) memcpy(state->delta, delta, sizeof(dc) * N);
    }
    free(grad); free(delta); free(r); free(trial);
    return status;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ====================================================================================
 * Scaled / joint / projected LM (the paper's PLM and PLM-J, Secs. 3.3 and 4.2-4.5).
 * The state is z = [O; P] (P present only for the joint problem); vectors over z are
 * stored as N (+ M) complex values and all inner products are real-coordinate ones.
 * ==================================================================================== */

/* z -> (O, P) views. */
typedef struct {
    const orc_geom* g;
    const int32_t* pos;
    const double* y;
    int joint;
    const dc* P_fixed;   /* probe when not joint */
} orc_problem;

static long zlen(const orc_problem* pb) {
    return (long)pb->g->ny * pb->g->nx + (pb->joint ? (long)pb->g->my * pb->g->mx : 0);
}
static const dc* zP(const orc_problem* pb, const dc* z) {
    return pb->joint ? z + (long)pb->g->ny * pb->g->nx : pb->P_fixed;
}

/* (G + lambda D) v for the z-vector v (D NULL = identity), at the point z. */
static void z_matvec(const orc_problem* pb, const dc* z, const dc* v, double lambda, const double* D, dc* out)
{
    const long N = (long)pb->g->ny * pb->g->nx;
    orc_ggn_matvec(pb->g, z, zP(pb, z), pb->pos, pb->y, v, pb->joint ? v + N : NULL, lambda,
                   D, D ? D + N : NULL, out, pb->joint ? out + N : NULL);
}

static void z_gradient(const orc_problem* pb, const dc* z, dc* gz)
{
    const long N = (long)pb->g->ny * pb->g->nx;
    orc_gradient(pb->g, z, zP(pb, z), pb->pos, pb->y, gz, pb->joint ? gz + N : NULL);
}

static double z_loss(const orc_problem* pb, const dc* z, double* dl2)
{
    return orc_loss(pb->g, z, zP(pb, z), pb->pos, pb->y, dl2);
}

/* Closed-form Dg(G) over z with the relative floor (App. B, Eq. ggn_joint_diag). */
static void z_diag(const orc_problem* pb, const dc* z, double floor_rel, double* D)
{
    const long N = (long)pb->g->ny * pb->g->nx;
    const int M = pb->g->my * pb->g->mx;
    if (pb->joint) {
        orc_ggn_diag(pb->g, z, zP(pb, z), pb->pos, pb->y, floor_rel, D, D + N);
    } else {
        double* dp = (double*)malloc(sizeof(double) * M);
        orc_ggn_diag(pb->g, z, zP(pb, z), pb->pos, pb->y, floor_rel, D, dp);
        free(dp);
    }
}

/* Radial projections of Eq. constraints: |O| <= rO, |P| <= rP (separable, Sec. 4.3). */
static void z_project(const orc_problem* pb, dc* z, double rO, double rP)
{
    const long N = (long)pb->g->ny * pb->g->nx;
    const long L = zlen(pb);
    for (long i = 0; i < L; ++i) {
        const double r = i < N ? rO : rP;
        const double a = cabs(z[i]);
        if (r > 0.0 && a > r) z[i] *= r / a;
    }
}

void orc_project(long n, dc* v, double radius)
{
    for (long i = 0; i < n; ++i) {
        double a = cabs(v[i]);
        if (radius > 0.0 && a > radius) v[i] *= radius / a;
    }
}

/* Truncated PCG for (G + lambda D) x = -g with the Jacobi preconditioner
 * Dg(G + lambda D) = (1 + lambda) D when D = Dg(G) (Sec. 3.3), or no preconditioner when
 * D is NULL (D = I).  Stopping rule Eq. lma_termination_magnitude on the unpreconditioned
 * residual.  x: warm start in, step out; r: final residual -g - (G + lambda D) x. */
static int z_pcg(const orc_problem* pb, const dc* z, const dc* grad, double lambda, const double* D, double eta,
                 int max_iter, dc* x, dc* r, int* conv_out)
{
    const long L = zlen(pb);
    dc* p = (dc*)malloc(sizeof(dc) * L);
    dc* q = (dc*)malloc(sizeof(dc) * L);
    dc* zz = (dc*)malloc(sizeof(dc) * L);
    z_matvec(pb, z, x, lambda, D, q);
    for (long i = 0; i < L; ++i) r[i] = -grad[i] - q[i];
    const double tol = eta * sqrt(rdot(grad, grad, L));
    for (long i = 0; i < L; ++i) zz[i] = D ? r[i] / ((1.0 + lambda) * D[i]) : r[i];
    for (long i = 0; i < L; ++i) p[i] = zz[i];
    double rz = rdot(r, zz, L), rr = rdot(r, r, L);
    int it = 0, conv = 0;
    while (1) {
        if (sqrt(rr) <= tol) { conv = 1; break; }
        if (it >= max_iter) break;
        z_matvec(pb, z, p, lambda, D, q);
        double pq = rdot(p, q, L);
        if (!(pq > 0.0)) break;
        double alpha = rz / pq;
        for (long i = 0; i < L; ++i) { x[i] += alpha * p[i]; r[i] -= alpha * q[i]; }
        for (long i = 0; i < L; ++i) zz[i] = D ? r[i] / ((1.0 + lambda) * D[i]) : r[i];
        double rz_new = rdot(r, zz, L);
        rr = rdot(r, r, L);
        double beta = rz_new / rz;
        rz = rz_new;
        for (long i = 0; i < L; ++i) p[i] = zz[i] + beta * p[i];
        ++it;
    }
    if (conv_out) *conv_out = conv;
    free(p); free(q); free(zz);
    return it;
}

/* Public PCG on z-vectors (tests). */
int orc_pcg(const orc_geom* g, const dc* z, const dc* P_fixed, const int32_t* pos, const double* y, int joint,
            const dc* grad, double lambda, const double* D, double eta, int max_iter, dc* x, dc* r,
            int* converged_out)
{
    orc_problem pb = {g, pos, y, joint, P_fixed};
    return z_pcg(&pb, z, grad, lambda, D, eta, max_iter, x, r, converged_out);
}

void orc_ggn_matvec_z(const orc_geom* g, const dc* z, const dc* P_fixed, const int32_t* pos, const double* y,
                      int joint, const dc* v, double lambda, const double* D, dc* out)
{
    orc_problem pb = {g, pos, y, joint, P_fixed};
    z_matvec(&pb, z, v, lambda, D, out);
}

typedef struct {
    double mu0, mu_min, kappa, nu, rho_min, beta, mu_max;
    int max_outer, max_cg;
    double target_err;
    int scaled;          /* D = Dg(G) with lambda = mu and Jacobi PCG (PLM), else D = I (LM) */
    int joint;           /* z = (O, P) (BPR), else O only (SPR) */
    int projected;       /* Algorithm 2 with the radial constraints below */
    double radius_O, radius_P;      /* Eq. constraints: 1 and 1e8 */
    double gamma, tau_s, p_s, sigma;  /* Algorithm 2 / Eq. armijo_criterion */
    int max_ls;
    double diag_floor;   /* D >= diag_floor * max D */
    double f_min;        /* subtracted from f in Algorithm 2's tests (Poisson: sum y - y log y) */
    /* App. E surrogate: h = |psihat|^2 + b + s_t with s_t decreasing on a logarithmic grid
     * from surrogate0 (t = 0) to surrogate_end (t = T - 1) and s_t = 0 from t = T on;
     * surrogate_T = 0 turns it off. */
    double surrogate0, surrogate_end;
    int surrogate_T;
} orc_lm2_params;

/* s_t of the App. E schedule (0 when off or when t >= T). */
double orc_surrogate_at(const orc_lm2_params* prm, int t)
{
    if (prm->surrogate_T <= 0 || t >= prm->surrogate_T) return 0.0;
    if (prm->surrogate_T == 1) return prm->surrogate0;
    const double u = (double)t / (double)(prm->surrogate_T - 1);
    return prm->surrogate0 * pow(prm->surrogate_end / prm->surrogate0, u);
}

/* Algorithm 1 with scaling, the joint state and the Algorithm 2 plug-in.
 * O_inout [N], P_inout [M] (updated when joint).  History and state as in orc_lm_solve
 * (state->t also places the run on the App. E surrogate schedule). */
int orc_lm_solve2(const orc_geom* g, dc* O_inout, dc* P_inout, const int32_t* pos, const double* y,
                  const orc_lm2_params* prm, const dc* O_ref, const unsigned char* mask,
                  int* n_outer_out, int* cg_total_out, double* hist_f, double* hist_gnorm, double* hist_mu,
                  int* hist_cg, double* hist_err, double* hist_rho, int hist_len, orc_lm_state* state)
{
    orc_problem pb = {g, pos, y, prm->joint, P_inout};
    const long N = (long)g->ny * g->nx;
    const int M = g->my * g->mx;
    const long L = zlen(&pb);
    dc* z = (dc*)malloc(sizeof(dc) * L);
    dc* grad = (dc*)malloc(sizeof(dc) * L);
    dc* delta = (dc*)calloc((size_t)L, sizeof(dc));
    dc* r = (dc*)malloc(sizeof(dc) * L);
    dc* trial = (dc*)malloc(sizeof(dc) * L);
    dc* s = (dc*)malloc(sizeof(dc) * L);
    double* D = prm->scaled ? (double*)malloc(sizeof(double) * L) : NULL;
    memcpy(z, O_inout, sizeof(dc) * N);
    if (prm->joint) memcpy(z + N, P_inout, sizeof(dc) * M);
    double mu = prm->mu0;
    int cg_total = 0, status = 0, t;
    const int t0 = state ? state->t : 0;   /* history entries are counted from t0 */
    if (state) {
        mu = state->mu;
        if (state->delta) memcpy(delta, state->delta, sizeof(dc) * L);
    }
    orc_geom gt = *g;   /* the geometry with the surrogate background of iteration t */
    pb.g = &gt;
    for (t = t0; t < t0 + prm->max_outer; ++t) {
        const int h = t - t0;
        gt.b = g->b + orc_surrogate_at(prm, t);
        double dl2 = 0.0;
        const double f = z_loss(&pb, z, &dl2);
        z_gradient(&pb, z, grad);
        const double gnorm = sqrt(rdot(grad, grad, L));
        const double eta = fmin(prm->beta, sqrt(gnorm));
        if (D) z_diag(&pb, z, prm->diag_floor, D);
        if (hist_f && h < hist_len) hist_f[h] = f;
        if (hist_gnorm && h < hist_len) hist_gnorm[h] = gnorm;
        double rho = 0.0;
        int cg_this = 0;
        while (!(rho > prm->rho_min)) {
            const double lambda = D ? mu : mu * pow(sqrt(dl2), prm->nu);
            int conv = 0;
            cg_this += z_pcg(&pb, z, grad, lambda, D, eta, prm->max_cg, delta, r, &conv);
            for (long i = 0; i < L; ++i) trial[i] = z[i] + delta[i];
            const double f_trial = z_loss(&pb, trial, NULL);
            double dd = 0.0;
            for (long i = 0; i < L; ++i) dd += (D ? D[i] : 1.0) * creal(delta[i] * conj(delta[i]));
            const double dfp = 0.5 * (lambda * dd - rdot(delta, grad, L)) + 0.5 * rdot(delta, r, L);
            rho = dfp > 0.0 ? (f - f_trial) / dfp : -1.0;
            if (rho > 0.75) mu = fmax(mu / prm->kappa, prm->mu_min);
            else if (rho > 0.25) { /* keep */ }
            else mu = prm->kappa * mu;
            if (rho > prm->rho_min) {
                if (!prm->projected) {
                    memcpy(z, trial, sizeof(dc) * L);
                } else {
                    /* Algorithm 2: projected step, descent test, Armijo backtracking. */
                    z_project(&pb, trial, prm->radius_O, prm->radius_P);
                    const double fp = z_loss(&pb, trial, NULL);
                    if (fp - prm->f_min < prm->gamma * (f - prm->f_min)) {
                        memcpy(z, trial, sizeof(dc) * L);
                    } else {
                        for (long i = 0; i < L; ++i) s[i] = trial[i] - z[i];
                        const double ss = rdot(s, s, L);
                        const int descent = rdot(grad, s, L) <= -prm->tau_s * pow(sqrt(ss), prm->p_s);
                        if (!descent) {
                            for (long i = 0; i < L; ++i) s[i] = -grad[i];
                        }
                        const double sn2 = rdot(s, s, L);
                        double alpha = 1.0;
                        int found = 0;
                        for (int ls = 0; ls < prm->max_ls; ++ls, alpha *= 0.5) {
                            for (long i = 0; i < L; ++i) trial[i] = z[i] + alpha * s[i];
                            z_project(&pb, trial, prm->radius_O, prm->radius_P);
                            if (z_loss(&pb, trial, NULL) <= f - prm->sigma * alpha * sn2) { found = 1; break; }
                        }
                        if (found) memcpy(z, trial, sizeof(dc) * L);
                    }
                }
            } else if (mu > prm->mu_max) {
                status = 6;
                break;
            }
        }
        cg_total += cg_this;
        if (hist_mu && h < hist_len) hist_mu[h] = mu;
        if (hist_cg && h < hist_len) hist_cg[h] = cg_this;
        if (hist_rho && h < hist_len) hist_rho[h] = rho;   /* gain ratio of the step that ended it */
        if (status) { ++t; break; }
        if (O_ref) {
            double e = orc_object_error(N, z, O_ref, mask);
            if (hist_err && h < hist_len) hist_err[h] = e;
            if (prm->target_err > 0.0 && e <= prm->target_err) { ++t; break; }
        }
    }
    memcpy(O_inout, z, sizeof(dc) * N);
    if (prm->joint) memcpy(P_inout, z + N, sizeof(dc) * M);
    if (n_outer_out) *n_outer_out = t - t0;
    if (cg_total_out) *cg_total_out = cg_total;
    if (state) {
        state->t = t;
        state->mu = mu;
        if (state->delta) memcpy(state->delta, delta, sizeof(dc) * L);
    }
    free(z); free(grad); free(delta); free(r); free(trial); free(s); free(D);
    return status;
}
