/*
 * fmm_oracle.c -- plain, slow FP64 CPU oracle for the Laplace treecode / fast
 * multipole method of Yokota & Barba, "Treecode and fast multipole method for
 * N-body simulation with CUDA" (GPU Computing Gems, 2011).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares no
 * code, header, table or helper with the CUDA path, and the CUDA path never
 * calls it.
 *
 * Every operator is written as its plain definition, in FP64, in the paper's
 * notation:
 *   Eq. 1   direct sum (potential and its gradient; the target mass m_i dropped,
 *           as Listing-1 style "acceleration" code does)
 *   Eq. 2   multipole coefficients M_n^m (P2M) and their evaluation (M2P)
 *   Eq. 3   local coefficients L_n^m and their evaluation (L2P)
 *   Eq. 4-5 multipole-to-local translation (M2L) with A_n^m
 *   Eq. 6   spherical harmonics Y_n^m
 *   Eq. 7-9 associated Legendre recurrences
 * M2M and L2L are not printed in the paper; they follow the translation theorems
 * of Cheng, Greengard & Rokhlin, J. Comput. Phys. 155 (1999), the reference the
 * paper cites for its translation operators (Section "Overview of Advanced
 * Techniques").
 *
 * Readings taken where the paper is silent or garbled:
 *   - Eq. 8 prints (2m-1)!; the Legendre recurrence needs the double factorial
 *     (2m-1)!! -- used here, with the Condon-Shortley phase (-1)^m.
 *   - Eq. 4 carries (-1)^j in the denominator; that is the textbook M2L for the
 *     vector v = (target centre - source centre), which is the direction used.
 *   - p is the number of degrees: n = 0..p-1 (Eq. 4 sums n up to p-1).
 *   - pairs at distance exactly zero contribute nothing; eps2 softens P2P only.
 *   - gradient: the analytic derivative of each series in spherical coordinates,
 *     with P_n^m / sin(alpha) taken from its own recurrence so that it stays finite
 *     on the expansion's z axis.
 *
 * Coefficient storage: complex, m >= 0 only (M_n^{-m} = conj(M_n^m)), index
 * n(n+1)/2 + m.
 *
 * Trees: (1) uniform octree of depth L over the root cube, dense per level: the cell
 * of level l with Morton key k has global index (8^l - 1)/7 + k; (2) adaptive octree
 * (cells split while they hold more than leaf_size particles) with the U, V, W, X lists
 * of Cheng, Greengard & Rokhlin (1999), numbered level by level in key order.
 */
#include <complex.h>
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define TRI(n, m) ((n) * ((n) + 1) / 2 + (m))
#define MAXDEG 80

static double FACT[2 * MAXDEG + 2];
static int fact_ready = 0;

static void init_fact(void)
{
    if (fact_ready) return;
    FACT[0] = 1.0;
    for (int i = 1; i < 2 * MAXDEG + 2; ++i) FACT[i] = FACT[i - 1] * i;
    fact_ready = 1;
}

int orc_version(void) { return 1; }

/* Number of OpenMP threads the parallel loops use. */
int orc_threads(void)
{
    int t = 1;
#pragma omp parallel
    {
#pragma omp single
        t = omp_get_num_threads();
    }
    return t;
}

/* ------------------------------------------------------------------------- */
/* Special functions                                                         */
/* ------------------------------------------------------------------------- */

/* Associated Legendre P_n^m(x), 0 <= m <= n < nmax, from Eq. 7 (three-term
 * recurrence in n), Eq. 8 (diagonal, read with the double factorial) and Eq. 9
 * (first off-diagonal).  Triangular storage TRI(n, m). */
void orc_legendre(int nmax, double x, double *P)
{
    double s = sqrt(fmax(0.0, 1.0 - x * x));
    double pmm = 1.0; /* P_m^m = (-1)^m (2m-1)!! (1-x^2)^{m/2} */
    for (int m = 0; m < nmax; ++m) {
        P[TRI(m, m)] = pmm;
        if (m + 1 < nmax) P[TRI(m + 1, m)] = x * (2 * m + 1) * pmm; /* Eq. 9 */
        for (int n = m + 1; n + 1 < nmax; ++n)                      /* Eq. 7 */
            P[TRI(n + 1, m)] = (x * (2 * n + 1) * P[TRI(n, m)] - (n + m) * P[TRI(n - 1, m)]) / (n - m + 1);
        pmm = -pmm * (2 * m + 1) * s;                                /* Eq. 8 */
    }
}

/* Q_n^m = P_n^m(cos a) / sin(a) for m >= 1 by the same recurrences started from
 * Q_m^m = (-1)^m (2m-1)!! sin(a)^{m-1}; finite at sin(a) = 0.  Q_n^0 set to 0. */
static void legendre_over_sin(int nmax, double x, double *Q)
{
    double s = sqrt(fmax(0.0, 1.0 - x * x));
    for (int n = 0; n < nmax; ++n) Q[TRI(n, 0)] = 0.0;
    double qmm = -1.0; /* Q_1^1 = -1 */
    for (int m = 1; m < nmax; ++m) {
        Q[TRI(m, m)] = qmm;
        if (m + 1 < nmax) Q[TRI(m + 1, m)] = x * (2 * m + 1) * qmm;
        for (int n = m + 1; n + 1 < nmax; ++n)
            Q[TRI(n + 1, m)] = (x * (2 * n + 1) * Q[TRI(n, m)] - (n + m) * Q[TRI(n - 1, m)]) / (n - m + 1);
        qmm = -qmm * (2 * m + 1) * s;
    }
}

/* d/d(alpha) of P_n^m(cos alpha):  m = 0 -> P_n^1;  m >= 1 -> n x Q_n^m - (n+m) Q_{n-1}^m
 * (from (1-x^2) dP_n^m/dx = (n+m) P_{n-1}^m - n x P_n^m). */
static double dlegendre_dalpha(int n, int m, double x, const double *P, const double *Q)
{
    if (m == 0) return (n >= 1) ? P[TRI(n, 1)] : 0.0;
    double q1 = (n - 1 >= m) ? Q[TRI(n - 1, m)] : 0.0;
    return n * x * Q[TRI(n, m)] - (n + m) * q1;
}

/* cart2sph: rho = |v|, alpha = polar angle from +z, beta = azimuth; 0,0 at the origin. */
static void cart2sph(const double *v, double *rho, double *alpha, double *beta)
{
    double r = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    *rho = r;
    if (r == 0.0) {
        *alpha = 0.0;
        *beta = 0.0;
        return;
    }
    double c = v[2] / r;
    if (c > 1.0) c = 1.0;
    if (c < -1.0) c = -1.0;
    *alpha = acos(c);
    *beta = atan2(v[1], v[0]);
}

/* Eq. 6: Y_n^m(alpha, beta) = sqrt((n-|m|)!/(n+|m|)!) P_n^{|m|}(cos alpha) e^{i m beta},
 * stored for m >= 0 (Y_n^{-m} = conj(Y_n^m)). */
void orc_ynm(int nmax, double alpha, double beta, double complex *Y)
{
    init_fact();
    double P[TRI(MAXDEG, 0) + MAXDEG];
    orc_legendre(nmax, cos(alpha), P);
    for (int n = 0; n < nmax; ++n)
        for (int m = 0; m <= n; ++m)
            Y[TRI(n, m)] = sqrt(FACT[n - m] / FACT[n + m]) * P[TRI(n, m)] * cexp(I * (m * beta));
}

/* Python-friendly wrapper: Y as interleaved (re, im). */
void orc_ynm_ri(int nmax, double alpha, double beta, double *Yri)
{
    double complex Y[TRI(MAXDEG, 0) + MAXDEG];
    orc_ynm(nmax, alpha, beta, Y);
    for (int i = 0; i < TRI(nmax, 0); ++i) {
        Yri[2 * i] = creal(Y[i]);
        Yri[2 * i + 1] = cimag(Y[i]);
    }
}

static double complex yfull(const double complex *Y, int n, int m)
{
    return (m >= 0) ? Y[TRI(n, m)] : conj(Y[TRI(n, -m)]);
}

static double complex cfull(const double complex *C, int n, int m)
{
    return (m >= 0) ? C[TRI(n, m)] : conj(C[TRI(n, -m)]);
}

/* Eq. 5: A_n^m = 1 / sqrt((n-m)! (n+m)!) */
static double Anm(int n, int m) { return 1.0 / sqrt(FACT[n - m] * FACT[n + m]); }

/* i^e for even e: (-1)^(e/2) */
static double ipow_even(int e)
{
    int h = e / 2;
    return (h % 2 == 0) ? 1.0 : -1.0;
}

static double neg1pow(int e) { return (e % 2 == 0) ? 1.0 : -1.0; }

/* ------------------------------------------------------------------------- */
/* Particle operators                                                        */
/* ------------------------------------------------------------------------- */

/* Eq. 1 restricted to a source set: phi_i = sum_j q_j / sqrt(r^2 + eps2),
 * grad_i = -sum_j q_j (x_i - x_j) / (r^2 + eps2)^{3/2}; pairs with r^2 == 0 skipped.
 * out4 accumulates (phi, dphi/dx, dphi/dy, dphi/dz). */
static void p2p_one(const double *xt, int64_t ns, const double *src, double eps2, double *out4)
{
    for (int64_t j = 0; j < ns; ++j) {
        double dx = xt[0] - src[4 * j + 0];
        double dy = xt[1] - src[4 * j + 1];
        double dz = xt[2] - src[4 * j + 2];
        double r2 = dx * dx + dy * dy + dz * dz;
        if (r2 == 0.0) continue;
        double q = src[4 * j + 3];
        double inv = 1.0 / sqrt(r2 + eps2);
        double inv3 = inv * inv * inv;
        out4[0] += q * inv;
        out4[1] -= q * dx * inv3;
        out4[2] -= q * dy * inv3;
        out4[3] -= q * dz * inv3;
    }
}

/* O(N^2) direct sum (Eq. 1) for nt targets against ns sources (xyzq, FP64).
 * out: 4*nt (phi, grad).  Parallel over targets only. */
void orc_direct(int64_t nt, const double *tgt_xyz3, int64_t ns, const double *src_xyzq, double eps2, double *out)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < nt; ++i) {
        double acc[4] = {0, 0, 0, 0};
        p2p_one(tgt_xyz3 + 3 * i, ns, src_xyzq, eps2, acc);
        for (int c = 0; c < 4; ++c) out[4 * i + c] = acc[c];
    }
}

/* Eq. 2 (the M_n^m factor): M_n^m += sum_j q_j rho_j^n Y_n^{-m}(alpha_j, beta_j),
 * (rho, alpha, beta) = x_j - centre.  n < p, m = 0..n. */
void orc_p2m(int p, const double *centre, int64_t np, const double *xyzq, double complex *M)
{
    init_fact();
    double complex Y[TRI(MAXDEG, 0) + MAXDEG];
    for (int64_t j = 0; j < np; ++j) {
        double v[3] = {xyzq[4 * j] - centre[0], xyzq[4 * j + 1] - centre[1], xyzq[4 * j + 2] - centre[2]};
        double rho, al, be;
        cart2sph(v, &rho, &al, &be);
        orc_ynm(p, al, be, Y);
        double q = xyzq[4 * j + 3];
        double rn = 1.0;
        for (int n = 0; n < p; ++n) {
            for (int m = 0; m <= n; ++m) M[TRI(n, m)] += q * rn * yfull(Y, n, -m);
            rn *= rho;
        }
    }
}

/* Shared body of M2P (Eq. 2 evaluation, radial factor r^{-n-1}) and L2P (Eq. 3
 * evaluation, radial factor r^n): value and analytic gradient at point x of the
 * series sum_{n<p} sum_{m=-n..n} C_n^m f_n(r) Y_n^m(theta, phi). */
static void eval_series(int p, int local, const double *centre, const double complex *C, const double *x, double *out4)
{
    init_fact();
    double v[3] = {x[0] - centre[0], x[1] - centre[1], x[2] - centre[2]};
    double r, th, ph;
    cart2sph(v, &r, &th, &ph);
    double ct = cos(th), st = sin(th);
    double P[TRI(MAXDEG, 0) + MAXDEG], Q[TRI(MAXDEG, 0) + MAXDEG];
    orc_legendre(p + 1, ct, P);
    legendre_over_sin(p + 1, ct, Q);
    double phi = 0, dr = 0, dth = 0, dph = 0;
    for (int n = 0; n < p; ++n) {
        double f, df, fr; /* f_n(r), f_n'(r), f_n(r)/r */
        if (local) {
            f = pow(r, n);
            df = (n >= 1) ? n * pow(r, n - 1) : 0.0;
            fr = (n >= 1) ? pow(r, n - 1) : 0.0; /* the n = 0 term has no angular gradient */
        } else {
            f = pow(r, -n - 1);
            df = -(n + 1) * pow(r, -n - 2);
            fr = pow(r, -n - 2);
        }
        for (int m = -n; m <= n; ++m) {
            int am = abs(m);
            double nrm = sqrt(FACT[n - am] / FACT[n + am]);
            double complex e = cexp(I * (m * ph));
            double complex c = cfull(C, n, m);
            double complex y = nrm * P[TRI(n, am)] * e;
            phi += creal(c * y) * f;
            dr += creal(c * y) * df;
            dth += creal(c * nrm * dlegendre_dalpha(n, am, ct, P, Q) * e) * fr;
            if (m != 0) dph += creal(c * nrm * (I * m) * Q[TRI(n, am)] * e) * fr;
        }
    }
    double cp = cos(ph), sp = sin(ph);
    out4[0] += phi;
    out4[1] += dr * st * cp + dth * ct * cp - dph * sp;
    out4[2] += dr * st * sp + dth * ct * sp + dph * cp;
    out4[3] += dr * ct - dth * st;
}

/* M2P: evaluate the multipole series of Eq. 2 (about `centre`) at x. */
void orc_m2p(int p, const double *centre, const double complex *M, const double *x, double *out4)
{
    eval_series(p, 0, centre, M, x, out4);
}

/* L2P: evaluate the local series of Eq. 3 (about `centre`) at x. */
void orc_l2p(int p, const double *centre, const double complex *L, const double *x, double *out4)
{
    eval_series(p, 1, centre, L, x, out4);
}

/* ------------------------------------------------------------------------- */
/* Translation operators                                                     */
/* ------------------------------------------------------------------------- */

/* Eq. 4 (M2L):
 *   L_j^k += sum_{n<p} sum_{m=-n..n} M_n^m i^{|k-m|-|k|-|m|} A_n^m A_j^k Y_{j+n}^{m-k}(alpha, beta)
 *                                   / ((-1)^j A_{j+n}^{m-k} rho^{j+n+1})
 * with (rho, alpha, beta) = target centre - source centre. */
void orc_m2l(int p, const double *src_centre, const double *tgt_centre, const double complex *M, double complex *L)
{
    init_fact();
    double v[3] = {tgt_centre[0] - src_centre[0], tgt_centre[1] - src_centre[1], tgt_centre[2] - src_centre[2]};
    double rho, al, be;
    cart2sph(v, &rho, &al, &be);
    double complex Y[TRI(2 * MAXDEG, 0) + 2 * MAXDEG];
    orc_ynm(2 * p - 1, al, be, Y);
    for (int j = 0; j < p; ++j)
        for (int k = 0; k <= j; ++k) {
            double complex acc = 0;
            for (int n = 0; n < p; ++n)
                for (int m = -n; m <= n; ++m) {
                    double c = ipow_even(abs(k - m) - abs(k) - abs(m)) * Anm(n, m) * Anm(j, k) /
                               (neg1pow(j) * Anm(j + n, m - k) * pow(rho, j + n + 1));
                    acc += cfull(M, n, m) * c * yfull(Y, j + n, m - k);
                }
            L[TRI(j, k)] += acc;
        }
}

/* M2M (Cheng, Greengard & Rokhlin 1999, translation of a multipole expansion):
 *   M_j^k(parent) += sum_{n=0..j} sum_{m=-n..n, |k-m| <= j-n}
 *        M_{j-n}^{k-m}(child) i^{|k|-|m|-|k-m|} A_n^m A_{j-n}^{k-m} rho^n Y_n^{-m}(alpha, beta) / A_j^k
 * with (rho, alpha, beta) = child centre - parent centre. */
void orc_m2m(int p, const double *child_centre, const double *parent_centre, const double complex *Mc, double complex *Mp)
{
    init_fact();
    double v[3] = {child_centre[0] - parent_centre[0], child_centre[1] - parent_centre[1],
                   child_centre[2] - parent_centre[2]};
    double rho, al, be;
    cart2sph(v, &rho, &al, &be);
    double complex Y[TRI(MAXDEG, 0) + MAXDEG];
    orc_ynm(p, al, be, Y);
    for (int j = 0; j < p; ++j)
        for (int k = 0; k <= j; ++k) {
            double complex acc = 0;
            for (int n = 0; n <= j; ++n)
                for (int m = -n; m <= n; ++m) {
                    if (abs(k - m) > j - n) continue;
                    double c = ipow_even(abs(k) - abs(m) - abs(k - m)) * Anm(n, m) * Anm(j - n, k - m) *
                               pow(rho, n) / Anm(j, k);
                    acc += cfull(Mc, j - n, k - m) * c * yfull(Y, n, -m);
                }
            Mp[TRI(j, k)] += acc;
        }
}

/* L2L (Cheng, Greengard & Rokhlin 1999, translation of a local expansion):
 *   L_j^k(child) += sum_{n=j..p-1} sum_{m=-n..n, |m-k| <= n-j}
 *        L_n^m(parent) i^{|m|-|m-k|-|k|} A_{n-j}^{m-k} A_j^k Y_{n-j}^{m-k}(alpha, beta) rho^{n-j}
 *        / ((-1)^{n+j} A_n^m)
 * with (rho, alpha, beta) = parent centre - child centre (the old expansion
 * centre seen from the new one). */
void orc_l2l(int p, const double *parent_centre, const double *child_centre, const double complex *Lp, double complex *Lc)
{
    init_fact();
    double v[3] = {parent_centre[0] - child_centre[0], parent_centre[1] - child_centre[1],
                   parent_centre[2] - child_centre[2]};
    double rho, al, be;
    cart2sph(v, &rho, &al, &be);
    double complex Y[TRI(MAXDEG, 0) + MAXDEG];
    orc_ynm(p, al, be, Y);
    for (int j = 0; j < p; ++j)
        for (int k = 0; k <= j; ++k) {
            double complex acc = 0;
            for (int n = j; n < p; ++n)
                for (int m = -n; m <= n; ++m) {
                    if (abs(m - k) > n - j) continue;
                    double c = ipow_even(abs(m) - abs(m - k) - abs(k)) * Anm(n - j, m - k) * Anm(j, k) *
                               pow(rho, n - j) / (neg1pow(n + j) * Anm(n, m));
                    acc += cfull(Lp, n, m) * c * yfull(Y, n - j, m - k);
                }
            Lc[TRI(j, k)] += acc;
        }
}

/* Interleaved (re, im) wrappers for the per-operator pins. */
static void ri2c(int cnt, const double *ri, double complex *c)
{
    for (int i = 0; i < cnt; ++i) c[i] = ri[2 * i] + I * ri[2 * i + 1];
}
static void c2ri(int cnt, const double complex *c, double *ri)
{
    for (int i = 0; i < cnt; ++i) {
        ri[2 * i] = creal(c[i]);
        ri[2 * i + 1] = cimag(c[i]);
    }
}
#define NT(p) ((p) * ((p) + 1) / 2)

void orc_p2m_ri(int p, const double *centre, int64_t np, const double *xyzq, double *Mri)
{
    double complex M[NT(MAXDEG)];
    ri2c(NT(p), Mri, M);
    orc_p2m(p, centre, np, xyzq, M);
    c2ri(NT(p), M, Mri);
}
void orc_m2p_ri(int p, const double *centre, const double *Mri, const double *x, double *out4)
{
    double complex M[NT(MAXDEG)];
    ri2c(NT(p), Mri, M);
    orc_m2p(p, centre, M, x, out4);
}
void orc_l2p_ri(int p, const double *centre, const double *Lri, const double *x, double *out4)
{
    double complex L[NT(MAXDEG)];
    ri2c(NT(p), Lri, L);
    orc_l2p(p, centre, L, x, out4);
}
void orc_m2l_ri(int p, const double *sc, const double *tc, const double *Mri, double *Lri)
{
    double complex M[NT(MAXDEG)], L[NT(MAXDEG)];
    ri2c(NT(p), Mri, M);
    ri2c(NT(p), Lri, L);
    orc_m2l(p, sc, tc, M, L);
    c2ri(NT(p), L, Lri);
}
void orc_m2m_ri(int p, const double *cc, const double *pc, const double *Mcri, double *Mpri)
{
    double complex Mc[NT(MAXDEG)], Mp[NT(MAXDEG)];
    ri2c(NT(p), Mcri, Mc);
    ri2c(NT(p), Mpri, Mp);
    orc_m2m(p, cc, pc, Mc, Mp);
    c2ri(NT(p), Mp, Mpri);
}
void orc_l2l_ri(int p, const double *pc, const double *cc, const double *Lpri, double *Lcri)
{
    double complex Lp[NT(MAXDEG)], Lc[NT(MAXDEG)];
    ri2c(NT(p), Lpri, Lp);
    ri2c(NT(p), Lcri, Lc);
    orc_l2l(p, pc, cc, Lp, Lc);
    c2ri(NT(p), Lc, Lcri);
}

/* ------------------------------------------------------------------------- */
/* Root box, Morton keys, uniform tree and interaction lists                 */
/* ------------------------------------------------------------------------- */

/* Root cube from the data: per-dimension min/max (exact as doubles), centre
 * c = (lo + hi) * 0.5, side S = max_d (hi_d - lo_d) (S = 1 if zero), origin
 * c - S * 0.5.  Returns 0, or 1 if a coordinate is not finite. */
int orc_root_box(int64_t n, const float *xyzq, double *origin3, double *side)
{
    double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    int bad = 0;
    for (int64_t i = 0; i < n; ++i)
        for (int d = 0; d < 3; ++d) {
            double x = (double)xyzq[4 * i + d];
            if (!isfinite(x)) {
                bad = 1;
                continue;
            }
            if (x < mn[d]) mn[d] = x;
            if (x > mx[d]) mx[d] = x;
        }
    if (n == 0 || bad) {
        for (int d = 0; d < 3; ++d) origin3[d] = 0.0;
        *side = 1.0;
        return bad;
    }
    double S = 0.0;
    for (int d = 0; d < 3; ++d)
        if (mx[d] - mn[d] > S) S = mx[d] - mn[d];
    if (S == 0.0) S = 1.0;
    for (int d = 0; d < 3; ++d) {
        double c = (mn[d] + mx[d]) * 0.5;
        origin3[d] = c - S * 0.5;
    }
    *side = S;
    return 0;
}

static uint64_t interleave3(uint64_t ix, uint64_t iy, uint64_t iz, int bits)
{
    uint64_t key = 0;
    for (int b = 0; b < bits; ++b) {
        key |= ((ix >> b) & 1ull) << (3 * b + 0);
        key |= ((iy >> b) & 1ull) << (3 * b + 1);
        key |= ((iz >> b) & 1ull) << (3 * b + 2);
    }
    return key;
}

static void deinterleave3(uint64_t key, int bits, int64_t *ix, int64_t *iy, int64_t *iz)
{
    int64_t a = 0, b2 = 0, c = 0;
    for (int b = 0; b < bits; ++b) {
        a |= (int64_t)((key >> (3 * b + 0)) & 1ull) << b;
        b2 |= (int64_t)((key >> (3 * b + 1)) & 1ull) << b;
        c |= (int64_t)((key >> (3 * b + 2)) & 1ull) << b;
    }
    *ix = a;
    *iy = b2;
    *iz = c;
}

/* 63-bit Morton keys at depth 21: with the scale s = 2^21 / S (one IEEE FP64 division),
 * k_d = clamp(floor((x_d - origin_d) * s), 0, 2^21 - 1), each operation one IEEE FP64
 * rounding (built with -ffp-contract=off); bit 3b+0 of the key is bit b of k_x, 3b+1 of
 * k_y, 3b+2 of k_z. */
void orc_keys(int64_t n, const float *xyzq, const double *origin3, double side, uint64_t *keys)
{
    const double scale = 2097152.0 / side;
    for (int64_t i = 0; i < n; ++i) {
        uint64_t k[3];
        for (int d = 0; d < 3; ++d) {
            double t = (double)xyzq[4 * i + d] - origin3[d];
            double v = t * scale;
            double f = floor(v);
            if (!(f >= 0.0)) f = 0.0; /* also maps NaN to 0 */
            if (f > 2097151.0) f = 2097151.0;
            k[d] = (uint64_t)f;
        }
        keys[i] = interleave3(k[0], k[1], k[2], 21);
    }
}

void orc_key_decode(uint64_t key, int bits, int64_t *ixyz)
{
    deinterleave3(key, bits, &ixyz[0], &ixyz[1], &ixyz[2]);
}

static int64_t level_offset(int l) { return (((int64_t)1 << (3 * l)) - 1) / 7; }

/* Geometric centre of the level-l cell with key `key`. */
void orc_cell_centre(const double *origin3, double side, int l, uint64_t key, double *c3)
{
    int64_t ix[3];
    deinterleave3(key, l, &ix[0], &ix[1], &ix[2]);
    double h = side / (double)((int64_t)1 << l);
    for (int d = 0; d < 3; ++d) c3[d] = origin3[d] + ((double)ix[d] + 0.5) * h;
}

/* Per-level cell ranges of a uniform depth-L tree from the sorted leaf keys:
 * begin[g], count[g] for every global cell index g (empty cells: 0, 0). */
void orc_cells(int L, int64_t n, const uint64_t *sorted_leaf_keys, int32_t *begin, int32_t *count)
{
    int64_t C = level_offset(L + 1);
    for (int64_t g = 0; g < C; ++g) {
        begin[g] = 0;
        count[g] = 0;
    }
    for (int l = 0; l <= L; ++l) {
        int64_t off = level_offset(l);
        for (int64_t i = 0; i < n; ++i) {
            uint64_t ck = sorted_leaf_keys[i] >> (3 * (L - l));
            if (count[off + ck] == 0) begin[off + ck] = (int32_t)i;
            count[off + ck] += 1;
        }
    }
}

/* P2P (near-field) list of each nonempty leaf: the nonempty level-L cells at
 * Chebyshev index distance <= 1, itself included (27 for an interior cell),
 * ascending key.  offs[8^L + 1], ids = global cell indices.  Returns entries. */
int64_t orc_list_p2p(int L, const int32_t *count, int32_t *offs, int32_t *ids)
{
    int64_t nl = (int64_t)1 << (3 * L), off = level_offset(L), side = (int64_t)1 << L, e = 0;
    for (int64_t t = 0; t < nl; ++t) {
        offs[t] = (int32_t)e;
        if (count[off + t] == 0) continue;
        int64_t x, y, z;
        deinterleave3((uint64_t)t, L, &x, &y, &z);
        /* candidates in ascending key order: collect then sort */
        int64_t cand[27];
        int nc = 0;
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    int64_t a = x + dx, b = y + dy, c = z + dz;
                    if (a < 0 || b < 0 || c < 0 || a >= side || b >= side || c >= side) continue;
                    int64_t k = (int64_t)interleave3(a, b, c, L);
                    if (count[off + k] == 0) continue;
                    cand[nc++] = k;
                }
        for (int i = 1; i < nc; ++i)
            for (int j = i; j > 0 && cand[j - 1] > cand[j]; --j) {
                int64_t tmp = cand[j];
                cand[j] = cand[j - 1];
                cand[j - 1] = tmp;
            }
        for (int i = 0; i < nc; ++i) ids[e++] = (int32_t)(off + cand[i]);
    }
    offs[nl] = (int32_t)e;
    return e;
}

/* M2L (well-separated) list of each nonempty cell at levels 2..L: nonempty
 * children of the parent's neighbours (parent included) that are not themselves
 * at Chebyshev index distance <= 1 (at most 189), ascending key.  offs[C + 1]
 * over all global cells (rows of levels 0, 1 and empty cells are empty). */
int64_t orc_list_m2l(int L, const int32_t *count, int32_t *offs, int32_t *ids)
{
    int64_t e = 0;
    for (int l = 0; l <= L; ++l) {
        int64_t nc_l = (int64_t)1 << (3 * l), off = level_offset(l), side = (int64_t)1 << l;
        for (int64_t t = 0; t < nc_l; ++t) {
            offs[off + t] = (int32_t)e;
            if (l < 2 || count[off + t] == 0) continue;
            int64_t x, y, z;
            deinterleave3((uint64_t)t, l, &x, &y, &z);
            int64_t px = x >> 1, py = y >> 1, pz = z >> 1;
            int64_t cand[216];
            int nc = 0;
            for (int dz = -1; dz <= 1; ++dz)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx)
                        for (int c = 0; c < 8; ++c) {
                            int64_t a = 2 * (px + dx) + (c & 1), b = 2 * (py + dy) + ((c >> 1) & 1),
                                    cz = 2 * (pz + dz) + ((c >> 2) & 1);
                            if (a < 0 || b < 0 || cz < 0 || a >= side || b >= side || cz >= side) continue;
                            if (llabs(a - x) <= 1 && llabs(b - y) <= 1 && llabs(cz - z) <= 1) continue;
                            int64_t k = (int64_t)interleave3(a, b, cz, l);
                            if (count[off + k] == 0) continue;
                            cand[nc++] = k;
                        }
            for (int i = 1; i < nc; ++i)
                for (int j = i; j > 0 && cand[j - 1] > cand[j]; --j) {
                    int64_t tmp = cand[j];
                    cand[j] = cand[j - 1];
                    cand[j - 1] = tmp;
                }
            for (int i = 0; i < nc; ++i) ids[e++] = (int32_t)(off + cand[i]);
        }
    }
    offs[level_offset(L + 1)] = (int32_t)e;
    return e;
}

/* ------------------------------------------------------------------------- */
/* The FMM / treecode passes over a uniform tree                             */
/* ------------------------------------------------------------------------- */

/*
 * Runs P2M -> M2M -> (FMM: M2L -> L2L -> L2P | treecode: M2P) and P2P over the
 * uniform depth-L tree (Fig. 1 flow).  Particles are already sorted by leaf key
 * (sxyzq: 4n FP64).  M and Lc (C * p(p+1)/2 complex as interleaved re, im) must
 * be zero on entry; out (4n, sorted order) accumulates (phi, grad).
 * need: optional mask over the 8^L leaves; when given, only the expansions that
 * feed the masked leaves are translated and only their particles evaluated
 * (every multipole is still formed).
 * method: 0 = FMM, 1 = treecode.
 */
int orc_fmm_passes(int p, int L, int method, double eps2, const double *origin3, double side, int64_t n,
                   const double *sxyzq, const int32_t *begin, const int32_t *count, const int32_t *p2p_offs,
                   const int32_t *p2p_ids, const int32_t *m2l_offs, const int32_t *m2l_ids, const uint8_t *need,
                   double *Mri, double *Lri, double *out)
{
    init_fact();
    (void)n;
    const int nt = NT(p);
    double complex *M = (double complex *)Mri;
    double complex *Lc = (double complex *)Lri;
    int64_t C = level_offset(L + 1);
    uint8_t *needc = (uint8_t *)calloc((size_t)C, 1);
    if (!needc) return -1;
    {
        int64_t nl = (int64_t)1 << (3 * L), offL = level_offset(L);
        for (int64_t t = 0; t < nl; ++t) {
            if (need && !need[t]) continue;
            for (int l = 0; l <= L; ++l) needc[level_offset(l) + (t >> (3 * (L - l)))] = 1;
        }
        (void)offL;
    }

    /* P2M at every nonempty leaf */
    {
        int64_t nl = (int64_t)1 << (3 * L), off = level_offset(L);
#pragma omp parallel for schedule(dynamic, 64)
        for (int64_t t = 0; t < nl; ++t) {
            int64_t g = off + t;
            if (count[g] == 0) continue;
            double c[3];
            orc_cell_centre(origin3, side, L, (uint64_t)t, c);
            orc_p2m(p, c, count[g], sxyzq + 4 * (int64_t)begin[g], M + g * nt);
        }
    }
    /* M2M from level L-1 up to 0 */
    for (int l = L - 1; l >= 0; --l) {
        int64_t ncl = (int64_t)1 << (3 * l), off = level_offset(l), offc = level_offset(l + 1);
#pragma omp parallel for schedule(dynamic, 16)
        for (int64_t t = 0; t < ncl; ++t) {
            if (count[off + t] == 0) continue;
            double pc[3];
            orc_cell_centre(origin3, side, l, (uint64_t)t, pc);
            for (int c = 0; c < 8; ++c) {
                int64_t ck = 8 * t + c;
                if (count[offc + ck] == 0) continue;
                double cc[3];
                orc_cell_centre(origin3, side, l + 1, (uint64_t)ck, cc);
                orc_m2m(p, cc, pc, M + (offc + ck) * nt, M + (off + t) * nt);
            }
        }
    }

    if (method == 0) {
        /* M2L at levels 2..L */
        for (int l = 2; l <= L; ++l) {
            int64_t ncl = (int64_t)1 << (3 * l), off = level_offset(l);
#pragma omp parallel for schedule(dynamic, 4)
            for (int64_t t = 0; t < ncl; ++t) {
                int64_t g = off + t;
                if (count[g] == 0 || !needc[g]) continue;
                double tc[3];
                orc_cell_centre(origin3, side, l, (uint64_t)t, tc);
                for (int32_t e = m2l_offs[g]; e < m2l_offs[g + 1]; ++e) {
                    int64_t s = m2l_ids[e];
                    double sc[3];
                    orc_cell_centre(origin3, side, l, (uint64_t)(s - off), sc);
                    orc_m2l(p, sc, tc, M + s * nt, Lc + g * nt);
                }
            }
        }
        /* L2L from level 2 down to L (parents at levels 2..L-1) */
        for (int l = 3; l <= L; ++l) {
            int64_t ncl = (int64_t)1 << (3 * l), off = level_offset(l), offp = level_offset(l - 1);
#pragma omp parallel for schedule(dynamic, 16)
            for (int64_t t = 0; t < ncl; ++t) {
                int64_t g = off + t;
                if (count[g] == 0 || !needc[g]) continue;
                double cc[3], pc[3];
                orc_cell_centre(origin3, side, l, (uint64_t)t, cc);
                orc_cell_centre(origin3, side, l - 1, (uint64_t)(t >> 3), pc);
                orc_l2l(p, pc, cc, Lc + (offp + (t >> 3)) * nt, Lc + g * nt);
            }
        }
        /* L2P at the leaves */
        if (L >= 2) {
            int64_t nl = (int64_t)1 << (3 * L), off = level_offset(L);
#pragma omp parallel for schedule(dynamic, 16)
            for (int64_t t = 0; t < nl; ++t) {
                int64_t g = off + t;
                if (count[g] == 0 || !needc[g]) continue;
                double c[3];
                orc_cell_centre(origin3, side, L, (uint64_t)t, c);
                for (int32_t i = begin[g]; i < begin[g] + count[g]; ++i)
                    orc_l2p(p, c, Lc + g * nt, sxyzq + 4 * (int64_t)i, out + 4 * (int64_t)i);
            }
        }
    } else {
        /* treecode: M2P from the M2L list of the leaf and of each ancestor at levels 2..L */
        int64_t nl = (int64_t)1 << (3 * L), offL = level_offset(L);
#pragma omp parallel for schedule(dynamic, 16)
        for (int64_t t = 0; t < nl; ++t) {
            int64_t g = offL + t;
            if (count[g] == 0 || !needc[g]) continue;
            for (int l = 2; l <= L; ++l) {
                int64_t a = level_offset(l) + (t >> (3 * (L - l)));
                for (int32_t e = m2l_offs[a]; e < m2l_offs[a + 1]; ++e) {
                    int64_t s = m2l_ids[e];
                    double sc[3];
                    orc_cell_centre(origin3, side, l, (uint64_t)(s - level_offset(l)), sc);
                    for (int32_t i = begin[g]; i < begin[g] + count[g]; ++i)
                        orc_m2p(p, sc, M + s * nt, sxyzq + 4 * (int64_t)i, out + 4 * (int64_t)i);
                }
            }
        }
    }

    /* P2P over the near-field list */
    {
        int64_t nl = (int64_t)1 << (3 * L), off = level_offset(L);
#pragma omp parallel for schedule(dynamic, 16)
        for (int64_t t = 0; t < nl; ++t) {
            int64_t g = off + t;
            if (count[g] == 0 || !needc[g]) continue;
            for (int32_t i = begin[g]; i < begin[g] + count[g]; ++i)
                for (int32_t e = p2p_offs[t]; e < p2p_offs[t + 1]; ++e) {
                    int64_t s = p2p_ids[e];
                    p2p_one(sxyzq + 4 * (int64_t)i, count[s], sxyzq + 4 * (int64_t)begin[s], eps2,
                            out + 4 * (int64_t)i);
                }
        }
    }
    free(needc);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Adaptive octree (Cheng, Greengard & Rokhlin 1999, the adaptive FMM the paper */
/* cites): a cell splits iff it holds more than leaf_size particles and is above */
/* max_level; only nonempty children exist.  Cells are numbered level by level, */
/* in ascending key order within a level, so the children of a cell are         */
/* consecutive.                                                                 */
/* ------------------------------------------------------------------------- */

/* Eq. 3 (the L_n^m factor), P2L: L_n^m += sum_j q_j rho_j^{-n-1} Y_n^{-m}(alpha_j, beta_j),
 * (rho, alpha, beta) = x_j - centre. */
void orc_p2l(int p, const double *centre, int64_t np, const double *xyzq, double complex *L)
{
    init_fact();
    double complex Y[TRI(MAXDEG, 0) + MAXDEG];
    for (int64_t j = 0; j < np; ++j) {
        double v[3] = {xyzq[4 * j] - centre[0], xyzq[4 * j + 1] - centre[1], xyzq[4 * j + 2] - centre[2]};
        double rho, al, be;
        cart2sph(v, &rho, &al, &be);
        orc_ynm(p, al, be, Y);
        double q = xyzq[4 * j + 3];
        for (int n = 0; n < p; ++n)
            for (int m = 0; m <= n; ++m) L[TRI(n, m)] += q * pow(rho, -n - 1) * yfull(Y, n, -m);
    }
}

void orc_p2l_ri(int p, const double *centre, int64_t np, const double *xyzq, double *Lri)
{
    double complex L[NT(MAXDEG)];
    ri2c(NT(p), Lri, L);
    orc_p2l(p, centre, np, xyzq, L);
    c2ri(NT(p), L, Lri);
}

/* Build the adaptive tree from the 63-bit keys of the particles sorted ascending.
 * Outputs (capacity cap cells): level, key prefix, begin, count, parent, child_begin,
 * nchild, and level_start[0..max_level+1].  Returns the number of cells, or -1 when cap
 * is too small. */
int64_t orc_adaptive_tree(int64_t n, const uint64_t *sk, int leaf_size, int max_level, int64_t cap, int32_t *level,
                          uint64_t *key, int32_t *begin, int32_t *count, int32_t *parent, int32_t *child_begin,
                          int32_t *nchild, int32_t *level_start)
{
    if (cap < 1) return -1;
    int64_t nc = 1;
    level[0] = 0;
    key[0] = 0;
    begin[0] = 0;
    count[0] = (int32_t)n;
    parent[0] = -1;
    level_start[0] = 0;
    int64_t lo = 0, hi = 1; /* cells of the current level */
    for (int l = 0; l <= max_level; ++l) {
        level_start[l + 1] = (int32_t)hi;
        for (int64_t c = lo; c < hi; ++c) {
            child_begin[c] = (int32_t)nc;
            nchild[c] = 0;
            if (count[c] <= leaf_size || l == max_level) continue;
            const int sh = 3 * (21 - (l + 1));
            for (int32_t i = begin[c]; i < begin[c] + count[c]; ++i) {
                uint64_t ck = sk[i] >> sh;
                if (i == begin[c] || (sk[i - 1] >> sh) != ck) {
                    if (nc >= cap) return -1;
                    level[nc] = l + 1;
                    key[nc] = ck;
                    begin[nc] = i;
                    count[nc] = 0;
                    parent[nc] = (int32_t)c;
                    nc++;
                    nchild[c]++;
                }
                count[nc - 1]++;
            }
        }
        lo = hi;
        hi = nc;
        if (lo == hi) {
            for (int k = l + 2; k <= max_level + 1; ++k) level_start[k] = (int32_t)hi;
            break;
        }
    }
    return nc;
}

/* integer box of a cell at depth 21: lo[d] inclusive, size */
static void cell_box(int l, uint64_t key, int64_t *lo, int64_t *size)
{
    int64_t ix[3];
    deinterleave3(key, l, &ix[0], &ix[1], &ix[2]);
    *size = (int64_t)1 << (21 - l);
    for (int d = 0; d < 3; ++d) lo[d] = ix[d] * (*size);
}

/* two boxes touch or overlap */
static int boxes_adjacent(int la, uint64_t ka, int lb, uint64_t kb)
{
    int64_t a[3], b[3], sa, sb;
    cell_box(la, ka, a, &sa);
    cell_box(lb, kb, b, &sb);
    for (int d = 0; d < 3; ++d)
        if (a[d] > b[d] + sb || b[d] > a[d] + sa) return 0;
    return 1;
}

static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* Lists of the adaptive tree (Cheng, Greengard & Rokhlin 1999):
 *   colleagues(B): cells of B's level adjacent to B, B included (coll[27 * c], -1 padded);
 *   U(B), B leaf: leaves adjacent to B, B included, any level;
 *   V(B): children of the colleagues of B's parent that are not adjacent to B;
 *   W(B), B leaf: descendants of B's colleagues whose parent is adjacent to B but which are
 *         not adjacent to B (the descent stops there);
 *   X(B): cells C with B in W(C) -- leaves C that are colleagues of a strict ancestor of B,
 *         adjacent to B's parent and not adjacent to B.
 * Rows ascending by cell index.  kind: 0 U, 1 V, 2 W, 3 X; offs[ncells + 1]; returns entries,
 * or -1 when cap is too small. */
int64_t orc_adaptive_list(int kind, int64_t ncells, const int32_t *level, const uint64_t *key, const int32_t *parent,
                          const int32_t *child_begin, const int32_t *nchild, const int32_t *coll, int32_t *offs,
                          int32_t *ids, int64_t cap)
{
    int64_t e = 0;
    const size_t scratch = (size_t)1 << 20; /* entries per row / descent stack */
    int32_t *row = (int32_t *)malloc(sizeof(int32_t) * scratch);
    int32_t *stack = (int32_t *)malloc(sizeof(int32_t) * scratch);
    if (!row || !stack) {
        free(row);
        free(stack);
        return -1;
    }
    for (int64_t b = 0; b < ncells; ++b) {
        offs[b] = (int32_t)e;
        int nr = 0;
        const int leaf = nchild[b] == 0;
        if (kind == 1 && parent[b] >= 0) {
            const int32_t *pc = coll + 27 * (int64_t)parent[b];
            for (int i = 0; i < 27 && pc[i] >= 0; ++i)
                for (int32_t c = child_begin[pc[i]]; c < child_begin[pc[i]] + nchild[pc[i]]; ++c)
                    if (!boxes_adjacent(level[b], key[b], level[c], key[c])) row[nr++] = c;
        } else if ((kind == 0 || kind == 2) && leaf) {
            const int32_t *bc = coll + 27 * b;
            for (int i = 0; i < 27 && bc[i] >= 0; ++i) {
                const int32_t a = bc[i];
                if (nchild[a] == 0) {
                    if (kind == 0) row[nr++] = a; /* same-level leaf colleagues, B included */
                    continue;
                }
                /* descend from a non-leaf colleague */
                int sp = 0;
                for (int32_t c = child_begin[a]; c < child_begin[a] + nchild[a]; ++c) stack[sp++] = c;
                while (sp > 0) {
                    const int32_t d = stack[--sp];
                    if (boxes_adjacent(level[b], key[b], level[d], key[d])) {
                        if (nchild[d] == 0) {
                            if (kind == 0) row[nr++] = d;
                        } else {
                            for (int32_t c = child_begin[d]; c < child_begin[d] + nchild[d]; ++c) stack[sp++] = c;
                        }
                    } else if (kind == 2) {
                        row[nr++] = d;
                    }
                }
            }
            if (kind == 0) /* coarser leaves: leaf colleagues of strict ancestors adjacent to B */
                for (int32_t anc = parent[b]; anc >= 0; anc = parent[anc]) {
                    const int32_t *ac = coll + 27 * (int64_t)anc;
                    for (int i = 0; i < 27 && ac[i] >= 0; ++i)
                        if (ac[i] != anc && nchild[ac[i]] == 0 &&
                            boxes_adjacent(level[b], key[b], level[ac[i]], key[ac[i]]))
                            row[nr++] = ac[i];
                }
        } else if (kind == 3 && parent[b] >= 0) {
            const int32_t pb = parent[b];
            for (int32_t anc = pb; anc >= 0; anc = parent[anc]) {
                const int32_t *ac = coll + 27 * (int64_t)anc;
                for (int i = 0; i < 27 && ac[i] >= 0; ++i) {
                    const int32_t c = ac[i];
                    if (c == anc || nchild[c] != 0) continue;
                    if (boxes_adjacent(level[pb], key[pb], level[c], key[c]) &&
                        !boxes_adjacent(level[b], key[b], level[c], key[c]))
                        row[nr++] = c;
                }
            }
        }
        qsort(row, (size_t)nr, sizeof(int32_t), cmp_i32);
        if (e + nr > cap) {
            free(row);
            free(stack);
            return -1;
        }
        for (int i = 0; i < nr; ++i) ids[e++] = row[i];
    }
    offs[ncells] = (int32_t)e;
    free(row);
    free(stack);
    return e;
}

/* Colleagues of every cell (same level, adjacent, itself included): children of the
 * colleagues of the parent that are adjacent.  coll[27 * c] ascending, -1 padded. */
void orc_adaptive_colleagues(int64_t ncells, const int32_t *level, const uint64_t *key, const int32_t *parent,
                             const int32_t *child_begin, const int32_t *nchild, int32_t *coll)
{
    for (int64_t c = 0; c < ncells; ++c)
        for (int i = 0; i < 27; ++i) coll[27 * c + i] = -1;
    if (ncells > 0) coll[0] = 0;
    /* cells are in level order, so parents are done before their children */
    for (int64_t b = 1; b < ncells; ++b) {
        const int32_t *pc = coll + 27 * (int64_t)parent[b];
        int nr = 0;
        int32_t row[27 * 8];
        for (int i = 0; i < 27 && pc[i] >= 0; ++i)
            for (int32_t c = child_begin[pc[i]]; c < child_begin[pc[i]] + nchild[pc[i]]; ++c) {
                int64_t a[3], d[3];
                deinterleave3(key[b], level[b], &a[0], &a[1], &a[2]);
                deinterleave3(key[c], level[c], &d[0], &d[1], &d[2]);
                if (llabs(a[0] - d[0]) <= 1 && llabs(a[1] - d[1]) <= 1 && llabs(a[2] - d[2]) <= 1) row[nr++] = c;
            }
        qsort(row, (size_t)nr, sizeof(int32_t), cmp_i32);
        for (int i = 0; i < nr; ++i) coll[27 * b + i] = row[i];
    }
}

/*
 * Adaptive passes (FP64).  method 0, the FMM: P2M at the leaves, M2M up the tree, M2L over
 * V, P2L over X, L2L down the tree, L2P at the leaves, M2P over W and P2P over U.
 * method 1, the treecode (Section "Fast N-body simulation": the treecode evaluates the
 * multipole expansions at the particles, no local expansions): P2M and M2M as above, then
 * at each leaf B, M2P over W(B) and over V(A) of B and of every ancestor A, and P2P over U(B)
 * and over X(A) of B and of every ancestor A.  X(A) holds leaves adjacent to A's parent and
 * larger than A, whose multipoles do not converge at A's particles: the FMM reaches them
 * through P2L, the treecode through direct sums.  The sources reached are the FMM's, each once.
 * Particles sorted by key (sxyzq); M, Lc zero on entry (ncells * p(p+1)/2 complex,
 * interleaved; Lc unused by the treecode); out accumulates (phi, grad) in sorted order.
 * need: optional mask over cells; when given, only leaves with need set are evaluated (and
 * only the local expansions they use are formed).
 */
int orc_adaptive_passes(int p, int method, double eps2, const double *origin3, double side, int64_t ncells, const int32_t *level,
                        const uint64_t *key, const int32_t *begin, const int32_t *count, const int32_t *parent,
                        const int32_t *child_begin, const int32_t *nchild, const int32_t *level_start, int max_level,
                        const double *sxyzq, const int32_t *u_offs, const int32_t *u_ids, const int32_t *v_offs,
                        const int32_t *v_ids, const int32_t *w_offs, const int32_t *w_ids, const int32_t *x_offs,
                        const int32_t *x_ids, const uint8_t *need, double *Mri, double *Lri, double *out)
{
    init_fact();
    const int nt = NT(p);
    double complex *M = (double complex *)Mri;
    double complex *Lc = (double complex *)Lri;
    uint8_t *needc = (uint8_t *)calloc((size_t)ncells, 1);
    if (!needc) return -1;
    for (int64_t c = 0; c < ncells; ++c)
        if (nchild[c] == 0 && (!need || need[c]))
            for (int32_t a = (int32_t)c; a >= 0; a = parent[a]) needc[a] = 1;

    /* P2M at every leaf at level >= 2 */
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t c = 0; c < ncells; ++c) {
        if (nchild[c] != 0 || level[c] < 2) continue;
        double ctr[3];
        orc_cell_centre(origin3, side, level[c], key[c], ctr);
        orc_p2m(p, ctr, count[c], sxyzq + 4 * (int64_t)begin[c], M + c * nt);
    }
    /* M2M bottom-up, parents at levels max_level-1 .. 2 */
    for (int l = max_level - 1; l >= 2; --l) {
#pragma omp parallel for schedule(dynamic, 16)
        for (int64_t c = level_start[l]; c < level_start[l + 1]; ++c) {
            if (nchild[c] == 0) continue;
            double pc[3];
            orc_cell_centre(origin3, side, l, key[c], pc);
            for (int32_t ch = child_begin[c]; ch < child_begin[c] + nchild[c]; ++ch) {
                double cc[3];
                orc_cell_centre(origin3, side, l + 1, key[ch], cc);
                orc_m2m(p, cc, pc, M + ch * nt, M + c * nt);
            }
        }
    }
    if (method == 1) {
        /* treecode: every needed leaf's particles take the multipoles of W(B) and of V along
         * its ancestor chain, and the particles of U(B) and of X along that chain */
#pragma omp parallel for schedule(dynamic, 8)
        for (int64_t b = 0; b < ncells; ++b) {
            if (nchild[b] != 0 || !needc[b]) continue;
            for (int32_t i = begin[b]; i < begin[b] + count[b]; ++i) {
                const double *xi = sxyzq + 4 * (int64_t)i;
                double *oi = out + 4 * (int64_t)i;
                for (int32_t e = w_offs[b]; e < w_offs[b + 1]; ++e) {
                    const int32_t s = w_ids[e];
                    double sc[3];
                    orc_cell_centre(origin3, side, level[s], key[s], sc);
                    orc_m2p(p, sc, M + (int64_t)s * nt, xi, oi);
                }
                for (int32_t e = u_offs[b]; e < u_offs[b + 1]; ++e) {
                    const int32_t s = u_ids[e];
                    p2p_one(xi, count[s], sxyzq + 4 * (int64_t)begin[s], eps2, oi);
                }
                for (int32_t a = (int32_t)b; a >= 0; a = parent[a]) {
                    for (int32_t e = v_offs[a]; e < v_offs[a + 1]; ++e) {
                        const int32_t s = v_ids[e];
                        double sc[3];
                        orc_cell_centre(origin3, side, level[s], key[s], sc);
                        orc_m2p(p, sc, M + (int64_t)s * nt, xi, oi);
                    }
                    for (int32_t e = x_offs[a]; e < x_offs[a + 1]; ++e) {
                        const int32_t s = x_ids[e];
                        p2p_one(xi, count[s], sxyzq + 4 * (int64_t)begin[s], eps2, oi);
                    }
                }
            }
        }
        free(needc);
        return 0;
    }
    /* M2L over V and P2L over X, into every needed cell */
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t b = 0; b < ncells; ++b) {
        if (!needc[b] || level[b] < 2) continue;
        double tc[3];
        orc_cell_centre(origin3, side, level[b], key[b], tc);
        for (int32_t e = v_offs[b]; e < v_offs[b + 1]; ++e) {
            const int32_t s = v_ids[e];
            double sc[3];
            orc_cell_centre(origin3, side, level[s], key[s], sc);
            orc_m2l(p, sc, tc, M + (int64_t)s * nt, Lc + b * nt);
        }
        for (int32_t e = x_offs[b]; e < x_offs[b + 1]; ++e) {
            const int32_t s = x_ids[e];
            orc_p2l(p, tc, count[s], sxyzq + 4 * (int64_t)begin[s], Lc + b * nt);
        }
    }
    /* L2L top-down, children at levels 3 .. max_level */
    for (int l = 3; l <= max_level; ++l) {
#pragma omp parallel for schedule(dynamic, 16)
        for (int64_t c = level_start[l]; c < level_start[l + 1]; ++c) {
            if (!needc[c]) continue;
            const int32_t pa = parent[c];
            double cc[3], pc[3];
            orc_cell_centre(origin3, side, l, key[c], cc);
            orc_cell_centre(origin3, side, l - 1, key[pa], pc);
            orc_l2l(p, pc, cc, Lc + (int64_t)pa * nt, Lc + c * nt);
        }
    }
    /* L2P, M2P over W and P2P over U at the needed leaves */
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t b = 0; b < ncells; ++b) {
        if (nchild[b] != 0 || !needc[b]) continue;
        double ctr[3];
        orc_cell_centre(origin3, side, level[b], key[b], ctr);
        for (int32_t i = begin[b]; i < begin[b] + count[b]; ++i) {
            const double *xi = sxyzq + 4 * (int64_t)i;
            double *oi = out + 4 * (int64_t)i;
            if (level[b] >= 2) orc_l2p(p, ctr, Lc + b * nt, xi, oi);
            for (int32_t e = w_offs[b]; e < w_offs[b + 1]; ++e) {
                const int32_t s = w_ids[e];
                double sc[3];
                orc_cell_centre(origin3, side, level[s], key[s], sc);
                orc_m2p(p, sc, M + (int64_t)s * nt, xi, oi);
            }
            for (int32_t e = u_offs[b]; e < u_offs[b + 1]; ++e) {
                const int32_t s = u_ids[e];
                p2p_one(xi, count[s], sxyzq + 4 * (int64_t)begin[s], eps2, oi);
            }
        }
    }
    free(needc);
    return 0;
}
