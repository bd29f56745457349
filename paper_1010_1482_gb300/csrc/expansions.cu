// Expansion kernels of the FMM / treecode: translation-operator tables (FP64 arithmetic,
// stored FP32), P2M, M2M, L2L, L2P and M2P (FP32).
//
// Notation (Section "Fast N-body simulation", Eq. 2-9): Y_n^m as Eq. 6 with the
// Condon-Shortley phase of Eq. 8; regular solid harmonics R_n^m(v) = |v|^n Y_n^m(v),
// irregular I_n^m(v) = |v|^(-n-1) Y_n^m(v).  Both are evaluated from Cartesian coordinates
// with the normalised three-term recurrence in n (Eq. 7 multiplied through by |v|^n) and the
// diagonal step R_m^m = -sqrt((2m-1)/(2m)) (x + iy) R_{m-1}^{m-1} (Eq. 8), so no
// trigonometric function is needed on the device.
//
//   P2M (Eq. 2):  M_n^m = sum_j q_j R_n^{-m}(x_j - c) = sum_j q_j conj(R_n^m(x_j - c))
//   L2P (Eq. 3):  phi = sum_{n,m} L_n^m R_n^m(x - c)
//   M2P (Eq. 2):  phi = sum_{n,m} M_n^m I_n^m(x - c)
// Gradients use the ladder relations of solid harmonics (d/dz and d/dx + i d/dy lower or
// raise the degree by one), which stay finite on the expansion's z axis.
// M2L (Eq. 4-5) and the M2M / L2L translations (Cheng, Greengard & Rokhlin 1999, cited by
// the paper for its translation operators) are linear maps on the real-packed coefficients;
// with coefficients scaled by the cell side they do not depend on the level, so each is a
// dense p^2 x p^2 FP32 matrix computed once per order in FP64.
#include "common.cuh"

#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

namespace gbfmm {

#define GBFMM_DISPATCH_P(P, CALL)      \
    switch (P) {                       \
    case 4: { constexpr int PQ = 4; CALL; } break;   \
    case 6: { constexpr int PQ = 6; CALL; } break;   \
    case 8: { constexpr int PQ = 8; CALL; } break;   \
    case 10: { constexpr int PQ = 10; CALL; } break; \
    }

constexpr int kMaxP = 10;
constexpr int kMaxDeg = 2 * kMaxP;  // harmonics up to degree 2P-2 (M2L) and P (M2P gradient)

// Recurrence and ladder constants, set once per device (init_expansion_constants).
__constant__ float c_rmm[kMaxDeg + 1];                 // sqrt((2m-1)/(2m))
__constant__ float c_ra[kMaxDeg + 1][kMaxDeg + 1];     // (2n+1) / sqrt((n+1-m)(n+1+m))
__constant__ float c_rb[kMaxDeg + 1][kMaxDeg + 1];     // sqrt((n-m)(n+m)) / sqrt((n+1-m)(n+1+m))
__constant__ float c_sq[2 * kMaxDeg + 4][2 * kMaxDeg + 4];  // sqrt(a*b)

void init_expansion_constants()
{
    float rmm[kMaxDeg + 1], ra[kMaxDeg + 1][kMaxDeg + 1], rb[kMaxDeg + 1][kMaxDeg + 1];
    static float sq[2 * kMaxDeg + 4][2 * kMaxDeg + 4];
    for (int m = 0; m <= kMaxDeg; ++m) rmm[m] = m ? (float)sqrt((2.0 * m - 1.0) / (2.0 * m)) : 0.f;
    for (int n = 0; n <= kMaxDeg; ++n)
        for (int m = 0; m <= kMaxDeg; ++m) {
            double den = (double)(n + 1 - m) * (double)(n + 1 + m);
            ra[n][m] = (m <= n) ? (float)((2.0 * n + 1.0) / sqrt(den)) : 0.f;
            rb[n][m] = (m <= n) ? (float)(sqrt((double)(n - m) * (double)(n + m)) / sqrt(den)) : 0.f;
        }
    for (int a = 0; a < 2 * kMaxDeg + 4; ++a)
        for (int b = 0; b < 2 * kMaxDeg + 4; ++b) sq[a][b] = (float)sqrt((double)a * (double)b);
    cudaMemcpyToSymbol(c_rmm, rmm, sizeof(rmm));
    cudaMemcpyToSymbol(c_ra, ra, sizeof(ra));
    cudaMemcpyToSymbol(c_rb, rb, sizeof(rb));
    cudaMemcpyToSymbol(c_sq, sq, sizeof(sq));
}

// real-packed index of Re C_n^m / Im C_n^m
GB_HD constexpr int re_idx(int n, int m) { return m == 0 ? n * n : n * n + 2 * m - 1; }
GB_HD constexpr int im_idx(int n, int m) { return n * n + 2 * m; }

// ------------------------------------------------------------------------------------------
// Operator tables (FP64 arithmetic, one CTA per operator).
// All three column-major, [op][col][row], rows padded to PR = round_up(p^2, 8) with zeros:
//   M2L  code < 343 (offset source - target, in cells)
//   M2M  child position c (bit0 x, bit1 y, bit2 z), child -> parent
//   L2L  parent -> child c
// ------------------------------------------------------------------------------------------
struct C64 {
    double re, im;
};
GB_HD C64 cmul(C64 a, C64 b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
GB_HD C64 conj64(C64 a) { return {a.re, -a.im}; }

GB_HD void dof_decode(int i, int &n, int &m, int &im)
{
    n = 0;
    while ((n + 1) * (n + 1) <= i) ++n;
    int r = i - n * n;
    if (r == 0) {
        m = 0;
        im = 0;
    } else {
        m = (r + 1) / 2;
        im = (r % 2 == 0);
    }
}

GB_HD double fact64(int k)
{
    double f = 1.0;
    for (int i = 2; i <= k; ++i) f *= i;
    return f;
}
GB_HD double Anm64(int n, int m) { return 1.0 / sqrt(fact64(n - m) * fact64(n + m)); }
GB_HD double ipow_even(int e) { return ((e / 2) % 2 == 0) ? 1.0 : -1.0; }

// regular (irreg = 0) or irregular (irreg = 1) solid harmonics H[n(n+1)/2 + m], m >= 0, n < nmax
GB_HD void harmonics64(int nmax, double x, double y, double z, int irreg, C64 *H)
{
    double r2 = x * x + y * y + z * z;
    double ir2 = 1.0 / r2;
    C64 hmm = {irreg ? 1.0 / sqrt(r2) : 1.0, 0.0};
    for (int m = 0; m < nmax; ++m) {
        if (m > 0) {
            double f = -sqrt((2.0 * m - 1.0) / (2.0 * m)) * (irreg ? ir2 : 1.0);
            C64 t = cmul(C64{x, y}, hmm);
            hmm = {f * t.re, f * t.im};
        }
        H[m * (m + 1) / 2 + m] = hmm;
        for (int n = m; n + 1 < nmax; ++n) {
            C64 a = H[n * (n + 1) / 2 + m];
            C64 b = (n - 1 >= m) ? H[(n - 1) * n / 2 + m] : C64{0.0, 0.0};
            double s = sqrt((double)(n - m) * (double)(n + m));
            double d = 1.0 / sqrt((double)(n + 1 - m) * (double)(n + 1 + m));
            double ca = (2.0 * n + 1.0) * z, cb = s * (irreg ? 1.0 : r2);
            C64 v = {(ca * a.re - cb * b.re) * d, (ca * a.im - cb * b.im) * d};
            if (irreg) {
                v.re *= ir2;
                v.im *= ir2;
            }
            H[(n + 1) * (n + 2) / 2 + m] = v;
        }
    }
}

GB_HD C64 hfull(const C64 *H, int n, int m)
{
    return m >= 0 ? H[n * (n + 1) / 2 + m] : conj64(H[n * (n + 1) / 2 - m]);
}

// complex coefficient of input C_n^m in output D_j^k for the three operators
GB_HD C64 k_m2l(const C64 *I, int j, int k, int n, int m)
{
    double f = ipow_even(abs(k - m) - abs(k) - abs(m)) * Anm64(n, m) * Anm64(j, k) / Anm64(j + n, m - k) *
               ((j & 1) ? -1.0 : 1.0);
    C64 h = hfull(I, j + n, m - k);
    return {f * h.re, f * h.im};
}

GB_DEV C64 k_m2m(const C64 *R, int j, int k, int n, int m)
{
    if (j < n || abs(k - m) > j - n) return {0.0, 0.0};
    int nn = j - n, mm = k - m;
    double f = ipow_even(abs(k) - abs(mm) - abs(k - mm)) * Anm64(nn, mm) * Anm64(n, m) / Anm64(j, k) / ldexp(1.0, j);
    C64 h = hfull(R, nn, -mm);
    return {f * h.re, f * h.im};
}

GB_DEV C64 k_l2l(const C64 *R, int j, int k, int n, int m)
{
    if (n < j || abs(m - k) > n - j) return {0.0, 0.0};
    double f = ipow_even(abs(m) - abs(m - k) - abs(k)) * Anm64(n - j, m - k) * Anm64(j, k) / Anm64(n, m) /
               ldexp(1.0, n + 1);
    C64 h = hfull(R, n - j, m - k);
    return {f * h.re, f * h.im};
}

__global__ void k_build_ops(int P, float *m2l, float *m2m, float *l2l)
{
    __shared__ C64 H[(2 * kMaxP) * (2 * kMaxP + 1) / 2];
    const int op = blockIdx.x;
    const int PP = P * P;
    int kind;  // 0 m2l, 1 m2m, 2 l2l
    double v[3];
    bool used = true;
    if (op < kM2LCodes) {
        kind = 0;
        int dx = op % 7 - 3, dy = (op / 7) % 7 - 3, dz = op / 49 - 3;
        used = !(abs(dx) <= 1 && abs(dy) <= 1 && abs(dz) <= 1);
        v[0] = dx;  // target centre - source centre = -(source - target); the list stores
        v[1] = dy;  // source - target, so the operator is built for the negated offset below
        v[2] = dz;
        v[0] = -v[0];
        v[1] = -v[1];
        v[2] = -v[2];
    } else {
        int c = (op - kM2LCodes) % 8;
        kind = (op - kM2LCodes) < 8 ? 1 : 2;
        v[0] = (c & 1) - 0.5;  // child centre - parent centre, in child cells
        v[1] = ((c >> 1) & 1) - 0.5;
        v[2] = ((c >> 2) & 1) - 0.5;
    }
    if (threadIdx.x == 0 && used) harmonics64(kind == 0 ? 2 * P - 1 : P, v[0], v[1], v[2], kind == 0, H);
    __syncthreads();
    const int PR = (PP + 7) / 8 * 8;
    float *table = kind == 0 ? m2l + (size_t)op * PP * PR
                 : kind == 1 ? m2m + (size_t)(op - kM2LCodes) * PP * PR
                             : l2l + (size_t)(op - kM2LCodes - 8) * PP * PR;
    for (int e = threadIdx.x; e < PP * (PR - PP); e += blockDim.x)  // zero padding rows
        table[(size_t)(e / (PR - PP)) * PR + PP + e % (PR - PP)] = 0.f;
    for (int e = threadIdx.x; e < PP * PP; e += blockDim.x) {
        int row = e / PP, col = e % PP;
        float out = 0.f;
        if (used) {
            int j, k, rim, n, m, cim;
            dof_decode(row, j, k, rim);
            dof_decode(col, n, m, cim);
            C64 u = cim ? C64{0.0, 1.0} : C64{1.0, 0.0};
            C64 a, b = {0.0, 0.0};
            if (kind == 0) {
                a = k_m2l(H, j, k, n, m);
                if (m > 0) b = k_m2l(H, j, k, n, -m);
            } else if (kind == 1) {
                a = k_m2m(H, j, k, n, m);
                if (m > 0) b = k_m2m(H, j, k, n, -m);
            } else {
                a = k_l2l(H, j, k, n, m);
                if (m > 0) b = k_l2l(H, j, k, n, -m);
            }
            C64 val = cmul(a, u);
            C64 w = cmul(b, conj64(u));
            val.re += w.re;
            val.im += w.im;
            out = (float)(rim ? val.im : val.re);
        }
        table[(size_t)col * PR + row] = out;
    }
}

void launch_build_operators(int P, float *m2l_ops, float *m2m_ops, float *l2l_ops, cudaStream_t s)
{
    k_build_ops<<<kM2LCodes + 16, 256, 0, s>>>(P, m2l_ops, m2m_ops, l2l_ops);
    note_launches(1);
}

// ------------------------------------------------------------------------------------------
// Rotation factors of the M2L operators (host, FP64).  For an offset code with translation
// v = target centre - source centre and a rotation Q taking v / |v| to +z,
//   T_v = F^-1 C_|v| F,
// F: block-diagonal in the degree, the map of a degree-n coefficient block under the change
//    of frame x -> Q x (multipole and local blocks alike: both are sums of q f(rho) R_n^-m);
//    found by least squares from the blocks of point charges at sample directions and at their
//    rotated images (the map is exactly linear, so the fit is exact up to rounding);
// F^-1: the same for Q^T;
// C: the M2L operator of the coaxial translation (0, 0, |v|), which couples equal orders only,
//    with one real coefficient for the real and the imaginary parts.
// The factorisation is checked against the dense operator before it is used.
// Layout per code (kM2LCodes slots of m2l_rot_code_floats): F blocks (n = 0..P-1, (2n+1)^2 each,
// [row][col]), F^-1 blocks, then C blocks (m = 0..P-1, (P-m)^2 each, [j-m][n-m]), zero padding.
// ------------------------------------------------------------------------------------------
namespace {

void packed_block_regular(int n, const double x[3], double *out)
{
    C64 H[(kMaxDeg + 1) * (kMaxDeg + 2) / 2];
    harmonics64(n + 1, x[0], x[1], x[2], 0, H);
    for (int m = 0; m <= n; ++m) {
        const C64 r = H[n * (n + 1) / 2 + m];  // the block holds conj(R_n^m)
        if (m == 0) {
            out[0] = r.re;
        } else {
            out[2 * m - 1] = r.re;
            out[2 * m] = -r.im;
        }
    }
}

// solve G X = B for X (s x s, G symmetric positive definite), partial pivoting
bool solve_dense(int s, std::vector<double> G, std::vector<double> &B)
{
    for (int c = 0; c < s; ++c) {
        int piv = c;
        for (int r = c + 1; r < s; ++r)
            if (fabs(G[r * s + c]) > fabs(G[piv * s + c])) piv = r;
        if (fabs(G[piv * s + c]) < 1e-300) return false;
        if (piv != c)
            for (int k = 0; k < s; ++k) {
                std::swap(G[c * s + k], G[piv * s + k]);
                std::swap(B[c * s + k], B[piv * s + k]);
            }
        for (int r = 0; r < s; ++r) {
            if (r == c) continue;
            const double f = G[r * s + c] / G[c * s + c];
            if (f == 0.0) continue;
            for (int k = 0; k < s; ++k) {
                G[r * s + k] -= f * G[c * s + k];
                B[r * s + k] -= f * B[c * s + k];
            }
        }
    }
    for (int r = 0; r < s; ++r)
        for (int k = 0; k < s; ++k) B[r * s + k] /= G[r * s + r];
    return true;
}

// F_n for the frame change x -> Q x, row-major (2n+1)^2
bool rotation_block(int n, const double Q[9], double *F)
{
    const int s = 2 * n + 1, K = 2 * s + 3;
    std::vector<double> G(s * s, 0.0), Hm(s * s, 0.0), p(s), q(s);
    for (int i = 0; i < K; ++i) {
        double x[3] = {sin(1.31 * i + 0.7), cos(2.17 * i + 0.23), sin(0.93 * i + 1.1) + 0.3 * cos(3.7 * i)};
        const double nx = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
        for (double &c : x) c /= nx;
        const double y[3] = {Q[0] * x[0] + Q[1] * x[1] + Q[2] * x[2], Q[3] * x[0] + Q[4] * x[1] + Q[5] * x[2],
                             Q[6] * x[0] + Q[7] * x[1] + Q[8] * x[2]};
        packed_block_regular(n, x, p.data());
        packed_block_regular(n, y, q.data());
        for (int a = 0; a < s; ++a)
            for (int b = 0; b < s; ++b) {
                G[a * s + b] += p[a] * p[b];
                Hm[a * s + b] += p[a] * q[b];  // (sum p q^T): F^T = G^-1 (sum p q^T)
            }
    }
    if (!solve_dense(s, G, Hm)) return false;
    for (int a = 0; a < s; ++a)
        for (int b = 0; b < s; ++b) F[a * s + b] = Hm[b * s + a];
    return true;
}

// the dense M2L operator (real-packed, [row][col]) of translation v, as k_build_ops builds it
void dense_m2l(int P, const double v[3], std::vector<double> &T)
{
    const int PP = P * P;
    std::vector<C64> H((2 * kMaxP) * (2 * kMaxP + 1) / 2);
    harmonics64(2 * P - 1, v[0], v[1], v[2], 1, H.data());
    T.assign((size_t)PP * PP, 0.0);
    for (int row = 0; row < PP; ++row)
        for (int col = 0; col < PP; ++col) {
            int j, k, rim, n, m, cim;
            dof_decode(row, j, k, rim);
            dof_decode(col, n, m, cim);
            const C64 u = cim ? C64{0.0, 1.0} : C64{1.0, 0.0};
            const C64 a = k_m2l(H.data(), j, k, n, m);
            const C64 b = m > 0 ? k_m2l(H.data(), j, k, n, -m) : C64{0.0, 0.0};
            C64 val = cmul(a, u);
            const C64 w = cmul(b, conj64(u));
            val.re += w.re;
            val.im += w.im;
            T[(size_t)row * PP + col] = rim ? val.im : val.re;
        }
}

}  // namespace

// floats per code: F, F^-1 and C, padded to a multiple of 4 (16-byte aligned codes)
size_t m2l_rot_code_floats(int P)
{
    size_t f = 0, c = 0;
    for (int n = 0; n < P; ++n) f += (size_t)(2 * n + 1) * (2 * n + 1);
    for (int m = 0; m < P; ++m) c += (size_t)(P - m) * (P - m);
    return (2 * f + c + 3) / 4 * 4;
}

int build_m2l_rot_table(int P, std::vector<float> &out)
{
    const int PP = P * P;
    const size_t RS = m2l_rot_code_floats(P);
    out.assign(RS * kM2LCodes, 0.f);
    std::vector<double> T, Cz, Fd((size_t)PP * PP), Fi((size_t)PP * PP);
    for (int code = 0; code < kM2LCodes; ++code) {
        const int dx = code % 7 - 3, dy = (code / 7) % 7 - 3, dz = code / 49 - 3;
        if (abs(dx) <= 1 && abs(dy) <= 1 && abs(dz) <= 1) continue;
        const double v[3] = {-(double)dx, -(double)dy, -(double)dz};  // target centre - source centre
        const double d = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        const double u[3] = {v[0] / d, v[1] / d, v[2] / d};
        double Q[9];  // rotation taking u to +z (Rodrigues about u x z)
        const double ax = u[1], ay = -u[0], s2 = ax * ax + ay * ay, c = u[2];
        if (s2 < 1e-30) {
            const double sg = c > 0 ? 1.0 : -1.0;  // u = +-z: identity or a half turn about x
            const double Qi[9] = {1, 0, 0, 0, sg, 0, 0, 0, sg};
            memcpy(Q, Qi, sizeof(Q));
        } else {
            const double sn = sqrt(s2), kx = ax / sn, ky = ay / sn, t = 1.0 - c;
            const double Qi[9] = {c + kx * kx * t, kx * ky * t, ky * sn, kx * ky * t, c + ky * ky * t, -kx * sn,
                                  -ky * sn, kx * sn, c};
            memcpy(Q, Qi, sizeof(Q));
        }
        const double Qt[9] = {Q[0], Q[3], Q[6], Q[1], Q[4], Q[7], Q[2], Q[5], Q[8]};
        const double z[3] = {0.0, 0.0, d};
        dense_m2l(P, v, T);
        dense_m2l(P, z, Cz);
        std::fill(Fd.begin(), Fd.end(), 0.0);
        std::fill(Fi.begin(), Fi.end(), 0.0);
        float *o = out.data() + RS * code;
        size_t at = 0;
        for (int pass = 0; pass < 2; ++pass)
            for (int n = 0; n < P; ++n) {
                const int s = 2 * n + 1;
                std::vector<double> B(s * s);
                if (!rotation_block(n, pass == 0 ? Q : Qt, B.data())) return -1;
                for (int a = 0; a < s; ++a)
                    for (int b = 0; b < s; ++b) {
                        (pass == 0 ? Fd : Fi)[(size_t)(n * n + a) * PP + n * n + b] = B[a * s + b];
                        o[at++] = (float)B[a * s + b];
                    }
            }
        // C: equal orders only, one coefficient for real and imaginary parts
        double cmax = 0.0, off = 0.0, imdiff = 0.0;
        for (int r = 0; r < PP; ++r)
            for (int cc = 0; cc < PP; ++cc) cmax = fmax(cmax, fabs(Cz[(size_t)r * PP + cc]));
        for (int r = 0; r < PP; ++r)
            for (int cc = 0; cc < PP; ++cc) {
                int j, k, rim, n, m, cim;
                dof_decode(r, j, k, rim);
                dof_decode(cc, n, m, cim);
                if (k != m || rim != cim) off = fmax(off, fabs(Cz[(size_t)r * PP + cc]));
            }
        for (int m = 0; m < P; ++m)
            for (int j = m; j < P; ++j)
                for (int n = m; n < P; ++n) {
                    const double cre = Cz[(size_t)(m == 0 ? j * j : j * j + 2 * m - 1) * PP + (m == 0 ? n * n : n * n + 2 * m - 1)];
                    if (m > 0) imdiff = fmax(imdiff, fabs(cre - Cz[(size_t)(j * j + 2 * m) * PP + n * n + 2 * m]));
                    o[at++] = (float)cre;
                }
        if (off > 1e-12 * cmax || imdiff > 1e-12 * cmax) return -2;
        // F^-1 C F against the dense operator
        std::vector<double> CF((size_t)PP * PP, 0.0);
        for (int r = 0; r < PP; ++r)
            for (int k2 = 0; k2 < PP; ++k2) {
                const double cv = Cz[(size_t)r * PP + k2];
                if (cv == 0.0) continue;
                for (int cc = 0; cc < PP; ++cc) CF[(size_t)r * PP + cc] += cv * Fd[(size_t)k2 * PP + cc];
            }
        double err = 0.0, tmax = 0.0;
        for (int r = 0; r < PP; ++r)
            for (int cc = 0; cc < PP; ++cc) {
                double acc = 0.0;
                for (int k2 = 0; k2 < PP; ++k2) acc += Fi[(size_t)r * PP + k2] * CF[(size_t)k2 * PP + cc];
                err = fmax(err, fabs(acc - T[(size_t)r * PP + cc]));
                tmax = fmax(tmax, fabs(T[(size_t)r * PP + cc]));
            }
        if (err > 1e-9 * tmax) return -3;
    }
    return 0;
}

// ------------------------------------------------------------------------------------------
// FP32 helpers
// ------------------------------------------------------------------------------------------
struct CellGeom {
    float cx, cy, cz, inv_h;
};

// ------------------------------------------------------------------------------------------
// Cell geometry tables.  The centre of a level-l cell with integer coordinates (ix, iy, iz) is
// origin + (i + 1/2) h_l per axis, h_l = side / 2^l, and its inverse side 1 / h_l: FP64
// expressions rounded to FP32.  FP64 runs at a small fraction of the FP32 rate, so they are
// evaluated once per level and axis (uniform tree) or once per cell (adaptive tree) into a
// table that the expansion kernels read, instead of once per particle or per (particle, cell)
// pair.
//   uniform: geo[l] = 1/h_l for l < kGeoLevels, then for l = 0..L the 2^l centre coordinates
//            along x, then y, then z, at offset kGeoLevels + 3 (2^l - 1)
//   adaptive: geom[c] = (cx, cy, cz, 1/h) of cell c
// ------------------------------------------------------------------------------------------
__global__ void k_geo_levels(const Box *__restrict__ box, int L, float *__restrict__ geo)
{
    const Box b = *box;
    const int64_t total = kGeoLevels + 3 * ((int64_t(2) << L) - 1);
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        if (t < kGeoLevels) {
            const double h = b.side / (double)(int64_t(1) << t);
            geo[t] = (float)(1.0 / h);
            continue;
        }
        const int64_t u = t - kGeoLevels;
        int l = 0;
        while (3 * ((int64_t(2) << l) - 1) <= u) ++l;
        const int64_t r = u - 3 * ((int64_t(1) << l) - 1);
        const int d = (int)(r >> l);
        const int i = (int)(r - ((int64_t)d << l));
        const double h = b.side / (double)(int64_t(1) << l);
        geo[t] = (float)(b.origin[d] + (i + 0.5) * h);
    }
}

void launch_geo_levels(const Box *box, int L, float *geo, cudaStream_t s)
{
    const int64_t total = kGeoLevels + 3 * ((int64_t(2) << L) - 1);
    k_geo_levels<<<(unsigned)std::min<int64_t>((total + 255) / 256, 1024), 256, 0, s>>>(box, L, geo);
    note_launches(1);
}

GB_DEV CellGeom geo_level_cell(const float *__restrict__ geo, int l, uint32_t key)
{
    int ix, iy, iz;
    demorton3(key, ix, iy, iz);
    const float *a = geo + kGeoLevels + 3 * ((1 << l) - 1);
    CellGeom g;
    g.cx = __ldg(a + ix);
    g.cy = __ldg(a + (1 << l) + iy);
    g.cz = __ldg(a + (2 << l) + iz);
    g.inv_h = __ldg(geo + l);
    return g;
}

GB_DEV CellGeom geo_cell(const float4 *__restrict__ geom, int64_t c)
{
    const float4 v = __ldg(&geom[c]);
    CellGeom g;
    g.cx = v.x;
    g.cy = v.y;
    g.cz = v.z;
    g.inv_h = v.w;
    return g;
}

// ------------------------------------------------------------------------------------------
// P2M: one warp per leaf; lanes stride over the leaf's particles, each accumulates the full
// real-packed expansion in registers, then a butterfly reduction sums the lanes.
// ------------------------------------------------------------------------------------------
// acc += sum over particles j = b0 + lane, b0 + lane + 32, ... < e0 of q_j conj(H_n^m(x^_j)),
// x^ = (x - c) / h, with H the regular harmonics R (P2M, Eq. 2) or the irregular harmonics I
// (P2L, Eq. 3), real-packed
template <int P, bool IRREG>
GB_DEV void p2x_particles(float (&acc)[P * P], const float4 *__restrict__ sx, int b0, int e0, int lane,
                          const CellGeom &cg)
{
    for (int j = b0 + lane; j < e0; j += 32) {
        float4 p = __ldg(&sx[j]);
        const float x = (p.x - cg.cx) * cg.inv_h, y = (p.y - cg.cy) * cg.inv_h, z = (p.z - cg.cz) * cg.inv_h;
        const float q = p.w, r2 = x * x + y * y + z * z;
        const float ir = IRREG ? rsqrt_ftz(r2) : 1.f;
        const float ir2 = ir * ir;
        float mre = ir, mim = 0.f;  // H_m^m
#pragma unroll
        for (int m = 0; m < P; ++m) {
            if (m > 0) {
                const float f = -c_rmm[m] * ir2;
                const float tr = f * (x * mre - y * mim), ti = f * (x * mim + y * mre);
                mre = tr;
                mim = ti;
            }
            float are = mre, aim = mim, bre = 0.f, bim = 0.f;  // H_n^m, H_{n-1}^m
#pragma unroll
            for (int n = m; n < P; ++n) {
                if (n > m) {
                    const float ca = c_ra[n - 1][m] * z, cb = c_rb[n - 1][m] * (IRREG ? 1.f : r2);
                    float nre = ca * are - cb * bre, nim = ca * aim - cb * bim;
                    if (IRREG) {
                        nre *= ir2;
                        nim *= ir2;
                    }
                    bre = are;
                    bim = aim;
                    are = nre;
                    aim = nim;
                }
                acc[re_idx(n, m)] += q * are;
                if (m > 0) acc[im_idx(n, m)] -= q * aim;
            }
        }
    }
}

// Warp-wide sum of acc over the lanes, stored to (or added into) dst: a transpose through the
// warp's shared-memory scratch in two halves of the coefficients (each lane writes its row,
// then lane j sums column j over the 32 rows).  scr holds 32 x (WS_H + 1) floats.
template <int P>
struct WarpSum {
    static constexpr int PP = P * P, H = (PP + 1) / 2, LD = H + 1;
};

template <int P>
GB_DEV void warp_store(float (&acc)[P * P], float *dst, int lane, bool add, float *scr)
{
    using W = WarpSum<P>;
#pragma unroll
    for (int part = 0; part < 2; ++part) {
        __syncwarp();
#pragma unroll
        for (int i = 0; i < W::H; ++i)
            if (part * W::H + i < W::PP) scr[lane * W::LD + i] = acc[part * W::H + i];
        __syncwarp();
        for (int i = lane; i < W::H && part * W::H + i < W::PP; i += 32) {
            float v = 0.f;
#pragma unroll 8
            for (int r = 0; r < 32; ++r) v += scr[r * W::LD + i];
            float *d = dst + part * W::H + i;
            *d = add ? *d + v : v;
        }
    }
}

template <int P>
__global__ void __launch_bounds__(128) k_p2m(int L, const float *__restrict__ geo, const float4 *__restrict__ sx,
                                             const int32_t *__restrict__ begin, const int32_t *__restrict__ end,
                                             float *__restrict__ M)
{
    __shared__ float scr[4][32 * WarpSum<P>::LD];
    const int lane = threadIdx.x & 31;
    const int64_t leaf = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
    if (leaf >= (int64_t(1) << (3 * L))) return;
    const int64_t g = level_offset(L) + leaf;
    const int b0 = begin[g], e0 = end[g];
    if (e0 <= b0) return;
    const CellGeom cg = geo_level_cell(geo, L, (uint32_t)leaf);
    float acc[P * P];
#pragma unroll
    for (int i = 0; i < P * P; ++i) acc[i] = 0.f;
    p2x_particles<P, false>(acc, sx, b0, e0, lane, cg);
    warp_store<P>(acc, M + g * (P * P), lane, false, scr[threadIdx.x >> 5]);
}

void launch_p2m(int P, int L, const float *geo, const float4 *sx, const int32_t *begin, const int32_t *end, float *M,
                cudaStream_t s)
{
    int64_t nl = int64_t(1) << (3 * L);
    unsigned grid = (unsigned)((nl + 3) / 4);
    switch (P) {
    case 4: k_p2m<4><<<grid, 128, 0, s>>>(L, geo, sx, begin, end, M); break;
    case 6: k_p2m<6><<<grid, 128, 0, s>>>(L, geo, sx, begin, end, M); break;
    case 8: k_p2m<8><<<grid, 128, 0, s>>>(L, geo, sx, begin, end, M); break;
    case 10: k_p2m<10><<<grid, 128, 0, s>>>(L, geo, sx, begin, end, M); break;
    }
    note_launches(1);
}

// ------------------------------------------------------------------------------------------
// M2M and L2L as batched FP32 contractions over 32 cells per CTA, the same register-blocked
// micro-kernel as M2L (4 operator rows x 8 cells per thread) on shared-memory-staged operands.
//   M2M (UP):  M~(parent q) = sum over child positions c of T^M2M_c M~(child 8q + c)
//   L2L (!UP): L~(child 8q + c) += T^L2L_c L~(parent q), one child position per CTA column
// M2M is block lower-triangular in degree (output degree j reads input degrees <= j) and L2L
// block upper-triangular (reads degrees >= j): each thread's k range is cut to its rows'
// degrees (rounded to whole k-groups of 4).
// ------------------------------------------------------------------------------------------
constexpr int kTrTN = 32, kTrCN = 8;

template <int P, bool UP, int TN = kTrTN, int CN = kTrCN>
struct TransCfg {
    static constexpr int PP = P * P, PR = ops_rows_padded(P), SB = staged_col_stride(P);
    static constexpr int NCG = TN / CN, NRG = PR / 4, NT = ((NRG * NCG + 31) / 32) * 32;
    static constexpr int AF = PP * PR, BF = TN * SB;  // floats of one operator / one column block
    static constexpr int NBUF = UP ? 2 : 1;           // M2M walks 8 child positions: double-buffered
    static constexpr size_t kSmem = (size_t)NBUF * (AF + BF) * sizeof(float);
};

GB_DEV int degree_of(int r)
{
    int d = 0;
    while ((d + 1) * (d + 1) <= r) ++d;
    return d;
}

GB_DEV void cp_async16_t(void *dst, const void *src, uint32_t src_bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(src_bytes)
                 : "memory");
}

// TN cells per CTA; the operator of each child position and the TN source columns are copied
// into shared memory with cp.async (zero-filled for missing cells), the next child position's
// copies in flight while the current one is applied
template <int P, bool UP, int TN, int CN>
__global__ void __launch_bounds__(TransCfg<P, UP, TN, CN>::NT) k_translate(int l, const int32_t *__restrict__ begin,
                                                                       const int32_t *__restrict__ end,
                                                                       const float *__restrict__ ops,
                                                                       float *__restrict__ X)
{
    using Cfg = TransCfg<P, UP, TN, CN>;
    constexpr int PP = Cfg::PP, PR = Cfg::PR, SB = Cfg::SB, NCG = Cfg::NCG, NRG = Cfg::NRG;
    extern __shared__ __align__(16) float tsm[];
    // parents: level l (M2M) or l - 1 (L2L)
    const int lp = UP ? l : l - 1;
    const int64_t np = int64_t(1) << (3 * lp);
    const int64_t q0 = blockIdx.x * (int64_t)TN;
    const int64_t offp = level_offset(lp), offc = level_offset(lp + 1);
    const int tid = threadIdx.x;
    const bool work = tid < NRG * NCG;
    const int cg = tid % NCG, rg = tid / NCG;
    int kbeg = 0, kend = PP;
    if (work) {
        const int r0 = min(rg * 4, PP - 1), r1 = min(rg * 4 + 3, PP - 1);
        if (UP) {
            const int d = degree_of(r1);
            kend = min(PP, ((d + 1) * (d + 1) + 3) / 4 * 4);
        } else {
            const int d = degree_of(r0);
            kbeg = (d * d) / 4 * 4;
        }
    }
    auto stage = [&](int c, int buf) {
        float *A = tsm + buf * (Cfg::AF + Cfg::BF);
        float *B = A + Cfg::AF;
        const float *src = ops + (size_t)c * PP * PR;
        for (int e = tid; e < PP * PR / 4; e += blockDim.x) cp_async16_t(A + 4 * e, src + 4 * e, 16u);
        for (int e = tid; e < TN * (PP / 4); e += blockDim.x) {
            const int i = e / (PP / 4), k4 = e % (PP / 4);
            const int64_t q = q0 + i;
            const float *gsrc = X;
            uint32_t bytes = 0;
            if (q < np) {
                const int64_t g = UP ? offc + 8 * q + c : offp + q;
                if (end[g] > begin[g]) {
                    gsrc = X + g * PP + 4 * k4;
                    bytes = 16u;
                }
            }
            cp_async16_t(B + i * SB + 4 * k4, gsrc, bytes);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    float acc[4][CN];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < CN; ++j) acc[i][j] = 0.f;
    const int c_first = UP ? 0 : blockIdx.y, c_last = UP ? 7 : blockIdx.y;
    stage(c_first, 0);
    for (int c = c_first; c <= c_last; ++c) {
        const int buf = UP ? (c - c_first) & 1 : 0;
        if (c < c_last) {
            stage(c + 1, buf ^ 1);
            asm volatile("cp.async.wait_group 1;" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        __syncthreads();
        if (work) {
            const float *Ar = tsm + buf * (Cfg::AF + Cfg::BF) + rg * 4;
            const float *Bc = tsm + buf * (Cfg::AF + Cfg::BF) + Cfg::AF + cg * SB;
#pragma unroll 2
            for (int k = kbeg; k < kend; k += 4) {
                Frag<CN, 4> f;
                f.load(Ar, Bc, k, PR, NCG * SB);
                f.fma(acc);
            }
        }
        __syncthreads();  // the buffer is refilled two positions later
    }
    if (!work) return;
#pragma unroll
    for (int j = 0; j < CN; ++j) {
        const int64_t q = q0 + cg + j * NCG;
        if (q >= np) continue;
        const int r = rg * 4;
        if (r >= PP) continue;
        const int64_t g = UP ? offp + q : offc + 8 * q + blockIdx.y;
        if (end[g] <= begin[g]) continue;
        float4 *dst = reinterpret_cast<float4 *>(X + g * PP + r);
        if (UP) {
            *dst = make_float4(acc[0][j], acc[1][j], acc[2][j], acc[3][j]);
        } else {
            float4 v = *dst;
            v.x += acc[0][j];
            v.y += acc[1][j];
            v.z += acc[2][j];
            v.w += acc[3][j];
            *dst = v;
        }
    }
}

template <int P, bool UP, int TN, int CN>
static void launch_translate_tn(int l, const int32_t *begin, const int32_t *end, const float *ops, float *X,
                                cudaStream_t s)
{
    using Cfg = TransCfg<P, UP, TN, CN>;
    cudaFuncSetAttribute(k_translate<P, UP, TN, CN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::kSmem);
    const int64_t np = int64_t(1) << (3 * (UP ? l : l - 1));
    dim3 grid((unsigned)((np + TN - 1) / TN), UP ? 1 : 8);
    k_translate<P, UP, TN, CN><<<grid, Cfg::NT, Cfg::kSmem, s>>>(l, begin, end, ops, X);
    note_launches(1);
}

// cells per CTA: 32 (8 per thread) when the level has enough cells to fill the GPU twice over,
// else 16 (2 per thread): small levels are bound by the latency of staging the operators, and
// seven times the threads per cell cut it (M2M levels 2-4 of a 2^20-particle p = 10 tree:
// 150 us -> 68 us)
template <int P, bool UP>
static void launch_translate_t(int l, const int32_t *begin, const int32_t *end, const float *ops, float *X,
                               cudaStream_t s)
{
    const int64_t np = int64_t(1) << (3 * (UP ? l : l - 1));
    const int64_t ctas32 = (np + 31) / 32 * (UP ? 1 : 8);
    if (ctas32 >= 2 * 152)
        launch_translate_tn<P, UP, 32, 8>(l, begin, end, ops, X, s);
    else
        launch_translate_tn<P, UP, 16, 2>(l, begin, end, ops, X, s);
}

void launch_m2m(int P, int l, const int32_t *begin, const int32_t *end, const float *ops, float *M, cudaStream_t s)
{
    switch (P) {
    case 4: launch_translate_t<4, true>(l, begin, end, ops, M, s); break;
    case 6: launch_translate_t<6, true>(l, begin, end, ops, M, s); break;
    case 8: launch_translate_t<8, true>(l, begin, end, ops, M, s); break;
    case 10: launch_translate_t<10, true>(l, begin, end, ops, M, s); break;
    }
}

void launch_l2l(int P, int l, const int32_t *begin, const int32_t *end, const float *ops, float *Lc, cudaStream_t s)
{
    switch (P) {
    case 4: launch_translate_t<4, false>(l, begin, end, ops, Lc, s); break;
    case 6: launch_translate_t<6, false>(l, begin, end, ops, Lc, s); break;
    case 8: launch_translate_t<8, false>(l, begin, end, ops, Lc, s); break;
    case 10: launch_translate_t<10, false>(l, begin, end, ops, Lc, s); break;
    }
}

// ------------------------------------------------------------------------------------------
// L2P: one thread per particle (sorted order).  phi = (1/h) sum L~ R(x^), grad = (1/h^2) x
// ladder sums, x^ = (x - c) / h:
//   dphi/dz            = sum_{n<P-1} sum_m sqrt((n+1-m)(n+1+m)) L_{n+1}^m R_n^m
//   dphi/dx + i dphi/dy = sum_{n<P-1} sum_m s(m) sqrt((n+2-m)(n+1-m)) L_{n+1}^{m-1} R_n^m,
//   s(m) = +1 for m >= 1, -1 for m <= 0.
// ------------------------------------------------------------------------------------------
// value and gradient of the scaled local expansion Lg at x^ (multiplied by 1/h and 1/h^2)
template <int P>
GB_DEV float4 l2p_eval(const float *__restrict__ Lg, float x, float y, float z, float ih)
{
    const float r2 = x * x + y * y + z * z;
    float phi = 0.f, gz = 0.f, gpr = 0.f, gpi = 0.f;
    float mre = 1.f, mim = 0.f;
#pragma unroll
    for (int m = 0; m < P; ++m) {
        if (m > 0) {
            const float f = -c_rmm[m];
            const float tr = f * (x * mre - y * mim), ti = f * (x * mim + y * mre);
            mre = tr;
            mim = ti;
        }
        float are = mre, aim = mim, bre = 0.f, bim = 0.f;
#pragma unroll
        for (int nn = m; nn < P; ++nn) {
            if (nn > m) {
                const float ca = c_ra[nn - 1][m] * z, cb = c_rb[nn - 1][m] * r2;
                const float nre = ca * are - cb * bre, nim = ca * aim - cb * bim;
                bre = are;
                bim = aim;
                are = nre;
                aim = nim;
            }
            // phi: L_nn^m R_nn^m
            {
                const float lre = __ldg(&Lg[re_idx(nn, m)]);
                const float lim = (m > 0) ? __ldg(&Lg[im_idx(nn, m)]) : 0.f;
                const float w = (m > 0) ? 2.f : 1.f;
                phi += w * (lre * are - lim * aim);
            }
            if (nn + 1 < P) {
                // d/dz: L_{nn+1}^m R_nn^m
                {
                    const float lre = __ldg(&Lg[re_idx(nn + 1, m)]);
                    const float lim = (m > 0) ? __ldg(&Lg[im_idx(nn + 1, m)]) : 0.f;
                    const float w = (m > 0) ? 2.f : 1.f;
                    gz += w * c_sq[nn + 1 - m][nn + 1 + m] * (lre * are - lim * aim);
                }
                // d/dx + i d/dy, term mu = m >= 1: + sqrt((nn+2-m)(nn+1-m)) L_{nn+1}^{m-1} R_nn^m
                if (m >= 1) {
                    const float lre = __ldg(&Lg[re_idx(nn + 1, m - 1)]);
                    const float lim = (m - 1 > 0) ? __ldg(&Lg[im_idx(nn + 1, m - 1)]) : 0.f;
                    const float c = c_sq[nn + 2 - m][nn + 1 - m];
                    gpr += c * (lre * are - lim * aim);
                    gpi += c * (lre * aim + lim * are);
                }
                // term mu = -m <= 0: - sqrt((nn+2+m)(nn+1+m)) conj(L_{nn+1}^{m+1} R_nn^m)
                {
                    const float lre = __ldg(&Lg[re_idx(nn + 1, m + 1)]);
                    const float lim = __ldg(&Lg[im_idx(nn + 1, m + 1)]);
                    const float c = c_sq[nn + 2 + m][nn + 1 + m];
                    gpr -= c * (lre * are - lim * aim);
                    gpi += c * (lre * aim + lim * are);
                }
            }
        }
    }
    const float ih2 = ih * ih;
    return make_float4(phi * ih, gpr * ih2, gpi * ih2, gz * ih2);
}

// the near-field compensated sums of particle i (sorted order: the sums, then their
// compensations) completed with the far field, in the order the P2P kernel adds it
GB_DEV float4 near_plus_far(const float4 *__restrict__ near, int64_t i, float4 f)
{
    const float4 s = near[2 * i], c = near[2 * i + 1];
    Kahan a{s.x, c.x}, bx{s.y, c.y}, by{s.z, c.z}, bz{s.w, c.w};
    a.add(f.x);
    bx.add(f.y);
    by.add(f.z);
    bz.add(f.w);
    return make_float4(a.s, bx.s, by.s, bz.s);
}

template <int P>
__global__ void __launch_bounds__(128) k_l2p(int L, const float *__restrict__ geo, int64_t n,
                                             const float4 *__restrict__ sx, const uint32_t *__restrict__ leafkey,
                                             const float *__restrict__ Lc, float4 *__restrict__ far,
                                             const float4 *__restrict__ near, const uint32_t *__restrict__ perm,
                                             float4 *__restrict__ out)
{
    constexpr int PP = P * P;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t key = leafkey[i];
    const int64_t g = level_offset(L) + key;
    const CellGeom cg = geo_level_cell(geo, L, key);
    float4 p = __ldg(&sx[i]);
    const float4 f = l2p_eval<P>(Lc + g * PP, (p.x - cg.cx) * cg.inv_h, (p.y - cg.cy) * cg.inv_h,
                                 (p.z - cg.cz) * cg.inv_h, cg.inv_h);
    if (near)
        out[perm[i]] = near_plus_far(near, i, f);
    else
        far[i] = f;
}

void launch_l2p(int P, int L, const float *geo, int64_t n, const float4 *sx, const uint32_t *leafkey, const float *Lc,
                float4 *far, cudaStream_t s, const float4 *near, const uint32_t *perm, float4 *out)
{
    if (n <= 0) return;
    unsigned grid = (unsigned)((n + 127) / 128);
    GBFMM_DISPATCH_P(P, (k_l2p<PQ><<<grid, 128, 0, s>>>(L, geo, n, sx, leafkey, Lc, far, near, perm, out)));
    note_launches(1);
}

// ------------------------------------------------------------------------------------------
// M2P (treecode far field; the adaptive FMM's W lists): the multipole of a source cell evaluated
// at a target particle.  With x^ = (x - c)/h:
//   phi = (1/h) sum M~_n^m I_n^m(x^)
//   dphi/dz             = -(1/h^2) sum sqrt((n+1-m)(n+1+m)) M~_n^m I_{n+1}^m
//   dphi/dx + i dphi/dy =  (1/h^2) sum s(m) sqrt((n+m+2)(n+m+1)) M~_n^m I_{n+1}^{m+1},
//   s(m) = +1 for m >= 0, -1 for m < 0.
// ------------------------------------------------------------------------------------------
// The constants of these sums are folded into the source cell's coefficients once per cell
// (staged in shared memory), so that each (particle, cell) evaluation spends two FMAs per real
// term: per (N, m), 0 <= m <= N <= P, two float4 (in two halves of the fold, F[q] and F[NM + q])
//   {w M_N^m (re, im), -w sqrt((N-m)(N+m)) M_{N-1}^m (re, im)},
//   {A - B (re, im), A + B (re, im)},  A = sqrt((N+m)(N+m-1)) M_{N-1}^{m-1},
//                                      B = sqrt((N-m)(N-m-1)) M_{N-1}^{m+1},
// w = 2 for m > 0; dphi/dx + i dphi/dy = sum A I - conj(B I), so its real part takes A - B
// against (Re I, -Im I) and its imaginary part A + B against (Im I, Re I).
template <int P>
struct M2PFold {
    static constexpr int NM = (P + 1) * (P + 2) / 2;
};

GB_HD constexpr int nm_idx(int N, int m) { return N * (N + 1) / 2 + m; }

// per (N, m) of the folded coefficients: where its four source coefficients sit in M (re and im
// index each, -1 for none) and their factors; built once per CTA by m2p_fold_table
template <int P>
struct M2PFoldTab {
    int4 re, im;   // source coefficient of {phi, dz, A, B}: real / imaginary part index, -1: zero
    float4 c;      // factors of {phi, dz, A, B}
};

template <int P>
GB_DEV void m2p_fold_table(M2PFoldTab<P> *__restrict__ T, int t, int nt)
{
    auto root = [](int a, int b) { return sqrtf((float)(a * b)); };
    for (int q = t; q < M2PFold<P>::NM; q += nt) {
        int N = 0;
        while ((N + 1) * (N + 2) / 2 <= q) ++N;
        const int m = q - N * (N + 1) / 2;
        const float w = m > 0 ? 2.f : 1.f;
        M2PFoldTab<P> e;
        e.re = make_int4(-1, -1, -1, -1);
        e.im = make_int4(-1, -1, -1, -1);
        e.c = make_float4(0.f, 0.f, 0.f, 0.f);
        if (N <= P - 1) {
            e.re.x = re_idx(N, m);
            e.im.x = m > 0 ? im_idx(N, m) : -1;
            e.c.x = w;
        }
        if (N >= 1 && m <= N - 1) {
            e.re.y = re_idx(N - 1, m);
            e.im.y = m > 0 ? im_idx(N - 1, m) : -1;
            e.c.y = -w * root(N - m, N + m);
        }
        if (N >= 1 && m >= 1) {
            e.re.z = re_idx(N - 1, m - 1);
            e.im.z = m - 1 > 0 ? im_idx(N - 1, m - 1) : -1;
            e.c.z = root(N + m, N + m - 1);
        }
        if (N >= 1 && m + 1 <= N - 1) {
            e.re.w = re_idx(N - 1, m + 1);
            e.im.w = im_idx(N - 1, m + 1);
            e.c.w = root(N - m, N - m - 1);
        }
        T[q] = e;
    }
}

// the block stages the cell's coefficients M[P^2] (coalesced) in sM, then threads t, t + nt,
// ... fill F[2 NM] through the table
template <int P>
GB_DEV void m2p_fold(const float *__restrict__ M, float *__restrict__ sM, const M2PFoldTab<P> *__restrict__ T,
                     float4 *__restrict__ F, int t, int nt)
{
    for (int k = t; k < P * P; k += nt) sM[k] = M[k];
    __syncthreads();
    auto at = [&](int k) { return k >= 0 ? sM[k] : 0.f; };
    for (int q = t; q < M2PFold<P>::NM; q += nt) {
        const M2PFoldTab<P> e = T[q];
        const float pr = e.c.x * at(e.re.x), pi = e.c.x * at(e.im.x);
        const float zr = e.c.y * at(e.re.y), zi = e.c.y * at(e.im.y);
        const float ar = e.c.z * at(e.re.z), ai = e.c.z * at(e.im.z);
        const float br = e.c.w * at(e.re.w), bi = e.c.w * at(e.im.w);
        F[q] = make_float4(pr, pi, zr, zi);
        F[M2PFold<P>::NM + q] = make_float4(ar - br, ai - bi, ar + br, ai + bi);
    }
}

// The M2P sums for NT targets at once against one source cell's folded
// coefficients (Fa[q] = {phi, dz} pair, Fb[q] = {A - B, A + B} pair of (N, m) = q), so that every
// coefficient load serves NT targets.  x, y, z: target minus cell centre over h; ih = 1/h.  The
// degree recurrence takes z/r^2 and the constants' products with it once per term:
// I_N = (a z/r^2) I_{N-1} - (b / r^2) I_{N-2}.
template <int P, int NT>
GB_DEV void m2p_acc_n(const float4 *__restrict__ Fa, const float4 *__restrict__ Fb, const float (&x)[NT],
                      const float (&y)[NT], const float (&z)[NT], float ih, float (&o)[NT][4])
{
    float ir2[NT], zi[NT], mre[NT], mim[NT], phi[NT], gz[NT], gpr[NT], gpi[NT];
#pragma unroll
    for (int k = 0; k < NT; ++k) {
        const float r2 = x[k] * x[k] + y[k] * y[k] + z[k] * z[k];
        const float ir = rsqrt_ftz(r2);
        ir2[k] = ir * ir;
        zi[k] = z[k] * ir2[k];
        mre[k] = ir;  // I_0^0 = 1/r
        mim[k] = 0.f;
        phi[k] = gz[k] = gpr[k] = gpi[k] = 0.f;
    }
#pragma unroll
    for (int m = 0; m <= P; ++m) {
        if (m > 0) {
#pragma unroll
            for (int k = 0; k < NT; ++k) {
                const float f = -c_rmm[m] * ir2[k];
                const float tr = f * (x[k] * mre[k] - y[k] * mim[k]), ti = f * (x[k] * mim[k] + y[k] * mre[k]);
                mre[k] = tr;
                mim[k] = ti;
            }
        }
        float are[NT], aim[NT], bre[NT], bim[NT];
#pragma unroll
        for (int k = 0; k < NT; ++k) {
            are[k] = mre[k];
            aim[k] = mim[k];
            bre[k] = bim[k] = 0.f;
        }
#pragma unroll
        for (int N = m; N <= P; ++N) {
            if (N > m) {
#pragma unroll
                for (int k = 0; k < NT; ++k) {
                    const float A = c_ra[N - 1][m] * zi[k], B = c_rb[N - 1][m] * ir2[k];
                    const float nre = fmaf(A, are[k], -B * bre[k]), nim = fmaf(A, aim[k], -B * bim[k]);
                    bre[k] = are[k];
                    bim[k] = aim[k];
                    are[k] = nre;
                    aim[k] = nim;
                }
            }
            const int q = nm_idx(N, m);
            if (N <= P - 1 || (N >= 1 && m <= N - 1)) {
                const float4 a = Fa[q];
#pragma unroll
                for (int k = 0; k < NT; ++k) {
                    if (N <= P - 1) phi[k] = fmaf(a.x, are[k], fmaf(-a.y, aim[k], phi[k]));
                    if (N >= 1 && m <= N - 1) gz[k] = fmaf(a.z, are[k], fmaf(-a.w, aim[k], gz[k]));
                }
            }
            if (N >= 1 && (m >= 1 || m + 1 <= N - 1)) {
                const float4 bb = Fb[q];
#pragma unroll
                for (int k = 0; k < NT; ++k) {
                    gpr[k] = fmaf(bb.x, are[k], fmaf(-bb.y, aim[k], gpr[k]));
                    gpi[k] = fmaf(bb.z, aim[k], fmaf(bb.w, are[k], gpi[k]));
                }
            }
        }
    }
    const float ih2 = ih * ih;
#pragma unroll
    for (int k = 0; k < NT; ++k) {
        o[k][0] += phi[k] * ih;
        o[k][1] += gpr[k] * ih2;
        o[k][2] += gpi[k] * ih2;
        o[k][3] += gz[k] * ih2;
    }
}

// M2P by warps (the treecode on both trees): two warps per target leaf and no block barrier.
// The leaf's targets go in chunks of up to 32, warp h of the leaf taking chunks h, h + 2, ...;
// a chunk of T targets takes G = min(4, 32 / T) source cells per step (lane l: target l % T,
// source group l / T), so small leaves and the remainder chunk still fill the warp.  Per step the warp stages the cells' coefficients and folds them into its own
// shared memory (the M2P constants of m2p_fold), then every active lane evaluates its target
// against its group's cell (m2p_acc_n).  At the end of a chunk the groups' partial sums are
// added in group order (deterministic).  Sources: the M2L rows of the leaf's ancestors at levels
// 2..L (uniform tree, UNI) or one cell-list row (adaptive tree).  ADD: add into far (else write).
template <int P>
struct M2PW {
    static constexpr int NM = M2PFold<P>::NM;
    static constexpr int GMAX = 4;
    static constexpr int NMP = NM % 8 == 0 ? NM + 1 : NM;  // float4 stride of the two halves (bank spread)
    static constexpr int WARPS = 4;                         // per CTA; two per leaf
};

template <int P, bool UNI, bool ADD>
__global__ void __launch_bounds__(128) k_m2p_warp(int L, const float *__restrict__ geo,
                                                  const int32_t *__restrict__ leaves, Span lv,
                                                  const float4 *__restrict__ geom, const int32_t *__restrict__ begin,
                                                  const int32_t *__restrict__ end, const uint32_t *__restrict__ offs,
                                                  const int32_t *__restrict__ ids, const float4 *__restrict__ sx,
                                                  const float *__restrict__ M, float4 *__restrict__ far)
{
    using W = M2PW<P>;
    constexpr int PP = P * P, NM = W::NM, G4 = W::GMAX, NMP = W::NMP;
    __shared__ M2PFoldTab<P> sT[NM];
    __shared__ float4 sF[W::WARPS][G4 * 2 * NMP];
    __shared__ float sM[W::WARPS][G4 * PP];
    __shared__ float4 sR[W::WARPS][32];
    m2p_fold_table<P>(sT, threadIdx.x, blockDim.x);
    __syncthreads();  // the only block barrier: the table
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t w = (blockIdx.x * (int64_t)W::WARPS + warp) >> 1;
    const int half = warp & 1;
    if (w >= span_count(lv)) return;
    const int64_t b = UNI ? level_offset(L) + w : (int64_t)leaves[w];
    const int b0 = begin[b], nt = end[b] - b0;
    if (nt <= 32 * half || (!UNI && offs[b] == offs[b + 1])) return;  // no chunk, or no sources (far untouched)
    float4 *F = sF[warp];
    float *Ms = sM[warp];
    for (int c0 = 32 * half; c0 < nt; c0 += 64) {
        const int T = min(32, nt - c0);
        const int G = min(G4, 32 / T);
        const int t = lane % T, g = lane / T;
        const bool act = g < G;
        const float4 p = __ldg(&sx[b0 + c0 + (act ? t : 0)]);
        float o[1][4] = {{0.f, 0.f, 0.f, 0.f}};
        auto row = [&](uint32_t e0, uint32_t e1, int l) {
            for (uint32_t e = e0; e < e1; e += G) {
                const int ng = (int)(e1 - e < (uint32_t)G ? e1 - e : (uint32_t)G);
                __syncwarp();
                for (int k = lane; k < ng * PP; k += 32) {
                    const int gg = k / PP, kk = k - gg * PP;
                    Ms[k] = M[(int64_t)ids[e + gg] * PP + kk];
                }
                __syncwarp();
                for (int q = lane; q < ng * NM; q += 32) {
                    const int gg = q / NM, qq = q - gg * NM;
                    const M2PFoldTab<P> en = sT[qq];
                    const float *m = Ms + gg * PP;
                    auto at = [&](int k) { return k >= 0 ? m[k] : 0.f; };
                    const float pr = en.c.x * at(en.re.x), pi = en.c.x * at(en.im.x);
                    const float zr = en.c.y * at(en.re.y), zi = en.c.y * at(en.im.y);
                    const float ar = en.c.z * at(en.re.z), ai = en.c.z * at(en.im.z);
                    const float br = en.c.w * at(en.re.w), bi = en.c.w * at(en.im.w);
                    F[gg * 2 * NMP + qq] = make_float4(pr, pi, zr, zi);
                    F[gg * 2 * NMP + NMP + qq] = make_float4(ar - br, ai - bi, ar + br, ai + bi);
                }
                __syncwarp();
                if (act && g < ng) {
                    const int64_t sc = ids[e + g];
                    const CellGeom cg = UNI ? geo_level_cell(geo, l, (uint32_t)(sc - level_offset(l))) : geo_cell(geom, sc);
                    const float4 *Fa = F + g * 2 * NMP;
                    float xs[1] = {(p.x - cg.cx) * cg.inv_h}, ys[1] = {(p.y - cg.cy) * cg.inv_h};
                    float zs[1] = {(p.z - cg.cz) * cg.inv_h};
                    m2p_acc_n<P, 1>(Fa, Fa + NMP, xs, ys, zs, cg.inv_h, o);
                }
            }
        };
        if (UNI) {
            for (int l = 2; l <= L; ++l) {
                const int64_t a = level_offset(l) + (w >> (3 * (L - l)));
                row(offs[a], offs[a + 1], l);
            }
        } else {
            row(offs[b], offs[b + 1], 0);
        }
        // the groups' partial sums, added in group order
        __syncwarp();
        sR[warp][lane] = make_float4(o[0][0], o[0][1], o[0][2], o[0][3]);
        __syncwarp();
        if (act && g == 0) {
            float4 r = sR[warp][t];
            for (int gg = 1; gg < G; ++gg) {
                const float4 v = sR[warp][t + gg * T];
                r.x += v.x;
                r.y += v.y;
                r.z += v.z;
                r.w += v.w;
            }
            const int64_t i = b0 + c0 + t;
            if (ADD) {
                float4 f = far[i];
                f.x += r.x;
                f.y += r.y;
                f.z += r.z;
                f.w += r.w;
                far[i] = f;
            } else {
                far[i] = r;
            }
        }
    }
}

void launch_m2p(int P, int L, const float *geo, const float4 *sx, const int32_t *begin, const int32_t *end,
                const uint32_t *m2l_offs, const int32_t *m2l_ids, const float *M, float4 *far, cudaStream_t s)
{
    const int64_t nl = int64_t(1) << (3 * L);
    const unsigned grid = (unsigned)((nl + 1) / 2);  // two warps per leaf, four per CTA
    const Span lv = host_span(0, nl);
    GBFMM_DISPATCH_P(P, (k_m2p_warp<PQ, true, false><<<grid, 128, 0, s>>>(L, geo, nullptr, lv, nullptr, begin, end,
                                                                          m2l_offs, m2l_ids, sx, M, far)));
    note_launches(1);
}

// ==========================================================================================
// Adaptive tree: cells are given by index; each carries its level and 63-bit key prefix.
// ==========================================================================================
GB_DEV CellGeom cell_geom63(const Box &b, int l, uint64_t key)
{
    int ix, iy, iz;
    demorton63(key, ix, iy, iz);
    double h = b.side / (double)(int64_t(1) << l);
    CellGeom g;
    g.cx = (float)(b.origin[0] + (ix + 0.5) * h);
    g.cy = (float)(b.origin[1] + (iy + 0.5) * h);
    g.cz = (float)(b.origin[2] + (iz + 0.5) * h);
    g.inv_h = (float)(1.0 / h);
    return g;
}

__global__ void k_cell_geom(Span cells, const int32_t *__restrict__ level, const uint64_t *__restrict__ key,
                            const Box *__restrict__ box, float4 *__restrict__ geom)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= span_count(cells)) return;
    const int64_t c = span_first(cells) + i;
    const CellGeom g = cell_geom63(*box, level[c], key[c]);
    geom[c] = make_float4(g.cx, g.cy, g.cz, g.inv_h);
}

void launch_cell_geom(Span cells, const int32_t *level, const uint64_t *key, const Box *box, float4 *geom,
                      cudaStream_t s)
{
    if (cells.cap <= 0) return;
    k_cell_geom<<<(unsigned)((cells.cap + 255) / 256), 256, 0, s>>>(cells, level, key, box, geom);
    note_launches(1);
}

// P2M at the listed leaves (levels >= 2), one warp per leaf
template <int P>
__global__ void __launch_bounds__(128) k_p2m_cells(const int32_t *__restrict__ leaves, Span lv,
                                                   const int32_t *__restrict__ level, const float4 *__restrict__ geom,
                                                   const int32_t *__restrict__ begin, const int32_t *__restrict__ count,
                                                   const float4 *__restrict__ sx, float *__restrict__ M)
{
    __shared__ float scr[4][32 * WarpSum<P>::LD];
    const int lane = threadIdx.x & 31;
    const int64_t w = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
    if (w >= span_count(lv)) return;
    const int32_t c = leaves[w];
    if (level[c] < 2) return;
    const CellGeom cg = geo_cell(geom, c);
    float acc[P * P];
#pragma unroll
    for (int i = 0; i < P * P; ++i) acc[i] = 0.f;
    p2x_particles<P, false>(acc, sx, begin[c], begin[c] + count[c], lane, cg);
    warp_store<P>(acc, M + (int64_t)c * (P * P), lane, false, scr[threadIdx.x >> 5]);
}

// P2L over the X list (Eq. 3's L from the particles of each X leaf), one warp per cell; adds
// into the cell's local expansion
template <int P>
__global__ void __launch_bounds__(128) k_p2l_cells(Span cells, const int32_t *__restrict__ level,
                                                   const float4 *__restrict__ geom, const int32_t *__restrict__ begin,
                                                   const int32_t *__restrict__ count,
                                                   const uint32_t *__restrict__ x_offs,
                                                   const int32_t *__restrict__ x_ids, const float4 *__restrict__ sx,
                                                   float *__restrict__ Lc)
{
    __shared__ float scr[4][32 * WarpSum<P>::LD];
    const int lane = threadIdx.x & 31;
    const int64_t w = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
    if (w >= span_count(cells)) return;
    const int64_t b = span_first(cells) + w;
    const uint32_t e0 = x_offs[b], e1 = x_offs[b + 1];
    if (e0 == e1 || level[b] < 2) return;
    const CellGeom cg = geo_cell(geom, b);
    float acc[P * P];
#pragma unroll
    for (int i = 0; i < P * P; ++i) acc[i] = 0.f;
    for (uint32_t e = e0; e < e1; ++e) {
        const int32_t c = x_ids[e];
        p2x_particles<P, true>(acc, sx, begin[c], begin[c] + count[c], lane, cg);
    }
    warp_store<P>(acc, Lc + b * (P * P), lane, true, scr[threadIdx.x >> 5]);
}

// L2P at every particle's leaf (leaves above level 2 carry no local expansion)
template <int P>
__global__ void __launch_bounds__(128) k_l2p_cells(int64_t n, const int32_t *__restrict__ leaf_of,
                                                   const int32_t *__restrict__ level, const float4 *__restrict__ geom,
                                                   const float4 *__restrict__ sx, const float *__restrict__ Lc,
                                                   float4 *__restrict__ far, const float4 *__restrict__ near,
                                                   const uint32_t *__restrict__ perm, float4 *__restrict__ out,
                                                   const int32_t *__restrict__ abort)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n || (abort && *abort)) return;
    const int32_t c = leaf_of[i];
    float4 f = make_float4(0.f, 0.f, 0.f, 0.f);
    if (level[c] >= 2) {
        const CellGeom cg = geo_cell(geom, c);
        float4 p = __ldg(&sx[i]);
        f = l2p_eval<P>(Lc + (int64_t)c * (P * P), (p.x - cg.cx) * cg.inv_h, (p.y - cg.cy) * cg.inv_h,
                        (p.z - cg.cz) * cg.inv_h, cg.inv_h);
    }
    if (near) {  // far holds the M2P (W list) sums
        const float4 w = far[i];
        f.x += w.x;
        f.y += w.y;
        f.z += w.z;
        f.w += w.w;
        out[perm[i]] = near_plus_far(near, i, f);
    } else {
        far[i] = f;
    }
}

// M2P over the W list, one CTA per listed leaf; adds into the far-field accumulator
template <int P>
__global__ void __launch_bounds__(64) k_m2p_cells(const int32_t *__restrict__ leaves, Span lv,
                                                  const float4 *__restrict__ geom, const int32_t *__restrict__ begin,
                                                  const int32_t *__restrict__ end,
                                                  const uint32_t *__restrict__ w_offs,
                                                  const int32_t *__restrict__ w_ids, const float4 *__restrict__ sx,
                                                  const float *__restrict__ M, float4 *__restrict__ far)
{
    __shared__ float4 sF[2 * M2PFold<P>::NM];
    __shared__ float sM[P * P];
    __shared__ M2PFoldTab<P> sT[M2PFold<P>::NM];
    if (blockIdx.x >= span_count(lv)) return;
    const int32_t b = leaves[blockIdx.x];
    const uint32_t e0 = w_offs[b], e1 = w_offs[b + 1];
    if (e0 == e1) return;
    m2p_fold_table<P>(sT, threadIdx.x, blockDim.x);  // read after the first fold's barrier
    const int b0 = begin[b], bend = end[b];
    for (int t0 = b0; t0 < bend; t0 += blockDim.x) {
        const int t = t0 + threadIdx.x;
        const bool act = t < bend;
        float4 p = act ? __ldg(&sx[t]) : make_float4(0.f, 0.f, 0.f, 0.f);
        float o[4] = {0.f, 0.f, 0.f, 0.f};
        for (uint32_t e = e0; e < e1; ++e) {
            const int32_t sc = w_ids[e];
            __syncthreads();
            m2p_fold<P>(M + (int64_t)sc * (P * P), sM, sT, sF, threadIdx.x, blockDim.x);
            __syncthreads();
            const CellGeom cg = geo_cell(geom, sc);
            if (act) {
                float xs[1] = {(p.x - cg.cx) * cg.inv_h}, ys[1] = {(p.y - cg.cy) * cg.inv_h};
                float zs[1] = {(p.z - cg.cz) * cg.inv_h};
                float o1[1][4] = {{o[0], o[1], o[2], o[3]}};
                m2p_acc_n<P, 1>(sF, sF + M2PFold<P>::NM, xs, ys, zs, cg.inv_h, o1);
#pragma unroll
                for (int k = 0; k < 4; ++k) o[k] = o1[0][k];
            }
        }
        if (act) {
            float4 f = far[t];
            f.x += o[0];
            f.y += o[1];
            f.z += o[2];
            f.w += o[3];
            far[t] = f;
        }
    }
}

// M2M (up) / L2L (down) over cells given by their parents' index range; children by position.
// As k_translate: the operator of each child position and the TN source columns are copied into
// shared memory with cp.async (zero-filled for missing children), the next child position's
// copies in flight while the current one is applied.
template <int P, bool UP, int TN, int CN>
__global__ void __launch_bounds__(TransCfg<P, UP, TN, CN>::NT) k_translate_cells(Span par,
                                                                         const int32_t *__restrict__ child_of,
                                                                         const int32_t *__restrict__ nchild,
                                                                         const float *__restrict__ ops,
                                                                         float *__restrict__ X)
{
    using Cfg = TransCfg<P, UP, TN, CN>;
    constexpr int PP = Cfg::PP, PR = Cfg::PR, SB = Cfg::SB, NCG = Cfg::NCG, NRG = Cfg::NRG;
    extern __shared__ __align__(16) float tsm[];
    const int64_t q0 = blockIdx.x * (int64_t)TN;
    const int64_t lo = span_first(par), np = span_count(par);
    if (q0 >= np) return;  // the whole CTA: beyond the parents
    const int tid = threadIdx.x;
    const bool work = tid < NRG * NCG;
    const int cg = tid % NCG, rg = tid / NCG;
    int kbeg = 0, kend = PP;
    if (work) {
        const int r0 = min(rg * 4, PP - 1), r1 = min(rg * 4 + 3, PP - 1);
        if (UP) {
            const int d = degree_of(r1);
            kend = min(PP, ((d + 1) * (d + 1) + 3) / 4 * 4);
        } else {
            const int d = degree_of(r0);
            kbeg = (d * d) / 4 * 4;
        }
    }
    auto stage = [&](int c, int buf) {
        float *A = tsm + buf * (Cfg::AF + Cfg::BF);
        float *B = A + Cfg::AF;
        const float *src = ops + (size_t)c * PP * PR;
        for (int e = tid; e < PP * PR / 4; e += blockDim.x) cp_async16_t(A + 4 * e, src + 4 * e, 16u);
        for (int e = tid; e < TN * (PP / 4); e += blockDim.x) {
            const int i = e / (PP / 4), k4 = e % (PP / 4);
            const int64_t q = q0 + i;
            const float *gsrc = X;
            uint32_t bytes = 0;
            if (q < np) {
                const int64_t pcell = lo + q;
                const int64_t g = UP ? child_of[pcell * 8 + c] : (child_of[pcell * 8 + c] >= 0 ? pcell : -1);
                if (g >= 0) {
                    gsrc = X + g * PP + 4 * k4;
                    bytes = 16u;
                }
            }
            cp_async16_t(B + i * SB + 4 * k4, gsrc, bytes);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    float acc[4][CN];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < CN; ++j) acc[i][j] = 0.f;
    const int c_first = UP ? 0 : blockIdx.y, c_last = UP ? 7 : blockIdx.y;
    stage(c_first, 0);
    for (int c = c_first; c <= c_last; ++c) {
        const int buf = UP ? (c - c_first) & 1 : 0;
        if (c < c_last) {
            stage(c + 1, buf ^ 1);
            asm volatile("cp.async.wait_group 1;" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        __syncthreads();
        if (work) {
            const float *Ar = tsm + buf * (Cfg::AF + Cfg::BF) + rg * 4;
            const float *Bc = tsm + buf * (Cfg::AF + Cfg::BF) + Cfg::AF + cg * SB;
#pragma unroll 2
            for (int k = kbeg; k < kend; k += 4) {
                Frag<CN, 4> f;
                f.load(Ar, Bc, k, PR, NCG * SB);
                f.fma(acc);
            }
        }
        __syncthreads();  // the buffer is refilled two positions later
    }
    if (!work) return;
#pragma unroll
    for (int j = 0; j < CN; ++j) {
        const int64_t q = q0 + cg + j * NCG;
        if (q >= np) continue;
        const int r = rg * 4;
        if (r >= PP) continue;
        const int64_t pcell = lo + q;
        int64_t g;
        if (UP) {
            if (nchild[pcell] == 0) continue;  // a leaf keeps its P2M expansion
            g = pcell;
        } else {
            g = child_of[pcell * 8 + blockIdx.y];
            if (g < 0) continue;
        }
        float4 *dst = reinterpret_cast<float4 *>(X + g * PP + r);
        if (UP) {
            *dst = make_float4(acc[0][j], acc[1][j], acc[2][j], acc[3][j]);
        } else {
            float4 v = *dst;
            v.x += acc[0][j];
            v.y += acc[1][j];
            v.z += acc[2][j];
            v.w += acc[3][j];
            *dst = v;
        }
    }
}

void launch_p2m_cells(int P, const int32_t *leaves, Span lv, const int32_t *level, const float4 *geom,
                      const int32_t *begin, const int32_t *count, const float4 *sx, float *M, cudaStream_t s)
{
    if (lv.cap <= 0) return;
    const unsigned grid = (unsigned)((lv.cap + 3) / 4);
    GBFMM_DISPATCH_P(P, (k_p2m_cells<PQ><<<grid, 128, 0, s>>>(leaves, lv, level, geom, begin, count, sx, M)));
    note_launches(1);
}

void launch_p2l_cells(int P, Span cells, const int32_t *level, const float4 *geom, const int32_t *begin,
                      const int32_t *count, const uint32_t *x_offs, const int32_t *x_ids, const float4 *sx, float *Lc,
                      cudaStream_t s)
{
    if (cells.cap <= 0) return;
    const unsigned grid = (unsigned)((cells.cap + 3) / 4);
    GBFMM_DISPATCH_P(P, (k_p2l_cells<PQ><<<grid, 128, 0, s>>>(cells, level, geom, begin, count, x_offs, x_ids, sx,
                                                              Lc)));
    note_launches(1);
}

void launch_l2p_cells(int P, int64_t n, const int32_t *leaf_of, const int32_t *level, const float4 *geom,
                      const float4 *sx, const float *Lc, float4 *far, cudaStream_t s, const float4 *near,
                      const uint32_t *perm, float4 *out, const int32_t *abort)
{
    if (n <= 0) return;
    const unsigned grid = (unsigned)((n + 127) / 128);
    GBFMM_DISPATCH_P(P, (k_l2p_cells<PQ><<<grid, 128, 0, s>>>(n, leaf_of, level, geom, sx, Lc, far, near, perm, out,
                                                              abort)));
    note_launches(1);
}

void launch_m2p_cells(int P, const int32_t *leaves, Span lv, const float4 *geom, const int32_t *begin,
                      const int32_t *end, const uint32_t *w_offs, const int32_t *w_ids, const float4 *sx,
                      const float *M, float4 *far, cudaStream_t s, bool long_rows)
{
    if (lv.cap <= 0) return;
    if (long_rows) {
        const unsigned grid = (unsigned)((lv.cap + 1) / 2);  // two warps per leaf, four per CTA
        GBFMM_DISPATCH_P(P, (k_m2p_warp<PQ, false, true><<<grid, 128, 0, s>>>(0, nullptr, leaves, lv, geom, begin,
                                                                              end, w_offs, w_ids, sx, M, far)));
    } else {
        GBFMM_DISPATCH_P(P, (k_m2p_cells<PQ><<<(unsigned)lv.cap, 64, 0, s>>>(leaves, lv, geom, begin, end, w_offs,
                                                                             w_ids, sx, M, far)));
    }
    note_launches(1);
}

template <int P, bool UP, int TN, int CN>
static void translate_cells_tn(Span par, const int32_t *child_of, const int32_t *nchild, const float *ops, float *X,
                               cudaStream_t s)
{
    using Cfg = TransCfg<P, UP, TN, CN>;
    const int smem = (int)Cfg::kSmem;  // operator + column block, double-buffered for M2M
    cudaFuncSetAttribute(k_translate_cells<P, UP, TN, CN>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    dim3 grid((unsigned)((par.cap + TN - 1) / TN), UP ? 1 : 8);
    k_translate_cells<P, UP, TN, CN><<<grid, Cfg::NT, smem, s>>>(par, child_of, nchild, ops, X);
    note_launches(1);
}

// the cells-per-CTA choice of the uniform tree's translations (launch_translate_t), on the
// launch's capacity
template <int P, bool UP>
static void translate_cells_t(Span par, const int32_t *child_of, const int32_t *nchild, const float *ops, float *X,
                              cudaStream_t s)
{
    const int64_t ctas32 = (par.cap + 31) / 32 * (UP ? 1 : 8), ctas64 = (par.cap + 63) / 64 * (UP ? 1 : 8);
    if constexpr (UP) {  // large levels: 128 (upward) or 64 cells per CTA share each staged operator
        if ((par.cap + 127) / 128 >= 4 * 152) return translate_cells_tn<P, UP, 128, 8>(par, child_of, nchild, ops, X, s);
    }
    if (ctas64 >= 4 * 152)
        translate_cells_tn<P, UP, 64, 8>(par, child_of, nchild, ops, X, s);
    else if (ctas32 >= 2 * 152)
        translate_cells_tn<P, UP, 32, 8>(par, child_of, nchild, ops, X, s);
    else
        translate_cells_tn<P, UP, 16, 2>(par, child_of, nchild, ops, X, s);
}

void launch_translate_cells(int P, bool up, Span parents, const int32_t *child_of, const int32_t *nchild,
                            const float *ops, float *X, cudaStream_t s)
{
    if (parents.cap <= 0) return;
    if (up) {
        GBFMM_DISPATCH_P(P, (translate_cells_t<PQ, true>(parents, child_of, nchild, ops, X, s)));
    } else {
        GBFMM_DISPATCH_P(P, (translate_cells_t<PQ, false>(parents, child_of, nchild, ops, X, s)));
    }
}
#undef GBFMM_DISPATCH_P

}  // namespace gbfmm
