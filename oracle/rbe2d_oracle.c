/*
 * RBE2D CPU oracle — plain, slow, FP64, written from the paper
 * (Gan, Gao, Liang, Xu, "Random Batch Ewald Method for Dielectrically Confined
 * Coulomb Systems", arXiv 2405.06333).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is compiled into liborc_rbe2d.so and may be
 * loaded only by tests/, __graft_entry__.smoke() and the cpu_baseline / reference
 * leg of bench.py.  It shares no code, header, table or constant generator with the
 * CUDA path, and the CUDA path never calls it.
 *
 * What it computes, by definition and in the paper's notation:
 *   - Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11), the counter-based generator
 *     both sides use to draw the k-batch.
 *   - The separable Gaussian weight w(k) = exp(-k^2/(4 alpha^2)) on the lattice
 *     k = 2 pi (nx/Lx, ny/Ly, nz/Lz), its normaliser S (Eq. 2.21) and i.i.d. draws from P(k) = w(k)/S (Sec. 2.3).
 *   - The image charges of the three-layer sandwich model (Eq. 3.2, positions
 *     Eq. 3.3).
 *   - The structure factors rho_k and rhobar^M_k of Theorem 3.3 (Eqs. 3.16-3.17),
 *     by explicit summation over all 2MN image charges, and alternatively by the
 *     structure-factor re-calibration of Sec. 3.4 (coefficients Y_odd, Y_even).
 *   - The random-batch k-space energy (2pi/V)(S/P) sum_l Re(rho rhobar^M)/k^2, the
 *     self term, U_IBC^M (Eq. 3.18), the RBE force (Eq. 3.26,
 *     gradient by the chain rule on the explicit image sum, or by Eq. 3.25), dU/dq and dU/dgamma.
 *   - The same with the full k-sum (weights w(k) instead of S/P).
 *   - The erfc real-space sum with images (Eq. 3.12) by brute force.
 *   - The parameter rules: L_z (Eq. 3.23), M (Eq. 3.10),
 *     alpha ~ (N/(Lx Ly H))^(1/3) (Sec. 2.3).
 *
 * Readings of the paper taken here:
 *   A1  the extra exp(-k^2/4alpha^2) in Eq. 2.20 is dropped: with
 *       importance sampling it would double-count the weight; Eq. 3.26 has none.
 *   A4  gamma_+^(l) = gt^ceil(l/2) gb^floor(l/2), gamma_-^(l) = gb^ceil(l/2) gt^floor(l/2):
 *       the first image above the slab (at 2H - z) is the reflection in the top
 *       interface, as beta_ij (Eq. 3.7) requires.
 *   A5  odd (mirrored) images carry k-hat = (kx, ky, -kz), as in Eq. 3.25; the
 *       swapped pairing printed in Eq. 3.27 is not used.
 *   A6  inside rhobar^M the exponent is -i k.r_j (the paper prints r_i).
 *   A13 per sampled k the product rho rhobar^M is complex; its real part is used.
 *   A14 U_IBC^M and its q-gradient use the written non-symmetric general form.
 *
 * Units are Gaussian (no 1/(4 pi eps0)); F = -grad U.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

typedef struct {
    double Lx, Ly, H, Lz;   /* cell Lx x Ly, slab z in [0,H], extended period Lz */
    double gamma_top;       /* dielectric contrast at z = H */
    double gamma_bot;       /* dielectric contrast at z = 0 */
    double alpha;           /* Ewald splitting parameter */
    int M;                  /* image reflection levels (0 = homogeneous) */
} orc_system;

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the following parallel regions (timing only: the per-k and per-particle sums do
 * not depend on it; the real-space energy total may differ in its last bits). */
void orc_set_num_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------------- */
/* Philox4x64-10, from its published definition (Salmon et al., SC'11).       */
/* ------------------------------------------------------------------------- */
static void orc_mulhilo64(uint64_t a, uint64_t b, uint64_t* hi, uint64_t* lo) {
    unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
    *hi = (uint64_t)(p >> 64);
    *lo = (uint64_t)p;
}

void orc_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
    uint64_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; r++) {
        if (r > 0) { k0 += W0; k1 += W1; }
        uint64_t hi0, lo0, hi1, lo1;
        orc_mulhilo64(M0, c0, &hi0, &lo0);
        orc_mulhilo64(M1, c2, &hi1, &lo1);
        uint64_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* ------------------------------------------------------------------------- */
/* Gaussian weight, normaliser S, CDF tables, sampling  (Sec. 2.3)            */
/* ------------------------------------------------------------------------- */

/* Per-dimension truncation: beyond n_d the 1-D factor exp(-(pi n/(alpha L))^2) is
 * below exp(-46), i.e. n_d = ceil(alpha L sqrt(46) / pi). */
int orc_nmax(double alpha, double L) {
    return (int)ceil(alpha * L * sqrt(46.0) / ORC_PI);
}

/* One-dimensional factor of w(k) = exp(-k^2/(4 alpha^2)) for k_d = 2 pi n / L:
 * (2 pi n / L)^2 / (4 alpha^2) = (pi n / (alpha L))^2. */
double orc_w1d(int n, double alpha, double L) {
    double a = ORC_PI * (double)n / (alpha * L);
    return exp(-(a * a));
}

/* S = sum_{k != 0} w(k) (Eq. 2.21).  Because w factorises, S = Sx Sy Sz - 1. */
double orc_S(const orc_system* s) {
    double Sd[3];
    double Ls[3] = {s->Lx, s->Ly, s->Lz};
    for (int d = 0; d < 3; d++) {
        int nd = orc_nmax(s->alpha, Ls[d]);
        double acc = 0.0;
        for (int n = -nd; n <= nd; n++) acc += orc_w1d(n, s->alpha, Ls[d]);
        Sd[d] = acc;
    }
    return Sd[0] * Sd[1] * Sd[2] - 1.0;
}

/* Normalised cumulative table of the 1-D factor over n = -n_d..n_d:
 * sequential left-to-right prefix sum, divided by the total, last entry 1. */
void orc_cdf(double alpha, double L, int nd, double* cdf) {
    int len = 2 * nd + 1;
    double acc = 0.0;
    for (int i = 0; i < len; i++) {
        acc += orc_w1d(i - nd, alpha, L);
        cdf[i] = acc;
    }
    double total = cdf[len - 1];
    for (int i = 0; i < len; i++) cdf[i] = cdf[i] / total;
    cdf[len - 1] = 1.0;
}

/* First index whose cumulative value exceeds u (plain linear scan). */
static int orc_first_above(const double* cdf, int len, double u) {
    for (int i = 0; i < len; i++)
        if (cdf[i] > u) return i;
    return len - 1;
}

/* Draw P i.i.d. wave-vector indices from P(k) = w(k)/S, k != 0.
 * Sample l, attempt a at step s uses the Philox block with counter
 * (l, a, s, 0) and key (seed, 0); words 0,1,2 give u_d = (word >> 11) 2^-53,
 * each index is the first CDF entry above u_d, and (0,0,0) is rejected.
 * Returns 0, or -6 if a sample was rejected 64 times. */
int orc_sample_k(const orc_system* s, uint64_t seed, uint64_t step, int P, int32_t* kidx) {
    double Ls[3] = {s->Lx, s->Ly, s->Lz};
    int nd[3];
    double* cdf[3];
    for (int d = 0; d < 3; d++) {
        nd[d] = orc_nmax(s->alpha, Ls[d]);
        cdf[d] = (double*)malloc(sizeof(double) * (size_t)(2 * nd[d] + 1));
        orc_cdf(s->alpha, Ls[d], nd[d], cdf[d]);
    }
    int status = 0;
    for (int l = 0; l < P && status == 0; l++) {
        int accepted = 0;
        for (int a = 0; a < 64 && !accepted; a++) {
            uint64_t ctr[4] = {(uint64_t)l, (uint64_t)a, step, 0};
            uint64_t key[2] = {seed, 0};
            uint64_t w[4];
            orc_philox4x64_10(ctr, key, w);
            int n[3];
            for (int d = 0; d < 3; d++) {
                double u = (double)(w[d] >> 11) * 0x1.0p-53;
                n[d] = orc_first_above(cdf[d], 2 * nd[d] + 1, u) - nd[d];
            }
            if (n[0] != 0 || n[1] != 0 || n[2] != 0) {
                kidx[3 * l + 0] = n[0];
                kidx[3 * l + 1] = n[1];
                kidx[3 * l + 2] = n[2];
                accepted = 1;
            }
        }
        if (!accepted) status = -6;
    }
    for (int d = 0; d < 3; d++) free(cdf[d]);
    return status;
}

/* Metropolis variant of the sampler (the paper draws the batch "by a Metropolis
 * procedure" without fixing the proposal; Sec. 2.3).  Reading taken here: one chain per
 * batch slot l on the lattice Z^3 \ {0} with target P(k) = w(k)/S restricted to the
 * sampler's box |n_d| <= n_d; a symmetric random-walk proposal n' = n + delta with
 * delta_d uniform on {-s_d, ..., s_d}, s_d = max(1, ceil(alpha L_d / (pi sqrt 2))) (about
 * one standard deviation of the 1-D factor); acceptance min(1, w(k')/w(k)), taken as
 * u w(k) < w(k'), with w(0) = 0 and w = 0 outside the box.  Update `it` of chain l at
 * step `step` draws Philox4x64-10 with counter (l, it, step, 1) and key (seed, 0):
 * delta_d = ((word_d >> 32) (2 s_d + 1)) >> 32 minus s_d for d = 0, 1, 2, and
 * u = (word_3 >> 11) 2^-53.  Each call applies `sweeps` updates to every chain.
 * The proposal is a reading (the paper fixes none); the chain is pinned by the tests
 * against its enumerated transition kernel and its target distribution. */
int orc_metropolis_halfwidth(double alpha, double L) {
    int s = (int)ceil(alpha * L / (ORC_PI * sqrt(2.0)));
    return s < 1 ? 1 : s;
}

static double orc_w3(const orc_system* s, const int nd[3], const int n[3]) {
    if (n[0] == 0 && n[1] == 0 && n[2] == 0) return 0.0;
    for (int d = 0; d < 3; d++)
        if (n[d] < -nd[d] || n[d] > nd[d]) return 0.0;
    return orc_w1d(n[0], s->alpha, s->Lx) * orc_w1d(n[1], s->alpha, s->Ly) * orc_w1d(n[2], s->alpha, s->Lz);
}

void orc_metropolis(const orc_system* s, uint64_t seed, uint64_t step, int sweeps, int P, int32_t* state,
                    int64_t* accepted) {
    double Ls[3] = {s->Lx, s->Ly, s->Lz};
    int nd[3], hw[3];
    for (int d = 0; d < 3; d++) {
        nd[d] = orc_nmax(s->alpha, Ls[d]);
        hw[d] = orc_metropolis_halfwidth(s->alpha, Ls[d]);
    }
    int64_t acc = 0;
    for (int l = 0; l < P; l++) {
        int n[3] = {state[3 * l], state[3 * l + 1], state[3 * l + 2]};
        for (int it = 0; it < sweeps; it++) {
            uint64_t ctr[4] = {(uint64_t)l, (uint64_t)it, step, 1};
            uint64_t key[2] = {seed, 0};
            uint64_t w[4];
            orc_philox4x64_10(ctr, key, w);
            int m[3];
            for (int d = 0; d < 3; d++) {
                uint64_t span = (uint64_t)(2 * hw[d] + 1);
                m[d] = n[d] + (int)(((w[d] >> 32) * span) >> 32) - hw[d];
            }
            double u = (double)(w[3] >> 11) * 0x1.0p-53;
            double wn = orc_w3(s, nd, n), wm = orc_w3(s, nd, m);
            if (u * wn < wm) {
                n[0] = m[0]; n[1] = m[1]; n[2] = m[2];
                acc++;
            }
        }
        state[3 * l] = n[0]; state[3 * l + 1] = n[1]; state[3 * l + 2] = n[2];
    }
    if (accepted) *accepted = acc;
}

/* Every lattice k != 0 with |n_d| <= nmax_d, with its weight w(k), in the order
 * nx outer, ny, nz inner.  Returns the count; kidx/w may be NULL to count only. */
int64_t orc_full_klist(const orc_system* s, const int32_t nmax[3], int32_t* kidx, double* w) {
    int64_t c = 0;
    for (int nx = -nmax[0]; nx <= nmax[0]; nx++)
        for (int ny = -nmax[1]; ny <= nmax[1]; ny++)
            for (int nz = -nmax[2]; nz <= nmax[2]; nz++) {
                if (nx == 0 && ny == 0 && nz == 0) continue;
                if (kidx) {
                    kidx[3 * c] = nx; kidx[3 * c + 1] = ny; kidx[3 * c + 2] = nz;
                }
                if (w) {
                    double kx = 2.0 * ORC_PI * nx / s->Lx, ky = 2.0 * ORC_PI * ny / s->Ly,
                           kz = 2.0 * ORC_PI * nz / s->Lz;
                    double k2 = kx * kx + ky * ky + kz * kz;
                    w[c] = exp(-k2 / (4.0 * s->alpha * s->alpha));
                }
                c++;
            }
    return c;
}

/* ------------------------------------------------------------------------- */
/* Image charges (Eq. 3.2 and Eq. 3.3, coefficient reading A4)                */
/* ------------------------------------------------------------------------- */
static int orc_ceil_half(int l) { return (l + 1) / 2; }
static int orc_floor_half(int l) { return l / 2; }

/* gamma_+^(l), gamma_-^(l) and their derivatives w.r.t. gamma_top, gamma_bot. */
void orc_image_coeff(const orc_system* s, int l, double* gp, double* gm,
                     double* dgp_dt, double* dgp_db, double* dgm_dt, double* dgm_db) {
    int c = orc_ceil_half(l), f = orc_floor_half(l);
    double gt = s->gamma_top, gb = s->gamma_bot;
    *gp = pow(gt, c) * pow(gb, f);
    *gm = pow(gb, c) * pow(gt, f);
    if (dgp_dt) *dgp_dt = (c == 0 ? 0.0 : c * pow(gt, c - 1)) * pow(gb, f);
    if (dgp_db) *dgp_db = pow(gt, c) * (f == 0 ? 0.0 : f * pow(gb, f - 1));
    if (dgm_dt) *dgm_dt = pow(gb, c) * (f == 0 ? 0.0 : f * pow(gt, f - 1));
    if (dgm_db) *dgm_db = (c == 0 ? 0.0 : c * pow(gb, c - 1)) * pow(gt, f);
}

/* z_{j+}^(l) = (-1)^l z + 2 ceil(l/2) H,  z_{j-}^(l) = (-1)^l z - 2 floor(l/2) H. */
void orc_image_z(const orc_system* s, int l, double z, double* zp, double* zm) {
    double sg = (l % 2 == 0) ? 1.0 : -1.0;
    *zp = sg * z + 2.0 * orc_ceil_half(l) * s->H;
    *zm = sg * z - 2.0 * orc_floor_half(l) * s->H;
}

/* c_M = 1 + sum_l (-1)^l (gamma_+^(l) + gamma_-^(l)): d(z_j + sum_l gamma z_img)/dz_j. */
double orc_cM(const orc_system* s) {
    double c = 1.0;
    for (int l = 1; l <= s->M; l++) {
        double gp, gm;
        orc_image_coeff(s, l, &gp, &gm, NULL, NULL, NULL, NULL);
        c += ((l % 2 == 0) ? 1.0 : -1.0) * (gp + gm);
    }
    return c;
}

/* ------------------------------------------------------------------------- */
/* Structure factors (Theorem 3.3, Eq. 3.17) and the k-space sum                        */
/* ------------------------------------------------------------------------- */
static double orc_phase(const orc_system* s, const int32_t* n, double x, double y, double z) {
    /* k . r = 2 pi (nx x / Lx + ny y / Ly + nz z / Lz) */
    return 2.0 * ORC_PI * ((double)n[0] * x / s->Lx + (double)n[1] * y / s->Ly + (double)n[2] * z / s->Lz);
}

/* rhobar^M-type sum of one charge at (x,y,z) with all its images:
 *   e^{-i k.r} + sum_l (gamma_+ e^{-i k.r_+} + gamma_- e^{-i k.r_-})
 * and, optionally, the same with the gamma derivatives as coefficients. */
static double complex orc_conj_with_images(const orc_system* s, const int32_t* n, double x, double y,
                                           double z, double complex* d_dt, double complex* d_db) {
    double complex acc = cexp(-I * orc_phase(s, n, x, y, z));
    double complex at = 0.0, ab = 0.0;
    for (int l = 1; l <= s->M; l++) {
        double gp, gm, gpt, gpb, gmt, gmb, zp, zm;
        orc_image_coeff(s, l, &gp, &gm, &gpt, &gpb, &gmt, &gmb);
        orc_image_z(s, l, z, &zp, &zm);
        double complex ep = cexp(-I * orc_phase(s, n, x, y, zp));
        double complex em = cexp(-I * orc_phase(s, n, x, y, zm));
        acc += gp * ep + gm * em;
        at += gpt * ep + gmt * em;
        ab += gpb * ep + gmb * em;
    }
    if (d_dt) *d_dt = at;
    if (d_db) *d_db = ab;
    return acc;
}

/* Explicit structure factors for K wave vectors:
 *   rho_k    = sum_j q_j e^{i k.r_j}
 *   rhobarM_k = sum_j q_j [e^{-i k.r_j} + sum_{l=1..M} (gamma_+ e^{-i k.r_{j+}} + gamma_- e^{-i k.r_{j-}})]
 * and d rhobarM / d gamma_top, d gamma_bot (each may be NULL). */
void orc_sf_explicit(const orc_system* s, int64_t N, const double* pos, const double* q, int64_t K,
                     const int32_t* kidx, double complex* rho, double complex* rhobarM,
                     double complex* drb_dt, double complex* drb_db) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t c = 0; c < K; c++) {
        const int32_t* n = kidx + 3 * c;
        double complex r = 0.0, rb = 0.0, rt = 0.0, rbb = 0.0;
        for (int64_t j = 0; j < N; j++) {
            double x = pos[3 * j], y = pos[3 * j + 1], z = pos[3 * j + 2];
            double complex dt, db;
            r += q[j] * cexp(I * orc_phase(s, n, x, y, z));
            rb += q[j] * orc_conj_with_images(s, n, x, y, z, &dt, &db);
            rt += q[j] * dt;
            rbb += q[j] * db;
        }
        if (rho) rho[c] = r;
        if (rhobarM) rhobarM[c] = rb;
        if (drb_dt) drb_dt[c] = rt;
        if (drb_db) drb_db[c] = rbb;
    }
}

/* Re-calibration coefficients of Sec. 3.4 (defined after Eq. 3.27):
 *   Y_odd(kz)  = sum_{l odd}  [gamma_+^(l) e^{ i kz (l+1) H} + gamma_-^(l) e^{-i kz (l-1) H}]
 *   Y_even(kz) = sum_{l even} [gamma_+^(l) e^{ i kz l H}     + gamma_-^(l) e^{-i kz l H}]   */
void orc_Y(const orc_system* s, double kz, double complex* Yodd, double complex* Yeven) {
    double complex yo = 0.0, ye = 0.0;
    for (int l = 1; l <= s->M; l++) {
        double gp, gm;
        orc_image_coeff(s, l, &gp, &gm, NULL, NULL, NULL, NULL);
        if (l % 2 == 1)
            yo += gp * cexp(I * kz * (l + 1) * s->H) + gm * cexp(-I * kz * (l - 1) * s->H);
        else
            ye += gp * cexp(I * kz * l * s->H) + gm * cexp(-I * kz * l * s->H);
    }
    *Yodd = yo;
    *Yeven = ye;
}

/* d Y_odd / d gamma and d Y_even / d gamma (gamma = gamma_top if which == 0, else
 * gamma_bot): the same sums with each gamma_+-^(l) replaced by its derivative. */
void orc_dY(const orc_system* s, double kz, int which, double complex* dYodd, double complex* dYeven) {
    double complex yo = 0.0, ye = 0.0;
    for (int l = 1; l <= s->M; l++) {
        double gp, gm, gpt, gpb, gmt, gmb;
        orc_image_coeff(s, l, &gp, &gm, &gpt, &gpb, &gmt, &gmb);
        double dp = which == 0 ? gpt : gpb, dm = which == 0 ? gmt : gmb;
        if (l % 2 == 1)
            yo += dp * cexp(I * kz * (l + 1) * s->H) + dm * cexp(-I * kz * (l - 1) * s->H);
        else
            ye += dp * cexp(I * kz * l * s->H) + dm * cexp(-I * kz * l * s->H);
    }
    *dYodd = yo;
    *dYeven = ye;
}

/* Re-calibrated structure factors: with sigma_k = sum_j q_j e^{i khat.r_j},
 * khat = (kx, ky, -kz), the image sum decouples (Sec. 3.4) into
 *   rhobarM_k = (1 + conj(Y_even)) conj(rho_k) + conj(Y_odd) conj(sigma_k).
 * Returns rho, sigma and rhobarM (any may be NULL). */
void orc_sf_recal(const orc_system* s, int64_t N, const double* pos, const double* q, int64_t K,
                  const int32_t* kidx, double complex* rho, double complex* sigma,
                  double complex* rhobarM) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t c = 0; c < K; c++) {
        const int32_t* n = kidx + 3 * c;
        int32_t nh[3] = {n[0], n[1], -n[2]};
        double complex r = 0.0, sg = 0.0;
        for (int64_t j = 0; j < N; j++) {
            double x = pos[3 * j], y = pos[3 * j + 1], z = pos[3 * j + 2];
            r += q[j] * cexp(I * orc_phase(s, n, x, y, z));
            sg += q[j] * cexp(I * orc_phase(s, nh, x, y, z));
        }
        double kz = 2.0 * ORC_PI * n[2] / s->Lz;
        double complex yo, ye;
        orc_Y(s, kz, &yo, &ye);
        if (rho) rho[c] = r;
        if (sigma) sigma[c] = sg;
        if (rhobarM) rhobarM[c] = (1.0 + conj(ye)) * conj(r) + conj(yo) * conj(sg);
    }
}

/* Sums over particles used by U_IBC^M (Eq. 3.18):
 *   mu  = sum_i q_i z_i
 *   Zs  = sum_j q_j [z_j + sum_l (gamma_+ z_{j+} + gamma_- z_{j-})]
 *   Zt, Zb = d Zs / d gamma_top, d gamma_bot. */
static void orc_ibc_sums(const orc_system* s, int64_t N, const double* pos, const double* q, double* mu,
                         double* Zs, double* Zt, double* Zb) {
    double m = 0, z0 = 0, zt = 0, zb = 0;
    for (int64_t j = 0; j < N; j++) {
        double z = pos[3 * j + 2];
        m += q[j] * z;
        double a = z, at = 0, ab = 0;
        for (int l = 1; l <= s->M; l++) {
            double gp, gm, gpt, gpb, gmt, gmb, zp, zm;
            orc_image_coeff(s, l, &gp, &gm, &gpt, &gpb, &gmt, &gmb);
            orc_image_z(s, l, z, &zp, &zm);
            a += gp * zp + gm * zm;
            at += gpt * zp + gmt * zm;
            ab += gpb * zp + gmb * zm;
        }
        z0 += q[j] * a;
        zt += q[j] * at;
        zb += q[j] * ab;
    }
    *mu = m; *Zs = z0; *Zt = zt; *Zb = zb;
}

/*
 * k-space energy, force and gradients for a list of K wave vectors with weights W_k:
 *   U_k    = (2 pi / V) sum_k W_k Re(rho_k rhobarM_k) / k^2
 *   U_self = -(alpha / sqrt(pi)) sum_i q_i^2
 *   U_IBC  = (2 pi / V) mu Zs
 * With W_k = S/P over a sampled batch this is the RBE estimator (Eq. 3.26 and the
 * matching energy); with W_k = w(k) over the lattice it is the full k-sum
 * (first term of Eq. 3.16).
 *
 * Forces (F = -grad U, U_k + U_IBC) and dU/dq_i (U_k + U_self + U_IBC) are
 * returned for n_targets particles (targets == NULL means all N).  The gradient
 * of Re(rho rhobarM) w.r.t. r_i is taken
 *   mode 0: by the chain rule on the explicit image sum: grad rho = i k q_i e^{ik.r_i},
 *           grad rhobarM = -i q_i [k e^{-ik.r_i} + sum_l gamma (kx,ky,(-1)^l kz) e^{-ik.r_img}];
 *   mode 1: by Eq. 3.25 with rho^M = conj(rhobarM) from the re-calibration.
 * energy[3] = {U_k, U_self, U_IBC}; dUdgamma[2] = {dU/dgamma_top, dU/dgamma_bot}
 * (mode 0: derivative of every explicit image coefficient; mode 1: the same
 * derivative taken through Y_odd, Y_even).  Any output may be NULL.
 */
int orc_kspace(const orc_system* s, int64_t N, const double* pos, const double* q, int64_t K,
               const int32_t* kidx, const double* W, int mode, int64_t n_targets,
               const int64_t* targets, double* energy, double* force, double* dUdq,
               double* dUdgamma) {
    double V = s->Lx * s->Ly * s->Lz;
    double pref = 2.0 * ORC_PI / V;
    double complex* rho = (double complex*)malloc(sizeof(double complex) * (size_t)K);
    double complex* rb = (double complex*)malloc(sizeof(double complex) * (size_t)K);
    double complex* rbt = NULL;
    double complex* rbb = NULL;
    double complex* sig = NULL;
    if (!rho || !rb) { free(rho); free(rb); return -7; }
    if (mode == 0) {
        rbt = (double complex*)malloc(sizeof(double complex) * (size_t)K);
        rbb = (double complex*)malloc(sizeof(double complex) * (size_t)K);
        orc_sf_explicit(s, N, pos, q, K, kidx, rho, rb, rbt, rbb);
    } else {
        sig = (double complex*)malloc(sizeof(double complex) * (size_t)K);
        orc_sf_recal(s, N, pos, q, K, kidx, rho, sig, rb);
        /* d rhobarM / d gamma = conj(dY_even) conj(rho) + conj(dY_odd) conj(sigma) */
        rbt = (double complex*)malloc(sizeof(double complex) * (size_t)K);
        rbb = (double complex*)malloc(sizeof(double complex) * (size_t)K);
        for (int64_t c = 0; c < K; c++) {
            double kz = 2.0 * ORC_PI * kidx[3 * c + 2] / s->Lz;
            double complex dyo, dye;
            orc_dY(s, kz, 0, &dyo, &dye);
            rbt[c] = conj(dye) * conj(rho[c]) + conj(dyo) * conj(sig[c]);
            orc_dY(s, kz, 1, &dyo, &dye);
            rbb[c] = conj(dye) * conj(rho[c]) + conj(dyo) * conj(sig[c]);
        }
    }
    double mu, Zs, Zt, Zb;
    orc_ibc_sums(s, N, pos, q, &mu, &Zs, &Zt, &Zb);
    double cM = orc_cM(s);

    if (energy) {
        double uk = 0.0, q2 = 0.0;
        for (int64_t c = 0; c < K; c++) {
            const int32_t* n = kidx + 3 * c;
            double kx = 2.0 * ORC_PI * n[0] / s->Lx, ky = 2.0 * ORC_PI * n[1] / s->Ly,
                   kz = 2.0 * ORC_PI * n[2] / s->Lz;
            double k2 = kx * kx + ky * ky + kz * kz;
            uk += W[c] * creal(rho[c] * rb[c]) / k2;
        }
        for (int64_t j = 0; j < N; j++) q2 += q[j] * q[j];
        energy[0] = pref * uk;
        energy[1] = -s->alpha / sqrt(ORC_PI) * q2;
        energy[2] = pref * mu * Zs;
    }
    if (dUdgamma) {
        double gt = 0.0, gb = 0.0;
        for (int64_t c = 0; c < K; c++) {
            const int32_t* n = kidx + 3 * c;
            double kx = 2.0 * ORC_PI * n[0] / s->Lx, ky = 2.0 * ORC_PI * n[1] / s->Ly,
                   kz = 2.0 * ORC_PI * n[2] / s->Lz;
            double k2 = kx * kx + ky * ky + kz * kz;
            gt += W[c] * creal(rho[c] * rbt[c]) / k2;
            gb += W[c] * creal(rho[c] * rbb[c]) / k2;
        }
        dUdgamma[0] = pref * (gt + mu * Zt);
        dUdgamma[1] = pref * (gb + mu * Zb);
    }
    int64_t nt = targets ? n_targets : N;
    if (force || dUdq) {
#pragma omp parallel for schedule(dynamic, 16)
        for (int64_t t = 0; t < nt; t++) {
            int64_t i = targets ? targets[t] : t;
            double x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2];
            double fx = 0, fy = 0, fz = 0, dq = 0;
            for (int64_t c = 0; c < K; c++) {
                const int32_t* n = kidx + 3 * c;
                double kx = 2.0 * ORC_PI * n[0] / s->Lx, ky = 2.0 * ORC_PI * n[1] / s->Ly,
                       kz = 2.0 * ORC_PI * n[2] / s->Lz;
                double k2 = kx * kx + ky * ky + kz * kz;
                double wk = W[c] / k2;
                double complex e = cexp(I * orc_phase(s, n, x, y, z));
                double gx, gy, gz;
                if (mode == 0) {
                    /* grad_i Re(rho rhobarM) = Re[(grad rho) rhobarM + rho (grad rhobarM)] */
                    double complex tx = I * kx * q[i] * e * rb[c];
                    double complex ty = I * ky * q[i] * e * rb[c];
                    double complex tz = I * kz * q[i] * e * rb[c];
                    double complex ce = conj(e);
                    double complex sx = -I * kx * ce, sy = -I * ky * ce, sz = -I * kz * ce;
                    for (int l = 1; l <= s->M; l++) {
                        double gp, gm, zp, zm;
                        orc_image_coeff(s, l, &gp, &gm, NULL, NULL, NULL, NULL);
                        orc_image_z(s, l, z, &zp, &zm);
                        double sgn = (l % 2 == 0) ? 1.0 : -1.0;
                        double complex ep = cexp(-I * orc_phase(s, n, x, y, zp));
                        double complex em = cexp(-I * orc_phase(s, n, x, y, zm));
                        double complex g = gp * ep + gm * em;
                        sx += -I * kx * g;
                        sy += -I * ky * g;
                        sz += -I * (sgn * kz) * g;
                    }
                    gx = creal(tx + rho[c] * q[i] * sx);
                    gy = creal(ty + rho[c] * q[i] * sy);
                    gz = creal(tz + rho[c] * q[i] * sz);
                } else {
                    /* Eq. 3.25: q_i k Im[e^{-ik.r_i}(rho + rho^M) + sum_{l even} (...) rho]
                     *         + q_i khat Im[sum_{l odd} (...) rho]                        */
                    double complex rhoM = conj(rb[c]);
                    double complex ce = conj(e);
                    double complex ev = 0.0, od = 0.0;
                    for (int l = 1; l <= s->M; l++) {
                        double gp, gm, zp, zm;
                        orc_image_coeff(s, l, &gp, &gm, NULL, NULL, NULL, NULL);
                        orc_image_z(s, l, z, &zp, &zm);
                        double complex g = gp * cexp(-I * orc_phase(s, n, x, y, zp)) +
                                           gm * cexp(-I * orc_phase(s, n, x, y, zm));
                        if (l % 2 == 0) ev += g; else od += g;
                    }
                    double a1 = cimag(ce * (rho[c] + rhoM) + ev * rho[c]);
                    double a2 = cimag(od * rho[c]);
                    gx = q[i] * (kx * a1 + kx * a2);
                    gy = q[i] * (ky * a1 + ky * a2);
                    gz = q[i] * (kz * a1 - kz * a2);
                }
                fx -= wk * gx;
                fy -= wk * gy;
                fz -= wk * gz;
                if (dUdq) {
                    double complex imgs = orc_conj_with_images(s, n, x, y, z, NULL, NULL);
                    dq += wk * creal(e * rb[c] + rho[c] * imgs);
                }
            }
            if (force) {
                /* -d U_IBC / d z_i = -(2pi/V) [q_i Zs + mu q_i c_M] */
                force[3 * t + 0] = pref * fx;
                force[3 * t + 1] = pref * fy;
                force[3 * t + 2] = pref * fz - pref * (q[i] * Zs + mu * q[i] * cM);
            }
            if (dUdq) {
                /* d U_IBC / d q_i = (2pi/V) [z_i Zs + mu Z_i] */
                double Zi = z;
                for (int l = 1; l <= s->M; l++) {
                    double gp, gm, zp, zm;
                    orc_image_coeff(s, l, &gp, &gm, NULL, NULL, NULL, NULL);
                    orc_image_z(s, l, z, &zp, &zm);
                    Zi += gp * zp + gm * zm;
                }
                dUdq[t] = pref * dq - 2.0 * s->alpha / sqrt(ORC_PI) * q[i] + pref * (z * Zs + mu * Zi);
            }
        }
    }
    free(rho); free(rb); free(rbt); free(rbb); free(sig);
    return 0;
}

/* Structure factors as the GPU boundary reports them: rho_k and
 * sigma_k = sum_j q_j e^{i khat.r_j} (re, im, re, im per k), mu = sum q z. */
void orc_rho_sigma(const orc_system* s, int64_t N, const double* pos, const double* q, int64_t K,
                   const int32_t* kidx, double* out4) {
    double complex* r = (double complex*)malloc(sizeof(double complex) * (size_t)K);
    double complex* g = (double complex*)malloc(sizeof(double complex) * (size_t)K);
    orc_sf_recal(s, N, pos, q, K, kidx, r, g, NULL);
    for (int64_t c = 0; c < K; c++) {
        out4[4 * c + 0] = creal(r[c]);
        out4[4 * c + 1] = cimag(r[c]);
        out4[4 * c + 2] = creal(g[c]);
        out4[4 * c + 3] = cimag(g[c]);
    }
    free(r); free(g);
}

/* ------------------------------------------------------------------------- */
/* Real space with images, by brute force (Eq. 3.12)                           */
/* ------------------------------------------------------------------------- */
/*
 * Sources seen by particle i: every real charge j in every xy replica except
 * (j = i, n = 0), and every image of every charge (own images included) in every
 * xy replica, with weight gamma_+^(l) or gamma_-^(l).  Pairs farther than r_c are
 * dropped.  The force is the erfc-screened field of the sources times q_i:
 *   F_i = q_i sum_src q_src g [erfc(a r)/r^2 + (2a/sqrt(pi)) e^{-a^2 r^2}/r] (r_i - r_src)/r
 * and the energy 1/2 sum_i q_i sum_src q_src g erfc(a r)/r.  This is the gradient of
 * Eq. 3.12 because every image term is symmetric under i <-> j.
 * energy (if not NULL) is summed over the targets.
 */
int orc_real_space(const orc_system* s, double r_c, int64_t N, const double* pos, const double* q,
                   int64_t n_targets, const int64_t* targets, double* force, double* energy) {
    int64_t nt = targets ? n_targets : N;
    int rx = (int)ceil(r_c / s->Lx), ry = (int)ceil(r_c / s->Ly);
    double a = s->alpha, rc2 = r_c * r_c;
    double twoa_sqpi = 2.0 * a / sqrt(ORC_PI);
    double etot = 0.0;
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : etot)
    for (int64_t t = 0; t < nt; t++) {
        int64_t i = targets ? targets[t] : t;
        double xi = pos[3 * i], yi = pos[3 * i + 1], zi = pos[3 * i + 2];
        double fx = 0, fy = 0, fz = 0, e = 0;
        for (int64_t j = 0; j < N; j++) {
            double xj = pos[3 * j], yj = pos[3 * j + 1], zj = pos[3 * j + 2];
            for (int l = 0; l <= s->M; l++) {
                int nimg = (l == 0) ? 1 : 2;
                for (int side = 0; side < nimg; side++) {
                    double g, zs;
                    if (l == 0) { g = 1.0; zs = zj; }
                    else {
                        double gp, gm, zp, zm;
                        orc_image_coeff(s, l, &gp, &gm, NULL, NULL, NULL, NULL);
                        orc_image_z(s, l, zj, &zp, &zm);
                        g = side == 0 ? gp : gm;
                        zs = side == 0 ? zp : zm;
                    }
                    double dz = zi - zs;
                    if (dz * dz >= rc2 || g == 0.0) continue;
                    for (int nx = -rx; nx <= rx; nx++)
                        for (int ny = -ry; ny <= ry; ny++) {
                            if (l == 0 && j == i && nx == 0 && ny == 0) continue;
                            double dx = xi - (xj + nx * s->Lx), dy = yi - (yj + ny * s->Ly);
                            double r2 = dx * dx + dy * dy + dz * dz;
                            if (r2 >= rc2) continue;
                            double r = sqrt(r2);
                            double ec = erfc(a * r);
                            double fr = q[j] * g * (ec / r2 + twoa_sqpi * exp(-a * a * r2) / r) / r;
                            fx += fr * dx; fy += fr * dy; fz += fr * dz;
                            e += q[j] * g * ec / r;
                        }
                }
            }
        }
        if (force) {
            force[3 * t] = q[i] * fx;
            force[3 * t + 1] = q[i] * fy;
            force[3 * t + 2] = q[i] * fz;
        }
        etot += 0.5 * q[i] * e;
    }
    if (energy) *energy = etot;
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Parameter rules                                                           */
/* ------------------------------------------------------------------------- */
/* Eq. 3.10: M ~ (2 ln eps - 4 pi H/L - ln|gt gb|) / (ln|gt gb| - 4 pi H/L), L = max(Lx,Ly),
 * rounded up and capped at 64.  With gt gb = 0 the series ends after the first
 * level (M = 1), or has no images at all when both contrasts vanish (M = 0). */
int orc_auto_M(double Lx, double Ly, double H, double gt, double gb, double eps) {
    if (gt == 0.0 && gb == 0.0) return 0;
    if (gt * gb == 0.0) return 1;
    double L = Lx > Ly ? Lx : Ly;
    double t = 4.0 * ORC_PI * H / L;
    double lg = log(fabs(gt * gb));
    double m = (2.0 * log(eps) - t - lg) / (lg - t);
    int M = (int)ceil(m);
    if (M < 1) M = 1;
    if (M > 64) M = 64;
    return M;
}

/* Eq. 3.23: L_z >= (M+1) H + max{ L/(2pi) ln(1/eps), sqrt(ln(1/eps))/alpha }, rounded
 * up to an integer.  With M = 0 this is the homogeneous rule of Eq. 2.19. */
double orc_auto_Lz(double Lx, double Ly, double H, int M, double alpha, double eps) {
    double L = Lx > Ly ? Lx : Ly;
    double a = L / (2.0 * ORC_PI) * log(1.0 / eps);
    double b = sqrt(log(1.0 / eps)) / alpha;
    return ceil((M + 1) * H + (a > b ? a : b));
}

/* Sec. 2.3: alpha ~ N^(1/3) / (Lx Ly H)^(1/3). */
double orc_auto_alpha(int64_t N, double Lx, double Ly, double H) {
    return cbrt((double)N / (Lx * Ly * H));
}
