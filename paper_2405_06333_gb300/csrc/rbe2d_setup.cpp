// Host-side setup of librbe2d: the automatic parameter rules, the k-sampler tables and
// the image-series constants.  Plain C++, float64, compiled with -ffp-contract=off so
// the tables are identical on every host architecture.
#include "rbe2d_setup.h"

#include <cmath>

namespace rbe2d {

static const double kPi = 3.14159265358979323846;

// Eq. 3.10: the number of reflection levels for tolerance eps,
//   M ~ (2 ln eps - 4 pi H/L - ln|gt gb|) / (ln|gt gb| - 4 pi H/L),  L = max(Lx, Ly),
// rounded up and capped at 64.  When gt gb = 0 the series has at most one level.
int auto_M(double Lx, double Ly, double H, double gt, double gb, double eps) {
    if (gt == 0.0 && gb == 0.0) return 0;
    const double g = gt * gb;
    if (g == 0.0) return 1;
    const double L = Lx > Ly ? Lx : Ly;
    const double aspect = 4.0 * kPi * H / L;
    const double lng = std::log(std::fabs(g));
    double m = std::ceil((2.0 * std::log(eps) - aspect - lng) / (lng - aspect));
    if (m < 1.0) m = 1.0;
    if (m > 64.0) m = 64.0;
    return (int)m;
}

// Eq. 3.23: Lz >= (M+1) H + max{ L ln(1/eps) / (2 pi), sqrt(ln(1/eps)) / alpha }, rounded up.
double auto_Lz(double Lx, double Ly, double H, int M, double alpha, double eps) {
    const double L = Lx > Ly ? Lx : Ly;
    const double l1 = L / (2.0 * kPi) * std::log(1.0 / eps);
    const double l2 = std::sqrt(std::log(1.0 / eps)) / alpha;
    return std::ceil((double)(M + 1) * H + (l1 > l2 ? l1 : l2));
}

// 1-D factor of the Gaussian weight: exp(-(2 pi n/L)^2 / (4 alpha^2)) = exp(-(pi n/(alpha L))^2).
static double w1(int n, double alpha, double L) {
    const double a = kPi * (double)n / (alpha * L);
    return std::exp(-(a * a));
}

int table_half_width(double alpha, double L) {
    // terms beyond this index are below exp(-46) of the central one
    return (int)std::ceil(alpha * L * std::sqrt(46.0) / kPi);
}

// Normalised cumulative table over n = -h..h, built left to right; the last entry is 1.
// Returns the sum of the 1-D factor (S_d).
double build_cdf(double alpha, double L, std::vector<double>* cdf) {
    const int h = table_half_width(alpha, L);
    cdf->assign(2 * h + 1, 0.0);
    double run = 0.0;
    for (int i = 0; i <= 2 * h; i++) {
        run += w1(i - h, alpha, L);
        (*cdf)[i] = run;
    }
    const double total = (*cdf)[2 * h];
    for (int i = 0; i <= 2 * h; i++) (*cdf)[i] = (*cdf)[i] / total;
    (*cdf)[2 * h] = 1.0;
    return total;
}

// The 1-D factor itself over n = -h..h (the Metropolis acceptance ratios use it).
void build_weights(double alpha, double L, std::vector<double>* w) {
    const int h = table_half_width(alpha, L);
    w->assign(2 * h + 1, 0.0);
    for (int i = 0; i <= 2 * h; i++) (*w)[i] = w1(i - h, alpha, L);
}

// Half-width of the Metropolis random-walk proposal in one dimension: about one standard
// deviation alpha L / (pi sqrt 2) of the 1-D factor, at least 1.
int metropolis_half_width(double alpha, double L) {
    const int s = (int)std::ceil(alpha * L / (kPi * std::sqrt(2.0)));
    return s < 1 ? 1 : s;
}

// Guide table of a normalised cumulative table: guide[g] = first index whose value
// exceeds g / len (g = 0..len-1).  A search for u starts at guide[floor(u len)].
void build_guide(const std::vector<double>& cdf, std::vector<int>* guide) {
    const int len = (int)cdf.size();
    guide->assign(len, len - 1);
    int i = 0;
    for (int g = 0; g < len; g++) {
        const double t = (double)g / (double)len;
        while (i < len - 1 && !(cdf[i] > t)) i++;
        (*guide)[g] = i;
    }
}

// Image-series constants of U_IBC^M (Eq. 3.18).  With gamma_+^(l) = gt^ceil(l/2) gb^floor(l/2),
// gamma_-^(l) = gb^ceil(l/2) gt^floor(l/2) and the image heights of Eq. 3.3,
//   sum_l (gamma_+ z_+ + gamma_- z_-) = z (cM - 1) + H dM
//   cM = 1 + sum_l (-1)^l (gamma_+ + gamma_-),  dM = sum_l (2 ceil(l/2) gamma_+ - 2 floor(l/2) gamma_-).
void image_constants(double gt, double gb, int M, ImageConsts* out) {
    ImageConsts c = {1.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int l = 1; l <= M; l++) {
        const int up = (l + 1) / 2, dn = l / 2;
        const double gp = std::pow(gt, up) * std::pow(gb, dn);
        const double gm = std::pow(gb, up) * std::pow(gt, dn);
        const double gp_t = (up ? up * std::pow(gt, up - 1) : 0.0) * std::pow(gb, dn);
        const double gp_b = std::pow(gt, up) * (dn ? dn * std::pow(gb, dn - 1) : 0.0);
        const double gm_t = std::pow(gb, up) * (dn ? dn * std::pow(gt, dn - 1) : 0.0);
        const double gm_b = (up ? up * std::pow(gb, up - 1) : 0.0) * std::pow(gt, dn);
        const double sgn = (l % 2 == 0) ? 1.0 : -1.0;
        c.cM += sgn * (gp + gm);
        c.dcM_t += sgn * (gp_t + gm_t);
        c.dcM_b += sgn * (gp_b + gm_b);
        c.dM += 2.0 * up * gp - 2.0 * dn * gm;
        c.ddM_t += 2.0 * up * gp_t - 2.0 * dn * gm_t;
        c.ddM_b += 2.0 * up * gp_b - 2.0 * dn * gm_b;
    }
    *out = c;
}

}  // namespace rbe2d
