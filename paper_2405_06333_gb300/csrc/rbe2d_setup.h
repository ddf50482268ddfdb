// Host-side setup helpers of librbe2d (parameter rules, sampler tables, image constants).
#pragma once

#include <vector>

namespace rbe2d {

struct ImageConsts {
    double cM, dM, dcM_t, dcM_b, ddM_t, ddM_b;
};

int auto_M(double Lx, double Ly, double H, double gt, double gb, double eps);
double auto_Lz(double Lx, double Ly, double H, int M, double alpha, double eps);
int table_half_width(double alpha, double L);
double build_cdf(double alpha, double L, std::vector<double>* cdf);
void build_weights(double alpha, double L, std::vector<double>* w);
int metropolis_half_width(double alpha, double L);
void build_guide(const std::vector<double>& cdf, std::vector<int>* guide);
void image_constants(double gt, double gb, int M, ImageConsts* out);

}  // namespace rbe2d
