// plan_host.h -- host-side helpers of the plan (wedges, boxes, KB kernel,
// Hermitian eigensolver, Jacobi SVD), shared by plan.cpp and the host utilities of api.cpp.
#pragma once

#include <complex>
#include <string>
#include <utility>
#include <vector>

#include "fio_internal.h"

namespace fio {

int default_L(int N);
int wedge_of(int k1, int k2, int L);
bool wedge_geometry(const std::vector<std::pair<int, int>> &pts, double sigma, int w,
                    WedgeDev &wd, std::vector<RowDev> &rows, std::vector<int> &k1s,
                    std::vector<int> &k2s, std::vector<int> &x1p, std::vector<int> &x2p,
                    std::string &err);
int kb_width_for(double eps);
double kb_beta_for(int w, double sigma);
double kb_phi_host(double s, int w, double beta);
double kb_phihat_host(double nu, int w, double beta);
void herm_eig(int n, std::vector<std::complex<double>> A, std::vector<double> &ev,
              std::vector<std::complex<double>> &V);
void svd_jacobi(int m, int n, std::vector<std::complex<double>> &A, std::vector<double> &sig,
                std::vector<std::complex<double>> &V);
void svd_right_pivoted(int n, const std::vector<std::complex<double>> &R, std::vector<double> &sig,
                       std::vector<std::complex<double>> &V);

}  // namespace fio
