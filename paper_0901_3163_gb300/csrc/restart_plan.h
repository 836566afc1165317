// The FP64 small problem at the end of one Lan-DR / MinRes-DR restart cycle
// (arXiv:0901.3163, Sec. 1-2), on the host.
#pragma once

#include <vector>

namespace dlz {

struct RestartPlan {
    std::vector<double> y;       // m     : x += V_m y
    std::vector<double> s, q;    // MinRes-DR: LS residual c - Tbar y, unit vector spanning range(Tbar)^perp
    double rho = 0.0;            // Lan-DR: the residual is rho v_{m+1}
    std::vector<double> P;       // (m+1) x (k+1): V_{k+1} <- V_{m+1} P
    std::vector<double> Tn, cn;  // new Tbar ((m+1) x m, rows/cols < k+1 filled) and c
    std::vector<double> theta, res;   // kept (harmonic) Ritz values and residuals
};

// The small FP64 problem of one cycle (host), in two parts so that the GPU can
// update x and compute the true residual while the host does the eigenproblem.
// T: (m+1) x m row-major Tbar_m.
// Part 1: the linear-system coefficients y (Lan-DR: Galerkin T_m y = c; MinRes-DR:
// least squares min ||c - Tbar y||, with s = c - Tbar y and q spanning range(Tbar)^perp).
int plan_solve(bool harmonic, int m, const std::vector<double> &T, const std::vector<double> &c, RestartPlan &o);
// Part 2: (harmonic) Ritz pairs, the restart matrix P and the new Tbar and c; Anorm
// becomes max(Anorm, max |eig T_m|).
int plan_finish(bool harmonic, int m, int k, const std::vector<double> &T, double &Anorm, RestartPlan &o);

}  // namespace dlz
