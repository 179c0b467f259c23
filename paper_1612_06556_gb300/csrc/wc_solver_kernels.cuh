// Launchers of the fused BiCGStab vector updates (wc_blas.cu) on FP64
// fields.  Each runs on S.stream, reduces into S.red and updates the scalars
// S.scal on the device (no host synchronisation).
#pragma once

#include "wc_internal.cuh"

namespace wc {

int reduce_grid(const ReduceScratch &rs, long long n);

// r = b - r (r holds M x), rhat = r, p = v = 0; scalars reset
cudaError_t bicg_init(wc_lattice lat, SolverState &S, const double2 *b, double2 *r, double2 *rhat, double2 *p,
                      double2 *v);
// p = r + beta (p - omega v); pp = |p|^2
cudaError_t bicg_p(wc_lattice lat, SolverState &S, const double2 *r, const double2 *v, double2 *p);
// alpha = rho / <rhat, v>
cudaError_t bicg_alpha(wc_lattice lat, SolverState &S, const double2 *rhat, const double2 *v);
// s = r - alpha v; ss = |s|^2
cudaError_t bicg_s(wc_lattice lat, SolverState &S, const double2 *r, const double2 *v, double2 *s);
// omega = <t, s> / <t, t>
cudaError_t bicg_omega(wc_lattice lat, SolverState &S, const double2 *t, const double2 *s);
// x += alpha phat + omega shat; r = s - omega t; rho, beta, rr updated
cudaError_t bicg_xr(wc_lattice lat, SolverState &S, double2 *x, const double2 *phat, const double2 *shat,
                    const double2 *s, const double2 *t, double2 *r, const double2 *rhat);
// r = b - r (r holds M x); rr = |r|^2
cudaError_t residual(wc_lattice lat, SolverState &S, const double2 *b, double2 *r);
// S.red.result[0] = |a|^2
cudaError_t norm2_to_result(wc_lattice lat, SolverState &S, const double2 *a);

}  // namespace wc
