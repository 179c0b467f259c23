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

// FP32 counterparts for the reliable-update solver (FP32 fields)
// rhat = r, p = v = xlo = 0; scalars reset from |r|^2
cudaError_t lo_init(wc_lattice lat, SolverState &S, const float4 *r, float4 *rhat, float4 *p, float4 *v,
                    float4 *xlo);
cudaError_t lo_p(wc_lattice lat, SolverState &S, const float4 *r, const float4 *v, float4 *p);
cudaError_t lo_alpha(wc_lattice lat, SolverState &S, const float4 *rhat, const float4 *v);
cudaError_t lo_s(wc_lattice lat, SolverState &S, const float4 *r, const float4 *v, float4 *s);
cudaError_t lo_omega(wc_lattice lat, SolverState &S, const float4 *t, const float4 *s);
// xlo += alpha phat + omega shat; r = s - omega t; rho, beta, rr updated
cudaError_t lo_xr(wc_lattice lat, SolverState &S, float4 *xlo, const float4 *phat, const float4 *shat,
                  const float4 *s, const float4 *t, float4 *r, const float4 *rhat);
// after r was replaced: rho = <rhat, r>, beta from rho0 (rr untouched)
cudaError_t lo_rho(wc_lattice lat, SolverState &S, const float4 *rhat, const float4 *r);
// x (FP64) += xlo (FP32); xlo = 0
cudaError_t hp_add_lo(wc_lattice lat, SolverState &S, double2 *x, float4 *xlo);

}  // namespace wc
