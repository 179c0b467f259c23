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

// Low-precision counterparts for the reliable-update and nested solvers:
// the BiCGStab vectors are FP32 fields, or FP16 fields (per-site scale,
// FP32 arithmetic); xlo, the accumulated correction, is always FP32.
// rhat = r, p = v = xlo = 0; scalars reset from |r|^2
cudaError_t lo_init(wc_lattice lat, SolverState &S, wc_field r, wc_field rhat, wc_field p, wc_field v,
                    wc_field xlo);
cudaError_t lo_p(wc_lattice lat, SolverState &S, wc_field r, wc_field v, wc_field p);
cudaError_t lo_alpha(wc_lattice lat, SolverState &S, wc_field rhat, wc_field v);
cudaError_t lo_s(wc_lattice lat, SolverState &S, wc_field r, wc_field v, wc_field s);
cudaError_t lo_omega(wc_lattice lat, SolverState &S, wc_field t, wc_field s);
// xlo += alpha phat + omega shat; r = s - omega t; rho, beta, rr updated
cudaError_t lo_xr(wc_lattice lat, SolverState &S, wc_field xlo, wc_field phat, wc_field shat, wc_field s,
                  wc_field t, wc_field r, wc_field rhat);
// r_hp = b - r_hp (r_hp holds op x), rr = |r_hp|^2, r = r_hp in the Krylov
// storage, rho = <rhat, r> and beta recomputed: one pass (FP64 b and r_hp)
cudaError_t refresh_tail(wc_lattice lat, SolverState &S, const wc_field b, wc_field r_hp, wc_field r, wc_field rhat);
// x (FP64) += xlo (FP32); xlo = 0
cudaError_t hp_add_lo(wc_lattice lat, SolverState &S, double2 *x, wc_field xlo);

// One member of a lockstep group: its vectors (values; per-site scales for
// FP16 storage, else null), accumulated correction, reduction scratch and
// scalars.
struct LoMember {
    void *r, *rhat, *p, *v, *s, *t, *phat, *shat;
    float *rn, *rhatn, *pn, *vn, *sn, *tn, *phatn, *shatn;
    float4 *xlo;
    ReduceScratch rs;
    SolverScalars *sc;
};
enum LoStep { LO_STEP_P, LO_STEP_ALPHA, LO_STEP_S, LO_STEP_OMEGA, LO_STEP_XR };
// Fill a LoMember from a member's state and vectors (host side).
LoMember lo_member(SolverState &S, wc_field r, wc_field rhat, wc_field p, wc_field v, wc_field s, wc_field t,
                   wc_field phat, wc_field shat, wc_field xlo);
// One step kernel (lo_p, lo_alpha, lo_s, lo_omega or lo_xr) for the m
// members of a lockstep group in one launch, blockIdx.y = member; members:
// device array of m entries, all on lat with one storage precision (half:
// FP16).  Each member reduces into its own scratch and updates its own
// scalars; a member whose skip word is set does nothing.
cudaError_t lo_group(LoStep step, wc_lattice lat, int m, const LoMember *members, bool half, int max_blocks,
                     cudaStream_t stream);
// alpha (step LO_STEP_ALPHA) or omega (LO_STEP_OMEGA) of the m members from
// the partial sums part[member][nblk][4] that the even multi-RHS Schur pass
// wrote (FP32 vectors), one CTA per member
cudaError_t lo_group_finalize(LoStep step, int m, int nblk, const double *part, const LoMember *members,
                              cudaStream_t stream);

}  // namespace wc
