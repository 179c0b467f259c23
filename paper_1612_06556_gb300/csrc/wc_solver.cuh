// BiCGStab building blocks shared by the single-RHS solve, the batched
// graph-captured solve and the action/force call (wc_solver.cu).
#pragma once

#include "wc_internal.cuh"

namespace wc {

// FP64 work vectors of one solve (phat/shat alias p/s without a
// preconditioner) and the two inner-precision fields of the RAS defect
// correction.
struct SolverVecs {
    wc_field r, rhat, p, v, s, t, phat, shat, lo_in, lo_out;
};

wc_status check_ras_params(wc_lattice lat, const wc_ras_params *p);
wc_status check_solve_args(wc_lattice lat, wc_field x, wc_field b, const wc_solve_params *p);
wc_status solver_vectors(wc_lattice lat, SolverState &S, const wc_solve_params &p, SolverVecs *w);
wc_status read_scalars(wc_lattice lat, SolverState &S);

// Queue (no host synchronisation) on S.stream:
//   init: r = b - op x, rhat = r, p = v = 0, scalars reset
//   iteration: one flexible BiCGStab step, scalars updated on the device
//   true residual: r = b - op x, S.scal->rr = |r|^2
wc_status enqueue_init(wc_lattice lat, SolverState &S, int kind, wc_field x, wc_field b, const SolverVecs &w,
                       bool x_zero = false);
wc_status enqueue_iteration(wc_lattice lat, SolverState &S, const wc_solve_params &p, int kind, wc_field x,
                            const SolverVecs &w);
wc_status enqueue_true_residual(wc_lattice lat, SolverState &S, int kind, wc_field x, wc_field b,
                                const SolverVecs &w);
// An even-odd reliable half solve (single or batched) ends unconfirmed at
// |r| <= m tol: m = 0.5 unless the environment variable WC_EO_DEFER_MARGIN
// gives another (0: the half solve always confirms in FP64 itself; a large
// m makes the full-residual confirmation fail, for tests of the resume).
double defer_margin();
// end of an even-odd solve of the full lattice lat from its half fields:
// x_o reconstructed, x = (x_e, x_o), *rr = |b - op x|^2 (one synchronisation)
wc_status eo_reconstruct_residual(wc_lattice lat, int kind, wc_field be, wc_field bo, wc_field xe, wc_field xo,
                                  wc_field x, double *rr);

// Host-driven solve of op x = b (kind 0: M, 1: M^+) with state S, counting
// iters_done iterations already spent; bb = |b|^2 or < 0 to compute it.
// defer_rr > 0 (reliable-update solver only): a caller that recomputes the
// true residual itself lets the solve end, without an FP64 operator
// application, once the low-precision recurrence residual |r|^2 is at most
// defer_rr; *unconfirmed is then set (x holds the folded correction).
wc_status bicgstab(wc_lattice lat, SolverState &S, int kind, wc_field x, wc_field b, const wc_solve_params &p,
                   wc_solve_info *info, int iters_done, double bb, double defer_rr = 0.0,
                   bool *unconfirmed = nullptr);
// Same with the lattice's own state and stream.
wc_status bicgstab(wc_lattice lat, int kind, wc_field x, wc_field b, const wc_solve_params &p, wc_solve_info *info);

// FP32 vectors of the reliable-update solver (r, rhat, p, v, s, t, phat,
// shat, xlo FP32; lo_in/lo_out FP16 casts of the RAS input/output when the
// inner precision is FP16)
struct LoVecs {
    wc_field r, rhat, p, v, s, t, phat, shat, xlo, lo_in, lo_out;
};
wc_status lo_vectors(wc_lattice lat, SolverState &S, const wc_solve_params &p, LoVecs *w);
// one FP32 BiCGStab step (scalars on the device)
wc_status enqueue_lo_iteration(wc_lattice lat, SolverState &S, const wc_solve_params &p, int kind,
                               const LoVecs &w);
// reliable update: x += xlo; r_hp = b - op x (FP64, S.scal->rr = |r_hp|^2);
// r = fl32(r_hp); rho and beta recomputed
wc_status enqueue_refresh_full(wc_lattice lat, SolverState &S, int kind, wc_field x, wc_field b, wc_field r_hp,
                               const LoVecs &w);
// start of a reliable solve: r_hp = b - op x (r_hp = b when the caller
// knows x = 0); r = fl32(r_hp); rhat = r, p = v = xlo = 0, scalars reset
// (rr = |r|^2 of the FP32 copy)
wc_status enqueue_lo_start(wc_lattice lat, SolverState &S, int kind, wc_field x, wc_field b, wc_field r_hp,
                           const LoVecs &w, bool x_zero = false);

cudaError_t ras_prepare();

}  // namespace wc
