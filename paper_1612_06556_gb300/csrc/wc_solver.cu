// BiCGStab drivers and the BLAS / RAS / solve entry points of the C ABI.
//
// The outer solver is a right-preconditioned flexible BiCGStab in FP64 (the
// paper's Sec. 2 replaces CCS-QCD's double-precision BiCGStab by a flexible
// one whose preconditioner is a lower-precision solve):
//
//   r = b - M x, rhat = r, rho0 = alpha = omega = 1, v = p = 0
//   repeat:  rho = <rhat, r>, beta = (rho / rho0)(alpha / omega)
//            p = r + beta (p - omega v), phat = K^-1 p, v = M phat
//            alpha = rho / <rhat, v>, s = r - alpha v, shat = K^-1 s, t = M shat
//            omega = <t, s> / <t, t>, x += alpha phat + omega shat, r = s - omega t
//   until |r| <= tol |b|; then r = b - M x is recomputed in FP64 and the
//   solve restarts from x (rhat = r) if the true residual misses tol.
//
// K = 1 gives the plain FP64 BiCGStab.  With RAS, K^-1 u = |u| RAS(u / |u|)
// is evaluated in FP32 arithmetic on FP32 or FP16 fields: a defect
// correction in which the low-precision preconditioner only ever sees a
// unit-norm vector, while residuals, inner products and the solution update
// stay FP64 on the GPU.  Every scalar (rho, alpha, omega, beta, norms) is
// computed on the device by the last block of the fused reduction kernels;
// the host reads one small struct per iteration to test convergence.
//
// The other drivers here: the reliable-update solver (the same recurrence
// in FP32 with FP64 refreshes of x and r), the nested three-level solver
// (the flexible one with an FP32 BiCGStab as K), and the even-odd wrapper
// that runs any of them on the Schur complement of a half lattice.
#include <math.h>
#include <stdlib.h>

#include <chrono>
#include <new>

#include "wc_internal.cuh"
#include "wc_solver_kernels.cuh"
#include "wc_solver.cuh"

namespace wc {

size_t ras_smem_bytes(const wc_ras_params &p);
bool ras_fits(const wc_ras_params &p);

wc_status check_ras_params(wc_lattice lat, const wc_ras_params *p)
{
    if (!p) return set_error(lat, WC_ERR_ARG, "RAS parameters are NULL");
    if (p->overlap < 0 || p->mr_iters < 0) return set_error(lat, WC_ERR_ARG, "RAS overlap and mr_iters must be >= 0");
    for (int m = 0; m < 4; ++m) {
        const int b = p->block[m], L = lat->g.L[m];
        if (b <= 0 || L % b != 0)
            return set_error(lat, WC_ERR_ARG, "RAS block extents must divide the lattice extents");
        if (L <= b + 2 * p->overlap)
            return set_error(lat, WC_ERR_ARG, "RAS extended block must be smaller than the lattice in every direction");
        if (b + 2 * p->overlap > 255) return set_error(lat, WC_ERR_ARG, "RAS extended block extent above 255");
    }
    if (!ras_fits(*p))
        return set_error(lat, WC_ERR_ARG, "RAS extended block too large for one CTA (shared memory / threads)");
    if (p->schur != 0 && p->schur != 1) return set_error(lat, WC_ERR_ARG, "RAS schur must be 0 or 1");
    if (p->schur && !ras_schur_fits(*p))
        return set_error(lat, WC_ERR_ARG,
                         "block-Schur RAS needs block[0] + 2 overlap even and at most 1536 extended sites");
    return WC_OK;
}

namespace {

double2 *d2(wc_field f) { return static_cast<double2 *>(f->data); }

}  // namespace

double defer_margin()
{
    const char *e = getenv("WC_EO_DEFER_MARGIN");
    if (!e || !*e) return 0.5;
    const double m = atof(e);
    return m > 0.0 && isfinite(m) ? m : 0.0;
}

wc_status read_scalars(wc_lattice lat, SolverState &S)
{
    wc_status st = check_cuda(lat,
                              cudaMemcpyAsync(S.scal_host, S.scal, sizeof(SolverScalars), cudaMemcpyDeviceToHost,
                                              S.stream),
                              "cudaMemcpyAsync(scalars)");
    if (st == WC_OK) st = check_cuda(lat, cudaStreamSynchronize(S.stream), "sync(scalars)");
    return st;
}

static wc_status eo_ras_temps(wc_lattice lat, SolverState &S, wc_prec prec);

wc_status solver_vectors(wc_lattice lat, SolverState &S, const wc_solve_params &p, SolverVecs *w)
{
    wc_status st = WC_OK;
    w->r = state_work(lat, S, 0, WC_F64, &st);
    if (st == WC_OK) w->rhat = state_work(lat, S, 1, WC_F64, &st);
    if (st == WC_OK) w->p = state_work(lat, S, 2, WC_F64, &st);
    if (st == WC_OK) w->v = state_work(lat, S, 3, WC_F64, &st);
    if (st == WC_OK) w->s = state_work(lat, S, 4, WC_F64, &st);
    if (st == WC_OK) w->t = state_work(lat, S, 5, WC_F64, &st);
    w->phat = w->p;
    w->shat = w->s;
    w->lo_in = w->lo_out = nullptr;
    if (st == WC_OK && lat->schur_parent) state_work(lat, S, kSchurSlot + WC_F64, WC_F64, &st);
    if (st == WC_OK && (p.precond == WC_PRECOND_RAS || p.solver == WC_SOLVER_NESTED)) {
        w->phat = state_work(lat, S, 6, WC_F64, &st);
        if (st == WC_OK) w->shat = state_work(lat, S, 7, WC_F64, &st);
    }
    if (st == WC_OK && p.precond == WC_PRECOND_RAS && p.solver != WC_SOLVER_NESTED) {
        st = eo_ras_temps(lat, S, p.inner_prec);
        const int lo = p.inner_prec == WC_F16 ? 22 : 10;
        if (st == WC_OK) w->lo_in = state_work(lat, S, lo, p.inner_prec, &st);
        if (st == WC_OK) w->lo_out = state_work(lat, S, lo + 1, p.inner_prec, &st);
    }
    return st;
}

// The full-lattice fields the RAS of an even-odd solve works in (on the
// parent lattice, precision prec), created with the solver's vectors so
// that nothing is allocated while a batch is being captured.
static wc_status eo_ras_temps(wc_lattice lat, SolverState &S, wc_prec prec)
{
    if (!lat->schur_parent) return WC_OK;
    const int base = kRasEoSlot + 2 * (prec == WC_F16);
    wc_status st = WC_OK;
    for (int i = 0; i < 2 && st == WC_OK; ++i)
        if (!S.work[base + i]) st = wc_field_create(lat->schur_parent, prec, &S.work[base + i]);
    return st;
}

// RAS for the operator of lat.  On a half lattice (even-odd) it is the full
// lattice's RAS applied to the even vector extended by zeros on the odd
// sites and restricted back to the even sites: M^^-1 is exactly the
// even-even block of M^-1, and RAS approximates M^-1.
static wc_status ras_apply(wc_lattice lat, SolverState &S, wc_field out, wc_field in, const wc_ras_params &ras,
                           int kind)
{
    if (!lat->schur_parent) return check_cuda(lat, launch_ras(lat, out, in, ras, kind, S.stream), "ras");
    wc_lattice full = lat->schur_parent;
    if (ras.schur) return check_cuda(lat, launch_ras_schur(full, out, in, ras, kind, S.stream), "ras_schur");
    const int base = kRasEoSlot + 2 * (in->prec == WC_F16);
    wc_field a = S.work[base], b = S.work[base + 1];
    if (!a || !b) return set_error(lat, WC_ERR_STATE, "even-odd RAS fields missing");
    wc_status st = check_cuda(lat, launch_merge(full, in, nullptr, a, S.stream), "embed");
    if (st == WC_OK) st = check_cuda(lat, launch_ras(full, b, a, ras, kind, S.stream), "ras");
    if (st == WC_OK) st = check_cuda(lat, launch_split(full, b, out, nullptr, S.stream), "restrict");
    return st;
}

// uhat = K^-1 u = |u| RAS(u / |u|); norm2_dev: |u|^2 on the device
static wc_status nested_inner(wc_lattice lat, SolverState &S, const wc_solve_params &p, int kind, wc_field u,
                              wc_field uhat, const double *norm2_dev);

static wc_status apply_precond(wc_lattice lat, SolverState &S, const wc_solve_params &p, int kind,
                               const SolverVecs &w, wc_field u, wc_field uhat, const double *norm2_dev)
{
    if (p.solver == WC_SOLVER_NESTED) return nested_inner(lat, S, p, kind, u, uhat, norm2_dev);
    if (p.precond == WC_PRECOND_NONE) return WC_OK;   // uhat aliases u
    wc_status st = check_cuda(lat, launch_copy(lat, w.lo_in, u, 1.0, norm2_dev, 1, S.stream), "defect cast down");
    if (st == WC_OK) st = ras_apply(lat, S, w.lo_out, w.lo_in, p.ras, kind);
    if (st == WC_OK)
        st = check_cuda(lat, launch_copy(lat, uhat, w.lo_out, 1.0, norm2_dev, 0, S.stream), "defect cast up");
    return st;
}

wc_status enqueue_init(wc_lattice lat, SolverState &S, int kind, wc_field x, wc_field b, const SolverVecs &w,
                       bool x_zero)
{
    wc_status st = x_zero ? check_cuda(lat, cudaMemsetAsync(w.r->data, 0, spinor_bytes(WC_F64, lat->g.V), S.stream),
                                       "memset")
                          : check_cuda(lat, launch_apply(lat, w.r, x, kind, S), "apply");
    if (st == WC_OK)
        st = check_cuda(lat, bicg_init(lat, S, d2(b), d2(w.r), d2(w.rhat), d2(w.p), d2(w.v)), "bicg_init");
    return st;
}

wc_status enqueue_iteration(wc_lattice lat, SolverState &S, const wc_solve_params &p, int kind, wc_field x,
                            const SolverVecs &w)
{
    wc_status st = check_cuda(lat, bicg_p(lat, S, d2(w.r), d2(w.v), d2(w.p)), "bicg_p");
    if (st == WC_OK) st = apply_precond(lat, S, p, kind, w, w.p, w.phat, &S.scal->pp);
    if (st == WC_OK) st = check_cuda(lat, launch_apply(lat, w.v, w.phat, kind, S), "apply");
    if (st == WC_OK) st = check_cuda(lat, bicg_alpha(lat, S, d2(w.rhat), d2(w.v)), "bicg_alpha");
    if (st == WC_OK) st = check_cuda(lat, bicg_s(lat, S, d2(w.r), d2(w.v), d2(w.s)), "bicg_s");
    if (st == WC_OK) st = apply_precond(lat, S, p, kind, w, w.s, w.shat, &S.scal->ss);
    if (st == WC_OK) st = check_cuda(lat, launch_apply(lat, w.t, w.shat, kind, S), "apply");
    if (st == WC_OK) st = check_cuda(lat, bicg_omega(lat, S, d2(w.t), d2(w.s)), "bicg_omega");
    if (st == WC_OK)
        st = check_cuda(lat, bicg_xr(lat, S, d2(x), d2(w.phat), d2(w.shat), d2(w.s), d2(w.t), d2(w.r), d2(w.rhat)),
                        "bicg_xr");
    return st;
}

wc_status enqueue_true_residual(wc_lattice lat, SolverState &S, int kind, wc_field x, wc_field b,
                                const SolverVecs &w)
{
    wc_status st = check_cuda(lat, launch_apply(lat, w.r, x, kind, S), "apply");
    if (st == WC_OK) st = check_cuda(lat, residual(lat, S, d2(b), d2(w.r)), "residual");
    return st;
}

static wc_status bicgstab_impl(wc_lattice lat, SolverState &S, int kind, wc_field x, wc_field b,
                               const wc_solve_params &p, double bb, wc_solve_info *info, int iters_done);

// End of an even-odd solve on the lattice's stream: x_o = A_oo^-1 (b_o +
// k H_oe x_e) together with the odd-site residual r_o = b_o - (A_oo x_o -
// k H_oe x_e) of the stored x_o (one pass), the even-site (M x)_e = A_ee x_e
// - k H_eo x_o, x = (x_e, x_o), and *rr = |b_e - (M x)_e|^2 + |r_o|^2, the
// squared true residual of the full system (M^+ for kind 1), in the FP64
// operator arithmetic of the lattice.  Scratch: slots kEoResSlot, +1 of the
// half lattice's own state; one synchronisation.
wc_status eo_reconstruct_residual(wc_lattice lat, int kind, wc_field be, wc_field bo, wc_field xe, wc_field xo,
                                  wc_field x, double *rr)
{
    wc_lattice h = nullptr;
    wc_status st = half_lattice(lat, &h);
    if (st != WC_OK) return st;
    SolverState &R = h->st;
    R.stream = lat->stream;
    cudaStream_t s = lat->stream;
    wc_field re = state_work(h, R, kEoResSlot, WC_F64, &st);
    wc_field ro = st == WC_OK ? state_work(h, R, kEoResSlot + 1, WC_F64, &st) : nullptr;
    if (st != WC_OK) return st;
    const double k = lat->kappa;
    st = check_cuda(lat, launch_eo(lat, 1, 5, kind, xe, bo, xo, k, s, ro), "x_o and r_o");
    if (st == WC_OK) st = check_cuda(lat, launch_eo(lat, 0, 1, kind, xo, xe, re, -k, s), "(M x)_e");
    if (st == WC_OK) st = check_cuda(lat, launch_merge(lat, xe, xo, x, s), "merge");
    if (st == WC_OK) st = check_cuda(lat, residual(h, R, d2(be), d2(re)), "residual");
    if (st == WC_OK) st = check_cuda(lat, norm2_to_result(h, R, d2(ro)), "norm2");
    if (st == WC_OK)
        st = check_cuda(lat, cudaMemcpyAsync(R.red.host_result, R.red.result, sizeof(double), cudaMemcpyDeviceToHost, s),
                        "copy");
    if (st == WC_OK) st = read_scalars(h, R);
    if (st == WC_OK) *rr = R.scal_host->rr + R.red.host_result[0];
    return st;
}

// x == 0 (one reduction and a synchronisation): the residual of a zero
// start vector is b and needs no FP64 operator application
static wc_status x_is_zero(wc_lattice lat, SolverState &S, wc_field x, bool *zero)
{
    wc_status st = check_cuda(lat, norm2_to_result(lat, S, static_cast<const double2 *>(x->data)), "norm2");
    if (st == WC_OK)
        st = check_cuda(lat, cudaMemcpyAsync(S.red.host_result, S.red.result, sizeof(double), cudaMemcpyDeviceToHost,
                                             S.stream), "copy");
    if (st == WC_OK) st = check_cuda(lat, cudaStreamSynchronize(S.stream), "sync");
    if (st == WC_OK) *zero = S.red.host_result[0] == 0.0;
    return st;
}
wc_status reliable_bicgstab(wc_lattice lat, SolverState &S, int kind, wc_field x, wc_field b,
                            const wc_solve_params &p, wc_solve_info *info, int iters_done, double bb,
                            double defer_rr, bool *unconfirmed);

// Solve op x = b (op = M for kind 0, M^+ for kind 1); x, b FP64 fields.
// S: solver state (scratch); S.stream: the stream everything is queued on.
wc_status bicgstab(wc_lattice lat, SolverState &S, int kind, wc_field x, wc_field b, const wc_solve_params &p,
                   wc_solve_info *info, int iters_done, double bb, double defer_rr, bool *unconfirmed)
{
    wc_solve_info local{};
    wc_solve_info *out = info ? info : &local;
    *out = wc_solve_info{};
    out->status = WC_ERR_CUDA;
    if (unconfirmed) *unconfirmed = false;
    const wc_status st = p.solver == WC_SOLVER_RELIABLE
                             ? reliable_bicgstab(lat, S, kind, x, b, p, out, iters_done, bb, defer_rr, unconfirmed)
                             : bicgstab_impl(lat, S, kind, x, b, p, bb, out, iters_done);
    if (st != WC_OK && (out->status == WC_OK || out->status == WC_ERR_CUDA)) out->status = st;
    return st;
}

static wc_status eo_bicgstab(wc_lattice lat, int kind, wc_field x, wc_field b, const wc_solve_params &p,
                             wc_solve_info *info);

wc_status bicgstab(wc_lattice lat, int kind, wc_field x, wc_field b, const wc_solve_params &p, wc_solve_info *info)
{
    lat->st.stream = lat->stream;
    if (p.even_odd) return eo_bicgstab(lat, kind, x, b, p, info);
    return bicgstab(lat, lat->st, kind, x, b, p, info, 0, -1.0);
}

// Even-odd solve of op x = b (op = M, or M^+ for kind 1):
//   t = A_oo^-1 b_o, b^_e = b_e + k H_eo t, solve M^ x_e = b^_e on the half
//   lattice (tolerance scaled so that |b - M x| <= tol |b|: the full
//   residual equals the Schur residual on the even sites and vanishes on
//   the odd ones), x_o = A_oo^-1 (b_o + k H_oe x_e); the true FP64 residual
//   of the full system is recomputed at the end.
// The reliable-update solver's last FP64 refresh of the Schur residual
// would compute, up to rounding, the same number as that final full
// residual, so the half solve ends without it once its low-precision
// recurrence residual is below half the tolerance (defer_margin): the
// full residual then confirms convergence.  Where it does not (the
// recurrence had drifted), the half solve resumes from x_e with its own
// FP64 confirmation and the full residual is taken again.
static wc_status eo_bicgstab(wc_lattice lat, int kind, wc_field x, wc_field b, const wc_solve_params &p,
                             wc_solve_info *info)
{
    auto t0 = std::chrono::steady_clock::now();
    wc_solve_info local{};
    wc_solve_info &inf = info ? *info : local;
    inf = wc_solve_info{};
    inf.status = WC_ERR_CUDA;
    wc_lattice h = nullptr;
    wc_status st = half_lattice(lat, &h);
    if (st != WC_OK) return inf.status = st;
    cudaStream_t s = lat->stream;
    h->st.stream = s;
    wc_field f[5] = {};   // be, bo, xe, xo, bh: kept in the half lattice's state between solves
    for (int i = 0; i < 5 && st == WC_OK; ++i) f[i] = state_work(h, h->st, kEoSlot + i, WC_F64, &st);
    wc_field be = f[0], bo = f[1], xe = f[2], xo = f[3], bh = f[4], t = h->schur_tmp[WC_F64];
    const double k = lat->kappa;
    if (st == WC_OK) st = check_cuda(lat, launch_split(lat, b, be, bo, s), "split");
    if (st == WC_OK) st = check_cuda(lat, launch_split(lat, x, xe, xo, s), "split");
    if (st == WC_OK) st = check_cuda(lat, launch_eo(lat, 1, 4, kind, nullptr, bo, t, 0.0, s), "A_oo^-1 b_o");
    if (st == WC_OK) st = check_cuda(lat, launch_eo(lat, 0, 2, kind, t, be, bh, k, s), "b^_e");
    double bb = 0.0, bbh = 0.0;
    if (st == WC_OK) st = reduce_norm2(lat, b, &bb);
    if (st == WC_OK) st = reduce_norm2(h, bh, &bbh);
    wc_solve_params q = p;
    q.even_odd = 0;
    if (bbh > 0.0 && bb > 0.0) q.tol = p.tol * sqrt(bb / bbh);
    const double m = defer_margin();
    const double defer_rr = p.solver == WC_SOLVER_RELIABLE ? m * m * q.tol * q.tol * bbh : 0.0;
    bool unconfirmed = false;
    if (st == WC_OK) {
        const wc_status sr = bicgstab(h, h->st, kind, xe, bh, q, &inf, 0, bbh, defer_rr, &unconfirmed);
        if (sr != WC_OK && sr != WC_ERR_NOT_CONVERGED && sr != WC_ERR_BREAKDOWN) st = sr;
    }
    int iters = inf.iters, restarts = inf.restarts;
    wc_status half_status = inf.status;
    bool ok = false;
    double rr = 0.0;
    for (int pass = 0; pass < 2 && st == WC_OK; ++pass) {
        if (pass == 1) {   // the deferred confirmation failed: resume from x_e
            const wc_status sr = bicgstab(h, h->st, kind, xe, bh, q, &inf, iters, bbh);
            if (sr != WC_OK && sr != WC_ERR_NOT_CONVERGED && sr != WC_ERR_BREAKDOWN) st = sr;
            iters = inf.iters;
            restarts += 1 + inf.restarts;
            half_status = inf.status;
            if (st != WC_OK) break;
        }
        st = eo_reconstruct_residual(lat, kind, be, bo, xe, xo, x, &rr);
        if (st != WC_OK) break;
        ok = bb == 0.0 || rr <= p.tol * p.tol * bb;
        if (ok || !unconfirmed) break;
    }
    if (st != WC_OK) return inf.status = st;
    inf = wc_solve_info{};
    inf.iters = iters;
    inf.restarts = restarts;
    inf.true_rel_resid = bb > 0.0 ? sqrt(rr / bb) : 0.0;
    inf.status = ok ? WC_OK : (half_status != WC_OK ? half_status : WC_ERR_NOT_CONVERGED);
    if (!ok) set_error(lat, inf.status, "even-odd solve: true residual above tol");
    inf.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return inf.status;
}

static wc_status bicgstab_impl(wc_lattice lat, SolverState &S, int kind, wc_field x, wc_field b,
                               const wc_solve_params &p, double bb, wc_solve_info *info, int iters_done)
{
    auto t0 = std::chrono::steady_clock::now();
    wc_solve_info &inf = *info;
    inf.iters = iters_done;
    inf.status = WC_ERR_NOT_CONVERGED;
    SolverVecs w;
    wc_status st = solver_vectors(lat, S, p, &w);
    if (st != WC_OK) return st;
    if (bb < 0.0) {
        st = check_cuda(lat, norm2_to_result(lat, S, d2(b)), "norm2");
        if (st == WC_OK)
            st = check_cuda(lat,
                            cudaMemcpyAsync(S.red.host_result, S.red.result, sizeof(double), cudaMemcpyDeviceToHost,
                                            S.stream),
                            "cudaMemcpyAsync(norm)");
        if (st == WC_OK) st = check_cuda(lat, cudaStreamSynchronize(S.stream), "sync(norm)");
        if (st != WC_OK) return st;
        bb = S.red.host_result[0];
    }
    if (!isfinite(bb)) {
        inf.status = WC_ERR_NAN;
        return set_error(lat, WC_ERR_NAN, "source has non-finite entries");
    }
    if (bb == 0.0) {
        st = check_cuda(lat, cudaMemsetAsync(x->data, 0, spinor_bytes(WC_F64, lat->g.V), S.stream), "memset");
        if (st == WC_OK) st = check_cuda(lat, cudaStreamSynchronize(S.stream), "sync");
        inf.status = st;
        inf.true_rel_resid = 0.0;
        return st;
    }
    const double tol2 = p.tol * p.tol * bb;
    wc_status result = WC_ERR_NOT_CONVERGED;
    bool x_zero = false;
    if (iters_done == 0) st = x_is_zero(lat, S, x, &x_zero);
    if (st != WC_OK) return st;

    for (int restart = 0; restart <= p.max_restarts; ++restart) {
        inf.restarts = restart;
        st = enqueue_init(lat, S, kind, x, b, w, restart == 0 && x_zero);
        if (st == WC_OK) st = read_scalars(lat, S);
        if (st != WC_OK) return st;
        if (S.scal_host->flags & FLAG_NAN) {
            result = set_error(lat, WC_ERR_NAN, "non-finite residual");
            break;
        }
        inf.true_rel_resid = sqrt(S.scal_host->rr / bb);
        if (S.scal_host->rr <= tol2) {
            result = WC_OK;
            break;
        }
        bool breakdown = false;
        while (inf.iters < p.max_iter) {
            st = enqueue_iteration(lat, S, p, kind, x, w);
            if (st == WC_OK) st = read_scalars(lat, S);
            if (st != WC_OK) return st;
            ++inf.iters;
            const SolverScalars &h = *S.scal_host;
            if (h.flags & FLAG_NAN) {
                result = set_error(lat, WC_ERR_NAN, "non-finite value in BiCGStab");
                break;
            }
            if (h.rr <= tol2) break;
            if (h.flags & FLAG_BREAKDOWN) {
                breakdown = true;
                break;
            }
        }
        if (result == WC_ERR_NAN) break;
        st = enqueue_true_residual(lat, S, kind, x, b, w);
        if (st == WC_OK) st = read_scalars(lat, S);
        if (st != WC_OK) return st;
        inf.true_rel_resid = sqrt(S.scal_host->rr / bb);
        if (!isfinite(inf.true_rel_resid)) {
            result = set_error(lat, WC_ERR_NAN, "non-finite true residual");
            break;
        }
        if (S.scal_host->rr <= tol2) {
            result = WC_OK;
            break;
        }
        if (inf.iters >= p.max_iter) {
            result = set_error(lat, WC_ERR_NOT_CONVERGED, "max_iter reached");
            break;
        }
        result = set_error(lat, breakdown ? WC_ERR_BREAKDOWN : WC_ERR_NOT_CONVERGED,
                           breakdown ? "BiCGStab breakdown" : "true residual above tol after all restarts");
    }
    inf.status = result;
    inf.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return result;
}

// ------------------------------------------------------------------------
// Reliable-update solve: BiCGStab in FP32 with FP64 refreshes
// ------------------------------------------------------------------------

namespace {


}  // namespace

wc_status lo_vectors(wc_lattice lat, SolverState &S, const wc_solve_params &p, LoVecs *w)
{
    wc_status st = WC_OK;
    // the eight BiCGStab vectors in FP32 (slots 12-19) or FP16 (36-43); the
    // correction xlo is always FP32 (slot 20)
    const bool half = p.krylov_prec == WC_F16;
    wc_field *slots[8] = {&w->r, &w->rhat, &w->p, &w->v, &w->s, &w->t, &w->phat, &w->shat};
    for (int i = 0; i < 8 && st == WC_OK; ++i)
        *slots[i] = half ? state_work(lat, S, kHalfKrylovSlot + i, WC_F16, &st) : state_work(lat, S, 12 + i, WC_F32, &st);
    if (st == WC_OK) w->xlo = state_work(lat, S, 20, WC_F32, &st);
    if (p.precond == WC_PRECOND_NONE) {   // no preconditioner: phat, shat are p, s
        w->phat = w->p;
        w->shat = w->s;
    }
    w->lo_in = w->lo_out = nullptr;
    const wc_prec kp = half ? WC_F16 : WC_F32;
    if (st == WC_OK && lat->schur_parent) state_work(lat, S, kSchurSlot + kp, kp, &st);
    if (st == WC_OK && lat->schur_parent) state_work(lat, S, kSchurSlot + WC_F64, WC_F64, &st);
    // RAS on FP16 storage when either the vectors or inner_prec are FP16
    const bool ras16 = half || p.inner_prec == WC_F16;
    if (st == WC_OK && p.precond == WC_PRECOND_RAS) st = eo_ras_temps(lat, S, ras16 ? WC_F16 : WC_F32);
    if (st == WC_OK && p.precond == WC_PRECOND_RAS && ras16 && !half) {
        w->lo_in = state_work(lat, S, 22, WC_F16, &st);
        if (st == WC_OK) w->lo_out = state_work(lat, S, 23, WC_F16, &st);
    }
    return st;
}

namespace {

// uhat = RAS(u) for FP32 u (through FP16 storage when inner_prec is FP16);
// nothing without a preconditioner (uhat aliases u)
wc_status lo_precond(wc_lattice lat, SolverState &S, const wc_solve_params &p, int kind, const LoVecs &w,
                     wc_field u, wc_field uhat)
{
    if (p.precond == WC_PRECOND_NONE) return WC_OK;
    if (u->prec == WC_F16 || p.inner_prec != WC_F16) return ras_apply(lat, S, uhat, u, p.ras, kind);
    wc_status st = check_cuda(lat, launch_copy(lat, w.lo_in, u, 1.0, nullptr, 0, S.stream), "cast to FP16");
    if (st == WC_OK) st = ras_apply(lat, S, w.lo_out, w.lo_in, p.ras, kind);
    if (st == WC_OK) st = check_cuda(lat, launch_copy(lat, uhat, w.lo_out, 1.0, nullptr, 0, S.stream), "cast");
    return st;
}

}  // namespace

wc_status enqueue_lo_iteration(wc_lattice lat, SolverState &S, const wc_solve_params &p, int kind,
                               const LoVecs &w)
{
    wc_status st = check_cuda(lat, lo_p(lat, S, w.r, w.v, w.p), "lo_p");
    if (st == WC_OK) st = lo_precond(lat, S, p, kind, w, w.p, w.phat);
    if (st == WC_OK) st = check_cuda(lat, launch_apply(lat, w.v, w.phat, kind, S), "apply");
    if (st == WC_OK) st = check_cuda(lat, lo_alpha(lat, S, w.rhat, w.v), "lo_alpha");
    if (st == WC_OK) st = check_cuda(lat, lo_s(lat, S, w.r, w.v, w.s), "lo_s");
    if (st == WC_OK) st = lo_precond(lat, S, p, kind, w, w.s, w.shat);
    if (st == WC_OK) st = check_cuda(lat, launch_apply(lat, w.t, w.shat, kind, S), "apply");
    if (st == WC_OK) st = check_cuda(lat, lo_omega(lat, S, w.t, w.s), "lo_omega");
    if (st == WC_OK)
        st = check_cuda(lat, lo_xr(lat, S, w.xlo, w.phat, w.shat, w.s, w.t, w.r, w.rhat),
                        "lo_xr");
    return st;
}

wc_status enqueue_refresh_full(wc_lattice lat, SolverState &S, int kind, wc_field x, wc_field b, wc_field r_hp,
                               const LoVecs &w);

wc_status enqueue_lo_start(wc_lattice lat, SolverState &S, int kind, wc_field x, wc_field b, wc_field r_hp,
                           const LoVecs &w, bool x_zero)
{
    wc_status st = x_zero ? check_cuda(lat, cudaMemsetAsync(r_hp->data, 0, spinor_bytes(WC_F64, lat->g.V), S.stream),
                                       "memset")
                          : check_cuda(lat, launch_apply(lat, r_hp, x, kind, S), "apply");
    if (st == WC_OK)
        st = check_cuda(lat, residual(lat, S, static_cast<const double2 *>(b->data),
                                      static_cast<double2 *>(r_hp->data)), "residual");
    if (st == WC_OK) st = check_cuda(lat, launch_copy(lat, w.r, r_hp, 1.0, nullptr, 0, S.stream), "cast residual");
    if (st == WC_OK)
        st = check_cuda(lat, lo_init(lat, S, w.r, w.rhat, w.p, w.v, w.xlo), "lo_init");
    return st;
}

// x += xlo; r_hp = b - op x (FP64); S.scal->rr = |r_hp|^2
static wc_status enqueue_refresh(wc_lattice lat, SolverState &S, int kind, wc_field x, wc_field b, wc_field r_hp,
                                 const LoVecs &w)
{
    wc_status st = check_cuda(lat, hp_add_lo(lat, S, static_cast<double2 *>(x->data), w.xlo), "hp_add_lo");
    if (st == WC_OK) st = check_cuda(lat, launch_apply(lat, r_hp, x, kind, S), "apply");
    if (st == WC_OK)
        st = check_cuda(lat, residual(lat, S, static_cast<const double2 *>(b->data), static_cast<double2 *>(r_hp->data)),
                        "residual");
    return st;
}

wc_status enqueue_refresh_full(wc_lattice lat, SolverState &S, int kind, wc_field x, wc_field b, wc_field r_hp,
                               const LoVecs &w)
{
    wc_status st = check_cuda(lat, hp_add_lo(lat, S, static_cast<double2 *>(x->data), w.xlo), "hp_add_lo");
    if (st == WC_OK) st = check_cuda(lat, launch_apply(lat, r_hp, x, kind, S), "apply");
    if (st == WC_OK) st = check_cuda(lat, refresh_tail(lat, S, b, r_hp, w.r, w.rhat), "refresh");
    return st;
}

// Inner level of the nested solver: uhat = |u| z with z an approximate
// solution of op z = u / |u| by FP32 BiCGStab (right-preconditioned by RAS
// unless precond is NONE),
// from z = 0, stopped at |r| <= inner_tol or after inner_iters steps.  Uses
// its own solver state so that the outer scalars are untouched.
static wc_status nested_inner(wc_lattice lat, SolverState &S, const wc_solve_params &p, int kind, wc_field u,
                              wc_field uhat, const double *norm2_dev)
{
    wc_status st = WC_OK;
    if (!S.inner) {
        S.inner = new (std::nothrow) SolverState();
        if (!S.inner) return set_error(lat, WC_ERR_ARG, "out of host memory");
        st = state_init(lat, *S.inner);
        if (st != WC_OK) {
            delete S.inner;
            S.inner = nullptr;
            return st;
        }
    }
    SolverState &I = *S.inner;
    I.stream = S.stream;
    LoVecs w;
    st = lo_vectors(lat, I, p, &w);
    if (st != WC_OK) return st;
    const double itol = (p.inner_tol > 0.0 && p.inner_tol < 1.0) ? p.inner_tol : 0.01;
    const int iters = p.inner_iters > 0 ? p.inner_iters : 100;
    st = check_cuda(lat, launch_copy(lat, w.r, u, 1.0, norm2_dev, 1, I.stream), "cast to unit norm");
    if (st == WC_OK)
        st = check_cuda(lat, lo_init(lat, I, w.r, w.rhat, w.p, w.v, w.xlo), "lo_init");
    if (st == WC_OK) st = read_scalars(lat, I);
    if (st != WC_OK) return st;
    const double rr0 = I.scal_host->rr;
    for (int it = 0; it < iters && rr0 > 0.0; ++it) {
        st = enqueue_lo_iteration(lat, I, p, kind, w);
        if (st == WC_OK) st = read_scalars(lat, I);
        if (st != WC_OK) return st;
        const SolverScalars &h = *I.scal_host;
        if (h.flags != 0 || !(h.rr > itol * itol * rr0)) break;
    }
    // a blown-up inner solve (NaN) falls back to the identity preconditioner
    if (I.scal_host->flags & FLAG_NAN)
        return check_cuda(lat, launch_copy(lat, uhat, u, 1.0, nullptr, 0, I.stream), "copy");
    return check_cuda(lat, launch_copy(lat, uhat, w.xlo, 1.0, norm2_dev, 0, I.stream), "cast back");
}

wc_status reliable_bicgstab(wc_lattice lat, SolverState &S, int kind, wc_field x, wc_field b,
                            const wc_solve_params &p, wc_solve_info *info, int iters_done, double bb,
                            double defer_rr, bool *unconfirmed)
{
    auto t0 = std::chrono::steady_clock::now();
    wc_solve_info &inf = *info;
    inf = wc_solve_info{};
    inf.iters = iters_done;
    inf.status = WC_ERR_NOT_CONVERGED;
    wc_status st = WC_OK;
    wc_field r_hp = state_work(lat, S, 0, WC_F64, &st);
    LoVecs w;
    if (st == WC_OK) st = lo_vectors(lat, S, p, &w);
    if (st != WC_OK) return st;
    if (bb < 0.0) {
        st = check_cuda(lat, norm2_to_result(lat, S, static_cast<const double2 *>(b->data)), "norm2");
        if (st == WC_OK)
            st = check_cuda(lat, cudaMemcpyAsync(S.red.host_result, S.red.result, sizeof(double),
                                                 cudaMemcpyDeviceToHost, S.stream), "copy");
        if (st == WC_OK) st = check_cuda(lat, cudaStreamSynchronize(S.stream), "sync");
        if (st != WC_OK) return st;
        bb = S.red.host_result[0];
    }
    if (!isfinite(bb)) {
        inf.status = WC_ERR_NAN;
        return set_error(lat, WC_ERR_NAN, "source has non-finite entries");
    }
    if (bb == 0.0) {
        st = check_cuda(lat, cudaMemsetAsync(x->data, 0, spinor_bytes(WC_F64, lat->g.V), S.stream), "memset");
        if (st == WC_OK) st = check_cuda(lat, cudaStreamSynchronize(S.stream), "sync");
        inf.status = st;
        return st;
    }
    const double tol2 = p.tol * p.tol * bb;
    const double delta = (p.delta > 0.0 && p.delta < 1.0) ? p.delta : 0.01;
    const double d2 = delta * delta;
    wc_status result = WC_ERR_NOT_CONVERGED;
    bool x_zero = false;
    if (iters_done == 0) st = x_is_zero(lat, S, x, &x_zero);
    if (st != WC_OK) return st;
    for (int restart = 0; restart <= p.max_restarts; ++restart) {
        inf.restarts = restart;
        // true residual, FP32 copy, BiCGStab state reset (xlo = 0)
        double rr_true = bb;
        if (restart == 0 && x_zero) {
            st = check_cuda(lat, launch_copy(lat, r_hp, b, 1.0, nullptr, 0, S.stream), "copy");
        } else {
            st = check_cuda(lat, launch_apply(lat, r_hp, x, kind, S), "apply");
            if (st == WC_OK)
                st = check_cuda(lat, residual(lat, S, static_cast<const double2 *>(b->data),
                                              static_cast<double2 *>(r_hp->data)), "residual");
            if (st == WC_OK) st = read_scalars(lat, S);
            if (st == WC_OK) rr_true = S.scal_host->rr;
        }
        if (st != WC_OK) return st;
        inf.true_rel_resid = sqrt(rr_true / bb);
        if (!isfinite(rr_true)) {
            result = set_error(lat, WC_ERR_NAN, "non-finite residual");
            break;
        }
        if (rr_true <= tol2) {
            result = WC_OK;
            break;
        }
        st = check_cuda(lat, launch_copy(lat, w.r, r_hp, 1.0, nullptr, 0, S.stream), "cast residual");
        if (st == WC_OK)
            st = check_cuda(lat, lo_init(lat, S, w.r, w.rhat, w.p, w.v, w.xlo), "lo_init");
        if (st != WC_OK) return st;
        double rmax2 = rr_true, rr_refresh = rr_true, rr_prev = rr_true;
        bool breakdown = false, converged = false, diverged = false;
        while (inf.iters < p.max_iter) {
            st = enqueue_lo_iteration(lat, S, p, kind, w);
            if (st == WC_OK) st = read_scalars(lat, S);
            if (st != WC_OK) return st;
            ++inf.iters;
            const SolverScalars h = *S.scal_host;
            if ((h.flags & FLAG_NAN) || h.rr > 1e8 * rr_refresh) {
                // the FP32 recurrence blew up: drop its pending correction and
                // restart from the last FP64-verified iterate
                diverged = true;
                break;
            }
            if (h.flags & FLAG_BREAKDOWN) {
                breakdown = true;
                break;
            }
            if (h.rr > rmax2) rmax2 = h.rr;
            const double prev = rr_prev;
            rr_prev = h.rr;
            if (defer_rr > 0.0 && h.rr <= defer_rr) {
                // the caller confirms with its own true residual: fold the
                // correction only
                st = check_cuda(lat, hp_add_lo(lat, S, static_cast<double2 *>(x->data), w.xlo), "hp_add_lo");
                if (st != WC_OK) return st;
                if (unconfirmed) *unconfirmed = true;
                inf.true_rel_resid = sqrt(h.rr / bb);
                converged = true;
                break;
            }
            // deferring, a recurrence below tol but above defer_rr refreshes
            // only once it stops decreasing
            const bool at_tol = h.rr <= tol2 && (defer_rr <= 0.0 || !(h.rr < prev));
            if (h.rr <= d2 * rmax2 || at_tol) {
                // reliable update: fold the FP32 correction into the FP64
                // solution and restart the recurrence from the true residual
                // (its low-precision copy and rho in the same pass)
                st = enqueue_refresh_full(lat, S, kind, x, b, r_hp, w);
                if (st == WC_OK) st = read_scalars(lat, S);
                if (st != WC_OK) return st;
                rr_true = S.scal_host->rr;
                inf.true_rel_resid = sqrt(rr_true / bb);
                if (rr_true <= tol2) {
                    converged = true;
                    break;
                }
                rmax2 = rr_true;
                rr_refresh = rr_true;
                rr_prev = rr_true;
            }
        }
        if (converged) {
            result = WC_OK;
            break;
        }
        if (diverged) {
            st = check_cuda(lat, cudaMemsetAsync(w.xlo->data, 0, spinor_bytes(WC_F32, lat->g.V), S.stream), "memset");
            if (st != WC_OK) return st;
            if (restart == p.max_restarts) {
                result = set_error(lat, WC_ERR_NAN, "FP32 recurrence diverged after all restarts");
                break;
            }
            continue;   // restart from x (true residual recomputed at the top)
        }
        // fold whatever correction is pending and test the true residual
        st = enqueue_refresh(lat, S, kind, x, b, r_hp, w);
        if (st == WC_OK) st = read_scalars(lat, S);
        if (st != WC_OK) return st;
        rr_true = S.scal_host->rr;
        inf.true_rel_resid = sqrt(rr_true / bb);
        if (rr_true <= tol2) {
            result = WC_OK;
            break;
        }
        if (inf.iters >= p.max_iter) {
            result = set_error(lat, WC_ERR_NOT_CONVERGED, "max_iter reached");
            break;
        }
        result = set_error(lat, breakdown ? WC_ERR_BREAKDOWN : WC_ERR_NOT_CONVERGED,
                           breakdown ? "BiCGStab breakdown" : "true residual above tol after all restarts");
    }
    inf.status = result;
    inf.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return result;
}

wc_status check_solve_args(wc_lattice lat, wc_field x, wc_field b, const wc_solve_params *p)
{
    if (!lat) return set_error(nullptr, WC_ERR_ARG, "lattice is NULL");
    if (!x || !b || !p) return set_error(lat, WC_ERR_ARG, "x, b and params must not be NULL");
    if (x->lat != lat || b->lat != lat) return set_error(lat, WC_ERR_ARG, "fields belong to another lattice");
    if (x->prec != WC_F64 || b->prec != WC_F64) return set_error(lat, WC_ERR_ARG, "x and b must be FP64 fields");
    if (x == b) return set_error(lat, WC_ERR_ARG, "x and b must be distinct");
    if (!(p->tol > 0.0) || p->max_iter < 0 || p->max_restarts < 0)
        return set_error(lat, WC_ERR_ARG, "tol must be > 0, max_iter and max_restarts >= 0");
    if (p->precond != WC_PRECOND_NONE && p->precond != WC_PRECOND_RAS)
        return set_error(lat, WC_ERR_ARG, "unknown preconditioner");
    if (p->solver != WC_SOLVER_FLEXIBLE && p->solver != WC_SOLVER_RELIABLE && p->solver != WC_SOLVER_NESTED)
        return set_error(lat, WC_ERR_ARG, "unknown solver kind");
    if (p->solver == WC_SOLVER_NESTED && (!(p->inner_tol >= 0.0 && p->inner_tol < 1.0) || p->inner_iters < 0))
        return set_error(lat, WC_ERR_ARG, "inner_tol must be in [0, 1) and inner_iters >= 0");
    if (p->krylov_prec != WC_F64 && p->krylov_prec != WC_F32 && p->krylov_prec != WC_F16)
        return set_error(lat, WC_ERR_ARG, "krylov_prec must be WC_F32 or WC_F16 (WC_F64 means WC_F32)");
    if (p->solver == WC_SOLVER_RELIABLE && !(p->delta >= 0.0 && p->delta < 1.0))
        return set_error(lat, WC_ERR_ARG, "delta must be in [0, 1)");
    if (p->precond == WC_PRECOND_RAS) {
        if (p->inner_prec != WC_F32 && p->inner_prec != WC_F16)
            return set_error(lat, WC_ERR_ARG, "RAS inner precision must be WC_F32 or WC_F16");
        wc_status st = check_ras_params(lat, &p->ras);
        if (st != WC_OK) return st;
    }
    return require_operator(lat);
}

}  // namespace wc

using namespace wc;

extern "C" {

wc_status wc_dot(wc_lattice lat, wc_field a, wc_field b, double *re_im)
{
    if (!lat || !a || !b || !re_im) return set_error(lat, WC_ERR_ARG, "NULL argument");
    if (a->lat != lat || b->lat != lat) return set_error(lat, WC_ERR_ARG, "fields belong to another lattice");
    return reduce_dot(lat, a, b, re_im);
}

wc_status wc_norm2(wc_lattice lat, wc_field a, double *out)
{
    if (!lat || !a || !out) return set_error(lat, WC_ERR_ARG, "NULL argument");
    if (a->lat != lat) return set_error(lat, WC_ERR_ARG, "field belongs to another lattice");
    return reduce_norm2(lat, a, out);
}

wc_status wc_axpy_norm(wc_lattice lat, const double *a, wc_field x, wc_field y, double *norm2_y)
{
    if (!lat || !a || !x || !y) return set_error(lat, WC_ERR_ARG, "NULL argument");
    if (x->lat != lat || y->lat != lat) return set_error(lat, WC_ERR_ARG, "fields belong to another lattice");
    if (x->prec != y->prec) return set_error(lat, WC_ERR_ARG, "x and y must have the same precision");
    if (x == y) return set_error(lat, WC_ERR_ARG, "x and y must be distinct");
    return axpy_norm(lat, a, x, y, norm2_y);
}

wc_status wc_ras_precond(wc_lattice lat, wc_field out, wc_field in, const wc_ras_params *p)
{
    if (!lat || !out || !in) return set_error(lat, WC_ERR_ARG, "NULL argument");
    if (out->lat != lat || in->lat != lat) return set_error(lat, WC_ERR_ARG, "fields belong to another lattice");
    if (out == in) return set_error(lat, WC_ERR_ARG, "out and in must be distinct");
    if (out->prec != in->prec || in->prec == WC_F64)
        return set_error(lat, WC_ERR_ARG, "RAS works on FP32 or FP16 fields of one precision");
    wc_status st = check_ras_params(lat, p);
    if (st != WC_OK) return st;
    st = require_operator(lat);
    if (st != WC_OK) return st;
    return check_cuda(lat, launch_ras(lat, out, in, *p, 0, lat->stream), "ras");
}

wc_status wc_ras_schur(wc_lattice lat, wc_field out, wc_field in, const wc_ras_params *p, int dagger)
{
    if (!lat || !out || !in || !p) return set_error(lat, WC_ERR_ARG, "NULL argument");
    if (out->lat != lat || in->lat != lat) return set_error(lat, WC_ERR_ARG, "fields belong to another lattice");
    if (out == in) return set_error(lat, WC_ERR_ARG, "out and in must be distinct");
    if (out->prec != in->prec || in->prec == WC_F64)
        return set_error(lat, WC_ERR_ARG, "RAS works on FP32 or FP16 fields of one precision");
    wc_ras_params q = *p;
    q.schur = 1;
    wc_status st = check_ras_params(lat, &q);
    if (st != WC_OK) return st;
    st = require_operator(lat);
    if (st != WC_OK) return st;
    wc_lattice h = nullptr;
    st = half_lattice(lat, &h);
    if (st != WC_OK) return st;
    wc_field *tmp = lat->ras_half[in->prec];
    for (int k = 0; k < 2 && st == WC_OK; ++k)
        if (!tmp[k]) st = wc_field_create(h, in->prec, &tmp[k]);
    if (st == WC_OK) st = check_cuda(lat, launch_split(lat, in, tmp[0], nullptr, lat->stream), "split");
    if (st == WC_OK)
        st = check_cuda(lat, launch_ras_schur(lat, tmp[1], tmp[0], q, dagger ? 1 : 0, lat->stream), "ras_schur");
    if (st == WC_OK) st = check_cuda(lat, launch_merge(lat, tmp[1], nullptr, out, lat->stream), "merge");
    return st;
}

wc_status wc_solve_bicgstab(wc_lattice lat, wc_field x, wc_field b, const wc_solve_params *p, wc_solve_info *info)
{
    wc_status st = check_solve_args(lat, x, b, p);
    if (st != WC_OK) {
        if (info) {
            *info = wc_solve_info{};
            info->status = st;
        }
        return st;
    }
    return bicgstab(lat, 0, x, b, *p, info);
}

}  // extern "C"
