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
#include <math.h>

#include <chrono>

#include "wc_internal.cuh"
#include "wc_solver_kernels.cuh"

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
    return WC_OK;
}

namespace {

wc_field work_field(wc_lattice lat, int slot, wc_prec prec, wc_status *st)
{
    if (!lat->work[slot]) {
        *st = wc_field_create(lat, prec, &lat->work[slot]);
        if (*st != WC_OK) return nullptr;
    }
    *st = WC_OK;
    return lat->work[slot];
}

double2 *d2(wc_field f) { return static_cast<double2 *>(f->data); }

wc_status read_scalars(wc_lattice lat)
{
    wc_status st = check_cuda(lat,
                              cudaMemcpyAsync(lat->scal_host, lat->scal, sizeof(SolverScalars),
                                              cudaMemcpyDeviceToHost, lat->stream),
                              "cudaMemcpyAsync(scalars)");
    if (st == WC_OK) st = check_cuda(lat, cudaStreamSynchronize(lat->stream), "sync(scalars)");
    return st;
}

struct Precond {
    wc_precond kind = WC_PRECOND_NONE;
    wc_ras_params ras{};
    wc_field lo_in = nullptr, lo_out = nullptr;   // inner-precision fields
    int dagger = 0;
};

// uhat = K^-1 u.  norm2_dev: |u|^2 on the device (written by the update kernel).
wc_status apply_precond(wc_lattice lat, const Precond &K, wc_field u, wc_field uhat, const double *norm2_dev)
{
    if (K.kind == WC_PRECOND_NONE) return WC_OK;   // callers use u itself
    wc_status st = check_cuda(lat, launch_copy(lat, K.lo_in, u, 1.0, norm2_dev, 1), "defect cast down");
    if (st == WC_OK) st = check_cuda(lat, launch_ras(lat, K.lo_out, K.lo_in, K.ras, K.dagger), "ras");
    if (st == WC_OK) st = check_cuda(lat, launch_copy(lat, uhat, K.lo_out, 1.0, norm2_dev, 0), "defect cast up");
    return st;
}

}  // namespace

// Solve op x = b (op = M for kind 0, M^+ for kind 1); x, b FP64 fields.
static wc_status bicgstab_impl(wc_lattice lat, int kind, wc_field x, wc_field b, const wc_solve_params &p,
                               wc_solve_info *info);

wc_status bicgstab(wc_lattice lat, int kind, wc_field x, wc_field b, const wc_solve_params &p, wc_solve_info *info)
{
    wc_solve_info local{};
    local.status = WC_ERR_CUDA;
    wc_solve_info *out = info ? info : &local;
    *out = local;
    const wc_status st = bicgstab_impl(lat, kind, x, b, p, out);
    if (st != WC_OK && out->status == WC_OK) out->status = st;
    if (st != WC_OK && out->status == WC_ERR_CUDA && st != WC_ERR_CUDA) out->status = st;
    return st;
}

static wc_status bicgstab_impl(wc_lattice lat, int kind, wc_field x, wc_field b, const wc_solve_params &p,
                               wc_solve_info *info)
{
    auto t0 = std::chrono::steady_clock::now();
    wc_solve_info inf{};
    inf.status = WC_ERR_NOT_CONVERGED;
    wc_status st = WC_OK;
    wc_field r = work_field(lat, 0, WC_F64, &st);
    wc_field rhat = st == WC_OK ? work_field(lat, 1, WC_F64, &st) : nullptr;
    wc_field pv = st == WC_OK ? work_field(lat, 2, WC_F64, &st) : nullptr;
    wc_field v = st == WC_OK ? work_field(lat, 3, WC_F64, &st) : nullptr;
    wc_field s = st == WC_OK ? work_field(lat, 4, WC_F64, &st) : nullptr;
    wc_field t = st == WC_OK ? work_field(lat, 5, WC_F64, &st) : nullptr;
    Precond K;
    K.kind = p.precond;
    K.ras = p.ras;
    K.dagger = kind;
    wc_field phat = pv, shat = s;
    if (st == WC_OK && K.kind == WC_PRECOND_RAS) {
        phat = work_field(lat, 6, WC_F64, &st);
        if (st == WC_OK) shat = work_field(lat, 7, WC_F64, &st);
        const int lo = p.inner_prec == WC_F16 ? 12 : 10;
        if (st == WC_OK) K.lo_in = work_field(lat, lo, p.inner_prec, &st);
        if (st == WC_OK) K.lo_out = work_field(lat, lo + 1, p.inner_prec, &st);
    }
    if (st != WC_OK) return st;

    double bb = 0.0;
    st = reduce_norm2(lat, b, &bb);
    if (st != WC_OK) return st;
    if (!isfinite(bb)) {
        inf.status = WC_ERR_NAN;
        if (info) *info = inf;
        return set_error(lat, WC_ERR_NAN, "source has non-finite entries");
    }
    if (bb == 0.0) {
        st = check_cuda(lat, cudaMemsetAsync(x->data, 0, spinor_bytes(WC_F64, lat->g.V), lat->stream), "memset");
        inf.status = WC_OK;
        inf.true_rel_resid = 0.0;
        if (info) *info = inf;
        return st;
    }
    const double tol2 = p.tol * p.tol * bb;
    const int apply_kind = kind;   // 0: M, 1: M^+
    wc_status result = WC_ERR_NOT_CONVERGED;

    for (int restart = 0; restart <= p.max_restarts; ++restart) {
        inf.restarts = restart;
        // r = b - op x
        st = check_cuda(lat, launch_apply(lat, r, x, apply_kind), "apply");
        if (st == WC_OK) st = check_cuda(lat, bicg_init(lat, d2(b), d2(r), d2(rhat), d2(pv), d2(v)), "bicg_init");
        if (st == WC_OK) st = read_scalars(lat);
        if (st != WC_OK) return st;
        if (lat->scal_host->flags & FLAG_NAN) {
            result = set_error(lat, WC_ERR_NAN, "non-finite residual");
            break;
        }
        if (lat->scal_host->rr <= tol2) {
            result = WC_OK;
            break;
        }
        bool breakdown = false;
        while (inf.iters < p.max_iter) {
            st = check_cuda(lat, bicg_p(lat, d2(r), d2(v), d2(pv)), "bicg_p");
            if (st == WC_OK) st = apply_precond(lat, K, pv, phat, &lat->scal->pp);
            if (st == WC_OK) st = check_cuda(lat, launch_apply(lat, v, phat, apply_kind), "apply");
            if (st == WC_OK) st = check_cuda(lat, bicg_alpha(lat, d2(rhat), d2(v)), "bicg_alpha");
            if (st == WC_OK) st = check_cuda(lat, bicg_s(lat, d2(r), d2(v), d2(s)), "bicg_s");
            if (st == WC_OK) st = apply_precond(lat, K, s, shat, &lat->scal->ss);
            if (st == WC_OK) st = check_cuda(lat, launch_apply(lat, t, shat, apply_kind), "apply");
            if (st == WC_OK) st = check_cuda(lat, bicg_omega(lat, d2(t), d2(s)), "bicg_omega");
            if (st == WC_OK)
                st = check_cuda(lat, bicg_xr(lat, d2(x), d2(phat), d2(shat), d2(s), d2(t), d2(r), d2(rhat)),
                                "bicg_xr");
            if (st == WC_OK) st = read_scalars(lat);
            if (st != WC_OK) return st;
            ++inf.iters;
            const SolverScalars &h = *lat->scal_host;
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
        // true residual in FP64
        st = check_cuda(lat, launch_apply(lat, r, x, apply_kind), "apply");
        if (st == WC_OK) st = check_cuda(lat, residual(lat, d2(b), d2(r)), "residual");
        if (st == WC_OK) st = read_scalars(lat);
        if (st != WC_OK) return st;
        inf.true_rel_resid = sqrt(lat->scal_host->rr / bb);
        if (!isfinite(inf.true_rel_resid)) {
            result = set_error(lat, WC_ERR_NAN, "non-finite true residual");
            break;
        }
        if (lat->scal_host->rr <= tol2) {
            result = WC_OK;
            break;
        }
        if (inf.iters >= p.max_iter) {
            result = set_error(lat, WC_ERR_NOT_CONVERGED, "max_iter reached");
            break;
        }
        if (breakdown && restart == p.max_restarts) {
            result = set_error(lat, WC_ERR_BREAKDOWN, "BiCGStab breakdown");
            break;
        }
        result = set_error(lat, breakdown ? WC_ERR_BREAKDOWN : WC_ERR_NOT_CONVERGED,
                           breakdown ? "BiCGStab breakdown" : "true residual above tol after all restarts");
    }
    if (result == WC_OK && inf.true_rel_resid == 0.0) {
        // converged at the initial residual check: report it
        inf.true_rel_resid = sqrt(lat->scal_host->rr / bb);
    }
    inf.status = result;
    inf.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (info) *info = inf;
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
    if (p->precond == WC_PRECOND_RAS) {
        if (p->inner_prec != WC_F32 && p->inner_prec != WC_F16)
            return set_error(lat, WC_ERR_ARG, "RAS inner precision must be WC_F32 or WC_F16");
        wc_status st = check_ras_params(lat, &p->ras);
        if (st != WC_OK) return st;
    }
    if (!lat->gauge_loaded || !lat->clover_loaded) return set_error(lat, WC_ERR_STATE, "gauge/clover not loaded");
    return WC_OK;
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
    if (!lat->gauge_loaded || !lat->clover_loaded) return set_error(lat, WC_ERR_STATE, "gauge/clover not loaded");
    return check_cuda(lat, launch_ras(lat, out, in, *p, 0), "ras");
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
