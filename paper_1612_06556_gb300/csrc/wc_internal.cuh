// Host-side internals of libwc: lattice and field handles, solver state,
// error helpers and the launchers each translation unit implements.  The
// device layouts and precision traits are in wc_device.cuh.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/wc.h"
#include "wc_device.cuh"

namespace wc {

// ------------------------------------------------------------------------
// host-side helpers shared by the translation units
// ------------------------------------------------------------------------

struct Lattice;

wc_status set_error(wc_lattice lat, wc_status st, const std::string &msg);
wc_status check_cuda(wc_lattice lat, cudaError_t e, const char *what);
wc_status check_launch(wc_lattice lat, const char *what);

// Number of SMs of the current device (cached).
int sm_count();

}  // namespace wc

// ------------------------------------------------------------------------
// handle definitions
// ------------------------------------------------------------------------

namespace wc {

// Per-solve state: device scalars and their pinned host mirror, reduction
// scratch, solver work fields (created on first use: slots 0-9 FP64, 10-21
// FP32, 22-23 FP16, 24 + precision: the odd-site intermediate of the
// even-odd operator on a half lattice, 27-31: the half-lattice FP64 fields
// b_e, b_o, x_e, x_o, b^_e of an even-odd solve, 32-35: full-lattice FP32
// and FP16 in/out fields of the RAS preconditioner of an even-odd solve,
// 36-43: the low-precision BiCGStab vectors when they are FP16, 44-45: the
// even and odd halves of the final full residual of an even-odd solve) and
// the stream the solve is queued on.  A lattice owns one for its single-RHS
// calls; a batched solve creates one per RHS.
constexpr int kSchurSlot = 24;
constexpr int kEoSlot = 27;
constexpr int kRasEoSlot = 32;
constexpr int kHalfKrylovSlot = 36;
constexpr int kEoResSlot = 44;
struct SolverState {
    SolverScalars *scal = nullptr;
    SolverScalars *scal_host = nullptr;
    ReduceScratch red;
    wc_field_s *work[46] = {};
    cudaStream_t stream = nullptr;
    SolverState *inner = nullptr;   // state of a nested inner solve, created on first use
};

}  // namespace wc

struct wc_lattice_s {
    wc::Geom g{};
    cudaStream_t stream = nullptr;
    bool gauge_loaded = false;
    bool clover_loaded = false;
    double csw = 0.0, kappa = 0.0;
    int fp64_arith = WC_ARITH_F64;            // arithmetic of the FP64 operator kernels
    wc::GaugeStore gauge;
    wc::CloverStore clover;
    wc::SolverState st;                       // scratch of single-RHS calls
    double2 *staging = nullptr;               // canonical-size device buffer
    size_t staging_bytes = 0;
    // asynchronous import/export: host-to-device copies run on copy_stream
    // into astage_in (ev_in_ready: copied; ev_in_free: consumed by the
    // import kernel); device-to-host copies run on copy_out_stream from two
    // alternating buffers astage_out[b] (ev_out_ready[b]: written by the
    // export kernel; ev_out_free[b]: copied out), so that a step's copy out
    // overlaps the next step's kernels
    cudaStream_t copy_stream = nullptr, copy_out_stream = nullptr;
    cudaEvent_t ev_in_ready = nullptr, ev_in_free = nullptr;
    cudaEvent_t ev_out_ready[2] = {nullptr, nullptr}, ev_out_free[2] = {nullptr, nullptr};
    double2 *astage_in = nullptr, *astage_out[2] = {nullptr, nullptr};
    int out_buf = 0;
    // even-odd: A^-1 (built on first use) and the half lattice whose
    // operator is the Schur complement M^ (V/2 sites, shares gauge/clover)
    wc::CloverStore cinv;                     // A^-1, parity-ordered planes (even-odd kernels)
    wc::CloverStore ceo;                      // A, parity-ordered copy (even-odd kernels)
    bool cinv_loaded = false;
    wc_lattice_s *half = nullptr;
    wc_lattice_s *schur_parent = nullptr;     // set on a half lattice
    wc_field_s *schur_tmp[3] = {};            // half lattice: odd-site temporaries
    // sub-domain of a decomposed lattice (wc_create_subdomain): extents of
    // the whole lattice, global coordinate of local site 0, bit mu of
    // split_mask: direction mu is cut (its faces border other sub-domains),
    // and the lattice extended by one site across every cut face, on which
    // the gauge field is loaded and the clover term built
    int global_L[4] = {0, 0, 0, 0};
    int offset[4] = {0, 0, 0, 0};
    int split_mask = 0;
    wc_lattice_s *ext = nullptr;
    // wc_solve_batch: the solver states of its right-hand sides on this
    // lattice, and (full lattice of an even-odd batch) five FP64
    // half-lattice fields per right-hand side, kept for the next batch (a
    // batch with k right-hand sides here takes the first k)
    std::vector<wc::SolverState> batch_states;
    std::vector<wc_field_s *> batch_fields;
    // wc_ras_schur: the even-site input and output on the half lattice, per
    // precision (created on first use)
    wc_field_s *ras_half[3][2] = {};
    std::string err;
};

struct wc_field_s {
    wc_lattice lat = nullptr;
    wc_prec prec = WC_F64;
    void *data = nullptr;
    float *nrm = nullptr;   // FP16 only: per-site scale
};

namespace wc {

inline size_t spinor_bytes(wc_prec p, int V)
{
    return p == WC_F64 ? (size_t)V * 12 * sizeof(double2)
         : p == WC_F32 ? (size_t)V * 6 * sizeof(float4)
                       : (size_t)V * 3 * sizeof(uint4);
}

// launchers implemented in the .cu files (all asynchronous on `stream`)
cudaError_t launch_apply(wc_lattice lat, wc_field out, wc_field in, int kind /*0 M, 1 Mdag, 2 H*/,
                         cudaStream_t stream);
// The operator of a solve on S.stream; on a half lattice (M^) the odd-site
// intermediate is the state's own (slot kSchurSlot + precision, when it
// exists), so that solves on one lattice may run concurrently.
cudaError_t launch_apply(wc_lattice lat, wc_field out, wc_field in, int kind, SolverState &S);
cudaError_t launch_copy(wc_lattice lat, wc_field dst, wc_field src, double scale, const double *dev_scale,
                        int invert_scale, cudaStream_t stream);
// RAS on block Schur complements, on half-lattice (even-site) fields of the
// half lattice of full (A^-1 built)
bool ras_schur_fits(const wc_ras_params &p);
cudaError_t launch_ras_schur(const wc_lattice_s *full, wc_field out, wc_field in, const wc_ras_params &p, int dagger,
                             cudaStream_t stream);
cudaError_t launch_ras(wc_lattice lat, wc_field out, wc_field in, const wc_ras_params &p, int dagger,
                       cudaStream_t stream);

bool apply_shape(wc_lattice lat, wc_prec prec, int kind, int force, int out[6]);

// WC_OK when the whole-lattice operator of lat can be applied: gauge field
// (and, with need_clover, the clover term) loaded, and lat not a sub-domain,
// whose operator needs its neighbours' face data (wc_halo_pack /
// wc_apply_interior / wc_apply_surface)
wc_status require_operator(wc_lattice lat, bool need_clover = true);

// sub-domains (wc_halo.cu): copy the interior of the extended lattice's
// gauge field / clover term into the sub-domain's stores
cudaError_t extract_gauge(wc_lattice sub, cudaStream_t stream);
cudaError_t extract_clover(wc_lattice sub, cudaStream_t stream);

// multi-right-hand-side FP32 operator (wc_mrhs.cu): outs[r] = M ins[r]
// (kind 0) or M^+ ins[r] (kind 1) for r < n <= kMrhsMax, links and clover
// read once per site; active (nullable, device): 0 skips right-hand side r
constexpr int kMrhsMax = 16;
cudaError_t launch_apply_multi(wc_lattice lat, int n, const wc_field *outs, const wc_field *ins, int kind,
                               const int *active, cudaStream_t stream);

// multi-right-hand-side Schur operator (wc_eomulti.cu): outs[r] = M^ ins[r]
// (M^+ with dagger) for FP32 or FP16 half-lattice fields of the half lattice
// `half`, tmps[r] its odd-site intermediates; skip (nullable) holds per field
// a device flag (nullable) whose nonzero value skips it
cudaError_t launch_schur_multi(wc_lattice half, int n, wc_field const *outs, wc_field const *ins,
                               wc_field const *tmps, int dagger, const int *const *skip, cudaStream_t stream,
                               int red = 0, wc_field const *dots = nullptr, double *part = nullptr);
// CTAs of one multi-RHS Schur pass on the half lattice `half` (the second
// dimension of its partial sums)
int schur_multi_blocks(wc_lattice half);

// even-odd preconditioning (wc_evenodd.cu)
// tmp: a half-lattice field of out's precision for the odd-site
// intermediate (nullptr: the half lattice's own, shared by its callers)
cudaError_t launch_schur(wc_lattice half, wc_field out, wc_field in, int dagger, cudaStream_t stream,
                         wc_field tmp = nullptr);
// out2: the second output of mode 5 (nullptr for the other modes)
cudaError_t launch_eo(const wc_lattice_s *full, int parity, int mode, int dagger, const wc_field_s *hin,
                      const wc_field_s *vin, wc_field_s *out, double beta, cudaStream_t stream,
                      wc_field_s *out2 = nullptr);
cudaError_t launch_split(const wc_lattice_s *full, const wc_field_s *f, wc_field_s *ev, wc_field_s *od,
                         cudaStream_t stream);
cudaError_t launch_merge(const wc_lattice_s *full, const wc_field_s *ev, const wc_field_s *od, wc_field_s *f,
                         cudaStream_t stream);
wc_status build_clover_inverse(wc_lattice lat);
wc_status half_lattice(wc_lattice lat, wc_lattice *out);
void free_half(wc_lattice lat);
// the solver states and fields a lattice keeps for wc_solve_batch
void free_batch_pool(wc_lattice lat);
int apply_shape_count();

// solver states
wc_status state_init(wc_lattice lat, SolverState &s);
void state_free(SolverState &s);
wc_field state_work(wc_lattice lat, SolverState &s, int slot, wc_prec prec, wc_status *st);

// reductions over fields of any precision (blocking, on the lattice's stream)
wc_status reduce_dot(wc_lattice lat, wc_field a, wc_field b, double out[2]);
wc_status reduce_norm2(wc_lattice lat, wc_field a, double *out);
wc_status axpy_norm(wc_lattice lat, const double a[2], wc_field x, wc_field y, double *norm2);

}  // namespace wc
