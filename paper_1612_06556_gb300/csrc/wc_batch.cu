// Batched solves: many right-hand sides on possibly different lattices in
// one CUDA graph launch.
//
// The paper's host proxy exists so that the accelerator never returns to the
// host between solver steps (Sec. 2, reverse offloading).  Here the whole
// BiCGStab iteration loop of every right-hand side runs inside one graph:
//
//   flexible (FP64 BiCGStab, FP32/FP16 RAS defect correction):
//     WHILE (any RHS active)                      <- device-side condition
//       IF (RHS 0 active) { one BiCGStab step }   \
//       IF (RHS 1 active) { one BiCGStab step }    > independent branches,
//       ...                                       /  run concurrently
//       check: per RHS, stop at |r| <= tol |b|, breakdown, NaN or max_iter
//
//   reliable update (FP32 BiCGStab, FP64 refreshes):
//     WHILE (any RHS active)
//       IF (RHS i active)  { one FP32 BiCGStab step }        for every i
//       check 1: refresh due?  (|r| <= delta max|r|, |r| <= tol |b|, or
//                max_iter reached)
//       IF (RHS i refresh) { x += x_lo; r = b - M x in FP64; r32 = r;
//                            rho, beta recomputed }            for every i
//       check 2: converged (true residual) or max_iter -> inactive
//
// Lockstep groups (reliable update without a preconditioner on the half
// lattices of an even-odd batch): the right-hand sides of one lattice -- the
// sources of a propagator -- step together in one IF branch per group, and
// each step's two Schur applications are one multi-right-hand-side launch
// for the whole group (links, A and A^-1 read once per site for all of
// them), each of its five vector updates one launch over all members.  A member that has stopped keeps its place: the check kernels set
// the skip word of its solver scalars, and its step kernels (and its part
// of the multi-RHS launch) return at once.
//
// Each branch is captured from the same enqueue code the single-RHS solves
// use, on that RHS's own solver state (scalars, reduction scratch, work
// vectors), so branches share nothing but the read-only gauge field and
// clover term of their lattice.  No host round trip happens until every RHS
// has stopped; then the true residual of each RHS is recomputed in FP64 and
// any RHS that missed tol (breakdown, drift) is continued by the host-driven
// solver.
//
// RAS block shapes: with ras.block = {0,0,0,0} the shape is chosen per
// lattice extent and inner precision by a small autotuner (candidate shapes
// timed on a short trial solve, result cached for the process).
#include <math.h>
#include <stdlib.h>

#include <chrono>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "wc_internal.cuh"
#include "wc_solver.cuh"
#include "wc_solver_kernels.cuh"

namespace wc {

bool ras_fits(const wc_ras_params &p);

namespace {

struct BatchItem {
    SolverScalars *scal;
    double tol2;    // tol^2 |b|^2
    double d2;      // delta^2 (reliable update)
    int max_iter;
    int pad;
    double defer2;  // > 0: stop unconfirmed once the recurrence |r|^2 <= defer2 (the caller confirms)
};

// Device-side per-RHS state of the loop.
struct BatchDev {
    const BatchItem *items;
    int *iters;
    int *active;
    int *refresh;
    double *rmax2;                              // [2n]: max |r|^2 since the last refresh, last |r|^2
    const cudaGraphConditionalHandle *h_iter;   // per RHS outside lockstep groups
    const cudaGraphConditionalHandle *h_ref;
    int *fresh;                                 // per RHS: 1 stopped right after a refresh, 2 stopped
                                                // unconfirmed (below defer2, no refresh)
    const int *group;                           // per RHS: lockstep group, -1 if none
    const cudaGraphConditionalHandle *h_group;  // per group
    int ngroups;
};

constexpr int kMaxGroups = 64;

// After the BiCGStab steps.  Flexible: decide which RHS continue and set
// the WHILE condition.  Reliable: decide which RHS refresh now.
__global__ void k_batch_check_iter(BatchDev d, int n, int reliable, cudaGraphConditionalHandle wh)
{
    __shared__ int any;
    if (threadIdx.x == 0) any = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const BatchItem &it = d.items[i];
        int a = d.active[i];
        int ref = 0;
        if (a) {
            const int k = ++d.iters[i];
            const SolverScalars &s = *it.scal;
            if (!reliable) {
                if (!(s.rr > it.tol2) || s.flags != 0 || k >= it.max_iter) a = 0;
            } else if (s.flags != 0) {
                a = 0;   // breakdown / NaN: the host takes over
                d.fresh[i] = 0;
                if (d.group[i] >= 0) it.scal->skip = 1;
            } else {
                const double prev = d.rmax2[n + i];
                d.rmax2[n + i] = s.rr;
                if (s.rr > d.rmax2[i]) d.rmax2[i] = s.rr;
                if (it.defer2 > 0.0 && s.rr <= it.defer2) {
                    a = 0;   // the caller folds the correction and confirms
                    d.fresh[i] = 2;
                } else {
                    // below tol but above defer2 the step refreshes only when
                    // the recurrence stopped decreasing
                    const bool at_tol = s.rr <= it.tol2 && (it.defer2 <= 0.0 || !(s.rr < prev));
                    ref = (s.rr <= it.d2 * d.rmax2[i] || at_tol || k >= it.max_iter) ? 1 : 0;
                }
            }
            d.active[i] = a;
        }
        if (reliable) {
            d.refresh[i] = ref;
            cudaGraphSetConditional(d.h_ref[i], ref ? 1u : 0u);
        } else {
            cudaGraphSetConditional(d.h_iter[i], a ? 1u : 0u);
            if (a) atomicOr(&any, 1);
        }
    }
    __syncthreads();
    if (!reliable && threadIdx.x == 0) cudaGraphSetConditional(wh, any ? 1u : 0u);
}

// Reliable update only, after the refreshes: stop converged RHS (FP64 true
// residual) and RHS at max_iter; set the IF conditions (per RHS, or per
// lockstep group with the members' skip words) and the WHILE condition.
__global__ void k_batch_check_refresh(BatchDev d, int n, cudaGraphConditionalHandle wh)
{
    __shared__ int any;
    __shared__ int gany[kMaxGroups];
    if (threadIdx.x == 0) any = 0;
    for (int g = threadIdx.x; g < d.ngroups; g += blockDim.x) gany[g] = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const BatchItem &it = d.items[i];
        int a = d.active[i];
        if (a && d.refresh[i]) {
            const double rr = it.scal->rr;   // FP64 true residual of the refresh
            if (!(rr > it.tol2) || d.iters[i] >= it.max_iter) {
                a = 0;
                d.fresh[i] = 1;   // x and the FP64 residual rr are current
            }
            d.rmax2[i] = rr;
            d.rmax2[n + i] = rr;
            d.active[i] = a;
        }
        const int g = d.group[i];
        if (g >= 0) {
            it.scal->skip = a ? 0 : 1;
            if (a) atomicOr(&gany[g], 1);
        } else {
            cudaGraphSetConditional(d.h_iter[i], a ? 1u : 0u);
        }
        if (a) atomicOr(&any, 1);
    }
    __syncthreads();
    for (int g = threadIdx.x; g < d.ngroups; g += blockDim.x) cudaGraphSetConditional(d.h_group[g], gany[g] ? 1u : 0u);
    if (threadIdx.x == 0) cudaGraphSetConditional(wh, any ? 1u : 0u);
}

struct Resources {
    std::vector<SolverState> S;
    std::vector<SolverVecs> W;
    std::vector<LoVecs> LW;
    std::vector<cudaStream_t> streams;
    BatchItem *d_items = nullptr;
    int *d_iters = nullptr, *d_active = nullptr, *d_refresh = nullptr, *d_group = nullptr, *d_fresh = nullptr;
    std::vector<std::pair<wc_lattice, int>> home;   // pool slot each state came from
    double *d_rmax2 = nullptr;
    cudaGraphConditionalHandle *d_hiter = nullptr, *d_href = nullptr, *d_hgroup = nullptr;
    std::vector<LoMember *> d_members;   // per lockstep group
    std::vector<double *> d_part;        // per lockstep group: fused partial sums (FP32 vectors)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;

    ~Resources()
    {
        for (auto s : streams)
            if (s) cudaStreamSynchronize(s);
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        cudaFree(d_items);
        cudaFree(d_iters);
        cudaFree(d_active);
        cudaFree(d_refresh);
        cudaFree(d_rmax2);
        cudaFree(d_hiter);
        cudaFree(d_href);
        cudaFree(d_group);
        cudaFree(d_hgroup);
        cudaFree(d_fresh);
        for (auto m : d_members) cudaFree(m);
        for (auto q : d_part) cudaFree(q);
        // states go back to their lattice's pool, with the work fields
        // this batch added
        for (size_t i = 0; i < S.size(); ++i) {
            S[i].stream = nullptr;
            if (i < home.size() && home[i].first)
                home[i].first->batch_states[home[i].second] = S[i];
            else
                state_free(S[i]);
        }
        for (auto s : streams)
            if (s) cudaStreamDestroy(s);
    }
};

template <class T>
cudaError_t to_device(T **dst, const std::vector<T> &src)
{
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(dst), sizeof(T) * src.size());
    if (e == cudaSuccess) e = cudaMemcpy(*dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice);
    return e;
}

// n IF-condition handles of graph `parent` with default values initial[i]
wc_status create_handles(cudaGraph_t parent, int n, const std::vector<int> &initial,
                         std::vector<cudaGraphConditionalHandle> *handles)
{
    handles->assign(n, 0);
    for (int i = 0; i < n; ++i) {
        wc_status st = check_cuda(nullptr, cudaGraphConditionalHandleCreate(&(*handles)[i], parent,
                                                                            initial[i] ? 1u : 0u,
                                                                            cudaGraphCondAssignDefault),
                                  "cudaGraphConditionalHandleCreate");
        if (st != WC_OK) return st;
    }
    return WC_OK;
}

// One IF node per handle, each depending on deps, whose body holds the
// launches `enqueue(k)` queues on the stream of right-hand side idx[k]
// while that stream is captured.
template <class Enqueue>
wc_status add_if_nodes(cudaGraph_t parent, const std::vector<cudaGraphNode_t> &deps,
                       const std::vector<cudaGraphConditionalHandle> &handles, const std::vector<int> &idx,
                       Resources &R, Enqueue enqueue, std::vector<cudaGraphNode_t> *nodes)
{
    for (size_t k = 0; k < handles.size(); ++k) {
        cudaGraphNodeParams ip = {};
        ip.type = cudaGraphNodeTypeConditional;
        ip.conditional.handle = handles[k];
        ip.conditional.type = cudaGraphCondTypeIf;
        ip.conditional.size = 1;
        cudaGraphNode_t node;
        wc_status st = check_cuda(nullptr, cudaGraphAddNode(&node, parent, deps.empty() ? nullptr : deps.data(),
                                                            nullptr, deps.size(), &ip), "add IF node");
        if (st != WC_OK) return st;
        nodes->push_back(node);
        cudaStream_t s = R.streams[idx[k]];
        st = check_cuda(nullptr, cudaStreamBeginCaptureToGraph(s, ip.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                                               cudaStreamCaptureModeRelaxed),
                        "cudaStreamBeginCaptureToGraph");
        if (st != WC_OK) return st;
        const wc_status est = enqueue((int)k);
        cudaGraph_t captured = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(s, &captured);
        if (est != WC_OK) return est;
        st = check_cuda(nullptr, ce, "cudaStreamEndCapture");
        if (st != WC_OK) return st;
    }
    return WC_OK;
}

// Lockstep groups for Krylov vectors of precision kp: WC_BATCH_LOCKSTEP=0
// keeps one branch per right-hand side, =1 groups FP32 and FP16 vectors;
// by default FP32 vectors step in lockstep and FP16 vectors do not (their
// multi-right-hand-side Schur passes gain only 1.13x over single ones, and
// on the 36-source batch the branches measured 5 % faster).
bool lockstep_enabled(wc_prec kp)
{
    const char *e = getenv("WC_BATCH_LOCKSTEP");
    if (e && e[0] == '0') return false;
    if (e && e[0] == '1') return true;
    return kp == WC_F32;
}

// One lockstep step of the reliable update for the right-hand sides idx of
// one half lattice, queued on stream s: each vector update is one launch for
// all members (member table dm on the device), each of the two Schur
// applications one multi-right-hand-side launch; the kernels of a stopped
// member return at once (its skip word).  With FP32 vectors the inner
// products of alpha (<rhat, v>) and omega (<t, s>, |t|^2, |s|^2) are summed
// by the even Schur pass that produces v and t (partials in part) and
// finished by a one-CTA-per-member kernel, instead of two more passes over
// the vectors.
wc_status enqueue_group_step(wc_lattice half, const std::vector<int> &idx, Resources &R, const LoMember *dm,
                             double *part, cudaStream_t s)
{
    const int m = (int)idx.size();
    std::vector<wc_field> p(m), v(m), sv(m), t(m), tmp(m);
    std::vector<const int *> skip(m);
    for (int k = 0; k < m; ++k) {
        const int i = idx[k];
        const LoVecs &w = R.LW[i];
        p[k] = w.phat;
        v[k] = w.v;
        sv[k] = w.shat;
        t[k] = w.t;
        tmp[k] = R.S[i].work[kSchurSlot + w.v->prec];
        skip[k] = &R.S[i].scal->skip;
        if (!tmp[k]) return set_error(half, WC_ERR_STATE, "lockstep: no odd-site intermediate");
    }
    const bool hv = R.LW[idx[0]].v->prec == WC_F16;
    const bool fused = !hv && part;
    const int mb = R.S[idx[0]].red.max_blocks, nblk = schur_multi_blocks(half);
    std::vector<wc_field> rh(m);
    for (int k = 0; k < m; ++k) rh[k] = R.LW[idx[k]].rhat;
    wc_status st = check_cuda(half, lo_group(LO_STEP_P, half, m, dm, hv, mb, s), "lo_p");
    if (st == WC_OK)
        st = check_cuda(half, launch_schur_multi(half, m, v.data(), p.data(), tmp.data(), 0, skip.data(), s,
                                                 fused ? 1 : 0, rh.data(), part), "schur_multi");
    if (st == WC_OK)
        st = fused ? check_cuda(half, lo_group_finalize(LO_STEP_ALPHA, m, nblk, part, dm, s), "alpha")
                   : check_cuda(half, lo_group(LO_STEP_ALPHA, half, m, dm, hv, mb, s), "lo_alpha");
    if (st == WC_OK) st = check_cuda(half, lo_group(LO_STEP_S, half, m, dm, hv, mb, s), "lo_s");
    if (st == WC_OK)
        st = check_cuda(half, launch_schur_multi(half, m, t.data(), sv.data(), tmp.data(), 0, skip.data(), s,
                                                 fused ? 2 : 0, nullptr, part), "schur_multi");
    if (st == WC_OK)
        st = fused ? check_cuda(half, lo_group_finalize(LO_STEP_OMEGA, m, nblk, part, dm, s), "omega")
                   : check_cuda(half, lo_group(LO_STEP_OMEGA, half, m, dm, hv, mb, s), "lo_omega");
    if (st == WC_OK) st = check_cuda(half, lo_group(LO_STEP_XR, half, m, dm, hv, mb, s), "lo_xr");
    return st;
}

wc_status add_kernel_node(cudaGraph_t g, const std::vector<cudaGraphNode_t> &deps, void *func, void **args,
                          cudaGraphNode_t *node)
{
    cudaKernelNodeParams kp = {};
    kp.func = func;
    kp.gridDim = dim3(1);
    kp.blockDim = dim3(256);
    kp.sharedMemBytes = 0;
    kp.kernelParams = args;
    return check_cuda(nullptr, cudaGraphAddKernelNode(node, g, deps.data(), deps.size(), &kp), "add check node");
}

// ---- RAS block-shape autotuner ------------------------------------------

std::mutex g_tune_mutex;
std::map<std::tuple<int, int, int, int, int, int>, wc_ras_params> g_tuned;

std::vector<wc_ras_params> ras_candidates(wc_lattice lat, const wc_ras_params &base)
{
    std::vector<wc_ras_params> out;
    const int opts[3] = {2, 4, 8};
    for (int a : opts)
        for (int b : opts)
            for (int c : opts)
                for (int d : opts) {
                    const int core = a * b * c * d;
                    if (core < 128 || core > 512) continue;
                    wc_ras_params q = base;
                    q.block[0] = a;
                    q.block[1] = b;
                    q.block[2] = c;
                    q.block[3] = d;
                    bool ok = ras_fits(q);
                    for (int m = 0; m < 4 && ok; ++m)
                        ok = lat->g.L[m] % q.block[m] == 0 && lat->g.L[m] > q.block[m] + 2 * q.overlap;
                    if (ok) out.push_back(q);
                }
    return out;
}

// Pick the block shape that reduces the residual fastest on a short trial
// solve of M x = b from x = 0 (log of the residual reduction per second).
wc_status autotune_ras(wc_lattice lat, wc_field b, const wc_solve_params &p, wc_ras_params *out)
{
    const auto key = std::make_tuple(lat->g.L[0], lat->g.L[1], lat->g.L[2], lat->g.L[3], (int)p.inner_prec,
                                     p.ras.overlap * 1000 + p.ras.mr_iters);
    {
        std::lock_guard<std::mutex> lk(g_tune_mutex);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) {
            *out = it->second;
            return WC_OK;
        }
    }
    wc_ras_params base = p.ras;
    std::vector<wc_ras_params> cands = ras_candidates(lat, base);
    if (cands.empty()) return set_error(lat, WC_ERR_ARG, "RAS autotuner: no block shape fits this lattice");
    wc_field x = nullptr;
    wc_status st = wc_field_create(lat, WC_F64, &x);
    if (st != WC_OK) return st;
    double best = -1.0;
    wc_ras_params best_p = cands[0];
    // the first trial also creates the solver's work fields: run it twice
    std::vector<wc_ras_params> trials;
    trials.push_back(cands[0]);
    trials.insert(trials.end(), cands.begin(), cands.end());
    for (size_t ti = 0; ti < trials.size(); ++ti) {
        const wc_ras_params &c = trials[ti];
        wc_solve_params q = p;
        q.ras = c;
        q.max_iter = 2;
        q.max_restarts = 0;
        q.tol = 1e-30;
        st = check_cuda(lat, cudaMemsetAsync(x->data, 0, spinor_bytes(WC_F64, lat->g.V), lat->stream), "memset");
        if (st != WC_OK) break;
        wc_solve_info info{};
        const wc_status r = bicgstab(lat, 0, x, b, q, &info);
        if (r != WC_OK && r != WC_ERR_NOT_CONVERGED) continue;
        if (ti == 0 || !(info.true_rel_resid > 0.0) || info.seconds <= 0.0) continue;
        const double rate = -log(info.true_rel_resid) / info.seconds;
        if (rate > best) {
            best = rate;
            best_p = c;
        }
    }
    wc_field_destroy(x);
    if (st != WC_OK) return st;
    {
        std::lock_guard<std::mutex> lk(g_tune_mutex);
        g_tuned[key] = best_p;
    }
    *out = best_p;
    return WC_OK;
}

}  // namespace

// The RAS parameters a solve on lat uses: p.ras, or the autotuned shape
// when p.ras.block is all zero (needs a right-hand side to tune on).
wc_status resolve_ras(wc_lattice lat, wc_field b, const wc_solve_params &p, wc_ras_params *out)
{
    if (p.precond != WC_PRECOND_RAS || p.ras.block[0] != 0) {
        *out = p.ras;
        return WC_OK;
    }
    if (p.ras.schur)
        return set_error(lat, WC_ERR_ARG, "give the block shape of the block-Schur RAS explicitly");
    return autotune_ras(lat, b, p, out);
}

}  // namespace wc

using namespace wc;

static wc_status batch_core(int n, const wc_lattice *lats, wc_field *xs, wc_field *bs, const wc_solve_params *p,
                            const double *tol_scale, wc_solve_info *infos, double defer_margin = 0.0,
                            int *unconfirmed = nullptr);
static wc_status batch_even_odd(int n, const wc_lattice *lats, wc_field *xs, wc_field *bs,
                                const wc_solve_params *p, wc_solve_info *infos);

extern "C" wc_status wc_solve_batch(int n, const wc_lattice *lats, wc_field *xs, wc_field *bs,
                                    const wc_solve_params *p, wc_solve_info *infos)
{
    if (n < 0 || (n > 0 && (!lats || !xs || !bs || !p || !infos)))
        return set_error(nullptr, WC_ERR_ARG, "wc_solve_batch: bad arguments");
    if (n == 0) return WC_OK;
    if (p->solver == WC_SOLVER_NESTED)
        return set_error(nullptr, WC_ERR_ARG, "wc_solve_batch: the nested solver is host-driven; use FLEXIBLE "
                                              "or RELIABLE");
    if (p->even_odd && p->precond == WC_PRECOND_RAS && p->ras.block[0] == 0)
        return set_error(nullptr, WC_ERR_ARG, "wc_solve_batch: with even_odd give the RAS block shape explicitly");
    for (int i = 0; i < n; ++i) {
        // the RAS shape is checked after autotuning when it is left to it
        wc_solve_params q = *p;
        if (q.precond == WC_PRECOND_RAS && q.ras.block[0] == 0) {
            for (int m = 0; m < 4; ++m) q.ras.block[m] = 1;
            q.ras.overlap = 0;
        }
        if (!lats[i]) return set_error(nullptr, WC_ERR_ARG, "wc_solve_batch: NULL lattice");
        const wc_status st = check_solve_args(lats[i], xs[i], bs[i], &q);
        if (st != WC_OK)
            return set_error(nullptr, st, "wc_solve_batch: RHS " + std::to_string(i) + ": " + lats[i]->err);
        for (int j = 0; j < i; ++j)
            if (xs[j] == xs[i] || xs[i] == bs[j])
                return set_error(nullptr, WC_ERR_ARG, "wc_solve_batch: solution fields must be distinct");
    }
    return p->even_odd ? batch_even_odd(n, lats, xs, bs, p, infos) : batch_core(n, lats, xs, bs, p, nullptr, infos);
}

// The batched solve proper, on checked arguments.  tol_scale (may be null):
// per-RHS factors on p->tol.  defer_margin > 0 (reliable solver, a caller
// that recomputes every true residual): an RHS whose recurrence residual
// falls below defer_margin tol stops without a last FP64 refresh, its
// correction folded into x; unconfirmed[i] (n entries) is then set to 1.
static wc_status batch_core(int n, const wc_lattice *lats, wc_field *xs, wc_field *bs, const wc_solve_params *p,
                            const double *tol_scale, wc_solve_info *infos, double defer_margin, int *unconfirmed)
{
    const bool reliable = p->solver == WC_SOLVER_RELIABLE;
    auto t0 = std::chrono::steady_clock::now();
    Resources R;
    R.S.resize(n);
    R.W.resize(n);
    R.LW.resize(n);
    R.streams.assign(n, nullptr);
    std::vector<wc_solve_params> P(n, *p);
    if (tol_scale)
        for (int i = 0; i < n; ++i) P[i].tol *= tol_scale[i];
    wc_status st = check_cuda(nullptr, ras_prepare(), "ras_prepare");
    for (int i = 0; i < n && st == WC_OK; ++i) {
        st = resolve_ras(lats[i], bs[i], *p, &P[i].ras);
        if (st == WC_OK && P[i].precond == WC_PRECOND_RAS) st = check_ras_params(lats[i], &P[i].ras);
        if (st != WC_OK) return set_error(nullptr, st, std::string("wc_solve_batch: ") + lats[i]->err);
    }
    // solver states from the lattices' pools (created on first use; their
    // work fields persist from batch to batch)
    R.home.assign(n, std::make_pair(wc_lattice(nullptr), 0));
    {
        std::map<wc_lattice, int> used;
        for (int i = 0; i < n && st == WC_OK; ++i) {
            const int k = used[lats[i]]++;
            auto &pool = lats[i]->batch_states;
            if (k == (int)pool.size()) {
                SolverState fresh;
                st = state_init(lats[i], fresh);
                if (st != WC_OK) break;
                pool.push_back(fresh);
            }
            R.S[i] = pool[k];
            pool[k] = SolverState{};   // held by this batch until it returns
            R.home[i] = std::make_pair(lats[i], k);
        }
    }
    for (int i = 0; i < n && st == WC_OK; ++i) {
        st = check_cuda(lats[i], cudaStreamCreateWithFlags(&R.streams[i], cudaStreamNonBlocking), "stream");
        if (st == WC_OK) {
            R.S[i].stream = R.streams[i];
            st = check_cuda(lats[i], cudaMemsetAsync(R.S[i].scal, 0, sizeof(SolverScalars), R.streams[i]), "memset");
        }
        if (st == WC_OK)
            st = check_cuda(lats[i], cudaMemsetAsync(R.S[i].red.ticket, 0, sizeof(unsigned), R.streams[i]), "memset");
        if (st == WC_OK) st = solver_vectors(lats[i], R.S[i], P[i], &R.W[i]);
        if (st == WC_OK && reliable) st = lo_vectors(lats[i], R.S[i], P[i], &R.LW[i]);
    }
    if (st != WC_OK) return st;

    // |b|^2 and |x|^2 (a zero start needs no operator application), then
    // the start of every solve, one synchronisation for each
    std::vector<double> bb(n), tol2(n);
    std::vector<char> x_zero(n, 0);
    for (int i = 0; i < n && st == WC_OK; ++i) {
        SolverState &S = R.S[i];
        st = check_cuda(lats[i], norm2_to_result(lats[i], S, static_cast<const double2 *>(xs[i]->data)), "norm2");
        if (st == WC_OK)
            st = check_cuda(lats[i], cudaMemcpyAsync(S.red.host_result + 1, S.red.result, sizeof(double),
                                                     cudaMemcpyDeviceToHost, S.stream), "copy");
        if (st == WC_OK)
            st = check_cuda(lats[i], norm2_to_result(lats[i], S, static_cast<const double2 *>(bs[i]->data)), "norm2");
        if (st == WC_OK)
            st = check_cuda(lats[i], cudaMemcpyAsync(S.red.host_result, S.red.result, sizeof(double),
                                                     cudaMemcpyDeviceToHost, S.stream), "copy");
    }
    for (int i = 0; i < n && st == WC_OK; ++i) st = check_cuda(lats[i], cudaStreamSynchronize(R.streams[i]), "sync");
    for (int i = 0; i < n && st == WC_OK; ++i) {
        SolverState &S = R.S[i];
        bb[i] = S.red.host_result[0];
        x_zero[i] = S.red.host_result[1] == 0.0;
        st = reliable ? enqueue_lo_start(lats[i], S, 0, xs[i], bs[i], R.W[i].r, R.LW[i], x_zero[i] != 0)
                      : enqueue_init(lats[i], S, 0, xs[i], bs[i], R.W[i], x_zero[i] != 0);
        if (st == WC_OK)
            st = check_cuda(lats[i], cudaMemcpyAsync(S.scal_host, S.scal, sizeof(SolverScalars),
                                                     cudaMemcpyDeviceToHost, S.stream), "copy");
    }
    for (int i = 0; i < n && st == WC_OK; ++i) st = check_cuda(lats[i], cudaStreamSynchronize(R.streams[i]), "sync");
    if (st != WC_OK) return st;
    std::vector<int> active(n, 0), iters(n, 0), zeros(n, 0), fresh(n, 0);
    // per RHS: the largest |r|^2 since the last refresh, then (entries n +
    // i) the |r|^2 of the previous step
    std::vector<double> rmax2(2 * (size_t)n, 0.0);
    int any = 0;
    for (int i = 0; i < n; ++i) {
        infos[i] = wc_solve_info{};
        tol2[i] = P[i].tol * P[i].tol * bb[i];
        const SolverScalars &h = *R.S[i].scal_host;
        rmax2[i] = h.rr;
        rmax2[n + i] = h.rr;
        if (!isfinite(bb[i]) || (h.flags & FLAG_NAN) || !isfinite(h.rr)) {
            infos[i].status = WC_ERR_NAN;
        } else if (bb[i] == 0.0 || h.rr <= tol2[i]) {
            infos[i].status = WC_OK;   // settled below (zero source: x = 0)
        } else if (P[i].max_iter > 0) {
            active[i] = 1;
            any = 1;
        }
    }

    // lockstep groups: reliable update without a preconditioner on a half
    // lattice, right-hand sides of the same lattice, up to kMrhsMax a group
    std::vector<int> group(n, -1);
    std::vector<std::vector<int>> members;
    if (reliable && lockstep_enabled(P[0].krylov_prec == WC_F16 ? WC_F16 : WC_F32)) {
        std::map<std::pair<wc_lattice, int>, int> open;   // (lattice, precision) -> group being filled
        for (int i = 0; i < n; ++i) {
            if (P[i].precond != WC_PRECOND_NONE || !lats[i]->schur_parent) continue;
            const int pr = (int)R.LW[i].v->prec;
            if (pr != WC_F32 && pr != WC_F16) continue;
            const auto key = std::make_pair(lats[i], pr);
            auto it = open.find(key);
            if (it == open.end() || (int)members[it->second].size() == kMrhsMax) {
                if ((int)members.size() == kMaxGroups) continue;
                open[key] = (int)members.size();
                members.emplace_back();
                it = open.find(key);
            }
            group[i] = it->second;
            members[it->second].push_back(i);
        }
        // a group of one gains nothing: back to its own branch
        for (auto &m : members)
            if (m.size() == 1) {
                group[m[0]] = -1;
                m.clear();
            }
        std::vector<std::vector<int>> kept;
        for (auto &m : members)
            if (!m.empty()) {
                for (int i : m) group[i] = (int)kept.size();
                kept.push_back(m);
            }
        members.swap(kept);
    }
    const int ngroups = (int)members.size();

    if (any) {
        std::vector<BatchItem> items(n);
        for (int i = 0; i < n; ++i) {
            const double dl = (P[i].delta > 0.0 && P[i].delta < 1.0) ? P[i].delta : 0.01;
            items[i] = BatchItem{R.S[i].scal, tol2[i], dl * dl, P[i].max_iter, 0,
                                 defer_margin * defer_margin * tol2[i]};
        }
        st = check_cuda(nullptr, to_device(&R.d_items, items), "copy");
        if (st == WC_OK) st = check_cuda(nullptr, to_device(&R.d_iters, iters), "copy");
        if (st == WC_OK) st = check_cuda(nullptr, to_device(&R.d_active, active), "copy");
        if (st == WC_OK) st = check_cuda(nullptr, to_device(&R.d_refresh, zeros), "copy");
        if (st == WC_OK) st = check_cuda(nullptr, to_device(&R.d_rmax2, rmax2), "copy");
        if (st == WC_OK) st = check_cuda(nullptr, to_device(&R.d_group, group), "copy");
        if (st == WC_OK) st = check_cuda(nullptr, to_device(&R.d_fresh, zeros), "copy");
        R.d_members.assign(ngroups, nullptr);
        R.d_part.assign(ngroups, nullptr);
        for (int g = 0; g < ngroups && st == WC_OK; ++g) {
            const int i0 = members[g][0];
            if (R.LW[i0].v->prec == WC_F32)
                st = check_cuda(nullptr, cudaMalloc(reinterpret_cast<void **>(&R.d_part[g]),
                                                    sizeof(double) * 4 * members[g].size() *
                                                        (size_t)schur_multi_blocks(lats[i0])),
                                "cudaMalloc");
            if (st != WC_OK) break;
            std::vector<LoMember> tab;
            for (int i : members[g]) {
                const LoVecs &w = R.LW[i];
                tab.push_back(lo_member(R.S[i], w.r, w.rhat, w.p, w.v, w.s, w.t, w.phat, w.shat, w.xlo));
            }
            st = check_cuda(nullptr, to_device(&R.d_members[g], tab), "copy");
        }
        // a member that starts inactive skips from the first step
        const int one = 1;
        for (int i = 0; i < n && st == WC_OK; ++i)
            if (group[i] >= 0 && !active[i])
                st = check_cuda(nullptr, cudaMemcpy(&R.S[i].scal->skip, &one, sizeof(int), cudaMemcpyHostToDevice),
                                "copy");
        // top level: one WHILE node
        if (st == WC_OK) st = check_cuda(nullptr, cudaGraphCreate(&R.graph, 0), "cudaGraphCreate");
        cudaGraphConditionalHandle wh = 0;
        cudaGraph_t body = nullptr;
        if (st == WC_OK)
            st = check_cuda(nullptr, cudaGraphConditionalHandleCreate(&wh, R.graph, 1, cudaGraphCondAssignDefault),
                            "cudaGraphConditionalHandleCreate");
        if (st == WC_OK) {
            cudaGraphNodeParams wp = {};
            wp.type = cudaGraphNodeTypeConditional;
            wp.conditional.handle = wh;
            wp.conditional.type = cudaGraphCondTypeWhile;
            wp.conditional.size = 1;
            cudaGraphNode_t wnode;
            st = check_cuda(nullptr, cudaGraphAddNode(&wnode, R.graph, nullptr, nullptr, 0, &wp), "add WHILE node");
            if (st == WC_OK) body = wp.conditional.phGraph_out[0];
        }
        // body: IF(active_i){step_i} -> check_iter [-> IF(refresh_i){refresh_i} -> check_refresh]
        //       IF(group g any active){lockstep step of group g}
        std::vector<cudaGraphConditionalHandle> h_iter(n, 0), h_ref, h_grp, h_own;
        std::vector<int> own, own_active, grp_lead, grp_active(ngroups, 0), all(n);
        for (int i = 0; i < n; ++i) {
            all[i] = i;
            if (group[i] < 0) {
                own.push_back(i);
                own_active.push_back(active[i]);
            } else if (active[i]) {
                grp_active[group[i]] = 1;
            }
        }
        for (const auto &m : members) grp_lead.push_back(m[0]);
        std::vector<cudaGraphNode_t> iter_nodes, ref_nodes;
        if (st == WC_OK) st = create_handles(body, (int)own.size(), own_active, &h_own);
        if (st == WC_OK) st = create_handles(body, ngroups, grp_active, &h_grp);
        for (size_t k = 0; k < own.size() && st == WC_OK; ++k) h_iter[own[k]] = h_own[k];
        if (st == WC_OK && reliable) st = create_handles(body, n, zeros, &h_ref);
        if (st == WC_OK) st = check_cuda(nullptr, to_device(&R.d_hiter, h_iter), "copy");
        if (st == WC_OK && reliable) st = check_cuda(nullptr, to_device(&R.d_href, h_ref), "copy");
        if (st == WC_OK && ngroups > 0) st = check_cuda(nullptr, to_device(&R.d_hgroup, h_grp), "copy");
        BatchDev dev{R.d_items, R.d_iters, R.d_active, R.d_refresh, R.d_rmax2, R.d_hiter, R.d_href,
                     R.d_fresh, R.d_group, R.d_hgroup, ngroups};
        int reliable_i = reliable ? 1 : 0;
        void *args1[] = {&dev, &n, &reliable_i, &wh};
        void *args2[] = {&dev, &n, &wh};
        if (st == WC_OK)
            st = add_if_nodes(body, {}, h_own, own, R, [&](int k) {
                const int i = own[k];
                return reliable ? enqueue_lo_iteration(lats[i], R.S[i], P[i], 0, R.LW[i])
                                : enqueue_iteration(lats[i], R.S[i], P[i], 0, xs[i], R.W[i]);
            }, &iter_nodes);
        if (st == WC_OK)
            st = add_if_nodes(body, {}, h_grp, grp_lead, R, [&](int g) {
                return enqueue_group_step(lats[members[g][0]], members[g], R, R.d_members[g], R.d_part[g],
                                          R.streams[members[g][0]]);
            }, &iter_nodes);
        cudaGraphNode_t check1 = nullptr, check2 = nullptr;
        if (st == WC_OK)
            st = add_kernel_node(body, iter_nodes, reinterpret_cast<void *>(k_batch_check_iter), args1, &check1);
        if (st == WC_OK && reliable) {
            st = add_if_nodes(body, {check1}, h_ref, all, R, [&](int i) {
                return enqueue_refresh_full(lats[i], R.S[i], 0, xs[i], bs[i], R.W[i].r, R.LW[i]);
            }, &ref_nodes);
            if (st == WC_OK)
                st = add_kernel_node(body, ref_nodes, reinterpret_cast<void *>(k_batch_check_refresh), args2,
                                     &check2);
        }
        if (st == WC_OK) st = check_cuda(nullptr, cudaGraphInstantiate(&R.exec, R.graph, 0), "cudaGraphInstantiate");
        if (st == WC_OK) st = check_cuda(nullptr, cudaGraphLaunch(R.exec, R.streams[0]), "cudaGraphLaunch");
        if (st == WC_OK) st = check_cuda(nullptr, cudaStreamSynchronize(R.streams[0]), "sync(graph)");
        if (st == WC_OK)
            st = check_cuda(nullptr, cudaMemcpy(iters.data(), R.d_iters, sizeof(int) * n, cudaMemcpyDeviceToHost),
                            "copy");
        if (st == WC_OK)
            st = check_cuda(nullptr, cudaMemcpy(fresh.data(), R.d_fresh, sizeof(int) * n, cudaMemcpyDeviceToHost),
                            "copy");
        // the host-driven continuation below runs the same step kernels
        for (int i = 0; i < n && st == WC_OK; ++i)
            if (group[i] >= 0)
                st = check_cuda(nullptr, cudaMemset(&R.S[i].scal->skip, 0, sizeof(int)), "memset");
        if (st != WC_OK) return st;
    }

    // true residuals in FP64 for every RHS (the reliable solver folded its
    // FP32 correction into x at its last refresh, whose FP64 residual is
    // still in the scalars when the RHS stopped right after it), then
    // host-driven continuation of any RHS that missed tol
    for (int i = 0; i < n && st == WC_OK; ++i) {
        if (infos[i].status == WC_ERR_NAN) continue;
        SolverState &S = R.S[i];
        if (bb[i] == 0.0) {
            st = check_cuda(lats[i], cudaMemsetAsync(xs[i]->data, 0, spinor_bytes(WC_F64, lats[i]->g.V), S.stream),
                            "memset");
            continue;
        }
        if (reliable && fresh[i] == 2) {   // stopped unconfirmed: fold the correction only
            st = check_cuda(lats[i], hp_add_lo(lats[i], S, static_cast<double2 *>(xs[i]->data), R.LW[i].xlo),
                            "hp_add_lo");
            if (unconfirmed) unconfirmed[i] = 1;
        }
        if (reliable && fresh[i]) {
            if (st == WC_OK)
                st = check_cuda(lats[i], cudaMemcpyAsync(S.scal_host, S.scal, sizeof(SolverScalars),
                                                         cudaMemcpyDeviceToHost, S.stream), "copy");
            continue;
        }
        if (reliable)
            st = check_cuda(lats[i], hp_add_lo(lats[i], S, static_cast<double2 *>(xs[i]->data), R.LW[i].xlo), "hp_add_lo");
        if (st == WC_OK) st = enqueue_true_residual(lats[i], S, 0, xs[i], bs[i], R.W[i]);
        if (st == WC_OK)
            st = check_cuda(lats[i], cudaMemcpyAsync(S.scal_host, S.scal, sizeof(SolverScalars),
                                                     cudaMemcpyDeviceToHost, S.stream), "copy");
    }
    for (int i = 0; i < n && st == WC_OK; ++i) st = check_cuda(lats[i], cudaStreamSynchronize(R.streams[i]), "sync");
    if (st != WC_OK) return st;
    const double batch_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    wc_status worst = WC_OK;
    for (int i = 0; i < n; ++i) {
        wc_solve_info &inf = infos[i];
        inf.iters = iters[i];
        if (inf.status != WC_ERR_NAN && bb[i] > 0.0) {
            const double rr = R.S[i].scal_host->rr;
            inf.true_rel_resid = sqrt(rr / bb[i]);
            if (!isfinite(rr)) {
                inf.status = WC_ERR_NAN;
            } else if (rr <= tol2[i]) {
                inf.status = WC_OK;
            } else if (iters[i] >= P[i].max_iter) {
                inf.status = WC_ERR_NOT_CONVERGED;
            } else {
                // missed tol (drift of the recursive residual or breakdown):
                // continue from x with the host-driven solver
                wc_solve_params q = P[i];
                q.max_restarts = p->max_restarts > 0 ? p->max_restarts - 1 : 0;
                const int done = iters[i];
                bicgstab(lats[i], R.S[i], 0, xs[i], bs[i], q, &inf, done, bb[i]);
                inf.restarts += 1;
            }
        }
        inf.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (inf.status == WC_OK) inf.seconds = batch_seconds;
        if (inf.status != WC_OK && worst == WC_OK) worst = inf.status;
    }
    return worst;
}

// Even-odd batch: every RHS is reduced to its Schur system on the half
// lattice (b^_e = b_e + k H_eo A_oo^-1 b_o, tolerance scaled by |b|/|b^_e|),
// all Schur systems are solved in one batched graph (each solve keeps its
// odd-site intermediate in its own state), then x_o = A_oo^-1 (b_o + k H_oe
// x_e) and the FP64 true residual of the full system are formed per RHS.
static wc_status batch_even_odd(int n, const wc_lattice *lats, wc_field *xs, wc_field *bs,
                                const wc_solve_params *p, wc_solve_info *infos)
{
    auto t0 = std::chrono::steady_clock::now();
    std::vector<wc_lattice> H(n, nullptr);
    std::vector<wc_field> fe(5 * (size_t)n, nullptr);   // per RHS: b_e, b_o, x_e, x_o, b^_e
    std::vector<double> bb(n, 0.0), bbh(n, 0.0), scale(n, 1.0);
    std::vector<int> unconfirmed(n, 0);
    wc_status st = WC_OK;
    auto F = [&](int i, int k) -> wc_field & { return fe[5 * (size_t)i + k]; };
    std::map<wc_lattice, int> used;   // right-hand sides so far per lattice
    for (int i = 0; i < n && st == WC_OK; ++i) {
        wc_lattice lat = lats[i];
        st = half_lattice(lat, &H[i]);
        if (st != WC_OK) {
            st = set_error(nullptr, st, "wc_solve_batch: RHS " + std::to_string(i) + ": " + lat->err);
            break;
        }
        // the five half-lattice fields of this RHS, from the lattice's pool
        const size_t base = 5 * (size_t)used[lat]++;
        auto &pool = lat->batch_fields;
        while (st == WC_OK && pool.size() < base + 5) {
            wc_field f = nullptr;
            st = wc_field_create(H[i], WC_F64, &f);
            if (st == WC_OK) pool.push_back(f);
        }
        for (int k = 0; k < 5 && st == WC_OK; ++k) F(i, k) = pool[base + k];
        cudaStream_t s = lat->stream;
        wc_field t = H[i]->schur_tmp[WC_F64];
        if (st == WC_OK) st = check_cuda(lat, launch_split(lat, bs[i], F(i, 0), F(i, 1), s), "split");
        if (st == WC_OK) st = check_cuda(lat, launch_split(lat, xs[i], F(i, 2), F(i, 3), s), "split");
        if (st == WC_OK) st = check_cuda(lat, launch_eo(lat, 1, 4, 0, nullptr, F(i, 1), t, 0.0, s), "A_oo^-1 b_o");
        if (st == WC_OK) st = check_cuda(lat, launch_eo(lat, 0, 2, 0, t, F(i, 0), F(i, 4), lat->kappa, s), "b^_e");
        if (st == WC_OK) st = reduce_norm2(lat, bs[i], &bb[i]);
        if (st == WC_OK) st = reduce_norm2(H[i], F(i, 4), &bbh[i]);
        if (st == WC_OK && bb[i] > 0.0 && bbh[i] > 0.0) scale[i] = sqrt(bb[i] / bbh[i]);
    }
    std::vector<wc_field> xe(n), bh(n);
    for (int i = 0; i < n; ++i) {
        xe[i] = F(i, 2);
        bh[i] = F(i, 4);
    }
    wc_solve_params q = *p;
    q.even_odd = 0;
    // reliable: the half solves end without their last FP64 refresh (the
    // full residual below confirms, as in the single even-odd solve)
    const double margin = p->solver == WC_SOLVER_RELIABLE ? defer_margin() : 0.0;
    if (st == WC_OK) {
        const wc_status sc = batch_core(n, H.data(), xe.data(), bh.data(), &q, scale.data(), infos, margin,
                                        unconfirmed.data());
        if (sc == WC_ERR_CUDA || sc == WC_ERR_ARG || sc == WC_ERR_STATE) st = sc;
    }
    wc_status worst = WC_OK;
    for (int i = 0; i < n && st == WC_OK; ++i) {
        wc_lattice lat = lats[i];
        double rr = 0.0;
        st = eo_reconstruct_residual(lat, 0, F(i, 0), F(i, 1), F(i, 2), F(i, 3), xs[i], &rr);
        if (st == WC_OK && unconfirmed[i] && bb[i] > 0.0 && !(rr <= p->tol * p->tol * bb[i])) {
            // the deferred confirmation failed: resume this Schur solve from
            // x_e on the host, confirming in FP64 itself
            wc_solve_params qi = q;
            qi.tol = p->tol * scale[i];
            wc_solve_info sub{};
            H[i]->st.stream = lat->stream;
            const wc_status sr = bicgstab(H[i], H[i]->st, 0, F(i, 2), F(i, 4), qi, &sub, infos[i].iters, bbh[i]);
            if (sr != WC_OK && sr != WC_ERR_NOT_CONVERGED && sr != WC_ERR_BREAKDOWN) st = sr;
            infos[i].iters = sub.iters;
            infos[i].restarts += 1 + sub.restarts;
            if (st == WC_OK) st = eo_reconstruct_residual(lat, 0, F(i, 0), F(i, 1), F(i, 2), F(i, 3), xs[i], &rr);
        }
        if (st != WC_OK) break;
        wc_solve_info &inf = infos[i];
        inf.true_rel_resid = bb[i] > 0.0 ? sqrt(rr / bb[i]) : 0.0;
        if (!isfinite(rr)) inf.status = WC_ERR_NAN;
        else if (bb[i] == 0.0 || rr <= p->tol * p->tol * bb[i]) inf.status = WC_OK;
        else if (inf.status == WC_OK) inf.status = WC_ERR_NOT_CONVERGED;
        inf.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (inf.status != WC_OK && worst == WC_OK) worst = inf.status;
    }
    if (st != WC_OK) return st;
    return worst;
}

extern "C" wc_status wc_ras_autotune(wc_lattice lat, wc_field b, const wc_solve_params *p, wc_ras_params *out)
{
    if (!lat) return set_error(nullptr, WC_ERR_ARG, "lattice is NULL");
    if (!b || !p || !out) return set_error(lat, WC_ERR_ARG, "NULL argument");
    if (b->lat != lat || b->prec != WC_F64) return set_error(lat, WC_ERR_ARG, "b must be an FP64 field of lat");
    wc_status st0 = require_operator(lat);
    if (st0 != WC_OK) return st0;
    if (p->inner_prec != WC_F32 && p->inner_prec != WC_F16) return set_error(lat, WC_ERR_ARG, "bad inner precision");
    if (p->ras.overlap < 0 || p->ras.mr_iters < 0) return set_error(lat, WC_ERR_ARG, "bad RAS overlap / mr_iters");
    wc_solve_params q = *p;
    q.precond = WC_PRECOND_RAS;
    for (int m = 0; m < 4; ++m) q.ras.block[m] = 0;
    if (!(q.tol > 0.0)) q.tol = 1e-10;
    return resolve_ras(lat, b, q, out);
}
