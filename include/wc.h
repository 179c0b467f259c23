/*
 * wc.h -- C ABI of the GB300 Wilson-Clover library (libwc.so).
 *
 * The library applies the Wilson-Clover quark matrix
 *     M = (1 + T) - kappa H
 * to colour-spinor fields on a 4-D lattice and solves M x = b with BiCGStab:
 * plain in FP64, as an FP64 flexible (defect-correction) outer loop around
 * an FP32/FP16-storage overlapped Restricted Additive Schwarz (RAS)
 * preconditioner whose blocks are solved inside CTAs, as FP32/FP16
 * BiCGStab with FP64 reliable updates, or as the three-level nested solver,
 * each on the full lattice or on its even-odd Schur complement; the FP64
 * operator steps may run in double-FP32 arithmetic on the FP32 pipes
 * (wc_set_fp64_arith), since GB300 executes FP64 at 1/64 of its FP32 rate.
 * This is the
 * solver stack of the paper's CCS-QCD benchmark (Sec. 2: double-precision
 * flexible BiCGStab, single-precision preconditioner, even-odd and
 * overlapped RAS preconditioning, SU(3) reconstruction; Sec. 3: the hopping
 * multiplication "MULT").
 *
 * Conventions (the paper names the operator but prints no formula; these
 * are this library's reading, identical to the test oracle's):
 *   - site index  s = x + Lx*(y + Ly*(z + Lz*t)), directions mu = x,y,z,t
 *   - chiral Dirac basis: gamma_k = [[0, i s_k], [-i s_k, 0]],
 *     gamma_t = [[0, 1], [1, 0]], gamma_5 = diag(-1, -1, 1, 1)
 *   - (H psi)(x) = sum_mu (1 - gamma_mu) U_mu(x) psi(x+mu)
 *                        + (1 + gamma_mu) U_mu(x-mu)^+ psi(x-mu);
 *     hops across the time boundary are multiplied by t_bc (+1 or -1)
 *   - T(x) = i csw kappa sum_{mu<nu} sigma_munu (x) Fhat_munu(x) with
 *     sigma_munu = (i/2)[gamma_mu, gamma_nu] and Fhat the traceless
 *     anti-Hermitian part of the four-leaf clover sum divided by 8
 *
 * Canonical (caller-side) layouts, all complex128 = interleaved (re, im)
 * doubles in C order (spinors may also be passed as complex64 through
 * wc_field_import_f32 / wc_field_export_f32):
 *   gauge   U[Lt][Lz][Ly][Lx][mu][3][3]   (row, column)
 *   spinor  psi[Lt][Lz][Ly][Lx][spin 4][colour 3]
 *   force   F[Lt][Lz][Ly][Lx][mu][3][3]
 * Any pointer argument named "data" below may be a device pointer or a host
 * pointer (pageable or pinned); the library detects which.  The library
 * copies what it needs into memory it owns and never keeps a caller pointer
 * after a call returns.
 *
 * Errors: every call returns a wc_status; no C++ exception crosses the ABI.
 * A human-readable message for the last failure on a lattice is returned by
 * wc_last_error(lat) (wc_last_error(NULL) for failures without a lattice).
 * Argument errors are reported before any kernel is launched.
 *
 * Streams: each lattice runs its kernels on one CUDA stream, given at
 * creation (NULL = the legacy default stream).  Applies, imports/exports of
 * device data, casts and RAS applications are asynchronous with respect to
 * the host; reductions, solves and the force call block until their result
 * is on the host.
 */
#ifndef WC_H
#define WC_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct wc_lattice_s *wc_lattice;
typedef struct wc_field_s *wc_field;

typedef enum {
    WC_OK = 0,
    WC_ERR_ARG = 1,           /* invalid argument; nothing was launched */
    WC_ERR_CUDA = 2,          /* a CUDA call failed; see wc_last_error */
    WC_ERR_STATE = 3,         /* gauge field / clover term not loaded yet */
    WC_ERR_NOT_CONVERGED = 4, /* solver hit max_iter before tol */
    WC_ERR_BREAKDOWN = 5,     /* BiCGStab breakdown: <rhat,r>, <rhat,v> or <t,t> = 0 */
    WC_ERR_NAN = 6,           /* a non-finite norm was met inside a reduction */
    WC_ERR_TIMEOUT = 7        /* reserved: no call returns it (no device-side wait is bounded by a
                                 timeout; batched solves loop inside a CUDA graph) */
} wc_status;

typedef enum { WC_F64 = 0, WC_F32 = 1, WC_F16 = 2 } wc_prec;

typedef enum { WC_PRECOND_NONE = 0, WC_PRECOND_RAS = 1 } wc_precond;

/* Arithmetic of the operator on FP64 fields (wc_set_fp64_arith). */
typedef enum { WC_ARITH_F64 = 0, WC_ARITH_DF32 = 1 } wc_fp64_arith;

/* Overlapped RAS (paper Sec. 2, "overlapped Restricted Additive Schwarz"):
 * the lattice is tiled from the origin by blocks of block[mu] sites; each
 * block is extended by `overlap` sites on every face (periodically), M is
 * restricted to the extended block with hops that leave it dropped, and
 * mr_iters minimal-residual steps from zero solve it; only the block's core
 * is written back.  Requires L[mu] % block[mu] == 0 and
 * L[mu] > block[mu] + 2*overlap.
 * schur (even-odd solves only): 0 -- the preconditioner of the even-site
 * system is the RAS above applied to the even vector extended by zeros to
 * the full lattice and restricted back to the even sites; 1 -- RAS on block
 * Schur complements: the MR steps solve the even-site Schur complement of
 * the cut block operator, M^_B = A_ee - kappa^2 H^B_eo A_oo^-1 H^B_oe (H^B:
 * hops with both ends in the extended block), on the block's even sites
 * (parity of the global coordinates), and the core's even sites are written
 * back (wc_ras_schur).  schur = 1 needs block[0] + 2*overlap even, at most
 * 1536 sites per extended block, and an explicit block shape. */
typedef struct {
    int block[4];
    int overlap;
    int mr_iters;
    int schur;
} wc_ras_params;

/* How a preconditioned solve splits its precisions.
 * FLEXIBLE (defect correction): FP64 flexible BiCGStab -- every vector,
 *   inner product and operator application in FP64 -- with the
 *   preconditioner K^-1 u = |u| RAS(u / |u|) evaluated in FP32 arithmetic on
 *   inner_prec storage.
 * RELIABLE: BiCGStab itself runs in FP32 (FP32 vectors, FP32 operator, RAS
 *   on inner_prec storage, FP64 sums of FP32 partials); the solution is held
 *   in FP64 and every time the FP32 residual falls below delta times its
 *   largest value since the last refresh, the correction is added to the FP64
 *   solution and the residual is recomputed as b - M x in FP64 (a "reliable
 *   update").  This trades FP64 work, slow on GB300, for FP32 work.
 * NESTED (the paper's three levels, Sec. 2): FP64 flexible BiCGStab whose
 *   preconditioner is an FP32 BiCGStab solve of M z = u / |u| that is itself
 *   right-preconditioned by RAS (MR block solves), run until its residual
 *   falls below inner_tol or for inner_iters steps.
 * With precond NONE, FLEXIBLE is plain FP64 BiCGStab, RELIABLE is FP32
 * BiCGStab with FP64 reliable updates and NESTED's inner FP32 BiCGStab runs
 * without RAS.  even_odd = 1 runs any of the three on the even-site Schur
 * complement (with or without RAS), as the paper's solvers do (Sec. 2).
 * The true residual |b - M x| / |b| reported and tested against tol is FP64
 * in all of them, on the full lattice.  An even-odd RELIABLE solve leaves
 * the convergence test to that full residual: its half-lattice solve stops,
 * without a last FP64 refresh, once the low-precision recurrence residual is
 * below 0.5 tol (the environment variable WC_EO_DEFER_MARGIN sets another
 * factor; 0 keeps the refresh), and resumes, confirming in FP64 itself, if
 * the full residual is then above tol. */
typedef enum { WC_SOLVER_FLEXIBLE = 0, WC_SOLVER_RELIABLE = 1, WC_SOLVER_NESTED = 2 } wc_solver_kind;

typedef struct {
    double tol;            /* stop when |b - M x| / |b| <= tol (true residual) */
    int max_iter;          /* total outer iterations over all restarts */
    int max_restarts;      /* restarts after a failed true-residual check */
    wc_precond precond;    /* NONE: plain FP64 BiCGStab; RAS: mixed precision */
    wc_prec inner_prec;    /* storage of the RAS preconditioner: WC_F32 or WC_F16 */
    wc_ras_params ras;
    wc_solver_kind solver; /* FLEXIBLE, RELIABLE or NESTED */
    double delta;          /* RELIABLE refresh threshold, 0 < delta < 1 (0: 0.01) */
    double inner_tol;      /* NESTED inner relative tolerance, 0 < inner_tol < 1 (0: 0.01) */
    int inner_iters;       /* NESTED inner step limit, >= 0 (0: 100) */
    wc_prec krylov_prec;   /* RELIABLE and NESTED: storage of the low-precision BiCGStab vectors and
                              of their operator: WC_F16 (values + one FP32 scale per site, FP32
                              arithmetic; RAS then also on FP16 storage) or WC_F32 (also for
                              WC_F64, the zero value); the accumulated FP32 correction and
                              every FP64 quantity are unaffected */
    int even_odd;          /* 1: solve the even-site Schur complement (see wc_apply_schur) and
                              reconstruct the odd sites; needs even extents; any solver kind;
                              with precond RAS the preconditioner is the full lattice's RAS on
                              the even vector extended by zeros, restricted to the even sites
                              (Sec. 2: the inner solver is even-odd and RAS preconditioned);
                              0: full lattice */
} wc_solve_params;

typedef struct {
    int iters;             /* BiCGStab iterations performed */
    int restarts;          /* restarts after a failed true-residual check (the resume of an even-odd
                              RELIABLE half solve whose deferred confirmation failed counts as one) */
    double true_rel_resid; /* |b - M x| / |b| recomputed in FP64 at the end */
    double seconds;        /* wall time of the solve on the host clock */
    wc_status status;
} wc_solve_info;

/* ---- lattices ------------------------------------------------------ */

/* Create a lattice of extent dims = {Lx, Ly, Lz, Lt} (each >= 2) with time
 * boundary factor t_bc (+1 periodic, -1 antiperiodic) whose kernels run on
 * cuda_stream (a cudaStream_t, or NULL).  Allocates the device workspace. */
wc_status wc_create_lattice(const int dims[4], int t_bc, void *cuda_stream, wc_lattice *out);
wc_status wc_destroy_lattice(wc_lattice lat);
/* Switch the stream later kernels of this lattice are queued on. */
wc_status wc_set_stream(wc_lattice lat, void *cuda_stream);

/* Arithmetic of every later FP64 operator application on this lattice:
 * wc_apply_M / _Mdag / _hop and wc_apply_schur on FP64 fields, and the FP64
 * operator steps inside the solvers (FP64 BiCGStab iterations, reliable
 * updates, true residuals, even-odd source preparation and
 * reconstruction).  WC_ARITH_F64 (the default): FP64 arithmetic.
 * WC_ARITH_DF32: double-FP32 arithmetic -- each value is carried as the
 * unevaluated sum of two floats (about 47 significant bits) and the
 * operations run on the FP32 pipes, which on GB300 are 64 times faster than
 * its FP64 pipe.  Storage stays FP64.  Results agree with FP64 arithmetic to
 * ~1e-14 relative to the largest input; inputs with |x| < 2^-103 keep only
 * 24 bits and |x| < 2^-126 reads as zero.  BLAS-1 steps and the force stay
 * in FP64.  Returns WC_ERR_ARG for any other value.  Host-side setting
 * only; graphs captured earlier (wc_solve_batch) keep the arithmetic they
 * were captured with. */
wc_status wc_set_fp64_arith(wc_lattice lat, int arith);

/* Load the gauge field U (canonical layout, data = device or host pointer).
 * Links are stored as their first two rows (12 reals; paper Sec. 2,
 * "SU(3)-reconstruction") in FP64, FP32 and FP16; the third row is rebuilt
 * as the complex conjugate of the cross product of the first two, so U must
 * be special unitary to working precision.  Invalidates the clover term. */
wc_status wc_load_gauge(wc_lattice lat, const double *data);

/* Build A = 1 + T from the loaded gauge field on the GPU (FP64 arithmetic)
 * and store it as two Hermitian 6x6 blocks per site (the chiral basis makes
 * T block diagonal in spin pairs {0,1} and {2,3}): 6 real diagonal + 15
 * complex lower entries each, 72 reals per site, in FP64, FP32 and FP16.
 * kappa is also the hopping parameter used by every later apply. */
wc_status wc_load_clover(wc_lattice lat, double csw, double kappa);

/* ---- fields --------------------------------------------------------- */

/* A colour-spinor field owned by the library, stored in prec:
 * FP64 / FP32 values, or FP16 values with one FP32 scale per site. */
wc_status wc_field_create(wc_lattice lat, wc_prec prec, wc_field *out);
wc_status wc_field_destroy(wc_field f);
/* canonical complex128 (device or host) -> field (rounded to nearest).
 * Host data goes through one copy-engine transfer into a device staging
 * buffer (reading host memory from the conversion kernel itself measured
 * 2.6x slower per import + export on GB300).  Device data: asynchronous on
 * the lattice stream; host data: blocking. */
wc_status wc_field_import(wc_field f, const double *data);
/* field -> canonical complex128 (device or host).  Same rules. */
wc_status wc_field_export(wc_field f, double *data);
/* The same with canonical complex64 data (float pairs, psi[V][4][3]), device
 * or host: half the bytes of complex128 across the host link, for callers
 * whose data is single precision.  Import widens (FP64 field) or rounds
 * (FP16 field); export of an FP64 field rounds to nearest FP32.  Same
 * synchronisation and error rules as the complex128 calls. */
wc_status wc_field_import_f32(wc_field f, const float *data);
wc_status wc_field_export_f32(wc_field f, float *data);
/* Asynchronous import / export for pipelines that stream host data through
 * the library: data (canonical complex128, or complex64 when complex64 is
 * nonzero) must be device memory or page-locked host memory (WC_ERR_ARG
 * otherwise, nothing queued); the call returns once the work is queued.
 * Host-to-device copies run on a second stream of the lattice and
 * device-to-host copies on a third one (from two alternating staging
 * buffers), so the copy of the next step's input and the copy out of the
 * current step's result overlap each other and the kernels; the import and
 * export kernels and everything between them stay in the lattice stream's
 * order.  The caller keeps imported host data unchanged and reads exported
 * host data only after wc_sync(lat).  The lattice holds three extra
 * canonical-size device buffers from the first asynchronous call with host
 * data until it is destroyed. */
wc_status wc_field_import_async(wc_field f, const void *data, int complex64);
wc_status wc_field_export_async(wc_field f, void *data, int complex64);
/* Block until every kernel and copy queued on the lattice (all three
 * streams) has finished. */
wc_status wc_sync(wc_lattice lat);
/* dst = src converted to dst's precision, times scale (any precisions). */
wc_status wc_field_copy(wc_field dst, wc_field src, double scale);

/* ---- operator --------------------------------------------------------- */

/* out = M in (paper Sec. 2-3: the Wilson-Clover matrix multiplication).
 * out and in: distinct fields of the same lattice and precision; the
 * arithmetic is FP64 for FP64 fields and FP32 otherwise.  Asynchronous. */
wc_status wc_apply_M(wc_lattice lat, wc_field out, wc_field in);
/* out = M^+ in = gamma5 M gamma5 in.  Same rules as wc_apply_M. */
wc_status wc_apply_Mdag(wc_lattice lat, wc_field out, wc_field in);
/* out = H in (hopping term only, no clover, no kappa).  Same rules. */
wc_status wc_apply_hop(wc_lattice lat, wc_field out, wc_field in);

/* Multi-right-hand-side operator for the sources of a propagator (Sec. 2:
 * the solver is applied per source; the sources share U and A):
 * outs[r] = M ins[r] (dagger = 0) or M^+ ins[r] (dagger != 0), r < n,
 * 1 <= n <= 16, all FP32 fields of lat.  One launch reads the links and the
 * clover term once per site for all n fields: 192 + 480/n bytes per site and
 * field instead of 672.  Every out distinct from every other out and every
 * in.  Asynchronous on the lattice stream; WC_ERR_ARG for other precisions
 * or sizes, before any launch. */
wc_status wc_apply_multi(wc_lattice lat, int n, wc_field *outs, wc_field *ins, int dagger);

/* Even-odd preconditioned operator (the matrix the paper's CCS-QCD solver
 * works on, Sec. 2).  With sites ordered by parity (even: x+y+z+t even),
 * M = [[A_ee, -k H_eo], [-k H_oe, A_oo]] and its Schur complement on the
 * even sites is  M^ = A_ee - k^2 H_eo A_oo^-1 H_oe.  out (even sites) =
 * M^ in (even sites), or M^+ = gamma5 M^ gamma5 with dagger != 0; the odd
 * sites of in are ignored and those of out set to zero.  A^-1 is built on
 * the first call (blocking; WC_ERR_BREAKDOWN if a clover block is
 * singular).  All four extents must be even (WC_ERR_ARG otherwise: a hop
 * across the boundary of an odd extent would keep the parity).  Fields:
 * distinct, same lattice and
 * precision.  Blocking. */
wc_status wc_apply_schur(wc_lattice lat, wc_field out, wc_field in, int dagger);

/* Launch shape of the operator kernels.  The site-to-thread mapping
 * (lexicographic or 4-D tiles), CTA size and register cap of wc_apply_M /
 * wc_apply_Mdag / wc_apply_hop are chosen per lattice extent, precision and
 * kind (0 M, 1 M^+, 2 H) by timing the candidates on the first apply (that
 * first call blocks; not done while the stream is being captured, where the
 * default shape is used).  force_index >= 0 pins candidate #force_index
 * (0..23; WC_ERR_ARG if its tile does not divide the lattice or it is a
 * register-capped shape with FP64); -1 only reports.  shape_out receives
 * {threads per CTA, tile x, y, z, t (all 0: lexicographic), flags}, flags
 * = register cap (0 none, 1: 64, 2: 85 registers per thread) + 4 if the
 * launch is persistent (grid = resident CTAs, each CTA walking the site
 * blocks) + 16 if it is a programmatic dependent launch (the kernel may
 * start while the previous kernel of the stream drains, prefetches its
 * links and clover into L2, then waits for that kernel; plain launch while
 * the stream is being captured); all -1 if nothing was chosen yet.  The choice is shared by lattices of equal
 * extent in the process.  With prec = WC_F64 on a lattice in WC_ARITH_DF32
 * mode (wc_set_fp64_arith) the call reports or pins the double-FP32
 * operator's shape, which is chosen separately from the FP64 one. */
wc_status wc_apply_shape(wc_lattice lat, wc_prec prec, int kind, int force_index, int shape_out[6]);

/* outs[r] (even sites) = M^ ins[r] (even sites), M^ = A_ee - kappa^2 H_eo
 * A_oo^-1 H_oe (M^+ with dagger = 1), odd sites of outs[r] set to zero, for
 * 1 <= n <= 16 full-lattice FP32 or FP16 fields of one precision (all
 * extents even).  One odd-site and one even-site pass serve all n fields:
 * the links, A and A^-1 of a site are read once for every field (the
 * right-hand sides of a propagator share them; paper Sec. 2: the solvers
 * act on the even-odd preconditioned matrix).  outs must be distinct from
 * each other and from ins.  Blocking. */
wc_status wc_apply_schur_multi(wc_lattice lat, int n, wc_field *outs, wc_field *ins, int dagger);

/* ---- fused BLAS-1 (FP64 accumulation; blocking) ---------------------- */

/* re_im[0] + i re_im[1] = <a, b> = sum conj(a) b over all sites */
wc_status wc_dot(wc_lattice lat, wc_field a, wc_field b, double *re_im);
wc_status wc_norm2(wc_lattice lat, wc_field a, double *out);
/* y += (a[0] + i a[1]) x, then *norm2_y = |y|^2 (norm2_y may be NULL). */
wc_status wc_axpy_norm(wc_lattice lat, const double *a, wc_field x, wc_field y,
                       double *norm2_y);

/* ---- allocation-free variant ------------------------------------------ */

/* out[0] + i out[1] = <a, b> = sum_i conj(a_i) b_i over n complex128 values.
 * The paper has no counterpart: this is wc_dot for callers that must not
 * allocate device memory (a framework that owns the memory pool, a
 * latency-critical path where cudaMalloc would synchronise the device).
 * a, b: device pointers to n interleaved (re, im) doubles, 16-byte aligned
 * (as every complex128 array allocation is); out: device pointer to 2
 * doubles, 8-byte aligned, written on the given CUDA stream (NULL = legacy
 * default stream); the call returns without waiting for the result.
 * WC_ERR_ARG, before any CUDA call, for NULL or misaligned pointers (a and
 * b may be NULL when n = 0: the result is then 0), n < 0 or n above the
 * maximum.
 * It allocates nothing: its scratch is a fixed 32 KiB array in the
 * library's device memory, held by every GPU that loads the library until
 * the process exits.  n may be at most 8,388,608 (WC_ERR_ARG beyond).
 * When that array comes to exist: with CUDA's lazy module loading (the
 * default since CUDA 12.2) the library code holding it is loaded into a
 * context on first use, and the first call of this function on a device is
 * such a use -- that first call may allocate device memory for the module
 * and may synchronise.  A caller that must not allocate at all makes one
 * call during its own set-up (or runs with CUDA_MODULE_LOADING=EAGER, where
 * the array exists from context creation); every later call on that device
 * and context allocates nothing.  The first call on a device also looks up
 * the array's device address (with that device current) and must come
 * before any stream capture that includes this call.  Every call shares the
 * one array, so calls whose kernels overlap on the GPU (e.g. on two streams)
 * race and give wrong sums; calls ordered on one stream are safe.
 * Deterministic for fixed n. */
wc_status wc_dot_noalloc(const double *a, const double *b, long long n, double *out, void *cuda_stream);

/* ---- domain decomposition: the overlapped MULT ------------------------ */

/* The paper's multi-node hopping multiplication overlaps the halo exchange
 * with computation (Sec. 2.2, communication-computation overlapping): a
 * pre-communication step prepares the face data, the interior sites are
 * computed while the messages travel, and the surface sites once they have
 * arrived.  These calls provide the three steps for one sub-domain; moving
 * the buffers between sub-domains (NCCL, MPI, device copies) is the
 * caller's.
 *
 * wc_create_subdomain: a lattice holding the sites [offset, offset +
 * local_dims) of a lattice of extents global_dims (every extent >= 2,
 * offset[mu] + local_dims[mu] <= global_dims[mu]).  Direction mu is cut when
 * local_dims[mu] < global_dims[mu] (at least one must be); along uncut
 * directions the sub-domain is periodic by itself.  Neighbouring
 * sub-domains across a cut face must have the same extents in the other
 * three directions.  t_bc applies to hops across the global time boundary.
 * On a sub-domain, wc_load_gauge takes the gauge field (canonical layout)
 * of the sites [offset - c, offset + local_dims + c) with c[mu] = 1 along
 * cut directions and 0 otherwise (periodic in the global lattice): the
 * clover leaves of a face site reach one site into the neighbour, so
 * wc_load_clover builds the clover term of the sub-domain exactly; the
 * extended field is kept for later clover rebuilds.  Fields, imports,
 * exports, copies and the BLAS-1 calls work on sub-domains (inner products
 * are then partial sums of the sub-domain's sites); the whole-lattice
 * operator, RAS and the solvers return WC_ERR_ARG.
 *
 * Face buffers: one per cut direction and side, wc_halo_bytes(mu) bytes
 * (12 FP32 reals per face site; 0 for uncut directions), 16-byte aligned
 * device memory.  send[2 mu] goes to the lower neighbour along mu and
 * arrives there as recv[2 mu + 1]; send[2 mu + 1] goes to the upper
 * neighbour and arrives as its recv[2 mu].  Entries of uncut directions are
 * ignored (may be NULL).  FP32 fields; dagger = 1 for M^+ (pack and surface
 * must use the same dagger).
 *
 * wc_halo_pack: fills the send buffers from in (lower face:
 * (1 -+ gamma_mu) in projected to two spinors; upper face: U_mu^+ times the
 * other projection).  wc_apply_interior: out = M in (M^+ in) on every site
 * that has no hop across a cut face; it needs no buffer and may run while
 * the buffers travel.  wc_apply_surface: out on the remaining sites, from in
 * and the received buffers.  The three calls queue kernels on the lattice
 * stream (wc_set_stream may switch it between calls to overlap them); the
 * two apply calls together give exactly the whole-lattice operator (bit for
 * bit with wc_apply_M / wc_apply_Mdag of the undivided lattice in FP32). */
wc_status wc_create_subdomain(const int local_dims[4], const int global_dims[4], const int offset[4], int t_bc,
                              void *cuda_stream, wc_lattice *out);
wc_status wc_halo_bytes(wc_lattice lat, int mu, long long *bytes);
wc_status wc_halo_pack(wc_lattice lat, wc_field in, int dagger, void *const send[8]);
wc_status wc_apply_interior(wc_lattice lat, wc_field out, wc_field in, int dagger);
wc_status wc_apply_surface(wc_lattice lat, wc_field out, wc_field in, int dagger, const void *const recv[8]);

/* ---- preconditioner and solvers --------------------------------------- */

/* out = RAS(in) (see wc_ras_params).  FP32 arithmetic on FP32 or FP16
 * fields of the same precision.  Asynchronous. */
wc_status wc_ras_precond(wc_lattice lat, wc_field out, wc_field in, const wc_ras_params *p);

/* out = the RAS on block Schur complements (see wc_ras_params, schur = 1;
 * p->schur itself is ignored) of the even sites of in, M^ (dagger = 0) or
 * M^+ (dagger = 1): FP32 arithmetic on FP32 or FP16 full-lattice fields of
 * one precision; the odd sites of in are ignored and those of out set to
 * zero.  All extents even.  Builds A^-1 on first use.  Asynchronous on the
 * lattice stream (two half-lattice temporaries per precision are kept by
 * the lattice). */
wc_status wc_ras_schur(wc_lattice lat, wc_field out, wc_field in, const wc_ras_params *p, int dagger);

/* Solve M x = b.  x (FP64) holds the initial guess on entry and the
 * solution on return; b is FP64.  Blocking; fills *info. */
wc_status wc_solve_bicgstab(wc_lattice lat, wc_field x, wc_field b, const wc_solve_params *p,
                            wc_solve_info *info);

/* Solve M_i x_i = b_i for n right-hand sides on possibly different
 * lattices (each x_i, b_i FP64 fields of lats[i]; x_i distinct) with the
 * parameters p.  All BiCGStab iterations of all right-hand sides run inside
 * one CUDA graph launch (a device-side loop with one convergence mask per
 * right-hand side; right-hand sides proceed concurrently), queued on
 * internal streams; the true residual of each is then recomputed in FP64 and
 * any that misses tol is continued by the host-driven solver (FLEXIBLE and
 * RELIABLE; NESTED is WC_ERR_ARG here).  With even_odd every right-hand side
 * is first reduced to its even-site Schur system (all extents even), the
 * Schur systems are solved in the graph, and each solution is completed on
 * the odd sites and checked on the full system.  Reliable update with FP32
 * Krylov vectors and without a preconditioner on even-odd systems runs the
 * right-hand sides of one lattice in lockstep groups of up to 16 (each
 * step's Schur applications are one multi-right-hand-side launch for the
 * group; a stopped member skips its kernels); the environment variable
 * WC_BATCH_LOCKSTEP=0 gives every right-hand side its own branch instead,
 * WC_BATCH_LOCKSTEP=1 groups FP16 Krylov vectors too.  An even-odd
 * RELIABLE batch leaves each right-hand side's convergence test to its full
 * residual, as a single even-odd solve does (see wc_solve_params;
 * WC_EO_DEFER_MARGIN).  A zero initial guess skips the
 * start's operator application.  Each lattice keeps the solver states and
 * work fields of its largest batch (and, with even_odd, five FP64
 * half-lattice fields per right-hand side) for the next batch, until
 * wc_destroy_lattice; calls on one lattice must not overlap.  With
 * p->precond = WC_PRECOND_RAS and p->ras.block = {0,0,0,0} the RAS block
 * shape of each lattice is chosen by wc_ras_autotune.  Blocking; fills
 * infos[0..n-1] (seconds: wall time of the whole batch); returns the first
 * non-OK status of any right-hand side. */
wc_status wc_solve_batch(int n, const wc_lattice *lats, wc_field *xs, wc_field *bs,
                         const wc_solve_params *p, wc_solve_info *infos);

/* Choose the RAS block shape (core extents from {2, 4, 8}, 128 to 512
 * sites, fitting one CTA and the lattice) that reduces the residual of
 * M x = b fastest in a short timed trial solve with p's overlap, mr_iters
 * and inner precision; the result is cached per lattice extent for the
 * process.  b: an FP64 field of lat.  Blocking; writes *out. */
wc_status wc_ras_autotune(wc_lattice lat, wc_field b, const wc_solve_params *p, wc_ras_params *out);

/* S = phi^+ (M^+ M)^-1 phi and its force F = dS/dU per link as traceless
 * anti-Hermitian 3x3 matrices (canonical force layout, data = device or
 * host), from two FP64 solves M^+ Y = phi, M X = Y.  Blocking. */
wc_status wc_action_force(wc_lattice lat, wc_field phi, double *S_out, double *force,
                          const wc_solve_params *p);

/* out = scale * F U for every link (3x3 complex products, canonical force
 * and gauge layouts [V][4][3][3]; all three device pointers; out may alias
 * neither input).  With F from wc_action_force and scale = -dL/dS this is
 * the gradient of a loss L(S) with respect to U on the tangent space of
 * SU(3): for U -> exp(eps X) U, dS/deps = tr(X F) = Re sum tr(G^+ X U) with
 * G = -F U.  The paper has no gradient; this is the step that turns the
 * force into the autograd gradient of the binding.  Asynchronous on the
 * lattice stream. */
wc_status wc_force_times_links(wc_lattice lat, const double *force, const double *U, double scale, double *out);

/* Diagnostics of the checked build (the library compiled with -DWC_CHECKED,
 * build.py --checked): every site, neighbour, block-local and shared-memory
 * index the operator, even-odd, RAS and multi-RHS kernels compute is tested
 * against its array's extent; an index out of range is counted and replaced
 * by 0 (no fault: the result is wrong and the count says so), and the RAS
 * kernels fill their shared memory with NaN before staging it.  *count =
 * the number of out-of-range indices since the library was loaded (waits
 * for the device first).  WC_ERR_STATE in the normal build.  The paper has
 * no counterpart: this stands in for a memory checker. */
wc_status wc_checked_violations(unsigned long long *count);

const char *wc_last_error(wc_lattice lat);

#ifdef __cplusplus
}
#endif
#endif
