/*
 * ok.h -- C ABI of the GB300 (sm_103a) library for the Oktay-Kronfeld (OK) action Dirac operator
 * in the precalculated-W form of Jang et al., "Optimization of the Oktay-Kronfeld Action Conjugate
 * Gradient Inverter" (PoS LATTICE2013, arXiv:1311.5029), and its BiCGStab inverter.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Lattice: dims = {X, Y, Z, T}; sites are ordered lexicographically with x fastest,
 *   site = x + X * (y + Y * (z + Z * t)).  Direction mu = 0, 1, 2, 3 is x, y, z, t (the paper's
 *   mu = 4 is t).  bc[mu] = +1 periodic, -1 antiperiodic boundary for the fermion field; the
 *   gauge field is always periodic.
 * Gauge links: [T][Z][Y][X][mu=4][3][3] complex (row-major 3x3), interleaved re/im, complex128
 *   (OK_F64) or complex64 (OK_F32).
 * Fermion fields: [T][Z][Y][X][spin=4][colour=3] complex, spin outer.  Spin basis: the Dirac
 *   representation of the paper's Ref. [EKM] as fixed by the block forms of W (Sec. 2.2):
 *   gamma_4 = diag(1, 1, -1, -1), gamma_i = [[0, sigma_i], [sigma_i, 0]].
 * Pointers: every array argument is a DEVICE pointer owned by the caller (for example
 *   torch.Tensor.data_ptr()), unless stated otherwise.  The library never frees caller memory.
 *   `stream` is a cudaStream_t (NULL = the legacy default stream); all work is enqueued on it.
 * Errors: every int-returning call returns OK_SUCCESS (0) or a negative OK_E* code and never
 *   throws across the ABI.  OK_ECUDA means a CUDA runtime call failed; the CUDA error is
 *   available from ok_last_cuda_error().  On any error no output is guaranteed.
 * Threads: a W handle is immutable after ok_precompute_W; concurrent applies and solves with
 *   the same handle on different streams are safe (each solve allocates its own workspace).
 */
#ifndef OK_GB300_H
#define OK_GB300_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status codes */
#define OK_SUCCESS      0
#define OK_EINVAL      -1   /* invalid argument (null pointer, bad size, missing precision) */
#define OK_ENOMEM      -2   /* device or host allocation failed */
#define OK_ECUDA       -3   /* a CUDA runtime call or kernel launch failed */
#define OK_ENOCONV     -4   /* solver hit maxiter (or max restarts) before reaching tol */
#define OK_EBREAKDOWN  -5   /* BiCGStab breakdown that restarts could not cure */
#define OK_ENONFINITE  -6   /* a non-finite value appeared in a solver scalar */
#define OK_EINTERNAL   -7   /* internal consistency check failed */

/* ------------------------------------------------------------------ types */
typedef struct {
    int dims[4];   /* X, Y, Z, T; each >= 1, product <= OK_MAX_SITES */
    int bc[4];     /* +1 periodic, -1 antiperiodic (fermion boundary phase) */
} ok_lattice;

#define OK_MAX_SITES (1 << 27)

/* Precision of an application of M: OK_F64 (complex128 fields, FP64-accurate W), OK_F32 (complex64
 * fields, FP32 W), OK_F32_W16 (complex64 fields and FP32 arithmetic with the FP16 copy of W) or
 * OK_F16_TC (several right-hand sides at once on the tensor cores: complex64 fields and the
 * OK_W_F16_TC copy of W enter the products as FP16, which accumulate in FP32) or OK_F32_OTF
 * (complex64 fields; no stored W: each W matrix of Eqs. shifted_W_first .. shifted_W_last is
 * rebuilt in FP32 from the links and clover fields of an OK_W_OTF handle where a hop needs it). */
typedef enum { OK_F64 = 0, OK_F32 = 1, OK_F32_W16 = 2, OK_F16_TC = 3, OK_F32_OTF = 4 } ok_prec;

/* Which stored copies a W handle carries (bit mask for ok_precompute_W).  OK_W_DF64 keeps FP64
 * accuracy as double-float pairs (hi + lo, two floats, about 48 significand bits): FP64 applications
 * and residuals on such a handle run on the FP32 pipes, which GB300 executes 58 times faster than its
 * FP64 pipe, with errors of about 1e-14 relative; it takes twice the memory of OK_W_F64.  Without
 * OK_W_F64 (and OK_W_F16_TC) in the mask, the clover fields and W themselves are computed in
 * double-float arithmetic on the FP32 pipes (about 1e-13 relative) instead of FP64.  When a
 * handle has both, ok_apply_M with OK_F64 uses the native OK_W_F64 copy (FP64 rounding exactly),
 * and the true residuals (ok_true_residual and those inside the solvers) use the double-float copy,
 * the faster of the two on GB300. */
#define OK_W_F64 1
#define OK_W_F32 2
#define OK_W_DF64 4
#define OK_W_F16 8   /* half-precision copy (relative rounding 2^-11) for the low-precision iteration */
#define OK_W_LINKS 16 /* also keep an FP32 copy of the links (for the learned preconditioner, ok_net_*) */
/* FP16 copy for the tensor-core multi-right-hand-side apply (OK_F16_TC): per site, the operator's
 * hops written as 6x6 complex blocks acting on the spin projections (u + l) / sqrt 2 and
 * (u - l) / sqrt 2 of the neighbour spinor, each entry rounded once from FP64 (relative 2^-11);
 * 3216 bytes per site, in a site-major layout. */
#define OK_W_F16_TC 32
/* Inputs of the on-the-fly apply (OK_F32_OTF) instead of a stored W: FP32 copies of the links
 * (288 bytes per site) and of the clover fields E_k, B_k (432 bytes per site), site-blocked. */
#define OK_W_OTF 64

/* Coefficients of the tree-level, tadpole-improved OK action (Sec. 1; they enter the W formulas,
 * Eqs. shifted_W_first .. shifted_W_last).  u0 <= 0: u0 is computed from the mean plaquette of
 * the links.  kappa <= 0: 1/(2 kappa) = am0 + 1 + 3 r_s zeta + 18 c4. */
typedef struct {
    double u0, am0, kappa;
    double zeta, r_s, c_B, c_E, c_EE, c1, c2, c3, c4, c5;
} ok_coeffs;

typedef struct {
    int iters;             /* BiCGStab iterations (each = two applications of M) */
    int restarts;          /* restarts from the true residual (breakdown or stagnation) */
    int reliable_updates;  /* FP64 residual recomputations of the mixed-precision solver */
    int fp64_applies;      /* FP64 applications of M, including true-residual checks */
    double true_relres;    /* |b - M x| / |b| recomputed in FP64 at exit */
    double iter_relres;    /* iterated residual norm / |b| at exit */
    double time_ms;        /* host wall time of the call */
} ok_solve_info;

#define OK_SOLVE_AUTO   0  /* mixed if the handle has OK_W_F32 and OK_W_F64, else plain FP64 */
#define OK_SOLVE_F64    1  /* plain FP64 BiCGStab (needs OK_W_F64) */
#define OK_SOLVE_MIXED  2  /* FP32 BiCGStab with FP64 reliable updates (needs both precisions) */
#define OK_SOLVE_MIXED16 3 /* as OK_SOLVE_MIXED with the FP16 W copy in the FP32 iteration (OK_W_F16) */
#define OK_SOLVE_MIXED_TC 4 /* ok_bicgstab_multi: as OK_SOLVE_MIXED with the tensor-core apply (OK_W_F16_TC) */
/* Flag, or-ed into OK_SOLVE_MIXED, OK_SOLVE_MIXED16 or OK_SOLVE_MIXED_TC: outer FP64 defect correction.
 * Each FP64 recomputation of r = b - M x (when the low-precision residual has dropped by delta)
 * starts a fresh low-precision BiCGStab on the correction equation M e = r (rhat = p = r), whose
 * increments accumulate into the FP64 x, instead of continuing the previous search direction
 * (the reliable update).  info->reliable_updates counts the corrections. */
#define OK_SOLVE_DEFECT 8

typedef struct {
    double tol;          /* stop when |b - M x| / |b| < tol (true FP64 residual) */
    int maxiter;         /* total BiCGStab iterations allowed */
    int mode;            /* OK_SOLVE_* */
    double delta;        /* mixed mode: reliable update when |r| < delta * max |r| since last */
    int max_restarts;    /* restarts from the true residual allowed */
    int check_every;     /* iterations enqueued between host convergence checks (>= 1) */
} ok_solve_params;

typedef struct ok_W ok_W;  /* opaque, library-owned precalculation-matrix set */
typedef struct ok_net ok_net;  /* opaque, library-owned learned preconditioner (see ok_net_create) */

/* ------------------------------------------------------------------ entry points */

/* Precompute the W matrices (Sec. 2.2, "Precalculation"; Eqs. shifted_W_first ..
 * shifted_W_last) for one gauge configuration: mean plaquette and u0, clover fields E_i and B_i,
 * and the forward set W^0_x, W^+_{mu,x}, W^{++}_{ii,x}, W^{++}_{ij,x}, W^{+-}_{ij,x} (i < j) per
 * site, unshifted, in a private site-blocked layout.  The backward matrices are not stored: they
 * follow from the forward ones by Eqs. conjugate and opp_diag_pre_mat.  Arithmetic is FP64;
 * W_precs selects the stored copies (at least one of OK_W_F64, OK_W_F32, OK_W_DF64, OK_W_F16,
 * OK_W_F16_TC),
 * plus OK_W_LINKS to keep an FP32 copy of the links in the handle.
 *   links: device [T][Z][Y][X][4][3][3] complex in links_prec; not retained after the call.
 *   W_out: receives a new handle owned by the caller, released with ok_free_W.
 * Synchronises `stream` before returning (u0 is read back).  Errors: OK_EINVAL (null pointer,
 * dims out of range, bad bc or mask), OK_ENOMEM, OK_ECUDA. */
int ok_precompute_W(const ok_lattice* lat, const void* links, ok_prec links_prec,
                    const ok_coeffs* coeffs, int W_precs, void* stream, ok_W** W_out);

/* Release a handle from ok_precompute_W (NULL is ignored).  Its arrays return to the device's
 * stream-ordered memory pool (ordered on the legacy default stream); call it only after work using
 * the handle has completed.  ok_precompute_W lets that pool keep up to 8 GiB of released memory
 * (if the pool's release threshold was still 0), so the next handle reuses it without mapping. */
void ok_free_W(ok_W* W);

/* u0 used by the handle (given or computed from the mean plaquette); NaN if W is NULL. */
double ok_W_u0(const ok_W* W);

/* Mean plaquette (1/3) Re tr U_plaq over all sites and six planes; its fourth root is u0. */
double ok_W_plaquette(const ok_W* W);

/* Lattice, stored-precision mask and device bytes held by the handle.  Any output may be NULL. */
int ok_W_info(const ok_W* W, ok_lattice* lat, int* W_precs, size_t* bytes);

/* out = M psi (Eq. dslash with M in the form of Eq. minFlopForm: the on-site W^0, the 8 nearest,
 * 6 next-to-nearest straight and 12 diagonal neighbours), using the handle's stored matrices of
 * precision `prec`, arithmetic in that precision (OK_F32_W16: complex64 fields, FP32 arithmetic,
 * matrices read from the OK_W_F16 copy and widened to FP32; OK_F32_OTF: complex64 fields, no stored
 * matrices: each W group of a hop is rebuilt in FP32 from the OK_W_OTF links and clover fields, at
 * x for a forward hop and at the neighbour for a backward one, Sec. 2.2's precalculation undone).
 *   psi, out: device [V][4][3] complex in `prec`; out must not overlap psi.
 * Errors: OK_EINVAL (null, aliasing, handle lacks `prec`), OK_ECUDA.  Asynchronous. */
int ok_apply_M(const ok_W* W, ok_prec prec, const void* psi, void* out, void* stream);

/* Solve M x = src by BiCGStab (the paper's bi-stabilized CG, Sec. 2.3) with default parameters
 * (OK_SOLVE_AUTO, delta 1e-3, 5 restarts, host check every 4 iterations).  src, x: device [V][4][3] complex128; x holds the
 * initial guess on entry and the solution on exit.  info (host, may be NULL) is filled on
 * success and on OK_ENOCONV / OK_EBREAKDOWN.  Synchronises `stream`. */
int ok_bicgstab(const ok_W* W, const void* src, void* x, double tol, int maxiter,
                ok_solve_info* info, void* stream);

/* As ok_bicgstab with explicit parameters (params on the host). */
int ok_bicgstab_ex(const ok_W* W, const void* src, void* x, const ok_solve_params* params,
                   ok_solve_info* info, void* stream);

/* Several right-hand sides at once (the 12 spin-colour sources of a propagator; the paper's
 * method solves one source at a time, Sec. 2.3).
 *
 * ok_apply_M_multi: out_k = M psi_k for k < nrhs in one launch.  prec OK_F32 (FP32 W) or
 * OK_F32_W16 (FP16 W): FP32 fields and arithmetic, every W matrix a thread loads applied to several
 * right-hand sides (the count chosen by ok_autotune).  prec OK_F16_TC (needs OK_W_F16_TC, nrhs <= 16):
 * on the tensor cores; per site and hop the right-hand sides times the hop's 6x6 spin-projected
 * blocks is a complex GEMM (warp-level mma.sync m16n8k16, FP16 operands, FP32 accumulation).  Each
 * right-hand side enters as FP16 scaled by a power of two that puts its largest component below
 * 2^14, so fields of any magnitude keep FP16's relative precision (components below 2^-24 of the
 * largest flush to zero); the result is FP32.  This entry converts to and from the private field
 * layout of the tensor-core kernel around the launch, in stream-ordered scratch.
 *   psi, out: device [nrhs][V][4][3] complex64, 16-byte aligned, not overlapping.
 * Errors: OK_EINVAL (null, nrhs < 1 or > 16 for OK_F16_TC, overlap, misalignment, copy missing),
 * OK_ENOMEM, OK_ECUDA.  Asynchronous.
 *
 * ok_bicgstab_multi: solves M x_k = src_k for k < nrhs with the mixed-precision method of
 * ok_bicgstab_ex run for all systems in lockstep: FP32 iteration on the FP32 (OK_SOLVE_MIXED) or
 * FP16 (OK_SOLVE_MIXED16) copy of W, or on the tensor cores (OK_SOLVE_MIXED_TC: FP32 iteration
 * vectors in the tensor-core kernel's layout, FP16 copies of the applied vectors scaled per system
 * from its residual norm, nrhs <= 16), with FP64 reliable updates, every system to its own true
 * FP64 residual below params->tol.  OK_SOLVE_AUTO picks OK_SOLVE_MIXED_TC when the handle has
 * OK_W_F16_TC and nrhs <= 16, else OK_SOLVE_MIXED16 when it has OK_W_F16, else OK_SOLVE_MIXED.  One
 * iteration is five launches for all systems, captured once into a CUDA graph and replayed
 * params->check_every iterations at a time.
 *   src, x: device [nrhs][V][4][3] complex128 (x: initial guess in, solution out), 1 <= nrhs <= 64;
 *   info: host array of nrhs records (may be NULL).
 * Needs OK_W_F64 or OK_W_DF64 for the residuals.  Returns OK_SUCCESS when every system converged,
 * else the first failing system's code (OK_ENOCONV, OK_EBREAKDOWN, OK_ENONFINITE); OK_EINVAL for
 * bad arguments (including params->delta outside (0, 1)), OK_ENOMEM, OK_ECUDA. */
int ok_apply_M_multi(const ok_W* W, ok_prec prec, int nrhs, const void* psi, void* out, void* stream);
int ok_bicgstab_multi(const ok_W* W, int nrhs, const void* src, void* x, const ok_solve_params* params,
                      ok_solve_info* info, void* stream);

/* Autotuner: times the candidate launch shapes of the FP32 (prec OK_F32) or FP16-W (OK_F32_W16)
 * application on scratch fields (two untimed and five timed launches each, CUDA events on
 * `stream`) and stores the fastest in the handle, which later applies and solves use.
 *   nrhs = 1: the single right-hand side kernel with the forward W read by ordinary loads or
 *             streamed into shared memory by TMA; *choice = 1 if streaming won;
 *   nrhs > 1: right-hand sides per thread (1, 2 or 4, dividing nrhs) and the persistent grid
 *             width; *choice = the right-hand sides per thread.
 * choice, best_us (the winner's time per launch, microseconds) may be NULL.  Synchronises
 * `stream`; allocates 2 nrhs V 96 bytes of scratch.  Not thread-safe against concurrent use of
 * the same handle.  OK_EINVAL for bad arguments or a missing copy, OK_ECUDA.  The paper has no
 * counterpart. */
int ok_autotune(ok_W* W, ok_prec prec, int nrhs, int* choice, double* best_us, void* stream);

/* Learned right preconditioner (an addition to the paper's unpreconditioned solver, Sec. 2.3).
 * P = L_K ... L_1 with gauge-covariant linear layers
 *   (L psi)(x) = sum_d A_d (T_d psi)(x),  d in {0, +x, -x, +y, -y, +z, -z, +t, -t},
 * T_0 = 1, (T_{+mu} psi)(x) = U_mu(x) psi(x + mu), (T_{-mu} psi)(x) = U_mu(x - mu)^dag psi(x - mu)
 * (the link transport of the hopping terms of Eq. minFlopForm, with the boundary sign of the
 * handle's bc) and A_d learned 4 x 4 complex spin matrices shared by all sites.  P is linear in
 * the source and gauge covariant; the links come from a handle made with OK_W_LINKS.
 *
 * Weights are host arrays of layers * 288 doubles: complex128 [layers][9 offsets][4][4] as
 * (re, im) pairs, offsets in the order above.  The network keeps FP32 weights, Adam moments and a
 * workspace allocated at first use: 2 V 96 bytes for applications, plus layers V 96 bytes once it
 * trains.  One network must not be used from two streams at once.
 *
 * ok_net_create: layers 1..16, weights NULL for the identity (A_0 = 1).  ok_net_free releases it.
 * ok_net_apply: out = P psi; psi, out: device [V][4][3] complex64, not overlapping.
 * ok_net_loss_grad: loss = |P b - x|^2 / |x|^2 for one pair (b, x: device complex64 fields) and,
 *   if grad is not NULL, its gradient (d/dRe + i d/dIm) into grad (host, layers * 288 doubles).
 *   Synchronises `stream`.
 * ok_net_train_step: one Adam step (lr, beta 0.9 / 0.999) on the mean loss of nb pairs
 *   (b, x: device [nb][V][4][3] complex64); *loss receives the mean loss before the step.
 *   Synchronises `stream`.
 * ok_bicgstab_net: ok_bicgstab_ex with the FP32 iteration preconditioned on the right by P
 *   (BiCGStab on M P y = b, x = x0 + P y); modes OK_SOLVE_MIXED or OK_SOLVE_MIXED16 only, the
 *   true FP64 residual of x judges convergence as without P.
 * Errors: OK_EINVAL (null or misaligned pointers, overlap, a handle without OK_W_LINKS, another
 * device, non-finite weights), OK_ENOMEM, OK_ECUDA; ok_bicgstab_net as ok_bicgstab_ex. */
int ok_net_create(int layers, const double* weights, ok_net** net);
void ok_net_free(ok_net* net);
int ok_net_layers(const ok_net* net);
int ok_net_get_weights(ok_net* net, double* weights);
int ok_net_set_weights(ok_net* net, const double* weights);
int ok_net_apply(ok_net* net, const ok_W* W, const void* psi, void* out, void* stream);
int ok_net_loss_grad(ok_net* net, const ok_W* W, const void* b, const void* x, double* loss, double* grad,
                     void* stream);
int ok_net_train_step(ok_net* net, const ok_W* W, int nb, const void* b, const void* x, double lr,
                      double* loss, void* stream);
int ok_bicgstab_net(const ok_W* W, ok_net* net, const void* src, void* x, const ok_solve_params* params,
                    ok_solve_info* info, void* stream);
/* ok_bicgstab_multi with every system's FP32 iteration right-preconditioned by the network (one
 * launch per network layer for all systems; arguments and results as ok_bicgstab_multi, the
 * handle needs OK_W_LINKS; the solve allocates four more FP32 fields per system). */
int ok_bicgstab_multi_net(const ok_W* W, ok_net* net, int nrhs, const void* src, void* x,
                          const ok_solve_params* params, ok_solve_info* info, void* stream);

/* Pin the launch shapes of the FP32 (OK_F32) or FP16-W (OK_F32_W16) application by hand instead
 * of measuring them: staged (0 or 1) for one right-hand side, nr (0 = default, else 1, 2 or 4
 * right-hand sides per thread) and blocks_x (0 = as many as fit, else 1..2^20) for several.
 * OK_EINVAL for other values. */
int ok_set_launch_shape(ok_W* W, ok_prec prec, int staged, int nr, int blocks_x);

/* The defaults used by ok_bicgstab, for the given tol and maxiter. */
ok_solve_params ok_default_solve_params(double tol, int maxiter);

/* True residual |b - M x| / |b| in FP64 (the check that judges every solve): one FP64
 * application of M fused with the norms.  b, x: device [V][4][3] complex128; relres: host.
 * Needs OK_W_F64 or OK_W_DF64.  Synchronises `stream`.  |b| = 0 gives relres = |M x|. */
int ok_true_residual(const ok_W* W, const void* b, const void* x, double* relres, void* stream);

/* Inspection: one application of M with the fused inner products that a BiCGStab half-iteration
 * takes from it (the paper's bi-stabilized CG, Sec. 2.3; van der Vorst 1992): the launch the
 * solver runs for v = M p (kind OK_REDUCE_DOT) and for t = M s (kind OK_REDUCE_TS).
 *   out = M psi, and
 *   OK_REDUCE_DOT: sums[0] + i sums[1] = <y, M psi> = sum conj(y) (M psi); sums[2] = 0;
 *   OK_REDUCE_TS:  sums[0] + i sums[1] = <M psi, y>, sums[2] = |M psi|^2.
 * prec OK_F64 (complex128 fields, OK_W_F64; OK_REDUCE_TS then needs y == psi), OK_F32 (complex64,
 * OK_W_F32) or OK_F32_W16 (complex64, OK_W_F16).  psi, y, out: device [V][4][3]; out must not
 * overlap psi or y; sums: host, 3 doubles.  The partial sums are FP64 and summed in a fixed order.
 * Allocates stream-ordered scratch and synchronises `stream`.
 * Errors: OK_EINVAL (null or misaligned pointers, overlap, a missing copy, an unknown kind),
 * OK_ENOMEM, OK_ECUDA. */
#define OK_REDUCE_DOT 1
#define OK_REDUCE_TS 2
int ok_apply_M_reduce(const ok_W* W, ok_prec prec, int kind, const void* psi, const void* y, void* out,
                      double* sums, void* stream);

/* Allocation-free true residual.  The paper has no counterpart: this entry exists for callers that
 * cannot let a library allocate device memory.  Two kinds of caller need it:
 *   - programs that reserve (nearly) all of the GPU's memory for their own pool at start-up, where
 *     a cudaMalloc issued here would fail or fragment that pool;
 *   - latency-critical loops that cannot afford the device-wide synchronisation cudaMalloc and
 *     cudaFree imply.
 * It computes r = b - M x with the OK_W_F64 copy (one fused application of M) and *relres = |r| / |b|
 * (|M x| when b = 0), like ok_true_residual, but calls no cudaMalloc, cudaFree or allocating
 * routine.
 *   b, x: device [V][4][3] complex128, inputs.  r: device [V][4][3] complex128, output, supplied by
 *   the caller, must not overlap b or x.  relres: host.
 * Its reduction scratch is one fixed array of about 2 MiB in the library's device memory.  Every GPU
 * that loads the library holds that array until the process exits.  Every call looks up the array's
 * address (cudaGetSymbolAddress, which allocates nothing) with the caller's device current, so a
 * device reset or a new context between calls is handled; the first call on a device may load the
 * library's module there, so make that first call before any stream capture.  All calls on a device share the array, so calls that overlap on
 * the GPU (different streams or threads) race: serialise them.  Synchronises `stream`.
 * Errors: OK_EINVAL for null or misaligned pointers, r overlapping an input, a handle without
 * OK_W_F64, or a lattice of more than OK_STATIC_MAX_SITES sites; OK_ECUDA. */
#define OK_STATIC_MAX_SITES (1 << 22)
int ok_true_residual_static(const ok_W* W, const void* b, const void* x, void* r, double* relres,
                            void* stream);

/* Inspection: write the dense 12x12 forward matrix of one kind for every site, reconstructed from
 * the stored representation of precision `prec` (OK_F32_W16: the half-precision copy; OK_F16_TC: the
 * tensor-core copy's blocks, W = T Q T / 2; OK_F64 reads OK_W_F64, else OK_W_DF64):
 * out = device [V][12][12] complex128 (row index
 * 3*spin + colour).  kind: 0 W^0; 1..4 W^+_mu (x, y, z, t); 5..7 W^{++}_ii (x, y, z);
 * 8..10 W^{++}_ij (xy, xz, yz); 11..13 W^{+-}_ij (xy, xz, yz; they multiply psi_{x+i-j}). */
int ok_W_expand(const ok_W* W, ok_prec prec, int kind, void* out, void* stream);

/* Number of kernels this library has launched since it was loaded (all devices, all threads). */
unsigned long long ok_launch_count(void);

/* Failure detection for the kernels' bounded waits.  The FP32 and FP16-W applies wait on shared-
 * memory barriers for the bulk copies of W; a wait that has not completed after about 2^30 SM
 * cycles gives up, so the launch ends instead of hanging, and counts itself in a device word.
 * *n receives that count for the current device (0 unless a copy failed: then every result since
 * the last reset is invalid); reset != 0 clears it.  Synchronous.  OK_EINVAL for a null n,
 * OK_ECUDA if the copy fails.  The paper has no counterpart. */
int ok_wait_timeouts(unsigned* n, int reset);

/* Failure injection for the test of the bounded waits: every later application that streams W
 * through shared memory (a handle pinned with ok_set_launch_shape(staged = 1)) makes block 0
 * declare extra_bytes more for its first bulk copy than the copy delivers, so that wait runs out
 * after about half a second; the launch then ends (its result is invalid), the timeouts are
 * counted for ok_wait_timeouts and the context stays usable.  extra_bytes = 0 turns it off;
 * other values must be multiples of 16 up to 65536 (else OK_EINVAL).  Synchronous. */
int ok_inject_wait_timeout(unsigned extra_bytes);

/* Kernel tracing (per-kernel-class timing with CUDA events recorded on the launching stream).
 * While enabled, every kernel launch of the library is bracketed by two CUDA events; ok_trace_read
 * waits for the recorded events, folds them into per-class totals and returns up to `max` entries
 * in `stats` (host array), the number of classes in *n.  Classes are named after the kernel and
 * its precision, e.g. "apply_f32_dot".  ok_trace_reset clears the totals.  Returns OK_EINVAL for
 * null outputs, OK_ECUDA if an event failed.  Tracing adds two event records per launch. */
typedef struct {
    char name[32];
    unsigned long long launches;
    double total_ms;
} ok_trace_stat;

void ok_trace_enable(int on);
int ok_trace_read(ok_trace_stat* stats, int max, int* n);
void ok_trace_reset(void);

/* Last CUDA error code seen by the library on this thread (0 if none). */
int ok_last_cuda_error(void);

/* Static description of a status code. */
const char* ok_strerror(int status);

#ifdef __cplusplus
}
#endif
#endif /* OK_GB300_H */
