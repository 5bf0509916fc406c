/* porowave_pt.h — C ABI of the GB300 pseudo-transient (PT) + Picard solver for 3-D nonlinear
 * poroviscoelastic two-phase flow (porosity waves).
 *
 * What it solves (thesis Art. 1): Biot poroelasticity extended with viscous compaction
 * (Eqs. 1-2), total momentum balance (Eq. 3), Darcy flow (Eq. 4), Maxwell viscoelastic shear
 * (Eq. 5), porosity evolution (Eq. 6), Carman-Kozeny permeability (Eq. 7), power-law shear
 * viscosity (Eq. 8), decompaction weakening (Eq. 9) of the bulk viscosity (Eq. 10) and total
 * density (Eq. 11), each physical time step solved implicitly by the PT iteration of
 * Section 2.2 (Eqs. 12-16, in the form Eqs. 17-27) on the staggered grid of Fig. 1, with
 * damped solid velocities, log-space porosity and Picard updates of the viscosities.
 *
 * Units are nondimensional; gravity acts along -z; pressures are excess over the lithostatic
 * pressure of the background density phi0 rho_f + (1 - phi0) rho_s. Boundaries are free slip
 * (zero normal velocity, zero shear stress) with zero normal Darcy flux (Eq. 34).
 *
 * ------------------------------------------------------------------------------------------
 * Memory layout (all fields, device memory, owned by the caller):
 *   Every staggered field is stored in the same padded box of dimensions
 *       pitch_x  x  pitch_y  x  (nz + 1)            with pitch_x = roundup(nx + 1, 16),
 *                                                        pitch_y = ny + 1,
 *   element (i, j, k) at offset i + pitch_x * (j + pitch_y * k), x fastest
 *   (pt_field_elems() gives the element count). Valid index ranges:
 *       cell centres (Pt, Pf, phi, mu, eta, txx, tyy, tzz, logk)   i < nx,  j < ny,  k < nz
 *       x-faces Vx (at x = i dx)                                    i <= nx, j < ny,  k < nz
 *       y-faces Vy                                                  i < nx,  j <= ny, k < nz
 *       z-faces Vz                                                  i < nx,  j < ny,  k <= nz
 *       xy-edges txy (at x = i dx, y = j dy)                        i <= nx, j <= ny, k < nz
 *       xz-edges txz                                                i <= nx, j < ny,  k <= nz
 *       yz-edges tyz                                                i < nx,  j <= ny, k <= nz
 *   Cell (i, j, k) is centred at ((i + 1/2) dx, (j + 1/2) dy, (k + 1/2) dz), dx = lx / nx.
 *   Entries outside the valid ranges are padding: the library never reads them as data.
 *   Field arrays must be 16-byte aligned and must not alias each other or the workspace.
 *
 * Threading and streams: every call is asynchronous on the stream given to pt_init except
 * where a call returns a report (pt_step, pt_iterate, pt_residual), which synchronise that
 * stream to read it. The library holds no global state; a context is used by one host thread
 * at a time.
 *
 * Errors: functions return PT_OK (0) or a negative code (pt_strerror gives its text). On any
 * error the fields hold the last complete iterate.
 */
#ifndef POROWAVE_PT_H
#define POROWAVE_PT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  PT_OK = 0,
  PT_EINVAL = -1,     /* bad argument: null pointer, size < 1, dt <= 0, misaligned, ...      */
  PT_ENOTCONV = -2,   /* max_iter reached before the residual fell below tol                  */
  PT_ENAN = -3,       /* a residual norm was not finite                                       */
  PT_ETIMEOUT = -4,   /* a bounded device-side wait expired (reserved: no kernel of this
                         library waits on another; every convergence decision is a host read
                         of a reduction or a non-spinning retire kernel)                       */
  PT_ECUDA = -5,      /* a CUDA call or kernel launch failed                                  */
  PT_ESPACE = -6      /* workspace smaller than pt_workspace_size()                            */
};

/* Arithmetic of the PT iterations. PT_FP64: FP64 throughout, in the FP64-lean form (two
 * fused kernels per iteration, coefficients refreshed at Picard updates). PT_FP64_STEPWISE:
 * FP64, one kernel per data-flow step (the straightforward form, kept for comparison).
 * PT_FP32: FP32 PT iterations with FP64 residuals, defect correction and porosity time
 * integration. PT_DF64: the FP64-lean form's iteration in double-float arithmetic (each value
 * the unevaluated sum of two FP32 numbers, a 48-bit significand in FP32's exponent range,
 * computed on the FP32 pipe): the iterate lives in the workspace from pt_step_begin on and is
 * written to the caller's FP64 fields when each call returns; residual norms and reports are
 * FP64. Fields at the boundary are FP64 in every mode. PT_DF64 serves pt_init / pt_step /
 * pt_iterate / pt_residual; the batched, sub-domain and adjoint entry points take PT_FP64. */
enum { PT_FP64 = 0, PT_FP32 = 1, PT_FP64_STEPWISE = 2, PT_DF64 = 3 };

/* Cell-centred grid on [0, lx] x [0, ly] x [0, lz]; dx = lx / nx. */
typedef struct {
  int32_t nx, ny, nz;
  double lx, ly, lz;
} pt_grid;

/* Physical parameters (Table 2 symbols, nondimensional). */
typedef struct {
  double phi0;      /* background porosity (sets the background density)                  */
  double k0;        /* reference permeability over fluid viscosity, k = k0 e^logk (phi/phi0)^3 */
  double mu0;       /* reference shear viscosity (Eq. 8)                                  */
  double eta0;      /* reference bulk viscosity, eta = eta0 mu / phi (Eq. 10)             */
  double R_weak;    /* bulk-viscosity multiplier where Pf > Pt (Eq. 9; 1 = no weakening)  */
  double n_pow;     /* power-law exponent n (Eq. 8)                                       */
  double tau0;      /* characteristic stress tau0 (Eq. 8)                                 */
  double alpha;     /* Biot-Willis coefficient                                            */
  double B;         /* Skempton coefficient                                               */
  double beta_d;    /* drained compressibility 1 / K_d                                    */
  double beta_phi;  /* effective bulk compressibility 1 / K_phi                           */
  double G;         /* elastic shear modulus                                              */
  double rhof_g;    /* fluid density times gravity                                        */
  double rhos_g;    /* solid density times gravity                                        */
  int32_t powerlaw_on;    /* 0: mu* = mu0 (no power law)                                  */
  int32_t compaction_on;  /* 0: no viscous compaction term (1 / eta = 0)                  */
  double tau_bg;          /* applied horizontal background shear stress (Eqs. 32-33; 0 =
                             none): tau_bg / (2 mu0) is added to the xy strain rate on every
                             xy-edge, the wall edges included (free slip for the unknown V) */
} pt_phys;

/* Numerical parameters of the PT iteration (Section 2.2 and the appendix two-phase script). */
typedef struct {
  double dt;              /* physical time step (> 0)                                      */
  double tol;             /* convergence: max of the residual max-norms < tol               */
  int32_t max_iter;       /* PT iteration cap per physical step                            */
  int32_t nup;            /* Picard update and residual check every nup-th iteration       */
  double damp[3];         /* velocity damping per direction, e.g. 1 - 1/n                  */
  double rho_i;           /* inertial density of the velocity pseudo-time step            */
  double beta_n;          /* numerical compressibility in the normal stresses               */
  double rel_mu, rel_eta; /* log-space Picard relaxation of mu and eta                      */
  double cfl_v;           /* dtau_V = cfl_v h^2 rho_i / (mu (1 + beta_n)),  h = min(dx,dy,dz) */
  double cfl_pf;          /* dtau_Pf = cfl_pf h^2 (1 + beta_d B / alpha) / max local k      */
  double dtpt_scale;      /* dtau_Pt = dtpt_scale mu (1 + beta_n) / nz                      */
  double xsi_w;           /* stress sub-step dtS = max(mu) / (G xsi_w)                      */
  int32_t precision;      /* PT_FP64, PT_FP64_STEPWISE, PT_FP32 or PT_DF64 (enum above)     */
  int32_t iters_per_graph;/* PT iterations per CUDA-graph replay; 0 = nup                  */
  double inner_rtol;      /* PT_FP32: each FP32 correction solve stops at this relative drop
                           * of its residual (0 = 0.1)                                     */
  int32_t mg_levels;      /* PT_FP32: 0 or 1 = each correction problem is solved by FP32 PT
                           * iterations; L >= 2 = by geometric-multigrid V-cycles over L grids
                           * (each with ceil(n / 2) cells per direction of the one above, over
                           * the same box: nested for even n; the coarsest at least 2 cells per
                           * direction), smoothed by the PT sweep (see pt_mixed_kernels.cu);
                           * PT_EINVAL otherwise, and for batched ensembles                   */
  int32_t mg_reserved;    /* 0                                                              */
} pt_num;

/* Caller-owned device fields, padded box layout above. logk may be NULL (logk = 0). */
typedef struct {
  double *Vx, *Vy, *Vz;                       /* solid velocity                (r/w)     */
  double *Pt, *Pf, *phi;                      /* total, fluid pressure, porosity (r/w)    */
  double *txx, *tyy, *tzz, *txy, *txz, *tyz;  /* deviatoric stress of the last step (r/w) */
  double *mu, *eta;                           /* Picard shear and bulk viscosity (r/w)    */
  const double *logk;                         /* log-permeability prefactor field (read)  */
} pt_fields;

/* Report of a step / iteration batch: residual max-norms of the last check. */
typedef struct {
  int32_t iters;      /* PT iterations taken                                                */
  int32_t status;     /* PT_OK, PT_ENOTCONV, PT_ENAN, ...                                   */
  double res_v;       /* max |F| momentum residual (Eq. 19 left side)                       */
  double res_pt;      /* max |numerical div V| (Eq. 17 left side)                           */
  double res_pf;      /* max |fluid-pressure residual| (Eq. 18 left side)                   */
  double res_pic;     /* max |log mu* - log mu|, |log eta* - log eta| (Eqs. 24, 26)         */
} pt_report;

typedef struct pt_ctx pt_ctx;

/* Elements per field array (padded box) for this grid; 0 if the grid is invalid. */
size_t pt_field_elems(const pt_grid *grid);
/* x pitch of the padded box (elements). */
int32_t pt_pitch_x(const pt_grid *grid);
/* Bytes of device workspace pt_init needs for this grid and numerics. */
size_t pt_workspace_size(const pt_grid *grid, const pt_num *num);

/* Create a solver context over caller-owned fields and workspace (device memory, at least
 * pt_workspace_size() bytes, 256-byte aligned). Initialises the Picard state
 * mu = mu0, eta = eta0 mu / phi (Eq. 26 with R = 1) unless keep_visc != 0, zeroes the damped
 * residuals, and validates every argument. `stream` is a cudaStream_t (NULL = default stream).
 * The context keeps the pointers: fields and workspace must outlive it. */
int pt_init(pt_ctx **ctx, const pt_grid *grid, const pt_phys *phys, const pt_num *num,
            const pt_fields *fields, void *workspace, size_t workspace_bytes, void *stream,
            int32_t keep_visc);

/* One physical time step (thesis Art. 1 Section 2.2): snapshot of the old state, PT + Picard
 * iterations until the residual max-norm < tol (checked every nup iterations) or max_iter,
 * then the step's final stresses. Returns PT_OK, PT_ENOTCONV (fields hold the last iterate,
 * `rep` the last norms) or an error. */
int pt_step(pt_ctx *ctx, pt_report *rep);

/* Lower-level pieces of pt_step, for fixed-iteration-count runs (benchmarks, parity tests):
 * pt_step_begin = old-state snapshot and stress sub-step; pt_iterate = `niter` PT iterations
 * numbered it0+1 .. it0+niter (Picard and norms on multiples of nup; no convergence exit;
 * `rep` may be NULL to skip the norm read-back); pt_step_end = final stresses and dt_cum. */
int pt_step_begin(pt_ctx *ctx);
int pt_iterate(pt_ctx *ctx, int32_t it0, int32_t niter, pt_report *rep);
int pt_step_end(pt_ctx *ctx);

/* Residual max-norms of the current state (no update). */
int pt_residual(pt_ctx *ctx, pt_report *rep);

/* Per-kernel device time, measured with CUDA events recorded on the context's stream around
 * every kernel launch between pt_profile_begin and pt_profile_end (a benchmarking aid; the
 * events are created on first use and kept by the context). pt_profile_end synchronises the
 * stream, writes up to max_out entries (one per kernel that ran) and the entry count. */
typedef struct {
  char name[24];
  int64_t launches;
  double total_ms;
} pt_kernel_time;
int pt_profile_begin(pt_ctx *ctx);
int pt_profile_end(pt_ctx *ctx, pt_kernel_time *out, int32_t max_out, int32_t *n_out);
/* Kernel launches issued by this context since pt_init. */
int64_t pt_launch_count(const pt_ctx *ctx);

/* ---- Measured peaks (benchmarking aids; thesis Art. 1 Eqs. 28-29 compare T_eff with a measured
 * copy throughput) ---------------------------------------------------------------------------
 * pt_peak_copy: dst = src over `bytes` (16-byte aligned device buffers, bytes rounded down to a
 * multiple of 16) with 16-byte vector loads and stores, grid-stride over 8 CTAs of 256 threads per
 * SM; best of `reps` timed launches after one warm-up; *gbs = read + write bytes / best time.
 * pt_peak_arith: kind 0 = FP64 (DFMA, DADD, DMUL, one each per step of 8 independent chains per
 * thread), kind 1 = FP32 FMA (8 chains); 2048 threads per SM, `steps` steps; *ginst = thread-
 * instructions per second / 1e9 (FP32 flops = 2 x that). `sink` is device memory of at least
 * 8 x (SM count) doubles (never written for these inputs). Both synchronise `stream`. */
int pt_peak_copy(const void *src, void *dst, size_t bytes, int32_t reps, void *stream, double *best_ms,
                 double *gbs);
int pt_peak_arith(int32_t kind, void *sink, int32_t steps, int32_t reps, void *stream, double *best_ms,
                  double *ginst);

/* ---- Check of the hand-written device arithmetic (test aid; no thesis counterpart) ----------
 * Applies one device routine of the PT kernels element-wise: out[e] = f(a[e] (, b[e])), n
 * elements, device pointers, synchronises `stream`. It exists so that each replacement of a
 * library operation can be compared with CUDA's own function and with its stated error bound:
 *   PT_MATH_RCP_PSEUDO   1/x, approximate FP64 reciprocal + one Newton-Raphson step (~2^-46)
 *   PT_MATH_RCP_FULL     1/x, approximate FP64 reciprocal + two Newton-Raphson steps (rounding)
 *   PT_MATH_EXPM1_POS/NEG  expm1(x), expm1(-x) from the split Taylor series of exp (tiers
 *                          |x| <= 2^-20, <= 2^-6; beyond, CUDA's expm1)
 *   PT_MATH_DF_ADD/SUB/MUL   double-float a + b, a - b, a * b (inputs rounded to double-float)
 *   PT_MATH_DF_FMA       double-float a * b + a
 *   PT_MATH_DF_RCP/SQRT  double-float 1/a, sqrt(a) (FP32 seed + one Newton step)
 *   PT_MATH_DF_ROOT      double-float a^(1/m), m = (int)b[e] (Newton's m-th root)
 *   PT_MATH_DF_EXPM1_POS/NEG  the split Taylor series in double-float
 * Returns PT_EINVAL for an unknown code or a missing operand. */
enum { PT_MATH_RCP_PSEUDO = 0, PT_MATH_RCP_FULL = 1, PT_MATH_EXPM1_POS = 2, PT_MATH_EXPM1_NEG = 3,
       PT_MATH_DF_ADD = 4, PT_MATH_DF_SUB = 5, PT_MATH_DF_MUL = 6, PT_MATH_DF_FMA = 7,
       PT_MATH_DF_RCP = 8, PT_MATH_DF_SQRT = 9, PT_MATH_DF_ROOT = 10, PT_MATH_DF_EXPM1_POS = 11,
       PT_MATH_DF_EXPM1_NEG = 12 };
int pt_math_check(int32_t fn, const double *a, const double *b, double *out, int64_t n, void *stream);

/* ---- Residual norms with no allocation at all -------------------------------------------
 * The paper has no counterpart to this entry point; it exists for callers that cannot
 * allocate device memory when they need the norms - e.g. a health check inside a run whose
 * HBM is entirely held by a pool allocator, where a raw cudaMalloc would fail or fragment the
 * pool, or a timing-critical loop that cannot afford the implicit device synchronisation of
 * cudaMalloc / cudaFree. It computes the same four norms as pt_residual from fields the caller
 * passes (current fields, old-step fields, the stress sub-step dtS) without a context or
 * workspace: its intermediate arrays live in one fixed device array inside this library,
 * PT_RESIDUAL_STATIC_SCRATCH_BYTES large, which every GPU that loads the library holds until
 * the process exits. Grids whose padded box needs more than 10 arrays of that array (boxes of
 * about 838,000 elements, e.g. 90^3 cells) are rejected with PT_ESPACE before any device work.
 * Layout, alignment and argument rules are those of pt_init (the same validation and the same
 * coefficient builder; the background shear tau_bg included); the current device must be the
 * one holding the fields. The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and caches it. Under CUDA's lazy module loading (the default) that
 * first call is also when the device reserves the array's memory, so make it early: before a
 * pool allocator claims the device's free memory, and before any stream capture. Every
 * call shares the array and clears its reduction block first; calls whose device work
 * overlaps (other streams or host threads) race on it. Calls no cudaMalloc / cudaFree and no
 * allocating library routine; synchronises `stream` to read the norms into `rep`. */
#define PT_RESIDUAL_STATIC_SCRATCH_BYTES (64u * 1024u * 1024u)
typedef struct {
  const double *Pto, *Pfo;                          /* pressures at the start of the step */
  const double *txxo, *tyyo, *tzzo, *txyo, *txzo, *tyzo;  /* old-step stresses          */
} pt_old_fields;
int pt_residual_static(const pt_grid *grid, const pt_phys *phys, const pt_num *num,
                       const pt_fields *fields, const pt_old_fields *old, double dtS,
                       void *stream, pt_report *rep);

/* ---- Adjoint (no thesis counterpart) -------------------------------------------------------
 * Gradient of an objective J(phi^N) of the porosity after N physical steps with respect to the
 * log-permeability field logk (k = k0 e^logk (phi/phi0)^3), by the discrete adjoint of the
 * converged implicit steps: for n = N..1, J_F(u^n)^T lambda^n = g^n is solved with the same
 * pseudo-transient scheme as the forward steps on the transposed staggered stencils, the
 * gradient accumulates -(dF/dlogk)^T lambda^n and g^{n-1} = -(dF^n/du^{n-1})^T lambda^n.
 * Scope: no weakening (R_weak = 1: Eq. 25 is a step function), beta_n = 0, no background shear,
 * and no old-stress refresh inside the window (the window starts at the context's first step
 * with zero stresses and the accumulated time stays below the stress sub-step dtS); other
 * settings return PT_EINVAL. With the power law on (Eq. 24) mu is an unknown of each step with
 * the Picard fixed-point row log mu - log mu*(tau_II), eta = eta0 mu / phi, the Maxwell moduli
 * 2 mu / (1 + xi) vary per centre and edge, and the step's dtS = max(mu of the previous step) /
 * (G xsi_w) is differentiated too (into the cell holding that maximum).
 * pt_adjoint_forward runs the N forward steps from the context's current state, keeping a
 * checkpoint of the full state every ckpt_every steps in the adjoint workspace
 * (pt_adjoint_workspace_size bytes, 256-byte aligned, device memory; ckpt_every = 1 stores every
 * step and the reverse sweep then runs no forward step again); pt_adjoint then sweeps
 * back, re-running each segment from its checkpoint, writes dJ/dlogk (device, box layout) given
 * dJ/dphi^N (device, box layout), and leaves the context at the state after step N.
 * reps (pt_adjoint_forward: N entries; pt_adjoint: 1) report iterations and the last norms. */
size_t pt_adjoint_workspace_size(const pt_grid *grid, int32_t nsteps, int32_t ckpt_every);
int pt_adjoint_forward(pt_ctx *ctx, int32_t nsteps, int32_t ckpt_every, void *adj_workspace,
                       size_t adj_bytes, pt_report *reps);
int pt_adjoint(pt_ctx *ctx, const double *dJ_dphi, double *dJ_dlogk, pt_report *rep);

/* One application of the transposed operator: out = J_F(u)^T lam, J_F the Jacobian of the
 * residual F = (F_V, F_Pt, F_Pf, F_L[, F_mu]) of the implicit step (Eqs. 17-22 and, with the
 * power law, 24; same scope as pt_adjoint) at the context's current fields u (k0 e^logk from
 * pt_init; the context's current dtS). Components are in box layout on the device: lam/out Vx,
 * Vy, Vz on faces (the wall-normal faces of lam must hold zero; those of out are set to zero),
 * Pt, Pf, phi and mu at centres (lam->Pt pairs with F_Pt, ... , lam->phi with F_L, lam->mu with
 * F_mu; out->phi is dF/dphi^T lam, out->mu dF/dmu^T lam). Requires a step begun (pt_step or
 * pt_step_begin); workspace: pt_adjoint_workspace_size(grid, 0, 1) bytes of device memory,
 * 256-byte aligned, used as scratch. Synchronises the stream. The thesis has no counterpart:
 * this exists so that the transposed stencils can be checked against an independent Jacobian. */
typedef struct {
  double *Vx, *Vy, *Vz, *Pt, *Pf, *phi;
  double *mu;   /* the Picard row / unknown mu (power law on; may be NULL when it is off) */
} pt_adj_vec;
int pt_adjoint_apply(pt_ctx *ctx, const pt_adj_vec *lam, pt_adj_vec *out, void *workspace, size_t bytes);

/* Test aid (host only): the multigrid transfer tables of one direction between nf fine and
 * nc = ceil(nf / 2) coarse cells (pt_num.mg_levels; see pt_mixed.cuh MgAxis for the layout:
 * box_i0[nc], box_w[3 nc], hat_i0[nc + 1], hat_w[4 (nc + 1)], lin_ab[2 nf], lin_w[2 nf],
 * fl_n0[nf + 1], fl_t[nf + 1], as 4-byte words, integers and FP32 values). Writes
 * pt_mg_axis_words(nf) words to out (PT_ESPACE if `words` is smaller; PT_EINVAL for nf < 2). */
size_t pt_mg_axis_words(int32_t nf);
int pt_mg_axis_tables(int32_t nf, uint32_t *out, size_t words);

/* ---- Batched ensemble --------------------------------------------------------------------
 * ninst independent instances (each its own grid, parameters, fields and numerics), all
 * PT_FP64 or all PT_FP32 (mixing returns PT_EINVAL), advanced together by one persistent engine:
 * one launch per phase covers all instances through a flat work list of (instance, tile) items
 * walked by a persistent grid-stride grid (SMs x resident CTAs), the launch sequence captured
 * in one CUDA graph per replay, and every decision (convergence, iteration cap, non-finite
 * norms) taken on the device per instance; the host reads a status table once per replay.
 * FP64 ensembles (the FP64-lean form): 2 nup (or 4 nup) PT iterations per replay; each instance
 * stops at its own first check with norms < tol (or at its max_iter / a non-finite norm). The
 * first pt_batch_step tunes the tile shape (32x4, 32x8, 64x4) and the iterations per replay.
 * FP32 ensembles (the FP32 + FP64 defect-correction form): a replay runs `rounds` rounds of
 * [FP64 residuals, stresses and Picard update of the instances starting an outer iteration;
 * their outer decision (converged, outer weight, inner target); nup FP32 correction iterations
 * of the instances in a correction solve; their inner decision (relative drop reached or budget
 * spent); the FP64 update and porosity integration of the instances ending one], the instances
 * split into contiguous groups whose rounds are parallel branches of the graph. The first
 * pt_batch_step tunes the correction tile depth (32, 64 levels), the CTAs per SM of the
 * correction kernel (3, 4), the rounds per replay (1, 2) and the groups (1, 4, 8, 16).
 * Either way each instance reproduces its single-instance pt_step: the same per-point code and
 * the same decisions in the same order, so the same iteration counts and statuses, and fields
 * equal to rounding (the shared bodies inlined into other kernels may round their multiply-adds
 * differently), whatever the configuration (tuning replays are real iterations). grids/phys/nums/fields are arrays of ninst; the workspace holds every instance's
 * workspace (pt_workspace_size) plus the descriptor tables. The batch works on a stream of its
 * own (graphs cannot be captured on the legacy default stream): pt_batch_init and pt_batch_step
 * first synchronise the caller's `stream`, and pt_batch_step returns after its work is done. */
typedef struct pt_batch pt_batch;
size_t pt_batch_workspace_size(int32_t ninst, const pt_grid *grids, const pt_num *nums);
int pt_batch_init(pt_batch **batch, int32_t ninst, const pt_grid *grids, const pt_phys *phys,
                  const pt_num *nums, const pt_fields *fields, void *workspace,
                  size_t workspace_bytes, void *stream);
/* One physical step of every instance. reps[ninst] receives each instance's report;
 * time_to_converge_ms[ninst] (may be NULL) its device time from the step's first iteration to
 * its stop. Returns PT_OK when every instance converged, PT_ENOTCONV if any hit its cap. */
int pt_batch_step(pt_batch *batch, pt_report *reps, double *time_to_converge_ms);
/* The tuned configuration (valid after the first pt_batch_step): the tile's x and y extents
 * (FP32 ensembles: the correction tile, 30 x 6 faces) and the (correction) iterations per replay. */
int pt_batch_config(const pt_batch *batch, int32_t *tile_x, int32_t *tile_y,
                    int32_t *iters_per_graph);
/* FP32 ensembles: the tuned correction tile depth (z levels), CTAs per SM of the correction
 * kernel and number of member groups (contiguous groups of near-equal cells whose rounds are
 * parallel branches of the replayed graph); PT_EINVAL for an FP64 ensemble. */
int pt_batch_config_fp32(const pt_batch *batch, int32_t *tile_z, int32_t *blocks_per_sm,
                         int32_t *groups);
void pt_batch_destroy(pt_batch *batch);

/* ---- Sub-domain (halo-exchange) form (Art. 1 Section 2.2) ----------------------------------
 * The distributed-memory decomposition of the thesis (Art. 1 Section 2.2; Art. 2: one
 * sub-domain per GPU, halos exchanged every iteration), run on one GPU: the grid is split into
 * parts[0] x parts[1] x parts[2] parts of near-equal size (at least 2 cells per part and
 * direction), each an FP64-lean instance of the batched engine with its own padded box and a
 * one-cell halo on every side that has a neighbour. After every PT iteration the halos of V,
 * Pt, Pf, phi (with 1/(1-phi) and k) and after every Picard update those of mu, eta are copied
 * from the owning parts; residual norms count owned points only; all parts stop together and
 * share one stress sub-step from the largest mu of the whole grid. The result is bitwise that
 * of the undivided grid run by the same kernels (parts = {1, 1, 1}).
 * pt_dd_init copies the caller's global fields (device, box layout of `grid`) into the parts
 * (workspace: pt_dd_workspace_size bytes of device memory, 256-byte aligned; precision must be
 * PT_FP64; viscosities are initialised from phi as by pt_init); pt_dd_step advances one
 * physical step to convergence (rep: iterations and the global norms); pt_dd_gather writes the
 * parts' owned values back into the global fields. Errors: PT_EINVAL (sizes, parts, precision),
 * PT_ESPACE, PT_ECUDA; pt_dd_step returns PT_ENOTCONV / PT_ENAN as pt_step does. */
typedef struct pt_dd pt_dd;
size_t pt_dd_workspace_size(const pt_grid *grid, const pt_num *num, const int32_t parts[3]);
int pt_dd_init(pt_dd **dd, const pt_grid *grid, const pt_phys *phys, const pt_num *num,
               const pt_fields *fields, const int32_t parts[3], void *workspace, size_t bytes,
               void *stream);
int pt_dd_step(pt_dd *dd, pt_report *rep);
int pt_dd_gather(pt_dd *dd);
/* Number of parts and the tuned configuration of the underlying batched engine. */
int pt_dd_config(const pt_dd *dd, int32_t *nparts, int32_t *tile_x, int32_t *tile_y, int32_t *iters_per_graph);
void pt_dd_destroy(pt_dd *dd);

/* Release the context (not the caller's memory). */
void pt_destroy(pt_ctx *ctx);

const char *pt_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif
