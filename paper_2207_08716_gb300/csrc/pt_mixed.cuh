// pt_mixed.cuh — argument structs and host launchers of the mixed-precision (PT_FP32) kernels
// in pt_mixed_kernels.cu.
#pragma once

#include "pt_lean.cuh"
#include "pt_kernels.cuh"

namespace pt {

struct MixPrepIn {
  const double *Vx, *Vy, *Vz, *Pt, *Pf, *phi, *mu, *eta, *perm, *Pto, *Pfo, *txxo, *tyyo, *tzzo;
};
struct MixPrepOut {
  double *txx, *tyy, *tzz;                                  // FP64 stresses at u
  float *r_pt, *r_pf, *cc, *perm, *idtp;
};
struct MixFaceIn {
  const double *txx, *tyy, *tzz, *txy, *txz, *tyz, *Pt, *phi;
};
struct MixCoefOut {
  float *mu;                                                // mu at centres (FP32)
  float *dtvc;                                              // velocity pseudo-step fac / mu at centres
};
struct MixPorosity {       // the porosity integration of Eq. 22 at the corrected state
  const double *Vx, *Vy, *Vz, *phi, *Pt1, *Pf1, *Pto, *Pfo, *Lo, *eta;
  double* phi1;
};
struct MixUpdate {
  double *Vx, *Vy, *Vz, *Pt, *Pf;
  const float *dVx, *dVy, *dVz, *dPt, *dPf;
  double omega;             // u <- u + omega delta
};

template <class T>
struct CorrCoef {
  T rdx, rdy, rdz, hrdx, hrdy, hrdz, hrdx2, hrdy2, hrdz2;
  T bd_rdt, bd_rdt_a, bda_B_rdt, beta_n, rrho_i, damp_x, damp_y, damp_z;
  T rG;         // 1 / (G dtS): xi = mu rG
  T ifac_pf;    // 1 / dtau_Pf = kmax ifac_pf
};
// One FP32 PT iteration on the correction, in one pass: the current correction (dV, dPt, dPf),
// the frozen coefficients and right-hand sides, and where the next correction goes.
template <class T>
struct CorrIn {
  const T *Vx, *Vy, *Vz, *Pt, *Pf;                 // current correction dV, dPt, dPf
  const T *cc, *perm, *idtp, *r_pt, *r_pf, *mu, *dtvc, *rfx, *rfy, *rfz;
};
template <class T>
struct CorrOut {
  T *Vx, *Vy, *Vz, *Pt, *Pf;                       // next dV, dPt, dPf (other buffers)
  T *Rx, *Ry, *Rz;                                 // damped residuals (in place)
  T *res_pt, *res_pf;                              // cell residuals rho_Pt, rho_Pf (when non-null)
  int eval;                                        // 1: evaluate only -- R = momentum residual of the
                                                   // current iterate (damp 0), no dV', dPt', dPf'
};

// One grid of the multigrid hierarchy of the FP32 correction problem (level 0 = the problem's
// own arrays; coarser levels live in the workspace).
// Transfer weights between a level and the finer one above it along one direction (n fine cells,
// nc = ceil(n / 2) coarse cells; built on the host from the cell and face positions, in the
// workspace): the coarse cell I covers fine cells box_i0[I] + 0..2 with weights box_w[3 I + t]
// (the covered fractions); the coarse face J gathers fine faces hat_i0[J] + 0..3 with weights
// hat_w[4 J + t] (a hat of half-width n / nc, normalised); fine cell i interpolates coarse cells
// lin_ab[2 i], lin_ab[2 i + 1] with weights lin_w[2 i], lin_w[2 i + 1]; fine face i interpolates
// coarse faces fl_n0[i], fl_n0[i] + 1 with weights 1 - fl_t[i], fl_t[i].
struct MgAxis {
  const int* box_i0;
  const float* box_w;
  const int* hat_i0;
  const float* hat_w;
  const int* lin_ab;
  const float* lin_w;
  const int* fl_n0;
  const float* fl_t;
};

struct MgLevel {
  Box b;
  MgAxis ax[3];                                    // transfers from the finer level (x, y, z)
  float *cc, *perm, *idtp, *mu, *dtvc;             // frozen coefficients
  float *rpt, *rpf, *rfx, *rfy, *rfz;              // right-hand sides
  float *dVx[2], *dVy[2], *dVz[2], *dPt[2], *dPf[2];
  float *Rx, *Ry, *Rz;
  float *res_pt, *res_pf;                          // cell residuals of an evaluation sweep
};

void mix_prepare(dim3 g, dim3 bl, cudaStream_t s, Box b, const Coef& c, const MixPrepIn& in,
                 const MixPrepOut& out, unsigned long long* red);
void mix_res_faces(dim3 g, dim3 bl, cudaStream_t s, Box b, const Coef& c, const MixFaceIn& in, float* rfx,
                   float* rfy, float* rfz, unsigned long long* red);
void mix_coef(dim3 g, dim3 bl, cudaStream_t s, Box b, const Coef& c, const double* mu, const MixCoefOut& out);
void mix_edges(dim3 g, dim3 bl, cudaStream_t s, Box b, const Coef& c, const EdgeIn& in, const EdgeOut& out);
void mix_porosity(dim3 g, dim3 bl, cudaStream_t s, Box b, const Coef& c, const MixPorosity& p);
void mix_update(dim3 g, dim3 bl, cudaStream_t s, Box b, const MixUpdate& u);
// One fused FP32 correction iteration over the whole grid (z-marching tiles, see the kernel).
void corr_iteration(cudaStream_t s, Box b, const CorrCoef<float>& c, const CorrIn<float>& in,
                    const CorrOut<float>& out, unsigned long long* red, int check);
// Multigrid transfers between level `f` (n cells per direction) and the coarser level `c`
// (ceil(n / 2) cells over the same box, so r = n / ceil(n / 2) fine cells per coarse cell: 2 for an
// even n, slightly less for an odd one, where the grids are not nested):
//   mg_coef      coarse mu, k, cc = means over the fine cells a coarse cell covers (weights = the
//                covered fractions, "box" weights); 1/dtau_Pt and dtau_V from the coarse mu with the
//                coarse grid's pseudo-step factors
//   mg_restrict  coarse right-hand sides from the fine residuals (cells: box weights; faces: the
//                hat function of half-width r along the normal, normalised -- (1/4, 1/2, 1/4) for
//                r = 2 -- times box weights across it; the fine momentum residual is rho_i R of the
//                evaluation sweep), zero coarse iterate and R
//   mg_prolong   fine iterate (buffers df) += coarse correction (buffers dc) interpolated: cells
//                trilinearly between coarse centres (3/4 and 1/4 for r = 2; zero gradient beyond the
//                first and last centre), faces linearly between coarse faces along the normal and
//                between centres across it
void mg_coef(cudaStream_t s, const MgLevel& f, const MgLevel& c, float dtaupt_fac, float dtauv_fac);
void mg_restrict(cudaStream_t s, const MgLevel& f, const MgLevel& c, float rho_i);
void mg_prolong(cudaStream_t s, const MgLevel& c, int dc, const MgLevel& f, int df);

// ---------------------------------------------------------------- batched FP32 ensembles
// Every member's defect-correction loop in one engine: the loop's decisions (outer convergence,
// outer weight, inner stop, iteration cap) are taken on the device per member, so the members
// advance together through one graph-captured launch sequence per replay:
//   PREP     FP64 residuals at u, stresses, Picard update               (members in MB_PREP)
//   decide   outer norms: converged / non-finite -> MB_DONE, else weight, inner target -> MB_INNER
//   INIT     frozen FP32 coefficients and a zero correction             (members starting a solve)
//   corr x nup   FP32 correction iterations, norms at the last          (members in MB_INNER)
//   decide   inner stop (drop reached, or the member's iteration budget spent) -> MB_UPDATE
//   UPDATE, POROSITY   u <- u + omega delta, FP64 porosity integration  (members in MB_UPDATE)
//   finish   parity flip, iterations counted, cap -> MB_DONE, else MB_PREP
// The per-point and per-tile bodies are those of the single-instance kernels, and the decisions
// are the host loop's, so a member reproduces its single-instance FP32 step: the same iteration
// counts, fields equal to rounding.
enum { MB_PREP = 0, MB_INNER = 1, MB_UPDATE = 2, MB_DONE = 3 };
enum { MB_PH_PERM = 0, MB_PH_PREP = 1, MB_PH_FACES = 2, MB_PH_INIT = 3, MB_PH_UPDATE = 4, MB_PH_POROSITY = 5 };

struct MixBatchInst {
  Box b;
  Coef k;                                   // FP64 residuals, porosity update
  LeanCoef<double> lc;                      // Picard update
  CorrCoef<float> cc;                       // FP32 correction iteration
  double *Vx, *Vy, *Vz, *Pt[2], *Pf[2], *phi[2], *mu, *eta, *perm, *rog, *Pto, *Pfo, *Lo;
  const double* logk;
  double *txxo, *tyyo, *tzzo, *txyo, *txzo, *tyzo;
  double *s_txx, *s_tyy, *s_tzz, *s_txy, *s_txz, *s_tyz;
  float *rpt, *rpf, *rfx, *rfy, *rfz, *ccf, *kf, *idtp, *muf, *dtvc;
  float *dVx[2], *dVy[2], *dVz[2], *dPt[2], *dPf[2], *Rx, *Ry, *Rz;
  const float* fbase;                       // the FP32 arrays above, kMixArrays consecutive arrays
  long long fstride;                        // fbase + slot * fstride (floats), in the order of pt_init
  CorrIn<float> cin[2];                     // correction iteration reading buffer d (0/1) ...
  CorrOut<float> cout[2];                   // ... and writing buffer 1 - d
  unsigned long long* red;                  // outer norms (RED_N slots)
  unsigned long long* ired;                 // inner norms (RED_N slots)
  double tol;                               // outer tolerance
  double rtol;                              // inner relative drop
  int max_iter;                             // FP32 iterations per step
  int gx, gy;                               // point tiles (32 x 8 of one z-level)
  int cgx, cgy, cgz;                        // correction tiles (kCorrTX x kCorrTY x zchunk)
  long long tile_base, ctile_base;          // first work item of this member in each list
};

struct MixBatchStatus {
  int phase;                                // MB_*
  int cur;                                  // parity of the buffers holding Pt, Pf, phi
  int inner;                                // FP32 iterations of the current correction solve
  int iters;                                // FP32 iterations of the step before this solve
  int outer;                                // outer iterations completed
  int status;                               // PT_OK, PT_ENOTCONV, PT_ENAN once MB_DONE
  int fresh;                                // 1 while a solve is being set up (INIT runs)
  int pad;
  double omega;                             // weight of the outer update
  double prev;                              // previous outer residual max (0 at the start)
  double target;                            // inner stop: drop to this residual max
  double res[4];                            // outer norms of the last check (v, pt, pf, pic)
  unsigned long long t_start, t_stop;       // device %globaltimer (ns)
};

// The kernels take a slice of the member table (inst, st: its first member; ninst members) and
// the range [t0, t1) of work items its members own (tile_base / ctile_base are global offsets).
void mb_points(int grid, cudaStream_t s, int phase, const MixBatchInst* inst, const MixBatchStatus* st, int ninst,
               long long t0, long long t1);
// Correction iteration number inner + step (1-based) of every member in MB_INNER within its budget;
// minb (3 or 4): the CTAs per SM the kernel's registers are budgeted for. Sets the kernel's
// shared-memory attribute first (mb_corr_blocks_per_sm, before any capture).
void mb_corr(int grid, int minb, cudaStream_t s, const MixBatchInst* inst, const MixBatchStatus* st, int ninst,
             long long t0, long long t1, int step, int nup, int zchunk);
void mb_decide_outer(cudaStream_t s, const MixBatchInst* inst, MixBatchStatus* st, int ninst);
void mb_decide_inner(cudaStream_t s, const MixBatchInst* inst, MixBatchStatus* st, int ninst, int nup);
void mb_finish(cudaStream_t s, const MixBatchInst* inst, MixBatchStatus* st, int ninst);
void mb_start(cudaStream_t s, const MixBatchInst* inst, MixBatchStatus* st, int ninst);
// Resident CTAs per SM of the point and correction kernels.
int mb_points_blocks_per_sm();
int mb_corr_blocks_per_sm(int minb);
// Correction tile extents in x and y (faces per tile).
int corr_tile_x();
int corr_tile_y();

}  // namespace pt
