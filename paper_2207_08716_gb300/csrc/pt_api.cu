// pt_api.cu — host side of the C ABI declared in include/porowave_pt.h.
//
// The context owns no device memory: fields belong to the caller, scratch lives in the
// caller's workspace. Iterate k of the centre fields (Pt, Pf, phi) alternates between the
// caller's arrays and their workspace partners (ping-pong); every API call that returns leaves
// the current iterate in the caller's arrays.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <algorithm>
#include <cstring>
#include <new>
#include <array>
#include <chrono>
#include <utility>
#include <vector>

#include "../../include/porowave_pt.h"
#include "pt_common.cuh"
#include "pt_kernels.cuh"
#include "pt_lean.cuh"
#include "pt_mixed.cuh"
#include "pt_batch.cuh"
#include "pt_adjoint.cuh"
#include "pt_dd.cuh"
#include "pt_host.h"

using namespace pt;

namespace {

constexpr size_t kAlign = 256;
constexpr int kRefArrays = 23;   // step-by-step path
constexpr int kLeanArrays = 26;  // extra arrays of the FP64-lean path
constexpr int kMixArrays = 23;   // FP32 arrays of the mixed-precision path
constexpr int kDfArrays = 28;    // double-float iterate, stresses, residuals, old fields (PT_DF64)
// Default relative drop at which the inner FP32 solves of the mixed-precision path stop. The
// outer loop's convergence is bound by the log-space Picard relaxation of mu and eta (one
// update per outer iteration), not by the inner accuracy: a drop of 0.3 per inner solve needs
// about as many FP32 iterations in total as the FP64 path needs FP64 iterations (measured on
// 32^3-96^3), while 1e-4 needs 3-4 times more.
constexpr double kInnerRtol = 0.1;
// Multigrid V-cycle of the FP32 correction problem (pt_num.mg_levels >= 2): nu1 = nu2 = 2 PT
// sweeps without damping before and after each coarse-grid correction, the velocity pseudo-step
// scaled by 0.8 and the Pf pseudo-step by 6/7 in them (the undamped PT sweep is a Jacobi
// iteration; these weights make it a smoother of the viscous and Darcy operators, whose Jacobi
// weights would otherwise be ~1.1 and ~1), kMgCoarseIters damped PT iterations on the coarsest grid.
constexpr int kMgNu1 = 2, kMgNu2 = 2, kMgCoarseIters = 24, kMgMaxLevels = 10;
constexpr double kMgSmoothV = 0.8, kMgSmoothPf = 6.0 / 7.0;
constexpr int kMgArrays = 25;      // FP32 arrays of one coarse level
constexpr int kMgFineArrays = 2;   // residual outputs of the finest level

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }


}  // namespace

struct pt_ctx {
  Box box;
  Coef coef;
  pt_grid grid;
  pt_grid metric;   // grid whose spacing (and nz) define the coefficients: `grid`, or for a part
                    // of a decomposed grid the whole grid
  pt_phys phys;
  pt_num num;
  cudaStream_t stream;
  // caller's fields
  double *Vx, *Vy, *Vz, *txx, *tyy, *tzz, *txy, *txz, *tyz, *mu, *eta;
  const double* logk;
  double* Pt[2];
  double* Pf[2];
  double* phi[2];
  int cur;  // 0: iterate k in the caller's arrays, 1: in the workspace partners
  // workspace
  double *Pto, *Pfo, *Lo, *txxo, *tyyo, *tzzo, *txyo, *txzo, *tyzo, *Rx, *Ry, *Rz, *perm, *rog;
  double *s_txx, *s_tyy, *s_tzz, *s_txy, *s_txz, *s_tyz;
  // FP64-lean path (precision PT_FP64)
  bool lean;
  double *lperm[2], *lw[2], *phio, *Eo, *iEo;
  double *toa_xx, *toa_yy, *toa_zz, *toa_xy, *toa_xz, *toa_yz, *cm2, *idtp, *ieta;
  double *em2_xy, *em2_xz, *em2_yz, *eb_xy, *eb_xz, *eb_yz, *dtv_x, *dtv_y, *dtv_z, *K0;
  LeanCoef<double> lcoef;
  // double-float path (precision PT_DF64): the lean arrays above hold df64 values; the iterate
  // lives in these df64 arrays between pt_step_begin and the return of each call, the caller's
  // FP64 fields receive it (export) when a call returns
  bool dfm, df_dirty;
  int fcur;
  df64 *fVx, *fVy, *fVz, *fPt[2], *fPf[2], *fphi[2], *fmu, *feta, *fRx, *fRy, *fRz;
  df64 *fs_txx, *fs_tyy, *fs_tzz, *fs_txy, *fs_txz, *fs_tyz;
  df64 *ftxxo, *ftyyo, *ftzzo, *ftxyo, *ftxzo, *ftyzo, *fPto, *fPfo;
  LeanCoef<df64> fcoef;
  // mixed-precision path (precision PT_FP32): FP32 correction problem
  bool mixed;
  double mix_omega;         // PT_FP32: weight of the outer update u <- u + omega delta
  double mix_prev;          // PT_FP32: the previous outer residual max (0 at a step's start)
  float *m_rpt, *m_rpf, *m_rfx, *m_rfy, *m_rfz, *m_cc, *m_perm, *m_idtp, *m_mu, *m_dtvc;
  float *m_dVx[2], *m_dVy[2], *m_dVz[2], *m_dPt[2], *m_dPf[2], *m_Rx, *m_Ry, *m_Rz;
  CorrCoef<float> ccoef;
  // multigrid V-cycle of the correction problem (mg_L >= 2): level 0 = the m_* arrays above
  int mg_L;
  std::vector<MgLevel> mg;
  std::vector<int> mg_d;                           // parity of each level's current iterate
  std::vector<CorrCoef<float>> mg_smooth, mg_eval; // per level: smoothing and evaluation sweeps
  CorrCoef<float> mg_coarse;                       // damped PT on the coarsest grid
  std::vector<float> mg_dtpt, mg_dtv;              // per level: dtau_Pt / mu and dtau_V mu factors
  // adjoint recording (pt_adjoint_forward / pt_adjoint)
  char* adj_ws;
  size_t adj_bytes;
  int adj_nsteps, adj_ckpt;
  std::vector<double> adj_dtS, adj_dtcum;
  std::vector<int> adj_nst;
  unsigned long long* red;       // device reduction block (RED_N slots)
  unsigned long long* h_red;     // pinned host copy
  // stress sub-stepping
  double dtS, dt_cum;
  int nsteps;
  // launch accounting and optional per-kernel event timing
  long long launches;
  bool profiling;
  struct Rec { int kid; cudaEvent_t a, b; };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  size_t pool_used;
};

namespace {

enum KernelId { K_PERM, K_CENTRES, K_EDGES, K_POROSITY, K_FACES, K_PICARD, K_BEGIN, K_INIT_VISC,
                K_RESIDUAL_FACES, K_LEAN_CELLS, K_LEAN_FACES, K_LEAN_PICARD, K_LEAN_COEF, K_LEAN_BEGIN,
                K_LEAN_K0, K_MIX_PREP, K_MIX_FACES, K_MIX_COEF, K_CORR_ITER,
                K_MIX_UPDATE, K_ADJ_PREP, K_ADJ_CELLS, K_ADJ_FACES, K_ADJ_CARRY, K_DF_CELLS, K_DF_FACES,
                K_DF_PICARD, K_DF_COEF, K_DF_BEGIN, K_DF_K0, K_DF_CONVERT, K_ADJ_EDGES_PL, K_ADJ_CELLS_PL,
                K_ADJ_FACES_PL, K_MG_FINE, K_MG_COARSE, K_MG_TRANSFER, K_MIX_EDGES, K_MIX_POROSITY, K_COUNT };
const char* const kKernelNames[K_COUNT] = {"k_perm", "k_centres", "k_edges", "k_porosity", "k_faces",
                                           "k_picard", "k_begin_step", "k_init_visc",
                                           "k_residual_faces", "k_lean_cells", "k_lean_faces",
                                           "k_lean_picard", "k_lean_coef", "k_lean_begin", "k_lean_k0",
                                           "k_mix_prepare", "k_mix_res_faces", "k_mix_coef",
                                           "k_corr_iteration", "k_mix_update",
                                           "k_adj_prep", "k_adj_cells", "k_adj_faces", "k_adj_carry",
                                           "k_lean_cells_df64", "k_lean_faces_df64", "k_lean_picard_df64",
                                           "k_lean_coef_df64", "k_lean_begin_df64", "k_lean_k0_df64",
                                           "k_df64_convert", "k_adj_edges_pl", "k_adj_cells_pl",
                                           "k_adj_faces_pl", "k_corr_iteration_mg_fine",
                                           "k_corr_iteration_mg_coarse", "k_mg_transfer", "k_mix_edges",
                                           "k_mix_porosity"};

cudaEvent_t pooled_event(pt_ctx* c) {
  if (c->pool_used == c->pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    c->pool.push_back(e);
  }
  return c->pool[c->pool_used++];
}

// Launch bracket: counts the launch and, while profiling, records an event pair around it.
struct LaunchScope {
  pt_ctx* c;
  int kid;
  cudaEvent_t b = nullptr;
  LaunchScope(pt_ctx* ctx, int id) : c(ctx), kid(id) {
    c->launches++;
    if (c->profiling) {
      cudaEvent_t a = pooled_event(c);
      b = pooled_event(c);
      if (a && b) {
        cudaEventRecord(a, c->stream);
        c->recs.push_back({kid, a, b});
      } else {
        b = nullptr;
      }
    }
  }
  ~LaunchScope() {
    if (b) cudaEventRecord(b, c->stream);
  }
};
#define PT_LAUNCH(ctx, kid, ...) \
  do {                           \
    LaunchScope scope_(ctx, kid); \
    __VA_ARGS__;                 \
  } while (0)

dim3 block_dims() { return dim3(32, 8, 1); }
dim3 grid_dims(const Box& b) {
  return dim3((unsigned)((b.nx + 1 + 31) / 32), (unsigned)((b.ny + 1 + 7) / 8), (unsigned)(b.nz + 1));
}

void fill_lean_coef(pt_ctx* c);
void fill_corr_coef(pt_ctx* c);

// m when the Picard relaxation weight is 1/m (2 <= m <= 64, to rounding), else 0: the
// double-float path takes x^(1/m) by Newton's m-th root instead of exp(rel log x).
int relax_root(double rel) {
  if (!(rel > 0.0) || !std::isfinite(rel)) return 0;
  const double m = std::nearbyint(1.0 / rel);
  if (m >= 2.0 && m <= 64.0 && std::fabs(m * rel - 1.0) <= 4.0 * 2.220446049250313e-16) return (int)m;
  return 0;
}

// The per-step scalars of the lean form rounded to double-float (each to ~2^-48 relative).
LeanCoef<df64> lean_coef_df64(const LeanCoef<double>& L) {
  LeanCoef<df64> F;
#define PT_DF(x) F.x = df64(L.x)
  PT_DF(rdx); PT_DF(rdy); PT_DF(rdz); PT_DF(hrdx); PT_DF(hrdy); PT_DF(hrdz);
  PT_DF(hrdx2); PT_DF(hrdy2); PT_DF(hrdz2); PT_DF(buoy_dz); PT_DF(bd_rdt); PT_DF(bda_B_rdt);
  PT_DF(alpha); PT_DF(alpha_B); PT_DF(bd_rdt_a); PT_DF(beta_n); PT_DF(beta_phi); PT_DF(dt);
  PT_DF(rphi0); PT_DF(k0); PT_DF(phi0); PT_DF(drho_g); PT_DF(ifac_pf); PT_DF(rrho_i);
  PT_DF(damp_x); PT_DF(damp_y); PT_DF(damp_z); PT_DF(rdx_r); PT_DF(rdy_r); PT_DF(rdz_r);
  PT_DF(drho_g_r); PT_DF(rho_i); PT_DF(ebg); PT_DF(mu0); PT_DF(eta0); PT_DF(R_weak);
  PT_DF(rtau0_2); PT_DF(rGdtS); PT_DF(dtaupt_fac); PT_DF(dtauv_fac);
#undef PT_DF
  F.compaction_on = L.compaction_on;
  F.powerlaw_on = L.powerlaw_on;
  F.bg_on = L.bg_on;
  F.tau0 = L.tau0;
  F.n_pow = L.n_pow;
  F.rel_mu = L.rel_mu;
  F.rel_eta = L.rel_eta;
  F.root_mu = L.root_mu;
  F.root_eta = L.root_eta;
  return F;
}

void fill_coef(pt_ctx* c) {
  c->coef = make_coef(c->metric, c->phys, c->num, c->dtS);
  fill_lean_coef(c);
  fill_corr_coef(c);
}

void fill_lean_coef(pt_ctx* c) {
  const Coef& k = c->coef;
  const pt_grid& g = c->metric;
  const pt_phys& p = c->phys;
  LeanCoef<double>& L = c->lcoef;
  const double dz = g.lz / g.nz;
  L.rdx = k.rdx; L.rdy = k.rdy; L.rdz = k.rdz;
  L.hrdx = 0.5 * k.rdx; L.hrdy = 0.5 * k.rdy; L.hrdz = 0.5 * k.rdz;
  L.hrdx2 = 0.5 * k.rdx * k.rdx; L.hrdy2 = 0.5 * k.rdy * k.rdy; L.hrdz2 = 0.5 * k.rdz * k.rdz;
  L.buoy_dz = (k.rhof_g - k.rho_bg_g) * dz;
  L.ebg = k.ebg;
  L.bg_on = k.bg_on;
  L.bd_rdt = k.beta_d * k.rdt;
  L.bda_B_rdt = k.beta_d * k.alpha / k.B * k.rdt;
  L.alpha = k.alpha;
  L.bd_rdt_a = k.beta_d * k.alpha * k.rdt;
  L.alpha_B = k.alpha / k.B;
  L.beta_n = k.beta_n;
  L.beta_phi = k.beta_phi;
  L.dt = k.dt;
  L.rphi0 = k.rphi0;
  L.k0 = k.k0;
  L.phi0 = k.phi0;
  L.drho_g = p.rhof_g - p.rhos_g;
  L.ifac_pf = 1.0 / k.dtaupf_fac;
  L.rrho_i = k.rrho_i;
  L.rho_i = 1.0 / k.rrho_i;
  L.rdx_r = k.rdx * k.rrho_i; L.rdy_r = k.rdy * k.rrho_i; L.rdz_r = k.rdz * k.rrho_i;
  L.drho_g_r = (p.rhof_g - p.rhos_g) * k.rrho_i;
  L.damp_x = k.damp_x; L.damp_y = k.damp_y; L.damp_z = k.damp_z;
  L.compaction_on = k.compaction_on;
  L.powerlaw_on = k.powerlaw_on;
  L.mu0 = k.mu0; L.eta0 = k.eta0; L.tau0 = k.tau0; L.n_pow = k.n_pow;
  L.rtau0_2 = 1.0 / (k.tau0 * k.tau0);
  L.rel_mu = k.rel_mu; L.rel_eta = k.rel_eta; L.R_weak = k.R_weak;
  L.rGdtS = k.rGdtS;
  L.dtaupt_fac = k.dtaupt_fac;
  L.dtauv_fac = k.dtauv_fac;
  L.root_mu = relax_root(k.rel_mu);
  L.root_eta = relax_root(k.rel_eta);
  c->fcoef = lean_coef_df64(L);
}

CorrCoef<float> corr_coef_of(const Coef& k) {
  CorrCoef<float> f;
  f.rdx = (float)k.rdx; f.rdy = (float)k.rdy; f.rdz = (float)k.rdz;
  f.hrdx = (float)(0.5 * k.rdx); f.hrdy = (float)(0.5 * k.rdy); f.hrdz = (float)(0.5 * k.rdz);
  f.hrdx2 = (float)(0.5 * k.rdx * k.rdx); f.hrdy2 = (float)(0.5 * k.rdy * k.rdy);
  f.hrdz2 = (float)(0.5 * k.rdz * k.rdz);
  f.bd_rdt = (float)(k.beta_d * k.rdt);
  f.bd_rdt_a = (float)(k.beta_d * k.rdt * k.alpha);
  f.bda_B_rdt = (float)(k.beta_d * k.alpha / k.B * k.rdt);
  f.beta_n = (float)k.beta_n;
  f.rrho_i = (float)k.rrho_i;
  f.damp_x = (float)k.damp_x; f.damp_y = (float)k.damp_y; f.damp_z = (float)k.damp_z;
  f.rG = (float)k.rGdtS;
  f.ifac_pf = (float)(1.0 / k.dtaupf_fac);
  return f;
}

// The grid of multigrid level l: each level has ceil(n / 2) cells per direction of the level
// above over the same box lengths (nested for an even n).
pt_grid mg_grid(const pt_grid& g, int l) {
  pt_grid h = g;
  for (int k = 0; k < l; ++k) {
    h.nx = (h.nx + 1) / 2;
    h.ny = (h.ny + 1) / 2;
    h.nz = (h.nz + 1) / 2;
  }
  return h;
}

bool mg_ok(const pt_grid& g, const pt_num& n) {
  if (n.mg_levels <= 1) return n.mg_levels >= 0;
  if (n.precision != PT_FP32 || n.mg_levels > kMgMaxLevels) return false;
  const pt_grid c = mg_grid(g, n.mg_levels - 1);   // the coarsest grid
  return c.nx >= 2 && c.ny >= 2 && c.nz >= 2;
}

// 4-byte words of the transfer tables of one direction (MgAxis) between nf fine and nc coarse cells.
size_t mg_axis_words(int nf, int nc) { return (size_t)9 * nc + (size_t)6 * nf + 7; }

// The transfer tables of one direction, built from the cell and face positions in FP64 (coarse
// cell I spans [I r, (I + 1) r] fine cells, coarse face J sits at J r, r = nf / nc); laid out as
// box_i0[nc], box_w[3 nc], hat_i0[nc + 1], hat_w[4 (nc + 1)], lin_ab[2 nf], lin_w[2 nf],
// fl_n0[nf + 1], fl_t[nf + 1] (MgAxis).
std::vector<uint32_t> mg_axis_tables(int nf, int nc) {
  std::vector<uint32_t> t(mg_axis_words(nf, nc), 0u);
  const double r = (double)nf / nc, rinv = (double)nc / nf;
  int32_t* box_i0 = (int32_t*)t.data();
  float* box_w = (float*)(box_i0 + nc);
  int32_t* hat_i0 = (int32_t*)(box_w + 3 * nc);
  float* hat_w = (float*)(hat_i0 + nc + 1);
  int32_t* lin_ab = (int32_t*)(hat_w + 4 * (nc + 1));
  float* lin_w = (float*)(lin_ab + 2 * nf);
  int32_t* fl_n0 = (int32_t*)(lin_w + 2 * nf);
  float* fl_t = (float*)(fl_n0 + nf + 1);
  for (int I = 0; I < nc; ++I) {   // covered fractions of fine cells i0, i0 + 1, i0 + 2
    const double a = I * r, b = (I + 1) * r;
    const int i0 = (int)std::floor(a);
    box_i0[I] = i0;
    for (int k = 0; k < 3; ++k) {
      const int i = i0 + k;
      const double lo = std::max(a, (double)i), hi = std::min(b, (double)(i + 1));
      box_w[3 * I + k] = (i < nf && hi > lo) ? (float)((hi - lo) / r) : 0.f;
    }
  }
  for (int J = 0; J <= nc; ++J) {  // normalised hat of half-width r around face J
    const double X = J * r;
    const int i0 = std::max((int)std::floor(X - r) + 1, 0);
    hat_i0[J] = i0;
    double w[4], sum = 0.0;
    for (int k = 0; k < 4; ++k) {
      const int i = i0 + k;
      const double v = i <= nf ? 1.0 - std::fabs(i - X) / r : 0.0;
      w[k] = v > 0.0 ? v : 0.0;
      sum += w[k];
    }
    for (int k = 0; k < 4; ++k) hat_w[4 * J + k] = sum > 0.0 ? (float)(w[k] / sum) : 0.f;
  }
  for (int i = 0; i < nf; ++i) {   // fine centre between two coarse centres (held beyond the ends)
    const double s = (i + 0.5) * rinv - 0.5;
    int i0 = (int)std::floor(s);
    double u = s - i0;
    if (i0 < 0) { i0 = 0; u = 0.0; }
    if (i0 >= nc - 1) { i0 = nc - 1; u = 0.0; }
    lin_ab[2 * i] = i0;
    lin_ab[2 * i + 1] = std::min(i0 + 1, nc - 1);
    lin_w[2 * i] = (float)(1.0 - u);
    lin_w[2 * i + 1] = (float)u;
  }
  for (int i = 0; i <= nf; ++i) {  // fine face between two coarse faces
    const double s = i * rinv;
    int n0 = std::min((int)std::floor(s), nc - 1);
    fl_n0[i] = n0;
    fl_t[i] = (float)(s - n0);
  }
  return t;
}

MgAxis mg_axis_at(char* base, int nf, int nc) {
  MgAxis a;
  int32_t* box_i0 = (int32_t*)base;
  float* box_w = (float*)(box_i0 + nc);
  int32_t* hat_i0 = (int32_t*)(box_w + 3 * nc);
  float* hat_w = (float*)(hat_i0 + nc + 1);
  int32_t* lin_ab = (int32_t*)(hat_w + 4 * (nc + 1));
  float* lin_w = (float*)(lin_ab + 2 * nf);
  int32_t* fl_n0 = (int32_t*)(lin_w + 2 * nf);
  float* fl_t = (float*)(fl_n0 + nf + 1);
  a.box_i0 = box_i0; a.box_w = box_w; a.hat_i0 = hat_i0; a.hat_w = hat_w;
  a.lin_ab = lin_ab; a.lin_w = lin_w; a.fl_n0 = fl_n0; a.fl_t = fl_t;
  return a;
}

// Workspace of the V-cycle's grids: the finest level's residual outputs, kMgArrays per coarser
// level and its transfer tables.
size_t mg_bytes(const pt_grid& g, const pt_num& n) {
  if (n.mg_levels < 2 || !mg_ok(g, n)) return 0;
  size_t total = kMgFineArrays * align_up((size_t)make_box(&g).n * sizeof(float), kAlign);
  for (int l = 1; l < n.mg_levels; ++l) {
    const pt_grid gl = mg_grid(g, l), gf = mg_grid(g, l - 1);
    total += kMgArrays * align_up((size_t)make_box(&gl).n * sizeof(float), kAlign);
    total += align_up(mg_axis_words(gf.nx, gl.nx) * 4, kAlign) + align_up(mg_axis_words(gf.ny, gl.ny) * 4, kAlign) +
             align_up(mg_axis_words(gf.nz, gl.nz) * 4, kAlign);
  }
  return total;
}

// Per-level coefficient sets of the V-cycle (they depend on the step's dtS through xi).
void fill_mg_coef(pt_ctx* c) {
  if (c->mg_L < 2) return;
  for (int l = 0; l < c->mg_L; ++l) {
    pt_num nl = c->num;
    for (int d = 0; d < 3; ++d)   // damping defect 1 - damp grows with the grid spacing
      nl.damp[d] = std::max(0.0, 1.0 - (1.0 - c->num.damp[d]) * (double)(1 << l));
    const Coef k = make_coef(mg_grid(c->metric, l), c->phys, nl, c->dtS);
    CorrCoef<float> sm = corr_coef_of(k), ev = sm;
    sm.damp_x = sm.damp_y = sm.damp_z = 0.0f;
    sm.rrho_i = (float)(k.rrho_i * kMgSmoothV);
    sm.ifac_pf = (float)(1.0 / (k.dtaupf_fac * kMgSmoothPf));
    ev.damp_x = ev.damp_y = ev.damp_z = 0.0f;
    c->mg_smooth[l] = sm;
    c->mg_eval[l] = ev;
    c->mg_dtpt[l] = (float)k.dtaupt_fac;
    c->mg_dtv[l] = (float)k.dtauv_fac;
    if (l == c->mg_L - 1) c->mg_coarse = corr_coef_of(k);
  }
}

void fill_corr_coef(pt_ctx* c) {
  c->ccoef = corr_coef_of(c->coef);
  fill_mg_coef(c);
}

int cuda_status(cudaError_t e) { return e == cudaSuccess ? PT_OK : PT_ECUDA; }

void df_export(pt_ctx* c);

int sync_current_to_caller(pt_ctx* c) {
  if (c->dfm) {
    df_export(c);
    return cuda_status(cudaGetLastError());
  }
  if (c->cur == 0) return PT_OK;
  const size_t bytes = (size_t)c->box.n * sizeof(double);
  cudaError_t e = cudaMemcpyAsync(c->Pt[0], c->Pt[1], bytes, cudaMemcpyDeviceToDevice, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->Pf[0], c->Pf[1], bytes, cudaMemcpyDeviceToDevice, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->phi[0], c->phi[1], bytes, cudaMemcpyDeviceToDevice, c->stream);
  if (c->lean) {
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->lw[0], c->lw[1], bytes, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->lperm[0], c->lperm[1], bytes, cudaMemcpyDeviceToDevice, c->stream);
  }
  c->cur = 0;
  return cuda_status(e);
}

// One PT iteration number `it` (1-based); check = Picard update + norms.
void launch_iteration_lean(pt_ctx* c, int check);
void launch_iteration_df(pt_ctx* c, int check);

void launch_iteration(pt_ctx* c, int check) {
  if (c->dfm) {
    launch_iteration_df(c, check);
    return;
  }
  if (c->lean) {
    launch_iteration_lean(c, check);
    return;
  }
  const Box& b = c->box;
  const Coef& k = c->coef;
  const dim3 bl = block_dims(), gr = grid_dims(b);
  const int a = c->cur, n = 1 - c->cur;
  if (check) cudaMemsetAsync(c->red, 0, RED_N * sizeof(unsigned long long), c->stream);
  PT_LAUNCH(c, K_PERM, k_perm<<<gr, bl, 0, c->stream>>>(b, k, c->phi[a], c->logk, c->perm, c->rog));
  CentreIn ci{c->Vx, c->Vy, c->Vz, c->Pt[a], c->Pf[a], c->phi[a], c->mu, c->eta, c->perm,
              c->Pto, c->Pfo, c->txxo, c->tyyo, c->tzzo};
  CentreOut co{c->Pt[n], c->Pf[n], c->s_txx, c->s_tyy, c->s_tzz};
  PT_LAUNCH(c, K_CENTRES, k_centres<<<gr, bl, 0, c->stream>>>(b, k, ci, co, 1, c->red, check));
  EdgeIn ei{c->Vx, c->Vy, c->Vz, c->mu, c->txyo, c->txzo, c->tyzo};
  EdgeOut eo{c->s_txy, c->s_txz, c->s_tyz};
  PT_LAUNCH(c, K_EDGES, k_edges<<<gr, bl, 0, c->stream>>>(b, k, ei, eo));
  PT_LAUNCH(c, K_POROSITY,
            k_porosity<<<gr, bl, 0, c->stream>>>(b, k, c->Vx, c->Vy, c->Vz, c->phi[a], c->Pt[n],
                                                  c->Pf[n], c->Pto, c->Pfo, c->Lo, c->eta, c->phi[n]));
  FaceIn fi{c->s_txx, c->s_tyy, c->s_tzz, c->s_txy, c->s_txz, c->s_tyz, c->Pt[n], c->rog, c->mu};
  PT_LAUNCH(c, K_FACES,
            k_faces<<<gr, bl, 0, c->stream>>>(b, k, fi, c->Vx, c->Vy, c->Vz, c->Rx, c->Ry, c->Rz, c->red, check));
  if (check) {
    PicardIn pi{c->s_txx, c->s_tyy, c->s_tzz, c->s_txy, c->s_txz, c->s_tyz, c->phi[n], c->Pt[n], c->Pf[n]};
    PT_LAUNCH(c, K_PICARD, k_picard<<<gr, bl, 0, c->stream>>>(b, k, pi, c->mu, c->eta, c->red, 1));
  }
  c->cur = n;
}

void launch_lean_coef(pt_ctx* c) {
  const Box& b = c->box;
  LeanCoefIn<double> ci{c->mu, c->eta, c->txxo, c->tyyo, c->tzzo, c->txyo, c->txzo, c->tyzo};
  LeanCoefOut<double> co{c->cm2, c->toa_xx, c->toa_yy, c->toa_zz, c->idtp, c->ieta, c->em2_xy,
                         c->em2_xz, c->em2_yz, c->eb_xy, c->eb_xz, c->eb_yz, c->toa_xy, c->toa_xz, c->toa_yz,
                         c->dtv_x, c->dtv_y,
                         c->dtv_z};
  PT_LAUNCH(c, K_LEAN_COEF, lean_coef<double>(grid_dims(b), block_dims(), c->stream, b, c->lcoef, ci, co));
}

// One PT iteration of the FP64-lean form: cells (pressures, stresses, porosity), faces
// (momentum, velocities), and on check iterations the Picard update and coefficient refresh.
void launch_iteration_lean(pt_ctx* c, int check) {
  const Box& b = c->box;
  const dim3 bl = block_dims(), gr = grid_dims(b);
  const int a = c->cur, n = 1 - c->cur;
  if (check) cudaMemsetAsync(c->red, 0, RED_N * sizeof(unsigned long long), c->stream);
  LeanCellIn<double> ci{c->Vx, c->Vy, c->Vz, c->Pt[a], c->Pf[a], c->phi[a], c->lw[a], c->lperm[a],
                        c->Pto, c->Pfo, c->phio, c->Eo, c->iEo, c->ieta, c->idtp, c->cm2,
                        c->toa_xx, c->toa_yy, c->toa_zz, c->em2_xy, c->em2_xz, c->em2_yz, c->eb_xy,
                        c->eb_xz, c->eb_yz,
                        c->toa_xy, c->toa_xz, c->toa_yz, c->logk ? c->K0 : nullptr};
  LeanCellOut<double> co{c->Pt[n], c->Pf[n], c->phi[n], c->lw[n], c->lperm[n], c->s_txx, c->s_tyy,
                         c->s_tzz, c->s_txy, c->s_txz, c->s_tyz};
  PT_LAUNCH(c, K_LEAN_CELLS, lean_cells<double>(gr, bl, c->stream, b, c->lcoef, ci, co, c->red, check));
  LeanFaceIn<double> fi{c->s_txx, c->s_tyy, c->s_tzz, c->s_txy, c->s_txz, c->s_tyz, c->Pt[n],
                        c->phi[a], c->dtv_x, c->dtv_y, c->dtv_z};
  PT_LAUNCH(c, K_LEAN_FACES, lean_faces<double>(gr, bl, c->stream, b, c->lcoef, fi, c->Vx, c->Vy, c->Vz, c->Rx,
                                                   c->Ry, c->Rz, c->red, check));
  if (check) {
    LeanPicardIn<double> pi{c->s_txx, c->s_tyy, c->s_tzz, c->s_txy, c->s_txz, c->s_tyz, c->phi[n],
                            c->Pt[n], c->Pf[n]};
    PT_LAUNCH(c, K_LEAN_PICARD, lean_picard<double>(gr, bl, c->stream, b, c->lcoef, pi, c->mu, c->eta, c->red));
    launch_lean_coef(c);
  }
  c->cur = n;
}

// ------------------------------------------------------ double-float path (PT_DF64)
// The lean-form kernels instantiated for df64: the same per-point code on double-float values,
// the lean arrays of the workspace reinterpreted (8 bytes per element either way).
df64* D(double* p) { return reinterpret_cast<df64*>(p); }

void df_convert(pt_ctx* c, double* const* d, df64* const* f, int n, bool to_df) {
  DfCopy cp;
  std::memset(&cp, 0, sizeof cp);
  for (int i = 0; i < n; ++i) {
    cp.d[i] = d[i];
    cp.f[i] = f[i];
  }
  PT_LAUNCH(c, K_DF_CONVERT, df64_convert(c->stream, cp, n, c->box.n, to_df));
}

// The caller's FP64 fields -> the double-float iterate (buffer 0).
void df_import(pt_ctx* c) {
  double* const d[8] = {c->Vx, c->Vy, c->Vz, c->Pt[0], c->Pf[0], c->phi[0], c->mu, c->eta};
  df64* const f[8] = {c->fVx, c->fVy, c->fVz, c->fPt[0], c->fPf[0], c->fphi[0], c->fmu, c->feta};
  df_convert(c, d, f, 8, true);
  c->fcur = 0;
  c->df_dirty = false;
}

// The double-float iterate -> the caller's FP64 fields (when iterations ran since the last one).
void df_export(pt_ctx* c) {
  if (!c->df_dirty) return;
  const int a = c->fcur;
  double* const d[8] = {c->Vx, c->Vy, c->Vz, c->Pt[0], c->Pf[0], c->phi[0], c->mu, c->eta};
  df64* const f[8] = {c->fVx, c->fVy, c->fVz, c->fPt[a], c->fPf[a], c->fphi[a], c->fmu, c->feta};
  df_convert(c, d, f, 8, false);
  c->df_dirty = false;
}

void launch_df_coef(pt_ctx* c) {
  const Box& b = c->box;
  LeanCoefIn<df64> ci{c->fmu, c->feta, c->ftxxo, c->ftyyo, c->ftzzo, c->ftxyo, c->ftxzo, c->ftyzo};
  LeanCoefOut<df64> co{D(c->cm2), D(c->toa_xx), D(c->toa_yy), D(c->toa_zz), D(c->idtp), D(c->ieta),
                       D(c->em2_xy), D(c->em2_xz), D(c->em2_yz), D(c->eb_xy), D(c->eb_xz), D(c->eb_yz),
                       D(c->toa_xy), D(c->toa_xz), D(c->toa_yz), D(c->dtv_x), D(c->dtv_x), D(c->dtv_x)};
  // (double-float form: em2_* hold the raw edge moduli, dtv_x the per-centre velocity pseudo-step)
  PT_LAUNCH(c, K_DF_COEF, lean_coef<df64>(grid_dims(b), block_dims(), c->stream, b, c->fcoef, ci, co));
}

// The cells kernel's inputs at double-float iterate a, outputs into buffer n.
void df_cells(pt_ctx* c, int a, int n, int check) {
  const Box& b = c->box;
  LeanCellIn<df64> ci{c->fVx, c->fVy, c->fVz, c->fPt[a], c->fPf[a], c->fphi[a], D(c->lw[a]), D(c->lperm[a]),
                      c->fPto, c->fPfo, D(c->phio), D(c->Eo), D(c->iEo), D(c->ieta), D(c->idtp), D(c->cm2),
                      D(c->toa_xx), D(c->toa_yy), D(c->toa_zz), D(c->em2_xy), D(c->em2_xz), D(c->em2_yz),
                      D(c->eb_xy), D(c->eb_xz), D(c->eb_yz), D(c->toa_xy), D(c->toa_xz), D(c->toa_yz),
                      c->logk ? D(c->K0) : nullptr};
  LeanCellOut<df64> co{c->fPt[n], c->fPf[n], c->fphi[n], D(c->lw[n]), D(c->lperm[n]), c->fs_txx, c->fs_tyy,
                       c->fs_tzz, c->fs_txy, c->fs_txz, c->fs_tyz};
  PT_LAUNCH(c, K_DF_CELLS, lean_cells<df64>(grid_dims(b), block_dims(), c->stream, b, c->fcoef, ci, co, c->red, check));
}

// One PT iteration in double-float: the lean form's kernels on the df64 iterate.
void launch_iteration_df(pt_ctx* c, int check) {
  const Box& b = c->box;
  const dim3 bl = block_dims(), gr = grid_dims(b);
  const int a = c->fcur, n = 1 - a;
  if (check) cudaMemsetAsync(c->red, 0, RED_N * sizeof(unsigned long long), c->stream);
  df_cells(c, a, n, check);
  LeanFaceIn<df64> fi{c->fs_txx, c->fs_tyy, c->fs_tzz, c->fs_txy, c->fs_txz, c->fs_tyz, c->fPt[n],
                      c->fphi[a], D(c->dtv_x), D(c->dtv_x), D(c->dtv_x)};
  PT_LAUNCH(c, K_DF_FACES, lean_faces<df64>(gr, bl, c->stream, b, c->fcoef, fi, c->fVx, c->fVy, c->fVz, c->fRx,
                                            c->fRy, c->fRz, c->red, check));
  if (check) {
    LeanPicardIn<df64> pi{c->fs_txx, c->fs_tyy, c->fs_tzz, c->fs_txy, c->fs_txz, c->fs_tyz, c->fphi[n],
                          c->fPt[n], c->fPf[n]};
    PT_LAUNCH(c, K_DF_PICARD, lean_picard<df64>(gr, bl, c->stream, b, c->fcoef, pi, c->fmu, c->feta, c->red));
    launch_df_coef(c);
  }
  c->fcur = n;
  c->df_dirty = true;
}

// End of a double-float step: the stresses of the final state (one cells evaluation at the
// current iterate; its pressure and porosity outputs land in the idle buffers and are dropped),
// written to the caller's stress fields together with the iterate.
int df_step_end(pt_ctx* c) {
  const int a = c->fcur;
  df_cells(c, a, 1 - a, 0);
  double* const d[6] = {c->txx, c->tyy, c->tzz, c->txy, c->txz, c->tyz};
  df64* const f[6] = {c->fs_txx, c->fs_tyy, c->fs_tzz, c->fs_txy, c->fs_txz, c->fs_tyz};
  df_convert(c, d, f, 6, false);
  df_export(c);
  return cuda_status(cudaGetLastError());
}

int read_report(pt_ctx* c, pt_report* rep) {
  cudaError_t e = cudaMemcpyAsync(c->h_red, c->red, RED_N * sizeof(unsigned long long),
                                  cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return PT_ECUDA;
  auto val = [&](int s) {
    double d;
    std::memcpy(&d, &c->h_red[s], sizeof d);
    return d;
  };
  rep->res_v = val(RED_V);
  rep->res_pt = val(RED_PT);
  rep->res_pf = val(RED_PF);
  rep->res_pic = val(RED_PIC);
  const bool finite = std::isfinite(rep->res_v) && std::isfinite(rep->res_pt) &&
                      std::isfinite(rep->res_pf) && std::isfinite(rep->res_pic);
  return finite ? PT_OK : PT_ENAN;
}

double report_max(const pt_report* r) {
  return std::fmax(std::fmax(r->res_v, r->res_pt), std::fmax(r->res_pf, r->res_pic));
}

// ---- multigrid V-cycle of the FP32 correction problem
// One sweep of the correction iteration on level l with coefficient set `cf`: from the level's
// current buffers into the other ones (then they become current), or, with eval, the residuals
// of the current iterate only (R = momentum residual / rho_i, rho_Pt and rho_Pf into res_*).
void mg_sweep(pt_ctx* c, int l, const CorrCoef<float>& cf, int eval, int check) {
  const MgLevel& L = c->mg[l];
  const int d = c->mg_d[l];
  const CorrIn<float> in{L.dVx[d], L.dVy[d], L.dVz[d], L.dPt[d], L.dPf[d], L.cc, L.perm, L.idtp, L.rpt, L.rpf,
                         L.mu, L.dtvc, L.rfx, L.rfy, L.rfz};
  const CorrOut<float> out{L.dVx[1 - d], L.dVy[1 - d], L.dVz[1 - d], L.dPt[1 - d], L.dPf[1 - d], L.Rx, L.Ry, L.Rz,
                           eval ? L.res_pt : nullptr, eval ? L.res_pf : nullptr, eval};
  PT_LAUNCH(c, l == 0 ? K_MG_FINE : K_MG_COARSE, corr_iteration(c->stream, L.b, cf, in, out, c->red, check));
  if (!eval) c->mg_d[l] = 1 - d;
}

// V-cycle on level l for the current right-hand sides: pre-smoothing, residual, restriction to a
// zero coarse correction, the coarse cycle (damped PT iterations on the coarsest grid),
// prolongation of the correction, post-smoothing.
void mg_vcycle(pt_ctx* c, int l) {
  if (l == c->mg_L - 1) {
    for (int s = 0; s < kMgCoarseIters; ++s) mg_sweep(c, l, c->mg_coarse, 0, 0);
    return;
  }
  for (int s = 0; s < kMgNu1; ++s) mg_sweep(c, l, c->mg_smooth[l], 0, 0);
  mg_sweep(c, l, c->mg_eval[l], 1, 0);
  PT_LAUNCH(c, K_MG_TRANSFER, mg_restrict(c->stream, c->mg[l], c->mg[l + 1], (float)c->num.rho_i));
  c->mg_d[l + 1] = 0;
  mg_vcycle(c, l + 1);
  PT_LAUNCH(c, K_MG_TRANSFER, mg_prolong(c->stream, c->mg[l + 1], c->mg_d[l + 1], c->mg[l], c->mg_d[l]));
  for (int s = 0; s < kMgNu2; ++s) mg_sweep(c, l, c->mg_smooth[l], 0, 0);
}

// One outer iteration of the mixed-precision path (see pt_mixed_kernels.cu): FP64 residuals
// and Picard update at u, then up to n_in FP32 PT iterations on the correction (stopping early
// at a relative drop kInnerRtol when early_exit), u <- u + delta, FP64 porosity update.
// `outer` receives the FP64 residual norms at u; *converged is set when they are below tol
// (then no correction is run).
int mixed_outer(pt_ctx* c, int n_in, bool early_exit, pt_report* outer, bool* converged, int* inner_done) {
  const Box& b = c->box;
  const Coef& k = c->coef;
  const dim3 bl = block_dims(), gr = grid_dims(b);
  const int a = c->cur;
  *converged = false;
  *inner_done = 0;
  cudaMemsetAsync(c->red, 0, RED_N * sizeof(unsigned long long), c->stream);
  // (i) FP64 residuals at u, frozen coefficients of the correction problem
  PT_LAUNCH(c, K_PERM, k_perm<<<gr, bl, 0, c->stream>>>(b, k, c->phi[a], c->logk, c->perm, c->rog));
  MixPrepIn pin{c->Vx, c->Vy, c->Vz, c->Pt[a], c->Pf[a], c->phi[a], c->mu, c->eta, c->perm, c->Pto,
                c->Pfo, c->txxo, c->tyyo, c->tzzo};
  MixPrepOut pout{c->s_txx, c->s_tyy, c->s_tzz, c->m_rpt, c->m_rpf, c->m_cc, c->m_perm, c->m_idtp};
  PT_LAUNCH(c, K_MIX_PREP, mix_prepare(gr, bl, c->stream, b, k, pin, pout, c->red));
  EdgeIn ei{c->Vx, c->Vy, c->Vz, c->mu, c->txyo, c->txzo, c->tyzo};
  EdgeOut eo{c->s_txy, c->s_txz, c->s_tyz};
  PT_LAUNCH(c, K_MIX_EDGES, mix_edges(gr, bl, c->stream, b, k, ei, eo));
  MixFaceIn fin{c->s_txx, c->s_tyy, c->s_tzz, c->s_txy, c->s_txz, c->s_tyz, c->Pt[a], c->phi[a]};
  PT_LAUNCH(c, K_MIX_FACES, mix_res_faces(gr, bl, c->stream, b, k, fin, c->m_rfx, c->m_rfy, c->m_rfz, c->red));
  // (ii) Picard update of mu, eta from the stresses at u
  LeanPicardIn<double> pi{c->s_txx, c->s_tyy, c->s_tzz, c->s_txy, c->s_txz, c->s_tyz, c->phi[a],
                          c->Pt[a], c->Pf[a]};
  PT_LAUNCH(c, K_LEAN_PICARD, lean_picard<double>(gr, bl, c->stream, b, c->lcoef, pi, c->mu, c->eta, c->red));
  if (cudaGetLastError() != cudaSuccess) return PT_ECUDA;
  int rc = read_report(c, outer);
  if (rc != PT_OK) return rc;
  if (early_exit && report_max(outer) < c->num.tol) {
    *converged = true;
    return PT_OK;
  }
  // globalisation of the outer loop: when the last update more than doubled the FP64 residual,
  // halve the weight of the next ones (down to 1/16); while it falls, let the weight grow back
  // to 1 (the fixed point does not depend on the weight)
  {
    const double r = report_max(outer);
    if (c->mix_prev > 0.0) {
      if (r > 2.0 * c->mix_prev) c->mix_omega = std::max(c->mix_omega * 0.5, 0.0625);
      else if (r < c->mix_prev) c->mix_omega = std::min(c->mix_omega * 1.25, 1.0);
    }
    c->mix_prev = r;
  }
  const double target = (c->num.inner_rtol > 0 ? c->num.inner_rtol : kInnerRtol) * report_max(outer);
  // (iii) FP32 PT on the correction, from delta = 0, R = 0
  MixCoefOut mco{c->m_mu, c->m_dtvc};
  PT_LAUNCH(c, K_MIX_COEF, mix_coef(gr, bl, c->stream, b, k, c->mu, mco));
  const size_t fb = (size_t)b.n * sizeof(float);
  // both correction-velocity buffers: the wall faces, never written by the iteration, stay zero
  float* zero[] = {c->m_dVx[0], c->m_dVy[0], c->m_dVz[0], c->m_dVx[1], c->m_dVy[1], c->m_dVz[1],
                   c->m_dPt[0], c->m_dPf[0], c->m_Rx, c->m_Ry, c->m_Rz};
  for (float* z : zero) cudaMemsetAsync(z, 0, fb, c->stream);
  int d = 0;
  const int nup = c->num.nup;
  if (c->mg_L >= 2) {
    // V-cycles until the same relative drop (checked by an evaluation sweep after each cycle) or
    // the budget; a cycle counts its finest-grid sweeps
    for (int l = 1; l < c->mg_L; ++l)
      PT_LAUNCH(c, K_MG_TRANSFER, mg_coef(c->stream, c->mg[l - 1], c->mg[l], c->mg_dtpt[l], c->mg_dtv[l]));
    c->mg_d[0] = 0;
    int it = 0;
    while (it < n_in) {
      mg_vcycle(c, 0);
      it += kMgNu1 + kMgNu2 + 1;
      *inner_done = it;
      if (!early_exit) continue;
      cudaMemsetAsync(c->red, 0, RED_N * sizeof(unsigned long long), c->stream);
      mg_sweep(c, 0, c->mg_eval[0], 1, 1);
      *inner_done = ++it;
      pt_report ir;
      rc = read_report(c, &ir);
      if (rc != PT_OK) return rc;
      if (std::fmax(std::fmax(ir.res_v, ir.res_pt), ir.res_pf) < target) break;
    }
    d = c->mg_d[0];
  }
  for (int it = 1; it <= n_in && c->mg_L < 2; ++it) {
    const int check = early_exit && (it % nup) == 0;
    if (check) cudaMemsetAsync(c->red, 0, RED_N * sizeof(unsigned long long), c->stream);
    const CorrIn<float> ci{c->m_dVx[d], c->m_dVy[d], c->m_dVz[d], c->m_dPt[d], c->m_dPf[d], c->m_cc, c->m_perm,
                           c->m_idtp, c->m_rpt, c->m_rpf, c->m_mu, c->m_dtvc, c->m_rfx, c->m_rfy, c->m_rfz};
    const CorrOut<float> co{c->m_dVx[1 - d], c->m_dVy[1 - d], c->m_dVz[1 - d], c->m_dPt[1 - d], c->m_dPf[1 - d],
                            c->m_Rx, c->m_Ry, c->m_Rz};
    PT_LAUNCH(c, K_CORR_ITER, corr_iteration(c->stream, b, c->ccoef, ci, co, c->red, check));
    d = 1 - d;
    *inner_done = it;
    if (check) {
      pt_report ir;
      rc = read_report(c, &ir);
      if (rc != PT_OK) return rc;
      if (std::fmax(std::fmax(ir.res_v, ir.res_pt), ir.res_pf) < target) break;
    }
  }
  // (iv) u <- u + delta in FP64, then the FP64 porosity time integration (Eq. 22, log space)
  MixUpdate mu{c->Vx, c->Vy, c->Vz, c->Pt[a], c->Pf[a], c->m_dVx[d], c->m_dVy[d], c->m_dVz[d], c->m_dPt[d], c->m_dPf[d],
               c->mix_omega};
  PT_LAUNCH(c, K_MIX_UPDATE, mix_update(gr, bl, c->stream, b, mu));
  PT_LAUNCH(c, K_MIX_POROSITY,
            mix_porosity(gr, bl, c->stream, b, k,
                         MixPorosity{c->Vx, c->Vy, c->Vz, c->phi[a], c->Pt[a], c->Pf[a], c->Pto, c->Pfo, c->Lo,
                                     c->eta, c->phi[1 - a]}));
  // Pt, Pf stay in buffer a; phi moves to 1 - a: copy the pressures along so cur stays paired
  cudaMemcpyAsync(c->Pt[1 - a], c->Pt[a], (size_t)b.n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
  cudaMemcpyAsync(c->Pf[1 - a], c->Pf[a], (size_t)b.n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
  c->cur = 1 - a;
  return cuda_status(cudaGetLastError());
}

// Step begin in three parts (a decomposed grid takes the largest mu over all its parts):
// old-state snapshot and the largest mu into the reduction block; read it; stress sub-step,
// old-stress refresh and coefficients from it.
int step_begin_launch(pt_ctx* c) {
  int rc = sync_current_to_caller(c);
  if (rc != PT_OK) return rc;
  const Box& b = c->box;
  cudaMemsetAsync(c->red, 0, RED_N * sizeof(unsigned long long), c->stream);
  if (c->dfm) {
    // the caller's fields become the double-float iterate; the FP64 old pressures are kept too
    // (pt_residual evaluates the FP64 residual of the caller's fields)
    df_import(c);
    const size_t bytes = (size_t)b.n * sizeof(double);
    cudaMemcpyAsync(c->Pto, c->Pt[0], bytes, cudaMemcpyDeviceToDevice, c->stream);
    cudaMemcpyAsync(c->Pfo, c->Pf[0], bytes, cudaMemcpyDeviceToDevice, c->stream);
    LeanBeginIn<df64> bi{c->fPt[0], c->fPf[0], c->fphi[0], c->fmu, c->logk ? D(c->K0) : nullptr};
    LeanBeginOut<df64> bo{c->fPto, c->fPfo, D(c->phio), D(c->Eo), D(c->iEo), D(c->lw[0]), D(c->lperm[0])};
    PT_LAUNCH(c, K_DF_BEGIN, lean_begin<df64>(grid_dims(b), block_dims(), c->stream, b, c->fcoef, bi, bo, c->red));
  } else if (c->lean) {
    LeanBeginIn<double> bi{c->Pt[0], c->Pf[0], c->phi[0], c->mu, c->logk ? c->K0 : nullptr};
    LeanBeginOut<double> bo{c->Pto, c->Pfo, c->phio, c->Eo, c->iEo, c->lw[0], c->lperm[0]};
    PT_LAUNCH(c, K_LEAN_BEGIN, lean_begin<double>(grid_dims(b), block_dims(), c->stream, b, c->lcoef, bi, bo, c->red));
  } else {
    PT_LAUNCH(c, K_BEGIN, k_begin_step<<<grid_dims(b), block_dims(), 0, c->stream>>>(
                               b, c->Pt[0], c->Pf[0], c->phi[0], c->mu, c->Pto, c->Pfo, c->Lo, c->red));
  }
  return cuda_status(cudaGetLastError());
}

int step_begin_mumax(pt_ctx* c, double* mu_max) {
  cudaError_t e =
      cudaMemcpyAsync(c->h_red, c->red, RED_N * sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return PT_ECUDA;
  std::memcpy(mu_max, &c->h_red[RED_MUMAX], sizeof *mu_max);
  return PT_OK;
}

int step_begin_finish(pt_ctx* c, double mu_max) {
  if (!std::isfinite(mu_max) || !(mu_max > 0)) return PT_ENAN;
  const Box& b = c->box;
  cudaError_t e = cudaSuccess;
  // stress sub-step of the appendix two-phase script: the largest xi = mu / (G dtS) is xsi_w;
  // the old stresses are refreshed at the first step and when dt_cum reaches dtS
  c->dtS = mu_max / (c->phys.G * c->num.xsi_w);
  if (c->nsteps == 0 || c->dt_cum >= c->dtS) {
    const size_t bytes = (size_t)b.n * sizeof(double);
    const double* src[6] = {c->txx, c->tyy, c->tzz, c->txy, c->txz, c->tyz};
    double* dst[6] = {c->txxo, c->tyyo, c->tzzo, c->txyo, c->txzo, c->tyzo};
    for (int s = 0; s < 6 && e == cudaSuccess; ++s)
      e = cudaMemcpyAsync(dst[s], src[s], bytes, cudaMemcpyDeviceToDevice, c->stream);
    if (c->dfm && e == cudaSuccess) {
      df64* const f[6] = {c->ftxxo, c->ftyyo, c->ftzzo, c->ftxyo, c->ftxzo, c->ftyzo};
      df_convert(c, dst, f, 6, true);
    }
    c->dt_cum = 0.0;
  }
  c->nsteps += 1;
  fill_coef(c);
  if (c->lean && e == cudaSuccess) {
    launch_lean_coef(c);
    e = cudaGetLastError();
  }
  if (c->dfm && e == cudaSuccess) {
    launch_df_coef(c);
    e = cudaGetLastError();
  }
  return cuda_status(e);
}

}  // namespace

extern "C" {

size_t pt_field_elems(const pt_grid* grid) {
  if (!grid_ok(grid)) return 0;
  return (size_t)make_box(grid).n;
}

int32_t pt_pitch_x(const pt_grid* grid) {
  if (!grid_ok(grid)) return 0;
  return make_box(grid).px;
}

size_t pt_workspace_size(const pt_grid* grid, const pt_num* num) {
  if (!grid_ok(grid) || !num) return 0;
  const Box b = make_box(grid);
  const bool df = num->precision == PT_DF64;
  const int arrays = kRefArrays + ((num->precision == PT_FP64 || df) ? kLeanArrays : 0) + (df ? kDfArrays : 0);
  const size_t mixed = num->precision == PT_FP32 ? kMixArrays * align_up((size_t)b.n * sizeof(float), kAlign) : 0;
  return arrays * align_up((size_t)b.n * sizeof(double), kAlign) + mixed + mg_bytes(*grid, *num) + kAlign;
}

int pt_init(pt_ctx** ctx, const pt_grid* grid, const pt_phys* phys, const pt_num* num,
            const pt_fields* f, void* workspace, size_t workspace_bytes, void* stream,
            int32_t keep_visc) {
  if (!ctx) return PT_EINVAL;
  *ctx = nullptr;
  if (!grid_ok(grid) || !phys || !num || !f || !workspace) return PT_EINVAL;
  if (!(num->dt > 0) || !std::isfinite(num->dt) || num->nup < 1 || num->max_iter < 0 || !(num->tol >= 0))
    return PT_EINVAL;
  if (!(num->rho_i > 0) || !(num->cfl_v > 0) || !(num->cfl_pf > 0) || !(num->dtpt_scale > 0) ||
      !(num->xsi_w > 0))
    return PT_EINVAL;
  if (num->precision != PT_FP64 && num->precision != PT_FP64_STEPWISE && num->precision != PT_FP32 &&
      num->precision != PT_DF64)
    return PT_EINVAL;
  if (!phys_ok(phys)) return PT_EINVAL;
  if (!mg_ok(*grid, *num)) return PT_EINVAL;
  // the fused FP32 correction iteration indexes the box with 32-bit integers
  if (num->precision == PT_FP32 && make_box(grid).n >= (1LL << 31)) return PT_EINVAL;
  double* const ptrs[] = {f->Vx, f->Vy, f->Vz, f->Pt, f->Pf, f->phi, f->txx, f->tyy,
                          f->tzz, f->txy, f->txz, f->tyz, f->mu, f->eta};
  for (double* p : ptrs)
    if (!p || !aligned16(p)) return PT_EINVAL;
  if (f->logk && !aligned16(f->logk)) return PT_EINVAL;
  if (((uintptr_t)workspace & (kAlign - 1)) != 0) return PT_EINVAL;
  if (workspace_bytes < pt_workspace_size(grid, num)) return PT_ESPACE;

  pt_ctx* c = new (std::nothrow) pt_ctx();
  if (!c) return PT_ECUDA;
  c->grid = *grid;
  c->metric = *grid;
  c->phys = *phys;
  c->num = *num;
  c->box = make_box(grid);
  c->stream = (cudaStream_t)stream;
  c->Vx = f->Vx; c->Vy = f->Vy; c->Vz = f->Vz;
  c->Pt[0] = f->Pt; c->Pf[0] = f->Pf; c->phi[0] = f->phi;
  c->txx = f->txx; c->tyy = f->tyy; c->tzz = f->tzz;
  c->txy = f->txy; c->txz = f->txz; c->tyz = f->tyz;
  c->mu = f->mu; c->eta = f->eta; c->logk = f->logk;
  const size_t stride = align_up((size_t)c->box.n * sizeof(double), kAlign);
  char* w = (char*)workspace;
  c->lean = num->precision == PT_FP64;
  double** slots[kRefArrays + kLeanArrays] = {
      &c->Pt[1], &c->Pf[1], &c->phi[1], &c->Pto, &c->Pfo, &c->Lo, &c->txxo, &c->tyyo, &c->tzzo,
      &c->txyo, &c->txzo, &c->tyzo, &c->Rx, &c->Ry, &c->Rz, &c->perm, &c->rog, &c->s_txx,
      &c->s_tyy, &c->s_tzz, &c->s_txy, &c->s_txz, &c->s_tyz,
      // FP64-lean extras
      &c->lperm[0], &c->lperm[1], &c->lw[0], &c->lw[1], &c->phio, &c->Eo, &c->iEo, &c->toa_xx,
      &c->toa_yy, &c->toa_zz, &c->toa_xy, &c->toa_xz, &c->toa_yz, &c->cm2, &c->idtp, &c->ieta,
      &c->em2_xy, &c->em2_xz, &c->em2_yz, &c->eb_xy, &c->eb_xz, &c->eb_yz, &c->dtv_x, &c->dtv_y, &c->dtv_z,
      &c->K0};
  c->dfm = num->precision == PT_DF64;
  c->df_dirty = false;
  c->fcur = 0;
  const int arrays = kRefArrays + ((c->lean || c->dfm) ? kLeanArrays : 0);
  for (int s = 0; s < arrays; ++s) *slots[s] = (double*)(w + s * stride);
  char* wend = w + arrays * stride;
  if (c->dfm) {
    df64** fslots[kDfArrays] = {&c->fVx, &c->fVy, &c->fVz, &c->fPt[0], &c->fPt[1], &c->fPf[0], &c->fPf[1],
                                &c->fphi[0], &c->fphi[1], &c->fmu, &c->feta, &c->fRx, &c->fRy, &c->fRz,
                                &c->fs_txx, &c->fs_tyy, &c->fs_tzz, &c->fs_txy, &c->fs_txz, &c->fs_tyz,
                                &c->ftxxo, &c->ftyyo, &c->ftzzo, &c->ftxyo, &c->ftxzo, &c->ftyzo, &c->fPto,
                                &c->fPfo};
    for (int s = 0; s < kDfArrays; ++s) *fslots[s] = (df64*)(wend + s * stride);
    wend += kDfArrays * stride;
  }
  c->mixed = num->precision == PT_FP32;
  c->mix_omega = 1.0;
  c->mix_prev = 0.0;
  if (c->mixed) {
    const size_t fstride = align_up((size_t)c->box.n * sizeof(float), kAlign);
    float** fslots[kMixArrays] = {
        &c->m_rpt, &c->m_rpf, &c->m_rfx, &c->m_rfy, &c->m_rfz, &c->m_cc, &c->m_perm, &c->m_idtp, &c->m_mu,
        &c->m_dtvc, &c->m_dVx[0], &c->m_dVx[1], &c->m_dVy[0], &c->m_dVy[1], &c->m_dVz[0], &c->m_dVz[1],
        &c->m_dPt[0], &c->m_dPt[1], &c->m_dPf[0], &c->m_dPf[1], &c->m_Rx, &c->m_Ry, &c->m_Rz};
    for (int s = 0; s < kMixArrays; ++s) *fslots[s] = (float*)(wend + s * fstride);
    wend += kMixArrays * fstride;
  }
  c->mg_L = (c->mixed && num->mg_levels >= 2) ? num->mg_levels : 0;
  std::vector<std::pair<char*, std::vector<uint32_t>>> mg_tables;   // (device address, host copy)
  if (c->mg_L) {
    const size_t fstride = align_up((size_t)c->box.n * sizeof(float), kAlign);
    c->mg.resize(c->mg_L);
    c->mg_d.assign(c->mg_L, 0);
    c->mg_smooth.resize(c->mg_L);
    c->mg_eval.resize(c->mg_L);
    c->mg_dtpt.assign(c->mg_L, 0.f);
    c->mg_dtv.assign(c->mg_L, 0.f);
    MgLevel& f0 = c->mg[0];
    f0.b = c->box;
    f0.cc = c->m_cc; f0.perm = c->m_perm; f0.idtp = c->m_idtp; f0.mu = c->m_mu; f0.dtvc = c->m_dtvc;
    f0.rpt = c->m_rpt; f0.rpf = c->m_rpf; f0.rfx = c->m_rfx; f0.rfy = c->m_rfy; f0.rfz = c->m_rfz;
    for (int d = 0; d < 2; ++d) {
      f0.dVx[d] = c->m_dVx[d]; f0.dVy[d] = c->m_dVy[d]; f0.dVz[d] = c->m_dVz[d];
      f0.dPt[d] = c->m_dPt[d]; f0.dPf[d] = c->m_dPf[d];
    }
    f0.Rx = c->m_Rx; f0.Ry = c->m_Ry; f0.Rz = c->m_Rz;
    f0.res_pt = (float*)wend;
    f0.res_pf = (float*)(wend + fstride);
    wend += kMgFineArrays * fstride;
    for (int l = 1; l < c->mg_L; ++l) {
      const pt_grid gl = mg_grid(*grid, l), gf = mg_grid(*grid, l - 1);
      MgLevel& L = c->mg[l];
      L.b = make_box(&gl);
      const int nf[3] = {gf.nx, gf.ny, gf.nz}, nc[3] = {gl.nx, gl.ny, gl.nz};
      const size_t st = align_up((size_t)L.b.n * sizeof(float), kAlign);
      float** slots[kMgArrays] = {&L.cc, &L.perm, &L.idtp, &L.mu, &L.dtvc, &L.rpt, &L.rpf, &L.rfx, &L.rfy,
                                  &L.rfz, &L.dVx[0], &L.dVx[1], &L.dVy[0], &L.dVy[1], &L.dVz[0], &L.dVz[1],
                                  &L.dPt[0], &L.dPt[1], &L.dPf[0], &L.dPf[1], &L.Rx, &L.Ry, &L.Rz,
                                  &L.res_pt, &L.res_pf};
      for (int a = 0; a < kMgArrays; ++a) *slots[a] = (float*)(wend + a * st);
      wend += kMgArrays * st;
      for (int d = 0; d < 3; ++d) {   // transfer tables from the finer level, copied in after the memset
        L.ax[d] = mg_axis_at(wend, nf[d], nc[d]);
        mg_tables.emplace_back(wend, mg_axis_tables(nf[d], nc[d]));
        wend += align_up(mg_axis_words(nf[d], nc[d]) * 4, kAlign);
      }
    }
  }
  c->red = (unsigned long long*)wend;
  if (cudaMallocHost(&c->h_red, RED_N * sizeof(unsigned long long)) != cudaSuccess) {
    delete c;
    return PT_ECUDA;
  }
  c->dtS = 0.0;
  c->dt_cum = 0.0;
  c->nsteps = 0;
  c->cur = 0;
  c->launches = 0;
  c->profiling = false;
  c->pool_used = 0;
  c->adj_ws = nullptr;
  c->adj_nsteps = 0;
  fill_coef(c);
  // zero the whole workspace (damped residuals, old stresses, scratch padding)
  cudaError_t e = cudaMemsetAsync(workspace, 0, pt_workspace_size(grid, num), c->stream);
  for (const auto& tb : mg_tables)   // the host copies live until the synchronisation below
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(tb.first, tb.second.data(), tb.second.size() * 4, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess && c->dfm && c->logk) {
    PT_LAUNCH(c, K_DF_K0, lean_k0<df64>(grid_dims(c->box), block_dims(), c->stream, c->box, c->phys.k0, c->logk,
                                        D(c->K0)));
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && c->lean && c->logk) {
    PT_LAUNCH(c, K_LEAN_K0, lean_k0<double>(grid_dims(c->box), block_dims(), c->stream, c->box, c->phys.k0, c->logk,
                                            c->K0));
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && !keep_visc) {
    PT_LAUNCH(c, K_INIT_VISC, k_init_visc<<<grid_dims(c->box), block_dims(), 0, c->stream>>>(
                                   c->box, c->coef, c->phi[0], c->mu, c->eta));
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    cudaFreeHost(c->h_red);
    delete c;
    return PT_ECUDA;
  }
  *ctx = c;
  return PT_OK;
}

int pt_step_begin(pt_ctx* c) {
  if (c) {
    c->mix_omega = 1.0;
    c->mix_prev = 0.0;
  }
  if (!c) return PT_EINVAL;
  int rc = step_begin_launch(c);
  double mu_max = 0.0;
  if (rc == PT_OK) rc = step_begin_mumax(c, &mu_max);
  if (rc == PT_OK) rc = step_begin_finish(c, mu_max);
  return rc;
}

int pt_iterate(pt_ctx* c, int32_t it0, int32_t niter, pt_report* rep) {
  if (!c || it0 < 0 || niter < 0) return PT_EINVAL;
  if (c->nsteps == 0) return PT_EINVAL;  // pt_step_begin first
  if (c->mixed) {
    // one outer iteration with exactly niter FP32 iterations on the correction
    pt_report outer;
    bool conv = false;
    int done = 0;
    int rc = mixed_outer(c, niter, false, &outer, &conv, &done);
    if (rc == PT_OK) rc = sync_current_to_caller(c);
    if (rc == PT_OK) rc = cuda_status(cudaStreamSynchronize(c->stream));
    if (rep) {
      *rep = outer;
      rep->iters = done;
      rep->status = rc;
    }
    return rc;
  }
  int checked = 0;
  for (int32_t it = it0 + 1; it <= it0 + niter; ++it) {
    const int check = (it % c->num.nup) == 0;
    launch_iteration(c, check);
    checked |= check;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return PT_ECUDA;
  int rc = sync_current_to_caller(c);
  if (rc != PT_OK) return rc;
  if (rep) {
    std::memset(rep, 0, sizeof *rep);
    rep->iters = niter;
    if (checked) {
      rc = read_report(c, rep);
    } else {
      rc = cuda_status(cudaStreamSynchronize(c->stream));
    }
    rep->status = rc;
  }
  return rc;
}

int pt_step_end(pt_ctx* c) {
  if (!c) return PT_EINVAL;
  if (c->dfm) {
    const int rc = df_step_end(c);
    c->dt_cum += c->num.dt;
    return rc;
  }
  int rc = sync_current_to_caller(c);
  if (rc != PT_OK) return rc;
  const Box& b = c->box;
  CentreIn ci{c->Vx, c->Vy, c->Vz, c->Pt[0], c->Pf[0], c->phi[0], c->mu, c->eta, c->perm,
              c->Pto, c->Pfo, c->txxo, c->tyyo, c->tzzo};
  CentreOut co{nullptr, nullptr, c->txx, c->tyy, c->tzz};
  PT_LAUNCH(c, K_CENTRES, k_centres<<<grid_dims(b), block_dims(), 0, c->stream>>>(b, c->coef, ci, co, 0, c->red, 0));
  EdgeIn ei{c->Vx, c->Vy, c->Vz, c->mu, c->txyo, c->txzo, c->tyzo};
  EdgeOut eo{c->txy, c->txz, c->tyz};
  PT_LAUNCH(c, K_EDGES, k_edges<<<grid_dims(b), block_dims(), 0, c->stream>>>(b, c->coef, ei, eo));
  c->dt_cum += c->num.dt;
  return cuda_status(cudaGetLastError());
}

int pt_step(pt_ctx* c, pt_report* rep) {
  if (!c) return PT_EINVAL;
  int rc = pt_step_begin(c);
  if (rc != PT_OK) return rc;
  pt_report r;
  std::memset(&r, 0, sizeof r);
  int it = 0;
  bool converged = false;
  const int nup = c->num.nup, cap = c->num.max_iter;
  while (c->mixed) {
    int done = 0;
    rc = mixed_outer(c, cap - it, true, &r, &converged, &done);
    it += done;
    if (rc != PT_OK || converged || it >= cap) break;
  }
  while (!c->mixed && it < cap) {
    const int n = std::min(nup - (it % nup), cap - it);
    for (int s = 1; s <= n; ++s) launch_iteration(c, ((it + s) % nup) == 0);
    it += n;
    if (cudaGetLastError() != cudaSuccess) return PT_ECUDA;
    if (it % nup == 0) {
      rc = read_report(c, &r);
      if (rc != PT_OK) break;
      if (report_max(&r) < c->num.tol) {
        converged = true;
        break;
      }
    }
  }
  int rc2 = sync_current_to_caller(c);
  if (rc == PT_OK) rc = rc2;
  if (rc == PT_OK) rc = pt_step_end(c);
  if (rc == PT_OK) rc = cuda_status(cudaStreamSynchronize(c->stream));
  if (rc == PT_OK && !converged) rc = PT_ENOTCONV;
  r.iters = it;
  r.status = rc;
  if (rep) *rep = r;
  return rc;
}

int pt_residual(pt_ctx* c, pt_report* rep) {
  if (!c || !rep) return PT_EINVAL;
  if (c->nsteps == 0) return PT_EINVAL;
  int rc = sync_current_to_caller(c);
  if (rc != PT_OK) return rc;
  const Box& b = c->box;
  const Coef& k = c->coef;
  const dim3 bl = block_dims(), gr = grid_dims(b);
  cudaMemsetAsync(c->red, 0, RED_N * sizeof(unsigned long long), c->stream);
  PT_LAUNCH(c, K_PERM, k_perm<<<gr, bl, 0, c->stream>>>(b, k, c->phi[0], c->logk, c->perm, c->rog));
  CentreIn ci{c->Vx, c->Vy, c->Vz, c->Pt[0], c->Pf[0], c->phi[0], c->mu, c->eta, c->perm,
              c->Pto, c->Pfo, c->txxo, c->tyyo, c->tzzo};
  CentreOut co{c->Pt[1], c->Pf[1], c->s_txx, c->s_tyy, c->s_tzz};   // updates go to scratch
  PT_LAUNCH(c, K_CENTRES, k_centres<<<gr, bl, 0, c->stream>>>(b, k, ci, co, 1, c->red, 1));
  EdgeIn ei{c->Vx, c->Vy, c->Vz, c->mu, c->txyo, c->txzo, c->tyzo};
  EdgeOut eo{c->s_txy, c->s_txz, c->s_tyz};
  PT_LAUNCH(c, K_EDGES, k_edges<<<gr, bl, 0, c->stream>>>(b, k, ei, eo));
  FaceIn fi{c->s_txx, c->s_tyy, c->s_tzz, c->s_txy, c->s_txz, c->s_tyz, c->Pt[0], c->rog, c->mu};
  PT_LAUNCH(c, K_RESIDUAL_FACES, k_residual_faces<<<gr, bl, 0, c->stream>>>(b, k, fi, c->red));
  PicardIn pi{c->s_txx, c->s_tyy, c->s_tzz, c->s_txy, c->s_txz, c->s_tyz, c->phi[0], c->Pt[0], c->Pf[0]};
  PT_LAUNCH(c, K_PICARD, k_picard<<<gr, bl, 0, c->stream>>>(b, k, pi, c->mu, c->eta, c->red, 0));
  if (cudaGetLastError() != cudaSuccess) return PT_ECUDA;
  std::memset(rep, 0, sizeof *rep);
  rc = read_report(c, rep);
  rep->status = rc;
  return rc;
}

int pt_profile_begin(pt_ctx* c) {
  if (!c) return PT_EINVAL;
  c->recs.clear();
  c->pool_used = 0;
  c->profiling = true;
  return PT_OK;
}

int pt_profile_end(pt_ctx* c, pt_kernel_time* out, int32_t max_out, int32_t* n_out) {
  if (!c || (max_out > 0 && !out)) return PT_EINVAL;
  c->profiling = false;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return PT_ECUDA;
  double ms[K_COUNT] = {0};
  long long cnt[K_COUNT] = {0};
  for (const auto& r : c->recs) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) return PT_ECUDA;
    ms[r.kid] += t;
    cnt[r.kid] += 1;
  }
  int32_t n = 0;
  for (int k = 0; k < K_COUNT; ++k) {
    if (!cnt[k]) continue;
    if (n < max_out) {
      std::memset(out[n].name, 0, sizeof out[n].name);
      std::strncpy(out[n].name, kKernelNames[k], sizeof out[n].name - 1);
      out[n].launches = cnt[k];
      out[n].total_ms = ms[k];
    }
    ++n;
  }
  if (n_out) *n_out = n < max_out ? n : max_out;
  c->recs.clear();
  c->pool_used = 0;
  return PT_OK;
}

int64_t pt_launch_count(const pt_ctx* c) { return c ? (int64_t)c->launches : -1; }

void pt_destroy(pt_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  for (cudaEvent_t e : c->pool) cudaEventDestroy(e);
  cudaFreeHost(c->h_red);
  delete c;
}

int pt_math_check(int32_t fn, const double* a, const double* b, double* out, int64_t n, void* stream) {
  if (fn < 0 || fn >= MATH_COUNT || !a || !out || n < 0) return PT_EINVAL;
  if ((fn == MATH_DF_ADD || fn == MATH_DF_SUB || fn == MATH_DF_MUL || fn == MATH_DF_FMA || fn == MATH_DF_ROOT) && !b)
    return PT_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  math_check(st, fn, a, b, out, (long long)n);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return cuda_status(e);
}

const char* pt_strerror(int code) {
  switch (code) {
    case PT_OK: return "ok";
    case PT_EINVAL: return "invalid argument";
    case PT_ENOTCONV: return "PT iteration cap reached before the tolerance";
    case PT_ENAN: return "non-finite residual";
    case PT_ETIMEOUT: return "bounded device wait expired";
    case PT_ECUDA: return "CUDA error";
    case PT_ESPACE: return "workspace too small";
    default: return "unknown error";
  }
}

}  // extern "C"

// ============================================================================ batched ensemble
struct pt_batch {
  int ninst;
  std::vector<pt_ctx*> ctx;
  cudaStream_t caller;      // the caller's stream (may be the legacy default stream)
  cudaStream_t stream;      // the batch's own stream: graphs are captured and replayed on it
  std::vector<BatchInst> h_inst;
  BatchInst* d_inst;
  BatchStatus* d_st;
  BatchStatus* h_st;
  int nup;
  int bx, by, ipg;          // tile shape, iterations per graph replay
  bool tuned;
  long long ntiles;
  int grid;
  cudaGraphExec_t exec;
  int exec_bx, exec_by, exec_ipg;
  // parts of one decomposed grid (pt_dd): coupled convergence, halo exchange, ownership
  int coupled;
  const HaloSlab* d_slabs;
  int nslabs, slab_elems;
  DDTables tables;
  std::vector<std::array<int, 6>> own;   // per instance: own_lo[3], own_hi[3]
  // FP32 ensembles (every instance PT_FP32): the defect-correction engine of pt_mixed.cuh, its
  // decisions taken on the device per member; one graph replay = `mult` rounds of nup
  // correction iterations with the outer phases between them
  bool mixed;
  std::vector<MixBatchInst> h_minst;
  MixBatchInst* d_minst;
  MixBatchStatus* d_mst;
  MixBatchStatus* h_mst;
  unsigned long long* d_ired;
  int zchunk, minb, mult;   // correction tile depth, CTAs per SM of the correction kernel, rounds per replay
  int groups;               // members split into this many contiguous groups, each a parallel graph branch
  long long nptiles, nctiles;
  int pgrid, cgrid;
  int exec_zchunk, exec_minb, exec_mult, exec_groups;
  std::vector<int> gm;                  // group g = members [gm[g], gm[g + 1])
  std::vector<cudaStream_t> gstream;    // capture streams of the branches
  std::vector<cudaEvent_t> gevent;      // fork (0) and one join per branch
};

namespace {

// Descriptor tables: the FP64 engine's (instances, statuses), then the FP32 engine's (members,
// statuses, inner reduction slots).
size_t batch_table_bytes(int ninst) {
  return align_up(sizeof(BatchInst) * ninst, kAlign) + align_up(sizeof(BatchStatus) * ninst, kAlign) +
         align_up(sizeof(MixBatchInst) * ninst, kAlign) + align_up(sizeof(MixBatchStatus) * ninst, kAlign) +
         align_up(sizeof(unsigned long long) * RED_N * ninst, kAlign);
}

// Descriptor of instance m for the batch's tile shape (pointers of both ping-pong parities).
void fill_batch_inst(pt_batch* B, int m, long long base) {
  pt_ctx* c = B->ctx[m];
  BatchInst& I = B->h_inst[m];
  I.b = c->box;
  I.c = c->lcoef;
  for (int a = 0; a < 2; ++a) {
    const int n = 1 - a;
    I.cin[a] = LeanCellIn<double>{c->Vx, c->Vy, c->Vz, c->Pt[a], c->Pf[a], c->phi[a], c->lw[a], c->lperm[a],
                                  c->Pto, c->Pfo, c->phio, c->Eo, c->iEo, c->ieta, c->idtp, c->cm2,
                                  c->toa_xx, c->toa_yy, c->toa_zz, c->em2_xy, c->em2_xz, c->em2_yz,
                                  c->eb_xy, c->eb_xz, c->eb_yz, c->toa_xy, c->toa_xz, c->toa_yz,
                                  c->logk ? c->K0 : nullptr};
    I.cout[a] = LeanCellOut<double>{c->Pt[n], c->Pf[n], c->phi[n], c->lw[n], c->lperm[n], c->s_txx,
                                    c->s_tyy, c->s_tzz, c->s_txy, c->s_txz, c->s_tyz};
    I.fin[a] = LeanFaceIn<double>{c->s_txx, c->s_tyy, c->s_tzz, c->s_txy, c->s_txz, c->s_tyz, c->Pt[n],
                                  c->phi[a], c->dtv_x, c->dtv_y, c->dtv_z};
    I.pin[a] = LeanPicardIn<double>{c->s_txx, c->s_tyy, c->s_tzz, c->s_txy, c->s_txz, c->s_tyz,
                                    c->phi[n], c->Pt[n], c->Pf[n]};
  }
  I.kin = LeanCoefIn<double>{c->mu, c->eta, c->txxo, c->tyyo, c->tzzo, c->txyo, c->txzo, c->tyzo};
  I.kout = LeanCoefOut<double>{c->cm2, c->toa_xx, c->toa_yy, c->toa_zz, c->idtp, c->ieta, c->em2_xy,
                               c->em2_xz, c->em2_yz, c->eb_xy, c->eb_xz, c->eb_yz, c->toa_xy, c->toa_xz,
                               c->toa_yz, c->dtv_x,
                               c->dtv_y, c->dtv_z};
  I.Vx = c->Vx; I.Vy = c->Vy; I.Vz = c->Vz;
  I.Rx = c->Rx; I.Ry = c->Ry; I.Rz = c->Rz;
  I.mu = c->mu; I.eta = c->eta;
  I.red = B->coupled ? B->ctx[0]->red : c->red;   // parts of one grid share the norms
  for (int d = 0; d < 3; ++d) {
    I.own_lo[d] = B->own.empty() ? 0 : B->own[m][d];
    I.own_hi[d] = B->own.empty() ? (d == 0 ? c->box.nx : d == 1 ? c->box.ny : c->box.nz) : B->own[m][3 + d];
  }
  I.tol = c->num.tol;
  I.max_iter = c->num.max_iter;
  I.gx = (c->box.nx + 1 + B->bx - 1) / B->bx;
  I.gy = (c->box.ny + 1 + B->by - 1) / B->by;
  I.tile_base = base;
}

// Descriptors for the current tile shape, uploaded; returns the work-list length.
cudaError_t upload_batch(pt_batch* B) {
  long long base = 0;
  for (int m = 0; m < B->ninst; ++m) {
    fill_batch_inst(B, m, base);
    base += (long long)B->h_inst[m].gx * B->h_inst[m].gy * (B->ctx[m]->box.nz + 1);
  }
  B->ntiles = base;
  const int dev_blocks = batch_blocks_per_sm(B->bx, B->by);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  B->grid = std::max(1, sms * dev_blocks);
  return cudaMemcpyAsync(B->d_inst, B->h_inst.data(), sizeof(BatchInst) * B->ninst, cudaMemcpyHostToDevice,
                         B->stream);
}

// The launches of `ipg` iterations starting from parity 0 (ipg is a multiple of 2 nup).
void record_batch_iterations(pt_batch* B, int ipg) {
  for (int it = 1; it <= ipg; ++it) {
    const int a = (it - 1) & 1;
    const int check = (it % B->nup) == 0;
    batch_phase(B->bx, B->by, B->grid, B->stream, BATCH_CELLS, B->d_inst, B->d_st, B->ninst, B->ntiles, a, check);
    batch_phase(B->bx, B->by, B->grid, B->stream, BATCH_FACES, B->d_inst, B->d_st, B->ninst, B->ntiles, a, check);
    if (B->coupled)
      dd_exchange(B->stream, B->d_inst, B->d_st, B->d_slabs, B->nslabs, B->slab_elems, B->tables, a, DD_STATE);
    if (check) {
      batch_phase(B->bx, B->by, B->grid, B->stream, BATCH_PICARD, B->d_inst, B->d_st, B->ninst, B->ntiles, a, 1);
      if (B->coupled)
        dd_exchange(B->stream, B->d_inst, B->d_st, B->d_slabs, B->nslabs, B->slab_elems, B->tables, a, DD_VISC);
      batch_phase(B->bx, B->by, B->grid, B->stream, BATCH_COEF, B->d_inst, B->d_st, B->ninst, B->ntiles, a, 0);
      batch_converge(B->stream, B->d_inst, B->d_st, B->ninst, B->nup, B->coupled);
    }
  }
}

int build_batch_graph(pt_batch* B) {
  if (B->exec && B->exec_bx == B->bx && B->exec_by == B->by && B->exec_ipg == B->ipg) return PT_OK;
  if (B->exec) {
    cudaGraphExecDestroy(B->exec);
    B->exec = nullptr;
  }
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(B->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return PT_ECUDA;
  record_batch_iterations(B, B->ipg);
  cudaError_t e = cudaStreamEndCapture(B->stream, &g);
  if (e == cudaSuccess) e = cudaGraphInstantiate(&B->exec, g, 0);
  if (g) cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    B->exec = nullptr;
    return PT_ECUDA;
  }
  B->exec_bx = B->bx;
  B->exec_by = B->by;
  B->exec_ipg = B->ipg;
  return PT_OK;
}

int batch_active(pt_batch* B, int* nactive) {
  cudaError_t e = cudaMemcpyAsync(B->h_st, B->d_st, sizeof(BatchStatus) * B->ninst, cudaMemcpyDeviceToHost,
                                  B->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(B->stream);
  if (e != cudaSuccess) return PT_ECUDA;
  int n = 0;
  for (int m = 0; m < B->ninst; ++m) n += B->h_st[m].active;
  *nactive = n;
  return PT_OK;
}

// ---- FP32 ensembles: descriptors, graph and decisions of the device-side engine
void fill_mix_inst(pt_batch* B, int m, long long base, long long cbase) {
  pt_ctx* c = B->ctx[m];
  MixBatchInst& I = B->h_minst[m];
  I.b = c->box;
  I.k = c->coef;
  I.lc = c->lcoef;
  I.cc = c->ccoef;
  I.Vx = c->Vx; I.Vy = c->Vy; I.Vz = c->Vz;
  for (int a = 0; a < 2; ++a) {
    I.Pt[a] = c->Pt[a]; I.Pf[a] = c->Pf[a]; I.phi[a] = c->phi[a];
    I.dVx[a] = c->m_dVx[a]; I.dVy[a] = c->m_dVy[a]; I.dVz[a] = c->m_dVz[a];
    I.dPt[a] = c->m_dPt[a]; I.dPf[a] = c->m_dPf[a];
  }
  I.mu = c->mu; I.eta = c->eta; I.perm = c->perm; I.rog = c->rog; I.Pto = c->Pto; I.Pfo = c->Pfo; I.Lo = c->Lo;
  I.logk = c->logk;
  I.txxo = c->txxo; I.tyyo = c->tyyo; I.tzzo = c->tzzo; I.txyo = c->txyo; I.txzo = c->txzo; I.tyzo = c->tyzo;
  I.s_txx = c->s_txx; I.s_tyy = c->s_tyy; I.s_tzz = c->s_tzz; I.s_txy = c->s_txy; I.s_txz = c->s_txz;
  I.s_tyz = c->s_tyz;
  I.rpt = c->m_rpt; I.rpf = c->m_rpf; I.rfx = c->m_rfx; I.rfy = c->m_rfy; I.rfz = c->m_rfz;
  I.ccf = c->m_cc; I.kf = c->m_perm; I.idtp = c->m_idtp; I.muf = c->m_mu; I.dtvc = c->m_dtvc;
  I.Rx = c->m_Rx; I.Ry = c->m_Ry; I.Rz = c->m_Rz;
  I.fbase = c->m_rpt;
  I.fstride = (long long)(c->m_rpf - c->m_rpt);
  for (int d = 0; d < 2; ++d) {
    I.cin[d] = CorrIn<float>{I.dVx[d], I.dVy[d], I.dVz[d], I.dPt[d], I.dPf[d], I.ccf, I.kf, I.idtp, I.rpt,
                             I.rpf, I.muf, I.dtvc, I.rfx, I.rfy, I.rfz};
    I.cout[d] = CorrOut<float>{I.dVx[1 - d], I.dVy[1 - d], I.dVz[1 - d], I.dPt[1 - d], I.dPf[1 - d], I.Rx, I.Ry,
                               I.Rz};
  }
  I.red = c->red;
  I.ired = B->d_ired + (size_t)RED_N * m;
  I.tol = c->num.tol;
  I.rtol = c->num.inner_rtol > 0 ? c->num.inner_rtol : kInnerRtol;
  I.max_iter = c->num.max_iter;
  I.gx = (c->box.nx + 1 + 31) / 32;
  I.gy = (c->box.ny + 1 + 7) / 8;
  I.cgx = (c->box.nx + 1 + corr_tile_x() - 1) / corr_tile_x();
  I.cgy = (c->box.ny + 1 + corr_tile_y() - 1) / corr_tile_y();
  I.cgz = (c->box.nz + 1 + B->zchunk - 1) / B->zchunk;
  I.tile_base = base;
  I.ctile_base = cbase;
}

cudaError_t upload_mix(pt_batch* B) {
  long long base = 0, cbase = 0;
  for (int m = 0; m < B->ninst; ++m) {
    fill_mix_inst(B, m, base, cbase);
    const MixBatchInst& I = B->h_minst[m];
    base += (long long)I.gx * I.gy * (I.b.nz + 1);
    cbase += (long long)I.cgx * I.cgy * I.cgz;
  }
  B->nptiles = base;
  B->nctiles = cbase;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  B->pgrid = std::max(1, sms * mb_points_blocks_per_sm());
  B->cgrid = std::max(1, sms * mb_corr_blocks_per_sm(B->minb));
  return cudaMemcpyAsync(B->d_minst, B->h_minst.data(), sizeof(MixBatchInst) * B->ninst, cudaMemcpyHostToDevice,
                         B->stream);
}

// Contiguous member groups of near-equal cells (the branches of a replay).
void split_mix_groups(pt_batch* B) {
  const int G = std::max(1, std::min(B->groups, B->ninst));
  long long total = 0;
  for (int m = 0; m < B->ninst; ++m) total += B->ctx[m]->box.n;
  B->gm.assign(1, 0);
  long long acc = 0;
  for (int m = 0; m < B->ninst; ++m) {
    acc += B->ctx[m]->box.n;
    const int g = (int)B->gm.size();   // the group being filled
    if (g < G && m + 1 < B->ninst && acc * G >= total * g && B->ninst - (m + 1) >= G - g) B->gm.push_back(m + 1);
  }
  B->gm.push_back(B->ninst);
}

// The rounds of one member group on stream `s`: outer phases, nup correction iterations, update.
void record_mix_group(pt_batch* B, int g, cudaStream_t s) {
  const int m0 = B->gm[g], m1 = B->gm[g + 1], n = m1 - m0;
  const MixBatchInst* inst = B->d_minst + m0;
  MixBatchStatus* st = B->d_mst + m0;
  const MixBatchInst& first = B->h_minst[m0];
  const long long p0 = first.tile_base, c0 = first.ctile_base;
  const long long p1 = m1 < B->ninst ? B->h_minst[m1].tile_base : B->nptiles;
  const long long c1 = m1 < B->ninst ? B->h_minst[m1].ctile_base : B->nctiles;
  for (int r = 0; r < B->mult; ++r) {
    mb_points(B->pgrid, s, MB_PH_PERM, inst, st, n, p0, p1);
    mb_points(B->pgrid, s, MB_PH_PREP, inst, st, n, p0, p1);
    mb_points(B->pgrid, s, MB_PH_FACES, inst, st, n, p0, p1);
    mb_decide_outer(s, inst, st, n);
    mb_points(B->pgrid, s, MB_PH_INIT, inst, st, n, p0, p1);
    for (int k = 1; k <= B->nup; ++k) mb_corr(B->cgrid, B->minb, s, inst, st, n, c0, c1, k, B->nup, B->zchunk);
    mb_decide_inner(s, inst, st, n, B->nup);
    mb_points(B->pgrid, s, MB_PH_UPDATE, inst, st, n, p0, p1);
    mb_points(B->pgrid, s, MB_PH_POROSITY, inst, st, n, p0, p1);
    mb_finish(s, inst, st, n);
  }
}

// One replay: the member groups as parallel branches (they share no data), forked from and
// joined into the batch's stream.
void record_mix_rounds(pt_batch* B) {
  split_mix_groups(B);
  const int G = (int)B->gm.size() - 1;
  if (G == 1) {
    record_mix_group(B, 0, B->stream);
    return;
  }
  cudaEventRecord(B->gevent[0], B->stream);
  for (int g = 0; g < G; ++g) {
    cudaStreamWaitEvent(B->gstream[g], B->gevent[0], 0);
    record_mix_group(B, g, B->gstream[g]);
    cudaEventRecord(B->gevent[1 + g], B->gstream[g]);
  }
  for (int g = 0; g < G; ++g) cudaStreamWaitEvent(B->stream, B->gevent[1 + g], 0);
}

int build_mix_graph(pt_batch* B) {
  if (B->exec && B->exec_zchunk == B->zchunk && B->exec_minb == B->minb && B->exec_mult == B->mult &&
      B->exec_groups == B->groups)
    return PT_OK;
  if (B->exec) {
    cudaGraphExecDestroy(B->exec);
    B->exec = nullptr;
  }
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(B->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return PT_ECUDA;
  record_mix_rounds(B);
  cudaError_t e = cudaStreamEndCapture(B->stream, &g);
  if (e == cudaSuccess) e = cudaGraphInstantiate(&B->exec, g, 0);
  if (g) cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    B->exec = nullptr;
    return PT_ECUDA;
  }
  B->exec_zchunk = B->zchunk;
  B->exec_minb = B->minb;
  B->exec_mult = B->mult;
  B->exec_groups = B->groups;
  return PT_OK;
}

int mix_active(pt_batch* B, int* nactive) {
  cudaError_t e = cudaMemcpyAsync(B->h_mst, B->d_mst, sizeof(MixBatchStatus) * B->ninst, cudaMemcpyDeviceToHost,
                                  B->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(B->stream);
  if (e != cudaSuccess) return PT_ECUDA;
  int n = 0;
  for (int m = 0; m < B->ninst; ++m) n += B->h_mst[m].phase != MB_DONE;
  *nactive = n;
  return PT_OK;
}

// The two timing events of a tuner, destroyed on every return path.
struct TunerEvents {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  bool create() { return cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess; }
  ~TunerEvents() {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  }
};

// FP32 ensemble step: every member's step begin (host, as pt_step), then graph replays until
// every member is done; the first step times one replay of each candidate configuration
// (correction tile depth, CTAs per SM, rounds per replay) and keeps the fastest per round.
int batch_step_mixed(pt_batch* B, pt_report* reps, double* ttc_ms) {
  int rc = PT_OK;
  int cap = 0;
  for (int m = 0; m < B->ninst && rc == PT_OK; ++m) {
    rc = pt_step_begin(B->ctx[m]);
    cap = std::max(cap, B->ctx[m]->num.max_iter);
  }
  if (rc != PT_OK) return rc;
  if (cudaStreamSynchronize(B->stream) != cudaSuccess) return PT_ECUDA;
  if (upload_mix(B) != cudaSuccess) return PT_ECUDA;
  mb_start(B->stream, B->d_minst, B->d_mst, B->ninst);
  // every round advances each member that is not done: an outer iteration takes at least one
  // round and at least min(nup, budget) correction iterations, so this many rounds end every member
  const long long max_rounds = 2LL * ((long long)cap / B->nup + 2) + 4;
  struct Cfg { int zchunk, minb, mult, groups; };
  const Cfg cands[] = {{64, 4, 1, 1}, {64, 3, 1, 4}, {64, 4, 1, 4}, {64, 3, 1, 8}, {64, 3, 1, 16}, {32, 3, 1, 8},
                       {64, 3, 2, 8}};
  const int ncand = B->tuned ? 0 : (int)(sizeof cands / sizeof cands[0]);
  float best_ms = 1e30f;
  Cfg best = {B->zchunk, B->minb, B->mult, B->groups};
  long long rounds = 0;
  int nactive = B->ninst;
  TunerEvents ev;
  if (ncand && !ev.create()) return PT_ECUDA;
  for (int t = 0; t < ncand && nactive > 0 && rounds < max_rounds; ++t) {
    B->zchunk = cands[t].zchunk;
    B->minb = cands[t].minb;
    B->mult = cands[t].mult;
    B->groups = cands[t].groups;
    if (upload_mix(B) != cudaSuccess) return PT_ECUDA;
    rc = build_mix_graph(B);
    if (rc != PT_OK) return rc;
    cudaEventRecord(ev.e0, B->stream);
    if (cudaGraphLaunch(B->exec, B->stream) != cudaSuccess) return PT_ECUDA;
    cudaEventRecord(ev.e1, B->stream);
    rounds += B->mult;
    rc = mix_active(B, &nactive);
    if (rc != PT_OK) return rc;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev.e0, ev.e1);
    if (ms / B->mult < best_ms) {
      best_ms = ms / B->mult;
      best = cands[t];
    }
  }
  if (ncand) {
    B->zchunk = best.zchunk;
    B->minb = best.minb;
    B->mult = best.mult;
    B->groups = best.groups;
    B->tuned = true;
    if (upload_mix(B) != cudaSuccess) return PT_ECUDA;
  }
  rc = build_mix_graph(B);
  if (rc != PT_OK) return rc;
  while (nactive > 0 && rounds < max_rounds) {
    if (cudaGraphLaunch(B->exec, B->stream) != cudaSuccess) return PT_ECUDA;
    rounds += B->mult;
    rc = mix_active(B, &nactive);
    if (rc != PT_OK) return rc;
  }
  if (nactive > 0) return PT_ECUDA;   // cannot happen: see max_rounds
  int any_nc = 0, any_nan = 0;
  for (int m = 0; m < B->ninst; ++m) {
    const MixBatchStatus& S = B->h_mst[m];
    pt_ctx* c = B->ctx[m];
    c->cur = S.cur;
    c->mix_omega = S.omega;
    c->mix_prev = S.prev;
    const int rc_end = pt_step_end(c);
    reps[m].iters = S.iters;
    reps[m].status = S.status;
    reps[m].res_v = S.res[0];
    reps[m].res_pt = S.res[1];
    reps[m].res_pf = S.res[2];
    reps[m].res_pic = S.res[3];
    if (ttc_ms) ttc_ms[m] = S.t_stop > S.t_start ? (double)(S.t_stop - S.t_start) * 1e-6 : -1.0;
    if (rc_end != PT_OK) return rc_end;
    any_nc |= S.status == PT_ENOTCONV;
    any_nan |= S.status == PT_ENAN;
  }
  if (cudaStreamSynchronize(B->stream) != cudaSuccess) return PT_ECUDA;
  return any_nan ? PT_ENAN : (any_nc ? PT_ENOTCONV : PT_OK);
}

}  // namespace

extern "C" {

size_t pt_batch_workspace_size(int32_t ninst, const pt_grid* grids, const pt_num* nums) {
  if (ninst < 1 || !grids || !nums) return 0;
  size_t total = 0;
  for (int m = 0; m < ninst; ++m) {
    const size_t s = pt_workspace_size(&grids[m], &nums[m]);
    if (s == 0) return 0;
    total += align_up(s, kAlign);
  }
  return total + batch_table_bytes(ninst);
}

int pt_batch_init(pt_batch** out, int32_t ninst, const pt_grid* grids, const pt_phys* phys, const pt_num* nums,
                  const pt_fields* fields, void* workspace, size_t workspace_bytes, void* stream) {
  if (!out) return PT_EINVAL;
  *out = nullptr;
  if (ninst < 1 || !grids || !phys || !nums || !fields || !workspace) return PT_EINVAL;
  if (((uintptr_t)workspace & (kAlign - 1)) != 0) return PT_EINVAL;
  const bool fp32 = nums[0].precision == PT_FP32;
  for (int m = 0; m < ninst; ++m)
    if (nums[m].precision != (fp32 ? PT_FP32 : PT_FP64) || nums[m].nup != nums[0].nup || nums[m].mg_levels > 1)
      return PT_EINVAL;
  const size_t need = pt_batch_workspace_size(ninst, grids, nums);
  if (need == 0) return PT_EINVAL;
  if (workspace_bytes < need) return PT_ESPACE;
  pt_batch* B = new (std::nothrow) pt_batch();
  if (!B) return PT_ECUDA;
  B->ninst = ninst;
  B->caller = (cudaStream_t)stream;
  // a stream of its own: the legacy default stream cannot be captured into a graph
  if (cudaStreamCreateWithFlags(&B->stream, cudaStreamNonBlocking) != cudaSuccess) {
    delete B;
    return PT_ECUDA;
  }
  if (cudaStreamSynchronize(B->caller) != cudaSuccess) {
    cudaStreamDestroy(B->stream);
    delete B;
    return PT_ECUDA;
  }
  B->nup = nums[0].nup;
  B->bx = 32;
  B->by = 8;
  B->ipg = 2 * B->nup;
  B->tuned = false;
  B->exec = nullptr;
  B->coupled = 0;
  B->d_slabs = nullptr;
  B->nslabs = 0;
  B->slab_elems = 0;
  B->ctx.assign(ninst, nullptr);
  B->h_inst.resize(ninst);
  B->mixed = fp32;
  B->zchunk = 64;
  B->minb = 4;
  B->mult = 1;
  B->groups = 1;
  B->exec_zchunk = B->exec_minb = B->exec_mult = B->exec_groups = 0;
  B->h_st = nullptr;
  B->h_mst = nullptr;
  if (fp32) B->h_minst.resize(ninst);
  char* w = (char*)workspace;
  int rc = PT_OK;
  if (fp32) {   // capture streams and events of the parallel member groups (up to 16)
    B->gstream.assign(16, nullptr);
    B->gevent.assign(17, nullptr);
    for (cudaStream_t& q : B->gstream)
      if (rc == PT_OK && cudaStreamCreateWithFlags(&q, cudaStreamNonBlocking) != cudaSuccess) rc = PT_ECUDA;
    for (cudaEvent_t& e : B->gevent)
      if (rc == PT_OK && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) rc = PT_ECUDA;
  }
  for (int m = 0; m < ninst && rc == PT_OK; ++m) {
    const size_t s = pt_workspace_size(&grids[m], &nums[m]);
    rc = pt_init(&B->ctx[m], &grids[m], &phys[m], &nums[m], &fields[m], w, s, (void*)B->stream, 0);
    w += align_up(s, kAlign);
  }
  if (rc == PT_OK) {
    char* t = w;
    B->d_inst = (BatchInst*)t;
    t += align_up(sizeof(BatchInst) * ninst, kAlign);
    B->d_st = (BatchStatus*)t;
    t += align_up(sizeof(BatchStatus) * ninst, kAlign);
    B->d_minst = (MixBatchInst*)t;
    t += align_up(sizeof(MixBatchInst) * ninst, kAlign);
    B->d_mst = (MixBatchStatus*)t;
    t += align_up(sizeof(MixBatchStatus) * ninst, kAlign);
    B->d_ired = (unsigned long long*)t;
    if (cudaMallocHost(&B->h_st, sizeof(BatchStatus) * ninst) != cudaSuccess) rc = PT_ECUDA;
    if (rc == PT_OK && cudaMallocHost(&B->h_mst, sizeof(MixBatchStatus) * ninst) != cudaSuccess) rc = PT_ECUDA;
  }
  if (rc != PT_OK) {
    for (pt_ctx* c : B->ctx) pt_destroy(c);
    if (B->h_st) cudaFreeHost(B->h_st);
    if (B->h_mst) cudaFreeHost(B->h_mst);
    for (cudaStream_t q : B->gstream)
      if (q) cudaStreamDestroy(q);
    for (cudaEvent_t e : B->gevent)
      if (e) cudaEventDestroy(e);
    cudaStreamDestroy(B->stream);
    delete B;
    return rc;
  }
  *out = B;
  return PT_OK;
}

int pt_batch_step(pt_batch* B, pt_report* reps, double* ttc_ms) {
  if (!B || !reps) return PT_EINVAL;
  // order after the caller's prior work on its stream
  if (cudaStreamSynchronize(B->caller) != cudaSuccess) return PT_ECUDA;
  if (B->mixed) return batch_step_mixed(B, reps, ttc_ms);
  int rc = PT_OK;
  int cap = 0;
  if (B->coupled) {
    // parts of one grid: one stress sub-step from the largest mu over all parts
    double mu_max = 0.0;
    for (int m = 0; m < B->ninst && rc == PT_OK; ++m) rc = step_begin_launch(B->ctx[m]);
    for (int m = 0; m < B->ninst && rc == PT_OK; ++m) {
      double v = 0.0;
      rc = step_begin_mumax(B->ctx[m], &v);
      mu_max = std::fmax(mu_max, v);
    }
    for (int m = 0; m < B->ninst && rc == PT_OK; ++m) rc = step_begin_finish(B->ctx[m], mu_max);
    cap = B->ctx[0]->num.max_iter;
  }
  for (int m = 0; m < B->ninst && rc == PT_OK && !B->coupled; ++m) {
    rc = pt_step_begin(B->ctx[m]);   // old-state snapshot, dtS, coefficients (per instance)
    cap = std::max(cap, B->ctx[m]->num.max_iter);
  }
  if (rc != PT_OK) return rc;
  if (upload_batch(B) != cudaSuccess) return PT_ECUDA;
  batch_start(B->stream, B->d_inst, B->d_st, B->ninst);
  // candidate configurations; the first step times one replay of each and keeps the fastest
  struct Cfg { int bx, by, mult; };
  const Cfg cands[] = {{32, 8, 2}, {32, 4, 2}, {64, 4, 2}, {32, 8, 4}};
  const int ncand = B->tuned ? 0 : (int)(sizeof cands / sizeof cands[0]);
  float best_ms = 1e30f;
  Cfg best = {B->bx, B->by, B->ipg / (2 * B->nup)};
  int done = 0, nactive = B->ninst;
  TunerEvents ev;
  if (ncand && !ev.create()) return PT_ECUDA;
  for (int t = 0; t < ncand && nactive > 0 && done < cap; ++t) {
    B->bx = cands[t].bx;
    B->by = cands[t].by;
    B->ipg = cands[t].mult * 2 * B->nup;
    if (upload_batch(B) != cudaSuccess) return PT_ECUDA;
    rc = build_batch_graph(B);
    if (rc != PT_OK) return rc;
    cudaEventRecord(ev.e0, B->stream);
    if (cudaGraphLaunch(B->exec, B->stream) != cudaSuccess) return PT_ECUDA;
    cudaEventRecord(ev.e1, B->stream);
    done += B->ipg;
    rc = batch_active(B, &nactive);
    if (rc != PT_OK) return rc;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev.e0, ev.e1);
    if (ms / B->ipg < best_ms) {
      best_ms = ms / B->ipg;
      best = cands[t];
    }
  }
  if (ncand) {
    B->bx = best.bx;
    B->by = best.by;
    B->ipg = best.mult * 2 * B->nup;
    B->tuned = true;
    if (upload_batch(B) != cudaSuccess) return PT_ECUDA;
  }
  rc = build_batch_graph(B);
  if (rc != PT_OK) return rc;
  while (nactive > 0 && done < cap) {
    if (cudaGraphLaunch(B->exec, B->stream) != cudaSuccess) return PT_ECUDA;
    done += B->ipg;
    rc = batch_active(B, &nactive);
    if (rc != PT_OK) return rc;
  }
  rc = batch_active(B, &nactive);
  if (rc != PT_OK) return rc;
  int any_nc = 0, any_nan = 0;
  for (int m = 0; m < B->ninst; ++m) {
    const BatchStatus& s = B->h_st[m];
    pt_ctx* c = B->ctx[m];
    c->cur = s.iters & 1;     // the instance's last iterate is in the buffer of its parity
    const int rc_end = pt_step_end(c);
    reps[m].iters = s.iters;
    reps[m].status = s.status;
    reps[m].res_v = s.res[0];
    reps[m].res_pt = s.res[1];
    reps[m].res_pf = s.res[2];
    reps[m].res_pic = s.res[3];
    if (ttc_ms) ttc_ms[m] = s.t_stop > s.t_start ? (double)(s.t_stop - s.t_start) * 1e-6 : -1.0;
    if (rc_end != PT_OK) return rc_end;
    any_nc |= s.status == PT_ENOTCONV;
    any_nan |= s.status == PT_ENAN;
  }
  if (cudaStreamSynchronize(B->stream) != cudaSuccess) return PT_ECUDA;
  return any_nan ? PT_ENAN : (any_nc ? PT_ENOTCONV : PT_OK);
}

size_t pt_mg_axis_words(int32_t nf) { return nf >= 2 ? mg_axis_words(nf, (nf + 1) / 2) : 0; }

int pt_mg_axis_tables(int32_t nf, uint32_t* out, size_t words) {
  if (nf < 2 || !out) return PT_EINVAL;
  const std::vector<uint32_t> t = mg_axis_tables(nf, (nf + 1) / 2);
  if (words < t.size()) return PT_ESPACE;
  std::memcpy(out, t.data(), t.size() * sizeof(uint32_t));
  return PT_OK;
}

int pt_batch_config(const pt_batch* B, int32_t* tile_x, int32_t* tile_y, int32_t* ipg) {
  if (!B) return PT_EINVAL;
  if (tile_x) *tile_x = B->mixed ? corr_tile_x() : B->bx;
  if (tile_y) *tile_y = B->mixed ? corr_tile_y() : B->by;
  if (ipg) *ipg = B->mixed ? B->mult * B->nup : B->ipg;
  return PT_OK;
}

int pt_batch_config_fp32(const pt_batch* B, int32_t* tile_z, int32_t* blocks_per_sm, int32_t* groups) {
  if (!B || !B->mixed) return PT_EINVAL;
  if (tile_z) *tile_z = B->zchunk;
  if (blocks_per_sm) *blocks_per_sm = B->minb;
  if (groups) *groups = std::max(1, std::min(B->groups, B->ninst));
  return PT_OK;
}

void pt_batch_destroy(pt_batch* B) {
  if (!B) return;
  cudaStreamSynchronize(B->stream);
  if (B->exec) cudaGraphExecDestroy(B->exec);
  for (pt_ctx* c : B->ctx) pt_destroy(c);
  cudaFreeHost(B->h_st);
  cudaFreeHost(B->h_mst);
  for (cudaStream_t q : B->gstream)
    if (q) cudaStreamDestroy(q);
  for (cudaEvent_t e : B->gevent)
    if (e) cudaEventDestroy(e);
  cudaStreamDestroy(B->stream);
  delete B;
}

}  // extern "C"

// ============================================================================ adjoint
namespace {

constexpr int kCkptArrays = 23;   // 14 caller fields, R (3), old stresses (6)
constexpr int kSegArrays = 7;     // converged Vx, Vy, Vz, Pt, Pf, phi, mu per step of a segment
// multipliers, residual memory, stresses, right-hand sides, coefficients (40), and for the power
// law lambda_mu (2), g_mu, Z (3), the power-law coefficients (26) and an accumulator
constexpr int kAdjArrays = 73;

int n_ckpts(int nsteps, int every) { return (nsteps + every - 1) / every + 1; }  // + final state

double** ckpt_sources(pt_ctx* c, double** s) {
  double* src[kCkptArrays] = {c->Vx, c->Vy, c->Vz, c->Pt[0], c->Pf[0], c->phi[0], c->txx, c->tyy, c->tzz,
                              c->txy, c->txz, c->tyz, c->mu, c->eta, c->Rx, c->Ry, c->Rz, c->txxo,
                              c->tyyo, c->tzzo, c->txyo, c->txzo, c->tyzo};
  for (int i = 0; i < kCkptArrays; ++i) s[i] = src[i];
  return s;
}

double* ws_array(char* base, const Box& b, size_t index) {
  return (double*)(base + index * align_up((size_t)b.n * sizeof(double), kAlign));
}
double* adj_array(pt_ctx* c, size_t index) { return ws_array(c->adj_ws, c->box, index); }

int ckpt_io(pt_ctx* c, int slot, bool save) {
  double* s[kCkptArrays];
  ckpt_sources(c, s);
  const size_t bytes = (size_t)c->box.n * sizeof(double);
  for (int i = 0; i < kCkptArrays; ++i) {
    double* d = adj_array(c, (size_t)slot * kCkptArrays + i);
    const cudaError_t e = save ? cudaMemcpyAsync(d, s[i], bytes, cudaMemcpyDeviceToDevice, c->stream)
                               : cudaMemcpyAsync(s[i], d, bytes, cudaMemcpyDeviceToDevice, c->stream);
    if (e != cudaSuccess) return PT_ECUDA;
  }
  if (save) {
    c->adj_dtS[slot] = c->dtS;
    c->adj_dtcum[slot] = c->dt_cum;
    c->adj_nst[slot] = c->nsteps;
  } else {
    c->dtS = c->adj_dtS[slot];
    c->dt_cum = c->adj_dtcum[slot];
    c->nsteps = c->adj_nst[slot];
    c->cur = 0;
    fill_coef(c);
  }
  return PT_OK;
}

bool adjoint_scope_ok(const pt_ctx* c) {
  return c->phys.compaction_on != 0 && c->phys.R_weak == 1.0 && c->phys.tau_bg == 0.0 &&
         c->num.beta_n == 0.0 && !c->mixed && !c->dfm && (c->lean || !c->logk);
}

// The adjoint's working arrays (kAdjArrays consecutive workspace arrays from `base`).
struct AdjArrays {
  double *Lx, *Ly, *Lz, *LRx, *LRy, *LRz, *lP[2], *lF[2], *lL[2], *mL[2];
  double *txx, *tyy, *tzz, *txy, *txz, *tyz, *gP, *gF, *gphi, *gth;
  double *lM[2], *gM, *Zxy, *Zxz, *Zyz, *acc;
  AdjPrep prep;
  AdjPrepPL pl;
  double* all[kAdjArrays];
  AdjArrays(char* base, const Box& b) {
    for (int i = 0; i < kAdjArrays; ++i) all[i] = ws_array(base, b, i);
    double** A = all;
    Lx = A[0]; Ly = A[1]; Lz = A[2]; LRx = A[3]; LRy = A[4]; LRz = A[5];
    lP[0] = A[6]; lP[1] = A[7]; lF[0] = A[8]; lF[1] = A[9]; lL[0] = A[10]; lL[1] = A[11];
    mL[0] = A[12]; mL[1] = A[13];
    txx = A[14]; tyy = A[15]; tzz = A[16]; txy = A[17]; txz = A[18]; tyz = A[19];
    gP = A[20]; gF = A[21]; gphi = A[22]; gth = A[23];
    prep = AdjPrep{A[24], A[25], A[26], A[27], A[28], A[29], A[30], A[31], A[32], A[33],
                   A[34], A[35], A[36], A[37], A[38], A[39], nullptr, nullptr};
    lM[0] = A[40]; lM[1] = A[41]; gM = A[42]; Zxy = A[43]; Zxz = A[44]; Zyz = A[45];
    double** P = A + 46;
    pl = AdjPrepPL{P[0], P[1], P[2], P[3], P[4], P[5], P[6], P[7], P[8], P[9], P[10], P[11], P[12],
                   P[13], P[14], P[15], P[16], P[17], P[18], P[19], P[20], P[21], P[22], P[23], P[24], P[25]};
    acc = A[72];
  }
  AdjEdgeIn edge_in(int cur) const {
    return AdjEdgeIn{Lx, Ly, Lz, lM[cur], pl.Axy, pl.Axz, pl.Ayz, pl.me_xy, pl.me_xz, pl.me_yz};
  }
  AdjPrep prep_for(int cur) const {
    AdjPrep p = prep;
    p.lL = lL[cur];
    p.mL = mL[cur];
    return p;
  }
  AdjCellIn cell_in(int cur, const double* K0) const {
    return AdjCellIn{Lx, Ly, Lz, lP[cur], lF[cur], lL[cur], mL[cur], gP, gF, gphi, K0,
                     prep.W, prep.cP, prep.cF, prep.Dg, prep.iD, prep.aPF, prep.a3k,
                     prep.kfx, prep.kfy, prep.kfz, prep.gkx, prep.gky, prep.gkz};
  }
};

// Scalars of the transposed system (mu = mu0 everywhere in the adjoint's scope).
AdjCoef adjoint_coef(const pt_ctx* c) {
  const Coef& k = c->coef;
  AdjCoef ac;
  ac.rdx = k.rdx; ac.rdy = k.rdy; ac.rdz = k.rdz;
  ac.m2 = 2.0 * c->phys.mu0 / (1.0 + c->phys.mu0 * k.rGdtS);   // d tau / d eps, fixed old stresses
  ac.third = 1.0 / 3.0;
  ac.hm2rdx = 0.5 * ac.m2 * k.rdx; ac.hm2rdy = 0.5 * ac.m2 * k.rdy; ac.hm2rdz = 0.5 * ac.m2 * k.rdz;
  ac.r_eta0mu0 = 1.0 / (c->phys.eta0 * c->phys.mu0);
  ac.bd_rdt = k.beta_d * k.rdt;
  ac.bd_rdt_a = k.beta_d * k.alpha * k.rdt;
  ac.bda_B_rdt = k.beta_d * k.alpha / k.B * k.rdt;
  ac.beta_phi = k.beta_phi;
  ac.dt = k.dt;
  ac.dt_r = k.dt * ac.r_eta0mu0;
  ac.idtp = 1.0 / (k.dtaupt_fac * c->phys.mu0);
  ac.ifac_pf = 1.0 / k.dtaupf_fac;
  ac.rphi0 = k.rphi0;
  ac.k0 = k.k0;
  ac.buoy = k.rhof_g - k.rho_bg_g;
  ac.hdrho_g = 0.5 * (c->phys.rhof_g - c->phys.rhos_g);
  ac.hdt_rdx = 0.5 * k.dt * k.rdx; ac.hdt_rdy = 0.5 * k.dt * k.rdy; ac.hdt_rdz = 0.5 * k.dt * k.rdz;
  ac.rrho_i = k.rrho_i;
  ac.damp_x = k.damp_x; ac.damp_y = k.damp_y; ac.damp_z = k.damp_z;
  ac.dtauv = k.dtauv_fac / c->phys.mu0;
  ac.powerlaw = c->phys.powerlaw_on != 0;
  ac.Gdt = c->phys.G * c->dtS;           // set per step from that step's dtS
  ac.rtau0_2 = 1.0 / (c->phys.tau0 * c->phys.tau0);
  ac.pw = 0.5 * (c->phys.n_pow - 1.0);
  ac.r_eta0 = 1.0 / c->phys.eta0;
  ac.dtauv_fac = k.dtauv_fac;
  ac.dtaupt_fac = k.dtaupt_fac;
  return ac;
}

}  // namespace

extern "C" {

size_t pt_adjoint_workspace_size(const pt_grid* grid, int32_t nsteps, int32_t every) {
  if (!grid_ok(grid) || nsteps < 0 || every < 1) return 0;
  const Box b = make_box(grid);
  const size_t stride = align_up((size_t)b.n * sizeof(double), kAlign);
  if (nsteps == 0) return (size_t)kAdjArrays * stride;                    // pt_adjoint_apply
  const int nck = n_ckpts(nsteps, every);
  return ((size_t)nck * kCkptArrays + (size_t)(every + 1) * kSegArrays + kAdjArrays) * stride;
}

int pt_adjoint_forward(pt_ctx* c, int32_t nsteps, int32_t every, void* ws, size_t bytes, pt_report* reps) {
  if (!c || !ws || nsteps < 1 || every < 1) return PT_EINVAL;
  if (!adjoint_scope_ok(c) || c->nsteps != 0) return PT_EINVAL;
  if (((uintptr_t)ws & (kAlign - 1)) != 0) return PT_EINVAL;
  const size_t need = pt_adjoint_workspace_size(&c->grid, nsteps, every);
  if (need == 0) return PT_EINVAL;
  if (bytes < need) return PT_ESPACE;
  if (sync_current_to_caller(c) != PT_OK) return PT_ECUDA;
  c->adj_ws = (char*)ws;
  c->adj_bytes = bytes;
  c->adj_nsteps = nsteps;
  c->adj_ckpt = every;
  const int nck = n_ckpts(nsteps, every);
  c->adj_dtS.assign(nck, 0.0);
  c->adj_dtcum.assign(nck, 0.0);
  c->adj_nst.assign(nck, 0);
  int rc = PT_OK;
  for (int n = 0; n < nsteps && rc == PT_OK; ++n) {
    if (n % every == 0) rc = ckpt_io(c, n / every, true);
    if (rc != PT_OK) break;
    pt_report r;
    rc = pt_step(c, &r);
    if (reps) reps[n] = r;
    if (rc == PT_ENOTCONV) rc = PT_OK;   // reported per step; the adjoint uses the iterate reached
    // the old stresses must not be refreshed after the first step inside the window
    if (rc == PT_OK && c->dt_cum < (n + 0.5) * c->num.dt) rc = PT_EINVAL;
  }
  if (rc == PT_OK) rc = ckpt_io(c, nck - 1, true);   // final state
  if (rc == PT_OK) rc = cuda_status(cudaStreamSynchronize(c->stream));
  if (rc != PT_OK) c->adj_nsteps = 0;
  return rc;
}

int pt_adjoint(pt_ctx* c, const double* dJ_dphi, double* grad, pt_report* rep) {
  if (!c || !dJ_dphi || !grad || !c->adj_ws || c->adj_nsteps < 1) return PT_EINVAL;
  const Box& b = c->box;
  const dim3 bl = block_dims(), gr = grid_dims(b);
  const int N = c->adj_nsteps, every = c->adj_ckpt, nck = n_ckpts(N, every);
  const size_t bytes = (size_t)b.n * sizeof(double);
  const size_t seg0 = (size_t)nck * kCkptArrays, adj0 = seg0 + (size_t)(every + 1) * kSegArrays;
  AdjArrays A(c->adj_ws + adj0 * align_up(bytes, kAlign), b);
  auto seg = [&](int slot, int f) { return adj_array(c, seg0 + (size_t)slot * kSegArrays + f); };
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < kAdjArrays && e == cudaSuccess; ++i) e = cudaMemsetAsync(A.all[i], 0, bytes, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(grad, 0, bytes, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(A.gphi, dJ_dphi, bytes, cudaMemcpyDeviceToDevice, c->stream);
  if (e != cudaSuccess) return PT_ECUDA;
  AdjCoef ac = adjoint_coef(c);
  const bool pl = ac.powerlaw;
  const double* K0 = (c->lean && c->logk) ? c->K0 : nullptr;
  std::vector<double> seg_dtS((size_t)every + 1, 0.0);   // each kept step's stress sub-step dtS
  long long total_iters = 0;
  pt_report last;
  std::memset(&last, 0, sizeof last);
  int rc = PT_OK;
  int cur = 0;   // parity of the multipliers' ping-pong
  for (int s = nck - 2; s >= 0 && rc == PT_OK; --s) {
    const int n0 = s * every, n1 = std::min(N, n0 + every);
    // re-run the segment from its checkpoint, keeping every converged state; its last state is
    // the next checkpoint (no recompute at all when every step is checkpointed)
    double* src[kSegArrays] = {c->Vx, c->Vy, c->Vz, c->Pt[0], c->Pf[0], c->phi[0], c->mu};
    auto keep = [&](int m) {
      for (int f = 0; f < kSegArrays && rc == PT_OK; ++f)
        if (cudaMemcpyAsync(seg(m, f), src[f], bytes, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess)
          rc = PT_ECUDA;
      seg_dtS[(size_t)m] = c->dtS;
    };
    rc = ckpt_io(c, s, false);
    if (rc == PT_OK) keep(0);
    for (int n = n0 + 1; n < n1 && rc == PT_OK; ++n) {
      pt_report r;
      rc = pt_step(c, &r);
      if (rc == PT_ENOTCONV) rc = PT_OK;
      if (rc == PT_OK) keep(n - n0);
    }
    if (rc == PT_OK) rc = ckpt_io(c, s + 1, false);
    if (rc == PT_OK) keep(n1 - n0);
    // adjoint steps n1 .. n0+1, warm-started from the previous step's multipliers
    for (int n = n1; n > n0 && rc == PT_OK; --n) {
      const int m = n - n0;
      const AdjState u{seg(m, 0), seg(m, 1), seg(m, 2), seg(m, 3), seg(m, 4), seg(m, 5), seg(m, 6)};
      ac.Gdt = c->phys.G * seg_dtS[(size_t)m];
      if (pl) {
        // the state's edge stresses go to the Z arrays as scratch (the iteration overwrites them)
        PT_LAUNCH(c, K_ADJ_PREP, adj_prep_pl(gr, bl, c->stream, b, ac, u, K0, A.prep_for(cur), A.pl, A.Zxy, A.Zxz,
                                             A.Zyz));
      } else {
        PT_LAUNCH(c, K_ADJ_PREP, adj_prep(gr, bl, c->stream, b, ac, u, K0, A.prep_for(cur)));
      }
      // convergence: residual max-norms below tol times the largest right-hand side |g|
      cudaMemsetAsync(c->red, 0, RED_N * sizeof(unsigned long long), c->stream);
      PT_LAUNCH(c, K_ADJ_CARRY, adj_gmax(gr, bl, c->stream, b, A.gP, A.gF, A.gphi, c->red));
      if (pl) PT_LAUNCH(c, K_ADJ_CARRY, adj_gmax(gr, bl, c->stream, b, A.gM, A.gM, A.gM, c->red));
      double gscale = 0.0;
      if (cudaMemcpyAsync(c->h_red, c->red, RED_N * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                          c->stream) != cudaSuccess ||
          cudaStreamSynchronize(c->stream) != cudaSuccess) {
        rc = PT_ECUDA;
        break;
      }
      std::memcpy(&gscale, &c->h_red[RED_GMAX], sizeof gscale);
      int it = 0;
      const int nup = c->num.nup, cap = c->num.max_iter;
      const AdjFaceIn fi0{A.txx, A.tyy, A.tzz, A.txy, A.txz, A.tyz, nullptr, nullptr, A.prep.bfx, A.prep.bfy,
                          A.prep.bfz, nullptr, nullptr, nullptr, 1, pl ? A.pl.dtvx : nullptr,
                          pl ? A.pl.dtvy : nullptr, pl ? A.pl.dtvz : nullptr};
      while (gscale > 0.0 && it < cap && rc == PT_OK) {
        ++it;
        const int check = (it % nup) == 0 || it == cap;
        if (check) cudaMemsetAsync(c->red, 0, RED_N * sizeof(unsigned long long), c->stream);
        const AdjCellOut co{A.txx, A.tyy, A.tzz, A.txy, A.txz, A.tyz, A.lP[1 - cur], A.lF[1 - cur],
                            A.lL[1 - cur], A.mL[1 - cur], check ? A.gth : nullptr, nullptr, nullptr, nullptr};
        if (pl) {
          PT_LAUNCH(c, K_ADJ_EDGES_PL, adj_edges_pl(gr, bl, c->stream, b, ac, A.edge_in(cur),
                                                    AdjEdgeOut{A.txy, A.txz, A.tyz, A.Zxy, A.Zxz, A.Zyz}));
          const AdjMuIn mi{A.lM[cur], A.gM, A.Zxy, A.Zxz, A.Zyz, A.lM[1 - cur], nullptr};
          PT_LAUNCH(c, K_ADJ_CELLS_PL, adj_cells_pl(gr, bl, c->stream, b, ac, u, A.cell_in(cur, K0), co, A.pl, mi,
                                                 c->red, check));
        } else {
          PT_LAUNCH(c, K_ADJ_CELLS, adj_cells(gr, bl, c->stream, b, ac, u, A.cell_in(cur, K0), co, c->red, check));
        }
        AdjFaceIn fi = fi0;
        fi.lP1 = A.lP[1 - cur];
        fi.mL = A.mL[1 - cur];
        PT_LAUNCH(c, pl ? K_ADJ_FACES_PL : K_ADJ_FACES,
                  adj_faces(gr, bl, c->stream, b, ac, fi, A.Lx, A.Ly, A.Lz, A.LRx, A.LRy, A.LRz, c->red, check));
        cur = 1 - cur;
        if (check) {
          rc = read_report(c, &last);
          if (rc != PT_OK) break;
          if (report_max(&last) < c->num.tol * gscale) break;
        }
      }
      total_iters += it;
      if (rc != PT_OK) break;
      if (gscale == 0.0) cudaMemsetAsync(A.gth, 0, bytes, c->stream);   // g = 0: lambda = 0
      // gradient and carry into step n-1 (phi_o = phi^{n-1})
      const AdjCarry ca{A.lP[cur], A.lF[cur], A.lL[cur], A.gth, seg(m - 1, 5), grad, A.gP, A.gF, A.gphi};
      PT_LAUNCH(c, K_ADJ_CARRY, adj_carry(gr, bl, c->stream, b, ac, ca));
      if (pl) {
        // the power law: this step's dtS = max(mu^{n-1}) / (G xsi_w) carries
        // -(d(lambda . F)/d(G dtS)) / xsi_w into row mu of step n-1 at the cell holding that maximum
        cudaMemsetAsync(A.gM, 0, bytes, c->stream);
        cudaMemsetAsync(A.acc, 0, sizeof(double), c->stream);
        PT_LAUNCH(c, K_ADJ_CARRY, adj_edges_pl(gr, bl, c->stream, b, ac, A.edge_in(cur),
                                               AdjEdgeOut{A.txy, A.txz, A.tyz, A.Zxy, A.Zxz, A.Zyz}));
        PT_LAUNCH(c, K_ADJ_CARRY, adj_dgdt_pl(gr, bl, c->stream, b, ac, u, A.pl, A.Lx, A.Ly, A.Lz, A.lM[cur],
                                              A.Zxy, A.Zxz, A.Zyz, A.acc));
        cudaMemsetAsync(c->red, 0, RED_N * sizeof(unsigned long long), c->stream);
        cudaMemsetAsync(c->red + RED_ARG, 0xff, sizeof(unsigned long long), c->stream);
        PT_LAUNCH(c, K_ADJ_CARRY, adj_argmax(gr, bl, c->stream, b, seg(m - 1, 6), c->red));
        PT_LAUNCH(c, K_ADJ_CARRY, adj_add_at(c->stream, b, A.gM, c->red, A.acc, -1.0 / c->num.xsi_w));
      }
      if (cudaGetLastError() != cudaSuccess) rc = PT_ECUDA;
    }
  }
  if (rc == PT_OK) rc = ckpt_io(c, nck - 1, false);   // back to the state after step N
  if (rc == PT_OK) rc = cuda_status(cudaStreamSynchronize(c->stream));
  if (rep) {
    *rep = last;
    rep->iters = (int32_t)std::min<long long>(total_iters, 0x7fffffff);
    rep->status = rc;
  }
  return rc;
}

int pt_adjoint_apply(pt_ctx* c, const pt_adj_vec* lam, pt_adj_vec* out, void* ws, size_t wbytes) {
  if (!c || !lam || !out || !ws) return PT_EINVAL;
  if (!lam->Vx || !lam->Vy || !lam->Vz || !lam->Pt || !lam->Pf || !lam->phi) return PT_EINVAL;
  if (!out->Vx || !out->Vy || !out->Vz || !out->Pt || !out->Pf || !out->phi) return PT_EINVAL;
  if (!adjoint_scope_ok(c) || c->nsteps < 1) return PT_EINVAL;
  const bool pl = c->phys.powerlaw_on != 0;
  if (pl && (!lam->mu || !out->mu)) return PT_EINVAL;
  if (((uintptr_t)ws & (kAlign - 1)) != 0) return PT_EINVAL;
  if (wbytes < pt_adjoint_workspace_size(&c->grid, 0, 1)) return PT_ESPACE;
  int rc = sync_current_to_caller(c);
  if (rc != PT_OK) return rc;
  const Box& b = c->box;
  const dim3 bl = block_dims(), gr = grid_dims(b);
  const size_t bytes = (size_t)b.n * sizeof(double);
  AdjArrays A((char*)ws, b);
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < kAdjArrays && e == cudaSuccess; ++i) e = cudaMemsetAsync(A.all[i], 0, bytes, c->stream);
  const double* src[7] = {lam->Vx, lam->Vy, lam->Vz, lam->Pt, lam->Pf, lam->phi, lam->mu};
  double* dst[7] = {A.Lx, A.Ly, A.Lz, A.lP[0], A.lF[0], A.lL[0], A.lM[0]};
  const int nv = pl ? 7 : 6;
  for (int i = 0; i < nv && e == cudaSuccess; ++i)
    e = cudaMemcpyAsync(dst[i], src[i], bytes, cudaMemcpyDeviceToDevice, c->stream);
  double* outs[7] = {out->Vx, out->Vy, out->Vz, out->Pt, out->Pf, out->phi, out->mu};
  for (int i = 0; i < nv && e == cudaSuccess; ++i) e = cudaMemsetAsync(outs[i], 0, bytes, c->stream);
  if (e != cudaSuccess) return PT_ECUDA;
  const AdjCoef ac = adjoint_coef(c);
  const double* K0 = (c->lean && c->logk) ? c->K0 : nullptr;
  const AdjState u{c->Vx, c->Vy, c->Vz, c->Pt[0], c->Pf[0], c->phi[0], c->mu};
  // with g = 0 the residual rows of the iteration kernels are J^T lambda itself
  const AdjCellOut co{A.txx, A.tyy, A.tzz, A.txy, A.txz, A.tyz, A.lP[1], A.lF[1], A.lL[1], A.mL[1],
                      nullptr, out->Pt, out->Pf, out->phi};
  if (pl) {
    PT_LAUNCH(c, K_ADJ_PREP, adj_prep_pl(gr, bl, c->stream, b, ac, u, K0, A.prep_for(0), A.pl, A.Zxy, A.Zxz,
                                         A.Zyz));
    PT_LAUNCH(c, K_ADJ_EDGES_PL, adj_edges_pl(gr, bl, c->stream, b, ac, A.edge_in(0),
                                              AdjEdgeOut{A.txy, A.txz, A.tyz, A.Zxy, A.Zxz, A.Zyz}));
    const AdjMuIn mi{A.lM[0], A.gM, A.Zxy, A.Zxz, A.Zyz, A.lM[1], out->mu};
    PT_LAUNCH(c, K_ADJ_CELLS_PL, adj_cells_pl(gr, bl, c->stream, b, ac, u, A.cell_in(0, K0), co, A.pl, mi, c->red, 0));
  } else {
    PT_LAUNCH(c, K_ADJ_PREP, adj_prep(gr, bl, c->stream, b, ac, u, K0, A.prep_for(0)));
    PT_LAUNCH(c, K_ADJ_CELLS, adj_cells(gr, bl, c->stream, b, ac, u, A.cell_in(0, K0), co, c->red, 0));
  }
  const AdjFaceIn fi{A.txx, A.tyy, A.tzz, A.txy, A.txz, A.tyz, A.lP[0], A.mL[0],
                     A.prep.bfx, A.prep.bfy, A.prep.bfz, out->Vx, out->Vy, out->Vz, 0, nullptr, nullptr, nullptr};
  PT_LAUNCH(c, pl ? K_ADJ_FACES_PL : K_ADJ_FACES,
            adj_faces(gr, bl, c->stream, b, ac, fi, A.Lx, A.Ly, A.Lz, A.LRx, A.LRy, A.LRz, c->red, 0));
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  return cuda_status(e);
}

}  // extern "C"

// ============================================================================ sub-domains
struct pt_dd {
  pt_grid grid;
  Box gbox;
  int nparts;
  pt_batch* B;
  std::vector<DDFields> h_parts;
  DDFields* d_global;
  DDFields* d_parts;
  Box* d_boxes;
  DDTables tables;
};

namespace {

// Split of a grid into parts: part p of a direction owns cells [cut[p], cut[p+1]) and its box
// adds one halo cell on each side that has a neighbour.
struct DDPlan {
  int parts[3];
  std::vector<int> cut[3];
  std::vector<pt_grid> grids;
  std::vector<std::array<int, 3>> off;
  std::vector<std::array<int, 6>> own;
  std::vector<HaloSlab> slabs;
  int slab_elems = 0;
};

bool dd_plan(const pt_grid* g, const int32_t* parts, DDPlan* P) {
  if (!grid_ok(g) || !parts) return false;
  const int n[3] = {g->nx, g->ny, g->nz};
  const double h[3] = {g->lx / g->nx, g->ly / g->ny, g->lz / g->nz};
  for (int d = 0; d < 3; ++d) {
    if (parts[d] < 1 || (parts[d] > 1 && n[d] / parts[d] < 2)) return false;   // >= 2 cells per part
    P->parts[d] = parts[d];
    P->cut[d].resize(parts[d] + 1);
    for (int p = 0; p <= parts[d]; ++p) P->cut[d][p] = (int)((long long)p * n[d] / parts[d]);
  }
  for (int pz = 0; pz < parts[2]; ++pz)
    for (int py = 0; py < parts[1]; ++py)
      for (int px = 0; px < parts[0]; ++px) {
        const int pc[3] = {px, py, pz};
        int nl[3];
        std::array<int, 3> off;
        std::array<int, 6> own;
        for (int d = 0; d < 3; ++d) {
          const int lo = P->cut[d][pc[d]], hi = P->cut[d][pc[d] + 1];
          const int hl = pc[d] > 0, hr = pc[d] < parts[d] - 1;
          nl[d] = hi - lo + hl + hr;
          off[d] = lo - hl;
          own[d] = hl;
          own[3 + d] = hl + (hi - lo);
        }
        pt_grid lg{nl[0], nl[1], nl[2], nl[0] * h[0], nl[1] * h[1], nl[2] * h[2]};
        const int m = (int)P->grids.size();
        P->grids.push_back(lg);
        P->off.push_back(off);
        P->own.push_back(own);
        for (int d = 0; d < 3; ++d)
          for (int side = 0; side < 2; ++side) {
            if (side == 0 ? pc[d] == 0 : pc[d] == parts[d] - 1) continue;
            int r0[3], r1[3];
            for (int e = 0; e < 3; ++e) {
              r0[e] = 0;
              r1[e] = nl[e] + 1;          // box indices include the upper face / edge plane
            }
            if (side == 0) {
              r0[d] = 0;
              r1[d] = 1;
            } else {
              r0[d] = nl[d] - 1;
              r1[d] = nl[d] + 1;
            }
            P->slabs.push_back(HaloSlab{m, r0[0], r1[0], r0[1], r1[1], r0[2], r1[2]});
            const long long el = (long long)(r1[0] - r0[0]) * (r1[1] - r0[1]) * (r1[2] - r0[2]);
            P->slab_elems = (int)std::max<long long>(P->slab_elems, el);
          }
      }
  return true;
}

size_t dd_part_bytes(const pt_grid& lg) {
  return (size_t)kDDFields * align_up((size_t)make_box(&lg).n * sizeof(double), kAlign);
}

size_t dd_table_bytes(const pt_grid* g, const DDPlan& P) {
  const size_t np = P.grids.size();
  return align_up(sizeof(HaloSlab) * std::max<size_t>(1, P.slabs.size()), kAlign) +
         align_up(sizeof(int) * (size_t)(g->nx + g->ny + g->nz + 3), kAlign) +
         align_up(sizeof(int) * 3 * np, kAlign) + align_up(sizeof(DDFields) * (np + 1), kAlign) +
         align_up(sizeof(Box) * np, kAlign);
}

}  // namespace

extern "C" {

size_t pt_dd_workspace_size(const pt_grid* grid, const pt_num* num, const int32_t parts[3]) {
  DDPlan P;
  if (!num || !dd_plan(grid, parts, &P)) return 0;
  size_t total = 0;
  for (const pt_grid& lg : P.grids) total += dd_part_bytes(lg);
  std::vector<pt_num> nums(P.grids.size(), *num);
  const size_t bw = pt_batch_workspace_size((int32_t)P.grids.size(), P.grids.data(), nums.data());
  if (bw == 0) return 0;
  return total + align_up(bw, kAlign) + dd_table_bytes(grid, P);
}

int pt_dd_init(pt_dd** out, const pt_grid* grid, const pt_phys* phys, const pt_num* num, const pt_fields* fields,
               const int32_t parts[3], void* workspace, size_t bytes, void* stream) {
  if (!out) return PT_EINVAL;
  *out = nullptr;
  if (!grid || !phys || !num || !fields || !parts || !workspace) return PT_EINVAL;
  if (num->precision != PT_FP64) return PT_EINVAL;
  if (((uintptr_t)workspace & (kAlign - 1)) != 0) return PT_EINVAL;
  DDPlan P;
  if (!dd_plan(grid, parts, &P)) return PT_EINVAL;
  const size_t need = pt_dd_workspace_size(grid, num, parts);
  if (need == 0) return PT_EINVAL;
  if (bytes < need) return PT_ESPACE;
  const int np = (int)P.grids.size();
  cudaStream_t s = (cudaStream_t)stream;
  pt_dd* D = new (std::nothrow) pt_dd();
  if (!D) return PT_ECUDA;
  D->grid = *grid;
  D->gbox = make_box(grid);
  D->nparts = np;
  // part fields, then the batch's workspace, then the tables
  char* w = (char*)workspace;
  D->h_parts.resize(np);
  std::vector<pt_fields> pf(np);
  for (int m = 0; m < np; ++m) {
    const size_t stride = align_up((size_t)make_box(&P.grids[m]).n * sizeof(double), kAlign);
    for (int f = 0; f < kDDFields; ++f) D->h_parts[m].f[f] = (double*)(w + f * stride);
    if (!fields->logk) D->h_parts[m].f[kDDFields - 1] = nullptr;
    double** F = D->h_parts[m].f;
    pf[m] = pt_fields{F[0], F[1], F[2], F[3], F[4], F[5], F[6], F[7], F[8], F[9], F[10], F[11], F[12], F[13],
                      F[14]};
    w += dd_part_bytes(P.grids[m]);
  }
  std::vector<pt_num> nums(np, *num);
  std::vector<pt_phys> phs(np, *phys);
  const size_t bw = pt_batch_workspace_size(np, P.grids.data(), nums.data());
  char* wb = w;
  w += align_up(bw, kAlign);
  HaloSlab* d_slabs = (HaloSlab*)w;
  w += align_up(sizeof(HaloSlab) * std::max<size_t>(1, P.slabs.size()), kAlign);
  int* d_own = (int*)w;
  w += align_up(sizeof(int) * (size_t)(grid->nx + grid->ny + grid->nz + 3), kAlign);
  int* d_off = (int*)w;
  w += align_up(sizeof(int) * 3 * np, kAlign);
  D->d_global = (DDFields*)w;
  D->d_parts = D->d_global + 1;
  w += align_up(sizeof(DDFields) * (np + 1), kAlign);
  D->d_boxes = (Box*)w;
  // host copies of the tables
  std::vector<int> own;
  const int n[3] = {grid->nx, grid->ny, grid->nz};
  for (int d = 0; d < 3; ++d)
    for (int G = 0; G <= n[d]; ++G) {
      int p = 0;
      while (p + 1 < P.parts[d] && G >= P.cut[d][p + 1]) ++p;
      own.push_back(p);
    }
  std::vector<int> off;
  std::vector<Box> boxes;
  for (int m = 0; m < np; ++m) {
    for (int d = 0; d < 3; ++d) off.push_back(P.off[m][d]);
    boxes.push_back(make_box(&P.grids[m]));
  }
  DDFields g;
  const double* gf[kDDFields] = {fields->Vx, fields->Vy, fields->Vz, fields->Pt, fields->Pf, fields->phi,
                                 fields->txx, fields->tyy, fields->tzz, fields->txy, fields->txz, fields->tyz,
                                 fields->mu, fields->eta, fields->logk};
  for (int f = 0; f < kDDFields; ++f) g.f[f] = const_cast<double*>(gf[f]);
  cudaError_t e = cudaSuccess;
  if (!P.slabs.empty())
    e = cudaMemcpyAsync(d_slabs, P.slabs.data(), sizeof(HaloSlab) * P.slabs.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_own, own.data(), sizeof(int) * own.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_off, off.data(), sizeof(int) * off.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(D->d_global, &g, sizeof g, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(D->d_parts, D->h_parts.data(), sizeof(DDFields) * np, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(D->d_boxes, boxes.data(), sizeof(Box) * np, cudaMemcpyHostToDevice, s);
  for (int m = 0; m < np && e == cudaSuccess; ++m) {
    dd_scatter(s, D->gbox, boxes[m], P.off[m][0], P.off[m][1], P.off[m][2], D->d_global, D->d_parts + m);
    e = cudaGetLastError();
  }
  // the host tables must outlive the copies
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    delete D;
    return PT_ECUDA;
  }
  int rc = pt_batch_init(&D->B, np, P.grids.data(), phs.data(), nums.data(), pf.data(), wb, bw, stream);
  if (rc != PT_OK) {
    delete D;
    return rc;
  }
  pt_batch* B = D->B;
  for (pt_ctx* c : B->ctx) {   // coefficients from the whole grid's spacing (and nz)
    c->metric = *grid;
    fill_coef(c);
  }
  B->coupled = 1;
  B->own = P.own;
  B->d_slabs = d_slabs;
  B->nslabs = (int)P.slabs.size();
  B->slab_elems = P.slab_elems;
  D->tables = DDTables{d_own, d_own + grid->nx + 1, d_own + grid->nx + grid->ny + 2, d_off, P.parts[0],
                       P.parts[1]};
  B->tables = D->tables;
  *out = D;
  return PT_OK;
}

int pt_dd_step(pt_dd* D, pt_report* rep) {
  if (!D || !rep) return PT_EINVAL;
  std::vector<pt_report> reps(D->nparts);
  const int rc = pt_batch_step(D->B, reps.data(), nullptr);
  *rep = reps[0];
  return rc;
}

int pt_dd_gather(pt_dd* D) {
  if (!D) return PT_EINVAL;
  dd_gather(D->B->stream, D->gbox, D->d_boxes, D->tables, D->d_global, D->d_parts);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(D->B->stream);
  return cuda_status(e);
}

int pt_dd_config(const pt_dd* D, int32_t* nparts, int32_t* tile_x, int32_t* tile_y, int32_t* ipg) {
  if (!D) return PT_EINVAL;
  if (nparts) *nparts = D->nparts;
  return pt_batch_config(D->B, tile_x, tile_y, ipg);
}

void pt_dd_destroy(pt_dd* D) {
  if (!D) return;
  pt_batch_destroy(D->B);
  delete D;
}

}  // extern "C"
