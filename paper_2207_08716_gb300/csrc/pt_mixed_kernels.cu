// pt_mixed_kernels.cu — mixed precision (PT_FP32): FP32 PT iterations on the correction of an
// FP64 defect-correction loop.
//
// One outer iteration at the FP64 state u = (V, Pt, Pf, phi; mu, eta):
//   (i)   FP64 residuals of Eqs. 17-19 at u: r_Pt (numerical div V), r_Pf (fluid pressure),
//         r_F (momentum) — stored in FP32 as the right-hand side of the correction problem —
//         and their max-norms (k_mix_prepare, k_edges, k_mix_res_faces);
//   (ii)  FP64 Picard update of mu, eta (Eqs. 24-26) from the stresses at u;
//   (iii) FP32 PT on the correction delta = (dV, dPt, dPf) of the system linearised at u with
//         frozen coefficients (k, 1/(eta(1-phi)), mu, pseudo-time steps): the same damped,
//         local-implicit scheme as the FP64 iteration, iterating on the small correction so
//         that FP32 keeps its relative precision on it (k_corr_iteration, one pass per iteration);
//   (iv)  u <- u + delta in FP64 (k_mix_update), then the porosity time integration of
//         Eq. 22 in FP64 (log space) from the corrected pressures and velocities.
// Converged when the FP64 residual max-norms and the Picard change are below tol.
#include "pt_mixed.cuh"
#include "pt_ref_points.cuh"
#include "pt_lean_body.cuh"
#include "../../include/porowave_pt.h"

namespace pt {

namespace {
template <class T>
__device__ inline T tabs(T x) { return x < T(0) ? -x : x; }
__device__ inline double pos_max64(double a, double b) {
  const long long ia = __double_as_longlong(a), ib = __double_as_longlong(b);
  return __longlong_as_double(ia > ib ? ia : ib);
}
}  // namespace

// (i) FP64 residuals at cell centres, normal stresses at u, and the frozen coefficients of the
// correction problem (in FP32).
__device__ __forceinline__ void mix_prepare_point(const Box& b, const Coef& c, const MixPrepIn& in,
                                                  const MixPrepOut& out, int i, int j, int k, double& r_pt,
                                                  double& r_pf) {
  if (i < b.nx && j < b.ny && k < b.nz) {
    const long long q = cidx(b, i, j, k);
    const long long px = b.px, pxy = b.pxy;
    const double Pt = in.Pt[q], Pf = in.Pf[q], Pto = in.Pto[q], Pfo = in.Pfo[q];
    const double ph = in.phi[q], mu = in.mu[q];
    const double divV = (in.Vx[q + 1] - in.Vx[q]) * c.rdx + (in.Vy[q + px] - in.Vy[q]) * c.rdy +
                        (in.Vz[q + pxy] - in.Vz[q]) * c.rdz;
    // reciprocals by the two-step Newton iteration (within an ulp; these phases run on the FP64 pipe)
    const double cc = c.compaction_on ? lean_detail::rcp_full(in.eta[q] * (1.0 - ph)) : 0.0;
    const double divVn = divV + c.beta_d * ((Pt - Pto) - c.alpha * (Pf - Pfo)) * c.rdt + (Pt - Pf) * cc;
    const double kc = in.perm[q];
    const double buoy = c.rhof_g - c.rho_bg_g;
    double kmax = kc, qxl = 0.0, qxr = 0.0, qyl = 0.0, qyr = 0.0, qzl = 0.0, qzr = 0.0;
    if (i > 0) {
      const double kn = in.perm[q - 1];
      kmax = pos_max64(kmax, kn);
      qxl = -0.5 * (kn + kc) * (Pf - in.Pf[q - 1]) * c.rdx;
    }
    if (i < b.nx - 1) {
      const double kn = in.perm[q + 1];
      kmax = pos_max64(kmax, kn);
      qxr = -0.5 * (kc + kn) * (in.Pf[q + 1] - Pf) * c.rdx;
    }
    if (j > 0) {
      const double kn = in.perm[q - px];
      kmax = pos_max64(kmax, kn);
      qyl = -0.5 * (kn + kc) * (Pf - in.Pf[q - px]) * c.rdy;
    }
    if (j < b.ny - 1) {
      const double kn = in.perm[q + px];
      kmax = pos_max64(kmax, kn);
      qyr = -0.5 * (kc + kn) * (in.Pf[q + px] - Pf) * c.rdy;
    }
    if (k > 0) {
      const double kn = in.perm[q - pxy];
      kmax = pos_max64(kmax, kn);
      qzl = -0.5 * (kn + kc) * ((Pf - in.Pf[q - pxy]) * c.rdz + buoy);
    }
    if (k < b.nz - 1) {
      const double kn = in.perm[q + pxy];
      kmax = pos_max64(kmax, kn);
      qzr = -0.5 * (kc + kn) * ((in.Pf[q + pxy] - Pf) * c.rdz + buoy);
    }
    const double divqD = (qxr - qxl) * c.rdx + (qyr - qyl) * c.rdy + (qzr - qzl) * c.rdz;
    const double rpf = divqD + c.beta_d * c.alpha * ((Pf - Pfo) / c.B - (Pt - Pto)) * c.rdt + (Pf - Pt) * cc;
    // stresses at u (Eq. 21) for the momentum residual and the Picard update
    const double xi = mu * c.rGdtS;
    const double s = lean_detail::rcp_full(1.0 + xi);
    const double bn = c.beta_n * divVn;
    out.txx[q] = (in.txxo[q] * xi + 2.0 * mu * ((in.Vx[q + 1] - in.Vx[q]) * c.rdx - divV / 3.0 + bn)) * s;
    out.tyy[q] = (in.tyyo[q] * xi + 2.0 * mu * ((in.Vy[q + px] - in.Vy[q]) * c.rdy - divV / 3.0 + bn)) * s;
    out.tzz[q] = (in.tzzo[q] * xi + 2.0 * mu * ((in.Vz[q + pxy] - in.Vz[q]) * c.rdz - divV / 3.0 + bn)) * s;
    // right-hand side and frozen coefficients of the correction problem (the iteration derives
    // 1/dtau_Pf from the largest neighbour k and the local-implicit denominators itself)
    (void)kmax;
    out.r_pt[q] = (float)divVn;
    out.r_pf[q] = (float)rpf;
    out.cc[q] = (float)cc;
    out.perm[q] = (float)kc;
    out.idtp[q] = (float)lean_detail::rcp_full(c.dtaupt_fac * mu);
    r_pt = fabs(divVn);
    r_pf = fabs(rpf);
  }
}

// The edge stresses and the porosity integration of the FP32 form's outer phases (the shared
// bodies with Newton reciprocals).
__global__ void __launch_bounds__(256) k_mix_edges(Box b, Coef c, EdgeIn in, EdgeOut out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  edges_point<true>(b, c, in, out, i, j, (int)blockIdx.z);
}
__global__ void __launch_bounds__(256) k_mix_porosity(Box b, Coef c, MixPorosity p) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  porosity_point<true>(b, c, p.Vx, p.Vy, p.Vz, p.phi, p.Pt1, p.Pf1, p.Pto, p.Pfo, p.Lo, p.eta, p.phi1, i, j,
                       (int)blockIdx.z);
}

__global__ void __launch_bounds__(256) k_mix_prepare(Box b, Coef c, MixPrepIn in, MixPrepOut out,
                                                     unsigned long long* red) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  double r_pt = 0.0, r_pf = 0.0;
  mix_prepare_point(b, c, in, out, i, j, k, r_pt, r_pf);
  block_max_atomic(r_pt, red + RED_PT);
  block_max_atomic(r_pf, red + RED_PF);
}

// (i) FP64 momentum residual at u (Eq. 19), stored in FP32; its max-norm.
__device__ __forceinline__ void mix_res_faces_point(const Box& b, const Coef& c, const MixFaceIn& in,
                                                    float* __restrict__ rfx, float* __restrict__ rfy,
                                                    float* __restrict__ rfz, int i, int j, int k, double& r_v) {
  if (i <= b.nx && j <= b.ny && k <= b.nz) {
    const long long q = cidx(b, i, j, k);
    const long long px = b.px, pxy = b.pxy;
    if (i > 0 && i < b.nx && j < b.ny && k < b.nz) {
      const double F = (in.txx[q] - in.txx[q - 1]) * c.rdx + (in.txy[q + px] - in.txy[q]) * c.rdy +
                       (in.txz[q + pxy] - in.txz[q]) * c.rdz - (in.Pt[q] - in.Pt[q - 1]) * c.rdx;
      rfx[q] = (float)F;
      r_v = fmax(r_v, fabs(F));
    }
    if (j > 0 && j < b.ny && i < b.nx && k < b.nz) {
      const double F = (in.txy[q + 1] - in.txy[q]) * c.rdx + (in.tyy[q] - in.tyy[q - px]) * c.rdy +
                       (in.tyz[q + pxy] - in.tyz[q]) * c.rdz - (in.Pt[q] - in.Pt[q - px]) * c.rdy;
      rfy[q] = (float)F;
      r_v = fmax(r_v, fabs(F));
    }
    if (k > 0 && k < b.nz && i < b.nx && j < b.ny) {
      const double rog = (0.5 * (in.phi[q - pxy] + in.phi[q]) - c.phi0) * (c.rhof_g - c.rhos_g);
      const double F = (in.txz[q + 1] - in.txz[q]) * c.rdx + (in.tyz[q + px] - in.tyz[q]) * c.rdy +
                       (in.tzz[q] - in.tzz[q - pxy]) * c.rdz - (in.Pt[q] - in.Pt[q - pxy]) * c.rdz - rog;
      rfz[q] = (float)F;
      r_v = fmax(r_v, fabs(F));
    }
  }
}

__global__ void __launch_bounds__(256) k_mix_res_faces(Box b, Coef c, MixFaceIn in, float* __restrict__ rfx,
                                                       float* __restrict__ rfy, float* __restrict__ rfz,
                                                       unsigned long long* red) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  double r_v = 0.0;
  mix_res_faces_point(b, c, in, rfx, rfy, rfz, i, j, k, r_v);
  block_max_atomic(r_v, red + RED_V);
}

// Frozen mu-dependent coefficients of the correction problem: mu and the velocity pseudo-step
// dtau_V = fac / mu at centres, in FP32 (the iteration forms 2 mu/(1+xi) at centres and edges and
// the face pseudo-steps from them).
__device__ __forceinline__ void mix_coef_point(const Box& b, const Coef& c, const double* __restrict__ mu,
                                               const MixCoefOut& out, int i, int j, int k) {
  if (i < b.nx && j < b.ny && k < b.nz) {
    const long long q = cidx(b, i, j, k);
    out.mu[q] = (float)mu[q];
    out.dtvc[q] = (float)(c.dtauv_fac / mu[q]);
  }
}

__global__ void __launch_bounds__(256) k_mix_coef(Box b, Coef c, const double* __restrict__ mu, MixCoefOut out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  mix_coef_point(b, c, mu, out, i, j, (int)blockIdx.z);
}

// (iii) one FP32 PT iteration on the correction in a single pass.
//
// The iteration's two halves depend on each other across neighbours: the faces (momentum,
// damped R, dV) of level k read the cells' stresses and new dPt at k and k-1 (own cell, x- and
// y-neighbours below) and the edge stresses at k and k+1 (own edge, x- and y-neighbours above).
// A 32 x 8 block owns a tile of 30 x 6 faces and cells and marches up a column of face levels:
// at level L every thread computes the cell and the three lower edges at its index for the tile
// plus a one-cell halo on each side (the halo is recomputed by the neighbouring tiles' blocks from
// the same inputs, bit for bit), into rings in shared memory; after a barrier the tile's threads
// compute the faces of level L-1 from the rings. Stresses and the new dPt never go to global
// memory: per cell the pass reads dV, dPt, dPf, R, the right-hand sides and the frozen cc, k,
// 1/dtau_Pt, mu, dtau_V (18 arrays) and writes dV', dPt', dPf', R (8 arrays): 104 B per cell
// against 200 B for a cells kernel plus a faces kernel. dV is read from one buffer and written to
// another (other blocks' halos still read the old dV). The pseudo-step of dPf (largest neighbour
// k), the local-implicit denominators, 2 mu/(1+xi) at centres and edges (mean of the four
// centres' mu) and the face pseudo-steps (mean of the two centres') are formed here.
//
// Staging: the 12 arrays read at a point's own index go into a three-slot shared-memory ring by
// cp.async, one level ahead (levels L-1 and L resident while L+1 is in flight), so every x-, y-
// and z-1 neighbour a point reads comes from shared memory; only the three z+1 values of a cell
// (Vz; k and dPf for the Darcy flux) and the faces' own right-hand side and R are plain loads.
// The Darcy part (dPf', its residual) is formed for the tile's own cells only: the halo cells
// feed the faces through their stresses and dPt' alone.
constexpr int kCorrTX = 30, kCorrTY = 6, kCorrZChunk = 64;
enum { C_VX, C_VY, C_VZ, C_PT, C_PF, C_CC, C_K, C_IDTP, C_RPT, C_RPF, C_MU, C_DTV, kCorrStage };
// Blocks per SM asked of the register allocator.
constexpr int kCorrMinBlocks = 4;
// rings: cells (4 values) over three levels, edges (3) over two, staged inputs over three
constexpr int kCorrSmemBytes = (3 * 4 + 2 * 3 + 3 * kCorrStage) * 8 * 32 * (int)sizeof(float);

__device__ __forceinline__ void corr_cp4(float* smem, const float* gmem) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gmem) : "memory");
}

__device__ __forceinline__ float corr_modulus(const CorrCoef<float>& c, float m) {
  return __fdividef(2.0f * m, 1.0f + m * c.rG);
}

// One tile of the iteration: faces and cells of columns [tbx kCorrTX, +kCorrTX) x [tby kCorrTY,
// +kCorrTY) and face levels [k0, k1), by a 32 x 8 block whose dynamic shared memory (kCorrSmemBytes)
// starts at corr_smem. Leaves no copy in flight: the block may start another tile after a barrier.
__device__ __forceinline__ void corr_tile(const Box& b, const CorrCoef<float>& c, const CorrIn<float>& in,
                                          const CorrOut<float>& out, int tbx, int tby, int k0, int k1,
                                          unsigned long long* red, int check, float* corr_smem) {
  using T = float;
  T(*s_cell)[4][8][32] = reinterpret_cast<T(*)[4][8][32]>(corr_smem);                 // txx, tyy, tzz, dPt'
  T(*s_edge)[3][8][32] = reinterpret_cast<T(*)[3][8][32]>(corr_smem + 3 * 4 * 8 * 32);  // txy, txz, tyz
  T(*s_in)[kCorrStage][8][32] = reinterpret_cast<T(*)[kCorrStage][8][32]>(corr_smem + (3 * 4 + 2 * 3) * 8 * 32);
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int i = tbx * kCorrTX - 1 + tx;
  const int j = tby * kCorrTY - 1 + ty;
  const bool own = tx >= 1 && tx <= kCorrTX && ty >= 1 && ty <= kCorrTY;
  const int ipx = b.px, ipxy = (int)b.pxy;   // the host keeps the box below 2^31 elements
  // residual norms as bit patterns of non-negative doubles: a NaN (largest pattern) stays in them
  unsigned long long r_pt = 0ull, r_pf = 0ull, r_v = 0ull;
  auto keep_max = [](unsigned long long& m, float x) {
    const unsigned long long u = (unsigned long long)__double_as_longlong((double)fabsf(x));
    m = u > m ? u : m;
  };
  auto slot = [](int L) { return (L + 6) % 3; };     // L >= -2
  const bool in_box = i >= 0 && j >= 0 && i <= b.nx && j <= b.ny;
  auto stage = [&](int L) {   // own-index values of level L (inside the box) into its ring slot
    if (in_box && L >= 0 && L <= b.nz) {
      const int q = i + ipx * j + ipxy * L;
      float(*st)[8][32] = s_in[slot(L)];
      corr_cp4(&st[C_VX][ty][tx], in.Vx + q);
      corr_cp4(&st[C_VY][ty][tx], in.Vy + q);
      corr_cp4(&st[C_VZ][ty][tx], in.Vz + q);
      corr_cp4(&st[C_PT][ty][tx], in.Pt + q);
      corr_cp4(&st[C_PF][ty][tx], in.Pf + q);
      corr_cp4(&st[C_CC][ty][tx], in.cc + q);
      corr_cp4(&st[C_K][ty][tx], in.perm + q);
      corr_cp4(&st[C_IDTP][ty][tx], in.idtp + q);
      corr_cp4(&st[C_RPT][ty][tx], in.r_pt + q);
      corr_cp4(&st[C_RPF][ty][tx], in.r_pf + q);
      corr_cp4(&st[C_MU][ty][tx], in.mu + q);
      corr_cp4(&st[C_DTV][ty][tx], in.dtvc + q);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  T dtv_zm = T(0);   // dtau_V at (i, j, F - 1) for the z-face of level F (carried up the column)
  stage(k0 - 2);
  stage(k0 - 1);
  for (int L = k0 - 1; L <= k1; ++L) {
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");   // this thread's copies of level L landed
    // every thread's copies are visible (points read their neighbours' staged values), and every
    // thread is done with the previous level: its faces' ring slots and the stage slot L - 2
    __syncthreads();
    stage(L + 1);                                             // in flight while this level computes
    const float(*S)[8][32] = s_in[slot(L)];
    const float(*Sm)[8][32] = s_in[slot(L - 1)];
    const int sl = slot(L), se = L & 1;
    // the faces of level L - 1 read these after the cell phase: their loads go out first
    const int F = L - 1;
    const bool face_here = own && F >= k0 && F < k1 && in_box && F <= b.nz;
    T rfx = T(0), rfy = T(0), rfz = T(0), Rx0 = T(0), Ry0 = T(0), Rz0 = T(0);
    const bool fx = face_here && i > 0 && i < b.nx && j < b.ny && F < b.nz;
    const bool fy = face_here && j > 0 && j < b.ny && i < b.nx && F < b.nz;
    const bool fz = face_here && F > 0 && F < b.nz && i < b.nx && j < b.ny;
    if (face_here) {
      const int q = i + ipx * j + ipxy * F;
      if (fx) { rfx = in.rfx[q]; Rx0 = out.Rx[q]; }
      if (fy) { rfy = in.rfy[q]; Ry0 = out.Ry[q]; }
      if (fz) { rfz = in.rfz[q]; Rz0 = out.Rz[q]; }
    }
    // ---------------- cell and lower edges at (i, j, L). Cells are needed for the tile and its
    // left / lower halo (tx <= 30, ty <= 6), edges for the tile and its right / upper halo
    // (tx >= 1, ty >= 1); x-, y- and z-1 neighbours come from the stage ring.
    T txx = T(0), tyy = T(0), tzz = T(0), P1 = T(0), exy = T(0), exz = T(0), eyz = T(0);
    if (in_box && L >= 0 && L <= b.nz) {
      const int q = i + ipx * j + ipxy * L;
      const T mu_c = S[C_MU][ty][tx], vx_c = S[C_VX][ty][tx], vy_c = S[C_VY][ty][tx], vz_c = S[C_VZ][ty][tx];
      if (tx >= 1 && ty >= 1) {
        if (L < b.nz && i > 0 && i < b.nx && j > 0 && j < b.ny) {
          const T m = T(0.25) * (S[C_MU][ty - 1][tx - 1] + S[C_MU][ty - 1][tx] + S[C_MU][ty][tx - 1] + mu_c);
          exy = corr_modulus(c, m) * ((vx_c - S[C_VX][ty - 1][tx]) * c.hrdy + (vy_c - S[C_VY][ty][tx - 1]) * c.hrdx);
        }
        if (j < b.ny && i > 0 && i < b.nx && L > 0 && L < b.nz) {
          const T m = T(0.25) * (Sm[C_MU][ty][tx - 1] + Sm[C_MU][ty][tx] + S[C_MU][ty][tx - 1] + mu_c);
          exz = corr_modulus(c, m) * ((vx_c - Sm[C_VX][ty][tx]) * c.hrdz + (vz_c - S[C_VZ][ty][tx - 1]) * c.hrdx);
        }
        if (i < b.nx && j > 0 && j < b.ny && L > 0 && L < b.nz) {
          const T m = T(0.25) * (Sm[C_MU][ty - 1][tx] + Sm[C_MU][ty][tx] + S[C_MU][ty - 1][tx] + mu_c);
          eyz = corr_modulus(c, m) * ((vy_c - Sm[C_VY][ty][tx]) * c.hrdz + (vz_c - S[C_VZ][ty - 1][tx]) * c.hrdy);
        }
      }
      if (tx <= kCorrTX && ty <= kCorrTY && i < b.nx && j < b.ny && L < b.nz) {
        const T dPt = S[C_PT][ty][tx], dPf = S[C_PF][ty][tx], cc = S[C_CC][ty][tx];
        const T rpt = S[C_RPT][ty][tx];
        const T gx = (S[C_VX][ty][tx + 1] - vx_c) * c.rdx, gy = (S[C_VY][ty + 1][tx] - vy_c) * c.rdy;
        const T gz = (in.Vz[q + ipxy] - vz_c) * c.rdz;
        const T divV = gx + gy + gz;
        const T cpl = c.bd_rdt_a + cc;                 // beta_d alpha / dt + cc
        const T rho_pt = rpt + divV + (c.bd_rdt + cc) * dPt - cpl * dPf;
        // dP' = dP - dtau rho(dP', ...) solved for dP' (local terms implicit; the quotient only
        // scales the pseudo-step, so the fast reciprocal does)
        const T idtp = S[C_IDTP][ty][tx];
        const T dPt1 = __fdividef(dPt * idtp - (rpt + divV - cpl * dPf), idtp + c.bd_rdt + cc);
        const T third = divV * T(1.0 / 3.0);
        const T bn = c.beta_n * (rho_pt - rpt);
        const T cm2 = corr_modulus(c, mu_c);
        txx = cm2 * (gx - third + bn);
        tyy = cm2 * (gy - third + bn);
        tzz = cm2 * (gz - third + bn);
        P1 = out.eval ? dPt : dPt1;
        if (own && L >= k0 && L < k1) {
          // Darcy flux divergence, the largest neighbour k and dPf' (the tile's own cells)
          const T rpf = S[C_RPF][ty][tx], kc = S[C_K][ty][tx];
          T kmax = kc, sx = T(0), sy = T(0), sz = T(0);
          if (i > 0) {
            const T kn = S[C_K][ty][tx - 1];
            kmax = fmaxf(kmax, kn);
            sx -= (kn + kc) * (dPf - S[C_PF][ty][tx - 1]);
          }
          if (i < b.nx - 1) {
            const T kn = S[C_K][ty][tx + 1];
            kmax = fmaxf(kmax, kn);
            sx += (kc + kn) * (S[C_PF][ty][tx + 1] - dPf);
          }
          if (j > 0) {
            const T kn = S[C_K][ty - 1][tx];
            kmax = fmaxf(kmax, kn);
            sy -= (kn + kc) * (dPf - S[C_PF][ty - 1][tx]);
          }
          if (j < b.ny - 1) {
            const T kn = S[C_K][ty + 1][tx];
            kmax = fmaxf(kmax, kn);
            sy += (kc + kn) * (S[C_PF][ty + 1][tx] - dPf);
          }
          if (L > 0) {
            const T kn = Sm[C_K][ty][tx];
            kmax = fmaxf(kmax, kn);
            sz -= (kn + kc) * (dPf - Sm[C_PF][ty][tx]);
          }
          if (L < b.nz - 1) {
            const T kn = in.perm[q + ipxy];
            kmax = fmaxf(kmax, kn);
            sz += (kc + kn) * (in.Pf[q + ipxy] - dPf);
          }
          const T divq = -(sx * c.hrdx2 + sy * c.hrdy2 + sz * c.hrdz2);
          const T rho_pf = rpf + divq + (c.bda_B_rdt + cc) * dPf - cpl * dPt;
          const T idtf = kmax * c.ifac_pf;
          const T dPf1 = __fdividef(dPf * idtf - (rpf + divq - cpl * dPt), idtf + c.bda_B_rdt + cc);
          if (!out.eval) {
            out.Pt[q] = dPt1;
            out.Pf[q] = dPf1;
          }
          if (out.res_pt) {
            out.res_pt[q] = rho_pt;
            out.res_pf[q] = rho_pf;
          }
          if (check) {
            keep_max(r_pt, rho_pt);
            keep_max(r_pf, rho_pf);
          }
        }
      }
    }
    s_cell[sl][0][ty][tx] = txx;
    s_cell[sl][1][ty][tx] = tyy;
    s_cell[sl][2][ty][tx] = tzz;
    s_cell[sl][3][ty][tx] = P1;
    s_edge[se][0][ty][tx] = exy;
    s_edge[se][1][ty][tx] = exz;
    s_edge[se][2][ty][tx] = eyz;
    __syncthreads();
    // ---------------- faces of level F = L - 1 (cells at F and F-1, edges at F and L = F+1;
    // V and dtau_V at F from the stage slot of F, dtau_V at F - 1 carried from the level below)
    if (face_here) {
      const int sf = slot(F), sb = slot(F - 1), ef = F & 1, eu = se;
      const int q = i + ipx * j + ipxy * F;
      const T Pc = s_cell[sf][3][ty][tx];
      const T dtv_c = Sm[C_DTV][ty][tx];
      T Fx = T(0), Fy = T(0), Fz = T(0);
      if (fx) {
        Fx = rfx + (s_cell[sf][0][ty][tx] - s_cell[sf][0][ty][tx - 1]) * c.rdx +
             (s_edge[ef][0][ty + 1][tx] - s_edge[ef][0][ty][tx]) * c.rdy +
             (s_edge[eu][1][ty][tx] - s_edge[ef][1][ty][tx]) * c.rdz - (Pc - s_cell[sf][3][ty][tx - 1]) * c.rdx;
        const T R1 = Fx * c.rrho_i + c.damp_x * Rx0;
        out.Rx[q] = R1;
        if (!out.eval) out.Vx[q] = Sm[C_VX][ty][tx] + T(0.5) * (Sm[C_DTV][ty][tx - 1] + dtv_c) * R1;
      }
      if (fy) {
        Fy = rfy + (s_edge[ef][0][ty][tx + 1] - s_edge[ef][0][ty][tx]) * c.rdx +
             (s_cell[sf][1][ty][tx] - s_cell[sf][1][ty - 1][tx]) * c.rdy +
             (s_edge[eu][2][ty][tx] - s_edge[ef][2][ty][tx]) * c.rdz - (Pc - s_cell[sf][3][ty - 1][tx]) * c.rdy;
        const T R1 = Fy * c.rrho_i + c.damp_y * Ry0;
        out.Ry[q] = R1;
        if (!out.eval) out.Vy[q] = Sm[C_VY][ty][tx] + T(0.5) * (Sm[C_DTV][ty - 1][tx] + dtv_c) * R1;
      }
      if (fz) {
        Fz = rfz + (s_edge[ef][1][ty][tx + 1] - s_edge[ef][1][ty][tx]) * c.rdx +
             (s_edge[ef][2][ty + 1][tx] - s_edge[ef][2][ty][tx]) * c.rdy +
             (s_cell[sf][2][ty][tx] - s_cell[sb][2][ty][tx]) * c.rdz - (Pc - s_cell[sb][3][ty][tx]) * c.rdz;
        const T R1 = Fz * c.rrho_i + c.damp_z * Rz0;
        out.Rz[q] = R1;
        if (!out.eval) out.Vz[q] = Sm[C_VZ][ty][tx] + T(0.5) * (dtv_zm + dtv_c) * R1;
      }
      if (check) {
        keep_max(r_v, Fx);
        keep_max(r_v, Fy);
        keep_max(r_v, Fz);
      }
    }
    // dtau_V at (i, j, L - 1), the z-face of the next level's lower pseudo-step
    dtv_zm = (in_box && L >= 1 && L - 1 <= b.nz) ? Sm[C_DTV][ty][tx] : T(0);
  }
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");   // the last level's look-ahead copies
  if (check) {
    block_max_atomic(__longlong_as_double((long long)r_pt), red + RED_PT);
    block_max_atomic(__longlong_as_double((long long)r_pf), red + RED_PF);
    block_max_atomic(__longlong_as_double((long long)r_v), red + RED_V);
  }
}

__global__ void __launch_bounds__(256, kCorrMinBlocks) k_corr_iteration(Box b, CorrCoef<float> c, CorrIn<float> in,
                                                        CorrOut<float> out, unsigned long long* red, int check) {
  extern __shared__ __align__(16) float corr_smem[];   // kCorrSmemBytes, dynamic (above 48 KB)
  const int k0 = blockIdx.z * kCorrZChunk;
  corr_tile(b, c, in, out, blockIdx.x, blockIdx.y, k0, min(k0 + kCorrZChunk, b.nz + 1), red, check, corr_smem);
}

// (iv) u <- u + delta (FP64 += FP32 correction).
__device__ __forceinline__ void mix_update_point(const Box& b, const MixUpdate& u, int i, int j, int k) {
  if (i > b.nx || j > b.ny || k > b.nz) return;
  const long long q = cidx(b, i, j, k);
  const double w = u.omega;
  if (i > 0 && i < b.nx && j < b.ny && k < b.nz) u.Vx[q] = fma(w, (double)u.dVx[q], u.Vx[q]);
  if (j > 0 && j < b.ny && i < b.nx && k < b.nz) u.Vy[q] = fma(w, (double)u.dVy[q], u.Vy[q]);
  if (k > 0 && k < b.nz && i < b.nx && j < b.ny) u.Vz[q] = fma(w, (double)u.dVz[q], u.Vz[q]);
  if (i < b.nx && j < b.ny && k < b.nz) {
    u.Pt[q] = fma(w, (double)u.dPt[q], u.Pt[q]);
    u.Pf[q] = fma(w, (double)u.dPf[q], u.Pf[q]);
  }
}

__global__ void __launch_bounds__(256) k_mix_update(Box b, MixUpdate u) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  mix_update_point(b, u, i, j, (int)blockIdx.z);
}

void mix_prepare(dim3 g, dim3 bl, cudaStream_t s, Box b, const Coef& c, const MixPrepIn& in,
                 const MixPrepOut& out, unsigned long long* red) {
  k_mix_prepare<<<g, bl, 0, s>>>(b, c, in, out, red);
}
void mix_res_faces(dim3 g, dim3 bl, cudaStream_t s, Box b, const Coef& c, const MixFaceIn& in, float* rfx,
                   float* rfy, float* rfz, unsigned long long* red) {
  k_mix_res_faces<<<g, bl, 0, s>>>(b, c, in, rfx, rfy, rfz, red);
}
void mix_edges(dim3 g, dim3 bl, cudaStream_t s, Box b, const Coef& c, const EdgeIn& in, const EdgeOut& out) {
  k_mix_edges<<<g, bl, 0, s>>>(b, c, in, out);
}
void mix_porosity(dim3 g, dim3 bl, cudaStream_t s, Box b, const Coef& c, const MixPorosity& p) {
  k_mix_porosity<<<g, bl, 0, s>>>(b, c, p);
}
void mix_coef(dim3 g, dim3 bl, cudaStream_t s, Box b, const Coef& c, const double* mu, const MixCoefOut& out) {
  k_mix_coef<<<g, bl, 0, s>>>(b, c, mu, out);
}
void mix_update(dim3 g, dim3 bl, cudaStream_t s, Box b, const MixUpdate& u) {
  k_mix_update<<<g, bl, 0, s>>>(b, u);
}
void corr_iteration(cudaStream_t s, Box b, const CorrCoef<float>& c, const CorrIn<float>& in,
                    const CorrOut<float>& out, unsigned long long* red, int check) {
  const dim3 g((unsigned)((b.nx + 1 + kCorrTX - 1) / kCorrTX), (unsigned)((b.ny + 1 + kCorrTY - 1) / kCorrTY),
               (unsigned)((b.nz + 1 + kCorrZChunk - 1) / kCorrZChunk));
  cudaFuncSetAttribute(k_corr_iteration, cudaFuncAttributeMaxDynamicSharedMemorySize, kCorrSmemBytes);
  k_corr_iteration<<<g, dim3(32, 8, 1), kCorrSmemBytes, s>>>(b, c, in, out, red, check);
}


// ============================================================ multigrid transfers (FP32)
// Level f (fine, n cells per direction) and level c (coarse, ceil(n / 2)), through the weight
// tables of c.ax (MgAxis).
__global__ void __launch_bounds__(256) k_mg_coef(MgLevel f, MgLevel c, float dtaupt_fac, float dtauv_fac) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x, J = blockIdx.y * blockDim.y + threadIdx.y;
  const int K = blockIdx.z;
  if (I >= c.b.nx || J >= c.b.ny || K >= c.b.nz) return;
  const int i0 = c.ax[0].box_i0[I], j0 = c.ax[1].box_i0[J], k0 = c.ax[2].box_i0[K];
  const float* wx = c.ax[0].box_w + 3 * I;
  const float* wy = c.ax[1].box_w + 3 * J;
  const float* wz = c.ax[2].box_w + 3 * K;
  float m = 0.f, k = 0.f, cc = 0.f;
  for (int dz = 0; dz < 3; ++dz)
    for (int dy = 0; dy < 3; ++dy)
      for (int dx = 0; dx < 3; ++dx) {
        const float w = wx[dx] * wy[dy] * wz[dz];
        if (w == 0.f) continue;
        const long long q = cidx(f.b, i0 + dx, j0 + dy, k0 + dz);
        m += w * f.mu[q];
        k += w * f.perm[q];
        cc += w * f.cc[q];
      }
  const long long qc = cidx(c.b, I, J, K);
  c.mu[qc] = m;
  c.perm[qc] = k;
  c.cc[qc] = cc;
  c.idtp[qc] = 1.0f / (dtaupt_fac * m);
  c.dtvc[qc] = dtauv_fac / m;
}

__global__ void __launch_bounds__(256) k_mg_restrict(MgLevel f, MgLevel c, float rho_i) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x, J = blockIdx.y * blockDim.y + threadIdx.y;
  const int K = blockIdx.z;
  const Box& B = c.b;
  if (I > B.nx || J > B.ny || K > B.nz) return;
  const long long qc = cidx(B, I, J, K);
  // a zero correction and damped residual on the coarse grid (walls included)
  c.dVx[0][qc] = 0.f; c.dVx[1][qc] = 0.f; c.dVy[0][qc] = 0.f; c.dVy[1][qc] = 0.f;
  c.dVz[0][qc] = 0.f; c.dVz[1][qc] = 0.f; c.dPt[0][qc] = 0.f; c.dPf[0][qc] = 0.f;
  c.Rx[qc] = 0.f; c.Ry[qc] = 0.f; c.Rz[qc] = 0.f;
  const Box& F = f.b;
  const MgAxis &X = c.ax[0], &Y = c.ax[1], &Z = c.ax[2];
  if (I < B.nx && J < B.ny && K < B.nz) {
    const int i0 = X.box_i0[I], j0 = Y.box_i0[J], k0 = Z.box_i0[K];
    const float *bx = X.box_w + 3 * I, *by = Y.box_w + 3 * J, *bz = Z.box_w + 3 * K;
    float a = 0.f, b = 0.f;
    for (int dz = 0; dz < 3; ++dz)
      for (int dy = 0; dy < 3; ++dy)
        for (int dx = 0; dx < 3; ++dx) {
          const float w = bx[dx] * by[dy] * bz[dz];
          if (w == 0.f) continue;
          const long long q = cidx(F, i0 + dx, j0 + dy, k0 + dz);
          a += w * f.res_pt[q];
          b += w * f.res_pf[q];
        }
    c.rpt[qc] = a;
    c.rpf[qc] = b;
  }
  // faces: hat weights along the normal, box weights across it
  if (I > 0 && I < B.nx && J < B.ny && K < B.nz) {
    const int i0 = X.hat_i0[I], j0 = Y.box_i0[J], k0 = Z.box_i0[K];
    const float *h = X.hat_w + 4 * I, *by = Y.box_w + 3 * J, *bz = Z.box_w + 3 * K;
    float s = 0.f;
    for (int dz = 0; dz < 3; ++dz)
      for (int dy = 0; dy < 3; ++dy)
        for (int dx = 0; dx < 4; ++dx) {
          const float w = h[dx] * by[dy] * bz[dz];
          if (w == 0.f) continue;
          s += w * f.Rx[cidx(F, i0 + dx, j0 + dy, k0 + dz)];
        }
    c.rfx[qc] = rho_i * s;
  }
  if (J > 0 && J < B.ny && I < B.nx && K < B.nz) {
    const int i0 = X.box_i0[I], j0 = Y.hat_i0[J], k0 = Z.box_i0[K];
    const float *bx = X.box_w + 3 * I, *h = Y.hat_w + 4 * J, *bz = Z.box_w + 3 * K;
    float s = 0.f;
    for (int dz = 0; dz < 3; ++dz)
      for (int dy = 0; dy < 4; ++dy)
        for (int dx = 0; dx < 3; ++dx) {
          const float w = bx[dx] * h[dy] * bz[dz];
          if (w == 0.f) continue;
          s += w * f.Ry[cidx(F, i0 + dx, j0 + dy, k0 + dz)];
        }
    c.rfy[qc] = rho_i * s;
  }
  if (K > 0 && K < B.nz && I < B.nx && J < B.ny) {
    const int i0 = X.box_i0[I], j0 = Y.box_i0[J], k0 = Z.hat_i0[K];
    const float *bx = X.box_w + 3 * I, *by = Y.box_w + 3 * J, *h = Z.hat_w + 4 * K;
    float s = 0.f;
    for (int dz = 0; dz < 4; ++dz)
      for (int dy = 0; dy < 3; ++dy)
        for (int dx = 0; dx < 3; ++dx) {
          const float w = bx[dx] * by[dy] * h[dz];
          if (w == 0.f) continue;
          s += w * f.Rz[cidx(F, i0 + dx, j0 + dy, k0 + dz)];
        }
    c.rfz[qc] = rho_i * s;
  }
}

__global__ void __launch_bounds__(256) k_mg_prolong(MgLevel c, int dc, MgLevel f, int df) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  const Box& B = f.b;
  if (i > B.nx || j > B.ny || k > B.nz) return;
  const long long q = cidx(B, i, j, k);
  const MgAxis &X = c.ax[0], &Y = c.ax[1], &Z = c.ax[2];
  if (i < B.nx && j < B.ny && k < B.nz) {   // cells: trilinear between coarse centres
    float pt = 0.f, pf = 0.f;
    for (int a = 0; a < 2; ++a)
      for (int bb = 0; bb < 2; ++bb)
        for (int cc = 0; cc < 2; ++cc) {
          const float w = Z.lin_w[2 * k + a] * Y.lin_w[2 * j + bb] * X.lin_w[2 * i + cc];
          const long long qc = cidx(c.b, X.lin_ab[2 * i + cc], Y.lin_ab[2 * j + bb], Z.lin_ab[2 * k + a]);
          pt += w * c.dPt[dc][qc];
          pf += w * c.dPf[dc][qc];
        }
    f.dPt[df][q] += pt;
    f.dPf[df][q] += pf;
  }
  // faces: linear between coarse faces along the normal (coarse wall faces are zero), between
  // coarse centres across it
  if (i > 0 && i < B.nx && j < B.ny && k < B.nz) {
    const int n0 = X.fl_n0[i];
    const float t = X.fl_t[i];
    float v = 0.f;
    for (int a = 0; a < 2; ++a)
      for (int bb = 0; bb < 2; ++bb) {
        const int y = Y.lin_ab[2 * j + bb], z = Z.lin_ab[2 * k + a];
        v += Z.lin_w[2 * k + a] * Y.lin_w[2 * j + bb] *
             ((1.f - t) * c.dVx[dc][cidx(c.b, n0, y, z)] + t * c.dVx[dc][cidx(c.b, n0 + 1, y, z)]);
      }
    f.dVx[df][q] += v;
  }
  if (j > 0 && j < B.ny && i < B.nx && k < B.nz) {
    const int n0 = Y.fl_n0[j];
    const float t = Y.fl_t[j];
    float v = 0.f;
    for (int a = 0; a < 2; ++a)
      for (int cc = 0; cc < 2; ++cc) {
        const int x = X.lin_ab[2 * i + cc], z = Z.lin_ab[2 * k + a];
        v += Z.lin_w[2 * k + a] * X.lin_w[2 * i + cc] *
             ((1.f - t) * c.dVy[dc][cidx(c.b, x, n0, z)] + t * c.dVy[dc][cidx(c.b, x, n0 + 1, z)]);
      }
    f.dVy[df][q] += v;
  }
  if (k > 0 && k < B.nz && i < B.nx && j < B.ny) {
    const int n0 = Z.fl_n0[k];
    const float t = Z.fl_t[k];
    float v = 0.f;
    for (int bb = 0; bb < 2; ++bb)
      for (int cc = 0; cc < 2; ++cc) {
        const int x = X.lin_ab[2 * i + cc], y = Y.lin_ab[2 * j + bb];
        v += Y.lin_w[2 * j + bb] * X.lin_w[2 * i + cc] *
             ((1.f - t) * c.dVz[dc][cidx(c.b, x, y, n0)] + t * c.dVz[dc][cidx(c.b, x, y, n0 + 1)]);
      }
    f.dVz[df][q] += v;
  }
}

void mg_coef(cudaStream_t s, const MgLevel& f, const MgLevel& c, float dtaupt_fac, float dtauv_fac) {
  const dim3 bl(32, 8, 1), g((c.b.nx + 31) / 32, (c.b.ny + 7) / 8, c.b.nz);
  k_mg_coef<<<g, bl, 0, s>>>(f, c, dtaupt_fac, dtauv_fac);
}
void mg_restrict(cudaStream_t s, const MgLevel& f, const MgLevel& c, float rho_i) {
  const dim3 bl(32, 8, 1), g((c.b.nx + 1 + 31) / 32, (c.b.ny + 1 + 7) / 8, c.b.nz + 1);
  k_mg_restrict<<<g, bl, 0, s>>>(f, c, rho_i);
}
void mg_prolong(cudaStream_t s, const MgLevel& c, int dc, const MgLevel& f, int df) {
  const dim3 bl(32, 8, 1), g((f.b.nx + 1 + 31) / 32, (f.b.ny + 1 + 7) / 8, f.b.nz + 1);
  k_mg_prolong<<<g, bl, 0, s>>>(c, dc, f, df);
}

// ============================================================ batched FP32 ensembles (engine)
namespace {

__device__ inline unsigned long long mb_global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Last member whose first work item (tile_base or ctile_base) is <= t.
template <long long MixBatchInst::*BASE>
__device__ inline int mb_find(const MixBatchInst* inst, int ninst, long long t) {
  int lo = 0, hi = ninst - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (inst[mid].*BASE <= t) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// The first work item >= `next` that this CTA visits in a grid stride starting at blockIdx.x:
// a CTA skips a member that has no work in a launch in one step instead of tile by tile.
__device__ inline long long mb_skip_to(long long next, long long t0) {
  const long long g = gridDim.x;
  return next + ((t0 + (long long)blockIdx.x - next) % g + g) % g;
}

__device__ inline bool mb_runs(int phase, const MixBatchStatus& s) {
  switch (phase) {
    case MB_PH_PERM: case MB_PH_PREP: case MB_PH_FACES: return s.phase == MB_PREP;
    case MB_PH_INIT: return s.phase == MB_INNER && s.fresh;
    default: return s.phase == MB_UPDATE;
  }
}

constexpr int kMbBX = 32, kMbBY = 8;   // point tiles: 32 x 8 cells of one z-level

}  // namespace

// The point phases over every member's tiles (grid-stride over the flat work list; a member not
// in the phase skips its tiles, uniformly per CTA, so the block-wide reductions stay collective).
template <int PHASE>
__global__ void __launch_bounds__(kMbBX * kMbBY) k_mb_points(const MixBatchInst* __restrict__ inst,
                                                            const MixBatchStatus* __restrict__ st, int ninst,
                                                            long long t0, long long t1) {
  for (long long t = t0 + blockIdx.x; t < t1; t += gridDim.x) {
    const int m = mb_find<&MixBatchInst::tile_base>(inst, ninst, t);
    const MixBatchStatus& S = st[m];
    if (!mb_runs(PHASE, S)) {   // uniform over the CTA: on to the next member's tiles
      t = mb_skip_to(m + 1 < ninst ? inst[m + 1].tile_base : t1, t0) - gridDim.x;
      continue;
    }
    const MixBatchInst& I = inst[m];
    const long long local = t - I.tile_base;
    const long long per_z = (long long)I.gx * I.gy;
    const int kz = (int)(local / per_z);
    const int r = (int)(local - (long long)kz * per_z);
    const int ty = r / I.gx, tx = r - ty * I.gx;
    const int i = tx * kMbBX + threadIdx.x, j = ty * kMbBY + threadIdx.y;
    const Box& b = I.b;
    const int a = S.cur;
    if (PHASE == MB_PH_PERM) {
      perm_point(b, I.k, I.phi[a], I.logk, I.perm, I.rog, i, j, kz);
    } else if (PHASE == MB_PH_PREP) {
      const MixPrepIn pin{I.Vx, I.Vy, I.Vz, I.Pt[a], I.Pf[a], I.phi[a], I.mu, I.eta, I.perm, I.Pto, I.Pfo,
                          I.txxo, I.tyyo, I.tzzo};
      const MixPrepOut pout{I.s_txx, I.s_tyy, I.s_tzz, I.rpt, I.rpf, I.ccf, I.kf, I.idtp};
      double r_pt = 0.0, r_pf = 0.0;
      mix_prepare_point(b, I.k, pin, pout, i, j, kz, r_pt, r_pf);
      edges_point<true>(b, I.k, EdgeIn{I.Vx, I.Vy, I.Vz, I.mu, I.txyo, I.txzo, I.tyzo},
                        EdgeOut{I.s_txy, I.s_txz, I.s_tyz}, i, j, kz);
      block_max_atomic(r_pt, I.red + RED_PT);
      block_max_atomic(r_pf, I.red + RED_PF);
    } else if (PHASE == MB_PH_FACES) {
      double r_v = 0.0, pic = 1.0;
      mix_res_faces_point(b, I.k, MixFaceIn{I.s_txx, I.s_tyy, I.s_tzz, I.s_txy, I.s_txz, I.s_tyz, I.Pt[a], I.phi[a]},
                          I.rfx, I.rfy, I.rfz, i, j, kz, r_v);
      lean_picard_point(b, I.lc,
                        LeanPicardIn<double>{I.s_txx, I.s_tyy, I.s_tzz, I.s_txy, I.s_txz, I.s_tyz, I.phi[a],
                                             I.Pt[a], I.Pf[a]},
                        I.mu, I.eta, i, j, kz, pic);
      block_max_atomic(r_v, I.red + RED_V);
      block_max_log_atomic(pic, I.red + RED_PIC);
    } else if (PHASE == MB_PH_INIT) {
      mix_coef_point(b, I.k, I.mu, MixCoefOut{I.muf, I.dtvc}, i, j, kz);
      if (i <= b.nx && j <= b.ny && kz <= b.nz) {   // a zero correction and damped residual
        const long long q = cidx(b, i, j, kz);
        I.dVx[0][q] = 0.f; I.dVx[1][q] = 0.f; I.dVy[0][q] = 0.f; I.dVy[1][q] = 0.f;
        I.dVz[0][q] = 0.f; I.dVz[1][q] = 0.f; I.dPt[0][q] = 0.f; I.dPf[0][q] = 0.f;
        I.Rx[q] = 0.f; I.Ry[q] = 0.f; I.Rz[q] = 0.f;
      }
    } else if (PHASE == MB_PH_UPDATE) {
      const int d = S.inner & 1;   // the last correction's buffer
      mix_update_point(b, MixUpdate{I.Vx, I.Vy, I.Vz, I.Pt[a], I.Pf[a], I.dVx[d], I.dVy[d], I.dVz[d], I.dPt[d],
                                    I.dPf[d], S.omega}, i, j, kz);
    } else {   // MB_PH_POROSITY: phi moves to the other buffer, the pressures follow it
      porosity_point<true>(b, I.k, I.Vx, I.Vy, I.Vz, I.phi[a], I.Pt[a], I.Pf[a], I.Pto, I.Pfo, I.Lo, I.eta,
                           I.phi[1 - a], i, j, kz);
      if (i < b.nx && j < b.ny && kz < b.nz) {
        const long long q = cidx(b, i, j, kz);
        I.Pt[1 - a][q] = I.Pt[a][q];
        I.Pf[1 - a][q] = I.Pf[a][q];
      }
    }
  }
}

// Correction iteration number inner + step of the members in MB_INNER (within their budget),
// one corr_tile per work item; the block's shared memory is reused from tile to tile.
template <int MINB>
__global__ void __launch_bounds__(256, MINB) k_mb_corr(const MixBatchInst* __restrict__ inst,
                                                       const MixBatchStatus* __restrict__ st, int ninst,
                                                       long long t0, long long t1, int step, int nup,
                                                       int zchunk) {
  extern __shared__ __align__(16) float corr_smem[];
  __shared__ CorrCoef<float> s_cc;   // the member's coefficients, read from shared memory by the tile
  for (long long t = t0 + blockIdx.x; t < t1; t += gridDim.x) {
    const int m = mb_find<&MixBatchInst::ctile_base>(inst, ninst, t);
    const MixBatchStatus& S = st[m];
    const MixBatchInst& I = inst[m];
    const int it = S.inner + step;
    if (S.phase != MB_INNER || it > I.max_iter - S.iters) {   // uniform over the CTA
      t = mb_skip_to(m + 1 < ninst ? inst[m + 1].ctile_base : t1, t0) - gridDim.x;
      continue;
    }
    const int d = (it - 1) & 1;
    if (threadIdx.x == 0 && threadIdx.y == 0) s_cc = I.cc;
    // the argument pointers as offsets of one base (cheap to recompute, unlike pointers loaded
    // from the descriptor): slots rpt, rpf, rfx, rfy, rfz, cc, k, idtp, mu, dtvc, dVx[2], dVy[2],
    // dVz[2], dPt[2], dPf[2], Rx, Ry, Rz
    float* const B = const_cast<float*>(I.fbase);
    const long long fs = I.fstride;
    auto P = [B, fs](int slot) { return B + slot * fs; };
    const CorrIn<float> ci{P(10 + d), P(12 + d), P(14 + d), P(16 + d), P(18 + d), P(5), P(6), P(7), P(0), P(1),
                           P(8), P(9), P(2), P(3), P(4)};
    const CorrOut<float> co{P(11 - d), P(13 - d), P(15 - d), P(17 - d), P(19 - d), P(20), P(21), P(22)};
    const long long local = t - I.ctile_base;
    const long long per_z = (long long)I.cgx * I.cgy;
    const int bz = (int)(local / per_z);
    const int r = (int)(local - (long long)bz * per_z);
    const int tby = r / I.cgx, tbx = r - tby * I.cgx;
    const int k0 = bz * zchunk;
    const Box b = I.b;
    unsigned long long* const ired = I.ired;
    __syncthreads();   // s_cc written
    corr_tile(b, s_cc, ci, co, tbx, tby, k0, min(k0 + zchunk, b.nz + 1), ired, step == nup, corr_smem);
    __syncthreads();   // the next tile's stage and rings overwrite this one's
  }
}

// Outer decision of the members in MB_PREP (the host loop's, in the same order): non-finite
// norms stop the member (PT_ENAN), norms below tol end its step (PT_OK); otherwise the outer
// weight adapts (halved down to 1/16 when the residual more than doubled, grown by 1.25 up to 1
// while it falls), the inner target is rtol times the residual, and a correction solve starts.
__global__ void k_mb_decide_outer(const MixBatchInst* __restrict__ inst, MixBatchStatus* __restrict__ st,
                                  int ninst) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= ninst || st[m].phase != MB_PREP) return;
  MixBatchStatus& S = st[m];
  unsigned long long* red = inst[m].red;
  const int slot[4] = {RED_V, RED_PT, RED_PF, RED_PIC};
  bool finite = true;
  double r = 0.0;
  for (int s = 0; s < 4; ++s) {
    const double v = __longlong_as_double((long long)red[slot[s]]);
    S.res[s] = v;
    finite = finite && isfinite(v);
    r = fmax(r, v);
    red[slot[s]] = 0ull;
  }
  if (!finite) {
    S.phase = MB_DONE;
    S.status = PT_ENAN;
    S.t_stop = mb_global_ns();
    return;
  }
  if (r < inst[m].tol) {
    S.phase = MB_DONE;
    S.status = PT_OK;
    S.t_stop = mb_global_ns();
    return;
  }
  if (S.prev > 0.0) {
    if (r > 2.0 * S.prev) S.omega = fmax(S.omega * 0.5, 0.0625);
    else if (r < S.prev) S.omega = fmin(S.omega * 1.25, 1.0);
  }
  S.prev = r;
  S.target = inst[m].rtol * r;
  S.phase = MB_INNER;
  S.fresh = 1;
  S.inner = 0;
}

// Inner decision after `nup` correction launches: the iterations that ran are counted; after a
// check iteration a non-finite norm stops the member (PT_ENAN) and a drop below the target ends
// the solve; so does a spent budget (max_iter - iters).
__global__ void k_mb_decide_inner(const MixBatchInst* __restrict__ inst, MixBatchStatus* __restrict__ st,
                                  int ninst, int nup) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= ninst || st[m].phase != MB_INNER) return;
  MixBatchStatus& S = st[m];
  S.fresh = 0;
  const int budget = inst[m].max_iter - S.iters;
  const int ran = min(nup, budget - S.inner);
  S.inner += ran;
  bool stop = S.inner >= budget;
  if (ran == nup) {   // the last launch was a check iteration
    unsigned long long* red = inst[m].ired;
    const double v = __longlong_as_double((long long)red[RED_V]);
    const double pt = __longlong_as_double((long long)red[RED_PT]);
    const double pf = __longlong_as_double((long long)red[RED_PF]);
    red[RED_V] = 0ull;
    red[RED_PT] = 0ull;
    red[RED_PF] = 0ull;
    if (!(isfinite(v) && isfinite(pt) && isfinite(pf))) {
      S.iters += S.inner;
      S.phase = MB_DONE;
      S.status = PT_ENAN;
      S.t_stop = mb_global_ns();
      return;
    }
    if (fmax(fmax(v, pt), pf) < S.target) stop = true;
  }
  if (stop) S.phase = MB_UPDATE;
}

// End of an outer iteration: the iterate moved to the other buffers; the solve's iterations are
// counted; a member whose budget is spent stops unconverged (PT_ENOTCONV), the others go on.
__global__ void k_mb_finish(const MixBatchInst* __restrict__ inst, MixBatchStatus* __restrict__ st, int ninst) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= ninst || st[m].phase != MB_UPDATE) return;
  MixBatchStatus& S = st[m];
  S.cur = 1 - S.cur;
  S.iters += S.inner;
  S.inner = 0;
  S.outer += 1;
  if (S.iters >= inst[m].max_iter) {
    S.phase = MB_DONE;
    S.status = PT_ENOTCONV;
    S.t_stop = mb_global_ns();
  } else {
    S.phase = MB_PREP;
  }
}

__global__ void k_mb_start(const MixBatchInst* __restrict__ inst, MixBatchStatus* __restrict__ st, int ninst) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= ninst) return;
  MixBatchStatus& S = st[m];
  S.phase = MB_PREP;
  S.cur = 0;
  S.inner = 0;
  S.iters = 0;
  S.outer = 0;
  S.status = PT_ENOTCONV;
  S.fresh = 0;
  S.omega = 1.0;
  S.prev = 0.0;
  S.target = 0.0;
  for (int s = 0; s < 4; ++s) S.res[s] = 0.0;
  for (int s = 0; s < RED_N; ++s) {
    inst[m].red[s] = 0ull;
    inst[m].ired[s] = 0ull;
  }
  S.t_start = mb_global_ns();
  S.t_stop = 0ull;
}

void mb_points(int grid, cudaStream_t s, int phase, const MixBatchInst* inst, const MixBatchStatus* st, int ninst,
               long long t0, long long t1) {
  const dim3 bl(kMbBX, kMbBY, 1);
  switch (phase) {
    case MB_PH_PERM: k_mb_points<MB_PH_PERM><<<grid, bl, 0, s>>>(inst, st, ninst, t0, t1); break;
    case MB_PH_PREP: k_mb_points<MB_PH_PREP><<<grid, bl, 0, s>>>(inst, st, ninst, t0, t1); break;
    case MB_PH_FACES: k_mb_points<MB_PH_FACES><<<grid, bl, 0, s>>>(inst, st, ninst, t0, t1); break;
    case MB_PH_INIT: k_mb_points<MB_PH_INIT><<<grid, bl, 0, s>>>(inst, st, ninst, t0, t1); break;
    case MB_PH_UPDATE: k_mb_points<MB_PH_UPDATE><<<grid, bl, 0, s>>>(inst, st, ninst, t0, t1); break;
    default: k_mb_points<MB_PH_POROSITY><<<grid, bl, 0, s>>>(inst, st, ninst, t0, t1); break;
  }
}

void mb_corr(int grid, int minb, cudaStream_t s, const MixBatchInst* inst, const MixBatchStatus* st, int ninst,
             long long t0, long long t1, int step, int nup, int zchunk) {
  if (minb == 3) {
    k_mb_corr<3><<<grid, dim3(32, 8, 1), kCorrSmemBytes, s>>>(inst, st, ninst, t0, t1, step, nup, zchunk);
  } else {
    k_mb_corr<4><<<grid, dim3(32, 8, 1), kCorrSmemBytes, s>>>(inst, st, ninst, t0, t1, step, nup, zchunk);
  }
}

void mb_decide_outer(cudaStream_t s, const MixBatchInst* inst, MixBatchStatus* st, int ninst) {
  k_mb_decide_outer<<<(ninst + 127) / 128, 128, 0, s>>>(inst, st, ninst);
}
void mb_decide_inner(cudaStream_t s, const MixBatchInst* inst, MixBatchStatus* st, int ninst, int nup) {
  k_mb_decide_inner<<<(ninst + 127) / 128, 128, 0, s>>>(inst, st, ninst, nup);
}
void mb_finish(cudaStream_t s, const MixBatchInst* inst, MixBatchStatus* st, int ninst) {
  k_mb_finish<<<(ninst + 127) / 128, 128, 0, s>>>(inst, st, ninst);
}
void mb_start(cudaStream_t s, const MixBatchInst* inst, MixBatchStatus* st, int ninst) {
  k_mb_start<<<(ninst + 127) / 128, 128, 0, s>>>(inst, st, ninst);
}

int mb_points_blocks_per_sm() {
  int n = 0;
  const cudaError_t e =
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_mb_points<MB_PH_PREP>, kMbBX * kMbBY, 0);
  return (e == cudaSuccess && n > 0) ? n : 1;
}

int mb_corr_blocks_per_sm(int minb) {
  int n = 0;
  cudaError_t e;
  if (minb == 3) {
    cudaFuncSetAttribute(k_mb_corr<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, kCorrSmemBytes);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_mb_corr<3>, 256, kCorrSmemBytes);
  } else {
    cudaFuncSetAttribute(k_mb_corr<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, kCorrSmemBytes);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_mb_corr<4>, 256, kCorrSmemBytes);
  }
  return (e == cudaSuccess && n > 0) ? n : 1;
}

int corr_tile_x() { return kCorrTX; }
int corr_tile_y() { return kCorrTY; }

}  // namespace pt
