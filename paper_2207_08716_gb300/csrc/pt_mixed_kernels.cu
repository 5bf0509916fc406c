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
__global__ void __launch_bounds__(256) k_mix_prepare(Box b, Coef c, MixPrepIn in, MixPrepOut out,
                                                     unsigned long long* red) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  double r_pt = 0.0, r_pf = 0.0;
  if (i < b.nx && j < b.ny && k < b.nz) {
    const long long q = cidx(b, i, j, k);
    const long long px = b.px, pxy = b.pxy;
    const double Pt = in.Pt[q], Pf = in.Pf[q], Pto = in.Pto[q], Pfo = in.Pfo[q];
    const double ph = in.phi[q], mu = in.mu[q];
    const double divV = (in.Vx[q + 1] - in.Vx[q]) * c.rdx + (in.Vy[q + px] - in.Vy[q]) * c.rdy +
                        (in.Vz[q + pxy] - in.Vz[q]) * c.rdz;
    const double cc = c.compaction_on ? 1.0 / (in.eta[q] * (1.0 - ph)) : 0.0;
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
    const double s = 1.0 / (1.0 + xi);
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
    out.idtp[q] = (float)(1.0 / (c.dtaupt_fac * mu));
    r_pt = fabs(divVn);
    r_pf = fabs(rpf);
  }
  block_max_atomic(r_pt, red + RED_PT);
  block_max_atomic(r_pf, red + RED_PF);
}

// (i) FP64 momentum residual at u (Eq. 19), stored in FP32; its max-norm.
__global__ void __launch_bounds__(256) k_mix_res_faces(Box b, Coef c, MixFaceIn in, float* __restrict__ rfx,
                                                       float* __restrict__ rfy, float* __restrict__ rfz,
                                                       unsigned long long* red) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  double r_v = 0.0;
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
  block_max_atomic(r_v, red + RED_V);
}

// Frozen mu-dependent coefficients of the correction problem: mu and the velocity pseudo-step
// dtau_V = fac / mu at centres, in FP32 (the iteration forms 2 mu/(1+xi) at centres and edges and
// the face pseudo-steps from them).
__global__ void __launch_bounds__(256) k_mix_coef(Box b, Coef c, const double* __restrict__ mu, MixCoefOut out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i < b.nx && j < b.ny && k < b.nz) {
    const long long q = cidx(b, i, j, k);
    out.mu[q] = (float)mu[q];
    out.dtvc[q] = (float)(c.dtauv_fac / mu[q]);
  }
}

// (iii) one FP32 PT iteration on the correction in a single pass.
//
// The iteration's two halves depend on each other across neighbours: the faces (momentum,
// damped R, dV) of level k read the cells' stresses and new dPt at k and k-1 (own cell, x- and
// y-neighbours below) and the edge stresses at k and k+1 (own edge, x- and y-neighbours above).
// A 32 x 8 block owns a tile of 30 x 6 faces and cells and marches up a column of kCorrZChunk
// levels: at level L every thread computes the cell and the three lower edges at its index for
// the tile plus a one-cell halo on each side (the halo is recomputed by the neighbouring tiles'
// blocks from the same inputs, bit for bit), into a three-level ring in shared memory; after a
// barrier the tile's threads compute the faces of level L-1 from the ring. Stresses and the new
// dPt never go to global memory: per cell the pass reads dV, dPt, dPf, R, the right-hand sides
// and the frozen cc, k, 1/dtau_Pt, mu, dtau_V (18 arrays) and writes dV', dPt', dPf', R (8 arrays):
// 104 B per cell against 200 B for a cells kernel plus a faces kernel. dV is read from one buffer
// and written to another (other blocks' halos still read the old dV). The pseudo-step of dPf
// (largest neighbour k), the local-implicit denominators, 2 mu/(1+xi) at centres and edges (mean
// of the four centres' mu) and the face pseudo-steps (mean of the two centres') are formed here.
constexpr int kCorrTX = 30, kCorrTY = 6, kCorrZChunk = 64;
// The 11 arrays the cell phase reads at its own index are copied into a shared-memory stage by
// cp.async ahead of their level; the cell phase reads its own values and its x- and y-neighbours
// inside the block's region from the stage.
enum { C_VX, C_VY, C_VZ, C_PT, C_PF, C_CC, C_K, C_IDTP, C_RPT, C_RPF, C_MU, kCorrStage };
// Stage depth: 2 = the next level's copies in flight while this level computes; 3 = two levels
// ahead, and the z+1 values read from the stage too. Blocks per SM asked of the register allocator.
constexpr int kCorrStages = 2, kCorrMinBlocks = 4;
// rings of three levels for cells (4 values) and edges (3), kCorrStages for the staged inputs
constexpr int kCorrSmemBytes = (3 * (4 + 3) + kCorrStages * kCorrStage) * 8 * 32 * (int)sizeof(float);

__device__ __forceinline__ void corr_cp4(float* smem, const float* gmem) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gmem) : "memory");
}

__device__ __forceinline__ float corr_modulus(const CorrCoef<float>& c, float m) {
  return __fdividef(2.0f * m, 1.0f + m * c.rG);
}

__global__ void __launch_bounds__(256, kCorrMinBlocks) k_corr_iteration(Box b, CorrCoef<float> c, CorrIn<float> in,
                                                        CorrOut<float> out, unsigned long long* red, int check) {
  using T = float;
  // ring of three levels: cells (txx, tyy, tzz, dPt') and edges (txy, txz, tyz) of the region
  extern __shared__ __align__(16) float corr_smem[];   // kCorrSmemBytes, dynamic (above 48 KB)
  T(*s_cell)[4][8][32] = reinterpret_cast<T(*)[4][8][32]>(corr_smem);
  T(*s_edge)[3][8][32] = reinterpret_cast<T(*)[3][8][32]>(corr_smem + 3 * 4 * 8 * 32);
  T(*s_in)[kCorrStage][8][32] = reinterpret_cast<T(*)[kCorrStage][8][32]>(corr_smem + 3 * 7 * 8 * 32);
  (void)kCorrSmemBytes;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int i = blockIdx.x * kCorrTX - 1 + tx;
  const int j = blockIdx.y * kCorrTY - 1 + ty;
  const int k0 = blockIdx.z * kCorrZChunk;
  const int k1 = min(k0 + kCorrZChunk, b.nz + 1);       // face levels [k0, k1) of this block
  const bool own = tx >= 1 && tx <= kCorrTX && ty >= 1 && ty <= kCorrTY;
  const int ipx = b.px, ipxy = (int)b.pxy;   // the host keeps the box below 2^31 elements
  // residual norms as bit patterns of non-negative doubles: a NaN (largest pattern) stays in them
  unsigned long long r_pt = 0ull, r_pf = 0ull, r_v = 0ull;
  auto keep_max = [](unsigned long long& m, float x) {
    const unsigned long long u = (unsigned long long)__double_as_longlong((double)fabsf(x));
    m = u > m ? u : m;
  };
  const bool in_box = i >= 0 && j >= 0 && i <= b.nx && j <= b.ny;
  auto stage = [&](int L) {   // own-index values of level L (inside the box) into stage L mod 3
    if (in_box && L >= 0 && L <= b.nz) {
      const int q = i + ipx * j + ipxy * L;
      float(*st)[8][32] = s_in[(L + kCorrStages) % kCorrStages];
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
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  for (int d = 0; d < kCorrStages - 1; ++d) stage(k0 - 1 + d);
  for (int L = k0 - 1; L <= k1; ++L) {
    const int sl = (L + 3) % 3;
    stage(L + kCorrStages - 1);                        // the level kCorrStages - 1 ahead goes out now
    asm volatile("cp.async.wait_group 1;\n" ::: "memory");   // this thread's copies up to level L landed
    // every thread's staged copies are visible (the cell phase reads neighbours' staged values),
    // and the previous level's faces are done with the ring slot this level overwrites
    __syncthreads();
    const float(*S)[8][32] = s_in[(L + kCorrStages) % kCorrStages];
    const float(*Su)[8][32] = s_in[(L + 1 + kCorrStages) % kCorrStages];   // level L + 1 (3 stages)
    // the faces of level L - 1 read these after the cell phase: their loads go out first
    const int F = L - 1;
    const bool face_here = own && F >= k0 && F < k1 && in_box && F <= b.nz;
    T rfx = T(0), rfy = T(0), rfz = T(0), Rx0 = T(0), Ry0 = T(0), Rz0 = T(0), Vx0 = T(0), Vy0 = T(0), Vz0 = T(0);
    T dtx = T(0), dty = T(0), dtz = T(0);
    const bool fx = face_here && i > 0 && i < b.nx && j < b.ny && F < b.nz;
    const bool fy = face_here && j > 0 && j < b.ny && i < b.nx && F < b.nz;
    const bool fz = face_here && F > 0 && F < b.nz && i < b.nx && j < b.ny;
    if (face_here) {
      const int q = i + ipx * j + ipxy * F;
      if (fx) { rfx = in.rfx[q]; Rx0 = out.Rx[q]; Vx0 = in.Vx[q]; dtx = T(0.5) * (in.dtvc[q - 1] + in.dtvc[q]); }
      if (fy) { rfy = in.rfy[q]; Ry0 = out.Ry[q]; Vy0 = in.Vy[q]; dty = T(0.5) * (in.dtvc[q - ipx] + in.dtvc[q]); }
      if (fz) { rfz = in.rfz[q]; Rz0 = out.Rz[q]; Vz0 = in.Vz[q]; dtz = T(0.5) * (in.dtvc[q - ipxy] + in.dtvc[q]); }
    }
    // ---------------- cell and lower edges at (i, j, L). Cells are needed for the tile and its
    // left / lower halo (tx <= 30, ty <= 6), edges for the tile and its right / upper halo
    // (tx >= 1, ty >= 1). Indices are 32-bit (the host keeps the box below 2^31 elements);
    // x- and y-neighbours inside the block's region come from this level's stage.
    T txx = T(0), tyy = T(0), tzz = T(0), P1 = T(0), exy = T(0), exz = T(0), eyz = T(0);
    if (in_box && L >= 0 && L <= b.nz) {
      const int q = i + ipx * j + ipxy * L;
      auto nb = [&](int slot, int dx, int dy, const float* g, int off) -> float {
        const int x = tx + dx, y = ty + dy;
        return (x >= 0 && x < 32 && y >= 0 && y < 8) ? S[slot][y][x] : g[q + off];
      };
      const T mu_c = S[C_MU][ty][tx], vx_c = S[C_VX][ty][tx], vy_c = S[C_VY][ty][tx], vz_c = S[C_VZ][ty][tx];
      if (tx >= 1 && ty >= 1) {
        if (L < b.nz && i > 0 && i < b.nx && j > 0 && j < b.ny) {
          const T m = T(0.25) * (nb(C_MU, -1, -1, in.mu, -1 - ipx) + nb(C_MU, 0, -1, in.mu, -ipx) +
                                 nb(C_MU, -1, 0, in.mu, -1) + mu_c);
          exy = corr_modulus(c, m) * ((vx_c - nb(C_VX, 0, -1, in.Vx, -ipx)) * c.hrdy +
                                      (vy_c - nb(C_VY, -1, 0, in.Vy, -1)) * c.hrdx);
        }
        if (j < b.ny && i > 0 && i < b.nx && L > 0 && L < b.nz) {
          const T m = T(0.25) * (in.mu[q - 1 - ipxy] + in.mu[q - ipxy] + nb(C_MU, -1, 0, in.mu, -1) + mu_c);
          exz = corr_modulus(c, m) * ((vx_c - in.Vx[q - ipxy]) * c.hrdz + (vz_c - nb(C_VZ, -1, 0, in.Vz, -1)) * c.hrdx);
        }
        if (i < b.nx && j > 0 && j < b.ny && L > 0 && L < b.nz) {
          const T m = T(0.25) * (in.mu[q - ipx - ipxy] + in.mu[q - ipxy] + nb(C_MU, 0, -1, in.mu, -ipx) + mu_c);
          eyz = corr_modulus(c, m) * ((vy_c - in.Vy[q - ipxy]) * c.hrdz + (vz_c - nb(C_VZ, 0, -1, in.Vz, -ipx)) * c.hrdy);
        }
      }
      if (tx <= kCorrTX && ty <= kCorrTY && i < b.nx && j < b.ny && L < b.nz) {
        const T dPt = S[C_PT][ty][tx], dPf = S[C_PF][ty][tx], cc = S[C_CC][ty][tx];
        const T rpt = S[C_RPT][ty][tx], rpf = S[C_RPF][ty][tx];
        const T gx = (nb(C_VX, 1, 0, in.Vx, 1) - vx_c) * c.rdx, gy = (nb(C_VY, 0, 1, in.Vy, ipx) - vy_c) * c.rdy;
        const T gz = (((kCorrStages > 2) ? Su[C_VZ][ty][tx] : in.Vz[q + ipxy]) - vz_c) * c.rdz;
        const T divV = gx + gy + gz;
        const T cpl = c.bd_rdt_a + cc;                 // beta_d alpha / dt + cc
        const T rho_pt = rpt + divV + (c.bd_rdt + cc) * dPt - cpl * dPf;
        const T kc = S[C_K][ty][tx];
        T kmax = kc, sx = T(0), sy = T(0), sz = T(0);
        if (i > 0) {
          const T kn = nb(C_K, -1, 0, in.perm, -1);
          kmax = fmaxf(kmax, kn);
          sx -= (kn + kc) * (dPf - nb(C_PF, -1, 0, in.Pf, -1));
        }
        if (i < b.nx - 1) {
          const T kn = nb(C_K, 1, 0, in.perm, 1);
          kmax = fmaxf(kmax, kn);
          sx += (kc + kn) * (nb(C_PF, 1, 0, in.Pf, 1) - dPf);
        }
        if (j > 0) {
          const T kn = nb(C_K, 0, -1, in.perm, -ipx);
          kmax = fmaxf(kmax, kn);
          sy -= (kn + kc) * (dPf - nb(C_PF, 0, -1, in.Pf, -ipx));
        }
        if (j < b.ny - 1) {
          const T kn = nb(C_K, 0, 1, in.perm, ipx);
          kmax = fmaxf(kmax, kn);
          sy += (kc + kn) * (nb(C_PF, 0, 1, in.Pf, ipx) - dPf);
        }
        if (L > 0) {
          const T kn = in.perm[q - ipxy];
          kmax = fmaxf(kmax, kn);
          sz -= (kn + kc) * (dPf - in.Pf[q - ipxy]);
        }
        if (L < b.nz - 1) {
          const T kn = (kCorrStages > 2) ? Su[C_K][ty][tx] : in.perm[q + ipxy];
          kmax = fmaxf(kmax, kn);
          sz += (kc + kn) * (((kCorrStages > 2) ? Su[C_PF][ty][tx] : in.Pf[q + ipxy]) - dPf);
        }
        const T divq = -(sx * c.hrdx2 + sy * c.hrdy2 + sz * c.hrdz2);
        const T rho_pf = rpf + divq + (c.bda_B_rdt + cc) * dPf - cpl * dPt;
        // dP' = dP - dtau rho(dP', ...) solved for dP' (local terms implicit; the quotients only
        // scale the pseudo-step, so the fast reciprocal does)
        const T idtp = S[C_IDTP][ty][tx], idtf = kmax * c.ifac_pf;
        const T dPt1 = __fdividef(dPt * idtp - (rpt + divV - cpl * dPf), idtp + c.bd_rdt + cc);
        const T dPf1 = __fdividef(dPf * idtf - (rpf + divq - cpl * dPt), idtf + c.bda_B_rdt + cc);
        const T third = divV * T(1.0 / 3.0);
        const T bn = c.beta_n * (rho_pt - rpt);
        const T cm2 = corr_modulus(c, mu_c);
        txx = cm2 * (gx - third + bn);
        tyy = cm2 * (gy - third + bn);
        tzz = cm2 * (gz - third + bn);
        P1 = dPt1;
        if (own && L >= k0 && L < k1) {
          out.Pt[q] = dPt1;
          out.Pf[q] = dPf1;
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
    s_edge[sl][0][ty][tx] = exy;
    s_edge[sl][1][ty][tx] = exz;
    s_edge[sl][2][ty][tx] = eyz;
    __syncthreads();
    // ---------------- faces of level F = L - 1 (cells at F and F-1, edges at F and L = F+1)
    if (face_here) {
      const int sf = (F + 3) % 3, sb = (F + 2) % 3, su = sl;
      const int q = i + ipx * j + ipxy * F;
      const T Pc = s_cell[sf][3][ty][tx];
      T Fx = T(0), Fy = T(0), Fz = T(0);
      if (fx) {
        Fx = rfx + (s_cell[sf][0][ty][tx] - s_cell[sf][0][ty][tx - 1]) * c.rdx +
             (s_edge[sf][0][ty + 1][tx] - s_edge[sf][0][ty][tx]) * c.rdy +
             (s_edge[su][1][ty][tx] - s_edge[sf][1][ty][tx]) * c.rdz - (Pc - s_cell[sf][3][ty][tx - 1]) * c.rdx;
        const T R1 = Fx * c.rrho_i + c.damp_x * Rx0;
        out.Rx[q] = R1;
        out.Vx[q] = Vx0 + dtx * R1;
      }
      if (fy) {
        Fy = rfy + (s_edge[sf][0][ty][tx + 1] - s_edge[sf][0][ty][tx]) * c.rdx +
             (s_cell[sf][1][ty][tx] - s_cell[sf][1][ty - 1][tx]) * c.rdy +
             (s_edge[su][2][ty][tx] - s_edge[sf][2][ty][tx]) * c.rdz - (Pc - s_cell[sf][3][ty - 1][tx]) * c.rdy;
        const T R1 = Fy * c.rrho_i + c.damp_y * Ry0;
        out.Ry[q] = R1;
        out.Vy[q] = Vy0 + dty * R1;
      }
      if (fz) {
        Fz = rfz + (s_edge[sf][1][ty][tx + 1] - s_edge[sf][1][ty][tx]) * c.rdx +
             (s_edge[sf][2][ty + 1][tx] - s_edge[sf][2][ty][tx]) * c.rdy +
             (s_cell[sf][2][ty][tx] - s_cell[sb][2][ty][tx]) * c.rdz - (Pc - s_cell[sb][3][ty][tx]) * c.rdz;
        const T R1 = Fz * c.rrho_i + c.damp_z * Rz0;
        out.Rz[q] = R1;
        out.Vz[q] = Vz0 + dtz * R1;
      }
      if (check) {
        keep_max(r_v, Fx);
        keep_max(r_v, Fy);
        keep_max(r_v, Fz);
      }
    }
  }
  if (check) {
    block_max_atomic(__longlong_as_double((long long)r_pt), red + RED_PT);
    block_max_atomic(__longlong_as_double((long long)r_pf), red + RED_PF);
    block_max_atomic(__longlong_as_double((long long)r_v), red + RED_V);
  }
}

// (iv) u <- u + delta (FP64 += FP32 correction).
__global__ void __launch_bounds__(256) k_mix_update(Box b, MixUpdate u) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
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

void mix_prepare(dim3 g, dim3 bl, cudaStream_t s, Box b, const Coef& c, const MixPrepIn& in,
                 const MixPrepOut& out, unsigned long long* red) {
  k_mix_prepare<<<g, bl, 0, s>>>(b, c, in, out, red);
}
void mix_res_faces(dim3 g, dim3 bl, cudaStream_t s, Box b, const Coef& c, const MixFaceIn& in, float* rfx,
                   float* rfy, float* rfz, unsigned long long* red) {
  k_mix_res_faces<<<g, bl, 0, s>>>(b, c, in, rfx, rfy, rfz, red);
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

}  // namespace pt
