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
//         that FP32 keeps its relative precision on it (k_corr_cells, k_corr_faces);
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
    // right-hand side and frozen coefficients of the correction problem
    const double idtp = 1.0 / (c.dtaupt_fac * mu);
    const double idtf = kmax / c.dtaupf_fac;
    out.r_pt[q] = (float)divVn;
    out.r_pf[q] = (float)rpf;
    out.cc[q] = (float)cc;
    out.perm[q] = (float)kc;
    out.idtp[q] = (float)idtp;
    out.iden_pt[q] = (float)(1.0 / (idtp + c.beta_d * c.rdt + cc));
    out.idtf[q] = (float)idtf;
    out.iden_pf[q] = (float)(1.0 / (idtf + c.beta_d * c.alpha / c.B * c.rdt + cc));
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

// Frozen mu-dependent coefficients of the correction problem: 2 mu/(1+xi) at centres and
// edges, dtau_V on faces (FP32).
__global__ void __launch_bounds__(256) k_mix_coef(Box b, Coef c, const double* __restrict__ mu, MixCoefOut out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i > b.nx || j > b.ny || k > b.nz) return;
  const long long q = cidx(b, i, j, k);
  const long long px = b.px, pxy = b.pxy;
  const double rG = c.rGdtS;
  // viscoelastic moduli 2 mu / (1 + xi) at centres and edges (mean of the four cells' mu)
  if (i < b.nx && j < b.ny && k < b.nz) {
    const double m = mu[q];
    out.cm2[q] = (float)(2.0 * m / (1.0 + m * rG));
  }
  if (k < b.nz && i > 0 && i < b.nx && j > 0 && j < b.ny) {
    const double m = 0.25 * (mu[q - 1 - px] + mu[q - px] + mu[q - 1] + mu[q]);
    out.em2_xy[q] = (float)(2.0 * m / (1.0 + m * rG));
  }
  if (j < b.ny && i > 0 && i < b.nx && k > 0 && k < b.nz) {
    const double m = 0.25 * (mu[q - 1 - pxy] + mu[q - pxy] + mu[q - 1] + mu[q]);
    out.em2_xz[q] = (float)(2.0 * m / (1.0 + m * rG));
  }
  if (i < b.nx && j > 0 && j < b.ny && k > 0 && k < b.nz) {
    const double m = 0.25 * (mu[q - px - pxy] + mu[q - pxy] + mu[q - px] + mu[q]);
    out.em2_yz[q] = (float)(2.0 * m / (1.0 + m * rG));
  }
  // pseudo-time steps of the velocity correction, mean of the two centres' dtau_V = fac / mu
  if (i > 0 && i < b.nx && j < b.ny && k < b.nz)
    out.dtv_x[q] = (float)(0.5 * c.dtauv_fac * (1.0 / mu[q - 1] + 1.0 / mu[q]));
  if (j > 0 && j < b.ny && i < b.nx && k < b.nz)
    out.dtv_y[q] = (float)(0.5 * c.dtauv_fac * (1.0 / mu[q - px] + 1.0 / mu[q]));
  if (k > 0 && k < b.nz && i < b.nx && j < b.ny)
    out.dtv_z[q] = (float)(0.5 * c.dtauv_fac * (1.0 / mu[q - pxy] + 1.0 / mu[q]));
}

// (iii) one FP32 PT iteration on the correction, cells: edge and centre stresses of dV (no
// old-stress term, it is in r_F), local-implicit dPt and dPf updates of the linearised Eqs.
// 17-18 with right-hand sides r_Pt, r_Pf and frozen coefficients.
template <class T>
__global__ void __launch_bounds__(256) k_corr_cells(Box b, CorrCoef<T> c, CorrIn<T> in,
                                                    CorrCellOut<T> out, unsigned long long* red, int check) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  double r_pt = 0.0, r_pf = 0.0;
  if (i <= b.nx && j <= b.ny && k <= b.nz) {
    const long long q = cidx(b, i, j, k);
    const long long px = b.px, pxy = b.pxy;
    if (k < b.nz) {
      T t = T(0);
      if (i > 0 && i < b.nx && j > 0 && j < b.ny)
        t = in.em2_xy[q] * ((in.Vx[q] - in.Vx[q - px]) * c.hrdy + (in.Vy[q] - in.Vy[q - 1]) * c.hrdx);
      out.txy[q] = t;
    }
    if (j < b.ny) {
      T t = T(0);
      if (i > 0 && i < b.nx && k > 0 && k < b.nz)
        t = in.em2_xz[q] * ((in.Vx[q] - in.Vx[q - pxy]) * c.hrdz + (in.Vz[q] - in.Vz[q - 1]) * c.hrdx);
      out.txz[q] = t;
    }
    if (i < b.nx) {
      T t = T(0);
      if (j > 0 && j < b.ny && k > 0 && k < b.nz)
        t = in.em2_yz[q] * ((in.Vy[q] - in.Vy[q - pxy]) * c.hrdz + (in.Vz[q] - in.Vz[q - px]) * c.hrdy);
      out.tyz[q] = t;
    }
    if (i < b.nx && j < b.ny && k < b.nz) {
      const T dPt = in.Pt[q], dPf = in.Pf[q], cc = in.cc[q];
      const T gx = (in.Vx[q + 1] - in.Vx[q]) * c.rdx, gy = (in.Vy[q + px] - in.Vy[q]) * c.rdy;
      const T gz = (in.Vz[q + pxy] - in.Vz[q]) * c.rdz;
      const T divV = gx + gy + gz;
      const T cpl = c.bd_rdt_a + cc;                 // beta_d alpha / dt + cc
      const T rho_pt = in.r_pt[q] + divV + (c.bd_rdt + cc) * dPt - cpl * dPf;
      const T kc = in.perm[q];
      T sx = T(0), sy = T(0), sz = T(0);
      if (i > 0) sx -= (in.perm[q - 1] + kc) * (dPf - in.Pf[q - 1]);
      if (i < b.nx - 1) sx += (kc + in.perm[q + 1]) * (in.Pf[q + 1] - dPf);
      if (j > 0) sy -= (in.perm[q - px] + kc) * (dPf - in.Pf[q - px]);
      if (j < b.ny - 1) sy += (kc + in.perm[q + px]) * (in.Pf[q + px] - dPf);
      if (k > 0) sz -= (in.perm[q - pxy] + kc) * (dPf - in.Pf[q - pxy]);
      if (k < b.nz - 1) sz += (kc + in.perm[q + pxy]) * (in.Pf[q + pxy] - dPf);
      const T divq = -(sx * c.hrdx2 + sy * c.hrdy2 + sz * c.hrdz2);
      const T rho_pf = in.r_pf[q] + divq + (c.bda_B_rdt + cc) * dPf - cpl * dPt;
      // dP' = dP - dtau rho(dP', ...) solved for dP' (local terms implicit)
      const T dPt1 = (dPt * in.idtp[q] - (in.r_pt[q] + divV - cpl * dPf)) * in.iden_pt[q];
      const T dPf1 = (dPf * in.idtf[q] - (in.r_pf[q] + divq - cpl * dPt)) * in.iden_pf[q];
      out.Pt[q] = dPt1;
      out.Pf[q] = dPf1;
      const T third = divV * T(1.0 / 3.0);
      const T bn = c.beta_n * (rho_pt - in.r_pt[q]);
      const T cm2 = in.cm2[q];
      out.txx[q] = cm2 * (gx - third + bn);
      out.tyy[q] = cm2 * (gy - third + bn);
      out.tzz[q] = cm2 * (gz - third + bn);
      if (check) {
        r_pt = (double)tabs(rho_pt);
        r_pf = (double)tabs(rho_pf);
      }
    }
  }
  if (check) {
    block_max_atomic(r_pt, red + RED_PT);
    block_max_atomic(r_pf, red + RED_PF);
  }
}

// (iii) faces: linearised momentum residual r_F + div tau(dV) - grad dPt', damped R, dV update.
// Reads 19 FP32 arrays and writes 6, all loads before the first store.
template <class T>
__global__ void __launch_bounds__(256) k_corr_faces(Box b, CorrCoef<T> c, CorrFaceIn<T> in,
                                                    T* __restrict__ Vx, T* __restrict__ Vy, T* __restrict__ Vz,
                                                    T* __restrict__ Rx, T* __restrict__ Ry, T* __restrict__ Rz,
                                                    unsigned long long* red, int check) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  double r_v = 0.0;
  if (i <= b.nx && j <= b.ny && k <= b.nz) {
    const long long q = cidx(b, i, j, k);
    const long long px = b.px, pxy = b.pxy;
    const bool fx = i > 0 && i < b.nx && j < b.ny && k < b.nz;
    const bool fy = j > 0 && j < b.ny && i < b.nx && k < b.nz;
    const bool fz = k > 0 && k < b.nz && i < b.nx && j < b.ny;
    T Fx = T(0), Fy = T(0), Fz = T(0), Rx1 = T(0), Ry1 = T(0), Rz1 = T(0), Vx1 = T(0), Vy1 = T(0), Vz1 = T(0);
    if (fx) {
      Fx = in.rfx[q] + (in.txx[q] - in.txx[q - 1]) * c.rdx + (in.txy[q + px] - in.txy[q]) * c.rdy +
           (in.txz[q + pxy] - in.txz[q]) * c.rdz - (in.Pt1[q] - in.Pt1[q - 1]) * c.rdx;
      Rx1 = Fx * c.rrho_i + c.damp_x * Rx[q];
      Vx1 = Vx[q] + in.dtv_x[q] * Rx1;
    }
    if (fy) {
      Fy = in.rfy[q] + (in.txy[q + 1] - in.txy[q]) * c.rdx + (in.tyy[q] - in.tyy[q - px]) * c.rdy +
           (in.tyz[q + pxy] - in.tyz[q]) * c.rdz - (in.Pt1[q] - in.Pt1[q - px]) * c.rdy;
      Ry1 = Fy * c.rrho_i + c.damp_y * Ry[q];
      Vy1 = Vy[q] + in.dtv_y[q] * Ry1;
    }
    if (fz) {
      Fz = in.rfz[q] + (in.txz[q + 1] - in.txz[q]) * c.rdx + (in.tyz[q + px] - in.tyz[q]) * c.rdy +
           (in.tzz[q] - in.tzz[q - pxy]) * c.rdz - (in.Pt1[q] - in.Pt1[q - pxy]) * c.rdz;
      Rz1 = Fz * c.rrho_i + c.damp_z * Rz[q];
      Vz1 = Vz[q] + in.dtv_z[q] * Rz1;
    }
    if (fx) { Rx[q] = Rx1; Vx[q] = Vx1; }
    if (fy) { Ry[q] = Ry1; Vy[q] = Vy1; }
    if (fz) { Rz[q] = Rz1; Vz[q] = Vz1; }
    if (check) r_v = fmax((double)tabs(Fx), fmax((double)tabs(Fy), (double)tabs(Fz)));
  }
  if (check) block_max_atomic(r_v, red + RED_V);
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
template <class T>
void corr_cells(dim3 g, dim3 bl, cudaStream_t s, Box b, const CorrCoef<T>& c, const CorrIn<T>& in,
                const CorrCellOut<T>& out, unsigned long long* red, int check) {
  k_corr_cells<T><<<g, bl, 0, s>>>(b, c, in, out, red, check);
}
template <class T>
void corr_faces(dim3 g, dim3 bl, cudaStream_t s, Box b, const CorrCoef<T>& c, const CorrFaceIn<T>& in, T* Vx,
                T* Vy, T* Vz, T* Rx, T* Ry, T* Rz, unsigned long long* red, int check) {
  k_corr_faces<T><<<g, bl, 0, s>>>(b, c, in, Vx, Vy, Vz, Rx, Ry, Rz, red, check);
}
template void corr_cells<float>(dim3, dim3, cudaStream_t, Box, const CorrCoef<float>&, const CorrIn<float>&,
                                const CorrCellOut<float>&, unsigned long long*, int);
template void corr_faces<float>(dim3, dim3, cudaStream_t, Box, const CorrCoef<float>&, const CorrFaceIn<float>&,
                                float*, float*, float*, float*, float*, float*, unsigned long long*, int);

}  // namespace pt
