// pt_ref_kernels.cu — the step-by-step ("reference") GPU form of one PT iteration: one kernel
// per data-flow step, intermediates in global memory, one thread per box index (i, j, k).
//
// Data flow of one iteration k -> k+1 (thesis Art. 1, Eqs. 17-27; staggered grid of Fig. 1):
//   k_perm      k = k0 e^logk (phi/phi0)^3 (Eq. 23), rho g - rho_BG g (Eq. 27)   from phi^k
//   k_centres   div V, numerical div V (Eq. 17), Pt^{k+1}, Pf^{k+1} local-implicit (Eqs. 17-18
//               with div qD from Eq. 20), normal deviatoric stresses (Eq. 21)
//   k_edges     shear stresses on edges (Eq. 21), zero on boundary edges (free slip) unless a
//               background shear stress is applied (Eqs. 32-33)
//   k_porosity  phi^{k+1} = 1 - exp(L), L from Eq. 22 in log(1 - phi) form
//   k_faces     momentum residual (Eq. 19) with Pt^{k+1}, damped R, V^{k+1} = V + dtau R
//   k_picard    every nup-th iteration: mu, eta towards Eqs. 24-26, log-space relaxation
// Residual max-norms are reduced into a small device block on check iterations.
#include "pt_ref_points.cuh"

namespace pt {

__device__ inline bool in_cells(const Box& b, int i, int j, int k) {
  return i < b.nx && j < b.ny && k < b.nz;
}

__device__ inline void thread_ijk(int& i, int& j, int& k) {
  i = blockIdx.x * blockDim.x + threadIdx.x;
  j = blockIdx.y * blockDim.y + threadIdx.y;
  k = blockIdx.z;
}

__global__ void k_perm(Box b, Coef c, const double* __restrict__ phi,
                       const double* __restrict__ logk, double* __restrict__ perm,
                       double* __restrict__ rog) {
  int i, j, k;
  thread_ijk(i, j, k);
  perm_point(b, c, phi, logk, perm, rog, i, j, k);
}


// update = 0: stresses only (end of step, residual evaluation); update = 1: also the pressures.
__global__ void k_centres(Box b, Coef c, CentreIn in, CentreOut out, int update,
                          unsigned long long* red, int check) {
  int i, j, k;
  thread_ijk(i, j, k);
  double r_pt = 0.0, r_pf = 0.0;
  if (in_cells(b, i, j, k)) {
    const long long q = cidx(b, i, j, k);
    const double Pt = in.Pt[q], Pf = in.Pf[q], Pto = in.Pto[q], Pfo = in.Pfo[q];
    const double ph = in.phi[q], mu = in.mu[q];
    const double divV = (in.Vx[q + 1] - in.Vx[q]) * c.rdx + (in.Vy[q + b.px] - in.Vy[q]) * c.rdy +
                        (in.Vz[q + b.pxy] - in.Vz[q]) * c.rdz;
    const double cc = c.compaction_on ? 1.0 / (in.eta[q] * (1.0 - ph)) : 0.0;
    const double divVn = divV + c.beta_d * ((Pt - Pto) - c.alpha * (Pf - Pfo)) * c.rdt + (Pt - Pf) * cc;
    if (update) {
      // Darcy flux on the 6 faces (zero normal flux on the boundary), its divergence, and the
      // largest permeability of the cell and its existing neighbours.
      const double kc = in.perm[q];
      const double buoy = c.rhof_g - c.rho_bg_g;
      double kmax = kc, qxl = 0.0, qxr = 0.0, qyl = 0.0, qyr = 0.0, qzl = 0.0, qzr = 0.0;
      if (i > 0) {
        const double kn = in.perm[q - 1];
        kmax = fmax(kmax, kn);
        qxl = -0.5 * (kn + kc) * (Pf - in.Pf[q - 1]) * c.rdx;
      }
      if (i < b.nx - 1) {
        const double kn = in.perm[q + 1];
        kmax = fmax(kmax, kn);
        qxr = -0.5 * (kc + kn) * (in.Pf[q + 1] - Pf) * c.rdx;
      }
      if (j > 0) {
        const double kn = in.perm[q - b.px];
        kmax = fmax(kmax, kn);
        qyl = -0.5 * (kn + kc) * (Pf - in.Pf[q - b.px]) * c.rdy;
      }
      if (j < b.ny - 1) {
        const double kn = in.perm[q + b.px];
        kmax = fmax(kmax, kn);
        qyr = -0.5 * (kc + kn) * (in.Pf[q + b.px] - Pf) * c.rdy;
      }
      if (k > 0) {
        const double kn = in.perm[q - b.pxy];
        kmax = fmax(kmax, kn);
        qzl = -0.5 * (kn + kc) * ((Pf - in.Pf[q - b.pxy]) * c.rdz + buoy);
      }
      if (k < b.nz - 1) {
        const double kn = in.perm[q + b.pxy];
        kmax = fmax(kmax, kn);
        qzr = -0.5 * (kc + kn) * ((in.Pf[q + b.pxy] - Pf) * c.rdz + buoy);
      }
      const double divqD = (qxr - qxl) * c.rdx + (qyr - qyl) * c.rdy + (qzr - qzl) * c.rdz;
      const double dtau_pt = c.dtaupt_fac * mu;
      const double dtau_pf = c.dtaupf_fac / kmax;
      out.Pt1[q] = (Pt - dtau_pt * (divV + c.beta_d * (-Pto - c.alpha * (Pf - Pfo)) * c.rdt - cc * Pf)) /
                   (1.0 + dtau_pt * (c.beta_d * c.rdt + cc));
      out.Pf1[q] = (Pf - dtau_pf * (divqD + c.beta_d * (-(c.alpha / c.B) * Pfo - c.alpha * (Pt - Pto)) * c.rdt -
                                    cc * Pt)) /
                   (1.0 + dtau_pf * (c.beta_d * c.alpha / c.B * c.rdt + cc));
      if (check) {
        r_pt = fabs(divVn);
        r_pf = fabs(divqD + c.beta_d * c.alpha * ((Pf - Pfo) / c.B - (Pt - Pto)) * c.rdt + (Pf - Pt) * cc);
      }
    }
    // normal deviatoric stresses, Maxwell backward Euler with xi = mu / (G dtS)
    const double xi = mu * c.rGdtS;
    const double s = 1.0 / (1.0 + xi);
    const double bn = c.beta_n * divVn;
    const double exx = (in.Vx[q + 1] - in.Vx[q]) * c.rdx - divV / 3.0;
    const double eyy = (in.Vy[q + b.px] - in.Vy[q]) * c.rdy - divV / 3.0;
    const double ezz = (in.Vz[q + b.pxy] - in.Vz[q]) * c.rdz - divV / 3.0;
    out.txx[q] = (in.txxo[q] * xi + 2.0 * mu * (exx + bn)) * s;
    out.tyy[q] = (in.tyyo[q] * xi + 2.0 * mu * (eyy + bn)) * s;
    out.tzz[q] = (in.tzzo[q] * xi + 2.0 * mu * (ezz + bn)) * s;
  }
  if (check) {
    block_max_atomic(r_pt, red + RED_PT);
    block_max_atomic(r_pf, red + RED_PF);
  }
}


__global__ void k_edges(Box b, Coef c, EdgeIn in, EdgeOut out) {
  int i, j, k;
  thread_ijk(i, j, k);
  edges_point(b, c, in, out, i, j, k);
}

// phi^{k+1} from Eq. 22 (porosity_point)
__global__ void k_porosity(Box b, Coef c, const double* __restrict__ Vx, const double* __restrict__ Vy,
                           const double* __restrict__ Vz, const double* __restrict__ phi,
                           const double* __restrict__ Pt1, const double* __restrict__ Pf1,
                           const double* __restrict__ Pto, const double* __restrict__ Pfo,
                           const double* __restrict__ Lo, const double* __restrict__ eta,
                           double* __restrict__ phi1) {
  int i, j, k;
  thread_ijk(i, j, k);
  porosity_point(b, c, Vx, Vy, Vz, phi, Pt1, Pf1, Pto, Pfo, Lo, eta, phi1, i, j, k);
}


__device__ inline double dtau_v(const Coef& c, double mu) { return c.dtauv_fac / mu; }

__global__ void k_faces(Box b, Coef c, FaceIn in, double* __restrict__ Vx, double* __restrict__ Vy,
                        double* __restrict__ Vz, double* __restrict__ Rx, double* __restrict__ Ry,
                        double* __restrict__ Rz, unsigned long long* red, int check) {
  int i, j, k;
  thread_ijk(i, j, k);
  double r_v = 0.0;
  if (i <= b.nx && j <= b.ny && k <= b.nz) {
    const long long q = cidx(b, i, j, k);
    const long long px = b.px, pxy = b.pxy;
    if (i > 0 && i < b.nx && j < b.ny && k < b.nz) {  // interior x-face
      const double F = (in.txx[q] - in.txx[q - 1]) * c.rdx + (in.txy[q + px] - in.txy[q]) * c.rdy +
                       (in.txz[q + pxy] - in.txz[q]) * c.rdz - (in.Pt1[q] - in.Pt1[q - 1]) * c.rdx;
      const double R = F * c.rrho_i + c.damp_x * Rx[q];
      Rx[q] = R;
      Vx[q] += 0.5 * (dtau_v(c, in.mu[q - 1]) + dtau_v(c, in.mu[q])) * R;
      r_v = fmax(r_v, fabs(F));
    }
    if (j > 0 && j < b.ny && i < b.nx && k < b.nz) {  // interior y-face
      const double F = (in.txy[q + 1] - in.txy[q]) * c.rdx + (in.tyy[q] - in.tyy[q - px]) * c.rdy +
                       (in.tyz[q + pxy] - in.tyz[q]) * c.rdz - (in.Pt1[q] - in.Pt1[q - px]) * c.rdy;
      const double R = F * c.rrho_i + c.damp_y * Ry[q];
      Ry[q] = R;
      Vy[q] += 0.5 * (dtau_v(c, in.mu[q - px]) + dtau_v(c, in.mu[q])) * R;
      r_v = fmax(r_v, fabs(F));
    }
    if (k > 0 && k < b.nz && i < b.nx && j < b.ny) {  // interior z-face
      const double F = (in.txz[q + 1] - in.txz[q]) * c.rdx + (in.tyz[q + px] - in.tyz[q]) * c.rdy +
                       (in.tzz[q] - in.tzz[q - pxy]) * c.rdz - (in.Pt1[q] - in.Pt1[q - pxy]) * c.rdz -
                       0.5 * (in.rog[q - pxy] + in.rog[q]);
      const double R = F * c.rrho_i + c.damp_z * Rz[q];
      Rz[q] = R;
      Vz[q] += 0.5 * (dtau_v(c, in.mu[q - pxy]) + dtau_v(c, in.mu[q])) * R;
      r_v = fmax(r_v, fabs(F));
    }
  }
  if (check) block_max_atomic(r_v, red + RED_V);
}


// Picard targets mu* = mu0 / (1 + (tau_II / tau0)^(n-1)) (Eq. 24) and
// eta* = eta0 mu / phi R (Eqs. 25-26, R = R_weak where Pf > Pt); log-space relaxation.
// update = 0: residual only (eta* from the current mu, nothing written).
__global__ void k_picard(Box b, Coef c, PicardIn in, double* __restrict__ mu, double* __restrict__ eta,
                         unsigned long long* red, int update) {
  int i, j, k;
  thread_ijk(i, j, k);
  double r = 0.0;
  if (in_cells(b, i, j, k)) {
    const long long q = cidx(b, i, j, k);
    const long long px = b.px, pxy = b.pxy;
    const double axy = 0.25 * (in.txy[q] + in.txy[q + 1] + in.txy[q + px] + in.txy[q + 1 + px]);
    const double axz = 0.25 * (in.txz[q] + in.txz[q + 1] + in.txz[q + pxy] + in.txz[q + 1 + pxy]);
    const double ayz = 0.25 * (in.tyz[q] + in.tyz[q + px] + in.tyz[q + pxy] + in.tyz[q + px + pxy]);
    const double sxx = in.txx[q], syy = in.tyy[q], szz = in.tzz[q];
    const double tII = sqrt(0.5 * (sxx * sxx + syy * syy + szz * szz) + axy * axy + axz * axz + ayz * ayz);
    const double mus = c.powerlaw_on ? c.mu0 / (1.0 + pow(tII / c.tau0, c.n_pow - 1.0)) : c.mu0;
    const double mu_old = mu[q], eta_old = eta[q];
    const double mu_new = update ? exp(c.rel_mu * log(mus) + (1.0 - c.rel_mu) * log(mu_old)) : mu_old;
    const double R = (in.Pf1[q] > in.Pt1[q]) ? c.R_weak : 1.0;
    const double etas = c.eta0 * mu_new / in.phi1[q] * R;
    r = fmax(fabs(log(mus) - log(mu_old)), fabs(log(etas) - log(eta_old)));
    if (update) {
      mu[q] = mu_new;
      eta[q] = exp(c.rel_eta * log(etas) + (1.0 - c.rel_eta) * log(eta_old));
    }
  }
  block_max_atomic(r, red + RED_PIC);
}

// Start of a physical step: Pto = Pt, Pfo = Pf, Lo = log(1 - phi), max(mu) for dtS.
__global__ void k_begin_step(Box b, const double* __restrict__ Pt, const double* __restrict__ Pf,
                             const double* __restrict__ phi, const double* __restrict__ mu,
                             double* __restrict__ Pto, double* __restrict__ Pfo, double* __restrict__ Lo,
                             unsigned long long* red) {
  int i, j, k;
  thread_ijk(i, j, k);
  double m = 0.0;
  if (in_cells(b, i, j, k)) {
    const long long q = cidx(b, i, j, k);
    Pto[q] = Pt[q];
    Pfo[q] = Pf[q];
    Lo[q] = log(1.0 - phi[q]);
    m = mu[q];
  }
  block_max_atomic(m, red + RED_MUMAX);
}

__global__ void k_init_visc(Box b, Coef c, const double* __restrict__ phi, double* __restrict__ mu,
                            double* __restrict__ eta) {
  int i, j, k;
  thread_ijk(i, j, k);
  if (!in_cells(b, i, j, k)) return;
  const long long q = cidx(b, i, j, k);
  mu[q] = c.mu0;
  eta[q] = c.eta0 * c.mu0 / phi[q];
}

// System residual of the current state (no update): momentum max-norm with the current Pt.
__global__ void k_residual_faces(Box b, Coef c, FaceIn in, unsigned long long* red) {
  int i, j, k;
  thread_ijk(i, j, k);
  double r_v = 0.0;
  if (i <= b.nx && j <= b.ny && k <= b.nz) {
    const long long q = cidx(b, i, j, k);
    const long long px = b.px, pxy = b.pxy;
    if (i > 0 && i < b.nx && j < b.ny && k < b.nz)
      r_v = fmax(r_v, fabs((in.txx[q] - in.txx[q - 1]) * c.rdx + (in.txy[q + px] - in.txy[q]) * c.rdy +
                           (in.txz[q + pxy] - in.txz[q]) * c.rdz - (in.Pt1[q] - in.Pt1[q - 1]) * c.rdx));
    if (j > 0 && j < b.ny && i < b.nx && k < b.nz)
      r_v = fmax(r_v, fabs((in.txy[q + 1] - in.txy[q]) * c.rdx + (in.tyy[q] - in.tyy[q - px]) * c.rdy +
                           (in.tyz[q + pxy] - in.tyz[q]) * c.rdz - (in.Pt1[q] - in.Pt1[q - px]) * c.rdy));
    if (k > 0 && k < b.nz && i < b.nx && j < b.ny)
      r_v = fmax(r_v, fabs((in.txz[q + 1] - in.txz[q]) * c.rdx + (in.tyz[q + px] - in.tyz[q]) * c.rdy +
                           (in.tzz[q] - in.tzz[q - pxy]) * c.rdz - (in.Pt1[q] - in.Pt1[q - pxy]) * c.rdz -
                           0.5 * (in.rog[q - pxy] + in.rog[q])));
  }
  block_max_atomic(r_v, red + RED_V);
}

}  // namespace pt
