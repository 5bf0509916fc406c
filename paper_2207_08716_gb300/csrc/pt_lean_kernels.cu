// pt_lean_kernels.cu — the FP64-lean form of one PT iteration (two kernels per iteration).
//
// GB300 issues 2 FP64 lanes per SM per clock (~1.26 TFLOP/s) against ~6.7 TB/s of HBM, so an
// FP64 PT iteration is bound by FP64 instructions, not bytes. This form therefore trades bytes
// for FP64 work wherever a quantity changes less often than every iteration:
//   * coefficients that depend only on mu, eta and the old stresses (which change at Picard
//     updates and step starts) are kept in arrays refreshed by k_lean_coef:
//       centres  cm2 = 2 mu / (1 + xi), toa_ii = tau_o_ii xi / (1 + xi), idtp = 1 / dtau_Pt,
//                ieta = 1 / eta
//       edges    em2 = 2 mu_e / (1 + xi_e), toa_e = tau_o_e xi_e / (1 + xi_e)
//       faces    dtv = dtau_V (mean of the two centres' values)
//     with xi = mu / (G dtS) (Eq. 21, backward-Euler Maxwell step);
//   * k = k0 e^logk (phi / phi0)^3 (Eq. 23) and w = 1 / (1 - phi) travel with phi: the
//     porosity update of iteration k writes them for iteration k+1;
//   * the log-space porosity update (Eq. 22) is L = Lo + delta, so
//       phi'  = phi_o - (1 - phi_o) expm1(delta),   1 / (1 - phi') = (1 / (1 - phi_o)) e^-delta,
//     with both exponentials from one Taylor polynomial of exp (|delta| is tiny; large |delta|
//     falls back to CUDA's expm1) — no exp, no division, no cancellation in 1 - e^L;
//   * the largest neighbour permeability (pseudo-time step of Pf) is found with 64-bit
//     integer compares of the positive doubles' bit patterns (exact, off the FP64 pipe).
// k_lean_cells: Darcy flux and divergence (Eq. 20), div V and numerical div V (Eq. 17),
// local-implicit Pt, Pf (Eqs. 17-18), stresses at centres and the cell's three lower edges
// (Eq. 21), porosity (Eq. 22). k_lean_faces: momentum residual (Eq. 19) with Pt^{k+1},
// damped R, V^{k+1}. k_lean_picard: Picard targets (Eqs. 24-26) with log-space relaxation.
#include "pt_lean.cuh"

namespace pt {

namespace {

// exp(d) - 1 and exp(-d) - 1 from the Taylor series of exp split into its odd part
// O = d + d^3/3! + ... and even part E = d^2/2! + d^4/4! + ... (both truncated after d^9 /
// d^8: for |d| <= 2^-6 the first dropped term is below 2^-60 |d|). expm1(d) = E + O,
// expm1(-d) = E - O.
__device__ inline void expm1_pair(double d, double& em_pos, double& em_neg) {
  if (fabs(d) <= 0.015625) {
    const double d2 = d * d;
    const double E = d2 * fma(d2, fma(d2, fma(d2, 1.0 / 40320.0, 1.0 / 720.0), 1.0 / 24.0), 0.5);
    const double O = d * fma(d2, fma(d2, fma(d2, fma(d2, 1.0 / 362880.0, 1.0 / 5040.0), 1.0 / 120.0), 1.0 / 6.0), 1.0);
    em_pos = E + O;
    em_neg = E - O;
  } else {
    em_pos = expm1(d);
    em_neg = expm1(-d);
  }
}
__device__ inline void expm1_pair(float d, float& em_pos, float& em_neg) {
  if (fabsf(d) <= 0.0625f) {
    const float d2 = d * d;
    const float E = d2 * fmaf(d2, fmaf(d2, 1.0f / 720.0f, 1.0f / 24.0f), 0.5f);
    const float O = d * fmaf(d2, fmaf(d2, 1.0f / 120.0f, 1.0f / 6.0f), 1.0f);
    em_pos = E + O;
    em_neg = E - O;
  } else {
    em_pos = expm1f(d);
    em_neg = expm1f(-d);
  }
}

// max of positive values through their bit patterns (monotone for x > 0)
__device__ inline double pos_max(double a, double b) {
  const long long ia = __double_as_longlong(a), ib = __double_as_longlong(b);
  return __longlong_as_double(ia > ib ? ia : ib);
}
__device__ inline float pos_max(float a, float b) {
  const int ia = __float_as_int(a), ib = __float_as_int(b);
  return __int_as_float(ia > ib ? ia : ib);
}

template <class T>
__device__ inline T tabs(T x) { return x < T(0) ? -x : x; }

}  // namespace

// ------------------------------------------------------------------------------ cells
template <class T>
__global__ void __launch_bounds__(256) k_lean_cells(Box b, LeanCoef<T> c, LeanCellIn<T> in,
                                                    LeanCellOut<T> out, unsigned long long* red,
                                                    int check) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  double r_pt = 0.0, r_pf = 0.0;
  if (i <= b.nx && j <= b.ny && k <= b.nz) {
    const long long q = cidx(b, i, j, k);
    const long long px = b.px, pxy = b.pxy;
    const bool cell = i < b.nx && j < b.ny && k < b.nz;
    // ---- edges owned by this index: xy (i, j, k), xz (i, j, k), yz (i, j, k)
    if (k < b.nz) {
      T t = T(0);
      if (i > 0 && i < b.nx && j > 0 && j < b.ny) {
        const T e = (in.Vx[q] - in.Vx[q - px]) * c.hrdy + (in.Vy[q] - in.Vy[q - 1]) * c.hrdx;
        t = in.toa_xy[q] + in.em2_xy[q] * e;
      }
      out.txy[q] = t;
    }
    if (j < b.ny) {
      T t = T(0);
      if (i > 0 && i < b.nx && k > 0 && k < b.nz) {
        const T e = (in.Vx[q] - in.Vx[q - pxy]) * c.hrdz + (in.Vz[q] - in.Vz[q - 1]) * c.hrdx;
        t = in.toa_xz[q] + in.em2_xz[q] * e;
      }
      out.txz[q] = t;
    }
    if (i < b.nx) {
      T t = T(0);
      if (j > 0 && j < b.ny && k > 0 && k < b.nz) {
        const T e = (in.Vy[q] - in.Vy[q - pxy]) * c.hrdz + (in.Vz[q] - in.Vz[q - px]) * c.hrdy;
        t = in.toa_yz[q] + in.em2_yz[q] * e;
      }
      out.tyz[q] = t;
    }
    if (cell) {
      const T Pt = in.Pt[q], Pf = in.Pf[q], Pto = in.Pto[q], Pfo = in.Pfo[q];
      const T ph = in.phi[q], w = in.w[q], ieta = in.ieta[q];
      const T vxl = in.Vx[q], vxr = in.Vx[q + 1], vyl = in.Vy[q], vyr = in.Vy[q + px];
      const T vzl = in.Vz[q], vzr = in.Vz[q + pxy];
      const T gx = (vxr - vxl) * c.rdx, gy = (vyr - vyl) * c.rdy, gz = (vzr - vzl) * c.rdz;
      const T divV = gx + gy + gz;
      const T cc = c.compaction_on ? ieta * w : T(0);
      const T dPt = Pt - Pto, dPf = Pf - Pfo;
      const T divVn = divV + c.bd_rdt * (dPt - c.alpha * dPf) + (Pt - Pf) * cc;
      // Darcy flux through the six faces (zero on the boundary) and the largest neighbour k
      const T kc = in.perm[q];
      T kmax = kc, sx = T(0), sy = T(0), sz = T(0);
      if (i > 0) {
        const T kn = in.perm[q - 1];
        kmax = pos_max(kmax, kn);
        sx -= (kn + kc) * (Pf - in.Pf[q - 1]);
      }
      if (i < b.nx - 1) {
        const T kn = in.perm[q + 1];
        kmax = pos_max(kmax, kn);
        sx += (kc + kn) * (in.Pf[q + 1] - Pf);
      }
      if (j > 0) {
        const T kn = in.perm[q - px];
        kmax = pos_max(kmax, kn);
        sy -= (kn + kc) * (Pf - in.Pf[q - px]);
      }
      if (j < b.ny - 1) {
        const T kn = in.perm[q + px];
        kmax = pos_max(kmax, kn);
        sy += (kc + kn) * (in.Pf[q + px] - Pf);
      }
      if (k > 0) {
        const T kn = in.perm[q - pxy];
        kmax = pos_max(kmax, kn);
        sz -= (kn + kc) * ((Pf - in.Pf[q - pxy]) + c.buoy_dz);
      }
      if (k < b.nz - 1) {
        const T kn = in.perm[q + pxy];
        kmax = pos_max(kmax, kn);
        sz += (kc + kn) * ((in.Pf[q + pxy] - Pf) + c.buoy_dz);
      }
      // div qD = -1/2 sum_d rd^2 [(k + k_r)(Pf_r - Pf) - (k_l + k)(Pf - Pf_l)]
      const T divqD = -(sx * c.hrdx2 + sy * c.hrdy2 + sz * c.hrdz2);
      // local-implicit pressure updates, Eqs. 17-18, written with 1 / dtau
      const T idtp = in.idtp[q];
      const T Pt1 = (Pt * idtp - (divV - c.bd_rdt * (Pto + c.alpha * dPf) - cc * Pf)) /
                    (idtp + c.bd_rdt + cc);
      const T idtf = kmax * c.ifac_pf;
      const T Pf1 = (Pf * idtf - (divqD - c.bd_rdt * (c.alpha_B * Pfo + c.alpha * dPt) - cc * Pt)) /
                    (idtf + c.bda_B_rdt + cc);
      out.Pt[q] = Pt1;
      out.Pf[q] = Pf1;
      // normal deviatoric stresses (Eq. 21): tau = tau_o xi/(1+xi) + 2 mu/(1+xi) (edot + beta_n divVn)
      const T third = divV * T(1.0 / 3.0);
      const T bn = c.beta_n * divVn;
      const T cm2 = in.cm2[q];
      out.txx[q] = in.toa_xx[q] + cm2 * (gx - third + bn);
      out.tyy[q] = in.toa_yy[q] + cm2 * (gy - third + bn);
      out.tzz[q] = in.toa_zz[q] + cm2 * (gz - third + bn);
      // porosity in log space (Eq. 22): L = Lo + delta,
      // delta = -[beta_phi ((Pf1 - Pfo) - (Pt1 - Pto)) + dt (Pf1 - Pt1) / eta + dt V.grad(1-phi)/(1-phi)]
      T ax = T(0), ay = T(0), az = T(0);
      if (i > 0) ax += vxl * (ph - in.phi[q - 1]);
      if (i < b.nx - 1) ax += vxr * (in.phi[q + 1] - ph);
      if (j > 0) ay += vyl * (ph - in.phi[q - px]);
      if (j < b.ny - 1) ay += vyr * (in.phi[q + px] - ph);
      if (k > 0) az += vzl * (ph - in.phi[q - pxy]);
      if (k < b.nz - 1) az += vzr * (in.phi[q + pxy] - ph);
      // V.grad(1-phi)/(1-phi) = -(1/2) w sum_d rd (...)
      const T adv = -(ax * c.hrdx + ay * c.hrdy + az * c.hrdz) * w;
      const T comp = c.compaction_on ? (Pf1 - Pt1) * ieta : T(0);
      const T delta = -(c.beta_phi * ((Pf1 - Pfo) - (Pt1 - Pto)) + c.dt * (comp + adv));
      T em_p, em_n;
      expm1_pair(delta, em_p, em_n);
      const T phio = in.phio[q], Eo = in.Eo[q], iEo = in.iEo[q];
      const T ph1 = phio - Eo * em_p;
      out.phi[q] = ph1;
      out.w[q] = iEo + iEo * em_n;
      const T r = ph1 * c.rphi0;
      out.perm[q] = (in.K0 ? in.K0[q] : c.k0) * r * r * r;
      if (check) {
        r_pt = (double)tabs(divVn);
        r_pf = (double)tabs(divqD + c.bda_B_rdt * dPf - c.bd_rdt * c.alpha * dPt + (Pf - Pt) * cc);
      }
    }
  }
  if (check) {
    block_max_atomic(r_pt, red + RED_PT);
    block_max_atomic(r_pf, red + RED_PF);
  }
}

// ------------------------------------------------------------------------------ faces
template <class T>
__global__ void __launch_bounds__(256) k_lean_faces(Box b, LeanCoef<T> c, LeanFaceIn<T> in,
                                                    T* __restrict__ Vx, T* __restrict__ Vy,
                                                    T* __restrict__ Vz, T* __restrict__ Rx,
                                                    T* __restrict__ Ry, T* __restrict__ Rz,
                                                    unsigned long long* red, int check) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  double r_v = 0.0;
  if (i <= b.nx && j <= b.ny && k <= b.nz) {
    const long long q = cidx(b, i, j, k);
    const long long px = b.px, pxy = b.pxy;
    if (i > 0 && i < b.nx && j < b.ny && k < b.nz) {
      const T F = (in.txx[q] - in.txx[q - 1]) * c.rdx + (in.txy[q + px] - in.txy[q]) * c.rdy +
                  (in.txz[q + pxy] - in.txz[q]) * c.rdz - (in.Pt1[q] - in.Pt1[q - 1]) * c.rdx;
      const T R = F * c.rrho_i + c.damp_x * Rx[q];
      Rx[q] = R;
      Vx[q] += in.dtv_x[q] * R;
      if (check) r_v = fmax(r_v, (double)tabs(F));
    }
    if (j > 0 && j < b.ny && i < b.nx && k < b.nz) {
      const T F = (in.txy[q + 1] - in.txy[q]) * c.rdx + (in.tyy[q] - in.tyy[q - px]) * c.rdy +
                  (in.tyz[q + pxy] - in.tyz[q]) * c.rdz - (in.Pt1[q] - in.Pt1[q - px]) * c.rdy;
      const T R = F * c.rrho_i + c.damp_y * Ry[q];
      Ry[q] = R;
      Vy[q] += in.dtv_y[q] * R;
      if (check) r_v = fmax(r_v, (double)tabs(F));
    }
    if (k > 0 && k < b.nz && i < b.nx && j < b.ny) {
      // buoyancy -(rho g - rho_BG g) averaged to the face, rho g - rho_BG g = (phi - phi0) drho_g
      const T rog = (T(0.5) * (in.phi[q - pxy] + in.phi[q]) - c.phi0) * c.drho_g;
      const T F = (in.txz[q + 1] - in.txz[q]) * c.rdx + (in.tyz[q + px] - in.tyz[q]) * c.rdy +
                  (in.tzz[q] - in.tzz[q - pxy]) * c.rdz - (in.Pt1[q] - in.Pt1[q - pxy]) * c.rdz - rog;
      const T R = F * c.rrho_i + c.damp_z * Rz[q];
      Rz[q] = R;
      Vz[q] += in.dtv_z[q] * R;
      if (check) r_v = fmax(r_v, (double)tabs(F));
    }
  }
  if (check) block_max_atomic(r_v, red + RED_V);
}

// ------------------------------------------------------------------------------ Picard
template <class T>
__global__ void __launch_bounds__(256) k_lean_picard(Box b, LeanCoef<T> c, LeanPicardIn<T> in,
                                                     T* __restrict__ mu, T* __restrict__ eta,
                                                     unsigned long long* red) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  double r = 0.0;
  if (i < b.nx && j < b.ny && k < b.nz) {
    const long long q = cidx(b, i, j, k);
    const long long px = b.px, pxy = b.pxy;
    const double axy = 0.25 * ((double)in.txy[q] + in.txy[q + 1] + in.txy[q + px] + in.txy[q + 1 + px]);
    const double axz = 0.25 * ((double)in.txz[q] + in.txz[q + 1] + in.txz[q + pxy] + in.txz[q + 1 + pxy]);
    const double ayz = 0.25 * ((double)in.tyz[q] + in.tyz[q + px] + in.tyz[q + pxy] + in.tyz[q + px + pxy]);
    const double sxx = in.txx[q], syy = in.tyy[q], szz = in.tzz[q];
    const double tII = sqrt(0.5 * (sxx * sxx + syy * syy + szz * szz) + axy * axy + axz * axz + ayz * ayz);
    double mus = c.mu0;
    if (c.powerlaw_on) {
      const double x = tII / c.tau0;
      const double p = c.n_pow - 1.0;
      mus = c.mu0 / (1.0 + (p == 2.0 ? x * x : pow(x, p)));
    }
    const double mu_old = mu[q], eta_old = eta[q];
    const double lmus = log(mus), lmu = log(mu_old);
    const double mu_new = exp(c.rel_mu * lmus + (1.0 - c.rel_mu) * lmu);
    const double R = (in.Pf1[q] > in.Pt1[q]) ? c.R_weak : 1.0;
    const double etas = c.eta0 * mu_new / (double)in.phi1[q] * R;
    const double letas = log(etas), leta = log(eta_old);
    r = fmax(fabs(lmus - lmu), fabs(letas - leta));
    mu[q] = (T)mu_new;
    eta[q] = (T)exp(c.rel_eta * letas + (1.0 - c.rel_eta) * leta);
  }
  block_max_atomic(r, red + RED_PIC);
}

// --------------------------------------------------------------------- coefficient refresh
// From mu, eta and the raw old stresses (after a Picard update or a step start).
template <class T>
__global__ void __launch_bounds__(256) k_lean_coef(Box b, LeanCoef<T> c, LeanCoefIn<T> in,
                                                   LeanCoefOut<T> out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i > b.nx || j > b.ny || k > b.nz) return;
  const long long q = cidx(b, i, j, k);
  const long long px = b.px, pxy = b.pxy;
  const double rG = c.rGdtS;
  if (i < b.nx && j < b.ny && k < b.nz) {
    const double m = in.mu[q];
    const double s = 1.0 / (1.0 + m * rG);
    const double a = 1.0 - s;                         // xi / (1 + xi)
    out.cm2[q] = (T)(2.0 * m * s);
    out.toa_xx[q] = (T)(in.txxo[q] * a);
    out.toa_yy[q] = (T)(in.tyyo[q] * a);
    out.toa_zz[q] = (T)(in.tzzo[q] * a);
    out.idtp[q] = (T)(1.0 / (c.dtaupt_fac * m));
    out.ieta[q] = (T)(1.0 / (double)in.eta[q]);
  }
  if (k < b.nz && i > 0 && i < b.nx && j > 0 && j < b.ny) {
    const double m = 0.25 * ((double)in.mu[q - 1 - px] + in.mu[q - px] + in.mu[q - 1] + in.mu[q]);
    const double s = 1.0 / (1.0 + m * rG);
    out.em2_xy[q] = (T)(2.0 * m * s);
    out.toa_xy[q] = (T)(in.txyo[q] * (1.0 - s));
  }
  if (j < b.ny && i > 0 && i < b.nx && k > 0 && k < b.nz) {
    const double m = 0.25 * ((double)in.mu[q - 1 - pxy] + in.mu[q - pxy] + in.mu[q - 1] + in.mu[q]);
    const double s = 1.0 / (1.0 + m * rG);
    out.em2_xz[q] = (T)(2.0 * m * s);
    out.toa_xz[q] = (T)(in.txzo[q] * (1.0 - s));
  }
  if (i < b.nx && j > 0 && j < b.ny && k > 0 && k < b.nz) {
    const double m = 0.25 * ((double)in.mu[q - px - pxy] + in.mu[q - pxy] + in.mu[q - px] + in.mu[q]);
    const double s = 1.0 / (1.0 + m * rG);
    out.em2_yz[q] = (T)(2.0 * m * s);
    out.toa_yz[q] = (T)(in.tyzo[q] * (1.0 - s));
  }
  // pseudo-time steps of the velocities, mean of the two centres' dtau_V = fac / mu
  if (i > 0 && i < b.nx && j < b.ny && k < b.nz)
    out.dtv_x[q] = (T)(0.5 * c.dtauv_fac * (1.0 / (double)in.mu[q - 1] + 1.0 / (double)in.mu[q]));
  if (j > 0 && j < b.ny && i < b.nx && k < b.nz)
    out.dtv_y[q] = (T)(0.5 * c.dtauv_fac * (1.0 / (double)in.mu[q - px] + 1.0 / (double)in.mu[q]));
  if (k > 0 && k < b.nz && i < b.nx && j < b.ny)
    out.dtv_z[q] = (T)(0.5 * c.dtauv_fac * (1.0 / (double)in.mu[q - pxy] + 1.0 / (double)in.mu[q]));
}

// ------------------------------------------------------------------------ step start
// phio = phi, Eo = 1 - phi, iEo = 1 / (1 - phi), w = iEo, k from phi; Pto, Pfo; max(mu).
template <class T>
__global__ void __launch_bounds__(256) k_lean_begin(Box b, LeanCoef<T> c, LeanBeginIn<T> in,
                                                    LeanBeginOut<T> out, unsigned long long* red) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  double m = 0.0;
  if (i < b.nx && j < b.ny && k < b.nz) {
    const long long q = cidx(b, i, j, k);
    const double ph = in.phi[q];
    const double Eo = 1.0 - ph;
    const double iEo = 1.0 / Eo;
    out.Pto[q] = in.Pt[q];
    out.Pfo[q] = in.Pf[q];
    out.phio[q] = (T)ph;
    out.Eo[q] = (T)Eo;
    out.iEo[q] = (T)iEo;
    out.w[q] = (T)iEo;
    const double r = ph * (double)c.rphi0;
    out.perm[q] = (T)((in.K0 ? (double)in.K0[q] : (double)c.k0) * r * r * r);
    m = in.mu[q];
  }
  block_max_atomic(m, red + RED_MUMAX);
}

// K0 = k0 e^logk / phi0^3 is folded into k = K0 phi^3; here K0 = k0 e^logk (phi0 via rphi0).
template <class T>
__global__ void k_lean_k0(Box b, double k0, const double* __restrict__ logk, T* __restrict__ K0) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i < b.nx && j < b.ny && k < b.nz) {
    const long long q = cidx(b, i, j, k);
    K0[q] = (T)(k0 * exp(logk[q]));
  }
}

template <class T>
void lean_cells(dim3 gr, dim3 bl, cudaStream_t st, Box b, const LeanCoef<T>& c, const LeanCellIn<T>& in,
                const LeanCellOut<T>& out, unsigned long long* red, int check) {
  k_lean_cells<T><<<gr, bl, 0, st>>>(b, c, in, out, red, check);
}
template <class T>
void lean_faces(dim3 gr, dim3 bl, cudaStream_t st, Box b, const LeanCoef<T>& c, const LeanFaceIn<T>& in,
                T* Vx, T* Vy, T* Vz, T* Rx, T* Ry, T* Rz, unsigned long long* red, int check) {
  k_lean_faces<T><<<gr, bl, 0, st>>>(b, c, in, Vx, Vy, Vz, Rx, Ry, Rz, red, check);
}
template <class T>
void lean_picard(dim3 gr, dim3 bl, cudaStream_t st, Box b, const LeanCoef<T>& c, const LeanPicardIn<T>& in,
                 T* mu, T* eta, unsigned long long* red) {
  k_lean_picard<T><<<gr, bl, 0, st>>>(b, c, in, mu, eta, red);
}
template <class T>
void lean_coef(dim3 gr, dim3 bl, cudaStream_t st, Box b, const LeanCoef<T>& c, const LeanCoefIn<T>& in,
               const LeanCoefOut<T>& out) {
  k_lean_coef<T><<<gr, bl, 0, st>>>(b, c, in, out);
}
template <class T>
void lean_begin(dim3 gr, dim3 bl, cudaStream_t st, Box b, const LeanCoef<T>& c, const LeanBeginIn<T>& in,
                const LeanBeginOut<T>& out, unsigned long long* red) {
  k_lean_begin<T><<<gr, bl, 0, st>>>(b, c, in, out, red);
}
template <class T>
void lean_k0(dim3 gr, dim3 bl, cudaStream_t st, Box b, double k0, const double* logk, T* K0) {
  k_lean_k0<T><<<gr, bl, 0, st>>>(b, k0, logk, K0);
}

template void lean_cells<double>(dim3, dim3, cudaStream_t, Box, const LeanCoef<double>&, const LeanCellIn<double>&,
                                 const LeanCellOut<double>&, unsigned long long*, int);
template void lean_faces<double>(dim3, dim3, cudaStream_t, Box, const LeanCoef<double>&, const LeanFaceIn<double>&,
                                 double*, double*, double*, double*, double*, double*, unsigned long long*, int);
template void lean_picard<double>(dim3, dim3, cudaStream_t, Box, const LeanCoef<double>&, const LeanPicardIn<double>&,
                                  double*, double*, unsigned long long*);
template void lean_coef<double>(dim3, dim3, cudaStream_t, Box, const LeanCoef<double>&, const LeanCoefIn<double>&,
                                const LeanCoefOut<double>&);
template void lean_begin<double>(dim3, dim3, cudaStream_t, Box, const LeanCoef<double>&, const LeanBeginIn<double>&,
                                 const LeanBeginOut<double>&, unsigned long long*);
template void lean_k0<double>(dim3, dim3, cudaStream_t, Box, double, const double*, double*);

}  // namespace pt
