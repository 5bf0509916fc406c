// pt_lean_body.cuh — per-point bodies of the FP64-lean PT kernels (see pt_lean_kernels.cu for
// the method), shared by the single-instance kernels and the batched (ensemble) kernels.
#pragma once

#include "pt_lean.cuh"

namespace pt {
namespace lean_detail {

// exp(d) - 1 and exp(-d) - 1 from the Taylor series of exp split into its odd part
// O = d + d^3/3! + ... and even part E = d^2/2! + d^4/4! + ... (truncated after d^3 / d^2 for
// |d| <= 2^-20 and after d^9 / d^8 for |d| <= 2^-6: in both cases the first dropped term is
// below 2^-60 |d|). expm1(d) = E + O, expm1(-d) = E - O.
__device__ inline void expm1_pair(double d, double& em_pos, double& em_neg) {
  if (fabs(d) <= 0x1p-20) {
    const double d2 = d * d;
    const double E = 0.5 * d2;
    const double O = d * fma(d2, 1.0 / 6.0, 1.0);
    em_pos = E + O;
    em_neg = E - O;
  } else if (fabs(d) <= 0.015625) {
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

// 1 / x for the local-implicit pseudo-step denominators (x > 0, far inside the normal range):
// the hardware's approximate reciprocal refined by one Newton step, r' = r + r (1 - x r), whose
// relative error is the square of the seed's (~2^-46 in FP64). It only scales the pseudo-time
// step of the update P - res / x, so the fixed point of the iteration does not depend on it.
__device__ inline double rcp_pseudo(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  return fma(r, fma(-x, r, 1.0), r);
}
__device__ inline float rcp_pseudo(float x) { return __frcp_rn(x); }

// 1 / x to rounding accuracy for the coefficients that set the fixed point (x > 0, normal):
// two Newton steps r' = r + r (1 - x r) on the hardware's approximate reciprocal.
__device__ inline double rcp_full(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  r = fma(r, fma(-x, r, 1.0), r);
  return fma(r, fma(-x, r, 1.0), r);
}


}  // namespace lean_detail

// Cells, stresses of the three lower edges, pressures, porosity at box index (i, j, k).
template <class T>
__device__ __forceinline__ void lean_cell_point(const Box& b, const LeanCoef<T>& c, const LeanCellIn<T>& in,
                                                const LeanCellOut<T>& out, int i, int j, int k, int check,
                                                double& r_pt, double& r_pf) {
  using namespace lean_detail;
  if (i <= b.nx && j <= b.ny && k <= b.nz) {
    const long long q = cidx(b, i, j, k);
    const long long px = b.px, pxy = b.pxy;
    const bool cell = i < b.nx && j < b.ny && k < b.nz;
    // ---- edges owned by this index: xy (i, j, k), xz (i, j, k), yz (i, j, k); stored at the end
    // with the cell's outputs, after every load (the arrays are not declared non-aliasing)
    T t_xy = T(0), t_xz = T(0), t_yz = T(0);
    if (k < b.nz && i > 0 && i < b.nx && j > 0 && j < b.ny) {   // toa_xy holds the background part too
      t_xy = fma(in.eb_xy[q], in.Vy[q] - in.Vy[q - 1], fma(in.em2_xy[q], in.Vx[q] - in.Vx[q - px], in.toa_xy[q]));
    } else if (k < b.nz && c.bg_on) {   // wall xy-edge under background shear (Eqs. 32-33)
      t_xy = in.toa_xy[q];
    }
    if (j < b.ny && i > 0 && i < b.nx && k > 0 && k < b.nz)
      t_xz = fma(in.eb_xz[q], in.Vz[q] - in.Vz[q - 1], fma(in.em2_xz[q], in.Vx[q] - in.Vx[q - pxy], in.toa_xz[q]));
    if (i < b.nx && j > 0 && j < b.ny && k > 0 && k < b.nz)
      t_yz = fma(in.eb_yz[q], in.Vz[q] - in.Vz[q - px], fma(in.em2_yz[q], in.Vy[q] - in.Vy[q - pxy], in.toa_yz[q]));
    if (cell) {
      const T Pt = in.Pt[q], Pf = in.Pf[q], Pto = in.Pto[q], Pfo = in.Pfo[q];
      const T ph = in.phi[q], w = in.w[q], ieta = in.ieta[q];
      const T vxl = in.Vx[q], vxr = in.Vx[q + 1], vyl = in.Vy[q], vyr = in.Vy[q + px];
      const T vzl = in.Vz[q], vzr = in.Vz[q + pxy];
      const T gx = (vxr - vxl) * c.rdx, gy = (vyr - vyl) * c.rdy, gz = (vzr - vzl) * c.rdz;
      const T divV = gx + gy + gz;
      const T cc = c.compaction_on ? ieta * w : T(0);
      const T dPt = Pt - Pto, dPf = Pf - Pfo, dpp = Pt - Pf;
      // explicit fused multiply-adds: the same rounding in every kernel that inlines this body
      const T divVn = fma(dpp, cc, fma(-c.bd_rdt_a, dPf, fma(c.bd_rdt, dPt, divV)));
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
      // local-implicit pressure updates, Eqs. 17-18: P1 = P - res / (1/dtau + d res/dP), the
      // residuals being divVn (row Pt) and resF (row Pf)
      const T resF = fma(-dpp, cc, fma(-c.bd_rdt_a, dPt, fma(c.bda_B_rdt, dPf, divqD)));
      const T Pt1 = Pt - rcp_pseudo(in.idtp[q] + cc) * divVn;   // idtp holds 1/dtau_Pt + beta_d/dt
      const T Pf1 = Pf - rcp_pseudo(kmax * c.ifac_pf + c.bda_B_rdt + cc) * resF;
      // normal deviatoric stresses (Eq. 21): tau = tau_o xi/(1+xi) + 2 mu/(1+xi) (edot + beta_n divVn)
      const T s3 = fma(c.beta_n, divVn, -(divV * T(1.0 / 3.0)));
      const T cm2 = in.cm2[q];
      const T sxx = fma(cm2, gx + s3, in.toa_xx[q]);
      const T syy = fma(cm2, gy + s3, in.toa_yy[q]);
      const T szz = fma(cm2, gz + s3, in.toa_zz[q]);
      // porosity in log space (Eq. 22): L = Lo + delta,
      // delta = -[beta_phi ((Pf1 - Pfo) - (Pt1 - Pto)) + dt (Pf1 - Pt1) / eta + dt V.grad(1-phi)/(1-phi)]
      // V.grad(1-phi)/(1-phi) = -(w/2) sum_d rd [v_r (phi_r - phi) + v_l (phi - phi_l)]
      //                      = -w [sum_d hrd (v_r phi_r - v_l phi_l) - phi divV / 2]
      // (the velocities of wall faces are zero, so the divergence term is div V exactly)
      T ax = T(0), ay = T(0), az = T(0);
      if (i > 0) ax = -vxl * in.phi[q - 1];
      if (i < b.nx - 1) ax = fma(vxr, in.phi[q + 1], ax);
      if (j > 0) ay = -vyl * in.phi[q - px];
      if (j < b.ny - 1) ay = fma(vyr, in.phi[q + px], ay);
      if (k > 0) az = -vzl * in.phi[q - pxy];
      if (k < b.nz - 1) az = fma(vzr, in.phi[q + pxy], az);
      const T adv = -w * fma(T(-0.5) * ph, divV, fma(ax, c.hrdx, fma(ay, c.hrdy, az * c.hrdz)));
      const T comp = c.compaction_on ? (Pf1 - Pt1) * ieta : T(0);
      const T delta = -(c.beta_phi * ((Pf1 - Pfo) - (Pt1 - Pto)) + c.dt * (comp + adv));
      T em_p, em_n;
      expm1_pair(delta, em_p, em_n);
      const T phio = in.phio[q], Eo = in.Eo[q], iEo = in.iEo[q];
      const T K0 = in.K0 ? in.K0[q] : c.k0;
      const T ph1 = phio - Eo * em_p;
      const T r = ph1 * c.rphi0;
      // every load above precedes the stores (the arrays are not declared non-aliasing)
      out.Pt[q] = Pt1;
      out.Pf[q] = Pf1;
      out.txx[q] = sxx;
      out.tyy[q] = syy;
      out.tzz[q] = szz;
      out.phi[q] = ph1;
      out.w[q] = iEo + iEo * em_n;
      out.perm[q] = K0 * r * r * r;
      if (check) {
        r_pt = (double)tabs(divVn);
        r_pf = (double)tabs(resF);
      }
    }
    if (k < b.nz) out.txy[q] = t_xy;
    if (j < b.ny) out.txz[q] = t_xz;
    if (i < b.nx) out.tyz[q] = t_yz;
  }
}

// Momentum residual, damped R and velocity update of the three lower faces of (i, j, k); bit d
// of `mask` includes the face normal to direction d in the residual norm r_v.
template <class T>
__device__ __forceinline__ void lean_face_point(const Box& b, const LeanCoef<T>& c, const LeanFaceIn<T>& in,
                                                T* __restrict__ Vx, T* __restrict__ Vy, T* __restrict__ Vz,
                                                T* __restrict__ Rx, T* __restrict__ Ry, T* __restrict__ Rz,
                                                int i, int j, int k, int check, double& r_v, int mask = 7) {
  using namespace lean_detail;
  if (i <= b.nx && j <= b.ny && k <= b.nz) {
    const long long q = cidx(b, i, j, k);
    const long long px = b.px, pxy = b.pxy;
    const bool fx = i > 0 && i < b.nx && j < b.ny && k < b.nz;
    const bool fy = j > 0 && j < b.ny && i < b.nx && k < b.nz;
    const bool fz = k > 0 && k < b.nz && i < b.nx && j < b.ny;
    // all loads before the first store (the arrays are not declared non-aliasing)
    T Fx = T(0), Fy = T(0), Fz = T(0), Rx1 = T(0), Ry1 = T(0), Rz1 = T(0), Vx1 = T(0), Vy1 = T(0), Vz1 = T(0);
    // F / rho_i directly (the spacings carry 1/rho_i); the norm takes |F| = rho_i |F / rho_i|
    if (fx) {
      Fx = (in.txx[q] - in.txx[q - 1]) * c.rdx_r + (in.txy[q + px] - in.txy[q]) * c.rdy_r +
           (in.txz[q + pxy] - in.txz[q]) * c.rdz_r - (in.Pt1[q] - in.Pt1[q - 1]) * c.rdx_r;
      Rx1 = fma(c.damp_x, Rx[q], Fx);
      Vx1 = fma(in.dtv_x[q], Rx1, Vx[q]);
    }
    if (fy) {
      Fy = (in.txy[q + 1] - in.txy[q]) * c.rdx_r + (in.tyy[q] - in.tyy[q - px]) * c.rdy_r +
           (in.tyz[q + pxy] - in.tyz[q]) * c.rdz_r - (in.Pt1[q] - in.Pt1[q - px]) * c.rdy_r;
      Ry1 = fma(c.damp_y, Ry[q], Fy);
      Vy1 = fma(in.dtv_y[q], Ry1, Vy[q]);
    }
    if (fz) {
      // buoyancy -(rho g - rho_BG g) averaged to the face, rho g - rho_BG g = (phi - phi0) drho_g
      const T rog = (T(0.5) * (in.phi[q - pxy] + in.phi[q]) - c.phi0) * c.drho_g_r;
      Fz = (in.txz[q + 1] - in.txz[q]) * c.rdx_r + (in.tyz[q + px] - in.tyz[q]) * c.rdy_r +
           (in.tzz[q] - in.tzz[q - pxy]) * c.rdz_r - (in.Pt1[q] - in.Pt1[q - pxy]) * c.rdz_r - rog;
      Rz1 = fma(c.damp_z, Rz[q], Fz);
      Vz1 = fma(in.dtv_z[q], Rz1, Vz[q]);
    }
    if (fx) { Rx[q] = Rx1; Vx[q] = Vx1; }
    if (fy) { Ry[q] = Ry1; Vy[q] = Vy1; }
    if (fz) { Rz[q] = Rz1; Vz[q] = Vz1; }
    if (check) {
      if (fx && (mask & 1)) r_v = fmax(r_v, (double)tabs(Fx) * (double)c.rho_i);
      if (fy && (mask & 2)) r_v = fmax(r_v, (double)tabs(Fy) * (double)c.rho_i);
      if (fz && (mask & 4)) r_v = fmax(r_v, (double)tabs(Fz) * (double)c.rho_i);
    }
  }
}

// Picard targets and relaxation at cell (i, j, k). m = max(x, 1/x) over the ratios x = mu*/mu
// and eta*/eta (>= 1): its log is the Picard change max(|log mu* - log mu|, |log eta* - log eta|),
// taken once per block by the caller (log is monotone).
template <class T>
__device__ __forceinline__ void lean_picard_point(const Box& b, const LeanCoef<T>& c, const LeanPicardIn<T>& in,
                                                  T* __restrict__ mu, T* __restrict__ eta, int i, int j, int k,
                                                  double& m) {
  using namespace lean_detail;
  if (i < b.nx && j < b.ny && k < b.nz) {
    const long long q = cidx(b, i, j, k);
    const long long px = b.px, pxy = b.pxy;
    const double axy = 0.25 * ((double)in.txy[q] + in.txy[q + 1] + in.txy[q + px] + in.txy[q + 1 + px]);
    const double axz = 0.25 * ((double)in.txz[q] + in.txz[q + 1] + in.txz[q + pxy] + in.txz[q + 1 + pxy]);
    const double ayz = 0.25 * ((double)in.tyz[q] + in.tyz[q + px] + in.tyz[q + pxy] + in.tyz[q + px + pxy]);
    const double sxx = in.txx[q], syy = in.tyy[q], szz = in.tzz[q];
    // tau_II^2 = (sxx^2 + syy^2 + szz^2) / 2 + axy^2 + axz^2 + ayz^2 (explicit FMAs: every form
    // that inlines this body rounds it alike)
    const double tII2 = fma(0.5, fma(sxx, sxx, fma(syy, syy, szz * szz)), fma(axy, axy, fma(axz, axz, ayz * ayz)));
    // Eq. 24: mu* = mu0 / (1 + (tau_II / tau0)^(n-1)); the log-space relaxation
    // exp(rel log mu* + (1 - rel) log mu) is written mu (mu* / mu)^rel (a square root for rel = 1/2)
    double den = 1.0;
    if (c.powerlaw_on) {
      const double x2 = tII2 * c.rtau0_2;                        // (tau_II / tau0)^2
      const double p = c.n_pow - 1.0;
      den = p == 2.0 ? 1.0 + x2 : 1.0 + exp(0.5 * p * log(x2));
    }
    const double mu_old = mu[q], eta_old = eta[q];
    const double x_mu = c.mu0 / (den * mu_old);                  // mu* / mu
    const double mu_new = mu_old * (c.rel_mu == 0.5 ? sqrt(x_mu) : exp(c.rel_mu * log(x_mu)));
    const double R = (in.Pf1[q] > in.Pt1[q]) ? c.R_weak : 1.0;
    // Eq. 26: eta* = eta0 mu / phi R (with the relaxed mu), relaxed the same way
    const double x_eta = c.eta0 * mu_new * R / ((double)in.phi1[q] * eta_old);
    m = fmax(fmax(x_mu, rcp_full(x_mu)), fmax(x_eta, rcp_full(x_eta)));
    if (!(x_mu == x_mu && x_eta == x_eta)) m = x_mu + x_eta;     // NaN stays NaN (fmax drops it)
    mu[q] = (T)mu_new;
    eta[q] = (T)(eta_old * (c.rel_eta == 0.5 ? sqrt(x_eta) : exp(c.rel_eta * log(x_eta))));
  }
}

// Coefficient refresh at box index (i, j, k).
template <class T>
__device__ __forceinline__ void lean_coef_point(const Box& b, const LeanCoef<T>& c, const LeanCoefIn<T>& in,
                                                const LeanCoefOut<T>& out, int i, int j, int k) {
  using namespace lean_detail;
  if (i > b.nx || j > b.ny || k > b.nz) return;
  const long long q = cidx(b, i, j, k);
  const long long px = b.px, pxy = b.pxy;
  const double rG = c.rGdtS;
  if (i < b.nx && j < b.ny && k < b.nz) {
    const double m = in.mu[q];
    const double s = rcp_full(fma(m, rG, 1.0));
    const double a = 1.0 - s;                         // xi / (1 + xi)
    out.cm2[q] = (T)(2.0 * m * s);
    out.toa_xx[q] = (T)(in.txxo[q] * a);
    out.toa_yy[q] = (T)(in.tyyo[q] * a);
    out.toa_zz[q] = (T)(in.tzzo[q] * a);
    out.idtp[q] = (T)(rcp_full(c.dtaupt_fac * m) + (double)c.bd_rdt);   // 1/dtau_Pt + beta_d/dt
    out.ieta[q] = (T)rcp_full((double)in.eta[q]);
  }
  if (k < b.nz && i > 0 && i < b.nx && j > 0 && j < b.ny) {
    const double m = 0.25 * ((double)in.mu[q - 1 - px] + in.mu[q - px] + in.mu[q - 1] + in.mu[q]);
    const double s = rcp_full(fma(m, rG, 1.0));
    out.em2_xy[q] = (T)(2.0 * m * s * (double)c.hrdy);
    out.eb_xy[q] = (T)(2.0 * m * s * (double)c.hrdx);
    // the background shear's stress 2 mu/(1+xi) tau_bg/(2 mu0) (Eqs. 32-33) joins the old-stress part
    out.toa_xy[q] = (T)(in.txyo[q] * (1.0 - s) + 2.0 * m * s * (double)c.ebg);
  } else if (k < b.nz && c.bg_on) {   // wall xy-edges carry the background stress
    const double m = edge_mean_mu_xy(b, in.mu, q, i, j);
    const double s = rcp_full(fma(m, rG, 1.0));
    out.toa_xy[q] = (T)(in.txyo[q] * (1.0 - s) + 2.0 * m * s * (double)c.ebg);
  }
  if (j < b.ny && i > 0 && i < b.nx && k > 0 && k < b.nz) {
    const double m = 0.25 * ((double)in.mu[q - 1 - pxy] + in.mu[q - pxy] + in.mu[q - 1] + in.mu[q]);
    const double s = rcp_full(fma(m, rG, 1.0));
    out.em2_xz[q] = (T)(2.0 * m * s * (double)c.hrdz);
    out.eb_xz[q] = (T)(2.0 * m * s * (double)c.hrdx);
    out.toa_xz[q] = (T)(in.txzo[q] * (1.0 - s));
  }
  if (i < b.nx && j > 0 && j < b.ny && k > 0 && k < b.nz) {
    const double m = 0.25 * ((double)in.mu[q - px - pxy] + in.mu[q - pxy] + in.mu[q - px] + in.mu[q]);
    const double s = rcp_full(fma(m, rG, 1.0));
    out.em2_yz[q] = (T)(2.0 * m * s * (double)c.hrdz);
    out.eb_yz[q] = (T)(2.0 * m * s * (double)c.hrdy);
    out.toa_yz[q] = (T)(in.tyzo[q] * (1.0 - s));
  }
  // pseudo-time steps of the velocities, mean of the two centres' dtau_V = fac / mu
  const double imu = (i < b.nx && j < b.ny && k < b.nz) ? rcp_full((double)in.mu[q]) : 0.0;
  if (i > 0 && i < b.nx && j < b.ny && k < b.nz)
    out.dtv_x[q] = (T)(0.5 * c.dtauv_fac * (rcp_full((double)in.mu[q - 1]) + imu));
  if (j > 0 && j < b.ny && i < b.nx && k < b.nz)
    out.dtv_y[q] = (T)(0.5 * c.dtauv_fac * (rcp_full((double)in.mu[q - px]) + imu));
  if (k > 0 && k < b.nz && i < b.nx && j < b.ny)
    out.dtv_z[q] = (T)(0.5 * c.dtauv_fac * (rcp_full((double)in.mu[q - pxy]) + imu));
}

}  // namespace pt
