// pt_lean_body.cuh — per-point bodies of the FP64-lean PT kernels (see pt_lean_kernels.cu for
// the method), shared by the single-instance kernels and the batched (ensemble) kernels.
#pragma once

#include "df64.cuh"
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
// relative error is the square of the seed's (the approximate FP64 reciprocal is good to about
// 2^-20, so ~2^-40 after the step; measured below 1e-12). It only scales the pseudo-time step of
// the update P - res / x, so the fixed point of the iteration does not depend on it.
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

// ---- the same operations in double-float (PT_DF64): one Newton step from the FP32 seed
// reaches the format's own rounding (~2^-46), so the pseudo-step and the fixed-point
// reciprocals are the same function
__device__ inline df64 rcp_pseudo(df64 x) { return df_rcp(x); }
__device__ inline df64 rcp_full(df64 x) { return df_rcp(x); }

__device__ inline df64 pos_max(df64 a, df64 b) { return a < b ? b : a; }

// Same tiers as the FP64 pair (the truncation stays below 2^-60 |d|, far under the format's
// 2^-48); outside them the library expm1 in FP64.
__device__ inline void expm1_pair(df64 d, df64& em_pos, df64& em_neg) {
  const float ad = fabsf(d.hi);
  if (ad <= 0x1p-20f) {
    const df64 d2 = d * d;
    const df64 E = scale2(d2, 0.5f);
    const df64 O = d * fma(d2, df64(1.0 / 6.0), df64(1.0));
    em_pos = E + O;
    em_neg = E - O;
  } else if (ad <= 0.015625f) {
    const df64 d2 = d * d;
    const df64 E = d2 * fma(d2, fma(d2, fma(d2, df64(1.0 / 40320.0), df64(1.0 / 720.0)), df64(1.0 / 24.0)),
                            df64(0.5));
    const df64 O = d * fma(d2, fma(d2, fma(d2, fma(d2, df64(1.0 / 362880.0), df64(1.0 / 5040.0)),
                                           df64(1.0 / 120.0)), df64(1.0 / 6.0)), df64(1.0));
    em_pos = E + O;
    em_neg = E - O;
  } else {
    const double x = (double)d;
    em_pos = df64(expm1(x));
    em_neg = df64(expm1(-x));
  }
}

// conversions between the field type and FP64 (identity for FP64)
__device__ inline double to_d(double x) { return x; }
__device__ inline double to_d(df64 x) { return (double)x; }
template <class T>
__device__ inline T from_d(double x) { return T(x); }

// a / b: the plain quotient in FP64, the refined reciprocal in double-float
__device__ inline double tdiv(double a, double b) { return a / b; }
__device__ inline df64 tdiv(df64 a, df64 b) { return a * df_rcp(b); }

__device__ inline double tmax(double a, double b) { return fmax(a, b); }
__device__ inline df64 tmax(df64 a, df64 b) { return a < b ? b : a; }

// x^rel of the log-space Picard relaxation (x > 0). FP64: sqrt for rel = 1/2, else
// exp(rel log x). Double-float: the square root for rel = 1/2, Newton's m-th root for
// rel = 1/m (root = m, set on the host), else exp(rel log x) in FP64.
__device__ inline double relax_pow(double x, double rel, int /*root*/) {
  return rel == 0.5 ? sqrt(x) : exp(rel * log(x));
}
__device__ inline df64 relax_pow(df64 x, double rel, int root) {
  if (root == 2) return df_sqrt(x);
  if (root > 2) return df_root(x, root);
  return df64(exp(rel * log((double)x)));
}


}  // namespace lean_detail

// Which arrays a form stores. The FP64 form is bound by the FP64 pipe and stores everything that
// changes less often than every iteration (1/(1-phi) and k travelling with phi, 1 - phi_o and its
// reciprocal, edge moduli pre-multiplied by both spacings, three face pseudo-steps). Double-float
// arithmetic is cheap and the double-float form is bound by HBM and instruction issue, so it
// recomputes 1/(1-phi), 1 - phi_o and its reciprocal, keeps one modulus per edge (em2_* hold
// 2 mu/(1+xi); eb_* unused) and one velocity pseudo-step per centre (dtv_x = dtv_y = dtv_z hold
// fac / mu, averaged to each face): 56 fewer bytes per cell and iteration.
template <class T>
struct LeanRecompute { static constexpr bool value = false; };
template <>
struct LeanRecompute<df64> { static constexpr bool value = true; };
// k(phi) travels with phi (written by the cells kernel for the next iteration) in both forms:
// recomputing it for the cell and its six neighbours costs more issue slots than its 16 bytes
template <class T>
struct LeanStoreK { static constexpr bool value = true; };

// Where the cells body reads the arrays it needs only at its own index q ("pointwise"): straight
// from global memory, or from a shared-memory stage that cp.async filled ahead (slot order below).
enum { S_PTO, S_PFO, S_PHIO, S_IETA, S_IDTP, S_CM2, S_TXX, S_TYY, S_TZZ, S_EXY, S_EXZ, S_EYZ, S_TXY, S_TXZ,
       S_TYZ, kStageSlots,
       // own-index values of the neighbour arrays (staged too when the whole level is staged)
       S_VX = kStageSlots, S_VY, S_VZ, S_PT, S_PF, S_PHI, S_K, kStageSlotsAll };
struct DirectPoint {
  template <class T>
  __device__ __forceinline__ T operator()(const T* a, long long q, int) const { return a[q]; }
};

// Cells, stresses of the three lower edges, pressures, porosity at box index (i, j, k).
template <class T, class PP = DirectPoint>
__device__ __forceinline__ void lean_cell_point(const Box& b, const LeanCoef<T>& c, const LeanCellIn<T>& in,
                                                const LeanCellOut<T>& out, int i, int j, int k, int check,
                                                double& r_pt, double& r_pf, const PP& pp = PP()) {
  using namespace lean_detail;
  if (i <= b.nx && j <= b.ny && k <= b.nz) {
    const long long q = cidx(b, i, j, k);
    const long long px = b.px, pxy = b.pxy;
    const bool cell = i < b.nx && j < b.ny && k < b.nz;
    // ---- edges owned by this index: xy (i, j, k), xz (i, j, k), yz (i, j, k); stored at the end
    // with the cell's outputs, after every load (the arrays are not declared non-aliasing)
    constexpr bool RC = LeanRecompute<T>::value;
    constexpr bool KS = LeanStoreK<T>::value;
    T t_xy = T(0), t_xz = T(0), t_yz = T(0);
    if (k < b.nz && i > 0 && i < b.nx && j > 0 && j < b.ny) {   // toa_xy holds the background part too
      if constexpr (RC)
        t_xy = fma(pp(in.em2_xy, q, S_EXY), fma(pp(in.Vy, q, S_VY) - in.Vy[q - 1], c.hrdx,
                                                (pp(in.Vx, q, S_VX) - in.Vx[q - px]) * c.hrdy),
                   pp(in.toa_xy, q, S_TXY));
      else
        t_xy = fma(in.eb_xy[q], in.Vy[q] - in.Vy[q - 1], fma(pp(in.em2_xy, q, S_EXY), in.Vx[q] - in.Vx[q - px],
                                                             pp(in.toa_xy, q, S_TXY)));
    } else if (k < b.nz && c.bg_on) {   // wall xy-edge under background shear (Eqs. 32-33)
      t_xy = pp(in.toa_xy, q, S_TXY);
    }
    if (j < b.ny && i > 0 && i < b.nx && k > 0 && k < b.nz) {
      if constexpr (RC)
        t_xz = fma(pp(in.em2_xz, q, S_EXZ), fma(pp(in.Vz, q, S_VZ) - in.Vz[q - 1], c.hrdx,
                                                (pp(in.Vx, q, S_VX) - in.Vx[q - pxy]) * c.hrdz),
                   pp(in.toa_xz, q, S_TXZ));
      else
        t_xz = fma(in.eb_xz[q], in.Vz[q] - in.Vz[q - 1], fma(pp(in.em2_xz, q, S_EXZ), in.Vx[q] - in.Vx[q - pxy],
                                                             pp(in.toa_xz, q, S_TXZ)));
    }
    if (i < b.nx && j > 0 && j < b.ny && k > 0 && k < b.nz) {
      if constexpr (RC)
        t_yz = fma(pp(in.em2_yz, q, S_EYZ), fma(pp(in.Vz, q, S_VZ) - in.Vz[q - px], c.hrdy,
                                                (pp(in.Vy, q, S_VY) - in.Vy[q - pxy]) * c.hrdz),
                   pp(in.toa_yz, q, S_TYZ));
      else
        t_yz = fma(in.eb_yz[q], in.Vz[q] - in.Vz[q - px], fma(pp(in.em2_yz, q, S_EYZ), in.Vy[q] - in.Vy[q - pxy],
                                                              pp(in.toa_yz, q, S_TYZ)));
    }
    if (cell) {
      const T Pt = pp(in.Pt, q, S_PT), Pf = pp(in.Pf, q, S_PF), Pto = pp(in.Pto, q, S_PTO), Pfo = pp(in.Pfo, q, S_PFO);
      const T ph = pp(in.phi, q, S_PHI), ieta = pp(in.ieta, q, S_IETA);
      // k = K0 (phi / phi0)^3 (Eq. 23) at box index e with porosity p (recomputing forms)
      auto kperm = [&](T p, long long e) {
        const T r = p * c.rphi0;
        return (in.K0 ? in.K0[e] : c.k0) * r * r * r;
      };
      T w;
      if constexpr (RC) w = rcp_full(T(1.0) - ph);
      else w = in.w[q];
      const T vxl = pp(in.Vx, q, S_VX), vxr = in.Vx[q + 1], vyl = pp(in.Vy, q, S_VY), vyr = in.Vy[q + px];
      const T vzl = pp(in.Vz, q, S_VZ), vzr = in.Vz[q + pxy];
      const T gx = (vxr - vxl) * c.rdx, gy = (vyr - vyl) * c.rdy, gz = (vzr - vzl) * c.rdz;
      const T divV = gx + gy + gz;
      const T cc = c.compaction_on ? ieta * w : T(0);
      const T dPt = Pt - Pto, dPf = Pf - Pfo, dpp = Pt - Pf;
      // explicit fused multiply-adds: the same rounding in every kernel that inlines this body
      const T divVn = fma(dpp, cc, fma(-c.bd_rdt_a, dPf, fma(c.bd_rdt, dPt, divV)));
      // Darcy flux through the six faces (zero on the boundary) and the largest neighbour k
      T kc;
      if constexpr (!KS) kc = kperm(ph, q);
      else kc = pp(in.perm, q, S_K);
      T kmax = kc, sx = T(0), sy = T(0), sz = T(0);
      if (i > 0) {
        T kn;
        if constexpr (!KS) kn = kperm(in.phi[q - 1], q - 1);
        else kn = in.perm[q - 1];
        kmax = pos_max(kmax, kn);
        sx -= (kn + kc) * (Pf - in.Pf[q - 1]);
      }
      if (i < b.nx - 1) {
        T kn;
        if constexpr (!KS) kn = kperm(in.phi[q + 1], q + 1);
        else kn = in.perm[q + 1];
        kmax = pos_max(kmax, kn);
        sx += (kc + kn) * (in.Pf[q + 1] - Pf);
      }
      if (j > 0) {
        T kn;
        if constexpr (!KS) kn = kperm(in.phi[q - px], q - px);
        else kn = in.perm[q - px];
        kmax = pos_max(kmax, kn);
        sy -= (kn + kc) * (Pf - in.Pf[q - px]);
      }
      if (j < b.ny - 1) {
        T kn;
        if constexpr (!KS) kn = kperm(in.phi[q + px], q + px);
        else kn = in.perm[q + px];
        kmax = pos_max(kmax, kn);
        sy += (kc + kn) * (in.Pf[q + px] - Pf);
      }
      if (k > 0) {
        T kn;
        if constexpr (!KS) kn = kperm(in.phi[q - pxy], q - pxy);
        else kn = in.perm[q - pxy];
        kmax = pos_max(kmax, kn);
        sz -= (kn + kc) * ((Pf - in.Pf[q - pxy]) + c.buoy_dz);
      }
      if (k < b.nz - 1) {
        T kn;
        if constexpr (!KS) kn = kperm(in.phi[q + pxy], q + pxy);
        else kn = in.perm[q + pxy];
        kmax = pos_max(kmax, kn);
        sz += (kc + kn) * ((in.Pf[q + pxy] - Pf) + c.buoy_dz);
      }
      // div qD = -1/2 sum_d rd^2 [(k + k_r)(Pf_r - Pf) - (k_l + k)(Pf - Pf_l)]
      const T divqD = -(sx * c.hrdx2 + sy * c.hrdy2 + sz * c.hrdz2);
      // local-implicit pressure updates, Eqs. 17-18: P1 = P - res / (1/dtau + d res/dP), the
      // residuals being divVn (row Pt) and resF (row Pf)
      const T resF = fma(-dpp, cc, fma(-c.bd_rdt_a, dPt, fma(c.bda_B_rdt, dPf, divqD)));
      const T Pt1 = Pt - rcp_pseudo(pp(in.idtp, q, S_IDTP) + cc) * divVn;   // idtp holds 1/dtau_Pt + beta_d/dt
      const T Pf1 = Pf - rcp_pseudo(kmax * c.ifac_pf + c.bda_B_rdt + cc) * resF;
      // normal deviatoric stresses (Eq. 21): tau = tau_o xi/(1+xi) + 2 mu/(1+xi) (edot + beta_n divVn)
      const T s3 = fma(c.beta_n, divVn, -(divV * T(1.0 / 3.0)));
      const T cm2 = pp(in.cm2, q, S_CM2);
      const T sxx = fma(cm2, gx + s3, pp(in.toa_xx, q, S_TXX));
      const T syy = fma(cm2, gy + s3, pp(in.toa_yy, q, S_TYY));
      const T szz = fma(cm2, gz + s3, pp(in.toa_zz, q, S_TZZ));
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
      const T phio = pp(in.phio, q, S_PHIO);
      T Eo, iEo;
      if constexpr (RC) {
        Eo = T(1.0) - phio;
        iEo = T(0.0);   // not needed: 1/(1-phi) is recomputed from phi
      } else {
        Eo = in.Eo[q];
        iEo = in.iEo[q];
      }
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
      if constexpr (!RC) out.w[q] = iEo + iEo * em_n;
      if constexpr (KS) out.perm[q] = K0 * r * r * r;
      if (check) {
        r_pt = to_d(tabs(divVn));
        r_pf = to_d(tabs(resF));
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
  constexpr bool RC = LeanRecompute<T>::value;
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
      T dtv;
      if constexpr (RC) dtv = T(0.5) * (in.dtv_x[q - 1] + in.dtv_x[q]);
      else dtv = in.dtv_x[q];
      Vx1 = fma(dtv, Rx1, Vx[q]);
    }
    if (fy) {
      Fy = (in.txy[q + 1] - in.txy[q]) * c.rdx_r + (in.tyy[q] - in.tyy[q - px]) * c.rdy_r +
           (in.tyz[q + pxy] - in.tyz[q]) * c.rdz_r - (in.Pt1[q] - in.Pt1[q - px]) * c.rdy_r;
      Ry1 = fma(c.damp_y, Ry[q], Fy);
      T dtv;
      if constexpr (RC) dtv = T(0.5) * (in.dtv_y[q - px] + in.dtv_y[q]);
      else dtv = in.dtv_y[q];
      Vy1 = fma(dtv, Ry1, Vy[q]);
    }
    if (fz) {
      // buoyancy -(rho g - rho_BG g) averaged to the face, rho g - rho_BG g = (phi - phi0) drho_g
      const T rog = (T(0.5) * (in.phi[q - pxy] + in.phi[q]) - c.phi0) * c.drho_g_r;
      Fz = (in.txz[q + 1] - in.txz[q]) * c.rdx_r + (in.tyz[q + px] - in.tyz[q]) * c.rdy_r +
           (in.tzz[q] - in.tzz[q - pxy]) * c.rdz_r - (in.Pt1[q] - in.Pt1[q - pxy]) * c.rdz_r - rog;
      Rz1 = fma(c.damp_z, Rz[q], Fz);
      T dtv;
      if constexpr (RC) dtv = T(0.5) * (in.dtv_z[q - pxy] + in.dtv_z[q]);
      else dtv = in.dtv_z[q];
      Vz1 = fma(dtv, Rz1, Vz[q]);
    }
    if (fx) { Rx[q] = Rx1; Vx[q] = Vx1; }
    if (fy) { Ry[q] = Ry1; Vy[q] = Vy1; }
    if (fz) { Rz[q] = Rz1; Vz[q] = Vz1; }
    if (check) {
      if (fx && (mask & 1)) r_v = fmax(r_v, to_d(tabs(Fx)) * to_d(c.rho_i));
      if (fy && (mask & 2)) r_v = fmax(r_v, to_d(tabs(Fy)) * to_d(c.rho_i));
      if (fz && (mask & 4)) r_v = fmax(r_v, to_d(tabs(Fz)) * to_d(c.rho_i));
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
    const T axy = T(0.25) * (in.txy[q] + in.txy[q + 1] + in.txy[q + px] + in.txy[q + 1 + px]);
    const T axz = T(0.25) * (in.txz[q] + in.txz[q + 1] + in.txz[q + pxy] + in.txz[q + 1 + pxy]);
    const T ayz = T(0.25) * (in.tyz[q] + in.tyz[q + px] + in.tyz[q + pxy] + in.tyz[q + px + pxy]);
    const T sxx = in.txx[q], syy = in.tyy[q], szz = in.tzz[q];
    // tau_II^2 = (sxx^2 + syy^2 + szz^2) / 2 + axy^2 + axz^2 + ayz^2 (explicit FMAs: every form
    // that inlines this body rounds it alike)
    const T tII2 = fma(T(0.5), fma(sxx, sxx, fma(syy, syy, szz * szz)), fma(axy, axy, fma(axz, axz, ayz * ayz)));
    // Eq. 24: mu* = mu0 / (1 + (tau_II / tau0)^(n-1)); the log-space relaxation
    // exp(rel log mu* + (1 - rel) log mu) is written mu (mu* / mu)^rel (a square root for rel = 1/2)
    T den = T(1.0);
    if (c.powerlaw_on) {
      const T x2 = tII2 * c.rtau0_2;                               // (tau_II / tau0)^2
      const double p = c.n_pow - 1.0;
      den = p == 2.0 ? T(1.0) + x2 : from_d<T>(1.0 + exp(0.5 * p * log(to_d(x2))));
    }
    const T mu_old = mu[q], eta_old = eta[q];
    const T x_mu = tdiv(c.mu0, den * mu_old);                        // mu* / mu
    const T mu_new = mu_old * relax_pow(x_mu, c.rel_mu, c.root_mu);
    const T R = (in.Pf1[q] > in.Pt1[q]) ? c.R_weak : T(1.0);
    // Eq. 26: eta* = eta0 mu / phi R (with the relaxed mu), relaxed the same way
    const T x_eta = tdiv(c.eta0 * mu_new * R, in.phi1[q] * eta_old);
    m = to_d(tmax(tmax(x_mu, rcp_full(x_mu)), tmax(x_eta, rcp_full(x_eta))));
    if (!(x_mu == x_mu && x_eta == x_eta)) m = to_d(x_mu) + to_d(x_eta);   // NaN stays NaN (fmax drops it)
    mu[q] = mu_new;
    eta[q] = eta_old * relax_pow(x_eta, c.rel_eta, c.root_eta);
  }
}

// Mean shear viscosity over the centres next to the xy-edge q = (i, j, .) that lie inside the
// grid (four inside, two on a wall, one in a corner), in a fixed order (1/n exact: n = 1, 2, 4).
template <class T>
__device__ inline T lean_edge_mean_mu_xy(const Box& b, const T* mu, long long q, int i, int j) {
  T s = T(0.0);
  int n = 0;
  if (i > 0 && j > 0) { s += mu[q - 1 - b.px]; ++n; }
  if (i < b.nx && j > 0) { s += mu[q - b.px]; ++n; }
  if (i > 0 && j < b.ny) { s += mu[q - 1]; ++n; }
  if (i < b.nx && j < b.ny) { s += mu[q]; ++n; }
  return s * T(n == 4 ? 0.25 : (n == 2 ? 0.5 : 1.0));
}

// Coefficient refresh at box index (i, j, k).
template <class T>
__device__ __forceinline__ void lean_coef_point(const Box& b, const LeanCoef<T>& c, const LeanCoefIn<T>& in,
                                                const LeanCoefOut<T>& out, int i, int j, int k) {
  using namespace lean_detail;
  if (i > b.nx || j > b.ny || k > b.nz) return;
  const long long q = cidx(b, i, j, k);
  const long long px = b.px, pxy = b.pxy;
  constexpr bool RC = LeanRecompute<T>::value;
  const T rG = c.rGdtS;
  const T one = T(1.0), two = T(2.0);
  if (i < b.nx && j < b.ny && k < b.nz) {
    const T m = in.mu[q];
    const T s = rcp_full(fma(m, rG, one));
    const T a = one - s;                              // xi / (1 + xi)
    out.cm2[q] = two * m * s;
    out.toa_xx[q] = in.txxo[q] * a;
    out.toa_yy[q] = in.tyyo[q] * a;
    out.toa_zz[q] = in.tzzo[q] * a;
    out.idtp[q] = rcp_full(c.dtaupt_fac * m) + c.bd_rdt;   // 1/dtau_Pt + beta_d/dt
    out.ieta[q] = rcp_full(in.eta[q]);
  }
  if (k < b.nz && i > 0 && i < b.nx && j > 0 && j < b.ny) {
    const T m = T(0.25) * (in.mu[q - 1 - px] + in.mu[q - px] + in.mu[q - 1] + in.mu[q]);
    const T s = rcp_full(fma(m, rG, one));
    if constexpr (RC) {
      out.em2_xy[q] = two * m * s;
    } else {
      out.em2_xy[q] = two * m * s * c.hrdy;
      out.eb_xy[q] = two * m * s * c.hrdx;
    }
    // the background shear's stress 2 mu/(1+xi) tau_bg/(2 mu0) (Eqs. 32-33) joins the old-stress part
    out.toa_xy[q] = in.txyo[q] * (one - s) + two * m * s * c.ebg;
  } else if (k < b.nz && c.bg_on) {   // wall xy-edges carry the background stress
    const T m = lean_edge_mean_mu_xy(b, in.mu, q, i, j);
    const T s = rcp_full(fma(m, rG, one));
    out.toa_xy[q] = in.txyo[q] * (one - s) + two * m * s * c.ebg;
  }
  if (j < b.ny && i > 0 && i < b.nx && k > 0 && k < b.nz) {
    const T m = T(0.25) * (in.mu[q - 1 - pxy] + in.mu[q - pxy] + in.mu[q - 1] + in.mu[q]);
    const T s = rcp_full(fma(m, rG, one));
    if constexpr (RC) {
      out.em2_xz[q] = two * m * s;
    } else {
      out.em2_xz[q] = two * m * s * c.hrdz;
      out.eb_xz[q] = two * m * s * c.hrdx;
    }
    out.toa_xz[q] = in.txzo[q] * (one - s);
  }
  if (i < b.nx && j > 0 && j < b.ny && k > 0 && k < b.nz) {
    const T m = T(0.25) * (in.mu[q - px - pxy] + in.mu[q - pxy] + in.mu[q - px] + in.mu[q]);
    const T s = rcp_full(fma(m, rG, one));
    if constexpr (RC) {
      out.em2_yz[q] = two * m * s;
    } else {
      out.em2_yz[q] = two * m * s * c.hrdz;
      out.eb_yz[q] = two * m * s * c.hrdy;
    }
    out.toa_yz[q] = in.tyzo[q] * (one - s);
  }
  // pseudo-time steps of the velocities, mean of the two centres' dtau_V = fac / mu (the
  // recomputing forms store the centre values and average them in the faces kernel)
  if constexpr (RC) {
    if (i < b.nx && j < b.ny && k < b.nz) out.dtv_x[q] = c.dtauv_fac * rcp_full(in.mu[q]);
    return;
  }
  const T imu = (i < b.nx && j < b.ny && k < b.nz) ? rcp_full(in.mu[q]) : T(0.0);
  if (i > 0 && i < b.nx && j < b.ny && k < b.nz)
    out.dtv_x[q] = T(0.5) * c.dtauv_fac * (rcp_full(in.mu[q - 1]) + imu);
  if (j > 0 && j < b.ny && i < b.nx && k < b.nz)
    out.dtv_y[q] = T(0.5) * c.dtauv_fac * (rcp_full(in.mu[q - px]) + imu);
  if (k > 0 && k < b.nz && i < b.nx && j < b.ny)
    out.dtv_z[q] = T(0.5) * c.dtauv_fac * (rcp_full(in.mu[q - pxy]) + imu);
}

}  // namespace pt
