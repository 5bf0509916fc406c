// pt_lean.cuh — argument structs and declarations of the FP64-lean PT kernels
// (pt_lean_kernels.cu). T is the field and arithmetic type: double (PT_FP64) or the
// double-float df64 (PT_DF64).
#pragma once

#include "df64.cuh"
#include "pt_common.cuh"

namespace pt {

// Per-step scalars in the field type, pre-folded so each kernel multiplies instead of divides.
template <class T>
struct LeanCoef {
  T rdx, rdy, rdz;              // 1 / dx
  T hrdx, hrdy, hrdz;           // 1 / (2 dx)
  T hrdx2, hrdy2, hrdz2;        // 1 / (2 dx^2)
  T buoy_dz;                    // (rho_f - rho_BG) g dz
  T bd_rdt, bda_B_rdt;          // beta_d / dt, beta_d alpha / (B dt)
  T alpha, alpha_B;             // alpha, alpha / B
  T bd_rdt_a;                   // beta_d alpha / dt
  T beta_n, beta_phi, dt;
  T rphi0, k0, phi0, drho_g;    // 1 / phi0, k0, phi0, (rho_f - rho_s) g
  T ifac_pf;                    // 1 / (cfl_pf h^2 (1 + beta_d B / alpha)): 1/dtau_Pf = kmax * ifac_pf
  T rrho_i, damp_x, damp_y, damp_z;
  T rdx_r, rdy_r, rdz_r, drho_g_r;  // 1/(d rho_i), (rho_f - rho_s) g / rho_i: the momentum residual over rho_i
  T rho_i;
  int compaction_on, powerlaw_on;
  T ebg;                        // background xy strain rate tau_bg / (2 mu0) (Eqs. 32-33)
  int bg_on;                    // tau_bg != 0: wall xy-edges carry the background stress
  // Picard update and coefficient refresh
  T mu0, eta0, R_weak;
  T rtau0_2;                    // 1 / tau0^2
  T rGdtS, dtaupt_fac, dtauv_fac;
  double tau0, n_pow, rel_mu, rel_eta;
  int root_mu, root_eta;        // m when rel = 1/m (2 <= m <= 64), else 0 (double-float roots)
};

template <class T>
struct LeanCellIn {
  const T *Vx, *Vy, *Vz, *Pt, *Pf, *phi, *w, *perm;
  const T *Pto, *Pfo, *phio, *Eo, *iEo;
  const T *ieta, *idtp, *cm2, *toa_xx, *toa_yy, *toa_zz;   // idtp holds 1/dtau_Pt + beta_d/dt
  // edge moduli 2 mu/(1+xi) pre-multiplied by the two half inverse spacings of each edge's strain
  // rate: em2_xy = m hrdy, eb_xy = m hrdx; em2_xz = m hrdz, eb_xz = m hrdx; em2_yz = m hrdz, eb_yz = m hrdy
  const T *em2_xy, *em2_xz, *em2_yz, *eb_xy, *eb_xz, *eb_yz, *toa_xy, *toa_xz, *toa_yz;
  const T *K0;  // k0 e^logk per cell, or null (scalar k0)
};
template <class T>
struct LeanCellOut {
  T *Pt, *Pf, *phi, *w, *perm, *txx, *tyy, *tzz, *txy, *txz, *tyz;
};
template <class T>
struct LeanFaceIn {
  const T *txx, *tyy, *tzz, *txy, *txz, *tyz, *Pt1, *phi, *dtv_x, *dtv_y, *dtv_z;
};
template <class T>
struct LeanPicardIn {
  const T *txx, *tyy, *tzz, *txy, *txz, *tyz, *phi1, *Pt1, *Pf1;
};
template <class T>
struct LeanCoefIn {
  const T *mu, *eta;
  const T *txxo, *tyyo, *tzzo, *txyo, *txzo, *tyzo;
};
template <class T>
struct LeanCoefOut {
  T *cm2, *toa_xx, *toa_yy, *toa_zz, *idtp, *ieta;
  T *em2_xy, *em2_xz, *em2_yz, *eb_xy, *eb_xz, *eb_yz, *toa_xy, *toa_xz, *toa_yz;
  T *dtv_x, *dtv_y, *dtv_z;
};
template <class T>
struct LeanBeginIn {
  const T *Pt, *Pf, *phi, *mu, *K0;
};
template <class T>
struct LeanBeginOut {
  T *Pto, *Pfo, *phio, *Eo, *iEo, *w, *perm;
};

// Host-side launchers (the kernels are templates and are launched from their own TU).
template <class T>
void lean_cells(dim3 gr, dim3 bl, cudaStream_t st, Box b, const LeanCoef<T>& c, const LeanCellIn<T>& in,
                const LeanCellOut<T>& out, unsigned long long* red, int check);
template <class T>
void lean_faces(dim3 gr, dim3 bl, cudaStream_t st, Box b, const LeanCoef<T>& c, const LeanFaceIn<T>& in,
                T* Vx, T* Vy, T* Vz, T* Rx, T* Ry, T* Rz, unsigned long long* red, int check);
template <class T>
void lean_picard(dim3 gr, dim3 bl, cudaStream_t st, Box b, const LeanCoef<T>& c, const LeanPicardIn<T>& in,
                 T* mu, T* eta, unsigned long long* red);
template <class T>
void lean_coef(dim3 gr, dim3 bl, cudaStream_t st, Box b, const LeanCoef<T>& c, const LeanCoefIn<T>& in,
               const LeanCoefOut<T>& out);
template <class T>
void lean_begin(dim3 gr, dim3 bl, cudaStream_t st, Box b, const LeanCoef<T>& c, const LeanBeginIn<T>& in,
                const LeanBeginOut<T>& out, unsigned long long* red);
template <class T>
void lean_k0(dim3 gr, dim3 bl, cudaStream_t st, Box b, double k0, const double* logk, T* K0);

// Up to 16 arrays converted in one launch between FP64 (d) and double-float (f), whole boxes.
struct DfCopy {
  double* d[16];
  df64* f[16];
};
void df64_convert(cudaStream_t st, const DfCopy& cp, int narrays, long long n, bool to_df);

// Element-wise application of one device math routine (pt_math_check; codes in porowave_pt.h).
enum { MATH_RCP_PSEUDO = 0, MATH_RCP_FULL = 1, MATH_EXPM1_POS = 2, MATH_EXPM1_NEG = 3, MATH_DF_ADD = 4,
       MATH_DF_SUB = 5, MATH_DF_MUL = 6, MATH_DF_FMA = 7, MATH_DF_RCP = 8, MATH_DF_SQRT = 9,
       MATH_DF_ROOT = 10, MATH_DF_EXPM1_POS = 11, MATH_DF_EXPM1_NEG = 12, MATH_COUNT = 13 };
void math_check(cudaStream_t st, int fn, const double* a, const double* b, double* out, long long n);

}  // namespace pt
