// rx.cuh — argument structs and launchers of the reactive porosity-wave kernels (rx_kernels.cu).
#pragma once

#include "pt_common.cuh"

namespace pt {

// Per-run scalars in the iteration type T (folded so the kernel multiplies).
template <class T>
struct RxCoef {
  T rdx, rdy, rdz;                       // 1/d
  T rhofg;                               // rho_f g (Darcy buoyancy)
  T rphi0, k0, reta;                     // 1/phi0, k0, 1/eta
  T beta_d, beta_s, beta_f;
  T beta_x, half_xs, xs_max, rtau;       // Xs_eq = clamp(beta_x Pf + half_xs, 0, xs_max); 1/tau
  T dt, rdt, dt_tau, r1dt_tau;           // dt, 1/dt, dt/tau, 1/(1 + dt/tau)
  T sr_opdx, opdx;                       // S_r (1 + dX), 1 + dX
  T pf_iscale;                           // 1 / pf_scale
  T rdx2, rdy2, rdz2;                    // 1/d^2 (Jacobi diagonal of the Darcy operator)
  T kc3;                                 // k0 / phi0^3: k = kc3 phi^3
  T rhofg_dz;                            // rho_f g dz (buoyancy as a pressure difference over a z face)
};

template <class T>
__device__ inline T rx_clamp(T v, T lo, T hi) { return v < lo ? lo : (v > hi ? hi : v); }
template <class T>
__device__ inline T rx_abs(T x) { return x < T(0) ? -x : x; }
// k = k0 (phi / phi0)^3
template <class T>
__device__ inline T rx_perm(const RxCoef<T>& c, T ph) {
  return c.kc3 * (ph * ph) * ph;
}
// beta_P = phi beta_f + beta_d - (1 + phi) beta_s
template <class T>
__device__ inline T rx_bp(const RxCoef<T>& c, T ph) {
  return ph * c.beta_f + c.beta_d - (T(1) + ph) * c.beta_s;
}
// 1 / x from the hardware's approximate reciprocal refined by Newton steps r' = r + r (1 - x r),
// each of which squares the relative error (FP64: ~2^-23 seed, rounding-limited after two). x is
// 1 - phi, 1 - Xs, beta_P or a Jacobi denominator here: positive and far inside the normal range.
// FP32 takes the fast reciprocal-multiply intrinsic (2 ulp).
__device__ inline double rx_rcp(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  r = fma(r, fma(-x, r, 1.0), r);
  return fma(r, fma(-x, r, 1.0), r);
}
__device__ inline float rx_rcp(float x) { return __fdividef(1.0f, x); }
// max of the three one-iteration changes; NaN if any is (fmax alone would drop it)
__device__ inline double rx_change(double d_phi, double d_pf, double d_xs) {
  const double s = d_phi + d_pf + d_xs;
  return s != s ? s : fmax(d_phi, fmax(d_pf, d_xs));
}

template <class T>
struct RxIn {
  const T *Pf, *phi, *Xs, *Pf_o, *phi_o, *Xs_o;
  const T* k;                            // k(phi) of the iterate (plain FP64 iteration; else null)
};
template <class T>
struct RxOut {
  T *Pf, *phi, *Xs, *R;                  // R written when non-null
  T* k;                                  // k(phi') for the next iteration (plain FP64 iteration)
};

// One PT iteration over the cells with pseudo step dtau; check: change norm into red[RED_V]
// and max k/beta_P of the new porosity into red[RED_MUMAX].
template <class T>
void rx_iter(cudaStream_t s, Box b, const RxCoef<T>& c, double dtau, const RxIn<T>& in, const RxOut<T>& out,
             unsigned long long* red, int check);
// max k / beta_P over the cells into red[RED_MUMAX]
template <class T>
void rx_kbmax(cudaStream_t s, Box b, const RxCoef<T>& c, const T* phi, unsigned long long* red);
// caller FP64 fields -> iterate and old-step arrays in T (start of a step); k1 (may be null):
// k(phi) of the iterate
template <class T>
void rx_begin(cudaStream_t s, Box b, const RxCoef<T>& c, const double* Pf, const double* phi, const double* Xs,
              T* Pf1, T* phi1, T* Xs1, T* Pf_o, T* phi_o, T* Xs_o, T* k1);
// iterate (and rate) in T -> caller FP64 fields (end of a step)
template <class T>
void rx_end(cudaStream_t s, Box b, const T* Pf, const T* phi, const T* Xs, const T* R, double* Pf1, double* phi1,
            double* Xs1, double* R1);

// ---- geometric multigrid (FAS V-cycle) of the implicit step: rx_mg_kernels.cu ----

// FAS sources of a coarse level (unused on the finest)
template <class T>
struct MgSrc {
  const T *fP, *fphi, *fX;
};
// What the restriction writes on the coarse level: the restricted iterate (twice: the
// iterate the coarse sweeps start from and the copy u0 the correction is measured against)
// and the restricted residual in the FAS source slots.
template <class T>
struct MgCoarse {
  T *Pf, *phi, *Xs, *Pf0, *phi0, *Xs0, *fP, *fphi, *fX;
};
// The coarse correction e = u - u0, written by the coarse level's last sweep over u0
template <class T>
struct MgE {
  T *Pf, *phi, *Xs;
};
template <class T>
struct MgCorr {
  const T *Pf, *phi, *Xs;
};

// One weighted-Jacobi sweep (the PT iteration with local pseudo steps); fas: add the FAS
// sources; laste (coarse levels, with fas): write e = u' - u0 over u0 instead of u' to out;
// check: change norm into red[RED_V]; out.R written when non-null.
template <class T>
void mg_smooth(cudaStream_t s, Box b, const RxCoef<T>& c, double omega, const RxIn<T>& in, const MgSrc<T>* fas,
               const RxOut<T>& out, const MgE<T>* laste, unsigned long long* red, int check);
// fine residual and iterate -> coarse iterate, u0 and (restricted residual) sources
template <class T>
void mg_restrict(cudaStream_t s, Box fine, Box coarse, const RxCoef<T>& c, const RxIn<T>& in, const MgSrc<T>* fas,
                 const MgCoarse<T>& out);
// coarse sources f -= g(u0) (the FAS right-hand side)
template <class T>
void mg_coarse_rhs(cudaStream_t s, Box coarse, const RxCoef<T>& c, const RxIn<T>& u0, const MgCoarse<T>& out);
// fine iterate += trilinear interpolation of the coarse correction e; phi kept in [1e-4, 1]
template <class T>
void mg_prolong(cudaStream_t s, Box fine, Box coarse, const MgCorr<T>& e, T* Pf, T* phi, T* Xs);
// old-step fields: 8-child means
template <class T>
void mg_restrict_old(cudaStream_t s, Box fine, Box coarse, const T* Pf_o, const T* phi_o, const T* Xs_o, T* cPf_o,
                     T* cphi_o, T* cXs_o);

}  // namespace pt
