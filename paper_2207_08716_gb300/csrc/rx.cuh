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
};

template <class T>
struct RxIn {
  const T *Pf, *phi, *Xs, *Pf_o, *phi_o, *Xs_o;
};
template <class T>
struct RxOut {
  T *Pf, *phi, *Xs, *R;                  // R written when non-null
};

// One PT iteration over the cells with pseudo step dtau; check: change norm into red[RED_V]
// and max k/beta_P of the new porosity into red[RED_MUMAX].
template <class T>
void rx_iter(cudaStream_t s, Box b, const RxCoef<T>& c, double dtau, const RxIn<T>& in, const RxOut<T>& out,
             unsigned long long* red, int check);
// max k / beta_P over the cells into red[RED_MUMAX]
template <class T>
void rx_kbmax(cudaStream_t s, Box b, const RxCoef<T>& c, const T* phi, unsigned long long* red);
// caller FP64 fields -> iterate and old-step arrays in T (start of a step)
template <class T>
void rx_begin(cudaStream_t s, Box b, const double* Pf, const double* phi, const double* Xs, T* Pf1, T* phi1, T* Xs1,
              T* Pf_o, T* phi_o, T* Xs_o);
// iterate (and rate) in T -> caller FP64 fields (end of a step)
template <class T>
void rx_end(cudaStream_t s, Box b, const T* Pf, const T* phi, const T* Xs, const T* R, double* Pf1, double* phi1,
            double* Xs1, double* R1);

}  // namespace pt
