// pt_mixed.cuh — argument structs and host launchers of the mixed-precision (PT_FP32) kernels
// in pt_mixed_kernels.cu.
#pragma once

#include "pt_common.cuh"

namespace pt {

struct MixPrepIn {
  const double *Vx, *Vy, *Vz, *Pt, *Pf, *phi, *mu, *eta, *perm, *Pto, *Pfo, *txxo, *tyyo, *tzzo;
};
struct MixPrepOut {
  double *txx, *tyy, *tzz;                                  // FP64 stresses at u
  float *r_pt, *r_pf, *cc, *perm, *iden_pt, *iden_pf;
};
struct MixFaceIn {
  const double *txx, *tyy, *tzz, *txy, *txz, *tyz, *Pt, *phi;
};
struct MixCoefOut {
  float *mu;                                                // FP32 copy of the Picard-updated mu
};
struct MixUpdate {
  double *Vx, *Vy, *Vz, *Pt, *Pf;
  const float *dVx, *dVy, *dVz, *dPt, *dPf;
};

template <class T>
struct CorrCoef {
  T rdx, rdy, rdz, hrdx, hrdy, hrdz, hrdx2, hrdy2, hrdz2;
  T bd_rdt, bd_rdt_a, bda_B_rdt, beta_n, rrho_i, damp_x, damp_y, damp_z;
  T rG;                                            // 1 / (G dtS): xi = mu rG
  T hdtv;                                          // dtau_V at a face = hdtv (1/mu_l + 1/mu_r)
};
// One FP32 PT iteration on the correction reads the current correction and the frozen
// coefficients and writes the next correction (ping-pong); R is updated in place.
template <class T>
struct CorrIn {
  const T *Vx, *Vy, *Vz, *Pt, *Pf;                 // current correction dV, dPt, dPf
  const T *cc, *perm, *iden_pt, *iden_pf, *r_pt, *r_pf, *mu, *rfx, *rfy, *rfz;
};
template <class T>
struct CorrOut {
  T *Vx, *Vy, *Vz, *Pt, *Pf;                       // next correction
};

void mix_prepare(dim3 g, dim3 bl, cudaStream_t s, Box b, const Coef& c, const MixPrepIn& in,
                 const MixPrepOut& out, unsigned long long* red);
void mix_res_faces(dim3 g, dim3 bl, cudaStream_t s, Box b, const Coef& c, const MixFaceIn& in, float* rfx,
                   float* rfy, float* rfz, unsigned long long* red);
void mix_coef(dim3 g, dim3 bl, cudaStream_t s, Box b, const Coef& c, const double* mu, const MixCoefOut& out);
void mix_update(dim3 g, dim3 bl, cudaStream_t s, Box b, const MixUpdate& u);
template <class T>
void corr_iter(dim3 g, dim3 bl, cudaStream_t s, Box b, const CorrCoef<T>& c, const CorrIn<T>& in,
               const CorrOut<T>& out, T* Rx, T* Ry, T* Rz, unsigned long long* red, int check);

}  // namespace pt
