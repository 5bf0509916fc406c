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
  float *r_pt, *r_pf, *cc, *perm, *idtp;
};
struct MixFaceIn {
  const double *txx, *tyy, *tzz, *txy, *txz, *tyz, *Pt, *phi;
};
struct MixCoefOut {
  float *mu;                                                // mu at centres (FP32)
  float *dtvc;                                              // velocity pseudo-step fac / mu at centres
};
struct MixUpdate {
  double *Vx, *Vy, *Vz, *Pt, *Pf;
  const float *dVx, *dVy, *dVz, *dPt, *dPf;
  double omega;             // u <- u + omega delta
};

template <class T>
struct CorrCoef {
  T rdx, rdy, rdz, hrdx, hrdy, hrdz, hrdx2, hrdy2, hrdz2;
  T bd_rdt, bd_rdt_a, bda_B_rdt, beta_n, rrho_i, damp_x, damp_y, damp_z;
  T rG;         // 1 / (G dtS): xi = mu rG
  T ifac_pf;    // 1 / dtau_Pf = kmax ifac_pf
};
// One FP32 PT iteration on the correction, in one pass: the current correction (dV, dPt, dPf),
// the frozen coefficients and right-hand sides, and where the next correction goes.
template <class T>
struct CorrIn {
  const T *Vx, *Vy, *Vz, *Pt, *Pf;                 // current correction dV, dPt, dPf
  const T *cc, *perm, *idtp, *r_pt, *r_pf, *mu, *dtvc, *rfx, *rfy, *rfz;
};
template <class T>
struct CorrOut {
  T *Vx, *Vy, *Vz, *Pt, *Pf;                       // next dV, dPt, dPf (other buffers)
  T *Rx, *Ry, *Rz;                                 // damped residuals (in place)
};

void mix_prepare(dim3 g, dim3 bl, cudaStream_t s, Box b, const Coef& c, const MixPrepIn& in,
                 const MixPrepOut& out, unsigned long long* red);
void mix_res_faces(dim3 g, dim3 bl, cudaStream_t s, Box b, const Coef& c, const MixFaceIn& in, float* rfx,
                   float* rfy, float* rfz, unsigned long long* red);
void mix_coef(dim3 g, dim3 bl, cudaStream_t s, Box b, const Coef& c, const double* mu, const MixCoefOut& out);
void mix_update(dim3 g, dim3 bl, cudaStream_t s, Box b, const MixUpdate& u);
// One fused FP32 correction iteration over the whole grid (z-marching tiles, see the kernel).
void corr_iteration(cudaStream_t s, Box b, const CorrCoef<float>& c, const CorrIn<float>& in,
                    const CorrOut<float>& out, unsigned long long* red, int check);

}  // namespace pt
