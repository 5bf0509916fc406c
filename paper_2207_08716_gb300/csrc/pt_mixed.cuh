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
  float *r_pt, *r_pf, *cc, *perm, *idtp, *iden_pt, *idtf, *iden_pf;
};
struct MixFaceIn {
  const double *txx, *tyy, *tzz, *txy, *txz, *tyz, *Pt, *phi;
};
struct MixCoefOut {
  float *cm2, *em2_xy, *em2_xz, *em2_yz;                    // 2 mu / (1 + xi) at centres and edges
  float *dtv_x, *dtv_y, *dtv_z;                             // velocity pseudo-steps at faces
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
};
// FP32 PT iteration on the correction: current correction and frozen coefficients.
template <class T>
struct CorrIn {
  const T *Vx, *Vy, *Vz, *Pt, *Pf;                 // current correction dV, dPt, dPf
  const T *cc, *perm, *idtp, *iden_pt, *idtf, *iden_pf, *r_pt, *r_pf, *cm2, *em2_xy, *em2_xz, *em2_yz;
};
template <class T>
struct CorrCellOut {
  T *Pt, *Pf, *txx, *tyy, *tzz, *txy, *txz, *tyz;  // next dPt, dPf; stresses of the correction
};
template <class T>
struct CorrFaceIn {
  const T *txx, *tyy, *tzz, *txy, *txz, *tyz, *Pt1, *dtv_x, *dtv_y, *dtv_z, *rfx, *rfy, *rfz;
};

void mix_prepare(dim3 g, dim3 bl, cudaStream_t s, Box b, const Coef& c, const MixPrepIn& in,
                 const MixPrepOut& out, unsigned long long* red);
void mix_res_faces(dim3 g, dim3 bl, cudaStream_t s, Box b, const Coef& c, const MixFaceIn& in, float* rfx,
                   float* rfy, float* rfz, unsigned long long* red);
void mix_coef(dim3 g, dim3 bl, cudaStream_t s, Box b, const Coef& c, const double* mu, const MixCoefOut& out);
void mix_update(dim3 g, dim3 bl, cudaStream_t s, Box b, const MixUpdate& u);
template <class T>
void corr_cells(dim3 g, dim3 bl, cudaStream_t s, Box b, const CorrCoef<T>& c, const CorrIn<T>& in,
                const CorrCellOut<T>& out, unsigned long long* red, int check);
template <class T>
void corr_faces(dim3 g, dim3 bl, cudaStream_t s, Box b, const CorrCoef<T>& c, const CorrFaceIn<T>& in, T* Vx,
                T* Vy, T* Vz, T* Rx, T* Ry, T* Rz, unsigned long long* red, int check);

}  // namespace pt
