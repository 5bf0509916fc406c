// pt_kernels.cuh — argument structs and declarations of the solver's kernels (defined in
// pt_ref_kernels.cu), launched by the host API in pt_api.cu.
#pragma once

#include "pt_common.cuh"

namespace pt {

struct CentreIn {
  const double *Vx, *Vy, *Vz, *Pt, *Pf, *phi, *mu, *eta, *perm, *Pto, *Pfo, *txxo, *tyyo, *tzzo;
};
struct CentreOut {
  double *Pt1, *Pf1, *txx, *tyy, *tzz;
};
struct EdgeIn {
  const double *Vx, *Vy, *Vz, *mu, *txyo, *txzo, *tyzo;
};
struct EdgeOut {
  double *txy, *txz, *tyz;
};
struct FaceIn {
  const double *txx, *tyy, *tzz, *txy, *txz, *tyz, *Pt1, *rog, *mu;
};
struct PicardIn {
  const double *txx, *tyy, *tzz, *txy, *txz, *tyz, *phi1, *Pt1, *Pf1;
};

__global__ void k_perm(Box b, Coef c, const double* __restrict__ phi, const double* __restrict__ logk,
                       double* __restrict__ perm, double* __restrict__ rog);
__global__ void k_centres(Box b, Coef c, CentreIn in, CentreOut out, int update,
                          unsigned long long* red, int check);
__global__ void k_edges(Box b, Coef c, EdgeIn in, EdgeOut out);
__global__ void k_porosity(Box b, Coef c, const double* __restrict__ Vx, const double* __restrict__ Vy,
                           const double* __restrict__ Vz, const double* __restrict__ phi,
                           const double* __restrict__ Pt1, const double* __restrict__ Pf1,
                           const double* __restrict__ Pto, const double* __restrict__ Pfo,
                           const double* __restrict__ Lo, const double* __restrict__ eta,
                           double* __restrict__ phi1);
__global__ void k_faces(Box b, Coef c, FaceIn in, double* __restrict__ Vx, double* __restrict__ Vy,
                        double* __restrict__ Vz, double* __restrict__ Rx, double* __restrict__ Ry,
                        double* __restrict__ Rz, unsigned long long* red, int check);
__global__ void k_picard(Box b, Coef c, PicardIn in, double* __restrict__ mu, double* __restrict__ eta,
                         unsigned long long* red, int update);
__global__ void k_begin_step(Box b, const double* __restrict__ Pt, const double* __restrict__ Pf,
                             const double* __restrict__ phi, const double* __restrict__ mu,
                             double* __restrict__ Pto, double* __restrict__ Pfo, double* __restrict__ Lo,
                             unsigned long long* red);
__global__ void k_init_visc(Box b, Coef c, const double* __restrict__ phi, double* __restrict__ mu,
                            double* __restrict__ eta);
__global__ void k_residual_faces(Box b, Coef c, FaceIn in, unsigned long long* red);

}  // namespace pt
