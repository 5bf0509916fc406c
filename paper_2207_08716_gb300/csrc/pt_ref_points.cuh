// pt_ref_points.cuh — per-point bodies of three step-by-step kernels that the FP32
// defect-correction loop also runs, one instance at a time (pt_ref_kernels.cu) and in the
// batched FP32 engine (pt_mixed_kernels.cu): the same inlined code in both, so a batched
// member reproduces its single-instance run to rounding.
//   perm_point      k = k0 e^logk (phi/phi0)^3 (Eq. 23), rho g - rho_BG g (Eq. 27)
//   edges_point     shear stresses on the three lower edges of (i, j, k) (Eq. 21), zero on
//                   boundary edges unless a background shear is applied (Eqs. 32-33)
//   porosity_point  phi^{k+1} = 1 - exp(L), L from Eq. 22 in log(1 - phi) form
#pragma once

#include "pt_kernels.cuh"
#include "pt_lean_body.cuh"

namespace pt {

// a / b: the IEEE quotient (FAST = false, the step-by-step form), or a times the two-step Newton
// reciprocal of the hardware's approximate one (within an ulp; the FP32 form's outer phases,
// which need far less and run on the FP64 pipe)
template <bool FAST>
__device__ __forceinline__ double ref_div(double a, double b) {
  if constexpr (FAST) return a * lean_detail::rcp_full(b);
  else return a / b;
}

__device__ __forceinline__ void perm_point(const Box& b, const Coef& c, const double* __restrict__ phi,
                                           const double* __restrict__ logk, double* __restrict__ perm,
                                           double* __restrict__ rog, int i, int j, int k) {
  if (i >= b.nx || j >= b.ny || k >= b.nz) return;
  const long long q = cidx(b, i, j, k);
  const double ph = phi[q];
  const double r = ph * c.rphi0;
  // without a log k field the factor e^0 is 1 exactly: no exponential evaluated
  perm[q] = c.k0 * (logk ? exp(logk[q]) : 1.0) * r * r * r;
  rog[q] = (ph * c.rhof_g + (1.0 - ph) * c.rhos_g) - c.rho_bg_g;
}

template <bool FAST = false>
__device__ __forceinline__ void edges_point(const Box& b, const Coef& c, const EdgeIn& in, const EdgeOut& out,
                                            int i, int j, int k) {
  if (i > b.nx || j > b.ny || k > b.nz) return;
  const long long q = cidx(b, i, j, k);
  const long long px = b.px, pxy = b.pxy;
  if (k < b.nz) {  // xy-edge (i, j, k); the background shear adds ebg to the strain rate
    double t = 0.0;
    if (i > 0 && i < b.nx && j > 0 && j < b.ny) {
      const double m = 0.25 * (in.mu[q - 1 - px] + in.mu[q - px] + in.mu[q - 1] + in.mu[q]);
      const double xi = m * c.rGdtS;
      const double e = 0.5 * ((in.Vx[q] - in.Vx[q - px]) * c.rdy + (in.Vy[q] - in.Vy[q - 1]) * c.rdx) + c.ebg;
      t = ref_div<FAST>(in.txyo[q] * xi + 2.0 * m * e, 1.0 + xi);
    } else if (c.bg_on) {   // wall edge: background part only
      const double m = edge_mean_mu_xy(b, in.mu, q, i, j);
      const double xi = m * c.rGdtS;
      t = ref_div<FAST>(in.txyo[q] * xi + 2.0 * m * c.ebg, 1.0 + xi);
    }
    out.txy[q] = t;
  }
  if (j < b.ny) {  // xz-edge (i, j, k)
    double t = 0.0;
    if (i > 0 && i < b.nx && k > 0 && k < b.nz) {
      const double m = 0.25 * (in.mu[q - 1 - pxy] + in.mu[q - pxy] + in.mu[q - 1] + in.mu[q]);
      const double xi = m * c.rGdtS;
      const double e = 0.5 * ((in.Vx[q] - in.Vx[q - pxy]) * c.rdz + (in.Vz[q] - in.Vz[q - 1]) * c.rdx);
      t = ref_div<FAST>(in.txzo[q] * xi + 2.0 * m * e, 1.0 + xi);
    }
    out.txz[q] = t;
  }
  if (i < b.nx) {  // yz-edge (i, j, k)
    double t = 0.0;
    if (j > 0 && j < b.ny && k > 0 && k < b.nz) {
      const double m = 0.25 * (in.mu[q - px - pxy] + in.mu[q - pxy] + in.mu[q - px] + in.mu[q]);
      const double xi = m * c.rGdtS;
      const double e = 0.5 * ((in.Vy[q] - in.Vy[q - pxy]) * c.rdz + (in.Vz[q] - in.Vz[q - px]) * c.rdy);
      t = ref_div<FAST>(in.tyzo[q] * xi + 2.0 * m * e, 1.0 + xi);
    }
    out.tyz[q] = t;
  }
}

// phi^{k+1} = 1 - exp(L),  L = Lo - dt [beta_phi ((Pf1 - Pfo) - (Pt1 - Pto)) / dt
//                                       + (Pf1 - Pt1) / eta + V . grad(1 - phi) / (1 - phi)]
template <bool FAST = false>
__device__ __forceinline__ void porosity_point(const Box& b, const Coef& c, const double* __restrict__ Vx,
                                               const double* __restrict__ Vy, const double* __restrict__ Vz,
                                               const double* __restrict__ phi, const double* __restrict__ Pt1,
                                               const double* __restrict__ Pf1, const double* __restrict__ Pto,
                                               const double* __restrict__ Pfo, const double* __restrict__ Lo,
                                               const double* __restrict__ eta, double* __restrict__ phi1, int i,
                                               int j, int k) {
  if (i >= b.nx || j >= b.ny || k >= b.nz) return;
  const long long q = cidx(b, i, j, k);
  const double omc = 1.0 - phi[q];
  double ax = 0.0, ay = 0.0, az = 0.0;
  if (i > 0) ax += Vx[q] * (omc - (1.0 - phi[q - 1])) * c.rdx;
  if (i < b.nx - 1) ax += Vx[q + 1] * ((1.0 - phi[q + 1]) - omc) * c.rdx;
  if (j > 0) ay += Vy[q] * (omc - (1.0 - phi[q - b.px])) * c.rdy;
  if (j < b.ny - 1) ay += Vy[q + b.px] * ((1.0 - phi[q + b.px]) - omc) * c.rdy;
  if (k > 0) az += Vz[q] * (omc - (1.0 - phi[q - b.pxy])) * c.rdz;
  if (k < b.nz - 1) az += Vz[q + b.pxy] * ((1.0 - phi[q + b.pxy]) - omc) * c.rdz;
  const double adv = ref_div<FAST>(0.5 * (ax + ay + az), omc);
  const double pt1 = Pt1[q], pf1 = Pf1[q];
  const double comp = c.compaction_on ? ref_div<FAST>(pf1 - pt1, eta[q]) : 0.0;
  const double L = Lo[q] - c.dt * (c.beta_phi * ((pf1 - Pfo[q]) - (pt1 - Pto[q])) * c.rdt + comp + adv);
  phi1[q] = 1.0 - exp(L);
}

}  // namespace pt
