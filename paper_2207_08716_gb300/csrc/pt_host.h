// pt_host.h — host-side helpers shared by every entry point of the porosity-wave PT library:
// argument rules for grids, the padded box, and the per-step scalars of Eqs. 17-27 built from
// the caller's parameter structs. One definition, so the context path (pt_init / pt_step /
// pt_residual) and the allocation-free residual path cannot drift apart.
#pragma once

#include <cmath>
#include <cstdint>
#include <cstring>

#include "../../include/porowave_pt.h"
#include "pt_common.cuh"

namespace pt {

constexpr int kPitchMultiple = 16;

// Grid sizes and extents the library accepts: at least one cell per direction, nx and ny below
// 2^20 (so every padded-box index fits the kernels' arithmetic), nz below the grid's z limit,
// positive finite extents.
inline bool grid_ok(const pt_grid* g) {
  return g && g->nx >= 1 && g->ny >= 1 && g->nz >= 1 && g->nx < (1 << 20) && g->ny < (1 << 20) &&
         g->nz < 65535 && g->lx > 0 && g->ly > 0 && g->lz > 0 && std::isfinite(g->lx) &&
         std::isfinite(g->ly) && std::isfinite(g->lz);
}

// Padded box of a grid accepted by grid_ok (64-bit arithmetic throughout).
inline Box make_box(const pt_grid* g) {
  Box b;
  b.nx = g->nx;
  b.ny = g->ny;
  b.nz = g->nz;
  const long long px = ((long long)g->nx + 1 + kPitchMultiple - 1) / kPitchMultiple * kPitchMultiple;
  b.px = (int)px;
  b.pxy = px * ((long long)g->ny + 1);
  b.n = b.pxy * ((long long)g->nz + 1);
  return b;
}

inline bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// Physical parameters the library accepts (positive moduli, viscosities, permeability,
// porosity in (0, 1), finite background shear).
inline bool phys_ok(const pt_phys* p) {
  return p && p->phi0 > 0 && p->phi0 < 1 && p->k0 > 0 && p->mu0 > 0 && p->eta0 > 0 && p->G > 0 &&
         p->alpha > 0 && p->B > 0 && p->tau0 > 0 && p->R_weak > 0 && std::isfinite(p->tau_bg);
}

// Per-step scalars from the grid whose spacing (and nz) define them, the physical and numerical
// parameters and the stress sub-step dtS (xi = mu / (G dtS), Eq. 21; dtS <= 0 leaves 1/(G dtS)
// at zero until the first step sets it).
inline Coef make_coef(const pt_grid& g, const pt_phys& p, const pt_num& n, double dtS) {
  Coef k;
  std::memset(&k, 0, sizeof k);
  const double dx = g.lx / g.nx, dy = g.ly / g.ny, dz = g.lz / g.nz;
  const double h = std::fmin(dx, std::fmin(dy, dz));
  k.rdx = 1.0 / dx;
  k.rdy = 1.0 / dy;
  k.rdz = 1.0 / dz;
  k.h2 = h * h;
  k.phi0 = p.phi0;
  k.rphi0 = 1.0 / p.phi0;
  k.k0 = p.k0;
  k.mu0 = p.mu0;
  k.eta0 = p.eta0;
  k.R_weak = p.R_weak;
  k.n_pow = p.n_pow;
  k.tau0 = p.tau0;
  k.alpha = p.alpha;
  k.B = p.B;
  k.beta_d = p.beta_d;
  k.beta_phi = p.beta_phi;
  k.G = p.G;
  k.rhof_g = p.rhof_g;
  k.rhos_g = p.rhos_g;
  k.rho_bg_g = p.phi0 * p.rhof_g + (1.0 - p.phi0) * p.rhos_g;   // Eq. 27 background density
  k.powerlaw_on = p.powerlaw_on;
  k.compaction_on = p.compaction_on;
  k.dt = n.dt;
  k.rdt = 1.0 / n.dt;
  k.damp_x = n.damp[0];
  k.damp_y = n.damp[1];
  k.damp_z = n.damp[2];
  k.rho_i = n.rho_i;
  k.rrho_i = 1.0 / n.rho_i;
  k.beta_n = n.beta_n;
  k.rel_mu = n.rel_mu;
  k.rel_eta = n.rel_eta;
  k.dtauv_fac = n.cfl_v * k.h2 * n.rho_i / (1.0 + n.beta_n);
  k.dtaupt_fac = n.dtpt_scale * (1.0 + n.beta_n) / g.nz;
  k.dtaupf_fac = n.cfl_pf * k.h2 * (1.0 + p.beta_d * p.B / p.alpha);
  k.rGdtS = dtS > 0 ? 1.0 / (p.G * dtS) : 0.0;
  // background shear (Eqs. 32-33): tau_bg / (2 mu0) joins the xy strain rate on every xy-edge
  k.ebg = 0.5 * p.tau_bg / p.mu0;
  k.bg_on = p.tau_bg != 0.0;
  return k;
}

}  // namespace pt
