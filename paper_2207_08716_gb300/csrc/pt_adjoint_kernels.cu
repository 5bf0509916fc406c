// pt_adjoint_kernels.cu — discrete adjoint of the converged implicit step (Art. 1, Eqs. 17-26;
// the thesis has no adjoint: the gradient of a final-porosity misfit w.r.t. the log-k field).
//
// Each physical step solves F(u; u_o, theta) = 0 for u = (V, Pt, Pf, phi) (Eqs. 17-22 with the
// power law off, no weakening switch, beta_n = 0 and fixed old stresses, so eta = eta0 mu0 / phi).
// For an objective J(phi^N) the adjoint of step n solves J_F(u^n)^T lambda = g^n with the same
// pseudo-transient scheme as the forward solve, on the transposed staggered stencils:
//   row V  (faces):  A lambda_V - grad lambda_P + (d adv / d V)^T lambda_L
//                    (A: the symmetric viscoelastic operator; damped PT, as the forward V)
//   row Pt (centres): div lambda_V + (beta_d/dt + c) lambda_P - (beta_d alpha/dt + c) lambda_F
//                    - (beta_phi + dt/eta) lambda_L - g_P     (local-implicit PT)
//   row Pf (centres): K lambda_F + (beta_d alpha/(B dt) + c) lambda_F - (beta_d alpha/dt + c) lambda_P
//                    + (beta_phi + dt/eta) lambda_L - g_F      (K: the symmetric Darcy operator)
//   row phi(centres): buoyancy, compaction, dk/dphi and advection transposes; lambda_L from its
//                    own diagonal dF_L/dphi = -1/(1-phi) + ... (Jacobi)
// with c = phi / ((1-phi) eta0 mu0) and k = k0 e^theta (phi/phi0)^3.
//
// GB300 form: FP64 throughput (not HBM) bounds these stencils, so everything that depends only
// on the frozen converged state — 1/(1-phi), k and its face averages, dPf/dn, the row diagonals
// and their inverses — is computed once per step by k_adj_prep, and the iteration kernels are
// left with multiply-adds: no division and no k(phi) evaluation per iteration.
#include "pt_adjoint.cuh"

namespace pt {

namespace {
__device__ inline double pos_max_d(double a, double b) {
  const long long ia = __double_as_longlong(a), ib = __double_as_longlong(b);
  return __longlong_as_double(ia > ib ? ia : ib);
}
__device__ inline double kperm(const AdjCoef& c, const double* K0, long long q, double ph) {
  const double r = ph * c.rphi0;
  return (K0 ? K0[q] : c.k0) * r * r * r;
}
}  // namespace

// Per-step coefficients from the converged state u (cells i < nx ... and their lower faces).
__global__ void __launch_bounds__(256) k_adj_prep(Box b, AdjCoef c, AdjState u, const double* __restrict__ K0,
                                                  AdjPrep o) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i > b.nx || j > b.ny || k > b.nz) return;
  const long long q = cidx(b, i, j, k);
  const long long px = b.px, pxy = b.pxy;
  // lower faces of the cell (i, j, k): interior faces only, zero elsewhere
  {
    double kf = 0.0, gk = 0.0, bf = 0.0;
    if (i > 0 && i < b.nx && j < b.ny && k < b.nz) {
      const double pl = u.phi[q - 1], pr = u.phi[q];
      kf = 0.5 * (kperm(c, K0, q - 1, pl) + kperm(c, K0, q, pr)) * c.rdx * c.rdx;
      gk = -0.5 * (u.Pf[q] - u.Pf[q - 1]) * c.rdx * c.rdx;
      bf = -c.hdt_rdx * (pr - pl);
    }
    o.kfx[q] = kf; o.gkx[q] = gk; o.bfx[q] = bf;
  }
  {
    double kf = 0.0, gk = 0.0, bf = 0.0;
    if (j > 0 && j < b.ny && i < b.nx && k < b.nz) {
      const double pl = u.phi[q - px], pr = u.phi[q];
      kf = 0.5 * (kperm(c, K0, q - px, pl) + kperm(c, K0, q, pr)) * c.rdy * c.rdy;
      gk = -0.5 * (u.Pf[q] - u.Pf[q - px]) * c.rdy * c.rdy;
      bf = -c.hdt_rdy * (pr - pl);
    }
    o.kfy[q] = kf; o.gky[q] = gk; o.bfy[q] = bf;
  }
  {
    double kf = 0.0, gk = 0.0, bf = 0.0;
    if (k > 0 && k < b.nz && i < b.nx && j < b.ny) {
      const double pl = u.phi[q - pxy], pr = u.phi[q];
      kf = 0.5 * (kperm(c, K0, q - pxy, pl) + kperm(c, K0, q, pr)) * c.rdz * c.rdz;
      gk = -0.5 * ((u.Pf[q] - u.Pf[q - pxy]) * c.rdz + c.buoy) * c.rdz;
      bf = -c.hdt_rdz * (pr - pl);
    }
    o.kfz[q] = kf; o.gkz[q] = gk; o.bfz[q] = bf;
  }
  if (i >= b.nx || j >= b.ny || k >= b.nz) return;
  const double ph = u.phi[q];
  const double w = 1.0 / (1.0 - ph);
  const double cc = ph * w * c.r_eta0mu0;
  const double kc = kperm(c, K0, q, ph);
  double kmax = kc;
  if (i > 0) kmax = pos_max_d(kmax, kperm(c, K0, q - 1, u.phi[q - 1]));
  if (i < b.nx - 1) kmax = pos_max_d(kmax, kperm(c, K0, q + 1, u.phi[q + 1]));
  if (j > 0) kmax = pos_max_d(kmax, kperm(c, K0, q - px, u.phi[q - px]));
  if (j < b.ny - 1) kmax = pos_max_d(kmax, kperm(c, K0, q + px, u.phi[q + px]));
  if (k > 0) kmax = pos_max_d(kmax, kperm(c, K0, q - pxy, u.phi[q - pxy]));
  if (k < b.nz - 1) kmax = pos_max_d(kmax, kperm(c, K0, q + pxy, u.phi[q + pxy]));
  const double Pt = u.Pt[q], Pf = u.Pf[q];
  o.W[q] = w;
  o.cP[q] = 1.0 / (c.idtp + c.bd_rdt + cc);
  o.cF[q] = 1.0 / (kmax * c.ifac_pf + c.bda_B_rdt + cc);
  o.aPF[q] = (Pt - Pf) * w * w * c.r_eta0mu0;
  o.a3k[q] = 3.0 * kc / ph;
  // diagonal of row phi: d/dphi [log(1-phi) + dt (Pf-Pt) phi/(eta0 mu0) + dt S / (2 (1-phi))],
  // S = sum over the cell's interior faces of V (om_r - om_l) / d, om = 1 - phi
  const double omc = 1.0 - ph;
  double S = 0.0, dS = 0.0;
  if (i > 0) { S += u.Vx[q] * (omc - (1.0 - u.phi[q - 1])) * c.rdx; dS -= u.Vx[q] * c.rdx; }
  if (i < b.nx - 1) { S += u.Vx[q + 1] * ((1.0 - u.phi[q + 1]) - omc) * c.rdx; dS += u.Vx[q + 1] * c.rdx; }
  if (j > 0) { S += u.Vy[q] * (omc - (1.0 - u.phi[q - px])) * c.rdy; dS -= u.Vy[q] * c.rdy; }
  if (j < b.ny - 1) { S += u.Vy[q + px] * ((1.0 - u.phi[q + px]) - omc) * c.rdy; dS += u.Vy[q + px] * c.rdy; }
  if (k > 0) { S += u.Vz[q] * (omc - (1.0 - u.phi[q - pxy])) * c.rdz; dS -= u.Vz[q] * c.rdz; }
  if (k < b.nz - 1) { S += u.Vz[q + pxy] * ((1.0 - u.phi[q + pxy]) - omc) * c.rdz; dS += u.Vz[q + pxy] * c.rdz; }
  const double diag = -w + c.dt_r * (Pf - Pt) + c.dt * 0.5 * (w * w * S + w * dS);
  o.Dg[q] = diag;
  o.iD[q] = 1.0 / diag;
  o.mL[q] = o.lL[q] * w;
}

// Cells: adjoint stresses of lambda_V at centres and the cell's lower edges, and the centre
// updates of lambda_P, lambda_F, lambda_L.
__global__ void __launch_bounds__(256) k_adj_cells(Box b, AdjCoef c, AdjState u, AdjCellIn in, AdjCellOut out,
                                                   unsigned long long* red, int check) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  double r_pt = 0.0, r_pf = 0.0, r_l = 0.0;
  if (i <= b.nx && j <= b.ny && k <= b.nz) {
    const long long q = cidx(b, i, j, k);
    const long long px = b.px, pxy = b.pxy;
    if (k < b.nz) {
      double t = 0.0;
      if (i > 0 && i < b.nx && j > 0 && j < b.ny)
        t = c.hm2rdy * (in.Lx[q] - in.Lx[q - px]) + c.hm2rdx * (in.Ly[q] - in.Ly[q - 1]);
      out.txy[q] = t;
    }
    if (j < b.ny) {
      double t = 0.0;
      if (i > 0 && i < b.nx && k > 0 && k < b.nz)
        t = c.hm2rdz * (in.Lx[q] - in.Lx[q - pxy]) + c.hm2rdx * (in.Lz[q] - in.Lz[q - 1]);
      out.txz[q] = t;
    }
    if (i < b.nx) {
      double t = 0.0;
      if (j > 0 && j < b.ny && k > 0 && k < b.nz)
        t = c.hm2rdz * (in.Ly[q] - in.Ly[q - pxy]) + c.hm2rdy * (in.Lz[q] - in.Lz[q - px]);
      out.tyz[q] = t;
    }
    if (i < b.nx && j < b.ny && k < b.nz) {
      const double ph = u.phi[q];
      const double cc = ph * in.W[q] * c.r_eta0mu0;
      const double lP = in.lP[q], lF = in.lF[q], lL = in.lL[q];
      // lambda_V at the cell's faces (wall faces are not unknowns and stay zero)
      const double Lz0 = in.Lz[q], Lz1 = in.Lz[q + pxy];
      const double gx = (in.Lx[q + 1] - in.Lx[q]) * c.rdx, gy = (in.Ly[q + px] - in.Ly[q]) * c.rdy;
      const double gz = (Lz1 - Lz0) * c.rdz;
      const double divL = gx + gy + gz;
      const double d3 = divL * c.third;
      out.txx[q] = c.m2 * (gx - d3);
      out.tyy[q] = c.m2 * (gy - d3);
      out.tzz[q] = c.m2 * (gz - d3);
      // ---- row Pt
      const double cplP = c.bd_rdt_a + cc, cplL = c.beta_phi + c.dt_r * ph;
      const double resP = divL + (c.bd_rdt + cc) * lP - cplP * lF - cplL * lL - in.gP[q];
      out.lP[q] = lP - in.cP[q] * resP;
      // ---- row Pf: K lambda_F and (dq/dk)^T lambda_F over the six faces; the advection
      // transpose of row phi over the same faces
      double Klf = 0.0, dkT = 0.0, offx = 0.0, offy = 0.0, offz = 0.0;
      if (i > 0) {
        const double dn = in.lF[q - 1] - lF;
        Klf -= in.kfx[q] * dn;
        dkT += in.gkx[q] * dn;
        offx -= u.Vx[q] * in.mL[q - 1];
      }
      if (i < b.nx - 1) {
        const double dn = in.lF[q + 1] - lF;
        Klf -= in.kfx[q + 1] * dn;
        dkT -= in.gkx[q + 1] * dn;
        offx += u.Vx[q + 1] * in.mL[q + 1];
      }
      if (j > 0) {
        const double dn = in.lF[q - px] - lF;
        Klf -= in.kfy[q] * dn;
        dkT += in.gky[q] * dn;
        offy -= u.Vy[q] * in.mL[q - px];
      }
      if (j < b.ny - 1) {
        const double dn = in.lF[q + px] - lF;
        Klf -= in.kfy[q + px] * dn;
        dkT -= in.gky[q + px] * dn;
        offy += u.Vy[q + px] * in.mL[q + px];
      }
      if (k > 0) {
        const double dn = in.lF[q - pxy] - lF;
        Klf -= in.kfz[q] * dn;
        dkT += in.gkz[q] * dn;
        offz -= u.Vz[q] * in.mL[q - pxy];
      }
      if (k < b.nz - 1) {
        const double dn = in.lF[q + pxy] - lF;
        Klf -= in.kfz[q + pxy] * dn;
        dkT -= in.gkz[q + pxy] * dn;
        offz += u.Vz[q + pxy] * in.mL[q + pxy];
      }
      const double off = offx * c.hdt_rdx + offy * c.hdt_rdy + offz * c.hdt_rdz;
      const double resF = Klf + (c.bda_B_rdt + cc) * lF - cplP * lP + cplL * lL - in.gF[q];
      out.lF[q] = lF - in.cF[q] * resF;
      const double a3k = in.a3k[q];
      if (out.gtheta) out.gtheta[q] = a3k * ph * c.third * dkT;   // k (dq/dk)^T lambda_F
      // ---- row phi: buoyancy (Eq. 19), compaction (Eqs. 17-18), k(phi) (Eq. 23), advection
      const double sL = -c.hdrho_g * (Lz0 + Lz1) + in.aPF[q] * (lP - lF) + a3k * dkT + off - in.gphi[q];
      const double lLn = -in.iD[q] * sL;
      out.lL[q] = lLn;
      out.mL[q] = lLn * in.W[q];
      if (check || out.rL) {
        const double resL = sL + in.Dg[q] * lL;
        if (out.rL) {
          out.rP[q] = resP;
          out.rF[q] = resF;
          out.rL[q] = resL;
        }
        r_pt = fabs(resP);
        r_pf = fabs(resF);
        r_l = fabs(resL);
      }
    }
  }
  if (check) {
    block_max_atomic(r_pt, red + RED_PT);
    block_max_atomic(r_pf, red + RED_PF);
    block_max_atomic(r_l, red + RED_PIC);
  }
}

// Faces: row V with lambda_P1 and mL = lambda_L / (1 - phi); damped R, lambda_V update.
__global__ void __launch_bounds__(256) k_adj_faces(Box b, AdjCoef c, AdjFaceIn in, double* Lx, double* Ly,
                                                   double* Lz, double* Rx, double* Ry, double* Rz,
                                                   unsigned long long* red, int check) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  double r_v = 0.0;
  if (i <= b.nx && j <= b.ny && k <= b.nz) {
    const long long q = cidx(b, i, j, k);
    const long long px = b.px, pxy = b.pxy;
    const bool fx = i > 0 && i < b.nx && j < b.ny && k < b.nz;
    const bool fy = j > 0 && j < b.ny && i < b.nx && k < b.nz;
    const bool fz = k > 0 && k < b.nz && i < b.nx && j < b.ny;
    double Fx = 0.0, Fy = 0.0, Fz = 0.0, Rx1 = 0.0, Ry1 = 0.0, Rz1 = 0.0, Lx1 = 0.0, Ly1 = 0.0, Lz1 = 0.0;
    if (fx) {
      Fx = (in.txx[q] - in.txx[q - 1]) * c.rdx + (in.txy[q + px] - in.txy[q]) * c.rdy +
           (in.txz[q + pxy] - in.txz[q]) * c.rdz - (in.lP1[q] - in.lP1[q - 1]) * c.rdx +
           in.bfx[q] * (in.mL[q - 1] + in.mL[q]);
      if (in.update) {
        Rx1 = Fx * c.rrho_i + c.damp_x * Rx[q];
        Lx1 = Lx[q] + c.dtauv * Rx1;
      }
    }
    if (fy) {
      Fy = (in.txy[q + 1] - in.txy[q]) * c.rdx + (in.tyy[q] - in.tyy[q - px]) * c.rdy +
           (in.tyz[q + pxy] - in.tyz[q]) * c.rdz - (in.lP1[q] - in.lP1[q - px]) * c.rdy +
           in.bfy[q] * (in.mL[q - px] + in.mL[q]);
      if (in.update) {
        Ry1 = Fy * c.rrho_i + c.damp_y * Ry[q];
        Ly1 = Ly[q] + c.dtauv * Ry1;
      }
    }
    if (fz) {
      Fz = (in.txz[q + 1] - in.txz[q]) * c.rdx + (in.tyz[q + px] - in.tyz[q]) * c.rdy +
           (in.tzz[q] - in.tzz[q - pxy]) * c.rdz - (in.lP1[q] - in.lP1[q - pxy]) * c.rdz +
           in.bfz[q] * (in.mL[q - pxy] + in.mL[q]);
      if (in.update) {
        Rz1 = Fz * c.rrho_i + c.damp_z * Rz[q];
        Lz1 = Lz[q] + c.dtauv * Rz1;
      }
    }
    if (in.update) {
      if (fx) { Rx[q] = Rx1; Lx[q] = Lx1; }
      if (fy) { Ry[q] = Ry1; Ly[q] = Ly1; }
      if (fz) { Rz[q] = Rz1; Lz[q] = Lz1; }
    }
    if (fx && in.rx) in.rx[q] = Fx;
    if (fy && in.ry) in.ry[q] = Fy;
    if (fz && in.rz) in.rz[q] = Fz;
    r_v = fmax(fabs(Fx), fmax(fabs(Fy), fabs(Fz)));
  }
  if (check) block_max_atomic(r_v, red + RED_V);
}

// After a converged adjoint step: dJ/dtheta -= k (dq/dk)^T lambda_F (already in gtheta), and
// the carry g = -(dF/du_o)^T lambda into the previous step (through Pto, Pfo, Lo = log(1-phi_o)).
__global__ void __launch_bounds__(256) k_adj_carry(Box b, AdjCoef c, AdjCarry a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= b.nx || j >= b.ny || k >= b.nz) return;
  const long long q = cidx(b, i, j, k);
  const double lP = a.lP[q], lF = a.lF[q], lL = a.lL[q];
  a.grad[q] -= a.gtheta[q];
  a.gP[q] = c.bd_rdt * lP - c.bd_rdt_a * lF - c.beta_phi * lL;
  a.gF[q] = -c.bd_rdt_a * lP + c.bda_B_rdt * lF + c.beta_phi * lL;
  a.gphi[q] = -lL / (1.0 - a.phi_o[q]);
}

// Largest |g| of the right-hand side of an adjoint step (its convergence scale).
__global__ void __launch_bounds__(256) k_adj_gmax(Box b, const double* gP, const double* gF, const double* gphi,
                                                  unsigned long long* red) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  double m = 0.0;
  if (i < b.nx && j < b.ny && k < b.nz) {
    const long long q = cidx(b, i, j, k);
    m = fmax(fabs(gP[q]), fmax(fabs(gF[q]), fabs(gphi[q])));
  }
  block_max_atomic(m, red + RED_GMAX);
}

void adj_prep(dim3 g, dim3 bl, cudaStream_t s, Box b, const AdjCoef& c, const AdjState& u, const double* K0,
              const AdjPrep& out) {
  k_adj_prep<<<g, bl, 0, s>>>(b, c, u, K0, out);
}
void adj_cells(dim3 g, dim3 bl, cudaStream_t s, Box b, const AdjCoef& c, const AdjState& u, const AdjCellIn& in,
               const AdjCellOut& out, unsigned long long* red, int check) {
  k_adj_cells<<<g, bl, 0, s>>>(b, c, u, in, out, red, check);
}
void adj_faces(dim3 g, dim3 bl, cudaStream_t s, Box b, const AdjCoef& c, const AdjFaceIn& in, double* Lx,
               double* Ly, double* Lz, double* Rx, double* Ry, double* Rz, unsigned long long* red, int check) {
  k_adj_faces<<<g, bl, 0, s>>>(b, c, in, Lx, Ly, Lz, Rx, Ry, Rz, red, check);
}
void adj_carry(dim3 g, dim3 bl, cudaStream_t s, Box b, const AdjCoef& c, const AdjCarry& a) {
  k_adj_carry<<<g, bl, 0, s>>>(b, c, a);
}
void adj_gmax(dim3 g, dim3 bl, cudaStream_t s, Box b, const double* gP, const double* gF, const double* gphi,
              unsigned long long* red) {
  k_adj_gmax<<<g, bl, 0, s>>>(b, gP, gF, gphi, red);
}

}  // namespace pt
