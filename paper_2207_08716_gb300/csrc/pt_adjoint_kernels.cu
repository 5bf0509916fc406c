// pt_adjoint_kernels.cu — discrete adjoint of the converged implicit step.
//
// Each physical step solves F(u; u_o, theta) = 0 for u = (V, Pt, Pf, phi) (Eqs. 17-22 with the
// power law off, no weakening switch, beta_n = 0 and fixed old stresses, so eta = eta0 mu0 / phi).
// For an objective J(phi^N) the adjoint of step n solves J_F(u^n)^T lambda = g^n with the same
// pseudo-transient scheme as the forward solve, on the transposed staggered stencils:
//   row V  (faces):  A lambda_V - grad lambda_P - dt/2 d(phi)/dx (w lambda_L)_l + (w lambda_L)_r
//                    (A: the symmetric viscoelastic operator; damped PT, as the forward V)
//   row Pt (centres): div lambda_V + (beta_d/dt + c) lambda_P - (beta_d alpha/dt + c) lambda_F
//                    - (beta_phi + dt/eta) lambda_L - g_P     (local-implicit PT)
//   row Pf (centres): K lambda_F + (beta_d alpha/(B dt) + c) lambda_F - (beta_d alpha/dt + c) lambda_P
//                    + (beta_phi + dt/eta) lambda_L - g_F      (K: the symmetric Darcy operator)
//   row phi(centres): buoyancy, compaction, d k/d phi and advection transposes; lambda_L by
//                    Jacobi on its diagonal dF_L/dphi = -1/(1-phi) + ...
// with w = 1/(1-phi), c = phi w/(eta0 mu0), k = k0 e^theta (phi/phi0)^3. After convergence,
// dJ/dtheta -= k (dq/dk)^T lambda_F and the carry into the previous step is g = -(dF/du_o)^T lambda.
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

// Cells: adjoint stresses of lambda_V at centres and the cell's lower edges, and the centre
// updates lambda_P, lambda_F, lambda_L.
__global__ void __launch_bounds__(256) k_adj_cells(Box b, AdjCoef c, AdjState u, AdjCellIn in, AdjCellOut out,
                                                   unsigned long long* red, int check) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  double r_pt = 0.0, r_pf = 0.0, r_l = 0.0;
  if (i <= b.nx && j <= b.ny && k <= b.nz) {
    const long long q = cidx(b, i, j, k);
    const long long px = b.px, pxy = b.pxy;
    const double m2 = c.m2;
    if (k < b.nz) {
      double t = 0.0;
      if (i > 0 && i < b.nx && j > 0 && j < b.ny)
        t = m2 * 0.5 * ((in.Lx[q] - in.Lx[q - px]) * c.rdy + (in.Ly[q] - in.Ly[q - 1]) * c.rdx);
      out.txy[q] = t;
    }
    if (j < b.ny) {
      double t = 0.0;
      if (i > 0 && i < b.nx && k > 0 && k < b.nz)
        t = m2 * 0.5 * ((in.Lx[q] - in.Lx[q - pxy]) * c.rdz + (in.Lz[q] - in.Lz[q - 1]) * c.rdx);
      out.txz[q] = t;
    }
    if (i < b.nx) {
      double t = 0.0;
      if (j > 0 && j < b.ny && k > 0 && k < b.nz)
        t = m2 * 0.5 * ((in.Ly[q] - in.Ly[q - pxy]) * c.rdz + (in.Lz[q] - in.Lz[q - px]) * c.rdy);
      out.tyz[q] = t;
    }
    if (i < b.nx && j < b.ny && k < b.nz) {
      const double ph = u.phi[q];
      const double w = 1.0 / (1.0 - ph);
      const double ieta = ph * c.r_eta0mu0;             // 1 / eta = phi / (eta0 mu0)
      const double cc = ph * w * c.r_eta0mu0;           // 1 / (eta (1 - phi))
      const double dcc = w * w * c.r_eta0mu0;           // d cc / d phi
      const double lP = in.lP[q], lF = in.lF[q], lL = in.lL[q];
      // lambda_V at the cell's faces (boundary faces are not unknowns: zero)
      const double gx = (in.Lx[q + 1] - in.Lx[q]) * c.rdx, gy = (in.Ly[q + px] - in.Ly[q]) * c.rdy;
      const double gz = (in.Lz[q + pxy] - in.Lz[q]) * c.rdz;
      const double divL = gx + gy + gz;
      out.txx[q] = m2 * (gx - divL / 3.0);
      out.tyy[q] = m2 * (gy - divL / 3.0);
      out.tzz[q] = m2 * (gz - divL / 3.0);
      // ---- row Pt
      const double cplP = c.bd_rdt_a + cc, cplL = c.beta_phi + c.dt * ieta;
      const double resP = divL + (c.bd_rdt + cc) * lP - cplP * lF - cplL * lL - in.gP[q];
      const double idtp = c.idtp;
      out.lP[q] = (lP * idtp - (divL - cplP * lF - cplL * lL - in.gP[q])) / (idtp + c.bd_rdt + cc);
      // ---- row Pf: symmetric Darcy operator on lambda_F, and the pieces of row phi that need
      // the face fluxes: (dq/dk)^T lambda_F with gr_f = dPf/dn (+ buoyancy on z-faces)
      const double kc = kperm(c, in.K0, q, ph);
      const double Pf = u.Pf[q];
      double kmax = kc, sK = 0.0, sdk = 0.0;
      if (i > 0) {
        const double kn = kperm(c, in.K0, q - 1, u.phi[q - 1]);
        kmax = pos_max_d(kmax, kn);
        sK -= (kn + kc) * (lF - in.lF[q - 1]) * c.rdx * c.rdx;
        sdk += (Pf - u.Pf[q - 1]) * c.rdx * (in.lF[q - 1] - lF) * c.rdx;
      }
      if (i < b.nx - 1) {
        const double kn = kperm(c, in.K0, q + 1, u.phi[q + 1]);
        kmax = pos_max_d(kmax, kn);
        sK += (kc + kn) * (in.lF[q + 1] - lF) * c.rdx * c.rdx;
        sdk += (u.Pf[q + 1] - Pf) * c.rdx * (lF - in.lF[q + 1]) * c.rdx;
      }
      if (j > 0) {
        const double kn = kperm(c, in.K0, q - px, u.phi[q - px]);
        kmax = pos_max_d(kmax, kn);
        sK -= (kn + kc) * (lF - in.lF[q - px]) * c.rdy * c.rdy;
        sdk += (Pf - u.Pf[q - px]) * c.rdy * (in.lF[q - px] - lF) * c.rdy;
      }
      if (j < b.ny - 1) {
        const double kn = kperm(c, in.K0, q + px, u.phi[q + px]);
        kmax = pos_max_d(kmax, kn);
        sK += (kc + kn) * (in.lF[q + px] - lF) * c.rdy * c.rdy;
        sdk += (u.Pf[q + px] - Pf) * c.rdy * (lF - in.lF[q + px]) * c.rdy;
      }
      if (k > 0) {
        const double kn = kperm(c, in.K0, q - pxy, u.phi[q - pxy]);
        kmax = pos_max_d(kmax, kn);
        sK -= (kn + kc) * (lF - in.lF[q - pxy]) * c.rdz * c.rdz;
        sdk += ((Pf - u.Pf[q - pxy]) * c.rdz + c.buoy) * (in.lF[q - pxy] - lF) * c.rdz;
      }
      if (k < b.nz - 1) {
        const double kn = kperm(c, in.K0, q + pxy, u.phi[q + pxy]);
        kmax = pos_max_d(kmax, kn);
        sK += (kc + kn) * (in.lF[q + pxy] - lF) * c.rdz * c.rdz;
        sdk += ((u.Pf[q + pxy] - Pf) * c.rdz + c.buoy) * (lF - in.lF[q + pxy]) * c.rdz;
      }
      const double Klf = -0.5 * sK;                     // K lambda_F (K = d div qD / d Pf)
      const double cplF = c.beta_phi + c.dt * ieta;
      const double resF = Klf + (c.bda_B_rdt + cc) * lF - cplP * lP + cplF * lL - in.gF[q];
      const double idtf = kmax * c.ifac_pf;
      out.lF[q] = (lF * idtf - (Klf - cplP * lP + cplF * lL - in.gF[q])) / (idtf + c.bda_B_rdt + cc);
      // (d div qD / d k)^T lambda_F at this cell: -1/2 sum_faces gr_f (lF_left - lF_right) / dx
      const double dkT = -0.5 * sdk;
      if (out.gtheta) out.gtheta[q] = kc * dkT;         // (dF_Pf/dtheta)^T lambda_F, dk/dtheta = k
      // ---- row phi
      const double Pt = u.Pt[q];
      double resL = -0.5 * c.drho_g * ((k > 0 ? in.Lz[q] : 0.0) + (k < b.nz - 1 ? in.Lz[q + pxy] : 0.0));
      resL += (Pt - Pf) * dcc * lP;                      // compaction in row Pt
      resL += (Pf - Pt) * dcc * lF + 3.0 * kc / ph * dkT; // compaction and k(phi) in row Pf
      // row L itself: log(1-phi), compaction dt (Pf - Pt) phi / (eta0 mu0), advection
      const double Vxl = u.Vx[q], Vxr = u.Vx[q + 1], Vyl = u.Vy[q], Vyr = u.Vy[q + px];
      const double Vzl = u.Vz[q], Vzr = u.Vz[q + pxy];
      const double omc = 1.0 - ph;
      double S = 0.0, dS = 0.0, off = 0.0;
      if (i > 0) {
        S += Vxl * (omc - (1.0 - u.phi[q - 1])) * c.rdx;
        dS -= Vxl * c.rdx;
        off -= 0.5 * in.lL[q - 1] / (1.0 - u.phi[q - 1]) * Vxl * c.rdx;
      }
      if (i < b.nx - 1) {
        S += Vxr * ((1.0 - u.phi[q + 1]) - omc) * c.rdx;
        dS += Vxr * c.rdx;
        off += 0.5 * in.lL[q + 1] / (1.0 - u.phi[q + 1]) * Vxr * c.rdx;
      }
      if (j > 0) {
        S += Vyl * (omc - (1.0 - u.phi[q - px])) * c.rdy;
        dS -= Vyl * c.rdy;
        off -= 0.5 * in.lL[q - px] / (1.0 - u.phi[q - px]) * Vyl * c.rdy;
      }
      if (j < b.ny - 1) {
        S += Vyr * ((1.0 - u.phi[q + px]) - omc) * c.rdy;
        dS += Vyr * c.rdy;
        off += 0.5 * in.lL[q + px] / (1.0 - u.phi[q + px]) * Vyr * c.rdy;
      }
      if (k > 0) {
        S += Vzl * (omc - (1.0 - u.phi[q - pxy])) * c.rdz;
        dS -= Vzl * c.rdz;
        off -= 0.5 * in.lL[q - pxy] / (1.0 - u.phi[q - pxy]) * Vzl * c.rdz;
      }
      if (k < b.nz - 1) {
        S += Vzr * ((1.0 - u.phi[q + pxy]) - omc) * c.rdz;
        dS += Vzr * c.rdz;
        off += 0.5 * in.lL[q + pxy] / (1.0 - u.phi[q + pxy]) * Vzr * c.rdz;
      }
      const double diag = -w + c.dt * (Pf - Pt) * c.r_eta0mu0 + c.dt * 0.5 * (w * w * S + w * dS);
      resL += diag * lL + c.dt * off - in.gphi[q];
      out.lL[q] = lL - resL / diag;
      if (check) {
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

// Faces: row V with the updated lambda_P, damped R, lambda_V update.
__global__ void __launch_bounds__(256) k_adj_faces(Box b, AdjCoef c, AdjState u, AdjFaceIn in, double* Lx,
                                                   double* Ly, double* Lz, double* Rx, double* Ry, double* Rz,
                                                   unsigned long long* red, int check) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  double r_v = 0.0;
  if (i <= b.nx && j <= b.ny && k <= b.nz) {
    const long long q = cidx(b, i, j, k);
    const long long px = b.px, pxy = b.pxy;
    // (d adv / d V)^T lambda_L on face f between cells l and r: -dt/2 (phi_r - phi_l)/dx (w lambda_L)_l+_r
    if (i > 0 && i < b.nx && j < b.ny && k < b.nz) {
      const double pl = u.phi[q - 1], pr = u.phi[q];
      const double adv = -0.5 * c.dt * (pr - pl) * c.rdx * (in.lL[q - 1] / (1.0 - pl) + in.lL[q] / (1.0 - pr));
      const double F = (in.txx[q] - in.txx[q - 1]) * c.rdx + (in.txy[q + px] - in.txy[q]) * c.rdy +
                       (in.txz[q + pxy] - in.txz[q]) * c.rdz - (in.lP1[q] - in.lP1[q - 1]) * c.rdx + adv;
      const double R = F * c.rrho_i + c.damp_x * Rx[q];
      Rx[q] = R;
      Lx[q] += c.dtauv * R;
      if (check) r_v = fmax(r_v, fabs(F));
    }
    if (j > 0 && j < b.ny && i < b.nx && k < b.nz) {
      const double pl = u.phi[q - px], pr = u.phi[q];
      const double adv = -0.5 * c.dt * (pr - pl) * c.rdy * (in.lL[q - px] / (1.0 - pl) + in.lL[q] / (1.0 - pr));
      const double F = (in.txy[q + 1] - in.txy[q]) * c.rdx + (in.tyy[q] - in.tyy[q - px]) * c.rdy +
                       (in.tyz[q + pxy] - in.tyz[q]) * c.rdz - (in.lP1[q] - in.lP1[q - px]) * c.rdy + adv;
      const double R = F * c.rrho_i + c.damp_y * Ry[q];
      Ry[q] = R;
      Ly[q] += c.dtauv * R;
      if (check) r_v = fmax(r_v, fabs(F));
    }
    if (k > 0 && k < b.nz && i < b.nx && j < b.ny) {
      const double pl = u.phi[q - pxy], pr = u.phi[q];
      const double adv = -0.5 * c.dt * (pr - pl) * c.rdz * (in.lL[q - pxy] / (1.0 - pl) + in.lL[q] / (1.0 - pr));
      const double F = (in.txz[q + 1] - in.txz[q]) * c.rdx + (in.tyz[q + px] - in.tyz[q]) * c.rdy +
                       (in.tzz[q] - in.tzz[q - pxy]) * c.rdz - (in.lP1[q] - in.lP1[q - pxy]) * c.rdz + adv;
      const double R = F * c.rrho_i + c.damp_z * Rz[q];
      Rz[q] = R;
      Lz[q] += c.dtauv * R;
      if (check) r_v = fmax(r_v, fabs(F));
    }
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

// Largest |g| of the right-hand side of an adjoint step (its convergence scale), into red[slot].
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

void adj_gmax(dim3 g, dim3 bl, cudaStream_t s, Box b, const double* gP, const double* gF, const double* gphi,
              unsigned long long* red) {
  k_adj_gmax<<<g, bl, 0, s>>>(b, gP, gF, gphi, red);
}
void adj_cells(dim3 g, dim3 bl, cudaStream_t s, Box b, const AdjCoef& c, const AdjState& u, const AdjCellIn& in,
               const AdjCellOut& out, unsigned long long* red, int check) {
  k_adj_cells<<<g, bl, 0, s>>>(b, c, u, in, out, red, check);
}
void adj_faces(dim3 g, dim3 bl, cudaStream_t s, Box b, const AdjCoef& c, const AdjState& u, const AdjFaceIn& in,
               double* Lx, double* Ly, double* Lz, double* Rx, double* Ry, double* Rz, unsigned long long* red,
               int check) {
  k_adj_faces<<<g, bl, 0, s>>>(b, c, u, in, Lx, Ly, Lz, Rx, Ry, Rz, red, check);
}
void adj_carry(dim3 g, dim3 bl, cudaStream_t s, Box b, const AdjCoef& c, const AdjCarry& a) {
  k_adj_carry<<<g, bl, 0, s>>>(b, c, a);
}

}  // namespace pt
