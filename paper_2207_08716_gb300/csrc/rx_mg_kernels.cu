// rx_mg_kernels.cu — geometric multigrid (FAS V-cycle) of the reactive porosity-wave step (thesis
// Art. 3, Eqs. 8-10; the thesis's future-work section on multigrid-accelerated PT iterations).
//
// The smoother is the reactive PT iteration with a local pseudo step: per cell
//   gP   = R - (Pf - Pf_o) / dt + fP
//   Pf'  = Pf + gP / (Dk / (omega BP) + 1/dt + a)        (Dk: Jacobi diagonal of the Darcy operator)
//   phi' = clamp(phi_o + dt dphi, 1e-4, 1) + fphi,   Xs' = (Xs_o + (dt/tau) Xs_eq) / (1 + dt/tau) + fX
// with every right-hand side at the sweep's input and f = 0 on the finest grid. Coarse grids are
// 2 x 2 x 2 agglomerations; the restriction takes 8-child means of the iterate and of the
// residual (g = target - current), the FAS source is f_c = mean(r) - g_c(u0_c), and the
// correction u_c - u0_c (written by the coarse level's last sweep) comes back by trilinear
// interpolation (3/4, 1/4 per direction, the neighbour held at the wall). The sweeps, the
// restriction and the right-hand side run one thread per cell, the prolongation one per fine
// x-pair.
#include "rx.cuh"

namespace pt {

namespace {

// Step equations at cell (i, j, k) of a grid: the rate R, gP, the Jacobi denominator (DEN) and
// the porosity and Xs targets (with the FAS sources when FAS).
template <class T>
struct MgEq {
  T R, gP, den, phi1, Xs1;
};

template <class T, bool FAS, bool DEN>
__device__ __forceinline__ MgEq<T> mg_eq(const Box& b, const RxCoef<T>& c, T romega, const RxIn<T>& in,
                                         const MgSrc<T>& f, long long q, int i, int j, int k) {
  const long long px = b.px, pxy = b.pxy;
  const T Pf = in.Pf[q], ph = in.phi[q], Xs = in.Xs[q];
  const T kc = rx_perm(c, ph);
  // Darcy flux through the six faces (zero through the walls): s_d = sum over the d-faces of the
  // face permeability (k + k_nb, twice the mean) times the pressure difference (z: minus the
  // buoyancy rho_f g dz across the face); k_d = the sum of those face permeabilities
  T sx = T(0), sy = T(0), sz = T(0), kx = T(0), ky = T(0), kz = T(0);
  if (i > 0) {
    const T kf = rx_perm(c, in.phi[q - 1]) + kc;
    sx = fma(kf, in.Pf[q - 1] - Pf, sx);
    kx += kf;
  }
  if (i < b.nx - 1) {
    const T kf = kc + rx_perm(c, in.phi[q + 1]);
    sx = fma(kf, in.Pf[q + 1] - Pf, sx);
    kx += kf;
  }
  if (j > 0) {
    const T kf = rx_perm(c, in.phi[q - px]) + kc;
    sy = fma(kf, in.Pf[q - px] - Pf, sy);
    ky += kf;
  }
  if (j < b.ny - 1) {
    const T kf = kc + rx_perm(c, in.phi[q + px]);
    sy = fma(kf, in.Pf[q + px] - Pf, sy);
    ky += kf;
  }
  if (k > 0) {
    const T kf = rx_perm(c, in.phi[q - pxy]) + kc;
    sz = fma(kf, (in.Pf[q - pxy] - Pf) + c.rhofg_dz, sz);
    kz += kf;
  }
  if (k < b.nz - 1) {
    const T kf = kc + rx_perm(c, in.phi[q + pxy]);
    sz = fma(kf, (in.Pf[q + pxy] - Pf) - c.rhofg_dz, sz);
    kz += kf;
  }
  // div qD = -(1/2) sum_d s_d / d^2
  const T divq = T(-0.5) * fma(sx, c.rdx2, fma(sy, c.rdy2, sz * c.rdz2));
  const T Pf_o = in.Pf_o[q], phi_o = in.phi_o[q], Xs_o = in.Xs_o[q];
  const T w = rx_rcp(T(1) - ph), ixs = rx_rcp(T(1) - Xs);
  const T xr = c.beta_x * Pf + c.half_xs;
  const T xseq = rx_clamp(xr, T(0), c.xs_max);
  const T dXs = (xseq - Xs) * c.rtau;
  const T bp = rx_bp(c, ph);
  const T rbp = rx_rcp(bp);
  const T src = c.sr_opdx * (T(1) - ph) * ixs;
  const T comp = Pf * w * c.reta;                        // -Pe / (eta (1 - phi)), Pe = -Pf
  MgEq<T> e;
  e.R = (-divq - comp + src * dXs) * rbp;
  e.gP = e.R - (Pf - Pf_o) * c.rdt;
  if (FAS) e.gP += f.fP[q];
  if (DEN) {
    const T dxs_dpf = (xr > T(0) && xr < c.xs_max) ? c.beta_x : T(0);
    const T a = (w * c.reta - src * dxs_dpf * c.rtau) * rbp;
    const T Dk = T(0.5) * fma(kx, c.rdx2, fma(ky, c.rdy2, kz * c.rdz2));
    e.den = Dk * rbp * romega + c.rdt + a;
  } else {
    e.den = T(1);
  }
  const T bphi = c.beta_d - c.beta_s * w;
  const T dphi = (T(1) - ph) * (bphi * e.R + comp - c.opdx * ixs * dXs);
  e.phi1 = rx_clamp(phi_o + c.dt * dphi, T(1e-4), T(1));
  e.Xs1 = (Xs_o + c.dt_tau * xseq) * c.r1dt_tau;
  if (FAS) {
    e.phi1 += f.fphi[q];
    e.Xs1 += f.fX[q];
  }
  return e;
}

// the coarse neighbour on the side of fine index i, held inside [0, m)
__device__ __forceinline__ int side_nb(int i, int m) {
  const int n = (i & 1) ? (i >> 1) + 1 : (i >> 1) - 1;
  return n < 0 ? 0 : (n > m - 1 ? m - 1 : n);
}

dim3 grid_of(const Box& b) { return dim3((unsigned)((b.nx + 31) / 32), (unsigned)((b.ny + 7) / 8), (unsigned)b.nz); }

}  // namespace

// LASTE: the last sweep of a coarse level's visit writes the correction e = u' - u0 into the u0
// slots (read and written by the same thread) instead of u', which nothing reads afterwards.
template <class T, bool FAS, bool LASTE>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 8 : 5) k_mg_smooth(Box b, RxCoef<T> c, T romega, RxIn<T> in, MgSrc<T> f,
                                                   RxOut<T> out, MgE<T> e0, unsigned long long* red, int check) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  double chg = 0.0;
  if (i < b.nx && j < b.ny && k < b.nz) {
    const long long q = cidx(b, i, j, k);
    const MgEq<T> e = mg_eq<T, FAS, true>(b, c, romega, in, f, q, i, j, k);
    const T Pf = in.Pf[q], ph = in.phi[q], Xs = in.Xs[q];
    const T Pf1 = Pf + e.gP * rx_rcp(e.den);
    if (LASTE) {
      e0.Pf[q] = Pf1 - e0.Pf[q];
      e0.phi[q] = e.phi1 - e0.phi[q];
      e0.Xs[q] = e.Xs1 - e0.Xs[q];
    } else {
      out.Pf[q] = Pf1;
      out.phi[q] = e.phi1;
      out.Xs[q] = e.Xs1;
      if (out.R) out.R[q] = e.R;
    }
    if (check)
      chg = rx_change((double)rx_abs(e.phi1 - ph), (double)rx_abs(Pf1 - Pf) * (double)c.pf_iscale,
                      (double)rx_abs(e.Xs1 - Xs));
  }
  if (check) block_max_atomic(chg, red + RED_V);
}

// One fine cell per thread: its residual (the step equations, without the Jacobi denominator) and
// iterate; the 8 children of a coarse cell sit in one block of 32 x 4 x 2 threads (x pairs
// summed by a warp shuffle, y and z pairs through shared memory), whose 16 x 2 x 1 coarse cells
// receive the 8-child means.
constexpr int kRbx = 32, kRby = 4, kRbz = 2;

template <class T, bool FAS>
__global__ void __launch_bounds__(kRbx * kRby * kRbz) k_mg_restrict(Box fb, Box cb, RxCoef<T> c, RxIn<T> in,
                                                                    MgSrc<T> f, MgCoarse<T> out) {
  const int tx = threadIdx.x, ty = threadIdx.y, tz = threadIdx.z;
  const int i = blockIdx.x * kRbx + tx, j = blockIdx.y * kRby + ty, k = blockIdx.z * kRbz + tz;
  T v[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};        // Pf, phi, Xs, gP, gphi, gX
  if (i < fb.nx && j < fb.ny && k < fb.nz) {
    const long long q = cidx(fb, i, j, k);
    const MgEq<T> e = mg_eq<T, FAS, false>(fb, c, T(1), in, f, q, i, j, k);
    const T ph = in.phi[q], Xs = in.Xs[q];
    v[0] = in.Pf[q];
    v[1] = ph;
    v[2] = Xs;
    v[3] = e.gP;
    v[4] = e.phi1 - ph;
    v[5] = e.Xs1 - Xs;
  }
  __shared__ T part[kRbz][kRby][kRbx / 2][6];
#pragma unroll
  for (int n = 0; n < 6; ++n) {
    const T o = __shfl_down_sync(0xffffffffu, v[n], 1);
    if ((tx & 1) == 0) part[tz][ty][tx >> 1][n] = v[n] + o;
  }
  __syncthreads();
  if (tz == 0 && (ty & 1) == 0 && tx < kRbx / 2) {
    const int I = blockIdx.x * (kRbx / 2) + tx, J = blockIdx.y * (kRby / 2) + (ty >> 1), K = blockIdx.z;
    if (I < cb.nx && J < cb.ny && K < cb.nz) {
      T s[6];
#pragma unroll
      for (int n = 0; n < 6; ++n)
        s[n] = T(0.125) * ((part[0][ty][tx][n] + part[0][ty + 1][tx][n]) + (part[1][ty][tx][n] + part[1][ty + 1][tx][n]));
      const long long Q = cidx(cb, I, J, K);
      out.Pf[Q] = s[0];
      out.phi[Q] = s[1];
      out.Xs[Q] = s[2];
      out.Pf0[Q] = s[0];
      out.phi0[Q] = s[1];
      out.Xs0[Q] = s[2];
      out.fP[Q] = s[3];
      out.fphi[Q] = s[4];
      out.fX[Q] = s[5];
    }
  }
}

template <class T>
__global__ void __launch_bounds__(256) k_mg_coarse_rhs(Box b, RxCoef<T> c, RxIn<T> u0, MgCoarse<T> out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= b.nx || j >= b.ny || k >= b.nz) return;
  const long long q = cidx(b, i, j, k);
  const MgEq<T> e = mg_eq<T, false, false>(b, c, T(1), u0, MgSrc<T>{nullptr, nullptr, nullptr}, q, i, j, k);
  out.fP[q] -= e.gP;
  out.fphi[q] -= e.phi1 - u0.phi[q];
  out.fX[q] -= e.Xs1 - u0.Xs[q];
}

// One thread per fine x-pair (the two x-children of coarse column I at fine row (j, k)): the
// correction's coarse columns I - 1, I, I + 1 (held inside the grid) are first weighted over the
// parent's row and the row on the child's side in y and z (3/4 x 3/4, 3/4 x 1/4, 1/4 x 1/4),
// then the low child takes 3/4 of column I and 1/4 of I - 1, the high child 1/4 of I + 1.
template <class T>
struct __align__(2 * sizeof(T)) MgPair {
  T lo, hi;
};

template <class T>
__device__ __forceinline__ void prolong_pair(const T* __restrict__ e, T* u, long long q0, const long long (&xo)[3],
                                             const long long (&ro)[4], bool clamp) {
  T col[3];
#pragma unroll
  for (int d = 0; d < 3; ++d)
    col[d] = fma(T(0.5625), e[ro[0] + xo[d]],
                 fma(T(0.1875), e[ro[1] + xo[d]] + e[ro[2] + xo[d]], T(0.0625) * e[ro[3] + xo[d]]));
  MgPair<T> p = *reinterpret_cast<const MgPair<T>*>(u + q0);
  p.lo += fma(T(0.75), col[1], T(0.25) * col[0]);
  p.hi += fma(T(0.75), col[1], T(0.25) * col[2]);
  if (clamp) {
    p.lo = rx_clamp(p.lo, T(1e-4), T(1));
    p.hi = rx_clamp(p.hi, T(1e-4), T(1));
  }
  *reinterpret_cast<MgPair<T>*>(u + q0) = p;
}

template <class T>
__global__ void __launch_bounds__(256) k_mg_prolong(Box fb, Box cb, MgCorr<T> e, T* Pf, T* phi, T* Xs) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (I >= cb.nx || j >= fb.ny || k >= fb.nz) return;
  const long long xo[3] = {max(I - 1, 0), I, min(I + 1, cb.nx - 1)};
  const long long yJ = (long long)cb.px * (j >> 1), yN = (long long)cb.px * side_nb(j, cb.ny);
  const long long zK = cb.pxy * (k >> 1), zN = cb.pxy * side_nb(k, cb.nz);
  const long long ro[4] = {yJ + zK, yN + zK, yJ + zN, yN + zN};   // weights 9/16, 3/16, 3/16, 1/16
  const long long q0 = cidx(fb, 2 * I, j, k);
  prolong_pair(e.Pf, Pf, q0, xo, ro, false);
  prolong_pair(e.phi, phi, q0, xo, ro, true);
  prolong_pair(e.Xs, Xs, q0, xo, ro, false);
}

template <class T>
__global__ void __launch_bounds__(256) k_mg_restrict_old(Box fb, Box cb, const T* __restrict__ a,
                                                         const T* __restrict__ b, const T* __restrict__ d, T* A, T* B,
                                                         T* D) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = blockIdx.y * blockDim.y + threadIdx.y;
  const int K = blockIdx.z;
  if (I >= cb.nx || J >= cb.ny || K >= cb.nz) return;
  T sa = T(0), sb = T(0), sd = T(0);
#pragma unroll
  for (int n = 0; n < 8; ++n) {
    const long long q = cidx(fb, 2 * I + (n & 1), 2 * J + ((n >> 1) & 1), 2 * K + (n >> 2));
    sa += a[q];
    sb += b[q];
    sd += d[q];
  }
  const long long Q = cidx(cb, I, J, K);
  A[Q] = sa * T(0.125);
  B[Q] = sb * T(0.125);
  D[Q] = sd * T(0.125);
}

template <class T>
void mg_smooth(cudaStream_t s, Box b, const RxCoef<T>& c, double omega, const RxIn<T>& in, const MgSrc<T>* fas,
               const RxOut<T>& out, const MgE<T>* laste, unsigned long long* red, int check) {
  const T romega = (T)(1.0 / omega);
  const MgSrc<T> none{nullptr, nullptr, nullptr};
  const MgE<T> noe{nullptr, nullptr, nullptr};
  const dim3 g = grid_of(b), blk(32, 8, 1);
  if (!fas)
    k_mg_smooth<T, false, false><<<g, blk, 0, s>>>(b, c, romega, in, none, out, noe, red, check);
  else if (!laste)
    k_mg_smooth<T, true, false><<<g, blk, 0, s>>>(b, c, romega, in, *fas, out, noe, red, check);
  else
    k_mg_smooth<T, true, true><<<g, blk, 0, s>>>(b, c, romega, in, *fas, out, *laste, red, check);
}

template <class T>
void mg_restrict(cudaStream_t s, Box fine, Box coarse, const RxCoef<T>& c, const RxIn<T>& in, const MgSrc<T>* fas,
                 const MgCoarse<T>& out) {
  const dim3 g((unsigned)((fine.nx + kRbx - 1) / kRbx), (unsigned)((fine.ny + kRby - 1) / kRby),
               (unsigned)((fine.nz + kRbz - 1) / kRbz));
  const dim3 blk(kRbx, kRby, kRbz);
  if (fas)
    k_mg_restrict<T, true><<<g, blk, 0, s>>>(fine, coarse, c, in, *fas, out);
  else
    k_mg_restrict<T, false><<<g, blk, 0, s>>>(fine, coarse, c, in, MgSrc<T>{nullptr, nullptr, nullptr}, out);
}

template <class T>
void mg_coarse_rhs(cudaStream_t s, Box coarse, const RxCoef<T>& c, const RxIn<T>& u0, const MgCoarse<T>& out) {
  k_mg_coarse_rhs<T><<<grid_of(coarse), dim3(32, 8, 1), 0, s>>>(coarse, c, u0, out);
}

template <class T>
void mg_prolong(cudaStream_t s, Box fine, Box coarse, const MgCorr<T>& e, T* Pf, T* phi, T* Xs) {
  const dim3 g((unsigned)((coarse.nx + 31) / 32), (unsigned)((fine.ny + 7) / 8), (unsigned)fine.nz);
  k_mg_prolong<T><<<g, dim3(32, 8, 1), 0, s>>>(fine, coarse, e, Pf, phi, Xs);
}

template <class T>
void mg_restrict_old(cudaStream_t s, Box fine, Box coarse, const T* Pf_o, const T* phi_o, const T* Xs_o, T* cPf_o,
                     T* cphi_o, T* cXs_o) {
  k_mg_restrict_old<T><<<grid_of(coarse), dim3(32, 8, 1), 0, s>>>(fine, coarse, Pf_o, phi_o, Xs_o, cPf_o, cphi_o,
                                                                  cXs_o);
}

#define MG_INSTANTIATE(T)                                                                                          \
  template void mg_smooth<T>(cudaStream_t, Box, const RxCoef<T>&, double, const RxIn<T>&, const MgSrc<T>*,        \
                             const RxOut<T>&, const MgE<T>*, unsigned long long*, int);                           \
  template void mg_restrict<T>(cudaStream_t, Box, Box, const RxCoef<T>&, const RxIn<T>&, const MgSrc<T>*,         \
                               const MgCoarse<T>&);                                                               \
  template void mg_coarse_rhs<T>(cudaStream_t, Box, const RxCoef<T>&, const RxIn<T>&, const MgCoarse<T>&);        \
  template void mg_prolong<T>(cudaStream_t, Box, Box, const MgCorr<T>&, T*, T*, T*);                             \
  template void mg_restrict_old<T>(cudaStream_t, Box, Box, const T*, const T*, const T*, T*, T*, T*);
MG_INSTANTIATE(double)
MG_INSTANTIATE(float)

}  // namespace pt
