// rx_kernels.cu — reactive porosity-wave solver (thesis Art. 3, Eqs. 8-10; appendix A.6 form):
// one fused pseudo-transient iteration per launch. Per cell it reads Pf and k = k0 (phi/phi0)^3
// (FP64: stored with phi; FP32: from phi) with their six neighbours (Darcy flux, k averaged to the
// faces), phi, Xs and the old step, and writes the next Pf, phi, Xs (FP64: and k(phi')): 7 or 8
// arrays read, 3 or 4 written (the rate dPf/dt only on check and final iterations). Divisions are Newton-refined hardware reciprocals (rx_rcp).
#include "rx.cuh"

namespace pt {

template <class T>
__global__ void __launch_bounds__(256) k_rx_iter(Box b, RxCoef<T> c, T dtau, RxIn<T> in, RxOut<T> out,
                                                 unsigned long long* red, int check) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  double chg = 0.0, kb = 0.0;
  if (i < b.nx && j < b.ny && k < b.nz) {
    const long long q = cidx(b, i, j, k);
    const long long px = b.px, pxy = b.pxy;
    const T Pf = in.Pf[q], ph = in.phi[q], Xs = in.Xs[q];
    // k = k0 (phi/phi0)^3: in FP64 (bound by the FP64 pipe) it travels with phi, each cell writing
    // k(phi') for the next iteration; in FP32 (bound by HBM) it is recomputed from phi
    constexpr bool kstored = sizeof(T) == 8;
    auto perm = [&](long long o) { return kstored ? in.k[o] : rx_perm(c, in.phi[o]); };
    const T kc = perm(q);
    // Darcy flux through the six faces, zero through the walls; z faces carry rho_f g
    T sx = T(0), sy = T(0), sz = T(0);
    if (i > 0) sx -= (perm(q - 1) + kc) * (Pf - in.Pf[q - 1]) * c.rdx;
    if (i < b.nx - 1) sx += (kc + perm(q + 1)) * (in.Pf[q + 1] - Pf) * c.rdx;
    if (j > 0) sy -= (perm(q - px) + kc) * (Pf - in.Pf[q - px]) * c.rdy;
    if (j < b.ny - 1) sy += (kc + perm(q + px)) * (in.Pf[q + px] - Pf) * c.rdy;
    if (k > 0) sz -= (perm(q - pxy) + kc) * ((Pf - in.Pf[q - pxy]) * c.rdz - c.rhofg);
    if (k < b.nz - 1) sz += (kc + perm(q + pxy)) * ((in.Pf[q + pxy] - Pf) * c.rdz - c.rhofg);
    // div qD = -(1/2) sum_d [(k + k_r)(dPf_r) - (k_l + k)(dPf_l)] / d
    const T divq = -(sx * c.rdx + sy * c.rdy + sz * c.rdz) * T(0.5);
    const T Pf_o = in.Pf_o[q], phi_o = in.phi_o[q], Xs_o = in.Xs_o[q];
    const T w = rx_rcp(T(1) - ph), ixs = rx_rcp(T(1) - Xs);
    const T xr = c.beta_x * Pf + c.half_xs;
    const T xseq = rx_clamp(xr, T(0), c.xs_max);
    const T dXs = (xseq - Xs) * c.rtau;
    const T bp = rx_bp(c, ph);
    const T rbp = rx_rcp(bp);
    const T src = c.sr_opdx * (T(1) - ph) * ixs;
    const T comp = Pf * w * c.reta;                       // -Pe / (eta (1 - phi)), Pe = -Pf
    const T R = (-divq - comp + src * dXs) * rbp;
    const T dxs_dpf = (xr > T(0) && xr < c.xs_max) ? c.beta_x : T(0);
    const T a = (w * c.reta - src * dxs_dpf * c.rtau) * rbp;   // -dR/dPf of the cell's own terms
    const T Xs1 = (Xs_o + c.dt_tau * xseq) * c.r1dt_tau;
    const T Pf1 = Pf + dtau * (R - (Pf - Pf_o) * c.rdt) * rx_rcp(T(1) + dtau * (c.rdt + a));
    const T bphi = c.beta_d - c.beta_s * w;
    const T dphi = (T(1) - ph) * (bphi * R + comp - c.opdx * ixs * dXs);
    const T phi1 = rx_clamp(phi_o + c.dt * dphi, T(1e-4), T(1));
    const T k1 = rx_perm(c, phi1);
    out.Pf[q] = Pf1;
    out.phi[q] = phi1;
    out.Xs[q] = Xs1;
    if (kstored) out.k[q] = k1;
    if (out.R) out.R[q] = R;
    if (check) {
      chg = rx_change((double)rx_abs(phi1 - ph), (double)rx_abs(Pf1 - Pf) * (double)c.pf_iscale,
                      (double)rx_abs(Xs1 - Xs));
      kb = (double)(k1 * rx_rcp(rx_bp(c, phi1)));
    }
  }
  if (check) {
    block_max_atomic(chg, red + RED_V);
    block_max_atomic(kb, red + RED_MUMAX);
  }
}

template <class T>
__global__ void __launch_bounds__(256) k_rx_kbmax(Box b, RxCoef<T> c, const T* __restrict__ phi,
                                                  unsigned long long* red) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  double kb = 0.0;
  if (i < b.nx && j < b.ny && k < b.nz) {
    const T ph = phi[cidx(b, i, j, k)];
    kb = (double)(rx_perm(c, ph) / rx_bp(c, ph));
  }
  block_max_atomic(kb, red + RED_MUMAX);
}

template <class T>
__global__ void __launch_bounds__(256) k_rx_begin(Box b, RxCoef<T> c, const double* __restrict__ Pf,
                                                  const double* __restrict__ phi, const double* __restrict__ Xs,
                                                  T* Pf1, T* phi1, T* Xs1, T* Pf_o, T* phi_o, T* Xs_o, T* k1) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= b.nx || j >= b.ny || k >= b.nz) return;
  const long long q = cidx(b, i, j, k);
  const T a = (T)Pf[q], p = (T)phi[q], x = (T)Xs[q];
  Pf1[q] = a; phi1[q] = p; Xs1[q] = x;
  Pf_o[q] = a; phi_o[q] = p; Xs_o[q] = x;
  if (k1) k1[q] = rx_perm(c, p);
}

template <class T>
__global__ void __launch_bounds__(256) k_rx_end(Box b, const T* __restrict__ Pf, const T* __restrict__ phi,
                                                const T* __restrict__ Xs, const T* __restrict__ R, double* Pf1,
                                                double* phi1, double* Xs1, double* R1) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= b.nx || j >= b.ny || k >= b.nz) return;
  const long long q = cidx(b, i, j, k);
  Pf1[q] = (double)Pf[q]; phi1[q] = (double)phi[q]; Xs1[q] = (double)Xs[q]; R1[q] = (double)R[q];
}

namespace {
dim3 rx_grid(const Box& b) {
  return dim3((unsigned)((b.nx + 31) / 32), (unsigned)((b.ny + 7) / 8), (unsigned)b.nz);
}
}  // namespace

template <class T>
void rx_iter(cudaStream_t s, Box b, const RxCoef<T>& c, double dtau, const RxIn<T>& in, const RxOut<T>& out,
             unsigned long long* red, int check) {
  k_rx_iter<T><<<rx_grid(b), dim3(32, 8, 1), 0, s>>>(b, c, (T)dtau, in, out, red, check);
}
template <class T>
void rx_kbmax(cudaStream_t s, Box b, const RxCoef<T>& c, const T* phi, unsigned long long* red) {
  k_rx_kbmax<T><<<rx_grid(b), dim3(32, 8, 1), 0, s>>>(b, c, phi, red);
}
template <class T>
void rx_begin(cudaStream_t s, Box b, const RxCoef<T>& c, const double* Pf, const double* phi, const double* Xs,
              T* Pf1, T* phi1, T* Xs1, T* Pf_o, T* phi_o, T* Xs_o, T* k1) {
  k_rx_begin<T><<<rx_grid(b), dim3(32, 8, 1), 0, s>>>(b, c, Pf, phi, Xs, Pf1, phi1, Xs1, Pf_o, phi_o, Xs_o, k1);
}
template <class T>
void rx_end(cudaStream_t s, Box b, const T* Pf, const T* phi, const T* Xs, const T* R, double* Pf1, double* phi1,
            double* Xs1, double* R1) {
  k_rx_end<T><<<rx_grid(b), dim3(32, 8, 1), 0, s>>>(b, Pf, phi, Xs, R, Pf1, phi1, Xs1, R1);
}

#define RX_INSTANTIATE(T)                                                                                         \
  template void rx_iter<T>(cudaStream_t, Box, const RxCoef<T>&, double, const RxIn<T>&, const RxOut<T>&,         \
                           unsigned long long*, int);                                                            \
  template void rx_kbmax<T>(cudaStream_t, Box, const RxCoef<T>&, const T*, unsigned long long*);                \
  template void rx_begin<T>(cudaStream_t, Box, const RxCoef<T>&, const double*, const double*, const double*,   \
                            T*, T*, T*, T*, T*, T*, T*);                                                         \
  template void rx_end<T>(cudaStream_t, Box, const T*, const T*, const T*, const T*, double*, double*, double*,  \
                          double*);
RX_INSTANTIATE(double)
RX_INSTANTIATE(float)

}  // namespace pt
