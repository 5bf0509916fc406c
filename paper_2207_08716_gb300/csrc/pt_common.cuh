// pt_common.cuh — device-side definitions shared by the solver's kernels.
//
// Padded box layout: every staggered field of an nx x ny x nz grid lives in a box of
// px x py x (nz + 1) elements, px = roundup(nx + 1, 16), py = ny + 1, element (i, j, k) at
// i + px * (j + py * k). A cell (i, j, k) and its lower x-, y-, z-faces and lower xy-, xz-,
// yz-edges share one index, so every stencil offset is one of +-1, +-px, +-pxy.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace pt {

struct Box {
  int nx, ny, nz;
  int px;             // x pitch (elements)
  long long pxy;      // px * py
  long long n;        // elements per field
};

// Scalars of one physical step, in FP64 (the FP32 path converts what it needs).
struct Coef {
  double rdx, rdy, rdz;        // 1 / dx, ...
  double h2;                   // min(dx, dy, dz)^2
  double phi0, rphi0, k0, mu0, eta0, R_weak, n_pow, tau0;
  double alpha, B, beta_d, beta_phi, G;
  double rhof_g, rhos_g, rho_bg_g;  // densities times gravity, background phi0 rho_f + (1-phi0) rho_s
  int powerlaw_on, compaction_on;
  double dt, rdt;
  double damp_x, damp_y, damp_z, rho_i, rrho_i, beta_n, rel_mu, rel_eta;
  double dtauv_fac;            // cfl_v h^2 rho_i / (1 + beta_n):   dtau_V = dtauv_fac / mu
  double dtaupt_fac;           // dtpt_scale (1 + beta_n) / nz:     dtau_Pt = dtaupt_fac * mu
  double dtaupf_fac;           // cfl_pf h^2 (1 + beta_d B / alpha): dtau_Pf = dtaupf_fac / kmax
  double rGdtS;                // 1 / (G dtS): xi = mu / (G dtS)
  double ebg;                  // background xy strain rate tau_bg / (2 mu0) (Eqs. 32-33)
  int bg_on;                   // tau_bg != 0: wall xy-edges carry the background stress
};

// Mean shear viscosity over the centres next to the xy-edge with box index q = (i, j, .)
// that lie inside the grid (four inside, two on a wall, one in a corner), in a fixed order.
template <class T>
__device__ inline double edge_mean_mu_xy(const Box& b, const T* mu, long long q, int i, int j) {
  double s = 0.0;
  int n = 0;
  if (i > 0 && j > 0) { s += (double)mu[q - 1 - b.px]; ++n; }
  if (i < b.nx && j > 0) { s += (double)mu[q - b.px]; ++n; }
  if (i > 0 && j < b.ny) { s += (double)mu[q - 1]; ++n; }
  if (i < b.nx && j < b.ny) { s += (double)mu[q]; ++n; }
  return s / n;
}

__host__ __device__ inline long long cidx(const Box& b, int i, int j, int k) {
  return (long long)i + (long long)b.px * j + b.pxy * k;
}

// Indices of the residual max-norm slots in the device reduction block.
enum { RED_V = 0, RED_PT = 1, RED_PF = 2, RED_PIC = 3, RED_MUMAX = 4, RED_GMAX = 5, RED_N = 8 };

// Max-reduction of non-negative doubles through their bit patterns (monotone for x >= 0; a
// NaN from fabs has the largest pattern and therefore surfaces in the norm). Every thread of
// the block must call it (it synchronises the block).
template <bool LOG>
__device__ inline void block_max_atomic_impl(double v, unsigned long long* slot) {
  unsigned long long u = (unsigned long long)__double_as_longlong(v);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long w = __shfl_xor_sync(0xffffffffu, u, o);
    u = w > u ? w : u;
  }
  __shared__ unsigned long long warp_max[32];
  const int lane = (threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z)) & 31;
  const int warp = (threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z)) >> 5;
  const int nwarps = (blockDim.x * blockDim.y * blockDim.z + 31) >> 5;
  if (lane == 0) warp_max[warp] = u;
  __syncthreads();
  if (warp == 0) {
    u = lane < nwarps ? warp_max[lane] : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      unsigned long long w = __shfl_xor_sync(0xffffffffu, u, o);
      u = w > u ? w : u;
    }
    if (LOG) {
      if (lane == 0) {
        const double l = log(__longlong_as_double((long long)u));
        if (!(l <= 0.0)) atomicMax(slot, (unsigned long long)__double_as_longlong(l));   // > 0 or NaN
      }
    } else if (lane == 0 && u != 0ull) {
      atomicMax(slot, u);
    }
  }
  __syncthreads();  // warp_max may be reused by the next call in the same kernel
}

__device__ inline void block_max_atomic(double v, unsigned long long* slot) { block_max_atomic_impl<false>(v, slot); }

// The same for values >= 1 whose log goes into the slot: log is monotone, so the block takes the
// max of the values and one thread the log (a NaN still has the largest pattern). Every thread of
// the block calls it; a thread with nothing to contribute passes 1.
__device__ inline void block_max_log_atomic(double v, unsigned long long* slot) { block_max_atomic_impl<true>(v, slot); }

}  // namespace pt
