// pt_lean_kernels.cu — the FP64-lean form of one PT iteration (two kernels per iteration).
//
// GB300 issues 2 FP64 lanes per SM per clock (~1.26 TFLOP/s) against ~6.7 TB/s of HBM, so an
// FP64 PT iteration is bound by FP64 instructions, not bytes. This form therefore trades bytes
// for FP64 work wherever a quantity changes less often than every iteration:
//   * coefficients that depend only on mu, eta and the old stresses (which change at Picard
//     updates and step starts) are kept in arrays refreshed by k_lean_coef:
//       centres  cm2 = 2 mu / (1 + xi), toa_ii = tau_o_ii xi / (1 + xi), idtp = 1 / dtau_Pt,
//                ieta = 1 / eta
//       edges    em2 = 2 mu_e / (1 + xi_e), toa_e = tau_o_e xi_e / (1 + xi_e)
//       faces    dtv = dtau_V (mean of the two centres' values)
//     with xi = mu / (G dtS) (Eq. 21, backward-Euler Maxwell step);
//   * k = k0 e^logk (phi / phi0)^3 (Eq. 23) and w = 1 / (1 - phi) travel with phi: the
//     porosity update of iteration k writes them for iteration k+1;
//   * the log-space porosity update (Eq. 22) is L = Lo + delta, so
//       phi'  = phi_o - (1 - phi_o) expm1(delta),   1 / (1 - phi') = (1 / (1 - phi_o)) e^-delta,
//     with both exponentials from one Taylor polynomial of exp (|delta| is tiny; large |delta|
//     falls back to CUDA's expm1) — no exp, no division, no cancellation in 1 - e^L;
//   * the largest neighbour permeability (pseudo-time step of Pf) is found with 64-bit
//     integer compares of the positive doubles' bit patterns (exact, off the FP64 pipe).
// k_lean_cells: Darcy flux and divergence (Eq. 20), div V and numerical div V (Eq. 17),
// local-implicit Pt, Pf (Eqs. 17-18), stresses at centres and the cell's three lower edges
// (Eq. 21), porosity (Eq. 22). k_lean_faces: momentum residual (Eq. 19) with Pt^{k+1},
// damped R, V^{k+1}. k_lean_picard: Picard targets (Eqs. 24-26) with log-space relaxation.
#include "pt_lean_body.cuh"

#include <algorithm>

namespace pt {

// ------------------------------------------------------------------------------ cells
template <class T>
__global__ void __launch_bounds__(256, 3) k_lean_cells(Box b, LeanCoef<T> c, LeanCellIn<T> in,
                                                    LeanCellOut<T> out, unsigned long long* red,
                                                    int check) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  double r_pt = 0.0, r_pf = 0.0;
  lean_cell_point(b, c, in, out, i, j, k, check, r_pt, r_pf);
  if (check) {
    block_max_atomic(r_pt, red + RED_PT);
    block_max_atomic(r_pf, red + RED_PF);
  }
}

// ------------------------------------------------- cells, z-marching with staged inputs
// The double-float cells kernel is limited by memory latency: with 80 registers a thread cannot
// hold all of its ~30 loads in flight, so memory time and issue time add up. Here each 32 x 8
// block marches through kLeanZChunk z-levels of its column; the 15 arrays read only at the
// thread's own index (kStageSlots, pointwise) of level k+1 are copied into a shared-memory stage
// by cp.async while level k computes (two stages, 61,440 B per block), so those loads take no
// registers and overlap the arithmetic. The neighbour arrays (V, Pt, Pf, phi, k) are loaded
// directly (z-neighbours of consecutive levels hit L1 / L2).
constexpr int kLeanZChunk = 16;
constexpr int kStageThreads = 256;
// stage the own-index values of the neighbour arrays too (22 slots, 102 registers, 2 blocks per
// SM: 10.4 ms per 511^3 launch) or only the pointwise arrays (15 slots, 80 registers, 3 blocks
// per SM: 9.9 ms)
constexpr bool kStageAll = false;
constexpr int kSlots = kStageAll ? (int)kStageSlotsAll : (int)kStageSlots;
constexpr int kZmarchBlocks = kStageAll ? 2 : 3;

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// Reads a staged slot from this level's stage (kSlots x kStageThreads values); slots outside the
// staged set are read from global memory (the stage holds nothing for them).
template <class T>
struct StagedPoint {
  const T* s;
  int tid;
  __device__ __forceinline__ T operator()(const T* a, long long q, int slot) const {
    return slot < kSlots ? s[slot * kStageThreads + tid] : a[q];
  }
};

template <class T>
__device__ __forceinline__ void stage_level(T* dst, const LeanCellIn<T>& in, long long q) {
  cp_async8(dst + S_PTO * kStageThreads, in.Pto + q);
  cp_async8(dst + S_PFO * kStageThreads, in.Pfo + q);
  cp_async8(dst + S_PHIO * kStageThreads, in.phio + q);
  cp_async8(dst + S_IETA * kStageThreads, in.ieta + q);
  cp_async8(dst + S_IDTP * kStageThreads, in.idtp + q);
  cp_async8(dst + S_CM2 * kStageThreads, in.cm2 + q);
  cp_async8(dst + S_TXX * kStageThreads, in.toa_xx + q);
  cp_async8(dst + S_TYY * kStageThreads, in.toa_yy + q);
  cp_async8(dst + S_TZZ * kStageThreads, in.toa_zz + q);
  cp_async8(dst + S_EXY * kStageThreads, in.em2_xy + q);
  cp_async8(dst + S_EXZ * kStageThreads, in.em2_xz + q);
  cp_async8(dst + S_EYZ * kStageThreads, in.em2_yz + q);
  cp_async8(dst + S_TXY * kStageThreads, in.toa_xy + q);
  cp_async8(dst + S_TXZ * kStageThreads, in.toa_xz + q);
  cp_async8(dst + S_TYZ * kStageThreads, in.toa_yz + q);
  if constexpr (kStageAll) {
    cp_async8(dst + S_VX * kStageThreads, in.Vx + q);
    cp_async8(dst + S_VY * kStageThreads, in.Vy + q);
    cp_async8(dst + S_VZ * kStageThreads, in.Vz + q);
    cp_async8(dst + S_PT * kStageThreads, in.Pt + q);
    cp_async8(dst + S_PF * kStageThreads, in.Pf + q);
    cp_async8(dst + S_PHI * kStageThreads, in.phi + q);
    cp_async8(dst + S_K * kStageThreads, in.perm + q);
  }
}

template <class T>
__global__ void __launch_bounds__(kStageThreads, kZmarchBlocks) k_lean_cells_zmarch(Box b, LeanCoef<T> c, LeanCellIn<T> in,
                                                                       LeanCellOut<T> out,
                                                                       unsigned long long* red, int check) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* stage = reinterpret_cast<T*>(smem_raw);   // [2][kSlots][kStageThreads]
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k0 = blockIdx.z * kLeanZChunk;
  const int k1 = min(k0 + kLeanZChunk, b.nz + 1);   // levels [k0, k1), all inside the box
  const bool active = i <= b.nx && j <= b.ny;      // the body's own index range
  constexpr int stage_elems = kSlots * kStageThreads;
  if (active) stage_level(stage + tid, in, cidx(b, i, j, k0));
  cp_async_commit();
  unsigned long long m_pt = 0ull, m_pf = 0ull;     // norms as bit patterns: a NaN stays the largest
  for (int k = k0; k < k1; ++k) {
    const int buf = (k - k0) & 1;
    if (active && k + 1 < k1) stage_level(stage + (buf ^ 1) * stage_elems + tid, in, cidx(b, i, j, k + 1));
    cp_async_commit();
    cp_async_wait_1();                              // this level's copies have landed
    double r_pt = 0.0, r_pf = 0.0;
    lean_cell_point(b, c, in, out, i, j, k, check, r_pt, r_pf, StagedPoint<T>{stage + buf * stage_elems, tid});
    const unsigned long long a = (unsigned long long)__double_as_longlong(r_pt);
    const unsigned long long d = (unsigned long long)__double_as_longlong(r_pf);
    m_pt = a > m_pt ? a : m_pt;
    m_pf = d > m_pf ? d : m_pf;
    __syncthreads();                                // every read of this stage precedes its refill
  }
  if (check) {
    block_max_atomic(__longlong_as_double((long long)m_pt), red + RED_PT);
    block_max_atomic(__longlong_as_double((long long)m_pf), red + RED_PF);
  }
}

// ------------------------------------------------------------------------------ faces
template <class T>
__global__ void __launch_bounds__(256) k_lean_faces(Box b, LeanCoef<T> c, LeanFaceIn<T> in,
                                                    T* __restrict__ Vx, T* __restrict__ Vy,
                                                    T* __restrict__ Vz, T* __restrict__ Rx,
                                                    T* __restrict__ Ry, T* __restrict__ Rz,
                                                    unsigned long long* red, int check) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  double r_v = 0.0;
  lean_face_point(b, c, in, Vx, Vy, Vz, Rx, Ry, Rz, i, j, k, check, r_v);
  if (check) block_max_atomic(r_v, red + RED_V);
}

// ------------------------------------------------------------------------------ Picard
template <class T>
__global__ void __launch_bounds__(256) k_lean_picard(Box b, LeanCoef<T> c, LeanPicardIn<T> in,
                                                     T* __restrict__ mu, T* __restrict__ eta,
                                                     unsigned long long* red) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  double m = 1.0;
  lean_picard_point(b, c, in, mu, eta, i, j, k, m);
  block_max_log_atomic(m, red + RED_PIC);
}

// --------------------------------------------------------------------- coefficient refresh
// From mu, eta and the raw old stresses (after a Picard update or a step start).
template <class T>
__global__ void __launch_bounds__(256) k_lean_coef(Box b, LeanCoef<T> c, LeanCoefIn<T> in,
                                                   LeanCoefOut<T> out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  lean_coef_point(b, c, in, out, i, j, k);
}

// ------------------------------------------------------------------------ step start
// phio = phi, Eo = 1 - phi, iEo = 1 / (1 - phi), w = iEo, k from phi; Pto, Pfo; max(mu).
template <class T>
__global__ void __launch_bounds__(256) k_lean_begin(Box b, LeanCoef<T> c, LeanBeginIn<T> in,
                                                    LeanBeginOut<T> out, unsigned long long* red) {
  using namespace lean_detail;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  double m = 0.0;
  if (i < b.nx && j < b.ny && k < b.nz) {
    const long long q = cidx(b, i, j, k);
    const T ph = in.phi[q];
    out.Pto[q] = in.Pt[q];
    out.Pfo[q] = in.Pf[q];
    out.phio[q] = ph;
    if constexpr (!LeanRecompute<T>::value) {   // the recomputing forms derive these from phi
      const T Eo = T(1.0) - ph;
      const T iEo = tdiv(T(1.0), Eo);
      out.Eo[q] = Eo;
      out.iEo[q] = iEo;
      out.w[q] = iEo;
    }
    if constexpr (LeanStoreK<T>::value) {
      const T r = ph * c.rphi0;
      out.perm[q] = (in.K0 ? in.K0[q] : c.k0) * r * r * r;
    }
    m = to_d(in.mu[q]);
  }
  block_max_atomic(m, red + RED_MUMAX);
}

// K0 = k0 e^logk / phi0^3 is folded into k = K0 phi^3; here K0 = k0 e^logk (phi0 via rphi0).
template <class T>
__global__ void k_lean_k0(Box b, double k0, const double* __restrict__ logk, T* __restrict__ K0) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i < b.nx && j < b.ny && k < b.nz) {
    const long long q = cidx(b, i, j, k);
    K0[q] = lean_detail::from_d<T>(k0 * exp(logk[q]));
  }
}

// ----------------------------------------------------------- FP64 <-> double-float copies
// Element-wise over whole padded boxes (padding included), one array per blockIdx.y.
__global__ void k_to_df64(DfCopy cp, long long n) {
  const double* __restrict__ src = cp.d[blockIdx.y];
  df64* __restrict__ dst = cp.f[blockIdx.y];
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    dst[e] = df64(src[e]);
}
__global__ void k_from_df64(DfCopy cp, long long n) {
  double* __restrict__ dst = cp.d[blockIdx.y];
  const df64* __restrict__ src = cp.f[blockIdx.y];
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    dst[e] = (double)src[e];
}

void df64_convert(cudaStream_t st, const DfCopy& cp, int narrays, long long n, bool to_df) {
  if (narrays <= 0) return;
  int sms = 152;
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long want = (n + 255) / 256;
  const unsigned gx = (unsigned)std::max(1LL, std::min<long long>(want, 8LL * sms));
  const dim3 gr(gx, (unsigned)narrays, 1);
  if (to_df) k_to_df64<<<gr, 256, 0, st>>>(cp, n);
  else k_from_df64<<<gr, 256, 0, st>>>(cp, n);
}

// ---------------------------------------------------------------- math check (test aid)
// One of the hand-written device routines applied element-wise, so that each can be compared
// with CUDA's own functions and with its stated error bound (the kernels inline the same code).
__global__ void k_math_check(int fn, const double* __restrict__ a, const double* __restrict__ b,
                             double* __restrict__ out, long long n) {
  using namespace lean_detail;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const double x = a[e], y = b ? b[e] : 0.0;
    double r = 0.0, p = 0.0, m = 0.0;
    df64 dp, dm;
    switch (fn) {
      case MATH_RCP_PSEUDO: r = rcp_pseudo(x); break;
      case MATH_RCP_FULL: r = rcp_full(x); break;
      case MATH_EXPM1_POS: expm1_pair(x, p, m); r = p; break;
      case MATH_EXPM1_NEG: expm1_pair(x, p, m); r = m; break;
      case MATH_DF_ADD: r = (double)(df64(x) + df64(y)); break;
      case MATH_DF_SUB: r = (double)(df64(x) - df64(y)); break;
      case MATH_DF_MUL: r = (double)(df64(x) * df64(y)); break;
      case MATH_DF_FMA: r = (double)fma(df64(x), df64(y), df64(x)); break;
      case MATH_DF_RCP: r = (double)df_rcp(df64(x)); break;
      case MATH_DF_SQRT: r = (double)df_sqrt(df64(x)); break;
      case MATH_DF_ROOT: r = (double)df_root(df64(x), (int)y); break;
      case MATH_DF_EXPM1_POS: expm1_pair(df64(x), dp, dm); r = (double)dp; break;
      case MATH_DF_EXPM1_NEG: expm1_pair(df64(x), dp, dm); r = (double)dm; break;
      default: r = nan(""); break;
    }
    out[e] = r;
  }
}

void math_check(cudaStream_t st, int fn, const double* a, const double* b, double* out, long long n) {
  if (n <= 0) return;
  const unsigned g = (unsigned)std::min<long long>((n + 255) / 256, 4096);
  k_math_check<<<g, 256, 0, st>>>(fn, a, b, out, n);
}

template <class T>
void lean_cells(dim3 gr, dim3 bl, cudaStream_t st, Box b, const LeanCoef<T>& c, const LeanCellIn<T>& in,
                const LeanCellOut<T>& out, unsigned long long* red, int check) {
  k_lean_cells<T><<<gr, bl, 0, st>>>(b, c, in, out, red, check);
}
// The double-float form's cells launch: the z-marching staged kernel (the block shape stays 32 x 8).
template <>
void lean_cells<df64>(dim3 gr, dim3 bl, cudaStream_t st, Box b, const LeanCoef<df64>& c, const LeanCellIn<df64>& in,
                      const LeanCellOut<df64>& out, unsigned long long* red, int check) {
  const int smem = 2 * kSlots * kStageThreads * (int)sizeof(df64);
  cudaFuncSetAttribute(k_lean_cells_zmarch<df64>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  const dim3 g(gr.x, gr.y, (unsigned)((b.nz + 1 + kLeanZChunk - 1) / kLeanZChunk));
  k_lean_cells_zmarch<df64><<<g, dim3(32, 8, 1), smem, st>>>(b, c, in, out, red, check);
}
template <class T>
void lean_faces(dim3 gr, dim3 bl, cudaStream_t st, Box b, const LeanCoef<T>& c, const LeanFaceIn<T>& in,
                T* Vx, T* Vy, T* Vz, T* Rx, T* Ry, T* Rz, unsigned long long* red, int check) {
  k_lean_faces<T><<<gr, bl, 0, st>>>(b, c, in, Vx, Vy, Vz, Rx, Ry, Rz, red, check);
}
template <class T>
void lean_picard(dim3 gr, dim3 bl, cudaStream_t st, Box b, const LeanCoef<T>& c, const LeanPicardIn<T>& in,
                 T* mu, T* eta, unsigned long long* red) {
  k_lean_picard<T><<<gr, bl, 0, st>>>(b, c, in, mu, eta, red);
}
template <class T>
void lean_coef(dim3 gr, dim3 bl, cudaStream_t st, Box b, const LeanCoef<T>& c, const LeanCoefIn<T>& in,
               const LeanCoefOut<T>& out) {
  k_lean_coef<T><<<gr, bl, 0, st>>>(b, c, in, out);
}
template <class T>
void lean_begin(dim3 gr, dim3 bl, cudaStream_t st, Box b, const LeanCoef<T>& c, const LeanBeginIn<T>& in,
                const LeanBeginOut<T>& out, unsigned long long* red) {
  k_lean_begin<T><<<gr, bl, 0, st>>>(b, c, in, out, red);
}
template <class T>
void lean_k0(dim3 gr, dim3 bl, cudaStream_t st, Box b, double k0, const double* logk, T* K0) {
  k_lean_k0<T><<<gr, bl, 0, st>>>(b, k0, logk, K0);
}

template void lean_cells<double>(dim3, dim3, cudaStream_t, Box, const LeanCoef<double>&, const LeanCellIn<double>&,
                                 const LeanCellOut<double>&, unsigned long long*, int);
template void lean_faces<double>(dim3, dim3, cudaStream_t, Box, const LeanCoef<double>&, const LeanFaceIn<double>&,
                                 double*, double*, double*, double*, double*, double*, unsigned long long*, int);
template void lean_picard<double>(dim3, dim3, cudaStream_t, Box, const LeanCoef<double>&, const LeanPicardIn<double>&,
                                  double*, double*, unsigned long long*);
template void lean_coef<double>(dim3, dim3, cudaStream_t, Box, const LeanCoef<double>&, const LeanCoefIn<double>&,
                                const LeanCoefOut<double>&);
template void lean_begin<double>(dim3, dim3, cudaStream_t, Box, const LeanCoef<double>&, const LeanBeginIn<double>&,
                                 const LeanBeginOut<double>&, unsigned long long*);
template void lean_k0<double>(dim3, dim3, cudaStream_t, Box, double, const double*, double*);

template void lean_faces<df64>(dim3, dim3, cudaStream_t, Box, const LeanCoef<df64>&, const LeanFaceIn<df64>&,
                                 df64*, df64*, df64*, df64*, df64*, df64*, unsigned long long*, int);
template void lean_picard<df64>(dim3, dim3, cudaStream_t, Box, const LeanCoef<df64>&, const LeanPicardIn<df64>&,
                                  df64*, df64*, unsigned long long*);
template void lean_coef<df64>(dim3, dim3, cudaStream_t, Box, const LeanCoef<df64>&, const LeanCoefIn<df64>&,
                                const LeanCoefOut<df64>&);
template void lean_begin<df64>(dim3, dim3, cudaStream_t, Box, const LeanCoef<df64>&, const LeanBeginIn<df64>&,
                                 const LeanBeginOut<df64>&, unsigned long long*);
template void lean_k0<df64>(dim3, dim3, cudaStream_t, Box, double, const double*, df64*);

}  // namespace pt
