// pt_dd_kernels.cu — halo exchange, scatter and gather of the sub-domain form (the thesis's
// distributed-memory decomposition, Art. 1 Section 2.2 and Art. 2, run on one GPU).
//
// Part p owns global cells [a_p, b_p) per direction; its box covers [a_p - h_lo, b_p + h_hi)
// with h = 1 on every side that has a neighbour. Halo values are what a neighbouring GPU would
// send: after each PT iteration the exchange copies, for every box index of a part's halo
// slabs, the value at the same global index from the part that owns that cell. Every owned
// cell and every face next to one is then computed from the same inputs as in the undivided
// grid, by the same per-point code, so the result is bitwise that of the undivided run.
#include "pt_dd.cuh"

namespace pt {

namespace {

__device__ inline int owner_part(const DDTables& t, int gx, int gy, int gz) {
  return (t.own_z[gz] * t.parts_y + t.own_y[gy]) * t.parts_x + t.own_x[gx];
}

}  // namespace

__global__ void __launch_bounds__(256) k_dd_exchange(const BatchInst* __restrict__ inst,
                                                     const BatchStatus* __restrict__ st,
                                                     const HaloSlab* __restrict__ slabs, DDTables t, int a,
                                                     int set) {
  const HaloSlab s = slabs[blockIdx.y];
  if (!st[s.inst].active) return;
  const int ni = s.i1 - s.i0, nj = s.j1 - s.j0, nk = s.k1 - s.k0;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)ni * nj * nk) return;
  const int i = s.i0 + (int)(e % ni);
  const int j = s.j0 + (int)((e / ni) % nj);
  const int k = s.k0 + (int)(e / ((long long)ni * nj));
  const int* om = t.off + 3 * s.inst;
  const int gx = i + om[0], gy = j + om[1], gz = k + om[2];
  const int o = owner_part(t, gx, gy, gz);
  if (o == s.inst) return;
  const int* oo = t.off + 3 * o;
  const BatchInst& D = inst[s.inst];
  const BatchInst& S = inst[o];
  const long long qd = cidx(D.b, i, j, k);
  const long long qs = cidx(S.b, gx - oo[0], gy - oo[1], gz - oo[2]);
  if (set == DD_STATE) {
    const LeanCellOut<double>& d = D.cout[a];   // the iterate written by the iteration of parity a
    const LeanCellOut<double>& r = S.cout[a];
    d.Pt[qd] = r.Pt[qs];
    d.Pf[qd] = r.Pf[qs];
    d.phi[qd] = r.phi[qs];
    d.w[qd] = r.w[qs];
    d.perm[qd] = r.perm[qs];
    D.Vx[qd] = S.Vx[qs];
    D.Vy[qd] = S.Vy[qs];
    D.Vz[qd] = S.Vz[qs];
  } else {
    D.mu[qd] = S.mu[qs];
    D.eta[qd] = S.eta[qs];
  }
}

__global__ void __launch_bounds__(256) k_dd_scatter(Box g, Box l, int ox, int oy, int oz,
                                                    const DDFields* __restrict__ src,
                                                    const DDFields* __restrict__ dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i > l.nx || j > l.ny || k > l.nz) return;
  const long long ql = cidx(l, i, j, k), qg = cidx(g, i + ox, j + oy, k + oz);
  for (int f = 0; f < kDDFields; ++f)
    if (src->f[f]) dst->f[f][ql] = src->f[f][qg];
}

__global__ void __launch_bounds__(256) k_dd_gather(Box g, const Box* __restrict__ boxes, DDTables t,
                                                   const DDFields* __restrict__ dst,
                                                   const DDFields* __restrict__ parts) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i > g.nx || j > g.ny || k > g.nz) return;
  const int o = owner_part(t, i, j, k);
  const int* oo = t.off + 3 * o;
  const long long qg = cidx(g, i, j, k), ql = cidx(boxes[o], i - oo[0], j - oo[1], k - oo[2]);
  for (int f = 0; f < kDDFields - 1; ++f) dst->f[f][qg] = parts[o].f[f][ql];   // logk is read-only
}

void dd_exchange(cudaStream_t s, const BatchInst* inst, const BatchStatus* st, const HaloSlab* slabs, int nslabs,
                 int max_elems, const DDTables& t, int a, int set) {
  if (nslabs == 0) return;
  const dim3 grid((unsigned)((max_elems + 255) / 256), (unsigned)nslabs, 1);
  k_dd_exchange<<<grid, 256, 0, s>>>(inst, st, slabs, t, a, set);
}

void dd_scatter(cudaStream_t s, Box global, Box local, int ox, int oy, int oz, const DDFields* g,
                const DDFields* part) {
  const dim3 bl(32, 8, 1), gr((unsigned)((local.nx + 1 + 31) / 32), (unsigned)((local.ny + 1 + 7) / 8),
                              (unsigned)(local.nz + 1));
  k_dd_scatter<<<gr, bl, 0, s>>>(global, local, ox, oy, oz, g, part);
}

void dd_gather(cudaStream_t s, Box global, const Box* boxes, const DDTables& t, const DDFields* g,
               const DDFields* parts) {
  const dim3 bl(32, 8, 1), gr((unsigned)((global.nx + 1 + 31) / 32), (unsigned)((global.ny + 1 + 7) / 8),
                              (unsigned)(global.nz + 1));
  k_dd_gather<<<gr, bl, 0, s>>>(global, boxes, t, g, parts);
}

}  // namespace pt
