// pt_batch_kernels.cu — batched ensemble kernels (many independent instances of the Art. 1 solver).
//
// All instances of an ensemble are advanced by one launch per PT phase (cells, faces, Picard,
// coefficients). The work list is the concatenation of every instance's tiles (bx x by cells of
// one z-level of its padded box); a persistent grid (SMs x resident CTAs) walks it with a grid
// stride, so instances of uneven size share the GPU without per-instance launches. Each tile
// runs the same per-point code as the single-instance FP64-lean kernels (pt_lean_body.cuh) with
// its instance's box, coefficients and fields, so a batched instance reproduces its
// single-instance run bit for bit. Retired instances' tiles return at once.
#include "pt_batch.cuh"
#include "pt_lean_body.cuh"

namespace pt {

namespace {

__device__ inline int find_instance(const BatchInst* inst, int ninst, long long t) {
  int lo = 0, hi = ninst - 1;
  while (lo < hi) {  // last instance whose tile_base <= t
    const int mid = (lo + hi + 1) >> 1;
    if (inst[mid].tile_base <= t) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__device__ inline unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

}  // namespace

template <int BX, int BY, int PHASE>
__global__ void __launch_bounds__(BX * BY) k_batch_phase(const BatchInst* __restrict__ inst,
                                                         const BatchStatus* __restrict__ st, int ninst,
                                                         long long ntiles, int a, int check) {
  for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int m = find_instance(inst, ninst, t);
    if (!st[m].active) {                              // uniform over the CTA: a retired instance's
      // tiles are skipped in one step, to the first tile of the next instance this CTA visits
      const long long next = m + 1 < ninst ? inst[m + 1].tile_base : ntiles;
      const long long g = gridDim.x;
      t = next + (((long long)blockIdx.x - next) % g + g) % g - g;
      continue;
    }
    const BatchInst& I = inst[m];
    const long long local = t - I.tile_base;
    const long long per_z = (long long)I.gx * I.gy;
    const int k = (int)(local / per_z);
    const int r = (int)(local - (long long)k * per_z);
    const int ty = r / I.gx, tx = r - ty * I.gx;
    const int i = tx * BX + threadIdx.x, j = ty * BY + threadIdx.y;
    // ownership of the cell (i, j, k) and of its lower faces: a face counts when one of its two
    // cells is owned (halo cells of a sub-domain are recomputed by their owner)
    const bool ox = i >= I.own_lo[0] && i < I.own_hi[0], oy = j >= I.own_lo[1] && j < I.own_hi[1];
    const bool oz = k >= I.own_lo[2] && k < I.own_hi[2];
    const bool own = ox && oy && oz;
    if (PHASE == BATCH_CELLS) {
      double r_pt = 0.0, r_pf = 0.0;
      lean_cell_point(I.b, I.c, I.cin[a], I.cout[a], i, j, k, check, r_pt, r_pf);
      if (check) {
        block_max_atomic(own ? r_pt : 0.0, I.red + RED_PT);
        block_max_atomic(own ? r_pf : 0.0, I.red + RED_PF);
      }
    } else if (PHASE == BATCH_FACES) {
      double r_v = 0.0;
      const bool fx = i >= I.own_lo[0] && i <= I.own_hi[0], fy = j >= I.own_lo[1] && j <= I.own_hi[1];
      const bool fz = k >= I.own_lo[2] && k <= I.own_hi[2];
      const int mask = (fx && oy && oz ? 1 : 0) | (ox && fy && oz ? 2 : 0) | (ox && oy && fz ? 4 : 0);
      lean_face_point(I.b, I.c, I.fin[a], I.Vx, I.Vy, I.Vz, I.Rx, I.Ry, I.Rz, i, j, k, check, r_v, mask);
      if (check) block_max_atomic(r_v, I.red + RED_V);
    } else if (PHASE == BATCH_PICARD) {
      double rp = 1.0;
      lean_picard_point(I.b, I.c, I.pin[a], I.mu, I.eta, i, j, k, rp);
      block_max_log_atomic(own ? rp : 1.0, I.red + RED_PIC);
    } else {
      lean_coef_point(I.b, I.c, I.kin, I.kout, i, j, k);
    }
  }
}

__global__ void k_batch_converge(const BatchInst* __restrict__ inst, BatchStatus* __restrict__ st,
                                 int ninst, int nup, int coupled) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (coupled) {
    // parts of one problem: instance 0's slots hold the global norms; one decision for all
    if (m != 0 || !st[0].active) return;
    unsigned long long* red = inst[0].red;
    double v[4], worst = 0.0;
    bool finite = true;
    const int slot[4] = {RED_V, RED_PT, RED_PF, RED_PIC};
    for (int s = 0; s < 4; ++s) {
      v[s] = __longlong_as_double((long long)red[slot[s]]);
      finite = finite && isfinite(v[s]);
      worst = fmax(worst, v[s]);
      red[slot[s]] = 0ull;
    }
    const int it = st[0].iters + nup;
    const bool stop = !finite || worst < inst[0].tol || it >= inst[0].max_iter;
    const unsigned long long now = global_ns();
    for (int p = 0; p < ninst; ++p) {
      for (int s = 0; s < 4; ++s) st[p].res[s] = v[s];
      st[p].iters = it;
      if (stop) {
        st[p].active = 0;
        st[p].status = !finite ? -3 : (worst < inst[0].tol ? 0 : -2);
        st[p].t_stop = now;
      }
    }
    return;
  }
  if (m >= ninst || !st[m].active) return;
  unsigned long long* red = inst[m].red;
  double v[4];
  const int slot[4] = {RED_V, RED_PT, RED_PF, RED_PIC};
  double worst = 0.0;
  bool finite = true;
  for (int s = 0; s < 4; ++s) {
    v[s] = __longlong_as_double((long long)red[slot[s]]);
    finite = finite && isfinite(v[s]);
    worst = fmax(worst, v[s]);
    st[m].res[s] = v[s];
    red[slot[s]] = 0ull;
  }
  const int it = st[m].iters + nup;
  st[m].iters = it;
  if (!finite || worst < inst[m].tol || it >= inst[m].max_iter) {
    st[m].active = 0;
    st[m].status = !finite ? -3 : (worst < inst[m].tol ? 0 : -2);
    st[m].t_stop = global_ns();
  }
}

__global__ void k_batch_start(const BatchInst* __restrict__ inst, BatchStatus* __restrict__ st, int ninst) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= ninst) return;
  st[m].active = 1;
  st[m].iters = 0;
  st[m].status = -2;
  for (int s = 0; s < 4; ++s) st[m].res[s] = 0.0;
  for (int s = 0; s < RED_N; ++s) inst[m].red[s] = 0ull;
  st[m].t_start = global_ns();
  st[m].t_stop = 0ull;
}

template <int BX, int BY>
void launch_phase(int grid, cudaStream_t s, int phase, const BatchInst* inst, const BatchStatus* st, int ninst,
                  long long ntiles, int a, int check) {
  const dim3 bl(BX, BY, 1);
  switch (phase) {
    case BATCH_CELLS: k_batch_phase<BX, BY, BATCH_CELLS><<<grid, bl, 0, s>>>(inst, st, ninst, ntiles, a, check); break;
    case BATCH_FACES: k_batch_phase<BX, BY, BATCH_FACES><<<grid, bl, 0, s>>>(inst, st, ninst, ntiles, a, check); break;
    case BATCH_PICARD: k_batch_phase<BX, BY, BATCH_PICARD><<<grid, bl, 0, s>>>(inst, st, ninst, ntiles, a, check); break;
    default: k_batch_phase<BX, BY, BATCH_COEF><<<grid, bl, 0, s>>>(inst, st, ninst, ntiles, a, check); break;
  }
}

void batch_phase(int bx, int by, int grid, cudaStream_t s, int phase, const BatchInst* inst,
                 const BatchStatus* st, int ninst, long long ntiles, int a, int check) {
  if (bx == 32 && by == 4) launch_phase<32, 4>(grid, s, phase, inst, st, ninst, ntiles, a, check);
  else if (bx == 64 && by == 4) launch_phase<64, 4>(grid, s, phase, inst, st, ninst, ntiles, a, check);
  else launch_phase<32, 8>(grid, s, phase, inst, st, ninst, ntiles, a, check);
}

void batch_converge(cudaStream_t s, const BatchInst* inst, BatchStatus* st, int ninst, int nup, int coupled) {
  k_batch_converge<<<(ninst + 127) / 128, 128, 0, s>>>(inst, st, ninst, nup, coupled);
}

void batch_start(cudaStream_t s, const BatchInst* inst, BatchStatus* st, int ninst) {
  k_batch_start<<<(ninst + 127) / 128, 128, 0, s>>>(inst, st, ninst);
}

int batch_blocks_per_sm(int bx, int by) {
  int n = 0;
  cudaError_t e;
  if (bx == 32 && by == 4)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch_phase<32, 4, BATCH_CELLS>, 128, 0);
  else if (bx == 64 && by == 4)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch_phase<64, 4, BATCH_CELLS>, 256, 0);
  else
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch_phase<32, 8, BATCH_CELLS>, 256, 0);
  return (e == cudaSuccess && n > 0) ? n : 1;
}

}  // namespace pt
