// pt_dd.cuh — the sub-domain (halo-exchange) form: the grid split into parts that are advanced
// together by the batched kernels, each part a padded box with a one-cell halo on its internal
// sides, refreshed from the owning part after every PT iteration (pt_dd_kernels.cu).
#pragma once

#include "pt_batch.cuh"

namespace pt {

constexpr int kDDFields = 15;   // the 14 caller fields and logk

// Box-index range [i0, i1) x [j0, j1) x [k0, k1) of part `inst` whose values are halo values.
struct HaloSlab {
  int inst, i0, i1, j0, j1, k0, k1;
};

// Decomposition tables (device memory).
struct DDTables {
  const int* own_x;        // part coordinate along x owning global box index G (nx + 1 entries)
  const int* own_y;
  const int* own_z;
  const int* off;          // 3 per part: global box index of the part's local index 0
  int parts_x, parts_y;    // part id = (pz * parts_y + py) * parts_x + px
};

// Field pointers of one part (device memory): the 14 caller fields and logk (may be null).
struct DDFields {
  double* f[kDDFields];
};

enum { DD_STATE = 0, DD_VISC = 1 };

// Halo refresh of the iterate written by an iteration of parity a (DD_STATE: V, Pt, Pf, phi,
// 1/(1-phi), k) or of mu, eta after a Picard update (DD_VISC). Parts that have retired skip.
void dd_exchange(cudaStream_t s, const BatchInst* inst, const BatchStatus* st, const HaloSlab* slabs, int nslabs,
                 int max_elems, const DDTables& t, int a, int set);
// Global fields -> part m (its whole box, halos included).
void dd_scatter(cudaStream_t s, Box global, Box local, int ox, int oy, int oz, const DDFields* g,
                const DDFields* part);
// Parts -> global fields: every global box index from the part that owns it.
void dd_gather(cudaStream_t s, Box global, const Box* boxes, const DDTables& t, const DDFields* g,
               const DDFields* parts);

}  // namespace pt
