// pt_batch.cuh — the batched ensemble: many independent instances (own grid, parameters and
// fields) advanced by one launch per PT phase over a flat work list of (instance, tile) items.
#pragma once

#include "pt_lean.cuh"

namespace pt {

// Per-instance descriptor read by the batched kernels (device memory, one per instance).
// Index 0/1 of the ping-pong sets is the parity of the iterate the launch reads.
struct BatchInst {
  Box b;
  LeanCoef<double> c;
  LeanCellIn<double> cin[2];
  LeanCellOut<double> cout[2];
  LeanFaceIn<double> fin[2];
  LeanPicardIn<double> pin[2];
  LeanCoefIn<double> kin;
  LeanCoefOut<double> kout;
  double *Vx, *Vy, *Vz, *Rx, *Ry, *Rz, *mu, *eta;
  unsigned long long* red;    // RED_N slots of this instance
  double tol;
  int max_iter;
  int gx, gy;                 // tiles per z-level for the current tile shape
  long long tile_base;        // first work item of this instance
  int own_lo[3], own_hi[3];   // cells [own_lo, own_hi) per direction enter the residual norms
};

// Per-instance status written by the convergence kernel (device memory).
struct BatchStatus {
  int active;                 // 1 while iterating
  int iters;                  // PT iterations taken when it stopped
  int status;                 // PT_OK, PT_ENOTCONV, PT_ENAN
  int pad;
  double res[4];              // residual norms of its last check (v, pt, pf, pic)
  unsigned long long t_start, t_stop;   // device %globaltimer (ns)
};

enum { BATCH_CELLS = 0, BATCH_FACES = 1, BATCH_PICARD = 2, BATCH_COEF = 3 };

// Launch `phase` over all active instances with parity `a` (0/1); tile shape bx x by.
void batch_phase(int bx, int by, int grid, cudaStream_t s, int phase, const BatchInst* inst,
                 const BatchStatus* st, int ninst, long long ntiles, int a, int check);
// After a check iteration: retire converged (or capped / non-finite) instances, add `nup` to
// the iteration counter of the active ones, clear their reduction slots. coupled: the instances
// are parts of one problem sharing instance 0's reduction slots and retire together.
void batch_converge(cudaStream_t s, const BatchInst* inst, BatchStatus* st, int ninst, int nup, int coupled);
// Start of a step: all instances active, counters zero, reduction slots clear, start time.
void batch_start(cudaStream_t s, const BatchInst* inst, BatchStatus* st, int ninst);
// Resident CTAs per SM of the batched cell kernel for a tile shape (occupancy of the widest phase).
int batch_blocks_per_sm(int bx, int by);

}  // namespace pt
