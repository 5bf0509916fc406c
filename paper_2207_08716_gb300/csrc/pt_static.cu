// pt_static.cu — residual max-norms of a solver state without any memory allocation.
//
// Who needs this: a caller that cannot allocate device memory at the moment it wants the
// norms, for example a health check inside a long run whose HBM is entirely held by a pool
// allocator (a raw cudaMalloc would fail or fragment that pool), or a timing-critical loop
// that cannot afford the implicit device synchronisation of cudaMalloc / cudaFree. Such a
// caller passes its fields and the old-step fields and gets the four norms back; the kernels'
// intermediate arrays (permeability, density, stresses, updated pressures) and the reduction
// block live in one file-scope device array of fixed size, so nothing is allocated, no
// workspace and no context is needed.
//
// The array is part of this library's device image: every GPU that loads the library holds
// it (PT_RESIDUAL_STATIC_SCRATCH_BYTES) until the process exits. All calls share it and it
// keeps the last call's contents: the reduction block is cleared at the start of every call,
// and calls whose device work overlaps (other streams, other host threads) race on it.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "../../include/porowave_pt.h"
#include "pt_common.cuh"
#include "pt_kernels.cuh"
#include "pt_host.h"

using namespace pt;

namespace {

static __device__ __align__(256) unsigned char g_residual_scratch[PT_RESIDUAL_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 128;
constexpr size_t kAlign = 256;
constexpr int kScratchArrays = 10;  // perm, rog, Pt1, Pf1, txx, tyy, tzz, txy, txz, tyz

std::mutex g_mutex;
void* g_device_addr[kMaxDevices];  // address of g_residual_scratch on each device, or null

// Device address of the scratch array on the current device. Host code cannot use the array's
// name as a device address (it is a host-side stand-in), so the address is looked up once per
// device with that device current, and cached.
int scratch_on_current_device(unsigned char** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return PT_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return PT_EINVAL;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_device_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_residual_scratch);
    if (e != cudaSuccess || !p) return PT_ECUDA;
    g_device_addr[dev] = p;
  }
  *out = (unsigned char*)g_device_addr[dev];
  return PT_OK;
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// The argument rules of pt_init (grid_ok, phys_ok, the numerics' positive pseudo-step factors,
// 16-byte aligned non-null fields), plus a positive finite stress sub-step.
bool args_ok(const pt_grid* g, const pt_phys* p, const pt_num* n, const pt_fields* f,
             const pt_old_fields* o, double dtS) {
  if (!grid_ok(g) || !phys_ok(p) || !n || !f || !o) return false;
  if (!(n->dt > 0) || !std::isfinite(n->dt) || !(n->rho_i > 0) || !(n->cfl_v > 0) || !(n->cfl_pf > 0) ||
      !(n->dtpt_scale > 0))
    return false;
  if (!(dtS > 0) || !std::isfinite(dtS)) return false;
  const void* ptrs[] = {f->Vx, f->Vy, f->Vz, f->Pt, f->Pf, f->phi, f->mu, f->eta, o->Pto,
                        o->Pfo, o->txxo, o->tyyo, o->tzzo, o->txyo, o->txzo, o->tyzo};
  for (const void* q : ptrs)
    if (!q || !aligned16(q)) return false;
  if (f->logk && !aligned16(f->logk)) return false;
  return true;
}

}  // namespace

extern "C" int pt_residual_static(const pt_grid* grid, const pt_phys* phys, const pt_num* num,
                                  const pt_fields* f, const pt_old_fields* old, double dtS,
                                  void* stream_handle, pt_report* rep) {
  if (!rep) return PT_EINVAL;
  std::memset(rep, 0, sizeof *rep);
  if (!args_ok(grid, phys, num, f, old, dtS)) return rep->status = PT_EINVAL;
  const Box b = make_box(grid);
  const size_t stride = align_up((size_t)b.n * sizeof(double), kAlign);
  if (kScratchArrays * stride + kAlign > (size_t)PT_RESIDUAL_STATIC_SCRATCH_BYTES)
    return rep->status = PT_ESPACE;

  unsigned char* base = nullptr;
  int rc = scratch_on_current_device(&base);
  if (rc != PT_OK) return rep->status = rc;
  double* s[kScratchArrays];
  for (int i = 0; i < kScratchArrays; ++i) s[i] = (double*)(base + i * stride);
  unsigned long long* red = (unsigned long long*)(base + kScratchArrays * stride);

  cudaStream_t st = (cudaStream_t)stream_handle;
  const Coef k = make_coef(*grid, *phys, *num, dtS);   // the same builder as pt_init's
  const dim3 bl(32, 8, 1);
  const dim3 gr((unsigned)((b.nx + 1 + 31) / 32), (unsigned)((b.ny + 1 + 7) / 8), (unsigned)(b.nz + 1));
  double *perm = s[0], *rog = s[1], *Pt1 = s[2], *Pf1 = s[3];
  double *txx = s[4], *tyy = s[5], *tzz = s[6], *txy = s[7], *txz = s[8], *tyz = s[9];

  cudaError_t e = cudaMemsetAsync(red, 0, RED_N * sizeof(unsigned long long), st);
  if (e != cudaSuccess) return rep->status = PT_ECUDA;
  k_perm<<<gr, bl, 0, st>>>(b, k, f->phi, f->logk, perm, rog);
  CentreIn ci{f->Vx, f->Vy, f->Vz, f->Pt, f->Pf, f->phi, f->mu, f->eta, perm,
              old->Pto, old->Pfo, old->txxo, old->tyyo, old->tzzo};
  CentreOut co{Pt1, Pf1, txx, tyy, tzz};
  k_centres<<<gr, bl, 0, st>>>(b, k, ci, co, 1, red, 1);
  EdgeIn ei{f->Vx, f->Vy, f->Vz, f->mu, old->txyo, old->txzo, old->tyzo};
  EdgeOut eo{txy, txz, tyz};
  k_edges<<<gr, bl, 0, st>>>(b, k, ei, eo);
  FaceIn fi{txx, tyy, tzz, txy, txz, tyz, f->Pt, rog, f->mu};
  k_residual_faces<<<gr, bl, 0, st>>>(b, k, fi, red);
  PicardIn pi{txx, tyy, tzz, txy, txz, tyz, f->phi, f->Pt, f->Pf};
  k_picard<<<gr, bl, 0, st>>>(b, k, pi, f->mu, f->eta, red, 0);  // update = 0: nothing written
  e = cudaGetLastError();
  unsigned long long h[RED_N];
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, red, sizeof h, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return rep->status = PT_ECUDA;
  double v[4];
  const int slot[4] = {RED_V, RED_PT, RED_PF, RED_PIC};
  for (int i = 0; i < 4; ++i) std::memcpy(&v[i], &h[slot[i]], sizeof(double));
  rep->res_v = v[0];
  rep->res_pt = v[1];
  rep->res_pf = v[2];
  rep->res_pic = v[3];
  const bool finite = std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]) && std::isfinite(v[3]);
  return rep->status = finite ? PT_OK : PT_ENAN;
}
