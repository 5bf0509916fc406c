// rx_api.cu — host side of the reactive porosity-wave C ABI (include/porowave_rx.h).
//
// A context keeps the iterate in the workspace in the iteration type (FP64 or FP32): the
// caller's FP64 fields are read at the start of each physical step and written back at its
// end. Plain PT step: old-step copies, the first pseudo step from max k / beta_P, then fused
// iterations (ping-pong of Pf, phi, Xs); every nup-th iteration reads the change norm and
// max k / beta_P of the new porosity (pseudo step of the next iterations) back to the host.
// Multigrid step (contexts made by rx_mg_init): the old-step fields are restricted down the
// hierarchy once, then FAS V-cycles run, each replayed from a CUDA graph with one host read of
// the change norm.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>

#include "porowave_rx.h"
#include "rx.cuh"

using namespace pt;

namespace {
constexpr int kMgMaxLevels = 16;
// One grid of the multigrid hierarchy (level 0 aliases the context's own arrays).
struct MgLevel {
  Box b;
  RxCoef<double> cd;
  RxCoef<float> cf;
  void* Pf[2];
  void* phi[2];
  void* Xs[2];
  void *Pf_o, *phi_o, *Xs_o;
  void *fP, *fphi, *fX;              // FAS sources (coarse levels)
  void *Pf0, *phi0, *Xs0;            // restricted iterate before the coarse solve
  int cur;                           // which of the ping-pong pair holds the iterate
};
}  // namespace

struct rx_ctx {
  Box box;
  rx_phys phys;
  rx_num num;
  cudaStream_t stream;
  rx_fields f;                       // caller's FP64 fields
  bool fp32;
  RxCoef<double> cd;
  RxCoef<float> cf;
  void* Pf[2];                       // iteration-type arrays (double* or float*)
  void* phi[2];
  void* Xs[2];
  void *Pf_o, *phi_o, *Xs_o, *R;
  void* k[2];                        // k(phi) of the ping-pong iterates (plain iteration)
  unsigned long long* red;
  unsigned long long* h_red;
  double hmin2;
  long long launches;
  rx_mg mg;                          // multigrid settings (mg.levels = 0: plain context)
  MgLevel lv[kMgMaxLevels];
  // One V-cycle (reduction reset, kernels, read-back of the change norm) as a CUDA graph per
  // parity of the finest level's ping-pong index at its start; captured on a stream of the
  // context's own (the legacy default stream cannot be captured), replayed on `stream`.
  cudaStream_t cap;
  cudaGraphExec_t cyc[2];
  long long cyc_launches[2];
  int cyc_end[2];
};

namespace {

constexpr size_t kRxAlign = 256;
constexpr int kRxArrays = 12;        // Pf, phi, Xs, k (x2), Pf_o, phi_o, Xs_o, R
constexpr int kMgArrays = 15;        // per coarse level: Pf, phi, Xs (x2), old (3), f (3), u0 (3)

size_t rx_align(size_t x) { return (x + kRxAlign - 1) / kRxAlign * kRxAlign; }

bool rx_box(const pt_grid* g, Box* b) {
  const size_t n = pt_field_elems(g);
  if (n == 0) return false;
  b->nx = g->nx;
  b->ny = g->ny;
  b->nz = g->nz;
  b->px = pt_pitch_x(g);
  b->pxy = (long long)b->px * (g->ny + 1);
  b->n = (long long)n;
  return true;
}

template <class T>
void fill(RxCoef<T>& c, const pt_grid& g, const rx_phys& p, const rx_num& n) {
  c.rdx = (T)(g.nx / g.lx);
  c.rdy = (T)(g.ny / g.ly);
  c.rdz = (T)(g.nz / g.lz);
  c.rhofg = (T)(p.rhof * p.g);
  c.rphi0 = (T)(1.0 / p.phi0);
  c.k0 = (T)p.k0;
  c.reta = (T)(1.0 / p.eta);
  c.beta_d = (T)p.beta_d;
  c.beta_s = (T)p.beta_s;
  c.beta_f = (T)p.beta_f;
  c.beta_x = (T)p.beta_x;
  c.half_xs = (T)(0.5 * p.xs_max);
  c.xs_max = (T)p.xs_max;
  c.rtau = (T)(1.0 / p.tau);
  c.dt = (T)n.dt;
  c.rdt = (T)(1.0 / n.dt);
  c.dt_tau = (T)(n.dt / p.tau);
  c.r1dt_tau = (T)(1.0 / (1.0 + n.dt / p.tau));
  const double sr = 1.0 - p.rhos / (p.rhof * (1.0 + p.dX));
  c.sr_opdx = (T)(sr * (1.0 + p.dX));
  c.opdx = (T)(1.0 + p.dX);
  c.pf_iscale = (T)(1.0 / n.pf_scale);
  c.rdx2 = (T)((g.nx / g.lx) * (g.nx / g.lx));
  c.rdy2 = (T)((g.ny / g.ly) * (g.ny / g.ly));
  c.rdz2 = (T)((g.nz / g.lz) * (g.nz / g.lz));
  c.kc3 = (T)(p.k0 / (p.phi0 * p.phi0 * p.phi0));
  c.rhofg_dz = (T)(p.rhof * p.g * g.lz / g.nz);
}

bool num_ok(const rx_num* n) {
  return n && n->dt > 0 && std::isfinite(n->dt) && n->tol >= 0 && n->cfl_div > 0 && n->pf_scale > 0 &&
         n->max_iter >= 1 && n->nup >= 1 && (n->precision == PT_FP64 || n->precision == PT_FP32);
}

bool phys_ok(const rx_phys* p) {
  return p && p->phi0 > 0 && p->k0 > 0 && p->eta > 0 && p->rhof > 0 && p->tau > 0 && p->xs_max > 0 &&
         p->dX > -1.0;
}

int status(cudaError_t e) { return e == cudaSuccess ? PT_OK : PT_ECUDA; }

// max k / beta_P from the reduction block (after a synchronising read) -> pseudo step
int read_red(rx_ctx* c, double* change, double* kb) {
  cudaError_t e = cudaMemcpyAsync(c->h_red, c->red, RED_N * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                                  c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return PT_ECUDA;
  std::memcpy(change, &c->h_red[RED_V], sizeof(double));
  std::memcpy(kb, &c->h_red[RED_MUMAX], sizeof(double));
  return PT_OK;
}

double pseudo_step(const rx_ctx* c, double kb) { return c->hmin2 / kb / c->num.cfl_div; }

template <class T>
const RxCoef<T>& coef_of(const rx_ctx* c);
template <>
const RxCoef<double>& coef_of<double>(const rx_ctx* c) { return c->cd; }
template <>
const RxCoef<float>& coef_of<float>(const rx_ctx* c) { return c->cf; }

template <class T>
int run_step(rx_ctx* c, int32_t niter, bool converge, pt_report* rep) {
  const Box& b = c->box;
  const RxCoef<T>& k = coef_of<T>(c);
  T* Pf[2] = {(T*)c->Pf[0], (T*)c->Pf[1]};
  T* phi[2] = {(T*)c->phi[0], (T*)c->phi[1]};
  T* Xs[2] = {(T*)c->Xs[0], (T*)c->Xs[1]};
  // k travels with phi in FP64 only (see k_rx_iter)
  T* kk[2] = {sizeof(T) == 8 ? (T*)c->k[0] : nullptr, sizeof(T) == 8 ? (T*)c->k[1] : nullptr};
  rx_begin<T>(c->stream, b, k, c->f.Pf, c->f.phi, c->f.Xs, Pf[0], phi[0], Xs[0], (T*)c->Pf_o, (T*)c->phi_o,
              (T*)c->Xs_o, kk[0]);
  cudaMemsetAsync(c->red, 0, RED_N * sizeof(unsigned long long), c->stream);
  rx_kbmax<T>(c->stream, b, k, phi[0], c->red);
  c->launches += 2;
  double change = 0.0, kb = 0.0;
  int rc = read_red(c, &change, &kb);
  if (rc != PT_OK) return rc;
  if (!(kb > 0) || !std::isfinite(kb)) return PT_ENAN;
  double dtau = pseudo_step(c, kb);
  int cur = 0, it = 0;
  bool converged = false;
  change = 0.0;
  while (it < niter) {
    ++it;
    const int check = (it % c->num.nup) == 0;
    const bool last = it == niter;
    if (check) cudaMemsetAsync(c->red, 0, RED_N * sizeof(unsigned long long), c->stream);
    const RxIn<T> in{Pf[cur], phi[cur], Xs[cur], (const T*)c->Pf_o, (const T*)c->phi_o, (const T*)c->Xs_o, kk[cur]};
    const RxOut<T> out{Pf[1 - cur], phi[1 - cur], Xs[1 - cur], (check || last) ? (T*)c->R : nullptr, kk[1 - cur]};
    rx_iter<T>(c->stream, b, k, dtau, in, out, c->red, check);
    ++c->launches;
    cur = 1 - cur;
    if (check) {
      rc = read_red(c, &change, &kb);
      if (rc != PT_OK) return rc;
      if (!std::isfinite(change) || !std::isfinite(kb)) {
        rc = PT_ENAN;
        break;
      }
      dtau = pseudo_step(c, kb);
      if (converge && change < c->num.tol) {   // this check iteration wrote the final rate
        converged = true;
        break;
      }
    }
  }
  if (rc == PT_OK) {
    rx_end<T>(c->stream, b, Pf[cur], phi[cur], Xs[cur], (const T*)c->R, c->f.Pf, c->f.phi, c->f.Xs, c->f.R);
    ++c->launches;
    rc = status(cudaStreamSynchronize(c->stream));
  }
  if (rc == PT_OK && converge && !converged) rc = PT_ENOTCONV;
  if (rep) {
    std::memset(rep, 0, sizeof *rep);
    rep->iters = it;
    rep->status = rc;
    rep->res_v = change;
  }
  return rc;
}

// ---- multigrid ----

bool mg_ok(const pt_grid* g, const rx_mg* m) {
  if (!g || !m || m->levels < 1 || m->levels > kMgMaxLevels || m->nu_pre < 0 || m->nu_coarse < 1 ||
      m->max_cycles < 1 || !(m->omega > 0.0 && m->omega <= 1.0))
    return false;
  if (m->levels > 1 && m->nu_post < 1) return false;
  const int32_t s = 1 << (m->levels - 1);
  return g->nx % s == 0 && g->ny % s == 0 && g->nz % s == 0;
}

pt_grid level_grid(const pt_grid& g, int l) {
  pt_grid c = g;
  c.nx = g.nx >> l;
  c.ny = g.ny >> l;
  c.nz = g.nz >> l;
  return c;
}

size_t mg_extra_bytes(const pt_grid& g, int levels, size_t elem) {
  size_t s = 0;
  for (int l = 1; l < levels; ++l) {
    const pt_grid c = level_grid(g, l);
    s += kMgArrays * rx_align(pt_field_elems(&c) * elem);
  }
  return s;
}

template <class T>
const RxCoef<T>& lcoef(const MgLevel& L);
template <>
const RxCoef<double>& lcoef<double>(const MgLevel& L) { return L.cd; }
template <>
const RxCoef<float>& lcoef<float>(const MgLevel& L) { return L.cf; }

template <class T>
RxIn<T> level_in(const MgLevel& L) {
  return RxIn<T>{(const T*)L.Pf[L.cur], (const T*)L.phi[L.cur], (const T*)L.Xs[L.cur],
                 (const T*)L.Pf_o,      (const T*)L.phi_o,      (const T*)L.Xs_o};
}

// one weighted-Jacobi sweep on level l; the last sweep of a cycle on the finest level writes
// the rate and the change norm, the last sweep of a coarse level's visit writes the correction
// e = u' - u0 over u0 (the iterate itself is not needed after it)
template <class T>
void mg_sweep(rx_ctx* c, int l, bool last) {
  MgLevel& L = c->lv[l];
  const bool fine = l == 0;
  const MgSrc<T> src{(const T*)L.fP, (const T*)L.fphi, (const T*)L.fX};
  const MgE<T> e{(T*)L.Pf0, (T*)L.phi0, (T*)L.Xs0};
  const int cur = L.cur;
  const RxOut<T> out{(T*)L.Pf[1 - cur], (T*)L.phi[1 - cur], (T*)L.Xs[1 - cur], (fine && last) ? (T*)c->R : nullptr};
  mg_smooth<T>(c->stream, L.b, lcoef<T>(L), c->mg.omega, level_in<T>(L), fine ? nullptr : &src, out,
               (!fine && last) ? &e : nullptr, c->red, fine && last);
  if (fine || !last) L.cur = 1 - cur;
  ++c->launches;
}

template <class T>
void vcycle(rx_ctx* c, int l) {
  const rx_mg& m = c->mg;
  MgLevel& L = c->lv[l];
  if (l == m.levels - 1) {
    for (int s = 0; s < m.nu_coarse; ++s) mg_sweep<T>(c, l, s == m.nu_coarse - 1);
    return;
  }
  for (int s = 0; s < m.nu_pre; ++s) mg_sweep<T>(c, l, false);
  MgLevel& C = c->lv[l + 1];
  C.cur = 0;
  const MgCoarse<T> co{(T*)C.Pf[0], (T*)C.phi[0], (T*)C.Xs[0], (T*)C.Pf0, (T*)C.phi0,
                       (T*)C.Xs0,   (T*)C.fP,     (T*)C.fphi,  (T*)C.fX};
  const MgSrc<T> src{(const T*)L.fP, (const T*)L.fphi, (const T*)L.fX};
  mg_restrict<T>(c->stream, L.b, C.b, lcoef<T>(L), level_in<T>(L), l == 0 ? nullptr : &src, co);
  const RxIn<T> u0{(const T*)C.Pf0, (const T*)C.phi0, (const T*)C.Xs0,
                   (const T*)C.Pf_o, (const T*)C.phi_o, (const T*)C.Xs_o};
  mg_coarse_rhs<T>(c->stream, C.b, lcoef<T>(C), u0, co);
  c->launches += 2;
  vcycle<T>(c, l + 1);
  const MgCorr<T> e{(const T*)C.Pf0, (const T*)C.phi0, (const T*)C.Xs0};   // the correction, see mg_sweep
  mg_prolong<T>(c->stream, L.b, C.b, e, (T*)L.Pf[L.cur], (T*)L.phi[L.cur], (T*)L.Xs[L.cur]);
  ++c->launches;
  for (int s = 0; s < m.nu_post; ++s) mg_sweep<T>(c, l, s == m.nu_post - 1);
}

template <class T>
int build_cycle_graph(rx_ctx* c, int parity) {
  MgLevel& F = c->lv[0];
  F.cur = parity;
  const long long l0 = c->launches;
  const cudaStream_t s = c->stream;
  if (cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return PT_ECUDA;
  c->stream = c->cap;
  cudaMemsetAsync(c->red, 0, RED_N * sizeof(unsigned long long), c->cap);
  vcycle<T>(c, 0);
  cudaMemcpyAsync(c->h_red, c->red, RED_N * sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->cap);
  c->stream = s;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(c->cap, &g);
  if (e == cudaSuccess) e = cudaGraphInstantiate(&c->cyc[parity], g, 0);
  if (g) cudaGraphDestroy(g);
  c->cyc_launches[parity] = c->launches - l0;
  c->launches = l0;
  c->cyc_end[parity] = F.cur;
  F.cur = parity;                     // the captured cycle has not run yet
  if (e != cudaSuccess) {
    c->cyc[parity] = nullptr;
    return PT_ECUDA;
  }
  return PT_OK;
}

template <class T>
int run_mg(rx_ctx* c, int32_t ncycles, bool converge, pt_report* rep) {
  MgLevel& F = c->lv[0];
  F.cur = 0;
  rx_begin<T>(c->stream, c->box, lcoef<T>(F), c->f.Pf, c->f.phi, c->f.Xs, (T*)F.Pf[0], (T*)F.phi[0], (T*)F.Xs[0],
              (T*)F.Pf_o, (T*)F.phi_o, (T*)F.Xs_o, nullptr);
  ++c->launches;
  for (int l = 1; l < c->mg.levels; ++l) {
    const MgLevel& A = c->lv[l - 1];
    MgLevel& B = c->lv[l];
    mg_restrict_old<T>(c->stream, A.b, B.b, (const T*)A.Pf_o, (const T*)A.phi_o, (const T*)A.Xs_o, (T*)B.Pf_o,
                       (T*)B.phi_o, (T*)B.Xs_o);
    ++c->launches;
  }
  int rc = PT_OK, it = 0;
  bool converged = false;
  double change = 0.0;
  while (it < ncycles) {
    ++it;
    const int parity = F.cur;
    if (!c->cyc[parity]) {
      rc = build_cycle_graph<T>(c, parity);
      if (rc != PT_OK) break;
    }
    if (cudaGraphLaunch(c->cyc[parity], c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess) {
      rc = PT_ECUDA;
      break;
    }
    c->launches += c->cyc_launches[parity];
    F.cur = c->cyc_end[parity];
    std::memcpy(&change, &c->h_red[RED_V], sizeof(double));
    if (!std::isfinite(change)) {
      rc = PT_ENAN;
      break;
    }
    if (converge && change < c->num.tol) {
      converged = true;
      break;
    }
  }
  if (rc == PT_OK) {
    rx_end<T>(c->stream, c->box, (const T*)F.Pf[F.cur], (const T*)F.phi[F.cur], (const T*)F.Xs[F.cur],
              (const T*)c->R, c->f.Pf, c->f.phi, c->f.Xs, c->f.R);
    ++c->launches;
    rc = status(cudaStreamSynchronize(c->stream));
  }
  if (rc == PT_OK && converge && !converged) rc = PT_ENOTCONV;
  if (rep) {
    std::memset(rep, 0, sizeof *rep);
    rep->iters = it;
    rep->status = rc;
    rep->res_v = change;
  }
  return rc;
}

}  // namespace

extern "C" {

size_t rx_workspace_size(const pt_grid* grid, const rx_num* num) {
  Box b;
  if (!rx_box(grid, &b) || !num_ok(num)) return 0;
  const size_t elem = num->precision == PT_FP32 ? sizeof(float) : sizeof(double);
  return kRxArrays * rx_align((size_t)b.n * elem) + rx_align(RED_N * sizeof(unsigned long long));
}

int rx_init(rx_ctx** out, const pt_grid* grid, const rx_phys* phys, const rx_num* num, const rx_fields* fields,
            void* workspace, size_t bytes, void* stream) {
  if (!out) return PT_EINVAL;
  *out = nullptr;
  Box b;
  if (!rx_box(grid, &b) || !phys_ok(phys) || !num_ok(num) || !fields || !workspace) return PT_EINVAL;
  if (!fields->Pf || !fields->phi || !fields->Xs || !fields->R) return PT_EINVAL;
  if (((uintptr_t)workspace & (kRxAlign - 1)) != 0) return PT_EINVAL;
  if (bytes < rx_workspace_size(grid, num)) return PT_ESPACE;
  rx_ctx* c = new (std::nothrow) rx_ctx();
  if (!c) return PT_ECUDA;
  c->box = b;
  c->phys = *phys;
  c->num = *num;
  c->stream = (cudaStream_t)stream;
  c->f = *fields;
  c->fp32 = num->precision == PT_FP32;
  fill(c->cd, *grid, *phys, *num);
  fill(c->cf, *grid, *phys, *num);
  const double h = std::fmin(grid->lx / grid->nx, std::fmin(grid->ly / grid->ny, grid->lz / grid->nz));
  c->hmin2 = h * h;
  const size_t stride = rx_align((size_t)b.n * (c->fp32 ? sizeof(float) : sizeof(double)));
  char* w = (char*)workspace;
  void** slots[kRxArrays] = {&c->Pf[0], &c->Pf[1], &c->phi[0], &c->phi[1], &c->Xs[0], &c->Xs[1],
                             &c->Pf_o, &c->phi_o, &c->Xs_o, &c->R,      &c->k[0],  &c->k[1]};
  for (int s = 0; s < kRxArrays; ++s) *slots[s] = w + s * stride;
  c->red = (unsigned long long*)(w + kRxArrays * stride);
  c->launches = 0;
  if (cudaMallocHost(&c->h_red, RED_N * sizeof(unsigned long long)) != cudaSuccess) {
    delete c;
    return PT_ECUDA;
  }
  if (cudaMemsetAsync(workspace, 0, rx_workspace_size(grid, num), c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess) {
    cudaFreeHost(c->h_red);
    delete c;
    return PT_ECUDA;
  }
  *out = c;
  return PT_OK;
}

int rx_step(rx_ctx* c, pt_report* rep) {
  if (!c) return PT_EINVAL;
  return c->fp32 ? run_step<float>(c, c->num.max_iter, true, rep) : run_step<double>(c, c->num.max_iter, true, rep);
}

int rx_iterate(rx_ctx* c, int32_t niter, pt_report* rep) {
  if (!c || niter < 1) return PT_EINVAL;
  return c->fp32 ? run_step<float>(c, niter, false, rep) : run_step<double>(c, niter, false, rep);
}

long long rx_launch_count(const rx_ctx* c) { return c ? c->launches : -1; }

size_t rx_mg_workspace_size(const pt_grid* grid, const rx_num* num, const rx_mg* mg) {
  const size_t base = rx_workspace_size(grid, num);
  if (base == 0 || !mg_ok(grid, mg)) return 0;
  const size_t elem = num->precision == PT_FP32 ? sizeof(float) : sizeof(double);
  return base + mg_extra_bytes(*grid, mg->levels, elem);
}

int rx_mg_init(rx_ctx** out, const pt_grid* grid, const rx_phys* phys, const rx_num* num, const rx_mg* mg,
               const rx_fields* fields, void* workspace, size_t bytes, void* stream) {
  if (!out) return PT_EINVAL;
  *out = nullptr;
  const size_t need = rx_mg_workspace_size(grid, num, mg);
  if (need == 0) return PT_EINVAL;
  if (bytes < need) return PT_ESPACE;
  const size_t base = rx_workspace_size(grid, num);
  rx_ctx* c = nullptr;
  int rc = rx_init(&c, grid, phys, num, fields, workspace, base, stream);
  if (rc != PT_OK) return rc;
  c->mg = *mg;
  if (cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) != cudaSuccess) {
    c->cap = nullptr;
    rx_destroy(c);
    return PT_ECUDA;
  }
  MgLevel& F = c->lv[0];
  F.b = c->box;
  F.cd = c->cd;
  F.cf = c->cf;
  for (int s = 0; s < 2; ++s) {
    F.Pf[s] = c->Pf[s];
    F.phi[s] = c->phi[s];
    F.Xs[s] = c->Xs[s];
  }
  F.Pf_o = c->Pf_o;
  F.phi_o = c->phi_o;
  F.Xs_o = c->Xs_o;
  F.fP = F.fphi = F.fX = F.Pf0 = F.phi0 = F.Xs0 = nullptr;
  const size_t elem = c->fp32 ? sizeof(float) : sizeof(double);
  char* w = (char*)workspace + base;
  for (int l = 1; l < mg->levels; ++l) {
    MgLevel& L = c->lv[l];
    const pt_grid g = level_grid(*grid, l);
    rx_box(&g, &L.b);
    fill(L.cd, g, *phys, *num);
    fill(L.cf, g, *phys, *num);
    const size_t stride = rx_align((size_t)L.b.n * elem);
    void** slots[kMgArrays] = {&L.Pf[0], &L.Pf[1], &L.phi[0], &L.phi[1], &L.Xs[0], &L.Xs[1], &L.Pf_o, &L.phi_o,
                               &L.Xs_o,   &L.fP,     &L.fphi,   &L.fX,     &L.Pf0,   &L.phi0,  &L.Xs0};
    for (int s = 0; s < kMgArrays; ++s) *slots[s] = w + s * stride;
    w += kMgArrays * stride;
    L.cur = 0;
  }
  if (cudaMemsetAsync((char*)workspace + base, 0, need - base, c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess) {
    rx_destroy(c);
    return PT_ECUDA;
  }
  *out = c;
  return PT_OK;
}

int rx_mg_step(rx_ctx* c, pt_report* rep) {
  if (!c || c->mg.levels < 1) return PT_EINVAL;
  return c->fp32 ? run_mg<float>(c, c->mg.max_cycles, true, rep) : run_mg<double>(c, c->mg.max_cycles, true, rep);
}

int rx_mg_cycles(rx_ctx* c, int32_t ncycles, pt_report* rep) {
  if (!c || c->mg.levels < 1 || ncycles < 1) return PT_EINVAL;
  return c->fp32 ? run_mg<float>(c, ncycles, false, rep) : run_mg<double>(c, ncycles, false, rep);
}

void rx_destroy(rx_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  for (int p = 0; p < 2; ++p)
    if (c->cyc[p]) cudaGraphExecDestroy(c->cyc[p]);
  if (c->cap) cudaStreamDestroy(c->cap);
  cudaFreeHost(c->h_red);
  delete c;
}

}  // extern "C"
