// Host side of the C ABI declared in include/ddlra.h: planning, allocation,
// initial factors, the time-step driver (optionally replayed from a CUDA graph),
// observables and factor exchange.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/ddlra.h"
#include "dd_internal.cuh"
#include "dd_launch.h"

namespace {

thread_local std::string g_err;

dd_status fail(dd_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

#define DD_CUDA(call)                                                                  \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return fail(DD_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));    \
  } while (0)

struct SubGeo {
  int N, nxk, nyk, cx0, cy0, rowoff;
  int nb[4];
  int inst, rlo, rhi, raug, fbase, fnx;
  double hx, hy, dt, sh;
};

// The device allocator set by dd_set_allocator (both callbacks null: cudaMalloc / cudaFree).
// A solver copies the one in effect when it is created and releases its memory through that
// copy; t_alloc points at the copy of the solver being created on this thread.
std::mutex g_alloc_mu;
dd_allocator g_alloc = {nullptr, nullptr, nullptr};
thread_local const dd_allocator* t_alloc = nullptr;

template <class T>
cudaError_t dalloc(T** p, size_t count) {
  const size_t bytes = sizeof(T) * std::max<size_t>(count, 1);
  if (t_alloc && t_alloc->alloc) {
    void* q = t_alloc->alloc(bytes, t_alloc->ctx);
    *p = nullptr;
    if (!q) return cudaErrorMemoryAllocation;
    if (reinterpret_cast<uintptr_t>(q) & 255u) {     // the tile loads need aligned rows
      t_alloc->release(q, t_alloc->ctx);
      return cudaErrorInvalidValue;
    }
    *p = static_cast<T*>(q);
    return cudaSuccess;
  }
  return cudaMalloc(reinterpret_cast<void**>(p), bytes);
}

void dfree(const dd_allocator& a, void* p) {
  if (!p) return;
  if (a.alloc) a.release(p, a.ctx);
  else cudaFree(p);
}

double legendre(int l, double x) {
  if (l == 0) return 1.0;
  double p0 = 1.0, p1 = x;
  for (int k = 1; k < l; ++k) {
    double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
    p0 = p1;
    p1 = p2;
  }
  return p1;
}

}  // namespace

struct dd_dlra {
  // problem
  int device;
  int ninst;
  std::vector<int> inst_sub0, inst_nsub, inst_fbase, inst_nx, inst_ny;
  long ncells_out;
  int nx, ny, tx, ty, nsub, n;
  double hx, hy, sh, ssum;
  dd_options opt;
  int RC, RS, MC, r_floor, maxlines, maxN;
  long Ntot;
  std::vector<SubGeo> geo;
  std::vector<double> sw_host;
  cudaStream_t stream;
  dd_allocator alloc;   // the device allocator in effect at create
  int use_graph;
  cudaGraphExec_t graph_exec;
  bool graph_ready;
  // device: geometry
  int *d_N, *d_nxk, *d_nyk, *d_rowoff, *d_nb, *d_cx0, *d_cy0;
  int *d_rlo, *d_rhi, *d_raug, *d_fbase, *d_fnx;
  double *d_hxk, *d_hyk, *d_dtk, *d_shk;
  double* d_dth;   // dt / 2 per subdomain (the half steps of the Strang splitting)
  // physical inflow per subdomain and side (x-lo, x-hi, y-lo, y-hi), null without inflow
  int* d_infl_on;
  double *d_infl_g, *d_infl_hw, *d_infl_sc;
  // device: problem data
  double *d_ox, *d_oy, *d_w, *d_sw, *d_sig_s, *d_sig_t, *d_sQ, *d_angcand;
  int n_angcand, angcand_complete, n_angorth;
  // device: state, double buffered
  double *d_X[2], *d_V[2], *d_S[2];
  int* d_r[2];
  // device: workspace
  double *d_L0, *d_Hw, *d_Hwa, *d_Vh, *d_K, *d_X1, *d_L, *d_V1, *d_Kb, *d_sm, *d_part;
  double *d_sig, *d_rho, *d_fluxw;
  int *d_m, *d_rt, *d_rx, *d_rc, *d_p, *d_keep, *d_cexp, *d_kcn, *d_kcur;
  // spatial completion family: cosine tables per subdomain
  double* d_sptab;
  long long* d_spoff;
  int* d_spnf;
  double *d_dm, *d_mvec;
  unsigned* d_status;
  double* d_noalloc;   // device address of the allocation-free readout's scratch array
  double tune_ms[8];   // the autotuner's timings (dd_dlra_tuning)
  dd::Problem P;
};

namespace {

dd::PhaseBufs bufs(dd_dlra* h, int in, int out) {
  dd::PhaseBufs B;
  B.X = h->d_X[in]; B.V = h->d_V[in]; B.S = h->d_S[in]; B.r = h->d_r[in];
  B.Xo = h->d_X[out]; B.Vo = h->d_V[out]; B.So = h->d_S[out]; B.ro = h->d_r[out];
  B.L0 = h->d_L0; B.Hw = h->d_Hw; B.Hwa = h->d_Hwa; B.Vh = h->d_Vh; B.K = h->d_K;
  B.X1 = h->d_X1; B.L = h->d_L; B.V1 = h->d_V1; B.Kb = h->d_Kb; B.sm = h->d_sm;
  B.part = h->d_part; B.m = h->d_m; B.rt = h->d_rt; B.rx = h->d_rx; B.rc = h->d_rc;
  B.sig = h->d_sig; B.p = h->d_p; B.status = h->d_status;
  B.keep = h->d_keep; B.kcn = h->d_kcn; B.kcur = h->d_kcur; B.cexp = h->d_cexp; B.dm = h->d_dm; B.mvec = h->d_mvec;
  return B;
}

// One time step of Algorithm 6: x-phase (state 0 -> 1), y-phase (1 -> 0),
// collision in place on state 0.
void enqueue_step(dd_dlra* h) {
  if (h->P.splitting == DD_SPLIT_STRANG) {
    // x(dt/2), y(dt/2), collision(dt), y(dt/2), x(dt/2); the state alternates 0 -> 1 -> 0
    // -> 0 -> 1 -> 0, so the step ends in state 0 as with the Lie order
    dd::Problem Ph = h->P;
    Ph.g.dtk = h->d_dth;
    dd::advection_phase(Ph, bufs(h, 0, 1), 0, h->stream);
    dd::advection_phase(Ph, bufs(h, 1, 0), 1, h->stream);
    dd::collision_phase(h->P, bufs(h, 0, 0), h->stream);
    dd::advection_phase(Ph, bufs(h, 0, 1), 1, h->stream);
    dd::advection_phase(Ph, bufs(h, 1, 0), 0, h->stream);
  } else {
    dd::advection_phase(h->P, bufs(h, 0, 1), 0, h->stream);
    dd::advection_phase(h->P, bufs(h, 1, 0), 1, h->stream);
    dd::collision_phase(h->P, bufs(h, 0, 0), h->stream);
  }
  if (h->P.mass_fix) {
    // correction state 0 -> 1, then back to 0 (the state between steps)
    dd::mass_fix_phase(h->P, bufs(h, 0, 1), h->stream);
    const long Nt = h->Ntot, RC = h->RC;
    cudaMemcpyAsync(h->d_X[0], h->d_X[1], sizeof(double) * Nt * RC, cudaMemcpyDeviceToDevice, h->stream);
    cudaMemcpyAsync(h->d_V[0], h->d_V[1], sizeof(double) * (long)h->nsub * h->n * RC,
                    cudaMemcpyDeviceToDevice, h->stream);
    cudaMemcpyAsync(h->d_S[0], h->d_S[1], sizeof(double) * (long)h->nsub * RC * RC,
                    cudaMemcpyDeviceToDevice, h->stream);
    cudaMemcpyAsync(h->d_r[0], h->d_r[1], sizeof(int) * h->nsub, cudaMemcpyDeviceToDevice, h->stream);
  }
}

dd_status check_status(dd_dlra* h) {
  unsigned st = 0;
  DD_CUDA(cudaMemcpyAsync(&st, h->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream));
  DD_CUDA(cudaStreamSynchronize(h->stream));
  if (st & dd::ST_NONFINITE) return fail(DD_ERR_NONFINITE, "non-finite value in the factors");
  if (st & dd::ST_COMPLETION) return fail(DD_ERR_COMPLETION, "basis completion family exhausted");
  if (st & dd::ST_RANKCAP) return fail(DD_ERR_RANK_CAP, "rank capacity exceeded");
  if (st & dd::ST_TIMEOUT)
    return fail(DD_ERR_TIMEOUT, "a kernel's bounded wait for its tile loads or tensor-core "
                                "products ran out");
  return DD_OK;
}

// Angular completion family: P_2l(mu) cos/sin(m phi), sqrt(w)-weighted rows.
void angular_family(const dd_quadrature* q, double ssum, std::vector<double>& tab, int max_count,
                    int* complete) {
  const int n = q->n;
  std::vector<double> phi(n), mu(n);
  for (int i = 0; i < n; ++i) {
    phi[i] = std::atan2(q->omega_y[i], q->omega_x[i]);
    double s2 = q->omega_x[i] * q->omega_x[i] + q->omega_y[i] * q->omega_y[i];
    mu[i] = std::sqrt(std::max(0.0, 1.0 - s2));
  }
  const int l_count = q->n_polar == 0 ? 1 : (q->n_polar + 1) / 2;
  const int m_max = q->n_azimuth / 2;
  int count = 0, total = 0;
  std::vector<double> c(n);
  for (int deg = 0; deg <= m_max + 2 * (l_count - 1); ++deg) {
    for (int m = std::min(deg, m_max); m >= 0; --m) {
      if ((deg - m) % 2) continue;
      int l = (deg - m) / 2;
      if (l >= l_count) continue;
      for (int trig = 0; trig < 2; ++trig) {
        if (trig == 1 && m == 0) continue;
        double nn = 0.0;
        for (int i = 0; i < n; ++i) {
          double p = legendre(2 * l, mu[i]);
          c[i] = p * (trig == 0 ? std::cos(m * phi[i]) : std::sin(m * phi[i]));
          nn += q->w[i] * c[i] * c[i];
        }
        if (nn < 1e-12 * ssum) continue;
        ++total;
        if (count == max_count) {                  // a candidate past the table: not complete
          *complete = 0;
          return;
        }
        for (int i = 0; i < n; ++i) tab.push_back(std::sqrt(q->w[i]) * c[i]);
        ++count;
      }
    }
  }
  *complete = (count == total) ? 1 : 0;
}

// G = T T^T of the nc leading rows of the n-column table T (device), one thread per entry
__global__ void k_tab_gram(const double* T, int nc, int n, double* G) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nc * nc) return;
  const int i = e / nc, j = e - i * nc;
  double y = 0.0;
  for (int q = 0; q < n; ++q) y += T[(size_t)i * n + q] * T[(size_t)j * n + q];
  G[e] = y;
}

// dst[i * ld] = src[i], i < n (column 0 of a row-major matrix from a compact vector)
__global__ void k_put_col0(double* dst, int ld, const double* src, long n) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    dst[i * ld] = src[i];
}

void free_all(dd_dlra* h) {
  void* ptrs[] = {h->d_N, h->d_nxk, h->d_nyk, h->d_rowoff, h->d_nb, h->d_cx0, h->d_cy0,
                  h->d_ox, h->d_oy, h->d_w, h->d_sw, h->d_sig_s, h->d_sig_t, h->d_sQ,
                  h->d_angcand, h->d_X[0], h->d_X[1], h->d_V[0], h->d_V[1], h->d_S[0],
                  h->d_S[1], h->d_r[0], h->d_r[1], h->d_L0, h->d_Hw, h->d_Hwa, h->d_Vh,
                  h->d_K, h->d_X1, h->d_L, h->d_V1, h->d_Kb, h->d_sm, h->d_part, h->d_sig,
                  h->d_rho, h->d_fluxw, h->d_m, h->d_rt, h->d_rx, h->d_rc, h->d_p, h->d_status,
                  h->d_keep, h->d_cexp, h->d_dm, h->d_mvec, h->d_rlo, h->d_rhi, h->d_raug, h->d_fbase,
                  h->d_fnx, h->d_hxk, h->d_hyk, h->d_dtk, h->d_shk, h->d_dth, h->d_infl_on, h->d_infl_g,
                  h->d_infl_hw, h->d_infl_sc, h->d_kcn, h->d_kcur, h->d_sptab, h->d_spoff,
                  h->d_spnf};
  // a caller's allocator may hand the blocks out again at once (cudaFree would wait for the
  // device): nothing of this solver, a failed create's launches included, may still run
  if (h->alloc.alloc) cudaDeviceSynchronize();
  for (void* p : ptrs) dfree(h->alloc, p);
  if (h->graph_ready) cudaGraphExecDestroy(h->graph_exec);
}

}  // namespace

namespace dd {

dd_status set_error(dd_status s, const char* msg) { return fail(s, msg); }

cudaError_t noalloc_scratch_address(double** addr);   // dd_noalloc.cu

// Scalar flux with the per-subdomain scratch in the fixed device array whose address
// the solver looked up at create time.
dd_status noalloc_flux_impl(dd_dlra_t h, int scratch_doubles, double* out) {
  g_err.clear();
  int dev = -1;
  DD_CUDA(cudaGetDevice(&dev));
  if (dev != h->device) return fail(DD_ERR_ARG, "call on the device the solver was created on");
  if ((long)h->nsub * h->RC > scratch_doubles)
    return fail(DD_ERR_ARG, "nsub * r_cap = " + std::to_string((long)h->nsub * h->RC) +
                                " exceeds the allocation-free scratch of " +
                                std::to_string(scratch_doubles) + " doubles");
  dd::scalar_flux(h->P, h->d_X[0], h->d_V[0], h->d_S[0], h->d_r[0], h->d_noalloc, out, h->nx,
                  h->stream);
  DD_CUDA(cudaGetLastError());
  return DD_OK;
}

}  // namespace dd

extern "C" {

const char* dd_last_error(void) { return g_err.c_str(); }

const char* dd_dlra_last_error(dd_dlra_t h) {
  (void)h;   // the message is kept per host thread, not per solver
  return g_err.c_str();
}

dd_status dd_set_allocator(const dd_allocator* a) {
  g_err.clear();
  if (a && (a->alloc == nullptr) != (a->release == nullptr))
    return fail(DD_ERR_ARG, "an allocator needs both alloc and release, or neither");
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  g_alloc = a ? *a : dd_allocator{nullptr, nullptr, nullptr};
  return DD_OK;
}

static dd_status check_instance(const dd_grid* grid, const dd_tiling* tiling,
                                const dd_fields* fields, const double* g0, const dd_options* opt) {
  if (!grid || !tiling || !fields || !g0 || !opt) return fail(DD_ERR_ARG, "null argument");
  if (!fields->sigma_s || !fields->sigma_a || !fields->source) return fail(DD_ERR_ARG, "null field");
  for (int sd = 0; sd < 4; ++sd)
    if ((fields->inflow_g[sd] == nullptr) != (fields->inflow_h[sd] == nullptr))
      return fail(DD_ERR_ARG, "inflow needs both g and h on a side");
  if (grid->nx <= 0 || grid->ny <= 0 || !(grid->x1 > grid->x0) || !(grid->y1 > grid->y0))
    return fail(DD_ERR_ARG, "bad grid");
  if (tiling->tx <= 0 || tiling->ty <= 0 || !tiling->xcuts || !tiling->ycuts)
    return fail(DD_ERR_ARG, "bad tiling");
  if (tiling->xcuts[0] != 0 || tiling->xcuts[tiling->tx] != grid->nx || tiling->ycuts[0] != 0 ||
      tiling->ycuts[tiling->ty] != grid->ny)
    return fail(DD_ERR_ARG, "tiling cuts must start at 0 and end at nx / ny");
  for (int i = 0; i < tiling->tx; ++i)
    if (tiling->xcuts[i + 1] <= tiling->xcuts[i]) return fail(DD_ERR_ARG, "xcuts not increasing");
  for (int j = 0; j < tiling->ty; ++j)
    if (tiling->ycuts[j + 1] <= tiling->ycuts[j]) return fail(DD_ERR_ARG, "ycuts not increasing");
  if (opt->rank_mode != DD_RANK_FIXED && opt->rank_mode != DD_RANK_TOL)
    return fail(DD_ERR_ARG, "rank_mode");
  if (opt->integrator != DD_EULER && opt->integrator != DD_RK4)
    return fail(DD_ERR_ARG, "integrator");
  if (opt->precision != DD_FP64 && opt->precision != DD_MIXED && opt->precision != DD_TF32 &&
      opt->precision != DD_BF16)
    return fail(DD_ERR_ARG, "precision");
  if (opt->mass_fix != 0 && opt->mass_fix != 1) return fail(DD_ERR_ARG, "mass_fix");
  if (opt->splitting != DD_SPLIT_LIE && opt->splitting != DD_SPLIT_STRANG)
    return fail(DD_ERR_ARG, "splitting");
  if (opt->kstep_split != DD_KSPLIT_EIGEN && opt->kstep_split != DD_KSPLIT_FLUX)
    return fail(DD_ERR_ARG, "kstep_split");
  if (opt->products != DD_PRODUCTS_TENSOR && opt->products != DD_PRODUCTS_FP64 &&
      opt->products != DD_PRODUCTS_AUTO)
    return fail(DD_ERR_ARG, "products");
  if (opt->autotune != 0 && opt->autotune != 1) return fail(DD_ERR_ARG, "autotune");
  if (!(opt->dt > 0.0) || !(opt->tau >= 0.0)) return fail(DD_ERR_ARG, "dt / tau");
  const int RS = opt->rank_mode == DD_RANK_FIXED ? opt->rank : opt->r_max;
  const int fl = opt->rank_mode == DD_RANK_FIXED ? opt->rank : opt->r_min;
  if (opt->r_aug_max < 1 || opt->r_aug_max > DD_MAXC)
    return fail(DD_ERR_ARG, "r_aug_max must be in [1, 64]");
  if (RS < 1 || RS > opt->r_aug_max) return fail(DD_ERR_ARG, "stored-rank cap must be in [1, r_aug_max]");
  if (3 * RS > DD_MAXC) return fail(DD_ERR_ARG, "3 * stored-rank cap must be <= 64");
  if (fl < 0 || fl > RS) return fail(DD_ERR_ARG, "rank floor");
  return DD_OK;
}

// Plan, allocate and initialise a solver over ninst independent problems that
// share the direction table; instance i's subdomains follow instance i-1's.
static dd_status create_impl(int ninst, const dd_grid* grids, const dd_tiling* tilings,
                             const dd_quadrature* quad, const dd_fields* fields,
                             const double* const* g0s, const dd_options* opts, void* stream,
                             dd_dlra_t* out) {
  g_err.clear();
  if (!out || !quad || !grids || !tilings || !fields || !g0s || !opts || ninst < 1)
    return fail(DD_ERR_ARG, "null argument");
  *out = nullptr;
  if (quad->n <= 0 || !quad->omega_x || !quad->omega_y || !quad->w)
    return fail(DD_ERR_ARG, "bad quadrature");
  for (int i = 0; i < quad->n; ++i)
    if (!(quad->w[i] > 0.0)) return fail(DD_ERR_ARG, "quadrature weights must be positive");
  for (int i = 0; i < ninst; ++i) {
    dd_status st = check_instance(&grids[i], &tilings[i], &fields[i], g0s[i], &opts[i]);
    if (st != DD_OK) return st;
    const dd_options& a = opts[0];
    const dd_options& b = opts[i];
    if (b.rank_mode != a.rank_mode || b.integrator != a.integrator || b.precision != a.precision ||
        b.c_adv != a.c_adv || b.tau != a.tau || b.tol != a.tol || b.mass_fix != a.mass_fix ||
        b.splitting != a.splitting || b.kstep_split != a.kstep_split || b.products != a.products ||
        b.autotune != a.autotune)
      return fail(DD_ERR_ARG, "instances of a batch must share rank mode, tolerance, integrator, "
                              "precision, mass_fix, splitting, kstep_split, products, autotune, c_adv and tau");
  }
  const dd_options* opt = &opts[0];

  dd_dlra* h = new dd_dlra();   // value-initialised: every device pointer starts null
  {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    h->alloc = g_alloc;
  }
  struct AllocScope {                // dalloc draws on this solver's allocator until create returns
    explicit AllocScope(const dd_allocator* a) { t_alloc = a; }
    ~AllocScope() { t_alloc = nullptr; }
  } alloc_scope(&h->alloc);
  cudaGetDevice(&h->device);
  h->ninst = ninst;
  h->nx = grids[0].nx; h->ny = grids[0].ny; h->tx = tilings[0].tx; h->ty = tilings[0].ty;
  h->n = quad->n;
  h->hx = (grids[0].x1 - grids[0].x0) / grids[0].nx;
  h->hy = (grids[0].y1 - grids[0].y0) / grids[0].ny;
  h->sh = std::sqrt(h->hx * h->hy);
  h->opt = *opt;
  h->stream = reinterpret_cast<cudaStream_t>(stream);
  h->ssum = 0.0;
  for (int i = 0; i < quad->n; ++i) h->ssum += quad->w[i];
  int RS = 0, raug_max = 0;
  for (int i = 0; i < ninst; ++i) {
    RS = std::max(RS, opts[i].rank_mode == DD_RANK_FIXED ? opts[i].rank : opts[i].r_max);
    raug_max = std::max(raug_max, opts[i].r_aug_max);
  }
  h->RS = RS;
  // inflow sides add up to two augmentation columns per axis (one per physical side)
  bool any_inflow = false;
  for (int i = 0; i < ninst; ++i)
    for (int sd = 0; sd < 4; ++sd) any_inflow |= fields[i].inflow_g[sd] != nullptr;
  h->MC = 3 * h->RS + (any_inflow ? 2 : 0);
  // column capacity of every tall and small matrix: the intermediate rank and the
  // augmentation input width both fit
  h->RC = std::max(raug_max, h->MC);
  // the tensor-core forms stage rows with TMA, which needs rows on 16-byte boundaries
  if (opt->precision == DD_TF32 || opt->precision == DD_BF16 || opt->products != DD_PRODUCTS_FP64)
    h->RC += h->RC & 1;
  h->r_floor = opt->rank_mode == DD_RANK_FIXED ? opt->rank : opt->r_min;
  auto bail = [&](dd_status s, const std::string& m) {
    free_all(h);
    delete h;
    return fail(s, m);
  };
  if (h->n < h->MC) return bail(DD_ERR_ARG, "need at least 3 * stored-rank cap directions");

  // geometry, instance after instance
  int rowoff = 0, fbase = 0;
  h->maxlines = 0;
  h->maxN = 0;
  for (int inst = 0; inst < ninst; ++inst) {
    const dd_grid* grid = &grids[inst];
    const dd_tiling* tiling = &tilings[inst];
    const dd_options* o = &opts[inst];
    const double hx = (grid->x1 - grid->x0) / grid->nx, hy = (grid->y1 - grid->y0) / grid->ny;
    const int k0 = (int)h->geo.size();
    const int tx = tiling->tx, ty = tiling->ty;
    h->inst_sub0.push_back(k0);
    h->inst_nsub.push_back(tx * ty);
    h->inst_fbase.push_back(fbase);
    h->inst_nx.push_back(grid->nx);
    h->inst_ny.push_back(grid->ny);
    for (int J = 0; J < ty; ++J)
      for (int I = 0; I < tx; ++I) {
        int k = k0 + J * tx + I;
        SubGeo s;
        s.cx0 = tiling->xcuts[I];
        s.cy0 = tiling->ycuts[J];
        s.nxk = tiling->xcuts[I + 1] - s.cx0;
        s.nyk = tiling->ycuts[J + 1] - s.cy0;
        s.N = s.nxk * s.nyk;
        s.rowoff = rowoff;
        rowoff += s.N;
        s.nb[0] = I > 0 ? k - 1 : -1;
        s.nb[1] = I < tx - 1 ? k + 1 : -1;
        s.nb[2] = J > 0 ? k - tx : -1;
        s.nb[3] = J < ty - 1 ? k + tx : -1;
        s.inst = inst;
        s.hx = hx; s.hy = hy; s.dt = o->dt; s.sh = std::sqrt(hx * hy);
        s.rlo = o->rank_mode == DD_RANK_FIXED ? o->rank : o->r_min;
        s.rhi = o->rank_mode == DD_RANK_FIXED ? o->rank : o->r_max;
        s.raug = o->r_aug_max;
        s.fbase = fbase;
        s.fnx = grid->nx;
        h->geo.push_back(s);
        h->maxlines = std::max(h->maxlines, std::max(s.nxk, s.nyk));
        h->maxN = std::max(h->maxN, s.N);
      }
    fbase += grid->nx * grid->ny;
  }
  h->nsub = (int)h->geo.size();
  h->ncells_out = fbase;
  h->Ntot = rowoff;
  // the K-step holds one whole line of K (side x r_t <= side x r_aug_max values) per CTA
  for (const SubGeo& s : h->geo)
    if (std::max(s.nxk, s.nyk) * s.raug > DD_THREADS * 24)
      return bail(DD_ERR_ARG, "subdomain side x r_aug_max exceeds the K-step tile (6144)");

  const int RC = h->RC, n = h->n, nsub = h->nsub, MC = h->MC;
  const long Nt = h->Ntot;
  {
    std::vector<int> vN(nsub), vnx(nsub), vny(nsub), vro(nsub), vnb(4 * nsub), vcx(nsub), vcy(nsub),
        vlo(nsub), vhi(nsub), vaug(nsub), vfb(nsub), vfnx(nsub);
    std::vector<double> vhx(nsub), vhy(nsub), vdt(nsub), vsh(nsub);
    for (int k = 0; k < nsub; ++k) {
      const SubGeo& g = h->geo[k];
      vN[k] = g.N; vnx[k] = g.nxk; vny[k] = g.nyk; vro[k] = g.rowoff; vcx[k] = g.cx0; vcy[k] = g.cy0;
      for (int s = 0; s < 4; ++s) vnb[4 * k + s] = g.nb[s];
      vlo[k] = g.rlo; vhi[k] = g.rhi; vaug[k] = g.raug; vfb[k] = g.fbase; vfnx[k] = g.fnx;
      vhx[k] = g.hx; vhy[k] = g.hy; vdt[k] = g.dt; vsh[k] = g.sh;
    }
#define UP_INT(dst, v)                                                                       \
  if (dalloc(&dst, v.size()) != cudaSuccess ||                                                \
      cudaMemcpy(dst, v.data(), sizeof(int) * v.size(), cudaMemcpyHostToDevice) != cudaSuccess) \
    return bail(DD_ERR_CUDA, "upload geometry");
#define UP_DBLV(dst, v)                                                                         \
  if (dalloc(&dst, v.size()) != cudaSuccess ||                                                   \
      cudaMemcpy(dst, v.data(), sizeof(double) * v.size(), cudaMemcpyHostToDevice) != cudaSuccess) \
    return bail(DD_ERR_CUDA, "upload geometry");
    UP_INT(h->d_N, vN); UP_INT(h->d_nxk, vnx); UP_INT(h->d_nyk, vny); UP_INT(h->d_rowoff, vro);
    UP_INT(h->d_nb, vnb); UP_INT(h->d_cx0, vcx); UP_INT(h->d_cy0, vcy);
    UP_INT(h->d_rlo, vlo); UP_INT(h->d_rhi, vhi); UP_INT(h->d_raug, vaug); UP_INT(h->d_fbase, vfb);
    UP_INT(h->d_fnx, vfnx);
    std::vector<double> vdth(nsub);
    for (int k = 0; k < nsub; ++k) vdth[k] = 0.5 * vdt[k];
    UP_DBLV(h->d_hxk, vhx); UP_DBLV(h->d_hyk, vhy); UP_DBLV(h->d_dtk, vdt); UP_DBLV(h->d_shk, vsh);
    UP_DBLV(h->d_dth, vdth);
#undef UP_INT
#undef UP_DBLV
  }
  // problem data
  std::vector<double> sw(n), sig_s(Nt), sig_t(Nt), sQ(Nt);
  for (int q = 0; q < n; ++q) sw[q] = std::sqrt(quad->w[q]);
  h->sw_host = sw;
  for (int k = 0; k < nsub; ++k) {
    const SubGeo& s = h->geo[k];
    const dd_fields* f = &fields[s.inst];
    for (int c = 0; c < s.N; ++c) {
      int gi = (s.cy0 + c / s.nxk) * s.fnx + s.cx0 + c % s.nxk;
      sig_s[s.rowoff + c] = f->sigma_s[gi];
      sig_t[s.rowoff + c] = f->sigma_s[gi] + f->sigma_a[gi];
      sQ[s.rowoff + c] = s.sh * f->source[gi];
    }
  }
  std::vector<double> tab;
  angular_family(quad, h->ssum, tab, 4 * RC + 16, &h->angcand_complete);
  h->n_angcand = (int)(tab.size() / n);
  // the longest leading part of the table whose candidates are mutually orthogonal (to
  // 1e-12 in cosine): only those enter the coefficient-space completion, which examines at
  // most kc_bmax(RC) of them (their Gram on the device, after the upload below)
  const int n_chk = std::min(h->n_angcand, dd::kc_bmax(RC));
#define UP_DBL(dst, ptr, count)                                                                 \
  if (dalloc(&dst, count) != cudaSuccess ||                                                      \
      cudaMemcpy(dst, ptr, sizeof(double) * (count), cudaMemcpyHostToDevice) != cudaSuccess)     \
    return bail(DD_ERR_CUDA, "upload problem data");
  UP_DBL(h->d_ox, quad->omega_x, n);
  UP_DBL(h->d_oy, quad->omega_y, n);
  UP_DBL(h->d_w, quad->w, n);
  UP_DBL(h->d_sw, sw.data(), n);
  UP_DBL(h->d_sig_s, sig_s.data(), Nt);
  UP_DBL(h->d_sig_t, sig_t.data(), Nt);
  UP_DBL(h->d_sQ, sQ.data(), Nt);
  UP_DBL(h->d_angcand, tab.data(), tab.size());
  {
    double* d_g = nullptr;
    std::vector<double> gh((size_t)n_chk * n_chk);
    if (n_chk > 0) {
      if (dalloc(&d_g, gh.size()) != cudaSuccess) return bail(DD_ERR_CUDA, "device allocation failed");
      k_tab_gram<<<(n_chk * n_chk + 255) / 256, 256>>>(h->d_angcand, n_chk, n, d_g);
      const cudaError_t e = cudaMemcpy(gh.data(), d_g, sizeof(double) * gh.size(), cudaMemcpyDeviceToHost);
      dfree(h->alloc, d_g);
      if (e != cudaSuccess) return bail(DD_ERR_CUDA, "angular table Gram");
    }
    h->n_angorth = dd::orthogonal_prefix_gram(gh.data(), n_chk, 1e-12);
  }
  {
    // spatial completion family (R11): per subdomain the cosines cos(pi f (i + 1/2) / n)
    // of the x and y frequencies that its first kc_bmax(RC) candidates use
    const int bm = dd::kc_bmax(RC);
    std::vector<double> sptab;
    std::vector<long long> spoff(nsub);
    std::vector<int> spnf(2 * nsub);
    for (int k = 0; k < nsub; ++k) {
      const int nx = h->geo[k].nxk, ny = h->geo[k].nyk;
      int dmax = nx + ny - 2, cum = 0;
      for (int d = 0; d <= nx + ny - 2; ++d) {
        cum += std::min(d, nx - 1) - std::max(0, d - (ny - 1)) + 1;
        if (cum >= bm) { dmax = d; break; }
      }
      const int nfx = std::min(dmax, nx - 1) + 1, nfy = std::min(dmax, ny - 1) + 1;
      spoff[k] = (long long)sptab.size();
      spnf[2 * k] = nfx;
      spnf[2 * k + 1] = nfy;
      const double pi = 3.141592653589793;
      for (int f = 0; f < nfx; ++f)
        for (int i = 0; i < nx; ++i) sptab.push_back(std::cos(pi * f * (i + 0.5) / nx));
      for (int f = 0; f < nfy; ++f)
        for (int j = 0; j < ny; ++j) sptab.push_back(std::cos(pi * f * (j + 0.5) / ny));
    }
    UP_DBL(h->d_sptab, sptab.data(), sptab.size());
    if (dalloc(&h->d_spoff, spoff.size()) != cudaSuccess ||
        cudaMemcpy(h->d_spoff, spoff.data(), sizeof(long long) * spoff.size(),
                   cudaMemcpyHostToDevice) != cudaSuccess ||
        dalloc(&h->d_spnf, spnf.size()) != cudaSuccess ||
        cudaMemcpy(h->d_spnf, spnf.data(), sizeof(int) * spnf.size(), cudaMemcpyHostToDevice) !=
            cudaSuccess)
      return bail(DD_ERR_CUDA, "upload problem data");
  }
  if (any_inflow) {
    // per subdomain and side: on/off, face values sqrt(hx hy) g(line), angular column
    // sqrt(w) m_in h and the augmentation scale |g|_x (the subdomain-sized virtual
    // neighbour)
    const int ML = h->maxlines;
    std::vector<int> on(nsub * 4, 0);
    std::vector<double> gf((size_t)nsub * 4 * ML, 0.0), hw((size_t)nsub * 4 * n, 0.0),
        sc(nsub * 4, 0.0);
    for (int k = 0; k < nsub; ++k) {
      const SubGeo& sg = h->geo[k];
      const dd_fields* f = &fields[sg.inst];
      for (int sd = 0; sd < 4; ++sd) {
        if (sg.nb[sd] >= 0 || !f->inflow_g[sd]) continue;
        on[k * 4 + sd] = 1;
        const bool xs = sd < 2;
        const int lines = xs ? sg.nyk : sg.nxk, len = xs ? sg.nxk : sg.nyk;
        double g2 = 0.0;
        for (int l = 0; l < lines; ++l) {
          const double gv = f->inflow_g[sd][xs ? sg.cy0 + l : sg.cx0 + l];
          gf[((size_t)k * 4 + sd) * ML + l] = sg.sh * gv;
          g2 += gv * gv;
        }
        sc[k * 4 + sd] = std::sqrt(sg.hx * sg.hy * len * g2);
        const double* om = xs ? quad->omega_x : quad->omega_y;
        for (int q = 0; q < n; ++q) {
          const bool in = (sd % 2 == 0) ? om[q] >= 0.0 : om[q] < 0.0;
          hw[((size_t)k * 4 + sd) * n + q] = in ? sw[q] * f->inflow_h[sd][q] : 0.0;
        }
      }
    }
    if (dalloc(&h->d_infl_on, on.size()) != cudaSuccess ||
        cudaMemcpy(h->d_infl_on, on.data(), sizeof(int) * on.size(), cudaMemcpyHostToDevice) != cudaSuccess)
      return bail(DD_ERR_CUDA, "upload inflow");
    UP_DBL(h->d_infl_g, gf.data(), gf.size());
    UP_DBL(h->d_infl_hw, hw.data(), hw.size());
    UP_DBL(h->d_infl_sc, sc.data(), sc.size());
  }
#undef UP_DBL
  // state and workspace
  bool ok = true;
  for (int b = 0; b < 2; ++b) {
    ok &= dalloc(&h->d_X[b], Nt * RC) == cudaSuccess;
    ok &= dalloc(&h->d_V[b], (long)nsub * n * RC) == cudaSuccess;
    ok &= dalloc(&h->d_S[b], (long)nsub * RC * RC) == cudaSuccess;
    ok &= dalloc(&h->d_r[b], nsub) == cudaSuccess;
  }
  ok &= dalloc(&h->d_L0, (long)nsub * n * MC) == cudaSuccess;
  const int WC = RC;
  ok &= dalloc(&h->d_Hw, Nt * WC) == cudaSuccess;
  ok &= dalloc(&h->d_Hwa, (long)nsub * n * WC) == cudaSuccess;
  ok &= dalloc(&h->d_Vh, (long)nsub * n * RC) == cudaSuccess;
  ok &= dalloc(&h->d_K, Nt * RC) == cudaSuccess;
  ok &= dalloc(&h->d_X1, Nt * RC) == cudaSuccess;
  ok &= dalloc(&h->d_L, (long)nsub * n * RC) == cudaSuccess;
  ok &= dalloc(&h->d_V1, (long)nsub * n * RC) == cudaSuccess;
  ok &= dalloc(&h->d_Kb, (long)nsub * 2 * h->maxlines * RC) == cudaSuccess;
  ok &= dalloc(&h->d_sm, (long)nsub * dd::NSMALL * RC * RC) == cudaSuccess;
  ok &= dalloc(&h->d_sig, (long)nsub * DD_MAXC) == cudaSuccess;
  ok &= dalloc(&h->d_rho, (long)h->ncells_out) == cudaSuccess;
  ok &= dalloc(&h->d_fluxw, (long)nsub * RC) == cudaSuccess;
  ok &= dalloc(&h->d_m, nsub) == cudaSuccess;
  ok &= dalloc(&h->d_rt, nsub) == cudaSuccess;
  ok &= dalloc(&h->d_rx, 2 * nsub) == cudaSuccess;
  ok &= dalloc(&h->d_rc, nsub) == cudaSuccess;
  ok &= dalloc(&h->d_p, nsub) == cudaSuccess;
  ok &= dalloc(&h->d_keep, nsub) == cudaSuccess;
  ok &= dalloc(&h->d_kcn, nsub) == cudaSuccess;
  ok &= dalloc(&h->d_kcur, nsub) == cudaSuccess;
  ok &= dalloc(&h->d_cexp, (long)nsub * 16) == cudaSuccess;
  ok &= dalloc(&h->d_dm, Nt) == cudaSuccess;
  ok &= dalloc(&h->d_mvec, (long)nsub * RC) == cudaSuccess;
  ok &= dalloc(&h->d_status, 1) == cudaSuccess;
  if (!ok) return bail(DD_ERR_CUDA, "device allocation failed");

  // problem descriptor
  dd::Problem& P = h->P;
  P.g.nsub = nsub; P.g.n = n; P.g.RC = RC; P.g.MC = MC;
  P.g.N = h->d_N; P.g.nxk = h->d_nxk; P.g.nyk = h->d_nyk; P.g.rowoff = h->d_rowoff;
  P.g.nb = h->d_nb; P.g.cx0 = h->d_cx0; P.g.cy0 = h->d_cy0;
  P.g.hxk = h->d_hxk; P.g.hyk = h->d_hyk; P.g.dtk = h->d_dtk; P.g.shk = h->d_shk;
  P.g.rlo = h->d_rlo; P.g.rhi = h->d_rhi; P.g.raug = h->d_raug; P.g.fbase = h->d_fbase;
  P.g.fnx = h->d_fnx;
  P.maxlines = h->maxlines; P.maxN = h->maxN;
  P.ox = h->d_ox; P.oy = h->d_oy; P.w = h->d_w; P.sw = h->d_sw;
  P.sig_s = h->d_sig_s; P.sig_t = h->d_sig_t; P.sQ = h->d_sQ;
  P.hx = h->hx; P.hy = h->hy; P.sh = h->sh; P.dt = opt->dt; P.c_adv = opt->c_adv; P.ssum = h->ssum;
  P.integrator = opt->integrator; P.rank_mode = opt->rank_mode; P.tol = opt->tol;
  P.prec = opt->precision == DD_MIXED  ? dd::PREC_MIXED
           : opt->precision == DD_TF32 ? dd::PREC_TF32
           : opt->precision == DD_BF16 ? dd::PREC_BF16
                                       : dd::PREC_FP64;
  P.Ntot = Nt;
  P.oz_sp = P.oz_ang = opt->products == DD_PRODUCTS_TENSOR ? 1 : 0;
  P.ozg_sp = P.ozg_ang = P.oz_sp;
  P.mass_fix = opt->mass_fix;
  P.splitting = opt->splitting;
  P.kstep_split = opt->kstep_split;
  P.infl_on = h->d_infl_on; P.infl_g = h->d_infl_g; P.infl_hw = h->d_infl_hw;
  P.infl_sc = h->d_infl_sc;
  P.tau = opt->tau; P.accept = 0.5;
  P.r_floor = h->r_floor; P.r_aug_max = raug_max; P.RS = h->RS; P.WC = WC;
  P.angcand = h->d_angcand; P.n_angcand = h->n_angcand; P.angcand_complete = h->angcand_complete;
  P.n_angorth = h->n_angorth;
  P.sptab = h->d_sptab; P.spoff = h->d_spoff; P.spnf = h->d_spnf;
  P.nchunk_sp = std::max(1, std::min(16, h->maxN / 64));
  {
    int nsm = 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess ||
        nsm <= 0)
      nsm = 1;
    P.nsm = nsm;
  }
  P.nchunk_ang = std::max(1, std::min(16, n / 64));
  P.ochunk_sp = P.nchunk_sp;
  P.ochunk_ang = P.nchunk_ang;
  if (dalloc(&h->d_part, dd::part_elems(P)) != cudaSuccess)
    return bail(DD_ERR_CUDA, "device allocation failed");
  if (dd::orth_init() != cudaSuccess || dd::phase_init() != cudaSuccess)
    return bail(DD_ERR_CUDA, "kernel attribute setup failed");
  if (opt->products == DD_PRODUCTS_AUTO) {      // the heuristic; the autotuner may revise it
    const long tiles_sp = (long)nsub * ((h->maxN + 127) / 128), tiles_ang = (long)nsub * ((n + 127) / 128);
    P.oz_sp = tiles_sp >= 2L * P.nsm;
    P.oz_ang = tiles_ang >= 2L * P.nsm;
  }
  if ((P.prec >= dd::PREC_TF32 || opt->products != DD_PRODUCTS_FP64) && dd::tc_init() != cudaSuccess)
    return bail(DD_ERR_CUDA, "tensor-core setup failed (tensor-map encoder or kernel attributes)");
  // the allocation-free readout's scratch array, looked up with this solver's device and
  // context current (no allocation)
  if (dd::noalloc_scratch_address(&h->d_noalloc) != cudaSuccess)
    return bail(DD_ERR_CUDA, "scratch array lookup failed");

  // isotropic initial data at rank 1 (rank 0 where g0 vanishes on the subdomain): only
  // column 0 of X and V is nonzero; it is uploaded compactly (staged in the orthonormalisation
  // workspaces) and scattered on the device into both state buffers, the rest cleared there
  {
    std::vector<double> x0((size_t)Nt, 0.0), v0((size_t)nsub * n, 0.0),
        S((size_t)nsub * RC * RC, 0.0);
    std::vector<int> r(nsub, 0);
    for (int k = 0; k < nsub; ++k) {
      const SubGeo& s = h->geo[k];
      const double* g0 = g0s[s.inst];
      double nn = 0.0;
      for (int c = 0; c < s.N; ++c) {
        double gv = g0[(s.cy0 + c / s.nxk) * s.fnx + s.cx0 + c % s.nxk];
        nn += gv * gv;
      }
      nn = std::sqrt(nn);
      if (!(nn > 0.0)) continue;
      r[k] = 1;
      for (int c = 0; c < s.N; ++c)
        x0[(size_t)s.rowoff + c] = g0[(s.cy0 + c / s.nxk) * s.fnx + s.cx0 + c % s.nxk] / nn;
      for (int q = 0; q < n; ++q) v0[(size_t)k * n + q] = sw[q] / std::sqrt(h->ssum);
      S[(size_t)k * RC * RC] = nn * s.sh * std::sqrt(h->ssum);
    }
    if (cudaMemcpy(h->d_Hw, x0.data(), sizeof(double) * x0.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(h->d_Hwa, v0.data(), sizeof(double) * v0.size(), cudaMemcpyHostToDevice) != cudaSuccess)
      return bail(DD_ERR_CUDA, "upload initial state");
    for (int b = 0; b < 2; ++b) {
      if (cudaMemset(h->d_X[b], 0, sizeof(double) * (size_t)Nt * RC) != cudaSuccess ||
          cudaMemset(h->d_V[b], 0, sizeof(double) * (size_t)nsub * n * RC) != cudaSuccess)
        return bail(DD_ERR_CUDA, "clear initial state");
      k_put_col0<<<256, 256>>>(h->d_X[b], RC, h->d_Hw, (long)Nt);
      k_put_col0<<<256, 256>>>(h->d_V[b], RC, h->d_Hwa, (long)nsub * n);
      if (cudaGetLastError() != cudaSuccess ||
          cudaMemcpy(h->d_S[b], S.data(), sizeof(double) * S.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
          cudaMemcpy(h->d_r[b], r.data(), sizeof(int) * nsub, cudaMemcpyHostToDevice) != cudaSuccess)
        return bail(DD_ERR_CUDA, "upload initial state");
    }
    // the staging areas are the autotuner's trial outputs next, on the solver's stream
    if (cudaDeviceSynchronize() != cudaSuccess) return bail(DD_ERR_CUDA, "upload initial state");
    if (cudaMemset(h->d_status, 0, sizeof(unsigned)) != cudaSuccess ||
        cudaMemset(h->d_sm, 0, sizeof(double) * (size_t)nsub * dd::NSMALL * RC * RC) != cudaSuccess ||
        cudaMemset(h->d_rx, 0, sizeof(int) * 2 * nsub) != cudaSuccess ||
        cudaMemset(h->d_dm, 0, sizeof(double) * (size_t)Nt) != cudaSuccess)
      return bail(DD_ERR_CUDA, "clear workspace");
  }
  for (int i = 0; i < 8; ++i) h->tune_ms[i] = -1.0;
  if (opt->autotune &&
      dd::autotune(P, bufs(h, 0, 1), h->stream, opt->products == DD_PRODUCTS_AUTO, 1, h->tune_ms) !=
          cudaSuccess)
    return bail(DD_ERR_CUDA, "autotuner");
  if (cudaDeviceSynchronize() != cudaSuccess) return bail(DD_ERR_CUDA, "create: device error");
  *out = h;
  return DD_OK;
}

dd_status dd_dlra_create(const dd_grid* grid, const dd_tiling* tiling, const dd_quadrature* quad,
                         const dd_fields* fields, const double* g0, const dd_options* opt,
                         void* stream, dd_dlra_t* out) {
  if (!grid || !tiling || !quad || !fields || !g0 || !opt || !out) {
    g_err = "null argument";
    return DD_ERR_ARG;
  }
  const double* g0s[1] = {g0};
  return create_impl(1, grid, tiling, quad, fields, g0s, opt, stream, out);
}

dd_status dd_dlra_create_batch(int ninst, const dd_grid* grids, const dd_tiling* tilings,
                               const dd_quadrature* quad, const dd_fields* fields,
                               const double* const* g0, const dd_options* opts, void* stream,
                               dd_dlra_t* out) {
  return create_impl(ninst, grids, tilings, quad, fields, g0, opts, stream, out);
}

dd_status dd_dlra_instance(dd_dlra_t h, int inst, int* first_subdomain, int* nsub,
                           int* flux_offset, int* nx, int* ny) {
  if (!h || inst < 0 || inst >= h->ninst) return fail(DD_ERR_ARG, "bad instance");
  if (first_subdomain) *first_subdomain = h->inst_sub0[inst];
  if (nsub) *nsub = h->inst_nsub[inst];
  if (flux_offset) *flux_offset = h->inst_fbase[inst];
  if (nx) *nx = h->inst_nx[inst];
  if (ny) *ny = h->inst_ny[inst];
  return DD_OK;
}

dd_status dd_dlra_set_graph(dd_dlra_t h, int use_graph) {
  if (!h) return fail(DD_ERR_ARG, "null handle");
  h->use_graph = use_graph;
  return DD_OK;
}

dd_status dd_dlra_step(dd_dlra_t h, int nsteps) {
  g_err.clear();
  if (!h || nsteps < 0) return fail(DD_ERR_ARG, "bad argument");
  if (h->use_graph) {
    if (!h->graph_ready) {
      // capture on a private stream (the legacy default stream cannot be captured);
      // the instantiated graph is then launched on the solver's stream
      cudaStream_t user = h->stream, cap;
      DD_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
      cudaGraph_t graph;
      h->stream = cap;
      cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        enqueue_step(h);
        e = cudaStreamEndCapture(cap, &graph);
      }
      h->stream = user;
      cudaStreamDestroy(cap);
      if (e != cudaSuccess) return fail(DD_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e));
      e = cudaGraphInstantiate(&h->graph_exec, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) return fail(DD_ERR_CUDA, std::string("graph: ") + cudaGetErrorString(e));
      h->graph_ready = true;
    }
    for (int s = 0; s < nsteps; ++s) DD_CUDA(cudaGraphLaunch(h->graph_exec, h->stream));
  } else {
    for (int s = 0; s < nsteps; ++s) enqueue_step(h);
  }
  DD_CUDA(cudaGetLastError());
  return DD_OK;
}

dd_status dd_dlra_scalar_flux(dd_dlra_t h, double* out, int out_on_device) {
  g_err.clear();
  if (!h || !out) return fail(DD_ERR_ARG, "bad argument");
  double* dst = out_on_device ? out : h->d_rho;
  dd::scalar_flux(h->P, h->d_X[0], h->d_V[0], h->d_S[0], h->d_r[0], h->d_fluxw, dst, h->nx, h->stream);
  DD_CUDA(cudaGetLastError());
  if (!out_on_device) {
    DD_CUDA(cudaMemcpyAsync(out, h->d_rho, sizeof(double) * (size_t)h->ncells_out,
                            cudaMemcpyDeviceToHost, h->stream));
    return check_status(h);
  }
  return DD_OK;
}

dd_status dd_dlra_scalar_flux_instance(dd_dlra_t h, int inst, double* out, int out_on_device) {
  g_err.clear();
  if (!h || !out || inst < 0 || inst >= h->ninst) return fail(DD_ERR_ARG, "bad argument");
  dd::scalar_flux(h->P, h->d_X[0], h->d_V[0], h->d_S[0], h->d_r[0], h->d_fluxw, h->d_rho, h->nx,
                  h->stream);
  DD_CUDA(cudaGetLastError());
  const size_t cnt = (size_t)h->inst_nx[inst] * (size_t)h->inst_ny[inst];
  DD_CUDA(cudaMemcpyAsync(out, h->d_rho + h->inst_fbase[inst], sizeof(double) * cnt,
                          out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                          h->stream));
  return out_on_device ? DD_OK : check_status(h);
}

dd_status dd_dlra_ranks(dd_dlra_t h, int* stored, int* intermediate) {
  g_err.clear();
  if (!h || !stored) return fail(DD_ERR_ARG, "bad argument");
  DD_CUDA(cudaMemcpyAsync(stored, h->d_r[0], sizeof(int) * h->nsub, cudaMemcpyDeviceToHost, h->stream));
  if (intermediate)
    DD_CUDA(cudaMemcpyAsync(intermediate, h->d_rx, sizeof(int) * 2 * h->nsub, cudaMemcpyDeviceToHost,
                            h->stream));
  return check_status(h);
}

dd_status dd_dlra_info(dd_dlra_t h, int* nsub, int* n, int* r_cap) {
  if (!h) return fail(DD_ERR_ARG, "null handle");
  if (nsub) *nsub = h->nsub;
  if (n) *n = h->n;
  if (r_cap) *r_cap = h->RC;
  return DD_OK;
}

dd_status dd_dlra_get_factors(dd_dlra_t h, int k, double* U, double* S, double* V, int* r) {
  g_err.clear();
  if (!h || k < 0 || k >= h->nsub || !U || !S || !V || !r) return fail(DD_ERR_ARG, "bad argument");
  const SubGeo& s = h->geo[k];
  const int RC = h->RC, n = h->n;
  int rk = 0;
  std::vector<double> X((size_t)s.N * RC), Vt((size_t)n * RC), Sm((size_t)RC * RC);
  DD_CUDA(cudaMemcpyAsync(&rk, h->d_r[0] + k, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  DD_CUDA(cudaMemcpyAsync(X.data(), h->d_X[0] + (size_t)s.rowoff * RC, sizeof(double) * X.size(),
                          cudaMemcpyDeviceToHost, h->stream));
  DD_CUDA(cudaMemcpyAsync(Vt.data(), h->d_V[0] + (size_t)k * n * RC, sizeof(double) * Vt.size(),
                          cudaMemcpyDeviceToHost, h->stream));
  DD_CUDA(cudaMemcpyAsync(Sm.data(), h->d_S[0] + (size_t)k * RC * RC, sizeof(double) * Sm.size(),
                          cudaMemcpyDeviceToHost, h->stream));
  dd_status st = check_status(h);
  if (st != DD_OK) return st;
  for (int c = 0; c < s.N; ++c)
    for (int t = 0; t < rk; ++t) U[(size_t)c * rk + t] = X[(size_t)c * RC + t] / s.sh;
  for (int q = 0; q < n; ++q)
    for (int t = 0; t < rk; ++t) V[(size_t)q * rk + t] = Vt[(size_t)q * RC + t] / h->sw_host[q];
  for (int i = 0; i < rk; ++i)
    for (int j = 0; j < rk; ++j) S[(size_t)i * rk + j] = Sm[(size_t)i * RC + j];
  *r = rk;
  return DD_OK;
}

dd_status dd_dlra_set_factors(dd_dlra_t h, int k, int r, const double* U, const double* S,
                              const double* V) {
  g_err.clear();
  if (!h || k < 0 || k >= h->nsub || r < 0 || r > h->RS || (r > 0 && (!U || !S || !V)))
    return fail(DD_ERR_ARG, "bad argument");
  const SubGeo& s = h->geo[k];
  const int RC = h->RC, n = h->n;
  std::vector<double> X((size_t)s.N * RC, 0.0), Vt((size_t)n * RC, 0.0), Sm((size_t)RC * RC, 0.0);
  for (int c = 0; c < s.N; ++c)
    for (int t = 0; t < r; ++t) X[(size_t)c * RC + t] = U[(size_t)c * r + t] * s.sh;
  for (int q = 0; q < n; ++q)
    for (int t = 0; t < r; ++t) Vt[(size_t)q * RC + t] = V[(size_t)q * r + t] * h->sw_host[q];
  for (int i = 0; i < r; ++i)
    for (int j = 0; j < r; ++j) Sm[(size_t)i * RC + j] = S[(size_t)i * r + j];
  DD_CUDA(cudaStreamSynchronize(h->stream));
  DD_CUDA(cudaMemcpy(h->d_X[0] + (size_t)s.rowoff * RC, X.data(), sizeof(double) * X.size(),
                     cudaMemcpyHostToDevice));
  DD_CUDA(cudaMemcpy(h->d_V[0] + (size_t)k * n * RC, Vt.data(), sizeof(double) * Vt.size(),
                     cudaMemcpyHostToDevice));
  DD_CUDA(cudaMemcpy(h->d_S[0] + (size_t)k * RC * RC, Sm.data(), sizeof(double) * Sm.size(),
                     cudaMemcpyHostToDevice));
  DD_CUDA(cudaMemcpy(h->d_r[0] + k, &r, sizeof(int), cudaMemcpyHostToDevice));
  return DD_OK;
}

int dd_profile_slots(void) { return dd::NSLOT; }

const char* dd_profile_slot_name(int slot) {
  return (slot >= 0 && slot < dd::NSLOT) ? dd::kSlotNames[slot] : nullptr;
}

dd_status dd_dlra_profile(dd_dlra_t h, int nsteps, double* ms, int* launches) {
  return dd_dlra_profile_work(h, nsteps, ms, launches, nullptr);
}

dd_status dd_dlra_tuning(dd_dlra_t h, int* choice, double* ms) {
  g_err.clear();
  if (!h) return fail(DD_ERR_ARG, "null handle");
  if (choice) {
    choice[0] = h->P.oz_sp;
    choice[1] = h->P.oz_ang;
    choice[2] = h->P.ochunk_sp;
    choice[3] = h->P.ochunk_ang;
    choice[4] = h->P.ozg_sp;
    choice[5] = h->P.ozg_ang;
  }
  if (ms)
    for (int i = 0; i < 8; ++i) ms[i] = h->tune_ms[i];
  return DD_OK;
}

dd_status dd_dlra_profile_work(dd_dlra_t h, int nsteps, double* ms, int* launches, double* flops) {
  g_err.clear();
  if (!h || nsteps < 0 || !ms || !launches) return fail(DD_ERR_ARG, "bad argument");
  for (int i = 0; i < dd::NSLOT; ++i) { ms[i] = 0.0; launches[i] = 0; }
  unsigned long long* d_work = nullptr;
  if (flops) {
    // the kernels add their algorithmic flops to these counters while this call runs
    DD_CUDA(cudaMalloc(&d_work, sizeof(unsigned long long) * dd::NSLOT));
    DD_CUDA(cudaMemsetAsync(d_work, 0, sizeof(unsigned long long) * dd::NSLOT, h->stream));
    h->P.g.work = d_work;
  }
  dd::Prof* prof = new dd::Prof();
  prof->n = 0;
  for (int i = 0; i < dd::Prof::MAXL; ++i) {
    cudaEventCreate(&prof->b[i]);
    cudaEventCreate(&prof->e[i]);
  }
  dd_status st = DD_OK;
  for (int s = 0; s < nsteps && st == DD_OK; ++s) {
    prof->n = 0;
    dd::g_prof = prof;
    enqueue_step(h);
    dd::g_prof = nullptr;
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) { st = fail(DD_ERR_CUDA, cudaGetErrorString(e)); break; }
    for (int i = 0; i < prof->n; ++i) {
      float t = 0.f;
      cudaEventElapsedTime(&t, prof->b[i], prof->e[i]);
      ms[prof->slot[i]] += t;
      launches[prof->slot[i]] += 1;
    }
  }
  dd::g_prof = nullptr;
  for (int i = 0; i < dd::Prof::MAXL; ++i) {
    cudaEventDestroy(prof->b[i]);
    cudaEventDestroy(prof->e[i]);
  }
  delete prof;
  if (d_work) {
    h->P.g.work = nullptr;
    unsigned long long w[dd::NSLOT];
    cudaError_t e = cudaMemcpy(w, d_work, sizeof(w), cudaMemcpyDeviceToHost);
    cudaFree(d_work);
    if (e != cudaSuccess && st == DD_OK) st = fail(DD_ERR_CUDA, cudaGetErrorString(e));
    for (int i = 0; i < dd::NSLOT; ++i) flops[i] = e == cudaSuccess ? (double)w[i] : 0.0;
  }
  if (st != DD_OK) return st;
  return check_status(h);
}

dd_status dd_selftest_wait(unsigned polls, int* timed_out) {
  g_err.clear();
  if (!timed_out) return fail(DD_ERR_ARG, "null argument");
  if (polls == 0 || polls > (1u << 21)) return fail(DD_ERR_ARG, "polls must be in 1 .. 2^21");
  *timed_out = 0;
  unsigned* d = nullptr;
  DD_CUDA(cudaMalloc(&d, sizeof(unsigned)));
  cudaError_t e = cudaMemset(d, 0, sizeof(unsigned));
  if (e == cudaSuccess) e = dd::wait_selftest(d, polls, nullptr);
  unsigned word = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&word, d, sizeof(unsigned), cudaMemcpyDeviceToHost);
  const cudaError_t ef = cudaFree(d);
  if (e == cudaSuccess) e = ef;
  if (e != cudaSuccess) return fail(DD_ERR_CUDA, std::string("wait self-test: ") + cudaGetErrorString(e));
  *timed_out = (word & dd::ST_TIMEOUT) ? 1 : 0;
  return DD_OK;
}

dd_status dd_dlra_sync(dd_dlra_t h) {
  if (!h) return fail(DD_ERR_ARG, "null handle");
  return check_status(h);
}

void dd_dlra_destroy(dd_dlra_t h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  free_all(h);
  delete h;
}

}  // extern "C"
