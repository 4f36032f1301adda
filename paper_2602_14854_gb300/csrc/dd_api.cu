// Host side of the C ABI declared in include/ddlra.h: planning, allocation,
// initial factors, the time-step driver (optionally replayed from a CUDA graph),
// observables and factor exchange.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
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
};

template <class T>
cudaError_t dalloc(T** p, size_t count) {
  return cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * std::max<size_t>(count, 1));
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
  int nx, ny, tx, ty, nsub, n;
  double hx, hy, sh, ssum;
  dd_options opt;
  int RC, RS, MC, r_floor, maxlines, maxN;
  long Ntot;
  std::vector<SubGeo> geo;
  std::vector<double> sw_host;
  cudaStream_t stream;
  int use_graph;
  cudaGraphExec_t graph_exec;
  bool graph_ready;
  // device: geometry
  int *d_N, *d_nxk, *d_nyk, *d_rowoff, *d_nb, *d_cx0, *d_cy0;
  // device: problem data
  double *d_ox, *d_oy, *d_w, *d_sw, *d_sig_s, *d_sig_t, *d_sQ, *d_angcand;
  int n_angcand, angcand_complete;
  // device: state, double buffered
  double *d_X[2], *d_V[2], *d_S[2];
  int* d_r[2];
  // device: workspace
  double *d_L0, *d_Hw, *d_Hwa, *d_Vh, *d_K, *d_X1, *d_L, *d_V1, *d_Kb, *d_sm, *d_part;
  double *d_sig, *d_rho, *d_fluxw;
  int *d_m, *d_rt, *d_rx, *d_rc, *d_p, *d_flag;
  double* d_scale;
  unsigned* d_status;
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
  B.flag = h->d_flag; B.scale = h->d_scale;
  return B;
}

// One time step of Algorithm 6: x-phase (state 0 -> 1), y-phase (1 -> 0),
// collision in place on state 0.
void enqueue_step(dd_dlra* h) {
  dd::advection_phase(h->P, bufs(h, 0, 1), 0, h->stream);
  dd::advection_phase(h->P, bufs(h, 1, 0), 1, h->stream);
  dd::collision_phase(h->P, bufs(h, 0, 0), h->stream);
}

dd_status check_status(dd_dlra* h) {
  unsigned st = 0;
  DD_CUDA(cudaMemcpyAsync(&st, h->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream));
  DD_CUDA(cudaStreamSynchronize(h->stream));
  if (st & dd::ST_NONFINITE) return fail(DD_ERR_NONFINITE, "non-finite value in the factors");
  if (st & dd::ST_COMPLETION) return fail(DD_ERR_COMPLETION, "basis completion family exhausted");
  if (st & dd::ST_RANKCAP) return fail(DD_ERR_RANK_CAP, "rank capacity exceeded");
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
        if (count < max_count) {
          for (int i = 0; i < n; ++i) tab.push_back(std::sqrt(q->w[i]) * c[i]);
          ++count;
        }
      }
    }
  }
  *complete = (count == total) ? 1 : 0;
}

void free_all(dd_dlra* h) {
  void* ptrs[] = {h->d_N, h->d_nxk, h->d_nyk, h->d_rowoff, h->d_nb, h->d_cx0, h->d_cy0,
                  h->d_ox, h->d_oy, h->d_w, h->d_sw, h->d_sig_s, h->d_sig_t, h->d_sQ,
                  h->d_angcand, h->d_X[0], h->d_X[1], h->d_V[0], h->d_V[1], h->d_S[0],
                  h->d_S[1], h->d_r[0], h->d_r[1], h->d_L0, h->d_Hw, h->d_Hwa, h->d_Vh,
                  h->d_K, h->d_X1, h->d_L, h->d_V1, h->d_Kb, h->d_sm, h->d_part, h->d_sig,
                  h->d_rho, h->d_fluxw, h->d_m, h->d_rt, h->d_rx, h->d_rc, h->d_p, h->d_status,
                  h->d_flag, h->d_scale};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (h->graph_ready) cudaGraphExecDestroy(h->graph_exec);
}

}  // namespace

namespace dd {

dd_status set_error(dd_status s, const char* msg) { return fail(s, msg); }

// Scalar flux with the per-subdomain scratch at a caller-supplied device address.
dd_status noalloc_flux_impl(dd_dlra_t h, double* scratch, int scratch_doubles, double* out) {
  g_err.clear();
  int dev = -1;
  DD_CUDA(cudaGetDevice(&dev));
  if (dev != h->device) return fail(DD_ERR_ARG, "call on the device the solver was created on");
  if ((long)h->nsub * h->RC > scratch_doubles)
    return fail(DD_ERR_ARG, "nsub * r_cap = " + std::to_string((long)h->nsub * h->RC) +
                                " exceeds the allocation-free scratch of " +
                                std::to_string(scratch_doubles) + " doubles");
  dd::scalar_flux(h->P, h->d_X[0], h->d_V[0], h->d_S[0], h->d_r[0], scratch, out, h->nx, h->stream);
  DD_CUDA(cudaGetLastError());
  return DD_OK;
}

}  // namespace dd

extern "C" {

const char* dd_last_error(void) { return g_err.c_str(); }

dd_status dd_dlra_create(const dd_grid* grid, const dd_tiling* tiling, const dd_quadrature* quad,
                         const dd_fields* fields, const double* g0, const dd_options* opt,
                         void* stream, dd_dlra_t* out) {
  g_err.clear();
  if (!grid || !tiling || !quad || !fields || !g0 || !opt || !out)
    return fail(DD_ERR_ARG, "null argument");
  *out = nullptr;
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
  if (quad->n <= 0 || !quad->omega_x || !quad->omega_y || !quad->w)
    return fail(DD_ERR_ARG, "bad quadrature");
  for (int i = 0; i < quad->n; ++i)
    if (!(quad->w[i] > 0.0)) return fail(DD_ERR_ARG, "quadrature weights must be positive");
  if (opt->rank_mode != DD_RANK_FIXED && opt->rank_mode != DD_RANK_TOL)
    return fail(DD_ERR_ARG, "rank_mode");
  if (opt->integrator != DD_EULER && opt->integrator != DD_RK4)
    return fail(DD_ERR_ARG, "integrator");
  if (opt->precision != DD_FP64 && opt->precision != DD_MIXED)
    return fail(DD_ERR_ARG, "precision");
  if (!(opt->dt > 0.0) || !(opt->tau >= 0.0)) return fail(DD_ERR_ARG, "dt / tau");

  dd_dlra* h = new dd_dlra();   // value-initialised: every device pointer starts null
  cudaGetDevice(&h->device);
  h->nx = grid->nx; h->ny = grid->ny; h->tx = tiling->tx; h->ty = tiling->ty;
  h->nsub = h->tx * h->ty; h->n = quad->n;
  h->hx = (grid->x1 - grid->x0) / grid->nx;
  h->hy = (grid->y1 - grid->y0) / grid->ny;
  h->sh = std::sqrt(h->hx * h->hy);
  h->opt = *opt;
  h->stream = reinterpret_cast<cudaStream_t>(stream);
  h->ssum = 0.0;
  for (int i = 0; i < quad->n; ++i) h->ssum += quad->w[i];
  h->RS = opt->rank_mode == DD_RANK_FIXED ? opt->rank : opt->r_max;
  h->MC = 3 * h->RS;
  // column capacity of every tall and small matrix: the intermediate rank and the
  // augmentation input width both fit
  h->RC = std::max(opt->r_aug_max, h->MC);
  h->r_floor = opt->rank_mode == DD_RANK_FIXED ? opt->rank : opt->r_min;
  auto bail = [&](dd_status s, const std::string& m) {
    free_all(h);
    delete h;
    return fail(s, m);
  };
  if (opt->r_aug_max < 1 || opt->r_aug_max > DD_MAXC)
    return bail(DD_ERR_ARG, "r_aug_max must be in [1, 64]");
  if (h->RS < 1 || h->RS > opt->r_aug_max)
    return bail(DD_ERR_ARG, "stored-rank cap must be in [1, r_aug_max]");
  if (h->MC > DD_MAXC) return bail(DD_ERR_ARG, "3 * stored-rank cap must be <= 64");
  if (h->n < h->MC) return bail(DD_ERR_ARG, "need at least 3 * stored-rank cap directions");
  if (h->r_floor < 0 || h->r_floor > h->RS) return bail(DD_ERR_ARG, "rank floor");

  // geometry
  h->geo.resize(h->nsub);
  int rowoff = 0;
  h->maxlines = 0;
  h->maxN = 0;
  for (int J = 0; J < h->ty; ++J)
    for (int I = 0; I < h->tx; ++I) {
      int k = J * h->tx + I;
      SubGeo& s = h->geo[k];
      s.cx0 = tiling->xcuts[I];
      s.cy0 = tiling->ycuts[J];
      s.nxk = tiling->xcuts[I + 1] - s.cx0;
      s.nyk = tiling->ycuts[J + 1] - s.cy0;
      s.N = s.nxk * s.nyk;
      s.rowoff = rowoff;
      rowoff += s.N;
      s.nb[0] = I > 0 ? k - 1 : -1;
      s.nb[1] = I < h->tx - 1 ? k + 1 : -1;
      s.nb[2] = J > 0 ? k - h->tx : -1;
      s.nb[3] = J < h->ty - 1 ? k + h->tx : -1;
      h->maxlines = std::max(h->maxlines, std::max(s.nxk, s.nyk));
      h->maxN = std::max(h->maxN, s.N);
    }
  h->Ntot = rowoff;
  if (h->maxlines * h->RC > DD_THREADS * 24)
    return bail(DD_ERR_ARG, "subdomain side x r_aug_max exceeds the K-step tile (6144)");

  const int RC = h->RC, n = h->n, nsub = h->nsub, MC = h->MC;
  const long Nt = h->Ntot;
  {
    std::vector<int> vN(nsub), vnx(nsub), vny(nsub), vro(nsub), vnb(4 * nsub), vcx(nsub), vcy(nsub);
    for (int k = 0; k < nsub; ++k) {
      vN[k] = h->geo[k].N; vnx[k] = h->geo[k].nxk; vny[k] = h->geo[k].nyk;
      vro[k] = h->geo[k].rowoff; vcx[k] = h->geo[k].cx0; vcy[k] = h->geo[k].cy0;
      for (int s = 0; s < 4; ++s) vnb[4 * k + s] = h->geo[k].nb[s];
    }
#define UP_INT(dst, v)                                                                       \
  if (dalloc(&dst, v.size()) != cudaSuccess ||                                                \
      cudaMemcpy(dst, v.data(), sizeof(int) * v.size(), cudaMemcpyHostToDevice) != cudaSuccess) \
    return bail(DD_ERR_CUDA, "upload geometry");
    UP_INT(h->d_N, vN); UP_INT(h->d_nxk, vnx); UP_INT(h->d_nyk, vny); UP_INT(h->d_rowoff, vro);
    UP_INT(h->d_nb, vnb); UP_INT(h->d_cx0, vcx); UP_INT(h->d_cy0, vcy);
#undef UP_INT
  }
  // problem data
  std::vector<double> sw(n), sig_s(Nt), sig_t(Nt), sQ(Nt);
  for (int q = 0; q < n; ++q) sw[q] = std::sqrt(quad->w[q]);
  h->sw_host = sw;
  for (int k = 0; k < nsub; ++k) {
    const SubGeo& s = h->geo[k];
    for (int c = 0; c < s.N; ++c) {
      int gi = (s.cy0 + c / s.nxk) * h->nx + s.cx0 + c % s.nxk;
      sig_s[s.rowoff + c] = fields->sigma_s[gi];
      sig_t[s.rowoff + c] = fields->sigma_s[gi] + fields->sigma_a[gi];
      sQ[s.rowoff + c] = h->sh * fields->source[gi];
    }
  }
  std::vector<double> tab;
  angular_family(quad, h->ssum, tab, 4 * RC + 16, &h->angcand_complete);
  h->n_angcand = (int)(tab.size() / n);
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
  ok &= dalloc(&h->d_rho, (long)h->nx * h->ny) == cudaSuccess;
  ok &= dalloc(&h->d_fluxw, (long)nsub * RC) == cudaSuccess;
  ok &= dalloc(&h->d_m, nsub) == cudaSuccess;
  ok &= dalloc(&h->d_rt, nsub) == cudaSuccess;
  ok &= dalloc(&h->d_rx, 2 * nsub) == cudaSuccess;
  ok &= dalloc(&h->d_rc, nsub) == cudaSuccess;
  ok &= dalloc(&h->d_p, nsub) == cudaSuccess;
  ok &= dalloc(&h->d_flag, nsub) == cudaSuccess;
  ok &= dalloc(&h->d_scale, nsub) == cudaSuccess;
  ok &= dalloc(&h->d_status, 1) == cudaSuccess;
  if (!ok) return bail(DD_ERR_CUDA, "device allocation failed");

  // problem descriptor
  dd::Problem& P = h->P;
  P.g.nsub = nsub; P.g.n = n; P.g.RC = RC; P.g.MC = MC;
  P.g.N = h->d_N; P.g.nxk = h->d_nxk; P.g.nyk = h->d_nyk; P.g.rowoff = h->d_rowoff;
  P.g.nb = h->d_nb; P.g.cx0 = h->d_cx0; P.g.cy0 = h->d_cy0;
  P.maxlines = h->maxlines; P.maxN = h->maxN;
  P.ox = h->d_ox; P.oy = h->d_oy; P.w = h->d_w; P.sw = h->d_sw;
  P.sig_s = h->d_sig_s; P.sig_t = h->d_sig_t; P.sQ = h->d_sQ;
  P.hx = h->hx; P.hy = h->hy; P.sh = h->sh; P.dt = opt->dt; P.c_adv = opt->c_adv; P.ssum = h->ssum;
  P.integrator = opt->integrator; P.rank_mode = opt->rank_mode; P.tol = opt->tol;
  P.prec = opt->precision == DD_MIXED ? 1 : 0;
  P.tau = opt->tau; P.accept = 0.5;
  P.r_floor = h->r_floor; P.r_aug_max = opt->r_aug_max; P.RS = h->RS; P.WC = WC;
  P.angcand = h->d_angcand; P.n_angcand = h->n_angcand; P.angcand_complete = h->angcand_complete;
  P.nchunk_sp = std::max(1, std::min(16, h->maxN / 64));
  P.nchunk_ang = std::max(1, std::min(16, n / 64));
  if (dalloc(&h->d_part, dd::part_elems(P)) != cudaSuccess)
    return bail(DD_ERR_CUDA, "device allocation failed");
  if (dd::orth_init() != cudaSuccess || dd::phase_init(P) != cudaSuccess)
    return bail(DD_ERR_CUDA, "kernel attribute setup failed");

  // isotropic initial data at rank 1 (rank 0 where g0 vanishes on the subdomain)
  {
    std::vector<double> X((size_t)Nt * RC, 0.0), V((size_t)nsub * n * RC, 0.0),
        S((size_t)nsub * RC * RC, 0.0);
    std::vector<int> r(nsub, 0);
    for (int k = 0; k < nsub; ++k) {
      const SubGeo& s = h->geo[k];
      double nn = 0.0;
      for (int c = 0; c < s.N; ++c) {
        double gv = g0[(s.cy0 + c / s.nxk) * h->nx + s.cx0 + c % s.nxk];
        nn += gv * gv;
      }
      nn = std::sqrt(nn);
      if (!(nn > 0.0)) continue;
      r[k] = 1;
      for (int c = 0; c < s.N; ++c)
        X[(size_t)(s.rowoff + c) * RC] = g0[(s.cy0 + c / s.nxk) * h->nx + s.cx0 + c % s.nxk] / nn;
      for (int q = 0; q < n; ++q) V[((size_t)k * n + q) * RC] = sw[q] / std::sqrt(h->ssum);
      S[(size_t)k * RC * RC] = nn * h->sh * std::sqrt(h->ssum);
    }
    for (int b = 0; b < 2; ++b) {
      if (cudaMemcpy(h->d_X[b], X.data(), sizeof(double) * X.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
          cudaMemcpy(h->d_V[b], V.data(), sizeof(double) * V.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
          cudaMemcpy(h->d_S[b], S.data(), sizeof(double) * S.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
          cudaMemcpy(h->d_r[b], r.data(), sizeof(int) * nsub, cudaMemcpyHostToDevice) != cudaSuccess)
        return bail(DD_ERR_CUDA, "upload initial state");
    }
    if (cudaMemset(h->d_status, 0, sizeof(unsigned)) != cudaSuccess ||
        cudaMemset(h->d_sm, 0, sizeof(double) * (size_t)nsub * dd::NSMALL * RC * RC) != cudaSuccess ||
        cudaMemset(h->d_rx, 0, sizeof(int) * 2 * nsub) != cudaSuccess)
      return bail(DD_ERR_CUDA, "clear workspace");
  }
  if (cudaDeviceSynchronize() != cudaSuccess) return bail(DD_ERR_CUDA, "create: device error");
  *out = h;
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
    DD_CUDA(cudaMemcpyAsync(out, h->d_rho, sizeof(double) * (size_t)h->nx * h->ny,
                            cudaMemcpyDeviceToHost, h->stream));
    return check_status(h);
  }
  return DD_OK;
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
    for (int t = 0; t < rk; ++t) U[(size_t)c * rk + t] = X[(size_t)c * RC + t] / h->sh;
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
    for (int t = 0; t < r; ++t) X[(size_t)c * RC + t] = U[(size_t)c * r + t] * h->sh;
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
  g_err.clear();
  if (!h || nsteps < 0 || !ms || !launches) return fail(DD_ERR_ARG, "bad argument");
  for (int i = 0; i < dd::NSLOT; ++i) { ms[i] = 0.0; launches[i] = 0; }
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
  if (st != DD_OK) return st;
  return check_status(h);
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
