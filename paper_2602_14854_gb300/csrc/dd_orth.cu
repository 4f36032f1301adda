// Rank-revealing orthonormalisation with deterministic basis completion.
//
// Serves three steps of the scheme:
//   ORTH_QR       "perform a QR decomposition of K (of L)" (Algorithms 1-3, steps 2
//                 and 5): an orthonormal basis of the numerically significant
//                 column span of K (L), completed to r_out columns;
//   ORTH_AUG      the SVD and rank choice of the augmentation (Algorithm 4, steps
//                 2-4): leading left singular vectors of
//                 L0 = [V S^T, V_L S_L^T, V_R S_R^T], r_t chosen by the tail rule,
//                 completed to r_t columns;
//   ORTH_COMPLETE pad an orthonormal basis to r_out columns (collision step started
//                 below the rank floor).
//
// A singular value sigma_j counts as significant when sigma_j > tau * sigma_1.
//
// Fast path (all SMs): CholeskyQR2 of the tall input.  Gram G1 = A^T A (chunked
// over rows), R1 = chol(G1), Q1 = A R1^-1, G2 = Q1^T Q1, R2 = chol(G2), R = R2 R1;
// one-sided Jacobi SVD of R gives the singular values and the left singular basis
// U_R; the output is Q1 (R2^-1 U_R).  It is taken only when every singular value
// is significant and no completion is needed (then the span it returns is the
// input's, to ~eps * cond <= 1e-11); otherwise the subdomain is flagged.
//
// Fallback (one CTA per flagged subdomain): exact power-of-two scaling of a copy,
// Householder QR (in shared memory when it fits), explicit Q_H by backward
// accumulation in place of the reflectors, one-sided Jacobi SVD of R (on the rows
// of R, accumulating the rotations: the accumulated orthogonal matrix is the left
// singular basis U_R), significant left singular vectors Q_H U_R, and missing
// columns taken in order from a fixed exactly-orthogonal candidate family, each
// Gram-Schmidt'd twice and accepted when its residual norm is >= accept:
//   space: cos(pi a (i+1/2)/nx_k) cos(pi b (j+1/2)/ny_k), by a+b then a descending;
//   angle: the table built at create time (P_2l(mu) x cos/sin(m phi), weighted by
//          sqrt(w)), then the unit vectors.
#include "dd_internal.cuh"
#include "dd_launch.h"

#include <math_constants.h>

namespace dd {

// Rank decision shared by both paths (one thread).  sig[] descending, scaled by
// 2^-e; returns p, sets *keep and *r_out.
__device__ int decide(const OrthArgs& a, int k, const double* sig, int nref, int e, int* keep,
                      int* r_out) {
  int p = 0;
  double s1 = nref > 0 ? sig[0] : 0.0;
  if (s1 > 0.0)
    for (int t = 0; t < nref; ++t)
      if (sig[t] > a.tau * s1) ++p;
  const double unscale = ldexp(1.0, e);
  if (a.sig_out)
    for (int t = 0; t < DD_MAXC; ++t) a.sig_out[(long)k * DD_MAXC + t] = t < nref ? sig[t] * unscale : 0.0;
  if (a.p_out) a.p_out[k] = p;
  if (a.mode == ORTH_QR) {
    *r_out = a.rout[k];
    *keep = min(p, *r_out);
  } else {  // ORTH_AUG
    int r_tail = p;
    if (a.rank_mode == 1) {
      r_tail = nref;
      for (int r = 0; r <= nref; ++r) {
        double ss = 0.0;
        for (int t = r; t < nref; ++t) {
          double x = sig[t] * unscale;
          ss += x * x;
        }
        if (sqrt(ss) <= a.tol) { r_tail = r; break; }
      }
    }
    int r_sig = min(r_tail, p);
    int cap = min(min(a.g.raug[k], a.g.n), a.g.N[k]);
    int fl = max(a.r_own[k], a.g.rlo[k]);
    int rt = min(max(r_sig, fl), cap);
    *r_out = rt;
    *keep = min(rt, p);
  }
  return p;
}

// ---------------------------------------------------------------------------
// fast path, small kernels (one CTA per subdomain)
// ---------------------------------------------------------------------------
// Cholesky s*G = R^T R of the m x m matrix G (row-major, ld) into upper R
// (row-major, ld), by one warp (lanes over columns); Gw is m x ld scratch.
// Returns 0 on a non-positive pivot.
__device__ int chol_upper_warp(const double* G, int ld, int m, double s, double* R, double* Gw) {
  const int lane = threadIdx.x & 31;
  for (int e = lane; e < m * ld; e += 32) Gw[e] = G[e] * s;
  __syncwarp();
  for (int j = 0; j < m; ++j) {
    const double d = Gw[j * ld + j];
    if (!(d > 0.0)) return 0;
    const double rd = sqrt(d);
    for (int c = lane; c < ld; c += 32)
      R[j * ld + c] = (c < j || c >= m) ? 0.0 : (c == j ? rd : Gw[j * ld + c] / rd);
    __syncwarp();
    for (int c = j + 1 + lane; c < m; c += 32) {
      const double rc = R[j * ld + c];
      for (int r = j + 1; r <= c; ++r) Gw[r * ld + c] -= R[j * ld + r] * rc;
    }
    __syncwarp();
  }
  for (int j = m; j < ld; ++j)
    for (int c = lane; c < ld; c += 32) R[j * ld + c] = 0.0;
  __syncwarp();
  return 1;
}

// Inverse of the upper-triangular R into Ri (lanes / threads over columns).
__device__ void tri_inv_upper(const double* R, int ld, int m, double* Ri, int tid, int nthr) {
  for (int c = tid; c < ld; c += nthr) {
    for (int i = ld - 1; i >= 0; --i) {
      double x = 0.0;
      if (c < m && i <= c) {
        x = (i == c) ? 1.0 : 0.0;
        for (int l = i + 1; l <= c; ++l) x -= R[i * ld + l] * Ri[l * ld + c];
        x /= R[i * ld + i];
      }
      Ri[i * ld + c] = x;
    }
  }
}

// pass 1 (one warp per subdomain): R1 = chol(s G1), R1^-1.  Flags the subdomain
// when the factorisation fails or the diagonal ratio exceeds 1e7.
__global__ void k_cqr1(OrthArgs a, const double* sm, int sG, int sR, int sRi, double* smw,
                       int* flag, double* scale) {
  extern __shared__ double shm[];
  const int k = blockIdx.x, RC = a.g.RC, lane = threadIdx.x & 31;
  const int m = a.acols[k];
  const double* G = sm + ((long)k * NSMALL + sG) * RC * RC;
  double* R = smw + ((long)k * NSMALL + sR) * RC * RC;
  double* Ri = smw + ((long)k * NSMALL + sRi) * RC * RC;
  double* Rs = shm;
  double* Gw = Rs + RC * RC;
  double dmax = 0.0;
  bool fin = true;
  for (int j = lane; j < m; j += 32) dmax = fmax(dmax, G[j * RC + j]);
  for (int e = lane; e < m * RC; e += 32) fin = fin && isfinite(G[e]);
  dmax = warp_max(dmax);
  fin = __all_sync(0xffffffffu, fin);
  int ok = 0;
  double s = 1.0;
  if (m > 0 && fin && dmax > 0.0 && isfinite(dmax)) {
    s = ldexp(1.0, -ilogb(dmax));
    ok = chol_upper_warp(G, RC, m, s, Rs, Gw);
    if (ok) {
      double lo = 1e300, hi = 0.0;
      for (int j = lane; j < m; j += 32) { lo = fmin(lo, Rs[j * RC + j]); hi = fmax(hi, Rs[j * RC + j]); }
      lo = -warp_max(-lo);
      hi = warp_max(hi);
      if (!(lo > 1e-7 * hi)) ok = 0;
    }
  }
  if (!fin && lane == 0) atomicOr(a.status, (unsigned)ST_NONFINITE);
  if (lane == 0) { flag[k] = ok ? 0 : 1; scale[k] = s; }
  if (!ok) return;
  for (int e = lane; e < RC * RC; e += 32) R[e] = Rs[e];
  tri_inv_upper(Rs, RC, m, Ri, lane, 32);
}

// pass 2: R2 = chol(G2), R = R2 R1.  Every singular value of the input is
// significant when |R|_F |R^-1|_F < 1/tau (the Frobenius condition bound is an
// upper bound of the 2-norm one).  Then, when the output keeps all m columns, the
// transform is M = R2^-1; when it keeps fewer (the augmentation's leading r_t of m
// singular vectors, or a tolerance rule), the one-sided Jacobi SVD of R supplies
// U_R and M = R2^-1 U_R[:, :keep].  Otherwise the subdomain is flagged.
__global__ void k_cqr2(OrthArgs a, const double* sm, int sG2, int sR1, int sR1i, double* smw,
                       int sM, int* flag, const double* scale) {
  extern __shared__ double shm[];
  const int k = blockIdx.x, RC = a.g.RC;
  if (flag[k]) return;
  const int m = a.acols[k];
  const double* G2 = sm + ((long)k * NSMALL + sG2) * RC * RC;
  const double* R1 = smw + ((long)k * NSMALL + sR1) * RC * RC;
  const double* R1i = smw + ((long)k * NSMALL + sR1i) * RC * RC;
  double* M = smw + ((long)k * NSMALL + sM) * RC * RC;
  double* R2 = shm;                   // RC*RC row-major
  double* R2i = R2 + RC * RC;
  double* Bc = R2i + RC * RC;         // column-major B = R^T
  double* Jc = Bc + RC * RC;
  double* sig = Jc + RC * RC;
  double* pw = sig + RC;              // 2 x RC power-iteration vectors
  int* perm = reinterpret_cast<int*>(pw + 2 * RC);
  int* iv = perm + RC;
  __shared__ double red[40];
  if (threadIdx.x < 32) {
    int ok = chol_upper_warp(G2, RC, m, 1.0, R2, Bc);
    if (threadIdx.x == 0) iv[0] = ok;
  }
  __syncthreads();
  if (!iv[0]) {
    if (threadIdx.x == 0) flag[k] = 1;
    return;
  }
  tri_inv_upper(R2, RC, m, R2i, threadIdx.x, blockDim.x);
  __syncthreads();
  // R = R2 R1 (into Bc as B = R^T, column-major) and R^-1 = R1^-1 R2^-1 (Frobenius norms)
  double nr = 0.0, ni = 0.0;
  for (int e = threadIdx.x; e < RC * RC; e += blockDim.x) {
    int col = e / RC, row = e % RC;
    double x = 0.0, y = 0.0;
    if (col < m && row < m && row >= col) {
      for (int l = col; l <= row; ++l) {
        x += R2[col * RC + l] * R1[l * RC + row];
        y += R1i[col * RC + l] * R2i[l * RC + row];
      }
    }
    Bc[col * RC + row] = x;
    Jc[col * RC + row] = (row == col) ? 1.0 : 0.0;
    nr += x * x;
    ni += y * y;
  }
  nr = block_sum(nr, red);
  ni = block_sum(ni, red);
  bool well = sqrt(nr) * sqrt(ni) * a.tau < 1.0;
  if (!well) {
    // exact certificate: every singular value of R exceeds tau * sigma_max iff
    // R^T R - tau^2 sigma_max^2 I is positive definite.  sigma_max^2 comes from a
    // power iteration (a lower estimate, so the shift carries a 1% margin);
    // cases within the margin go to the exact SVD / fallback.
    double* GR = R2i;                 // scratch; R2^-1 is recomputed below
    double* wv = pw;
    double* wn = pw + RC;
    __shared__ double lam;
    __shared__ int cert;
    // GR = R^T R from B (column c of B = row c of R)
    __syncthreads();
    double* G = Jc + 0;               // Jc is re-initialised before the SVD
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
      int i = e / m, j = e % m;
      double x = 0.0;
      for (int l = 0; l < m; ++l) x += Bc[l * RC + i] * Bc[l * RC + j];
      G[i * RC + j] = x;
    }
    for (int i = threadIdx.x; i < m; i += blockDim.x) wv[i] = 1.0 + 0.01 * i;
    __syncthreads();
    for (int it = 0; it < 40; ++it) {
      for (int i = threadIdx.x; i < m; i += blockDim.x) {
        double x = 0.0;
        for (int j = 0; j < m; ++j) x += G[i * RC + j] * wv[j];
        wn[i] = x;
      }
      __syncthreads();
      double nn = 0.0;
      for (int i = threadIdx.x; i < m; i += blockDim.x) nn += wn[i] * wn[i];
      nn = block_sum(nn, red);
      double dn = 0.0;
      for (int i = threadIdx.x; i < m; i += blockDim.x) dn += wn[i] * wv[i];
      dn = block_sum(dn, red);
      const double inv = nn > 0.0 ? rsqrt(nn) : 0.0;
      for (int i = threadIdx.x; i < m; i += blockDim.x) wv[i] = wn[i] * inv;
      if (threadIdx.x == 0) lam = dn;   // Rayleigh quotient (w normalised after the first pass)
      __syncthreads();
    }
    if (threadIdx.x < 32) {
      const double shift = 1.01 * a.tau * a.tau * lam;
      if (threadIdx.x == 0)
        for (int i = 0; i < m; ++i) G[i * RC + i] -= shift;
      __syncwarp();
      int ok = lam > 0.0 ? chol_upper_warp(G, RC, m, 1.0, GR, Bc) : 0;
      if (threadIdx.x == 0) cert = ok;
    }
    __syncthreads();
    well = cert != 0;
    // restore what the rest of the kernel reads: B = R^T, J = I, R2^-1
    for (int e = threadIdx.x; e < RC * RC; e += blockDim.x) {
      int col = e / RC, row = e % RC;
      double x = 0.0;
      if (col < m && row < m && row >= col)
        for (int l = col; l <= row; ++l) x += R2[col * RC + l] * R1[l * RC + row];
      Bc[col * RC + row] = x;
      Jc[col * RC + row] = (row == col) ? 1.0 : 0.0;
    }
    __syncthreads();
    tri_inv_upper(R2, RC, m, R2i, threadIdx.x, blockDim.x);
    __syncthreads();
  }
  int need_svd = 0;
  if (threadIdx.x == 0) {
    int keep_all = 0;
    if (well) {
      if (a.mode == ORTH_QR) keep_all = (a.rout[k] == m);
      else if (a.rank_mode == 0) {                      // fixed mode: r_t = min(max(m, floor), cap)
        int cap = min(min(a.g.raug[k], a.g.n), a.g.N[k]);
        int rt = min(max(m, max(a.r_own[k], a.g.rlo[k])), cap);
        keep_all = (rt == m);
        if (keep_all) a.rt_out[k] = m;
      }
    }
    iv[2] = keep_all;
    iv[3] = m;
    need_svd = well && !keep_all && a.mode == ORTH_AUG;
    iv[4] = need_svd;
    if (!well || (!keep_all && !need_svd)) flag[k] = 1;
  }
  __syncthreads();
  if (iv[4]) {
    // leading singular vectors needed: leave B = R^T and R2^-1 for the SVD launch
    double* Bo = smw + ((long)k * NSMALL + sG2) * RC * RC;
    double* Ro = smw + ((long)k * NSMALL + sR1i) * RC * RC;
    for (int e = threadIdx.x; e < RC * RC; e += blockDim.x) {
      Bo[e] = Bc[e];
      Ro[e] = R2i[e];
    }
    if (threadIdx.x == 0) flag[k] = 2;
    return;
  }
  if (!iv[2]) return;
  const int keep = iv[3];
  // M = R2^-1 (all columns kept); zero elsewhere
  for (int e = threadIdx.x; e < RC * RC; e += blockDim.x) {
    int i = e / RC, t = e % RC;
    M[e] = (i < m && t < keep) ? R2i[i * RC + t] : 0.0;
  }
}

size_t cqr2_smem_bytes(int RC) {
  return sizeof(double) * (4 * RC * RC + 3 * RC) + sizeof(int) * (RC + 8);
}

// ---------------------------------------------------------------------------
// fallback (one CTA per flagged subdomain)
// ---------------------------------------------------------------------------
struct OrthSmem {
  double* Bc;   // mcap x mcap, column-major: column j of B = R^T = row j of R
  double* Jc;   // mcap x mcap, column-major accumulated rotations
  double* tau;  // Householder scalars
  double* sig;  // singular values
  double* wv;   // dot products
  double* red;  // reduction scratch (40)
  double* dv;   // double scalars
  int* perm;    // descending order of sig
  int* iv;      // integer scalars
  double* X;    // scratch of the mixed-precision SVD (jacobi_mixed_scratch_bytes(mcap))
  double* W;    // staged matrix (shared-memory variant), column-major rows x m
};

__device__ OrthSmem carve(void* base, int mcap) {
  OrthSmem s;
  double* d = reinterpret_cast<double*>(base);
  s.Bc = d; d += mcap * mcap;
  s.Jc = d; d += mcap * mcap;
  s.tau = d; d += DD_MAXC;
  s.sig = d; d += DD_MAXC;
  s.wv = d; d += DD_MAXC;
  s.red = d; d += 40;
  s.dv = d; d += 8;
  s.perm = reinterpret_cast<int*>(d);
  s.iv = s.perm + DD_MAXC;
  d += (DD_MAXC + 16) / 2;
  s.X = d;
  d += (jacobi_mixed_scratch_bytes(mcap) + 7) / 8;
  s.W = d;
  return s;
}

size_t orth_smem_base(int mcap) {
  return sizeof(double) * (2 * mcap * mcap + 3 * DD_MAXC + 48) + sizeof(int) * (DD_MAXC + 16) +
         8 * ((jacobi_mixed_scratch_bytes(mcap) + 7) / 8);
}

template <bool SMEM>
__global__ void __launch_bounds__(DD_THREADS) k_orth(OrthArgs a, int mcap, const int* flag,
                                                      const double* sm_small, int sB, int sR2i) {
  extern __shared__ double smem_raw[];
  const int k = blockIdx.x;
  if (flag && flag[k] == 0) return;
  const int how = flag ? flag[k] : 1;     // 1: full fallback, 2: SVD of the fast path's R
  OrthSmem sm = carve(smem_raw, mcap);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  const Geo& g = a.g;
  const int rows = a.spatial ? g.N[k] : g.n;
  const long rbase = a.spatial ? (long)g.rowoff[k] : (long)k * g.n;
  const double* A = a.A + rbase * a.lda;
  double* Wg = a.W + rbase * a.ldw;
  double* Q = a.Q + rbase * a.ldq;
  const int m = a.acols[k];
  int* iv = sm.iv;
  double* dv = sm.dv;
  // element (i, j) of the working copy
  auto Wp = [&](int i, int j) -> double& {
    return SMEM ? sm.W[(long)j * rows + i] : Wg[(long)i * a.ldw + j];
  };

  int keep = 0, r_out = 0;

  if (a.mode == ORTH_COMPLETE) {
    for (int i = tid; i < rows; i += blockDim.x)
      for (int t = 0; t < m; ++t) Q[(long)i * a.ldq + t] = A[(long)i * a.lda + t];
    keep = m;
    r_out = a.rout[k];
    __syncthreads();
  } else if (how == 2) {
    // The fast path proved the input well conditioned and left B = R^T (A = Q1 R2^-1 R,
    // Q1 in the workspace) and R2^-1: the left singular vectors of A are
    // Q1 R2^-1 U_R, U_R from the SVD of R.
    const int RC = g.RC;
    const double* Bs = sm_small + ((long)k * NSMALL + sB) * RC * RC;
    const double* R2i = sm_small + ((long)k * NSMALL + sR2i) * RC * RC;
    for (int idx = tid; idx < mcap * mcap; idx += blockDim.x) {
      int col = idx / mcap, row = idx % mcap;
      sm.Bc[idx] = (col < m && row < m) ? Bs[col * RC + row] : 0.0;
      sm.Jc[idx] = (row == col) ? 1.0 : 0.0;
    }
    __syncthreads();
    jacobi_svd_mixed(sm.Bc, sm.Jc, m, mcap, &iv[0], sm.sig, sm.X);
    for (int j = warp; j < m; j += nwarps) {
      double s = 0.0;
      for (int l = lane; l < m; l += 32) s += sm.Bc[j * mcap + l] * sm.Bc[j * mcap + l];
      s = warp_sum(s);
      if (lane == 0) sm.sig[j] = sqrt(s);
    }
    __syncthreads();
    if (tid == 0) {
      for (int t = 0; t < m; ++t) sm.perm[t] = t;
      for (int t = 0; t < m; ++t) {
        int best = t;
        for (int u = t + 1; u < m; ++u)
          if (sm.sig[sm.perm[u]] > sm.sig[sm.perm[best]]) best = u;
        int tmp = sm.perm[t]; sm.perm[t] = sm.perm[best]; sm.perm[best] = tmp;
      }
      double ss[DD_MAXC];
      for (int t = 0; t < m; ++t) ss[t] = sm.sig[sm.perm[t]];
      decide(a, k, ss, m, 0, &keep, &r_out);
      if (a.mode == ORTH_AUG) a.rt_out[k] = r_out;
      iv[1] = keep;
      iv[2] = r_out;
    }
    __syncthreads();
    keep = iv[1];
    r_out = iv[2];
    // M = R2^-1 U_R[:, :keep] (column-major m x keep, in the mixed-SVD scratch)
    double* M = sm.X;
    for (int e = tid; e < m * keep; e += blockDim.x) {
      int t = e / m, i = e % m;
      double x = 0.0;
      for (int l = i; l < m; ++l) x += R2i[i * RC + l] * sm.Jc[sm.perm[t] * mcap + l];
      M[t * m + i] = x;
    }
    __syncthreads();
    for (long idx = tid; idx < (long)rows * keep; idx += blockDim.x) {
      int i = (int)(idx / keep), t = (int)(idx % keep);
      const double* q1 = Wg + (long)i * a.ldw;
      double x = 0.0;
      for (int j = 0; j < m; ++j) x += q1[j] * M[t * m + j];
      Q[(long)i * a.ldq + t] = x;
    }
    __syncthreads();
  } else {
    // ---- 1. exact power-of-two scaling of a copy --------------------------------
    double mx = 0.0;
    bool bad = false;
    for (int i = tid; i < rows; i += blockDim.x)
      for (int t = 0; t < m; ++t) {
        double x = A[(long)i * a.lda + t];
        if (!isfinite(x)) bad = true;
        mx = fmax(mx, fabs(x));
      }
    if (bad) atomicOr(a.status, (unsigned)ST_NONFINITE);
    double amax = block_max(mx, sm.red);
    int e = 0;
    if (amax > 0.0 && isfinite(amax)) e = ilogb(amax) + 1;
    const double sc = ldexp(1.0, -e);
    for (long idx = tid; idx < (long)rows * m; idx += blockDim.x) {
      int i = (int)(idx / m), t = (int)(idx % m);
      Wp(i, t) = A[(long)i * a.lda + t] * sc;
    }
    __syncthreads();

    const bool zero = !(amax > 0.0) || !isfinite(amax);
    const int nref = zero ? 0 : min(m, rows);

    // ---- 2. Householder QR in place ------------------------------------------------
    for (int j = 0; j < nref; ++j) {
      double s = 0.0;
      for (int i = j + 1 + tid; i < rows; i += blockDim.x) {
        double x = Wp(i, j);
        s += x * x;
      }
      double xn2 = block_sum(s, sm.red);
      if (tid == 0) {
        double alpha = Wp(j, j);
        if (xn2 == 0.0) {
          sm.tau[j] = 0.0;
          dv[0] = 0.0;
        } else {
          double beta = -copysign(sqrt(alpha * alpha + xn2), alpha);
          sm.tau[j] = (beta - alpha) / beta;
          dv[0] = 1.0 / (alpha - beta);
          dv[1] = beta;
        }
      }
      __syncthreads();
      const double tj = sm.tau[j];
      if (tj != 0.0) {
        const double vs = dv[0];
        for (int i = j + 1 + tid; i < rows; i += blockDim.x) Wp(i, j) *= vs;
        __syncthreads();
        if (tid == 0) Wp(j, j) = dv[1];
        for (int c = j + 1 + warp; c < m; c += nwarps) {
          double d = (lane == 0) ? Wp(j, c) : 0.0;
          for (int i = j + 1 + lane; i < rows; i += 32) d += Wp(i, j) * Wp(i, c);
          d = warp_sum(d);
          if (lane == 0) sm.wv[c] = d;
        }
        __syncthreads();
        const int nc = m - j - 1;
        if (nc > 0) {
          const long tot = (long)(rows - j) * nc;
          for (long idx = tid; idx < tot; idx += blockDim.x) {
            int c = j + 1 + (int)(idx / (rows - j));
            int i = j + (int)(idx % (rows - j));
            double v = (i == j) ? 1.0 : Wp(i, j);
            Wp(i, c) -= tj * v * sm.wv[c];
          }
        }
        __syncthreads();
      }
    }

    // ---- 3. R -> B = R^T (column-major); explicit Q_H in place (backward accumulation)
    for (int idx = tid; idx < mcap * mcap; idx += blockDim.x) {
      int col = idx / mcap, row = idx % mcap;
      double b = 0.0;
      if (col < nref && row < nref && row >= col) b = Wp(col, row);
      sm.Bc[idx] = b;
      sm.Jc[idx] = (row == col) ? 1.0 : 0.0;
    }
    __syncthreads();
    for (int j = nref - 1; j >= 0; --j) {
      const double tj = sm.tau[j];
      if (tj != 0.0 && j < nref - 1) {
        for (int c = j + 1 + warp; c < nref; c += nwarps) {
          double d = 0.0;   // row j of the already formed columns is zero
          for (int i = j + 1 + lane; i < rows; i += 32) d += Wp(i, j) * Wp(i, c);
          d = warp_sum(d);
          if (lane == 0) sm.wv[c] = d;
        }
        __syncthreads();
        const int nc = nref - j - 1;
        const long tot = (long)(rows - j) * nc;
        for (long idx = tid; idx < tot; idx += blockDim.x) {
          int c = j + 1 + (int)(idx / (rows - j));
          int i = j + (int)(idx % (rows - j));
          double v = (i == j) ? 1.0 : Wp(i, j);
          Wp(i, c) -= tj * v * sm.wv[c];
        }
        __syncthreads();
      }
      for (int i = tid; i < rows; i += blockDim.x) {
        double x;
        if (i < j) x = 0.0;
        else if (i == j) x = 1.0 - tj;
        else x = -tj * Wp(i, j);
        Wp(i, j) = x;
      }
      __syncthreads();
    }

    // ---- 4. one-sided Jacobi SVD of R, rank decision --------------------------------
    jacobi_svd_mixed(sm.Bc, sm.Jc, nref, mcap, &iv[0], sm.sig, sm.X);
    for (int j = warp; j < nref; j += nwarps) {
      double s = 0.0;
      for (int l = lane; l < nref; l += 32) s += sm.Bc[j * mcap + l] * sm.Bc[j * mcap + l];
      s = warp_sum(s);
      if (lane == 0) sm.sig[j] = sqrt(s);
    }
    __syncthreads();
    if (tid == 0) {
      for (int t = 0; t < nref; ++t) sm.perm[t] = t;
      for (int t = 0; t < nref; ++t) {          // selection sort, descending, stable
        int best = t;
        for (int u = t + 1; u < nref; ++u)
          if (sm.sig[sm.perm[u]] > sm.sig[sm.perm[best]]) best = u;
        int tmp = sm.perm[t]; sm.perm[t] = sm.perm[best]; sm.perm[best] = tmp;
      }
      double ss[DD_MAXC];
      for (int t = 0; t < nref; ++t) ss[t] = sm.sig[sm.perm[t]];
      decide(a, k, ss, nref, e, &keep, &r_out);
      if (a.mode == ORTH_AUG) a.rt_out[k] = r_out;
      iv[1] = keep;
      iv[2] = r_out;
    }
    __syncthreads();
    keep = iv[1];
    r_out = iv[2];

    // ---- 5. significant left singular vectors: Q_H U_R[:, :keep] -----------------------
    for (long idx = tid; idx < (long)rows * keep; idx += blockDim.x) {
      int i = (int)(idx / keep), t = (int)(idx % keep);
      const double* u = sm.Jc + sm.perm[t] * mcap;
      double x = 0.0;
      for (int j = 0; j < nref; ++j) x += Wp(i, j) * u[j];
      Q[(long)i * a.ldq + t] = x;
    }
    __syncthreads();
  }

  // ---- 6. completion from the fixed family ---------------------------------------------
  int cur = keep;
  if (tid == 0) { iv[3] = 0; iv[4] = 0; iv[8] = 0; }   // spatial degree d, next a; angular index
  __syncthreads();
  const int nxk = a.spatial ? g.nxk[k] : 0, nyk = a.spatial ? g.nyk[k] : 0;
  const int nang = a.n_angcand + (a.angcand_complete ? g.n : 0);
  while (cur < r_out) {
    if (tid == 0) {
      int ok = 0;
      if (a.spatial) {
        // (a,b) with d = a+b ascending, a descending from min(d, nx-1), b < ny
        int d = iv[3], aa = iv[4];
        while (d <= nxk + nyk - 2) {
          if (aa >= 0 && d - aa < nyk) { ok = 1; break; }
          ++d;
          aa = min(d, nxk - 1);
        }
        if (ok) { iv[6] = aa; iv[7] = d - aa; iv[3] = d; iv[4] = aa - 1; }
        else { iv[3] = d; }
      } else {
        int ci = iv[8]++;
        if (ci < nang) { ok = 1; iv[6] = ci; }
      }
      iv[9] = ok;
    }
    __syncthreads();
    if (!iv[9]) {
      if (tid == 0) atomicOr(a.status, (unsigned)ST_COMPLETION);
      break;
    }
    double s = 0.0;
    if (a.spatial) {
      const int ca = iv[6], cb = iv[7];
      for (int i = tid; i < rows; i += blockDim.x) {
        int il = i % nxk, jl = i / nxk;
        double v = cos(CUDART_PI * ca * (il + 0.5) / nxk) * cos(CUDART_PI * cb * (jl + 0.5) / nyk);
        Q[(long)i * a.ldq + cur] = v;
        s += v * v;
      }
    } else {
      const int ci = iv[6];
      for (int i = tid; i < rows; i += blockDim.x) {
        double v = (ci < a.n_angcand) ? a.angcand[(long)ci * g.n + i] : ((i == ci - a.n_angcand) ? 1.0 : 0.0);
        Q[(long)i * a.ldq + cur] = v;
        s += v * v;
      }
    }
    double n2 = block_sum(s, sm.red);
    if (n2 == 0.0) { __syncthreads(); continue; }
    const double inv = 1.0 / sqrt(n2);
    for (int i = tid; i < rows; i += blockDim.x) Q[(long)i * a.ldq + cur] *= inv;
    __syncthreads();
    for (int pass = 0; pass < 2; ++pass) {
      for (int t = warp; t < cur; t += nwarps) {
        double d = 0.0;
        for (int i = lane; i < rows; i += 32) d += Q[(long)i * a.ldq + t] * Q[(long)i * a.ldq + cur];
        d = warp_sum(d);
        if (lane == 0) sm.wv[t] = d;
      }
      __syncthreads();
      for (int i = tid; i < rows; i += blockDim.x) {
        double v = Q[(long)i * a.ldq + cur];
        for (int t = 0; t < cur; ++t) v -= sm.wv[t] * Q[(long)i * a.ldq + t];
        Q[(long)i * a.ldq + cur] = v;
      }
      __syncthreads();
    }
    s = 0.0;
    for (int i = tid; i < rows; i += blockDim.x) {
      double v = Q[(long)i * a.ldq + cur];
      s += v * v;
    }
    double rn = sqrt(block_sum(s, sm.red));
    if (rn >= a.accept) {
      const double ir = 1.0 / rn;
      for (int i = tid; i < rows; i += blockDim.x) Q[(long)i * a.ldq + cur] *= ir;
      ++cur;
    }
    __syncthreads();
  }
  // zero the unused columns of the output block so later products may read them
  for (long idx = tid; idx < (long)rows * (a.ldq - cur); idx += blockDim.x) {
    int i = (int)(idx / (a.ldq - cur)), t = cur + (int)(idx % (a.ldq - cur));
    Q[(long)i * a.ldq + t] = 0.0;
  }
}

static const size_t kSmemLimit = 220 * 1024;

// Launch the fallback kernel: shared-memory staging when rows x mcap fits.
void launch_orth_fallback(const OrthArgs& a, int mcap, int maxrows, const int* flag,
                          const double* sm_small, int sB, int sR2i, cudaStream_t st) {
  const size_t base = orth_smem_base(mcap);
  // the staged copy holds the input's columns: at most r_aug_max for a QR, mcap otherwise
  const int wcols = a.mode == ORTH_QR ? min(mcap, a.r_aug_max) : mcap;
  const size_t need = base + sizeof(double) * ((size_t)maxrows * wcols + 8);
  pbeg(st, a.mode == ORTH_AUG ? KS_ORTH_AUG : KS_ORTH);
  if (need <= kSmemLimit)
    k_orth<true><<<a.g.nsub, DD_THREADS, need, st>>>(a, mcap, flag, sm_small, sB, sR2i);
  else
    k_orth<false><<<a.g.nsub, DD_THREADS, base, st>>>(a, mcap, flag, sm_small, sB, sR2i);
  pend(st);
}

void launch_cqr1(const OrthArgs& a, const double* sm, int sG, int sR, int sRi, double* smw,
                 int* flag, double* scale, cudaStream_t st) {
  pbeg(st, KS_CQR1);
  k_cqr1<<<a.g.nsub, 32, sizeof(double) * 2 * a.g.RC * a.g.RC, st>>>(a, sm, sG, sR, sRi, smw,
                                                                       flag, scale);
  pend(st);
}

void launch_cqr2(const OrthArgs& a, const double* sm, int sG2, int sR1, int sR1i, double* smw,
                 int sM, int* flag, const double* scale, cudaStream_t st) {
  pbeg(st, KS_CQR2);
  k_cqr2<<<a.g.nsub, DD_THREADS, cqr2_smem_bytes(a.g.RC), st>>>(a, sm, sG2, sR1, sR1i, smw, sM,
                                                                 flag, scale);
  pend(st);
}

cudaError_t orth_init() {
  cudaError_t e = cudaFuncSetAttribute(k_orth<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kSmemLimit);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_orth<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)orth_smem_base(DD_MAXC) + 64);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_cqr1, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(sizeof(double) * 2 * DD_MAXC * DD_MAXC));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_cqr2, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)cqr2_smem_bytes(DD_MAXC));
}

}  // namespace dd
