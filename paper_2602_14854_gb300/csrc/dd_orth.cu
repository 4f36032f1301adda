// Rank-revealing orthonormalisation with deterministic basis completion.
//
// Serves three steps of the scheme:
//   ORTH_QR       the QR decomposition of K (of L) in the K- and L-steps
//                 (Algorithms 1-3): an orthonormal basis of the numerically
//                 significant column span of K (L), completed to r_out columns;
//   ORTH_AUG      the SVD and rank choice of the augmentation (Algorithm 4):
//                 leading left singular vectors of
//                 L0 = [V S^T, V_L S_L^T, V_R S_R^T], r_t chosen by the tail rule,
//                 completed to r_t columns;
//   ORTH_COMPLETE pad an orthonormal basis to r_out columns (collision step started
//                 below the rank floor).
//
// A singular value sigma_j counts as significant when sigma_j > tau * sigma_1.
//
// Method (every pass over the rows runs on all SMs; only m x m work is per
// subdomain):
//   G1 = A^T A                      chunked Gram (k_gram; partials summed by k_geig)
//   G1 = V diag(lambda) V^T         k_geig: pivoted Cholesky G1 = X X^T, one-sided
//                                   Jacobi on X (FP32 sweeps, double-float finish),
//                                   one FP64 refinement; sigma_j = lambda_j^1/2 give
//                                   the rank decision; M = V_keep diag(sigma)^-1
//   U1 = A M                        k_tall: the leading left singular vectors, up to
//                                   errors of order eps |A|^2 / sigma_j^2
//   G2 = U1^T U1                    k_gram + k_chol_inv (G2^-1/2 by Newton-Schulz in
//                                   double-float)
//   Q  = U1 G2^-1/2                 k_tall: orthonormal to ~1e-14
//   completion                      k_kc_w / k_kca_w, k_kc_sel, k_kc_apply (QR and
//                                   augmentation: Gram-Schmidt in coefficient space),
//                                   then k_complete (what that leaves; the collision's
//                                   padding)
// The span of Q is that of the leading left singular vectors of A.  The
// eigenvector error eps |G1| / gap enters the result weighted by the discarded
// sigma_j, orders of magnitude below the FP64 parity bound (the CPU oracle takes
// the SVD of A itself).
//
// Completion: missing columns are taken in order from a fixed exactly-orthogonal
// candidate family, each Gram-Schmidt'd against the columns so far and accepted when
// its residual norm is >= accept:
//   space: cos(pi a (i+1/2)/nx_k) cos(pi b (j+1/2)/ny_k), by a+b then a descending;
//   angle: the table built at create time (P_2l(mu) x cos/sin(m phi), weighted by
//          sqrt(w)), then the unit vectors.
#include "dd_internal.cuh"
#include "dd_launch.h"

#include <climits>
#include <math_constants.h>

namespace dd {

// Rank decision (one thread).  sig[] descending; returns p, sets *keep and *r_out.
__device__ int decide(const OrthArgs& a, int k, const double* sig, int nref, int* keep,
                      int* r_out) {
  int p = 0;
  double s1 = nref > 0 ? sig[0] : 0.0;
  if (s1 > 0.0)
    for (int t = 0; t < nref; ++t)
      if (sig[t] > a.tau * s1) ++p;
  if (a.sig_out)
    for (int t = 0; t < DD_MAXC; ++t) a.sig_out[(long)k * DD_MAXC + t] = t < nref ? sig[t] : 0.0;
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
        for (int t = r; t < nref; ++t) ss += sig[t] * sig[t];
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

// On this GPU one FP64 warp instruction holds the SM's FP64 pipe for ~18 cycles
// whatever the number of active lanes, so the small FP64 algebra below keeps its FP64
// instructions few and full: scalar FP64 work is done by one lane and broadcast, loops
// map whole warps onto rows, and comparisons use the integer order of the bit
// patterns (positive doubles order as their bits).

// Pivoted Cholesky of the m x m (m <= 64) positive semidefinite A (column-major,
// leading dimension ld; overwritten by its Schur complements): A = X X^T up to a
// remainder whose diagonal is <= thr_rel times the largest diagonal entry of A.  X is
// m x k, written to the first k columns of X with the rows in the original order
// (column t is row t of the triangular factor in pivot order).  The pivot is the
// largest remaining positive finite diagonal entry (lowest index on ties); *piv gets
// the pivoted indices as a bit mask.  Block-wide; returns k.
__device__ int pchol_cols(double* A, double* X, int m, int ld, double thr_rel,
                          unsigned long long* piv) {
  __shared__ double pc[2];
  __shared__ int pi[1];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  unsigned long long done = 0ull;
  long long thr_bits = 0;                          // lane 0 of warp 0 only
  int k = 0;
  for (; k < m; ++k) {
    if (warp == 0) {
      long long best = 0;
      int bi = m;
      for (int i = lane; i < m; i += 32) {
        const long long b = __double_as_longlong(A[i * ld + i]);
        const bool ok = !((done >> i) & 1ull) && b > 0 && b < 0x7ff0000000000000ll;
        if (ok && b > best) { best = b; bi = i; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const long long ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (lane == 0) {
        if (k == 0) thr_bits = __double_as_longlong(thr_rel * __longlong_as_double(best));
        const bool go = bi < m && best > thr_bits;
        if (go) {
          const double dv = __longlong_as_double(best), id = rsqrt(dv);
          pc[0] = dv * id;
          pc[1] = id;
        }
        pi[0] = go ? bi : -1;
      }
    }
    __syncthreads();
    const int bi = pi[0];
    if (bi < 0) break;
    const double d = pc[0], id = pc[1];
    // column k of X (warp 0) and the Schur update (every warp) both read the pivot
    // column of A, which no thread writes in this step (bi is done)
    if (warp == 0)
      for (int i = lane; i < m; i += 32)
        X[k * ld + i] = ((done >> i) & 1ull) ? 0.0 : (i == bi ? d : A[bi * ld + i] * id);
    done |= 1ull << bi;
    for (int j = warp; j < m; j += nw) {
      if ((done >> j) & 1ull) continue;
      const double f = (A[bi * ld + j] * id) * id;   // one FMA per entry of the update
      for (int i = lane; i < m; i += 32)
        if (!((done >> i) & 1ull)) A[j * ld + i] = fma(-A[bi * ld + i], f, A[j * ld + i]);
    }
    __syncthreads();
  }
  *piv = done;
  return k;
}

// Completes the orthonormal columns 0..cur-1 of the m x m column-major V (leading
// dimension ld) to m columns with unit vectors, first those of the indices outside
// mask (in index order), then the others, each accepted when its squared norm after
// Gram-Schmidt exceeds 0.01 (at every stage some unit vector keeps at least 1/m).
// The candidates outside mask are taken as a block: the span of the first cur columns
// is removed from all of them at once (twice), then each is Gram-Schmidt'd against the
// block columns accepted before it; the rest, when needed, one by one against
// everything (twice).  coef: m doubles, W: 2 ld^2 doubles of shared scratch.
__device__ void complete_unit(double* V, int m, int cur, int ld, unsigned long long mask,
                              double* coef, double* W, unsigned* status) {
  __shared__ double cred[40];
  __shared__ int cidx[64];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  if (cur >= m) return;
  // indices outside mask, ascending
  const unsigned long long out = ~mask & (m >= 64 ? ~0ull : ((1ull << m) - 1ull));
  const int q = __popcll(out);
  for (int t = tid; t < m; t += blockDim.x)
    if ((out >> t) & 1ull) cidx[__popcll(out & ((1ull << t) - 1ull))] = t;
  __syncthreads();
  const int c0 = cur;
  double* C = W + (long)ld * ld;
  for (int e = tid; e < m * q; e += blockDim.x) {          // W = E - V V^T E
    const int r = e % m, t = e / m, i = cidx[t];
    double s = r == i ? 1.0 : 0.0;
    for (int l = 0; l < c0; ++l) s -= V[l * ld + i] * V[l * ld + r];
    W[t * ld + r] = s;
  }
  __syncthreads();
  for (int e = tid; e < c0 * q; e += blockDim.x) {         // C = V^T W
    const int l = e % c0, t = e / c0;
    double s = 0.0;
    for (int r = 0; r < m; ++r) s += V[l * ld + r] * W[t * ld + r];
    C[t * ld + l] = s;
  }
  __syncthreads();
  for (int e = tid; e < m * q; e += blockDim.x) {          // W -= V C
    const int r = e % m, t = e / m;
    double s = W[t * ld + r];
    for (int l = 0; l < c0; ++l) s -= C[t * ld + l] * V[l * ld + r];
    W[t * ld + r] = s;
  }
  __syncthreads();
  for (int t = 0; t < q && cur < m; ++t) {
    const int na = cur - c0;
    for (int l = warp; l < na; l += nw) {
      double s = 0.0;
      for (int r = lane; r < m; r += 32) s += V[(c0 + l) * ld + r] * W[t * ld + r];
      s = warp_sum(s);
      if (lane == 0) coef[l] = s;
    }
    __syncthreads();
    double* x = V + (long)cur * ld;
    double n2 = 0.0;
    for (int r = tid; r < m; r += blockDim.x) {
      double s = W[t * ld + r];
      for (int l = 0; l < na; ++l) s -= coef[l] * V[(c0 + l) * ld + r];
      x[r] = s;
      n2 += s * s;
    }
    n2 = block_sum(n2, cred);
    if (n2 > 0.01) {
      for (int r = tid; r < m; r += blockDim.x) x[r] *= rsqrt(n2);
      ++cur;
    }
    __syncthreads();
  }
  for (int cand = 0; cand < 2 * m && cur < m; ++cand) {    // not expected: one by one
    const int i = cand < m ? cand : cand - m;
    const bool inmask = (mask >> i) & 1ull;
    if ((cand < m) == inmask) continue;
    double* x = V + (long)cur * ld;
    for (int r = tid; r < m; r += blockDim.x) {
      double s = r == i ? 1.0 : 0.0;
      for (int l = 0; l < cur; ++l) s -= V[l * ld + i] * V[l * ld + r];
      x[r] = s;
    }
    __syncthreads();
    for (int l = warp; l < cur; l += nw) {
      double s = 0.0;
      for (int r = lane; r < m; r += 32) s += V[l * ld + r] * x[r];
      s = warp_sum(s);
      if (lane == 0) coef[l] = s;
    }
    __syncthreads();
    double n2 = 0.0;
    for (int r = tid; r < m; r += blockDim.x) {
      double s = x[r];
      for (int l = 0; l < cur; ++l) s -= coef[l] * V[l * ld + r];
      x[r] = s;
      n2 += s * s;
    }
    n2 = block_sum(n2, cred);
    if (n2 > 0.01) {
      for (int r = tid; r < m; r += blockDim.x) x[r] *= rsqrt(n2);
      ++cur;
    }
    __syncthreads();
  }
  if (cur < m && threadIdx.x == 0) atomicOr(status, (unsigned)ST_COMPLETION);
}

size_t geig_smem_bytes(int RC) {
  return sizeof(double) * (3 * RC * RC + 2 * RC) + 8 * ((jacobi_mixed_scratch_bytes(RC) + 7) / 8) +
         sizeof(int) * (RC + 16);
}

// Eigendecomposition of G1 (m x m): one-sided Jacobi (FP32 sweeps, double-float
// finish; the columns of G1 V are orthogonal with norms lambda_j, G1 being positive
// semidefinite), then one FP64 refinement step of the eigenvectors (Ogita and
// Aishima, 2018): with R = I - V^T V, S = V^T G1 V, lambda_i = s_ii / (1 - r_ii),
// V <- V (I + E), e_ij = (s_ij + lambda_j r_ij) / (lambda_j - lambda_i) for
// separated pairs, r_ij / 2 within clusters and on the diagonal.  The double-float
// solution is accurate to ~1e-14 |G1|; the step brings it to the FP64 level, which the
// parity with an FP64 SVD needs for eigenvectors whose eigenvalues sit near the rank
// threshold (tau^2 lambda_1).  Writes M = V_keep diag(sigma_keep)^-1 (row-major,
// slot sM), keep (per subdomain) and, for the augmentation, r_t.
__global__ void __launch_bounds__(DD_THREADS, 1) k_geig(OrthArgs a, const double* part,
                                                     const int* cexp, int nchunk, double* sm,
                                                     int sM, int* keep_out) {
  extern __shared__ double shg[];
  const int k = blockIdx.x, RC = a.g.RC;
  const int m = a.acols[k];
  const double* G = part + (long)k * nchunk * RC * RC;      // nchunk partial Grams
  double* M = sm + ((long)k * NSMALL + sM) * RC * RC;
  double* Bc = shg;                 // column-major working copy
  double* Jc = Bc + RC * RC;        // accumulated rotations
  double* Gs = Jc + RC * RC;        // G1 (scaled), kept for the refinement
  double* lam = Gs + RC * RC;       // eigenvalues
  double* sig = lam + RC;           // singular values of A, descending
  double* X = sig + RC;             // scratch of the SVD
  int* perm = reinterpret_cast<int*>(X + (jacobi_mixed_scratch_bytes(RC) + 7) / 8);
  int* iv = perm + RC;
  const int tid = threadIdx.x;
  // the chunk partials are Grams of 2^-e_c A: G1 of 2^-emax A is their sum with
  // weights 4^(e_c - emax)
  __shared__ double fac[64];
  int emax = INT_MIN;
  for (int c = 0; c < nchunk; ++c) emax = max(emax, cexp[(long)k * nchunk + c]);
  for (int c = tid; c < nchunk; c += blockDim.x) {
    const int ec = cexp[(long)k * nchunk + c];
    fac[c] = ec == INT_MIN ? 0.0 : ldexp(1.0, 2 * max(ec - emax, -600));
  }
  __syncthreads();
  bool fin = true;
  for (int e = tid; e < RC * RC; e += blockDim.x) {
    const int col = e / RC, row = e % RC;
    double x = 0.0;
    if (col < m && row < m && emax != INT_MIN)
      for (int c = 0; c < nchunk; ++c) x += G[(long)c * RC * RC + row * RC + col] * fac[c];
    if (!isfinite(x)) { fin = false; x = 0.0; }
    Bc[e] = x;
    Gs[e] = x;
    Jc[e] = (row == col) ? 1.0 : 0.0;
  }
  if (emax == INT_MIN) emax = 0;
  if (!fin) atomicOr(a.status, (unsigned)ST_NONFINITE);
  __syncthreads();
  // G1 = X X^T by pivoted Cholesky (X in Jc, its k columns ordered by decreasing pivot);
  // one-sided Jacobi on X then gives X J = W with orthogonal columns, G1 = W W^T: the
  // normalised columns of W are eigenvectors of G1 (eigenvalues |w_j|^2), completed
  // by unit vectors for the null space below the Cholesky threshold (1e-13 of the
  // largest diagonal entry, far below the rank threshold tau^2).  Jacobi on the
  // triangular factor needs a fraction of the sweeps Jacobi on G1 does (the graded
  // columns are nearly orthogonal from the start).  (The Jacobi of G1 itself remains
  // only for a rank beyond the 64-column capacity, which does not occur.)
  unsigned long long pmask = 0ull;
  const int kr = pchol_cols(Bc, Jc, m, RC, 1e-13, &pmask);
  if (kr <= 64) {
    orth_cols_mixed(Jc, m, kr, RC, X);
    complete_unit(Jc, m, kr, RC, pmask, lam, X, a.status);
  } else {
    for (int e = tid; e < RC * RC; e += blockDim.x) {
      const int col = e / RC, row = e % RC;
      Bc[e] = Gs[e];
      Jc[e] = (row == col) ? 1.0 : 0.0;
    }
    __syncthreads();
    jacobi_svd_mixed(Bc, Jc, m, RC, &iv[0], lam, X);
  }
  // FP64 refinement of the eigenvectors (V is Jc: V_ij = Jc[j * RC + i])
  refine_sym_eig(Gs, Jc, lam, m, RC, X);
  for (int j = tid; j < m; j += blockDim.x) {
    const double l = lam[j];
    if (!isfinite(l)) atomicOr(a.status, (unsigned)ST_NONFINITE);
    lam[j] = l > 0.0 ? l : 0.0;       // G1 is positive semidefinite
  }
  __syncthreads();
  rank_sort_desc_nonneg(lam, m, perm);
  __syncthreads();
  for (int t = tid; t < m; t += blockDim.x) sig[t] = sqrt(lam[perm[t]]);   // of 2^-emax A
  __syncthreads();
  for (int t = tid; t < m; t += blockDim.x) lam[t] = ldexp(sig[t], emax);  // of A
  __syncthreads();
  if (tid == 0) {
    int keep = 0, r_out = 0;
    decide(a, k, lam, m, &keep, &r_out);
    if (a.mode == ORTH_AUG) a.rt_out[k] = r_out;
    keep_out[k] = keep;
    iv[1] = keep;
  }
  __syncthreads();
  const int keep = iv[1];
  // M = V_keep diag(sigma)^-1 for A itself: 2^-emax / sigma_scaled
  for (int t = tid; t < keep; t += blockDim.x) lam[t] = ldexp(1.0 / sig[t], -emax);
  __syncthreads();
  for (int e = tid; e < RC * RC; e += blockDim.x) {
    const int i = e / RC, t = e % RC;
    M[e] = (i < m && t < keep) ? Jc[perm[t] * RC + i] * lam[t] : 0.0;
  }
}

size_t chol_smem_bytes(int RC) { return sizeof(float2) * 5 * RC * RC; }

// Z = G2^-1/2 (q x q, q = keep) into slot sRi, so that Q = U1 Z is orthonormal.  G2,
// summed here from its nchunk partial Grams, is the Gram of U1 = A V diag(sigma)^-1,
// the identity up to E = G2 - I (|E| <~ 1e-3, set by the eigensolver's accuracy
// relative to the smallest kept sigma^2).  Coupled Newton-Schulz iteration in
// double-float (Y <- Y T, Z <- T Z, T = (3I - Z Y)/2; Y -> G2^1/2, Z -> G2^-1/2, the
// error e maps to ~3/4 e^2), iterated until the predicted error is below 1e-16: a few
// parallel matrix products instead of a sequential factorisation.  |E|_F >= 0.9 (not
// expected; only through non-finite or inconsistent data) is reported and leaves the
// identity.
__global__ void __launch_bounds__(DD_THREADS) k_chol_inv(OrthArgs a, const double* part,
                                                         int nchunk, double* sm, int sRi,
                                                         const int* keep) {
  extern __shared__ float2 shc[];
  const int k = blockIdx.x, RC = a.g.RC, tid = threadIdx.x;
  const int q = keep[k];
  const double* G = part + (long)k * nchunk * RC * RC;
  double* Ri = sm + ((long)k * NSMALL + sRi) * RC * RC;
  float2* Y = shc;
  float2* Z = Y + RC * RC;
  float2* T = Z + RC * RC;
  float2* W1 = T + RC * RC;
  float2* W2 = W1 + RC * RC;
  __shared__ double red[40];
  double e2 = 0.0;
  for (int e = tid; e < q * q; e += blockDim.x) {
    const int i = e / q, j = e % q;
    double x = 0.0;
    for (int c = 0; c < nchunk; ++c) x += G[(long)c * RC * RC + i * RC + j];
    const double d = x - (i == j ? 1.0 : 0.0);
    e2 += d * d;
    Y[i * RC + j] = df_from_double(x);
    Z[i * RC + j] = make_float2(i == j ? 1.f : 0.f, 0.f);
  }
  const double err = sqrt(block_sum(e2, red));
  const bool ok = isfinite(err) && err < 0.9;
  int iters = 0;
  for (double e = err; e > 1e-16 && iters < 12; e = 0.75 * e * e) ++iters;
  // Y, Z and T are polynomials in G2: symmetric and commuting, so every product is
  // symmetric; only its upper triangle is computed (pairs enumerated densely) and mirrored.
  const int ntri = q * (q + 1) / 2;
  if (ok) {
    for (int it = 0; it < iters; ++it) {
      for (int p = tid; p < ntri; p += blockDim.x) {            // T = (3I - Z Y) / 2
        int j = (int)((sqrtf(8.f * p + 1.f) - 1.f) * 0.5f);
        j += (j + 1) * (j + 2) / 2 <= p;
        j -= j * (j + 1) / 2 > p;
        const int i = p - j * (j + 1) / 2;
        float2 x = make_float2(0.f, 0.f);
        for (int l = 0; l < q; ++l) x = df_add(x, df_mul(Z[i * RC + l], Y[l * RC + j]));
        const float2 t = df_mulf(df_add(make_float2(i == j ? 3.f : 0.f, 0.f), df_neg(x)), 0.5f);
        T[i * RC + j] = t;
        T[j * RC + i] = t;
      }
      __syncthreads();
      for (int p = tid; p < ntri; p += blockDim.x) {            // W1 = Y T, W2 = T Z
        int j = (int)((sqrtf(8.f * p + 1.f) - 1.f) * 0.5f);
        j += (j + 1) * (j + 2) / 2 <= p;
        j -= j * (j + 1) / 2 > p;
        const int i = p - j * (j + 1) / 2;
        float2 x = make_float2(0.f, 0.f), y = make_float2(0.f, 0.f);
        for (int l = 0; l < q; ++l) {
          x = df_add(x, df_mul(Y[i * RC + l], T[l * RC + j]));
          y = df_add(y, df_mul(T[i * RC + l], Z[l * RC + j]));
        }
        W1[i * RC + j] = x; W1[j * RC + i] = x;
        W2[i * RC + j] = y; W2[j * RC + i] = y;
      }
      __syncthreads();
      float2* tmp = Y; Y = W1; W1 = tmp;
      tmp = Z; Z = W2; W2 = tmp;
    }
  }
  if (!ok && tid == 0 && q > 0) atomicOr(a.status, (unsigned)ST_NONFINITE);
  for (int e = tid; e < RC * RC; e += blockDim.x) {
    const int i = e / RC, c = e % RC;
    double v = 0.0;
    if (i < q && c < q) v = ok ? df_to_double(Z[i * RC + c]) : (i == c ? 1.0 : 0.0);
    Ri[e] = v;
  }
}

// Completion to r_out columns (one CTA per subdomain; idle where keep >= r_out).
// ORTH_COMPLETE first copies the input's columns.  Columns from the last accepted
// one up to ldq are zero on return.
#define KC_TAB 512
__global__ void __launch_bounds__(DD_THREADS) k_complete(OrthArgs a, const int* keep_in) {
  __shared__ double cxy[2 * KC_TAB];   // the two cosine vectors of a spatial candidate
  __shared__ double red[40];
  __shared__ double wv[DD_MAXC];
  __shared__ int iv[12];
  const int k = blockIdx.x;
  const Geo& g = a.g;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  const int rows = a.spatial ? g.N[k] : g.n;
  const long rbase = a.spatial ? (long)g.rowoff[k] : (long)k * g.n;
  double* Q = a.Q + rbase * a.ldq;
  int cur, r_out;
  if (a.mode == ORTH_COMPLETE) {
    const double* A = a.A + rbase * a.lda;
    cur = a.acols[k];
    r_out = a.rout[k];
    for (long idx = tid; idx < (long)rows * a.ldq; idx += blockDim.x) {
      const int i = (int)(idx / a.ldq), t = (int)(idx % a.ldq);
      Q[(long)i * a.ldq + t] = t < cur ? A[(long)i * a.lda + t] : 0.0;
    }
    __syncthreads();
  } else {
    cur = keep_in[k];
    r_out = a.mode == ORTH_AUG ? a.rt_out[k] : a.rout[k];
  }
  if (cur >= r_out) return;
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
      // the candidate is a product of two cosine vectors: evaluate each once (the same
      // expressions as per cell, so the candidate is bitwise the same)
      const int ca = iv[6], cb = iv[7];
      const bool tab = nxk + nyk <= 2 * KC_TAB;
      if (tab) {
        for (int i = tid; i < nxk + nyk; i += blockDim.x)
          cxy[i] = i < nxk ? cos(CUDART_PI * ca * (i + 0.5) / nxk)
                           : cos(CUDART_PI * cb * (i - nxk + 0.5) / nyk);
        __syncthreads();
      }
      for (int i = tid; i < rows; i += blockDim.x) {
        int il = i % nxk, jl = i / nxk;
        double v = tab ? cxy[il] * cxy[nxk + jl]
                       : cos(CUDART_PI * ca * (il + 0.5) / nxk) * cos(CUDART_PI * cb * (jl + 0.5) / nyk);
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
    // scalar FP64 work (square roots, reciprocals) by one lane, broadcast through red[34]
    double n2 = block_sum(s, red);
    if (n2 == 0.0) { __syncthreads(); continue; }
    if (tid == 0) red[34] = rsqrt(n2);
    __syncthreads();
    const double inv = red[34];
    for (int i = tid; i < rows; i += blockDim.x) Q[(long)i * a.ldq + cur] *= inv;
    __syncthreads();
    // Gram-Schmidt against the accepted columns, a second pass only when the first one
    // cancelled more than half of the squared norm (with at least 1/sqrt(2) of the unit
    // candidate left, one pass already leaves it orthogonal to ~sqrt(2) eps: "twice is
    // enough"); the squared norm after the last pass decides acceptance
    double rn2 = 0.0;
    for (int pass = 0; pass < 2; ++pass) {
      for (int t = warp; t < cur; t += nwarps) {
        double d = 0.0;
        for (int i = lane; i < rows; i += 32) d += Q[(long)i * a.ldq + t] * Q[(long)i * a.ldq + cur];
        d = warp_sum(d);
        if (lane == 0) wv[t] = d;
      }
      __syncthreads();
      s = 0.0;
      for (int i = tid; i < rows; i += blockDim.x) {
        double v = Q[(long)i * a.ldq + cur];
        for (int t = 0; t < cur; ++t) v -= wv[t] * Q[(long)i * a.ldq + t];
        Q[(long)i * a.ldq + cur] = v;
        s += v * v;
      }
      rn2 = block_sum(s, red);
      if (rn2 >= 0.5) break;
    }
    if (rn2 >= a.accept * a.accept) {
      if (tid == 0) red[34] = rsqrt(rn2);
      __syncthreads();
      const double ir = red[34];
      for (int i = tid; i < rows; i += blockDim.x) Q[(long)i * a.ldq + cur] *= ir;
      ++cur;
    }
    __syncthreads();
  }
  // a rejected last candidate leaves a non-zero column at cur
  for (long idx = tid; idx < (long)rows * (a.ldq - cur); idx += blockDim.x) {
    int i = (int)(idx / (a.ldq - cur)), t = cur + (int)(idx % (a.ldq - cur));
    Q[(long)i * a.ldq + t] = 0.0;
  }
}

void launch_geig(const OrthArgs& a, const double* part, const int* cexp, int nchunk, double* sm,
                 int sM, int* keep, cudaStream_t st) {
  pbeg(st, a.mode == ORTH_AUG ? KS_GEIG_AUG : KS_GEIG);
  k_geig<<<a.g.nsub, DD_THREADS, geig_smem_bytes(a.g.RC), st>>>(a, part, cexp, nchunk, sm, sM, keep);
  pend(st);
}

void launch_chol_inv(const OrthArgs& a, const double* part, int nchunk, double* sm, int sRi,
                     const int* keep, cudaStream_t st) {
  pbeg(st, KS_CHOL);
  k_chol_inv<<<a.g.nsub, DD_THREADS, chol_smem_bytes(a.g.RC), st>>>(a, part, nchunk, sm, sRi, keep);
  pend(st);
}

// ---------------------------------------------------------------------------------------
// Spatial completion in coefficient space.  The cosine candidates c_j are mutually
// orthogonal, so Gram-Schmidt of c_j against the first cur0 columns Q0 and the columns
// q_k = C a_k + Q0 b_k accepted before it needs only w_j = Q0^T c_j / |c_j|:
//   q_k^T c_j / |c_j| = b_k^T w_j =: g_k,   |residual|^2 = 1 - |w_j|^2 - |g|^2,
//   accepted (|residual| >= accept):  a = (e_j / |c_j| - sum g_k a_k) / |residual|,
//                                     b = (-w_j - sum g_k b_k) / |residual|.
// The same candidates in the same order with the same acceptance rule as the one-by-one
// completion (and R11's definition), equal to it up to rounding; the passes over the
// rows (W and the new columns) run on all SMs instead of one CTA per subdomain.
// ---------------------------------------------------------------------------------------
#define KC_TR 128    // rows per tile of k_kca_w
#define KC_TR3 32    // rows per CTA of k_kc_apply
#define KCA_JC 4     // candidates per CTA of k_kca_w
#define KC_JB 32     // grid rows per block of k_kc_w
static_assert(DD_THREADS >= 160, "k_kc_w gives each of up to kc_bmax(DD_MAXC) candidates a thread");

// Subdomain k's completion: columns done (cur0), target (r_out), rows, and the number of
// candidates examined at once (0: nothing to add).  Angle: the leading table candidates
// that are mutually orthogonal (all of them under a product quadrature); the rest and the
// unit vectors after them are left to the one-by-one completion.
__device__ __forceinline__ int kc_plan(const OrthArgs& a, const int* keep, int k, int* cur0,
                                       int* r_out, int* rows) {
  const int RC = a.g.RC;
  *cur0 = keep[k];
  *r_out = a.mode == ORTH_AUG ? a.rt_out[k] : a.rout[k];
  if (a.spatial) {
    *rows = a.g.N[k];
    return kc_b(a.g.nxk[k], a.g.nyk[k], *cur0, *r_out, RC);
  }
  *rows = a.g.n;
  const int need = *r_out - *cur0;
  if (need <= 0) return 0;
  int b = need + (4 * *cur0 + 2) / 3 + 1;
  b = min(b, a.n_angorth);
  return min(b, kc_bmax(RC));
}

size_t kca_w_smem(int RC) { return sizeof(double) * KC_TR * ((RC | 1) + KCA_JC); }
size_t kc_w_smem(int RC) { return sizeof(double) * KC_JB * kc_bmax(RC); }   // nfa <= b <= bmax
size_t kc_sel_smem(int RC) { return sizeof(double) * ((size_t)(kc_bmax(RC) + RC) * RC + 2 * RC); }
size_t kc_apply_smem(int RC) { return sizeof(double) * KC_TR3 * ((kc_bmax(RC) | 1) + (RC | 1)); }

// W = Q0^T C and the candidates' squared norms.  A candidate is the product of an
// x-cosine cx_a and a y-cosine cy_b, so W[l][j] = sum_jl cy_b(jl) sum_il Q0[jl nx + il][l]
// cx_a(il): one CTA per (column l, subdomain) contracts x first for the nfa frequencies
// in use (N nfa FMAs instead of N b) in blocks of KC_JB grid rows, then y per candidate;
// CTA l = RC writes |c_j|^2 = |cx_a|^2 |cy_b|^2.
__global__ void __launch_bounds__(DD_THREADS) k_kc_w(OrthArgs a, const double* tab,
                                                     const long long* off, const int* nf,
                                                     const int* keep, double* part) {
  extern __shared__ double kq[];
  __shared__ int cab[2 * 160];
  const int k = blockIdx.y, l = blockIdx.x, RC = a.g.RC, bm = kc_bmax(RC), tid = threadIdx.x;
  const int cur0 = keep[k], nxk = a.g.nxk[k], nyk = a.g.nyk[k];
  const int b = kc_b(nxk, nyk, cur0, a.rout[k], RC);
  if (b <= 0 || (l >= cur0 && l != RC)) return;
  // candidate frequencies (all inside the tables, else k_kc_sel leaves it all to the
  // sequential completion and nothing here is read)
  __shared__ int nfa_s, okc;
  if (tid == 0) { nfa_s = 0; okc = 1; }
  __syncthreads();
  for (int j = tid; j < b; j += blockDim.x) {
    int ca = 0, cb = 0;
    const bool ok = kc_cand(j, nxk, nyk, &ca, &cb) && ca < nf[2 * k] && cb < nf[2 * k + 1];
    if (!ok) okc = 0;
    cab[2 * j] = ok ? ca : 0;
    cab[2 * j + 1] = ok ? cb : 0;
    atomicMax(&nfa_s, ca + 1);
  }
  __syncthreads();
  if (!okc) return;
  const int nfa = nfa_s;
  const double* tx = tab + off[k];
  const double* ty = tx + (size_t)nf[2 * k] * nxk;
  double* W = part + (size_t)k * kc_region(RC) + (size_t)(bm + RC) * RC;
  if (l == RC) {
    for (int j = tid; j < b; j += blockDim.x) {
      const double* cx = tx + (size_t)cab[2 * j] * nxk;
      const double* cy = ty + (size_t)cab[2 * j + 1] * nyk;
      double sx = 0.0, sy = 0.0;
      for (int i = 0; i < nxk; ++i) sx += cx[i] * cx[i];
      for (int i = 0; i < nyk; ++i) sy += cy[i] * cy[i];
      W[(size_t)RC * bm + j] = sx * sy;
    }
    return;
  }
  const double* Q = a.Q + (size_t)a.g.rowoff[k] * a.ldq + l;
  double* T = kq;                                  // KC_JB x nfa
  double acc = 0.0;                                // thread j < b: W[l][j]
  for (int j0 = 0; j0 < nyk; j0 += KC_JB) {
    const int nj = min(KC_JB, nyk - j0);
    for (int e = tid; e < nj * nfa; e += blockDim.x) {
      const int jl = e / nfa, fa = e - jl * nfa;
      const double* row = Q + (size_t)(j0 + jl) * nxk * a.ldq;
      const double* cx = tx + (size_t)fa * nxk;
      double x = 0.0;
      for (int i = 0; i < nxk; ++i) x += row[(size_t)i * a.ldq] * cx[i];
      T[jl * nfa + fa] = x;
    }
    __syncthreads();
    if (tid < b) {
      const int ca = cab[2 * tid];
      const double* cy = ty + (size_t)cab[2 * tid + 1] * nyk + j0;
      for (int jl = 0; jl < nj; ++jl) acc += T[jl * nfa + ca] * cy[jl];
    }
    __syncthreads();
  }
  if (tid < b) W[(size_t)l * bm + tid] = acc;
}

// W for the angular table candidates: one CTA per (KCA_JC candidates, subdomain), 128-row
// tiles of Q0 staged in shared memory once for all of them (odd pitch), lane = row, warp w
// accumulating columns w + 8 q; warp 0 also sums |c_j|^2.  Every W[l][j] is summed over
// the same rows in the same order as with one candidate per CTA.
__global__ void __launch_bounds__(DD_THREADS) k_kca_w(OrthArgs a, const int* keep, double* part) {
  extern __shared__ double kq[];
  const int k = blockIdx.y, j0 = blockIdx.x * KCA_JC, RC = a.g.RC, bm = kc_bmax(RC);
  int cur0 = 0, r_out = 0, rows = 0;
  const int b = kc_plan(a, keep, k, &cur0, &r_out, &rows);
  if (j0 >= b) return;
  const int jn = min(KCA_JC, b - j0);
  const double* Q = a.Q + (size_t)k * a.g.n * a.ldq;
  const int pitch = cur0 | 1;
  double* cv = kq + KC_TR * pitch;                 // KCA_JC x KC_TR
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  double acc[8][KCA_JC], nn[KCA_JC];
#pragma unroll
  for (int jj = 0; jj < KCA_JC; ++jj) {
    nn[jj] = 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q][jj] = 0.0;
  }
  for (int r0 = 0; r0 < rows; r0 += KC_TR) {
    const int nr = min(KC_TR, rows - r0);
    for (int r = warp; r < nr; r += DD_THREADS / 32)
      for (int l = lane; l < cur0; l += 32) kq[r * pitch + l] = Q[(size_t)(r0 + r) * a.ldq + l];
    for (int e = tid; e < KCA_JC * KC_TR; e += DD_THREADS) {
      const int jj = e / KC_TR, r = e - jj * KC_TR;
      cv[e] = (jj < jn && r < nr) ? a.angcand[(size_t)(j0 + jj) * a.g.n + r0 + r] : 0.0;
    }
    __syncthreads();
    for (int r = lane; r < nr; r += 32) {
      double x[KCA_JC];
#pragma unroll
      for (int jj = 0; jj < KCA_JC; ++jj) x[jj] = cv[jj * KC_TR + r];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int l = warp + 8 * q;
        if (l < cur0) {
          const double qv = kq[r * pitch + l];
#pragma unroll
          for (int jj = 0; jj < KCA_JC; ++jj) acc[q][jj] += qv * x[jj];
        }
      }
      if (warp == 0)
#pragma unroll
        for (int jj = 0; jj < KCA_JC; ++jj) nn[jj] += x[jj] * x[jj];
    }
    __syncthreads();
  }
  double* W = part + (size_t)k * kc_region(RC) + (size_t)(bm + RC) * RC;
#pragma unroll
  for (int q = 0; q < 8; ++q)
#pragma unroll
    for (int jj = 0; jj < KCA_JC; ++jj) {
      const double x = warp_sum(acc[q][jj]);
      const int l = warp + 8 * q;
      if (lane == 0 && l < cur0 && jj < jn) W[(size_t)l * bm + j0 + jj] = x;
    }
#pragma unroll
  for (int jj = 0; jj < KCA_JC; ++jj) {
    const double x = warp_sum(nn[jj]);
    if (tid == 0 && jj < jn) W[(size_t)RC * bm + j0 + jj] = x;
  }
}

// The selection in coefficient space (one CTA per subdomain): kcn = accepted count,
// kcur = cur0 + kcn (cur0 when the tables do not cover the candidates: the sequential
// completion then does all of it); the coefficients a_t (rows of A, b x kcn) and b_t
// (rows of B, cur0 x kcn) go to the subdomain's scratch.
__global__ void __launch_bounds__(DD_THREADS) k_kc_sel(OrthArgs a, const int* nf, const int* keep,
                                                       double* part, int* kcn, int* kcur) {
  extern __shared__ double ks[];
  __shared__ int okf;
  __shared__ double sc[2];
  const int k = blockIdx.x, RC = a.g.RC, bm = kc_bmax(RC), tid = threadIdx.x;
  int cur0 = 0, r_out = 0, rows = 0;
  const int b = kc_plan(a, keep, k, &cur0, &r_out, &rows);
  if (tid == 0) {
    int ok = b > 0;
    if (a.spatial) {
      const int nxk = a.g.nxk[k], nyk = a.g.nyk[k];
      for (int j = 0; j < b && ok; ++j) {
        int ca = 0, cb = 0;
        ok = kc_cand(j, nxk, nyk, &ca, &cb) && ca < nf[2 * k] && cb < nf[2 * k + 1];
      }
    }
    okf = ok;
  }
  __syncthreads();
  if (!okf) {
    if (tid == 0) { kcn[k] = 0; kcur[k] = cur0; }
    return;
  }
  double* R = part + (size_t)k * kc_region(RC);
  double* Ac = R;                                   // bm x RC
  double* Bc = R + (size_t)bm * RC;                 // RC x RC
  const double* W = R + (size_t)(bm + RC) * RC;     // (RC + 1) x bm
  double* As = ks;                                  // b x RC
  double* Bs = As + (size_t)bm * RC;                // cur0 x RC
  double* wt = Bs + (size_t)RC * RC;                // cur0
  double* g = wt + RC;                              // accepted count
  const int need = r_out - cur0;
  int nacc = 0;
  for (int j = 0; j < b && nacc < need; ++j) {
    // scalar FP64 work on one lane, broadcast through sc
    if (tid == 0) {
      const double n2 = W[(size_t)RC * bm + j];
      sc[0] = n2 > 0.0 ? rsqrt(n2) : 0.0;
    }
    __syncthreads();
    const double inv = sc[0];
    if (inv != 0.0) {
      for (int l = tid; l < cur0; l += blockDim.x) wt[l] = W[(size_t)l * bm + j] * inv;
      __syncthreads();
      for (int t = tid; t < nacc; t += blockDim.x) {
        double x = 0.0;
        for (int l = 0; l < cur0; ++l) x += Bs[l * RC + t] * wt[l];
        g[t] = x;
      }
      __syncthreads();
      if (tid < 32) {
        double x = 0.0;
        for (int i = tid; i < cur0; i += 32) x += wt[i] * wt[i];
        for (int i = tid; i < nacc; i += 32) x += g[i] * g[i];
        x = warp_sum(x);
        if (tid == 0) {
          const double rn2 = 1.0 - x;
          sc[1] = rn2 >= a.accept * a.accept ? rsqrt(rn2) : 0.0;
        }
      }
      __syncthreads();
      const double ir = sc[1];
      if (ir != 0.0) {
        for (int i = tid; i < b + cur0; i += blockDim.x) {
          if (i < b) {
            double x = i == j ? inv : 0.0;
            for (int t = 0; t < nacc; ++t) x -= g[t] * As[i * RC + t];
            As[i * RC + nacc] = x * ir;
          } else {
            const int l = i - b;
            double x = -wt[l];
            for (int t = 0; t < nacc; ++t) x -= g[t] * Bs[l * RC + t];
            Bs[l * RC + nacc] = x * ir;
          }
        }
        ++nacc;
      }
    }
    __syncthreads();
  }
  for (int e = tid; e < b * nacc; e += blockDim.x) {
    const int i = e / nacc, t = e - i * nacc;
    Ac[i * RC + t] = As[i * RC + t];
  }
  for (int e = tid; e < cur0 * nacc; e += blockDim.x) {
    const int l = e / nacc, t = e - l * nacc;
    Bc[l * RC + t] = Bs[l * RC + t];
  }
  if (tid == 0) { kcn[k] = nacc; kcur[k] = cur0 + nacc; }
}

// The accepted columns Q[:, cur0 + t] = C a_t + Q0 b_t, 32 rows per CTA (candidate
// values and Q0 rows staged in shared memory).
__global__ void __launch_bounds__(DD_THREADS) k_kc_apply(OrthArgs a, const double* tab,
                                                         const long long* off, const int* nf,
                                                         const int* keep, const int* kcn,
                                                         const double* part) {
  extern __shared__ double kt[];
  __shared__ int cab[2 * 160];
  const int k = blockIdx.y, RC = a.g.RC, bm = kc_bmax(RC), tid = threadIdx.x;
  const int nacc = kcn[k];
  if (nacc <= 0) return;
  int cur0 = 0, r_out = 0, rows = 0;
  const int b = kc_plan(a, keep, k, &cur0, &r_out, &rows);
  const int r0 = blockIdx.x * KC_TR3;
  if (r0 >= rows) return;
  const int nxk = a.spatial ? a.g.nxk[k] : 1, nyk = a.spatial ? a.g.nyk[k] : 1;
  const int nr = min(KC_TR3, rows - r0);
  const int cp = b | 1, qp = cur0 | 1;
  double* Ct = kt;                                  // KC_TR3 x cp
  double* Qt = Ct + KC_TR3 * (bm | 1);              // KC_TR3 x qp
  double* Q = a.Q + (a.spatial ? (size_t)a.g.rowoff[k] : (size_t)k * a.g.n) * a.ldq;
  if (a.spatial)
    for (int j = tid; j < b; j += blockDim.x) {
      int ca = 0, cb = 0;
      kc_cand(j, nxk, nyk, &ca, &cb);
      cab[2 * j] = ca;
      cab[2 * j + 1] = cb;
    }
  for (int e = tid; e < nr * cur0; e += blockDim.x) {
    const int r = e / cur0, l = e - r * cur0;
    Qt[r * qp + l] = Q[(size_t)(r0 + r) * a.ldq + l];
  }
  __syncthreads();
  if (a.spatial) {
    const double* tx = tab + off[k];
    const double* ty = tx + (size_t)nf[2 * k] * nxk;
    for (int e = tid; e < nr * b; e += blockDim.x) {
      const int r = e / b, j = e - r * b, i = r0 + r;
      Ct[r * cp + j] = tx[(size_t)cab[2 * j] * nxk + i % nxk] * ty[(size_t)cab[2 * j + 1] * nyk + i / nxk];
    }
  } else {
    for (int e = tid; e < nr * b; e += blockDim.x) {
      const int r = e / b, j = e - r * b;
      Ct[r * cp + j] = a.angcand[(size_t)j * a.g.n + r0 + r];
    }
  }
  __syncthreads();
  const double* Ac = part + (size_t)k * kc_region(RC);
  const double* Bc = Ac + (size_t)bm * RC;
  for (int e = tid; e < nr * nacc; e += blockDim.x) {
    const int r = e / nacc, t = e - r * nacc;
    double x = 0.0;
    for (int j = 0; j < b; ++j) x += Ct[r * cp + j] * Ac[j * RC + t];
    for (int l = 0; l < cur0; ++l) x += Qt[r * qp + l] * Bc[l * RC + t];
    Q[(size_t)(r0 + r) * a.ldq + cur0 + t] = x;
  }
}

void launch_kc(const OrthArgs& a, const double* tab, const long long* off, const int* nf,
               const int* keep, double* part, int* kcn, int* kcur, int maxN, cudaStream_t st) {
  const int RC = a.g.RC, nsub = a.g.nsub;
  pbeg(st, KS_KC_W);
  if (a.spatial)
    k_kc_w<<<dim3(RC + 1, nsub), DD_THREADS, kc_w_smem(RC), st>>>(a, tab, off, nf, keep, part);
  else
    k_kca_w<<<dim3((kc_bmax(RC) + KCA_JC - 1) / KCA_JC, nsub), DD_THREADS, kca_w_smem(RC), st>>>(
        a, keep, part);
  pend(st);
  pbeg(st, KS_KC_SEL);
  k_kc_sel<<<nsub, DD_THREADS, kc_sel_smem(RC), st>>>(a, nf, keep, part, kcn, kcur);
  pend(st);
  pbeg(st, KS_KC_APPLY);
  const int rows_max = a.spatial ? maxN : a.g.n;
  k_kc_apply<<<dim3((rows_max + KC_TR3 - 1) / KC_TR3, nsub), DD_THREADS, kc_apply_smem(RC), st>>>(
      a, tab, off, nf, keep, kcn, part);
  pend(st);
}

void launch_complete(const OrthArgs& a, const int* keep, cudaStream_t st) {
  pbeg(st, KS_COMPLETE);
  k_complete<<<a.g.nsub, DD_THREADS, 0, st>>>(a, keep);
  pend(st);
}

cudaError_t orth_init() {
  cudaError_t e = cudaFuncSetAttribute(k_geig, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)geig_smem_bytes(DD_MAXC));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_kc_w, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kc_w_smem(DD_MAXC));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_kca_w, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kca_w_smem(DD_MAXC));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_kc_sel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kc_sel_smem(DD_MAXC));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_kc_apply, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kc_apply_smem(DD_MAXC));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_chol_inv, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)chol_smem_bytes(DD_MAXC));
}

}  // namespace dd
