// Phase kernels of the DD-DLRA time step (FP64).
//
// advection_phase() runs, for every subdomain at once, Algorithm 4 (augmentation)
// -> Algorithm 1 or 2 (projector-splitting integrator for x- or y-advection with
// the inflow boundary data of Eq. (generate_Kboundary) and the eigen-upwind
// K-step of Appendix A) -> Algorithm 5 (truncation).  collision_phase() runs
// Algorithm 3.  Storage is the Euclidean-rescaled form described in
// dd_internal.cuh: X = sqrt(hx hy) U, Vt = sqrt(w) V, S unchanged.
//
// Discrete operators (per subdomain, along the advection axis, h = cell width):
//   K-step  dK/dt = -(c/h) [K |C| - K_prev C+ + K_next C-],  C = Vh^T diag(Omega) Vh,
//           C+- the positive / negative parts of C (Appendix A: each eigenvector of
//           C upwinded by the sign of its eigenvalue); K_prev/K_next take the
//           frozen ghost rows K^b at the line ends.
//   S-step  dS/dt = (c/h) [S |C| - (T S + G_lo) C+ + (T^T S + G_hi) C-],
//           T = X^T shift_prev(X), G_lo/hi = X_face^T K^b_lo/hi  (the K-step
//           operator projected on the new basis, Eq. (advx_evolS)).
//   L-step  per direction q:  dL_q/dt = -(c Omega_q/h) [(I - T) L_q - G_lo Vh_q]  (Omega_q > 0)
//                              dL_q/dt = -(c Omega_q/h) [(T^T - I) L_q + G_hi Vh_q] (Omega_q < 0)
//           (per-direction upwinding of f = U L^T with ghost f^b = K^b V^T, Eq. (advx_evolL)).
#include <map>
#include <mutex>
#include <vector>

#include "dd_internal.cuh"

#include <climits>
#include "dd_launch.h"

namespace dd {

#define SMB(B, P, k, idx) ((B).sm + ((long)(k) * NSMALL + (idx)) * (long)(P).g.RC * (P).g.RC)

namespace {

__constant__ double c_rk_a[4] = {0.0, 0.5, 0.5, 1.0};
__constant__ double c_rk_b[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};

// out[i][j] (+)= alpha * sum_l A[i][l] B[l][j], block-wide, threads over (i, j)
__device__ void bmm(double* out, int ldo, double alpha, const double* A, int lda, const double* Bm,
                    int ldb, int ni, int nj, int nl, bool accumulate) {
  for (int e = threadIdx.x; e < ni * nj; e += blockDim.x) {
    int i = e / nj, j = e % nj;
    double s = 0.0;
    for (int l = 0; l < nl; ++l) s += A[i * lda + l] * Bm[l * ldb + j];
    out[i * ldo + j] = accumulate ? out[i * ldo + j] + alpha * s : alpha * s;
  }
}

// ---------------------------------------------------------------------------
// augmentation input  L0 = [Vt S^T, Vt_lo S_lo^T, Vt_hi S_hi^T]
// ---------------------------------------------------------------------------
// Columns of L0: the own block, the neighbours' blocks and one column per physical
// inflow side of the axis (the inflow's angular profile, a virtual neighbour).
__global__ void k_aug_cols(Geo g, const int* r, int axis, int* m, const int* infl_on) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= g.nsub) return;
  int lo = g.nb[k * 4 + 2 * axis], hi = g.nb[k * 4 + 2 * axis + 1];
  const int il = (lo < 0 && infl_on && infl_on[k * 4 + 2 * axis]) ? 1 : 0;
  const int ih = (hi < 0 && infl_on && infl_on[k * 4 + 2 * axis + 1]) ? 1 : 0;
  m[k] = r[k] + (lo >= 0 ? r[lo] : 0) + (hi >= 0 ? r[hi] : 0) + il + ih;
}

__global__ void k_build_L0(Geo g, const double* V, const double* S, const int* r, int axis,
                           double* L0, const int* infl_on, const double* infl_hw,
                           const double* infl_sc) {
  extern __shared__ double sh[];
  const int k = blockIdx.y, RC = g.RC;
  const int lo = g.nb[k * 4 + 2 * axis], hi = g.nb[k * 4 + 2 * axis + 1];
  const int src[3] = {k, lo, hi};
  int rr[3];
  for (int b = 0; b < 3; ++b) rr[b] = src[b] >= 0 ? r[src[b]] : 0;
  const int sl = 2 * axis, shi = 2 * axis + 1;
  const int il = (lo < 0 && infl_on && infl_on[k * 4 + sl]) ? 1 : 0;
  const int ih = (hi < 0 && infl_on && infl_on[k * 4 + shi]) ? 1 : 0;
  // stage the three S blocks
  for (int b = 0; b < 3; ++b)
    for (int e = threadIdx.x; e < RC * RC; e += blockDim.x)
      sh[b * RC * RC + e] = src[b] >= 0 ? S[(long)src[b] * RC * RC + e] : 0.0;
  __syncthreads();
  const int mn = rr[0] + rr[1] + rr[2], m = mn + il + ih;
  const int q0 = blockIdx.x * 32;
  for (int e = threadIdx.x; e < 32 * m; e += blockDim.x) {
    int q = q0 + e / m, col = e % m;
    if (q >= g.n) continue;
    if (col >= mn) {                               // inflow column: sqrt(w) m_in h |g|_x
      const int side = (col == mn && il) ? sl : shi;
      L0[((long)k * g.n + q) * g.MC + col] =
          infl_hw[((long)k * 4 + side) * g.n + q] * infl_sc[k * 4 + side];
      continue;
    }
    int b = 0, t = col;
    while (t >= rr[b]) { t -= rr[b]; ++b; }
    const double* Vq = V + ((long)src[b] * g.n + q) * RC;
    const double* Sb = sh + b * RC * RC + t * RC;     // row t of S_b
    double s = 0.0;
    for (int l = 0; l < rr[b]; ++l) s += Vq[l] * Sb[l];
    L0[((long)k * g.n + q) * g.MC + col] = s;
  }
}

// ---------------------------------------------------------------------------
// angular Galerkin coefficients (partial sums over direction chunks)
//   C = Vh^T diag(Om) Vh, Mout_lo = Vh^T diag(Om<0) Vh, Mout_hi = Vh^T diag(Om>=0) Vh,
//   M = Vt^T Vh, Min_lo = Vt_lo^T diag(Om>=0) Vh, Min_hi = Vt_hi^T diag(Om<0) Vh
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(DD_THREADS) k_ang_coeffs(Geo g, const double* om,
                                                            const double* Vh, const double* V,
                                                            const int* r, const int* rt, int axis,
                                                            int nchunk, int nblk, double* part,
                                                            const int* infl_on,
                                                            const double* infl_hw) {
  // Work items, enumerated densely so that every lane of an FP64 instruction is used:
  // the rt(rt+1)/2 pairs i <= j of the three symmetric blocks C, Mout_lo, Mout_hi (one
  // product v_i v_j per direction feeds all three), then the pairs of M, Min_lo and
  // Min_hi.  The sign of Om is taken from its bits (Om < 0 <=> sign bit set, not -0).
  // nblk = 8 adds the direction split C+ = <Vh, Om+ Vh>, C- = <Vh, Om- Vh> (flux-split
  // K-step) as blocks 6 and 7, from the same products.
  const int k = blockIdx.y, c = blockIdx.x, RC = g.RC, n = g.n;
  const int ch = (n + nchunk - 1) / nchunk;
  const int q0 = c * ch, q1 = min(n, q0 + ch);
  const int lo = g.nb[k * 4 + 2 * axis], hi = g.nb[k * 4 + 2 * axis + 1];
  // a physical inflow side takes the neighbour's place with one row, the inflow's
  // angular column sqrt(w) m_in h (already masked): Min = that column^T Vh
  const bool il = lo < 0 && infl_on && infl_on[k * 4 + 2 * axis];
  const bool ih = hi < 0 && infl_on && infl_on[k * 4 + 2 * axis + 1];
  const int rtk = rt[k], rk = r[k];
  const int rlo = lo >= 0 ? r[lo] : (il ? 1 : 0), rhi = hi >= 0 ? r[hi] : (ih ? 1 : 0);
  const double* Vhk = Vh + (long)k * n * RC;
  const double* Vk = V + (long)k * n * RC;
  const double* Vlo = lo >= 0 ? V + (long)lo * n * RC
                              : (il ? infl_hw + ((long)k * 4 + 2 * axis) * n : V);
  const double* Vhi = hi >= 0 ? V + (long)hi * n * RC
                              : (ih ? infl_hw + ((long)k * 4 + 2 * axis + 1) * n : V);
  const int slo = lo >= 0 ? RC : 1, shi = hi >= 0 ? RC : 1;   // row strides
  double* out = part + ((long)k * nchunk + c) * nblk * RC * RC;
  for (int e = threadIdx.x; e < nblk * RC * RC; e += blockDim.x) out[e] = 0.0;
  __syncthreads();
  const int nsym = rtk * (rtk + 1) / 2;
  const int n3 = rk * rtk, n4 = rlo * rtk, n5 = rhi * rtk;
  const int nwork = nsym + n3 + n4 + n5;
  count_work(g, KS_ANG_COEFFS, (double)(q1 - q0) * (nsym * (nblk == 8 ? 8.0 : 5.0) + 2.0 * (n3 + n4 + n5)));
  for (int w = threadIdx.x; w < nwork; w += blockDim.x) {
    if (w < nsym) {
      int j = (int)((sqrtf(8.f * w + 1.f) - 1.f) * 0.5f);
      j += (j + 1) * (j + 2) / 2 <= w;
      j -= j * (j + 1) / 2 > w;
      const int i = w - j * (j + 1) / 2;
      double sc = 0.0, sl = 0.0, sh = 0.0, sp = 0.0, sm = 0.0;
      if (nblk == 8) {
        #pragma unroll 8
        for (int q = q0; q < q1; ++q) {
          const double o = om[q];
          const long long ob = __double_as_longlong(o);
          const double t = Vhk[q * RC + i] * Vhk[q * RC + j];
          sc += o * t;
          if (ob < 0 && ob != (long long)0x8000000000000000ull) { sl += t; sm += o * t; }
          else { sh += t; sp += o * t; }
        }
      } else {                                     // C+ and C- not wanted: three FP64 ops a term
        #pragma unroll 8
        for (int q = q0; q < q1; ++q) {
          const double o = om[q];
          const long long ob = __double_as_longlong(o);
          const double t = Vhk[q * RC + i] * Vhk[q * RC + j];
          sc += o * t;
          if (ob < 0 && ob != (long long)0x8000000000000000ull) sl += t;
          else sh += t;
        }
      }
      out[i * RC + j] = sc; out[j * RC + i] = sc;
      out[RC * RC + i * RC + j] = sl; out[RC * RC + j * RC + i] = sl;
      out[2 * RC * RC + i * RC + j] = sh; out[2 * RC * RC + j * RC + i] = sh;
      if (nblk == 8) {
        out[6 * RC * RC + i * RC + j] = sp; out[6 * RC * RC + j * RC + i] = sp;
        out[7 * RC * RC + i * RC + j] = sm; out[7 * RC * RC + j * RC + i] = sm;
      }
    } else {
      int u = w - nsym, blk;
      const double* Va;
      int sel, sa;                                 // sel: 0 all directions, 1 Om >= 0, 2 Om < 0
      if (u < n3) { blk = 3; Va = Vk; sel = 0; sa = RC; }
      else if ((u -= n3) < n4) { blk = 4; Va = Vlo; sel = 1; sa = slo; }
      else { u -= n4; blk = 5; Va = Vhi; sel = 2; sa = shi; }
      const int i = u / rtk, j = u - i * rtk;
      double s = 0.0;
      #pragma unroll 8
      for (int q = q0; q < q1; ++q) {
        const long long ob = __double_as_longlong(om[q]);
        const bool ng = ob < 0 && ob != (long long)0x8000000000000000ull;
        if (sel == 0 || (sel == 1 && !ng) || (sel == 2 && ng)) s += Va[q * sa + i] * Vhk[q * RC + j];
      }
      out[blk * RC * RC + i * RC + j] = s;
    }
  }
}

struct Dst {
  int idx[8];
  int ident = 0;   // bit b: block b holds E and the slot receives I - E
};

// Sum the chunk partials in fixed order into the small matrices.
__global__ void k_reduce(const double* part, int nchunk, int nblk, Dst dst, double* sm, int RC) {
  const int k = blockIdx.y;
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < nblk * RC * RC; o += gridDim.x * blockDim.x) {
    const int b = o / (RC * RC), e = o % (RC * RC);
    double s = 0.0;
    for (int c = 0; c < nchunk; ++c) s += part[(((long)k * nchunk + c) * nblk + b) * RC * RC + e];
    if ((dst.ident >> b) & 1) s = (e / RC == e % RC ? 1.0 : 0.0) - s;
    sm[((long)k * NSMALL + dst.idx[b]) * RC * RC + e] = s;
  }
}

// Generic chunked Gram  G = A^T diag(w) B  over the rows of one subdomain.
// spatial != 0: rows are the subdomain's cells; else its directions.
// B may be a per-row vector (ldb = 1, bcols = 1).
struct GramArgs {
  int spatial;
  const double* A; int lda; const int* acnt; int afix;
  const double* Bm; int ldb; const int* bcnt; int bfix; int b_per_sub;  // b_per_sub: B has per-subdomain rows
  const double* wrow;   // row weights (indexed like a per-row vector of the same layout), or null
  double* part; int nchunk;
  int* cexp;            // A^T A only (Bm == A): chunk exponents, see k_gram
  int sym;              // A^T W A: the upper triangle is computed and mirrored
};
// Chunked Gram A^T diag(w) B: block (c, k) sums over row chunk c of subdomain k.  Each
// thread owns whole (i, j) pairs, enumerated densely (the upper triangle only for a
// symmetric product) so that every lane of an FP64 instruction does useful work; the
// RC x RC partial is assembled in shared memory and stored whole (zeros outside).
__global__ void __launch_bounds__(DD_THREADS) k_gram(Geo g, GramArgs a) {
  extern __shared__ double gt[];
  __shared__ long long mred[DD_THREADS / 32];
  const int k = blockIdx.y, c = blockIdx.x, RC = g.RC;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int rows = a.spatial ? g.N[k] : g.n;
  const long rb = a.spatial ? (long)g.rowoff[k] : (long)k * g.n;
  const long rbB = a.b_per_sub ? rb : 0;
  const int ch = (rows + a.nchunk - 1) / a.nchunk;
  const int i0 = c * ch, i1 = min(rows, i0 + ch);
  const int na = a.acnt ? a.acnt[k] : a.afix, nbc = a.bcnt ? a.bcnt[k] : a.bfix;
  double* out = a.part + ((long)k * a.nchunk + c) * RC * RC;
  // A^T A squares the entries: a chunk whose largest |entry| 2^e is far from 1
  // (|e| > 400) is scaled by 2^-e first, so that tiny data keep their significant
  // bits (e is stored; INT_MIN marks a chunk below 2^-1000, taken as zero).  The
  // largest |entry| is found on the integer order of the bit patterns (NaN ignored).
  int ex = 0;
  bool scl = false, zero = false;
  if (a.cexp) {
    long long mb = 0;
    for (int row = i0 + warp; row < i1; row += DD_THREADS / 32)
      for (int l = lane; l < na; l += 32) {
        const long long b = __double_as_longlong(a.A[(rb + row) * a.lda + l]) & 0x7fffffffffffffffll;
        if (b <= 0x7ff0000000000000ll) mb = max(mb, b);
      }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, o));
    if (lane == 0) mred[warp] = mb;
    __syncthreads();
    mb = 0;
    for (int w = 0; w < DD_THREADS / 32; ++w) mb = max(mb, mred[w]);
    const double mx = __longlong_as_double(mb);
    const int e0 = (mx > 0.0 && isfinite(mx)) ? ilogb(mx) : 0;
    zero = !(mx > 0.0) || e0 < -1000;
    scl = !zero && (e0 < -400 || e0 > 400);
    ex = scl ? e0 : 0;
    if (tid == 0) a.cexp[(long)k * a.nchunk + c] = zero ? INT_MIN : ex;
  }
  const double f = scl ? ldexp(1.0, -ex) : 1.0;
  for (int e = tid; e < RC * RC; e += DD_THREADS) gt[e] = 0.0;
  __syncthreads();
  const int npair = zero ? 0 : (a.sym ? na * (na + 1) / 2 : na * nbc);
  count_work(g, KS_GRAM, 2.0 * (i1 - i0) * npair * (a.wrow ? 1.5 : 1.0));
  for (int p = tid; p < npair; p += DD_THREADS) {
    int i, j;
    if (a.sym) {                                   // p -> (i <= j)
      j = (int)((sqrtf(8.f * p + 1.f) - 1.f) * 0.5f);
      j += (j + 1) * (j + 2) / 2 <= p;
      j -= j * (j + 1) / 2 > p;
      i = p - j * (j + 1) / 2;
    } else {
      i = p / nbc;
      j = p - i * nbc;
    }
    const double* Ac = a.A + rb * a.lda + i;
    const double* Bc = a.Bm + rbB * a.ldb + j;
    double s0 = 0.0;
    if (scl) {
      for (int row = i0; row < i1; ++row)
        s0 += (Ac[(long)row * a.lda] * f) * (Bc[(long)row * a.ldb] * f);
    } else if (a.wrow) {
      for (int row = i0; row < i1; ++row)
        s0 += Ac[(long)row * a.lda] * a.wrow[rb + row] * Bc[(long)row * a.ldb];
    } else {
      for (int row = i0; row < i1; ++row) s0 += Ac[(long)row * a.lda] * Bc[(long)row * a.ldb];
    }
    const double sv = s0;
    gt[i * RC + j] = sv;
    if (a.sym) gt[j * RC + i] = sv;
  }
  __syncthreads();
  for (int e = tid; e < RC * RC; e += DD_THREADS) out[e] = gt[e];
}

// ---------------------------------------------------------------------------
// small per-subdomain algebra: B = S M, B_lo = S_lo Min_lo, B_hi = S_hi Min_hi,
// Jacobi eigendecomposition of C -> C+, C-, |C|  (Appendix A)
// ---------------------------------------------------------------------------
size_t small_adv1_smem(int RC) {
  return sizeof(double) * (2 * RC * RC + RC) + 8 * ((jacobi_mixed_scratch_bytes(RC) + 7) / 8) +
         sizeof(int) * 16;
}

__global__ void __launch_bounds__(DD_THREADS) k_small_adv1(Problem P, PhaseBufs B, int axis) {
  extern __shared__ double sh[];
  const int k = blockIdx.x, RC = P.g.RC;
  const int lo = P.g.nb[k * 4 + 2 * axis], hi = P.g.nb[k * 4 + 2 * axis + 1];
  const int rk = B.r[k], rt = B.rt[k];
  const int rlo = lo >= 0 ? B.r[lo] : 0, rhi = hi >= 0 ? B.r[hi] : 0;
  const double* Sk = B.S + (long)k * RC * RC;
  // products (inputs read from global; outputs to the small buffers)
  bmm(SMB(B, P, k, SM_B), RC, 1.0, Sk, RC, SMB(B, P, k, SM_M), RC, rk, rt, rk, false);
  if (lo >= 0)
    bmm(SMB(B, P, k, SM_B_LO), RC, 1.0, B.S + (long)lo * RC * RC, RC, SMB(B, P, k, SM_MIN_LO), RC,
        rlo, rt, rlo, false);
  if (hi >= 0)
    bmm(SMB(B, P, k, SM_B_HI), RC, 1.0, B.S + (long)hi * RC * RC, RC, SMB(B, P, k, SM_MIN_HI), RC,
        rhi, rt, rhi, false);
  // a physical inflow side: its face values carry the whole amplitude, B = Min (one row)
  for (int side = 0; side < 2; ++side) {
    const int nbs = side ? hi : lo;
    if (nbs >= 0 || !P.infl_on || !P.infl_on[k * 4 + 2 * axis + side]) continue;
    const double* Mi = SMB(B, P, k, side ? SM_MIN_HI : SM_MIN_LO);
    double* Bs = SMB(B, P, k, side ? SM_B_HI : SM_B_LO);
    for (int t = threadIdx.x; t < RC; t += blockDim.x) Bs[t] = t < rt ? Mi[t] : 0.0;
  }
  if (P.kstep_split == 1) {
    // flux split: C+ and C- came with the Galerkin coefficients; |C| = C+ - C-
    const double* Cp = SMB(B, P, k, SM_CP);
    const double* Cn = SMB(B, P, k, SM_CM);
    double* Ca = SMB(B, P, k, SM_CABS);
    for (int e = threadIdx.x; e < RC * RC; e += blockDim.x) Ca[e] = Cp[e] - Cn[e];
    return;
  }
  // Eigendecomposition of the symmetric rt x rt matrix C: one-sided Jacobi of the
  // positive semidefinite C + s I (s = |C|_F >= its spectral radius); the column
  // norms of (C + s I) P are lambda + s.  FP32 sweeps and a double-float finish,
  // accurate to ~1e-13 |C|, then one FP64 refinement step, in every precision: the upwind
  // split feeds every stencil application (FP32 errors here were the largest part of the
  // mixed form's; the double-float level still put single steps of narrow sources 1e-10
  // off the oracle).
  double* Bc = sh;                      // RC*RC column-major
  double* Pm = Bc + RC * RC;            // RC*RC eigenvectors: column l = Pm[l*RC + i]
  double* lam = Pm + RC * RC;           // RC
  double* X = lam + RC;                 // SVD scratch
  int* iv = reinterpret_cast<int*>(X + (jacobi_mixed_scratch_bytes(RC) + 7) / 8);
  __shared__ double red[40];
  const double* Csrc = SMB(B, P, k, SM_C);
  double nf = 0.0;
  for (int e = threadIdx.x; e < rt * rt; e += blockDim.x) {
    const int i = e / rt, j = e % rt;
    const double x = 0.5 * (Csrc[i * RC + j] + Csrc[j * RC + i]);
    nf += x * x;
  }
  const double shift = sqrt(block_sum(nf, red));
  for (int e = threadIdx.x; e < RC * RC; e += blockDim.x) {
    const int col = e / RC, row = e % RC;
    double x = 0.0;
    if (row < rt && col < rt) x = 0.5 * (Csrc[row * RC + col] + Csrc[col * RC + row]) + (row == col ? shift : 0.0);
    Bc[e] = x;
    Pm[e] = (row == col) ? 1.0 : 0.0;
  }
  __syncthreads();
  jacobi_svd_mixed(Bc, Pm, rt, RC, &iv[0], lam, X);
  {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int j = warp; j < rt; j += nwarps) {
      double s2 = 0.0;
      for (int l = lane; l < rt; l += 32) s2 += Bc[j * RC + l] * Bc[j * RC + l];
      s2 = warp_sum(s2);
      if (lane == 0) lam[j] = sqrt(s2) - shift;
    }
  }
  __syncthreads();
  // one FP64 refinement step of P and lambda (C itself, symmetrised, in Bc): the split's
  // sensitivity to P is |C| / (the gap between positive and negative eigenvalues), and
  // the double-float Jacobi alone left splits ~1e-13 |C| / gap off the FP64 ones
  for (int e = threadIdx.x; e < RC * RC; e += blockDim.x) {
    const int i = e / RC, j = e % RC;
    Bc[e] = (i < rt && j < rt) ? 0.5 * (Csrc[i * RC + j] + Csrc[j * RC + i]) : 0.0;
  }
  __syncthreads();
  refine_sym_eig(Bc, Pm, lam, rt, RC, X);
  // C+ = P diag(max(l,0)) P^T, C- = P diag(min(l,0)) P^T
  double* Cp = SMB(B, P, k, SM_CP);
  double* Cn = SMB(B, P, k, SM_CM);
  double* Ca = SMB(B, P, k, SM_CABS);
  // (upper triangles, mirrored: the products P_li P_lj are symmetric bit for bit)
  for (int e = threadIdx.x; e < RC * RC; e += blockDim.x) {
    const int i = e / RC, j = e - i * RC;
    if (i >= rt || j >= rt) { Cp[e] = 0.0; Cn[e] = 0.0; Ca[e] = 0.0; }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < rt * (rt + 1) / 2; e += blockDim.x) {
    int j = (int)((sqrtf(8.f * e + 1.f) - 1.f) * 0.5f);
    j += (j + 1) * (j + 2) / 2 <= e;
    j -= j * (j + 1) / 2 > e;
    const int i = e - j * (j + 1) / 2;              // i <= j
    double sp = 0.0, sm = 0.0;
    for (int l = 0; l < rt; ++l) {
      const double pp = Pm[l * RC + i] * Pm[l * RC + j];
      if (lam[l] > 0.0) sp += lam[l] * pp;
      else if (lam[l] < 0.0) sm += lam[l] * pp;
    }
    Cp[i * RC + j] = sp; Cn[i * RC + j] = sm; Ca[i * RC + j] = sp - sm;
    Cp[j * RC + i] = sp; Cn[j * RC + i] = sm; Ca[j * RC + i] = sp - sm;
  }
  // P and lambda for the eigenbasis K-step (slots S3T and VB are free until the S-step)
  double* Pout = SMB(B, P, k, SM_S3T);
  double* lout = SMB(B, P, k, SM_VB);
  for (int e = threadIdx.x; e < RC * RC; e += blockDim.x) {
    const int u = e / RC, j = e % RC;
    Pout[e] = (u < rt && j < rt) ? Pm[j * RC + u] : 0.0;
  }
  for (int j = threadIdx.x; j < RC; j += blockDim.x) lout[j] = j < rt ? lam[j] : 0.0;
}

// ---------------------------------------------------------------------------
// tall x small product  Y = A Bm  (per subdomain counts), zero-filled to ldy
// ---------------------------------------------------------------------------
struct TallArgs {
  int spatial;
  const double* A; int lda; const int* ninner; int ninner_fix;
  const double* Bm; int bsmall;     // small matrix index inside the subdomain block (or -1: Bm is per-k RC*RC stride)
  const int* ncols; int ncols_fix;
  double* Y; int ldy;
  // optional: the Gram Y^T Y of each row tile (nc x nc, RC x RC stride) to
  // gpart[k * gridDim.x + tile], the chunk partials of the next orthonormalisation step
  double* gpart;
};
#define TALL_ROWS 32
size_t tall_smem(int RC, int ldy) {
  return sizeof(double) * ((size_t)RC * RC + 4 + TALL_ROWS * (RC | 1) + TALL_ROWS * (ldy | 1));
}
// Y = A M (rows of subdomain k; columns nc..ldy-1 of Y set to zero).  A block takes
// TALL_ROWS rows: the rows of A, M and the output tile live in shared memory (loads
// and stores coalesced); lane = row, each warp takes tiles of 4 output columns, so
// every lane of an FP64 instruction does useful work.
__global__ void __launch_bounds__(DD_THREADS) k_tall(Geo g, TallArgs a, double* smbase) {
  extern __shared__ double sh[];
  const int k = blockIdx.y, RC = g.RC;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int rows = a.spatial ? g.N[k] : g.n;
  const long rb = a.spatial ? (long)g.rowoff[k] : (long)k * g.n;
  const int ni = a.ninner ? a.ninner[k] : a.ninner_fix;
  const int nc = a.ncols ? a.ncols[k] : a.ncols_fix;
  const int r0 = blockIdx.x * TALL_ROWS;
  const int nrow = min(TALL_ROWS, rows - r0);
  double* gp = a.gpart ? a.gpart + ((long)k * gridDim.x + blockIdx.x) * RC * RC : nullptr;
  if (nrow <= 0) {
    if (gp)
      for (int e = tid; e < nc * nc; e += DD_THREADS) gp[(e / nc) * RC + e % nc] = 0.0;
    return;
  }
  const double* Bk = (a.bsmall >= 0) ? smbase + ((long)k * NSMALL + a.bsmall) * RC * RC
                                     : a.Bm + (long)k * RC * RC;
  const int SA = ni | 1, SY = a.ldy | 1;
  count_work(g, KS_TALL, 2.0 * nrow * ni * nc + (gp ? (double)nrow * nc * (nc + 1) : 0.0));
  double* Ms = sh;                                  // RC x RC (+4 so a tile never reads past it)
  double* As = Ms + RC * RC + 4;                    // TALL_ROWS x SA
  double* Ys = As + TALL_ROWS * (RC | 1);           // TALL_ROWS x SY
  for (int e = tid; e < RC * RC + 4; e += DD_THREADS) Ms[e] = e < ni * RC ? Bk[e] : 0.0;
  for (int r = warp; r < nrow; r += DD_THREADS / 32)
    for (int l = lane; l < ni; l += 32) As[r * SA + l] = a.A[(rb + r0 + r) * a.lda + l];
  __syncthreads();
  const int ntile = (a.ldy + 3) >> 2;
  for (int t = warp; t < ntile; t += DD_THREADS / 32) {
    const int j0 = t * 4;
    double c0 = 0.0, c1 = 0.0, c2 = 0.0, c3 = 0.0;
    if (j0 < nc && lane < nrow) {
      const double* ar = As + lane * SA;
      for (int l = 0; l < ni; ++l) {
        const double x = ar[l];
        const double* mr = Ms + l * RC + j0;
        c0 += x * mr[0]; c1 += x * mr[1]; c2 += x * mr[2]; c3 += x * mr[3];
      }
    }
    if (lane < nrow) {
      double* yr = Ys + lane * SY + j0;
      if (j0 < a.ldy) yr[0] = j0 < nc ? c0 : 0.0;
      if (j0 + 1 < a.ldy) yr[1] = j0 + 1 < nc ? c1 : 0.0;
      if (j0 + 2 < a.ldy) yr[2] = j0 + 2 < nc ? c2 : 0.0;
      if (j0 + 3 < a.ldy) yr[3] = j0 + 3 < nc ? c3 : 0.0;
    }
  }
  __syncthreads();
  for (int r = warp; r < nrow; r += DD_THREADS / 32)
    for (int j = lane; j < a.ldy; j += 32) a.Y[(rb + r0 + r) * a.ldy + j] = Ys[r * SY + j];
  if (gp) {
    // the tile's Gram, pairs (i <= j) enumerated densely, rows in order
    const int npair = nc * (nc + 1) / 2;
    for (int p = tid; p < npair; p += DD_THREADS) {
      int j = (int)((sqrtf(8.f * p + 1.f) - 1.f) * 0.5f);
      j += (j + 1) * (j + 2) / 2 <= p;
      j -= j * (j + 1) / 2 > p;
      const int i = p - j * (j + 1) / 2;
      double x = 0.0;
      for (int r = 0; r < nrow; ++r) x += Ys[r * SY + i] * Ys[r * SY + j];
      gp[i * RC + j] = x;
      gp[j * RC + i] = x;
    }
  }
}

// ---------------------------------------------------------------------------
// ghost rows (Eq. (generate_Kboundary)): K^b_lo = (X_lo S_lo)|face Min_lo + K|own lo face Mout_lo
// ---------------------------------------------------------------------------
// One warp per (side, line) ghost row, lane = output column t: the blocks of a
// subdomain split its 2 * nlines rows, so every SM takes part.
__global__ void __launch_bounds__(DD_THREADS) k_ghost(Problem P, PhaseBufs B, int axis) {
  const int k = blockIdx.y, RC = P.g.RC;
  const Lines L = lines_of(P.g, k, axis);
  const int rt = B.rt[k];
  const int row = blockIdx.x * (DD_THREADS / 32) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (row >= 2 * L.nlines) return;
  const int side = row >= L.nlines, line = side ? row - L.nlines : row;
  const int nbk = P.g.nb[k * 4 + 2 * axis + side];
  const double* Mout = SMB(B, P, k, side == 0 ? SM_MOUT_LO : SM_MOUT_HI);
  const int own = cell_of(L, line, side == 0 ? 0 : L.len - 1);
  const double* Kr = B.K + ((long)P.g.rowoff[k] + own) * RC;
  const double* Xr = nullptr;
  const double* Bb = SMB(B, P, k, side == 0 ? SM_B_LO : SM_B_HI);
  int rn = 0;
  if (nbk >= 0) {
    const Lines Ln = lines_of(P.g, nbk, axis);
    const int cell = cell_of(Ln, line, side == 0 ? Ln.len - 1 : 0);
    Xr = B.X + ((long)P.g.rowoff[nbk] + cell) * RC;
    rn = B.r[nbk];
  } else if (P.infl_on && P.infl_on[k * 4 + 2 * axis + side]) {
    // physical inflow: the face value sqrt(hx hy) g(line) times B = Min
    Xr = P.infl_g + ((long)k * 4 + 2 * axis + side) * P.maxlines + line;
    rn = 1;
  }
  double* out = B.Kb + (((long)k * 2 + side) * P.maxlines + line) * RC;
  for (int t = lane; t < RC; t += 32) {
    double s = 0.0;
    if (t < rt) {
      for (int u = 0; u < rt; ++u) s += Kr[u] * Mout[u * RC + t];
      for (int u = 0; u < rn; ++u) s += Xr[u] * Bb[u * RC + t];
    }
    out[t] = s;
  }
}

// ---------------------------------------------------------------------------
// K-step of the advection (Appendix A), all RK stages fused; a CTA owns whole lines
// ---------------------------------------------------------------------------
#define KS_EPT 24    // entries per thread of k_kstep_adv (lines x cells x r_t <= 256 x 24)
#define KE_EPT 16    // entries per thread of k_kstep_eig (<= 256 x 16)
// TC: arithmetic type (double for the FP64 path, float for the mixed path); the
// factors stay FP64 in memory.  big_only: only the subdomains whose line does not fit
// k_kstep_eig's tile (len r_t > 256 KE_EPT; that kernel skips them).
template <typename TC>
__global__ void __launch_bounds__(DD_THREADS) k_kstep_adv(Problem P, PhaseBufs B, int axis, int lpb,
                                                          int big_only) {
  extern __shared__ double sh_raw[];
  TC* sh = reinterpret_cast<TC*>(sh_raw);
  const int k = blockIdx.y, RC = P.g.RC;
  const Lines L = lines_of(P.g, k, axis);
  const int l0 = blockIdx.x * lpb;
  if (l0 >= L.nlines) return;
  const int nl = min(lpb, L.nlines - l0);
  const int rt = B.rt[k];
  const int len = L.len;
  if (big_only && (long)len * rt <= (long)DD_THREADS * KE_EPT) return;
  count_work(P.g, KS_KSTEP_ADV, (double)nl * len * rt * (6.0 * rt + 4.0) * (P.integrator == 1 ? 4 : 1));
  TC* Cp = sh;
  TC* Cn = Cp + RC * RC;
  TC* Ca = Cn + RC * RC;
  TC* Glo = Ca + RC * RC;          // lpb x RC
  TC* Ghi = Glo + lpb * RC;
  TC* Kst = Ghi + lpb * RC;        // lpb x len x rt
  for (int e = threadIdx.x; e < RC * RC; e += blockDim.x) {
    Cp[e] = (TC)SMB(B, P, k, SM_CP)[e];
    Cn[e] = (TC)SMB(B, P, k, SM_CM)[e];
    Ca[e] = (TC)SMB(B, P, k, SM_CABS)[e];
  }
  for (int e = threadIdx.x; e < nl * RC; e += blockDim.x) {
    int li = e / RC, t = e % RC;
    Glo[e] = (TC)B.Kb[(((long)k * 2 + 0) * P.maxlines + l0 + li) * RC + t];
    Ghi[e] = (TC)B.Kb[(((long)k * 2 + 1) * P.maxlines + l0 + li) * RC + t];
  }
  const int tot = nl * len * rt;
  TC k0[KS_EPT], acc[KS_EPT];
  for (int i = 0; i < KS_EPT; ++i) {
    int e = threadIdx.x + i * blockDim.x;
    k0[i] = 0; acc[i] = 0;
    if (e < tot) {
      int li = e / (len * rt), pos = (e / rt) % len, t = e % rt;
      int cell = cell_of(L, l0 + li, pos);
      k0[i] = (TC)B.K[((long)P.g.rowoff[k] + cell) * RC + t];
      Kst[e] = k0[i];
    }
  }
  __syncthreads();
  const TC coef = (TC)(-P.c_adv / (axis == 0 ? P.g.hxk[k] : P.g.hyk[k]));
  const TC dt = (TC)P.g.dtk[k];
  const int nst = P.integrator == 1 ? 4 : 1;
  for (int s = 0; s < nst; ++s) {
    TC kv[KS_EPT];
    for (int i = 0; i < KS_EPT; ++i) {
      int e = threadIdx.x + i * blockDim.x;
      kv[i] = 0;
      if (e < tot) {
        int li = e / (len * rt), pos = (e / rt) % len, t = e % rt;
        const TC* Kc = Kst + (li * len + pos) * rt;
        const TC* Kp = pos > 0 ? Kc - rt : Glo + li * RC;
        const TC* Kn = pos < len - 1 ? Kc + rt : Ghi + li * RC;
        TC a1 = 0, a2 = 0, a3 = 0;
        for (int u = 0; u < rt; ++u) {
          a1 += Kc[u] * Ca[u * RC + t];
          a2 += Kp[u] * Cp[u * RC + t];
          a3 += Kn[u] * Cn[u * RC + t];
        }
        kv[i] = coef * (a1 - a2 + a3);
      }
    }
    __syncthreads();
    const TC bs = (TC)((nst == 4) ? c_rk_b[s] : 1.0);
    const TC an = (TC)((s + 1 < nst) ? c_rk_a[s + 1] : 0.0);
    for (int i = 0; i < KS_EPT; ++i) {
      int e = threadIdx.x + i * blockDim.x;
      if (e < tot) {
        acc[i] += bs * kv[i];
        if (s + 1 < nst) Kst[e] = k0[i] + an * dt * kv[i];
      }
    }
    __syncthreads();
  }
  for (int i = 0; i < KS_EPT; ++i) {
    int e = threadIdx.x + i * blockDim.x;
    if (e < tot) {
      int li = e / (len * rt), pos = (e / rt) % len, t = e % rt;
      int cell = cell_of(L, l0 + li, pos);
      double* Ke = B.K + ((long)P.g.rowoff[k] + cell) * RC + t;
      // the increment is formed in TC, the update itself in FP64 (the start value is
      // re-read, so FP32 arithmetic never rounds the state)
      *Ke = *Ke + (double)(dt * acc[i]);
    }
  }
}

// K-step of the advection in the eigenbasis of C, where Appendix A's upwinding acts
// column by column: with K~ = K P (ghost rows likewise) each RK stage is
//   R~_ij = coef (lambda+_j (K~_ij - K~_(i-1)j) + lambda-_j (K~_(i+1)j - K~_ij)),
// O(1) per entry instead of the 3 r_t products of the matrix stencil; the increment
// dt sum_s b_s R~_s is rotated back with P^T and added to the FP64 state.  P and lambda
// come from k_small_adv1 (small slots S3T and VB, free until the S-step).  Same lines-
// per-CTA layout as k_kstep_adv; the entry indices are decoded once.
// The explicit-Euler K-step in the eigenbasis, the stencil alone: on K~ = K P (in X1, formed
// by a tall product) along the lines of the sweep, with the ghosts K^b P at the line ends,
// the increment dt coef (lambda+_j (K~_c - K~_p) + lambda-_j (K~_n - K~_c)) of column j
// (Appendix A's per-eigenvector upwinding) into Hw (zero in the columns from r_t; rotated
// back and added to K by the next tall product).  One line per CTA: warp w takes the
// columns 32 (w % 2) .. + 31 of the line's segment w / 2 (of KE1_SEGS), each thread walking
// its column along the segment with the previous and current entries in registers.  The
// one-stage form of k_kstep_eig's stencil, expanded into one coefficient per neighbour.
#define KE1_SEGS 4
static_assert(DD_THREADS == 64 * KE1_SEGS, "k_kstep_eig1: two warps per segment");
__global__ void __launch_bounds__(DD_THREADS) k_kstep_eig1(Problem P, PhaseBufs B, int axis) {
  __shared__ double gh[2][DD_MAXC];
  const int k = blockIdx.y, RC = P.g.RC, line = blockIdx.x;
  const Lines L = lines_of(P.g, k, axis);
  if (line >= L.nlines) return;
  const int len = L.len, rt = B.rt[k];
  count_work(P.g, KS_KSTEP_ADV, (double)len * rt * 8.0);
  const double* Pg = SMB(B, P, k, SM_S3T);
  const double* lam = SMB(B, P, k, SM_VB);
  for (int e = threadIdx.x; e < 2 * rt; e += blockDim.x) {     // ghosts in the eigenbasis
    const int side = e >= rt, j = e - side * rt;
    const double* kb = B.Kb + (((long)k * 2 + side) * P.maxlines + line) * RC;
    double x = 0.0;
    for (int u = 0; u < rt; ++u) x += kb[u] * Pg[u * RC + j];
    gh[side][j] = x;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, j = (warp & 1) * 32 + (threadIdx.x & 31);
  const int sl = (len + KE1_SEGS - 1) / KE1_SEGS, p0 = (warp >> 1) * sl, p1 = min(len, p0 + sl);
  if (j >= RC || p0 >= p1) return;
  const double coef = -P.c_adv / (axis == 0 ? P.g.hxk[k] : P.g.hyk[k]);
  const double dt = P.g.dtk[k];
  const long base = ((long)P.g.rowoff[k] + cell_of(L, line, 0)) * RC + j;
  const long step = (long)L.stride_pos * RC;
  if (j >= rt) {                                 // whole rows: the product reads pairs of columns
    for (int pos = p0; pos < p1; ++pos) B.Hw[base + pos * step] = 0.0;
    return;
  }
  // inc = cc kc + cp kp + cn kn with the column's coefficients (three FP64 operations per
  // entry: the kernel is bound by the FP64 pipe, whose warp instructions cost the same
  // however many lanes are active)
  const double l = lam[j], lp = l > 0.0 ? l : 0.0, ln = l < 0.0 ? l : 0.0;
  const double cpk = -dt * coef * lp, cnk = dt * coef * ln, cck = dt * coef * (lp - ln);
  double kp = p0 > 0 ? B.X1[base + (p0 - 1) * step] : gh[0][j], kc = B.X1[base + p0 * step];
#pragma unroll 4
  for (int pos = p0; pos < p1; ++pos) {
    const double kn = pos < len - 1 ? B.X1[base + (pos + 1) * step] : gh[1][j];
    B.Hw[base + pos * step] = fma(cnk, kn, fma(cpk, kp, cck * kc));
    kp = kc;
    kc = kn;
  }
}

template <typename TC>
__global__ void __launch_bounds__(DD_THREADS) k_kstep_eig(Problem P, PhaseBufs B, int axis, int lpb,
                                                      int ebasis) {
  extern __shared__ double sh_raw[];
  TC* sh = reinterpret_cast<TC*>(sh_raw);
  const int k = blockIdx.y, RC = P.g.RC;
  const Lines L = lines_of(P.g, k, axis);
  const int l0 = blockIdx.x * lpb;
  if (l0 >= L.nlines) return;
  const int nl = min(lpb, L.nlines - l0);
  const int rt = B.rt[k];
  const int len = L.len;
  // a tile larger than the register tile (only with lpb = 1: a line longer than
  // 256 KE_EPT / r_t) is left to k_kstep_adv, launched after this kernel for exactly these
  if ((long)nl * len * rt > (long)DD_THREADS * KE_EPT) return;
  count_work(P.g, KS_KSTEP_ADV,
             (double)nl * len * rt * ((ebasis ? 0.0 : 4.0 * rt) + 8.0 * (P.integrator == 1 ? 4 : 1)));
  // ebasis: K~ = K P was formed outside (in X1, by the tall products); the stages run on it
  // and the increment dt sum_s b_s R~_s is written back there (rotated back and added to K
  // outside)
  const double* Ksrc = ebasis ? B.X1 : B.K;
  TC* Pm = sh;                     // Pm[u * RC + j]: component u of eigenvector j
  TC* lp = Pm + RC * RC;           // max(lambda, 0)
  TC* ln = lp + RC;                // min(lambda, 0)
  TC* Glo = ln + RC;               // lpb x RC ghost rows in the eigenbasis
  TC* Ghi = Glo + lpb * RC;
  TC* Kst = Ghi + lpb * RC;        // lpb x len x rt
  const double* Pg = SMB(B, P, k, SM_S3T);
  const double* lam = SMB(B, P, k, SM_VB);
  for (int e = threadIdx.x; e < RC * RC; e += blockDim.x) Pm[e] = (TC)Pg[e];
  for (int j = threadIdx.x; j < RC; j += blockDim.x) {
    const double l = j < rt ? lam[j] : 0.0;
    lp[j] = (TC)(l > 0.0 ? l : 0.0);
    ln[j] = (TC)(l < 0.0 ? l : 0.0);
  }
  const int tot = nl * len * rt;
  int code[KE_EPT];                // li << 20 | pos << 8 | t (li < 2^11, pos < 2^12, t < 2^8)
#pragma unroll
  for (int i = 0; i < KE_EPT; ++i) {
    const int e = threadIdx.x + i * blockDim.x;
    code[i] = 0;
    if (e < tot) {
      const int li = e / (len * rt), pos = (e / rt) % len, t = e % rt;
      code[i] = (li << 20) | (pos << 8) | t;
      Kst[e] = (TC)Ksrc[((long)P.g.rowoff[k] + cell_of(L, l0 + li, pos)) * RC + t];
    }
  }
  __syncthreads();
  // ghosts and K into the eigenbasis
  for (int e = threadIdx.x; e < 2 * nl * rt; e += blockDim.x) {
    const int side = e >= nl * rt, r = e - side * nl * rt, li = r / rt, j = r - li * rt;
    const double* kb = B.Kb + (((long)k * 2 + side) * P.maxlines + l0 + li) * RC;
    TC x = 0;
    for (int u = 0; u < rt; ++u) x += (TC)kb[u] * Pm[u * RC + j];
    (side ? Ghi : Glo)[li * RC + j] = x;
  }
  TC k0[KE_EPT], acc[KE_EPT];
#pragma unroll
  for (int i = 0; i < KE_EPT; ++i) {
    const int e = threadIdx.x + i * blockDim.x;
    k0[i] = 0; acc[i] = 0;
    if (e < tot) {
      if (ebasis) {
        k0[i] = Kst[e];
      } else {
        const int t = code[i] & 255, rowe = e - t;   // entry of column 0 of this cell
        TC x = 0;
        for (int u = 0; u < rt; ++u) x += Kst[rowe + u] * Pm[u * RC + t];
        k0[i] = x;
      }
    }
  }
  __syncthreads();
  if (!ebasis) {
#pragma unroll
    for (int i = 0; i < KE_EPT; ++i) {
      const int e = threadIdx.x + i * blockDim.x;
      if (e < tot) Kst[e] = k0[i];
    }
  }
  __syncthreads();
  const TC coef = (TC)(-P.c_adv / (axis == 0 ? P.g.hxk[k] : P.g.hyk[k]));
  const TC dt = (TC)P.g.dtk[k];
  const int nst = P.integrator == 1 ? 4 : 1;
  for (int s = 0; s < nst; ++s) {
    TC kv[KE_EPT];
  #pragma unroll
  for (int i = 0; i < KE_EPT; ++i) {
      const int e = threadIdx.x + i * blockDim.x;
      kv[i] = 0;
      if (e < tot) {
        const int li = code[i] >> 20, pos = (code[i] >> 8) & 4095, j = code[i] & 255;
        const TC kc = Kst[e];
        const TC kp = pos > 0 ? Kst[e - rt] : Glo[li * RC + j];
        const TC kn = pos < len - 1 ? Kst[e + rt] : Ghi[li * RC + j];
        kv[i] = coef * (lp[j] * (kc - kp) + ln[j] * (kn - kc));
      }
    }
    __syncthreads();
    const TC bs = (TC)((nst == 4) ? c_rk_b[s] : 1.0);
    const TC an = (TC)((s + 1 < nst) ? c_rk_a[s + 1] : 0.0);
  #pragma unroll
  for (int i = 0; i < KE_EPT; ++i) {
      const int e = threadIdx.x + i * blockDim.x;
      if (e < tot) {
        acc[i] += bs * kv[i];
        Kst[e] = (s + 1 < nst) ? k0[i] + an * dt * kv[i] : acc[i];
      }
    }
    __syncthreads();
  }
  if (ebasis) {                     // the increment dt acc~, in the eigenbasis
#pragma unroll
    for (int i = 0; i < KE_EPT; ++i) {
      const int e = threadIdx.x + i * blockDim.x;
      if (e < tot) {
        const int li = code[i] >> 20, pos = (code[i] >> 8) & 4095, t = code[i] & 255;
        B.X1[((long)P.g.rowoff[k] + cell_of(L, l0 + li, pos)) * RC + t] = (double)(dt * Kst[e]);
      }
    }
    return;
  }
  // back to the original basis: increment_t = dt sum_j acc~_j P_tj, added in FP64
#pragma unroll
  for (int i = 0; i < KE_EPT; ++i) {
    const int e = threadIdx.x + i * blockDim.x;
    if (e < tot) {
      const int li = code[i] >> 20, pos = (code[i] >> 8) & 4095, t = code[i] & 255;
      const int rowe = e - t;
      TC x = 0;
      for (int j = 0; j < rt; ++j) x += Kst[rowe + j] * Pm[t * RC + j];
      double* Ke = B.K + ((long)P.g.rowoff[k] + cell_of(L, l0 + li, pos)) * RC + t;
      *Ke = *Ke + (double)(dt * x);
    }
  }
}

// ---------------------------------------------------------------------------
// spatial coefficients of the S- and L-steps (partial sums over cell chunks)
//   S1 = X1^T K1, T = X1^T shift_prev(X1), G_lo = X1_loface^T K^b_lo, G_hi = X1_hiface^T K^b_hi
// ---------------------------------------------------------------------------
// skip_t: every block but T (block 1), which the tensor-core Gram writes in its
// difference form E = I - T.
__global__ void k_sp_coeffs(Problem P, PhaseBufs B, int axis, int skip_t) {
  const int k = blockIdx.y, c = blockIdx.x, RC = P.g.RC, nchunk = P.nchunk_sp;
  const Lines L = lines_of(P.g, k, axis);
  // chunks of whole lines: every cell's shift partner and the two face cells of a
  // line are in the same chunk, and no index is divided inside the loops
  const int lch = (L.nlines + nchunk - 1) / nchunk;
  const int l0 = c * lch, l1 = min(L.nlines, l0 + lch);
  const int rt = B.rt[k];
  count_work(P.g, KS_SP_COEFFS, 2.0 * rt * rt * (max(0, l1 - l0) * (double)L.len * (skip_t ? 1 : 2) +
                                                 2.0 * max(0, l1 - l0)));
  const double* X1 = B.X1 + (long)P.g.rowoff[k] * RC;
  const double* K = B.K + (long)P.g.rowoff[k] * RC;
  const double* Kb = B.Kb + (long)k * 2 * P.maxlines * RC;
  double* out = B.part + ((long)k * nchunk + c) * 4 * RC * RC;
  // work items (block, i, j) enumerated densely over i, j < rt, so that every lane of
  // an FP64 instruction is used; the partial is zeroed first
  for (int o = threadIdx.x; o < 4 * RC * RC; o += blockDim.x)
    if (!(skip_t && o / (RC * RC) == 1)) out[o] = 0.0;
  __syncthreads();
  const int rt2 = rt * rt;
  for (int w = threadIdx.x; w < 4 * rt2; w += blockDim.x) {
    const int blk = w / rt2, e = w - blk * rt2, i = e / rt, j = e - i * rt;
    if (skip_t && blk == 1) continue;
    double s = 0.0;
    {
      if (blk == 0) {
        for (int line = l0; line < l1; ++line)
          for (int pos = 0, cell = line * L.stride_line; pos < L.len; ++pos, cell += L.stride_pos)
            s += X1[(long)cell * RC + i] * K[(long)cell * RC + j];
      } else if (blk == 1) {
        for (int line = l0; line < l1; ++line)
          for (int pos = 1, cell = line * L.stride_line + L.stride_pos; pos < L.len;
               ++pos, cell += L.stride_pos)
            s += X1[(long)cell * RC + i] * X1[(long)(cell - L.stride_pos) * RC + j];
      } else if (blk == 2) {
        for (int line = l0; line < l1; ++line)
          s += X1[(long)(line * L.stride_line) * RC + i] * Kb[(long)line * RC + j];
      } else {
        for (int line = l0; line < l1; ++line)
          s += X1[(long)(line * L.stride_line + (L.len - 1) * L.stride_pos) * RC + i] *
               Kb[((long)P.maxlines + line) * RC + j];
      }
    }
    out[blk * RC * RC + i * RC + j] = s;
  }
}

// ---------------------------------------------------------------------------
// S-step of the advection (small, one CTA per subdomain), and the L-step matrices
// ---------------------------------------------------------------------------
// One RK stage per launch, rows of each subdomain split over CL blocks: the FP64
// products of this r_t x r_t ODE would otherwise run on one SM per subdomain.  Block
// (k, c) takes rows [c*rpb, (c+1)*rpb): it reads the full stage value of S, computes its
// rows of U1 = T S + G_lo, U2 = T^T S + G_hi and F = coef (S |C| - U1 C+ + U2 C-),
// accumulates Ac = sum_s b_s F_s and writes its rows of the next stage value
// S1 + a_{s+1} dt F (at the last stage S2 = S1 + dt Ac and the L-step matrices).  The
// stage values alternate between the small slots S3T and UB, and Ac lives in VB: those
// are free between the QR of K and the QR of L.  Every element is computed in the same
// order as by a single block, so the result does not depend on CL.
size_t sstep_smem(int RC) { return sizeof(double) * 3 * (size_t)RC * RC; }

__global__ void __launch_bounds__(DD_THREADS) k_sstep_adv(Problem P, PhaseBufs B, int axis,
                                                          int s, int CL) {
  extern __shared__ double sh[];
  const int k = blockIdx.x / CL, cr = blockIdx.x - k * CL, RC = P.g.RC;
  const int rt = B.rt[k];
  const int rpb = (rt + CL - 1) / CL;
  const int i0 = min(rt, cr * rpb), i1 = min(rt, i0 + rpb), nr = i1 - i0;
  const int nst = P.integrator == 1 ? 4 : 1;
  double* Ss = sh;                                   // full stage value (rows < rt)
  double* U1 = Ss + RC * RC;                         // rows i0..i1 (local index)
  double* U2 = U1 + rpb * RC;
  const double* S1 = SMB(B, P, k, SM_S1);
  const double* Sin = s == 0 ? S1 : SMB(B, P, k, (s & 1) ? SM_S3T : SM_UB);
  double* Sout = SMB(B, P, k, (s & 1) ? SM_UB : SM_S3T);
  double* Ac = SMB(B, P, k, SM_VB);
  const double* T = SMB(B, P, k, SM_T);
  const double* Glo = SMB(B, P, k, SM_G_LO);
  const double* Ghi = SMB(B, P, k, SM_G_HI);
  const double* Cp = SMB(B, P, k, SM_CP);
  const double* Cn = SMB(B, P, k, SM_CM);
  const double* Ca = SMB(B, P, k, SM_CABS);
  for (int e = threadIdx.x; e < rt * RC; e += blockDim.x) Ss[e] = Sin[e];
  __syncthreads();
  for (int e = threadIdx.x; e < nr * rt; e += blockDim.x) {
    const int li = e / rt, j = e - li * rt, i = i0 + li;
    double a1 = Glo[i * RC + j], a2 = Ghi[i * RC + j];
    for (int l = 0; l < rt; ++l) {
      a1 += T[i * RC + l] * Ss[l * RC + j];
      a2 += T[l * RC + i] * Ss[l * RC + j];
    }
    U1[li * RC + j] = a1; U2[li * RC + j] = a2;
  }
  __syncthreads();
  const double coef = P.c_adv / (axis == 0 ? P.g.hxk[k] : P.g.hyk[k]);
  const double dtk = P.g.dtk[k];
  const double bs = (nst == 4) ? c_rk_b[s] : 1.0;
  const double an = (s + 1 < nst) ? c_rk_a[s + 1] : 0.0;
  double* S2 = SMB(B, P, k, SM_S2);
  for (int e = threadIdx.x; e < nr * rt; e += blockDim.x) {
    const int li = e / rt, j = e - li * rt, i = i0 + li;
    double f = 0.0;
    for (int l = 0; l < rt; ++l)
      f += Ss[i * RC + l] * Ca[l * RC + j] - U1[li * RC + l] * Cp[l * RC + j] + U2[li * RC + l] * Cn[l * RC + j];
    f = coef * f;
    const double acc = (s == 0 ? 0.0 : Ac[i * RC + j]) + bs * f;
    if (s + 1 < nst) {
      Ac[i * RC + j] = acc;
      Sout[i * RC + j] = S1[i * RC + j] + an * dtk * f;
    } else {
      S2[i * RC + j] = S1[i * RC + j] + dtk * acc;
    }
  }
  if (s + 1 == nst) {                                // L-step matrices and zero padding
    double* Ap = SMB(B, P, k, SM_AP);
    double* Am = SMB(B, P, k, SM_AM);
    for (int e = threadIdx.x; e < nr * RC; e += blockDim.x) {
      const int li = e / RC, j = e - li * RC, i = i0 + li;
      const bool in = j < rt;
      if (!in) S2[i * RC + j] = 0.0;
      Ap[i * RC + j] = in ? ((i == j ? 1.0 : 0.0) - T[i * RC + j]) : 0.0;
      Am[i * RC + j] = in ? (T[j * RC + i] - (i == j ? 1.0 : 0.0)) : 0.0;
    }
    if (cr == 0)
      for (int e = rt * RC + threadIdx.x; e < RC * RC; e += blockDim.x) {
        S2[e] = 0.0; Ap[e] = 0.0; Am[e] = 0.0;
      }
  }
}

// ---------------------------------------------------------------------------
// L-step of the advection with explicit Euler as products over all directions.  The
// Euler step of direction q's ODE is L_q = S2 v_q + dt kappa_q (A_s S2 v_q + g_q), with s
// the upwind side of Omega_q, g_q = -G_lo v_q (Omega_q > 0) or G_hi v_q (Omega_q < 0) and
// kappa_q = -c Omega_q / h.  With W_+ = A_+ S2 - G_lo and W_- = A_- S2 + G_hi it is
// L_q = S2 v_q + dt kappa_q W_s v_q: the tall product L = V S2^T over the direction rows,
// then L += diag(rs_+) V W_+^T and L += diag(rs_-) V W_-^T with rs_s,q = dt kappa_q on the
// directions of side s and 0 on the others (the Ozaki products' accumulating epilogue, FP64
// accumulation).  The arithmetic is that of k_lstep_adv's FP64 form but for the association
// ((A S2) v instead of A (S2 v), (dt kappa) y instead of dt (kappa y)); the reduced-precision
// forms take it too (FP64-accurate, and faster than their FP32 stages).
// k_lstep_w: blockIdx.x = 0 writes W_+^T (slot VB), S2^T (slot UB) and rs_+, 1 writes W_-^T
// (slot S3T) and rs_-; the three slots are free between the S-step and the truncation.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(DD_THREADS) k_lstep_w(Problem P, PhaseBufs B, int axis,
                                                        double* rs) {
  __shared__ double s2[DD_MAXC * DD_MAXC];
  const int k = blockIdx.y, side = blockIdx.x, RC = P.g.RC, rt = B.rt[k];
  const double* S2 = SMB(B, P, k, SM_S2);
  for (int e = threadIdx.x; e < rt * RC; e += blockDim.x) s2[e] = S2[e];
  __syncthreads();
  const double* A = SMB(B, P, k, side ? SM_AM : SM_AP);
  const double* G = SMB(B, P, k, side ? SM_G_HI : SM_G_LO);
  const double gs = side ? 1.0 : -1.0;
  double* Wt = SMB(B, P, k, side ? SM_S3T : SM_VB);
  double* St = SMB(B, P, k, SM_UB);
  for (int e = threadIdx.x; e < RC * RC; e += blockDim.x) {
    const int i = e / RC, j = e - i * RC;            // W[i][j] -> Wt[j][i]
    double w = 0.0;
    if (i < rt && j < rt) {
      for (int l = 0; l < rt; ++l) w += A[i * RC + l] * s2[l * RC + j];
      w += gs * G[i * RC + j];
    }
    Wt[j * RC + i] = w;
    if (side == 0) St[j * RC + i] = (i < rt && j < rt) ? s2[i * RC + j] : 0.0;
  }
  // row scales dt kappa_q of this side's directions (kappa_q = -c Omega_q / h), 0 elsewhere
  const int n = P.g.n;
  const double* om = axis == 0 ? P.ox : P.oy;
  const double hinv = 1.0 / (axis == 0 ? P.g.hxk[k] : P.g.hyk[k]), dt = P.g.dtk[k];
  double* r = rs + ((long)side * P.g.nsub + k) * n;
  for (int q = threadIdx.x; q < n; q += blockDim.x) {
    const double oq = om[q];
    const bool mine = side ? oq < 0.0 : oq > 0.0;
    r[q] = mine ? dt * (-P.c_adv * oq * hinv) : 0.0;
  }
}

// ---------------------------------------------------------------------------
// L-step of the advection: every direction is an independent r_t-dimensional
// linear ODE; one warp per direction, all RK stages fused.  In FP32 (TC = float) the
// first-stage right-hand side a0 = g + A L0 is formed in FP64 (the interior and ghost
// terms are large and cancel where a direction's flux through the subdomain is nearly
// balanced) and the later stages add only A times the stage increment, so FP32 rounds
// no term larger than the result it contributes to.
// ---------------------------------------------------------------------------
template <typename TC>
__global__ void __launch_bounds__(DD_THREADS) k_lstep_adv(Problem P, PhaseBufs B, int axis) {
  extern __shared__ double sh_raw[];
  TC* sh = reinterpret_cast<TC*>(sh_raw);
  const int k = blockIdx.y, RC = P.g.RC, n = P.g.n;
  const int rt = B.rt[k];
  TC* S2 = sh;
  TC* Ap = S2 + RC * RC;
  TC* Am = Ap + RC * RC;
  TC* Glo = Am + RC * RC;
  TC* Ghi = Glo + RC * RC;
  TC* wsp = Ghi + RC * RC;          // per warp: vh, L0, Ls, g  (4*RC)
  double* S2d = sh_raw + 5 * RC * RC + 8 * 4 * RC;   // FP64 copy for the start value
  double* vhd = S2d + RC * RC;                         // per warp: FP64 vh (RC)
  constexpr bool f32 = sizeof(TC) == sizeof(float);
  for (int e = threadIdx.x; e < RC * RC; e += blockDim.x) {
    S2d[e] = SMB(B, P, k, SM_S2)[e];
    S2[e] = SMB(B, P, k, SM_S2)[e];
    Ap[e] = SMB(B, P, k, SM_AP)[e];
    Am[e] = SMB(B, P, k, SM_AM)[e];
    Glo[e] = SMB(B, P, k, SM_G_LO)[e];
    Ghi[e] = SMB(B, P, k, SM_G_HI)[e];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  TC* vh = wsp + warp * 4 * RC;
  TC* L0 = vh + RC;
  TC* Ls = L0 + RC;
  TC* gv = Ls + RC;
  double* vw = vhd + warp * RC;
  double* l0w = vhd + (8 + warp) * RC;                 // per warp: FP64 L0 (FP32 form)
  const double* om = axis == 0 ? P.ox : P.oy;
  const TC dt = (TC)P.g.dtk[k];
  const TC hinv = (TC)(1.0 / (axis == 0 ? P.g.hxk[k] : P.g.hyk[k]));
  const int nst = P.integrator == 1 ? 4 : 1;
  count_work(P.g, KS_LSTEP_ADV, (double)max(0, min(n, (int)(blockIdx.x + 1) * 32) - (int)blockIdx.x * 32) *
                                    rt * rt * (4.0 + 2.0 * nst));
  for (int q = blockIdx.x * 32 + warp; q < min(n, (int)(blockIdx.x + 1) * 32); q += nw) {
    const double* Vq = B.Vh + ((long)k * n + q) * RC;
    for (int t = lane; t < RC; t += 32) {
      vh[t] = t < rt ? Vq[t] : 0.0;
      vw[t] = t < rt ? Vq[t] : 0.0;
    }
    __syncwarp();
    const TC oq = om[q];
    const TC* A = oq > 0.0 ? Ap : Am;
    const TC kap = (TC)(-P.c_adv) * oq * hinv;
    TC accv[2] = {0.0, 0.0}, l0v[2] = {0.0, 0.0};
    double l0d[2] = {0.0, 0.0};
    for (int h = 0; h < 2; ++h) {
      int i = lane + 32 * h;
      if (i < rt) {
        TC gg = 0.0;
        double sd = 0.0;
        for (int j = 0; j < rt; ++j) {
          sd += S2d[i * RC + j] * vw[j];
          if (oq > 0.0) gg -= Glo[i * RC + j] * vh[j];
          else if (oq < 0.0) gg += Ghi[i * RC + j] * vh[j];
        }
        const TC s = (TC)sd;
        L0[i] = s; Ls[i] = s; gv[i] = gg; l0v[h] = s; l0d[h] = sd;
        if (f32) l0w[i] = sd;
      }
    }
    __syncwarp();
    if (f32 && oq != 0.0) {
      // a0 = g + A L0 in FP64 into gv; Ls holds the stage increment (0 at stage 0)
      const double* A64 = SMB(B, P, k, oq > 0.0 ? SM_AP : SM_AM);
      const double* G64 = SMB(B, P, k, oq > 0.0 ? SM_G_LO : SM_G_HI);
      const double gs = oq > 0.0 ? -1.0 : 1.0;
      for (int h = 0; h < 2; ++h) {
        int i = lane + 32 * h;
        if (i < rt) {
          double g64 = 0.0, a64 = 0.0;
          for (int j = 0; j < rt; ++j) {
            g64 += G64[i * RC + j] * vw[j];
            a64 += A64[i * RC + j] * l0w[j];
          }
          gv[i] = (TC)(gs * g64 + a64);
          Ls[i] = 0;
        }
      }
      __syncwarp();
    }
    if (oq != 0.0) {
      for (int s = 0; s < nst; ++s) {
        TC kv[2] = {0.0, 0.0};
        for (int h = 0; h < 2; ++h) {
          int i = lane + 32 * h;
          if (i < rt) {
            TC a = gv[i];
            for (int j = 0; j < rt; ++j) a += A[i * RC + j] * Ls[j];
            kv[h] = kap * a;
          }
        }
        __syncwarp();
        const TC bs = (nst == 4) ? c_rk_b[s] : 1.0;
        const TC an = (s + 1 < nst) ? c_rk_a[s + 1] : 0.0;
        for (int h = 0; h < 2; ++h) {
          int i = lane + 32 * h;
          if (i < rt) {
            accv[h] += bs * kv[h];
            if (s + 1 < nst) Ls[i] = f32 ? an * dt * kv[h] : l0v[h] + an * dt * kv[h];
          }
        }
        __syncwarp();
      }
    }
    double* Lq = B.L + ((long)k * n + q) * RC;
    for (int h = 0; h < 2; ++h) {
      int i = lane + 32 * h;
      if (i < RC) Lq[i] = i < rt ? l0d[h] + (double)(dt * accv[h]) : 0.0;
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// truncation (Algorithm 5): SVD of S3 by one-sided Jacobi on the columns of S3^T
// ---------------------------------------------------------------------------
__global__ void k_trunc(Problem P, PhaseBufs B) {
  extern __shared__ double sh[];
  const int k = blockIdx.x, RC = P.g.RC;
  const int rt = B.rt[k];
  double* Bc = sh;                 // column-major, column j = column j of S3^T = row j of S3
  double* Jc = Bc + RC * RC;       // column-major rotations
  double* sig = Jc + RC * RC;
  double* X = sig + RC;            // scratch of the mixed-precision SVD
  int* perm = reinterpret_cast<int*>(X + (jacobi_mixed_scratch_bytes(RC) + 7) / 8);
  int* iv = perm + RC;
  const double* S3T = SMB(B, P, k, SM_S3T);
  for (int e = threadIdx.x; e < RC * RC; e += blockDim.x) {
    int col = e / RC, row = e % RC;
    // B = S3^T: B[row][col] = S3T[row][col]
    Bc[col * RC + row] = (row < rt && col < rt) ? S3T[row * RC + col] : 0.0;
    Jc[col * RC + row] = (row == col) ? 1.0 : 0.0;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  jacobi_svd_mixed(Bc, Jc, rt, RC, &iv[0], sig, X);
  for (int j = warp; j < rt; j += nwarps) {
    double s = 0.0;
    for (int l = lane; l < rt; l += 32) s += Bc[j * RC + l] * Bc[j * RC + l];
    s = warp_sum(s);
    if (lane == 0) {
      sig[j] = sqrt(s);
      if (!isfinite(sig[j])) atomicOr(B.status, (unsigned)ST_NONFINITE);
    }
  }
  __syncthreads();
  rank_sort_desc(sig, rt, perm);
  __syncthreads();
  if (threadIdx.x == 0) {
    int p = 0;
    double s1 = rt > 0 ? sig[perm[0]] : 0.0;
    if (s1 > 0.0)
      for (int t = 0; t < rt; ++t)
        if (sig[perm[t]] > P.tau * s1) ++p;
    int r1;
    if (P.rank_mode == 1) {
      int rtail = rt;
      for (int rr = 0; rr <= rt; ++rr) {
        double ss = 0.0;
        for (int t = rr; t < rt; ++t) ss += sig[perm[t]] * sig[perm[t]];
        if (sqrt(ss) <= P.tol) { rtail = rr; break; }
      }
      r1 = min(max(rtail, P.g.rlo[k]), P.g.rhi[k]);
    } else {
      r1 = P.g.rhi[k];
    }
    r1 = min(r1, p);
    iv[1] = r1;
    B.ro[k] = r1;
  }
  __syncthreads();
  const int r1 = iv[1];
  // S3 = J diag(sig) W^T with W = B J / sig: U_bar = J, V_bar = (B J)/sig
  double* Ub = SMB(B, P, k, SM_UB);
  double* Vb = SMB(B, P, k, SM_VB);
  double* So = B.So + (long)k * RC * RC;
  for (int e = threadIdx.x; e < RC * RC; e += blockDim.x) {
    int i = e / RC, t = e % RC;
    double u = 0.0, v = 0.0;
    if (i < rt && t < r1) {
      int c = perm[t];
      u = Jc[c * RC + i];
      v = Bc[c * RC + i] / sig[c];
    }
    Ub[e] = u; Vb[e] = v;
    So[e] = (i == t && t < r1) ? sig[perm[t]] : 0.0;
  }
}

// ---------------------------------------------------------------------------
// conserved-moment correction (optional; not part of the paper's scheme)
// ---------------------------------------------------------------------------
// mvec[k] = S (V^T sqrt(w)) over the first cnt[k] columns (S null: the identity):
// with it, the scalar flux of X S V^T (or of K V^T) is X mvec / sqrt(hx hy).
__global__ void k_mf_vec(Problem P, const double* V, const double* S, const int* cnt,
                         double* mvec) {
  __shared__ double a[DD_MAXC];
  const int k = blockIdx.x, RC = P.g.RC, n = P.g.n, c = cnt[k];
  const double* Vk = V + (long)k * n * RC;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int t = warp; t < RC; t += nw) {
    double x = 0.0;
    if (t < c)
      for (int q = lane; q < n; q += 32) x += Vk[(long)q * RC + t] * P.sw[q];
    x = warp_sum(x);
    if (lane == 0) a[t] = x;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < RC; i += blockDim.x) {
    double x = 0.0;
    if (i < c) {
      if (S) {
        const double* Sk = S + (long)k * RC * RC;
        for (int t = 0; t < c; ++t) x += Sk[i * RC + t] * a[t];
      } else {
        x = a[i];
      }
    }
    mvec[(long)k * RC + i] = x;
  }
}

// dm[cell] += sign * (A[cell, :cnt] . mvec[k]) / sqrt(hx hy)
__global__ void k_mf_acc(Problem P, const double* A, const int* cnt, const double* mvec,
                         double sign, double* dm) {
  const int k = blockIdx.y, RC = P.g.RC, N = P.g.N[k], c = cnt[k];
  const long rb = P.g.rowoff[k];
  const double* v = mvec + (long)k * RC;
  const double f = sign / P.g.shk[k];
  for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < N; row += gridDim.x * blockDim.x) {
    double x = 0.0;
    for (int t = 0; t < c; ++t) x += A[(rb + row) * RC + t] * v[t];
    dm[rb + row] += f * x;
  }
}

// K_a = [X S | sqrt(hx hy) dm] (the isotropic term's spatial factor), then dm = 0
__global__ void k_mf_build_x(Problem P, const double* X, const double* S, const int* r,
                             double* dm, double* Ka) {
  const int k = blockIdx.y, RC = P.g.RC, N = P.g.N[k], rk = r[k];
  const long rb = P.g.rowoff[k];
  const double* Sk = S + (long)k * RC * RC;
  for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < N; row += gridDim.x * blockDim.x) {
    const double* Xr = X + (rb + row) * RC;
    double* Kr = Ka + (rb + row) * RC;
    for (int t = 0; t < RC; ++t) {
      double x = 0.0;
      if (t < rk) {
        for (int u = 0; u < rk; ++u) x += Xr[u] * Sk[u * RC + t];
      } else if (t == rk) {
        x = P.g.shk[k] * dm[rb + row];
      }
      Kr[t] = x;
    }
    dm[rb + row] = 0.0;
  }
}

// V_a = [V | sqrt(w) / |S|] (the isotropic term's angular factor), m = r + 1
__global__ void k_mf_build_v(Problem P, const double* V, const int* r, double* Va, int* m) {
  const int k = blockIdx.y, RC = P.g.RC, n = P.g.n, rk = r[k];
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x)
    for (int t = 0; t < RC; ++t)
      Va[((long)k * n + q) * RC + t] =
          t < rk ? V[((long)k * n + q) * RC + t] : (t == rk ? P.sw[q] / P.ssum : 0.0);
  if (blockIdx.x == 0 && threadIdx.x == 0) m[k] = rk + 1;
}

// ---------------------------------------------------------------------------
// collision (Algorithm 3)
// ---------------------------------------------------------------------------
__global__ void k_coll_rank(Problem P, const int* r, int* rc) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= P.g.nsub) return;
  rc[k] = min(min(max(r[k], P.g.rlo[k]), P.g.n), P.g.N[k]);
}

// a = Vh^T sqrt(w)  (the paper's <V_j>_phi)
__global__ void k_coll_a(Problem P, PhaseBufs B) {
  const int k = blockIdx.x, RC = P.g.RC, n = P.g.n;
  const int rc = B.rc[k];
  __shared__ double red[40];
  double* vec = SMB(B, P, k, SM_VEC);
  for (int t = 0; t < RC; ++t) {
    double s = 0.0;
    if (t < rc)
      for (int q = threadIdx.x; q < n; q += blockDim.x) s += B.Vh[((long)k * n + q) * RC + t] * P.sw[q];
    s = block_sum(s, red);
    if (threadIdx.x == 0) vec[t] = s;
  }
}

// row-local collision K-step: dK_c/dt = (sig_s/|S|)(K_c . a) a - sig_t K_c + sQ_c a
template <typename TC>
__global__ void k_coll_kstep(Problem P, PhaseBufs B) {
  const int k = blockIdx.y, RC = P.g.RC;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int N = P.g.N[k], rc = B.rc[k];
  const double* a = SMB(B, P, k, SM_VEC);
  const TC dt = (TC)P.g.dtk[k];
  const int nst = P.integrator == 1 ? 4 : 1;
  // a cell per W lanes (W the power of two >= r_c, up to 32), G = 32 / W cells per warp: FP64
  // instructions hold the pipe whether or not their lanes are active.  The dot product's
  // butterfly over W lanes is the full warp's with the steps that add zero lanes left out.
  int W = 1;
  while (W < rc && W < 32) W <<= 1;
  const int G = 32 / W, slot = lane / W, tl = lane - slot * W;
  {
    double cells = 0.0;
    for (long c0 = (long)blockIdx.x * nw * G; c0 < N; c0 += (long)gridDim.x * nw * G)
      cells += (double)min((long)nw * G, (long)N - c0);
    count_work(P.g, KS_COLL_KSTEP, cells * rc * 6.0 * nst);
  }
  for (int c0 = (blockIdx.x * nw + warp) * G; c0 < N; c0 += gridDim.x * nw * G) {
    const int cell = c0 + slot;
    const bool valid = cell < N;
    const long row = (long)P.g.rowoff[k] + (valid ? cell : c0);
    const TC ss = (TC)(P.sig_s[row] / P.ssum), st = (TC)P.sig_t[row], sq = (TC)P.sQ[row];
    TC k0[2], ks[2], acc[2] = {0.0, 0.0}, av[2];
    double k0d[2];
    for (int h = 0; h < 2; ++h) {
      int t = tl + 32 * h;
      k0d[h] = (valid && t < rc) ? B.K[row * RC + t] : 0.0;
      k0[h] = (TC)k0d[h];
      av[h] = t < rc ? a[t] : 0.0;
      ks[h] = k0[h];
    }
    // the upper half of the columns only where r_c > 32
    const int nh = rc > 32 ? 2 : 1;
    for (int s = 0; s < nst; ++s) {
      TC d = ks[0] * av[0];
      if (nh > 1) d += ks[1] * av[1];
      for (int o = W >> 1; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
      TC kv[2] = {0.0, 0.0};
      for (int h = 0; h < nh; ++h) kv[h] = ss * d * av[h] - st * ks[h] + sq * av[h];
      const TC bs = (nst == 4) ? c_rk_b[s] : 1.0;
      const TC an = (s + 1 < nst) ? c_rk_a[s + 1] : 0.0;
      for (int h = 0; h < nh; ++h) {
        acc[h] += bs * kv[h];
        ks[h] = k0[h] + an * dt * kv[h];
      }
    }
    if (valid)
      for (int t = tl; t < RC; t += W) {
        const int h = t >> 5;
        B.K[row * RC + t] = t < rc ? k0d[h] + (double)(dt * acc[h]) : 0.0;
      }
  }
}

// The collision K-step with explicit Euler in FP64, a thread per cell (the warp form above
// issues its FP64 instructions for one cell at a time, and a warp instruction holds the FP64
// pipe however many of its lanes are active): K_c <- K_c + dt ((sig_s/|S|)(K_c . a) a
// - sig_t K_c + sQ_c a) on the first r_c columns, zero beyond.
__global__ void __launch_bounds__(DD_THREADS) k_coll_kstep1(Problem P, PhaseBufs B) {
  __shared__ double av[DD_MAXC];
  const int k = blockIdx.y, RC = P.g.RC, N = P.g.N[k], rc = B.rc[k];
  const double* a = SMB(B, P, k, SM_VEC);
  for (int t = threadIdx.x; t < RC; t += blockDim.x) av[t] = t < rc ? a[t] : 0.0;
  __syncthreads();
  const int c0 = blockIdx.x * blockDim.x;
  if (c0 >= N) return;
  count_work(P.g, KS_COLL_KSTEP, (double)min((int)blockDim.x, N - c0) * rc * 6.0);
  const int cell = c0 + threadIdx.x;
  if (cell >= N) return;
  const long row = (long)P.g.rowoff[k] + cell;
  const double ss = P.sig_s[row] / P.ssum, st = P.sig_t[row], sq = P.sQ[row];
  const double dt = P.g.dtk[k];
  double* Kr = B.K + row * RC;
  double d = 0.0;
  for (int t = 0; t < rc; ++t) d += Kr[t] * av[t];
  for (int t = 0; t < RC; ++t) {
    const double k0 = Kr[t];
    Kr[t] = t < rc ? k0 + dt * (ss * d * av[t] - st * k0 + sq * av[t]) : 0.0;
  }
}

// The collision L-step with explicit Euler in FP64, a thread per direction row (the warp
// form below issues its FP64 instructions for one direction at a time, and a warp
// instruction holds the FP64 pipe however many lanes are active): L0 = S2 v,
// a = sw b_0 - Mt L0, L = L0 + dt a, every sum in the warp form's order (bitwise the same).
// Dynamic shared memory: S2 and Mt (r_c rows each), b_0, and each thread's L0 (entry j of
// thread t at j blockDim + t).
size_t coll_lstep1_smem(int RC) { return sizeof(double) * (2 * RC * RC + RC + DD_THREADS * RC); }
__global__ void __launch_bounds__(DD_THREADS) k_coll_lstep1(Problem P, PhaseBufs B) {
  extern __shared__ double sc1[];
  const int k = blockIdx.y, RC = P.g.RC, n = P.g.n, rc = B.rc[k], T = blockDim.x;
  double* S2 = sc1;
  double* Mt = S2 + rc * RC;
  double* b0 = Mt + rc * RC;
  double* L0 = b0 + RC;
  for (int e = threadIdx.x; e < rc * RC; e += T) {
    S2[e] = SMB(B, P, k, SM_S2)[e];
    Mt[e] = SMB(B, P, k, SM_MT)[e];
  }
  for (int i = threadIdx.x; i < RC; i += T) b0[i] = SMB(B, P, k, SM_VEC)[2 * RC + i];
  __syncthreads();
  const int q0 = blockIdx.x * T;
  if (q0 >= n) return;
  count_work(P.g, KS_COLL_LSTEP, (double)min(T, n - q0) * rc * rc * 4.0);
  const int q = q0 + threadIdx.x;
  if (q >= n) return;
  const double* Vq = B.Vh + ((long)k * n + q) * RC;
  double* Lq = B.L + ((long)k * n + q) * RC;
  double* l0 = L0 + threadIdx.x;
  for (int i = 0; i < rc; ++i) l0[i * T] = 0.0;
  for (int j = 0; j < rc; ++j) {                   // sd_i += S2_ij v_j, j ascending
    const double vj = Vq[j];
    for (int i = 0; i < rc; ++i) l0[i * T] += S2[i * RC + j] * vj;
  }
  const double swq = P.sw[q], dt = P.g.dtk[k];
  for (int i = 0; i < RC; ++i) {
    double out = 0.0;
    if (i < rc) {
      double a = swq * b0[i];
      for (int j = 0; j < rc; ++j) a -= Mt[i * RC + j] * l0[j * T];
      out = l0[i * T] + dt * a;
    }
    Lq[i] = out;
  }
}

// collision S-step and the stage values b_s of the L-step's direction mean
__global__ void k_coll_small(Problem P, PhaseBufs B) {
  extern __shared__ double sh[];
  const int k = blockIdx.x, RC = P.g.RC;
  const int rc = B.rc[k];
  double* vec = SMB(B, P, k, SM_VEC);   // row 0: a, row 1: q, rows 2..5: b stages
  const double* Ms = SMB(B, P, k, SM_MS);
  const double* Mt = SMB(B, P, k, SM_MT);
  double* S0 = sh;
  double* Ss = S0 + RC * RC;
  double* Ac = Ss + RC * RC;
  double* F = Ac + RC * RC;
  double* Wv = F + RC * RC;             // Ss a  (RC)
  double* mv = Wv + RC;                 // m stage (RC)
  double* m0 = mv + RC;
  double* km = m0 + RC;
  double* qv = km + RC;                 // q = X1^T sQ, column 0 of the scratch block
  const double* av = vec;
  const double iS = 1.0 / P.ssum;
  for (int i = threadIdx.x; i < RC; i += blockDim.x) qv[i] = i < rc ? SMB(B, P, k, SM_UB)[i * RC] : 0.0;
  for (int e = threadIdx.x; e < RC * RC; e += blockDim.x) {
    S0[e] = SMB(B, P, k, SM_S1)[e];
    Ss[e] = S0[e];
    Ac[e] = 0.0;
  }
  __syncthreads();
  const int nst = P.integrator == 1 ? 4 : 1;
  // S-step:  dS/dt = -[(1/|S|) Ms S a a^T - Mt S + q a^T]
  for (int s = 0; s < nst; ++s) {
    for (int i = threadIdx.x; i < rc; i += blockDim.x) {
      double w = 0.0;
      for (int j = 0; j < rc; ++j) w += Ss[i * RC + j] * av[j];
      Wv[i] = w;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < rc * rc; e += blockDim.x) {
      int i = e / rc, j = e % rc;
      double msw = 0.0, mts = 0.0;
      for (int l = 0; l < rc; ++l) {
        msw += Ms[i * RC + l] * Wv[l];
        mts += Mt[i * RC + l] * Ss[l * RC + j];
      }
      F[i * RC + j] = -(iS * msw * av[j] - mts + qv[i] * av[j]);
    }
    __syncthreads();
    const double bs = (nst == 4) ? c_rk_b[s] : 1.0;
    const double an = (s + 1 < nst) ? c_rk_a[s + 1] : 0.0;
    for (int e = threadIdx.x; e < rc * rc; e += blockDim.x) {
      int i = e / rc, j = e % rc;
      Ac[i * RC + j] += bs * F[i * RC + j];
      if (s + 1 < nst) Ss[i * RC + j] = S0[i * RC + j] + an * P.g.dtk[k] * F[i * RC + j];
    }
    __syncthreads();
  }
  double* S2 = SMB(B, P, k, SM_S2);
  for (int e = threadIdx.x; e < RC * RC; e += blockDim.x) {
    int i = e / RC, j = e % RC;
    S2[e] = (i < rc && j < rc) ? S0[e] + P.g.dtk[k] * Ac[e] : 0.0;
  }
  __syncthreads();
  // m0 = S2 a ; dm/dt = (Ms - Mt) m + |S| q ; b_s = (1/|S|) Ms m_s + q
  for (int i = threadIdx.x; i < rc; i += blockDim.x) {
    double w = 0.0;
    for (int j = 0; j < rc; ++j) w += S2[i * RC + j] * av[j];
    m0[i] = w; mv[i] = w;
  }
  __syncthreads();
  for (int s = 0; s < nst; ++s) {
    for (int i = threadIdx.x; i < rc; i += blockDim.x) {
      double bsv = qv[i], d = P.ssum * qv[i];
      for (int j = 0; j < rc; ++j) {
        bsv += iS * Ms[i * RC + j] * mv[j];
        d += (Ms[i * RC + j] - Mt[i * RC + j]) * mv[j];
      }
      vec[(2 + s) * RC + i] = bsv;
      km[i] = d;
    }
    __syncthreads();
    const double an = (s + 1 < nst) ? c_rk_a[s + 1] : 0.0;
    for (int i = threadIdx.x; i < rc; i += blockDim.x) mv[i] = m0[i] + an * P.g.dtk[k] * km[i];
    __syncthreads();
  }
}

// collision L-step per direction:  dL_q/dt = sqrt(w_q) b(t) - Mt L_q
template <typename TC>
__global__ void __launch_bounds__(DD_THREADS) k_coll_lstep(Problem P, PhaseBufs B) {
  extern __shared__ double sh_raw[];
  TC* sh = reinterpret_cast<TC*>(sh_raw);
  const int k = blockIdx.y, RC = P.g.RC, n = P.g.n;
  const int rc = B.rc[k];
  TC* S2 = sh;
  TC* Mt = S2 + RC * RC;
  TC* bst = Mt + RC * RC;         // 4 x RC
  TC* wsp = bst + 4 * RC;         // per warp: vh, Ls (2*RC)
  double* S2d = sh_raw + 2 * RC * RC + 4 * RC + 8 * 2 * RC;   // FP64 copy for the start value
  double* vhd = S2d + RC * RC;                                  // per warp: FP64 vh (RC)
  for (int e = threadIdx.x; e < RC * RC; e += blockDim.x) {
    S2d[e] = SMB(B, P, k, SM_S2)[e];
    S2[e] = SMB(B, P, k, SM_S2)[e];
    Mt[e] = SMB(B, P, k, SM_MT)[e];
  }
  for (int e = threadIdx.x; e < 4 * RC; e += blockDim.x) bst[e] = SMB(B, P, k, SM_VEC)[2 * RC + e];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  TC* vh = wsp + warp * 2 * RC;
  TC* Ls = vh + RC;
  double* vw = vhd + warp * RC;
  const int nst = P.integrator == 1 ? 4 : 1;
  const TC dt = (TC)P.g.dtk[k];
  count_work(P.g, KS_COLL_LSTEP, (double)max(0, min(n, (int)(blockIdx.x + 1) * 32) - (int)blockIdx.x * 32) *
                                     rc * rc * (2.0 + 2.0 * nst));
  for (int q = blockIdx.x * 32 + warp; q < min(n, (int)(blockIdx.x + 1) * 32); q += nw) {
    const double* Vq = B.Vh + ((long)k * n + q) * RC;
    for (int t = lane; t < RC; t += 32) {
      vh[t] = t < rc ? Vq[t] : 0.0;
      vw[t] = t < rc ? Vq[t] : 0.0;
    }
    __syncwarp();
    const TC swq = P.sw[q];
    TC l0v[2] = {0.0, 0.0}, accv[2] = {0.0, 0.0};
    double l0d[2] = {0.0, 0.0};
    for (int h = 0; h < 2; ++h) {
      int i = lane + 32 * h;
      if (i < rc) {
        double sd = 0.0;
        for (int j = 0; j < rc; ++j) sd += S2d[i * RC + j] * vw[j];
        l0v[h] = (TC)sd; Ls[i] = (TC)sd; l0d[h] = sd;
      }
    }
    __syncwarp();
    for (int s = 0; s < nst; ++s) {
      TC kv[2] = {0.0, 0.0};
      for (int h = 0; h < 2; ++h) {
        int i = lane + 32 * h;
        if (i < rc) {
          TC a = swq * bst[s * RC + i];
          for (int j = 0; j < rc; ++j) a -= Mt[i * RC + j] * Ls[j];
          kv[h] = a;
        }
      }
      __syncwarp();
      const TC bs = (nst == 4) ? c_rk_b[s] : 1.0;
      const TC an = (s + 1 < nst) ? c_rk_a[s + 1] : 0.0;
      for (int h = 0; h < 2; ++h) {
        int i = lane + 32 * h;
        if (i < rc) {
          accv[h] += bs * kv[h];
          if (s + 1 < nst) Ls[i] = l0v[h] + an * dt * kv[h];
        }
      }
      __syncwarp();
    }
    double* Lq = B.L + ((long)k * n + q) * RC;
    for (int h = 0; h < 2; ++h) {
      int i = lane + 32 * h;
      if (i < RC) Lq[i] = i < rc ? l0d[h] + (double)(dt * accv[h]) : 0.0;
    }
    __syncwarp();
  }
}

// S_out = (S3^T)^T, rank = r_c
__global__ void k_coll_final(Problem P, PhaseBufs B) {
  const int k = blockIdx.x, RC = P.g.RC;
  const int rc = B.rc[k];
  const double* S3T = SMB(B, P, k, SM_S3T);
  double* So = B.So + (long)k * RC * RC;
  for (int e = threadIdx.x; e < RC * RC; e += blockDim.x) {
    int i = e / RC, j = e % RC;
    So[e] = (i < rc && j < rc) ? S3T[j * RC + i] : 0.0;
  }
  if (threadIdx.x == 0) B.ro[k] = rc;
}

// ---------------------------------------------------------------------------
// scalar flux  rho_c = X_c (S a) / sqrt(hx hy),  a = Vt^T sqrt(w)
// ---------------------------------------------------------------------------
__global__ void k_flux_prep(Problem P, const double* V, const double* S, const int* r, double* work) {
  const int k = blockIdx.x, RC = P.g.RC, n = P.g.n;
  const int rk = r[k];
  __shared__ double red[40];
  __shared__ double av[DD_MAXC];
  for (int t = 0; t < rk; ++t) {
    double s = 0.0;
    for (int q = threadIdx.x; q < n; q += blockDim.x) s += V[((long)k * n + q) * RC + t] * P.sw[q];
    s = block_sum(s, red);
    if (threadIdx.x == 0) av[t] = s;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < RC; i += blockDim.x) {
    double s = 0.0;
    if (i < rk)
      for (int j = 0; j < rk; ++j) s += S[(long)k * RC * RC + i * RC + j] * av[j];
    work[(long)k * RC + i] = s;
  }
}

__global__ void k_flux(Problem P, const double* X, const int* r, const double* work, double* rho,
                       int nx) {
  const int k = blockIdx.y, RC = P.g.RC;
  const int N = P.g.N[k], rk = r[k], nxk = P.g.nxk[k];
  const double* sa = work + (long)k * RC;
  for (int cell = blockIdx.x * blockDim.x + threadIdx.x; cell < N; cell += gridDim.x * blockDim.x) {
    const double* Xr = X + ((long)P.g.rowoff[k] + cell) * RC;
    double s = 0.0;
    for (int t = 0; t < rk; ++t) s += Xr[t] * sa[t];
    int il = cell % nxk, jl = cell / nxk;
    rho[(long)P.g.fbase[k] + (long)(P.g.cy0[k] + jl) * P.g.fnx[k] + P.g.cx0[k] + il] = s / P.g.shk[k];
  }
}

// TC working set plus an FP64 copy of S2 and one FP64 vh per warp
size_t lstep_smem(int RC) {
  return sizeof(double) * (5 * RC * RC + 8 * 4 * RC + RC * RC + 2 * 8 * RC);
}

size_t coll_lstep_smem(int RC) {
  return sizeof(double) * (2 * RC * RC + 4 * RC + 8 * 2 * RC + RC * RC + 8 * RC);
}

size_t trunc_smem(int RC) {
  return sizeof(double) * (2 * RC * RC + RC) + 8 * ((jacobi_mixed_scratch_bytes(RC) + 7) / 8) +
         sizeof(int) * (RC + 8);
}

size_t kstep_smem(const Problem& P, int lpb, int len) {
  const int RC = P.g.RC;
  return sizeof(double) * (3 * RC * RC + 2 * lpb * RC + (size_t)lpb * len * RC);
}

size_t kstep_eig_smem(const Problem& P, int lpb, int len) {
  const int RC = P.g.RC;
  return sizeof(double) * ((size_t)RC * RC + 2 * RC + 2 * lpb * RC + (size_t)lpb * len * RC);
}

int kstep_eig_lpb(const Problem& P, int len) {
  const int RC = P.g.RC;
  int lpb = max(1, (DD_THREADS * KE_EPT) / (len * RC));
  while (lpb > 1 && kstep_eig_smem(P, lpb, len) > 200 * 1024) --lpb;
  const long lines = (long)P.maxlines * P.g.nsub;
  while (lpb > 1 && (lines + lpb - 1) / lpb < 2L * P.nsm) --lpb;
  return lpb;
}

int kstep_lpb(const Problem& P, int len) {
  // lines per CTA: bounded by the register tile (KS_EPT per thread) and shared memory,
  // and small enough that the grid covers every SM about twice (the kernel is bound
  // by the FP64 pipe of the SMs it occupies)
  const int RC = P.g.RC;
  int lpb = max(1, (DD_THREADS * KS_EPT) / (len * RC));
  while (lpb > 1 && kstep_smem(P, lpb, len) > 200 * 1024) --lpb;
  const long lines = (long)P.maxlines * P.g.nsub;
  while (lpb > 1 && (lines + lpb - 1) / lpb < 2L * P.nsm) --lpb;
  return lpb;
}

}  // namespace

const char* const kSlotNames[NSLOT] = {
    "k_aug_cols", "k_build_L0", "k_geig(aug)", "k_ang_coeffs", "k_reduce", "k_small_adv1", "k_tall",
    "k_ghost", "k_kstep_adv", "k_sp_coeffs", "k_sstep_adv", "k_lstep_adv", "k_gram", "k_trunc",
    "k_coll_rank", "k_coll_a", "k_coll_kstep", "k_coll_small", "k_coll_lstep", "k_coll_final",
    "k_flux", "memcpy", "k_geig", "k_chol_inv", "k_complete", "k_mass_fix", "k_kc_w", "k_kc_sel",
    "k_kc_apply", "k_tc_tall", "k_tc_gram", "k_lstep_prod", "k_oz_tall", "k_oz_gram"};
thread_local Prof* g_prof = nullptr;

size_t part_elems(const Problem& P) {
  const int nc = P.nchunk_sp > P.nchunk_ang ? P.nchunk_sp : P.nchunk_ang;
  const size_t grams = (size_t)P.g.nsub * nc * 8 * P.g.RC * P.g.RC;
  const size_t kc = (size_t)P.g.nsub * kc_region(P.g.RC);   // the spatial completion's scratch
  return grams > kc ? grams : kc;
}

// Kernel attributes are per process, not per solver: they are set for the largest
// capacity (DD_MAXC) so that solvers of different widths can coexist.
cudaError_t phase_init() {
  const int RC = DD_MAXC;
  cudaError_t e;
  e = cudaFuncSetAttribute(k_kstep_adv<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 210 * 1024);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_kstep_adv<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 210 * 1024);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_kstep_eig<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 210 * 1024);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_sstep_adv, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)sstep_smem(RC));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_lstep_adv<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(lstep_smem(RC)));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_lstep_adv<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(lstep_smem(RC)));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_small_adv1, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)small_adv1_smem(RC));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_trunc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)trunc_smem(RC));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_coll_small, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(sizeof(double) * (4 * RC * RC + 5 * RC)));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_coll_lstep<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(coll_lstep_smem(RC)));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_coll_lstep1, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(coll_lstep1_smem(RC)));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_coll_lstep<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(coll_lstep_smem(RC)));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_build_L0, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(sizeof(double) * 3 * RC * RC));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_tall, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)tall_smem(RC, RC));
  return e;
}

// one thread per output element of the nblk small matrices of every subdomain
static dim3 reduce_grid(const Geo& g, int nblk) {
  return dim3((nblk * g.RC * g.RC + DD_THREADS - 1) / DD_THREADS, g.nsub);
}

static void gram(const Problem& P, const PhaseBufs& B, cudaStream_t st, int spatial,
                 const double* A, int lda, const int* acnt, int afix, const double* Bm, int ldb,
                 const int* bcnt, int bfix, int b_per_sub, const double* wrow, int dst_small) {
  GramArgs a;
  a.spatial = spatial; a.A = A; a.lda = lda; a.acnt = acnt; a.afix = afix;
  a.Bm = Bm; a.ldb = ldb; a.bcnt = bcnt; a.bfix = bfix; a.b_per_sub = b_per_sub;
  a.wrow = wrow; a.part = B.part; a.nchunk = spatial ? P.nchunk_sp : P.nchunk_ang;
  a.cexp = nullptr;
  a.sym = A == Bm && lda == ldb && acnt == bcnt && afix == bfix && b_per_sub;
  pbeg(st, KS_GRAM);
  k_gram<<<dim3(a.nchunk, P.g.nsub), DD_THREADS, sizeof(double) * P.g.RC * P.g.RC, st>>>(P.g, a);
  pend(st);
  Dst d;
  d.idx[0] = dst_small;
  pbeg(st, KS_REDUCE);
  k_reduce<<<reduce_grid(P.g, 1), DD_THREADS, 0, st>>>(B.part, a.nchunk, 1, d, B.sm, P.g.RC);
  pend(st);
}

// chunked Gram A^T A left as partial sums in B.part (summed by the consumer); returns
// the number of chunks
static int gram_partials(const Problem& P, const PhaseBufs& B, cudaStream_t st, int spatial,
                         const double* A, int lda, const int* acnt, int* cexp) {
  GramArgs a;
  a.spatial = spatial; a.A = A; a.lda = lda; a.acnt = acnt; a.afix = 0;
  a.Bm = A; a.ldb = lda; a.bcnt = acnt; a.bfix = 0; a.b_per_sub = 1;
  a.wrow = nullptr; a.part = B.part; a.nchunk = spatial ? P.ochunk_sp : P.ochunk_ang;
  a.cexp = cexp;
  a.sym = 1;
  if ((spatial ? P.ozg_sp : P.ozg_ang) &&
      oz_gram(P, B.status, st, spatial, A, lda, acnt, B.part, a.nchunk, cexp))
    return a.nchunk;
  pbeg(st, KS_GRAM);
  k_gram<<<dim3(a.nchunk, P.g.nsub), DD_THREADS, sizeof(double) * P.g.RC * P.g.RC, st>>>(P.g, a);
  pend(st);
  return a.nchunk;
}

// The same product on the tensor cores in the DD_TF32 / DD_BF16 forms (the Galerkin
// products: K0, the truncation's rotations, the collision's X S); FP64 otherwise, and for
// the orthonormalisation's products, which call tall() directly.
static void tall(const Problem& P, const PhaseBufs& B, cudaStream_t st, int spatial,
                 const double* A, int lda, const int* ninner, int ninner_fix, const double* Bm,
                 int bsmall, const int* ncols, int ncols_fix, double* Y, int ldy,
                 double* gpart = nullptr);
static void galerkin_tall(const Problem& P, const PhaseBufs& B, cudaStream_t st, int spatial,
                          const double* A, int lda, const int* ninner, const double* Bm,
                          int bsmall, const int* ncols, double* Y, int ldy) {
  if (P.prec >= PREC_TF32 && tc_tall(P, B.status, st, spatial, A, lda, ninner, 0, Bm, bsmall,
                                     B.sm, ncols, 0, Y, ldy, 1.0, 0))
    return;
  tall(P, B, st, spatial, A, lda, ninner, 0, Bm, bsmall, ncols, 0, Y, ldy);
}

static void tall(const Problem& P, const PhaseBufs& B, cudaStream_t st, int spatial,
                 const double* A, int lda, const int* ninner, int ninner_fix, const double* Bm,
                 int bsmall, const int* ncols, int ncols_fix, double* Y, int ldy,
                 double* gpart) {
  if ((spatial ? P.oz_sp : P.oz_ang) && !gpart &&
      oz_tall(P, B.status, st, spatial, A, lda, ninner, ninner_fix, Bm, bsmall,
                                B.sm, ncols, ncols_fix, Y, ldy))
    return;
  TallArgs a;
  a.spatial = spatial; a.A = A; a.lda = lda; a.ninner = ninner; a.ninner_fix = ninner_fix;
  a.Bm = Bm; a.bsmall = bsmall; a.ncols = ncols; a.ncols_fix = ncols_fix; a.Y = Y; a.ldy = ldy;
  a.gpart = gpart;
  const int rows = spatial ? P.maxN : P.g.n;
  dim3 grid((rows + TALL_ROWS - 1) / TALL_ROWS, P.g.nsub);
  pbeg(st, KS_TALL);
  k_tall<<<grid, DD_THREADS, tall_smem(P.g.RC, ldy), st>>>(P.g, a, B.sm);
  pend(st);
}

static TcGramSrc gsrc(const double* ptr, int ld, const int* cnt, int blk, int wsel = W_NONE,
                      const double* wrow = nullptr, int transpose = 0) {
  TcGramSrc s;
  s.ptr = ptr; s.ld = ld; s.cnt = cnt; s.fix = 0; s.nbside = -1; s.same_as_b = 0; s.shift = 0;
  s.wsel = wsel; s.wrow = wrow; s.blk = blk; s.transpose = transpose;
  return s;
}
static TcGram tgram(const Problem& P, const PhaseBufs& B, int spatial, int axis, const double* Bop,
                    const int* bcnt, int nchunk, int nblk) {
  TcGram a;
  a.g = P.g; a.spatial = spatial; a.axis = axis; a.B = Bop; a.ldb = P.g.RC; a.bcnt = bcnt;
  a.bfix = 0; a.nsrc = 0; a.part = B.part; a.nchunk = nchunk; a.nblk = nblk;
  a.ox = P.ox; a.oy = P.oy; a.status = B.status;
  return a;
}
static void reduce_to(const Problem& P, const PhaseBufs& B, cudaStream_t st, int nchunk, int nblk,
                      const Dst& d) {
  pbeg(st, KS_REDUCE);
  k_reduce<<<reduce_grid(P.g, nblk), DD_THREADS, 0, st>>>(B.part, nchunk, nblk, d, B.sm, P.g.RC);
  pend(st);
}

// ---------------------------------------------------------------------------------------
// Autotuner
// ---------------------------------------------------------------------------------------
// deterministic trial values in [-1, 1) (a multiplicative hash of the index)
__global__ void k_trial_fill(double* a, long n) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    a[i] = (double)((unsigned)(i * 2654435761ull) >> 8) * (1.0 / 8388608.0) - 1.0;
}

namespace {
struct TuneChoice {
  int oz_sp, oz_ang, nch_sp, nch_ang, ozg_sp, ozg_ang;
  double ms[8];
};
std::mutex g_tune_mu;
std::map<std::vector<long>, TuneChoice> g_tune_cache;

// average time of fn() on st over reps launches after one untimed call (ms; -1 on error)
template <class F>
double time_on(cudaStream_t st, int reps, F fn) {
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess) return -1.0;
  if (cudaEventCreate(&b) != cudaSuccess) { cudaEventDestroy(a); return -1.0; }
  fn();
  cudaEventRecord(a, st);
  for (int i = 0; i < reps; ++i) fn();
  cudaEventRecord(b, st);
  float t = -1.0f;
  const bool ok = cudaEventSynchronize(b) == cudaSuccess && cudaEventElapsedTime(&t, a, b) == cudaSuccess;
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return ok ? (double)t / reps : -1.0;
}
}  // namespace

cudaError_t autotune(Problem& P, const PhaseBufs& B, cudaStream_t st, int tune_products,
                     int tune_chunks, double* ms) {
  for (int i = 0; i < 8; ++i) ms[i] = -1.0;
  if (!tune_products && !tune_chunks) return cudaSuccess;
  const int RC = P.g.RC, nsub = P.g.nsub;
  const std::vector<long> key = {nsub, P.maxN, P.g.n, RC, P.prec, P.Ntot, tune_products,
                                 tune_chunks, P.ochunk_sp, P.ochunk_ang};
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      const TuneChoice& c = it->second;
      if (tune_products) {
        P.oz_sp = c.oz_sp; P.oz_ang = c.oz_ang; P.ozg_sp = c.ozg_sp; P.ozg_ang = c.ozg_ang;
      }
      if (tune_chunks) { P.ochunk_sp = c.nch_sp; P.ochunk_ang = c.nch_ang; }
      for (int i = 0; i < 8; ++i) ms[i] = c.ms[i];
      return cudaSuccess;
    }
  }
  // trial operands in the workspace: A = K (spatial) / L (angular), Y = Hw / Hwa, the
  // small matrices filled with trial values, every column count = RC (in keep)
  const long nsm_elems = (long)nsub * NSMALL * RC * RC;
  k_trial_fill<<<P.nsm * 4, 256, 0, st>>>(B.K, P.Ntot * RC);
  k_trial_fill<<<P.nsm * 4, 256, 0, st>>>(B.L, (long)nsub * P.g.n * RC);
  k_trial_fill<<<P.nsm * 4, 256, 0, st>>>(B.sm, nsm_elems);
  {
    std::vector<int> cnt(nsub, RC);
    cudaError_t e = cudaMemcpyAsync(B.keep, cnt.data(), sizeof(int) * nsub, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
  }
  const int REPS = 3;
  for (int sp = 1; sp >= 0; --sp) {
    const double* A = sp ? B.K : B.L;
    double* Y = sp ? B.Hw : B.Hwa;
    const int f = sp ? 0 : 1;
    if (tune_products) {
      // both engines at two column counts (half and full capacity).  The FP64 kernel also
      // forms the Gram of its output from the same tiles in the orthonormalisation (one of
      // its two products there): the tensor-core side is charged half a separate Gram
      // reduction per product.
      // The orthonormalisation's Gram engine (k_gram or k_oz_gram) is timed the same way
      // and the faster one kept (by 3%; k_gram on a tie).
      const int half = std::max(2, (RC / 2) & ~1);
      Problem Q = P;
      Q.oz_sp = Q.oz_ang = 0;
      Q.ozg_sp = Q.ozg_ang = 0;
      Problem Qg = Q;
      Qg.ozg_sp = Qg.ozg_ang = 1;
      auto gram_trial = [&](const Problem& R) {
        return time_on(st, REPS, [&] {
          const int n = gram_partials(R, B, st, sp, A, RC, B.keep, nullptr);
          Dst d;
          for (int i = 0; i < 8; ++i) d.idx[i] = SM_QM;
          reduce_to(R, B, st, n, 1, d);
        });
      };
      const double tg64 = gram_trial(Q), tgoz = gram_trial(Qg);
      const int gpick = tgoz > 0.0 && tg64 > 0.0 && tgoz < 0.97 * tg64 ? 1 : 0;
      if (sp) P.ozg_sp = gpick; else P.ozg_ang = gpick;
      const double tg = gpick ? tgoz : tg64;
      double t64 = 0.0, toz = tg > 0.0 ? tg : 0.0;
      bool oz_ok = true;
      for (int c : {half, RC}) {
        t64 += time_on(st, REPS, [&] {
          tall(Q, B, st, sp, A, RC, nullptr, c, nullptr, SM_QM, nullptr, c, Y, P.WC);
        });
        toz += time_on(st, REPS, [&] {
          oz_ok = oz_ok && oz_tall(P, B.status, st, sp, A, RC, nullptr, c, nullptr, SM_QM, B.sm,
                                   nullptr, c, Y, P.WC);
        });
      }
      ms[4 * f + 0] = t64;
      ms[4 * f + 1] = oz_ok ? toz : -1.0;
      const int pick = oz_ok && toz > 0.0 && toz < t64 ? 1 : 0;
      if (sp) P.oz_sp = pick; else P.oz_ang = pick;
    }
    if (tune_chunks) {
      // the orthonormalisations' Gram A^T A with its fixed-order reduction, at the
      // heuristic's chunk count and at a half and a quarter of it (the partials buffer is
      // sized for the heuristic's; the Galerkin products keep it)
      int& nch = sp ? P.ochunk_sp : P.ochunk_ang;
      const int h = nch;
      double best = -1.0, worst = -1.0;
      int pick = h;
      for (int cand : {h, h / 2, h / 4}) {
        if (cand < 1 || (cand != h && cand == pick)) continue;
        Problem Q = P;
        (sp ? Q.ochunk_sp : Q.ochunk_ang) = cand;
        const double t = time_on(st, REPS, [&] {
          const int n = gram_partials(Q, B, st, sp, A, RC, B.keep, nullptr);
          Dst d;
          for (int i = 0; i < 8; ++i) d.idx[i] = SM_QM;
          reduce_to(Q, B, st, n, 1, d);
        });
        if (t > 0.0 && (best < 0.0 || t < 0.97 * best)) { best = t; pick = cand; }
        worst = std::max(worst, t);
      }
      nch = pick;
      ms[4 * f + 2] = best;
      ms[4 * f + 3] = worst;
    }
  }
  // leave the workspace as a new solver has it
  cudaError_t e = cudaMemsetAsync(B.sm, 0, sizeof(double) * nsm_elems, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return e;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    TuneChoice c;
    c.oz_sp = P.oz_sp; c.oz_ang = P.oz_ang; c.nch_sp = P.ochunk_sp; c.nch_ang = P.ochunk_ang;
    c.ozg_sp = P.ozg_sp; c.ozg_ang = P.ozg_ang;
    for (int i = 0; i < 8; ++i) c.ms[i] = ms[i];
    g_tune_cache[key] = c;
  }
  return cudaSuccess;
}

// dm += sign * scalar flux of A (spatial, cnt columns) in the angular basis V (with
// core S when given); the conserved-moment correction's bookkeeping
static void mass_acc(const Problem& P, const PhaseBufs& B, cudaStream_t st, const double* A,
                     const double* V, const double* S, const int* cnt, double sign) {
  pbeg(st, KS_MASS);
  k_mf_vec<<<P.g.nsub, DD_THREADS, 0, st>>>(P, V, S, cnt, B.mvec);
  k_mf_acc<<<dim3((P.maxN + DD_THREADS - 1) / DD_THREADS, P.g.nsub), DD_THREADS, 0, st>>>(
      P, A, cnt, B.mvec, sign, B.dm);
  pend(st);
}

static OrthArgs orth_args(const Problem& P, const PhaseBufs& B, int spatial, int mode) {
  OrthArgs a;
  a.g = P.g; a.spatial = spatial; a.mode = mode;
  a.rank_mode = P.rank_mode; a.tol = P.tol; a.r_floor = P.r_floor; a.r_aug_max = P.r_aug_max;
  a.tau = P.tau; a.accept = P.accept;
  a.angcand = P.angcand; a.n_angcand = P.n_angcand; a.angcand_complete = P.angcand_complete;
  a.n_angorth = P.n_angorth;
  a.sig_out = B.sig; a.p_out = B.p; a.status = B.status;
  a.r_own = B.r; a.rt_out = B.rt;
  return a;
}

// Orthonormal basis of the significant left singular span of A (per subdomain),
// completed to the requested width: Gram, its eigendecomposition, U1 = A V S^-1,
// one CholeskyQR pass on U1, completion (dd_orth.cu).
static void orthonormalize(const Problem& P, const PhaseBufs& B, cudaStream_t st, OrthArgs a) {
  const int sp = a.spatial;
  double* W = sp ? B.Hw : B.Hwa;
  int nch = gram_partials(P, B, st, sp, a.A, a.lda, a.acols, B.cexp);
  launch_geig(a, B.part, B.cexp, nch, B.sm, SM_QM, B.keep, st);
  // U1 = A M; its Gram from the same tiles when their partials fit the buffer (one partial
  // per 32-row tile, counted from each subdomain's first row), else by k_gram
  const int ntile = ((sp ? P.maxN : P.g.n) + TALL_ROWS - 1) / TALL_ROWS;
  const bool fuse = !(sp ? P.oz_sp : P.oz_ang) && ntile <= 8 * std::max(P.nchunk_sp, P.nchunk_ang);
  tall(P, B, st, sp, a.A, a.lda, a.acols, 0, nullptr, SM_QM, B.keep, 0, W, P.WC,
       fuse ? B.part : nullptr);
  nch = fuse ? ntile : gram_partials(P, B, st, sp, W, P.WC, B.keep, nullptr);
  launch_chol_inv(a, B.part, nch, B.sm, SM_R1I, B.keep, st);
  tall(P, B, st, sp, W, P.WC, B.keep, 0, nullptr, SM_R1I, B.keep, 0, a.Q, a.ldq);
  if (a.mode == ORTH_QR || (!sp && a.mode == ORTH_AUG)) {
    // mutually orthogonal candidates (the cosines; the angular table): coefficient-space
    // Gram-Schmidt on all SMs, then the one-by-one completion for whatever that leaves
    // (normally nothing; in angle the unit vectors after the table)
    launch_kc(a, P.sptab, P.spoff, P.spnf, B.keep, B.part, B.kcn, B.kcur, P.maxN, st);
    launch_complete(a, B.kcur, st);
  } else {
    launch_complete(a, B.keep, st);
  }
}

void advection_phase(const Problem& P, const PhaseBufs& B, int axis, cudaStream_t st) {
  const Geo& g = P.g;
  const int RC = g.RC, nsub = g.nsub;
  // 1. augmentation (Algorithm 4)
  pbeg(st, KS_AUG_COLS);
  k_aug_cols<<<(nsub + 127) / 128, 128, 0, st>>>(g, B.r, axis, B.m, P.infl_on);
  pend(st);
  pbeg(st, KS_BUILD_L0);
  k_build_L0<<<dim3((g.n + 31) / 32, nsub), DD_THREADS, sizeof(double) * 3 * RC * RC, st>>>(
      g, B.V, B.S, B.r, axis, B.L0, P.infl_on, P.infl_hw, P.infl_sc);
  pend(st);
  {
    OrthArgs a = orth_args(P, B, 0, ORTH_AUG);
    a.A = B.L0; a.lda = g.MC; a.acols = B.m; a.Q = B.Vh; a.ldq = RC; a.rout = nullptr;
    orthonormalize(P, B, st, a);
  }
  pbeg(st, KS_COPY);
  cudaMemcpyAsync(B.rx + axis * nsub, B.rt, sizeof(int) * nsub, cudaMemcpyDeviceToDevice, st);
  pend(st);
  // 2. angular Galerkin coefficients, boundary masses
  // twice the angular chunks (more blocks than SMs), as far as the partial buffer holds
  const int nch_ac = std::min(2 * P.nchunk_ang, std::max(P.nchunk_sp, P.nchunk_ang));
  const int nblk_ac = P.kstep_split == 1 ? 8 : 6;
  bool tc_done = false;
  if (P.prec >= PREC_TF32 && !P.infl_on) {
    // the six (eight) blocks as weighted Grams against Vh; the sources that read Vh itself
    // take the even slots, the own and neighbour V the odd ones
    TcGram a = tgram(P, B, 0, axis, B.Vh, B.rt, nch_ac, nblk_ac);
    TcGramSrc vh = gsrc(nullptr, RC, B.rt, 0, W_OMEGA);
    vh.same_as_b = 1;
    TcGramSrc v = gsrc(B.V, RC, B.r, 3);
    a.src[0] = vh;                                   // C
    a.src[1] = v;                                    // M
    a.src[2] = vh; a.src[2].blk = 1; a.src[2].wsel = W_NEG;      // Mout_lo
    a.src[3] = v; a.src[3].blk = 4; a.src[3].nbside = 0; a.src[3].wsel = W_NONNEG;  // Min_lo
    a.src[4] = vh; a.src[4].blk = 2; a.src[4].wsel = W_NONNEG;   // Mout_hi
    a.src[5] = v; a.src[5].blk = 5; a.src[5].nbside = 1; a.src[5].wsel = W_NEG;     // Min_hi
    a.nsrc = 6;
    if (nblk_ac == 8) {
      a.src[6] = vh; a.src[6].blk = 6; a.src[6].wsel = W_OMEGA_POS;                  // C+
      a.src[7] = vh; a.src[7].blk = 7; a.src[7].wsel = W_OMEGA_NEG;                  // C-
      a.nsrc = 8;
    }
    tc_done = tc_gram(P, st, a);
  }
  if (!tc_done) {
    pbeg(st, KS_ANG_COEFFS);
    k_ang_coeffs<<<dim3(nch_ac, nsub), DD_THREADS, 0, st>>>(
        g, axis == 0 ? P.ox : P.oy, B.Vh, B.V, B.r, B.rt, axis, nch_ac, nblk_ac, B.part,
        P.infl_on, P.infl_hw);
    pend(st);
  }
  {
    Dst d;
    d.idx[0] = SM_C; d.idx[1] = SM_MOUT_LO; d.idx[2] = SM_MOUT_HI;
    d.idx[3] = SM_M; d.idx[4] = SM_MIN_LO; d.idx[5] = SM_MIN_HI;
    d.idx[6] = SM_CP; d.idx[7] = SM_CM;
    pbeg(st, KS_REDUCE);
    k_reduce<<<reduce_grid(g, nblk_ac), DD_THREADS, 0, st>>>(B.part, nch_ac, nblk_ac, d, B.sm, RC);
    pend(st);
  }
  // 3. S M products, eigen-split of C
  pbeg(st, KS_SMALL_ADV1);
  k_small_adv1<<<nsub, DD_THREADS, small_adv1_smem(RC), st>>>(P, B, axis);
  pend(st);
  // 4. K^0 = X (S <V, Vh>)
  galerkin_tall(P, B, st, 1, B.X, RC, B.r, nullptr, SM_B, B.rt, B.K, RC);
  // 5. boundary data
  pbeg(st, KS_GHOST);
  k_ghost<<<dim3((2 * P.maxlines + DD_THREADS / 32 - 1) / (DD_THREADS / 32), nsub), DD_THREADS, 0, st>>>(P, B, axis);
  pend(st);
  // 6. K-step
  {
    const int len = P.maxlines;
    // with the spatial tall products on the tensor cores (and, for RK4, every line within
    // the eigenbasis tile): the two basis changes as tall products (K~ = K P into X1, free
    // until the QR; K += increment P^T, accumulated in FP64 by the product's epilogue:
    // rotating the whole K back would put rounding of K's size on entries whose increment is
    // tiny), the stages in the eigenbasis in between
    const bool euler = P.integrator == 0;
    const bool ebasis = P.kstep_split == 0 && P.oz_sp &&
                        (euler || (long)len * g.RC <= (long)DD_THREADS * KE_EPT);
    if (ebasis && oz_tall(P, B.status, st, 1, B.K, RC, B.rt, 0, nullptr, SM_S3T, B.sm, B.rt, 0,
                          B.X1, RC, 0)) {
      // the stages on K~ (the increment into Hw with Euler, in place in X1 with RK4), then
      // K += increment P^T by the second product (the same shape as the first: it cannot be
      // refused where that one was not)
      pbeg(st, KS_KSTEP_ADV);
      if (euler) {
        k_kstep_eig1<<<dim3(P.maxlines, nsub), DD_THREADS, 0, st>>>(P, B, axis);
      } else {
        const int lpb = kstep_eig_lpb(P, len);
        dim3 grid((P.maxlines + lpb - 1) / lpb, nsub);
        k_kstep_eig<double><<<grid, DD_THREADS, kstep_eig_smem(P, lpb, len), st>>>(P, B, axis, lpb, 1);
      }
      pend(st);
      (void)oz_tall(P, B.status, st, 1, euler ? B.Hw : B.X1, RC, B.rt, 0, nullptr, SM_S3T, B.sm,
                    B.rt, 0, B.K, RC, 1, 1);
    } else {
    pbeg(st, KS_KSTEP_ADV);
    if (P.kstep_split == 0 && len < 4096) {
      // FP64 eigen-split in the eigenbasis, in the mixed form too: the FP32 matrix
      // stencil rounds |C| K_i, C+ K_i-1 and C- K_i+1, which cancel to the much smaller
      // increment, and its error grew to 1e-4..1e-3 of the flux on narrow sources
      const int lpb = kstep_eig_lpb(P, len);
      dim3 grid((P.maxlines + lpb - 1) / lpb, nsub);
      k_kstep_eig<double><<<grid, DD_THREADS, kstep_eig_smem(P, lpb, len), st>>>(P, B, axis, lpb, 0);
      if ((long)len * g.RC > (long)DD_THREADS * KE_EPT) {
        // subdomains whose line exceeds the eigenbasis kernel's tile: the FP64 matrix
        // stencil (the same discrete operator)
        const int lpb2 = kstep_lpb(P, len);
        dim3 grid2((P.maxlines + lpb2 - 1) / lpb2, nsub);
        k_kstep_adv<double><<<grid2, DD_THREADS, kstep_smem(P, lpb2, len), st>>>(P, B, axis, lpb2, 1);
      }
    } else {
      const int lpb = kstep_lpb(P, len);
      dim3 grid((P.maxlines + lpb - 1) / lpb, nsub);
      if (P.prec >= PREC_MIXED)
        k_kstep_adv<float><<<grid, DD_THREADS, kstep_smem(P, lpb, len), st>>>(P, B, axis, lpb, 0);
      else
        k_kstep_adv<double><<<grid, DD_THREADS, kstep_smem(P, lpb, len), st>>>(P, B, axis, lpb, 0);
    }
    pend(st);
    }
  }
  if (P.mass_fix) mass_acc(P, B, st, B.K, B.Vh, nullptr, B.rt, 1.0);
  // 7. QR of K
  {
    OrthArgs a = orth_args(P, B, 1, ORTH_QR);
    a.A = B.K; a.lda = RC; a.acols = B.rt; a.Q = B.X1; a.ldq = RC; a.rout = B.rt;
    orthonormalize(P, B, st, a);
  }
  // 8. S-step coefficients and S-step
  bool sp_tc = false;
  {
    // the spatial coefficient T = X1^T shift(X1) on the tensor cores in its difference form
    // E = X1^T (X1 - shift(X1)) = I - T (a Gram against X1, written transposed; the
    // reduction forms T = I - E); S1 = X1^T K (the R factor of the QR of K) and the face
    // products G_lo, G_hi in FP64
    bool& tcd = sp_tc;
    if (P.prec >= PREC_TF32) {
      TcGram a = tgram(P, B, 1, axis, B.X1, B.rt, P.nchunk_sp, 4);
      a.src[0] = gsrc(B.X1, RC, B.rt, 1, W_NONE, nullptr, 1);
      a.src[0].shift = 1;
      a.nsrc = 1;
      tcd = tc_gram(P, st, a);
    }
    pbeg(st, KS_SP_COEFFS);
    k_sp_coeffs<<<dim3(P.nchunk_sp, nsub), DD_THREADS, 0, st>>>(P, B, axis, tcd ? 1 : 0);
    pend(st);
  }
  {
    Dst d;
    d.idx[0] = SM_S1; d.idx[1] = SM_T; d.idx[2] = SM_G_LO; d.idx[3] = SM_G_HI;
    d.ident = sp_tc ? 2 : 0;
    pbeg(st, KS_REDUCE);
    k_reduce<<<reduce_grid(g, 4), DD_THREADS, 0, st>>>(B.part, P.nchunk_sp, 4, d, B.sm, RC);
    pend(st);
  }
  pbeg(st, KS_SSTEP_ADV);
  {
    // blocks per subdomain: enough to cover the SMs, at most 8
    const int CL = std::max(1, std::min(8, P.nsm / std::max(1, nsub)));
    const int nst = P.integrator == 1 ? 4 : 1;
    for (int s = 0; s < nst; ++s)
      k_sstep_adv<<<nsub * CL, DD_THREADS, sstep_smem(RC), st>>>(P, B, axis, s, CL);
  }
  pend(st);
  // 9. L-step
  bool lprod = false;
  if (P.integrator == 0 && P.oz_ang) {
    // as three products over the direction rows, FP64-accurate in every form: L = V S2^T,
    // then L += dt kappa_q (V W_s^T)_q by the products' accumulating epilogue, with the
    // per-row scales of k_lstep_w (zero for the other upwind side)
    double* rs = B.Hwa;                            // 2 x nsub x n row scales
    pbeg(st, KS_LSTEP_PROD);
    k_lstep_w<<<dim3(2, nsub), DD_THREADS, 0, st>>>(P, B, axis, rs);
    pend(st);
    lprod = oz_tall(P, B.status, st, 0, B.Vh, RC, B.rt, 0, nullptr, SM_UB, B.sm, B.rt, 0, B.L, RC);
    if (lprod) {                                   // the same shape: not refused either
      (void)oz_tall(P, B.status, st, 0, B.Vh, RC, B.rt, 0, nullptr, SM_VB, B.sm, B.rt, 0, B.L, RC,
                    0, 1, rs);
      (void)oz_tall(P, B.status, st, 0, B.Vh, RC, B.rt, 0, nullptr, SM_S3T, B.sm, B.rt, 0, B.L, RC,
                    0, 1, rs + (long)nsub * g.n);
    }
  }
  if (!lprod) {
    pbeg(st, KS_LSTEP_ADV);
    if (P.prec >= PREC_MIXED) {
      k_lstep_adv<float><<<dim3((g.n + 31) / 32, nsub), DD_THREADS, lstep_smem(RC),
                    st>>>(P, B, axis);
    } else {
      k_lstep_adv<double><<<dim3((g.n + 31) / 32, nsub), DD_THREADS, lstep_smem(RC),
                    st>>>(P, B, axis);
    }
    pend(st);
  }
  // 10. QR of L
  {
    OrthArgs a = orth_args(P, B, 0, ORTH_QR);
    a.A = B.L; a.lda = RC; a.acols = B.rt; a.Q = B.V1; a.ldq = RC; a.rout = B.rt;
    orthonormalize(P, B, st, a);
  }
  gram(P, B, st, 0, B.V1, RC, B.rt, 0, B.L, RC, B.rt, 0, 1, nullptr, SM_S3T);
  // 11. truncation (Algorithm 5)
  pbeg(st, KS_TRUNC);
  k_trunc<<<nsub, DD_THREADS, trunc_smem(RC), st>>>(
      P, B);
  pend(st);
  galerkin_tall(P, B, st, 1, B.X1, RC, B.rt, nullptr, SM_UB, B.ro, B.Xo, RC);
  galerkin_tall(P, B, st, 0, B.V1, RC, B.rt, nullptr, SM_VB, B.ro, B.Vo, RC);
  if (P.mass_fix) mass_acc(P, B, st, B.Xo, B.Vo, B.So, B.ro, -1.0);
}

void collision_phase(const Problem& P, const PhaseBufs& B, cudaStream_t st) {
  const Geo& g = P.g;
  const int RC = g.RC, nsub = g.nsub;
  pbeg(st, KS_COLL_RANK);
  k_coll_rank<<<(nsub + 127) / 128, 128, 0, st>>>(P, B.r, B.rc);
  pend(st);
  {
    OrthArgs a = orth_args(P, B, 0, ORTH_COMPLETE);
    a.A = B.V; a.lda = RC; a.acols = B.r; a.Q = B.Vh; a.ldq = RC; a.rout = B.rc;
    launch_complete(a, nullptr, st);
  }
  pbeg(st, KS_COLL_A);
  k_coll_a<<<nsub, DD_THREADS, 0, st>>>(P, B);
  pend(st);
  galerkin_tall(P, B, st, 1, B.X, RC, B.r, B.S, -1, B.rc, B.K, RC);
  pbeg(st, KS_COLL_KSTEP);
  if (P.prec >= PREC_MIXED) {
    k_coll_kstep<float><<<dim3(64, nsub), DD_THREADS, 0, st>>>(P, B);
  } else if (P.integrator == 0) {
    k_coll_kstep1<<<dim3((P.maxN + DD_THREADS - 1) / DD_THREADS, nsub), DD_THREADS, 0, st>>>(P, B);
  } else {
    k_coll_kstep<double><<<dim3(64, nsub), DD_THREADS, 0, st>>>(P, B);
  }
  pend(st);
  if (P.mass_fix) mass_acc(P, B, st, B.K, B.Vh, nullptr, B.rc, 1.0);
  {
    OrthArgs a = orth_args(P, B, 1, ORTH_QR);
    a.A = B.K; a.lda = RC; a.acols = B.rc; a.Q = B.Xo; a.ldq = RC; a.rout = B.rc;
    orthonormalize(P, B, st, a);
  }
  // S1 = Xo^T K (the R factor of the QR of K) in FP64; the Galerkin contractions
  // Ms = Xo^T diag(sigma_s) Xo, Mt = Xo^T diag(sigma_t) Xo on the tensor cores in the
  // DD_TF32 / DD_BF16 forms
  gram(P, B, st, 1, B.Xo, RC, B.rc, 0, B.K, RC, B.rc, 0, 1, nullptr, SM_S1);
  {
    bool tcd = false;
    if (P.prec >= PREC_TF32) {
      TcGram a = tgram(P, B, 1, 0, B.Xo, B.rc, P.nchunk_sp, 2);
      a.src[0] = gsrc(nullptr, RC, B.rc, 0, W_ROW, P.sig_s);
      a.src[0].same_as_b = 1;
      a.src[1] = a.src[0];
      a.src[1].blk = 1;
      a.src[1].wrow = P.sig_t;
      a.nsrc = 2;
      if ((tcd = tc_gram(P, st, a))) {
        Dst d;
        d.idx[0] = SM_MS; d.idx[1] = SM_MT;
        reduce_to(P, B, st, P.nchunk_sp, 2, d);
      }
    }
    if (!tcd) {
      gram(P, B, st, 1, B.Xo, RC, B.rc, 0, B.Xo, RC, B.rc, 0, 1, P.sig_s, SM_MS);
      gram(P, B, st, 1, B.Xo, RC, B.rc, 0, B.Xo, RC, B.rc, 0, 1, P.sig_t, SM_MT);
    }
  }
  // q = X1^T sQ  -> row 1 of the vector block (reduce into a scratch small, then copy)
  {
    GramArgs a;
    a.spatial = 1; a.A = B.Xo; a.lda = RC; a.acnt = B.rc; a.afix = 0;
    a.Bm = P.sQ; a.ldb = 1; a.bcnt = nullptr; a.bfix = 1; a.b_per_sub = 1;
    a.wrow = nullptr; a.part = B.part; a.nchunk = P.nchunk_sp; a.cexp = nullptr; a.sym = 0;
    pbeg(st, KS_GRAM);
    k_gram<<<dim3(a.nchunk, nsub), DD_THREADS, sizeof(double) * RC * RC, st>>>(g, a);
    pend(st);
    Dst d;
    d.idx[0] = SM_UB;   // scratch: column 0 holds q
    pbeg(st, KS_REDUCE);
    k_reduce<<<reduce_grid(g, 1), DD_THREADS, 0, st>>>(B.part, a.nchunk, 1, d, B.sm, RC);
    pend(st);
  }
  pbeg(st, KS_COLL_SMALL);
  k_coll_small<<<nsub, DD_THREADS, sizeof(double) * (4 * RC * RC + 5 * RC), st>>>(P, B);
  pend(st);
  pbeg(st, KS_COLL_LSTEP);
  if (P.prec >= PREC_MIXED) {
    k_coll_lstep<float><<<dim3((g.n + 31) / 32, nsub), DD_THREADS,
                   coll_lstep_smem(RC), st>>>(P, B);
  } else if (P.integrator == 0) {
    k_coll_lstep1<<<dim3((g.n + DD_THREADS - 1) / DD_THREADS, nsub), DD_THREADS,
                    coll_lstep1_smem(RC), st>>>(P, B);
  } else {
    k_coll_lstep<double><<<dim3((g.n + 31) / 32, nsub), DD_THREADS,
                   coll_lstep_smem(RC), st>>>(P, B);
  }
  pend(st);
  {
    OrthArgs a = orth_args(P, B, 0, ORTH_QR);
    a.A = B.L; a.lda = RC; a.acols = B.rc; a.Q = B.Vo; a.ldq = RC; a.rout = B.rc;
    orthonormalize(P, B, st, a);
  }
  gram(P, B, st, 0, B.Vo, RC, B.rc, 0, B.L, RC, B.rc, 0, 1, nullptr, SM_S3T);
  pbeg(st, KS_COLL_FINAL);
  k_coll_final<<<nsub, DD_THREADS, 0, st>>>(P, B);
  pend(st);
  if (P.mass_fix) mass_acc(P, B, st, B.Xo, B.Vo, B.So, B.ro, -1.0);
}

// Conserved-moment correction at the end of a step (optional; not part of the
// paper's scheme): f <- X S V^T + dm (x) 1/|S|, orthonormalised and truncated by
// Algorithm 5's rule.  In the stored (Euclidean) form f = K_a V_a^T with
// K_a = [X S | sqrt(hx hy) dm] and V_a = [V | sqrt(w)/|S|]; V_a = Q_v, K' = K_a (V_a^T Q_v),
// K' = Q_x S', and the truncation of the (r+1) x (r+1) core S' as in the advection.
void mass_fix_phase(const Problem& P, const PhaseBufs& B, cudaStream_t st) {
  const Geo& g = P.g;
  const int RC = g.RC, nsub = g.nsub;
  pbeg(st, KS_MASS);
  k_mf_build_x<<<dim3((P.maxN + DD_THREADS - 1) / DD_THREADS, nsub), DD_THREADS, 0, st>>>(
      P, B.X, B.S, B.r, B.dm, B.K);
  k_mf_build_v<<<dim3((g.n + DD_THREADS - 1) / DD_THREADS, nsub), DD_THREADS, 0, st>>>(
      P, B.V, B.r, B.L, B.m);
  pend(st);
  {
    OrthArgs a = orth_args(P, B, 0, ORTH_QR);
    a.A = B.L; a.lda = RC; a.acols = B.m; a.Q = B.V1; a.ldq = RC; a.rout = B.m;
    orthonormalize(P, B, st, a);
  }
  gram(P, B, st, 0, B.L, RC, B.m, 0, B.V1, RC, B.m, 0, 1, nullptr, SM_B);
  tall(P, B, st, 1, B.K, RC, B.m, 0, nullptr, SM_B, B.m, 0, B.X1, RC);
  {
    OrthArgs a = orth_args(P, B, 1, ORTH_QR);
    a.A = B.X1; a.lda = RC; a.acols = B.m; a.Q = B.K; a.ldq = RC; a.rout = B.m;
    orthonormalize(P, B, st, a);
  }
  gram(P, B, st, 1, B.X1, RC, B.m, 0, B.K, RC, B.m, 0, 1, nullptr, SM_S3T);
  pbeg(st, KS_COPY);
  cudaMemcpyAsync(B.rt, B.m, sizeof(int) * nsub, cudaMemcpyDeviceToDevice, st);
  pend(st);
  pbeg(st, KS_TRUNC);
  k_trunc<<<nsub, DD_THREADS, trunc_smem(RC), st>>>(P, B);
  pend(st);
  tall(P, B, st, 1, B.K, RC, B.rt, 0, nullptr, SM_UB, B.ro, 0, B.Xo, RC);
  tall(P, B, st, 0, B.V1, RC, B.rt, 0, nullptr, SM_VB, B.ro, 0, B.Vo, RC);
}

void scalar_flux(const Problem& P, const double* X, const double* V, const double* S, const int* r,
                 double* work, double* rho, int nx, cudaStream_t st) {
  pbeg(st, KS_FLUX);
  k_flux_prep<<<P.g.nsub, DD_THREADS, 0, st>>>(P, V, S, r, work);
  pend(st);
  pbeg(st, KS_FLUX);
  k_flux<<<dim3(16, P.g.nsub), DD_THREADS, 0, st>>>(P, X, r, work, rho, nx);
  pend(st);
}

}  // namespace dd
