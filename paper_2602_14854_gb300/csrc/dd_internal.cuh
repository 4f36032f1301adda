// Internal declarations of the DD-DLRA CUDA library (not part of the ABI).
//
// Storage convention on the device (the factors of the paper, rescaled so that
// every orthonormality is Euclidean):
//   X = sqrt(hx*hy) * U        (N_k x r, row-major, X^T X = I)
//   Vt = diag(sqrt(w)) * V     (n x r,   row-major, Vt^T Vt = I)
//   S                          (r x r,   the paper's S)
// so f_{c,q} = X_c S Vt_q^T / (sqrt(hx*hy) sqrt(w_q)) and the singular values of S
// are the paper's weighted L2 singular values (Section 3.4 matrix form).
//
// Spatial tall arrays hold all subdomains back to back: row rowoff[k] + c for
// cell c (x-fastest inside subdomain k).  Angular tall arrays hold n rows per
// subdomain: row k*n + q.  Small per-subdomain matrices are RC x RC blocks.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define DD_MAXC 64          // maximum columns of any tall or small matrix
#define DD_THREADS 256

namespace dd {

enum OrthMode { ORTH_QR = 0, ORTH_AUG = 1, ORTH_COMPLETE = 2 };
enum StatusBits { ST_NONFINITE = 1, ST_COMPLETION = 2, ST_RANKCAP = 4, ST_TIMEOUT = 8 };
// arithmetic of the step (dd_options.precision)
enum Prec { PREC_FP64 = 0, PREC_MIXED = 1, PREC_TF32 = 2, PREC_BF16 = 3 };

// Geometry of the tiling, device arrays (read-only inside kernels).
struct Geo {
  int nsub, n, RC, MC;
  const int* N;      // cells of subdomain k
  const int* nxk;    // width
  const int* nyk;    // height
  const int* rowoff; // first spatial row of subdomain k
  const int* nb;     // 4 per subdomain: x-lo, x-hi, y-lo, y-hi neighbour, -1 = physical boundary
  const int* cx0;    // x offset of the subdomain inside its problem's grid
  const int* cy0;    // y offset
  // per-subdomain problem parameters (a batch holds several independent problems
  // that share the direction table; every subdomain carries its problem's values)
  const double* hxk;  // cell widths
  const double* hyk;
  const double* dtk;  // time step
  const double* shk;  // sqrt(hx hy)
  const int* rlo;     // rank floor / lower truncation clamp (fixed mode: the rank)
  const int* rhi;     // upper truncation clamp (fixed mode: the rank)
  const int* raug;    // cap of the intermediate rank
  const int* fbase;   // first cell of the problem in the concatenated density output
  const int* fnx;     // width of the problem's grid
  // algorithmic flops per kernel slot, counted by the kernels while dd_dlra_profile_work
  // runs (null otherwise: nothing is counted)
  unsigned long long* work;
};

// Adds one CTA's algorithmic flops to the slot's counter (profiling only).
__device__ __forceinline__ void count_work(const Geo& g, int slot, double flops) {
  if (g.work && threadIdx.x == 0 && flops > 0.0)
    atomicAdd(&g.work[slot], (unsigned long long)flops);
}

// Line geometry along an axis (0 = x, 1 = y) for subdomain k.
struct Lines {
  int nlines, len, stride_line, stride_pos;
};
__device__ __forceinline__ Lines lines_of(const Geo& g, int k, int axis) {
  Lines L;
  int nx = g.nxk[k], ny = g.nyk[k];
  if (axis == 0) { L.nlines = ny; L.len = nx; L.stride_line = nx; L.stride_pos = 1; }
  else           { L.nlines = nx; L.len = ny; L.stride_line = 1; L.stride_pos = nx; }
  return L;
}
__device__ __forceinline__ int cell_of(const Lines& L, int line, int pos) {
  return line * L.stride_line + pos * L.stride_pos;
}

// ---------------------------------------------------------------------------
// reductions
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <typename T>
__device__ __forceinline__ T warp_sum_t(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <typename T>
__device__ __forceinline__ T warp_max_t(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
// Block-wide sum returned to every thread; red must hold >= 33 doubles.
__device__ __forceinline__ double block_sum(double v, double* red) {
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  if (wid == 0) {
    double t = (lane < nw) ? red[lane] : 0.0;
    t = warp_sum(t);
    if (lane == 0) red[32] = t;
  }
  __syncthreads();
  return red[32];
}
// Three block-wide FP32 sums in one reduction, returned to every thread; red must hold
// >= 99 floats.
__device__ __forceinline__ void block_sum3f(float* a, float* b, float* c, float* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  float x = *a, y = *b, z = *c;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    x += __shfl_xor_sync(0xffffffffu, x, o);
    y += __shfl_xor_sync(0xffffffffu, y, o);
    z += __shfl_xor_sync(0xffffffffu, z, o);
  }
  __syncthreads();
  if (lane == 0) { red[wid] = x; red[32 + wid] = y; red[64 + wid] = z; }
  __syncthreads();
  if (wid == 0) {
    x = lane < nw ? red[lane] : 0.f;
    y = lane < nw ? red[32 + lane] : 0.f;
    z = lane < nw ? red[64 + lane] : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      x += __shfl_xor_sync(0xffffffffu, x, o);
      y += __shfl_xor_sync(0xffffffffu, y, o);
      z += __shfl_xor_sync(0xffffffffu, z, o);
    }
    if (lane == 0) { red[96] = x; red[97] = y; red[98] = z; }
  }
  __syncthreads();
  *a = red[96]; *b = red[97]; *c = red[98];
}
__device__ __forceinline__ double block_max(double v, double* red) {
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_max(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  if (wid == 0) {
    double t = (lane < nw) ? red[lane] : 0.0;
    t = warp_max(t);
    if (lane == 0) red[32] = t;
  }
  __syncthreads();
  return red[32];
}

// Stable descending order of v[0..n) by ranks (block-wide, one thread per entry):
// perm[t] is the index of the t-th largest value, ties by index.  NaN ranks as
// -infinity, so perm is a permutation for any input.
__device__ __forceinline__ double rank_key(double x) { return x == x ? x : -INFINITY; }
__device__ __forceinline__ void rank_sort_desc(const double* v, int n, int* perm) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double x = rank_key(v[i]);
    int r = 0;
    for (int j = 0; j < n; ++j) {
      const double y = rank_key(v[j]);
      r += (y > x) || (y == x && j < i);
    }
    perm[r] = i;
  }
}

// The same order for non-negative, non-NaN values, compared by their bit patterns
// (which order as the values).
__device__ __forceinline__ void rank_sort_desc_nonneg(const double* v, int n, int* perm) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const long long x = __double_as_longlong(v[i]);
    int r = 0;
    for (int j = 0; j < n; ++j) {
      const long long y = __double_as_longlong(v[j]);
      r += (y > x) || (y == x && j < i);
    }
    perm[r] = i;
  }
}

// Spatial completion candidates (the cosine products of the completion family, by
// a + b, then a descending): at most kc_bmax(RC) of them are examined at once.
__host__ __device__ __forceinline__ int kc_bmax(int RC) { return RC + (4 * RC + 2) / 3 + 1; }
// doubles of scratch per subdomain: coefficients A (bmax x RC), B (RC x RC), then
// W = Q0^T C ((RC + 1) x bmax, the candidates' squared norms in row RC)
__host__ __device__ __forceinline__ size_t kc_region(int RC) {
  return (size_t)(kc_bmax(RC) + RC) * RC + (size_t)(RC + 1) * kc_bmax(RC);
}
// Length of the longest leading run of nc candidates that are mutually orthogonal to rel_tol
// in cosine and non-zero, from their Gram G (nc x nc, row-major, host memory): only those
// take the coefficient-space completion (a product quadrature makes the whole angular table
// so).
inline int orthogonal_prefix_gram(const double* G, int nc, double rel_tol) {
  int po = 0;
  for (; po < nc; ++po) {
    const double np = __builtin_sqrt(G[(size_t)po * nc + po]);
    bool ok = np > 0.0;
    for (int i = 0; i < po && ok; ++i)
      ok = __builtin_fabs(G[(size_t)i * nc + po]) <=
           rel_tol * __builtin_sqrt(G[(size_t)i * nc + i]) * np;
    if (!ok) break;
  }
  return po;
}

// Candidate j of an nxk x nyk subdomain: frequencies (a, b); false past the family.
__host__ __device__ __forceinline__ bool kc_cand(int j, int nxk, int nyk, int* ca, int* cb) {
  for (int d = 0; d <= nxk + nyk - 2; ++d) {
    const int ahi = d < nxk - 1 ? d : nxk - 1;
    const int alo = d - (nyk - 1) > 0 ? d - (nyk - 1) : 0;
    const int cnt = ahi - alo + 1;
    if (j < cnt) { *ca = ahi - j; *cb = d - *ca; return true; }
    j -= cnt;
  }
  return false;
}
// Candidates examined for cur0 columns done out of r_out: the missing ones plus 4 cur0 / 3
// for rejections.  The unit candidates are orthonormal, so their squared projections
// onto the span of the cur0 first columns sum to at most cur0, and a candidate rejected
// for that projection alone carries more than 3/4 of it; when the block still falls
// short, the sequential completion adds the rest.
__host__ __device__ __forceinline__ int kc_b(int nxk, int nyk, int cur0, int r_out, int RC) {
  const int need = r_out - cur0;
  if (need <= 0) return 0;
  int b = need + (4 * cur0 + 2) / 3 + 1;
  if (b > nxk * nyk) b = nxk * nyk;
  if (b > kc_bmax(RC)) b = kc_bmax(RC);
  return b;
}

// Round-robin (circle method) pairing for parallel Jacobi sweeps over mm
// (even) indices: round r in [0, mm-1), pair i in [0, mm/2).  Both sums are below
// 2 (mm - 1), so each reduction modulo mm - 1 is one compare-and-subtract.
__device__ __forceinline__ void rr_pair(int mm, int r, int i, int* p, int* q) {
  const int M = mm - 1;
  if (i == 0) { *p = 0; *q = (mm > 1) ? 1 + r : 0; return; }
  int a = i + r, b = M - i + r;
  a = a >= M ? a - M : a;
  b = b >= M ? b - M : b;
  *p = 1 + a; *q = 1 + b;
}

#define JACOBI_TOL 1e-15

__device__ __forceinline__ float rsqrt_t(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_t(double x) { return rsqrt(x); }

// ---------------------------------------------------------------------------
// Double-float ("float-float") arithmetic: a value is the unevaluated sum hi + lo of
// two floats, |lo| <= ulp(hi)/2, about 48 significant bits.  Built from the exact
// error-free transformations of Knuth (TwoSum) and Dekker (Fast2Sum), with the product
// error taken by one FMA.  Explicit _rn intrinsics keep the compiler from contracting
// or reassociating the compensated sequences.  On this GPU FP32 issues at 64x the
// FP64 rate, so small sequential linear algebra runs several times faster this way
// than in FP64 while keeping ~1e-14 relative accuracy.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float v = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, v)), __fsub_rn(b, v));
  return make_float2(s, e);
}
__device__ __forceinline__ float2 df_fast_sum(float a, float b) {   // needs |a| >= |b| or a == 0
  const float s = __fadd_rn(a, b);
  return make_float2(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
  const float2 s = df_two_sum(a.x, b.x);
  return df_fast_sum(s.x, __fadd_rn(s.y, __fadd_rn(a.y, b.y)));
}
__device__ __forceinline__ float2 df_neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 df_mul(float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  float e = __fmaf_rn(a.x, b.x, -p);
  e = __fmaf_rn(a.x, b.y, e);
  e = __fmaf_rn(a.y, b.x, e);
  return df_fast_sum(p, e);
}
__device__ __forceinline__ float2 df_mulf(float2 a, float b) {
  const float p = __fmul_rn(a.x, b);
  float e = __fmaf_rn(a.x, b, -p);
  e = __fmaf_rn(a.y, b, e);
  return df_fast_sum(p, e);
}
__device__ __forceinline__ float2 df_sqrt(float2 a) {          // a > 0
  const float y = sqrtf(a.x);
  const float p = __fmul_rn(y, y);
  const float2 r = df_add(a, make_float2(-p, -__fmaf_rn(y, y, -p)));
  return df_fast_sum(y, r.x / (2.f * y));
}
__device__ __forceinline__ float2 df_div(float2 a, float2 b) {
  const float q1 = a.x / b.x;
  const float2 r = df_add(a, df_neg(df_mulf(b, q1)));
  return df_fast_sum(q1, r.x / b.x);
}
__device__ __forceinline__ float2 df_from_double(double x) {
  const float h = __double2float_rn(x);
  return make_float2(h, __double2float_rn(x - (double)h));
}
__device__ __forceinline__ double df_to_double(float2 a) { return (double)a.x + (double)a.y; }
__device__ __forceinline__ float2 z2f() { return make_float2(0.f, 0.f); }
__device__ __forceinline__ float2 df_shfl_xor(unsigned mask, float2 v, int o) {
  return make_float2(__shfl_xor_sync(mask, v.x, o), __shfl_xor_sync(mask, v.y, o));
}
__device__ __forceinline__ float2 df_shfl(unsigned mask, float2 v, int src) {
  return make_float2(__shfl_sync(mask, v.x, src), __shfl_sync(mask, v.y, src));
}

// ---------------------------------------------------------------------------
// One-sided (Hestenes) Jacobi on the m columns (length m <= 64) of the column-major
// matrix B (leading dimension ld), accumulating the rotations in J, until no pair
// has |b_p . b_q| > tol |b_p| |b_q| and > 1e-30 |B|_F^2 (pairs negligible against
// the whole matrix are left alone: rotating rounding noise never converges and
// cannot change the significant directions).  Pairs follow the round-robin order;
// a half-warp owns a pair (each of its 16 lanes holds up to 4 entries of a column),
// so the 8 warps of a CTA rotate 16 disjoint pairs at once.  Squared column norms
// are recomputed at the start of every sweep and updated in between (a rotation
// with tangent t annihilating gamma = b_p . b_q maps them to alpha - t gamma and
// beta + t gamma).  The rotation is computed by the first lane of the half-warp.
// Block-wide; nrm holds m values of shared scratch (flag is unused).
// ---------------------------------------------------------------------------
#define JAC_PER 4   // entries per lane: m <= 16 * JAC_PER

__device__ __forceinline__ float half_sum(float v, unsigned hm) {
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(hm, v, o);
  return v;
}
__device__ __forceinline__ float2 half_sum_df(float2 v, unsigned hm) {
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) v = df_add(v, df_shfl_xor(hm, v, o));
  return v;
}

// FP32 sweeps.  Every lane of the half-warp computes the rotation itself (no
// broadcasts) with the fast reciprocal / reciprocal-square-root units: any exactly
// orthogonal rotation that reduces b_p . b_q will do, and c = (1 + t^2)^-1/2, s = c t
// is orthogonal to FP32 rounding whatever t is.  Each thread keeps the largest
// relative off-diagonal |b_p . b_q| / (|b_p| |b_q|) it saw; the sweep ends the
// iteration when the block-wide largest is <= tol (nothing was rotated) or below stop
// (in the quadratic regime that leaves them at ~stop^2).
__device__ __forceinline__ void jacobi_f32(float* Bc, float* Jc, int m, int ld, int* flag,
                                           float* nrm, float tol, float stop, int max_sweeps) {
  (void)flag;
  const int lane = threadIdx.x & 31, hl = lane & 15, half = lane >> 4;
  const int slot0 = (threadIdx.x >> 5) * 2 + half, nslot = (blockDim.x >> 5) * 2;
  const unsigned hm = half ? 0xffff0000u : 0x0000ffffu;
  const int mm = m + (m & 1);
  __shared__ double jred[40];
  double nf = 0.0;
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    double x = (double)Bc[(e / m) * ld + e % m];
    nf += x * x;
  }
  const float abs_thr = (float)(1e-30 * block_sum(nf, jred));
  for (int sweep = 0; sweep < max_sweeps && m > 1; ++sweep) {
    for (int j = slot0; j < m; j += nslot) {
      float s2 = 0.f;
#pragma unroll
      for (int i = 0; i < JAC_PER; ++i) {
        const int l = hl + 16 * i;
        if (l < m) s2 = __fmaf_rn(Bc[j * ld + l], Bc[j * ld + l], s2);
      }
      s2 = half_sum(s2, hm);
      if (hl == 0) nrm[j] = s2;
    }
    __syncthreads();
    float lmax = 0.f;
    for (int r = 0; r < mm - 1; ++r) {
      for (int pi = slot0; pi < mm / 2; pi += nslot) {
        int p, q;
        rr_pair(mm, r, pi, &p, &q);
        if (p >= m || q >= m) continue;
        float* bp = Bc + p * ld;
        float* bq = Bc + q * ld;
        const float al = nrm[p], be = nrm[q];      // read before this half-warp writes them
        float ga = 0.f;
#pragma unroll
        for (int i = 0; i < JAC_PER; ++i) {
          const int l = hl + 16 * i;
          if (l < m) ga = __fmaf_rn(bp[l], bq[l], ga);
        }
        ga = half_sum(ga, hm);
        const float pr = al * be;
        if (!(fabsf(ga) > abs_thr) || !(pr > 0.f)) continue;
        const float rel = fabsf(ga) * rsqrtf(pr);
        lmax = fmaxf(lmax, rel);
        if (!(rel > tol)) continue;
        const float zeta = __fdividef(be - al, 2.f * ga);
        float t;
        if (fabsf(zeta) > 1e8f) {
          t = __fdividef(0.5f, zeta);
        } else {
          const float w = 1.f + zeta * zeta;
          t = __fdividef(zeta >= 0.f ? 1.f : -1.f, fabsf(zeta) + w * rsqrtf(w));
        }
        const float c = rsqrtf(1.f + t * t), s = c * t;
        __syncwarp(hm);                              // every lane has read al, be
        if (hl == 0) {
          nrm[p] = al - t * ga;
          nrm[q] = be + t * ga;
        }
        float* jp = Jc + p * ld;
        float* jq = Jc + q * ld;
#pragma unroll
        for (int i = 0; i < JAC_PER; ++i) {
          const int l = hl + 16 * i;
          if (l < m) {
            float x = bp[l], y = bq[l];
            bp[l] = c * x - s * y; bq[l] = s * x + c * y;
            x = jp[l]; y = jq[l];
            jp[l] = c * x - s * y; jq[l] = s * x + c * y;
          }
        }
      }
      __syncthreads();
    }
    const float mrel = (float)block_max((double)lmax, jred);
    if (mrel <= tol || mrel < stop) break;
  }
}

// double-float sweeps (same algorithm; the rotation's tangent comes from the hi parts
// in FP32 and c = (1 + t^2)^-1/2 is refined by one Newton step in double-float, so
// every rotation is orthogonal to double-float rounding)
__device__ __forceinline__ void jacobi_df(float2* Bd, float2* Jd, int m, int ld, int* flag,
                                          float2* nrm, float tol, float stop, int max_sweeps) {
  (void)flag;
  const int lane = threadIdx.x & 31, hl = lane & 15, half = lane >> 4;
  const int slot0 = (threadIdx.x >> 5) * 2 + half, nslot = (blockDim.x >> 5) * 2;
  const unsigned hm = half ? 0xffff0000u : 0x0000ffffu;
  const int mm = m + (m & 1);
  __shared__ double jred[40];
  double nf = 0.0;
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    double x = (double)Bd[(e / m) * ld + e % m].x;
    nf += x * x;
  }
  const float abs_thr = (float)(1e-30 * block_sum(nf, jred));
  for (int sweep = 0; sweep < max_sweeps && m > 1; ++sweep) {
    for (int j = slot0; j < m; j += nslot) {
      float2 s2 = make_float2(0.f, 0.f);
#pragma unroll
      for (int i = 0; i < JAC_PER; ++i) {
        const int l = hl + 16 * i;
        if (l < m) s2 = df_add(s2, df_mul(Bd[j * ld + l], Bd[j * ld + l]));
      }
      s2 = half_sum_df(s2, hm);
      if (hl == 0) nrm[j] = s2;
    }
    __syncthreads();
    float lmax = 0.f;
    for (int r = 0; r < mm - 1; ++r) {
      for (int pi = slot0; pi < mm / 2; pi += nslot) {
        int p, q;
        rr_pair(mm, r, pi, &p, &q);
        if (p >= m || q >= m) continue;
        float2* bp = Bd + p * ld;
        float2* bq = Bd + q * ld;
        const float2 al = nrm[p], be = nrm[q];     // read before this half-warp writes them
        float2 ga = make_float2(0.f, 0.f);
#pragma unroll
        for (int i = 0; i < JAC_PER; ++i) {
          const int l = hl + 16 * i;
          if (l < m) ga = df_add(ga, df_mul(bp[l], bq[l]));
        }
        ga = half_sum_df(ga, hm);
        const float pr = al.x * be.x;
        if (!(fabsf(ga.x) > abs_thr) || !(pr > 0.f)) continue;
        const float rel = fabsf(ga.x) * rsqrtf(pr);
        lmax = fmaxf(lmax, rel);
        if (!(rel > tol)) continue;
        const float zeta = __fdividef(df_add(be, df_neg(al)).x, 2.f * ga.x);
        float t;
        if (fabsf(zeta) > 1e8f) {
          t = __fdividef(0.5f, zeta);
        } else {
          const float w = 1.f + zeta * zeta;
          t = __fdividef(zeta >= 0.f ? 1.f : -1.f, fabsf(zeta) + w * rsqrtf(w));
        }
        // w = 1 + t^2 exactly enough; c = w^-1/2 by one Newton step from rsqrtf
        const float2 w = df_add(make_float2(1.f, 0.f), df_mulf(make_float2(t, 0.f), t));
        const float y0 = rsqrtf(w.x);
        const float2 h = df_add(make_float2(1.f, 0.f), df_neg(df_mulf(df_mulf(w, y0), y0)));
        const float2 c = df_add(make_float2(y0, 0.f), df_mulf(h, 0.5f * y0));
        const float2 s = df_mulf(c, t);
        __syncwarp(hm);                              // every lane has read al, be
        if (hl == 0) {
          const float2 tg = df_mulf(ga, t);
          nrm[p] = df_add(al, df_neg(tg));
          nrm[q] = df_add(be, tg);
        }
        const float2 ns = df_neg(s);
        float2* jp = Jd + p * ld;
        float2* jq = Jd + q * ld;
#pragma unroll
        for (int i = 0; i < JAC_PER; ++i) {
          const int l = hl + 16 * i;
          if (l < m) {
            float2 x = bp[l], y = bq[l];
            bp[l] = df_add(df_mul(c, x), df_mul(ns, y));
            bq[l] = df_add(df_mul(s, x), df_mul(c, y));
            x = jp[l]; y = jq[l];
            jp[l] = df_add(df_mul(c, x), df_mul(ns, y));
            jq[l] = df_add(df_mul(s, x), df_mul(c, y));
          }
        }
      }
      __syncthreads();
    }
    const float mrel = (float)block_max((double)lmax, jred);
    if (mrel <= tol || mrel < stop) break;
  }
}

// ---------------------------------------------------------------------------
// Column-per-lane one-sided Jacobi for at most 32 columns (the same iteration and
// stopping rules as jacobi_f32 / jacobi_df, laid out for latency): lane j of every
// warp holds column j of B (and of J) in registers, the rows interleaved over the
// block's JW_WARPS warps (row i in warp i % JW_WARPS).  In each round every column
// meets its round-robin partner: the partner's entries arrive by shuffle, the dot
// product's per-warp parts are summed in a fixed order through shared memory (one
// barrier per round), and both lanes of a pair compute the same rotation from
// bit-identical inputs, so no value is broadcast.  Every warp computes every
// rotation, so the stopping test needs no block-wide reduction.  B is nr x nc
// (nr <= JW_WARPS * ROWS rows, nc <= 32 columns), J is nc x nc.
// ---------------------------------------------------------------------------
#define JW_WARPS (DD_THREADS / 32)
#define JW_JROWS ((32 + JW_WARPS - 1) / JW_WARPS)   // rows of J per warp (nc <= 32)

// Partner of index j in round r of the circle method over mm (even) indices: 0 is
// fixed and meets 1 + r; otherwise a = j - 1 meets b with a + b = 2r (mod mm - 1).
// Indices >= mm (lanes beyond the matrix) are their own partner.
__device__ __forceinline__ int jw_partner(int j, int r, int mm) {
  const int M = mm - 1, a = j - 1;
  int b = 2 * r - a;
  b = b < 0 ? b + M : b;
  b = b >= M ? b - M : b;
  int p = a == r ? 0 : 1 + b;
  p = j == 0 ? 1 + r : p;
  return j >= mm ? j : p;
}

// Sum over the warps of the per-lane value x (fixed pairwise order, identical in
// every warp).  buf: 2 x JW_WARPS x 32 values of shared memory, alternated by *ph.
template <typename T, typename Add>
__device__ __forceinline__ T jw_sum(T x, T* buf, int* ph, Add add) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T* b = buf + (*ph & 1) * JW_WARPS * 32;
  ++*ph;
  b[warp * 32 + lane] = x;
  __syncthreads();
  T u[JW_WARPS];
#pragma unroll
  for (int w = 0; w < JW_WARPS; ++w) u[w] = b[w * 32 + lane];
#pragma unroll
  for (int h = 1; h < JW_WARPS; h <<= 1)
#pragma unroll
    for (int w = 0; w + h < JW_WARPS; w += 2 * h) u[w] = add(u[w], u[w + h]);
  return u[0];
}
// The exchange buffer of the column sweeps: one per kernel, shared by every
// instantiation (2 x JW_WARPS x 32 double-float values).
__device__ __forceinline__ float2* jw_buffer() {
  __shared__ float2 jwb[2 * JW_WARPS * 32];
  return jwb;
}
struct JwAddF { __device__ float operator()(float a, float b) const { return a + b; } };
struct JwAddDF { __device__ float2 operator()(float2 a, float2 b) const { return df_add(a, b); } };

// Double-float product whose rounding does not depend on the operand order (the two
// lanes of a pair form their dot product with the operands swapped).
__device__ __forceinline__ float2 df_mul_sym(float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  const float e = __fadd_rn(__fmaf_rn(a.x, b.x, -p),
                            __fadd_rn(__fmul_rn(a.x, b.y), __fmul_rn(a.y, b.x)));
  return df_fast_sum(p, e);
}

// Rotation of the pair (lo, hi) annihilating g = b_lo . b_hi, from a = |b_lo|^2 and
// b = |b_hi|^2 (both lanes pass them in the same roles): t = sgn(z) / (|z| + (1 + z^2)^1/2),
// z = (b - a) / (2g), c = (1 + t^2)^-1/2, s = c t, written without t: with
// D = |z| + (1 + z^2)^1/2, s = sgn(z) (1 + D^2)^-1/2 and c = D |s| (three dependent
// special-function operations); for |z| > 1e8, t = 1 / (2z) and c = 1.  Returns t in *t.
__device__ __forceinline__ void jw_rotation(float a, float b, float g, float* c, float* s,
                                            float* t) {
  const float z = __fdividef(b - a, 2.f * g);
  const float az = fabsf(z);
  const float w = __fmaf_rn(z, z, 1.f);
  const float D = az + w * rsqrtf(w);
  const float q = rsqrtf(__fmaf_rn(D, D, 1.f));
  const float iD = __fdividef(1.f, D);
  const bool huge = az > 1e8f;
  const float sg = z >= 0.f ? 1.f : -1.f;
  const float th = __fdividef(0.5f, z);
  *c = huge ? 1.f : D * q;
  *s = huge ? th : sg * q;
  *t = huge ? th : sg * iD;
}

// FP32 sweeps of the column-major nr x nc Bf with J accumulated in Jf when WJ (both
// shared memory, leading dimension ld; Jf holds the starting J).  Block-wide, blockDim
// = DD_THREADS.  Same contract as jacobi_f32.
template <int ROWS, bool WJ>
__device__ __forceinline__ void jacobi_f32_cols(float* Bf, float* Jf, int nr, int nc, int ld,
                                                float tol, float stop, int max_sweeps) {
  float* xb = reinterpret_cast<float*>(jw_buffer());
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int mm = nc + (nc & 1);
  int ph = 0;
  float b[ROWS], v[JW_JROWS];
#pragma unroll
  for (int k = 0; k < ROWS; ++k) {
    const int i = warp + JW_WARPS * k;
    b[k] = (lane < nc && i < nr) ? Bf[lane * ld + i] : 0.f;
  }
#pragma unroll
  for (int k = 0; k < JW_JROWS; ++k) {
    const int i = warp + JW_WARPS * k;
    v[k] = (WJ && lane < nc && i < nc) ? Jf[lane * ld + i] : 0.f;
  }
  __syncthreads();                                 // Bf, Jf are rewritten at the end
  float al = 0.f, abs_thr = 0.f;
  for (int sweep = 0; sweep < max_sweeps && nc > 1; ++sweep) {
    {                                              // squared norms afresh every sweep
      float t = 0.f;
#pragma unroll
      for (int k = 0; k < ROWS; ++k) t = __fmaf_rn(b[k], b[k], t);
      al = jw_sum(t, xb, &ph, JwAddF());
      if (sweep == 0) abs_thr = 1e-30f * warp_sum_t(al);
    }
    float lmax = 0.f;
    for (int r = 0; r < mm - 1; ++r) {
      const int p = jw_partner(lane, r, mm);
      const float be = __shfl_sync(0xffffffffu, al, p);
      float pb[ROWS];
#pragma unroll
      for (int k = 0; k < ROWS; ++k) pb[k] = __shfl_sync(0xffffffffu, b[k], p);
      float g = 0.f;
#pragma unroll
      for (int k = 0; k < ROWS; ++k) g = __fmaf_rn(b[k], pb[k], g);
      g = jw_sum(g, xb, &ph, JwAddF());
      const float pr = al * be;
      const bool ok = p != lane && p < nc && lane < nc && fabsf(g) > abs_thr && pr > 0.f;
      const float rel = ok ? fabsf(g) * rsqrtf(pr) : 0.f;
      lmax = fmaxf(lmax, rel);
      const bool lo = lane < p;
      float c, s, t;
      jw_rotation(lo ? al : be, lo ? be : al, g, &c, &s, &t);
      const bool rot = rel > tol;
      // b_lo' = c b_lo - s b_hi, b_hi' = s b_lo + c b_hi; |b_lo'|^2 = a - t g, |b_hi'|^2 = b + t g
      c = rot ? c : 1.f;
      const float sn = rot ? (lo ? -s : s) : 0.f;
      const float tg = rot ? (lo ? -(t * g) : t * g) : 0.f;
#pragma unroll
      for (int k = 0; k < ROWS; ++k) b[k] = c * b[k] + sn * pb[k];
      al += tg;
      if (WJ) {
#pragma unroll
        for (int k = 0; k < JW_JROWS; ++k) {
          const float pv = __shfl_sync(0xffffffffu, v[k], p);
          v[k] = c * v[k] + sn * pv;
        }
      }
    }
    const float mrel = warp_max_t(lmax);
    if (mrel <= tol || mrel < stop) break;
  }
#pragma unroll
  for (int k = 0; k < ROWS; ++k) {
    const int i = warp + JW_WARPS * k;
    if (lane < nc && i < nr) Bf[lane * ld + i] = b[k];
  }
  if (WJ) {
#pragma unroll
    for (int k = 0; k < JW_JROWS; ++k) {
      const int i = warp + JW_WARPS * k;
      if (lane < nc && i < nc) Jf[lane * ld + i] = v[k];
    }
  }
  __syncthreads();
}

// Double-float sweeps, column per lane (same contract as jacobi_df; J accumulated in
// Jd when WJ).  The tangent comes from the hi parts in FP32 and c = (1 + t^2)^-1/2 is
// refined by one Newton step in double-float, so every rotation is orthogonal to
// double-float rounding.
template <int ROWS, bool WJ>
__device__ __forceinline__ void jacobi_df_cols(float2* Bd, float2* Jd, int nr, int nc, int ld,
                                               float tol, float stop, int max_sweeps,
                                               float2* nrm_out = nullptr) {
  float2* xd = jw_buffer();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int mm = nc + (nc & 1);
  int ph = 0;
  const float2 z2 = make_float2(0.f, 0.f);
  float2 b[ROWS], v[JW_JROWS];
#pragma unroll
  for (int k = 0; k < ROWS; ++k) {
    const int i = warp + JW_WARPS * k;
    b[k] = (lane < nc && i < nr) ? Bd[lane * ld + i] : z2;
  }
#pragma unroll
  for (int k = 0; k < JW_JROWS; ++k) {
    const int i = warp + JW_WARPS * k;
    v[k] = (WJ && lane < nc && i < nc) ? Jd[lane * ld + i] : z2;
  }
  __syncthreads();
  float2 al = z2;
  float abs_thr = 0.f;
  for (int sweep = 0; sweep < max_sweeps && nc > 1; ++sweep) {
    {
      float2 t = z2;
#pragma unroll
      for (int k = 0; k < ROWS; ++k) t = df_add(t, df_mul_sym(b[k], b[k]));
      al = jw_sum(t, xd, &ph, JwAddDF());
      if (sweep == 0) abs_thr = 1e-30f * warp_sum_t(al.x);
    }
    float lmax = 0.f;
    for (int r = 0; r < mm - 1; ++r) {
      const int p = jw_partner(lane, r, mm);
      const float2 be = df_shfl(0xffffffffu, al, p);
      float2 pb[ROWS];
#pragma unroll
      for (int k = 0; k < ROWS; ++k) pb[k] = df_shfl(0xffffffffu, b[k], p);
      float2 g = z2;
#pragma unroll
      for (int k = 0; k < ROWS; ++k) g = df_add(g, df_mul_sym(b[k], pb[k]));
      g = jw_sum(g, xd, &ph, JwAddDF());
      const float pr = al.x * be.x;
      const bool ok = p != lane && p < nc && lane < nc && fabsf(g.x) > abs_thr && pr > 0.f;
      const float rel = ok ? fabsf(g.x) * rsqrtf(pr) : 0.f;
      lmax = fmaxf(lmax, rel);
      const bool lo = lane < p;
      const float2 a_lo = lo ? al : be, a_hi = lo ? be : al;
      float c32, s32, t;
      jw_rotation(0.f, df_add(a_hi, df_neg(a_lo)).x, g.x, &c32, &s32, &t);
      const bool rot = rel > tol;
      // c = (1 + t^2)^-1/2 by one Newton step in double-float from rsqrtf
      const float2 w = df_add(make_float2(1.f, 0.f), df_mulf(make_float2(t, 0.f), t));
      const float y0 = rsqrtf(w.x);
      const float2 h = df_add(make_float2(1.f, 0.f), df_neg(df_mulf(df_mulf(w, y0), y0)));
      float2 c = df_add(make_float2(y0, 0.f), df_mulf(h, 0.5f * y0));
      const float2 s = df_mulf(c, t), gt = df_mulf(g, t);
      c = rot ? c : make_float2(1.f, 0.f);
      const float2 sn = rot ? (lo ? df_neg(s) : s) : z2;
      const float2 tg = rot ? (lo ? df_neg(gt) : gt) : z2;
#pragma unroll
      for (int k = 0; k < ROWS; ++k) b[k] = df_add(df_mul(c, b[k]), df_mul(sn, pb[k]));
      al = df_add(al, tg);
      if (WJ) {
#pragma unroll
        for (int k = 0; k < JW_JROWS; ++k) {
          const float2 pv = df_shfl(0xffffffffu, v[k], p);
          v[k] = df_add(df_mul(c, v[k]), df_mul(sn, pv));
        }
      }
    }
    const float mrel = warp_max_t(lmax);
    if (mrel <= tol || mrel < stop) break;
  }
  if (nrm_out) {                                   // squared column norms afresh
    float2 t = z2;
#pragma unroll
    for (int k = 0; k < ROWS; ++k) t = df_add(t, df_mul_sym(b[k], b[k]));
    t = jw_sum(t, xd, &ph, JwAddDF());
    if (warp == 0 && lane < nc) nrm_out[lane] = t;
  }
#pragma unroll
  for (int k = 0; k < ROWS; ++k) {
    const int i = warp + JW_WARPS * k;
    if (lane < nc && i < nr) Bd[lane * ld + i] = b[k];
  }
  if (WJ) {
#pragma unroll
    for (int k = 0; k < JW_JROWS; ++k) {
      const int i = warp + JW_WARPS * k;
      if (lane < nc && i < nc) Jd[lane * ld + i] = v[k];
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Column-pair sweeps for 33..64 columns (see jacobi_f32_pairs below).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float4* jw_buffer4() {
  __shared__ float4 jwb4[2 * JW_WARPS * 32];
  return jwb4;
}
struct JwAddF2 {
  __device__ float2 operator()(float2 a, float2 b) const { return make_float2(a.x + b.x, a.y + b.y); }
};
struct JwAddDF2 {
  __device__ float4 operator()(float4 a, float4 b) const {
    const float2 x = df_add(make_float2(a.x, a.y), make_float2(b.x, b.y));
    const float2 y = df_add(make_float2(a.z, a.w), make_float2(b.z, b.w));
    return make_float4(x.x, x.y, y.x, y.y);
  }
};

// Column pairs per lane (nc <= 64): lane l < np = mm / 2 (mm = nc rounded up to even) holds
// the pair (top_l, bot_l) of columns, rows interleaved over the warps as in the other
// column sweeps.  A sweep is mm - 1 rounds of the circle method: each round every lane
// rotates its own pair (one dot product, one rotation for both columns), then the columns
// move one place around the circle with top_0 fixed: top_l <- top_(l-1) (l >= 2),
// top_1 <- bot_0, bot_l <- bot_(l+1), bot_(np-1) <- top_(np-1); over mm - 1 rounds every
// pair of columns meets once.  The column indices travel with the data (a column index
// >= nc is the empty partner of odd nc), and the columns return to their places at the
// end.  Same contract as jacobi_f32_cols.
#define JW_PROWS (64 / JW_WARPS)          // rows per warp for nr <= 64 (B and J alike)

template <bool WJ>
__device__ __forceinline__ void jacobi_f32_pairs(float* Bf, float* Jf, int nr, int nc, int ld,
                                                 float tol, float stop, int max_sweeps) {
  float2* xb = jw_buffer();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int mm = nc + (nc & 1), np = mm >> 1;
  int ph = 0;
  int it = lane, ib = lane + np;                  // column indices of top and bottom
  float bt[JW_PROWS], bb[JW_PROWS], vt[JW_PROWS], vb[JW_PROWS];
#pragma unroll
  for (int k = 0; k < JW_PROWS; ++k) {
    const int i = warp + JW_WARPS * k;
    const bool on = lane < np;
    bt[k] = (on && it < nc && i < nr) ? Bf[it * ld + i] : 0.f;
    bb[k] = (on && ib < nc && i < nr) ? Bf[ib * ld + i] : 0.f;
    vt[k] = (WJ && on && it < nc && i < nc) ? Jf[it * ld + i] : 0.f;
    vb[k] = (WJ && on && ib < nc && i < nc) ? Jf[ib * ld + i] : 0.f;
  }
  __syncthreads();                                 // Bf, Jf are rewritten at the end
  float at = 0.f, ab = 0.f, abs_thr = 0.f;
  for (int sweep = 0; sweep < max_sweeps && nc > 1; ++sweep) {
    {                                              // squared norms afresh every sweep
      float2 t = make_float2(0.f, 0.f);
#pragma unroll
      for (int k = 0; k < JW_PROWS; ++k) {
        t.x = __fmaf_rn(bt[k], bt[k], t.x);
        t.y = __fmaf_rn(bb[k], bb[k], t.y);
      }
      t = jw_sum(t, xb, &ph, JwAddF2());
      at = t.x; ab = t.y;
      if (sweep == 0) abs_thr = 1e-30f * warp_sum_t(lane < np ? at + ab : 0.f);
    }
    float lmax = 0.f;
    for (int r = 0; r < mm - 1; ++r) {
      float g = 0.f;
#pragma unroll
      for (int k = 0; k < JW_PROWS; ++k) g = __fmaf_rn(bt[k], bb[k], g);
      g = jw_sum(make_float2(g, 0.f), xb, &ph, JwAddF2()).x;
      const float pr = at * ab;
      const bool ok = lane < np && it < nc && ib < nc && fabsf(g) > abs_thr && pr > 0.f;
      const float rel = ok ? fabsf(g) * rsqrtf(pr) : 0.f;
      lmax = fmaxf(lmax, rel);
      const bool lo = it < ib;                     // top is the pair's lower column
      float c, s, t;
      jw_rotation(lo ? at : ab, lo ? ab : at, g, &c, &s, &t);
      if (rel > tol) {
        // b_lo' = c b_lo - s b_hi, b_hi' = s b_lo + c b_hi; |b_lo'|^2 = a - t g, |b_hi'|^2 = b + t g
        const float st = lo ? -s : s, tg = t * g;
#pragma unroll
        for (int k = 0; k < JW_PROWS; ++k) {
          const float x = bt[k], y = bb[k];
          bt[k] = c * x + st * y;
          bb[k] = c * y - st * x;
        }
        if (WJ) {
#pragma unroll
          for (int k = 0; k < JW_PROWS; ++k) {
            const float x = vt[k], y = vb[k];
            vt[k] = c * x + st * y;
            vb[k] = c * y - st * x;
          }
        }
        at += lo ? -tg : tg;
        ab += lo ? tg : -tg;
      }
      if (np > 1) {                                // one place around the circle
        const int sp = lane > 0 ? lane - 1 : 0, sn = lane + 1 < np ? lane + 1 : lane;
#pragma unroll
        for (int k = 0; k < JW_PROWS; ++k) {
          const float pt = __shfl_sync(0xffffffffu, lane == 0 ? bb[k] : bt[k], sp);
          const float pb = __shfl_sync(0xffffffffu, bb[k], sn);
          const float own = bt[k];
          bt[k] = lane == 0 ? own : pt;
          bb[k] = lane == np - 1 ? own : pb;
        }
        if (WJ) {
#pragma unroll
          for (int k = 0; k < JW_PROWS; ++k) {
            const float pt = __shfl_sync(0xffffffffu, lane == 0 ? vb[k] : vt[k], sp);
            const float pb = __shfl_sync(0xffffffffu, vb[k], sn);
            const float own = vt[k];
            vt[k] = lane == 0 ? own : pt;
            vb[k] = lane == np - 1 ? own : pb;
          }
        }
        {
          const float pt = __shfl_sync(0xffffffffu, lane == 0 ? ab : at, sp);
          const float pb = __shfl_sync(0xffffffffu, ab, sn);
          const int qt = __shfl_sync(0xffffffffu, lane == 0 ? ib : it, sp);
          const int qb = __shfl_sync(0xffffffffu, ib, sn);
          const float oa = at;
          const int oi = it;
          at = lane == 0 ? oa : pt;
          ab = lane == np - 1 ? oa : pb;
          it = lane == 0 ? oi : qt;
          ib = lane == np - 1 ? oi : qb;
        }
      }
    }
    const float mrel = warp_max_t(lmax);
    if (mrel <= tol || mrel < stop) break;
  }
#pragma unroll
  for (int k = 0; k < JW_PROWS; ++k) {
    const int i = warp + JW_WARPS * k;
    if (lane < np && i < nr) {
      if (it < nc) Bf[it * ld + i] = bt[k];
      if (ib < nc) Bf[ib * ld + i] = bb[k];
    }
    if (WJ && lane < np && i < nc) {
      if (it < nc) Jf[it * ld + i] = vt[k];
      if (ib < nc) Jf[ib * ld + i] = vb[k];
    }
  }
  __syncthreads();
}

// Double-float sweeps on column pairs (same layout and schedule as jacobi_f32_pairs; same
// contract as jacobi_df_cols): the tangent from the hi parts in FP32, c = (1 + t^2)^-1/2
// refined by one Newton step in double-float.
template <bool WJ>
__device__ __forceinline__ void jacobi_df_pairs(float2* Bd, float2* Jd, int nr, int nc, int ld,
                                                float tol, float stop, int max_sweeps,
                                                float2* nrm_out = nullptr) {
  float4* xd = jw_buffer4();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int mm = nc + (nc & 1), np = mm >> 1;
  int ph = 0;
  const float2 z2 = make_float2(0.f, 0.f);
  int it = lane, ib = lane + np;
  float2 bt[JW_PROWS], bb[JW_PROWS], vt[WJ ? JW_PROWS : 1], vb[WJ ? JW_PROWS : 1];
#pragma unroll
  for (int k = 0; k < JW_PROWS; ++k) {
    const int i = warp + JW_WARPS * k;
    const bool on = lane < np;
    bt[k] = (on && it < nc && i < nr) ? Bd[it * ld + i] : z2;
    bb[k] = (on && ib < nc && i < nr) ? Bd[ib * ld + i] : z2;
  }
  if (WJ) {
#pragma unroll
    for (int k = 0; k < (WJ ? JW_PROWS : 1); ++k) {
      const int i = warp + JW_WARPS * k;
      const bool on = lane < np && i < nc;
      vt[k] = (on && it < nc) ? Jd[it * ld + i] : z2;
      vb[k] = (on && ib < nc) ? Jd[ib * ld + i] : z2;
    }
  }
  __syncthreads();
  float2 at = z2, ab = z2;
  float abs_thr = 0.f;
  for (int sweep = 0; sweep < max_sweeps && nc > 1; ++sweep) {
    {
      float2 t0 = z2, t1 = z2;
#pragma unroll
      for (int k = 0; k < JW_PROWS; ++k) {
        t0 = df_add(t0, df_mul_sym(bt[k], bt[k]));
        t1 = df_add(t1, df_mul_sym(bb[k], bb[k]));
      }
      const float4 t = jw_sum(make_float4(t0.x, t0.y, t1.x, t1.y), xd, &ph, JwAddDF2());
      at = make_float2(t.x, t.y); ab = make_float2(t.z, t.w);
      if (sweep == 0) abs_thr = 1e-30f * warp_sum_t(lane < np ? at.x + ab.x : 0.f);
    }
    float lmax = 0.f;
    for (int r = 0; r < mm - 1; ++r) {
      float2 g0 = z2;
#pragma unroll
      for (int k = 0; k < JW_PROWS; ++k) g0 = df_add(g0, df_mul_sym(bt[k], bb[k]));
      const float4 gs = jw_sum(make_float4(g0.x, g0.y, 0.f, 0.f), xd, &ph, JwAddDF2());
      const float2 g = make_float2(gs.x, gs.y);
      const float pr = at.x * ab.x;
      const bool ok = lane < np && it < nc && ib < nc && fabsf(g.x) > abs_thr && pr > 0.f;
      const float rel = ok ? fabsf(g.x) * rsqrtf(pr) : 0.f;
      lmax = fmaxf(lmax, rel);
      const bool lo = it < ib;
      if (rel > tol) {
        const float2 a_lo = lo ? at : ab, a_hi = lo ? ab : at;
        float c32, s32, t;
        jw_rotation(0.f, df_add(a_hi, df_neg(a_lo)).x, g.x, &c32, &s32, &t);
        const float2 w = df_add(make_float2(1.f, 0.f), df_mulf(make_float2(t, 0.f), t));
        const float y0 = rsqrtf(w.x);
        const float2 h = df_add(make_float2(1.f, 0.f), df_neg(df_mulf(df_mulf(w, y0), y0)));
        const float2 cc = df_add(make_float2(y0, 0.f), df_mulf(h, 0.5f * y0));
        const float2 ss = df_mulf(cc, t), gt = df_mulf(g, t);
        const float2 st = lo ? df_neg(ss) : ss;    // top' = c top + st bot, bot' = c bot - st top
#pragma unroll
        for (int k = 0; k < JW_PROWS; ++k) {
          const float2 x = bt[k], y = bb[k];
          bt[k] = df_add(df_mul(cc, x), df_mul(st, y));
          bb[k] = df_add(df_mul(cc, y), df_neg(df_mul(st, x)));
        }
        if (WJ) {
#pragma unroll
          for (int k = 0; k < (WJ ? JW_PROWS : 1); ++k) {
            const float2 x = vt[k], y = vb[k];
            vt[k] = df_add(df_mul(cc, x), df_mul(st, y));
            vb[k] = df_add(df_mul(cc, y), df_neg(df_mul(st, x)));
          }
        }
        at = df_add(at, lo ? df_neg(gt) : gt);
        ab = df_add(ab, lo ? gt : df_neg(gt));
      }
      if (np > 1) {
        const int sp = lane > 0 ? lane - 1 : 0, sn = lane + 1 < np ? lane + 1 : lane;
#pragma unroll
        for (int k = 0; k < JW_PROWS; ++k) {
          const float2 pt = df_shfl(0xffffffffu, lane == 0 ? bb[k] : bt[k], sp);
          const float2 pb = df_shfl(0xffffffffu, bb[k], sn);
          const float2 own = bt[k];
          bt[k] = lane == 0 ? own : pt;
          bb[k] = lane == np - 1 ? own : pb;
        }
        if (WJ) {
#pragma unroll
          for (int k = 0; k < (WJ ? JW_PROWS : 1); ++k) {
            const float2 pt = df_shfl(0xffffffffu, lane == 0 ? vb[k] : vt[k], sp);
            const float2 pb = df_shfl(0xffffffffu, vb[k], sn);
            const float2 own = vt[k];
            vt[k] = lane == 0 ? own : pt;
            vb[k] = lane == np - 1 ? own : pb;
          }
        }
        {
          const float2 pt = df_shfl(0xffffffffu, lane == 0 ? ab : at, sp);
          const float2 pb = df_shfl(0xffffffffu, ab, sn);
          const int qt = __shfl_sync(0xffffffffu, lane == 0 ? ib : it, sp);
          const int qb = __shfl_sync(0xffffffffu, ib, sn);
          const float2 oa = at;
          const int oi = it;
          at = lane == 0 ? oa : pt;
          ab = lane == np - 1 ? oa : pb;
          it = lane == 0 ? oi : qt;
          ib = lane == np - 1 ? oi : qb;
        }
      }
    }
    const float mrel = warp_max_t(lmax);
    if (mrel <= tol || mrel < stop) break;
  }
  if (nrm_out) {
    float2 t0 = z2, t1 = z2;
#pragma unroll
    for (int k = 0; k < JW_PROWS; ++k) {
      t0 = df_add(t0, df_mul_sym(bt[k], bt[k]));
      t1 = df_add(t1, df_mul_sym(bb[k], bb[k]));
    }
    const float4 t = jw_sum(make_float4(t0.x, t0.y, t1.x, t1.y), xd, &ph, JwAddDF2());
    if (warp == 0 && lane < np) {
      if (it < nc) nrm_out[it] = make_float2(t.x, t.y);
      if (ib < nc) nrm_out[ib] = make_float2(t.z, t.w);
    }
  }
#pragma unroll
  for (int k = 0; k < JW_PROWS; ++k) {
    const int i = warp + JW_WARPS * k;
    if (lane < np && i < nr) {
      if (it < nc) Bd[it * ld + i] = bt[k];
      if (ib < nc) Bd[ib * ld + i] = bb[k];
    }
  }
  if (WJ) {
#pragma unroll
    for (int k = 0; k < (WJ ? JW_PROWS : 1); ++k) {
      const int i = warp + JW_WARPS * k;
      if (lane < np && i < nc) {
        if (it < nc) Jd[it * ld + i] = vt[k];
        if (ib < nc) Jd[ib * ld + i] = vb[k];
      }
    }
  }
  __syncthreads();
}

// Two Newton-Schulz steps J <- J (3I - J^T J) / 2 on the n x n column-major Jd in
// double-float (T, W: n x n scratch), making a J orthogonal to ~1e-7 orthogonal to
// double-float rounding.
__device__ __forceinline__ void ns_orthogonalize_df(float2* Jd, float2* T, float2* W, int n,
                                                    int ld) {
  for (int it = 0; it < 2; ++it) {
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
      int i = e / n, j = e % n;
      float2 x = make_float2(0.f, 0.f);
      for (int l = 0; l < n; ++l) x = df_add(x, df_mul(Jd[i * ld + l], Jd[j * ld + l]));
      T[i * ld + j] = df_add(make_float2(i == j ? 3.f : 0.f, 0.f), df_neg(x));
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
      int c = e / n, r = e % n;
      float2 x = make_float2(0.f, 0.f);
      for (int l = 0; l < n; ++l) x = df_add(x, df_mul(Jd[l * ld + r], T[c * ld + l]));
      W[c * ld + r] = df_mulf(x, 0.5f);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
      int c = e / n, r = e % n;
      Jd[c * ld + r] = W[c * ld + r];
    }
    __syncthreads();
  }
}

// Shared scratch of jacobi_svd_mixed for leading dimension ld: the FP32 copies of B
// and J (reused as a double-float temporary afterwards), m norms, and the
// double-float B and J.
// One FP64 refinement step of approximate eigenvectors of a symmetric matrix (Ogita and
// Aishima, 2018): with R = I - V^T V, S = V^T G V, lambda_i = s_ii / (1 - r_ii),
// V <- V (I + E), e_ij = (s_ij + lambda_j r_ij) / (lambda_j - lambda_i) for separated pairs,
// r_ij / 2 within clusters and on the diagonal; the error of V maps to about its square.
// G: m x m, row-major with stride RC; V: V_ij = V[j * RC + i] (refined in place); lam: the
// refined eigenvalues (not sorted).  S and R are symmetric (upper triangles computed,
// mirrored); the norms that set the cluster threshold, the quotients of E (a first-order
// correction) and the product V E are taken in FP32.  Scratch X: 3 RC^2 doubles.  Block-wide.
static __device__ __noinline__ void refine_sym_eig(const double* G, double* V, double* lam, int m,
                                                   int RC, double* X) {
  double* T = X;
  double* S = T + RC * RC;
  double* R = S + RC * RC;
  __shared__ double rred[50];            // >= 99 floats for block_sum3f
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {            // T = G1 V
    const int i = e / m, j = e % m;
    double x = 0.0;
    for (int l = 0; l < m; ++l) x += G[i * RC + l] * V[j * RC + l];
    T[i * RC + j] = x;
  }
  __syncthreads();
  float offn = 0.f, rn = 0.f, gn = 0.f;
  const int ntri = m * (m + 1) / 2;
  for (int e = threadIdx.x; e < ntri; e += blockDim.x) {             // S = V^T T, R = I - V^T V
    int j = (int)((sqrtf(8.f * e + 1.f) - 1.f) * 0.5f);
    j += (j + 1) * (j + 2) / 2 <= e;
    j -= j * (j + 1) / 2 > e;
    const int i = e - j * (j + 1) / 2;                       // i <= j
    double x = 0.0, y = 0.0;
    for (int l = 0; l < m; ++l) {
      x += V[i * RC + l] * T[l * RC + j];
      y += V[i * RC + l] * V[j * RC + l];
    }
    const double rr = (i == j ? 1.0 : 0.0) - y;
    S[i * RC + j] = x; S[j * RC + i] = x;
    R[i * RC + j] = rr; R[j * RC + i] = rr;
    const float xf = (float)x, rf = (float)rr, gf = (float)G[i * RC + j];
    const float wgt = i == j ? 1.f : 2.f;
    if (i != j) offn += 2.f * xf * xf;
    rn += wgt * rf * rf;
    gn += wgt * gf * gf;
  }
  block_sum3f(&offn, &rn, &gn, reinterpret_cast<float*>(rred));
  const float delta = 2.f * (sqrtf(offn) + sqrtf(gn) * sqrtf(rn));   // cluster separation
  for (int i = threadIdx.x; i < m; i += blockDim.x) lam[i] = S[i * RC + i] / (1.0 - R[i * RC + i]);
  __syncthreads();
  float* Ef = reinterpret_cast<float*>(T);      // E in FP32 (T = G V is dead)
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    const int i = e / m, j = e % m;
    float x = (float)(0.5 * R[i * RC + j]);
    if (i != j) {
      const float d = (float)(lam[j] - lam[i]);
      if (fabsf(d) > delta) x = __fdividef((float)(S[i * RC + j] + lam[j] * R[i * RC + j]), d);
    }
    Ef[i * RC + j] = x;
  }
  __syncthreads();
  float* Vf = reinterpret_cast<float*>(R);      // V in FP32 (R is dead)
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    const int i = e / m, j = e % m;
    Vf[j * RC + i] = (float)V[j * RC + i];
  }
  __syncthreads();
  // V (I + E) into S (dead): V + V E with the correction V E in FP32 (E is itself a
  // first-order FP32 quantity of the size of V's error, so FP32 rounding of V E lies far
  // below FP64 rounding of V)
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    const int i = e / m, j = e % m;
    float x = 0.f;
    for (int l = 0; l < m; ++l) x = __fmaf_rn(Vf[l * RC + i], Ef[l * RC + j], x);
    S[j * RC + i] = V[j * RC + i] + (double)x;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    const int i = e / m, j = e % m;
    V[j * RC + i] = S[j * RC + i];
  }
  __syncthreads();
}

__host__ __device__ __forceinline__ size_t jacobi_mixed_scratch_bytes(int ld) {
  return sizeof(float) * (2 * ld * ld + 2 * ld) + sizeof(float2) * (2 * ld * ld);
}

// FP32 variant for the mixed-precision path: the sweeps alone (columns orthogonal to
// ~1e-6, J orthogonal to ~1e-7); on return Bc = B J and Jc = J as with the FP64-accurate
// version.  Same scratch.
__device__ __forceinline__ void jacobi_svd_f32(double* Bc, double* Jc, int m, int ld, int* flag,
                                               void* scratch) {
  float* B32 = reinterpret_cast<float*>(scratch);
  float* J32 = B32 + ld * ld;
  float* n32 = J32 + ld * ld;
  if (m <= 0) return;
  __shared__ double fred[40];
  double mx = 0.0;
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) mx = fmax(mx, fabs(Bc[(e / m) * ld + e % m]));
  mx = block_max(mx, fred);
  if (!(mx > 0.0) || !isfinite(mx)) return;
  const int ex = ilogb(mx);              // scalbn: 2^-ex itself may not be representable
  for (int e = threadIdx.x; e < ld * ld; e += blockDim.x) {
    int c = e / ld, r = e % ld;
    B32[e] = (c < m && r < m) ? (float)scalbn(Bc[e], -ex) : 0.f;
    J32[e] = (c == r) ? 1.f : 0.f;
  }
  __syncthreads();
  jacobi_f32(B32, J32, m, ld, flag, n32, 1e-6f, 1e-3f, 30);
  for (int e = threadIdx.x; e < ld * ld; e += blockDim.x) {
    int c = e / ld, r = e % ld;
    if (c < m && r < m) {
      Bc[e] = scalbn((double)B32[e], ex);
      Jc[e] = (double)J32[e];
    }
  }
  __syncthreads();
}

// SVD of the m x m (m <= 64) column-major B by one-sided Jacobi, accurate to about
// 1e-13 relative to |B|: FP32 sweeps on a power-of-two scaled float copy until the
// columns are orthogonal to ~1e-6; the accumulated rotation, converted to
// double-float, is made orthogonal by two Newton-Schulz steps J <- J (3I - J^T J)/2;
// B <- B J in double-float; double-float sweeps finish (typically two or three).
// On return B J (in Bc, FP64) has orthogonal columns and Jc (FP64) is orthogonal.
// Jc must hold the identity on entry; flag and nrm as for the sweeps.
__device__ __forceinline__ void jacobi_svd_mixed(double* Bc, double* Jc, int m, int ld, int* flag,
                                                 double* nrm, void* scratch) {
  (void)nrm;
  float* B32 = reinterpret_cast<float*>(scratch);
  float* J32 = B32 + ld * ld;
  float* n32 = J32 + ld * ld;
  float2* T = reinterpret_cast<float2*>(B32);           // after the FP32 sweeps
  float2* Bd = reinterpret_cast<float2*>(n32 + 2 * ld);
  float2* Jd = Bd + ld * ld;
  if (m <= 0) return;
  __shared__ double mred[40];
  double mx = 0.0;
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) mx = fmax(mx, fabs(Bc[(e / m) * ld + e % m]));
  mx = block_max(mx, mred);
  if (!(mx > 0.0) || !isfinite(mx)) return;
  const int ex = ilogb(mx);              // scalbn: 2^-ex itself may not be representable
  for (int e = threadIdx.x; e < ld * ld; e += blockDim.x) {
    int c = e / ld, r = e % ld;
    B32[e] = (c < m && r < m) ? (float)scalbn(Bc[e], -ex) : 0.f;
    J32[e] = (c == r) ? 1.f : 0.f;
  }
  __syncthreads();
  if (m <= 32 && blockDim.x == DD_THREADS)
    jacobi_f32_cols<JW_JROWS, true>(B32, J32, m, m, ld, 1e-6f, 1e-3f, 30);
  else if (m <= 64 && blockDim.x == DD_THREADS)
    jacobi_f32_pairs<true>(B32, J32, m, m, ld, 1e-6f, 1e-3f, 30);
  else
    jacobi_f32(B32, J32, m, ld, flag, n32, 1e-6f, 1e-3f, 30);
  for (int e = threadIdx.x; e < ld * ld; e += blockDim.x) Jd[e] = make_float2(J32[e], 0.f);
  __syncthreads();
  ns_orthogonalize_df(Jd, T, Bd, m, ld);
  // B <- (sc B) J in double-float
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    int c = e / m, r = e % m;
    T[c * ld + r] = df_from_double(scalbn(Bc[c * ld + r], -ex));
  }
  __syncthreads();
  for (int e = threadIdx.x; e < ld * ld; e += blockDim.x) {
    int c = e / ld, r = e % ld;
    float2 x = make_float2(0.f, 0.f);
    if (c < m && r < m)
      for (int l = 0; l < m; ++l) x = df_add(x, df_mul(T[l * ld + r], Jd[c * ld + l]));
    Bd[e] = x;
  }
  __syncthreads();
  if (m <= 32 && blockDim.x == DD_THREADS)
    jacobi_df_cols<JW_JROWS, true>(Bd, Jd, m, m, ld, 1e-13f, 3e-7f, 10);
  else if (m <= 64 && blockDim.x == DD_THREADS)
    jacobi_df_pairs<true>(Bd, Jd, m, m, ld, 1e-13f, 3e-7f, 10);
  else
    jacobi_df(Bd, Jd, m, ld, flag, T, 1e-13f, 3e-7f, 10);
  for (int e = threadIdx.x; e < ld * ld; e += blockDim.x) {
    int c = e / ld, r = e % ld;
    if (c < m && r < m) {
      Bc[e] = scalbn(df_to_double(Bd[e]), ex);
      Jc[e] = df_to_double(Jd[e]);
    }
  }
  __syncthreads();
}

// Orthonormal basis of the column span of the nr x nc (nc <= nr <= 64) column-major
// FP64 X of full column rank (leading dimension ld), by one-sided Jacobi: on return the
// columns of X are those of X J / |X J| (J orthogonal, X J with orthogonal columns), to
// double-float accuracy (~1e-13).  FP32 sweeps on a power-of-two scaled copy accumulate
// J; J is made orthogonal by two Newton-Schulz steps and X J formed in double-float;
// double-float sweeps finish on the rotated columns (J itself is not needed further),
// whose norms give the normalisation.  Loops put whole warps on rows (warp per column,
// lane per row).  Scratch as for jacobi_svd_mixed.
__device__ __forceinline__ void orth_cols_mixed(double* X, int nr, int nc, int ld, void* scratch) {
  float* B32 = reinterpret_cast<float*>(scratch);
  float* J32 = B32 + ld * ld;
  float* n32 = J32 + ld * ld;
  float2* T = reinterpret_cast<float2*>(B32);           // after the FP32 sweeps
  float2* Bd = reinterpret_cast<float2*>(n32 + 2 * ld);
  float2* Jd = Bd + ld * ld;
  float2* nd = reinterpret_cast<float2*>(n32);          // nc squared norms
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (nr <= 0 || nc <= 0) return;
  __shared__ long long rbits[JW_WARPS + 1];
  long long mb = 0;                                     // largest |x| by its bit pattern
  for (int c = warp; c < nc; c += nw)
    for (int r = lane; r < nr; r += 32)
      mb = max(mb, __double_as_longlong(X[c * ld + r]) & 0x7fffffffffffffffll);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, o));
  if (lane == 0) rbits[warp] = mb;
  __syncthreads();
  mb = 0;
  for (int w = 0; w < nw; ++w) mb = max(mb, rbits[w]);
  const double mx = __longlong_as_double(mb);
  if (!(mx > 0.0) || mb >= 0x7ff0000000000000ll) return;
  const int ex = ilogb(mx);
  const double f = ldexp(1.0, -ex);
  for (int c = warp; c < nc; c += nw) {
    for (int r = lane; r < nr; r += 32) B32[c * ld + r] = (float)(X[c * ld + r] * f);
    for (int r = lane; r < nc; r += 32) J32[c * ld + r] = (c == r) ? 1.f : 0.f;
  }
  __syncthreads();
  if (nc > 32)                                          // then nr >= nc > 32
    jacobi_f32_pairs<true>(B32, J32, nr, nc, ld, 1e-6f, 1e-3f, 30);
  else if (nr <= 32)
    jacobi_f32_cols<32 / JW_WARPS, true>(B32, J32, nr, nc, ld, 1e-6f, 1e-3f, 30);
  else
    jacobi_f32_cols<64 / JW_WARPS, true>(B32, J32, nr, nc, ld, 1e-6f, 1e-3f, 30);
  for (int c = warp; c < nc; c += nw)
    for (int r = lane; r < nc; r += 32) Jd[c * ld + r] = make_float2(J32[c * ld + r], 0.f);
  __syncthreads();
  ns_orthogonalize_df(Jd, T, Bd, nc, ld);
  for (int c = warp; c < nc; c += nw)
    for (int r = lane; r < nr; r += 32) T[c * ld + r] = df_from_double(X[c * ld + r] * f);
  __syncthreads();
  for (int c = warp; c < nc; c += nw)
    for (int r = lane; r < nr; r += 32) {
      float2 x = make_float2(0.f, 0.f);
      for (int l = 0; l < nc; ++l) x = df_add(x, df_mul(T[l * ld + r], Jd[c * ld + l]));
      Bd[c * ld + r] = x;
    }
  __syncthreads();
  if (nc > 32)
    jacobi_df_pairs<false>(Bd, nullptr, nr, nc, ld, 1e-13f, 3e-7f, 10, nd);
  else if (nr <= 32)
    jacobi_df_cols<32 / JW_WARPS, false>(Bd, nullptr, nr, nc, ld, 1e-13f, 3e-7f, 10, nd);
  else
    jacobi_df_cols<64 / JW_WARPS, false>(Bd, nullptr, nr, nc, ld, 1e-13f, 3e-7f, 10, nd);
  for (int c = warp; c < nc; c += nw) {
    // 1 / |w_c| in double-float: one Newton step from rsqrtf
    const float2 n2 = nd[c];
    float2 y = z2f();
    if (n2.x > 0.f) {
      const float y0 = rsqrtf(n2.x);
      const float2 h = df_add(make_float2(1.f, 0.f), df_neg(df_mulf(df_mulf(n2, y0), y0)));
      y = df_add(make_float2(y0, 0.f), df_mulf(h, 0.5f * y0));
    }
    for (int r = lane; r < nr; r += 32) X[c * ld + r] = df_to_double(df_mul(Bd[c * ld + r], y));
  }
  __syncthreads();
}

}  // namespace dd
