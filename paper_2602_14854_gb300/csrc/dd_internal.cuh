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
enum StatusBits { ST_NONFINITE = 1, ST_COMPLETION = 2, ST_RANKCAP = 4 };

// Geometry of the tiling, device arrays (read-only inside kernels).
struct Geo {
  int nsub, n, RC, MC;
  const int* N;      // cells of subdomain k
  const int* nxk;    // width
  const int* nyk;    // height
  const int* rowoff; // first spatial row of subdomain k
  const int* nb;     // 4 per subdomain: x-lo, x-hi, y-lo, y-hi neighbour, -1 = physical boundary
  const int* cx0;    // global x offset of the subdomain
  const int* cy0;    // global y offset
};

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

// Round-robin (circle method) pairing for parallel Jacobi sweeps over mm
// (even) indices: round r in [0, mm-1), pair i in [0, mm/2).
__device__ __forceinline__ void rr_pair(int mm, int r, int i, int* p, int* q) {
  int a0 = (mm > 1) ? 1 + (r % (mm - 1)) : 0;
  if (i == 0) { *p = 0; *q = a0; }
  else {
    int ai = 1 + ((i + r) % (mm - 1));
    int aj = 1 + ((mm - 1 - i + r) % (mm - 1));
    *p = ai; *q = aj;
  }
}

#define JACOBI_TOL 1e-15

// One-sided Jacobi (Hestenes) on the m columns (length m) of the column-major
// matrix Bc (leading dimension ld), accumulating the rotations in Jc, until no
// pair has |b_p . b_q| > 1e-15 |b_p| |b_q| and > 1e-30 |B|_F^2 (pairs of columns
// negligible against the whole matrix are left alone: rotating rounding noise
// never converges and cannot change the significant directions).
// Column norms are recomputed at the start of every sweep and updated exactly in
// between (a rotation with tangent t that annihilates gamma = b_p . b_q maps the
// squared norms to alpha - t gamma and beta + t gamma), so each pair needs one
// dot product.  The rotation is computed by lane 0 of the warp that owns the pair.
// Block-wide; flag is shared scratch, nrm is m doubles of shared scratch.
__device__ __forceinline__ void jacobi_columns(double* Bc, double* Jc, int m, int ld, int* flag,
                                               double* nrm) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int mm = m + (m & 1);
  __shared__ double jred[40];
  double nf = 0.0;
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    double x = Bc[(e / m) * ld + e % m];
    nf += x * x;
  }
  const double abs_thr = 1e-30 * block_sum(nf, jred);
  for (int sweep = 0; sweep < 40 && m > 1; ++sweep) {
    for (int j = warp; j < m; j += nwarps) {
      double s2 = 0.0;
      for (int l = lane; l < m; l += 32) s2 += Bc[j * ld + l] * Bc[j * ld + l];
      s2 = warp_sum(s2);
      if (lane == 0) nrm[j] = s2;
    }
    if (threadIdx.x == 0) *flag = 0;
    __syncthreads();
    for (int r = 0; r < mm - 1; ++r) {
      for (int pi = warp; pi < mm / 2; pi += nwarps) {
        int p, q;
        rr_pair(mm, r, pi, &p, &q);
        if (p >= m || q >= m) continue;
        double* bp = Bc + p * ld;
        double* bq = Bc + q * ld;
        double ga = 0.0;
        for (int l = lane; l < m; l += 32) ga += bp[l] * bq[l];
        ga = warp_sum(ga);
        const double al = nrm[p], be = nrm[q];
        if (!(fabs(ga) > abs_thr && fabs(ga) > JACOBI_TOL * sqrt(al * be))) continue;
        double c = 0.0, s = 0.0, t = 0.0;
        if (lane == 0) {
          const double zeta = (be - al) / (2.0 * ga);
          if (fabs(zeta) > 1e8) t = 0.5 / zeta;   // small angle: exact to rounding
          else t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
          c = rsqrt(1.0 + t * t);
          s = c * t;
          nrm[p] = al - t * ga;
          nrm[q] = be + t * ga;
          *flag = 1;
        }
        c = __shfl_sync(0xffffffffu, c, 0);
        s = __shfl_sync(0xffffffffu, s, 0);
        double* jp = Jc + p * ld;
        double* jq = Jc + q * ld;
        for (int l = lane; l < m; l += 32) {
          double x = bp[l], y = bq[l];
          bp[l] = c * x - s * y; bq[l] = s * x + c * y;
          x = jp[l]; y = jq[l];
          jp[l] = c * x - s * y; jq[l] = s * x + c * y;
        }
      }
      __syncthreads();
    }
    int f = *flag;
    __syncthreads();
    if (f == 0) break;
  }
}

}  // namespace dd
