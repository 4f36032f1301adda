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
template <typename T>
__device__ __forceinline__ T warp_sum_t(T v) {
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
// pair has |b_p . b_q| > tol |b_p| |b_q| and > 1e-30 |B|_F^2 (pairs of columns
// negligible against the whole matrix are left alone: rotating rounding noise
// never converges and cannot change the significant directions).
// Column norms are recomputed at the start of every sweep and updated exactly in
// between (a rotation with tangent t that annihilates gamma = b_p . b_q maps the
// squared norms to alpha - t gamma and beta + t gamma), so each pair needs one
// dot product.  The rotation is computed by lane 0 of the warp that owns the pair.
// Block-wide; flag is shared scratch, nrm is m values of shared scratch.
__device__ __forceinline__ float rsqrt_t(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_t(double x) { return rsqrt(x); }

template <typename T>
__device__ __forceinline__ void jacobi_columns_t(T* Bc, T* Jc, int m, int ld, int* flag, T* nrm,
                                                 T tol, int max_sweeps) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int mm = m + (m & 1);
  __shared__ double jred[40];
  double nf = 0.0;
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    double x = (double)Bc[(e / m) * ld + e % m];
    nf += x * x;
  }
  const T abs_thr = (T)(1e-30 * block_sum(nf, jred));
  for (int sweep = 0; sweep < max_sweeps && m > 1; ++sweep) {
    for (int j = warp; j < m; j += nwarps) {
      T s2 = 0;
      for (int l = lane; l < m; l += 32) s2 += Bc[j * ld + l] * Bc[j * ld + l];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
      if (lane == 0) nrm[j] = s2;
    }
    if (threadIdx.x == 0) *flag = 0;
    __syncthreads();
    for (int r = 0; r < mm - 1; ++r) {
      for (int pi = warp; pi < mm / 2; pi += nwarps) {
        int p, q;
        rr_pair(mm, r, pi, &p, &q);
        if (p >= m || q >= m) continue;
        T* bp = Bc + p * ld;
        T* bq = Bc + q * ld;
        T ga = 0;
        for (int l = lane; l < m; l += 32) ga += bp[l] * bq[l];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ga += __shfl_xor_sync(0xffffffffu, ga, o);
        const T al = nrm[p], be = nrm[q];
        if (!(fabs(ga) > abs_thr && fabs(ga) > tol * sqrt(al * be))) continue;
        T c = 0, s = 0, t = 0;
        if (lane == 0) {
          const T zeta = (be - al) / (2 * ga);
          if (fabs(zeta) > (T)1e8) t = (T)0.5 / zeta;   // small angle: exact to rounding
          else t = (zeta >= 0 ? (T)1 : (T)-1) / (fabs(zeta) + sqrt((T)1 + zeta * zeta));
          c = rsqrt_t((T)1 + t * t);
          s = c * t;
          nrm[p] = al - t * ga;
          nrm[q] = be + t * ga;
          *flag = 1;
        }
        c = __shfl_sync(0xffffffffu, c, 0);
        s = __shfl_sync(0xffffffffu, s, 0);
        T* jp = Jc + p * ld;
        T* jq = Jc + q * ld;
        for (int l = lane; l < m; l += 32) {
          T x = bp[l], y = bq[l];
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

__device__ __forceinline__ void jacobi_columns(double* Bc, double* Jc, int m, int ld, int* flag,
                                               double* nrm) {
  jacobi_columns_t<double>(Bc, Jc, m, ld, flag, nrm, JACOBI_TOL, 40);
}

// Shared scratch of jacobi_svd_mixed for leading dimension ld.
__host__ __device__ __forceinline__ size_t jacobi_mixed_scratch_bytes(int ld) {
  return sizeof(float) * (2 * ld * ld + ld) + sizeof(double) * (2 * ld * ld);
}

// The same result as jacobi_columns (FP64 accuracy, Jc orthogonal to rounding),
// with most of the sweeps on the FP32 pipe: FP32 sweeps on a float copy until the
// columns are orthogonal to ~1e-6, two Newton-Schulz steps J <- J (3I - J^T J)/2
// in FP64 make the accumulated rotation orthogonal to rounding, B <- B J in FP64,
// then FP64 sweeps finish (typically two).  Jc must hold the identity on entry.
__device__ __forceinline__ void jacobi_svd_mixed(double* Bc, double* Jc, int m, int ld, int* flag,
                                                 double* nrm, void* scratch) {
  float* B32 = reinterpret_cast<float*>(scratch);
  float* J32 = B32 + ld * ld;
  float* n32 = J32 + ld * ld;
  double* T1 = reinterpret_cast<double*>(n32 + ld + (ld & 1));
  double* T2 = T1 + ld * ld;
  if (m <= 2) { jacobi_columns(Bc, Jc, m, ld, flag, nrm); return; }
  // power-of-two scaling keeps the float copy clear of underflow and overflow
  __shared__ double mred[40];
  double mx = 0.0;
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) mx = fmax(mx, fabs(Bc[(e / m) * ld + e % m]));
  mx = block_max(mx, mred);
  const double sc = (mx > 0.0 && isfinite(mx)) ? ldexp(1.0, -ilogb(mx)) : 1.0;
  for (int e = threadIdx.x; e < ld * ld; e += blockDim.x) {
    int c = e / ld, r = e % ld;
    B32[e] = (c < m && r < m) ? (float)(Bc[e] * sc) : 0.f;
    J32[e] = (c == r) ? 1.f : 0.f;
  }
  __syncthreads();
  jacobi_columns_t<float>(B32, J32, m, ld, flag, n32, 1e-6f, 30);
  // J = float -> double, two Newton-Schulz steps (column-major m x m)
  for (int e = threadIdx.x; e < ld * ld; e += blockDim.x) Jc[e] = (double)J32[e];
  __syncthreads();
  for (int it = 0; it < 2; ++it) {
    // T1 = J^T J
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
      int i = e / m, j = e % m;
      double x = 0.0;
      for (int l = 0; l < m; ++l) x += Jc[i * ld + l] * Jc[j * ld + l];
      T1[i * ld + j] = (i == j ? 3.0 : 0.0) - x;
    }
    __syncthreads();
    // T2 = J T1 / 2   (column j of T2 = J * column j of T1)
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
      int c = e / m, r = e % m;
      double x = 0.0;
      for (int l = 0; l < m; ++l) x += Jc[l * ld + r] * T1[l * ld + c];
      T2[c * ld + r] = 0.5 * x;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
      int c = e / m, r = e % m;
      Jc[c * ld + r] = T2[c * ld + r];
    }
    __syncthreads();
  }
  // B <- B J
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    int c = e / m, r = e % m;
    double x = 0.0;
    for (int l = 0; l < m; ++l) x += Bc[l * ld + r] * Jc[c * ld + l];
    T2[c * ld + r] = x;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    int c = e / m, r = e % m;
    Bc[c * ld + r] = T2[c * ld + r];
  }
  __syncthreads();
  jacobi_columns(Bc, Jc, m, ld, flag, nrm);
}

}  // namespace dd
