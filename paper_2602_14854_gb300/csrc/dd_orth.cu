// Rank-revealing orthonormalisation with deterministic basis completion.
//
// One CTA per subdomain.  Serves three steps of the scheme:
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
// Method: scale by a power of two (exact), Householder QR of the copy, one-sided
// Jacobi SVD of R (Hestenes, on the rows of R, accumulating the rotations: the
// accumulated orthogonal matrix is the left singular basis of R), a singular value
// sigma_j counts as significant when sigma_j > tau * sigma_1, the significant left
// singular vectors of the input are Q_H [U_R; 0], and missing columns come in order
// from a fixed exactly-orthogonal candidate family, each Gram-Schmidt'd twice and
// accepted when its residual norm is >= accept:
//   space: cos(pi a (i+1/2)/nx_k) cos(pi b (j+1/2)/ny_k), by a+b then a descending;
//   angle: the table built at create time (P_2l(mu) x cos/sin(m phi), weighted by
//          sqrt(w)), then the unit vectors.
#include "dd_internal.cuh"
#include "dd_launch.h"

#include <math_constants.h>

namespace dd {

namespace {

struct OrthSmem {
  double* Bc;   // DD_MAXC x DD_MAXC, column-major: column j of B = R^T = row j of R
  double* Jc;   // DD_MAXC x DD_MAXC, column-major accumulated rotations
  double* tau;  // Householder scalars
  double* sig;  // singular values
  double* wv;   // dot products
  double* red;  // reduction scratch (40)
  int* perm;    // descending order of sig
  int* iv;      // integer scalars
  double* dv;   // double scalars
};

__device__ OrthSmem carve(void* base) {
  OrthSmem s;
  double* d = reinterpret_cast<double*>(base);
  s.Bc = d; d += DD_MAXC * DD_MAXC;
  s.Jc = d; d += DD_MAXC * DD_MAXC;
  s.tau = d; d += DD_MAXC;
  s.sig = d; d += DD_MAXC;
  s.wv = d; d += DD_MAXC;
  s.red = d; d += 40;
  s.dv = d; d += 8;
  s.perm = reinterpret_cast<int*>(d);
  s.iv = s.perm + DD_MAXC;
  return s;
}

}  // namespace

size_t orth_smem_bytes() {
  return sizeof(double) * (2 * DD_MAXC * DD_MAXC + 3 * DD_MAXC + 48) + sizeof(int) * (DD_MAXC + 16);
}

__global__ void __launch_bounds__(DD_THREADS) k_orth(OrthArgs a) {
  extern __shared__ double smem_raw[];
  OrthSmem sm = carve(smem_raw);
  const int k = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  const Geo& g = a.g;
  const int rows = a.spatial ? g.N[k] : g.n;
  const long rbase = a.spatial ? (long)g.rowoff[k] : (long)k * g.n;
  const double* A = a.A + rbase * a.lda;
  double* W = a.W + rbase * a.ldw;
  double* Q = a.Q + rbase * a.ldq;
  const int m = a.acols[k];
  int* iv = sm.iv;
  double* dv = sm.dv;

  int keep = 0, r_out = 0;

  if (a.mode == ORTH_COMPLETE) {
    // copy the orthonormal input columns, then pad below
    for (int i = tid; i < rows; i += blockDim.x)
      for (int t = 0; t < m; ++t) Q[(long)i * a.ldq + t] = A[(long)i * a.lda + t];
    keep = m;
    r_out = a.rout[k];
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
    for (int i = tid; i < rows; i += blockDim.x)
      for (int t = 0; t < m; ++t) W[(long)i * a.ldw + t] = A[(long)i * a.lda + t] * sc;
    __syncthreads();

    const bool zero = !(amax > 0.0) || !isfinite(amax);
    const int nref = zero ? 0 : min(m, rows);

    // ---- 2. Householder QR in place ------------------------------------------------
    for (int j = 0; j < nref; ++j) {
      double s = 0.0;
      for (int i = j + 1 + tid; i < rows; i += blockDim.x) {
        double x = W[(long)i * a.ldw + j];
        s += x * x;
      }
      double xn2 = block_sum(s, sm.red);
      if (tid == 0) {
        double alpha = W[(long)j * a.ldw + j];
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
        for (int i = j + 1 + tid; i < rows; i += blockDim.x) W[(long)i * a.ldw + j] *= vs;
        __syncthreads();
        if (tid == 0) W[(long)j * a.ldw + j] = dv[1];
        for (int c = j + 1 + warp; c < m; c += nwarps) {
          double d = (lane == 0) ? W[(long)j * a.ldw + c] : 0.0;
          for (int i = j + 1 + lane; i < rows; i += 32)
            d += W[(long)i * a.ldw + j] * W[(long)i * a.ldw + c];
          d = warp_sum(d);
          if (lane == 0) sm.wv[c] = d;
        }
        __syncthreads();
        const int nc = m - j - 1;
        if (nc > 0) {
          const long tot = (long)(rows - j) * nc;
          for (long idx = tid; idx < tot; idx += blockDim.x) {
            int i = j + (int)(idx / nc);
            int c = j + 1 + (int)(idx % nc);
            double v = (i == j) ? 1.0 : W[(long)i * a.ldw + j];
            W[(long)i * a.ldw + c] -= tj * v * sm.wv[c];
          }
        }
        __syncthreads();
      }
    }

    // ---- 3. one-sided Jacobi SVD of R ------------------------------------------------
    for (int idx = tid; idx < DD_MAXC * DD_MAXC; idx += blockDim.x) {
      int col = idx / DD_MAXC, row = idx % DD_MAXC;
      double b = 0.0;
      if (col < nref && row < nref && row >= col) b = W[(long)col * a.ldw + row];
      sm.Bc[idx] = b;
      sm.Jc[idx] = (row == col) ? 1.0 : 0.0;
    }
    __syncthreads();
    const int mm = nref + (nref & 1);
    for (int sweep = 0; sweep < 60 && nref > 1; ++sweep) {
      if (tid == 0) iv[0] = 0;
      __syncthreads();
      for (int r = 0; r < mm - 1; ++r) {
        for (int pi = warp; pi < mm / 2; pi += nwarps) {
          int p, q;
          rr_pair(mm, r, pi, &p, &q);
          if (p >= nref || q >= nref) continue;
          double* bp = sm.Bc + p * DD_MAXC;
          double* bq = sm.Bc + q * DD_MAXC;
          double al = 0.0, be = 0.0, ga = 0.0;
          for (int l = lane; l < nref; l += 32) {
            double x = bp[l], y = bq[l];
            al += x * x; be += y * y; ga += x * y;
          }
          al = warp_sum(al); be = warp_sum(be); ga = warp_sum(ga);
          if (ga != 0.0 && fabs(ga) > 2.220446049250313e-16 * sqrt(al * be)) {
            double zeta = (be - al) / (2.0 * ga);
            double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
            double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
            double* jp = sm.Jc + p * DD_MAXC;
            double* jq = sm.Jc + q * DD_MAXC;
            for (int l = lane; l < nref; l += 32) {
              double x = bp[l], y = bq[l];
              bp[l] = c * x - s * y; bq[l] = s * x + c * y;
              x = jp[l]; y = jq[l];
              jp[l] = c * x - s * y; jq[l] = s * x + c * y;
            }
            if (lane == 0) iv[0] = 1;
          }
        }
        __syncthreads();
      }
      if (iv[0] == 0) break;
      __syncthreads();
    }
    for (int j = warp; j < nref; j += nwarps) {
      double s = 0.0;
      for (int l = lane; l < nref; l += 32) s += sm.Bc[j * DD_MAXC + l] * sm.Bc[j * DD_MAXC + l];
      s = warp_sum(s);
      if (lane == 0) sm.sig[j] = sqrt(s);
    }
    __syncthreads();

    // ---- 4. rank decision (one thread) ----------------------------------------------
    if (tid == 0) {
      for (int t = 0; t < nref; ++t) sm.perm[t] = t;
      for (int t = 0; t < nref; ++t) {          // selection sort, descending, stable
        int best = t;
        for (int u = t + 1; u < nref; ++u)
          if (sm.sig[sm.perm[u]] > sm.sig[sm.perm[best]]) best = u;
        int tmp = sm.perm[t]; sm.perm[t] = sm.perm[best]; sm.perm[best] = tmp;
      }
      int p = 0;
      double s1 = nref > 0 ? sm.sig[sm.perm[0]] : 0.0;
      if (s1 > 0.0)
        for (int t = 0; t < nref; ++t)
          if (sm.sig[sm.perm[t]] > a.tau * s1) ++p;
      const double unscale = ldexp(1.0, e);
      if (a.sig_out)
        for (int t = 0; t < DD_MAXC; ++t)
          a.sig_out[(long)k * DD_MAXC + t] = t < nref ? sm.sig[sm.perm[t]] * unscale : 0.0;
      if (a.p_out) a.p_out[k] = p;
      if (a.mode == ORTH_QR) {
        r_out = a.rout[k];
        keep = min(p, r_out);
      } else {  // ORTH_AUG
        int r_tail = p;
        if (a.rank_mode == 1) {
          r_tail = nref;
          for (int r = 0; r <= nref; ++r) {
            double ss = 0.0;
            for (int t = r; t < nref; ++t) {
              double x = sm.sig[sm.perm[t]] * unscale;
              ss += x * x;
            }
            if (sqrt(ss) <= a.tol) { r_tail = r; break; }
          }
        }
        int r_sig = min(r_tail, p);
        int cap = min(min(a.r_aug_max, g.n), g.N[k]);
        int fl = max(a.r_own[k], a.r_floor);
        int rt = min(max(r_sig, fl), cap);
        r_out = rt;
        keep = min(rt, p);
        a.rt_out[k] = rt;
      }
      iv[1] = keep;
      iv[2] = r_out;
    }
    __syncthreads();
    keep = iv[1];
    r_out = iv[2];

    // ---- 5. significant left singular vectors: Q_H [U_R; 0] ----------------------------
    for (long idx = tid; idx < (long)rows * keep; idx += blockDim.x) {
      int i = (int)(idx / keep), t = (int)(idx % keep);
      Q[(long)i * a.ldq + t] = (i < nref) ? sm.Jc[sm.perm[t] * DD_MAXC + i] : 0.0;
    }
    __syncthreads();
    for (int j = nref - 1; j >= 0 && keep > 0; --j) {
      const double tj = sm.tau[j];
      if (tj == 0.0) continue;
      for (int t = warp; t < keep; t += nwarps) {
        double d = (lane == 0) ? Q[(long)j * a.ldq + t] : 0.0;
        for (int i = j + 1 + lane; i < rows; i += 32) d += W[(long)i * a.ldw + j] * Q[(long)i * a.ldq + t];
        d = warp_sum(d);
        if (lane == 0) sm.wv[t] = d;
      }
      __syncthreads();
      const long tot = (long)(rows - j) * keep;
      for (long idx = tid; idx < tot; idx += blockDim.x) {
        int i = j + (int)(idx / keep), t = (int)(idx % keep);
        double v = (i == j) ? 1.0 : W[(long)i * a.ldw + j];
        Q[(long)i * a.ldq + t] -= tj * v * sm.wv[t];
      }
      __syncthreads();
    }
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

void launch_orth(const OrthArgs& a, cudaStream_t st) {
  pbeg(st, KS_ORTH);
  k_orth<<<a.g.nsub, DD_THREADS, orth_smem_bytes(), st>>>(a);
  pend(st);
}

cudaError_t orth_init() {
  return cudaFuncSetAttribute(k_orth, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)orth_smem_bytes());
}

}  // namespace dd
