// Tensor-core (tcgen05) form of the dense Galerkin contractions of the step, for the
// DD_TF32 and DD_BF16 precisions.
//
// The factors stay FP64 in memory.  Tiles are staged in shared memory by TMA
// (cp.async.bulk.tensor), split in shared memory into a high and a low part of the
// tensor-core type (x = hi + lo to ~2^-22 |x| in TF32, ~2^-17 in BF16), and multiplied as
// hi*hi + hi*lo + lo*hi with FP32 accumulation in tensor memory: the error-compensated
// splitting of Ootomo and Yokota (2022, "Recovering single precision accuracy from Tensor
// Cores while surpassing the FP32 theoretical peak performance") for TF32 and of Henry,
// Tang and Heinecke (2019, "Leveraging the bfloat16 artificial intelligence datatype for
// higher-precision computations") for BF16, so each product carries FP32-level error
// instead of the type's own 2^-11 / 2^-8.  Results are written back in FP64.
//
//   k_tc_tall  Y = alpha A M (or Y += alpha A M): A tall (rows x ni), M small (ni x nc),
//              per subdomain; 128-row tiles, M = 128 MMAs, double-buffered TMA loads.
//   k_tc_gram  partial Galerkin Grams D_p = A_p^T diag(w_p) B over a chunk of rows, two
//              A operands stacked along M = 128 per CTA, written to the chunk partials that
//              k_reduce sums in FP64 (the same layout as the FP64 Gram kernels).
#include <cuda.h>

#include <climits>

#include "dd_internal.cuh"
#include "dd_launch.h"
#include "dd_tc.cuh"

namespace dd {

namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn g_encode = nullptr;

// Tensor map of a row-major FP64 array (rows x ld) whose boxes are box_rows x ld
// (ld even: rows start on 16-byte boundaries).  Rows outside the array read as zero.
bool make_map(CUtensorMap* m, const double* ptr, int ld, long rows, int box_rows) {
  if (!g_encode || (ld & 1) || ld > 256 || rows < 1) return false;
  cuuint64_t dims[2] = {(cuuint64_t)ld, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 8};
  cuuint32_t box[2] = {(cuuint32_t)ld, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  return g_encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<double*>(ptr), dims, strides,
                  box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

constexpr uint32_t kWait = 1u << 21;   // polls of a bounded mbarrier wait (about a second)

// Split f into the operand byte offset `off` of the hi (base) and lo (base + lo_off)
// planes.
template <int FMT>
__device__ __forceinline__ void put_split(uint8_t* base, uint32_t lo_off, uint32_t off, float f) {
  if (FMT == tc::FMT_TF32) {
    uint32_t h, l;
    tc::split_tf32(f, &h, &l);
    *reinterpret_cast<uint32_t*>(base + off) = h;
    *reinterpret_cast<uint32_t*>(base + lo_off + off) = l;
  } else {
    uint16_t h, l;
    tc::split_bf16(f, &h, &l);
    *reinterpret_cast<uint16_t*>(base + off) = h;
    *reinterpret_cast<uint16_t*>(base + lo_off + off) = l;
  }
}

// hi*hi + hi*lo + lo*hi over nslab K-slabs of 32 bytes (accumulating into d from `acc`)
template <int FMT>
__device__ __forceinline__ void mma_split(uint32_t d, uint32_t a_hi, uint32_t a_lo, uint32_t b_hi,
                                          uint32_t b_lo, int nslab, uint32_t sbo_a,
                                          uint32_t sbo_b, uint32_t id, uint32_t acc) {
  const uint32_t as[3] = {a_hi, a_lo, a_hi}, bs[3] = {b_lo, b_hi, b_hi};
#pragma unroll
  for (int p = 0; p < 3; ++p)
    for (int s = 0; s < nslab; ++s) {
      const uint64_t ad = tc::sdesc(as[p] + 256 * s, 128, sbo_a);
      const uint64_t bd = tc::sdesc(bs[p] + 256 * s, 128, sbo_b);
      if (FMT == tc::FMT_TF32) tc::mma_tf32(d, ad, bd, id, acc);
      else tc::mma_bf16(d, ad, bd, id, acc);
      acc = 1;
    }
}

}  // namespace

// ---------------------------------------------------------------------------------------
// tall x small:  Y = alpha A M  (or Y += alpha A M)
// ---------------------------------------------------------------------------------------
struct TcTall {
  Geo g;
  int spatial;
  int lda;                          // leading dimension of A (its tensor map's box width)
  const int* ninner; int ninner_fix;
  const double* Bm; int bsmall;     // M: small slot bsmall of smbase, or Bm + k RC^2 (bsmall < 0)
  const double* smbase;
  const int* ncols; int ncols_fix;
  double* Y; int ldy;
  double alpha; int accumulate;     // accumulate: Y += alpha A M on columns < nc only
  int tps;                          // 128-row tiles per subdomain (of the largest)
  unsigned* status;
};

#define TT_ROWS 128
#define TT_THREADS 256
#define TT_STAGE (TT_ROWS * DD_MAXC * 8)          // 64 KiB: FP64 tile, then its hi / lo planes
#define TT_BPLANE (DD_MAXC * DD_MAXC * 4)         // 16 KiB: one plane of M^T
size_t tc_tall_smem() { return 1024 + 2 * TT_STAGE + 2 * TT_BPLANE; }

// CTA b takes a contiguous range of the (subdomain, 128-row tile) pairs; the tile after
// the current one is loaded by TMA while the current one is split and multiplied.  Eight
// warps split; warp w reads TMEM lanes 32 (w % 4).. and the 16-column groups of parity w / 4.
template <int FMT>
__global__ void __launch_bounds__(TT_THREADS, 1) k_tc_tall(const __grid_constant__ CUtensorMap mapA,
                                                           TcTall a) {
  extern __shared__ uint8_t raw_tt[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(raw_tt) + 1023) &
                                             ~uintptr_t(1023));
  uint8_t* stage[2] = {base, base + TT_STAGE};
  uint8_t* bop = base + 2 * TT_STAGE;
  __shared__ uint64_t bar_tma[2], bar_mma;
  __shared__ uint32_t tmem_s;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int RC = a.g.RC, es = FMT == tc::FMT_TF32 ? 4 : 2, kq = 32 / es;
  const long ntot = (long)a.g.nsub * a.tps;
  const long f0 = blockIdx.x * ntot / gridDim.x, f1 = (blockIdx.x + 1) * ntot / gridDim.x;
  auto rows_of = [&](int k) { return a.spatial ? a.g.N[k] : a.g.n; };
  auto valid = [&](long f) { return (int)(f % a.tps) * TT_ROWS < rows_of((int)(f / a.tps)); };
  auto next_valid = [&](long f) {
    while (f < f1 && !valid(f)) ++f;
    return f;
  };
  auto row0 = [&](long f) {
    const int k = (int)(f / a.tps);
    return (a.spatial ? (long)a.g.rowoff[k] : (long)k * a.g.n) + (long)(f % a.tps) * TT_ROWS;
  };
  long f = next_valid(f0);
  if (f >= f1) return;                                // nothing here (before any setup)
  if (tid == 0) {
    tc::mbar_init(&bar_tma[0], 1);
    tc::mbar_init(&bar_tma[1], 1);
    tc::mbar_init(&bar_mma, 1);
    tc::mbar_init_fence();
  }
  if (warp == 0) tc::tmem_alloc(&tmem_s, 64);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_s;
  const uint32_t box_bytes = (uint32_t)TT_ROWS * a.lda * 8;
  if (tid == 0) {
    tc::mbar_arrive_expect_tx(&bar_tma[0], box_bytes);
    tc::tma_load_2d(stage[0], &mapA, 0, (int)row0(f), &bar_tma[0]);
  }
  int kB = -1, it = 0;
  bool alive = true;
  for (; f < f1 && alive; f = next_valid(f + 1), ++it) {
    const int buf = it & 1;
    const long fn = next_valid(f + 1);
    if (tid == 0 && fn < f1) {                         // the other buffer's MMA completed
      tc::mbar_arrive_expect_tx(&bar_tma[buf ^ 1], box_bytes);
      tc::tma_load_2d(stage[buf ^ 1], &mapA, 0, (int)row0(fn), &bar_tma[buf ^ 1]);
    }
    const int k = (int)(f / a.tps), rows = rows_of(k);
    const int r0 = (int)(f % a.tps) * TT_ROWS;
    const int ni = a.ninner ? a.ninner[k] : a.ninner_fix;
    const int nc = a.ncols ? a.ncols[k] : a.ncols_fix;
    const int Kp = ni <= kq ? kq : (ni + kq - 1) / kq * kq;
    const int KB = Kp * es;
    const int N = nc <= 16 ? 16 : (nc + 15) / 16 * 16;
    count_work(a.g, KS_TC_TALL, 2.0 * min(TT_ROWS, rows - r0) * ni * nc);
    if (k != kB) {                                     // M^T as the B operand (N x Kp)
      const double* Mk = a.bsmall >= 0 ? a.smbase + ((long)k * NSMALL + a.bsmall) * RC * RC
                                       : a.Bm + (long)k * RC * RC;
      for (int e = tid; e < N * Kp; e += TT_THREADS) {
        const int n = e / Kp, kk = e - n * Kp;
        const float x = (n < nc && kk < ni) ? tc::f64_to_f32(Mk[kk * RC + n]) : 0.f;
        put_split<FMT>(bop, TT_BPLANE, tc::op_off(n, kk * es, KB), x);
      }
      kB = k;
    }
    const bool got = tc::mbar_wait(&bar_tma[buf], (it >> 1) & 1, kWait);
    // split the FP64 tile in place: every value read before any plane is written
    const double* st = reinterpret_cast<const double*>(stage[buf]);
    float v[DD_MAXC / 2];
#pragma unroll
    for (int j = 0; j < DD_MAXC / 2; ++j) {
      v[j] = 0.f;
      const int e = tid + TT_THREADS * j;
      if (e < TT_ROWS * Kp) {
        const int r = e / Kp, kk = e - r * Kp;
        if (got && kk < ni && r0 + r < rows) v[j] = tc::f64_to_f32(st[r * a.lda + kk]);
      }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < DD_MAXC / 2; ++j) {
      const int e = tid + TT_THREADS * j;
      if (e < TT_ROWS * Kp) {
        const int r = e / Kp, kk = e - r * Kp;
        put_split<FMT>(stage[buf], TT_STAGE / 2, tc::op_off(r, kk * es, KB), v[j]);
      }
    }
    tc::fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      const uint32_t sa = tc::smem_u32(stage[buf]), sb = tc::smem_u32(bop);
      mma_split<FMT>(tmem, sa, sa + TT_STAGE / 2, sb, sb + TT_BPLANE, Kp / kq, 8 * KB, 8 * KB,
                     tc::idesc(FMT, 128, N), 0);
      tc::mma_commit(&bar_mma);
    }
    __syncwarp();
    const bool done = tc::mbar_wait(&bar_mma, it & 1, kWait);
    tc::fence_after_sync();
    const int r = r0 + (warp & 3) * 32 + lane;
    double* y = a.Y + (row0(f) - r0 + r) * a.ldy;
    for (int c0 = (warp >> 2) * 16; c0 < N; c0 += 32) {
      float d[16];
      tc::tmem_ld16(tmem + ((uint32_t)((warp & 3) * 32) << 16) + c0, d);
      if (r < rows) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int c = c0 + j;
          const double x = tc::f32_to_f64(d[j]);
          if (c < nc) y[c] = a.accumulate ? y[c] + a.alpha * x : (a.alpha == 1.0 ? x : a.alpha * x);
          else if (!a.accumulate && c < a.ldy) y[c] = 0.0;
        }
      }
    }
    if (r < rows && !a.accumulate && warp < 4)
      for (int c = N; c < a.ldy; ++c) y[c] = 0.0;
    tc::fence_before_sync();
    alive = __syncthreads_and(got && done) != 0;        // block-uniform
    if (!alive && tid == 0) atomicOr(a.status, (unsigned)ST_TIMEOUT);
  }
  if (!alive && tid == 0) {                           // bounded waits for work in flight
    tc::mbar_wait(&bar_mma, (it - 1) & 1, kWait);
    if (f < f1) tc::mbar_wait(&bar_tma[it & 1], (it >> 1) & 1, kWait);
  }
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 64);
}

// ---------------------------------------------------------------------------------------
// Galerkin Grams:  D_p = A_p^T diag(w_p) B  over a chunk of rows
// ---------------------------------------------------------------------------------------
#define TG_ROWS 32                                  // rows (the MMA's K) per stage
#define TG_THREADS 256
#define TG_STAGE (TG_ROWS * DD_MAXC * 8)            // 16 KiB FP64 tile
#define TG_APLANE (128 * TG_ROWS * 4)               // 16 KiB: one plane of the stacked A^T
#define TG_BPLANE (DD_MAXC * TG_ROWS * 4)           // 8 KiB: one plane of B^T
#define TG_OPS (2 * TG_APLANE + 2 * TG_BPLANE)      // one set of operands (hi and lo)
size_t tc_gram_smem() { return 1024 + 2 * 3 * TG_STAGE + 2 * TG_OPS; }

// One CTA per (row chunk, subdomain, source pair).  Stages of 32 rows: the FP64 tiles of
// the next stage load (TMA) while the current stage is split; the operands alternate
// between two buffers, each guarded by its own MMA barrier, so the split of stage s + 1
// overlaps the products of stage s.
template <int FMT>
__global__ void __launch_bounds__(TG_THREADS, 1) k_tc_gram(const __grid_constant__ CUtensorMap mapB,
                                                           const __grid_constant__ CUtensorMap mapA0,
                                                           const __grid_constant__ CUtensorMap mapA1,
                                                           TcGram a) {
  extern __shared__ uint8_t raw_tg[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(raw_tg) + 1023) &
                                             ~uintptr_t(1023));
  // stage tiles: [buf][0] B, [buf][1] A0, [buf][2] A1; operands: [buf] A hi, A lo, B hi, B lo
  auto tile = [&](int b, int t) { return base + (b * 3 + t) * TG_STAGE; };
  auto ops = [&](int b) { return base + 6 * TG_STAGE + b * TG_OPS; };
  __shared__ uint64_t bar_tma[2], bar_mma[2];
  __shared__ uint32_t tmem_s;
  __shared__ float wgt[2][TG_ROWS];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int k = blockIdx.y, c = blockIdx.x, grp = blockIdx.z, RC = a.g.RC;
  const int rows = a.spatial ? a.g.N[k] : a.g.n;
  const long rb = a.spatial ? (long)a.g.rowoff[k] : (long)k * a.g.n;
  const int ch = (rows + a.nchunk - 1) / a.nchunk;
  const int i0 = min(rows, c * ch), i1 = min(rows, i0 + ch);
  const int nb = a.bcnt ? a.bcnt[k] : a.bfix;
  const int N = nb <= 16 ? 16 : (nb + 15) / 16 * 16;
  const int es = FMT == tc::FMT_TF32 ? 4 : 2, KB = TG_ROWS * es;
  // the two sources of this CTA: column counts, row bases (own or a neighbour's rows)
  int ma[2], src[2], sh[2];
  long arb[2];
  bool from_b[2];
  for (int h = 0; h < 2; ++h) {
    src[h] = 2 * grp + h;
    ma[h] = 0;
    arb[h] = 0;
    sh[h] = 0;
    from_b[h] = false;
    if (src[h] >= a.nsrc) continue;
    const TcGramSrc& s = a.src[src[h]];
    int kk = k;
    if (s.nbside >= 0) kk = a.g.nb[k * 4 + 2 * a.axis + s.nbside];
    if (kk < 0) continue;
    ma[h] = s.cnt ? s.cnt[kk] : s.fix;
    arb[h] = a.spatial ? (long)a.g.rowoff[kk] : (long)kk * a.g.n;
    from_b[h] = s.same_as_b;
    sh[h] = s.shift ? (a.axis == 0 ? 1 : a.g.nxk[k]) : 0;
  }
  // output: every source's RC x RC partial block, written whole (zeros outside the
  // product) so that k_reduce can sum the chunk partials
  auto out_of = [&](int p) {
    return a.part + (((long)k * a.nchunk + c) * a.nblk + a.src[p].blk) * RC * RC;
  };
  const bool any = (ma[0] > 0 || ma[1] > 0) && nb > 0 && i1 > i0;
  if (!any) {
    for (int h = 0; h < 2; ++h)
      if (src[h] < a.nsrc) {
        double* o = out_of(src[h]);
        for (int e = tid; e < RC * RC; e += blockDim.x) o[e] = 0.0;
      }
    return;
  }
  count_work(a.g, KS_TC_GRAM, 2.0 * (i1 - i0) * nb * (ma[0] + ma[1]));
  if (tid == 0) {
    tc::mbar_init(&bar_tma[0], 1);
    tc::mbar_init(&bar_tma[1], 1);
    tc::mbar_init(&bar_mma[0], 1);
    tc::mbar_init(&bar_mma[1], 1);
    tc::mbar_init_fence();
  }
  if (warp == 0) tc::tmem_alloc(&tmem_s, 128);        // two FP32 accumulators of 64 columns
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_s;
  const double* om = a.axis == 0 ? a.ox : a.oy;
  const int nst = (i1 - i0 + TG_ROWS - 1) / TG_ROWS;
  auto issue = [&](int s) {                            // thread 0: the tiles of stage s
    const int b = s & 1, r0 = i0 + s * TG_ROWS;
    uint32_t bytes = (uint32_t)TG_ROWS * a.ldb * 8;
    for (int h = 0; h < 2; ++h)
      if (ma[h] > 0 && !from_b[h]) bytes += (uint32_t)TG_ROWS * a.src[src[h]].ld * 8;
    tc::mbar_arrive_expect_tx(&bar_tma[b], bytes);
    tc::tma_load_2d(tile(b, 0), &mapB, 0, (int)(rb + r0), &bar_tma[b]);
    if (ma[0] > 0 && !from_b[0])                       // a shifted source reads rows earlier
      tc::tma_load_2d(tile(b, 1), &mapA0, 0, (int)(arb[0] + r0 - sh[0]), &bar_tma[b]);
    if (ma[1] > 0 && !from_b[1])
      tc::tma_load_2d(tile(b, 2), &mapA1, 0, (int)(arb[1] + r0 - sh[1]), &bar_tma[b]);
  };
  // Every stage's products go to a fresh FP32 accumulator in TMEM (two, alternating) and
  // are added into double-float sums (TwoSum) once the stage completes: the FP32 rounding
  // then spans one 32-row stage, not the whole chunk.  Thread: row m = 32 (w % 4) + lane of
  // D, the 16-column groups of parity w / 4.
  float2 acc[2][16];
#pragma unroll
  for (int q = 0; q < 2; ++q)
#pragma unroll
    for (int j = 0; j < 16; ++j) acc[q][j] = make_float2(0.f, 0.f);
  bool ok = true;
  auto readout = [&](int j) {                          // stage j's products into acc
    const bool d = tc::mbar_wait(&bar_mma[j & 1], (j >> 1) & 1, kWait);
    ok = ok && d;
    tc::fence_after_sync();
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int c0 = (warp >> 2) * 16 + 32 * q;
      if (c0 < N) {
        float v[16];
        tc::tmem_ld16(tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)((j & 1) * 64 + c0), v);
#pragma unroll
        for (int t = 0; t < 16; ++t) acc[q][t] = df_add(acc[q][t], make_float2(v[t], 0.f));
      }
    }
    tc::fence_before_sync();
  };
  if (tid == 0) issue(0);
  int s = 0;
  for (; s < nst && ok; ++s) {
    const int b = s & 1, r0 = i0 + s * TG_ROWS, nr = min(TG_ROWS, i1 - r0);
    if (tid == 0 && s + 1 < nst) issue(s + 1);         // its buffers' stage s - 1 is split
    // (the operands of buffer b were read by stage s - 2, read out in the last iteration)
    const bool got = tc::mbar_wait(&bar_tma[b], (s >> 1) & 1, kWait);
    // row weights of the two sources (FP32)
    if (tid < 2 * TG_ROWS) {
      const int h = tid / TG_ROWS, r = tid % TG_ROWS, row = r0 + r;
      float wv = 1.f;
      if (src[h] < a.nsrc && r < nr) {
        const TcGramSrc& so = a.src[src[h]];
        const long long ob = __double_as_longlong(om[min(row, a.g.n - 1)]);
        const bool ng = ob < 0 && ob != (long long)0x8000000000000000ull;
        switch (so.wsel) {
          case W_OMEGA: wv = tc::f64_to_f32(om[row]); break;
          case W_NEG: wv = ng ? 1.f : 0.f; break;
          case W_NONNEG: wv = ng ? 0.f : 1.f; break;
          case W_OMEGA_POS: wv = ng ? 0.f : tc::f64_to_f32(om[row]); break;
          case W_OMEGA_NEG: wv = ng ? tc::f64_to_f32(om[row]) : 0.f; break;
          case W_ROW: wv = tc::f64_to_f32(so.wrow[rb + row]); break;
          default: break;
        }
      }
      wgt[h][r] = wv;
    }
    __syncthreads();
    uint8_t* op = ops(b);
    // B^T (N x 32 rows) and the stacked, weighted A^T (128 x 32 rows)
    const double* sB = reinterpret_cast<const double*>(tile(b, 0));
    for (int e = tid; e < N * TG_ROWS; e += TG_THREADS) {
      const int n = e / TG_ROWS, r = e - n * TG_ROWS;
      const float x = (got && n < nb && r < nr) ? tc::f64_to_f32(sB[r * a.ldb + n]) : 0.f;
      put_split<FMT>(op + 2 * TG_APLANE, TG_BPLANE, tc::op_off(n, r * es, KB), x);
    }
    for (int e = tid; e < 128 * TG_ROWS; e += TG_THREADS) {
      const int m = e / TG_ROWS, r = e - m * TG_ROWS, h = m >> 6, i = m & 63;
      float x = 0.f;
      if (got && i < ma[h] && r < nr) {
        const double* sA = reinterpret_cast<const double*>(from_b[h] ? tile(b, 0) : tile(b, 1 + h));
        const int ld = from_b[h] ? a.ldb : a.src[src[h]].ld;
        if (sh[h]) {
          // the row minus the row one cell earlier along the axis (0 before a line start),
          // formed in FP64 before the split: the Gram is then the small difference E = I - T
          // itself, not T ~ I, whose FP32-level error would dominate I - T
          const int row = r0 + r;
          const int pos = a.axis == 0 ? row % a.g.nxk[k] : row / a.g.nxk[k];
          x = tc::f64_to_f32(sB[r * a.ldb + i] - (pos == 0 ? 0.0 : sA[r * ld + i]));
        } else {
          x = tc::f64_to_f32(sA[r * ld + i]);
        }
        x *= wgt[h][r];
      }
      put_split<FMT>(op, TG_APLANE, tc::op_off(m, r * es, KB), x);
    }
    tc::fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      const uint32_t sa = tc::smem_u32(op), sb = sa + 2 * TG_APLANE;
      mma_split<FMT>(tmem + (uint32_t)(b * 64), sa, sa + TG_APLANE, sb, sb + TG_BPLANE,
                     TG_ROWS / (32 / es), 8 * KB, 8 * KB, tc::idesc(FMT, 128, N), 0u);
      tc::mma_commit(&bar_mma[b]);
    }
    if (s >= 1) readout(s - 1);                        // overlaps the products of stage s
    ok = __syncthreads_and(ok && got) != 0;            // block-uniform
  }
  if (s >= 1) readout(s - 1);
  ok = __syncthreads_and(ok) != 0;
  if (!ok) {
    if (tid == 0) {
      atomicOr(a.status, (unsigned)ST_TIMEOUT);
      if (s < nst) tc::mbar_wait(&bar_tma[s & 1], (s >> 1) & 1, kWait);   // load in flight
    }
  }
  // epilogue: the double-float sums of row m (source h = m / 64, column i = m % 64 of A_h)
  {
    const int m = (warp & 3) * 32 + lane, h = m >> 6, i = m & 63;
    double* o = src[h] < a.nsrc ? out_of(src[h]) : nullptr;
    const bool tr = o && a.src[src[h]].transpose;
    if (o && i < RC) {
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int c0 = (warp >> 2) * 16 + 32 * q;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int cc = c0 + j;
          if (cc >= RC) continue;
          const double x = (ok && c0 < N && i < ma[h] && cc < nb)
                               ? tc::f32_to_f64(acc[q][j].x) + tc::f32_to_f64(acc[q][j].y)
                               : 0.0;
          if (tr) o[cc * RC + i] = x;
          else o[i * RC + cc] = x;
        }
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 128);
}

// ---------------------------------------------------------------------------------------
// FP64-accurate tall x small products on the BF16 tensor cores (Ozaki scheme)
// ---------------------------------------------------------------------------------------
// Y = A M with the error-free splitting of Ozaki, Ogita, Oishi and Rump (2012, "Error-free
// transformations of matrix multiplication by using fast routines of matrix multiplication
// and its applications"): per 128-row tile the columns of A are equalised by powers of two
// 2^-c_k (folded into the rows of M), each row of A and each column of M get a power-of-two
// scale, and every value becomes a fixed-point integer with 56 fraction bits, split into 7
// balanced base-256 digits (|digit| <= 256: exact in BF16).  Digit products of orders s, t
// go to the TMEM accumulator of g = s + t (pairs with g <= 6; 28 of 49): every partial sum is
// an integer below 2^23, so the FP32 accumulation is exact.  The epilogue combines the seven
// sums in 64-bit integers and builds the FP64 result from bits.  Error: a few units of 2^-56
// of max|A row| max|M column| per entry (FP64 rounding of the products is 2^-53 each).  No
// FP64 instruction runs anywhere in the kernel.
#define OZ_DIG 7
#define OZ_ASL (TT_ROWS * 32 * 2)            // 8 KiB: one digit plane of 128 rows x 32 k
#define OZ_MSL (DD_MAXC * DD_MAXC * 2)       // 8 KiB: one digit plane of M^T (64 x 64)
size_t oz_tall_smem() { return 1024 + TT_STAGE + OZ_DIG * OZ_ASL + OZ_DIG * OZ_MSL; }

// biased FP64 exponent of x (0 for zero and subnormals)
__device__ __forceinline__ int f64_bexp(double x) {
  return (int)(((unsigned long long)__double_as_longlong(x) >> 52) & 0x7ff);
}
// x * 2^(56 - e) rounded to an integer (|x| < 2^e), by integer operations
__device__ __forceinline__ long long oz_fixed(double x, int e) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const int E = (int)((u >> 52) & 0x7ff);
  if (E == 0) return 0;
  const long long m = (long long)((u & 0xfffffffffffffull) | 0x10000000000000ull);
  const int sh = E - 1019 - e;
  long long T = 0;
  if (sh >= 0) T = m << sh;
  else if (sh > -62) T = (m + (1ll << (-sh - 1))) >> (-sh);
  return (u >> 63) ? -T : T;
}
// the 7 balanced base-256 digits of T (T = sum_s d_s 2^(48 - 8 s), |T| < 2^56) as BF16 bit
// patterns: the bytes of |T| by 32-bit operations, balanced from the lowest up (a byte
// >= 128 becomes byte - 256 with a carry into the next), then the sign
__device__ __forceinline__ void oz_digits(long long T, uint16_t* d) {
  const bool neg = T < 0;
  const unsigned long long U = neg ? (unsigned long long)(-T) : (unsigned long long)T;
  const unsigned tl = (unsigned)U, th = (unsigned)(U >> 32);
  int b[OZ_DIG] = {(int)(th >> 16), (int)((th >> 8) & 255u), (int)(th & 255u), (int)(tl >> 24),
                   (int)((tl >> 16) & 255u), (int)((tl >> 8) & 255u), (int)(tl & 255u)};
#pragma unroll
  for (int s = OZ_DIG - 1; s > 0; --s) {
    const int c = b[s] >= 128;
    b[s] -= c << 8;
    b[s - 1] += c;
  }
#pragma unroll
  for (int s = 0; s < OZ_DIG; ++s)
    d[s] = __bfloat16_as_ushort(__float2bfloat16_rn((float)(neg ? -b[s] : b[s])));
}
// J * 2^sc as an FP64 (round to nearest even), by integer operations
__device__ __forceinline__ double oz_to_f64(long long J, int sc) {
  if (J == 0) return 0.0;
  const unsigned long long sg = J < 0 ? 0x8000000000000000ull : 0ull;
  unsigned long long u = J < 0 ? (unsigned long long)(-J) : (unsigned long long)J;
  int msb = 63 - __clzll((long long)u);
  unsigned long long r;
  if (msb > 52) {
    const int sh = msb - 52;
    r = u >> sh;
    const unsigned long long rem = u & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
    if (rem > half || (rem == half && (r & 1ull))) ++r;
    if (r >> 53) { r >>= 1; ++msb; }
  } else {
    r = u << (52 - msb);
  }
  const int be = 1023 + msb + sc;
  if (be <= 0) return __longlong_as_double((long long)sg);
  if (be >= 2047) return __longlong_as_double((long long)(sg | 0x7ff0000000000000ull));
  return __longlong_as_double((long long)(sg | ((unsigned long long)be << 52) | (r & 0xfffffffffffffull)));
}

__global__ void __launch_bounds__(TT_THREADS, 1) k_oz_tall(const __grid_constant__ CUtensorMap mapA,
                                                           TcTall a) {
  extern __shared__ uint8_t raw_oz[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(raw_oz) + 1023) &
                                             ~uintptr_t(1023));
  const double* st = reinterpret_cast<const double*>(base);
  uint8_t* asl = base + TT_STAGE;                      // OZ_DIG planes of 128 x 32 (K-major)
  uint8_t* msl = asl + OZ_DIG * OZ_ASL;                // OZ_DIG planes of 64 x 64
  __shared__ uint64_t bar_tma, bar_mma;
  __shared__ uint32_t tmem_s;
  __shared__ int cmax[DD_MAXC], rexp[TT_ROWS], fexp[DD_MAXC];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int RC = a.g.RC;
  const long ntot = (long)a.g.nsub * a.tps;
  const long f0 = blockIdx.x * ntot / gridDim.x, f1 = (blockIdx.x + 1) * ntot / gridDim.x;
  auto rows_of = [&](int k) { return a.spatial ? a.g.N[k] : a.g.n; };
  auto valid = [&](long f) { return (int)(f % a.tps) * TT_ROWS < rows_of((int)(f / a.tps)); };
  auto next_valid = [&](long f) {
    while (f < f1 && !valid(f)) ++f;
    return f;
  };
  auto row0 = [&](long f) {
    const int k = (int)(f / a.tps);
    return (a.spatial ? (long)a.g.rowoff[k] : (long)k * a.g.n) + (long)(f % a.tps) * TT_ROWS;
  };
  long f = next_valid(f0);
  if (f >= f1) return;
  if (tid == 0) {
    tc::mbar_init(&bar_tma, 1);
    tc::mbar_init(&bar_mma, 1);
    tc::mbar_init_fence();
  }
  if (warp == 0) tc::tmem_alloc(&tmem_s, 512);          // OZ_DIG accumulators of 64 columns
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_s;
  const uint32_t box_bytes = (uint32_t)TT_ROWS * a.lda * 8;
  if (tid == 0) {
    tc::mbar_arrive_expect_tx(&bar_tma, box_bytes);
    tc::tma_load_2d(base, &mapA, 0, (int)row0(f), &bar_tma);
  }
  bool alive = true;
  int it = 0, nmma = 0;
  for (; f < f1 && alive; f = next_valid(f + 1), ++it) {
    const long fn = next_valid(f + 1);
    const int k = (int)(f / a.tps), rows = rows_of(k);
    const int r0 = (int)(f % a.tps) * TT_ROWS, nrow = min(TT_ROWS, rows - r0);
    const int ni = a.ninner ? a.ninner[k] : a.ninner_fix;
    const int nc = a.ncols ? a.ncols[k] : a.ncols_fix;
    const int N = nc <= 16 ? 16 : (nc + 15) / 16 * 16;
    count_work(a.g, KS_OZ_TALL, 2.0 * nrow * ni * nc);
    const double* Mk = a.bsmall >= 0 ? a.smbase + ((long)k * NSMALL + a.bsmall) * RC * RC
                                     : a.Bm + (long)k * RC * RC;
    if (tid < DD_MAXC) cmax[tid] = 0;
    const bool got = tc::mbar_wait(&bar_tma, it & 1, kWait);
    __syncthreads();
    // column exponents of the tile: c_k = max_r E(A[r][k]) - 1022
    for (int e = tid; e < TT_ROWS * DD_MAXC; e += TT_THREADS) {
      const int kk = e & (DD_MAXC - 1), r = e >> 6;
      if (kk < ni && r < nrow) atomicMax(&cmax[kk], f64_bexp(st[r * a.lda + kk]));
    }
    __syncthreads();
    // row exponents of A 2^-c: e_r = max_k (E(A[r][k]) - c_k) - 1022 (2 threads per row)
    {
      const int r = tid >> 1, h = tid & 1;
      int mx = -100000;
      if (r < nrow)
        for (int kk = h; kk < ni; kk += 2) {
          const int E = f64_bexp(st[r * a.lda + kk]);
          if (E) mx = max(mx, E - (cmax[kk] - 1022));
        }
      mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
      if (h == 0) rexp[r] = mx - 1022;
    }
    // column exponents of 2^c M: f_n = max_k (E(M[k][n]) + c_k) - 1022
    if (tid < DD_MAXC) {
      int mx = -100000;
      if (tid < nc)
        for (int kk = 0; kk < ni; ++kk) {
          const int E = f64_bexp(Mk[kk * RC + tid]);
          if (E && cmax[kk]) mx = max(mx, E + (cmax[kk] - 1022));
        }
      fexp[tid] = mx - 1022;
    }
    __syncthreads();
    // digit planes of (2^c M)^T: element (n, k) relative to 2^(f_n - c_k) (the N rows and
    // K halves the products read)
    const int kw = ni > 32 ? 64 : 32;
    for (int e = tid; e < N * kw; e += TT_THREADS) {
      const int n = e / kw, kk = e - n * kw;
      uint16_t d[OZ_DIG];
      const long long T = (n < nc && kk < ni && cmax[kk])
                              ? oz_fixed(Mk[kk * RC + n], fexp[n] - (cmax[kk] - 1022)) : 0;
      oz_digits(T, d);
      const uint32_t off = tc::op_off(n, kk * 2, 128);
#pragma unroll
      for (int s2 = 0; s2 < OZ_DIG; ++s2) *reinterpret_cast<uint16_t*>(msl + s2 * OZ_MSL + off) = d[s2];
    }
    const int nh = ni > 32 ? 2 : 1;
    for (int h = 0; h < nh; ++h) {
      if (h > 0) alive = tc::mbar_wait(&bar_mma, nmma++ & 1, kWait) && alive;   // planes free
      // digit planes of the tile's columns 32 h .. 32 h + 31: element (r, k) of A 2^-c
      // relative to 2^(e_r + c_k)
      for (int e = tid; e < TT_ROWS * 32; e += TT_THREADS) {
        const int r = e >> 5, kk = 32 * h + (e & 31);
        uint16_t d[OZ_DIG];
        const long long T = (got && r < nrow && kk < ni && cmax[kk])
                                ? oz_fixed(st[r * a.lda + kk], rexp[r] + (cmax[kk] - 1022)) : 0;
        oz_digits(T, d);
        const uint32_t off = tc::op_off(r, (e & 31) * 2, 64);
#pragma unroll
        for (int s2 = 0; s2 < OZ_DIG; ++s2) *reinterpret_cast<uint16_t*>(asl + s2 * OZ_ASL + off) = d[s2];
      }
      tc::fence_async_smem();
      __syncthreads();
      if (tid == 0) {
        tc::fence_after_sync();
        if (h == nh - 1 && fn < f1) {                  // the stage is no longer read
          tc::mbar_arrive_expect_tx(&bar_tma, box_bytes);
          tc::tma_load_2d(base, &mapA, 0, (int)row0(fn), &bar_tma);
        }
        const uint32_t id = tc::idesc(tc::FMT_BF16, 128, N);
        const uint32_t sa = tc::smem_u32(asl), sb = tc::smem_u32(msl);
        for (int g = 0; g < OZ_DIG; ++g)
          for (int s1 = 0; s1 <= g; ++s1)
#pragma unroll
            for (int j = 0; j < 2; ++j) {
              const uint64_t ad = tc::sdesc(sa + s1 * OZ_ASL + 256 * j, 128, 512);
              const uint64_t bd = tc::sdesc(sb + (g - s1) * OZ_MSL + 256 * (2 * h + j), 128, 1024);
              tc::mma_bf16(tmem + (uint32_t)(g * 64), ad, bd, id,
                           (h > 0 || s1 > 0 || j > 0) ? 1u : 0u);
            }
        tc::mma_commit(&bar_mma);
      }
      __syncwarp();
    }
    alive = tc::mbar_wait(&bar_mma, nmma++ & 1, kWait) && alive && got;
    tc::fence_after_sync();
    // epilogue: row m of the tile, the 16-column groups of parity w / 4
    const int m = (warp & 3) * 32 + lane, r = r0 + m;
    double* y = a.Y + (row0(f) + m) * a.ldy;
    const int er = m < nrow ? rexp[m] : 0;
    for (int c0 = (warp >> 2) * 16; c0 < N; c0 += 32) {
      float D[OZ_DIG][16];
#pragma unroll
      for (int g = 0; g < OZ_DIG; ++g)
        tc::tmem_ld16(tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(g * 64 + c0), D[g]);
      if (r < rows) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int c = c0 + j;
          if (c < nc) {
            long long J = 0;
#pragma unroll
            for (int g = 0; g < OZ_DIG - 1; ++g) J += (long long)__float2int_rn(D[g][j]) << (40 - 8 * g);
            J += (long long)(__float2int_rn(D[OZ_DIG - 1][j]) >> 8);
            y[c] = oz_to_f64(J, er + fexp[c] - 56);
          } else if (c < a.ldy) {
            y[c] = 0.0;
          }
        }
      }
    }
    if (r < rows && warp < 4)
      for (int c = N; c < a.ldy; ++c) y[c] = 0.0;
    tc::fence_before_sync();
    alive = __syncthreads_and(alive) != 0;
    if (!alive && tid == 0) atomicOr(a.status, (unsigned)ST_TIMEOUT);
  }
  if (!alive && tid == 0 && f < f1) tc::mbar_wait(&bar_tma, it & 1, kWait);   // load in flight
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

// ---------------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------------
cudaError_t tc_init() {
  if (!g_encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                     cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    g_encode = reinterpret_cast<EncodeTiledFn>(fn);
  }
  cudaError_t e;
  e = cudaFuncSetAttribute(k_tc_tall<tc::FMT_TF32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)tc_tall_smem());
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_tc_tall<tc::FMT_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)tc_tall_smem());
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_tc_gram<tc::FMT_TF32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)tc_gram_smem());
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_oz_tall, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)oz_tall_smem());
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_tc_gram<tc::FMT_BF16>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_gram_smem());
}

bool tc_tall(const Problem& P, unsigned* status, cudaStream_t st, int spatial, const double* A,
             int lda, const int* ninner, int ninner_fix, const double* Bm, int bsmall,
             const double* smbase, const int* ncols, int ncols_fix, double* Y, int ldy,
             double alpha, int accumulate) {
  const long rows_all = spatial ? P.Ntot : (long)P.g.nsub * P.g.n;
  CUtensorMap map;
  if (!make_map(&map, A, lda, rows_all, TT_ROWS)) return false;
  TcTall a;
  a.g = P.g; a.spatial = spatial; a.lda = lda; a.ninner = ninner; a.ninner_fix = ninner_fix;
  a.Bm = Bm; a.bsmall = bsmall; a.smbase = smbase; a.ncols = ncols; a.ncols_fix = ncols_fix;
  a.Y = Y; a.ldy = ldy; a.alpha = alpha; a.accumulate = accumulate; a.status = status;
  a.tps = ((spatial ? P.maxN : P.g.n) + TT_ROWS - 1) / TT_ROWS;
  const long ntot = (long)P.g.nsub * a.tps;
  const int grid = (int)std::min<long>(ntot, P.nsm);
  pbeg(st, KS_TC_TALL);
  if (P.prec == PREC_BF16)
    k_tc_tall<tc::FMT_BF16><<<grid, TT_THREADS, tc_tall_smem(), st>>>(map, a);
  else
    k_tc_tall<tc::FMT_TF32><<<grid, TT_THREADS, tc_tall_smem(), st>>>(map, a);
  pend(st);
  return true;
}

bool oz_tall(const Problem& P, unsigned* status, cudaStream_t st, int spatial, const double* A,
             int lda, const int* ninner, int ninner_fix, const double* Bm, int bsmall,
             const double* smbase, const int* ncols, int ncols_fix, double* Y, int ldy) {
  const long rows_all = spatial ? P.Ntot : (long)P.g.nsub * P.g.n;
  CUtensorMap map;
  if (!make_map(&map, A, lda, rows_all, TT_ROWS)) return false;
  TcTall a;
  a.g = P.g; a.spatial = spatial; a.lda = lda; a.ninner = ninner; a.ninner_fix = ninner_fix;
  a.Bm = Bm; a.bsmall = bsmall; a.smbase = smbase; a.ncols = ncols; a.ncols_fix = ncols_fix;
  a.Y = Y; a.ldy = ldy; a.alpha = 1.0; a.accumulate = 0; a.status = status;
  a.tps = ((spatial ? P.maxN : P.g.n) + TT_ROWS - 1) / TT_ROWS;
  const long ntot = (long)P.g.nsub * a.tps;
  const int grid = (int)std::min<long>(ntot, P.nsm);
  pbeg(st, KS_OZ_TALL);
  k_oz_tall<<<grid, TT_THREADS, oz_tall_smem(), st>>>(map, a);
  pend(st);
  return true;
}

bool tc_gram(const Problem& P, cudaStream_t st, const TcGram& a0) {
  TcGram a = a0;
  a.g = P.g;
  a.ox = P.ox;
  a.oy = P.oy;
  const long rows_all = a.spatial ? P.Ntot : (long)P.g.nsub * P.g.n;
  CUtensorMap mb, ma[2];
  if (!make_map(&mb, a.B, a.ldb, rows_all, TG_ROWS)) return false;
  // one tensor map per source slot of a CTA (slot h holds sources h, h + 2, ...: the same
  // array is required across a slot's sources)
  for (int h = 0; h < 2; ++h) {
    const TcGramSrc* s = nullptr;                     // the slot's first loaded source
    for (int p = h; p < a.nsrc; p += 2) {
      if (a.src[p].same_as_b) continue;
      if (!s) s = &a.src[p];
      else if (a.src[p].ptr != s->ptr || a.src[p].ld != s->ld) return false;
    }
    if (!make_map(&ma[h], s ? s->ptr : a.B, s ? s->ld : a.ldb, rows_all, TG_ROWS)) return false;
  }
  dim3 grid(a.nchunk, P.g.nsub, (a.nsrc + 1) / 2);
  pbeg(st, KS_TC_GRAM);
  if (P.prec == PREC_BF16)
    k_tc_gram<tc::FMT_BF16><<<grid, TG_THREADS, tc_gram_smem(), st>>>(mb, ma[0], ma[1], a);
  else
    k_tc_gram<tc::FMT_TF32><<<grid, TG_THREADS, tc_gram_smem(), st>>>(mb, ma[0], ma[1], a);
  pend(st);
  return true;
}

}  // namespace dd
