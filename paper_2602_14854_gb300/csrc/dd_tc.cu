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

#include <algorithm>
#include <atomic>
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
// looked up once by tc_init; solvers may be created from several host threads
std::atomic<EncodeTiledFn> g_encode{nullptr};

// Tensor map of a row-major FP64 array (rows x ld) whose boxes are box_rows x ld
// (ld even: rows start on 16-byte boundaries).  Rows outside the array read as zero.
bool make_map(CUtensorMap* m, const double* ptr, int ld, long rows, int box_rows) {
  const EncodeTiledFn encode = g_encode.load(std::memory_order_acquire);
  if (!encode || (ld & 1) || ld > 256 || rows < 1) return false;
  cuuint64_t dims[2] = {(cuuint64_t)ld, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 8};
  cuuint32_t box[2] = {(cuuint32_t)ld, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  return encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<double*>(ptr), dims, strides,
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
  const double* A;                  // A itself (the kernels that load it without a tensor map)
  int mtrans;                       // M read transposed (the Ozaki kernel)
  const double* rowscale;           // accumulate: Y_r += rowscale_r (A M)_r (the Ozaki kernel; null: 1)
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
// and its applications").  The rows of M are equalised by powers of two, M' = diag(2^-mu) M
// with mu_k the exponent of row k's largest entry, the inverse scale folded into the columns
// of A (A' = A diag(2^mu)); each row r of A' gets the power-of-two bound 2^e_r and each column
// n of M' the bound 2^f_n, and every value becomes a fixed-point integer with 56 fraction bits
// relative to its bound (truncated), split into 7 balanced base-256 digits (the top digit is at
// most 256, the others at most 128 in magnitude: exact in BF16).  Digit products of
// orders s, t go to the TMEM accumulator of g = s + t (pairs with g <= 6; 28 of 49): with at
// most 64 terms of at most 7 pairs every partial sum is an integer below 2^24, so the FP32
// accumulation is exact.  The epilogue combines the seven sums in 64-bit integers and builds
// the FP64 result from bits.  Error: a few units of 2^-56 of max_k |A'[r][k]| max_k
// |M'[k][n]| per entry (the FP64 rounding of each product is 2^-53 of the product).  No FP64
// arithmetic runs in the kernel.
//
// A CTA (one per SM: 16 worker warps and one warp that issues the MMAs) walks a contiguous
// range of 128-row tiles.  M's digit planes
// are formed once per subdomain.  Per tile, each warp loads 8 rows straight into registers
// (16-byte loads, 8 rows x 64 bytes per instruction), takes the row bounds by shuffles and
// writes the digit planes (two digits per 32-bit shared store); one thread then issues the
// 28 x (K / 16) MMAs.  The planes are double-buffered: tile i's MMAs run while the warps
// convert tile i + 1, and tile i's epilogue (TMEM -> registers -> FP64 -> a per-warp
// transposition buffer -> whole-row stores) follows.  When two buffers of a whole row's
// planes do not fit beside M's (lda > 48), K runs in two passes of 32: the stages (one pass
// of one tile each) alternate between the two buffers all the same.
#define OZ_DIG 7
#define OZ_WORKERS 512                       // 16 warps: loads, digits, epilogue
#define OZ_THREADS (OZ_WORKERS + 32)         // + one warp that issues the MMAs
#define OZ_WARPS (OZ_WORKERS / 32)
#define OZ_NONE (-(1 << 20))                 // exponent of an all-zero row / column
#define OZ_EPI (OZ_WARPS * 32 * 5 * 8)       // epilogue buffers: 32 rows x 4 (+1) per warp
#define OZ_SMEM_LIMIT (227 * 1024 - 4096)    // dynamic shared memory (the static part is < 4 KiB)

struct OzPlan {
  int KP, KA, npass, nbuf;                   // K extent of M's planes, of a pass; passes; buffers (2)
  size_t mpl, apl, abuf, total;              // bytes: one M plane, one A plane, one A buffer, all
};
// the shared-memory plan for inner dimensions up to lda (even, <= 64)
OzPlan oz_plan(int lda, size_t limit) {
  OzPlan p;
  p.KP = (lda + 15) / 16 * 16;
  p.mpl = (size_t)DD_MAXC * 2 * p.KP;
  for (int mode = 0; mode < 2; ++mode) {
    p.KA = mode ? 32 : p.KP;
    p.nbuf = 2;
    p.npass = (p.KP + p.KA - 1) / p.KA;
    p.apl = (size_t)TT_ROWS * 2 * p.KA;
    p.abuf = std::max((size_t)OZ_DIG * p.apl, (size_t)OZ_EPI);
    p.total = 128 + OZ_DIG * p.mpl + p.nbuf * p.abuf;
    if (p.total <= limit) break;
  }
  return p;
}

// biased FP64 exponent of x (0 for zero and subnormals)
__device__ __forceinline__ int f64_bexp(double x) {
  return (int)((unsigned)(__double_as_longlong(x) >> 52) & 0x7ffu);
}
// The 7 digits of T = trunc(x 2^(56 - e)) (|x| < 2^e, so |T| < 2^56), T = sum_s d_s 2^(48 - 8 s),
// as exact FP32 values, by integer operations: with the mantissa left-aligned (implicit bit
// at bit 63) T is one right shift; adding 128 at each of the six low byte positions makes
// every low byte of V = T + 0x808080808080 equal to d_s + 128 with the borrows and carries
// of a balanced representation (d_s in [-128, 127] for s >= 1, and d_0 = V >> 48 in
// [-256, 256]); byte b becomes the FP32 (0x4B4000bb = 1.5 2^23 + b) minus 1.5 2^23 + 128.
// Signed T needs nothing more: the identity is modular.
__device__ __forceinline__ void oz_digits(double x, int e, float* d) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(u >> 32);
  const int E = (int)((hi >> 20) & 0x7ffu);
  const int sh = 1030 + e - E;                       // >= 8
  const unsigned long long m = (u << 11) | 0x8000000000000000ull;
  long long T = (E != 0 && sh < 64) ? (long long)(m >> sh) : 0ll;
  if (hi >> 31) T = -T;
  const unsigned long long V = (unsigned long long)T + 0x808080808080ull;
  const unsigned vl = (unsigned)V, vh = (unsigned)(V >> 32);
  const float c = 12583040.0f;                       // 1.5 2^23 + 128
  d[6] = __int_as_float((int)__byte_perm(vl, 0x4B400000u, 0x7650)) - c;
  d[5] = __int_as_float((int)__byte_perm(vl, 0x4B400000u, 0x7651)) - c;
  d[4] = __int_as_float((int)__byte_perm(vl, 0x4B400000u, 0x7652)) - c;
  d[3] = __int_as_float((int)__byte_perm(vl, 0x4B400000u, 0x7653)) - c;
  d[2] = __int_as_float((int)__byte_perm(vh, 0x4B400000u, 0x7650)) - c;
  d[1] = __int_as_float((int)__byte_perm(vh, 0x4B400000u, 0x7651)) - c;
  d[0] = __int_as_float(0x4B400000 + ((int)vh >> 16)) - 12582912.0f;
}
// the BF16 digits of two values packed in one word (each digit has <= 8 significant bits:
// its BF16 is the top half of its FP32)
__device__ __forceinline__ uint32_t oz_pack(float lo, float hi) {
  return __byte_perm(__float_as_uint(lo), __float_as_uint(hi), 0x7632);
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
// tcgen05.ld of 4 columns without the wait (the caller waits once for several)
__device__ __forceinline__ void oz_tmem_ld4(uint32_t taddr, uint32_t* r) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(taddr));
}

// one tile's shape
struct OzTile {
  int k, nrow, ni, nc, N;
  long row0;
};
// a warp's 8 rows of the tile: lane (rho, q) loads row 8 w + rho, columns 8 c + 2 q and
// 8 c + 2 q + 1 (c < KP / 8) with 16-byte loads (8 rows x 64 bytes per instruction)
__device__ __forceinline__ void oz_load_rows(double2 (&x)[8], const double* A, int lda,
                                             const OzTile& t, int r, int q, int KP) {
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int kk = 8 * c + 2 * q;
    x[c] = make_double2(0.0, 0.0);
    if (c < KP / 8 && r < t.nrow && kk < t.ni)
      x[c] = __ldg(reinterpret_cast<const double2*>(A + (t.row0 + r) * lda + kk));
  }
}

__global__ void __launch_bounds__(OZ_THREADS, 1) k_oz_tall(TcTall a, int KP, int KA, int npass,
                                                           int nbuf) {
  extern __shared__ uint8_t raw_oz[];
  uint8_t* msl = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(raw_oz) + 127) &
                                            ~uintptr_t(127));   // OZ_DIG planes DD_MAXC x KP
  const uint32_t MPL = DD_MAXC * 2 * KP, APL = TT_ROWS * 2 * KA;
  const uint32_t ABUF = max(OZ_DIG * APL, (uint32_t)OZ_EPI);
  uint8_t* asl0 = msl + OZ_DIG * MPL;                          // 2 x (OZ_DIG planes 128 x KA)
  __shared__ uint64_t bar_mma[2];                              // MMAs of the stages in buffer 0 / 1
  __shared__ uint32_t tmem_s;
  __shared__ int mexp[DD_MAXC], fexp[DD_MAXC], rexp[2][TT_ROWS], red[8][DD_MAXC];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool worker = warp < OZ_WARPS;
  const int RC = a.g.RC, tps = a.tps;
  const int ntot = a.g.nsub * tps;
  const int f0 = (int)((long)blockIdx.x * ntot / gridDim.x);
  const int f1 = (int)((long)(blockIdx.x + 1) * ntot / gridDim.x);
  auto rows_of = [&](int k) { return a.spatial ? a.g.N[k] : a.g.n; };
  auto next_valid = [&](int f) {
    while (f < f1 && (f % tps) * TT_ROWS >= rows_of(f / tps)) ++f;
    return f;
  };
  auto shape = [&](int f) {
    OzTile t;
    t.k = f / tps;
    const int r0 = (f - t.k * tps) * TT_ROWS;
    t.nrow = min(TT_ROWS, rows_of(t.k) - r0);
    t.row0 = (a.spatial ? (long)a.g.rowoff[t.k] : (long)t.k * a.g.n) + r0;
    t.ni = a.ninner ? a.ninner[t.k] : a.ninner_fix;
    t.nc = a.ncols ? a.ncols[t.k] : a.ncols_fix;
    t.N = t.nc <= 16 ? 16 : (t.nc + 15) / 16 * 16;
    return t;
  };
  int f = next_valid(f0);
  if (f >= f1) return;
  if (tid == 0) {
    tc::mbar_init(&bar_mma[0], 1);
    tc::mbar_init(&bar_mma[1], 1);
    tc::mbar_init_fence();
  }
  if (warp == 0) tc::tmem_alloc(&tmem_s, 512);          // OZ_DIG accumulators of 64 columns
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_s;
  bool alive = true;
  // A stage is one pass of one tile: its digit planes go to buffer (stage & 1) and its MMAs
  // commit to that buffer's barrier, completing that barrier's phase (stage >> 1).
  int ns = 0, kcur = -1, tb = 0, prev_tb = 0;           // stages issued, tile parity (rexp)
  bool pending = false;                                 // a tile's MMAs issued, epilogue not done
  OzTile prev{};
  auto wait_stage = [&](int j) {
    alive = tc::mbar_wait(&bar_mma[j & 1], (j >> 1) & 1, kWait) && alive;
  };

  // epilogue of tile t (its MMAs complete; row bounds rexp[rb]), planes buffer b as scratch;
  // worker warp w: TMEM lanes 32 (w % 4) .., 4-column groups w / 4, w / 4 + 4, ...
  auto epilogue = [&](const OzTile& t, int rb, int b) {
    const int q4 = warp & 3, m = q4 * 32 + lane;
    const int er = rexp[rb][m];
    double* ebuf = reinterpret_cast<double*>(asl0 + (size_t)b * ABUF) + warp * (32 * 5);
    double* ybase = a.Y + t.row0 * a.ldy;
    for (int c0 = (warp >> 2) * 4; c0 < t.N; c0 += 16) {
      uint32_t D[OZ_DIG][4];
#pragma unroll
      for (int g = 0; g < OZ_DIG; ++g)
        oz_tmem_ld4(tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(g * t.N + c0), D[g]);
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int g = 0; g < OZ_DIG; ++g)
#pragma unroll
        for (int j = 0; j < 4; ++j) asm volatile("" : "+r"(D[g][j]));
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c = c0 + j;
        double v = 0.0;
        if (c < t.nc && m < t.nrow && alive) {
          long long J = 0;
#pragma unroll
          for (int g = 0; g < OZ_DIG - 1; ++g)
            J += (long long)__float2int_rn(__uint_as_float(D[g][j])) << (40 - 8 * g);
          J += (long long)(__float2int_rn(__uint_as_float(D[OZ_DIG - 1][j])) >> 8);
          v = oz_to_f64(J, er + fexp[c] - 56);
        }
        ebuf[lane * 5 + j] = v;
      }
      __syncwarp();
      const int cc = c0 + (lane & 3);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int rl = 8 * i + (lane >> 2), rr = q4 * 32 + rl;
        if (rr < t.nrow && cc < a.ldy) {
          double* yp = ybase + (long)rr * a.ldy + cc;
          if (!a.accumulate) *yp = ebuf[rl * 5 + (lane & 3)];
          else if (cc < t.nc) *yp += (a.rowscale ? a.rowscale[t.row0 + rr] : 1.0) * ebuf[rl * 5 + (lane & 3)];
        }
      }
      __syncwarp();
    }
    if (warp < 4 && a.ldy > t.N && !a.accumulate)       // columns N .. ldy - 1
      for (int e = lane; e < 32 * (a.ldy - t.N); e += 32) {
        const int rr = q4 * 32 + e / (a.ldy - t.N), c = t.N + e % (a.ldy - t.N);
        if (rr < t.nrow) ybase[(long)rr * a.ldy + c] = 0.0;
      }
  };
  auto finish_prev = [&]() {          // wait for prev's MMAs (its last stage), its epilogue
    wait_stage(ns - 1);
    tc::fence_after_sync();
    if (worker) epilogue(prev, prev_tb, (ns - 1) & 1);
    tc::fence_before_sync();
    alive = __syncthreads_and(alive) != 0;
    pending = false;
  };
  // MMAs of tile t, K range k0 .. k0 + KA - 1 of its planes in buffer b.  M's planes are
  // stacked along N (plane u = rows u N .. u N + N - 1) and accumulator g sits at TMEM
  // columns g N .., so one MMA of A's plane s with planes u0 .. u0 + nu - 1 adds the pairs
  // (s, u) into accumulators s + u0 .. s + u0 + nu - 1: at most 256 / N planes an MMA
  auto issue = [&](const OzTile& t, int b, int k0, int acc0) {
    tc::fence_after_sync();
    const int ns = max(k0 == 0 ? 1 : 0, (min(t.ni, k0 + KA) - k0 + 15) >> 4);
    const int nper = 256 / t.N;
    const uint32_t MPLt = (uint32_t)t.N * 2 * KP;
    const uint64_t ad0 = tc::sdesc(tc::smem_u32(asl0 + (size_t)b * ABUF), 128, 16 * KA);
    const uint64_t bd0 = tc::sdesc(tc::smem_u32(msl) + 256 * (k0 / 16), 128, 16 * KP);
    for (int j = 0; j < ns; ++j)
      for (int s1 = 0; s1 < OZ_DIG; ++s1)
        for (int u0 = 0; u0 < OZ_DIG - s1; u0 += nper) {
          const int nu = min(nper, OZ_DIG - s1 - u0);
          tc::mma_bf16(tmem + (uint32_t)((s1 + u0) * t.N), ad0 + ((s1 * APL + 256 * j) >> 4),
                       bd0 + ((u0 * MPLt + 256 * j) >> 4), tc::idesc(tc::FMT_BF16, 128, nu * t.N),
                       (acc0 || j > 0 || s1 > 0) ? 1u : 0u);
        }
    tc::mma_commit(&bar_mma[b]);
  };

  const int rho = lane & 7, q = lane >> 3, r = 8 * warp + rho;
  double2 x[8];                                          // the warp's rows of the tile
  OzTile t = shape(f);
  if (worker) oz_load_rows(x, a.A, a.lda, t, r, q, KP);
  while (alive) {
    count_work(a.g, KS_OZ_TALL, 2.0 * t.nrow * t.ni * t.nc);
    if (t.k != kcur) {
      if (pending) finish_prev();                       // its MMAs read the old M planes
      if (!alive) break;
      // ---- M's digit planes, once per subdomain: M staged as FP64 [kk][DD_MAXC] in the
      // (free) first planes buffer by coalesced loads, then bounds and digits from there
      kcur = t.k;
      const double* Mk = a.bsmall >= 0 ? a.smbase + ((long)t.k * NSMALL + a.bsmall) * RC * RC
                                       : a.Bm + (long)t.k * RC * RC;
      double* Ms = reinterpret_cast<double*>(asl0);
#pragma unroll
      for (int i = 0; i < DD_MAXC * DD_MAXC / OZ_WORKERS; ++i) {
        const int e = tid + OZ_WORKERS * i, kk = e >> 6, n = e & (DD_MAXC - 1);
        if (worker && kk < KP)
          Ms[e] = (kk < t.ni && n < t.nc)
                      ? __ldg(Mk + (a.mtrans ? (long)n * RC + kk : (long)kk * RC + n)) : 0.0;
      }
      __syncthreads();
      for (int kk = worker ? warp : KP; kk < KP; kk += OZ_WARPS) {   // mu_k: warp per row
        int mx = OZ_NONE;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int E = f64_bexp(Ms[kk * DD_MAXC + lane + 32 * h]);
          if (E) mx = max(mx, E - 1022);
        }
        mx = __reduce_max_sync(0xffffffffu, mx);
        if (lane == 0) mexp[kk] = mx;
      }
      __syncthreads();
      if (worker) {                                     // f_n: 8 threads per column
        const int n = tid & (DD_MAXC - 1), q = tid >> 6;
        int mx = OZ_NONE;
        for (int kk = q; kk < t.ni; kk += 8) {
          const int E = f64_bexp(Ms[kk * DD_MAXC + n]);
          if (E) mx = max(mx, E - 1022 - mexp[kk]);
        }
        red[q][n] = mx;
      }
      __syncthreads();
      if (tid < DD_MAXC) {
        int mx = red[0][tid];
#pragma unroll
        for (int q = 1; q < 8; ++q) mx = max(mx, red[q][tid]);
        fexp[tid] = mx;
      }
      __syncthreads();
      // digits of M'[kk][n] relative to 2^f_n, two adjacent kk per thread; plane u holds
      // rows u N + n
      const uint32_t MPLt = (uint32_t)t.N * 2 * KP;
      for (int e = worker ? tid : t.N * (KP / 2); e < t.N * (KP / 2); e += OZ_WORKERS) {
        const int n = e / (KP / 2), kk = 2 * (e - n * (KP / 2));
        const double m0 = Ms[kk * DD_MAXC + n], m1 = Ms[(kk + 1) * DD_MAXC + n];
        float d0[OZ_DIG], d1[OZ_DIG];
        oz_digits(m0, fexp[n] + mexp[kk], d0);
        oz_digits(m1, fexp[n] + mexp[kk + 1], d1);
        const uint32_t off = tc::op_off(n, kk * 2, 2 * KP);
#pragma unroll
        for (int u = 0; u < OZ_DIG; ++u)
          *reinterpret_cast<uint32_t*>(msl + u * MPLt + off) = oz_pack(d0[u], d1[u]);
      }
      __syncthreads();
    }
    // ---- the tile's rows (loaded during the previous tile): row bounds, digit planes
    int mx = OZ_NONE;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int kk = 8 * c + 2 * q;
      if (worker && c < KP / 8 && kk < t.ni) {
        const int E0 = f64_bexp(x[c].x), E1 = f64_bexp(x[c].y);
        if (E0 && mexp[kk] != OZ_NONE) mx = max(mx, E0 - 1022 + mexp[kk]);
        if (E1 && kk + 1 < t.ni && mexp[kk + 1] != OZ_NONE) mx = max(mx, E1 - 1022 + mexp[kk + 1]);
      }
    }
    mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, 8));
    mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, 16));
    if (worker && q == 0) rexp[tb][r] = mx;
    const int fn = next_valid(f + 1);
    const OzTile tn = fn < f1 ? shape(fn) : t;
    for (int p = 0; p < npass; ++p) {
      const int k0 = p * KA, buf = ns & 1;
      if (ns >= 2) wait_stage(ns - 2);                  // the buffer's previous stage is read
      uint8_t* asl = asl0 + (size_t)buf * ABUF;
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const int kk = 8 * c + 2 * q;
        if (worker && c < KP / 8 && kk >= k0 && kk < k0 + KA) {
          // entries past ni, or whose row of M is zero, are zero (their digits too)
          const double x0 = (kk < t.ni && mexp[kk] != OZ_NONE) ? x[c].x : 0.0;
          const double x1 = (kk + 1 < t.ni && mexp[kk + 1] != OZ_NONE) ? x[c].y : 0.0;
          float d0[OZ_DIG], d1[OZ_DIG];
          oz_digits(x0, mx - mexp[kk], d0);
          oz_digits(x1, mx - mexp[min(kk + 1, DD_MAXC - 1)], d1);
          const uint32_t off = tc::op_off(r, (kk - k0) * 2, 2 * KA);
#pragma unroll
          for (int s = 0; s < OZ_DIG; ++s)
            *reinterpret_cast<uint32_t*>(asl + s * APL + off) = oz_pack(d0[s], d1[s]);
        }
      }
      if (worker && p == npass - 1 && fn < f1) oz_load_rows(x, a.A, a.lda, tn, r, q, KP);
      tc::fence_async_smem();
      alive = __syncthreads_and(alive) != 0;
      if (alive && p == 0 && pending) finish_prev();    // overlapped with the previous MMAs
      if (!alive) break;
      if (tid == OZ_WORKERS) issue(t, buf, k0, p > 0);   // the issuing warp
      ++ns;
      __syncwarp();
    }
    if (!alive) break;
    pending = true;
    prev = t;
    prev_tb = tb;
    tb ^= 1;
    if (fn >= f1) break;
    f = fn;
    t = tn;
  }
  if (pending && alive) finish_prev();
  if (!alive) {
    if (tid == 0) atomicOr(a.status, (unsigned)ST_TIMEOUT);
    if (ns > 0) tc::mbar_wait(&bar_mma[(ns - 1) & 1], ((ns - 1) >> 1) & 1, kWait);   // in flight
  }
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

// ---------------------------------------------------------------------------------------
// FP64-accurate symmetric Gram partials on the BF16 tensor cores (Ozaki scheme)
// ---------------------------------------------------------------------------------------
// G_c = A_c^T A_c over a chunk of rows, with the chunks and the output of k_gram: one
// RC x RC partial per (subdomain, chunk), zero outside the ma x ma block; with chunk
// exponents, the Gram of 2^-e A_c (e = the chunk's scale when it is far from 1; INT_MIN for a
// chunk below 2^-1000).  A pre-pass over the chunk's rows bounds every column i by 2^c_i;
// the values become 7 balanced base-256 digits relative to 2^(c_i + 1) (as for the tall
// products, one bit higher, so that every digit, the leading one included, is in
// [-128, 128]), and the chunk's rows are taken in stages of 64 (double-buffered digit
// planes of A'^T, the K dimension of the stage's MMAs).
// The M = 128 A operand of an MMA starting at plane s1 covers h = 128 / P consecutive
// planes (P = the padded column count): lanes u P .. u P + P - 1 ("band" u) hold plane
// s1 + u.  One MMA per s1 in {0, h, 2h, ..} with the B operand's planes t = 0 .. 6 - s1
// stacked along N (accumulator column block s1 + t) therefore serves every band at once:
// in band u, column block c accumulates the digit pairs (s, t) of order s + t = c + u.
// At most 4 pairs of products <= 2^14 meet in one band's block, so 128 rows (two stages)
// stay below 2^24 and exact in FP32: the accumulators are read out every two stages.  The
// read-out combines each band's blocks in 64-bit integers (< 2^62), exchanges the bands
// through the free plane buffer (rows padded to P + 1 entries), sums them in a fixed order and adds the result, made FP64
// with the chunk's column scales, to per-thread FP64 accumulators (thread t owns the
// upper-triangle entries t + 512 m of the P x P block); a chunk's partial is written after
// its last read-out.  Persistent CTAs (one per SM: 16 worker warps, one MMA-issue warp)
// walk the (subdomain, chunk) items.
#define OG_KS 64                          // rows per stage (K of one stage's MMAs)
#define OG_RO 2                           // stages per read-out (128 rows)
#define OG_PAD (128 * 2 * OG_KS)          // the M = 128 A operand reads past the last plane

struct OzGram {
  Geo g;
  int spatial;
  const double* A; int lda;
  const int* acnt;
  double* part; int nchunk;
  int* cexp;
  unsigned* status;
};

// dynamic shared memory of k_oz_gram for a column capacity RC <= DD_MAXC: two plane buffers
// (and the alignment slack); at most 147.6 KB, beside 5.2 KB of static shared memory
static size_t og_smem(int RC) {
  const int PMAX = (RC + 15) / 16 * 16;
  return 128 + 2 * ((size_t)OZ_DIG * PMAX * 2 * OG_KS + OG_PAD);
}

// what a read-out needs to know
struct OgGroup {
  int k, c, ma, P, ex, last, cp;
};

__global__ void __launch_bounds__(OZ_THREADS, 1) k_oz_gram(OzGram a) {
  extern __shared__ uint8_t raw_og[];
  uint8_t* buf0 = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(raw_og) + 127) &
                                             ~uintptr_t(127));
  const int RC = a.g.RC, PMAX = (RC + 15) / 16 * 16;
  const uint32_t BUF = OZ_DIG * PMAX * 2 * OG_KS + OG_PAD;
  __shared__ uint64_t bar_mma[2];
  __shared__ uint32_t tmem_s;
  __shared__ int cs[2][DD_MAXC];                 // column bound exponents (item parity)
  __shared__ long long cred[8][DD_MAXC];
  __shared__ long long cmb[DD_MAXC];             // column maxima (bits) of the item
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool worker = warp < OZ_WARPS;
  const int nitems = a.g.nsub * a.nchunk;
  if ((int)blockIdx.x >= nitems) return;
  if (tid == 0) {
    tc::mbar_init(&bar_mma[0], 1);
    tc::mbar_init(&bar_mma[1], 1);
    tc::mbar_init_fence();
  }
  if (warp == 0) tc::tmem_alloc(&tmem_s, 512);   // OZ_DIG column blocks of up to 64 columns
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_s;
  bool alive = true;
  int ns = 0;                                    // stages issued
  int gs = 0;                                    // stages in the open read-out group
  int cp = 0;                                    // item parity (cs)
  bool pending = false;                          // a closed group not yet read out
  OgGroup prev{};
  double acc[8];
#pragma unroll
  for (int m = 0; m < 8; ++m) acc[m] = 0.0;
  auto wait_stage = [&](int j) {
    alive = tc::mbar_wait(&bar_mma[j & 1], (j >> 1) & 1, kWait) && alive;
  };
  // read out the closed group prev (its MMAs complete) into acc; write the chunk's partial
  // after its last group.  Scratch: the planes buffer of the group's last stage.
  auto readout = [&]() {
    wait_stage(ns - 1);
    tc::fence_after_sync();
    const int P = prev.P, h = 128 / P, nb = h < OZ_DIG ? h : OZ_DIG;
    long long* X = reinterpret_cast<long long*>(buf0 + (size_t)((ns - 1) & 1) * BUF);
    if (worker) {
      // worker warp w: TMEM lanes 32 (w % 4) .. (band u = lane / P, row i), 4-column groups
      // 4 (w / 4) + 16 t
      const int q4 = warp & 3, L = q4 * 32 + lane, u = L / P, i = L - u * P;
      const bool lv = u < nb && i < prev.ma;
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int c0 = 4 * (warp >> 2) + 16 * t;
        if (c0 >= P) continue;                   // warp-uniform
        uint32_t D[OZ_DIG][4];
#pragma unroll
        for (int c = 0; c < OZ_DIG; ++c)
          oz_tmem_ld4(tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(c * P + c0), D[c]);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int c = 0; c < OZ_DIG; ++c)
#pragma unroll
          for (int jj = 0; jj < 4; ++jj) asm volatile("" : "+r"(D[c][jj]));
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
          const int j = c0 + jj;
          if (lv && j < prev.ma && j >= i) {
            long long J = 0;
#pragma unroll
            for (int c = 0; c < OZ_DIG; ++c) {
              const int g = c + u;                 // the digit order this block holds
              const int d = __float2int_rn(__uint_as_float(D[c][jj]));
              if (g < OZ_DIG - 1) J += (long long)d << (40 - 8 * g);
              else if (g == OZ_DIG - 1) J += (long long)(d >> 8);
            }
            X[(u * P + i) * (P + 1) + j] = J;
          }
        }
      }
    }
    __syncthreads();
    if (worker && alive) {
      const int* csr = cs[prev.cp];
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        const int e = tid + OZ_WORKERS * m, i = e / P, j = e - i * P;
        if (e < P * P && i < prev.ma && j < prev.ma && j >= i) {
          long long J = 0;
          for (int u = 0; u < nb; ++u) J += X[(u * P + i) * (P + 1) + j];
          acc[m] += oz_to_f64(J, csr[i] + csr[j] + 2 - 56 - 2 * prev.ex);
        }
      }
    }
    if (prev.last && worker) {
      double* out = a.part + ((long)prev.k * a.nchunk + prev.c) * RC * RC;
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        const int e = tid + OZ_WORKERS * m, i = e / P, j = e - i * P;
        if (e < P * P && i < prev.ma && j < prev.ma && j >= i) {
          out[i * RC + j] = acc[m];
          out[j * RC + i] = acc[m];
        }
        acc[m] = 0.0;
      }
      for (int e = tid; e < RC * RC; e += OZ_WORKERS) {
        const int r = e / RC, cc = e - r * RC;
        if (r >= prev.ma || cc >= prev.ma) out[e] = 0.0;
      }
    }
    tc::fence_before_sync();
    alive = __syncthreads_and(alive) != 0;
    pending = false;
  };
  // MMAs of one stage from plane buffer b (planes of P rows): for s1 = 0, h, 2h, .. the
  // A operand is planes s1 .. s1 + h - 1 (one per band; past the last plane it reads junk
  // into blocks never read out), the B operand planes u0 .. u0 + nu - 1 (u0 + nu <= 7 - s1)
  // stacked along N into column blocks s1 + u0 ..
  auto issue = [&](int b, int P, bool first) {
    tc::fence_after_sync();
    const int nper = 256 / P, h = 128 / P;
    const uint32_t PL = (uint32_t)P * 2 * OG_KS;
    const uint64_t d0 = tc::sdesc(tc::smem_u32(buf0 + (size_t)b * BUF), 128, 16 * OG_KS);
    for (int j = 0; j < OG_KS / 16; ++j)
      for (int s1 = 0; s1 < OZ_DIG; s1 += h)
        for (int u0 = 0; u0 < OZ_DIG - s1; u0 += nper) {
          const int nu = min(nper, OZ_DIG - s1 - u0);
          tc::mma_bf16(tmem + (uint32_t)((s1 + u0) * P), d0 + ((s1 * PL + 256 * j) >> 4),
                       d0 + ((u0 * PL + 256 * j) >> 4), tc::idesc(tc::FMT_BF16, 128, nu * P),
                       (!first || j > 0 || s1 > 0) ? 1u : 0u);
        }
    tc::mma_commit(&bar_mma[b]);
  };

  for (int w = blockIdx.x; w < nitems && alive; w += gridDim.x) {
    const int k = w / a.nchunk, c = w - k * a.nchunk;
    const int rows = a.spatial ? a.g.N[k] : a.g.n;
    const long rb = a.spatial ? (long)a.g.rowoff[k] : (long)k * a.g.n;
    const int ch = (rows + a.nchunk - 1) / a.nchunk;
    const int i0 = min(rows, c * ch), i1 = min(rows, i0 + ch);
    const int ma = a.acnt[k], P = ma <= 16 ? 16 : (ma + 15) / 16 * 16;
    // ---- pre-pass: column bounds (largest |entry| of each column on the integer order of
    // its bits; non-finite entries other than infinities are left out) and the chunk scale,
    // into the parity cn of cs (a pending read-out of the previous item uses parity cp)
    const int ci = tid & 63, rg = tid >> 6, cn = cp ^ 1;
    {
      long long mb = 0;
      if (worker && ci < ma)
        for (int row = i0 + rg; row < i1; row += 8) {
          const long long bits =
              __double_as_longlong(a.A[(rb + row) * a.lda + ci]) & 0x7fffffffffffffffll;
          if (bits <= 0x7ff0000000000000ll) mb = max(mb, bits);
        }
      if (worker) cred[rg][ci] = mb;
    }
    __syncthreads();
    if (tid < DD_MAXC) {
      long long m2 = cred[0][tid];
#pragma unroll
      for (int r = 1; r < 8; ++r) m2 = max(m2, cred[r][tid]);
      const int E = (int)((unsigned long long)m2 >> 52);
      cs[cn][tid] = E ? E - 1022 : OZ_NONE;
      cmb[tid] = tid < ma ? m2 : 0;
    }
    __syncthreads();                              // cred is read before the next item's writes
    int ex = 0;
    bool zero = ma == 0 || i1 <= i0;
    if (a.cexp) {
      long long cmx = 0;                          // the chunk's largest |entry|
      for (int q = 0; q < DD_MAXC; ++q) cmx = max(cmx, cmb[q]);
      const double mx = __longlong_as_double(cmx);
      const int e0 = (mx > 0.0 && isfinite(mx)) ? ilogb(mx) : 0;
      zero = zero || !(mx > 0.0) || e0 < -1000;
      ex = (!zero && (e0 < -400 || e0 > 400)) ? e0 : 0;
      if (tid == 0) a.cexp[(long)k * a.nchunk + c] = zero ? INT_MIN : ex;
    }
    if (zero) {                                   // an all-zero partial, no stages
      double* out = a.part + ((long)k * a.nchunk + c) * RC * RC;
      for (int e = tid; e < RC * RC; e += OZ_THREADS) out[e] = 0.0;
      continue;
    }
    cp = cn;
    count_work(a.g, KS_OZ_GRAM, 2.0 * (i1 - i0) * (ma * (ma + 1) / 2));
    const int nst = (i1 - i0 + OG_KS - 1) / OG_KS;
    const int e1 = cs[cp][ci] + 1;                // this thread's column: digits relative to 2^e1
    for (int sgi = 0; sgi < nst; ++sgi) {
      const int r0 = i0 + sgi * OG_KS, b = ns & 1;
      // ---- loads: thread (column ci, row pairs tid / 64 + 8 t)
      double2 x[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int rp = rg + 8 * t, r = r0 + 2 * rp;
        x[t] = make_double2(0.0, 0.0);
        if (worker && ci < ma) {
          if (r < i1) x[t].x = __ldg(a.A + (rb + r) * a.lda + ci);
          if (r + 1 < i1) x[t].y = __ldg(a.A + (rb + r + 1) * a.lda + ci);
        }
      }
      if (ns >= 2) wait_stage(ns - 2);           // buffer b's previous stage is done
      // ---- digit planes: element (i, r) of A'^T at op_off(i, 2 (r - r0), 2 OG_KS)
      if (worker && ci < ma) {
        uint8_t* pl = buf0 + (size_t)b * BUF;
        const uint32_t PL = (uint32_t)P * 2 * OG_KS;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int rp = rg + 8 * t;
          float d0[OZ_DIG], d1[OZ_DIG];
          oz_digits(x[t].x, e1, d0);
          oz_digits(x[t].y, e1, d1);
          const uint32_t off = tc::op_off(ci, rp * 4, 2 * OG_KS);
#pragma unroll
          for (int s = 0; s < OZ_DIG; ++s)
            *reinterpret_cast<uint32_t*>(pl + s * PL + off) = oz_pack(d0[s], d1[s]);
        }
      }
      tc::fence_async_smem();
      alive = __syncthreads_and(alive) != 0;
      if (alive && pending) readout();            // the closed group's MMAs, under this conversion
      if (!alive) break;
      if (tid == OZ_WORKERS) issue(b, P, gs == 0);
      ++ns;
      ++gs;
      if (gs == OG_RO || sgi == nst - 1) {       // close the group
        pending = true;
        prev.k = k; prev.c = c; prev.ma = ma; prev.P = P; prev.ex = ex; prev.cp = cp;
        prev.last = sgi == nst - 1;
        gs = 0;
      }
      __syncwarp();
    }
  }
  if (pending && alive) readout();
  if (!alive) {
    if (tid == 0) atomicOr(a.status, (unsigned)ST_TIMEOUT);
    if (ns > 0) tc::mbar_wait(&bar_mma[(ns - 1) & 1], ((ns - 1) >> 1) & 1, kWait);
  }
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

// ---------------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------------
// Failure-detection self-test of the bounded wait that every tensor-core kernel uses for its
// tile loads and MMAs: one thread initialises an mbarrier expecting one arrival that nothing
// makes and waits on its phase 0 for at most `polls` polls.  When the wait runs out it records
// ST_TIMEOUT in *status, as the production kernels do, then makes the arrival itself so that
// the barrier's phase is complete when the CTA exits.
__global__ void k_wait_selftest(unsigned* status, uint32_t polls) {
  __shared__ uint64_t bar;
  if (threadIdx.x != 0) return;
  tc::mbar_init(&bar, 1);
  tc::mbar_init_fence();
  if (!tc::mbar_wait(&bar, 0, polls)) {
    atomicOr(status, (unsigned)ST_TIMEOUT);
    tc::mbar_arrive(&bar);
  }
}

cudaError_t wait_selftest(unsigned* status, unsigned polls, cudaStream_t st) {
  k_wait_selftest<<<1, 32, 0, st>>>(status, polls);
  return cudaGetLastError();
}

cudaError_t tc_init() {
  if (!g_encode.load(std::memory_order_acquire)) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                     cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    g_encode.store(reinterpret_cast<EncodeTiledFn>(fn), std::memory_order_release);
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
                           (int)OZ_SMEM_LIMIT);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_oz_gram, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)og_smem(DD_MAXC));
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
  a.A = A; a.mtrans = 0; a.rowscale = nullptr;
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
             const double* smbase, const int* ncols, int ncols_fix, double* Y, int ldy,
             int mtrans, int accumulate, const double* rowscale) {
  if (lda > DD_MAXC || (lda & 1)) return false;
  const OzPlan pl = oz_plan(lda, OZ_SMEM_LIMIT);
  if (pl.total > OZ_SMEM_LIMIT) return false;
  TcTall a;
  a.g = P.g; a.spatial = spatial; a.lda = lda; a.ninner = ninner; a.ninner_fix = ninner_fix;
  a.Bm = Bm; a.bsmall = bsmall; a.smbase = smbase; a.ncols = ncols; a.ncols_fix = ncols_fix;
  a.Y = Y; a.ldy = ldy; a.alpha = 1.0; a.accumulate = accumulate; a.status = status;
  a.A = A;
  a.mtrans = mtrans;
  a.rowscale = rowscale;
  a.tps = ((spatial ? P.maxN : P.g.n) + TT_ROWS - 1) / TT_ROWS;
  const long ntot = (long)P.g.nsub * a.tps;
  const int grid = (int)std::min<long>(ntot, P.nsm);
  pbeg(st, KS_OZ_TALL);
  k_oz_tall<<<grid, OZ_THREADS, pl.total, st>>>(a, pl.KP, pl.KA, pl.npass, pl.nbuf);
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

bool oz_gram(const Problem& P, unsigned* status, cudaStream_t st, int spatial, const double* A,
             int lda, const int* acnt, double* part, int nchunk, int* cexp) {
  if (P.g.RC > DD_MAXC) return false;
  const size_t smem = og_smem(P.g.RC);
  OzGram a;
  a.g = P.g; a.spatial = spatial; a.A = A; a.lda = lda; a.acnt = acnt; a.part = part;
  a.nchunk = nchunk; a.cexp = cexp; a.status = status;
  const int grid = (int)std::min<long>((long)P.g.nsub * nchunk, P.nsm);
  pbeg(st, KS_OZ_GRAM);
  k_oz_gram<<<grid, OZ_THREADS, smem, st>>>(a);
  pend(st);
  return true;
}

}  // namespace dd
