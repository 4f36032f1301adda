// Host-side launch interface between the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include "dd_internal.cuh"

namespace dd {

// Kernel classes timed by dd_dlra_profile (one slot per kernel function).
enum KernelSlot {
  KS_AUG_COLS = 0, KS_BUILD_L0, KS_GEIG_AUG, KS_ANG_COEFFS, KS_REDUCE, KS_SMALL_ADV1, KS_TALL,
  KS_GHOST, KS_KSTEP_ADV, KS_SP_COEFFS, KS_SSTEP_ADV, KS_LSTEP_ADV, KS_GRAM, KS_TRUNC,
  KS_COLL_RANK, KS_COLL_A, KS_COLL_KSTEP, KS_COLL_SMALL, KS_COLL_LSTEP, KS_COLL_FINAL,
  KS_FLUX, KS_COPY, KS_GEIG, KS_CHOL, KS_COMPLETE, KS_MASS, KS_KC_W, KS_KC_SEL, KS_KC_APPLY,
  KS_TC_TALL, KS_TC_GRAM, KS_LSTEP_PROD, KS_OZ_TALL, KS_OZ_GRAM, NSLOT
};
extern const char* const kSlotNames[NSLOT];

// Event-pair recorder around kernel launches (active only inside dd_dlra_profile).
struct Prof {
  static const int MAXL = 512;
  int n;
  cudaEvent_t b[MAXL], e[MAXL];
  int slot[MAXL];
};
extern thread_local Prof* g_prof;
inline void pbeg(cudaStream_t st, int slot) {
  if (g_prof && g_prof->n < Prof::MAXL) {
    cudaEventRecord(g_prof->b[g_prof->n], st);
    g_prof->slot[g_prof->n] = slot;
  }
}
inline void pend(cudaStream_t st) {
  if (g_prof && g_prof->n < Prof::MAXL) {
    cudaEventRecord(g_prof->e[g_prof->n], st);
    ++g_prof->n;
  }
}

struct OrthArgs {
  Geo g;
  int spatial;            // rows are cells (1) or directions (0)
  int mode;               // OrthMode
  const double* A; int lda;
  const int* acols;       // input columns per subdomain
  double* Q; int ldq;     // output basis
  const int* rout;        // output columns per subdomain (QR, COMPLETE)
  const int* r_own;       // AUG: current stored rank
  int* rt_out;            // AUG: chosen intermediate rank
  int rank_mode; double tol; int r_floor; int r_aug_max;
  double tau; double accept;
  const double* angcand; int n_angcand; int angcand_complete;
  int n_angorth;          // leading table candidates that are mutually orthogonal
  double* sig_out; int* p_out;
  unsigned* status;
};

cudaError_t orth_init();
// the per-subdomain steps of the orthonormalisation (dd_orth.cu)
void launch_geig(const OrthArgs& a, const double* part, const int* cexp, int nchunk, double* sm,
                 int sM, int* keep, cudaStream_t st);
void launch_chol_inv(const OrthArgs& a, const double* part, int nchunk, double* sm, int sRi,
                     const int* keep, cudaStream_t st);
void launch_complete(const OrthArgs& a, const int* keep, cudaStream_t st);
// Spatial completion of a QR basis by Gram-Schmidt in coefficient space (dd_orth.cu):
// tab/off/nf are the cosine tables of the candidate family, part the scratch region
// (kc_region doubles per subdomain), kcn the accepted count, kcur the columns done.
void launch_kc(const OrthArgs& a, const double* tab, const long long* off, const int* nf,
               const int* keep, double* part, int* kcn, int* kcur, int maxN, cudaStream_t st);

// Phase kernels (dd_phase.cu).  All buffers follow the layout described in
// dd_internal.cuh; "small" matrices are RC x RC blocks, per subdomain stride RC*RC.
struct PhaseBufs {
  // state (read) and state (write)
  const double* X; const double* V; const double* S; const int* r;
  double* Xo; double* Vo; double* So; int* ro;
  // workspace
  double* L0;      // angular rows, ld MC
  double* Hw;      // orthonormalisation workspace, spatial rows, ld WC
  double* Hwa;     // orthonormalisation workspace, angular rows, ld WC
  double* Vh;      // angular rows, ld RC (augmented basis)
  double* K;       // spatial rows, ld RC
  double* X1;      // spatial rows, ld RC
  double* L;       // angular rows, ld RC
  double* V1;      // angular rows, ld RC
  double* Kb;      // ghosts: nsub x 2 sides x maxlines x RC
  double* sm;      // small matrices: nsub x NSMALL x RC*RC
  double* part;    // partial sums for chunked reductions
  int* m;          // L0 columns per subdomain
  int* rt;         // intermediate rank
  int* rx;         // last r_t of x / y phases (2*nsub)
  int* rc;         // collision rank
  double* sig;     // diagnostics
  int* p;          // diagnostics
  int* keep;       // per subdomain: significant columns kept by the orthonormalisation
  int* kcn;        // per subdomain: candidates accepted by the coefficient-space completion
  int* kcur;       // per subdomain: columns done before the sequential completion
  int* cexp;       // per subdomain and row chunk: power-of-two exponent of a scaled Gram
  double* dm;      // per cell: scalar-flux change of the non-conservative parts (mass fix)
  double* mvec;    // per subdomain: RC-vector scratch of the mass bookkeeping
  unsigned* status;
};

// indices of small matrices inside a subdomain's block of NSMALL matrices
enum Small {
  SM_C = 0, SM_MOUT_LO, SM_MOUT_HI, SM_M, SM_MIN_LO, SM_MIN_HI,   // angular Galerkin coefficients
  SM_B, SM_B_LO, SM_B_HI,                                          // S M, S_lo Min_lo, S_hi Min_hi
  SM_CP, SM_CM, SM_CABS,                                           // C+, C-, |C|
  SM_S1, SM_T, SM_G_LO, SM_G_HI,                                   // S-step coefficients
  SM_S2, SM_AP, SM_AM,                                             // S-step result, L-step matrices
  SM_S3T, SM_UB, SM_VB,                                            // S3^T, truncation rotations
  SM_MS, SM_MT, SM_VEC,                                            // collision: Ms, Mt, vectors (a, q, b-stages)
  SM_R1I, SM_QM,                                                   // orthonormalisation
  NSMALL
};

struct Problem {
  Geo g;
  int maxlines;           // longest line (max subdomain width or height)
  int maxN;               // most cells in a subdomain
  const double* ox; const double* oy; const double* w; const double* sw;
  const double* sig_s; const double* sig_t; const double* sQ;  // per cell (spatial row order); sQ = sqrt(hx hy) Q
  double hx, hy, sh, dt, c_adv, ssum;
  int integrator;         // 0 Euler, 1 RK4
  int prec;               // Prec: FP64 throughout; FP32 increments (MIXED); in addition the
                          // Galerkin contractions on tensor cores (TF32, BF16)
  int mass_fix;           // conserved-moment correction at the end of every step
  int splitting;          // 0 Lie (x, y, collision), 1 Strang (x/2, y/2, collision, y/2, x/2)
  int kstep_split;        // C+/C- of the advection K-step: 0 eigen-split, 1 direction split
  int oz_sp, oz_ang;      // FP64 tall products on the tensor cores (Ozaki splitting), for
                          // the spatial / the angular row family
  int ozg_sp, ozg_ang;    // the orthonormalisations' Grams likewise
  // physical inflow (null without): per subdomain and side (x-lo, x-hi, y-lo, y-hi) an
  // on flag, face values sqrt(hx hy) g per line (maxlines), the angular column
  // sqrt(w) m_in h (n) and its augmentation scale |g|_x
  const int* infl_on; const double* infl_g; const double* infl_hw; const double* infl_sc;
  int rank_mode; double tol; double tau; double accept;
  int r_floor, r_aug_max, RS;
  int WC;                 // leading dimension of the orthonormalisation workspaces
  const double* angcand; int n_angcand; int angcand_complete;
  int n_angorth;          // leading table candidates mutually orthogonal to 1e-12
  // spatial candidate family: per subdomain the cosines cos(pi f (i + 1/2) / n_x) for
  // f < nf[2k] and cos(pi f (j + 1/2) / n_y) for f < nf[2k + 1], from offset spoff[k]
  const double* sptab; const long long* spoff; const int* spnf;
  int nchunk_sp, nchunk_ang;   // chunks of the two-stage reductions
  int ochunk_sp, ochunk_ang;   // chunks of the orthonormalisations' Grams (<= nchunk_*)
  int nsm;                     // streaming multiprocessors of the device
  long Ntot;                   // spatial rows of all subdomains
};

// ---- tensor-core contractions (dd_tc.cu), DD_TF32 / DD_BF16 --------------------------
// Row weights of a Gram source: none, the advection axis' velocity Omega, its sign masks
// (Omega < 0 / Omega >= 0, -0 counting as >= 0), Omega+ = max(Omega, 0), Omega- =
// min(Omega, 0), or a per-row array (spatial rows).
enum GramWeight { W_NONE = 0, W_OMEGA, W_NEG, W_NONNEG, W_OMEGA_POS, W_OMEGA_NEG, W_ROW };
struct TcGramSrc {
  const double* ptr; int ld;   // the tall array (ignored when same_as_b)
  const int* cnt; int fix;     // columns per subdomain (cnt[k'] or fix)
  int nbside;                  // -1: the subdomain's own rows; 0 / 1: the low / high
                               // neighbour's along the axis (absent neighbour: no product)
  int same_as_b;               // the rows of the common operand B (no separate load)
  int shift;                   // the difference B - shift(B): each row of the common operand
                               // minus the row one cell earlier along the axis (0 before a
                               // line start); ptr must be B
  int wsel; const double* wrow;
  int blk;                     // partial block written
  int transpose;               // write D^T
};
#define TC_MAXSRC 8
struct TcGram {
  Geo g;
  int spatial, axis;
  const double* B; int ldb; const int* bcnt; int bfix;   // the common operand
  int nsrc; TcGramSrc src[TC_MAXSRC];  // sources 2j and 2j + 1 share a CTA; the sources
                                       // of one slot (even / odd) not same_as_b share ptr, ld
  double* part; int nchunk, nblk;
  const double* ox; const double* oy;
  unsigned* status;
};
cudaError_t tc_init();
// the bounded-wait self-test (failure detection): ST_TIMEOUT into *status when it runs out
cudaError_t wait_selftest(unsigned* status, unsigned polls, cudaStream_t st);
// Y = alpha A M (accumulate: Y += alpha A M); false when the operands do not suit TMA
// (odd leading dimension), then nothing is launched
bool tc_tall(const Problem& P, unsigned* status, cudaStream_t st, int spatial, const double* A,
             int lda, const int* ninner, int ninner_fix, const double* Bm, int bsmall,
             const double* smbase, const int* ncols, int ncols_fix, double* Y, int ldy,
             double alpha, int accumulate);
bool tc_gram(const Problem& P, cudaStream_t st, const TcGram& a);
// Y = A M to FP64 accuracy on the BF16 tensor cores (Ozaki splitting); false when the
// operands do not suit TMA, then nothing is launched
// (mtrans: M is read transposed, Y = A M^T, M still the RC x RC block of its slot;
// accumulate: Y += A M on the columns < ncols, the others untouched, each row r scaled by
// rowscale[r] (global row index) when rowscale is not null)
bool oz_tall(const Problem& P, unsigned* status, cudaStream_t st, int spatial, const double* A,
             int lda, const int* ninner, int ninner_fix, const double* Bm, int bsmall,
             const double* smbase, const int* ncols, int ncols_fix, double* Y, int ldy,
             int mtrans = 0, int accumulate = 0, const double* rowscale = nullptr);
// The chunk partials of the symmetric Gram A^T A (the layout and chunk exponents of k_gram)
// FP64-accurate on the BF16 tensor cores; false when the capacity does not fit.
bool oz_gram(const Problem& P, unsigned* status, cudaStream_t st, int spatial, const double* A,
             int lda, const int* acnt, double* part, int nchunk, int* cexp);
void advection_phase(const Problem& P, const PhaseBufs& B, int axis, cudaStream_t st);
void collision_phase(const Problem& P, const PhaseBufs& B, cudaStream_t st);
void mass_fix_phase(const Problem& P, const PhaseBufs& B, cudaStream_t st);
void scalar_flux(const Problem& P, const double* X, const double* V, const double* S, const int* r,
                 double* work, double* rho, int nx, cudaStream_t st);
cudaError_t phase_init();   // kernel attributes for every capacity up to DD_MAXC
size_t part_elems(const Problem& P);
// Launch choices timed on the solver's own workspace (called once, when a solver is
// created): the engine of the FP64 tall x small products per row family (when
// tune_products) and the chunk counts of the chunked Gram reductions (when tune_chunks).
// The winners are written to P; each family's times are reported in ms[8] (FP64 products,
// tensor-core products, then the chunk candidates' best and worst), -1 where not timed.
// Choices are cached per shape (subdomains, cells, directions, column capacity,
// precision): a later solver of the same shape reuses them without timing.
cudaError_t autotune(Problem& P, const PhaseBufs& B, cudaStream_t st, int tune_products,
                     int tune_chunks, double* ms);

}  // namespace dd
