/*
 * ddlra.h — C ABI of the GB300 (sm_103a) domain-decomposition dynamical low-rank
 * (DD-DLRA) time step for the 2D-space x angle radiative transfer equation
 * (Brunner, Einkemmer, Haut, arXiv 2602.14854).
 *
 * Model (Section 2, Eq. (rt)):
 *     d_t f + c_adv Omega . grad f = sigma_s/|S| * rho - sigma_t f + Q,
 *     sigma_t = sigma_s + sigma_a,   rho = sum_q w_q f_q,   |S| = sum_q w_q,
 * discretised by cell-centred first-order upwind finite volumes on a uniform
 * grid and a discrete direction table (Omega_x, Omega_y, w).
 *
 * On every subdomain k of a block tiling the solution is kept in low-rank form
 * f = U_k S_k V_k^T (Section 3.4) with U orthonormal in the spatial product
 * <u,v> = hx*hy*sum u v and V orthonormal in <a,b> = sum_q w_q a b.  One time
 * step is Algorithm 6: x-augmentation (Algorithm 4), x-advection by the
 * projector-splitting integrator (Algorithm 1) with inflow boundary data
 * (Eq. (generate_Kboundary)) and eigen-upwinding (Appendix A), truncation
 * (Algorithm 5), the same in y (Algorithm 2), then absorption/scattering/source
 * (Algorithm 3).
 *
 * Conventions
 *  - Every call returns a dd_status; DD_OK is 0.  On failure the call has no
 *    effect on the solver state unless stated, and dd_last_error() returns a
 *    thread-local message.  No call throws across the ABI.
 *  - All host arrays passed in are copied; the caller keeps ownership.
 *  - Cells are numbered x-fastest over the global grid: c = j*nx + i.
 *    Within subdomain k cells are numbered x-fastest over the subdomain.
 *  - Subdomain k = J*tx + I for tile column I and tile row J.
 *  - Device memory is allocated by the library at create time (by cudaMalloc, or
 *    by the caller's allocator, see dd_set_allocator) and released by
 *    dd_dlra_destroy.  All device work is issued on the stream given at create.
 *  - Errors detected on the device (non-finite values, an exhausted basis
 *    completion family) are recorded in a device status word and reported by
 *    the next call that synchronises (dd_dlra_scalar_flux, dd_dlra_ranks,
 *    dd_dlra_get_factors, dd_dlra_sync).
 */
#ifndef DDLRA_H
#define DDLRA_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum dd_status {
  DD_OK = 0,
  DD_ERR_ARG = 1,        /* invalid argument (sizes, tiling, options)          */
  DD_ERR_CUDA = 2,       /* a CUDA runtime call failed                           */
  DD_ERR_RANK_CAP = 3,   /* a rank exceeds the capacity fixed at create time     */
  DD_ERR_NONFINITE = 4,  /* a non-finite value appeared in the factors          */
  DD_ERR_COMPLETION = 5, /* the fixed basis-completion family was exhausted      */
  DD_ERR_STATE = 6,      /* call not valid in the current state                 */
  DD_ERR_TIMEOUT = 7     /* a kernel's bounded wait (tile load, tensor-core      */
                         /* product) ran out; the step's results are not valid  */
} dd_status;

typedef struct dd_grid {
  int nx, ny;                 /* global cell counts                               */
  double x0, x1, y0, y1;      /* domain [x0,x1] x [y0,y1], uniform cells           */
} dd_grid;

typedef struct dd_tiling {
  int tx, ty;                 /* subdomain counts in x and y                      */
  const int* xcuts;           /* host, tx+1 cell indices 0 = c_0 < ... < c_tx = nx */
  const int* ycuts;           /* host, ty+1 cell indices 0 = c_0 < ... < c_ty = ny */
} dd_tiling;

typedef struct dd_quadrature {
  int n;                      /* number of discrete directions                    */
  const double* omega_x;      /* host, n: x velocity components                   */
  const double* omega_y;      /* host, n: y velocity components                   */
  const double* w;            /* host, n: positive quadrature weights, |S| = sum  */
  int n_polar;                /* polar (mu) levels of a product set; 0 = circle    */
  int n_azimuth;              /* azimuths per level (phi count)                   */
} dd_quadrature;

typedef struct dd_fields {
  const double* sigma_s;      /* host, nx*ny: scattering coefficient  (>= 0)      */
  const double* sigma_a;      /* host, nx*ny: absorption coefficient  (>= 0)      */
  const double* source;       /* host, nx*ny: isotropic source Q                  */
  /* Physical inflow f(s, Omega) = g(s) h(Omega), constant in time, for the directions
   * entering through a side (Omega_x >= 0 at x = x0, Omega_x < 0 at x = x1, likewise in
   * y): the Hohlraum and boundary point-source inflow of Section 4.  Sides in the order
   * x0, x1, y0, y1; a null g or h means zero inflow on that side.  In the scheme an
   * inflow side acts as a neighbour: its data enter the ghost rows of the K-step and the
   * augmentation of Algorithm 4 (one column m_in h |g|, |g|^2 = hx hy len sum g^2 over
   * the subdomain's face, len its cell count along the axis). */
  const double* inflow_g[4];  /* host: ny values (x sides) or nx values (y sides)  */
  const double* inflow_h[4];  /* host: n values                                    */
} dd_fields;

enum { DD_RANK_FIXED = 0, DD_RANK_TOL = 1 };
enum { DD_EULER = 0, DD_RK4 = 1 };
/* Arithmetic of the step (the paper fixes none).  DD_FP64: FP64 throughout, except that
 * the small eigen/singular value problems (m x m, m <= 64) run FP32 Jacobi sweeps finished
 * in double-float arithmetic (~1e-13 relative; the eigensolver of the orthonormalisation
 * adds one FP64 refinement).  DD_MIXED: in addition, FP32 arithmetic for the increments of
 * the collision-step ODEs and for the L-step's stage corrections (its first-stage
 * right-hand side is formed in FP64); each update itself is added in FP64.  DD_TF32 /
 * DD_BF16: DD_MIXED plus the Galerkin contractions on the tensor cores (tcgen05) in TF32 /
 * BF16 with FP32 accumulation, each FP64 operand split into a high and a low part of that
 * type and multiplied hi*hi + hi*lo + lo*hi (FP32-level error per product): the angular
 * coefficients <V, Omega V> and boundary masses, the spatial coefficients X^T K and
 * X^T shift(X), the collision's X^T diag(sigma) X and X^T K, the projection V^T L, and the
 * products K0 = X (S <V, V_hat>), the truncation's rotations and the collision's X S.
 * The orthonormalisations, the small SVDs and eigendecompositions, the advection K-step
 * (Appendix A's eigenbasis form) and the storage stay FP64.  With physical inflow the
 * angular coefficients stay FP64.  The advection K-step is FP64 in every form except the
 * matrix stencil of the flux-split form outside DD_FP64. */
enum { DD_FP64 = 0, DD_MIXED = 1, DD_TF32 = 2, DD_BF16 = 3 };

typedef struct dd_options {
  int rank_mode;      /* DD_RANK_FIXED: stored rank <= rank; DD_RANK_TOL: tolerance tol   */
  int rank;           /* fixed mode: stored rank r (also the augmentation floor)         */
  double tol;         /* tolerance mode: absolute tail tolerance of Algorithms 4 and 5    */
  int r_min, r_max;   /* tolerance mode: stored-rank clamp after truncation               */
  int r_aug_max;      /* cap on the intermediate rank r_t (<= 64)                         */
  int integrator;     /* DD_EULER or DD_RK4 for every sub-step ODE                        */
  double c_adv;       /* advection speed                                                  */
  double dt;          /* time step                                                        */
  double tau;         /* relative numerical-rank threshold (sigma_j <= tau*sigma_1 -> 0)  */
  int precision;      /* DD_FP64, DD_MIXED, DD_TF32 or DD_BF16                            */
  int mass_fix;       /* 1: conserved-moment correction at the end of every step (not part */
                      /* of the paper's scheme): the scalar-flux change of the S-, L-steps  */
                      /* and truncations of the step is added back as the isotropic        */
                      /* rank-one term delta(x) (x) 1/|S|, then Algorithm 5 truncates; 0: off */
  int splitting;      /* DD_SPLIT_LIE: x, y, collision (Algorithm 6); DD_SPLIT_STRANG:       */
                      /* x(dt/2), y(dt/2), collision(dt), y(dt/2), x(dt/2), the second-order */
                      /* splitting Section 3 refers to; every advection phase is a whole    */
                      /* Algorithm 1/2 with the half step                                    */
  int kstep_split;    /* DD_KSPLIT_EIGEN: the K-step's C+ and C- from the eigendecomposition */
                      /* of C (Appendix A); DD_KSPLIT_FLUX: from the direction split,        */
                      /* C+- = <V, max/min(Omega, 0) V> (the L-step's per-direction upwind   */
                      /* flux projected on the angular basis; equal to Appendix A's at full  */
                      /* rank; not the paper's scheme at low rank; no eigendecomposition)    */
  int products;       /* the FP64 tall x small products (orthonormalisations, truncation,     */
                      /* K0 = X S <V, V_hat>): DD_PRODUCTS_FP64: FP64 CUDA-core arithmetic;    */
                      /* DD_PRODUCTS_TENSOR: these and the orthonormalisations' Grams on the  */
                      /* BF16 tensor cores with the error-free                                 */
                      /* splitting of Ozaki et al. (seven 8-bit digits per value, exact FP32   */
                      /* accumulation, FP64-level error).  Results agree to FP64 rounding, not */
                      /* bits.  DD_PRODUCTS_AUTO: per row family (spatial rows, angular rows)  */
                      /* the faster of the two: timed when the solver is created if autotune  */
                      /* is set, else the tensor cores where the family has at least two      */
                      /* 128-row tiles per SM (the Grams then stay on the CUDA cores).         */
  int autotune;       /* 1: when the solver is created, time the launch choices on its own    */
                      /* workspace and keep the fastest: the products' and the               */
                      /* orthonormalisations' Grams' engines per row family (with            */
                      /* DD_PRODUCTS_AUTO) and the chunk counts of the orthonormalisations'  */
                      /* chunked Gram reductions (the heuristic's, a half and a quarter of it; */
                      /* every count keeps a fixed summation order).  Cached per problem     */
                      /* shape in the process.  0: fixed heuristics.  See dd_dlra_tuning.      */
} dd_options;

enum { DD_SPLIT_LIE = 0, DD_SPLIT_STRANG = 1 };
enum { DD_KSPLIT_EIGEN = 0, DD_KSPLIT_FLUX = 1 };
enum { DD_PRODUCTS_FP64 = 0, DD_PRODUCTS_TENSOR = 1, DD_PRODUCTS_AUTO = 2 };

typedef struct dd_dlra* dd_dlra_t;

/*
 * dd_dlra_create — plan, allocate and initialise a DD-DLRA solver.
 *
 * g0 (host, nx*ny) is the isotropic initial data f(0,x,y,Omega) = g0(x,y); it is
 * stored at rank 1 per subdomain (rank 0 where g0 vanishes on a subdomain).
 * Tilings are block-aligned (Section 3, Figure "block domain decomposition"):
 * every subdomain in a tile row has the same height, in a tile column the same
 * width.  stream is a cudaStream_t (NULL = the legacy default stream).
 * Errors: DD_ERR_ARG for inconsistent sizes or options (r_aug_max > 64,
 * 3*stored-rank cap > 64, fewer directions than 3*stored-rank cap, a subdomain side
 * times r_aug_max above 6144: the K-step keeps a whole line of K in one CTA), DD_ERR_CUDA.
 */
dd_status dd_dlra_create(const dd_grid* grid, const dd_tiling* tiling,
                         const dd_quadrature* quad, const dd_fields* fields,
                         const double* g0, const dd_options* opt, void* stream,
                         dd_dlra_t* out);

/*
 * dd_dlra_create_batch — one solver over ninst independent problems that share the
 * direction table `quad`: grids, tilings, materials, initial data, dt, ranks and the
 * intermediate-rank cap may differ per problem; rank_mode, tol, integrator,
 * precision, c_adv and tau must agree (else DD_ERR_ARG).  Every problem's subdomains
 * advance in the same kernel launches, so a batch is one CUDA graph per step.
 * grids, tilings, fields, g0 and opts hold ninst entries (g0[i] = problem i's
 * isotropic initial data).  Subdomains are numbered problem after problem; the
 * density (dd_dlra_scalar_flux) holds the problems back to back.  (The batched
 * form has no counterpart in the paper: independent problems are independent.)
 */
dd_status dd_dlra_create_batch(int ninst, const dd_grid* grids, const dd_tiling* tilings,
                               const dd_quadrature* quad, const dd_fields* fields,
                               const double* const* g0, const dd_options* opts, void* stream,
                               dd_dlra_t* out);

/* Layout of problem inst of a batch: its first subdomain index, subdomain count, the
 * offset of its density in the dd_dlra_scalar_flux output and its grid size. */
dd_status dd_dlra_instance(dd_dlra_t h, int inst, int* first_subdomain, int* nsub,
                           int* flux_offset, int* nx, int* ny);

/*
 * dd_dlra_step — advance every subdomain by nsteps time steps of Algorithm 6.
 * Asynchronous on the solver's stream.  With use_graph != 0 the step is
 * captured once into a CUDA graph and replayed.
 */
dd_status dd_dlra_step(dd_dlra_t h, int nsteps);
dd_status dd_dlra_set_graph(dd_dlra_t h, int use_graph);

/*
 * dd_dlra_scalar_flux — rho = sum_q w_q f_q on all nx*ny cells, global x-fastest
 * order (Section 2, density); for a batch, the problems' densities back to back.
 * out has nx*ny doubles (a batch: the sum over problems); out_on_device != 0 means
 * a device pointer (written asynchronously on the solver's stream), else a host
 * pointer (the call synchronises).
 */
dd_status dd_dlra_scalar_flux(dd_dlra_t h, double* out, int out_on_device);

/*
 * dd_dlra_scalar_flux_instance — the density of problem inst of a batch alone (for a single
 * problem, inst = 0 gives the same as dd_dlra_scalar_flux): its nx*ny cells (the grid size
 * dd_dlra_instance reports), global x-fastest order of that problem.  The density of every
 * problem is formed in the solver's workspace and problem inst's part copied to out; out is
 * a device pointer when out_on_device != 0 (asynchronous on the solver's stream), else a
 * host pointer (the call synchronises).  Errors: DD_ERR_ARG for a null handle or out, or inst
 * outside 0 .. ninst-1; DD_ERR_CUDA.
 */
dd_status dd_dlra_scalar_flux_instance(dd_dlra_t h, int inst, double* out, int out_on_device);

/* Stored ranks per subdomain after the last step (host, nsub ints), and the
 * intermediate ranks r_t of the last x- and y-augmentation (host, 2*nsub ints,
 * may be NULL).  Synchronises. */
dd_status dd_dlra_ranks(dd_dlra_t h, int* stored, int* intermediate);

/* Number of subdomains, directions and the rank capacity. */
dd_status dd_dlra_info(dd_dlra_t h, int* nsub, int* n, int* r_cap);

/*
 * Factors of subdomain k in the paper's weighted form, host row-major:
 * U (N_k x r), S (r x r), V (n x r), N_k = cells of subdomain k.  get: buffers
 * sized for r_cap columns are enough; *r receives the rank.  set: r <= stored-
 * rank cap; U must be orthonormal in hx*hy*sum and V in sum w (not checked).
 * Both synchronise.
 */
dd_status dd_dlra_get_factors(dd_dlra_t h, int k, double* U, double* S, double* V, int* r);
dd_status dd_dlra_set_factors(dd_dlra_t h, int k, int r, const double* U, const double* S,
                              const double* V);

/*
 * Instrumentation (no counterpart in the paper).  dd_dlra_profile runs nsteps
 * time steps without the CUDA graph, with a CUDA event pair recorded around
 * every kernel launch, and accumulates per kernel function (slot) the total
 * device milliseconds (ms, dd_profile_slots() doubles) and the launch count
 * (launches, dd_profile_slots() ints).  It advances the solver like
 * dd_dlra_step and synchronises.  dd_profile_slot_name returns a static name,
 * or NULL for an out-of-range slot.
 */
int dd_profile_slots(void);
const char* dd_profile_slot_name(int slot);
dd_status dd_dlra_profile(dd_dlra_t h, int nsteps, double* ms, int* launches);
/* dd_dlra_profile, and (flops != NULL, dd_profile_slots() doubles) the algorithmic
 * floating-point operations of every kernel slot over the nsteps steps, counted by the
 * kernels themselves from the sizes they process (the method's operation count for the
 * ranks actually used: 2 per multiply-add of the products, per stage of the fused
 * integrators; the tensor-core slots count the products once, not their three partial
 * products).  The latency-bound slots (small eigen/singular-value problems, completions,
 * reductions) count nothing.  Allocates a small device buffer for the counters. */
dd_status dd_dlra_profile_work(dd_dlra_t h, int nsteps, double* ms, int* launches, double* flops);

/*
 * dd_dlra_tuning — the launch choices the solver runs with (host outputs, either may be
 * NULL): choice[6] = {tensor-core products for spatial rows (0/1), for angular rows (0/1),
 * chunks per subdomain of the orthonormalisations' Grams for spatial rows, for angular rows
 * (the Galerkin products keep the heuristic's count), the orthonormalisations' Grams on the
 * tensor cores for spatial rows (0/1), for angular rows (0/1)}; ms[8] = the autotuner's
 * timings per family (spatial, then angular): FP64 products, tensor-core products, the
 * best and the worst chunk count (ms for one trial Gram and reduction); -1 where nothing
 * was timed (autotune off, or a choice fixed by the options).
 */
dd_status dd_dlra_tuning(dd_dlra_t h, int* choice, double* ms);

/*
 * dd_dlra_scalar_flux_noalloc — the density of dd_dlra_scalar_flux written to the
 * device pointer out (same size and layout), by a call that allocates nothing: no
 * cudaMalloc, no cudaFree, no allocating library routine.  It is for callers that
 * must not allocate device memory at the moment they read the density, for instance
 * under a policy that allows device allocation only at start-up.  (No counterpart in
 * the paper: this is a property of the library, not of the method.)
 *
 * The per-subdomain scratch (nsub * r_cap doubles) lives in one file-scope device
 * array of 16384 doubles (128 KiB) that every GPU loading the library keeps until
 * the process exits; larger solvers get DD_ERR_ARG.  Each solver looks up the array's
 * device address when it is created (with its device and context current), so the
 * address is valid exactly as long as the solver's own memory.  Call it with the
 * solver's device current (else DD_ERR_ARG, checked before anything else).  All calls
 * share the array and each overwrites every element it later reads, so nothing needs
 * clearing; calls that overlap on the GPU (other streams, other solvers) race on it.
 * Asynchronous on the solver's stream, like dd_dlra_scalar_flux with out_on_device != 0.
 * The call can be recorded into a CUDA graph by stream capture when the capturing
 * stream is the solver's own stream (the one given at create): it issues two kernel
 * launches on that stream and nothing else.
 */
dd_status dd_dlra_scalar_flux_noalloc(dd_dlra_t h, double* out);

/* Wait for the solver's stream and report any device-side error. */
dd_status dd_dlra_sync(dd_dlra_t h);

/*
 * dd_selftest_wait — failure-detection self-test (no counterpart in the paper: a property of
 * the library).  Runs, on the current device, one CTA that waits with the same bounded wait
 * the tensor-core kernels use for their tile loads and MMAs on an mbarrier that nothing
 * completes, for at most `polls` polls (1 .. 2^21; the production kernels allow 2^21, about a
 * second).  The wait runs out, the kernel records the timeout bit in a device status word as
 * the production kernels do (they then report DD_ERR_TIMEOUT from the next synchronising
 * call) and returns; the call reads the word back and sets *timed_out = 1.  The CUDA context
 * stays usable.  Synchronous (legacy default stream); allocates and frees one device word.
 * Errors: DD_ERR_ARG for a null pointer or polls out of range, DD_ERR_CUDA for a failed CUDA
 * call.
 */
dd_status dd_selftest_wait(unsigned polls, int* timed_out);

/* Release all device and host memory of the solver.  NULL is ignored. */
void dd_dlra_destroy(dd_dlra_t h);

/* Thread-local message of the last failing call on this thread ("" if none). */
const char* dd_last_error(void);

/* The same message, under the per-solver name: the message is kept per host thread, so h
 * (which may be NULL, e.g. after a failed create) does not select it. */
const char* dd_dlra_last_error(dd_dlra_t h);

/*
 * dd_allocator / dd_set_allocator — device memory from the caller's allocator, e.g. a
 * framework's caching allocator, instead of cudaMalloc / cudaFree.  (No counterpart in the
 * paper: a property of the library.)
 *
 * alloc(bytes, ctx) returns device memory of the current device of at least `bytes` bytes,
 * 256-byte aligned, or NULL; release(ptr, ctx) gives back one pointer alloc returned.  The
 * setter is process-wide and thread-safe; NULL, or both callbacks NULL, restores cudaMalloc /
 * cudaFree.  Each solver copies the allocator in effect when it is created: every device
 * buffer of its state and workspace is drawn through it during dd_dlra_create /
 * dd_dlra_create_batch (on the creating thread) and released through the same copy by
 * dd_dlra_destroy (on the destroying thread, after the solver's stream is synchronised), so
 * changing the allocator later affects only solvers created later.  The memory must stay
 * valid until release; it is used on the solver's stream.  Not drawn through it: the
 * allocation-free readout's fixed array, the counters of dd_dlra_profile_work and the
 * status word of dd_selftest_wait.  Errors: DD_ERR_ARG when exactly one callback is NULL; a NULL or
 * misaligned block makes the create fail with DD_ERR_CUDA.
 */
typedef struct dd_allocator {
  void* (*alloc)(size_t bytes, void* ctx);
  void (*release)(void* ptr, void* ctx);
  void* ctx;
} dd_allocator;

dd_status dd_set_allocator(const dd_allocator* a);

#ifdef __cplusplus
}
#endif
#endif /* DDLRA_H */
