/*
 * ftsp2.h -- C ABI of the GB300 (sm_103a) machine-learned finite-temperature
 * SP2 hot path (arXiv 2605.08523).
 *
 * Given dense symmetric Hamiltonians H (one large matrix or a ragged batch),
 * a chemical potential mu and an electronic temperature kT per instance, the
 * library
 *   (a1) bounds each spectrum with Gershgorin circles (Appendix A),
 *   (a2) maps (H, beta, mu) onto a trained model (beta0, mu0) by the affine
 *        rescaling of Sec. III A (Eqs. H', mu', beta', H0), choosing the flip
 *        of Eq. flip and a model whose region of validity (Eq. conditions)
 *        contains (beta', mu'),
 *   (a3) runs the L-layer learned recursion x <- a x^2 + b x + c, A <- A + d x
 *        (Eq. mlsp2) on the matrix, one symmetric square per layer on the
 *        tensor cores,
 *   (a4) returns D = A + X (or I - (A + X) when flipped) with Tr D and
 *        ||D||_F^2 (Eq. tr(D^2)),
 *   (a5, a6) runs the entropy recursion (Eqs. entropy expansion and
 *        entropy expansion-s) and returns S = 4 ln2 (Tr F - Tr F^2),
 * and (a7) trains the per-layer coefficients by Levenberg-Marquardt on scalar
 * samples (Sec. II C).
 *
 * Conventions shared by every entry point
 *   - Energies are in eV with k_B absorbed: beta = 1/kT.  S is returned per
 *     spin channel in units of k_B.
 *   - Matrices are row-major.  H is FP64 and must be symmetric; every element
 *     is read.  D is FP32.
 *   - Pointers named d... are device pointers; all others are host pointers.
 *     The caller owns every buffer; the library never allocates device memory
 *     in these calls (model sets are the one library-owned allocation).
 *   - Every launch goes to the caller's stream (`stream`, a cudaStream_t
 *     passed as void*; NULL = legacy default stream) and the call returns
 *     without synchronising, unless FTSP2_SYNC is set in `flags`, in which case
 *     it synchronises the stream and returns the worst per-instance status.
 *     Without FTSP2_SYNC only host-side argument errors and launch errors are
 *     returned; device-detected conditions (validity, non-finite input,
 *     timeouts) are left in the per-instance records.
 *   - Calls that share a workspace must not overlap on the GPU.
 */
#ifndef FTSP2_H
#define FTSP2_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FTSP2_OK = 0,
    FTSP2_E_ARG = -1,          /* bad argument detected on the host           */
    FTSP2_E_CUDA = -2,         /* a CUDA runtime/driver call failed           */
    FTSP2_E_WORKSPACE = -3,    /* workspace too small or misaligned           */
    FTSP2_E_VALIDITY = -4,     /* beta' beyond every model's region of validity */
    FTSP2_E_NONFINITE = -5,    /* NaN/Inf in H, mu or kT                       */
    FTSP2_E_TIMEOUT = -6,      /* a bounded device-side wait gave up           */
    FTSP2_E_NOMODEL = -7,      /* empty or inconsistent model set              */
    FTSP2_E_UNSUPPORTED = -8   /* device is not sm_103 / mode not built        */
} ftsp2_status;

/* Arithmetic of the layer products X^2 (Sec. IV A): every mode keeps the state
 * in FP32 and accumulates in FP32; they differ in how X is split into
 * tensor-core operands. */
typedef enum {
    FTSP2_FP32 = 0,    /* CUDA-core FP32 FMA products (no tensor cores)        */
    FTSP2_TF32X3 = 1,  /* X = hi + lo in TF32, 3 products (hi hi, hi lo, lo hi)  */
    FTSP2_BF16X3 = 2,  /* X = b0 + b1 + b2 in BF16, 6 products (terms >= 2^-16)  */
    FTSP2_FP16X2 = 3   /* X = hi + lo in FP16 with a per-layer power-of-two
                          scale, 3 products (the paper's Eq. emulated matmul)  */
} ftsp2_mode;

/* flags */
#define FTSP2_SYNC          0x1  /* synchronise and return the worst status   */
#define FTSP2_CLAMP         0x2  /* outside validity: lower beta' to the largest
                                    valid value of the largest-beta0 model, as
                                    the paper's Appendix A program does (this
                                    changes the temperature); default: status
                                    FTSP2_E_VALIDITY and no result           */
#define FTSP2_REFINE1       0x4  /* last layer in FTSP2_FP32 arithmetic       */
#define FTSP2_REFINE2       0x8  /* last two layers in FTSP2_FP32 arithmetic  */
/* Tile shape of the tensor-core layer launches.  By default a batch runs with
 * the shape ftsp2_autotune recorded for it or, if none was recorded, with the
 * shape a padding model prefers; these two flags override both. */
#define FTSP2_PAIR_TILES    0x10 /* 256 x 256 tiles on CTA pairs (cta_group::2) */
#define FTSP2_SINGLE_TILES  0x20 /* 128 x 128 tiles on single CTAs             */
/* Spectral bounds: by default the Gershgorin interval of Appendix A.  With this
 * flag it is tightened by 24 Lanczos steps in FP64 (start vector from
 * splitmix64 of the row index, no re-orthogonalisation): the extreme Ritz
 * values of the tridiagonal, widened by their residual bounds, by 1 % of their
 * spread and by 1e-6 of their magnitude (the products H v are formed in FP32),
 * intersected with the Gershgorin interval.  A narrower interval
 * lowers beta' = W beta, so a model of smaller beta0 (fewer layers, less
 * amplified rounding) may be chosen.  Cost: 24 matrix-vector products in FP64
 * per instance.  The interval is not a rigorous enclosure (the residual bound
 * and the margin are safety terms, checked on the workload families of the
 * tests); a few eigenvalues slightly outside it map just outside [0, 1], where
 * the shipped tables stay within their fit error for excursions up to 0.02. */
#define FTSP2_LANCZOS       0x40
/* Model choice (workflow step 4) among the models whose region of validity
 * contains (beta', mu'): by default the smallest beta0 (least amplified
 * rounding), ties to fewer layers; with this flag the fewest Fermi-chain layers
 * (the fastest), ties to the smaller beta0. */
#define FTSP2_MIN_LAYERS    0x80
/* With FTSP2_REFINE1/2: the refinement layers run on the tensor cores as
 * BF16X3 layers (6 products of 3-way BF16 splits, FP32 accumulation in
 * 64-element chunks: FP32-class products) instead of FP32 FMA on the CUDA
 * cores, which on this GPU cost ten times a tensor-core layer.  No effect in
 * FTSP2_BF16X3 mode (its layers are BF16X3 already). */
#define FTSP2_REFINE_TC     0x100
/* Final epilogue of the 256 x 256 pair tiles in the layers of the main format
 * (Z_{k+1}, A_{k+1} and the next layer's operands from a finished tile).  By
 * default it is deferred when the tiles are long (mean order n over the pair
 * tiles >= 3072): the accumulating warps pass a finished tile's sums to two
 * store warps per CTA through a scratch in the workspace (128 KB per CTA, at
 * most 192 CTAs) and go on with the next tile, so that the epilogue's memory
 * traffic overlaps the next tile's MMAs; for shorter tiles the accumulating
 * warps run it inline.  These two flags force one or the other (results are
 * identical). */
#define FTSP2_EPI_DEFERRED  0x200
#define FTSP2_EPI_INLINE    0x400
/* Operand storage of the FP16X2 / BF16X3 tensor-core layers.  The square of a
 * symmetric matrix needs its full row panels, but by default a layer stores
 * the next operands only for the upper triangle (plus the diagonal tile
 * blocks), and the next layer loads the K-slices left of a panel's diagonal
 * block as transposed panels of the upper triangle (MN-major tcgen05
 * operands).  This halves the operand stores of the epilogue.  With this flag
 * every layer writes and reads full matrices (results are identical). */
#define FTSP2_FULL_OPERANDS 0x800
/* Layer launches.  When a launch of the tensor-core layer kernel would run a
 * few waves of tiles (at most 8 per unit), consecutive layers of the main
 * format run in one persistent cooperative launch.  Its work items are (layer,
 * tile) in layer order, and an item of layer g starts once every tile of layer
 * g - 1 of the same chain is finished (device-side counters; bounded waits
 * that end in FTSP2_E_TIMEOUT).  The last tiles of one layer then overlap the
 * first tiles of the next chain's layer, instead of leaving units idle at the
 * end of every launch.  This flag forces one launch per layer (results are
 * identical). */
#define FTSP2_LAYER_LAUNCHES 0x1000

/* One Hamiltonian of a (ragged) batch.  H_b starts at dH + offset and is
 * n x n row-major; D_b starts at dD + offset.  Offsets are in elements. */
typedef struct {
    int32_t n;          /* order, >= 1                                        */
    int32_t reserved;
    int64_t offset;     /* element offset into dH and dD                      */
    double mu;          /* chemical potential (eV)                            */
    double kT;          /* electronic temperature (eV), > 0                   */
} ftsp2_instance;

/* One trained model (Sec. III A 2, "a set of models").
 *
 * family FTSP2_FAMILY_MLSP2: theta holds L rows (a, b, c, d) = (theta_i1,
 * theta_i2, theta_i3, theta_i4) of Eq. mlsp2, acting on the layer-0 input
 * x0 = H0 without an inner flip and approximating 1/(1 + exp(-beta0 (x - mu0)))
 * on [0, 1].
 *
 * family FTSP2_FAMILY_SKIP: Skip-SP2 (Sec. II A 3) with one stored layer and
 * one accumulator; theta holds L + 1 rows of 4 doubles: layer rows
 * (delta_i, alpha_i, beta_i, gamma_i) with u_i = delta_i + alpha_i x_i +
 * beta_i A_i, A_{i+1} = A_i + gamma_i x_i, x_{i+1} = u_i^2, and the output row
 * (A_0, gamma_L, 0, 0): the accumulator starts at A_0 and
 * f = A_L + gamma_L x_L.  The accumulator feeding back into the squared
 * combination (beta_i) is what the family adds; beta = 0 covers Eq. mlsp2
 * through the embedding of the Appendix on model embeddings.
 *
 * family FTSP2_FAMILY_MAX: Max-SP2 (Sec. II A 2, Eq. maxsp2), every layer the
 * square of an affine combination of all the layers before it:
 * u_i = delta_i + sum_{j<=i} theta_{i,j} x_j, x_{i+1} = u_i^2, and
 * f = c + sum_{j<=L} gamma_j x_j (Eq. maxsp2 has c = 0; Alg. maxsp2 a
 * constant in place of gamma_0 x_0).  theta is flat: for i = 0 .. L-1 the
 * block (delta_i, gamma_i, theta_{i,0}, ..., theta_{i,i}), then (c, gamma_L):
 * L (L + 5) / 2 + 2 doubles, L <= 20.  The layers keep every x_j, so a solve
 * holds L + 1 FP32 state planes per chain (size workspaces with
 * ftsp2_workspace_size_set).  These tables run in FTSP2_FP32 mode only
 * (FTSP2_E_UNSUPPORTED otherwise).  Skip-SP2 tables with k stored layers and
 * K accumulators run through their Max-SP2 embedding (ftsp2_skip_to_max).
 *
 * theta_entropy holds the entropy recursion's rows (Eq. entropy expansion) in
 * the same family (L_entropy layers) or is NULL to reuse theta (the
 * theta_fermi strategy).  alpha is the entropy input scale of Eq. entropy
 * expansion.  All pointers are host pointers, copied at creation.  A set may
 * mix families. */
#define FTSP2_FAMILY_MLSP2 0
#define FTSP2_FAMILY_SKIP  1
#define FTSP2_FAMILY_MAX   2
typedef struct {
    int32_t L;
    int32_t L_entropy;
    double beta0;
    double mu0;
    double alpha;
    const double* theta;
    const double* theta_entropy;
    int32_t family;          /* FTSP2_FAMILY_*                               */
    int32_t reserved;
} ftsp2_table;

typedef struct ftsp2_model_set ftsp2_model_set;   /* opaque */

/* Per-instance record written by ftsp2_rescale / ftsp2_density /
 * ftsp2_entropy (device memory, 64 bytes each). */
typedef struct {
    double e_min, e_max;   /* Gershgorin bounds (Appendix A)                  */
    double mu_p;           /* mu' after the flip (Eq. mu', Eq. flip)          */
    double beta_p;         /* beta' (after clamping, if any)                  */
    double scale;          /* X0 = mu0 I + scale (mu I - H): scale = +-beta_eff/beta0 */
    int32_t flip;          /* 1 if Eq. flip was applied (mu' > 1/2)           */
    int32_t model;         /* index into the model set, -1 if none is valid   */
    int32_t status;        /* ftsp2_status of this instance                   */
    int32_t layers;        /* layers run for this instance                    */
    int32_t valid;         /* 1 if inside the chosen model's region          */
    int32_t reserved;
} ftsp2_rescale_rec;

/* ---- model sets -------------------------------------------------------- */

/* Copies `ntab` tables to the device (one cudaMalloc, owned by the set) and
 * precomputes the per-layer constants the kernels use.  Tables must satisfy
 * 1 <= L <= 64, beta0 > 0, 0 < mu0 < 1.  Returns FTSP2_E_NOMODEL for ntab < 1. */
ftsp2_status ftsp2_model_set_create(const ftsp2_table* tabs, int ntab, ftsp2_model_set** out);

/* Model set holding the 26-layer table printed in the paper's Appendix A
 * (beta0 = 1500, mu0 = 1/3; theta_fermi entropy with alpha = 0.842704). */
ftsp2_status ftsp2_model_set_builtin(ftsp2_model_set** out);

void ftsp2_model_set_destroy(ftsp2_model_set* set);

/* Number of tables and the largest layer count in the set. */
ftsp2_status ftsp2_model_set_info(const ftsp2_model_set* set, int* ntab, int* max_layers);

/* Copy of table `idx` of the set: *L layers, theta_out (host, room for 4*64
 * doubles) receives the table's rows as given at creation (Eq. mlsp2: L rows
 * (a, b, c, d); Skip-SP2: L + 1 rows; Max-SP2: the flat table); any output
 * pointer may be NULL.  A Skip-SP2 table has at most 63 layers. */
ftsp2_status ftsp2_model_set_table(const ftsp2_model_set* set, int idx, int* L, double* theta_out,
                                   double* beta0, double* mu0, double* alpha);

/* ---- workspace ------------------------------------------------------------ */

/* Bytes of device workspace needed by a density/entropy call with these
 * instances and mode.  `want` = 1 density, 2 entropy, 3 both.  The size covers
 * every flag (refinement layers, Lanczos bounds, the deferred epilogue's
 * scratch). */
ftsp2_status ftsp2_workspace_size(const ftsp2_instance* inst, int nb, ftsp2_mode mode,
                                  int want, size_t* bytes);

/* The same for a given model set: also covers the state planes that Max-SP2
 * tables of the set keep (L + 1 per chain instead of 2).  Equal to
 * ftsp2_workspace_size for sets without such tables. */
ftsp2_status ftsp2_workspace_size_set(const ftsp2_instance* inst, int nb, const ftsp2_model_set* set,
                                      ftsp2_mode mode, int want, size_t* bytes);

/* ---- the hot path ------------------------------------------------------------ */

/* Bytes of device workspace ftsp2_rescale needs for nb instances (any
 * workspace sized by ftsp2_workspace_size for the same instances also fits). */
ftsp2_status ftsp2_rescale_workspace_size(int nb, size_t* bytes);

/* (a1)+(a2) only: Gershgorin bounds, normalisation, flip, validity and model
 * choice for every instance; writes dRec[nb].  dInst is a device copy of inst
 * (same contents; the kernels read it, the host plans from inst).  ws must be
 * 1024-byte aligned and hold ftsp2_rescale_workspace_size(nb) bytes, or, with
 * FTSP2_LANCZOS, ftsp2_workspace_size(inst, nb, any mode, 1) bytes
 * (FTSP2_E_WORKSPACE otherwise). */
ftsp2_status ftsp2_rescale(const double* dH, const ftsp2_instance* inst,
                           const ftsp2_instance* dInst, int nb,
                           const ftsp2_model_set* set, int flags,
                           ftsp2_rescale_rec* dRec, void* ws, size_t ws_bytes,
                           void* stream);

/* (a1)-(a4): density matrices.  dD receives D_b at its offset (full symmetric
 * matrix, FP32).  dTrace (nullable) receives 2 doubles per instance:
 * Tr D_b and ||D_b||_F^2 (Eq. tr(D^2)), accumulated in FP64.  dRec receives
 * the per-instance records.  ws must hold ftsp2_workspace_size(..., want=1)
 * bytes and be 1024-byte aligned. */
ftsp2_status ftsp2_density(const double* dH, const ftsp2_instance* inst,
                           const ftsp2_instance* dInst, int nb,
                           const ftsp2_model_set* set, ftsp2_mode mode, int flags,
                           float* dD, double* dTrace, ftsp2_rescale_rec* dRec,
                           void* ws, size_t ws_bytes, void* stream);

/* (a1), (a2), (a5), (a6): entropies only.  dS receives one double per
 * instance: S_b = 4 ln2 (Tr F - Tr F^2), F = A_S + Y (Eq. entropy expansion-s,
 * taken with the sign that makes S >= 0). */
ftsp2_status ftsp2_entropy(const double* dH, const ftsp2_instance* inst,
                           const ftsp2_instance* dInst, int nb,
                           const ftsp2_model_set* set, ftsp2_mode mode, int flags,
                           double* dS, ftsp2_rescale_rec* dRec,
                           void* ws, size_t ws_bytes, void* stream);

/* CUDA graphs.  ftsp2_density, ftsp2_entropy and ftsp2_density_entropy only
 * launch kernels on `stream` (planning is host-side arithmetic; the workspace
 * is the caller's), so a call may be recorded by stream capture and the graph
 * replayed: each replay recomputes the batch from the current contents of dH
 * and the device copy dInst, into the same output buffers.  The pointers,
 * instance sizes, model set and flags are fixed at capture; mu and kT may be
 * changed between replays through dInst.  Make one uncaptured call with the
 * same arguments first (it sets per-kernel attributes), and do not pass
 * FTSP2_SYNC while capturing (FTSP2_E_ARG).  Layer profiling
 * (ftsp2_profile_layers) skips captured launches. */

/* (a1)-(a6) in one pass: both recursions share the bounds and the rescale and
 * run as two problems of the same grouped launch per layer (Alg. 2 runs them
 * in one loop).  Any of dD, dTrace, dS may be NULL (dD and dS not both). */
ftsp2_status ftsp2_density_entropy(const double* dH, const ftsp2_instance* inst,
                                   const ftsp2_instance* dInst, int nb,
                                   const ftsp2_model_set* set, ftsp2_mode mode, int flags,
                                   float* dD, double* dTrace, double* dS,
                                   ftsp2_rescale_rec* dRec,
                                   void* ws, size_t ws_bytes, void* stream);

/* Density without allocation.  Same computation and arguments as
 * ftsp2_density, but the workspace comes from an 8 MiB array inside the
 * library's device image instead of from the caller.  It is meant for callers
 * that cannot allocate device memory where they need D: code running while a
 * stream is being captured into a CUDA graph, plug-ins whose host application
 * owns all device memory, loops that must not pay for cudaMalloc.  (The paper
 * has no counterpart; this is an interface convenience of this library.)
 *   - Allocates nothing: no cudaMalloc, no cudaFree, no host buffers.  The
 *     model set must have been created beforehand.
 *   - Limit: the batch must fit the 8 MiB array.  It needs about
 *     nb * P^2 * (8 + 2 b) bytes plus a few KiB of bookkeeping, where P is the
 *     largest n rounded up to 128 and b the operand bytes per element (4 for
 *     FTSP2_FP16X2 and FTSP2_FP32, 6 for FTSP2_BF16X3, 8 for FTSP2_TF32X3;
 *     FTSP2_REFINE1/2 add 8, or 12 with FTSP2_REFINE_TC).  A single FP16X2
 *     instance fits up to n = 640.
 *     Larger batches are rejected with FTSP2_E_WORKSPACE before any launch.
 *     FTSP2_SYNC is refused (FTSP2_E_ARG); read dRec instead.
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.  A first call made while `stream` is being
 *     captured is refused with FTSP2_E_ARG, before the lookup and before any
 *     launch.
 *   - Every call uses the same array and leaves its contents behind; each call
 *     rewrites everything it reads before reading it.  Calls that overlap on
 *     the GPU (other streams, other host threads) race on the array: serialise
 *     them. */
ftsp2_status ftsp2_density_noalloc(const double* dH, const ftsp2_instance* inst,
                                   const ftsp2_instance* dInst, int nb,
                                   const ftsp2_model_set* set, ftsp2_mode mode, int flags,
                                   float* dD, double* dTrace, ftsp2_rescale_rec* dRec,
                                   void* stream);

/* ---- chemical potential for a prescribed electron count -------------------------- */

/* Newton-Raphson on g(mu) = N_occ - Tr D(mu) (Sec. III A 4, Eqs. g, dg,
 * delta_mu), entirely on the device.  Differentiating the Fermi operator
 * (Eq. FD_Func) gives dD/dmu = +beta D (I - D) (the printed Eq. drho has the
 * opposite sign), so one update is
 *     Delta mu = (N_occ - Tr D) / (beta (Tr D - ||D||_F^2)),
 * from the traces the density call already returns (Eq. tr(D^2)), limited to
 * |Delta mu| <= (e_max - e_min) / 16.  An instance takes no step once
 * |N_occ - Tr D| <= tol, when Tr D - ||D||_F^2 <= 0, or while it has no valid
 * model.
 *   - The starting mu is dInst[b].mu; every update is written there (device
 *     memory, the caller's table; inst on the host is not changed and is used
 *     for planning only).
 *   - The call runs `iterations` + 1 evaluations of the hot path (bounds,
 *     rescale and model choice are redone for every mu) and `iterations`
 *     updates in between; dD, dTrace, dS (nullable: then no entropy chain) and
 *     dRec hold the result at the final mu.  dSteps[b] receives the number of
 *     updates instance b took.  dNocc: nb doubles (device), the electron counts
 *     per spin channel (0 <= N_occ <= n).
 *   - Workspace as for ftsp2_density_entropy (want = 3 when dS is given, else 1).
 *   - Launches only; no host synchronisation unless FTSP2_SYNC (then the worst
 *     final per-instance status is returned).  Capturable into a CUDA graph.
 *   - Errors: FTSP2_E_ARG for iterations outside [0, 64], tol < 0 or NULL
 *     dNocc / dTrace / dSteps; otherwise those of ftsp2_density_entropy. */
ftsp2_status ftsp2_density_mu(const double* dH, const ftsp2_instance* inst, ftsp2_instance* dInst, int nb,
                              const double* dNocc, const ftsp2_model_set* set, ftsp2_mode mode, int flags,
                              int iterations, double tol, float* dD, double* dTrace, double* dS,
                              ftsp2_rescale_rec* dRec, int32_t* dSteps, void* ws, size_t ws_bytes,
                              void* stream);

/* ---- tile-shape autotuner ------------------------------------------------------ */

/* Measures the batch with both tensor-core tile shapes and records the faster.
 * Arguments are those of ftsp2_density_entropy (the buffers are written as by
 * that call; the results of the last run are left in them).  For each shape
 * the batch runs once untimed and then `reps` times between CUDA events on
 * `stream`; ms[0] receives the mean time of the 128 x 128 single-CTA shape,
 * ms[1] that of the 256 x 256 pair shape (ms nullable), *choice the shape kept
 * (0 single, 1 pair; -1 in FTSP2_FP32 mode, which has no tensor-core layers and
 * is not timed).  The record is keyed by device, mode, density/entropy
 * selection, refinement flags and the sorted list of orders n, lives for the
 * life of the process, and is shared by all threads (guarded by a mutex).
 * Synchronises `stream`.  Not usable during stream capture.  FTSP2_PAIR_TILES
 * and FTSP2_SINGLE_TILES in `flags` are ignored here.  Errors: those of
 * ftsp2_density_entropy; FTSP2_E_ARG if reps < 1. */
ftsp2_status ftsp2_autotune(const double* dH, const ftsp2_instance* inst,
                            const ftsp2_instance* dInst, int nb,
                            const ftsp2_model_set* set, ftsp2_mode mode, int flags,
                            float* dD, double* dTrace, double* dS,
                            ftsp2_rescale_rec* dRec, void* ws, size_t ws_bytes,
                            int reps, int* choice, float* ms, void* stream);

/* The tile shape a call with these arguments would use on the current device:
 * 1 pair, 0 single, -1 none (FTSP2_FP32 mode).  `want` as in
 * ftsp2_workspace_size.  *from_tuner is set to 1 if the shape comes from an
 * ftsp2_autotune record, 0 if from the flags or the padding model.  Host-only
 * apart from reading the device's SM count. */
ftsp2_status ftsp2_tile_shape(const ftsp2_instance* inst, int nb, ftsp2_mode mode, int want,
                              int flags, int* shape, int* from_tuner);

/* Forgets every ftsp2_autotune record. */
ftsp2_status ftsp2_autotune_clear(void);

/* ---- training (a7) -------------------------------------------------------------- */

typedef struct {
    int32_t iterations;     /* LM iterations run                               */
    int32_t accepted;       /* accepted steps                                  */
    double cost0, cost;     /* 0.5 sum r^2 at start and end                    */
    double max_err;         /* max |model - target| on the samples              */
    double lambda;          /* final damping                                    */
} ftsp2_train_report;

#define FTSP2_TARGET_FERMI   0  /* 1/(1 + exp(-beta0 (x - mu0)))                */
#define FTSP2_TARGET_ENTROPY 1  /* s(beta0 (x - mu0)) of Eq. entropy, model
                                   4 ln2 F (1 - F) with x0 = alpha (x - mu0) + mu0 */

/* Levenberg-Marquardt with optional geodesic acceleration (Sec. II C 2) of
 * an L-layer Eq. mlsp2 table on nsamples scalar samples.
 *   - Samples (Sec. II C 1): the library builds them (ftsp2_train_samples with
 *     the same beta0, mu0, nsamples, seed) and keeps them fixed for the whole
 *     fit; seed 0 gives the deterministic quantile grid.
 *   - theta_init (host, L*4, nullable): the starting table; NULL starts from
 *     ftsp2_train_init(L, beta0, mu0) (the SP2 sequence at mu0 with its slope
 *     matched to beta0/4).  theta_out (host, L*4) receives the result.
 *   - target FTSP2_TARGET_FERMI or FTSP2_TARGET_ENTROPY (then the model input
 *     is alpha (x - mu0) + mu0, Eq. entropy expansion); iterations >= 0 LM
 *     steps; accel != 0 enables geodesic acceleration.
 *   - Residuals, Jacobian rows and the reductions J^T J, J^T r run on the GPU
 *     in FP64; the damped normal equations are solved on the host by Cholesky
 *     in FP64.
 *   - dWork (device) must hold ftsp2_train_workspace_size(nsamples, L) bytes
 *     (the samples live there too).  Synchronous on `stream`.
 * Errors: FTSP2_E_ARG for L outside 1..64, nsamples < 1, beta0 <= 0, mu0
 * outside (0, 1), a bad target, NULL outputs or non-finite start entries;
 * FTSP2_E_WORKSPACE for a short workspace. */
size_t ftsp2_train_workspace_size(int nsamples, int L);
ftsp2_status ftsp2_train_coeffs(int target, double beta0, double mu0, int L, double alpha,
                                int nsamples, uint64_t seed, int iterations, int accel,
                                const double* theta_init, double* theta_out,
                                ftsp2_train_report* rep, void* dWork, size_t work_bytes,
                                void* stream);

/* The training sample set (Sec. II C 1), host only: x_out[nsamples] in [0, 1]
 * at the quantiles of the density p(x) = 1 + |f'(x)|, f the increasing
 * logistic 1/(1 + exp(-beta0 (x - mu0))): the CDF of p is integrated by the
 * trapezoid rule on 2,000,001 evenly spaced points and inverted by linear
 * interpolation at q_s = (s + 1/2)/nsamples (seed 0) or
 * q_s = (s + u_s)/nsamples with u_s the top 53 bits of splitmix64(seed + s)
 * scaled to [0, 1) (one point in each equal-probability cell). */
ftsp2_status ftsp2_train_samples(double beta0, double mu0, int nsamples, uint64_t seed, double* x_out);

/* Starting tables, host only (reading of the "scaled and truncated SP2"
 * initial guess of Sec. II A 1):
 *   ftsp2_train_init: the SP2 sequence for a known chemical potential
 *     (Eq. sp2-mu) at mu0 as Eq. mlsp2 rows (Appendix C: X^2 -> (1, 0, 0, 0),
 *     2X - X^2 -> (-1, 2, 0, 0)), with the contraction x -> mu0 + kappa
 *     (x - mu0) folded into layer 0, kappa = min(1, (beta0/4) / slope), the
 *     slope of the sequence at mu0 being the product of the layers'
 *     derivatives along the trajectory of mu0 (L*4 doubles out);
 *   ftsp2_train_init_alt: the same SP2 sequence in the one-term form
 *     (Eq. mlsp2_alt; (L + 1)*2 doubles out);
 *   ftsp2_mlsp2_to_skip: the Appendix embedding of L Eq. mlsp2 rows (every
 *     a_i != 0) as a Skip-SP2 table with one stored layer and one accumulator
 *     ((L + 1)*4 doubles out; L <= 63).
 * ftsp2_layer_count: Eq. layer count, ln(beta'/4) / ln(2 / varphi), the
 * fewest layers a table needs to reach the slope beta'/4 (NaN for beta' <= 0). */
ftsp2_status ftsp2_train_init(int L, double beta0, double mu0, double* theta_out);
ftsp2_status ftsp2_train_init_alt(int L, double mu0, double* alt_out);
ftsp2_status ftsp2_mlsp2_to_skip(int L, const double* theta, double* skip_out);
double ftsp2_layer_count(double beta_p);

/* Residuals model - target of a table (family FTSP2_FAMILY_MLSP2: L rows of
 * 4; FTSP2_FAMILY_SKIP: L + 1 rows of 4; FTSP2_FAMILY_MAX: the flat table,
 * L <= 20) at npoints device points dX, into dR (device), FP64, no Jacobian:
 * used to measure a table's error on a grid. */
ftsp2_status ftsp2_train_residuals(int family, int target, double beta0, double mu0, int L, double alpha,
                                   const double* table, const double* dX, int npoints, double* dR,
                                   void* stream);

/* The one-term form of the recursion (Eq. mlsp2_alt).  A table of this form
 * holds L + 1 rows (t_i1, t_i2), (L + 1) * 2 doubles: layers
 * x_{i+1} = (t_i1 + x_i)^2, A_{i+1} = A_i + t_i2 x_i for i < L, and the output
 * row (t_L1, t_L2) with f = A_L + t_L1 + t_L2 x_L (Eq. mlsp2_alt-output).
 * ftsp2_alt_to_mlsp2 writes the L rows (a, b, c, d) of Eq. mlsp2 that compute
 * the same function (the embedding of the Appendix on model embeddings):
 * (1, 2 t_i1, t_i1^2, t_i2), with the last layer's (a, b, c) multiplied by
 * t_L2 and t_L1 added to its c.  Such rows go into an ftsp2_table like any
 * other; the layer kernels run them unchanged (their centred epilogue folds
 * every term of a layer into one pass whichever form the table has).
 * FTSP2_E_ARG for L outside 1..64 or non-finite entries. */
ftsp2_status ftsp2_alt_to_mlsp2(int L, const double* alt, double* theta_out);

/* Embeddings in Max-SP2 (the Appendix on model embeddings: MLSP2 in Skip-SP2
 * in Max-SP2), host only; max_out receives the flat Max-SP2 table
 * (L (L + 5) / 2 + 2 doubles) computing the same function.
 *   ftsp2_mlsp2_to_max: L Eq. mlsp2 rows (every a_i != 0), through the
 *     Skip-SP2 embedding of ftsp2_mlsp2_to_skip.
 *   ftsp2_skip_to_max: a Skip-SP2 table with k stored layers and K
 *     accumulators (Sec. II A 3): u_i = alpha_{i,k} + sum_{j<min(k,i+1)}
 *     alpha_{i,j} x_{i-j} + sum_l beta_{i,l} A_{i,l},
 *     A_{i+1,l} = A_{i,l} + gamma_{i,l} x_i, x_{i+1} = u_i^2,
 *     f = gamma_L x_L + sum_l A_{L,l} (the paper writes gamma_L = 1; the
 *     embedding of Eq. mlsp2 needs the weight); alpha is L x (k + 1)
 *     row-major (the constant alpha_{i,k} last), beta and gamma L x K, A0
 *     the K initial accumulators (beta, gamma, A0 may be NULL when K = 0).
 *     With A_{i,l} = A_{0,l} + sum_{j<i} gamma_{j,l} x_j:
 *     delta_i = alpha_{i,k} + sum_l beta_{i,l} A_{0,l},
 *     theta_{i,j} = sum_l beta_{i,l} gamma_{j,l} [j < i] + alpha_{i,i-j} [i - j < k],
 *     c = sum_l A_{0,l}, gamma_j = sum_l gamma_{j,l} (j < L), and gamma_L.
 * FTSP2_E_ARG for L outside 1..20, k < 1, K < 0, or non-finite entries. */
ftsp2_status ftsp2_mlsp2_to_max(int L, const double* theta, double* max_out);
ftsp2_status ftsp2_skip_to_max(int L, int k, int K, const double* alpha, const double* beta, const double* gamma,
                               const double* A0, double gamma_L, double* max_out);

/* Levenberg-Marquardt training in the one-term form: as ftsp2_train_coeffs,
 * with alt_init / alt_out (host) of (L + 1) * 2 doubles (alt_init NULL:
 * ftsp2_train_init_alt(L, mu0)).  The GPU computes the
 * Eq. mlsp2 Jacobian of the mapped table and its reductions J^T J, J^T r; the
 * host applies the chain rule of ftsp2_alt_to_mlsp2 (P^T J^T J P, P^T J^T r,
 * P = d theta / d t) and solves for the 2L + 2 parameters.  Same workspace
 * (ftsp2_train_workspace_size(nsamples, L)). */
ftsp2_status ftsp2_train_coeffs_alt(int target, double beta0, double mu0, int L, double alpha,
                                    int nsamples, uint64_t seed, int iterations, int accel,
                                    const double* alt_init, double* alt_out, ftsp2_train_report* rep,
                                    void* dWork, size_t work_bytes, void* stream);

/* Levenberg-Marquardt training of a Skip-SP2 table (FTSP2_FAMILY_SKIP, one
 * stored layer and one accumulator): as ftsp2_train_coeffs, with skip_init /
 * skip_out (host) of (L + 1) * 4 doubles (layer rows, then the output row
 * (A_0, gamma_L, 0, 0)); skip_init NULL starts from the embedding of
 * ftsp2_train_init(L, beta0, mu0).  The 4L + 2 parameters get their own
 * forward and reverse sweep on the GPU.  dWork must hold
 * ftsp2_train_workspace_size(nsamples, L + 1) bytes; L <= 63. */
ftsp2_status ftsp2_train_coeffs_skip(int target, double beta0, double mu0, int L, double alpha,
                                     int nsamples, uint64_t seed, int iterations, int accel,
                                     const double* skip_init, double* skip_out, ftsp2_train_report* rep,
                                     void* dWork, size_t work_bytes, void* stream);

/* Levenberg-Marquardt training of the families that keep stored layers
 * (Sec. II A 2 and II A 3), as ftsp2_train_coeffs otherwise (samples, seed,
 * geodesic acceleration, report, stream).  L <= 20; dWork must hold
 * ftsp2_train_workspace_size_max(nsamples, L) bytes (room for the
 * L (L + 5) / 2 + 3 columns of the augmented Max-SP2 Jacobian).
 * ftsp2_train_coeffs_max: a flat Max-SP2 table (FTSP2_FAMILY_MAX layout);
 *   max_init NULL starts from ftsp2_mlsp2_to_max of ftsp2_train_init(L,
 *   beta0, mu0).  The GPU runs the Max-SP2 forward and reverse sweep.
 * ftsp2_train_coeffs_skipk: a Skip-SP2 table with k stored layers and K
 *   accumulators (1 <= k <= L, K >= 1) as the vector
 *   (alpha (L x (k + 1), constant last), beta (L x K), gamma (L x K),
 *   A_{0,1}, gamma_L): (1 + k + 2K) L + 2 doubles, the paper's count, the
 *   other initial accumulators zero.  The model is its Max-SP2 embedding
 *   (ftsp2_skipk_to_max), the GPU forms the Max-SP2 Jacobian and its
 *   reductions, the host applies the embedding's exact Jacobian
 *   (P^T J^T J P, P^T J^T r); a parameter whose J^T J diagonal is zero at the
 *   current point is damped with the smallest positive diagonal entry.
 *   skip_init NULL starts from ftsp2_train_init_skipk.
 * ftsp2_train_init_skipk (host): the default start, the one-accumulator
 *   embedding (ftsp2_mlsp2_to_skip) of ftsp2_train_init(L, beta0, mu0) in
 *   stored-layer slot 0 and accumulator 1; the further stored layers and
 *   accumulator inputs gamma zero, the further accumulators' feedback beta
 *   0.01 (no effect on the function while those accumulators are zero).
 * ftsp2_skipk_to_max (host): the flat Max-SP2 table of such a vector. */
size_t ftsp2_train_workspace_size_max(int nsamples, int L);
ftsp2_status ftsp2_train_coeffs_max(int target, double beta0, double mu0, int L, double alpha, int nsamples,
                                    uint64_t seed, int iterations, int accel, const double* max_init,
                                    double* max_out, ftsp2_train_report* rep, void* dWork, size_t work_bytes,
                                    void* stream);
ftsp2_status ftsp2_train_coeffs_skipk(int target, double beta0, double mu0, int L, int k, int K, double alpha,
                                      int nsamples, uint64_t seed, int iterations, int accel,
                                      const double* skip_init, double* skip_out, ftsp2_train_report* rep,
                                      void* dWork, size_t work_bytes, void* stream);
ftsp2_status ftsp2_train_init_skipk(int L, int k, int K, double beta0, double mu0, double* skip_out);
ftsp2_status ftsp2_skipk_to_max(int L, int k, int K, const double* skip, double* max_out);

/* Building blocks of one LM iteration, exposed for parity tests.
 * ftsp2_train_residual_jacobian: residuals dR[nsamples] = model(theta) - target
 * and (if dM != NULL) the augmented Jacobian dM[(4L+1) * nsamples],
 * parameter-major: dM[j * nsamples + s] = d model(x_s) / d theta_j for the
 * flattened table (a_0, b_0, c_0, d_0, a_1, ...), j < 4L, by reverse
 * accumulation, and dM[4L * nsamples + s] = r_s.  theta is a host array.
 * ftsp2_train_normal_equations: dG[(4L+1)^2] = M^T M (row-major), i.e.
 * [[J^T J, J^T r], [r^T J, r^T r]], reduced in FP64 in a fixed order; dWork
 * must hold ftsp2_train_workspace_size(nsamples, L) bytes. */
ftsp2_status ftsp2_train_residual_jacobian(int target, double beta0, double mu0, int L,
                                           double alpha, const double* theta,
                                           const double* dX, int nsamples,
                                           double* dR, double* dM, void* stream);
ftsp2_status ftsp2_train_normal_equations(const double* dM, int nsamples, int L, double* dG,
                                          void* dWork, size_t work_bytes, void* stream);

/* ---- measurement support ------------------------------------------------- */

/* While enabled, every tensor-core layer launch is bracketed by a CUDA event
 * pair recorded on the caller's stream (host-side events, created on demand;
 * not usable during stream capture).  ftsp2_profile_read synchronises those
 * events and returns the summed layer-kernel time (ms) and the number of
 * layers measured since the last read (a multi-layer launch counts its
 * layers), then clears the record. */
ftsp2_status ftsp2_profile_layers(int enable);
ftsp2_status ftsp2_profile_read(double* total_ms, uint64_t* launches);

/* ---- misc ---------------------------------------------------------------- */

const char* ftsp2_status_string(ftsp2_status s);

/* Number of kernels this library launched since load (all entry points). */
uint64_t ftsp2_kernel_launch_count(void);

/* ---- bounded device-side waits ------------------------------------------------- */

/* Every wait inside a layer kernel is bounded by this limit (ns; default 4e9,
 * process-wide, read at each call).  The waits are those of the multi-layer
 * launches (an item waits until every tile of the previous layer of its chain
 * has finished) and of the kernel's internal pipeline barriers.  When a
 * dependency wait runs out, the kernel records FTSP2_E_TIMEOUT in the call's
 * status word and every CTA finishes its work list in a skip mode that keeps
 * the barrier protocol (no loads, MMAs or stores), so nothing is left in
 * flight and the context stays usable; the per-instance records then carry
 * FTSP2_E_TIMEOUT (returned with FTSP2_SYNC) and the outputs are not valid.
 * The next call starts from a cleared status word.  (No counterpart in the
 * paper: a property of this implementation's persistent launches.)
 * FTSP2_E_ARG unless 1e5 <= ns <= 6e10. */
ftsp2_status ftsp2_set_wait_limit_ns(uint64_t ns);
uint64_t ftsp2_wait_limit_ns(void);

/* Test hook for the bounded waits: while layer >= 0, items of that global
 * layer inside a multi-layer launch wait for one completion more than their
 * predecessor layer can give, so their dependency wait runs out after the
 * wait limit.  -1 (the default) turns it off.  Process-wide; for tests only.
 * FTSP2_E_ARG for layer < -1 or >= 64. */
ftsp2_status ftsp2_debug_stall_layer(int layer);

#ifdef __cplusplus
}
#endif

#endif /* FTSP2_H */
