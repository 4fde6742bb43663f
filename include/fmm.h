/*
 * fmm.h -- C ABI of the B300 adaptive FMM Poisson solver.
 *
 * The library computes the gravitational potential and acceleration of every
 * leaf cell of a graded AMR octree with isolated boundaries, following the
 * adaptive FMM of Lee & Teyssier (arXiv 2607.19489): one FMM tree per AMR level
 * (Sec. 3.1), P2M/M2M upward pass (Eqs. 1-2), M2L over the 6^3-3^3 interaction
 * list and L2L downward pass (Eqs. 3-4, Alg. 3), and the far / intermediate /
 * near / nearest field evaluation (Sec. 3.2, Fig. 2, Alg. 4).
 *
 * Geometry.  The domain is the unit box [0,1)^3.  Level l has 2^l cells per
 * axis of size h_l = 2^-l; cell (i,j,k) has centre ((i,j,k)+1/2) h_l and is a
 * point mass there.  Levels lmin..lmax hold leaf cells; a cell is refined when
 * cells exist one level finer inside it.  RAMSES rules apply: refined cells
 * have all 8 children (octs), level lmin covers the whole box, and a cell may
 * be refined only if the 3^3 neighbours of its father are refined (Sec. 3.2).
 *
 * Conventions.  g(R) = -1/|R|; phi_i = G sum_{j != i} m_j g(x_i - x_j) as
 * approximated by the FMM; accel = -grad phi.  Expansion order p applies to
 * multipoles and locals alike; M2L keeps |alpha|+|beta| <= p (Eq. 3).
 *
 * Errors.  Every call returns an fmm_status.  No call aborts or throws.
 * Device-side errors found by kernels are latched in the context and returned
 * by the next call that synchronises (fmm_set_levels, fmm_sync).
 *
 * Streams.  `stream` is a cudaStream_t passed as void*; NULL is the legacy
 * default stream.  fmm_solve is asynchronous on that stream; it allocates
 * nothing and never synchronises (all workspace is sized by fmm_set_levels).
 *
 * Threading.  A context may be used by one host thread at a time.
 */
#ifndef FMM_H
#define FMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fmm_ctx fmm_ctx;

typedef enum {
  FMM_OK = 0,
  FMM_ERR_ARG = -1,         /* bad argument (NULL pointer, level range, p, ...) */
  FMM_ERR_NOT_GRADED = -2,  /* hierarchy violates the graded-octree rule (Sec. 3.2) */
  FMM_ERR_DUPLICATE = -3,   /* a cell given twice, or given as a leaf while refined */
  FMM_ERR_OUT_OF_BOX = -4,  /* a cell index outside [0, 2^l) */
  FMM_ERR_OOM = -5,         /* device allocation failed or exceeded the budget */
  FMM_ERR_CUDA = -6,        /* a CUDA runtime call failed (fmm_last_error has the text) */
  FMM_ERR_NONFINITE = -7,   /* a mass is NaN or infinite */
  FMM_ERR_STATE = -8,       /* call out of order (e.g. solve before set_levels) */
  FMM_ERR_TIMEOUT = -9,     /* a bounded device-side wait gave up */
  FMM_ERR_INCOMPLETE = -10  /* a refined cell lacks some of its 8 children, or the
                               base level does not cover the box */
} fmm_status;

typedef enum {
  FMM_FP64 = 0,          /* every step in FP64 (DFMA) */
  FMM_MIXED_BF16X3 = 1,  /* M2L/M2P on tcgen05 tensor cores in split-BF16 (3 products,
                            FP32 accumulation), everything else in FP32; with
                            config.fp64_top the M2M of box levels <= 3 and the L2L
                            chain with its local-expansion accumulation run in FP64 */
  FMM_MIXED_TF32 = 2     /* as FMM_MIXED_BF16X3, but M2L/M2P in one TF32 product per
                            term (tcgen05 kind::tf32, FP32 accumulation) */
} fmm_precision;

/* The bottom intermediate field of a target cell t at level l: the sources in the
 * interaction list of t's parent box F (level l-1). */
typedef enum {
  FMM_BOTTOM_M2P = 0,     /* the paper's (Fig. 2, Alg. 4): M2P from each source to t */
  FMM_BOTTOM_M2L_L2P = 1  /* M2L (Eq. 3) / P2L from each source into F's local
                             expansion, which also receives F's parent's by L2L
                             (Eq. 4); t evaluates it by L2P.  The downward pass runs one
                             level further; the truncation differs from M2P's. */
} fmm_bottom_mode;

typedef struct {
  int p;              /* expansion order of the local expansions, 1..8 (Eq. 3 truncation) */
  int precision;      /* fmm_precision */
  double G;           /* gravitational constant (outputs scale linearly) */
  int out_fp32;       /* 0: phi/accel outputs are double, 1: float */
  size_t mem_budget;  /* 0: unlimited; else fmm_set_levels fails with FMM_ERR_OOM when
                         the device workspace would exceed this many bytes */
  int bottom_mode;    /* fmm_bottom_mode */
  int p_m;            /* multipole order used by M2L and M2P, 1..p; 0 means p.  Eq. 3
                         sums n <= p - m over the multipoles that exist: with the
                         paper's quadrupoles and p = 3 (Sec. 2) that is p_m = 2, p = 3.
                         Terms with |alpha| > p_m are dropped from every translation. */
  int mass_fp32;      /* 0: masses passed to fmm_set_levels / fmm_update_masses are
                         double, 1: float (widened exactly to double on the device) */
  int fp64_top;       /* mixed precisions: 1 keeps FP64 for the M2M of box levels <= 3
                         and for the L2L chain and the accumulation of the local
                         expansions; 0 runs them in FP32 (the default: on B300 the
                         FP64 version costs ~20 % of a solve and, measured, gains no
                         accuracy against the FP64 path).  Ignored by FMM_FP64. */
  int delta_l;        /* levels between the cells and the finest FMM box: 1 (the
                         paper's choice for AMR and ATS; 0 also means 1) or 2 (the
                         generalisation of the footnote of Sec. 2, which Paper I
                         tested on unigrids): the finest box is a 4^3 block of cells,
                         the near field the cells of its 3^3 neighbour blocks (12^3
                         cells), the bottom intermediate field the M2P from its
                         interaction list and M2L stops one box level higher.  With 2,
                         fmm_set_levels takes one complete level only (lmin == lmax
                         >= 3; otherwise FMM_ERR_ARG) and the bottom mode must be
                         FMM_BOTTOM_M2P; fmm_solve_adjoint and the static unigrid
                         entry return FMM_ERR_ARG. */
  int periodic;       /* 0: isolated boundaries (the paper's); 1: periodic boundaries
                         (Sec. 6 names them as the next step): the box tiles space, a
                         uniform background of the opposite total mass is added (lap
                         phi = 4 pi G (rho - mean rho)), and phi is Ewald's periodic
                         potential (zero mean over the box; a cell's own images act on
                         it).  Every neighbour and interaction list wraps around the
                         box, M2L also runs at box level 1, and the images beyond the
                         root's 3^3 reach level 1 through a lattice tensor built on the
                         host.  Needs lmin >= 3 (fmm_set_levels returns FMM_ERR_ARG),
                         the graded rule across the box edges (FMM_ERR_NOT_GRADED),
                         bottom mode FMM_BOTTOM_M2P and delta_l 1; fmm_solve_adjoint,
                         fmm_direct_sum, fmm_set_drift and the static unigrid entry
                         return FMM_ERR_ARG. */
} fmm_config;

/* Device memory for the library, supplied by the caller (for instance a caching
 * allocator).  Called with ptr == NULL to allocate `bytes` (return the device
 * pointer, 256-byte aligned, or NULL when out of memory) and with ptr != NULL to
 * release an earlier allocation of `bytes` (the return value is ignored).
 * `stream` is the stream of the library call that needs the memory; the library
 * orders all its own work on that stream before it returns memory. */
typedef void* (*fmm_alloc_fn)(void* user, void* ptr, size_t bytes, void* stream);

/* Create a context on the current CUDA device.  The config is copied.  `alloc`
 * (with its `alloc_user` pointer) supplies every device allocation the context
 * makes (its workspace, and the translation tables it shares with the other
 * contexts of the same device, order, precision and allocator); NULL uses
 * cudaMalloc / cudaFree.  Returns FMM_ERR_ARG for p outside 1..8, p_m outside
 * 0..p, an unknown precision or bottom mode, delta_l outside 0..2 (2 with
 * bottom mode FMM_BOTTOM_M2L_L2P), or periodic outside 0..1 (1 with another
 * bottom mode or delta_l = 2). */
fmm_status fmm_create(const fmm_config* cfg, fmm_alloc_fn alloc, void* alloc_user, fmm_ctx** out);

/* Set the AMR hierarchy, or replace its levels lo..lmax (adaptive time
 * stepping: Alg. 1 rebuilds the trees of the active levels only).
 *
 *   n[k]    host int64, number of leaf cells of level lo+k, k = 0..lmax-lo
 *   ijk[k]  int32 [n[k]][3] cell indices of level lo+k, each in [0, 2^(lo+k))
 *   mass[k] [n[k]] masses, double (or float when config.mass_fp32)
 * ijk/mass may be device or host pointers (host data is copied in on
 * `stream`).  The caller keeps ownership; the library copies what it needs
 * before returning, so the buffers may be reused afterwards.  A call with
 * lo == lmin replaces the whole hierarchy (lmin and lmax may change); a call
 * with lo > lmin must keep lmin and lmax (FMM_ERR_STATE), and levels below lo
 * keep their previous cells and masses.  The first call must have lo == lmin.
 * The tree index of the whole hierarchy (Morton-sorted octs, parents,
 * children, 27-neighbour tables) is rebuilt and validated, as a CUDA graph
 * when graphs are on (fmm_set_graphs); this call synchronises `stream` once.
 * Requires 2 <= lmin <= lmax <= 20. */
fmm_status fmm_set_levels(fmm_ctx* ctx, int lmin, int lmax, int lo, const int64_t* n,
                          const int32_t* const* ijk, const void* const* mass, void* stream);

/* Replace the masses of levels lo..lmax of the current hierarchy, cells
 * unchanged (a time step that moves mass but not the mesh).  mass[k]: double
 * (float when config.mass_fp32) [n] for level lo+k in the order of the last fmm_set_levels of that level,
 * device or host pointer, copied on `stream` before the call returns (host
 * memory) or in stream order (device memory).  No tree rebuild and no
 * synchronisation; the next solve recomputes what depends on these levels.
 * The values are not validated (fmm_set_levels rejects non-finite masses). */
fmm_status fmm_update_masses(fmm_ctx* ctx, int lo, const void* const* mass, void* stream);

/* Multipole drifting of stale trees (Sec. 4 names it as future work, after
 * SWIFT).  In a solve from level lo > lmin the trees of levels j < lo are stale:
 * their multipoles hold the masses last given to those levels.  With drifting
 * on, every box of such a tree at box level >= 2 is moved by d = v dt[j], v the
 * centre-of-mass velocity of the tree's cells inside the box: its moments about
 * the box centre become those of the moved mass (the shift of Eq. 2).  Cells
 * used as point masses (P2P, P2L) stay at their centres.
 *
 * fmm_set_velocities: vel[k] double [n][3], velocity of each leaf of level lo+k
 * in the order of the last fmm_set_levels of that level, device or host
 * pointer, copied on `stream`.  fmm_set_levels of a level invalidates its
 * velocities; a drifting solve that needs them returns FMM_ERR_STATE.
 *
 * fmm_set_drift: dt[k], k = 0..n-1 with n = lmax - lmin + 1: the time elapsed
 * since level lmin+k was set (only levels below a solve's lo are drifted); NULL
 * turns drifting off.  A drifting solve recomputes every multipole from the
 * masses (a full upward pass) before it adds the drift; the first call after a
 * new hierarchy sizes the drift scratch (the solves then allocate nothing).
 * Periodic contexts (whose level-1 multipoles would need drifting too):
 * FMM_ERR_ARG. */
fmm_status fmm_set_velocities(fmm_ctx* ctx, int lo, const double* const* vel, void* stream);
fmm_status fmm_set_drift(fmm_ctx* ctx, const double* dt, int n);

/* Solve for the leaf cells of levels lo..lmax (Alg. 1 for l = lo..lmax, which
 * share one upward and one downward pass: the far field of a box does not
 * depend on the target level).  phi[k] / accel[k] receive level lo+k in the
 * caller's input order: phi [n][1], accel [n][3], double or float per
 * config.out_fp32.  Device or host pointers (host outputs are copied back on
 * `stream`; the caller synchronises before reading them).  Asynchronous. */
fmm_status fmm_solve(fmm_ctx* ctx, int lo, void* const* phi, void* const* accel, void* stream);

/* Solves many independent hierarchies (one context each, same device) in one
 * CUDA graph launch: the contexts' solves are branches of one graph, so small
 * hierarchies run side by side.  The paper has no counterpart (it solves one
 * hierarchy per MPI domain).
 *   ctxs[i]     distinct contexts with a hierarchy set
 *   lo[i]       first solved level of context i (as fmm_solve)
 *   phi[i][k], accel[i][k]  DEVICE outputs of level lo[i]+k of context i
 * The graph is captured on the first call for a given set of contexts,
 * layouts, levels and output pointers (a few are cached) and launched on
 * `stream`; later calls with the same arguments only launch it.
 * Asynchronous; errors as fmm_solve (FMM_ERR_ARG for host outputs). */
fmm_status fmm_batch_solve(fmm_ctx* const* ctxs, int nctx, const int* lo, void* const* const* phi,
                           void* const* const* accel, void* stream);

/* Autotuner: times the candidate launch shapes of the context's kernels on its
 * current hierarchy (solves of levels lo..lmax into scratch outputs) and keeps
 * the fastest: the split-K factor of the tcgen05 M2P and M2L contractions
 * (mixed precision) and the target octs per block of the near-field kernel.
 * Synchronises `stream`.  The choices stay with the context (also for later
 * hierarchies) and are read back with fmm_get_tuning: out3 = {split M2P,
 * split M2L (0 = built-in heuristic), near-field octs per block}.  The split
 * factors serve solves from the same lo only (a sub-cycle from a finer level
 * has much smaller contractions and keeps the built-in choice); the
 * octs-per-block choice serves every solve. */
fmm_status fmm_autotune(fmm_ctx* ctx, int lo, void* stream);
fmm_status fmm_get_tuning(const fmm_ctx* ctx, int* out3);
/* Sets the same three values (for instance one autotuned context's choices on
 * the other contexts of a batch); values set here serve solves from every
 * level.  Unsupported octs-per-block values fall back to the built-in choice. */
fmm_status fmm_set_tuning(fmm_ctx* ctx, const int* in3);

/* Adjoint of fmm_solve (not in the paper: the exact transpose of its linear
 * map from masses to outputs).  Given cotangents of the outputs of levels
 * lo..lmax, writes the gradient of <g_phi, phi> + <g_accel, accel> with
 * respect to the mass of every leaf of every level:
 *   g_phi[k], g_accel[k]  level lo+k, [n][1] and [n][3] in the caller's input
 *                         order, double or float per config.out_fp32
 *   g_mass[k]             level lmin+k (all levels: far fields couple them),
 *                         double [n]
 * Device or host pointers.  The transposed chain runs in reverse (P2P^T,
 * L2P^T, near-field M2P^T, M2P^T, M2L^T, L2L^T, M2M^T); the map is linear, so
 * no forward state is kept or recomputed.  Needs an FMM_FP64 context
 * (FMM_ERR_ARG otherwise).  The first call after fmm_set_levels builds the
 * lists of source octs and synchronises `stream` once; the first call of a
 * context builds the transposed operators (host work, about 130 MB of device
 * memory at p = 6).  Asynchronous otherwise. */
fmm_status fmm_solve_adjoint(fmm_ctx* ctx, int lo, const void* const* g_phi, const void* const* g_accel,
                             double* const* g_mass, void* stream);

/* Wait for all work of the context on its last stream and return any
 * latched device error (FMM_ERR_TIMEOUT from a bounded wait, FMM_ERR_CUDA).
 * After FMM_ERR_TIMEOUT the outputs of that solve are invalid; the context
 * clears its partial sums, and the next solve recomputes everything. */
fmm_status fmm_sync(fmm_ctx* ctx);

/* Every wait of a tensor-core contraction on one of its pipeline barriers gives
 * up after `seconds` of wall-clock time (default 2; 0 gives up at the first
 * wait that is not already complete, for tests).  A CTA that gives up latches
 * FMM_ERR_TIMEOUT (returned by fmm_sync), waits for its own copies and tensor
 * operations in flight, frees its tensor memory and exits.  FMM_ERR_ARG for a
 * negative or non-finite value. */
fmm_status fmm_set_wait_limit(fmm_ctx* ctx, double seconds);

/* Text of the last error of this context (static storage inside ctx). */
const char* fmm_last_error(const fmm_ctx* ctx);

void fmm_destroy(fmm_ctx* ctx);

/* Solve a complete unigrid of level 2..4 (n = 8^level cells, at most 16^3)
 * without allocating any device memory.  The paper has no counterpart to this
 * call; it exists for callers that cannot call cudaMalloc while they run, such
 * as host codes whose device memory is owned by another allocator (one that
 * reserves the whole GPU at start-up, say) or loops that must not allocate
 * after initialisation.
 *   ctx       an existing context (any precision, p <= 6); only its translation
 *             tables are used, its own hierarchy is left as it was
 *   ijk/mass  device pointers, int32 [n][3] and double [n], every cell of the
 *             grid exactly once, any order
 *   phi/accel device pointers, [n] and [n][3], double or float per
 *             ctx's out_fp32, written in the input order
 * All per-hierarchy scratch lives in one static device array of 2 MiB inside
 * the library (every GPU that loads the library holds it until the process
 * exits).  The first call on a device looks up that array's address; make it
 * before any stream capture on the device.  All calls share the array, so
 * calls that overlap on the GPU race.  The call synchronises `stream` once, to
 * report invalid cells.  Returns FMM_ERR_ARG (with fmm_last_error set) for a
 * level outside 2..4, n != 8^level or p > 6, and FMM_ERR_OUT_OF_BOX,
 * FMM_ERR_DUPLICATE or FMM_ERR_NONFINITE for invalid cells. */
fmm_status fmm_solve_unigrid_static(fmm_ctx* ctx, int level, int64_t n, const int32_t* ijk,
                                    const double* mass, void* phi, void* accel, void* stream);

/* The exact sum the FMM approximates (Sec. 2; the reference of the accuracy
 * checks of Sec. 4): phi and accel of selected leaf cells of `level` from every
 * leaf cell of the current hierarchy, G sum_{j != i} m_j g(x_i - x_j) and its
 * negative gradient, in FP64, O(n_sel x cells) work on the device.
 *   sel    DEVICE int64 [n_sel], indices into the level's cells in the order of
 *          the last fmm_set_levels of that level (an index outside gives NaN)
 *   phi    DEVICE double [n_sel];  accel  DEVICE double [n_sel][3]
 * Asynchronous on `stream`.  FMM_ERR_STATE before fmm_set_levels, FMM_ERR_ARG
 * for a level outside lmin..lmax, n_sel < 0 or non-device pointers. */
fmm_status fmm_direct_sum(fmm_ctx* ctx, int level, int64_t n_sel, const int64_t* sel, double* phi,
                          double* accel, void* stream);

/* ---- introspection (tests and tools) ---------------------------------- */

/* Number of octs per level l = 0..lmax (n_oct[0] = 0) of the current tree. */
fmm_status fmm_tree_counts(const fmm_ctx* ctx, int64_t* n_oct);

/* Copy the tree index of level l (1..lmax) to host buffers, in canonical
 * order: octs sorted by the Morton key of their parent cell (x in the lowest
 * bit of each triple), cell id = 8*oct + (x&1 | (y&1)<<1 | (z&1)<<2).
 *   oct_key  uint64 [n_oct]     Morton key of the parent cell (level l-1)
 *   status   int64  [8 n_oct]   refined: child oct id at l+1; leaf: -1 - input index
 *   nbr      int64  [27 n_oct]  oct whose parent is the parent's neighbour
 *            (dx,dy,dz) at index (dx+1)+3(dy+1)+9(dz+1); -2 - (cell id at l-1)
 *            if that neighbour is a leaf; -1 outside the unit box. */
fmm_status fmm_tree_export(const fmm_ctx* ctx, int level, uint64_t* oct_key, int64_t* status,
                           int64_t* nbr);

/* Host-only: integer numerators P_gamma(u) of d^gamma (1/r) = P_gamma(u) /
 * |u|^(2|gamma|+1) at an integer point u, for all |gamma| <= q (q <= 12), in
 * graded order (degree, then a descending, then b descending).  These build
 * the library's translation tables.  Needs no GPU. */
fmm_status fmm_host_numerators(int q, const int64_t* u, int64_t* out);

/* Host-only: the FP64 translation operators the library builds, for checks.
 * which = 0: bottom M2P   [256][26*8*nc]   (n = (f*8+t)*4+comp; k = (q*8+s)*nc+alpha)
 *         1: M2L          [8*nc][26*8*nc]  (n = b*nc+beta)
 *         2: near M2P     [343][nc][4]     (R = target - source in [-3,3]^3)
 *         3: L2P          [64][nc][4]      (position f*8+t inside the level l-2 box)
 *         4: M2M          [8][nc][nc]      (child c, output alpha, input gamma)
 *         5: L2L          [8][nc][nc]      (child c, output beta, input gamma)
 *         6: lattice tensor [ncoef(p)]     (T_gamma = d^gamma psi_far(0), periodic
 *                                           boundaries; psi_far = Ewald's potential of
 *                                           a unit mass with its background minus g over
 *                                           the 27 nearest images; physical units)
 *         7: level-1 lattice operator [8*nc][8*nc] (the level-1 local expansions
 *                                           from the level-1 multipoles through the root)
 *         8: Delta l = 2 M2P [2048][26*8*nc] (n = ((g*8+f)*8+t)*4+comp)
 *         9: Delta l = 2 near-field ring [256][26*64] (k = (q*8+s)*8+child)
 * Expansions are in box units (multipoles / h^|alpha|, locals * h^(|beta|+1));
 * comp 0 is phi, comps 1..3 are accel = -grad phi.  Returns FMM_ERR_ARG if
 * `n` (doubles) is too small.  Needs no GPU. */
fmm_status fmm_host_table(int p, int which, double* out, int64_t n);

/* Counters since fmm_create: out[0] = launches of this library's own kernels,
 * out[1] = calls into CUB primitives (radix sort, scan, select) during tree
 * builds, out[2] = fmm_solve calls, out[3] = fmm_set_levels calls. */
fmm_status fmm_stats(const fmm_ctx* ctx, int64_t* out4);

/* fmm_solve replays its device work as a CUDA graph (on by default): the
 * first solve for a given lo, output pointers and tree layout captures it on
 * a stream of the library's own, later ones launch it on `stream`.  A new
 * hierarchy with other list lengths, or a reallocated workspace, captures
 * again.  on = 0 launches every kernel directly.  With timing on (below) the
 * solve never uses a graph. */
fmm_status fmm_set_graphs(fmm_ctx* ctx, int on);

/* Per-stage device times (ms) of the last solve when timing is enabled with
 * fmm_set_timing(ctx, 1), 5 doubles: upward (P2M, M2M), downward (M2L, L2L),
 * m2p (the bottom M2P contraction; 0 in bottom mode 1), near-field M2P, near
 * field (P2P, nearest field, L2P, scatter).  With timing on the stages run one
 * after the other on one stream; otherwise the bottom M2P runs beside the
 * downward pass. */
fmm_status fmm_set_timing(fmm_ctx* ctx, int on);
fmm_status fmm_stage_times(const fmm_ctx* ctx, double* ms5);

#ifdef __cplusplus
}
#endif
#endif /* FMM_H */
