/*
 * decbpm.h -- C ABI of the B300 (sm_103a) DEC beam-propagation library.
 *
 * The library marches a complex transverse field psi along z on an
 * unstructured mesh, solving the normalized NLSE of Eq. 1
 *
 *     i dpsi/dz = -sum_n p_n lap^n psi - V psi - chi |psi|^2 psi
 *
 * discretized with discrete exterior calculus as in Eqs. 10-12: psi is a
 * primal 0-form (one value per vertex), the transverse Laplacian is
 * -*0^{-1} d0^T *1 d0 (Table I), *0 is the barycentric (diagonal) Hodge star
 * and *1 the Galerkin Hodge star of Eq. 9, whose stiffness d0^T *1 d0 equals
 * the cotangent-weight stiffness used here.  Higher-order diffraction terms
 * are powers of the same operator (Table I, "Higher-order" row).  Potential
 * and Kerr coefficients are per triangle, lumped to vertices with *0(V) and
 * *0(chi) (Sec. "Discrete Hodge star").
 *
 * One z-step of length h is the Strang split D_{h/2} E_h D_{h/2}:
 *   E_h  = exp(i h sum_n p_n (-A)^n), A = *0^{-1} d0^T *1 d0, applied by a
 *          Chebyshev expansion on an interval [0, rho] that contains the
 *          spectrum of A (rho: see DECBPM_BOUND_*);
 *   D_h  = exact flow of dpsi/dz = i (v + chib |psi|^2) psi - sigma psi per
 *          vertex (potential, Kerr phase and absorber damping).
 *
 * Conventions shared by every entry point
 *   - Return value: DECBPM_OK (0) or a negative DECBPM_ERR_* code.  The
 *     message of the last failure on the calling thread is returned by
 *     decbpm_last_error().  No entry point aborts, traps or exits.
 *   - Fields live on the device in the caller's vertex order, interleaved
 *     complex (re, im), field-minor: element (vertex p, field f) is at
 *     index p * n_fields + f.  complex64 for DECBPM_C64, complex128 for
 *     DECBPM_C128.  The caller owns these buffers; the library updates them
 *     in place.
 *   - Host arrays (mesh description, diagnostics) are read or written only
 *     during the call.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is
 *     enqueued on it; calls that return diagnostics or check device status
 *     synchronize that stream before returning.
 *   - A handle may be used by one thread at a time.
 */
#ifndef DECBPM_H
#define DECBPM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes -------------------------------------------------------- */
#define DECBPM_OK                 0
#define DECBPM_ERR_INVALID_ARG   -1   /* bad pointer, size, dz, precision ... */
#define DECBPM_ERR_BAD_MESH      -2   /* inverted / degenerate triangle, non-manifold edge, isolated vertex */
#define DECBPM_ERR_NONFINITE     -3   /* NaN or Inf in an input, or in the field after a step block */
#define DECBPM_ERR_TIMEOUT       -4   /* a device-side grid barrier gave up waiting (bounded spin) */
#define DECBPM_ERR_CUDA          -5   /* a CUDA runtime call failed */
#define DECBPM_ERR_OOM           -6   /* device or host allocation failed */
#define DECBPM_ERR_UNSUPPORTED   -7   /* valid request that this library does not implement */
#define DECBPM_ERR_DEVICE_CHECK  -8   /* a device-side consistency check failed; the kernel skipped the work */

/* ---- enumerations -------------------------------------------------------- */
#define DECBPM_C64   1   /* complex64 field, FP32 arithmetic, FP64 diagnostics */
#define DECBPM_C128  2   /* complex128 field, FP64 arithmetic */

#define DECBPM_KERR_LUMPED   0   /* N_p = chib_p |psi_p|^2 (per-vertex, "pointwise") */
#define DECBPM_KERR_ELEMENT  1   /* N_p = [*0^{-1} Q^T D Q |psi|^2]_p, triangle-averaged (Eq. 14) */

#define DECBPM_VARIANT_FUSED  0  /* persistent kernel, fused Chebyshev/Clenshaw terms and diagonal step */
#define DECBPM_VARIANT_PLAIN  1  /* unfused reference path: one CSR SpMV launch + one update launch per term */
#define DECBPM_VARIANT_ROWS   2  /* fused, operands read straight from global memory (never the tile-staged
                                    kernel that FUSED selects for complex64 plans with 9..16 fields) */
#define DECBPM_VARIANT_PAIRS  3  /* fused, two Clenshaw stages per grid-wide pass (stage-pair kernel, complex64
                                    plans with 9..16 fields whose tiles' depth-two halos fit its capacities; other
                                    plans run FUSED).  It stores a_k psi - b_{k+2} in place of b_{k+2}, so its
                                    fields differ from FUSED's at the level of FP32 rounding.  FUSED runs it once
                                    decbpm_plan_autotune has chosen it. */
#define DECBPM_VARIANT_FLOW   4  /* fused, the tile-staged kernel without grid barriers between Clenshaw stages
                                    (dataflow kernel): a tile waits only for the tiles adjacent to it in the
                                    operator graph to finish the previous stage (per-tile completion counters),
                                    so CTAs are not held in lockstep.  Same arithmetic per row as FUSED's
                                    tile-staged kernel (bitwise identical fields); complex64 plans with 9..16
                                    fields whose tiles have at most 31 such neighbours, other plans run FUSED.
                                    FUSED runs it once decbpm_plan_autotune has chosen it. */

#define DECBPM_ORDER_DEFAULT  0  /* Hilbert curve in 2D, coordinate order in 1D */
#define DECBPM_ORDER_RCM      1  /* reverse Cuthill-McKee (small bandwidth, thin level sets) */
#define DECBPM_ORDER_HILBERT  2  /* Hilbert space-filling curve of the vertex positions (compact blocks) */

/* The Chebyshev interval [0, rho] must contain the spectrum of A (outside it
 * the truncated series of exp(-i h A) grows like cosh(k acosh x)).
 * GERSHGORIN: rho = min(Gershgorin bound, element bound max_t lambda_max(K_t, M_t)), both
 *   deterministic upper bounds, times 1 + 1e-6 (DECBPM_RHO_RIGOROUS).
 * LANCZOS (default): theta = the largest Ritz value of lanczos_steps (default 200) Lanczos
 *   steps on *0^{-1/2} K *0^{-1/2} from a fixed pseudo-random start; theta <= lambda_max
 *   and is typically within a fraction of a percent of it on these meshes, 1.6x tighter
 *   than Gershgorin on graded meshes (the Chebyshev degree, hence the work per step,
 *   shrinks nearly in proportion).  The candidate 1.01 theta is then checked for each
 *   mesh: a degree-128 Chebyshev polynomial of the operator on [0, 1.01 theta / 1.002],
 *   applied in FP64 to a seeded probe vector (pseudo-random plus spikes at the vertices
 *   with the largest Gershgorin rows), must not raise the probe's norm; an eigenvalue
 *   above the candidate would raise it by cosh(128 acosh x).  If it passes, rho =
 *   1.01 theta (DECBPM_RHO_LANCZOS_CHECKED); otherwise rho falls back to the rigorous
 *   bound (DECBPM_RHO_LANCZOS_REJECTED).  The check shows the bound for every
 *   eigenvector whose component in the probe is at least 1e-3 of its norm; it is no
 *   proof for an eigenvector orthogonal to the probe, and no probability is claimed. */
#define DECBPM_BOUND_DEFAULT     0
#define DECBPM_BOUND_LANCZOS     1
#define DECBPM_BOUND_GERSHGORIN  2

/* which bound rho is (decbpm_mesh_info_t.rho_kind) */
#define DECBPM_RHO_RIGOROUS          0   /* min(Gershgorin, element bound) (DECBPM_BOUND_GERSHGORIN, or
                                            Lanczos not tighter) */
#define DECBPM_RHO_LANCZOS_CHECKED   1   /* 1.01 x the Lanczos Ritz value, passed the per-mesh check */
#define DECBPM_RHO_LANCZOS_REJECTED  2   /* the Lanczos candidate failed the check: the rigorous bound */

typedef struct decbpm_mesh_s *decbpm_mesh_t;
typedef struct decbpm_plan_s *decbpm_plan_t;

/* ---- mesh description (host memory, read during decbpm_mesh_create) ---------
 * dim 2: cells are triangles [v1, v2, v3], counter-clockwise (positive signed
 *        area), as the paper assumes for 2-simplices; dim 1: segments [a, b].
 * V_cell / chi_cell: potential and Kerr coefficient per cell, evaluated at the
 *        cell centroid (NULL = 0 and 1).  sigma_vertex: absorber rate >= 0
 *        per vertex (NULL = none).  p_n: diffraction coefficients p_1..p_np of
 *        Eq. 1 (NULL or n_p = 0 means p_1 = 1). */
typedef struct {
    int32_t dim;
    int64_t n_vertices;
    int64_t n_cells;
    const double  *coords;        /* [n_vertices * dim] */
    const int32_t *cells;         /* [n_cells * (dim + 1)] */
    const double  *V_cell;        /* [n_cells] or NULL */
    const double  *chi_cell;      /* [n_cells] or NULL */
    const double  *sigma_vertex;  /* [n_vertices] or NULL */
    const double  *p_n;           /* [n_p] or NULL */
    int32_t        n_p;
    int32_t        ordering;      /* internal vertex order: DECBPM_ORDER_DEFAULT / _RCM / _HILBERT */
    int32_t        spectral_bound;/* rho of the Chebyshev interval: DECBPM_BOUND_DEFAULT / _LANCZOS / _GERSHGORIN */
    int32_t        lanczos_steps; /* Lanczos steps of the LANCZOS bound (0 = 200; fewer: faster set-up,
                                     a looser candidate that the per-mesh check may reject) */
} decbpm_mesh_desc;

typedef struct {
    int64_t n_vertices, n_edges, n_cells;
    int64_t nnz_offdiag;       /* off-diagonal entries of the stiffness K (2 per edge) */
    int32_t max_degree;        /* largest vertex degree */
    int32_t n_p;               /* number of diffraction coefficients */
    int64_t bandwidth;         /* max |new(p) - new(q)| over edges in the internal order */
    double  rho;               /* upper end of the Chebyshev interval of A = *0^{-1} K (see DECBPM_BOUND_*) */
    double  area;              /* sum of cell measures = sum of *0 */
    double  mean_degree;       /* nnz_offdiag / n_vertices */
    int64_t sell_entries;      /* padded off-diagonal entries stored (SELL-32) */
    int64_t device_bytes;      /* device memory held by the handle (operators, no workspaces) */
    int32_t rho_kind;          /* DECBPM_RHO_*: which bound rho is */
    int32_t pad_;
    double  rho_lanczos;       /* largest Lanczos Ritz value theta (0 if not run) */
    double  rho_rigorous;      /* (1 + 1e-6) min(Gershgorin bound, element bound) */
} decbpm_mesh_info_t;

/* ---- propagation parameters ---------------------------------------------- */
typedef struct {
    double  dz;          /* step length h > 0 */
    int64_t n_steps;     /* >= 0 */
    int32_t precision;   /* DECBPM_C64 | DECBPM_C128: element type of the field buffers */
    int32_t kerr_mode;   /* DECBPM_KERR_LUMPED | DECBPM_KERR_ELEMENT */
    int32_t diag_every;  /* > 0: diagnostics after every diag_every steps; 0: only after the last step */
    int32_t variant;     /* DECBPM_VARIANT_FUSED | _ROWS | _PAIRS | _FLOW | _PLAIN (C128, one mesh, one
                            field); decbpm_vjp and decbpm_propagate_noalloc take FUSED */
    double  cheb_tol;    /* Chebyshev truncation: tail bound; 0 = 1e-16 (C128) / 1e-9 (C64) */
} decbpm_params;

/* Diagnostics of one field at one z (FP64 accumulation, fixed reduction order):
 *   power       P = sum_p m_p |psi_p|^2                    (m = *0)
 *   hamiltonian H = psi^H *0 L_diff psi - sum_p m_p v_p |psi_p|^2 - 1/2 sum_p m_p chib_p |psi_p|^4
 *               (conserved by the lumped system without absorber; NaN when n_p > 2)
 *   max_intensity = max_p |psi_p|^2                                             */
typedef struct { double z, power, hamiltonian, max_intensity; } decbpm_diag;

/* ---- library ------------------------------------------------------------- */
/* Library name and target; the bounds-check build (-DDECBPM_BOUNDS_CHECK,
   libdecbpm_checked.so) says "bounds-checked": its march kernels test every
   gather index against its buffer and report DECBPM_ERR_DEVICE_CHECK. */
const char *decbpm_version(void);
/* Message of the last failed call on this thread ("" if none).  Owned by the library. */
const char *decbpm_last_error(void);

/* ---- mesh ---------------------------------------------------------------- *
 * Assembles the DEC operators in FP64 on the host (Sec. "DEC computational
 * framework" through Eq. 12): canonical edges (a < b), the cotangent form of
 * d0^T *1 d0 (equal to the Galerkin *1 of Eq. 9 with xi = 1), *0, *0(V),
 * *0(chi), the spectral bound rho of A; renumbers vertices (Hilbert curve or
 * reverse Cuthill-McKee), packs the operator as SELL-32 and uploads it (FP64 and FP32
 * copies) to the current CUDA device.  The handle owns that device memory.
 * Errors: INVALID_ARG (NULL/size), BAD_MESH, NONFINITE, CUDA, OOM.          */
int decbpm_mesh_create(const decbpm_mesh_desc *desc, decbpm_mesh_t *out);
int decbpm_mesh_destroy(decbpm_mesh_t mesh);
int decbpm_mesh_info(decbpm_mesh_t mesh, decbpm_mesh_info_t *info);

/* Host-only assembly (no device needed), for inspection and testing.
 * First call with every output NULL to fill *info (sizes); then call again
 * with outputs of those sizes (any output may stay NULL):
 *   m, v, chib   [n_vertices]            *0, lumped potential, lumped Kerr coefficient (caller order)
 *   K_rowptr     [n_vertices + 1]        stiffness K = d0^T *1 d0 in CSR, caller order,
 *   K_col, K_val [nnz_offdiag + n_vertices]   diagonal included, columns ascending
 *   perm         [n_vertices]            internal order: perm[new] = caller index
 * The internal order is reverse Cuthill-McKee or a Hilbert curve (desc->ordering).           */
int decbpm_assemble_host(const decbpm_mesh_desc *desc, decbpm_mesh_info_t *info,
                         double *m, double *v, double *chib,
                         int64_t *K_rowptr, int32_t *K_col, double *K_val, int32_t *perm);

/* Host-only: Chebyshev coefficients used for E_h.  For p = (p_1) the
 * expansion is exp(-i a x) = sum_k (2 - delta_k0) (-i)^k J_k(a) T_k(x)
 * (Jacobi-Anger), so this returns J_0(a) .. J_{n-1}(a) by Miller's backward
 * recurrence, n = smallest degree + 1 whose tail 2 sum_{k>=n} |J_k(a)| <= tol.
 * J_out has room for max_terms values; *n_out receives n (or the needed size
 * with INVALID_ARG if max_terms is too small).                               */
int decbpm_bessel_coefficients(double a, double tol, int32_t max_terms, double *J_out, int32_t *n_out);

/* ---- propagation (single mesh) --------------------------------------------
 * Advances n_fields independent fields psi_dev[n_vertices * n_fields] by
 * params->n_steps Strang steps.  diag_out (host, may be NULL) receives
 * n_fields records per diagnostic point, field-minor:
 *   n_diag = n_steps / diag_every (+1 if n_steps % diag_every != 0), or 1 if diag_every == 0.
 * Workspaces (internal-order field copy, three Clenshaw buffers, barrier
 * words) are allocated on first use and cached in the handle.
 * On a mesh with a PML (decbpm_mesh_set_pml) the march runs on the
 * stretched operators, complex64 or complex128, lumped Kerr, p_1 only.
 * Errors: INVALID_ARG, NONFINITE (field became non-finite), TIMEOUT, CUDA, OOM,
 * UNSUPPORTED (n_fields > 64, the PLAIN variant with C64 or several fields
 * on a mesh without a layer, element Kerr or p_2.. with a layer).          */
int decbpm_propagate(decbpm_mesh_t mesh, const decbpm_params *params, void *psi_dev, int64_t n_fields,
                     void *stream, decbpm_diag *diag_out);

/* Same with host buffers: copies psi_host (pinned or pageable) to the device,
 * propagates, copies the result back into psi_host.                          */
int decbpm_propagate_host(decbpm_mesh_t mesh, const decbpm_params *params, void *psi_host, int64_t n_fields,
                          void *stream, decbpm_diag *diag_out);

/* Diagnostics of fields already on the device (caller order). diag_out: n_fields records. */
int decbpm_diagnostics(decbpm_mesh_t mesh, const void *psi_dev, int64_t n_fields, int32_t precision,
                       void *stream, decbpm_diag *diag_out);

/* ---- batched propagation: many meshes x many fields, one persistent launch ----
 * A plan binds n_meshes mesh handles, each carrying fields_per_mesh[i] fields
 * (all <= 64), at one precision.  It owns the workspaces and a CUDA graph per
 * step block.  All meshes advance the same n_steps with the same dz; each
 * mesh uses its own Chebyshev degree.  In complex64 a mesh with more than 16
 * fields runs as field groups of at most 16 (decbpm_plan_config.field_groups;
 * so do decbpm_propagate, decbpm_propagate_host and decbpm_propagate_batch):
 * the same stages on each group, the caller's layout unchanged.             */
int decbpm_plan_create(const decbpm_mesh_t *meshes, int32_t n_meshes, const int32_t *fields_per_mesh,
                       int32_t precision, decbpm_plan_t *out);
int decbpm_plan_destroy(decbpm_plan_t plan);
/* psi_dev[i] is mesh i's field buffer [n_vertices_i * fields_per_mesh_i].
 * diag_out (host, may be NULL): for each diagnostic point, for each mesh, its
 * fields' records (sum_i fields_per_mesh_i records per point).              */
int decbpm_plan_propagate(decbpm_plan_t plan, const decbpm_params *params, void *const *psi_dev,
                          void *stream, decbpm_diag *diag_out);
/* Host-buffer version of decbpm_plan_propagate (copies in, propagates, copies out). */
int decbpm_plan_propagate_host(decbpm_plan_t plan, const decbpm_params *params, void *const *psi_host,
                               void *stream, decbpm_diag *diag_out);
/* Plan information: Chebyshev degree used by mesh i for step dz (0 if i is out of range). */
int32_t decbpm_plan_degree(decbpm_plan_t plan, int32_t mesh_index, double dz, int32_t precision, double cheb_tol);

/* Launch configuration of a plan. */
typedef struct {
    int32_t grid;          /* CTAs of the persistent cooperative launch (all co-resident) */
    int32_t block;         /* threads per CTA */
    int32_t fields_padded; /* fields per vertex in the internal layout (power of two >= max fields of an
                              entry, see field_groups) */
    int32_t graphs;        /* 1 if step blocks are replayed from captured CUDA graphs */
    int32_t stages;        /* grid-wide stages per step for the last configured dz (max degree) */
    int32_t n_meshes;
    int32_t tile_slots;    /* > 0: the FUSED variant runs a tile-staged kernel with this many shared-memory
                              slots (complex64 with 9..16 fields, or one field per mesh); 0: the row kernel */
    int32_t tile_slot_bytes;
    int32_t tile_grid;     /* CTAs of the tile-staged launch */
    int32_t tile_block;    /* threads per CTA of the tile-staged launch (16 compute + 3 copy warps) */
    int32_t tuned;         /* 1 once decbpm_plan_autotune chose the launch shapes below */
    int32_t fused_kernel;  /* FUSED runs: 3 the dataflow kernel, 2 the stage-pair kernel, 1 the tile-staged
                              kernel, 0 the row kernel */
    int32_t tile_slots_used; /* ring slots the tile-staged kernel uses */
    int32_t forward_walk;  /* 1: odd stages do not walk backwards */
    int32_t pair_slots;    /* > 0: the plan can run the stage-pair kernel with this many ring slots */
    int32_t pair_slot_bytes;
    int32_t pair_grid;     /* CTAs of the stage-pair launch */
    int32_t passes;        /* grid-wide passes per step of the stage-pair kernel (last configured dz) */
    int32_t values_per_thread; /* row kernel: complex values per thread (a row is fields_padded / this lanes) */
    int32_t rows_per_item; /* row kernel: vertex rows per warp work item */
    int32_t flow_grid;     /* > 0: the plan can run the dataflow kernel with this many CTAs (one more warp
                              than the tile-staged kernel's: a publisher of tile completions) */
    int32_t flow_skip;     /* dataflow kernel: a reversed walk starts this many tiles before the previous
                              walk's end */
    int32_t flow_ranges;   /* dataflow kernel: 1 = the tile-staged kernel's contiguous ranges of the active
                              tiles per CTA, 0 = fixed per-CTA chunks of every mesh */
    int32_t tile_rows;     /* rows per tile of the tile-staged kernel: 128 (16 fields, march_tile_kernel),
                              512 (one field, march_tile1_kernel), 0: none */
    int32_t meta_items;    /* row kernel, single-mesh plans: warp items per CTA whose operator metadata
                              (columns, weights, slice widths) a launch caches in shared memory once, so
                              that no stage reads it from L2 again; 0: not cached (several meshes, the
                              cache switched off, or it does not fit with the launch's CTAs per SM) */
    int32_t field_groups;  /* plan entries the march runs: n_meshes, or more when a complex64 plan has more
                              than 16 fields on a mesh and runs it as field groups of at most 16 fields
                              (balanced sizes, consecutive, sharing the mesh's operator) so that every entry
                              fits the tile-staged kernels; the caller's layout and records are unchanged */
} decbpm_plan_config;
int decbpm_plan_get_config(decbpm_plan_t plan, decbpm_plan_config *cfg);

/* Autotuner of the FUSED variant's launch shapes (no counterpart in the paper:
 * the kernels' own tuning).  Times short trial marches of `trial_steps` steps
 * (1..1000) at step dz on the plan's internal buffers, for every candidate:
 * the stage-pair kernel with 3 or 2 ring slots, the tile-staged kernel
 * with 3 or 2 ring slots and the dataflow kernel with walk skips 4, 8 and 16
 * (per-CTA chunks) or 8 (contiguous ranges)
 * (complex64 plans with 9..16 fields), the row kernel
 * with 1..max co-resident CTAs per SM and (complex64 plans with 4+ fields) 4 or
 * 2 complex values per thread, each with and without the reverse walk
 * of odd stages; keeps the fastest for this plan and caches it for the
 * process (key: the meshes' content, field counts, precision, dz, kerr_mode),
 * so another plan of the same problem takes it without timing
 * (out->from_cache = 1).  The single-stage candidates do the same arithmetic
 * per row (bitwise identical fields); the stage-pair kernel differs from them
 * at the level of FP32 rounding (see DECBPM_VARIANT_PAIRS).  Synchronous; the
 * plan's internal buffers are overwritten (they hold nothing between calls). */
typedef struct {
    int32_t variant;       /* DECBPM_VARIANT_PAIRS: the stage-pair kernel; DECBPM_VARIANT_FUSED: the tile-staged
                              kernel; DECBPM_VARIANT_FLOW: the dataflow kernel; DECBPM_VARIANT_ROWS: the row
                              kernel */
    int32_t ctas_per_sm;   /* row kernel: co-resident CTAs per SM (tile kernel: 1) */
    int32_t tile_slots;    /* tile kernel: ring slots (0 for the row kernel) */
    int32_t forward_walk;  /* 1: odd stages walk forwards */
    double  ms_per_step;   /* best trial time per step */
    int32_t candidates;    /* configurations timed (0 when taken from the cache) */
    int32_t from_cache;
    int32_t values_per_thread; /* row kernel: complex values per thread (complex64 plans of 4+ fields: 4 or 2;
                                  so rows per warp item = 32 x this / padded fields); others: the default */
    int32_t walk_skip;     /* dataflow kernel: see decbpm_plan_config.flow_skip (0: the default, 8) */
    int32_t no_meta_cache; /* row kernel: 1 reads the operator metadata every stage (see
                              decbpm_plan_config.meta_items); 0: cached where it fits */
    int32_t flow_ranges;   /* dataflow kernel: see decbpm_plan_config.flow_ranges */
} decbpm_tune_result;
int decbpm_plan_autotune(decbpm_plan_t plan, double dz, int32_t kerr_mode, int32_t trial_steps, void *stream,
                         decbpm_tune_result *out);
/* Apply a launch shape without timing (for example one that decbpm_plan_autotune
 * returned in an earlier process): variant (PAIRS, FUSED = tile-staged, FLOW,
 * ROWS), ctas_per_sm, values_per_thread and no_meta_cache (ROWS), tile_slots
 * (PAIRS, FUSED, FLOW), walk_skip and flow_ranges (FLOW), forward_walk; ms_per_step,
 * candidates and from_cache are ignored.  Shapes the
 * plan cannot run return DECBPM_ERR_UNSUPPORTED or DECBPM_ERR_INVALID_ARG. */
int decbpm_plan_set_shape(decbpm_plan_t plan, const decbpm_tune_result *shape);

/* Device time in ms, from CUDA events recorded on the launch stream, from the
 * start of the first march-kernel launch to the end of the last one in the
 * most recent decbpm_plan_propagate call (one launch when diag_every = 0). */
int decbpm_plan_last_march_ms(decbpm_plan_t plan, double *ms);

/* ---- potential and adjoint --------------------------------------------------
 * Replace the per-vertex potential v_p used by the diagonal flow (host array
 * in caller order; NULL restores the lumped *0^{-1} *0(V) 1 of the mesh).  A
 * per-vertex refractive-index perturbation enters as dv_p = (k0 L)^2 d(n^2)_p. */
int decbpm_mesh_set_potential(decbpm_mesh_t mesh, const double *v_vertex);

/* Device-side potential offset: v_p = base_p + dv_dev[p] for every vertex, where
 * base is the mesh's lumped *0^{-1} *0(V) 1 or the last array given to
 * decbpm_mesh_set_potential, and dv_dev is an FP64 device array [n_vertices]
 * in caller order (NULL: v = base).  Enqueued on `stream` (one kernel; no host
 * copy, no synchronization), so it orders with the propagations on that stream;
 * it changes the mesh for every later call.  A per-vertex refractive-index
 * perturbation enters as dv_p = (k0 L)^2 ((n_p)^2 - n_ref^2) in the
 * normalisation of Eq. 1, so dJ/dn_p = 2 (k0 L)^2 n_p dJ/dv_p.             */
int decbpm_mesh_set_potential_offset(decbpm_mesh_t mesh, const double *dv_dev, void *stream);

/* Vector-Jacobian product of the whole march psi_N = (D_{h/2} E_h D_{h/2})^N psi_0
 * (lumped Kerr, fused variant) for n_fields fields on one mesh:
 *   gN_dev         [n_vertices * n_fields] Euclidean cotangent of psi_N (dJ = Re sum conj(gN) dpsi_N),
 *   grad_psi0_dev  out: dJ/dpsi_0 in the same convention (the gradient torch uses for complex inputs),
 *   grad_v_dev     out (may be NULL): FP64 [n_vertices] dJ/dv_p for the per-vertex potential,
 *   psiN_dev       out (may be NULL): the forward result.
 * The E-step adjoint in the *0 inner product is E_{-h} (same Chebyshev kernel,
 * conjugate coefficients); the diagonal-flow adjoint is its real-pair
 * linearization.  Memory: checkpoints every checkpoint_every steps (0 =
 * ceil(sqrt(n_steps))) plus one segment of states are kept on the device.     */
int decbpm_vjp(decbpm_mesh_t mesh, const decbpm_params *params, const void *psi0_dev, const void *gN_dev,
               void *psiN_dev, void *grad_psi0_dev, double *grad_v_dev, int64_t n_fields, int32_t checkpoint_every,
               void *stream);

/* Gradient of the overlap objective of a march (the inverse-design use the
 * paper's Conclusion names as a motivation): for each field f,
 *   J_f = |<phi_f, psi_N,f>_{*0}|^2 = |sum_p m_p conj(phi_p,f) psi_N,p,f|^2,
 * psi_N = (D_{h/2} E_h D_{h/2})^N psi_0 (lumped Kerr, fused variant).  The
 * overlap is formed on the device from the forward result in FP64 (fixed-order
 * reduction), its cotangent 2 c_f m phi_f starts the same checkpointed backward
 * march as decbpm_vjp.
 *   psi0_dev, target_dev  [n_vertices * n_fields], caller order, field-minor, the
 *                         element type of params->precision (phi_f = target)
 *   J_out                 host [n_fields]: J_f
 *   grad_v_dev            out (may be NULL): FP64 [n_vertices] d(sum_f J_f)/dv_p
 *   grad_psi0_dev         out (may be NULL): dJ_f/dpsi_0,f (dJ = Re sum conj(g) dpsi)
 * Synchronous.  Errors: INVALID_ARG, UNSUPPORTED (element Kerr, PLAIN/ROWS
 * variant, a PML), NONFINITE, TIMEOUT, CUDA, OOM.                           */
int decbpm_adjoint(decbpm_mesh_t mesh, const decbpm_params *params, const void *psi0_dev, const void *target_dev,
                   int64_t n_fields, double *J_out, double *grad_v_dev, void *grad_psi0_dev, int32_t checkpoint_every,
                   void *stream);

/* ---- the paper's integrator ---------------------------------------------------
 * Adaptive Dormand-Prince 5(4) (the "RK45" the paper runs through scipy) on
 * the full DEC ODE of Eq. 10, dPsi/dz = -i (L Psi + N(|psi|^2) Psi), with the
 * potential inside L as in Eq. 11 (sign per Eq. 1) and the absorber as
 * -sigma psi; FP64, one complex128 field in caller order on the device,
 * integrated in place from z = 0 to z_end.  Step control: accept when the
 * RMS of err / (atol + rtol max(|y|, |y_new|)) over real and imaginary parts
 * is <= 1; next step h min(10, 0.9 E^-1/5) (no growth right after a
 * rejection), or h max(0.2, 0.9 E^-1/5) after a rejection; h0 = 0 chooses
 * the first step automatically.  p_n with n <= 2.                          */
typedef struct { double rtol, atol, h0; int64_t max_steps; } decbpm_rk45_opts;
typedef struct { int64_t n_accepted, n_rejected, n_rhs; double h_last, z; } decbpm_rk45_stats;
int decbpm_rk45(decbpm_mesh_t mesh, double z_end, int32_t kerr_mode, const decbpm_rk45_opts *opts, void *psi_dev,
                void *stream, decbpm_rk45_stats *stats);

/* ---- discrete soliton --------------------------------------------------------
 * The fundamental nonlinear mode used as the launch field of the paper's
 * soliton case (computed there by a self-consistent eigenmode solver on the
 * same mesh, Supp. Note 4): a field phi with  H(phi) phi = mu phi,
 * H(phi) = p1 A - diag(v + N(|phi|^2))  (the generator of Eq. 10, sign per
 * Eq. 1), and power sum_p m_p |phi_p|^2 = power; then psi(z) = phi e^{-i mu z}
 * solves Eq. 10.  Method: imaginary-z iteration with the nonlinearity frozen
 * per iteration, phi <- e^{-tau H(phi)} phi renormalised (FP64 Chebyshev
 * series of the exponential; its fixed points are exactly the self-consistent
 * eigenmodes), until || H phi - mu phi ||_*0 / || phi ||_*0 < tol.  psi_dev is
 * one complex128 field [N0] in caller order: the start on input (e.g. a
 * Gaussian on the core), the mode on output.  p_1 > 0 only.               */
typedef struct {
    double power;        /* sum_p m_p |phi_p|^2 > 0 */
    double tau;          /* imaginary-z step of one iteration > 0 (e.g. 0.5) */
    double tol;          /* stop when the relative residual is below tol */
    double mix;          /* (0, 1]: the frozen potential uses I <- mix |phi|^2 + (1 - mix) I */
    int64_t max_iter;    /* >= 1 */
    int32_t kerr_mode;   /* DECBPM_KERR_LUMPED | DECBPM_KERR_ELEMENT */
} decbpm_soliton_opts;
typedef struct { double mu, residual; int64_t iterations, cheb_terms; } decbpm_soliton_stats;
int decbpm_soliton(decbpm_mesh_t mesh, const decbpm_soliton_opts *opts, void *psi_dev, void *stream,
                   decbpm_soliton_stats *stats);

/* Host only: e^{-a} I_k(a), k = 0..n-1, with every later term < tol e^{-a} I_0(a)
 * (the coefficients of the Chebyshev series of e^{-a x}); *n_out = n; out may
 * be NULL to query n; at most n_max values are written. */
int decbpm_bessel_i_scaled(double a, double tol, int32_t n_max, double *out, int32_t *n_out);

/* ---- perfectly matched layer ---------------------------------------------------
 * Absorbing layer by complex stretching of the discrete Hodge stars, the
 * extension the paper proposes in its Conclusion (exterior complex scaling):
 * about (x0, y0), beyond r_inner the radius continues into the complex plane,
 * r~ = r + i int sigma dr, sigma = sigma_max ((r - r_inner)/(r_outer - r_inner))^order
 * (order 0: constant sigma_max beyond r_inner).  Per triangle the Whitney
 * inner product of *1 (Eq. 9) takes the tensor (r~/(s r)) e_r e_r^T +
 * (s r/r~) e_t e_t^T, s = 1 + i sigma, and *0 the factor s r~ / r; v and chib
 * keep their lumped definitions with the stretched *0.  FP64, assembled on the
 * host (the split-step's weights a_pq / r are also kept in FP32, with FP32
 * copies of v and chib).  Once set, the mesh runs with decbpm_rk45 (lumped
 * Kerr) and with decbpm_propagate for any number of fields (1..64, layout
 * as without a layer), complex64 or complex128, lumped Kerr and p_1 only:
 * the Strang split-step on the stretched operators, E_h by the Chebyshev
 * series of exp(-i a x) evaluated on the complex spectrum (degree from the
 * Bernstein ellipse of the Gershgorin box of A~), D_h the exact flow with
 * the complex v and chib (their imaginary parts damp the intensity by a
 * Bernoulli equation).  One persistent launch per step block where one
 * thread per (vertex, field) element fits the grid (up to about 220k
 * elements on 148 SMs), else one launch per Chebyshev term and per flow
 * (params->variant = DECBPM_VARIANT_PLAIN forces the latter); complex64
 * rounds the last stage of each step once (double-float FP32 sums).
 * decbpm_propagate_host runs the same march from host buffers.  Every other
 * split-step entry point (plans, batches over meshes, the adjoint, the
 * soliton solver, the allocation-free call) returns DECBPM_ERR_UNSUPPORTED.  pml = NULL or sigma_max = 0
 * removes the layer.  2D meshes only. */
typedef struct { double x0, y0, r_inner, r_outer, sigma_max; int32_t order; } decbpm_pml;
int decbpm_mesh_set_pml(decbpm_mesh_t mesh, const decbpm_pml *pml);
/* Chebyshev degree M of the split-step on the stretched operators for step
 * dz at precision's default tolerance (or cheb_tol > 0): M grid-wide stages
 * per step.  Host only; 0 if the mesh has no layer or an argument is bad. */
int32_t decbpm_mesh_pml_degree(decbpm_mesh_t mesh, double dz, int32_t precision, double cheb_tol);

/* One-shot convenience: plan_create + plan_propagate + plan_destroy. */
int decbpm_propagate_batch(const decbpm_mesh_t *meshes, int32_t n_meshes, const int32_t *fields_per_mesh,
                           const decbpm_params *params, void *const *psi_dev, void *stream,
                           decbpm_diag *diag_out);

/* ---- allocation-free propagation -------------------------------------------
 * No counterpart in the paper: a service for callers that cannot allocate
 * device memory at the moment they propagate -- for example code running while
 * another allocator (a framework's caching allocator) owns the whole memory
 * budget, or a loop that must keep a fixed memory footprint.  Same march as
 * decbpm_propagate on one mesh (fused row kernel, either precision and Kerr
 * mode, bit for bit the same field), but the scratch (internal-order field
 * copy, three Clenshaw buffers, stage tables, barrier/status words) lives in
 * one static 32 MiB device array of the library instead of allocated
 * workspaces; this call makes no cudaMalloc, cudaFree or pinned-memory
 * allocation.  The scratch needed is about 4 * n_vertices * padded_fields *
 * (8 bytes for C64, 16 for C128) plus 64 KiB; larger requests fail with
 * DECBPM_ERR_INVALID_ARG and a message giving the sizes.  The mesh handle
 * (created beforehand with decbpm_mesh_create, on the device that is current
 * at this call, else DECBPM_ERR_INVALID_ARG) and psi_dev are the caller's.
 * No diagnostics are returned.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress, with that device current) and
 * keeps it for the process.  A cudaDeviceReset drops the module, so the kept address is stale after it:
 * do not call this entry point after resetting the device.  All calls share
 * the one array, which keeps the last call's contents (the call clears what
 * must start at zero), so calls that can overlap on the GPU (on different
 * streams or from different host threads of one process) race on it:
 * serialize them.  Each process has its own copy.  The call synchronizes
 * `stream` before returning.                                                 */
int decbpm_propagate_noalloc(decbpm_mesh_t mesh, const decbpm_params *params, void *psi_dev, int64_t n_fields,
                             void *stream);

/* ---- failure-path self test ------------------------------------------------
 * Launches a small cooperative kernel whose CTAs meet at the same bounded
 * grid barrier the march kernel uses, but wait for `missing_arrivals` more
 * arrivals than the grid provides, giving up after timeout_ns.  Returns
 * DECBPM_ERR_TIMEOUT when missing_arrivals > 0 (the wait runs out, the kernel
 * exits normally and the context stays usable) and DECBPM_OK when it is 0.   */
int decbpm_selftest_barrier(int32_t missing_arrivals, int64_t timeout_ns, void *stream);

/* Index-check self test: one tiny kernel passes an out-of-range index (n for
 * an n-element buffer) through the march kernels' gather-index check and
 * writes back what the check returned; the index is not used to access
 * memory.  The bounds-check build (libdecbpm_checked.so) returns
 * DECBPM_ERR_DEVICE_CHECK (the check fired and replaced the index by 0), the
 * default build DECBPM_OK (no check compiled in).                            */
int decbpm_selftest_bounds_check(void *stream);

#ifdef __cplusplus
}
#endif

#endif /* DECBPM_H */
