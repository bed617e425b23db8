/*
 * alphac: alpha complexes of weighted points (atoms) on one GB300 GPU.
 *
 * The method is the Delaunay-free construction of Masood, Ray and Natarajan,
 * "Parallel Computation of Alpha Complexes for Biomolecules" (arXiv 1908.05944):
 * an estimation pass builds, bottom-up, every edge, triangle and tetrahedron
 * whose OrthoSize is at most alpha (Section 4.3, Step 1 of Section 3.1), and a
 * pruning pass keeps those whose orthocentre passes the empty-orthosphere test
 * AC2, inserting the faces of kept simplices directly (Section 4.4, Steps 2-5).
 *
 * Conventions
 *   - Lengths in angstrom, alpha in angstrom^2. Centres and radii are quantised
 *     to 1/1024 A and alpha to 2^-20 A^2, each rounded half to even. Every
 *     predicate is decided exactly on these integers.
 *   - Ties (the paper's "symbolic perturbation", Section 2) are broken by
 *     perturbing the squared radii, W_k + eps_k, with eps_k decreasing steeply
 *     in the INPUT index k. The alpha bound itself (AC3) is not perturbed and
 *     is inclusive.
 *   - A simplex is a tuple of input indices in ascending order; each dimension
 *     is returned as one row-major int32 array (count, d+1) sorted
 *     lexicographically.
 *   - "Device" pointers are CUDA global memory of the current device; "host"
 *     pointers are ordinary (pageable or pinned) memory. Where an argument may
 *     be either, the library asks the CUDA driver which it is.
 *   - stream arguments are cudaStream_t values passed as void* (NULL = the
 *     legacy default stream).
 *   - Every call returns AC_OK (0) or a negative AC_ERR_* code; no exception
 *     crosses this boundary. ac_last_error_detail() gives a message for the
 *     calling thread's last failure.
 *   - Results live in device memory owned by the context and stay valid until
 *     the next ac_build on it or ac_destroy.
 *   - A context is not thread safe: one host thread at a time may use it.
 */
#ifndef ALPHAC_H
#define ALPHAC_H

#include <stdint.h>

#if defined(__GNUC__)
#define AC_API __attribute__((visibility("default")))
#else
#define AC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define AC_OK 0
#define AC_ERR_INVALID_ARG -1 /* NULL pointer, n < 0, NaN/Inf, radius <= 0, bad dim */
#define AC_ERR_DEGENERATE -2  /* two centres coincide after quantisation */
#define AC_ERR_RANGE -3       /* inputs beyond the exact-integer ranges (see ac_create) */
#define AC_ERR_CAPACITY -4    /* an internal list outgrew what regrowth allows */
#define AC_ERR_OOM -5         /* device allocation failed */
#define AC_ERR_CUDA -6        /* a CUDA runtime call failed (the sticky error is not cleared) */
#define AC_ERR_TIMEOUT -7     /* a bounded device-side wait gave up */
#define AC_ERR_STATE -8       /* results asked for before ac_build, or after a failed one */

/* precision of the predicate evaluation; every mode decides every predicate exactly */
#define AC_PRECISION_FILTERED 0  /* FP32 with a forward error bound -> FP64 -> exact integers */
#define AC_PRECISION_PLAIN_FP64 1 /* FP64 with a forward error bound -> exact integers */

/* which value ac_filtration_values returns */
#define AC_FILTRATION_SIZE 0      /* Size (Section 2.3): radius^2 of the smallest empty orthosphere */
#define AC_FILTRATION_ORTHOSIZE 1 /* OrthoSize: the simplex's own orthosphere */

typedef struct ac_ctx ac_ctx;

/* Zero-initialised options select the defaults. */
typedef struct {
    int32_t precision;     /* AC_PRECISION_* */
    int32_t filtration;    /* AC_FILTRATION_* */
    double cell_factor;    /* grid cell side = cell_factor * sqrt(r_max^2 + alpha); 0 = 1.0 */
    int32_t block_warps;   /* warps per block of the per-atom kernel; 0 = 8 */
    int32_t keep_candidates; /* 1: also keep the estimation-pass lists Sigma_ortho^1..3 */
    int32_t no_graph;        /* 1: every ac_build synchronises with the host at each list size
                                (default 0: later builds of a context replay its first build's
                                launch sequence as one CUDA graph, see ac_build) */
    int32_t host_results;    /* 1: ac_build also copies every list (rows, filtration values,
                                attached flags) to page-locked host memory owned by the context,
                                each list as soon as it is final, overlapping the rest of the
                                build; read them with ac_get_simplices_host. The blocks go back
                                to a process-wide cache (at most 8 GB) at ac_destroy, for the
                                next context */
    int32_t reserved[6];
} ac_options;

typedef struct {
    int64_t n_atoms;
    int64_t candidates[4]; /* |Sigma_ortho^d|: simplices with OrthoSize <= alpha (Step 1) */
    int64_t simplices[4];  /* |K_alpha^d| */
    int64_t neighbour_pairs; /* ordered pairs of atoms whose grown balls meet */
    int32_t max_degree;
    int32_t grid_dims[3];
    /* predicate decisions by the level that settled them: [0] FP32, [1] FP64, [2] exact */
    int64_t ac2_tests_tet[3];
    int64_t ac2_tests_tri[3];
    int64_t ac2_tests_edge; /* exact 64-bit integers */
    int64_t ac3_tests[4];   /* AC3 tests per dimension (edges: exact 64-bit integers) */
    int64_t ac3_exact;      /* triangle/tetrahedron AC3 tests the filter left to exact integers */
    double ms_total;        /* device time of the last ac_build (CUDA events) */
    double ms_stage[8];     /* grid, neighbours, per-atom pass, canonical K3, K2, K1+K0+lists, filtration,
                               and the per-atom kernel's own launch */
    int64_t kernel_launches; /* kernels the last ac_build launched (graph nodes when replayed) */
    int32_t replayed;        /* 1: the last ac_build ran as a CUDA graph replay */
    int32_t host_syncs;      /* host waits for the device during the last ac_build */
    int64_t escalated;       /* simplices whose AC3 or AC2 the per-atom kernel's bounds left open,
                                settled by the FP64 / exact-integer kernel */
} ac_stats;

/*
 * Create a context for one set of balls (Section 2: B = {(p_i, r_i)}) and one
 * alpha (Section 2.4). Copies and quantises the input; the caller keeps its
 * buffers. centres: n x 3 row-major doubles (A); radii: n doubles (A), both
 * host or device. opt may be NULL.
 * Ranges checked here (else AC_ERR_RANGE): |coordinate| < 2^20 A (below 2^30
 * quanta of 1/1024 A after rounding to the nearest quantum, so that any two
 * coordinates differ by less than 2^31 quanta), and
 * r_max^2 + alpha <= 16 A^2 (h = sqrt(r_max^2 + alpha) <= 4 A keeps every
 * predicate inside 128-bit integers). n must be below 2^31.
 * Errors: AC_ERR_INVALID_ARG (NULL out, n < 0, NaN/Inf, radius <= 0),
 * AC_ERR_RANGE, AC_ERR_OOM, AC_ERR_CUDA. On error *out is NULL.
 */
AC_API int ac_create(const double* centres, const double* radii, int64_t n, double alpha, const ac_options* opt,
              ac_ctx** out);

/*
 * Create a context for a batch of independent molecules sharing one alpha.
 * Molecule m is atoms [offsets[m], offsets[m+1]) of centres/radii; offsets is
 * a HOST array of n_mol + 1 non-decreasing int64 starting at 0. Indices in the
 * results are per molecule (0-based within the molecule). Each molecule's
 * complex is the one ac_create would give it alone (Section 3.1, Steps 1-5):
 * molecules never interact. Same errors as ac_create.
 */
AC_API int ac_create_batch(const double* centres, const double* radii, const int64_t* offsets, int64_t n_mol,
                    double alpha, const ac_options* opt, ac_ctx** out);

/*
 * Compute the alpha complex (Steps 1-5 of Section 3.1; Sections 4.2-4.4) and
 * the filtration values. Enqueued on stream; returns after the device work is
 * finished. The first build of a context reads each list size back to size
 * the next step (a few host waits). A context's inputs never change, so later
 * builds (unless opt.no_graph) replay the same launch sequence, captured once
 * as a CUDA graph, with every size the first build read checked on the device;
 * a mismatch (not expected: the computation is deterministic) makes that call
 * fall back to a synchronised build. Results are identical either way.
 * Errors: AC_ERR_DEGENERATE, AC_ERR_CAPACITY, AC_ERR_OOM, AC_ERR_CUDA,
 * AC_ERR_TIMEOUT: a bounded device-side wait ran out. Scans of more than 4 M
 * elements (list offsets) are single-pass, each tile waiting for the sums of
 * the tiles before it; a tile polls one flag at most 2^24 times, or the
 * number the environment variable ALPHAC_SCAN_SPIN_LIMIT gives when the scan
 * is launched (a negative value makes every tile stop waiting once, to test
 * this path). A tile whose wait runs out adds the missing sum from the
 * inputs itself, so every offset, and every list built from them, is still
 * exact and the context stays usable; the call reports AC_ERR_TIMEOUT all the
 * same (a wait of that length means something else is holding the GPU), and
 * the next ac_build on the context starts afresh.
 */
AC_API int ac_build(ac_ctx* ctx, void* stream);

/*
 * Device pointer to the simplices of dimension dim (0..3) of the alpha
 * complex K_alpha (Section 2.4; K^3..K^0 of Steps 2-5 of Section 3.1): *count
 * rows of dim+1 ascending int32 input indices, sorted lexicographically. mol selects a
 * molecule of a batch context (-1 for a single-molecule context). Owned by ctx.
 * Errors: AC_ERR_INVALID_ARG, AC_ERR_STATE.
 */
AC_API int ac_get_simplices(ac_ctx* ctx, int dim, int64_t mol, const int32_t** d_tuples, int64_t* count);

/*
 * Device pointer to one double per simplex of ac_get_simplices(dim, mol), in
 * the same order: Size (Section 2.3) in A^2, or OrthoSize when the context was
 * created with AC_FILTRATION_ORTHOSIZE. Owned by ctx.
 * Errors: AC_ERR_INVALID_ARG, AC_ERR_STATE (as ac_get_simplices).
 */
AC_API int ac_filtration_values(ac_ctx* ctx, int dim, int64_t mol, const double** d_f, int64_t* count);

/*
 * Device pointer to one uint8 per simplex of (dim, mol): 1 if AC2 fails at the
 * simplex's own orthocentre (it is in the complex as a face of a larger
 * simplex, "attached"; Section 2.3 and Steps 3-5 of Section 3.1), else 0.
 * Owned by ctx. Errors: AC_ERR_INVALID_ARG, AC_ERR_STATE (as ac_get_simplices).
 */
AC_API int ac_attached_flags(ac_ctx* ctx, int dim, int64_t mol, const uint8_t** d_flags, int64_t* count);

/*
 * Device pointers to the estimation-pass lists Sigma_ortho^dim (dim 1..3; Step
 * 1 of Section 3.1, Section 4.3) of a context created with keep_candidates = 1
 * (single molecule only): rows of ascending input indices, sorted
 * lexicographically. Owned by ctx. Errors: AC_ERR_INVALID_ARG (NULL, dim
 * outside 1..3), AC_ERR_STATE (no build, or candidates not kept).
 */
AC_API int ac_get_candidates(ac_ctx* ctx, int dim, const int32_t** d_tuples, int64_t* count);

/*
 * Re-evaluate the filtration values at other centres/radii (device, same
 * layout as ac_create, n atoms) with the combinatorics of the last build held
 * fixed: each simplex keeps its source simplex (the one whose orthocentre is
 * its closest witness) and takes that source's OrthoSize, in FP64.
 * d_f_out[dim] receives one double per simplex of dim (device, caller-owned;
 * NULL skips that dimension). For finite-difference checks of ac_backward.
 * The value is the Size of Section 2.3 through its source. Errors:
 * AC_ERR_INVALID_ARG (NULL ctx or inputs), AC_ERR_STATE (no build),
 * AC_ERR_OOM, AC_ERR_CUDA.
 */
AC_API int ac_eval_filtration(ac_ctx* ctx, const double* d_centres, const double* d_radii, double* const d_f_out[4],
                       void* stream);

/*
 * The filtration values of the last build evaluated in FP32 arithmetic, as a
 * measure of the error single precision would make (the build itself takes
 * every value from the exact rational, rounded to FP64). Each simplex takes
 * its source's OrthoSize (the same source as ac_filtration_values), computed
 * in single precision from the quantised centres and radii (exact in FP32):
 * offsets, Gram matrix, its solve and the squared orthoradius, every
 * operation rounded to FP32 (Section 2.3 definitions). d_f_out[dim]: device,
 * caller-owned, one float per simplex of dim in list order (NULL skips it).
 * Returns after the device work is finished. Errors: AC_ERR_INVALID_ARG
 * (NULL), AC_ERR_STATE (no build), AC_ERR_CUDA.
 */
AC_API int ac_eval_filtration_fp32(ac_ctx* ctx, float* const d_f_out[4], void* stream);

/*
 * Gradient of L = sum_dim sum_s dLdf[dim][s] * f[dim][s] with respect to the
 * centres and radii, combinatorics fixed (FP64). With lambda the barycentric
 * coordinates of the source's orthocentre c in its affine hull:
 * df/dp_k = 2 lambda_k (p_k - c), df/dr_k = -2 r_k lambda_k.
 * d_dLdf[dim]: device, one double per simplex (NULL = zero). Outputs are
 * device, caller-owned, n x 3 and n doubles, OVERWRITTEN (not accumulated).
 * The paper gives no gradient: this is the derivative of the Size of Section
 * 2.3, taken through the source simplex's OrthoSize with the source held fixed
 * (an envelope argument: the multipliers of the equal-power constraints are
 * the barycentric coordinates of c). Every sum is taken in a fixed order (up
 * the build's coface links to each source simplex, then per atom; no
 * floating-point atomics), so repeated calls give bit-identical gradients.
 * Scratch: 8 bytes per simplex and 32 per vertex of each simplex, allocated by
 * the context on first use. Returns after the device work is finished.
 * Errors: AC_ERR_INVALID_ARG (NULL), AC_ERR_STATE (no build), AC_ERR_OOM,
 * AC_ERR_CUDA.
 */
AC_API int ac_backward(ac_ctx* ctx, const double* const d_dLdf[4], double* d_dLdcentres, double* d_dLdradii,
                void* stream);

/*
 * ac_backward without any device allocation. The paper has no counterpart:
 * this serves callers that cannot allocate device memory (a training step
 * whose memory belongs to another allocator, a service with a fixed device
 * memory budget). It runs the one-pass backward kernel (one thread per
 * simplex, FP64 atomic adds into the outputs), whose only scratch is a table
 * of the 4 per-dimension list pointers; here that table is a static device
 * array (32 bytes, 256-byte aligned) that every GPU loading the library holds
 * until exit. Same arguments and errors as ac_backward (AC_ERR_CAPACITY if a
 * context had more lists than the table holds); the gradients agree with
 * ac_backward's to rounding, the atomics adding in no fixed order. The first
 * call on a device looks up the table's device address (with that device
 * current) and keeps it for the process, so it is stale after a
 * cudaDeviceReset; make that first call before any stream capture. Every call
 * rewrites the whole table and synchronises the stream before returning;
 * calls that overlap on the GPU share the table and race.
 */
AC_API int ac_backward_noalloc(ac_ctx* ctx, const double* const d_dLdf[4], double* d_dLdcentres, double* d_dLdradii,
                               void* stream);

/*
 * Choose the grid cell side (cell_factor in units of sqrt(r_max^2 + alpha),
 * the side Section 4.2 fixes)
 * and the warps per block of the per-atom kernel by timing builds of this
 * context over a small grid of both (cell factors 0.5 to 2, 4 to 8 warps: 36
 * builds); the fastest is
 * kept in the context, a final ac_build leaves valid results, and the choice
 * is copied to *chosen (may be NULL). Results do not depend on the choice.
 * Same errors as ac_build.
 */
AC_API int ac_autotune(ac_ctx* ctx, void* stream, ac_options* chosen);

/*
 * The alpha complex at a smaller alpha from a built one (the filtration
 * restricted; the alpha sweep of Section 6): K_alpha2 = {sigma in K_alpha :
 * Size(sigma) <= alpha2} (Section 2.4, inclusive), decided exactly on the
 * rational Size (not on its FP64 rounding). alpha2 is quantised like alpha
 * (rint(2^20 alpha2)) and must not exceed the context's alpha.
 * d_flags: caller-owned DEVICE array of the list's length (ac_get_simplices'
 * count for dim and mol); entry j is set to 1 if row j is in K_alpha2, else 0.
 * *count_in receives the number of rows set. Synchronises the stream.
 * Errors: AC_ERR_INVALID_ARG (bad dim/mol, NULL, alpha2 > alpha), AC_ERR_STATE
 * (no build yet), AC_ERR_CUDA.
 */
AC_API int ac_subcomplex(ac_ctx* ctx, int dim, int64_t mol, double alpha2, uint8_t* d_flags, int64_t* count_in,
                         void* stream);

/*
 * ---- Out-of-core build: host-resident inputs and results ----------------
 *
 * For a molecule whose lists do not fit in device memory at once (Section
 * 4.6: partitions processed one at a time with their border, results copied
 * back to host memory): the atoms are cut into
 * slabs along z, and each slab is built on the GPU as the alpha complex of its
 * atoms plus a halo, the atoms within reach of the slab (|dZ| <= 2 h, in
 * quanta, h = ceil(sqrt(r_max^2 + alpha))). A simplex belongs to the slab that
 * holds its first (smallest-index) vertex. Every simplex with that vertex in
 * the slab, its AC2 and AC3 decisions, its attached flag and its Size depend
 * only on atoms whose grown balls meet that vertex's (the simplex's cofaces
 * contain the vertex; their violators are common neighbours of their
 * vertices), so the halo makes each slab's share exactly that of the whole
 * molecule, and no simplex is produced twice (Section 4.6 removes duplicates
 * instead). The shares are brought to host memory and placed in order of
 * their first vertex: the result equals what ac_build returns for the whole
 * molecule, list for list.
 */
typedef struct ac_chunked ac_chunked;

typedef struct {
    int64_t n_chunks;      /* slabs with at least one atom */
    int64_t reach;         /* halo width in quanta (2 h) */
    int64_t core_max;      /* most atoms in one slab */
    int64_t subset_max;    /* most atoms in one slab plus its halo (what one device build holds) */
    int64_t subset_total;  /* atoms built over all slabs (halo atoms counted in every slab) */
    double ms_plan;        /* host: quantised z, slab cuts, slab membership (wall clock) */
    double ms_device;      /* wall clock of the slab builds, incl. host<->device copies */
    double ms_assemble;    /* host: placement of the shares in first-vertex order */
} ac_chunked_stats;

/*
 * The slab cut of ac_build_chunked alone (Section 4.6; host only, no GPU
 * needed). centres n x 3 and radii n
 * are HOST doubles (A). Slab k holds the atoms with thresholds[k] <= Z <
 * thresholds[k+1], Z = rint(1024 z); the cuts keep at most max_core_atoms
 * atoms in a slab unless more than that share one cut interval (a run of
 * atoms with the same Z, or, for z spans above 2^22 quanta, the same
 * 2^-22 of the span). thresholds: caller array of cap entries, filled with
 * *n_chunks + 1 values; *reach = 2 ceil(sqrt(max W + A)) quanta (0 if no ball
 * survives alpha). Errors: AC_ERR_INVALID_ARG (NULL, n < 0, max_core_atoms
 * < 1, NaN/Inf, radius <= 0, cap too small: *n_chunks is still set),
 * AC_ERR_RANGE (as ac_create).
 */
AC_API int ac_chunk_plan(const double* centres, const double* radii, int64_t n, double alpha, int64_t max_core_atoms,
                         int64_t* thresholds, int64_t cap, int64_t* n_chunks, int64_t* reach);

/*
 * Build the alpha complex of n HOST balls slab by slab (Section 4.6: the data
 * split into parts processed one at a time, each with its border), at most
 * max_core_atoms atoms per slab (plus halo) on the device at a time. opt as
 * for ac_create (keep_candidates must be 0). The slabs run one after another
 * on stream; *out receives a result whose lists live in host memory (read
 * them with ac_chunked_simplices; free with ac_chunked_free). Synchronous.
 * Errors: those of ac_chunk_plan, ac_create and ac_build, AC_ERR_OOM (host
 * memory). On error *out is NULL.
 */
AC_API int ac_build_chunked(const double* centres, const double* radii, int64_t n, double alpha,
                            const ac_options* opt, int64_t max_core_atoms, void* stream, ac_chunked** out);

/*
 * One molecule over several processes (Section 4.6: the grid split into
 * parts, each processed with its border; here each part on its own GPU):
 * ac_part_plan cuts the quantised z of the n HOST balls into n_parts ranges
 * of about n / n_parts atoms each (host only, no GPU): thresholds (n_parts + 1
 * int64, caller-owned) are in 1/1024 A, part p holding the atoms with
 * thresholds[p] <= Z < thresholds[p + 1]; *reach is the halo, 2 sqrt(r_max^2 +
 * alpha) in 1/1024 A (rounded up). Parts hold about equal numbers of atoms, or
 * none when many atoms share one z. Errors: AC_ERR_INVALID_ARG (NULL, n < 0,
 * n_parts < 1, non-finite input), AC_ERR_RANGE (as ac_create).
 */
AC_API int ac_part_plan(const double* centres, const double* radii, int64_t n, double alpha, int64_t n_parts,
                        int64_t* thresholds, int64_t* reach);

/*
 * Part `part` of n_parts (the cut of ac_part_plan; Section 4.6, a part with
 * its border) of the alpha complex of n HOST balls: every simplex whose first (smallest input index) vertex lies in
 * the part, with its attached flag and filtration value, exactly as the whole
 * molecule's build has them. Built like ac_build_chunked, restricted to the
 * part: slabs of at most max_core_atoms atoms of the part, each with every
 * atom within the halo (from all n). Every coface of such a simplex, and every
 * ball that can violate AC2 at their orthocentres, has a grown ball meeting
 * the first vertex's, so the halo holds them all; the shares of the parts are
 * disjoint and together make the whole complex. The result (host lists, as
 * ac_chunked_simplices reads them; free with ac_chunked_free) lists the rows
 * in first-vertex order. Synchronous. Errors: those of ac_build_chunked,
 * AC_ERR_INVALID_ARG (part outside [0, n_parts)). On error *out is NULL.
 */
AC_API int ac_build_part(const double* centres, const double* radii, int64_t n, double alpha, const ac_options* opt,
                         int64_t n_parts, int64_t part, int64_t max_core_atoms, void* stream, ac_chunked** out);

/*
 * The whole complex from the shares of the parts (host only; Section 4.6
 * concatenates the parts' results and removes duplicates, which first-vertex
 * ownership makes unnecessary here): counts
 * (n_parts x 4 int64, part-major) gives the rows of each part and dimension,
 * tuples/f/attached (n_parts x 4 host pointers, the arrays ac_chunked_simplices
 * gives for that part) the rows, values and flags. Each first vertex's rows
 * come from one part, in order: they are placed at that vertex's place in the
 * lexicographic order, with no search for duplicates. The result is read with
 * ac_chunked_simplices and freed with ac_chunked_free. Errors:
 * AC_ERR_INVALID_ARG (NULL, a negative count, a first vertex outside [0, n),
 * two parts with rows of the same first vertex, a share out of order),
 * AC_ERR_OOM. On error *out is NULL.
 */
AC_API int ac_merge_parts(int64_t n, int64_t n_parts, const int64_t* counts, const int32_t* const* tuples,
                          const double* const* f, const uint8_t* const* attached, ac_chunked** out);

/*
 * Host pointers to dimension dim of a chunked result: tuples (count, dim+1)
 * int32 input indices, ascending in a row, rows lexicographically sorted;
 * f: the filtration values (opt.filtration); attached: the attached flags
 * (as ac_attached_flags). Owned by the result. Any output pointer may be NULL.
 * Errors: AC_ERR_INVALID_ARG (NULL result, dim outside 0..3).
 */
AC_API int ac_chunked_simplices(const ac_chunked* res, int dim, const int32_t** tuples, const double** f,
                                const uint8_t** attached, int64_t* count);

/* Slab counts and times of a chunked build. Errors: AC_ERR_INVALID_ARG. */
AC_API int ac_chunked_info(const ac_chunked* res, ac_chunked_stats* out);

/* Free a chunked result. NULL is a no-op. */
AC_API void ac_chunked_free(ac_chunked* res);

/*
 * Host copies of the K_alpha lists (Section 2.4) of dimension dim (0..3) of
 * molecule mol (-1 for a single-molecule context), made by the last ac_build
 * of a context created with
 * opt.host_results = 1: *count rows of dim+1 int32 indices (as
 * ac_get_simplices), their filtration values (as ac_filtration_values) and
 * attached flags (as ac_attached_flags). Page-locked host memory owned by the
 * context, valid until the next ac_build or ac_destroy. Any output pointer
 * but count may be NULL.
 * Errors: AC_ERR_INVALID_ARG (bad dim/mol), AC_ERR_STATE (no build, or the
 * context does not keep host results).
 */
AC_API int ac_get_simplices_host(ac_ctx* ctx, int dim, int64_t mol, const int32_t** h_tuples, const double** h_f,
                                 const uint8_t** h_attached, int64_t* count);

/* Counters and stage times of the last ac_build (all zero before one), copied
 * to *out. Errors: AC_ERR_INVALID_ARG (NULL). */
AC_API int ac_get_stats(ac_ctx* ctx, ac_stats* out);

/* Number of molecules (1 for a single-molecule context) and atoms; either
 * output may be NULL. Errors: AC_ERR_INVALID_ARG (NULL ctx). */
AC_API int ac_get_sizes(ac_ctx* ctx, int64_t* n_mol, int64_t* n_atoms);

/* Measurement helper; the paper has no counterpart (it is not part of the
 * method, Section 5 reports timings only): the device's FMA throughput in
 * FP32 (fp64 = 0) or FP64 (fp64 = 1), in floating-point operations per second
 * (an FMA counts two), from independent FMA chains in registers over a launch
 * that fills every SM for `iters` steps per chain (one untimed launch of an
 * eighth of them first), timed with CUDA events on `stream` (NULL: the default
 * stream). The denominator that the per-atom kernel's arithmetic is compared
 * with beside the peak derived from unit counts and clock. *ms (may be NULL)
 * receives the timed launch's duration. Synchronises the stream.
 * Errors: AC_ERR_INVALID_ARG (NULL output, iters < 1), AC_ERR_CUDA, AC_ERR_OOM. */
AC_API int ac_fma_peak(int fp64, int iters, void* stream, double* flops_per_s, float* ms);

/* Free the context and everything it owns. NULL is a no-op. */
AC_API void ac_destroy(ac_ctx* ctx);

/* Static description of an AC_* code. */
AC_API const char* ac_error_string(int code);

/* Detail of the calling thread's last failure (empty string if none). */
AC_API const char* ac_last_error_detail(void);

#ifdef __cplusplus
}
#endif
#endif /* ALPHAC_H */
