/*
 * vfmm: adaptive volume-potential box FMM on one GB300 (sm_103a).
 *
 * Computes, at every collocation node of every leaf of a level-restricted
 * quadtree, the volume integral of Section 3 (Eq. volumeint3)
 *     u(x) = V[f~](x) = -(1/2 pi) int_B log|x - y| f~(y) dy
 * and its gradient (Section 3.2, Eq. volumeint3x), where B is the root box and
 * f~ is the piecewise polynomial interpolant of f on the leaves (Section 3.1).
 *
 * Conventions shared by every entry point
 *  - Root box: centre (cx, cy), width W. A box at level l has width W 2^-l and
 *    integer coordinates (ix, iy) in [0, 2^l)^2. Boxes are numbered in
 *    canonical order: by level, then by Morton key (bit b of ix -> bit 2b,
 *    bit b of iy -> bit 2b + 1). Leaves are numbered in the same order.
 *  - Leaf nodes: tensor first-kind Chebyshev nodes, k per side; node (i, j) of
 *    a leaf of width h and lower-left corner (lo_x, lo_y) sits at
 *    x = lo_x + h (i_box + 1/2 + xhat_i), xhat_i = -cos(pi (2i+1) / (2k)) / 2,
 *    stored x-fastest: flat index j*k + i.
 *  - Values arrays (f, u, u_x, u_y) are FP64, [nrhs][n_leaves][k*k], leaf-major
 *    in canonical leaf order, row-major, no padding.
 *  - Level restriction (Section 3.1): adjacent leaves (corner contact counts)
 *    differ by at most one level.
 *  - Refinement (Section 3.1, Section 6.1): a box at level l < max_depth is
 *    split when the largest |c_mn| with max(m, n) >= k - 2 of its 2-D Chebyshev
 *    coefficients exceeds tol * F, F = max |f| over the nodes of the uniform
 *    tree of level min(5, max_depth); boxes above min_depth always split.
 *  - Pointers named *_dev are CUDA device pointers on the current device;
 *    everything else is host memory. The caller owns every buffer it passes;
 *    the library owns the memory behind vfmm_tree and vfmm_ops handles and
 *    frees it in the matching destroy call.
 *  - Streams: `stream` is a cudaStream_t (NULL = legacy default stream). Calls
 *    that fill device buffers are stream-ordered and return before the work
 *    completes, unless stated otherwise.
 *  - Errors: every call returns VFMM_OK (0) or a negative VFMM_ERR_* code and
 *    never aborts; vfmm_strerror() names the code and vfmm_last_error_detail()
 *    gives the last failure's message (thread-local).
 */
#ifndef VFMM_H
#define VFMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define VFMM_OK 0
#define VFMM_ERR_INVALID_ARG (-1)
#define VFMM_ERR_OOM (-2)
#define VFMM_ERR_CUDA (-3)
#define VFMM_ERR_NOT_BUILT (-4)
#define VFMM_ERR_TIMEOUT (-5)
#define VFMM_ERR_WORKSPACE (-6)
#define VFMM_ERR_INTERNAL (-7)

/* Source kinds; params layouts (host FP64 arrays):
 *  CONSTANT  : [A]                                         f = A
 *  GAUSS_SUM : n rows [cx, cy, sigma, A]                   f = sum A exp(-|x-c|^2 / (2 sigma^2))
 *  KINKED    : [a_2..a_8, c_2..c_8, 5 g rows, 5 h rows]    f = g max(0, phi) + h,
 *              phi = r_chi(x)^2 - |x|^2, r_chi = 0.6 + chi(|x|) sum_m a_m cos(m theta + c_m),
 *              chi(rho) = psi((rho - 0.1)/0.2), psi(t) = e^{-1/t} / (e^{-1/t} + e^{-1/(1-t)}),
 *              g and h Gaussian sums in the GAUSS_SUM row layout (n = 5). */
#define VFMM_SRC_CONSTANT 0
#define VFMM_SRC_GAUSS_SUM 1
#define VFMM_SRC_KINKED 2

/* Arithmetic of the solve. */
#define VFMM_FP64 0  /* every product and sum in FP64 */
/* VFMM_MIXED: every dense contraction (near-field tables, S2M, M2L, S2L, L2T + M2T) as split-BF16
 * tcgen05 products with FP32 accumulators; FP64 for the log(h) terms, coefficient 0 of every
 * expansion, M2M, L2L and the final per-target sums. */
#define VFMM_MIXED 1

#define VFMM_LIST_U 0 /* leaves: the leaf itself and every adjacent leaf (near field) */
#define VFMM_LIST_V 1 /* boxes: children of parent's colleagues not adjacent to the box (M2L) */
#define VFMM_LIST_W 2 /* leaves: children of colleagues not adjacent to the leaf (M2T) */
#define VFMM_LIST_X 3 /* boxes: leaves c with the box in W(c) (S2L) */

typedef struct vfmm_tree vfmm_tree;
typedef struct vfmm_ops vfmm_ops;

typedef struct {
    double cx, cy, width; /* root box */
    int32_t k;            /* nodes per side, 4 <= k <= 16 */
    int32_t max_depth;    /* 0 <= max_depth <= 16 */
    int32_t min_depth;    /* 0 <= min_depth <= max_depth */
    double tol;           /* refinement tolerance (relative to F) */
} vfmm_tree_params;

typedef struct {
    int32_t kind;         /* VFMM_SRC_* */
    int32_t n;            /* GAUSS_SUM: number of rows; ignored otherwise */
    const double* params; /* host, layout above */
} vfmm_source;

typedef struct {
    int64_t n_boxes, n_leaves;
    int32_t depth, k;
    int64_t list_len[4]; /* entries in the U, V, W, X lists */
    double f_scale;      /* F of the refinement test (0 for uniform trees) */
    double min_margin;   /* min over refinement decisions of |q / (tol F) - 1|, q the split test's
                            quantity (the tail, or a vfmm_tree_build_rule rule's weighted error) */
    int64_t n_depth_capped; /* leaves at max_depth whose split test still fails (informational:
                               the tree is complete but that refinement stopped at the depth cap;
                               0 for uniform trees, -1 where not tested: leaf-count and pull builds) */
} vfmm_tree_info_t;

/* Adaptive build (Section 3.1): level-by-level refinement of the root box by the
 * tail test on f, then the minimal refinement that meets the level restriction,
 * canonical numbering and the U/V/W/X lists, all on the device.
 * Synchronises `stream` (box counts are read back per level).
 * Errors: INVALID_ARG (bad k, depths, width <= 0, tol < 0, unknown source kind),
 * OOM, CUDA. */
int vfmm_tree_build(const vfmm_tree_params* prm, const vfmm_source* src, void* stream, vfmm_tree** out);

/* Refinement rules of vfmm_tree_build_rule. */
#define VFMM_REFINE_TAIL 0          /* trailing Chebyshev coefficients (vfmm_tree_build) */
#define VFMM_REFINE_INTERP 1        /* interpolation error */
#define VFMM_REFINE_INTERP_AREA 2   /* interpolation error x (h / width)^2 */
#define VFMM_REFINE_INTERP_MIXED 3  /* x (h / width)^2 on boxes meeting the boundary, x h / width elsewhere */

/* vfmm_tree_build with the a-priori rules of Section 6.1 (on adaptivity) as the split
 * test: the interpolation error e = max |f - p| over the nodes of the box's four children, p the
 * interpolant of f on the box's own nodes, compared with tol * F unweighted (INTERP), times the
 * relative area (INTERP_AREA), or times the relative area where the box meets the source's
 * boundary and the relative side length elsewhere (INTERP_MIXED). Boundary: the curve where the
 * kinked source is only continuous (its level set takes both signs on those nodes); other
 * sources have none. F, depths, balance, numbering and lists as vfmm_tree_build; TAIL is
 * vfmm_tree_build itself. Errors as vfmm_tree_build, and INVALID_ARG for an unknown rule. */
int vfmm_tree_build_rule(const vfmm_tree_params* prm, const vfmm_source* src, int32_t rule, void* stream,
                         vfmm_tree** out);

/* Tree with a leaf-count target (for batches of uneven problems; the paper refines to a
 * tolerance only): starting from the root, the leaf of highest priority is split, one at a
 * time, until the tree has >= n_leaves leaves or no leaf below prm->max_depth is left; then
 * the same level restriction, numbering and lists as vfmm_tree_build. Priority of a leaf =
 * the binary exponent e of its tail (the same trailing-coefficient test quantity, tail in
 * [2^(e-1), 2^e)), raised to at least e_F - 30 where F = max |f| as for vfmm_tree_build
 * (tails near rounding level all tie); ties go to the coarser leaf, then the smaller Morton
 * key. The queue is kept on the host; tails are computed on the device in batches.
 * tree_info.min_margin = smallest relative distance of a deciding tail to a power of two.
 * prm->tol and prm->min_depth are ignored. Synchronises `stream`.
 * Errors: INVALID_ARG (bad k, max_depth, width, n_leaves outside [1, 2^26], source), OOM, CUDA. */
int vfmm_tree_build_leaves(const vfmm_tree_params* prm, const vfmm_source* src, int64_t n_leaves, void* stream,
                           vfmm_tree** out);

/* Builds n independent trees at once (a batch of uneven problems; no counterpart in the paper):
 * tree i as vfmm_tree_build_leaves(&prm[i], &src[i], n_leaves[i], ...) when n_leaves[i] > 0, else as
 * vfmm_tree_build(&prm[i], &src[i], ...). Up to n_threads host threads (<= 0: one per host core, at
 * most 16) take trees in turn, each on a CUDA stream of its own on the current device, so that the
 * host work (priority queues, lists, plans) and the device work of different trees overlap. The
 * trees are the same as the single builds' (bit for bit). Returns when all are built; out[n] holds
 * them. Errors: those of the single builds (the first failing tree's code; every tree built so far
 * is then destroyed and out[] zeroed), INVALID_ARG (null pointers, n < 0). */
int vfmm_tree_build_many(const vfmm_tree_params* prm, const vfmm_source* src, const int64_t* n_leaves, int32_t n,
                         int32_t n_threads, vfmm_tree** out);

/* Uniform tree of the given depth (prm->tol and depths ignored). Synchronises. */
int vfmm_tree_build_uniform(const vfmm_tree_params* prm, int32_t depth, void* stream, vfmm_tree** out);

/* Adaptive build for an f the caller evaluates (Section 3.1 refinement; the method asks the
 * user for nothing about f but a way to evaluate it, Section 7): a pull protocol over an
 * opaque builder.
 *   vfmm_tree_begin            starts a build with vfmm_tree_build's parameters, on `stream`;
 *   vfmm_tree_pending          number of nodes where f is wanted next (0: refinement complete);
 *   vfmm_tree_pending_nodes    writes those nodes' x and y to caller-owned device buffers of
 *                              that length (enqueued on the builder's stream);
 *   vfmm_tree_submit           takes f at those nodes (device, same order; read on the builder's
 *                              stream, which the call synchronises before returning);
 *   vfmm_tree_finish           after pending reached 0: the level restriction, numbering and
 *                              lists, as vfmm_tree_build; returns the tree (once per builder);
 *   vfmm_tree_builder_destroy  frees the builder (the tree stays valid).
 * Rounds: first the k*k nodes of every box of the uniform level min(5, max_depth) (their max |f|
 * is the F of the tail test), then, per level from min_depth on, the k*k nodes of every candidate
 * box (box-major, node j*k + i with x varying fastest, as leaf nodes). Levels below min_depth
 * split without f. With f equal to a built-in source at the same nodes the tree equals
 * vfmm_tree_build's. Errors: INVALID_ARG (parameters as vfmm_tree_build, null pointers, nodes
 * or f requested when none are pending, finish before refinement completes or twice), OOM,
 * CUDA. */
typedef struct vfmm_tree_builder vfmm_tree_builder;
int vfmm_tree_begin(const vfmm_tree_params* prm, void* stream, vfmm_tree_builder** out);
int vfmm_tree_pending(const vfmm_tree_builder* b, int64_t* n_nodes);
int vfmm_tree_pending_nodes(const vfmm_tree_builder* b, double* x_dev, double* y_dev);
int vfmm_tree_submit(vfmm_tree_builder* b, const double* f_dev);
int vfmm_tree_finish(vfmm_tree_builder* b, vfmm_tree** out);
int vfmm_tree_builder_destroy(vfmm_tree_builder* b);

int vfmm_tree_info(const vfmm_tree* tree, vfmm_tree_info_t* info);

/* Host copies of the box table: level, ix, iy, each [n_boxes] int32. Synchronous. */
int vfmm_tree_export_boxes(const vfmm_tree* tree, int32_t* level, int32_t* ix, int32_t* iy);

/* Host copy of one list in CSR form: ptr [n_boxes + 1], idx [len], cfg [len] (box
 * indices ascending within a row). D = (centre of the entry - centre of the row's box)
 * / h, h the width of the row's box. cfg:
 *  U -> 0..8 for a leaf of the same level, (dy + 1) * 3 + (dx + 1) with (dx, dy) = D;
 *       9..20 for a leaf one level coarser, 9 + the position of 2D and 21..32 for a
 *       leaf one level finer, 21 + the position of 4D in the 12-entry pattern
 *       {(+-3, +-1), (+-1, +-3), (+-3, +-3)} sorted by (y, x);
 *  V -> the position of D in the 40 offsets of [-3, 3]^2 outside [-1, 1]^2, row-major
 *       (dy outer, dx inner, ascending);
 *  W -> the position of 4D, X -> the position of 2D, in the 20-entry pattern
 *       {(+-5, +-1), (+-1, +-5), (+-5, +-3), (+-3, +-5), (+-5, +-5)} sorted by (y, x).
 * Any output pointer may be NULL. Synchronous. */
int vfmm_tree_export_list(const vfmm_tree* tree, int32_t which, int32_t* ptr, int32_t* idx, int32_t* cfg);

/* Node coordinates of every leaf, x_dev and y_dev [n_leaves * k * k]. */
int vfmm_tree_leaf_nodes(const vfmm_tree* tree, double* x_dev, double* y_dev, void* stream);

/* f at every leaf node, f_dev [n_leaves * k * k]. */
int vfmm_source_sample(const vfmm_tree* tree, const vfmm_source* src, double* f_dev, void* stream);

int vfmm_tree_destroy(vfmm_tree* tree);

/* Unit-scale operators of the box code for (k, p) (Section 3.1: tables computed once for a unit
 * box and reused at every level up to scale; Section 3.2 for the gradient tables), generated on the
 * device: 33 near-field tables of the potential and both gradient components,
 * S2M, S2L (20), M2T geometry (20), L2T, M2M (4), M2L (40), L2L (4).
 * 4 <= k <= 16, 1 <= p <= 60. Synchronises. Errors: INVALID_ARG, OOM, CUDA. */
int vfmm_ops_create(int32_t k, int32_t p, int32_t precision, void* stream, vfmm_ops** out);

/* Host copy of one operator table for parity tests (layouts in the binding). */
#define VFMM_OP_NEAR 0 /* [33][3][k*k][k*k] */
#define VFMM_OP_S2M 1  /* [p+1][k*k] complex (re, im interleaved) */
#define VFMM_OP_S2L 2  /* [20][p+1][k*k] complex */
#define VFMM_OP_M2M 3  /* [4][p+1][p+1] complex */
#define VFMM_OP_L2L 4  /* [4][p+1][p+1] complex */
#define VFMM_OP_M2L 5  /* [40][p+1][p+1] complex */
int vfmm_ops_export(const vfmm_ops* ops, int32_t which, double* host, int64_t n_doubles);

int vfmm_ops_destroy(vfmm_ops* ops);

/* Slices of the split-BF16 contractions of a VFMM_MIXED operator set (no counterpart in the paper,
 * which computes in double precision). Every operand of a contraction is stored as 8 balanced
 * base-128 digits (56 bits below its power-of-two scale); a contraction that takes S of them
 * (6 <= S <= 8) issues the S (S + 1) / 2 slice products i + j <= S + 1 and rounds each operand at
 * 2^(-7 S - 1) of its scale: fewer tensor-core products and fewer gathered bytes, less accuracy.
 * slices[5] = near field, S2M, M2L, S2L, leaf far field (L2T + M2T); a new operator set takes 6
 * for all, the fewest allowed: the error against the FP64 form stays at or below 6e-12 on the
 * adaptive 20-Gaussian (k = 16, p = 40), kinked and uniform depth-7 (k = 16) workloads.
 * Host-only; applies to later calls and graph captures (a graph keeps the counts it captured); not
 * while a solve with these operators is being launched. Errors: INVALID_ARG (null pointer, not
 * VFMM_MIXED, a count outside [6, 8]). */
int vfmm_ops_set_slices(vfmm_ops* ops, const int32_t* slices);
int vfmm_ops_get_slices(const vfmm_ops* ops, int32_t* slices);

/* Form of the M2L translation (the V-list far field of Section 3.1). The paper's box code
 * diagonalises it with plane waves (Section 3.1, citing [Ethridge] and [Hrycak98]); this library
 * also keeps the dense (p+1) x (p+1) Laurent-to-Taylor matrix per V offset, which the tensor-core
 * form needs.
 *  VFMM_M2L_DENSE      dense translation per V entry (the default; the only form of VFMM_MIXED);
 *  VFMM_M2L_PLANEWAVE  VFMM_FP64 only: per box, the multipole goes to s exponential (plane-wave)
 *                      coefficients for each of the four sides (1/u^n as a Laplace integral,
 *                      discretised by an s-node rule built for the 14 rotated V offsets and
 *                      every order the translation needs); a V entry is then one complex
 *                      multiplication per coefficient, and each box turns the sum back into its
 *                      local expansion. The log term of the multipole is added exactly. s = 57,
 *                      73, 83, 88 for p <= 10, 20, 30, 60; the result differs from the dense form by
 *                      about 1e-15 of the potential's scale.
 * vfmm_ops_set_m2l changes the solve's workspace size (query vfmm_workspace_size again); a graph
 * keeps the form it captured. Host-only; not while a solve with these operators is being launched.
 * vfmm_ops_get_m2l returns the form and s (n_waves may be NULL). Errors: INVALID_ARG (null ops,
 * unknown form, PLANEWAVE on a VFMM_MIXED operator set). */
#define VFMM_M2L_DENSE 0
#define VFMM_M2L_PLANEWAVE 1
int vfmm_ops_set_m2l(vfmm_ops* ops, int32_t form);
int vfmm_ops_get_m2l(const vfmm_ops* ops, int32_t* form, int32_t* n_waves);

/* Device workspace the solve needs for this tree, operator set and nrhs
 * (multipole and local expansions, near-field partial products). with_io != 0
 * adds room for the device copies vfmm_volume_potential_host stages through.
 * VFMM_MIXED with nrhs > 1 builds (once per tree and nrhs, host-side, cached in the
 * tree under a lock) the contraction schedules with the right-hand sides folded in. */
int vfmm_workspace_size(const vfmm_tree* tree, const vfmm_ops* ops, int32_t nrhs, int32_t with_io,
                        size_t* bytes);

/* The box code (Section 3.1): u, u_x, u_y at every leaf node for nrhs right-hand
 * sides: upward pass (S2M, M2M), downward pass (M2L over V, S2L over X, L2L),
 * leaf pass (near-field tables over U with the log(h) scale term, L2T, M2T over W).
 * Layout: f, u, u_x, u_y are [nrhs][n_leaves][k*k] doubles (canonical leaf order, x-fastest
 * nodes). VFMM_FP64 solves the right-hand sides one after another; VFMM_MIXED folds them
 * into one solve whose tensor-core contractions carry nrhs rows per leaf or box (no
 * counterpart in the paper, which solves one right-hand side at a time).
 * Everything is ordered on `stream`, with no host synchronisation and no allocation (the first
 * VFMM_MIXED call for a new nrhs builds its schedules on the host, see vfmm_workspace_size).
 * VFMM_MIXED forks its work onto internal streams that the library keeps per host thread and
 * device (created by the thread's first call made outside stream capture): S2L and the near field
 * on a lowest-priority stream, the rest of the solve on a highest-priority one (coefficient 0 on
 * a third), all joined back into `stream` by events before the call returns; under stream
 * capture the fork becomes parallel branches of the graph (kernel nodes keep their priorities).
 * Errors: INVALID_ARG (k or p of ops differ from the tree's k, nrhs < 1), WORKSPACE
 * (workspace_bytes below vfmm_workspace_size), CUDA. A bounded device wait that runs out
 * (VFMM_ERR_TIMEOUT) happens after this call has returned: it is recorded in a status word at
 * the start of the workspace, cleared by each call, which vfmm_workspace_status reads once
 * `stream` has been synchronised. */
int vfmm_volume_potential(const vfmm_tree* tree, const vfmm_ops* ops, const double* f_dev, int32_t nrhs,
                          double* u_dev, double* ux_dev, double* uy_dev, void* workspace_dev,
                          size_t workspace_bytes, void* stream);

/* Same, from host buffers: copies f to the device, solves, copies u, u_x, u_y back
 * and synchronises `stream`. Host buffers should be pinned for full copy speed.
 * The workspace must be sized with with_io = 1. Synchronous, so a bounded wait that ran
 * out is returned as VFMM_ERR_TIMEOUT by this call itself. */
int vfmm_volume_potential_host(const vfmm_tree* tree, const vfmm_ops* ops, const double* f_host, int32_t nrhs,
                               double* u_host, double* ux_host, double* uy_host, void* workspace_dev,
                               size_t workspace_bytes, void* stream);

/* Status of the last solve that used this workspace (no counterpart in the paper). The
 * asynchronous calls (vfmm_volume_potential, graph replays, batch items, the allocation-free
 * entry point) cannot return a timeout themselves; every bounded device wait that runs out
 * records where in the status word at the start of the workspace that the solve used. Call
 * this after synchronising the solve's stream: it copies the word to the host (synchronous) and
 * returns VFMM_OK, or VFMM_ERR_TIMEOUT with the site in vfmm_last_error_detail; the results of
 * such a solve are incomplete. workspace_dev = NULL reads the word of the allocation-free entry
 * point's static scratch on the current device. Errors: CUDA. */
int vfmm_workspace_status(const void* workspace_dev);

/* v~: values at arbitrary points (Section 3.1: away from the collocation nodes the paper takes
 * the polynomial that interpolates the computed values on the leaf holding the point; Section
 * 3.3 on its error). For each point (x_dev[i], y_dev[i]) and each of the n_fields fields
 * (1..8; fields_dev and out_dev are host arrays of n_fields device pointers), out_dev[q][i] =
 * the tensor Lagrange interpolant on the leaf's k x k nodes of fields_dev[q] ([n_leaves][k*k],
 * the layout of f and u, e.g. u, u_x, u_y of one right-hand side) at the point.
 * The leaf of a point comes from its integer coordinates at the finest level,
 * floor(2^depth (x - lo) / width) (clamped to 2^depth - 1 on the root's upper edges), so a
 * point on an edge shared by two leaves belongs to the one above or to its right; leaf_dev
 * (optional, [n_points] int32) receives its canonical leaf index. Points outside the closed
 * root box or with a NaN coordinate get NaN and leaf -1. Stream-ordered, no allocation.
 * Errors: INVALID_ARG (null tree or pointers, n_fields outside [1, 8], n_points < 0), CUDA. */
int vfmm_leaf_interpolate(const vfmm_tree* tree, int32_t n_fields, const double* const* fields_dev,
                          int64_t n_points, const double* x_dev, const double* y_dev, double* const* out_dev,
                          int32_t* leaf_dev, void* stream);

/* The computed potential at arbitrary points from the stored expansions (Section 5.3: the FMM's
 * multipole and local expansions are kept after the call, so that a new target costs O(p) for its
 * far field instead of a new FMM). For each point t (x_dev[i], y_dev[i]) of leaf b (located as
 * vfmm_leaf_interpolate locates it): u, u_x, u_y = the far field of b's local expansion and of the
 * multipoles of b's W list at t, plus the near field of every leaf of b's U list, integrated
 * against f~ at t itself by on-the-fly quadrature (tanh-sinh rules on triangles with apex at the
 * source box's point nearest to t). At a leaf node it gives the solve's value there; elsewhere it is
 * V f~(t), not the interpolant v~. Reads the expansions a vfmm_volume_potential call with nrhs = 1
 * and the same tree, ops and f_dev ([n_leaves][k*k]) left in workspace_dev (workspace_bytes as
 * given to that call), so it must follow that call on the same stream and precede any other use of
 * the workspace. Points outside the closed root box or with a NaN coordinate get NaN. FP64;
 * stream-ordered, no allocation. Errors: INVALID_ARG (null pointers, n_points < 0 or > 2^31 - 1,
 * k differs), WORKSPACE (smaller than a one-right-hand-side workspace), CUDA. */
int vfmm_evaluate_points(const vfmm_tree* tree, const vfmm_ops* ops, const double* f_dev, const void* workspace_dev,
                         size_t workspace_bytes, int64_t n_points, const double* x_dev, const double* y_dev,
                         double* u_dev, double* ux_dev, double* uy_dev, void* stream);

/* Allocation-free solve. The paper has no counterpart: this entry point exists for
 * callers that cannot allocate device memory, such as hosts whose device memory is
 * owned entirely by their own pool allocator (so neither a workspace buffer nor a
 * cudaMalloc is available to this library). It runs vfmm_volume_potential with its
 * workspace in a fixed 32 MiB static device array that every GPU loading the library
 * holds until the process exits, and never calls cudaMalloc or cudaFree.
 *  - Size limit: trees whose vfmm_workspace_size (nrhs = 1, with_io = 0) exceeds 32 MiB
 *    are rejected with VFMM_ERR_WORKSPACE (roughly a few hundred leaves at k = 8).
 *  - Right-hand sides are solved one after another in the same scratch (the mixed form
 *    does not fold them here, since that would build new schedules in device memory),
 *    every launch on `stream` (no second stream is created).
 *  - Set-up: the first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call before
 *    any stream capture.
 *  - Sharing: all calls on a device use the same array, which keeps the last call's
 *    contents; calls that overlap on the GPU (different streams, or concurrent host
 *    threads) race with each other and must be serialised by the caller.
 *  - Status: each call clears the array's status word once and every right-hand side's
 *    solve adds to it; vfmm_workspace_status(NULL) reads it after `stream` is synchronised.
 * Inputs and outputs are as for vfmm_volume_potential. */
int vfmm_volume_potential_noalloc(const vfmm_tree* tree, const vfmm_ops* ops, const double* f_dev, int32_t nrhs,
                                  double* u_dev, double* ux_dev, double* uy_dev, void* stream);

/* CUDA-graph form of vfmm_volume_potential for repeated solves with the same buffers: the
 * solve (all its kernels, copies and memsets) is captured once on `stream` into an executable
 * graph; each launch replays it, reading f_dev and writing u_dev, ux_dev, uy_dev, using the
 * workspace given at creation. The buffers must stay allocated for the graph's lifetime.
 * Creation runs one ordinary solve first (so one-time kernel attributes are set outside the
 * capture), then captures; it synchronises `stream`. Errors as vfmm_volume_potential. */
typedef struct vfmm_graph vfmm_graph;
int vfmm_graph_create(const vfmm_tree* tree, const vfmm_ops* ops, const double* f_dev, int32_t nrhs, double* u_dev,
                      double* ux_dev, double* uy_dev, void* workspace_dev, size_t workspace_bytes, void* stream,
                      vfmm_graph** out);
int vfmm_graph_launch(const vfmm_graph* graph, void* stream);
int vfmm_graph_destroy(vfmm_graph* graph);

/* ---------------------------------------------------------------- batches of problems
 * Many independent solves in one stream-ordered call (no counterpart in the paper, which
 * solves one problem at a time). Each item is exactly one vfmm_volume_potential call:
 * its own tree, operator set (shared between items is fine: read-only), nrhs, device
 * buffers f/u/u_x/u_y laid out as for vfmm_volume_potential, and its own workspace (sized
 * by vfmm_workspace_size; two items never share a workspace, since they may run at the
 * same time). Buffers stay owned by the caller.
 *
 * A batch handle owns `n_streams` side streams (1..VFMM_BATCH_MAX_STREAMS) and events. A
 * call forks the active side streams from `stream`, deals the items to them by estimated
 * work (longest first, to the least loaded stream), and joins them back into `stream`, so
 * the batch is ordered like one kernel on `stream` and independent items overlap on the
 * GPU. Each item runs on its side stream alone (no further fork inside an item). One handle serves one host thread at a time. Errors: INVALID_ARG (null handle,
 * item without tree or ops), and every error of vfmm_volume_potential (the first one
 * stops the launches; streams are still joined). */
#define VFMM_BATCH_MAX_STREAMS 64
typedef struct vfmm_batch vfmm_batch;
typedef struct {
    const vfmm_tree* tree;
    const vfmm_ops* ops;
    int32_t nrhs;
    const double* f;  /* device, [nrhs][n_leaves][k*k] */
    double* u;        /* device, same layout */
    double* ux;
    double* uy;
    void* workspace;  /* device, >= vfmm_workspace_size(tree, ops, nrhs, 0) bytes */
    size_t workspace_bytes;
} vfmm_batch_item;
int vfmm_batch_create(int32_t n_streams, vfmm_batch** out);
int vfmm_batch_destroy(vfmm_batch* batch);
int vfmm_batch_potential(vfmm_batch* batch, int32_t n, const vfmm_batch_item* items, void* stream);
/* The whole batch captured as one CUDA graph (replayed with vfmm_graph_launch, freed with
 * vfmm_graph_destroy); runs the batch once before capturing and synchronises `stream`,
 * which must not be the default stream. Item buffers must outlive the graph. */
int vfmm_batch_graph_create(vfmm_batch* batch, int32_t n, const vfmm_batch_item* items, void* stream,
                            vfmm_graph** out);
/* Schedule autotuner: captures the batch with 1, 2, 4, ... (up to n_streams) side streams,
 * times three graph replays of each with CUDA events on `stream`, keeps the fastest count
 * as the handle's active one and returns it with its mean time in milliseconds. */
int vfmm_batch_tune(vfmm_batch* batch, int32_t n, const vfmm_batch_item* items, void* stream,
                    int32_t* best_streams, float* best_ms);
int vfmm_batch_streams(const vfmm_batch* batch, int32_t* active);

/* Failure-path self-test (no counterpart in the paper). Every wait inside the tensor-core kernels
 * is bounded; when one runs out the kernel records an error word and returns, and the call
 * reports VFMM_ERR_TIMEOUT instead of hanging. This call exercises that path without any fault:
 * a one-warp kernel waits, through the same bounded wait, on an mbarrier that nothing arrives on,
 * gives up after `polls` polls (1..2^20) and records the word, which is read back as a solve does.
 * Returns VFMM_ERR_TIMEOUT (the expected outcome; the context stays usable), INVALID_ARG for a
 * bad `polls`, INTERNAL if the wait completed, CUDA on a CUDA error. Synchronises `stream`. */
int vfmm_selftest_wait_timeout(int64_t polls, void* stream);

/* Schedule autotuner (no counterpart in the paper): for the VFMM_MIXED form, times each small
 * split contraction of this tree and nrhs (near field, M2L, S2L, leaf far field: those with fewer
 * CTAs than two per SM) with split-K factors 1, 2, 4, 8, 16 on the caller's data, and where the
 * schedule holds both forms of a contraction (targets grouped, or one column per list entry with
 * a per-target sum) times both; keeps the fastest in the tree's schedule (used by every later
 * call with this nrhs) and returns the split-K factors in splits[4] (near, M2L, S2L, far; may be
 * NULL; 1 for the entry-major form, see vfmm_solve_work out[7]). Where the near field runs as one
 * persistent CTA per SM and the tree passes are persistent, it then times the whole forked solve
 * (near field beside the main chain, as vfmm_volume_potential and its graphs run it) with the near
 * field capped at 8/8, 7/8, 6/8, 5/8 and 4/8 of the SMs and the tree passes' grids capped to the SMs left
 * free, and keeps the fastest (out[8], out[9] of vfmm_solve_work). Runs two ordinary solves around the timing, so
 * u, u_x, u_y hold the solution afterwards; synchronises `stream`. Must not overlap other calls
 * on the same tree; graphs captured earlier keep the schedule they captured. No-op (splits = 1)
 * for VFMM_FP64. Errors as vfmm_volume_potential. */
int vfmm_tune(const vfmm_tree* tree, const vfmm_ops* ops, const double* f_dev, int32_t nrhs, double* u_dev,
              double* ux_dev, double* uy_dev, void* workspace_dev, size_t workspace_bytes, void* stream,
              int32_t* splits);

/* Work accounting for roofline reports, for a call with nrhs right-hand sides: out[VFMM_N_WORK] =
 * [0] BF16 tensor-core FLOPs the near-field contraction issues per call (VFMM_MIXED: every
 *     slice product of every tile at the operator set's slice counts, zero-padded rows included;
 *     0 for VFMM_FP64),
 * [1] the same for M2L, [2] for the leaf far field (L2T + M2T), [3] for S2L, [4] for S2M,
 * [5] FP64-equivalent FLOPs of the near field, 2 * 3k^2 * k^2 per U-list entry and right-hand side,
 * [6] number of U-list entries, [7] which contractions run in the entry-major form (one column
 *     per list entry, summed per target afterwards): bit 0 near field, 1 M2L, 2 leaf far field,
 *     3 S2L, [8] the near-field contraction's CTA cap (0: one CTA per work item), [9] the grid cap of
 *     the persistent tree passes (0: one CTA per box of the widest level, at most one per SM).
 *     Host-only; no device work. */
#define VFMM_N_WORK 10
int vfmm_solve_work(const vfmm_tree* tree, const vfmm_ops* ops, int32_t nrhs, double* out);

/* Co-schedule of a VFMM_MIXED solve with nrhs right-hand sides on this tree (no counterpart in the
 * paper): near_ctas caps the near-field contraction's grid (0: one CTA per work item; a positive
 * cap makes its CTAs persistent, each walking several work items), pass_ctas caps the grid of the
 * persistent tree passes (0: one CTA per box of the widest level, at most one per SM). vfmm_tune
 * picks both by timing the forked solve; these calls read or override its choice (results do not
 * depend on either: every work item is computed the same way whichever CTA takes it). The set call
 * applies to later calls and graph captures; not while a solve on this tree is being launched.
 * Host-only. Errors: INVALID_ARG (null pointers, nrhs < 1, a negative cap). */
int vfmm_schedule_get(const vfmm_tree* tree, int32_t nrhs, int32_t* near_ctas, int32_t* pass_ctas);
int vfmm_schedule_set(vfmm_tree* tree, int32_t nrhs, int32_t near_ctas, int32_t pass_ctas);

/* Stage timers (tracing): the same solve as vfmm_volume_potential with CUDA events
 * recorded on `stream` between its stages; synchronises `stream` and returns the
 * elapsed milliseconds of each stage summed over the right-hand sides
 * (stage_ms[VFMM_N_STAGES]: S2M, M2M, DOWN (M2L + S2L + L2L), NEAR, L2T, LEAF, then for
 * VFMM_MIXED the split tensor-core contractions alone (each with its partial-sum reduction):
 * NEAR_TC, S2M_TC, M2L_TC, S2L_TC, FAR_TC; these five are 0 for VFMM_FP64) and the number of
 * kernels the solve launched (*launches). */
#define VFMM_N_STAGES 11
int vfmm_volume_potential_profiled(const vfmm_tree* tree, const vfmm_ops* ops, const double* f_dev, int32_t nrhs,
                                   double* u_dev, double* ux_dev, double* uy_dev, void* workspace_dev,
                                   size_t workspace_bytes, void* stream, float* stage_ms, int32_t* launches);

const char* vfmm_strerror(int code);
const char* vfmm_last_error_detail(void);

#ifdef __cplusplus
}
#endif

#endif /* VFMM_H */
