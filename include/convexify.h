/*
 * convexify.h -- C ABI of the GB300 per-point rank-one convexification library
 * (libconvexify.so).
 *
 * Method: Balzani, Koehler, Neumeier, Peter, Peterseim, "Multidimensional
 * rank-one convexification of incremental damage models at finite strains"
 * (arXiv 2211.14318).  For every quadrature point F in R^{2x2} with history
 * beta_k, the incremental stress potential W (Eq. 2.9) is sampled along rank-one
 * lines F + t a (x) b (Eq. 4.4, restated per point), each line is convexified
 * (Algorithm 1) and read at t = 0, the minimum over directions is taken
 * (Eq. 4.3), and the split is recursed to the lamination depth K (Eq. 3.3).
 * W^R and P = dW^R/dF are evaluated over the resulting lamination tree
 * (Eq. 5.2, Algorithm 3).
 *
 * Conventions
 *  - Every function returns an int status: CVX_OK (0) or a negative CVX_ERR_*.
 *    cvx_last_error() returns the message of the calling thread's last error.
 *    No C++ exception crosses this boundary.
 *  - F is row-major (F11, F12, F21, F22).  All array arguments of the compute
 *    calls are caller-owned DEVICE pointers unless stated otherwise; the caller
 *    keeps them alive until the stream has reached the end of the call.
 *  - Calls are asynchronous on the given stream (NULL = legacy default stream),
 *    except where marked "synchronous".  Arguments are validated (parameters
 *    first, then the handle and pointers) before anything is enqueued or any
 *    CUDA call is made.  Kernel faults surface as
 *    CVX_ERR_CUDA from this or a later call.
 *  - The library owns the handle's workspace (grown on demand with cudaMalloc)
 *    and its direction tables.  A handle may be used by one host thread at a
 *    time; work of one handle is serialised on the streams it is given.
 *  - Arithmetic: every line is first sampled in FP32 on the CUDA cores, and
 *    that pass bounds the value at t = 0 of its lower hull from below and
 *    above (rigorously, for the FP32 samples).  It screens the directions:
 *    only those whose lower bound lies within a tolerance of the best upper
 *    bound (several times the FP32 sampling error) are resampled in FP64, and
 *    the node's direction, split and value are decided on those FP64
 *    samples.  Split points, W^R and P are evaluated in FP64.
 */
#ifndef CONVEXIFY_H
#define CONVEXIFY_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status */
enum cvx_error {
    CVX_OK = 0,
    CVX_ERR_INVALID_ARG = -1, /* argument out of range, NULL where required     */
    CVX_ERR_CUDA = -2,        /* CUDA runtime error (message has the CUDA text) */
    CVX_ERR_OOM = -3,         /* workspace allocation failed                    */
    CVX_ERR_TIMEOUT = -4,     /* a bounded device-side wait gave up             */
    CVX_ERR_NOT_TRAINED = -5, /* surrogate used before training or loading      */
    CVX_ERR_UNSUPPORTED = -6  /* configuration not built into this library      */
};

/* per-point status bits (int32 per point) */
enum cvx_point_status {
    CVX_PT_OK = 0,
    CVX_PT_NONPOS_DET = 1, /* det F <= 0: W^R and P are NaN, no tree          */
    CVX_PT_TIE = 2,        /* some node's two best directions were closer than
                              the FP32 sampling error bound (warning only)     */
    CVX_PT_EDGE = 4,       /* some split point lies on the end of its line     */
    CVX_PT_ITER_CAP = 8,   /* a hull search hit its iteration cap (warning)    */
    CVX_PT_OVERFLOW = 16,  /* the decision at some node is not certified
                              against every direction (warning)               */
    CVX_PT_FALLBACK = 32   /* surrogate_propose: some node fell back to the
                              full scan                                       */
};

/* energy kinds */
enum cvx_energy_kind {
    CVX_ENERGY_NH_DAMAGE = 0,  /* plane-strain Neo-Hooke with exponential damage,
                                  Eqs. (2.3)-(2.9)                              */
    CVX_ENERGY_DOUBLE_WELL = 1, /* test energy (F11^2-1)^2 + F12^2 + F21^2 +
                                  (F22-1)^2, closed-form envelope; not in the
                                  paper                                         */
    CVX_ENERGY_STVK_DAMAGE = 2 /* St. Venant-Kirchhoff, Eq. (2.2), with the
                                  damage of Eqs. (2.4)-(2.9); the global-grid
                                  calls only (CVX_ERR_UNSUPPORTED elsewhere)    */
};

typedef struct cvx_handle cvx_handle;
typedef struct CUstream_st *cvx_stream; /* same object as cudaStream_t */

/* Problem parameters.  Material of Sec. 2 (mu, lambda, D_inf, D_0 of Eq. 2.6).
 * Directions: the angle grid a_i = (cos pi i/Na, sin pi i/Na), b_j likewise,
 * direction index j_dir = i * Nb + j (a discrete subset of the rank-one cone
 * of Sec. 4.1); or, if dirs != NULL, n_dirs custom (a1, a2, b1, b2) rows
 * (HOST pointer, copied), e.g. the reduced set R^1_1 of Eq. (5.1).
 * Line: L = line_points samples t_m = (m - m0) h, m0 = (L-1)/2,
 * h = 2 t_half / (L-1), so t = 0 (the point itself) is sampled exactly;
 * samples with det(F + t R) <= 0 are excluded.  depth = K, 0 <= K <= 8. */
typedef struct cvx_params {
    double mu;
    double lambda_L;
    double D_inf;
    double D0;
    double t_half;
    const double *dirs; /* host, n_dirs x 4, or NULL for the angle grid */
    int32_t energy;     /* enum cvx_energy_kind                          */
    int32_t n_theta_a;
    int32_t n_theta_b;
    int32_t n_dirs;
    int32_t line_points; /* odd, 3 <= L <= 2079                          */
    int32_t depth;
    int32_t flags; /* CVX_FLAG_* bits (0: the plain grid method)        */
    int32_t recentre; /* surrogate_propose: re-centrings of a proposal window
                         whose best direction lies on its border, 0..8
                         (0: none); ignored by the other calls          */
} cvx_params;

/* cvx_params.flags.
 * CVX_FLAG_REFINE_NEWTON: after a node's split is decided on the grid, refine
 * its ends t-, t+ by FP64 Newton on the common-tangent conditions
 * g'(t-) = g'(t+) = (g(t+) - g(t-)) / (t+ - t-), g(t) = W(F + t R*), seeded by
 * the grid bridge, at most 8 iterations.  The refinement is kept only if it
 * converged with both ends inside the line window and its chord value at 0 is
 * not above the grid bridge's; the node is then flagged CVX_NODE_NEWTON and
 * its children, xi and h use the refined ends.  The paper takes laminates from
 * its grids only; this is an addition (the direction is still the grid's). */
/* CVX_FLAG_GAP_ONE_SIDED (surrogate_propose only): the energy-gap fallback
 * test becomes (V - E_pred) / (1e-8 + |V|) > gap_tol, i.e. a node falls back
 * only when the proposed laminate is better than what its window found. */
/* CVX_FLAG_MIRROR_WINDOW (surrogate_propose only): mirror window.  An
 * isotropic W (Sec. 2: W depends on F through I1 and J) takes the same values
 * on the line F + t a(x)b and on its reflection F + t (M1 a)(x)(M2 b), M1 and
 * M2 the reflections about the principal axes of F (F = Q1 S Q2^T,
 * M = Q diag(1, -1) Q^T, M1 F M2 = F), so the node value over the angles has
 * mirrored twin basins of nearly equal value on the grid.  A node whose window
 * split along d is scanned once more in a window of half-width (w + 1) / 2
 * around the grid cell of the mirror of d (theta_a -> 2 phi1 - theta_a,
 * theta_b -> 2 phi2 - theta_b, phi the principal angles), with the same
 * re-centring; it takes the lower of the two values (the lower direction index
 * on equal values) and falls back to the full scan if the mirror window's best
 * direction still lies on its border.  Skipped when the mirror window lies
 * inside the node's last window. */
/* CVX_FLAG_WINDOW_DOUBLINGS(n), n = 1..8 (convexify_points and
 * convexify_batch): adaptive line window.  Sec. 4.1 asks for a radius
 * "sufficiently large"; a node whose split has an end on the end of its line
 * (CVX_NODE_EDGE) is scanned again with the line window doubled (t_half 2^e,
 * the same L), at most n doublings; the node's children start from its
 * window, and cvx_node.window_exp records e.  0 (the default): the window is
 * t_half for every node. */
enum cvx_param_flags {
    CVX_FLAG_REFINE_NEWTON = 1,
    CVX_FLAG_GAP_ONE_SIDED = 2,
    CVX_FLAG_MIRROR_WINDOW = 4
};
#define CVX_FLAG_WINDOW_DOUBLINGS(n) ((int32_t)(n) << 8)
#define CVX_WINDOW_DOUBLINGS_OF(flags) (((flags) >> 8) & 15)

/* Node of the per-point lamination tree (Sec. 4.3, Algorithm 2), heap layout:
 * node i has children 2i+1 (F-) and 2i+2 (F+); 2^{K+1}-1 nodes per point. */
typedef struct cvx_node {
    double F[4];     /* deformation gradient of this node                     */
    double w;        /* W(F), FP64                                            */
    double h;        /* node value: FP64 bridge value at t = 0 along the chosen
                        direction (the refined chord value if CVX_NODE_NEWTON);
                        W(F) if the node does not split                       */
    double xi;       /* weight of F+ in this node's split, (m0-m-)/(m+-m-)
                        (-t-/(t+ - t-) with the refined ends)                 */
    double weight;   /* product of split weights from the root                */
    int32_t dir;     /* chosen direction index, -1 if the node was not scanned */
    int32_t m_minus; /* sample index of F- on the chosen line (0..L-1)         */
    int32_t m_plus;  /* sample index of F+                                     */
    int32_t flags;   /* CVX_NODE_* bits                                        */
    float gap;       /* gap between the two best directions' FP64 hull values,
                        rounded to FP32; where the second best was not
                        resampled in FP64 (its FP32 screen bound already lay
                        above the best), a lower bound of that gap           */
    int32_t window_exp; /* the node's line window is t_half 2^window_exp       */
} cvx_node;

enum cvx_node_flags {
    CVX_NODE_EXISTS = 1,
    CVX_NODE_SCANNED = 2,
    CVX_NODE_LAMINATED = 4,
    CVX_NODE_LEAF = 8,
    CVX_NODE_TIE = 16,
    CVX_NODE_EDGE = 32,
    CVX_NODE_ITER_CAP = 64,  /* a hull search hit its iteration cap          */
    CVX_NODE_OVERFLOW = 128, /* decision not certified against every direction */
    CVX_NODE_NEWTON = 256,   /* split refined by CVX_FLAG_REFINE_NEWTON        */
    CVX_NODE_FALLBACK = 512  /* surrogate_propose: decided by the full scan     */
};

/* Root laminate of a point: direction a (x) b = dirs[dir], volume fraction xi
 * of F+, and F+- (Fig. fig:RankOneConvexification1D). */
typedef struct cvx_laminate {
    int32_t laminated; /* 0: the point is rank-one convex on its lines */
    int32_t dir;
    int32_t m_minus;
    int32_t m_plus;
    double xi;
    double h;
    double F_plus[4];
    double F_minus[4];
} cvx_laminate;

/* Counters accumulated on the device over all calls since the last reset. */
typedef struct cvx_stats {
    int64_t points;         /* points convexified                          */
    int64_t nodes_scanned;  /* tree nodes whose lines were scanned         */
    int64_t lines;          /* (node, direction) lines sampled             */
    int64_t valid_samples;  /* samples with det > 0 (algorithmic work)     */
    int64_t laminated;      /* nodes that split                            */
    int64_t fp64_checks;    /* FP64 spot samples of the refinement certificates */
    int64_t full_passes;    /* full-line argmin passes of the hull search  */
    int64_t rare_paths;     /* hull searches that left the fast path       */
    int64_t ties;           /* nodes flagged CVX_NODE_TIE                  */
    int64_t iter_caps;      /* hull searches that hit the iteration cap    */
    int64_t window_steps;   /* supporting-slope steps inside the windows   */
    int64_t rounds;         /* verification rounds of the hull searches    */
    int64_t fp64_window;    /* FP64 fallbacks in the window checks         */
    int64_t fp64_rare;      /* FP64 fallbacks on the rare path             */
    int64_t fp64_center;    /* FP64 fallbacks deciding the centre          */
    int64_t refined;        /* candidate lines resampled and decided in FP64 */
    int64_t overflow;       /* nodes with more screened candidates than kept */
    int64_t window_nodes;   /* surrogate_propose: nodes scanned in a window */
    int64_t fallbacks;      /* ... of which deferred to the full scan       */
    int64_t refine_full;    /* FP64 refinements that resampled the whole line
                               (the windowed FP64 bridge was not certified) */
    int64_t lines_bounded;  /* lines excluded by their sampling-pass bound,
                               without a hull search                        */
    int64_t lines_flat;     /* lines whose sampling-pass bound is within the
                               FP32 sample error of the centre value: no
                               hull search, the bound is their lower bound  */
    int64_t recentred;      /* surrogate_propose: window re-centrings        */
    int64_t lines_certified; /* lines certified not to split their node (the
                               tangent line at the centre supports every
                               sample): no FP64 refinement needed           */
    int64_t edge_splits;    /* splits with an end on the end of its line
                               (CVX_NODE_EDGE): the laminate is limited by the
                               line window t_half (Sec. 4.1 asks for a radius
                               "sufficiently large")                        */
    int64_t window_doublings; /* nodes rescanned with a doubled line window
                               (CVX_FLAG_WINDOW_DOUBLINGS)                  */
    int64_t mirror_windows; /* surrogate_propose: nodes scanned in a mirror
                               window (CVX_FLAG_MIRROR_WINDOW)              */
    int64_t mirror_won;     /* ... whose mirror window held the lower value  */
} cvx_stats;

/* ----------------------------------------------------------------- handles */

/* Creates a handle bound to CUDA device `device` (the calling thread's current
 * device is left unchanged).  Synchronous.  Errors: INVALID_ARG, CUDA. */
int cvx_create(cvx_handle **out, int device);

/* Frees the handle's workspace and tables.  Synchronous (waits for the
 * device).  NULL is accepted. */
int cvx_destroy(cvx_handle *h);

/* Copies the calling thread's last error message (NUL-terminated, truncated
 * to len) into buf.  Returns the length of the full message. */
int cvx_last_error(char *buf, size_t len);

/* Reads (synchronous: waits for the handle's device) and optionally resets
 * the counters. */
int cvx_get_stats(cvx_handle *h, cvx_stats *out, int reset);

/* Enables (1) or disables (0) CUDA-event timing of every line-scan kernel
 * launch (events recorded on the launching stream around each launch). */
int cvx_set_profiling(cvx_handle *h, int enable);

/* Synchronous: total device time in ms and number of line-scan kernel launches
 * timed since the last reset (requires cvx_set_profiling(h, 1)). */
int cvx_get_scan_timing(cvx_handle *h, double *ms, int64_t *launches, int reset);

/* sizeof of the ABI structs, for bindings to check their layouts:
 * which = 0 cvx_params, 1 cvx_node, 2 cvx_laminate, 3 cvx_stats, 4 cvx_problem,
 * 5 cvx_grid; -1 otherwise. */
int cvx_struct_size(int which);

/* Sets the launch shape of the line-scan kernel of convexify_points: warps per
 * CTA (1..8) and directions per work item (>= 1; 0 = automatic).  For the
 * damage energy the line scan runs one line per lane (the environment
 * variable CVX_SCAN_KERNEL=warp selects the warp-per-line scan instead); it
 * ignores warps_per_cta and caps the directions per item at 256.
 * convexify_batch chooses its own (see cvx_get_batch_tuning). */
int cvx_set_tuning(cvx_handle *h, int warps_per_cta, int dirs_per_item);

/* ----------------------------------------------------- steps of the method */

/* W(F) and P = dW/dF in FP64 at n points (Eqs. 2.9, 2.12), plane strain.
 * F: n x 4, beta_k: n, W: n, P: n x 4 (P may be NULL).  det F <= 0 gives NaN. */
int cvx_energy(cvx_handle *h, const cvx_params *p, int64_t n, const double *F,
               const double *beta_k, double *W, double *P, cvx_stream s);

/* History update between load steps, Eq. (2.5): beta_out = max(beta_in,
 * psi0(F)).  beta_in may be NULL (treated as 0); beta_out may alias beta_in. */
int cvx_history_update(cvx_handle *h, const cvx_params *p, int64_t n, const double *F,
                       const double *beta_in, double *beta_out, cvx_stream s);

/* FP32 samples of W along n_lines lines F_i + t a (x) b with direction
 * dir_i (Eq. 4.4 per point): w is n_lines x L, NaN where det <= 0.
 * F: n_lines x 4, beta_k: n_lines, dir: n_lines (int32).  The same samples
 * the convexification kernel computes. */
int cvx_sample_lines(cvx_handle *h, const cvx_params *p, int64_t n_lines, const double *F,
                     const double *beta_k, const int32_t *dir, float *w, cvx_stream s);

/* Lower hull (Algorithm 1) of n_lines given FP32 lines of L samples at the
 * integer abscissae m - m0 (NaN = excluded; the non-NaN samples must be
 * contiguous and include m0), read at x = 0: bridge vertices m_minus <= m0 <=
 * m_plus (both m0 if m0 is a strict vertex) and the value h in FP64.
 * Exact: the result is the hull of the FP32 values.  3 <= L <= 2079, odd. */
int cvx_hull_bridge(cvx_handle *h, int64_t n_lines, int32_t L, const float *w,
                    int32_t *m_minus, int32_t *m_plus, double *hval, cvx_stream s);

/* --------------------------------------------------------- the hot path */

/* Per-point rank-one convexification of n points (Sec. 4-5):
 *   W_R (n), P (n x 4)            relaxed energy and stress, FP64;
 *   status (n)                    CVX_PT_* bits;
 *   root (n, nullable)            root laminate;
 *   tree (n x (2^{K+1}-1), nullable) full lamination tree.
 * Workspace: the handle's (grown with cudaMalloc when needed). */
int convexify_points(cvx_handle *h, const cvx_params *p, int64_t n, const double *F,
                     const double *beta_k, double *W_R, double *P, cvx_laminate *root,
                     cvx_node *tree, int32_t *status, cvx_stream s);

/* Tangent of the relaxed energy over lamination trees (the tree output of
 * convexify_points or surrogate_propose with the same parameters): with the
 * laminates held fixed, Eq. (5.2) differentiated once more, i.e. Algorithm 3
 * evaluating the second derivative at the leaves,
 *   A = sum over the leaves of (product of split weights) d^2W/dFdF(F_leaf),
 * d^2W/dFdF from Eq. (2.12) in FP64.  A is n x 16 (DEVICE), row-major
 * A[16 p + 4 a + b] = dP_a / dF_b over the row-major entries of F; NaN for a
 * point whose root does not exist or has det F <= 0.  beta_k (n) and tree
 * (n x (2^{K+1}-1), K = p->depth) are DEVICE arrays.  Asynchronous. */
int cvx_tree_tangent(cvx_handle *h, const cvx_params *p, int64_t n, const double *beta_k,
                     const cvx_node *tree, double *A, cvx_stream s);

/* --------------------------------------------------------- global-grid form */

/* The paper's own algorithm (Secs. 4.1-4.3, 5.1-5.3): W is stored on a grid of
 * deformation gradients and Eq. (4.3) is iterated on the whole grid,
 *   W^{k+1}(F) = min( W^k(F), min_R hull_l[ W^k(F + l R) ](0) ),
 * where the inner term is Algorithm 1's lower hull of the values of W^k at the
 * grid points of the line through F, read at F.  The lamination forest records
 * per iteration and grid point the winning laminate; Algorithm 2 builds the
 * tree of an arbitrary F from it (multilinear-interpolation corners where F is
 * not a grid point, Sec. 5.3) and Algorithm 3 evaluates W and P over it.
 * Both the two-dimensional studies (F in R^{2x2}, plane strain, Sec. 6.1) and
 * the nine-dimensional one (F in R^{3x3}, Sec. 6.8) are covered.
 *
 * Grid (Sec. 5.2, the cuboid form): dim = d = 2 or 3; the D = d^2 components
 * of F (row-major: F11, F12, ...) take the values lo[c] + i delta[c],
 * i = 0 .. n[c] - 1; flat index with the last component fastest;
 * 1 <= n[c] <= 512, at most 2^31 - 1 points.  Entries c >= D are ignored.
 *
 * Directions are grid-index offsets o (nd x D int32, HOST): one step of a line
 * moves component c by o[c] grid steps, i.e. F + l R with R_c = o[c] delta[c]
 * (the matrix a (x) b of Eq. 5.1 scaled by delta when all delta[c] are equal,
 * as in the studies of Secs. 6.1 and 6.8).  Every offset must be nonzero and
 * rank-one as a d x d matrix, |o[c]| <= 512, 1 <= nd <= 4096.  cvx_grid_r11
 * writes the directions of Eq. (5.1) in the order used by the ties rule below.
 *
 * Lines are the maximal runs of grid points F + l R inside the grid.  Values
 * that are not finite (excluded by det_rule) are left out of the hulls and
 * keep their value.  A point laminates along the lowest direction index whose
 * hull value is strictly below both W^k(F) and every lower-indexed
 * direction's; its record is (dir, l-, l+) with l- < 0 < l+ the hull vertices
 * around it in line steps, and F+- = F + l+- R with weight xi = -l-/(l+ - l-)
 * of F+ (Algorithm 2's |F - F-|_1 / |F+ - F-|_1); (-1, 0, 0) if it does not.
 * Hull predicates and chord values are FP64 with every operation rounded on
 * its own, so a step is reproducible bit for bit.
 *
 * Energy: the material of p (mu, lambda_L, D_inf, D0; energy NH_DAMAGE,
 * STVK_DAMAGE, or DOUBLE_WELL for dim = 2; the line fields are not used).
 * det_rule (what det F <= 0 means, the readings of the studies of Sec. 6.1):
 * 0 = excluded (NaN), as on the per-point path; 1 = kept: the Neo-Hooke term
 * takes ln|det F| (det F < 0 mirrors det F > 0; det F = 0 stays excluded) and
 * Eq. (2.2), a polynomial in F, is kept everywhere. */
typedef struct cvx_grid {
    int32_t dim;
    int32_t n[9];
    double lo[9];
    double delta[9];
} cvx_grid;

/* The reduced direction set R^1_1 of Eq. (5.1) as grid-index offsets, one of
 * each pair +-a (x) b (the sign gives the same line), row-major a_i b_j.
 * dim = 2: a, b over (1,0), (0,1), (1,1), (1,-1); row 4 ia + ib; off is
 * 16 x 4.  dim = 3: a, b over the 13 vectors of {-1,0,1}^3 whose first
 * nonzero entry is +1, in the order (1,0,0), (0,1,0), (0,0,1), (1,1,0),
 * (1,-1,0), (1,0,1), (1,0,-1), (0,1,1), (0,1,-1), (1,1,1), (1,1,-1), (1,-1,1),
 * (1,-1,-1); row 13 ia + ib; off is 169 x 9.  off: HOST. */
int cvx_grid_r11(int32_t dim, int32_t *off);

/* W^0 on the grid: W (DEVICE, N values in flat order) = the energy at every
 * grid point with history beta_k. */
int cvx_grid_energy(cvx_handle *h, const cvx_params *p, const cvx_grid *g, double beta_k,
                    int32_t det_rule, double *W, cvx_stream s);

/* One iteration of Eq. (4.3): W_out from W_in (DEVICE, N each, no aliasing);
 * lam (DEVICE, N x 3 int32, nullable) = the laminate records; dec (DEVICE
 * scalar, nullable) = the largest decrease W_in - W_out over the points where
 * both are finite.  Workspace: the handle's (12 bytes per point and
 * direction, in chunks of at most 1 GB, plus the line starts). */
int cvx_grid_step(cvx_handle *h, const cvx_grid *g, int32_t nd, const int32_t *off,
                  const double *W_in, double *W_out, int32_t *lam, double *dec, cvx_stream s);

/* The global iteration (Sec. 4.1): W^0 = cvx_grid_energy, then Eq. (4.3) until
 * the largest decrease of a step is at most tol or kmax steps were taken
 * (1 <= kmax <= 64; the studies of Sec. 6 use tol = 1e-4, kmax = 20).  The
 * stop is decided on the device: nothing waits on the host, and the steps
 * after the stop return at once.  Outputs (DEVICE): W (N) = W^K; iters (one
 * int32) = K; forest (kmax x N x 3 int32, nullable) = the records of step k at
 * forest + 3 N k (rows k >= K are not written); decs (kmax, nullable) = the
 * largest decrease of each step (0 after the stop). */
int cvx_grid_convexify(cvx_handle *h, const cvx_params *p, const cvx_grid *g, double beta_k,
                       int32_t det_rule, int32_t nd, const int32_t *off, int32_t kmax, double tol,
                       double *W, int32_t *forest, double *decs, int32_t *iters, cvx_stream s);

/* Relaxed energy and stress at n arbitrary points F (DEVICE, n x D) after K
 * iterations (WK = W^K, forest = K x N x 3 records, both DEVICE):
 *   W_interp (n): the multilinear interpolation of W^K (Sec. 4.1, values off
 *     the grid by interpolation);
 *   W_tree (n), P (n x D): Algorithm 3 over Algorithm 2's tree: the cell
 *     corners of F (up to 2^D) with their interpolation weights (one corner if
 *     F is a grid point; coordinates within 1e-12 grid steps of a grid value
 *     count as on it) at order K, each expanded through the latest iteration
 *     k <= order that split it (children at order k - 1), W and P (Eq. 2.12)
 *     at the leaves;
 *   A (n x D x D, nullable): the tangent d^2W/dFdF over the same tree
 *     (Algorithm 3's third output; A[D^2 q + D a + b] = dP_a / dF_b);
 *   leaves (n int64, nullable): the leaves of the tree.
 * NaN (leaves 0) outside the grid.  nd and off must be those of the run that
 * made the forest.  0 <= K <= 64.  The trees are tabulated per grid point and
 * order first (K sweeps over the grid); workspace: three tables of W, P,
 * (A,) leaf count per grid point ((D + 2) 8 bytes per point, D^2 8 more with
 * A). */
int cvx_grid_query(cvx_handle *h, const cvx_params *p, const cvx_grid *g, double beta_k,
                   int32_t det_rule, int32_t nd, const int32_t *off, int32_t K, const double *WK,
                   const int32_t *forest, int64_t n, const double *F, double *W_interp,
                   double *W_tree, double *P, double *A, int64_t *leaves, cvx_stream s);

/* ------------------------------------------------------------ batched form */

/* One problem of a batch: its own parameters and caller-owned DEVICE arrays
 * (as for convexify_points; root may be NULL). */
typedef struct cvx_problem {
    cvx_params params;
    int64_t n;
    const double *F;       /* n x 4 */
    const double *beta_k;  /* n */
    double *W_R;           /* n */
    double *P;             /* n x 4 */
    int32_t *status;       /* n */
    cvx_laminate *root;    /* n, nullable */
} cvx_problem;

/* Many independent problems (meshes, load steps) of uneven sizes in one run:
 * the points of all problems share the same per-level persistent kernels
 * (work items handed out by an atomic counter, so uneven problems balance),
 * and the whole multi-level run is a CUDA graph.  Results are those of
 * convexify_points on each problem.  All problems must use the same energy
 * kind; n_problems <= 65536; the problems array is a HOST array.
 * The first call with a given set of problems (shapes, parameters and
 * pointers) picks the launch shape with a short timed trial on a sample of the
 * points (the autotuner; result cached in the handle, and in the JSON file
 * named by the environment variable CVX_AUTOTUNE_CACHE if set), captures the
 * graph and launches it; later calls with the same set replay the graph.
 * The first call is therefore synchronous; later calls are asynchronous.
 * The trial runs write their results into the leading points' outputs (later
 * overwritten) and add to the handle's statistics counters.  A later
 * convexify_points call that grows the handle's workspace makes the next
 * batch call capture again. */
int convexify_batch(cvx_handle *h, int n_problems, const cvx_problem *problems, cvx_stream s);

/* The launch shape the autotuner chose for the last batch (0s before any):
 * warps_per_cta 4 or 8 for the warp-per-line scan, 0 for the lane-per-line
 * scan (damage energy); dirs_per_item_cap 0 = no cap. */
int cvx_get_batch_tuning(cvx_handle *h, int *warps_per_cta, int *dirs_per_item_cap,
                         int *from_cache);

/* ------------------------------------------- surrogate proposal network */

/* A small network that proposes, per tree node, where the line scan should
 * look (not in the paper: an addition; the full scan stays the reference and
 * the fallback).  Inputs per node x = (F11, F12, F21, F22, beta_k, ln det F),
 * standardised with a per-feature mean and std; 4 hidden layers of width 256
 * with GELU; 7 outputs: the angles theta_a, theta_b of a (x) b (period pi),
 * the logit of the volume fraction xi of F+, the four entries of the jump
 * F+ - F- (row-major).  Training and inference run on the BF16 tensor cores
 * (tcgen05, FP32 accumulation); the FP32 master weights and Adam state live
 * in the handle.
 *
 * Parameters: one flat FP32 vector of CVX_SURROGATE_PARAMS values,
 *   W0 (256 x 6), b0 (256), W1 (256 x 256), b1, W2, b2, W3, b3,
 *   W4 (7 x 256), b4 (7), weights row-major as (out, in).
 * Labels Y (n x 7): theta_a, theta_b, xi, jump (4); a node that does not
 * split has NaN angles and xi (masked out of the loss) and a zero jump.
 * Loss per sample: sum_i (1 - cos 2 (o_i - theta_i)) over the two angles
 * + (sigmoid(o_2) - xi)^2 + |o_{3..6} - jump|^2, averaged over the batch. */
#define CVX_SURROGATE_PARAMS 200967

typedef struct cvx_train_cfg {
    int32_t epochs; /* passes over the data                                  */
    int32_t batch;  /* samples per Adam step, 16..65536                       */
    float lr;       /* Adam step size (beta1 0.9, beta2 0.999, eps 1e-8)      */
    int32_t init;   /* 1: standardise from X and draw fresh weights from seed */
    uint64_t seed;  /* weight init and shuffling                             */
} cvx_train_cfg;

/* Sets / reads the FP32 weights (HOST arrays) and the input standardisation
 * (mean[6], std[6], std > 0). */
int surrogate_set_weights(cvx_handle *h, const float *params, const float *mean,
                          const float *std);
int surrogate_get_weights(cvx_handle *h, float *params, float *mean, float *std);

/* Raw outputs (n x 7, DEVICE) of DEVICE inputs X (n x 6, unstandardised). */
int surrogate_forward(cvx_handle *h, int64_t n, const float *X, float *out, cvx_stream s);

/* Mean loss (DEVICE scalar) and its gradient (DEVICE, CVX_SURROGATE_PARAMS)
 * over one batch of n <= 2^20 DEVICE samples, with the current weights. */
int surrogate_loss_grad(cvx_handle *h, int64_t n, const float *X, const float *Y, float *loss,
                        float *grad, cvx_stream s);

/* Trains on n DEVICE samples (X n x 6, Y n x 7) with Adam; loss_log (HOST,
 * cfg->epochs values, nullable) receives each epoch's mean batch loss.
 * Synchronous. */
int surrogate_train(cvx_handle *h, int64_t n, const float *X, const float *Y,
                    const cvx_train_cfg *cfg, float *loss_log, cvx_stream s);

/* Training samples from lamination trees (e.g. convexify_points with a tree
 * output, angle-grid directions): one sample per scanned node, X = the node's
 * inputs, Y = (pi i / Na, pi j / Nb) of its direction i Nb + j, its xi and
 * jump F+ - F-; NaN angles and xi, zero jump for a node that does not split.
 * X (n (2^{K+1} - 1) x 6) and Y (... x 7) are DEVICE arrays of that capacity;
 * *count (HOST) receives the number written, in point then heap order.
 * Synchronous. */
int surrogate_labels(cvx_handle *h, const cvx_params *p, int64_t n, const double *beta_k,
                     const cvx_node *tree, float *X, float *Y, int64_t *count, cvx_stream s);

/* The surrogate-proposed form of convexify_points (same arguments and
 * results; angle-grid directions only).  At every tree node the network
 * proposes a direction; its nearest cell (ia, ib) of the Na x Nb grid centres
 * a window of (2 window + 1)^2 directions (indices wrap), and only those lines
 * are scanned.  If the window's best direction lies on its border (and the
 * energy gap test passes), the window is moved to be centred on that
 * direction's cell and scanned again, at most p->recentre times.  The node
 * falls back to the full scan of all Na Nb directions if (i) the window's
 * best direction still lies on its border, or (ii) the energy gap
 * |E_pred - V| / (1e-8 + |V|) exceeds gap_tol, where V is the
 * window's node value and E_pred = xi W(F+) + (1 - xi) W(F-) the proposed
 * laminate evaluated exactly (F+ = F + (1 - xi) amp R, F- = F - xi amp R,
 * R = a (x) b of the proposed angles, amp = jump : R).  fell_back (n, DEVICE,
 * nullable) = 1 where some node of the point fell back (also status bit
 * CVX_PT_FALLBACK; nodes flagged CVX_NODE_FALLBACK).  Requires weights
 * (surrogate_train / set_weights / load); 0 <= 2 window + 1 <= min(Na, Nb). */
int surrogate_propose(cvx_handle *h, const cvx_params *p, int64_t n, const double *F,
                      const double *beta_k, int window, double gap_tol, double *W_R, double *P,
                      cvx_laminate *root, cvx_node *tree, uint8_t *fell_back, int32_t *status,
                      cvx_stream s);

/* Weights and standardisation to / from a file (little-endian FP32). */
int surrogate_save(cvx_handle *h, const char *path);
int surrogate_load(cvx_handle *h, const char *path);

/* The tensor-core building block of the network: C (M x N, FP32, DEVICE) =
 * A (M x K) B (N x K)^T with A, B bfloat16 (raw 16-bit patterns), DEVICE,
 * row-major, 16-byte aligned; K a positive multiple of 16.  Synchronous. */
int cvx_gemm_bf16(cvx_handle *h, int M, int N, int K, const uint16_t *A, const uint16_t *B,
                  float *C, cvx_stream s);

/* ------------------------------------------------ allocation-free variant */

/* convexify_points for callers that may not allocate device memory — for
 * example a material routine plugged into a host finite-element code that
 * owns all device memory through its own pool, or a latency-critical caller
 * that cannot accept cudaMalloc's implicit device synchronisation.  The paper
 * has no counterpart; this is a packaging of the same computation.
 *
 * Same arguments and results as convexify_points (no handle, no root/tree
 * outputs; W_R, P, status, F, beta_k are caller-owned device pointers).  All
 * scratch lives in one fixed 64 MiB device array of the library (every GPU
 * that loads the library holds it until the process exits); nothing in this
 * call allocates device memory.  Limits: at most 16384 directions, and a
 * problem whose scratch (tree, queues, candidate records; roughly
 * n * (88 (2^{K+1} - 1) + 600 * 2^{K-1}) bytes plus 48 bytes per direction)
 * fits in 64 MiB; larger problems are rejected with CVX_ERR_INVALID_ARG.
 * Runs on the calling thread's current device.  The first call on a device
 * looks up the array's device address there (cudaGetSymbolAddress).  Every
 * call shares the array and leaves its contents behind (each call clears what
 * must start at zero), so calls that overlap on the GPU — on different streams, or from different
 * host threads — race and must be serialised by the caller. */
int convexify_points_static(const cvx_params *p, int64_t n, const double *F,
                            const double *beta_k, double *W_R, double *P, int32_t *status,
                            cvx_stream s);

#ifdef __cplusplus
}
#endif
#endif /* CONVEXIFY_H */
