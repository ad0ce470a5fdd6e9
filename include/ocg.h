/*
 * ocg.h - C ABI of libocg: multigrid-preconditioned conjugate gradient for
 * div(beta grad p) = b on a 2:1-balanced adaptive octree with cut cells, on one
 * B300 GPU (sm_103a).
 *
 * Method: "Matrix-Free Multigrid with Algebraically Consistent Coarsening on Adaptive
 * Octrees" (Wang, Sun, Zhu).  Operator: Sec. 2.1 (Eq. projection-poisson-system) with
 * the T-junction ghost rule of Sec. 3.1 (Eq. t-junction-ghost-values); coarsening:
 * Sec. 2.5, Alg. 3; preconditioner: the FAS-style mu-cycle of Sec. 3.2, Alg. 4, with
 * red-black Gauss-Seidel smoothing (Sec. 2.3); Krylov loop: Alg. 1 (Sec. 2.2).
 *
 * Conventions
 *  - Every function returns an int status: OCG_OK (0) or a negative OCG_E* code;
 *    ocg_last_error() returns a message for the calling thread's last failure.
 *  - Handles (ocg_octree, ocg_hier) are opaque and owned by the library; release them
 *    with the matching *_destroy.  A hierarchy keeps a pointer to its octree: destroy
 *    the hierarchy first.
 *  - Vector arguments named *_dev are caller-owned device pointers; *_host are
 *    caller-owned host pointers.  Leaf vectors are indexed in canonical leaf order:
 *    sorted by (depth, Morton key of (i,j,k) with x in bit 0).
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).  A call
 *    is asynchronous on that stream unless its comment says it synchronises.
 *  - Device: an octree's tables go to the device that is current at its first
 *    ocg_setup_hierarchy, and a hierarchy belongs to that device.  Every later call on
 *    either (set-up of another hierarchy on the octree, applies, cycles, solves, batches)
 *    must run with that device current, else it returns OCG_EINVAL.
 *  - Boundary codes per wall in the order x-, x+, y-, y+, z-, z+: OCG_BC_NEUMANN (0) or
 *    OCG_BC_DIRICHLET (1, value held at the wall face, weight 2*h, beta = 1 on walls;
 *    a non-zero wall value enters through the right-hand side).
 */
#ifndef OCG_H
#define OCG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define OCG_OK 0
#define OCG_EINVAL (-1)    /* malformed argument or unsupported size */
#define OCG_ENOMEM (-2)    /* device or host allocation failed */
#define OCG_ECUDA (-3)     /* a CUDA runtime call failed */
#define OCG_ENOTCONV (-4)  /* max_iter reached before the tolerance; stats are filled */
#define OCG_ENAN (-5)      /* a non-finite residual norm was detected */
#define OCG_ESTATE (-6)    /* handle in the wrong state for this call */

#define OCG_BC_NEUMANN 0
#define OCG_BC_DIRICHLET 1

#define OCG_REFINE_NONE 0        /* uniform root grid */
#define OCG_REFINE_BALL_CENTRE 1 /* refine iff |centre - c|^2 < r^2 (first sphere) */
#define OCG_REFINE_SDF_BAND 2    /* refine iff |phi(centre)| < band + (sqrt(3)/2) h */
#define OCG_REFINE_SINE_BAND 3   /* refine iff |phi(c)| < band + |grad phi(c)| (sqrt(3)/2) h,
                                    phi a normalised sum of plane sine waves */
#define OCG_REFINE_STAR_BAND 4   /* refine iff |phi(c)| < band + L (sqrt(3)/2) h, phi the star
                                    surface r - (r0 + a cos(k theta) cos(k phi)) (Sec. 4.1) */

#define OCG_F64 0
#define OCG_F32 1

#define OCG_PREC_FP64 0        /* FP64 PCG and FP64 cycle; needs coef_dtype OCG_F64 */
#define OCG_PREC_FP32 1        /* FP32 vectors throughout, FP64 dot products */
#define OCG_PREC_MIXED 2       /* FP64 PCG vectors and dots, FP32 cycle */

typedef struct ocg_octree ocg_octree;
typedef struct ocg_hier ocg_hier;

/* Refinement description (Sec. 3, Sec. 4.1 grids).  Root grid n0^3 cells on the unit
 * cube (n0 even, 2 <= n0, n0 * 2^max_depth <= 2^20), leaves at depths 0..max_depth.
 * A depth-d cell with d < max_depth is refined when the predicate holds at its centre
 * x = (i + 0.5) / (n0 2^d); predicate arithmetic is IEEE float64 in a fixed order:
 *   BALL_CENTRE: (dx*dx + dy*dy) + dz*dz < r*r with d = x - centre of spheres[0]
 *   SDF_BAND:    |phi| < band + (0.5*sqrt(3)) * (1/(n0 2^d)), phi = min over
 *                spheres sqrt(dx*dx+dy*dy+dz*dz) - r and boxes (lo, hi):
 *                q = |x - 0.5*(lo+hi)| - 0.5*(hi-lo),
 *                sqrt(mx*mx+my*my+mz*mz) + min(max(qx, max(qy, qz)), 0), m = max(q, 0)
 *   STAR_BAND:   (cx, cy, cz, r0) = spheres[0], (a, k, L) = spheres[1][0..2] (k an
 *                integer 0..16): d = x - c, rho2 = dx*dx + dy*dy, r = sqrt(rho2 + dz*dz),
 *                rho = sqrt(rho2), u = dz / r (1 if r = 0), v = dx / rho (1 if rho = 0),
 *                T_k by the Chebyshev recurrence t0 = 1, t1 = w, t(n+1) = (2*w)*t(n) - t(n-1)
 *                (cos(k theta) = T_k(u), cos(k phi) = T_k(v) with theta the polar angle
 *                from +z and phi the azimuth from +x), phi = r - (r0 + (a * T_k(u)) * T_k(v));
 *                refined iff |phi| < band + (L * (0.5*sqrt(3))) * (1/(n0 2^d)).
 *   SINE_BAND:   phi = s / n and |grad phi| = sqrt((gx*gx + gy*gy) + gz*gz) / n over the
 *                n = n_sines waves (kappa, dx, dy, dz, theta) = sines[w], accumulated in
 *                w order from 0: w2 = TWO_PI * kappa, a = w2 * ((dx*x + dy*y) + dz*z) + theta,
 *                s += sin(a), g += (w2 * cos(a)) * (dx, dy, dz); refined iff
 *                |phi| < band + (|grad phi| * (0.5*sqrt(3))) * (1/(n0 2^d)).
 *                TWO_PI is 2 pi rounded to double.  sin and cos are the library's own
 *                deterministic forms (so that any implementation can reproduce the tree
 *                bit for bit): k = rint(a * (2/pi)), r = ((a - k P1) - k P2) - k P3 with
 *                pi/2 = P1 + P2 + P3 (P1 = 0x1.921fb544p+0, P2 = 0x1.0b4611a6p-34,
 *                P3 = 0x1.3198a2e037073p-69), Taylor polynomials in r2 = r*r evaluated by
 *                Horner from the highest term, sin r = r + (r*r2) * sum_{j=0..7}
 *                (-1)^(j+1)/(2j+3)! r2^j and cos r = 1 + r2 * sum_{j=0..8} (-1)^(j+1)/(2j+2)!
 *                r2^j, coefficients formed as 1.0 / n! in double, and the quadrant
 *                q = k mod 4 selecting (sin r, cos r, -sin r, -cos r) for sin(a) and
 *                (cos r, -sin r, -cos r, sin r) for cos(a).  Valid for |a| < 2^20.
 * With tile_log2 = t > 0 every aligned tile of 2^t x 2^t x 2^t depth-d cells takes one
 * decision, the predicate above evaluated for the depth-(d - t) cell that covers the tile
 * (i, j, k replaced by i >> t, j >> t, k >> t and n0 2^d by (n0 2^d) >> t): the paper's
 * grids refine the 8^3 tiles that meet the surface (Sec. 4.1, t = 3).
 * followed by the minimal refinement that makes face-neighbouring leaves differ by at
 * most one depth (Sec. 3). */
typedef struct {
    int32_t n0;
    int32_t max_depth;
    int32_t refine;
    int32_t n_spheres;      /* <= 4 */
    int32_t n_boxes;        /* <= 4 */
    int32_t tile_log2;      /* 0..4: the predicate decides per aligned tile of 2^tile_log2
                               cells per axis (n0 a multiple of 2^tile_log2); 0 = per cell */
    double band;
    double spheres[4][4];   /* cx, cy, cz, r */
    double boxes[4][6];     /* lox, loy, loz, hix, hiy, hiz */
    int32_t n_sines;        /* 1..8 for SINE_BAND, else ignored */
    int32_t reserved2;
    double sines[8][5];     /* kappa, dx, dy, dz, theta per wave (|a| < 2^20 required) */
} ocg_octree_desc;

/* Build the octree and its multigrid tables on the host (no device call; the tables are
 * uploaded to the current device by the first ocg_setup_hierarchy on this octree).
 * Errors: EINVAL (bad desc), ENOMEM. */
int ocg_octree_build(const ocg_octree_desc* desc, ocg_octree** out);

/* Octree of desc built from a previous octree after a local change of the geometry (a
 * moved or resized obstacle: the tables are recomputed whenever the grid topology
 * changes, Sec. 3.4).  box = (lox, loy, loz, hix, hiy, hiz) in the unit cube's
 * coordinates.  The refinement predicate is evaluated again only for the cells that meet
 * the box (with one cell of margin per depth) and for the children of cells whose flag
 * changed; every other cell keeps its flag from prev; the 2:1 closure and all tables are
 * then formed as by ocg_octree_build.
 * Contract: the predicate of desc equals that of prev's description on every cell that
 * does not meet the box (for SDF_BAND: the box holds the moved primitive's old and new
 * positions grown by band + sqrt(3)/2 / n0).  Under it the result is the octree that
 * ocg_octree_build(desc) makes, table for table; without it the result is a valid
 * 2:1-balanced octree but not necessarily that one.  prev is not modified and stays
 * valid; the new octree is independent of it.
 * Errors: EINVAL (null argument, bad desc, n0 / max_depth / refine / tile_log2 differing from prev's,
 * box not finite or lo > hi), ENOMEM. */
int ocg_octree_rebuild(const ocg_octree* prev, const ocg_octree_desc* desc, const double box[6],
                       ocg_octree** out);
void ocg_octree_destroy(ocg_octree* t);

/* counts[0] leaves, [1] canonical faces, [2] max depth D, [3] coarsest level mc (<= 0),
 * [4] cells over all levels (padded), [5] T-junction octet records, [6] cells of the
 * tree levels 0..D (leaves and inner), [7] octets over all levels. */
int ocg_octree_counts(const ocg_octree* t, int64_t counts[8]);

/* Canonical tables for bit-exact comparison (host buffers sized from counts).
 * Leaves: depth, i, j, k (coordinates at the leaf's depth), n_leaves each. */
int ocg_octree_export_leaves(const ocg_octree* t, int32_t* depth, int32_t* i, int32_t* j,
                             int32_t* k);
/* Per leaf and direction (x-,x+,y-,y+,z-,z+), 6 entries per leaf: kind 0 wall,
 * 1 same-depth leaf, 2 coarser leaf (fine side of a T-junction), 3 refined neighbour
 * (coarse side); rank = canonical rank of the neighbour leaf for kinds 1 and 2, else -1. */
int ocg_octree_export_neighbours(const ocg_octree* t, int8_t* kind, int64_t* rank);
/* Faces in canonical order (axis, depth of the finer side, Morton key of the cell on
 * the + side at that depth); minus/plus = canonical leaf ranks of the two sides. */
int ocg_octree_export_faces(const ocg_octree* t, int32_t* axis, int32_t* depth, int32_t* i,
                            int32_t* j, int32_t* k, int64_t* minus, int64_t* plus);
/* The same for canonical faces first .. first+count-1 only (buffers of count entries), so
 * that trees with hundreds of millions of faces can be read in pieces.  NULL buffers are
 * skipped.  Errors: EINVAL (range outside 0..n_faces). */
int ocg_octree_export_faces_range(const ocg_octree* t, int64_t first, int64_t count, int32_t* axis,
                                  int32_t* depth, int32_t* i, int32_t* j, int32_t* k,
                                  int64_t* minus, int64_t* plus);
/* Cells of multigrid level m (mc <= m <= D) in Morton order of the level's grid: depth-m
 * cells for m >= 0, the uniform root coarsening n0/2^-m for m < 0 (padding cells of an
 * odd coarsest grid excluded).  Call with i == NULL to get *n only. leaf: 1 for leaves. */
int ocg_octree_export_level(const ocg_octree* t, int32_t m, int64_t* n, int32_t* i,
                            int32_t* j, int32_t* k, int8_t* leaf);

/* Multigrid parameters (Sec. 2.3, 3.3). */
typedef struct {
    int32_t mu;            /* cycle index: 1 V-cycle, 2 W-cycle */
    int32_t nu_pre;        /* RBGS iterations before the coarse correction (red->black) */
    int32_t nu_post;       /* after it (black->red) */
    int32_t nu_coarsest;   /* at the coarsest level: half red->black, half black->red */
    double beta_restrict;  /* beta applied on the restriction (Alg. 4): 2 */
    double alpha;          /* R = P^T / alpha (Sec. 3.3): 2 */
    int32_t coef_dtype;    /* OCG_F64 or OCG_F32 storage of the matrix-free coefficients */
    int32_t bf16_coarse;   /* 1: the cycle reads BF16 copies of levels below the finest */
    int32_t sweep_form;    /* OCG_SWEEP_AUTO (time every form per level at set-up and keep
                              the fastest), OCG_SWEEP_OCTET, OCG_SWEEP_CELL, OCG_SWEEP_QUAD or
                              OCG_SWEEP_TILE */
    int32_t mu_min_cells;  /* 0: mu applies on every level (the paper's cycle).  > 0 (an
                              extension): the recursion into a coarser level is repeated mu
                              times only when that level has at least this many cells
                              (leaves and inner, padding excluded), once otherwise — a
                              W-cycle on the large levels, a V-cycle on the small ones whose
                              cost on the GPU is launch latency.  Negative: EINVAL. */
    int32_t coarsening;    /* OCG_COARSEN_ALGEBRAIC (Alg. 3: the paper's algebraically
                              consistent coarsening) or OCG_COARSEN_GEOMETRIC (the geometric
                              multigrid of Sec. 3.3, for ablation): every cell with children
                              on the levels below the finest takes the coefficients the grid
                              gives it at its own size H: w = beta H per face, beta the fluid
                              fraction of the face from the SDF of the description's spheres
                              and boxes (positive in fluid) at its four corners, split into
                              two triangles along the face's (0,0)-(1,1) diagonal in the
                              other two axes, phi linear on each, positive area exact,
                              clamped to [1e-3, 1] and rounded to FP32; a wall face 2H
                              (Dirichlet) or 0 (Neumann); c = the sum of the six (0 kept
                              where Alg. 3 gives 0).  For cut-cell problems whose face beta
                              is that fraction.  Needs OCG_REFINE_SDF_BAND; else EINVAL. */
    int32_t reserved;      /* must be 0 */
} ocg_mg_params;
#define OCG_COARSEN_ALGEBRAIC 0
#define OCG_COARSEN_GEOMETRIC 1

#define OCG_SWEEP_AUTO (-1)
#define OCG_SWEEP_OCTET 0      /* one thread per octet (8 cells in registers) */
#define OCG_SWEEP_CELL 1       /* one thread per cell (octet in 8 lanes) */
#define OCG_SWEEP_QUAD 2       /* two threads per octet (one z-layer of 4 cells each) */
#define OCG_SWEEP_TILE 3       /* one thread per octet, the block's octets shared in shared memory */

/* Fill leaf coefficients from face beta (canonical face order, float32, device) and the
 * wall codes (Sec. 2.1; T sub-faces per Sec. 3.1), then coarsen every level with Alg. 3
 * (FP64 arithmetic, stored in coef_dtype).  Synchronises.
 * beta = 0 on every face of a leaf (e.g. exact fluid fractions inside a solid) leaves it
 * without a coefficient: an inactive cell that every kernel skips (its solution stays 0;
 * means over octets count active cells only, 0 when there is none).  With inactive cells
 * a constant null space is not supported (the mean shift would reach them), and the
 * transposed operator's T-junction correction assumes every cell active.
 * Errors: EINVAL (negative or non-finite beta, bad params), ENOMEM, ECUDA. */
int ocg_setup_hierarchy(const ocg_octree* t, const float* face_beta_dev, const int32_t bc[6],
                        const ocg_mg_params* prm, void* stream, ocg_hier** out);
void ocg_hier_destroy(ocg_hier* h);

/* Refresh the hierarchy for new face fractions beta (device, canonical face order, FP32)
 * on the same octree, walls and parameters (no counterpart in the paper; the per-step
 * refresh of a moving-boundary simulation whose topology is unchanged): the leaf
 * coefficients, Alg. 3 (or the geometric rediscretisation) and the FP32 / BF16 copies are
 * recomputed in place, so solves, graphs captured on the hierarchy and batches built from
 * it keep working on the new coefficients; sweep and tail choices made at set-up are kept.
 * Synchronises the stream.  Errors: EINVAL (null argument, negative or non-finite beta:
 * the coefficients are then undefined until a successful update), ECUDA. */
int ocg_hier_update_beta(ocg_hier* h, const float* beta_dev, void* stream);

/* Sweep form chosen for level m and, if the set-up timed them, the measured time of one
 * colour sweep in each form (microseconds, captured in a CUDA graph; -1 if not timed).
 * Levels run inside the shared-memory coarse kernel report form -1. */
int ocg_hier_tuning(const ocg_hier* h, int32_t m, int32_t* form, double* us_octet, double* us_cell,
                    double* us_quad, double* us_tile);

/* Stored coefficients (c, c_x-, c_y-, c_z-) of level m, cells in the order of
 * ocg_octree_export_level, as float64 host arrays.  Synchronises. */
int ocg_hier_export_coefs(const ocg_hier* h, int32_t m, double* c, double* cx, double* cy,
                          double* cz);

/* y = A x for the composite leaf operator (Sec. 2.1 flux sums, Sec. 3.1 ghosts; inner
 * values are the mean of their active children).  dtype OCG_F64 or OCG_F32 for both x
 * and y (device, canonical leaf order, n_leaves).  transpose = 1 gives y = A^T x (the
 * operator of the adjoint solve; no counterpart in the paper): A x plus the rows of
 * A^T - A, which only T-junctions make non-zero (every tree cell is taken as active
 * there).  Other transpose values: EINVAL.  The first transposed call builds and
 * uploads the octree's adjoint tables (host work, synchronous). */
int ocg_apply_A(ocg_hier* h, int32_t dtype, const void* x_dev, void* y_dev, int32_t transpose,
                void* stream);

/* z = one FAS-style mu-cycle from zero applied to r (Alg. 4), dtype OCG_F64 or OCG_F32
 * (F64 needs coef_dtype OCG_F64; F32 needs OCG_F32); device, canonical leaf order. */
int ocg_vcycle(ocg_hier* h, int32_t dtype, const void* r_dev, void* z_dev, void* stream);

/* r = M^T z, the transpose of the linear map z = M r of ocg_vcycle (no counterpart in the
 * paper): the transposes of the cycle's steps (Alg. 4: colour sweeps, FAS restriction with
 * u* = Avg(u), recursion, prolongation) applied in reverse order to adjoint states.  It is
 * the preconditioner of the adjoint solve: A^T M^T = (M A)^T has the spectrum of A M.
 * Every level runs as plain launches (no shared-memory coarse tail).  Same dtype rules and
 * layout as ocg_vcycle; allocates two scratch vectors over all cells on first use.
 * Errors: EINVAL, ENOMEM, ECUDA. */
int ocg_vcycle_transpose(ocg_hier* h, int32_t dtype, const void* z_dev, void* r_dev, void* stream);

#define OCG_SOLVE_EAGER 1      /* flags: launch kernel by kernel, test convergence on the host */
#define OCG_SOLVE_TRANSPOSE 2  /* flags: solve A^T x = b (adjoint system) by BiCGStab */
#define OCG_SOLVE_UNROLLED 4   /* flags (measurement): run exactly max_iter iterations as one
                                  flat CUDA graph without the WHILE node, so that a probe's
                                  events become graph nodes around the probed kernels */
#define OCG_SOLVE_BICGSTAB 8   /* flags, with OCG_SOLVE_TRANSPOSE: solve A^T x = b by BiCGStab
                                  instead of Alg. 1 (both preconditioned by M^T) */
#define OCG_SOLVE_WARM 16      /* flags: x_dev holds the initial guess x0 on input (else
                                  x0 = 0); r0 = b - A x0 (A^T x0), the stop test stays
                                  ||r|| <= tol ||b|| */

typedef struct {
    double tol;              /* stop when ||r||_2 <= tol ||b||_2 (recursive residual) */
    int32_t max_iter;        /* >= 1 */
    int32_t precision;       /* OCG_PREC_* */
    int32_t nullspace;       /* -1 auto (all walls Neumann), 0 off, 1 zero-mean residual */
    int32_t flags;           /* OCG_SOLVE_* */
} ocg_solve_params;

#define OCG_HIST 128
typedef struct {
    int32_t iterations;      /* operator applications inside the loop */
    int32_t converged;
    double rel_res;          /* last recursive ||r|| / ||b|| */
    double true_rel_res;     /* ||b - A x|| / ||b|| recomputed in FP64 at exit */
    int64_t kernels;         /* kernel launches this solve executed */
    double hist[OCG_HIST];   /* rel_res after each iteration, hist[0] = 1 */
} ocg_solve_stats;

/* Solve A x = b (Alg. 1 preconditioned by one mu-cycle per iteration, x0 = 0).  b and x
 * are float64 device vectors in canonical leaf order.  By default the loop runs as a
 * CUDA graph (captured on the first solve of each precision / null-space mode and kept
 * with the hierarchy) whose iterations sit under a conditional WHILE node: the test
 * ||r|| <= tol ||b|| is made on the device and the call synchronises once, at the end.
 * With OCG_SOLVE_EAGER, or while a probe is set, kernels are launched one by one and the
 * host tests convergence after every iteration.  The true residual is recomputed in FP64
 * at exit.  With the null space on, b is shifted to zero mean and x is returned with
 * zero mean over the leaves.
 * With OCG_SOLVE_TRANSPOSE the call solves A^T x = b (adjoint system; no counterpart in
 * the paper) by Alg. 1 on A^T preconditioned by the transposed cycle M^T
 * (ocg_vcycle_transpose): its scalars (r, M^T r) = (M r, r) and (p, A^T p) = (A p, p) are
 * the forward method's quadratic forms.  With OCG_SOLVE_TRANSPOSE | OCG_SOLVE_BICGSTAB it
 * uses BiCGStab (van der Vorst 1992), right-preconditioned by M^T, whose iteration applies
 * M^T and A^T twice.  Alg. 1 with the forward cycle M stagnates on A^T, which T-junctions
 * make differ from A, and BiCGStab with M diverges at high coefficient contrast.
 * `iterations` counts iterations.  A hierarchy serves one solve at a time (its work
 * vectors are shared).
 * Known limit: partly solid cells kept as unknowns (exact fractions on every face, so a
 * cell with tiny fluid faces stays active) beside T-junctions give rows whose T ghost
 * outweighs the diagonal; where many sit on a thin obstacle (e.g. the star tank on the
 * 128^3-root cell-by-cell band grid) the iteration can stagnate (ENOTCONV).  Classifying
 * the solid cells as the ghost-fluid method of Sec. 2.1 does (a cell whose centre is in
 * the solid is no unknown: give every face touching it beta = 0) removes those rows, and
 * the tank solves then converge at the paper's rates on band and tile grids.
 * Errors: ENOTCONV (stats filled), ENAN, EINVAL (also unknown flags), ECUDA. */
int ocg_pcg_solve(ocg_hier* h, const double* b_dev, double* x_dev, const ocg_solve_params* prm,
                  ocg_solve_stats* stats, void* stream);

/* Batched solves: many independent problems advanced together (no counterpart in the
 * paper).  A batch groups n hierarchies (each set up by ocg_setup_hierarchy with FP32
 * coefficients, no BF16, the same mu of 1 or 2 with mu_min_cells 0, nu_post >= 1, equal
 * nu / alpha / beta_restrict, and a shared-memory coarse tail, i.e. an even root grid of
 * at least 8 cells per axis).  One launch per phase serves all problems: the cycle's
 * phases are aligned at the problems' finest levels, so Alg. 4's recursion (mu visits of
 * the next height per visit) is one schedule for all; the coarse tails that sit at one
 * height run in one launch (one CTA per problem); the sweep form of each height is
 * timed at creation when the first hierarchy's sweep_form is OCG_SWEEP_AUTO.  The batch uses the hierarchies' work vectors: while it exists, do not
 * run other solves on those hierarchies concurrently with it, and destroy it before them.
 * Synchronises the stream.  Errors: EINVAL (incompatible hierarchies), ENOMEM, ECUDA. */
typedef struct ocg_batch ocg_batch;
int ocg_batch_create(ocg_hier* const* hs, int32_t n, void* stream, ocg_batch** out);
void ocg_batch_destroy(ocg_batch* b);

/* Heights of the batch's V-cycle above the coarse tails (*heights) and, for height h
 * (1..*heights), the chosen sweep form and the timed microseconds of one colour sweep
 * of all problems in each form (-1 if not timed). */
int ocg_batch_info(const ocg_batch* b, int32_t h, int32_t* heights, int32_t* form, double* us_octet,
                   double* us_cell);

/* Solve A_p x_p = b_p for every problem p of the batch by Alg. 1 preconditioned by one
 * V-cycle (mixed precision: FP32 cycle, FP64 Krylov vectors; prm->precision must be
 * OCG_PREC_MIXED, prm->flags 0).  b_dev[p] / x_dev[p]: float64 device vectors of problem
 * p in canonical leaf order (host arrays of n device pointers).  Per-problem alpha, beta,
 * residual and stop test; a problem that has converged is frozen while the others go on;
 * the loop is one CUDA graph whose WHILE node runs while any problem is open.  stats: n
 * entries, filled per problem (kernels = launches of the whole batch).  Synchronises
 * once.  Errors: ENOTCONV (some problem hit max_iter; stats filled), ENAN, EINVAL. */
int ocg_pcg_solve_batched(ocg_batch* b, const double* const* b_dev, double* const* x_dev,
                          const ocg_solve_params* prm, ocg_solve_stats* stats, void* stream);

/* Face gradient of a loss through the solve (adjoint; no counterpart in the paper).
 * With p the solution of A p = b and lambda that of A^T lambda = dL/dp, writes
 * dbeta[f] = dL/dbeta_f = -lambda^T (dA/dbeta_f) p for every canonical face f (the order
 * of ocg_octree_export_faces): -h_f (lambda_i - lambda_j)(p_i - p_j) for the face between
 * equal-depth leaves i (- side) and j, and -(h_f/2)(lambda_i - lambda_K)(pbar_P - p_K) for
 * a T sub-face of the fine leaf i against the coarser leaf K, pbar_P the mean of the
 * leaves under i's parent (Sec. 3.1 ghost).  p, lambda: float64 device vectors in
 * canonical leaf order; dbeta: float64 device vector of n_faces.  Uses the hierarchy's
 * work vectors (one call at a time per hierarchy). */
int ocg_face_grad(ocg_hier* h, const double* p_dev, const double* lambda_dev, double* dbeta_dev,
                  void* stream);

/* Operator apply that allocates nothing (no counterpart in the paper).
 * For callers that must not allocate device memory at call time, e.g. code running
 * under a memory budget enforced by an external allocator, a real-time loop that may not
 * block on cudaMalloc, or a host framework that forbids allocations outside its own
 * pool.  Computes the same y = A x as ocg_apply_A with dtype OCG_F32 and transpose 0
 * (float32 x_dev / y_dev, canonical leaf order, caller-owned), but its two work vectors
 * live in a fixed device array compiled into the library (8 MiB, held by every GPU that
 * loads the library until the process exits), so at most OCG_NOALLOC_MAX_CELLS cells of
 * the tree levels 0..D (counts[6] of ocg_octree_counts) are accepted; larger trees get
 * OCG_EINVAL.  The first call on a device looks up that array's device address (with
 * that device current); make the first call before any stream capture.  All calls share
 * the array: calls that overlap on the GPU (other streams, other threads) race and must
 * be serialised by the caller.  Calls no cudaMalloc / cudaFree. */
#define OCG_NOALLOC_MAX_CELLS (1 << 20)
int ocg_apply_A_f32_noalloc(ocg_hier* h, const float* x_dev, float* y_dev, void* stream);

/* Measurement hooks (no counterpart in the paper; used by the benchmark).
 * ocg_probe_set: from now on, bracket every launch of kernel `kind` on level `level`
 * with CUDA events recorded on the launching stream (kind 0 off, 1 red-black sweep,
 * 2 residual+restriction, 3 prolongation, 4 composite operator (level 0), 5 the
 * shared-memory coarse kernel (level = its finest level)).
 * ocg_probe_read: synchronises the stream, returns the number of bracketed launches,
 * their summed duration in ms and the cells one launch processes, and resets. */
#define OCG_PROBE_OFF 0
#define OCG_PROBE_SWEEP 1
#define OCG_PROBE_RESTRICT 2
#define OCG_PROBE_PROLONG 3
#define OCG_PROBE_APPLY 4
#define OCG_PROBE_TAIL 5
int ocg_probe_set(ocg_hier* h, int32_t kind, int32_t level);
int ocg_probe_read(ocg_hier* h, void* stream, int64_t* launches, double* total_ms,
                   int64_t* cells_per_launch);

/* Device memory hooks: from now on the library obtains every device buffer (octree
 * tables, coefficients, work vectors, graphs' scratch) from alloc(bytes, ctx), which must
 * return memory of the current device aligned to 256 bytes or NULL (ENOMEM), and releases
 * it with free(ptr, ctx) — e.g. a framework's caching allocator.  Both NULL restores
 * cudaMalloc / cudaFree.  A block is always released by the hooks that made it, so the
 * hooks may change while objects live, but they must stay callable until those objects
 * are destroyed.  Pinned host buffers stay cudaMallocHost.  Thread-safe.
 * Errors: EINVAL (one hook given without the other). */
typedef void* (*ocg_alloc_fn)(size_t bytes, void* ctx);
typedef void (*ocg_free_fn)(void* ptr, void* ctx);
int ocg_set_allocator(ocg_alloc_fn alloc, ocg_free_fn free_fn, void* ctx);

/* Total kernel launches issued by this library in this process. */
int ocg_launch_count(int64_t* n);

const char* ocg_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* OCG_H */
