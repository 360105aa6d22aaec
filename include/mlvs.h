/*
 * mlvs.h -- C ABI of the MLVS-DUGKS hot-path library (sm_103a).
 *
 * The library advances the reduced distributions (g, h) of the BGK/Shakhov model with the
 * discrete unified gas-kinetic scheme (Sec. 2.2, Eqs. phi_update ... recover_phi) over every
 * (physical cell x discrete velocity) pair, on one or several velocity spaces built on a
 * quadtree-structured Newton--Cotes base grid (Sec. 2.3, 3.1-3.2).  Multi-level parts follow
 * Sec. 3.2 (criterion, grouping), Sec. 3.3 (linear moment-constrained correction) and
 * Sec. 3.4 (inter-level coupling).  Cartesian and structured curvilinear meshes use
 * mlvs_handle; unstructured meshes of polygonal cells (one velocity space) use mlvs_uhandle
 * (mlvs_ucreate ... mlvs_udestroy), whose errors are read with mlvs_last_error(NULL).
 *
 * Conventions
 *  - Every entry point returns an mlvs_status; MLVS_OK is 0 and errors are negative.
 *  - Pointers marked "host" are read (or written) during the call only; the caller keeps
 *    ownership.  The handle owns all device memory it allocates and frees it in
 *    mlvs_destroy.
 *  - A handle is single-threaded: calls on one handle must not overlap.  All device work is
 *    ordered on the stream given in mlvs_config.stream (NULL: the legacy default stream).
 *  - Asynchronous device errors (non-finite or negative moments, an exhausted bounded wait)
 *    surface as the status of the next mlvs_step or mlvs_moments call.  After such an
 *    error the handle answers MLVS_ERR_STATE until destroyed.
 *  - mlvs_last_error returns a diagnostic string describing the last failing call.
 */
#ifndef MLVS_H
#define MLVS_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mlvs_handle mlvs_handle;

typedef enum {
  MLVS_OK = 0,
  MLVS_ERR_ARG = -1,        /* an argument is out of range or inconsistent              */
  MLVS_ERR_OOM = -2,        /* a device or host allocation failed                       */
  MLVS_ERR_CUDA = -3,       /* a CUDA runtime call failed                               */
  MLVS_ERR_NONFINITE = -4,  /* a moment became NaN/Inf                                  */
  MLVS_ERR_POSITIVITY = -5, /* density or temperature became non-positive               */
  MLVS_ERR_SINGULAR = -6,   /* a moment-correction matrix is singular                   */
  MLVS_ERR_TIMEOUT = -7,    /* a bounded device-side wait ran out                       */
  MLVS_ERR_STATE = -8       /* call order violated, or the handle holds an earlier error */
} mlvs_status;

/* boundary kinds, per side x-low, x-high, y-low, y-high */
enum { MLVS_BC_PERIODIC = 0, MLVS_BC_ZEROGRAD = 1, MLVS_BC_WALL = 2, MLVS_BC_FREESTREAM = 3 };
/* storage type of the distributions */
enum { MLVS_F64 = 0, MLVS_F32 = 1, MLVS_BF16 = 2 };
/* Newton--Cotes rule of the base grid (Sec. 2.3; the order is not named in the paper) */
enum { MLVS_QUAD_BOOLE = 0, MLVS_QUAD_SIMPSON = 1, MLVS_QUAD_TRAPZ = 2 };
/* slope limiter of Eq. reconstruction (Venkatakrishnan: unstructured meshes only) */
enum { MLVS_LIMITER_VANLEER = 0, MLVS_LIMITER_NONE = 1, MLVS_LIMITER_VENKAT = 2 };

typedef struct {
  int dim;              /* velocity/space dimension D: 1 or 2 (Sec. 2.1)                      */
  int n_instances;      /* independent cases advanced together (>= 1)                          */
  int nx, ny;           /* uniform Cartesian mesh; ny = 1 when dim = 1                         */
  double Lx, Ly;        /* domain lengths; cell sizes are Lx/nx, Ly/ny                         */
  int bc[4];            /* MLVS_BC_* for x-low, x-high, y-low, y-high                          */
  double wall[4][3];    /* (u_w, v_w, T_w) of each wall side (diffuse isothermal wall)         */
  double R;             /* gas constant                                                       */
  double K_internal;    /* internal degrees of freedom K (monatomic: 0)                        */
  double Pr;            /* Prandtl number; 1 gives the BGK model (Eq. shakhov_eq)              */
  double omega;         /* viscosity exponent of mu = mu_ref (T/T_ref)^omega (Sec. 4)          */
  double Kn;            /* Knudsen number, used when mu_ref <= 0 (VHS relation, alpha = 1)      */
  double mu_ref;        /* reference viscosity; > 0 overrides Kn                               */
  double L_ref, T_ref, rho_ref;
  double cfl;           /* dt = cfl * min(dx, dy) / max |xi|_inf, unless dt > 0                */
  double dt;            /* > 0: fixed time step                                               */
  int storage;          /* MLVS_F64 | MLVS_F32 | MLVS_BF16                                     */
  int compat_cell;      /* 1: four-moment compatibility correction at cells (Sec. 3.3.1)      */
  int compat_face;      /* 1: the same correction of the face model distribution              */
  int limiter;          /* MLVS_LIMITER_*                                                     */
  const double* init_W; /* host [n_instances][ny][nx][4] = (rho, u, v, T); copied              */
  void* stream;         /* cudaStream_t the library orders its work on                        */
  double far[4];        /* freestream (rho, u, v, T) of MLVS_BC_FREESTREAM sides: velocities
                           entering take its (corrected) Maxwellian, leaving ones the
                           reconstruction                                                  */
  int mesh_kind;        /* 0: the box Lx x Ly; 1: structured curvilinear mesh from node_xy    */
  const double* node_xy;/* mesh_kind 1: host [ny+1][nx+1][2] node coordinates, copied. Cell
                           (i,j) has nodes (i,j),(i+1,j),(i+1,j+1),(i,j+1) counter-clockwise;
                           on a periodic side the last node column/row repeats the first (an
                           O-grid) or is its translate.  Slopes along the index directions
                           become physical through J^{-T}; dt = cfl min |V|/max|S| / max|xi| */
  int positive_mapping; /* 1 (dim 2): a level switch or a cross-level ghost state whose additive
                           four-moment result has a negative g where the projection has none
                           takes the exponential correction of the same targets instead
                           (Sec. 3.3.2, Eq. exponential_moment_correction); ghost routes are
                           then launched one by one                                         */
  int map_moments;      /* 9 (dim 2): level switches, cross-level ghost states and cross-level
                           microfluxes use the nine-moment mapping (Sec. 3.3.2, Eqs.
                           mapping_nine_targets to mapping_h_residual_correction: the source's
                           raw moments up to G and J as targets), one launch per route;
                           0 or 4: the four-moment mapping                                   */
  int compat_moments;   /* 8 (dim 2): the compatibility correction at cells and faces
                           (compat_cell, compat_face) is the eight-moment correction of Sec.
                           3.3.1 (Eq. eq_eight_basis, Eq. eq_eight_moment_constraint), whose
                           heat-flux target is the Shakhov model's own heat flux (1 - Pr) q;
                           freestream sides keep the four-moment correction.  Runs on one
                           level (mlvs_set_velocity_levels with one level and adaptive = 0;
                           else MLVS_ERR_ARG): a uniform level or a kappa space, whose
                           model sums come from its rows of level groups.  0 or 4: the
                           four-moment correction                                            */
} mlvs_config;

/* One representative velocity space, described on the base grid (Sec. 3.2). */
typedef struct {
  int uniform_L;               /* >= 0: every axis grouped at level L; -1: use kappa         */
  const unsigned char* kappa;  /* host [N1][N1] coarsening index per 2x2 block, 0..3         */
} mlvs_level_desc;

typedef struct {
  int profile;               /* in: nonzero records CUDA events around every launch          */
  double dt;                 /* out: time step in use                                        */
  long long cell_velocity_updates; /* out: sum over levels of cells x velocities, per call   */
  int n_levels;              /* out                                                          */
  int launches;              /* out: kernels launched by the call                            */
  float ms_total;            /* out: device time of the call (CUDA events), ms               */
  float ms_phase[6];         /* out (profile): summed device time, ms, of the cell
                                finalisation, face-sum, face finalisation, update, ghost
                                mapping and flux mapping launches                            */
} mlvs_step_stats;

/* Create a handle for the problem in cfg (Sec. 2.1-2.2: mesh, gas model, boundaries, initial
 * state).  No velocity space exists yet.
 * Errors: MLVS_ERR_ARG (bad sizes/kinds), MLVS_ERR_CUDA, MLVS_ERR_OOM. */
mlvs_status mlvs_create(const mlvs_config* cfg, mlvs_handle** out);

/* Build the base grid (n_base points per axis on [umin, umax], rule `quadrature`,
 * Sec. 2.3) and the velocity spaces `levels` (Sec. 3.2), allocate the distributions of
 * every instance on level 0, and initialise them to the compatibility-corrected Maxwellian
 * of cfg.init_W (phi~ = phi^eq at rest in equilibrium).  n_base must be odd.
 * adaptive selects what mlvs_adapt does with the cell masks of the criterion: 1 groups them
 * into new representative spaces (Sec. 3.2; the level set is replaced); 0 keeps this level
 * set and moves every cell to the coarsest level (fewest velocities) whose space encloses
 * its mask, the finest level when none does.
 * Errors: MLVS_ERR_ARG, MLVS_ERR_OOM, MLVS_ERR_CUDA, MLVS_ERR_SINGULAR. */
mlvs_status mlvs_set_velocity_levels(mlvs_handle* h, int n_base, double umin, double umax,
                                     int quadrature, int n_levels,
                                     const mlvs_level_desc* levels, int adaptive);

/* Advance every instance by n_steps DUGKS steps (Sec. 2.2).  stats may be NULL; when given,
 * stats->profile is read and the other fields are written.
 * Errors: MLVS_ERR_STATE, MLVS_ERR_NONFINITE, MLVS_ERR_POSITIVITY, MLVS_ERR_CUDA. */
mlvs_status mlvs_step(mlvs_handle* h, int n_steps, mlvs_step_stats* stats);

/* Assign every cell of one instance to a velocity level (host levels[ny*nx], values in
 * 0..n_levels-1, copied).  A cell whose space changes is remapped by the hierarchical
 * projection and the four-moment correction with its own moments as targets
 * (Sec. 3.3.2, Eq. level_switch_conservation).  Cross-level faces are then evaluated on the
 * common refinement of the two spaces and their fluxes mapped back with the four-moment flux
 * correction (Sec. 3.4).
 * Errors: MLVS_ERR_ARG, MLVS_ERR_STATE, MLVS_ERR_OOM, MLVS_ERR_CUDA. */
mlvs_status mlvs_set_cell_levels(mlvs_handle* h, int instance, const int* levels);

/* Extra (the representative space of Sec. 3.2): number of velocities of a level and (if the
 * arrays are non-NULL, capacity cap) its coordinates and weights. */
mlvs_status mlvs_level_info(const mlvs_handle* h, int level, int* nv, double* xi_x, double* xi_y,
                            double* w, int cap);

/* Adaptation thresholds (Sec. 3.2). */
typedef struct {
  double C_split;    /* I_B above C_split: the block stays fine (Eq. block-hysteresis-rule)  */
  double C_merge;    /* I_B below C_merge: the block merges, subject to the transport test  */
  double eps_merge;  /* tolerance of Eq. merge-transport-error; <= 0 switches the test off   */
  double tau_clust;  /* graded-distance threshold of the grouping                          */
  int max_level;     /* coarsest candidate block: 1 (2x2), 2 (4x4) or 3 (8x8)              */
} mlvs_adapt_params;

typedef struct {
  int n_levels;                  /* representative spaces after the call                  */
  int n_distinct;                /* distinct cell masks                                   */
  int n_changed;                 /* cells (all instances) whose velocity space changed    */
  long long updates_per_step;    /* sum over levels of cells x velocities, all instances  */
  float ms_criterion;            /* device time of the criterion kernels                  */
  float ms_group;                /* wall time of the mask download and the grouping       */
  float ms_remap;                /* wall time of the level rebuild and the remap          */
  float ms_total;                /* wall time of the call                                 */
  int n_interior_faces;          /* faces between two cells, all instances (N_int, Sec. 3.5) */
  int n_cross_faces;             /* of those, faces between two levels (N_cross)          */
  int n_exp_corrected;           /* positive_mapping: cells remapped with the exponential
                                    correction                                            */
  int n_exp_failed;              /* positive_mapping: cells whose Newton iteration did not
                                    converge (they keep the additive result)              */
} mlvs_adapt_stats;

/* Velocity-space requirement of every cell of one instance (Sec. 3.2, criterion only): the
 * cell's (g~, h~) is read on the base grid by inheritance, the block indicator I_B of
 * Eq. block-contribution-indicator is compared with C_split / C_merge with hysteresis
 * against the cell's current space, the transport test applies below C_merge, and the
 * candidate blocks are scanned 8x8 -> 4x4 -> 2x2.  kappa_out is [ny*nx][N1*N1] bytes (N1 =
 * level-1 groups per axis of the base grid; row-major blocks, y major), host or device memory
 * (out_on_device).  2-D only.
 * Errors: MLVS_ERR_ARG (1-D, bad thresholds), MLVS_ERR_STATE, MLVS_ERR_CUDA. */
mlvs_status mlvs_criterion(mlvs_handle* h, int instance, const mlvs_adapt_params* p,
                           unsigned char* kappa_out, int out_on_device);

/* Adapt the velocity levels (Sec. 3.2): the criterion on every cell of every instance, then
 * (adaptive = 1) the grouping of the cell masks (mlvs_cluster) with one level per distinct
 * representative space (the blockwise minimum of its members, made parent-child
 * consistent), the level set being replaced so that level indices refer to the new set
 * afterwards; or (adaptive = 0) the coarsest enclosing level of the fixed set per cell.
 * Every cell whose space changed is remapped conservatively.  stats may be NULL
 * (n_distinct is 0 with adaptive = 0).
 * Errors: as mlvs_criterion, and MLVS_ERR_OOM. */
mlvs_status mlvs_adapt(mlvs_handle* h, const mlvs_adapt_params* p, mlvs_adapt_stats* stats);

/* Run mlvs_adapt with p after every `interval` steps taken by mlvs_step (interval 0: never);
 * the update interval of the representative spaces in the runs of Sec. 4.
 * p is copied. */
mlvs_status mlvs_set_adaptation(mlvs_handle* h, const mlvs_adapt_params* p, int interval);

/* Host-only: the velocity space of a coarsening mask (Sec. 3.1-3.2), built as the library
 * builds a representative space.  The base grid has n_base points per axis on [umin, umax] with
 * rule `quadrature` (MLVS_QUAD_*); kappa[nkappa] holds one byte per level-1 block (nkappa =
 * n1 * n1, y major) and is first made parent-child consistent (a block keeps level L only if
 * every level-1 block of its level-L parent allows L).  The space's points and weights (2-D,
 * in the library's point order) go to xi_x, xi_y, w of capacity cap; *nv_out receives the point
 * count and *n1_out (may be NULL) the level-1 groups per axis.  With kappa NULL only *n1_out is
 * written; with all three outputs NULL only the sizes are.  Needs no GPU.
 * Errors: MLVS_ERR_ARG (base size or rule invalid, nkappa != n1 * n1, cap too small). */
mlvs_status mlvs_space_points(int n_base, double umin, double umax, int quadrature,
                              const unsigned char* kappa, int nkappa, double* xi_x, double* xi_y,
                              double* w, int cap, int* nv_out, int* n1_out);

/* Host-only: the curvilinear geometry the library derives from a node grid (what a handle
 * created with mesh_kind = 1 uses): the face areas and normals of Eq. explicit_update and the
 * slope and offset geometry of Eq. reconstruction on the O-grid of the cylinder case (Sec. 4).
 * node_xy[(ny + 1) * (nx + 1)][2] row-major (row j = node
 * row), cells counter-clockwise; periodic_x, periodic_y say which pairs of sides are periodic.
 * cell_geo[5][nx * ny]: J^{-T} row-major (four rows; index-direction slopes times it give
 * physical slopes), then the area.  face_geo[7][nface]: x-faces first (nfx * ny, nfx = nx if
 * periodic_x else nx + 1), then y-faces (nx * nfy): unit normal (2 rows, towards the cell of
 * higher index), length, midpoint minus the lower-index side's centroid (2), midpoint minus the
 * higher-index side's centroid (2); a ghost's centroid is the boundary cell's reflected through
 * the face midpoint, a periodic image's is moved by the mean offset of the periodic node rows.
 * width[nx * ny] (may be NULL): area over the longest edge.  Needs no GPU.
 * Errors: MLVS_ERR_ARG (null pointers, sizes below 1, a cell that is not counter-clockwise). */
mlvs_status mlvs_mesh_geometry(int nx, int ny, int periodic_x, int periodic_y, const double* node_xy,
                               double* cell_geo, double* face_geo, double* width);

/* Host-only: the geometry of an unstructured mesh of polygonal cells, what the update of
 * Eq. explicit_update and the reconstruction of Eq. reconstruction need on general polygons
 * (the two-cavity expansion of Sec. 4.5 runs on unstructured cells).  node_xy[n_node][2];
 * cell c has the counter-clockwise nodes cell_nodes[cell_ptr[c] .. cell_ptr[c + 1]) (at least
 * three; cell_ptr[0] = 0).  A face is an edge used by one cell (boundary) or by two cells in
 * opposite directions; faces are numbered in the order of (smaller node, larger node); L is
 * the lower-numbered cell using the edge and the unit normal points out of L.  Outputs, all
 * NULL to get *n_face only, else all given (caller-owned, host memory):
 *   cell_geo[7][n_cell]: area, centroid x, y, width (area over the longest edge), and the
 *     inverse of the least-squares normal matrix sum d d^T (xx, xy, yy), d the centroid across
 *     each face minus the cell's, or twice the face midpoint minus the centroid on a boundary
 *     face (the cell reflected through the face);
 *   cell_face[cell_ptr[n_cell]]: per cell, in the order of its edges, f when the cell is L
 *     of face f and -f - 1 when it is R;
 *   face_cells[2][face_cap]: L, then R (-1 on a boundary face), rows face_cap apart;
 *   face_nodes[2][face_cap]: the edge's nodes in L's direction of traversal;
 *   face_geo[5][face_cap]: unit normal x, y, length, midpoint x, y.
 * Needs no GPU.  Errors: MLVS_ERR_ARG (null pointers, a node index out of range, a cell with
 * fewer than three nodes or with area <= 0, an edge used by more than two cells or twice in
 * the same direction, a singular normal matrix, face_cap below the face count). */
mlvs_status mlvs_umesh_geometry(int n_node, const double* node_xy, int n_cell, const int* cell_ptr,
                                const int* cell_nodes, int face_cap, int* n_face, double* cell_geo,
                                int* cell_face, int* face_cells, int* face_nodes, double* face_geo);

/* Host-only, no counterpart in the paper (data layout): a cell order along a Hilbert curve
 * through the bounding box of the centroids cx[n_cell], cy[n_cell] (16 bits per axis), so
 * that consecutive cells are spatially compact when the cells are renumbered in this order.
 * order[k] receives the cell visited k-th (caller-owned, n_cell entries); cells on the same
 * curve position keep their order.  Needs no GPU.
 * Errors: MLVS_ERR_ARG (null pointers, n_cell < 1, a non-finite centroid). */
mlvs_status mlvs_umesh_order(int n_cell, const double* cx, const double* cy, int* order);

/* Host-only grouping of nrow masks of nb bytes each (Sec. 3.2): distinct masks by decreasing
 * frequency (ties: lexicographic order), each joins the nearest existing centre when the
 * graded distance sum|ka - kb| / (3 nb) is <= tau (ties: lowest cluster), else it seeds a new
 * cluster.  labels[nrow] receives the cluster of every row, reps[reps_cap][nb] the blockwise
 * minimum over the members of each cluster, *n_reps the cluster count.  Needs no GPU.
 * Errors: MLVS_ERR_ARG (null pointers, nb < 1, reps_cap < *n_reps). */
mlvs_status mlvs_cluster(const unsigned char* kappa, long nrow, int nb, double tau, int* labels,
                         unsigned char* reps, int reps_cap, int* n_reps);

/* No counterpart in the paper (launch mechanics). CUDA graphs for mlvs_step: on != 0 replays the
 * launch sequence of two steps (the ping-pong buffers return to their parity after two) as one
 * graph, captured on first use and again whenever the levels change; an adaptation or a moments
 * call in between falls back to regular launches for the step concerned. Profiled steps never
 * use graphs. The handle's stream may be any stream, including the legacy default stream. */
mlvs_status mlvs_set_graph(mlvs_handle* h, int on);

/* No counterpart in the paper (batching). Advance several handles (independent cases, e.g.
 * different meshes and Knudsen numbers) by n_steps together. use_graph != 0: every two steps are
 * one graph launch on hs[0]'s stream whose branches are the instances of all handles, so their
 * kernels can run concurrently; the other handles' streams are ordered before and after it.
 * stats (may be NULL) sums over the group; ms_phase is not filled. A handle may appear only
 * once. Errors: as mlvs_step, for the first handle that fails. */
mlvs_status mlvs_step_many(mlvs_handle* const* hs, int n_handles, int n_steps, int use_graph,
                           mlvs_step_stats* stats);

/* No counterpart in the paper (launch tuning). Autotune the velocity chunking of the tile
 * launches: for each candidate number of CTAs per tile launch (148, 296, 444, 592, 888, 1184,
 * 1776) re-chunk the velocities of every level, run one warm step and `steps` timed steps, and
 * keep the fastest. *cta_target and ms_table[7] (ms per step of every candidate) are written
 * when non-NULL. The state advances by 7 (steps + 1) real steps. Errors: MLVS_ERR_ARG,
 * MLVS_ERR_STATE, MLVS_ERR_OOM, MLVS_ERR_CUDA. */
mlvs_status mlvs_autotune(mlvs_handle* h, int steps, int* cta_target, float* ms_table);

/* No counterpart in the paper. Set the chunking target directly (one of the values mlvs_autotune
 * chooses from, or any other positive CTA count). */
mlvs_status mlvs_set_tuning(mlvs_handle* h, int cta_target);

/* ----------------------------------------------------------------------------------------
 * Level selector.  Not part of the paper: a 10 -> 64 -> 64 -> 4 ReLU network that predicts a
 * cell's level in a fixed set of four levels from cell features, trained on labels of the
 * criterion, used by mlvs_adapt_mlp with the criterion as fallback below a confidence
 * threshold.  Weights: 5,124 FP32 master values (layout W1 [64][10], b1 [64], W2 [64][64],
 * b2 [64], W3 [4][64], b3 [4]) and their BF16 copy, which the forward and backward passes
 * read with FP32 accumulation.  Reductions run in a fixed order (results reproducible).
 * -------------------------------------------------------------------------------------- */
typedef struct mlvs_mlp mlvs_mlp;

/* Selector, no counterpart in the paper.  Create a network with zero weights; its work is
 * ordered on `stream` (cudaStream_t). */
mlvs_status mlvs_mlp_create(void* stream, mlvs_mlp** out);
void mlvs_mlp_destroy(mlvs_mlp* m);
/* Selector, no counterpart in the paper. host w[5124]: FP32 master weights (the BF16 copy is
 * their nearest-even rounding); resets the momentum. */
mlvs_status mlvs_mlp_set_weights(mlvs_mlp* m, const float* w, int n);
/* Selector, no counterpart in the paper. host master[5124] and/or bf16_values[5124] (the BF16
 * weights as floats); either may be NULL. */
mlvs_status mlvs_mlp_get_weights(const mlvs_mlp* m, float* master, float* bf16_values, int n);
/* Selector, no counterpart in the paper. device X[n][10] -> device logits[n][4] and/or softmax
 * prob[n][4] (either may be NULL); asynchronous on the network's stream. */
mlvs_status mlvs_mlp_forward(mlvs_mlp* m, const float* X, int n, float* logits, float* prob);
/* Selector, no counterpart in the paper. Gradient of the mean softmax cross-entropy of device
 * X[n][10], labels y[n] (0..3) into device grad[5124]; *loss (host, may be NULL) receives the
 * loss. Synchronous. Errors: MLVS_ERR_ARG (a label outside 0..3), MLVS_ERR_OOM, MLVS_ERR_CUDA. */
mlvs_status mlvs_mlp_gradient(mlvs_mlp* m, const float* X, const int* y, int n, float* grad, float* loss);
/* Selector, no counterpart in the paper. One SGD step with momentum on the same batch: v =
 * momentum v + grad, w -= lr v (FP32 master), BF16 copy refreshed. *loss (host, may be NULL):
 * the loss before the step. */
mlvs_status mlvs_mlp_train_step(mlvs_mlp* m, const float* X, const int* y, int n, float lr, float momentum,
                                float* loss);

/* Selector, no counterpart in the paper (features from the moments of Sec. 2.1).  The ten
 * selector features of every cell of one instance (out [ny*nx][10] floats, host or
 * device): log rho, u / sqrt(R T_ref), v / sqrt(R T_ref), log(T / T_ref),
 * q / (rho (RT)^1.5) (two), dx |grad rho| / rho, dx |grad T| / T, dx |grad u| / sqrt(RT),
 * log10 Kn_local (lambda = (mu/p) sqrt(pi R T / 2) over L_ref); gradients by central
 * differences with neighbours wrapped on periodic sides and clamped on the others,
 * dx = min(dx, dy).  Errors: MLVS_ERR_ARG, MLVS_ERR_STATE, MLVS_ERR_CUDA. */
mlvs_status mlvs_features(mlvs_handle* h, int instance, float* out, int out_on_device);

/* Sec. 3.2 masks read with the fixed-level-set rule. The level the fixed-level-set rule
 * (mlvs_set_velocity_levels, adaptive = 0) gives every cell of one instance from its criterion
 * mask (host levels[ny*nx]); the cells do not move. Errors: as mlvs_criterion. */
mlvs_status mlvs_criterion_levels(mlvs_handle* h, int instance, const mlvs_adapt_params* p, int* levels);

/* Selector, no counterpart in the paper.  Fixed-level-set adaptation (adaptive = 0, four levels)
 * with the selector: every cell whose largest softmax probability reaches `confidence` takes
 * the predicted level; the others
 * take the level of the criterion (run on those cells only).  stats->n_distinct receives the
 * number of cells that fell back to the criterion.
 * Errors: MLVS_ERR_ARG (not four levels, adaptive = 1, confidence outside [0, 1]), and as
 * mlvs_adapt. */
mlvs_status mlvs_adapt_mlp(mlvs_handle* h, mlvs_mlp* m, const mlvs_adapt_params* p, float confidence,
                           mlvs_adapt_stats* stats);

/* Extra: the parent-child consistent coarsening index (Sec. 3.2) of a level's space. *nb_out
 * receives its length (N1*N1 in 2-D, N1 in 1-D); out (capacity cap) may be NULL to query it. */
mlvs_status mlvs_level_kappa(const mlvs_handle* h, int level, unsigned char* out, int cap,
                             int* nb_out);

/* field bits for mlvs_moments; fields are written in this bit order */
enum {
  MLVS_RHO = 1, MLVS_U = 2, MLVS_V = 4, MLVS_T = 8, MLVS_QX = 16, MLVS_QY = 32,
  MLVS_LEVEL = 64, MLVS_RHOE = 128, MLVS_SXX = 256, MLVS_SXY = 512, MLVS_SYY = 1024
};
/* Cell moments of one instance at the current time (Eqs. discrete_W, discrete_q):
 * out is [n_fields][ny*nx] doubles (row-major cells), host or device memory (out_on_device).
 * q is the heat flux of phi (q = 2 tau/(2 tau + dt Pr) q~); SXX, SXY, SYY the stress
 * deviator of phi, 2 tau/(2 tau + dt) (P~ - p I) with P~ = sum w c c g~ (c = xi - u).
 * Errors: MLVS_ERR_ARG, MLVS_ERR_STATE, MLVS_ERR_CUDA. */
mlvs_status mlvs_moments(mlvs_handle* h, int instance, unsigned fields, double* out,
                         int out_on_device);

/* No counterpart in the paper (a test accessor). Copy the distributions g~, h~ of cells [cell0,
 * cell0+ncells) of one instance to host arrays out_g/out_h laid out [ncells][nv] (nv of the
 * cell's level; all cells in the range must share a level). *nv_out receives nv. */
mlvs_status mlvs_read_cells(mlvs_handle* h, int instance, int cell0, int ncells,
                            double* out_g, double* out_h, int cap, int* nv_out);

/* Extra: the time step in use (the CFL 0.5 reading of Sec. 4). */
mlvs_status mlvs_time_step(const mlvs_handle* h, double* dt);

/* Conservative moments without device allocation.  The paper has no counterpart: this entry
 * point exists for callers that must not have the library allocate device memory, such as a
 * process that reserves its GPU memory once at start-up and forbids later allocations (an
 * allocation synchronises the device and can fail under memory pressure), or code that records
 * its work into a CUDA graph, where an allocation inside the recorded region breaks it.
 *
 * Input: g, h are caller-owned device arrays of FP32 reduced distributions laid out [nv][ncell]
 * (velocity-plane-major, the library's own layout); xi_x, xi_y, w_x, w_y are device arrays of
 * nv velocity coordinates and per-axis weights (weight = w_x * w_y; D = 1: xi_y = 0, w_y = 1).
 * Output: out is a caller-owned device array [4][ncell] = (rho, rho u, rho v, rho E) in FP64.
 * Work is queued on `stream` (cudaStream_t, NULL = default stream); the call does not wait.
 *
 * Scratch: an 8 MiB file-scope device array (16 velocity chunks x 4 moments x 16384 cells of
 * FP64 partial sums) that every GPU which loads the library holds until the process exits.
 * ncell above 16384 is rejected with MLVS_ERR_ARG.  The library calls no cudaMalloc, cudaFree or
 * other allocating routine here.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call before any stream capture.
 * The address found is kept per device ordinal for the life of the process and belongs to the
 * device's primary context: a host program that destroys that context (cudaDeviceReset) must not
 * call this entry point again on that device.
 * All calls share the one array and leave their partial sums in it; every call overwrites all the
 * entries it later reads, so nothing needs clearing, but calls that overlap on the GPU (on
 * different streams, or different threads) race on the array and must be serialised by the caller.
 * Errors: MLVS_ERR_ARG (null pointer, non-positive or too large sizes), MLVS_ERR_CUDA; the
 * message is available from mlvs_last_error(NULL). */
mlvs_status mlvs_moments_noalloc(const float* g, const float* h, int nv, int ncell,
                                 const float* xi_x, const float* xi_y, const float* w_x,
                                 const float* w_y, double* out, void* stream);

/* ---- Unstructured meshes of polygonal cells, one velocity space ----
 * The DUGKS step of Sec. 2.2 on general polygons (the two-cavity expansion of Sec. 4.5 runs on
 * unstructured cells): Eq. explicit_update with each face's length and outward normal, Eq.
 * reconstruction with a least-squares gradient per cell and velocity (a boundary face adds the
 * cell reflected through it, a zero difference) limited by Venkatakrishnan's function with
 * eps^2 = (K h)^3 P_c^2, K = 1, h = sqrt(area), P_c the cell's value; every boundary face is a
 * diffuse isothermal wall. */
typedef struct mlvs_uhandle mlvs_uhandle;

typedef struct {
  int storage;          /* MLVS_F64 | MLVS_F32: storage and compute type                     */
  double R, K_internal, Pr, omega, mu_ref, T_ref;  /* gas; mu = mu_ref (T/T_ref)^omega (Sec. 4)  */
  double Kn;            /* used when mu_ref <= 0: the VHS relation with alpha = 1, rho_ref = 1,
                           L_ref = 1 (as mlvs_config's Kn)                                    */
  double cfl;           /* dt = cfl * min over cells (area / longest edge) / max |xi|_inf      */
  double dt;            /* > 0: fixed time step instead                                      */
  int compat_cell;      /* 1: four-moment compatibility correction at cells (Sec. 3.3.1)      */
  int compat_face;      /* 1: the same correction of the face model distribution              */
  int limiter;          /* MLVS_LIMITER_VENKAT | MLVS_LIMITER_NONE                            */
  int compat_moments;   /* 4 (or 0): Eq. eq_four_basis; 8: the eight-moment correction of
                           Eq. eq_eight_basis, whose heat-flux target is the model's own
                           (1 - Pr) q and whose deviatoric-stress target is zero            */
  int n_base;           /* velocity space: the n_base x n_base tensor product (Sec. 2.3)      */
  double umin, umax;    /* on [umin, umax]^2                                                  */
  int quadrature;       /* MLVS_QUAD_*                                                        */
  int n_wall;           /* walls named by edge_wall, 1..8                                     */
  double wall[8][3];    /* (u_w, v_w, T_w) of each wall                                       */
  int vpc;              /* velocities per chunk of the moment sums (0: 64)                    */
  void* stream;         /* cudaStream_t the handle orders its work on                         */
} mlvs_uconfig;

/* Sec. 2.2 on polygons; the two-cavity case of Sec. 4.5.  Create a handle on the mesh of
 * mlvs_umesh_geometry (node_xy[n_node][2], counter-clockwise cells in CSR cell_ptr /
 * cell_nodes) with the initial state phi~ = the Maxwellian of init_W[n_cell][4] = (rho, u, v, T),
 * corrected as compat_cell says.  edge_wall[cell_ptr[n_cell]] (NULL: all 0) names the wall of
 * every boundary edge, in the order of cell_nodes (entries of interior edges are ignored).  All
 * inputs are copied.  Device memory: about (8 n_cell + 4 n_face) x nv values of the storage type.
 * Errors: MLVS_ERR_ARG (any defect mlvs_umesh_geometry reports, bad gas constants or space, a
 * boundary edge naming no wall, non-positive initial density or temperature), MLVS_ERR_OOM,
 * MLVS_ERR_CUDA, MLVS_ERR_SINGULAR; the message is available from mlvs_last_error(NULL). */
mlvs_status mlvs_ucreate(const mlvs_uconfig* cfg, int n_node, const double* node_xy, int n_cell,
                         const int* cell_ptr, const int* cell_nodes, const int* edge_wall,
                         const double* init_W, mlvs_uhandle** out);

/* Sec. 2.2, Eqs. phi_update to recover_phi on polygons.  Advance n_steps steps, ordered on the
 * handle's stream; returns after they completed.  *ms (may be NULL) receives their device time.
 * Errors: MLVS_ERR_NONFINITE / MLVS_ERR_POSITIVITY / MLVS_ERR_SINGULAR when a cell or face state
 * failed (the handle then refuses further steps with MLVS_ERR_STATE), MLVS_ERR_CUDA. */
mlvs_status mlvs_ustep(mlvs_uhandle* h, int n_steps, float* ms);

/* No counterpart in the paper.  Copy (g~, h~) to host g[n_cell][nv], hh[n_cell][nv] in the
 * caller's cell order, velocity v = iy * n_base + ix.  Errors: MLVS_ERR_ARG, MLVS_ERR_CUDA. */
mlvs_status mlvs_uread(const mlvs_uhandle* h, double* g, double* hh);

/* Eqs. discrete_W, discrete_q: the cell state at the start of the last step taken (after
 * mlvs_ucreate: zeros), W[11][n_cell] = rho, u, v, T, q_x, q_y, rho E, tau, then the stress
 * deviator of phi (xx, xy, yy), caller's cell order.  Errors: MLVS_ERR_ARG, MLVS_ERR_CUDA. */
mlvs_status mlvs_ucells(const mlvs_uhandle* h, double* W);

/* No counterpart in the paper.  Sizes and time step (each pointer may be NULL). */
mlvs_status mlvs_uinfo(const mlvs_uhandle* h, int* nv, int* n_face, double* dt);

/* No counterpart in the paper.  Release everything the handle owns.  NULL is allowed. */
void mlvs_udestroy(mlvs_uhandle* h);

/* No counterpart in the paper.  Release everything the handle owns.  NULL is allowed. */
void mlvs_destroy(mlvs_handle* h);

/* No counterpart in the paper. Diagnostic text of the last failing call on h (or of the last
 * failing create if h is NULL). */
const char* mlvs_last_error(const mlvs_handle* h);

#ifdef __cplusplus
}
#endif
#endif /* MLVS_H */
