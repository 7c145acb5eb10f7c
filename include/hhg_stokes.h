/*
 * hhg_stokes.h -- C ABI of the GB300 all-at-once Uzawa multigrid Stokes solver.
 *
 * Method (Gmeiner, Huber, John, Ruede, Wohlmuth, "A quantitative performance
 * analysis for Stokes solvers at the extreme scale", arXiv:1511.02134):
 *   - stabilised equal-order P1-P1 Stokes system in the Laplace formulation,
 *     K = [A B^T; B -C], with PSPG stabilisation c_l, g_l (Sec. 2.1, the
 *     linear system of Sec. 3);
 *   - hierarchy by uniform refinement of a macro tetrahedral mesh (Sec. 2.1);
 *   - all-at-once multigrid with the inexact Uzawa smoother (Sec. 3.3),
 *     velocity: symmetric colour Gauss-Seidel (forward + backward sweep,
 *     Sec. 3.4-3.5), pressure: forward colour Gauss-Seidel on C with
 *     under-relaxation omega (Sec. 3.5), variable V-cycle V_var(3,3)
 *     (Sec. 3.5), block-preconditioned MINRES on the coarsest level
 *     (Sec. 3.7), relative-residual stopping rule (Sec. 3.6);
 *   - a mixed-precision mode: FP32 V-cycles inside FP64 iterative refinement.
 *
 * Conventions shared by every entry point
 *   Return value: 0 (HHG_OK) on success, a negative HHG_E* code otherwise.
 *     No function aborts the process; hhg_last_error() gives a message.
 *   Memory: every pointer argument may point to host memory (pageable or
 *     pinned) or to device memory of the mesh's device (unified addressing).
 *     The library copies inputs before returning and never keeps a caller
 *     pointer.  Outputs are written to caller buffers of the documented size.
 *     All device memory is owned by the mesh and released by hhg_destroy.
 *   Streams: all device work of a mesh is ordered on the stream given to
 *     hhg_create_mesh (NULL = a non-blocking stream the library creates,
 *     which does not wait on the legacy default stream).  Device inputs must
 *     be complete with respect to that stream when a call is made.
 *     Functions that return host data synchronise that stream.
 *   Node order: nodal arrays cover the bounding-box lattice of a level,
 *     (n_x, n_y, n_z) nodes with n_a = cells_a * 2^level + 1, node (i,j,k)
 *     at flat index i + n_x (j + n_y k) (x fastest).  Vector fields are
 *     (n, 3) row-major (x, y, z per node); scalar fields (n,).  Values at
 *     nodes that carry no unknown are ignored on input and 0 on output,
 *     except that velocity outputs carry the Dirichlet data on Dirichlet nodes.
 *   Levels: level k means k regular refinements of the macro tetrahedra
 *     (2^k + 1 nodes per macro edge); the paper's level L is k = L + 2.
 */
#ifndef HHG_STOKES_H
#define HHG_STOKES_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HHG_OK 0
#define HHG_EINVAL (-1)     /* bad argument (null pointer, size, level, option) */
#define HHG_EMESH (-2)      /* macro mesh not a set of lattice Kuhn tetrahedra, duplicate or non-manifold */
#define HHG_ENOMEM (-3)     /* device allocation failed */
#define HHG_EDIVERGED (-4)  /* residual became NaN/Inf or grew beyond 1e3 x the initial one */
#define HHG_EMAXIT (-5)     /* tolerance not reached within max_cycles (results still written) */
#define HHG_ECUDA (-6)      /* CUDA runtime error (message in hhg_last_error) */
#define HHG_ESTATE (-7)     /* call out of order (e.g. solve before hhg_set_rhs) */

#define HHG_MODE_FP64 0     /* plain FP64 V-cycles */
#define HHG_MODE_FP32_IR 1  /* FP32 V-cycles inside FP64 iterative refinement */

/* Boundary flags per macro face (face f of a tetrahedron is the face opposite
 * its local vertex f); only faces on the boundary of the macro mesh matter. */
#define HHG_BC_AUTO 0       /* boundary face: Dirichlet */
#define HHG_BC_DIRICHLET 1  /* prescribed velocity (Sec. 2) */
#define HHG_BC_OUTFLOW 2    /* do-nothing boundary nu du/dn - p n = 0 (natural, Sec. 6.1) */
#define HHG_BC_SLIP 3       /* free slip (Sec. 6.1): u . n_i = 0 with the mass-conservative normal
                               n_i = <grad phi_i, 1> / |<grad phi_i, 1>|, and no tangential stress
                               (the momentum rows are tested in the admissible directions only).
                               Where two non-parallel free-slip face planes meet (an obstacle
                               edge) the velocity is along the edge.  A node on a Dirichlet face
                               is Dirichlet; so are corners of three slip planes and nodes whose
                               integral vanishes (slip faces back to back: obstacles touching
                               along an edge or at a corner); they take the boundary data given
                               there.  Nodes also on an outflow face keep the normal n_i */

/* Node flag bits returned by hhg_node_flags. */
#define HHG_NODE_ACTIVE 1   /* carries a pressure unknown */
#define HHG_NODE_VFREE 2    /* carries velocity unknowns */
#define HHG_NODE_IRREG 4    /* near the boundary: some incident tetrahedra are missing (or the
                               mesh is an affine lattice: every active node) */
#define HHG_NODE_DIRICHLET 8
#define HHG_NODE_OUTFLOW 16
#define HHG_NODE_SLIP 32    /* velocity node on a free-slip face (carries HHG_NODE_IRREG) */

/* Solver parameters; hhg_default_options gives the paper's UMG set-up
 * (Tab. "settings" of Sec. 3.7 and the text of Sec. 2.1, 3.5, 4.1). */
typedef struct hhg_options {
  double nu;                 /* viscosity (1) */
  double delta;              /* PSPG parameter delta_T (1/12, Sec. 2.1) */
  double omega;              /* pressure smoother under-relaxation (0.3, Sec. 3.5) */
  int32_t nu_pre;            /* pre-smoothing steps on the finest level (3) */
  int32_t nu_post;           /* post-smoothing steps on the finest level (3) */
  int32_t var_increment;     /* extra steps per coarser level (2: V_var) */
  int32_t coarsest_level;    /* level of the coarse-grid solve (2 = the paper's T_0) */
  int32_t coarse_minres_max; /* MINRES iterations at most (5, Sec. 4.1) */
  double coarse_minres_rtol; /* MINRES relative tolerance (5e-3, Sec. 3.7) */
  int32_t coarse_cg_max;     /* inner CG iterations at most (50) */
  double coarse_cg_rtol;     /* inner CG relative tolerance (1e-3, Sec. 3.7) */
  int32_t use_graphs;        /* 1: replay each V-cycle as a captured CUDA graph */
  int32_t fuse_coarse_levels;/* 1: run the coarse levels (see fuse_max_nodes) and the coarse
                                solve as one fused kernel per cycle; 2: the same with the
                                levels held in the shared memory of one thread-block cluster
                                (falls back to 1 where they do not fit; default); 0: off */
  int32_t fuse_max_nodes;    /* largest level (lattice nodes) of the fused kernel; 0 = default
                                (1024 for mode 1, 65536 for mode 2) */
  int32_t team_blocks;       /* CTAs of the fused kernel's thread-block cluster (1 = one block,
                                at most 16); 0 = default (1 for mode 1; for mode 2, 8 in FP32
                                and 16 in FP64) */
  int32_t fused_min_nodes;   /* FP32 Uzawa steps on levels of at least this many lattice nodes
                                run as three colour-fused passes (a z-march over (x, y) tiles
                                staged into shared memory by tensor copies, several colour
                                phases per pass); 0 = default (never: slower than the
                                per-colour launches on GB300), -1 = never */
  int32_t ir_fixed_point;    /* FP32+IR mode: 1 (default) keeps the refined iterate in 64-bit
                                fixed point (per-field power-of-two scale, updated in integer
                                arithmetic) and evaluates the FP64 refinement residual's
                                regular-node stencils exactly on it; 0: FP64 iterate and
                                residual */
  int32_t spec_max_nodes;    /* levels with fewer lattice nodes evaluate the regular-node update
                                before reading a node's flags (hides load latency on small,
                                latency-bound levels); 0 = default (2^20), -1 = never */
  int32_t colour_block_z;    /* planes per thread block of the colour kernels (1, 2 or 4; 0 =
                                default: 1) */
  int32_t resident_node_lists; /* cluster-resident levels (fuse_coarse_levels 2): 1 runs each
                                velocity / pressure colour phase over per-CTA lists of its
                                regular nodes and then its boundary nodes; 0 = default (1),
                                -1 = over all lattice positions of the colour with flag tests */
  int32_t fused_tile_rows;   /* rows (y) per tile of the fused passes; 0 = chosen per level and
                                pass (most nodes per staged row at the fewest CTA waves) */
  int64_t wait_poll_limit;   /* tests of one mbarrier wait of the fused passes before the pass
                                gives up and reports HHG_ECUDA; 0 = default (2^20) */
  int32_t operator_form;     /* velocity block of the discretisation (Sec. 2.1): 0 = Laplace form
                                a_1 (default), 1 = D form a_2(u, v) = 2 nu <D(u), D(v)> (the
                                velocity smoother then updates the three components of a node
                                at once with its 3 x 3 block; the FP32+IR mode keeps its iterate
                                and refinement residual in FP64) */
  int32_t colour_pairs;      /* 1: FP32 colour kernels of the levels in the flags-first form (see
                                spec_max_nodes) update two neighbouring nodes of the colour per
                                thread with 8-byte loads; 0 = default (off: slower on GB300,
                                the kernels are bound by the loads in flight), -1 = off */
  int32_t fused_wait_test;   /* tests only: 1 makes each fused pass announce 16 bytes more than its
                                first staged plane delivers, so that its first wait runs out (the
                                pass then withdraws them, waits for its copies to land and reports
                                HHG_ECUDA); 0 = off */
  int32_t quad_min_nodes;    /* FP32 Laplace-form levels with at least this many lattice nodes
                                compute the residual four nodes per thread, sharing their
                                neighbours' loads; 0 = default (2^25: the level-9 cube, 5.10 ->
                                4.30 ms; no gain at level 8, a loss at level 7), -1 = never */
} hhg_options;

/* Per-solve statistics. */
typedef struct hhg_stats {
  int32_t cycles;            /* V-cycles performed */
  int32_t status;            /* HHG_OK, HHG_EMAXIT or HHG_EDIVERGED */
  double rel_residual;       /* ||K x - f~|| / ||K x_0 - f~|| at exit */
  double r0;                 /* ||K x_0 - f~|| (FP64, Euclidean over all unknowns) */
  double seconds;            /* wall time of the solve (host clock, stream synchronised) */
  int64_t kernel_launches;   /* kernels launched (graph nodes counted per replay) */
  double history[64];        /* relative residual after cycle c (history[0] = 1) */
  int32_t fx_rescales;       /* FP32+IR fixed point: cycles whose update was redone in FP64
                                with fresh scales (a correction too large for the scale, or
                                the iterate's range grown or shrunk past its bounds) */
} hhg_stats;

typedef struct hhg_mesh hhg_mesh;

/* Fill *opt with the defaults listed above. */
void hhg_default_options(hhg_options* opt);

/* Build the level hierarchy coarsest_level..finest_level on the current CUDA
 * device (Sec. 2.1 refinement, Sec. 3.4 primitives).
 *   macro_vertices: nv x 3 doubles; macro_tets: nt x 4 int32 vertex ids
 *   (0-based); bc_flags: nt x 4 bytes (HHG_BC_*), may be NULL (all AUTO).
 *   Every tetrahedron must be a Kuhn tetrahedron of a cell of a lattice,
 *   with its vertices listed along the path o, o+H e_a, o+H(e_a+e_b),
 *   o+H(1,1,1) or along the reverse path: the order defines the regular
 *   refinement.  The lattice is axis-aligned with spacing H when the first
 *   tetrahedron's edges v1-v0, v2-v1, v3-v2 are axis-aligned of one length;
 *   otherwise it is the affine lattice spanned by those three edges (a
 *   sheared or stretched cube, for example), on which every node takes the
 *   stencil rows of its class (HHG_NODE_IRREG set on every active node)
 *   and nodal arrays cover the bounding box in lattice coordinates.
 *   Otherwise HHG_EMESH.
 *   finest_level >= coarsest_level >= 0, finest_level <= 12.
 *   opt may be NULL (defaults).  cuda_stream: a cudaStream_t or NULL.
 *   On success *out owns all device memory of the hierarchy. */
int hhg_create_mesh(const double* macro_vertices, int64_t nv,
                    const int32_t* macro_tets, int64_t nt,
                    const uint8_t* bc_flags, int32_t finest_level,
                    const hhg_options* opt, void* cuda_stream, hhg_mesh** out);

/* Release every resource of the mesh (NULL is accepted). */
void hhg_destroy(hhg_mesh* mesh);

/* Static message for an error code. */
const char* hhg_strerror(int code);

/* Message of the last failed call on this mesh (or of the last failed
 * hhg_create_mesh when mesh is NULL); never NULL. */
const char* hhg_last_error(const hhg_mesh* mesh);

/* dims[3] = lattice nodes per axis of `level`. */
int hhg_lattice_dims(const hhg_mesh* mesh, int32_t level, int64_t dims[3]);

/* *n = number of lattice nodes of `level` (the length of nodal arrays). */
int hhg_num_nodes(const hhg_mesh* mesh, int32_t level, int64_t* n);

/* Unknown counts of `level`: velocity nodes (3 unknowns each) and pressure
 * nodes; free DoFs = 3 * n_velocity_nodes + n_pressure_nodes (the paper's count). */
int hhg_num_dofs(const hhg_mesh* mesh, int32_t level, int64_t* n_velocity_nodes,
                 int64_t* n_pressure_nodes);

/* Node coordinates of `level`, (n, 3) doubles: origin + h basis (i, j, k). */
int hhg_node_coords(const hhg_mesh* mesh, int32_t level, double* xyz);

/* Node flags (HHG_NODE_* bits) of `level`, n bytes. */
int hhg_node_flags(const hhg_mesh* mesh, int32_t level, uint8_t* flags);

/* Outflow weights w_i = int_{Gamma_out} phi_i n dS of `level`, (n, 3)
 * doubles (zero away from do-nothing faces).  The flux functional of
 * Sec. 6 is J(u) = sum_i w_i . u_i. */
int hhg_outflow_weights(const hhg_mesh* mesh, int32_t level, double* w);

/* Device bytes held by the mesh (fields of all levels and modes allocated so far). */
int hhg_device_bytes(const hhg_mesh* mesh, int64_t* bytes);

/* Right-hand side of the finest level from a nodal body force and Dirichlet
 * data (Sec. 2.1 forms f and g_l with the body force interpolated):
 *   f_h = M (I_h f) on velocity nodes, g_h = sum_d G_d (I_h f)_d,
 *   then the lift f -= A_{I,D} u_D, g -= B_{.,D} u_D; for meshes without
 *   an outflow face g is projected onto range(K) (its mean is removed).
 *   f_nodal: (n, 3) or NULL (= 0); u_dirichlet: (n, 3) or NULL (= 0), read
 *   on Dirichlet nodes only.  Resets the iterate to zero. */
int hhg_set_rhs(hhg_mesh* mesh, const double* f_nodal, const double* u_dirichlet);

/* Initial iterate: u (n, 3) on velocity nodes and p (n,) on pressure nodes;
 * either may be NULL (= 0).  The velocity of a free-slip node is kept
 * tangential (its normal part is dropped).  Call after hhg_set_rhs. */
int hhg_set_initial(hhg_mesh* mesh, const double* u, const double* p);

/* `count` FP64 V_var cycles on the current iterate, each followed by the
 * pressure-mean projection (meshes without outflow).  rel_residual_out
 * (may be NULL) receives ||K x - f~|| / ||K x_before - f~||. */
int hhg_vcycle(hhg_mesh* mesh, int32_t count, double* rel_residual_out);

/* Solve from the current iterate until ||K x_k - f~|| / ||K x_0 - f~|| <= tol
 * (Sec. 3.6) or max_cycles cycles.  mode: HHG_MODE_FP64 or HHG_MODE_FP32_IR.
 * u_out (n, 3) and p_out (n,) may be NULL (the solution stays on the device
 * and can be read with hhg_get_solution).  stats may be NULL.
 * Returns HHG_OK, HHG_EMAXIT (outputs written) or HHG_EDIVERGED. */
int hhg_solve(hhg_mesh* mesh, double tol, int32_t max_cycles, int32_t mode,
              double* u_out, double* p_out, hhg_stats* stats);

/* Full multigrid (Sec. 5).  From a nodal body force and Dirichlet data (as
 * for hhg_set_rhs, which this call also performs for the finest level) the
 * right-hand side is rediscretised on every level from the data's values at
 * that level's nodes.  Starting from zero, the coarsest level is solved by
 * the coarse solver; on every finer level l the iterate starts from the P1
 * interpolant of level l-1's velocity (its Dirichlet values included) and
 * pressure and runs `cycles` V_var(nu, nu) cycles rooted at l
 * (nu + var_increment (l - k) smoothing steps on level k), each followed by
 * the pressure-mean projection on meshes without outflow.  The paper's FMG
 * V_var(2,2) is cycles = 1, nu = 2, its "2V" variant cycles = 2.
 *   mode: HHG_MODE_FP64, or HHG_MODE_FP32_IR (each cycle an FP32 correction
 *   cycle on the level's FP64 residual, the update in FP64; the coarsest
 *   level is solved in FP64 either way).
 *   f_nodal, u_dirichlet: (n, 3) or NULL (= 0), finest lattice order.
 *   u_out, p_out: as hhg_solve (may be NULL); stats (may be NULL): cycles =
 *   V-cycles run, rel_residual = ||K x - f~|| / ||f~|| of the result.
 * The finest iterate stays on the device: hhg_solve may continue from it.
 * Overwrites the right-hand sides and iterates of every level. */
int hhg_fmg_solve(hhg_mesh* mesh, const double* f_nodal, const double* u_dirichlet, int32_t cycles, int32_t nu,
                  int32_t mode, double* u_out, double* p_out, hhg_stats* stats);

/* Current iterate as nodal fields (Dirichlet values included in u). */
int hhg_get_solution(hhg_mesh* mesh, double* u_out, double* p_out);

/* (ku, kp) = K (u, p) on `level` for nodal fields (unknown nodes only;
 * zero elsewhere), FP64.  For tests of the operator. */
int hhg_apply_operator(hhg_mesh* mesh, int32_t level, const double* u, const double* p,
                       double* ku, double* kp);

/* Gradient of a linear functional J(u, p) = sum_i ju_i . u_i + jp_i p_i of
 * the solution with respect to the nodal body force: solves the adjoint
 * system K lambda = (ju, jp) (K is symmetric, Sec. 3) with the same
 * multigrid, then grad_f = R^T lambda with R f = (M f, sum_d G_d f_d).
 * Needs a mesh with an outflow face (non-singular K).  ju (n, 3), jp (n,)
 * (NULL = 0); grad_f (n, 3).  The adjoint iterate starts from zero and is
 * solved to `tol` in `mode`.  The forward iterate is left untouched. */
int hhg_adjoint_gradient(hhg_mesh* mesh, const double* ju, const double* jp, double tol,
                         int32_t max_cycles, int32_t mode, double* grad_f, hhg_stats* stats);

/* ---- step-level access, for parity tests of single kernels ----------------
 * Fields of one level and precision (0 = FP64 hierarchy, 1 = FP32 hierarchy). */
#define HHG_FIELD_U 0   /* velocity iterate, (n, 3) */
#define HHG_FIELD_P 1   /* pressure iterate, (n,) */
#define HHG_FIELD_F 2   /* velocity right-hand side, (n, 3) */
#define HHG_FIELD_G 3   /* pressure right-hand side, (n,) */
#define HHG_FIELD_RU 4  /* velocity residual / smoother scratch, (n, 3) */
#define HHG_FIELD_RP 5  /* pressure residual / smoother scratch, (n,) */

/* write = 1: copy buf into the field (values on non-unknown nodes dropped);
 * write = 0: copy the field into buf.  buf holds doubles in both precisions. */
int hhg_level_field(hhg_mesh* mesh, int32_t level, int32_t precision, int32_t field,
                    int32_t write, double* buf);

#define HHG_OP_UZAWA_STEP 0   /* one inexact Uzawa step on (U, P) with (F, G) */
#define HHG_OP_VEL_FORWARD 1  /* forward velocity colour sweep with RU as right-hand side */
#define HHG_OP_VEL_BACKWARD 2 /* backward velocity colour sweep with RU as right-hand side */
#define HHG_OP_VEL_RHS 3      /* RU = F - B^T P */
#define HHG_OP_PRES_RHS 4     /* RP = B U - G */
#define HHG_OP_PRES_SWEEP 5   /* forward pressure colour sweep with RP */
#define HHG_OP_RESIDUAL 6     /* (RU, RP) = (F, G) - K (U, P) */
#define HHG_OP_RESTRICT 7     /* level-1 (F, G) = P^T (RU, RP) of level, level-1 (U, P) = 0 */
#define HHG_OP_PROLONG_ADD 8  /* (U, P) of level += P (U, P) of level-1 */
#define HHG_OP_COARSE_SOLVE 9 /* (U, P) += MINRES correction on the coarsest level */
#define HHG_OP_VCYCLE 10      /* one V_var cycle rooted at `level` */
#define HHG_OP_PROJECT 11     /* remove the m-weighted pressure mean */
#define HHG_OP_VEL_FORWARD_F 12 /* forward velocity colour sweep with F - B^T P formed at each node
                                   (the velocity colours of an FP32 Uzawa step) */
#define HHG_OP_PRES_SWEEP_F 13  /* forward pressure colour sweep with B U - G formed at each node
                                   (the pressure colours of an Uzawa step) */
#define HHG_OP_REFINE 14        /* finest level, precision 1: FP64 iterate += FP32 correction and
                                   the FP64 residual into the FP32 right-hand side (the refinement
                                   around each FP32 V-cycle) */
#define HHG_OP_CYCLE 15         /* finest level: one cycle of hhg_solve in that precision (FP64:
                                   V-cycle, projection, residual norm; FP32: zeroed correction,
                                   V-cycle, refinement), without the host's convergence test */
#define HHG_OP_FUSED_PASS0 16   /* precision 1, a level with fused passes: pass 0 alone (velocity
                                   colours 0 1 2 3 from (U, P) into RU) */
#define HHG_OP_FUSED_PASS1 17   /* pass 1 alone (velocity colours 2 1, velocity + pressure colour
                                   0, from (RU, P) into (U, RP)) */
#define HHG_OP_FUSED_PASS2 18   /* pass 2 alone (pressure colours 1 2 3 from (U, RP) into P) */

/* Run `op` `count` times on `level` in `precision`. */
int hhg_level_op(hhg_mesh* mesh, int32_t level, int32_t precision, int32_t op, int32_t count);

/* Device time of `reps` back-to-back runs of `op` on `level` (CUDA events on
 * the mesh's stream, after one untimed run); *ms_per_rep receives the mean.
 * The fields are modified as by hhg_level_op, except that HHG_OP_REFINE and
 * HHG_OP_CYCLE with ir_fixed_point skip the per-step check and recovery of
 * the fixed-point iterate (hhg_level_op and hhg_solve do both).  For
 * measurement. */
int hhg_time_op(hhg_mesh* mesh, int32_t level, int32_t precision, int32_t op, int32_t reps,
                double* ms_per_rep);

/* Kernels launched by this mesh so far (graph nodes counted per replay). */
int hhg_kernel_launches(const hhg_mesh* mesh, int64_t* count);

/* Allocations (cudaMalloc and pinned cudaMallocHost calls) made for this mesh
 * so far, including the temporaries of hhg_apply_operator and
 * hhg_level_field that are freed before those calls return. */
int hhg_allocations(const hhg_mesh* mesh, int64_t* count);

/* ---- allocation-free coarse-grid solve ---------------------------------------
 * The paper has no counterpart to this entry point; it exists for callers
 * that must not allocate device memory after set-up: code whose device
 * memory comes from a fixed arena or a framework-owned pool, and real-time or
 * latency-bound loops that cannot afford cudaMalloc/cudaFree (both may block
 * on the whole device and may fail under memory pressure).  Once a mesh has
 * been created (creation allocates), this call performs the coarse-grid
 * MINRES correction of hhg_level_op(HHG_OP_COARSE_SOLVE) without allocating:
 * its scratch is a 2 MiB file-scope device array (held by every GPU that
 * loads the library until the process exits).
 *   f (n, 3), g (n,): right-hand side on the coarsest level; u (n, 3), p (n,):
 *   iterate on input, corrected iterate on output; n = hhg_num_nodes of the
 *   coarsest level; host or device pointers, lattice order.
 *   The mesh's coarsest-level fields and staging buffer are used as work
 *   space, so do not overlap this call with other calls on the same mesh.
 *   Errors: HHG_EINVAL when the coarsest level needs more than 2^18 scratch
 *   doubles (11 (3 nv + np) + 9 nv for nv free velocity nodes and np
 *   pressure nodes), HHG_ECUDA on CUDA errors.  On HHG_EINVAL nothing is
 *   written: neither the caller's u, p nor the mesh's fields.
 *   The first call on a device looks up the array's device address (one
 *   cudaGetSymbolAddress); make that first call before any stream capture.
 *   Every call shares the one array per device, which keeps the last call's
 *   contents; the solve clears what must start at zero.  Calls that overlap
 *   on the GPU, from any mesh or thread, race on the array. */
int hhg_coarse_solve_noalloc(hhg_mesh* mesh, const double* f, const double* g, double* u, double* p);

/* ---- host-only lattice logic (no GPU needed) -------------------------------
 * Classify the nodes of `level` for a macro mesh (same arguments as
 * hhg_create_mesh); flags (n bytes) receives HHG_NODE_* bits and dims[3] the
 * lattice size.  With flags = NULL only dims is written. */
int hhg_lattice_classify(const double* macro_vertices, int64_t nv, const int32_t* macro_tets,
                         int64_t nt, const uint8_t* bc_flags, int32_t level, int64_t dims[3],
                         uint8_t* flags);

/* The saddle-point matrix K of `level` (the forms of Sec. 2.1: a_1 or, with
 * opt->operator_form = 1, a_2; b; the PSPG term c_l; free-slip nodes
 * constrained as in Sec. 6.1: Pi A Pi + (I - Pi), Pi B^T, B Pi), assembled on
 * the host in CSR from the stencil classes and closed-form rows the kernels
 * apply, with the level's scale factors (opt->nu, opt->delta; NULL =
 * defaults).  No device is touched.  Unknowns: the free velocity nodes
 * component by component, then the active pressure nodes, each in lattice
 * order; rows in that order, the pressure rows being (B u - C p).
 * sizes[0] receives the number of rows, sizes[1] of stored entries, sizes[2]
 * of free velocity nodes; with kptr = NULL nothing else is written.  Else
 * kptr (rows + 1), kcol and kval (entries), vnode (velocity nodes) and pnode
 * (rows - 3 velocity nodes) receive the matrix and the lattice index of each
 * unknown's node, and pmass (pressure nodes; NULL = not wanted) the lumped
 * mass of each pressure unknown (the coarse solver's preconditioner and the
 * weights of the pressure mean).  Errors: HHG_EINVAL, HHG_EMESH
 * (hhg_last_error(NULL)). */
int hhg_assemble_operator_host(const double* macro_vertices, int64_t nv, const int32_t* macro_tets,
                               int64_t nt, const uint8_t* bc_flags, int32_t level, const hhg_options* opt,
                               int64_t sizes[3], int32_t* kptr, int32_t* kcol, double* kval,
                               int64_t* vnode, int64_t* pnode, double* pmass);

#ifdef __cplusplus
}
#endif

#endif /* HHG_STOKES_H */
