/* ipcsim: one IPC time step on one GPU (sm_103a), behind a plain C ABI.
 *
 * What a step computes (Eq. 3 and §III-C.2 of the paper): the positions at
 * t+1 minimise one incremental potential over every free degree of freedom,
 *
 *   E(z) = 1/2 (z - z~)^T M (z - z~)
 *        + dt^2 [ E_FEM + E_barrier + E_friction + E_stitch + E_ABD + E_joint ],
 *
 * with E_FEM the Neo-Hookean energy of the tetrahedral fingertips and
 * deformable objects (§III-C.1), E_barrier the log-barrier contact potential
 * on point-triangle and edge-edge pairs, E_friction the lagged, smoothly
 * mollified friction potential, E_stitch the stitch springs of Eq. 2 that
 * attach fingertip vertices to the gripper bases, and E_ABD the stiff
 * orthogonality energy of affine bodies (§III-C.1).  Kinematic bodies
 * (arm links and finger bases in the grasping scenes) follow the rigid
 * transforms given to each step; links modelled as affine bodies are instead
 * driven by E_joint, the quadratic joint drive potentials of Eq. 3 (springs
 * between body-frame points and directions of two affine bodies, or of one
 * body and the world, with per-step targets), and are solved with
 * everything else.  The step is a projected Newton iteration with a
 * preconditioned PCG linear solve, an additive-CCD bound on every step length
 * and a backtracking line search, so no pair of primitives ever
 * interpenetrates.
 *
 * Conventions for every entry point
 *   - Units are SI.  Positions are double, row-major (n, 3).
 *   - Pointers named *_host point to host memory and are read (or written)
 *     during the call only; the caller keeps ownership.  Pointers named
 *     *_dev are CUDA device pointers of the library's device.
 *   - A 3x4 transform is 12 doubles, row-major [R | t]: x = R xbar + t.
 *   - ABD generalised coordinates q are 12 doubles [p, A(:,0), A(:,1), A(:,2)]
 *     with x = p + A xbar.
 *   - Every call returns IPC_OK (0) or a negative ipc_status; no call aborts
 *     or exits.  sim_last_error() gives a human-readable reason.
 *   - On a failed sim_step the state stays at the start of that step.
 *   - All device work is enqueued on the stream given to sim_create.
 */
#ifndef IPCSIM_H
#define IPCSIM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ipcsim ipcsim;
typedef int ipc_status;

enum {
  IPC_OK = 0,
  IPC_ERR_ARG = -1,           /* bad argument or scene description */
  IPC_ERR_INVERTED = -2,      /* a rest tetrahedron has non-positive volume */
  IPC_ERR_INTERSECTING = -3,  /* initial state has a pair at zero distance */
  IPC_ERR_NEWTON_MAXIT = -4,  /* Newton did not reach the tolerance */
  IPC_ERR_PCG = -5,           /* PCG broke down (p^T A p <= 0) */
  IPC_ERR_LS_STALL = -6,      /* line search halved 40 times without decrease */
  IPC_ERR_NAN = -7,           /* non-finite energy, gradient or direction */
  IPC_ERR_BVH_OVERFLOW = -8,  /* BVH traversal stack overflow */
  IPC_ERR_CUDA = -9,          /* a CUDA runtime call failed */
  IPC_ERR_CAPACITY = -10      /* a pair buffer could not grow */
};

/* Scene description, read once by sim_create.  Vertex ids are 0-based and
 * local to their body (FEM ids index fem_X). */
typedef struct {
  /* deformable (FEM) bodies: tetrahedral meshes (§III-C.1) */
  int n_fem_verts;
  const double* fem_X_host;     /* (n_fem_verts, 3) rest = initial positions */
  const double* fem_V0_host;    /* (n_fem_verts, 3) initial velocity, or NULL for 0 */
  int n_tets;
  const int* tets_host;         /* (n_tets, 4), positively oriented */
  const double* logE_host;      /* (n_tets) ln Young's modulus */
  const double* nu_host;        /* (n_tets) Poisson ratio */
  const double* rho_host;       /* (n_tets) density */
  const int* fem_body_host;     /* (n_tets) FEM body id, or NULL for one body */
  /* affine bodies (ABD): closed outward triangle meshes in body frame */
  int n_abd;
  const int* abd_nverts_host;   /* (n_abd) */
  const double* abd_X_host;     /* concatenated (sum nverts, 3) */
  const int* abd_ntris_host;    /* (n_abd) */
  const int* abd_tris_host;     /* concatenated (sum ntris, 3), ids local to the body */
  const double* abd_rho_host;   /* (n_abd) density */
  const double* abd_q0_host;    /* (n_abd, 12) initial q */
  /* kinematic bodies: arm links, finger bases, plates, fixed obstacles */
  int n_kin;
  const int* kin_nverts_host;   /* (n_kin) */
  const double* kin_X_host;     /* concatenated local rest vertices */
  const int* kin_ntris_host;    /* (n_kin) */
  const int* kin_tris_host;     /* concatenated, ids local to the body */
  const double* kin_T0_host;    /* (n_kin, 12) transforms at t = 0 */
  /* stitch springs of Eq. 2: FEM vertex -> point fixed to a kinematic body */
  int n_stitch;
  const int* stitch_v_host;     /* (n_stitch) FEM vertex id */
  const int* stitch_b_host;     /* (n_stitch) kinematic body id */
  const double* stitch_X_host;  /* (n_stitch, 3) anchor in that body's frame */
  double gravity[3];
  /* joint drives of Eq. 3 (E_joint, revolute and prismatic joints as
   * quadratic drive potentials): joint j adds
   *   E_j = k_j / 2 | J_a q_a - J_b q_b - t_j |^2
   * where q_a, q_b are the q of affine bodies a and b, J q = p + A v for a
   * body-frame point v (kind 0) and A v for a body-frame direction (kind 1).
   * Body b = -1 is the world (its term drops; t_j is then a world point or
   * direction).  A revolute joint is two point springs on the hinge axis plus
   * a direction spring whose b-side direction turns with the drive angle; a
   * prismatic joint is a point spring whose b-side point slides with the
   * drive offset.  The b-side vectors and t change per step
   * (sim_set_joint_targets); a-side vectors are fixed. */
  int n_joints;
  const int* joint_body_host;   /* (n_joints, 2) bodies a (>= 0) and b (>= -1), ABD ids of this scene */
  const int* joint_kind_host;   /* (n_joints, 2) 0 point, 1 direction, for sides a and b */
  const double* joint_vec_host; /* (n_joints, 2, 3) v on side a, initial v on side b (body frames) */
  const double* joint_k_host;   /* (n_joints) stiffness (N/m for points, J for directions), >= 0 */
  const double* joint_t_host;   /* (n_joints, 3) initial target offset t (world frame) */
} ipc_scene_desc;

enum { IPC_PREC_FP64 = 0, IPC_PREC_MIXED = 1 };

typedef struct {
  double dt;          /* time step (s) */
  double dhat;        /* barrier activation distance (m) */
  double kappa;       /* barrier stiffness; <= 0: kbar / B''(dhat/2), kbar = E_max * mean soft edge */
  double mu;          /* friction coefficient */
  double eps_v;       /* friction velocity threshold (m/s); mollifier width eps_v * dt */
  double k_c;         /* stitch stiffness (N/m); <= 0: 100 * E_max * mean soft edge */
  double kappa_A;     /* ABD orthogonality stiffness (Pa) */
  double newton_tol;  /* stop when max|p| / (dt * L_bbox) < newton_tol and kinematic DOFs reached */
  double pcg_rtol;    /* PCG stops when |r|_2 <= pcg_rtol |b|_2 */
  double s_ccd;       /* ACCD minimum-separation fraction (0.1) */
  int max_newton;     /* Newton iteration cap */
  int max_pcg;        /* PCG iteration cap; <= 0: 10 * sqrt(n_dof) + 100 */
  int precision;      /* IPC_PREC_FP64 or IPC_PREC_MIXED */
  int pair_capacity;  /* initial contact-pair capacity; <= 0: automatic (grows on demand) */
  int broad_phase;    /* IPC_BROAD_LBVH (default) or IPC_BROAD_ALL_PAIRS (every pair tested; for checks) */
  int pair_capacity_max; /* largest contact-pair buffer (pairs) the simulator grows to; a step that needs
                            more fails with IPC_ERR_CAPACITY; <= 0: 2^23 */
  int preconditioner; /* IPC_PRECOND_TWO_LEVEL (default) or IPC_PRECOND_BLOCK_JACOBI */
  int coarse_rebuild; /* two-level coarse matrix: 0 rebuilt at the first Newton iteration of every step
                         (default); n > 0 kept up to n steps while the PCG iterations per solve stay
                         within 30 % of the step it was built in; -1 rebuilt at every Newton iteration */
  int kappa_adaptive; /* adaptive barrier stiffness (IPC's kappa growth; the paper keeps IPC's barrier
                         without stating its stiffness policy): != 0: after every Newton iteration whose
                         iterate had its smallest primitive distance below kappa_dmin * dhat while that
                         distance had not grown since the step's previous iterate, the scene's kappa
                         doubles, up to kappa_max_factor times its initial value; kappa carries over to
                         the following steps.  sim_adjoint is not available with it. */
  double kappa_dmin;       /* fraction of dhat (<= 0: 1e-2) */
  double kappa_max_factor; /* (<= 0: 100) */
} ipc_params;

/* PCG preconditioners (the paper names StiffGIPC's solver without its
 * details; both are this library's).  Block Jacobi: the inverse 3x3 diagonal
 * blocks.  Two-level: block Jacobi plus a coarse correction
 * P (P^T A P)^-1 P^T whose columns are the rigid-body motions (3
 * translations, 3 rotations about the centre) of runs of FEM row segments of
 * the PCG launch (at most 768 coarse unknowns per solve); P^T A P is
 * assembled and inverted (FP64 Gauss-Jordan) as coarse_rebuild says.
 * Number FEM vertices in spatial order (e.g. Morton order) so that row
 * segments are compact clusters. */
enum { IPC_PRECOND_TWO_LEVEL = 0, IPC_PRECOND_BLOCK_JACOBI = 1 };

enum { IPC_BROAD_LBVH = 0, IPC_BROAD_ALL_PAIRS = 1 };

typedef struct {
  int status;             /* ipc_status of the step */
  int newton_iters;
  int pcg_iters_total;
  int pcg_iters_max;
  int n_pairs_max;        /* most active barrier pairs seen in one iterate */
  int n_friction_pairs;   /* lagged friction pairs of the step */
  int n_ccd_max;          /* most CCD candidates seen in one iteration */
  int ls_halvings;        /* total line-search halvings */
  double alpha_min;       /* smallest accepted step fraction */
  double min_dist;        /* smallest primitive distance over the accepted iterates (m) */
  double energy_end;      /* incremental potential at the solution */
  double pnorm_end;       /* max|p| / (dt L) of the last Newton direction */
  int pcg_unconverged;    /* PCG solves that stopped at max_pcg (or stagnated) above pcg_rtol: the
                             Newton direction of those iterations is inexact (the step still ends
                             only when the Newton test holds) */
  int pcg_fallbacks;      /* two-level solves that broke down or ended far above pcg_rtol (the coarse
                             inverse not positive definite on that system) and were repeated with
                             block Jacobi; their iterations are in pcg_iters_total */
  double kappa_end;       /* barrier stiffness of the first scene after the step */
} ipc_step_stats;

/* Build a simulator of the scene the paper's physics layer simulates
 * (§III-C.1: FEM soft bodies, ABD rigid bodies, IPC contact; Eqs. 1-2: the
 * fingertips coupled to the gripper by stitch springs; §III-C.2: arm links
 * driven along the planned motion).  Validates the scene (IPC_ERR_INVERTED for a rest tet
 * with det(Dm) <= 0), prepares rest shapes, masses, the BSR pattern and the
 * contact surfaces on the host, uploads them, and allocates device memory
 * with cudaMalloc.  stream: a cudaStream_t (NULL = legacy default stream). */
ipc_status sim_create(const ipc_scene_desc* desc, const ipc_params* params, void* stream, ipcsim** out);

/* Batched data generation (the paper's pipeline generates many simulated
 * demonstrations, Fig. 2 and §III-C.3; running several independent scenes
 * in one simulator is this library's, the paper does not describe it): one
 * simulator for n independent scenes.  The
 * scenes are concatenated (FEM vertices, tets, ABD bodies, kinematic bodies
 * and stitch springs in scene order, ids shifted accordingly); pairs between
 * different scenes are never formed; every scene keeps its own barrier and
 * stitch stiffness (auto-scaled from its own material and mesh).  One
 * sim_step then advances all scenes with one shared Newton loop in which
 * every scene keeps its own control: its own convergence test (with the
 * smallest scene bounding box as L_bbox), CCD step bound and backtracking
 * line search, so each advances as it would alone; a converged scene stops
 * moving while the others continue.  The linear systems are solved in one
 * cooperative launch holding one independent PCG solve per scene (its own
 * scalars, tolerance and stop; converged scenes are left out) when every
 * scene's rows are contiguous, there are at most 256 scenes and the launch
 * has room for CTAs of every scene; otherwise one solve covers the whole
 * block-diagonal system.  sim_step takes the kinematic transforms of all
 * scenes concatenated; sim_get_state / sim_set_state use the concatenated
 * layout.  Gravity is taken from the first scene. */
ipc_status sim_create_batch(const ipc_scene_desc* descs, int n, const ipc_params* params, void* stream, ipcsim** out);

/* Device-memory hook (not part of the paper's method: it lets a host
 * framework own the simulator's device memory, e.g. PyTorch's caching
 * allocator).  alloc returns `bytes` of device memory of the current device
 * for use on `stream` (the simulator's stream), or NULL on failure; free
 * returns a block alloc gave, with the same stream (work already queued on it
 * may still read the block, so a caching allocator must order its reuse after
 * that work, as stream-ordered allocators do).  ctx is passed through. */
typedef struct {
  void* (*alloc)(size_t bytes, void* stream, void* ctx);
  void (*free)(void* ptr, void* stream, void* ctx);
  void* ctx;
} ipc_allocator;

/* sim_create (n == 1) or sim_create_batch (n > 1) with every device buffer
 * of the simulator taken from `allocator` (required) instead of cudaMalloc:
 * the scene data, the state, the work buffers, the contact-pair and
 * candidate lists (which grow on demand during sim_step), the BVHs and the
 * PCG buffers.  Blocks are given back when a list grows and at sim_destroy.
 * Pinned host staging buffers still come from cudaMallocHost.  The
 * allocator must stay valid until sim_destroy. */
ipc_status sim_create_with_allocator(const ipc_scene_desc* descs, int n, const ipc_params* params,
                                     const ipc_allocator* allocator, void* stream, ipcsim** out);

/* Device memory accounting: out3 = [blocks taken from the caller's
 * allocator, blocks taken by cudaMalloc, bytes held now]. */
ipc_status sim_memory(const ipcsim* sim, long long* out3);

/* Advance one time step (Eq. 3).  kin_T_next_host: (n_kin, 12) transforms of
 * the kinematic bodies at t+1 (may be NULL when n_kin == 0).  stats_host may
 * be NULL.  Synchronises the stream once per Newton iteration to read the
 * convergence data and returns when the step is done. */
ipc_status sim_step(ipcsim* sim, const double* kin_T_next_host, ipc_step_stats* stats_host);

/* Advance n independent simulators by one step each (Eq. 3 for each; the
 * concurrency is this library's, not described in the paper), concurrently: every
 * simulator runs its own Newton loop (its own convergence, step lengths and
 * line search) on its own stream, driven from its own host thread, so the
 * kernels of different scenes overlap on the GPU.  Simulators must be
 * distinct, each created with its own stream, and of the current device.
 * kin_T_next_host[i] as for sim_step (may be NULL for scenes without
 * kinematic bodies, or the whole array NULL); stats_host and status_host
 * (n entries each) may be NULL.  Returns IPC_OK if every step succeeded,
 * else the first failing status. */
ipc_status sim_step_many(ipcsim* const* sims, int n, const double* const* kin_T_next_host, ipc_step_stats* stats_host,
                         ipc_status* status_host);

/* The simulated part of the trajectory record of Eq. 4 (X_deform, the
 * deformable positions; T_rigid, the affine bodies' q).  Copy the state out: FEM positions and velocities (n_fem_verts, 3) and ABD
 * q / qdot (n_abd, 12).  Any pointer may be NULL.  `on_device` != 0 means the
 * pointers are device pointers, else host pointers.  Synchronous. */
ipc_status sim_get_state(const ipcsim* sim, double* x, double* v, double* abd_q, double* abd_qd, int on_device);

/* Every vertex position of the current state in the global vertex order
 * (FEM vertices, ABD surface vertices x = p + A xbar, kinematic vertices at
 * their current transforms) into xv_dev ((n_vertices_all, 3) doubles,
 * device): the geometry a frame of Eq. 4's trajectory is rendered from.
 * Synchronous. */
ipc_status sim_positions(const ipcsim* sim, double* xv_dev);

/* Overwrite the state (same layouts; e.g. to restart a rollout of Eq. 3 from
 * a recorded step).  Kinematic bodies keep their pose. */
ipc_status sim_set_state(ipcsim* sim, const double* x, const double* v, const double* abd_q, const double* abd_qd,
                         int on_device);

/* Counts: [n_fem_verts, n_tets, n_abd, n_kin, n_surface_tris, n_surface_edges,
 * n_surface_verts, n_nodes, bsr_blocks] written to out9. */
ipc_status sim_sizes(const ipcsim* sim, int* out9);

/* Derived scalars fixed at create: [kappa, k_c, L_bbox, dhat] (kappa: the
 * barrier stiffness of E_barrier in Eq. 3; k_c: the stitch stiffness of
 * Eq. 2; both auto-scaled when the parameters leave them 0, the paper gives
 * no values). */
ipc_status sim_scalars(const ipcsim* sim, double* out4);

/* Place the kinematic bodies (the arm links and finger bases that follow the
 * planned motion of §III-C.2; T_link of Eq. 4) at the given transforms (host, (n_kin, 12)),
 * e.g. to restart a trajectory from an earlier step together with
 * sim_set_state. */
ipc_status sim_set_kinematic(ipcsim* sim, const double* kin_T_host);

/* Material and friction parameters (§III-C.1 specifies the FEM material by
 * Young's modulus and Poisson ratio; mu is the friction coefficient of
 * E_friction in Eq. 3) for the following steps (the parameters
 * the adjoint differentiates): per-tet ln Young's modulus (n_tets host
 * doubles, or NULL to keep) and the friction coefficient (mu < 0 keeps it).
 * The barrier stiffness and stitch stiffness fixed at create do not change. */
ipc_status sim_set_params(ipcsim* sim, const double* logE_host, double mu);

/* Joint drive targets for the following steps (E_joint of Eq. 3: the
 * reference trajectory q_ref enters only through these): vec_b_host
 * (n_joints, 3) the b-side body-frame vectors, t_host (n_joints, 3) the
 * target offsets, all joints of all scenes concatenated; either may be NULL to
 * keep it.  sim_adjoint uses the targets set last, so set those of the step
 * being differentiated before calling it.  IPC_ERR_ARG on a non-finite value. */
ipc_status sim_set_joint_targets(ipcsim* sim, const double* vec_b_host, const double* t_host);

/* Implicit adjoint of one step (implicit function theorem applied to the
 * minimisation of Eq. 3; the paper's simulator is not differentiated, this
 * is an extension for identifying material and friction parameters from
 * trajectories).  Given the
 * state at t (z_t_dev, zd_t_dev: DOF vectors (n_nodes, 3), FEM vertices then
 * ABD pseudo-nodes), the converged state z_next_dev of the step t -> t+1, the
 * kinematic transforms at t and t+1 (host, (n_kin, 12)) and the loss
 * gradients gz_next_dev, gzd_next_dev w.r.t. z_{t+1} and zd_{t+1} = (z_{t+1} - z_t)/dt:
 * recomputes the unprojected Hessian H at z_next, solves H lam = gz + gzd/dt
 * by FP64 PCG (relative residual 1e-12; IPC_ERR_PCG if H is not positive
 * definite there) and writes gz_t_dev = dL/dz_t and gzd_t_dev = dL/dzd_t
 * (overwritten), adds dL/dlogE into glogE_dev (n_tets, may be NULL) and
 * dL/dmu into *gmu_host (may be NULL).  dL/dz_t includes the dependence of
 * the lagged friction data (normal forces, normals and closest-point weights,
 * all computed at x_t) on x_t.  Uses the simulator's work buffers; the
 * simulator's state is not changed. */
ipc_status sim_adjoint(ipcsim* sim, const double* z_t_dev, const double* zd_t_dev, const double* z_next_dev,
                       const double* kin_T_t_host, const double* kin_T_next_host, const double* gz_next_dev,
                       const double* gzd_next_dev, double* gz_t_dev, double* gzd_t_dev, double* glogE_dev,
                       double* gmu_host);

/* Launch shape of the cooperative PCG (the linear solve inside every Newton
 * iteration of Eq. 3's minimisation; the paper names StiffGIPC's solver
 * without its parallel layout, this is the library's): threads per FEM row (rowg = 1, 2, 4
 * or 8; <= 0 keeps the current value) and CTAs per SM (1 to 4; <= 0 keeps;
 * fewer are launched when the kernel cannot keep that many resident).  With
 * autotune_next_step != 0 the next sim_step times every shape (2 x 4) on its
 * first linear system and keeps the fastest.  out4 (may be NULL) receives
 * [rowg, blocks_per_sm, CTAs of the last PCG launch (0 before the first),
 * 1 if that launch kept its operator rows in shared memory]; ms8 (may be
 * NULL) the last autotuning times in ms, index 4 * (blocks_per_sm - 1) +
 * log2(rowg) (-1: no co-resident plan with that shape). */
ipc_status sim_tuning(ipcsim* sim, int rowg, int blocks_per_sm, int autotune_next_step, int* out4, float* ms8);

/* Where the cooperative PCG keeps its operator (the solver of the Newton
 * step; the paper does not describe its solver's layout).  streamed == 0
 * (default): each CTA copies its rows of the BSR operator and of the
 * block-Jacobi preconditioner into shared memory once per solve when every
 * CTA's rows fit, else they are read from global memory in every iteration;
 * streamed != 0: always read from global memory.  Both give the same
 * arithmetic in the same order.  Takes effect at the next solve. */
ipc_status sim_pcg_residency(ipcsim* sim, int streamed);

/* The coarse level of the two-level preconditioner as last built: out4 =
 * [aggregates (FEM CTAs of the launch), independent solves, coarse unknowns
 * of the largest solve (6 per aggregate), 1 if the last build succeeded
 * (0: that solve ran with block Jacobi alone)]. */
ipc_status sim_coarse_info(const ipcsim* sim, long long* out4);

/* Accounting of the library, no counterpart in the paper.  Per-stage timing
 * with CUDA events recorded on the simulator's stream
 * around each stage of sim_step (cheap; intervals are read at the
 * synchronisation points sim_step already has).  enable == 1 starts (and
 * clears) accounting, enable == 2 resumes it without clearing, 0 pauses it
 * (keeping what was accumulated); sim_profile_read returns accumulated milliseconds and
 * interval counts per stage [PCG, elastic, barrier, culling, CCD, friction,
 * other, PCG setup (incidence lists, FP32 copies, operator layout)] and work4
 * = [PCG iterations, sum over iterations of barrier
 * pairs, of friction pairs, BSR blocks]. */
ipc_status sim_profile(ipcsim* sim, int enable);
ipc_status sim_profile_read(const ipcsim* sim, double* ms8, long long* n8, long long* work4);

/* Host only (no GPU, no simulator): the partition of the rows among the CTAs
 * of a cooperative PCG launch of `grid` CTAs, as sim_step plans it (block-
 * Jacobi PCG of the Newton system, the solver of the Newton step; the paper
 * does not describe its solver's parallel layout).  row: (nf + 4 nab + 1)
 * BSR row offsets, FEM rows first, then the 4 pseudo-node rows of every ABD
 * body; node_scene: (nf + 4 nab) scene of every row, or NULL with
 * n_scenes = 1 (one solve); row_extra: (nf) added cost of every FEM row, or
 * NULL (every FEM row costs its stored blocks + 2, plus this; sim_step
 * passes none in this version).  Outputs
 * (caller-owned): out4 = [FEM CTAs, ABD
 * CTAs, independent solves (n_scenes when every scene got CTAs of its own,
 * else 1), most FEM rows of one CTA]; seg (grid + 1): FEM row boundaries of
 * the FEM CTAs; abd_seg (grid + 1): body boundaries of the ABD CTAs;
 * cta_scene (grid): the solve every CTA serves (-1: none).  IPC_ERR_ARG for
 * NULL outputs or non-positive sizes. */
ipc_status sim_pcg_partition(const int* row, int nf, int nab, int grid, const int* node_scene, int n_scenes,
                             const int* row_extra, int* out4, int* seg, int* abd_seg, int* cta_scene);

/* Measured arithmetic roofs of the current device (not part of the paper's
 * method: they are the denominators of the solver kernels' roofline, which
 * on this part is set by the FP64 pipe rather than by memory): out2[0] =
 * FP64 FMA rate, out2[1] = FP32 FMA rate, both in TFLOP/s (2 flops per FMA),
 * from independent register FMA chains on every SM, best of five timed
 * launches (about 0.2 s in all).  Allocates a small scratch buffer;
 * synchronises the device's legacy default stream. */
ipc_status sim_device_peaks(double* out2);

/* Accounting of the library, no counterpart in the paper.  Total number of
 * CUDA kernels this library has launched in this process
 * (all simulators, all threads), for launch accounting. */
unsigned long long sim_kernel_launches(void);

/* Error reporting of the library, no counterpart in the paper.  Reason of the
 * last failure of `sim`; with sim == NULL, of the last failed
 * sim_create on the calling thread. */
const char* sim_last_error(const ipcsim* sim);
void sim_destroy(ipcsim* sim);

/* ------------------------------------------------------------------------
 * Stage entry points (the hot-path kernels one by one, for parity checks
 * and profiling).  Positions are device pointers to (n_vertices_all, 3)
 * doubles in the library's global vertex order: FEM vertices, then the
 * ABD surface vertices body by body, then the kinematic vertices body by
 * body (sim_sizes gives the counts).
 * ---------------------------------------------------------------------- */

/* E_FEM of Eq. 3, the Stable Neo-Hookean energy of §III-C.1.  Elastic energy,
 * gradient (n_fem_verts, 3) and, if H_dev != NULL, the
 * per-tet 12x12 Hessians (n_tets, 144), PSD-projected when project != 0, at
 * FEM positions x_dev (n_fem_verts, 3).  Energies are V_e Psi (not scaled by
 * dt^2).  E_dev: one double.  grad_dev is overwritten. */
ipc_status sim_eval_elastic(ipcsim* sim, const double* x_dev, int project, double* E_dev, double* grad_dev,
                            double* H_dev);

/* The contact pairs of IPC (§III-C.1: barrier potentials between primitives
 * closer than dhat).  Active contact pairs at all-vertex positions x_dev: every point-triangle
 * and edge-edge pair with squared distance < dhat^2 after the exclusion
 * rules.  Records (cap, 8) int32: kind (0 PT / 1 EE), primitive a, primitive b,
 * distance type, 4 vertex ids; s_dev (cap) squared distances.  Writes the
 * count to *n_host.  Returns IPC_ERR_CAPACITY (with the needed count in
 * *n_host) when cap is too small.  Primitive numbering: surface vertices,
 * triangles and edges as returned by sim_surface. */
ipc_status sim_active_pairs(ipcsim* sim, const double* x_dev, int cap, int* rec_dev, double* s_dev, int* n_host);

/* The contact surfaces of the bodies of §III-C.1.  Surface topology (host
 * buffers of sizes from sim_sizes): surface vertex
 * ids, triangles (3 ids), edges (2 ids), all in the global vertex order. */
ipc_status sim_surface(const ipcsim* sim, int* sv_host, int* tris_host, int* edges_host);

/* E_barrier of Eq. 3 (the log barrier of IPC).  Barrier energy kappa * sum
 * m_k b(s_k) (not scaled by dt^2), its gradient
 * with respect to the free DOF nodes (n_nodes, 3: FEM vertices, then the 4
 * pseudo-nodes of each ABD body) and the per-pair vertex-space 12x12
 * Hessians (n, 144), PSD-projected when project != 0, of n pair records (as
 * from sim_active_pairs) at x_dev.  Allocates scratch with cudaMalloc. */
ipc_status sim_eval_barrier(ipcsim* sim, const double* x_dev, int n, const int* rec_dev, int project, double* E_dev,
                            double* grad_dev, double* H_dev);

/* sim_eval_barrier without device allocation.  The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory once
 * they run (a control loop on a fixed memory budget, or a process in which
 * another allocator owns the device memory), because sim_eval_barrier
 * allocates its scratch with cudaMalloc on every call.  Same arguments,
 * outputs and error codes as sim_eval_barrier; the caller still provides
 * every input and output buffer.  Its scratch is one static device array of
 * 2^20 8-byte slots (8 MiB) that every GPU loading this library holds until
 * the process exits (its sums are kept as three-word order-independent
 * accumulators, 48 slots per node); scenes needing more (more than about
 * 21 800 nodes) are rejected with IPC_ERR_ARG and a message naming the size.  The first call
 * on a device looks up the array's device address (cudaGetSymbolAddress)
 * with that device current.  With CUDA's lazy module loading (the default)
 * that first call may also load this library's device code onto the device,
 * and with it the 8 MiB array: make the first call early, before the device
 * memory is handed to another allocator and before any stream capture.
 * All calls share the array and it keeps the previous call's contents (the
 * call clears what it accumulates into): calls that overlap on the GPU, from
 * any simulator, race.  No cudaMalloc, cudaFree or allocating library
 * routine is called. */
ipc_status sim_eval_barrier_noalloc(ipcsim* sim, const double* x_dev, int n, const int* rec_dev, int project,
                                    double* E_dev, double* grad_dev, double* H_dev);

/* The continuous collision detection of §III-C.1 (the guarantee of no
 * interpenetration).  Largest step fraction in (0, 1] along the vertex displacement p_dev
 * (n_vertices_all, 3) from x_dev: minimum additive-CCD time of impact over
 * all pairs whose swept boxes overlap.  *n_cand_host: candidates tested. */
ipc_status sim_ccd_alpha(ipcsim* sim, const double* x_dev, const double* p_dev, double* alpha_host, int* n_cand_host);

/* ------------------------------------------------------------------------
 * Physics-to-render dual-mesh mapping (§III-D.1, Eqs. 5-6): the render mesh
 * of a deformable body is its simulation surface after L levels of Loop
 * subdivision, precomputed as one sparse matrix W (N_fine x N_coarse, Eq. 5);
 * every frame X_f = W X_c (Eq. 6).
 * ---------------------------------------------------------------------- */
typedef struct ipc_dual_mesh ipc_dual_mesh;

/* Build W for the coarse triangle mesh tris_host ((n_tris, 3) ids into
 * n_verts coarse vertices; outward orientation is kept by the subdivision)
 * and 0 <= levels <= 6 (Loop's rules per level: an interior edge vertex
 * 3/8 (a + b) + 1/8 (c + d), a boundary edge vertex (a + b) / 2, an old
 * vertex of valence n (1 - n beta) v + beta sum of neighbours with
 * beta = (5/8 - (3/8 + cos(2 pi / n) / 4)^2) / n, a boundary vertex
 * 3/4 v + 1/8 of each boundary neighbour; new vertices follow the old ones,
 * one per edge in increasing (min id, max id) order).  Host work; with
 * upload != 0 also one upload of W (CSR: int row offsets, int columns,
 * double weights) with cudaMalloc (upload == 0: host only, for
 * sim_dual_mesh_topology; sim_dual_mesh_apply then returns IPC_ERR_ARG).
 * IPC_ERR_ARG for ids out of range or levels outside [0, 6]. */
ipc_status sim_dual_mesh_create(const int* tris_host, int n_tris, int n_verts, int levels, int upload,
                                ipc_dual_mesh** out);
/* out4 = [N_coarse, N_fine, fine triangles, nonzeros of W]. */
ipc_status sim_dual_mesh_sizes(const ipc_dual_mesh* m, long long* out4);
/* Host copies (any may be NULL): fine triangles (fine triangles, 3); W as CSR:
 * row offsets (N_fine + 1), columns and weights (nonzeros). */
ipc_status sim_dual_mesh_topology(const ipc_dual_mesh* m, int* fine_tris_host, int* row_host, int* col_host,
                                  double* val_host);
/* X_f = W X_c on the device: xc_dev (N_coarse, 3), xf_dev (N_fine, 3),
 * enqueued on `stream` (a cudaStream_t); does not synchronise. */
ipc_status sim_dual_mesh_apply(const ipc_dual_mesh* m, const double* xc_dev, double* xf_dev, void* stream);
/* Reason of the last failed sim_dual_mesh_create on the calling thread. */
const char* sim_dual_mesh_last_error(void);
void sim_dual_mesh_destroy(ipc_dual_mesh* m);

/* ------------------------------------------------------------------------
 * Headless path tracer of the simulated frames (§III-D.2, "real-time path
 * tracing", with the appearance-preserving shadow-receiving material of
 * §III-D.3, Eq. 7), written as plain CUDA (no graphics API): triangles in an
 * LBVH rebuilt per frame, one thread per pixel, spp paths of up to max_depth
 * diffuse bounces with next-event estimation toward the area lights, linear
 * RGB out (no tone mapping; the LUT calibration of §III-D.4 needs real frames).
 * ---------------------------------------------------------------------- */
enum { IPC_MAT_DIFFUSE = 0,      /* Lambertian; rgb = albedo */
       IPC_MAT_EMISSIVE = 1,     /* area light (two-sided); rgb = radiance */
       IPC_MAT_BACKGROUND = 2,   /* reconstructed background, Eq. 7; rgb = C_tex of the triangle; paths end here */
       IPC_MAT_TRANSPARENT = 3   /* thin sheet: paths pass with throughput x rgb; casts no shadow */ };

typedef struct {
  int n_verts;
  int n_tris;
  const int* tris_host;    /* (n_tris, 3) vertex ids */
  const int* type_host;    /* (n_tris) IPC_MAT_* */
  const float* rgb_host;   /* (n_tris, 3) colour of the material (see IPC_MAT_*) */
} ipc_render_scene;

typedef struct {
  float eye[3], fwd[3], right[3], up[3];  /* pinhole camera: unit forward, right, up */
  float tan_half_fov;                     /* tan of half the vertical field of view */
  int width, height;
} ipc_camera;

typedef struct {
  int spp;                  /* paths per pixel */
  int max_depth;            /* diffuse bounces after the first hit */
  int n_shadow;             /* N light samples of the visibility V of Eq. 7 */
  float lambda_s;           /* shadow strength lambda_s of Eq. 7, in [0, 1] */
  float eps;                /* ray offset from a surface (m) */
  unsigned long long seed;  /* every random number is a hash of (seed, pixel, sample, dimension) */
} ipc_render_params;

typedef struct ipc_render ipc_render;

/* Upload the topology and materials (host arrays, copied).  The light
 * triangles (IPC_MAT_EMISSIVE) are sampled in proportion to their area.
 * IPC_ERR_ARG for ids out of range or an unknown material. */
ipc_status sim_render_create(const ipc_render_scene* scene, ipc_render** out);
/* Render one frame at vertex positions x_dev ((n_verts, 3) doubles, device)
 * into rgb_dev ((height, width, 3) floats, device, row-major from the top
 * left), enqueued on `stream` (a cudaStream_t); does not synchronise.  The
 * frame is a deterministic function of its inputs (counter-based random
 * numbers; FP32 arithmetic without contraction). */
ipc_status sim_render_frame(ipc_render* r, const double* x_dev, const ipc_camera* cam, const ipc_render_params* p,
                            float* rgb_dev, void* stream);
/* Reason of the last failed sim_render_create on the calling thread. */
const char* sim_render_last_error(void);
void sim_render_destroy(ipc_render* r);

#ifdef __cplusplus
}
#endif
#endif /* IPCSIM_H */
