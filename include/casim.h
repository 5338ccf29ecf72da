/*
 * casim -- collision-aware local-global soft-robot simulation on one GPU.
 *
 * C ABI of the CUDA library.  The method is the paper's projection-based
 * local-global solver with virtual-spring collision response (Fang, Tian,
 * Weightman, Wang, "Collision-Aware Fast Simulation for Soft Robots by
 * Optimization-Based Geometric Computing", Sec. II-III, Algorithm 1).
 *
 * One outer iteration i (the inner while-loop of Algorithm 1, run a fixed
 * number of times) maps positions X_i to X_{i+1}:
 *   1. collision check on X_i (Sec. II-B, Eq. 3, Eq. 4): every non-fixed
 *      boundary vertex strictly inside a tet that does not contain it, or
 *      inside an obstacle sphere;
 *   2. spring update (Sec. II-C, Eq. 5, Sec. III-A.3): create, re-target or
 *      release one virtual spring per boundary vertex;
 *   3. local step (Sec. III-A, Eq. 6, Eq. 7): per-tet rotation by SVD and the
 *      chamber / body target shape;
 *   4. global step (Sec. III-B, Eq. 8): assemble the right-hand side and solve
 *      the SPD system for the free vertex positions by PCG.
 *
 * Conventions for every entry point:
 *   - Return value: 0 (CASIM_OK) on success, a negative CASIM_E_* code on
 *     error, a positive CASIM_W_* code for a warning.  No C++ exception ever
 *     crosses this boundary.  casim_last_error() describes the last failure.
 *   - Host input arrays are copied before the call returns; the caller keeps
 *     ownership.  Output buffers belong to the caller.
 *   - Device pointers ("dev_*") are CUDA device addresses on the device that
 *     was current when the simulation was created.
 *   - All device work is enqueued on the stream given at creation (NULL means
 *     the legacy default stream); the stream belongs to the caller.
 *   - A simulation handle must be used from one host thread at a time.
 *   - Vertex and tet ids are always the caller's ids (0-based, as uploaded).
 */
#ifndef CASIM_H
#define CASIM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define CASIM_OK 0
#define CASIM_E_INVALID (-1)   /* bad argument (null pointer, size, value)      */
#define CASIM_E_CUDA (-2)      /* a CUDA runtime call failed                     */
#define CASIM_E_SINGULAR (-3)  /* a connected component has no fixed vertex      */
#define CASIM_E_STATE (-4)     /* call out of order (e.g. step before upload)    */
#define CASIM_E_CAPACITY (-5)  /* caller's output buffer is too small            */
#define CASIM_E_NONFINITE (-6) /* NaN or Inf met on the device                   */
#define CASIM_E_TIMEOUT (-7)   /* a device-side wait ran out of its budget       */
#define CASIM_E_OVERFLOW (-8)  /* a device work list exceeded its capacity       */
#define CASIM_E_BOUNDS (-9)    /* a checked build met an out-of-range gather
                                  index (see casim_build_checked)                */
#define CASIM_W_PCG_MAXIT 1    /* PCG stopped at its iteration cap (warning)     */
#define CASIM_W_PAIRS_TRUNCATED 2 /* a vertex lay in more tets than
                                     max_pairs_per_vertex; its pair list (not its
                                     spring) was truncated (warning)             */

/* ---- precision modes ---------------------------------------------------- */
#define CASIM_FP64 0   /* every quantity in FP64                                  */
#define CASIM_MIXED 1  /* positions, rotations, targets and PCG vectors in FP32;
                          dot products, norms and PCG scalars in FP64; collision
                          predicates exact                                        */

/* ---- collision modes ---------------------------------------------------- */
#define CASIM_COLLISION_OFF 0
#define CASIM_COLLISION_SELF 1
#define CASIM_COLLISION_SELF_OBSTACLE 2

typedef struct casim_sim casim_sim;

/* Solver parameters.  casim_default_params() fills every field. */
typedef struct {
  int32_t precision;        /* CASIM_FP64 or CASIM_MIXED                              */
  int32_t collision;        /* CASIM_COLLISION_*                                      */
  double k_spring;          /* spring weight k of Eq. 5 (Eq. 8 uses 1)                */
  double eps;               /* contact offset epsilon of Sec. II-C (length units)     */
  double pcg_tol;           /* stop when |r|_2 <= pcg_tol * |b|_2                     */
  int32_t pcg_max_iter;     /* PCG iteration cap per outer iteration                  */
  int32_t n_w_knots;        /* number of (strain, w) knots of R_omega, >= 1           */
  const double* w_knots;    /* host, 2*n_w_knots doubles (eps_i, w_i), eps ascending;
                               copied at casim_create                                 */
  double cell_size;         /* spatial-hash cell edge (length units), > 0             */
  int32_t stats;            /* 1: record the Eq. 8 energy per iteration               */
  int32_t max_pairs_per_vertex; /* self pairs stored per vertex (1..16)              */
  uint64_t wait_budget_cycles;  /* SM clock cycles a grid-barrier wait may spin
                                   before the kernel gives up with CASIM_E_TIMEOUT;
                                   0 selects the default (about 2 s)                 */
  int32_t pcg_kernel;       /* PCG kernel: 0 auto (one robot: MIXED 5 if it fits,
                               else 2 if it fits, else 1; several robots: 4 if it
                               fits, else 3, else 1);
                               1 streaming (whole grid, vectors in memory, any
                               size); 2 register-resident (whole grid, one row per
                               thread, grid barriers); 3 cluster (one 16-CTA
                               cluster per robot, vectors in shared memory, robots
                               from a work queue); 4 segmented streaming (blocks
                               assigned to robots, one CG per robot, shared grid
                               barriers); 5 dataflow (MIXED only: register-resident
                               without grid barriers; every shared value carries
                               its CG epoch and readers wait for the rows they
                               read).
                               A forced kernel that does not fit gives
                               CASIM_E_INVALID at upload                           */
  int32_t debug_flags;      /* test-only fault injection, 0 in normal use:
                               CASIM_DEBUG_BARRIER_NEVER_COMPLETES makes the PCG
                               grid barrier (kernels 1, 2 and 4) or the partial
                               poll (kernel 5) wait for one block more than it
                               has (the cluster kernel uses the hardware cluster
                               barrier), so every wait runs out of
                               wait_budget_cycles and the step ends with
                               CASIM_E_TIMEOUT; CASIM_DEBUG_CORRUPT_INCIDENCE
                               (checked builds only, else CASIM_E_INVALID) plants
                               an out-of-range gather index                      */
  int32_t pcg_precond;      /* preconditioner of the dataflow kernel (5): 0 auto =
                               two-level (Jacobi plus an additive coarse
                               correction over aggregates of a third of a block,
                               Galerkin
                               coarse matrix of the Laplacian, its inverse formed
                               at upload); 1 Jacobi only.  Other kernels use
                               Jacobi                                            */
  int32_t broad_phase;      /* collision broad phase: 0 spatial hash rebuilt every
                               iteration; 1 AABB trees (Sec. II-B) over the tets
                               and the boundary faces, built once at upload (median
                               split of the rest centroids) and refitted every
                               iteration.  Both give the same contact pairs and
                               spring targets (exact leaf tests, same tie rules) */
  int32_t local_block;      /* launch shapes (threads per block; 0 = default):   */
  int32_t rhs_block;        /*   local step 64/128/256 (128), RHS gather          */
  int32_t narrow_block;     /*   128/256/512 (256), narrow phase 128/256/512 (256,
                               one warp per query vertex).  Results do not depend
                               on them except for the summation order of the
                               energy statistic; the autotuner picks them        */
  int32_t pcg_block;        /* rows (threads) per block of the dataflow PCG (5): 0
                               auto = 288 (9 warps; aggregates of 96 rows) when the
                               system fits one such block per SM, else 384
                               (aggregates of 128); 288 or 384 forces it          */
} casim_params;

#define CASIM_DEBUG_BARRIER_NEVER_COMPLETES 1
/* test-only, accepted by checked builds only: the upload writes one entry of
   the vertex-to-tet incidence list out of range on the device, so the right-
   hand-side gather meets it and the step ends with CASIM_E_BOUNDS           */
#define CASIM_DEBUG_CORRUPT_INCIDENCE 2

/* Per-iteration record (Eq. 8 energy at X_i with the targets of iteration i). */
typedef struct {
  double energy;            /* 0 unless params.stats                                 */
  double pcg_rel_residual;  /* |r|/|b| at PCG exit (recursive residual)              */
  int32_t n_self_pairs;     /* |P_self| found on X_i                                 */
  int32_t n_obstacle_pairs; /* |P_obs| found on X_i                                  */
  int32_t n_springs;        /* |V_col| after the spring update                       */
  int32_t pcg_iters;        /* PCG iterations of this outer iteration                */
  /* Signatures of the iteration's discrete state (0 unless params.stats): the
     sum mod 2^64 of a 64-bit mix of (tet id, interval of the w(eps) table its
     strain fell in) over body tets, and of (boundary-vertex index, decision:
     0 self spring kept from its record / 1 sphere spring / 2 tetrahedral-
     obstacle spring / 3 self spring cast in this iteration, face, sphere or
     obstacle face id) over the springs after the update.  Two runs with
     equal signatures at every iteration took the same discrete decisions
     (with overwhelming probability), e.g. the two sides of a finite
     difference. */
  uint64_t knot_signature;
  uint64_t spring_signature;
} casim_iter_record;

typedef struct {
  int64_t iterations;       /* outer iterations run since the last upload            */
  int64_t total_pcg_iters;
  casim_iter_record last;   /* record of the most recent iteration                   */
  int32_t status;           /* device status code of the last casim_sync             */
  int32_t pcg_kernel;       /* PCG kernel chosen at upload (1..5, see casim_params)   */
  int32_t status_bits;      /* OR of every device status word casim_sync has read
                               since the mesh upload: 1 non-finite value, 2 wait
                               timeout, 4 PCG iteration cap, 8 hash / pair
                               overflow, 16 a vertex's pair list truncated at
                               params.max_pairs_per_vertex, 32 an out-of-range
                               input id, 64 an out-of-range gather index
                               (checked builds)                                      */
  int32_t pad;
} casim_stats;

/* Fills *p with the defaults: MIXED, self collision, k = 1, eps = 0.005,
   pcg_tol = 1e-6, pcg_max_iter = 1000, w == 1 (one knot), cell_size = 0.5,
   stats = 1, max_pairs_per_vertex = 8, wait budget default. */
void casim_default_params(casim_params* p);

/* Creates a simulation.  cuda_stream: a cudaStream_t (NULL: default stream).
   Errors: CASIM_E_INVALID for out-of-range parameters. */
int casim_create(const casim_params* params, void* cuda_stream, casim_sim** out);

/* Uploads a tetrahedral mesh M = M_c + M_b (Sec. II-A) and resets the state to
   the rest shape with no springs.
     rest_xyz  host, n_verts*3 doubles, vertex positions of the rest shape V
     tets      host, n_tets*4 int32 vertex ids, positively oriented
               (det[v1-v0, v2-v0, v3-v0] > 0)
     tet_group host, n_tets int32: -1 body element, g >= 0 chamber group g
     fixed     host, n_verts uint8: nonzero = position held fixed
   Errors: CASIM_E_INVALID (ids out of range, non-positive rest volume, group
   ids not dense from 0), CASIM_E_SINGULAR (a connected component without a
   fixed vertex), CASIM_E_CUDA. */
int casim_upload_mesh(casim_sim* sim, int32_t n_verts, const double* rest_xyz, int32_t n_tets,
                      const int32_t* tets, const int32_t* tet_group, const uint8_t* fixed);

/* One robot of a batch (same conventions as casim_upload_mesh). */
typedef struct {
  int32_t n_verts;
  const double* rest_xyz;    /* n_verts*3 */
  int32_t n_tets;
  const int32_t* tets;       /* n_tets*4, ids local to this robot */
  const int32_t* tet_group;  /* n_tets: -1 body, g >= 0 this robot's chamber g */
  const uint8_t* fixed;      /* n_verts */
} casim_mesh_desc;

/* Uploads n_robots independent robots (no counterpart in the paper, which
   simulates one robot; a batching service).  They are simulated together:
   one collision check over all robots that never pairs a vertex with another
   robot's tet, one local step over all tets, and one PCG solve per robot
   (independent stopping tests), all in the same launches.  Afterwards the
   robots behave as one mesh whose vertices, tets and chamber groups are the
   robots' own, concatenated in robot order (robot r's chamber g becomes group
   g + the number of groups of robots 0..r-1), so casim_set_actuation takes
   the concatenated ratios and casim_get_positions the concatenated vertices.
   Obstacle spheres act on every robot.  Each robot needs a fixed vertex in
   every connected component.  Errors as casim_upload_mesh. */
int casim_upload_batch(casim_sim* sim, int32_t n_robots, const casim_mesh_desc* robots);

/* Volume ratios alpha_g per chamber group (Eq. 2; chamber targets are scaled
   by cbrt(alpha_g), Sec. III-A.1).  n_groups must equal 1 + the largest group
   id of the mesh.  Errors: CASIM_E_INVALID (alpha <= 0), CASIM_E_STATE. */
int casim_set_actuation(casim_sim* sim, int32_t n_groups, const double* alpha);

/* Rigid obstacle spheres O_obs (Eq. 4): host, n*4 doubles (cx, cy, cz, r). */
int casim_set_spheres(casim_sim* sim, int32_t n, const double* cxyzr);

/* Rigid tetrahedral obstacle O_obs (Sec. II-B, Eq. 4): the paper builds AABB
   trees over the robot and over the obstacle, with one tetrahedron per leaf.
   A non-fixed robot boundary vertex strictly inside an obstacle tetrahedron
   (exact signs) is in contact with the obstacle; its spring (kind 2 in the
   spring records) targets the closest point of the obstacle's boundary,
   offset by eps along that face's outward normal (Sec. II-C), and is released
   like a self spring once the vertex is more than eps outside the stored face
   point.  When a vertex is also inside a sphere, the obstacle whose signed
   surface distance is smallest wins (spheres on ties).  Requires collision
   mode CASIM_COLLISION_SELF_OBSTACLE to take effect.
     n_verts, xyz   host, n_verts*3 doubles (rounded to the working precision)
     n_tets, tets   host, n_tets*4 int32, positively oriented; 0 removes the
                    obstacle
   The obstacle's AABB trees (tets and boundary faces) are built and fitted
   here; it never moves.  Copies its inputs; replaces any previous obstacle;
   must follow casim_upload_mesh (an upload removes the obstacle).
   Errors: CASIM_E_STATE before an upload, CASIM_E_INVALID for ids out of
   range, non-positive volumes or non-finite positions, CASIM_E_CUDA. */
int casim_set_obstacle_mesh(casim_sim* sim, int32_t n_verts, const double* xyz, int32_t n_tets,
                            const int32_t* tets);

/* Overwrites all vertex positions (host, n_verts*3 doubles, caller order).
   In MIXED mode the values are rounded to FP32.  Clears the last step: the
   next global solve starts from these positions. */
int casim_set_positions(casim_sim* sim, const double* xyz);

/* Asynchronously restores the rest positions (or the positions of the last
   casim_set_positions / casim_load_state call) and clears every spring and
   the last step, on the stream, without host copies.  History and counters
   are kept. */
int casim_reset(casim_sim* sim);

/* Enqueues n_iters outer iterations on the stream (asynchronous).
   Errors: CASIM_E_STATE (no mesh or actuation), CASIM_E_CUDA. */
int casim_step(casim_sim* sim, int32_t n_iters);

/* Runs n_iters outer iterations from the current state (like casim_step)
   while saving a checkpoint of the positions and spring records before
   iterations 0, ckpt_every, 2*ckpt_every, ... for casim_backward (no
   counterpart in the paper; the adjoint is a service built on its loop).
   Memory: ceil(n_iters/ckpt_every) checkpoints plus ckpt_every recomputed
   position sets.  Synchronous with respect to the stream's earlier work only
   through the copies it enqueues; errors as casim_step. */
int casim_forward_ckpt(casim_sim* sim, int32_t n_iters, int32_t ckpt_every);

/* Reverse pass of the last casim_forward_ckpt: given dL/dX of the final
   positions (host, n_verts*3 doubles, caller order; rows of fixed vertices
   are ignored) writes dL/dalpha (host, n_groups doubles) for the chamber
   volume ratios.  The discrete decisions of each iteration (contact pairs,
   spring kinds, faces and spheres, which springs were cast) are held fixed,
   so the result is the derivative of the unrolled map on the region of
   parameters where those decisions do not change.  Each segment between
   checkpoints is recomputed; the final forward state and the history
   counters are restored afterwards.  Errors: CASIM_E_STATE (no preceding
   casim_forward_ckpt, or the actuation or positions changed since),
   CASIM_E_NONFINITE, CASIM_E_CUDA.  Synchronises the stream. */
int casim_backward(casim_sim* sim, const double* dL_dX, double* dL_dalpha);

/* Waits for the stream and returns the device status: CASIM_OK,
   CASIM_W_PCG_MAXIT, CASIM_W_PAIRS_TRUNCATED, CASIM_E_NONFINITE,
   CASIM_E_TIMEOUT or CASIM_E_OVERFLOW (a tet's box spans more than 512 hash
   cells or the hash entries exceed 16 per tet and face: contacts may be lost).
   The device status is cleared after it is read. */
int casim_sync(casim_sim* sim);

/* Current positions, caller order, as n_verts*3 doubles into host_out (may be
   NULL) and/or as n_verts*3 values of the working precision (float in MIXED,
   double in FP64) into dev_out (may be NULL).  Synchronises the stream when
   host_out is given. */
int casim_get_positions(casim_sim* sim, double* host_out, void* dev_out);

/* Contact sets found by the last collision check (on X_i of the last
   iteration run): self pairs (v, e) sorted by (v, e) into pairs[2*k], and the
   vertices inside an obstacle sphere (sorted) into obstacle_verts.  On entry
   *n_pairs / *n_obst hold the capacities (in pairs / vertices); on exit the
   counts.  Returns CASIM_E_CAPACITY (with the counts set) when too small.
   A vertex whose self pairs exceeded max_pairs_per_vertex keeps the smallest
   tet ids and sets the CASIM_W_PAIRS_TRUNCATED device status. */
int casim_get_contacts(casim_sim* sim, int32_t* pairs, int64_t* n_pairs, int32_t* obstacle_verts,
                       int64_t* n_obst);

/* Spring records after the last spring update, one per non-fixed boundary
   vertex in ascending vertex id.  Any output pointer may be NULL.
     verts   int32 vertex id            active  uint8 1 = spring present
     kind    int32 0 self, 1 obstacle   face    int32 boundary face id (self),
                                                 sphere id (obstacle), -1 none
     bary    2 doubles (weights of the face's 2nd and 3rd vertex)
     target  3 doubles, the spring's other end v_c
   *n (in: capacity, out: count).  Boundary faces are numbered by (tet id,
   local face k), face k being the face opposite the tet's k-th vertex. */
int casim_get_springs(casim_sim* sim, int64_t* n, int32_t* verts, uint8_t* active, int32_t* kind,
                      int32_t* face, double* bary, double* target);

/* Replaces the spring records (same layout as casim_get_springs; verts must
   list the non-fixed boundary vertices in ascending order). */
int casim_set_springs(casim_sim* sim, int64_t n, const int32_t* verts, const uint8_t* active,
                      const int32_t* kind, const int32_t* face, const double* bary,
                      const double* target);

/* Element targets of the last local step: host n_tets*12 doubles, P_e as a
   row-major 3x4 matrix per tet (not weighted by omega_e). */
int casim_get_targets(casim_sim* sim, double* host_out);

/* Per-iteration records of the last min(cap, iterations) iterations, oldest
   first; *n receives the count. */
int casim_get_history(casim_sim* sim, int32_t cap, casim_iter_record* out, int32_t* n);

int casim_get_stats(casim_sim* sim, casim_stats* out);

/* Saves / restores positions and spring records (checkpoint / resume), and
   the last outer iteration's step x_i - x_(i-1), from which the next global
   solve of the single-robot MIXED path starts (so a resumed run repeats the
   uninterrupted one bit for bit).  casim_save_state with buf == NULL stores
   the required size in *len.  casim_load_state also accepts the earlier
   layout without the step (the next solve then starts from x_i). */
int casim_save_state(casim_sim* sim, void* buf, size_t* len);
int casim_load_state(casim_sim* sim, const void* buf, size_t len);

/* Sizes of the uploaded mesh (any pointer may be NULL). */
int casim_get_sizes(casim_sim* sim, int32_t* n_verts, int32_t* n_tets, int32_t* n_free,
                    int32_t* n_boundary_faces, int32_t* n_query_verts);

/* Last launch configuration and device time split of the previous
   casim_step (milliseconds per phase: collision, springs, local, rhs, pcg),
   measured with CUDA events when params.stats >= 2; zero otherwise. */
int casim_get_phase_times(casim_sim* sim, double* ms_out5);

/* Allocation-free contact check (no counterpart in the paper; a service for
   callers that cannot allocate device memory while they run, such as real-time
   controllers that must not allocate inside a control loop, or host programs
   whose own allocator owns the GPU memory pool and forbids outside
   cudaMalloc calls).

   Computes the self-collision pairs of Eq. 3 exactly as a casim_step
   iteration does (spatial hash + exact strict point-in-tet test), for
   positions given by the caller, without allocating: all intermediate data
   lives in one static device array of about 6.2 MiB that every GPU which
   loads the library holds until the process exits.
     n_verts, dev_xyz   device, n_verts*3 floats, vertex positions
     n_tets, dev_tets   device, n_tets*4 int32 vertex ids (16-byte aligned),
                        positively oriented
     n_query, dev_query device, n_query int32 vertex ids to test
     cell_size          hash cell edge (length units), > 0
     max_pairs          pairs kept per query vertex, 1..16
     dev_pair_count     device, n_query int32: number of tets strictly
                        containing the vertex (capped at max_pairs)
     dev_pair_tet       device, n_query*max_pairs int32: their tet ids,
                        ascending, in the first dev_pair_count[q] slots
     cuda_stream        cudaStream_t (NULL: default stream)
   Limits: n_verts <= 32768, n_tets <= 65536, n_query <= 16384; larger sizes
   are rejected with CASIM_E_INVALID before any GPU work.  Other errors:
   CASIM_E_INVALID (null or misaligned pointer, id out of range, bad
   cell_size / max_pairs), CASIM_E_OVERFLOW (more pairs than max_pairs for
   some vertex, or more hash entries than the scratch holds),
   CASIM_E_NONFINITE, CASIM_E_CUDA.  Ids are checked on the device before
   any position is read through them.  casim_last_error(NULL) on the calling
   thread tells which check failed.
   Calls no cudaMalloc or cudaFree.  The first call on a device looks up the
   static array's device address (cudaGetSymbolAddress), so make that first
   call outside any stream capture.  The address is cached per device for the
   life of the process and does not survive cudaDeviceReset.  The call waits for its stream before it
   returns.  Every call reuses the same array, which keeps the last call's
   contents (the call clears what must start at zero): calls whose GPU work
   overlaps, from several host threads or streams, race with each other. */
int casim_contacts_noalloc(int32_t n_verts, const float* dev_xyz, int32_t n_tets, const int32_t* dev_tets,
                           int32_t n_query, const int32_t* dev_query, double cell_size, int32_t max_pairs,
                           int32_t* dev_pair_count, int32_t* dev_pair_tet, void* cuda_stream);

/* Remesh trigger (Sec. III-C; Algorithm 1, the check after the inner loop).
   Remeshing itself is not part of this library; this reports which chamber
   elements (tet_group >= 0) would trigger it.  For every chamber element,
   F is the affine map taking the element's reference shape to its current
   shape (F = D_cur D_ref^-1, D the edge matrix v1 - v0, v2 - v0, v3 - v0):
     bit 1 (value 1): volume change  det F = Vol(cur) / Vol(ref) > alpha_max
     bit 2 (value 2): distortion     largest singular value of F > d_max
   (the paper's norm of the diagonal factor of F's SVD), evaluated in FP64 from
   the current positions.  Body elements get 0.  The paper uses
   alpha_max = d_max = 4.
     ref_xyz             host, n_verts*3 doubles in the caller's vertex order:
                         the reference shape (Algorithm 1 compares with the
                         shape at the previous outer step); NULL = rest shape
     flags_out           host, n_tets bytes, caller's tet order (written)
     n_flagged           host, number of elements with any flag (may be NULL)
     group_volume_ratio  host, n_groups doubles (may be NULL): per chamber
                         group, the sum of current over the sum of reference
                         element volumes
   Synchronous: waits for the work queued on the simulation's stream.
   Returns CASIM_E_INVALID for bad arguments (n_groups must equal 1 + the
   largest group id when group_volume_ratio is given). */
int casim_remesh_flags(casim_sim* sim, const double* ref_xyz, double alpha_max, double d_max,
                       uint8_t* flags_out, int32_t* n_flagged, int32_t n_groups,
                       double* group_volume_ratio);

/* One outer step of casim_progressive. */
typedef struct {
  int32_t k;                       /* outer step, from 1                                   */
  int32_t status;                  /* casim_sync of the step's inner loop (0 or a warning) */
  int32_t n_volume;                /* chamber elements with bit 1 against the step's start */
  int32_t n_distortion;            /* chamber elements with bit 2 against the step's start */
  int32_t n_flagged;               /* chamber elements with either bit                     */
  int32_t pad;
  double applied_max;              /* largest volume ratio applied at this step             */
  double chamber_volume_ratio_min; /* smallest per-group chamber volume ratio against rest  */
  double chamber_volume_ratio_max; /* largest one                                          */
} casim_outer_record;

/* Progressive actuation: the outer loop of Algorithm 1 without the
   remeshing step.  Outer step k = 1, 2, ... sets the volume ratios
   a_g = min(alpha_target[g], k * alpha_step) (the paper's alpha_k = k alpha_max,
   capped so that the last step applies exactly the target), runs n_inner
   iterations of the loop from the current state (positions and springs carry
   over), and records the remesh flags of the step against the shape it
   started from and the chamber volume ratios against the rest shape.  It stops
   after the step that applies every target, or after max_outer steps.
     alpha_target   host, n_groups volume ratios (> 0)
     records        host, room for max_outer records; *n_outer gets the count
   Synchronous.  Leaves the targets' last applied ratios set.  Errors of the
   inner loop are returned as by casim_sync. */
int casim_progressive(casim_sim* sim, int32_t n_groups, const double* alpha_target, double alpha_step,
                      int32_t n_inner, int32_t max_outer, double alpha_max, double d_max,
                      casim_outer_record* records, int32_t* n_outer);

/* One step of casim_step_anderson. */
typedef struct {
  double e_prev;     /* Eq. 8 energy at x_k, the point the step came from (NaN without a proposal) */
  double e_acc;      /* energy at the accelerated proposal                                         */
  int32_t accepted;  /* 1: the proposal became x_{k+1}; 0: x_{k+1} = g_k                         */
  int32_t proposed;  /* 1: a proposal was formed (history non-empty, solve succeeded)           */
} casim_aa_record;

#define CASIM_AA_MAX_M 16

/* Anderson acceleration of the loop (Sec. III-B: the paper accelerates the
   local-global iteration with the method of Peng et al. 2018).  Runs n_iters
   iterations x_k -> g_k = G(x_k) of the loop (as casim_step) from the current
   state and, with memory m (0 <= m <= CASIM_AA_MAX_M; 0 = plain loop), after
   each one forms the proposal x_acc = g_k - dG theta, where dF, dG hold the
   differences of the last m + 1 residuals f_j = g_j - x_j and images g_j, and
   theta solves (dF^T dF + lambda I) theta = dF^T f_k, lambda = 1e-12
   trace(dF^T dF) / m.  Safeguard (Peng et al.'s energy test): the proposal
   becomes x_{k+1} only if its Eq. 8 energy is below that of x_k, both with the
   local projections at the point and iteration k's spring targets;
   otherwise x_{k+1} = g_k.
   Each call starts with an empty history.
     records     host, n_iters records (may be NULL)
     n_accepted  host, number of accepted proposals (may be NULL)
   Synchronous (waits for its work); the history records of casim_get_history
   are those of the n_iters loop iterations.  Errors as casim_step. */
int casim_step_anderson(casim_sim* sim, int32_t n_iters, int32_t m, casim_aa_record* records,
                        int32_t* n_accepted);

void casim_destroy(casim_sim* sim);

/* Message of the last failure on this handle.  With sim NULL: the message of
   the last failure, on the calling host thread, of a call that takes no
   handle (casim_create, casim_contacts_noalloc).  Valid until the next call
   on the handle (or the next handle-free call on the thread). */
const char* casim_last_error(const casim_sim* sim);

/* 1 when the library was built with -DCASIM_CHECKED (libcasim_checked.so):
   every gather index of the hot kernels (tet and face vertices, hash items,
   incidence entries, matrix columns, PCG halo rows and columns, cast list) is
   checked on the device, and an index outside its array sets a status bit
   and reads element 0 instead, so the step ends with CASIM_E_BOUNDS rather
   than an out-of-range access.  It stands in for a memory checker.  0
   otherwise.  No error. */
int casim_build_checked(void);

#ifdef __cplusplus
}
#endif

#endif /* CASIM_H */
