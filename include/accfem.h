/*
 * accfem.h -- C ABI of the GB300 (sm_103a) contact-FEM hot path of Acc-FEM
 * (H. Chen et al., "Accelerated Quasi-Static FEM for Real-Time Modeling of Continuum
 * Robots with Multiple Contacts and Large Deformation", arXiv 2503.06922).
 *
 * One handle = one robot in one lumen, resident on the current CUDA device.  A call to
 * accfem_solve is one quasi-static step of the paper (Sec. II-III): Newton iterations, each
 * made of the corotational element force/tangent and their block-tridiagonal assembly
 * (Eq. 20, Sec. III.C), node-vs-triangle collision detection (Eq. 3-10, Sec. III.C), the
 * block factorisation and the contact-space solve of the QP of Eq. 23 through its LCP
 * (Eq. 12-13, 22), and the step limiter (Eq. 25-27).  Every step runs in CUDA kernels.
 *
 * Units: metres, newtons, newton-metres, radians; all reals are IEEE binary64.
 * Node i has material arc length s_i = i L / M; node 0 is the base, node M the tip.
 * Quaternions are (w, x, y, z) and map the section triad to global coordinates
 * (column 0 = robot axis, column 1 = entrance_up at rest).
 *
 * Ownership: every pointer argument is host memory owned by the caller, read or written
 * only during the call (inputs are copied at create); the handle owns all device memory.
 * Calls are synchronous on the handle's stream.  A handle is not thread-safe: use one
 * host thread per handle.  No call aborts: every failure is reported as a status and, for
 * calls taking a handle, a message retrievable with accfem_last_error.
 */
#ifndef ACCFEM_H
#define ACCFEM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct accfem_handle accfem_handle;

#define ACCFEM_MAX_CABLES 8     /* cables per robot; also the row stride of batched tensions     */

typedef enum {
  ACCFEM_OK = 0,
  ACCFEM_E_INVALID_ARG = 1,     /* a descriptor, option or argument is out of range        */
  ACCFEM_E_NOMEM = 2,           /* device or host allocation failed                          */
  ACCFEM_E_CUDA = 3,            /* a CUDA runtime call failed (message has the CUDA error)    */
  ACCFEM_E_NOT_CONVERGED = 4,   /* max_newton_iters reached; best iterate is still returned   */
  ACCFEM_E_CONTACT_CAPACITY = 5,/* more constraint rows than max_contacts / result capacity  */
  ACCFEM_E_NOT_SPD = 6,         /* a non-positive pivot in the tangent factorisation          */
  ACCFEM_E_TIMEOUT = 7,         /* the contact LCP exceeded max_contact_iters pivots          */
  ACCFEM_E_PENETRATION = 8      /* reserved: converged state violates non-penetration         */
} accfem_status;

/* Robot (Sec. II.A-B, Table 1 columns): hollow circular section, M equal two-node 6-DOF
 * beam elements of length l0 = length / n_elements.  Cables (Eq. 16-18): cable j is welded
 * to the tip at distance cable_radius from the axis, at angle cable_angles[j] from the
 * section's second axis towards its third; n_cables <= ACCFEM_MAX_CABLES. */
typedef struct {
  double length, outer_radius, inner_radius, youngs_modulus, poisson_ratio;
  int32_t n_elements;           /* M >= 1; N = M + 1 nodes                                  */
  int32_t n_cables;             /* 0..8                                                       */
  double cable_radius;
  const double* cable_angles;   /* n_cables values (radians)                                 */
} accfem_robot_desc;

/* Lumen (Eq. 3, Sec. III.C): triangle soup, outward winding (counter-clockwise seen from
 * outside the lumen).  The clamp that feeds the robot sits at entrance_point, pushing along
 * entrance_dir; entrance_up fixes the rest section triad (orthogonalised against dir). */
typedef struct {
  const double* vertices;       /* 3 * n_vertices, xyz                                       */
  int64_t n_vertices;
  const int32_t* triangles;     /* 3 * n_triangles vertex indices; n_triangles may be 0       */
  int64_t n_triangles;
  double entrance_point[3], entrance_dir[3], entrance_up[3];
} accfem_lumen_desc;

/* Options.  Defaults (accfem_default_options): activation_gap 1e-3 m (a constraint row is
 * created when the clearance to a locally closest wall feature is below r_o + gap),
 * step_limit beta0 = 5e-4 m (Eq. 25-26, applied to the largest nodal translation),
 * newton_tol 1e-11 m (stop when the unlimited step has max(|du_i|, r_o |dtheta_i|) below it
 * and the constraint set did not change), contact_tol 1e-11 (relative sign tolerance of the
 * LCP pivoting), max_newton_iters 200, max_contact_iters 1000, max_contacts 256 (constraint
 * rows, at most 8192), tangent_mode 0 (material tangent K = B^T K_l B; the only mode on the GPU).
 * The contact solve of a Newton iteration runs over a working set of at most min(max_contacts, 512)
 * rows: the rows active or violated in the previous iteration and the rows whose gap is at most
 * step_limit / 5; every other row is checked against the applied step (a violated row joins the
 * working set and the iteration cannot converge), so a converged solve solves the contact problem
 * of all rows. */
typedef struct {
  double activation_gap, step_limit, newton_tol, contact_tol;
  int32_t max_newton_iters, max_contact_iters, max_contacts, tangent_mode;
} accfem_options;

/* Result of one solve.  The caller owns every buffer; node_pos holds 3*(M+1) doubles,
 * node_quat 4*(M+1); the contact arrays hold contact_capacity entries (contact_point and
 * contact_normal 3 per entry).  On return n_contacts is the number of constraint rows of
 * the last Newton iteration (if it exceeds contact_capacity only the first
 * contact_capacity are written and the status is ACCFEM_E_CONTACT_CAPACITY).
 * contact_force[i] >= 0 is the multiplier y_i of Eq. 11 (newtons along -normal on the
 * robot) of the last Newton step (at convergence: the equilibrium contact force); contact_normal points from the robot to the far side of the wall (Eq. 3).
 * base_reaction is the force and moment (global) that the clamp exerts on the last
 * prescribed node, i.e. F(x) at that node (Eq. 14-15).  residual is max |F - F_a + A_c^T y|
 * over the free DOFs at the last iterate. */
typedef struct {
  double* node_pos;
  double* node_quat;
  int32_t contact_capacity;
  int32_t n_contacts;
  int32_t* contact_node;
  int32_t* contact_tri;
  double* contact_point;
  double* contact_normal;
  double* contact_force;
  double base_reaction[6];
  int32_t newton_iters, contact_iters;
  double residual;
} accfem_result;

/* Warm start: full nodal poses to start the Newton iterations from (prescribed nodes are
 * reset to their clamp poses). */
typedef struct {
  const double* node_pos;   /* 3*(M+1) */
  const double* node_quat;  /* 4*(M+1) */
} accfem_state;

/* Fills *out with the defaults above.  E_INVALID_ARG if out is NULL. */
accfem_status accfem_default_options(accfem_options* out);

/* Creates a handle on the current CUDA device: copies robot and lumen, builds the lumen's
 * uniform grid, allocates all device memory for M elements and max_contacts rows.
 * options may be NULL (defaults).  On failure *out is NULL and the status says why.  The handle
 * records its device: calls that launch work on it (solves, state reads, kernel timing, the
 * allocation-free query, batches of it) return ACCFEM_E_INVALID_ARG with a message when another
 * device is current. */
accfem_status accfem_create(const accfem_robot_desc* robot, const accfem_lumen_desc* lumen,
                            const accfem_options* options, accfem_handle** out);

/* One quasi-static step (Sec. II-III): cable tensions (n_cables values, >= 0) mapped to the
 * tip load of Eq. 16-18 (follower), insertion depth in [0, length] (nodes with
 * s_i <= length - insertion are clamped on the entrance axis), optional warm start (NULL:
 * the resident state of the previous call moved along the robot's own path by the change of
 * insertion, or the straight pose on the first call).  Writes *out (see accfem_result).
 * On E_NOT_CONVERGED the last iterate is still written and becomes the resident state. */
accfem_status accfem_solve(accfem_handle* h, const double* cable_tensions, double insertion,
                           const accfem_state* warm, accfem_result* out);

/* Same step with a direct tip load instead of the cables: force f and moment m, given in the
 * tip section frame and following it (follower != 0) or fixed in global axes (follower == 0).
 * Used to check the path against closed forms (cantilever, end moment, ...). */
accfem_status accfem_solve_tip_load(accfem_handle* h, const double f[3], const double m[3],
                                    int32_t follower, double insertion, const accfem_state* warm,
                                    accfem_result* out);

/* Same step as accfem_solve, with cable_tensions in DEVICE memory and no result copied back:
 * the solution stays resident (read it with accfem_get_state).  newton_iters (may be NULL)
 * receives the iteration count.  For callers that keep their inputs on the GPU. */
accfem_status accfem_solve_resident(accfem_handle* h, const double* device_cable_tensions,
                                    double insertion, int32_t* newton_iters);

/* Forgets the resident state: the next solve without warm start begins from the straight pose. */
accfem_status accfem_reset(accfem_handle* h);

/* Makes the handle enqueue its work on the caller's CUDA stream (a cudaStream_t passed as
 * void*; NULL restores the handle's own stream).  Calls stay synchronous with respect to it. */
accfem_status accfem_set_stream(accfem_handle* h, void* stream);

/* Arithmetic of the element kernel.  ACCFEM_PRECISION_FP64 (the default): everything FP64.
 * ACCFEM_PRECISION_MIXED: the element tangent products (K_l B E^T and the 78 entries of
 * K = (B E^T)^T K_l B E^T) take FP32 operands with FP32 accumulation; the element force (the
 * Newton residual), the factorisation, the contact Schur complement and the contact solve stay
 * FP64.  Collision always prunes in FP32 and decides in FP64.  The tangent only steers the Newton
 * iteration, whose FP64 residual refines every step, so a converged solve meets the same
 * tolerance in both modes.  The assembled tangent's condition number grows like the cube of the
 * element count, past FP32 precision from a few hundred elements: when the FP32 tangent gives a
 * non-positive pivot, the solve switches to the FP64 tangent and repeats that iteration
 * (accfem_solve_stats reports it).  A batch takes each member's mode when the batch is created. */
#define ACCFEM_PRECISION_FP64 0
#define ACCFEM_PRECISION_MIXED 1
accfem_status accfem_set_precision(accfem_handle* h, int32_t mode);

/* Per-element Young's modulus (Sec. II.A: the robot is not uniform; its distal section is much
 * less rigid than the rest).  youngs_modulus: host array of n_elements moduli in Pa, element e
 * joining nodes e and e + 1 (node 0 at the base), copied before return; NULL restores the robot's
 * own modulus everywhere.  The section (radii) and Poisson's ratio stay the robot's, so element e
 * has EA = E_e A, EI = E_e I, GJ = E_e / (2 (1 + nu)) 2 I.  Call between solves (it waits for the
 * handle's work); the resident state is kept.  A batch reads its members' moduli at every
 * iteration, so it applies to batched solves too.  E_INVALID_ARG if n_elements differs from the
 * robot's or a modulus is not finite and positive (nothing is changed then). */
accfem_status accfem_set_element_modulus(accfem_handle* h, const double* youngs_modulus, int32_t n_elements);

/* Frame mode: the paper's real-time scheme, one linearisation per frame (Eq. 20-23 at x_t, the
 * limited step of Eq. 25-27 gives x_{t+1}).  iters_per_frame > 0: every later solve performs at most
 * that many Newton iterations and returns ACCFEM_OK when it reaches them, with the state after the
 * last iteration resident and reported (newton_iters tells how many ran; a solve that converges
 * earlier stops there).  Each iteration then solves the QP over every detected constraint row (the
 * working set is all rows), so a frame's state is the paper's step from the previous frame's, and
 * max_contacts is bounded by the working-set cap (512).  0 restores solves to convergence with the
 * options' iteration cap.  Call between solves; a batch takes each member's mode when the batch is
 * created.  E_INVALID_ARG for a negative count or one above 10^6. */
accfem_status accfem_set_frame_mode(accfem_handle* h, int32_t iters_per_frame);

/* Contact solver of each Newton iteration (the QP of Eq. 23 in contact space, min 1/2 y^T W y + q^T y
 * over y >= 0, W = A K^{-1} A^T over the working set).  Both return its exact solution.
 * ACCFEM_CONTACT_ACTIVE_SET (the default): a primal active-set method started from the rows active
 * in the previous iteration.  ACCFEM_CONTACT_ADMM: the paper's scheme (Sec. III.B: the MLCP as a QP
 * solved by OSQP): OSQP's ADMM iteration (sigma 1e-6, rho 0.1 max diag W, relaxation 1.6, relative
 * tolerance 1e-3, at most 4000 iterations) on the whole working-set W, factored once, whose guess
 * of the free rows the active-set method then polishes to the exact solution.
 * ACCFEM_CONTACT_PRIMAL_ADMM: OSQP's ADMM on the primal QP of Eq. 23 as the paper states it (min
 * 1/2 dx^T K dx + g^T dx subject to A dx <= b over every constraint row; sigma 1e-6, rho 0.1 max diag
 * K, relaxation 1.6, tolerance 1e-3, at most 4000 iterations): K + sigma I + rho A^T A keeps K's
 * block-tridiagonal form and is factored once per Newton iteration, each ADMM iteration is one
 * solve with that factor, and the rows whose multiplier is positive start the active-set method,
 * which gives the exact solution; node contacts only (E_INVALID_ARG with the segment model), and not
 * in batches (accfem_batch_create refuses such members).  Call between solves; a batch takes each
 * member's solver when the batch is created.  E_INVALID_ARG otherwise. */
#define ACCFEM_CONTACT_ACTIVE_SET 0
#define ACCFEM_CONTACT_ADMM 1
#define ACCFEM_CONTACT_PRIMAL_ADMM 2
accfem_status accfem_set_contact_solver(accfem_handle* h, int32_t solver);

/* Contact model (Eq. 3-7).  ACCFEM_CONTACT_NODE (the default): a contact point sits at a node (xi = 0 of
 * an element; Sec. III.C pairs nodes with triangles), one constraint row per wall feature the node lies
 * over.  ACCFEM_CONTACT_SEGMENT: a contact point may lie anywhere on an element's chord, at chord
 * fraction s, and its displacement is interpolated from the element's two nodal translations by N(xi)
 * of Eq. 4-6 in the element frame (axial P1, P2 along the chord, transverse P3, P4 across it); one row
 * per wall feature the chord lies over (the node rule with the chord's closest point for the node), a
 * row at a shared node kept once, on the lower element; per element at most 144 triangles reach the
 * exact test and 32 rows are kept (ACCFEM_E_CONTACT_CAPACITY beyond).  In segment mode a result's contact_node is the
 * element's far node (element contact_node - 1 joins nodes contact_node - 1 and contact_node) and
 * contact_point the wall point.  Call between solves; a batch takes each member's model when the batch
 * is created.  The allocation-free query always detects node rows.  E_INVALID_ARG otherwise. */
#define ACCFEM_CONTACT_NODE 0
#define ACCFEM_CONTACT_SEGMENT 1
accfem_status accfem_set_contact_model(accfem_handle* h, int32_t model);

/* Cumulative bytes copied host->device and device->host by this handle's solve and state calls. */
accfem_status accfem_transfer_bytes(const accfem_handle* h, int64_t* h2d, int64_t* d2h);

/* Hot-path kernels that accfem_time_kernel can time standalone on the resident state. */
typedef enum {
  ACCFEM_KERNEL_ELEMENT = 0,    /* corotational force + tangent, one warp per element            */
  ACCFEM_KERNEL_COLLIDE = 1,    /* node-vs-triangle detection, one warp per free node            */
  ACCFEM_KERNEL_ASSEMBLE = 2,   /* block-tridiagonal assembly, RHS columns, level-1 eliminations  */
  ACCFEM_KERNEL_CONTACT = 3,    /* W = A K^-1 A^T and the contact LCP (needs a completed solve)  */
  ACCFEM_KERNEL_FACTOR = 4      /* assembly + block cyclic reduction factor and multi-RHS solve:
                                   every launch of one iteration's sequence, timed as one unit   */
} accfem_kernel;

/* Launches one hot-path kernel (or, for ACCFEM_KERNEL_FACTOR, the whole assembly + factor + solve
 * sequence) reps times on the resident state of the last solve (the listed kernels only read the
 * poses and rewrite their own outputs) and returns the mean device time of one launch (sequence)
 * in *us, measured with CUDA events on the handle's stream.  For measurement. */
accfem_status accfem_time_kernel(accfem_handle* h, accfem_kernel kernel, int32_t reps, double* us);

/* As accfem_time_kernel, but the reps launches (sequences) are captured, one after another, into
 * one CUDA graph that is replayed once untimed and once timed: the kernels then follow each other
 * through graph dependencies, as inside the device-side Newton loop, without the host's launch
 * overhead.  *us is the mean device time of one launch (sequence) of the timed replay.  The handle's
 * stream must not be capturing already; ACCFEM_E_CUDA (with the message in accfem_last_error) when
 * the capture or the replay fails.  For measurement. */
accfem_status accfem_time_kernel_graph(accfem_handle* h, accfem_kernel kernel, int32_t reps, double* us);

/* Collision query that allocates no memory.  The paper has no counterpart: this entry point exists
 * for callers that must not call cudaMalloc (or any allocating routine) once they run, for example a
 * real-time control loop that reserves all of its device memory at start-up and may not grow it, or
 * a host application that hands this library a fixed device-memory budget and owns every allocation
 * itself.  It is the constraint detection of accfem_solve for n_nodes caller positions (device memory,
 * 3 doubles each, node i = entry i) against the handle's lumen, with the same rule, the same
 * per-node limits (at most 64 triangles reach the exact FP64 test and at most 16 rows per node) and
 * the same rows as accfem_solve reports.  Inputs and outputs are caller-owned DEVICE buffers: up to
 * row_capacity rows are written in (node, triangle) order to row_node, row_tri, row_point (3 per row),
 * row_normal (3 per row) and row_gap (the b_i of Eq. 10); *n_rows (device int32) receives the total
 * row count.  The work runs on stream (a cudaStream_t; NULL = the handle's stream) and the call waits
 * for it.  Per-node scratch lives in one fixed device array of the library sized for n_nodes <= 4096
 * (about 4 MB, held by every GPU that loads the library until the process exits); larger n_nodes
 * returns ACCFEM_E_INVALID_ARG, as does a current device other than the handle's.
 * ACCFEM_E_CONTACT_CAPACITY when a node exceeds the per-node limits above or the rows exceed
 * row_capacity.  The first call on a device looks up the array's device address (once per device,
 * with that device current); make that first call before any stream capture.  All calls share the
 * one array, which keeps the last call's contents: calls that overlap on the GPU (other streams or
 * threads) race and must not be issued concurrently. */
accfem_status accfem_detect_contacts_noalloc(accfem_handle* h, const double* node_pos, int32_t n_nodes,
                                             int32_t row_capacity, int32_t* row_node, int32_t* row_tri,
                                             double* row_point, double* row_normal, double* row_gap,
                                             int32_t* n_rows, void* stream);

/* ---- Batched solves.  The paper solves one robot at a time; these calls are an extension for
 * throughput with no counterpart in it.  A batch groups member handles (each its own robot and
 * lumen, created by accfem_create on the current device) and advances every member that has a
 * solve in flight with one persistent kernel launch per Newton phase: each member runs exactly the
 * kernel code of accfem_solve on its own buffers, so its results are the ones accfem_solve gives.
 * Solves start and finish independently (continuous batching): stage solves on idle members with
 * accfem_batch_begin, run accfem_batch_advance, collect the finished ones with accfem_batch_poll and
 * accfem_batch_results, stage more.  The members stay owned by the caller and must outlive the
 * batch; a member must not be passed to other calls while a batch solve of it is staged or in
 * flight (between those solves it may be used alone; its resident state is shared).  Batch calls are
 * synchronous on the batch's stream; a batch is not thread-safe. */
typedef struct accfem_batch accfem_batch;

/* Groups members[0..n_members), 1 <= n_members <= 1024 distinct handles.  Builds the batch's CUDA
 * graph once (one iteration of all members as a conditional loop body). */
accfem_status accfem_batch_create(accfem_handle* const* members, int32_t n_members, accfem_batch** out);

/* Stages one quasi-static solve of member `member`, as accfem_solve with warm = NULL: cable_tensions
 * holds the member's n_cables values (host), insertion in [0, length]; the start pose follows the
 * member's resident state (straight on its first solve).  The solve starts at the next advance.
 * ACCFEM_E_INVALID_ARG if the member already has a solve staged or in flight. */
accfem_status accfem_batch_begin(accfem_batch* b, int32_t member, const double* cable_tensions, double insertion);

/* Starts the staged solves, then runs up to max_iters (>= 1) Newton iterations of every solve in
 * flight and waits; a solve stops at convergence, at an error or at its member's max_newton_iters.
 * *n_in_flight (may be NULL) receives the number of solves still unfinished. */
accfem_status accfem_batch_advance(accfem_batch* b, int32_t max_iters, int32_t* n_in_flight);

/* *done = 1 when member `member` has no solve staged or in flight; then *solve_status and
 * *newton_iters (either may be NULL) describe its last finished solve (ACCFEM_OK and 0 if none). */
accfem_status accfem_batch_poll(const accfem_batch* b, int32_t member, int32_t* done, accfem_status* solve_status,
                                int32_t* newton_iters);

/* Copies the results of the last finished solves of members[0..count) into out[0..count) (fields as
 * accfem_solve fills them) through one device gather and one device-to-host copy; statuses[j] (may
 * be NULL) receives member j's solve status.  Returns the first non-OK solve status, or an argument
 * or CUDA error. */
accfem_status accfem_batch_results(accfem_batch* b, const int32_t* members, int32_t count, accfem_result* out,
                                   accfem_status* statuses);

/* One solve of every member i with mask[i] != 0 (mask NULL = all members): tensions of member i at
 * cable_tensions[ACCFEM_MAX_CABLES * i ...], insertion insertions[i]; begins them, advances until
 * all finished and, if results is not NULL, fills results[i] (indexed by member).  statuses[i] (may be
 * NULL) receives each solved member's status.  Returns the first non-OK solve status. */
accfem_status accfem_batch_solve(accfem_batch* b, const double* cable_tensions, const double* insertions,
                                 const int32_t* mask, accfem_status* statuses, accfem_result* results);

/* One timed request for accfem_batch_serve: a quasi-static solve of scene `member` with the given
 * cable tensions (the member's n_cables values; the rest are ignored) and insertion, arriving
 * `arrival` seconds after the start of the run. */
typedef struct {
  double arrival;
  int32_t member;
  int32_t pad;
  double cable_tensions[ACCFEM_MAX_CABLES];
  double insertion;
} accfem_request;

/* Answer to one request: solve status and Newton iterations, the times (seconds after the start of
 * the run) at which its solve began and its answer was ready (latency = t_end - arrival), the tip
 * node pose (position 3, quaternion 4) and the constraint-row count. */
typedef struct {
  accfem_status status;
  int32_t newton_iters;
  double t_begin, t_end;
  double tip[7];
  int32_t n_contacts;
  int32_t pad;
} accfem_response;

/* Serves requests[0..n_requests) (non-decreasing arrival times) in real time by continuous batching:
 * a request waits until it has arrived and its scene is idle (requests of one scene are solved in
 * arrival order, each warm started from the scene's resident state left by the previous one), then
 * joins the solves in flight; everything in flight advances chunk_iters Newton iterations per
 * launch, and a solve's answer is ready after the launch in which it finished.  Admission by device
 * footprint: the batch's own memory, then members in index order while the total stays within
 * hbm_cap_bytes (<= 0: no cap); requests of members left out are answered ACCFEM_E_NOMEM without a
 * solve.  Returns when every request is answered (responses[k] for requests[k]); all members must
 * be idle at the call.  results (may be NULL): n_requests caller-owned results with buffers sized for
 * each request's member, as for accfem_solve; when given, every solved request's full result (poses,
 * constraint rows, contact forces, base reaction, counts) is also written to results[k], gathered with
 * the other solves that finished in the same launch (one more kernel and copy per launch, before the
 * answers of that launch are ready). */
accfem_status accfem_batch_serve(accfem_batch* b, const accfem_request* requests, int32_t n_requests,
                                 int32_t chunk_iters, int64_t hbm_cap_bytes, accfem_response* responses,
                                 accfem_result* results);

/* Autotuning of the work packing and the element mapping.  The batch's phase kernels are persistent;
 * they can run on their full resident grid or on 1/2, 1/4 or 1/8 of it (more units per block, fewer
 * idle blocks), and the element phase maps one warp to an element in blocks of 2, 4 or 8 warps: 12
 * variants, variant v dividing the grids by 2^(v % 4) with element blocks of 2 << (v / 4) warps.  After
 * this call the next 12 x trials advances take the variants in turn, each timed on the device per
 * Newton iteration, and the fastest is kept; results do not depend on the variant. */
accfem_status accfem_batch_autotune(accfem_batch* b, int32_t trials);

/* Variant in use (0..11 as above; -1 while tuning) and, if ms_per_pass is not NULL, the measured
 * milliseconds per Newton iteration of each variant (12 values, -1 if not measured). */
accfem_status accfem_batch_tuning(const accfem_batch* b, int32_t* variant, double* ms_per_pass);

/* Times one phase kernel of the batch (ACCFEM_KERNEL_ELEMENT, _COLLIDE or _ASSEMBLE) on the work plan of
 * the next iteration: call it after an accfem_batch_advance that left solves in flight.  The kernel
 * runs reps times (1..1000) on the members still iterating, each launch after a 256 MiB write that
 * evicts the L2 cache (a temporary device buffer of that size is allocated for the call), timed with
 * CUDA events on the batch's stream; *us receives the mean microseconds per launch and *items (may be
 * NULL) the free nodes the launch covers (elements for the element phase).  These phases only read the
 * poses and rewrite their own outputs, which the next iteration recomputes.  For measurement. */
accfem_status accfem_batch_time_phase(accfem_batch* b, accfem_kernel kernel, int32_t reps, double* us, int64_t* items);

/* Work stream of the batch's calls (a cudaStream_t; NULL = the batch's own stream). */
accfem_status accfem_batch_set_stream(accfem_batch* b, void* stream);

/* Cumulative bytes copied host->device and device->host by this batch's calls. */
accfem_status accfem_batch_transfer_bytes(const accfem_batch* b, int64_t* h2d, int64_t* d2h);

/* Number of kernel launches issued by this batch since creation. */
int64_t accfem_batch_kernel_launches(const accfem_batch* b);

/* Message of the last failure on this batch ("" if none). */
const char* accfem_batch_last_error(const accfem_batch* b);

/* Frees the batch (not its members); NULL is a no-op. */
void accfem_batch_destroy(accfem_batch* b);

/* Sizes of the contact problem in the last Newton iteration of the handle's last solve: constraint
 * rows, rows of the working set, active rows (y > 0); and 1 in *fp64_fallback when that solve, in
 * mixed precision, switched to the FP64 tangent.  Any pointer may be NULL. */
accfem_status accfem_solve_stats(const accfem_handle* h, int32_t* rows, int32_t* working_rows, int32_t* active_rows,
                                 int32_t* fp64_fallback);

/* ADMM iterations of the handle's last solve, summed over its Newton iterations (0 unless the
 * contact solver is ACCFEM_CONTACT_ADMM or ACCFEM_CONTACT_PRIMAL_ADMM; the scheme of Sec. III.B,
 * accfem_set_contact_solver).
 * ACCFEM_E_INVALID_ARG for NULL pointers. */
accfem_status accfem_solve_admm_iterations(const accfem_handle* h, int32_t* iters);

/* Device memory held by the handle, in bytes. */
accfem_status accfem_device_bytes(const accfem_handle* h, int64_t* bytes);

/* Copies the resident nodal poses (3*(M+1) and 4*(M+1) doubles) to host buffers. */
accfem_status accfem_get_state(accfem_handle* h, double* node_pos, double* node_quat);

/* Number of kernel launches issued by this handle since creation (for launch accounting). */
int64_t accfem_kernel_launches(const accfem_handle* h);

/* Frees the handle and its device memory; NULL is a no-op. */
void accfem_destroy(accfem_handle* h);

/* Static description of a status code. */
const char* accfem_status_string(accfem_status s);

/* Message of the last failure on this handle ("" if none); valid until the next call. */
const char* accfem_last_error(const accfem_handle* h);

#ifdef __cplusplus
}
#endif
#endif /* ACCFEM_H */
