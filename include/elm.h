/* elm.h -- C ABI of libelm.so: the advection step of the modified method of
 * characteristics (MMOC) on block-structured simplex meshes, for one GB300 GPU.
 *
 * Method: Kohl, Mohr, Eibl, Ruede, "A massively parallel Eulerian-Lagrangian
 * method for advection-dominated transport in viscous fluids" (arXiv
 * 2103.02388).  The library computes lines 3-4 of Algorithm 1 (departure
 * points and advection; the diffusion solve of line 5 is elm_diffusion_step):
 * for every P2 (or P1) node x_i of a
 * mesh of macro triangles / tetrahedra refined uniformly L times (Sec. 2.1),
 * the departure point X(x_i, t_{n+1}, t_n) of Eq. (departure point) by classic
 * RK4 backwards in time through the P2 (P1) velocity, linearly interpolated in
 * time (Eq. linear interpolation), then T^{n+1}_i = T^n_h(X_i) (Sec. 2.3.1,
 * step (iii)).
 *
 * Conventions shared by every call:
 *  - Elements: P2 (quadratic Lagrange, nodes = micro vertices and edge
 *    midpoints) by default, or P1 (linear, nodes = micro vertices) with
 *    ELM_P1 (Sec. 3.1: linear or quadratic elements for the temperature and
 *    the velocity).  M = 2^(L+1) node lattice points per macro edge for P2,
 *    M = 2^L for P1.
 *  - Node vectors live in STORAGE layout: macro after macro, each macro's
 *    nodes p = (p1 >= p2 [>= p3] >= 0), p1 <= M, packed row by row
 *    (index p1(p1+1)(p1+2)/6 + p2(p2+1)/2 + p3 in 3D, p1(p1+1)/2 + p2 in 2D).
 *    Nodes on macro interfaces appear once per macro that holds them; the
 *    copy in the lowest-numbered macro is the owner.  elm_mesh_unique_map
 *    gives storage -> unique ids; elm_to_storage / elm_to_unique convert.
 *  - Scalars are [n] and velocities [n, dim] row-major, in the mesh's
 *    precision (double for ELM_FP64, float for ELM_FP32).
 *  - Device pointers are borrowed, caller-owned, and used in stream order on
 *    the CUDA stream passed as `stream` (a cudaStream_t; NULL = legacy
 *    default stream).  Device memory is allocated only by elm_mesh_create
 *    (its tables and the buffers its flags ask for), elm_mesh_set_annulus (the
 *    sector table, and the blended diffusion tables and work lists) and
 *    elm_batch_create;
 *    the per-step calls allocate nothing.  No call synchronises, except
 *    elm_get_status (which synchronises `stream`) and elm_diffusion_step
 *    (below).
 *  - Errors: argument errors are returned synchronously and leave the
 *    mesh unchanged; device-side conditions (walk limit, non-finite values)
 *    set flags that elm_get_status reports.  No call traps or exits.
 *    (elm_diffusion_step is the one call that also synchronises: the host
 *    reads the device's convergence decision between batches of CG
 *    iterations.)
 *    elm_last_error() returns a thread-local message for the last failure.
 */
#ifndef ELM_H
#define ELM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct elm_mesh_s* elm_mesh;
typedef struct elm_batch_s* elm_batch;

typedef enum {
  ELM_OK = 0,
  ELM_ERR_ARG = 1,        /* invalid argument (null pointer, size, level, dtype) */
  ELM_ERR_CUDA = 2,       /* a CUDA runtime call failed */
  ELM_ERR_TOPOLOGY = 3,   /* degenerate macro or a face shared by > 2 macros */
  ELM_ERR_WALK_LIMIT = 4, /* a point needed more macro hops than the limit */
  ELM_ERR_NONFINITE = 5,  /* a velocity or result value was NaN / Inf */
  ELM_ERR_STATE = 6,      /* call order violated (e.g. advect before set_velocity) */
  ELM_ERR_NOT_CONVERGED = 7 /* an iterative solve stopped at its iteration limit */
} elm_status;

enum { ELM_FP64 = 0, ELM_FP32 = 1 };

/* Flag OR-ed into `precision` of elm_mesh_create: build the host tables only
 * (node coordinates, unique map; no device memory, no CUDA call).  Calls that
 * need the device then return ELM_ERR_STATE.  Lets a host without a GPU
 * prepare inputs and check a mesh. */
enum { ELM_HOST_ONLY = 0x100 };

/* Flag OR-ed into `precision` of elm_mesh_create: also allocate the scratch
 * of elm_advect_adjoint (64-bit accumulators and per-slot scale statistics:
 * (1 + 2 dim) * 8 + 6 * 8 + 3 * 4 bytes per storage node). */
enum { ELM_ADJOINT = 0x200 };

/* Flag OR-ed into `precision` of elm_mesh_create: linear (P1) elements for
 * the velocity and the scalar instead of quadratic (P2) ones (Sec. 3.1, test
 * setup; Tables 1 and 3 use P1).  The location is the same; a field is
 * evaluated from the d+1 vertices of the micro simplex with the micro
 * barycentrics as basis.  Combinable with ELM_ADJOINT (the adjoint then
 * differentiates the P1 interpolants) and with the batched form. */
enum { ELM_P1 = 0x400 };

/* Flag OR-ed into `precision` of elm_mesh_create: also build the diffusion
 * solver of elm_diffusion_step (per macro the element mass matrix, one
 * stiffness matrix per micro-simplex orientation and the node-centred stencil
 * weights of its interior; the work lists of the interior rows and of the
 * cells touching a macro face; boundary and owner masks; 2^dim colour
 * accumulators and 7 solver vectors per storage node in the mesh precision,
 * and the FP32 copies of the inner solves on FP64 meshes). */
enum { ELM_DIFFUSION = 0x800 };

/* Flag OR-ed into `precision` of elm_mesh_create: also set up elm_advect_host
 * (two sets of device staging buffers, (2 dim + 2) values per storage node in
 * the mesh precision each, and two internal non-blocking copy streams). */
enum { ELM_HOST_STAGING = 0x1000 };

/* Builds the refined mesh (Sec. 2.1: coarse mesh T_0 refined uniformly after
 * Bey; Sec. 2.3.1, grid data structure: one DoF owner per interface node).
 *  dim            2 (triangles) or 3 (tetrahedra).
 *  vertex_xyz     host, [n_vertices, dim] doubles.
 *  macro_vertices host, [n_macros, dim+1] vertex ids in [0, n_vertices).  The
 *                 order within a macro is irrelevant: vertices are sorted by
 *                 id, which makes the refinement conforming across faces.
 *  level          P2: 0..9 in 2D, 0..7 in 3D; P1: 0..10 in 2D, 0..8 in 3D.
 *  precision      ELM_FP64 or ELM_FP32, optionally | ELM_HOST_ONLY,
 *                 | ELM_ADJOINT, | ELM_P1, | ELM_DIFFUSION, | ELM_HOST_STAGING.
 * Copies everything it needs; allocates the mesh's device tables on the
 * current device.  Returns ELM_ERR_TOPOLOGY for a degenerate macro or a
 * non-manifold face.  *out is set only on success. */
elm_status elm_mesh_create(int dim, int64_t n_vertices, const double* vertex_xyz,
                           int64_t n_macros, const int64_t* macro_vertices,
                           int level, int precision, elm_mesh* out);

/* Frees the mesh and its device tables (after pending work on its streams). */
elm_status elm_mesh_destroy(elm_mesh mesh);

/* Blending onto an annulus (Sec. 2.1, blending map Phi; the curved domain of
 * Sec. 3.4).  The 2D macro mesh must be a ring of n_sectors sectors: every
 * vertex on a circle of radius in [r_min, r_max] at an angle
 * theta0 + k 2 pi / n_sectors, every macro spanning one sector.  Phi maps
 * each sector in polar form: the computational point
 * rho ((1 - lam) e_k + lam e_{k+1}) (e_k the unit vector at angle theta_k)
 * goes to rho e(theta_k + lam 2 pi / n_sectors), so chords become arcs with
 * uniform angle and the vertices stay.  Afterwards node coordinates are
 * physical, traced points live in the physical annulus (stage and departure
 * points with a radius outside [r_min, r_max] are projected radially onto
 * it), and every field evaluation pulls its point back with Phi^{-1} before
 * the location.  With ELM_DIFFUSION the call also builds the diffusion
 * solver's per-micro-simplex mass and stiffness matrices of the blended
 * geometry (the stiffness with the metric DPhi^{-1} DPhi^{-T} |det DPhi| by a
 * 5 x 5 collapsed Gauss rule; 2 nb^2 doubles per micro simplex).  Meshes:
 * ELM_FP64, 2D, P1 or P2, without ELM_ADJOINT; blended meshes are not
 * batched.  Returns ELM_ERR_TOPOLOGY for a mesh that is not such a ring.
 * Call once, before elm_set_velocity. */
elm_status elm_mesh_set_annulus(elm_mesh mesh, double r_min, double r_max, int n_sectors, double theta0);

/* Storage length n of every node vector of this mesh (0 for a null mesh). */
int64_t elm_mesh_num_nodes(elm_mesh mesh);

/* Number of distinct (unique) nodes. */
int64_t elm_mesh_num_unique(elm_mesh mesh);

/* Node coordinates in storage order into host_out [n, dim] doubles. */
elm_status elm_mesh_node_coords(elm_mesh mesh, double* host_out);

/* Storage slot -> unique node id into host_out [n] (unique ids follow the
 * storage order of the owner slots). */
elm_status elm_mesh_unique_map(elm_mesh mesh, int64_t* host_out);

/* Device copy between layouts, ncomp values per node, mesh precision:
 * storage_dev[s] = unique_dev[unique_map[s]]  /  unique_dev[u] = storage_dev[owner(u)]. */
elm_status elm_to_storage(elm_mesh mesh, const void* unique_dev, void* storage_dev, int ncomp, void* stream);
elm_status elm_to_unique(elm_mesh mesh, const void* storage_dev, void* unique_dev, int ncomp, void* stream);

/* Sets the nodal velocity at t_n (u_old) and t_{n+1} (u_new), storage layout
 * [n, dim], mesh precision (Sec. 2.3.1 step (ii), Eq. linear interpolation).
 * u_new == u_old means a steady velocity (no time interpolation).  The call
 * enqueues, on `stream`, a copy of the velocity into the mesh's own
 * device buffers in a padded 4-component record layout (one vector load per
 * stencil node in the kernel); the caller's buffers are not used afterwards.
 * Work on other streams must be ordered after it by the caller. */
elm_status elm_set_velocity(elm_mesh mesh, const void* u_old_dev, const void* u_new_dev, void* stream);

/* The velocity pair of the next older interval of a look-back over a
 * time-dependent velocity (Sec. 2.3.3, intervals taken newest first, each
 * with the linear time interpolation of its pair, Eq. linear
 * interpolation): with (u^{k-1}, u^k) set, the current u_old becomes u_new
 * (its packed records are kept, the caller's buffer is not read again) and
 * u_old_dev ([n, dim], device, mesh precision) is packed as the new u_old,
 * giving (u^{k-2}, u^{k-1}) for half the packing work of elm_set_velocity.
 * After a steady velocity the current field becomes u_new.  Enqueued on
 * `stream`, which must be the stream of the calls that read the previous
 * pair (the repacked buffer is the previous u_new's).  ELM_ERR_STATE without
 * a velocity; allocates nothing. */
elm_status elm_shift_velocity(elm_mesh mesh, const void* u_old_dev, void* stream);

/* Most RK4 substeps of one forward step (elm_advect, elm_advect_noalloc,
 * elm_batch_advect); elm_advect_adjoint, whose cost grows with the square of
 * the substep count, takes at most ELM_MAX_ADJOINT_SUBSTEPS. */
#define ELM_MAX_SUBSTEPS 65536
#define ELM_MAX_ADJOINT_SUBSTEPS 64

/* One advection step (Algorithm 1, lines 3-4; Sec. 2.3.1 steps (i)-(iii)):
 * T_new[i] = T_old_h(X_i), X_i traced back over dt from node i with n_sub
 * equal RK4 substeps.  T_old and T_new are [n] in storage layout and must
 * not overlap.  Stage and departure points outside the domain are clamped
 * to the mesh's bounding box.  1 <= n_sub <= ELM_MAX_SUBSTEPS; dt finite
 * and >= 0.
 * Look-back distance b (Sec. 2.3.3) for a steady velocity: tracing back b
 * steps of tau with s RK4 substeps each and interpolating T^{n+1-b} is
 * exactly elm_advect(T^{n+1-b}, b*tau, b*s); b = infinity is T^0 with
 * dt = t_{n+1} (one trace over the whole time, no interpolation error
 * accumulated between steps).
 * Each node is computed once, by its owner copy (Sec. 2.3.1: one owner per
 * degree of freedom); a second launch copies the result to the node's other
 * storage copies, so all copies hold the same value.  Two kernel launches
 * on `stream`; allocates nothing. */
elm_status elm_advect(elm_mesh mesh, const void* T_old_dev, void* T_new_dev, double dt, int n_sub,
                      void* stream);

/* The advection step of elm_advect with every buffer in HOST memory, for a
 * caller whose fields live on the host (Algorithm 1, lines 3-4: the step's
 * inputs are the velocity at t_n and t_{n+1} and T^n; its result is T^{n+1}).
 * Needs a mesh created with ELM_HOST_STAGING.
 *  u_old_host, u_new_host  velocity [n, dim] (equal pointers: steady); both
 *                          NULL: the mesh's current velocity (from
 *                          elm_set_velocity or an earlier call) is used and
 *                          only T moves (ELM_ERR_STATE if none is set).
 *  T_old_host, T_new_host  [n]; they may be the same buffer (in-place).
 *  dt, n_sub, stream       as for elm_advect.
 * The buffers given must be page-locked host memory (cudaHostAlloc, cudaHostRegister
 * or a pinned torch tensor): the call checks the first and last byte of each
 * and returns ELM_ERR_ARG for pageable memory.  Everything is enqueued
 * asynchronously; when `stream` has completed, T_new_host holds the result,
 * and until then the caller must neither change the inputs nor read or reuse
 * the output.  A velocity given becomes the mesh's current velocity, as
 * after elm_set_velocity.
 * Pipelining: consecutive calls alternate between the two staging sets, and
 * the copies run on the mesh's own streams, so the host-to-device copy of a
 * call overlaps the step of the call before it, and each quarter of the
 * result is copied back while the rest is computed.  A call whose inputs
 * overlap the host result of the call in flight before it waits for that
 * result first, so feeding T_new_host back as the next T_old_host is
 * correct.  Successive calls on one mesh must use one stream (or be ordered
 * by the caller).  Not capturable into a CUDA graph: returns ELM_ERR_STATE
 * while `stream` is capturing. */
elm_status elm_advect_host(elm_mesh mesh, const void* u_old_host, const void* u_new_host, const void* T_old_host,
                           void* T_new_host, double dt, int n_sub, void* stream);

/* The advection step of elm_advect for callers that cannot allocate device
 * memory where they advect (for example an application whose device memory
 * is handed out by its own pool, or a time-critical loop that cannot take the
 * implicit device synchronisation of cudaMalloc / cudaFree).  The paper has no
 * counterpart: this entry point changes only where the working copy of the
 * velocity lives.  It allocates and frees nothing.
 *  u_old_dev, u_new_dev  the caller's velocity, [n, dim] row-major in the mesh
 *                        precision (equal pointers: steady velocity); packed on
 *                        `stream` into a fixed scratch array inside the library
 *                        (32 MiB of device memory held by every GPU that loads
 *                        the library until exit), then read by the step.
 *  T_old_dev, T_new_dev, dt, n_sub, stream  as for elm_advect.
 * elm_set_velocity is not needed and the mesh's own velocity is untouched.
 * Limit: meshes of at most 524288 (2^19) storage nodes; larger meshes return
 * ELM_ERR_ARG.  The first call on a device looks up the scratch array's device
 * address (with that device current); make that first call before any stream
 * capture.  That address is kept for the life of the process, so the device's
 * context must not be reset (cudaDeviceReset) after the first call.  Every call
 * shares the one scratch array, so calls that overlap on the GPU (other
 * streams, other threads) race; order them.  Launches exactly what elm_advect
 * launches (the step and the interface-copy pass), plus the velocity packing. */
elm_status elm_advect_noalloc(elm_mesh mesh, const void* u_old_dev, const void* u_new_dev, const void* T_old_dev,
                              void* T_new_dev, double dt, int n_sub, void* stream);

/* Adjoint of elm_advect (Eq. departure point and step (iii) of Sec. 2.3.1,
 * differentiated) for the velocity last given to elm_set_velocity:
 *   gT_old = W^T gT_new, W the interpolation matrix of the step
 *            (W_ij = phi_j(X_i)), and
 *   gU_old, gU_new = dL/du^n, dL/du^{n+1} through the backward RK4 stages,
 *            the P1 / P2 velocity evaluations, the time interpolation and the box
 *            clamps (a clamped coordinate passes no derivative), for
 *            L = <gT_new, T_new(u)>.
 * T_old, gT_new, gT_old: [n]; gU_old, gU_new: [n, dim]; storage layout, mesh
 * precision.  Steady velocity (u_old == u_new in elm_set_velocity): gU_old
 * receives the whole velocity gradient and gU_new must be NULL; otherwise
 * gU_new may be NULL to receive the sum in gU_old.  Gradients are
 * accumulated onto each node's owner slot (duplicate slots get 0), so
 * elm_to_unique gives per-node gradients.  Deterministic: contributions are
 * summed as 64-bit fixed-point integers with one scale per output slot, set
 * by a first pass from the slot's largest contribution and its number of
 * contributions so that no sum can overflow (however many departure points
 * meet at one node) and every entry keeps its relative precision; repeated
 * calls give bitwise equal results.  Requires ELM_ADJOINT at
 * creation; allocates nothing; a few kernel launches on `stream`.  The map
 * is only piecewise smooth (P1 and P2 are C0); on element faces the derivative of
 * the element the point is located in is used.
 * 1 <= n_sub <= ELM_MAX_ADJOINT_SUBSTEPS (the reverse sweep recomputes each
 * substep's start from the node, O(n_sub^2) work). */
elm_status elm_advect_adjoint(elm_mesh mesh, const void* T_old_dev, const void* gT_new_dev, void* gT_old_dev,
                              void* gU_old_dev, void* gU_new_dev, double dt, int n_sub, void* stream);

/* ---- Look-back over a time-dependent velocity (Sec. 2.3.3) ----
 * Tracing back b time steps needs the velocity of every intermediate step
 * (b = infinity: of every step since t_0).  elm_trace continues backward
 * traces over one interval at a time, with that interval's velocity pair
 * from elm_set_velocity; elm_trace_eval then interpolates the temperature
 * of the time the traces reached.  For T^{n+1} with look-back b:
 *   D = NULL;  for k = n+1 down to n+2-b:
 *     elm_set_velocity(u^{k-1}, u^k); elm_trace(D, D', tau, s); D = D';
 *   elm_trace_eval(D, T^{n+1-b}, T^{n+1}).
 * A steady velocity needs none of this: elm_advect(T^{n+1-b}, b tau, b s).
 *
 * elm_trace: for every node x_i, starts at x_i + D_in[i] (at x_i when D_in
 * is NULL), traces back over dt with n_sub classic RK4 substeps through the
 * current velocity (time-interpolated as in elm_advect, t_{n+1} being the
 * start of this backward interval), clamps to the bounding box like
 * elm_advect and writes the offset D_out[i] = X_i - x_i.
 *  D_in, D_out  [n, dim] departure offsets, storage layout, mesh precision;
 *               they must not overlap.  Every storage copy of an interface
 *               node continues from the offset of the node's owner copy and
 *               all copies receive the same result.
 *  1 <= n_sub <= ELM_MAX_SUBSTEPS; dt finite and >= 0.
 * Two kernel launches on `stream` (the traces, then the copy of each
 * interface node's result to its other storage copies); allocates nothing;
 * device conditions go to elm_get_status as for elm_advect. */
elm_status elm_trace(elm_mesh mesh, const void* D_in_dev, void* D_out_dev, double dt, int n_sub, void* stream);

/* T_dst[i] = T_src_h(x_i + D[i]) (Sec. 2.3.1, step (iii), at the end of
 * traces made by elm_trace).  D is [n, dim], T_src and T_dst [n] (must not
 * overlap), storage layout, mesh precision.  Needs no velocity.  Two kernel
 * launches on `stream` (evaluation, interface copies); allocates nothing. */
elm_status elm_trace_eval(elm_mesh mesh, const void* D_dev, const void* T_src_dev, void* T_dst_dev, void* stream);

/* ---- Diffusion step (Sec. 2.2, Eq. finite-dimensional Galerkin approximation
 * and Eq. linear system; Algorithm 1 line 5 and the fractional steps of the
 * Strang splitting, Algorithm 2) ----
 * Solves, for the P1 / P2 mass matrix M and stiffness matrix A of the mesh,
 *   (M + tau theta kappa A) c_new = (M - tau (1 - theta) kappa A) c_hat + tau M q
 * with c_new = c_bnd on the boundary of the macro mesh (Dirichlet), by
 * Jacobi-preconditioned conjugate gradients on the interior unknowns, to
 * |r| <= rtol |b| (b the interior right-hand side).  theta = 1: implicit
 * Euler; theta = 1/2: Crank-Nicolson.
 *  c_hat_dev  [n] storage layout, mesh precision: the advected field.
 *  c_bnd_dev  [n] boundary values (NULL: c_hat's values there).
 *  q_dev      [n] nodal source values q (NULL: q = 0); the caller combines
 *             theta q^{n+1} + (1 - theta) q^n.
 *  c_new_dev  [n] result; must not overlap an input.  Every storage copy of a
 *             node receives the node's value.
 *  iterations, residual  optional host outputs: CG iterations and the final
 *             relative residual.
 * FP64 meshes (affine macros) solve by defect correction: the residual in
 * FP64, the corrections by the same PCG in FP32 (to 3e-5 of their start), so
 * `iterations` counts the FP32 iterations; blended FP64 meshes and FP32 meshes
 * run the PCG in their own precision.
 * The operator is matrix-free: a node-centred stencil for the nodes inside a
 * macro and an element pass over the cells touching a macro face (blended
 * meshes: over every cell); it uses no atomics and sums in a fixed order, so
 * repeated calls give bitwise equal results.  Requires ELM_DIFFUSION at
 * creation.  Unlike the other calls this one synchronises `stream`: the
 * device decides convergence, and the host reads the CG scalars once per 8
 * iterations.  Returns ELM_ERR_NOT_CONVERGED (with c_new the last iterate)
 * when max_iter iterations do not reach rtol. */
elm_status elm_diffusion_step(elm_mesh mesh, const void* c_hat_dev, const void* c_bnd_dev, const void* q_dev,
                              void* c_new_dev, double tau, double kappa, double theta, double rtol, int max_iter,
                              int* iterations, double* residual, void* stream);

/* Synchronises `stream`, returns the first device-side condition raised by
 * work on this mesh since the previous call (ELM_ERR_WALK_LIMIT or
 * ELM_ERR_NONFINITE), else ELM_OK, and clears the flags. */
elm_status elm_get_status(elm_mesh mesh, void* stream);

/* ---- Batched form: many independent advection instances in one launch ----
 * Each instance is a P2 or P1 mesh with its own level, dimension, velocity
 * (elm_set_velocity on that mesh), dt and n_sub; every instance performs the
 * step of elm_advect (Algorithm 1, lines 3-4).  One persistent kernel takes
 * (instance, chunk) items from a shared work list, so small and large
 * instances share the GPU in a single launch (one launch per element order
 * present: P2 instances first, then P1).  The paper has no batched form; it
 * traces one field per run.
 *
 * elm_batch_create: count in 1..128 meshes, all of one precision and device,
 * borrowed (they must outlive the batch).  blocks_per_sm (0..32) sets the
 * persistent grid (resident blocks per SM; 0 = default 6) and with it the
 * kernel's register budget (8 or more: the 8-block budget, else the 6-block
 * one); chunks_per_item (0..64; 0 = 1) is the tile a block takes per fetch
 * from the work list: that many consecutive 128-node chunks of one instance.
 * The autotuner picks both.  Allocates the batch's small device tables. */
elm_status elm_batch_create(const elm_mesh* meshes, int count, int blocks_per_sm, int chunks_per_item,
                            elm_batch* out);
elm_status elm_batch_destroy(elm_batch batch);
/* Number of work items (runs of chunks of one instance) of the batch. */
int64_t elm_batch_num_items(elm_batch batch);
/* One step of every instance k: T_new[k] = advect(T_old[k], dt[k], n_sub[k]).
 * T_old, T_new, dt, n_sub are host arrays of `count` entries (device
 * pointers in storage layout, mesh precision).  Their values are copied into
 * the launch's parameters, so the call can be captured in a CUDA graph and
 * replayed with the same pointers.  Zeroes the device counters and launches
 * one kernel per element order present on `stream`, then one kernel that
 * copies every instance's interface nodes from their owners (each node is
 * computed once, by its owner copy, as in elm_advect); allocates nothing.
 * Each instance's device flags are reported by elm_get_status on its mesh. */
elm_status elm_batch_advect(elm_batch batch, const void* const* T_old, void* const* T_new, const double* dt,
                            const int* n_sub, void* stream);

/* Thread-local description of the last error returned on this thread. */
const char* elm_last_error(void);

/* Measured throughput of the SM pipes the advection kernels are bound by, on
 * the current device (a timed loop of each instruction kind, 8 independent
 * chains per thread, 8 resident 256-thread blocks per SM); the benchmark's
 * compute roofline divides by these.  The paper has no counterpart.
 *  rates_host  [n >= 5] doubles, written: FP32 FMAs per second issued as FFMA,
 *              FP32 FMAs per second issued as packed FFMA2 (2 per instruction),
 *              FP32 min/max per second, 32-bit integer min/max per second,
 *              FP64 FMAs per second.
 *  stream      as elsewhere; the call synchronises it (it reads CUDA events).
 * Takes about 20 ms; allocates no device memory; ELM_ERR_ARG for n < 5. */
elm_status elm_probe_pipes(double* rates_host, int n, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* ELM_H */
