/*
 * cellfsi.h - C ABI of the GB300 cell/fluid time-step library (libcellfsi.so).
 *
 * One time step of a hyperelastic tetrahedral cell immersed in a lattice-
 * Boltzmann fluid (Mueller et al., "A hyperelastic model for simulating cells
 * in flow"):
 *   (a) Mooney-Rivlin nodal forces f_i^a = -V_0 dU/du_i^a on every tet
 *       (Sec. 2, Sec. 3.1-3.2), summed per vertex;
 *   (b) immersed-boundary coupling: vertex forces spread onto the lattice and
 *       fluid velocity interpolated back with a discrete delta kernel (Sec. 6);
 *   (c) D3Q19 lattice-Boltzmann stream-collide with forcing and moving walls
 *       (Sec. 6.1: plane Couette flow, walls moving at -/+u_wall in x).
 *
 * Conventions shared by every call
 * --------------------------------
 * - Units are lattice units: nodes at integer coordinates 0..n-1, time step 1.
 *   The walls sit half a spacing outside rows y = 0 and y = ny-1; x and z are
 *   periodic.
 * - All pointer arguments are HOST pointers, row-major, owned by the caller.
 *   The library copies inputs before returning and writes outputs into
 *   caller-allocated arrays; it keeps no reference to caller memory.
 * - Vertex arrays are [nv][3] doubles; tets are [nt][4] int32 vertex indices
 *   local to the cell, corner 3 being the paper's vertex 4 (the origin of the
 *   tet's local coordinates, Sec. 3.2).
 * - Every call returns a cf_status. On failure cf_last_error() describes it;
 *   the context stays usable unless the status is CF_ECUDA.
 * - The library owns all device memory of a context and frees it in
 *   cf_destroy(). Device work runs on the context's stream; calls that return
 *   data synchronise that stream. No call traps or hangs the GPU: device-side
 *   faults of the inputs (inverted tets, non-finite values, a delta support
 *   that crosses a wall) are reported through status codes.
 * - A context is not thread-safe; use one per host thread.
 * - Call order: cf_create, then cf_lbm_init and/or cf_mesh_init (any order,
 *   repeatable), cf_set_material, then cf_step. cf_step needs cf_lbm_init;
 *   cf_compute_forces needs only meshes. Otherwise CF_ESTATE.
 */
#ifndef CELLFSI_H
#define CELLFSI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cf_ctx cf_ctx;

typedef enum {
    CF_OK = 0,
    CF_EINVAL = 1,      /* bad argument: size, index range, repeated vertex, parameter range */
    CF_EDEGENERATE = 2, /* reference tet with |det J| <= 1e-12 (longest edge)^3 */
    CF_EINVERTED = 3,   /* a tet reached det F <= 0 during the run */
    CF_ENONFINITE = 4,  /* NaN or Inf in forces, positions or populations */
    CF_EDOMAIN = 5,     /* a vertex's delta support left 0 <= y <= ny-1 */
    CF_ESTATE = 6,      /* call out of order */
    CF_ECUDA = 7,       /* CUDA runtime error; context must be destroyed */
    CF_ETIMEOUT = 8,    /* device work did not finish within the host timeout */
    CF_ENOMEM = 9,      /* device allocation failed */
    CF_EUNSTABLE = 10   /* a vertex moved a lattice spacing or more in one step */
} cf_status;

/* Create a context on CUDA device `device`. `cuda_stream` is a cudaStream_t
 * the caller owns (for example PyTorch's current stream) or NULL, in which
 * case the context creates and owns a non-blocking stream. */
cf_status cf_create(cf_ctx **out, int device, void *cuda_stream);

/* Free all device memory of the context. NULL is ignored. */
void cf_destroy(cf_ctx *ctx);

/* Storage of the lattice populations, used by the next cf_lbm_init (which
 * re-initialises the fluid). The populations are kept as deviations
 * f_q - w_q from the rest equilibrium; FP16 and BF16 store them multiplied by
 * a power of two per weight class. The collide always computes in FP32.
 * CF_POP_F16 and CF_POP_BF16 round each store to nearest; CF_POP_F16_SR and
 * CF_POP_BF16_SR round stochastically (unbiased: up with probability equal to
 * the dropped fraction, from a counter-based hash of the node, the direction
 * and a per-step seed held on the device), so that increments smaller than
 * half a unit in the last place are not lost on average.
 * Default CF_POP_F32. Errors: CF_EINVAL for an unknown format. */
enum { CF_POP_F32 = 0, CF_POP_F16 = 1, CF_POP_BF16 = 2, CF_POP_F16_SR = 3, CF_POP_BF16_SR = 4 };
cf_status cf_set_population_format(cf_ctx *ctx, int32_t format);

/* How the spread accumulates the force field, from the next cf_lbm_init on.
 * CF_SPREAD_FLOAT (default): one float4 atomic add per vertex and support
 * node; the field is exact up to the order of those additions, so two runs
 * can differ by rounding, and a chaotic flow amplifies that. CF_SPREAD_FIXED:
 * the field is held in 64-bit fixed point (units of 2^-48 per component),
 * each contribution is its FP32 value scaled by 2^48 and rounded once, and
 * the integer sums are exact whatever the order: every run, launch shape
 * (tiles, block sizes, near-field form, where the region is marked) and
 * schedule (pipelined, one step per call, profiled) gives bit-identical
 * results; the force kernel's form (tets per thread, lanes per tet) still
 * changes its rounding. Costs 8 more bytes per node of the field (24 instead
 * of 16), three 64-bit reductions per support node instead of one vector
 * one, and disables the staged spread. |F| must stay below 2^15 per
 * component. Not a paper feature: a service for reproducible runs. */
#define CF_SPREAD_FLOAT 0
#define CF_SPREAD_FIXED 1
cf_status cf_set_spread(cf_ctx *ctx, int32_t mode);

/* Immersed-boundary delta kernel for the spreading of vertex forces and the
 * interpolation of the fluid velocity (the paper does not name its kernel),
 * from the next cf_lbm_init on: delta_h(r) = phi(r_x) phi(r_y) phi(r_z) with
 *   CF_DELTA_TRILINEAR (2): phi(r) = max(0, 1 - |r|), 2 nodes per axis;
 *   CF_DELTA_PESKIN4   (4): Peskin's four-point kernel (Acta Numerica 2002),
 *     phi(r) = (3 - 2|r| + sqrt(1 + 4|r| - 4r^2))/8 for |r| <= 1,
 *              (5 - 2|r| - sqrt(-7 + 12|r| - 4r^2))/8 for 1 <= |r| <= 2,
 *     4 nodes per axis.
 * The value is the support width. Every support node must lie in
 * 0 <= y <= ny-1 (else CF_EDOMAIN from the step). Default
 * CF_DELTA_TRILINEAR. Errors: CF_EINVAL for any other value. */
enum { CF_DELTA_TRILINEAR = 2, CF_DELTA_PESKIN4 = 4 };
cf_status cf_set_delta(cf_ctx *ctx, int32_t kernel);

/* Lattice-Boltzmann fluid on nx*ny*nz nodes (Sec. 6.1 box), D3Q19 BGK with
 * relaxation time tau (> 1/2), Guo forcing, halfway bounce-back walls at
 * y = -1/2 moving at (u_wall_lo_x, 0, 0) and y = ny-1/2 moving at
 * (u_wall_hi_x, 0, 0) (|u| < 0.1), and a uniform body-force density
 * body_force[3] (NULL = none), e.g. for a pressure-driven channel. The fluid
 * starts at rest with density 1. nx, ny, nz >= 1, ny, nz <= 65535,
 * nx*ny*nz < 2^30 (node indices are 32-bit; 2^30 FP32 nodes take about
 * 200 GB); CF_ENOMEM if the device cannot hold the lattice.
 * Re-initialises the fluid if called again. */
cf_status cf_lbm_init(cf_ctx *ctx, int32_t nx, int32_t ny, int32_t nz, double tau,
                      double u_wall_lo_x, double u_wall_hi_x, const double *body_force);

/* Add one cell (Sec. 3): reference positions x_ref[nv][3] (absolute lattice
 * coordinates), tets[nt][4] (local vertex indices) and current positions
 * y0[nv][3] (NULL = x_ref). Computes once per tet the Jacobian
 * J_ik = x_i^k - x_i^4, B = J^-1 and V_0 = |det J|/6 (Sec. 3.2); tets with
 * det J < 0 get corners 1 and 2 swapped so that all are positively oriented.
 * Builds the vertex -> (tet, corner) incidence rows used to sum vertex forces
 * in a fixed order. Returns the new cell's id (0, 1, ...) in *cell_id_out.
 * Errors: CF_EINVAL (nv < 4, nt < 1, index out of range, repeated vertex),
 * CF_EDEGENERATE. Material defaults to mu = kappa = 0 (no force). */
cf_status cf_mesh_init(cf_ctx *ctx, int32_t nv, const double *x_ref, int32_t nt, const int32_t *tets,
                       const double *y0, int32_t *cell_id_out);

/* Add ncells cells at once (one reallocation and one incidence-row build
 * for all of them; for suspensions of hundreds of cells). nv[ncells],
 * nt[ncells]: sizes; x_ref [sum nv][3], tets [sum nt][4] (indices local to
 * each cell), y0 [sum nv][3] or NULL: the cells' arrays concatenated in
 * order. cell_ids_out[ncells] receives the ids. Same per-cell set-up and
 * errors as cf_mesh_init (the message names the cell); on error no cell is
 * added. */
cf_status cf_mesh_init_batch(cf_ctx *ctx, int32_t ncells, const int32_t *nv, const double *x_ref, const int32_t *nt,
                             const int32_t *tets, const double *y0, int32_t *cell_ids_out);

/* Mooney-Rivlin material of one cell (Sec. 2): shear modulus mu >= 0, bulk
 * modulus kappa >= 0 and ratio w in [0, 1], with mu_1 = w mu and
 * mu_2 = (1 - w) mu; w = 1 is neo-Hookean. A nearly incompressible material,
 * kappa >= 100 mu (Poisson ratio 0.495 and above), has the volume change
 * J - 1 of its tets evaluated in FP64 (from the FP32 displacements and an
 * FP64 copy of B kept from the set-up): the volume term kappa (J - 1)
 * amplifies any rounding of J - 1 by kappa / mu. The rest of the force is
 * FP32. */
cf_status cf_set_material(cf_ctx *ctx, int32_t cell_id, double mu, double kappa, double w);

/* Materials of several cells at once: ids[ncells], mu, kappa, w as in
 * cf_set_material (all validated before any is applied). Setting a cell's
 * material makes it uniform again after cf_set_tet_materials. */
cf_status cf_set_materials(cf_ctx *ctx, int32_t ncells, const int32_t *ids, const double *mu, const double *kappa,
                           const double *w);

/* Materials per tet within one cell (Sec. 3.1: the force is local to each
 * tet, so regions of a cell such as a nucleus or a cortex may carry their
 * own elastic parameters). region[nt] assigns each of the cell's tets
 * (in its cf_mesh_init order, after the orientation fix, which keeps tet
 * order) to one of nreg >= 1 regions; mu[nreg], kappa[nreg], w[nreg] as in
 * cf_set_material. Forces, energies, steps and the force JVP use the per-tet
 * materials; the parameter gradients (cf_force_param_vjp,
 * cf_relax_adjoint, cf_adjoint_gradients) are per cell and return
 * CF_ESTATE while any cell has per-tet materials. Errors: CF_EINVAL (unknown
 * cell, region index out of range, parameter range). */
cf_status cf_set_tet_materials(cf_ctx *ctx, int32_t cell_id, const int32_t *region, int32_t nreg, const double *mu,
                               const double *kappa, const double *w);

/* Advance n >= 0 coupled time steps t -> t+1, each: elastic forces at y^t,
 * vertex sums, spread onto the lattice, one stream-collide with that force,
 * interpolation of the fluid velocity u(t) at y^t and y^{t+1} = y^t + u.
 * Synchronises and returns the first error any step raised. */
cf_status cf_step(cf_ctx *ctx, int32_t n);

/* Same as cf_step but returns after enqueueing the work on the stream; the
 * error word is read by the next synchronising call (cf_synchronize or any
 * cf_get_*). */
cf_status cf_step_async(cf_ctx *ctx, int32_t n);

/* One round trip for callers that drive the cells from the host: set the
 * positions of all cells (y_in [V][3], every vertex in cell order as with
 * CF_ALL_CELLS; NULL keeps them), advance n >= 0 steps as cf_step, then
 * read the positions of all cells into y_out [V][3] (NULL skips it), with a
 * single wait at the end. Host buffers that are page-locked and mapped into
 * the device's address space (cudaHostAlloc, cudaMallocHost, or registered
 * as mapped) are read and written in place by the conversion kernels over
 * the host link; other buffers go through a device staging copy. The caller
 * keeps both buffers unchanged and unread until the call returns. Errors as
 * cf_set_positions, cf_step and cf_get_positions; CF_ESTATE without cells
 * when y_in or y_out is given. */
cf_status cf_step_exchange(cf_ctx *ctx, int32_t n, const double *y_in, double *y_out);

/* Build, without running anything, every CUDA graph that cf_step or
 * cf_step_async of n steps would build on first use, from the current state
 * and from every other buffer parity and region phase (the step counter
 * modulo 2 and 3), so that repeated n-step calls only launch (graph capture
 * and instantiation take milliseconds). Positions, populations and the step
 * counter are unchanged. CF_ESTATE before cf_lbm_init, CF_EINVAL for n < 0. */
cf_status cf_prepare_steps(cf_ctx *ctx, int32_t n);

/* Wait for the context's stream (polling, with the host timeout) and return
 * the accumulated device error status. */
cf_status cf_synchronize(cf_ctx *ctx);

/* Measurement support: advance n >= 1 steps with the same kernels as
 * cf_step, but launched one after another on the context's stream (no
 * graph, no overlap) with a CUDA event around each launch. kernel_ms[5]
 * receives the mean duration in ms per step of: tet forces, vertex sums +
 * spread, far-field stream-collide (the whole lattice when there are no
 * cells), near-field stream-collide, interpolate + advect. *near_nodes (may
 * be NULL) receives the number of nodes in the last step's force region.
 * Synchronises; returns the first device error. */
cf_status cf_step_profiled(cf_ctx *ctx, int32_t n, double *kernel_ms, int64_t *near_nodes);

/* Launch shapes of the step kernels, as CF_SHAPE_LEN int32 values:
 *   [0..2] x, y, z extent in nodes of the force-region tiles: 16x4x4
 *          (default), 32x4x2, 32x2x4 or 8x8x4 (the lattice is cut into tiles;
 *          the near-field stream-collide updates the tiles that meet a
 *          vertex's delta support, the far field the others);
 *   [3]    threads per block of the tet-force kernel (default 64);
 *   [4]    threads per block of the vertex-sum + spread kernel (default 128);
 *   [5]    threads per block of the interpolation kernel (default 128);
 *   [6]    1: the tet forces and the vertex sums + spread run as one
 *          persistent launch over work items of all cells, vertex sums of a
 *          cell starting as soon as its tets are done; 0 (default): two
 *          launches ([3] and [4] apply only then);
 *   [7]    1: the near-field stream-collide runs in rows of 128 nodes over
 *          the whole lattice, threads outside the region returning at once
 *          (for regions that cover much of the lattice); 0 (default): blocks
 *          stride over the region's tile list;
 *   [8]    1: the far field issues a node's loads before its region test
 *          resolves (saves a round trip per far node, wastes the loads of
 *          region nodes); 0 (default): region nodes return first;
 *   [9]    form of the force kernel: 0 (default) one thread per tet; 1 two
 *          tets per thread, both tets' loads in flight before either is
 *          computed; 2 four lanes per tet (one corner each, the tet's
 *          deformation gradient and corner forces shared by shuffles: more
 *          threads for meshes too small to fill the GPU);
 *   [10]   1: with FP32 populations the far and near fields cache them in
 *          L2 at normal priority (for lattices whose stream-collide gains
 *          more from L2 reuse than the cell kernels lose); 0 (default):
 *          populations are streamed with evict-first hints, so that the
 *          cells' data stays in L2;
 *   [11]   1 (default): with 16-bit populations and nx even the
 *          whole-lattice, far-field and row-form near-field stream-collide
 *          take two x-neighbours per thread (32-bit population access,
 *          packed FP32 collide); 0: one node per thread;
 *   [12]   where the force region of a step is marked (the tiles that meet
 *          the vertices' delta supports grown by one node): 0 (default) by
 *          the force kernel of the step before, one extra thread per vertex
 *          running under the tets; 1 by the interpolation two steps before,
 *          right after it moves the vertices, its eight lanes per vertex
 *          sharing the vertex's tiles (a shorter chain for small meshes);
 *   [13]   1: the spread is staged in shared memory: a block of 256
 *          consecutive vertices accumulates its forces in the bounding box
 *          of their supports, then adds each node that received force to
 *          the lattice with one atomic (for the four-point kernel, whose
 *          supports overlap a dozen-fold); 0 (default): one atomic per
 *          vertex and support node;
 *   [14]   form of the interpolation + advection: 0 (default) eight
 *          threads per vertex, each summing an eighth of the support, the
 *          eighths combined by shuffles; 1 one thread per vertex (fewer
 *          instructions per vertex, less parallelism). Both sum the same
 *          eight partial sums in the same tree with every operation rounded
 *          explicitly: the same positions, bit for bit ([5] gives the
 *          threads per block of either).
 * Block sizes are multiples of 32 in [32, 256].
 * No shape changes a computed value beyond rounding: the order of the
 * spread's float atomics (none with cf_set_spread(ctx, CF_SPREAD_FIXED)) and
 * the force kernel's form [9]. cf_set_launch_shape applies from the next cf_step call;
 * CF_EINVAL for a value outside these sets. */
#define CF_SHAPE_LEN 15
cf_status cf_get_launch_shape(cf_ctx *ctx, int32_t *shape);
cf_status cf_set_launch_shape(cf_ctx *ctx, const int32_t *shape);

/* Bounds of the waits in the fused cell chain (launch shape [6] = 1). A
 * vertex-sum work item waits for the completion count of its cell's tet
 * items; the wait gives up after max_polls polls (default 2^24, each with a
 * 64 ns back-off: about a second), and the step then returns CF_ETIMEOUT
 * instead of hanging. extra_need > 0 raises every cell's required count by
 * that much, so that no wait can succeed: a host-side way to make the waits
 * run out and check that the call reports CF_ETIMEOUT and leaves the
 * context usable (the paper has no counterpart: this exercises the
 * library's failure detection). Defaults: cf_set_chain_wait(ctx, 1 << 24,
 * 0). Applies from the next step call. CF_EINVAL for max_polls < 1 or
 * extra_need < 0. */
cf_status cf_set_chain_wait(cf_ctx *ctx, int64_t max_polls, int32_t extra_need);

/* Autotuner: picks the launch shape by timing coupled steps on the
 * context's own state. One knob at a time (tile shape, fused or separate
 * cell chain, near-field form, far-field load order, force-kernel form,
 * caching of FP32 populations, node pairs of 16-bit populations, where the
 * region is marked, staged spread, form of the interpolation, tet-force,
 * spread and interpolation block sizes), every candidate runs
 * steps_per_candidate (>= 1) coupled steps exactly as cf_step runs them
 * (the same step graphs, far field and cell chain overlapping), timed as a
 * whole with CUDA events, and the fastest candidate is kept. The simulation
 * advances by those steps exactly as under cf_step (32 candidates in all). A fluid-only context has nothing to
 * tune and does not advance. shape_out (may be NULL) receives the chosen
 * shape (CF_SHAPE_LEN values). CF_ESTATE before cf_lbm_init; device errors
 * of the steps as cf_step. */
cf_status cf_autotune(cf_ctx *ctx, int32_t steps_per_candidate, int32_t *shape_out);

/* Elastic vertex forces at the current positions only (Sec. 3.1 per tet,
 * summed per vertex), without touching the fluid. */
cf_status cf_compute_forces(cf_ctx *ctx);

/* cell_id value that addresses every vertex of every cell, in cell order
 * (cf_get_forces, cf_get_positions, cf_set_positions, cf_cell_verts,
 * cf_cell_tets). */
#define CF_ALL_CELLS (-1)

/* Vertex forces [nv][3] of a cell from the last cf_compute_forces or cf_step
 * (the forces at y^t of the last step). */
cf_status cf_get_forces(cf_ctx *ctx, int32_t cell_id, double *out);

/* Current positions y = x_ref + u of a cell, [nv][3]. */
cf_status cf_get_positions(cf_ctx *ctx, int32_t cell_id, double *out);

/* Overwrite the current positions of a cell, [nv][3]. */
cf_status cf_set_positions(cf_ctx *ctx, int32_t cell_id, const double *y);

/* Fluid velocity u(t) of the last step on every node, [nz][ny][nx][3]:
 * rho u = sum_i c_i f_i + F/2 with the force F of that step. */
cf_status cf_get_velocity(cf_ctx *ctx, double *out);

/* Fluid density rho of the last step on every node, [nz][ny][nx]. */
cf_status cf_get_density(cf_ctx *ctx, double *out);

/* Elastic energy E = sum over the cell's tets of V_0 U (Sec. 2-3.1) at the
 * current positions, accumulated in double. */
cf_status cf_get_energy(cf_ctx *ctx, int32_t cell_id, double *out);

/* Taylor deformation of a cell at its current positions (Sec. 3.3), computed
 * on the device: inertia tensor Theta = sum_l V_l (r.r I - r r^T) over the
 * tets (r = tet centroid relative to the volume-weighted cell centroid, V_l
 * the current tet volume), its eigenvalues theta_1 >= theta_2 >= theta_3, the
 * semi-axes a_i (square roots of the paper's expressions, which have units of
 * length squared) and D = (a3 - a1)/(a3 + a1). out[10] = D, D computed from
 * the squared expressions as printed, inclination of the major axis to x in
 * the x-y plane (degrees, (-90, 90]), a1, a2, a3, theta1, theta2, theta3,
 * cell volume. */
cf_status cf_get_taylor(cf_ctx *ctx, int32_t cell_id, double *out);

/* Cell strain (Sec. 6.1, Eq. for the net strain): out[0] = d_max, the
 * largest distance between two vertices of the cell at the current positions
 * (all pairs, on the device, in FP32 from the cell-relative positions),
 * out[1] = (d_max - d_ref) / d_ref with d_ref the reference diameter (2R for a
 * sphere of radius R). CF_EINVAL for an unknown cell, a null output or d_ref
 * not positive and finite. */
cf_status cf_get_cell_strain(cf_ctx *ctx, int32_t cell_id, double d_ref, double *out);

/* Incidence rows of a cell: ptr[nv+1], idx[4 nt] with entries 4*t + c (t
 * local to the cell, ascending within each row). */
cf_status cf_get_csr(cf_ctx *ctx, int32_t cell_id, int32_t *ptr, int32_t *idx);

/* Oriented tets [nt][4] (local indices), B [nt][3][3] with B[k][j] =
 * (J^-1)_kj and V0 [nt] as stored on the device (FP32 values widened).
 * Any output pointer may be NULL. */
cf_status cf_get_mesh(cf_ctx *ctx, int32_t cell_id, int32_t *tets, double *B, double *V0);

/* ------------------------------------------------------------------------
 * Compression between plates and the adjoint (fitting the moduli).
 *
 * The paper compresses a cell between a resting plate and a moving one, with
 * a repulsive force keeping the vertices out of the plates (Sec. 4.2), and
 * fits E and w to force-deformation curves (Sec. 4.3). Here: cells without
 * fluid, a one-sided harmonic plate penalty f_z = k (z_lo - z)_+ -
 * k (z - z_hi)_+ per vertex, quasi-static relaxation by damped steps
 * y <- y + dt (f_el(y) + f_plate(y)), and the top plate's force
 * F = sum_v k (z_v - z_hi)_+ per cell. The adjoint gives dL/d(mu, kappa, w)
 * per cell for any loss L of the plate forces at the ends of recorded
 * relaxation calls.
 * ------------------------------------------------------------------------ */

/* Plate stiffness k >= 0 and plate heights z_lo[c] < z_hi[c] per cell
 * (absolute lattice coordinates). Takes effect for the following calls. */
cf_status cf_plates_set(cf_ctx *ctx, double k_plate, const double *z_lo, const double *z_hi);

/* n >= 1 damped relaxation steps of all cells (unit-mass vertices; the fluid,
 * if any, is not advanced): v <- damping v + dt (f_el + f_plate),
 * y <- y + dt v, with 0 <= damping < 1 (damping = 0: first-order gradient
 * flow y <- y + dt^2 f). Velocities start at zero after cf_tape_clear.
 * record != 0 appends the call to the context's tape, keeping device
 * checkpoints of positions and velocities every 50 steps and at the end
 * (32 bytes per vertex per checkpoint). Errors: CF_ESTATE without cells or
 * plates, CF_ENONFINITE if a position blows up (dt too large for the
 * stiffness), CF_EINVERTED if a tet inverts. */
cf_status cf_relax(cf_ctx *ctx, int32_t n, double dt, double damping, int32_t record);

/* Top-plate force per cell at the current positions, out[ncells]. */
cf_status cf_plate_force(cf_ctx *ctx, double *out);

/* Drop the tape, zero the relaxation velocities and the adjoint state
 * (dL/dy, dL/dv and the accumulated parameter gradients). */
cf_status cf_tape_clear(cf_ctx *ctx);

/* Generation of the context's tape, *out: a counter that grows every time
 * the tape is emptied (cf_tape_clear, or cells added since the last
 * relaxation). A caller that records a forward pass and reverses it later
 * (an autograd function) keeps the generation of its forward and checks it
 * before the reverse pass: a different value means the tape now holds
 * another forward. */
cf_status cf_tape_generation(cf_ctx *ctx, int64_t *out);

/* Reverse the most recent recorded cf_relax call not yet reversed: dF[ncells]
 * is dL/dF for the plate forces at the end of that call. Adds the call's
 * contribution to dL/d(mu, kappa, w) per cell (accumulated in double) and
 * carries dL/dy back to its start (recomputing positions from the
 * checkpoints). Reverse the calls last to first. CF_ESTATE if the tape is
 * empty, or if some cell's material differs from the one the recorded call
 * ran with (the reverse pass would differentiate another forward). */
cf_status cf_relax_adjoint(cf_ctx *ctx, const double *dF);

/* Accumulated dL/d(mu, kappa, w) per cell, out[ncells][3]. */
cf_status cf_adjoint_gradients(cf_ctx *ctx, double *out);

/* Directional derivative of the elastic vertex forces along v[V][3] at the
 * current positions (all cells): out = J v, J = df/dy = -(Hessian of the
 * elastic energy), so J is symmetric and this is also the vector-Jacobian
 * product. */
cf_status cf_force_jvp(cf_ctx *ctx, const double *v, double *out);

/* lambda . df/d(mu, kappa, w) per cell for lambda[V][3] at the current
 * positions, out[ncells][3] (double). */
cf_status cf_force_param_vjp(cf_ctx *ctx, const double *lambda, double *out);

/* Number of vertices / tets of a cell (0 if the id is unknown). */
int32_t cf_cell_verts(const cf_ctx *ctx, int32_t cell_id);
int32_t cf_cell_tets(const cf_ctx *ctx, int32_t cell_id);

/* Message of the last failing call on this context ("" if none). */
const char *cf_last_error(const cf_ctx *ctx);

/* ------------------------------------------------------------------------
 * Vertex forces for callers that cannot allocate device memory.
 *
 * The paper has no counterpart: this is a service of the library. It is for
 * code that is not allowed to call cudaMalloc or any allocating library
 * routine - for example a solver running as a plugin inside a host
 * application that owns all device memory, or a real-time loop whose memory
 * is fixed before it starts. It computes the same elastic vertex forces as
 * cf_compute_forces (Sec. 3.1-3.2 per tet, summed per vertex in incidence-row
 * order) for one cell with one material, without a context, and allocates
 * nothing: the per-corner forces between the two kernels live in a static
 * device array of CF_STATIC_MAX_TETS * 64 bytes (4 MiB), plus 256 KiB of
 * zeros, reserved on every GPU that loads the library until the process
 * exits.
 *
 * All array pointers are DEVICE pointers owned by the caller; the layouts are
 * those the library uses internally (cf_get_mesh and cf_get_csr return the
 * same data on the host):
 *   tets    [nt][4] int32, positively oriented, corner 3 = the paper's
 *           vertex 4, 16-byte aligned;
 *   B       [9][nt] float, B[(3k + j) * nt + t] = (J^-1)_kj of tet t;
 *   V0      [nt] float, reference tet volumes;
 *   u       [nv][4] float, displacement y - x_ref in the first three, 16-byte
 *           aligned;
 *   csr_ptr [nv+1], csr_idx [4 nt] int32: incidence rows, entries 4 t + c
 *           ascending within each row;
 *   f       [nv][4] float output, vertex force in the first three, 16-byte
 *           aligned.
 * mu, kappa, w: the material as in cf_set_material. cuda_stream: the stream
 * to run on (NULL = legacy default stream); the call synchronises it.
 *
 * Returns CF_EINVAL for nt > CF_STATIC_MAX_TETS (the scratch would not fit),
 * nv < 1, nt < 1, a null or misaligned pointer, or a material out of range;
 * CF_EINVERTED / CF_ENONFINITE as cf_compute_forces; CF_ECUDA on a runtime
 * error. Indices are not validated here (cf_mesh_init validates them).
 *
 * The first call on each device (and again the first call after the
 * device's CUDA context was destroyed and created anew, e.g. by
 * cudaDeviceReset) looks up the static array's device address
 * (cudaGetSymbolAddress, with that device current). Every call copies the
 * material from host memory, reads the error word back and synchronises
 * the stream, so no call may be made while its stream is being captured
 * into a CUDA graph. Every call shares the one array: calls that overlap on
 * the GPU (several streams or host threads at once) race and must be
 * serialised by the caller. Each call clears the error word and overwrites
 * the scratch it reads.
 * ------------------------------------------------------------------------ */
#define CF_STATIC_MAX_TETS 65536
cf_status cf_vertex_forces_static(int32_t nv, int32_t nt, const int32_t *tets, const float *B, const float *V0,
                                  const float *u, const int32_t *csr_ptr, const int32_t *csr_idx, double mu,
                                  double kappa, double w, float *f, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* CELLFSI_H */
