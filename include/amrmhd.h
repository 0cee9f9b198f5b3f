/*
 * amrmhd: GB300 (sm_103a) patch-based AMR ideal-MHD level advance.
 *
 * C ABI of libamrmhd.so. Plain pointers and sizes only. Every call returns an
 * amrmhd_status; after an error, amrmhd_last_error() describes it. All device
 * work is ordered on the stream given to amrmhd_create. A context is not
 * thread-safe.
 *
 * The objects follow the paper's statement of patch-based AMR (Carroll-Nellenback
 * et al., "Efficient Parallelization for AMR MHD Multiphysics Calculations",
 * Sec. 2): a patch (grid) is a regular cell array on one level l; cells of level l
 * are R = 2 times finer than level l-1; every patch above level 0 is nested in the
 * coarser level. Ghost zones decouple the hyperbolic advance of each patch
 * (Abstract, Sec. 1); the levels advance in the recursive order 0,1,2,2,1,2,2 with
 * prolongation, advance, synchronization (reflux) and restriction (Sec. 4).
 *
 * Memory ownership: the caller allocates the arena (one device allocation of the
 * size amrmhd_set_hierarchy reports, e.g. a torch tensor) and owns it; the
 * library owns its integer maps, small device scalars and CUDA graphs.
 *
 * State layout inside the arena (for reference; use get/set_state to move data):
 * two state buffers (ping-pong), each holding, for every patch in (level, id)
 * order, 8 field arrays rho, mx, my, mz, E, Bx, By, Bz. A patch with interior
 * n_x x n_y x n_z stores each field over its ghosted box of extent
 * (n_x+9) x (n_y+9) x (n_z+9) (2D: z extent 1), x fastest, index
 * (i+4) + (n_x+9)*((j+4) + (n_y+9)*(k+4)) for patch-local cell (i,j,k),
 * i in [-4, n_x+4); face field B_d at that index is the face at the low side of
 * cell (i,j,k) along d. In 2D, Bz is cell-centred. Element type: double
 * (AMRMHD_FP64) or float (AMRMHD_MIXED).
 */
#ifndef AMRMHD_H
#define AMRMHD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct amrmhd_ctx amrmhd_ctx; /* opaque, library-owned */

typedef enum {
  AMRMHD_OK = 0,
  AMRMHD_EINVAL = -1,    /* bad argument or malformed patch list */
  AMRMHD_ENEST = -2,     /* proper nesting violated (Sec. 2 nesting, 3-cell margin) */
  AMRMHD_EOVERLAP = -3,  /* two patches of one level overlap */
  AMRMHD_ENOMEM = -4,    /* arena too small or a library allocation failed */
  AMRMHD_ECUDA = -5,     /* a CUDA runtime call failed */
  AMRMHD_ENONPHYS = -6,  /* non-finite or non-positive density/pressure found by the CFL reduction */
  AMRMHD_ETIMEOUT = -7,  /* a bounded device wait gave up */
  AMRMHD_ESTATE = -8     /* call out of order (no hierarchy, no arena, wrong step sequence) */
} amrmhd_status;

enum { AMRMHD_FP64 = 0, AMRMHD_MIXED = 1 };
/* Boundary kinds per side of a dimension. A dimension is periodic with
 * AMRMHD_BC_PERIODIC on both sides. Otherwise each side is a zero-gradient
 * outflow (ghost cells copy the nearest domain cell; a ghost face normal to the
 * boundary copies the boundary face) or a fixed inflow (ghost cells and faces
 * take cfg.inflow). */
enum { AMRMHD_BC_PERIODIC = 0, AMRMHD_BC_OUTFLOW = 1, AMRMHD_BC_INFLOW = 2 };

typedef struct {
  int32_t dim;         /* 2 or 3 */
  int32_t base[3];     /* level-0 cells per dimension (base[2] = 1 in 2D) */
  double lo[3], hi[3]; /* physical domain */
  int32_t nghost;      /* must be 4 (= R x stencil reach 2) */
  int32_t ratio;       /* must be 2 */
  int32_t max_level;   /* highest level index allowed (levels 0..max_level) */
  int32_t precision;   /* AMRMHD_FP64: all FP64; AMRMHD_MIXED: FP32 stencil, FP64
                          primitive recovery, registers, dt and CFL */
  int32_t bc[3][2];    /* AMRMHD_BC_* per dimension and side (low, high) */
  double gamma;        /* ratio of specific heats */
  double cfl;          /* Courant number of the sum-form rate (e.g. 0.4) */
  int32_t strict_fp64; /* 1: FP64 kernels compiled without FMA contraction (bitwise
                          reproducible parity build); 0: contraction allowed */
  double inflow[8];    /* conserved inflow state (rho, mx, my, mz, E, Bx, By, Bz) */
} amrmhd_config;

/* A patch: level and half-open box [lo, hi) in level-l cell indices, inside
 * [0, base*2^l). Above level 0, lo and hi must be even (aligned to parent
 * cells). Patch ids are positions in the array given to set_hierarchy. */
typedef struct {
  int32_t level;
  int32_t lo[3];
  int32_t hi[3];
} amrmhd_patch;

/* Creates a context: one AMR mesh of Sec. 2 (levels of grids, refinement ratio
 * R = 2). The paper names the hyperbolic advance but neither its equations nor
 * its boundary kinds: ideal MHD with the ratio of specific heats cfg.gamma and
 * the per-side boundary kinds above are this library's readings. cfg is copied. cuda_stream: the cudaStream_t all work of
 * the context is ordered on; NULL makes the library create its own
 * non-blocking stream at bind_arena (the legacy default stream cannot be
 * captured into a CUDA graph). No device call is made until bind_arena. */
amrmhd_status amrmhd_create(const amrmhd_config* cfg, void* cuda_stream, amrmhd_ctx** out);

/* Destroys a context and frees library-owned memory (not the arena). The paper
 * is silent (a resource call of this library). */
amrmhd_status amrmhd_destroy(amrmhd_ctx* ctx);

/* Installs a hierarchy (patches copied). Validates: boxes inside the level
 * domain and aligned, level 0 tiles the domain, no same-level overlap
 * (AMRMHD_EOVERLAP), every level-l cell's parent cell has all cells within 3
 * parent cells in the parent region (AMRMHD_ENEST). Builds the neighbour lists
 * by inheritance from the parents' neighbours (Sec. 3.1) and all ghost,
 * prolongation, register and restriction maps. *arena_bytes receives the arena
 * size the caller must allocate and bind. Host-only: needs no GPU. */
amrmhd_status amrmhd_set_hierarchy(amrmhd_ctx* ctx, const amrmhd_patch* patches, int32_t n,
                                   size_t* arena_bytes);

/* Binds caller-owned device memory of at least arena_bytes bytes (256-byte
 * aligned) and uploads the maps. Must follow set_hierarchy. The paper is silent
 * on memory layout (its grids live in per-processor arrays); this library's
 * reading is the arena layout above: patches in (level, id) order, 8 fields per
 * patch over its ghosted box. */
amrmhd_status amrmhd_bind_arena(amrmhd_ctx* ctx, void* dev_ptr, size_t bytes);

/* Copies one field of one patch in or out of the current state buffer. The
 * paper is silent on I/O; the fields are the scheme's conserved variables
 * (rho, m, E cell-centred; B on faces for constrained transport).
 * Values are double. Layout: the patch's interior, x fastest: cell fields
 * n_z x n_y x n_x; the face field along d has n_d + 1 entries along d (both
 * boundary faces). src/dst is device memory if *_on_device is 1, else host
 * memory. set_state synchronises nothing; get_state to host synchronises the
 * context stream. */
amrmhd_status amrmhd_set_state(amrmhd_ctx* ctx, int32_t patch, int32_t field, const void* src,
                               int32_t src_on_device);
amrmhd_status amrmhd_get_state(amrmhd_ctx* ctx, int32_t patch, int32_t field, void* dst,
                               int32_t dst_on_device);

/* Packed form of the same: all patches in id order, each in the layout above,
 * concatenated; field f of every patch. amrmhd_packed_size gives the element
 * count of one packed field. */
amrmhd_status amrmhd_packed_size(amrmhd_ctx* ctx, int32_t field, int64_t* count);
amrmhd_status amrmhd_set_state_packed(amrmhd_ctx* ctx, int32_t field, const double* src, int32_t src_on_device);
amrmhd_status amrmhd_get_state_packed(amrmhd_ctx* ctx, int32_t field, double* dst, int32_t dst_on_device);

/* The whole state as one packed array: the 8 packed fields of
 * amrmhd_set_state_packed one after the other (field 0's array, then field
 * 1's, ...; the amrmhd_backward layout). With a page-locked host pointer
 * (cudaHostAlloc, cudaHostRegister, a pinned torch tensor) the packing kernels
 * read or write the host memory directly; with any other host pointer the data
 * moves in one copy per direction through a library-owned staging buffer
 * (allocated on first use); either way the call synchronises the stream. With
 * a device pointer it is stream-ordered. */
amrmhd_status amrmhd_set_state_all(amrmhd_ctx* ctx, const double* src, int32_t on_device);
amrmhd_status amrmhd_get_state_all(amrmhd_ctx* ctx, double* dst, int32_t on_device);

/* The same with float elements (the stored type of AMRMHD_MIXED, so no
 * rounding there; an FP64 context rounds on the way out and widens on the way in). */
amrmhd_status amrmhd_set_state_all_f32(amrmhd_ctx* ctx, const float* src, int32_t on_device);
amrmhd_status amrmhd_get_state_all_f32(amrmhd_ctx* ctx, float* dst, int32_t on_device);

/* Integer parity export. The neighbour rows are the connections Sec. 2 calls
 * neighbors, built by the inheritance of Sec. 3.1; the paper is silent on every
 * row format, and the canonical layout below (ghosts in z,y,x order, sources
 * by smallest (id, index), local indices into the ghosted box) is this
 * library's reading.
 * Exports integer map `which` (AMRMHD_MAP_*) as rows of int32; *width receives
 * the row width, *len the total int count; up to cap ints are written to dst
 * (host memory; dst may be NULL to query the size). Host-only. Row formats:
 *  NEIGHBORS      (p, q, sx, sy, sz): same-level q, periodic shift s, whose
 *                 shifted interior meets p's ghosted box; sorted.
 *  GHOST_CELLS    (p, Ldst, kind, src, Lsrc) for every ghost cell of p in z,y,x
 *                 order; kind 0 = same-level copy, 1 = prolongation from the parent
 *                 cell Lsrc of coarse patch src, 2 = boundary copy from p's own
 *                 Lsrc (the nearest domain position), 3 = inflow (src = Lsrc = -1).
 *  GHOST_FACES    (p, d, Ldst, kind, src, Lsrc), faces not owned by p; the
 *                 same-level source is the owner with the smallest (id, index).
 *  CF_FACES       (l, qc, d, Lface, side, pf, Lfine): coarse faces between a
 *                 covered and an uncovered level-(l-1) cell; qc owns the uncovered
 *                 cell; side = +1 if the face is that cell's low face; pf holds the
 *                 fine sub-faces, Lfine is the first (z,y,x order).
 *  CF_EDGES       (l, qc, c, Ledge, pf, Lfine): c-edges with 1..3 covered cells
 *                 around; owners with the smallest (id, index).
 *  EMF_FACES      (l, qc, d, Lface, e0, e1, e2, e3): every owner copy of a coarse
 *                 face with both cells uncovered touching a C/F edge; e* are
 *                 CF_EDGES row numbers or -1 (slots: t2-edges at the face and
 *                 one up along t1, t1-edges at the face and one up along t2,
 *                 t1 = (d+1)%3, t2 = (d+2)%3).
 *  RESTRICT_CELLS (l, qc, Lcell, pf, Lchild0).
 *  RESTRICT_FACES (l, qc, d, Lface, pf, Lfine0) for every owner copy.
 *  REFLUX_CELLS   (l, qc, Lcell, f0..f5): CF_FACES row numbers of the cell's
 *                 x-, x+, y-, y+, z-, z+ faces or -1.
 * Local indices L are into the patch's ghosted box of extent n+9 per dimension. */
enum {
  AMRMHD_MAP_NEIGHBORS = 0, AMRMHD_MAP_GHOST_CELLS = 1, AMRMHD_MAP_GHOST_FACES = 2,
  AMRMHD_MAP_CF_FACES = 3, AMRMHD_MAP_CF_EDGES = 4, AMRMHD_MAP_EMF_FACES = 5,
  AMRMHD_MAP_RESTRICT_CELLS = 6, AMRMHD_MAP_RESTRICT_FACES = 7, AMRMHD_MAP_REFLUX_CELLS = 8
};
amrmhd_status amrmhd_export_map(amrmhd_ctx* ctx, int32_t which, int32_t* dst, int64_t cap, int64_t* len,
                                int32_t* width);

/* Ghost fill of every patch of `level` (same-level copies incl. periodic
 * images; with substep 1 on a level above 0 also prolongation of the other
 * ghosts from the parent level's state at the start of its current sub-step).
 * Substep 2 refreshes only same-level ghosts (prolonged ghosts keep the values
 * evolved by substep 1: extended ghost zones, Abstract and Sec. 1). */
amrmhd_status amrmhd_fill_ghosts(amrmhd_ctx* ctx, int32_t level, int32_t substep);

/* The (A)dvance of Sec. 4 for every grid of `level`: the hyperbolic advance of
 * each grid decoupled by its ghost zones (Abstract, Sec. 1). The paper does not
 * give the scheme; this library's reading is MUSCL-Hancock with the primitive
 * half-step predictor and minmod slopes, HLLD fluxes (Miyoshi & Kusano 2005)
 * and constrained transport with Gardiner-Stone edge EMFs.
 * Advances every patch of `level` by dt.
 * Level 0 updates the interior; above level 0, substep 1 updates the interior
 * plus 2 ghost layers and substep 2 the interior. Records the coarse-side
 * registers of the next finer level's C/F boundary and the fine-side registers
 * of this level's boundary for this substep. Must follow fill_ghosts(level). */
amrmhd_status amrmhd_advance_level(amrmhd_ctx* ctx, int32_t level, double dt, int32_t substep);

/* Synchronization and restriction of fine_level into fine_level-1 (Sec. 4's S
 * and R): reflux of the C/F flux and EMF registers into uncovered coarse cells
 * and faces, then averaging of the covered coarse cells and of the coarse
 * faces in the closure of the fine region. Must follow both substeps of
 * fine_level after advance_level(fine_level-1). */
amrmhd_status amrmhd_reflux_restrict(amrmhd_ctx* ctx, int32_t fine_level);

/* Time step of the coarse step. The paper is silent on the time step; this
 * library's reading is the sum-form rate and one global dt0 per coarse step:
 * dt0 = cfl / max_l (2^-l max over level-l cells of sum_d (|v_d| + c_f,d)/dx_d),
 * computed on the device in FP64; synchronises the stream.
 * AMRMHD_ENONPHYS if a density or pressure is not finite and positive. */
amrmhd_status amrmhd_cfl_dt(amrmhd_ctx* ctx, double* dt0);

/* n_coarse full coarse steps (CFL dt each, then the whole recursion of Sec. 4:
 * level order 0,1,2,2,1,2,2 with P, O, A, S, R per level; finer levels advance
 * concurrently with the coarser advance, Sec. 4's threads; the paper does
 * not fix the ghost refresh: here fine ghosts are prolonged once per parent step
 * and self-evolved, same-level ghosts refreshed every sub-step), run as a
 * captured CUDA graph. dt_used (host, may be NULL) receives the n_coarse dt0
 * values. Synchronises the stream at the end and reports device errors. */
amrmhd_status amrmhd_step(amrmhd_ctx* ctx, int32_t n_coarse, double* dt_used);

/* The same n_coarse coarse steps, stream-ordered: the call returns once the
 * steps are queued on the context's stream, without waiting for them, so that
 * a caller can queue further work (state I/O with device pointers, copies on
 * its own streams ordered by events) while they run. Device errors of the
 * steps (a non-physical state, a queue wait that ran out) stay in the
 * context's error word and are reported by the next synchronising call
 * (amrmhd_sync, amrmhd_step, amrmhd_cfl_dt); a dt0 of a step that follows such
 * an error is 0 (the state does not change). Like amrmhd_step, the paper is
 * silent on how the steps are issued. */
amrmhd_status amrmhd_step_async(amrmhd_ctx* ctx, int32_t n_coarse);

/* Waits for the work queued on the context's stream and reports (then clears)
 * a device error: AMRMHD_ENONPHYS, AMRMHD_ETIMEOUT, else AMRMHD_OK. */
amrmhd_status amrmhd_sync(amrmhd_ctx* ctx);

/* n_coarse coarse steps with the prescribed dt0 sequence dt_seq (host, n_coarse
 * positive values; level l steps with dt0 2^-l) instead of the CFL dt, with
 * plain launches: the forward map that amrmhd_backward differentiates.
 * Synchronises the stream. */
amrmhd_status amrmhd_step_dt(amrmhd_ctx* ctx, int32_t n_coarse, const double* dt_seq);

/* Discrete adjoint of n_coarse coarse steps with the dt0 sequence dt_seq (host;
 * dt is a constant of the map, not differentiated). The paper has no adjoint;
 * the conventions here (dt fixed, the forward's branch at every kink, one entry
 * per stored copy) are this library's. The level advance
 * (Sec. 4: prolongation, advance, reflux and restriction of the recursive
 * level order) is differentiated exactly: the call returns
 *   dL_dU0 = (dU_final / dU0)^T dL_dUfinal
 * where U0 is the context's state at the call and U_final the state after the
 * steps. Both are DEVICE arrays of float64 in the packed state layout of all
 * 8 fields one after the other (field 0's packed array, then field 1's, ...;
 * each as amrmhd_set_state_packed: patches in id order, a patch's interior
 * cells, or its own faces along the field's direction, x fastest). A face
 * stored by two patches has one entry per copy: dL_dUfinal may split the
 * derivative of a shared face among its copies in any way, and dL_dU0 gives
 * each copy its own partial derivative (the derivative with respect to the
 * face value is their sum).
 * The forward is run up to the last segment's start storing a checkpoint of
 * every level's state every ckpt_every coarse steps, then each segment is
 * recomputed storing the filled state of every level sub-step, and swept
 * backwards (ckpt_every >= n_coarse: one segment, no separate forward pass). Branches (minmod, HLLD
 * cases, upwinding) take the forward's decisions. Adjoint accumulation is FP64;
 * the local Jacobians of the HLLD flux and the half-step predictor are
 * evaluated in the forward's compute type (FP64, or FP32 in mixed precision, on
 * the mixed-precision trajectory), the others in FP64.
 * The first call (and any call needing more checkpoint or snapshot room) allocates
 * device memory owned by the context: about state + 70 scratch arrays per patch
 * in FP64, n_coarse/ckpt_every checkpoints and ckpt_every x (2^nlevels - 1)
 * level snapshots. On return the context holds U0 again. Synchronises the stream. */
amrmhd_status amrmhd_backward(amrmhd_ctx* ctx, int32_t n_coarse, const double* dt_seq, int32_t ckpt_every,
                              const double* dL_dUfinal, double* dL_dU0);

/* The forward of amrmhd_backward recorded: the n_coarse steps of amrmhd_step_dt
 * storing a checkpoint of every level's state every ckpt_every coarse steps, so
 * that amrmhd_backward_recorded can differentiate them without running the
 * forward again (the state-changing calls of this header drop the record:
 * stepping, advancing, refluxing, setting the state, a new hierarchy or arena,
 * a regrid, a backward). Same errors as amrmhd_backward. Synchronises the stream. */
amrmhd_status amrmhd_step_dt_ckpt(amrmhd_ctx* ctx, int32_t n_coarse, const double* dt_seq, int32_t ckpt_every);

/* amrmhd_backward of the steps of the last amrmhd_step_dt_ckpt, the context
 * still at their final state: dL_dU0 = (dU_final / dU0)^T dL_dUfinal with U0
 * the state before those steps (layouts and conventions of amrmhd_backward); the
 * segments are recomputed from the recorded checkpoints and swept backwards. On
 * return the context holds U0 and the record is dropped. AMRMHD_ESTATE if no
 * record matches the current state. Synchronises the stream. */
amrmhd_status amrmhd_backward_recorded(amrmhd_ctx* ctx, const double* dL_dUfinal, double* dL_dU0);

/* The gradient with respect to the initial velocity (the configuration's
 * control: the adjoint of the level advance gives dL/dU0; the paper has no
 * adjoint, and the chain rule here is this library's reading: rho, p and B are
 * held while v varies). From the packed initial state u0 and dL/dU0 (DEVICE
 * arrays in the amrmhd_backward layout; only the cell fields rho, mx, my, mz,
 * E are read: the first 5 packed fields, ncells entries each) it writes
 * dL_dv0 (DEVICE, 3 packed cell fields vx, vy, vz, ncells each):
 * dL/dv_c = rho (dL/dm_c + v_c dL/dE), v = m / rho. Stream-ordered on
 * cuda_stream (NULL: the legacy default stream). AMRMHD_EINVAL for bad
 * arguments, AMRMHD_ECUDA if the launch fails. */
amrmhd_status amrmhd_grad_velocity(int64_t ncells, const double* u0, const double* dL_dU0, double* dL_dv0,
                                   void* cuda_stream);

/* The local transposed Jacobians that amrmhd_backward applies at every face
 * and cell, exposed for verification: gx = J^T g at n points, FP64, one point
 * per row, all arrays HOST, row-major.
 *  which 0: the HLLD flux (the scheme's Riemann solver, Miyoshi & Kusano
 *           2005; the paper names no solver)
 *           of a rotated face, x = (rho, u_n, u_t, u_u, p, B_t, B_u) of the left
 *           state, the same of the right state, then B_n (15 per row);
 *           g = the 7 flux components (rho, m_n, m_t, m_u, E, B_t, B_u);
 *           dim is ignored.
 *  which 1: the half-step primitive predictor of one cell, wh = w -
 *           sum_d h[d] A_d(w) s_d, x = (w[8], s_0[8], .., s_{dim-1}[8]) with
 *           w = (rho, vx, vy, vz, p, Bx, By, Bz) and s_d its slopes along d
 *           (8 + 8 dim per row); g = 8 per row; h[dim] the factors dt/(2 dx_d).
 *  method 0: the hand-written transposes amrmhd_backward uses in FP64; 1: the
 *            same formulas evaluated with forward-mode dual numbers (FP64);
 *            2: the hand-written transposes in FP32 (x, g and h rounded to
 *            FP32), as the mixed-precision adjoint applies them.
 * Branches are the ones the forward takes at x. Allocates and frees device
 * memory for the call and synchronises the device. Errors: AMRMHD_EINVAL for a
 * bad which/dim/method, a negative n, NULL arrays or gamma <= 1; AMRMHD_ECUDA if
 * an allocation, copy or launch fails. */
amrmhd_status amrmhd_local_vjp(int32_t which, int32_t dim, int64_t n, const double* x, const double* g, double gamma,
                               const double* h, int32_t method, double* gx);

/* Diagnostic: the FP32 <-> FP64 conversions of the mixed-precision recovery
 * (the paper says nothing about precision; the mixed mode's split, FP64 for the
 * energy balance p = (gamma-1)(E - ke - me), is this library's design: the mixed path widens its FP32 operands and rounds
 * the FP64 pressure back to FP32 with integer operations on the bit patterns). For i < n (host arrays):
 * x_narrow[i] = x[i] rounded to FP32 (nearest even, results below 2^-126
 * flushed to a signed zero), y_widen[i] = y[i] widened to FP64 (FP32
 * subnormals flushed), and x_narrow_hw[i], y_widen_hw[i] the same conversions
 * by the compiler's casts. on_device 0 evaluates everything on the host CPU;
 * 1 in a kernel compiled as the mixed path is (FP32 denormals flushed), with
 * the hardware conversion instructions as the reference. Allocates and frees
 * device memory for on_device 1 and synchronises the device. Errors:
 * AMRMHD_EINVAL for on_device not 0/1, n < 0 or NULL arrays with n > 0;
 * AMRMHD_ECUDA if an allocation, copy or launch fails. */
amrmhd_status amrmhd_fp_convert(int32_t on_device, int64_t n, const double* x, const float* y, float* x_narrow,
                                double* y_widen, float* x_narrow_hw, double* y_widen_hw);

/* Measurement: the device's floating-point multiply-add throughput (FP32 with
 * fp64 = 0, FP64 with fp64 = 1) in operations per second (a multiply-add counts
 * 2), from a kernel of independent multiply-add chains on every SM (8 blocks of
 * 256 threads per SM, best of 5 timed launches after one warm-up, CUDA events on
 * the legacy default stream); *sms (may be NULL) receives the SM count. The
 * roofline of an ALU-bound kernel is taken against this number. Allocates and
 * frees a small device buffer and synchronises the device. Errors:
 * AMRMHD_EINVAL for bad arguments, AMRMHD_ECUDA if a CUDA call fails. */
amrmhd_status amrmhd_alu_peak(int32_t fp64, double* flops_per_s, int32_t* sms);

/* Diagnostic: the primitive recovery (conservative -> primitive, the first
 * step of the advance; the paper is silent on it) exactly as the mixed-precision
 * advance runs it, for n cells (host arrays, row-major): u = (rho, mx, my, mz, E)
 * (5 per cell), bl and br = the low and high face values of (Bx, By, Bz) (3 per
 * cell) -> w = (rho, vx, vy, vz, p, Bx, By, Bz) with B the face means (8 per
 * cell). All FP32 except the energy balance p = (gamma-1)(E - ke - me), which
 * runs in FP64 with ke and me formed as double-float FP32 pairs. Allocates and
 * frees device memory for the call and synchronises the device. Errors:
 * AMRMHD_EINVAL for n < 0, NULL arrays with n > 0 or gamma <= 1; AMRMHD_ECUDA if
 * an allocation, copy or launch fails. */
amrmhd_status amrmhd_recover_mixed(int64_t n, const float* u, const float* bl, const float* br, double gamma,
                                   float* w);

/* Regrid: rebuilds every level above 0, coarse to fine, up to max_levels
 * levels (Sec. 2: the grids follow the flagged regions; a new grid takes its
 * data from the preceding overlapping grid of its level, else from the coarser
 * level). For each level l < max_levels - 1, in order:
 *  1. flag the level-l cells with max_d |rho(i+1) - rho(i-1)| / (2 rho) > theta
 *     (FP64 from the stored values, ghosts filled first);
 *  2. buffer the flags by 2 cells inside the level-l region;
 *  3. mark the aligned blocks of 4^dim level-l cells that hold a buffered flag
 *     and whose surrounding 3 cells lie in the level-l region (proper nesting);
 *  4. merge the marked blocks greedily in z,y,x order (runs along x, then y,
 *     then z, at most 4 blocks per side) and refine by 2: new level-(l+1)
 *     patches of 8..32 cells per side, aligned to 8 fine cells;
 *  5. fill the new level: cells and faces copied from the old level l+1 where
 *     it covered the parent cell, else prolonged from level l; where copied and
 *     prolonged fine faces meet on a coarse face, the interior faces of the
 *     prolonged coarse cell get the least-norm correction that makes every
 *     child divergence-free.
 * The first level without boxes ends the hierarchy. Level 0 is kept. Patch ids
 * of the result: level 0 as before, then each level's boxes in creation order
 * (amrmhd_get_patches). After the call the context owns a new arena allocated
 * with cudaMalloc (a caller's arena is no longer referenced); the adjoint
 * workspace and captured graphs are released. Base sizes must be divisible by 4.
 * Steps 1-3 run on the device by default (AMRMHD_OPT_DEVICE_CLUSTER; step 4 on
 * the host from the block marks), the maps of the intermediate and final
 * hierarchies and of step 5 on the device when AMRMHD_OPT_DEVICE_MAPS allows;
 * the results do not depend on either option. With AMRMHD_REGRID_TRACE set in
 * the environment each stage's host timings are printed to stderr.
 * Synchronises the stream. */
amrmhd_status amrmhd_regrid(amrmhd_ctx* ctx, double theta, int32_t max_levels);

/* Steps 2-4 of amrmhd_regrid alone on the context's hierarchy (host only, no
 * device work): the level+1 boxes (n x 7 int32: level, lo[3], hi[3]) from the
 * flagged level cells given as nflags (x, y, z) triples; flags outside the
 * level's region are ignored. out may be NULL to query *n. */
amrmhd_status amrmhd_regrid_boxes(amrmhd_ctx* ctx, int32_t level, const int32_t* flags, int64_t nflags,
                                  int32_t* out, int32_t cap, int32_t* n);

/* The current patch list (ids in order); out may be NULL to query *n. */
amrmhd_status amrmhd_get_patches(amrmhd_ctx* ctx, amrmhd_patch* out, int32_t cap, int32_t* n);

/* Integer queries: AMRMHD_Q_* */
enum {
  AMRMHD_Q_NPATCH = 0, AMRMHD_Q_NLEVEL = 1, AMRMHD_Q_CELLS = 2, AMRMHD_Q_CELL_UPDATES_PER_STEP = 3,
  AMRMHD_Q_ARENA_BYTES = 4, AMRMHD_Q_KERNEL_LAUNCHES = 5,
  /* host wall time of the last amrmhd_regrid in microseconds: flagging (the
   * fills; with the host clustering also the flag kernel and list copy),
   * clustering, building the stage hierarchies, maps and arenas, and the data
   * transfer */
  AMRMHD_Q_REGRID_FLAG_US = 6, AMRMHD_Q_REGRID_CLUSTER_US = 7, AMRMHD_Q_REGRID_BUILD_US = 8,
  AMRMHD_Q_REGRID_TRANSFER_US = 9,
  /* of AMRMHD_Q_REGRID_BUILD_US, the building of hierarchies and maps
   * (amrmhd_set_hierarchy; the rest is device memory and map upload) */
  AMRMHD_Q_REGRID_MAPS_US = 10,
  /* of AMRMHD_Q_REGRID_TRANSFER_US, the building of the transfer maps */
  AMRMHD_Q_REGRID_TRANSFER_MAPS_US = 12,
  /* host wall time of the last amrmhd_set_hierarchy in microseconds: validation and
   * neighbour lists (host), the ghost boxes, the register/reflux/restriction maps */
  AMRMHD_Q_MAPS_HOST_US = 13, AMRMHD_Q_MAPS_GHOST_US = 14, AMRMHD_Q_MAPS_REGISTERS_US = 15,
  /* raises by the density and pressure floors since bind_arena (amrmhd_set_floors);
   * synchronises the stream */
  AMRMHD_Q_FLOOR_EVENTS = 11
};
amrmhd_status amrmhd_query(amrmhd_ctx* ctx, int32_t what, int64_t* value);

/* Density and pressure floors (0, 0: off, the default). The paper is silent on
 * floors; the reading for strong shocks: every recovery of the advance and the
 * CFL reduction raises a density below rho_min to rho_min before forming the
 * velocity and pressure, then a pressure below p_min to p_min, counting every
 * raise (AMRMHD_Q_FLOOR_EVENTS). Floors act on the primitives only, so where
 * they act the advance is not conservative; they are never needed in smooth
 * problems. amrmhd_backward refuses to run with floors set (AMRMHD_ESTATE).
 * AMRMHD_EINVAL for negative or non-finite values. Captured graphs are
 * rebuilt at the next step. */
amrmhd_status amrmhd_set_floors(amrmhd_ctx* ctx, double rho_min, double p_min);

/* Options (set before set_hierarchy): AMRMHD_OPT_* */
enum {
  AMRMHD_OPT_ADVANCE = 0,  /* 0 (default): mixed precision in 3D uses one fused kernel per
                              level advance (no scratch); FP64 and 2D use the staged kernels
                              batched over the level; 1: the staged kernels launched one
                              patch at a time (baseline); 2: the staged kernels batched;
                              3: the fused kernel (3D) in either precision */
  AMRMHD_OPT_GRAPH = 1,    /* 1 (default): amrmhd_step replays a CUDA graph; 0: plain launches */
  AMRMHD_OPT_TILE = 2,     /* fused 3D advance tile: -1 default (the autotuned tile per level and
                              sub-step kind after amrmhd_autotune, else 16x8 FP32, 8x8 FP64), 0: 16x16
                              tile with 256 threads, 1: 16x16 / 512, 2: 16x8 / 256, 3: 8x8 / 256,
                              4: 12x12 / 256 */
  AMRMHD_OPT_CONCURRENT = 3, /* 1 (default): in a coarse step the two sub-steps of level l+1 run on a
                              side stream concurrently with the advance of level l (they meet
                              before the reflux), and the CFL reduction runs beside the level-0
                              ghost fill; 0: one stream, strictly in the recursive order */
  AMRMHD_OPT_HOST_IO = 4,   /* whole-state I/O with host buffers (amrmhd_set/get_state_all*): 0 (default):
                              page-locked buffers are read and written in place by the packing kernels
                              over the host link, other host memory through a device staging buffer;
                              1: every host buffer through the staging buffer (copy engine) */
  AMRMHD_OPT_DIRECT_HALO = 5, /* 1 (default): the 3D base level of a one-level hierarchy whose equal patches
                              tile the fully periodic domain is advanced by the fused kernel reading its
                              halo from the neighbour patches' interiors, and amrmhd_step skips that
                              level's same-level ghost fill (its ghost cells are then not kept up to
                              date; amrmhd_fill_ghosts still fills them); 0: fill, then read the
                              ghosts. The results are the same either way. */
  AMRMHD_OPT_QUEUE = 6,      /* 1: a 3D hierarchy of 2 to 12 levels on the fused path advances through the
                              device work queue: per sub-step of the finest level one persistent launch
                              of the resident CTAs takes tasks in ticket order, finest level first (the
                              paper's threaded level advances with preference to the finer levels,
                              Sec. 4): the finest level's same-level ghost copies, then every starting
                              level's advance tiles, each tile after the copies into its patch (bounded
                              waits on per-patch counters; a wait that runs out makes amrmhd_step return
                              AMRMHD_ETIMEOUT). Results equal the level-by-level launches. 0 (default):
                              per-level launches, finer levels on side streams. */
  AMRMHD_OPT_QUEUE_TILE = 7, /* tile of the queue's advance tasks: 3 (default) 8x8, 2 16x8 */
  AMRMHD_OPT_QUEUE_WITHHOLD = 8, /* test switch, 0 (default) or 1: the first patch of the finest level
                              waits in the first batch of a coarse step for one fill task more than
                              exist, so the wait runs out (after 0.5 s) and amrmhd_step returns
                              AMRMHD_ETIMEOUT; the device stays usable */
  AMRMHD_OPT_QUEUE_BALANCE = 9 /* how a coarser level's advance tiles are shared out over the queue
                              launches of its sub-step: 1 (default) so that every launch's predicted
                              total work (the finer levels' tiles included) reaches one common level,
                              the paper's load balancing (Sec. 5) with the launches of a coarse step
                              as its processors; 0 equal numbers of tiles per launch */,
  AMRMHD_OPT_DEVICE_MAPS = 10 /* where amrmhd_set_hierarchy builds the register, reflux and restriction
                              maps (the coarse-fine faces and edges of the synchronize step, Sec. 4, and
                              the restricted cells and faces): -1 (default) on the device when the
                              process sees one, else on the host; 1 on the device (then
                              amrmhd_set_hierarchy needs a device and returns AMRMHD_ECUDA or
                              AMRMHD_ENOMEM if it fails); 0 on the host. Both give the same rows in the
                              same order (amrmhd_export_map copies device-built rows back on demand).
                              Takes effect at the next amrmhd_set_hierarchy or amrmhd_regrid. */,
  AMRMHD_OPT_DEVICE_CLUSTER = 11 /* where amrmhd_regrid clusters the flagged cells into new boxes (its
                              steps 2-4): 1 (default) on the device (flag test, 2-cell buffer and
                              block marks in dense bytes of the clustering frame; only the block marks
                              are copied back for the greedy merge), 0 on the host (the flag list is
                              copied back). Both give the same boxes in the same order. */,
  AMRMHD_OPT_ZCHUNK = 12 /* z planes per CTA of the fused 3D advance: -1 (default) the length
                              amrmhd_autotune chose for the level and sub-step kind (the whole column
                              before it runs), 0 the whole column, n in 1..4096 chunks of n planes
                              (each chunk restarts the z march 2 planes below its first plane: more
                              CTAs with shorter marches, for levels of few or tall patches, at the cost
                              of recomputed planes), -2 whole columns except those of the launch's last
                              partial wave of resident CTAs, which run as two halves each when they
                              fill at most half of that wave (a level of many columns). The results
                              are the same bit for bit for every choice. May be changed between steps (it is read at the next launch or
                              graph capture). */
};
amrmhd_status amrmhd_set_option(amrmhd_ctx* ctx, int32_t option, int64_t value);

/* Autotuner of the fused 3D advance: for every level, and separately for its
 * interior-only advance and (above level 0) its advance with 2 extended ghost
 * layers (sub-step 1), times `trials` advances with each tile variant
 * (AMRMHD_OPT_TILE 0..4) and each z chunk (AMRMHD_OPT_ZCHUNK 0, -2, 4, 8 and 16 where
 * shorter than the level's column) on the current state with CUDA events and
 * keeps the fastest pair (used while AMRMHD_OPT_TILE, respectively
 * AMRMHD_OPT_ZCHUNK, is -1; amrmhd_tile_choice reads it). The state is not changed: an
 * advance reads the current buffer and writes the other one. tiles (host, may
 * be NULL) receives the interior-only choice per level (-1 where the staged
 * kernels are used, i.e. FP64 by default and 2D). The variants compute the
 * same formulas in the same order: identical results in the strict FP64 build,
 * FP32 rounding differences in mixed precision (where the compiler may
 * contract multiply-adds differently per variant). Synchronises the stream. */
amrmhd_status amrmhd_autotune(amrmhd_ctx* ctx, int32_t trials, int32_t* tiles);

/* The fused 3D advance's launch shape in use for level `level`: kind 0 its
 * interior-only advance, kind 1 its advance with 2 extended ghost layers
 * (levels above 0). *tile (host) receives the tile variant (AMRMHD_OPT_TILE
 * numbering; -1 where the staged kernels advance the level), *zlen (host) the z
 * planes per CTA (AMRMHD_OPT_ZCHUNK numbering: 0 the whole column, -2 the last
 * partial wave's columns halved), both after the options and the
 * autotuner's choice. The paper is silent on launch shapes (they are this
 * implementation's mapping of a level's grids onto the GPU). Errors:
 * AMRMHD_ESTATE without a hierarchy; AMRMHD_EINVAL for a null pointer, a level
 * out of range or kind not 0 or 1. */
amrmhd_status amrmhd_tile_choice(amrmhd_ctx* ctx, int32_t level, int32_t kind, int32_t* tile, int32_t* zlen);

const char* amrmhd_last_error(const amrmhd_ctx* ctx);

/* SM partitions, for the single-GPU analogue of the paper's weak-scaling
 * experiment (Sec. 6: the work per processor fixed while processors are
 * added). amrmhd_sm_partition_create makes a stream of the current device whose
 * kernels run only on one group of at least sm_count SMs (a green context of
 * the CUDA driver; the group is rounded up to the device's partition
 * granularity): *sms receives the group's SM count, *stream the stream (pass it
 * to amrmhd_create and set AMRMHD_OPT_CONCURRENT to 0, so that no work of the
 * context leaves it), *handle the partition. amrmhd_sm_partition_destroy
 * synchronises and releases the stream and the partition (contexts using the
 * stream must be destroyed first). Device memory allocated outside the
 * partition (the arena) is used as is. Errors: AMRMHD_EINVAL for bad arguments
 * or a count above the device's SMs, AMRMHD_ECUDA if a driver call fails. */
amrmhd_status amrmhd_sm_partition_create(int32_t sm_count, void** stream, int32_t* sms, void** handle);
amrmhd_status amrmhd_sm_partition_destroy(void* handle);
/* The calling thread's last failure of amrmhd_sm_partition_create (the step
 * that failed and its driver code), "" if none. */
const char* amrmhd_sm_partition_error(void);

/* Advance of ONE patch that allocates no device memory (no counterpart in the
 * paper: it exists for callers that cannot call cudaMalloc, e.g. code running
 * under a memory pool that forbids new allocations, a real-time loop that must
 * not enter the allocator, or a library handed only the state pointers).
 * Mixed precision (FP32 stencil, FP64 primitive recovery), the same staged
 * kernels as advance_level. Its intermediate arrays live in one fixed device
 * array of 256 B + 70 x 16384 x 4 B (about 4.6 MB) that every GPU loading the
 * library holds until the process exits.
 *  u_in:  device pointer, 8 consecutive float arrays (rho, mx, my, mz, E, Bx,
 *         By, Bz), each over the ghosted box of extent (n_x+9)(n_y+9)(n_z+9)
 *         (2D: (n_x+9)(n_y+9)), x fastest, index as in the state layout above;
 *         the caller fills the 4 ghost layers (cells and faces).
 *  u_out: device pointer, same layout; the cells of the interior widened by w
 *         layers and their faces are written, nothing else.
 *  dim 2 or 3; n[dim] interior extents; dx[dim] cell sizes; gamma; dt; w = 0
 *  (interior) or 2 (interior + 2 ghost layers); cuda_stream (NULL = legacy
 *  default stream). Returns AMRMHD_EINVAL for bad arguments or when
 *  (n_x+9)(n_y+9)(n_z+9) > 16384 (e.g. 3D patches above 16^3), AMRMHD_ECUDA if
 *  a CUDA call fails. The first call on a device looks up the array's device
 *  address (once per device, with that device current): make that first call
 *  before any stream capture. Every call shares the array and it keeps the last
 *  call's contents (every entry read is written earlier in the same call, so
 *  nothing needs clearing); calls that overlap on the GPU race on it. */
amrmhd_status amrmhd_advance_patch_noalloc(const float* u_in, float* u_out, int32_t dim, const int32_t* n,
                                           const double* dx, double gamma, double dt, int32_t w, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* AMRMHD_H */
