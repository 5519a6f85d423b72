/*
 * ewave.h -- C ABI of the GB300 (sm_103a) library for the 2D acoustic PML wave operator of
 * Ravelo, Schreiber & Peixoto, "High-order exponential integration for seismic wave
 * modeling" (arXiv 2401.16322), and of the time integrators the paper compares.
 *
 * Problem statement (Sec. 3, Eq. 1st_ord): dU/dt = H U + f(t), U = (u, v, w_x, w_y), with H
 * the semi-discrete operator of Eq. (1) (Sec. 2): PML damping beta (Sec. 2), 8th-order (or
 * 4th-order) staggered finite differences (Sec. 2.1, Eqs. spatial_8th_1/2), zero extension
 * on the sides and bottom, and the free-surface rows of Sec. 2.2 / Appendix A on top.
 * f is a Ricker point source in the v-row.
 *
 * Conventions
 *  - Plain C, no exceptions.  Every function returns an int status (EWV_OK = 0, negative on
 *    error); ewv_last_error() gives a one-line message for the last failing call on a handle.
 *  - Memory ownership: the caller owns every grid-sized device buffer (state, model
 *    parameters, integrator workspace, seismograms) and passes raw device pointers plus byte
 *    sizes; sizes come from ewv_layout() / ewv_workspace_bytes().  The library owns only
 *    small device metadata (descriptors, per-step scalars, reduction partials, Hessenberg
 *    matrices, coefficients).  Host arrays passed in are copied and never kept.
 *  - Device pointers must be 256-byte aligned (torch allocations are); sizes are checked.
 *  - Threading: calls on one handle are serialised on its stream (ewv_set_stream); distinct
 *    handles are independent.  Calls return after enqueueing work unless stated otherwise.
 *  - Asynchronous errors: a step call ends its GPU work with a scan of every shot's state;
 *    a non-finite value (NaN or infinity) or a TMA pipeline wait that gave up sets the
 *    handle's error word, which is copied to the host without waiting.  The next step call
 *    on the handle, or ewv_sync, returns EWV_ERR_NONFINITE or EWV_ERR_TIMEOUT for it (and
 *    clears it); such a step call enqueues nothing.
 *  - Grid: nodes (i, j), i = 0..nx-1 left to right, j = 0..ny-1 top to bottom (j = 0 is the
 *    free surface when enabled).  w_x lives at (i+1/2, j), i = 0..nx-2; w_y at (i, j+1/2),
 *    j = 0..ny-2; w_y is the paper's w_y for its upward y axis.
 *  - Device state layout ("padded"): one state vector = 4 fields (u, v, w_x, w_y), each
 *    [ny][pitch] of the model's precision, field-major; w_x column nx-1, w_y row ny-1 and
 *    columns nx..pitch-1 are padding and hold zeros.  A model with nshots shots stores
 *    nshots such vectors back to back (the "state" buffer).
 *  - Compact host layout (ewv_set_state / ewv_get_state): float64, u [ny][nx], v [ny][nx],
 *    w_x [ny][nx-1], w_y [ny-1][nx], concatenated (n = 2 nx ny + (nx-1) ny + nx (ny-1)).
 *  - Three dimensions (dims = 3; not in the paper, which is 2D): the PML of Eq. (1) carried
 *    to three axes with an auxiliary field psi (psi_t = u), U = (u, v, w_x, w_y, w_z, psi):
 *      v_t   = -(bx by + by bz + bx bz) u - (bx + by + bz) v - bx by bz psi
 *              + c^2 (u_xx + u_yy + u_zz + d_x w_x + d_y w_y + d_z w_z) + f,
 *      w_a,t = -b_a w_a + (sum of the other two b's - b_a) d_a u
 *              + (product of the other two b's) d_a psi              (a = x, y, z),
 *      psi_t = u.
 *    With one axis undamped and a field constant along it, the u, v and remaining w rows are
 *    exactly Eq. (1) on the other two axes.  z is vertical, with node planes k = 0..nz-1 and
 *    k = 0 the free surface: z takes the role of the 2D y axis (upward derivative, Appendix A
 *    rows, no top damping).  x and y are horizontal.  w_z lives at (i, j, k+1/2), psi at the
 *    nodes (its half-point derivatives use the stencils of d_a u).
 *    - Device layout: 6 fields, each [nz][ny][pitch].
 *    - Compact host layout: each field [ez][ey][ex] with its own extents.
 *    - Leap-frog advances psi by the trapezoid rule, psi^{n+1} = psi^n + dt (u^n + u^{n+1})/2.
 *    - Supported: forward steps of every integrator and H x.  The transpose and the
 *      adjoint are not (UNSUPPORTED).
 */
#ifndef EWAVE_H
#define EWAVE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------------------ */
#define EWV_OK 0
#define EWV_ERR_INVALID_ARG -1
#define EWV_ERR_BAD_SIZE_OR_ALIGNMENT -2
#define EWV_ERR_WORKSPACE_TOO_SMALL -3
#define EWV_ERR_CUDA -4
#define EWV_ERR_NONFINITE -5
#define EWV_ERR_TIMEOUT -6
#define EWV_ERR_UNSUPPORTED -7
#define EWV_ERR_NOT_BOUND -8

/* ---- enums ------------------------------------------------------------------------- */
#define EWV_F32 0
#define EWV_F64 1

#define EWV_METHOD_APPLY 0    /* plain H x (no integrator)                               */
#define EWV_METHOD_FABER 1    /* Sec. 3.2 Faber three-term recurrence                    */
#define EWV_METHOD_KRYLOV 2   /* Sec. 3.2 Arnoldi (modified Gram-Schmidt) + Pade exp     */
#define EWV_METHOD_HORK 3     /* Sec. 3.2 high-order (SSP) Runge-Kutta                   */
#define EWV_METHOD_RK32 4     /* Sec. 3.1 RK3-2                                          */
#define EWV_METHOD_RK44 5     /* Sec. 3.1 classical RK4-4                                */
#define EWV_METHOD_LEAPFROG 6 /* Sec. 3.1 two-step leap-frog                             */
#define EWV_METHOD_ADJOINT_FABER 7 /* discrete adjoint of the Faber step (workspace query) */
#define EWV_METHOD_ADJOINT_KRYLOV 8 /* linearised adjoint of the Krylov step (workspace query) */
#define EWV_METHOD_ADJOINT_LEAPFROG 9 /* discrete adjoint of the leap-frog step (workspace query) */
#define EWV_METHOD_KRYLOV_ADAPTIVE 10 /* adaptive Krylov step (workspace query, m = m_max)      */

#define EWV_LEAPFROG_AVERAGED 0 /* time-averaged PML damping of w (stable reading)       */
#define EWV_LEAPFROG_LITERAL 1  /* explicit -beta w^n damping, as the formula reads      */
/* The averaged scheme with u advanced in difference form: d^{n+1} = u^{n+1} - u^n follows
 * from d^n, and u^{n+1} = u^n + d^{n+1} (the same scheme in exact arithmetic).  2u^n - u^{n-1}
 * is never formed, so FP32 rounding no longer acts as a velocity error every step.  d is
 * kept in the v field (2D only; the v field then holds no velocity).  Switching to or from
 * this form restarts the history (u^{-1} = u^0). */
#define EWV_LEAPFROG_DIFFERENCE 2

/* Largest Krylov dimension and Faber degree the library accepts. */
#define EWV_MAX_KRYLOV_M 48
#define EWV_MAX_FABER_DEGREE 128
#define EWV_MAX_TAIL_P 24

/* ---- model description ------------------------------------------------------------- */
typedef struct ewv_model_desc {
    int dims;            /* 2 (the paper's case) or 3 (the extension above)               */
    int nx, ny;          /* grid nodes; 2 <= nx, ny <= 2^30                               */
    double dx;           /* grid spacing (m), dx = dy (Sec. 2.1)                          */
    int fd_order;        /* 8 (paper, Sec. 2.1) or 4 (no free surface only)               */
    int pml_width;       /* PML thickness delta in grid points (0 = no damping)           */
    double beta0;        /* damping magnitude beta0 of Sec. 2's profile (1/s)             */
    int free_surface;    /* 1: Sec. 2.2 free surface on top; 0: PML + zero extension      */
    int precision;       /* EWV_F32 or EWV_F64                                            */
    int nshots;          /* independent shots (states) sharing this velocity model        */
    int src_taylor_p;    /* p of the augmented matrix H~ (Eq. matrix_ampli), 1..24        */
    int max_receivers;   /* receivers per shot (seismogram row width)                     */
    int nz;              /* dims = 3: node planes along z (2..2^30); ignored for dims = 2 */
} ewv_model_desc;

typedef struct ewv_layout_info {
    int pitch;                 /* elements per padded row (multiple of 128 bytes)          */
    int elem_bytes;            /* 4 or 8                                                   */
    size_t field_elems;        /* ny * pitch (2D); nz * ny * pitch (3D)                    */
    size_t vector_bytes;       /* fields (4; 6 in 3D) * field_elems * elem_bytes           */
    size_t state_bytes;        /* nshots * vector_bytes                                    */
    size_t params_bytes;       /* c^2 on the padded grid: field_elems * elem_bytes         */
    size_t compact_n;          /* length of the compact host state vector                  */
} ewv_layout_info;

typedef struct ewv_model* ewv_model_t;
typedef struct ewv_batch* ewv_batch_t;

/* ---- lifetime and binding ---------------------------------------------------------- */

/* Create a model from desc (copied).  Uses the current CUDA device.  Errors:
 * INVALID_ARG (a field out of range, e.g. p, or a padded grid nz * ny * pitch above
 * 2^31 - 1 elements: receiver offsets are 32-bit), checked before any CUDA call;
 * UNSUPPORTED (a free surface with fd_order 4); CUDA (allocation failed). */
int ewv_create_model(const ewv_model_desc* desc, ewv_model_t* out);
int ewv_destroy_model(ewv_model_t model);

/* Stream (a cudaStream_t, e.g. torch.cuda.current_stream().cuda_stream) for all work. */
int ewv_set_stream(ewv_model_t model, void* cuda_stream);

/* Padded layout and buffer sizes of this model. */
int ewv_layout(ewv_model_t model, ewv_layout_info* out);

/* Device workspace bytes that `method` needs at Krylov dimension / Faber degree / HORK
 * stages m (ignored by the others), for all shots. */
int ewv_workspace_bytes(ewv_model_t model, int method, int m, size_t* bytes);

/* Bind caller-owned device buffers.  state: state_bytes; params: params_bytes (c^2);
 * work: workspace (may be NULL with work_bytes 0 until a method needs it).  Binding zeroes
 * state and work on the stream.  Errors: BAD_SIZE_OR_ALIGNMENT. */
int ewv_bind_buffers(ewv_model_t model, void* state, size_t state_bytes, void* params,
                     size_t params_bytes, void* work, size_t work_bytes);

/* Rebind only the workspace (zeroed on the stream); state and params are left untouched. */
int ewv_bind_workspace(ewv_model_t model, void* work, size_t work_bytes);

/* Seismogram buffer: [nshots][capacity][max_receivers] of the model's precision.  Sample s
 * holds u at the receivers after the s-th step since the last ewv_reset_recording(). */
int ewv_bind_seismogram(ewv_model_t model, void* seismo, size_t bytes, int capacity);
int ewv_reset_recording(ewv_model_t model);

/* Zero every shot's state on the stream, forget the leap-frog history and rewind the
 * recording cursor (a fresh simulation from rest). */
int ewv_reset_state(ewv_model_t model);

/* ---- model inputs ------------------------------------------------------------------ */

/* Velocity c (m/s) at the nodes, host float64 [ny][nx] (count = nx*ny; 3D: [nz][ny][nx],
 * count = nx*ny*nz); stores c^2 in the params buffer and records c_max (used by the Faber
 * ellipse).  Synchronous. */
int ewv_set_velocity(ewv_model_t model, const double* c_host, size_t count);

/* Ricker source of shot `shot` at (sx, depth sy) metres, peak frequency f_peak, delay t0,
 * amplitude amp: f = amp r(t)/dx^2 added to the v-row at the nearest node (index
 * floor(pos/dx + 1/2), Sec. 4.1's Ricker wavelet).  Receivers: nrec (x, depth) pairs in
 * rxy (metres).  The node indices are echoed (src_idx_out[2] = {i, j}; rec_idx_out[2*nrec])
 * when the pointers are non-NULL.  Errors: INVALID_ARG for positions off the grid or
 * nrec > max_receivers. */
int ewv_set_source_receivers(ewv_model_t model, int shot, double sx, double sy, double f_peak,
                             double t0, double amp, int nrec, const double* rxy,
                             int32_t* src_idx_out, int32_t* rec_idx_out);

/* The same for a 3D model: source at (sx, sy, depth sz); receivers as nrec (x, y, depth)
 * triples in rxyz; echoed indices src_idx_out[3] = {i, j, k}, rec_idx_out[3*nrec].  The
 * 2D call on a 3D model (and this call on a 2D model) returns INVALID_ARG. */
int ewv_set_source_receivers3d(ewv_model_t model, int shot, double sx, double sy, double sz,
                               double f_peak, double t0, double amp, int nrec,
                               const double* rxyz, int32_t* src_idx_out, int32_t* rec_idx_out);

/* Override the Faber ellipse (gamma, c0, c1) of Sec. 3.2's recurrence.  By default it is
 * the ellipse centred at -dims beta0 / 2 with semi-axes sqrt(2) x (dims beta0 / 2) (real)
 * and sqrt(2) x omega (imaginary), omega = kappa c_max sqrt(dims |S2|) / dx, S2 the minimum
 * of the centred second-derivative symbol, kappa = 1.30 with a free surface, else 1.05. */
int ewv_set_faber_ellipse(ewv_model_t model, double gamma, double c0, double c1);
int ewv_get_faber_ellipse(ewv_model_t model, double* gamma, double* c0, double* c1);

/* ---- state transfer (synchronous) --------------------------------------------------- */

/* Compact float64 host state of one shot <-> the padded device state. */
int ewv_set_state(ewv_model_t model, int shot, const double* host, size_t n);
int ewv_get_state(ewv_model_t model, int shot, double* host, size_t n);
/* Compact host vector <-> one padded device vector at `dev` (vector_bytes). */
int ewv_pack_vector(ewv_model_t model, const double* host, size_t n, void* dev);
int ewv_unpack_vector(ewv_model_t model, const void* dev, double* host, size_t n);

/* Storage-precision experiment (the paper keeps every vector in its working precision; this
 * is the library's own probe of bfloat16 storage).  With EWV_STORE_BF16 every value that a
 * stencil pass stores (the integrator's Y and ACC vectors of Faber, HORK, RK3-2 and RK4-4
 * steps) is rounded to the nearest bfloat16 (ties to even) and kept in the FP32 buffer, so
 * the arithmetic sees exactly what a bfloat16 store and load would give.  The FP32 plain
 * stencil kernel serves these passes (the TMA pipeline is not used), so the experiment
 * measures accuracy, not speed.  Krylov's final combination and the leap-frog step are not
 * rounded.  2D FP32 models only (UNSUPPORTED otherwise). */
#define EWV_STORE_FP32 0
#define EWV_STORE_BF16 1
int ewv_set_storage_rounding(ewv_model_t model, int mode);

/* ---- operator (Eq. 1, Secs. 2.1-2.2) ------------------------------------------------- */

/* y = H x (transpose = 0) or y = H^T x (transpose = 1) for padded device vectors x, y of
 * this model (no source term).  x and y must not overlap. */
int ewv_apply_operator(ewv_model_t model, int transpose, const void* x, void* y);

/* ---- time integrators: advance every shot by nsteps steps of dt from time t --------- */

/* Sec. 3.2 Faber: u^{n+1} = sum_{j=0}^{degree} a_j F_j(H~) [u^n; e_p]. */
int ewv_step_faber(ewv_model_t model, double t, double dt, int degree, int nsteps);

/* Sec. 3.2 Krylov: Arnoldi (MGS) on dt H~ with m matrix-vector products, exp of the m x m
 * Hessenberg by [13/13] Pade with scaling and squaring.  The start vector is [U^n; eta e_p]
 * with the source column scaled by 1/eta, eta = |U^n| (1 if U^n = 0), which leaves the
 * exponential unchanged and keeps the wavefield and the tail on one scale.  *info (may be NULL) receives the
 * smallest effective dimension over shots and steps (< m after a happy breakdown); with a
 * non-NULL info the call waits for the GPU to read it and returns EWV_ERR_NONFINITE itself
 * when the Arnoldi process met a non-finite value.  With info NULL it returns after
 * enqueueing, like the other step calls. */
int ewv_step_krylov(ewv_model_t model, double t, double dt, int m, int nsteps, int* info);

/* One ewv_step_krylov step (nsteps = 1, no info) that also writes the step's dense states
 *   x_q = [I 0] beta V_m exp(tau_q H_m) e_1 ~ [I 0] exp(tau_q dt H~) [U^n; e_p],  q = 0..3,
 * tau_q the 4-point Gauss-Legendre nodes on [0, 1], from the step's own Arnoldi basis and
 * Hessenberg matrix (Sec. 3.2) into dense: 4 x nshots padded state vectors of the model's
 * precision, device memory, caller-owned, 256-B aligned, laid out [q][shot].  These are the
 * forward states the adjoint of the step's exponential integrates against (see
 * ewv_adjoint_step_krylov_dense): storing them trades 4 vectors per step of memory (Sec. 3.3,
 * N_mem) for the forward Arnoldi the adjoint would otherwise recompute.  The call runs
 * without step graphs.  Errors as ewv_step_krylov; BAD_SIZE_OR_ALIGNMENT for a misaligned
 * buffer. */
int ewv_step_krylov_dense(ewv_model_t model, double t, double dt, int m, void* dense);

/* Adaptive Krylov step (KIOPS-style; the paper names adaptive dimensions and substeps as the
 * improvement it leaves out, Secs. 3.2 and 6): advance every shot by nsteps steps of dt of
 * U^{n+1} = [I 0] exp(dt H~) [U^n; eta e_p] (the balanced start vector of ewv_step_krylov),
 * each step in substeps tau of the normalised step.  A substep grows its Arnoldi basis one
 * vector at a time from m_min to m_max and stops at the first dimension j whose estimate
 *   beta h_{j+1,j} (tau |[phi_1(tau H_j)]_{j,1}| + tau^2 |[phi_2(tau H_j)]_{j,1}| |A v_{j+1}|)
 * (the first two terms of Saad's error series; A v_{j+1} is the next column's product,
 * reused when the basis grows) is at most tol tau beta, beta the norm of the substep's
 * augmented start vector.  At m_max the substep shrinks tau on the same basis (no new
 * products); after a substep tau grows by at most 2x; a happy breakdown takes the rest of
 * the step at once.  phi_1, phi_2 and exp come from one exponential of the twice-bordered
 * Hessenberg matrix, in FP64 on the host, which reads the Krylov scalars after every basis
 * vector: the call waits for the GPU once per vector and launches directly (no graphs).
 * Every shot has its own dimensions and substeps.  The orthogonalisation window of
 * ewv_set_krylov_window applies.  stats (may be NULL) receives {substeps, matrix-vector
 * products, largest dimension} summed over shots and steps.  Workspace:
 * ewv_workspace_bytes(EWV_METHOD_KRYLOV_ADAPTIVE, m_max) (m_max + 1 vectors).  Errors:
 * INVALID_ARG (tol <= 0, 1 <= m_min <= m_max <= EWV_MAX_KRYLOV_M - 1 violated), NONFINITE
 * (also when a substep cannot meet tol at m_max after 60 shrinks). */
int ewv_step_krylov_adaptive(ewv_model_t model, double t, double dt, double tol, int m_min,
                             int m_max, int nsteps, int* stats);

/* Incomplete orthogonalisation for the Krylov step (the library's option; the paper names
 * incomplete or non-orthonormal bases as the way to cut the Arnoldi cost, Secs. 3.2 and 6):
 * with window q > 0 each new vector is orthogonalised, in modified Gram-Schmidt order, only
 * against the q most recent basis vectors, so the Hessenberg matrix is banded and a step
 * costs m + q m Gram-Schmidt passes instead of m (m + 1) / 2; the Arnoldi relation
 * A V_m = V_{m+1} H still holds, the basis is no longer orthonormal.  q = 0 (default): full
 * Gram-Schmidt.  A batch uses the window of its first model. */
int ewv_set_krylov_window(ewv_model_t model, int window);

/* Sec. 3.2 HORK (scheme EWV_METHOD_HORK, `stages` = m) or Sec. 3.1 RK3-2 / RK4-4
 * (EWV_METHOD_RK32 / EWV_METHOD_RK44; stages ignored). */
int ewv_step_rk(ewv_model_t model, double t, double dt, int scheme, int stages, int nsteps);

/* Evaluation order of HORK(m) (Sec. 3.2).  For the linear system one HORK step is the
 * degree-m Taylor polynomial of exp(dt H~) applied to [u^n; e_p]; both forms compute it with
 * m operator passes and agree up to rounding.
 *   EWV_HORK_LOW_STORAGE (default): the paper's low-storage stages k_i = (I + dt H~) k_{i-1}
 *     with the accumulator sum_i lambda_i k_i (17 FP32 words per grid point and pass).
 *   EWV_HORK_HORNER: V_j = V_0 + (dt/j) H~ V_{j+1}, j = m .. 1, V_{m+1} = V_0,
 *     u^{n+1} = V_1.  A pass reads V_{j+1}, V_0 and c^2 and writes V_j (13 words).  Rounding
 *     made in pass j reaches the result multiplied by (dt H~)^(j-1)/(j-1)!, so in FP32 at
 *     large steps (|dt lambda| near 10) it is less accurate than the low-storage form.
 * The setting drops the model's captured step graphs; a batch uses its first model's form.
 * Returns EWV_ERR_INVALID_ARG for an unknown form. */
#define EWV_HORK_HORNER 0
#define EWV_HORK_LOW_STORAGE 1
int ewv_set_hork_form(ewv_model_t model, int form);

/* Sec. 3.1 leap-frog.  The state's u, w_x, w_y hold time level n; the previous level lives
 * in the workspace and is initialised from the state on the first call after a state
 * change (u^{-1} = u^0, w^{-1} = w^0).  The v field is not advanced. */
int ewv_step_leapfrog(ewv_model_t model, double t, double dt, int nsteps);
int ewv_set_leapfrog_variant(ewv_model_t model, int variant);

/* ---- discrete adjoint: FWI gradient with respect to m = c^2 ------------------------------
 * Misfit J = 1/2 sum_n |R U^n - d^n|^2 over the recorded samples; U^n = Phi_n(U^{n-1}) is one
 * Faber step (Sec. 3.2).  The inverse problem stores one state per step (Secs. 3.3, 6:
 * N_mem = T/dt); these calls run the exact discrete adjoint of the recurrence.
 *
 * ewv_adjoint_step: for every shot, given the checkpoint U^{n-1} (nshots padded state
 * vectors) and the cotangent lambda = dJ/dU^n (nshots padded vectors, in/out), replaces
 * lambda by (dPhi_n/dU)^T lambda and accumulates grad += (dPhi_n/dm)^T lambda into grad
 * (nshots padded fields [ny][pitch] of the model's precision, one per shot; sum them for
 * the model gradient).  t = t_{n-1}, dt, m as in the forward ewv_step_faber call (same
 * ellipse).  method EWV_METHOD_FABER (reverse three-term recurrence) or EWV_METHOD_HORK
 * (m = stages; reverse of the (I + dt H~) chain): exact discrete adjoints, needing
 * ewv_workspace_bytes(EWV_METHOD_ADJOINT_FABER, m) of workspace (the step is recomputed
 * from the checkpoint: m tape vectors + 3 cotangents).  method EWV_METHOD_KRYLOV (m = Krylov
 * dimension, <= EWV_MAX_KRYLOV_M): the Krylov step depends nonlinearly on U (its basis and
 * Hessenberg matrix do).  By default (EWV_KRYLOV_ADJOINT_EXACT) this is the exact discrete
 * adjoint of the computed step: the basis is recomputed from the checkpoint and the reverse
 * mode runs through the output combination, the Frechet derivative of exp(H_m) (FP64, on the
 * host: one stream synchronisation per call), every modified Gram-Schmidt update in reverse
 * order (the orthogonalisation window of ewv_set_krylov_window included) and the start
 * vector with its tail scaling eta = |U|.  With EWV_KRYLOV_ADJOINT_EXPONENTIAL
 * (ewv_set_krylov_adjoint) it is the adjoint of the step's exact exponential,
 * U^n = [I 0] exp(dt H~) [U^{n-1}; e_p]: lambda <- exp(dt H)^T lambda by Arnoldi on dt H^T
 * (m products), and grad += int_0^dt [exp((dt-s) H)^T lambda]_v (L u + D w)(s) ds by 4-point
 * Gauss-Legendre with dense output from the two bases; it agrees with the Krylov forward
 * only to that step's time accuracy.  Workspace: ewv_workspace_bytes(EWV_METHOD_ADJOINT_KRYLOV,
 * m) (2m + 9 vectors) for either.
 * method EWV_METHOD_LEAPFROG (m ignored; averaged damping of w, in the plain or the
 * difference form, which are one scheme): the exact discrete adjoint of one Sec. 3.1 step
 * z^{n-1} -> z^n, z = (u, u_prev, w, w_prev).  checkpoint: level n-1 in the u, w_x, w_y
 * fields (the state before the step); adj_state: 2 nshots padded vectors, the first nshots
 * holding the cotangents of (u, u_prev, w_x, w_y) of level n (u_prev in the v field), the
 * next nshots those of w_prev in their w fields; both are replaced by the cotangents of
 * level n-1.  One H^T pass and two pointwise passes; workspace
 * ewv_workspace_bytes(EWV_METHOD_ADJOINT_LEAPFROG, 0) (3 vectors).  UNSUPPORTED for the
 * literal damping variant.
 * 2D models only.  Buffers 256-B aligned, caller-owned.  In FP32 the stencil passes run on
 * the persistent TMA kernels (Faber, HORK, leap-frog: forward recompute, H^T and gradient;
 * Krylov's exponential form: both Arnoldi processes and the gradient), and the call then
 * synchronises the stream once to read their pipeline-timeout flag (EWV_ERR_TIMEOUT).
 *
 * ewv_adjoint_inject: lambda_u += R^T values at the receivers, values [nshots][max_receivers]
 * of the model's precision (the seismogram cotangent of one sample).
 *
 * ewv_checkpoint_stride: checkpoint every stride-th step so that at most `budget` states
 * are stored: stride = 1 if nsteps <= budget, else ceil(nsteps / budget); the states of a
 * segment are recomputed from its checkpoint during the backward pass. */
int ewv_adjoint_step(ewv_model_t model, int method, double t, double dt, int m,
                     const void* checkpoint, void* adj_state, void* grad);
#define EWV_KRYLOV_ADJOINT_EXACT 0        /* reverse mode through the computed Krylov step */
#define EWV_KRYLOV_ADJOINT_EXPONENTIAL 1  /* adjoint of exp(dt H~), the step's limit          */
int ewv_set_krylov_adjoint(ewv_model_t model, int mode);
/* The adjoint of one Krylov step's exponential (as EWV_KRYLOV_ADJOINT_EXPONENTIAL, whatever
 * mode ewv_set_krylov_adjoint holds) from the forward step's dense states instead of its
 * checkpoint: dense is the buffer ewv_step_krylov_dense wrote for that step (4 x nshots
 * padded vectors, [q][shot]); t, dt, m as in that call; adj_state and grad as in
 * ewv_adjoint_step.  Only the adjoint Arnoldi on dt H^T runs (m products, none of the forward
 * process).  Workspace: ewv_workspace_bytes(EWV_METHOD_ADJOINT_KRYLOV, m). */
int ewv_adjoint_step_krylov_dense(ewv_model_t model, double t, double dt, int m, const void* dense,
                                  void* adj_state, void* grad);
int ewv_adjoint_inject(ewv_model_t model, void* adj_state, const void* values);
int ewv_checkpoint_stride(int nsteps, int budget, int* stride);
/* out[o] = sum over shots of per_shot[shot][o] (fields [ny][pitch]), shots summed in order:
 * the model gradient from the per-shot gradients of ewv_adjoint_step. */
int ewv_sum_shot_fields(ewv_model_t model, const void* per_shot, void* out);

/* ---- batches: many models (of uneven sizes) stepped together ----------------------- */

/* A batch steps every shot of every listed model in the same kernel launches (one tile
 * work list across all grids).  Models keep their own buffers; they must share the
 * precision, fd order and free-surface setting.  The batch uses the first model's stream
 * unless ewv_batch_set_stream is called. */
int ewv_create_batch(const ewv_model_t* models, int nmodels, ewv_batch_t* out);
int ewv_destroy_batch(ewv_batch_t batch);
int ewv_batch_set_stream(ewv_batch_t batch, void* cuda_stream);
int ewv_batch_step_faber(ewv_batch_t batch, double t, double dt, int degree, int nsteps);
int ewv_batch_step_krylov(ewv_batch_t batch, double t, double dt, int m, int nsteps,
                          int* info);
int ewv_batch_step_rk(ewv_batch_t batch, double t, double dt, int scheme, int stages,
                      int nsteps);
int ewv_batch_step_krylov_adaptive(ewv_batch_t batch, double t, double dt, double tol, int m_min,
                                   int m_max, int nsteps, int* stats);
int ewv_batch_step_leapfrog(ewv_batch_t batch, double t, double dt, int nsteps);

/* ---- allocation-free Faber step ------------------------------------------------------ */

/* The paper has no counterpart to this entry point; it serves callers that cannot call
 * cudaMalloc (code running inside someone else's memory pool, environments that forbid
 * run-time device allocation, or a process that must not grow the device heap while other
 * work holds the GPU).  It advances one FP32 state by nsteps Faber steps exactly like
 * ewv_step_faber, but needs no model handle and allocates nothing: the two Faber work
 * vectors and all per-step metadata live in one fixed file-scope device array of the
 * library (16 MB + 256 KB, held by every GPU that loads the library until the process
 * exits), so grids are limited to ny * pitch <= EWV_NOALLOC_MAX_FIELD_ELEMS.
 *  - state: padded FP32 state vector (4 fields of [ny][pitch], see the layout above),
 *    advanced in place; c2: c^2 on the padded grid; both 16-byte aligned, caller-owned.
 *  - args: grid, stencil, damping, optional source and the Faber ellipse (gamma, c0, c1).
 *  - stream: cudaStream_t (NULL = default stream).
 * Errors: INVALID_ARG for bad arguments, BAD_SIZE_OR_ALIGNMENT when ny * pitch exceeds
 * EWV_NOALLOC_MAX_FIELD_ELEMS (nothing is launched) or a pointer is misaligned, CUDA.
 * The first call on each device (with that device current) looks up the array's device
 * address; make that first call before any stream capture.  Calls share the array:
 * calls whose GPU work overlaps race.  The call reads the Faber coefficients back from the
 * GPU once, so it synchronises the stream before launching the steps.  Unlike the handle
 * calls it does not scan the state for non-finite values: check the state if that matters. */
#define EWV_NOALLOC_MAX_FIELD_ELEMS (1 << 19)
typedef struct ewv_noalloc_faber_args {
    int nx, ny, pitch;     /* grid nodes; pitch: elements per row, >= nx, multiple of 32 */
    double dx;
    int fd_order;          /* 8 or 4 (4 without free surface)                            */
    int pml_width;
    double beta0;
    int free_surface;
    int has_source;        /* 0: no source term                                         */
    int src_i, src_j;      /* source node                                                */
    int src_taylor_p;      /* p of the augmented block, 1..24                            */
    double f_peak, t0, amp;
    double gamma, c0, c1;  /* Faber ellipse                                              */
} ewv_noalloc_faber_args;
int ewv_faber_step_noalloc(const ewv_noalloc_faber_args* args, float* state, const float* c2,
                           double t, double dt, int degree, int nsteps, void* stream);

/* ---- diagnostics -------------------------------------------------------------------- */

/* Last error message on this handle ("" if none); valid until the next call on it. */
const char* ewv_last_error(ewv_model_t model);
const char* ewv_batch_last_error(ewv_batch_t batch);
/* Library version string. */
const char* ewv_version(void);
/* CUDA graphs (default on): a step call launches its first step directly, captures the
 * launch sequence of one step into a CUDA graph (once per method, m, dt and Faber ellipse)
 * and replays it for the remaining steps; steps read their time from a device-side clock,
 * so the graph has no per-step parameters.  Off: every kernel is launched directly.
 * With kernel timing enabled, the captured step carries its own event pairs and every
 * replay waits on the host for them (one wait per step). */
int ewv_enable_graphs(ewv_model_t model, int enable);
int ewv_batch_enable_graphs(ewv_batch_t batch, int enable);

/* Tile-shape autotuner of the FP32 persistent TMA pass.  Variants (tile height, consumer
 * warps, pipeline stages): 0 = (16, 16, 3), 1 = (16, 8, 3), 2 = (8, 8, 5), 3 = (8, 16, 5),
 * 5 = (20, 20, 3), 6 = (18, 18, 3), each consumer thread on one column; 7 = (18, 9, 3),
 * 8 = (16, 8, 3), 9 = (18, 18, 3), 10 = (24, 12, 2), each consumer thread on two adjacent
 * columns (8-byte shared loads, packed FP32 pair arithmetic); 11 = (24, 12, 3),
 * 12 = (36, 9, 2), 13 = (28, 14, 3) and 14 = (30, 15, 3) are composite: passes without an A
 * operand (Horner HORK passes, Krylov products) run these column-pair shapes without the A
 * stage buffer, passes with one run
 * variant 7 (the reported shape is the no-A one).  The autotuner's score is the sum of a
 * probe pass with and one without an A operand.  The leap-frog step and the FWI gradient
 * pass always run the column-pair form on 64 x 30 tiles with 15 warps, the transposed pass
 * on 64 x 18 tiles with 9 warps;
 * tiles are 64 columns wide with a 4-column / R-row halo.  With v = -1 (default) the first
 * FP32 step call times every variant on the probe passes over the engine's own problems and
 * keeps the fastest; ewv_*kernel_variant reports the choice, its shape and the probe times
 * (us[EWV_NUM_KERNEL_VARIANTS], -1 where a variant could not launch).  Variant 4 = (16, 16,
 * 4) without the U stage buffer: passes that read a U vector run variant 0 under it.
 * 3D models: 0 (default) = TMA pipeline with 16 consumer warps, 2 = 8 warps, 1 = plain
 * z-marching kernel. */
#define EWV_NUM_KERNEL_VARIANTS 15
int ewv_set_kernel_variant(ewv_model_t model, int variant);
int ewv_kernel_variant(ewv_model_t model, int* variant, int* tile_height, int* warps,
                       int* stages, double* probe_us);
int ewv_batch_set_kernel_variant(ewv_batch_t batch, int variant);
int ewv_batch_kernel_variant(ewv_batch_t batch, int* variant, int* tile_height, int* warps,
                             int* stages, double* probe_us);

/* Event timing of the fused stencil passes (the hot kernel): when enabled, every stencil
 * pass launch (each integrator pass and each leap-frog step, inside captured step graphs
 * too) is bracketed by a pair of CUDA events on the stream the pass runs on.
 * ewv_*kernel_timing synchronises the stream, returns the summed device time (ms) and the
 * number of timed launches since the last read, and resets both. */
int ewv_enable_kernel_timing(ewv_model_t model, int enable);
int ewv_kernel_timing(ewv_model_t model, double* total_ms, long long* launches);
int ewv_batch_enable_kernel_timing(ewv_batch_t batch, int enable);
int ewv_batch_kernel_timing(ewv_batch_t batch, double* total_ms, long long* launches);

/* Number of kernel launches this handle has enqueued since creation (for reporting). */
int ewv_launch_count(ewv_model_t model, long long* count);

/* Wait until every call enqueued on the handle has finished on the GPU, then report (and
 * clear) its asynchronous error word: EWV_OK, EWV_ERR_NONFINITE or EWV_ERR_TIMEOUT. */
int ewv_sync(ewv_model_t model);
int ewv_batch_sync(ewv_batch_t batch);

/* Testing aid: the limit, in ns (at most 1e9, the default), after which a pipeline wait of
 * the 2D FP32 TMA pass, or a grid-barrier wait of the Gram-Schmidt column kernel, on the
 * current device gives up.  The TMA kernel then waits (up to 1 s) for its copies in flight;
 * either sets the timeout bit of the error word and returns, so that a test can check the
 * EWV_ERR_TIMEOUT path on a healthy GPU with a limit a normal pass outruns (e.g. 0).  Waits
 * for the device to be idle first; applies to later launches, graph replays included.
 * Restore 1000000000 afterwards.  INVALID_ARG above 1e9. */
int ewv_debug_set_wait_limit(unsigned long long ns);

/* Testing aid: whether Krylov steps (and the exponential Krylov adjoint) run each Arnoldi
 * column's modified Gram-Schmidt steps on the column kernel -- one cooperative launch per
 * column with q_{j+1} in shared memory and a bounded grid barrier per step, taken when every
 * flat chunk of the engine fits one co-resident grid -- (1, the default) or on one flat
 * pass per step (0).  In FP32 both give the same values bit for bit; in FP64 the flat form
 * fuses the first dot of a column into the stencil pass, so they agree to rounding.
 * Process-wide; waits for the device to be idle first. */
int ewv_debug_set_column_kernel(int enable);

#ifdef __cplusplus
}
#endif
#endif /* EWAVE_H */
