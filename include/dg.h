/*
 * dg.h -- C ABI of the GB300 DGSEM operator library (libdg_gb300.so).
 *
 * The library evaluates the semi-discrete time derivative Ut = DG_Operator(U)
 * of the 3D compressible Navier-Stokes equations with the split-form
 * discontinuous Galerkin spectral element method on Legendre-Gauss-Lobatto
 * nodes (paper Sec. 2.2 "split-form DG scheme"; Sec. 4 "split DGSE
 * formulation"), and advances it with the five-stage fourth-order low-storage
 * Runge-Kutta scheme (paper Sec. 4).  The operator is:
 *   - BR1 lifting of the primitive gradients grad(u, v, w, T);
 *   - the kinetic-energy-preserving two-point volume flux differencing on
 *     curvilinear hexahedra (curl-form metrics);
 *   - the Riemann (central / local Lax-Friedrichs / Roe with Harten's entropy
 *     fix, Sec. 4) and BR1 viscous surface fluxes, with the equilibrium
 *     wall-stress model on slip walls (Sec. 3.1-3.2, Algorithms 1-2:
 *     Van Driest transform, Spalding or Reichardt law, Newton solve);
 *   - the surface integral, the 1/J scaling and a constant body force.
 *
 * Conventions shared by every entry point
 *   - Return value: 0 (DG_OK) or a negative DG_ERR_* code; the message of the
 *     last error of a context is returned by dg_last_error().
 *   - Field layout ("SoA"): double U[5][K][n^3], n = N + 1, variable v in
 *     (rho, rho u, rho v, rho w, E), node p = i + n (j + n k) of element e.
 *   - Ownership: the context owns all device storage (mesh, metrics, state,
 *     scratch).  Caller pointers are borrowed for the duration of the call
 *     only.  "on_device" arguments say whether a caller pointer is a device
 *     pointer (1) or a host pointer (0); host pointers may be pageable or
 *     pinned.
 *   - Stream: every device operation of a context is enqueued on the stream
 *     given to dg_init_mesh / dg_set_stream (a cudaStream_t, 0 = legacy
 *     default stream).  Calls that return results to the host synchronise
 *     that stream; the others are asynchronous.  With dg_set_overlap the
 *     wall-model kernel may run on a side stream that forks from and joins
 *     back into that stream within each call, so the ordering seen by the
 *     caller is that of the one stream.
 *   - Errors never trap or hang the GPU: device-side failures (non-finite
 *     state, wall-model Newton without convergence) set flags that the host
 *     reads with dg_check_status().
 */
#ifndef DG_GB300_H
#define DG_GB300_H

#ifdef __cplusplus
extern "C" {
#endif

enum dg_status_code {
  DG_OK = 0,
  DG_ERR_ARG = -1,             /* invalid argument (null pointer, bad enum, bad size) */
  DG_ERR_NOT_INIT = -2,        /* state not set before use */
  DG_ERR_MESH = -3,            /* non-positive Jacobian, non-matching faces, bad neighbour */
  DG_ERR_CUDA = -4,            /* CUDA runtime error (message has the CUDA error string) */
  DG_ERR_NONFINITE = -5,       /* a non-finite value appeared in the state */
  DG_ERR_WM_NOCONV = -6,       /* wall-model Newton iteration did not converge */
  DG_ERR_DEVICE_BOUNDS = -7,   /* device index check failed (debug builds) */
  DG_ERR_NOT_IMPLEMENTED = -8, /* option combination not available */
  DG_ERR_OOM = -9              /* device allocation failed */
};

enum dg_precision { DG_FP64 = 0, DG_FP32_MIXED = 1 };
/* Volume two-point fluxes: the kinetic-energy-preserving split forms of
 * Pirozzoli and of Kennedy-Gruber (Sec. 2.2), and Chandrashekar's entropy-
 * conserving and kinetic-energy-preserving flux (Sec. 4, the production
 * scheme).  The central surface flux uses the same two-point flux. */
enum dg_vol_flux { DG_VOL_KEP_PIROZZOLI = 0, DG_VOL_KEP_KENNEDY_GRUBER = 1, DG_VOL_EC_CHANDRASHEKAR = 2 };
enum dg_surf_flux { DG_SURF_CENTRAL = 0, DG_SURF_LLF = 1, DG_SURF_ROE = 2 };
enum dg_wall_law { DG_LAW_SPALDING = 0, DG_LAW_REICHARDT = 1 };

/* Neighbour codes of boundary faces in dg_mesh_desc.nbr.
 *   DG_BC_WALL     slip wall with the equilibrium wall model (Sec. 3.2);
 *   DG_BC_INFLOW   Dirichlet inflow: the exterior state is dg_phys.U_in;
 *   DG_BC_OUTFLOW  subsonic pressure outflow: the exterior state has the
 *                  interior density and velocity and pressure dg_phys.p_out
 *                  (the cascade boundaries of Sec. 4).
 * At inflow and outflow faces the inviscid flux is the selected Riemann
 * solver between the interior trace and the exterior state, the BR1 lifting
 * averages with the exterior state, and the viscous flux is the interior one. */
#define DG_BC_WALL (-1)
#define DG_BC_INFLOW (-2)
#define DG_BC_OUTFLOW (-3)
/* Halo face h of a partitioned mesh (the neighbour lives on another rank):
 * neighbour code DG_BC_HALO_BASE - h, h = 0 .. n_halo-1, each once.  See the
 * partitioning section below. */
#define DG_BC_HALO_BASE (-16)

typedef struct dg_ctx dg_ctx;

/* Mesh of K conforming hexahedra of degree N (paper Sec. 2.2: tensor-product
 * LGL nodes; the unstructured meshes of Sec. 4 and the space-filling-curve
 * subdomains of Sec. 2.1).
 *   X        host, double[3][K][n^3]: node coordinates at the LGL nodes
 *            returned by dg_lgl_nodes (degree-N geometry).
 *   nbr      host, int[K][6]: neighbour across local face l (0 -xi, 1 +xi,
 *            2 -eta, 3 +eta, 4 -zeta, 5 +zeta), or a negative boundary code
 *            (DG_BC_WALL, DG_BC_INFLOW, DG_BC_OUTFLOW, halo codes).
 *   nbr_face host, int[K][6] or NULL: the neighbour's local face that face l
 *            is joined to (NULL: l ^ 1 everywhere, the structured case).
 *   orient   host, int[K][6] or NULL (all 0): orientation code o in 0..7 of
 *            the joined faces.  Face-local node coordinates (a, b) in 0..N
 *            are (j, k) on the xi faces, (i, k) on the eta faces and (i, j) on
 *            the zeta faces; node (a, b) of face l of e coincides with node
 *            (a', b') of face nbr_face[e][l] of nbr[e][l], where
 *              (s, t) = (o & 1) ? (b, a) : (a, b),
 *              a' = (o & 2) ? N - s : s,   b' = (o & 4) ? N - t : t.
 *            The neighbour must list e back with the inverse code (o with
 *            the bits 2 and 4 exchanged when bit 1 is set, else o itself).
 *            On the local mesh of a partition (dg_partition_local) a halo
 *            face's code carries 8 when the local element is the face's
 *            master.
 * The joined faces must coincide node by node up to one translation
 * (periodic images), else DG_ERR_MESH.  Each interior face is evaluated once,
 * from its master side (the side with the odd local face when the two local
 * faces differ in parity, else the side with the smaller (element, face)
 * pair), whose metrics give the face normal.  All arrays are copied during
 * dg_init_mesh. */
typedef struct {
  int N;
  int K;
  const double* X;
  const int* nbr;
  const int* nbr_face;
  const int* orient;
} dg_mesh_desc;

/* Ideal gas and wall-model constants (paper Sec. 4: ideal gas with
 * Sutherland's law; Sec. 3.2: law of the wall).  mu is the viscosity:
 * constant when suth_S <= 0, else the reference value of Sutherland's law
 * mu(T) = mu (T / T_ref)^(3/2) (T_ref + suth_S) / (T + suth_S) (T_ref > 0
 * required), which then also sets the conductivity mu(T) cp / Pr and the
 * wall-model viscosity at the wall temperature; kappa and B are the law's constants;
 * hwm the sampling distance of the wall model; force a constant body force
 * per unit volume entering momentum (and its work f.u the energy).
 * p_ref: a constant subtracted from the pressure inside the momentum fluxes.
 * A constant pressure integrates to zero over every element (discrete
 * metric identities of the curl-form metrics), so the operator is unchanged
 * in exact arithmetic; setting p_ref to the ambient pressure removes the
 * cancellation of O(p_ref) terms at low Mach number (0 disables it). */
typedef struct {
  double gamma, R, mu, Pr;
  double force[3];
  double kappa, B, hwm;
  int law; /* dg_wall_law */
  double p_ref;
  double suth_S, T_ref; /* Sutherland's law (suth_S <= 0: constant mu) */
  double U_in[5];       /* inflow state (conservative), used by DG_BC_INFLOW faces */
  double p_out;         /* outflow pressure, used by DG_BC_OUTFLOW faces */
  double T_wall;        /* > 0: isothermal wall-modelled walls at this temperature
                           (Crocco-Busemann in the Van Driest transform, wall heat
                           flux q_w = -(cp/Pr) tau_w (T_aw - T_w) / u_s into the
                           energy equation); <= 0: adiabatic walls */
  double rho_ref;       /* FP32-mixed form only (>= 0; 0 disables): its FP32
                           primitives hold rho - rho_ref and h - h_ref,
                           h_ref = gamma p_ref / ((gamma - 1) rho_ref), formed
                           from the FP64 state, so that the differences of
                           neighbouring nodes in its flux-difference form carry
                           the FP32 rounding of the deviations from the reference
                           state instead of that of the values (the reference
                           density of the flow, e.g. 1 in units of rho0) */
} dg_phys;

typedef struct {
  int precision; /* dg_precision */
  int vol_flux;  /* dg_vol_flux */
  int surf_flux; /* dg_surf_flux */
  int viscous;   /* 1: Navier-Stokes (lifting + viscous fluxes), 0: Euler */
} dg_options;

/* LGL nodes xi[n] and weights w[n] on [-1, 1] (host arrays of N + 1 doubles).
 * 1 <= N <= 8. */
int dg_lgl_nodes(int N, double* xi, double* w);

/* Builds the geometry (curl-form metrics, Jacobians, face normals, wall-model
 * sampling points) on the host, validates it, allocates the device storage
 * and uploads it.  stream: cudaStream_t (may be 0).  On success *out owns
 * everything; free it with dg_destroy.  Device storage at N = 7: about 500
 * bytes per DOF in the FP64 viscous form (state, RK register, metrics and the
 * stored products Ja / J and (Ja Ja^T) / J, the stored primitives, scratch),
 * about 280 in the FP32-mixed form.  Errors: DG_ERR_ARG, DG_ERR_MESH,
 * DG_ERR_OOM, DG_ERR_CUDA (the message is then available through
 * dg_last_error(NULL)). */
int dg_init_mesh(dg_ctx** out, const dg_mesh_desc* m, const dg_phys* p, const dg_options* o,
                 void* stream);
int dg_destroy(dg_ctx* c);

/* Last error message of c (or of the last failed dg_init_mesh if c is NULL). */
const char* dg_last_error(const dg_ctx* c);

int dg_set_stream(dg_ctx* c, void* stream);

/* Meshes with wall-modelled walls: enable = 1 (the default) runs the
 * wall-model kernel (which reads only the state and writes only the wall
 * faces' fluxes) on a side stream of the highest priority, beside the lifting
 * and the interior-face kernels, rejoining the caller's stream before the
 * volume kernel (the prioritised streams and events of the paper's Sec. 2.1).
 * enable = 0 launches it in line on the caller's stream.  Results are bitwise
 * the same either way; a CUDA graph captured by dg_rk_steps_graph records the
 * fork and join of the setting in force when it is captured. */
int dg_set_overlap(dg_ctx* c, int enable);

/* Sizes: number of elements, nodes per element and total doubles of U. */
int dg_sizes(const dg_ctx* c, int* N, int* K, long long* n_state);

/* Copies U (5 K n^3 doubles) into / out of the context's state.
 * dg_set_state also clears the wall model's warm starts: each wall node's
 * law-of-the-wall solve starts from its previous solution (a few Newton steps,
 * the bracketed solve from scratch if they do not converge, Sec. 3.2 Alg. 1),
 * so results depend on the evaluations since the last dg_set_state, to the
 * solve's stopping tolerance (a Newton step below 1e-12 of max(1, |ln w|)). */
int dg_set_state(dg_ctx* c, const double* U, int on_device);
int dg_get_state(dg_ctx* c, double* U, int on_device);

/* Ut = DG_Operator(U) at time t (paper Sec. 2.2 / Sec. 4).  U: caller
 * array, or NULL for the context's state.  Ut: caller array (5 K n^3).
 * Both on the device or both on the host as on_device says. */
int dg_time_derivative(dg_ctx* c, const double* U, double* Ut, double t, int on_device);

/* One LSERK4 stage s (0..4) of the context's state (Carpenter-Kennedy
 * five-stage fourth-order 2N-storage scheme, paper Sec. 4):
 *   dU = A_s dU + dt Ut(U, t + c_s dt);  U = U + B_s dU.
 * A_0 = 0, so a step (s = 0..4) needs no reset of dU.  The volume kernel
 * applies the update in registers, in place. */
int dg_rk_stage(dg_ctx* c, int s, double t, double dt);

/* nsteps full LSERK4 steps from time t. */
int dg_rk_steps(dg_ctx* c, double t, double dt, int nsteps);

/* Vector-Jacobian product of the operator (the hand-written adjoint):
 *   gU     = (dUt/dU)^T lam,
 *   gtheta = (dUt/d(kappa, B))^T lam  (wall-law constants; zero without walls).
 * U: device array or NULL for the context's state; lam, gU: device arrays
 * double[5][K][n^3]; gtheta: device double[2] or NULL.  The transposed
 * split-form volume integral, viscous flux, BR1 lifting and primitive
 * recovery are written out by hand, and so is the reverse mode of the
 * Riemann flux (one forward sweep keeping the intermediates of the two-point
 * flux and of its dissipation, one backward sweep); the local derivatives of
 * the wall model come from forward-mode dual numbers, with the implicit
 * function theorem for the law-of-the-wall solve (Sec. 3.2).  FP64
 * contexts with the Pirozzoli or the entropy-conserving volume flux (the
 * paper's Sec. 4 scheme, with Roe + Harten faces), constant viscosity or
 * Sutherland's law, adiabatic or isothermal walls (the wall heat flux's
 * derivative with the stress's), inflow and outflow faces (through the
 * exterior state's dependence on the interior one) (else
 * DG_ERR_NOT_IMPLEMENTED); partitioned contexts run it in phases
 * (dg_vjp_phase; dg_vjp answers DG_ERR_ARG there).
 * The first call allocates the adjoint scratch of the context. */
int dg_vjp(dg_ctx* c, const double* U, const double* lam, double* gU, double* gtheta);

/* The adjoint of a partitioned context (see the partitioned-mesh section
 * below), in four phases with an exchange of the halo buffers after each of
 * the first three (send_U -> recv_U, send_G -> recv_G, send_U -> recv_U), the
 * reverse of an evaluation's:
 *   phase 1  packs the state traces of the halo faces (send_U);
 *   phase 2  the face, wall-model and boundary kernels: the cotangents of
 *            the peers' viscous-flux traces into send_G and of their state
 *            traces into send_U (needs the peers' state traces in recv_U);
 *            zeroes gtheta first;
 *   phase 3  adds the peers' viscous-flux cotangents (recv_G) and runs the
 *            element kernel, which adds its lifting's share to send_U;
 *   phase 4  gU from the local cotangents and the peers' state cotangents
 *            (recv_U).
 * Arguments as dg_vjp (the same U, lam, gU and gtheta in every phase);
 * gtheta holds this rank's share of (dUt/d(kappa, B))^T lam, to be summed
 * over the ranks.  The sum over ranks of the gU rows equals dg_vjp on the
 * unpartitioned mesh to rounding.  DG_ERR_ARG on an unpartitioned context or
 * a phase outside 1..4; option checks as dg_vjp. */
int dg_vjp_phase(dg_ctx* c, int phase, const double* U, const double* lam, double* gU, double* gtheta);

/* Sets the wall-law constants (kappa, B) used by later calls (Sec. 3.2). */
int dg_set_params(dg_ctx* c, double kappa, double B);

/* Arithmetic of the FP64 viscous form's lifting kernel at odd N (BR1
 * lifting, viscous flux, weak viscous divergence): mode 1 double-float (the
 * default at odd N: each value an unevaluated sum of two floats, the
 * operations built from error-free transformations on the FP32 pipe, about
 * 2^-47 relative rounding per operation; the state, the primitives, the
 * metric data and the kernel's outputs stay FP64, the temperature is lifted
 * relative to p_ref / (rho_ref R); the viscous terms are a small part of Ut,
 * and the operator's parity with the oracle is unchanged), 0 FP64.  Mode 1
 * keeps (hi, lo) float pairs of the metric data and of the lifted
 * primitives: 224 more bytes per DOF.  Even degrees and other forms ignore it.
 * DG_ERR_ARG for another mode.  Used by later calls. */
int dg_set_lifting_arithmetic(dg_ctx* c, int mode);

/* Iteration cap of the wall model's law-of-the-wall solve (SolveWallStress,
 * Sec. 3.2 Algorithms 1-2): bracket growth and Newton steps together, at
 * most max_iter evaluations of the law per wall node (default 200; the
 * converged solve takes about eight).  A wall node whose solve reaches the
 * cap keeps its last iterate and sets the status flag that dg_check_status
 * reports as DG_ERR_WM_NOCONV; nothing waits or traps on the GPU.
 * max_iter >= 1, else DG_ERR_ARG.  Used by later calls. */
int dg_set_wall_solve_limit(dg_ctx* c, int max_iter);

/* Independent states from host memory through the LSERK4 stages, with the
 * host transfers overlapped with the computation (a serving-style batch):
 * for every item i < nitems, U_in[i] (host double[5][K][n^3]) is copied to
 * the device, stages 0 .. nstages-1 of one step of size dt run on it with
 * the item's own register dU (zero at the start, as at a step's start), and
 * the result is copied to U_out[i] (host).  Two device slots: the copy of
 * item i+1 in and of item i-1 out run on their own streams while item i
 * computes on the context's stream (2 x 2 x 5 K n^3 doubles, allocated at the
 * first call).  Results equal those of dg_set_state, the stages and
 * dg_get_state bitwise.  The context's own state and register are not
 * touched; wall-law solves start afresh for every item.  Host buffers should
 * be page-locked for the copies to overlap; U_out[i] must not alias a later
 * item's input.  Synchronises the stream.  1 <= nstages <= 5; unpartitioned
 * contexts only (else DG_ERR_ARG). */
int dg_rk_stage_batch(dg_ctx* c, int nitems, const double* const* U_in, double* const* U_out, int nstages,
                      double t, double dt);

/* Explicit time step dt = cfl * 2/(2N+1) * min_nodes J / sum_dir(|u . Ja^dir|
 * + c |Ja^dir|) (CFL-based step of the explicit LSERK4, paper Sec. 4 uses
 * CFL 0.9).  U: device array or NULL for the state; dt: host double.
 * Synchronises the stream. */
int dg_time_step(dg_ctx* c, const double* U, double cfl, double* dt);

/* Volume-averaged kinetic energy (1/|Omega|) sum_nodes w_i w_j w_k J rho|u|^2/2
 * (the Taylor-Green diagnostic).  U: device array or NULL for the state; ke:
 * host double.  Synchronises the stream. */
int dg_kinetic_energy(dg_ctx* c, const double* U, double* ke);

/* Mean wall shear: the surface-quadrature-weighted mean of tau_w t_x over
 * all wall-modelled faces (t: unit wall-parallel sample velocity).  U: device
 * array or NULL for the state; loss: host double.  Synchronises the stream.
 * DG_ERR_ARG without wall-modelled walls. */
int dg_wall_shear(dg_ctx* c, const double* U, double* loss);

/* The FP64 <-> FP32 conversions of the FP32-mixed kernels, built from the
 * bit patterns with integer operations (the conversion instructions issue to
 * GB300's FP64 pipe), for testing them: for i < n (device arrays)
 *   f[i]   = d[i] rounded to the nearest float, ties to even (signed zero
 *            below the FP32 normal range, infinity above it, NaN kept),
 *   rem[i] = d[i] - f[i] as a float, to 2^-46 |d[i]| (zero where that
 *            scale is below the FP32 normal range, and for non-finite d[i]),
 *   gd[i]  = g[i] widened exactly (FP32 subnormals give signed zero).
 * Runs on the current device and synchronises it.  DG_ERR_ARG for n < 0 or
 * null arrays, DG_ERR_CUDA on a launch failure. */
int dg_convert_fp32(long long n, const double* d, float* f, float* rem, const float* g, double* gd);

/* Rollout adjoint: runs nsteps LSERK4 steps of size dt from U0 (device),
 * keeping one checkpoint of U per step (A_0 = 0, so U alone restarts a
 * step; checkpoints take nsteps * 5 K n^3 doubles of device memory), takes
 * L = mean wall shear of the final state, then sweeps the steps backwards,
 * recomputing each step's five stage inputs from its checkpoint and applying
 * the transposed 2N-storage recurrence with dg_vjp per stage.  Returns L
 * (host double), gU0 = dL/dU0 (device array) and gtheta = dL/d(kappa, B)
 * (device double[2] or NULL).  The context's state is not touched.
 * FP64 contexts with wall-modelled walls and the options dg_vjp accepts. */
int dg_rollout_vjp(dg_ctx* c, const double* U0, int nsteps, double dt, double* loss, double* gU0,
                   double* gtheta);

/* As dg_rk_steps, but replays a CUDA graph of one full step (the fifteen
 * kernel launches of the five stages), captured on an internal stream at
 * the first call and again whenever dt changes; the replays run on the
 * context's stream.  Results are identical to dg_rk_steps.  Per-kernel
 * profiling does not see graph replays. */
int dg_rk_steps_graph(dg_ctx* c, double t, double dt, int nsteps);

/* Copies the LSERK4 register dU (5 K n^3 doubles) out of / into the context
 * (checkpoint and restart inside a step; between steps dU needs no saving
 * because A_0 = 0). */
int dg_get_rk_register(dg_ctx* c, double* dU, int on_device);
int dg_set_rk_register(dg_ctx* c, const double* dU, int on_device);

/* Reads and clears the device status flags.  Returns DG_OK,
 * DG_ERR_DEVICE_BOUNDS, DG_ERR_NONFINITE or DG_ERR_WM_NOCONV (in that order
 * of precedence; synchronises the stream).  DG_ERR_DEVICE_BOUNDS comes only
 * from the bounds-checking build of the library (libdg_gb300_debug.so,
 * compiled with DG_DEBUG_BOUNDS): there every index that a kernel gathers
 * through the mesh tables (neighbour and face elements, face ids, halo
 * indices, wall-model sample elements) is checked against its range, and an
 * out-of-range one sets the flag and is replaced by 0 instead of being used,
 * so the GPU never reads outside an array. */
int dg_check_status(dg_ctx* c);

/* ---------------------------------------------------------------------------
 * Partitioned meshes (Sec. 2.1: non-overlapping subdomains along a
 * space-filling curve, one per rank and GPU).  Host functions need no GPU.
 *
 * dg_partition_sfc: part[K] (host) <- the rank of every element: elements
 *   ordered by the Morton key of their node-average centroid in the mesh's
 *   bounding box (21 bits per axis), cut into nranks contiguous runs of
 *   floor(K / nranks) or one more elements.  1 <= nranks <= K.
 *   X: host double[3][K][n^3] as in dg_mesh_desc.
 * dg_partition_local: the local mesh of `rank`: K_local elements (its own,
 *   in ascending global order; l2g[K_local] their global ids), nbr_local
 *   [K_local][6] with local neighbours, the global boundary codes, and
 *   DG_BC_HALO_BASE - h for the h-th face shared with another rank;
 *   nbr_face_local and orient_local [K_local][6] (may be NULL) the neighbour
 *   faces and orientation codes of the local elements (from nbr_face and
 *   orient, which may be NULL for the structured case), with 8 added to the
 *   code of a halo face whose master is the local element.
 *   halo[n_halo][4] (peer rank, local element, local face, 1 if the local
 *   element is the face's master by the rule of dg_mesh_desc).  The halo
 *   faces are ordered by peer, then by (global master element, master face),
 *   so two ranks list the faces they share in the same order and their halo
 *   buffers line up.  Call once with NULL arrays to get K_local and n_halo,
 *   then with arrays of those sizes.
 *
 * A context built from a local mesh (dg_init_mesh with nbr_local,
 * nbr_face_local and orient_local) owns halo buffers: recv_U/send_U
 * double[n_halo][5][n^2] (state traces at the halo faces' nodes, in the
 * face-node order of the face's master, which both ranks know)
 * and recv_G/send_G [n_halo][4][n^2] in the flux type (float in the
 * FP32-mixed form): each side's outward viscous flux there.  The caller moves
 * send_* of one rank into recv_* of the peer (the rows of the faces they
 * share, in the same order) between the phases of an evaluation:
 *   phase 1  packs send_U;                 then exchange U traces,
 *   phase 2  lifting, packs send_G;        then exchange viscous traces,
 *   phase 4  face fluxes (a halo face's flux is evaluated by both ranks from
 *            the same master and slave data) and the volume kernel.
 * Before the first evaluation the slave side of each halo face must receive
 * the master's normals: dg_halo_geometry writes the context's halo-face
 * geometry [n_halo][4][n^2] (unit normal of the master, surface element) to a
 * host array; send it to the peer, whose dg_halo_set_geometry installs the
 * rows of the faces where its element is the slave.  The fused calls
 * (dg_time_derivative, dg_rk_stage, ...) refuse partitioned contexts with
 * DG_ERR_ARG (the adjoint: dg_vjp_phase; the rollout adjoint answers
 * DG_ERR_NOT_IMPLEMENTED).  Wall-model sample
 * points must lie in local elements (else dg_init_mesh fails, DG_ERR_MESH).
 * Results equal those of the unpartitioned mesh bitwise.
 * ------------------------------------------------------------------------- */
int dg_partition_sfc(int N, int K, const double* X, int nranks, int* part);
int dg_partition_local(int K, const int* nbr, const int* nbr_face, const int* orient, const int* part, int rank,
                       int* K_local, int* l2g, int* nbr_local, int* nbr_face_local, int* orient_local, int* n_halo,
                       int* halo);
int dg_halo_buffers(dg_ctx* c, int* n_halo, void** send_U, void** recv_U, void** send_G, void** recv_G);
int dg_halo_geometry(dg_ctx* c, double* fgeo);
int dg_halo_set_geometry(dg_ctx* c, const double* fgeo);
/* One LSERK4 stage s (0..4) of the context's state, in phases 1, 2, 4 (in
 * that order, halo exchanges between them). */
int dg_stage_phase(dg_ctx* c, int phase, int s, double t, double dt);
/* Ut = DG_Operator(U) in phases 1, 2, 4; U (device, or NULL for the
 * context's state) and Ut (device) must be the same in the three calls. */
int dg_time_derivative_phase(dg_ctx* c, int phase, const double* U, double* Ut);

/* Per-kernel timing with CUDA events on the context's stream (tracing).
 * dg_profile_enable(c, 1) records events around the lift, face, wall and
 * volume kernels of every subsequent operator evaluation (in the FP64
 * viscous form the lift window also holds the kernel that forms the input
 * state's primitives, when they are not already stored); dg_profile_read
 * synchronises the stream, returns the summed milliseconds ms[4] and the
 * launch counts launches[4] (order: lift, face, wall, volume) since the last
 * read, and resets them. */
int dg_profile_enable(dg_ctx* c, int enable);
int dg_profile_read(dg_ctx* c, double* ms, int* launches);

/* Size in bytes of the static scratch array of dg_time_derivative_noalloc. */
#define DG_NOALLOC_SCRATCH_BYTES (32u << 20)

/* Ut = DG_Operator(U) like dg_time_derivative with device pointers, but
 * without the context's scratch buffers: the intermediate arrays of the
 * kernels come from one static device array of DG_NOALLOC_SCRATCH_BYTES
 * (32 MiB), which every GPU that loads the library holds until the process
 * exits.  The call allocates nothing.  The paper has no counterpart.
 *
 * It is meant for host programs that own all device memory through their
 * own allocator and cannot let a library call cudaMalloc when it computes
 * (as the paper's Fortran core does for its HIP kernels), and for callers
 * that run many contexts but want one shared scratch area instead of one
 * per context.  The mesh arrays still come from the context, which
 * dg_init_mesh allocated during set-up.
 *   U, Ut  device pointers, double[5][K][n^3]; U is read, Ut written.
 *   Errors DG_ERR_ARG if the mesh needs more scratch than the static array
 *   holds (the viscous FP64 operator needs about 84 bytes per DOF at N = 5
 *   and 72 at N = 7, so about 4e5 DOF fit, e.g. the 221,184-DOF channel;
 *   the message gives the bytes needed) or if the current device is not
 *   the one the context was created on, DG_ERR_CUDA on a CUDA failure.
 * In the FP32-mixed form the call also rewrites the context's own FP32
 * primitive array (allocated by dg_init_mesh) with those of U.
 * The first call on a device looks up the array's device address (the host
 * symbol is only a stand-in) and caches it; make that first call before any
 * stream capture.  All calls share the array: calls whose kernels overlap on
 * the GPU (different streams, different host threads) race on it.  Every
 * scratch word is rewritten before it is read in each call, so nothing
 * carries over from the previous call. */
int dg_time_derivative_noalloc(dg_ctx* c, const double* U, double* Ut);

/* Host copies of the geometry (for checking): Ja[K][n^3][3 dir][3 comp],
 * J[K][n^3]. */
int dg_get_metrics(const dg_ctx* c, double* Ja, double* J);

#ifdef __cplusplus
}
#endif

#endif /* DG_GB300_H */
