/*
 * mm.h -- C ABI of the GB300 finite-difference LLG solver core (libmm).
 *
 * What is computed (arXiv 2406.16064, MicroMagnetic.jl):
 *   the Landau-Lifshitz-Gilbert right-hand side on a regular cell mesh,
 *   dm/dt = -g~ m x H - alpha g~ m x (m x H), g~ = gamma/(1+alpha^2)
 *   (Sec. "LLG equation", LL form), with the effective field (Eq. 1) the sum of
 *     exchange             Sec. "Exchange energy", Eq. 5 (6-neighbour stencil;
 *                          uniform A or cell-based A with harmonic-mean pairs)
 *     DMI                  Sec. "Dzyaloshinskii-Moriya Energy", Eq. 14 and its
 *                          unified form: interfacial, bulk or D_2d vectors,
 *                          uniform or cell-based D
 *     uniaxial / cubic     Sec. "Anisotropy"
 *     Zeeman               Sec. "Zeeman energy"
 *     demagnetising field  Sec. "Magnetostatic energy", Eqs. 6-8: the discrete
 *                          convolution with the Newell tensor, evaluated by
 *                          zero-padded FFTs;
 *   plus, optionally, the spin-transfer and spin-orbit torques of Sec. "Spin
 *   transfer torques" in the right-hand side; integrated with adaptive
 *   Dormand-Prince RK45 and projection onto |m| = 1 after every accepted step
 *   (Sec. "LLG equation") or fixed-step RK4 with projection or on the Cayley
 *   variable (Sec. "Cayley transform"), minimised by steepest descent (Sec.
 *   "Steepest descent energy minimization"), and the nudged elastic band of
 *   Sec. "Miscellaneous".
 *
 * Conventions
 *   Units are SI: lengths m, fields A/m, Ms A/m, A J/m, D J/m^2, K J/m^3,
 *   gamma m/(A s), time s, energy J.  mu0 = 4e-7*pi.
 *   A magnetisation state of one simulation is structure-of-arrays
 *   m[c][z][y][x] (c = x,y,z; x fastest): 3*nx*ny*nz numbers.  A batch state
 *   is the concatenation of its simulations' blocks in the order they were
 *   added (mm_batch_layout gives the offsets).  Device buffers have the
 *   context's precision (double for MM_F64, float for MM_F32); host buffers
 *   are always double.
 *   Boundaries are free: a neighbour outside the mesh or with Ms = 0 is
 *   dropped from the exchange and DMI sums; cells with Ms = 0 have no field
 *   and no torque.
 *
 * Ownership and errors
 *   The library owns every device buffer it allocates; the *_dev arguments
 *   are caller-owned device pointers (for example a torch tensor's
 *   data_ptr()), contiguous, read or written on the context stream.  Host
 *   pointers are read or written before the call returns.
 *   Every call returns MM_OK (0) or a negative status; mm_last_error gives a
 *   message.  No call falls back to the CPU; without a usable GPU mm_create
 *   fails with MM_ECUDA.
 */
#ifndef MM_H
#define MM_H

#ifdef __cplusplus
extern "C" {
#endif

enum {
    MM_OK = 0,
    MM_EINVAL = -1,     /* bad argument or call order */
    MM_ENOMEM = -2,     /* device allocation failed */
    MM_ECUDA = -3,      /* CUDA runtime error */
    MM_ENAN = -4,       /* non-finite error norm in a step */
    MM_ESTEP = -5,      /* step size underflow */
    MM_ETIMEOUT = -6,   /* a bounded device wait ran out */
    MM_EBOUNDS = -7     /* a work item or block offset of the plan would leave its buffer
                           (checked on the host before the first launch) */
};

/* Context precision.  MM_F64: FP64 state, stage vectors, fields and
 * reductions; the FFT transforms, the tensor product and the z convolution
 * compute in double-float arithmetic (an FP32 pair hi + lo, about 48
 * significant bits) on the FP32 pipe, since GB300's FP64 rate is a small
 * fraction of its FP32 rate; fields agree with native FP64 to ~1e-14.
 * MM_F32: FP32 state and arithmetic with FP64-accurate norms, error norm and
 * energies.  MM_F64_NATIVE: FP64 arithmetic in every kernel. */
enum { MM_F64 = 0, MM_F32 = 1, MM_F64_NATIVE = 2 };
enum { MM_HOST = 0, MM_DEVICE = 1 };      /* where a buffer lives */
/* DMI symmetry class (Sec. "Dzyaloshinskii-Moriya Energy"): DMI vectors e_ij
 * for the neighbours (-x, +x, -y, +y, -z, +z): interfacial (C_nv)
 * (-e_y, e_y, e_x, -e_x, 0, 0); bulk (T, O) r_ij = (-e_x, e_x, -e_y, e_y, -e_z,
 * e_z); D_2d (e_x, -e_x, -e_y, e_y, 0, 0). */
enum { MM_DMI_NONE = 0, MM_DMI_INTERFACIAL = 1, MM_DMI_BULK = 2, MM_DMI_D2D = 3 };

typedef struct mm_ctx mm_ctx;             /* opaque */

/* Regular mesh of nx*ny*nz cells of size dx*dy*dz (FDMesh, Sec. "Design"). */
typedef struct { int nx, ny, nz; double dx, dy, dz; } mm_mesh;

/* Per-simulation material.  Kc is the cubic constant of the paper's form
 * E = Kc (mx^4 + my^4 + mz^4) (Sec. "Anisotropy"); u is normalised by the
 * library; precession = 0 drops the -g~ m x H term (relaxation / NEB);
 * demag = 0 switches the demagnetising field off. */
typedef struct {
    double Ms, A, D;
    int dmi_kind;
    double Ku, u[3], Kc;
    double H[3];
    double alpha, gamma;
    int precession;
    int demag;
} mm_material;

/* Per-simulation integration status (mm_get_status). */
typedef struct {
    double t, h, err, max_dmdt;
    long long n_accepted, n_rejected;
    int status;           /* 0 running, 1 reached t_end, 2 relaxed, <0 error code */
    int pad;
} mm_status;

/* Create a context on CUDA device `device` with precision MM_F64 or MM_F32.
 * cuda_stream is a cudaStream_t (NULL = the library creates its own). */
int mm_create(mm_ctx **out, int device, int precision, void *cuda_stream);
int mm_destroy(mm_ctx *ctx);
const char *mm_last_error(const mm_ctx *ctx);

/* Add a simulation (mesh + material + optional per-cell Ms, host double
 * array of nx*ny*nz values, NULL for uniform Ms = mat->Ms; Ms = 0 marks
 * cells outside the shape, Listing 1).  Must precede mm_precompute_demag.
 * Limits: each padded FFT length (next power of two >= 2n-1) <= 8192 in an
 * FP32 context, <= 4096 in an FP64 context (one row or column tile in shared
 * memory); MM_EINVAL otherwise. */
int mm_add_sim(mm_ctx *ctx, const mm_mesh *mesh, const mm_material *mat,
               const double *Ms_cells, int *sim_id);

/* Offsets (in elements) of each simulation's [3][N] block inside a batch
 * state buffer, and the total length; offsets has room for n_sims entries. */
int mm_batch_layout(const mm_ctx *ctx, long long *offsets, long long *total);
int mm_num_sims(const mm_ctx *ctx);

/* Tile shapes and schedules of one simulation's passes (an implementation
 * choice: the paper's kernels use library FFTs and have no counterpart).
 * 0 in a field keeps the library's fixed rule.
 *   Ty          kx columns per spectrum block and column tile (power of two, 1..32)
 *   Rx          rows per x-pass CTA (1..ny)
 *   x_threads   threads per x-pass CTA (multiple of 32, <= 1024 FP32 / 512 FP64)
 *   col_threads threads per column-pass CTA of meshes with one plane or more
 *               than 8 planes (same limits)
 *   col_group   cluster pass (2..8 planes): column FFT stages per register
 *               group, 1 = 16-point groups, 2 = 32-point groups
 *   col_occ     cluster pass: CTAs per SM its kernel is built for, 3 or 4 (FP32
 *               up to 4 planes, column tiles small enough for that many CTAs'
 *               shared memory; fewer registers a thread, and 8-point column
 *               groups at 4) or 0 / 2 (the rule)
 *   x_stage     1: the x-inverse pass stages its tile's state rows, with their
 *               +-y and +-z neighbours, in shared memory by bulk copies
 *               (cp.async.bulk, completed on an mbarrier) that overlap its
 *               inverse FFT; 0 / 2: the rule (the epilogue loads them directly)
 * The two CTA widths act per launch, which covers the whole batch: they apply
 * when every simulation of the context has the same value (else the rule). */
typedef struct { int Ty, Rx, x_threads, col_threads, col_group, col_occ, x_stage; } mm_tuning;

/* Set the tuning of one simulation (sim_id = -1: every simulation); must
 * precede mm_precompute_demag.  MM_EINVAL if the tiles do not fit the kernels
 * (shared memory, limits above). */
int mm_set_tuning(mm_ctx *ctx, int sim_id, const mm_tuning *t);

/* The tuning in use by one simulation, every field resolved (rule values
 * filled in; col_group 0 for a simulation without the cluster pass). */
int mm_get_tuning(const mm_ctx *ctx, int sim_id, mm_tuning *out);

/* Autotune the mesh of simulation sim_id (before mm_precompute_demag): time
 * candidate tunings -- kx block width and column register groups, then rows
 * per x tile and x-pass CTA width, then column-pass CTA width, each phase
 * starting from the best of the last, the fixed rule first -- as `reps` RK45
 * attempts each (CUDA events, after two untimed ones) of a scratch copy of the
 * whole batch (every simulation with its material, per-cell constants and
 * current tuning) on the same device, the candidate on the simulations of that
 * mesh, and set the fastest on them; its CTA widths, which act on the whole
 * batch, go to every simulation.  best (nullable) receives the chosen values
 * (0 where the rule was kept), best_ms / rule_ms (nullable) the milliseconds
 * per attempt of the batch with the best and with the starting tuning.  The
 * scratch context allocates and frees device memory. */
int mm_autotune(mm_ctx *ctx, int sim_id, int reps, mm_tuning *best, double *best_ms, double *rule_ms);

/* Which kernels run the RK45 attempts of mm_rk45_attempts, mm_rk45_step and
 * mm_relax (an implementation choice: the paper's integrator has no
 * counterpart).  MM_ATTEMPT_AUTO (the default): when every simulation of the
 * context has one plane and padded FFT lengths Px, Py <= 64 (at most 32 x 32
 * cells), no extended terms (bulk / D_2d DMI, per-cell A or D, spin torques)
 * and no NEB chain, the attempts run in ONE launch per call (per 1024 attempts
 * of a call): one thread-block
 * cluster per simulation keeps y_n, the stage vectors and both transform
 * stages in shared memory and runs all n attempts of the call, with the same
 * stage, error-norm, controller and projection arithmetic as the pass kernels
 * (the controller's err^-1/5 from a Newton-refined fifth root, within two ulps
 * of pow) and its transforms as warp-shuffle FFTs in the context's transform
 * precision; otherwise, and with MM_ATTEMPT_PASSES, every attempt replays the
 * pass kernels from a CUDA graph.  kind = 2, 4, 8 or 16 chooses the single
 * launch (where it applies) on a cluster of that many CTAs per simulation
 * instead of the largest the device co-schedules (a tuning choice).  May be
 * called at any time after mm_create; MM_EINVAL for another kind. */
enum { MM_ATTEMPT_AUTO = 0, MM_ATTEMPT_PASSES = 1 };
int mm_set_attempt_kernel(mm_ctx *ctx, int kind);
/* The path the next attempt takes (after mm_precompute_demag): *single = 1 for
 * the single launch (cluster: its CTAs per simulation), 0 for the pass kernels
 * (cluster: 0).  Either pointer may be NULL. */
int mm_get_attempt_kernel(mm_ctx *ctx, int *single, int *cluster);

/* Applied field of one simulation (field sweeps, Listing 2), A/m. */
int mm_set_field(mm_ctx *ctx, int sim_id, const double H[3]);

/* Cell-based exchange and DMI constants of one simulation (host double arrays
 * of nx*ny*nz values, J/m and J/m^2; NULL keeps that constant uniform, both
 * NULL return to uniform A and D).  Neighbours couple with the harmonic means
 * A_ij = 2 A_i A_j / (A_i + A_j) and D_ij = 2 D_i D_j / (D_i + D_j), 0 where
 * the two values sum to 0 (Sec. "Exchange energy", Sec. "Dzyaloshinskii-
 * Moriya Energy").  Must precede mm_precompute_demag; MM_EINVAL for a
 * non-finite value.  The arrays are copied. */
int mm_set_cell_params(mm_ctx *ctx, int sim_id, const double *A_cells, const double *D_cells);

/* Spin torques of one simulation (Sec. "Spin transfer torques"), added to
 * the implicit LLG equation dm/dt = -gamma m x H + alpha m x dm/dt + T with
 *   T = m x (m x (u.grad)m) + beta m x (u.grad)m      (Zhang-Li, u in m/s)
 *       - a_J m x (m x p) - b_J m x p                 (Slonczewski / spin-orbit,
 *                                                       a_J, b_J in 1/s)
 * and solved for dm/dt: the right-hand side gains (T + alpha m x T)/(1 + alpha^2).
 * (u.grad)m is the central difference (m_+ - m_-)/(2 Delta) along each axis,
 * a neighbour outside the mesh or with Ms = 0 taken as the cell itself; p is
 * normalised (it must be non-zero when a_J or b_J is).  The torques act with
 * and without the precession term, enter the RK45 attempts, relax, rhs_eval
 * and mm_rk4 with cayley = 0 (mm_rk4 with cayley = 1 returns MM_EINVAL), and
 * not the minimiser or the energies, which use H_eff only.  May be called at
 * any time; zeros switch the torques off.  MM_EINVAL for a non-finite value. */
int mm_set_spin_torque(mm_ctx *ctx, int sim_id, const double u[3], double beta, double a_J, double b_J,
                       const double p[3]);

/* Finalise the batch: allocate device state, compute the Newell tensor in
 * FP64 for every distinct (mesh, cell) geometry (Eq. 7, Newell 1993; closed
 * form near, tent-averaged dipole quadrature far) and its spectrum, and
 * store -N^/(Px Py Pz) in the context precision.  Simulations with the same
 * geometry share one spectrum. */
int mm_precompute_demag(mm_ctx *ctx);

/* Real-space tensor of one simulation's geometry, FP64, for offsets
 * |i| < nx etc: out_host has 6*(2nz-1)*(2ny-1)*(2nx-1) doubles laid out
 * [c][k+nz-1][j+ny-1][i+nx-1], c in (xx, yy, zz, xy, xz, yz). */
int mm_newell_tensor(mm_ctx *ctx, int sim_id, double *out_host);

/* Integration state m (sim_id = -1: the whole batch in batch layout).  Host
 * buffers are double in every context; in an FP32 context a page-locked host
 * buffer (cudaMallocHost or registered) moves its FP64 values by DMA and is
 * converted on the device, any other host buffer is converted on the host
 * through a pinned staging buffer (the same rounding either way). */
int mm_set_m(mm_ctx *ctx, int sim_id, const void *m, int where);
int mm_get_m(mm_ctx *ctx, int sim_id, void *m, int where);

/* One right-hand-side evaluation (Eqs. 1-14 + LL form, with the spin torques
 * when set) of caller-owned device buffers: m_dev in, dmdt_dev out, heff_dev
 * (nullable) out, all in the context precision, [3][N] per simulation
 * (sim_id = -1: whole batch layout).  H_eff holds the field terms only (the
 * spin torques are not fields).  Asynchronous on the context stream. */
int mm_rhs_eval(mm_ctx *ctx, int sim_id, const void *m_dev, void *dmdt_dev, void *heff_dev);

/* Demagnetising field of one simulation through the magnetic scalar potential
 * (Sec. "Magnetostatic energy": with the scalar potential the three inverse
 * transforms reduce to one): u_i = sum_j S(r_i - r_j) . Ms_j m_j with S_c the
 * exact potential of a cell magnetised along c (the potential of its two
 * charged c-faces), evaluated by zero-padded FFTs on a grid padded to the
 * smallest power of two >= 2n + 1 per axis (three forward transforms of M,
 * one inverse of u), then H_d = -grad u by central differences, u taken one
 * cell outside the mesh where a neighbour lies outside.  This is a different
 * discretisation from the Newell field of mm_rhs_eval: the two agree inside
 * smooth magnetisation to second order in the cell size and differ by tens of
 * percent of Ms at charged surfaces.  m_dev in, hd_dev out, caller-owned
 * device buffers [3][nz][ny][nx] in the context precision (FP64 contexts
 * compute in FP64); asynchronous on the context stream.  The kernel spectrum
 * is computed (FP64) and kept on the first call for each geometry, which
 * allocates device memory.  MM_EINVAL for a padded length above 2048 (an axis
 * of more than 1023 cells). */
int mm_demag_potential(mm_ctx *ctx, int sim_id, const void *m_dev, void *hd_dev);

/* The same evaluation with host double buffers (copies inside the call). */
int mm_rhs_eval_host(mm_ctx *ctx, int sim_id, const double *m_host, double *dmdt_host,
                     double *heff_host);

/* Adaptive Dormand-Prince RK45 (Sec. "LLG equation").  mm_rk45_attempts
 * issues n_attempts attempted steps for every running simulation without
 * synchronising (7 right-hand sides each, the error-norm reduction, the
 * controller and the projection, captured once as a CUDA graph).
 * mm_rk45_step repeats attempts until every running simulation accepted one
 * step.  rtol is the error tolerance of the step controller (max-norm of the
 * embedded error, absolute = relative as |m| = 1). */
int mm_rk45_setup(mm_ctx *ctx, double rtol, double t_end, double max_dmdt);
int mm_rk45_attempts(mm_ctx *ctx, int n_attempts);
int mm_rk45_step(mm_ctx *ctx, int *n_accepted, int *n_rejected);

/* Integrate every simulation until t >= t_end (t_end > 0) or until
 * max_i |dm/dt|_i < max_dmdt rad/s (max_dmdt > 0), at most max_steps
 * attempts; sync_every attempts are issued between status checks. */
int mm_relax(mm_ctx *ctx, double rtol, double t_end, double max_dmdt, long long max_steps,
             int sync_every, long long *attempts_done);

int mm_get_status(mm_ctx *ctx, int sim_id, mm_status *out);
int mm_reset_time(mm_ctx *ctx);

/* Integrator state of one simulation, for checkpoint and resume.  Together
 * with its magnetisation (mm_get_m / mm_set_m; a host round trip is exact in
 * both precisions) it is everything the next RK45 attempt reads: there is no
 * first-same-as-last stage carried between attempts, and the reduction
 * fields an attempt accumulates start from zero.  Restoring both into the
 * same context, or into one built with the same simulations and precision,
 * continues the integration exactly as the uninterrupted run would.
 * mm_set_checkpoint returns MM_EINVAL for rtol <= 0, a negative or
 * non-finite h or t, or a status outside {0, 1, 2} and the error codes. */
typedef struct {
    double t;             /* simulated time, s */
    double h;             /* next step size, s (0: chosen at the next attempt) */
    double t_end;         /* stop time, s (0: none) */
    double rtol;          /* step-controller tolerance */
    double max_dmdt;      /* relax threshold, rad/s (0: none) */
    long long n_accepted, n_rejected;
    int status;           /* as in mm_status */
    int pad;
} mm_checkpoint;
int mm_get_checkpoint(mm_ctx *ctx, int sim_id, mm_checkpoint *out);
int mm_set_checkpoint(mm_ctx *ctx, int sim_id, const mm_checkpoint *in);

/* Energies of one simulation at its current m, J:
 * E[0..6] = exchange, dmi, uniaxial, cubic, zeeman, demag, total. */
int mm_energy(mm_ctx *ctx, int sim_id, double E[7]);

/* Nudged elastic band (Sec. "Miscellaneous"; geodesic NEB of Bessarab et
 * al. 2015 for the details the paper leaves out).  Makes simulations
 * [first_sim, first_sim + n_images) one chain: their end images are fixed,
 * the free images move along -alpha g~ m x (m x F) with F the effective
 * field minus its tangent part plus the spring force k_spring (A/m per
 * radian) along the tangent; the chain shares one step size. */
int mm_neb_setup(mm_ctx *ctx, int first_sim, int n_images, double k_spring);
/* n_steps attempted RK45 steps of every chain; energies_out (nullable,
 * host) receives the energy of every simulation afterwards. */
int mm_neb_relax(mm_ctx *ctx, double rtol, long long n_steps, double *energies_out);

/* Steepest-descent energy minimisation of every simulation (Sec. "Steepest
 * descent energy minimization"): per cell, with f = m x H_eff and
 * g = m x (m x H_eff), m_{k+1} = ((1 - a) m_k - tau_k g_k) / (1 + a),
 * a = tau_k^2 |f|^2 / 4 (the paper's explicit form of its norm-preserving
 * midpoint step), and Barzilai-Borwein step sizes from the sums over a
 * simulation's cells, tau^1 = s.s / s.y on odd steps and tau^2 = s.y / y.y on
 * even ones (s = m_k - m_{k-1}, y = g_k - g_{k-1}); tau_0 = 0.01 / max|g|; a
 * rule that is not positive falls back to 0.01 / max|g|, and every step is
 * capped at tau <= 1 / max|g| (no cell turns by more than about one radian).
 * Starts from the current m
 * (mm_set_m) with no history; a simulation stops once max|dm/dt| of its LL
 * right-hand side (material alpha, gamma, precession flag) falls below
 * max_dmdt rad/s (0: never).  Runs at most max_steps steps, checking every
 * sync_every steps; steps_done (nullable) receives the largest step count,
 * converged (nullable) 1 if every simulation stopped on the criterion.  The
 * step sums are FP64 (compensated per thread in FP32 contexts), tau is FP64,
 * the update runs in the context precision and is followed by the projection
 * onto |m| = 1 (the update keeps |m| only in exact arithmetic).  Returns
 * MM_ENAN on a non-finite field and MM_EINVAL in a context with NEB chains.
 * Leaves the RK45 state (t, h) untouched. */
int mm_minimize(mm_ctx *ctx, double max_dmdt, long long max_steps, int sync_every, long long *steps_done,
                int *converged);
/* Last minimiser state of one simulation: steps taken, tau (m/A), max|dm/dt|
 * (rad/s) at the last step's m, status (0 running, 2 converged, -4 NaN). */
int mm_minimize_info(mm_ctx *ctx, int sim_id, long long *steps, double *tau, double *max_dmdt, int *status);

/* n_steps fixed steps of size h (seconds) of classical four-stage Runge-Kutta
 * on every simulation (Sec. "Cayley transform"), from the current m, in the
 * context precision.  cayley = 0: RK4 on the LL right-hand side dm/dt, then
 * m <- m / |m| after each step.  cayley = 1: with dm/dt = f x m,
 * f = gamma (H + alpha m x H) / (1 + alpha^2) (only the alpha term without
 * precession), RK4 on d omega/dt = f - omega x f / 2 + (omega . f) omega / 4
 * from omega = 0 and m_{n+1} = Q(omega_{n+1}) m_n with the Cayley transform
 * Q = (I - Omega/2)^-1 (I + Omega/2), Omega x = omega x x (a rotation: |m|
 * is kept to rounding).  Cells with Ms = 0 do not move.  Each simulation's
 * time advances by n_steps * h; its RK45 step size and status are untouched.
 * There is no error control and no check of the values.  Returns MM_EINVAL
 * for h not positive and finite, n_steps < 0, a context with NEB chains, or
 * cayley = 1 with spin torques set (f is built from H_eff). */
int mm_rk4(mm_ctx *ctx, double h, long long n_steps, int cayley);

/* Profiling aid: runs `reps` RK45 attempts (NEB attempts in a context with
 * chains) with direct launches (no graph) and a CUDA event recorded on the
 * context stream after every kernel kind.
 * ms[k] / counts[k] receive the summed duration and the launch count of each
 * kernel kind k: 0 x-forward pass (with the RK prologue), 1 y forward,
 * 2 z fused, 3 y inverse, 4 y fused (films), 5 x-inverse + field/torque
 * epilogue, 6 step control, 7 projection, 8 NEB, 9 cluster-fused y/z pass;
 * arrays of 10 entries. */
int mm_profile_attempts(mm_ctx *ctx, int reps, double *ms, long long *counts);

/* Debugging aid: bounded-wait check.  Runs a kernel that waits on a device
 * flag nobody sets, for at most `spins` polls, and returns MM_ETIMEOUT.
 * `spins` must lie in [0, MM_MAX_WAIT_SPINS] (2^22 polls, about a second of
 * polling at most); other values return MM_EINVAL before anything runs. */
#define MM_MAX_WAIT_SPINS (1LL << 22)
int mm_debug_bounded_wait(mm_ctx *ctx, long long spins);

/* Number of kernels this context launched (graph launches count their
 * kernel nodes). */
long long mm_kernel_launches(const mm_ctx *ctx);

/* The right-hand-side evaluation of ONE simulation for callers that cannot
 * allocate device memory.  The paper has no counterpart: this is a service of
 * this library.  Callers such as a plugin handed device pointers by its host
 * application, or code whose process owns the allocator, may not call
 * cudaMalloc; this call allocates nothing (no cudaMalloc, cudaFree or
 * allocating library routine).  The caller passes the state m_dev and the
 * outputs dmdt_dev and heff_dev (nullable), [3][nz][ny][nx] each in the given
 * precision (MM_F64: double, MM_F32: float), and a cudaStream_t (NULL = the
 * default stream); the result equals mm_rhs_eval's for the same simulation
 * (uniform Ms, A and D, no or interfacial DMI, no spin torques; another DMI
 * class returns MM_EINVAL).  Everything else -- twiddle tables, the FP64 Newell
 * tensor and its spectrum (recomputed on every call), the demag spectrum,
 * descriptors and work lists -- lives in one static device array of 32 MiB
 * that every GPU loading libmm holds until the process exits.  A mesh whose
 * padded FFT grid, Newell octant, tensor and spectrum do not fit returns
 * MM_EINVAL with a message (mm_last_error(NULL)); for example 256x256x1 fits,
 * 512x512x1 does not.  The first call in each CUDA context (with the
 * runtime's primary contexts: the first call on each device) looks the
 * array's device address up (cudaGetSymbolAddress) and remembers it under the
 * context's unique id: make that first call before any stream capture.  All
 * calls share the array and it keeps the last call's contents, so calls that
 * overlap on the GPU race: serialise them.  The call synchronises the stream
 * once (after the tensor), then returns with the evaluation queued. */
int mm_rhs_eval_static(const mm_mesh *mesh, const mm_material *mat, int precision,
                       const void *m_dev, void *dmdt_dev, void *heff_dev, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* MM_H */
