/*
 * dh.h — C ABI of the B300 (sm_103a) finite-volume Euler library.
 *
 * The library advances the compressible Euler equations (arXiv:2512.13403, Sec. 3, Eq. 2) on a
 * periodic uniform Cartesian grid with the pure update (U^{n+1}, theta^{n+1}) = H(U^n, theta^n)
 * of Sec. 2.1: primitive recovery and MUSCL reconstruction with the MC limiter (App. A.1), HLLC
 * fluxes with Davis wave speeds (App. A.2), the unsplit divergence integrated by SSP-RK2
 * (App. A.3), the CFL time step (App. A.4), and the operator-split sources — Ornstein-Uhlenbeck
 * forcing (Sec. 3.1.1), optically thin cooling (Sec. 4.3) and multigrid self-gravity (Sec. 5.2).
 *
 * Data layout.  A state is five structure-of-arrays planes (rho, m_x, m_y, m_z, E), each
 * nx*ny*nz contiguous values with x fastest, then y, then z: element (f, k, j, i) sits at
 * offset f*nx*ny*nz + (k*ny + j)*nx + i.  Values are float (DH_F32) or double (DH_F64) as
 * chosen at dh_create; every pointer argument that carries a state uses that type.
 *
 * Ownership.  A context owns every device buffer it needs (allocated once in dh_create and
 * released in dh_destroy) and the CUDA stream passed to dh_create (not owned: the caller keeps
 * it alive).  Caller buffers are only read or written during the call that receives them, and
 * all device work of a call is ordered on the context's stream.  Pointers flagged `on_device`
 * are device pointers (for example torch CUDA tensors on the same device); otherwise host
 * pointers (pinned or pageable).
 *
 * Errors.  Every entry point returns a dh_status; none aborts, traps or waits without bound.
 * DH_ERR_ARG leaves the context unchanged.  After DH_ERR_NONFINITE or DH_ERR_POSITIVITY the
 * context's state, time, step count and forcing state are those of the last good step.
 * dh_last_error() returns a message for the most recent failure on that context.
 */
#ifndef DH_H
#define DH_H

#ifdef __cplusplus
extern "C" {
#endif

#define DH_API_VERSION 1

typedef enum {
  DH_OK = 0,
  DH_ERR_ARG = 1,          /* invalid argument or unsupported configuration               */
  DH_ERR_CUDA = 2,         /* a CUDA runtime call failed (message in dh_last_error)       */
  DH_ERR_NONFINITE = 3,    /* a non-finite value appeared in the state                    */
  DH_ERR_POSITIVITY = 4,   /* rho <= 0 or P <= 0 after a step                             */
  DH_ERR_MG_NOCONV = 5,    /* multigrid did not reach its tolerance within mg_max_cycles  */
  DH_ERR_STATE = 6         /* call out of order (e.g. step before init_state)             */
} dh_status;

typedef enum { DH_F32 = 0, DH_F64 = 1 } dh_precision;

typedef struct dh_ctx dh_ctx;

/* Run configuration.  Fill with dh_config_default, then override fields. */
typedef struct dh_config {
  int nx, ny, nz;            /* cells per axis; each >= 4                                  */
  int precision;             /* DH_F32 (production) or DH_F64 (parity checks)              */
  double dx, dy, dz;         /* cell widths (default 1/n: unit periodic box)               */
  double gamma;              /* adiabatic index (default 5/3)                              */
  double cfl;                /* Courant number C of App. A.4 (default 0.4)                 */
  double dt_max;             /* upper bound on dt (default +inf)                           */
  /* Ornstein-Uhlenbeck forcing, Sec. 3.1.1: modes 1 <= |n| <= 2, solenoidal.
     Needs nx, ny, nz >= 5 so that the forced modes do not alias on the grid. */
  int forcing;               /* 0/1                                                        */
  double ou_tau;             /* autocorrelation time (default 0.5)                         */
  double ou_arms;            /* rms acceleration a_rms (default 1.0)                       */
  unsigned long long ou_seed;/* seed of the counter-based SplitMix64 draws (default 1)      */
  /* Optically thin cooling, Sec. 4.3, Lambda = n^2 T^(1/2), code units T = P / rho. */
  int cooling;               /* 0/1                                                        */
  double t_floor;            /* temperature floor (default 0.05)                           */
  double cool_frac;          /* first-substep fractional change limit f (default 0.1)      */
  int nsub_max;              /* substep cap (default 1024)                                 */
  /* (c_cool, the cooling time-step factor, is the last field below.) */
  /* Multigrid self-gravity, Sec. 5.2 and App. C: A phi = 4 pi G (rho - <rho>) by V- or
     W-cycles smoothed by red-black Gauss-Seidel or weighted Jacobi.  Needs dx == dy == dz;
     halving stops at dims < 8 or odd, coarsest <= 1024 cells. */
  int gravity;               /* 0/1                                                        */
  double four_pi_G;          /* 4 pi G (default 1)                                         */
  double mg_tol;             /* ||F - A phi||_2 / ||F||_2 stop tolerance (default 1e-6)   */
  int mg_max_cycles;         /* cycle cap (default 30)                                     */
  int mg_pre, mg_post;       /* smoothing sweeps before / after the coarse correction (2,2)*/
  int mg_smoother;           /* 0: red-black Gauss-Seidel (default); 1: weighted Jacobi     */
  double mg_omega;           /* Jacobi weight, 0 < omega <= 1 (default 2/3, Sec. 5.2)       */
  int mg_cycle;              /* 1: V-cycle (default); 2: W-cycle, two visits of each coarser
                                level above the coarsest (App. C)                          */
  /* Scheme (App. A.1, A.3). */
  int limiter;               /* 0: MC (default); 1: van Leer 2ab/(a+b)                     */
  int integrator;            /* 2: RK2 / Heun (default); 3: SSPRK3 (Shu-Osher form)        */
  /* Cooling time-step limit, Sec. 4.3: with cooling on and c_cool finite, the step is
     min(CFL step, c_cool * min over cells of t_cool, dt_max), t_cool = E_th / |Edot| over the
     cells above the floor energy.  Default +inf: off (cooling subcycles per cell instead). */
  double c_cool;
} dh_config;

/* Fills *cfg with the defaults above for an nx*ny*nz grid. */
void dh_config_default(dh_config* cfg, int nx, int ny, int nz);

/* Creates a context: validates *cfg (copied), allocates all device buffers on the current
   device and records `cuda_stream` (a cudaStream_t; NULL = legacy default stream).
   DH_ERR_ARG on an invalid configuration, DH_ERR_CUDA if allocation fails. */
dh_status dh_create(const dh_config* cfg, void* cuda_stream, dh_ctx** out);

/* Releases every buffer of the context.  NULL is ignored. */
void dh_destroy(dh_ctx* ctx);

/* Copies a state (layout above, context precision) into the context and resets time, step
   count, forcing state (draw 0 of Sec. 3.1.1) and the gravitational potential (zero). */
dh_status dh_init_state(dh_ctx* ctx, const void* U, int on_device);

/* Copies the current state out (layout above, context precision). */
dh_status dh_get_state(dh_ctx* ctx, void* U_out, int on_device);

/* One step (Sec. 2.1 update H): dt > 0 imposes the time step, dt <= 0 uses the CFL value of
   App. A.4 computed on the device from the current state.  *dt_used (nullable) receives the dt
   taken; reading it synchronises the stream. */
dh_status dh_step(dh_ctx* ctx, double dt, double* dt_used);

/* n_steps CFL steps with no host synchronisation between them; *t_out (nullable) receives the
   simulation time afterwards.  Synchronises once at the end to report errors. */
dh_status dh_advance(dh_ctx* ctx, int n_steps, double* t_out);

/* Time and completed step count of the current state. */
dh_status dh_get_time(dh_ctx* ctx, double* t, long long* nstep);

/* File checkpoint of the context (the restart the paper's pure update H(U^n, theta^n) of
   Sec. 2.1 implies: theta = time, step count, OU table, gravity warm start).  dh_save writes
   the current state, t, dt, the step count (which also numbers the OU draws), the OU tables
   and hold flag, and with gravity the potential that warm-starts the next solve (its float-float
   words: n hi floats then n lo floats), with a checksum; it settles pending steps first.  dh_load
   reads such a file into a context created with the same configuration in every dh_config
   field (grid, precision, cell widths, gamma, CFL and dt_max, limiter and integrator, the
   forcing, cooling and multigrid settings; else DH_ERR_ARG naming the first differing field,
   context unchanged), after which stepping continues bit for bit as in the saved context.  DH_ERR_ARG for unreadable, truncated or corrupted files.  Both synchronise. */
dh_status dh_save(dh_ctx* ctx, const char* path);
dh_status dh_load(dh_ctx* ctx, const char* path);

/* Diagnostics of the run so far (a metrics record per step when called after each step).
   The paper keeps none beyond its figures; the record carries what the method's failure and
   accuracy conditions depend on: the time and step, the status bits raised since the state was
   set (DH_FLAG_*: DH_FLAG_COOL_CAP is informational, a cell reached the cooling substep cap of
   Sec. 4.3), the largest cooling substep count of any cell since the previous dh_get_metrics
   (1 when cooling ran without subcycling, 0 without cooling or steps), the last Poisson
   solve's cycle count and relative residual (Sec. 5.2), the float64 conserved totals and the
   minima over cells of rho and P of the current state.  Settles enqueued steps and returns
   their status; synchronises. */
enum { DH_FLAG_NONFINITE = 1, DH_FLAG_POSITIVITY = 2, DH_FLAG_MG_NOCONV = 4, DH_FLAG_COOL_CAP = 8,
       DH_FLAG_TIMEOUT = 16 /* a kernel's bounded wait for its own copies gave up (fatal) */ };
typedef struct dh_metrics {
  double t, dt;             /* time after the last completed step, and its dt            */
  long long nstep;          /* completed steps                                           */
  unsigned flags;           /* DH_FLAG_* bits                                            */
  int cool_max_substeps;    /* largest cooling substep count since the previous read     */
  long long slope_fallbacks; /* positivity fallbacks of the PLM slopes since the previous
                                read: (cell, axis, RK stage) triples whose slopes were zeroed
                                because a face state had rho <= 0 or P <= 0 (App. A.2)     */
  int mg_cycles;            /* cycles of the last Poisson solve (0 without gravity)      */
  double mg_residual;       /* its ||F - A phi||_2 / ||F||_2                             */
  double totals[5];         /* sums over cells of rho, m_x, m_y, m_z, E (float64)        */
  double rho_min, p_min;    /* minima over cells of rho and P                            */
} dh_metrics;
dh_status dh_get_metrics(dh_ctx* ctx, dh_metrics* out);

/* CFL time step C * min_cells,axes dx_a / (|v_a| + c_s) of the current state (App. A.4). */
dh_status dh_compute_dt(dh_ctx* ctx, double* dt);

/* Sum over cells of each conserved field, accumulated in float64 on the device
   (deterministic order).  out[5] is a host array. */
dh_status dh_conserved_totals(dh_ctx* ctx, double out[5]);

/* Normalised forcing acceleration a(x) of the most recent forcing update (Sec. 3.1.1), three
   planes (a_x, a_y, a_z) in the state layout and context precision.  DH_ERR_STATE if forcing
   is off. */
dh_status dh_forcing_field(dh_ctx* ctx, void* a_out, int on_device);

/* Forcing mode table a_hat[m][c] (16 modes x 3 components, unnormalised) as interleaved
   (re, im) float64 pairs: out[2*(3*m + c) + {0,1}].  Modes are the half-space
   {1 <= |n|^2 <= 4, first nonzero component of n positive} in lexicographic (n_x, n_y, n_z)
   order. */
dh_status dh_forcing_modes(dh_ctx* ctx, double out[96]);

/* Sets the forcing mode table (same layout as dh_forcing_modes).  hold = 1 keeps it: later
   steps skip the OU update of Sec. 3.1.1 and force with this table (renormalised to a_rms) until
   the next call with hold = 0.  Used to drive several runs (a coarse and a fine grid) with one
   acceleration history.  DH_ERR_STATE if forcing is off. */
dh_status dh_set_forcing_modes(dh_ctx* ctx, const double modes[96], int hold);

/* Block mean of a float32 state (device, state layout, nx*ny*nz) over factor^3 cells into
   U_coarse (device, (nx/factor)*(ny/factor)*(nz/factor)): the conservative restriction of the
   conserved fields onto a coarser grid.  Dimensions must be divisible by factor. */
dh_status dh_downsample(const float* U_fine, int nx, int ny, int nz, int factor, float* U_coarse,
                        void* cuda_stream);

/* Gravitational potential phi of the last solve (one plane, float64, state index order),
   and the cycles / final relative residual of that solve (nullable outputs).  The context holds
   phi in float-float (about 48 significant bits) in whatever gauge the solves left it (only
   differences of phi enter a step); phi_out receives phi - <phi> rounded to float64. */
dh_status dh_get_potential(dh_ctx* ctx, double* phi_out, int on_device, int* cycles,
                           double* rel_residual);

/* The same Poisson problem solved exactly by the discrete Fourier transform (the FFT solver
   named beside the multigrid one, Sec. 2.3 and 5): F = four_pi_G (rho - <rho>) from one density
   plane `rho` (state index order, context precision; on_device as in dh_init_state), then
   phi_hat = F_hat / lambda(k) with lambda(k) = -(4/h^2) sum_a sin^2(pi k_a / n_a) the
   eigenvalues of the seven-point operator, phi_hat(0) = 0.  Float64 complex arithmetic; every
   dimension a power of two in [2, 1024] (else DH_ERR_ARG).  phi_out: n float64 values, device
   or host memory (out_on_device).  Needs gravity on (four_pi_G, cubic cells).  Leaves the
   context's potential and state alone; synchronises.  A cross-check of the multigrid. */
dh_status dh_fft_poisson(dh_ctx* ctx, const void* rho, int on_device, double* phi_out,
                         int out_on_device);

/* Sets the potential, the warm start of the next Poisson solve, to zero (the cold start of
   dh_init_state) without touching the state.  Needs gravity on.  Asynchronous on the stream. */
dh_status dh_reset_potential(dh_ctx* ctx);

/* Poisson solve of Sec. 5.2 on its own: F = four_pi_G (rho - <rho>) from one density plane
   `rho` (state index order, context precision), red-black Gauss-Seidel V-cycles warm-started from
   the context's potential until ||F - A phi||_2 / ||F||_2 <= mg_tol; the potential stays in the
   context (read it with dh_get_potential).  Needs gravity on.  DH_ERR_MG_NOCONV if mg_max_cycles
   cycles do not reach the tolerance (the potential is then the last iterate). */
dh_status dh_solve_poisson(dh_ctx* ctx, const void* rho, int on_device);

/* Reverse-mode product through n_steps steps (hand adjoint, App. A.3 stages transposed; dt of
   every step frozen at the value the forward took, App. A.4): given the current state U^0,
   runs the forward n_steps CFL steps (storing U every `ckpt_every` steps, Sec. 2.3
   checkpointing; an interval above n_steps is taken as n_steps), then returns dL/dU^0 in
   dLdU0 for dL/dU^{n} = dLdU_final.  n_steps = 0 copies dLdU_final; n_steps < 0 or
   ckpt_every < 1 is DH_ERR_ARG.  Both buffers use
   the state layout and precision; the context is left at U^{n} and steps on as if no adjoint
   had run.  The operator-split sources are differentiated too: the OU kick with each step's
   field held fixed (Sec. 3.1.1; the draws do not depend on U), self-gravity (Sec. 5: the kick
   transposed pointwise, then the potential's share through one more Poisson solve with the
   symmetric seven-point operator, to mg_tol) and cooling (Sec. 4.3: forward-mode tangents of
   the trapezoid or subcycled update along the branches the forward took).  DH_ERR_MG_NOCONV if
   an adjoint Poisson solve misses mg_tol. */
dh_status dh_adjoint_advance(dh_ctx* ctx, int n_steps, int ckpt_every, const void* dLdU_final,
                             void* dLdU0, int on_device);
/* dh_adjoint_advance with every step of the forward sweep taken at the imposed dt > 0 (as
   dh_step(dt)); dt = 0 is the CFL step of dh_adjoint_advance.  The form a rollout whose steps
   must land on fixed times (solver-in-the-loop training against a reference trajectory) needs. */
dh_status dh_adjoint_advance_dt(dh_ctx* ctx, int n_steps, int ckpt_every, double dt,
                                const void* dLdU_final, void* dLdU0, int on_device);

/* ---- Corrector building blocks (residual 3D CNN, BF16 tensor cores, FP32 accumulation) ----
   A 3x3x3 periodic convolution over an nx*ny*nz grid as an implicit GEMM on tcgen05:
   out[cell, n] = sum_{tap, c} act[cell + offset(tap), c] * W[n, c, tap] (+ bias[n]), the
   closure network of Sec. 7 in 3D.  Every dimension must be >= 3.  All pointers are device
   pointers; work is ordered on `stream`.

   Padded activation layout (bf16): C channels (C = 8, up to 8 real with the rest zero, or 32)
   are stored as C/8 channel groups of R = dh_conv_padded_rows(nx, ny, nz) rows of 8 bf16
   (16 bytes), group after group, C/8 * R * 16 bytes in all.  In group g, row
   guard + ((z+1)(ny+2) + (y+1))(nx+2) + (x+1) holds channels 8g..8g+7 of cell (x, y, z) for
   x, y, z in [-1, n]: coordinates -1 and n are periodic images (x = -1 is cell nx-1, and so on
   for faces, edges and corners).  The guard rows before and after the padded volume must be
   zero: allocate the buffer zeroed once; the kernels below write only cell rows and their
   images.  A tap is then a fixed row offset, which is what lets the tensor-core operand of
   every tap be a shifted view of one shared-memory window.

   dh_conv_padded_rows: R above (-1 if a dimension is < 3).
   dh_conv_pad: channel-last bf16 [cell][channels] -> padded layout (cell rows and images).
   dh_conv_unpad: padded layout -> channel-last bf16 [cell][channels].  channels is 8 or 32.

   dh_pack_conv_weights: converts fp32 weights W[cout][cin][3][3][3] (cross-correlation order,
   kernel index (kz, ky, kx) = offset + 1) into the packed bf16 operand `packed` of
   n_pad * k_pad elements (n_pad = 32 if the packed output count is 32, else 16; k_pad = 864
   for 9..32 input channels, 224 for <= 8).  transpose_flip = 0 packs the forward
   convolution (outputs = cout); 1 packs its data gradient (outputs = cin, taps mirrored), so
   that the same kernel maps an output gradient to an input gradient.

   dh_conv3d_bf16: act in the padded layout with cin_pad channels.  Modes: 0 = GELU (out bf16
   padded, 32 channels, = bf16(gelu(z)); z_out fp32 [cell][32] = acc + bias, nullable);
   1 = linear (out fp32 planar [n_real][cell] = acc + bias); 2 = GELU gradient (out bf16
   padded, 32 channels, = bf16(acc * gelu'(z_in)), z_in fp32 [cell][32]).  Supported
   (cin_pad, nout_pad, mode): (8,32,0), (8,32,2), (32,32,0), (32,32,2), (32,16,1), (32,32,1).
   Shared-memory windows of (130 + 2 (nx+2)) rows per tap plane must fit next to the weights:
   two or three of them (copies overlapping the MMAs) up to nx of about 160 with 32 input
   channels, one beyond; DH_ERR_ARG for nx beyond about 330.  *err_flag (device
   unsigned) becomes nonzero if a bounded wait inside the kernel gave up. */
long long dh_conv_padded_rows(int nx, int ny, int nz);
dh_status dh_conv_pad(const void* src, int channels, int nx, int ny, int nz, void* dst,
                      void* stream);
dh_status dh_conv_unpad(const void* src, int channels, int nx, int ny, int nz, void* dst,
                        void* stream);
dh_status dh_pack_conv_weights(const float* W, int cout, int cin, int transpose_flip,
                               void* packed, void* stream);
dh_status dh_conv3d_bf16(const void* act, int cin_pad, const void* packed, int nout_pad,
                         const float* bias, int mode, const float* z_in, void* out,
                         float* z_out, int n_real, int nx, int ny, int nz, unsigned* err_flag,
                         void* stream);

/* dh_conv3d_wgrad_bf16: weight gradient of such a convolution,
   dW[n][c][tap] = sum_cells grad[cell][n] * act[cell + offset(tap)][c], written in the fp32
   master layout W[cout][cin][27].  act: padded layout with cin_pad channels (cin real); grad:
   padded layout with grad_stride channels (8 or 32; cout real, the rest zero).  `partial` is
   caller-owned fp32 scratch of nctas * ceil(27*cin_pad/128) * 128 * (cout > 16 ? 32 : 16)
   values; the per-CTA partial sums are added in a fixed order. */
dh_status dh_conv3d_wgrad_bf16(const void* act, int cin_pad, int cin, const void* grad,
                               int grad_stride, int cout, int nx, int ny, int nz, float* partial,
                               int nctas, float* dW, unsigned* err_flag, void* stream);

/* The corrector network (Sec. 7 closure, a residual 3D CNN): x0 = bf16((U - mu)/sigma),
   z1 = conv(x0, W1) + b1, h1 = bf16(gelu(z1)), z2 = conv(h1, W2) + b2, h2 = bf16(gelu(z2)),
   y = conv(h2, W3) + b3, all 3x3x3 periodic, channels 5 -> 32 -> 32 -> 5.  Parameters are one
   flat fp32 device array of dh_cnn_param_count() = 36357 values: W1[32][5][27], b1[32],
   W2[32][32][27], b2[32], W3[5][32][27], b3[5]; norm15 = mu[5], sigma[5], s[5] (host, sigma > 0):
   input normalisation (U - mu)/sigma and per-channel output scale s of the correction.
   A dh_cnn owns the activations of one grid (every dimension >= 3). */
typedef struct dh_cnn dh_cnn;
long long dh_cnn_param_count(void);
dh_status dh_cnn_create(int nx, int ny, int nz, void* cuda_stream, dh_cnn** out);
/* The same network in either correction form (Sec. 7: a learned correction of the state, or a
   learned flux added in divergence form).  form 0 = state form above (5 outputs).  form 1 =
   flux form: W3[15][32][27], b3[15] (dh_cnn_param_count_form(1) = 45007 values), y[5 a + c] is
   the flux of field c through the face i + 1/2 along axis a (x, y, z), and the correction is
   dU_c(i) = -s_c sum_a (y_{a,c}(i) - y_{a,c}(i - e_a)), periodic: it changes no conserved total.
   Every call below takes either form; dh_cnn_backward then compares the divergence with the
   residual target.  DH_ERR_ARG for another form. */
long long dh_cnn_param_count_form(int form);
dh_status dh_cnn_create_form(int nx, int ny, int nz, int form, void* cuda_stream, dh_cnn** out);
void dh_cnn_destroy(dh_cnn* cnn);
/* Copies the parameters and packs the tensor-core operands (synchronises). */
dh_status dh_cnn_set_params(dh_cnn* cnn, const float* params, const float* norm15);
/* y = network(U) for a float32 state U (device, state layout); y_out (nullable, device) gets
   y as 5 planes.  Keeps the activations for dh_cnn_backward. */
dh_status dh_cnn_forward(dh_cnn* cnn, const float* U, float* y_out);
/* For the last forward (on U_in): residual target t = (U_target - U_in) / s per channel,
   loss = mean over 5 channels and cells of (y - t)^2; writes d loss / d params into grads
   (device, 36357 floats) and the loss into *loss (host, nullable).  U_in, U_target: float32
   states (device).  Synchronises. */
dh_status dh_cnn_backward(dh_cnn* cnn, const float* U_in, const float* U_target, float* grads,
                          double* loss);
/* Vector-Jacobian product of the correction dU(U) (before the floors) for the last
   dh_cnn_forward (on U): given dL_dcorr = dL/d(dU) (device, 5 planes float32), writes
   dL/d(params) into grads (device, param count floats) and, if dL_dU is not NULL,
   dL/dU = (d dU / dU)^T dL_dcorr into dL_dU (device, 5 planes float32).  The identity part of
   U + dU is the caller's.  The bf16 roundings of the forward are taken as the identity.  The
   building block of solver-in-the-loop training (Sec. 7), where the loss of a rollout is
   carried back through the corrector and the solver's adjoint.  Synchronises. */
dh_status dh_cnn_vjp(dh_cnn* cnn, const float* dL_dcorr, float* grads, float* dL_dU);
/* U <- U + dU(U) in place (float32 state, device; dU = s * network(U) in the state form),
   then rho >= rho_floor and E >= |m|^2/(2 rho) + rho T_floor/(gamma - 1).  An inference pass: it keeps no activations
   for dh_cnn_backward (call dh_cnn_forward again before the next backward).  Synchronises.
   DH_ERR_NONFINITE if a corrected value is not finite (U then holds the corrected values). */
dh_status dh_cnn_correct_state(dh_cnn* cnn, float* U, double rho_floor, double T_floor,
                               double gamma);
/* Solver-in-the-loop rollout training (Sec. 7: the loss of a rollout of solver steps, each
   followed by the correction, differentiated through both).  One term of the rollout loss for
   a state U and its reference T (float32, 5 planes of the network's grid, device):
   coef * sum over fields c and cells of ((U - T) / w_c)^2, with w5 five positive per-field
   weights (host).  With lam (nullable, device, same layout) also its gradient
   2 coef (U - T) / w_c^2, written (accumulate = 0) or added (accumulate = 1).  With loss_acc
   (nullable, one device double) the term is added to *loss_acc.  Asynchronous on the
   network's stream; DH_ERR_ARG for a non-positive weight. */
dh_status dh_cnn_rollout_misfit(dh_cnn* cnn, const float* U, const float* T, const float* w5,
                                double coef, float* lam, int accumulate, double* loss_acc);
/* The floors of the correction transposed (Sec. 7 corrector with the temperature floor of
   Sec. 4.3).  The last dh_cnn_forward must have been on V (the state before the correction);
   lam (device, 5 planes) holds dL/dU' for U' = floors(V + dU(V)) and is overwritten with
   dL/d(V + dU).  rho' = max(rho, rho_floor) passes the gradient where rho >= rho_floor;
   E' = max(E, |m|^2/(2 rho') + rho' T_floor/(gamma - 1)) gives it to the larger argument and
   splits an exact tie evenly, the floor's share flowing on to m and rho'.  Asynchronous.
   DH_ERR_STATE without a forward. */
dh_status dh_cnn_floor_vjp(dh_cnn* cnn, const float* V, float* lam, double rho_floor,
                           double T_floor, double gamma);
/* Per-field mean and standard deviation (n - 1 normalisation) over `count` samples of A - B
   (B nullable: A alone), each sample 5 planes of the network's grid (float32, device,
   contiguous): the normalisation statistics of the corrector's training set (Sec. 7).  out10
   (host): 5 means, then 5 standard deviations.  Float64 sums in a fixed order.  Synchronises. */
dh_status dh_cnn_field_moments(dh_cnn* cnn, const float* A, const float* B, long long count,
                               double* out10);
/* y <- y + a x over n floats (device), on `stream`: the sums of gradient contributions in
   rollout training. */
dh_status dh_axpy(long long n, double a, const float* x, float* y, void* stream);
/* Adam (Kingma & Ba) on n parameters: m, v are caller-owned moment buffers (device), step >= 1
   the 1-based step count for the bias corrections. */
dh_status dh_adam_step(float* params, const float* grads, float* m, float* v, long long n,
                       double lr, double beta1, double beta2, double eps, int step, void* stream);
/* Corrector of a float32 context: dh_set_corrector copies the parameters (as dh_cnn_set_params);
   dh_correct applies U <- U + s * network(U) to the current state with the floors above
   (rho_floor = 1e-6 <rho>, the context's T_floor and gamma); it settles enqueued steps first.
   DH_ERR_STATE without a corrector; DH_ERR_NONFINITE if the corrected state is not finite, in
   which case the context keeps the uncorrected state. */
dh_status dh_set_corrector(dh_ctx* ctx, const float* params, const float* norm15);
/* dh_set_corrector for either form (see dh_cnn_create_form); replaces a corrector of the
   other form. */
dh_status dh_set_corrector_form(dh_ctx* ctx, int form, const float* params, const float* norm15);
dh_status dh_correct(dh_ctx* ctx);
/* Sec. 7 (the corrector applied after each coarse step): with on = 1, every step that dh_step
   and dh_advance enqueue applies the corrector in place after its sources, on the device and
   without a host synchronisation (the same kernels and floors as dh_correct), and the next
   step's CFL time step is that of the corrected state.  A non-finite corrected state fails the
   step like a non-finite update: DH_ERR_NONFINITE, and the state holds the last good step.
   DH_ERR_STATE for on = 1 without a corrector.  While it is on, dh_adjoint_advance and
   dh_adjoint_advance_dt return DH_ERR_STATE (their adjoint covers the solver step only). */
dh_status dh_set_correct_every_step(dh_ctx* ctx, int on);

/* Conserved totals (as dh_conserved_totals) for callers that cannot allocate device memory,
   such as a host framework whose allocator owns the whole device-memory budget, or a
   time-critical loop that must not pay for the implicit device synchronisation of cudaMalloc.
   The paper has no counterpart; this entry point exists for such integrations only.
   Needs no context and allocates nothing: the per-block partial sums live in a fixed
   file-scope device array of 160 KiB (4096 blocks x 5 doubles) that every device which loads
   the library keeps until the process exits.
     U          device pointer to a state (layout above) of `precision` (DH_F32 or DH_F64)
     n_cells    nx*ny*nz, at most 268435456 (4096 blocks of 65536 cells); larger or < 1 is
                DH_ERR_ARG with the limit in dh_last_error(NULL)
     totals_out device pointer to 5 doubles (rho, m_x, m_y, m_z, E), caller-owned
     cuda_stream cudaStream_t on which the work is ordered (NULL = legacy default stream)
   Asynchronous: the result is ready when the stream reaches this point.  A call on a stream
   that is not being captured looks the array's device address up (cudaGetSymbolAddress) and
   caches it per device; a call on a stream under capture uses the cached address, so make one
   call on the device before capturing (and again after a cudaDeviceReset).  All calls share the array, which
   keeps the last call's contents (every slot a call reads is written earlier in the same call);
   calls whose kernels overlap on the GPU race on it and may return wrong sums. */
dh_status dh_conserved_totals_static(const void* U, int precision, long long n_cells,
                                     double* totals_out, void* cuda_stream);

/* Profiling: when enabled, device time of every kernel launch is accumulated per kernel kind
   with CUDA events on the context stream.  dh_profile_read returns, for kernel kind `kind`
   (see DH_KERNEL_*), the number of launches and their total milliseconds since the last
   enable.  dh_launch_count returns the number of library kernels launched since creation. */
enum {
  DH_KERNEL_STAGE1 = 0, DH_KERNEL_STAGE2 = 1, DH_KERNEL_PROLOGUE = 2, DH_KERNEL_REDUCE = 3,
  DH_KERNEL_SOURCES = 4, DH_KERNEL_MG = 5, DH_KERNEL_ADJOINT = 6, DH_KERNEL_CONV = 7,
  DH_KERNEL_KINDS = 8
};
dh_status dh_profile_enable(dh_ctx* ctx, int enable);
dh_status dh_profile_read(dh_ctx* ctx, int kind, long long* launches, double* total_ms);
dh_status dh_launch_count(dh_ctx* ctx, long long* launches);

/* Message of the most recent failure on ctx (or of the last failed dh_create when ctx is
   NULL); owned by the library, valid until the next call on the same context. */
const char* dh_last_error(const dh_ctx* ctx);

/* Name of a status code. */
const char* dh_status_string(dh_status s);

#ifdef __cplusplus
}
#endif
#endif /* DH_H */
