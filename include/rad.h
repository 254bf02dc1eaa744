/*
 * rad.h -- C ABI of the GB300 finite-solid-angle GR radiation library.
 *
 * The library advances the gray specific intensity I(x, n) of White et al.,
 * "General Relativistic Radiation with a Finite-Solid-Angle Method" (2023),
 * on one logically rectangular block of cells held on one GPU:
 *   - Sec. 2.6:      geodesic and latitude-longitude angle grids
 *                    (rad_init_angles, rad_init_angles_latlong, rad_get_angles)
 *   - Secs. 2.1-2.2: metric, normal-observer tetrad, Ricci rotation
 *                    coefficients, exact cell volumes (rad_set_metric)
 *   - Secs. 2.3-2.4, Eq. radiation_integral: reconstruction, upwind spatial
 *                    and angular fluxes, flux divergence (rad_step)
 *   - Sec. 2.5:      locally implicit coupling via a quartic for T (rad_step)
 *   - Sec. 2.4:      n0crit guard (rad_step)
 *   - Sec. 2.5:      R^{mu nu} = sum I n^mu n^nu dOmega (rad_moments)
 *   - gradient of an outgoing-flux loss through a step (rad_step_adjoint,
 *     rad_loss_outer)
 *
 * Conventions shared by every call
 *   - Status: every int-returning call returns RAD_OK (0) or a negative
 *     rad_status.  rad_last_error() gives a message for the last failure of
 *     that context.  No C++ exception crosses this interface.
 *   - Memory: the caller owns every buffer it passes (device pointers unless
 *     stated "host"), contiguous, at least 16-byte aligned; the library
 *     never frees them.  The context owns its tables and scratch.
 *   - Streams: all device work is enqueued on the stream given to
 *     rad_create (NULL = legacy default stream).  Calls are asynchronous
 *     except rad_init_angles(_latlong), rad_get_angles, rad_set_metric, rad_cfl_dt and
 *     rad_check, which synchronise that stream.
 *   - Device errors (non-finite intensity, unbracketed quartic, divergent
 *     Newton iteration) set a sticky error word in device memory instead of
 *     trapping; rad_check reads and clears it.
 *   - Intensity layout: I[k][j][i][n] for k < n[2], j < n[1], i < n[0],
 *     n < n_ang_padded (angle fastest).  Bins n >= n_ang are padding: their
 *     values are never used, and rad_step writes them as 0.  Element type is
 *     double (RAD_F64) or
 *     float (RAD_F32).  A block may hold at most 2^32 elements.  There are no
 *     ghost cells in the array: boundary
 *     conditions are applied by index mapping when neighbours are read.
 *   - Coordinates are (x1, x2, x3); for spherical metrics (r, theta, phi).
 */
#ifndef RAD_H
#define RAD_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rad_ctx rad_ctx;

typedef enum {
  RAD_OK = 0,
  RAD_EINVAL = -1,        /* bad argument (checked on the host, nothing enqueued) */
  RAD_ENOMEM = -2,        /* device or host allocation failed */
  RAD_ECUDA = -3,         /* a CUDA runtime call failed */
  RAD_ENOCONV = -4,       /* quartic without a bracketed root / Newton cap hit */
  RAD_ENONFINITE = -5,    /* a non-finite intensity or temperature was produced */
  RAD_ESTATE = -6,        /* call out of order (e.g. step before set_metric) */
  RAD_EUNSUPPORTED = -7   /* a valid request the library does not implement */
} rad_status;

enum { RAD_MINK_CART = 0, RAD_MINK_SPH = 1, RAD_KS_SPH = 2 };
enum { RAD_BC_PERIODIC = 0, RAD_BC_OUTFLOW = 1, RAD_BC_POLAR = 2,
       RAD_BC_HALO = 3   /* face shared with another block: ghosts from a halo buffer (rad_step_stage) */ };
enum { RAD_F64 = 0, RAD_F32 = 1 };
enum { RAD_RECON_DC = 0, RAD_RECON_PLM = 1, RAD_RECON_PPM = 2, RAD_RECON_MAPR = 3 /* angular only */ };
enum { RAD_COUPLE_THERMAL = 0, RAD_COUPLE_EMISSIVITY = 1, RAD_COUPLE_NONE = 2 };
enum { RAD_FRAME_TETRAD = 0, RAD_FRAME_COORD = 1, RAD_FRAME_FLUID = 2 };
enum { RAD_MOM_SIMT = 0, RAD_MOM_BF16X3 = 1 };

/* Create a context bound to a CUDA stream (cudaStream_t passed as void*). */
int rad_create(rad_ctx **out, void *cuda_stream);
/* Free the context, its tables and scratch.  NULL is ignored. */
void rad_destroy(rad_ctx *ctx);
/* Message of the last failing call on ctx ("" if none).  Owned by ctx. */
const char *rad_last_error(const rad_ctx *ctx);

/*
 * Build the level-N geodesic angle grid (Sec. 2.6: icosahedron, faces cut
 * flat into N^2 triangles, cells around the lattice vertices bounded by
 * great-circle arcs through the projected triangle centroids).
 * n_ang = 10 N^2 + 2; n_ang_padded rounds it up to a multiple of 4.
 * Orientation: a pentagon centred on +3hat, the 2hat axis a two-fold axis.
 * Bin numbering: the library's own (rad_get_angles gives each bin's
 * direction).  Bins 2t and 2t + 1 have no direction component of opposite
 * sign wherever the grid allows such a pairing (levels 3, 4, 5, 7, 8, 9,
 * ...); the flat-space stage kernels use it.
 * level must be in [1, 32].  Synchronous; replaces any previous grid (and
 * invalidates the metric, which must be set again).
 */
int rad_init_angles(rad_ctx *ctx, int level, int *n_ang_out, int *n_ang_padded_out);

/*
 * Latitude-longitude angle grid (Sec. 2.6) instead of the geodesic one:
 * n_zeta bands between latitude lines equally spaced in cos(zeta) from +1
 * to -1 (zeta measured from 3hat) and n_psi sectors between longitude lines
 * equally spaced in psi from 0 to 2 pi, n_ang = n_zeta n_psi cells of solid
 * angle 4 pi / n_ang.  Bin n = band * n_psi + sector; its direction lies
 * halfway between its lines in cos(zeta) and in psi.  Angular fluxes cross
 * the cell sides (meridian and latitude arcs, DC upwind as on the geodesic
 * grid); the poles carry none.  n_psi must be even and >= 4 (the pi
 * rotation about 2hat, used by polar boundaries, must map cells to cells),
 * n_zeta >= 1, n_ang <= 4096 (rad_step takes up to 812): RAD_EINVAL
 * otherwise.  Synchronous; invalidates the metric like rad_init_angles.
 */
int rad_init_angles_latlong(rad_ctx *ctx, int n_zeta, int n_psi, int *n_ang_out,
                            int *n_ang_padded_out);

/*
 * Copy the grid to host arrays (each may be NULL):
 *   dir[n_ang][3] unit directions (components on 1hat, 2hat, 3hat),
 *   dOmega[n_ang] exact spherical-polygon solid angles (sum 4 pi),
 *   nbr[n_ang][6] neighbour bins, -1 padding (the 12 pentagons of a
 *                 geodesic grid, every cell of a lat/long grid).
 */
int rad_get_angles(rad_ctx *ctx, double *dir, double *dOmega, int *nbr);

typedef struct {
  int kind;        /* RAD_MINK_CART, RAD_MINK_SPH or RAD_KS_SPH */
  double spin;     /* Kerr spin a (M = 1), |a| < 1; ignored for flat space */
} rad_metric;

typedef struct {
  int ndim;               /* dimensions carrying fluxes: 1, 2 or 3 */
  int n[3];               /* cells per dimension; n[d] = 1 for d >= ndim */
  const double *xf[3];    /* host face coordinates, n[d] + 1 increasing values;
                             xf[2] must be uniformly spaced */
  int bc_lo[3], bc_hi[3]; /* RAD_BC_*; polar only on x2 of a spherical metric,
                             which then needs theta faces at 0 / pi and an even
                             n[2] (or n[2] = 1) covering 2 pi in phi */
} rad_grid;

/*
 * Compute the per-cell and per-face geometry in FP64 (Secs. 2.1-2.2):
 * metric, normal-observer tetrad (Cartesian: identity; spherical:
 * theta -> 3hat, phi -> 1hat, r -> 2hat by Gram-Schmidt), Ricci rotation
 * coefficients (Eq. ricci) from exact forward-mode derivatives, exact
 * Delta V and Delta A.  Requires rad_init_angles.  Synchronous.
 */
int rad_set_metric(rad_ctx *ctx, const rad_metric *metric, const rad_grid *grid);

/* Gas state: device FP64 arrays over active cells, [k][j][i] (u: [k][j][i][3]). */
typedef struct {
  const double *rho;      /* rest-mass density (c_v = rho / (Gamma - 1)) */
  const double *u;        /* fluid four-velocity u^ihat in the tetrad frame */
  const double *alpha_a;  /* fluid-frame absorption coefficient (alpha_P = alpha_a) */
  const double *alpha_s;  /* fluid-frame scattering coefficient */
  const double *eta;      /* fluid-frame emissivity; only for RAD_COUPLE_EMISSIVITY */
  double *T;              /* gas temperature, updated in place by rad_step */
} rad_gas;

typedef struct {
  int precision;     /* RAD_F64 or RAD_F32: element type of I and of the
                        per-angle transport / coupling arithmetic; the
                        geometry, the quartic and the temperature are FP64 */
  int recon;         /* RAD_RECON_DC, RAD_RECON_PLM (van Leer) or RAD_RECON_PPM
                        (Colella & Woodward; three-cell stencil: polar
                        boundaries need n[1] >= 3; not in rad_step_adjoint) */
  int coupling;      /* RAD_COUPLE_THERMAL, _EMISSIVITY or _NONE */
  double n0crit;     /* guard threshold on |n_0| (Sec. 2.4), default 0.1 */
  int zero_guard;    /* apply the guard (default 1) */
  double a_rad;      /* radiation constant, default 1 */
  double gamma;      /* adiabatic index, default 5/3 */
  double tau_const;  /* C of the optical-depth weighting of the spatial fluxes
                        (Sec. 2.4): tau = C alpha_E dt / u^0hat at each face,
                        f = -expm1(-tau^2), upwind state times (1 - g_up + g)
                        with g_L/R = -f (1 + 1/n^0bar_L/R) and g their face
                        average; u and alpha_E = alpha_a + alpha_s are face
                        averages of the two cells.  0 (default) is the
                        free-streaming flux.  > 0 needs gas u, alpha_a and
                        alpha_s; rad_step_adjoint requires 0. */
  int rad_dom;       /* 1: radiation-dominated velocity substitution (end of
                        Sec. 2.5) in every coupling: where the fluid-frame
                        radiation energy exceeds rho + u_gas the coupling
                        runs at u^a = (1 - f^a) u_gas^a + f^a u_rad^a, with
                        u_rad from v_rad^a = R^{0a}/R^{00} and
                        f^a = G^a dt / (T_rad^{0a} - T_gas^{0a}) clamped to
                        [0, 1] (read without the printed extra factor u^a).
                        Needs RAD_COUPLE_THERMAL; each stage then runs the
                        transport and the coupling as two kernels.  Default 0;
                        rad_step_adjoint requires 0. */
  int recon_ang;     /* angular reconstruction: RAD_RECON_DC (default; the
                        geodesic grid's scheme, Sec. 2.6), RAD_RECON_PLM:
                        the spatial PLM applied along the lines of a
                        latitude-longitude grid (bands along a side of
                        constant psi, sectors through both poles for a
                        side of constant zeta; RAD_EUNSUPPORTED on a
                        geodesic grid), or RAD_RECON_MAPR: minimum-angle
                        plane reconstruction on a geodesic grid (Sec. 2.6
                        names it; here each bin keeps the least inclined of
                        the planes through itself and two cyclically
                        adjacent neighbours in its gnomonic tangent plane,
                        evaluated at the side midpoints; RAD_EUNSUPPORTED on
                        a latitude-longitude grid).  rad_step_adjoint takes
                        all three. */
} rad_opts;

/* Fill *opts with the defaults above (FP64, PLM, thermal coupling). */
void rad_opts_default(rad_opts *opts);

/*
 * dt = cfl * min(dt_space, dt_angle): dt_space = min over cells, flux
 * dimensions and bins of dx^d / |n^d / n^0|; dt_angle = min over cells and
 * bins of dOmega n^0 / sum_edges l_e |V . nu_e|.  Synchronous.
 */
int rad_cfl_dt(rad_ctx *ctx, double cfl, double *dt_out);

/*
 * One SSP-RK2 step of Eq. radiation_integral with the Sec. 2.5 coupling
 * after each stage (dt, then dt/2; the gas T entering stage 2 is the
 * average of T before and after stage 1) and the n0crit guard after each
 * coupling.  I (device, layout above) and gas->T are updated in place.
 * gas_src (device [k][j][i][4], nullable) receives -(dR^1/2 + dR^2), the
 * RK-weighted change of R^0_mu from the two couplings (the gas's share).
 * Allocates its stage scratch (one intensity array) on first use.
 * Geodesic levels up to 9 (812 bins: one CTA of at most 512 threads holds
 * every bin of a cell) and fewer than 2^32 intensity elements per block;
 * RAD_EUNSUPPORTED otherwise.
 */
int rad_step(rad_ctx *ctx, void *I, const rad_gas *gas, double dt,
             const rad_opts *opts, double *gas_src);

/*
 * rad_step without any device allocation (the paper has no counterpart; this
 * is a service of this library).  For callers that may not allocate device
 * memory once running: a host framework that owns all device memory through
 * its own pool, or a loop that cannot take the implicit synchronisation of
 * cudaMalloc / cudaFree.  Same arguments, options (every recon, recon_ang,
 * tau_const, rad_dom and coupling that rad_step takes), host-side checks,
 * kernels and results (bit for bit) as rad_step, but the stage scratch (one intensity array and one temperature
 * array) lives in a 32 MiB static device array that every GPU loading this
 * library holds until the process exits.  Grids needing more
 * (n_cells * n_ang_padded * element size, rounded up to 256 bytes, plus
 * 8 bytes per cell) are refused with RAD_EINVAL.  Calls share that array:
 * calls that overlap on the GPU (other streams or contexts on the same
 * device) race.  The first call on a device, with that device current, looks
 * up the array's device address; make that first call before any stream
 * capture.  Calls no cudaMalloc or cudaFree.  Gray transport only: a
 * context with groups set (rad_set_groups) gives RAD_EUNSUPPORTED.
 */
int rad_step_noalloc(rad_ctx *ctx, void *I, const rad_gas *gas, double dt,
                     const rad_opts *opts, double *gas_src);

/*
 * Gas update from the step's radiation source (end of Sec. 2.5: the change
 * of R^0_mu produced by the coupling is taken from the gas).  rho, u
 * ([cell][3], tetrad-frame u^ihat) and T (device FP64, per cell of this
 * context's grid) hold the gas state the step started from (keep a copy of
 * gas->T before rad_step, which overwrites it) and receive the state after
 * the source: T^0_mu = w u^0 u_mu + p delta^0_mu (ideal gas, p = rho T,
 * w = rho + gamma p / (gamma - 1)) gains src_mu, summed over n_src arrays
 * [n_src][cell][4] (rad_step's gas_src; n_src = n_groups for multigroup),
 * while rho u^0 is kept, and (rho, u, T) are recovered from the new
 * conserved state (one pressure equation per cell, solved in FP64).  A
 * cell whose new state is not physical (E <= (S^2 + D^2)^(1/2) in the
 * normal observer's frame) is left unchanged and sets the sticky
 * RAD_ENOCONV.  1 < gamma <= 2.  Asynchronous.
 */
int rad_gas_update(rad_ctx *ctx, double *rho, double *u, double *T, const double *src, int n_src,
                   double gamma);

/*
 * Multigroup transport (Sec. 2.2, Eq. radiation_integral_frequency): the
 * intensity is resolved in n_groups intervals of the tetrad-frame
 * frequency, nu_edges[0] < ... < nu_edges[n_groups] (host array; the first
 * >= 0, every edge finite except possibly the last, which may be +inf).
 * Each group's intensity (the integral of I_nu over its interval) takes the
 * gray spatial and angular fluxes plus the difference of the frequency
 * fluxes n^nu n_0 I_nu at its edges, n^nu = -nu omega^0hat_{AB} n^A n^B
 * (cell-centre geometry), donor cell in frequency: the upwind group's mean
 * I_g / dnu_g, the lower group where n^nu > 0, the upper where n^nu < 0; the
 * end edges pass radiation out of the resolved range and none in, and an
 * edge at 0 or infinity carries nothing.  While groups are set:
 *   - rad_step takes I as [n_groups][n3][n2][n1][n_ang_padded], gas->alpha_a,
 *     alpha_s and eta as [n_groups][n3][n2][n1] (rho, u and T per cell as
 *     before) and gas_src as [n_groups][n3][n2][n1][4];
 *   - coupling is RAD_COUPLE_EMISSIVITY (each group coupled on its own with
 *     the gray formulas; the gas temperature stays fixed) or
 *     RAD_COUPLE_NONE; RAD_COUPLE_THERMAL and rad_dom give RAD_EUNSUPPORTED,
 *     as do rad_step_stage, rad_step_noalloc, rad_step_host and
 *     rad_step_adjoint;
 *   - rad_cfl_dt also bounds dt by n^0 dnu_g / (nu_{g+1} |omega^0hat n n|) for
 *     every finite group;
 *   - rad_moments and rad_loss_outer take one group's array at a time.
 * n_groups = 0 returns to gray transport.  One group spanning [0, inf) is
 * the gray step.  Synchronous.
 */
int rad_set_groups(rad_ctx *ctx, int n_groups, const double *nu_edges);

/*
 * Decomposed domains (the task list of Sec. 2: a block's fluxes need its
 * neighbours' cells next to every shared face, exchanged before each
 * stage; Sec. 5 runs one block per GPU).  A context holds one block: its
 * rad_grid gives the block's own cells and face coordinates, and
 * RAD_BC_HALO on every face it shares with another block (a face of the
 * whole domain keeps its own boundary kind; a periodic direction split into
 * blocks becomes RAD_BC_HALO on the wrapped faces).  A block needs at least
 * 3 cells across a shared face; a block touching a polar axis must hold the
 * whole phi range.  rad_step refuses such blocks: they step one stage at a
 * time so that the halos of the stage-1 result can be exchanged:
 *
 *   for each shared face f: rad_halo_pack(ctx, I, prec, d, side, send[f])
 *   exchange: the neighbour across f receives send[f] as its halo of the
 *             opposite face (same layout, layer 0 next to the shared face)
 *   rad_step_stage(ctx, 1, I, gas, dt, opts, src, halo)
 *   for each shared face f: rad_halo_pack(ctx, NULL, prec, d, side, send[f])
 *   exchange
 *   rad_step_stage(ctx, 2, I, gas, dt, opts, src, halo)
 *
 * which computes, cell by cell, exactly what rad_step computes on the whole
 * domain.  The time step is the minimum of every block's rad_cfl_dt.  The
 * optical-depth weighting (it reads the neighbour's gas) and the adjoint
 * take single blocks only (RAD_EUNSUPPORTED).
 */
/*
 * One SSP-RK2 stage of rad_step.  stage 1: I (I^0, not modified) and gas->T
 * -> the context's stage scratch (I^1, T^1; allocated on first use like
 * rad_step's).  stage 2: the scratch and I -> I^2 written over I, T^2 over
 * gas->T, and gas_src as rad_step (stage 1 writes its half, stage 2 adds its
 * share).  halo: 6 device pointers, face (d, side) at 2 d + side, each the
 * ghost layers of a RAD_BC_HALO face of the stage's input (I for stage 1,
 * the stage-1 result for stage 2) in rad_halo_pack's layout; entries of
 * other faces are ignored (halo may be NULL when there are none).  Stage 2
 * must follow a stage 1 of the same precision on this context.  Same
 * options, checks and arithmetic as rad_step otherwise.
 */
int rad_step_stage(rad_ctx *ctx, int stage, void *I, const rad_gas *gas, double dt,
                   const rad_opts *opts, double *gas_src, const void *const *halo);

/*
 * Copy the 3 layers of an intensity array next to face (dim, side) of this
 * block into buf (device, 16-byte aligned), layer 0 adjacent to the face:
 *   dim 0: buf[3][n3][n2][n_ang_padded]   dim 1: buf[3][n3][n1][n_ang_padded]
 *   dim 2: buf[3][n2][n1][n_ang_padded]
 * I = NULL packs the context's stage-1 result (after rad_step_stage(.., 1, ..)
 * of this precision).  dim must carry fluxes and have >= 3 cells.
 * Asynchronous.
 */
int rad_halo_pack(rad_ctx *ctx, const void *I, int precision, int dim, int side, void *buf);

/*
 * Moments R^{AB} = sum_n I_n n^A n^B dOmega_n of every cell, written as 10
 * components [cell][10] in the order 00 01 02 03 11 12 13 22 23 33.
 * precision: element type of I (and of R for RAD_MOM_BF16X3, which writes
 * float).  frame: tetrad, coordinate (e e R) or fluid (Lambda Lambda R,
 * needs gas->u).  method: RAD_MOM_SIMT (CUDA cores, I's precision) or
 * RAD_MOM_BF16X3 (RAD_F32 only: tensor cores, I and the weights split into
 * bf16 hi + lo, three products, FP32 accumulation).
 */
int rad_moments(rad_ctx *ctx, const void *I, int precision, int frame, int method,
                const rad_gas *gas, void *R);

/*
 * Host-resident data (the paper has no counterpart; it takes the fields to
 * be resident on the device).  One item is one problem on this context's
 * grid: its intensity and gas state in host memory (same layouts and
 * precisions as for rad_step; I is not modified), and host buffers for the
 * results.
 */
typedef struct {
  const void *I;          /* [n3][n2][n1][n_ang_padded], opts->precision */
  const double *rho, *u, *alpha_a, *alpha_s;
  const double *eta;      /* only for RAD_COUPLE_EMISSIVITY */
  double *T;              /* in/out: the gas temperature after the steps */
  void *R;                /* out: [k][j][i][10] moments (FP64 for RAD_F64, FP32 for RAD_F32) */
  void *I_out;            /* out, nullable: the intensity after the steps */
} rad_host_item;

/*
 * For each of n_items items: copy I and the gas state to the device, take
 * nsteps rad_step steps (no gas source), contract with rad_moments (frame,
 * method as there), and copy R, T (and I_out if given) back.  Three device
 * slots owned by the context rotate (item i in slot i mod 3); uploads,
 * moment contractions and read-backs run on three streams of their own, so
 * that the uploads of the next two items and the contraction and read-back
 * of the previous one overlap the steps of item i (the copies hide when the
 * host buffers are pinned).  Items in flight together are independent: an
 * output array (T, R, I_out) of one item must not be an array of another
 * item among the two before or after it (inputs may be shared).
 * Synchronous: returns when every result is in host memory.  Errors as rad_step / rad_moments; a null host array of an
 * item is RAD_EINVAL and nothing is enqueued.
 */
int rad_step_host(rad_ctx *ctx, int n_items, const rad_host_item *items, double dt,
                  const rad_opts *opts, int nsteps, int frame, int method);

/*
 * Reverse-mode step: given the state I_n (checkpoint, not modified), the gas
 * state gas->T = T_n, and the adjoints lam_np1 = dL/dI_{n+1} and
 * lamT_np1 = dL/dT_{n+1}, write lam_n = dL/dI_n and lamT_n = dL/dT_n and
 * ACCUMULATE (+=) dL/dalpha_a, dL/dalpha_s, dL/deta (device FP64 [k][j][i])
 * through the step rad_step would take from (I_n, T_n).  With
 * RAD_COUPLE_THERMAL the gradient runs through the root of the quartic of
 * Sec. 2.5 (implicit-function theorem) and through the temperature between
 * the stages; with RAD_COUPLE_EMISSIVITY or RAD_COUPLE_NONE the temperature
 * is frozen and lamT_n = lamT_np1.  With opts->tau_const > 0 (the
 * optical-depth weighting of Sec. 2.4) the opacity gradients include the
 * path through the face weights.  Any spatial reconstruction (DC, PLM, PPM)
 * and any angular one (DC, line PLM, MAPR), the limiters and the plane choice
 * differentiated on their active branches.  With rad_dom = 1 the gradient
 * also runs through the substituted velocity (the radiation velocity, the
 * momentum fractions on their unclamped range, the trigger held fixed) into
 * the intensities, the temperature and the opacities.  lam arrays use the intensity
 * layout and precision; lamT arrays are device FP64 [k][j][i].  lamT_np1 may
 * be NULL (zero), lamT_n may be NULL (not written) and may equal lamT_np1;
 * g_eta may be NULL.
 */
int rad_step_adjoint(rad_ctx *ctx, const void *I_n, const rad_gas *gas, double dt,
                     const rad_opts *opts, const void *lam_np1, void *lam_n,
                     const double *lamT_np1, double *lamT_n,
                     double *g_alpha_a, double *g_alpha_s, double *g_eta);

/*
 * Outgoing-flux loss L = sum_{k,j} sum_{n: n^1 > 0 at the outer x1 face}
 * I[k][j][n1-1][n] dOmega_n, written to *L_dev (device double); if dL_dI is
 * not NULL it receives dL/dI (the seed of rad_step_adjoint).
 */
int rad_loss_outer(rad_ctx *ctx, const void *I, int precision, double *L_dev, void *dL_dI);

/* Read and clear the sticky device error word.  Synchronous.  Returns
 * RAD_OK or one recorded status, in this order: RAD_ECUDA (a bounded device
 * wait gave up), RAD_ENOCONV (a quartic without a bracketed root, or a gas
 * update that did not converge), RAD_ENONFINITE (a non-finite intensity),
 * RAD_ESTATE (a flat-space stage met a bin pair with opposite upwind sides,
 * which the library's bin numbering excludes). */
int rad_check(rad_ctx *ctx);

/* Self-test of the bounded device waits (no paper counterpart): enqueue a
 * kernel that waits on an mbarrier nothing arrives at; after `seconds`
 * (0 < seconds <= 10) the wait gives up and records the timeout bit that the
 * stage and moment kernels record, so that the next rad_check returns
 * RAD_ECUDA ("a device wait timed out").  The context stays usable.
 * Asynchronous; RAD_EINVAL for a bad duration. */
int rad_selftest_wait(rad_ctx *ctx, double seconds);

/* Measured FP64 fused multiply-add rate of the current device, in TFLOP/s
 * (no paper counterpart: the denominator for the FP64 stage kernels, which
 * the FP64 pipe bounds rather than HBM).  Every SM runs independent DFMA
 * chains; the best of three launches of about seconds/3 each (CUDA events)
 * is returned.  0 < seconds <= 30.  Synchronous, on the legacy default
 * stream; allocates and frees a small output buffer.  Reads no clock or
 * setting of the GPU and changes none. */
int rad_fp64_fma_rate(double seconds, double *tflops_out);

#ifdef __cplusplus
}
#endif
#endif /* RAD_H */
