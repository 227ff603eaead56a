/*
 * emm.h -- C ABI of the B300 fictitious-wave-domain FDTD library (libemm).
 *
 * The library advances the diffusive Maxwell equations transformed to the
 * fictitious wave domain (Yang, libEMM, arXiv 2304.00233, Sec. 2.2 Eq. 3-5)
 * with a 2r-th order staggered leapfrog on a non-uniform rectilinear grid
 * (Sec. 3.1 Eq. 8, 13-14), CPML absorbing layers (Sec. 3.4 Eq. 22-24), an
 * electric dipole source, and an on-the-fly DTFT (Sec. 3.5 Eq. 25) that yields
 * frequency-domain Green's functions (Sec. 2.2 Eq. 7) at receivers and,
 * optionally, over the model volume.  The time loop runs in CUDA kernels on
 * one GPU (sm_103a).
 *
 * Conventions shared by every entry point
 *   - Axes are x, y, z (index 0, 1, 2); z is positive down.  Every 3-D array
 *     is C order [n3][n2][n1] with x fastest (Sec. 3.8).
 *   - Field components are numbered 0..5 = Ex, Ey, Ez, Hx, Hy, Hz on the Yee
 *     grid: Ex at (x_{i+1/2}, y_j, z_k), Ey at (x_i, y_{j+1/2}, z_k),
 *     Ez at (x_i, y_j, z_{k+1/2}), Hx at (x_i, y_{j+1/2}, z_{k+1/2}),
 *     Hy at (x_{i+1/2}, y_j, z_{k+1/2}), Hz at (x_{i+1/2}, y_{j+1/2}, z_k).
 *   - The model (n1 x n2 x n3 nodes) is padded with ne buffer layers and nb
 *     CPML layers on every face: npad = n + 2 (nb + ne) (Sec. 3.4).  Pads
 *     repeat the edge spacing; half nodes are midpoints.  The grid holds
 *     integer samples 0..npad-1 and half samples 0..npad-2.
 *   - All functions return EMM_OK (0) or one of the EMM_E* codes below.  No
 *     C++ exception crosses the ABI.  Functions are thread-safe for distinct
 *     grids and distinct workspaces.
 *   - "host" pointers are ordinary CPU memory owned by the caller; "device"
 *     pointers are CUDA global memory owned by the caller.  The library never
 *     allocates or frees device memory.
 */
#ifndef EMM_H
#define EMM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ------------------------------------------------------- */
#define EMM_OK 0
#define EMM_EINVAL 1      /* invalid argument (sizes, ranges, NULL, non-monotone nodes) */
#define EMM_ENOMEM 2      /* host allocation failed */
#define EMM_EOUTSIDE 3    /* a source/receiver stencil leaves the non-CPML region */
#define EMM_ECFL 4        /* dt > 1/eta: the leapfrog would be unstable (Sec. 3.2) */
#define EMM_ECUDA 5       /* a CUDA runtime call or kernel launch failed */
#define EMM_EWORKSPACE 6  /* workspace too small or misaligned */
#define EMM_EDEVICE 7     /* the device flagged a bad input (see emm_status) */
#define EMM_ETIMEOUT 8    /* a bounded device-side wait ran out (see emm_status) */

/* Opaque grid handle: padded nodes, half nodes, FD tables (host, FP64).
 * Immutable after emm_make_grid; owns no device memory. */
typedef struct emm_grid emm_grid;

/* CUDA stream handle (layout-compatible with cudaStream_t); NULL = default stream. */
typedef struct CUstream_st *emm_stream;

typedef struct {
  int n[3];            /* interior node counts along x, y, z; each >= 2 */
  const double *x[3];  /* host: strictly ascending node coordinates (m), n[a] each */
  int rd;              /* FD half length r, order 2r: 1..4 (Sec. 3.1, 5.7) */
  int nb;              /* CPML layers per face, rd <= nb */
  int ne;              /* buffer layers between CPML and model, >= 0 */
} emm_grid_desc;

typedef struct {
  int n[3];            /* interior node counts */
  int npad[3];         /* padded sample counts n + 2 (nb + ne) */
  int rd, nb, ne;
  size_t cells;        /* npad[0] * npad[1] * npad[2] */
} emm_grid_info;

/* Build a grid: pads the nodes (Sec. 3.4), forms half nodes, and tabulates
 * the D+ / D- rows of every sample (row 1 of [V^T]^{-1}, Sec. 3.1 Eq. 9-14).
 * desc (host, read only during the call).  *out receives a handle that the
 * caller releases with emm_free_grid.  EMM_EINVAL for bad sizes, rd outside
 * 1..4, nb < rd, ne < 0, or non-ascending nodes; EMM_ENOMEM. */
int emm_make_grid(const emm_grid_desc *desc, emm_grid **out);

/* Release a grid (NULL is a no-op). */
void emm_free_grid(emm_grid *grid);

/* Sizes of a grid.  EMM_EINVAL on NULL arguments. */
int emm_grid_query(const emm_grid *grid, emm_grid_info *info);

/* Table kinds for emm_grid_tables. */
#define EMM_TAB_NODES 0      /* coef[npad+1]: padded integer nodes X (X[npad] only bounds the last half cell) */
#define EMM_TAB_HALF 1       /* coef[npad]: half nodes Xh[i] = (X[i] + X[i+1]) / 2 */
#define EMM_TAB_DPLUS 2      /* coef[npad][2rd]: D+ rows at Xh[i] over F[i-rd+1 .. i+rd] (Eq. 13);
                                idx[npad]: first tap i-rd+1, or -1 where the row is off the grid */
#define EMM_TAB_DMINUS 3     /* coef[npad][2rd]: D- rows at X[i] over half samples F[i-rd .. i+rd-1] (Eq. 14);
                                idx[npad]: first tap i-rd, or -1 */
#define EMM_TAB_SLAB_INT 4   /* idx[npad]: CPML slab entry 0..2nb-1 of integer sample i, or -1 */
#define EMM_TAB_SLAB_HALF 5  /* idx[npad]: CPML slab entry 0..2nb-1 of half sample i, or -1 */

/* Copy one table of axis `axis` (0..2) into host arrays (either may be NULL
 * when the kind does not fill it).  Used by the index-map parity tests.
 * EMM_EINVAL on a bad axis or kind. */
int emm_grid_tables(const emm_grid *grid, int axis, int kind, double *coef, int *idx);

/* Time step of the stability condition (Sec. 3.2 Eq. 15-16):
 * vmax = sqrt(2 omega0 / (mu0 sigma_min)), eta = vmax/2 sqrt(sum_a Dmax_a^2),
 * Dmax_a = largest absolute row sum of the D+ and D- tables of axis a.
 * *dt = 0.99 / eta; *eta and *vmax (both may be NULL) receive the others.
 * EMM_EINVAL if sigma_min or omega0 is not positive. */
int emm_time_step(const emm_grid *grid, double sigma_min, double omega0,
                  double *dt, double *eta, double *vmax);

/* CPML coefficients of axis `axis` for a given vmax, fmax and dt (Eq. 23-24,
 * kappa = 1, profile d = d0 (xi/L)^2 with d0 = -3 vmax ln(1e-3) / (2L),
 * alpha = pi fmax (1 - xi/L)); ab (host) receives [4][2nb]:
 * a at integer samples, b at integer samples, a at half samples, b at half
 * samples, indexed by slab entry (EMM_TAB_SLAB_*).  EMM_EINVAL on bad input. */
int emm_cpml_tables(const emm_grid *grid, int axis, double vmax, double fmax,
                    double dt, double *ab);

/* Stencil of a point source/receiver for component comp (0..5) at pos[3]
 * (m): along each axis, on the component's own node array P, i = max{i :
 * P[i] <= p}; knots i-rd+1 .. i+rd; start[a] = i-rd+1; w (host, [3][2rd])
 * receives the Lagrange interpolation weights (row 0 of [V^T]^{-1}, Sec. 3.1).
 * EMM_EOUTSIDE if a knot falls in a CPML slab or off the grid. */
int emm_locate(const emm_grid *grid, int comp, const double pos[3], int start[3], double *w);

/* One transmitter and its receivers. */
typedef struct {
  double omega0;        /* rad/s, > 0: fictitious permittivity eps = sigma / (2 omega0) (Eq. 3) */
  double fmax;          /* Hz, > 0: Gaussian wavelet exp(-(pi fmax (t - 1.5/fmax))^2) and CPML alpha */
  double sigma_min;     /* S/m, > 0: smallest conductivity in the model (sets vmax) */
  double dt;            /* s: time step; <= 0 selects 0.99/eta; > 1/eta is EMM_ECFL */
  int nt;               /* number of leapfrog steps, >= 0 (with 0 no step runs, J' of Eq. 7 is 0
                           and every Green's function is returned as 0) */
  double src[3];        /* source position (m) */
  double src_az;        /* rad: azimuth of the electric dipole */
  double src_dip;       /* rad: dip; direction (cos dip cos az, cos dip sin az, sin dip) */
  double moment;        /* A m: dipole moment (Green's functions do not depend on it) */
  int nrec;             /* >= 0 */
  const double *rec;    /* host [nrec][3] receiver positions (m) */
  int nfreq;            /* >= 1 */
  const double *freqs;  /* host [nfreq] frequencies (Hz, > 0) */
  int volume;           /* 1: also accumulate the DTFT of all six components on
                           every interior sample (the n1 x n2 x n3 samples of each
                           component's own staggered positions) */
  int src_kind;         /* 0: electric dipole J, injected in the E update at
                           t_{n+1/2}; outputs G^EE = sqrt(-i w/(2 w0)) E'/J' and
                           G^HE = H'/J' (Eq. 7).  1: magnetic dipole M (Eq. 1),
                           on the H samples, injected in the H update at t_{n+1}
                           (mu dH/dt = -(curl E + M)); outputs, from the
                           correspondence of Eq. 5 (E' = E, H' = sqrt(-i w/(2 w0)) H,
                           M' = M), G^EH = E'/M' and G^HH = H'/(sqrt(-i w/(2 w0)) M').
                           Same orientation (src_az, src_dip) and wavelet. */
  double src_length;    /* m, >= 0.  0: a point dipole at src.  > 0: an antenna of
                           this length along the dipole direction, centred at src,
                           carrying the moment spread evenly over src_points
                           sub-dipoles at the midpoints of equal segments (the
                           paper's uniformly distributed current, Sec. 7) */
  int src_points;       /* 1 .. 256 sub-dipoles when src_length > 0 */
  int airwave;          /* 1: air above the top interior node (Sec. 3.3): no CPML
                           on the top face; after every E update E_x, E_y on the
                           rd-1 integer rows above the interface, and after every
                           H update H_x, H_y on the rd half rows above it, are the
                           harmonic continuation of the interface plane (per
                           horizontal wavenumber k: e^{-|k| h} at height h, and
                           H_x,y = i k_x,y / |k| H_z, shifted to their own x-y
                           positions), through the 2-D DFT of the padded plane.
                           Needs uniform x and y spacing (EMM_EINVAL) and source
                           stencils below the interface (EMM_EOUTSIDE).  An
                           electric point-dipole solve without the volume DTFT
                           runs the layers next to the interface and the air
                           transforms on a second stream of the library's (one per
                           host thread and device, of the greatest priority),
                           forked from `stream` and joined back to it within the
                           call: work enqueued on `stream` before and after is
                           ordered with all of it, as with one stream.
                           emm_forward_timed and convergence runs keep one stream. */
  int tile_shape;       /* stencil tile of one CTA of the E and H launches, 128
                           threads each: 0 = 32 x 8 x 2 cells (x, y, z), 1 =
                           32 x 4 x 4.  Used by emm_forward, emm_forward_timed,
                           emm_forward_static, emm_forward_batch and the plans;
                           convergence runs, gradients, work lists and the
                           wavefront take 0.  Results do not depend on it. */
} emm_survey;

/* Leapfrog steps of fields a one-transmitter solve with the volume DTFT
 * keeps: its half-steps write into a ring of EMM_VOLUME_RING field slots
 * (E and H), and one volume-DTFT launch adds that many steps' terms to each
 * accumulator (Eq. 25), in step order, so that the accumulators are read and
 * written once per EMM_VOLUME_RING steps. */
#define EMM_VOLUME_RING 8

/* Device workspace bytes emm_forward needs for this grid and survey
 * (fields, CPML memory, 1/eps, tables; with survey->volume the accumulators
 * and EMM_VOLUME_RING - 1 more copies of E and H, the field ring).
 * EMM_EINVAL on bad input. */
int emm_workspace_size(const emm_grid *grid, const emm_survey *survey, size_t *bytes);

/* Run the forward time loop (Algorithm 1 without the airwave step) on
 * `stream` and write the Green's functions.
 *   sigma    device float [3][n3][n2][n1]: staggered sigma_xx at Ex, sigma_yy
 *            at Ey, sigma_zz at Ez positions of the interior (Sec. 5.5); the
 *            pads replicate the edge values.  Every value must be finite,
 *            positive and >= survey->sigma_min (else the device status word
 *            reports EMM_EDEVICE and the outputs are undefined).
 *   ws       device workspace of at least emm_workspace_size bytes, 256-byte
 *            aligned; its contents on entry do not matter.
 *   rec_out  device double [nrec][6][nfreq][2]: (re, im) of G^EE (V/m per
 *            A m) for components 0..2 and G^HE (A/m per A m) for 3..5 (Eq. 7).
 *   vol_out  device double [6][nfreq][n3][n2][n1][2] when survey->volume, else
 *            ignored (may be NULL).
 * The call validates on the host, uploads tables with cudaMemcpyAsync, and
 * enqueues every kernel asynchronously; it returns before the GPU finishes.
 * Host-detected errors (EMM_EINVAL, EMM_EOUTSIDE, EMM_ECFL, EMM_EWORKSPACE)
 * enqueue nothing; EMM_ECUDA reports a failed runtime call or launch. */
int emm_forward(const emm_grid *grid, const emm_survey *survey, const float *sigma,
                void *ws, size_t ws_bytes, double *rec_out, double *vol_out,
                emm_stream stream);

/* Per-kernel timing of a forward run (the per-phase breakdown of Sec. 6,
 * Table 1, measured on the device). */
typedef struct {
  int every;       /* in: time the launches of every `every`-th step (>= 1) */
  int samples;     /* out: number of steps timed */
  double e_ms;     /* out: mean duration (ms) of one E half step: the E launch
                      and the source and air launches after it */
  double h_ms;     /* out: mean duration (ms) of one H half step: the H launch
                      and the source and air launches after it */
  double total_ms; /* out: duration (ms) of the whole enqueued forward run */
  double loop_ms;  /* out: duration (ms) of the time loop alone: every E and H
                      launch back to back, from the first to the last */
  double v_ms;     /* out: volume-DTFT time (ms) per leapfrog step: the
                      duration of the timed DTFT launches over the steps they
                      covered (0 when survey->volume is 0).  With the volume
                      DTFT one launch covers up to eight steps, and the timed
                      steps are the last steps of such launches. */
} emm_timing;

/* emm_forward, with CUDA events recorded on `stream` around the E and H
 * launches of every timing->every-th step, around the time loop and around
 * the whole run.  Same
 * arguments, outputs and errors as emm_forward; in addition it synchronises
 * `stream` before returning and fills *timing (host).  EMM_EINVAL if timing
 * is NULL or timing->every < 1. */
int emm_forward_timed(const emm_grid *grid, const emm_survey *survey, const float *sigma,
                      void *ws, size_t ws_bytes, double *rec_out, double *vol_out,
                      emm_stream stream, emm_timing *timing);

/* emm_forward with the paper's stopping rule (Sec. 4.1): after step 0, and
 * after every step it = 100, 200, ..., a one-warp kernel compares the DTFT of
 * the six components at the 8 corners of the model interior (the samples
 * nb+ne and nb+ne+n-1 of each axis) for the lowest frequency with its value
 * at the previous check.  The run has converged after step it when, at every
 * corner, the change is at most 1e-5 of the current value and that value is
 * nonzero; it then keeps nt_run = it + 1 steps, and every leapfrog launch
 * already enqueued returns at once.  At most survey->nt steps run.
 * The verdicts reach the host through mapped pinned host memory (allocated
 * and freed by the call: 8 bytes), polled with one chunk of launches enqueued
 * ahead, each poll bounded (EMM_ETIMEOUT after 600 s without progress; the
 * environment variable EMM_POLL_TIMEOUT_S, in seconds, lowers the bound, for
 * tests of that path).  On a poll timeout the call still drains `stream`
 * (the enqueued launches finish) before it returns EMM_ETIMEOUT.
 * Synchronous: returns with `stream` drained.  *nt_run (host) receives the
 * steps taken.  Arguments, workspace (emm_workspace_size) and outputs as
 * emm_forward, the outputs being those of emm_forward with nt = *nt_run.
 * EMM_EINVAL if nt_run is NULL; other errors as emm_forward. */
int emm_forward_converge(const emm_grid *grid, const emm_survey *survey, const float *sigma,
                         void *ws, size_t ws_bytes, double *rec_out, double *vol_out,
                         emm_stream stream, int *nt_run);

/* Read the device status word of a workspace after emm_forward: synchronises
 * `stream`, then *status = EMM_OK, EMM_EDEVICE (a sigma value was not finite,
 * not positive, or below sigma_min) or EMM_ETIMEOUT (a kernel gave up on a
 * bounded wait for its asynchronous copies and returned early; the outputs
 * are then undefined).  EMM_ECUDA if the copy fails. */
int emm_status(const void *ws, int *status, emm_stream stream);

/* Device workspace bytes emm_forward_batch needs for nsrc transmitters (one
 * shared dt/eps and table set, nsrc field and CPML state blocks).
 * EMM_EINVAL on bad input, nsrc < 1 or survey->volume set. */
int emm_batch_workspace_size(const emm_grid *grid, const emm_survey *survey, int nsrc, size_t *bytes);

/* emm_forward for nsrc transmitters on one grid and one conductivity, all
 * advanced in the same launches (the independent transmitters of a survey,
 * one MPI rank each in the paper's Sec. 5.3 set-up).  Each transmitter has
 * its own fields and CPML memory; dt/eps, the tables, the receivers, the
 * wavelet and the source orientation and moment (from `survey`) are shared.
 *   src_pos   host double [nsrc][3]: transmitter positions (survey->src is
 *             ignored); each must pass the checks of emm_locate.
 *   rec_out   device double [nsrc][nrec][6][nfreq][2].
 *   ws        device workspace of emm_batch_workspace_size bytes.
 * Other arguments, asynchrony and errors as emm_forward; no volume DTFT. */
int emm_forward_batch(const emm_grid *grid, const emm_survey *survey, int nsrc, const double *src_pos,
                      const float *sigma, void *ws, size_t ws_bytes, double *rec_out, emm_stream stream);

/* Forward-solve plan: the time loop of emm_forward for one grid, survey,
 * workspace and outputs, captured once as a CUDA graph (every stencil,
 * source, air and volume launch with its dependent-launch edges) and
 * replayed by emm_plan_run for each conductivity.  The paper has no
 * counterpart; it removes the per-launch host work of a solve (2 nt + more
 * launches) for callers that solve the same survey many times.
 *   emm_plan_create: validates like emm_forward, enqueues one set-up on
 *     `stream` (with `sigma`; the launch parameters the graph keeps come
 *     from it), captures the loop and instantiates the graph; the loop is
 *     not run.  The plan keeps copies of the survey's arrays; `grid`, `ws`,
 *     `rec_out` and `vol_out` must stay valid (and are reused) for the
 *     plan's life.  EMM_ECUDA if capture or instantiation fails.
 *   emm_plan_run: the solve for `sigma` (device float [3][n3][n2][n1]) on
 *     `stream`: set-up, graph launch, normalisation; rec_out and vol_out
 *     receive exactly what emm_forward writes.  Asynchronous; emm_status on
 *     ws reads its device status.
 *   emm_plan_destroy: releases the plan (a run in flight completes).
 * A plan and the work-list entry points (emm_forward_jobs, emm_jobs_tune)
 * may be used in one process in either order. */
typedef struct emm_plan emm_plan;
int emm_plan_create(const emm_grid *grid, const emm_survey *survey, const float *sigma, void *ws,
                    size_t ws_bytes, double *rec_out, double *vol_out, emm_stream stream, emm_plan **plan);
int emm_plan_run(emm_plan *plan, const float *sigma, emm_stream stream);
void emm_plan_destroy(emm_plan *plan);

/* One problem of a work-list solve: a grid, a survey (one transmitter),
 * its conductivity and its receiver output, as emm_forward takes them. */
typedef struct emm_job {
  const emm_grid *grid;
  const emm_survey *survey;
  const float *sigma;  /* device float [3][n3][n2][n1] */
  double *rec_out;     /* device double [nrec][6][nfreq][2] */
} emm_job;

/* Workspace of emm_forward_jobs: each problem's emm_workspace_size, 256-byte
 * aligned, one after the other.  offsets: NULL, or a host array of njobs
 * that receives each problem's byte offset in the workspace (emm_status on
 * ws + offsets[j] reads problem j's device status).  EMM_EINVAL if njobs is
 * outside 1..16, the problems' FD orders differ, or a survey asks for the
 * volume DTFT, the air boundary, a magnetic source or an antenna. */
int emm_jobs_workspace_size(int njobs, const emm_job *jobs, size_t *bytes, size_t *offsets);

/* How emm_forward_jobs advances its problems. */
enum {
  EMM_JOBS_LIST = 0,        /* every leapfrog step is one E and one H launch over a work list of
                               all the problems' tiles (and receiver CTAs): their launch tails
                               overlap instead of each draining alone */
  EMM_JOBS_SEQUENTIAL = 1,  /* each problem's whole time loop in turn on `stream` */
  EMM_JOBS_STREAMS = 2      /* each problem on a stream of its own, forked from `stream` and
                               joined back to it (the library creates and releases the streams);
                               on these streams each launch waits for the whole launch before
                               it (no programmatic dependent launches) */
};

/* Forward solves of up to 16 problems of any grid sizes (one FD order, an
 * electric point dipole each) by one of the strategies above (emm_jobs_tune
 * picks the fastest for a given set of problems).  Each problem runs its own
 * survey->nt steps (under EMM_JOBS_LIST a problem that is done returns at
 * once from the later launches); each rec_out receives exactly what
 * emm_forward would write for that problem, whatever the strategy (the
 * same arithmetic on the same data).  The paper runs one transmitter per
 * MPI rank; this is the single-GPU form of running many, including grids of
 * uneven sizes.
 *   ws   device workspace of emm_jobs_workspace_size bytes, 256-byte aligned.
 * Asynchronous on `stream`; errors as emm_forward and emm_jobs_workspace_size,
 * and EMM_EINVAL for an unknown strategy. */
int emm_forward_jobs(int njobs, const emm_job *jobs, int strategy, void *ws, size_t ws_bytes,
                     emm_stream stream);

/* Autotuner of emm_forward_jobs: runs `steps` leapfrog steps of the problems
 * by each strategy (after a short warm-up of each), timed with CUDA events on
 * `stream`, and returns the times in ms[3] (host, indexed by EMM_JOBS_*) and
 * the fastest strategy in *best.  Synchronises `stream`.  The workspace is
 * left in no particular state (every solve prepares it again).  EMM_EINVAL
 * if steps < 1 or ms or best is NULL; otherwise as emm_forward_jobs. */
int emm_jobs_tune(int njobs, const emm_job *jobs, void *ws, size_t ws_bytes, int steps, emm_stream stream,
                  double *ms, int *best);

/* ---- Wavefront solve: several time steps in flight, through L2 ----
 * emm_forward's results (bit for bit) from ONE persistent cooperative
 * launch that advances z-layers of tiles through `depth` leapfrog steps per
 * sweep of the grid, so that a layer's fields, read from DRAM once, serve
 * several half-steps while they sit in the 126 MB L2 (the paper's solver
 * launches one kernel per half-step and re-reads every field each time,
 * Sec. 4).  The CTAs claim tiles in a fixed global order and each tile waits
 * (bounded, 1 s of device time) until the z-layers it reads are complete;
 * a wait that runs out writes EMM_ETIMEOUT to the status word (emm_status)
 * and every CTA stops.  One electric point dipole, no volume DTFT, no air
 * boundary; nt < 2^18.
 *   depth  time steps per sweep (1 .. 64).
 *   ws     device workspace of emm_wave_workspace_size bytes, 256-byte
 *          aligned (the forward workspace, then the tile order and the
 *          layer counters).
 * Other arguments as emm_forward.  Asynchronous on `stream`; EMM_EINVAL for
 * a survey outside the limits above, otherwise the errors of emm_forward;
 * EMM_ECUDA if the launch fails. */
int emm_wave_workspace_size(const emm_grid *grid, const emm_survey *survey, int depth, size_t *bytes);
int emm_forward_wave(const emm_grid *grid, const emm_survey *survey, const float *sigma, int depth, void *ws,
                     size_t ws_bytes, double *rec_out, emm_stream stream);

/* ---- Persistent work list: many problems in one cooperative launch ----
 * The paper runs one MPI rank per transmitter (Sec. 5); on one GPU the
 * transmitters of a survey and problems on grids of uneven sizes advance
 * together in ONE persistent launch: the resident CTAs walk the E half-step
 * tiles (and receiver CTAs) of every problem, meet at a grid barrier, walk
 * the H half-step tiles, meet again, for every leapfrog step.  Each item runs
 * the per-CTA code of the problem's own launch, so every problem's G equals
 * its emm_forward (or emm_forward_batch) result bit for bit.
 *
 * One task: a grid and survey with its conductivity (device float
 * [3][n3][n2][n1]); nsrc >= 1 transmitters sharing them (as
 * emm_forward_batch) at src_pos (host double [nsrc][3]; may be NULL when
 * nsrc == 1: survey->src); rec_out device double [nsrc][nrec][6][nfreq][2]. */
typedef struct emm_task {
  const emm_grid *grid;
  const emm_survey *survey;
  const float *sigma;
  int nsrc;
  const double *src_pos;
  double *rec_out;
} emm_task;

/* Launch options of the persistent work list. */
typedef struct {
  int ctas_per_sm;   /* resident CTAs per SM: 0 = as many as fit, else at most this many */
  int max_ctas;      /* 0 = no further limit, else at most this many CTAs in all */
  double wait_s;     /* bound of one grid-barrier wait, seconds (<= 0: 1 s) */
  int skip_arrival;  /* testing only: the index of one CTA that leaves without arriving at the
                        first grid barrier, so that every other CTA's bounded wait runs out and the
                        run ends with EMM_ETIMEOUT; -1 (or any index >= the CTA count) normally */
  int tile_shape;    /* stencil tile of one work item, 128 threads each: 0 = 32 x 8 x 2 cells
                        (x, y, z; the shape of the plain launches), 1 = 32 x 4 x 4 cells */
} emm_persist_opts;

/* Workspace of emm_forward_persistent: a 256-byte header (the work list's
 * status word first, so emm_status(ws) reads it), then each task's forward
 * workspace (emm_batch_workspace_size of its nsrc), 256-byte aligned.
 * offsets: NULL or a host array of ntasks receiving each task's byte offset
 * (emm_status(ws + offsets[j]) reads task j's own status word).  EMM_EINVAL
 * if ntasks is outside 1..16, the tasks' FD orders differ, nsrc < 1, src_pos
 * is NULL with nsrc > 1, or a survey asks for the volume DTFT, the air
 * boundary, a magnetic source or an antenna. */
int emm_persist_workspace_size(int ntasks, const emm_task *tasks, size_t *bytes, size_t *offsets);

/* Forward solves of the tasks in one persistent cooperative launch (after
 * each task's set-up, enqueued on `stream`, and before its normalisation).
 * opts NULL: the defaults {0, 0, 1.0, -1, 0}.  Every grid-barrier wait is
 * bounded by opts->wait_s of device time; a wait that runs out writes
 * EMM_ETIMEOUT to the header's status word and every CTA returns at its next
 * barrier (the outputs are then undefined).  Asynchronous on `stream`;
 * host-detected errors as emm_forward and emm_persist_workspace_size: the
 * layout and option checks enqueue nothing, while an error found in a
 * task's own set-up (EMM_ECFL, EMM_EOUTSIDE) returns after the set-up of
 * the tasks before it was enqueued (no launch follows); EMM_ECUDA if the
 * launch fails (for instance when the CTAs cannot all be resident). */
int emm_forward_persistent(int ntasks, const emm_task *tasks, const emm_persist_opts *opts, void *ws,
                           size_t ws_bytes, emm_stream stream);

/* Autotuner of the persistent launch: the candidates are every tile shape
 * (tile_shape 0, 1) with 1, 2, ... resident CTAs per SM up to that shape's
 * occupancy limit, in that order; it times `steps` leapfrog steps (each
 * task's own count at most) of the first *ncand candidates, each after a
 * warm-up run, with CUDA events on `stream`.  Returns in cands[k] and ms[k]
 * (host arrays of *ncand) each timed candidate's options and time, in
 * *ncand the number timed and in *best the fastest.  Synchronises `stream`;
 * the workspace is left to be prepared again.  EMM_EINVAL if steps < 1,
 * *ncand < 1 or a pointer is NULL; otherwise as emm_forward_persistent. */
int emm_persist_tune(int ntasks, const emm_task *tasks, void *ws, size_t ws_bytes, int steps, emm_stream stream,
                     int *ncand, emm_persist_opts *cands, double *ms, emm_persist_opts *best);

/* The whole persistent solve of fixed tasks captured once as a CUDA graph:
 * the tasks' set-up (state cleared, dt/eps from the conductivity at each
 * task's sigma pointer; the tables are uploaded once, at creation), the
 * cooperative launch and the normalisation.  emm_persist_plan_run replays
 * it on `stream` for the current contents of the bound sigma buffers into
 * the bound outputs; the plan keeps its own copies of the host arrays the
 * tasks point to.  Errors as emm_forward_persistent; EMM_ECUDA if the
 * capture or instantiation fails.  Destroy frees the graph (a launch in
 * flight completes first). */
typedef struct emm_persist_plan emm_persist_plan;
int emm_persist_plan_create(int ntasks, const emm_task *tasks, const emm_persist_opts *opts, void *ws,
                            size_t ws_bytes, emm_stream stream, emm_persist_plan **out);
int emm_persist_plan_run(emm_persist_plan *plan, emm_stream stream);
void emm_persist_plan_destroy(emm_persist_plan *plan);

/* Device workspace bytes emm_gradient needs (the forward workspace, the
 * checkpoints of every ckpt_every-th step, the E snapshots of one checkpoint
 * segment, the adjoint fields and the FP64 gradient accumulators).
 * EMM_EINVAL on bad input, ckpt_every < 1 or survey->volume set. */
int emm_gradient_workspace_size(const emm_grid *grid, const emm_survey *survey, int ckpt_every,
                                size_t *bytes);

/* Gradient of the receiver Green's functions with respect to the
 * conductivity: for a cotangent dG it computes
 *     grad = d/d sigma  Re( sum_{r,c,f} conj(dG[r][c][f]) G[r][c][f] ),
 * the vector-Jacobian product of the forward map sigma -> G.  The paper
 * stops at the forward solver (inversion is named as future work); this is
 * the exact discrete adjoint of the time loop emm_forward runs (Sec. 3.1,
 * Eq. 8; CPML Eq. 22-24; DTFT Eq. 25; Eq. 7), with dt, nt and the CPML
 * coefficients fixed by the survey constants.  Forward states are recomputed
 * from checkpoints taken every ckpt_every steps.
 *   sigma     device float [3][n3][n2][n1], as for emm_forward.
 *   dG        device double [nrec][6][nfreq][2] (re, im) cotangent.
 *   ws        device workspace of emm_gradient_workspace_size bytes, 256-byte
 *             aligned; contents on entry do not matter.
 *   rec_out   device double [nrec][6][nfreq][2]: G of the forward sweep.
 *   grad      device double [3][n3][n2][n1]: the gradient with respect to
 *             the interior staggered sigma_xx, sigma_yy, sigma_zz (the pads'
 *             replicated values folded onto the edge samples).
 * Asynchronous on `stream`; errors as emm_forward (survey->volume must be 0
 * survey->src_kind 0, survey->src_length 0 and survey->airwave 0: EMM_EINVAL
 * otherwise). */
int emm_gradient(const emm_grid *grid, const emm_survey *survey, const float *sigma, const double *dG,
                 int ckpt_every, void *ws, size_t ws_bytes, double *rec_out, double *grad,
                 emm_stream stream);

/* emm_gradient with a memory budget for the reverse sweep: the forward
 * sweep keeps the E snapshot of every step of the last
 * floor(stored_steps / ckpt_every) checkpoint segments (at most all of them)
 * in the workspace, and the reverse sweep recomputes only the earlier
 * segments.  Workspace: emm_gradient_stored_workspace_size with the same
 * ckpt_every and stored_steps (each stored step adds one E state: the three
 * E arrays).  stored_steps = 0 is emm_gradient.  The gradient and G equal
 * emm_gradient's bit for bit (recomputation restarts from full checkpointed
 * states through the same deterministic kernels).  EMM_EINVAL if
 * stored_steps < 0; otherwise as emm_gradient. */
int emm_gradient_stored_workspace_size(const emm_grid *grid, const emm_survey *survey, int ckpt_every,
                                       int stored_steps, size_t *bytes);
int emm_gradient_stored(const emm_grid *grid, const emm_survey *survey, const float *sigma, const double *dG,
                        int ckpt_every, int stored_steps, void *ws, size_t ws_bytes, double *rec_out,
                        double *grad, emm_stream stream);

/* Least-squares data misfit of one transmitter and its gradient, in one
 * call (no separate forward solve for the residual):
 *     misfit += 1/2 sum_{r,c,f} w[r][c][f] |G[r][c][f] - d_obs[r][c][f]|^2
 *     grad    = d/d sigma of that misfit
 * The forward sweep gives G; a device kernel forms the weighted residual
 * w (G - d_obs) and adds the misfit (a fixed-order reduction, so repeated
 * calls are reproducible); the residual is the cotangent of the adjoint
 * sweep, i.e. the result is emm_gradient_stored with dG = w (G - d_obs).
 * The paper names inversion as future work; this is the data-fit term an
 * inversion of its Green's functions minimises.
 *   d_obs     device double [nrec][6][nfreq][2] observed data (re, im).
 *   weight    device double [nrec][6][nfreq], non-negative, or NULL for
 *             all ones (a zero weight drops a datum, e.g. a channel not
 *             recorded).
 *   misfit    device double; the misfit is ADDED to it, so calls for the
 *             transmitters of a survey accumulate their sum.
 * Workspace: emm_gradient_stored_workspace_size with the same ckpt_every
 * and stored_steps.  Other arguments, asynchrony and errors as
 * emm_gradient_stored; EMM_EINVAL if d_obs or misfit is NULL. */
int emm_misfit_gradient(const emm_grid *grid, const emm_survey *survey, const float *sigma,
                        const double *d_obs, const double *weight, int ckpt_every, int stored_steps,
                        void *ws, size_t ws_bytes, double *rec_out, double *misfit, double *grad,
                        emm_stream stream);

/* Staggered conductivity from cell values (Sec. 3.6).  Cells lie between
 * adjacent interior nodes: [n3-1][n2-1][n1-1] arrays, x fastest, of the
 * horizontal (sigma_h) and vertical (sigma_v) conductivity.  sigma_xx at the
 * E_x sample (x_{i+1/2}, y_j, z_k) is the mean of sigma_h over the cells
 * around that edge in y and z (cells j-1, j and k-1, k, clamped to the
 * model), weighted by their y-z face areas dy dz; along x the sample takes
 * cell min(i, n1-2).  sigma_yy likewise (x and z neighbours), sigma_zz the
 * same mean of sigma_v over the x and y neighbours.  The map is linear.
 *   ws        device scratch of emm_stagger_workspace_size bytes, 8-byte
 *             aligned (the interior cell widths are copied there).
 *   sigma_h, sigma_v  device double [n3-1][n2-1][n1-1].
 *   sigma     device float [3][n3][n2][n1] output, as emm_forward takes it
 *             (each mean computed in FP64, rounded once).
 * Asynchronous on `stream`.  EMM_EINVAL on NULL arguments, EMM_EWORKSPACE
 * on a short or misaligned ws, EMM_ECUDA on a launch error. */
int emm_stagger_workspace_size(const emm_grid *grid, size_t *bytes);
int emm_stagger_sigma(const emm_grid *grid, const double *sigma_h, const double *sigma_v, void *ws,
                      size_t ws_bytes, float *sigma, emm_stream stream);

/* Transpose of emm_stagger_sigma: carries a gradient with respect to the
 * staggered conductivity, device double [3][n3][n2][n1] (emm_gradient's
 * output), to the cells, and ADDS it to grad_h and grad_v (device double
 * [n3-1][n2-1][n1-1]), so the transmitters of a survey accumulate.  Each
 * cell gathers its own terms in a fixed order (deterministic).  Arguments
 * and errors as emm_stagger_sigma. */
int emm_stagger_sigma_adjoint(const emm_grid *grid, const double *grad, void *ws, size_t ws_bytes,
                              double *grad_h, double *grad_v, emm_stream stream);

/* Size of the scratch array that emm_forward_static works in. */
#define EMM_STATIC_SCRATCH_BYTES (64u << 20)

/* emm_forward for callers that cannot allocate device memory: for instance a
 * plug-in inside a host application that owns every device allocation and
 * forbids its modules to call cudaMalloc, or code that must not call it at
 * solve time because an allocation can synchronise the device.  The paper has
 * no counterpart of this call; it computes what emm_forward computes.
 *   Instead of a caller workspace it uses one file-scope device array of
 *   EMM_STATIC_SCRATCH_BYTES (64 MiB) inside the library, which every GPU that
 *   loads the library holds until the process exits.  The call itself
 *   allocates nothing: no cudaMalloc, no cudaFree, no allocating library
 *   routine.  The array is created when the library's device code is loaded
 *   into a context, which the CUDA runtime does at the first library call that
 *   touches that device (with lazy module loading, possibly at this call's
 *   first use); that load can allocate and synchronise like any module load,
 *   so make one library call on each device before the code that must not
 *   allocate.  The first call in a context looks up the array's address there
 *   (the context of the device current at the call) and caches it per
 *   context; make this first call on each device before any stream capture.
 *   After a device reset the module is loaded again in a new context, and the
 *   next call looks the address up again.
 *   Arguments sigma, rec_out, vol_out and stream are those of emm_forward
 *   (device buffers the caller owns).  status: NULL, or a host int that, after
 *   the call has synchronised `stream`, receives the device status word of
 *   the run (EMM_OK, EMM_EDEVICE or EMM_ETIMEOUT, as emm_status reports it);
 *   with status NULL the call returns before the GPU finishes.
 *   Errors: those of emm_forward; EMM_EWORKSPACE when the problem needs more
 *   than EMM_STATIC_SCRATCH_BYTES (emm_workspace_size gives the need), with
 *   nothing enqueued; EMM_ECUDA if the address lookup fails.
 *   Every call shares the one array and finds the previous call's contents in
 *   it; the call clears what must start at zero.  Calls whose work overlaps
 *   on the GPU (different streams, or several host threads) race on the array
 *   and give undefined results: serialise them on one stream. */
int emm_forward_static(const emm_grid *grid, const emm_survey *survey, const float *sigma,
                       double *rec_out, double *vol_out, emm_stream stream, int *status);

/* Static description of an error code (never NULL). */
const char *emm_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* EMM_H */
