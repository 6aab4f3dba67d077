/*
 * pbs.h -- C ABI of the GB300 (sm_103a) proton pencil-beam depth-march solver.
 *
 * The library computes the deterministic linear-Boltzmann proton-beam model of
 * Zhang, Bai & Tang (arXiv 2504.00340): the phase-space density
 * psi(x; y, z, E, u, v) is marched in depth x (the time-like variable,
 * Section 3.3) by Strang splitting into three Crank-Nicolson subsystems:
 *   E  energy loss, DG-P1 in energy (Section 3.2, Eq. 0041-d),
 *   T  lateral transport, flux-limited MUSCL finite volumes (Section 3.4,
 *      Eq. distansport, Remark 3),
 *   A  angular diffusion, five-point Laplacian diagonalised by sine transforms
 *      (Section 3.4, Eqs. sd and fly),
 * applied as E(h/2) T(h/2) A(h) T(h/2) E(h/2) per depth step h.  Protons are
 * split into the primary field and K catastrophically scattered fields by
 * source iteration (Section 3.1, Eq. pri-se; Remark 1), and dose is tallied per
 * voxel from the energy lost in the E substeps (Section 4, Eq. en_d).
 *
 * Conventions for every entry point:
 *   - All functions return pbs_status; no C++ exception crosses the ABI.
 *   - Host arrays passed in are borrowed for the duration of the call only
 *     (copied in).  Host arrays passed out are written by the call.
 *   - Device memory: the caller owns the workspace it binds with
 *     pbs_bind_workspace; the library allocates no device memory itself
 *     (its coefficient tables and device status word live in the workspace;
 *     only the CUDA graph that pbs_run records holds driver-owned memory).
 *   - Stream: all device work is issued on the stream given to pbs_create
 *     (a cudaStream_t passed as void*; NULL = the legacy default stream).
 *     pbs_launch_beam, pbs_step and the substep calls are asynchronous;
 *     pbs_read_* synchronise the stream.
 *   - A context is bound to the CUDA device current at pbs_create; call it
 *     with that device current.  A context is not thread-safe.
 *   - Calling out of order (e.g. pbs_step before pbs_launch_beam) returns
 *     PBS_ERR_STATE; bad sizes or NULL pointers return PBS_ERR_ARG; CUDA
 *     failures return PBS_ERR_CUDA; a device wait that gave up returns
 *     PBS_ERR_TIMEOUT.  pbs_last_error describes the last failure.
 *
 * Logical layout of one component of psi (row-major, used by pbs_read_psi,
 * pbs_write_psi and on the device):  psi[g][c][j][i][p][q] with
 *   g energy group 0..ng-1 (0 = lowest energy), c DG coefficient
 *   (0 = group mean psi^1, 1 = slope psi^2), j,i angle indices in v,u,
 *   p,q lateral cell indices in y,z.
 */
#ifndef PBS_H
#define PBS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PBS_OK = 0,
  PBS_ERR_ARG = -1,
  PBS_ERR_CUDA = -2,
  PBS_ERR_NOMEM = -3,
  PBS_ERR_STATE = -4,
  PBS_ERR_TIMEOUT = -5,
  PBS_ERR_UNSUPPORTED = -6
} pbs_status;

typedef enum {
  PBS_FP64 = 0,   /* psi, arithmetic and the source contraction in FP64       */
  PBS_FP32 = 1,   /* psi and arithmetic in FP32, FP64 dose tally              */
  PBS_MIXED = 2   /* FP32 psi; the catastrophic-source angle contraction on
                     tensor cores in BF16 with FP32 accumulation             */
} pbs_precision;

/* Discretisation.  Lateral cells are centred on (y,z) = 0; angle nodes are
 * u_i = (i - (nu-1)/2) du with du = 2 u_max / (nu + 1) (zero Dirichlet values
 * one spacing beyond the outermost nodes, Section 3.4); energy faces are
 * given explicitly (ng+1 values, strictly ascending, MeV). */
typedef struct {
  int ny, nz;              /* lateral cells (y, z)                          */
  int ng;                  /* energy groups                                 */
  int nu, nv;              /* angle nodes (u, v); the device path needs even
                              nu, nv with nu, nv <= 16                      */
  int nx;                  /* depth steps the context can hold dose for     */
  int n_scatter;           /* K: number of scattered components (0 = primary
                              only)                                         */
  int n_beams;             /* independent pencil beams held by the context
                              (>= 1): each has its own psi_p..psi_sK, beam
                              projection, dose and fluence; all share the
                              grid, physics and density field and march in
                              lock-step, each kernel launch covering all    */
  double dy, dz;           /* lateral cell sizes (cm)                       */
  double dx;               /* depth step h (cm)                             */
  double u_max, v_max;     /* half-widths of the angle box                  */
  const double *e_faces;   /* ng+1 ascending group faces (MeV), borrowed    */
} pbs_grid;

/* Physics of water-equivalent media.  model = 0 (Appendix A with
 * substitutes): mass stopping power from the Bragg-Kleeman range law
 * R = bk_alpha E^bk_p, multiple-scattering power (Highland form)
 * T = (es / pv)^2 / x0 used as rho * sigma_tr.  model = 1 (Appendix A as
 * printed, for water): Bethe-Bloch stopping power per element with the
 * piecewise I-value rule, combined by Bragg additivity over the mass
 * fractions of H and O (density correction 0; held constant below
 * max(dE_1 / 2, 0.5 MeV)), and the screened-Rutherford momentum-transfer
 * cross section summed over the atoms of a gram (group-averaged by 8-point
 * Gauss-Legendre); bk_*, x0 and es are then unused.  Both: catastrophic
 * removal sigma_ct (cm^2/g), exponential energy transfer P^1 with rate
 * lambda_p1 (1/MeV) and Gamma(g_alpha, g_beta) angular deflection P^2
 * (Section 4 and Appendix A.4); s_scale and ts_scale multiply S and the
 * scattering power (0 switches a process off); mp is the proton rest
 * energy (MeV).  t_scale multiplies the energy-straggling coefficient of
 * Appendix A.2 (Williams' binding-corrected Bohr coefficient of water, per
 * element with the I-values above, held below 0.5 MeV; either model); 0
 * (the default) leaves straggling out (see pbs_set_straggling for how the
 * energy substep takes it). */
typedef struct {
  double bk_alpha, bk_p;
  double x0;
  double mp;
  double es;
  double sigma_ct;
  double lambda_p1;
  double g_alpha, g_beta;
  double s_scale, ts_scale;
  int model;
  double t_scale;
} pbs_physics;

/* Pencil beam of Eq. (bdy): Gaussian in y, z (cm), u, v and E (MeV). */
typedef struct {
  double e0, sigma_e, y0, z0, sigma_y, sigma_z, u0, v0, sigma_u, sigma_v;
} pbs_beam;

typedef struct pbs_ctx pbs_ctx;

/* Create a context for the grid on the current device.  precision is a
 * pbs_precision.  stream is a cudaStream_t (may be NULL).  *out receives the
 * context; destroy it with pbs_destroy.  Returns PBS_ERR_UNSUPPORTED for
 * grids the device kernels do not handle (odd or > 16 angle counts, nz > 1024,
 * ng > 2048). */
pbs_status pbs_create(pbs_ctx **out, const pbs_grid *grid, int precision, void *stream);

/* Bytes of device workspace the context needs: psi of all K+1 components
 * (the primary and scattered fields of the source iteration, Section 3.1,
 * Eq. pri-se, each with both DG coefficients of Section 3.2), the source
 * buffers of Remark 1, the density slabs, the dose and fluence tallies of
 * Section 4 and the coefficient tables.  The library's own addition: the
 * paper names no memory layout. */
pbs_status pbs_workspace_size(const pbs_ctx *ctx, size_t *bytes);

/* Bind caller-owned device memory of at least pbs_workspace_size bytes,
 * 256-byte aligned; the call zeroes it (synchronously on the context's
 * stream).  The caller keeps ownership and must keep it alive until
 * pbs_destroy or a new bind.  A new bind forgets the material and the beam. */
pbs_status pbs_bind_workspace(pbs_ctx *ctx, void *dev_ptr, size_t bytes);

/* Build the FP64 coefficient tables on the host from the physics model and
 * upload them (group faces' stopping power, group-averaged scattering power,
 * removal cross section, P^1 decay factors, P^2 matrices). */
pbs_status pbs_set_physics(pbs_ctx *ctx, const pbs_physics *phys);

/* Caller-supplied tables instead of the built-in physics (e.g. tabulated
 * stopping powers): s_face[ng+1] mass stopping power at the group faces
 * (MeV cm^2/g, > 0), ts[ng] group-averaged scattering power (rad^2 cm^2/g,
 * >= 0: d<u^2>/dx per unit density, the rho sigma_tr of Eq. 0041-d),
 * sig_ct[ng] catastrophic removal cross section of each emitting group
 * (cm^2/g, >= 0), lambda_p1 (1/MeV, > 0) the rate of the exponential energy
 * transfer P^1 (Appendix A.4; normalised to sum 1 over the receiving groups),
 * and p2[ng*na*na] ([g][a][a'], the outgoing-angle density, normalised by
 * the caller) or NULL to keep the P^2 of the previous pbs_set_physics /
 * pbs_set_tables call.  Host arrays, copied during the call.  PBS_ERR_ARG
 * for a value out of range; PBS_ERR_STATE for p2 = NULL with n_scatter > 0
 * and no previous P^2. */
pbs_status pbs_set_tables(pbs_ctx *ctx, const double *s_face, const double *ts, const double *sig_ct,
                          double lambda_p1, const double *p2);

/* Energy straggling (Section 3.2, the Q_1 / Q_2 terms of Eq. 0041-d;
 * Appendix A.2) with a caller-given coefficient: t_face[ng+1] the mass
 * straggling coefficient at the group faces (MeV^2 cm^2/g, finite, >= 0;
 * linear within each group), or NULL to switch straggling off.  Replaces the
 * coefficient pbs_set_physics built (its t_scale) and keeps every other
 * table; pbs_set_tables switches straggling off again.  The term splits into
 * (rho/2) d/dE(T dpsi/dE), discretised by the symmetric interior-penalty
 * method (penalty 2 T_f over the mean width of the two groups at face f, no
 * flux through the two outer faces) and applied explicitly to the old state
 * inside each Crank-Nicolson energy substep, and the drift
 * (rho/2) d/dE(T' psi), added to the face stopping powers as T'/2 (T' at an
 * inner face: the mean of its two groups' slopes).  The explicit part is
 * stable while h rho_max lambda_max / 2 <= 2 (lambda_max bounded by the row
 * sums of the straggling blocks, h = dx/2); pbs_step, pbs_run, pbs_autotune
 * and pbs_substep_energy return PBS_ERR_ARG beyond it.  Host array, copied
 * during the call.  PBS_ERR_STATE before pbs_set_physics / pbs_set_tables. */
pbs_status pbs_set_straggling(pbs_ctx *ctx, const double *t_face);

/* Copy out the straggling coefficient at the faces t_face[ng+1] (zeros when
 * off) and the face stopping power before the drift is added, s_base[ng+1]
 * (pbs_get_tables returns the stopping power with the drift).  Either
 * pointer may be NULL. */
pbs_status pbs_get_straggling(const pbs_ctx *ctx, double *t_face, double *s_base);

/* Copy the FP64 host tables out (any pointer may be NULL):
 * s_face[ng+1] (MeV cm^2/g), ts[ng] (rad^2 cm^2/g), sig[ng] (cm^2/g),
 * p1[ng*ng] ([g'][g], probability g' -> g), p2[ng*na*na] ([g][a][a'],
 * density in (u,v) of a' -> a), u[nu], v[nv]. */
pbs_status pbs_get_tables(const pbs_ctx *ctx, double *s_face, double *ts, double *sig, double *p1, double *p2,
                          double *u, double *v);

/* Density rho[s][p][q] (g/cm^3) for depth steps s = 0..n_slabs-1
 * (n_slabs <= grid.nx), host FP64, copied during the call.  The density
 * multiplies the stopping power and the removal cross section of the energy
 * operator (Eq. 0041-do) and the scattering power of the angular subsystem
 * (Section 3.4); Section 4's heterogeneous phantoms (slabs, inserts) are
 * density fields.  Step s uses slab s in all five substeps (the cell-centred
 * reading of a depth step).  PBS_ERR_ARG for n_slabs out of range or a
 * negative or non-finite density; PBS_ERR_STATE before a workspace is
 * bound. */
pbs_status pbs_set_material(pbs_ctx *ctx, const double *rho, int n_slabs);

/* Project the beam of Eq. (bdy) onto psi_p (cell averages in y, z, u, v;
 * DG L2 projection in E; normalised to one proton), zero psi_s1..psi_sK,
 * the dose and the fluence, and reset the depth counter to 0.  With
 * n_beams > 1 every beam of the context gets this beam. */
pbs_status pbs_launch_beam(pbs_ctx *ctx, const pbs_beam *beam);

/* As pbs_launch_beam with one beam description per beam of the context
 * (n must equal grid.n_beams). */
pbs_status pbs_launch_beams(pbs_ctx *ctx, const pbs_beam *beams, int n);

/* March n_steps depth steps (Strang order E T A T E per step, all
 * components in lock-step).  Asynchronous.  PBS_ERR_ARG if the march would
 * pass the material's last slab.  The closing E(h/2) of the last step is
 * deferred so that it can be fused with the opening E(h/2) of the next call
 * (one pass over psi for the two); pbs_flush applies it, and every read,
 * write, substep or material call applies it first. */
pbs_status pbs_step(pbs_ctx *ctx, int n_steps);

/* Apply a deferred closing E(h/2), if any.  Asynchronous. */
pbs_status pbs_flush(pbs_ctx *ctx);

/* One depth step in four stages (Section 3.3's Strang sequence), for callers
 * that act between the substeps, e.g. to exchange halo rows between lateral
 * parts held by different processes:
 *   stage 0  E(h/2) opening the step (fused with a deferred closing half)
 *   stage 1  T(h/2)      stage 2  A(h)      stage 3  T(h/2)
 * after which the step is counted and its closing E(h/2) deferred, exactly
 * as pbs_step does.  Stages must come in the order 0, 1, 2, 3 (PBS_ERR_STATE
 * otherwise); pbs_step, pbs_run and pbs_domain_step refuse to start while a
 * staged step is incomplete.  Stage 0 returns PBS_ERR_ARG if the step would
 * pass the material's last slab.  Asynchronous. */
pbs_status pbs_step_stage(pbs_ctx *ctx, int stage);

/* Lateral domain decomposition of one beam (Remark 2: the energy and
 * angular subsystems are independent at every lateral point, only the
 * transport couples neighbouring cells).  Declares this context's rows
 * 0..ny-1 to be rows y_offset..y_offset+ny-1 of a grid of ny_global rows
 * (the same z, energy and angle grids and cell sizes), of which the first
 * halo_lo and the last halo_hi are halo rows: copies of the neighbouring
 * parts' own rows, refreshed before every transport substep.  A part at the
 * grid's lower edge (y_offset = 0) has halo_lo = 0, at the upper edge
 * halo_hi = 0, and every interior side has a halo (PBS_ERR_ARG otherwise).
 * The beam projection then evaluates the part's rows of the whole grid with
 * the whole grid's normalisation, so that the parts hold exactly the values
 * of the undivided grid.  Call it before pbs_launch_beam (PBS_ERR_STATE
 * after); contexts with n_beams > 1 return PBS_ERR_UNSUPPORTED.  Each part's
 * material is its own rows of the density field. */
pbs_status pbs_set_lateral_part(pbs_ctx *ctx, int y_offset, int ny_global, int halo_lo, int halo_hi);

/* March n_steps depth steps of one beam split into n_parts lateral parts
 * (pbs_set_lateral_part), ordered by y, in lock-step: stages 0-3 of each step
 * on every part, and before stages 1 and 3 the halo rows of every interior
 * interface copied from the neighbour's own rows into each part's own
 * workspace (cudaMemcpy2DAsync, every psi plane of every component; parts on
 * different streams or devices are ordered by event waits).  Interior halos
 * need at least 4 rows, the reach of the two stages of the explicit
 * trapezoid; the Crank-Nicolson transport (pbs_options) couples whole rows
 * and returns PBS_ERR_UNSUPPORTED.  The parts must share precision, z,
 * energy and angle grids, cell sizes, options, tables and depth, and their
 * own rows must tile the grid (PBS_ERR_ARG / PBS_ERR_STATE otherwise).  A
 * part's own rows of psi then equal those of the undivided march bit for bit
 * when both run the same kernel forms (pbs_tuning; FP64 has one form): the
 * arithmetic of each cell is the same.  Its halo rows hold nothing
 * meaningful between steps, and the dose and fluence of its own rows equal
 * the undivided ones up to the order of the FP64 tally's atomic sums.  The closing E(h/2) of the last step is deferred on every part as
 * in pbs_step.  Asynchronous on the parts' streams. */
pbs_status pbs_domain_step(pbs_ctx *const *parts, int n_parts, int n_steps);

/* Copy rows first_row..first_row+n_rows-1 of every psi plane of every
 * component (the [k][g][c][j][i] planes of ny x nz cells) to (to_buffer = 1)
 * or from (to_buffer = 0) a caller-owned device buffer laid out
 * [plane][row][q], planes * n_rows * nz values of the working precision.
 * With pbs_step_stage this is a halo exchange between lateral parts held by
 * different processes: pack the rows a neighbour needs, send them with the
 * caller's own transport, unpack the received rows into the halo.
 * Asynchronous on the context's stream. */
pbs_status pbs_copy_rows(pbs_ctx *ctx, int first_row, int n_rows, int to_buffer, void *dev_buf);

/* Depth range of each beam of a batch: beam b marches steps[b] depth steps
 * (capped by the material's n_slabs) and then only receives its closing
 * E(h/2); later launches skip it.  steps must be non-increasing in b (order
 * the beams by range) so that the marching beams always form a prefix and
 * every launch covers a contiguous block of components.  Default: nx for
 * every beam.  PBS_ERR_ARG for n != n_beams, a value outside [0, nx] or an
 * increase; PBS_ERR_STATE after the march has started (launch the beams
 * again first). */
pbs_status pbs_set_beam_steps(pbs_ctx *ctx, const int *steps, int n);

/* The whole march of every beam: restart psi, dose and fluence from the
 * launched beams' projections, march each beam to its depth
 * (pbs_set_beam_steps) and apply the closing half, so that the dose and
 * fluence are final.  use_graph != 0 records the sequence once into a CUDA
 * graph on a stream of the context (again after a change of beam depths,
 * material extent, launch shapes or workspace) and launches the graph on the
 * context's stream: one launch for the whole batch.  Asynchronous.  The
 * first graph call records; call it once before capturing the caller's own
 * work around it. */
pbs_status pbs_run(pbs_ctx *ctx, int use_graph);

/* Persistent batch of pencil beams (spots): the whole march of n_beams
 * independent beams in one persistent kernel launch, each beam a context of
 * its own (its own lateral grid, energy groups, tables, density, depth range
 * (pbs_set_beam_steps / material extent) and workspace).  A device work queue
 * hands out the tiles of every beam's passes (per depth step E(h/2) fused
 * across steps, T(h/2), A(h), T(h/2); Section 3.3), round-robin over the
 * beams; per-beam completion counters order a beam's passes, so beams of
 * different depth and size fill the GPU together with no bucketing and no
 * empty energy groups.  Every tile is the same device code as the matching
 * block of the per-substep kernels, so each beam's psi equals its own
 * pbs_run with the tuning {energy_angles 8, energy_form 1, angular_form 2 to 7}
 * bit for bit (the dose up to the order of its atomic FP64 sums).
 *   use_graph      nonzero: record the batch (every beam's restart from its
 *                  projection, the queue reset, the launch) into a CUDA graph
 *                  on first use and replay it; the graph is kept by beams[0]
 *                  until the batch (contexts, depths, workspace, options)
 *                  changes.  Record it before capturing around it.
 *   wait_limit_ms  bound of every device wait of a tile for the beam's
 *                  earlier passes (<= 0: 2000 ms).  A wait that runs out sets
 *                  every beam's device status word and the launch stops at
 *                  the next tile boundary with no copy in flight; the next
 *                  synchronising call on any beam (e.g. pbs_read_dose)
 *                  returns PBS_ERR_TIMEOUT, and the next pbs_run_batch
 *                  starts afresh.
 *   hold_beam      failure-detection test hook (-1 in normal use): beam
 *                  hold_beam's second pass waits for one tile more than its
 *                  first pass has, so its waits can only run out.
 *   shape          CTA shape of the launch (same results, different speed):
 *                  0  256 threads, two per SM (16-angle energy tiles, 4
 *                     transport columns per lane);
 *                  1  128 threads, three per SM (8-angle energy tiles, 4 or 6
 *                     transport columns).
 *   transport_cols 4 or 6 columns per lane of the transport tiles (6 only with
 *                  shape 1 and rows that split evenly into 6-column lanes,
 *                  else 4), or 0 for the default rule (6 where that fills the
 *                  warps better).
 *   pipeline       0: a beam's passes follow one another whole.  1: the
 *                  T(h/2) A(h) T(h/2) passes of a step are cut into chunks of
 *                  32 slab stacks (component, group, coefficient), and the
 *                  angular step of a chunk starts as soon as its first
 *                  transport is done, its second transport as soon as its
 *                  angular step is (the angular step couples only the angles
 *                  of one stack, the transport only the cells of one plane):
 *                  one beam's passes overlap, at the cost of more tasks.
 *   pbs_batch_autotune picks shape, columns and pipeline.  16 x 16 angles
 *   run with shape 0 only. */
typedef struct {
  int use_graph;
  double wait_limit_ms;
  int hold_beam;
  int shape;
  int transport_cols;
  int pipeline;
} pbs_batch_options;

/* Bytes of the device workspace pbs_run_batch needs for these beams with
 * their current depth ranges (descriptors, task list, queue counters), with
 * or without pipelined passes. */
pbs_status pbs_batch_workspace_size(pbs_ctx *const *beams, int n_beams, size_t *bytes);

/* Restart every beam from its projection (as pbs_run does) and march all of
 * them to their own depths in one persistent launch (see pbs_batch_options),
 * on the beams' common stream.  dev_ws: caller-owned device memory of at
 * least pbs_batch_workspace_size bytes, 256-byte aligned, kept alive while
 * the batch runs; opts may be NULL (no graph, 2000 ms waits).  The beams
 * must be FP32 or mixed-precision contexts with n_scatter = 0 and n_beams =
 * 1, the default integrators and no straggling, ny*nz even, nz a multiple
 * of 4, one square angle grid for all (at most 8 x 8, or 16 x 16 with shape
 * 0), one device and one stream
 * (PBS_ERR_UNSUPPORTED / PBS_ERR_ARG otherwise), each with a workspace,
 * tables, material and a launched beam (PBS_ERR_STATE otherwise).
 * Asynchronous; afterwards every beam's dose and fluence are final (read
 * them per context). */
pbs_status pbs_run_batch(pbs_ctx *const *beams, int n_beams, void *dev_ws, size_t bytes,
                         const pbs_batch_options *opts);

/* Batch autotuner: times the CTA shapes, transport column counts and
 * pipelined passes of pbs_batch_options (best of two trials each) on the
 * batch with every beam
 * cut to at most `steps` depth steps, with CUDA events on the beams' stream,
 * and writes the fastest into opts->shape, opts->transport_cols and
 * opts->pipeline (the other fields are kept).  The trials march the beams, so they restart from
 * their projections afterwards.  dev_ws as for pbs_run_batch.
 * Synchronises. */
pbs_status pbs_batch_autotune(pbs_ctx *const *beams, int n_beams, void *dev_ws, size_t bytes, int steps,
                              pbs_batch_options *opts);

/* Method options (each changes the computed result, unlike pbs_tuning):
 *   angular_integrator    time integration of each sine mode of the angular
 *                         diffusion (Section 3.4): 0 Crank-Nicolson (Section
 *                         3.3, the default), 1 the mode's exact exponential
 *                         exp(h kappa lam / 2) (the "ODE solver" reading).
 *   transport_integrator  depth integration of the lateral transport
 *                         (Remark 3): 0 the explicit trapezoid (Heun) of the
 *                         limited upwind operator L (the default); 1
 *                         Crank-Nicolson whose implicit half keeps the
 *                         first-order upwind part L1 implicit and takes the
 *                         limited slope from the old state:
 *                         (I - h/2 L1) psi_new = psi + h L(psi) - h/2 L1(psi),
 *                         solved exactly by one sweep in the upwind
 *                         direction (stable beyond the explicit Courant
 *                         limit).  Needs nz <= 256.
 *   straggling_integrator with energy straggling on (pbs_set_straggling):
 *                         0 the interior-penalty part explicit inside the
 *                         Crank-Nicolson energy step (the default; one scan
 *                         per fused pair of substeps); 1 inside the
 *                         Crank-Nicolson step as well, as the printed scheme
 *                         reads: the block-tridiagonal system is solved by
 *                         block elimination from the top group down and
 *                         substitution upward (two passes over psi per
 *                         substep, no fused pair, no stability bound). */
typedef struct {
  int angular_integrator;
  int transport_integrator;
  int straggling_integrator;
} pbs_options;

/* Set / read the method options; PBS_ERR_ARG for an unknown value,
 * PBS_ERR_UNSUPPORTED for transport_integrator 1 with nz > 256.  The
 * deferred closing E(h/2) of the march, if any, is applied first. */
pbs_status pbs_set_options(pbs_ctx *ctx, const pbs_options *options);
pbs_status pbs_get_options(const pbs_ctx *ctx, pbs_options *options);

/* Launch shapes and kernel forms of the march.  Every setting computes the
 * same method; forms differ in how the work maps onto the GPU, and the
 * packed forms differ from the plain ones by rounding only.
 *   energy_angles   angles per block of the energy pass: 4, 8 or 16
 *   energy_form     FP32 energy pass: 0 one lane per thread, 1 two lateral
 *                   points per thread on the packed FP32x2 datapath (needs
 *                   ny*nz even, else form 0 runs)
 *   transport_ctas  resident CTAs per SM of the streaming transport, 0..64
 *                   (0 = as many as fit)
 *   transport_cols  columns of a row per lane of the streaming transport: 4,
 *                   6, 8 or 0 (chosen by the row width nz: 6 where nz is a
 *                   multiple of 6 and that fills the warps better, else 4)
 *   angular_form    angular substep: 0 direct, 1 TMA-staged persistent
 *                   (needs a row pitch of ny*nz elements that is a multiple of
 *                   16 bytes), 2 packed FP32x2 (FP32, ny*nz even), 3 packed
 *                   at 64 registers per thread (more CTAs per SM), 4 packed
 *                   with two slab stacks per CTA (the second's rows prefetched
 *                   into the L2 during the first), 5 packed with the sine
 *                   coefficients held in registers (the N/2 distinct
 *                   magnitudes, signs fixed at compile time) instead of read
 *                   from the constant bank, 6 as 5 at most 85 registers per
 *                   thread, 7 as 5 with two slab stacks per CTA (as 4); a form
 *                   the grid does not allow falls back to 0
 *   source_form     BF16 source contraction on the tensor cores (mixed
 *                   precision, n_scatter > 0): 0 tile by tile, 1 pipelined
 *                   (TMA loads, MMAs and epilogue of consecutive tiles
 *                   overlapped), 2 pipelined with 128-byte swizzled R tiles */
typedef struct {
  int energy_angles;
  int energy_form;
  int transport_ctas;
  int transport_cols;
  int angular_form;
  int source_form;
} pbs_tuning;

/* Launch-shape autotuner: times the candidate energy forms and shapes (angles
 * per block 4, 8, 16), transport residencies (1, 2, 3, 4, as many as fit) and
 * angular forms on the launched beams with CUDA events, best of reps trials
 * each, and keeps the fastest.  The trials advance the state, so the beams
 * restart from their projections afterwards (depth 0).  Synchronises. */
pbs_status pbs_autotune(pbs_ctx *ctx, int reps);

/* Set / read the launch shapes directly (PBS_ERR_ARG for a value outside the
 * ranges above). */
pbs_status pbs_set_tuning(pbs_ctx *ctx, const pbs_tuning *tuning);
pbs_status pbs_get_tuning(const pbs_ctx *ctx, pbs_tuning *tuning);

/* Checkpoint / resume of the march state (the library's own addition; the
 * paper marches once from the entrance): psi of every component of every
 * beam (working precision), dose, fluence, the beam projection factors, the
 * per-beam depth ranges, the depth counter and a deferred closing E(h/2)
 * (kept deferred, not applied).  The material, the tables and the method
 * options are inputs, not state: set them on the restoring context before
 * pbs_checkpoint_load, equal to those of the saving context (the checkpoint
 * records the options and hashes of the FP64 tables and of the density
 * field, and load compares them).  pbs_checkpoint_size gives the bytes of
 * the host buffer; save copies the state into it (synchronises); load
 * restores a checkpoint written by a context with the same grid, precision,
 * n_scatter and n_beams.  load returns PBS_ERR_STATE before the tables and
 * the material are set, and PBS_ERR_ARG for another grid, options, tables or
 * density, or for a buffer that is not a consistent checkpoint (flags other
 * than 0/1, a deferred half with no marched step, depths out of range); it
 * rejects before touching the device.  Host buffers are the caller's. */
pbs_status pbs_checkpoint_size(const pbs_ctx *ctx, size_t *bytes);
pbs_status pbs_checkpoint_save(pbs_ctx *ctx, void *host, size_t bytes);
pbs_status pbs_checkpoint_load(pbs_ctx *ctx, const void *host, size_t bytes);

/* Depth steps marched since pbs_launch_beam. */
pbs_status pbs_get_depth(const pbs_ctx *ctx, int *steps_done);

/* Dose D[b][s][p][q] (MeV/g per source proton of beam b, Section 4:
 * D = E_dep / rho) for the first n_slabs slabs of every beam; n must equal
 * n_beams*n_slabs*ny*nz. Synchronises. */
pbs_status pbs_read_dose(pbs_ctx *ctx, double *host_out, size_t n);

/* Planar fluence F[b][s][p][q] = du dv sum_{k,g,a} psi^1 dE (protons/cm^2)
 * of beam b at depths s*dx, s = 0..n_planes-1 (s = 0 is the entrance): the
 * zeroth angular and energy moment of the phase-space density of Section 2
 * (integrating the DG expansion of Section 3.2 over each group leaves
 * psi^1 dE), summed over the primary and scattered fields; the particle
 * count whose loss the removal term of Eq. 0041-do drives.  n must equal
 * n_beams*n_planes*ny*nz with n_planes <= steps done + 1 (PBS_ERR_ARG
 * otherwise).  Synchronises. */
pbs_status pbs_read_fluence(pbs_ctx *ctx, double *host_out, size_t n);

/* Copy component k of psi to / from the host as FP64 in the logical layout
 * above (n = ng*2*nu*nv*ny*nz); component k = b*(n_scatter+1) + j is
 * component j of beam b.  Synchronises. */
pbs_status pbs_read_psi(pbs_ctx *ctx, int k, double *host_out, size_t n);
pbs_status pbs_write_psi(pbs_ctx *ctx, int k, const double *host_in, size_t n);

/* Single substeps for testing and for callers composing their own march.
 * energy: E(h) on all components in lock-step with the source chain, dose
 *   added to slab `slab`, fluence written to plane `fluence_plane` if >= 0.
 * transport: T(h) on all components.  angular: A(h) on all components with
 *   the density of slab `slab`. */
pbs_status pbs_substep_energy(pbs_ctx *ctx, double h, int slab, int fluence_plane);
pbs_status pbs_substep_transport(pbs_ctx *ctx, double h);
pbs_status pbs_substep_angular(pbs_ctx *ctx, double h, int slab);

/* Catastrophic source of Remark 1 from component k_from at its current
 * state with the density of slab `slab`: host_out[g][j][i][p][q] (FP64),
 * n = ng*nu*nv*ny*nz.  Synchronises. */
pbs_status pbs_eval_source(pbs_ctx *ctx, int k_from, int slab, double *host_out, size_t n);

/* Allocation-free variant of pbs_eval_source, for callers that cannot
 * allocate device memory (no cudaMalloc and no caching allocator: e.g. code
 * embedded in a host framework that hands it pre-carved device buffers, or a
 * process whose device memory belongs to another owner).  The paper has no
 * counterpart to this call.  It evaluates the same catastrophic source as
 * pbs_eval_source on an FP32 context (one removal cross section for every
 * group), without a context or workspace:
 *   psi_k    device, FP32 component [g][c][j][i][p][q] (ng*2*nu*nv*ny*nz)
 *   rho_yz   device, FP32 density of the slab [p][q]
 *   p2       device, FP32 P^2 matrices [g][a][a'] (ng*na*na), e.g. the FP64
 *            tables of pbs_get_tables converted to float
 *   e_faces  host, ng+1 ascending group faces (MeV), read during the call
 *   sigma_ct, lambda_p1  as in pbs_physics;  u_max, v_max  as in pbs_grid
 *   src_out  device, FP32 [g][j][i][p][q] (ng*nu*nv*ny*nz), written
 *   stream   cudaStream_t (may be NULL); the call is asynchronous.
 * Its only scratch is a 16 MiB array in the library's own device memory
 * (a file-scope __device__ array that every device loading the library holds
 * until exit), so ng*nu*nv*ny*nz must not exceed 4 Mi (= 4194304) elements
 * and ng must not exceed 2048: larger calls return PBS_ERR_UNSUPPORTED.  The
 * call allocates no device memory.  Its first call on a device looks up the
 * array's device address (once per device, with that device current): make
 * that first call before any stream capture.  Each device has its own copy
 * of the array, so calls on different devices are independent; on one
 * device every call shares the one array, whose contents each call fully
 * overwrites, so calls that overlap on the same device (e.g. on different
 * streams) race on it and must be serialised by the caller. */
pbs_status pbs_eval_source_noalloc(const float *psi_k, const float *rho_yz, const float *p2, const double *e_faces,
                                   int ng, int nu, int nv, int ny, int nz, double u_max, double v_max,
                                   double sigma_ct, double lambda_p1, float *src_out, void *stream);

/* Kernel kinds for per-kernel timing. */
typedef enum {
  PBS_KERNEL_ENERGY = 0,     /* energy substep scan (incl. dose/fluence/R)   */
  PBS_KERNEL_TRANSPORT = 1,  /* lateral transport substep                    */
  PBS_KERNEL_ANGULAR = 2,    /* angular substep                              */
  PBS_KERNEL_SOURCE = 3,     /* catastrophic-source angle contraction        */
  PBS_KERNEL_QUEUE = 4,      /* persistent batch: claiming tiles and waiting
                                for a beam's earlier passes                 */
  PBS_KERNEL_KINDS = 5
} pbs_kernel_kind;

/* Per-kernel timing.  pbs_set_profiling(ctx, 1) clears the totals and makes
 * every later kernel launch of the march be bracketed by a CUDA event pair
 * recorded on the context's stream (0 stops recording).  pbs_profile_read
 * synchronises the stream and returns, for one pbs_kernel_kind, the number of
 * launches timed and their summed device time in milliseconds.  A persistent
 * batch (pbs_run_batch) led by a profiling context is one launch, so its time
 * is split by tile kind instead: the kernel sums the SM clocks its CTAs spend
 * in energy, transport and angular tiles and in claiming and waiting
 * (PBS_KERNEL_QUEUE), and pbs_profile_read reports, per kind, the tiles run
 * and those clocks per CTA converted to milliseconds at the device's
 * nominal SM clock (kinds sum to about the launch's duration). */
pbs_status pbs_set_profiling(pbs_ctx *ctx, int on);
pbs_status pbs_profile_read(pbs_ctx *ctx, int kind, long long *launches, double *total_ms);

/* Number of kernel launches the library has issued since pbs_create. */
pbs_status pbs_kernel_launches(const pbs_ctx *ctx, long long *count);

const char *pbs_last_error(const pbs_ctx *ctx);
const char *pbs_status_string(int status);
void pbs_destroy(pbs_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif
