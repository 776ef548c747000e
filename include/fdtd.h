/*
 * fdtd.h -- C ABI of the GB300 Maxwell-Bloch FDTD library (libfdtd.so).
 *
 * The library steps the 3D Yee finite-difference time-domain leapfrog over a
 * per-node permittivity map of an fcc inverted opal, with absorbing (CPML),
 * PEC or periodic faces, a Gaussian-pulse source, field probes and Poynting
 * flux planes, coupled cell by cell to a four-level Maxwell-Bloch gain medium
 * (polarization oscillator per field component, rate equations for the four
 * level populations, pump and seeded spontaneous-emission noise).
 * Paper: Conti & Fratalocchi, "Dynamic light diffusion, Anderson localization
 * and lasing in disordered inverted opals: 3D ab-initio Maxwell-Bloch
 * computation", Sec. "Sample and numerical approach" (method, geometry,
 * disorder), Secs. "Wide-band excitation" and "Dynamical diffusion" (pulses,
 * probes, transmitted flux T(t)), Sec. "3+1D simulation of lasing" (pumped gain).
 *
 * Units (normalized, exact rescalings of SI):
 *   E in V/m; H~ = eta0 H in V/m; P~ = P / eps0 in V/m; populations in m^-3.
 *   S = c dt / dx = courant / sqrt(3).   Cell (i,j,k) spans [i,i+1)x[j,j+1)x[k,k+1)
 *   in grid units; Ex at (i+1/2,j,k), Ey at (i,j+1/2,k), Ez at (i,j,k+1/2),
 *   H~x at (i,j+1/2,k+1/2), H~y at (i+1/2,j,k+1/2), H~z at (i+1/2,j+1/2,k).
 * Arrays crossing the ABI are in memory order [k][j][i] (x fastest).
 *
 * Conventions
 *   - Every function returns 0 (FDTD_OK) or a negative FDTD_E_* code;
 *     fdtd_last_error() gives a message for the calling thread.  No C++
 *     exception crosses the ABI.
 *   - Handles are opaque and owned by the library.  Input arrays are owned by
 *     the caller and copied before return.  Output buffers are caller-owned
 *     HOST memory unless stated otherwise.
 *   - Device memory comes from the optional allocator (NULL: cudaMalloc /
 *     cudaFree).  Streams are cudaStream_t passed as void* (NULL: the legacy
 *     default stream).  Work is enqueued asynchronously on the grid's stream;
 *     read functions synchronize that stream.
 *   - The library runs on the device current at fdtd_create_grid.  There is no
 *     CPU fallback: without a usable CUDA device every call that needs one
 *     returns FDTD_E_CUDA.
 */
#ifndef FDTD_H
#define FDTD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
enum {
  FDTD_OK = 0,
  FDTD_E_INVAL = -1,     /* bad argument (size, index, range, NULL)            */
  FDTD_E_NOMEM = -2,     /* allocator returned NULL                            */
  FDTD_E_CUDA = -3,      /* CUDA runtime error (message has the CUDA string)   */
  FDTD_E_STATE = -4,     /* call not allowed in the object's current state     */
  FDTD_E_NONFINITE = -5, /* a probe, flux or energy value became NaN or Inf    */
  FDTD_E_BUSY = -6,      /* request still pending                              */
  FDTD_E_TIMEOUT = -7,   /* a bounded wait ran out                             */
  FDTD_E_BUDGET = -8     /* request can never fit the server's memory budget   */
};

enum { FDTD_FP32 = 0, FDTD_FP64 = 1 };
enum { FDTD_INIT_STEADY = 0, FDTD_INIT_GROUND = 1 };
enum { FDTD_SRC_POINT = 0, FDTD_SRC_SHEET = 1 };

typedef struct fdtd_grid fdtd_grid;

/* Device allocator.  alloc returns device memory of `bytes` usable on
 * `stream`, aligned to 256 bytes, or NULL (a block that is not 256-byte
 * aligned is freed again and the call that needed it fails with E_NOMEM);
 * free releases it.  ctx is passed through. */
typedef struct fdtd_allocator {
  void* (*alloc)(size_t bytes, void* stream, void* ctx);
  void (*free)(void* ptr, size_t bytes, void* stream, void* ctx);
  void* ctx;
} fdtd_allocator;

/* Grid description (paper, Sec. "Sample and numerical approach": a box of
 * n^3 Yee cells with an absorbing layer, Courant step half the 3D limit).
 *   nx, ny, nz       cells per axis (each >= 1)
 *   npml[6]          absorbing-slab thickness on faces x-,x+,y-,y+,z-,z+
 *                    (0 = bare PEC wall; must be 0 on periodic axes)
 *   periodic[3]      1 = wrap the axis
 *   precision        FDTD_FP32 (fields, polarization, populations in binary32
 *                    with compensated population sums) or FDTD_FP64
 *   res, a           cells per lattice constant; lattice constant in metres
 *   courant          fraction of the 3D stability limit (S = courant/sqrt 3)
 *   eps[3]           relative permittivity of classes outside / background /
 *                    sphere (see fdtd_set_eps_from_spheres)
 *   cpml_*           grading order m, sigma_max factor (sigma_max dt/eps0 =
 *                    factor (m+1) S / sqrt(eps_outside)), kappa_max, alpha_max
 *                    (alpha dt/eps0 = alpha_max 2 pi f_ref dt), f_ref (a/lambda)
 *   seed             64-bit key of the spontaneous-emission noise
 *   record_capacity  probe / flux history kept on the device (steps, >= 1);
 *                    older entries are overwritten (ring) */
typedef struct fdtd_grid_desc {
  int32_t nx, ny, nz;
  int32_t npml[6];
  int32_t periodic[3];
  int32_t precision;
  int32_t reserved;   /* set to 0 (keeps the record free of padding) */
  double res, a, courant;
  double eps[3];
  double cpml_m, cpml_sigma_factor, cpml_kappa_max, cpml_alpha_max, cpml_f_hat;
  uint64_t seed;
  int64_t record_capacity;
} fdtd_grid_desc;

/* Create a grid: allocates the Yee fields (three sets of the six components:
 * a grid frozen on a TMA-staged kernel, paired or not, cycles through all
 * three so the observation of a step can overlap the next one, other grids
 * through two), the material bytes, the CPML auxiliary slabs and the
 * recorders, all zeroed.
 * The material starts as background class everywhere.
 * Errors: E_INVAL (sizes, npml on a periodic axis, npml >= axis length),
 * E_NOMEM, E_CUDA. */
int fdtd_create_grid(const fdtd_grid_desc* desc, const fdtd_allocator* alloc, void* stream,
                     fdtd_grid** out);

/* Release every device buffer (after synchronizing the grid's stream). NULL is a no-op. */
int fdtd_destroy_grid(fdtd_grid* g);

/* Rasterize the inverted opal on the device (paper, Sec. "Sample and
 * numerical approach": air spheres of radius r0 = a/(2 sqrt 2) in the fcc
 * lattice, disorder on radii).  spheres: n rows (cx, cy, cz, r) in grid units
 * (double, host).  box_lo/box_hi: structure box in grid units.  Per cell byte:
 * bits 2c..2c+1 = class of the E_c node (0 outside the box, 1 background,
 * 2 inside a sphere: strict (dx*dx+dy*dy)+dz*dz < r*r in FP64, each operation
 * rounded), bit 6 = cell centre inside a sphere and the box (gain cell).
 * Allowed before the first step only (E_STATE after). */
int fdtd_set_eps_from_spheres(fdtd_grid* g, const double* spheres, int64_t n, const double box_lo[3],
                              const double box_hi[3]);

/* Set / read the material bytes directly (uint8[nz][ny][nx], host), in the
 * layout above.  set: before the first step only; E_INVAL if a byte holds
 * class 3 in any of its three 2-bit fields or has bit 7 set. */
int fdtd_set_material(fdtd_grid* g, const uint8_t* mat);
int fdtd_get_material(fdtd_grid* g, uint8_t* mat);

/* Four-level gain medium in the cells whose bit 6 is set (paper, Secs.
 * "Sample and numerical approach" and "3+1D simulation of lasing").
 *   n_total    number density (m^-3)          fa_hat   transition a/lambda
 *   dw_rel     linewidth / omega_a            tau32, tau21, tau10  lifetimes (s)
 *   pump       rate 0 -> 3 (s^-1)             kappa    coupling (0: 6 pi eps0 c^3/(omega_a^2 tau21))
 *   noise_amp  std of the P~ kick per step (V/m) in gain cells
 *   init       FDTD_INIT_STEADY (N = N_eq) or FDTD_INIT_GROUND (all in level 0)
 * Polarization: P~^{n+1} = a1 P~^n - a2 P~^{n-1} + a3 (N1-N2) E^n + noise_amp xi.
 * Populations: Crank-Nicolson, stored as deviations from the pumped
 * equilibrium (FP32 runs add a compensation word per population).
 * Before the first step only; E_INVAL on non-positive lifetimes or density. */
typedef struct fdtd_gain_params {
  double n_total, fa_hat, dw_rel, tau32, tau21, tau10, pump, kappa, noise_amp;
  int32_t init;
} fdtd_gain_params;
int fdtd_set_gain(fdtd_grid* g, const fdtd_gain_params* p);

/* Where the Bloch variables of a gain cell live (paper, Sec. "Sample and
 * numerical approach": solved in the middle of the Yee cell).
 * FDTD_COUPLING_CELL (default): the polarization P~_c of cell (i,j,k) sits on
 * the node of E_c(i,j,k) and the cell's populations see its own three nodes.
 * FDTD_COUPLING_CENTRED: P~ and the populations sit at the cell centre; the
 * oscillator is driven by the average of the four E_c edges around the centre
 * (beyond the grid 0, or the periodic wrap), each E_c node receives the
 * average polarization current of the four cells that share it, and the
 * populations see the centre average of (E^{n+1}+E^n)/2, so the exchange of
 * energy between field and medium balances exactly.  Centred grids step their
 * fields with the passive step kernel plus three centred kernels per step,
 * and step alone (fdtd_batch_create refuses them).  Before the first step
 * only (E_STATE after); E_INVAL for another value. */
enum { FDTD_COUPLING_CELL = 0, FDTD_COUPLING_CENTRED = 1 };
int fdtd_set_gain_coupling(fdtd_grid* g, int32_t coupling);

/* Soft current source (paper, Secs. "Wide-band excitation" and "Dynamical
 * diffusion": single-cycle and 100 fs Gaussian pulses).  Waveform
 * g(n) = exp(-(t-t0)^2/(2 tau^2)) sin(2 pi f0 (t-t0)) at t = (n+1/2) dt,
 * tau = sqrt(ln 2)/(pi rel_bw f0), t0 = 5 tau unless t0_steps > 0.  The update
 * of E_comp subtracts amplitude * profile * g(n) / eps_r at the source nodes.
 * POINT: node (i,j,k).  SHEET: plane `index` normal to `axis`, over the
 * non-absorbing interior of the two transverse axes, profile
 * exp(-(du^2+dv^2)/waist^2) about the interior centre (waist 0 = uniform).
 * At most 8 sources; before the first step only. */
typedef struct fdtd_source_desc {
  int32_t kind, comp;
  int32_t i, j, k;
  int32_t axis, index;
  double waist, f0_hat, rel_bw, t0_steps, amplitude;
} fdtd_source_desc;
int fdtd_add_source(fdtd_grid* g, const fdtd_source_desc* s, int32_t* id);

/* Field probe at cell (i,j,k): after update n it records E^{n+1} (three
 * components) of that cell (paper, Sec. "Wide-band excitation": the field is
 * sampled at a generic point inside the crystal).  At most 64 probes; before
 * the first step only. */
int fdtd_add_probe(fdtd_grid* g, int32_t i, int32_t j, int32_t k, int32_t* id);

/* Poynting flux plane (paper, Sec. "Dynamical diffusion": the transmitted
 * power T(t) is the Poynting vector summed across the exit side of the
 * crystal).  Plane `index` normal
 * to `axis`; faces at ((u+1/2), (v+1/2)) for u in [u0,u1), v in [v0,v1) along
 * the cyclic transverse axes (axis+1)%3, (axis+2)%3.  During update n it
 * records T^n = sign dx^2 sum (E x H).n in watts, E at time n averaged onto the
 * face, H averaged over the two half steps and the two planes around it.
 * Requires 1 <= index <= n_axis-1 and ranges within [0, n-1].  At most 16
 * planes; before the first step only. */
int fdtd_add_flux_plane(fdtd_grid* g, int32_t axis, int32_t index, double sign, int32_t u0, int32_t u1,
                        int32_t v0, int32_t v1, int32_t* id);

/* Advance the grid by n >= 0 time steps (asynchronous on the grid's stream).
 * The first call freezes the set-up (sources, probes, flux planes, gain).
 * E_STATE if no permittivity map was set.  The recorders are rings: stepping
 * past record_capacity overwrites the oldest entries. */
int fdtd_step_n(fdtd_grid* g, int64_t n);

/* Launch shape of the step kernel: tile rows `by` (see fdtd_set_kernel for
 * how each kernel reads bx and by; before this call every kernel uses its
 * default tile), z-ranges of `zdepth` planes per work item (0: chosen from
 * the grid size; the TMA kernels cap it at 31), and grid_blocks > 0 makes the
 * launch persistent with that many blocks looping over the work items (0: one
 * block per item, except the paired kernel, which then runs one wave of
 * resident blocks and fetches each block's next item ahead).  Results do not
 * depend on the shape.  Needs bx, by >= 2, bx*by a multiple of 32, <= 512. */
int fdtd_set_launch(fdtd_grid* g, int32_t bx, int32_t by, int32_t zdepth, int32_t grid_blocks);

/* Order of the single-node kernels' work items within a launch:
 * FDTD_ORDER_COSTLIEST (default) issues the items whose tiles or planes
 * cross absorbing slabs first (items of equal cost in z order);
 * FDTD_ORDER_Z issues every item in z order (z-range, then row, then column
 * of tiles), so neighbouring tiles run together and the halo rows and
 * columns they share are read from DRAM once.  The paired kernel keeps its
 * own cost-bucketed z order.  Results do not depend on the order.  A launch
 * parameter of this library: the paper has no counterpart.  E_INVAL for
 * another value. */
enum { FDTD_ORDER_COSTLIEST = 0, FDTD_ORDER_Z = 1 };
int fdtd_set_item_order(fdtd_grid* g, int32_t order);

/* Absorbing layer of the grid's slabs (paper, Sec. "Sample and numerical
 * approach": a uniaxial PML).  FDTD_ABSORBER_CPML (default): the convolutional
 * PML of the descriptor's grading, inside the fused step kernels.
 * FDTD_ABSORBER_UPML: the uniaxial PML on the same grading of sigma and
 * kappa (alpha unused), at each field node's own position on every axis; a
 * node where any axis is graded steps through an auxiliary D~ (E) or B~ (H~):
 * D~' = [(k1 - s1/2) D~ + S curl H~]/(k1 + s1/2) on the axis d1 after the
 * component c, E' = [(k2 - s2/2) E + ((kc + sc/2) D~' - (kc - sc/2) D~)/eps_r]
 * /(k2 + s2/2) on c and the axis d2 after d1 (s = sigma dt/eps0), and H~
 * likewise with -S curl E.  Sources act outside the layer only.  UPML grids
 * step with two launches per step (H~, then E, one thread per node;
 * fdtd_kernel_in_use reports kind 4), passive grids only (E_INVAL with a
 * gain medium), stepping alone (fdtd_batch_create refuses them).  Before the
 * first step only (E_STATE after). */
enum { FDTD_ABSORBER_CPML = 0, FDTD_ABSORBER_UPML = 1 };
int fdtd_set_absorber(fdtd_grid* g, int32_t absorber);

/* Step-kernel variant: 0 = automatic (the paired kernel for binary32 and
 * the TMA-staged kernel for binary64 grids when no axis is periodic, else the
 * plain-load kernel), 1 = plain-load kernel (blocks of bx x by threads own
 * (bx-1) x (by-1) columns; default 32 x 8), 2 = TMA-staged kernel (blocks of
 * 32 x by threads own 32 x by columns, by 4 or 8, default 8; E_INVAL on
 * periodic grids), 3 = paired TMA-staged kernel, binary32 grids only (each
 * thread updates two x-adjacent nodes with packed f32x2 arithmetic; tiles of
 * 32 x by columns, by 8 or 16, default 16; E_INVAL on periodic or binary64
 * grids).  A launch shape a kernel cannot take selects the next more general
 * one (3 -> 2 -> 1).  All perform the same arithmetic per node and give
 * identical results. */
int fdtd_set_kernel(fdtd_grid* g, int32_t kind);

/* Persisting L2 window of the CPML memory: on = 1 (the default) keeps the
 * grid's CPML auxiliary arrays in a persisting L2 window on the grid's
 * stream while it steps.  One grid per device holds the window at a time:
 * the one that stepped alone most recently (another grid's step, a batch's
 * step, switching it off or destroying the grid clears the window and returns
 * its lines to normal).  It raises the context's persisting-L2 set-aside
 * (cudaLimitPersistingL2CacheSize) to the arrays' size, at most the device's
 * maximum, and replaces any access-policy window the caller set on that
 * stream.  A cache placement of this library, no counterpart in the paper:
 * no result changes.  E_INVAL for another value. */
int fdtd_set_l2_residency(fdtd_grid* g, int32_t on);

/* The step kernel the grid's launches use under its current settings
 * (1 plain, 2 TMA, 3 paired, 4 the UPML launches), and the rows of its tile (*rows: the tile of
 * owned columns is 32 x rows for kinds 2 and 3, (bx-1) x (by-1) for kind 1).
 * Valid after the first step (or a batch build); E_STATE before. */
int fdtd_kernel_in_use(fdtd_grid* g, int32_t* kind, int32_t* rows);

/* Launch-shape autotuner (no counterpart in the paper: it serves the
 * stepping of many realizations).  Times each candidate launch shape (step
 * kernel, tile rows, z-range depth, and for batches the persistent grid) for
 * trial_steps steps after two warm-up steps, starting every trial from the
 * current state and restoring the state afterwards (fields, CPML and gain
 * memory, recorder rings, step counters), then keeps the fastest shape.  The
 * candidates perform identical arithmetic, so no result changes.  Needs free
 * device memory for one copy of the state (plain cudaMalloc, not the grid's
 * allocator; E_NOMEM otherwise).  out (nullable) receives the choice. */
typedef struct fdtd_tune_result {
  int32_t kernel;       /* fdtd_set_kernel kind (0 = automatic)             */
  int32_t bx, by;       /* launch shape (by 0 = the kernel's default rows)  */
  int32_t zdepth;       /* planes per work item (0 = automatic)            */
  int32_t grid_blocks;  /* persistent blocks (0 = the kernel's default)     */
  int32_t candidates;   /* shapes timed                                     */
  double ms_per_step;   /* time of one step with the chosen shape           */
  int32_t order;        /* item order (fdtd_set_item_order)                 */
} fdtd_tune_result;
int fdtd_autotune(fdtd_grid* g, int32_t trial_steps, fdtd_tune_result* out);

/* Per-launch timing of the step kernel: on = 0 switches it off; on = k >= 1
 * brackets every k-th step-kernel launch (the first, the (k+1)-th, ...) by a
 * pair of CUDA events on the grid's stream (k > 1 keeps the event overhead
 * off most launches).  fdtd_kernel_time synchronizes and returns the summed
 * duration (ms) of the bracketed launches and their number. */
int fdtd_set_timing(fdtd_grid* g, int32_t on);
int fdtd_kernel_time(fdtd_grid* g, double* ms, int64_t* launches);

/* Wait for the grid's stream; returns E_NONFINITE if the device raised the
 * non-finite flag (checked on probes, flux and energy). */
int fdtd_sync(fdtd_grid* g);

/* Steps completed (host-side count of enqueued steps). */
int fdtd_steps_done(fdtd_grid* g, int64_t* n);

/* Probe history: out[count][3] (double, host) for updates t0 .. t0+count-1.
 * E_INVAL if the range is not within the last record_capacity steps. */
int fdtd_read_probes(fdtd_grid* g, int32_t id, int64_t t0, int64_t count, double* out);

/* Flux history: out[count] (double, host) of T^n for n = t0 .. t0+count-1. */
int fdtd_read_flux(fdtd_grid* g, int32_t id, int64_t t0, int64_t count, double* out);

/* Current fields, comp 0..5 = Ex, Ey, Ez, H~x, H~y, H~z: E at time n, H~ at
 * time n-1/2 (n = steps done), as double[nz][ny][nx] (host). */
int fdtd_read_fields(fdtd_grid* g, int32_t comp, double* out);
/* Overwrite one field component of the current time level (before the first
 * step only), same layout. */
int fdtd_write_fields(fdtd_grid* g, int32_t comp, const double* in);

/* Gain state as double[3][nz][ny][nx] (host): what = 0 -> P~^n, 1 -> P~^{n-1},
 * 2 -> populations N1, N2, N3 (m^-3; N0 = n_total - N1 - N2 - N3 in gain
 * cells), 3 -> deviations N1..N3 - N_eq (m^-3) as carried by the update;
 * zero outside gain cells.  E_STATE without gain. */
int fdtd_read_gain(fdtd_grid* g, int32_t what, double* out);

/* Field energy 1/2 eps0 dx^3 (sum eps_r E^2 + sum H~^2) in joules at the
 * current time level (E^n, H~^{n-1/2}), reduced on the device in FP64 in a
 * fixed order (bitwise reproducible for a given grid size). */
int fdtd_field_energy(fdtd_grid* g, double* out);

/* Stop a grid at update `limit`: steps n >= limit are not performed (by
 * fdtd_step_n or a batch).  Default: no limit. */
int fdtd_set_step_limit(fdtd_grid* g, int64_t limit);

/* Limit, in nanoseconds, of every wait of the TMA-staged step kernels for a
 * staged plane of this grid (default 2e9).  A wait that runs out makes the
 * kernel let its copies in flight land (each within 2 s), stop its block and
 * flag the grid, and the next fdtd_sync / read returns FDTD_E_TIMEOUT; the
 * CUDA context stays usable, the grid's state is then undefined.  0 makes
 * every such wait give up at once without looking at the copy (a healthy
 * run's way to test that error path).  The paper has no counterpart: this is
 * the library's guard against a copy that never completes.  E_INVAL if
 * ns < 0.  Takes effect at the next step call; a batch takes each member's
 * limit when it is created. */
int fdtd_set_wait_limit(fdtd_grid* g, int64_t ns);

/* ---------------------------------------------------------------- batches
 * Many grids of mixed size stepped together (the disorder realizations of the
 * paper, Sec. "Wide-band excitation and gap filling", are independent runs):
 * one step-kernel launch per time step covers the work items of every member,
 * followed by one observation launch.  Members keep their own counters and
 * step limits; reads go through the member grids as usual.  All members must
 * have the same precision; the batch does not own them (destroy the batch
 * first).  Set-up of the members must be complete (their first step freezes
 * it).  Work is enqueued on the batch's stream; member streams are made to
 * wait for it. */
typedef struct fdtd_batch fdtd_batch;
int fdtd_batch_create(fdtd_grid* const* grids, int32_t n, void* stream, fdtd_batch** out);
int fdtd_batch_destroy(fdtd_batch* b);
/* kernel: as fdtd_set_kernel; by: rows of the tile (0: the kernel's
 * default); zdepth: planes per work item (0: 16); grid_blocks > 0: persistent
 * launch with that many blocks.  Members that cannot share the kernel or the
 * tile all fall back to the more general kernel. */
int fdtd_batch_set_launch(fdtd_batch* b, int32_t kernel, int32_t by, int32_t zdepth, int32_t grid_blocks);
/* Capture `steps_per_graph` steps (step + observation launches and the
 * counter update) into a CUDA graph replayed by fdtd_batch_step_n; 0 = off.
 * Per-launch timing (fdtd_batch_set_timing) uses direct launches. */
int fdtd_batch_set_graph(fdtd_batch* b, int32_t steps_per_graph);
int fdtd_batch_step_n(fdtd_batch* b, int64_t n);
int fdtd_batch_sync(fdtd_batch* b);
int fdtd_batch_set_timing(fdtd_batch* b, int32_t on);
int fdtd_batch_kernel_time(fdtd_batch* b, double* ms, int64_t* launches);
/* As fdtd_autotune, over the batch's launch shapes, restoring every member. */
int fdtd_batch_autotune(fdtd_batch* b, int32_t trial_steps, fdtd_tune_result* out);

/* ---------------------------------------------------------------- serving
 * A request server keeps runs (disorder realizations, pulse or lasing runs of
 * any grid size) resident on the device and steps them together: requests
 * arriving while others run are admitted at chunk boundaries as slots and
 * memory free up (first in, first out), their work shares the step launches,
 * and each run stops exactly at its own step count, so its results do not
 * depend on the other runs.  Device memory comes from the stream-ordered
 * pool; admission keeps the estimated bytes of resident runs within the
 * budget.  A worker thread does all device work. */
typedef struct fdtd_server fdtd_server;

typedef struct fdtd_server_desc {
  int64_t hbm_budget_bytes;  /* device bytes resident runs may hold */
  int32_t max_slots;         /* resident runs at most */
  int32_t steps_per_chunk;   /* steps between admission / retirement points */
  int32_t precision;         /* FDTD_FP32 or FDTD_FP64 (all requests) */
  int32_t graph;             /* 1: replay chunks as CUDA graphs */
} fdtd_server_desc;

typedef struct fdtd_flux_desc {
  int32_t axis, index, u0, u1, v0, v1;
  double sign;
} fdtd_flux_desc;

/* One run.  All arrays are caller-owned and copied by fdtd_submit. */
typedef struct fdtd_request {
  fdtd_grid_desc grid;              /* record_capacity is set to `steps` */
  const double* spheres;            /* n_spheres x (cx, cy, cz, r), grid units */
  int64_t n_spheres;
  double box_lo[3], box_hi[3];
  const fdtd_gain_params* gain;     /* NULL: passive */
  const fdtd_source_desc* sources;
  int32_t n_sources;
  const int32_t* probes;            /* n_probes x (i, j, k) */
  int32_t n_probes;
  const fdtd_flux_desc* fluxes;
  int32_t n_fluxes;
  int64_t steps;
} fdtd_request;

typedef struct fdtd_result {
  int32_t status;         /* FDTD_OK, FDTD_E_BUSY (pending) or the run's error */
  int64_t steps;
  double submit_s, admit_s, done_s;  /* seconds since the server started */
  double field_energy;    /* joules after the last step */
  int32_t n_probes, n_fluxes;
} fdtd_result;

typedef struct fdtd_server_stats {
  int64_t submitted, admitted, completed, failed, chunks;
  int64_t cell_updates;   /* of completed runs */
  int32_t resident, queued;
  int64_t used_bytes;
} fdtd_server_stats;

/* E_INVAL for a null argument or a budget, slot count or chunk that is not
 * positive; E_CUDA without a CUDA device; E_NOMEM if the worker thread cannot
 * start.  `stream` is unused (the worker owns its stream).  As everywhere in
 * this header, failures come back as codes: no C++ exception leaves a call. */
int fdtd_server_create(const fdtd_server_desc* desc, void* stream, fdtd_server** out);
/* Fails queued requests, finishes resident runs, joins the worker. */
int fdtd_server_destroy(fdtd_server* s);
/* E_BUDGET if the run alone exceeds the budget; E_INVAL on bad arrays. */
int fdtd_submit(fdtd_server* s, const fdtd_request* req, uint64_t* ticket);
/* timeout_ms 0: returns FDTD_E_BUSY while pending; > 0: waits up to that long
 * and returns FDTD_E_TIMEOUT if still pending.  Fills `out` in every case. */
int fdtd_poll(fdtd_server* s, uint64_t ticket, fdtd_result* out, int32_t timeout_ms);
/* Results of a completed run: probes as double[steps][n_probes][3], flux as
 * double[n_fluxes][steps] (caller-owned host buffers). */
int fdtd_result_probes(fdtd_server* s, uint64_t ticket, double* out);
int fdtd_result_flux(fdtd_server* s, uint64_t ticket, double* out);
/* Forget a finished run's results. */
int fdtd_result_release(fdtd_server* s, uint64_t ticket);
int fdtd_server_get_stats(fdtd_server* s, fdtd_server_stats* out);

/* Field energy 1/2 eps0 dx^3 (sum eps_r E^2 + sum H~^2) in joules of
 * caller-owned DEVICE arrays, computed without allocating any memory.
 * The paper has no counterpart: this is for callers that cannot allocate
 * device memory where they need the number (another framework owns the
 * allocator, a real-time loop must not enter it, a tool inspects fields in
 * place).  fields: six device pointers Ex, Ey, Ez, H~x, H~y, H~z, each
 * [nz][ny][pitch] elements of the given precision with x fastest; mat: device
 * material bytes in the same layout (eps[class] per E node, as in
 * fdtd_set_eps_from_spheres); dx: cell size in metres; stream: cudaStream_t
 * or NULL; out: HOST double.  The reduction scratch is a fixed file-scope
 * device array holding 2048 partial sums: at most 134,217,728 cells (2048 x
 * 65536); larger inputs return E_INVAL.  The call synchronizes `stream`.
 * Every call shares that scratch and leaves the last call's contents there;
 * calls that overlap on the GPU race, so serialize them.  The scratch's
 * device address is looked up on every call whose stream is not being
 * captured (a device reset may move it) and remembered per device for calls
 * made during a capture, so make the first call on each device before
 * capturing a stream into a CUDA graph. */
int fdtd_field_energy_noalloc(const void* const fields[6], const uint8_t* mat, int32_t nx, int32_t ny, int32_t nz,
                              int32_t pitch, int32_t precision, const double eps[3], double dx, void* stream,
                              double* out);

/* Checkpoint: write / read every state array (fields, CPML slabs, gain state,
 * step count, recorders) to / from a file.  load requires a grid created
 * with the same description; it may step with another kernel than the grid
 * that saved (the current field set is moved into its own cycle). */
int fdtd_save_state(fdtd_grid* g, const char* path);
int fdtd_load_state(fdtd_grid* g, const char* path);

/* Message of the last error on the calling thread ("" if none). */
const char* fdtd_last_error(void);

/* Library build information (static string). */
const char* fdtd_version(void);

#ifdef __cplusplus
}
#endif
#endif /* FDTD_H */
