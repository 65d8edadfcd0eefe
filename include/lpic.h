/*
 * lpic.h -- C ABI of liblpic: the hot path of the explicit electromagnetic
 * particle-in-cell timestep of lambdaPIC (Algorithm 1 without QED, load
 * balancing or MPI) on one NVIDIA B300 (sm_103a).
 *
 * Per particle: field gather from the Yee grid (Sec. 3.1), relativistic Boris
 * push (Sec. 3.1), Esirkepov charge-conserving current deposit (Sec. 3.1); per
 * grid: the Yee FDTD update split in two dt/2 halves (Sec. 3.2 Eq. 1-4,
 * Algorithm 1), with periodic or absorbing (first-order Mur) x edges and an
 * incoming laser at x-min (Sec. 4.2).
 *
 * Conventions shared by every call
 * --------------------------------
 * Units: normalised, c = eps0 = 1, charges in |e|, masses in m_e.
 * Memory: every data pointer is a DEVICE pointer owned by the caller
 *   (borrowed: it must stay valid until lpic_destroy_grid).  The library owns
 *   only its scratch (sort keys, tile tables, status word), allocated in
 *   lpic_create_grid / lpic_add_species and freed in lpic_destroy_grid.  No
 *   call allocates after lpic_add_species.
 * Streams: calls taking a cudaStream_t enqueue work on that stream and return
 *   without synchronising, except where "synchronises" is stated.  The
 *   non-synchronising calls are capturable in a CUDA graph.
 * Errors: every call returns an lpic_status.  Argument errors are detected on
 *   the host and returned at once (nothing is enqueued); CUDA launch errors
 *   return LPIC_ECUDA.  Errors found by kernels (a particle that moved a full
 *   cell, left its tile's halo or an absorbing edge region, a non-finite
 *   momentum) set bits of a device status word that lpic_check_status
 *   returns.  lpic_last_error() gives a message for the calling thread's last
 *   failure.  No C++ exception crosses this interface.
 *
 * Field layout: each component is a dense row-major array [nz][ny][fx]
 *   (nz = 1 in 2D), fx = nx for periodic x and nx + 1 for absorbing x.  Index
 *   (i, j, k) of a component stands for its staggered Yee position:
 *     E_x (i+1/2, j, k)   E_y (i, j+1/2, k)   E_z (i, j, k+1/2)
 *     B_x (i, j+1/2, k+1/2)   B_y (i+1/2, j, k+1/2)   B_z (i+1/2, j+1/2, k)
 *   and J is co-located with E.  In 2D the k offsets are dropped.  Element
 *   types: LPIC_FP64 -> E, B, J double; LPIC_FP32_FIXED -> E, B float and J
 *   int64 fixed point (J_c = J_int * lpic_grid_info.j_scale[c]).
 *
 * Particle layout: a species lives in two caller-owned device buffers (ping
 *   and pong).  The sort moves particles from the current buffer to the other
 *   one and flips them; lpic_species_query tells which one is current.  Each
 *   buffer is a struct of arrays, every array `capacity` entries long, in
 *   this order (capacity must be a multiple of 64, so every array starts on
 *   a 256-byte boundary):
 *     LPIC_FP32_FIXED: int32 cell, float off[dim], float u[3], float w, int32 id
 *        cell = (k * ny + j) * nx + i of the particle's cell (-1 = removed),
 *        off = in-cell offsets in [0, 1) (cell units).
 *     LPIC_FP64:       double x[dim], double u[3], double w, int32 id
 *        x = physical position, w = 0 marks a removed particle.
 *   u = gamma v / c.  Particles are stored leapfrog-style: at the loop
 *   boundary t_n the buffers hold x^{n+1/2} = x^n + (dt/2) v^n and u^n (the
 *   second half push of one step and the first half push of the next, which
 *   use the same velocity, are fused).  lpic_positions_at_step returns x^n.
 */
#ifndef LPIC_H
#define LPIC_H

#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LPIC_OK = 0,
    LPIC_EINVAL = 1,        /* bad argument or descriptor */
    LPIC_ENOMEM = 2,        /* scratch allocation failed */
    LPIC_ECUDA = 3,         /* a CUDA runtime call or launch failed */
    LPIC_EDEVICE = 4,       /* lpic_check_status: a kernel set status bits */
    LPIC_EUNSUPPORTED = 5   /* valid but not supported combination */
} lpic_status;

/* device status bits (lpic_check_status) */
#define LPIC_ST_CFL       0x1u  /* a particle moved >= 1 cell in a step */
#define LPIC_ST_HALO      0x2u  /* a particle outside its tile's box where no global-
                                   memory path exists (unfused stages, ensembles); it is
                                   skipped */
#define LPIC_ST_NAN       0x4u  /* non-finite momentum */
#define LPIC_ST_OUTSIDE   0x8u  /* a deposit or gather reached past an absorbing edge */
#define LPIC_ST_OVERFLOW  0x10u /* a fixed-point value exceeded its bound */
#define LPIC_ST_BOUNDS    0x20u /* checked build (liblpic_check.so, LPIC_CHECK=1) only:
                                   a shared-memory index of the gather or the current
                                   box fell outside its box; the access was skipped */

enum { LPIC_FP64 = 0, LPIC_FP32_FIXED = 1 };

typedef struct lpic_grid *lpic_grid_t;    /* opaque, owned by the library */

/* Incoming laser at x-min (Sec. 4.2): E_y polarised,
 * E_inc(x, y, z, t) = a0 sin^2(pi s / tau) exp(-r^2 / w0^2) sin(omega s),
 * s = t - x in (0, tau), r^2 = (y - yc)^2 + (z - zc)^2 (no z term in 2D). */
typedef struct {
    double a0, w0, tau, omega, yc, zc;
} lpic_laser_desc;

typedef struct {
    int dim;                    /* 2 (2D3V) or 3 (3D3V) */
    int nx, ny, nz;             /* cells per dimension; nz ignored in 2D */
    double dx, dy, dz, dt;      /* cell sizes and time step; dz ignored in 2D.
                                   dt must satisfy the Courant limit of Sec. 3.2 */
    int absorb_x;               /* 0: periodic x; 1: absorbing x edges (first-order Mur,
                                   laser entering through the x-min edge); 2: CPML layers
                                   (pml_* below, laser entering as a current sheet on
                                   node plane pml_cells + 2) */
    int shape_order;            /* 1: cloud-in-cell, 2: quadratic spline (TSC) */
    int precision;              /* LPIC_FP64 or LPIC_FP32_FIXED */
    int tile[3];                /* cells per tile for the FP32 path; 0 = default */
    int block_particles;        /* FP32 path: at most this many particles per thread block
                                   (a crowded tile is split into several work items);
                                   0 = default (4096), else in [256, 2^20] */
    int sort_interval;          /* FP32 path: lpic_step sorts every sort_interval steps
                                   (0 or 1: every step); the tiles then carry a margin of
                                   ceil((sort_interval - 1) c dt / h) cells for the drift
                                   (less if the boxes would not fit in shared memory);
                                   particles beyond it take a global-memory path */
    void *E[3], *B[3], *J[3];   /* caller-owned device field arrays (see layout) */
    const lpic_laser_desc *laser; /* NULL: no laser; copied at create (needs absorb_x) */
    /* CPML (absorb_x = 2; Sec. 3.2 names CPML absorbing boundaries): layers of
     * pml_cells cells at both x ends in which the x derivatives of the field
     * updates become (1/kappa) d/dx + psi with the recursive convolution
     * psi <- b psi + a d/dx, b = exp(-(sigma/kappa + alpha) dt/2),
     * a = sigma (b - 1) / (sigma kappa + kappa^2 alpha), per half step; over the
     * depth d in [0, 1] into a layer sigma = pml_sigma_max d^pml_m,
     * kappa = 1 + (pml_kappa_max - 1) d^pml_m, alpha = pml_alpha_max (1 - d).
     * The outer faces are perfect conductors.  Requires 1 <= pml_cells and
     * 2 pml_cells + 8 <= nx; ignored unless absorb_x = 2. */
    int pml_cells;
    double pml_m, pml_sigma_max, pml_kappa_max, pml_alpha_max;
    /* FP32_FIXED path only: 1 keeps FP64 master fields (E and B are double
     * arrays; the Maxwell half steps of Sec. 3.2, Eq. 1-4, run in double with
     * the int64 current converted in double, and the particle kernels round
     * the fields to float once, when the tile kernel stages them in shared
     * memory).  The Gauss-law residual then stays constant to double
     * rounding.  Not with the QED passes or in an ensemble. */
    int maxwell_fp64;
} lpic_grid_desc;

typedef struct {
    double q, m;                /* charge (|e| units, signed) and mass (m_e units); m = 0 with
                                   q = 0 is a massless species (photons; FP32_FIXED path): it
                                   moves at c along u, sees no field, deposits nothing, and its
                                   energy in lpic_diagnostics is w |u| */
    long long count;            /* particles in buffers[0] at add time (first count entries) */
    long long capacity;         /* entries per array, multiple of 64, >= count */
    void *buffers[2];           /* two device buffers of lpic_species_bytes() bytes */
    int staggered;              /* 0: buffers hold x^0, add_species advances them by dt/2;
                                   1: they already hold x^{1/2} */
    double max_weight;          /* bound on |w| of particles created in this species later
                                   (Breit-Wheeler pairs); the fixed-point shift covers
                                   max(this, the largest |w| in the buffer); 0 = none */
} lpic_species_desc;

typedef struct {
    int fixed_shift;            /* F: FP32 path J_int unit is 2^-F charge */
    double j_scale[3];          /* J_c = J_int * j_scale[c] (FP32 path) */
    double rho_scale;           /* rho = rho_int * rho_scale (FP32 path) */
    int tile[3];                /* tile shape in use */
    long long ntiles;
    int fx;                     /* stored x extent of the field arrays */
    long long launches;         /* kernel launches issued so far by calls on this grid */
} lpic_grid_info;

typedef struct {
    double kinetic;             /* sum_p w m (gamma - 1), gamma from u^n */
    double field;               /* (1/2) sum (E^2 + B^2) dV over stored positions */
    double charge;              /* sum_p q w */
    long long particles;        /* alive particles, all species */
} lpic_diag;

/* Size in bytes of one species buffer (ping or pong). */
size_t lpic_species_bytes(int dim, int precision, long long capacity);

/* Create a grid from a descriptor (Sec. 3.2 grid; Sec. 2.1 Patches
 * replaced by one guard-less global grid per instance).  Checks the
 * descriptor (dimensions: at least 4 cells each and field arrays of fewer
 * than 2^31 nodes; Courant limit, shape order, laser needs absorbing x, tile
 * shape) and allocates the library's scratch.  Synchronous. */
lpic_status lpic_create_grid(const lpic_grid_desc *desc, lpic_grid_t *out);

/* Free the library's scratch (not the caller's buffers).  Synchronises the
 * device.  NULL is accepted. */
lpic_status lpic_destroy_grid(lpic_grid_t grid);

/* Register a species (Sec. 2.1 Species): checks the descriptor, allocates the
 * per-species scratch, computes the fixed-point shift F from the bound
 * sum_s capacity_s * max|q w|_s so that no int64 current can overflow, and,
 * unless staggered, advances positions by dt/2.  Must be called before the
 * first lpic_gather_push_deposit.  Synchronises `stream`. */
lpic_status lpic_add_species(lpic_grid_t grid, const lpic_species_desc *desc,
                             cudaStream_t stream, int *species_id);

/* Which buffer is current (0 or 1) and how many particles it holds (alive
 * particles first after a sort).  Synchronises `stream`. */
lpic_status lpic_species_query(lpic_grid_t grid, int species_id, cudaStream_t stream,
                               int *current_buffer, long long *count);

/* What a checkpoint needs besides the caller-owned buffers: the weight bound
 * the species was registered with (max |w| at add time, or max_weight if
 * larger; it sets the fixed-point shift, so a restored grid given the same
 * bounds and capacities gets the same shift and can take the saved integer
 * current as it is) and the id its next created particle will get.
 * Synchronises `stream`. */
lpic_status lpic_species_checkpoint_info(lpic_grid_t grid, int species_id, cudaStream_t stream,
                                         double *max_weight, long long *next_id);

/* Sort a species by cell tile (Algorithm 1 "sort particles by cell index"):
 * counting sort (histogram, scan, scatter) from the current buffer into the
 * other one, dropping removed particles; then the buffers flip.  Within a
 * tile the order is not specified.  species_id -1 sorts every species. */
lpic_status lpic_sort_particles(lpic_grid_t grid, int species_id, cudaStream_t stream);

/* Zero the current array J (before the species loop of a step). */
lpic_status lpic_zero_current(lpic_grid_t grid, cudaStream_t stream);

/* The fused particle kernel (Sec. 2.3 "unified pusher", Algorithm 1 particle
 * loop): for each particle of the species, gather E and B at x^{n+1/2}
 * (Sec. 3.1), Boris u^n -> u^{n+1} (Sec. 3.1), advance the position by
 * dt v^{n+1} to x^{n+3/2}, and add the Esirkepov current of that straight
 * path (Sec. 3.1) to J.  FP64 path: one thread per particle, double atomics.
 * FP32 path: needs the species sorted by tile within its last sort_interval
 * pushes; one thread block per tile with the tile's E/B halo and
 * an int64 fixed-point J accumulator in shared memory, flushed once per tile
 * with integer atomics (deterministic, bit-exact continuity). */
lpic_status lpic_gather_push_deposit(lpic_grid_t grid, int species_id, cudaStream_t stream);

/* One Maxwell half step (Sec. 3.2 Eq. 3-4, split as in Algorithm 1) from t to
 * t + dt/2.  half = 0: E += (dt/2)(curl B - J), then B -= (dt/2) curl E;
 * half = 1: B first, then E.  Absorbing x edges use first-order Mur on E_y,
 * E_z with the laser (if any) entering at x-min. */
lpic_status lpic_maxwell_half_step(lpic_grid_t grid, int half, double t, cudaStream_t stream);

/* One full step t -> t + dt (Algorithm 1): Maxwell half 0, zero J, per
 * species sort (FP32 path, every sort_interval steps; the push before a sort
 * also builds the next sort's tile histogram) and gather_push_deposit,
 * Maxwell half 1. */
lpic_status lpic_step(lpic_grid_t grid, double t, cudaStream_t stream);

/* Set the device clock that captured steps read the laser time from. */
lpic_status lpic_set_clock(lpic_grid_t grid, double t, cudaStream_t stream);

/* Run nsteps full steps (as lpic_step) by replaying CUDA graphs: the first
 * call for a given buffer parity captures one step on `stream` (thread-local
 * capture) and instantiates it; later calls only launch.  The laser time is
 * the device clock (lpic_set_clock), which each replay advances by dt.  A
 * graph holds the species buffer pointers of its parity, so adding species or
 * changing buffers after the first capture is not supported.  `stream` must
 * be a created stream (the legacy default stream cannot be captured). */
lpic_status lpic_graph_steps(lpic_grid_t grid, int nsteps, cudaStream_t stream);

/* Charge density of the stored positions x^{n+1/2} (the charge the deposit
 * conserves, Sec. 3.1), added into rho[nz][ny][fx]: FP64 path double
 * q w S / dV; FP32 path int64 sum of rint(2^F q w S) with the same shape
 * arithmetic as the deposit (rho = rho_int * rho_scale). */
lpic_status lpic_deposit_charge(lpic_grid_t grid, int species_id, void *rho, cudaStream_t stream);

/* The unfused path (Sec. 2.3 "Callback system" and Sec. 3.3: the paper fuses
 * position push, field interpolation, momentum push and deposition into one
 * loop only when no callback sits between them).  Stage 1,
 * lpic_gather_fields, sorts the species by tile if it was pushed since its
 * last sort, then writes each particle's six interpolated field components
 * (E_x, E_y, E_z, B_x, B_y, B_z at x^{n+1/2}, the fused kernel's gather) to
 * the caller's device array fields[6][capacity] (float), indexed like the
 * current particle buffer.  Between the stages the caller may read or change
 * those fields with its own kernels on `stream` (an external field, a
 * per-particle diagnostic).  Stage 2, lpic_push_deposit_fields, then pushes
 * and deposits the species exactly as lpic_gather_push_deposit would, with
 * the fields read from the array; it must follow stage 1 of the same species
 * with no sort or push in between (else LPIC_EINVAL).  With unchanged fields
 * the two stages give bit-identical results to the fused call.  FP32 path
 * only (LPIC_EUNSUPPORTED otherwise).  Asynchronous on `stream`. */
lpic_status lpic_gather_fields(lpic_grid_t grid, int species_id, float *fields, cudaStream_t stream);
lpic_status lpic_push_deposit_fields(lpic_grid_t grid, int species_id, const float *fields,
                                     cudaStream_t stream);

/* Species-resolved fields (Sec. 6.1): one lpic_step of `grid` that also
 * advances the fields of `aux` with the current of species `species_id`
 * alone as the source (Maxwell's equations are linear, so aux holds the
 * field that species radiates).  aux is another grid with the same
 * geometry, time step, precision and x boundary and no species (its laser,
 * if any, is its own); the species is deposited first and its current copied
 * into aux's J, then the other species deposit on top.  Asynchronous on
 * `stream`. */
lpic_status lpic_step_resolved(lpic_grid_t grid, double t, int species_id, lpic_grid_t aux,
                               cudaStream_t stream);

/* Gauss's law diagnostic (Sec. 3.2; Sec. 4.1 checks charge conservation):
 * the discrete divergence of the current E at the integer nodes,
 * sum_d (E_d(i+1/2) - E_d(i-1/2)) / h_d, in double, written to the caller's
 * device array out[nz][ny][fx] (overwritten; periodic wrap, E_x = 0 below an
 * absorbing x-min edge).  After each step the residual
 * div E - (rho(x^{n+3/2}) + rho(x^{n+1/2})) / 2 of the stored positions before
 * and after the step is the same at every node, because E changes only
 * through the current, which conserves that charge. */
lpic_status lpic_div_e(lpic_grid_t grid, double *out, cudaStream_t stream);

/* Write x^n = x^{n+1/2} - (dt/2) v^n as doubles, out[d * capacity + p] for
 * d < dim, in current-buffer order (removed particles give NaN). */
lpic_status lpic_positions_at_step(lpic_grid_t grid, int species_id, double *out,
                                   cudaStream_t stream);

/* FP64 energy and charge reductions (Sec. 4.1 energy diagnostic).
 * Synchronises `stream`. */
lpic_status lpic_diagnostics(lpic_grid_t grid, lpic_diag *out, cudaStream_t stream);

lpic_status lpic_grid_get_info(lpic_grid_t grid, lpic_grid_info *out);

/* Benchmark timing of the fused particle kernel: lpic_kernel_timing(g, n)
 * (re)starts recording CUDA events on the launching stream around the next n
 * launches of that kernel (0 stops); lpic_kernel_time waits for them and
 * returns the summed elapsed milliseconds and the number of timed launches.
 * Eager calls only (not under graph capture). */
lpic_status lpic_kernel_timing(lpic_grid_t grid, int max_launches);
lpic_status lpic_kernel_time(lpic_grid_t grid, double *ms, long long *launches);

/* Synchronise `stream`, return the device status bits in *bits and clear
 * them; returns LPIC_EDEVICE when any bit was set. */
lpic_status lpic_check_status(lpic_grid_t grid, cudaStream_t stream, unsigned *bits);

/* Ensembles: many independent grids stepped together (batched scheduling).
 * One launch per field pass and per sort pass covers every grid, and one
 * persistent particle kernel takes (species, work item) entries from a
 * device queue that visits the densest species first.  Each grid keeps its
 * own tile shape and block_particles (a sparse member can take larger tiles
 * than a dense one); the persistent kernel reserves the largest member's
 * shared memory per block.  Requirements: at least one grid; all grids on the
 * FP32_FIXED path with the same dimension and shape order, sort_interval <= 1,
 * periodic boundaries and no laser; every grid has its species added and all
 * species buffers at the same parity.  The grids stay owned by the caller and must
 * outlive the ensemble; while it exists they are stepped through it (queries
 * and diagnostics on the grids remain valid). */
typedef struct lpic_ensemble *lpic_ensemble_t;
lpic_status lpic_create_ensemble(lpic_grid_t *grids, int n, lpic_ensemble_t *out);
lpic_status lpic_destroy_ensemble(lpic_ensemble_t ensemble);
/* One step of every grid (as lpic_step). */
lpic_status lpic_ensemble_step(lpic_ensemble_t ensemble, cudaStream_t stream);
/* nsteps ensemble steps replayed from captured CUDA graphs (one per buffer
 * parity); `stream` must be a created stream. */
lpic_status lpic_ensemble_graph_steps(lpic_ensemble_t ensemble, int nsteps, cudaStream_t stream);
/* Synchronise; status bits of the ensemble and of every grid, cleared. */
lpic_status lpic_ensemble_check_status(lpic_ensemble_t ensemble, cudaStream_t stream, unsigned *bits);
/* Kernel launches issued by the ensemble so far. */
lpic_status lpic_ensemble_launches(lpic_ensemble_t ensemble, long long *launches);

/* Counting sort by cell tile of one FP32_FIXED particle buffer that allocates
 * nothing (the paper has no counterpart; it serves callers that cannot
 * allocate device memory: a host framework that owns all device memory
 * through its own pool, a thread whose process is capturing a CUDA graph in
 * global capture mode, or a real-time loop that cannot take the device
 * synchronisation of cudaMalloc/cudaFree).  It needs no grid: the geometry is
 * given directly.  src and dst are two distinct buffers in the FP32_FIXED
 * particle layout above (capacity entries per array, multiple of 64, 256-byte
 * aligned); count_in (device int) is the number of particles in src (a
 * value above capacity is taken as capacity, a negative one as 0);
 * count_out (device int) receives the number of particles written to dst
 * (removed particles, cell < 0, and cells at or beyond nx ny nz, are
 * dropped); tile_start (device array of
 * ntiles + 1 ints, tiles numbered x fastest) receives each tile's first index
 * in dst and, last, the total.  Order inside a tile is not specified.
 * Scratch: one fixed array in device global memory, held by every device that
 * loads the library until the process exits, sized for at most
 * LPIC_NOALLOC_MAX_TILES tiles; larger tilings return LPIC_EINVAL.  The first
 * call on a device looks up the array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * Every call uses the same array, so calls whose work overlaps on the GPU
 * (other streams, other threads) race and give wrong results; serialise them.
 * Asynchronous on `stream`. */
#define LPIC_NOALLOC_MAX_TILES 65536
lpic_status lpic_sort_tiles_static(int dim, int nx, int ny, int nz, const int tile[3],
                                   const void *src, void *dst, long long capacity,
                                   const int *count_in, int *count_out, int *tile_start,
                                   cudaStream_t stream);

/* Nonlinear Compton emission (Sec. 3.4: the nonlinear Compton module emits
 * photons from energetic electrons in strong fields; Sec. 2.1: particle
 * attributes such as chi and the optical depth tau).  FP32_FIXED path only.
 * Locally-constant-field approximation in normalised units (momenta in m c,
 * fields in m c omega / e for the unit frequency omega, time in 1/omega),
 * eps_ref = hbar omega / (m c^2):
 *   chi = eps_ref gamma sqrt((E + beta x B)^2 - (beta . E)^2),
 *   dW/dxi = alpha / (eps_ref sqrt(3) pi gamma) S(xi, chi),
 *   S = (1 - xi + 1/(1 - xi)) K_{2/3}(delta) - int_delta^inf K_{1/3},
 *   delta = 2 xi / (3 chi (1 - xi)),  W = int_0^1 dW/dxi.
 * Event Monte Carlo: each particle has an optical depth tau[id] (a caller-owned
 * device float array indexed by the particle id).  Per call tau decreases by
 * W dt with chi from the grid's fields gathered (the grid's shape order) at
 * x - (dt/2) v, the particle's position at the time of its momentum; when it
 * reaches 0 a photon with momentum xi gamma u/|u| is created at the
 * particle's stored position with its weight, the particle's momentum
 * becomes u (1 - xi gamma / |u|) and tau restarts at -ln r2.  xi solves
 * P(xi; chi) = r1 with P the normalised cumulative of S.  Random numbers:
 * Philox4x32-10 with counter (id, step, 0, 0) (r1 from word 0, r2 from word 1)
 * and key (seed low 32 bits, seed high 32 bits); r = (x + 1/2) 2^-32.
 * The rate and the spectrum come from tables built at lpic_qed_init over
 * chi in [1e-4, 1e3] (32 rows a decade, the cumulative of S on 513 nodes
 * per row); below 1e-4 the classical limit (W and xi proportional to chi),
 * above 1e3 the rate is extrapolated in log-log and the spectrum is that of
 * chi = 1e3.  Accuracy against the defining integrals: rate ~1e-4 relative,
 * xi ~2e-4 relative (FP32 table lookups). */

/* Build the tables (on the host, about a second, once per grid), and set
 * eps_ref and the seed.  Synchronises `stream`. */
lpic_status lpic_qed_init(lpic_grid_t grid, double eps_ref, uint64_t seed, cudaStream_t stream);

/* tau[id] = -ln r for id in [0, n_ids), r from counter (id, 0, 2, 0) for the
 * depths of emitting particles (photons = 0) or (id, 0, 3, 0) for the
 * pair-creation depths of photons (photons = 1). */
lpic_status lpic_qed_initial_tau(lpic_grid_t grid, float *tau, long long n_ids, int photons,
                                 cudaStream_t stream);

/* One emission pass over species `electron_species` (any massive species),
 * optionally setting each new photon's pair-creation depth
 * photon_tau[photon id] (counter (id, 0, 3, 0); photon_tau may be NULL with
 * photon_n_ids = 0; an id outside [0, photon_n_ids) sets LPIC_ST_OVERFLOW),
 * normally right after lpic_step (the grid's fields at call time are used).
 * Photons are appended to `photon_species` (a species added with m = 0 and
 * q = 0), which gets new particle ids count, count + 1, ... (count = its
 * particles at add time) in an unspecified order.  A particle id outside
 * [0, n_ids), or more photons than the photon species' capacity (an emitter
 * whose photon finds no room keeps its momentum and its spent depth, and
 * emits at a later pass), sets LPIC_ST_OVERFLOW; a gather past an absorbing edge sets LPIC_ST_OUTSIDE and
 * skips the particle.  step is the counter word (0 <= step < 2^32).
 * Asynchronous. */
lpic_status lpic_qed_compton(lpic_grid_t grid, int electron_species, int photon_species, float *tau,
                             long long n_ids, float *photon_tau, long long photon_n_ids, long long step,
                             cudaStream_t stream);

/* Nonlinear Compton emission inside the fused particle kernel (Algorithm 1
 * places the QED events between the field interpolation and the momentum
 * push).  From this call on, every push of `electron_species` (lpic_step,
 * lpic_gather_push_deposit, captured steps) runs the kernel form with
 * emission: after the gather of E and B at x^{n+1/2}, chi is formed from u^n
 * and those fields, tau[id] decreases by W dt, and on an event (counter
 * (id, step, 0, 0) as in lpic_qed_compton) a photon of momentum xi gamma
 * u^n/|u^n| leaves from x^{n+1/2} with the particle's weight, the particle
 * recoils, its depth restarts, and the Boris push, move and deposit use the
 * recoiled momentum.  Photons are appended to `photon_species` (massless,
 * with an index above electron_species, so that the same step's photon push
 * carries them to x^{n+3/2}); photon_tau as in lpic_qed_compton.  The counter
 * word is a device counter of the grid: set to first_step here (and by
 * lpic_qed_set_step), advanced by one at the end of every lpic_step, read by
 * each fused push.  Overflow and id rules as in lpic_qed_compton (a photon
 * without room leaves its emitter untouched, which is pushed without recoil).
 * photon_species = -1 turns the emission of electron_species off.  The
 * unfused stages and ensembles refuse a species with emission
 * (LPIC_EUNSUPPORTED).  Drops the grid's captured steps; synchronises the
 * device. */
lpic_status lpic_qed_fuse(lpic_grid_t grid, int electron_species, int photon_species, float *tau,
                          long long n_ids, float *photon_tau, long long photon_n_ids, long long first_step,
                          cudaStream_t stream);
/* Set the counter word of the fused emission (0 <= step < 2^32).  Asynchronous. */
lpic_status lpic_qed_set_step(lpic_grid_t grid, long long step, cudaStream_t stream);

/* Id given to the next particle that species `species_id` gains on the
 * device (emitted photons, Breit-Wheeler pairs); by default its count at add
 * time.  Ids key the optical depths and the random draws, so species that
 * share a depth array need disjoint ranges: set each species' next id past
 * every id in use.  Ids are int32: next_id plus the particles created later
 * must stay below 2^31.  Asynchronous. */
lpic_status lpic_species_set_next_id(lpic_grid_t grid, int species_id, long long next_id, cudaStream_t stream);

/* Breit-Wheeler pair creation (Sec. 3.4: pairs from energetic photons, the
 * energy split by the pair spectrum, the pair inserted into the electron and
 * positron species).  Same approximation and Monte Carlo as above, for a
 * photon of momentum k (energy k m c^2) along khat:
 *   chi_g = eps_ref k sqrt((E + khat x B)^2 - (khat . E)^2),
 *   dW/deta = alpha / (eps_ref sqrt(3) pi k) F(eta, chi_g),
 *   F = (eta/(1 - eta) + (1 - eta)/eta) K_{2/3}(z) + int_z^inf K_{1/3},
 *   z = 2 / (3 chi_g eta (1 - eta)),
 * eta the electron's share; r from counter (id, step, 1, 0) word 0; the
 * electron gets momentum eta k, the positron (1 - eta) k, both the photon's
 * stored position and weight; the photon is removed.  Photons with |k| <= 2
 * (below the pair threshold) never convert.  Tables over chi_g in
 * [1e-2, 1e3] (the rate is 0 below, where it is under 1e-110 of its scale,
 * and flushes to 0 in float below chi_g ~ 0.03); rate ~1e-4, eta ~1e-4.
 * One pass over `photon_species` with depths tau[photon id] (n_ids entries).
 * New particles get ids count, count + 1, ... of their species; a pair that
 * exceeds a capacity or whose weight exceeds a receiving species' bound
 * (max_weight at add time) is not created and sets LPIC_ST_OVERFLOW: its
 * photon stays, with its spent depth, and converts at a later pass.  The two pair species need a sort before their next
 * push (lpic_step does it).  Asynchronous. */
lpic_status lpic_qed_breit_wheeler(lpic_grid_t grid, int photon_species, int electron_species,
                                   int positron_species, float *tau, long long n_ids, long long step,
                                   cudaStream_t stream);

/* The pair tables' lookups for n (chi_g, r) pairs (device arrays): H =
 * int_0^1 F deta at chi_g (W = alpha H / (eps_ref sqrt(3) pi k)) and eta(chi_g, r).
 * Asynchronous. */
lpic_status lpic_qed_pair_eval(lpic_grid_t grid, const double *chi, const double *r, long long n, double *h,
                               double *eta, cudaStream_t stream);

/* The table lookups for n given (chi, r) pairs (device arrays): h = int_0^1 S
 * dxi at chi (W = alpha h / (eps_ref sqrt(3) pi gamma)) and xi(chi, r).
 * Asynchronous. */
lpic_status lpic_qed_eval(lpic_grid_t grid, const double *chi, const double *r, long long n, double *h,
                          double *xi, cudaStream_t stream);

/* Fault injection for tests: from this call on, the nth device allocation
 * the library makes (counted over all grids, species, ensembles and tables)
 * fails as if the device were out of memory; the call that made it unwinds
 * what it had allocated and returns LPIC_ENOMEM.  nth = 0 turns injection
 * off.  Not thread-safe; for tests only. */
lpic_status lpic_debug_fail_alloc(long long nth);

/* Message for the calling thread's last failed call ("" if none). */
const char *lpic_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* LPIC_H */
