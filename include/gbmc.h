/*
 * gbmc.h -- C ABI of the GB300 library for checkerboard Metropolis sweeps of
 * Ising-type lattices and population annealing (arXiv:1709.04394).
 *
 * Conventions (apply to every entry point):
 *  - Every call returns a gbmc_status: 0 on success, a negative code on error.
 *    No exception crosses the ABI. gbmc_last_error() returns a message for the
 *    calling host thread's last failed call.
 *  - Work is enqueued asynchronously on the context's CUDA stream unless the
 *    entry point says it synchronises. Device pointers passed in are owned by
 *    the caller and must stay valid until the enqueued work has completed.
 *  - Handles (gbmc_ctx, gbmc_lattice, gbmc_pa) are owned by the library and
 *    released with gbmc_destroy / lattice_free / pa_free.
 *  - Spin layout ("int8 layout"): int8 values +1 / -1, one byte per site,
 *    [instance][replica][site], site index row-major with x fastest:
 *    2D site = y*L + x, 3D site = (z*L + y)*L + x. Periodic boundaries.
 *  - Random numbers: Philox4x32-10 (Sec. 4, counter-based generators) with
 *    key = (seed & 0xffffffff, seed >> 32) and counter (q, t, r, c3), where
 *    c3 = purpose<<28 | colour<<27 | instance. Metropolis (purpose 0): for the
 *    k-th site of colour c in row-major order, q = k>>2 and the site uses
 *    output word k&3; t = the lattice's sweep counter; r = replica index
 *    within its instance. Random start (purpose 1): q = site>>2, word site&3,
 *    t = 0, s = +1 if the word's top bit is 0. Resampling draw k (purpose 2):
 *    q = k>>1, t = annealing step, r = 0, 64-bit value (w[2l+1]<<32)|w[2l],
 *    l = k&1. Couplings (purpose 3): bond b = 3*site + mu, q = b>>2, word b&3,
 *    t = r = 0, J = +1 if the top bit is 0. Parallel-tempering exchanges
 *    (purpose 4), multi-spin-coded sweeps (purpose 5) and Swendsen-Wang bonds
 *    and cluster coins (purposes 6 and 7) are defined at their entry points.
 *    These numbers depend only on these indices, never on how the work is
 *    spread over the GPU (Sec. 4).
 *  - Metropolis acceptance (Sec. 3.1, Eq. (8)): a site with dE <= 0 flips;
 *    otherwise it flips iff its 32-bit word u satisfies u <= T(dE), with
 *    T(dE) = ceil(exp(-beta dE) * 2^32) - 1 computed in fp64 on the host, i.e.
 *    r = u 2^-32 < exp(-beta dE). Even sub-lattice ((x+y[+z]) even) first.
 */
#ifndef GBMC_H
#define GBMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GBMC_OK = 0,
    GBMC_ERR_ARG = -1,     /* invalid argument, size or layout */
    GBMC_ERR_OOM = -2,     /* device or host allocation failed */
    GBMC_ERR_CUDA = -3,    /* a CUDA runtime call failed (message has the CUDA error) */
    GBMC_ERR_TIMEOUT = -4, /* a bounded device-side wait gave up; results are invalid */
    GBMC_ERR_STATE = -5    /* call not valid in the handle's current state */
} gbmc_status;

enum { GBMC_ISING_FM = 0, GBMC_EA_PMJ = 1 };            /* model */
enum { GBMC_INT8 = 0, GBMC_BITPACK = 1 };               /* storage layout */
enum { GBMC_START_ALL_UP = 0, GBMC_START_RANDOM = 1 };  /* initial state */

typedef struct gbmc_ctx gbmc_ctx;
typedef struct gbmc_lattice gbmc_lattice;
typedef struct gbmc_pa gbmc_pa;
typedef struct gbmc_pt gbmc_pt;

/* Library version (major*10000 + minor*100 + patch). */
int gbmc_version(void);
/* 1 for the bounds-checked build (libgbmc_check.so, compiled with GBMC_CHECK):
 * its kernels verify their array indices, replace a bad one by 0 (so the access
 * stays in bounds) and record the first failure; gbmc_sync and every other
 * call that checks the device's error flags then return GBMC_ERR_STATE with
 * "bounds check failed in <file>:<line>". 0 for the normal build, which has no
 * checks. The checked build is for testing small and uneven lattices, not for
 * timing. */
int32_t gbmc_checked_build(void);

/* Message of the calling thread's last failed call ("" if none). The pointer
 * stays valid until the thread's next gbmc call. */
const char *gbmc_last_error(void);

/* Create a context on CUDA device `device`, enqueueing on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream). The stream is borrowed. */
gbmc_status gbmc_create(gbmc_ctx **out, int device, void *cuda_stream);
gbmc_status gbmc_set_stream(gbmc_ctx *ctx, void *cuda_stream);
/* Synchronise the context's stream and report any device-side error flag
 * (GBMC_ERR_TIMEOUT) raised by a bounded wait since the last check. */
gbmc_status gbmc_sync(gbmc_ctx *ctx);
gbmc_status gbmc_destroy(gbmc_ctx *ctx);

/* Resampling path of population annealing: fused = 1 (default when the device
 * supports cooperative launches) runs the weights, ln Q / prefix sums,
 * multinomial draws and child placement of one lattice in ONE cooperative
 * launch with grid-wide barriers; fused = 0 uses one launch per phase. Both
 * give identical results. */
gbmc_status gbmc_set_resample_mode(gbmc_ctx *ctx, int32_t fused);

/* Launch form of the shared-memory sweep kernel (Sec. 3.1 checkerboard sweeps
 * of copies resident in shared memory; no counterpart in the paper, which
 * launches one thread block per tile). A work unit is one group of copies of
 * one (lattice, instance). GRID: one thread block per unit. PERSISTENT: as
 * many blocks as fit on the device at once, each claiming units from a
 * counter in the context until none is left, lattices with the largest
 * copies first. AUTO (default): persistent when the autotuned shape of the
 * lattice class says so or when several lattices share a launch, else grid.
 * Every form gives bit-identical results. Persistent launches of one context
 * share its counter, so a context's work must stay on one stream (no two of
 * its sweep launches in flight at once). 2D ferromagnets too large for one
 * thread block's shared memory (int8: L % 256 == 0; bit-packed: L % 1024 ==
 * 0) with at most (SM count / 8) copies, whose strips of rows (about
 * L x copies / SM count rows plus two halo rows each) fit in 200 KB of shared
 * memory (int8 on 152 SMs: L <= 5376 for one copy): AUTO and PERSISTENT run
 * all sweeps of a metropolis_sweeps call without E/M series as one cooperative
 * launch, each thread block keeping a strip of rows in shared memory and
 * trading its first and last rows with its neighbours through global memory
 * after every half-sweep (bounded waits; GBMC_ERR_TIMEOUT if one runs out);
 * GRID uses the per-launch kernels (halo tiles of up to 4 sweeps, resp. one
 * launch per half-sweep). Double-checkerboard sweeps with bit-sliced tiles
 * (metropolis_sweeps_dcb): PERSISTENT runs every round of a call in one
 * launch whenever all tile pairs fit on the device at once, GRID one launch
 * per coarse colour and round, AUTO the first for small k (k <= 3 with tiles
 * of 64, k <= 7 with tiles of 128), the second otherwise. Unknown mode:
 * GBMC_ERR_ARG. */
enum { GBMC_LAUNCH_AUTO = 0, GBMC_LAUNCH_GRID = 1, GBMC_LAUNCH_PERSISTENT = 2 };
gbmc_status gbmc_set_sweep_launch(gbmc_ctx *ctx, int32_t mode);
/* Kernel of the resident sweeps (checkerboard sweeps of copies held on chip,
 * Sec. 3.1). BYTES: one byte per spin in colour planes (any lattice whose copy
 * fits in a thread block's shared memory). BITS: one bit per spin, 32 sites of
 * a colour per word (the multi-spin coding of sites of Sec. 3.1 applied to the
 * copy on chip; the population stays in the int8 layout in device memory and
 * is converted on load and store), for 2D ferromagnets with L in {16, 32, 64,
 * 128, 256} and 3D lattices (ferromagnet or +-J) with L = 8 or 16; other lattices of the
 * same call take the BYTES kernel. AUTO (default): BITS for a supported lattice
 * class unless gbmc_autotune timed BYTES faster for it. The mode also picks the
 * strip-resident sweeps of large int8 2D ferromagnets (gbmc_set_sweep_launch):
 * BYTES runs them on the int8 strips; AUTO and BITS, where the bit-packed strip
 * kernel fits (L % 1024 == 0, at most SM count / 8 copies), pack the
 * configuration to one bit per spin in a library buffer (N / 8 bytes per copy,
 * kept with the lattice), run every sweep of the call there and unpack it (three
 * launches per call). All give bit-identical results (same Philox words per
 * site). Unknown kernel: GBMC_ERR_ARG. */
enum { GBMC_KERNEL_AUTO = 0, GBMC_KERNEL_BYTES = 1, GBMC_KERNEL_BITS = 2 };
gbmc_status gbmc_set_sweep_kernel(gbmc_ctx *ctx, int32_t kernel);
/* Test aid for the bounded waits: each grid barrier of the fused resampling
 * waits for `phantom_arrivals` CTAs more than the launch has, and each
 * neighbour wait of the strip-resident sweeps for that many half-sweeps more
 * (so with 1 a wait can only end by running out of its budget); waits give up
 * after `budget_cycles` SM cycles (default 2e9). A wait that runs out makes the
 * kernel return early and the next synchronising call (gbmc_sync, pa_run,
 * pa_step with statistics) return GBMC_ERR_TIMEOUT; the context stays usable.
 * Pass (0, 2000000000) to restore the defaults. */
gbmc_status gbmc_test_barrier_wait(gbmc_ctx *ctx, uint32_t phantom_arrivals, uint64_t budget_cycles);

/* Per-kernel timing with CUDA events recorded on the context stream around
 * every launch the library enqueues (off by default). gbmc_profile(ctx, 1)
 * clears the counters and starts recording; 0 stops. gbmc_profile_read
 * synchronises the stream and fills up to `capacity` entries (one per kernel
 * kind that ran), *n_out = their number. Times are device times between the
 * events bracketing the launches of that kind, in milliseconds. */
typedef struct {
    char name[32];
    uint64_t launches;  /* kernels of this kind enqueued while recording */
    double total_ms;    /* summed event-to-event device time */
} gbmc_kernel_time;
gbmc_status gbmc_profile(gbmc_ctx *ctx, int32_t enable);
gbmc_status gbmc_profile_read(gbmc_ctx *ctx, gbmc_kernel_time *out, uint32_t capacity, uint32_t *n_out);
/* Number of kernels this library has enqueued in this process so far (a
 * replayed CUDA graph of pa_run_graph counts its kernel nodes at each launch,
 * not when it is captured). */
uint64_t gbmc_kernel_launches(void);

/* ------------------------------------------------------------------------ */
/* Lattices: one or more independent copies of an L^dim periodic lattice.    */
/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t dim;            /* 2 or 3 */
    int32_t L;              /* linear size, even, 2 <= L <= 32768 (dim 2) / 1024 (dim 3) */
    int32_t model;          /* GBMC_ISING_FM (J = 1) or GBMC_EA_PMJ (bimodal +-J, Sec. 6) */
    int32_t layout;         /* GBMC_INT8, or GBMC_BITPACK (2D ferromagnet, L % 64 == 0): one bit per
                               spin, per copy two colour planes, plane c row y word w = sites
                               j = 32w..32w+31 of colour c (x = 2j + ((y+c)&1)), bit 1 where s = -1.
                               Sweeps and observables only (population annealing uses int8). */
    int32_t start;          /* GBMC_START_ALL_UP or GBMC_START_RANDOM */
    uint32_t n_instances;   /* disorder instances (independent couplings), >= 1 */
    uint32_t n_replicas;    /* replicas per instance, >= 1 */
    uint32_t instance_base; /* Philox instance id of the first instance (< 2^27) */
    uint64_t seed;          /* Philox key */
} gbmc_lattice_desc;

typedef struct {
    int64_t n_sites;        /* N = L^dim */
    int64_t n_copies;       /* n_instances * n_replicas */
    int64_t spin_bytes;     /* bytes of one configuration buffer in the lattice's layout */
    uint32_t sweep_counter; /* t of the next sweep */
    uint32_t pad;
    void *spins_dev;        /* buffer that holds the current configuration */
} gbmc_lattice_info;

/* Create a lattice and write its initial state (Sec. 3.1, step 1).
 * spins_dev: caller-owned device buffer of at least info.spin_bytes bytes
 * (int8 layout: n_instances*n_replicas*N bytes; bit-packed: N/8 bytes per
 * copy), 16-byte aligned; NULL lets the library allocate it. For GBMC_EA_PMJ
 * the couplings of every instance are drawn here from the seed (purpose 3)
 * and kept in library memory. Enqueued on the context stream. */
gbmc_status lattice_init(gbmc_ctx *ctx, const gbmc_lattice_desc *desc, void *spins_dev,
                         size_t spins_bytes, gbmc_lattice **out);
gbmc_status lattice_free(gbmc_lattice *lat);
gbmc_status lattice_info(const gbmc_lattice *lat, gbmc_lattice_info *out);
gbmc_status lattice_set_sweep_counter(gbmc_lattice *lat, uint32_t t);

/* Copy the current configuration out in the int8 layout (bytes must equal
 * n_copies*N). dst may be host (pageable or pinned) or device memory. For a
 * bit-packed lattice the copy is unpacked on the device first. Synchronises
 * the context stream when dst is host memory. */
gbmc_status lattice_copy_out(gbmc_ctx *ctx, const gbmc_lattice *lat, int8_t *dst, size_t bytes);
/* Overwrite the configuration from an int8-layout buffer (host or device);
 * values must be +1/-1 (others give undefined dynamics). */
gbmc_status lattice_copy_in(gbmc_ctx *ctx, gbmc_lattice *lat, const int8_t *src, size_t bytes);
/* Couplings of a GBMC_EA_PMJ lattice as int8 +-1, [instance][site][mu], mu = x,y,z
 * forward bonds (bytes = n_instances*N*3). */
gbmc_status lattice_couplings_out(gbmc_ctx *ctx, const gbmc_lattice *lat, int8_t *dst, size_t bytes);

/* n_sweeps checkerboard Metropolis sweeps at inverse temperature beta of every
 * copy (Sec. 3.1; Eq. (8)), sweep counters t .. t+n_sweeps-1; the lattice's
 * counter advances by n_sweeps. 0 <= beta*4*dim <= 700.
 * E_series_dev / M_series_dev: NULL, or device int32 [n_sweeps][n_copies]
 * receiving E (Eq. (7)) and M = sum_i s_i after every sweep. */
gbmc_status metropolis_sweeps(gbmc_ctx *ctx, gbmc_lattice *lat, double beta, uint32_t n_sweeps,
                              int32_t *E_series_dev, int32_t *M_series_dev);

/* Double-checkerboard sweeps with k hits per tile (Sec. 3.1, Fig. 5 right,
 * the multi-hit variant). The lattice is cut into tile x tile tiles, tile
 * (a, b) holding the sites with x / tile = a, y / tile = b and having coarse
 * colour (a + b) mod 2. A round updates every tile of coarse colour 0, then
 * every tile of coarse colour 1; a tile gets k full checkerboard sweeps (fine
 * colour 0, then 1) held on chip while every site outside it stays fixed.
 * Tiles of 64 and 128 are held one bit per spin in registers, one launch per
 * coarse colour and round; with no E/M series asked for, a cooperative-capable
 * device and every tile pair of the call resident at once, all rounds can
 * instead run in one launch, each tile kept on chip for the whole call and
 * trading only its edge rows and columns with its neighbours through bounded
 * waits (a wait that runs out raises GBMC_ERR_TIMEOUT at the next
 * synchronising call): the choice follows gbmc_set_sweep_launch (AUTO: one
 * launch for small k, where the per-launch loads dominate). GBMC_KERNEL_BYTES
 * (gbmc_set_sweep_kernel) forces the byte-plane tiles, the only ones for 32.
 * Every variant gives the same spins. The j-th sweep of round m uses sweep counter
 * t + k m + j (t = the lattice's counter on entry) for the Philox words of the
 * tile's sites, the words plain sweeps would use, and the counter advances by
 * k n_rounds; the configurations differ from plain sweeps because the order
 * of the updates does. Every update is a Metropolis step of one site, so the
 * chain keeps the Boltzmann distribution. Requirements (else GBMC_ERR_ARG):
 * 2D ferromagnet, int8 layout, tile in {32, 64, 128}, L a multiple of
 * 2 tile, k >= 1. E_series_dev / M_series_dev: NULL, or device int32
 * [n_rounds][n_copies] receiving E and M after every round. */
gbmc_status metropolis_sweeps_dcb(gbmc_ctx *ctx, gbmc_lattice *lat, double beta, uint32_t n_rounds,
                                  uint32_t k, uint32_t tile, int32_t *E_series_dev, int32_t *M_series_dev);

/* Checkerboard sweeps with multi-spin coding across replicas (Sec. 5.4: 32
 * copies coded together, their random numbers from a linear congruential
 * generator re-seeded by Philox). Replica slots 32 w .. 32 w + 31 of an
 * instance form group w; at each site of colour c with colour rank k and
 * sweep t, the Philox word of counter (k >> 2, t, w, 5 << 28 | c << 27 |
 * instance), word k & 3, seeds x -> 1664525 x + 1013904223 mod 2^32, and
 * replica 32 w + b takes the (b + 1)-th output as its uniform u in the
 * Metropolis rule u <= T(dE) (Eq. (8), as in metropolis_sweeps). The same
 * Metropolis chain as metropolis_sweeps with other random numbers. Inside the
 * kernel a site update serves 32 replicas with bitwise neighbour counting.
 * Requirements (else GBMC_ERR_ARG): 2D ferromagnet, int8 layout, L a multiple
 * of 16, 9 L^2 / 2 bytes of shared memory per 32 replicas (L <= 208). The
 * sweep counter advances by n_sweeps. */
enum { GBMC_RNG_PHILOX = 0, GBMC_RNG_MSC = 1 };
gbmc_status metropolis_sweeps_msc(gbmc_ctx *ctx, gbmc_lattice *lat, double beta, uint32_t n_sweeps);

/* Swendsen-Wang cluster updates of a ferromagnet (Sec. 3.3, its three steps),
 * every copy in place, update u using counter t = the lattice's sweep counter
 * + u (which advances by n_updates):
 *  1. forward bond b = dim i + mu (mu = axis) is active iff s_i = s_j and its
 *     Philox word (counter (b >> 2, t, replica, 6 << 28 | instance), word
 *     b & 3) is <= ceil((1 - exp(-2 beta)) 2^32) - 1 ("r < p" of the paper as
 *     an integer comparison);
 *  2. clusters = connected components of the active bonds, named by their
 *     smallest site index (a lock-free union-find on the GPU);
 *  3. the cluster named r flips iff the top bit of the Philox word of counter
 *     (r >> 2, t, replica, 7 << 28 | instance), word r & 3, is 1.
 * E_series_dev / M_series_dev: NULL or device int32 [n_updates][n_copies] (E
 * and M after each update); labels_dev: NULL or device int32 [n_copies][N],
 * the cluster name of every site in the last update. A lazily allocated
 * workspace stays with the lattice: 6 bytes per site and copy for 2D
 * L % 32 == 0 (the union-find forest and the 32 x 32 tiles' labels), 4 for 3D
 * L % 16 == 0, 5 otherwise. Requirements
 * (else GBMC_ERR_ARG): ferromagnet (dim 2 or 3), int8 layout. */
gbmc_status swendsen_wang(gbmc_ctx *ctx, gbmc_lattice *lat, double beta, uint32_t n_updates,
                          int32_t *E_series_dev, int32_t *M_series_dev, int32_t *labels_dev);

/* Energy E = -sum_<ij> J_ij s_i s_j (Eq. (7), forward bonds) and magnetisation
 * M = sum_i s_i of every copy, into device int32 arrays [n_copies]. */
gbmc_status observables(gbmc_ctx *ctx, const gbmc_lattice *lat, int32_t *E_dev, int32_t *M_dev);

/* Launch-shape autotuner for the shared-memory sweep kernel (lattices whose
 * copy fits in one CTA's shared memory). Candidate shapes -- threads per copy
 * (powers of two), copies per CTA, row-wise or flat walk over the words of a
 * colour plane -- are timed with CUDA events on a scratch copy of the first
 * (up to 32768) copies of the lattice, swept as one instance (n_sweeps sweeps
 * at beta, the lattice itself is left unchanged), then the fastest of them
 * once more as a persistent launch, and the fastest is recorded for the
 * lattice class (dim, model, L) for the rest of the process; for the classes
 * the bit-sliced kernel supports it is timed too (kernel). Untuned classes
 * use threads per copy = the power of two covering a quarter of a colour's
 * words (8..256; about four words per thread and half-sweep) in 256-thread
 * blocks. Every shape gives bit-identical results: the random words depend
 * only on (seed, sweep, replica, site). Synchronises. out->resident = 0 when
 * the lattice uses another kernel. */
typedef struct {
    int32_t resident;
    uint32_t threads_per_copy;
    uint32_t copies_per_cta;
    int32_t row_walk;
    double ms_per_sweep;      /* best time of one sweep of the timed replicas */
    uint32_t n_candidates;
    int32_t persistent;       /* 1: persistent launch (gbmc_set_sweep_launch) */
    int32_t kernel;           /* GBMC_KERNEL_BITS: the bit-sliced kernel was fastest (gbmc_set_sweep_kernel);
                                 GBMC_KERNEL_BYTES: the byte-plane shape above */
} gbmc_tuning;
gbmc_status gbmc_autotune(gbmc_ctx *ctx, const gbmc_lattice *lat, double beta, uint32_t n_sweeps,
                          gbmc_tuning *out);
/* Force (shape != NULL) or clear (NULL) the shape of a lattice class; used by
 * tests to check that every shape gives the same spins. threads_per_copy: a
 * power of two <= 256; copies_per_cta in 1..64 with product <= 256; kernel
 * GBMC_KERNEL_BITS selects the bit-sliced kernel in AUTO mode, anything else
 * the byte-plane shape. */
gbmc_status gbmc_set_tuning(int32_t dim, int32_t model, int32_t L, const gbmc_tuning *shape);

/* ------------------------------------------------------------------------ */
/* Population annealing (Sec. 5.4): every (lattice, instance) pair is one     */
/* population of n_replicas replicas annealed from beta_0 = 0.               */
/* ------------------------------------------------------------------------ */
/* Resampling laws (Sec. 5.4 step 2):
 *  MULTINOMIAL: R draws from the integer weights W_j = floor(2^s
 *    exp(-dbeta (E_j - Emin))), s = 63 - ceil(log2 R); the population stays R.
 *  NEAREST: replica j gets floor(tau_j) copies and one more with probability
 *    frac(tau_j), tau_j = R_0 W_j / sum_k W_k (s from the capacity): the weight
 *    e^{-dbeta E_j} / Q_i of the paper rescaled so that the expected population
 *    is R_0 at every step; the size R_i varies and Q_i of Eq. (13) uses
 *    R_{i-1}. The extra copy is decided exactly in integers: floor(U64_j C /
 *    2^64) < (R_0 W_j mod C), C = sum_k W_k, U64_j the resampling word of
 *    replica j. The first R_i slots of each population are live; a step that
 *    would need more slots than the capacity keeps the first `capacity`
 *    children, and the next gbmc_sync / pa_step / pa_run returns
 *    GBMC_ERR_STATE (the run is then invalid); so does a step that leaves a
 *    population empty. Fixed schedules only.
 *  POISSON: as NEAREST, but replica j gets Poisson(tau_j) copies, tau_j =
 *    double(R_0 W_j) / double(C) (correctly rounded fp64), drawn by inversion
 *    from u = the top 53 bits of U64_j: the least n with u < F(n), F summed
 *    term by term from p_0 = e^{-tau} with p_n = p_{n-1} (tau / n), stopping
 *    early once past the mode a term no longer changes F. e^{-tau} comes from
 *    a fixed sequence of correctly rounded operations (Cody-Waite reduction
 *    by ln2, Taylor series to degree 20), not from a math library, so the
 *    counts are reproducible on any IEEE machine. A mean tau_j > 500 is drawn
 *    as the sum of m = ceil(tau_j / 500) Poisson(tau_j / m) counts, piece p
 *    from the resampling word of replica j with counter field r = p. */
enum { GBMC_RESAMPLE_MULTINOMIAL = 0, GBMC_RESAMPLE_NEAREST = 1, GBMC_RESAMPLE_POISSON = 2 };

enum {
    GBMC_SCHED_LINEAR = 0,    /* beta_i = (beta_f * i) / n_steps, i = 0..n_steps */
    GBMC_SCHED_LIST = 1,      /* beta_i = betas[i], i = 0..n_steps, betas[0] = 0 */
    GBMC_SCHED_BISECTION = 2, /* per lattice: dbeta from histogram overlap bisection */
    GBMC_SCHED_MLP = 3        /* per lattice: MLP proposal, judged by the overlap */
};

typedef struct {
    uint32_t theta;          /* Metropolis sweeps per temperature step */
    uint32_t n_steps;        /* resampling steps S (LINEAR, LIST); step cap (adaptive) */
    int32_t schedule;        /* GBMC_SCHED_* */
    int32_t init;            /* 1: random start of every replica (exact at beta_0 = 0);
                                0: keep the lattices' current spins (taken as beta_0 = 0 samples) */
    double beta_f;           /* final inverse temperature */
    const double *betas;     /* host [n_steps+1] for GBMC_SCHED_LIST (copied) */
    double target_overlap;   /* adaptive schedules: histogram overlap to aim at (0.85) */
    double dbeta_max;        /* adaptive schedules: largest step */
    const float *mlp_params; /* GBMC_SCHED_MLP: host fp32 parameters, gbmc_mlp_param_count() */
    double overlap_lo;       /* GBMC_SCHED_MLP: accept a proposal if lo <= overlap <= hi */
    double overlap_hi;
    int32_t resample;        /* GBMC_RESAMPLE_MULTINOMIAL (0, constant R), _NEAREST or _POISSON */
    uint32_t initial_replicas; /* NEAREST / POISSON: R_0 (0 = n_replicas); the lattices'
                                  n_replicas is then the capacity of each population */
    int32_t sweep_rng;       /* GBMC_RNG_PHILOX (0): per-site Philox words (metropolis_sweeps);
                                GBMC_RNG_MSC: multi-spin-coded sweeps (metropolis_sweeps_msc) */
    int32_t pad;
} gbmc_pa_config;

/* Per-population record of one annealing step (after its sweeps). */
typedef struct {
    double beta;             /* beta_i */
    double dbeta;            /* beta_i - beta_{i-1} (0 at i = 0) */
    double lnQ;              /* ln Q_i, Eq. (13) */
    double lnZ;              /* N ln 2 + sum_{k<=i} ln Q_k */
    int64_t sumE, sumE2;     /* exact sums over the population of E and E^2 */
    int64_t sumAbsM, sumM2;  /* exact sums of |M| and M^2 */
    int32_t Emin, Emax;      /* population energy range */
    uint32_t step;           /* i */
    uint32_t n_replicas;     /* R_i: population size after step i (R for multinomial) */
    double overlap;          /* adaptive schedules: realised histogram overlap, else 0 */
    int32_t proposal_kind;   /* 0 fixed, 1 bisection, 2 accepted MLP proposal */
    int32_t pad;
} gbmc_pa_stats;

/* Create an annealing run over n_lattices lattices advanced together (one
 * sweep launch covers all of them). Library-owned device workspace: a second
 * configuration buffer per lattice, energies, histograms, resampling scratch,
 * and the fp64 weight tables. If cfg->init, every replica is randomised and
 * step 0 (beta_0 = 0) is recorded. Lattices must outlive the run. */
gbmc_status pa_create(gbmc_ctx *ctx, gbmc_lattice *const *lattices, uint32_t n_lattices,
                      const gbmc_pa_config *cfg, gbmc_pa **out);
gbmc_status pa_free(gbmc_pa *pa);
/* Start the run over from beta_0 = 0 without reallocating: step counter, ln Z
 * and accumulators are reset, the sweep counters return to their values at
 * pa_create, and step 0 is measured again. seed != 0 replaces every lattice's
 * Philox seed first. init != 0 draws a fresh random start from the (new)
 * seed; init == 0 keeps the current spins as the beta_0 = 0 population. */
gbmc_status pa_reset(gbmc_ctx *ctx, gbmc_pa *pa, int32_t init, uint64_t seed);
/* Number of populations (sum over lattices of n_instances); stats arrays are
 * indexed [step][population], lattices in creation order, instances within. */
gbmc_status pa_populations(const gbmc_pa *pa, uint32_t *n_populations);

/* One annealing step (Sec. 5.4 steps 2-4): resample every population to its
 * next inverse temperature, theta sweeps there, population measurements.
 * beta_next: NULL = the schedule's next value; else (adaptive schedules only)
 * host [n_lattices] explicit next betas, each above the lattice's current one.
 * out_host: NULL or host [n_populations] (rows of lattices that have already
 * reached beta_f are zero). Synchronises when out_host != NULL or the
 * schedule is adaptive. Returns GBMC_ERR_STATE once the schedule is done. */
gbmc_status pa_step(gbmc_ctx *ctx, gbmc_pa *pa, const double *beta_next, gbmc_pa_stats *out_host);

/* All remaining steps; stats_host: NULL or host [n_steps_max+1][n_populations]
 * (record of step 0 included); n_steps_done: number of steps taken by the run
 * so far. Synchronises. */
gbmc_status pa_run(gbmc_ctx *ctx, gbmc_pa *pa, gbmc_pa_stats *stats_host, uint32_t stats_capacity,
                   uint32_t *n_steps_done);

/* Adaptive schedules (GBMC_SCHED_BISECTION, GBMC_SCHED_MLP; one population per
 * lattice): every step reads the population's energy histogram h(E) and picks
 * dbeta with the overlap alpha(dbeta) = sum_E min(h/R, P1), P1 ~ h e^{-dbeta E}
 * (Sec. 5.4 cites adaptive steps without fixing them): bisection (50 halvings
 * of [0, min(dbeta_max, beta_f - beta)]) for the largest dbeta with alpha >=
 * target_overlap; or the MLP proposes dbeta and is kept if its alpha lies in
 * [overlap_lo, overlap_hi], else bisection. The chosen dbeta is read back by
 * the host, which builds the step's fp64 weight tables (libm exp) -- so these
 * schedules synchronise once per step. Each step is logged: */
typedef struct {
    double beta;            /* beta_i reached by the step */
    double dbeta;           /* beta_i - beta_{i-1} */
    double alpha;           /* overlap of the chosen step */
    double proposal;        /* MLP proposal (0 in bisection mode) */
    double alpha_proposal;  /* its overlap */
    double var;             /* variance of E of the population the step started from */
    float features[6];      /* MLP inputs: E/N mean, log(Var E/N + 1e-6), skewness, beta, log L, log R */
    int32_t kind;           /* 1 bisection, 2 accepted MLP proposal, 0 explicit beta_next */
    int32_t clamped;        /* the step hit its upper bound */
    int32_t evals;          /* overlap evaluations spent choosing it */
    int32_t pad;
} gbmc_schedule_record;
gbmc_status pa_schedule_log(const gbmc_pa *pa, uint32_t lattice, gbmc_schedule_record *out, uint32_t capacity,
                            uint32_t *n_out);
/* The inverse temperatures beta_0 .. beta_i reached so far by a lattice. */
gbmc_status pa_betas(const gbmc_pa *pa, uint32_t lattice, double *out, uint32_t capacity, uint32_t *n_out);

/* pa_run for fixed schedules (linear, list) as ONE CUDA graph: from step 0
 * (after pa_create or pa_reset) the whole run -- every resampling launch,
 * sweep launch and record of steps 1..S -- is captured once and replayed;
 * later calls replay it again while the stream, the lattices' seeds, starting
 * buffers and sweep counters and the resampling mode are unchanged (else it
 * is captured anew). The graph uses one launch per resampling phase (plain
 * kernel nodes). Same results as pa_run. Synchronises. */
gbmc_status pa_run_graph(gbmc_ctx *ctx, gbmc_pa *pa, gbmc_pa_stats *stats_host, uint32_t stats_capacity,
                         uint32_t *n_steps_done);

/* Replica each slot was copied from in the last resampling (device or host
 * dst, uint32 [n_copies] of that lattice; indices within the instance). */
gbmc_status pa_parents_out(gbmc_ctx *ctx, const gbmc_pa *pa, uint32_t lattice, uint32_t *dst,
                           size_t count);
/* Energies and magnetisations of the current population of a lattice
 * (device or host int32 [n_copies]). */
gbmc_status pa_energies_out(gbmc_ctx *ctx, const gbmc_pa *pa, uint32_t lattice, int32_t *E_dst,
                            int32_t *M_dst, size_t count);

/* Checkpoint and resume of an annealing run between steps. The random numbers
 * are a function of (seed, step, sweep, replica, site) only (Sec. 4,
 * counter-based generators), so a run continued from a saved state is
 * bit-identical to the uninterrupted run. The state holds the step index,
 * every lattice's seed, sweep counters, temperatures reached and schedule log,
 * ln Z, the energies, magnetisations, energy histogram and range of the
 * current population, the population sizes (variable-population laws) and the
 * step records; the spins are not part of it (lattice_copy_out before saving,
 * lattice_copy_in after loading).
 * pa_state_bytes: size of the state as it is now (adaptive schedules grow it
 * step by step). pa_state_save: writes it into host memory of exactly that
 * size; synchronises. pa_state_load: restores it into a run created by
 * pa_create with the same configuration on lattices of the same shapes
 * (GBMC_ERR_ARG otherwise, leaving the run unchanged); then copy the saved
 * configuration in with lattice_copy_in and continue with pa_step / pa_run.
 * Synchronises. The format is this library's own (host byte order). */
gbmc_status pa_state_bytes(const gbmc_pa *pa, size_t *bytes);
gbmc_status pa_state_save(gbmc_ctx *ctx, const gbmc_pa *pa, void *host, size_t bytes);
gbmc_status pa_state_load(gbmc_ctx *ctx, gbmc_pa *pa, const void *host, size_t bytes);

/* ------------------------------------------------------------------------ */
/* Parallel tempering (Sec. 5.1, Eq. (10)), on the same sweep kernel: each    */
/* instance's n_replicas copies are the T replicas, temperature k at          */
/* betas[k] (ascending). One step: theta sweeps of every copy at the beta of  */
/* its current temperature, then one exchange round over the pairs (k, k+1),  */
/* k = round mod 2, round mod 2 + 2, ...: accepted with probability           */
/* min(1, exp((beta_k - beta_{k+1})(E_a - E_b))) -- always if E_b >= E_a, else */
/* iff the pair's Philox word (purpose 4: q = k>>2, word k&3, t = round,      */
/* r = 0) is <= ceil(exp(-(beta_{k+1}-beta_k)(E_a-E_b)) 2^32) - 1 (host fp64). */
/* Swaps exchange temperature labels (two maps), not configurations. The     */
/* lattice (int8, shared-memory resident) belongs to the run until pt_free.  */
/* ------------------------------------------------------------------------ */
gbmc_status pt_create(gbmc_ctx *ctx, gbmc_lattice *lat, const double *betas /* host [n_replicas] */,
                      uint32_t theta, gbmc_pt **out);
gbmc_status pt_step(gbmc_ctx *ctx, gbmc_pt *pt, uint32_t n_steps);
/* rep_of: [n_instances][T] configuration at each temperature; accepted:
 * [n_instances][T-1] accepted swaps of each pair so far; E: [n_instances][T]
 * energy of each configuration after the last step. Host or device; any may
 * be NULL. Synchronises. */
gbmc_status pt_state_out(gbmc_ctx *ctx, const gbmc_pt *pt, uint32_t *rep_of, uint32_t *accepted, int32_t *E);
gbmc_status pt_free(gbmc_pt *pt);

/* ------------------------------------------------------------------------ */
/* Schedule MLP: 6 inputs -> 64 tanh -> 64 tanh -> 1, output y = log(dbeta   */
/* sigma_E). Parameters: fp32 vector [W1 (64x6 row-major), b1 (64), W2       */
/* (64x64), b2 (64), W3 (64), b3 (1)]; forward and backward use their bf16   */
/* roundings with fp32 accumulation. Trained on the GPU on (features,        */
/* bisection dbeta) pairs logged by pa_schedule_log. All device buffers.     */
/* ------------------------------------------------------------------------ */
uint32_t gbmc_mlp_param_count(void); /* 4673 */
/* Y[b] = network(X[b][0..5]) for b < B. */
gbmc_status mlp_forward(gbmc_ctx *ctx, const float *params, const float *X, uint32_t B, float *Y);
/* grad = d/dparams of (1/B) sum_b (y_b - T_b)^2 / 2 and loss[0] = that loss;
 * B <= 128 (one CTA, deterministic order). */
gbmc_status mlp_grad(gbmc_ctx *ctx, const float *params, const float *X, const float *T, uint32_t B, float *grad,
                     float *loss);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias correction at step k >= 1). */
gbmc_status mlp_adam(gbmc_ctx *ctx, float *params, const float *grad, float *m, float *v, uint32_t k, float lr);
/* epochs x ceil(n/batch) minibatches in data order (mlp_grad + mlp_adam each);
 * loss_out: NULL or device float [epochs][ceil(n/batch)] minibatch losses.
 * Uses stream-ordered scratch (cudaMallocAsync) for gradients and moments. */
gbmc_status mlp_train(gbmc_ctx *ctx, float *params, const float *X, const float *T, uint32_t n, uint32_t epochs,
                      uint32_t batch, float lr, float *loss_out);

/* ------------------------------------------------------------------------ */
/* Allocation-free resampling. The paper has no counterpart: this entry point */
/* exists for callers that must not allocate device memory -- processes      */
/* whose device memory belongs to another allocator or pool that must not be */
/* bypassed or fragmented, embedded or real-time drivers that reserve all    */
/* memory at start-up, and latency-critical code that cannot take the        */
/* implicit device-wide synchronisation of cudaMalloc / cudaFree.            */
/* ------------------------------------------------------------------------ */
/* One resampling step of population annealing for n_instances populations of
 * n_replicas replicas each, identical to the resampling inside pa_step (same
 * kernels, same Philox words, same parents and ln Q), but its scratch space
 * (histograms, integer cumulative weights, counts, weight tables, a copy of
 * the energies; about 8.1 MiB) is a fixed array compiled into the library, which every GPU that
 * loads the library holds until the process exits. It calls no cudaMalloc,
 * cudaFree or other allocating routine.
 *   cuda_stream: stream to enqueue on (NULL = legacy default stream).
 *   device: CUDA device index; made current by the call.
 *   dim, n_sites: lattice dimension (2 or 3) and N = L^dim, which fix the
 *     energy range [-dim N, dim N] and its bins of width 4.
 *   instance_base, seed, step: Philox instance id of the first population,
 *     key, and annealing step index i (draw k uses counter (k>>1, i, 0, c3)).
 *   dbeta: beta_i - beta_{i-1} >= 0.
 *   E_dev: device int32 [n_instances][n_replicas], the energies (each
 *     population's energies must differ by multiples of 4, as Metropolis
 *     dynamics keep them; values outside [-dim N, dim N] are clamped into it,
 *     so invalid input gives meaningless parents but no out-of-range access).
 *   parent_dev: device uint32 [n_instances][n_replicas] out: slot -> replica
 *     (within its instance) it copies; children contiguous, parents in order.
 *   lnQ_dev: device double [n_instances] out: per population, the log of the
 *     mean Boltzmann reweighting factor exp(-dbeta E) of its replicas.
 * Limits (GBMC_ERR_ARG beyond them): n_instances * n_replicas <= 131072,
 * n_instances <= 1024, dim*n_sites/2 + 1 <= 65537, n_instances *
 * (dim*n_sites/2 + 1) <= 524288.
 * The weight tables are computed on the host and copied from host memory on
 * every call (the host buffer is free again when the call returns). The first
 * call on a device (and the first after its context was reset) looks up the
 * array's device address with that device current; make that first call
 * before any stream capture. Every call
 * shares the one array and it keeps the last call's contents (each call
 * clears what must start at zero), so calls whose work overlaps on the GPU
 * -- on different streams, or from different host threads -- race and give
 * wrong results: serialise them. Asynchronous: results are ready when the
 * stream reaches them. */
gbmc_status pa_resample_static(void *cuda_stream, int32_t device, int32_t dim, int64_t n_sites,
                               uint32_t n_instances, uint32_t n_replicas, uint32_t instance_base,
                               uint64_t seed, uint32_t step, double dbeta, const int32_t *E_dev,
                               uint32_t *parent_dev, double *lnQ_dev);

#ifdef __cplusplus
}
#endif
#endif /* GBMC_H */
