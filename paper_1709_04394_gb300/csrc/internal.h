// internal.h -- host/device shared structures of the library and the host-side
// launchers of its kernels (not part of the public ABI).
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

namespace gbmc {

// Kernels enqueued by this library in this process (every <<<>>> adds one).
void count_launch();
// Message returned by gbmc_last_error() on the calling thread.
void set_last_error(const char* msg);

constexpr int kMaxJobs = 8;

// One lattice's share of a sweep launch (Sec. 3.1 checkerboard sweeps of all
// copies of one lattice; with PA, the resampling gather of Sec. 5.4 on load).
struct SweepJob {
    const int8_t* src;        // configuration read: copy c from src + parent(c)*N (or c*N)
    int8_t* dst;              // configuration written: copy c to dst + c*N (may be src if no parent)
    const uint32_t* parent;   // [n_inst*R] source replica (within its instance) of each slot, or null
    const uint8_t* jbits;     // +-J bonds: [n_inst][3][N], byte 1 where J = -1; null for J = 1
    const uint8_t* jsplit;    // +-J bonds per colour plane: [n_inst][2][6][N/2], byte 4 where J = -1
    int32_t* E;               // [n_inst*R] energy after the last sweep, or null
    int32_t* M;               // [n_inst*R] magnetisation after the last sweep, or null
    int32_t* Eser;            // [nsweeps][n_inst*R] per-sweep energy, or null
    int32_t* Mser;            // [nsweeps][n_inst*R] per-sweep magnetisation, or null
    uint32_t* hist;           // [n_inst][nbins] energy histogram accumulated, or null (PA)
    int32_t* emin;            // [n_inst] atomic min of E (PA), or null
    int32_t* emax;            // [n_inst] atomic max of E (PA), or null
    unsigned long long* sums; // [n_inst][4] sum E, E^2, |M|, M^2 (two's complement), or null
    uint64_t seed;
    uint32_t thr[3];          // thresholds T(4), T(8), T(12)
    uint32_t L, N, R, n_inst, inst_base;
    uint32_t t0, nsweeps;
    int32_t e_lo;             // histogram bin b = (E - e_lo) >> 2
    uint32_t nbins;
    uint32_t rpc;             // replicas per CTA (CTAs never straddle instances)
    uint32_t ctas_per_inst;
    const uint32_t* thr_temp; // parallel tempering: [T][3] thresholds per temperature, or null
    const uint32_t* temp_of;  // parallel tempering: [n_inst*R] temperature of each copy, or null
    const uint32_t* nlive;    // variable populations: [n_inst] live copies (the first ones); null: R
    const uint32_t* jb3;      // +-J bonds of the bit-sliced 3D L = 8 sweep: [n_inst][2][6][8] words, bit 1
                              // where J = -1; null for J = 1
};

struct SweepLaunch {
    SweepJob jobs[kMaxJobs];
    uint32_t cta_begin[kMaxJobs + 1];  // job j owns CTAs [cta_begin[j], cta_begin[j+1])
    int32_t njobs;
    int32_t dim;
    int32_t ea;
    int32_t swar;                      // 1: every job has L % 8 == 0 (split colour planes)
    int32_t rowwise;                   // 1: every job's threads per copy are a multiple of L/8
    uint32_t total;                    // work units (= cta_begin[njobs])
    unsigned int* work;                // persistent launch: [claim counter, finished CTAs], both 0
                                       // at launch; null: one CTA per unit
};

// ---- launchers (return cudaError_t of the launch) ----
cudaError_t launch_init_spins(int8_t* spins, int dim, uint32_t L, uint32_t n_inst, uint32_t R,
                              uint32_t inst_base, uint64_t seed, int random_start, cudaStream_t s);
cudaError_t launch_couplings(uint8_t* jbits, uint32_t L, uint32_t n_inst, uint32_t inst_base,
                             uint64_t seed, cudaStream_t s);
// Bond planes of the split layout (L % 8 == 0): for colour c and each site of
// that colour, the bonds to its 6 neighbours in the order used by the sweep.
cudaError_t launch_split_bonds(const uint8_t* jbits, uint8_t* jsplit, uint32_t L, uint32_t n_inst,
                               cudaStream_t s);
cudaError_t launch_jbits_to_int8(const uint8_t* jbits, int8_t* out, uint32_t N, uint32_t n_inst,
                                 cudaStream_t s);
cudaError_t launch_observables(const int8_t* spins, const uint8_t* jbits, int dim, uint32_t L,
                               uint32_t n_inst, uint32_t R, int32_t* E, int32_t* M, cudaStream_t s);

// Bit-packed 2D ferromagnet layout (one bit per spin, per-colour planes).
cudaError_t launch_bp_init(uint32_t* P, uint32_t L, uint64_t copies, uint32_t R, uint32_t inst_base, uint64_t seed,
                           int random_start, cudaStream_t s);
cudaError_t launch_bp_pack(const int8_t* src, uint32_t* P, uint32_t L, uint64_t copies, cudaStream_t s);
cudaError_t launch_bp_unpack(const uint32_t* P, int8_t* dst, uint32_t L, uint64_t copies, cudaStream_t s);
cudaError_t launch_bp_halfsweep(uint32_t* P, uint32_t L, uint64_t copies, uint32_t R, uint32_t inst_base,
                                uint64_t seed, uint32_t colour, uint32_t t, uint32_t T4, uint32_t T8, cudaStream_t s);
// All half-sweeps of a call in one cooperative launch, strips of rows resident
// in shared memory (bitpack.cu). progress: copies * Gc counters, zeroed by the
// launch; a wait that outlasts `budget` cycles raises *err and the kernel
// returns. phantom: extra half-sweeps a wait asks for (0 in production; tests
// set 1 to make a wait run out).
struct BpStrips {
    uint32_t* P;
    unsigned int* progress;
    unsigned int* err;
    long long budget;
    uint64_t seed;
    uint32_t L, Gc, rmax, R, inst_base, t0, n_half, T4, T8, phantom;
};
bool bp_strips_shape(uint32_t L, uint64_t copies, int sm_count, uint32_t& Gc, uint32_t& rmax, uint32_t& threads,
                     size_t& smem);
cudaError_t launch_bp_strips(const BpStrips& S, uint64_t copies, uint32_t threads, size_t smem, int sm_count,
                             cudaStream_t s);
cudaError_t launch_bp_observables(const uint32_t* P, uint32_t L, uint64_t copies, int32_t* E, int32_t* M,
                                  cudaStream_t s);

// Resident sweep: every copy fits in one CTA's shared memory.
size_t resident_smem_bytes(const SweepLaunch& P);
cudaError_t launch_sweep_resident(const SweepLaunch& P, uint32_t n_ctas, uint32_t threads,
                                  size_t smem, cudaStream_t s);
// Tiled sweeps of large 2D ferromagnets (T | L, T % 8 == 0): up to 4 exact
// sweeps per launch from src into dst (different buffers).
struct TileLaunch {
    const int8_t* src;
    int8_t* dst;
    uint64_t seed;
    uint32_t L, T, R, inst_base, copy0;
    uint32_t t0, nsweeps;     // nsweeps <= 4 (halo tiles); k hits per tile (double checkerboard)
    uint32_t thr[2];          // T(4), T(8)
    uint32_t coarse;          // double checkerboard: coarse colour of the tiles of this launch
};
size_t tile_smem_bytes(uint32_t T);
cudaError_t launch_sweep_tiles(const TileLaunch& P, uint64_t copies, cudaStream_t s);
// Strip-resident sweeps of large 2D ferromagnets, int8 layout (tiles.cu): all
// half-sweeps of a call in one cooperative launch, the same protocol and
// fields as BpStrips (thr = T(4), T(8)).
struct StripLaunch {
    int8_t* spins;
    unsigned int* progress;
    unsigned int* err;
    long long budget;
    uint64_t seed;
    uint32_t L, Gc, rmax, R, inst_base, t0, n_half, phantom;
    uint32_t thr[2];
};
bool strips_shape(uint32_t L, uint64_t copies, int sm_count, uint32_t& Gc, uint32_t& rmax, uint32_t& threads,
                  size_t& smem);
cudaError_t launch_sweep_strips(const StripLaunch& S, uint64_t copies, uint32_t threads, size_t smem, int sm_count,
                                cudaStream_t s);
// Double checkerboard (Fig. 5 right): the tiles of coarse colour P.coarse, each
// swept P.nsweeps times in place (src == dst); T in {32, 64, 128}, L % 2T == 0.
cudaError_t launch_sweep_dcb(const TileLaunch& P, uint64_t copies, cudaStream_t s);
// The same double checkerboard with each tile bit-sliced in registers
// (dcb_bits.cu): T in {64, 128}, the same spins.
bool dcb_bits_supported(uint32_t T);
cudaError_t launch_dcb_bits(const TileLaunch& P, uint64_t copies, cudaStream_t s);
// Every round of a call in one cooperative launch, tiles resident in
// registers, tile edges traded through `edges` and announced by `progress`
// (one counter per tile; both in one buffer of dcb_resident_bytes, progress
// after the edges). Waits give up after `budget` cycles or when *err is
// raised, raising *err; phantom: extra rounds a wait asks for (0 in
// production; tests set 1 to make a wait run out).
struct DcbResident {
    int8_t* spins;
    uint32_t* edges;
    unsigned int* progress;
    unsigned int* err;
    long long budget;
    uint64_t seed;
    uint32_t L, T, R, inst_base, t0, k, n_rounds, phantom;
    uint32_t thr[2];  // T(4), T(8)
};
size_t dcb_resident_bytes(uint32_t L, uint32_t T, uint64_t copies);
bool dcb_resident_fits(uint32_t L, uint32_t T, uint64_t copies, int sm_count);
cudaError_t launch_dcb_resident(const DcbResident& D, uint64_t copies, cudaStream_t s);
// Global-memory half-sweep over one job (large lattices); colour 0 or 1.
cudaError_t launch_halfsweep_global(const SweepJob& J, int dim, int colour, uint32_t t,
                                    cudaStream_t s);

// Bit-sliced resident sweeps (bitsweep.cu): every copy converted to one bit
// per spin on chip, same results as launch_sweep_resident. Supported lattices:
// 2D ferromagnets with L in {16, 32, 64, 128, 256}, 3D lattices with L = 8 or 16 (all
// jobs of a launch of one dimension and model; 2D lattices with L <= 32 and L >= 64,
// and 3D lattices with L = 8 and L = 16, go to separate launches). Uses its own
// block layout (P.cta_begin and P.total are recomputed).
bool bits_supported(int dim, int L);
cudaError_t launch_sweep_bits(const SweepLaunch& P, cudaStream_t s);
// +-J bonds of 3D lattices (L = 8 or 16) as the bit-sliced sweeps' bond words:
// bits3_bond_words(L) words per instance.
size_t bits3_bond_words(uint32_t L);
cudaError_t launch_bits3_bonds(const uint8_t* jbits, uint32_t* jb3, uint32_t L, uint32_t n_inst, cudaStream_t s);

// Multi-spin-coded sweeps (2D ferromagnet, L % 16 == 0): jobs with rpc = 32 G
// replicas per CTA; G in 1..4 groups of 32.
size_t msc_smem_bytes(uint32_t N, uint32_t G);
uint32_t msc_pick_groups(uint32_t N, uint64_t groups, int sms);
cudaError_t launch_sweep_msc(const SweepLaunch& P, uint32_t n_ctas, uint32_t G, cudaStream_t s);

// Swendsen-Wang update (Sec. 3.3) of `copies` copies of a ferromagnet, in place.
// (instance, replica) of copy index `copy` with R replicas per instance; a
// 32-bit division whenever the index fits in 32 bits (a 64-bit one is a long
// software routine).
__device__ __forceinline__ void split_copy(uint64_t copy, uint32_t R, uint32_t& inst, uint32_t& r) {
    if (copy < 0x100000000ull) {
        const uint32_t c = (uint32_t)copy;
        inst = c / R;
        r = c - inst * R;
    } else {
        inst = (uint32_t)(copy / R);
        r = (uint32_t)(copy - (uint64_t)inst * R);
    }
}

struct SwLaunch {
    int8_t* spins;            // [copies][N]
    uint8_t* bonds;           // [copies][N] bit mu: forward bond along mu active
    uint32_t* parent;         // [copies][N] union-find forest
    int32_t* labels;          // [copies][N] cluster name (smallest site) of every site, or null
    uint16_t* lab;            // [copies][N] 2D tiles: tile-local index of each site's tile root
    unsigned int* err;        // raised if a hook loop ran out of its cap
    uint64_t seed;
    uint64_t copy0;
    long long T_bond;         // active iff parallel and u <= T_bond (-1: never)
    uint32_t L, N, dim, R, inst_base, t;
    uint32_t lshift;          // log2 L when L is a power of two, else 0
};
cudaError_t launch_sw_update(const SwLaunch& P, uint64_t copies, cudaStream_t s);
// Lattices labelled tile by tile (2D: 32 x 32 tiles, 3D: 16 x 8 x 8) need no
// bond-flag array; the others use the global union-find over stored flags.
inline bool sw_tiled(uint32_t dim, uint32_t L) { return (dim == 2 && L % 32 == 0) || (dim == 3 && L % 16 == 0); }

// ---- population annealing resampling (Sec. 5.4, Eq. (13)) ----
struct PaLattice {
    const int32_t* E;         // [n_inst*R] current energies
    uint32_t* hist;           // [n_inst][nbins]
    int32_t* emin;            // [n_inst]
    int32_t* emax;            // [n_inst]
    unsigned long long* sums; // [n_inst][4]
    const double* wexp;       // [nbins] exp(-dbeta*4k) of this step
    const unsigned long long* wint;  // [nbins] floor(2^s exp(-dbeta*4k))
    unsigned long long* cloc; // [n_inst*R] inclusive weight sums within each chunk
    unsigned long long* ctot; // [n_inst][nchunks] chunk totals
    unsigned long long* cpre; // [n_inst][nchunks+1] exclusive chunk prefix (last = total)
    uint32_t* counts;         // [n_inst*R] copies of each replica
    uint32_t* sloc;           // [n_inst*R] exclusive count prefix within the chunk
    uint32_t* ntot;           // [n_inst][nchunks] chunk count totals
    uint32_t* parent;         // [n_inst*R] out: source replica of each slot
    void* stats;              // gbmc_pa_stats [n_inst] record of this step (device)
    double dbeta, beta, log_R, lnZ0;
    double overlap;           // realised overlap of an adaptive step (recorded)
    uint64_t seed;
    uint32_t R, n_inst, inst_base, nbins, nchunks, step;
    int32_t e_lo;
    int32_t kind;             // how the step was chosen (recorded)
    // nearest-integer resampling with variable populations (R = capacity):
    const uint32_t* nprev;    // [n_inst] R_{i-1} (read), or null (multinomial, constant R)
    uint32_t* nnext;          // [n_inst] R_i (written by the placement), or null
    unsigned int* overflow;   // raised when children exceed the capacity
    uint32_t R0;              // target population
    int32_t nearest;          // 1: nearest-integer law, 2: Poisson law (instead of multinomial draws)
};

constexpr uint32_t kScanChunk = 2048;  // replicas per resampling chunk (512 threads x 4)

// Grid-wide barrier of a cooperative launch. counter: zeroed before each
// launch; err: raised when a wait exceeds `budget` cycles (the kernel then
// returns early and the host reports GBMC_ERR_TIMEOUT). phantom: extra arrivals
// a barrier waits for (0 in production; tests set 1 to make a wait run out).
struct GridBarrier {
    unsigned int* counter;
    unsigned int* err;
    long long budget;
    uint32_t phantom;
};

cudaError_t launch_pa_resample_fused(const PaLattice& P, double* lnZ, const GridBarrier& B, int n_sms,
                                     cudaStream_t s);
cudaError_t launch_pa_weights(const PaLattice& P, cudaStream_t s);
cudaError_t launch_pa_reduce(const PaLattice& P, double* lnZ, int first_step, cudaStream_t s);
cudaError_t launch_pa_draws(const PaLattice& P, cudaStream_t s);
cudaError_t launch_pa_nearest(const PaLattice& P, cudaStream_t s);
cudaError_t launch_pa_place(const PaLattice& P, cudaStream_t s);
cudaError_t launch_pa_record(const PaLattice& P, const double* lnZ, double lnQ_unused, cudaStream_t s);
cudaError_t launch_pa_reset(const PaLattice& P, cudaStream_t s);

// ---- parallel tempering exchanges (Sec. 5.1, Eq. (10)) ----
struct PtExchange {
    const int32_t* E;          // [n_inst*T] energy of each configuration
    uint32_t* rep_of;          // [n_inst*T] configuration at each temperature
    uint32_t* temp_of;         // [n_inst*T] temperature of each configuration
    uint32_t* accepted;        // [n_inst*(T-1)] accepted swaps per pair
    const long long* tab;      // [T-1][M+1] threshold of pair k at energy gap 4m (-1: never)
    uint64_t seed;
    uint32_t T, M, n_inst, inst_base, round;
};
cudaError_t launch_pt_exchange(const PtExchange& X, cudaStream_t s);

// ---- schedule MLP (6 -> 64 -> 64 -> 1) ----
constexpr int kMlpIn = 6;
constexpr int kMlpHidden = 64;
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kMlpHidden * kMlpIn;
constexpr int kOffW2 = kOffB1 + kMlpHidden;
constexpr int kOffB2 = kOffW2 + kMlpHidden * kMlpHidden;
constexpr int kOffW3 = kOffB2 + kMlpHidden;
constexpr int kOffB3 = kOffW3 + kMlpHidden;
constexpr int kMlpParams = kOffB3 + 1;  // 4673
constexpr uint32_t kMlpMaxBatch = 128;

cudaError_t launch_mlp_forward(const float* p, const float* X, uint32_t B, float* Y, cudaStream_t s);
cudaError_t launch_mlp_grad(const float* p, const float* X, const float* T, uint32_t B, float* g, float* loss,
                            cudaStream_t s);
cudaError_t launch_mlp_adam(float* p, const float* g, float* m, float* v, uint32_t k, float lr, cudaStream_t s);

// ---- adaptive annealing steps: overlap bisection and MLP proposals ----
// One population per lattice (n_instances == 1).
struct SchedJob {
    const uint32_t* hist;     // [nbins] energy histogram of the current population
    const int32_t* emin;
    const int32_t* emax;
    int32_t e_lo;
    uint32_t nbins, R, N, L;
    double beta, dmax;        // current beta; largest allowed step (<= beta_f - beta)
};

struct SchedOut {             // result per lattice (device, copied to the host)
    double dbeta;             // chosen step
    double alpha;             // realised overlap of the chosen step
    double proposal;          // MLP proposal (0 in bisection mode)
    double alpha_proposal;    // overlap of the proposal
    double var;               // population variance of E
    float feat[6];            // MLP inputs
    int32_t kind;             // 1 bisection, 2 accepted MLP proposal
    int32_t clamped;          // 1: the step hit dmax
    int32_t evals;            // overlap evaluations spent
    int32_t emin, emax;
    int32_t pad;
};

struct SchedLaunch {
    SchedJob jobs[kMaxJobs];
    SchedOut* out;            // [njobs]
    const float* mlp;         // fp32 master parameters, or null (bisection only)
    double target, lo, hi;    // bisection target; MLP acceptance band
    int32_t njobs;
    int32_t mode;             // 1 bisection, 2 MLP with bisection fallback
};

cudaError_t launch_schedule(const SchedLaunch& S, cudaStream_t s);

}  // namespace gbmc
