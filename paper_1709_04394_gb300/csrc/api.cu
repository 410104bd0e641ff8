// api.cu -- the C ABI declared in include/gbmc.h: contexts, lattices, sweeps,
// observables and population annealing runs. Host code here only validates,
// sizes launches, computes the per-beta tables (thresholds of Eq. (8), fp64
// resampling weights of Eq. (13)) and enqueues the kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <map>
#include <mutex>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/gbmc.h"
#include "check.cuh"
#include "internal.h"

using namespace gbmc;

namespace {

thread_local std::string g_err;

gbmc_status fail(gbmc_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

#define CUDA_TRY(call)                                                                         \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return fail(e_ == cudaErrorMemoryAllocation ? GBMC_ERR_OOM : GBMC_ERR_CUDA,       \
                        "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

constexpr size_t kSmemLimit = 227 * 1024;

std::atomic<uint64_t> g_launches{0};

enum ProfKind {
    PK_INIT, PK_COUPLINGS, PK_SWEEP_RES, PK_HALFSWEEP, PK_OBS, PK_PA_WEIGHTS, PK_PA_REDUCE,
    PK_PA_DRAWS, PK_PA_PLACE, PK_PA_RECORD, PK_PA_RESET, PK_SWEEP_TILES, PK_SCHEDULE, PK_PA_FUSED,
    PK_BP_HALFSWEEP, PK_SWEEP_DCB, PK_SWEEP_MSC, PK_SW, PK_BP_STRIPS, PK_SWEEP_STRIPS, PK_PT_EXCHANGE, PK_SWEEP_BITS,
    PK_BP_PACK, PK_SWEEP_DCB_BITS, PK_SWEEP_DCB_RES, PK_COUNT
};
const char* const kProfNames[PK_COUNT] = {"init_spins", "couplings", "sweep_resident", "halfsweep_global",
                                          "observables", "pa_weights", "pa_reduce", "pa_draws", "pa_place",
                                          "pa_record", "pa_reset", "sweep_tiles", "schedule", "pa_resample",
                                          "bitpack_halfsweep", "sweep_dcb", "sweep_msc", "swendsen_wang",
                                          "bitpack_strips", "sweep_strips", "pt_exchange", "sweep_bits",
                                          "bitpack_convert", "sweep_dcb_bits",
                                          "sweep_dcb_resident"};

// Device words of a context: 8 flags and counters, then the progress
// counters of strip-resident sweeps (one per CTA, one CTA per SM).
constexpr size_t kCtxWords = 8 + 1024;

// Interior size of the tiles of large 2D lattices (window = kTile + 16).
constexpr uint32_t kTile = 128;

}  // namespace

namespace gbmc {
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void set_last_error(const char* msg) { g_err = msg; }
#ifdef GBMC_CHECK
namespace {
struct CheckEntry {
    CheckReader read;
    const char* file;
};
std::vector<CheckEntry>& check_entries() {
    static std::vector<CheckEntry> v;
    return v;
}
}  // namespace
void check_register(CheckReader reader, const char* file) { check_entries().push_back({reader, file}); }
#endif
}  // namespace gbmc

struct gbmc_ctx {
    int device;
    cudaStream_t stream;
    int sm_count;
    unsigned int* words = nullptr;  // device [barrier counter, error flag, unit claims, finished CTAs,
                                    //         population overflow flag, 3 spare, strip progress[1024]]
    bool fused = true;              // one cooperative resampling launch per lattice and step
    bool coop = false;              // the device supports cooperative launches
    int32_t launch_mode = GBMC_LAUNCH_AUTO;  // grid or persistent resident sweeps
    int32_t sweep_kernel = GBMC_KERNEL_AUTO; // bit-sliced or byte-plane resident sweeps
    uint32_t phantom = 0;           // test hook: extra barrier arrivals to wait for
    long long budget = 2000000000;  // cycles a barrier wait may last (about 1 s)
    bool prof = false;
    struct Pending {
        int kind;
        uint64_t launches;
        cudaEvent_t a, b;
    };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> pool;
    double ms[PK_COUNT] = {};
    uint64_t launches[PK_COUNT] = {};

    cudaEvent_t event() {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
};

namespace {
// Brackets one launcher call with an NVTX range named after its kernel kind
// (free unless a profiler is attached) and, when profiling is on, with CUDA
// events.
struct ProfScope {
    gbmc_ctx* c;
    int kind;
    uint64_t n0;
    cudaEvent_t a = nullptr;
    ProfScope(gbmc_ctx* ctx, int k) : c(ctx), kind(k), n0(g_launches.load()) {
        nvtxRangePushA(kProfNames[k]);
        if (c->prof) {
            a = c->event();
            cudaEventRecord(a, c->stream);
        }
    }
    ~ProfScope() {
        nvtxRangePop();
        const uint64_t n = g_launches.load() - n0;
        if (c->prof) {
            cudaEvent_t b = c->event();
            cudaEventRecord(b, c->stream);
            c->pending.push_back({kind, n, a, b});
        }
    }
};
}  // namespace

struct gbmc_lattice {
    gbmc_ctx* ctx;
    gbmc_lattice_desc d;
    uint64_t N;
    uint64_t ncopies;
    int8_t* spins;     // caller's (or library-allocated) buffer
    bool owns_spins;
    int8_t* cur;       // buffer holding the current configuration
    uint8_t* jbits;    // +-J bond planes [inst][3][N]
    uint8_t* jsplit;   // the same bonds per colour plane [inst][2][6][N/2] (L % 8 == 0)
    uint32_t* jb3;     // the same bonds as bit words of the bit-sliced 3D sweeps [inst][2][6][L^3 / 64]
    uint32_t* packed;  // bit-packed copy of the configuration for the strip-resident bit sweeps (int8 layout)
    int8_t* alt;       // second configuration buffer of the tiled large-lattice sweeps
    uint32_t* dcb_scratch;    // tile edges and progress counters of the resident double checkerboard
    size_t dcb_scratch_bytes;
    uint8_t* sw_bonds; // Swendsen-Wang workspace: bond flags, union-find forest, 2D tile labels
    uint32_t* sw_parent;
    uint16_t* sw_lab;
    uint32_t t;        // sweep counter
    gbmc_pa* run;      // annealing run using this lattice
};

namespace {

struct PaLat {
    gbmc_lattice* lat = nullptr;
    int8_t* alt = nullptr;
    int32_t *E = nullptr, *M = nullptr;
    uint32_t* hist = nullptr;
    int32_t *emin = nullptr, *emax = nullptr;
    unsigned long long* sums = nullptr;
    double* lnZ = nullptr;  // [2*n_inst]: lnZ, then lnQ of the last step
    unsigned long long *cloc = nullptr, *ctot = nullptr, *cpre = nullptr;
    uint32_t *counts = nullptr, *sloc = nullptr, *ntot = nullptr, *parent = nullptr;
    double* wexp = nullptr;                // [n_tables][nbins]
    unsigned long long* wint = nullptr;    // [n_tables][nbins]
    std::vector<double> betas;             // beta_0 .. beta_S
    std::vector<uint32_t> thr;             // [S+1][3]
    uint32_t nbins = 0, nchunks = 0;
    int32_t e_lo = 0;
    int s_bits = 0;
    uint32_t pop0 = 0;                     // first population index
    uint32_t t_start = 0;
    // adaptive schedules: weight tables of the current step in a 2-slot ring
    bool ring = false;
    double* hexp = nullptr;                // pinned host staging [2][nbins]
    unsigned long long* hint = nullptr;
    uint32_t steps = 0;                    // steps taken by this lattice
    bool done = false;                     // reached beta_f
    bool stepping = false;                 // takes part in the step being enqueued
    double overlap = 0.0;                  // realised overlap of the last step
    int32_t kind = 0;                      // how the last step was chosen
    std::vector<gbmc_schedule_record> log;
    uint32_t* nrep = nullptr;              // nearest-integer law: [2][n_inst] R_i by step parity
};

}  // namespace

struct gbmc_pa {
    gbmc_ctx* ctx;
    gbmc_pa_config cfg;
    std::vector<PaLat> lats;
    uint32_t P = 0;
    uint32_t S = 0;        // steps of a fixed schedule; step cap of an adaptive one
    uint32_t step = 0;     // steps enqueued
    bool adaptive = false;
    bool nearest = false;  // nearest-integer or Poisson resampling, variable populations
    bool poisson = false;  // Poisson counts
    bool msc = false;      // multi-spin-coded sweeps
    uint32_t R0 = 0;       // its initial (and expected) population
    gbmc_pa_stats* stats = nullptr;  // device [S+1][P]
    SchedOut* sched_dev = nullptr;   // [kMaxJobs]
    SchedOut* sched_host = nullptr;  // pinned copy
    float* mlp_dev = nullptr;        // MLP parameters (GBMC_SCHED_MLP)
    std::vector<void*> allocs;
    std::vector<void*> host_allocs;
    // CUDA graph of a whole fixed-schedule run (pa_run_graph) and the state it
    // starts from / leaves behind
    cudaGraphExec_t graph = nullptr;
    cudaStream_t capture_stream = nullptr;  // capture cannot use the legacy default stream
    std::vector<uint64_t> graph_key;
    uint64_t graph_kernels = 0;             // kernel nodes of the captured run
    std::vector<int8_t*> graph_end_cur;
    std::vector<uint32_t> graph_end_t;
};

namespace {

bool is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// T(dE) = ceil(exp(-beta dE) 2^32) - 1 (Eq. (8) as an integer comparison).
void thresholds(double beta, uint32_t out[3]) {
    for (int m = 0; m < 3; ++m) {
        const double dE = 4.0 * (double)(m + 1);
        const double p = std::exp(-(beta * dE));
        const double scaled = std::ldexp(p, 32);
        const int64_t t = (int64_t)std::ceil(scaled) - 1;
        out[m] = (uint32_t)(t < 0 ? 0 : (t > 0xFFFFFFFFll ? 0xFFFFFFFFll : t));
    }
}

bool beta_ok(double beta, int dim) { return std::isfinite(beta) && beta >= 0.0 && beta * 4.0 * dim <= 700.0; }

struct Tuning {
    bool resident;
    uint32_t tpr, rpc, threads;
    size_t smem;
    bool rowwise;     // allow the division-free row walk (needs tpr % (L/8) == 0)
    bool persistent;  // resident CTAs claim work units instead of one CTA per unit
    bool bits;        // the bit-sliced kernel (where it supports the lattice)
};

// Launch shapes chosen by gbmc_autotune (or set with gbmc_set_tuning), per
// lattice class (dim, model, L); every shape gives bit-identical results
// because the random numbers depend only on (seed, sweep, replica, site).
struct ShapeKey {
    int dim, model, L;
    bool operator<(const ShapeKey& o) const {
        return dim != o.dim ? dim < o.dim : (model != o.model ? model < o.model : L < o.L);
    }
};
struct Shape {
    uint32_t tpr, copies_per_cta;
    bool rowwise;
    bool persistent;
    bool bits;
};
std::mutex g_shape_mu;
std::map<ShapeKey, Shape> g_shapes;

size_t bond_bytes(const gbmc_lattice* l) {
    if (l->d.model != GBMC_EA_PMJ) return 0;
    return (l->d.L % 8 == 0 ? 6 : 3) * l->N;
}

uint64_t units_per_copy(const gbmc_lattice* l) {
    return (l->d.L % 8 == 0) ? l->N / 8 : ((l->N / 2) + 3) / 4;
}

// Shape for (tpr, copies per CTA): clamp to the replica count and shared memory.
Tuning make_tuning(const gbmc_lattice* l, uint32_t tpr, uint32_t rpc, bool rowwise, bool persistent = false) {
    Tuning t{};
    const uint64_t stride = (l->N + 15) & ~15ull;
    const size_t bonds = bond_bytes(l);
    if (stride + bonds > kSmemLimit || l->N > (1ull << 31)) {
        t.resident = false;
        return t;
    }
    if (rpc > l->d.n_replicas) rpc = l->d.n_replicas;
    if (rpc < 1) rpc = 1;
    while (rpc > 1 && rpc * stride + bonds > kSmemLimit) --rpc;
    t.resident = true;
    t.tpr = tpr;
    t.rpc = rpc;
    t.threads = tpr * rpc;
    if (t.threads < 32) t.threads = 32, t.tpr = 32 / rpc;
    t.smem = rpc * stride + bonds;
    t.rowwise = rowwise;
    t.persistent = persistent;
    return t;
}

// Default shape: threads per copy = the power of two covering a quarter of
// the copy's units (8..256: about four units per thread and half-sweep, the
// range the autotuner picks from), copies per CTA filling 256 threads; or the
// tuned one.
Tuning tune(const gbmc_lattice* l, bool use_table = true) {
    if (use_table) {
        std::lock_guard<std::mutex> g(g_shape_mu);
        auto it = g_shapes.find(ShapeKey{l->d.dim, l->d.model, l->d.L});
        if (it != g_shapes.end()) {
            Tuning t = make_tuning(l, it->second.tpr, it->second.copies_per_cta, it->second.rowwise,
                                   it->second.persistent);
            t.bits = it->second.bits;
            return t;
        }
    }
    const uint64_t units = units_per_copy(l);
    uint32_t tpr = 8;
    while (4 * tpr < units && tpr < 256) tpr <<= 1;
    Tuning t = make_tuning(l, tpr, 256 / tpr, true);
    t.bits = true;  // untuned classes take the bit-sliced kernel where it applies
    return t;
}

// Shapes for lattices launched together: they must share the CTA size, so
// tuned shapes are used only if they agree; otherwise the defaults.
std::vector<Tuning> tune_batch(const std::vector<const gbmc_lattice*>& ls) {
    std::vector<Tuning> t;
    for (auto* l : ls) t.push_back(tune(l));
    for (auto& x : t)
        if (x.threads != t[0].threads) {
            t.clear();
            for (auto* l : ls) t.push_back(tune(l, false));
            break;
        }
    return t;
}

SweepJob base_job(const gbmc_lattice* l, const Tuning& tu) {
    SweepJob J;
    std::memset(&J, 0, sizeof(J));
    J.src = l->cur;
    J.dst = l->cur;
    J.jbits = l->jbits;
    J.jsplit = l->jsplit;
    J.jb3 = l->jb3;
    J.seed = l->d.seed;
    J.L = (uint32_t)l->d.L;
    J.N = (uint32_t)l->N;
    J.R = l->d.n_replicas;
    J.n_inst = l->d.n_instances;
    J.inst_base = l->d.instance_base;
    J.t0 = l->t;
    J.rpc = tu.rpc;
    J.ctas_per_inst = (J.R + tu.rpc - 1) / tu.rpc;
    J.e_lo = -(int32_t)(l->d.dim * l->N);
    J.nbins = (uint32_t)(l->d.dim * l->N / 2 + 1);
    return J;
}

// Multi-spin-coded sweeps: supported lattices and groups of 32 per CTA (the
// count that fills the last wave of CTAs best).
bool msc_ok(const gbmc_lattice* l) {
    return l->d.dim == 2 && l->d.model == GBMC_ISING_FM && l->d.layout == GBMC_INT8 && l->d.L % 16 == 0 &&
           msc_smem_bytes((uint32_t)l->N, 1) <= kSmemLimit;
}

uint32_t msc_groups(const gbmc_ctx* ctx, const gbmc_lattice* l) {
    const uint64_t groups = (uint64_t)l->d.n_instances * ((l->d.n_replicas + 31) / 32);
    uint32_t G = msc_pick_groups((uint32_t)l->N, groups, ctx->sm_count);
    const uint32_t need = (l->d.n_replicas + 31) / 32;
    return G > need ? need : G;
}

// One multi-spin-coded sweep launch of P's jobs (their rpc = 32 G).
gbmc_status launch_msc_jobs(gbmc_ctx* ctx, SweepLaunch& P, uint32_t G) {
    uint32_t total = 0;
    for (int j = 0; j < P.njobs; ++j) {
        P.jobs[j].rpc = 32 * G;
        P.jobs[j].ctas_per_inst = (P.jobs[j].R + 32 * G - 1) / (32 * G);
        P.cta_begin[j] = total;
        total += P.jobs[j].n_inst * P.jobs[j].ctas_per_inst;
    }
    P.cta_begin[P.njobs] = total;
    P.total = total;
    ProfScope ps_(ctx, PK_SWEEP_MSC);
    CUDA_TRY(launch_sweep_msc(P, total, G, ctx->stream));
    return GBMC_OK;
}

// Enqueues one resident sweep launch of P's jobs. force_persistent: -1 takes
// the context's launch mode (AUTO: the tuned shapes' choice, persistent for
// batches of several lattices), 0 / 1 force a grid / persistent launch.
gbmc_status launch_bytes(gbmc_ctx* ctx, const SweepLaunch& P0, const std::vector<Tuning>& tu,
                         int force_persistent) {
    bool persistent = P0.njobs > 1;
    for (int j = 0; j < P0.njobs; ++j) persistent = persistent || tu[j].persistent;
    if (ctx->launch_mode == GBMC_LAUNCH_GRID) persistent = false;
    if (ctx->launch_mode == GBMC_LAUNCH_PERSISTENT) persistent = true;
    if (force_persistent >= 0) persistent = force_persistent != 0;
    SweepLaunch P = P0;
    if (persistent && P.njobs > 1) {
        // units are claimed in job order: largest copies first shortens the tail
        int order[kMaxJobs];
        for (int j = 0; j < P.njobs; ++j) order[j] = j;
        for (int a = 1; a < P.njobs; ++a)
            for (int b = a; b > 0 && P0.jobs[order[b]].N > P0.jobs[order[b - 1]].N; --b) {
                const int t = order[b];
                order[b] = order[b - 1];
                order[b - 1] = t;
            }
        for (int j = 0; j < P.njobs; ++j) P.jobs[j] = P0.jobs[order[j]];
    }
    uint32_t total = 0, threads = 0;
    for (int j = 0; j < P.njobs; ++j) {
        P.cta_begin[j] = total;
        total += P.jobs[j].n_inst * P.jobs[j].ctas_per_inst;
        if (tu[j].threads > threads) threads = tu[j].threads;
    }
    P.cta_begin[P.njobs] = total;
    P.total = total;
    P.work = persistent ? ctx->words + 2 : nullptr;
    P.rowwise = 1;
    for (int j = 0; j < P0.njobs; ++j) {
        const uint32_t W = P0.jobs[j].L / 8, tpr = threads / P0.jobs[j].rpc;
        if (W == 0 || tpr % W != 0 || !tu[j].rowwise) P.rowwise = 0;
    }
    // every job must use the same thread count: copies per CTA scale with it
    for (int j = 0; j < P0.njobs; ++j)
        if (tu[j].threads != threads)
            return fail(GBMC_ERR_ARG, "lattices of one launch need equal CTA shapes");
    const size_t smem = resident_smem_bytes(P);
    ProfScope ps_(ctx, PK_SWEEP_RES);
    CUDA_TRY(launch_sweep_resident(P, total, threads, smem, ctx->stream));
    return GBMC_OK;
}

// Whether the bit-sliced kernel takes job J of launch P under kernel mode k.
bool job_takes_bits(const SweepLaunch& P, const SweepJob& J, const Tuning& tu, int kernel) {
    if (kernel == GBMC_KERNEL_BYTES || !bits_supported(P.dim, (int)J.L)) return false;
    if (P.ea && !J.jb3) return false;
    return kernel == GBMC_KERNEL_BITS || tu.bits;
}

// Enqueues the sweep launches of P's jobs: the jobs the bit-sliced kernel
// takes in one launch of it, the others in one byte-plane resident launch.
// force_kernel: -1 takes the context's kernel mode.
gbmc_status launch_jobs(gbmc_ctx* ctx, const SweepLaunch& P0, const std::vector<Tuning>& tu,
                        int force_persistent = -1, int force_kernel = -1) {
    const int kernel = force_kernel >= 0 ? force_kernel : ctx->sweep_kernel;
    SweepLaunch B = P0, Y = P0;
    B.njobs = Y.njobs = 0;
    std::vector<Tuning> ty;
    for (int j = 0; j < P0.njobs; ++j) {
        if (job_takes_bits(P0, P0.jobs[j], tu[j], kernel)) {
            B.jobs[B.njobs++] = P0.jobs[j];
        } else {
            Y.jobs[Y.njobs++] = P0.jobs[j];
            ty.push_back(tu[j]);
        }
    }
    if (B.njobs) {
        ProfScope ps_(ctx, PK_SWEEP_BITS);
        CUDA_TRY(launch_sweep_bits(B, ctx->stream));
    }
    if (Y.njobs == 0) return GBMC_OK;
    return launch_bytes(ctx, Y, ty, force_persistent);
}

gbmc_status dalloc(gbmc_pa* pa, void** p, size_t bytes) {
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) return fail(GBMC_ERR_OOM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
    pa->allocs.push_back(*p);
    return GBMC_OK;
}

}  // namespace

extern "C" {

int gbmc_version(void) { return 100; }

int32_t gbmc_checked_build(void) {
#ifdef GBMC_CHECK
    return 1;
#else
    return 0;
#endif
}

const char* gbmc_last_error(void) { return g_err.c_str(); }

gbmc_status gbmc_create(gbmc_ctx** out, int device, void* cuda_stream) {
    if (!out) return fail(GBMC_ERR_ARG, "out is NULL");
    int n = 0;
    CUDA_TRY(cudaGetDeviceCount(&n));
    if (device < 0 || device >= n) return fail(GBMC_ERR_ARG, "device %d out of range (%d devices)", device, n);
    CUDA_TRY(cudaSetDevice(device));
    gbmc_ctx* c = new (std::nothrow) gbmc_ctx();
    if (!c) return fail(GBMC_ERR_OOM, "host allocation");
    c->device = device;
    c->stream = (cudaStream_t)cuda_stream;
    CUDA_TRY(cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device));
    int coop = 0;
    CUDA_TRY(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device));
    c->fused = coop != 0;
    c->coop = coop != 0;
    {
        cudaError_t e = cudaMalloc(&c->words, kCtxWords * sizeof(unsigned int));
        if (e != cudaSuccess) {
            delete c;
            return fail(GBMC_ERR_OOM, "cudaMalloc(context words): %s", cudaGetErrorString(e));
        }
        e = cudaMemset(c->words, 0, kCtxWords * sizeof(unsigned int));
        if (e != cudaSuccess) {
            cudaFree(c->words);
            delete c;
            return fail(GBMC_ERR_CUDA, "cudaMemset: %s", cudaGetErrorString(e));
        }
    }
    *out = c;
    return GBMC_OK;
}

gbmc_status gbmc_set_stream(gbmc_ctx* ctx, void* cuda_stream) {
    if (!ctx) return fail(GBMC_ERR_ARG, "ctx is NULL");
    ctx->stream = (cudaStream_t)cuda_stream;
    return GBMC_OK;
}

// Reads (and clears) the device error flags: a bounded wait that ran out
// (word 1) and a population that outgrew its capacity (word 4); the stream
// must have been synchronised.
static gbmc_status check_device_error(gbmc_ctx* ctx) {
#ifdef GBMC_CHECK
    for (const auto& c : check_entries()) {
        unsigned line = 0;
        if (c.read(&line)) {
            const char* f = std::strrchr(c.file, '/');
            return fail(GBMC_ERR_STATE, "bounds check failed in %s:%u", f ? f + 1 : c.file, line);
        }
    }
#endif
    unsigned int w[8] = {};
    CUDA_TRY(cudaMemcpy(w, ctx->words, sizeof(w), cudaMemcpyDeviceToHost));
    if (w[1]) {
        CUDA_TRY(cudaMemset(ctx->words + 1, 0, sizeof(unsigned int)));
        return fail(GBMC_ERR_TIMEOUT, "a grid barrier wait ran out of its cycle budget; results since the last "
                                      "check are invalid");
    }
    if (w[4]) {
        CUDA_TRY(cudaMemset(ctx->words + 4, 0, sizeof(unsigned int)));
        return fail(GBMC_ERR_STATE, "a population outgrew its capacity (nearest-integer resampling); the run "
                                    "is invalid");
    }
    return GBMC_OK;
}

gbmc_status gbmc_sync(gbmc_ctx* ctx) {
    if (!ctx) return fail(GBMC_ERR_ARG, "ctx is NULL");
    CUDA_TRY(cudaSetDevice(ctx->device));
    CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    return check_device_error(ctx);
}

gbmc_status gbmc_set_sweep_launch(gbmc_ctx* ctx, int32_t mode) {
    if (!ctx) return fail(GBMC_ERR_ARG, "ctx is NULL");
    if (mode != GBMC_LAUNCH_AUTO && mode != GBMC_LAUNCH_GRID && mode != GBMC_LAUNCH_PERSISTENT)
        return fail(GBMC_ERR_ARG, "unknown sweep launch mode %d", mode);
    ctx->launch_mode = mode;
    return GBMC_OK;
}

gbmc_status gbmc_set_sweep_kernel(gbmc_ctx* ctx, int32_t kernel) {
    if (!ctx) return fail(GBMC_ERR_ARG, "ctx is NULL");
    if (kernel != GBMC_KERNEL_AUTO && kernel != GBMC_KERNEL_BYTES && kernel != GBMC_KERNEL_BITS)
        return fail(GBMC_ERR_ARG, "unknown sweep kernel %d", kernel);
    ctx->sweep_kernel = kernel;
    return GBMC_OK;
}

gbmc_status gbmc_set_resample_mode(gbmc_ctx* ctx, int32_t fused) {
    if (!ctx) return fail(GBMC_ERR_ARG, "ctx is NULL");
    int coop = 0;
    CUDA_TRY(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, ctx->device));
    if (fused && !coop) return fail(GBMC_ERR_STATE, "device has no cooperative launch");
    ctx->fused = fused != 0;
    return GBMC_OK;
}

gbmc_status gbmc_test_barrier_wait(gbmc_ctx* ctx, uint32_t phantom_arrivals, uint64_t budget_cycles) {
    if (!ctx) return fail(GBMC_ERR_ARG, "ctx is NULL");
    if (budget_cycles == 0 || budget_cycles > (1ull << 40)) return fail(GBMC_ERR_ARG, "budget out of range");
    ctx->phantom = phantom_arrivals;
    ctx->budget = (long long)budget_cycles;
    return GBMC_OK;
}

gbmc_status gbmc_destroy(gbmc_ctx* ctx) {
    if (!ctx) return GBMC_OK;
    cudaStreamSynchronize(ctx->stream);
    for (auto& p : ctx->pending) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    for (auto e : ctx->pool) cudaEventDestroy(e);
    if (ctx->words) cudaFree(ctx->words);
    delete ctx;
    return GBMC_OK;
}

gbmc_status gbmc_profile(gbmc_ctx* ctx, int32_t enable) {
    if (!ctx) return fail(GBMC_ERR_ARG, "ctx is NULL");
    CUDA_TRY(cudaSetDevice(ctx->device));
    CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    for (auto& p : ctx->pending) {
        ctx->pool.push_back(p.a);
        ctx->pool.push_back(p.b);
    }
    ctx->pending.clear();
    if (enable)
        for (int k = 0; k < PK_COUNT; ++k) ctx->ms[k] = 0.0, ctx->launches[k] = 0;
    ctx->prof = enable != 0;
    return GBMC_OK;
}

gbmc_status gbmc_profile_read(gbmc_ctx* ctx, gbmc_kernel_time* out, uint32_t capacity, uint32_t* n_out) {
    if (!ctx) return fail(GBMC_ERR_ARG, "ctx is NULL");
    CUDA_TRY(cudaSetDevice(ctx->device));
    CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    for (auto& p : ctx->pending) {
        float ms = 0.f;
        CUDA_TRY(cudaEventElapsedTime(&ms, p.a, p.b));
        ctx->ms[p.kind] += ms;
        ctx->launches[p.kind] += p.launches;
        ctx->pool.push_back(p.a);
        ctx->pool.push_back(p.b);
    }
    ctx->pending.clear();
    uint32_t n = 0;
    for (int k = 0; k < PK_COUNT; ++k) {
        if (ctx->launches[k] == 0) continue;
        if (out && n < capacity) {
            std::memset(&out[n], 0, sizeof(out[n]));
            std::snprintf(out[n].name, sizeof(out[n].name), "%s", kProfNames[k]);
            out[n].launches = ctx->launches[k];
            out[n].total_ms = ctx->ms[k];
        }
        ++n;
    }
    if (n_out) *n_out = n;
    return GBMC_OK;
}

uint64_t gbmc_kernel_launches(void) { return g_launches.load(); }

gbmc_status lattice_init(gbmc_ctx* ctx, const gbmc_lattice_desc* d, void* spins_dev, size_t spins_bytes,
                         gbmc_lattice** out) {
    if (!ctx || !d || !out) return fail(GBMC_ERR_ARG, "NULL argument");
    if (d->dim != 2 && d->dim != 3) return fail(GBMC_ERR_ARG, "dim must be 2 or 3 (got %d)", d->dim);
    if (d->L < 2 || (d->L & 1)) return fail(GBMC_ERR_ARG, "L must be even and >= 2 (got %d)", d->L);
    if ((d->dim == 2 && d->L > 32768) || (d->dim == 3 && d->L > 1024))
        return fail(GBMC_ERR_ARG, "L too large");
    if (d->model != GBMC_ISING_FM && d->model != GBMC_EA_PMJ) return fail(GBMC_ERR_ARG, "unknown model");
    if (d->model == GBMC_EA_PMJ && d->dim != 3) return fail(GBMC_ERR_ARG, "the +-J model is three-dimensional");
    if (d->layout != GBMC_INT8 && d->layout != GBMC_BITPACK) return fail(GBMC_ERR_ARG, "unknown layout %d", d->layout);
    if (d->layout == GBMC_BITPACK && (d->dim != 2 || d->model != GBMC_ISING_FM || d->L % 64 != 0))
        return fail(GBMC_ERR_ARG, "the bit-packed layout needs a 2D ferromagnet with L %% 64 == 0");
    if (d->start != GBMC_START_ALL_UP && d->start != GBMC_START_RANDOM) return fail(GBMC_ERR_ARG, "unknown start");
    if (d->n_instances == 0 || d->n_replicas == 0) return fail(GBMC_ERR_ARG, "empty lattice set");
    if ((uint64_t)d->instance_base + d->n_instances > (1ull << 27)) return fail(GBMC_ERR_ARG, "instance ids exceed 2^27");
    uint64_t N = 1;
    for (int i = 0; i < d->dim; ++i) N *= (uint64_t)d->L;
    const uint64_t ncopies = (uint64_t)d->n_instances * d->n_replicas;
    if (d->n_replicas > 0xFFFFFFFFull || N * (uint64_t)d->dim > 0x7FFFFFFFull)
        return fail(GBMC_ERR_ARG, "lattice too large for 32-bit energies");
    const uint64_t bytes = d->layout == GBMC_BITPACK ? ncopies * (N / 8) : ncopies * N;
    if (spins_dev) {
        if (spins_bytes < bytes) return fail(GBMC_ERR_ARG, "spins buffer has %zu bytes, need %llu", spins_bytes, (unsigned long long)bytes);
        if (((uintptr_t)spins_dev & 15) != 0) return fail(GBMC_ERR_ARG, "spins buffer must be 16-byte aligned");
        if (!is_device_ptr(spins_dev)) return fail(GBMC_ERR_ARG, "spins buffer is not device memory");
    }
    CUDA_TRY(cudaSetDevice(ctx->device));
    gbmc_lattice* l = new (std::nothrow) gbmc_lattice;
    if (!l) return fail(GBMC_ERR_OOM, "host allocation");
    std::memset(l, 0, sizeof(*l));
    l->ctx = ctx;
    l->d = *d;
    l->N = N;
    l->ncopies = ncopies;
    if (spins_dev) {
        l->spins = (int8_t*)spins_dev;
    } else {
        cudaError_t e = cudaMalloc(&l->spins, bytes);
        if (e != cudaSuccess) {
            delete l;
            return fail(GBMC_ERR_OOM, "cudaMalloc(%llu): %s", (unsigned long long)bytes, cudaGetErrorString(e));
        }
        l->owns_spins = true;
    }
    l->cur = l->spins;
    if (d->model == GBMC_EA_PMJ) {
        cudaError_t e = cudaMalloc(&l->jbits, 3 * N * d->n_instances);
        if (e != cudaSuccess) {
            if (l->owns_spins) cudaFree(l->spins);
            delete l;
            return fail(GBMC_ERR_OOM, "cudaMalloc(couplings): %s", cudaGetErrorString(e));
        }
        ProfScope ps_(ctx, PK_COUPLINGS);
        CUDA_TRY(launch_couplings(l->jbits, (uint32_t)d->L, d->n_instances, d->instance_base, d->seed, ctx->stream));
        if (d->L % 8 == 0) {
            e = cudaMalloc(&l->jsplit, 6 * N * d->n_instances);
            if (e != cudaSuccess) {
                cudaFree(l->jbits);
                if (l->owns_spins) cudaFree(l->spins);
                delete l;
                return fail(GBMC_ERR_OOM, "cudaMalloc(split couplings): %s", cudaGetErrorString(e));
            }
            CUDA_TRY(launch_split_bonds(l->jbits, l->jsplit, (uint32_t)d->L, d->n_instances, ctx->stream));
        }
        if (bits_supported(d->dim, d->L)) {
            e = cudaMalloc(&l->jb3, bits3_bond_words((uint32_t)d->L) * 4 * d->n_instances);
            if (e != cudaSuccess) {
                if (l->jsplit) cudaFree(l->jsplit);
                cudaFree(l->jbits);
                if (l->owns_spins) cudaFree(l->spins);
                delete l;
                return fail(GBMC_ERR_OOM, "cudaMalloc(bond words): %s", cudaGetErrorString(e));
            }
            CUDA_TRY(launch_bits3_bonds(l->jbits, l->jb3, (uint32_t)d->L, d->n_instances, ctx->stream));
        }
    }
    {
        ProfScope ps_(ctx, PK_INIT);
        if (d->layout == GBMC_BITPACK)
            CUDA_TRY(launch_bp_init((uint32_t*)l->spins, (uint32_t)d->L, ncopies, d->n_replicas, d->instance_base,
                                    d->seed, d->start == GBMC_START_RANDOM, ctx->stream));
        else
            CUDA_TRY(launch_init_spins(l->spins, d->dim, (uint32_t)d->L, d->n_instances, d->n_replicas,
                                       d->instance_base, d->seed, d->start == GBMC_START_RANDOM, ctx->stream));
    }
    *out = l;
    return GBMC_OK;
}

gbmc_status lattice_free(gbmc_lattice* l) {
    if (!l) return GBMC_OK;
    if (l->run) return fail(GBMC_ERR_STATE, "lattice still used by an annealing run");
    if (l->owns_spins) cudaFree(l->spins);
    if (l->jbits) cudaFree(l->jbits);
    if (l->jsplit) cudaFree(l->jsplit);
    if (l->jb3) cudaFree(l->jb3);
    if (l->packed) cudaFree(l->packed);
    if (l->dcb_scratch) cudaFree(l->dcb_scratch);
    if (l->alt) cudaFree(l->alt);
    if (l->sw_bonds) cudaFree(l->sw_bonds);
    if (l->sw_parent) cudaFree(l->sw_parent);
    if (l->sw_lab) cudaFree(l->sw_lab);
    delete l;
    return GBMC_OK;
}

gbmc_status lattice_info(const gbmc_lattice* l, gbmc_lattice_info* out) {
    if (!l || !out) return fail(GBMC_ERR_ARG, "NULL argument");
    out->n_sites = (int64_t)l->N;
    out->n_copies = (int64_t)l->ncopies;
    out->spin_bytes = (int64_t)(l->d.layout == GBMC_BITPACK ? (l->N / 8) * l->ncopies : l->N * l->ncopies);
    out->sweep_counter = l->t;
    out->pad = 0;
    out->spins_dev = l->cur;
    return GBMC_OK;
}

gbmc_status lattice_set_sweep_counter(gbmc_lattice* l, uint32_t t) {
    if (!l) return fail(GBMC_ERR_ARG, "NULL lattice");
    l->t = t;
    return GBMC_OK;
}

gbmc_status lattice_copy_out(gbmc_ctx* ctx, const gbmc_lattice* l, int8_t* dst, size_t bytes) {
    if (!ctx || !l || !dst) return fail(GBMC_ERR_ARG, "NULL argument");
    if (bytes != l->N * l->ncopies) return fail(GBMC_ERR_ARG, "bytes must be %llu", (unsigned long long)(l->N * l->ncopies));
    if (l->d.layout == GBMC_BITPACK) {
        const bool dev = is_device_ptr(dst);
        int8_t* tmp = dst;
        if (!dev) CUDA_TRY(cudaMallocAsync((void**)&tmp, bytes, ctx->stream));
        CUDA_TRY(launch_bp_unpack((const uint32_t*)l->cur, tmp, (uint32_t)l->d.L, l->ncopies, ctx->stream));
        if (!dev) {
            CUDA_TRY(cudaMemcpyAsync(dst, tmp, bytes, cudaMemcpyDeviceToHost, ctx->stream));
            CUDA_TRY(cudaFreeAsync(tmp, ctx->stream));
            CUDA_TRY(cudaStreamSynchronize(ctx->stream));
        }
        return GBMC_OK;
    }
    CUDA_TRY(cudaMemcpyAsync(dst, l->cur, bytes, cudaMemcpyDefault, ctx->stream));
    if (!is_device_ptr(dst)) CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    return GBMC_OK;
}

gbmc_status lattice_copy_in(gbmc_ctx* ctx, gbmc_lattice* l, const int8_t* src, size_t bytes) {
    if (!ctx || !l || !src) return fail(GBMC_ERR_ARG, "NULL argument");
    if (bytes != l->N * l->ncopies) return fail(GBMC_ERR_ARG, "bytes must be %llu", (unsigned long long)(l->N * l->ncopies));
    if (l->d.layout == GBMC_BITPACK) {
        const bool dev = is_device_ptr(src);
        const int8_t* tsrc = src;
        int8_t* tmp = nullptr;
        if (!dev) {
            CUDA_TRY(cudaMallocAsync((void**)&tmp, bytes, ctx->stream));
            CUDA_TRY(cudaMemcpyAsync(tmp, src, bytes, cudaMemcpyHostToDevice, ctx->stream));
            tsrc = tmp;
        }
        CUDA_TRY(launch_bp_pack(tsrc, (uint32_t*)l->cur, (uint32_t)l->d.L, l->ncopies, ctx->stream));
        if (tmp) {
            CUDA_TRY(cudaFreeAsync(tmp, ctx->stream));
            CUDA_TRY(cudaStreamSynchronize(ctx->stream));
        }
        return GBMC_OK;
    }
    CUDA_TRY(cudaMemcpyAsync(l->cur, src, bytes, cudaMemcpyDefault, ctx->stream));
    if (!is_device_ptr(src)) CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    return GBMC_OK;
}

gbmc_status lattice_couplings_out(gbmc_ctx* ctx, const gbmc_lattice* l, int8_t* dst, size_t bytes) {
    if (!ctx || !l || !dst) return fail(GBMC_ERR_ARG, "NULL argument");
    if (!l->jbits) return fail(GBMC_ERR_STATE, "lattice has no couplings (ferromagnet)");
    const size_t need = 3 * l->N * l->d.n_instances;
    if (bytes != need) return fail(GBMC_ERR_ARG, "bytes must be %zu", need);
    int8_t* tmp = dst;
    const bool dev = is_device_ptr(dst);
    if (!dev) CUDA_TRY(cudaMallocAsync((void**)&tmp, need, ctx->stream));
    CUDA_TRY(launch_jbits_to_int8(l->jbits, tmp, (uint32_t)l->N, l->d.n_instances, ctx->stream));
    if (!dev) {
        CUDA_TRY(cudaMemcpyAsync(dst, tmp, need, cudaMemcpyDeviceToHost, ctx->stream));
        CUDA_TRY(cudaFreeAsync(tmp, ctx->stream));
        CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    }
    return GBMC_OK;
}

gbmc_status metropolis_sweeps(gbmc_ctx* ctx, gbmc_lattice* l, double beta, uint32_t n_sweeps, int32_t* E_series,
                              int32_t* M_series) {
    if (!ctx || !l) return fail(GBMC_ERR_ARG, "NULL argument");
    if (!beta_ok(beta, l->d.dim)) return fail(GBMC_ERR_ARG, "beta must satisfy 0 <= 4*dim*beta <= 700 (got %g)", beta);
    if (l->run) return fail(GBMC_ERR_STATE, "lattice is owned by an annealing run");
    if (n_sweeps == 0) return GBMC_OK;
    if ((uint64_t)l->t + n_sweeps > 0xFFFFFFFFull) return fail(GBMC_ERR_ARG, "sweep counter would wrap");
    CUDA_TRY(cudaSetDevice(ctx->device));
    if (l->d.layout == GBMC_BITPACK) {
        uint32_t thr[3];
        thresholds(beta, thr);
        uint32_t Gc = 0, rmax = 0, threads = 0;
        size_t smem = 0;
        if (!E_series && !M_series && ctx->launch_mode != GBMC_LAUNCH_GRID && ctx->coop && n_sweeps <= 0x40000000u &&
            ctx->sm_count <= (int)(kCtxWords - 8) &&
            bp_strips_shape((uint32_t)l->d.L, l->ncopies, ctx->sm_count, Gc, rmax, threads, smem)) {
            // every sweep of the call in one cooperative launch, strips resident in shared memory
            BpStrips S;
            std::memset(&S, 0, sizeof(S));
            S.P = (uint32_t*)l->cur;
            S.progress = ctx->words + 8;
            S.err = ctx->words + 1;
            S.budget = ctx->budget;
            S.seed = l->d.seed;
            S.L = (uint32_t)l->d.L;
            S.Gc = Gc;
            S.rmax = rmax;
            S.R = l->d.n_replicas;
            S.inst_base = l->d.instance_base;
            S.t0 = l->t;
            S.n_half = 2 * n_sweeps;
            S.T4 = thr[0];
            S.T8 = thr[1];
            S.phantom = ctx->phantom;
            {
                ProfScope ps_(ctx, PK_BP_STRIPS);
                CUDA_TRY(launch_bp_strips(S, l->ncopies, threads, smem, ctx->sm_count, ctx->stream));
            }
            l->t += n_sweeps;
            return GBMC_OK;
        }
        for (uint32_t s = 0; s < n_sweeps; ++s) {
            for (uint32_t colour = 0; colour < 2; ++colour) {
                ProfScope ps_(ctx, PK_BP_HALFSWEEP);
                CUDA_TRY(launch_bp_halfsweep((uint32_t*)l->cur, (uint32_t)l->d.L, l->ncopies, l->d.n_replicas,
                                             l->d.instance_base, l->d.seed, colour, l->t + s, thr[0], thr[1],
                                             ctx->stream));
            }
            if (E_series || M_series) {
                ProfScope ps_(ctx, PK_OBS);
                CUDA_TRY(launch_bp_observables((const uint32_t*)l->cur, (uint32_t)l->d.L, l->ncopies,
                                               E_series ? E_series + (uint64_t)s * l->ncopies : nullptr,
                                               M_series ? M_series + (uint64_t)s * l->ncopies : nullptr, ctx->stream));
            }
        }
        l->t += n_sweeps;
        return GBMC_OK;
    }
    const Tuning tu = tune(l);
    SweepJob J = base_job(l, tu);
    thresholds(beta, J.thr);
    {
        // large 2D ferromagnets in the int8 layout, every sweep of the call in one
        // launch of the bit-packed strip kernel: the configuration is packed to one
        // bit per spin first and unpacked after (same Philox words, same spins as
        // the byte strip kernel, a fraction of its instructions per update)
        uint32_t Gc = 0, rmax = 0, threads = 0;
        size_t smem = 0;
        if (!tu.resident && ctx->sweep_kernel != GBMC_KERNEL_BYTES && l->d.dim == 2 &&
            l->d.model == GBMC_ISING_FM && !E_series && !M_series && ctx->launch_mode != GBMC_LAUNCH_GRID &&
            ctx->coop && n_sweeps <= 0x40000000u && ctx->sm_count <= (int)(kCtxWords - 8) &&
            bp_strips_shape((uint32_t)l->d.L, l->ncopies, ctx->sm_count, Gc, rmax, threads, smem)) {
            if (!l->packed) {
                cudaError_t e = cudaMalloc(&l->packed, l->ncopies * (l->N / 8));
                if (e != cudaSuccess) return fail(GBMC_ERR_OOM, "cudaMalloc(packed copy): %s", cudaGetErrorString(e));
            }
            {
                ProfScope ps_(ctx, PK_BP_PACK);
                CUDA_TRY(launch_bp_pack(l->cur, l->packed, (uint32_t)l->d.L, l->ncopies, ctx->stream));
            }
            BpStrips S;
            std::memset(&S, 0, sizeof(S));
            S.P = l->packed;
            S.progress = ctx->words + 8;
            S.err = ctx->words + 1;
            S.budget = ctx->budget;
            S.seed = l->d.seed;
            S.L = (uint32_t)l->d.L;
            S.Gc = Gc;
            S.rmax = rmax;
            S.R = l->d.n_replicas;
            S.inst_base = l->d.instance_base;
            S.t0 = l->t;
            S.n_half = 2 * n_sweeps;
            S.T4 = J.thr[0];
            S.T8 = J.thr[1];
            S.phantom = ctx->phantom;
            {
                ProfScope ps_(ctx, PK_BP_STRIPS);
                CUDA_TRY(launch_bp_strips(S, l->ncopies, threads, smem, ctx->sm_count, ctx->stream));
            }
            {
                ProfScope ps_(ctx, PK_BP_PACK);
                CUDA_TRY(launch_bp_unpack(l->packed, l->cur, (uint32_t)l->d.L, l->ncopies, ctx->stream));
            }
            l->t += n_sweeps;
            return GBMC_OK;
        }
    }
    // strips of rows resident in shared memory for the whole call (large 2D ferromagnets, no E/M series)
    uint32_t sGc = 0, srmax = 0, sthreads = 0;
    size_t ssmem = 0;
    const bool strips = !tu.resident && l->d.dim == 2 && l->d.model == GBMC_ISING_FM && !E_series && !M_series &&
                        ctx->launch_mode != GBMC_LAUNCH_GRID && ctx->coop && n_sweeps <= 0x40000000u &&
                        ctx->sm_count <= (int)(kCtxWords - 8) &&
                        strips_shape((uint32_t)l->d.L, l->ncopies, ctx->sm_count, sGc, srmax, sthreads, ssmem);
    if (tu.resident) {
        SweepLaunch P;
        std::memset(&P, 0, sizeof(P));
        J.nsweeps = n_sweeps;
        J.Eser = E_series;
        J.Mser = M_series;
        P.jobs[0] = J;
        P.njobs = 1;
        P.dim = l->d.dim;
        P.ea = l->d.model == GBMC_EA_PMJ;
        P.swar = (l->d.L % 8) == 0;
        gbmc_status st = launch_jobs(ctx, P, std::vector<Tuning>{tu});
        if (st != GBMC_OK) return st;
    } else if (strips) {
        // large 2D lattices: every sweep of the call in one cooperative launch, strips resident in shared memory
        StripLaunch S;
        std::memset(&S, 0, sizeof(S));
        S.spins = l->cur;
        S.progress = ctx->words + 8;
        S.err = ctx->words + 1;
        S.budget = ctx->budget;
        S.seed = l->d.seed;
        S.L = (uint32_t)l->d.L;
        S.Gc = sGc;
        S.rmax = srmax;
        S.R = l->d.n_replicas;
        S.inst_base = l->d.instance_base;
        S.t0 = l->t;
        S.n_half = 2 * n_sweeps;
        S.phantom = ctx->phantom;
        S.thr[0] = J.thr[0];
        S.thr[1] = J.thr[1];
        ProfScope ps_(ctx, PK_SWEEP_STRIPS);
        CUDA_TRY(launch_sweep_strips(S, l->ncopies, sthreads, ssmem, ctx->sm_count, ctx->stream));
    } else if (l->d.dim == 2 && l->d.model == GBMC_ISING_FM && l->d.L % kTile == 0) {
        // large 2D lattices: shared-memory tiles with halos, up to 4 sweeps per launch
        if (!l->alt) {
            cudaError_t e = cudaMalloc(&l->alt, l->N * l->ncopies);
            if (e != cudaSuccess) return fail(GBMC_ERR_OOM, "cudaMalloc(second buffer): %s", cudaGetErrorString(e));
        }
        TileLaunch TL;
        std::memset(&TL, 0, sizeof(TL));
        TL.seed = l->d.seed;
        TL.L = (uint32_t)l->d.L;
        TL.T = kTile;
        TL.R = l->d.n_replicas;
        TL.inst_base = l->d.instance_base;
        TL.thr[0] = J.thr[0];
        TL.thr[1] = J.thr[1];
        const uint32_t chunk = (E_series || M_series) ? 1u : 4u;
        for (uint32_t s = 0; s < n_sweeps; s += chunk) {
            TL.src = l->cur;
            TL.dst = l->cur == l->spins ? l->alt : l->spins;
            TL.t0 = l->t + s;
            TL.nsweeps = (n_sweeps - s) < chunk ? (n_sweeps - s) : chunk;
            {
                ProfScope ps_(ctx, PK_SWEEP_TILES);
                CUDA_TRY(launch_sweep_tiles(TL, l->ncopies, ctx->stream));
            }
            l->cur = TL.dst;
            if (E_series || M_series) {
                ProfScope ps_(ctx, PK_OBS);
                CUDA_TRY(launch_observables(l->cur, l->jbits, l->d.dim, (uint32_t)l->d.L, l->d.n_instances,
                                            l->d.n_replicas, E_series ? E_series + (uint64_t)s * l->ncopies : nullptr,
                                            M_series ? M_series + (uint64_t)s * l->ncopies : nullptr, ctx->stream));
            }
        }
        if (l->cur != l->spins) {
            CUDA_TRY(cudaMemcpyAsync(l->spins, l->cur, l->N * l->ncopies, cudaMemcpyDeviceToDevice, ctx->stream));
            l->cur = l->spins;
        }
    } else {
        for (uint32_t s = 0; s < n_sweeps; ++s) {
            for (int colour = 0; colour < 2; ++colour) {
                ProfScope ps_(ctx, PK_HALFSWEEP);
                CUDA_TRY(launch_halfsweep_global(J, l->d.dim, colour, l->t + s, ctx->stream));
            }
            if (E_series || M_series) {
                ProfScope ps_(ctx, PK_OBS);
                CUDA_TRY(launch_observables(l->cur, l->jbits, l->d.dim, (uint32_t)l->d.L, l->d.n_instances,
                                            l->d.n_replicas, E_series ? E_series + (uint64_t)s * l->ncopies : nullptr,
                                            M_series ? M_series + (uint64_t)s * l->ncopies : nullptr, ctx->stream));
            }
        }
    }
    l->t += n_sweeps;
    return GBMC_OK;
}

gbmc_status swendsen_wang(gbmc_ctx* ctx, gbmc_lattice* l, double beta, uint32_t n_updates, int32_t* E_series,
                          int32_t* M_series, int32_t* labels) {
    if (!ctx || !l) return fail(GBMC_ERR_ARG, "NULL argument");
    if (!beta_ok(beta, l->d.dim)) return fail(GBMC_ERR_ARG, "beta must satisfy 0 <= 4*dim*beta <= 700 (got %g)", beta);
    if (l->run) return fail(GBMC_ERR_STATE, "lattice is owned by an annealing run");
    if (l->d.model != GBMC_ISING_FM || l->d.layout != GBMC_INT8)
        return fail(GBMC_ERR_ARG, "Swendsen-Wang updates need a ferromagnet in the int8 layout");
    if (l->N > 0x7FFFFFFFull) return fail(GBMC_ERR_ARG, "lattice too large for 32-bit cluster names");
    if (n_updates == 0) return GBMC_OK;
    if ((uint64_t)l->t + n_updates > 0xFFFFFFFFull) return fail(GBMC_ERR_ARG, "update counter would wrap");
    CUDA_TRY(cudaSetDevice(ctx->device));
    if (!l->sw_parent) {
        const bool tiled = sw_tiled((uint32_t)l->d.dim, (uint32_t)l->d.L);
        cudaError_t e = cudaMalloc(&l->sw_parent, 4 * l->N * l->ncopies);
        if (e == cudaSuccess && !tiled) e = cudaMalloc(&l->sw_bonds, l->N * l->ncopies);
        if (e == cudaSuccess && tiled && l->d.dim == 2) e = cudaMalloc(&l->sw_lab, 2 * l->N * l->ncopies);
        if (e != cudaSuccess) {
            cudaFree(l->sw_parent);
            cudaFree(l->sw_bonds);
            l->sw_bonds = nullptr;
            l->sw_parent = nullptr;
            return fail(GBMC_ERR_OOM, "cudaMalloc(Swendsen-Wang workspace): %s", cudaGetErrorString(e));
        }
    }
    SwLaunch P;
    std::memset(&P, 0, sizeof(P));
    P.spins = l->cur;
    P.bonds = l->sw_bonds;
    P.parent = l->sw_parent;
    P.lab = l->sw_lab;
    P.err = ctx->words + 1;
    P.seed = l->d.seed;
    // T_bond = ceil(p 2^32) - 1, p = 1 - exp(-2 beta): "r < p" as an integer comparison
    P.T_bond = (long long)std::ceil(std::ldexp(1.0 - std::exp(-2.0 * beta), 32)) - 1;
    P.L = (uint32_t)l->d.L;
    P.N = (uint32_t)l->N;
    P.dim = (uint32_t)l->d.dim;
    P.R = l->d.n_replicas;
    P.inst_base = l->d.instance_base;
    if ((P.L & (P.L - 1)) == 0)
        while ((1u << P.lshift) < P.L) ++P.lshift;
    for (uint32_t u = 0; u < n_updates; ++u) {
        P.t = l->t + u;
        P.labels = u + 1 == n_updates ? labels : nullptr;
        {
            ProfScope ps_(ctx, PK_SW);
            CUDA_TRY(launch_sw_update(P, l->ncopies, ctx->stream));
        }
        if (E_series || M_series) {
            ProfScope ps_(ctx, PK_OBS);
            CUDA_TRY(launch_observables(l->cur, l->jbits, l->d.dim, (uint32_t)l->d.L, l->d.n_instances,
                                        l->d.n_replicas, E_series ? E_series + (uint64_t)u * l->ncopies : nullptr,
                                        M_series ? M_series + (uint64_t)u * l->ncopies : nullptr, ctx->stream));
        }
    }
    l->t += n_updates;
    return GBMC_OK;
}

gbmc_status metropolis_sweeps_msc(gbmc_ctx* ctx, gbmc_lattice* l, double beta, uint32_t n_sweeps) {
    if (!ctx || !l) return fail(GBMC_ERR_ARG, "NULL argument");
    if (!beta_ok(beta, l->d.dim)) return fail(GBMC_ERR_ARG, "beta must satisfy 0 <= 4*dim*beta <= 700 (got %g)", beta);
    if (l->run) return fail(GBMC_ERR_STATE, "lattice is owned by an annealing run");
    if (!msc_ok(l))
        return fail(GBMC_ERR_ARG, "multi-spin-coded sweeps need a 2D ferromagnet, int8 layout, L %% 16 == 0, L <= 208");
    if (n_sweeps == 0) return GBMC_OK;
    if ((uint64_t)l->t + n_sweeps > 0xFFFFFFFFull) return fail(GBMC_ERR_ARG, "sweep counter would wrap");
    CUDA_TRY(cudaSetDevice(ctx->device));
    const Tuning tu = tune(l, false);
    SweepJob J = base_job(l, tu);
    thresholds(beta, J.thr);
    J.nsweeps = n_sweeps;
    SweepLaunch P;
    std::memset(&P, 0, sizeof(P));
    P.jobs[0] = J;
    P.njobs = 1;
    P.dim = 2;
    gbmc_status st = launch_msc_jobs(ctx, P, msc_groups(ctx, l));
    if (st != GBMC_OK) return st;
    l->t += n_sweeps;
    return GBMC_OK;
}

gbmc_status metropolis_sweeps_dcb(gbmc_ctx* ctx, gbmc_lattice* l, double beta, uint32_t n_rounds, uint32_t k,
                                  uint32_t tile, int32_t* E_series, int32_t* M_series) {
    if (!ctx || !l) return fail(GBMC_ERR_ARG, "NULL argument");
    if (!beta_ok(beta, l->d.dim)) return fail(GBMC_ERR_ARG, "beta must satisfy 0 <= 4*dim*beta <= 700 (got %g)", beta);
    if (l->run) return fail(GBMC_ERR_STATE, "lattice is owned by an annealing run");
    if (l->d.dim != 2 || l->d.model != GBMC_ISING_FM || l->d.layout != GBMC_INT8)
        return fail(GBMC_ERR_ARG, "double-checkerboard sweeps need a 2D ferromagnet in the int8 layout");
    if (tile != 32 && tile != 64 && tile != 128) return fail(GBMC_ERR_ARG, "tile must be 32, 64 or 128 (got %u)", tile);
    if (l->d.L % (2 * tile) != 0) return fail(GBMC_ERR_ARG, "L = %d is not a multiple of 2 * tile", (int)l->d.L);
    if (k == 0) return fail(GBMC_ERR_ARG, "k must be >= 1");
    if (n_rounds == 0) return GBMC_OK;
    if ((uint64_t)l->t + (uint64_t)n_rounds * k > 0xFFFFFFFFull) return fail(GBMC_ERR_ARG, "sweep counter would wrap");
    CUDA_TRY(cudaSetDevice(ctx->device));
    uint32_t thr[3];
    thresholds(beta, thr);
    TileLaunch TL;
    std::memset(&TL, 0, sizeof(TL));
    TL.src = TL.dst = l->cur;
    TL.seed = l->d.seed;
    TL.L = (uint32_t)l->d.L;
    TL.T = tile;
    TL.R = l->d.n_replicas;
    TL.inst_base = l->d.instance_base;
    TL.thr[0] = thr[0];
    TL.thr[1] = thr[1];
    TL.nsweeps = k;
    // bit-sliced tiles (the same spins) unless the byte-plane kernels are forced
    const bool bits = dcb_bits_supported(tile) && ctx->sweep_kernel != GBMC_KERNEL_BYTES;
    // every round in one launch, the tiles resident in registers: worth it for
    // small k, where loading and storing the tiles every round dominates; for
    // larger k the per-round launches are faster (a launch ends when its SM
    // work is done, while resident tiles that run ahead of their neighbours
    // take issue slots from the slower ones)
    const uint32_t k_resident = tile == 64 ? 3u : 7u;
    const bool resident_mode = ctx->launch_mode == GBMC_LAUNCH_PERSISTENT ||
                               (ctx->launch_mode == GBMC_LAUNCH_AUTO && k <= k_resident);
    if (bits && !E_series && !M_series && resident_mode && ctx->coop &&
        dcb_resident_fits(TL.L, tile, l->ncopies, ctx->sm_count)) {
        const size_t need = dcb_resident_bytes(TL.L, tile, l->ncopies);
        if (l->dcb_scratch_bytes < need) {
            if (l->dcb_scratch) {
                CUDA_TRY(cudaStreamSynchronize(ctx->stream));
                cudaFree(l->dcb_scratch);
                l->dcb_scratch = nullptr;
                l->dcb_scratch_bytes = 0;
            }
            cudaError_t e = cudaMalloc(&l->dcb_scratch, need);
            if (e != cudaSuccess) return fail(GBMC_ERR_OOM, "cudaMalloc(tile edges): %s", cudaGetErrorString(e));
            l->dcb_scratch_bytes = need;
        }
        const uint64_t tiles = (uint64_t)(TL.L / tile) * (TL.L / tile) * l->ncopies;
        DcbResident D;
        std::memset(&D, 0, sizeof(D));
        D.spins = l->cur;
        D.edges = l->dcb_scratch;
        D.progress = l->dcb_scratch + tiles * (tile / 8);
        D.err = ctx->words + 1;
        D.budget = ctx->budget;
        D.seed = l->d.seed;
        D.L = TL.L;
        D.T = tile;
        D.R = l->d.n_replicas;
        D.inst_base = l->d.instance_base;
        D.t0 = l->t;
        D.k = k;
        D.n_rounds = n_rounds;
        D.phantom = ctx->phantom;
        D.thr[0] = thr[0];
        D.thr[1] = thr[1];
        {
            ProfScope ps_(ctx, PK_SWEEP_DCB_RES);
            CUDA_TRY(launch_dcb_resident(D, l->ncopies, ctx->stream));
        }
        l->t += n_rounds * k;
        return GBMC_OK;
    }
    for (uint32_t m = 0; m < n_rounds; ++m) {
        TL.t0 = l->t + m * k;
        for (uint32_t coarse = 0; coarse < 2; ++coarse) {
            TL.coarse = coarse;
            ProfScope ps_(ctx, bits ? PK_SWEEP_DCB_BITS : PK_SWEEP_DCB);
            if (bits) CUDA_TRY(launch_dcb_bits(TL, l->ncopies, ctx->stream));
            else CUDA_TRY(launch_sweep_dcb(TL, l->ncopies, ctx->stream));
        }
        if (E_series || M_series) {
            ProfScope ps_(ctx, PK_OBS);
            CUDA_TRY(launch_observables(l->cur, l->jbits, l->d.dim, (uint32_t)l->d.L, l->d.n_instances,
                                        l->d.n_replicas, E_series ? E_series + (uint64_t)m * l->ncopies : nullptr,
                                        M_series ? M_series + (uint64_t)m * l->ncopies : nullptr, ctx->stream));
        }
    }
    l->t += n_rounds * k;
    return GBMC_OK;
}

gbmc_status observables(gbmc_ctx* ctx, const gbmc_lattice* l, int32_t* E, int32_t* M) {
    if (!ctx || !l) return fail(GBMC_ERR_ARG, "NULL argument");
    if (!E && !M) return GBMC_OK;
    CUDA_TRY(cudaSetDevice(ctx->device));
    ProfScope ps_(ctx, PK_OBS);
    if (l->d.layout == GBMC_BITPACK) {
        CUDA_TRY(launch_bp_observables((const uint32_t*)l->cur, (uint32_t)l->d.L, l->ncopies, E, M, ctx->stream));
        return GBMC_OK;
    }
    CUDA_TRY(launch_observables(l->cur, l->jbits, l->d.dim, (uint32_t)l->d.L, l->d.n_instances, l->d.n_replicas, E, M,
                                ctx->stream));
    return GBMC_OK;
}

// ------------------------------------------------------------------------
// Population annealing
// ------------------------------------------------------------------------

static PaLattice pa_params(gbmc_pa* pa, PaLat& pl, uint32_t step) {
    PaLattice P;
    std::memset(&P, 0, sizeof(P));
    gbmc_lattice* l = pl.lat;
    P.E = pl.E;
    P.hist = pl.hist;
    P.emin = pl.emin;
    P.emax = pl.emax;
    P.sums = pl.sums;
    P.cloc = pl.cloc;
    P.ctot = pl.ctot;
    P.cpre = pl.cpre;
    P.counts = pl.counts;
    P.sloc = pl.sloc;
    P.ntot = pl.ntot;
    P.parent = pl.parent;
    P.stats = pa->stats + (uint64_t)step * pa->P + pl.pop0;
    P.beta = pl.betas[step];
    P.dbeta = step == 0 ? 0.0 : pl.betas[step] - pl.betas[step - 1];
    if (step > 0) {
        const uint64_t row = pl.ring ? (uint64_t)(step & 1u) : (uint64_t)(step - 1);
        P.wexp = pl.wexp + row * pl.nbins;
        P.wint = pl.wint + row * pl.nbins;
    }
    P.log_R = std::log((double)l->d.n_replicas);
    P.seed = l->d.seed;
    P.R = l->d.n_replicas;
    P.n_inst = l->d.n_instances;
    P.inst_base = l->d.instance_base;
    P.nbins = pl.nbins;
    P.nchunks = pl.nchunks;
    P.step = step;
    P.e_lo = pl.e_lo;
    P.overlap = step == 0 ? 0.0 : pl.overlap;
    P.kind = step == 0 ? 0 : pl.kind;
    if (pa->nearest) {
        const uint32_t I = l->d.n_instances;
        P.nnext = pl.nrep + (uint64_t)(step & 1u) * I;
        P.nprev = step == 0 ? nullptr : pl.nrep + (uint64_t)((step - 1) & 1u) * I;
        P.overflow = pa->ctx->words + 4;
        P.R0 = pa->R0;
        P.nearest = pa->poisson ? 2 : 1;
    }
    return P;
}

// Sweep launch over the lattices taking part in this step: theta sweeps with
// the resampling gather (step > 0), or a measurement-only pass (step 0).
static gbmc_status pa_sweep_launch(gbmc_pa* pa, bool first) {
    SweepLaunch P;
    std::memset(&P, 0, sizeof(P));
    std::vector<const gbmc_lattice*> ls;
    std::vector<PaLat*> act;
    for (auto& pl : pa->lats)
        if (pl.stepping) {
            ls.push_back(pl.lat);
            act.push_back(&pl);
        }
    if (act.empty()) return GBMC_OK;
    const std::vector<Tuning> tus = tune_batch(ls);
    const gbmc_lattice* l0 = act[0]->lat;
    P.dim = l0->d.dim;
    P.ea = l0->d.model == GBMC_EA_PMJ;
    P.swar = 1;
    for (size_t li = 0; li < act.size(); ++li) {
        PaLat& pl = *act[li];
        gbmc_lattice* l = pl.lat;
        const Tuning& tu = tus[li];
        SweepJob J = base_job(l, tu);
        if (l->d.L % 8) P.swar = 0;
        const uint32_t step = pl.steps;
        thresholds(pl.betas[step], J.thr);
        J.E = pl.E;
        J.M = pl.M;
        J.hist = pl.hist;
        J.emin = pl.emin;
        J.emax = pl.emax;
        J.sums = pl.sums;
        if (pa->nearest) J.nlive = pl.nrep + (uint64_t)(step & 1u) * l->d.n_instances;
        if (first) {
            J.nsweeps = 0;
            J.src = J.dst = l->cur;
        } else {
            J.nsweeps = pa->cfg.theta;
            J.t0 = pl.t_start + (step - 1) * pa->cfg.theta;
            J.src = l->cur;
            J.dst = (l->cur == l->spins) ? pl.alt : l->spins;
            J.parent = pl.parent;
        }
        P.jobs[P.njobs++] = J;
    }
    gbmc_status st;
    if (pa->msc) {
        uint32_t G = 4;
        for (auto* pl : act) G = std::min(G, msc_groups(pa->ctx, pl->lat));
        st = launch_msc_jobs(pa->ctx, P, G);
    } else {
        st = launch_jobs(pa->ctx, P, tus);
    }
    if (st != GBMC_OK) return st;
    if (!first) {
        for (size_t li = 0; li < act.size(); ++li) {
            gbmc_lattice* l = act[li]->lat;
            l->cur = P.jobs[li].dst;
            l->t = act[li]->t_start + act[li]->steps * pa->cfg.theta;
        }
    }
    return GBMC_OK;
}

static gbmc_status pa_record(gbmc_pa* pa) {
    for (auto& pl : pa->lats) {
        if (!pl.stepping) continue;
        PaLattice P = pa_params(pa, pl, pl.steps);
        ProfScope ps_(pa->ctx, PK_PA_RECORD);
        CUDA_TRY(launch_pa_record(P, pl.lnZ, 0.0, pa->ctx->stream));
    }
    return GBMC_OK;
}

// Step 0: random start (exact equilibrium at beta_0 = 0, Sec. 5.4 step 1)
// and its measurement.
static gbmc_status pa_begin(gbmc_pa* pa, int init) {
    cudaStream_t s = pa->ctx->stream;
    CUDA_TRY(cudaMemsetAsync(pa->stats, 0, (uint64_t)(pa->S + 1) * pa->P * sizeof(gbmc_pa_stats), s));
    for (auto& pl : pa->lats) {
        gbmc_lattice* l = pl.lat;
        if (init) {
            l->cur = l->spins;
            ProfScope ps_(pa->ctx, PK_INIT);
            CUDA_TRY(launch_init_spins(l->spins, l->d.dim, (uint32_t)l->d.L, l->d.n_instances, l->d.n_replicas,
                                       l->d.instance_base, l->d.seed, 1, s));
        }
        l->t = pl.t_start;
        pl.steps = 0;
        pl.done = false;
        pl.stepping = true;
        pl.overlap = 0.0;
        pl.kind = 0;
        pl.log.clear();
        if (pa->adaptive) pl.betas.assign(1, 0.0);
        std::vector<double> z(2 * l->d.n_instances, 0.0);
        for (uint32_t k = 0; k < l->d.n_instances; ++k) z[k] = (double)l->N * std::log(2.0);
        CUDA_TRY(cudaMemcpyAsync(pl.lnZ, z.data(), z.size() * 8, cudaMemcpyHostToDevice, s));
        CUDA_TRY(cudaStreamSynchronize(s));  // z is a host temporary
        CUDA_TRY(cudaMemsetAsync(pl.counts, 0, l->ncopies * 4, s));
        PaLattice P = pa_params(pa, pl, 0);
        ProfScope ps_(pa->ctx, PK_PA_RESET);
        CUDA_TRY(launch_pa_reset(P, s));
    }
    pa->step = 0;
    gbmc_status st = pa_sweep_launch(pa, true);
    if (st != GBMC_OK) return st;
    return pa_record(pa);
}

gbmc_status pa_create(gbmc_ctx* ctx, gbmc_lattice* const* lattices, uint32_t n_lattices, const gbmc_pa_config* cfg,
                      gbmc_pa** out) {
    if (!ctx || !lattices || !cfg || !out) return fail(GBMC_ERR_ARG, "NULL argument");
    if (n_lattices == 0 || n_lattices > (uint32_t)kMaxJobs) return fail(GBMC_ERR_ARG, "1..%d lattices per run", kMaxJobs);
    const int sched = cfg->schedule;
    if (sched != GBMC_SCHED_LINEAR && sched != GBMC_SCHED_LIST && sched != GBMC_SCHED_BISECTION &&
        sched != GBMC_SCHED_MLP)
        return fail(GBMC_ERR_ARG, "unknown schedule %d", sched);
    const bool adaptive = sched == GBMC_SCHED_BISECTION || sched == GBMC_SCHED_MLP;
    if (cfg->n_steps == 0) return fail(GBMC_ERR_ARG, "n_steps must be >= 1");
    if (cfg->theta == 0) return fail(GBMC_ERR_ARG, "theta must be >= 1");
    if (sched == GBMC_SCHED_LIST && !cfg->betas) return fail(GBMC_ERR_ARG, "betas required for a list schedule");
    if (sched == GBMC_SCHED_MLP && !cfg->mlp_params) return fail(GBMC_ERR_ARG, "mlp_params required for the MLP schedule");
    if (cfg->resample != GBMC_RESAMPLE_MULTINOMIAL && cfg->resample != GBMC_RESAMPLE_NEAREST &&
        cfg->resample != GBMC_RESAMPLE_POISSON)
        return fail(GBMC_ERR_ARG, "unknown resampling law %d", cfg->resample);
    // both variable-population laws share the live-slot machinery
    const bool nearest = cfg->resample != GBMC_RESAMPLE_MULTINOMIAL;
    if (nearest && adaptive) return fail(GBMC_ERR_ARG, "variable-population resampling needs a fixed schedule");
    if (cfg->sweep_rng != GBMC_RNG_PHILOX && cfg->sweep_rng != GBMC_RNG_MSC)
        return fail(GBMC_ERR_ARG, "unknown sweep random-number scheme %d", cfg->sweep_rng);
    const bool msc = cfg->sweep_rng == GBMC_RNG_MSC;
    if (adaptive) {
        if (!(cfg->beta_f > 0.0) || !(cfg->dbeta_max > 0.0)) return fail(GBMC_ERR_ARG, "adaptive schedules need beta_f > 0 and dbeta_max > 0");
        if (!(cfg->target_overlap > 0.0 && cfg->target_overlap < 1.0)) return fail(GBMC_ERR_ARG, "target_overlap must lie in (0, 1)");
        if (sched == GBMC_SCHED_MLP && !(cfg->overlap_lo <= cfg->overlap_hi))
            return fail(GBMC_ERR_ARG, "overlap_lo must not exceed overlap_hi");
    }
    const gbmc_lattice* l0 = lattices[0];
    if (!l0) return fail(GBMC_ERR_ARG, "NULL lattice");
    CUDA_TRY(cudaSetDevice(ctx->device));
    std::vector<const gbmc_lattice*> ls;
    for (uint32_t i = 0; i < n_lattices; ++i) {
        const gbmc_lattice* l = lattices[i];
        if (!l) return fail(GBMC_ERR_ARG, "NULL lattice");
        if (l->run) return fail(GBMC_ERR_STATE, "lattice %u already in an annealing run", i);
        if (l->d.dim != l0->d.dim || l->d.model != l0->d.model)
            return fail(GBMC_ERR_ARG, "lattices of one run share dim and model");
        if (l->d.layout != GBMC_INT8)
            return fail(GBMC_ERR_ARG, "population annealing runs on the int8 layout (lattice %u is bit-packed)", i);
        if (msc && !msc_ok(l))
            return fail(GBMC_ERR_ARG, "multi-spin-coded sweeps need 2D ferromagnets with L %% 16 == 0, L <= 208");
        if (adaptive && l->d.n_instances != 1)
            return fail(GBMC_ERR_ARG, "adaptive schedules anneal one population per lattice (n_instances = 1)");
        if (l->d.n_replicas != l0->d.n_replicas && nearest)
            return fail(GBMC_ERR_ARG, "nearest-integer resampling: every lattice has the same capacity");
        if (nearest && cfg->initial_replicas > l->d.n_replicas)
            return fail(GBMC_ERR_ARG, "initial_replicas exceeds the capacity n_replicas of lattice %u", i);
        if (!nearest && cfg->initial_replicas != 0 && cfg->initial_replicas != l->d.n_replicas)
            return fail(GBMC_ERR_ARG, "multinomial resampling keeps R = n_replicas (initial_replicas must be 0)");
        for (uint32_t k = 0; k < i; ++k)
            if (lattices[k] == l) return fail(GBMC_ERR_ARG, "lattice %u listed twice", i);
        ls.push_back(l);
    }
    {
        const std::vector<Tuning> tus = tune_batch(ls);
        for (uint32_t i = 0; i < n_lattices; ++i) {
            if (!tus[i].resident)
                return fail(GBMC_ERR_ARG, "lattice %u too large for shared-memory resident annealing", i);
            if (tus[i].threads != tus[0].threads)
                return fail(GBMC_ERR_ARG, "lattices of one run need the same CTA size");
        }
    }
    gbmc_pa* pa = new (std::nothrow) gbmc_pa;
    if (!pa) return fail(GBMC_ERR_OOM, "host allocation");
    pa->ctx = ctx;
    pa->cfg = *cfg;
    pa->cfg.betas = nullptr;
    pa->cfg.mlp_params = nullptr;
    pa->S = cfg->n_steps;
    pa->adaptive = adaptive;
    pa->nearest = nearest;
    pa->poisson = cfg->resample == GBMC_RESAMPLE_POISSON;
    pa->msc = msc;
    pa->R0 = cfg->initial_replicas ? cfg->initial_replicas : l0->d.n_replicas;
    pa->lats.resize(n_lattices);
    gbmc_status st = GBMC_OK;
    uint32_t pop = 0;
    for (uint32_t i = 0; i < n_lattices && st == GBMC_OK; ++i) {
        PaLat& pl = pa->lats[i];
        gbmc_lattice* l = lattices[i];
        pl.lat = l;
        pl.pop0 = pop;
        pop += l->d.n_instances;
        pl.t_start = l->t;
        pl.ring = adaptive;
        const uint32_t I = l->d.n_instances, R = l->d.n_replicas;
        const uint64_t C = (uint64_t)I * R;
        pl.nbins = (uint32_t)(l->d.dim * l->N / 2 + 1);
        pl.e_lo = -(int32_t)(l->d.dim * l->N);
        pl.nchunks = (R + kScanChunk - 1) / kScanChunk;
        int lg = 0;
        while ((1ull << lg) < R) ++lg;
        pl.s_bits = 63 - lg;
        if (!adaptive) {
            pl.betas.resize(pa->S + 1);
            for (uint32_t k = 0; k <= pa->S; ++k)
                pl.betas[k] = sched == GBMC_SCHED_LIST ? cfg->betas[k] : (cfg->beta_f * (double)k) / (double)pa->S;
            if (pl.betas[0] != 0.0) st = fail(GBMC_ERR_ARG, "beta_0 must be 0");
            for (uint32_t k = 1; k <= pa->S && st == GBMC_OK; ++k) {
                if (!(pl.betas[k] >= pl.betas[k - 1]) || !beta_ok(pl.betas[k], l->d.dim))
                    st = fail(GBMC_ERR_ARG, "schedule must be non-decreasing with 0 <= 4*dim*beta <= 700");
            }
        } else {
            pl.betas.assign(1, 0.0);
            if (!beta_ok(cfg->beta_f, l->d.dim)) st = fail(GBMC_ERR_ARG, "beta_f out of range");
        }
        if (st != GBMC_OK) break;
        void* p;
        if ((st = dalloc(pa, &p, C * l->N)) != GBMC_OK) break;
        pl.alt = (int8_t*)p;
        if ((st = dalloc(pa, &p, C * 4)) != GBMC_OK) break;
        pl.E = (int32_t*)p;
        if ((st = dalloc(pa, &p, C * 4)) != GBMC_OK) break;
        pl.M = (int32_t*)p;
        if ((st = dalloc(pa, &p, (uint64_t)I * pl.nbins * 4)) != GBMC_OK) break;
        pl.hist = (uint32_t*)p;
        if ((st = dalloc(pa, &p, I * 4)) != GBMC_OK) break;
        pl.emin = (int32_t*)p;
        if ((st = dalloc(pa, &p, I * 4)) != GBMC_OK) break;
        pl.emax = (int32_t*)p;
        if ((st = dalloc(pa, &p, I * 32)) != GBMC_OK) break;
        pl.sums = (unsigned long long*)p;
        if ((st = dalloc(pa, &p, I * 16)) != GBMC_OK) break;
        pl.lnZ = (double*)p;
        if ((st = dalloc(pa, &p, C * 8)) != GBMC_OK) break;
        pl.cloc = (unsigned long long*)p;
        if ((st = dalloc(pa, &p, (uint64_t)I * pl.nchunks * 8)) != GBMC_OK) break;
        pl.ctot = (unsigned long long*)p;
        if ((st = dalloc(pa, &p, (uint64_t)I * (pl.nchunks + 1) * 8)) != GBMC_OK) break;
        pl.cpre = (unsigned long long*)p;
        if ((st = dalloc(pa, &p, C * 4)) != GBMC_OK) break;
        pl.counts = (uint32_t*)p;
        if ((st = dalloc(pa, &p, C * 4)) != GBMC_OK) break;
        pl.sloc = (uint32_t*)p;
        if ((st = dalloc(pa, &p, (uint64_t)I * pl.nchunks * 4)) != GBMC_OK) break;
        pl.ntot = (uint32_t*)p;
        if ((st = dalloc(pa, &p, C * 4)) != GBMC_OK) break;
        pl.parent = (uint32_t*)p;
        if (nearest) {
            if ((st = dalloc(pa, &p, 2ull * I * 4)) != GBMC_OK) break;
            pl.nrep = (uint32_t*)p;
        }
        cudaError_t ce = cudaMemsetAsync(pl.counts, 0, C * 4, ctx->stream);
        // every slot starts with a valid parent, so a step whose resampling was
        // abandoned (timed-out barrier) still gathers in bounds
        if (ce == cudaSuccess) ce = cudaMemsetAsync(pl.parent, 0, C * 4, ctx->stream);
        if (ce != cudaSuccess) { st = fail(GBMC_ERR_CUDA, "memset: %s", cudaGetErrorString(ce)); break; }
        // fp64 weight tables (Eq. (13)), host libm exp: every step of a fixed
        // schedule now; for adaptive schedules a 2-slot ring filled per step
        const uint64_t tb = (adaptive ? 2ull : (uint64_t)pa->S) * pl.nbins;
        if ((st = dalloc(pa, &p, tb * 8)) != GBMC_OK) break;
        pl.wexp = (double*)p;
        if ((st = dalloc(pa, &p, tb * 8)) != GBMC_OK) break;
        pl.wint = (unsigned long long*)p;
        if (adaptive) {
            void* hp = nullptr;
            ce = cudaMallocHost(&hp, tb * 8);
            if (ce != cudaSuccess) { st = fail(GBMC_ERR_OOM, "cudaMallocHost: %s", cudaGetErrorString(ce)); break; }
            pa->host_allocs.push_back(hp);
            pl.hexp = (double*)hp;
            ce = cudaMallocHost(&hp, tb * 8);
            if (ce != cudaSuccess) { st = fail(GBMC_ERR_OOM, "cudaMallocHost: %s", cudaGetErrorString(ce)); break; }
            pa->host_allocs.push_back(hp);
            pl.hint = (unsigned long long*)hp;
        } else {
            std::vector<double> we(tb);
            std::vector<unsigned long long> wi(tb);
            for (uint32_t k = 1; k <= pa->S; ++k) {
                const double dbeta = pl.betas[k] - pl.betas[k - 1];
                double* row = we.data() + (uint64_t)(k - 1) * pl.nbins;
                unsigned long long* irow = wi.data() + (uint64_t)(k - 1) * pl.nbins;
                for (uint32_t b = 0; b < pl.nbins; ++b) {
                    const double w = std::exp(-(dbeta * (double)(4ll * b)));
                    row[b] = w;
                    irow[b] = (unsigned long long)std::floor(std::ldexp(w, pl.s_bits));
                }
            }
            ce = cudaMemcpy(pl.wexp, we.data(), tb * 8, cudaMemcpyHostToDevice);
            if (ce == cudaSuccess) ce = cudaMemcpy(pl.wint, wi.data(), tb * 8, cudaMemcpyHostToDevice);
            if (ce != cudaSuccess) { st = fail(GBMC_ERR_CUDA, "table upload: %s", cudaGetErrorString(ce)); break; }
        }
    }
    if (st == GBMC_OK) {
        pa->P = pop;
        void* p;
        st = dalloc(pa, &p, (uint64_t)(pa->S + 1) * pa->P * sizeof(gbmc_pa_stats));
        if (st == GBMC_OK) pa->stats = (gbmc_pa_stats*)p;
    }
    if (st == GBMC_OK && adaptive) {
        void* p;
        st = dalloc(pa, &p, kMaxJobs * sizeof(SchedOut));
        if (st == GBMC_OK) pa->sched_dev = (SchedOut*)p;
        if (st == GBMC_OK) {
            cudaError_t ce = cudaMallocHost(&p, kMaxJobs * sizeof(SchedOut));
            if (ce != cudaSuccess) st = fail(GBMC_ERR_OOM, "cudaMallocHost: %s", cudaGetErrorString(ce));
            else {
                pa->host_allocs.push_back(p);
                pa->sched_host = (SchedOut*)p;
            }
        }
        if (st == GBMC_OK && sched == GBMC_SCHED_MLP) {
            st = dalloc(pa, &p, kMlpParams * sizeof(float));
            if (st == GBMC_OK) {
                pa->mlp_dev = (float*)p;
                cudaError_t ce = cudaMemcpy(p, cfg->mlp_params, kMlpParams * sizeof(float), cudaMemcpyHostToDevice);
                if (ce != cudaSuccess) st = fail(GBMC_ERR_CUDA, "MLP upload: %s", cudaGetErrorString(ce));
            }
        }
    }
    if (st != GBMC_OK) {
        for (void* p : pa->allocs) cudaFree(p);
        for (void* p : pa->host_allocs) cudaFreeHost(p);
        delete pa;
        return st;
    }
    for (auto& pl : pa->lats) pl.lat->run = pa;
    st = pa_begin(pa, cfg->init);
    if (st != GBMC_OK) return st;
    *out = pa;
    return GBMC_OK;
}

gbmc_status pa_free(gbmc_pa* pa) {
    if (!pa) return GBMC_OK;
    cudaStreamSynchronize(pa->ctx->stream);
    for (auto& pl : pa->lats) {
        // leave the current configuration in the lattice's own buffer
        gbmc_lattice* l = pl.lat;
        if (l->cur != l->spins) {
            cudaMemcpy(l->spins, l->cur, l->N * l->ncopies, cudaMemcpyDeviceToDevice);
            l->cur = l->spins;
        }
        l->run = nullptr;
    }
    if (pa->graph) cudaGraphExecDestroy(pa->graph);
    if (pa->capture_stream) cudaStreamDestroy(pa->capture_stream);
    for (void* p : pa->allocs) cudaFree(p);
    for (void* p : pa->host_allocs) cudaFreeHost(p);
    delete pa;
    return GBMC_OK;
}

gbmc_status pa_reset(gbmc_ctx* ctx, gbmc_pa* pa, int32_t init, uint64_t seed) {
    if (!ctx || !pa) return fail(GBMC_ERR_ARG, "NULL argument");
    pa->ctx = ctx;
    CUDA_TRY(cudaSetDevice(ctx->device));
    if (seed != 0)
        for (auto& pl : pa->lats) pl.lat->d.seed = seed;
    return pa_begin(pa, init);
}

gbmc_status pa_populations(const gbmc_pa* pa, uint32_t* n) {
    if (!pa || !n) return fail(GBMC_ERR_ARG, "NULL argument");
    *n = pa->P;
    return GBMC_OK;
}

// Resampling kernels, sweeps and the record of the step for every lattice
// with `stepping` set (its next beta already appended to pl.betas).
static gbmc_status pa_enqueue_common(gbmc_pa* pa) {
    cudaStream_t s = pa->ctx->stream;
    for (auto& pl : pa->lats) {
        if (!pl.stepping) continue;
        PaLattice P = pa_params(pa, pl, pl.steps);
        if (pa->ctx->fused) {
            GridBarrier B{pa->ctx->words, pa->ctx->words + 1, pa->ctx->budget, pa->ctx->phantom};
            ProfScope ps_(pa->ctx, PK_PA_FUSED);
            CUDA_TRY(launch_pa_resample_fused(P, pl.lnZ, B, pa->ctx->sm_count, s));
            continue;
        }
        {
            ProfScope ps_(pa->ctx, PK_PA_WEIGHTS);
            CUDA_TRY(launch_pa_weights(P, s));
        }
        {
            ProfScope ps_(pa->ctx, PK_PA_REDUCE);
            CUDA_TRY(launch_pa_reduce(P, pl.lnZ, 0, s));
        }
        {
            ProfScope ps_(pa->ctx, PK_PA_DRAWS);
            if (pa->nearest) CUDA_TRY(launch_pa_nearest(P, s));
            else CUDA_TRY(launch_pa_draws(P, s));
        }
        {
            ProfScope ps_(pa->ctx, PK_PA_PLACE);
            CUDA_TRY(launch_pa_place(P, s));
        }
    }
    gbmc_status st = pa_sweep_launch(pa, false);
    if (st != GBMC_OK) return st;
    st = pa_record(pa);
    if (st != GBMC_OK) return st;
    ++pa->step;
    return GBMC_OK;
}

static gbmc_status pa_enqueue_fixed(gbmc_pa* pa) {
    for (auto& pl : pa->lats) {
        pl.stepping = true;
        ++pl.steps;
    }
    return pa_enqueue_common(pa);
}

// Smallest step an adaptive schedule takes (guards against a target overlap
// that no positive step reaches).
constexpr double kMinStep = 1e-7;

static gbmc_status pa_enqueue_adaptive(gbmc_pa* pa, const double* beta_next) {
    cudaStream_t s = pa->ctx->stream;
    std::vector<PaLat*> act;
    for (auto& pl : pa->lats) {
        pl.stepping = !pl.done;
        if (pl.stepping) act.push_back(&pl);
    }
    if (act.empty()) return fail(GBMC_ERR_STATE, "every lattice has reached beta_f");
    if (pa->step >= pa->S) return fail(GBMC_ERR_STATE, "step cap of %u reached", pa->S);
    if (!beta_next) {
        SchedLaunch S;
        std::memset(&S, 0, sizeof(S));
        for (PaLat* pl : act) {
            SchedJob& J = S.jobs[S.njobs++];
            J.hist = pl->hist;
            J.emin = pl->emin;
            J.emax = pl->emax;
            J.e_lo = pl->e_lo;
            J.nbins = pl->nbins;
            J.R = pl->lat->d.n_replicas;
            J.N = (uint32_t)pl->lat->N;
            J.L = (uint32_t)pl->lat->d.L;
            J.beta = pl->betas.back();
            const double rest = pa->cfg.beta_f - J.beta;
            J.dmax = pa->cfg.dbeta_max < rest ? pa->cfg.dbeta_max : rest;
        }
        S.out = pa->sched_dev;
        S.mlp = pa->cfg.schedule == GBMC_SCHED_MLP ? pa->mlp_dev : nullptr;
        S.target = pa->cfg.target_overlap;
        S.lo = pa->cfg.overlap_lo;
        S.hi = pa->cfg.overlap_hi;
        S.mode = pa->cfg.schedule == GBMC_SCHED_MLP ? 2 : 1;
        {
            ProfScope ps_(pa->ctx, PK_SCHEDULE);
            CUDA_TRY(launch_schedule(S, s));
        }
        CUDA_TRY(cudaMemcpyAsync(pa->sched_host, pa->sched_dev, S.njobs * sizeof(SchedOut), cudaMemcpyDeviceToHost, s));
    }
    // the staging slot written below was last read two steps ago
    CUDA_TRY(cudaStreamSynchronize(s));
    {
        gbmc_status est = check_device_error(pa->ctx);
        if (est != GBMC_OK) return est;
    }
    for (size_t j = 0; j < act.size(); ++j) {
        PaLat& pl = *act[j];
        gbmc_lattice* l = pl.lat;
        const double beta = pl.betas.back();
        gbmc_schedule_record rec;
        std::memset(&rec, 0, sizeof(rec));
        double bnew;
        uint32_t kmax = pl.nbins - 1;
        if (beta_next) {
            const size_t li = (size_t)(&pl - pa->lats.data());
            bnew = beta_next[li];
            if (!(bnew > beta) || !beta_ok(bnew, l->d.dim)) return fail(GBMC_ERR_ARG, "beta_next[%zu] must exceed the current beta", li);
            if (bnew > pa->cfg.beta_f) bnew = pa->cfg.beta_f;
            rec.kind = 0;
        } else {
            const SchedOut& o = pa->sched_host[j];
            double d = o.dbeta > kMinStep ? o.dbeta : kMinStep;
            bnew = beta + d;
            if (pa->cfg.beta_f - bnew <= 1e-12 * (pa->cfg.beta_f > 1.0 ? pa->cfg.beta_f : 1.0)) bnew = pa->cfg.beta_f;
            rec.alpha = o.alpha;
            rec.proposal = o.proposal;
            rec.alpha_proposal = o.alpha_proposal;
            rec.var = o.var;
            for (int i = 0; i < 6; ++i) rec.features[i] = o.feat[i];
            rec.kind = o.kind;
            rec.clamped = o.clamped;
            rec.evals = o.evals;
            kmax = (uint32_t)((o.emax - o.emin) >> 2);
        }
        rec.beta = bnew;
        rec.dbeta = bnew - beta;
        pl.betas.push_back(bnew);
        ++pl.steps;
        if (bnew >= pa->cfg.beta_f) pl.done = true;
        pl.overlap = rec.alpha;
        pl.kind = rec.kind;
        pl.log.push_back(rec);
        // weight tables of this step (Eq. (13)), host libm exp, into the ring
        const double dbeta = rec.dbeta;
        const uint64_t slot = (uint64_t)(pl.steps & 1u) * pl.nbins;
        for (uint32_t b = 0; b <= kmax; ++b) {
            const double w = std::exp(-(dbeta * (double)(4ll * b)));
            pl.hexp[slot + b] = w;
            pl.hint[slot + b] = (unsigned long long)std::floor(std::ldexp(w, pl.s_bits));
        }
        CUDA_TRY(cudaMemcpyAsync(pl.wexp + slot, pl.hexp + slot, (uint64_t)(kmax + 1) * 8, cudaMemcpyHostToDevice, s));
        CUDA_TRY(cudaMemcpyAsync(pl.wint + slot, pl.hint + slot, (uint64_t)(kmax + 1) * 8, cudaMemcpyHostToDevice, s));
    }
    return pa_enqueue_common(pa);
}

static bool pa_finished(const gbmc_pa* pa) {
    if (pa->adaptive) {
        if (pa->step >= pa->S) return true;
        for (auto& pl : pa->lats)
            if (!pl.done) return false;
        return true;
    }
    return pa->step >= pa->S;
}

gbmc_status pa_step(gbmc_ctx* ctx, gbmc_pa* pa, const double* beta_next, gbmc_pa_stats* out_host) {
    if (!ctx || !pa) return fail(GBMC_ERR_ARG, "NULL argument");
    if (!pa->adaptive && pa->step >= pa->S) return fail(GBMC_ERR_STATE, "schedule finished after %u steps", pa->S);
    if (beta_next && !pa->adaptive) return fail(GBMC_ERR_ARG, "explicit beta_next needs an adaptive schedule");
    pa->ctx = ctx;
    CUDA_TRY(cudaSetDevice(ctx->device));
    gbmc_status st = pa->adaptive ? pa_enqueue_adaptive(pa, beta_next) : pa_enqueue_fixed(pa);
    if (st != GBMC_OK) return st;
    if (out_host) {
        CUDA_TRY(cudaMemcpyAsync(out_host, pa->stats + (uint64_t)pa->step * pa->P, pa->P * sizeof(gbmc_pa_stats),
                                 cudaMemcpyDeviceToHost, ctx->stream));
        CUDA_TRY(cudaStreamSynchronize(ctx->stream));
        return check_device_error(ctx);
    }
    return GBMC_OK;
}

gbmc_status pa_run(gbmc_ctx* ctx, gbmc_pa* pa, gbmc_pa_stats* stats_host, uint32_t capacity, uint32_t* n_done) {
    if (!ctx || !pa) return fail(GBMC_ERR_ARG, "NULL argument");
    pa->ctx = ctx;
    CUDA_TRY(cudaSetDevice(ctx->device));
    while (!pa_finished(pa)) {
        gbmc_status st = pa->adaptive ? pa_enqueue_adaptive(pa, nullptr) : pa_enqueue_fixed(pa);
        if (st != GBMC_OK) return st;
    }
    if (stats_host) {
        const uint32_t rows = capacity < pa->step + 1 ? capacity : pa->step + 1;
        CUDA_TRY(cudaMemcpyAsync(stats_host, pa->stats, (uint64_t)rows * pa->P * sizeof(gbmc_pa_stats),
                                 cudaMemcpyDeviceToHost, ctx->stream));
    }
    CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    if (n_done) *n_done = pa->step;
    return check_device_error(ctx);
}

// What a captured run depends on besides the run's own buffers: stream, each
// lattice's seed, starting buffer and sweep counter, and the resampling mode.
static std::vector<uint64_t> graph_key(const gbmc_pa* pa) {
    std::vector<uint64_t> k{(uint64_t)(uintptr_t)pa->ctx->stream, (uint64_t)pa->ctx->fused,
                            (uint64_t)pa->ctx->launch_mode};
    for (auto& pl : pa->lats) {
        k.push_back(pl.lat->d.seed);
        k.push_back((uint64_t)(uintptr_t)pl.lat->cur);
        k.push_back(pl.t_start);
    }
    return k;
}

gbmc_status pa_run_graph(gbmc_ctx* ctx, gbmc_pa* pa, gbmc_pa_stats* stats_host, uint32_t capacity, uint32_t* n_done) {
    if (!ctx || !pa) return fail(GBMC_ERR_ARG, "NULL argument");
    if (pa->adaptive) return fail(GBMC_ERR_ARG, "graph runs need a fixed schedule (linear or list)");
    if (pa->step != 0) return fail(GBMC_ERR_STATE, "graph runs start from step 0 (call pa_reset)");
    pa->ctx = ctx;
    CUDA_TRY(cudaSetDevice(ctx->device));
    const std::vector<uint64_t> key = graph_key(pa);
    if (!pa->graph || key != pa->graph_key) {
        if (pa->graph) {
            cudaGraphExecDestroy(pa->graph);
            pa->graph = nullptr;
        }
        // capture steps 1..S exactly as pa_run would enqueue them
        std::vector<int8_t*> cur0;
        std::vector<uint32_t> t0;
        for (auto& pl : pa->lats) {
            cur0.push_back(pl.lat->cur);
            t0.push_back(pl.lat->t);
        }
        // captured on a library stream (the caller's may be the legacy default
        // stream), with one launch per resampling phase (plain kernel nodes)
        if (!pa->capture_stream) CUDA_TRY(cudaStreamCreateWithFlags(&pa->capture_stream, cudaStreamNonBlocking));
        const bool prof = ctx->prof, fused = ctx->fused;
        cudaStream_t user_stream = ctx->stream;
        ctx->prof = false;
        ctx->fused = false;
        ctx->stream = pa->capture_stream;
        cudaGraph_t g = nullptr;
        const uint64_t launches0 = g_launches.load();
        cudaError_t ce = cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal);
        gbmc_status st = GBMC_OK;
        if (ce == cudaSuccess) {
            while (st == GBMC_OK && !pa_finished(pa)) st = pa_enqueue_fixed(pa);
            ce = cudaStreamEndCapture(ctx->stream, &g);
        }
        // kernels recorded in the graph run only when it is launched: count them then
        pa->graph_kernels = g_launches.load() - launches0;
        g_launches.fetch_sub(pa->graph_kernels);
        ctx->stream = user_stream;
        ctx->prof = prof;
        ctx->fused = fused;
        pa->graph_end_cur.clear();
        pa->graph_end_t.clear();
        for (auto& pl : pa->lats) {
            pa->graph_end_cur.push_back(pl.lat->cur);
            pa->graph_end_t.push_back(pl.lat->t);
        }
        // the capture only recorded the work: put the host state back to step 0
        for (size_t i = 0; i < pa->lats.size(); ++i) {
            pa->lats[i].lat->cur = cur0[i];
            pa->lats[i].lat->t = t0[i];
            pa->lats[i].steps = 0;
        }
        pa->step = 0;
        if (st != GBMC_OK) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        if (ce != cudaSuccess) return fail(GBMC_ERR_CUDA, "stream capture: %s", cudaGetErrorString(ce));
        ce = cudaGraphInstantiate(&pa->graph, g, 0);
        cudaGraphDestroy(g);
        if (ce != cudaSuccess) {
            pa->graph = nullptr;
            return fail(GBMC_ERR_CUDA, "graph instantiation: %s", cudaGetErrorString(ce));
        }
        pa->graph_key = key;
    }
    CUDA_TRY(cudaGraphLaunch(pa->graph, ctx->stream));
    g_launches.fetch_add(pa->graph_kernels);
    for (size_t i = 0; i < pa->lats.size(); ++i) {
        pa->lats[i].lat->cur = pa->graph_end_cur[i];
        pa->lats[i].lat->t = pa->graph_end_t[i];
        pa->lats[i].steps = pa->S;
    }
    pa->step = pa->S;
    if (stats_host) {
        const uint32_t rows = capacity < pa->step + 1 ? capacity : pa->step + 1;
        CUDA_TRY(cudaMemcpyAsync(stats_host, pa->stats, (uint64_t)rows * pa->P * sizeof(gbmc_pa_stats),
                                 cudaMemcpyDeviceToHost, ctx->stream));
    }
    CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    if (n_done) *n_done = pa->step;
    return check_device_error(ctx);
}

gbmc_status pa_schedule_log(const gbmc_pa* pa, uint32_t lattice, gbmc_schedule_record* out, uint32_t capacity,
                            uint32_t* n_out) {
    if (!pa) return fail(GBMC_ERR_ARG, "NULL argument");
    if (lattice >= pa->lats.size()) return fail(GBMC_ERR_ARG, "lattice index out of range");
    const auto& log = pa->lats[lattice].log;
    const uint32_t n = (uint32_t)log.size();
    if (out)
        for (uint32_t i = 0; i < n && i < capacity; ++i) out[i] = log[i];
    if (n_out) *n_out = n;
    return GBMC_OK;
}

gbmc_status pa_betas(const gbmc_pa* pa, uint32_t lattice, double* out, uint32_t capacity, uint32_t* n_out) {
    if (!pa) return fail(GBMC_ERR_ARG, "NULL argument");
    if (lattice >= pa->lats.size()) return fail(GBMC_ERR_ARG, "lattice index out of range");
    const PaLat& pl = pa->lats[lattice];
    const uint32_t n = pa->adaptive ? (uint32_t)pl.betas.size() : pl.steps + 1;
    if (out)
        for (uint32_t i = 0; i < n && i < capacity; ++i) out[i] = pl.betas[i];
    if (n_out) *n_out = n;
    return GBMC_OK;
}

gbmc_status pa_parents_out(gbmc_ctx* ctx, const gbmc_pa* pa, uint32_t lattice, uint32_t* dst, size_t count) {
    if (!ctx || !pa || !dst) return fail(GBMC_ERR_ARG, "NULL argument");
    if (lattice >= pa->lats.size()) return fail(GBMC_ERR_ARG, "lattice index out of range");
    const PaLat& pl = pa->lats[lattice];
    if (count != pl.lat->ncopies) return fail(GBMC_ERR_ARG, "count must be %llu", (unsigned long long)pl.lat->ncopies);
    CUDA_TRY(cudaMemcpyAsync(dst, pl.parent, count * 4, cudaMemcpyDefault, ctx->stream));
    CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    return GBMC_OK;
}

gbmc_status pa_energies_out(gbmc_ctx* ctx, const gbmc_pa* pa, uint32_t lattice, int32_t* E_dst, int32_t* M_dst,
                            size_t count) {
    if (!ctx || !pa) return fail(GBMC_ERR_ARG, "NULL argument");
    if (lattice >= pa->lats.size()) return fail(GBMC_ERR_ARG, "lattice index out of range");
    const PaLat& pl = pa->lats[lattice];
    if (count != pl.lat->ncopies) return fail(GBMC_ERR_ARG, "count must be %llu", (unsigned long long)pl.lat->ncopies);
    if (E_dst) CUDA_TRY(cudaMemcpyAsync(E_dst, pl.E, count * 4, cudaMemcpyDefault, ctx->stream));
    if (M_dst) CUDA_TRY(cudaMemcpyAsync(M_dst, pl.M, count * 4, cudaMemcpyDefault, ctx->stream));
    CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    return GBMC_OK;
}

// ---- checkpoint / resume of an annealing run ----
}  // extern "C"

namespace {

constexpr uint32_t kStateMagic = 0x41504247u;  // "GBPA"
constexpr uint32_t kStateVersion = 1u;

// Plain byte serialisation of the run state (host byte order; the state is
// meant to be restored by this library on a machine of the same byte order).
struct StateOut {
    uint8_t* p;
    size_t left;
    bool ok = true;
    void put(const void* v, size_t n) {
        if (!ok || n > left) {
            ok = false;
            return;
        }
        if (n) std::memcpy(p, v, n);
        p += n;
        left -= n;
    }
    template <typename T>
    void put(const T& v) { put(&v, sizeof(T)); }
};
struct StateIn {
    const uint8_t* p;
    size_t left;
    bool ok = true;
    void get(void* v, size_t n) {
        if (!ok || n > left) {
            ok = false;
            return;
        }
        if (n) std::memcpy(v, p, n);
        p += n;
        left -= n;
    }
    template <typename T>
    T get() {
        T v{};
        get(&v, sizeof(T));
        return v;
    }
};

size_t pa_state_size(const gbmc_pa* pa) {
    size_t b = 10 * 4 + (size_t)(pa->S + 1) * pa->P * sizeof(gbmc_pa_stats);
    for (const auto& pl : pa->lats) {
        const gbmc_lattice* l = pl.lat;
        const uint64_t I = l->d.n_instances, C = l->ncopies;
        b += 5 * 4 + 8 + 5 * 4 + 8;                          // shape, seed, counters, overlap
        b += 4 + pl.betas.size() * 8 + 4 + pl.log.size() * sizeof(gbmc_schedule_record);
        b += C * 8 + I * pl.nbins * 4 + I * 8 + I * 32 + I * 16;  // E, M, hist, range, sums, ln Z
        if (pa->nearest) b += 2 * I * 4;
    }
    return b;
}

}  // namespace

extern "C" {

gbmc_status pa_state_bytes(const gbmc_pa* pa, size_t* bytes) {
    if (!pa || !bytes) return fail(GBMC_ERR_ARG, "NULL argument");
    *bytes = pa_state_size(pa);
    return GBMC_OK;
}

gbmc_status pa_state_save(gbmc_ctx* ctx, const gbmc_pa* pa, void* host, size_t bytes) {
    if (!ctx || !pa || !host) return fail(GBMC_ERR_ARG, "NULL argument");
    if (bytes != pa_state_size(pa)) return fail(GBMC_ERR_ARG, "bytes must be %zu", pa_state_size(pa));
    CUDA_TRY(cudaSetDevice(ctx->device));
    CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    StateOut o{(uint8_t*)host, bytes};
    o.put(kStateMagic);
    o.put(kStateVersion);
    o.put((uint32_t)pa->lats.size());
    o.put(pa->P);
    o.put(pa->S);
    o.put((uint32_t)pa->cfg.schedule);
    o.put((uint32_t)pa->cfg.resample);
    o.put((uint32_t)pa->cfg.sweep_rng);
    o.put(pa->cfg.theta);
    o.put(pa->step);
    const size_t sb = (size_t)(pa->S + 1) * pa->P * sizeof(gbmc_pa_stats);
    if (o.ok && sb <= o.left) CUDA_TRY(cudaMemcpy(o.p, pa->stats, sb, cudaMemcpyDeviceToHost));
    o.p += sb <= o.left ? sb : 0;
    o.left -= sb <= o.left ? sb : 0;
    for (const auto& pl : pa->lats) {
        const gbmc_lattice* l = pl.lat;
        const uint64_t I = l->d.n_instances, C = l->ncopies;
        o.put((uint32_t)l->d.dim);
        o.put((uint32_t)l->d.L);
        o.put((uint32_t)l->d.model);
        o.put(l->d.n_instances);
        o.put(l->d.n_replicas);
        o.put(l->d.seed);
        o.put(l->t);
        o.put(pl.t_start);
        o.put(pl.steps);
        o.put((uint32_t)pl.done);
        o.put((uint32_t)pl.kind);
        o.put(pl.overlap);
        o.put((uint32_t)pl.betas.size());
        o.put(pl.betas.data(), pl.betas.size() * 8);
        o.put((uint32_t)pl.log.size());
        o.put(pl.log.data(), pl.log.size() * sizeof(gbmc_schedule_record));
        struct {
            const void* d;
            size_t n;
        } arrays[] = {{pl.E, C * 4}, {pl.M, C * 4}, {pl.hist, I * pl.nbins * 4}, {pl.emin, I * 4},
                      {pl.emax, I * 4}, {pl.sums, I * 32}, {pl.lnZ, I * 16}, {pa->nearest ? pl.nrep : nullptr, 2 * I * 4}};
        for (const auto& a : arrays) {
            if (!a.d) continue;
            if (!o.ok || a.n > o.left) {
                o.ok = false;
                break;
            }
            CUDA_TRY(cudaMemcpy(o.p, a.d, a.n, cudaMemcpyDeviceToHost));
            o.p += a.n;
            o.left -= a.n;
        }
    }
    if (!o.ok || o.left != 0) return fail(GBMC_ERR_STATE, "annealing state does not fit its size");
    return GBMC_OK;
}

gbmc_status pa_state_load(gbmc_ctx* ctx, gbmc_pa* pa, const void* host, size_t bytes) {
    if (!ctx || !pa || !host) return fail(GBMC_ERR_ARG, "NULL argument");
    CUDA_TRY(cudaSetDevice(ctx->device));
    StateIn in{(const uint8_t*)host, bytes};
    if (in.get<uint32_t>() != kStateMagic || in.get<uint32_t>() != kStateVersion)
        return fail(GBMC_ERR_ARG, "not an annealing state of this library version");
    const uint32_t nl = in.get<uint32_t>(), P = in.get<uint32_t>(), S = in.get<uint32_t>();
    const uint32_t sched = in.get<uint32_t>(), law = in.get<uint32_t>(), rng = in.get<uint32_t>();
    const uint32_t theta = in.get<uint32_t>(), step = in.get<uint32_t>();
    if (!in.ok || nl != pa->lats.size() || P != pa->P || S != pa->S || sched != (uint32_t)pa->cfg.schedule ||
        law != (uint32_t)pa->cfg.resample || rng != (uint32_t)pa->cfg.sweep_rng || theta != pa->cfg.theta ||
        step > S)
        return fail(GBMC_ERR_ARG, "annealing state belongs to a run of another configuration");
    const size_t sb = (size_t)(S + 1) * P * sizeof(gbmc_pa_stats);
    if (sb > in.left) return fail(GBMC_ERR_ARG, "annealing state truncated");
    const uint8_t* stats_h = in.p;
    in.p += sb;
    in.left -= sb;
    // validate every lattice record before changing anything
    struct LatState {
        uint64_t seed;
        uint32_t t, t_start, steps, done, kind;
        double overlap;
        std::vector<double> betas;
        std::vector<gbmc_schedule_record> log;
        const uint8_t* arrays;
    };
    std::vector<LatState> ls(nl);
    for (uint32_t i = 0; i < nl; ++i) {
        const PaLat& pl = pa->lats[i];
        const gbmc_lattice* l = pl.lat;
        const uint32_t dim = in.get<uint32_t>(), L = in.get<uint32_t>(), model = in.get<uint32_t>();
        const uint32_t I = in.get<uint32_t>(), R = in.get<uint32_t>();
        if (!in.ok || dim != (uint32_t)l->d.dim || L != (uint32_t)l->d.L || model != (uint32_t)l->d.model ||
            I != l->d.n_instances || R != l->d.n_replicas)
            return fail(GBMC_ERR_ARG, "annealing state: lattice %u has another shape", i);
        LatState& st = ls[i];
        st.seed = in.get<uint64_t>();
        st.t = in.get<uint32_t>();
        st.t_start = in.get<uint32_t>();
        st.steps = in.get<uint32_t>();
        st.done = in.get<uint32_t>();
        st.kind = in.get<uint32_t>();
        st.overlap = in.get<double>();
        const uint32_t nb = in.get<uint32_t>();
        if (!in.ok || nb > in.left / 8 || nb == 0 || st.steps + 1 > nb || st.steps > S)
            return fail(GBMC_ERR_ARG, "annealing state: lattice %u has a bad temperature list", i);
        st.betas.resize(nb);
        in.get(st.betas.data(), nb * 8);
        if (!pa->adaptive && st.betas != pl.betas)
            return fail(GBMC_ERR_ARG, "annealing state: lattice %u follows another schedule", i);
        const uint32_t nlog = in.get<uint32_t>();
        if (!in.ok || nlog > in.left / sizeof(gbmc_schedule_record))
            return fail(GBMC_ERR_ARG, "annealing state truncated");
        st.log.resize(nlog);
        in.get(st.log.data(), nlog * sizeof(gbmc_schedule_record));
        const uint64_t C = l->ncopies;
        const size_t ab = C * 8 + (size_t)I * pl.nbins * 4 + (size_t)I * 56 + (pa->nearest ? 2ull * I * 4 : 0);
        if (!in.ok || ab > in.left) return fail(GBMC_ERR_ARG, "annealing state truncated");
        st.arrays = in.p;
        in.p += ab;
        in.left -= ab;
    }
    if (in.left != 0) return fail(GBMC_ERR_ARG, "annealing state has %zu trailing bytes", in.left);
    CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    pa->ctx = ctx;
    CUDA_TRY(cudaMemcpy(pa->stats, stats_h, sb, cudaMemcpyHostToDevice));
    for (uint32_t i = 0; i < nl; ++i) {
        PaLat& pl = pa->lats[i];
        gbmc_lattice* l = pl.lat;
        const LatState& st = ls[i];
        const uint64_t I = l->d.n_instances, C = l->ncopies;
        l->d.seed = st.seed;
        l->t = st.t;
        l->cur = l->spins;  // lattice_copy_in writes the saved configuration here
        pl.t_start = st.t_start;
        pl.steps = st.steps;
        pl.done = st.done != 0;
        pl.kind = (int32_t)st.kind;
        pl.overlap = st.overlap;
        pl.betas = st.betas;
        pl.log = st.log;
        pl.stepping = !pl.done;
        const uint8_t* a = st.arrays;
        struct {
            void* d;
            size_t n;
        } arrays[] = {{pl.E, C * 4}, {pl.M, C * 4}, {pl.hist, I * pl.nbins * 4}, {pl.emin, I * 4},
                      {pl.emax, I * 4}, {pl.sums, I * 32}, {pl.lnZ, I * 16}, {pa->nearest ? pl.nrep : nullptr, 2 * I * 4}};
        for (const auto& x : arrays) {
            if (!x.d) continue;
            CUDA_TRY(cudaMemcpy(x.d, a, x.n, cudaMemcpyHostToDevice));
            a += x.n;
        }
    }
    pa->step = step;
    // a captured whole-run graph no longer describes the run
    pa->graph_key.clear();
    return GBMC_OK;
}

gbmc_status gbmc_set_tuning(int32_t dim, int32_t model, int32_t L, const gbmc_tuning* shape) {
    std::lock_guard<std::mutex> g(g_shape_mu);
    const ShapeKey k{dim, model, L};
    if (!shape) {
        g_shapes.erase(k);
        return GBMC_OK;
    }
    const uint32_t tpr = shape->threads_per_copy, rpc = shape->copies_per_cta;
    if (tpr == 0 || (tpr & (tpr - 1)) || tpr > 256 || rpc == 0 || rpc > 64 || tpr * rpc > 256)
        return fail(GBMC_ERR_ARG, "threads_per_copy must be a power of two <= 256, copies_per_cta in 1..64, product <= 256");
    g_shapes[k] = Shape{tpr, rpc, shape->row_walk != 0, shape->persistent != 0, shape->kernel == GBMC_KERNEL_BITS};
    return GBMC_OK;
}

// One untimed launch, then two launches timed with CUDA events (synchronises).
static gbmc_status time_launches(gbmc_ctx* ctx, const SweepLaunch& P, const std::vector<Tuning>& tv,
                                 int persistent, cudaEvent_t e0, cudaEvent_t e1, float* ms,
                                 int kernel = GBMC_KERNEL_BYTES) {
    gbmc_status st;
    if ((st = launch_jobs(ctx, P, tv, persistent, kernel)) != GBMC_OK) return st;
    cudaEventRecord(e0, ctx->stream);
    if ((st = launch_jobs(ctx, P, tv, persistent, kernel)) != GBMC_OK) return st;
    if ((st = launch_jobs(ctx, P, tv, persistent, kernel)) != GBMC_OK) return st;
    cudaEventRecord(e1, ctx->stream);
    cudaError_t ce = cudaEventSynchronize(e1);
    if (ce == cudaSuccess) ce = cudaEventElapsedTime(ms, e0, e1);
    if (ce != cudaSuccess) return fail(GBMC_ERR_CUDA, "autotune timing: %s", cudaGetErrorString(ce));
    return GBMC_OK;
}

gbmc_status gbmc_autotune(gbmc_ctx* ctx, const gbmc_lattice* l, double beta, uint32_t n_sweeps, gbmc_tuning* out) {
    if (!ctx || !l || !out) return fail(GBMC_ERR_ARG, "NULL argument");
    if (!beta_ok(beta, l->d.dim)) return fail(GBMC_ERR_ARG, "beta out of range");
    if (n_sweeps == 0) n_sweeps = 1;
    std::memset(out, 0, sizeof(*out));
    CUDA_TRY(cudaSetDevice(ctx->device));
    if (l->d.layout != GBMC_INT8) return GBMC_OK;
    const Tuning def = tune(l, false);
    if (!def.resident) return GBMC_OK;
    // time on the first (at most 32768) copies, all instances in order, as one
    // instance (instance 0's couplings), on a scratch copy
    const uint32_t R = l->ncopies < 32768u ? (uint32_t)l->ncopies : 32768u;
    const size_t bytes = (size_t)R * l->N;
    int8_t* scratch = nullptr;
    CUDA_TRY(cudaMallocAsync((void**)&scratch, bytes, ctx->stream));
    CUDA_TRY(cudaMemcpyAsync(scratch, l->cur, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
    cudaEvent_t e0 = ctx->event(), e1 = ctx->event();
    const uint32_t W = (uint32_t)l->d.L / 8;
    const uint64_t units = units_per_copy(l);
    double best = 1e30;
    Shape best_shape{def.tpr, def.rpc, true, false, false};
    uint32_t n_cand = 0;
    gbmc_status st = GBMC_OK;
    for (uint32_t tpr = 8; tpr <= 256 && st == GBMC_OK; tpr <<= 1) {
        if (tpr > 2 * units && tpr > 32) break;
        for (uint32_t threads : {128u, 256u}) {
            if (tpr > threads) continue;
            for (int rw = 1; rw >= 0; --rw) {
                if (rw && (l->d.L % 8 != 0 || tpr % W != 0)) continue;
                const Tuning tu = make_tuning(l, tpr, threads / tpr, rw != 0);
                if (!tu.resident || tu.threads != threads) continue;
                SweepLaunch P;
                std::memset(&P, 0, sizeof(P));
                SweepJob J = base_job(l, tu);
                J.src = J.dst = scratch;
                J.R = R;
                J.n_inst = 1;
                J.ctas_per_inst = (R + tu.rpc - 1) / tu.rpc;
                J.nsweeps = n_sweeps;
                J.t0 = 0;
                thresholds(beta, J.thr);
                P.jobs[0] = J;
                P.njobs = 1;
                P.dim = l->d.dim;
                P.ea = l->d.model == GBMC_EA_PMJ;
                P.swar = (l->d.L % 8) == 0;
                std::vector<Tuning> tv{tu};
                float ms = 0.f;
                if ((st = time_launches(ctx, P, tv, 0, e0, e1, &ms)) != GBMC_OK) break;
                ++n_cand;
                if (ms < best) {
                    best = ms;
                    best_shape = Shape{tu.tpr, tu.rpc, rw != 0, false, false};
                }
            }
        }
    }
    if (st == GBMC_OK) {
        // the best grid shape again as a persistent launch
        Tuning tu = make_tuning(l, best_shape.tpr, best_shape.copies_per_cta, best_shape.rowwise, true);
        SweepLaunch P;
        std::memset(&P, 0, sizeof(P));
        SweepJob J = base_job(l, tu);
        J.src = J.dst = scratch;
        J.R = R;
        J.n_inst = 1;
        J.ctas_per_inst = (R + tu.rpc - 1) / tu.rpc;
        J.nsweeps = n_sweeps;
        J.t0 = 0;
        thresholds(beta, J.thr);
        P.jobs[0] = J;
        P.njobs = 1;
        P.dim = l->d.dim;
        P.ea = l->d.model == GBMC_EA_PMJ;
        P.swar = (l->d.L % 8) == 0;
        std::vector<Tuning> tv{tu};
        float ms = 0.f;
        st = time_launches(ctx, P, tv, 1, e0, e1, &ms);
        if (st == GBMC_OK) {
            ++n_cand;
            if (ms < best) {
                best = ms;
                best_shape.persistent = true;
            }
        }
        // the bit-sliced kernel, where it supports the lattice
        if (st == GBMC_OK && bits_supported(l->d.dim, l->d.L) && (l->d.model != GBMC_EA_PMJ || l->jb3)) {
            st = time_launches(ctx, P, tv, 0, e0, e1, &ms, GBMC_KERNEL_BITS);
            if (st == GBMC_OK) {
                ++n_cand;
                if (ms < best) {
                    best = ms;
                    best_shape.bits = true;
                }
            }
        }
    }
    ctx->pool.push_back(e0);
    ctx->pool.push_back(e1);
    cudaFreeAsync(scratch, ctx->stream);
    if (st != GBMC_OK) return st;
    {
        std::lock_guard<std::mutex> g(g_shape_mu);
        g_shapes[ShapeKey{l->d.dim, l->d.model, l->d.L}] = best_shape;
    }
    out->resident = 1;
    out->threads_per_copy = best_shape.tpr;
    out->copies_per_cta = best_shape.copies_per_cta;
    out->row_walk = best_shape.rowwise ? 1 : 0;
    out->persistent = best_shape.persistent ? 1 : 0;
    out->kernel = best_shape.bits ? GBMC_KERNEL_BITS : GBMC_KERNEL_BYTES;
    out->ms_per_sweep = best / (2.0 * n_sweeps);
    out->n_candidates = n_cand;
    return GBMC_OK;
}

// ------------------------------------------------------------------------
// Schedule MLP
// ------------------------------------------------------------------------

uint32_t gbmc_mlp_param_count(void) { return (uint32_t)kMlpParams; }

gbmc_status mlp_forward(gbmc_ctx* ctx, const float* params, const float* X, uint32_t B, float* Y) {
    if (!ctx || !params || !X || !Y) return fail(GBMC_ERR_ARG, "NULL argument");
    if (B == 0) return GBMC_OK;
    CUDA_TRY(cudaSetDevice(ctx->device));
    CUDA_TRY(launch_mlp_forward(params, X, B, Y, ctx->stream));
    return GBMC_OK;
}

gbmc_status mlp_grad(gbmc_ctx* ctx, const float* params, const float* X, const float* T, uint32_t B, float* grad,
                     float* loss) {
    if (!ctx || !params || !X || !T || !grad || !loss) return fail(GBMC_ERR_ARG, "NULL argument");
    if (B == 0 || B > kMlpMaxBatch) return fail(GBMC_ERR_ARG, "batch must be 1..%u", kMlpMaxBatch);
    CUDA_TRY(cudaSetDevice(ctx->device));
    CUDA_TRY(launch_mlp_grad(params, X, T, B, grad, loss, ctx->stream));
    return GBMC_OK;
}

gbmc_status mlp_adam(gbmc_ctx* ctx, float* params, const float* grad, float* m, float* v, uint32_t k, float lr) {
    if (!ctx || !params || !grad || !m || !v) return fail(GBMC_ERR_ARG, "NULL argument");
    if (k == 0) return fail(GBMC_ERR_ARG, "Adam step count starts at 1");
    CUDA_TRY(cudaSetDevice(ctx->device));
    CUDA_TRY(launch_mlp_adam(params, grad, m, v, k, lr, ctx->stream));
    return GBMC_OK;
}

gbmc_status mlp_train(gbmc_ctx* ctx, float* params, const float* X, const float* T, uint32_t n, uint32_t epochs,
                      uint32_t batch, float lr, float* loss_out) {
    if (!ctx || !params || !X || !T) return fail(GBMC_ERR_ARG, "NULL argument");
    if (n == 0 || epochs == 0) return GBMC_OK;
    if (batch == 0 || batch > kMlpMaxBatch) return fail(GBMC_ERR_ARG, "batch must be 1..%u", kMlpMaxBatch);
    CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t s = ctx->stream;
    float* work = nullptr;  // grad, m, v
    CUDA_TRY(cudaMallocAsync((void**)&work, 3 * kMlpParams * sizeof(float) + 16, s));
    float* g = work;
    float* m = work + kMlpParams;
    float* v = work + 2 * kMlpParams;
    gbmc_status st = GBMC_OK;
    cudaError_t e = cudaMemsetAsync(m, 0, 2 * kMlpParams * sizeof(float), s);
    uint32_t k = 0;
    const uint32_t nb = (n + batch - 1) / batch;
    for (uint32_t ep = 0; ep < epochs && e == cudaSuccess; ++ep) {
        for (uint32_t bi = 0; bi < nb && e == cudaSuccess; ++bi) {
            const uint32_t b0 = bi * batch, B = (n - b0) < batch ? (n - b0) : batch;
            float* lp = loss_out ? loss_out + (uint64_t)ep * nb + bi : work + 3 * kMlpParams;
            e = launch_mlp_grad(params, X + (uint64_t)b0 * kMlpIn, T + b0, B, g, lp, s);
            if (e == cudaSuccess) e = launch_mlp_adam(params, g, m, v, ++k, lr, s);
        }
    }
    if (e != cudaSuccess) st = fail(GBMC_ERR_CUDA, "mlp_train: %s", cudaGetErrorString(e));
    cudaFreeAsync(work, s);
    return st;
}

// ------------------------------------------------------------------------
// Parallel tempering (Sec. 5.1)
// ------------------------------------------------------------------------

struct gbmc_pt {
    gbmc_ctx* ctx;
    gbmc_lattice* lat;
    std::vector<double> betas;
    uint32_t T, M, theta, round;
    uint32_t* thr_temp = nullptr;
    uint32_t *temp_of = nullptr, *rep_of = nullptr, *accepted = nullptr;
    int32_t *E = nullptr, *Mag = nullptr;
    long long* tab = nullptr;
    std::vector<void*> allocs;
};

gbmc_status pt_create(gbmc_ctx* ctx, gbmc_lattice* l, const double* betas, uint32_t theta, gbmc_pt** out) {
    if (!ctx || !l || !betas || !out) return fail(GBMC_ERR_ARG, "NULL argument");
    if (l->run) return fail(GBMC_ERR_STATE, "lattice is used by an annealing run");
    if (l->d.layout != GBMC_INT8) return fail(GBMC_ERR_ARG, "parallel tempering runs on the int8 layout");
    const Tuning tu = tune(l);
    if (!tu.resident) return fail(GBMC_ERR_ARG, "lattice too large for shared-memory resident sweeps");
    const uint32_t T = l->d.n_replicas;
    for (uint32_t k = 0; k < T; ++k) {
        if (!beta_ok(betas[k], l->d.dim)) return fail(GBMC_ERR_ARG, "beta[%u] out of range", k);
        if (k > 0 && !(betas[k] >= betas[k - 1])) return fail(GBMC_ERR_ARG, "betas must be ascending");
    }
    CUDA_TRY(cudaSetDevice(ctx->device));
    gbmc_pt* pt = new (std::nothrow) gbmc_pt;
    if (!pt) return fail(GBMC_ERR_OOM, "host allocation");
    pt->ctx = ctx;
    pt->lat = l;
    pt->betas.assign(betas, betas + T);
    pt->T = T;
    pt->M = (uint32_t)(l->d.dim * l->N / 2);
    pt->theta = theta;
    pt->round = 0;
    const uint64_t C = l->ncopies;
    auto alloc = [&](void** p, size_t bytes) -> bool {
        if (cudaMalloc(p, bytes ? bytes : 16) != cudaSuccess) return false;
        pt->allocs.push_back(*p);
        return true;
    };
    bool ok = alloc((void**)&pt->thr_temp, 12ull * T) && alloc((void**)&pt->temp_of, 4 * C) &&
              alloc((void**)&pt->rep_of, 4 * C) && alloc((void**)&pt->accepted, 4ull * l->d.n_instances * (T > 1 ? T - 1 : 1)) &&
              alloc((void**)&pt->E, 4 * C) && alloc((void**)&pt->Mag, 4 * C) &&
              alloc((void**)&pt->tab, 8ull * (T > 1 ? T - 1 : 1) * (pt->M + 1));
    if (!ok) {
        for (void* p : pt->allocs) cudaFree(p);
        delete pt;
        return fail(GBMC_ERR_OOM, "cudaMalloc for parallel tempering");
    }
    std::vector<uint32_t> thr(3ull * T), ident(C);
    for (uint32_t k = 0; k < T; ++k) thresholds(betas[k], &thr[3ull * k]);
    for (uint64_t c = 0; c < C; ++c) ident[c] = (uint32_t)(c % T);
    std::vector<long long> tab((uint64_t)(T > 1 ? T - 1 : 1) * (pt->M + 1), 0);
    for (uint32_t k = 0; k + 1 < T; ++k) {
        const double dbeta = betas[k + 1] - betas[k];
        for (uint32_t m = 0; m <= pt->M; ++m) {
            const double p = std::exp(-(dbeta * (double)(4ll * m)));
            tab[(uint64_t)k * (pt->M + 1) + m] = (long long)std::ceil(std::ldexp(p, 32)) - 1;
        }
    }
    cudaError_t e = cudaMemcpy(pt->thr_temp, thr.data(), 12ull * T, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(pt->temp_of, ident.data(), 4 * C, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(pt->rep_of, ident.data(), 4 * C, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(pt->accepted, 0, 4ull * l->d.n_instances * (T > 1 ? T - 1 : 1));
    if (e == cudaSuccess) e = cudaMemcpy(pt->tab, tab.data(), tab.size() * 8, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        for (void* p : pt->allocs) cudaFree(p);
        delete pt;
        return fail(GBMC_ERR_CUDA, "parallel tempering set-up: %s", cudaGetErrorString(e));
    }
    l->run = (gbmc_pa*)pt;  // the lattice is owned by this run until pt_free
    *out = pt;
    return GBMC_OK;
}

gbmc_status pt_step(gbmc_ctx* ctx, gbmc_pt* pt, uint32_t n_steps) {
    if (!ctx || !pt) return fail(GBMC_ERR_ARG, "NULL argument");
    pt->ctx = ctx;
    CUDA_TRY(cudaSetDevice(ctx->device));
    gbmc_lattice* l = pt->lat;
    if ((uint64_t)l->t + (uint64_t)n_steps * pt->theta > 0xFFFFFFFFull) return fail(GBMC_ERR_ARG, "sweep counter would wrap");
    for (uint32_t n = 0; n < n_steps; ++n) {
        const Tuning tu = tune(l);
        SweepJob J = base_job(l, tu);
        J.nsweeps = pt->theta;
        J.E = pt->E;
        J.M = pt->Mag;
        J.thr_temp = pt->thr_temp;
        J.temp_of = pt->temp_of;
        SweepLaunch P;
        std::memset(&P, 0, sizeof(P));
        P.jobs[0] = J;
        P.njobs = 1;
        P.dim = l->d.dim;
        P.ea = l->d.model == GBMC_EA_PMJ;
        P.swar = (l->d.L % 8) == 0;
        gbmc_status st = launch_jobs(ctx, P, std::vector<Tuning>{tu});
        if (st != GBMC_OK) return st;
        l->t += pt->theta;
        PtExchange X;
        X.E = pt->E;
        X.rep_of = pt->rep_of;
        X.temp_of = pt->temp_of;
        X.accepted = pt->accepted;
        X.tab = pt->tab;
        X.seed = l->d.seed;
        X.T = pt->T;
        X.M = pt->M;
        X.n_inst = l->d.n_instances;
        X.inst_base = l->d.instance_base;
        X.round = pt->round++;
        ProfScope ps_(ctx, PK_PT_EXCHANGE);
        CUDA_TRY(launch_pt_exchange(X, ctx->stream));
    }
    return GBMC_OK;
}

gbmc_status pt_state_out(gbmc_ctx* ctx, const gbmc_pt* pt, uint32_t* rep_of, uint32_t* accepted, int32_t* E) {
    if (!ctx || !pt) return fail(GBMC_ERR_ARG, "NULL argument");
    CUDA_TRY(cudaSetDevice(ctx->device));
    const gbmc_lattice* l = pt->lat;
    if (rep_of) CUDA_TRY(cudaMemcpyAsync(rep_of, pt->rep_of, 4 * l->ncopies, cudaMemcpyDefault, ctx->stream));
    if (accepted)
        CUDA_TRY(cudaMemcpyAsync(accepted, pt->accepted, 4ull * l->d.n_instances * (pt->T > 1 ? pt->T - 1 : 0),
                                 cudaMemcpyDefault, ctx->stream));
    if (E) CUDA_TRY(cudaMemcpyAsync(E, pt->E, 4 * l->ncopies, cudaMemcpyDefault, ctx->stream));
    CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    return GBMC_OK;
}

gbmc_status pt_free(gbmc_pt* pt) {
    if (!pt) return GBMC_OK;
    cudaStreamSynchronize(pt->ctx->stream);
    pt->lat->run = nullptr;
    for (void* p : pt->allocs) cudaFree(p);
    delete pt;
    return GBMC_OK;
}

}  // extern "C"
