// static_resample.cu -- pa_resample_static: the population-annealing
// resampling step for callers that cannot allocate device memory.
//
// Some callers must not call cudaMalloc: processes whose device memory belongs
// to another allocator (a framework's memory pool that has reserved the
// device and must not be bypassed or fragmented), embedded or real-time
// drivers that reserve all memory at start-up and forbid allocation later,
// and code on a latency-critical path where the implicit device-wide
// synchronisation of cudaMalloc / cudaFree would stall other streams. This
// entry point gives them the same resampling as pa_step (same kernels, same
// results) using a fixed scratch area that is part of the library image: a
// file-scope __device__ array of kStaticScratchBytes, which every GPU that
// loads the library holds until the process exits. The caller passes the
// energies in and receives the parent map and ln Q.
#include <cuda.h>

#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/gbmc.h"
#include "device.cuh"
#include "internal.h"

namespace gbmc {

namespace {

constexpr uint64_t kStaticMaxCopies = 1ull << 17;     // instances x replicas per call
constexpr uint64_t kStaticMaxInstances = 1024;
constexpr uint64_t kStaticMaxBins = 65537;            // dim * N / 2 + 1
constexpr uint64_t kStaticMaxHist = 1ull << 19;       // instances x bins

// Byte offsets of the regions inside the static array (each 256-aligned).
constexpr uint64_t align256(uint64_t x) { return (x + 255) & ~255ull; }
constexpr uint64_t kOffHist = 0;
constexpr uint64_t kOffEmin = align256(kOffHist + 4 * kStaticMaxHist);
constexpr uint64_t kOffEmax = align256(kOffEmin + 4 * kStaticMaxInstances);
constexpr uint64_t kOffSums = align256(kOffEmax + 4 * kStaticMaxInstances);
constexpr uint64_t kOffLnZ = align256(kOffSums + 32 * kStaticMaxInstances);
constexpr uint64_t kOffCloc = align256(kOffLnZ + 16 * kStaticMaxInstances);
constexpr uint64_t kOffCtot = align256(kOffCloc + 8 * kStaticMaxCopies);
constexpr uint64_t kOffCpre = align256(kOffCtot + 8 * kStaticMaxCopies);
constexpr uint64_t kOffCounts = align256(kOffCpre + 8 * (kStaticMaxCopies + kStaticMaxInstances));
constexpr uint64_t kOffSloc = align256(kOffCounts + 4 * kStaticMaxCopies);
constexpr uint64_t kOffNtot = align256(kOffSloc + 4 * kStaticMaxCopies);
constexpr uint64_t kOffWexp = align256(kOffNtot + 4 * kStaticMaxCopies);
constexpr uint64_t kOffWint = align256(kOffWexp + 8 * kStaticMaxBins);
constexpr uint64_t kOffE = align256(kOffWint + 8 * kStaticMaxBins);
constexpr uint64_t kStaticScratchBytes = align256(kOffE + 4 * kStaticMaxCopies);

}  // namespace

// The scratch area (8,454,656 bytes, about 8.1 MiB). Every call shares it and it keeps the
// last call's contents; each call clears what must start at zero.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Histogram and range of the given energies (the accumulators the sweep
// kernel fills in pa_step), taken on a copy clamped to the lattice's energy
// range [e_lo, -e_lo] so that caller-supplied values can never index outside
// the tables (valid energies are unchanged).
__global__ void k_static_stats(const int32_t* E, int32_t* Ecopy, uint64_t total, uint32_t R, int32_t e_lo,
                               uint32_t nbins, uint32_t* hist, int32_t* emin, int32_t* emax) {
    for (uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; g < total;
         g += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t inst = (uint32_t)(g / R);
        const int32_t e = min(max(E[g], e_lo), -e_lo);
        Ecopy[g] = e;
        atomicAdd(&hist[(uint64_t)inst * nbins + (uint32_t)((e - e_lo) >> 2)], 1u);
        atomicMin(&emin[inst], e);
        atomicMax(&emax[inst], e);
    }
}

}  // namespace gbmc

using namespace gbmc;

namespace {

gbmc_status static_fail(gbmc_status st, const char* msg, cudaError_t e = cudaSuccess) {
    char buf[256];
    if (e != cudaSuccess)
        snprintf(buf, sizeof(buf), "pa_resample_static: %s: %s", msg, cudaGetErrorString(e));
    else
        snprintf(buf, sizeof(buf), "pa_resample_static: %s", msg);
    set_last_error(buf);
    return st;
}

// Device address of the scratch array and the SM count, looked up with the
// device current (in host code the array's name is only a host-side handle,
// not a device address). The address belongs to the device's current context:
// it is cached together with that context's id (unique for the life of the
// process) and looked up again when the id changes, e.g. after the primary
// context was reset and the library's module was loaded anew.
constexpr int kMaxDevices = 64;
std::mutex g_addr_mu;
struct DevScratch {
    unsigned long long ctx_id;
    void* addr;
    int sms;
};
DevScratch g_dev[kMaxDevices] = {};

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

// Id of the calling thread's current context, through the driver entry points
// the runtime hands out (no link-time dependence on the driver library).
cudaError_t current_ctx_id(unsigned long long* id) {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static cudaError_t status = cudaErrorUnknown;
    static std::once_flag once;
    std::call_once(once, [] {
        cudaDriverEntryPointQueryResult q1, q2;
        void *f1 = nullptr, *f2 = nullptr;
        status = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1);
        if (status == cudaSuccess)
            status = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2);
        if (status == cudaSuccess && (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess))
            status = cudaErrorSymbolNotFound;
        get_current = (CtxGetCurrentFn)f1;
        get_id = (CtxGetIdFn)f2;
    });
    if (status != cudaSuccess) return status;
    CUcontext c = nullptr;
    if (get_current(&c) != CUDA_SUCCESS || c == nullptr || get_id(c, id) != CUDA_SUCCESS) return cudaErrorDeviceUninitialized;
    return cudaSuccess;
}

// Host staging of the weight tables (copied to the device before returning).
double g_host_wexp[kStaticMaxBins];
unsigned long long g_host_wint[kStaticMaxBins];
std::mutex g_host_mu;

}  // namespace

extern "C" gbmc_status pa_resample_static(void* cuda_stream, int32_t device, int32_t dim, int64_t n_sites,
                                          uint32_t n_instances, uint32_t n_replicas, uint32_t instance_base,
                                          uint64_t seed, uint32_t step, double dbeta, const int32_t* E_dev,
                                          uint32_t* parent_dev, double* lnQ_dev) {
    if (!E_dev || !parent_dev || !lnQ_dev) return static_fail(GBMC_ERR_ARG, "NULL buffer");
    if (dim != 2 && dim != 3) return static_fail(GBMC_ERR_ARG, "dim must be 2 or 3");
    if (device < 0 || device >= kMaxDevices) return static_fail(GBMC_ERR_ARG, "device out of range");
    if (n_instances == 0 || n_replicas == 0 || n_sites < 4) return static_fail(GBMC_ERR_ARG, "empty population");
    if (!(std::isfinite(dbeta) && dbeta >= 0.0)) return static_fail(GBMC_ERR_ARG, "dbeta must be finite and >= 0");
    const uint64_t total = (uint64_t)n_instances * n_replicas;
    const uint64_t nbins = (uint64_t)dim * (uint64_t)n_sites / 2 + 1;
    if (total > kStaticMaxCopies)
        return static_fail(GBMC_ERR_ARG, "n_instances * n_replicas exceeds the static limit of 131072");
    if (n_instances > kStaticMaxInstances) return static_fail(GBMC_ERR_ARG, "n_instances exceeds 1024");
    if (nbins > kStaticMaxBins) return static_fail(GBMC_ERR_ARG, "dim * n_sites / 2 + 1 exceeds 65537 energy bins");
    if ((uint64_t)n_instances * nbins > kStaticMaxHist)
        return static_fail(GBMC_ERR_ARG, "n_instances * energy bins exceeds 524288");
    if ((uint64_t)instance_base + n_instances > (1ull << 27)) return static_fail(GBMC_ERR_ARG, "instance ids exceed 2^27");

    cudaStream_t s = (cudaStream_t)cuda_stream;
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return static_fail(GBMC_ERR_CUDA, "cudaSetDevice", e);
    unsigned char* base = nullptr;
    int sms = 0;
    {
        std::lock_guard<std::mutex> g(g_addr_mu);
        unsigned long long id = 0;
        if ((e = current_ctx_id(&id)) != cudaSuccess) return static_fail(GBMC_ERR_CUDA, "current context", e);
        DevScratch& d = g_dev[device];
        if (!d.addr || d.ctx_id != id) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_static_scratch);
            if (e != cudaSuccess) return static_fail(GBMC_ERR_CUDA, "cudaGetSymbolAddress", e);
            int n = 0;
            e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, device);
            if (e != cudaSuccess) return static_fail(GBMC_ERR_CUDA, "SM count", e);
            d.addr = p;
            d.sms = n > 0 ? n : 1;
            d.ctx_id = id;
        }
        base = (unsigned char*)d.addr;
        sms = d.sms;
    }

    PaLattice P;
    std::memset(&P, 0, sizeof(P));
    const uint32_t nchunks = (n_replicas + kScanChunk - 1) / kScanChunk;
    double* lnZ = (double*)(base + kOffLnZ);
    P.E = (const int32_t*)(base + kOffE);
    P.hist = (uint32_t*)(base + kOffHist);
    P.emin = (int32_t*)(base + kOffEmin);
    P.emax = (int32_t*)(base + kOffEmax);
    P.sums = (unsigned long long*)(base + kOffSums);
    P.cloc = (unsigned long long*)(base + kOffCloc);
    P.ctot = (unsigned long long*)(base + kOffCtot);
    P.cpre = (unsigned long long*)(base + kOffCpre);
    P.counts = (uint32_t*)(base + kOffCounts);
    P.sloc = (uint32_t*)(base + kOffSloc);
    P.ntot = (uint32_t*)(base + kOffNtot);
    P.parent = parent_dev;
    P.wexp = (const double*)(base + kOffWexp);
    P.wint = (const unsigned long long*)(base + kOffWint);
    P.dbeta = dbeta;
    P.log_R = std::log((double)n_replicas);
    P.seed = seed;
    P.R = n_replicas;
    P.n_inst = n_instances;
    P.inst_base = instance_base;
    P.nbins = (uint32_t)nbins;
    P.nchunks = nchunks;
    P.step = step;
    P.e_lo = -(int32_t)(dim * n_sites);

    // weight tables W(k) = exp(-dbeta 4k), floor(2^s W), s = 63 - ceil(log2 R)
    int lg = 0;
    while ((1ull << lg) < n_replicas) ++lg;
    const int s_bits = 63 - lg;
    {
        std::lock_guard<std::mutex> g(g_host_mu);
        for (uint64_t b = 0; b < nbins; ++b) {
            const double w = std::exp(-(dbeta * (double)(4ll * (long long)b)));
            g_host_wexp[b] = w;
            g_host_wint[b] = (unsigned long long)std::floor(std::ldexp(w, s_bits));
        }
        // pageable source: the copy has taken the host arrays when the call returns
        e = cudaMemcpyAsync(base + kOffWexp, g_host_wexp, 8 * nbins, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(base + kOffWint, g_host_wint, 8 * nbins, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return static_fail(GBMC_ERR_CUDA, "table upload", e);
    }
    // clear what must start at zero: counts, ln Z slots; hist/min/max/sums by k_pa_reset
    e = cudaMemsetAsync(P.counts, 0, 4 * total, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(lnZ, 0, 16 * n_instances, s);
    if (e != cudaSuccess) return static_fail(GBMC_ERR_CUDA, "scratch clear", e);
    if ((e = launch_pa_reset(P, s)) != cudaSuccess) return static_fail(GBMC_ERR_CUDA, "reset", e);
    {
        uint64_t blocks = (total + 255) / 256;
        if (blocks > 16ull * (uint64_t)sms) blocks = 16ull * (uint64_t)sms;
        k_static_stats<<<(uint32_t)blocks, 256, 0, s>>>(E_dev, (int32_t*)(base + kOffE), total, n_replicas, P.e_lo,
                                                        P.nbins, P.hist, P.emin, P.emax);
        count_launch();
        if ((e = cudaGetLastError()) != cudaSuccess) return static_fail(GBMC_ERR_CUDA, "stats", e);
    }
    if ((e = launch_pa_weights(P, s)) != cudaSuccess) return static_fail(GBMC_ERR_CUDA, "weights", e);
    if ((e = launch_pa_reduce(P, lnZ, 0, s)) != cudaSuccess) return static_fail(GBMC_ERR_CUDA, "reduce", e);
    if ((e = launch_pa_draws(P, s)) != cudaSuccess) return static_fail(GBMC_ERR_CUDA, "draws", e);
    if ((e = launch_pa_place(P, s)) != cudaSuccess) return static_fail(GBMC_ERR_CUDA, "place", e);
    // ln Q of every instance sits after the n_instances ln Z slots
    e = cudaMemcpyAsync(lnQ_dev, lnZ + n_instances, 8 * n_instances, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return static_fail(GBMC_ERR_CUDA, "lnQ copy", e);
    return GBMC_OK;
}
