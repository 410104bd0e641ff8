// pa.cu -- population-annealing resampling (Sec. 5.4, step 2; Eq. (13)).
//
// Per population (one instance of one lattice, R replicas), from the energies
// left by the previous sweep launch and its histogram/min/max accumulators:
//   k_pa_weights : integer weight W_j = floor(2^s exp(-dbeta (E_j - Emin))) from
//                  the host-computed table; inclusive sums within 2048-replica
//                  chunks, chunk totals.
//   k_pa_reduce  : ln Q_i = -dbeta Emin + ln sum_E h(E) exp(-dbeta (E-Emin)) - ln R
//                  over the histogram (fixed-order fp64 tree), ln Z += ln Q;
//                  exclusive scan of the chunk totals -> the cumulative weights
//                  C_j = cpre[chunk] + cloc[j] in replica order; reset of the
//                  accumulators for the next sweep.
//   k_pa_draws   : R multinomial draws x_k = floor(U64_k C_R / 2^64) (Philox,
//                  purpose 2), parent = least j with C_j > x_k (two-level
//                  bisection), counts[parent] += 1 (integer atomics: the result
//                  does not depend on their order).
//   k_pa_count_scan, k_pa_place : exclusive scan of the counts; parent j fills
//                  slots [S_j, S_j + n_j): children contiguous, parents in order.
// The sweep kernel then gathers slot c from parent[c] while loading.
//
// Nearest-integer law (variable populations, P.nprev / P.nnext set): the
// draws are replaced by k_pa_nearest -- replica j gets floor(tau_j) copies
// plus one with probability frac(tau_j), tau_j = R0 W_j / C, decided in
// integers -- every phase only looks at the R_{i-1} live replicas, ln Q uses
// R_{i-1}, and the placement writes R_i (at most the capacity P.R).
#include <climits>

#include "../../include/gbmc.h"
#include "check.cuh"
#include "device.cuh"
#include "internal.h"

namespace gbmc {

constexpr int kScanThreads = 512;
constexpr int kPerThread = kScanChunk / kScanThreads;  // 4

// Replicas of population `inst` before this step's resampling: R_{i-1}.
__device__ __forceinline__ uint32_t live_prev(const PaLattice& P, uint32_t inst) {
    return P.nprev ? __ldcg(P.nprev + inst) : P.R;
}

// 64-bit uniform of resampling draw (or replica) k of population `inst`;
// r > 0: the extra pieces of a large Poisson mean.
__device__ __forceinline__ unsigned long long resample_u64(const PaLattice& P, uint32_t inst, uint32_t k,
                                                           uint32_t r = 0u) {
    const uint4 w = philox4x32_10(
        make_uint4(k >> 1, P.step, r, c3_word(kPurposeResample, 0u, P.inst_base + inst)),
        (uint32_t)P.seed, (uint32_t)(P.seed >> 32));
    return (k & 1u) ? (((unsigned long long)w.w << 32) | w.z) : (((unsigned long long)w.y << 32) | w.x);
}

// ---- the five phases, as block-level device functions ----

// Integer weights of one chunk and their inclusive sums within the chunk.
__device__ __forceinline__ void phase_weights(const PaLattice& P, uint32_t inst, uint32_t chunk,
                                              unsigned long long* sh) {
    const uint64_t base = (uint64_t)inst * P.R;
    const uint32_t live = live_prev(P, inst);
    const uint32_t j0 = chunk * kScanChunk + threadIdx.x * kPerThread;
    const int32_t emin = P.emin[inst];
    unsigned long long w[kPerThread];
    unsigned long long run = 0;
#pragma unroll
    for (int i = 0; i < kPerThread; ++i) {
        const uint32_t j = j0 + i;
        unsigned long long v = 0;
        if (j < live) v = P.wint[GBMC_IDX((uint32_t)(P.E[base + j] - emin) >> 2, P.nbins)];
        run += v;
        w[i] = run;
    }
    unsigned long long total;
    const unsigned long long incl = block_inclusive_scan<unsigned long long>(run, sh, &total);
    const unsigned long long excl = incl - run;
#pragma unroll
    for (int i = 0; i < kPerThread; ++i) {
        const uint32_t j = j0 + i;
        if (j < P.R) P.cloc[base + j] = excl + w[i];
    }
    if (threadIdx.x == 0) P.ctot[(uint64_t)inst * P.nchunks + chunk] = total;
}

// ln Q of one population (fixed-order fp64 tree), ln Z += ln Q, exclusive
// scan of its chunk totals, reset of the accumulators for the next sweep.
__device__ __forceinline__ void phase_reduce(const PaLattice& P, uint32_t inst, double* lnZ, double* lnQ_out,
                                             double* sd, unsigned long long* su) {
    const int32_t emin = P.emin[inst], emax = P.emax[inst];
    uint32_t* h = P.hist + (uint64_t)inst * P.nbins;
    double acc = 0.0;
    if (emin <= emax) {  // an empty population (variable sizes) has no range
        const uint32_t bmin = (uint32_t)(emin - P.e_lo) >> 2, bmax = (uint32_t)(emax - P.e_lo) >> 2;
        for (uint32_t b = bmin + threadIdx.x; b <= bmax; b += blockDim.x) {
            const uint32_t hb = h[b];
            if (hb) acc += (double)hb * P.wexp[GBMC_IDX(b - bmin, P.nbins)];
            h[b] = 0u;
        }
    }
    acc = warp_sum(acc);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    if (lane == 0) sd[warp] = acc;
    __syncthreads();
    if (warp == 0) {
        double v = lane < nwarps ? sd[lane] : 0.0;
        v = warp_sum(v);
        if (lane == 0) {
            const double log_R = P.nprev ? log((double)live_prev(P, inst)) : P.log_R;
            const double lnQ = -P.dbeta * (double)emin + log(v) - log_R;
            lnQ_out[inst] = lnQ;
            lnZ[inst] += lnQ;
        }
    }
    const unsigned long long* ct = P.ctot + (uint64_t)inst * P.nchunks;
    unsigned long long* cp = P.cpre + (uint64_t)inst * (P.nchunks + 1);
    unsigned long long carry = 0;
    for (uint32_t c0 = 0; c0 < P.nchunks; c0 += blockDim.x) {
        const uint32_t c = c0 + threadIdx.x;
        const unsigned long long v = c < P.nchunks ? __ldcg(ct + c) : 0ull;
        unsigned long long tot;
        const unsigned long long incl = block_inclusive_scan<unsigned long long>(v, su, &tot);
        if (c < P.nchunks) cp[c] = carry + incl - v;
        carry += tot;
    }
    if (threadIdx.x == 0) {
        cp[P.nchunks] = carry;
        P.emin[inst] = INT_MAX;
        P.emax[inst] = INT_MIN;
        unsigned long long* sums = P.sums + (uint64_t)inst * 4;
        sums[0] = sums[1] = sums[2] = sums[3] = 0ull;
    }
    __syncthreads();
}

// Multinomial draw g (global over the lattice's populations).
__device__ __forceinline__ void phase_draw(const PaLattice& P, uint64_t g) {
    const uint32_t inst = (uint32_t)(g / P.R), k = (uint32_t)(g - (uint64_t)inst * P.R);
    const unsigned long long U = resample_u64(P, inst, k);
    const unsigned long long* cp = P.cpre + (uint64_t)inst * (P.nchunks + 1);
    // data written by other CTAs earlier in a fused launch: read through L2 (__ldcg)
    const unsigned long long x = __umul64hi(U, __ldcg(cp + P.nchunks));
    // least chunk c with cp[c+1] > x
    uint32_t lo = 0, hi = P.nchunks - 1;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (__ldcg(cp + mid + 1) > x) hi = mid;
        else lo = mid + 1;
    }
    const uint32_t c = lo;
    const unsigned long long xr = x - __ldcg(cp + c);  // least j of the chunk with cloc[j] > xr
    const uint64_t base = (uint64_t)inst * P.R;
    uint32_t a = c * kScanChunk, b = min(P.R, (c + 1) * kScanChunk) - 1;
    while (a < b) {
        const uint32_t mid = (a + b) >> 1;
        if (__ldcg(P.cloc + base + mid) > xr) b = mid;
        else a = mid + 1;
    }
    atomicAdd(&P.counts[base + GBMC_IDX(a, P.R)], 1u);
}

// Nearest-integer copies of replica g (global over the lattice's populations):
// n_j = floor(R0 W_j / C) + [floor(U64_j C / 2^64) < (R0 W_j mod C)], C = sum W.
// R0 W_j <= capacity 2^s <= 2^63 and C <= R_{i-1} 2^s <= 2^63 by the choice of s.
__device__ __forceinline__ void phase_nearest(const PaLattice& P, uint64_t g) {
    const uint32_t inst = (uint32_t)(g / P.R), j = (uint32_t)(g - (uint64_t)inst * P.R);
    if (j >= live_prev(P, inst)) return;
    const uint64_t base = (uint64_t)inst * P.R;
    // W_j from the inclusive in-chunk sums (E_min was already reset by ln Q's phase)
    const unsigned long long W = __ldcg(P.cloc + base + j) - ((j % kScanChunk) ? __ldcg(P.cloc + base + j - 1) : 0ull);
    const unsigned long long C = __ldcg(P.cpre + (uint64_t)inst * (P.nchunks + 1) + P.nchunks);
    const unsigned long long num = (unsigned long long)P.R0 * W;
    const unsigned long long n0 = num / C, rem = num - n0 * C;
    const unsigned long long x = __umul64hi(resample_u64(P, inst, j), C);
    P.counts[base + j] = (uint32_t)n0 + (x < rem ? 1u : 0u);
}

// e^{-x}, x >= 0, in a fixed sequence of correctly rounded fp64 operations
// (so host and device agree bit for bit): Cody and Waite's reduction x = k ln2
// + r, |r| <= ln2/2, with ln2 = head + tail (the head's last 11 mantissa bits
// zero, so k * head is exact), e^{-r} by Horner's rule on its Taylor series to
// degree 20 (s <- 1 - (r/n) s, n = 20..1), then exact scaling by 2^-k; 0 for
// x > 700.
__device__ __forceinline__ double exp_neg_ieee(double x) {
    if (x > 700.0) return 0.0;
    const double k = floor(__dadd_rn(__ddiv_rn(x, 0.6931471805599453094172321), 0.5));
    const double r = __dsub_rn(__dsub_rn(x, __dmul_rn(k, 0.693147180559890330187045037746429443359375)),
                               __dmul_rn(k, 5.4979230187083711552420206887059365096458314e-14));
    double s = 1.0;
#pragma unroll 1
    for (int n = 20; n >= 1; --n) s = __dsub_rn(1.0, __dmul_rn(__ddiv_rn(r, (double)n), s));
    return ldexp(s, -(int)k);
}

// Poisson(tau) copies by inversion from the 64-bit uniform U: the least n with
// u < F(n), u = the top 53 bits of U as a fraction, F built term by term; a
// term that no longer changes F past the mode ends the search (tau <= 500
// here, so e^{-tau} is a normal number).
__device__ __forceinline__ uint32_t poisson_count(double tau, unsigned long long U) {
    if (tau > 700.0) return 0xFFFFFFFFu;
    const double u = __dmul_rn(__ull2double_rn(U >> 11), 1.1102230246251565404236316680908203125e-16);
    double p = exp_neg_ieee(tau), F = p;
    uint32_t n = 0;
    while (u >= F && n < 100000u) {
        n += 1;
        p = __dmul_rn(p, __ddiv_rn(tau, (double)n));
        const double Fn = __dadd_rn(F, p);
        if (Fn == F && (double)n > tau) break;
        F = Fn;
    }
    return n;
}

// Poisson copies of replica g: Poisson(tau_j), tau_j = R0 W_j / C in fp64; a
// mean above 500 as the sum of m = ceil(tau / 500) Poisson(tau / m) pieces,
// piece p from the replica's resampling word with counter field r = p.
__device__ __forceinline__ void phase_poisson(const PaLattice& P, uint64_t g) {
    const uint32_t inst = (uint32_t)(g / P.R), j = (uint32_t)(g - (uint64_t)inst * P.R);
    if (j >= live_prev(P, inst)) return;
    const uint64_t base = (uint64_t)inst * P.R;
    const unsigned long long W = __ldcg(P.cloc + base + j) - ((j % kScanChunk) ? __ldcg(P.cloc + base + j - 1) : 0ull);
    const unsigned long long C = __ldcg(P.cpre + (uint64_t)inst * (P.nchunks + 1) + P.nchunks);
    const double tau = __ddiv_rn(__ull2double_rn((unsigned long long)P.R0 * W), __ull2double_rn(C));
    uint32_t n = 0;
    if (tau <= 500.0) {
        n = poisson_count(tau, resample_u64(P, inst, j));
    } else {
        const uint32_t m = (uint32_t)ceil(__ddiv_rn(tau, 500.0));
        const double part = __ddiv_rn(tau, (double)m);
        for (uint32_t p = 0; p < m; ++p) n += poisson_count(part, resample_u64(P, inst, j, p));
    }
    P.counts[base + j] = n;
}

// Exclusive scan of the counts within one chunk, chunk total.
__device__ __forceinline__ void phase_count_scan(const PaLattice& P, uint32_t inst, uint32_t chunk, uint32_t* sh) {
    const uint64_t base = (uint64_t)inst * P.R;
    const uint32_t live = live_prev(P, inst);
    const uint32_t j0 = chunk * kScanChunk + threadIdx.x * kPerThread;
    uint32_t v[kPerThread];
    uint32_t run = 0;
#pragma unroll
    for (int i = 0; i < kPerThread; ++i) {
        const uint32_t j = j0 + i;
        v[i] = run;  // exclusive within the thread
        if (j < live) run += __ldcg(P.counts + base + j);
    }
    uint32_t total;
    const uint32_t incl = block_inclusive_scan<uint32_t>(run, sh, &total);
    const uint32_t excl = incl - run;
#pragma unroll
    for (int i = 0; i < kPerThread; ++i) {
        const uint32_t j = j0 + i;
        if (j < live) P.sloc[base + j] = excl + v[i];
    }
    if (threadIdx.x == 0) P.ntot[(uint64_t)inst * P.nchunks + chunk] = total;
}

// Parent j fills slots [S_j, S_j + n_j); counts are cleared for the next step.
// Variable populations: slots at or beyond the capacity are not written (the
// overflow flag is raised instead) and the last chunk's CTA records R_i.
__device__ __forceinline__ void phase_place(const PaLattice& P, uint32_t inst, uint32_t chunk, uint32_t* prefix) {
    const uint64_t base = (uint64_t)inst * P.R;
    const uint32_t live = live_prev(P, inst);
    if (threadIdx.x < 32) {
        uint32_t acc = 0;
        for (uint32_t c = threadIdx.x; c < chunk; c += 32) acc += __ldcg(P.ntot + (uint64_t)inst * P.nchunks + c);
        acc = warp_sum(acc);
        if (threadIdx.x == 0) *prefix = acc;
    }
    __syncthreads();
    const uint32_t pre = *prefix;
    if (P.nnext && threadIdx.x == 0 && chunk + 1 == P.nchunks) {
        uint64_t total = (uint64_t)pre + __ldcg(P.ntot + (uint64_t)inst * P.nchunks + chunk);
        if (total > P.R || total == 0) {  // outgrown its capacity, or died out
            atomicExch(P.overflow, 1u);
            if (total > P.R) total = P.R;
        }
        P.nnext[inst] = (uint32_t)total;
    }
    for (uint32_t i = threadIdx.x; i < kScanChunk; i += blockDim.x) {
        const uint32_t j = chunk * kScanChunk + i;
        if (j >= live) break;
        const uint32_t n = __ldcg(P.counts + base + j);
        if (n) {
            const uint64_t S = (uint64_t)pre + __ldcg(P.sloc + base + j);
            for (uint32_t m = 0; m < n; ++m) {
                if (S + m >= P.R) {
                    atomicExch(P.overflow, 1u);
                    break;
                }
                P.parent[base + GBMC_IDX(S + m, P.R)] = j;
            }
            P.counts[base + j] = 0u;
        }
    }
    __syncthreads();
}

// ---- separate kernels (one per phase) ----

__global__ void __launch_bounds__(kScanThreads) k_pa_weights(const __grid_constant__ PaLattice P) {
    __shared__ unsigned long long sh[32];
    phase_weights(P, blockIdx.y, blockIdx.x, sh);
}

cudaError_t launch_pa_weights(const PaLattice& P, cudaStream_t s) {
    dim3 grid(P.nchunks, P.n_inst);
    k_pa_weights<<<grid, kScanThreads, 0, s>>>(P);
    count_launch();
    return cudaGetLastError();
}

// One CTA per population.
__global__ void __launch_bounds__(1024) k_pa_reduce(const __grid_constant__ PaLattice P, double* lnZ,
                                                    double* lnQ_out) {
    __shared__ double sd[32];
    __shared__ unsigned long long su[32];
    phase_reduce(P, blockIdx.x, lnZ, lnQ_out, sd, su);
}

cudaError_t launch_pa_reduce(const PaLattice& P, double* lnZ, int /*first_step*/, cudaStream_t s) {
    // lnQ of the step is kept next to lnZ: lnZ[n_inst .. 2 n_inst)
    k_pa_reduce<<<P.n_inst, 1024, 0, s>>>(P, lnZ, lnZ + P.n_inst);
    count_launch();
    return cudaGetLastError();
}

__global__ void __launch_bounds__(256) k_pa_draws(const __grid_constant__ PaLattice P) {
    const uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (g >= (uint64_t)P.n_inst * P.R) return;
    phase_draw(P, g);
}

cudaError_t launch_pa_draws(const PaLattice& P, cudaStream_t s) {
    const uint64_t total = (uint64_t)P.n_inst * P.R;
    k_pa_draws<<<(uint32_t)((total + 255) / 256), 256, 0, s>>>(P);
    count_launch();
    return cudaGetLastError();
}

__global__ void __launch_bounds__(256) k_pa_nearest(const __grid_constant__ PaLattice P) {
    const uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (g >= (uint64_t)P.n_inst * P.R) return;
    if (P.nearest == 2) phase_poisson(P, g);
    else phase_nearest(P, g);
}

cudaError_t launch_pa_nearest(const PaLattice& P, cudaStream_t s) {
    const uint64_t total = (uint64_t)P.n_inst * P.R;
    k_pa_nearest<<<(uint32_t)((total + 255) / 256), 256, 0, s>>>(P);
    count_launch();
    return cudaGetLastError();
}

__global__ void __launch_bounds__(kScanThreads) k_pa_count_scan(const __grid_constant__ PaLattice P) {
    __shared__ uint32_t sh[32];
    phase_count_scan(P, blockIdx.y, blockIdx.x, sh);
}

__global__ void __launch_bounds__(kScanThreads) k_pa_place(const __grid_constant__ PaLattice P) {
    __shared__ uint32_t prefix;
    phase_place(P, blockIdx.y, blockIdx.x, &prefix);
}

cudaError_t launch_pa_place(const PaLattice& P, cudaStream_t s) {
    dim3 grid(P.nchunks, P.n_inst);
    k_pa_count_scan<<<grid, kScanThreads, 0, s>>>(P);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_pa_place<<<grid, kScanThreads, 0, s>>>(P);
    count_launch();
    return cudaGetLastError();
}

// ---- fused resampling: one cooperative launch, phases separated by grid barriers ----

// Grid barrier on a monotone arrival counter. Every wait is bounded: after
// `budget` cycles the waiting thread raises *err and gives up, the kernel
// returns, and the host reports GBMC_ERR_TIMEOUT at its next check; nothing
// spins forever. Returns false once *err is set.
__device__ bool grid_barrier(const GridBarrier& B, uint32_t& target) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        target += gridDim.x + B.phantom;
        __threadfence();
        atomicAdd(B.counter, 1u);
        const long long t0 = clock64();
        int ok = 1;
        while (atomicAdd(B.counter, 0u) < target) {
            if (atomicAdd(B.err, 0u) != 0u || clock64() - t0 > B.budget) {
                atomicExch(B.err, 1u);
                ok = 0;
                break;
            }
            __nanosleep(64);
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

__global__ void __launch_bounds__(kScanThreads) k_pa_resample_fused(const __grid_constant__ PaLattice P, double* lnZ,
                                                                     const __grid_constant__ GridBarrier B) {
    __shared__ unsigned long long sh64[32];
    __shared__ double sd[32];
    __shared__ uint32_t sh32[32];
    __shared__ uint32_t prefix;
    uint32_t target = 0;
    const uint32_t nch = P.n_inst * P.nchunks;
    for (uint32_t c = blockIdx.x; c < nch; c += gridDim.x) phase_weights(P, c / P.nchunks, c % P.nchunks, sh64);
    if (!grid_barrier(B, target)) return;
    for (uint32_t inst = blockIdx.x; inst < P.n_inst; inst += gridDim.x)
        phase_reduce(P, inst, lnZ, lnZ + P.n_inst, sd, sh64);
    if (!grid_barrier(B, target)) return;
    const uint64_t total = (uint64_t)P.n_inst * P.R;
    for (uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; g < total; g += (uint64_t)gridDim.x * blockDim.x) {
        if (P.nearest == 2) phase_poisson(P, g);
        else if (P.nearest) phase_nearest(P, g);
        else phase_draw(P, g);
    }
    if (!grid_barrier(B, target)) return;
    for (uint32_t c = blockIdx.x; c < nch; c += gridDim.x) phase_count_scan(P, c / P.nchunks, c % P.nchunks, sh32);
    if (!grid_barrier(B, target)) return;
    for (uint32_t c = blockIdx.x; c < nch; c += gridDim.x) phase_place(P, c / P.nchunks, c % P.nchunks, &prefix);
}

cudaError_t launch_pa_resample_fused(const PaLattice& P, double* lnZ, const GridBarrier& B, int n_sms,
                                     cudaStream_t s) {
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pa_resample_fused, kScanThreads, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const uint64_t work = (uint64_t)P.n_inst * P.nchunks;
    uint64_t grid = (uint64_t)n_sms * (uint64_t)per_sm;
    if (grid > work * 4) grid = work * 4;  // draws use more CTAs than chunks
    if (grid < 1) grid = 1;
    e = cudaMemsetAsync(B.counter, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    PaLattice Pc = P;
    double* lz = lnZ;
    GridBarrier Bc = B;
    void* args[] = {&Pc, &lz, &Bc};
    e = cudaLaunchCooperativeKernel((const void*)k_pa_resample_fused, dim3((uint32_t)grid), dim3(kScanThreads), args,
                                    0, s);
    count_launch();
    return e;
}

// Record of one step for every population of a lattice, after its sweeps.
__global__ void k_pa_record(const __grid_constant__ PaLattice P, const double* lnZ) {
    const uint32_t inst = blockIdx.x * blockDim.x + threadIdx.x;
    if (inst >= P.n_inst) return;
    gbmc_pa_stats* st = reinterpret_cast<gbmc_pa_stats*>(P.stats) + inst;
    const unsigned long long* su = P.sums + (uint64_t)inst * 4;
    st->beta = P.beta;
    st->dbeta = P.dbeta;
    st->lnQ = P.step == 0 ? 0.0 : lnZ[P.n_inst + inst];
    st->lnZ = lnZ[inst];
    st->sumE = (int64_t)su[0];
    st->sumE2 = (int64_t)su[1];
    st->sumAbsM = (int64_t)su[2];
    st->sumM2 = (int64_t)su[3];
    st->Emin = P.emin[inst];
    st->Emax = P.emax[inst];
    st->step = P.step;
    st->n_replicas = P.nnext ? P.nnext[inst] : P.R;
    st->overlap = P.overlap;
    st->proposal_kind = P.kind;
    st->pad = 0;
}

cudaError_t launch_pa_record(const PaLattice& P, const double* lnZ, double, cudaStream_t s) {
    k_pa_record<<<(P.n_inst + 127) / 128, 128, 0, s>>>(P, lnZ);
    count_launch();
    return cudaGetLastError();
}

// Reset of the accumulators before the first measurement (step 0).
__global__ void k_pa_reset(const __grid_constant__ PaLattice P) {
    const uint32_t inst = blockIdx.x;
    uint32_t* h = P.hist + (uint64_t)inst * P.nbins;
    for (uint32_t b = threadIdx.x; b < P.nbins; b += blockDim.x) h[b] = 0u;
    if (threadIdx.x == 0) {
        P.emin[inst] = INT_MAX;
        P.emax[inst] = INT_MIN;
        unsigned long long* sums = P.sums + (uint64_t)inst * 4;
        sums[0] = sums[1] = sums[2] = sums[3] = 0ull;
        if (P.nnext) P.nnext[inst] = P.R0;  // R_0
    }
}

cudaError_t launch_pa_reset(const PaLattice& P, cudaStream_t s) {
    k_pa_reset<<<P.n_inst, 256, 0, s>>>(P);
    count_launch();
    return cudaGetLastError();
}

}  // namespace gbmc
