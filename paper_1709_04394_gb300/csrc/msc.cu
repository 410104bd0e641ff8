// msc.cu -- checkerboard Metropolis sweeps with multi-spin coding across
// replicas (Sec. 5.4: 32 copies coded in one word, their random numbers from a
// cheap linear congruential generator re-seeded by Philox).
//
// A CTA takes G groups of 32 consecutive replica slots of one (lattice,
// instance). On load it gathers each replica through the resampling parent
// map (population annealing) from the int8 layout and transposes it into
// shared memory, one 32-bit word per site and group (bit b = replica
// 32 w + b, 1 = spin down), with warp ballots. A site update then serves all
// 32 replicas at once: the neighbour words give, bit-parallel, the masks of
// replicas with a >= 2, a = 1 and a = 0 unsatisfied bonds (dE = 8 - 4a in the
// 2D ferromagnet); a >= 2 always flips, a = 1 flips iff u_b <= T(4), a = 0 iff
// u_b <= T(8). The uniforms u_b: the Philox word of (q = k >> 2, sweep t,
// group w, purpose 5 | colour | instance), word k & 3 (k = the site's rank
// among its colour, as in the per-site path), seeds the LCG x -> 1664525 x +
// 1013904223 mod 2^32, and u_b is its (b + 1)-th output. After the last sweep
// the words are transposed back (lane b = replica b), which also yields each
// replica's count of down spins and unsatisfied bonds, hence E and M.
// Site i of a group is stored at word i + i / 8: threads update sites 8 words
// apart, which the padding spreads over all 32 banks.
#include <climits>

#include "bits.cuh"
#include "device.cuh"
#include "internal.h"

namespace gbmc {

constexpr uint32_t kPurposeMsc = 5u;
constexpr uint32_t kLcgA = 1664525u, kLcgC = 1013904223u;
constexpr uint32_t kMscThreads = 256;

__device__ __forceinline__ uint32_t pad(uint32_t i) { return i + (i >> 3); }

__host__ __device__ __forceinline__ uint32_t padded_words(uint32_t N) { return N + (N >> 3); }

// 3 CTAs per SM: the register cap (80) measured faster than the 100 registers
// the compiler picks unbounded (2 CTAs per SM).
__global__ void __launch_bounds__(kMscThreads, 3) k_sweep_msc(const __grid_constant__ SweepLaunch P, uint32_t G) {
    extern __shared__ __align__(16) uint32_t wsm[];  // [G][N + N/8]
    __shared__ int cntD[4 * 32], cntU[4 * 32];
    int jid = 0;
    while (jid + 1 < P.njobs && blockIdx.x >= P.cta_begin[jid + 1]) ++jid;
    const SweepJob& J = P.jobs[jid];
    const uint32_t local = blockIdx.x - P.cta_begin[jid];
    const uint32_t inst = local / J.ctas_per_inst;
    const uint32_t r0 = (local - inst * J.ctas_per_inst) * J.rpc;  // rpc = 32 G
    const uint32_t live = J.nlive ? J.nlive[inst] : J.R;
    if (r0 >= live) return;  // uniform over the CTA, before any barrier
    const uint32_t L = J.L, N = J.N, lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint32_t nwarps = kMscThreads / 32;
    const uint64_t slot0 = (uint64_t)inst * J.R + r0;
    const uint32_t chunks = N >> 4;  // 16 sites per chunk
    const uint32_t NW = padded_words(N);

    // ---- load: gather + transpose (lane b = replica r0 + 32 g + b) ----
    for (uint32_t gc = warp; gc < G * chunks; gc += nwarps) {
        const uint32_t g = gc / chunks, ch = gc - g * chunks;
        const uint32_t r = r0 + 32 * g + lane;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (r < live) {
            const uint64_t slot = slot0 + 32 * g + lane;
            const uint64_t src = J.parent ? (uint64_t)inst * J.R + J.parent[slot] : slot;
            v = *reinterpret_cast<const uint4*>(J.src + src * N + 16ull * ch);
        }
        uint32_t mine = 0;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const uint32_t w = j < 4 ? v.x : j < 8 ? v.y : j < 12 ? v.z : v.w;
            const uint32_t word = __ballot_sync(0xffffffffu, (w >> (8 * (j & 3) + 7)) & 1u);
            if (lane == (uint32_t)j) mine = word;
        }
        if (lane < 16) wsm[(uint64_t)g * NW + pad(16 * ch + lane)] = mine;
    }
    for (uint32_t i = threadIdx.x; i < 32 * G; i += kMscThreads) {
        cntD[i] = 0;
        cntU[i] = 0;
    }
    __syncthreads();

    // ---- sweeps ----
    const uint32_t k0 = (uint32_t)J.seed, k1 = (uint32_t)(J.seed >> 32);
    const uint32_t T4 = J.thr[0], T8 = J.thr[1];
    const uint32_t instance = J.inst_base + inst, half = L >> 1, quads = N >> 3;
    for (uint32_t s = 0; s < J.nsweeps; ++s) {
        const uint32_t t = J.t0 + s;
        for (uint32_t colour = 0; colour < 2; ++colour) {
            const uint32_t c3 = c3_word(kPurposeMsc, colour, instance);
            for (uint32_t u = threadIdx.x; u < G * quads; u += kMscThreads) {
                const uint32_t g = u / quads, quad = u - g * quads;
                const uint32_t w_group = (r0 >> 5) + g;
                const uint4 seeds = philox4x32_10(make_uint4(quad, t, w_group, c3), k0, k1);
                uint32_t* W = wsm + (uint64_t)g * NW;
                const uint32_t k = 4 * quad, y = k / half, j0 = k - y * half;
                const uint32_t off = (y + colour) & 1u;
                const uint32_t ru = (y == 0 ? L - 1 : y - 1) * L, rd = (y + 1 == L ? 0 : y + 1) * L, rw = y * L;
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    const uint32_t x = 2 * (j0 + m) + off;
                    const uint32_t xl = x == 0 ? L - 1 : x - 1, xr = x + 1 == L ? 0 : x + 1;
                    const uint32_t sv = W[pad(rw + x)];
                    const uint32_t x1 = sv ^ W[pad(rw + xl)], x2 = sv ^ W[pad(rw + xr)];
                    const uint32_t x3 = sv ^ W[pad(ru + x)], x4 = sv ^ W[pad(rd + x)];
                    const uint32_t o12 = x1 ^ x2, o34 = x3 ^ x4;
                    const uint32_t ge2 = (x1 & x2) | (x3 & x4) | (o12 & o34);  // a >= 2: dE <= 0
                    const uint32_t any = x1 | x2 | x3 | x4;
                    const uint32_t a1 = any & ~ge2;                              // a = 1: dE = 4
                    const uint32_t a0 = ~any;                                    // a = 0: dE = 8
                    uint32_t xs = m == 0 ? seeds.x : m == 1 ? seeds.y : m == 2 ? seeds.z : seeds.w;
                    uint32_t r4 = 0, r8 = 0;
#pragma unroll
                    for (int b = 0; b < 32; ++b) {
                        xs = kLcgA * xs + kLcgC;
                        accept_bits(r4, r8, T4, T8, xs);
                    }
                    // replica b's bits were shifted in first-to-last: bit 31 - b
                    W[pad(rw + x)] = sv ^ (ge2 | (a1 & __brev(r4)) | (a0 & __brev(r8)));
                }
            }
            __syncthreads();
        }
    }

    // ---- store + measure: transpose back (lane b = replica r0 + 32 g + b) ----
    const bool store = J.nsweeps > 0 || J.dst != J.src || J.parent;
    const bool want = J.E || J.M || J.hist;
    const uint32_t cpr = L >> 4;  // chunks per row
    for (uint32_t gc = warp; gc < G * chunks; gc += nwarps) {
        const uint32_t g = gc / chunks, ch = gc - g * chunks;
        const uint32_t y = ch / cpr, x0 = (ch - y * cpr) << 4;
        const uint32_t* W = wsm + (uint64_t)g * NW;
        const uint32_t rw = y * L, rd = (y + 1 == L ? 0 : y + 1) * L;
        const uint32_t xn = x0 + 16 == L ? 0 : x0 + 16;
        uint32_t p = 0, pd = 0;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            p |= ((W[pad(rw + x0 + j)] >> lane) & 1u) << j;
            pd |= ((W[pad(rd + x0 + j)] >> lane) & 1u) << j;
        }
        const uint32_t pr = (p >> 1) | (((W[pad(rw + xn)] >> lane) & 1u) << 15);
        const uint32_t r = r0 + 32 * g + lane;
        if (r < live) {
            if (want) {
                atomicAdd(&cntD[32 * g + lane], __popc(p));
                atomicAdd(&cntU[32 * g + lane], __popc(p ^ pr) + __popc(p ^ pd));
            }
            if (store) {
                uint4 v;
                uint32_t* vw = reinterpret_cast<uint32_t*>(&v);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const uint32_t nib = (p >> (4 * q)) & 0xFu;
                    const uint32_t spread = (nib * 0x00204081u) & 0x01010101u;  // bit i -> byte i
                    vw[q] = 0x01010101u + 0xFEu * spread;                      // +1 -> 0x01, -1 -> 0xFF
                }
                *reinterpret_cast<uint4*>(J.dst + (slot0 + 32 * g + lane) * N + rw + x0) = v;
            }
        }
    }
    if (!want) return;
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < 32 * G; i += kMscThreads) {
        const uint32_t r = r0 + i;
        if (r >= live) continue;
        const uint64_t slot = slot0 + i;
        const int E = 2 * cntU[i] - 2 * (int)N;  // 2N bonds: satisfied - unsatisfied, negated
        const int M = (int)N - 2 * cntD[i];
        if (J.E) J.E[slot] = E;
        if (J.M) J.M[slot] = M;
        if (J.hist) {
            atomicAdd(&J.hist[(uint64_t)inst * J.nbins + (uint32_t)((E - J.e_lo) >> 2)], 1u);
            atomicMin(&J.emin[inst], E);
            atomicMax(&J.emax[inst], E);
            unsigned long long* su = J.sums + (uint64_t)inst * 4;
            const long long el = E, ml = M;
            atomicAdd(&su[0], (unsigned long long)el);
            atomicAdd(&su[1], (unsigned long long)(el * el));
            atomicAdd(&su[2], (unsigned long long)(ml < 0 ? -ml : ml));
            atomicAdd(&su[3], (unsigned long long)(ml * ml));
        }
    }
}

size_t msc_smem_bytes(uint32_t N, uint32_t G) { return (size_t)G * padded_words(N) * 4; }

// Groups of 32 per CTA for `groups` groups of N-site copies in one launch:
// among G = 1..4 whose shared memory fits, the one whose last wave of CTAs is
// fullest (ties: more groups per CTA).
uint32_t msc_pick_groups(uint32_t N, uint64_t groups, int sms) {
    uint32_t best = 1;
    double best_eff = -1.0;
    for (uint32_t G = 1; G <= 4; ++G) {
        const size_t smem = msc_smem_bytes(N, G);
        if (smem > 227 * 1024) break;
        if (smem > 48 * 1024 &&
            cudaFuncSetAttribute(k_sweep_msc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            break;
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sweep_msc, kMscThreads, smem) != cudaSuccess ||
            per_sm < 1)
            break;
        const uint64_t ctas = (groups + G - 1) / G, slots = (uint64_t)per_sm * (uint64_t)sms;
        const uint64_t waves = (ctas + slots - 1) / slots;
        const double eff = (double)ctas / (double)(waves * slots);
        if (eff >= best_eff - 1e-9) {
            best_eff = eff;
            best = G;
        }
        if (ctas <= 1) break;
    }
    return best;
}

cudaError_t launch_sweep_msc(const SweepLaunch& P, uint32_t n_ctas, uint32_t G, cudaStream_t s) {
    size_t smem = 0;
    for (int j = 0; j < P.njobs; ++j) {
        const size_t b = msc_smem_bytes(P.jobs[j].N, G);
        if (b > smem) smem = b;
    }
    if (G < 1 || G > 4) return cudaErrorInvalidValue;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_sweep_msc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_sweep_msc<<<n_ctas, kMscThreads, smem, s>>>(P, G);
    count_launch();
    return cudaGetLastError();
}

}  // namespace gbmc
