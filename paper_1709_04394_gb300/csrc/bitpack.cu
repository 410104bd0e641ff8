// bitpack.cu -- the bit-packed ("multi-spin coded", Sec. 3.1) layout of 2D
// ferromagnets: one bit per spin. Per copy, two colour planes; plane c, row y,
// word w holds the sites j = 32w .. 32w+31 of colour c in row y (site
// x = 2j + ((y+c)&1)), bit = 1 where s = -1. L % 64 == 0.
//
// Sweeps use the same Philox words as the int8 layouts (the counter of a site
// depends only on its colour rank), so both layouts give identical spins.
// For the 32 sites of a word, the four neighbours are the same word of the
// other plane in rows y-1, y, y+1 and that word shifted by one bit; the
// number of unsatisfied bonds a (0..4) is summed bit-sliced (a0 + 2 a1 + 4 a2)
// and a site flips iff a >= 2, or a = 1 and u <= T(4), or a = 0 and u <= T(8).
//
// Two sweep kernels:
//  k_bp_halfsweep : one launch per half-sweep, one thread per word of the plane
//                   (any L % 64 == 0, any number of copies);
//  k_bp_strips    : all sweeps of a call in one cooperative launch. Each CTA
//                   keeps a strip of rows of both planes in shared memory for the
//                   whole run, with one halo row above and below. After each
//                   half-sweep it writes only its first and last rows back to
//                   global memory (updated first, then published by a progress
//                   counter) and, before the next one, reads its two neighbours'
//                   boundary rows once their counters show them. Each half-sweep
//                   reads the other plane as the previous half-sweep left it, so
//                   the result is that of the per-half-sweep launches.
#include "bits.cuh"
#include "device.cuh"
#include "internal.h"
#include "strips.cuh"

namespace gbmc {

// Random (or all-up) start written directly in packed form: word (copy,
// colour, row, w); the INIT word of site i is word i&3 of q = i>>2.
__global__ void k_bp_init(uint32_t* P, uint32_t L, uint64_t words_total, uint32_t R, uint32_t inst_base, uint32_t k0,
                          uint32_t k1, int random_start) {
    const uint32_t Wr = L >> 6;                    // words per plane row
    const uint64_t per_copy = 2ull * L * Wr;
    for (uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; g < words_total;
         g += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t word = 0;
        if (random_start) {
            const uint64_t copy = g / per_copy;
            const uint32_t rem = (uint32_t)(g - copy * per_copy);
            const uint32_t c = rem / (L * Wr), rw = rem - c * (L * Wr);
            const uint32_t y = rw / Wr, w = rw - y * Wr;
            const uint32_t inst = (uint32_t)(copy / R), r = (uint32_t)(copy - (uint64_t)inst * R);
            const uint32_t o = (y + c) & 1u;
            const uint32_t c3 = c3_word(kPurposeInit, 0u, inst_base + inst);
            // sites x = 64w + o + 2b, b = 0..31: 64 consecutive columns from 64w
            for (uint32_t qq = 0; qq < 16; ++qq) {
                const uint32_t site0 = y * L + 64 * w + 4 * qq;
                const uint4 v = philox4x32_10(make_uint4(site0 >> 2, 0u, r, c3), k0, k1);
                // columns 64w + 4qq + {0,1,2,3}; those with parity o are bits b = 2qq + (col-o)/2
                const uint32_t u[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (uint32_t l = 0; l < 4; ++l) {
                    if ((l & 1u) != o) continue;
                    const uint32_t b = 2 * qq + (l >> 1);
                    word |= (u[l] >> 31) << b;
                }
            }
        }
        P[g] = word;
    }
}

cudaError_t launch_bp_init(uint32_t* P, uint32_t L, uint64_t copies, uint32_t R, uint32_t inst_base, uint64_t seed,
                           int random_start, cudaStream_t s) {
    const uint64_t total = copies * 2ull * L * (L >> 6);
    uint64_t blocks = (total + 255) / 256;
    if (blocks > 152ull * 32) blocks = 152ull * 32;
    k_bp_init<<<(uint32_t)blocks, 256, 0, s>>>(P, L, total, R, inst_base, (uint32_t)seed, (uint32_t)(seed >> 32),
                                               random_start);
    count_launch();
    return cudaGetLastError();
}

// int8 row-major <-> packed planes; one thread per packed word.
__global__ void k_bp_pack(const int8_t* src, uint32_t* P, uint32_t L, uint64_t words_total) {
    const uint32_t Wr = L >> 6;
    const uint64_t per_copy = 2ull * L * Wr;
    for (uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; g < words_total;
         g += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t copy = g / per_copy;
        const uint32_t rem = (uint32_t)(g - copy * per_copy);
        const uint32_t c = rem / (L * Wr), rw = rem - c * (L * Wr);
        const uint32_t y = rw / Wr, w = rw - y * Wr;
        const uint32_t o = (y + c) & 1u;
        const int8_t* row = src + copy * (uint64_t)L * L + (uint64_t)y * L + 64ull * w + o;
        uint32_t word = 0;
        for (uint32_t b = 0; b < 32; ++b) word |= (uint32_t)(row[2 * b] < 0) << b;
        P[g] = word;
    }
}

__global__ void k_bp_unpack(const uint32_t* P, int8_t* dst, uint32_t L, uint64_t words_total) {
    const uint32_t Wr = L >> 6;
    const uint64_t per_copy = 2ull * L * Wr;
    for (uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; g < words_total;
         g += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t copy = g / per_copy;
        const uint32_t rem = (uint32_t)(g - copy * per_copy);
        const uint32_t c = rem / (L * Wr), rw = rem - c * (L * Wr);
        const uint32_t y = rw / Wr, w = rw - y * Wr;
        const uint32_t o = (y + c) & 1u;
        int8_t* row = dst + copy * (uint64_t)L * L + (uint64_t)y * L + 64ull * w + o;
        const uint32_t word = P[g];
        for (uint32_t b = 0; b < 32; ++b) row[2 * b] = ((word >> b) & 1u) ? -1 : 1;
    }
}

cudaError_t launch_bp_pack(const int8_t* src, uint32_t* P, uint32_t L, uint64_t copies, cudaStream_t s) {
    const uint64_t total = copies * 2ull * L * (L >> 6);
    uint64_t blocks = (total + 255) / 256;
    if (blocks > 152ull * 32) blocks = 152ull * 32;
    k_bp_pack<<<(uint32_t)blocks, 256, 0, s>>>(src, P, L, total);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_bp_unpack(const uint32_t* P, int8_t* dst, uint32_t L, uint64_t copies, cudaStream_t s) {
    const uint64_t total = copies * 2ull * L * (L >> 6);
    uint64_t blocks = (total + 255) / 256;
    if (blocks > 152ull * 32) blocks = 152ull * 32;
    k_bp_unpack<<<(uint32_t)blocks, 256, 0, s>>>(P, dst, L, total);
    count_launch();
    return cudaGetLastError();
}

// Neighbours of the colour-c word (y, w): the other plane's words in rows
// y-1, y+1, y and the row-y word shifted by one site towards j-1 (even x) or
// j+1 (odd x).
__device__ __forceinline__ void bp_neighbours(const uint32_t* oth, uint32_t L, uint32_t Wr, uint32_t y, uint32_t w,
                                              uint32_t o, uint32_t& up, uint32_t& dn, uint32_t& same,
                                              uint32_t& side) {
    const uint32_t yu = y == 0 ? L - 1 : y - 1, yd = y + 1 == L ? 0 : y + 1;
    up = __ldcg(oth + yu * Wr + w);
    dn = __ldcg(oth + yd * Wr + w);
    same = __ldcg(oth + y * Wr + w);
    if (o) {
        const uint32_t nx = __ldcg(oth + y * Wr + (w + 1 == Wr ? 0 : w + 1));
        side = __funnelshift_r(same, nx, 1);   // bits j+1
    } else {
        const uint32_t pv = __ldcg(oth + y * Wr + (w == 0 ? Wr - 1 : w - 1));
        side = __funnelshift_l(pv, same, 1);   // bits j-1
    }
}

// One half-sweep of colour c over every copy: one thread per word of plane c.
__global__ void __launch_bounds__(256) k_bp_halfsweep(uint32_t* P, uint32_t L, uint64_t copies, uint32_t R,
                                                      uint32_t inst_base, uint32_t colour, uint32_t t, uint32_t k0,
                                                      uint32_t k1, uint32_t T4, uint32_t T8) {
    const uint32_t Wr = L >> 6;
    const uint64_t plane_words = (uint64_t)L * Wr;
    const uint64_t total = copies * plane_words;
    const uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (g >= total) return;
    const uint64_t copy = g / plane_words;
    const uint32_t rw = (uint32_t)(g - copy * plane_words);
    const uint32_t y = rw / Wr, w = rw - y * Wr;
    const uint32_t inst = (uint32_t)(copy / R), r = (uint32_t)(copy - (uint64_t)inst * R);
    uint32_t* own = P + copy * 2 * plane_words + colour * plane_words;
    const uint32_t* oth = P + copy * 2 * plane_words + (colour ^ 1u) * plane_words;
    const uint32_t o = (y + colour) & 1u;
    uint32_t up, dn, same, side;
    bp_neighbours(oth, L, Wr, y, w, o, up, dn, same, side);
    const PhiloxFixed pf = philox_fix(t, r, c3_word(kPurposeMetro, colour, inst_base + inst), k0, k1);
    own[rw] = bp_word_update(own[rw], up, dn, same, side, pf, y * (L >> 3) + 8 * w, T4, T8);
}

cudaError_t launch_bp_halfsweep(uint32_t* P, uint32_t L, uint64_t copies, uint32_t R, uint32_t inst_base,
                                uint64_t seed, uint32_t colour, uint32_t t, uint32_t T4, uint32_t T8, cudaStream_t s) {
    const uint64_t total = copies * (uint64_t)L * (L >> 6);
    const uint64_t blocks = (total + 255) / 256;
    if (blocks > 0x7FFFFFFFull) return cudaErrorInvalidValue;
    k_bp_halfsweep<<<(uint32_t)blocks, 256, 0, s>>>(P, L, copies, R, inst_base, colour, t, (uint32_t)seed,
                                                    (uint32_t)(seed >> 32), T4, T8);
    count_launch();
    return cudaGetLastError();
}

// ---- strip-resident sweeps ----

constexpr uint32_t kBpStripThreads = 1024;

__global__ void __launch_bounds__(kBpStripThreads, 1) k_bp_strips(const __grid_constant__ BpStrips S) {
    extern __shared__ uint32_t sm[];
    __shared__ int s_ok;
    const uint32_t tid = threadIdx.x, B = blockDim.x;
    const uint32_t L = S.L, Wr = L >> 6;
    const uint32_t copy = blockIdx.x / S.Gc, g = blockIdx.x - copy * S.Gc;
    const uint32_t y0 = (uint32_t)((uint64_t)g * L / S.Gc), y1 = (uint32_t)((uint64_t)(g + 1) * L / S.Gc);
    const uint32_t rs = y1 - y0;  // >= 2
    const uint32_t inst = copy / S.R, r = copy - inst * S.R;
    const uint32_t k0 = (uint32_t)S.seed, k1 = (uint32_t)(S.seed >> 32);
    const uint32_t ps = (S.rmax + 2) * Wr;  // words per plane in shared memory
    uint32_t* gp = S.P + (uint64_t)copy * 2 * L * Wr;
    // local row lr: 0 = the row above the strip, 1..rs = rows y0..y1-1, rs+1 = the row below
    const uint32_t yu = y0 == 0 ? L - 1 : y0 - 1, yd = y1 == L ? 0 : y1;
    auto grow = [&](uint32_t lr) { return lr == 0 ? yu : (lr == rs + 1 ? yd : y0 + lr - 1); };
    for (uint32_t k = tid; k < 2 * (rs + 2) * Wr; k += B) {
        const uint32_t c = k / ((rs + 2) * Wr), rem = k - c * (rs + 2) * Wr, lr = rem / Wr, w = rem - lr * Wr;
        sm[c * ps + lr * Wr + w] = __ldcg(gp + ((uint64_t)c * L + grow(lr)) * Wr + w);
    }
    if (tid == 0) s_ok = 1;
    __syncthreads();  // all loads done before this CTA publishes anything
    const unsigned int* pu = S.progress + copy * S.Gc + (g == 0 ? S.Gc - 1 : g - 1);
    const unsigned int* pd = S.progress + copy * S.Gc + (g + 1 == S.Gc ? 0 : g + 1);
    // Warps 0 .. nb/32 - 1 (thread k < nb) own the first and last rows: thread
    // k < Wr word k of row 1, thread Wr + w word w of row rs. Each also
    // refreshes the one halo word its update reads (row 0, resp. rs + 1), so
    // only these warps wait for the neighbours, on named barrier 1; the other
    // warps go straight to the interior rows.
    const uint32_t nb = 2 * Wr, total = rs * Wr;
    // this thread's interior words k = k0, k0 + B, ... (fixed for the whole
    // launch: rows and columns worked out once), two updated at a time below
    constexpr uint32_t kMaxOwn = 4;
    uint32_t own_lr[kMaxOwn], own_w[kMaxOwn], n_own = 0;
    bool listed = true;
    for (uint32_t k = tid + (tid < nb ? B : 0u); k < total; k += B) {  // k >= nb: B >= nb by the launch shape
        if (n_own == kMaxOwn) {
            listed = false;  // more than kMaxOwn words per thread: the generic walk
            break;
        }
        const uint32_t kk = k - nb, lr = 2 + kk / Wr;
#pragma unroll
        for (uint32_t i = 0; i < kMaxOwn; ++i)
            if (i == n_own) {
                own_lr[i] = lr;
                own_w[i] = kk - (lr - 2) * Wr;
            }
        ++n_own;
    }
    for (uint32_t h = 0; h < S.n_half; ++h) {
        const uint32_t c = h & 1u;
        uint32_t* own = sm + c * ps;
        const uint32_t* oth = sm + (c ^ 1u) * ps;
        const PhiloxFixed pf = philox_fix(S.t0 + (h >> 1), r, c3_word(kPurposeMetro, c, S.inst_base + inst), k0, k1);
        auto update = [&](uint32_t lr, uint32_t w) {
            const uint32_t y = y0 + lr - 1, o = (y + c) & 1u;
            const uint32_t* orow = oth + lr * Wr;
            const uint32_t same = orow[w];
            const uint32_t side = o ? __funnelshift_r(same, orow[w + 1 == Wr ? 0 : w + 1], 1)   // bits j+1
                                    : __funnelshift_l(orow[w == 0 ? Wr - 1 : w - 1], same, 1);  // bits j-1
            const uint32_t v = bp_word_update(own[lr * Wr + w], oth[(lr - 1) * Wr + w], oth[(lr + 1) * Wr + w], same,
                                              side, pf, y * (L >> 3) + 8 * w, S.T4, S.T8);
            own[lr * Wr + w] = v;
            return v;
        };
        if (tid < nb) {
            const uint32_t lr = tid < Wr ? 1 : rs, w = tid < Wr ? tid : tid - Wr;
            if (h > 0) {
                // the neighbours' boundary rows of the other plane from half-sweep h - 1
                if (tid == 0 && !strip_wait(pu, pd, h + S.phantom, S.err, S.budget)) s_ok = 0;
                asm volatile("bar.sync 1, %0;" ::"r"(nb) : "memory");
                const uint32_t hr = tid < Wr ? 0 : rs + 1;
                sm[(c ^ 1u) * ps + hr * Wr + w] = __ldcg(gp + ((uint64_t)(c ^ 1u) * L + grow(hr)) * Wr + w);
            }
            if (s_ok) gp[((uint64_t)c * L + y0 + lr - 1) * Wr + w] = update(lr, w);
            // the boundary warps meet; one fence then orders all their stores
            asm volatile("bar.sync 1, %0;" ::"r"(nb) : "memory");
            if (tid == 0 && s_ok) {
                __threadfence();
                atomicExch(S.progress + blockIdx.x, h + 1u);
            }
        }
        if (listed) {
            // two words at a time: both loaded and updated before either is
            // stored (they read only the other plane)
            auto gather = [&](uint32_t lr, uint32_t w, uint32_t& up, uint32_t& dn, uint32_t& same, uint32_t& side,
                              uint32_t& q) {
                const uint32_t y = y0 + lr - 1, o = (y + c) & 1u;
                const uint32_t* orow = oth + lr * Wr;
                same = orow[w];
                side = o ? __funnelshift_r(same, orow[w + 1 == Wr ? 0 : w + 1], 1)   // bits j+1
                         : __funnelshift_l(orow[w == 0 ? Wr - 1 : w - 1], same, 1);  // bits j-1
                up = oth[(lr - 1) * Wr + w];
                dn = oth[(lr + 1) * Wr + w];
                q = y * (L >> 3) + 8 * w;
            };
#pragma unroll
            for (uint32_t i = 0; i < kMaxOwn; i += 2) {
                if (i + 1 < n_own) {
                    uint32_t ua, da, sa, xa, qa, ub, db, sb, xb, qb;
                    gather(own_lr[i], own_w[i], ua, da, sa, xa, qa);
                    gather(own_lr[i + 1], own_w[i + 1], ub, db, sb, xb, qb);
                    uint32_t* pa = own + own_lr[i] * Wr + own_w[i];
                    uint32_t* pb = own + own_lr[i + 1] * Wr + own_w[i + 1];
                    const uint32_t na = bp_word_update(*pa, ua, da, sa, xa, pf, qa, S.T4, S.T8);
                    const uint32_t nbw = bp_word_update(*pb, ub, db, sb, xb, pf, qb, S.T4, S.T8);
                    *pa = na;
                    *pb = nbw;
                } else if (i < n_own) {
                    update(own_lr[i], own_w[i]);
                }
            }
        } else {
            for (uint32_t k = tid + (tid < nb ? B : 0u); k < total; k += B) {
                const uint32_t kk = k - nb, lr = 2 + kk / Wr;
                update(lr, kk - (lr - 2) * Wr);
            }
        }
        __syncthreads();
        if (!s_ok) return;
    }
    for (uint32_t k = tid; k < 2 * total; k += B) {
        const uint32_t c = k / total, rem = k - c * total, lr = 1 + rem / Wr, w = rem - (lr - 1) * Wr;
        gp[((uint64_t)c * L + y0 + lr - 1) * Wr + w] = sm[c * ps + lr * Wr + w];
    }
}

bool bp_strips_shape(uint32_t L, uint64_t copies, int sm_count, uint32_t& Gc, uint32_t& rmax, uint32_t& threads,
                     size_t& smem) {
    // L % 1024 == 0: the 2 L/64 words of a strip's first and last rows are whole
    // warps (they meet on a named barrier); at least 8 strips per copy, one per SM
    if (L % 1024 != 0 || copies == 0 || sm_count < 8 || copies > (uint64_t)sm_count / 8) return false;
    const uint32_t Wr = L >> 6;
    Gc = (uint32_t)((uint64_t)sm_count / copies);
    if (Gc > L / 2) Gc = L / 2;  // two rows or more per strip
    rmax = (L + Gc - 1) / Gc;
    const uint32_t words = rmax * Wr, iters = (words + kBpStripThreads - 1) / kBpStripThreads;
    threads = ((words + iters - 1) / iters + 31) / 32 * 32;
    smem = 2ull * (rmax + 2) * Wr * sizeof(uint32_t);
    if (2 * Wr > threads || smem > 200u * 1024u) return false;
    int fit = 0;
    if (cudaFuncSetAttribute(k_bp_strips, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, k_bp_strips, (int)threads, smem) != cudaSuccess)
        return false;
    return fit >= 1;
}

cudaError_t launch_bp_strips(const BpStrips& S, uint64_t copies, uint32_t threads, size_t smem, int sm_count,
                             cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(k_bp_strips, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bp_strips, (int)threads, smem);
    if (e != cudaSuccess) return e;
    const uint64_t grid = copies * S.Gc;
    if (per_sm < 1 || grid > (uint64_t)per_sm * sm_count) return cudaErrorCooperativeLaunchTooLarge;
    e = cudaMemsetAsync(S.progress, 0, grid * sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    BpStrips Sc = S;
    void* args[] = {&Sc};
    e = cudaLaunchCooperativeKernel((const void*)k_bp_strips, dim3((uint32_t)grid), dim3(threads), args, smem, s);
    count_launch();
    return e;
}

// E and M of every copy: E = -sum over odd sites of s_i h_i = -(4 N/2 - 2 sum a_i),
// M = N - 2 (number of down spins). One block per copy.
__global__ void k_bp_observables(const uint32_t* P, uint32_t L, int32_t* E, int32_t* M) {
    const uint32_t Wr = L >> 6;
    const uint64_t plane_words = (uint64_t)L * Wr;
    const uint64_t copy = blockIdx.x;
    const uint32_t* p0 = P + copy * 2 * plane_words;
    const uint32_t* p1 = p0 + plane_words;
    long long unsat = 0, down = 0;
    for (uint32_t rw = threadIdx.x; rw < plane_words; rw += blockDim.x) {
        const uint32_t y = rw / Wr, w = rw - y * Wr;
        const uint32_t o = (y + 1u) & 1u;
        uint32_t up, dn, same, side;
        bp_neighbours(p0, L, Wr, y, w, o, up, dn, same, side);
        const uint32_t s = p1[rw];
        unsat += __popc(s ^ up) + __popc(s ^ dn) + __popc(s ^ same) + __popc(s ^ side);
        down += __popc(s) + __popc(p0[rw]);
    }
    unsat = warp_sum(unsat);
    down = warp_sum(down);
    __shared__ long long su[32], sd[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        su[warp] = unsat;
        sd[warp] = down;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long a = 0, b = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) a += su[i], b += sd[i];
        const long long N = (long long)L * L;
        if (E) E[copy] = (int32_t)(-(2 * N - 2 * a));
        if (M) M[copy] = (int32_t)(N - 2 * b);
    }
}

cudaError_t launch_bp_observables(const uint32_t* P, uint32_t L, uint64_t copies, int32_t* E, int32_t* M,
                                  cudaStream_t s) {
    if (copies > 0x7FFFFFFFull) return cudaErrorInvalidValue;
    k_bp_observables<<<(uint32_t)copies, 256, 0, s>>>(P, L, E, M);
    count_launch();
    return cudaGetLastError();
}

}  // namespace gbmc
