// tiles.cu -- checkerboard Metropolis sweeps of 2D ferromagnets too large for
// one CTA's shared memory (Sec. 3.1): strips of rows resident in shared memory
// for a whole call and halo tiles, both reproducing the plain two-phase sweeps
// exactly, and the double checkerboard of Fig. 5 (right) with k sweeps per
// tile load.
#include "device.cuh"
#include "internal.h"
#include "strips.cuh"
#include "units.cuh"

namespace gbmc {

// ---- tiled sweeps of large 2D lattices: shared-memory tiles with a halo ----
// Each CTA loads a (T + 16) x (T + 16) window (an 8-site halo on every side,
// periodic wrap) of one copy into shared memory as colour planes, runs up to 4
// full sweeps on it, and writes back the T x T interior to the other buffer.
// Half-sweep s updates rows [s + 1, W - s - 1) of the window: the region whose
// neighbours are still exact shrinks by one site per half-sweep, so after 2k
// <= 8 half-sweeps the interior equals the two-phase checkerboard sweeps of the
// whole lattice (Sec. 3.1). Halo sites get updated with stale neighbours and
// are discarded. The 8-site halo keeps every plane word aligned with a whole
// Philox call (4 same-colour sites = 8 lattice columns).
template <uint32_t T>
__global__ void __launch_bounds__(256) k_sweep_tiles(const __grid_constant__ TileLaunch P) {
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ __align__(16) uint32_t s_tbl[8];
    constexpr uint32_t Wd = T + 16, Wg = Wd >> 3, H = (Wd * Wd) >> 1;
    const uint32_t L = P.L, Lw = L >> 3;
    const uint32_t tiles_x = L / T;
    const uint32_t ty = blockIdx.x / tiles_x, tx = blockIdx.x - ty * tiles_x;
    const uint64_t copy = (uint64_t)P.copy0 + blockIdx.y;
    uint32_t inst, r;
    split_copy(copy, P.R, inst, r);
    const int8_t* src = P.src + copy * (uint64_t)L * L;
    int8_t* dst = P.dst + copy * (uint64_t)L * L;
    const uint32_t y0 = (ty * T + L - 8) % L;  // global row of window row 0
    const uint32_t xw0 = ((tx * T + L - 8) % L) >> 3;  // global 8-column chunk of window chunk 0
    // load with periodic wrap; chunks never straddle the wrap (L % 8 == 0)
    uint32_t* pl = reinterpret_cast<uint32_t*>(smem);
    for (uint32_t idx = threadIdx.x; idx < Wd * Wg; idx += blockDim.x) {
        const uint32_t rr = idx / Wg, cx = idx - rr * Wg;
        uint32_t gy = y0 + rr, gc = xw0 + cx;
        if (gy >= L) gy -= L;
        if (gc >= Lw) gc -= Lw;
        const uint2 v = *reinterpret_cast<const uint2*>(src + (uint64_t)gy * L + 8ull * gc);
        const uint32_t pe = gy & 1u;  // colour of the even columns of this row
        pl[pe * (H >> 2) + idx] = __byte_perm(v.x, v.y, 0x6420);
        pl[(pe ^ 1u) * (H >> 2) + idx] = __byte_perm(v.x, v.y, 0x7531);
    }
    if (threadIdx.x < 8) {
        const int d = 2 - (int)threadIdx.x;
        s_tbl[threadIdx.x] = d <= 0 ? 0xFFFFFFFFu : (d == 1 ? P.thr[0] : P.thr[1]);
    }
    __syncthreads();
    const uint8_t* tbl = reinterpret_cast<const uint8_t*>(s_tbl);
    const uint32_t k0 = (uint32_t)P.seed, k1 = (uint32_t)(P.seed >> 32);
    const uint32_t instance = P.inst_base + inst;
    int e = 0, m = 0;
    for (uint32_t s = 0; s < 2 * P.nsweeps; ++s) {
        const uint32_t colour = s & 1u, t = P.t0 + (s >> 1);
        const PhiloxFixed pf = philox_fix(t, r, c3_word(kPurposeMetro, colour, instance), k0, k1);
        const uint32_t row_lo = s + 1, rows = Wd - 2 * (s + 1);
        for (uint32_t u = threadIdx.x; u < rows * Wg; u += blockDim.x) {
            const uint32_t rr = u / Wg, g = u - rr * Wg;
            const uint32_t row = row_lo + rr;
            uint32_t gy = y0 + row, gc = xw0 + g;
            if (gy >= L) gy -= L;
            if (gc >= Lw) gc -= Lw;
            const uint32_t q = gy * Lw + gc;
            unit_split<2, false, false>(smem, nullptr, Wd, Wd * Wd, row, row, 0, g, colour, pf, tbl, true, e, m, q);
        }
        __syncthreads();
    }
    // store the T x T interior: window rows [8, 8 + T), chunks [1, 1 + T/8)
    constexpr uint32_t Tc = T >> 3;
    for (uint32_t idx = threadIdx.x; idx < T * Tc; idx += blockDim.x) {
        const uint32_t rr = idx / Tc, cx = idx - rr * Tc;
        const uint32_t wrow = rr + 8, wc = cx + 1;
        const uint32_t gy = ty * T + rr, gx = tx * T + 8 * cx;
        const uint32_t pe = gy & 1u;
        const uint32_t ev = pl[pe * (H >> 2) + wrow * Wg + wc], od = pl[(pe ^ 1u) * (H >> 2) + wrow * Wg + wc];
        uint2 v;
        v.x = __byte_perm(ev, od, 0x5140);
        v.y = __byte_perm(ev, od, 0x7362);
        *reinterpret_cast<uint2*>(dst + (uint64_t)gy * L + gx) = v;
    }
}

size_t tile_smem_bytes(uint32_t T) { return (size_t)(T + 16) * (T + 16); }

cudaError_t launch_sweep_tiles(const TileLaunch& P, uint64_t copies, cudaStream_t s) {
    const size_t smem = tile_smem_bytes(P.T);
    if (P.T != 128 && P.T != 256) return cudaErrorInvalidValue;
    auto kern = P.T == 128 ? k_sweep_tiles<128> : k_sweep_tiles<256>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const uint32_t tiles = (P.L / P.T) * (P.L / P.T);
    for (uint64_t c0 = 0; c0 < copies; c0 += 65535) {
        TileLaunch Q = P;
        Q.copy0 = (uint32_t)c0;
        const uint32_t nc = (uint32_t)((copies - c0) < 65535 ? (copies - c0) : 65535);
        kern<<<dim3(tiles, nc), 256, smem, s>>>(Q);
        count_launch();
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// ---- strip-resident sweeps of large 2D lattices ----
constexpr uint32_t kStripThreads = 1024;
// All sweeps of a call in one cooperative launch: CTA g of a copy keeps rows
// [y0, y1) of the copy, plus the row above and the row below, as colour planes
// in shared memory for the whole run. After each half-sweep only its first and
// last rows go back to global memory (updated first, then published through a
// progress counter); before the next one the CTA reads its neighbours' first
// and last rows once their counters show them. Each half-sweep sees the other
// colour as the previous half-sweep left it: the plain two-phase sweeps of
// the whole lattice, in place, with no halo recomputation.

// Each half-sweep: the threads with boundary units (first and last rows)
// update them, write them back and meet on a named barrier, after which one
// thread publishes the half-sweep; then every thread walks its word column
// (t % W) down the interior rows, B/W rows apart. Two passes into that walk,
// the boundary threads wait for the neighbours' same half-sweep (lane 0 of
// each warp polls) and fetch the halo words their next units read. One
// CTA-wide barrier ends the half-sweep.
__global__ void __launch_bounds__(kStripThreads, 1) k_sweep_strips(const __grid_constant__ StripLaunch S) {
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ __align__(16) uint32_t s_tbl[8];
    __shared__ int s_ok;
    const uint32_t tid = threadIdx.x, B = blockDim.x;
    const uint32_t L = S.L, W = L >> 3;  // words per plane row = 8-site chunks per lattice row
    const uint32_t copy = blockIdx.x / S.Gc, g = blockIdx.x - copy * S.Gc;
    const uint32_t y0 = (uint32_t)((uint64_t)g * L / S.Gc), y1 = (uint32_t)((uint64_t)(g + 1) * L / S.Gc);
    const uint32_t rs = y1 - y0;  // >= 2
    const uint32_t inst = copy / S.R, r = copy - inst * S.R;
    const uint32_t k0 = (uint32_t)S.seed, k1 = (uint32_t)(S.seed >> 32);
    const uint32_t NL = (S.rmax + 2) * L, ps = NL >> 3;  // bytes of both planes; words per plane
    uint32_t* pl = reinterpret_cast<uint32_t*>(smem);
    int8_t* gs = S.spins + (uint64_t)copy * L * L;
    // local row lr: 0 = the row above the strip, 1..rs = rows y0..y1-1, rs+1 = the row below
    const uint32_t yu = y0 == 0 ? L - 1 : y0 - 1, yd = y1 == L ? 0 : y1;
    auto grow = [&](uint32_t lr) { return lr == 0 ? yu : (lr == rs + 1 ? yd : y0 + lr - 1); };
    // the even columns of row y have colour y & 1
    for (uint32_t idx = tid; idx < (rs + 2) * W; idx += B) {
        const uint32_t lr = idx / W, gy = grow(lr);
        const uint2 v = __ldcg(reinterpret_cast<const uint2*>(gs + (uint64_t)gy * L) + (idx - lr * W));
        const uint32_t pe = gy & 1u;
        pl[pe * ps + idx] = __byte_perm(v.x, v.y, 0x6420);
        pl[(pe ^ 1u) * ps + idx] = __byte_perm(v.x, v.y, 0x7531);
    }
    if (tid < 8) {
        const int d = 2 - (int)tid;
        s_tbl[tid] = d <= 0 ? 0xFFFFFFFFu : (d == 1 ? S.thr[0] : S.thr[1]);
    }
    if (tid == 0) s_ok = 1;
    __syncthreads();  // all loads done before this CTA publishes anything
    const uint8_t* tbl = reinterpret_cast<const uint8_t*>(s_tbl);
    const unsigned int* pu = S.progress + copy * S.Gc + (g == 0 ? S.Gc - 1 : g - 1);
    const unsigned int* pd = S.progress + copy * S.Gc + (g + 1 == S.Gc ? 0 : g + 1);
    // unit_split walks rows of an L-wide lattice: pass it a row index with the
    // parity of the global row that never wraps (2 or 3 above the local row)
    const uint32_t ydelta = 2 + ((y0 + 1) & 1u);
    const uint32_t nb = 2 * W, total = rs * W, w = tid % W, rstep = B / W;
    const uint32_t nbth = nb < B ? nb : B;  // threads with boundary units
    int e = 0, m = 0;
    for (uint32_t h = 0; h < S.n_half; ++h) {
        const uint32_t c = h & 1u;
        const PhiloxFixed pf = philox_fix(S.t0 + (h >> 1), r, c3_word(kPurposeMetro, c, S.inst_base + inst), k0, k1);
        auto update = [&](uint32_t lr, uint32_t wc) {
            unit_split<2, false, false>(smem, nullptr, L, NL, lr, lr + ydelta, 0, wc, c, pf, tbl, true, e, m,
                                        (y0 + lr - 1) * W + wc);
        };
        // four rows of the column at a time: all four units are loaded and
        // updated before any word is stored (rows of one plane: none reads what
        // another writes)
        uint32_t* own = pl + c * ps;
        auto update4 = [&](uint32_t lr) {
            uint32_t ii[4], vv[4];
#pragma unroll
            for (uint32_t k = 0; k < 4; ++k) {
                const uint32_t rk = lr + k * rstep;
                unit_split<2, false, false, false>(smem, nullptr, L, NL, rk, rk + ydelta, 0, w, c, pf, tbl, true, e,
                                                   m, (y0 + rk - 1) * W + w, &ii[k], &vv[k]);
            }
#pragma unroll
            for (uint32_t k = 0; k < 4; ++k) own[ii[k]] = vv[k];
        };
        // boundary unit k < W: word k of row 1 (next to halo row 0); W + w: word
        // w of row rs (next to rs + 1)
        if (tid < nb) {
            for (uint32_t k = tid; k < nb; k += B) {
                const uint32_t lr = k < W ? 1 : rs, wk = k < W ? k : k - W;
                update(lr, wk);
                const uint32_t gy = y0 + lr - 1, pe = gy & 1u;
                const uint32_t ev = pl[pe * ps + lr * W + wk], od = pl[(pe ^ 1u) * ps + lr * W + wk];
                uint2 v;
                v.x = __byte_perm(ev, od, 0x5140);
                v.y = __byte_perm(ev, od, 0x7362);
                reinterpret_cast<uint2*>(gs + (uint64_t)gy * L)[wk] = v;
            }
            // the boundary threads (whole warps) meet; one fence then orders all their stores
            asm volatile("bar.sync 1, %0;" ::"r"(nbth) : "memory");
            if (tid == 0) {
                __threadfence();
                atomicExch(S.progress + blockIdx.x, h + 1u);
            }
        }
        // interior rows 2 .. rs - 1. After the first two passes (the neighbours
        // publish at the start of their half-sweep), the halo words the next
        // half-sweep's boundary units read: this plane as the neighbours left it
        // after this half-sweep, each fetched by the thread that uses it (the
        // halo rows of this plane are not read in this half-sweep)
        uint32_t lr = 2 + tid / W;
        for (uint32_t i = 0; i < 2 && lr < rs; ++i, lr += rstep) update(lr, w);
        if (tid < nb && h + 1 < S.n_half) {
            // lane 0 of each warp polls (W % 32 == 0: whole warps here, in step)
            int ok = 1;
            if ((tid & 31u) == 0) ok = strip_wait(pu, pd, h + 1 + S.phantom, S.err, S.budget);
            if (!__shfl_sync(0xffffffffu, ok, 0)) s_ok = 0;
            for (uint32_t k = tid; k < nb; k += B) {
                const uint32_t hr = k < W ? 0 : rs + 1, wk = k < W ? k : k - W, gy = grow(hr);
                const uint2 v = __ldcg(reinterpret_cast<const uint2*>(gs + (uint64_t)gy * L) + wk);
                pl[c * ps + hr * W + wk] = __byte_perm(v.x, v.y, (gy & 1u) == c ? 0x6420 : 0x7531);
            }
        }
        for (; lr + 3 * rstep < rs; lr += 4 * rstep) update4(lr);
        for (; lr < rs; lr += rstep) update(lr, w);
        __syncthreads();
        if (!s_ok) return;
    }
    for (uint32_t idx = tid; idx < total; idx += B) {
        const uint32_t lr = 1 + idx / W, wk = idx - (lr - 1) * W, gy = y0 + lr - 1, pe = gy & 1u;
        const uint32_t ev = pl[pe * ps + lr * W + wk], od = pl[(pe ^ 1u) * ps + lr * W + wk];
        uint2 v;
        v.x = __byte_perm(ev, od, 0x5140);
        v.y = __byte_perm(ev, od, 0x7362);
        reinterpret_cast<uint2*>(gs + (uint64_t)gy * L)[wk] = v;
    }
}

bool strips_shape(uint32_t L, uint64_t copies, int sm_count, uint32_t& Gc, uint32_t& rmax, uint32_t& threads,
                  size_t& smem) {
    // L % 256 == 0: a plane row is whole warps' worth of words (W % 32 == 0), so
    // a warp's threads share their rows; at least 8 strips per copy, one per SM
    if (L % 256 != 0 || copies == 0 || sm_count < 8 || copies > (uint64_t)sm_count / 8) return false;
    const uint32_t W = L >> 3;
    if (W > kStripThreads) return false;
    Gc = (uint32_t)((uint64_t)sm_count / copies);
    if (Gc > L / 2) Gc = L / 2;
    rmax = (L + Gc - 1) / Gc;
    // whole rows per pass: a thread keeps one word column
    const uint32_t rows = kStripThreads / W < rmax ? kStripThreads / W : rmax;
    threads = rows * W;
    smem = (size_t)(rmax + 2) * L;
    if (smem > 200u * 1024u) return false;
    int fit = 0;
    if (cudaFuncSetAttribute(k_sweep_strips, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, k_sweep_strips, (int)threads, smem) != cudaSuccess)
        return false;
    return fit >= 1;
}

cudaError_t launch_sweep_strips(const StripLaunch& S, uint64_t copies, uint32_t threads, size_t smem, int sm_count,
                                cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(k_sweep_strips, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sweep_strips, (int)threads, smem);
    if (e != cudaSuccess) return e;
    const uint64_t grid = copies * S.Gc;
    if (per_sm < 1 || grid > (uint64_t)per_sm * sm_count) return cudaErrorCooperativeLaunchTooLarge;
    e = cudaMemsetAsync(S.progress, 0, grid * sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    StripLaunch Sc = S;
    void* args[] = {&Sc};
    e = cudaLaunchCooperativeKernel((const void*)k_sweep_strips, dim3((uint32_t)grid), dim3(threads), args, smem, s);
    count_launch();
    return e;
}

// ---- double checkerboard with k hits per tile (Sec. 3.1, Fig. 5 right) ----
// One launch updates every T x T tile of one coarse colour ((tx + ty) mod 2)
// of a 2D ferromagnet in place: a CTA loads its tile with an 8-site halo as
// colour planes (the halo belongs to tiles of the other coarse colour, which
// no CTA of this launch writes), runs k full checkerboard sweeps of the tile
// interior -- sweep j with counter t0 + j, the random word of every site the
// plain sweep j would use -- and stores the interior back. The halo keeps
// each plane word a whole Philox call (4 same-colour sites, 8 columns).
template <uint32_t T, uint32_t NT>
__global__ void __launch_bounds__(NT) k_sweep_dcb(const __grid_constant__ TileLaunch P) {
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ __align__(16) uint32_t s_tbl[8];
    constexpr uint32_t Wd = T + 16, Wg = Wd >> 3, H = (Wd * Wd) >> 1, Tc = T >> 3;
    constexpr uint32_t U = T * Tc / NT;  // units per thread and half-sweep (NT is a multiple of Tc)
    static_assert(NT % Tc == 0 && (T * Tc) % NT == 0 && (U < 4 || U % 4 == 0), "tile / block shape");
    const uint32_t L = P.L, Lw = L >> 3;
    const uint32_t half_x = (L / T) >> 1;
    const uint32_t ty = blockIdx.x / half_x;
    const uint32_t tx = 2 * (blockIdx.x - ty * half_x) + ((ty + P.coarse) & 1u);
    const uint64_t copy = (uint64_t)P.copy0 + blockIdx.y;
    uint32_t inst, r;
    split_copy(copy, P.R, inst, r);
    int8_t* sp = P.dst + copy * (uint64_t)L * L;
    const uint32_t y0 = (ty * T + L - 8) % L;          // global row of window row 0
    const uint32_t xw0 = ((tx * T + L - 8) % L) >> 3;  // global 8-column chunk of window chunk 0
    uint32_t* pl = reinterpret_cast<uint32_t*>(smem);
    for (uint32_t idx = threadIdx.x; idx < Wd * Wg; idx += NT) {
        const uint32_t rr = idx / Wg, cx = idx - rr * Wg;
        uint32_t gy = y0 + rr, gc = xw0 + cx;
        if (gy >= L) gy -= L;
        if (gc >= Lw) gc -= Lw;
        const uint2 v = *reinterpret_cast<const uint2*>(sp + (uint64_t)gy * L + 8ull * gc);
        const uint32_t pe = gy & 1u;  // colour of the even columns of this row
        pl[pe * (H >> 2) + idx] = __byte_perm(v.x, v.y, 0x6420);
        pl[(pe ^ 1u) * (H >> 2) + idx] = __byte_perm(v.x, v.y, 0x7531);
    }
    if (threadIdx.x < 8) {
        const int d = 2 - (int)threadIdx.x;
        s_tbl[threadIdx.x] = d <= 0 ? 0xFFFFFFFFu : (d == 1 ? P.thr[0] : P.thr[1]);
    }
    __syncthreads();
    const uint8_t* tbl = reinterpret_cast<const uint8_t*>(s_tbl);
    const uint32_t k0 = (uint32_t)P.seed, k1 = (uint32_t)(P.seed >> 32);
    const uint32_t instance = P.inst_base + inst;
    int e = 0, m = 0;
    for (uint32_t s = 0; s < 2 * P.nsweeps; ++s) {
        const uint32_t colour = s & 1u, t = P.t0 + (s >> 1);
        const PhiloxFixed pf = philox_fix(t, r, c3_word(kPurposeMetro, colour, instance), k0, k1);
        // interior: window rows [8, 8 + T), chunks [1, 1 + T/8). Thread t keeps
        // chunk t % Tc and takes rows t / Tc + i NT/Tc, i < U, four at a time:
        // all four units are loaded and updated before any word is stored (rows
        // of one plane: none reads what another writes)
        uint32_t* own = pl + colour * (H >> 2);
        const uint32_t g = threadIdx.x % Tc, r0 = threadIdx.x / Tc;
#pragma unroll
        for (uint32_t base = 0; base < U; base += 4) {
            constexpr uint32_t G4 = U < 4 ? U : 4;
            uint32_t ii[G4], vv[G4];
#pragma unroll
            for (uint32_t k = 0; k < G4; ++k) {
                const uint32_t rr = r0 + (base + k) * (NT / Tc);
                const uint32_t q = (ty * T + rr) * Lw + tx * Tc + g;
                unit_split<2, false, false, false>(smem, nullptr, Wd, Wd * Wd, rr + 8, rr + 8, 0, g + 1, colour, pf,
                                                   tbl, true, e, m, q, &ii[k], &vv[k]);
            }
#pragma unroll
            for (uint32_t k = 0; k < G4; ++k) own[ii[k]] = vv[k];
        }
        __syncthreads();
    }
    for (uint32_t idx = threadIdx.x; idx < T * Tc; idx += NT) {
        const uint32_t rr = idx / Tc, cx = idx - rr * Tc;
        const uint32_t wrow = rr + 8, wc = cx + 1;
        const uint32_t gy = ty * T + rr, gx = tx * T + 8 * cx;
        const uint32_t pe = gy & 1u;
        const uint32_t ev = pl[pe * (H >> 2) + wrow * Wg + wc], od = pl[(pe ^ 1u) * (H >> 2) + wrow * Wg + wc];
        uint2 v;
        v.x = __byte_perm(ev, od, 0x5140);
        v.y = __byte_perm(ev, od, 0x7362);
        *reinterpret_cast<uint2*>(sp + (uint64_t)gy * L + gx) = v;
    }
}

template <uint32_t T, uint32_t NT>
static cudaError_t launch_dcb_t(const TileLaunch& P, uint64_t copies, cudaStream_t s) {
    const size_t smem = tile_smem_bytes(T);
    auto kern = k_sweep_dcb<T, NT>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const uint32_t tiles = (P.L / T) * (P.L / T) / 2;
    for (uint64_t c0 = 0; c0 < copies; c0 += 65535) {
        TileLaunch Q = P;
        Q.copy0 = (uint32_t)c0;
        const uint32_t nc = (uint32_t)((copies - c0) < 65535 ? (copies - c0) : 65535);
        kern<<<dim3(tiles, nc), NT, smem, s>>>(Q);
        count_launch();
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_sweep_dcb(const TileLaunch& P, uint64_t copies, cudaStream_t s) {
    if (P.src != P.dst || P.L % (2 * P.T) != 0) return cudaErrorInvalidValue;
    if (P.T == 32) return launch_dcb_t<32, 64>(P, copies, s);
    if (P.T == 64) return launch_dcb_t<64, 128>(P, copies, s);
    if (P.T == 128) return launch_dcb_t<128, 256>(P, copies, s);
    return cudaErrorInvalidValue;
}

}  // namespace gbmc
