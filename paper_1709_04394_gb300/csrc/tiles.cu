// tiles.cu -- checkerboard Metropolis sweeps of 2D ferromagnets too large for
// one CTA's shared memory (Sec. 3.1): halo tiles that reproduce the plain
// two-phase sweeps exactly, and the double checkerboard of Fig. 5 (right)
// with k sweeps per tile load.
#include "device.cuh"
#include "internal.h"
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
    const uint32_t inst = (uint32_t)(copy / P.R), r = (uint32_t)(copy - (uint64_t)inst * P.R);
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
    const uint32_t L = P.L, Lw = L >> 3;
    const uint32_t half_x = (L / T) >> 1;
    const uint32_t ty = blockIdx.x / half_x;
    const uint32_t tx = 2 * (blockIdx.x - ty * half_x) + ((ty + P.coarse) & 1u);
    const uint64_t copy = (uint64_t)P.copy0 + blockIdx.y;
    const uint32_t inst = (uint32_t)(copy / P.R), r = (uint32_t)(copy - (uint64_t)inst * P.R);
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
        // interior: window rows [8, 8 + T), chunks [1, 1 + T/8)
        for (uint32_t u = threadIdx.x; u < T * Tc; u += NT) {
            const uint32_t rr = u / Tc, g = u - rr * Tc;
            const uint32_t q = (ty * T + rr) * Lw + tx * Tc + g;
            unit_split<2, false, false>(smem, nullptr, Wd, Wd * Wd, rr + 8, rr + 8, 0, g + 1, colour, pf, tbl, true,
                                        e, m, q);
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
