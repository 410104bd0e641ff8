// dcb_bits.cu -- the double checkerboard of Sec. 3.1 (Fig. 5, right) with the
// tile held bit-sliced in registers: one bit per spin, one word per 32 sites
// of one colour in one row (the separate sub-lattice storage of Sec. 3.1 with
// multi-spin coding), so that the k sweeps of a tile load cost the Philox
// words and their threshold comparisons and little else.
//
// A launch updates every tile of one coarse colour ((tx + ty) & 1 == coarse)
// of every copy, k full sweeps each, in place: the tiles of a launch only
// read the fixed sites of the other coarse colour around them (the one-site
// halo: a row above and below, a column to the left and right). Lane l of
// warp w holds the rows y = (32 w + l) RPL + i, i < RPL, of its tile, both
// colours, WR = T / 64 words per row and colour: word v of colour c in row y
// holds the sites j = 32 v .. 32 v + 31 of colour c in that row (x = 2 j +
// ((y + c) & 1)), bit j - 32 v, 1 = down. Neighbours within a row are the
// other colour's word shifted by one site (its end bit from the halo column),
// those of rows y -/+ 1 the neighbouring lanes' words (warp ends: shared
// memory, filled with the halo rows or the next warp's edge rows).
//
// The sites use the Philox words of every other sweep kernel (colour rank k
// = y L / 2 + j of the site in the lattice, q = k >> 2, word k & 3; t = the
// call's sweep counter + the sweep within the tile load, as the byte-plane
// double checkerboard), so the spins are bit-identical to it.
#include "bits.cuh"
#include "check.cuh"
#include "device.cuh"
#include "internal.h"

namespace gbmc {

namespace {

// Warps per tile: one row per lane (64 x 64 tiles: two warps; 128 x 128: four).
constexpr uint32_t kWarps64 = 2, kWarps128 = 4;

// T: tile side (64 or 128); NW: warps per tile.
template <uint32_t T, uint32_t NW>
__global__ void __launch_bounds__(32 * NW) k_dcb_bits(const __grid_constant__ TileLaunch P) {
    constexpr uint32_t WR = T / 64;          // words per row and colour
    constexpr uint32_t RPL = T / (32 * NW);  // rows per lane
    constexpr uint32_t CH = T / 16;          // 16-byte chunks per tile row
    static_assert(WR >= 1 && RPL >= 1 && RPL * 32 * NW == T, "tile / block shape");
    // above[w]: the row over warp w's first row (w = 0: halo row -1, else warp
    // w - 1's last row); below[w]: the row under warp w's last row (w = NW - 1:
    // halo row T, else warp w + 1's first row). [colour][word]
    __shared__ __align__(16) uint32_t above[NW][2][WR];
    __shared__ __align__(16) uint32_t below[NW][2][WR];
    const uint32_t lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
    const uint32_t L = P.L;
    const uint32_t half_x = (L / T) >> 1;
    const uint32_t ty = blockIdx.x / half_x;
    const uint32_t tx = 2 * (blockIdx.x - ty * half_x) + ((ty + P.coarse) & 1u);
    const uint64_t copy = (uint64_t)P.copy0 + blockIdx.y;
    uint32_t inst, r;
    split_copy(copy, P.R, inst, r);
    const uint64_t LL = (uint64_t)L * L;
    int8_t* sp = P.dst + copy * LL;
    const uint32_t x0 = tx * T, yt = ty * T;
    const uint32_t xl = (x0 + L - 1u) % L, xr = (x0 + T) % L;  // halo columns

    // ---- load: rows of int8 -> bit words. Chunk m of a row (16 sites) gives 8
    // even-x and 8 odd-x sites: bits 8 m .. 8 m + 7 of the two colours' row
    // (even-x sites have colour y & 1) ----
    uint32_t s[RPL][2][WR];  // spins, 1 = down
    uint32_t hl[RPL], hr[RPL];  // down bits of the halo columns x0 - 1 and x0 + T
#pragma unroll
    for (uint32_t i = 0; i < RPL; ++i) {
        const uint32_t yl = (32u * wid + lane) * RPL + i, gy = yt + yl;
        const int8_t* row = sp + (uint64_t)GBMC_IDX(gy, L) * L;
        uint32_t ev[WR], od[WR];
#pragma unroll
        for (uint32_t v = 0; v < WR; ++v) ev[v] = od[v] = 0u;
#pragma unroll
        for (uint32_t m = 0; m < CH; ++m) {
            const uint4 c = *reinterpret_cast<const uint4*>(row + GBMC_IDX(x0 + 16u * m, L));
            uint32_t e0, o0, e1, o1;
            pack8(c.x, c.y, e0, o0);
            pack8(c.z, c.w, e1, o1);
            ev[m >> 2] |= (e0 | (e1 << 4)) << (8u * (m & 3u));
            od[m >> 2] |= (o0 | (o1 << 4)) << (8u * (m & 3u));
        }
        const uint32_t ce = yl & 1u;
#pragma unroll
        for (uint32_t v = 0; v < WR; ++v) {
            s[i][0][v] = ce ? od[v] : ev[v];
            s[i][1][v] = ce ? ev[v] : od[v];
        }
        hl[i] = row[GBMC_IDX(xl, L)] < 0 ? 1u : 0u;
        hr[i] = row[GBMC_IDX(xr, L)] < 0 ? 1u : 0u;
    }
    // halo rows -1 (even-x sites: colour 1) and T (colour 0) through the byte
    // image of the shared rows: byte m of a colour's row = chunk m's 8 bits
    if (wid == 0 && lane < CH) {
        const uint32_t gy = (yt + L - 1u) % L;
        const uint4 c = *reinterpret_cast<const uint4*>(sp + (uint64_t)gy * L + GBMC_IDX(x0 + 16u * lane, L));
        uint32_t e0, o0, e1, o1;
        pack8(c.x, c.y, e0, o0);
        pack8(c.z, c.w, e1, o1);
        uint8_t* b = reinterpret_cast<uint8_t*>(above[0]);
        b[GBMC_IDX(4u * WR + lane, 8u * WR)] = (uint8_t)(e0 | (e1 << 4));  // colour 1
        b[GBMC_IDX(lane, 8u * WR)] = (uint8_t)(o0 | (o1 << 4));            // colour 0
    }
    if (wid == NW - 1u && lane >= 32u - CH) {
        const uint32_t m = lane - (32u - CH);
        const uint32_t gy = (yt + T) % L;
        const uint4 c = *reinterpret_cast<const uint4*>(sp + (uint64_t)gy * L + GBMC_IDX(x0 + 16u * m, L));
        uint32_t e0, o0, e1, o1;
        pack8(c.x, c.y, e0, o0);
        pack8(c.z, c.w, e1, o1);
        uint8_t* b = reinterpret_cast<uint8_t*>(below[NW - 1]);
        b[GBMC_IDX(m, 8u * WR)] = (uint8_t)(e0 | (e1 << 4));            // colour 0
        b[GBMC_IDX(4u * WR + m, 8u * WR)] = (uint8_t)(o0 | (o1 << 4));  // colour 1
    }
    // edge rows between the warps of the tile, both colours
    if (NW > 1) {
#pragma unroll
        for (uint32_t c = 0; c < 2; ++c)
#pragma unroll
            for (uint32_t v = 0; v < WR; ++v) {
                if (lane == 31u && wid + 1u < NW) above[wid + 1u][c][v] = s[RPL - 1][c][v];
                if (lane == 0u && wid > 0u) below[wid - 1u][c][v] = s[0][c][v];
            }
    }
    __syncthreads();

    const uint32_t k0 = (uint32_t)P.seed, k1 = (uint32_t)(P.seed >> 32);
    const uint32_t instance = P.inst_base + inst;
    const uint32_t T4 = P.thr[0], T8 = P.thr[1];
    const uint32_t Lq = L >> 3;  // Philox counters per row (4 sites of one colour each)
#pragma unroll 1
    for (uint32_t sw = 0; sw < P.nsweeps; ++sw) {
        const uint32_t t = P.t0 + sw;
#pragma unroll
        for (uint32_t c = 0; c < 2; ++c) {
            const uint32_t o = c ^ 1u;
            const PhiloxFixed pf = philox_fix(t, r, c3_word(kPurposeMetro, c, instance), k0, k1);
            // rows over and under this lane's rows (the other colour)
            uint32_t up0[WR], dnL[WR];
#pragma unroll
            for (uint32_t v = 0; v < WR; ++v) {
                const uint32_t a = __shfl_up_sync(0xffffffffu, s[RPL - 1][o][v], 1);
                const uint32_t b = __shfl_down_sync(0xffffffffu, s[0][o][v], 1);
                up0[v] = lane == 0u ? above[wid][o][v] : a;
                dnL[v] = lane == 31u ? below[wid][o][v] : b;
            }
            uint32_t nw[RPL][WR];
#pragma unroll
            for (uint32_t i = 0; i < RPL; ++i) {
                const uint32_t yl = (32u * wid + lane) * RPL + i;
                // sites of colour c in row y have odd x iff (y + c) odd: their
                // in-row neighbour off the same j is j + 1, else j - 1
                const bool odd = ((yl + c) & 1u) != 0u;
                const uint32_t qrow = (yt + yl) * Lq + (x0 >> 3);
#pragma unroll
                for (uint32_t v = 0; v < WR; ++v) {
                    const uint32_t up = i > 0 ? s[i - 1][o][v] : up0[v];
                    const uint32_t dn = i + 1 < RPL ? s[i + 1][o][v] : dnL[v];
                    const uint32_t same = s[i][o][v];
                    const uint32_t nxt = v + 1 < WR ? s[i][o][v + 1 < WR ? v + 1 : v] : hr[i];
                    const uint32_t prv = v > 0 ? s[i][o][v > 0 ? v - 1 : 0] : hl[i] << 31;
                    const uint32_t side = odd ? __funnelshift_r(same, nxt, 1) : __funnelshift_l(prv, same, 1);
                    nw[i][v] = bp_word_update(s[i][c][v], up, dn, same, side, pf, qrow + 8u * v, T4, T8);
                }
            }
#pragma unroll
            for (uint32_t i = 0; i < RPL; ++i)
#pragma unroll
                for (uint32_t v = 0; v < WR; ++v) s[i][c][v] = nw[i][v];
            if (NW > 1) {
                // hand the new edge rows of colour c to the neighbouring warps;
                // the next half-sweep reads only colour c, this one read only
                // colour o, so one barrier per half-sweep orders both
#pragma unroll
                for (uint32_t v = 0; v < WR; ++v) {
                    if (lane == 31u && wid + 1u < NW) above[wid + 1u][c][v] = s[RPL - 1][c][v];
                    if (lane == 0u && wid > 0u) below[wid - 1u][c][v] = s[0][c][v];
                }
                __syncthreads();
            }
        }
    }

    // ---- store: bit words -> int8 rows (the tile interior only) ----
#pragma unroll
    for (uint32_t i = 0; i < RPL; ++i) {
        const uint32_t yl = (32u * wid + lane) * RPL + i, gy = yt + yl;
        int8_t* row = sp + (uint64_t)GBMC_IDX(gy, L) * L;
        const uint32_t ce = yl & 1u;
#pragma unroll
        for (uint32_t m = 0; m < CH; ++m) {
            const uint32_t sh = 8u * (m & 3u);
            const uint32_t ev = (s[i][ce][m >> 2] >> sh) & 0xFFu, od = (s[i][ce ^ 1u][m >> 2] >> sh) & 0xFFu;
            const uint2 lo = unpack8(ev & 15u, od & 15u), hi = unpack8(ev >> 4, od >> 4);
            *reinterpret_cast<uint4*>(row + GBMC_IDX(x0 + 16u * m, L)) = make_uint4(lo.x, lo.y, hi.x, hi.y);
        }
    }
}

template <uint32_t T, uint32_t NW>
cudaError_t launch_dcb_bits_t(const TileLaunch& P, uint64_t copies, cudaStream_t st) {
    const uint32_t tiles = (P.L / T) * (P.L / T) / 2;
    for (uint64_t c0 = 0; c0 < copies; c0 += 65535) {
        TileLaunch Q = P;
        Q.copy0 = (uint32_t)c0;
        const uint32_t nc = (uint32_t)((copies - c0) < 65535 ? (copies - c0) : 65535);
        k_dcb_bits<T, NW><<<dim3(tiles, nc), 32 * NW, 0, st>>>(Q);
        count_launch();
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

bool dcb_bits_supported(uint32_t T) { return T == 64 || T == 128; }

cudaError_t launch_dcb_bits(const TileLaunch& P, uint64_t copies, cudaStream_t st) {
    if (P.src != P.dst || !dcb_bits_supported(P.T) || P.L % (2 * P.T) != 0 || P.nsweeps == 0)
        return cudaErrorInvalidValue;
    if (P.T == 64) return launch_dcb_bits_t<64, kWarps64>(P, copies, st);
    return launch_dcb_bits_t<128, kWarps128>(P, copies, st);
}

}  // namespace gbmc
