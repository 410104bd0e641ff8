// dcb_bits.cu -- the double checkerboard of Sec. 3.1 (Fig. 5, right) with the
// tiles held bit-sliced in registers: one bit per spin, one word per 32 sites
// of one colour in one row (the separate sub-lattice storage of Sec. 3.1 with
// multi-spin coding), so that the k sweeps of a tile visit cost the Philox
// words and their threshold comparisons and little else.
//
// A tile of coarse colour b ((tx + ty) & 1 == b) takes k full sweeps while
// the tiles of the other coarse colour around it stay fixed: it reads only
// their sites next to it (the one-site halo: a row above and below, a column
// to the left and right). Lane l of warp w holds the rows y = (32 w + l) RPL
// + i, i < RPL, of a tile, both colours, WR = T / 64 words per row and colour:
// word v of colour c in row y holds the sites j = 32 v .. 32 v + 31 of colour
// c in that row (x = 2 j + ((y + c) & 1)), bit j - 32 v, 1 = down. Neighbours
// within a row are the other colour's word shifted by one site (its end bit
// from the halo column), those of rows y -/+ 1 the neighbouring lanes' words
// (warp ends: shared memory, filled with the halo rows or the next warp's
// edge rows).
//
//  * k_dcb_bits: one launch per coarse colour and round; every tile of that
//    colour is loaded from the int8 lattice with its halo, swept and stored.
//  * k_dcb_resident: every round of a call in one cooperative launch. A CTA
//    holds one tile of each coarse colour in registers for the whole call and
//    trades only tile edges (top and bottom rows, left and right columns as
//    bit masks) through global memory, each tile announcing its edges of a
//    round by a progress counter that its four neighbours wait for (a bounded
//    wait, as in the strip-resident sweeps).
//
// The sites use the Philox words of every other sweep kernel (colour rank k
// = y L / 2 + j of the site in the lattice, q = k >> 2, word k & 3; t = the
// call's sweep counter + the sweep within the round), so the spins are
// bit-identical to the byte-plane double checkerboard and to the oracle.
#include "bits.cuh"
#include "check.cuh"
#include "device.cuh"
#include "internal.h"
#include "strips.cuh"

namespace gbmc {

namespace {

// Warps per tile: one row per lane (64 x 64 tiles: two warps; 128 x 128: four).
constexpr uint32_t kWarps64 = 2, kWarps128 = 4;

template <uint32_t T, uint32_t NW>
struct Shape {
    static constexpr uint32_t WR = T / 64;          // words per row and colour
    static constexpr uint32_t RPL = T / (32 * NW);  // rows per lane
    static constexpr uint32_t CH = T / 16;          // 16-byte chunks per tile row
    static constexpr uint32_t MW = T / 32;          // words of a column mask
    static constexpr uint32_t EW = 4 * WR + 2 * MW; // edge words of a tile: top, bottom row, left, right column
    static_assert(WR >= 1 && RPL >= 1 && RPL * 32 * NW == T, "tile / block shape");
};

// The tile rows of this lane (tile origin x0, yt) from the int8 lattice sp
// into bit words s[i][colour][word]. Chunk m of a row (16 sites) gives 8
// even-x and 8 odd-x sites: bits 8 m .. 8 m + 7 of the two colours' row
// (even-x sites have colour y & 1).
template <uint32_t T, uint32_t NW>
__device__ __forceinline__ void load_rows(const int8_t* sp, uint32_t L, uint32_t x0, uint32_t yt, uint32_t lane,
                                          uint32_t wid, uint32_t (&s)[Shape<T, NW>::RPL][2][Shape<T, NW>::WR]) {
    using S = Shape<T, NW>;
#pragma unroll
    for (uint32_t i = 0; i < S::RPL; ++i) {
        const uint32_t yl = (32u * wid + lane) * S::RPL + i;
        const int8_t* row = sp + (uint64_t)GBMC_IDX(yt + yl, L) * L;
        uint32_t ev[S::WR], od[S::WR];
#pragma unroll
        for (uint32_t v = 0; v < S::WR; ++v) ev[v] = od[v] = 0u;
#pragma unroll
        for (uint32_t m = 0; m < S::CH; ++m) {
            const uint4 c = *reinterpret_cast<const uint4*>(row + GBMC_IDX(x0 + 16u * m, L));
            uint32_t e0, o0, e1, o1;
            pack8(c.x, c.y, e0, o0);
            pack8(c.z, c.w, e1, o1);
            ev[m >> 2] |= (e0 | (e1 << 4)) << (8u * (m & 3u));
            od[m >> 2] |= (o0 | (o1 << 4)) << (8u * (m & 3u));
        }
        const uint32_t ce = yl & 1u;
#pragma unroll
        for (uint32_t v = 0; v < S::WR; ++v) {
            s[i][0][v] = ce ? od[v] : ev[v];
            s[i][1][v] = ce ? ev[v] : od[v];
        }
    }
}

// The inverse: this lane's tile rows back to the int8 lattice.
template <uint32_t T, uint32_t NW>
__device__ __forceinline__ void store_rows(int8_t* sp, uint32_t L, uint32_t x0, uint32_t yt, uint32_t lane,
                                           uint32_t wid, const uint32_t (&s)[Shape<T, NW>::RPL][2][Shape<T, NW>::WR]) {
    using S = Shape<T, NW>;
#pragma unroll
    for (uint32_t i = 0; i < S::RPL; ++i) {
        const uint32_t yl = (32u * wid + lane) * S::RPL + i;
        int8_t* row = sp + (uint64_t)GBMC_IDX(yt + yl, L) * L;
        const uint32_t ce = yl & 1u;
#pragma unroll
        for (uint32_t m = 0; m < S::CH; ++m) {
            const uint32_t sh = 8u * (m & 3u);
            const uint32_t ev = (s[i][ce][m >> 2] >> sh) & 0xFFu, od = (s[i][ce ^ 1u][m >> 2] >> sh) & 0xFFu;
            const uint2 lo = unpack8(ev & 15u, od & 15u), hi = unpack8(ev >> 4, od >> 4);
            *reinterpret_cast<uint4*>(row + GBMC_IDX(x0 + 16u * m, L)) = make_uint4(lo.x, lo.y, hi.x, hi.y);
        }
    }
}

// load_rows / store_rows for one row per lane, staged through a byte image
// of the warp's 32 rows in shared memory (img: [colour][row][word]) so that
// the global accesses are whole rows: in step m, lane l moves chunk l % CH of
// row m (32 / CH) + l / CH.
template <uint32_t T, uint32_t NW>
__device__ __forceinline__ void load_rows_staged(const int8_t* sp, uint32_t L, uint32_t x0, uint32_t yt,
                                                 uint32_t lane, uint32_t wid,
                                                 uint32_t (&img)[2][32][Shape<T, NW>::WR],
                                                 uint32_t (&s)[1][2][Shape<T, NW>::WR]) {
    using S = Shape<T, NW>;
    constexpr uint32_t CH = S::CH, WR = S::WR, RPI = 32 / CH;
    static_assert(S::RPL == 1, "one row per lane");
    uint8_t* b = reinterpret_cast<uint8_t*>(&img[0][0][0]);
    const uint32_t ch = lane % CH, rsub = lane / CH;
#pragma unroll
    for (uint32_t m = 0; m < CH; ++m) {
        const uint32_t rw = m * RPI + rsub, yl = 32u * wid + rw;
        const uint4 c = *reinterpret_cast<const uint4*>(sp + (uint64_t)GBMC_IDX(yt + yl, L) * L +
                                                        GBMC_IDX(x0 + 16u * ch, L));
        uint32_t e0, o0, e1, o1;
        pack8(c.x, c.y, e0, o0);
        pack8(c.z, c.w, e1, o1);
        const uint32_t ce = yl & 1u;  // colour of the even-x sites
        b[GBMC_IDX((ce * 32u + rw) * 4u * WR + ch, 256u * WR)] = (uint8_t)(e0 | (e1 << 4));
        b[GBMC_IDX(((ce ^ 1u) * 32u + rw) * 4u * WR + ch, 256u * WR)] = (uint8_t)(o0 | (o1 << 4));
    }
    __syncwarp();
#pragma unroll
    for (uint32_t c = 0; c < 2; ++c)
#pragma unroll
        for (uint32_t v = 0; v < WR; ++v) s[0][c][v] = img[c][lane][v];
    __syncwarp();
}

template <uint32_t T, uint32_t NW>
__device__ __forceinline__ void store_rows_staged(int8_t* sp, uint32_t L, uint32_t x0, uint32_t yt, uint32_t lane,
                                                  uint32_t wid, uint32_t (&img)[2][32][Shape<T, NW>::WR],
                                                  const uint32_t (&s)[1][2][Shape<T, NW>::WR]) {
    using S = Shape<T, NW>;
    constexpr uint32_t CH = S::CH, WR = S::WR, RPI = 32 / CH;
    static_assert(S::RPL == 1, "one row per lane");
#pragma unroll
    for (uint32_t c = 0; c < 2; ++c)
#pragma unroll
        for (uint32_t v = 0; v < WR; ++v) img[c][lane][v] = s[0][c][v];
    __syncwarp();
    const uint8_t* b = reinterpret_cast<const uint8_t*>(&img[0][0][0]);
    const uint32_t ch = lane % CH, rsub = lane / CH;
#pragma unroll
    for (uint32_t m = 0; m < CH; ++m) {
        const uint32_t rw = m * RPI + rsub, yl = 32u * wid + rw;
        const uint32_t ce = yl & 1u;
        const uint32_t ev = b[GBMC_IDX((ce * 32u + rw) * 4u * WR + ch, 256u * WR)];
        const uint32_t od = b[GBMC_IDX(((ce ^ 1u) * 32u + rw) * 4u * WR + ch, 256u * WR)];
        const uint2 lo = unpack8(ev & 15u, od & 15u), hi = unpack8(ev >> 4, od >> 4);
        *reinterpret_cast<uint4*>(sp + (uint64_t)GBMC_IDX(yt + yl, L) * L + GBMC_IDX(x0 + 16u * ch, L)) =
            make_uint4(lo.x, lo.y, hi.x, hi.y);
    }
}

// Both warp-end rows of every warp but the tile's first (last) one into
// above (below) of its neighbour warp, both colours.
template <uint32_t T, uint32_t NW>
__device__ __forceinline__ void share_warp_edges(const uint32_t (&s)[Shape<T, NW>::RPL][2][Shape<T, NW>::WR],
                                                 uint32_t (&above)[NW][2][Shape<T, NW>::WR],
                                                 uint32_t (&below)[NW][2][Shape<T, NW>::WR], uint32_t lane,
                                                 uint32_t wid) {
    using S = Shape<T, NW>;
    if (NW > 1) {
#pragma unroll
        for (uint32_t c = 0; c < 2; ++c)
#pragma unroll
            for (uint32_t v = 0; v < S::WR; ++v) {
                if (lane == 31u && wid + 1u < NW) above[wid + 1u][c][v] = s[S::RPL - 1][c][v];
                if (lane == 0u && wid > 0u) below[wid - 1u][c][v] = s[0][c][v];
            }
    }
}

// k sweeps of one tile (rows yt.., columns x0..; its halo rows in above[0] and
// below[NW - 1], its halo column bits in hl, hr; sweep counters t0 ..), the
// colour-c half-sweep reading only colour 1 - c. Ends with the block's
// threads synchronised.
template <uint32_t T, uint32_t NW>
__device__ __forceinline__ void tile_sweeps(uint32_t (&s)[Shape<T, NW>::RPL][2][Shape<T, NW>::WR],
                                            const uint32_t (&hl)[Shape<T, NW>::RPL],
                                            const uint32_t (&hr)[Shape<T, NW>::RPL],
                                            uint32_t (&above)[NW][2][Shape<T, NW>::WR],
                                            uint32_t (&below)[NW][2][Shape<T, NW>::WR], uint32_t lane, uint32_t wid,
                                            uint32_t L, uint32_t x0, uint32_t yt, uint32_t t0, uint32_t nsweeps,
                                            uint32_t r, uint32_t instance, uint64_t seed, uint32_t T4, uint32_t T8) {
    using S = Shape<T, NW>;
    constexpr uint32_t WR = S::WR, RPL = S::RPL;
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    const uint32_t Lq = L >> 3;  // Philox counters per row (4 sites of one colour each)
#pragma unroll 1
    for (uint32_t sw = 0; sw < nsweeps; ++sw) {
        const uint32_t t = t0 + sw;
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
                    const uint32_t up = i > 0 ? s[i > 0 ? i - 1 : 0][o][v] : up0[v];
                    const uint32_t dn = i + 1 < RPL ? s[i + 1 < RPL ? i + 1 : i][o][v] : dnL[v];
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
    if (NW == 1) __syncthreads();
}

// ---- one launch per coarse colour and round ----

// T: tile side (64 or 128); NW: warps per tile.
template <uint32_t T, uint32_t NW>
__global__ void __launch_bounds__(32 * NW, T == 64 ? 16 : 4) k_dcb_bits(const __grid_constant__ TileLaunch P) {
    using S = Shape<T, NW>;
    constexpr uint32_t WR = S::WR, RPL = S::RPL, CH = S::CH;
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
    int8_t* sp = P.dst + copy * ((uint64_t)L * L);
    const uint32_t x0 = tx * T, yt = ty * T;
    const uint32_t xl = (x0 + L - 1u) % L, xr = (x0 + T) % L;  // halo columns

    __shared__ __align__(16) uint32_t img[NW][2][32][WR];  // staging of the warps' rows
    uint32_t s[RPL][2][WR];     // spins, 1 = down
    uint32_t hl[RPL], hr[RPL];  // down bits of the halo columns x0 - 1 and x0 + T
    load_rows_staged<T, NW>(sp, L, x0, yt, lane, wid, img[wid], s);
#pragma unroll
    for (uint32_t i = 0; i < RPL; ++i) {
        const int8_t* row = sp + (uint64_t)GBMC_IDX(yt + (32u * wid + lane) * RPL + i, L) * L;
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
    share_warp_edges<T, NW>(s, above, below, lane, wid);
    __syncthreads();
    tile_sweeps<T, NW>(s, hl, hr, above, below, lane, wid, L, x0, yt, P.t0, P.nsweeps, r, P.inst_base + inst, P.seed,
                       P.thr[0], P.thr[1]);
    store_rows_staged<T, NW>(sp, L, x0, yt, lane, wid, img[wid], s);
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

// ---- every round of a call in one launch ----

// Tile edges, per tile EW words: the top row (colour c, word v at c WR + v),
// the bottom row (2 WR + c WR + v), the left column x0 (4 WR + y / 32: bit
// y % 32 = site (x0, y) is down) and the right column x0 + T - 1 (4 WR + MW +
// y / 32). Written by one tile's CTA, read through L2 by its neighbours'.
template <uint32_t T, uint32_t NW>
__device__ __forceinline__ void publish_edges(uint32_t* e, const uint32_t (&s)[1][2][Shape<T, NW>::WR],
                                              uint32_t lane, uint32_t wid) {
    using S = Shape<T, NW>;
    constexpr uint32_t WR = S::WR;
    const uint32_t yl = 32u * wid + lane, ce = yl & 1u;
    // site x0 of row y: colour y & 1, word 0 bit 0; x0 + T - 1: the other colour, word WR - 1 bit 31
    const uint32_t lm = __ballot_sync(0xffffffffu, (s[0][ce][0] & 1u) != 0u);
    const uint32_t rm = __ballot_sync(0xffffffffu, (s[0][ce ^ 1u][WR - 1] >> 31) != 0u);
    if (lane == 0u) {
        __stcg(e + GBMC_IDX(4u * WR + wid, S::EW), lm);
        __stcg(e + GBMC_IDX(4u * WR + S::MW + wid, S::EW), rm);
    }
#pragma unroll
    for (uint32_t c = 0; c < 2; ++c)
#pragma unroll
        for (uint32_t v = 0; v < WR; ++v) {
            if (wid == 0u && lane == 0u) __stcg(e + GBMC_IDX(c * WR + v, S::EW), s[0][c][v]);
            if (wid == NW - 1u && lane == 31u) __stcg(e + GBMC_IDX(2u * WR + c * WR + v, S::EW), s[0][c][v]);
        }
}

template <uint32_t T, uint32_t NW>
__global__ void __launch_bounds__(32 * NW, T == 64 ? 14 : 4) k_dcb_resident(const __grid_constant__ DcbResident D) {
    using S = Shape<T, NW>;
    constexpr uint32_t WR = S::WR, EW = S::EW, MW = S::MW;
    static_assert(S::RPL == 1, "one row per lane (the column masks are warp ballots)");
    __shared__ __align__(16) uint32_t above[NW][2][WR];
    __shared__ __align__(16) uint32_t below[NW][2][WR];
    __shared__ uint32_t park[2][2][WR][32 * NW];  // [tile][colour][word][thread]
    __shared__ int s_ok;
    const uint32_t lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
    const uint32_t L = D.L, nt = L / T, pairs = nt >> 1;
    const uint32_t ty = blockIdx.x / pairs, px = blockIdx.x - ty * pairs;
    const uint64_t copy = blockIdx.y;
    uint32_t inst, r;
    split_copy(copy, D.R, inst, r);
    int8_t* sp = D.spins + copy * ((uint64_t)L * L);
    const uint32_t tiles = nt * nt;
    uint32_t* eb = D.edges + copy * ((uint64_t)tiles * EW);
    unsigned int* pg = D.progress + copy * (uint64_t)tiles;
    const uint32_t yt = ty * T;
    // the CTA's two tiles in row ty: coarse colour 0, then 1
    const uint32_t tx0 = 2u * px + (ty & 1u), tx1 = 2u * px + 1u - (ty & 1u);
    const uint32_t tyu = ty == 0 ? nt - 1u : ty - 1u, tyd = ty + 1u == nt ? 0u : ty + 1u;

    // the tile not being swept waits in shared memory (one slot per thread)
    uint32_t s[1][2][WR];
    load_rows<T, NW>(sp, L, tx1 * T, yt, lane, wid, s);
#pragma unroll
    for (uint32_t c = 0; c < 2; ++c)
#pragma unroll
        for (uint32_t v = 0; v < WR; ++v) park[1][c][v][threadIdx.x] = s[0][c][v];
    if (threadIdx.x == 0) s_ok = 1;
    // the coarse-1 tile's edges before any sweep: the halo of round 0's coarse-0 tiles
    publish_edges<T, NW>(eb + (uint64_t)GBMC_IDX(ty * nt + tx1, tiles) * EW, s, lane, wid);
    load_rows<T, NW>(sp, L, tx0 * T, yt, lane, wid, s);
#pragma unroll
    for (uint32_t c = 0; c < 2; ++c)
#pragma unroll
        for (uint32_t v = 0; v < WR; ++v) park[0][c][v][threadIdx.x] = s[0][c][v];
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicExch(pg + GBMC_IDX(ty * nt + tx1, tiles), 1u);
    }
    const uint32_t instance = D.inst_base + inst;
    bool ok = true;
#pragma unroll 1
    for (uint32_t m = 0; m < D.n_rounds && ok; ++m) {
#pragma unroll 1
        for (uint32_t b = 0; b < 2; ++b) {
            const uint32_t tx = (b ? tx1 : tx0), x0 = tx * T;
            const uint32_t txl = tx == 0 ? nt - 1u : tx - 1u, txr = tx + 1u == nt ? 0u : tx + 1u;
            const uint32_t tl = ty * nt + txl, tr = ty * nt + txr, tu = tyu * nt + tx, td = tyd * nt + tx;
            // progress of a tile: 1 = its edges before any sweep (coarse colour 1),
            // m + 2 = after round m. Round m of coarse colour b needs the other
            // colour's neighbours at m + 1 + b.
            const uint32_t need = m + 1u + b + D.phantom;
            if (threadIdx.x == 0 &&
                !(strip_wait(pg + GBMC_IDX(tl, tiles), pg + GBMC_IDX(tr, tiles), need, D.err, D.budget) &&
                  strip_wait(pg + GBMC_IDX(tu, tiles), pg + GBMC_IDX(td, tiles), need, D.err, D.budget)))
                s_ok = 0;
            __syncthreads();
            if (!s_ok) {
                ok = false;
                break;
            }
#pragma unroll
            for (uint32_t c = 0; c < 2; ++c)
#pragma unroll
                for (uint32_t v = 0; v < WR; ++v) s[0][c][v] = park[b][c][v][threadIdx.x];
            // the halo from the neighbours' edges (written by other CTAs: read from L2)
            if (wid == 0u && lane < 2u * WR)
                (&above[0][0][0])[lane] = __ldcg(eb + (uint64_t)GBMC_IDX(tu, tiles) * EW + 2u * WR + lane);
            if (wid == NW - 1u && lane >= 32u - 2u * WR)
                (&below[NW - 1][0][0])[lane - (32u - 2u * WR)] =
                    __ldcg(eb + (uint64_t)GBMC_IDX(td, tiles) * EW + (lane - (32u - 2u * WR)));
            uint32_t hl[1], hr[1];
            hl[0] = (__ldcg(eb + (uint64_t)GBMC_IDX(tl, tiles) * EW + 4u * WR + MW + wid) >> lane) & 1u;
            hr[0] = (__ldcg(eb + (uint64_t)GBMC_IDX(tr, tiles) * EW + 4u * WR + wid) >> lane) & 1u;
            share_warp_edges<T, NW>(s, above, below, lane, wid);
            __syncthreads();
            tile_sweeps<T, NW>(s, hl, hr, above, below, lane, wid, L, x0, yt, D.t0 + m * D.k, D.k, r, instance,
                               D.seed, D.thr[0], D.thr[1]);
            publish_edges<T, NW>(eb + (uint64_t)GBMC_IDX(ty * nt + tx, tiles) * EW, s, lane, wid);
#pragma unroll
            for (uint32_t c = 0; c < 2; ++c)
#pragma unroll
                for (uint32_t v = 0; v < WR; ++v) park[b][c][v][threadIdx.x] = s[0][c][v];
            __syncthreads();  // every edge store of the CTA before the announcement
            if (threadIdx.x == 0) {
                __threadfence();
                atomicExch(pg + GBMC_IDX(ty * nt + tx, tiles), m + 2u);
            }
        }
    }
    if (!ok) return;  // a wait ran out: the error is raised, the lattice keeps its old spins here
#pragma unroll 1
    for (uint32_t b = 0; b < 2; ++b) {
#pragma unroll
        for (uint32_t c = 0; c < 2; ++c)
#pragma unroll
            for (uint32_t v = 0; v < WR; ++v) s[0][c][v] = park[b][c][v][threadIdx.x];
        store_rows<T, NW>(sp, L, (b ? tx1 : tx0) * T, yt, lane, wid, s);
    }
}

template <uint32_t T, uint32_t NW>
bool resident_fits_t(uint32_t L, uint64_t copies, int sm_count) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dcb_resident<T, NW>, 32 * NW, 0) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    const uint64_t grid = (uint64_t)(L / T) * (L / T) / 2 * copies;
    return per_sm >= 1 && grid <= (uint64_t)per_sm * sm_count;
}

template <uint32_t T, uint32_t NW>
cudaError_t launch_resident_t(const DcbResident& D, uint64_t copies, cudaStream_t st) {
    const uint32_t nt = D.L / T;
    cudaError_t e = cudaMemsetAsync(D.progress, 0, (uint64_t)nt * nt * copies * sizeof(unsigned int), st);
    if (e != cudaSuccess) return e;
    DcbResident Dc = D;
    void* args[] = {&Dc};
    e = cudaLaunchCooperativeKernel((const void*)k_dcb_resident<T, NW>, dim3(nt * nt / 2, (uint32_t)copies),
                                    dim3(32 * NW), args, 0, st);
    count_launch();
    return e;
}

}  // namespace

bool dcb_bits_supported(uint32_t T) { return T == 64 || T == 128; }

cudaError_t launch_dcb_bits(const TileLaunch& P, uint64_t copies, cudaStream_t st) {
    if (P.src != P.dst || !dcb_bits_supported(P.T) || P.L % (2 * P.T) != 0 || P.nsweeps == 0)
        return cudaErrorInvalidValue;
    if (P.T == 64) return launch_dcb_bits_t<64, kWarps64>(P, copies, st);
    return launch_dcb_bits_t<128, kWarps128>(P, copies, st);
}

size_t dcb_resident_bytes(uint32_t L, uint32_t T, uint64_t copies) {
    const uint64_t tiles = (uint64_t)(L / T) * (L / T) * copies;
    return (size_t)(tiles * (T / 8 + 1) * sizeof(uint32_t));  // T / 8 edge words and a progress counter
}

bool dcb_resident_fits(uint32_t L, uint32_t T, uint64_t copies, int sm_count) {
    if (!dcb_bits_supported(T) || L % (2 * T) != 0 || copies == 0 || copies > 65535) return false;
    if (T == 64) return resident_fits_t<64, kWarps64>(L, copies, sm_count);
    return resident_fits_t<128, kWarps128>(L, copies, sm_count);
}

cudaError_t launch_dcb_resident(const DcbResident& D, uint64_t copies, cudaStream_t st) {
    if (!dcb_bits_supported(D.T) || D.L % (2 * D.T) != 0 || D.k == 0 || copies == 0 || copies > 65535)
        return cudaErrorInvalidValue;
    if (D.T == 64) return launch_resident_t<64, kWarps64>(D, copies, st);
    return launch_resident_t<128, kWarps128>(D, copies, st);
}

}  // namespace gbmc
