// bitsweep.cu -- checkerboard Metropolis sweeps (Sec. 3.1, Eq. (8)) of copies
// held bit-sliced on chip: one bit per spin in per-colour planes (the separate
// sub-lattice storage of Sec. 3.1 with multi-spin coding of the sites), so that
// the neighbour count of 32 sites costs a handful of word operations and the
// per-site work is the Philox word and its threshold comparisons.
//
// The population stays in the int8 layout of the ABI in global memory; each
// warp converts its copy to bit planes on load (through the resampling gather
// of Sec. 5.4 when a parent map is given) and back on store. The sites use the
// same Philox words as every other sweep kernel (colour rank k of a site, q =
// k >> 2, word k & 3), so the spins are bit-identical to theirs.
//
//  * k_sweep_bits2: 2D ferromagnet, L in {16, 32, 64, 128, 256}. The copy in
//    shared memory, each colour plane as N / 64 words of 32 consecutive colour
//    ranks: for L >= 64 plane c, row y, word w = the sites j = 32 w .. 32 w +
//    31 of colour c in row y (x = 2 j + ((y + c) & 1)), bit j - 32 w; for
//    L = 32 (16) a word holds 2 (4) rows of L / 2 sites. One warp per copy for
//    L >= 64, one lane per word and 2 (8) copies per warp for L = 32 (16). No
//    block-wide barrier: the warps of a block are independent.
//  * k_sweep_bits3: 3D lattices with L = 8 (ferromagnet or +-J spin glass,
//    Sec. 6). Eight lanes per copy, four copies per warp, the copy in
//    registers: lane z holds word z of both planes = the 32 sites of colour c
//    in the slab z (bit 4 y + j, x = 2 j + ((y + z + c) & 1)), i.e. colour
//    ranks 32 z .. 32 z + 31. Neighbours along x and y are rotations of the
//    other plane's word, along z the words of the neighbouring lanes.
//  * k_sweep_bits3w: 3D lattices with L = 16, one warp per copy in registers:
//    word w = 4 z + q of a plane holds rows y = 4 q .. 4 q + 3 of slab z, bit
//    8 (y & 3) + j = the site x = 2 j + ((y + z + c) & 1) (colour ranks 32 w ..
//    32 w + 31); lane l holds words l and l + 32 (slabs l / 4 and 8 + l / 4).
//    Neighbours along x are rotations within a row's byte, along y byte shifts
//    (across the words of the slab's four lanes), along z the words of the
//    lanes l -/+ 4.
#include "bits.cuh"
#include "check.cuh"
#include "device.cuh"
#include "internal.h"

namespace gbmc {

namespace {

constexpr uint32_t kBitsWarps = 4;  // warps per block: 4 copies (2D) or 16 copies (3D)

// Which job a block belongs to (jobs own consecutive blocks).
__device__ __forceinline__ int job_of(const SweepLaunch& P, uint32_t block) {
    int j = 0;
    while (j + 1 < P.njobs && block >= P.cta_begin[j + 1]) ++j;
    return j;
}

// Thresholds of one copy: the job's, or its temperature's (parallel tempering).
__device__ __forceinline__ void copy_thresholds(const SweepJob& J, uint64_t slot, uint32_t& T4, uint32_t& T8,
                                                uint32_t& T12) {
    if (J.temp_of) {
        const uint32_t* th = J.thr_temp + 3ull * J.temp_of[slot];
        T4 = th[0];
        T8 = th[1];
        T12 = th[2];
    } else {
        T4 = J.thr[0];
        T8 = J.thr[1];
        T12 = J.thr[2];
    }
}

// Energy and magnetisation of one copy after the last sweep (or of every
// sweep when a series is asked for): lane 0 writes them and, for annealing
// runs, adds them to the population's histogram, range and exact sums.
__device__ __forceinline__ void record_copy(const SweepJob& J, uint64_t slot, uint32_t inst, uint32_t s, bool sweep,
                                            bool last, int E, int M) {
    const uint64_t ncopies = (uint64_t)J.n_inst * J.R;
    if (J.Eser && sweep) J.Eser[(uint64_t)s * ncopies + slot] = E;
    if (J.Mser && sweep) J.Mser[(uint64_t)s * ncopies + slot] = M;
    if (!last) return;
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

// ---------------------------------------------------------------------------
// 2D
// ---------------------------------------------------------------------------

// Neighbour words of the colour-c word idx = (y, w) when a row spans
// L / 64 >= 1 words: the other plane's words in rows y - 1 and y + 1 and in
// row y, and the row-y word shifted by one site towards j + 1 (odd x) or
// j - 1 (even x), wrapping around the row.
__device__ __forceinline__ void nb2(const uint32_t* oth, uint32_t idx, uint32_t lgW, uint32_t L, uint32_t colour,
                                    uint32_t& up, uint32_t& dn, uint32_t& same, uint32_t& side, uint32_t& q0) {
    const uint32_t Wm = (1u << lgW) - 1u;
    const uint32_t y = idx >> lgW, w = idx & Wm;
    const uint32_t PW = L << lgW;
    up = oth[GBMC_IDX((((y - 1u) & (L - 1u)) << lgW) + w, PW)];
    dn = oth[GBMC_IDX((((y + 1u) & (L - 1u)) << lgW) + w, PW)];
    same = oth[GBMC_IDX(idx, PW)];
    const bool odd = ((y + colour) & 1u) != 0u;
    const uint32_t nbw = oth[GBMC_IDX((y << lgW) + ((odd ? w + 1u : w - 1u) & Wm), PW)];
    side = odd ? __funnelshift_r(same, nbw, 1) : __funnelshift_l(nbw, same, 1);
    q0 = y * (L >> 3) + 8u * w;
}

// The same when a word holds 64 / L rows of S = L / 2 sites (L = 16: four
// rows of 8, L = 32: two rows of 16): row s of word w is y = (64 / L) w + s,
// bits S s .. S s + S - 1. Rows y -/+ 1 are the neighbouring S-bit segments
// (across words at the ends); the x neighbour not sharing j is a rotation
// by one site within each row, towards j + 1 in the rows of odd x
// ((s + c) odd) and towards j - 1 in the others.
__device__ __forceinline__ void nb2_rows(const uint32_t* oth, uint32_t w, uint32_t PW, uint32_t S, uint32_t colour,
                                         uint32_t& up, uint32_t& dn, uint32_t& same, uint32_t& side, uint32_t& q0) {
    const uint32_t wm = PW - 1u;
    same = oth[GBMC_IDX(w, PW)];
    const uint32_t prev = oth[GBMC_IDX((w - 1u) & wm, PW)], next = oth[GBMC_IDX((w + 1u) & wm, PW)];
    up = __funnelshift_l(prev, same, S);  // (same << S) | (prev >> (32 - S))
    dn = __funnelshift_r(same, next, S);  // (same >> S) | (next << (32 - S))
    const uint32_t top = S == 16u ? 0x80008000u : 0x80808080u;  // last site of each row
    const uint32_t bot = S == 16u ? 0x00010001u : 0x01010101u;  // first site of each row
    const uint32_t to_next = ((same >> 1) & ~top) | ((same << (S - 1u)) & top);  // bit j <- bit j + 1
    const uint32_t to_prev = ((same << 1) & ~bot) | ((same >> (S - 1u)) & bot);  // bit j <- bit j - 1
    const uint32_t odd_s = S == 16u ? 0xFFFF0000u : 0xFF00FF00u;                 // rows s odd
    const uint32_t odd_x = colour ? ~odd_s : odd_s;                               // rows with odd x
    side = (to_next & odd_x) | (to_prev & ~odd_x);
    q0 = 8u * w;
}

// ROWS: every job has L <= 32 (words of several rows), else every job has L >= 64.
template <bool ROWS>
__global__ void __launch_bounds__(128) k_sweep_bits2(const __grid_constant__ SweepLaunch P, uint32_t wpb,
                                                     uint32_t words_per_warp) {
    extern __shared__ __align__(16) uint32_t smw[];
    const uint32_t lane = threadIdx.x & 31u, wib = threadIdx.x >> 5;
    const int jid = job_of(P, blockIdx.x);
    const SweepJob& J = P.jobs[jid];
    const uint32_t L = J.L, N = J.N;
    const uint32_t lgL = 31u - __clz(L);
    const uint32_t PW = N >> 6;                    // words per colour plane
    // lanes per copy: 32 (L >= 64), or one per word (L <= 32: a plane has 4 or 16 words)
    const uint32_t lpc = ROWS ? PW : 32u, lgl = ROWS ? 31u - __clz(lpc) : 5u;
    const uint32_t li = ROWS ? lane & (lpc - 1u) : lane, grp = ROWS ? lane >> lgl : 0u;
    const uint32_t per_warp = ROWS ? 32u >> lgl : 1u;
    const uint64_t ncopies = (uint64_t)J.n_inst * J.R;
    const uint64_t wslot = ((uint64_t)(blockIdx.x - P.cta_begin[jid]) * wpb + wib) * per_warp;
    if (wslot >= ncopies) return;                  // whole warp; no block barriers follow
    const uint64_t slot = wslot + grp;
    uint32_t inst = 0, r = 0;
    bool active = slot < ncopies;
    if (active) {
        split_copy(slot, J.R, inst, r);
        if (J.nlive && r >= J.nlive[inst]) active = false;  // variable populations: only live slots
    }
    if (!ROWS && !active) return;                  // one copy per warp: the whole warp
    // every lane of the warp takes part in its syncs and reductions
    uint32_t* sm = smw + (uint64_t)wib * words_per_warp + (uint64_t)grp * 2u * PW;
    uint8_t* smb = reinterpret_cast<uint8_t*>(sm);
    const uint32_t bytes = words_per_warp * 4u;
    const uint32_t cshift = lgL - 4u;              // 16-byte chunks per row = L / 16

    // ---- load: int8 rows -> bit planes. A chunk of 16 sites holds 8 even-x sites
    // (colour y & 1) and 8 odd-x sites, consecutive colour ranks in each plane:
    // their down bits are byte c16 of the two planes ----
    if (active) {
        const uint64_t srcslot = J.parent ? (uint64_t)inst * J.R + J.parent[slot] : slot;
        const uint4* g = reinterpret_cast<const uint4*>(J.src + GBMC_IDX(srcslot, ncopies) * N);
        for (uint32_t c16 = li; c16 < (N >> 4); c16 += lpc) {
            const uint4 v = g[c16];
            uint32_t e0, o0, e1, o1;
            pack8(v.x, v.y, e0, o0);
            pack8(v.z, v.w, e1, o1);
            const uint32_t ce = (c16 >> cshift) & 1u;  // colour of the even-x sites of row y
            smb[GBMC_IDX((ce * PW << 2) + c16, bytes)] = (uint8_t)(e0 | (e1 << 4));
            smb[GBMC_IDX(((ce ^ 1u) * PW << 2) + c16, bytes)] = (uint8_t)(o0 | (o1 << 4));
        }
    }
    __syncwarp();

    uint32_t T4, T8, T12;
    copy_thresholds(J, active ? slot : 0, T4, T8, T12);
    const uint32_t instance = J.inst_base + inst;
    const uint32_t k0 = (uint32_t)J.seed, k1 = (uint32_t)(J.seed >> 32);
    const bool want_final = J.E || J.M || J.hist;
    constexpr bool rows = ROWS;
    const uint32_t lgW = rows ? 0u : lgL - 6u, S = L >> 1;
    const uint32_t nsw = J.nsweeps;
    for (uint32_t s = 0; s <= nsw; ++s) {
        if (s == nsw && nsw != 0) break;  // s == nsw: measurement-only pass when nothing is swept
        const bool sweep = s < nsw;
        if (sweep) {
            const uint32_t t = J.t0 + s;
            for (uint32_t colour = 0; colour < 2; ++colour) {
                const PhiloxFixed pf = philox_fix(t, r, c3_word(kPurposeMetro, colour, instance), k0, k1);
                uint32_t* own = sm + colour * PW;
                const uint32_t* oth = sm + (colour ^ 1u) * PW;
                if (active && rows) {
                    uint32_t u, d, sa, x, q;
                    nb2_rows(oth, li, PW, S, colour, u, d, sa, x, q);
                    const uint32_t nw = bp_word_update(own[li], u, d, sa, x, pf, q, T4, T8);
                    own[li] = nw;
                } else if (active) {
                    // two words per lane and step (PW is a multiple of 64): both are
                    // loaded and updated before either is stored (they only read the
                    // other plane)
                    for (uint32_t ia = li; ia < PW; ia += 64u) {
                        const uint32_t ib = ia + 32u;
                        uint32_t ua, da, sa, xa, qa, ub, db, sb, xb, qb;
                        nb2(oth, ia, lgW, L, colour, ua, da, sa, xa, qa);
                        nb2(oth, ib, lgW, L, colour, ub, db, sb, xb, qb);
                        const uint32_t wa = own[ia], wb = own[ib];
                        const uint32_t na = bp_word_update(wa, ua, da, sa, xa, pf, qa, T4, T8);
                        const uint32_t nb = bp_word_update(wb, ub, db, sb, xb, pf, qb, T4, T8);
                        own[ia] = na;
                        own[ib] = nb;
                    }
                }
                __syncwarp();
            }
        }
        const bool last = sweep ? s + 1 == nsw : true;
        if ((J.Eser && sweep) || (J.Mser && sweep) || (last && want_final)) {
            // E = -sum over bonds s_i s_j: every bond has one colour-0 end, so
            // E = 2 (unsatisfied bonds of the colour-0 sites) - 2 N
            int U = 0, D = 0;
            if (active) {
                for (uint32_t idx = li; idx < PW; idx += lpc) {
                    uint32_t up, dn, same, side, q0;
                    if (rows) nb2_rows(sm + PW, idx, PW, S, 0u, up, dn, same, side, q0);
                    else nb2(sm + PW, idx, lgW, L, 0u, up, dn, same, side, q0);
                    const uint32_t w0 = sm[idx];
                    U += __popc(w0 ^ up) + __popc(w0 ^ dn) + __popc(w0 ^ same) + __popc(w0 ^ side);
                    D += __popc(w0) + __popc(sm[PW + idx]);
                }
            }
            for (uint32_t o = lpc >> 1; o > 0; o >>= 1) {  // within the copy's lanes
                U += __shfl_xor_sync(0xffffffffu, U, o);
                D += __shfl_xor_sync(0xffffffffu, D, o);
            }
            if (active && li == 0) record_copy(J, slot, inst, s, sweep, last, 2 * U - 2 * (int)N, (int)N - 2 * D);
        }
    }

    // ---- store: bit planes -> int8 rows ----
    if (active && (nsw > 0 || J.dst != J.src || J.parent)) {
        uint4* d = reinterpret_cast<uint4*>(J.dst + slot * N);
        for (uint32_t c16 = li; c16 < (N >> 4); c16 += lpc) {
            const uint32_t ce = (c16 >> cshift) & 1u;
            const uint32_t ev = smb[GBMC_IDX((ce * PW << 2) + c16, bytes)];
            const uint32_t od = smb[GBMC_IDX(((ce ^ 1u) * PW << 2) + c16, bytes)];
            const uint2 lo = unpack8(ev & 15u, od & 15u), hi = unpack8(ev >> 4, od >> 4);
            d[c16] = make_uint4(lo.x, lo.y, hi.x, hi.y);
        }
    }
}

// ---------------------------------------------------------------------------
// 3D, L = 8
// ---------------------------------------------------------------------------

// Rotation of each 4-bit row (nibble) of a slab word by one site: bit j takes
// bit j - 1 (lft) or bit j + 1 (rgt), wrapping within the row.
__device__ __forceinline__ uint32_t rot_nib_lft(uint32_t w) {
    return ((w << 1) & 0xEEEEEEEEu) | ((w >> 3) & 0x11111111u);
}
__device__ __forceinline__ uint32_t rot_nib_rgt(uint32_t w) {
    return ((w >> 1) & 0x77777777u) | ((w << 3) & 0x88888888u);
}

// The six neighbour words of the colour-c word of slab z, in the bond order
// (same-j x neighbour, other x neighbour, y - 1, y + 1, z - 1, z + 1), from the
// other plane's word of this lane and of the lanes of slabs z -/+ 1.
__device__ __forceinline__ void nb3(uint32_t oth, uint32_t z, uint32_t colour, uint32_t gbase, uint32_t nb[6]) {
    // rows whose sites of colour c have odd x: (y + z + c) odd
    const uint32_t odd_rows = ((z + colour) & 1u) ? 0x0F0F0F0Fu : 0xF0F0F0F0u;
    nb[0] = oth;
    nb[1] = (rot_nib_lft(oth) & ~odd_rows) | (rot_nib_rgt(oth) & odd_rows);
    nb[2] = __funnelshift_l(oth, oth, 4);  // row y takes row y - 1
    nb[3] = __funnelshift_r(oth, oth, 4);  // row y takes row y + 1
    nb[4] = __shfl_sync(0xffffffffu, oth, gbase | ((z - 1u) & 7u));
    nb[5] = __shfl_sync(0xffffffffu, oth, gbase | ((z + 1u) & 7u));
}

template <bool EA>
__global__ void __launch_bounds__(128) k_sweep_bits3(const __grid_constant__ SweepLaunch P, uint32_t wpb) {
    __shared__ __align__(16) uint32_t stage[kBitsWarps][4][16];  // [warp][copy][plane * 8 + z]
    const uint32_t lane = threadIdx.x & 31u, wib = threadIdx.x >> 5;
    const int jid = job_of(P, blockIdx.x);
    const SweepJob& J = P.jobs[jid];
    const uint64_t ncopies = (uint64_t)J.n_inst * J.R;
    const uint64_t warp_slot0 = ((uint64_t)(blockIdx.x - P.cta_begin[jid]) * wpb + wib) * 4u;
    if (warp_slot0 >= ncopies) return;  // whole warp
    const uint32_t g = lane >> 3, z = lane & 7u, gbase = lane & ~7u;
    const uint64_t slot = warp_slot0 + g;
    uint32_t inst = 0, r = 0;
    bool active = slot < ncopies;
    if (active) {
        split_copy(slot, J.R, inst, r);
        if (J.nlive && r >= J.nlive[inst]) active = false;
    }
    // every lane takes part in the shuffles; inactive copies compute on zeros
    constexpr uint32_t N = 512u;
    uint8_t* stb = reinterpret_cast<uint8_t*>(stage[wib][g]);

    // ---- load: chunk m of 16 bytes = rows y, y + 1 (y = 2 (m & 3)) of slab m >> 2 ----
    const uint64_t srcslot = active ? (J.parent ? (uint64_t)inst * J.R + J.parent[slot] : slot) : 0;
#pragma unroll
    for (uint32_t k = 0; k < 4; ++k) {
        const uint32_t m = z + 8u * k, zz = m >> 2, y = (m & 3u) << 1;
        uint4 v = make_uint4(0x01010101u, 0x01010101u, 0x01010101u, 0x01010101u);
        if (active) v = reinterpret_cast<const uint4*>(J.src + srcslot * N)[m];
        uint32_t ey, oy, ey1, oy1;
        pack8(v.x, v.y, ey, oy);    // row y
        pack8(v.z, v.w, ey1, oy1);  // row y + 1
        // plane A = (y + z) & 1 holds the even-x sites of row y and the odd-x sites of row y + 1
        const uint32_t A = (y + zz) & 1u;
        stb[((A * 8u + zz) << 2) + (y >> 1)] = (uint8_t)(ey | (oy1 << 4));
        stb[(((A ^ 1u) * 8u + zz) << 2) + (y >> 1)] = (uint8_t)(oy | (ey1 << 4));
    }
    __syncwarp();
    uint32_t pl[2] = {stage[wib][g][z], stage[wib][g][8 + z]};
    __syncwarp();

    uint32_t jb[2][6];
#pragma unroll
    for (uint32_t c = 0; c < 2; ++c)
#pragma unroll
        for (uint32_t k = 0; k < 6; ++k)
            jb[c][k] = (EA && active) ? J.jb3[GBMC_IDX((((uint64_t)inst * 2u + c) * 6u + k) * 8u + z, J.n_inst * 96ull)]
                                      : 0u;

    uint32_t T4, T8, T12;
    copy_thresholds(J, active ? slot : 0, T4, T8, T12);
    const uint32_t instance = J.inst_base + inst;
    const uint32_t k0 = (uint32_t)J.seed, k1 = (uint32_t)(J.seed >> 32);
    const bool want_final = J.E || J.M || J.hist;
    const uint32_t nsw = J.nsweeps;
    for (uint32_t s = 0; s <= nsw; ++s) {
        if (s == nsw && nsw != 0) break;
        const bool sweep = s < nsw;
        if (sweep) {
            const uint32_t t = J.t0 + s;
#pragma unroll 1
            for (uint32_t colour = 0; colour < 2; ++colour) {
                const PhiloxFixed pf = philox_fix(t, r, c3_word(kPurposeMetro, colour, instance), k0, k1);
                uint32_t nb[6];
                nb3(colour ? pl[0] : pl[1], z, colour, gbase, nb);
                const uint32_t w = colour ? pl[1] : pl[0];
                uint32_t d[6];
#pragma unroll
                for (uint32_t k = 0; k < 6; ++k) d[k] = w ^ nb[k] ^ (colour ? jb[1][k] : jb[0][k]);
                const uint32_t nw = bp3_word_update(w, d[0], d[1], d[2], d[3], d[4], d[5], pf, 8u * z, T4, T8, T12);
                if (colour) pl[1] = nw;
                else pl[0] = nw;
            }
        }
        const bool last = sweep ? s + 1 == nsw : true;
        if ((J.Eser && sweep) || (J.Mser && sweep) || (last && want_final)) {
            uint32_t nb[6];
            nb3(pl[1], z, 0u, gbase, nb);
            int U = 0;
#pragma unroll
            for (uint32_t k = 0; k < 6; ++k) U += __popc(pl[0] ^ nb[k] ^ jb[0][k]);
            int D = __popc(pl[0]) + __popc(pl[1]);
#pragma unroll
            for (uint32_t o = 4; o > 0; o >>= 1) {
                U += __shfl_xor_sync(0xffffffffu, U, o);
                D += __shfl_xor_sync(0xffffffffu, D, o);
            }
            // E = 2 (unsatisfied bonds of the colour-0 sites) - 3 N
            if (active && z == 0) record_copy(J, slot, inst, s, sweep, last, 2 * U - 3 * (int)N, (int)N - 2 * D);
        }
    }

    // ---- store ----
    if (nsw > 0 || J.dst != J.src || J.parent) {
        stage[wib][g][z] = pl[0];
        stage[wib][g][8 + z] = pl[1];
        __syncwarp();
        if (active) {
#pragma unroll
            for (uint32_t k = 0; k < 4; ++k) {
                const uint32_t m = z + 8u * k, zz = m >> 2, y = (m & 3u) << 1;
                const uint32_t A = (y + zz) & 1u;
                const uint32_t ba = stb[((A * 8u + zz) << 2) + (y >> 1)];
                const uint32_t bb = stb[(((A ^ 1u) * 8u + zz) << 2) + (y >> 1)];
                const uint2 row0 = unpack8(ba & 15u, bb & 15u);  // row y: even from A, odd from B
                const uint2 row1 = unpack8(bb >> 4, ba >> 4);     // row y + 1: even from B, odd from A
                reinterpret_cast<uint4*>(J.dst + slot * N)[m] = make_uint4(row0.x, row0.y, row1.x, row1.y);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// 3D, L = 16
// ---------------------------------------------------------------------------

// Rotation of each 8-site row (byte) of a word by one site: bit j takes bit
// j - 1 (lft) or bit j + 1 (rgt), wrapping within the row.
__device__ __forceinline__ uint32_t rot_byte_lft(uint32_t w) {
    return ((w << 1) & 0xFEFEFEFEu) | ((w >> 7) & 0x01010101u);
}
__device__ __forceinline__ uint32_t rot_byte_rgt(uint32_t w) {
    return ((w >> 1) & 0x7F7F7F7Fu) | ((w << 7) & 0x80808080u);
}

// The six neighbour words (order of nb3) of this lane's two colour-c words,
// from the other plane's words oth[h] (h = 0: slab l / 4, h = 1: slab 8 + l / 4).
__device__ __forceinline__ void nb3w(const uint32_t oth[2], uint32_t lane, uint32_t colour, uint32_t nb[2][6]) {
    const uint32_t prevl = (lane & ~3u) | ((lane - 1u) & 3u), nextl = (lane & ~3u) | ((lane + 1u) & 3u);
#pragma unroll
    for (uint32_t h = 0; h < 2; ++h) {
        const uint32_t z = (lane >> 2) + 8u * h;
        // rows (bytes) whose sites of colour c have odd x: (y + z + c) odd
        const uint32_t odd_rows = ((z + colour) & 1u) ? 0x00FF00FFu : 0xFF00FF00u;
        nb[h][0] = oth[h];
        nb[h][1] = (rot_byte_lft(oth[h]) & ~odd_rows) | (rot_byte_rgt(oth[h]) & odd_rows);
        const uint32_t prev = __shfl_sync(0xffffffffu, oth[h], prevl);  // rows y - 4 .. y - 1
        const uint32_t next = __shfl_sync(0xffffffffu, oth[h], nextl);
        nb[h][2] = __funnelshift_l(prev, oth[h], 8);  // row y takes row y - 1
        nb[h][3] = __funnelshift_r(oth[h], next, 8);  // row y takes row y + 1
    }
    // slabs z -/+ 1: lanes l -/+ 4, the other half across the wrap
    const uint32_t a0 = __shfl_sync(0xffffffffu, oth[0], (lane - 4u) & 31u);
    const uint32_t a1 = __shfl_sync(0xffffffffu, oth[1], (lane - 4u) & 31u);
    const uint32_t b0 = __shfl_sync(0xffffffffu, oth[0], (lane + 4u) & 31u);
    const uint32_t b1 = __shfl_sync(0xffffffffu, oth[1], (lane + 4u) & 31u);
    nb[0][4] = lane >= 4u ? a0 : a1;
    nb[1][4] = lane >= 4u ? a1 : a0;
    nb[0][5] = lane < 28u ? b0 : b1;
    nb[1][5] = lane < 28u ? b1 : b0;
}

template <bool EA>
__global__ void __launch_bounds__(128) k_sweep_bits3w(const __grid_constant__ SweepLaunch P, uint32_t wpb) {
    __shared__ __align__(16) uint32_t stage[kBitsWarps][2][64];  // [warp][plane][word]
    const uint32_t lane = threadIdx.x & 31u, wib = threadIdx.x >> 5;
    const int jid = job_of(P, blockIdx.x);
    const SweepJob& J = P.jobs[jid];
    const uint64_t ncopies = (uint64_t)J.n_inst * J.R;
    const uint64_t slot = (uint64_t)(blockIdx.x - P.cta_begin[jid]) * wpb + wib;
    if (slot >= ncopies) return;  // whole warp; no block barriers follow
    uint32_t inst = 0, r = 0;
    split_copy(slot, J.R, inst, r);
    if (J.nlive && r >= J.nlive[inst]) return;  // variable populations: only live slots
    constexpr uint32_t N = 4096u;
    uint8_t* stb = reinterpret_cast<uint8_t*>(stage[wib]);

    // ---- load: chunk m of 16 bytes = row y = m & 15 of slab z = m >> 4; its 8
    // even-x sites (colour (y + z) & 1) and 8 odd-x sites are byte m of the two planes ----
    const uint64_t srcslot = J.parent ? (uint64_t)inst * J.R + J.parent[slot] : slot;
    const uint4* g = reinterpret_cast<const uint4*>(J.src + GBMC_IDX(srcslot, ncopies) * N);
#pragma unroll
    for (uint32_t k = 0; k < 8; ++k) {
        const uint32_t m = lane + 32u * k;
        const uint4 v = g[m];
        uint32_t e0, o0, e1, o1;
        pack8(v.x, v.y, e0, o0);
        pack8(v.z, v.w, e1, o1);
        const uint32_t ce = ((m & 15u) + (m >> 4)) & 1u;
        stb[GBMC_IDX(ce * 256u + m, 512u)] = (uint8_t)(e0 | (e1 << 4));
        stb[GBMC_IDX((ce ^ 1u) * 256u + m, 512u)] = (uint8_t)(o0 | (o1 << 4));
    }
    __syncwarp();
    uint32_t pl[2][2] = {{stage[wib][0][lane], stage[wib][0][lane + 32u]},
                         {stage[wib][1][lane], stage[wib][1][lane + 32u]}};  // [colour][half]
    __syncwarp();

    uint32_t jb[2][2][6];  // [colour][half][bond kind]
#pragma unroll
    for (uint32_t c = 0; c < 2; ++c)
#pragma unroll
        for (uint32_t h = 0; h < 2; ++h)
#pragma unroll
            for (uint32_t k = 0; k < 6; ++k)
                jb[c][h][k] = EA ? J.jb3[GBMC_IDX((((uint64_t)inst * 2u + c) * 6u + k) * 64u + lane + 32u * h,
                                                  J.n_inst * 768ull)]
                                 : 0u;

    uint32_t T4, T8, T12;
    copy_thresholds(J, slot, T4, T8, T12);
    const uint32_t instance = J.inst_base + inst;
    const uint32_t k0 = (uint32_t)J.seed, k1 = (uint32_t)(J.seed >> 32);
    const bool want_final = J.E || J.M || J.hist;
    const uint32_t nsw = J.nsweeps;
    for (uint32_t s = 0; s <= nsw; ++s) {
        if (s == nsw && nsw != 0) break;
        const bool sweep = s < nsw;
        if (sweep) {
            const uint32_t t = J.t0 + s;
#pragma unroll 1
            for (uint32_t colour = 0; colour < 2; ++colour) {
                const PhiloxFixed pf = philox_fix(t, r, c3_word(kPurposeMetro, colour, instance), k0, k1);
                uint32_t nb[2][6];
                nb3w(colour ? pl[0] : pl[1], lane, colour, nb);
#pragma unroll
                for (uint32_t h = 0; h < 2; ++h) {
                    const uint32_t w = colour ? pl[1][h] : pl[0][h];
                    uint32_t d[6];
#pragma unroll
                    for (uint32_t k = 0; k < 6; ++k) d[k] = w ^ nb[h][k] ^ (colour ? jb[1][h][k] : jb[0][h][k]);
                    const uint32_t nw =
                        bp3_word_update(w, d[0], d[1], d[2], d[3], d[4], d[5], pf, 8u * (lane + 32u * h), T4, T8, T12);
                    if (colour) pl[1][h] = nw;
                    else pl[0][h] = nw;
                }
            }
        }
        const bool last = sweep ? s + 1 == nsw : true;
        if ((J.Eser && sweep) || (J.Mser && sweep) || (last && want_final)) {
            uint32_t nb[2][6];
            nb3w(pl[1], lane, 0u, nb);
            int U = 0;
#pragma unroll
            for (uint32_t h = 0; h < 2; ++h)
#pragma unroll
                for (uint32_t k = 0; k < 6; ++k) U += __popc(pl[0][h] ^ nb[h][k] ^ jb[0][h][k]);
            int D = __popc(pl[0][0]) + __popc(pl[0][1]) + __popc(pl[1][0]) + __popc(pl[1][1]);
#pragma unroll
            for (uint32_t o = 16; o > 0; o >>= 1) {
                U += __shfl_xor_sync(0xffffffffu, U, o);
                D += __shfl_xor_sync(0xffffffffu, D, o);
            }
            // E = 2 (unsatisfied bonds of the colour-0 sites) - 3 N
            if (lane == 0) record_copy(J, slot, inst, s, sweep, last, 2 * U - 3 * (int)N, (int)N - 2 * D);
        }
    }

    // ---- store ----
    if (nsw > 0 || J.dst != J.src || J.parent) {
        stage[wib][0][lane] = pl[0][0];
        stage[wib][0][lane + 32u] = pl[0][1];
        stage[wib][1][lane] = pl[1][0];
        stage[wib][1][lane + 32u] = pl[1][1];
        __syncwarp();
        uint4* d = reinterpret_cast<uint4*>(J.dst + slot * N);
#pragma unroll
        for (uint32_t k = 0; k < 8; ++k) {
            const uint32_t m = lane + 32u * k;
            const uint32_t ce = ((m & 15u) + (m >> 4)) & 1u;
            const uint32_t ev = stb[GBMC_IDX(ce * 256u + m, 512u)], od = stb[GBMC_IDX((ce ^ 1u) * 256u + m, 512u)];
            const uint2 lo = unpack8(ev & 15u, od & 15u), hi = unpack8(ev >> 4, od >> 4);
            d[m] = make_uint4(lo.x, lo.y, hi.x, hi.y);
        }
    }
}

// Bond words of the 3D L = 8 bit-sliced sweep: for instance i, colour c, bond
// kind k and slab z, bit 4 y + j = 1 iff the bond between the colour-c site
// (x = 2 j + ((y + z + c) & 1), y, z) and its k-th neighbour (order of nb3)
// has J = -1. jbits: [inst][mu][site] bytes, 1 where the forward bond of the
// site along mu has J = -1.
__global__ void k_bits3_bonds(const uint8_t* jbits, uint32_t* jb3, uint32_t n_inst) {
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n_inst * 96u) return;
    const uint32_t inst = g / 96u, rem = g - inst * 96u;
    const uint32_t c = rem / 48u, k = (rem / 8u) % 6u, z = rem & 7u;
    constexpr uint32_t L = 8u, N = 512u;
    const uint8_t* jb = jbits + (uint64_t)inst * 3u * N;
    uint32_t word = 0;
    for (uint32_t y = 0; y < L; ++y)
        for (uint32_t j = 0; j < 4; ++j) {
            const uint32_t o = (y + z + c) & 1u, x = 2u * j + o;
            const uint32_t i = (z * L + y) * L + x;
            const uint32_t xm = (z * L + y) * L + ((x + L - 1u) & (L - 1u));  // site x - 1
            uint32_t bond;
            switch (k) {
                case 0: bond = o ? jb[xm] : jb[i]; break;                                     // same-j x neighbour
                case 1: bond = o ? jb[i] : jb[xm]; break;                                     // the other x neighbour
                case 2: bond = jb[N + (z * L + ((y + L - 1u) & (L - 1u))) * L + x]; break;    // y - 1
                case 3: bond = jb[N + i]; break;                                              // y + 1
                case 4: bond = jb[2u * N + ((((z + L - 1u) & (L - 1u)) * L + y) * L + x)]; break;  // z - 1
                default: bond = jb[2u * N + i]; break;                                        // z + 1
            }
            word |= (bond ? 1u : 0u) << (4u * y + j);
        }
    jb3[g] = word;
}

// The same for L = 16 (word w = 4 z + q of k_sweep_bits3w, bit 8 (y & 3) + j,
// y = 4 q + (y & 3)): for instance i, colour c, bond kind k, word w at
// ((i * 2 + c) * 6 + k) * 64 + w.
__global__ void k_bits3w_bonds(const uint8_t* jbits, uint32_t* jb3, uint32_t n_inst) {
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n_inst * 768u) return;
    const uint32_t inst = g / 768u, rem = g - inst * 768u;
    const uint32_t c = rem / 384u, k = (rem / 64u) % 6u, w = rem & 63u;
    const uint32_t z = w >> 2, q = w & 3u;
    constexpr uint32_t L = 16u, N = 4096u;
    const uint8_t* jb = jbits + (uint64_t)inst * 3u * N;
    uint32_t word = 0;
    for (uint32_t yy = 0; yy < 4; ++yy)
        for (uint32_t j = 0; j < 8; ++j) {
            const uint32_t y = 4u * q + yy;
            const uint32_t o = (y + z + c) & 1u, x = 2u * j + o;
            const uint32_t i = (z * L + y) * L + x;
            const uint32_t xm = (z * L + y) * L + ((x + L - 1u) & (L - 1u));  // site x - 1
            uint32_t bond;
            switch (k) {
                case 0: bond = o ? jb[xm] : jb[i]; break;                                     // same-j x neighbour
                case 1: bond = o ? jb[i] : jb[xm]; break;                                     // the other x neighbour
                case 2: bond = jb[N + (z * L + ((y + L - 1u) & (L - 1u))) * L + x]; break;    // y - 1
                case 3: bond = jb[N + i]; break;                                              // y + 1
                case 4: bond = jb[2u * N + ((((z + L - 1u) & (L - 1u)) * L + y) * L + x)]; break;  // z - 1
                default: bond = jb[2u * N + i]; break;                                        // z + 1
            }
            word |= (bond ? 1u : 0u) << (8u * yy + j);
        }
    jb3[g] = word;
}

}  // namespace

bool bits_supported(int dim, int L) {
    return (dim == 2 && (L == 16 || L == 32 || L == 64 || L == 128 || L == 256)) || (dim == 3 && (L == 8 || L == 16));
}

size_t bits3_bond_words(uint32_t L) { return L == 8 ? 96u : 768u; }

cudaError_t launch_bits3_bonds(const uint8_t* jbits, uint32_t* jb3, uint32_t L, uint32_t n_inst, cudaStream_t s) {
    if (L != 8 && L != 16) return cudaErrorInvalidValue;
    const uint32_t n = n_inst * (uint32_t)bits3_bond_words(L);
    if (L == 8) k_bits3_bonds<<<(n + 255u) / 256u, 256, 0, s>>>(jbits, jb3, n_inst);
    else k_bits3w_bonds<<<(n + 255u) / 256u, 256, 0, s>>>(jbits, jb3, n_inst);
    count_launch();
    return cudaGetLastError();
}

static cudaError_t launch_bits_group(const SweepLaunch& P0, bool rows, cudaStream_t s) {
    constexpr uint32_t kWarps = kBitsWarps;
    SweepLaunch P = P0;
    // largest copies first: their blocks are dispatched first, shortening the tail
    for (int a = 1; a < P.njobs; ++a)
        for (int b = a; b > 0 && P.jobs[b].N > P.jobs[b - 1].N; --b) {
            const SweepJob t = P.jobs[b];
            P.jobs[b] = P.jobs[b - 1];
            P.jobs[b - 1] = t;
        }
    uint32_t total = 0, words = 0;
    for (int j = 0; j < P.njobs; ++j) {
        const SweepJob& J = P.jobs[j];
        if (!bits_supported(P.dim, (int)J.L)) return cudaErrorInvalidValue;
        P.cta_begin[j] = total;
        // 2D: one copy per warp, or 32 / (N / 64) copies when a plane has fewer
        // than 32 words (L = 16: 8, L = 32: 2); 3D L = 8: 4 copies per warp
        const uint32_t pw = J.N / 64u;
        const uint32_t per_warp = P.dim == 2 ? (pw < 32u ? 32u / pw : 1u) : (J.L == 8 ? 4u : 1u);
        const uint64_t nb = ((uint64_t)J.n_inst * J.R + per_warp * kWarps - 1) / (per_warp * kWarps);
        if (total + nb > 0x7FFFFFFFull) return cudaErrorInvalidValue;
        total += (uint32_t)nb;
        const uint32_t w = per_warp * 2u * pw;  // two planes of N / 2 bits per copy
        if (w > words) words = w;
    }
    P.cta_begin[P.njobs] = total;
    P.total = total;
    if (total == 0) return cudaSuccess;
    if (P.dim == 2) {
        const size_t smem = (size_t)kWarps * words * 4u;
        auto kern = rows ? k_sweep_bits2<true> : k_sweep_bits2<false>;
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        kern<<<total, 32u * kWarps, smem, s>>>(P, kWarps, words);
    } else if (P.jobs[0].L == 16) {
        if (P.ea) k_sweep_bits3w<true><<<total, 32u * kWarps, 0, s>>>(P, kWarps);
        else k_sweep_bits3w<false><<<total, 32u * kWarps, 0, s>>>(P, kWarps);
    } else if (P.ea) {
        k_sweep_bits3<true><<<total, 32u * kWarps, 0, s>>>(P, kWarps);
    } else {
        k_sweep_bits3<false><<<total, 32u * kWarps, 0, s>>>(P, kWarps);
    }
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_sweep_bits(const SweepLaunch& P0, cudaStream_t s) {
    // 2D: lattices whose words hold several rows (L <= 32) in their own launch;
    // 3D: L = 8 and L = 16 in launches of their own kernels
    SweepLaunch A = P0, B = P0;
    A.njobs = B.njobs = 0;
    for (int j = 0; j < P0.njobs; ++j) {
        if (P0.dim == 2 ? P0.jobs[j].L <= 32 : P0.jobs[j].L == 16) A.jobs[A.njobs++] = P0.jobs[j];
        else B.jobs[B.njobs++] = P0.jobs[j];
    }
    cudaError_t e = cudaSuccess;
    if (B.njobs) e = launch_bits_group(B, false, s);
    if (e == cudaSuccess && A.njobs) e = launch_bits_group(A, true, s);
    return e;
}

}  // namespace gbmc
