// units.cuh -- the site updates of one word of a copy (Sec. 3.1, Eq. (8)),
// shared by the resident, tiled, double-checkerboard and global sweep kernels.
//
// Spins are bytes +1 (0x01) / -1 (0xFF). For L % 8 == 0 the kernels keep each
// copy (or tile window) in shared memory as two colour planes (the separate
// sub-lattice storage of Sec. 3.1): plane c, row r = z*L + y, holds the L/2
// sites of colour c of that row in x order. A thread updates one 32-bit word
// of a plane = 4 consecutive same-colour sites = the 4 words of one Philox
// call. Their vertical neighbours are the same word of the other plane in the
// rows above/below; the horizontal ones are the same word and the word shifted
// by one byte (funnel shift). Byte-parallel (s_i ^ s_j) & 4 summed over the
// neighbours gives 4a per site, a = number of unsatisfied bonds
// (s_i J_ij s_j = -1), so dE = 4 (dim - a); 4a is also the byte offset of the
// site's threshold in a shared table (dE <= 0 -> 0xffffffff, i.e. always
// accept), and the site flips iff u <= table[a]. The global-memory kernel
// works on the row-major layout with 8-byte chunks; L % 8 != 0 uses a per-site
// path with the same Philox words.
#pragma once
#include "check.cuh"
#include "device.cuh"

namespace gbmc {

__device__ __forceinline__ uint64_t down_bits(uint64_t w) { return (w >> 1) & 0x0101010101010101ull; }

template <typename P>
__device__ __forceinline__ uint64_t ld8(const P* p) {
    return *reinterpret_cast<const uint64_t*>(p);
}

struct Thr {
    uint32_t t4, t8, t12;
};

// One 8-site chunk (row `row`, chunk `g`) of one copy: update the 4 sites of
// `colour`. sp: copy base; jb: bond planes of its instance (or null).
template <int DIM, bool EA, bool MEASURE>
__device__ __forceinline__ void unit_swar(uint8_t* sp, const uint8_t* jb, uint32_t L, uint32_t N,
                                          uint32_t row, uint32_t g, uint32_t colour,
                                          const PhiloxFixed& pf, const Thr& T, bool flip, int& e_acc,
                                          int& m_acc) {
    const uint32_t G = L >> 3;
    const uint32_t y = DIM == 3 ? row % L : row;
    const uint32_t z = DIM == 3 ? row / L : 0;
    const uint32_t off = (y + z + colour) & 1u;
    const uint32_t base = row * L;
    const uint32_t gl = g == 0 ? G - 1 : g - 1;
    const uint32_t gr = g + 1 == G ? 0 : g + 1;
    const uint32_t rowu = y == 0 ? row + L - 1 : row - 1;       // y - 1
    const uint32_t rowd = y + 1 == L ? row + 1 - L : row + 1;   // y + 1
    const uint64_t cur = ld8(sp + GBMC_IDX(base + 8 * g, N - 7));
    const uint64_t prv = ld8(sp + GBMC_IDX(base + 8 * gl, N - 7));
    const uint64_t nxt = ld8(sp + GBMC_IDX(base + 8 * gr, N - 7));
    const uint64_t up = ld8(sp + GBMC_IDX(rowu * L + 8 * g, N - 7));
    const uint64_t dn = ld8(sp + GBMC_IDX(rowd * L + 8 * g, N - 7));
    const uint64_t dc = down_bits(cur);
    uint64_t lft = down_bits((cur << 8) | (prv >> 56));
    uint64_t rgt = down_bits((cur >> 8) | (nxt << 56));
    uint64_t upb = down_bits(up), dnb = down_bits(dn);
    uint64_t bkb = 0, frb = 0;
    uint32_t rowb = 0;
    if (DIM == 3) {
        rowb = z == 0 ? row + (L - 1) * L : row - L;              // z - 1
        const uint32_t rowf = z + 1 == L ? row - (L - 1) * L : row + L;  // z + 1
        bkb = down_bits(ld8(sp + GBMC_IDX(rowb * L + 8 * g, N - 7)));
        frb = down_bits(ld8(sp + GBMC_IDX(rowf * L + 8 * g, N - 7)));
    }
    if (EA) {
        // bond planes: byte 1 where J = -1; an unsatisfied bond has d_i ^ d_j ^ b = 1
        const uint64_t jx = ld8(jb + base + 8 * g);
        const uint64_t jxp = ld8(jb + base + 8 * gl);
        rgt ^= jx;
        lft ^= (jx << 8) | (jxp >> 56);
        dnb ^= ld8(jb + N + base + 8 * g);
        upb ^= ld8(jb + N + rowu * L + 8 * g);
        if (DIM == 3) {
            frb ^= ld8(jb + 2 * N + base + 8 * g);
            bkb ^= ld8(jb + 2 * N + rowb * L + 8 * g);
        }
    }
    uint64_t a = (dc ^ lft) + (dc ^ rgt) + (dc ^ upb) + (dc ^ dnb);
    if (DIM == 3) a += (dc ^ bkb) + (dc ^ frb);

    uint4 w = make_uint4(0, 0, 0, 0);
    if (flip) w = philox_q(pf, row * G + g);
    uint64_t mask = 0;
    int e = 0;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const uint32_t pos = off + 2 * m;
        const int am = (int)((a >> (8 * pos)) & 0xFFu);
        const int d = DIM - am;  // dE / 4
        const uint32_t u = m == 0 ? w.x : m == 1 ? w.y : m == 2 ? w.z : w.w;
        const uint32_t thr = d == 1 ? T.t4 : (d == 2 ? T.t8 : T.t12);
        const bool acc = flip && (d <= 0 || u <= thr);
        mask |= acc ? (0xFEull << (8 * pos)) : 0ull;
        if (MEASURE) {
            const int sh = 2 * DIM - 2 * am;  // s_i h_i before the update
            e += acc ? sh : -sh;
        }
    }
    const uint64_t nw = cur ^ mask;
    if (flip) *reinterpret_cast<uint64_t*>(sp + base + 8 * g) = nw;
    if (MEASURE) {
        e_acc += e;
        m_acc += 8 - 2 * (int)__popcll(down_bits(nw));
    }
}

__device__ __forceinline__ uint32_t neq4(uint32_t a, uint32_t b) { return (a ^ b) & 0x04040404u; }

// Split-plane unit: word g of row `row` of colour plane `colour`; q is the
// Philox counter word of its 4 sites (row-major rank of the word over the
// whole lattice, which differs from row * (L/8) + g inside a tile). sp: copy
// base (plane 0 then plane 1, N/2 bytes each); jb: this colour's 2*DIM bond
// planes (bytes 0x04 where J = -1; order same-j x, shifted x, y-1, y+1, z-1,
// z+1); tbl: byte-addressed threshold table (entry a at byte 4a).
// STORE = false: the new word is returned in *st_idx / *st_val (index into the
// colour plane) instead of being written, so that a caller can load a second
// unit before storing the first.
template <int DIM, bool EA, bool MEASURE, bool STORE = true>
__device__ __forceinline__ void unit_split(uint8_t* sp, const uint8_t* jb, uint32_t L, uint32_t N,
                                           uint32_t row, uint32_t y, uint32_t z, uint32_t g, uint32_t colour,
                                           const PhiloxFixed& pf, const uint8_t* tbl, bool doflip, int& e_acc,
                                           int& m_acc, uint32_t q, uint32_t* st_idx = nullptr,
                                           uint32_t* st_val = nullptr) {
    const uint32_t W = L >> 3, H = N >> 1;
    const uint32_t o = (y + z + colour) & 1u;
    uint32_t* own = reinterpret_cast<uint32_t*>(sp + colour * H);
    const uint32_t* oth = reinterpret_cast<const uint32_t*>(sp + (colour ^ 1u) * H);
    const uint32_t rw = row * W;
    const uint32_t PW = H >> 2;  // words per colour plane
    const uint32_t cur = own[GBMC_IDX(rw + g, PW)];
    const uint32_t same = oth[GBMC_IDX(rw + g, PW)];
    // horizontal neighbour not sharing j: j+1 (odd x) or j-1 (even x)
    const uint32_t side = o ? __funnelshift_r(same, oth[GBMC_IDX(rw + (g + 1 == W ? 0 : g + 1), PW)], 8)
                            : __funnelshift_l(oth[GBMC_IDX(rw + (g == 0 ? W - 1 : g - 1), PW)], same, 8);
    const uint32_t rowu = y == 0 ? row + L - 1 : row - 1;
    const uint32_t rowd = y + 1 == L ? row + 1 - L : row + 1;
    const uint32_t up = oth[GBMC_IDX(rowu * W + g, PW)], dn = oth[GBMC_IDX(rowd * W + g, PW)];
    uint32_t a4;
    const uint32_t* b = EA ? reinterpret_cast<const uint32_t*>(jb) + rw + g : nullptr;
    const uint32_t P = H >> 2;  // words per plane
    if (EA) {
        a4 = (neq4(cur, same) ^ b[0]) + (neq4(cur, side) ^ b[P]) + (neq4(cur, up) ^ b[2 * P]) +
             (neq4(cur, dn) ^ b[3 * P]);
    } else {
        a4 = neq4(cur, same) + neq4(cur, side) + neq4(cur, up) + neq4(cur, dn);
    }
    if (DIM == 3) {
        const uint32_t rowb = z == 0 ? row + (L - 1) * L : row - L;
        const uint32_t rowf = z + 1 == L ? row - (L - 1) * L : row + L;
        const uint32_t bk = oth[GBMC_IDX(rowb * W + g, PW)], fr = oth[GBMC_IDX(rowf * W + g, PW)];
        if (EA) a4 += (neq4(cur, bk) ^ b[4 * P]) + (neq4(cur, fr) ^ b[5 * P]);
        else a4 += neq4(cur, bk) + neq4(cur, fr);
    }
    uint32_t flip = 0;
    if (doflip) {
        const uint4 w = philox_q(pf, q);
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const uint32_t am = __byte_perm(a4, 0u, 0x4440u + m);  // 4a of site m
            const uint32_t thr = *reinterpret_cast<const uint32_t*>(tbl + am);
            const uint32_t u = m == 0 ? w.x : m == 1 ? w.y : m == 2 ? w.z : w.w;
            flip |= (u <= thr) ? (0xFEu << (8 * m)) : 0u;
        }
    }
    const uint32_t nw = cur ^ flip;
    if constexpr (STORE) {
        if (doflip) own[GBMC_IDX(rw + g, PW)] = nw;
    } else {
        *st_idx = rw + g;
        *st_val = nw;
    }
    if (MEASURE) {
        // E contribution -sum s_new h = sum_acc s h - sum_rej s h, s h = 2 DIM - (4a)/2
        const int s_all = (int)__dp4a(a4, 0x01010101u, 0u);
        const int s_acc = (int)__dp4a(a4 & flip, 0x01010101u, 0u);
        const int nacc = __popc(flip & 0x02020202u);
        e_acc += 4 * DIM * nacc - s_acc - 8 * DIM + s_all / 2;
        // the other plane's word `same` pairs each of its sites with one site here
        m_acc += 8 - 2 * (__popc(nw & 0x02020202u) + __popc(same & 0x02020202u));
    }
}

// Per-site path for any even L: quad q covers colour ranks k = 4q .. 4q+3.
template <int DIM, bool EA, bool MEASURE>
__device__ __forceinline__ void unit_scalar(int8_t* sp, const uint8_t* jb, uint32_t L, uint32_t N,
                                            uint32_t q, uint32_t colour, const PhiloxFixed& pf,
                                            const Thr& T, bool flip, int& e_acc, int& m_acc) {
    const uint32_t half = L >> 1;
    const uint32_t ncol = N >> 1;
    uint4 w = make_uint4(0, 0, 0, 0);
    if (flip) w = philox_q(pf, q);
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const uint32_t k = 4 * q + m;
        if (k >= ncol) break;
        const uint32_t row = k / half, j = k - row * half;
        const uint32_t y = DIM == 3 ? row % L : row;
        const uint32_t z = DIM == 3 ? row / L : 0;
        const uint32_t x = 2 * j + ((y + z + colour) & 1u);
        const uint32_t i = row * L + x;
        const uint32_t xl = x == 0 ? L - 1 : x - 1, xr = x + 1 == L ? 0 : x + 1;
        const uint32_t yu = y == 0 ? L - 1 : y - 1, yd = y + 1 == L ? 0 : y + 1;
        const uint32_t zb = DIM == 3 ? row - y : 0;  // z*L
        const uint32_t i_l = row * L + xl, i_r = row * L + xr;
        const uint32_t i_u = (zb + yu) * L + x, i_d = (zb + yd) * L + x;
        int jl = 1, jr = 1, ju = 1, jd = 1, jbk = 1, jf = 1;
        if (EA) {
            jr = jb[i] ? -1 : 1;
            jl = jb[i_l] ? -1 : 1;
            jd = jb[N + i] ? -1 : 1;
            ju = jb[N + i_u] ? -1 : 1;
        }
        int h = jl * sp[GBMC_IDX(i_l, N)] + jr * sp[GBMC_IDX(i_r, N)] + ju * sp[GBMC_IDX(i_u, N)] +
                jd * sp[GBMC_IDX(i_d, N)];
        if (DIM == 3) {
            const uint32_t zbk = z == 0 ? L - 1 : z - 1, zf = z + 1 == L ? 0 : z + 1;
            const uint32_t i_b = (zbk * L + y) * L + x, i_f = (zf * L + y) * L + x;
            if (EA) {
                jf = jb[2 * N + i] ? -1 : 1;
                jbk = jb[2 * N + i_b] ? -1 : 1;
            }
            h += jbk * sp[GBMC_IDX(i_b, N)] + jf * sp[GBMC_IDX(i_f, N)];
        }
        const int si = sp[GBMC_IDX(i, N)];
        const int dE = 2 * si * h;
        const uint32_t u = m == 0 ? w.x : m == 1 ? w.y : m == 2 ? w.z : w.w;
        const uint32_t thr = dE == 4 ? T.t4 : (dE == 8 ? T.t8 : T.t12);
        const bool acc = flip && (dE <= 0 || u <= thr);
        const int snew = acc ? -si : si;
        if (flip) sp[i] = (int8_t)snew;
        if (MEASURE) {
            e_acc -= snew * h;
            m_acc += snew + sp[i_r];
        }
    }
}

}  // namespace gbmc
